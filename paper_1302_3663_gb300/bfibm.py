"""Python binding of libbfibm (include/bfibm.h): argument marshalling only.

Every call goes through the C ABI; every arithmetic step runs in the CUDA
kernels of the library. There is no CPU path: if the shared library cannot be
built or loaded, importing ``lib()`` raises.

Fields are exchanged as float64 numpy arrays in the ABI's dense layout:
shape ``(s2, s1, s0)`` in 3D and ``(s1, s0)`` in 2D, with ``s[a] = n[a] + 1``
on wall axes and ``n[a]`` on periodic axes.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ENOCONV, ETIMEOUT, ESTATE = range(7)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "ENOCONV", "ETIMEOUT", "ESTATE"]

FIELD = {"u": 0, "ut": 1, "urhs": 2, "p": 3, "prhs": 4, "rho": 5, "force": 6, "muc": 7,
         "mue": 8, "beta": 9, "m": 10, "ures": 11, "pres": 12, "idg": 13}
STAGE = {"rhs": 0, "divergence": 1, "project": 2, "interp_advance": 3, "springs": 4}
OPT_STATS, OPT_GRAPH, OPT_FUSED, OPT_TMA, OPT_INNER, OPT_KRYLOV, OPT_WAIT_NS, OPT_TAIL = range(8)
BATCH_PERSISTENT, BATCH_TUNE, BATCH_UNROLL, BATCH_TAIL = range(4)


class BfibmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 7 else status, msg))
        self.status = status


class bfibm_params(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32 * 3), ("periodic", C.c_int32 * 3),
                ("flow_axis", C.c_int32), ("phi_kind", C.c_int32), ("mg_levels_max", C.c_int32),
                ("nu1", C.c_int32), ("nu2", C.c_int32), ("vc_visc", C.c_int32),
                ("vc_p", C.c_int32), ("max_cycles", C.c_int32), ("coarse_sweeps", C.c_int32),
                ("precision", C.c_int32),
                ("h", C.c_double), ("rho_f", C.c_double), ("mu_f", C.c_double),
                ("rho_ratio", C.c_double), ("mu_ratio", C.c_double), ("omega", C.c_double),
                ("omega_mu", C.c_double), ("d0_vol", C.c_double), ("dt", C.c_double),
                ("sigma", C.c_double), ("euler", C.c_double), ("inv_re", C.c_double),
                ("c_force", C.c_double), ("body_force", C.c_double), ("u_center", C.c_double),
                ("ic_scale", C.c_double), ("rtol", C.c_double), ("gamma_coarse", C.c_double),
                ("gamma_levels", C.c_double * 8), ("div_tol", C.c_double),
                ("open_flow", C.c_int32)]


class bfibm_stats(C.Structure):
    _fields_ = [("cycles_visc", C.c_int32), ("cycles_p", C.c_int32),
                ("broken_total", C.c_int32), ("clamped_total", C.c_int32),
                ("res_visc", C.c_double), ("res_p", C.c_double), ("div_max", C.c_double),
                ("kinetic", C.c_double), ("step", C.c_int64),
                ("nonfinite_total", C.c_int32), ("wait_timeouts", C.c_int32),
                ("nonconv_total", C.c_int32), ("div_violations", C.c_int32),
                ("div_max_step", C.c_double), ("div_max_steps", C.c_double)]


_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int32)
_V = C.c_void_p
_i = C.c_int
_L = C.c_int64

# name -> argument types (all return bfibm_status unless listed in _RES)
SIGNATURES = {
    "bfibm_create": [C.POINTER(bfibm_params), _V, C.POINTER(_V)],
    "bfibm_set_nodes": [_V, _L, _DP],
    "bfibm_set_springs": [_V, _L, _IP, _DP, _DP, _DP],
    "bfibm_set_velocity": [_V, _i, _DP],
    "bfibm_step": [_V, _i],
    "bfibm_get_velocity": [_V, _i, _DP],
    "bfibm_get_pressure": [_V, _DP],
    "bfibm_get_nodes": [_V, _DP],
    "bfibm_get_broken": [_V, _L, C.POINTER(_L), _IP, _IP],
    "bfibm_get_stats": [_V, C.POINTER(bfibm_stats)],
    "bfibm_last_error": [_V],
    "bfibm_destroy": [_V],
    "bfibm_get_field": [_V, _i, _i, _i, _DP],
    "bfibm_set_field": [_V, _i, _i, _i, _DP],
    "bfibm_tma_plan": [_V, _i, _i, _IP],
    "bfibm_sweep_shape": [_V, _i, _i, _IP],
    "bfibm_sweep_set_shape": [_V, _i, _i, _IP],
    "bfibm_set_gamma": [_V, _DP],
    "bfibm_state_bytes": [_V, C.POINTER(_L)],
    "bfibm_save_state": [_V, _V, _L],
    "bfibm_load_state": [_V, _V, _L],
    "bfibm_tma_set_plan": [_V, _i, _i, _IP],
    "bfibm_get_field_f32": [_V, _i, _i, _i, C.POINTER(C.c_float)],
    "bfibm_set_field_f32": [_V, _i, _i, _i, C.POINTER(C.c_float)],
    "bfibm_get_field_dev": [_V, _i, _i, _i, _V],
    "bfibm_set_field_dev": [_V, _i, _i, _i, _V],
    "bfibm_get_node_forces": [_V, _DP],
    "bfibm_refresh": [_V],
    "bfibm_build_coefficients": [_V],
    "bfibm_stage": [_V, _i],
    "bfibm_solve_pressure": [_V, _i, _IP],
    "bfibm_solve_viscous": [_V, _i, _IP],
    "bfibm_smooth_pressure": [_V, _i, _i],
    "bfibm_smooth_viscous": [_V, _i, _i],
    "bfibm_synchronize": [_V],
    "bfibm_smooth_f32": [_V, _i, _i, _i],
    "bfibm_residual_pressure": [_V, _i],
    "bfibm_residual_viscous": [_V, _i],
    "bfibm_levels": [_V, _IP],
    "bfibm_level_dims": [_V, _i, _IP, _IP],
    "bfibm_body_force": [_V, _DP],
    "bfibm_set_option": [_V, _i, _L],
    "bfibm_launches_per_step": [_V, C.POINTER(_L)],
    "bfibm_launch_counts": [_V, C.POINTER(_L)],
    "bfibm_footprint": [C.POINTER(bfibm_params), _L, _L, C.POINTER(_L)],
    "bfibm_divergence_noalloc": [C.POINTER(bfibm_params), _V, _V, _V, _V, _V],
    "bfibm_batch_create": [C.POINTER(_V)],
    "bfibm_batch_add": [_V, _V, _IP],
    "bfibm_batch_remove": [_V, C.c_int32],
    "bfibm_batch_step": [_V, _IP],
    "bfibm_batch_wait": [_V],
    "bfibm_batch_slot_ms": [_V, C.c_int32, C.POINTER(C.c_float)],
    "bfibm_batch_destroy": [_V],
    "bfibm_batch_set_option": [_V, _i, _L],
    "bfibm_batch_info": [_V, C.POINTER(_L)],
    "bfibm_batch_sweep_shape": [_V, _i, _i, _IP],
    "bfibm_batch_error": [_V],
    "bfibm_batch_set_sweep_shape": [_V, _i, _i, _IP],
}
_RES = {"bfibm_last_error": C.c_char_p, "bfibm_destroy": None, "bfibm_batch_destroy": None,
        "bfibm_batch_error": C.c_char_p}

_LIB = None


def lib():
    """Load (building first if needed) libbfibm.so and set the prototypes."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = _build.build()
    L = C.CDLL(path)
    for name, args in SIGNATURES.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = _RES.get(name, C.c_int)
    _LIB = L
    return L


def library_path():
    return _build.LIB


def make_params(prm):
    """bfibm_params from a workload parameter dict."""
    P = bfibm_params()
    P.dim = prm["dim"]
    for a in range(3):
        P.n[a] = int(prm["n"][a])
        P.periodic[a] = int(prm["periodic"][a])
    for k in ("flow_axis", "phi_kind", "mg_levels_max", "nu1", "nu2", "vc_visc", "vc_p",
              "max_cycles", "coarse_sweeps", "precision"):
        setattr(P, k, int(prm.get(k, 0)))
    for k in ("h", "rho_f", "mu_f", "rho_ratio", "mu_ratio", "omega", "omega_mu", "d0_vol", "dt",
              "sigma", "euler", "inv_re", "c_force", "body_force", "u_center", "ic_scale", "rtol",
              "gamma_coarse"):
        setattr(P, k, float(prm[k]))
    for l, v in enumerate(prm.get("gamma_levels", [])[:8]):
        P.gamma_levels[l] = float(v)
    P.div_tol = float(prm.get("div_tol", 0.0))
    P.open_flow = int(prm.get("open_flow", 0))
    return P


def _dp(a):
    return a.ctypes.data_as(_DP)


def _out(out, shape):
    """A caller's output buffer, checked before the library writes into it
    (a wrong one would be written past its end), or a new one."""
    if out is None:
        return np.empty(shape)
    if (not isinstance(out, np.ndarray) or out.dtype != np.float64 or
            not out.flags.c_contiguous or not out.flags.writeable or tuple(out.shape) != tuple(shape)):
        raise ValueError("out must be a writeable C-contiguous float64 array of shape %s"
                         % (tuple(shape),))
    return out


def footprint(prm, eta=0, nsprings=0):
    out = _L(0)
    P = make_params(prm)
    st = lib().bfibm_footprint(C.byref(P), int(eta), int(nsprings), C.byref(out))
    if st != OK:
        raise BfibmError(st, "bfibm_footprint")
    return out.value


def divergence_noalloc(prm, u_ptrs, b_ptr, stream=None):
    """bfibm_divergence_noalloc on device pointers (ints); queues only."""
    P = make_params(prm)
    u = list(u_ptrs) + [None] * (3 - len(u_ptrs))
    st = lib().bfibm_divergence_noalloc(C.byref(P), u[0], u[1], u[2], b_ptr,
                                        _stream_handle(stream))
    if st != OK:
        raise BfibmError(st, "bfibm_divergence_noalloc")


def _stream_handle(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


class Context:
    """One simulation on the current CUDA device (see bfibm_create). `prm`
    holds the fields of bfibm_params and, for mixed precision, two solver
    options: `inner_cycles` (FP32 V-cycles per FP64 residual) and `krylov`
    (1: flexible CG around the V-cycles for the viscous solve)."""

    def __init__(self, prm, stream=None):
        self.lib = lib()
        self.prm = dict(prm)
        self.dim = prm["dim"]
        self._P = make_params(prm)
        h = _V()
        st = self.lib.bfibm_create(C.byref(self._P), _stream_handle(stream), C.byref(h))
        if st != OK:
            raise BfibmError(st, "bfibm_create rejected the parameters or failed")
        self.h = h
        self.eta = 0
        nl = C.c_int32(0)
        self.lib.bfibm_levels(self.h, C.byref(nl))
        self.levels = nl.value
        # FP32 V-cycles per FP64 defect-correction iteration (an option of the
        # context, not a field of bfibm_params)
        if int(prm.get("inner_cycles", 1)) != 1:
            self.set_option(OPT_INNER, int(prm["inner_cycles"]))
        # flexible CG around the FP32 V-cycles for the viscous solve
        if int(prm.get("krylov", 0)) != 0:
            self.set_option(OPT_KRYLOV, int(prm["krylov"]))

    def _chk(self, st, what, allow=(OK,)):
        if st not in allow:
            msg = self.lib.bfibm_last_error(self.h)
            raise BfibmError(st, "%s: %s" % (what, msg.decode() if msg else ""))
        return st

    def close(self):
        if getattr(self, "h", None):
            self.lib.bfibm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # geometry ----------------------------------------------------------------
    def dims(self, level=0):
        n = (C.c_int32 * 3)()
        s = (C.c_int32 * 3)()
        self._chk(self.lib.bfibm_level_dims(self.h, level, n, s), "bfibm_level_dims")
        return tuple(n), tuple(s)

    def shape(self, level=0):
        _, s = self.dims(level)
        return (s[2], s[1], s[0]) if self.dim == 3 else (s[1], s[0])

    @property
    def body_force(self):
        g = C.c_double(0)
        self._chk(self.lib.bfibm_body_force(self.h, C.byref(g)), "bfibm_body_force")
        return g.value

    # state -------------------------------------------------------------------
    def set_nodes(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, self.dim)
        self._chk(self.lib.bfibm_set_nodes(self.h, X.shape[0], _dp(X)), "bfibm_set_nodes")
        self.eta = X.shape[0]

    def set_springs(self, ab, rest, K, brk):
        ab = np.ascontiguousarray(ab, dtype=np.int32).reshape(-1, 2)
        rest, K, brk = (np.ascontiguousarray(a, dtype=np.float64) for a in (rest, K, brk))
        self._chk(self.lib.bfibm_set_springs(self.h, ab.shape[0], ab.ctypes.data_as(_IP),
                                             _dp(rest), _dp(K), _dp(brk)), "bfibm_set_springs")

    def set_velocity(self, comp, u):
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(self.shape())
        self._chk(self.lib.bfibm_set_velocity(self.h, comp, _dp(u)), "bfibm_set_velocity")

    def step(self, n=1):
        return self._chk(self.lib.bfibm_step(self.h, int(n)), "bfibm_step", (OK, ENOCONV))

    def get_velocity(self, comp, out=None):
        out = _out(out, self.shape())
        self._chk(self.lib.bfibm_get_velocity(self.h, comp, _dp(out)), "bfibm_get_velocity")
        return out

    def get_pressure(self, out=None):
        out = _out(out, self.shape())
        self._chk(self.lib.bfibm_get_pressure(self.h, _dp(out)), "bfibm_get_pressure")
        return out

    def get_nodes(self, out=None):
        out = _out(out, (self.eta, self.dim))
        self._chk(self.lib.bfibm_get_nodes(self.h, _dp(out)), "bfibm_get_nodes")
        return out

    def get_node_forces(self):
        out = np.empty((self.eta, self.dim))
        self._chk(self.lib.bfibm_get_node_forces(self.h, _dp(out)), "bfibm_get_node_forces")
        return out

    def get_broken(self):
        n = _L(0)
        self._chk(self.lib.bfibm_get_broken(self.h, 0, C.byref(n), None, None), "bfibm_get_broken")
        cnt = n.value
        ids = np.zeros(max(cnt, 1), dtype=np.int32)
        steps = np.zeros(max(cnt, 1), dtype=np.int32)
        self._chk(self.lib.bfibm_get_broken(self.h, cnt, C.byref(n), ids.ctypes.data_as(_IP),
                                            steps.ctypes.data_as(_IP)), "bfibm_get_broken")
        return ids[:cnt].copy(), steps[:cnt].copy()

    def get_stats(self):
        st = bfibm_stats()
        self._chk(self.lib.bfibm_get_stats(self.h, C.byref(st)), "bfibm_get_stats")
        return {k: getattr(st, k) for k, _ in bfibm_stats._fields_}

    # operator-level ----------------------------------------------------------
    def get_field(self, which, comp=0, level=0):
        out = np.empty(self.shape(level))
        self._chk(self.lib.bfibm_get_field(self.h, FIELD[which], comp, level, _dp(out)),
                  "bfibm_get_field")
        return out

    def set_field(self, which, arr, comp=0, level=0):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape(level))
        self._chk(self.lib.bfibm_set_field(self.h, FIELD[which], comp, level, _dp(a)),
                  "bfibm_set_field")

    def set_gamma(self, gamma_levels):
        """gamma_lh per coarse level (index 1 = grid 2h; 0 falls back to
        gamma_coarse); see bfibm_set_gamma."""
        g = np.zeros(8)
        g[:len(gamma_levels)] = gamma_levels
        self._chk(self.lib.bfibm_set_gamma(self.h, _dp(g)), "bfibm_set_gamma")

    def save_state(self):
        """The checkpoint of the evolving state as a uint8 array (see
        bfibm_save_state)."""
        n = _L()
        self._chk(self.lib.bfibm_state_bytes(self.h, C.byref(n)), "bfibm_state_bytes")
        buf = np.empty(n.value, dtype=np.uint8)
        self._chk(self.lib.bfibm_save_state(self.h, buf.ctypes.data, n.value), "bfibm_save_state")
        return buf

    def load_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        self._chk(self.lib.bfibm_load_state(self.h, buf.ctypes.data, buf.size), "bfibm_load_state")

    def tma_plan(self, level=0, kind=0):
        """(tile rows, planes per chunk, planes prefetched, strip columns, grid)
        of the tuned TMA sweep on a level, or None where the level does not
        use it."""
        out = (C.c_int32 * 5)()
        st = self.lib.bfibm_tma_plan(self.h, level, kind, out)
        return tuple(out) if st == OK else None

    def sweep_shape(self, level=0, kind=0):
        """(tile rows, planes per chunk, planes per phase, threads per row,
        kernel) of the tuned one-pass FP32 sweep on a level (kernel 0: ring
        sweep, 1: pair sweep; 0 in the first four: built-in choice), or None
        where the level has not been tuned."""
        out = (C.c_int32 * 5)()
        st = self.lib.bfibm_sweep_shape(self.h, level, kind, out)
        return tuple(out) if st == OK else None

    def sweep_set_shape(self, level, kind, shape):
        """Pin (tile rows, planes per chunk, planes per phase, threads per
        row, kernel) of the one-pass FP32 sweep for the shape of a level (a
        4-tuple pins the ring sweep); see bfibm_sweep_set_shape."""
        shape = list(shape) + [0] * (5 - len(shape))
        arr = (C.c_int32 * 5)(*[int(v) for v in shape])
        self._chk(self.lib.bfibm_sweep_set_shape(self.h, level, kind, arr),
                  "bfibm_sweep_set_shape")

    def sweep_plans(self):
        """Every tuned FP32 sweep choice of this context's levels: a list of
        (level, kind, TMA plan or None, one-pass shape)."""
        out = []
        for level in range(self.levels):
            for kind in list(range(self.dim)) + [3]:
                shape = self.sweep_shape(level, kind)
                if shape is not None:
                    out.append((level, kind, self.tma_plan(level, kind), shape))
        return out

    def pin_sweep_plans(self, plans):
        """Pin choices recorded by sweep_plans (of a context with the same
        level shapes), so that another process runs the same kernels."""
        for level, kind, tma, shape in plans:
            if tma is not None:
                self.tma_set_plan(level, kind, tma)
            else:
                self.sweep_set_shape(level, kind, shape)

    def tma_set_plan(self, level, kind, plan):
        """Pin (tile rows, planes per chunk, planes prefetched, strip columns,
        grid) for the shape of a level; see bfibm_tma_set_plan."""
        arr = (C.c_int32 * 5)(*plan)
        self._chk(self.lib.bfibm_tma_set_plan(self.h, level, kind, arr), "bfibm_tma_set_plan")

    def get_field_f32(self, which, comp=0, level=0):
        out = np.empty(self.shape(level), dtype=np.float32)
        self._chk(self.lib.bfibm_get_field_f32(self.h, FIELD[which], comp, level,
                                               out.ctypes.data_as(C.POINTER(C.c_float))),
                  "bfibm_get_field_f32")
        return out

    def set_field_f32(self, which, arr, comp=0, level=0):
        a = np.ascontiguousarray(arr, dtype=np.float32).reshape(self.shape(level))
        self._chk(self.lib.bfibm_set_field_f32(self.h, FIELD[which], comp, level,
                                               a.ctypes.data_as(C.POINTER(C.c_float))),
                  "bfibm_set_field_f32")

    def get_field_dev(self, which, dev_ptr, comp=0, level=0):
        self._chk(self.lib.bfibm_get_field_dev(self.h, FIELD[which], comp, level, int(dev_ptr)),
                  "bfibm_get_field_dev")

    def set_field_dev(self, which, dev_ptr, comp=0, level=0):
        self._chk(self.lib.bfibm_set_field_dev(self.h, FIELD[which], comp, level, int(dev_ptr)),
                  "bfibm_set_field_dev")

    def refresh(self):
        self._chk(self.lib.bfibm_refresh(self.h), "bfibm_refresh")

    def build_coefficients(self):
        self._chk(self.lib.bfibm_build_coefficients(self.h), "bfibm_build_coefficients")

    def stage(self, name):
        self._chk(self.lib.bfibm_stage(self.h, STAGE[name]), "bfibm_stage")

    def solve_pressure(self, ncycles):
        cyc = C.c_int32(0)
        self._chk(self.lib.bfibm_solve_pressure(self.h, int(ncycles), C.byref(cyc)),
                  "bfibm_solve_pressure", (OK, ENOCONV))
        return cyc.value

    def solve_viscous(self, ncycles):
        cyc = C.c_int32(0)
        self._chk(self.lib.bfibm_solve_viscous(self.h, int(ncycles), C.byref(cyc)),
                  "bfibm_solve_viscous", (OK, ENOCONV))
        return cyc.value

    def smooth_pressure(self, level=0, nsweeps=1, sync=True):
        self._chk(self.lib.bfibm_smooth_pressure(self.h, level, nsweeps), "bfibm_smooth_pressure")
        if sync:
            self.synchronize()

    def smooth_viscous(self, level=0, nsweeps=1, sync=True):
        self._chk(self.lib.bfibm_smooth_viscous(self.h, level, nsweeps), "bfibm_smooth_viscous")
        if sync:
            self.synchronize()

    def smooth_f32(self, which, level=0, nsweeps=1, sync=True):
        self._chk(self.lib.bfibm_smooth_f32(self.h, which, level, nsweeps), "bfibm_smooth_f32")
        if sync:
            self.synchronize()

    def synchronize(self):
        self._chk(self.lib.bfibm_synchronize(self.h), "bfibm_synchronize")

    def residual_pressure(self, level=0):
        self._chk(self.lib.bfibm_residual_pressure(self.h, level), "bfibm_residual_pressure")
        return self.get_field("pres", 0, level)

    def residual_viscous(self, level=0):
        self._chk(self.lib.bfibm_residual_viscous(self.h, level), "bfibm_residual_viscous")
        return [self.get_field("ures", d, level) for d in range(self.dim)]

    def launch_counts(self):
        """{top, body_visc, body_p, iters_visc, iters_p}: see bfibm_launch_counts."""
        out = (_L * 5)()
        self._chk(self.lib.bfibm_launch_counts(self.h, out), "bfibm_launch_counts")
        return dict(zip(("top", "body_visc", "body_p", "iters_visc", "iters_p"), out))

    def launches_per_step(self):
        n = _L(0)
        self._chk(self.lib.bfibm_launches_per_step(self.h, C.byref(n)), "bfibm_launches_per_step")
        return n.value

    def set_option(self, opt, value):
        self._chk(self.lib.bfibm_set_option(self.h, opt, int(value)), "bfibm_set_option")


def load_instance(inst, stream=None, prm_override=None):
    """Context with a workload instance's parameters, nodes and springs loaded."""
    prm = dict(inst["params"])
    if prm_override:
        prm.update(prm_override)
    ctx = Context(prm, stream=stream)
    ctx.set_nodes(inst["X"])
    ctx.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    return ctx


class Batch:
    """Independent contexts stepped together (see bfibm_batch_*). With
    persistent=True the members step in lock step, each multigrid level of
    their solves one launch over all of them (BFIBM_BATCH_PERSISTENT)."""

    def __init__(self, persistent=False, tune=True):
        self.lib = lib()
        h = _V()
        st = self.lib.bfibm_batch_create(C.byref(h))
        if st != OK:
            raise BfibmError(st, "bfibm_batch_create")
        self.h = h
        self.members = {}
        if persistent:
            self.set_option(BATCH_PERSISTENT, 1)
        if not tune:
            self.set_option(BATCH_TUNE, 0)

    def set_option(self, option, value):
        st = self.lib.bfibm_batch_set_option(self.h, int(option), int(value))
        if st != OK:
            raise BfibmError(st, "bfibm_batch_set_option")

    def info(self):
        """dict of bfibm_batch_info's fields"""
        out = (_L * 8)()
        st = self.lib.bfibm_batch_info(self.h, out)
        if st != OK:
            raise BfibmError(st, "bfibm_batch_info")
        keys = ("persistent", "builds", "members", "graph_kernels", "visc_body_kernels",
                "p_body_kernels", "visc_iterations", "p_iterations")
        return dict(zip(keys, [int(v) for v in out]))

    def sweep_shape(self, level, kind):
        """(tile rows, chunk planes, planes per phase, threads per row, one
        block per item, grid, kernel: 0 ring, 1 pair) of the plan's batched
        sweep; kind 0 viscous, 1 pressure"""
        out = (C.c_int32 * 7)()
        st = self.lib.bfibm_batch_sweep_shape(self.h, int(level), int(kind), out)
        if st != OK:
            raise BfibmError(st, "bfibm_batch_sweep_shape")
        return tuple(int(v) for v in out)

    def set_sweep_shape(self, level, kind, shape):
        """shape: (rows, chunk planes, planes per phase, threads per row, one
        block per item[, kernel: 0 ring, 1 pair])"""
        shape = list(shape[:6]) + [0] * (6 - len(shape[:6]))
        a = (C.c_int32 * 6)(*[int(v) for v in shape])
        st = self.lib.bfibm_batch_set_sweep_shape(self.h, int(level), int(kind), a)
        if st != OK:
            raise BfibmError(st, "bfibm_batch_set_sweep_shape: " +
                             (self.lib.bfibm_batch_error(self.h) or b"").decode())

    def sweep_shapes(self):
        """{level: (viscous shape, pressure shape)} of the current plan"""
        out = {}
        for lev in range(8):
            try:
                v, p = self.sweep_shape(lev, 0), self.sweep_shape(lev, 1)
                out[lev] = (v[:5] + v[6:], p[:5] + p[6:])
            except BfibmError:
                break
        return out

    def pin_sweep_shapes(self, shapes):
        for lev, (v, p) in shapes.items():
            self.set_sweep_shape(int(lev), 0, v)
            self.set_sweep_shape(int(lev), 1, p)

    def add(self, ctx):
        slot = C.c_int32(-1)
        st = self.lib.bfibm_batch_add(self.h, ctx.h, C.byref(slot))
        if st != OK:
            raise BfibmError(st, "bfibm_batch_add")
        self.members[slot.value] = ctx
        return slot.value

    def remove(self, slot):
        st = self.lib.bfibm_batch_remove(self.h, int(slot))
        if st != OK:
            raise BfibmError(st, "bfibm_batch_remove")
        return self.members.pop(slot)

    def step(self, nsteps=None):
        arr = None
        if nsteps is not None:
            n = max(self.members) + 1 if self.members else 0
            a = np.zeros(max(n, 1), dtype=np.int32)
            for k, v in nsteps.items():
                a[k] = v
            arr = a.ctypes.data_as(_IP)
            self._keep = a
        st = self.lib.bfibm_batch_step(self.h, arr)
        if st not in (OK, ENOCONV):
            msg = (self.lib.bfibm_batch_error(self.h) or b"").decode()
            raise BfibmError(st, "bfibm_batch_step: " + "; ".join(
                m for m in (msg, self._member_errors()) if m))

    def _member_errors(self):
        msgs = []
        for slot, ctx in self.members.items():
            m = self.lib.bfibm_last_error(ctx.h)
            if m:
                msgs.append("slot %d: %s" % (slot, m.decode()))
        return "; ".join(msgs)

    def wait(self):
        """Wait for every member; returns ENOCONV when a member reports it
        (its statistics say which) and raises on any other failure."""
        st = self.lib.bfibm_batch_wait(self.h)
        if st not in (OK, ENOCONV):
            raise BfibmError(st, "bfibm_batch_wait: " + self._member_errors())
        return st

    def slot_ms(self, slot):
        ms = C.c_float(0)
        st = self.lib.bfibm_batch_slot_ms(self.h, int(slot), C.byref(ms))
        if st != OK:
            raise BfibmError(st, "bfibm_batch_slot_ms")
        return ms.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.bfibm_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
