"""ctypes wrapper of the FP64 CPU oracle (test infrastructure).

Only the tests, the smoke check and the benchmark's CPU-baseline leg import
this module. It never touches the CUDA library. Fields are exchanged as numpy
arrays in the oracle's storage layout: extent ``s[a] = n[a] + 1`` along a wall
axis and ``n[a]`` along a periodic axis, shape ``(s_z, s_y, s_x)`` (3D) or
``(s_y, s_x)`` (2D).
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

FIELD = {"u": 0, "ut": 1, "urhs": 2, "p": 3, "prhs": 4, "rho": 5, "force": 6,
         "muc": 7, "mue": 8, "beta": 9, "m": 10, "ures": 11, "pres": 12}

# grid kinds for the transfer entries: faces of axis 0..2, centres, edges xy, xz, yz
KIND_FACE = (0, 1, 2)
KIND_CELL = 3
KIND_EDGE = {(0, 1): 4, (0, 2): 5, (1, 2): 6}


class OrParams(C.Structure):
    _fields_ = [("dim", C.c_int32), ("n", C.c_int32 * 3), ("periodic", C.c_int32 * 3),
                ("flow_axis", C.c_int32), ("phi_kind", C.c_int32), ("mg_levels_max", C.c_int32),
                ("nu1", C.c_int32), ("nu2", C.c_int32), ("vc_visc", C.c_int32), ("vc_p", C.c_int32),
                ("max_cycles", C.c_int32), ("coarse_sweeps", C.c_int32), ("pad0", C.c_int32),
                ("h", C.c_double), ("rho_f", C.c_double), ("mu_f", C.c_double),
                ("rho_ratio", C.c_double), ("mu_ratio", C.c_double), ("omega", C.c_double),
                ("omega_mu", C.c_double), ("d0_vol", C.c_double), ("dt", C.c_double),
                ("sigma", C.c_double), ("euler", C.c_double), ("inv_re", C.c_double),
                ("c_force", C.c_double), ("body_force", C.c_double), ("u_center", C.c_double),
                ("ic_scale", C.c_double), ("rtol", C.c_double), ("gamma_coarse", C.c_double),
                ("gamma_levels", C.c_double * 8), ("div_tol", C.c_double),
                ("open_flow", C.c_int32)]


class OrStats(C.Structure):
    _fields_ = [("cycles_visc", C.c_int32), ("cycles_p", C.c_int32),
                ("broken_total", C.c_int32), ("clamped_total", C.c_int32),
                ("res_visc", C.c_double), ("res_p", C.c_double), ("div_max", C.c_double),
                ("kinetic", C.c_double), ("step", C.c_int64)]


_LIBS = {}
_DP = C.POINTER(C.c_double)


# A test that plants a mistake in a copy of the oracle's source loads that
# build instead (both variants) by naming it in this environment variable.
OVERRIDE_ENV = "BFIBM_ORACLE_LIB"


def _lib(omp=False):
    if omp in _LIBS:
        return _LIBS[omp]
    path = os.environ.get(OVERRIDE_ENV)
    if not path:
        _build.build()
        path = _build.lib_path(omp)
    lib = C.CDLL(path)
    v, p, i, d, l = None, C.c_void_p, C.c_int, C.c_double, C.c_long
    sig = {
        "or_create": (p, [C.POINTER(OrParams)]), "or_destroy": (v, [p]),
        "or_phi": (d, [i, d]), "or_levels": (i, [p]), "or_body_force": (d, [p]),
        "or_outflow_pressure": (d, [p]),
        "or_level_dims": (v, [p, i, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "or_level_size": (l, [p, i]),
        "or_set_nodes": (v, [p, l, _DP]),
        "or_set_springs": (v, [p, l, C.POINTER(C.c_int32), _DP, _DP, _DP]),
        "or_refresh": (v, [p]), "or_step": (v, [p, i]),
        "or_get_field": (i, [p, i, i, i, _DP]), "or_set_field": (i, [p, i, i, i, _DP]),
        "or_get_nodes": (v, [p, _DP]), "or_get_node_forces": (v, [p, _DP]),
        "or_get_node_velocity": (v, [p, _DP]),
        "or_get_broken": (l, [p, l, C.POINTER(C.c_int32), C.POINTER(C.c_int32)]),
        "or_get_stats": (v, [p, C.POINTER(OrStats)]),
        "or_apply_p": (v, [p, i, _DP, _DP]),
        "or_apply_visc": (v, [p, i, C.POINTER(_DP), C.POINTER(_DP)]),
        "or_advection": (v, [p, C.POINTER(_DP), C.POINTER(_DP)]),
        "or_restrict": (v, [p, i, i, _DP, _DP]), "or_prolong_add": (v, [p, i, i, _DP, _DP]),
        "or_visc_diag": (d, [p, i, i, i, i, i]), "or_p_diag": (d, [p, i, i, i, i]),
        "or_solve_p": (i, [p, i]), "or_solve_visc": (i, [p, i]),
        "or_vcycle_p": (v, [p]), "or_vcycle_visc": (v, [p]),
        "or_rbgs_p": (v, [p, i]), "or_rbgs_visc": (v, [p, i]),
        "or_residual_p": (v, [p, i]), "or_residual_visc": (v, [p, i]),
        "or_build_coefficients": (v, [p]),
        "or_stage_rhs": (v, [p]), "or_stage_divergence": (v, [p]),
        "or_stage_project": (v, [p]), "or_stage_interp_advance": (v, [p]),
        "or_stage_springs": (v, [p]),
        "or_spread_sum": (v, [p, i, _DP, _DP, d]),
        "or_spread_max": (v, [p, i, _DP, d, d, d]),
        "or_interp": (v, [p, i, _DP, d, _DP]),
        "or_laminar_unit": (d, [p, d, d]),
        "or_num_threads": (i, []),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _LIBS[omp] = lib
    return lib


def phi(kind, r):
    """Delta-kernel profile phi_kind(r) as the oracle evaluates it."""
    lib = _lib()
    return np.array([lib.or_phi(int(kind), float(x)) for x in np.ravel(r)]).reshape(np.shape(r))


def make_params(prm):
    """Fill the oracle's parameter struct from a workload parameter dict."""
    P = OrParams()
    P.dim = prm["dim"]
    for a in range(3):
        P.n[a] = prm["n"][a]
        P.periodic[a] = int(prm["periodic"][a])
    for k in ("flow_axis", "phi_kind", "mg_levels_max", "nu1", "nu2", "vc_visc", "vc_p",
              "max_cycles", "coarse_sweeps"):
        setattr(P, k, int(prm[k]))
    for k in ("h", "rho_f", "mu_f", "rho_ratio", "mu_ratio", "omega", "omega_mu", "d0_vol",
              "dt", "sigma", "euler", "inv_re", "c_force", "body_force", "u_center", "ic_scale",
              "rtol", "gamma_coarse"):
        setattr(P, k, float(prm[k]))
    for l, v in enumerate(prm.get("gamma_levels", [])[:8]):
        P.gamma_levels[l] = float(v)
    P.div_tol = float(prm.get("div_tol", 0.0))
    P.open_flow = int(prm.get("open_flow", 0))
    return P


def _dp(a):
    return a.ctypes.data_as(_DP)


class Oracle:
    """One oracle simulation instance."""

    def __init__(self, prm, omp=False):
        self.lib = _lib(omp)
        self.prm = dict(prm)
        self._P = make_params(prm)
        self.h = self.lib.or_create(C.byref(self._P))
        if not self.h:
            raise ValueError("oracle rejected the parameters")
        self.dim = prm["dim"]
        self.levels = self.lib.or_levels(self.h)

    def close(self):
        if self.h:
            self.lib.or_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- geometry ---------------------------------------------------------
    def dims(self, l=0):
        n = (C.c_int32 * 3)()
        s = (C.c_int32 * 3)()
        self.lib.or_level_dims(self.h, l, n, s)
        return tuple(n), tuple(s)

    def shape(self, l=0):
        _, s = self.dims(l)
        return (s[2], s[1], s[0]) if self.dim == 3 else (s[1], s[0])

    @property
    def body_force(self):
        return self.lib.or_body_force(self.h)

    def outflow_pressure(self):
        """The pressure held at the outflow of an open duct (0 otherwise)."""
        return self.lib.or_outflow_pressure(self.h)

    # -- state ------------------------------------------------------------
    def set_nodes(self, X):
        X = np.ascontiguousarray(X, dtype=np.float64).reshape(-1, self.dim)
        self.lib.or_set_nodes(self.h, X.shape[0], _dp(X))
        self.eta = X.shape[0]

    def set_springs(self, ab, rest, K, brk):
        ab = np.ascontiguousarray(ab, dtype=np.int32).reshape(-1, 2)
        rest = np.ascontiguousarray(rest, dtype=np.float64)
        K = np.ascontiguousarray(K, dtype=np.float64)
        brk = np.ascontiguousarray(brk, dtype=np.float64)
        self.lib.or_set_springs(self.h, ab.shape[0], ab.ctypes.data_as(C.POINTER(C.c_int32)),
                                _dp(rest), _dp(K), _dp(brk))

    def refresh(self):
        self.lib.or_refresh(self.h)

    def step(self, n=1):
        self.lib.or_step(self.h, int(n))

    def get(self, which, comp=0, level=0):
        out = np.zeros(self.shape(level), dtype=np.float64)
        rc = self.lib.or_get_field(self.h, FIELD[which], comp, level, _dp(out))
        assert rc == 0
        return out

    def set(self, which, arr, comp=0, level=0):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape(level))
        rc = self.lib.or_set_field(self.h, FIELD[which], comp, level, _dp(a))
        assert rc == 0

    def nodes(self):
        out = np.zeros((self.eta, self.dim))
        self.lib.or_get_nodes(self.h, _dp(out))
        return out

    def node_forces(self):
        out = np.zeros((self.eta, self.dim))
        self.lib.or_get_node_forces(self.h, _dp(out))
        return out

    def node_velocity(self):
        out = np.zeros((self.eta, self.dim))
        self.lib.or_get_node_velocity(self.h, _dp(out))
        return out

    def broken(self):
        n = self.lib.or_get_broken(self.h, 0, None, None)
        ids = np.zeros(max(n, 1), dtype=np.int32)
        steps = np.zeros(max(n, 1), dtype=np.int32)
        self.lib.or_get_broken(self.h, n, ids.ctypes.data_as(C.POINTER(C.c_int32)),
                               steps.ctypes.data_as(C.POINTER(C.c_int32)))
        return ids[:n].copy(), steps[:n].copy()

    def stats(self):
        st = OrStats()
        self.lib.or_get_stats(self.h, C.byref(st))
        return {k: getattr(st, k) for k, _ in OrStats._fields_}

    # -- operators ----------------------------------------------------------
    def apply_p(self, p, level=0):
        p = np.ascontiguousarray(p, dtype=np.float64).reshape(self.shape(level))
        out = np.zeros_like(p)
        self.lib.or_apply_p(self.h, level, _dp(p), _dp(out))
        return out

    def _vec3(self, arrs, level):
        keep = [np.ascontiguousarray(a, dtype=np.float64).reshape(self.shape(level)) for a in arrs]
        while len(keep) < 3:
            keep.append(np.zeros(self.shape(level)))
        return keep, (_DP * 3)(*[_dp(a) for a in keep])

    def apply_visc(self, u, level=0):
        keep, ptr = self._vec3(u, level)
        outs, optr = self._vec3([np.zeros(self.shape(level)) for _ in range(3)], level)
        self.lib.or_apply_visc(self.h, level, ptr, optr)
        return [outs[d].copy() for d in range(self.dim)]

    def advection(self, u):
        keep, ptr = self._vec3(u, 0)
        outs, optr = self._vec3([np.zeros(self.shape(0)) for _ in range(3)], 0)
        self.lib.or_advection(self.h, ptr, optr)
        return [outs[d].copy() for d in range(self.dim)]

    def restrict(self, fine, level=0, comp=-1):
        """Restriction from `level` to `level + 1`: comp < 0 cell-centred, else the
        faces of velocity component comp."""
        f = np.ascontiguousarray(fine, dtype=np.float64).reshape(self.shape(level))
        out = np.zeros(self.shape(level + 1))
        self.lib.or_restrict(self.h, level, int(comp), _dp(f), _dp(out))
        return out

    def prolong_add(self, coarse, fine, level=0, comp=-1):
        """fine (on `level`) plus the prolongation of coarse (on `level + 1`)."""
        c = np.ascontiguousarray(coarse, dtype=np.float64).reshape(self.shape(level + 1))
        out = np.array(fine, dtype=np.float64).reshape(self.shape(level)).copy()
        self.lib.or_prolong_add(self.h, level, int(comp), _dp(c), _dp(out))
        return out

    def visc_diag(self, level, d, i, j, k=0):
        return self.lib.or_visc_diag(self.h, level, d, i, j, k)

    def p_diag(self, level, i, j, k=0):
        return self.lib.or_p_diag(self.h, level, i, j, k)

    def solve_p(self, ncycles):
        return self.lib.or_solve_p(self.h, int(ncycles))

    def solve_visc(self, ncycles):
        return self.lib.or_solve_visc(self.h, int(ncycles))

    def vcycle_p(self):
        self.lib.or_vcycle_p(self.h)

    def vcycle_visc(self):
        self.lib.or_vcycle_visc(self.h)

    def rbgs_p(self, level=0):
        self.lib.or_rbgs_p(self.h, level)

    def rbgs_visc(self, level=0):
        self.lib.or_rbgs_visc(self.h, level)

    def residual_p(self, level=0):
        self.lib.or_residual_p(self.h, level)
        return self.get("pres", 0, level)

    def residual_visc(self, level=0):
        self.lib.or_residual_visc(self.h, level)
        return [self.get("ures", d, level) for d in range(self.dim)]

    def build_coefficients(self):
        self.lib.or_build_coefficients(self.h)

    def stage(self, name):
        getattr(self.lib, "or_stage_" + name)(self.h)

    def spread_sum(self, kind, amp, w):
        arr = np.zeros(self.shape(0))
        amp = np.ascontiguousarray(amp, dtype=np.float64)
        self.lib.or_spread_sum(self.h, kind, _dp(arr), _dp(amp), float(w))
        return arr

    def spread_max(self, kind, w, mu_out, mu_max):
        arr = np.full(self.shape(0), float(mu_out))
        self.lib.or_spread_max(self.h, kind, _dp(arr), float(w), float(mu_out), float(mu_max))
        return arr

    def interp(self, kind, arr, w):
        a = np.ascontiguousarray(arr, dtype=np.float64).reshape(self.shape(0))
        out = np.zeros(self.eta)
        self.lib.or_interp(self.h, kind, _dp(a), float(w), _dp(out))
        return out

    def laminar_unit(self, y0, y1=0.0):
        return self.lib.or_laminar_unit(self.h, float(y0), float(y1))


def num_threads(omp=True):
    return _lib(omp).or_num_threads()
