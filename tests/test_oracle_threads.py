"""The oracle's OpenMP build splits only loops whose iterations are
independent (one colour of a sweep, residuals, transfers) and keeps every
reduction serial, so it gives the same bits as the single-threaded build:
whole time steps of the 2D biofilm case and of the 64^3 duct with its mound,
in tolerance mode, compared element by element."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_1302_3663_gb300 import workloads as W


def run(inst, prm, omp, steps):
    o = O.Oracle(prm, omp=omp)
    o.set_nodes(inst["X"])
    o.set_springs(inst["ab"], inst["rest"], inst["K"], inst["brk"])
    o.step(steps)
    out = [o.get("u", d) for d in range(o.dim)] + [o.get("p"), o.nodes()]
    st = o.stats()
    o.close()
    return out, (st["cycles_visc"], st["cycles_p"])


@pytest.mark.parametrize("name,steps", [("c1", 3), ("c2", 1)])
def test_openmp_build_gives_the_single_threaded_bits(name, steps):
    if O.num_threads(True) < 2:
        pytest.skip("one host thread: nothing to compare")
    inst = W.CONFIGS[name]()
    prm = dict(inst["params"], vc_visc=0, vc_p=0, rtol=1e-10, max_cycles=100)
    a, ca = run(inst, prm, False, steps)
    b, cb = run(inst, prm, True, steps)
    assert ca == cb
    for k, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x, y), "array %d: max |diff| %.3e" % (k, np.abs(x - y).max())
