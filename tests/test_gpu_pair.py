"""The pair sweep (a thread per (red, black) pair of a row, marching over the
planes) against the ring sweep on the same FP32 inputs. The per-point
arithmetic and its order are the same, and a wall term the ring sweep skips
gets a zero weight. So every viscous component and the pressure must come
out bit-identical, over several sweeps, for row tiles and plane chunks that
do not divide the grid, and on the 128 x 128 x 256 grid of the benchmark."""
import numpy as np
import pytest

from paper_1302_3663_gb300 import bfibm, workloads as W

from test_gpu_tma import context, random_inputs, sweep

pytestmark = pytest.mark.gpu

RING = (4, 8, 1, 0, 0)


def sweep_with(c, f, shape, nsweeps=3):
    for d in range(3):
        c.sweep_set_shape(0, d, shape)
    return sweep(c, f, 1, False, nsweeps)


@pytest.mark.parametrize("n,pair", [((48, 20, 40), (6, 7)), ((64, 64, 64), (14, 16)),
                                    ((30, 26, 18), (4, 5)), ((16, 9, 12), (8, 32))],
                         ids=["ragged", "c2", "odd_rows", "tall_tiles"])
def test_pair_sweep_bit_identical_to_ring_sweep(n, pair):
    c = context(n, (0, 0, 1), 2)
    f = random_inputs(c, np.random.default_rng(5))
    a = sweep_with(c, f, RING)
    b = sweep_with(c, f, (pair[0], pair[1], 1, 0, 1))
    assert c.sweep_shape(0, 0)[4] == 1
    for d, (x, y) in enumerate(zip(a, b)):
        assert np.isfinite(x).all()
        assert np.array_equal(x, y), "component %d: max |diff| %.3e" % (d, np.abs(x - y).max())
    c.close()


@pytest.mark.parametrize("n,pair", [((48, 20, 40), (6, 7)), ((64, 64, 64), (14, 16)),
                                    ((30, 26, 18), (4, 5)), ((16, 9, 12), (8, 32))],
                         ids=["ragged", "c2", "odd_rows", "tall_tiles"])
def test_pressure_pair_sweep_bit_identical_to_ring_sweep(n, pair):
    # the pressure's pair sweep: the same px_acc / px_final arithmetic, a
    # neighbour beyond a wall entering with weight 0
    c = context(n, (0, 0, 1), 2)
    f = random_inputs(c, np.random.default_rng(9))
    c.sweep_set_shape(0, 3, RING)
    a = sweep(c, f, 0, False, 3)
    c.sweep_set_shape(0, 3, (pair[0], pair[1], 1, 0, 1))
    b = sweep(c, f, 0, False, 3)
    assert c.sweep_shape(0, 3)[4] == 1
    assert np.isfinite(a[0]).all()
    assert np.array_equal(a[0], b[0]), "max |diff| %.3e" % np.abs(a[0] - b[0]).max()
    c.close()


def test_pair_sweep_bit_identical_on_the_benchmark_grid():
    inst = W.c3()
    c = bfibm.load_instance(inst)
    c.step(1)
    f = {}
    for d in range(3):
        for name in ("ut", "urhs", "m", "beta", "mue", "idg"):
            f[(name, d)] = c.get_field_f32(name, d, 0)
    for name in ("muc", "p", "prhs"):
        f[(name, 0)] = c.get_field_f32(name, 0, 0)
    a = sweep_with(c, f, RING, 2)
    for shape in ((6, 24, 1, 0, 1), (4, 9, 1, 0, 1)):
        b = sweep_with(c, f, shape, 2)
        for x, y in zip(a, b):
            assert np.array_equal(x, y)
    c.sweep_set_shape(0, 3, RING)
    a = sweep(c, f, 0, False, 2)
    for shape in ((6, 20, 1, 0, 1), (2, 7, 1, 0, 1)):
        c.sweep_set_shape(0, 3, shape)
        b = sweep(c, f, 0, False, 2)
        assert np.array_equal(a[0], b[0])
    c.close()


def test_pair_sweep_shapes_outside_its_range_are_refused():
    c = context((48, 20, 40), (0, 0, 1), 2)
    for bad in ((4, 8, 2, 0, 1), (4, 8, 1, 32, 1), (0, 8, 1, 0, 1), (4, 0, 1, 0, 1),
                (40, 8, 1, 0, 1)):
        with pytest.raises(bfibm.BfibmError):
            c.sweep_set_shape(0, 0, bad)
    c.close()
    c = context((40, 22, 44), (1, 0, 1), 2)   # periodic x: the ring sweep only
    with pytest.raises(bfibm.BfibmError):
        c.sweep_set_shape(0, 0, (4, 8, 1, 0, 1))
    c.close()
