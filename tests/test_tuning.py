"""Host-side bookkeeping of the solver studies (Sec. 4.3.1): the work units
one V-cycle costs, counted in relaxations of the finest grid."""
import math

from paper_1302_3663_gb300 import tuning


def test_one_level_is_plain_relaxation():
    # one level: the coarsest solve is the whole cycle
    assert tuning.work_units_per_cycle(3, 1, 2, 2, 16) == 16.0


def test_two_levels():
    # nu1 + nu2 sweeps on the fine grid, the coarse sweeps at 2^-D of its cost
    assert tuning.work_units_per_cycle(3, 2, 2, 2, 16) == 4.0 + 16.0 / 8.0
    assert tuning.work_units_per_cycle(2, 2, 3, 3, 16) == 6.0 + 16.0 / 4.0


def test_deep_hierarchy_approaches_the_geometric_sum():
    # sum over levels of (nu1 + nu2) 2^(-D l) -> (nu1 + nu2) / (1 - 2^-D)
    for dim in (2, 3):
        wu = tuning.work_units_per_cycle(dim, 30, 2, 2, 16)
        assert math.isclose(wu, 4.0 / (1.0 - 2.0 ** -dim), rel_tol=1e-12)
