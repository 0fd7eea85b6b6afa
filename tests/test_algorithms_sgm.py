"""The shifted geometric mean of Section 5's comparison (shift 10) against its
closed form, and the comparison table's setup (CPU)."""
import math

import pytest

import bench


def test_sgm10_closed_form():
    # (90 + 10)(990 + 10) = 1e5: the geometric mean is sqrt(1e5), minus the shift
    assert bench.sgm10([90, 990]) == pytest.approx(math.sqrt(1e5) - 10.0, rel=1e-12)
    assert bench.sgm10([37, 37, 37]) == pytest.approx(37.0, rel=1e-12)
    assert bench.sgm10([0]) == pytest.approx(0.0, abs=1e-12)
    # an unsolved instance counts at the iteration limit
    assert bench.sgm10([bench.SGM_LIMIT]) == pytest.approx(bench.SGM_LIMIT, rel=1e-12)


def test_algorithm_table_covers_section5():
    names = [a[0] for a in bench.ALGORITHMS]
    # the four algorithms, the three fixed restart lengths, and the Section 6 rules
    assert {(a[1], a[2]) for a in bench.ALGORITHMS[:4]} == {(1, 1), (1, 3), (0, 1), (0, 3)}
    assert sorted(a[3] for a in bench.ALGORITHMS if a[2] == 2) == [10, 100, 1000]
    assert len(set(names)) == len(names)


def test_instance_set_is_seeded():
    import qpgen
    a = bench.algorithm_set(qpgen.SEED_BASE + 5000)
    b = bench.algorithm_set(qpgen.SEED_BASE + 5000)
    assert len(a) == 26
    assert all((x.c == y.c).all() and (x.A != y.A).nnz == 0 for x, y in zip(a, b))
