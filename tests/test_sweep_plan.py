"""Host-side checks of how the sweep divides its work (no GPU): the work list
of one launch (every row of every running problem in exactly one unit, a
problem's units owning consecutive column-partial slots, at most min(R, n)
units per problem and R + count - 1 in all, loads even across clusters,
a problem owning whole shares swept interleaved) and the size classes of a
batch (boundaries at 512 x 2^(j/4), small classes merged upward)."""
import numpy as np
import pytest

from paper_0910_1650_gb300 import build as b
from paper_0910_1650_gb300 import capi


@pytest.fixture(scope="module", autouse=True)
def lib():
    b.build()
    return capi.lib()


def _check_plan(n, cluster, resident):
    units, ubeg = capi.ap_sweep_plan(n, cluster, resident)
    count = len(n)
    clusters = len(ubeg) - 1
    assert 1 <= clusters <= resident
    assert ubeg[0] == 0 and ubeg[-1] == len(units)
    assert all(ubeg[c + 1] > ubeg[c] for c in range(clusters))      # no empty cluster
    assert len(units) <= resident + count - 1
    seen = [np.zeros(m, dtype=np.int64) for m in n]
    slots = [[] for _ in n]
    for (p, g, first, cnt, stride) in units:
        assert cnt >= 1 and stride >= 1
        rows = first + stride * np.arange(cnt)
        assert rows[0] >= 0 and rows[-1] < n[p]
        seen[p][rows] += 1
        slots[p].append(g)
    for p in range(count):
        assert (seen[p] == 1).all(), p                               # every row exactly once
        assert sorted(slots[p]) == list(range(len(slots[p])))       # slots 0 .. G-1
        assert len(slots[p]) <= min(resident, n[p])
    return units, ubeg


def _loads(units, ubeg, n):
    return np.array([sum(units[u][3] * n[units[u][0]] for u in range(ubeg[c], ubeg[c + 1]))
                     for c in range(len(ubeg) - 1)], dtype=np.float64)


def test_single_problem_is_interleaved_over_every_cluster():
    for n, R in ((20000, 36), (1000, 760), (256, 760), (4097, 4096)):
        units, ubeg = _check_plan([n], 8 if n == 20000 else 1, R)
        G = min(n, R)
        assert len(units) == G and len(ubeg) - 1 == G
        # unit g sweeps rows g, g + G, g + 2G, ...: clusters side by side in memory
        assert sorted((u[2], u[4]) for u in units) == [(g, G) for g in range(G)]


def test_equal_problems_fill_every_cluster_evenly():
    n = [2000] * 50
    units, ubeg = _check_plan(n, 1, 456)
    assert len(ubeg) - 1 == 456
    loads = _loads(units, ubeg, n)
    # shares of 50 * 2000^2 / 456 elements, up to one row of rounding
    assert loads.max() <= loads.sum() / 456 + 2 * 2000
    # the problems that own whole shares are swept interleaved
    assert sum(1 for u in units if u[4] > 1) >= 400


def test_batch_of_many_small_problems_packs_them_into_shares():
    n = [256] * 2048
    units, ubeg = _check_plan(n, 1, 760)
    assert len(ubeg) - 1 == 760
    loads = _loads(units, ubeg, n)
    assert loads.max() <= loads.sum() / 760 + 2 * 256


@pytest.mark.parametrize("seed", range(6))
def test_random_batches_keep_every_invariant(seed):
    g = np.random.default_rng(seed)
    count = int(g.integers(1, 60))
    n = [int(x) for x in g.integers(2, 5000, size=count)]
    cluster = int(2 ** g.integers(0, 5))
    resident = int(g.integers(1, 900))
    _check_plan(n, cluster, resident)


def test_plan_rejects_bad_arguments():
    for args in (([1, 10], 1, 10), ([10], 3, 10), ([10], 1, 0), ([10], 32, 10)):
        with pytest.raises(capi.ApgbError):
            capi.ap_sweep_plan(*args)


def test_size_classes():
    # boundaries at 512 x 2^(j/4): 512 | 513 .. 608 | .. 724 | 725 ..
    n = [512] * 40 + [513] * 40 + [724] * 40 + [725] * 40
    cls = capi.ap_sweep_classes(n)
    assert cls == [0] * 40 + [1] * 40 + [2] * 40 + [3] * 40
    # a class with less than 8e6 elements of work joins the next larger one
    cls = capi.ap_sweep_classes([300] * 10 + [4000] * 3)
    assert cls == [0] * 13
    # the largest class is never merged away, and order follows size
    cls = capi.ap_sweep_classes([4000, 2, 3000, 100])
    assert cls[0] >= cls[2] >= cls[3] and cls[1] == cls[3]
    g = np.random.default_rng(7)
    n = [int(x) for x in g.integers(200, 4001, size=256)]
    cls = capi.ap_sweep_classes(n)
    order = np.argsort(n, kind="stable")
    assert np.all(np.diff(np.array(cls)[order]) >= 0)
    assert max(cls) + 1 <= 12
    with pytest.raises(capi.ApgbError):
        capi.ap_sweep_classes([5, 1])
