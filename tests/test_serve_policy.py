"""Admission policy of the serving loop (host logic, no GPU)."""
import collections

from paper_2003_01216_gb300.serve import Request, plan_admissions


def bytes_for(code, n, nseg=1):
    return n * (4 if code == 0 else 8) * 2 + 1000 * nseg


def q(*reqs):
    return collections.deque(Request(i, 0.0, c, n) for i, (c, n) in enumerate(reqs))


def test_large_head_goes_alone_small_heads_batch_by_type():
    w = q((0, 5000), (0, 10), (0, 20), (2, 30), (0, 40))
    groups = plan_admissions(w, 8, 0, 1 << 40, 0, bytes_for, small_keys=1000, batch_max_keys=10_000,
                             batch_max_reqs=64)
    sizes = [[r.n for r in g] for g, _ in groups]
    assert sizes == [[5000], [10, 20], [30], [40]]   # a type change or a large request ends a batch
    assert not w


def test_batch_caps():
    w = q(*[(0, 100)] * 10)
    groups = plan_admissions(w, 8, 0, 1 << 40, 0, bytes_for, 1000, batch_max_keys=350, batch_max_reqs=64)
    assert [len(g) for g, _ in groups] == [3, 3, 3, 1]
    w = q(*[(0, 1)] * 10)
    groups = plan_admissions(w, 8, 0, 1 << 40, 0, bytes_for, 1000, batch_max_keys=10_000, batch_max_reqs=4)
    assert [len(g) for g, _ in groups] == [4, 4, 2]


def test_slots_limit_admissions():
    w = q(*[(2, 5000)] * 5)
    groups = plan_admissions(w, 2, 0, 1 << 40, 0, bytes_for, 1000, 10_000, 64)
    assert len(groups) == 2 and len(w) == 3


def test_budget_queues_but_never_stalls():
    w = q((0, 5000), (0, 5000))
    need = bytes_for(0, 5000)
    # something in flight and no room: wait
    assert plan_admissions(w, 8, 0, need - 1, 1, bytes_for, 1000, 10_000, 64) == [] and len(w) == 2
    # nothing in flight: the head runs alone even over budget, the next one waits
    groups = plan_admissions(w, 8, 0, need - 1, 0, bytes_for, 1000, 10_000, 64)
    assert len(groups) == 1 and len(w) == 1
    # room for exactly two
    w = q((0, 5000), (0, 5000), (0, 5000))
    groups = plan_admissions(w, 8, 0, 2 * need, 0, bytes_for, 1000, 10_000, 64)
    assert len(groups) == 2 and len(w) == 1
