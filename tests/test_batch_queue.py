"""The persistent batch kernel's work queue (host logic, no GPU).

Every wait of the kernel is for items that sit earlier in the queue, which is
what makes each wait end (a CTA only ever waits for an item that a running CTA
already holds).  These tests build queues for random operator sizes, item
sizes and queue orders and check that each operator's work appears exactly
once and that every item comes after everything it waits for:
  permute chunks  <  gather tasks and near-field runs
  gather tasks    <  split-box reductions
  gathers, reductions, near-field runs  <  leaf runs.
"""
import numpy as np
import pytest

from paper_2307_16303_gb300 import api

GATHER, NEAR, REDUCE, LEAF, PERM = 0, 1, 2, 3, 4
PERM_CHUNK = 1024


def check_queue(q, npts, ng, ns, nl, near_group, leaf_group):
    nops = len(npts)
    pos = np.arange(len(q))
    for o in range(nops):
        mine = q[:, 0] == o
        kinds = {k: (q[mine & (q[:, 1] == k)], pos[mine & (q[:, 1] == k)]) for k in (GATHER, NEAR, REDUCE, LEAF, PERM)}
        # each piece of work exactly once
        assert sorted(kinds[PERM][0][:, 2].tolist()) == list(range(0, int(npts[o]), PERM_CHUNK))
        assert sorted(kinds[GATHER][0][:, 2].tolist()) == list(range(ng[o]))
        assert sorted(kinds[REDUCE][0][:, 2].tolist()) == list(range(ns[o]))
        for k, g in ((NEAR, near_group), (LEAF, leaf_group)):
            runs = kinds[k][0]
            covered = np.zeros(nl[o], np.int32)
            for first, cnt in runs[:, 2:4]:
                assert 1 <= cnt <= g
                covered[first:first + cnt] += 1
            assert covered.min() == 1 and covered.max() == 1
        last = lambda k: kinds[k][1].max() if len(kinds[k][1]) else -1
        first = lambda k: kinds[k][1].min() if len(kinds[k][1]) else len(q)
        assert last(PERM) < min(first(GATHER), first(NEAR))
        assert last(GATHER) < first(REDUCE)
        assert max(last(GATHER), last(REDUCE), last(NEAR)) < first(LEAF)
    assert set(np.unique(q[:, 1]).tolist()) <= {GATHER, NEAR, REDUCE, LEAF, PERM}


@pytest.mark.parametrize("lag", [0, 1, 2, 8])
@pytest.mark.parametrize("groups", [(4, 2), (1, 1), (8, 4), (3, 5)])
def test_queue_order_and_coverage(lag, groups):
    rng = np.random.default_rng(7 + lag)
    nops = 11
    npts = rng.integers(1, 5000, nops)
    ng = rng.integers(0, 40, nops)
    ng[3] = 0                                   # an operator without far field
    ns = np.minimum(rng.integers(0, 6, nops), ng)
    nl = np.maximum(1, npts // rng.integers(8, 60, nops))
    nl[5] = 1                                   # a one-leaf operator
    q = api.batch_queue(npts, ng, ns, nl, near_group=groups[0], leaf_group=groups[1], lag=lag)
    check_queue(q, npts, ng, ns, nl, *groups)


def test_phase_major_order_puts_every_leaf_after_every_stream():
    npts, ng, ns, nl = [3000, 9000, 40], [12, 30, 0], [1, 4, 0], [60, 200, 1]
    q = api.batch_queue(npts, ng, ns, nl)
    kinds = q[:, 1]
    assert np.all(kinds[:int(np.sum(kinds == PERM))] == PERM)
    first_leaf = np.argmax(kinds == LEAF)
    assert not np.any(np.isin(kinds[first_leaf:], [GATHER, NEAR, PERM]))


def test_queue_rejects_bad_sizes():
    with pytest.raises(api.H3DError):
        api.batch_queue([100], [1], [0], [0])          # no leaf
    with pytest.raises(api.H3DError):
        api.batch_queue([100], [1], [0], [2], near_group=0)
    with pytest.raises(api.H3DError):
        api.batch_queue([0], [1], [0], [1])            # no point
