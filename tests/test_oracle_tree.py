"""Pins for the oracle's Morton keys, ordering, depth rule and boxes (Sec. 2.1, Alg. 1)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I


def test_morton_corners_and_octants():
    eps = 1e-9
    pts = np.array([[-1.0, -1.0, -1.0], [1.0, 1.0, 1.0]])
    k = O.morton(pts)
    assert k[0] == 0
    assert k[1] == (1 << 63) - 1  # upper faces clamp into the last cell
    # level-1 octant (bx, by, bz) is the top triple, x most significant
    for bx in (0, 1):
        for by in (0, 1):
            for bz in (0, 1):
                c = np.array([[-0.5 + bx, -0.5 + by, -0.5 + bz]])
                assert int(O.morton(c)[0]) >> 60 == (bx << 2) | (by << 1) | bz
    # one step below the midplane stays in the lower half, the midplane goes up
    lohi = O.morton(np.array([[-eps, 0.0, 0.0], [0.0, 0.0, 0.0]]))
    assert int(lohi[0]) >> 62 == 0 and int(lohi[1]) >> 62 == 1


def test_morton_matches_integer_coordinates():
    # a key is the bit interleave of floor((x+1)/2 * 2^21): check by de-interleaving
    p = I.uniform(500, 21)
    k = O.morton(p).astype(object)
    q = np.minimum(np.floor((p + 1.0) / 2.0 * 2.0 ** 21), 2 ** 21 - 1).astype(np.int64)
    for key, (a, b, c) in zip(k, q):
        x = y = z = 0
        for bit in range(21):
            t = (key >> (3 * bit)) & 7
            x |= ((t >> 2) & 1) << bit
            y |= ((t >> 1) & 1) << bit
            z |= (t & 1) << bit
        assert (x, y, z) == (a, b, c)


def test_outside_domain_rejected():
    with pytest.raises(O.OracleError) as e:
        O.Oracle(np.array([[0.0, 0.0, 1.0 + 1e-12]]), leaf_size=4)
    assert e.value.status == 2
    with pytest.raises(O.OracleError):
        O.morton(np.array([[np.nan, 0.0, 0.0]]))


def test_grid_depth_and_full_leaves():
    # cell-centred 16^3 grid: leaf 64 -> depth 2 with exactly 64 points per leaf
    o = O.Oracle(I.grid(16), leaf_size=64)
    t = o.tree()
    assert o.L == 2 and list(t["nbox"]) == [1, 8, 64]
    off = np.concatenate([[0], np.cumsum(t["nbox"])])
    sizes = t["box_end"][off[2]:] - t["box_start"][off[2]:]
    assert np.all(sizes == 64)
    # "at most" leaf_size: 63 forces one more level (8 per leaf)
    assert O.Oracle(I.grid(16), leaf_size=63).L == 3


def test_depth_zero_and_one():
    p = I.uniform(64, 2)
    assert O.Oracle(p, leaf_size=64).L == 0
    assert O.Oracle(I.uniform(65, 2), leaf_size=64).L >= 1


def test_boxes_partition_and_contain_their_points():
    p = I.uniform(3000, 9)
    o = O.Oracle(p, leaf_size=20)
    t = o.tree()
    perm = t["perm"]
    assert np.array_equal(np.sort(perm), np.arange(3000))
    assert np.all(np.diff(t["keys"].astype(np.float64)) >= 0)
    sp = p[perm]
    off = np.concatenate([[0], np.cumsum(t["nbox"])])
    for l in range(o.L + 1):
        bs, be, bk = (t[k][off[l]:off[l + 1]] for k in ("box_start", "box_end", "box_key"))
        assert bs[0] == 0 and be[-1] == 3000 and np.all(bs[1:] == be[:-1]) and np.all(be > bs)
        # every point lies in the closed cube of its box: integer coords from geometry
        q = np.minimum(np.floor((sp + 1.0) / 2.0 * 2 ** l), 2 ** l - 1).astype(np.int64)
        for b in range(len(bs)):
            key = int(bk[b])
            bx = sum(((key >> (3 * i + 2)) & 1) << i for i in range(l))
            by = sum(((key >> (3 * i + 1)) & 1) << i for i in range(l))
            bz = sum(((key >> (3 * i)) & 1) << i for i in range(l))
            assert np.all(q[bs[b]:be[b]] == [bx, by, bz])
        assert l < o.L or (be - bs).max() <= 20
    assert (t["box_end"][off[o.L - 1]:off[o.L]] - t["box_start"][off[o.L - 1]:off[o.L]]).max() > 20


def test_ties_broken_by_original_index():
    p = np.array([[0.5, 0.5, 0.5]] * 5 + [[-0.5, -0.5, -0.5]] * 3)
    o = O.Oracle(p, leaf_size=5)
    assert list(o.tree()["perm"]) == [5, 6, 7, 0, 1, 2, 3, 4]
    with pytest.raises(O.OracleError) as e:
        O.Oracle(p, leaf_size=4)  # 5 coincident points never split
    assert e.value.status == 8
