"""Pins for the oracle's neighbour classes, interaction lists and near lists.

* A geometric brute force classifies box pairs by the dimension of the
  intersection of the two closed cubes (face / edge / vertex / nothing), as the
  Table "Notations" and Definition "admh3d" state them, and builds the clan and
  interaction list literally; the oracle (which uses integer offsets) must agree
  pair by pair.
* Block counts on full trees match closed forms derived by hand and, at L = 1,
  the values printed in the paper's Tables dense3d / lrfar / lrvert.
* Every entry of the N x N matrix is covered by exactly one block.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2307_16303_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))


def _coords(key: int, level: int):
    x = sum(((key >> (3 * i + 2)) & 1) << i for i in range(level))
    y = sum(((key >> (3 * i + 1)) & 1) << i for i in range(level))
    z = sum(((key >> (3 * i)) & 1) << i for i in range(level))
    return (x, y, z)


def _geometric_class(a, b):
    """Dimension of the intersection of closed unit cubes at integer corners a, b."""
    dims = 0
    for k in range(3):
        overlap = min(a[k] + 1, b[k] + 1) - max(a[k], b[k])
        if overlap < 0:
            return "far"
        if overlap > 0:
            dims += 1
    return {3: "self", 2: "face", 1: "edge", 0: "vertex"}[dims]


def _brute_lists(tree):
    L = tree["L"]
    off = np.concatenate([[0], np.cumsum(tree["nbox"])])
    blocks, near = set(), set()
    for l in range(1, L + 1):
        keys = [int(k) for k in tree["box_key"][off[l]:off[l + 1]]]
        co = [_coords(k, l) for k in keys]
        par = [tuple(c >> 1 for c in p) for p in co]
        for i in range(len(keys)):
            for j in range(len(keys)):
                if i == j:
                    continue
                pc = _geometric_class(par[i], par[j])
                in_clan = pc == "self" or pc in ("edge", "face")  # siblings or children of E/F of parent
                cls = _geometric_class(co[i], co[j])
                if in_clan and cls in ("vertex", "far"):
                    blocks.add((l, keys[i], keys[j], cls))
    keys = [int(k) for k in tree["box_key"][off[L]:off[L + 1]]]
    co = [_coords(k, L) for k in keys]
    for i in range(len(keys)):
        for j in range(len(keys)):
            cls = _geometric_class(co[i], co[j])
            if cls in ("self", "face", "edge"):
                near.add((keys[i], keys[j], cls))
    return blocks, near


def _oracle_sets(o):
    t, li = o.tree(), o.lists()
    off = np.concatenate([[0], np.cumsum(t["nbox"])])
    bk = t["box_key"]
    blocks = {(int(l), int(bk[off[l] + a]), int(bk[off[l] + b]), O.CLS_NAMES[int(c)])
              for l, a, b, c in zip(li["level"], li["tgt"], li["src"], li["cls"])}
    near = {(int(bk[off[o.L] + a]), int(bk[off[o.L] + b]), O.CLS_NAMES[int(c)])
            for a, b, c in zip(li["near_tgt"], li["near_src"], li["near_cls"])}
    return blocks, near, li


@pytest.mark.parametrize("pts,leaf", [
    (I.grid(8), 8),                 # full tree, L = 2
    (I.uniform(900, 31), 12),       # sparse boxes, ragged
    (I.sphere(1500, 32) * 0.99, 16),  # surface cloud, many empty boxes
])
def test_lists_match_geometric_brute_force(pts, leaf):
    o = O.Oracle(pts, leaf_size=leaf)
    blocks, near, li = _oracle_sets(o)
    bb, bn = _brute_lists(o.tree())
    assert blocks == bb
    assert near == bn
    assert len(blocks) == o.n_blocks and len(near) == o.n_near  # no duplicates
    # target-major order: (level, target, source) ascending
    order = np.lexsort((li["src"], li["tgt"], li["level"]))
    assert np.array_equal(order, np.arange(o.n_blocks))


def _count_by_class(o):
    li = o.lists()
    out = {"near": o.n_near}
    for l in range(1, o.L + 1):
        sel = li["level"] == l
        out[(l, "vertex")] = int(np.sum(sel & (li["cls"] == 3)))
        out[(l, "far")] = int(np.sum(sel & (li["cls"] == 4)))
    return out


def test_paper_counts_at_depth_one():
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "paper_block_counts.txt"))
            if ln.strip() and not ln.startswith("#")]
    hdr, vals = rows[0], dict(zip(rows[0], map(int, rows[1])))
    assert hdr == ["L", "dense", "far", "vertex"] and vals["L"] == 1
    c = _count_by_class(O.Oracle(I.grid(2), leaf_size=1))
    assert c["near"] == vals["dense"]
    assert c[(1, "far")] == vals["far"]
    assert c[(1, "vertex")] == vals["vertex"]


@pytest.mark.parametrize("L", [1, 2, 3])
def test_full_tree_closed_forms(L):
    """n = 2^L boxes per axis, every box non-empty.

    near (self+face+edge, ordered)  n^3 + 3*2*(n-1)n^2 + 3*4*(n-1)^2 n = 19n^3 - 30n^2 + 12n
    vertex blocks at level l        8(n_l-1)^3 - 8(n_{l-1}-1)^3  (V pairs whose parents are not V pairs;
                                    each V parent pair has exactly one touching V child pair)
    far blocks at level l           64*near(n_{l-1}) - n_l^3 - (near(n_l) - n_l^3) - vertex_l
                                    (clan pairs, minus the face/edge/vertex pairs inside the clan)
    """
    o = O.Oracle(I.grid(2 ** (L + 1)), leaf_size=8)
    assert o.L == L
    c = _count_by_class(o)

    def near(n):
        return 19 * n ** 3 - 30 * n ** 2 + 12 * n

    assert c["near"] == near(2 ** L)
    for l in range(1, L + 1):
        n, m = 2 ** l, 2 ** (l - 1)
        v = 8 * (n - 1) ** 3 - 8 * (m - 1) ** 3
        assert c[(l, "vertex")] == v
        assert c[(l, "far")] == 64 * near(m) - n ** 3 - (near(n) - n ** 3) - v
    assert sum(c[(l, "vertex")] for l in range(1, L + 1)) == (2 * 2 ** L - 2) ** 3


@pytest.mark.parametrize("pts,leaf", [(I.uniform(700, 41), 9), (I.grid(8), 8), (I.sphere(600, 42) * 0.9, 10)])
def test_every_entry_covered_exactly_once(pts, leaf):
    o = O.Oracle(pts, leaf_size=leaf)
    t, li = o.tree(), o.lists()
    off = np.concatenate([[0], np.cumsum(t["nbox"])])
    N = pts.shape[0]
    cover = np.zeros((N, N), np.int32)
    for a, b in zip(li["near_tgt"], li["near_src"]):
        ia, ib = off[o.L] + a, off[o.L] + b
        cover[t["box_start"][ia]:t["box_end"][ia], t["box_start"][ib]:t["box_end"][ib]] += 1
    for l, a, b in zip(li["level"], li["tgt"], li["src"]):
        ia, ib = off[l] + a, off[l] + b
        cover[t["box_start"][ia]:t["box_end"][ia], t["box_start"][ib]:t["box_end"][ib]] += 1
    assert cover.min() == 1 and cover.max() == 1


def test_lists_symmetric():
    o = O.Oracle(I.uniform(2000, 43), leaf_size=16)
    li = o.lists()
    fwd = set(zip(li["level"], li["tgt"], li["src"], li["cls"]))
    assert fwd == set(zip(li["level"], li["src"], li["tgt"], li["cls"]))
    nf = set(zip(li["near_tgt"], li["near_src"]))
    assert nf == set(zip(li["near_src"], li["near_tgt"]))


# --- the paper's comparison formats (H-matrix eta = sqrt(3), HODLR) ---------------

def _strong_admissible(a, b):
    """Eq. adm with eta = sqrt(3) for unit cubes at integer corners a, b:
    max(diam) = sqrt(3) <= sqrt(3) * dist  <=>  dist^2 >= 1 (exact in integers)."""
    dist2 = sum(max(0, abs(a[k] - b[k]) - 1) ** 2 for k in range(3))
    return dist2 >= 1


def _brute_lists_mode(tree, adm):
    L = tree["L"]
    off = np.concatenate([[0], np.cumsum(tree["nbox"])])
    blocks, near = set(), set()
    for l in range(1, L + 1):
        keys = [int(k) for k in tree["box_key"][off[l]:off[l + 1]]]
        co = [_coords(k, l) for k in keys]
        par = [tuple(c >> 1 for c in p) for p in co]
        for i in range(len(keys)):
            for j in range(len(keys)):
                if i == j:
                    continue
                if par[i] != par[j] and adm(par[i], par[j]):
                    continue   # covered by the parents' block
                if adm(co[i], co[j]):
                    blocks.add((l, keys[i], keys[j]))
    keys = [int(k) for k in tree["box_key"][off[L]:off[L + 1]]]
    co = [_coords(k, L) for k in keys]
    for i in range(len(keys)):
        for j in range(len(keys)):
            if i == j or not adm(co[i], co[j]):
                near.add((keys[i], keys[j]))
    return blocks, near


MODES = {"strong": _strong_admissible, "weak": lambda a, b: a != b}


@pytest.mark.parametrize("mode", ["strong", "weak"])
@pytest.mark.parametrize("pts,leaf", [(I.grid(8), 8), (I.uniform(900, 35), 12), (I.sphere(1200, 36) * 0.99, 14)])
def test_variant_lists_match_definitions(mode, pts, leaf):
    o = O.Oracle(pts, leaf_size=leaf, admissibility=mode)
    t, li = o.tree(), o.lists()
    off = np.concatenate([[0], np.cumsum(t["nbox"])])
    bk = t["box_key"]
    blocks = {(int(l), int(bk[off[l] + a]), int(bk[off[l] + b])) for l, a, b in zip(li["level"], li["tgt"], li["src"])}
    near = {(int(bk[off[o.L] + a]), int(bk[off[o.L] + b])) for a, b in zip(li["near_tgt"], li["near_src"])}
    bb, bn = _brute_lists_mode(t, MODES[mode])
    assert blocks == bb and near == bn


def test_variant_counts_from_paper_tables():
    rows = [ln.split() for ln in open(os.path.join(HERE, "golden", "paper_block_counts_variants.txt"))
            if ln.strip() and not ln.startswith("#")]
    assert rows[0] == ["format", "L", "dense", "vertex", "edge_plus_face", "far"]
    for fmt, L, dense, vert, ef, far in rows[1:]:
        L = int(L)
        o = O.Oracle(I.grid(2 ** (L + 1)), leaf_size=8, admissibility=fmt)
        assert o.L == L
        li = o.lists()
        assert o.n_near == int(dense)
        assert int(np.sum(li["cls"] == 3)) == int(vert)
        assert int(np.sum((li["cls"] == 1) | (li["cls"] == 2))) == int(ef)
        assert int(np.sum(li["cls"] == 4)) == int(far)


@pytest.mark.parametrize("mode", ["strong", "weak"])
def test_variant_covers_every_entry_once(mode):
    pts = I.uniform(600, 37)
    o = O.Oracle(pts, leaf_size=9, admissibility=mode)
    t, li = o.tree(), o.lists()
    off = np.concatenate([[0], np.cumsum(t["nbox"])])
    cover = np.zeros((600, 600), np.int32)
    for a, b in zip(li["near_tgt"], li["near_src"]):
        ia, ib = off[o.L] + a, off[o.L] + b
        cover[t["box_start"][ia]:t["box_end"][ia], t["box_start"][ib]:t["box_end"][ib]] += 1
    for l, a, b in zip(li["level"], li["tgt"], li["src"]):
        ia, ib = off[l] + a, off[l] + b
        cover[t["box_start"][ia]:t["box_end"][ia], t["box_start"][ib]:t["box_end"][ib]] += 1
    assert cover.min() == 1 and cover.max() == 1
