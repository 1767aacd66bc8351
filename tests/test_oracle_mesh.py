"""Pins of the oracle's octree mesh: tiling, 2:1 balance, refinement predicate, hanging nodes.

Checked by brute force, independently of the oracle's own search structures: every pair of
touching leaves, every leaf corner against every touching leaf.
"""
import numpy as np
import pytest

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import inputs as I


def _morton(ijk):
    x = ijk.astype(np.uint64)
    r = np.zeros(x.shape[0], np.uint64)
    for b in range(21):
        for k in range(3):
            r |= ((x[:, k] >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + k)
    return r


@pytest.fixture(scope="module")
def adaptive():
    reg = [I.Region(I.REGION_SPHERE_BAND, 5, (0.45, 0.5, 0.55, 0.2, 0.04)),
           I.Region(I.REGION_BOX, 4, (0.6, 0.3, 0.3, 0.9, 0.45, 0.5))]
    return OracleMesh((0, 0, 0), (1, 1, 1), 2, reg)


def _boxes(m):
    size = (1 << (20 - m.levels.astype(np.int64)))
    lo = m.anchors.astype(np.int64)
    return lo, lo + size[:, None], size


def test_leaves_tile_the_domain(adaptive):
    m = adaptive
    lo, hi, size = _boxes(m)
    assert (size.astype(np.float64) ** 3).sum() == float(np.prod(m.hiI.astype(np.float64)))
    keys = _morton(lo)
    assert np.all(np.diff(keys.astype(np.float64)) > 0)          # Morton-sorted, distinct
    # disjoint: no leaf contains another leaf's anchor
    for e in range(0, m.n_elem, 7):
        inside = np.all((lo >= lo[e]) & (lo < hi[e]), axis=1)
        assert inside.sum() == 1


def test_two_to_one_balance_brute_force(adaptive):
    m = adaptive
    lo, hi, _ = _boxes(m)
    lev = m.levels.astype(np.int64)
    for s in range(0, m.n_elem, 256):
        a = slice(s, s + 256)
        touch = np.all((lo[a, None, :] <= hi[None, :, :]) & (hi[a, None, :] >= lo[None, :, :]), axis=2)
        dl = np.abs(lev[a, None] - lev[None, :])
        assert not np.any(touch & (dl > 1))


def test_refinement_predicate_met(adaptive):
    m = adaptive
    lo, hi, _ = _boxes(m)
    b0 = lo * m.scale
    b1 = hi * m.scale
    c = np.array([0.45, 0.5, 0.55])
    near = np.maximum(np.maximum(b0 - c, c - b1), 0.0)
    dmin = np.sqrt((near ** 2).sum(1))
    far = np.maximum(np.abs(b0 - c), np.abs(b1 - c))
    dmax = np.sqrt((far ** 2).sum(1))
    band = (dmin <= 0.24) & (dmax >= 0.16)
    assert np.all(m.levels[band] >= 5)
    box = np.all((b0 <= np.array([0.9, 0.45, 0.5])) & (b1 >= np.array([0.6, 0.3, 0.3])), axis=1)
    assert np.all(m.levels[box] >= 4)
    assert np.all(m.levels >= 2)


def test_hanging_nodes_are_edge_or_face_midpoints(adaptive):
    m = adaptive
    assert m.n_hang > 0
    for h in range(m.n_hang):
        k = m.hang_np[h]
        assert k in (2, 4)
        P = m.node_ijk[m.hang_parents[h, :k]].astype(np.int64)
        assert np.array_equal(P.sum(0), k * m.hang_ijk[h].astype(np.int64))


def test_corners_are_nodes_exactly_when_corners_of_every_touching_leaf(adaptive):
    m = adaptive
    lo, hi, size = _boxes(m)
    nodes = {tuple(x) for x in m.node_ijk.astype(np.int64)}
    hang = {tuple(x) for x in m.hang_ijk.astype(np.int64)}
    assert len(nodes) == m.n_nodes and not (nodes & hang)
    for e in range(0, m.n_elem, 3):
        for c in range(8):
            P = lo[e] + np.array([(c >> k) & 1 for k in range(3)]) * size[e]
            touching = np.all((lo <= P) & (hi >= P), axis=1)
            corner = np.all((P == lo[touching]) | (P == hi[touching]), axis=1)
            idx = m.conn[e, c]
            if corner.all():
                assert idx < m.n_nodes and tuple(m.node_ijk[idx]) == tuple(P)
            else:
                assert idx >= m.n_nodes and tuple(m.hang_ijk[idx - m.n_nodes]) == tuple(P)


def test_linear_field_is_continuous_across_hanging_faces(adaptive):
    m = adaptive
    X = m.node_xyz
    f = 0.3 + X @ np.array([1.25, -0.5, 2.0])
    for h in range(m.n_hang):
        k = m.hang_np[h]
        v = f[m.hang_parents[h, :k]].sum() / k
        x = m.lo + m.hang_ijk[h] * m.scale
        assert abs(v - (0.3 + x @ np.array([1.25, -0.5, 2.0]))) <= 1e-14


def test_nodes_sorted_by_morton(adaptive):
    keys = _morton(adaptive.node_ijk)
    assert np.all(np.diff(keys.astype(np.float64)) > 0)


def test_carved_box_domain():
    # 2 x 1 x 1 box in a root cube of side 2: only leaves inside the box are kept
    m = OracleMesh((0, 0, 0), (2, 1, 1), 2, [I.Region(I.REGION_SPHERE_BAND, 4, (0.7, 0.5, 0.5, 0.2, 0.05))])
    lo, hi, size = _boxes(m)
    assert np.all(hi <= m.hiI[None, :])
    assert (size.astype(np.float64) ** 3).sum() == float(np.prod(m.hiI.astype(np.float64)))
