"""Pins of the oracle's geometry: in/out classification, markers, adaptive and surface quadrature.

References that do not come from the oracle:
* the 2-point Gauss abscissae printed in the paper's adaptive-quadrature figure (golden file);
* exact volumes and exact integrals of trilinear functions for cuts along dyadic sub-cell planes;
* the analytic sphere (inscribed / circumscribed radii of the faceted surface);
* an independent brute-force ray-parity count written here with numpy along a random direction;
* the divergence theorem for the triangulated surface (sum w n = 0, sum w x.n = 3 V, and the
  quadratic fluxes x_i x_j n_k against the first moment of the polyhedron);
* the barycentric moment formula int_T l_a l_b dA = A (1 + delta_ab) / 12 on each triangle.
"""
import os

import numpy as np
import pytest

from oracle import oracle as O
from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden", "fig_gp_gauss_abscissae.txt")


def box_body(lo, hi):
    return I.rounded_box(lo, hi, 0.0, 1)


def test_box_body_is_closed_and_outward():
    t = box_body((-1, -1, -1), (0.25, 2, 2))
    assert t.shape == (12, 3, 3)
    n = np.cross(t[:, 1] - t[:, 0], t[:, 2] - t[:, 0])
    vol = np.einsum("ij,ij->i", t[:, 0], np.cross(t[:, 1], t[:, 2])).sum() / 6.0
    assert abs(vol - 1.25 * 3 * 3) < 1e-12
    assert np.abs(n.sum(0)).max() < 1e-12


def test_first_split_points_match_printed_gauss_abscissae():
    printed = np.loadtxt(GOLD)
    m = OracleMesh((0, 0, 0), (1, 1, 1), 1, [], box_body((-1, -1, -1), (0.25, 2, 2)), lmax=3)
    mk, _, _ = m.markers()
    e = 0                                   # [0, 0.5]^3, cut by the plane x = 0.25 through its middle
    assert mk[e] == 2
    q = m.cut_points(e)
    assert q.shape[0] == 32                 # four level-1 children fully Out, 8 points each
    assert np.allclose(q[:, 3], 1.0 / 8.0)
    frac = np.mod(q[:, :3] + 1.0, 1.0)      # position inside the level-1 child, unit edge
    for k in range(3):
        vals = np.unique(np.round(frac[:, k], 9))
        assert np.allclose(np.sort(vals), np.sort(printed), atol=1e-10)
    assert np.all(q[:, 0] > 0.0)            # only the Out half (x > 0.25) carries points


def test_dyadic_plane_cut_is_exact():
    # plane x = 0.3125 lies on a level-3 sub-cell face of [0, 0.5]^3 (xi = 0.25)
    m = OracleMesh((0, 0, 0), (1, 1, 1), 1, [], box_body((-1, -1, -1), (0.3125, 2, 2)), lmax=3)
    q = m.cut_points(0)
    w = q[:, 3]
    assert abs(w.sum() - 8.0 * 0.375) <= 1e-14
    f = (1.0 + q[:, 0]) * (2.0 - q[:, 1]) * (0.5 + q[:, 2]) * (1.0 + 0.5 * q[:, 0] ** 2)
    # int_{0.25}^1 (1+x)(1+x^2/2) dx * int_{-1}^1 (2-y) dy * int_{-1}^1 (0.5+z) dz
    fx = lambda x: x + x ** 2 / 2 + x ** 3 / 6 + x ** 4 / 8
    exact = (fx(1.0) - fx(0.25)) * 4.0 * 1.0
    assert abs((w * f).sum() - exact) <= 1e-13


def _halfspace_volume(a, d):
    """Volume of {y in [0,1]^3 : a.y <= d} for a > 0 (inclusion-exclusion over the cube's corners)."""
    s = 0.0
    for v in range(8):
        bits = np.array([(v >> k) & 1 for k in range(3)], dtype=float)
        s += (-1) ** int(bits.sum()) * max(d - a @ bits, 0.0) ** 3
    return s / (6.0 * np.prod(a))


def _plane_body(a, d):
    """Tetrahedron whose face lies on a.x = d, every other face ~20 units away: inside the unit
    cube the body is the half-space a.x < d."""
    an = a / np.linalg.norm(a)
    c0 = an * d / np.linalg.norm(a)
    u = np.cross(an, [0.0, 0.0, 1.0])
    u /= np.linalg.norm(u)
    w = np.cross(an, u)
    P = [c0 + 20.0 * (np.cos(t) * u + np.sin(t) * w) for t in (0.0, 2 * np.pi / 3, 4 * np.pi / 3)]
    apex = c0 - 20.0 * an
    return np.array([[P[0], P[1], P[2]], [apex, P[1], P[0]], [apex, P[2], P[1]], [apex, P[0], P[2]]])


def test_oblique_plane_cut_quadrature():
    """Sub-cells are judged by their 8 Gauss points (Fig. GP caption): an Intercepted element
    whose level-0 Gauss points all fall on one side keeps all 8 (all Out) or none (all In);
    the others approach the exact clipped volume as the split level grows."""
    a, d, h = np.array([1.0, 0.7, 0.4]), 0.83, 1.0 / 8.0
    tri = _plane_body(a, d)
    G = 1.0 / np.sqrt(3.0)
    gp = np.array([[G if (g >> k) & 1 else -G for k in range(3)] for g in range(8)])
    errs = []
    for lmax in (1, 2, 3):
        m = OracleMesh((0, 0, 0), (1, 1, 1), 3, [], tri, lmax=lmax)
        mk, cf, _ = m.markers()
        E = 0.0
        for el in range(m.n_elem):
            x0 = m.anchors[el] * m.scale
            corners = x0 + np.array([[(c >> k) & 1 for k in range(3)] for c in range(8)]) * h
            cin = corners @ a < d
            assert mk[el] == (1 if cin.all() else 0 if not cin.any() else 2)
            if mk[el] != 2:
                continue
            got = m.cut_points(el)[:, 3].sum() * (h / 2) ** 3
            side_out = (x0 + (gp + 1.0) * h / 2) @ a > d
            if side_out.all():
                assert got == h ** 3
            elif not side_out.any():
                assert got == 0.0
            else:
                exact = h ** 3 * (1.0 - _halfspace_volume(a * h, d - a @ x0))
                assert abs(got - exact) <= h ** 3
                E += abs(got - exact)
        errs.append(E)
    assert errs[1] < errs[0] / 2.0 and errs[2] < errs[0] / 3.0


# ---------------------------------------------------------------------------------------
# in/out
# ---------------------------------------------------------------------------------------
def brute_parity(pts, tri, d):
    """Independent ray-parity count (numpy), direction d; returns (inside, ok) where ok is
    False for rays that pass within 1e-9 of a triangle edge."""
    v0, v1, v2 = tri[:, 0], tri[:, 1], tri[:, 2]
    e1, e2 = v1 - v0, v2 - v0
    pv = np.cross(d, e2)
    det = np.einsum("ij,ij->i", e1, pv)
    tv = pts[:, None, :] - v0[None]
    with np.errstate(divide="ignore", invalid="ignore"):
        u = np.einsum("pij,ij->pi", tv, pv) / det
        qv = np.cross(tv, e1[None])
        v = np.einsum("pij,j->pi", qv, d) / det
        t = np.einsum("pij,ij->pi", qv, e2) / det
    hit = (u >= 0) & (v >= 0) & (u + v <= 1) & (t > 0)
    near = (np.minimum(np.minimum(np.abs(u), np.abs(v)), np.abs(1 - u - v)) < 1e-9) & (t > 0) & \
           (u > -1e-9) & (v > -1e-9) & (u + v < 1 + 1e-9)
    return (hit.sum(1) % 2 == 1), ~near.any(1)


def _check_classification(m, tri, pts, seed):
    d = I.normal(seed, 3)
    d /= np.linalg.norm(d)
    truth, ok = brute_parity(pts, tri, d)
    got = m.classify(pts).astype(bool)
    assert ok.mean() > 0.99
    assert np.array_equal(got[ok], truth[ok])
    return got, truth


def test_inout_icosphere_vs_brute_force_and_analytic():
    c = np.array([0.5, 0.5, 0.5])
    tri = I.icosphere(2, 0.3, c, 1e-4, 3)
    m = OracleMesh((0, 0, 0), (1, 1, 1), 3, [I.Region(I.REGION_SPHERE_BAND, 5, (*c, 0.3, 0.04))], tri)
    pts = I.uniform(21, 3 * 4000).reshape(-1, 3)
    got, _ = _check_classification(m, tri, pts, 5)
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    n /= np.linalg.norm(n, axis=1)[:, None]
    r_in = np.min(np.einsum("ij,ij->i", tri[:, 0] - c, n))
    r_out = np.max(np.linalg.norm(tri.reshape(-1, 3) - c, axis=1))
    r = np.linalg.norm(pts - c, axis=1)
    assert np.all(got[r < r_in - 1e-9]) and not np.any(got[r > r_out + 1e-9])
    cnt = m.counters()
    assert cnt["normal_decided"] > 0.5 * cnt["normal_tests"]


def binned_parity(pts, tri, d):
    """Ray parity along d like brute_parity, for many points: the points are sorted by their
    coordinate along one axis perpendicular to d, so that each triangle only tests the points in
    its slab.  Returns (inside, ok), ok False within 1e-9 of a triangle edge."""
    d = d / np.linalg.norm(d)
    a = np.cross(d, [1.0, 0.0, 0.0] if abs(d[0]) < 0.9 else [0.0, 1.0, 0.0])
    a /= np.linalg.norm(a)
    b = np.cross(d, a)
    pa, pb = pts @ a, pts @ b
    order = np.argsort(pa)
    sa = pa[order]
    hits = np.zeros(pts.shape[0], np.int64)
    near = np.zeros(pts.shape[0], bool)
    for t in tri:
        ta, tb = t @ a, t @ b
        i0, i1 = np.searchsorted(sa, ta.min() - 1e-9), np.searchsorted(sa, ta.max() + 1e-9, side="right")
        idx = order[i0:i1]
        idx = idx[(pb[idx] >= tb.min() - 1e-9) & (pb[idx] <= tb.max() + 1e-9)]
        if idx.size == 0:
            continue
        e1, e2 = t[1] - t[0], t[2] - t[0]
        pv = np.cross(d, e2)
        det = e1 @ pv
        if det == 0.0:
            continue
        tv = pts[idx] - t[0]
        u = (tv @ pv) / det
        qv = np.cross(tv, e1)
        v = (qv @ d) / det
        tt = (qv @ e2) / det
        hit = (u >= 0) & (v >= 0) & (u + v <= 1) & (tt > 0)
        close = (np.minimum(np.minimum(np.abs(u), np.abs(v)), np.abs(1 - u - v)) < 1e-9) & (tt > 0) & \
                (u > -1e-9) & (v > -1e-9) & (u + v < 1 + 1e-9)
        hits[idx] += hit
        near[idx] |= close
    return hits % 2 == 1, ~near


def _grid_plane_boxes(seed):
    """Two filleted boxes (fillet 1/32) whose flat faces lie on planes of the level-5 grid of the
    unit cube, up to a vertex jitter of 1e-5."""
    return np.concatenate([I.rounded_box((0.25, 0.25, 0.3125), (0.75, 0.625, 0.6875), 1.0 / 32, 16, 1e-5, seed),
                           I.rounded_box((0.78125, 0.25, 0.3125), (0.90625, 0.5, 0.5), 1.0 / 32, 8, 1e-5, seed + 7)])


def _inout_errors(pad, seed=1):
    """Oracle in/out against binned ray parity along a random direction, for the 5^3 Gauss points
    of every Intercepted element and the corners of every element with background triangles.
    Returns (point errors, corner errors, points checked)."""
    tri = _grid_plane_boxes(seed)
    O.set_bt_pad(pad)
    try:
        m = OracleMesh((0, 0, 0), (1, 1, 1), 5, [], tri, 3)
        mk, cf, nbt = m.markers()
        h = 1.0 / 32
        xi = np.polynomial.legendre.leggauss(5)[0]
        G = np.stack(np.meshgrid(xi, xi, xi, indexing="ij"), -1).reshape(-1, 3)
        x0 = m.anchors.astype(np.float64) * m.scale
        cut = np.where(mk == 2)[0]
        pts = (x0[cut][:, None, :] + 0.5 * h * (G[None] + 1.0)).reshape(-1, 3)
        got = m.classify(pts).astype(bool)
        has = np.where(nbt > 0)[0]
        off = np.array([[(c >> k) & 1 for k in range(3)] for c in range(8)], dtype=np.float64)
        corners = (x0[has][:, None, :] + h * off[None]).reshape(-1, 3)
        cflag = (((cf[has][:, None] >> np.arange(8)[None]) & 1) == 1).reshape(-1)
    finally:
        O.set_bt_pad(1e-2)
    d = I.normal(5, 3)
    truth, ok = binned_parity(pts, tri, d)
    ctruth, cok = binned_parity(corners, tri, d)
    assert ok.mean() > 0.999 and cok.mean() > 0.99
    return int((got != truth)[ok].sum()), int((cflag != ctruth)[cok].sum()), int(ok.sum())


def test_inout_exact_with_faces_on_grid_planes():
    """Faces on grid planes: with B_T taken over the element box widened by 1e-2 of its edge, the
    normal test with ray fallback (Algorithm 6) and the markers (Algorithm 5) agree with ray
    parity at every Gauss point and every corner."""
    pe, ce, n = _inout_errors(1e-2)
    assert (pe, ce) == (0, 0) and n > 200000


def test_inout_plain_box_overlap_misclassifies_with_faces_on_grid_planes():
    """The same body with B_T over the exact closed box: points just in front of a face whose
    triangles miss the element box, behind the planes of the triangles that reach in, are called
    In.  This is what the widening removes."""
    pe, ce, n = _inout_errors(0.0)
    assert pe > 0 and ce > 0


def test_inout_two_disjoint_bodies_and_polyhedra():
    tri = np.concatenate([I.icosphere(2, 0.15, (0.3, 0.5, 0.5), 1e-4, 1), I.icosphere(1, 0.12, (0.72, 0.45, 0.55), 1e-4, 2),
                          box_body((0.1, 0.1, 0.1), (0.3, 0.25, 0.2))])
    tet = np.array([[[0.6, 0.8, 0.7], [0.9, 0.8, 0.7], [0.6, 0.95, 0.7]], [[0.6, 0.8, 0.7], [0.6, 0.8, 0.9], [0.9, 0.8, 0.7]],
                    [[0.6, 0.8, 0.7], [0.6, 0.95, 0.7], [0.6, 0.8, 0.9]], [[0.9, 0.8, 0.7], [0.6, 0.8, 0.9], [0.6, 0.95, 0.7]]])
    cen = tet.reshape(-1, 3).mean(0)
    nrm = np.cross(tet[:, 1] - tet[:, 0], tet[:, 2] - tet[:, 0])
    flip = np.einsum("ij,ij->i", nrm, tet.mean(1) - cen) < 0
    tet[flip] = tet[flip][:, [0, 2, 1]]
    tri = np.concatenate([tri, tet])
    m = OracleMesh((0, 0, 0), (1, 1, 1), 3, [I.Region(I.REGION_BOX, 5, (0.05, 0.05, 0.05, 0.95, 0.95, 0.95))], tri)
    pts = I.uniform(33, 3 * 3000).reshape(-1, 3)
    got, truth = _check_classification(m, tri, pts, 7)
    assert truth.sum() > 50


def test_markers_vs_analytic_corner_distances(small_sphere_oracle):
    w, m = small_sphere_oracle
    tri = w.triangles()
    c = np.array([0.5, 0.5, 0.5])
    n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
    n /= np.linalg.norm(n, axis=1)[:, None]
    r_in = np.min(np.einsum("ij,ij->i", tri[:, 0] - c, n)) - 1e-9
    r_out = np.max(np.linalg.norm(tri.reshape(-1, 3) - c, axis=1)) + 1e-9
    mk, cf, _ = m.markers()
    size = (1 << (20 - m.levels.astype(np.int64))) * m.scale
    corners = m.anchors[:, None, :] * m.scale + np.array([[(k >> j) & 1 for j in range(3)] for k in range(8)])[None] * size[:, None, None]
    r = np.linalg.norm(corners - c, axis=2)
    out_all = np.all(r > r_out, axis=1)
    in_all = np.all(r < r_in, axis=1)
    mixed = np.any(r < r_in, axis=1) & np.any(r > r_out, axis=1)
    assert np.all(mk[out_all] == 0) and np.all(mk[in_all] == 1) and np.all(mk[mixed] == 2)
    assert (mk == 2).sum() > 100
    # corner flags agree with the analytic verdict wherever it is unambiguous
    cin = ((cf[:, None] >> np.arange(8)[None]) & 1).astype(bool)
    assert np.all(cin[r < r_in]) and not np.any(cin[r > r_out])


def test_surface_quadrature_identities(small_sphere_oracle):
    w, m = small_sphere_oracle
    tri = w.triangles()
    sq = m.surface_points()
    assert sq.shape[0] == 3 * tri.shape[0]
    area = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1).sum()
    vol = np.einsum("ij,ij->i", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum() / 6.0
    x, n, wq, hb, el = sq[:, :3], sq[:, 3:6], sq[:, 6], sq[:, 7], sq[:, 8].astype(np.int64)
    assert abs(wq.sum() - area) <= 1e-14 * area * 10
    assert np.abs((wq[:, None] * n).sum(0)).max() <= 1e-15 * 10
    assert abs((wq * np.einsum("ij,ij->i", x, n)).sum() + 3.0 * vol) <= 1e-13
    h = (1 << (20 - m.levels[el].astype(np.int64))) * m.scale
    assert np.all(hb >= 0.01 * h - 1e-18) and np.all(hb <= np.sqrt(3) * h)
    # every point lies in the closed box of its owning element
    lo = m.anchors[el] * m.scale
    assert np.all((x >= lo - 1e-15) & (x <= lo + h[:, None] + 1e-15))


def test_surface_quadrature_is_exact_for_quadratics(small_sphere_oracle):
    """The Nitsche integrands of Eq. (weakbc) are products of trilinear fields restricted to flat
    triangles; the surface rule must integrate every quadratic exactly on each triangle.  Two
    closed forms that do not involve the rule's points:
    * per triangle, int_T x_i x_j dA = A/12 (sum_a v_ai v_aj + s_i s_j), s = v_0 + v_1 + v_2,
      from the barycentric moments int_T l_a l_b dA = A (1 + delta_ab) / 12;
    * over the closed surface, by the divergence theorem applied to x_i x_j e_k with the
      fluid-outward (body-inward) normal, sum_q w x_i x_j n_k = -(delta_ik M_j + delta_jk M_i),
      M = int_V x dV summed over the signed tetrahedra (0, a, b, c) as vol (a + b + c) / 4."""
    w, m = small_sphere_oracle
    tri = w.triangles()
    sq = m.surface_points()
    x, n, wq, t = sq[:, :3], sq[:, 3:6], sq[:, 6], sq[:, 9].astype(np.int64)
    A = 0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1)
    s = tri.sum(axis=1)
    exact = (A[:, None, None] / 12.0) * (np.einsum("tai,taj->tij", tri, tri) + s[:, :, None] * s[:, None, :])
    got = np.zeros_like(exact)
    np.add.at(got, t, wq[:, None, None] * x[:, :, None] * x[:, None, :])
    assert np.abs(got - exact).max() <= 1e-14 * np.abs(exact).max()
    # linear moments per triangle: int_T x dA = A s / 3
    lin = np.zeros((tri.shape[0], 3))
    np.add.at(lin, t, wq[:, None] * x)
    assert np.abs(lin - A[:, None] * s / 3.0).max() <= 1e-14 * np.abs(s).max() * A.max()
    vol_t = np.einsum("ti,ti->t", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])) / 6.0
    M = (vol_t[:, None] * s / 4.0).sum(axis=0)
    D = np.eye(3)
    want = -(D[:, None, :] * M[None, :, None] + D[None, :, :] * M[:, None, None])   # [i, j, k]
    flux = np.einsum("q,qi,qj,qk->ijk", wq, x, x, n)
    assert np.abs(flux - want).max() <= 1e-13 * np.abs(want).max()
    # the rule is the degree-2 one: the third central moment of x over a triangle is not exact
    c = s / 3.0
    d = tri[:, :, 0] - c[:, 0:1]                                   # vertices relative to the centroid
    cub = np.zeros(tri.shape[0])
    np.add.at(cub, t, wq * (x[:, 0] - c[t, 0]) ** 3)
    e3 = 6 * (d ** 3).sum(1) + 6 * sum(d[:, a] ** 2 * d[:, b] for a in range(3) for b in range(3) if a != b) \
        + 6 * d[:, 0] * d[:, 1] * d[:, 2]
    cub_exact = (2.0 * A / 120.0) * e3                             # int l^a l^b l^c = 2A a!b!c!/(a+b+c+2)!
    big = np.abs(cub_exact) > 1e-3 * np.abs(cub_exact).max()
    assert np.median(np.abs(cub - cub_exact)[big] / np.abs(cub_exact)[big]) > 0.1


def test_total_quadrature_volume_is_box_minus_body(small_sphere_oracle):
    """Sum of all volume weights = box volume - polyhedron volume, within the sub-cell resolution:
    Out elements give h^3, Intercepted elements the weights of their kept sub-cell points
    (reference weight x h^3 / 8), In elements nothing.  The polyhedron volume is exact (divergence
    theorem over the triangles); the error is bounded by the surface area times the finest
    sub-cell edge h / 2^L_max (a quarter of it is asserted)."""
    w, m = small_sphere_oracle
    mk, _, _ = m.markers()
    root = max(np.subtract(w.hi, w.lo))
    h = root * 2.0 ** -m.levels.astype(np.float64)
    vol = float(np.sum(h[mk == 0] ** 3))
    for e in np.where(mk == 2)[0]:
        vol += float(m.cut_points(e)[:, 3].sum()) * h[e] ** 3 / 8.0
    tri = w.triangles()
    v_body = float(np.einsum("ij,ij->i", tri[:, 0], np.cross(tri[:, 1], tri[:, 2])).sum()) / 6.0
    area = float(0.5 * np.linalg.norm(np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0]), axis=1).sum())
    exact = float(np.prod(np.subtract(w.hi, w.lo))) - v_body
    h_fine = h[mk == 2].min() / 2 ** w.lmax
    assert abs(vol - exact) <= 0.25 * area * h_fine, (vol, exact, area * h_fine)   # measured 7e-6 vs 6e-5
    # the sub-cell quadrature matters: counting Intercepted elements whole is off by far more
    crude = vol - sum(float(m.cut_points(e)[:, 3].sum()) * h[e] ** 3 / 8.0 for e in np.where(mk == 2)[0]) \
        + float(np.sum(h[mk == 2] ** 3))
    assert abs(crude - exact) > 5 * abs(vol - exact)
