"""CPU checks of the C-ABI library: it builds for sm_103a, loads, exports every declared entry
point, validates its arguments, and its host mesh builder agrees bit for bit with the oracle's
(octree, nodes, hanging nodes, background triangles).  No GPU is touched (device < 0)."""
import ctypes as C
import os
import re

import numpy as np
import pytest

from oracle.oracle import OracleMesh
from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    _lib.build()
    return _lib.load()


def declared_entry_points():
    names = set()
    for h in os.listdir(os.path.join(ROOT, "include")):
        if h.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", h)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(imga_\w+)\s*\(", txt))
    return names


def test_every_declared_symbol_is_exported(lib):
    names = declared_entry_points()
    assert {"imga_build_mesh", "imga_classify", "imga_residual", "imga_jvp"} <= names
    for n in names:
        assert hasattr(lib, n), n
    assert names <= set(_lib.SIGNATURES), names - set(_lib.SIGNATURES)


def _compare(w_lo, w_hi, base, regions, tri, lmax=3):
    m = api.Mesh(w_lo, w_hi, base, regions, tri, lmax, device=-1)
    o = OracleMesh(w_lo, w_hi, base, regions, tri, lmax)
    ex = m.export()
    assert m.n_elem == o.n_elem and m.n_nodes == o.n_nodes and m.n_hang == o.n_hang
    assert np.array_equal(ex["anchors"], o.anchors)
    assert np.array_equal(ex["levels"], o.levels)
    assert np.array_equal(ex["conn"], o.conn)
    assert np.array_equal(ex["node_ijk"], o.node_ijk)
    assert np.array_equal(ex["hang_parents"], o.hang_parents)
    assert np.array_equal(ex["hang_np"], o.hang_np)
    off, ids = m.background()
    for e in range(m.n_elem):
        assert np.array_equal(ids[off[e]:off[e + 1]], o.background_triangles(e)), e
    return m


def test_host_mesh_matches_oracle_small_sphere(lib):
    w = I.small_sphere()
    m = _compare(w.lo, w.hi, w.base_level, w.regions, w.triangles(), w.lmax)
    assert m.n_hang > 0


def test_host_mesh_matches_oracle_carved_box_and_cone(lib):
    regs = [I.Region(I.REGION_SPHERE_BAND, 6, (1.0, 0.5, 0.5, 0.12, 0.04)),
            I.Region(I.REGION_CONE, 5, (1.0, 0.5, 0.5, 0.7, 0.1, 0.27)),
            I.Region(I.REGION_BOX, 4, (0.2, 0.1, 0.1, 0.5, 0.4, 0.3))]
    tri = I.icosphere(2, 0.12, (1.0, 0.5, 0.5), 1e-4, 4)
    _compare((0, 0, 0), (2, 1, 1), 2, regs, tri)


@pytest.mark.parametrize("c", [(0.501, 0.502, 0.497), (0.26, 0.51, 0.74), (0.126, 0.377, 0.624)])
def test_host_mesh_matches_oracle_deep_refinement(lib, c):
    # a level-9 band in a level-1 mesh: 2:1 balance ripples outwards over 5 to 7 passes, the
    # later ones probing only from the leaves that the previous pass created or that found a
    # violation; the oracle rescans every leaf on every pass
    m = _compare((0, 0, 0), (1, 1, 1), 1, [I.Region(I.REGION_SPHERE_BAND, 9, (*c, 0.01, 0.002))], None)
    assert m.n_hang > 0 and int(m.export()["levels"].max()) == 9


def test_host_mesh_without_body(lib):
    _compare((0, 0, 0), (1, 1, 1), 2, [I.Region(I.REGION_SPHERE_BAND, 4, (0.3, 0.6, 0.5, 0.2, 0.05))], None)


def test_bsr_pattern_matches_oracle_assembly(lib):
    """The block pattern of the assembled Jacobian (imga_bsr_pattern, built on the host) equals the
    pattern of the oracle's block assembly, index for index."""
    from oracle import sparse as S
    c = (0.5, 0.5, 0.5)
    regs = [I.Region(I.REGION_SPHERE_BAND, 4, (*c, 0.2, 0.05))]
    tri = I.icosphere(2, 0.2, c, 1e-4, 3)
    m = api.Mesh((0, 0, 0), (1, 1, 1), 2, regs, tri, 3, device=-1)
    o = OracleMesh((0, 0, 0), (1, 1, 1), 2, regs, tri, 3)
    ptr, idx = m.bsr_pattern()
    u, up, _ = I.state(o.n_nodes, 2)
    A = S.assemble_bsr(o, I.Physics(), u, up)
    assert m.n_hang > 0 and ptr[-1] == idx.size == A.indices.size
    assert np.array_equal(ptr, A.indptr) and np.array_equal(idx, A.indices)
    # a mesh without a body, and a repeated call (the pattern is kept)
    m2 = api.Mesh((0, 0, 0), (2, 1, 1), 1, [I.Region(I.REGION_BOX, 3, (0.2, 0.1, 0.1, 0.5, 0.4, 0.3))], None, 3, device=-1)
    p1, i1 = m2.bsr_pattern()
    p2, i2 = m2.bsr_pattern()
    assert np.array_equal(p1, p2) and np.array_equal(i1, i2) and np.all(np.diff(p1) >= 8)


def test_node_coords_match_oracle(lib):
    w = I.small_sphere()
    m = api.Mesh(w.lo, w.hi, w.base_level, w.regions, w.triangles(), w.lmax, device=-1)
    o = OracleMesh(w.lo, w.hi, w.base_level, w.regions, w.triangles(), w.lmax)
    xyz = m.node_coords()
    assert xyz.shape == (o.n_nodes, 3) and np.array_equal(xyz, o.node_xyz)
    assert lib.imga_node_coords(None, xyz.ctypes.data_as(C.c_void_p), None) == 1
    assert lib.imga_node_coords(m.h, None, None) == 1


def test_invalid_arguments_are_rejected(lib):
    with pytest.raises(_lib.ImgaError) as e:
        api.Mesh((0, 0, 0), (1, 0.3, 1), 1, [], None, 3, device=-1)      # edge not a whole number of cells
    assert e.value.status == 1
    with pytest.raises(_lib.ImgaError):
        api.Mesh((0, 0, 0), (1, 1, 1), 1, [], None, 7, device=-1)        # L_max out of range
    with pytest.raises(_lib.ImgaError) as e:
        bad = np.zeros((1, 3, 3))
        api.Mesh((0, 0, 0), (1, 1, 1), 1, [], bad, 3, device=-1)         # zero-area triangle
    assert e.value.status == 4
    m = api.Mesh((0, 0, 0), (1, 1, 1), 1, [], None, 3, device=-1)
    ph = api.physics_struct(I.Physics())
    st = lib.imga_residual(m.h, C.c_void_p(16), C.c_void_p(16), None, None, C.byref(ph), 0, C.c_void_p(16), None)
    assert st == 1                                                        # host-only mesh: no compute
    assert b"host-only" in lib.imga_last_error()


def test_options_and_queries_reject_bad_arguments(lib):
    m = api.Mesh((0, 0, 0), (1, 1, 1), 1, [], None, 3, device=-1)
    # graphs, autotune, ray-only classify, deterministic, fused, fused split, side streams
    for opt in (1, 2, 3, 4, 5, 6, 7):
        assert lib.imga_set_option(m.h, opt, 1) == 1                      # host-only mesh
    assert lib.imga_set_option(None, 1, 1) == 1
    fused = np.zeros(6, np.int64)
    assert lib.imga_fused_info(None, fused.ctypes.data_as(C.c_void_p)) == 1
    assert lib.imga_fused_info(m.h, None) == 1
    assert lib.imga_fused_info(m.h, fused.ctypes.data_as(C.c_void_p)) == 0
    assert fused[0] == 0 and fused[5] == 4                                # off; all 4 warps start on costly items
    bps = np.zeros(4, np.int32)
    assert lib.imga_tuning_interior(None, bps.ctypes.data_as(C.c_void_p), None) == 1
    assert lib.imga_tuning_interior(m.h, bps.ctypes.data_as(C.c_void_p), None) == 0 and (bps == 0).all()   # not tuned
    counts = np.zeros(4, np.int64)
    assert lib.imga_classify_counts(m.h, counts.ctypes.data_as(C.c_void_p), 0) == 1   # host-only: no counts
    assert lib.imga_classify_counts(None, counts.ctypes.data_as(C.c_void_p), 0) == 1
    assert lib.imga_classify_counts(m.h, None, 0) == 1
    assert lib.imga_bsr_pattern(None, C.byref(C.c_int64()), None, None) == 1
    assert lib.imga_bsr_pattern(m.h, None, None, None) == 1
    assert lib.imga_tuning(None, None, None) == 1
    shape = np.zeros(8, np.int32)
    assert lib.imga_tuning(m.h, shape.ctypes.data_as(C.c_void_p), None) == 0
    assert (shape.reshape(2, 2, 2)[..., 0] == 4).all() and (shape.reshape(2, 2, 2)[..., 1] == 0).all()   # defaults
    bad = C.c_int64()
    assert lib.imga_selftest_conversions(0, -1, 1, C.byref(bad)) == 1    # n < 0
    assert lib.imga_selftest_conversions(0, 10, 1, None) == 1             # null output
