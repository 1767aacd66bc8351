"""Python handle on the plain FP64 CPU oracle (imga_oracle.cpp).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the CPU-baseline leg of the
benchmark use it; the product path never imports it.  It shares no code with the CUDA path.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "imga_oracle.cpp")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None

f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def build(force: bool = False) -> str:
    """Compile the oracle (plain g++, -ffp-contract=off so in/out decisions are reproducible)."""
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        os.makedirs(os.path.dirname(_OUT), exist_ok=True)
        tmp = _OUT + f".{os.getpid()}.tmp"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", tmp,
                               _SRC])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        vp, i64, i32, dp = C.c_void_p, C.c_int64, C.c_int, C.POINTER(C.c_double)
        L.or_build.restype = vp
        L.or_build.argtypes = [dp, dp, i32, i32, C.c_void_p, C.c_void_p, C.c_void_p, C.c_char_p, i32]
        L.or_free.argtypes = [vp]
        L.or_sizes.argtypes = [vp, C.c_void_p, C.c_void_p]
        L.or_export.argtypes = [vp] + [C.c_void_p] * 7
        L.or_find_leaf.argtypes = [vp, i64, i64, i64]
        L.or_find_leaf.restype = i32
        L.or_set_surface.argtypes = [vp, C.c_void_p, i64, i32]
        L.or_classify.argtypes = [vp, C.c_void_p, i64, C.c_void_p]
        L.or_markers.argtypes = [vp, C.c_void_p, i64, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_bt.argtypes = [vp, i64, C.c_void_p, i64]
        L.or_bt.restype = i64
        L.or_cut_points.argtypes = [vp, i64, C.c_void_p, i64]
        L.or_cut_points.restype = i64
        L.or_surface_points.argtypes = [vp, C.c_void_p, i64]
        L.or_surface_points.restype = i64
        L.or_counters.argtypes = [vp, C.c_void_p]
        L.or_set_bt_pad.argtypes = [C.c_double]
        L.or_set_threads.argtypes = [i32]
        L.or_surface_force.argtypes = [vp, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_set_dirichlet.argtypes = [vp, C.c_void_p, C.c_void_p]
        L.or_set_surface_velocity.argtypes = [vp, C.c_void_p, i64]
        L.or_set_surface_velocity.restype = i32
        L.or_residual_jvp.argtypes = [vp, C.c_void_p] + [C.c_void_p] * 5 + [C.c_void_p, i64, C.c_void_p, C.c_void_p]
        L.or_residual_jvp_complex_step.argtypes = L.or_residual_jvp.argtypes
        L.or_element_matrix.argtypes = [vp, C.c_void_p] + [C.c_void_p] * 4 + [i64, C.c_void_p]
        L.or_element_matrix.restype = i32
        L.or_element_residual.argtypes = [vp, C.c_void_p] + [C.c_void_p] * 4 + [i64, C.c_void_p]
        L.or_element_residual.restype = i32
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


def set_threads(n: int) -> None:
    """Threads of the oracle's element loop in residual / J v (default 1); each thread scatters into
    its own vectors, added in thread order afterwards."""
    lib().or_set_threads(int(n))


def set_bt_pad(pad: float) -> None:
    """Widening of the background-triangle boxes as a fraction of the element edge (default 1e-2);
    applies to meshes built afterwards.  A test knob: 0 restores the plain closed-box overlap."""
    lib().or_set_bt_pad(float(pad))


class OracleMesh:
    """Octree mesh + immersed surface, evaluated by the oracle."""

    def __init__(self, lo, hi, base_level, regions, triangles=None, lmax=3):
        L = lib()
        n = len(regions)
        kind = np.array([r.kind for r in regions] or [0], dtype=np.int32)
        level = np.array([r.level for r in regions] or [0], dtype=np.int32)
        par = np.array([r.packed() for r in regions] or [[0.0] * 8], dtype=np.float64)
        err = C.create_string_buffer(256)
        lo_ = (C.c_double * 3)(*lo)
        hi_ = (C.c_double * 3)(*hi)
        self._keep = (kind, level, par)
        h = L.or_build(lo_, hi_, base_level, n, _p(kind), _p(level), _p(par), err, 256)
        if not h:
            raise ValueError("oracle mesh: " + err.value.decode())
        self.h = h
        sz = np.zeros(6, dtype=np.int64)
        sc = np.zeros(1)
        L.or_sizes(h, _p(sz), _p(sc))
        self.n_elem, self.n_nodes, self.n_hang = int(sz[0]), int(sz[1]), int(sz[2])
        self.hiI = sz[3:6].copy()
        self.scale = float(sc[0])
        self.lo = np.array(lo, dtype=np.float64)
        self.anchors = np.zeros((self.n_elem, 3), np.uint32)
        self.levels = np.zeros(self.n_elem, np.uint8)
        self.conn = np.zeros((self.n_elem, 8), np.int32)
        self.node_ijk = np.zeros((self.n_nodes, 3), np.uint32)
        self.hang_parents = np.zeros((max(self.n_hang, 1), 4), np.int32)
        self.hang_np = np.zeros(max(self.n_hang, 1), np.int8)
        self.hang_ijk = np.zeros((max(self.n_hang, 1), 3), np.uint32)
        L.or_export(h, _p(self.anchors), _p(self.levels), _p(self.conn), _p(self.node_ijk), _p(self.hang_parents),
                    _p(self.hang_np), _p(self.hang_ijk))
        self.hang_parents = self.hang_parents[: self.n_hang]
        self.hang_np = self.hang_np[: self.n_hang]
        self.hang_ijk = self.hang_ijk[: self.n_hang]
        self.node_xyz = self.lo + self.node_ijk.astype(np.float64) * self.scale
        self.n_tri = 0
        self.set_surface(np.zeros((0, 3, 3)) if triangles is None else triangles, lmax)

    def __del__(self):
        try:
            if getattr(self, "h", None):
                lib().or_free(self.h)
                self.h = None
        except Exception:
            pass

    def set_surface(self, triangles, lmax=3):
        t = np.ascontiguousarray(triangles, dtype=np.float64).reshape(-1, 9)
        if t.shape[0] == 0:
            t = np.zeros((1, 9))[:0]
        self._tri = t
        self.n_tri = t.shape[0]
        lib().or_set_surface(self.h, _p(t) if t.shape[0] else None, t.shape[0], lmax)

    def find_leaf(self, ijk):
        return lib().or_find_leaf(self.h, int(ijk[0]), int(ijk[1]), int(ijk[2]))

    def classify(self, pts):
        pts = _f64(pts).reshape(-1, 3)
        out = np.zeros(pts.shape[0], np.uint8)
        lib().or_classify(self.h, _p(pts), pts.shape[0], _p(out))
        return out

    def markers(self, elems=None):
        if elems is None:
            n = self.n_elem
            ep = None
        else:
            elems = np.ascontiguousarray(elems, dtype=np.int64)
            n = elems.size
            ep = elems
        mk = np.zeros(n, np.int8)
        cf = np.zeros(n, np.uint8)
        nbt = np.zeros(n, np.int32)
        lib().or_markers(self.h, _p(ep), n, _p(mk), _p(cf), _p(nbt))
        return mk, cf, nbt

    def background_triangles(self, e):
        cap = self.n_tri
        out = np.zeros(max(cap, 1), np.int32)
        n = lib().or_bt(self.h, int(e), _p(out), cap)
        return out[:n]

    def cut_points(self, e):
        cap = 8 ** 5
        out = np.zeros((cap, 4))
        n = lib().or_cut_points(self.h, int(e), _p(out), cap)
        return out[:n].copy()

    def surface_points(self):
        cap = 3 * max(self.n_tri, 1)
        out = np.zeros((cap, 10))
        n = lib().or_surface_points(self.h, _p(out), cap)
        return out[:n].copy()

    def counters(self):
        out = np.zeros(4, np.int64)
        lib().or_counters(self.h, _p(out))
        return {"rays": int(out[0]), "normal_tests": int(out[1]), "normal_decided": int(out[2]),
                "elements_evaluated": int(out[3])}

    def set_dirichlet(self, mask, vals):
        mask = np.ascontiguousarray(mask, dtype=np.uint8)
        vals = _f64(vals).reshape(-1, 4)
        self._bc = (mask, vals)
        lib().or_set_dirichlet(self.h, _p(mask), _p(vals))

    def set_surface_velocity(self, g=None):
        """Velocity g of Eq. (weakbc) at every surface point, [n_surface_points, 3] in the order of
        surface_points(); None returns to the uniform body velocity of the physics."""
        if g is None:
            lib().or_set_surface_velocity(self.h, None, 0)
            self._g = None
            return
        g = _f64(g).reshape(-1, 3)
        self._g = g
        if lib().or_set_surface_velocity(self.h, _p(g), g.shape[0]) != 0:
            raise ValueError("one velocity per surface point is needed")

    def residual_jvp(self, phys, u, u_prev, u_prev2=None, f=None, v=None, nodes=None):
        """Returns (R, Jv) as [n_nodes, 4]; with `nodes`, only those rows are meaningful."""
        ph = np.array(phys.packed(), dtype=np.float64)
        u, up, up2, f, v = _f64(u), _f64(u_prev), _f64(u_prev2), _f64(f), _f64(v)
        if f is not None:
            f4 = np.zeros((self.n_nodes, 4))
            f4[:, :3] = f.reshape(self.n_nodes, -1)[:, :3]
            f = f4
        sel = None if nodes is None else np.ascontiguousarray(nodes, dtype=np.int64)
        R = np.zeros((self.n_nodes, 4))
        J = np.zeros((self.n_nodes, 4))
        lib().or_residual_jvp(self.h, _p(ph), _p(u), _p(up), _p(up2), _p(f), _p(v), _p(sel),
                              0 if sel is None else sel.size, _p(R), _p(J))
        return R, J

    def wpart_weights(self, ts_over_tv):
        """Eq. (Wpart), the cost of element e relative to an Out element:
        W(e) = n_Vgp(e) / n_Tgp + (T_s / T_v) n_Sgp(e) / n_Tgp, with n_Tgp = 8 for trilinear
        hexahedra.  n_Vgp is the number of volume Gauss points evaluated (8 for Out elements, the
        kept sub-cell points for Intercepted ones, none for In ones) and n_Sgp the number of its
        surface points."""
        mk, _, _ = self.markers()
        W = np.zeros(self.n_elem)
        W[mk == 0] = 1.0
        for e in np.where(mk == 2)[0]:
            W[e] = self.cut_points(int(e)).shape[0] / 8.0
        sq = self.surface_points()
        if sq.shape[0]:
            ns = np.bincount(sq[:, 8].astype(np.int64), minlength=self.n_elem)
            W += ts_over_tv * ns / 8.0
        return W

    def surface_force(self, phys, u, u_prev):
        """Force of the fluid on the body from the weak-boundary terms (float64 [3])."""
        ph = np.array(phys.packed(), dtype=np.float64)
        F = np.zeros(3)
        lib().or_surface_force(self.h, _p(ph), _p(_f64(u)), _p(_f64(u_prev)), _p(F))
        return F

    def jvp_complex_step(self, phys, u, u_prev, v, u_prev2=None, f=None):
        """J v as Im R(u + i eps v) / eps (eps = 1e-30): the complex step, independent of the dual numbers."""
        ph = np.array(phys.packed(), dtype=np.float64)
        u, up, up2, f, v = _f64(u), _f64(u_prev), _f64(u_prev2), _f64(f), _f64(v)
        if f is not None:
            f4 = np.zeros((self.n_nodes, 4))
            f4[:, :3] = f.reshape(self.n_nodes, -1)[:, :3]
            f = f4
        J = np.zeros((self.n_nodes, 4))
        lib().or_residual_jvp_complex_step(self.h, _p(ph), _p(u), _p(up), _p(up2), _p(f), _p(v), None, 0, None, _p(J))
        return J

    def residual(self, phys, u, u_prev, u_prev2=None, f=None, nodes=None):
        return self.residual_jvp(phys, u, u_prev, u_prev2, f, None, nodes)[0]

    def jvp(self, phys, u, u_prev, v, u_prev2=None, f=None, nodes=None):
        return self.residual_jvp(phys, u, u_prev, u_prev2, f, v, nodes)[1]

    def element_matrix(self, phys, u, u_prev, e, u_prev2=None, f=None):
        ph = np.array(phys.packed(), dtype=np.float64)
        K = np.zeros((32, 32))
        u, up, up2 = _f64(u), _f64(u_prev), _f64(u_prev2)
        if f is not None:
            f4 = np.zeros((self.n_nodes, 4))
            f4[:, :3] = _f64(f).reshape(self.n_nodes, -1)[:, :3]
            f = f4
        mk = lib().or_element_matrix(self.h, _p(ph), _p(u), _p(up), _p(up2), _p(f), int(e), _p(K))
        return K, mk

    def element_residual(self, phys, u, u_prev, e, u_prev2=None, f=None):
        ph = np.array(phys.packed(), dtype=np.float64)
        r = np.zeros(32)
        u, up, up2 = _f64(u), _f64(u_prev), _f64(u_prev2)
        if f is not None:
            f4 = np.zeros((self.n_nodes, 4))
            f4[:, :3] = _f64(f).reshape(self.n_nodes, -1)[:, :3]
            f = f4
        lib().or_element_residual(self.h, _p(ph), _p(u), _p(up), _p(up2), _p(f), int(e), _p(r))
        return r.reshape(8, 4)

    # M_e: element corner values from global node values (hanging interpolation)
    def gather_matrix(self, e):
        M = np.zeros((8, self.n_nodes))
        for c in range(8):
            idx = self.conn[e, c]
            if idx < self.n_nodes:
                M[c, idx] = 1.0
            else:
                h = idx - self.n_nodes
                for p in range(self.hang_np[h]):
                    M[c, self.hang_parents[h, p]] = 1.0 / self.hang_np[h]
        return M
