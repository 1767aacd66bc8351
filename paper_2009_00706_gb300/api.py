"""Thin Python binding of the imga C ABI (same names, argument marshalling only).

Device vectors are torch CUDA tensors (float64, [n_nodes, 4], contiguous); the stream is
torch's current stream unless one is given.  Every step of the computation runs in the
library's CUDA kernels; this module only converts arguments.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import MeshInfo, MeshParams, Physics, Problem, Region, SolverOpts, SolverStats, check

PRECISION_FP64, PRECISION_MIXED = 0, 1


def physics_struct(ph, g_points=None) -> Physics:
    """imga_physics from an inputs.Physics (or anything with the same fields); g_points: the
    velocity per surface point, a float64 CUDA tensor [n_surface_points, 3] in the order of
    Mesh.surface_points(), or None (g_body everywhere)."""
    s = Physics()
    s.rho, s.mu, s.dt, s.time_scheme = ph.rho, ph.mu, ph.dt, int(ph.scheme)
    s.C_b, s.C_I = ph.Cb, ph.CI
    s.g_body = (C.c_double * 3)(*ph.g)
    s.u_inf = (C.c_double * 3)(*ph.uinf)
    s.drop_visc_strong = int(ph.drop_visc)
    if g_points is not None:
        if not (g_points.is_cuda and str(g_points.dtype).endswith("float64") and g_points.is_contiguous()):
            raise ValueError("g_points: expected a contiguous float64 CUDA tensor [n_surface_points, 3]")
    s.g_points = None if g_points is None else g_points.data_ptr()
    return s


def _ptr(t):
    if t is None:
        return None
    return C.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        import torch
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return C.c_void_p(stream)
    return C.c_void_p(stream.cuda_stream)


def _vec(t, n_nodes, name):
    if t is None:
        return None
    if not (t.is_cuda and t.dtype.__repr__().endswith("float64") and t.is_contiguous() and t.numel() == 4 * n_nodes):
        raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor of {n_nodes} x 4")
    return t


class Mesh:
    """imga_build_mesh / imga_destroy_mesh and the calls that take the mesh handle."""

    def __init__(self, lo=None, hi=None, base_level=None, regions=None, triangles=None, lmax=3, device=0, _handle=None):
        L = _lib.load()
        if _handle is not None:
            self._adopt(_handle, device)
            return
        tri = np.ascontiguousarray(np.zeros((0, 3, 3)) if triangles is None else triangles, dtype=np.float64)
        regs = (Region * max(1, len(regions)))()
        for i, r in enumerate(regions):
            regs[i].kind, regs[i].level = r.kind, r.level
            regs[i].par = (C.c_double * 8)(*r.packed())
        P = MeshParams()
        P.lo = (C.c_double * 3)(*lo)
        P.hi = (C.c_double * 3)(*hi)
        P.base_level = base_level
        P.n_regions = len(regions)
        P.regions = C.cast(regs, C.POINTER(Region))
        P.quad_max_split = lmax
        h = C.c_void_p()
        n_tri = tri.shape[0]
        check(L.imga_build_mesh(tri.ctypes.data_as(C.c_void_p) if n_tri else None, n_tri, C.byref(P), device,
                                C.byref(h)))
        self._adopt(h, device)
        self.lo = np.array(lo, dtype=np.float64)

    def _adopt(self, h, device):
        L = _lib.load()
        self.h = h
        self.device = device
        info = MeshInfo()
        check(L.imga_mesh_get_info(h, C.byref(info)))
        self.info = {k: (list(getattr(info, k)) if k in ("hi_int", "setup_ms") else getattr(info, k))
                     for k, _ in MeshInfo._fields_}
        self.n_elem = info.n_elem
        self.n_nodes = info.n_nodes
        self.n_hang = info.n_hanging
        self.scale = info.scale
        np_ = C.c_int()
        L.imga_mesh_problems(h, C.byref(np_), None, None)
        self.n_problems = np_.value
        eo = np.zeros(self.n_problems + 1, np.int64)
        no = np.zeros(self.n_problems + 1, np.int64)
        L.imga_mesh_problems(h, C.byref(np_), eo.ctypes.data_as(C.c_void_p), no.ctypes.data_as(C.c_void_p))
        self.elem_off, self.node_off = eo, no

    @classmethod
    def batch(cls, workloads, mus=None, device=0):
        """imga_build_mesh_batch over a list of inputs.Workload (viscosity: each workload's physics.mu)."""
        L = _lib.load()
        n = len(workloads)
        probs = (Problem * n)()
        keep = []
        for i, w in enumerate(workloads):
            tri = np.ascontiguousarray(w.triangles(), dtype=np.float64)
            regs = (Region * max(1, len(w.regions)))()
            for j, r in enumerate(w.regions):
                regs[j].kind, regs[j].level = r.kind, r.level
                regs[j].par = (C.c_double * 8)(*r.packed())
            keep += [tri, regs]
            probs[i].tri_xyz_host = tri.ctypes.data_as(C.c_void_p) if tri.shape[0] else None
            probs[i].n_tri = tri.shape[0]
            P = probs[i].params
            P.lo = (C.c_double * 3)(*w.lo)
            P.hi = (C.c_double * 3)(*w.hi)
            P.base_level = w.base_level
            P.n_regions = len(w.regions)
            P.regions = C.cast(regs, C.POINTER(Region))
            P.quad_max_split = w.lmax
            probs[i].mu = w.physics.mu if mus is None else mus[i]
        h = C.c_void_p()
        check(L.imga_build_mesh_batch(probs, n, device, C.byref(h)))
        return cls(_handle=h, device=device)

    @classmethod
    def from_workload(cls, w, device=0, triangles=None):
        return cls(w.lo, w.hi, w.base_level, w.regions, w.triangles() if triangles is None else triangles, w.lmax,
                   device)

    def close(self):
        if getattr(self, "h", None):
            _lib.load().imga_destroy_mesh(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ---- host exports ------------------------------------------------------------------
    def export(self):
        L = _lib.load()
        ne, nn, nh = self.n_elem, self.n_nodes, self.n_hang
        anc = np.zeros((ne, 3), np.uint32)
        lev = np.zeros(ne, np.uint8)
        conn = np.zeros((ne, 8), np.int32)
        ijk = np.zeros((nn, 3), np.uint32)
        hp = np.zeros((max(nh, 1), 4), np.int32)
        hn = np.zeros(max(nh, 1), np.int8)
        f = lambda a: a.ctypes.data_as(C.c_void_p)
        check(L.imga_mesh_export(self.h, f(anc), f(lev), f(conn), f(ijk), f(hp), f(hn)))
        return {"anchors": anc, "levels": lev, "conn": conn, "node_ijk": ijk, "hang_parents": hp[:nh], "hang_np": hn[:nh]}

    def _gp(self, g_points):
        if g_points is not None and g_points.numel() != 3 * self.info["n_surface_points"]:
            raise ValueError(f"g_points: expected {self.info['n_surface_points']} x 3 values")
        return g_points

    def markers(self):
        mk = np.zeros(self.n_elem, np.int8)
        cf = np.zeros(self.n_elem, np.uint8)
        check(_lib.load().imga_export_markers(self.h, mk.ctypes.data_as(C.c_void_p), cf.ctypes.data_as(C.c_void_p)))
        return mk, cf

    def cut_points(self):
        off = np.zeros(self.n_elem + 1, np.int64)
        pts = np.zeros((max(1, self.info["n_cut_points"]), 4))
        check(_lib.load().imga_export_cut_points(self.h, off.ctypes.data_as(C.c_void_p), pts.ctypes.data_as(C.c_void_p)))
        return off, pts[: self.info["n_cut_points"]]

    def background(self):
        off = np.zeros(self.n_elem + 1, np.int32)
        ids = np.zeros(max(1, self.info["n_bt"]), np.int32)
        check(_lib.load().imga_export_background(self.h, off.ctypes.data_as(C.c_void_p), ids.ctypes.data_as(C.c_void_p)))
        return off, ids[: self.info["n_bt"]]

    def surface_points(self):
        n = self.info["n_surface_points"]
        out = np.zeros((max(1, n), 10))
        if n:
            check(_lib.load().imga_export_surface_points(self.h, out.ctypes.data_as(C.c_void_p)))
        return out[:n]

    # ---- device calls --------------------------------------------------------------------
    def classify(self, pts, flags=None, stream=None):
        import torch
        n = pts.shape[0]
        if flags is None:
            flags = torch.empty(n, dtype=torch.uint8, device=pts.device)
        check(_lib.load().imga_classify(self.h, _ptr(pts), n, _ptr(flags), _stream(stream)))
        return flags

    def residual(self, phys, u, u_prev, u_prev2=None, f=None, precision=PRECISION_FP64, out=None, stream=None,
                 g_points=None):
        import torch
        nn = self.n_nodes
        if out is None:
            out = torch.empty((nn, 4), dtype=torch.float64, device=u.device)
        ps = physics_struct(phys, self._gp(g_points))
        check(_lib.load().imga_residual(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                        _ptr(_vec(u_prev2, nn, "u_prev2")), _ptr(_vec(f, nn, "f")), C.byref(ps),
                                        precision, _ptr(out), _stream(stream)))
        return out

    def jvp(self, phys, u, u_prev, v, u_prev2=None, f=None, precision=PRECISION_FP64, out=None, stream=None,
            g_points=None):
        import torch
        nn = self.n_nodes
        if out is None:
            out = torch.empty((nn, 4), dtype=torch.float64, device=u.device)
        ps = physics_struct(phys, self._gp(g_points))
        check(_lib.load().imga_jvp(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                   _ptr(_vec(u_prev2, nn, "u_prev2")), _ptr(_vec(f, nn, "f")), C.byref(ps), precision,
                                   _ptr(_vec(v, nn, "v")), _ptr(out), _stream(stream)))
        return out

    def element_jacobians(self, phys, u, u_prev, elems, u_prev2=None, f=None, precision=PRECISION_FP64, out=None,
                          stream=None, g_points=None):
        """k_e [n, 32, 32] (float64, device) of the elements in `elems` (int32 device tensor)."""
        import torch
        nn = self.n_nodes
        n = elems.numel()
        if out is None:
            out = torch.empty((n, 32, 32), dtype=torch.float64, device=u.device)
        ps = physics_struct(phys, self._gp(g_points))
        check(_lib.load().imga_element_jacobians(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                                 _ptr(_vec(u_prev2, nn, "u_prev2")), _ptr(_vec(f, nn, "f")),
                                                 C.byref(ps), precision, _ptr(elems), n, _ptr(out), _stream(stream)))
        return out

    def newton_step(self, phys, u, u_prev, u_prev2=None, f=None, gmres_m=50, max_newton=20, max_krylov=1000,
                    rtol=1e-8, atol=0.0, krylov_rtol=1e-3, precision=PRECISION_FP64, precond=1, line_search=1,
                    stream=None, raise_on_failure=True, learned=None, learned_omega=0.5, g_points=None,
                    linear_solver=0, ml_agg=0, ml_coarse_max=0, ml_sweeps=0, ml_omega=0.0):
        """Newton-GMRES (linear_solver 0) or Newton-BiCGStab on the assembled Jacobian (1) in place on u;
        returns a stats dict.  precond 2 needs learned = an Mlp; precond 4 is the multilevel V-cycle."""
        nn = self.n_nodes
        o = SolverOpts(gmres_m, max_newton, max_krylov, rtol, atol, krylov_rtol, precision, precond, line_search,
                       learned.h if learned is not None else None, learned_omega, linear_solver, ml_agg,
                       ml_coarse_max, ml_sweeps, ml_omega)
        st = SolverStats()
        ps = physics_struct(phys, self._gp(g_points))
        status = _lib.load().imga_newton_step(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                              _ptr(_vec(u_prev2, nn, "u_prev2")), _ptr(_vec(f, nn, "f")),
                                              C.byref(ps), C.byref(o), C.byref(st), _stream(stream))
        out = {"status": status, "newton_its": st.newton_its, "krylov_its": st.krylov_its,
               "krylov_per_newton": list(st.krylov_per_newton)[: st.newton_its],
               "res_norm": list(st.res_norm)[: st.newton_its + 1], "time_ms": st.time_ms, "converged": st.converged,
               "fallbacks": st.fallbacks, "krylov_rel": list(st.krylov_rel)[: st.newton_its]}
        if raise_on_failure and status != 0:
            check(status)
        return out

    def bsr_assemble(self, phys, u, u_prev, u_prev2=None, f=None, precision=PRECISION_FP64, out=None, stream=None,
                     g_points=None):
        """The assembled Jacobian: float64 CUDA tensor [n_blocks, 4, 4] on the pattern of bsr_pattern()."""
        import torch
        nn = self.n_nodes
        nb = self.bsr_pattern()[1].size
        if out is None:
            out = torch.empty((nb, 4, 4), dtype=torch.float64, device=u.device)
        ps = physics_struct(phys, self._gp(g_points))
        check(_lib.load().imga_bsr_assemble(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                            _ptr(_vec(u_prev2, nn, "u_prev2")), _ptr(_vec(f, nn, "f")), C.byref(ps),
                                            precision, _ptr(out), _stream(stream)))
        return out

    def bsr_spmv(self, vals, x, out=None, stream=None):
        import torch
        nn = self.n_nodes
        if out is None:
            out = torch.empty((nn, 4), dtype=torch.float64, device=x.device)
        check(_lib.load().imga_bsr_spmv(self.h, _ptr(vals), _ptr(_vec(x, nn, "x")), _ptr(out), _stream(stream)))
        return out

    def time_steps(self, phys, u, u_prev, n_steps, f=None, gmres_m=50, max_newton=20, max_krylov=1000, rtol=1e-8,
                   atol=0.0, krylov_rtol=1e-3, precision=PRECISION_FP64, precond=4, line_search=1, stream=None,
                   g_points=None, linear_solver=0, raise_on_failure=True):
        """imga_time_steps: n_steps Newton-solved time steps in place on (u, u_prev); returns the force
        history [n_steps, 3] (host) and the Newton and Krylov iterations per step."""
        nn = self.n_nodes
        o = SolverOpts(gmres_m, max_newton, max_krylov, rtol, atol, krylov_rtol, precision, precond, line_search,
                       None, 0.5, linear_solver, 0, 0, 0, 0.0)
        ps = physics_struct(phys, self._gp(g_points))
        F = np.zeros((max(1, n_steps), 3))
        nh = np.zeros(max(1, n_steps), np.int32)
        kh = np.zeros(max(1, n_steps), np.int32)
        status = _lib.load().imga_time_steps(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                             _ptr(_vec(f, nn, "f")), C.byref(ps), C.byref(o), n_steps,
                                             F.ctypes.data_as(C.c_void_p), nh.ctypes.data_as(C.c_void_p),
                                             kh.ctypes.data_as(C.c_void_p), _stream(stream))
        if raise_on_failure and status != 0:
            check(status)
        return {"status": status, "force": F[:n_steps], "newton_its": nh[:n_steps], "krylov_its": kh[:n_steps]}

    def surface_force(self, phys, u, u_prev, out=None, stream=None, g_points=None):
        """Force of the fluid on the body (float64 CUDA tensor [3])."""
        import torch
        nn = self.n_nodes
        if out is None:
            out = torch.empty(3, dtype=torch.float64, device=u.device)
        ps = physics_struct(phys, self._gp(g_points))
        check(_lib.load().imga_surface_force(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                             C.byref(ps), _ptr(out), _stream(stream)))
        return out

    def multilevel_setup(self, phys, u, u_prev, u_prev2=None, f=None, precision=PRECISION_FP64, agg=6, coarse_max=16,
                         sweeps=1, omega=0.5, stream=None, g_points=None):
        nn = self.n_nodes
        ps = physics_struct(phys, self._gp(g_points))
        check(_lib.load().imga_multilevel_setup(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                                _ptr(_vec(u_prev2, nn, "u_prev2")), _ptr(_vec(f, nn, "f")),
                                                C.byref(ps), precision, agg, coarse_max, sweeps, omega, _stream(stream)))

    def multilevel_apply(self, r, out=None, stream=None):
        import torch
        nn = self.n_nodes
        if out is None:
            out = torch.empty((nn, 4), dtype=torch.float64, device=r.device)
        check(_lib.load().imga_multilevel_apply(self.h, _ptr(_vec(r, nn, "r")), _ptr(out), _stream(stream)))
        return out

    def multilevel_info(self):
        """(block rows per level, whether the dense last level met a singular pivot)"""
        n = C.c_int(0)
        rows = np.zeros(24, np.int64)
        sing = C.c_int(0)
        check(_lib.load().imga_multilevel_info(self.h, C.byref(n), rows.ctypes.data_as(C.c_void_p), C.byref(sing)))
        return rows[: n.value].copy(), bool(sing.value)

    def precond_dataset(self, phys, u, u_prev, elems, u_prev2=None, f=None, precision=PRECISION_MIXED, targets=True,
                        ldx=1040, stream=None):
        """(X [n, ldx], T [n, 1024] or None, scale [n]) float32 device tensors of the listed elements."""
        import torch
        n = elems.numel()
        X = torch.empty((n, ldx), dtype=torch.float32, device=u.device)
        T = torch.empty((n, 1024), dtype=torch.float32, device=u.device) if targets else None
        sc = torch.empty(n, dtype=torch.float32, device=u.device)
        ps = physics_struct(phys)
        nn = self.n_nodes
        check(_lib.load().imga_precond_dataset(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                               _ptr(_vec(u_prev2, nn, "u_prev2")), _ptr(_vec(f, nn, "f")), C.byref(ps),
                                               precision, _ptr(elems), n, ldx, _ptr(X), _ptr(T), _ptr(sc),
                                               _stream(stream)))
        return X, T, sc

    def profile(self, enable=True):
        check(_lib.load().imga_profile(self.h, 1 if enable else 0))

    def deterministic(self, on=True):
        """IMGA_OPT_DETERMINISTIC: slot writes + ordered node sums (on, default) or float64 atomics."""
        check(_lib.load().imga_set_option(self.h, 4, 1 if on else 0))

    def use_graphs(self, on=True):
        """imga_set_option(IMGA_OPT_GRAPHS): replay residual / J v calls as CUDA graphs."""
        check(_lib.load().imga_set_option(self.h, 1, 1 if on else 0))

    def autotune(self, on=True):
        """imga_set_option(IMGA_OPT_AUTOTUNE): tune the Intercepted-element tile shape on the next call
        of each precision and kind."""
        check(_lib.load().imga_set_option(self.h, 2, 1 if on else 0))

    def node_coords(self, out=None, stream=None):
        """float64 [n_nodes, 3] node coordinates: a tensor on the mesh's device (or `out`), or a
        numpy array for a host-only mesh."""
        if self.device < 0:
            xyz = np.zeros((self.n_nodes, 3))
            check(_lib.load().imga_node_coords(self.h, xyz.ctypes.data_as(C.c_void_p), None))
            return xyz
        import torch
        if out is None:
            out = torch.empty((self.n_nodes, 3), dtype=torch.float64, device=torch.device("cuda", self.device))
        check(_lib.load().imga_node_coords(self.h, _ptr(out), _stream(stream)))
        return out

    def bsr_pattern(self):
        """(indptr int64 [n_nodes + 1], indices int32 [n_blocks]) of the Jacobian's 4 x 4 block
        pattern (host arrays)."""
        L = _lib.load()
        nb = C.c_int64()
        check(L.imga_bsr_pattern(self.h, C.byref(nb), None, None))
        indptr = np.zeros(self.n_nodes + 1, np.int64)
        indices = np.zeros(max(1, nb.value), np.int32)
        check(L.imga_bsr_pattern(self.h, C.byref(nb), indptr.ctypes.data_as(C.c_void_p),
                                 indices.ctypes.data_as(C.c_void_p)))
        return indptr, indices[:nb.value]

    def classify_rays_only(self, on=True):
        """imga_set_option(IMGA_OPT_CLASSIFY_RAYS): classify every point by ray parity."""
        check(_lib.load().imga_set_option(self.h, 3, 1 if on else 0))

    def classify_counts(self, reset=False):
        """How imga_classify settled its points since the last reset (synchronises):
        {'marker', 'normal_tests', 'normal_decided', 'rays'}."""
        c = np.zeros(4, np.int64)
        check(_lib.load().imga_classify_counts(self.h, c.ctypes.data_as(C.c_void_p), 1 if reset else 0))
        return {"marker": int(c[0]), "normal_tests": int(c[1]), "normal_decided": int(c[2]), "rays": int(c[3])}

    def tuning(self):
        """{(precision, 'residual' | 'jvp'): (warps per block, longest first, candidate ms[6])}."""
        shape = np.zeros(8, np.int32)
        ms = np.zeros(24, np.float32)
        check(_lib.load().imga_tuning(self.h, shape.ctypes.data_as(C.c_void_p), ms.ctypes.data_as(C.c_void_p)))
        out = {}
        for p in range(2):
            for j, kind in enumerate(("residual", "jvp")):
                out[(p, kind)] = (int(shape[4 * p + 2 * j]), int(shape[4 * p + 2 * j + 1]), ms[12 * p + 6 * j:12 * p + 6 * j + 6].tolist())
        return out

    def fused(self, on=True):
        """IMGA_OPT_FUSED: the Out and Intercepted buckets in one persistent launch (surface kernels beside it)."""
        check(_lib.load().imga_set_option(self.h, 5, int(bool(on))))

    def concurrent(self, on=True):
        """IMGA_OPT_CONCURRENT: Intercepted / surface kernels on side streams beside the Out kernel."""
        check(_lib.load().imga_set_option(self.h, 7, 1 if on else 0))

    def fused_split(self, heavy_warps):
        """IMGA_OPT_FUSED_SPLIT: warps per block (1 .. 4) that start on the Intercepted elements."""
        check(_lib.load().imga_set_option(self.h, 6, int(heavy_warps)))

    def fused_info(self):
        c = np.zeros(6, np.int64)
        check(_lib.load().imga_fused_info(self.h, c.ctypes.data_as(C.c_void_p)))
        return {"on": bool(c[0]), "cut_items": int(c[1]), "dense_surface_elements": int(c[2]),
                "sparse_surface_points": int(c[3]), "out_elements": int(c[4]), "heavy_first_warps": int(c[5])}

    def tuning_interior(self):
        """{(precision, 'residual' | 'jvp'): (blocks per SM in use (0: occupancy limit), candidate ms[5])}"""
        bps = np.zeros(4, np.int32)
        ms = np.zeros(20, np.float32)
        check(_lib.load().imga_tuning_interior(self.h, bps.ctypes.data_as(C.c_void_p), ms.ctypes.data_as(C.c_void_p)))
        return {(p, kind): (int(bps[2 * p + j]), ms[10 * p + 5 * j:10 * p + 5 * j + 5].tolist())
                for p in range(2) for j, kind in enumerate(("residual", "jvp"))}

    def profile_read(self):
        """{kernel: (total ms, launches)} since profiling was enabled (synchronises)."""
        ms = np.zeros(6)
        n = np.zeros(6, np.int64)
        check(_lib.load().imga_profile_read(self.h, ms.ctypes.data_as(C.c_void_p), n.ctypes.data_as(C.c_void_p)))
        names = ("out_elements", "cut_elements", "nitsche", "strong_rows", "node_prep", "fused")
        return {k: (float(ms[i]), int(n[i])) for i, k in enumerate(names)}

    def set_dirichlet(self, mask=None, vals=None, stream=None):
        check(_lib.load().imga_set_dirichlet(self.h, _ptr(mask), _ptr(vals), _stream(stream)))


class Mlp:
    """imga_mlp: the learned block preconditioner's network (3 layers, BF16 tensor cores)."""

    def __init__(self, n_in=1027, width=128, n_out=1024, seed=0, device=0):
        h = C.c_void_p()
        check(_lib.load().imga_mlp_create(n_in, width, n_out, seed, device, C.byref(h)))
        self.h = h
        npar, pad = C.c_int64(), C.c_int()
        check(_lib.load().imga_mlp_shape(h, C.byref(npar), C.byref(pad)))
        self.n_params, self.n_in_pad = npar.value, pad.value
        self.n_in, self.width, self.n_out = n_in, width, n_out

    def close(self):
        if getattr(self, "h", None):
            _lib.load().imga_mlp_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def params(self):
        out = np.zeros(self.n_params, np.float32)
        check(_lib.load().imga_mlp_params(self.h, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        check(_lib.load().imga_mlp_params(self.h, p.ctypes.data_as(C.c_void_p), 1))

    def unpack(self, p):
        """(W1 [w, n_in], b1, W2, b2, W3, b3) float64 views of a flat parameter vector."""
        w, pad, nin, no = self.width, self.n_in_pad, self.n_in, self.n_out
        o = 0
        W1 = p[o:o + w * pad].reshape(w, pad)[:, :nin].astype(np.float64); o += w * pad
        b1 = p[o:o + w].astype(np.float64); o += w
        W2 = p[o:o + w * w].reshape(w, w).astype(np.float64); o += w * w
        b2 = p[o:o + w].astype(np.float64); o += w
        W3 = p[o:o + no * w].reshape(no, w).astype(np.float64); o += no * w
        b3 = p[o:o + no].astype(np.float64)
        return [W1, b1, W2, b2, W3, b3]

    def forward(self, X, stream=None):
        import torch
        n = X.shape[0]
        Y = torch.empty((n, self.n_out), dtype=torch.float32, device=X.device)
        check(_lib.load().imga_mlp_forward(self.h, _ptr(X), X.shape[1], n, _ptr(Y), _stream(stream)))
        return Y

    def gradient(self, X, T, stream=None):
        g = np.zeros(self.n_params, np.float32)
        loss = C.c_double()
        check(_lib.load().imga_mlp_gradient(self.h, _ptr(X), X.shape[1], _ptr(T), X.shape[0], C.byref(loss),
                                            g.ctypes.data_as(C.c_void_p), _stream(stream)))
        return loss.value, g

    def train(self, X, T, epochs=10, batch=1024, lr=1e-3, stream=None):
        hist = np.zeros(max(1, epochs))
        check(_lib.load().imga_mlp_train(self.h, _ptr(X), X.shape[1], _ptr(T), X.shape[0], epochs, batch, lr,
                                         hist.ctypes.data_as(C.c_void_p), _stream(stream)))
        return hist[:epochs]


class Partition:
    """imga_partition_*: the mesh split into k weighted Morton ranges with halo exchange."""

    def __init__(self, mesh, k, ts_over_tv=0.0):
        self.mesh = mesh
        h = C.c_void_p()
        check(_lib.load().imga_partition_build(mesh.h, k, ts_over_tv, C.byref(h)))
        self.h = h
        kk = C.c_int(0)
        self.elem_off = np.zeros(k + 1, np.int64)
        self.weight = np.zeros(k)
        self.n_owned = np.zeros(k, np.int64)
        self.n_ghost = np.zeros(k, np.int64)
        f = lambda a: a.ctypes.data_as(C.c_void_p)
        check(_lib.load().imga_partition_info(h, C.byref(kk), f(self.elem_off), f(self.weight), f(self.n_owned),
                                              f(self.n_ghost)))
        self.k = kk.value

    def nodes(self, p):
        """(global nodes of part p, owned first; owning part of every ghost)"""
        n = np.zeros(max(1, int(self.n_owned[p] + self.n_ghost[p])), np.int64)
        o = np.zeros(max(1, int(self.n_ghost[p])), np.int32)
        check(_lib.load().imga_partition_nodes(self.h, p, n.ctypes.data_as(C.c_void_p), o.ctypes.data_as(C.c_void_p)))
        return n[: self.n_owned[p] + self.n_ghost[p]], o[: self.n_ghost[p]]

    def residual(self, phys, u, u_prev, u_prev2=None, f=None, precision=PRECISION_FP64, out=None, stream=None):
        import torch
        nn = self.mesh.n_nodes
        if out is None:
            out = torch.empty((nn, 4), dtype=torch.float64, device=u.device)
        ps = physics_struct(phys)
        check(_lib.load().imga_partition_residual(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                                  _ptr(_vec(u_prev2, nn, "u_prev2")), _ptr(_vec(f, nn, "f")),
                                                  C.byref(ps), precision, _ptr(out), _stream(stream)))
        return out

    def jvp(self, phys, u, u_prev, v, u_prev2=None, f=None, precision=PRECISION_FP64, out=None, stream=None):
        import torch
        nn = self.mesh.n_nodes
        if out is None:
            out = torch.empty((nn, 4), dtype=torch.float64, device=u.device)
        ps = physics_struct(phys)
        check(_lib.load().imga_partition_jvp(self.h, _ptr(_vec(u, nn, "u")), _ptr(_vec(u_prev, nn, "u_prev")),
                                             _ptr(_vec(u_prev2, nn, "u_prev2")), _ptr(_vec(f, nn, "f")), C.byref(ps),
                                             precision, _ptr(_vec(v, nn, "v")), _ptr(out), _stream(stream)))
        return out

    def close(self):
        if getattr(self, "h", None):
            _lib.load().imga_partition_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def peak_flops(kind, device=0):
    """Measured TFLOP/s of an arithmetic pipe: kind 0 FP32 FMA, 1 packed FP32x2 FMA, 2 FP64 FMA."""
    t = C.c_double(0.0)
    check(_lib.load().imga_peak_flops(device, kind, C.byref(t)))
    return t.value


def selftest_conversions(n=1 << 24, seed=1, device=0):
    """imga_selftest_conversions: number of float64 <-> float32 conversion cases (of n) whose result
    differs from the hardware conversion."""
    bad = C.c_int64()
    check(_lib.load().imga_selftest_conversions(device, n, seed, C.byref(bad)))
    return bad.value


def gemm_bf16(A, B, stream=None):
    """C = A B^T with A, B rounded to BF16, FP32 accumulate (float32 CUDA tensors)."""
    import torch
    M, K = A.shape
    N = B.shape[0]
    Cm = torch.empty((M, N), dtype=torch.float32, device=A.device)
    check(_lib.load().imga_gemm_bf16(M, N, K, _ptr(A), _ptr(B), _ptr(Cm), _stream(stream)))
    return Cm
