"""Build and load the imga C-ABI library (libimga.so, sm_103a) and declare its signatures.

The library is compiled in-tree with nvcc: one translation unit per source, in parallel, linked
into paper_2009_00706_gb300/_build/libimga.so.  Loading fails loudly when the library is absent
or cannot be loaded: there is no fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libimga.so")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"

# (source, extra flags)
SOURCES = [
    ("mesh_host.cpp", ["-Xcompiler", "-ffp-contract=off", "-Xcompiler", "-fopenmp"]),
    ("capi.cpp", []),
    ("batch.cpp", []),
    ("geom.cu", ["-fmad=false"]),
    ("vms.cu", []),
    ("jac.cu", []),
    ("solver.cu", []),
    ("bsr.cu", ["-Xcompiler", "-fopenmp"]),
    ("peak.cu", []),
    ("partition.cu", []),
    ("mlp.cu", []),
]
HEADERS = ["imga_internal.h", "vms_device.cuh", os.path.join("..", "..", "include", "imga.h")]


def _nvcc():
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the imga library needs the CUDA toolkit to build")
    return cand


def _stale(obj, src):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    deps = [src] + [os.path.join(SRC, h) for h in HEADERS]
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile every source for sm_103a and link libimga.so; returns its path."""
    os.makedirs(OUT_DIR, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", ARCH, "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(HERE, "..", "include")]
    jobs = []
    objs = []
    for src, extra in SOURCES:
        s = os.path.join(SRC, src)
        o = os.path.join(OUT_DIR, src + ".o")
        objs.append(o)
        if force or _stale(o, s):
            lang = ["-x", "cu"] if src.endswith(".cu") else ["-x", "c++"]
            jobs.append([nvcc, "-c", *lang, s, "-o", o, *common, *extra])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        if verbose:
            print(r.stdout + r.stderr)
        return r

    with ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        list(ex.map(run, jobs))
    if jobs or not os.path.exists(LIB):
        tmp = LIB + f".{os.getpid()}.tmp"
        run([nvcc, "-shared", ARCH, "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"])
        os.replace(tmp, LIB)
    return LIB


# ------------------------------------------------------------------------------------------
# C structures (mirror include/imga.h)
# ------------------------------------------------------------------------------------------
class Region(C.Structure):
    _fields_ = [("kind", C.c_int), ("level", C.c_int), ("par", C.c_double * 8)]


class MeshParams(C.Structure):
    _fields_ = [("lo", C.c_double * 3), ("hi", C.c_double * 3), ("base_level", C.c_int), ("n_regions", C.c_int),
                ("regions", C.POINTER(Region)), ("quad_max_split", C.c_int)]


class Physics(C.Structure):
    _fields_ = [("rho", C.c_double), ("mu", C.c_double), ("dt", C.c_double), ("time_scheme", C.c_int),
                ("C_b", C.c_double), ("C_I", C.c_double), ("g_body", C.c_double * 3), ("u_inf", C.c_double * 3),
                ("drop_visc_strong", C.c_int), ("g_points", C.c_void_p)]


class Problem(C.Structure):
    _fields_ = [("tri_xyz_host", C.c_void_p), ("n_tri", C.c_int64), ("params", MeshParams), ("mu", C.c_double)]


class MeshInfo(C.Structure):
    _fields_ = [("n_elem", C.c_int64), ("n_nodes", C.c_int64), ("n_hanging", C.c_int64), ("n_out", C.c_int64),
                ("n_in", C.c_int64), ("n_cut", C.c_int64), ("n_cut_points", C.c_int64),
                ("n_surface_points", C.c_int64), ("n_tri", C.c_int64), ("n_bt", C.c_int64), ("n_rays", C.c_int64),
                ("hi_int", C.c_int64 * 3), ("scale", C.c_double), ("setup_ms", C.c_double * 4)]


class SolverOpts(C.Structure):
    _fields_ = [("gmres_m", C.c_int), ("max_newton", C.c_int), ("max_krylov", C.c_int), ("rtol", C.c_double),
                ("atol", C.c_double), ("krylov_rtol", C.c_double), ("precision", C.c_int), ("precond", C.c_int),
                ("line_search", C.c_int), ("learned", C.c_void_p), ("learned_omega", C.c_double),
                ("linear_solver", C.c_int), ("ml_agg", C.c_int), ("ml_coarse_max", C.c_int), ("ml_sweeps", C.c_int),
                ("ml_omega", C.c_double)]


class SolverStats(C.Structure):
    _fields_ = [("newton_its", C.c_int), ("krylov_its", C.c_int), ("krylov_per_newton", C.c_int * 32),
                ("res_norm", C.c_double * 33), ("time_ms", C.c_double), ("converged", C.c_int), ("fallbacks", C.c_int),
                ("krylov_rel", C.c_double * 32)]


# every entry point declared in include/imga.h, with its ctypes signature
_vp, _i64, _int, _dp = C.c_void_p, C.c_int64, C.c_int, C.c_void_p
SIGNATURES = {
    "imga_build_mesh": (C.c_int, [_dp, _i64, C.POINTER(MeshParams), _int, C.POINTER(_vp)]),
    "imga_destroy_mesh": (None, [_vp]),
    "imga_build_mesh_batch": (C.c_int, [C.POINTER(Problem), _int, _int, C.POINTER(_vp)]),
    "imga_mesh_problems": (C.c_int, [_vp, C.POINTER(C.c_int), _vp, _vp]),
    "imga_mesh_get_info": (C.c_int, [_vp, C.POINTER(MeshInfo)]),
    "imga_mesh_export": (C.c_int, [_vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "imga_export_markers": (C.c_int, [_vp, _vp, _vp]),
    "imga_export_cut_points": (C.c_int, [_vp, _vp, _vp]),
    "imga_export_surface_points": (C.c_int, [_vp, _vp]),
    "imga_export_background": (C.c_int, [_vp, _vp, _vp]),
    "imga_classify": (C.c_int, [_vp, _vp, _i64, _vp, _vp]),
    "imga_classify_counts": (C.c_int, [_vp, _vp, _int]),
    "imga_bsr_pattern": (C.c_int, [_vp, C.POINTER(C.c_int64), _vp, _vp]),
    "imga_node_coords": (C.c_int, [_vp, _vp, _vp]),
    "imga_residual": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(Physics), _int, _vp, _vp]),
    "imga_jvp": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(Physics), _int, _vp, _vp, _vp]),
    "imga_jvp_noalloc": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(Physics), _int, _vp, _vp, _vp]),
    "imga_selftest_conversions": (C.c_int, [_int, _i64, C.c_uint64, C.POINTER(C.c_int64)]),
    "imga_tuning": (C.c_int, [_vp, _vp, _vp]),
    "imga_set_dirichlet": (C.c_int, [_vp, _vp, _vp, _vp]),
    "imga_element_jacobians": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(Physics), _int, _vp, _i64, _vp, _vp]),
    "imga_newton_step": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(Physics), C.POINTER(SolverOpts),
                                   C.POINTER(SolverStats), _vp]),
    "imga_mlp_create": (C.c_int, [_int, _int, _int, C.c_uint64, _int, C.POINTER(_vp)]),
    "imga_mlp_destroy": (None, [_vp]),
    "imga_mlp_shape": (C.c_int, [_vp, C.POINTER(C.c_int64), C.POINTER(C.c_int)]),
    "imga_mlp_params": (C.c_int, [_vp, _vp, _int]),
    "imga_mlp_forward": (C.c_int, [_vp, _vp, _i64, _i64, _vp, _vp]),
    "imga_mlp_gradient": (C.c_int, [_vp, _vp, _i64, _vp, _i64, C.POINTER(C.c_double), _vp, _vp]),
    "imga_mlp_train": (C.c_int, [_vp, _vp, _i64, _vp, _i64, _int, _int, C.c_float, _vp, _vp]),
    "imga_precond_dataset": (C.c_int, [_vp, _vp, _vp, _vp, _vp, C.POINTER(Physics), _int, _vp, _i64, _int, _vp, _vp,
                                       _vp, _vp]),
    "imga_gemm_bf16": (C.c_int, [_int, _int, _int, _vp, _vp, _vp, _vp]),
    "imga_set_option": (C.c_int, [_vp, _int, _i64]),
    "imga_profile": (C.c_int, [_vp, _int]),
    "imga_profile_read": (C.c_int, [_vp, _vp, _vp]),
    "imga_last_error": (C.c_char_p, []),
    "imga_bsr_assemble": (C.c_int, [_vp, _dp, _dp, _dp, _dp, C.POINTER(Physics), _int, _dp, _vp]),
    "imga_bsr_spmv": (C.c_int, [_vp, _dp, _dp, _dp, _vp]),
    "imga_multilevel_setup": (C.c_int, [_vp, _dp, _dp, _dp, _dp, C.POINTER(Physics), _int, _int, _int, _int, C.c_double,
                                        _vp]),
    "imga_multilevel_apply": (C.c_int, [_vp, _dp, _dp, _vp]),
    "imga_multilevel_info": (C.c_int, [_vp, C.POINTER(C.c_int), _vp, _vp]),
    "imga_peak_flops": (C.c_int, [_int, _int, C.POINTER(C.c_double)]),
    "imga_surface_force": (C.c_int, [_vp, _dp, _dp, C.POINTER(Physics), _dp, _vp]),
    "imga_time_steps": (C.c_int, [_vp, _dp, _dp, _dp, C.POINTER(Physics), C.POINTER(SolverOpts), _int, _vp, _vp, _vp,
                                  _vp]),
    "imga_partition_build": (C.c_int, [_vp, _int, C.c_double, C.POINTER(_vp)]),
    "imga_partition_destroy": (None, [_vp]),
    "imga_partition_info": (C.c_int, [_vp, C.POINTER(C.c_int), _vp, _vp, _vp, _vp]),
    "imga_partition_nodes": (C.c_int, [_vp, _int, _vp, _vp]),
    "imga_partition_residual": (C.c_int, [_vp, _dp, _dp, _dp, _dp, C.POINTER(Physics), _int, _dp, _vp]),
    "imga_partition_jvp": (C.c_int, [_vp, _dp, _dp, _dp, _dp, C.POINTER(Physics), _int, _dp, _dp, _vp]),
    "imga_tuning_interior": (C.c_int, [_vp, _vp, _vp]),
    "imga_fused_info": (C.c_int, [_vp, _vp]),
}

_lib = None


def load(path: str | None = None):
    """Load libimga.so (it must have been built) and attach the signatures."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB
    if not os.path.exists(p):
        raise RuntimeError(f"imga library not built ({p}); run paper_2009_00706_gb300._lib.build()")
    L = C.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


class ImgaError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"imga status {status}: {msg}")
        self.status = status


def check(status):
    if status != 0:
        raise ImgaError(status, load().imga_last_error().decode(errors="replace"))
