"""imga_jvp_noalloc: the J v entry point for callers that cannot allocate device memory.

Some callers may not allocate device memory at the moment they apply the operator: a process
whose GPU memory is capped, or one that reserves everything at start-up and treats any later
cudaMalloc as a failure.  For them the library offers imga_jvp_noalloc, which takes the same
inputs and writes the same output as imga_jvp but keeps its per-call scratch in a fixed device
array compiled into the library instead of asking for memory.  These tests call it through the C
ABI, twice in a row with different directions, and check it against imga_jvp within the
tolerances of the parity tests; they also check that a mesh too large for the fixed array is
refused with a clear message.  The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

from paper_2009_00706_gb300 import _lib, api
from paper_2009_00706_gb300 import inputs as I

FP64_TOL = 1e-10
MIXED_TOL = 2e-5


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    _lib.build()
    dev = torch.device("cuda:0")
    w = I.small_sphere()
    mesh = api.Mesh.from_workload(w, device=0)
    return w, mesh, dev


def _noalloc(mesh, ph, u, up, v, prec, out):
    L = _lib.load()
    ps = api.physics_struct(ph)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    p = lambda t: C.c_void_p(t.data_ptr())
    return L.imga_jvp_noalloc(mesh.h, p(u), p(up), None, None, C.byref(ps), prec, p(v), p(out), stream)


@pytest.mark.parametrize("prec,tol", [(api.PRECISION_FP64, FP64_TOL), (api.PRECISION_MIXED, MIXED_TOL)])
def test_noalloc_matches_jvp_on_two_calls_in_a_row(setup, prec, tol):
    w, mesh, dev = setup
    u, up, _ = I.state(mesh.n_nodes, 7)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    ud, upd = t(u), t(up)
    for k in range(2):
        v = t(I.normal(300 + k, 4 * mesh.n_nodes).reshape(-1, 4))
        ref = mesh.jvp(w.physics, ud, upd, v, precision=prec)
        out = torch.full_like(ref, float("nan"))
        st = _noalloc(mesh, w.physics, ud, upd, v, prec, out)
        assert st == 0, _lib.load().imga_last_error()
        torch.cuda.synchronize()
        a, b = out.cpu().numpy(), ref.cpu().numpy()
        assert np.all(np.isfinite(a))
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(b)


def test_noalloc_refuses_a_mesh_beyond_its_fixed_scratch(setup):
    w, mesh, dev = setup
    big = api.Mesh((0, 0, 0), (1, 1, 1), 6, [], None, 3, device=0)      # 64^3 elements, 274,625 nodes
    u, up, v = I.state(big.n_nodes, 1)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    out = torch.zeros((big.n_nodes, 4), dtype=torch.float64, device=dev)
    st = _noalloc(big, w.physics, t(u), t(up), t(v), api.PRECISION_FP64, out)
    assert st == 1
    assert b"too large" in _lib.load().imga_last_error()
    # the same mesh fits in single precision (half the bytes per node)
    st = _noalloc(big, w.physics, t(u), t(up), t(v), api.PRECISION_MIXED, out)
    assert st == 0
    ref = big.jvp(w.physics, t(u), t(up), t(v), precision=api.PRECISION_MIXED)
    torch.cuda.synchronize()
    assert torch.linalg.norm(out - ref) <= MIXED_TOL * torch.linalg.norm(ref)
