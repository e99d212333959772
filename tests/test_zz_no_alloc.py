"""The entry point that allocates no device memory.

Callers that cannot call cudaMalloc (a host framework owning all device
memory, a fixed memory budget, a loop that must not synchronise on
allocation) use mlba_residual_noalloc, whose reduction scratch is a fixed
array inside the library.  This test calls it through the C ABI twice in a
row, with different sizes and boundary treatments so that the shared scratch
is reused, and checks each result against the existing operator entry point
mlba_op_blur (r = g - A f computed from its output) at the FP32 tolerance of
the other operator tests.  The file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import mlba_inputs as I

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def M():
    from paper_1504_07234_gb300.build import build
    build()
    import paper_1504_07234_gb300 as mod
    return mod


def one_case(M, torch, psf, n, bc, seed):
    ctx = M.Context(psf, n, bc, "none", dtype="f32")
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((ctx.nf, ctx.nf)).astype(np.float32)
    g = rng.standard_normal((n, n)).astype(np.float32)
    af = ctx.blur(f).astype(np.float64)                    # existing entry point
    ctx.close()
    r_ref = g.astype(np.float64) - af
    df = torch.from_numpy(f).cuda()
    dg = torch.from_numpy(g).cuda()
    dh = torch.from_numpy(psf.astype(np.float32)).cuda()
    dr = torch.empty((n, n), dtype=torch.float32, device="cuda")
    dn = torch.zeros(1, dtype=torch.float64, device="cuda")
    stream = torch.cuda.current_stream().cuda_stream
    rc = M.load_library().mlba_residual_noalloc(
        ctypes.c_void_p(df.data_ptr()), ctypes.c_void_p(dg.data_ptr()), ctypes.c_void_p(dh.data_ptr()),
        psf.shape[0], n, M.BC[bc], ctypes.c_void_p(dr.data_ptr()), ctypes.c_void_p(dn.data_ptr()),
        ctypes.c_void_p(stream))
    assert rc == 0
    torch.cuda.synchronize()
    r = dr.cpu().numpy().astype(np.float64)
    assert np.abs(r - r_ref).max() <= TOL * np.abs(r_ref).max()
    norm2 = float(dn.item())
    assert abs(norm2 - float((r_ref ** 2).sum())) <= TOL * float((r_ref ** 2).sum())


def test_noalloc_residual_two_calls_match_existing_entry_point(M):
    import torch
    one_case(M, torch, I.psf_motion(9, 0.4), 150, "reflective", 1)
    one_case(M, torch, I.psf_gaussian(2.0, 13), 67, "rect", 2)


def test_noalloc_rejects_oversize(M):
    lib = M.load_library()
    p = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    assert lib.mlba_residual_noalloc(p, p, p, 5, 4097, 1, p, p, None) == -7
    assert lib.mlba_residual_noalloc(p, p, p, 43, 1000, 1, p, p, None) == -7
