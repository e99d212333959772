"""The entry point that allocates no device memory.

Callers that cannot call cudaMalloc (a host framework owning all device
memory, a fixed memory budget, a loop that must not synchronise on
allocation) use mlba_residual_noalloc, whose reduction scratch is a fixed
array inside the library.  These tests call it through the C ABI several
times in a row, with different sizes and boundary treatments so that the
shared scratch is reused, and check each result against the existing operator
entry point mlba_op_blur (r = g - A f computed from its output) at the FP32
tolerance of the other operator tests, and against the FP64 oracle's blur
(whole image, or windows of the largest image).  The file is named to be
collected last.
"""
import ctypes

import numpy as np
import pytest

import mlba_inputs as I
from oracle import mlba_oracle as O

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def M():
    from paper_1504_07234_gb300.build import build
    build()
    import paper_1504_07234_gb300 as mod
    return mod


def call_noalloc(M, torch, f, g, psf, bc):
    n = g.shape[0]
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
    return dr.cpu().numpy().astype(np.float64), float(dn.item())


def one_case(M, torch, psf, n, bc, seed, windows=None):
    ctx = M.Context(psf, n, bc, "none", dtype="f32")
    rng = np.random.default_rng(seed)
    f = rng.standard_normal((ctx.nf, ctx.nf)).astype(np.float32)
    g = rng.standard_normal((n, n)).astype(np.float32)
    af = ctx.blur(f).astype(np.float64)                    # existing entry point
    ctx.close()
    r_lib = g.astype(np.float64) - af
    r, norm2 = call_noalloc(M, torch, f, g, psf, bc)
    assert np.abs(r - r_lib).max() <= TOL * np.abs(r_lib).max()
    ss = float((r_lib ** 2).sum())
    assert abs(norm2 - ss) <= TOL * ss
    # the FP64 oracle: whole image, or windows (p x p blur of a crop of the
    # Table 1 extension of f, which is the rectangular operator on the crop)
    f64, g64 = f.astype(np.float64), g.astype(np.float64)
    if windows is None:
        r_or = g64 - O.blur(f64, psf, bc)
        assert np.abs(r - r_or).max() <= TOL * np.abs(r_or).max()
        so = float((r_or ** 2).sum())
        assert abs(norm2 - so) <= TOL * so
    else:
        p = psf.shape[0]
        c = (p - 1) // 2
        fe = f64 if bc == "rect" else O.extend(f64, c, bc)
        for (y0, x0, w) in windows:
            crop = fe[y0:y0 + w + p - 1, x0:x0 + w + p - 1]
            r_or = g64[y0:y0 + w, x0:x0 + w] - O.blur(crop, psf, "rect")
            got = r[y0:y0 + w, x0:x0 + w]
            assert np.abs(got - r_or).max() <= TOL * np.abs(r_or).max(), (y0, x0)


def test_noalloc_residual_calls_in_a_row_match_existing_entry_point_and_oracle(M):
    import torch
    one_case(M, torch, I.psf_motion(9, 0.4), 150, "reflective", 1)
    one_case(M, torch, I.psf_gaussian(2.0, 13), 67, "rect", 2)
    one_case(M, torch, I.psf_disk(3), 83, "zero", 3)
    one_case(M, torch, np.array([[0.0, 0.1, 0.05], [0.2, 0.3, 0.0], [0.15, 0.1, 0.1]]), 45,
             "periodic", 4)


def test_noalloc_largest_tile_count_and_halo(M):
    """n = 4096 fills the fixed scratch exactly (16384 tiles) and p = 41 is
    the largest halo; one call, checked against the existing entry point and
    on corner, edge and interior windows against the oracle."""
    import torch
    n = 4096
    wins = [(0, 0, 48), (0, n - 48, 48), (n - 48, n - 48, 48), (2000, 17, 48), (1234, 3000, 48)]
    one_case(M, torch, I.psf_gaussian(6.0, 41), n, "periodic", 5, windows=wins)


def test_noalloc_rejects_oversize(M):
    lib = M.load_library()
    p = ctypes.c_void_p(16)   # never dereferenced: the size check comes first
    assert lib.mlba_residual_noalloc(p, p, p, 5, 4097, 1, p, p, None) == -7
    assert lib.mlba_residual_noalloc(p, p, p, 43, 1000, 1, p, p, None) == -7
