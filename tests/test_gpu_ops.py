"""GPU parity per operator: each kernel pass, called through the C ABI, against
the FP64 oracle on the same seeded inputs.

Tolerances: FP64 path max|err| <= 1e-11 * max|ref| (rounding-order only);
FP32 path <= 1e-5 relative in the max norm (per-operator bar of the design)
and 2e-2 for the bf16-stored Bregman variable (8 significant bits).
Sizes span several 32 x 32 tiles with ragged tails, sizes below one tile, and
FFT lengths with radix 2, 3, 4 and 5 factors and with prime factors above 5
(direct-sum passes: 196 = 2^2 7^2, 226 = 2 x 113, the prime 197, 4093).
"""
import numpy as np
import pytest

import mlba_inputs as I
from oracle import mlba_oracle as O

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-11, "f32": 1e-5}


@pytest.fixture(scope="module")
def M():
    from paper_1504_07234_gb300.build import build
    build()
    import paper_1504_07234_gb300 as mod
    return mod


def rel_err(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


PSFS = {
    "gauss9": I.psf_gaussian(2.0, 9),               # separable path
    "disk2": I.psf_disk(2),                         # dense tap list, symmetric
    "motion7": I.psf_motion(7, 0.7),                # sparse, nonsymmetric
    "asym3": np.array([[0.0, 0.1, 0.05], [0.2, 0.3, 0.0], [0.15, 0.1, 0.1]]),
    "gauss31": I.psf_gaussian(5.0, 31),
    "gauss41": I.psf_gaussian(7.0, 41),             # separable, p > 33: row pass into a second tile
    "disk17": I.psf_disk(17),                       # 37 x 37 dense runs: full groups of 8 taps + remainders
}


@pytest.mark.parametrize("path", ["direct", "fft"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["zero", "periodic", "reflective", "rect", "antireflective"])
@pytest.mark.parametrize("psf,n", [("gauss9", 70), ("disk2", 33), ("motion7", 45), ("asym3", 17),
                                   ("gauss31", 64), ("gauss41", 80), ("disk17", 72)])
def test_blur_and_adjoint(M, path, dtype, bc, psf, n):
    """A and A^T by the direct stencils and by FFT convolution on a padded
    size (Sections 2.1, 2.2); for antireflective BCs A^T is the reblurring
    matrix A'."""
    h = PSFS[psf]
    ctx = M.Context(h, n, bc, "none", dtype=dtype, blur_path=path)
    rng = np.random.default_rng(n)
    f = rng.standard_normal((ctx.nf, ctx.nf))
    t = rng.standard_normal((n, n))
    assert rel_err(ctx.blur(f), O.blur(f, h, bc)) <= TOL[dtype]
    ref = O.reblur(t, h, bc) if bc == "antireflective" else O.blur_adjoint(t, h, bc)
    assert rel_err(ctx.blur_adjoint(t), ref) <= TOL[dtype]
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [48, 60, 64, 100, 128, 192, 250, 256, 42, 196, 226, 197])
@pytest.mark.parametrize("transform,psf", [("dft", "motion7"), ("dct", "disk2"), ("dft", "gauss9"),
                                           ("dct", "gauss9")])
def test_spectrum_and_precond(M, dtype, n, transform, psf):
    h = PSFS[psf]
    ctx = M.Context(h, n, "periodic", "bccb", dtype=dtype, transform=transform)
    pre = O.SpectralPrecond(h, n, transform)
    lam = ctx.spectrum()
    if transform == "dft":
        ref = pre.lam[:, : n // 2 + 1]
    else:
        ref = pre.lam
    assert float(np.abs(lam - ref).max()) <= (1e-13 if dtype == "f64" else 2e-7)
    rng = np.random.default_rng(n + 1)
    r = rng.standard_normal((n, n))
    for which in ("inv", "tikh"):
        for alpha in (0.05, 1e-3):
            ref_t = pre.inv(r, alpha) if which == "inv" else pre.tikh(r, alpha)
            got = ctx.precond(r, alpha, which)
            assert rel_err(got, ref_t) <= (1e-11 if dtype == "f64" else 2e-5), (which, alpha)
    ctx.close()


@pytest.mark.parametrize("dtype,zs", [("f64", "f64"), ("f32", "f32"), ("f32", "bf16")])
@pytest.mark.parametrize("levels", [1, 2, 3, 4])
@pytest.mark.parametrize("bc,n", [("periodic", 70), ("reflective", 20), ("rect", 37), ("zero", 64),
                                  ("reflective", 11)])
def test_frame_step(M, dtype, zs, levels, bc, n):
    """L = 4 is the paper's setting (Section 6.1): dilation 8, reach 30 pixels
    per side, wider than the 11 x 11 and 20 x 20 images (repeated mirroring)."""
    h = PSFS["asym3"]
    ctx = M.Context(h, n, bc, "none", dtype=dtype, z_store=zs, levels=levels)
    nf = ctx.nf
    rng = np.random.default_rng(levels * 100 + n)
    z_in = 0.05 * rng.standard_normal((8 * levels + 1, nf, nf))
    if zs == "bf16":
        import torch
        z_in = torch.tensor(z_in, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    u = 0.1 * rng.standard_normal((nf, nf))
    mu = 0.03
    zo, f = ctx.frame(z_in, u, mu)
    z_ref = z_in + O.framelet_analysis(u, levels)
    f_ref = O.framelet_synthesis(O.soft(z_ref, mu), levels)
    tol_z = {"f64": 1e-12, "f32": 2e-6, "bf16": 1e-2}[zs]
    assert rel_err(zo.double().cpu().numpy(), z_ref) <= tol_z
    # f is synthesised from the FP32 update before z is rounded for storage
    assert rel_err(f.double().cpu().numpy(), f_ref) <= (1e-11 if dtype == "f64" else 1e-5)
    ctx.close()


def test_frame_tight_frame_on_gpu(M):
    """mu = 0 and z_in = 0: f = W^T W u = u (Section 3) through the fused kernel."""
    ctx = M.Context(PSFS["asym3"], 53, "reflective", "none", dtype="f64", levels=2)
    u = np.random.default_rng(7).standard_normal((53, 53))
    zo, f = ctx.frame(np.zeros((17, 53, 53)), u, 0.0)
    assert rel_err(f.cpu().numpy(), u) <= 1e-13
    ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("transform,psf,n", [("dct", "disk2", 64), ("dft", "motion7", 96),
                                             ("dct", "gauss9", 60), ("dft", "motion7", 300),
                                             ("dct", "disk2", 200), ("dct", "disk2", 196),
                                             ("dft", "motion7", 226), ("dft", "motion7", 197)])
def test_ns_alpha(M, dtype, transform, psf, n):
    """Also at sizes whose spectrum rows do not tile the per-block element
    count (300: 151 half-spectrum columns; 200: 200 DCT columns).  FP32 is
    held to the per-operator 1e-5: the root moves by less than 5e-8 when the
    oracle's spectrum and eigenvalues are rounded to FP32, so the FP32
    spectrum is not the limit, and the FP32 candidate sums measured at most
    1.2e-6 on these cases."""
    h = PSFS[psf]
    ctx = M.Context(h, n, "reflective" if transform == "dct" else "periodic", "tikh_ns",
                    dtype=dtype, transform=transform)
    pre = O.SpectralPrecond(h, n, transform)
    r = np.random.default_rng(3).standard_normal((n, n))
    for qn in (0.5, 0.8, 0.95):
        ref = O.ns_alpha(np.abs(pre.forward(r)) ** 2, pre.sigma, qn)
        got = ctx.ns_alpha(r, qn)
        assert abs(got - ref) <= (1e-10 if dtype == "f64" else 1e-5) * ref, (qn, got, ref)
    ctx.close()


@pytest.mark.parametrize("transform,psf", [("dft", "motion7"), ("dct", "gauss9")])
def test_precond_largest_prime_length(M, transform, psf):
    """n = 4093, the largest prime below the 4096 limit: one direct-sum pass
    of radix 4093 per 1-D transform (FP32).  Checked against the oracle's
    preconditioner on the whole image."""
    n = 4093
    h = PSFS[psf]
    ctx = M.Context(h, n, "periodic" if transform == "dft" else "reflective", "bccb",
                    dtype="f32", transform=transform)
    pre = O.SpectralPrecond(h, n, transform)
    r = np.random.default_rng(11).standard_normal((n, n))
    got = ctx.precond(r, 0.05, "inv")
    assert rel_err(got, pre.inv(r, 0.05)) <= 2e-5
    ctx.close()


@pytest.mark.parametrize("zs", ["f32", "bf16"])
@pytest.mark.parametrize("shape", range(8))
@pytest.mark.parametrize("levels", [1, 2])
def test_frame_step_every_tile_shape(M, zs, shape, levels):
    """Every tile shape of the fused framelet kernel (register queue or ring
    of z rows filled by bulk asynchronous copies, with per-lane copies where
    a warp's columns cross the image edge) against the oracle; 150 x 150 with
    the reflective BC and 97 x 97 rectangular (103 x 103 unknown) put warps on
    both sides of that split."""
    for bc, n in (("reflective", 150), ("rect", 97)):
        ctx = M.Context(PSFS["gauss9"] if bc == "rect" else PSFS["asym3"], n, bc, "none",
                        dtype="f32", z_store=zs, levels=levels, frame_shape=shape)
        assert ctx.tiles()["frame_shape"] == shape
        nf = ctx.nf
        rng = np.random.default_rng(shape * 10 + levels)
        z_in = 0.05 * rng.standard_normal((8 * levels + 1, nf, nf))
        if zs == "bf16":
            import torch
            z_in = torch.tensor(z_in, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
        u = 0.1 * rng.standard_normal((nf, nf))
        zo, f = ctx.frame(z_in, u, 0.03)
        z_ref = z_in + O.framelet_analysis(u, levels)
        f_ref = O.framelet_synthesis(O.soft(z_ref, 0.03), levels)
        assert rel_err(zo.double().cpu().numpy(), z_ref) <= (2e-6 if zs == "f32" else 1e-2)
        assert rel_err(f.double().cpu().numpy(), f_ref) <= 1e-5
        ctx.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n", [3, 17, 48, 100, 197, 256])
@pytest.mark.parametrize("psf", ["gauss9", "disk2"])
def test_antireflective_transform_precond(M, dtype, n, psf):
    """The antireflective transform (Section 2.2) for antireflective BCs and a
    quadrantally symmetric PSF: eigenvalues and (CC' + alpha I)^{-1},
    C'(CC' + alpha I)^{-1} against the oracle's dense transform."""
    h = PSFS[psf]
    if h.shape[0] > n:
        h = I.psf_gaussian(0.6, 3)
    ctx = M.Context(h, n, "antireflective", "bccb", dtype=dtype, transform="ar")
    pre = O.SpectralPrecond(h, n, "ar")
    assert float(np.abs(ctx.spectrum() - pre.lam).max()) <= (1e-13 if dtype == "f64" else 2e-7)
    r = np.random.default_rng(n + 7).standard_normal((n, n))
    for which in ("inv", "tikh"):
        for alpha in (0.05, 1e-3):
            ref = pre.inv(r, alpha) if which == "inv" else pre.tikh(r, alpha)
            got = ctx.precond(r, alpha, which)
            assert rel_err(got, ref) <= (1e-11 if dtype == "f64" else 2e-5), (which, alpha)
    ctx.close()
