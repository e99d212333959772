"""GPU parity of whole MLBA runs (Eq. MLBA2, Algorithms 1-4, 4-NS) against the
FP64 oracle, called through the C ABI.

FP64 path: the restoration f, the residual-norm history, alpha_n and beta_n
match the oracle to rounding (tolerances below).  FP32 path (FP64 norms,
denominators and alpha_n): restoration-level bars — RRE within 1e-3, PSNR
within 0.05 dB, the discrepancy stop within one iteration — plus a relative
image difference bound.
"""
import math

import numpy as np
import pytest

import mlba_inputs as I
from oracle import mlba_oracle as O

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def M():
    from paper_1504_07234_gb300.build import build
    build()
    import paper_1504_07234_gb300 as mod
    return mod


def run_gpu(M, pr, dtype="f64", z_store=None, iters=None, stop=None):
    stop = pr.stop if stop is None else stop
    max_iter = pr.max_iter if iters is None else iters
    ctx = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype=dtype, z_store=z_store,
                    mu=pr.mu, alpha=pr.alpha, levels=pr.levels, max_iter=max_iter, stop=stop,
                    gamma=pr.gamma, q=pr.q, rho=pr.rho, transform=pr.transform,
                    rect_ns_hybrid=pr.rect_ns_hybrid)
    ctx.set_data(pr.g, pr.delta)
    st = ctx.run(max_iter)
    f = ctx.result()
    res, al, be = ctx.history()
    ctx.close()
    return f, st, res, al, be


def run_oracle(pr, iters=None, stop=None):
    stop = pr.stop if stop is None else stop
    return O.mlba(pr.g, pr.psf, pr.delta, pr.bc, pr.precond, pr.mu, pr.alpha, pr.levels,
                  pr.max_iter if iters is None else iters, stop=stop, gamma=pr.gamma, q=pr.q,
                  rho=pr.rho, transform=pr.transform, rect_ns_hybrid=pr.rect_ns_hybrid)


def small(bc, precond, n=40, psf=None, levels=2, alpha=0.3, mu=10 / 255, iters=12,
          transform="auto", nu=0.01, seed=21):
    psf = I.psf_motion(7, 0.9) if psf is None else psf
    p = psf.shape[0]
    f = I.true_image(n + p - 1, seed)
    g, delta = I.observe(f, psf, nu, seed)
    return I.Problem(g=g, psf=psf, delta=delta, bc=bc, precond=precond, mu=mu, alpha=alpha,
                     levels=levels, max_iter=iters, stop=False, transform=transform, f_true=f,
                     rect_ns_hybrid=(bc == "rect" and precond == "tikh_ns"))


CASES = [
    ("rect", "none", "auto", I.psf_motion(7, 0.9), 0.3),
    ("rect", "bccb", "dft", I.psf_motion(7, 0.9), 0.3),
    ("rect", "bccb", "dct", I.psf_gaussian(1.5, 7), 0.1),
    ("rect", "krylov", "dft", I.psf_motion(7, 0.9), 0.05),
    ("rect", "sym", "auto", I.psf_motion(7, 0.9), 0.5),
    ("rect", "tikh_ns", "dct", I.psf_gaussian(1.5, 7), 0.05),
    ("zero", "bccb", "dft", I.psf_motion(7, 0.9), 0.3),
    ("zero", "krylov", "dft", I.psf_motion(7, 0.9), 0.05),
    ("zero", "tikh", "dft", I.psf_motion(7, 0.9), 0.05),
    ("periodic", "bccb", "dft", I.psf_motion(7, 0.9), 0.05),
    ("periodic", "tikh_ns", "dft", I.psf_motion(7, 0.9), 0.05),
    ("reflective", "sym", "auto", I.psf_motion(7, 0.9), 0.3),
    ("reflective", "tikh", "dct", I.psf_disk(3), 0.02),
    ("reflective", "tikh_ns", "dct", I.psf_disk(3), 0.05),
    ("reflective", "krylov", "dct", I.psf_disk(3), 0.02),
]


@pytest.mark.parametrize("bc,precond,transform,psf,alpha", CASES,
                         ids=[f"{c[0]}-{c[1]}-{c[2]}" for c in CASES])
def test_fp64_loop_matches_oracle(M, bc, precond, transform, psf, alpha):
    n = 48 if bc != "rect" else 42       # several tiles, ragged tails, FFT radix 2, 3, 16, 7
    pr = small(bc, precond, n=n, psf=psf, alpha=alpha, transform=transform)
    f, st, res, al, be = run_gpu(M, pr, "f64")
    ref = run_oracle(pr)
    assert st["iter"] == ref["iters"]
    scale = np.abs(ref["f"]).max()
    assert np.abs(f - ref["f"]).max() <= 1e-9 * scale
    np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-9)
    if precond == "tikh_ns":
        np.testing.assert_allclose(al, ref["alphas"], rtol=1e-8)
    if precond == "krylov":
        assert list(be) == ref["betas"]


ANY_N = [(196, "reflective", "tikh_ns", "dct", I.psf_disk(3), 0.05),   # 2^2 7^2 (Example 3's size)
         (226, "zero", "bccb", "dft", I.psf_motion(7, 0.9), 0.3),         # 2 x 113 (Example 4's size)
         (197, "periodic", "tikh", "dft", I.psf_motion(7, 0.9), 0.05),    # prime
         (197, "rect", "sym", "auto", I.psf_motion(7, 0.9), 0.5)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("n,bc,precond,transform,psf,alpha", ANY_N,
                         ids=[f"{c[0]}-{c[1]}-{c[2]}" for c in ANY_N])
def test_any_length_loop_matches_oracle(M, dtype, n, bc, precond, transform, psf, alpha):
    """Transform lengths with prime factors above 5 (the field-of-view sizes
    of Examples 3 and 4, Section 6, and a prime): FP64 to rounding, FP32 to
    the restoration bars."""
    pr = small(bc, precond, n=n, psf=psf, alpha=alpha, transform=transform, iters=8)
    f, st, res, al, be = run_gpu(M, pr, dtype)
    ref = run_oracle(pr)
    assert st["iter"] == ref["iters"]
    if dtype == "f64":
        assert np.abs(f - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max()
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-9)
        if precond == "tikh_ns":
            np.testing.assert_allclose(al, ref["alphas"], rtol=1e-8)
    else:
        restoration_bars(f, ref, pr)
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-3)


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc,precond,transform,n", [("reflective", "tikh_ns", "dct", 64),
                                                    ("rect", "bccb", "dft", 50)])
def test_four_level_loop_matches_oracle(M, dtype, bc, precond, transform, n):
    """Four framelet levels, the paper's setting (Section 6.1)."""
    psf = I.psf_disk(3) if transform == "dct" else I.psf_motion(7, 0.9)
    pr = small(bc, precond, n=n, psf=psf, levels=4, alpha=0.05 if precond == "tikh_ns" else 0.3,
               transform=transform, iters=8)
    f, st, res, al, be = run_gpu(M, pr, dtype)
    ref = run_oracle(pr)
    assert st["iter"] == ref["iters"]
    if dtype == "f64":
        assert np.abs(f - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max()
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-9)
    else:
        restoration_bars(f, ref, pr)
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-3)


ASYM3 = np.array([[0.0, 0.1, 0.05], [0.2, 0.3, 0.0], [0.15, 0.1, 0.1]])
# (parameters at which the oracle converges: with antireflective BCs the BCCB
# preconditioner needs the larger alpha of Algorithm 1, Section 4.1)
AR_CASES = [("none", "auto", I.psf_motion(7, 0.9), 0.3),
            ("bccb", "dft", I.psf_motion(7, 0.9), 1.0),
            ("tikh", "dft", ASYM3, 0.05),
            ("tikh_ns", "dft", ASYM3, 0.05),
            ("bccb", "dct", I.psf_gaussian(1.5, 7), 0.1)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("precond,transform,psf,alpha", AR_CASES,
                         ids=[f"{c[0]}-{c[1]}" for c in AR_CASES])
def test_antireflective_loop_matches_oracle(M, dtype, precond, transform, psf, alpha):
    """Antireflective BCs with the reblurring matrix A' in place of A^T
    (Section 2.2; the paper's Examples 3 and 4 run Alg-BC1, BC4 and BC4-NS
    with the BCCB preconditioner this way)."""
    pr = small("antireflective", precond, n=58, psf=psf, alpha=alpha, transform=transform, iters=10)
    f, st, res, al, be = run_gpu(M, pr, dtype)
    ref = run_oracle(pr)
    assert st["iter"] == ref["iters"]
    if dtype == "f64":
        assert np.abs(f - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max()
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-9)
        if precond == "tikh_ns":
            np.testing.assert_allclose(al, ref["alphas"], rtol=1e-8)
    else:
        restoration_bars(f, ref, pr)
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-3)


@pytest.mark.parametrize("levels", [2, 4])
def test_antireflective_batch_with_other_bcs(M, levels):
    """Antireflective problems batched with the other boundary treatments
    (two-group schedule), FP64, against the oracle."""
    probs = [small("antireflective", "bccb", n=44, transform="dft", iters=6, levels=levels,
                   alpha=1.0),
             small("reflective", "tikh_ns", n=48, psf=I.psf_disk(3), transform="dct", iters=6,
                   seed=3, levels=levels),
             small("antireflective", "tikh_ns", n=40, psf=ASYM3, iters=6, seed=4,
                   alpha=0.05, levels=levels),
             small("rect", "bccb", n=36, transform="dft", iters=6, seed=5, levels=levels)]
    descs = [dict(psf=p.psf, g=p.g, delta=p.delta, bc=p.bc, precond=p.precond, mu=p.mu,
                  alpha=p.alpha, transform=p.transform, max_iter=6) for p in probs]
    b = M.Batch(descs, dtype="f64", levels=levels, stop=False, max_iter=6, rect_ns_hybrid=True)
    b.iterate(7)
    for i, p in enumerate(probs):
        ref = run_oracle(p)
        assert np.abs(b.result(i) - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max(), i
    b.close()


AR_TR_CASES = [("bccb", I.psf_gaussian(1.5, 7), 0.1),     # auto: the antireflective transform, C = A
               ("tikh", I.psf_disk(3), 0.05),
               ("sym", I.psf_motion(7, 0.9), 0.3)]        # Q from H~ under antireflective BCs


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("precond,psf,alpha", AR_TR_CASES, ids=[c[0] for c in AR_TR_CASES])
def test_antireflective_transform_loop_matches_oracle(M, dtype, precond, psf, alpha):
    """Alg-BC1 / BC4 with C = A and Alg-BC3 (Q = antireflective matrix of H~,
    Section 4.3) through the antireflective transform, as the paper runs
    Examples 3 and 4."""
    pr = small("antireflective", precond, n=61, psf=psf, alpha=alpha, iters=10)
    f, st, res, al, be = run_gpu(M, pr, dtype)
    ref = run_oracle(pr)
    assert st["iter"] == ref["iters"]
    if dtype == "f64":
        assert np.abs(f - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max()
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-9)
    else:
        restoration_bars(f, ref, pr)
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-3)


def test_antireflective_rejects_alg2_and_ns_transform(M):
    h = I.psf_gaussian(1.5, 7)
    with pytest.raises(M.MlbaError):
        M.Context(h, 40, "antireflective", "krylov", dtype="f64")
    with pytest.raises(M.MlbaError):
        M.Context(h, 40, "antireflective", "tikh_ns", dtype="f64", transform="ar")
    with pytest.raises(M.MlbaError):
        M.Context(h, 40, "reflective", "bccb", dtype="f64", transform="ar")


FFT_CASES = [("rect", "bccb", "dft", I.psf_motion(7, 0.9), 0.3),
             ("reflective", "tikh_ns", "dct", I.psf_disk(3), 0.05),
             ("zero", "tikh", "dft", I.psf_motion(7, 0.9), 0.05),
             ("antireflective", "bccb", "dft", I.psf_motion(7, 0.9), 1.0),
             ("periodic", "none", "auto", I.psf_disk(17), 0.3)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc,precond,transform,psf,alpha", FFT_CASES,
                         ids=[f"{c[0]}-{c[1]}" for c in FFT_CASES])
def test_fft_blur_path_loop_matches_oracle(M, dtype, bc, precond, transform, psf, alpha):
    """Loops whose A and A^T run as FFT convolutions (opts.blur_path = 1),
    including a 37 x 37 dense disk, the case the path exists for."""
    n = 48 if bc != "rect" else 42
    pr = small(bc, precond, n=n, psf=psf, alpha=alpha, transform=transform, iters=8)
    descs = [dict(psf=pr.psf, g=pr.g, delta=pr.delta, bc=pr.bc, precond=pr.precond, mu=pr.mu,
                  alpha=pr.alpha, transform=pr.transform, max_iter=8)]
    b = M.Batch(descs, dtype=dtype, levels=pr.levels, stop=False, max_iter=8, blur_path="fft",
                rect_ns_hybrid=pr.rect_ns_hybrid)
    assert b.blur_fft(0)[0] and b.blur_fft(0)[1] >= n + psf.shape[0] - 1
    b.iterate(9)
    f = b.result(0)
    b.close()
    ref = run_oracle(pr)
    if dtype == "f64":
        assert np.abs(f - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max()
    else:
        restoration_bars(f, ref, pr)


def test_fft_blur_path_chosen_per_problem(M):
    """opts.blur_path = 2: every problem gets the faster path, measured at
    create; the results equal the all-direct batch to rounding (FP64)."""
    probs = [small("rect", "bccb", n=40, transform="dft", iters=5),
             small("reflective", "tikh_ns", n=64, psf=I.psf_disk(8), transform="dct", iters=5, seed=3),
             small("periodic", "none", n=50, psf=I.psf_disk(17), iters=5, seed=4)]
    descs = [dict(psf=p.psf, g=p.g, delta=p.delta, bc=p.bc, precond=p.precond, mu=p.mu,
                  alpha=p.alpha, transform=p.transform, max_iter=5) for p in probs]
    out = []
    for path in ("direct", "auto"):
        b = M.Batch(descs, dtype="f64", levels=2, stop=False, max_iter=5, blur_path=path)
        b.iterate(6)
        out.append([b.result(i) for i in range(len(probs))])
        if path == "auto":
            choices = [b.blur_fft(i)[0] for i in range(len(probs))]
        b.close()
    for i in range(len(probs)):
        assert np.abs(out[0][i] - out[1][i]).max() <= 1e-10 * np.abs(out[0][i]).max(), i
    assert len(choices) == 3


BAL_CASES = [("rect", "bccb", "dft", I.psf_motion(7, 0.9), 0.3, 2),
             ("reflective", "tikh_ns", "dct", I.psf_disk(3), 0.05, 2),
             ("zero", "bccb", "dft", I.psf_motion(7, 0.9), 0.3, 4),
             ("antireflective", "tikh", "auto", I.psf_gaussian(1.5, 7), 0.05, 2),
             ("periodic", "krylov", "dft", I.psf_motion(7, 0.9), 0.05, 1)]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc,precond,transform,psf,alpha,levels", BAL_CASES,
                         ids=[f"{c[0]}-{c[1]}-L{c[5]}" for c in BAL_CASES])
def test_balanced_formulation_matches_oracle(M, dtype, bc, precond, transform, psf, alpha, levels):
    """The balanced formulation x = S_mu(W (f + u)) with the paper's
    preconditioners (Section 1, Conclusions) against the oracle."""
    n = 48 if bc != "rect" else 42
    pr = small(bc, precond, n=n, psf=psf, alpha=alpha, transform=transform, iters=8, levels=levels)
    ctx = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype=dtype, mu=pr.mu, alpha=pr.alpha,
                    levels=levels, max_iter=8, stop=False, transform=pr.transform,
                    formulation="balanced")
    ctx.set_data(pr.g, pr.delta)
    ctx.iterate(9)
    f = ctx.result()
    res, al, be = ctx.history()
    ctx.close()
    ref = O.mlba(pr.g, pr.psf, pr.delta, pr.bc, pr.precond, pr.mu, pr.alpha, levels, 8,
                 stop=False, transform=pr.transform, formulation="balanced")
    if dtype == "f64":
        assert np.abs(f - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max()
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-9)
    else:
        restoration_bars(f, ref, pr)


def test_fp64_stop_rule_matches_oracle(M):
    pr = I.config(2, n=64)
    pr.precond, pr.transform = "tikh", "dct"
    pr.alpha = 0.02
    pr.max_iter = 300
    f, st, res, al, be = run_gpu(M, pr, "f64", stop=True)
    ref = run_oracle(pr, stop=True)
    assert st["stopped"] == 1 and st["stop_iter"] == ref["stop_iter"] == st["iter"]
    assert np.abs(f - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max()


NS_PAST = [("periodic", "dft", I.psf_motion(7, 0.9)), ("reflective", "dct", I.psf_disk(3)),
           ("rect", "dct", I.psf_gaussian(1.5, 7))]


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("bc,transform,psf", NS_PAST, ids=[c[0] for c in NS_PAST])
def test_ns_past_discrepancy_point_matches_oracle(M, dtype, bc, transform, psf):
    """Algorithm 4-NS run past its discrepancy point with stop = 0 (reading
    c15): from there on alpha_n is kept, and the forward column pass applies
    the weight and the inverse transform itself (no separate inverse pass).
    The iterates, residual norms and the alpha_n history follow the oracle;
    the noise level puts the discrepancy point at iterations 11, 14 and 26."""
    pr = small(bc, "tikh_ns", n=48, psf=psf, alpha=0.05, transform=transform, iters=30, nu=0.05)
    f, st, res, al, be = run_gpu(M, pr, dtype)
    ref = run_oracle(pr)
    assert ref["stop_iter"] is not None and ref["stop_iter"] < 28
    assert st["iter"] == ref["iters"] == 30
    if dtype == "f64":
        assert st["stop_iter"] == ref["stop_iter"]
        assert np.abs(f - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max()
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-9)
        np.testing.assert_allclose(al, ref["alphas"], rtol=1e-8)
    else:
        assert abs(st["stop_iter"] - ref["stop_iter"]) <= 1
        restoration_bars(f, ref, pr)
        np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-3)
        if st["stop_iter"] == ref["stop_iter"]:
            np.testing.assert_allclose(al, ref["alphas"], rtol=1e-3)


def test_config1_fp64_plain(M):
    """Workload 1: 64x64 rectangular FP64, BCCB (DFT), L = 1, 200 iterations."""
    pr = I.config(1)
    f, st, res, al, be = run_gpu(M, pr, "f64")
    ref = run_oracle(pr)
    assert st["iter"] == 200
    assert np.abs(f - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max()
    np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-9)


def restoration_bars(f_gpu, ref, pr):
    t = pr.truth_in_fov()
    rre_g, rre_o = O.rre(f_gpu, t), O.rre(ref["f"], t)
    ps_g, ps_o = O.psnr(f_gpu, t), O.psnr(ref["f"], t)
    assert abs(rre_g - rre_o) <= 1e-3, (rre_g, rre_o)
    assert abs(ps_g - ps_o) <= 0.05, (ps_g, ps_o)
    return rre_g, rre_o


def test_config2_fp32_ns(M):
    """Workload 2: reflective 256x256, 15x15 disk, Algorithm 4-NS (DCT), L = 2,
    discrepancy stop at tau*delta; FP32 with FP64 norms / alpha_n."""
    pr = I.config(2)
    f, st, res, al, be = run_gpu(M, pr, "f32")
    ref = run_oracle(pr)
    assert abs(st["stop_iter"] - ref["stop_iter"]) <= 1
    restoration_bars(f, ref, pr)
    k = min(len(al), len(ref["alphas"]))
    np.testing.assert_allclose(al[:k], ref["alphas"][:k], rtol=1e-3)


def test_config2_fp64_ns(M):
    pr = I.config(2)
    f, st, res, al, be = run_gpu(M, pr, "f64")
    ref = run_oracle(pr)
    assert st["stop_iter"] == ref["stop_iter"]
    assert np.abs(f - ref["f"]).max() <= 1e-8 * np.abs(ref["f"]).max()
    np.testing.assert_allclose(al, ref["alphas"], rtol=1e-8)


@pytest.mark.parametrize("variant", ["rect1", "rect2", "rect3"])
def test_config3_reduced_fp32_bf16(M, variant):
    """Workload 3 at 192x192 for 30 iterations: FP32 transforms and stencils
    with the Bregman variable stored in bf16 (and in FP32 for comparison)."""
    pr = I.config(3, variant=variant, n=192)
    ref = run_oracle(pr, iters=30)
    f32, st, *_ = run_gpu(M, pr, "f32", iters=30)
    restoration_bars(f32, ref, pr)
    fb, st, *_ = run_gpu(M, pr, "f32", z_store="bf16", iters=30)
    t = pr.truth_in_fov()
    assert abs(O.rre(fb, t) - O.rre(ref["f"], t)) <= 5e-3


def test_batch_matches_single(M):
    """Mixed batch (sizes, PSFs, BCs, preconditioners) advanced by one graph
    launch per step equals the problems run one by one (FP64, bit-for-bit
    identical kernels, so up to reduction order: same kernels, same order)."""
    probs = [small("rect", "bccb", n=40, transform="dft", iters=10),
             small("reflective", "tikh_ns", n=48, psf=I.psf_disk(3), transform="dct", iters=10, seed=3),
             small("periodic", "tikh_ns", n=36, psf=I.psf_motion(5, 0.2), iters=10, seed=4),
             small("rect", "bccb", n=60, psf=I.psf_gaussian(1.2, 7), transform="dct", iters=10, seed=5)]
    descs = [dict(psf=p.psf, g=p.g, delta=p.delta, bc=p.bc, precond=p.precond, mu=p.mu,
                  alpha=p.alpha, transform=p.transform, max_iter=p.max_iter) for p in probs]
    b = M.Batch(descs, dtype="f64", levels=2, stop=False, max_iter=10, rect_ns_hybrid=True)
    b.iterate(11)
    for i, p in enumerate(probs):
        ref = run_oracle(p)
        fb = b.result(i)
        assert b.stats(i)["iter"] == 10
        assert np.abs(fb - ref["f"]).max() <= 1e-9 * np.abs(ref["f"]).max(), i
    b.close()


def test_batch_set_data_all_and_result_all(M):
    """The batch-wide upload and download (one synchronisation each) give
    the per-problem calls' iterates bit for bit, and reject bad arguments
    before copying anything."""
    import ctypes
    probs = [small("rect", "bccb", n=40, transform="dft", iters=6),
             small("reflective", "tikh_ns", n=48, psf=I.psf_disk(3), transform="dct", iters=6, seed=3),
             small("periodic", "tikh_ns", n=36, psf=I.psf_motion(5, 0.2), iters=6, seed=4)]
    descs = [dict(psf=p.psf, g=p.g, delta=p.delta, bc=p.bc, precond=p.precond, mu=p.mu,
                  alpha=p.alpha, transform=p.transform) for p in probs]
    # new data: the observations scaled, the noise levels with them
    g2 = [(1.25 * p.g).astype(np.float32) for p in probs]
    d2 = [1.25 * p.delta for p in probs]
    out = []
    for batched in (False, True):
        b = M.Batch(descs, dtype="f32", levels=2, stop=False, max_iter=6)
        if batched:
            b.set_data_all(g2, d2)
        else:
            for i in range(len(probs)):
                b.set_data(i, g2[i], d2[i])
        b.reset()
        b.iterate(7)
        fs = b.result_all() if batched else [b.result(i) for i in range(len(probs))]
        out.append((fs, [b.stats(i) for i in range(len(probs))]))
        if batched:
            # a missing source or a zero delta for a 4-NS problem: MLBA_E_INVAL
            bad = (ctypes.c_void_p * 3)(None, None, None)
            d = (ctypes.c_double * 3)(*d2)
            assert b.lib.mlba_batch_set_data_all(b.h, bad, 0, d) == -1
            gp = [np.ascontiguousarray(x) for x in g2]
            ptrs = (ctypes.c_void_p * 3)(*[x.ctypes.data_as(ctypes.c_void_p) for x in gp])
            assert b.lib.mlba_batch_set_data_all(b.h, ptrs, 0, (ctypes.c_double * 3)(d2[0], 0.0, d2[2])) == -1
            assert b.lib.mlba_batch_result_all(b.h, bad, 0) == -1
            # nothing was changed by the rejected calls
            np.testing.assert_array_equal(b.result(1), fs[1])
        b.close()
    for i in range(len(probs)):
        np.testing.assert_array_equal(out[0][0][i], out[1][0][i])
        assert out[0][1][i] == out[1][1][i]


@pytest.mark.parametrize("dtype", ["f32", "f64"])
def test_two_group_schedule_equals_one_group(M, dtype):
    """The two-group schedule (two groups half a step apart on two streams)
    runs the same kernels on the same data as the one-group schedule: the
    iterates, stop iterations and statistics are bit-identical, also when the
    steps come in several iterate() calls and some problems stop early."""
    probs = [small("rect", "bccb", n=40, transform="dft", iters=9),
             small("reflective", "tikh_ns", n=48, psf=I.psf_disk(3), transform="dct", iters=9, seed=3),
             small("periodic", "tikh_ns", n=36, psf=I.psf_motion(5, 0.2), iters=9, seed=4),
             small("zero", "krylov", n=48, iters=9, alpha=0.05, seed=6),
             small("rect", "none", n=32, iters=9, seed=7),
             small("rect", "bccb", n=60, psf=I.psf_gaussian(1.2, 7), transform="dct", iters=9, seed=5)]
    descs = [dict(psf=p.psf, g=p.g, delta=p.delta, bc=p.bc, precond=p.precond, mu=p.mu,
                  alpha=p.alpha, transform=p.transform,
                  max_iter=3 if i == 1 else p.max_iter) for i, p in enumerate(probs)]
    out = []
    for two in (False, True):
        b = M.Batch(descs, dtype=dtype, levels=2, stop=True, max_iter=9, rect_ns_hybrid=True,
                    two_group=two)
        for k in (1, 3, 2, 4):
            b.iterate(k)
        out.append(([b.result(i) for i in range(len(probs))],
                    [b.stats(i) for i in range(len(probs))]))
        b.close()
    (f1, s1), (f2, s2) = out
    for i in range(len(probs)):
        assert np.array_equal(f1[i], f2[i]), i
        assert s1[i] == s2[i], (i, s1[i], s2[i])
    assert s2[1]["iter"] == 3 and s2[1]["stopped"] == 1


def test_batch_own_stop_rules(M):
    """Each problem of a batch stops on its own discrepancy rule."""
    probs = I.batch_problems(count=6, sizes=(64, 96, 128), max_iter=300)
    descs = [dict(psf=p.psf, g=p.g, delta=p.delta, bc=p.bc, precond=p.precond, mu=p.mu,
                  alpha=p.alpha, max_iter=p.max_iter) for p in probs]
    b = M.Batch(descs, dtype="f32", levels=2, stop=True, max_iter=300)
    b.iterate(301)
    assert b.active() == 0
    for i, p in enumerate(probs):
        ref = run_oracle(p)
        st = b.stats(i)
        if ref["stop_iter"] is not None:
            assert abs(st["stop_iter"] - ref["stop_iter"]) <= 1, (i, st, ref["stop_iter"])
        restoration_bars(b.result(i), ref, p)
    b.close()


@pytest.mark.parametrize("bc,precond,transform,psf,alpha,levels,n", [
    ("periodic", "tikh_ns", "dft", I.psf_motion(7, 0.9), 0.05, 2, 48),
    ("zero", "krylov", "dft", I.psf_motion(7, 0.9), 0.05, 2, 48),
    ("rect", "bccb", "dft", I.psf_motion(7, 0.9), 0.3, 2, 40),
    # L >= 3: z of levels 2.. kept in polyphase order, converted to band-major
    # planes in the blob and back
    ("rect", "bccb", "dft", I.psf_motion(7, 0.9), 0.3, 4, 37),
    ("reflective", "tikh_ns", "dct", I.psf_disk(3), 0.05, 3, 45)])
def test_checkpoint_resume_matches_uninterrupted(M, bc, precond, transform, psf, alpha, levels, n):
    """mlba_get_state after 5 iterations, mlba_set_state into a fresh context,
    5 more iterations: the same f, residual history and alpha_n / beta_n as 10
    uninterrupted iterations (the same kernels run on the same data), and the
    resumed context's z (band-major) equals the one it was saved from."""
    pr = small(bc, precond, n=n, psf=psf, alpha=alpha, transform=transform, iters=10, levels=levels)
    kw = dict(mu=pr.mu, alpha=pr.alpha, levels=pr.levels, max_iter=10, stop=False, gamma=pr.gamma,
              q=pr.q, rho=pr.rho, transform=pr.transform)
    full = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype="f64", **kw)
    full.set_data(pr.g, pr.delta)
    full.iterate(11)
    f_ref = full.result()
    res_ref, al_ref, be_ref = full.history()
    full.close()
    a = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype="f64", **kw)
    a.set_data(pr.g, pr.delta)
    a.iterate(5)
    blob = a.get_state()
    z_saved = a.get_z().cpu().numpy()
    a.close()
    b = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype="f64", **kw)
    b.set_data(pr.g, pr.delta)
    b.set_state(blob)
    assert b.stats()["iter"] == 5
    assert np.array_equal(b.get_z().cpu().numpy(), z_saved)
    b.iterate(6)
    f = b.result()
    res, al, be = b.history()
    b.close()
    assert np.abs(f - f_ref).max() <= 1e-12 * np.abs(f_ref).max()
    np.testing.assert_allclose(res, res_ref, rtol=1e-12)
    np.testing.assert_allclose(al, al_ref, rtol=1e-12)
    assert list(be) == list(be_ref)


def test_set_state_rejects_a_foreign_blob(M):
    pr = small("periodic", "bccb", n=48, transform="dft", alpha=0.05)
    a = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype="f64", mu=pr.mu, alpha=pr.alpha,
                  levels=2, max_iter=10, stop=False)
    a.set_data(pr.g, pr.delta)
    blob = a.get_state()
    b = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype="f64", mu=pr.mu, alpha=pr.alpha,
                  levels=1, max_iter=10, stop=False)
    b.set_data(pr.g, pr.delta)
    with pytest.raises(M.MlbaError):
        b.set_state(blob)
    b.close()
    # same shape, another preconditioner or threshold: the blob would continue
    # a different iteration, so it is refused too
    for kw in (dict(precond="tikh"), dict(mu=2 * pr.mu), dict(alpha=2 * pr.alpha)):
        o = dict(precond=pr.precond, mu=pr.mu, alpha=pr.alpha)
        o.update(kw)
        c = M.Context(pr.psf, pr.n, pr.bc, o["precond"], dtype="f64", mu=o["mu"],
                      alpha=o["alpha"], levels=2, max_iter=10, stop=False, transform="dft")
        c.set_data(pr.g, pr.delta)
        with pytest.raises(M.MlbaError):
            c.set_state(blob)
        c.close()
    a.close()


@pytest.mark.parametrize("dtype", ["f64", "f32"])
def test_nonfinite_data_reports_divergence(M, dtype):
    """Host-side fault injection: a NaN planted in g makes ||r^0|| NaN; the
    device stop rule records MLBA_E_DIVERGED and stops the problem, and later
    steps do nothing."""
    pr = small("reflective", "tikh_ns", n=48, psf=I.psf_disk(3), transform="dct", alpha=0.05)
    g = pr.g.copy()
    g[17, 5] = np.nan
    ctx = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype=dtype, mu=pr.mu, alpha=pr.alpha,
                    levels=2, max_iter=10, stop=True, transform="dct")
    ctx.set_data(g, pr.delta)
    ctx.iterate(5)
    st = ctx.stats()
    assert st["status"] == -5 and st["stopped"] == 1 and st["iter"] == 0
    assert st["nres"] == 1
    ctx.close()


@pytest.mark.parametrize("zs", ["f32", "bf16"])
def test_tile_shapes_give_identical_iterates(M, zs, tmp_path, monkeypatch):
    """Every tile shape the autotuner chooses from computes the same values in
    the same order: forced shapes give bit-identical iterates and statistics,
    and a tuned batch (measured at create, then read back from the on-disk
    cache) equals them too."""
    monkeypatch.setenv("MLBA_TUNE_CACHE", str(tmp_path / "tune.txt"))
    probs = [small("rect", "bccb", n=70, transform="dft", iters=6),
             small("reflective", "tikh_ns", n=100, psf=I.psf_disk(3), transform="dct", iters=6, seed=3),
             small("periodic", "tikh_ns", n=36, psf=I.psf_motion(5, 0.2), iters=6, seed=4)]
    descs = [dict(psf=p.psf, g=p.g, delta=p.delta, bc=p.bc, precond=p.precond, mu=p.mu,
                  alpha=p.alpha, transform=p.transform, max_iter=6) for p in probs]
    runs = []
    kw = dict(dtype="f32", z_store=zs, levels=2, stop=False, max_iter=6, rect_ns_hybrid=True)
    cases = [dict(frame_shape=k) for k in range(8)] + [dict(autotune=2), dict(autotune=1)]
    for extra in cases:
        b = M.Batch(descs, **kw, **extra)
        t = b.tiles()
        if "frame_shape" in extra:
            assert t["frame_shape"] == extra["frame_shape"] and t["how"] == "forced"
        elif extra["autotune"] == 2:
            assert t["how"] == "measured" and t["us"] > 0
        else:
            assert t["how"] == "cache"
        b.iterate(7)
        runs.append(([b.result(i) for i in range(len(probs))], [b.stats(i) for i in range(len(probs))]))
        b.close()
    f0, s0 = runs[0]
    for fk, sk in runs[1:]:
        for i in range(len(probs)):
            assert np.array_equal(f0[i], fk[i]), i
            assert s0[i] == sk[i], i
    assert (tmp_path / "tune.txt").read_text().startswith("frame3 ")
