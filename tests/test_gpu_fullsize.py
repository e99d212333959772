"""GPU parity at the full sizes of the measured workloads, in the launch
configuration the benchmark times (FP32, L = 2, one graph launch per step).

- The 64-problem batch (sizes up to 1024^2): the whole batch advances
  together; sampled problems of every kind (periodic / reflective 4-NS,
  rectangular Algorithm 1, Algorithm 3, smallest and largest sizes) are
  compared with the FP64 oracle run on its own for the same iterations.
- 1024^2 rectangular motion blur (Rect1 / Rect2 / Rect3, FP32 and BF16 z):
  a few iterations against the oracle.
- 4096^2 rectangular Gaussian with the nonstationary alpha_n (hybrid): the
  oracle's full loop is far too slow at this size, so the first iterate is
  checked on sampled windows the oracle computes one by one.  Everything in
  f^1 = W^T S_mu(W A^T (CC^T + alpha_0 I)^{-1} g) is local except the
  preconditioner and alpha_0, which the oracle computes on the whole image
  with library transforms; A^T and the framelets run on windows with a
  margin wider than their reach (A^T: 2c, one framelet step: 6 pixels).
  The forward blur is checked the same way on a random image.
"""
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


def oracle_run(pr, iters):
    return O.mlba(pr.g, pr.psf, pr.delta, pr.bc, pr.precond, pr.mu, pr.alpha, pr.levels, iters,
                  stop=False, gamma=pr.gamma, q=pr.q, rho=pr.rho, transform=pr.transform,
                  rect_ns_hybrid=pr.rect_ns_hybrid)


def test_batch64_full_size_sampled(M):
    import bench
    probs = bench.problems_for_rank(0)
    iters = 3
    b = M.Batch(bench.descs(probs), dtype="f32", levels=2, stop=False, max_iter=iters,
                rect_ns_hybrid=True)
    b.iterate(iters + 1)
    # one problem of each kind, the smallest and the largest sizes
    kinds = {}
    for i, p in enumerate(probs):
        kinds.setdefault((p.bc, p.precond), []).append(i)
    sample = {max(ix, key=lambda i: probs[i].n) for ix in kinds.values()}
    sample.add(min(range(len(probs)), key=lambda i: probs[i].n))
    for i in sorted(sample):
        p = probs[i]
        ref = oracle_run(p, iters)
        st = b.stats(i)
        assert st["iter"] == iters, (i, st)
        f = b.result(i).astype(np.float64)
        scale = np.abs(ref["f"]).max()
        assert np.abs(f - ref["f"]).max() <= 1e-4 * scale, (i, p.n, p.bc, p.precond)
        np.testing.assert_allclose(st["resnorm"], ref["resnorms"][-1], rtol=1e-5)
        if p.precond == "tikh_ns":
            np.testing.assert_allclose(st["alpha_n"], ref["alphas"][-1], rtol=1e-4)
    b.close()


def test_batch64_over_the_timed_iterations(M):
    """The 64-problem batch exactly as the benchmark runs it (FP32, two-group
    graph schedule, autotuned framelet tile, every problem running its budget
    with the discrepancy point recorded) for 25 steps, the span of a short
    timed run (5 warm-up + 20 timed) during which the alpha_n solves are
    active.  Sampled problems of every kind up to 384^2 are compared with the
    FP64 oracle run for the same 25 iterations: f, the last residual norm and
    alpha_n, the discrepancy point (within one iteration) and the
    restoration bars (RRE within 1e-3, PSNR within 0.05 dB)."""
    import bench
    probs = bench.problems_for_rank(0)
    iters = 25
    b = M.Batch(bench.descs(probs), dtype="f32", levels=2, stop=False, max_iter=iters,
                rect_ns_hybrid=True, autotune=bench.AUTOTUNE)
    b.iterate(iters + 1)
    kinds = {}
    for i, p in enumerate(probs):
        if p.n <= 384:
            kinds.setdefault((p.bc, p.precond), []).append(i)
    sample = set()
    for ix in kinds.values():
        ix = sorted(ix, key=lambda i: (probs[i].n, i))
        sample.update(ix[:2])
        sample.add(ix[-1])
    for i in sorted(sample):
        p = probs[i]
        ref = oracle_run(p, iters)
        st = b.stats(i)
        assert st["iter"] == iters, (i, st)
        f = b.result(i).astype(np.float64)
        scale = np.abs(ref["f"]).max()
        where = (i, p.n, p.bc, p.precond)
        assert np.abs(f - ref["f"]).max() <= 1e-3 * scale, where
        np.testing.assert_allclose(st["resnorm"], ref["resnorms"][-1], rtol=1e-4, err_msg=str(where))
        if ref["stop_iter"] is None:
            assert st["stop_iter"] < 0 or st["stop_iter"] >= iters - 1, where
        else:
            assert abs(st["stop_iter"] - ref["stop_iter"]) <= 1, where
        if p.precond == "tikh_ns":
            if ref["stop_iter"] is None:
                np.testing.assert_allclose(st["alpha_n"], ref["alphas"][-1], rtol=1e-3,
                                           err_msg=str(where))
            elif st["stop_iter"] == ref["stop_iter"]:
                # past the discrepancy point alpha_n is the one kept from the
                # iteration before it, where tau_n -> tau and q_n -> 1: the
                # root of Eq. Alg4_rev_7 is ill-conditioned there (a relative
                # change of 1e-6 in ||r|| moved it by ~3e-3 in these runs)
                np.testing.assert_allclose(st["alpha_n"], ref["alphas"][-1], rtol=2e-2,
                                           err_msg=str(where))
        t = p.truth_in_fov()
        assert abs(O.rre(f, t) - O.rre(ref["f"], t)) <= 1e-3, where
        assert abs(O.psnr(f, t) - O.psnr(ref["f"], t)) <= 0.05, where
    b.close()


@pytest.mark.parametrize("variant,z_store", [("rect1", None), ("rect2", None), ("rect3", None),
                                             ("rect1", "bf16")])
def test_config3_full_size(M, variant, z_store):
    """1024^2 rectangular, 21x21 motion blur, L = 2: FP32 (and BF16 z) against
    the FP64 oracle after a few iterations."""
    pr = I.config(3, variant=variant)
    iters = 2 if variant == "rect2" else 3
    ctx = M.Context(pr.psf, pr.n, pr.bc, pr.precond, dtype="f32", z_store=z_store, mu=pr.mu,
                    alpha=pr.alpha, levels=pr.levels, max_iter=iters, stop=False, gamma=pr.gamma,
                    q=pr.q, rho=pr.rho, transform=pr.transform)
    ctx.set_data(pr.g, pr.delta)
    ctx.run(iters)
    f = ctx.result().astype(np.float64)
    res, al, be = ctx.history()
    ctx.close()
    ref = oracle_run(pr, iters)
    scale = np.abs(ref["f"]).max()
    # BF16 z keeps 8 significant bits per coefficient: unit roundoff 2^-8
    tol = 1e-4 if z_store is None else 1e-2
    assert np.abs(f - ref["f"]).max() <= tol * scale
    np.testing.assert_allclose(res, ref["resnorms"], rtol=1e-5 if z_store is None else 2.0 ** -8)
    if variant == "rect2":
        assert list(be) == ref["betas"]


def _spectrum_dct_windowed(h, n):
    """The oracle's DCT eigenvalues, dct2(A e1) ./ dct2(e1), with A e1 formed on
    a 2p x 2p corner: e1 and its reflective extension are supported within
    the PSF radius of the corner, so the far edges do not enter (n >= 2p)."""
    from scipy import fft as sfft
    p = h.shape[0]
    m = 2 * p
    e = np.zeros((m, m))
    e[0, 0] = 1.0
    corner = O.blur(e, h, "reflective")[:p, :p]
    a_e1 = np.zeros((n, n))
    a_e1[:p, :p] = corner
    e1 = np.zeros((n, n))
    e1[0, 0] = 1.0
    return sfft.dctn(a_e1, type=2, norm="ortho") / sfft.dctn(e1, type=2, norm="ortho")


def test_config5_first_iterate_windows(M):
    """4096^2 rectangular, 31x31 Gaussian, NS alpha (hybrid), L = 2, FP32."""
    pr = I.config(5)
    n, h = pr.n, pr.psf
    p = h.shape[0]
    c = (p - 1) // 2
    nf = n + p - 1
    ctx = M.Context(h, n, "rect", "tikh_ns", dtype="f32", mu=pr.mu, alpha=pr.alpha, levels=2,
                    max_iter=1, stop=False, gamma=pr.gamma, q=pr.q, rho=pr.rho, transform="dct",
                    rect_ns_hybrid=True)
    ctx.set_data(pr.g, pr.delta)
    ctx.run(1)
    f1 = ctx.result().astype(np.float64)
    res, al, _ = ctx.history()
    # forward blur of a random image on the same context
    rng = np.random.default_rng(55)
    fr = rng.random((nf, nf)).astype(np.float32)
    af = ctx.blur(fr).astype(np.float64)
    ctx.close()

    # whole-image pieces: ||r^0|| = ||g||, alpha_0, t = (CC^T + alpha_0 I)^{-1} g
    g = pr.g.astype(np.float64)
    rn = float(np.linalg.norm(g))
    np.testing.assert_allclose(res[0], rn, rtol=1e-5)
    lam = _spectrum_dct_windowed(h, n)
    sigma = lam ** 2
    from scipy import fft as sfft
    ghat = sfft.dctn(g, type=2, norm="ortho")
    qn = O.ns_qn(rn, pr.delta, pr.q, pr.rho)
    a0 = max(O.ns_alpha(ghat ** 2, sigma, qn), pr.alpha)
    np.testing.assert_allclose(al[0], a0, rtol=1e-4)
    t = sfft.idctn(ghat / (sigma + a0), type=2, norm="ortho")

    w, mg = 64, 8
    for (y0, x0) in [(0, 0), (1900, 2300), (nf - w, nf - w)]:
        # u = A^T t on [u0, u1)^2 needs t on [u0 - 2c, u1) (zero outside the image)
        u0y, u1y = max(0, y0 - mg), min(nf, y0 + w + mg)
        u0x, u1x = max(0, x0 - mg), min(nf, x0 + w + mg)
        assert u1y - u0y == u1x - u0x            # square windows for the framelets
        t0y, t1y = max(0, u0y - 2 * c), min(n, u1y)
        t0x, t1x = max(0, u0x - 2 * c), min(n, u1x)
        tc = np.zeros((u1y - u0y + 2 * c, u1x - u0x + 2 * c))
        tc[t0y - (u0y - 2 * c):t1y - (u0y - 2 * c), t0x - (u0x - 2 * c):t1x - (u0x - 2 * c)] = \
            t[t0y:t1y, t0x:t1x]
        # the full correlation of the padded crop; its entries 2c.. are the
        # global u on [u0, u1)
        uc = O.blur_adjoint(tc, h, "rect")[2 * c:2 * c + (u1y - u0y), 2 * c:2 * c + (u1x - u0x)]
        # framelet step on the window: exact where the window edge is the image
        # edge (same half-sample reflection), and at least 6 pixels inside elsewhere
        fw = O.framelet_synthesis(O.soft(O.framelet_analysis(uc, 2), pr.mu), 2)
        sy, sx = y0 - u0y, x0 - u0x
        ref = fw[sy:sy + w, sx:sx + w]
        got = f1[y0:y0 + w, x0:x0 + w]
        assert np.abs(got - ref).max() <= 1e-4 * max(np.abs(ref).max(), 1e-30), (y0, x0)
        # forward blur: valid convolution of the (w + p - 1)^2 crop of f
        if y0 + w <= n and x0 + w <= n:
            ref_a = O.blur(fr[y0:y0 + w + p - 1, x0:x0 + w + p - 1].astype(np.float64), h, "rect")
            assert np.abs(af[y0:y0 + w, x0:x0 + w] - ref_a).max() <= 1e-5 * np.abs(ref_a).max()


def test_config5_alpha_n_root_after_several_steps(M):
    """4096^2 workload, alpha_n at a later iteration.  The oracle's loop is far
    too slow at this size, so this checks a property that holds at any size:
    the alpha_n the device chose at iteration k is the root of Eq. Alg4_rev_7
    for the residual r^k = g - A f^k of its own iterate (Algorithm 4-NS):
        alpha^2 sum w |r^|^2 / (sigma + alpha)^2 = q_k^2 sum w |r^|^2,
    q_k = max{q, 2 rho + (1 + rho)/tau_k}, tau_k = ||r^k|| / delta, with the
    orthonormal DCT and sigma the squared eigenvalues of the reflective
    matrix of the symmetric PSF; the rectangular hybrid floors it at alpha.
    r^k is formed here in FP64 from the device's f^k (valid convolution)."""
    from scipy import fft as sfft
    from scipy import signal
    pr = I.config(5)
    n, h = pr.n, pr.psf
    k = 5
    ctx = M.Context(h, n, "rect", "tikh_ns", dtype="f32", mu=pr.mu, alpha=pr.alpha, levels=2,
                    max_iter=k + 1, stop=False, gamma=pr.gamma, q=pr.q, rho=pr.rho,
                    transform="dct", rect_ns_hybrid=True)
    ctx.set_data(pr.g, pr.delta)
    ctx.iterate(k)
    fk = ctx.result().astype(np.float64)
    ctx.iterate(1)
    res, al, _ = ctx.history()
    ctx.close()
    assert len(al) >= k + 1
    r = pr.g.astype(np.float64) - signal.fftconvolve(fk, h, mode="valid")
    rn = float(np.linalg.norm(r))
    np.testing.assert_allclose(res[k], rn, rtol=1e-5)
    tau = rn / pr.delta
    qk = max(pr.q, 2 * pr.rho + (1 + pr.rho) / tau)
    sigma = _spectrum_dct_windowed(h, n) ** 2
    pw = sfft.dctn(r, type=2, norm="ortho") ** 2
    P = pw.sum()

    def h_and_slope(a):
        x = a / (sigma + a)
        return (pw * x * x).sum() / P - qk * qk, 2.0 * (pw * x * x * (1 - x)).sum() / P

    a = al[k]
    hv, d = h_and_slope(a)
    if a > pr.alpha * (1 + 1e-6):
        # |log alpha - log root| ~ |h| / h' (h increases with log alpha)
        assert abs(hv) / d <= 1e-4, (a, hv, d)
    else:
        # floored: the root lies at or below the floor
        assert a == pytest.approx(pr.alpha, rel=1e-6) and hv >= -1e-4 * d, (a, hv, d)
