"""Pins of the oracle's MLBA loop (Eq. MLBA2, Algorithms 1-4 and 4-NS)."""
import numpy as np
import pytest

import mlba_inputs as I
from oracle import mlba_oracle as O
from test_oracle_blur import dense_blur_matrix
from test_oracle_framelet import dense_w


def small_problem(n=16, bc="periodic", psf=None, seed=11, nu=0.01):
    psf = I.psf_motion(5, 0.8) if psf is None else psf
    p = psf.shape[0]
    f = I.true_image(n + p - 1, seed)
    g, delta = I.observe(f, psf, nu, seed)
    return g, psf, delta


@pytest.mark.parametrize("precond", ["bccb", "tikh"])
def test_mu_zero_periodic_is_iterated_tikhonov(precond):
    """mu = 0, periodic BC, C = A: x = z and W^T W = I turn Algorithms 1 and 4
    into f^{n+1} = f^n + C^T (CC^T + alpha I)^{-1}(g - C f^n), whose closed
    form in the Fourier domain is f^_n = (1 - rho^n) g^/lambda with
    rho = alpha/(|lambda|^2 + alpha) (derived from Eq. MLBA2, Section 4.1)."""
    g, h, delta = small_problem()
    n = g.shape[0]
    alpha, iters = 0.05, 7
    out = O.mlba(g, h, delta, "periodic", precond, mu=0.0, alpha=alpha, levels=2,
                 max_iter=iters, stop=False, transform="dft")
    # independent closed form with a direct DFT of the centred PSF
    c = (h.shape[0] - 1) // 2
    lam = np.zeros((n, n), complex)
    yy, xx = np.mgrid[0:n, 0:n]
    for a in range(h.shape[0]):
        for b in range(h.shape[1]):
            lam += h[a, b] * np.exp(-2j * np.pi * ((a - c) * yy + (b - c) * xx) / n)
    rho = alpha / (np.abs(lam) ** 2 + alpha)
    ghat = np.fft.fft2(g)
    fhat = (1 - rho ** iters) * ghat / lam
    np.testing.assert_allclose(out["f"], np.real(np.fft.ifft2(fhat)), atol=1e-10)


def test_first_iterate_dense():
    """z^1 = W A^T P g and f^1 = W^T S_mu(z^1) with dense A, P, W (Eq. Alg1)."""
    h = I.psf_motion(3, 0.5)
    g, _, delta = small_problem(n=6, psf=h)
    n, p = 6, h.shape[0]
    m = n + p - 1
    alpha, mu, levels = 0.1, 0.02, 1
    out = O.mlba(g, h, delta, "rect", "bccb", mu=mu, alpha=alpha, levels=levels,
                 max_iter=1, stop=False, transform="dft")
    a = dense_blur_matrix(h, n, "rect")
    cper = dense_blur_matrix(h, n, "periodic")
    pmat = np.linalg.inv(cper @ cper.T + alpha * np.eye(n * n))
    w = dense_w(m, levels)
    z1 = w @ (a.T @ (pmat @ g.ravel()))
    f1 = w.T @ O.soft(z1, mu)
    np.testing.assert_allclose(out["z"].ravel(), z1, atol=1e-12)
    np.testing.assert_allclose(out["f"].ravel(), f1, atol=1e-12)
    # and the recorded residual of iterate 1
    r1 = g.ravel() - a @ f1
    assert abs(out["resnorms"][1] - np.linalg.norm(r1)) < 1e-12


def test_discrepancy_stop_rule():
    """Eq. discrpr: stop at the first n > 0 with ||r^n|| <= gamma delta."""
    pr = I.config(2, n=64)
    out = O.mlba(pr.g, pr.psf, pr.delta, "reflective", "tikh", pr.mu, alpha=0.02,
                 levels=2, max_iter=300, stop=True, transform="dct")
    rn = out["resnorms"]
    k = out["stop_iter"]
    assert k is not None and k == out["iters"] and k > 0
    assert rn[k] <= pr.gamma * pr.delta
    assert all(x > pr.gamma * pr.delta for x in rn[1:k])


def test_ns_stop_rule_and_alpha_sequence():
    """Algorithm 4-NS stops at ||r|| <= tau delta (Eq. Alg4_rev_12) and every
    alpha_n solves Eq. Alg4_rev_7 for its own residual."""
    pr = I.config(2, n=64)
    out = O.mlba(pr.g, pr.psf, pr.delta, "reflective", "tikh_ns", pr.mu,
                 levels=2, max_iter=300, stop=True, transform="dct")
    tau = O.ns_tau(pr.rho)
    rn = out["resnorms"]
    k = out["stop_iter"]
    assert rn[k] <= tau * pr.delta and all(x > tau * pr.delta for x in rn[:k])
    assert len(out["alphas"]) == k


def test_ns_may_stop_at_zero():
    """Algorithm 4-NS checks the rule before the first step (n >= 0)."""
    g, h, _ = small_problem(n=12)
    huge = 10 * np.linalg.norm(g)
    out = O.mlba(g, h, huge, "periodic", "tikh_ns", 0.01, levels=1, max_iter=10)
    assert out["iters"] == 0 and out["stop_iter"] == 0
    np.testing.assert_array_equal(out["f"], 0.0)


def test_alg3_symmetric_psf_equals_alg1_dct():
    """Section 6 Example 4: for a symmetric PSF, H~ = H and Alg-Rect3 is
    Alg-Rect1 with the DCT."""
    g, h, delta = small_problem(n=14, psf=I.psf_gaussian(1.0, 5))
    a = O.mlba(g, h, delta, "rect", "sym", 0.02, alpha=0.3, levels=2, max_iter=6, stop=False)
    b = O.mlba(g, h, delta, "rect", "bccb", 0.02, alpha=0.3, levels=2, max_iter=6,
               stop=False, transform="dct")
    np.testing.assert_allclose(a["f"], b["f"], atol=1e-13)


def test_alg2_periodic_equals_alg1():
    """With periodic BC the PCG of Algorithm 2 converges in one step to the
    Algorithm 1 correction."""
    g, h, delta = small_problem(n=12)
    a = O.mlba(g, h, delta, "periodic", "krylov", 0.02, alpha=0.05, levels=1, max_iter=5,
               stop=False, transform="dft")
    b = O.mlba(g, h, delta, "periodic", "bccb", 0.02, alpha=0.05, levels=1, max_iter=5,
               stop=False, transform="dft")
    assert a["betas"] == [1] * 5
    np.testing.assert_allclose(a["f"], b["f"], atol=1e-11)


def test_alg4_with_c_equal_a_is_alg1():
    """Section 5: with C = A (periodic BC) Algorithm 4 is the standard MLBA."""
    g, h, delta = small_problem(n=12)
    a = O.mlba(g, h, delta, "periodic", "tikh", 0.03, alpha=0.05, levels=2, max_iter=5,
               stop=False, transform="dft")
    b = O.mlba(g, h, delta, "periodic", "bccb", 0.03, alpha=0.05, levels=2, max_iter=5,
               stop=False, transform="dft")
    np.testing.assert_allclose(a["f"], b["f"], atol=1e-12)


def test_rect_rejects_alg4():
    g, h, delta = small_problem(n=10)
    with pytest.raises(ValueError):
        O.mlba(g, h, delta, "rect", "tikh", 0.01)


def test_first_iterate_dense_antireflective():
    """Antireflective BCs (Section 2.2): z^1 = W A' P g and the residual of
    iterate 1 with the dense A (NumPy odd-reflection pad) and the dense
    reblurring matrix A' (the same pad on the 180-degree rotated PSF), P the
    BCCB preconditioner (Eq. Alg1)."""
    h = np.array([[0.0, 0.1, 0.05], [0.2, 0.3, 0.0], [0.15, 0.1, 0.1]])
    n = 7
    rng = np.random.default_rng(9)
    g = rng.random((n, n))
    alpha, mu, levels = 0.1, 0.02, 1
    out = O.mlba(g, h, 1.0, "antireflective", "bccb", mu=mu, alpha=alpha, levels=levels,
                 max_iter=1, stop=False, transform="dft")
    a = dense_blur_matrix(h, n, "antireflective")
    a_re = dense_blur_matrix(h[::-1, ::-1], n, "antireflective")
    cper = dense_blur_matrix(h, n, "periodic")
    pmat = np.linalg.inv(cper @ cper.T + alpha * np.eye(n * n))
    w = dense_w(n, levels)
    z1 = w @ (a_re @ (pmat @ g.ravel()))
    f1 = w.T @ O.soft(z1, mu)
    np.testing.assert_allclose(out["z"].ravel(), z1, atol=1e-12)
    np.testing.assert_allclose(out["f"].ravel(), f1, atol=1e-12)
    assert abs(out["resnorms"][1] - np.linalg.norm(g.ravel() - a @ f1)) < 1e-12
    with pytest.raises(ValueError):
        O.mlba(g, h, 1.0, "antireflective", "krylov", mu=mu)


@pytest.mark.parametrize("precond", ["bccb", "tikh"])
def test_balanced_mu_zero_equals_synthesis(precond):
    """With mu = 0 both the synthesis MLBA and the balanced iteration reduce
    to the preconditioned Landweber step f += u (W^T W = I), so they agree."""
    h = I.psf_motion(5, 0.4)
    n = 12
    g = np.random.default_rng(1).random((n, n))
    kw = dict(mu=0.0, alpha=0.1, levels=2, max_iter=5, stop=False, transform="dft")
    a = O.mlba(g, h, 1.0, "periodic", precond, **kw)
    b = O.mlba(g, h, 1.0, "periodic", precond, formulation="balanced", **kw)
    np.testing.assert_allclose(b["f"], a["f"], atol=1e-12)


def test_balanced_second_iterate_dense():
    """Balanced approach: x^1 = S(W A^T P g) (as the synthesis form), then
    x^2 = S(W (W^T x^1 + A^T P (g - A W^T x^1))), with dense A, P, W; the
    synthesis form's second iterate S(W A^T P g + W A^T P r^1) differs."""
    h = I.psf_motion(3, 0.5)
    n = 6
    p = h.shape[0]
    m = n + p - 1
    rng = np.random.default_rng(5)
    g = rng.random((n, n))
    alpha, mu, levels = 0.1, 0.02, 1
    out = O.mlba(g, h, 1.0, "rect", "bccb", mu=mu, alpha=alpha, levels=levels, max_iter=2,
                 stop=False, transform="dft", formulation="balanced")
    a = dense_blur_matrix(h, n, "rect")
    cper = dense_blur_matrix(h, n, "periodic")
    pmat = np.linalg.inv(cper @ cper.T + alpha * np.eye(n * n))
    w = dense_w(m, levels)
    x1 = O.soft(w @ (a.T @ (pmat @ g.ravel())), mu)
    f1 = w.T @ x1
    x2 = O.soft(w @ (f1 + a.T @ (pmat @ (g.ravel() - a @ f1))), mu)
    np.testing.assert_allclose(out["f"].ravel(), w.T @ x2, atol=1e-12)
    syn = O.mlba(g, h, 1.0, "rect", "bccb", mu=mu, alpha=alpha, levels=levels, max_iter=2,
                 stop=False, transform="dft")
    assert np.abs(syn["f"] - out["f"]).max() > 1e-6
