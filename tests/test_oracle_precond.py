"""Pins of the oracle's preconditioners (Sections 4 and 5)."""
import math

import numpy as np
import pytest

import mlba_inputs as I
from oracle import mlba_oracle as O
from test_oracle_blur import dense_blur_matrix


def dct_matrix(n):
    """Orthonormal DCT-II from its cosine definition."""
    k = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    d = np.sqrt(2.0 / n) * np.cos(np.pi * k * (2 * j + 1) / (2 * n))
    d[0] /= np.sqrt(2.0)
    return d


def test_bccb_eigenvalues_are_dft_of_padded_psf():
    """Section 2.2 / 4.1: the periodic-BC matrix is diagonalised by the 2-D
    DFT; its eigenvalue for the Fourier mode k is the spectrum entry."""
    h = I.psf_motion(5, 0.9)
    n = 8
    c = dense_blur_matrix(h, n, "periodic")
    lam = O.spectrum_dft(h, n)
    yy, xx = np.mgrid[0:n, 0:n]
    for k1 in range(n):
        for k2 in range(n):
            v = np.exp(2j * np.pi * (k1 * yy + k2 * xx) / n).ravel()
            np.testing.assert_allclose(c @ v, lam[k1, k2] * v, atol=1e-13)


def test_reflective_matrix_diagonalised_by_dct():
    """Section 2.2: reflective BC with a quadrantally symmetric PSF is
    D^T diag(Lambda) D with D the orthonormal 2-D DCT-II."""
    h = I.psf_disk(2)
    n = 9
    a = dense_blur_matrix(h, n, "reflective")
    d1 = dct_matrix(n)
    d = np.kron(d1, d1)
    diag = d @ a @ d.T
    lam = O.spectrum_dct(h, n)
    np.testing.assert_allclose(diag, np.diag(lam.ravel()), atol=1e-13)
    # closed form: Lambda(k1,k2) = sum_h h(dy,dx) cos(pi k1 dy/n) cos(pi k2 dx/n)
    p = h.shape[0]
    cc = (p - 1) // 2
    k = np.arange(n)
    closed = np.zeros((n, n))
    for a_ in range(p):
        for b_ in range(p):
            closed += h[a_, b_] * np.outer(np.cos(np.pi * k * (a_ - cc) / n),
                                           np.cos(np.pi * k * (b_ - cc) / n))
    np.testing.assert_allclose(lam, closed, atol=1e-13)


@pytest.mark.parametrize("transform,bc,psf", [
    ("dft", "periodic", I.psf_motion(5, 0.3)),
    ("dct", "reflective", I.psf_gaussian(1.1, 5)),
])
def test_spectral_precond_matches_dense(transform, bc, psf):
    n = 8
    c = dense_blur_matrix(psf, n, bc)
    pre = O.SpectralPrecond(psf, n, transform)
    alpha = 0.07
    rng = np.random.default_rng(2)
    r = rng.standard_normal((n, n))
    m = np.linalg.inv(c @ c.T + alpha * np.eye(n * n))
    np.testing.assert_allclose(pre.inv(r, alpha).ravel(), m @ r.ravel(), atol=1e-12)
    np.testing.assert_allclose(pre.tikh(r, alpha).ravel(), c.T @ m @ r.ravel(), atol=1e-12)
    np.testing.assert_allclose(pre.apply_C(r).ravel(), c @ r.ravel(), atol=1e-12)


def test_symmetrize():
    """Section 4.3: H~ is quadrantally symmetric, equals H for a symmetric H,
    and is the Frobenius-nearest quadrantally symmetric PSF (orthogonal
    projection: H - H~ is orthogonal to every symmetric S)."""
    h = I.psf_motion(7, 0.4)
    hs = O.symmetrize(h)
    assert O.quadrantally_symmetric(hs)
    assert not O.quadrantally_symmetric(h)
    g = I.psf_gaussian(1.2, 7)
    np.testing.assert_allclose(O.symmetrize(g), g, atol=1e-16)
    rng = np.random.default_rng(0)
    s = O.symmetrize(rng.standard_normal((7, 7)))
    assert abs(np.vdot(h - hs, s)) < 1e-15
    assert abs(hs.sum() - 1.0) < 1e-14


def test_pcg_against_dense_solve():
    """Section 4.2: PCG with enough steps solves (A A^T + alpha I) t = r."""
    h = I.psf_motion(5, 1.3)
    n = 7
    a = dense_blur_matrix(h, n, "rect")
    alpha = 0.02
    pre = O.SpectralPrecond(h, n, "dft")
    rng = np.random.default_rng(4)
    r = rng.standard_normal((n, n))
    t, steps = O.pcg(r, lambda v: O.blur(O.blur_adjoint(v, h, "rect"), h, "rect"),
                     lambda v: pre.inv(v, alpha), alpha, tol=1e-14, max_steps=200)
    exact = np.linalg.solve(a @ a.T + alpha * np.eye(n * n), r.ravel())
    np.testing.assert_allclose(t.ravel(), exact, atol=1e-10)
    assert 1 <= steps <= n * n
    # the cap beta_n <= 5 of Eq. bet
    _, capped = O.pcg(r, lambda v: O.blur(O.blur_adjoint(v, h, "rect"), h, "rect"),
                      lambda v: pre.inv(v, alpha), alpha, tol=1e-14, max_steps=5)
    assert capped == 5


def test_pcg_one_step_when_preconditioner_exact():
    """With periodic BC, A = C and the preconditioner is exact: one step."""
    h = I.psf_motion(5, 1.3)
    n = 10
    alpha = 0.03
    pre = O.SpectralPrecond(h, n, "dft")
    rng = np.random.default_rng(6)
    r = rng.standard_normal((n, n))
    t, steps = O.pcg(r, lambda v: O.blur(O.blur_adjoint(v, h, "periodic"), h, "periodic"),
                     lambda v: pre.inv(v, alpha), alpha)
    assert steps == 1
    np.testing.assert_allclose(t, pre.inv(r, alpha), atol=1e-12)


def test_ns_parameters():
    """Algorithm 4-NS: tau = (1+2rho)/(1-2rho); q_n in [q, 1) while
    ||r|| > tau delta."""
    rho, q = 1e-4, 0.5
    tau = O.ns_tau(rho)
    assert abs(tau - (1 + 2e-4) / (1 - 2e-4)) < 1e-16
    for tn in (tau * 1.0000001, 1.01, 1.5, 2.0, 10.0, 1e6):
        qn = O.ns_qn(tn * 3.0, 3.0, q, rho)
        assert q <= qn < 1.0
    assert O.ns_qn(1e9, 1.0, q, rho) == q


@pytest.mark.parametrize("transform,bc", [("dft", "periodic"), ("dct", "reflective")])
def test_ns_alpha_solves_defining_equation(transform, bc):
    """Eq. Alg4_rev_7 in the image domain with the dense C:
    alpha ||(CC^T + alpha I)^{-1} r|| = q_n ||r||."""
    h = I.psf_gaussian(1.4, 5)
    n = 8
    c = dense_blur_matrix(h, n, bc)
    pre = O.SpectralPrecond(h, n, transform)
    rng = np.random.default_rng(8)
    r = rng.standard_normal((n, n))
    for qn in (0.5, 0.8, 0.99):
        a = O.ns_alpha(np.abs(pre.forward(r)) ** 2, pre.sigma, qn)
        m = np.linalg.inv(c @ c.T + a * np.eye(n * n))
        lhs = a * np.linalg.norm(m @ r.ravel())
        assert abs(lhs - qn * np.linalg.norm(r)) <= 1e-12 * np.linalg.norm(r)
    # unique root, increasing in q_n
    a1 = O.ns_alpha(np.abs(pre.forward(r)) ** 2, pre.sigma, 0.6)
    a2 = O.ns_alpha(np.abs(pre.forward(r)) ** 2, pre.sigma, 0.7)
    assert a2 > a1


def test_convergence_condition_workload_1():
    """Eq. condconvalg1: ||K^T (CC^T+alpha I)^{-1} K|| < 1 at the alpha used by
    the 64x64 rectangular FP64 workload (W^T W = I so the norm is that of
    A^T P A).  Power iteration."""
    pr = I.config(1)
    pre = O.SpectralPrecond(pr.psf, pr.n, "dft")
    rng = np.random.default_rng(0)
    v = rng.standard_normal((pr.nf, pr.nf))
    lam = 0.0
    for _ in range(150):
        w = O.blur_adjoint(pre.inv(O.blur(v, pr.psf, "rect"), pr.alpha), pr.psf, "rect")
        lam = np.linalg.norm(w) / np.linalg.norm(v)
        v = w / np.linalg.norm(w)
    assert lam < 1.0


def test_convergence_condition_batch_workload():
    """Eq. condconvalg1 at the alpha of the batched workload for every
    rectangular problem's PSF (checked at n = 48: the norm depends on the PSF
    and the transform, hardly on n)."""
    probs = I.batch_problems()
    rng = np.random.default_rng(1)
    seen = set()
    for p in probs:
        if p.bc != "rect":
            continue
        key = (p.psf.shape[0], round(float(p.psf.sum() * 1e6 + p.psf[0, 0] * 1e9), 3))
        if key in seen:
            continue
        seen.add(key)
        tr = O.choose_transform(p.psf, "bccb", "auto")
        pre = O.SpectralPrecond(p.psf, 48, tr)
        m = 48 + p.psf.shape[0] - 1
        v = rng.standard_normal((m, m))
        lam = 0.0
        for _ in range(40):
            w = O.blur_adjoint(pre.inv(O.blur(v, p.psf, "rect"), p.alpha), p.psf, "rect")
            lam = np.linalg.norm(w) / np.linalg.norm(v)
            v = w / np.linalg.norm(w)
        assert lam < 0.95, (p.name, lam)


def _dense_precond(h, n, alpha):
    """M = (CC^T + alpha I)^{-1} as a dense matrix, C the periodic-BC matrix
    of h, built from the unitary 2-D DFT matrix and the spectrum (Section 4.1)."""
    f1 = np.fft.fft(np.eye(n)) / math.sqrt(n)
    f2 = np.kron(f1, f1)
    lam = O.spectrum_dft(h, n).ravel()
    return np.real(f2.conj().T @ np.diag(1.0 / (np.abs(lam) ** 2 + alpha)) @ f2)


def _galerkin_pcg_iterates(a, m, alpha, r, kmax):
    """The k-th PCG iterate without the CG recurrence: the Galerkin solution
    of (A A^T + alpha I) x = r over the Krylov space spanned by
    (M S)^j M r, j < k (S = A A^T + alpha I), which is the minimiser of the
    S-norm error there.  Returns, per k, the iterate and both relative
    residual norms: the preconditioned sqrt(r_k^T M r_k / r_0^T M r_0) and
    the plain ||r_k|| / ||r_0||."""
    s = a @ a.T + alpha * np.eye(a.shape[0])
    r0 = r.ravel()
    m0 = r0 @ m @ r0
    basis = [m @ r0]
    out = []
    for _ in range(kmax):
        v, _ = np.linalg.qr(np.stack(basis, axis=1))
        x = v @ np.linalg.solve(v.T @ s @ v, v.T @ r0)
        rk = r0 - s @ x
        out.append((x, math.sqrt(rk @ m @ rk / m0), np.linalg.norm(rk) / np.linalg.norm(r0)))
        basis.append(m @ s @ basis[-1])
    return out


PCG_STOP_CASE = dict(h=np.array([[0.0, 0.1, 0.05], [0.2, 0.3, 0.0], [0.15, 0.1, 0.1]]),
                     n=16, bc="zero", alpha=0.1, tol=1e-2, seed=4)


def test_pcg_stops_on_preconditioned_relative_residual():
    """Section 4.2 (Eqs. psys, bet; reading c12): beta_n is the first step
    at which sqrt(r_k^T M r_k / r_0^T M r_0) <= tol, capped at 5.  The
    expected step and iterate come from dense matrices (Galerkin projection
    on the Krylov space, no CG recurrence).  The case is chosen so that the
    plain criterion ||r_k|| / ||r_0|| <= tol would stop at a later step."""
    cs = PCG_STOP_CASE
    h, n, bc, alpha, tol = cs["h"], cs["n"], cs["bc"], cs["alpha"], cs["tol"]
    a = dense_blur_matrix(h, n, bc)
    m = _dense_precond(h, n, alpha)
    r = np.random.default_rng(cs["seed"]).standard_normal((n, n))
    its = _galerkin_pcg_iterates(a, m, alpha, r, 5)
    k_pre = next(k for k, (_, rel, _) in enumerate(its, 1) if rel <= tol)
    k_plain = next((k for k, (_, _, rel) in enumerate(its, 1) if rel <= tol), 6)
    assert 1 < k_pre < 5 and k_plain != k_pre      # the case discriminates
    pre = O.SpectralPrecond(h, n, "dft")
    t, steps = O.pcg(r, lambda v: O.blur(O.blur_adjoint(v, h, bc), h, bc),
                     lambda v: pre.inv(v, alpha), alpha, tol=tol, max_steps=5)
    assert steps == k_pre
    np.testing.assert_allclose(t.ravel(), its[k_pre - 1][0], atol=1e-10)
    # at the design tolerance 1e-3 the same system runs to the cap of Eq. bet
    t5, steps5 = O.pcg(r, lambda v: O.blur(O.blur_adjoint(v, h, bc), h, bc),
                       lambda v: pre.inv(v, alpha), alpha, tol=1e-3, max_steps=5)
    assert all(rel > 1e-3 for _, rel, _ in its[:4]) and steps5 == 5
    np.testing.assert_allclose(t5.ravel(), its[4][0], atol=1e-10)


@pytest.mark.parametrize("psf", [I.psf_gaussian(1.1, 5), I.psf_disk(2)])
@pytest.mark.parametrize("n", [6, 9])
def test_antireflective_transform_diagonalises_ar_matrix(psf, n):
    """Section 2.2: the antireflective matrix of a quadrantally symmetric PSF
    (dense, NumPy odd-reflection pad; separable Gaussian and non-separable
    disk) equals (T x T) diag(Lambda) (T x T)^{-1} with T the antireflective
    transform and Lambda the cosine symbol at j pi / (n-1) (0 for the two
    linear basis vectors)."""
    a = dense_blur_matrix(psf, n, "antireflective")
    tt = np.kron(O.ar_transform(n), O.ar_transform(n))
    lam = O.spectrum_ar(psf, n)
    np.testing.assert_allclose(tt @ np.diag(lam.ravel()) @ np.linalg.inv(tt), a, atol=1e-13)


def test_antireflective_precond_against_dense():
    """(QQ' + alpha I)^{-1} and Q'(QQ' + alpha I)^{-1} with Q the dense
    antireflective matrix of a symmetric PSF and Q' its reblurring matrix
    (Eq. Alg3 with antireflective BCs, Section 4.3; Eq. Alg4)."""
    h = I.psf_disk(2)
    n, alpha = 8, 0.03
    q = dense_blur_matrix(h, n, "antireflective")
    q_re = dense_blur_matrix(h[::-1, ::-1], n, "antireflective")
    np.testing.assert_allclose(q_re, q, atol=1e-15)          # symmetric PSF: Q' = Q
    pre = O.SpectralPrecond(h, n, "ar")
    r = np.random.default_rng(8).standard_normal((n, n))
    m = q @ q_re + alpha * np.eye(n * n)
    np.testing.assert_allclose(pre.inv(r, alpha).ravel(), np.linalg.solve(m, r.ravel()), atol=1e-11)
    np.testing.assert_allclose(pre.tikh(r, alpha).ravel(), q_re @ np.linalg.solve(m, r.ravel()),
                               atol=1e-11)


def test_alg3_antireflective_symmetric_psf_is_alg1_ar():
    """Section 4.3 with antireflective BCs: for a quadrantally symmetric PSF
    H~ = H, so Algorithm 3 equals Algorithm 1 with the antireflective C."""
    h = I.psf_gaussian(1.2, 5)
    n = 16
    rng = np.random.default_rng(3)
    g = rng.random((n, n))
    a3 = O.mlba(g, h, 1.0, "antireflective", "sym", mu=0.02, alpha=0.2, levels=1, max_iter=4,
                stop=False)
    a1 = O.mlba(g, h, 1.0, "antireflective", "bccb", mu=0.02, alpha=0.2, levels=1, max_iter=4,
                stop=False, transform="ar")
    np.testing.assert_allclose(a3["f"], a1["f"], atol=1e-12)
