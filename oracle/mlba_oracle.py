"""Plain FP64 CPU oracle of the preconditioned modified linearized Bregman
algorithm (MLBA) for frame-based deblurring with boundary treatment.

TEST INFRASTRUCTURE ONLY.  This module exists to check the CUDA library
against the paper.  Only the test suite, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import it.
It shares no code with the CUDA path and never imports it.

Everything is float64 numpy, written for readability, not speed: direct
convolution by a loop over PSF taps, the framelet as explicit sparse 1-D filter
matrices applied level by level, library FFT/DCT as the transform step, the
textbook PCG, and a bracketing root finder for the nonstationary parameter.
Where the paper is silent or garbled the reading taken is stated in the
function's docstring (readings c1..c19 of the design notes).

Pins (tests/test_oracle_*.py): dense-matrix brute force of A and A^T built
from the padding definitions of Table 1, the adjoint identity, W^T W = I and
the printed 1-D framelet matrices of Section 6.1, BCCB eigenvalues against the
dense periodic matrix, the DCT diagonalisation of the reflective matrix for a
symmetric PSF, the closed-form soft threshold, the closed-form iterated
Tikhonov sequence (mu = 0, periodic BC), the closed-form first iterate, the
PCG against a dense solve, and the defining equation of alpha_n.
"""
from __future__ import annotations

import math

import numpy as np
import scipy.fft as sfft
import scipy.sparse as sp

BCS = ("zero", "periodic", "reflective", "rect", "antireflective")
PRECONDS = ("none", "bccb", "krylov", "sym", "tikh", "tikh_ns")


# ---------------------------------------------------------------------------
# Section 2: the blurring matrix
# ---------------------------------------------------------------------------

def psf_centre(h: np.ndarray) -> int:
    """Centre index of an odd p x p PSF (reading c17: only odd p)."""
    p = h.shape[0]
    if h.shape != (p, p) or p % 2 == 0:
        raise ValueError("PSF must be square with odd size")
    return (p - 1) // 2


def bc_index(e: np.ndarray, n: int, bc: str) -> np.ndarray:
    """Field-of-view index that the extended index ``e`` copies (Table 1).

    zero: outside pixels are 0 (returned as -1); periodic: e mod n;
    reflective: fliplr/flipud mirror, i.e. e = -1 copies 0, e = n copies n-1,
    repeated with period 2n.
    """
    e = np.asarray(e)
    if bc == "zero":
        return np.where((e >= 0) & (e < n), e, -1)
    if bc == "periodic":
        return np.mod(e, n)
    if bc == "reflective":
        q = np.mod(e, 2 * n)
        return np.where(q < n, q, 2 * n - 1 - q)
    raise ValueError(bc)


def antireflect_1d(f: np.ndarray, c: int, axis: int) -> np.ndarray:
    """Antireflective pad by c along one axis (Section 2.2): outside the left
    edge F(1 - i) = 2 F(1) - F(i + 1), outside the right edge
    F(n + i) = 2 F(n) - F(n - i), i = 1..c (1-based, as printed).  Needs
    c <= n - 1."""
    f = np.moveaxis(f, axis, 0)
    n = f.shape[0]
    if c > n - 1:
        raise ValueError("antireflective pad wider than the image")
    out = np.empty((n + 2 * c,) + f.shape[1:])
    out[c:c + n] = f
    for i in range(1, c + 1):
        out[c - i] = 2.0 * f[0] - f[i]
        out[c + n - 1 + i] = 2.0 * f[n - 1] - f[n - 1 - i]
    return np.moveaxis(out, 0, axis)


def extend(f: np.ndarray, c: int, bc: str) -> np.ndarray:
    """Pad the n x n image by c pixels on every side as in Table 1; the
    antireflective pad of Section 2.2 antireflects the rows first and then
    the columns of the result, which gives the printed corner formulas."""
    if bc == "antireflective":
        return antireflect_1d(antireflect_1d(f, c, 0), c, 1)
    n = f.shape[0]
    idx = bc_index(np.arange(-c, n + c), n, bc)
    ok = idx >= 0
    out = np.zeros((n + 2 * c, n + 2 * c))
    sel = np.where(ok, idx, 0)
    out[:, :] = f[np.ix_(sel, sel)]
    out[~ok, :] = 0.0
    out[:, ~ok] = 0.0
    return out


def blur(f: np.ndarray, h: np.ndarray, bc: str) -> np.ndarray:
    """A f for the model g = A f + eta (Eq. model2 / modeld).

    True convolution (reading c10): (A f)(i, j) = sum_{a,b} H[a,b]
    f_ext(i + c - (a - c) - c, ...) i.e. the PSF entry at offset (dy, dx) from
    its centre multiplies f at (i - dy, j - dx).  ``bc == 'rect'``: f is
    m x m and A is the rectangular n^2 x m^2 'valid' operator A = M A_big of
    Eq. Arect (n = m - p + 1).  Otherwise f is n x n and is first padded by the
    boundary condition of Table 1 (zero / periodic / reflective).
    """
    p = h.shape[0]
    c = psf_centre(h)
    if bc == "rect":
        fe = f
        n = f.shape[0] - p + 1
    else:
        fe = extend(f, c, bc)
        n = f.shape[0]
    out = np.zeros((n, n))
    for a in range(p):
        for b in range(p):
            if h[a, b] != 0.0:
                out += h[a, b] * fe[p - 1 - a:p - 1 - a + n, p - 1 - b:p - 1 - b + n]
    return out


def reblur(t: np.ndarray, h: np.ndarray, bc: str) -> np.ndarray:
    """A' t, the reblurring matrix of Section 2.2: the same boundary condition
    imposed on the PSF rotated by 180 degrees.  With antireflective BCs it
    replaces A^T; with zero and periodic BCs A' = A^T."""
    return blur(t, h[::-1, ::-1], bc)


def blur_adjoint(t: np.ndarray, h: np.ndarray, bc: str) -> np.ndarray:
    """A^T t, the exact transpose of :func:`blur` (reading c11).

    The transpose of the tap loop scatters every tap onto the extended
    (n + p - 1)^2 domain (zero padding then full correlation, Section 2.1);
    for a boundary condition the extended domain is then folded back onto the
    field of view by the transpose of the Table 1 padding (each padded pixel
    adds into the pixel it copied; zero-BC padding is dropped).
    """
    n = t.shape[0]
    p = h.shape[0]
    c = psf_centre(h)
    v = np.zeros((n + p - 1, n + p - 1))
    for a in range(p):
        for b in range(p):
            if h[a, b] != 0.0:
                v[p - 1 - a:p - 1 - a + n, p - 1 - b:p - 1 - b + n] += h[a, b] * t
    if bc == "rect":
        return v
    idx = bc_index(np.arange(-c, n + c), n, bc)
    ok = idx >= 0
    rows = np.zeros((n, n + 2 * c))
    np.add.at(rows, idx[ok], v[ok, :])
    u = np.zeros((n, n))
    np.add.at(u.T, idx[ok], rows.T[ok, :])
    return u


# ---------------------------------------------------------------------------
# Section 6.1: piecewise-linear B-spline tight framelets
# ---------------------------------------------------------------------------

# masks b0, b1, b2 of Section 6.1 as taps at offsets -1, 0, +1 (reading c1)
MASKS = (
    (0.25, 0.5, 0.25),
    (math.sqrt(2.0) / 4.0, 0.0, -math.sqrt(2.0) / 4.0),
    (-0.25, 0.5, -0.25),
)
# band order within a level: (i, j) != (0, 0) lexicographically (reading c2)
HIGH_BANDS = tuple((i, j) for i in range(3) for j in range(3) if (i, j) != (0, 0))


def reflect_half(e: np.ndarray, n: int) -> np.ndarray:
    """Half-sample symmetric extension index (x[-1] = x[0], x[n] = x[n-1])."""
    q = np.mod(e, 2 * n)
    return np.where(q < n, q, 2 * n - 1 - q)


def filter_matrix(k: int, n: int, dilation: int = 1) -> sp.csr_matrix:
    """n x n matrix of mask b_k dilated by ``dilation`` under the reflective
    boundary of Section 6.1: row i holds b_k[t] at column refl(i + t*dilation).
    For dilation 1 this gives the printed B_0 and the printed [-1, 2, -1]
    matrix exactly (reading c1)."""
    rows, cols, vals = [], [], []
    i = np.arange(n)
    for t, w in zip((-1, 0, 1), MASKS[k]):
        if w == 0.0:
            continue
        rows.append(i)
        cols.append(reflect_half(i + t * dilation, n))
        vals.append(np.full(n, w))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(n, n))


def n_bands(levels: int) -> int:
    return 8 * levels + 1


def framelet_analysis(u: np.ndarray, levels: int) -> np.ndarray:
    """W u: the undecimated multilevel framelet transform (reading c2).

    Level l uses the masks dilated by 2^(l-1) on the level-(l-1) low-pass;
    the nine 2-D filters are B_i (rows) x B_j (columns), i.e. B_i X B_j^T.
    Output: (8*levels + 1, N, N) with the eight high-pass bands of level 1,
    then level 2, ..., and the final low-pass band last.
    """
    n = u.shape[0]
    bands = []
    cur = u
    for lev in range(1, levels + 1):
        d = 2 ** (lev - 1)
        b = [filter_matrix(k, n, d) for k in range(3)]
        for i, j in HIGH_BANDS:
            bands.append(np.asarray(b[i] @ cur @ b[j].T))
        cur = np.asarray(b[0] @ cur @ b[0].T)
    bands.append(cur)
    return np.stack(bands)


def framelet_synthesis(x: np.ndarray, levels: int) -> np.ndarray:
    """W^T x, the transpose of :func:`framelet_analysis`."""
    n = x.shape[-1]
    s = x[-1]
    for lev in range(levels, 0, -1):
        d = 2 ** (lev - 1)
        b = [filter_matrix(k, n, d) for k in range(3)]
        acc = np.asarray(b[0].T @ s @ b[0])
        for k, (i, j) in enumerate(HIGH_BANDS):
            acc = acc + np.asarray(b[i].T @ x[(lev - 1) * 8 + k] @ b[j])
        s = acc
    return s


def soft(x: np.ndarray, mu: float) -> np.ndarray:
    """S_mu of Eq. soft: sgn(x) max(|x| - mu, 0), componentwise."""
    return np.sign(x) * np.maximum(np.abs(x) - mu, 0.0)


# ---------------------------------------------------------------------------
# Section 4: preconditioners
# ---------------------------------------------------------------------------

def quadrantally_symmetric(h: np.ndarray, tol: float = 1e-14) -> bool:
    """True when H equals its left-right and up-down flips (Section 4.1)."""
    s = np.abs(h).max()
    return (np.abs(h - h[::-1, :]).max() <= tol * s) and (np.abs(h - h[:, ::-1]).max() <= tol * s)


def symmetrize(h: np.ndarray) -> np.ndarray:
    """H~ of Section 4.3: mean over the four sign flips of the offsets from
    the PSF centre (reading c8)."""
    return 0.25 * (h + h[::-1, :] + h[:, ::-1] + h[::-1, ::-1])


def spectrum_dft(h: np.ndarray, n: int) -> np.ndarray:
    """Eigenvalues of the periodic-BC (BCCB, Strang) matrix C of Section 4.1:
    2-D DFT of the PSF zero-padded to n x n with its centre moved to (0, 0)."""
    c = psf_centre(h)
    p = h.shape[0]
    pad = np.zeros((n, n))
    for a in range(p):
        for b in range(p):
            pad[(a - c) % n, (b - c) % n] += h[a, b]
    return np.fft.fft2(pad)


def spectrum_dct(h: np.ndarray, n: int) -> np.ndarray:
    """Eigenvalues of the reflective-BC matrix of a quadrantally symmetric PSF
    (Section 2.2, Section 4.1): dct2(A e_1) ./ dct2(e_1) with the orthonormal
    2-D DCT-II (reading c9)."""
    e1 = np.zeros((n, n))
    e1[0, 0] = 1.0
    a_e1 = blur(e1, h, "reflective")
    return sfft.dctn(a_e1, type=2, norm="ortho") / sfft.dctn(e1, type=2, norm="ortho")


def ar_transform(n: int) -> np.ndarray:
    """The antireflective transform of Section 2.2 as an n x n matrix: the
    sine vectors sin(j pi i / (n-1)), j = 1..n-2 (zero at both ends), with a
    uniform sampling of the linear functions 1 - i/(n-1) and i/(n-1) as the
    first and last columns (together they span the constant and linear
    functions).  Not orthogonal."""
    i = np.arange(n)[:, None]
    j = np.arange(n)[None, :]
    t = np.sin(j * np.pi * i / (n - 1))
    t[:, 0] = 1.0 - np.arange(n) / (n - 1)
    t[:, n - 1] = np.arange(n) / (n - 1)
    return t


def ar_angles(n: int) -> np.ndarray:
    """Frequency of each column of :func:`ar_transform`: j pi / (n-1) for the
    sine vectors, 0 for the two linear ones."""
    th = np.arange(n) * np.pi / (n - 1)
    th[0] = th[n - 1] = 0.0
    return th


def spectrum_ar(h: np.ndarray, n: int) -> np.ndarray:
    """Eigenvalues of the antireflective matrix of a quadrantally symmetric
    PSF in the basis of :func:`ar_transform` (tensor products in 2-D):
    Lambda(j, k) = sum h(d1, d2) cos(d1 th_j) cos(d2 th_k)."""
    c = psf_centre(h)
    p = h.shape[0]
    th = ar_angles(n)
    lam = np.zeros((n, n))
    for a in range(p):
        for b in range(p):
            if h[a, b] != 0.0:
                lam += h[a, b] * np.outer(np.cos((a - c) * th), np.cos((b - c) * th))
    return lam


class SpectralPrecond:
    """(CC^T + alpha I)^{-1} and C^T (CC^T + alpha I)^{-1} for a C diagonalised
    by the DFT (periodic BC), the DCT (reflective BC, symmetric PSF) or the
    antireflective transform (antireflective BC, symmetric PSF; C^T is then
    the reblurring matrix C' = C, Section 2.2).  The antireflective transform
    is not unitary: forward is its inverse, applied by a dense solve."""

    def __init__(self, h: np.ndarray, n: int, transform: str):
        self.transform = transform
        self.n = n
        if transform == "dft":
            self.lam = spectrum_dft(h, n)
        elif transform == "dct":
            self.lam = spectrum_dct(h, n)
        elif transform == "ar":
            self.lam = spectrum_ar(h, n)
            self.t = ar_transform(n)
            self.tinv = np.linalg.inv(self.t)
        else:
            raise ValueError(transform)
        self.sigma = np.abs(self.lam) ** 2

    def forward(self, r):
        if self.transform == "dft":
            return np.fft.fft2(r) / self.n       # unitary scaling
        if self.transform == "ar":
            return self.tinv @ r @ self.tinv.T
        return sfft.dctn(r, type=2, norm="ortho")

    def inverse(self, rhat):
        if self.transform == "dft":
            return np.real(np.fft.ifft2(rhat * self.n))
        if self.transform == "ar":
            return self.t @ rhat @ self.t.T
        return sfft.idctn(rhat, type=2, norm="ortho")

    def inv(self, r, alpha):
        """(CC^T + alpha I)^{-1} r (Eq. Alg1, Alg3)."""
        return self.inverse(self.forward(r) / (self.sigma + alpha))

    def tikh(self, r, alpha):
        """C^T (CC^T + alpha I)^{-1} r (Eq. Alg4)."""
        return self.inverse(self.forward(r) * np.conj(self.lam) / (self.sigma + alpha))

    def apply_C(self, f):
        return self.inverse(self.forward(f) * self.lam)


def pcg(r, apply_aat, apply_m, alpha, tol=1e-3, max_steps=5):
    """Algorithm 2 inner solve (Section 4.2, Eqs. syscg, psys, bet).

    Preconditioned CG for (A A^T + alpha I) t = r with preconditioner
    M = (CC^T + alpha I)^{-1} and zero initial guess.  Stops after
    beta_n = min(5, beta_tol) steps, beta_tol being the first step at which
    the relative residual of the symmetric system (psys),
    sqrt(r_k^T M r_k / r_0^T M r_0), is <= tol (reading c12).
    Returns (t, beta_n).
    """
    x = np.zeros_like(r)
    res = r.copy()
    zz = apply_m(res)
    rho = float(np.vdot(res, zz))
    rho0 = rho
    if rho0 == 0.0:
        return x, 0
    p = zz.copy()
    steps = 0
    for k in range(1, max_steps + 1):
        q = apply_aat(p) + alpha * p
        a = rho / float(np.vdot(p, q))
        x = x + a * p
        res = res - a * q
        steps = k
        zz = apply_m(res)
        rho_new = float(np.vdot(res, zz))
        if math.sqrt(max(rho_new, 0.0) / rho0) <= tol:
            break
        p = zz + (rho_new / rho) * p
        rho = rho_new
    return x, steps


def ns_qn(resnorm: float, delta: float, q: float, rho: float) -> float:
    """q_n = max{q, 2 rho + (1 + rho)/tau_n}, tau_n = ||r^n|| / delta (Eq. Alg4_rev_7)."""
    tau_n = resnorm / delta
    return max(q, 2.0 * rho + (1.0 + rho) / tau_n)


def ns_tau(rho: float) -> float:
    """tau = (1 + 2 rho)/(1 - 2 rho) of Algorithm 4-NS."""
    return (1.0 + 2.0 * rho) / (1.0 - 2.0 * rho)


ALPHA_FLOOR = 1e-14


def ns_alpha(rhat2: np.ndarray, sigma: np.ndarray, qn: float) -> float:
    """alpha_n solving alpha ||(CC^T + alpha I)^{-1} r|| = q_n ||r||
    (Eq. Alg4_rev_7, reading c13).

    With a unitary transform, ||(CC^T + a I)^{-1} r||^2 = sum |r^_k|^2/(s_k+a)^2
    and ||r||^2 = sum |r^_k|^2, so the equation is
    psi(a) = sum |r^_k|^2 a^2/(s_k+a)^2 = q_n^2 sum |r^_k|^2.  psi increases
    with a, so the root is unique (Remark after Algorithm 4-NS).  It is found
    by bisection on log(a) to a relative bracket of 1e-3 and then by
    safeguarded Newton steps to a relative change below 1e-15.  If even
    a = ALPHA_FLOOR over-shoots the target, ALPHA_FLOOR is returned.
    """
    total = float(rhat2.sum())
    target = qn * qn * total

    def psi(a):
        w = a / (sigma + a)
        return float((rhat2 * w * w).sum())

    def dpsi(a):
        # d psi / d a = sum 2 |r^|^2 a s /(s + a)^3
        return float((rhat2 * 2.0 * a * sigma / (sigma + a) ** 3).sum())

    lo, hi = ALPHA_FLOOR, 1.0
    if psi(lo) >= target:
        return lo
    while psi(hi) < target:
        lo, hi = hi, hi * 16.0
        if hi > 1e30:
            return hi
    while hi / lo > 1.001:
        mid = math.sqrt(lo * hi)
        if psi(mid) < target:
            lo = mid
        else:
            hi = mid
    a = math.sqrt(lo * hi)
    for _ in range(100):
        fa = psi(a) - target
        da = dpsi(a)
        step = fa / da if da > 0 else 0.0
        a_new = a - step
        if not (lo < a_new < hi):
            a_new = 0.5 * (lo + hi)
        if fa < 0:
            lo = max(lo, a)
        else:
            hi = min(hi, a)
        if abs(a_new - a) <= 1e-15 * a:
            a = a_new
            break
        a = a_new
    return a


# ---------------------------------------------------------------------------
# Section 3 / 4 / 5: the iteration
# ---------------------------------------------------------------------------

def choose_transform(h: np.ndarray, precond: str, transform: str, bc: str = "rect") -> str:
    """Diagonalising transform of C (Section 4.1).

    Algorithm 3 uses the DCT of the symmetrised PSF (the antireflective
    transform with antireflective BCs, Section 4.3).  An explicit choice wins
    otherwise.  'auto': with periodic BCs the periodic C equals A and the DFT
    is used; with antireflective BCs the antireflective transform (C = A) for
    a quadrantally symmetric PSF outside 4-NS, the BCCB C (DFT) otherwise, as
    the paper's Examples 3 and 4 do; otherwise the DCT when the PSF is
    quadrantally symmetric (the reflective C approximates A better, Section
    4.1) and the DFT when it is not."""
    if precond == "sym":
        return "ar" if bc == "antireflective" else "dct"
    if transform in ("dft", "dct", "ar"):
        return transform
    if bc == "periodic":
        return "dft"
    if bc == "antireflective":
        # C = A through the antireflective transform for a symmetric PSF
        # (Section 2.2); 4-NS needs a unitary transform for Eq. Alg4_rev_7
        return "ar" if (quadrantally_symmetric(h) and precond != "tikh_ns") else "dft"
    return "dct" if quadrantally_symmetric(h) else "dft"


def mlba(g, h, delta, bc, precond, mu, alpha=0.05, levels=1, max_iter=200,
         stop=True, gamma=1.0 + 1e-15, q=0.5, rho=1e-4, transform="auto",
         rect_ns_hybrid=False, pcg_tol=1e-3, pcg_max=5, formulation="synthesis"):
    """Run the preconditioned MLBA of Eq. MLBA2 in the variant ``precond``.

    - 'none'   : P = I (linearized Bregman, Eq. iterLinBreg with lambda = 1)
    - 'bccb'   : Algorithm 1, z += W A^T (CC^T + alpha I)^{-1} r
    - 'krylov' : Algorithm 2, t from :func:`pcg`, z += W A^T t
    - 'sym'    : Algorithm 3, Q = reflective BC of H~, z += W A^T (QQ^T+alpha I)^{-1} r
    - 'tikh'   : Algorithm 4, z += W C^T (CC^T + alpha I)^{-1} r (BC only)
    - 'tikh_ns': Algorithm 4-NS with alpha_n from Eq. Alg4_rev_7; with
                 ``bc == 'rect'`` (only if ``rect_ns_hybrid``) the Algorithm-1
                 form z += W A^T (CC^T + alpha_n I)^{-1} r with alpha_n floored
                 at ``alpha``, which must satisfy Eq. condconvalg1 (reading c14).

    with x = S_mu(z), f = W^T x, z^0 = x^0 = 0 and r^n = g - A f^n.  With
    antireflective BCs every A^T is the reblurring matrix A' (Section 2.2);
    Algorithm 2 is not defined for them here (the paper finds it of no use
    there, Example 4), nor 4-NS with the antireflective transform, which is
    not unitary (Eq. Alg4_rev_7 is solved in the transform domain).
    Stopping (Eq. discrpr, Eq. Alg4_rev_12): the first n > 0 with
    ||r^n|| <= gamma delta (Algorithms 1-4), or the first n >= 0 with
    ||r^n|| <= tau delta (4-NS) (readings c4, c16).  With ``stop=False``
    exactly ``max_iter`` updates run and the iteration at which the rule would
    have fired is recorded (reading c15); past that point 4-NS keeps alpha_n
    at its last value.

    ``formulation='balanced'``: the balanced approach the paper names as the
    other home of its preconditioners (Section 1; Conclusions), in its
    proximal form x^{n+1} = S_mu(W (W^T x^n + u^n)) with u^n the same
    preconditioned correction (A^T P r^n, or C^T (CC^T + alpha I)^{-1} r^n),
    f = W^T x; z holds W (f^n + u^n).  (The analysis approach written as a
    linearized Bregman iteration, z += u, f = W^T S_mu(W z), is Eq. MLBA2
    after the change of variable z <- W z, so it needs no separate form.)

    Returns a dict: f (restoration), z, iters (updates done), stop_iter,
    resnorms (||r^0|| .. ||r^iters||), alphas, betas.
    """
    if bc not in BCS or precond not in PRECONDS or formulation not in ("synthesis", "balanced"):
        raise ValueError((bc, precond, formulation))
    n = g.shape[0]
    p = h.shape[0]
    nf = n + p - 1 if bc == "rect" else n
    if precond in ("tikh", "tikh_ns") and bc == "rect" and not (precond == "tikh_ns" and rect_ns_hybrid):
        raise ValueError("Algorithm 4 needs a square A (Section 5)")
    if bc == "antireflective" and precond == "krylov":
        raise ValueError("Algorithm 2 is not defined for antireflective BCs here")
    adj = (lambda v: reblur(v, h, bc)) if bc == "antireflective" else (lambda v: blur_adjoint(v, h, bc))
    ns = precond == "tikh_ns"
    tr = choose_transform(h, precond, transform, bc)
    if tr == "ar" and (bc != "antireflective" or precond == "tikh_ns"):
        raise ValueError("the antireflective transform serves antireflective BCs outside 4-NS")
    pre = None
    if precond in ("bccb", "krylov", "tikh", "tikh_ns"):
        pre = SpectralPrecond(h, n, tr)
    elif precond == "sym":
        pre = SpectralPrecond(symmetrize(h), n, tr)
    tau = ns_tau(rho)

    B = n_bands(levels)
    z = np.zeros((B, nf, nf))
    f = np.zeros((nf, nf))
    resnorms, alphas, betas = [], [], []
    stop_iter = None
    alpha_n = alpha
    it = 0
    while True:
        r = g - blur(f, h, bc)
        rn = float(np.linalg.norm(r))
        resnorms.append(rn)
        crossed = (rn <= tau * delta) if ns else (it > 0 and rn <= gamma * delta)
        if crossed and stop_iter is None:
            stop_iter = it
        if stop and crossed:
            break
        if it >= max_iter:
            break
        if precond == "none":
            u = adj(r)
        elif precond in ("bccb", "sym"):
            u = adj(pre.inv(r, alpha))
        elif precond == "krylov":
            t, beta = pcg(r, lambda v: blur(blur_adjoint(v, h, bc), h, bc),
                          lambda v: pre.inv(v, alpha), alpha, pcg_tol, pcg_max)
            betas.append(beta)
            u = adj(t)
        elif precond == "tikh":
            u = pre.tikh(r, alpha)
        else:  # tikh_ns
            if not (rn <= tau * delta):
                qn = ns_qn(rn, delta, q, rho)
                rhat = pre.forward(r)
                alpha_n = ns_alpha(np.abs(rhat) ** 2, pre.sigma, qn)
                if bc == "rect":
                    alpha_n = max(alpha_n, alpha)
            alphas.append(alpha_n)
            if bc == "rect":
                u = adj(pre.inv(r, alpha_n))
            else:
                u = pre.tikh(r, alpha_n)
        if formulation == "balanced":
            z = framelet_analysis(f + u, levels)
        else:
            z = z + framelet_analysis(u, levels)
        f = framelet_synthesis(soft(z, mu), levels)
        it += 1
    return {"f": f, "z": z, "iters": it, "stop_iter": stop_iter,
            "resnorms": resnorms, "alphas": alphas, "betas": betas}


def rre(f_est: np.ndarray, f_true: np.ndarray) -> float:
    """Relative restoration error ||f - f~|| / ||f||."""
    return float(np.linalg.norm(f_est - f_true) / np.linalg.norm(f_true))


def psnr(f_est: np.ndarray, f_true: np.ndarray) -> float:
    """PSNR of Section 6 with peak 1 instead of 255 (reading c6):
    20 log10(N / ||f - f~||) for N x N images."""
    nn = f_true.shape[0]
    return 20.0 * math.log10(nn / np.linalg.norm(f_est - f_true))
