"""Seeded synthetic inputs for the MLBA deblurring workloads.

This module is shared by the tests, the benchmark and the oracle checks.  It
draws random numbers and builds the observed data of the degradation model
g = A f + eta of Section 1 (Eq. model2 / modeld): a true image F of size m x m,
a p x p PSF, and the observed n x n field of view obtained by blurring F and
keeping only the pixels that do not depend on anything outside F (the protocol
of Example 3 in Section 6), plus white Gaussian noise.  It holds none of the
restoration method's arithmetic: the blur of the synthetic truth is done with
SciPy's FFT convolution, a library routine that neither the oracle nor the CUDA
path uses.

The paper's own images (Saturn, Galaxy, Boat, Cameraman) and its RestoreTools
PSFs are not available; seeded piecewise-smooth images and analytic PSFs stand
in for them.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
from scipy.ndimage import convolve as nd_convolve
from scipy.signal import fftconvolve

__all__ = [
    "true_image", "psf_gaussian", "psf_disk", "psf_motion", "observe",
    "Problem", "config", "batch_problems", "CONFIG_NAMES",
]


# ---------------------------------------------------------------------------
# images and PSFs
# ---------------------------------------------------------------------------

def true_image(m: int, seed: int, n_shapes: int = 20) -> np.ndarray:
    """Piecewise-smooth m x m image in [0, 1].

    A random linear ramp scaled to [0, 0.4] plus ``n_shapes`` rectangles and
    disks of constant random intensity in [0, 1]; later shapes overwrite
    earlier ones; the result is clipped to [0, 1].
    """
    rng = np.random.default_rng([seed, 0x1a9e])
    yy, xx = np.mgrid[0:m, 0:m].astype(np.float64) / max(m - 1, 1)
    a, b = rng.uniform(-1.0, 1.0, size=2)
    ramp = a * xx + b * yy
    lo, hi = ramp.min(), ramp.max()
    img = 0.4 * (ramp - lo) / (hi - lo) if hi > lo else np.zeros((m, m))
    for _ in range(n_shapes):
        kind = rng.integers(0, 2)
        cy, cx = rng.uniform(0, m, size=2)
        size = rng.uniform(m / 16.0, m / 4.0)
        val = rng.uniform(0.0, 1.0)
        if kind == 0:
            h, w = size, rng.uniform(m / 16.0, m / 4.0)
            mask = (np.abs(yy * (m - 1) - cy) <= h / 2) & (np.abs(xx * (m - 1) - cx) <= w / 2)
        else:
            mask = (yy * (m - 1) - cy) ** 2 + (xx * (m - 1) - cx) ** 2 <= (size / 2) ** 2
        img[mask] = val
    return np.clip(img, 0.0, 1.0)


def psf_gaussian(sigma: float, p: int | None = None) -> np.ndarray:
    """Centred Gaussian PSF, p = 2*ceil(3 sigma)+1 unless given; sums to 1.

    Built as the outer product of a normalised 1-D Gaussian, so it is exactly
    rank one up to the rounding of the products.
    """
    if p is None:
        p = 2 * int(math.ceil(3.0 * sigma)) + 1
    c = (p - 1) // 2
    t = np.arange(p, dtype=np.float64) - c
    g = np.exp(-(t * t) / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def psf_disk(r: int, p: int | None = None) -> np.ndarray:
    """Out-of-focus disk: indicator of i^2 + j^2 <= r^2, p = 2r+3 unless given."""
    if p is None:
        p = 2 * r + 3
    c = (p - 1) // 2
    t = np.arange(p) - c
    h = ((t[:, None] ** 2 + t[None, :] ** 2) <= r * r).astype(np.float64)
    return h / h.sum()


def psf_motion(length: int, angle: float, p: int | None = None) -> np.ndarray:
    """Linear motion blur of the given length through the centre.

    The segment is sampled at 4*length points and each sample is splatted
    bilinearly onto the grid; p = length (odd) unless given.
    """
    if p is None:
        p = length if length % 2 == 1 else length + 1
    c = (p - 1) / 2.0
    h = np.zeros((p, p))
    ns = 4 * length
    s = np.linspace(-(length - 1) / 2.0, (length - 1) / 2.0, ns)
    ys = c + s * math.sin(angle)
    xs = c + s * math.cos(angle)
    for y, x in zip(ys, xs):
        y0, x0 = int(math.floor(y)), int(math.floor(x))
        fy, fx = y - y0, x - x0
        for dy, wy in ((0, 1 - fy), (1, fy)):
            for dx, wx in ((0, 1 - fx), (1, fx)):
                yy, xx = y0 + dy, x0 + dx
                if 0 <= yy < p and 0 <= xx < p:
                    h[yy, xx] += wy * wx
    return h / h.sum()


def observe(f_true: np.ndarray, psf: np.ndarray, nu: float, seed: int):
    """Observed field of view g (n x n, n = m - p + 1) and noise norm delta.

    g = valid part of the convolution of the m x m truth with the PSF, plus
    eta = nu * ||A f|| * e / ||e|| with e standard normal.  Returns (g, delta)
    with delta = ||eta|| exactly.
    """
    blurred = fftconvolve(f_true, psf, mode="valid")
    rng = np.random.default_rng([seed, 0x5eed])
    e = rng.standard_normal(blurred.shape)
    eta = nu * np.linalg.norm(blurred) * e / np.linalg.norm(e)
    return blurred + eta, float(np.linalg.norm(eta))


def observe_periodic(f_true: np.ndarray, psf: np.ndarray, nu: float, seed: int):
    """Observed n x n image of an n x n truth under periodic boundary
    conditions (the truth repeats outside the field of view), plus noise as
    in :func:`observe`.  Uses SciPy's wrap-mode convolution."""
    blurred = nd_convolve(f_true, psf, mode="wrap")
    rng = np.random.default_rng([seed, 0x5eed])
    e = rng.standard_normal(blurred.shape)
    eta = nu * np.linalg.norm(blurred) * e / np.linalg.norm(e)
    return blurred + eta, float(np.linalg.norm(eta))


def quadrant_symmetric(psf: np.ndarray) -> bool:
    return bool(np.array_equal(psf, psf[::-1, :]) and np.array_equal(psf, psf[:, ::-1]))


# ---------------------------------------------------------------------------
# problem descriptions of the measured workloads
# ---------------------------------------------------------------------------

# boundary treatment and preconditioner names (same integer codes as the C ABI)
BC = {"zero": 0, "periodic": 1, "reflective": 2, "rect": 3}
PRECOND = {"none": 0, "bccb": 1, "krylov": 2, "sym": 3, "tikh": 4, "tikh_ns": 5}
TRANSFORM = {"auto": 0, "dft": 1, "dct": 2}


@dataclass
class Problem:
    """One deblurring problem: data, PSF and the run parameters."""
    g: np.ndarray
    psf: np.ndarray
    delta: float
    bc: str
    precond: str
    mu: float
    alpha: float = 0.05
    levels: int = 1
    transform: str = "auto"
    gamma: float = 1.0 + 1e-15
    q: float = 0.5
    rho: float = 1e-4
    max_iter: int = 200
    stop: bool = True            # False: run max_iter iterations, no early stop
    rect_ns_hybrid: bool = False
    f_true: np.ndarray | None = None
    name: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.g.shape[0]

    @property
    def p(self) -> int:
        return self.psf.shape[0]

    @property
    def nf(self) -> int:
        return self.n + self.p - 1 if self.bc == "rect" else self.n

    def truth_in_fov(self) -> np.ndarray:
        """The part of the truth a restoration is compared with."""
        if self.f_true.shape[0] == self.nf:
            return self.f_true
        c = (self.p - 1) // 2
        return self.f_true[c:c + self.n, c:c + self.n]


def _make(n, psf, nu, seed, **kw):
    p = psf.shape[0]
    m = n + p - 1
    f = true_image(m, seed)
    g, delta = observe(f, psf, nu, seed)
    return Problem(g=g, psf=psf, delta=delta, f_true=f, **kw)


CONFIG_NAMES = {
    1: "plain-fp64 rect 64x64, 9x9 Gaussian, Alg-Rect1 (DFT), L=1, 200 it",
    2: "reflective 256x256, 15x15 disk r=6, Alg-BC4-NS (DCT), L=2",
    3: "rect 1024x1024, 21x21 motion, Alg-Rect1/2/3, L=2, 200 it, bf16 z",
    4: "batch of 64 problems, n in {128..1024}, mixed PSF/BC, L=2",
    5: "rect 4096x4096, 31x31 Gaussian sigma=5, DCT + NS alpha, L=2, 500 it",
}


def config(i: int, variant: str | None = None, n: int | None = None) -> Problem:
    """Single-problem workloads 1, 2, 3 and 5 (``n`` overrides the size)."""
    mu = 10.0 / 255.0
    if i == 1:
        return _make(n or 64, psf_gaussian(2.0, 9), 0.01, 1, bc="rect", precond="bccb",
                     transform="dft", mu=mu, alpha=0.3, levels=1, max_iter=200,
                     stop=False, name="C1")
    if i == 2:
        return _make(n or 256, psf_disk(6, 15), 0.02, 2, bc="reflective",
                     precond="tikh_ns", transform="dct", mu=mu, alpha=0.05, levels=2,
                     max_iter=500, stop=True, name="C2")
    if i == 3:
        rng = np.random.default_rng([3, 0xa76])
        ang = float(rng.uniform(0.0, math.pi))
        psf = psf_motion(21, ang)
        variant = variant or "rect1"
        pc, al = {"rect1": ("bccb", 0.5), "rect2": ("krylov", 0.05),
                  "rect3": ("sym", 0.5)}[variant]
        return _make(n or 1024, psf, 0.01, 3, bc="rect", precond=pc, mu=mu,
                     alpha=al, levels=2, max_iter=200, stop=False,
                     name=f"C3-{variant}")
    if i == 5:
        return _make(n or 4096, psf_gaussian(5.0, 31), 0.01, 5, bc="rect",
                     precond="tikh_ns", transform="dct", mu=mu, alpha=0.05, levels=2,
                     max_iter=500, stop=False, rect_ns_hybrid=True, name="C5")
    raise ValueError(f"no single-problem workload {i}")


BATCH_SIZES = (128, 192, 256, 384, 512, 768, 1024)


def batch_problems(count: int = 64, seed: int = 4, sizes=BATCH_SIZES,
                   max_iter: int = 500) -> list[Problem]:
    """Workload 4: independent problems of mixed size, PSF, BC and noise.

    Sizes uniform in ``sizes``; PSF family uniform over Gaussian sigma~U[1,4],
    disk r~U{2..8}, motion length~U{5,7,..,21} at angle~U[0,pi); BC uniform
    over periodic / reflective / rectangular; noise nu~U[0.005, 0.03].  BC
    problems run the nonstationary Algorithm 4-NS where C = A (periodic BC
    with the DFT; reflective BC with a quadrantally symmetric PSF and the
    DCT), reflective problems with a nonsymmetric PSF run Algorithm 3
    (symmetrised PSF, alpha = 0.3), rectangular ones the BCCB-preconditioned
    Algorithm 1 with alpha = 0.5 (the smallest of 0.3 / 0.5 at which
    Eq. condconvalg1 holds for every PSF of the family).  Periodic problems
    observe a periodic scene (the BC is the right model); the others observe
    the field of view of a larger scene (Example 3's protocol).  Each problem
    stops on its own discrepancy rule.
    """
    rng = np.random.default_rng([seed, 0xba7c])
    out = []
    for k in range(count):
        n = int(rng.choice(sizes))
        fam = int(rng.integers(0, 3))
        if fam == 0:
            psf = psf_gaussian(float(rng.uniform(1.0, 4.0)))
        elif fam == 1:
            psf = psf_disk(int(rng.integers(2, 9)))
        else:
            psf = psf_motion(int(rng.choice(np.arange(5, 22, 2))),
                             float(rng.uniform(0.0, math.pi)))
        bc = ("periodic", "reflective", "rect")[int(rng.integers(0, 3))]
        nu = float(rng.uniform(0.005, 0.03))
        kw = dict(mu=10.0 / 255.0, levels=2, max_iter=max_iter, stop=True, name=f"C4-{k}")
        if bc == "rect":
            out.append(_make(n, psf, nu, 1000 + k, bc=bc, precond="bccb", alpha=0.5, **kw))
        elif bc == "periodic":
            f = true_image(n, 1000 + k)
            g, delta = observe_periodic(f, psf, nu, 1000 + k)
            out.append(Problem(g=g, psf=psf, delta=delta, f_true=f, bc=bc, precond="tikh_ns",
                               alpha=0.05, **kw))
        elif quadrant_symmetric(psf):
            out.append(_make(n, psf, nu, 1000 + k, bc=bc, precond="tikh_ns", alpha=0.05, **kw))
        else:
            out.append(_make(n, psf, nu, 1000 + k, bc=bc, precond="sym", alpha=0.3, **kw))
    return out
