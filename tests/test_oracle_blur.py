"""Pins of the oracle's blur operator A and its transpose (Section 2).

The reference matrices are built column by column from the padding pictures
of Table 1, using numpy's own padding modes and SciPy's 'valid' 2-D
convolution; neither shares the oracle's index arithmetic.
"""
import numpy as np
import pytest
from scipy.signal import convolve2d

import mlba_inputs as I
from oracle import mlba_oracle as O

PAD_MODE = {"zero": "constant", "periodic": "wrap", "reflective": "symmetric"}


def dense_blur_matrix(h, n, bc):
    """A as a dense matrix: column k is the blur of the k-th unit image.

    BC: pad the n x n unit image by c on each side (Table 1: zeros, periodic
    copies, or fliplr/flipud mirrors) then keep the valid convolution.
    rect: the unit image is m x m and the valid convolution is n x n.
    """
    p = h.shape[0]
    c = (p - 1) // 2
    nf = n + p - 1 if bc == "rect" else n
    cols = []
    for k in range(nf * nf):
        e = np.zeros(nf * nf)
        e[k] = 1.0
        e = e.reshape(nf, nf)
        if bc != "rect":
            e = np.pad(e, c, mode=PAD_MODE[bc])
        cols.append(convolve2d(e, h, mode="valid").ravel())
    return np.stack(cols, axis=1)


PSFS = {
    "motion": I.psf_motion(5, 0.6),          # not symmetric: orientation matters
    "gauss": I.psf_gaussian(1.0, 5),
    "asym3": np.array([[0.0, 0.1, 0.05], [0.2, 0.3, 0.0], [0.15, 0.1, 0.1]]),
}


@pytest.mark.parametrize("bc", ["zero", "periodic", "reflective", "rect"])
@pytest.mark.parametrize("psf", list(PSFS))
def test_blur_matches_dense_definition(bc, psf):
    h = PSFS[psf]
    n = 7
    a = dense_blur_matrix(h, n, bc)
    nf = a.shape[1]
    side = int(round(np.sqrt(nf)))
    rng = np.random.default_rng(3)
    f = rng.standard_normal((side, side))
    np.testing.assert_allclose(O.blur(f, h, bc).ravel(), a @ f.ravel(), atol=1e-13)
    t = rng.standard_normal((n, n))
    np.testing.assert_allclose(O.blur_adjoint(t, h, bc).ravel(), a.T @ t.ravel(), atol=1e-13)


@pytest.mark.parametrize("bc", ["zero", "periodic", "reflective", "rect"])
def test_adjoint_identity_larger(bc):
    h = I.psf_disk(3)
    n = 40
    nf = n + h.shape[0] - 1 if bc == "rect" else n
    rng = np.random.default_rng(5)
    x = rng.standard_normal((nf, nf))
    y = rng.standard_normal((n, n))
    lhs = np.vdot(O.blur(x, h, bc), y)
    rhs = np.vdot(x, O.blur_adjoint(y, h, bc))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


@pytest.mark.parametrize("bc", ["periodic", "reflective", "rect"])
def test_psf_sum_one_preserves_constants(bc):
    """Nonnegative PSF with sum 1 (Section 4.2): A maps 1 to 1."""
    h = I.psf_motion(9, 1.1)
    n = 20
    nf = n + h.shape[0] - 1 if bc == "rect" else n
    out = O.blur(np.ones((nf, nf)), h, bc)
    np.testing.assert_allclose(out, 1.0, atol=1e-14)


def test_reflective_blur_symmetric_for_symmetric_psf():
    """Reflective BC with a quadrantally symmetric PSF gives a symmetric A
    (it is diagonalised by the orthonormal DCT, Section 2.2)."""
    a = dense_blur_matrix(I.psf_gaussian(1.3, 5), 6, "reflective")
    np.testing.assert_allclose(a, a.T, atol=1e-15)


def test_rect_equals_valid_crop_of_big_periodic():
    """Eq. Arect: A = M A_big for any BC of A_big (here periodic on m x m)."""
    h = I.psf_motion(5, 2.0)
    n, p = 9, h.shape[0]
    m = n + p - 1
    c = (p - 1) // 2
    rng = np.random.default_rng(1)
    f = rng.standard_normal((m, m))
    big = O.blur(f, h, "periodic")
    np.testing.assert_allclose(O.blur(f, h, "rect"), big[c:c + n, c:c + n], atol=1e-14)
