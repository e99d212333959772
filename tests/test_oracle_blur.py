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
            if bc == "antireflective":
                # NumPy's odd reflection: 2 x[edge] - x[edge -+ i], one axis after
                # the other (the corner rule of Section 2.2)
                e = np.pad(e, c, mode="reflect", reflect_type="odd")
            else:
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


# ---------------------------------------------------------------------------
# antireflective BCs and reblurring (Section 2.2)

@pytest.mark.parametrize("psf", ["motion", "gauss", "asym3"])
@pytest.mark.parametrize("n", [6, 9])
def test_antireflective_matches_dense_odd_reflection(psf, n):
    """A with antireflective BCs from the oracle's pad equals the dense matrix
    built with NumPy's odd reflection (2 x[edge] - x[edge -+ i], per axis)."""
    h = PSFS[psf]
    a = dense_blur_matrix(h, n, "antireflective")
    f = np.random.default_rng(n).standard_normal((n, n))
    np.testing.assert_allclose(O.blur(f, h, "antireflective").ravel(), a @ f.ravel(), atol=1e-13)


def test_antireflective_corner_formula():
    """The corner of the antireflective pad is 4 F(1,1) - 2 F(1,j+1) -
    2 F(i+1,1) + F(i+1,j+1) (Section 2.2), checked at every corner offset on
    a random image (1-based i, j as printed)."""
    n, c = 7, 3
    f = np.random.default_rng(2).standard_normal((n, n))
    e = O.extend(f, c, "antireflective")
    F = lambda i, j: f[i - 1, j - 1]            # 1-based access to the FOV
    E = lambda i, j: e[c + i - 1, c + j - 1]    # 1-based access to the pad
    for i in range(1, c + 1):
        for j in range(1, c + 1):
            assert abs(E(1 - i, 1 - j) - (4 * F(1, 1) - 2 * F(1, j + 1) - 2 * F(i + 1, 1) + F(i + 1, j + 1))) < 1e-13
            assert abs(E(1 - i, n + j) - (4 * F(1, n) - 2 * F(1, n - j) - 2 * F(i + 1, n) + F(i + 1, n - j))) < 1e-13
            assert abs(E(n + i, 1 - j) - (4 * F(n, 1) - 2 * F(n, j + 1) - 2 * F(n - i, 1) + F(n - i, j + 1))) < 1e-13
            assert abs(E(n + i, n + j) - (4 * F(n, n) - 2 * F(n, n - j) - 2 * F(n - i, n) + F(n - i, n - j))) < 1e-13


def test_antireflective_preserves_linear_images():
    """Antireflective BCs extend a linear image linearly, so a normalised
    quadrantally symmetric PSF maps every affine image to itself; the
    reflective and zero BCs do not."""
    n = 12
    h = I.psf_gaussian(1.3, 7)
    y, x = np.mgrid[0:n, 0:n].astype(float)
    lin = 0.3 + 0.05 * y - 0.02 * x
    np.testing.assert_allclose(O.blur(lin, h, "antireflective"), lin, atol=1e-13)
    assert np.abs(O.blur(lin, h, "reflective") - lin).max() > 1e-3
    assert np.abs(O.blur(lin, h, "zero") - lin).max() > 1e-3


def test_antireflective_sine_eigenvectors():
    """For a symmetric 1-D PSF the antireflective matrix has the sine vectors
    sin(j pi i / (n-1)), i = 0..n-1 (zero at both ends), as eigenvectors with
    eigenvalue sum_d h(d) cos(d j pi / (n-1)), and the constant and linear
    vectors with eigenvalue sum h: the structure behind the antireflective
    transform (Section 2.2).  Checked on the 2-D operator with a separable
    PSF, one factor a delta."""
    n, p = 10, 5
    g1 = np.exp(-0.5 * (np.arange(p) - 2.0) ** 2 / 1.1 ** 2)
    g1 /= g1.sum()
    h = np.zeros((p, p))
    h[2, :] = g1                                  # acts along the columns only
    a = dense_blur_matrix(h, n, "antireflective")
    i = np.arange(n)
    for j in range(1, n - 1):
        v1 = np.sin(j * np.pi * i / (n - 1))
        v = np.tile(v1, (n, 1)).ravel()           # the same row everywhere
        lam = sum(g1[k] * np.cos((k - 2) * j * np.pi / (n - 1)) for k in range(p))
        np.testing.assert_allclose(a @ v, lam * v, atol=1e-13)
    for v1 in (np.ones(n), i / (n - 1.0)):
        v = np.tile(v1, (n, 1)).ravel()
        np.testing.assert_allclose(a @ v, v, atol=1e-13)


@pytest.mark.parametrize("bc", ["zero", "periodic"])
def test_reblur_is_transpose_for_zero_and_periodic(bc):
    """Section 2.2: the reblurring matrix A' (the same BCs imposed on the PSF
    rotated by 180 degrees) equals A^T for zero and periodic BCs."""
    h = PSFS["asym3"]
    n = 8
    a = dense_blur_matrix(h, n, bc)
    t = np.random.default_rng(5).standard_normal((n, n))
    np.testing.assert_allclose(O.reblur(t, h, bc).ravel(), a.T @ t.ravel(), atol=1e-13)
    np.testing.assert_allclose(O.blur_adjoint(t, h, bc), O.reblur(t, h, bc), atol=1e-13)


def test_reblur_differs_from_transpose_for_antireflective():
    """With antireflective BCs A' is not A^T (that is why the paper replaces
    A^T by A'); for a symmetric PSF A' = A."""
    n = 8
    h = PSFS["asym3"]
    a = dense_blur_matrix(h, n, "antireflective")
    t = np.random.default_rng(6).standard_normal((n, n))
    assert np.abs(O.reblur(t, h, "antireflective").ravel() - a.T @ t.ravel()).max() > 1e-3
    g = PSFS["gauss"]
    np.testing.assert_allclose(O.reblur(t, g, "antireflective"), O.blur(t, g, "antireflective"), atol=1e-14)
