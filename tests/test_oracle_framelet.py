"""Pins of the oracle's tight framelet W and soft threshold (Sections 3, 6.1)."""
import math
import os

import numpy as np
import pytest

from oracle import mlba_oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "framelet_1d_printed_n6.txt")


def load_printed():
    mats, cur, name = {}, [], None
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        if line.startswith("B"):
            if name:
                mats[name] = np.array(cur, dtype=float) / 4.0
            name, cur = line, []
        else:
            cur.append([float(v) for v in line.split()])
    mats[name] = np.array(cur, dtype=float) / 4.0
    return mats


def test_filter_matrices_match_printed_section_6_1():
    printed = load_printed()
    b0 = O.filter_matrix(0, 6).toarray()
    b1 = O.filter_matrix(1, 6).toarray()
    b2 = O.filter_matrix(2, 6).toarray()
    np.testing.assert_allclose(b0, printed["B0"], atol=1e-15)
    # the printed "B_1" is the matrix of mask b2 = [-1, 2, -1]/4
    np.testing.assert_allclose(b2, printed["B1"], atol=1e-15)
    # the printed "B_2" is mask b1 without its sqrt(2) and with the opposite sign
    np.testing.assert_allclose(b1, -math.sqrt(2.0) * printed["B2"], atol=1e-15)


def test_mask_sums():
    assert abs(sum(O.MASKS[0]) - 1.0) < 1e-15
    assert abs(sum(O.MASKS[1])) < 1e-15
    assert abs(sum(O.MASKS[2])) < 1e-15


def dense_w(n, levels):
    cols = []
    for k in range(n * n):
        e = np.zeros(n * n)
        e[k] = 1.0
        cols.append(O.framelet_analysis(e.reshape(n, n), levels).ravel())
    return np.stack(cols, axis=1)


@pytest.mark.parametrize("n,levels", [(5, 1), (8, 2), (7, 3), (3, 3), (2, 2)])
def test_tight_frame_dense(n, levels):
    """W^T W = I (Section 1, Eq. wavecoeff; Section 3), including dilations
    larger than the image (reflection folded repeatedly)."""
    w = dense_w(n, levels)
    assert w.shape == (O.n_bands(levels) * n * n, n * n)
    np.testing.assert_allclose(w.T @ w, np.eye(n * n), atol=1e-14)


@pytest.mark.parametrize("levels", [1, 2, 4])
def test_synthesis_is_transpose(levels):
    rng = np.random.default_rng(levels)
    n = 19
    u = rng.standard_normal((n, n))
    x = rng.standard_normal((O.n_bands(levels), n, n))
    lhs = np.vdot(O.framelet_analysis(u, levels), x)
    rhs = np.vdot(u, O.framelet_synthesis(x, levels))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)
    np.testing.assert_allclose(O.framelet_synthesis(O.framelet_analysis(u, levels), levels), u, atol=1e-13)


def test_constant_image_has_only_lowpass():
    n, levels = 12, 2
    w = O.framelet_analysis(np.full((n, n), 0.7), levels)
    np.testing.assert_allclose(w[:-1], 0.0, atol=1e-15)
    np.testing.assert_allclose(w[-1], 0.7, atol=1e-15)


def test_frame_is_redundant():
    """W W^T != I for a tight frame that is not a basis (Section 3)."""
    w = dense_w(4, 1)
    assert np.abs(w @ w.T - np.eye(w.shape[0])).max() > 0.1


def test_soft_threshold_closed_form():
    """Eq. soft: S_mu(x) = sgn(x) max(|x| - mu, 0)."""
    x = np.array([-3.0, -1.0, -0.5, 0.0, 0.25, 0.5, 0.75, 2.0])
    expect = np.array([-2.5, -0.5, 0.0, 0.0, 0.0, 0.0, 0.25, 1.5])
    np.testing.assert_array_equal(O.soft(x, 0.5), expect)
    np.testing.assert_array_equal(O.soft(x, 0.0), x)


def test_level2_a_trous_impulse_response():
    """Reading c2 (undecimated, masks dilated by 2 at level 2): the level-2
    response to an interior impulse is the cascade of b0 with the dilated
    masks, e.g. low-pass rows [1,2,3,4,3,2,1]/16 and, for band (0,1), columns
    sqrt(2)/16 [-1,-2,-1,0,1,2,1] (analysis filters act as correlations)."""
    n, c0 = 21, 10
    u = np.zeros((n, n))
    u[c0, c0] = 1.0
    w = O.framelet_analysis(u, 2)
    k7 = np.array([1, 2, 3, 4, 3, 2, 1]) / 16.0
    v7 = math.sqrt(2.0) / 16.0 * np.array([-1, -2, -1, 0, 1, 2, 1])
    low = np.zeros((n, n))
    low[c0 - 3:c0 + 4, c0 - 3:c0 + 4] = np.outer(k7, k7)
    np.testing.assert_allclose(w[-1], low, atol=1e-16)
    band01 = np.zeros((n, n))
    band01[c0 - 3:c0 + 4, c0 - 3:c0 + 4] = np.outer(k7, v7)
    np.testing.assert_allclose(w[8 + O.HIGH_BANDS.index((0, 1))], band01, atol=1e-16)
