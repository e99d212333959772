"""The pins have teeth: plant plausible mistakes in the oracle (on the CPU,
through monkeypatching) and check that a pin then fails."""
import numpy as np
import pytest

import mlba_inputs as I
from oracle import mlba_oracle as O
from test_oracle_blur import dense_blur_matrix
import test_oracle_framelet as TF
import test_oracle_mlba as TM


def test_correlation_instead_of_convolution_is_caught(monkeypatch):
    # a motion PSF is centrally symmetric, so use one that is not
    h = np.array([[0.0, 0.1, 0.05], [0.2, 0.3, 0.0], [0.15, 0.1, 0.1]])
    good = O.blur

    def flipped(f, hh, bc):
        return good(f, hh[::-1, ::-1], bc)
    monkeypatch.setattr(O, "blur", flipped)
    a = dense_blur_matrix(h, 7, "zero")
    f = np.random.default_rng(0).standard_normal((7, 7))
    assert np.abs(O.blur(f, h, "zero").ravel() - a @ f.ravel()).max() > 1e-3


def test_wrong_lowpass_mask_is_caught(monkeypatch):
    monkeypatch.setattr(O, "MASKS", ((1 / 3, 1 / 3, 1 / 3),) + O.MASKS[1:])
    with pytest.raises(AssertionError):
        TF.test_tight_frame_dense(5, 1)


def test_missing_sqrt2_is_caught(monkeypatch):
    monkeypatch.setattr(O, "MASKS", (O.MASKS[0], (0.25, 0.0, -0.25), O.MASKS[2]))
    with pytest.raises(AssertionError):
        TF.test_tight_frame_dense(5, 1)


def test_dropped_alpha_in_denominator_is_caught(monkeypatch):
    monkeypatch.setattr(O.SpectralPrecond, "tikh",
                        lambda self, r, a: self.inverse(self.forward(r) * np.conj(self.lam)
                                                        / (self.sigma + 2 * a)))
    with pytest.raises(AssertionError):
        TM.test_mu_zero_periodic_is_iterated_tikhonov("tikh")


def test_wrong_dilation_is_caught(monkeypatch):
    good = O.filter_matrix
    monkeypatch.setattr(O, "filter_matrix", lambda k, n, d=1: good(k, n, 1))
    TF.test_tight_frame_dense(8, 2)          # still a tight frame ...
    with pytest.raises(AssertionError):      # ... but not the a-trous cascade
        TF.test_level2_a_trous_impulse_response()
