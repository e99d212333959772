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


def test_unpreconditioned_pcg_stop_rule_is_caught(monkeypatch):
    """Reading c12 fixes the relative residual of the preconditioned system
    (psys); a stop on ||r_k|| / ||r_0|| must fail the pin."""
    import test_oracle_precond as TP

    def pcg_plain(r, apply_aat, apply_m, alpha, tol=1e-3, max_steps=5):
        x = np.zeros_like(r)
        res = r.copy()
        zz = apply_m(res)
        rho = float(np.vdot(res, zz))
        p = zz.copy()
        n0 = float(np.linalg.norm(r))
        steps = 0
        for k in range(1, max_steps + 1):
            q = apply_aat(p) + alpha * p
            a = rho / float(np.vdot(p, q))
            x = x + a * p
            res = res - a * q
            steps = k
            zz = apply_m(res)
            rho_new = float(np.vdot(res, zz))
            if float(np.linalg.norm(res)) / n0 <= tol:
                break
            p = zz + (rho_new / rho) * p
            rho = rho_new
        return x, steps
    monkeypatch.setattr(O, "pcg", pcg_plain)
    with pytest.raises(AssertionError):
        TP.test_pcg_stops_on_preconditioned_relative_residual()


def test_reflective_pad_instead_of_antireflective_is_caught(monkeypatch):
    """Planting the reflective pad in place of the antireflective one must
    fail the linear-preservation pin."""
    import test_oracle_blur as TB
    good = O.extend

    def wrong(f, c, bc):
        return good(f, c, "reflective" if bc == "antireflective" else bc)
    monkeypatch.setattr(O, "extend", wrong)
    with pytest.raises(AssertionError):
        TB.test_antireflective_preserves_linear_images()


def test_wrong_antireflective_angles_are_caught(monkeypatch):
    """The sine vectors of the antireflective transform have frequencies
    j pi / (n - 1); a DCT-like j pi / n must fail the diagonalisation pin."""
    import test_oracle_precond as TP

    def wrong(n):
        th = np.arange(n) * np.pi / n
        th[0] = th[n - 1] = 0.0
        return th
    monkeypatch.setattr(O, "ar_angles", wrong)
    with pytest.raises(AssertionError):
        TP.test_antireflective_transform_diagonalises_ar_matrix(I.psf_disk(2), 6)
