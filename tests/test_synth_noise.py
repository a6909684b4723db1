"""The App. D.1 Poisson-Gaussian sensor model used for the noise ablation
(synth.ppa_noise): its parameter vectors are the paper's, and its moments,
quantisation and saturation follow the model's closed forms."""
import json
import os

import numpy as np
import pytest

import synth

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
GOLD = json.load(open(os.path.join(ROOT, "tests", "golden", "paper_constants.json")))


def theta(alpha=1.0, sig_r=0.0, lam_d=0.0, sig_p=0.0, F=1000.0, g=1.0, bits=16, t_e=0.0):
    return (alpha, sig_r, lam_d, sig_p, F, g, bits, t_e)


def test_parameter_vectors_are_the_papers():
    assert tuple(synth.THETA_STRONG) == pytest.approx(tuple(GOLD["appD1_theta_strong"]))
    assert tuple(synth.THETA_MILD) == pytest.approx(tuple(GOLD["appD1_theta_mild"]))


def test_output_is_on_the_adc_grid_and_in_range():
    rng = np.random.default_rng(0)
    x = rng.random((64, 64))
    for th in (synth.THETA_MILD, synth.THETA_STRONG):
        y = synth.ppa_noise(x, th, rng).astype(np.float64)
        full = 2 ** th[6] - 1
        assert y.min() >= 0.0 and y.max() <= 1.0
        assert np.allclose(y * full, np.round(y * full), atol=1e-3)


def test_shot_noise_moments():
    """Signal electrons only (no PRNU, read noise or dark current, unit gain, no
    clipping): n_DN ~ Poisson(alpha F x), so mean = variance = alpha F x."""
    rng = np.random.default_rng(1)
    n, x = 200_000, 0.5
    th = theta(alpha=0.2, F=1000.0)
    full = 2 ** th[6] - 1
    y = synth.ppa_noise(np.full(n, x), th, rng).astype(np.float64) * full
    lam = 0.2 * 1000.0 * x
    assert abs(y.mean() - lam) < 5 * np.sqrt(lam / n)
    assert abs(y.var() - lam) < 5 * lam * np.sqrt(2.0 / n)


def test_read_noise_is_clipped_at_zero():
    """No signal: n_e ~ N(0, sigma_r^2) clipped at 0 has mean sigma_r / sqrt(2 pi)
    (rounding to whole DN changes it by far less than the tolerance)."""
    rng = np.random.default_rng(2)
    n, sig = 200_000, 25.0
    th = theta(alpha=0.0, sig_r=sig)
    y = synth.ppa_noise(np.zeros(n), th, rng).astype(np.float64) * (2 ** th[6] - 1)
    assert y.min() == 0.0
    assert abs(y.mean() - sig / np.sqrt(2 * np.pi)) < 0.1


def test_highlights_saturate_where_the_signal_exceeds_the_adc_range():
    """alpha F x / g above 2^b - 1 DN saturates: x > 0.51 for strong, x > 0.85 for
    mild ('earlier highlight saturation' for the strong setting)."""
    rng = np.random.default_rng(3)
    for th, x_sat in ((synth.THETA_STRONG, (2 ** 10 - 1) * 1.5 / (0.20 * 15000)),
                      (synth.THETA_MILD, (2 ** 10 - 1) * 1.5 / (0.12 * 15000))):
        bright = synth.ppa_noise(np.full(4096, min(1.0, x_sat * 1.15)), th, rng)
        dim = synth.ppa_noise(np.full(4096, x_sat * 0.85), th, rng)
        assert (bright == 1.0).mean() > 0.99
        assert (dim == 1.0).mean() < 0.01
    assert (2 ** 10 - 1) * 1.5 / (0.20 * 15000) < (2 ** 10 - 1) * 1.5 / (0.12 * 15000)
