"""The evaluation metrics (paper_2506_23568_gb300.metrics) against closed forms: the
point response of a uniformly weighted aperture is a sinc, whose -3 dB width (0.8859 of the
first-null half-width), first sidelobe (-13.26 dB) and integrated sidelobe ratio (-9.68 dB
over an unbounded slice) are textbook values.  CPU only."""
import numpy as np
import pytest

from paper_2506_23568_gb300 import metrics


def test_psf_metrics_of_a_sinc():
    d = 1e-2  # first-null half-width
    x = np.arange(-8000, 8001) * (d / 40)  # +/- 200 nulls: the sidelobe energy beyond is 5e-4 of the total
    line = np.sinc(x / d) * np.exp(1j * 0.3)
    width, pslr, islr = metrics.psf_metrics(line, d / 40)
    assert width == pytest.approx(0.88589 * d, rel=2e-3)
    assert pslr == pytest.approx(-13.26, abs=0.02)
    assert islr == pytest.approx(-9.68, abs=0.05)


def test_psf_metrics_shifted_and_scaled():
    d = 7e-3
    x = np.arange(-300, 301) * 1e-4
    a = metrics.psf_metrics(3.0 * np.sinc((x - 1.3e-3) / d), 1e-4)
    b = metrics.psf_metrics(np.sinc(x / d), 1e-4)
    assert a == pytest.approx(b, rel=2e-2, abs=2e-2)


def test_psnr_and_nrmse_definitions():
    rng = np.random.default_rng(1)
    ref = rng.normal(size=500) + 1j * rng.normal(size=500)
    err = 1e-3 * (rng.normal(size=500) + 1j * rng.normal(size=500))
    f = ref + err
    m = np.abs(ref).max()
    assert metrics.psnr_db(f, ref) == pytest.approx(-10 * np.log10(np.mean(np.abs(err) ** 2) / m ** 2), rel=1e-12)
    assert metrics.nrmse_db(f, ref) == pytest.approx(20 * np.log10(np.linalg.norm(err) / np.linalg.norm(ref)),
                                                     rel=1e-12)
    # the magnitude variant ignores a global phase
    assert metrics.psnr_db(ref * np.exp(1j), ref, magnitude=True) > 250
