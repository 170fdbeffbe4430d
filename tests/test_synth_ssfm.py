"""Pins for the split-step Manakov generator that makes the learned equaliser's
training data (CPU only): the linear limit, the pure-nonlinearity closed form,
energy conservation, second-order step convergence, the ASE variance, and the
torch implementation against the NumPy one on the same draws."""

import numpy as np
import pytest

from synth.channel import LinkParams, fibre_dispersion
from synth.ssfm import FibreLink, H_PLANCK, propagate, propagate_torch, transmit
from synth.channel import C_LIGHT

P = LinkParams(bits_per_sym=4, symbol_rate=32e9, n_sym=2**10, linewidth=0.0, freq_offset=0.0, jones=False)


def tx(p=P, seed=0):
    return transmit(p, seed)[2]


def launch_scale(x, link):
    p_launch = 1e-3 * 10.0 ** (link.launch_dbm / 10.0)
    return np.sqrt(p_launch / np.mean(np.sum(np.abs(x) ** 2, axis=0)))


def test_linear_limit_is_the_dispersion_all_pass():
    link = FibreLink(spans=2, span_km=40.0, gamma=0.0, ase=False)
    x = tx()
    y = propagate(x, P.fs, P.wavelength, P.dispersion, link, np.random.default_rng(0))
    f = np.fft.fftfreq(P.n_samp, d=1.0 / P.fs)
    H = fibre_dispersion(f, P.with_(length=80e3))
    ref = np.fft.ifft(np.fft.fft(x, axis=1) * H[None], axis=1) * launch_scale(x, link)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-10


def test_pure_nonlinearity_closed_form():
    """No loss, no dispersion, one sample per simulated sample: every step is an exact phase
    rotation by 8/9 gamma (|A_x|^2 + |A_y|^2) h, so the field ends rotated by the total."""
    link = FibreLink(spans=3, span_km=50.0, alpha_db_km=0.0, gamma=1.3, ase=False, sim_sps=2, launch_dbm=6.0)
    x = tx()
    y = propagate(x, P.fs, P.wavelength, 0.0, link, np.random.default_rng(0))
    a = x * launch_scale(x, link)
    phi = 8.0 / 9.0 * 1.3e-3 * np.sum(np.abs(a) ** 2, axis=0) * 150e3
    ref = a * np.exp(1j * phi)[None]
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) < 1e-11
    assert phi.mean() > 0.5     # the test is not vacuous


def test_lossless_link_conserves_energy():
    # simulated at the input rate: the final spectral truncation would drop the SPM-broadened tails
    link = FibreLink(spans=2, span_km=40.0, alpha_db_km=0.0, ase=False, launch_dbm=8.0, sim_sps=2)
    x = tx()
    y = propagate(x, P.fs, P.wavelength, P.dispersion, link, np.random.default_rng(0))
    e_in = np.sum(np.abs(x * launch_scale(x, link)) ** 2)
    assert abs(np.sum(np.abs(y) ** 2) / e_in - 1.0) < 1e-12


def test_symmetric_steps_converge_at_second_order():
    link = FibreLink(spans=1, span_km=80.0, alpha_db_km=0.0, ase=False, launch_dbm=10.0, sim_sps=2)
    x = tx()
    run = lambda ph: propagate(x, P.fs, P.wavelength, P.dispersion, link.with_(max_phase=ph),
                               np.random.default_rng(0))
    ref = run(2.5e-4)
    e1 = np.linalg.norm(run(8e-3) - ref)
    e2 = np.linalg.norm(run(4e-3) - ref)
    assert 3.0 < e1 / e2 < 5.0, e1 / e2


def test_ase_variance():
    """Linear link (gamma 0): the received noise per polarisation and 2-samples/symbol sample is
    spans * n_sp h nu (G - 1) f_sim / up, f_sim = up f_s (white ASE band-limited by the final
    spectral truncation); each span's noise passes later spans unchanged in power."""
    p = P.with_(n_sym=2**13)
    link = FibreLink(spans=4, span_km=80.0, gamma=0.0, launch_dbm=0.0)
    x = tx(p)
    y_clean = propagate(x, p.fs, p.wavelength, p.dispersion, link.with_(ase=False), np.random.default_rng(1))
    y = propagate(x, p.fs, p.wavelength, p.dispersion, link, np.random.default_rng(1))
    n = y - y_clean
    alpha = 0.2 / (10.0 * np.log10(np.e)) / 1e3
    G = np.exp(alpha * 80e3)
    up = link.sim_sps // 2
    var = 4 * (10.0 ** 0.5 / 2.0) * H_PLANCK * (C_LIGHT / p.wavelength) * (G - 1.0) * (p.fs * up) / up
    meas = np.mean(np.abs(n) ** 2)
    assert abs(meas / var - 1.0) < 0.03, meas / var


def test_torch_matches_numpy_on_the_same_draws():
    torch = pytest.importorskip("torch")
    link = FibreLink(spans=2, span_km=80.0, launch_dbm=5.0)
    x = tx()
    Su = P.n_samp * (link.sim_sps // 2)
    rng = np.random.default_rng(9)
    draws = [rng.standard_normal((2, Su)) + 1j * rng.standard_normal((2, Su)) for _ in range(link.spans)]
    y_np = propagate(x, P.fs, P.wavelength, P.dispersion, link, np.random.default_rng(9))
    y_t = propagate_torch(torch.from_numpy(x), P.fs, P.wavelength, P.dispersion, link,
                          [torch.from_numpy(d) for d in draws]).numpy()
    assert np.linalg.norm(y_t - y_np) / np.linalg.norm(y_np) < 1e-10
