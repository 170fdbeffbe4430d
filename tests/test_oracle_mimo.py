"""Pins for the oracle's A2 (CMA), A3 (FO estimate) and A4 (segmented DD-LMS)."""

import numpy as np
import pytest

from oracle import cdc, mimo, qam, theory
from oracle.receiver import RxConfig, receive
from synth import LinkParams, generate, workload


def test_butterfly_and_gradient_by_explicit_loops():
    rng = np.random.default_rng(0)
    T, S, off = 5, 40, 1
    x = rng.normal(size=(2, S)) + 1j * rng.normal(size=(2, S))
    h = rng.normal(size=(2, 2, T)) + 1j * rng.normal(size=(2, 2, T))
    n = np.arange(-1, 22)
    X = mimo.gather(x, n, T, off)
    y = mimo.butterfly(h, X)
    e = rng.normal(size=(2, n.size)) + 1j * rng.normal(size=(2, n.size))
    g = mimo.gradient(e, X)
    c = (T - 1) // 2
    xs = lambda p, i: x[p, i] if 0 <= i < S else 0.0
    for q in range(2):
        for i, nn in enumerate(n):
            ref = sum(h[q, p, k] * xs(p, off + 2 * nn + c - k) for p in range(2) for k in range(T))
            assert abs(y[q, i] - ref) < 1e-12
        for p in range(2):
            for k in range(T):
                ref = sum(e[q, i] * np.conj(xs(p, off + 2 * nn + c - k)) for i, nn in enumerate(n))
                assert abs(g[q, p, k] - ref) < 1e-12


def test_dd_block_update_by_explicit_loops():
    """One DD-LMS block (phase, decision, error, update) written out symbol by symbol."""
    rng = np.random.default_rng(1)
    m, T, L = 4, 3, 6
    x = 0.5 * (rng.normal(size=(2, 40)) + 1j * rng.normal(size=(2, 40)))
    h = mimo.identity_taps(T) + 0.05 * (rng.normal(size=(2, 2, T)) + 1j * rng.normal(size=(2, 2, T)))
    mu = 0.01
    y, h2, _ = mimo._dd_blocks(x, h[None], np.arange(5, 5 + L)[None], m, mu, 0)
    c = 1
    ref_h = h.copy()
    for q in range(2):
        yq = [sum(h[q, p, k] * x[p, 2 * n + c - k] for p in range(2) for k in range(T)) for n in range(5, 5 + L)]
        assert np.allclose(y[0, q], yq, atol=1e-13)
        s4 = sum(v ** 4 for v in yq)
        psi = np.arctan2((-s4).imag, (-s4).real) / 4
        for i, n in enumerate(range(5, 5 + L)):
            d = qam.decide(np.array([yq[i] * np.exp(-1j * psi)]), m)[0]
            err = d * np.exp(1j * psi) - yq[i]
            for p in range(2):
                for k in range(T):
                    ref_h[q, p, k] += mu * err * np.conj(x[p, 2 * n + c - k])
    assert np.allclose(h2[0], ref_h, atol=1e-13)


def _noiseless_link(m=2, **kw):
    base = dict(bits_per_sym=m, symbol_rate=32e9, n_sym=1 << 14, length=80e3, linewidth=0.0,
                freq_offset=0.0, snr_db=None, jones=True)
    base.update(kw)
    return LinkParams(**base)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_cma_recovers_a_unitary_on_noiseless_input(seed):
    p = _noiseless_link()
    fr = generate(p, seed)
    cfg = RxConfig(bits_per_sym=2, symbol_rate=p.symbol_rate, length=p.length, fft_size=1024,
                   n_taps=15, lms_block=64, bps_phases=32, bps_window=64)
    r = receive(fr.samples, cfg, fr.ref_words)
    # combined DC response of the acquired CMA taps times the channel's Jones matrix
    W = r.taps_cma.sum(axis=-1) * r.scale[None, :]
    G = W @ fr.jones
    P = np.abs(G)
    if P[0, 1] > P[0, 0]:
        G = G[::-1]
    D = G / np.abs(np.diag(G)).mean()
    assert np.max(np.abs(D @ D.conj().T - np.eye(2))) < 1e-2        # unitary x diag, up to a permutation
    assert np.max(np.abs(D - np.diag(np.diag(D)))) < 1e-2        # crosstalk below -40 dB
    evm2 = r.counts["evm_num"] / r.counts["evm_den"]
    assert 10 * np.log10(evm2) < -30
    assert r.counts["bit_errors"] == 0


def test_large_offset_is_removed_on_noiseless_input():
    p = _noiseless_link(freq_offset=1.3e9)
    fr = generate(p, 4)
    cfg = RxConfig(bits_per_sym=2, symbol_rate=p.symbol_rate, length=p.length, fft_size=1024,
                   n_taps=15, lms_block=64, bps_phases=32, bps_window=64)
    r = receive(fr.samples, cfg, fr.ref_words)
    assert r.fo_code == 13000
    # the matched filter sits ahead of the derotation, so a 4 % offset clips the band edge: about -26 dB
    assert 10 * np.log10(r.counts["evm_num"] / r.counts["evm_den"]) < -24
    assert r.counts["bit_errors"] == 0
    # the corrected taps on the derotated samples give the CMA outputs, derotated:
    # y'[n] = y[n] exp(-j 2 w n) with w the offset per sample
    n = np.arange(2048, 4096)
    xd = mimo.derotate(r.cdc, r.fo_code, cfg.fo_grid_hz, cfg.fs, 0)
    y1 = mimo.butterfly(r.taps_foe, mimo.gather(xd, n, cfg.n_taps, 0))
    y0 = mimo.butterfly(r.taps_cma, mimo.gather(r.cdc, n, cfg.n_taps, 0))
    w = 2 * np.pi * r.fo_code * cfg.fo_grid_hz / cfg.fs
    assert np.max(np.abs(y1 - y0 * np.exp(-1j * w * 2 * n))) < 1e-9


def test_foe_exact_code_on_noiseless_grid_offset():
    rng = np.random.default_rng(3)
    Rs, grid, L_b = 32e9, 100e3, 128
    for true_code in (0, 7, -4321, 5000, 30000):
        s = qam.alphabet(2)[rng.integers(0, 4, size=(2, 4096))]
        w = 2 * np.pi * true_code * grid / Rs
        y = s * np.exp(1j * (w * np.arange(4096) + rng.uniform(0, 6, (2, 1))))
        code, what, _ = mimo.foe_code(y, Rs, grid, L_b)
        assert code == true_code
        assert what == pytest.approx(w, abs=1e-9)


@pytest.mark.parametrize("m", [2, 4])
def test_foe_within_one_grid_step_at_12db(m):
    rng = np.random.default_rng(4)
    Rs, grid, L_b = 32e9, 100e3, 128
    for trial in range(4):
        f0 = rng.uniform(-1e9, 1e9)
        s = qam.alphabet(m)[rng.integers(0, 2**m, size=(2, 8192))]
        sig = np.sqrt(1 / (2 * 10 ** 1.2))
        y = s * np.exp(1j * 2 * np.pi * f0 / Rs * np.arange(8192)) + sig * (
            rng.normal(size=s.shape) + 1j * rng.normal(size=s.shape))
        code, _, _ = mimo.foe_code(y, Rs, grid, L_b)
        assert abs(code * grid - f0) < grid


def test_segment_schedule_costs_nothing():
    """Segmented DD-LMS BER lies within binomial 3 sigma of the fully serial schedule."""
    w = workload("dp-16qam-32gbd", n_sym=1 << 16)
    p = w["link"].with_(snr_db=15.0)
    fr = generate(p, 5)
    cfg = RxConfig.from_dict(w["rx"])
    seg = receive(fr.samples, cfg, fr.ref_words).counts
    cfg_serial = RxConfig.from_dict(dict(w["rx"], seg_blocks=1 << 20))
    ser = receive(fr.samples, cfg_serial, fr.ref_words).counts
    b1, b2 = seg["bit_errors"] / seg["bits"], ser["bit_errors"] / ser["bits"]
    pth = theory.gray_qam_ber(4, 15.0)
    sigma = np.sqrt(pth * (1 - pth) / seg["bits"])
    assert abs(b1 - b2) < 3 * sigma * 1.5


def test_decision_margin_by_brute_force():
    """Distance to the nearest interior decision boundary, against a scan of all boundaries."""
    rng = np.random.default_rng(5)
    for m in (2, 4, 6):
        L, a = qam.n_levels(m), qam.amp(m)
        bounds = (2 * np.arange(1, L) - L) * a              # midpoints between adjacent levels
        u = rng.uniform(-1.5, 1.5, size=(3, 50)) + 1j * rng.uniform(-1.5, 1.5, size=(3, 50))
        got = mimo.decision_margin(u, m)
        dist = lambda v: np.min(np.abs(v[..., None] - bounds), axis=-1)
        want = np.minimum(dist(u.real), dist(u.imag)).min(axis=-1)
        assert np.allclose(got, want, atol=1e-12)


# ----------------------------------------------------------------------------
# A2 singularity recovery (reading: outputs correlated beyond 0.5 at a lag up
# to (T-1)/2 -> second row rebuilt from the first, acquisition rerun once)
# ----------------------------------------------------------------------------

@pytest.mark.parametrize("d", [-7, -3, 0, 1, 5, 7])
def test_output_correlation_of_a_delayed_copy_is_the_overlap_fraction(d):
    """y1 = e^{j theta} y0 delayed by d on unit-modulus symbols: |rho_d| = (L - |d|) / L exactly.

    Over the second half (L samples) the lag-d sum runs over the L - |d| aligned samples, each
    |y0|^2 = 1, and both energies are L; the other lags are sums of random QPSK products, far lower.
    """
    rng = np.random.default_rng(11 + d)
    L = 512
    y0 = qam.alphabet(2)[rng.integers(0, 4, size=2 * L)]
    y0 = y0 / np.abs(y0)
    y1 = np.exp(1j * 0.7) * np.roll(y0, d)
    got = mimo.output_correlation(np.stack([y0, y1]), 7)
    assert got == pytest.approx((L - abs(d)) / L, abs=1e-12)


def test_output_correlation_ignores_lags_beyond_the_window_and_independent_outputs():
    rng = np.random.default_rng(12)
    L = 2048
    y0 = np.exp(1j * np.pi / 2 * rng.integers(0, 4, size=2 * L))
    assert mimo.output_correlation(np.stack([y0, np.roll(y0, 9)]), 7) < 0.15
    y1 = np.exp(1j * np.pi / 2 * rng.integers(0, 4, size=2 * L))
    assert mimo.output_correlation(np.stack([y0, y1]), 7) < 0.15


def _freq_response(h, w):
    """H[..., q, p] at radian frequencies w [F], taps indexed about the centre tap."""
    T = h.shape[-1]
    c = (T - 1) // 2
    E = np.exp(-1j * np.outer(w, np.arange(T) - c))          # [F, T]
    return np.einsum("qpk,fk->fqp", h, E)


@pytest.mark.parametrize("T", [3, 15, 21])
def test_rebuilt_second_row_makes_a_scaled_unitary_at_every_frequency(T):
    """[[H_xx, H_xy], [-conj H_xy, conj H_xx]]: W W^H = (|H_xx|^2 + |H_xy|^2) I for all w.

    A dropped minus sign, a missing time reversal or a missing conjugate each leave an
    off-diagonal term on frequency-selective taps.
    """
    rng = np.random.default_rng(T)
    h = rng.normal(size=(2, 2, T)) + 1j * rng.normal(size=(2, 2, T))
    h2 = mimo.rebuild_second_row(h)
    assert np.array_equal(h2[0], h[0])
    w = np.linspace(-np.pi, np.pi, 97)
    W = _freq_response(h2, w)
    G = W @ np.conj(np.swapaxes(W, -1, -2))
    p = np.abs(W[:, 0, 0]) ** 2 + np.abs(W[:, 0, 1]) ** 2
    assert np.max(np.abs(G - p[:, None, None] * np.eye(2))) < 1e-10 * np.max(p)


def test_rebuilt_second_row_inverts_the_other_polarisation_of_a_jones_matrix():
    """First row = first row of J^H for J = [[a, b], [-conj b, conj a]] (|a|^2 + |b|^2 = 1):
    the rebuilt matrix is J^H itself, so W J = I."""
    rng = np.random.default_rng(13)
    for _ in range(5):
        v = rng.normal(size=2) + 1j * rng.normal(size=2)
        a, b = v / np.linalg.norm(v)
        J = np.array([[a, b], [-np.conj(b), np.conj(a)]])
        T = 9
        h = np.zeros((2, 2, T), dtype=np.complex128)
        h[0, :, (T - 1) // 2] = np.conj(J.T)[0]
        W = mimo.rebuild_second_row(h).sum(axis=-1)
        assert np.max(np.abs(W @ J - np.eye(2))) < 1e-13


def test_cma_rerun_recovers_from_a_singular_start():
    """Both rows started on the same polarisation lock onto one source (rho ~ 1); the rebuild
    and rerun then demultiplex: -40 dB crosstalk through the channel's Jones matrix and
    uncorrelated outputs, as from the identity start."""
    p = _noiseless_link()
    fr = generate(p, 2)
    cfg = RxConfig(bits_per_sym=2, symbol_rate=p.symbol_rate, length=p.length, fft_size=1024,
                   n_taps=15, lms_block=64, bps_phases=32, bps_window=64)
    T, L_b, n_cma = cfg.n_taps, cfg.lms_block, cfg.cma_blocks
    scale = cdc.power_scale(fr.samples, 2 * n_cma * L_b)
    H = cdc.cdc_response(cfg.fft_size, cfg.fs, cfg.dispersion, cfg.length, cfg.wavelength,
                         cfg.symbol_rate, cfg.rrc_rolloff, cfg.sps)
    buf = cdc.overlap_save(fr.samples * scale[:, None], H)
    h0 = np.zeros((2, 2, T), dtype=np.complex128)
    h0[:, 0, (T - 1) // 2] = 1.0                                # both outputs read polarisation x
    h1, y1 = mimo.cma_pass(buf, h0, L_b, n_cma, cfg.mu_cma, qam.cma_radius(2), 0)
    assert mimo.output_correlation(y1, (T - 1) // 2) > 0.99       # the first pass is singular
    h, y, rho, reran = mimo.cma_acquire(buf, T, L_b, n_cma, cfg.mu_cma, qam.cma_radius(2), 0, h0=h0)
    assert reran and rho > 0.99
    assert mimo.output_correlation(y, (T - 1) // 2) < 0.1
    G = (h.sum(axis=-1) * scale[None, :]) @ fr.jones
    if np.abs(G[0, 1]) > np.abs(G[0, 0]):
        G = G[::-1]
    D = G / np.abs(np.diag(G)).mean()
    assert np.max(np.abs(D - np.diag(np.diag(D)))) < 1e-2       # crosstalk below -40 dB
    # constant modulus reached on both outputs over the second half of the rerun
    half = y[:, y.shape[1] // 2:]
    assert np.mean(np.abs(np.abs(half) ** 2 - 1.0)) < 0.05
