"""Pins for the oracle's Kramers-Kronig front end (Sec. IV, Steps 1-8).

* the front end's amplitude and log-amplitude, value by value;
* the overlap-save Hilbert transform is exact on tones of the block grid (the
  Hilbert transform of cos is sin) and approximates the full-length transform
  (scipy.signal.hilbert) of a band-limited sequence, closer for longer blocks;
* KK reconstruction is exact for a field exp(g) with g analytic (a
  minimum-phase field whose log-amplitude and phase are a Hilbert pair on the
  block grid), and on a synthetic QAM link it recovers the known field, more
  closely as the carrier-to-signal power ratio rises;
* the matched-filter decimation returns every other sample of on-grid tones
  scaled by the filter's amplitude (2 RRC) at their frequencies;
* end to end, the symbols of noiseless QPSK and 16QAM KK links at the
  paper's CSPRs (6 and 11 dB) come back error-free.
"""

import math

import numpy as np
import pytest

from oracle import kk, qam
from oracle.cdc import rrc_amplitude
from synth.kk import KKLink, generate_kk


def test_front_end_values():
    codes = np.array([0, 1, 17, 2048, 4095], dtype=np.uint16)
    scale, dc, i_min = 0.01, -0.1, 1e-6
    a, l = kk.front_end(codes, scale, dc, i_min)
    for c, av, lv in zip(codes, a, l):
        I = max(scale * float(c) + dc, i_min)
        assert abs(av - math.sqrt(I)) <= 1e-15 * math.sqrt(I)
        assert abs(lv - 0.5 * math.log(I)) <= 1e-14


def _interior(S, N):
    """Samples kept by blocks whose input window lies inside the frame."""
    hop, lead = N // 2, N // 4
    lo = hop                                  # block 1 is the first with start >= 0
    hi = ((S - (N - lead)) // hop) * hop + hop   # last block with start + N <= S keeps [j hop, j hop + hop)
    return slice(lo, min(hi, S))


def test_hilbert_is_exact_on_grid_tones():
    N, S = 1024, 8 * 1024
    rng = np.random.default_rng(1)
    n = np.arange(S)
    l = np.full(S, 0.7)
    ref = np.zeros(S)
    for k in rng.integers(1, N // 2, size=6):
        c, th = rng.uniform(0.1, 1.0), rng.uniform(0, 2 * np.pi)
        l += c * np.cos(2 * np.pi * k * n / N + th)
        ref += c * np.sin(2 * np.pi * k * n / N + th)
    phi = kk.hilbert_os(l, N)
    sl = _interior(S, N)
    # FP64 rounding of the tone phases (arguments up to 2.5e4 rad) is about 3e-12
    assert np.max(np.abs(phi[sl] - ref[sl])) < 1e-10


def test_hilbert_approximates_the_full_transform():
    signal = pytest.importorskip("scipy.signal")
    fr = generate_kk(KKLink(n_sym=1 << 14, cspr_db=12.0), 1)
    _, l = kk.front_end(fr.intensity, 1.0, 0.0, 1e-12)
    ref = np.imag(signal.hilbert(l))
    errs = []
    for N in (1024, 4096):
        phi = kk.hilbert_os(l, N)
        sl = slice(N, l.size - N)
        errs.append(np.linalg.norm(phi[sl] - ref[sl]) / np.linalg.norm(ref[sl] - ref[sl].mean()))
    assert errs[0] < 5e-3 and errs[1] < 0.5 * errs[0], errs


@pytest.mark.parametrize("tone", [0.0, 0.13675])
def test_kk_is_exact_for_an_analytic_log_field(tone):
    """h = exp(g), g = sum c_i exp(j (2 pi k_i n / N + th_i)) with 0 < k_i < N/2: ln|h| = Re g and
    arg h = Im g = H{Re g}, so |h|^2 alone gives h back (times the downshift)."""
    N, S = 1024, 6 * 1024
    rng = np.random.default_rng(2)
    n = np.arange(S)
    g = np.full(S, 0.3 + 0j)
    for k in rng.integers(1, N // 2, size=5):
        g += rng.uniform(0.05, 0.3) * np.exp(1j * (2 * np.pi * k * n / N + rng.uniform(0, 2 * np.pi)))
    h = np.exp(g)
    a, l = kk.front_end(np.abs(h) ** 2, 1.0, 0.0, 1e-300)
    E = kk.reconstruct(a, kk.hilbert_os(l, N), tone)
    sl = _interior(S, N)
    ref = h * np.exp(-2j * np.pi * tone * n)
    assert np.max(np.abs(E[sl] - ref[sl])) < 1e-10 * np.max(np.abs(h))


def _field_error_db(cspr_db, N=1024):
    p = KKLink(n_sym=1 << 13, cspr_db=cspr_db)
    fr = generate_kk(p, 2)
    E, _ = kk.kk_receive(fr.codes, fr.scale, fr.dc, 1e-9, p.tone_offset / p.fs, p.rolloff, N)
    n = np.arange(E.size)
    ref = fr.field * np.exp(-2j * np.pi * p.tone_offset / p.fs * n)
    sl = slice(N, E.size - N)
    return 10 * np.log10(np.sum(np.abs(E[sl] - ref[sl]) ** 2) / np.sum(np.abs(fr.signal[sl]) ** 2))


def test_kk_recovers_the_field_better_at_higher_cspr():
    errs = [_field_error_db(c) for c in (8.0, 11.0, 14.0, 18.0)]
    assert errs[0] < -20.0, errs
    assert all(b < a - 2.0 for a, b in zip(errs, errs[1:])), errs


def test_matched_decimation_of_grid_tones():
    """Tones on the block grid, inside and inside the roll-off of the matched filter, at positive and
    negative frequencies: y[m] = sum_i c_i 2 RRC(f_i) exp(j 2 pi f_i 2m) (the filter's gain is
    sqrt(4) = 2, so that with the transmitter's RRC of gain 2 the symbols come back at unit scale)."""
    N, S, rolloff = 1024, 8 * 1024, 0.25
    n = np.arange(S)
    m = np.arange(S // 2)
    rng = np.random.default_rng(3)
    E = np.zeros(S, dtype=np.complex128)
    ref = np.zeros(S // 2, dtype=np.complex128)
    for k in (3, 40, 100, 140, 150, N - 7, N - 120, N - 145):
        f = (k if k < N // 2 else k - N) / N
        c = rng.normal() + 1j * rng.normal()
        E += c * np.exp(2j * np.pi * f * n)
        ref += c * 2.0 * rrc_amplitude(np.array([f]), 0.25, rolloff)[0] * np.exp(2j * np.pi * f * 2 * m)
    y = kk.matched_decimate(E, N, rolloff)
    sl = _interior(S, N)
    sl2 = slice(sl.start // 2, sl.stop // 2)
    assert np.max(np.abs(y[sl2] - ref[sl2])) < 1e-10
    # a tone beyond fs/4 is removed
    y2 = kk.matched_decimate(np.exp(2j * np.pi * 300 / N * n), N, rolloff)
    assert np.max(np.abs(y2[sl2])) < 1e-10


@pytest.mark.parametrize("m", [2, 4])
def test_noiseless_link_end_to_end(m):
    p = KKLink(bits_per_sym=m, n_sym=1 << 13, cspr_db=6.0 if m == 2 else 11.0)
    fr = generate_kk(p, 4)
    _, y = kk.kk_receive(fr.codes, fr.scale, fr.dc, 1e-9, p.tone_offset / p.fs, p.rolloff, 1024)
    ys, s = y[::2][256:-256], fr.symbols[256:-256]
    evm_db = 10 * np.log10(np.mean(np.abs(ys - s) ** 2))
    assert evm_db < -25.0, evm_db
    assert np.array_equal(qam.decide(ys, m), qam.decide(s, m))


def test_joined_buffers_reproduce_the_whole_stream():
    """The ingest reading: buffers of S samples, each processed as a frame joined to the previous
    buffer's last 2N codes (zero codes before the first) with the downshift counted from the stream
    index, give outputs N/2 .. N/2 + S/2 of every joined frame that continue one another and equal the
    front end on the whole stream as one frame; only the stream's first N/2 outputs (2 samples/symbol)
    differ, where the first buffer's carry holds no data."""
    N, S, nb = 1024, 8192, 4
    fr = generate_kk(KKLink(bits_per_sym=4, n_sym=nb * S // 4, cspr_db=11.0, snr_db=25.0), seed=6)
    p = fr.link
    f = p.tone_offset / p.fs
    _, y_ref = kk.kk_receive(fr.codes, fr.scale, fr.dc, 1e-6, f, p.rolloff, N)
    carry = np.zeros(2 * N, dtype=np.uint16)
    outs = []
    for i in range(nb):
        joined = np.concatenate([carry, fr.codes[i * S:(i + 1) * S]])
        carry = joined[S:S + 2 * N].copy()
        a, l = kk.front_end(joined, fr.scale, fr.dc, 1e-6)
        n = np.arange(joined.size) + i * S - 2 * N
        E = a * np.exp(1j * kk.hilbert_os(l, N)) * np.exp(-2j * np.pi * f * n)
        outs.append(kk.matched_decimate(E, N, p.rolloff)[N // 2:N // 2 + S // 2])
    got = np.concatenate(outs)[N // 2:]          # stream outputs from index 0
    ref = y_ref[:got.size]
    assert np.max(np.abs(got[N // 2:] - ref[N // 2:])) < 1e-9 * np.max(np.abs(ref))
    assert np.max(np.abs(got[:N // 2] - ref[:N // 2])) > 1e-3 * np.max(np.abs(ref))


def test_step9_single_polarisation_equaliser_by_explicit_loops():
    """One segment of the single-polarisation widely-linear DD-LMS written out sample by sample: the
    row-0 reduction of the dual-polarisation oracle equals it (a pol-1 leak, a conjugate on the wrong
    factor or a swapped step would not)."""
    from oracle import kk as okk
    from oracle import qam as oq
    rng = np.random.default_rng(21)
    T, L_b, nb, m = 5, 8, 6, 4
    n_sym = L_b * nb
    x = 0.3 * (rng.normal(size=2 * n_sym + 4) + 1j * rng.normal(size=2 * n_sym + 4))
    h0 = np.zeros(T, dtype=np.complex128)
    h0[T // 2] = 1.0
    g0 = 0.05 * (rng.normal(size=T) + 1j * rng.normal(size=T))
    mu, mu_c = 0.01, 0.02
    y, hf, gf, _ = okk.kk_equalise(x, h0, g0, n_sym, L_b, 10 ** 6, 0, m, mu, mu_c)
    c = (T - 1) // 2
    xs = lambda i: x[i] if 0 <= i < x.size else 0.0
    h, g = h0.copy(), g0.copy()
    for b in range(nb):
        ns = range(b * L_b, (b + 1) * L_b)
        yb = [sum(h[k] * xs(2 * n + c - k) + g[k] * np.conj(xs(2 * n + c - k)) for k in range(T)) for n in ns]
        assert np.allclose(y[b * L_b:(b + 1) * L_b], yb, atol=1e-13)
        psi = np.angle(-sum(v ** 4 for v in yb)) / 4
        dh, dg = np.zeros(T, complex), np.zeros(T, complex)
        for i, n in enumerate(ns):
            d = oq.decide(np.array([yb[i] * np.exp(-1j * psi)]), m)[0]
            e = d * np.exp(1j * psi) - yb[i]
            for k in range(T):
                dh[k] += e * np.conj(xs(2 * n + c - k))
                dg[k] += e * xs(2 * n + c - k)
        h, g = h + mu * dh, g + mu_c * dg
    assert np.allclose(hf, h, atol=1e-13) and np.allclose(gf, g, atol=1e-13)


def test_step9_undoes_a_transmitter_iq_imbalance_on_the_kk_link():
    """Noiseless KK link with a transmitter IQ imbalance: the widely-linear Step 9 decides every
    symbol right and reaches a far lower EVM than the linear form (conjugate step 0)."""
    from oracle import kk as okk
    from oracle import qam as oq
    from synth.kk import KKLink, generate_kk
    link = KKLink(bits_per_sym=4, n_sym=1 << 13, cspr_db=14.0, iq_imbalance=(0.08, 0.06))
    fr = generate_kk(link, seed=5)
    _, y2 = okk.kk_receive(fr.codes, fr.scale, fr.dc, 1e-3, link.tone_offset / link.fs, link.rolloff, 1024)
    T = 15
    h0 = np.zeros(T, dtype=np.complex128)
    h0[T // 2] = 1.0
    g0 = np.zeros(T, dtype=np.complex128)
    n = link.n_sym
    runs = {}
    for name, mu_c in (("wl", 1e-3), ("linear", 0.0)):
        y, _, _, bits = okk.kk_equalise(y2, h0, g0, n, 64, 10 ** 6, 0, 4, 1e-3, mu_c)
        tail = slice(n // 2, n - 64)
        runs[name] = (10 * np.log10(np.mean(np.abs(y[tail] - fr.symbols[tail]) ** 2)), bits, y)
    evm_wl, bits_wl, y_wl = runs["wl"]
    assert evm_wl < runs["linear"][0] - 6.0
    tail = slice(n // 2, n - 64)
    assert np.array_equal(oq.decide(y_wl[tail], 4), oq.decide(fr.symbols[tail], 4))
    assert np.array_equal(bits_wl.reshape(n, 4)[tail], fr.bits.reshape(n, 4)[tail])
