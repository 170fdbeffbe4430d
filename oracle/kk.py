"""Kramers-Kronig self-coherent front end (Sec. IV, Steps 1-8), FP64.

TEST INFRASTRUCTURE (see the package docstring).

The paper's KK chain at 4 samples/symbol: the ADC's 12-bit unsigned codes
become floats plus a static DC offset (the AC-coupled digitiser loses the
DC term the reconstruction needs); the front end takes the square root (the
field amplitude) and the logarithm (for the phase); a 1024-point 100 %
overlap-save FFT, the Hilbert transform in the frequency domain and an IFFT
give the phase; amplitude and phase form the field, which is shifted down
by the tone offset; a second 1024-point FFT, a static FD filter (matched
filter) and a 512-point IFFT return the signal at 2 samples/symbol (Steps
1-8). Readings taken:

* v = scale * code + dc; intensities below ``i_min`` are raised to it (the
  logarithm needs I > 0; a minimum-phase field never reaches zero);
  a = sqrt(v), l = ln a;
* overlap-save blocks as in ``cdc.overlap_save``: block j takes the N samples
  from j N/2 - N/4 (zero outside the frame) and keeps its centre half;
* Hilbert transform: the block spectrum times -j sgn(k) (sgn = +1 for bins
  0 < k < N/2, -1 for N/2 < k < N, 0 at k = 0 and k = N/2); the phase is the
  real part of the inverse transform;
* the field E = a exp(j phi) is that of the tone's frame, where the signal
  lies above the tone (minimum phase, Mecozzi et al.); the signal is moved to
  DC by E exp(-j 2 pi f_t n / fs), n the sample index from the frame start
  (the tone then sits at -f_t and the matched filter removes it);
* matched filter and decimation: the second pass's block spectrum X times
  H[k] = 2 RRC(f_k) (gain sqrt(4)); the N/2-point inverse transform takes the
  bins |f| < fs/4: bin k' of the short transform is bin k' (k' < N/4) or
  k' + N/2 (k' >= N/4) of the long one; y = IFFT_{N/2}(Y) / 2 returns the
  filtered signal at every other sample; the block keeps its centre half
  [N/8, 3N/8) of the N/2 outputs.
"""

from __future__ import annotations

import numpy as np

from .cdc import rrc_amplitude

SPS = 4


def front_end(codes: np.ndarray, scale: float, dc: float, i_min: float):
    """Step 1: (a, l) = (sqrt(I), ln sqrt(I)), I = max(scale * code + dc, i_min)."""
    v = scale * codes.astype(np.float64) + dc
    I = np.maximum(v, i_min)
    a = np.sqrt(I)
    return a, np.log(a)


def _blocks(S: int, N: int):
    hop, lead = N // 2, N // 4
    for j in range((S + hop - 1) // hop):
        yield j, j * hop - lead


def _segment(x: np.ndarray, start: int, N: int) -> np.ndarray:
    seg = np.zeros(N, dtype=x.dtype)
    lo, hi = max(start, 0), min(start + N, x.shape[0])
    if hi > lo:
        seg[lo - start:hi - start] = x[lo:hi]
    return seg


def hilbert_sign(N: int) -> np.ndarray:
    """-j sgn(k) on the N FFT bins (0 at DC and at N/2)."""
    k = np.arange(N)
    sgn = np.where((k > 0) & (k < N // 2), 1.0, np.where(k > N // 2, -1.0, 0.0))
    return -1j * sgn


def hilbert_os(l: np.ndarray, N: int) -> np.ndarray:
    """Steps 2-3: overlap-save Hilbert transform of the real sequence l."""
    S = l.shape[0]
    hop, lead = N // 2, N // 4
    G = hilbert_sign(N)
    out = np.zeros(S, dtype=np.float64)
    for j, start in _blocks(S, N):
        seg = _segment(l, start, N)
        phi = np.real(np.fft.ifft(np.fft.fft(seg) * G))
        keep = min(hop, S - j * hop)
        out[j * hop:j * hop + keep] = phi[lead:lead + keep]
    return out


def reconstruct(a: np.ndarray, phi: np.ndarray, tone_over_fs: float) -> np.ndarray:
    """Step 4: E = a exp(j phi) exp(-j 2 pi (f_t / fs) n)."""
    n = np.arange(a.shape[0], dtype=np.float64)
    return a * np.exp(1j * phi) * np.exp(-2j * np.pi * tone_over_fs * n)


def matched_response(N: int, rolloff: float) -> np.ndarray:
    """H[k] = 2 RRC(f_k) on the N bins of the 4-sample/symbol grid (symbol rate fs/4)."""
    f = np.fft.fftfreq(N, d=1.0)            # cycles per sample; the symbol rate is 1/4
    return np.sqrt(SPS) * rrc_amplitude(f, 0.25, rolloff)


def decimation_bins(N: int) -> np.ndarray:
    """Bin of the N-point spectrum that bin k' of the N/2-point spectrum takes (|f| < fs/4)."""
    k_short = np.arange(N // 2)
    return np.where(k_short < N // 4, k_short, k_short + N // 2)


def matched_decimate(E: np.ndarray, N: int, rolloff: float) -> np.ndarray:
    """Steps 6-8: FD matched filter and 4 -> 2 samples/symbol by spectral truncation."""
    S = E.shape[0]
    hop, lead = N // 2, N // 4
    H = matched_response(N, rolloff)
    k_long = decimation_bins(N)
    out = np.zeros(S // 2, dtype=np.complex128)
    for j, start in _blocks(S, N):
        seg = _segment(E, start, N)
        X = np.fft.fft(seg) * H
        y = np.fft.ifft(X[k_long]) / 2.0
        keep = min(hop // 2, S // 2 - j * (hop // 2))
        if keep > 0:
            out[j * (hop // 2):j * (hop // 2) + keep] = y[lead // 2:lead // 2 + keep]
    return out


def kk_receive(codes: np.ndarray, scale: float, dc: float, i_min: float, tone_over_fs: float, rolloff: float,
               N: int = 1024):
    """Steps 1-8. Returns (E [S] at 4 samples/symbol, y [S/2] at 2 samples/symbol)."""
    a, l = front_end(codes, scale, dc, i_min)
    phi = hilbert_os(l, N)
    E = reconstruct(a, phi, tone_over_fs)
    return E, matched_decimate(E, N, rolloff)


# ----------------------------------------------------------------------------
# Step 9 (Sec. IV-D): the KK receiver's TD widely-linear DD-LMS, then the
# decision and demapping, on the front end's output at 2 samples/symbol.
# Reading: the single-polarisation equaliser is the widely-linear A4 with one
# input and one output (y = h * x + g * conj(x) per output symbol, the A4
# block phase, decisions, update and segment schedule); the front end keeps
# the tone's phase, so the decisions need no quarter-turn search.
# ----------------------------------------------------------------------------

def kk_equalise(x: np.ndarray, h: np.ndarray, g: np.ndarray, n_sym: int, L_b: int, seg_blocks: int,
                warmup_blocks: int, m: int, mu: float, mu_conj: float, diag=None):
    """x: [S2] complex at 2 samples/symbol; h, g: [T] initial direct and conjugate taps.
    Returns (y [n_sym], final h, final g, bits uint8 [n_sym m] of the Gray-demapped decisions).

    Runs the dual-polarisation widely-linear segmented DD-LMS of ``mimo.dd_lms_wl`` with the second
    input plane zero and row 0 holding (h, 0, g, 0): the second input's taps then receive e x_2 = 0
    and stay zero, so row 0 is exactly the single-polarisation equaliser (row 1 is not used).
    ``diag`` (a dict) receives the per-segment decision margins of ``mimo.dd_lms`` (row 0 in [:, 0])."""
    from . import mimo, qam
    T = h.shape[0]
    xbuf = np.zeros((2, x.shape[0]), dtype=np.complex128)
    xbuf[0] = x
    taps = mimo.wl_identity_taps(T)
    taps[0, 0], taps[0, 1], taps[0, 2], taps[0, 3] = h, 0.0, g, 0.0
    y, hf = mimo.dd_lms_wl(xbuf, taps, n_sym, L_b, seg_blocks, warmup_blocks, m, mu, mu_conj, diag=diag)
    li, lq = qam.decide_levels(y[0], m)
    return y[0], hf[0, 0].copy(), hf[0, 2].copy(), qam.levels_to_bits(li, lq, m).reshape(-1)
