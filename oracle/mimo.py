"""A2 CMA acquisition, A3 frequency-offset estimate, A4 segmented DD-LMS (linear
and widely linear), FP64.

TEST INFRASTRUCTURE (see the package docstring).

The paper's only adaptive equaliser is a serial 4-tap widely-linear TD
DD-LMS that also decides and demaps (Sec. IV-D); it has no polarisation
demultiplexer, CMA or frequency-offset estimator. Everything below follows
the textbook methods named beside each function, with these readings:

* 2x2 butterfly FIR at 2 samples/symbol, centre tap c = (T-1)/2:
  y_q[n] = sum_p sum_{k<T} h_qp[k] x_p[2n + c - k], x zero outside the buffer;
* block LMS: the output of a block is computed with the taps it started with,
  then h_qp[k] += mu * sum_{n in block} e_q[n] conj(x_p[2n + c - k]);
* CMA (Godard, p = 2): e_q = y_q (R2 - |y_q|^2), R2 = E|s|^4 / E|s|^2, on the
  first ``cma_blocks`` blocks of the first frame only, from h_xx[c] = h_yy[c] = 1;
  if the two outputs then correlate (|rho_d| > 0.5 for some symbol lag
  |d| <= (T-1)/2 over the second half of the acquisition outputs: both locked
  onto one polarisation, possibly at different delays) the second row is
  rebuilt from the first
  (h_yy[k] = conj h_xx[T-1-k], h_yx[k] = -conj h_xy[T-1-k]) and the acquisition
  reruns once;
* FO estimate, two stages, all in FP64, on the outputs of the *final* CMA
  taps (held fixed) over the second half of the acquisition window (an
  adapting CMA lets the output phase wander, which biases any FO estimate).
  Coarse: the peak of the 4th-power periodogram,
  P[k] = sum_q |FFT_Nf(y_q^4)[k]|^2, Nf = the power of two >= 2x the window
  (at least 512),
  first maximum, signed bin kappa -> w_c = 2 pi kappa / (4 Nf) rad/symbol.
  Fine: per block j of L_b symbols a_j = sum_q sum_n (y_q[n] e^{-j w_c n})^4,
  phi_j = arg a_j unwrapped in sequence (a step of more than pi is folded back
  by 2 pi), w_f = 1/4 of the least-squares slope of phi_j against the block
  centres. w = w_c + w_f is quantised to code = round(w Rs / (2 pi) / grid);
  the input is derotated by exp(-j 2 pi code grid g / fs) (g = the sample
  counter) and the acquired taps by exp(-j 2 pi code grid (k - c) / fs);
* DD acquisition: the corrected taps then run ``dd_acq_blocks`` DD-LMS blocks
  (below) serially from the first symbol of the compensated, derotated input;
  their final taps start the segments of the first frame (CMA, then DD-LMS);
* DD-LMS: the frame's symbols are cut into segments of seg_blocks * L_b
  symbols; every segment starts from the same taps (the corrected acquisition
  taps in the first frame, the previous frame's final taps later), runs
  warmup_blocks blocks on the symbols just before it (outputs discarded;
  none for segment 0), then its own blocks. Per block the phase
  psi_q = arg(-sum_n y_q[n]^4) / 4, d_q = dec(y_q e^{-j psi_q}),
  e_q = d_q e^{j psi_q} - y_q. The taps carried to the next frame are the
  last segment's final taps.
"""

from __future__ import annotations

import numpy as np

from . import qam


def identity_taps(T: int) -> np.ndarray:
    h = np.zeros((2, 2, T), dtype=np.complex128)
    c = (T - 1) // 2
    h[0, 0, c] = 1.0
    h[1, 1, c] = 1.0
    return h


def gather(xbuf: np.ndarray, n: np.ndarray, T: int, off: int) -> np.ndarray:
    """X[..., p, i, k] = xbuf[p, off + 2 n_i + c - k] (zero outside the buffer).

    ``n`` has shape [..., L]; the result has shape [..., 2, L, T].
    """
    c = (T - 1) // 2
    idx = off + 2 * n[..., None] + c - np.arange(T)          # [..., L, T]
    S = xbuf.shape[1]
    valid = (idx >= 0) & (idx < S)
    X = xbuf[:, np.clip(idx, 0, S - 1)]                      # [2, ..., L, T]
    X = np.where(valid[None], X, 0.0)
    return np.moveaxis(X, 0, -3)


def butterfly(h: np.ndarray, X: np.ndarray) -> np.ndarray:
    """y[..., q, n] = sum_p sum_k h[..., q, p, k] X[..., p, n, k]."""
    return np.einsum("...qpk,...pnk->...qn", h, X)


def gradient(e: np.ndarray, X: np.ndarray) -> np.ndarray:
    """g[..., q, p, k] = sum_n e[..., q, n] conj(X[..., p, n, k])."""
    return np.einsum("...qn,...pnk->...qpk", e, np.conj(X))


# ----------------------------------------------------------------------------
# A2: CMA acquisition (Godard 1980)
# ----------------------------------------------------------------------------

def cma_pass(xbuf, h0, L_b, n_blocks, mu, R2, off):
    h = h0.copy()
    T = h.shape[-1]
    ys = []
    for b in range(n_blocks):
        n = np.arange(b * L_b, (b + 1) * L_b)
        X = gather(xbuf, n, T, off)
        y = butterfly(h, X)
        e = y * (R2 - np.abs(y) ** 2)
        h = h + mu * gradient(e, X)
        ys.append(y)
    y = np.concatenate(ys, axis=1) if ys else np.zeros((2, 0), dtype=np.complex128)
    return h, y


def output_correlation(y: np.ndarray, max_lag: int) -> float:
    """max over |d| <= max_lag of |rho_d| between the two outputs, second half of y.

    rho_d = sum_n y0[n] conj(y1[n + d]) / sqrt(sum |y0|^2 sum |y1|^2), n over
    the indices where both samples lie in the second half.
    """
    half = y[:, y.shape[1] // 2:]
    L = half.shape[1]
    den = np.sqrt(np.sum(np.abs(half[0]) ** 2) * np.sum(np.abs(half[1]) ** 2))
    if L == 0 or den == 0:
        return 0.0
    best = 0.0
    for d in range(-max_lag, max_lag + 1):
        a = half[0, max(0, -d):L - max(0, d)]
        b = half[1, max(0, d):L - max(0, -d)]
        best = max(best, float(np.abs(np.sum(a * np.conj(b))) / den))
    return best


def rebuild_second_row(h: np.ndarray) -> np.ndarray:
    """Singularity recovery: keep the first row, replace the second by the
    time-reversed conjugates h_yy[k] = conj h_xx[T-1-k], h_yx[k] = -conj h_xy[T-1-k].

    About the centre tap the reversal conjugates the frequency response, so
    the rebuilt 2x2 response is [[H_xx, H_xy], [-conj H_xy, conj H_xx]] at every
    frequency: a scaled unitary whose second row extracts the polarisation the
    first row rejects.
    """
    h2 = h.copy()
    h2[1, 1, :] = np.conj(h[0, 0, ::-1])
    h2[1, 0, :] = -np.conj(h[0, 1, ::-1])
    return h2


def cma_acquire(xbuf, T, L_b, n_blocks, mu, R2, off=0, h0=None):
    """Returns (taps, y_acq, rho, reran). ``h0`` (default: identity taps) starts the first pass."""
    h, y = cma_pass(xbuf, identity_taps(T) if h0 is None else h0, L_b, n_blocks, mu, R2, off)
    rho = output_correlation(y, (T - 1) // 2)
    reran = False
    if rho > 0.5:
        h, y = cma_pass(xbuf, rebuild_second_row(h), L_b, n_blocks, mu, R2, off)
        reran = True
    return h, y, rho, reran


# ----------------------------------------------------------------------------
# A3: frequency offset (4th-power periodogram peak, then the least-squares
# slope of the per-block 4th-power phase)
# ----------------------------------------------------------------------------

def foe_window(xbuf, h, n_acq, T, off):
    """Outputs of the fixed taps h over the second half of the acquisition window."""
    n = np.arange(n_acq // 2, n_acq)
    return butterfly(h, gather(xbuf, n, T, off))


def foe_coarse(y: np.ndarray) -> float:
    nw = y.shape[1]
    nf = 512
    while nf < 2 * nw:
        nf *= 2
    P = np.sum(np.abs(np.fft.fft(y ** 4, n=nf, axis=1)) ** 2, axis=0)
    k = int(np.argmax(P))
    kappa = k if k < nf // 2 else k - nf
    return 2.0 * np.pi * kappa / (4.0 * nf)


def foe_fine(y: np.ndarray, w_c: float, L_b: int) -> float:
    nb = y.shape[1] // L_b
    if nb < 2:
        return 0.0
    n = np.arange(nb * L_b)
    v = (y[:, :nb * L_b] * np.exp(-1j * w_c * n)[None, :]) ** 4
    a = v.reshape(2, nb, L_b).sum(axis=(0, 2))
    phi = np.angle(a)
    for j in range(1, nb):                         # sequential unwrap
        d = phi[j] - phi[j - 1]
        if d > np.pi:
            phi[j:] -= 2.0 * np.pi
        elif d < -np.pi:
            phi[j:] += 2.0 * np.pi
    centre = np.arange(nb) * L_b + (L_b - 1) / 2.0
    cc = centre - centre.mean()
    slope = np.sum(cc * (phi - phi.mean())) / np.sum(cc * cc)
    return float(slope / 4.0)


def foe_code(y: np.ndarray, symbol_rate: float, grid: float, L_b: int):
    """FO code from the fixed-tap window outputs y [2, n].

    Returns (code, w_hat [rad/symbol], distance of w_hat*Rs/(2 pi grid) to the
    rounding boundary, in grid steps).
    """
    if y.shape[1] < 2:
        return 0, 0.0, 0.5
    w_c = foe_coarse(y)
    w = w_c + foe_fine(y, w_c, L_b)
    u = w * symbol_rate / (2.0 * np.pi) / grid
    code = int(np.rint(u))
    return code, w, abs(abs(u - np.floor(u)) - 0.5)


def fo_correct_taps(h: np.ndarray, code: int, grid: float, fs: float) -> np.ndarray:
    T = h.shape[-1]
    c = (T - 1) // 2
    k = np.arange(T)
    return h * np.exp(-1j * 2.0 * np.pi * code * grid * (k - c) / fs)


def derotate(x: np.ndarray, code: int, grid: float, fs: float, g0: int) -> np.ndarray:
    g = g0 + np.arange(x.shape[1], dtype=np.float64)
    return x * np.exp(-1j * 2.0 * np.pi * code * grid * g / fs)[None, :]


# ----------------------------------------------------------------------------
# A4: segmented block DD-LMS
# ----------------------------------------------------------------------------

def decision_margin(u: np.ndarray, m: int) -> np.ndarray:
    """Distance (amplitude units) of each point's nearer component to an interior decision
    boundary of the square-QAM grid, minimised over the last axis. Diagnostic only: it tells
    how close a decision came to flipping; no arithmetic of the receiver uses it."""
    L = qam.n_levels(m)
    a = qam.amp(m)

    def one(v):
        t = (v / a + (L - 1)) / 2.0                       # level coordinate; boundaries at k + 1/2
        b = np.clip(np.floor(t) + 0.5, 0.5, L - 1.5)
        return np.abs(t - b) * 2.0 * a

    return np.minimum(one(np.real(u)), one(np.imag(u))).min(axis=-1)


def _dd_blocks(xbuf, h, n, m, mu, off):
    """One DD-LMS block on a batch of segments. n: [nS, L]; h: [nS, 2, 2, T].
    Returns (y, updated taps, decision margin [nS, 2])."""
    T = h.shape[-1]
    X = gather(xbuf, n, T, off)                       # [nS, 2, L, T]
    y = butterfly(h, X)                               # [nS, 2, L]
    psi = np.angle(-np.sum(y ** 4, axis=-1)) / 4.0    # [nS, 2]
    rot = np.exp(-1j * psi)[..., None]
    d = qam.decide(y * rot, m)
    e = d / rot - y
    return y, h + mu * gradient(e, X), decision_margin(y * rot, m)


def _run_segments(xbuf, h0, starts, n_main, L_b, n_warm, m, mu, off, last_len=None):
    """Segments with identical block structure, vectorised across segments.

    starts: [nS] first symbol of each segment; n_main full blocks each (the
    last one may be cut to ``last_len`` symbols); n_warm warm-up blocks.
    Returns (y, final taps, smallest decision margin of each segment and row [nS, 2]).
    """
    nS = len(starts)
    h = np.broadcast_to(h0, (nS,) + h0.shape).copy()
    margin = np.full((nS, 2), np.inf)
    for w in range(n_warm):
        b0 = starts - (n_warm - w) * L_b
        n = b0[:, None] + np.arange(L_b)[None, :]
        _, h, mg = _dd_blocks(xbuf, h, n, m, mu, off)
        margin = np.minimum(margin, mg)
    ys = []
    for j in range(n_main):
        L = L_b if (last_len is None or j < n_main - 1) else last_len
        n = (starts + j * L_b)[:, None] + np.arange(L)[None, :]
        y, h, mg = _dd_blocks(xbuf, h, n, m, mu, off)
        margin = np.minimum(margin, mg)
        ys.append(y)
    return np.concatenate(ys, axis=-1), h, margin


def dd_lms(xbuf, h_init, n_sym, L_b, seg_blocks, warmup_blocks, m, mu, off=0, diag=None):
    """Returns (y [2, n_sym], final taps of the last segment). When ``diag`` is a dict it receives
    "margin" [nseg, 2]: the smallest decision margin (``decision_margin``) met by each segment and
    row over its warm-up and main blocks."""
    L_seg = seg_blocks * L_b
    y = np.zeros((2, n_sym), dtype=np.complex128)
    if n_sym <= 0:
        return y, h_init.copy()
    nseg = (n_sym + L_seg - 1) // L_seg
    h_last = None
    margin = np.full((nseg, 2), np.inf)

    def place(starts, ys):
        for i, s in enumerate(starts):
            y[:, s:s + ys.shape[-1]] = ys[i]

    def one_segment(s, warm):
        start = s * L_seg
        length = min(L_seg, n_sym - start)
        n_main = (length + L_b - 1) // L_b
        last_len = length - (n_main - 1) * L_b
        ys, h, mg = _run_segments(xbuf, h_init, np.array([start]), n_main, L_b, warm, m, mu, off, last_len)
        place([start], ys)
        margin[s] = mg[0]
        return h[0]

    h_last = one_segment(0, 0)
    full = [s for s in range(1, nseg) if (s + 1) * L_seg <= n_sym]
    if full:
        starts = np.array(full) * L_seg
        ys, hs, mg = _run_segments(xbuf, h_init, starts, seg_blocks, L_b, warmup_blocks, m, mu, off)
        place(starts, ys)
        margin[full] = mg
        h_last = hs[-1]
    if nseg > 1 and nseg - 1 not in full:
        h_last = one_segment(nseg - 1, warmup_blocks)
    if diag is not None:
        diag["margin"] = margin
    return y, h_last


# ----------------------------------------------------------------------------
# Widely-linear segmented DD-LMS (Sec. IV-D: the paper's TD equaliser is
# widely linear, after Silva et al., to undo transmitter IQ imbalance)
# ----------------------------------------------------------------------------
#
# A widely-linear filter is a linear filter on the augmented input
# [x_0, x_1, conj x_0, conj x_1]:
#   y_q[n] = sum_p sum_k h_qp[k] x_p[2n + c - k] + g_qp[k] conj(x_p[2n + c - k]),
# and its LMS update is the linear one on that input:
#   h_qp[k] += mu   * sum_n e_q[n] conj(x_p[2n + c - k]),
#   g_qp[k] += mu_c * sum_n e_q[n] x_p[2n + c - k].
# Taps are [2 (q)][4][T]: [:, 0:2] multiply x_p, [:, 2:4] multiply conj(x_p).
# Phase, decision, error and the segment schedule are the A4 ones above.

def augment(xbuf: np.ndarray) -> np.ndarray:
    """[x_0, x_1] -> [x_0, x_1, conj x_0, conj x_1]."""
    return np.concatenate([xbuf, np.conj(xbuf)], axis=0)


def wl_step(mu: float, mu_conj: float) -> np.ndarray:
    """Step sizes of the four augmented inputs, shaped to broadcast over taps [..., q, 4, T]."""
    return np.array([mu, mu, mu_conj, mu_conj], dtype=np.float64)[:, None]


def wl_identity_taps(T: int) -> np.ndarray:
    h = np.zeros((2, 4, T), dtype=np.complex128)
    h[:, :2] = identity_taps(T)
    return h


def dd_lms_wl(xbuf, h_init, n_sym, L_b, seg_blocks, warmup_blocks, m, mu, mu_conj, off=0, diag=None):
    """Widely-linear A4 on the segment schedule of ``dd_lms``. h_init: [2, 4, T].
    Returns (y [2, n_sym], final taps [2, 4, T] of the last segment)."""
    return dd_lms(augment(xbuf), h_init, n_sym, L_b, seg_blocks, warmup_blocks, m,
                  wl_step(mu, mu_conj), off, diag)
