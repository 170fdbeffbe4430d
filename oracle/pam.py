"""IM/DD PAM-M chain with frequency-domain clock recovery (Sec. III, Steps 1-9), FP64.

TEST INFRASTRUCTURE (see the package docstring).

The paper's chain at 2 samples/symbol: 1024-point 100 % overlap-save FFT;
static FD equaliser; block-wise clock-phase estimate in the frequency domain
(by the method of its cited reference, whose equations the paper does not
give); the estimates averaged over 105 blocks (52 before, 52 after) by
vector addition and unwrapped; clock recovery as a phase ramp in the
frequency domain, IFFT, extraction of 256 symbols per block give or take a
slip; buffer-wise DC and amplitude normalisation; PAM decision with
thresholds and demapping. Readings taken:

* v = scale * code + dc (12-bit codes, static offset); blocks as in
  ``cdc.overlap_save`` (block j from j N/2 - N/4, zero outside the frame);
* the static FD equaliser is the RRC matched filter sqrt(2) RRC(f) (its
  offline-optimised 503 taps need the lab receiver);
* clock phase of block j: c_j = sum_{k < N/2} X_j[k] conj(X_j[k + N/2]) on
  the filtered spectrum (the spectral-line estimator: spectral components one
  symbol rate apart correlate, with phase -2 pi Rs tau for a delay tau);
* averaging: cbar_j = sum of c_i over |i - j| <= 52 inside the frame,
  phi_j = arg cbar_j in (-pi, pi];
* unwrapping in integers: w_0 = 0, w_j = w_{j-1} - 1 if phi_j - phi_{j-1} >
  pi, + 1 if < -pi, else unchanged; the unwrapped phase is phi_j + 2 pi w_j;
* clock recovery: block j's filtered spectrum times exp(-j phi_j f_k / Rs)
  (advances the signal by the residual delay; f_k / Rs = k_signed / (N/2)),
  inverse transform, real part;
* variable-rate extraction: the residual correction leaves symbol k at slot
  m = k - w_j (time m T) of block j (the unwrapped delay is the residual one
  minus w_j symbols); block j outputs the symbols k = j N/4 + w_j ..
  (j+1) N/4 + w_{j+1} - 1, i.e. its block-local samples N/4 + 2 i for
  i < N/4 + w_{j+1} - w_j (255, 256 or 257 symbols); the last block outputs
  N/4 (clipped to the frame); output i of block j sits at O_j + i,
  O_j = j N/4 + w_j - w_0;
* normalisation over the buffer's outputs: mean, then the mean absolute
  deviation mapped to M/2 (the mean |level| of uniform PAM-M):
  u = (y - mean) * (M/2) / mean|y - mean|;
* decision at the level midpoints (the offline-optimised thresholds need the
  lab receiver): level index l = clip(round((u + M - 1) / 2), 0, M - 1),
  Gray word l ^ (l >> 1), most significant bit first.
"""

from __future__ import annotations

import numpy as np

from .cdc import rrc_amplitude

AVG_HALF = 52


def front_end(codes: np.ndarray, scale: float, dc: float) -> np.ndarray:
    return scale * codes.astype(np.float64) + dc


def blocks(v: np.ndarray, N: int) -> np.ndarray:
    """[J, N] overlap-save input blocks (zero outside the frame)."""
    S = v.shape[0]
    hop, lead = N // 2, N // 4
    J = (S + hop - 1) // hop
    out = np.zeros((J, N))
    for j in range(J):
        start = j * hop - lead
        lo, hi = max(start, 0), min(start + N, S)
        if hi > lo:
            out[j, lo - start:hi - start] = v[lo:hi]
    return out


def matched_response(N: int, rolloff: float) -> np.ndarray:
    """sqrt(2) RRC(f_k), symbol rate fs/2."""
    return np.sqrt(2.0) * rrc_amplitude(np.fft.fftfreq(N, d=1.0), 0.5, rolloff)


def clock_products(X: np.ndarray) -> np.ndarray:
    """c_j = sum_{k < N/2} X_j[k] conj(X_j[k + N/2])."""
    N = X.shape[1]
    return np.sum(X[:, :N // 2] * np.conj(X[:, N // 2:]), axis=1)


def average(c: np.ndarray, half: int = AVG_HALF) -> np.ndarray:
    J = c.shape[0]
    out = np.zeros(J, dtype=np.complex128)
    for j in range(J):
        out[j] = np.sum(c[max(0, j - half):min(J, j + half + 1)])
    return out


def winding(phi: np.ndarray) -> np.ndarray:
    w = np.zeros(phi.shape[0], dtype=np.int64)
    for j in range(1, phi.shape[0]):
        d = phi[j] - phi[j - 1]
        w[j] = w[j - 1] + (-1 if d > np.pi else (1 if d < -np.pi else 0))
    return w


def correct(X: np.ndarray, phi: np.ndarray) -> np.ndarray:
    """Blocks' time signals after the residual clock correction exp(-j phi_j f_k / Rs)."""
    N = X.shape[1]
    k = np.arange(N)
    ks = np.where(k < N // 2, k, k - N).astype(np.float64)
    ks[N // 2] = 0.0                                    # the Nyquist bin (zero after the matched filter)
    ramp = np.exp(-1j * phi[:, None] * ks[None, :] / (N // 2))
    return np.real(np.fft.ifft(X * ramp, axis=1))


def extract(y_blocks: np.ndarray, w: np.ndarray, n_out_slots: int) -> np.ndarray:
    """Variable-rate extraction; n_out_slots = slots of the frame's kept range (S/2)."""
    J, N = y_blocks.shape
    q = N // 4
    out = []
    for j in range(J):
        wn = w[j + 1] if j + 1 < J else w[j]
        n = q + wn - w[j] if j + 1 < J else q
        n = min(n, n_out_slots - j * q) if j == J - 1 else n
        for i in range(max(n, 0)):
            out.append(y_blocks[j, q + 2 * i])
    return np.array(out)


def normalise(y: np.ndarray, M: int) -> np.ndarray:
    mu = np.mean(y)
    return (y - mu) * (M / 2.0) / np.mean(np.abs(y - mu))


def decide(u: np.ndarray, M: int):
    """(level index, bits [len * log2 M]) at the midpoint thresholds, Gray demapped."""
    l = np.clip(np.rint((u + (M - 1)) / 2.0), 0, M - 1).astype(np.int64)
    g = l ^ (l >> 1)
    m = int(np.log2(M))
    bits = ((g[:, None] >> np.arange(m - 1, -1, -1)[None, :]) & 1).astype(np.uint8).reshape(-1)
    return l, bits


def pam_receive(codes: np.ndarray, scale: float, dc: float, M: int, rolloff: float, N: int = 1024) -> dict:
    """Steps 1-9. Returns the per-block clock products, averaged phases, winding numbers, the
    extracted samples, their normalised values, level indices and bits."""
    v = front_end(codes, scale, dc)
    X = np.fft.fft(blocks(v, N), axis=1) * matched_response(N, rolloff)[None, :]
    c = clock_products(X)
    phi = np.angle(average(c))
    w = winding(phi)
    y = extract(correct(X, phi), w, codes.shape[0] // 2)
    u = normalise(y, M)
    lev, bits = decide(u, M)
    return dict(c=c, phi=phi, w=w, y=y, u=u, levels=lev, bits=bits)
