"""A0 power normalisation and A1 overlap-save FD dispersion compensation, FP64.

TEST INFRASTRUCTURE (see the package docstring).

Paper anchor: the receiver filters block-wise in the frequency domain with a
1024-point FFT and "100 % overlap-save", i.e. 512 valid outputs per block,
with a static FD filter multiplied bin by bin (Sec. III-A); an overlap kernel
carries one block of input across buffer boundaries and converts the ADC
integers to float (Sec. II-D, Steps 3-4). The paper's static filter equalises
the receiver bandwidth; here the FD filter is the chromatic-dispersion
all-pass, which the paper does not treat. Readings taken:

* H_cdc[k] = exp(+j pi D L lambda^2 f_k^2 / c), f_k the signed FFT bin
  frequency k*fs/N (the exact inverse of a fibre of dispersion D*L);
* the same FD multiply also applies the RRC matched filter
  sqrt(sps) * RRC(f_k; rolloff) when rolloff > 0, as the paper's QAM chain
  does matched filtering in its FD static filter (Sec. IV-C);
* a block of N = 2^K samples starts N/4 before the N/2 samples it keeps and
  outputs its centre half [N/4, 3N/4) (the CD impulse response is two-sided);
  a single frame is zero-padded outside [0, S); a stream carries the last N/2
  input samples to the next frame and delays its output by N/4 samples;
* the per-polarisation scale 1/sqrt(P) (A0) uses the mean power P of the
  first 2*N_acq samples of the first frame and is then held.
"""

from __future__ import annotations

import numpy as np

C_LIGHT = 299_792_458.0


def power_scale(x: np.ndarray, n_samples: int) -> np.ndarray:
    """A0: per-polarisation 1/sqrt(mean |x|^2) over the first n_samples samples.

    A polarisation whose window has zero power keeps scale 1.
    """
    n = min(int(n_samples), x.shape[1])
    out = np.ones(x.shape[0])
    for p in range(x.shape[0]):
        P = np.mean(np.abs(x[p, :n]) ** 2) if n > 0 else 0.0
        if P > 0:
            out[p] = 1.0 / np.sqrt(P)
    return out


def rrc_amplitude(f: np.ndarray, symbol_rate: float, rolloff: float) -> np.ndarray:
    """Root-raised-cosine amplitude response, 1 at DC."""
    af = np.abs(f)
    lo = (1.0 - rolloff) * symbol_rate / 2.0
    hi = (1.0 + rolloff) * symbol_rate / 2.0
    out = np.where(af <= lo, 1.0, 0.0)
    band = (af > lo) & (af <= hi)
    out[band] = np.cos(np.pi / (2.0 * rolloff * symbol_rate) * (af[band] - lo))
    return out


def cdc_response(nfft: int, fs: float, dispersion: float, length: float, wavelength: float,
                 symbol_rate: float = 0.0, rolloff: float = 0.0, sps: int = 2) -> np.ndarray:
    """FD filter on the nfft FFT bins (complex128 [nfft]): H_cdc, times the matched filter if rolloff > 0."""
    f = np.fft.fftfreq(nfft, d=1.0 / fs)
    H = np.exp(1j * np.pi * dispersion * length * wavelength**2 * f**2 / C_LIGHT)
    if rolloff > 0:
        H = H * np.sqrt(sps) * rrc_amplitude(f, symbol_rate, rolloff)
    return H


def overlap_save(x: np.ndarray, H: np.ndarray) -> np.ndarray:
    """A1 on one frame: [P, S] -> [P, S], zero-padded outside the frame."""
    nfft = H.shape[0]
    hop, lead = nfft // 2, nfft // 4
    P, S = x.shape
    out = np.zeros((P, S), dtype=np.complex128)
    nblk = (S + hop - 1) // hop
    for j in range(nblk):
        start = j * hop - lead
        seg = np.zeros((P, nfft), dtype=np.complex128)
        lo, hi = max(start, 0), min(start + nfft, S)
        if hi > lo:
            seg[:, lo - start:hi - start] = x[:, lo:hi]
        y = np.fft.ifft(np.fft.fft(seg, axis=1) * H[None, :], axis=1)
        keep = min(hop, S - j * hop)
        out[:, j * hop:j * hop + keep] = y[:, lead:lead + keep]
    return out


def overlap_save_stream(x: np.ndarray, H: np.ndarray, tail: np.ndarray):
    """A1 on one frame of a stream.

    ``tail`` holds the last N/2 input samples of the previous frame (zeros
    before the first). Returns (out [P, S], new tail); out[:, i] is the
    compensated sample at stream index (frame_start - N/4 + i).
    """
    nfft = H.shape[0]
    hop, lead = nfft // 2, nfft // 4
    P, S = x.shape
    if S % hop:
        raise ValueError("stream frames must hold a whole number of N/2 hops")
    v = np.concatenate([tail, x], axis=1)
    out = np.zeros((P, S), dtype=np.complex128)
    for j in range(S // hop):
        seg = v[:, j * hop:j * hop + nfft]
        y = np.fft.ifft(np.fft.fft(seg, axis=1) * H[None, :], axis=1)
        out[:, j * hop:(j + 1) * hop] = y[:, lead:lead + hop]
    return out, v[:, -hop:].copy()
