"""Nonlinear fibre link: symmetric split-step Fourier solution of the Manakov equation.

Channel physics only (no receiver arithmetic). Per step of length h the
field A = [A_x, A_y] (W^0.5) takes a half linear step, a nonlinear step and a
half linear step:
  linear:     A(w) <- A(w) exp((-alpha/2 + j beta2/2 w^2) h/2),  beta2 = -D lambda^2 / (2 pi c)
  nonlinear:  A <- A exp(+j 8/9 gamma (|A_x|^2 + |A_y|^2) h_eff),  h_eff = (1 - e^{-alpha h}) / alpha
(the same sign conventions as the linear channel in ``channel.py``). Step
lengths follow the mean power: h keeps 8/9 gamma P(z) h <= max_phase, capped
by the span end. Every span ends in an EDFA that restores the span loss,
G = e^{alpha L}, and adds complex Gaussian ASE of variance
n_sp h nu (G - 1) f_s per polarisation (n_sp = NF/2, f_s the simulation
sample rate). The link is simulated at ``sim_sps`` samples per symbol
(spectral zero padding of the 2-samples/symbol transmitted field) and
brought back to 2 samples/symbol by spectral truncation.

Two implementations share this module's structure: ``propagate`` on NumPy
(FP64, the reference for tests) and ``propagate_torch`` on torch tensors
(any device/dtype, used to generate long training frames on a GPU).
"""

from __future__ import annotations

from dataclasses import dataclass, replace

import numpy as np

from .channel import C_LIGHT, LinkParams, _streams, haar_unitary, modulate, pack_bits, rrc_spectrum, Frame

H_PLANCK = 6.62607015e-34


@dataclass(frozen=True)
class FibreLink:
    spans: int = 10
    span_km: float = 80.0
    alpha_db_km: float = 0.2
    gamma: float = 1.3                 # 1/(W km)
    nf_db: float = 5.0
    launch_dbm: float = 4.0            # total over both polarisations
    max_phase: float = 1e-3            # rad per step
    sim_sps: int = 4
    ase: bool = True                   # amplifier noise on/off

    def with_(self, **kw) -> "FibreLink":
        return replace(self, **kw)


def _plan(link: FibreLink, p_launch_w: float):
    """Step lengths [m] of one span (they repeat every span)."""
    alpha = link.alpha_db_km / (10.0 * np.log10(np.e)) / 1e3      # 1/m
    gam = link.gamma / 1e3 * 8.0 / 9.0                             # 1/(W m)
    L = link.span_km * 1e3
    steps, z = [], 0.0
    while z < L - 1e-9:
        P = p_launch_w * np.exp(-alpha * z)
        h = L - z if gam * P == 0.0 else min(link.max_phase / (gam * P), L - z)
        steps.append(h)
        z += h
    return alpha, gam, L, steps


def _heff(alpha: float, h: float) -> float:
    return h if alpha == 0.0 else (1.0 - np.exp(-alpha * h)) / alpha


def _ase_var(link: FibreLink, alpha: float, L: float, wavelength: float, fsu: float) -> float:
    if not link.ase:
        return 0.0
    nsp = 10.0 ** (link.nf_db / 10.0) / 2.0
    return nsp * H_PLANCK * (C_LIGHT / wavelength) * (np.exp(alpha * L) - 1.0) * fsu


def propagate(x: np.ndarray, fs: float, wavelength: float, dispersion: float, link: FibreLink,
              rng: np.random.Generator) -> np.ndarray:
    """x: [2, S] field at 2 samples/symbol (any scale) -> received [2, S] field (W^0.5)."""
    S = x.shape[1]
    up = link.sim_sps // 2
    Su = S * up
    fsu = fs * up
    X = np.fft.fft(x, axis=1)
    Xu = np.zeros((2, Su), dtype=np.complex128)
    half = S // 2
    Xu[:, :half] = X[:, :half]
    Xu[:, Su - (S - half):] = X[:, half:]
    a = np.fft.ifft(Xu, axis=1) * up
    p_launch = 1e-3 * 10.0 ** (link.launch_dbm / 10.0)
    a = a * np.sqrt(p_launch / np.mean(np.sum(np.abs(a) ** 2, axis=0)))
    alpha, gam, L, steps = _plan(link, p_launch)
    beta2 = -dispersion * wavelength ** 2 / (2.0 * np.pi * C_LIGHT)
    w = 2.0 * np.pi * np.fft.fftfreq(Su, d=1.0 / fsu)
    G = np.exp(alpha * L)
    ase_var = _ase_var(link, alpha, L, wavelength, fsu)
    for _ in range(link.spans):
        for h in steps:
            lin = np.exp((-alpha / 2.0 + 1j * beta2 / 2.0 * w * w) * (h / 2.0))
            a = np.fft.ifft(np.fft.fft(a, axis=1) * lin[None, :], axis=1)
            heff = _heff(alpha, h)
            a = a * np.exp(1j * gam * np.sum(np.abs(a) ** 2, axis=0) * heff)[None, :]
            a = np.fft.ifft(np.fft.fft(a, axis=1) * lin[None, :], axis=1)
        a = a * np.sqrt(G)
        a = a + np.sqrt(ase_var / 2.0) * (rng.standard_normal((2, Su)) + 1j * rng.standard_normal((2, Su)))
    A = np.fft.fft(a, axis=1)
    Y = np.concatenate([A[:, :half], A[:, Su - (S - half):]], axis=1)
    return np.fft.ifft(Y, axis=1) / up


def propagate_torch(x, fs: float, wavelength: float, dispersion: float, link: FibreLink, noise: list):
    """Same as :func:`propagate` on a torch complex tensor [2, S]; ``noise`` holds one
    [2, S*sim_sps] complex tensor of unit-variance ASE draws per span (drawn by the caller)."""
    import torch
    S = x.shape[1]
    up = link.sim_sps // 2
    Su = S * up
    fsu = fs * up
    X = torch.fft.fft(x, dim=1)
    Xu = torch.zeros((2, Su), dtype=x.dtype, device=x.device)
    half = S // 2
    Xu[:, :half] = X[:, :half]
    Xu[:, Su - (S - half):] = X[:, half:]
    a = torch.fft.ifft(Xu, dim=1) * up
    p_launch = 1e-3 * 10.0 ** (link.launch_dbm / 10.0)
    a = a * float(np.sqrt(p_launch / torch.mean(torch.sum(torch.abs(a) ** 2, dim=0)).item()))
    alpha, gam, L, steps = _plan(link, p_launch)
    beta2 = -dispersion * wavelength ** 2 / (2.0 * np.pi * C_LIGHT)
    w = 2.0 * np.pi * np.fft.fftfreq(Su, d=1.0 / fsu)
    G = np.exp(alpha * L)
    ase_var = _ase_var(link, alpha, L, wavelength, fsu)
    lins = {}
    for si in range(link.spans):
        for h in steps:
            if h not in lins:
                lins[h] = torch.from_numpy(np.exp((-alpha / 2.0 + 1j * beta2 / 2.0 * w * w) * (h / 2.0))).to(
                    device=x.device, dtype=x.dtype)
            lin = lins[h]
            a = torch.fft.ifft(torch.fft.fft(a, dim=1) * lin[None, :], dim=1)
            heff = _heff(alpha, h)
            a = a * torch.exp(1j * gam * heff * torch.sum(torch.abs(a) ** 2, dim=0))[None, :]
            a = torch.fft.ifft(torch.fft.fft(a, dim=1) * lin[None, :], dim=1)
        a = a * float(np.sqrt(G)) + float(np.sqrt(ase_var / 2.0)) * noise[si]
    A = torch.fft.fft(a, dim=1)
    Y = torch.cat([A[:, :half], A[:, Su - (S - half):]], dim=1)
    return torch.fft.ifft(Y, dim=1) / up


def transmit(p: LinkParams, seed: int):
    """Bits, symbols and the RRC-shaped 2-samples/symbol field (before the fibre)."""
    rng_bits, rng_jones, rng_phase, rng_awgn, rng_nl = _streams(seed)
    m = p.bits_per_sym
    bits = rng_bits.integers(0, 2, size=(2, p.n_sym * m), dtype=np.uint8)
    symbols = modulate(bits, m)
    x = np.zeros((2, p.n_samp), dtype=np.complex128)
    x[:, ::p.sps] = symbols
    f = np.fft.fftfreq(p.n_samp, d=1.0 / p.fs)
    x = np.fft.ifft(np.fft.fft(x, axis=1) * (np.sqrt(p.sps) * rrc_spectrum(f, p.symbol_rate, p.rolloff))[None], axis=1)
    return bits, symbols, x, (rng_jones, rng_phase, rng_awgn, rng_nl)


def receive_front(x: np.ndarray, p: LinkParams, rngs) -> tuple:
    """Jones rotation, laser phase noise and frequency offset at the receiver."""
    rng_jones, rng_phase, _, _ = rngs
    J = haar_unitary(rng_jones) if p.jones else np.eye(2, dtype=np.complex128)
    x = J @ x
    S = x.shape[1]
    i = np.arange(S, dtype=np.float64)
    wiener = np.cumsum(rng_phase.normal(0.0, np.sqrt(2.0 * np.pi * p.linewidth / p.fs), size=S)) \
        if p.linewidth > 0 else np.zeros(S)
    phase = 2.0 * np.pi * p.freq_offset * i / p.fs + wiener
    return x * np.exp(1j * phase)[None, :], J, phase


def generate_nonlinear(p: LinkParams, link: FibreLink, seed: int, device: str | None = None) -> Frame:
    """A frame through the nonlinear link (NumPy FP64, or torch on ``device`` for long frames)."""
    bits, symbols, x, rngs = transmit(p, seed)
    rng_nl = rngs[3]
    if device is None:
        y = propagate(x, p.fs, p.wavelength, p.dispersion, link, rng_nl)
    else:
        import torch
        Su = p.n_samp * (link.sim_sps // 2)
        noise = [torch.from_numpy(rng_nl.standard_normal((2, Su)) + 1j * rng_nl.standard_normal((2, Su)))
                 .to(device=device, dtype=torch.complex64) for _ in range(link.spans)]
        xt = torch.from_numpy(x).to(device=device, dtype=torch.complex64)
        y = propagate_torch(xt, p.fs, p.wavelength, p.dispersion, link, noise).cpu().numpy().astype(np.complex128)
    y, J, phase = receive_front(y, p, rngs)
    return Frame(params=p, seed=seed, samples=y, bits=bits, ref_words=pack_bits(bits), symbols=symbols, jones=J,
                 phase=phase, noise_var=np.zeros(2), extra={"fibre": link})
