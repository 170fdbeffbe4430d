"""End-to-end pins of the oracle chain (single frame and stream)."""

import numpy as np
import pytest

from oracle import cdc, theory
from oracle.receiver import Receiver, RxConfig, receive
from synth import generate, workload


def test_qpsk_workload_end_to_end():
    w = workload("dp-qpsk-25gbd")
    fr = generate(w["link"], 1)
    r = receive(fr.samples, RxConfig.from_dict(w["rx"]), fr.ref_words)
    c = r.counts
    assert abs(r.fo_code * 100e3 - w["link"].freq_offset) < 1.5e6
    assert all(s[3] >= 0.99 * r.sync_len for s in r.sync)
    assert {s[0] for s in r.sync} == {0, 1}                       # both polarisations found
    assert 10 * np.log10(c["evm_num"] / c["evm_den"]) < -w["link"].snr_db + 0.3
    assert c["bit_errors"] <= 2
    assert c["bits"] == 2 * 2 * (w["link"].n_sym - 1024)


def test_16qam_workload_reduced_frame_within_half_a_db():
    w = workload("dp-16qam-32gbd", n_sym=1 << 16)
    fr = generate(w["link"], 2)
    r = receive(fr.samples, RxConfig.from_dict(w["rx"]), fr.ref_words)
    c = r.counts
    evm_db = 10 * np.log10(c["evm_num"] / c["evm_den"])
    assert evm_db < -w["link"].snr_db + 0.8
    # BER no worse than theory at 1 dB lower SNR
    assert c["bit_errors"] / c["bits"] <= theory.gray_qam_ber(4, w["link"].snr_db - 1.0) * 3 + 3 / c["bits"]


def test_stream_bookkeeping_with_identity_taps():
    """Stream frames with frozen identity taps: y at global symbol g is the compensated sample 2g."""
    w = workload("dp-64qam-48gbd-stream", n_frames=4, frame_sym=1 << 12)
    fr = generate(w["link"].with_(n_sym=4 << 12), 3)
    cfg = RxConfig.from_dict(dict(w["rx"], cma_blocks=0, mu_dd=0.0, fft_size=1024))
    rx = Receiver(cfg, stream=True)
    S = 2 << 12
    ys = [rx.process(fr.samples[:, f * S:(f + 1) * S]).y for f in range(4)]
    y = np.concatenate(ys, axis=1)
    H = cdc.cdc_response(cfg.fft_size, cfg.fs, cfg.dispersion, cfg.length, cfg.wavelength,
                         cfg.symbol_rate, cfg.rrc_rolloff)
    lead = cfg.fft_size // 4                    # same block placement as the stream
    whole = cdc.overlap_save(np.concatenate([np.zeros((2, lead)), fr.samples], axis=1), H)
    lat = cfg.stream_latency
    g = np.arange(y.shape[1]) - lat
    ok = (g >= 0)
    assert np.max(np.abs(y[:, ok] - whole[:, 2 * g[ok] + lead])) < 1e-12


def test_stream_of_64qam_frames_tracks_and_counts():
    w = workload("dp-64qam-48gbd-stream", n_frames=4, frame_sym=1 << 15)
    fr = generate(w["link"].with_(n_sym=4 << 15), 4)
    cfg = RxConfig.from_dict(w["rx"])
    rx = Receiver(cfg, stream=True)
    S = 2 << 15
    tot = dict(bits=0, bit_errors=0)
    from synth.channel import pack_bits
    for f in range(4):
        ref = pack_bits(fr.bits[:, f * (S // 2) * 6:(f + 1) * (S // 2) * 6])
        r = rx.process(fr.samples[:, f * S:(f + 1) * S], ref)
        tot["bits"] += r.counts["bits"]
        tot["bit_errors"] += r.counts["bit_errors"]
        evm_db = 10 * np.log10(r.counts["evm_num"] / r.counts["evm_den"])
        assert evm_db < -w["link"].snr_db + 1.5
    assert tot["bits"] == 4 * 2 * 6 * ((1 << 15) - 2 * max(512, cfg.stream_latency + 16))
    assert tot["bit_errors"] / tot["bits"] < 10 * theory.gray_qam_ber(6, w["link"].snr_db)
