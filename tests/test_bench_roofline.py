"""The bench's roofline arithmetic on the CPU: the algorithmic work each stage is credited with, and the
fractions against the peaks, for the 16QAM 32 GBd frame of 2^20 symbols per polarisation."""

from __future__ import annotations

import pytest

import bench
from synth.workloads import workload

PK = {"hbm_gbs": 6790.0, "sm_max_mhz": 2070.0}
N = 1 << 20


@pytest.fixture(scope="module")
def w():
    return workload("dp-16qam-32gbd")


def test_lms_stages_count_64_T_flop_per_dp_symbol(w):
    T, Lb = w["rx"]["n_taps"], w["rx"]["lms_block"]
    r = bench.stage_roofline("dd_acq", 1.0, w, N, PK, None)
    # 2 output rows x (outputs + gradient), 2T complex MACs of 8 flop each, per symbol of 128 blocks
    assert r["algorithmic_flops"] == w["rx"]["dd_acq_blocks"] * Lb * 64 * T
    assert r["bound"] == "alu" and r["occupied_sms"] == 2
    assert r["peak"] == pytest.approx(152 * 128 * 2 * 2.07e9 / 1e12)
    assert r["frac_of_occupied_sms"] == pytest.approx(r["frac"] * 76)
    seg = bench.stage_roofline("lms", 1.0, w, N, PK, None)
    assert seg["algorithmic_flops"] == pytest.approx(N * (1 + 4 / 16) * 64 * T)


def test_hbm_stages_count_compulsory_bytes(w):
    fft, Lb = w["rx"]["fft_size"], w["rx"]["lms_block"]
    acq = 2 * max(w["rx"]["cma_blocks"], w["rx"]["dd_acq_blocks"]) * Lb + fft
    first = bench.stage_roofline("cdc", 1.0, w, N, PK, None)
    rest = bench.stage_roofline("cdc_rest", 1.0, w, N, PK, None)
    # both FD compensation parts together read and write every sample of both polarisations once
    assert first["algorithmic_bytes"] + rest["algorithmic_bytes"] == 2 * (2 * N) * 8 * 2
    assert first["algorithmic_bytes"] == 2 * acq * 8 * 2
    power = bench.stage_roofline("power", 1.0, w, N, PK, None)
    assert power["algorithmic_bytes"] == 2 * (2 * w["rx"]["cma_blocks"] * Lb) * 8
    assert power["frac"] == pytest.approx(power["achieved"] / 6790.0)


def test_whole_step_hbm_roofline():
    r = bench.hbm_step_roofline(35_651_584, 0.707, PK)
    assert r["achieved"] == pytest.approx(35_651_584 / 0.707e-3 / 1e9)
    assert r["frac"] == pytest.approx(r["achieved"] / 6790.0) and r["bound"] == "hbm"
