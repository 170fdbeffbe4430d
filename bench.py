"""Throughput benchmark of the dual-polarisation coherent receiver on GB300.

Workload: DP-16QAM at 32 GBd, one frame of 2^20 symbols per polarisation at
2 samples/symbol (complex64), 80 km SSMF dispersion, Jones rotation, 100 kHz
linewidth, 500 MHz offset, SNR 20 dB; FFT 4096 (50 % overlap), 21-tap 2x2
MIMO with 128-symbol blocks, 64 BPS phases over 64 symbols. Synthetic, seeded.

A step is one rx_process call over the whole frame (every stage A0-A6,
including the per-frame acquisition, alignment and BER counting). `value` is
decided line rate (2 * m * N bits per frame, edges included) over the CUDA
event time of the step with the input already in HBM; `e2e` is the same
metric through rx_process_host from pinned host memory, copies included. L2
is flushed (a 512 MiB write) between timed steps, outside the timed region.

`--impl reference` times the FP64 CPU oracle (the reference arm here) on a
bounded sample of the same workload on the host cores.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "dp-16qam-32gbd"
SEED = 1
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
SM_COUNT_GB300 = 152          # used only when no device is visible (CPU tests of the arithmetic)
FP32_LANES_PER_SM = 128


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-forms", action="store_true",
                    help="frame workload only: skip the precision, batched and learned forms (profiling runs)")
    ap.add_argument("--n-sym", type=int, default=0, help="smaller frame for profiling captures (not a bench line)")
    ap.add_argument("--workload", default="frame",
                    choices=["frame", "stream", "batch", "inflight", "learned", "cnn", "wl", "kk", "ingest", "pam",
                             "forms"],
                    help="frame: the 16QAM frame (the bench line); stream: 64QAM int8/FP16 stream of 64 frames; "
                         "batch: 16 channels in one graph launch; inflight: --frames independent 16QAM frames in "
                         "one graph launch; learned: split-step link, chain + "
                         "trained post-equaliser; cnn: the post-equaliser forward alone; wl: the "
                         "widely-linear segmented DD-LMS alone on an IQ-imbalanced 16QAM frame; kk: the "
                         "Kramers-Kronig front end on a 2^22-sample 12-bit buffer; ingest: real-time ingest "
                         "emulation of 2^22-sample buffers at 4 GSa/s through the KK front end; pam: the IM/DD "
                         "PAM-4 chain with FD clock recovery on a 2^22-sample buffer")
    ap.add_argument("--launch-dbm", type=float, default=4.0, help="launch power of the learned workload")
    ap.add_argument("--train-steps", type=int, default=3000, help="Adam steps of the learned workload")
    ap.add_argument("--window", type=int, default=16384, help="symbols per training step of the learned workload")
    ap.add_argument("--lr", type=float, default=7e-4, help="initial Adam learning rate of the learned workload")
    ap.add_argument("--frames", type=int, default=4, help="frames in flight of the inflight workload")
    ap.add_argument("--fmt", default="i8", choices=["i8", "f16", "c64"], help="input format of the stream workload")
    ap.add_argument("--wl-taps", type=int, default=21, help="tap count of the wl workload")
    ap.add_argument("--wl-threads", type=int, default=0,
                    help="CTA size of the wl workload (0: library choice; 512 runs the generic kernel)")
    return ap.parse_args()


def peaks():
    try:
        return json.load(open(PEAKS_FILE))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "fallback": True}


# --------------------------------------------------------------------------------------
# CPU baseline / reference arm: the FP64 oracle on a bounded sample
# --------------------------------------------------------------------------------------

CPU_SAMPLE_SYMBOLS = 1 << 18


def oracle_worker(n_sym: int, reps: int) -> dict:
    from oracle.receiver import Receiver, RxConfig
    from synth import generate, workload
    w = workload(WORKLOAD, n_sym=n_sym)
    fr = generate(w["link"], SEED)
    cfg = RxConfig.from_dict(w["rx"])
    rx = Receiver(cfg)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        rx.process(fr.samples, fr.ref_words)
        times.append(time.perf_counter() - t0)
    bits = 2 * w["link"].bits_per_sym * n_sym
    return dict(times=times, bits=bits)


def run_oracle_subprocess(n_sym: int, reps: int) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.oracle_worker(%d, %d)))" % (ROOT, n_sym, reps))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def cpu_baseline(reps: int = 3) -> dict:
    res = run_oracle_subprocess(CPU_SAMPLE_SYMBOLS, reps)
    t = statistics.median(res["times"])
    return {"value": res["bits"] / t / 1e9, "unit": "Gb/s", "cores": 1, "kind": "oracle",
            "sample": f"{WORKLOAD} frame of {CPU_SAMPLE_SYMBOLS} symbols/pol (of 2^20), full chain A0-A6 in FP64 "
                      f"NumPy, single thread, median of {reps}"}


def reference_arm(args) -> None:
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    res = run_oracle_subprocess(CPU_SAMPLE_SYMBOLS, args.warmup + args.steps)
    times = res["times"][args.warmup:]
    t = sum(times) / len(times)
    v = res["bits"] / t / 1e9
    line = {"metric": "processed line rate", "value": v, "unit": "Gb/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "symbols_per_pol": CPU_SAMPLE_SYMBOLS, "sample_of": 1 << 20},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "Gb/s", "cores": 1, "kind": "oracle",
                             "sample": f"{CPU_SAMPLE_SYMBOLS} symbols/pol per step, FP64 NumPy, single thread"},
            "e2e": {"value": v, "unit": "Gb/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


# --------------------------------------------------------------------------------------
# clocks during the timed region
# --------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            # a timed region of a few milliseconds falls between two 100 ms samples: take the first
            # sample before it starts and (on exit) one after it ends, so the record brackets it
            t0 = time.time()
            while not self.lines and self.proc.poll() is None and time.time() - t0 < 3.0:
                time.sleep(0.005)
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            n, t0 = len(self.lines), time.time()
            while len(self.lines) == n and self.proc.poll() is None and time.time() - t0 < 0.5:
                time.sleep(0.005)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# --------------------------------------------------------------------------------------
# roofline of a stage
# --------------------------------------------------------------------------------------

# DRAM traffic per launch from one ncu capture (profiles/), valid while the kernel's source file is
# unchanged since the capture: stage -> (source file, sha1 of it at capture, bytes read + written).
PROFILED_TRAFFIC = {
    # DRAM bytes read + written, one ncu capture of this launch
    "dd_acq": ("k_lms_tile.cuh", "b23aec6f6da92bcbfffa6aceeb6794cf68d1c9cd", 563456),
    # captured on the 2^18-symbol frame (4,316,416 B: the equalised symbols read once, under ncu's
    # cache flush) and scaled by the symbols of the 2^20-symbol launch (traffic in proportion)
    "bps": ("k_bps.cu", "a6a86046abed1084d0a65f4aa2c6ebe9be2e1228", 17265664),
    "wl": ("k_lms_fast.cuh", "fca5f277b4ecd771cc2e0b0acdff6c7ea8cf98cc", 33638912),
}


def _traffic(stage: str):
    import hashlib
    rec = PROFILED_TRAFFIC.get(stage)
    if not rec:
        return None
    path = os.path.join(ROOT, "paper_2011_13695_gb300", "csrc", rec[0])
    try:
        sha = hashlib.sha1(open(path, "rb").read()).hexdigest()
    except OSError:
        return None
    return rec[2] if sha == rec[1] else None


def fp32_peak(pk: dict) -> tuple[float, float, int, str]:
    """(FP32 flop/s peak, lane-op/s peak, SM count, note). The measured FMA rate when the bench
    measured it (``measure_fp32_peak``), else the unit count: SMs x 128 lanes x 2 flops x max clock."""
    sms = int(pk.get("sm_count", SM_COUNT_GB300))
    if pk.get("fp32_flops"):
        f = float(pk["fp32_flops"])
        return f, f / 2, sms, (f"measured: FMA-chain microkernel on every SM ({pk.get('fp32_form', '')}), "
                               f"{f / 1e12:.1f} TFLOP/s at SM clock {pk.get('fp32_sm_mhz')} MHz")
    clock_mhz = pk.get("sm_max_mhz", 2070.0)
    lanes = sms * FP32_LANES_PER_SM * clock_mhz * 1e6
    return 2 * lanes, lanes, sms, f"nominal: {sms} SMs x 128 lanes x 2 flops x {clock_mhz:.0f} MHz"


def measure_fp32_peak(rx, stream_handle, device_index: int = 0) -> dict:
    """FP32 FMA throughput of this GPU through the library's microkernel (scalar and packed FP32x2
    FMA chains on every SM), the SM clock sampled during it: the denominator of the ALU rooflines."""
    import torch
    sms = torch.cuda.get_device_properties(device_index).multi_processor_count
    best = {}
    with ClockSampler(device_index) as clk:
        for packed in (False, True):
            rates = [rx.rx_fp32_fma_rate(packed, 1 << 16, stream_handle)[0] for _ in range(3)]
            best["packed" if packed else "scalar"] = max(rates)
    form = max(best, key=best.get)
    return {"fp32_flops": best[form], "fp32_form": form, "fp32_scalar_flops": best["scalar"],
            "fp32_packed_flops": best["packed"], "sm_count": sms, "fp32_sm_mhz": clk.summary().get("sm_mhz")}


def stage_roofline(stage: str, ms: float, w: dict, n_sym: int, pk: dict, sm_mhz: float | None) -> dict:
    """Roofline of one stage's dominant kernel: algorithmic work of one launch over its duration.

    FP32 arithmetic is counted in flops (an FMA is 2) against the FMA pipes' peak (measured by the
    FMA-chain microkernel when available, else SMs x 128 lanes x 2 flops x max SM clock); BPS, whose
    work is compare/round/select as much as FMA, in lane-operations against half that flop rate;
    HBM-bound stages in compulsory bytes against the measured copy bandwidth."""
    rxs = w["rx"]
    m = rxs["bits_per_sym"]
    T, Lb = rxs["n_taps"], rxs["lms_block"]
    flop_peak, lane_peak, sms, note = fp32_peak(pk)
    t = ms * 1e-3
    lms_flops_per_symbol = 2 * (16 * T + 16 * T)          # 2 rows x (outputs + gradient), 2T complex MACs each
    alu = {
        # serial block recursions: one CTA per output row, blocks one after another
        "cma": ("k_lms (CMA acquisition, serial blocks)", rxs["cma_blocks"] * Lb * lms_flops_per_symbol),
        "dd_acq": ("k_lms (DD acquisition, serial blocks)", rxs["dd_acq_blocks"] * Lb * lms_flops_per_symbol),
        "lms": ("k_lms (segmented DD-LMS)",
                n_sym * (1 + rxs["warmup_blocks"] / rxs["seg_blocks"]) * lms_flops_per_symbol),
    }
    if stage in alu:
        name, flops = alu[stage]
        peak = flop_peak / 1e12
        a = flops / t / 1e12
        r = {"kernel": name, "bound": "alu", "achieved": a, "peak": peak, "unit": "TFLOP/s", "frac": a / peak,
             "traffic": _traffic(stage), "algorithmic_flops": flops, "peak_note": "FP32 FMA pipes, " + note}
        if stage in ("cma", "dd_acq"):
            # a serial chain of block steps, one CTA (holding a whole SM) per output row: the fraction of
            # the two SMs it can occupy is the meaningful one
            r["occupied_sms"] = 2
            r["frac_of_occupied_sms"] = a / (peak * 2 / sms)
        return r
    if stage == "bps":
        ops = 2 * n_sym * rxs["bps_phases"] * 16          # lane-ops per (symbol, test phase)
        peak = lane_peak / 1e12
        a = ops / t / 1e12
        return {"kernel": "k_bps2", "bound": "alu", "achieved": a, "peak": peak, "unit": "Tops/s",
                "frac": a / peak, "traffic": _traffic(stage), "algorithmic_ops": ops,
                "peak_note": "lane-operations: half the FP32 flop peak, " + note}
    # FD compensation: the acquisition's blocks first ("cdc": its window plus one FFT of reach), the
    # rest beside the acquisition ("cdc_rest"); the power estimate reads the CMA window only
    acq_samples = min(2 * n_sym, 2 * max(rxs["cma_blocks"], rxs["dd_acq_blocks"]) * Lb + rxs["fft_size"])
    byts = {"cdc": 2 * acq_samples * 8 * 2, "cdc_rest": 2 * (2 * n_sym - acq_samples) * 8 * 2,
            "power": 2 * min(2 * n_sym, 2 * rxs["cma_blocks"] * Lb) * 8, "unwrap": 2 * n_sym * (8 + 1 + 8 + 4),
            "count": 2 * n_sym * 8 + 2 * 2 * n_sym * m / 8, "sync": 0, "foe": 0}.get(stage, 0)
    a = byts / t / 1e9 if t > 0 else 0.0
    peak = pk.get("hbm_gbs", 6800.0)
    return {"kernel": stage, "bound": "hbm", "achieved": a, "peak": peak, "unit": "GB/s", "frac": a / peak,
            "traffic": _traffic(stage), "algorithmic_bytes": byts}


# --------------------------------------------------------------------------------------
# replicas on several GPUs (host side; the data path has no collective)
# --------------------------------------------------------------------------------------

def max_over_ranks(values, dist=None, device="cpu"):
    """Each value replaced by its maximum over the ranks of the process group (the job's time is its
    slowest replica's); without a process group the values are returned unchanged."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def free_port() -> int:
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def _spawned_rank(rank: int, world: int, port: int, fn, fn_args: tuple) -> None:
    os.environ.update(RANK=str(rank), LOCAL_RANK=str(rank), WORLD_SIZE=str(world), LOCAL_WORLD_SIZE=str(world),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    fn(*fn_args)


def spawn_ranks(world: int, fn, *fn_args) -> None:
    """Run fn(*fn_args) in `world` processes that see the rendezvous environment torchrun gives its
    ranks (RANK = LOCAL_RANK, WORLD_SIZE, MASTER_ADDR 127.0.0.1, a free MASTER_PORT): one replica per
    GPU of this host when bench.py is started without torchrun."""
    import torch.multiprocessing as mp
    mp.spawn(_spawned_rank, args=(world, free_port(), fn, fn_args), nprocs=world, join=True)


def hbm_step_roofline(bytes_per_step: int, ms_per_step: float, pk: dict) -> dict:
    """A whole step's compulsory HBM bytes over its time, against the measured copy bandwidth."""
    gbs = bytes_per_step / (ms_per_step * 1e-3) / 1e9
    peak = pk.get("hbm_gbs", 6800.0)
    return {"bound": "hbm", "bytes_per_step": bytes_per_step, "achieved": gbs, "peak": peak, "unit": "GB/s",
            "frac": gbs / peak}


def chain_flops_per_dp_symbol(rxs: dict) -> float:
    """Algorithmic FP32 flops per DP symbol of the chain: the FD compensation's FFT pair and multiply
    ((20 log2 N_fft + 12) x 4 per symbol: two polarisations, 2 samples/symbol, half of each block kept),
    the butterfly's outputs and gradient (64 T) and BPS (36 B)."""
    import math
    return (20 * math.log2(rxs["fft_size"]) + 12) * 4 + 64 * rxs["n_taps"] + 36 * rxs["bps_phases"]


def alu_step_roofline(w: dict, n_sym: int, ms_per_step: float, pk: dict) -> dict:
    flops = n_sym * chain_flops_per_dp_symbol(w["rx"])
    peak = fp32_peak(pk)[0]
    a = flops / (ms_per_step * 1e-3)
    return {"bound": "alu", "flops_per_step": flops, "achieved": a / 1e12, "peak": peak / 1e12, "unit": "TFLOP/s",
            "frac": a / peak}


def replica_line_rate(world: int, bits_per_step: int, steps: int, total_ms: float) -> float:
    """Whole-job line rate in Gb/s: every rank processes its own frame of bits_per_step bits per step,
    and the job takes the slowest rank's time for the steps."""
    return world * bits_per_step * steps / (total_ms * 1e-3) / 1e9


# --------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------

def our_arm(args) -> None:
    import numpy as np
    import torch

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.receiver import Receiver
    from synth import generate, workload

    w = workload(WORKLOAD, **({"n_sym": args.n_sym} if args.n_sym else {}))
    link = w["link"]
    N = link.n_sym
    m = link.bits_per_sym
    fr = generate(link, SEED + rank)
    x_host = np.ascontiguousarray(fr.samples.astype(np.complex64))
    ref_host = np.ascontiguousarray(fr.ref_words.astype(np.uint32))
    x = torch.from_numpy(x_host.view(np.float32)).cuda()
    ref = torch.from_numpy(ref_host.view(np.int32)).cuda()
    rcv = Receiver(w["rx"], N)
    out = torch.zeros(2 * rcv.words(N), dtype=torch.int32, device="cuda")
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    bits_per_step = 2 * m * N

    def barrier():
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    # device-resident steps (the library replays each frame's launches as one CUDA graph)
    for _ in range(args.warmup):
        rcv.process(x, N, ref, out)
    barrier()
    launches0 = rx.rx_launch_count(rcv.h)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            rcv.process(x, N, ref, out)
            evs[i][1].record(stream)
        barrier()
    launches = rx.rx_launch_count(rcv.h) - launches0
    step_ms = [a.elapsed_time(b) for a, b in evs]
    total_ms = sum(step_ms)
    # per-stage kernel times: a second timed pass of the same steps with CUDA events between the
    # stages on the streams they run on (the events cost time, so the headline pass runs without them)
    rx.rx_set_timing(rcv.h, True)
    rcv.process(x, N, ref, out)
    barrier()
    rx.rx_set_timing(rcv.h, True)
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        rcv.process(x, N, ref, out)
    barrier()
    stages = rx.rx_stage_times(rcv.h)
    rx.rx_set_timing(rcv.h, False)
    total_ms = max_over_ranks([total_ms], dist, "cuda")[0]
    st = rcv.stats()

    # end to end from pinned host memory
    xh = torch.from_numpy(x_host.view(np.float32)).pin_memory()
    rh = torch.from_numpy(ref_host.view(np.int32)).pin_memory()
    oh = torch.zeros(2 * rcv.words(N), dtype=torch.int32).pin_memory()
    e2e_ms = float("nan")
    if not args.no_e2e:
        for _ in range(args.warmup):
            rcv.process_host(xh, N, rh, oh)
        barrier()
        e_evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                 for _ in range(args.steps)]
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            e_evs[i][0].record(stream)
            rcv.process_host(xh, N, rh, oh)
            e_evs[i][1].record(stream)
        barrier()
        e2e_ms = sum(a.elapsed_time(b) for a, b in e_evs)
    e2e_ms = max_over_ranks([e2e_ms], dist, "cuda")[0]

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return
    pk = dict(peaks(), **measure_fp32_peak(rx, stream.cuda_stream, local))
    csum = clk.summary()
    per_stage = {k: v[0] / max(v[1], 1) for k, v in stages.items() if v[1] > 0}
    # the dominant kernel: the longest stage that is one kernel launch ("cma" also holds the
    # singularity check, its rerun and the tap rebuild; "unwrap", "sync" and "foe" are several launches)
    single = {k: v for k, v in per_stage.items() if k in ("dd_acq", "lms", "bps", "cdc", "cdc_rest", "count", "power")}
    dom = max(single or per_stage, key=(single or per_stage).get)
    roof = stage_roofline(dom, per_stage[dom], w, N, pk, csum.get("sm_mhz"))
    roof["peak_source"] = ("fallback" if pk.get("fallback") else
                           "measured: HBM copy from MEASURED_PEAKS.json, FP32 FMA rate by the FMA-chain microkernel")
    value = replica_line_rate(world, bits_per_step, args.steps, total_ms)
    e2e = replica_line_rate(world, bits_per_step, args.steps, e2e_ms) if e2e_ms == e2e_ms else None
    line = {
        "metric": "processed line rate", "value": value, "unit": "Gb/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "symbols_per_pol": N, "bits_per_sym": m, "symbol_rate_gbd": 32,
                   "fft": 4096, "taps": 21, "bps_phases": 64, "parallelism": f"replicas{world}",
                   "l2": "flushed between timed steps (512 MiB write)",
                   "stage_times": "second pass of the same steps with per-stage CUDA events"},
        "e2e": {"value": e2e, "unit": "Gb/s", "h2d_bytes_per_step": int(x_host.nbytes + ref_host.nbytes),
                "d2h_bytes_per_step": int(oh.numel() * 4)},
        "gpu_launches": int(launches),
        "roofline": roof,
        # the whole step against HBM: its compulsory bytes (the frame's samples and reference bits in,
        # the decided bits out) over the step time; the chain is ALU- and latency-bound, so this is small
        "hbm_roofline": hbm_step_roofline(int(x_host.nbytes + ref_host.nbytes + 2 * rcv.words(N) * 4),
                                          total_ms / args.steps, pk),
        # the whole step against the FP32 FMA peak: the chain's algorithmic flops per DP symbol (FFT pair
        # of the FD compensation, butterfly outputs and gradient, BPS) over the step time
        "alu_roofline": alu_step_roofline(w, N, total_ms / args.steps, pk),
        "fp32_peak": {"tflops": pk["fp32_flops"] / 1e12, "form": pk["fp32_form"],
                      "scalar_tflops": pk["fp32_scalar_flops"] / 1e12, "packed_tflops": pk["fp32_packed_flops"] / 1e12,
                      "sm_count": pk["sm_count"], "sm_mhz": pk["fp32_sm_mhz"]},
        "stage_ms": {k: round(v, 4) for k, v in per_stage.items()},
        # every stage against its own bound (algorithmic work of the stage over its time)
        "stage_roofline": {k: {"bound": r["bound"], "frac": round(r["frac"], 5), "unit": r["unit"],
                               "achieved": round(r["achieved"], 3)}
                           for k, r in ((k, stage_roofline(k, v, w, N, pk, csum.get("sm_mhz")))
                                        for k, v in per_stage.items() if k not in ("sync", "foe"))},
        "ber": st["ber"], "evm": st["evm"], "fo_code": st["fo_code"],
        "clocks": csum,
    }
    if not args.no_cpu_baseline and world == 1:
        try:
            line["cpu_baseline"] = cpu_baseline()
        except Exception as e:  # report, do not hide
            line["cpu_baseline"] = {"error": str(e)[:300]}
    if not args.no_forms and world == 1 and not args.n_sym:
        line["forms"] = other_forms(args)
    print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def stream_form(fmt: str, steps: int, warmup: int) -> dict:
    """64QAM 48 GBd stream: 64 frames of 2^18 symbols/pol with carried state, from one seeded signal in
    the input format fmt ("c64": the plain FP32 chain's complex64 input; "f16": FP16; "i8": 8-bit ADC,
    4-sigma mid-tread). Each timed step is the whole 64-frame stream through a fresh handle."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.receiver import Receiver
    from synth import generate, workload
    from synth.channel import pack_bits, quantise_int8, to_fp16

    w = workload("dp-64qam-48gbd-stream")
    F, n = w["n_frames"], w["frame_sym"]
    fr = generate(w["link"], SEED)
    S = 2 * n
    if fmt == "i8":
        codes, delta = quantise_int8(fr.samples)
        data, rfmt, scale = codes, rx.RX_IN_I8, float(delta[0])
    elif fmt == "f16":
        data, rfmt, scale = to_fp16(fr.samples).view(np.int16), rx.RX_IN_F16, 1.0
    else:
        data, rfmt, scale = fr.samples.astype(np.complex64).view(np.float32).reshape(2, -1, 2), rx.RX_IN_C64, 1.0
    xs = [torch.from_numpy(np.ascontiguousarray(data[:, f * S:(f + 1) * S])).cuda() for f in range(F)]
    m = w["link"].bits_per_sym
    refs = [torch.from_numpy(pack_bits(fr.bits[:, f * n * m:(f + 1) * n * m]).astype(np.uint32).view(np.int32)).cuda()
            for f in range(F)]
    stream = torch.cuda.current_stream()
    times = []
    for rep in range(warmup + steps):
        rcv = Receiver(w["rx"], n, input_format=rfmt, input_scale=scale, streaming=True)
        out = torch.zeros(2 * rcv.words(n), dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for f in range(F):
            rcv.process(xs[f], n, refs[f], out)
        e1.record(stream)
        torch.cuda.synchronize()
        if rep >= warmup:
            times.append(e0.elapsed_time(e1))
        st = rcv.stats()
        rcv.close()
    t = sum(times) / len(times)
    bits = 2 * m * n * F
    in_bytes = int(sum(x.numel() * x.element_size() for x in xs))
    return {"metric": "processed line rate", "value": bits / (t * 1e-3) / 1e9, "unit": "Gb/s",
            "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": t, "higher_is_better": True,
            "dtype": f"{fmt} in, f32", "data": "synthetic",
            "config": {"workload": "dp-64qam-48gbd-stream", "frames": F, "symbols_per_frame": n, "input": fmt,
                       "input_bytes": in_bytes, "l2": "inputs of the stream (64 frames) exceed L2 only for c64; "
                                                      "every step is a fresh handle over the whole stream"},
            "ber": st["ber"], "evm": st["evm"], "q_db": st["q_db"], "error_word": st["error_word"]}


def other_forms(args) -> dict:
    """The chain's other forms on the same GPU, each beside its plain counterpart: the precision form
    (64QAM 48 GBd stream of 64 x 2^18 symbols with complex64, FP16 and int8 input), the batched form (16
    channels in one graph launch, and the same frames through single handles in turn) and the learned
    form (split-step 16QAM link: chain + post-equaliser + decisions against the chain alone). A few
    timed steps each, so that the whole run stays within minutes."""
    import argparse
    out = {}
    try:
        out["stream"] = {fmt: stream_form(fmt, 3, 3) for fmt in ("c64", "f16", "i8")}
        base = out["stream"]["c64"]
        for fmt in ("f16", "i8"):
            f = out["stream"][fmt]
            f["vs_c64"] = {"rate_ratio": f["value"] / base["value"], "ber_c64": base["ber"], "ber": f["ber"]}
    except Exception as e:  # report, do not hide
        out["stream"] = {"error": str(e)[:300]}
    try:
        out["batch"] = batch_form(5, 3)
    except Exception as e:
        out["batch"] = {"error": str(e)[:300]}
    try:
        out["inflight"] = inflight_form(4, 5, 3)
    except Exception as e:
        out["inflight"] = {"error": str(e)[:300]}
    try:
        la = argparse.Namespace(**vars(args))
        la.steps, la.warmup, la.n_sym = 5, 3, 0
        out["learned"] = learned_form(la)
    except Exception as e:
        out["learned"] = {"error": str(e)[:300]}
    return out


def stream_arm(args) -> None:
    print(json.dumps(stream_form(args.fmt, args.steps, args.warmup)))


def batch_form(steps: int, warmup: int) -> dict:
    """16 seeded channels (16..64 GBd, QPSK/16QAM/64QAM, 2^16..2^20 symbols) in one graph launch,
    beside the same frames through single handles of the same (tuned) configurations one after the
    other on the same stream (the plain chain, channel by channel)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.receiver import config_from
    from synth import generate
    from synth.workloads import batch_channels

    chans = batch_channels(42)
    xs, refs, outs, cfgs, n_sym, bits = [], [], [], [], [], 0
    for ch in chans:
        fr = generate(ch["link"], ch["seed"])
        N, m = ch["link"].n_sym, ch["link"].bits_per_sym
        xs.append(torch.from_numpy(np.ascontiguousarray(fr.samples.astype(np.complex64)).view(np.float32)).cuda())
        refs.append(torch.from_numpy(fr.ref_words.astype(np.uint32).view(np.int32)).cuda())
        outs.append(torch.zeros(2 * ((N * m + 31) // 32), dtype=torch.int32, device="cuda"))
        cfgs.append(config_from(ch["rx"], N))
        n_sym.append(N)
        bits += 2 * m * N
    t0 = time.perf_counter()
    b = rx.rx_batch_create(cfgs)
    tune_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    args_ = ([t.data_ptr() for t in xs], n_sym, [t.data_ptr() for t in refs], [t.data_ptr() for t in outs],
             stream.cuda_stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def timed(run):
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        ms = []
        for i in range(steps):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sum(ms) / len(ms)

    t = timed(lambda: rx.rx_batch_process(b, *args_))
    tuned = [(rx.rx_batch_config(b, i).fft_size, rx.rx_batch_config(b, i).lms_threads) for i in range(len(chans))]
    errs = sum(rx.rx_batch_stats(b, i)["bit_errors"] for i in range(len(chans)))
    counted = sum(rx.rx_batch_stats(b, i)["bits_counted"] for i in range(len(chans)))
    # the plain chain: one handle per channel with the tuned configuration, frames one after another
    hs = [rx.rx_create(rx.rx_batch_config(b, i)) for i in range(len(chans))]

    def singles():
        for i, h in enumerate(hs):
            rx.rx_process(h, xs[i].data_ptr(), n_sym[i], refs[i].data_ptr(), outs[i].data_ptr(), stream.cuda_stream)
    t1 = timed(singles)
    s_errs = sum(rx.rx_stats(h)["bit_errors"] for h in hs)
    s_counted = sum(rx.rx_stats(h)["bits_counted"] for h in hs)
    for h in hs:
        rx.rx_destroy(h)
    rx.rx_batch_destroy(b)
    return {"metric": "processed line rate", "value": bits / (t * 1e-3) / 1e9, "unit": "Gb/s",
            "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": t, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch16-seed42", "channels": len(chans), "symbols": sum(n_sym),
                       "tuned_fft_and_lms_threads": tuned, "tune_s": round(tune_s, 2),
                       "l2": "flushed between timed steps"},
            "graph_launches_per_step": 1, "ber": errs / max(counted, 1),
            "plain_sequential": {"value": bits / (t1 * 1e-3) / 1e9, "ms_per_step": t1,
                                 "ber": s_errs / max(s_counted, 1),
                                 "note": "same frames, one rx_process call per channel in turn"}}


def inflight_form(frames: int, steps: int, warmup: int) -> dict:
    """Independent DP-16QAM 32 GBd frames of 2^20 symbols/pol (the headline frame, one seed each), F of
    them in one graph launch (one handle and forked stream per frame, the configuration unchanged:
    FFT 4096, 128-thread LMS CTAs, no tuning): while one frame's serial acquisition holds two SMs,
    the others' throughput stages use the rest. Beside it, the same frames one rx_process call after
    another on one stream."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.receiver import config_from
    from synth import generate, workload

    w = workload("dp-16qam-32gbd")
    N, m = w["link"].n_sym, w["link"].bits_per_sym
    xs, refs, outs, bits = [], [], [], 0
    for f in range(frames):
        fr = generate(w["link"], SEED + f)
        xs.append(torch.from_numpy(np.ascontiguousarray(fr.samples.astype(np.complex64)).view(np.float32)).cuda())
        refs.append(torch.from_numpy(fr.ref_words.astype(np.uint32).view(np.int32)).cuda())
        outs.append(torch.zeros(2 * ((N * m + 31) // 32), dtype=torch.int32, device="cuda"))
        bits += 2 * m * N
    cfg = config_from(w["rx"], N)
    cfg.lms_threads = 128
    b = rx.rx_batch_create([cfg] * frames)
    stream = torch.cuda.current_stream()
    n_sym = [N] * frames
    args_ = ([t.data_ptr() for t in xs], n_sym, [t.data_ptr() for t in refs], [t.data_ptr() for t in outs],
             stream.cuda_stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")

    def timed(run):
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        ms = []
        for i in range(steps):
            flush.fill_(i & 0xFF)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        return sum(ms) / len(ms)

    t = timed(lambda: rx.rx_batch_process(b, *args_))
    errs = sum(rx.rx_batch_stats(b, i)["bit_errors"] for i in range(frames))
    counted = sum(rx.rx_batch_stats(b, i)["bits_counted"] for i in range(frames))
    h = rx.rx_create(cfg)

    def singles():
        for i in range(frames):
            rx.rx_process(h, xs[i].data_ptr(), N, refs[i].data_ptr(), outs[i].data_ptr(), stream.cuda_stream)
    t1 = timed(singles)
    s_errs, s_counted = rx.rx_stats(h)["bit_errors"], rx.rx_stats(h)["bits_counted"]
    rx.rx_destroy(h)
    rx.rx_batch_destroy(b)
    return {"metric": "processed line rate", "value": bits / (t * 1e-3) / 1e9, "unit": "Gb/s",
            "n_gpus": 1, "steps": steps, "warmup": warmup, "ms_per_step": t, "higher_is_better": True,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "dp-16qam-32gbd frames in flight", "frames": frames, "symbols_per_pol": N,
                       "l2": "flushed between timed steps"},
            "graph_launches_per_step": 1, "ber": errs / max(counted, 1),
            "plain_sequential": {"value": bits / (t1 * 1e-3) / 1e9, "ms_per_step": t1,
                                 "ber": s_errs / max(s_counted, 1),
                                 "note": "same frames, one rx_process call per frame in turn"}}


def batch_arm(args) -> None:
    print(json.dumps(batch_form(args.steps, args.warmup)))


# per position of the sequence: one position is one DP symbol (4 input channels I_x, Q_x, I_y, Q_y),
# so a frame of N symbols per polarisation is N positions
CNN_FWD_FLOP = 2 * 9 * (4 * 64 + 64 * 64 + 64 * 64 + 64 * 4)
CNN_TRAIN_FLOP = 2 * CNN_FWD_FLOP + 2 * 9 * (64 * 64 + 64 * 64 + 64 * 4)         # + weight and data gradients


def learned_form(args) -> dict:
    """Learned post-equaliser on split-step DP-16QAM 32 GBd, 10 x 80 km: the plain chain on training
    frames, training by the library's kernels, then timed steps of chain + post-equaliser + decisions
    on a frame of another seed; BER/EVM of both forms reported."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300 import rx
    from paper_2011_13695_gb300.learned import PostEqualiser, chain_pairs, decide_stats, he_init
    from paper_2011_13695_gb300.receiver import Receiver
    from synth.ssfm import generate_nonlinear
    from synth.workloads import workload

    kw = {"launch_dbm": args.launch_dbm}
    if args.n_sym:
        kw["n_sym"] = args.n_sym
    w = workload("dp-16qam-32gbd-ssfm", **kw)
    link, fibre = w["link"], w["fibre"]
    N, m = link.n_sym, link.bits_per_sym

    def on_device(fr):
        return (torch.from_numpy(np.ascontiguousarray(fr.samples.astype(np.complex64))).cuda(),
                torch.from_numpy(np.ascontiguousarray(fr.ref_words).view(np.int32)).cuda(),
                torch.from_numpy(np.ascontiguousarray(fr.symbols.astype(np.complex64))).cuda())

    t0 = time.perf_counter()
    rcv = Receiver(w["rx"], N)
    zs, ts, train_stats = [], [], []
    for seed in w["train_seeds"]:
        xs_, ref_, sym_ = on_device(generate_nonlinear(link, fibre, seed, device="cuda"))
        z, t, st = chain_pairs(rcv, xs_, N, ref_, sym_)
        zs.append(z)
        ts.append(t)
        train_stats.append(st)
    x, ref, sym = on_device(generate_nonlinear(link, fibre, w["test_seed"], device="cuda"))
    gen_s = time.perf_counter() - t0

    window, steps = args.window, args.train_steps
    pe = PostEqualiser(N, he_init(seed=0))
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    losses = pe.train(zs, ts, 1024, N - 1024, steps=steps, window=window, lr=args.lr, lr_final=args.lr / 10, seed=0)
    e1.record(stream)
    torch.cuda.synchronize()
    train_ms = e0.elapsed_time(e1)

    out = torch.empty((2, N), dtype=torch.complex64, device="cuda")
    for _ in range(args.warmup):
        rcv.process(x, N, ref, None)
        pe.forward(rcv.symbols(N), out)
    torch.cuda.synchronize()
    # plain chain and learned form on the test frame (statistics of one pass each)
    rcv.reset()
    z_test, _, plain = chain_pairs(rcv, x, N, ref, sym)
    pe.forward(z_test, out)
    learned = decide_stats(rcv, out, N, ref)

    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    zbuf = torch.empty((2, N), dtype=torch.complex64, device="cuda")
    zbytes = rx.rx_buffer_bytes(rcv.h, rx.RX_BUF_Z)
    step_ms, cnn_ms = [], []
    launches0 = rx.rx_launch_count(rcv.h)
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, b, c = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            a.record(stream)
            rcv.process(x, N, ref, None)
            rx.rx_get_buffer(rcv.h, rx.RX_BUF_Z, zbuf.data_ptr(), zbytes, stream.cuda_stream)
            b.record(stream)
            pe.forward(zbuf, out)
            c.record(stream)
            rcv.decide(out, N, ref, None)
            d = torch.cuda.Event(enable_timing=True)
            d.record(stream)
            torch.cuda.synchronize()
            step_ms.append(a.elapsed_time(d))
            cnn_ms.append(b.elapsed_time(c))
    launches = rx.rx_launch_count(rcv.h) - launches0 + args.steps * 4
    t = sum(step_ms) / len(step_ms)
    tc = sum(cnn_ms) / len(cnn_ms)
    pk = peaks()
    bf16_peak = pk.get("bf16_tflops", 1900.0)
    fwd_tflops = N * CNN_FWD_FLOP / (tc * 1e-3) / 1e12
    train_tflops = steps * window * CNN_TRAIN_FLOP / (train_ms * 1e-3) / 1e12
    bits = 2 * m * N
    pe.close()
    line = {
        "metric": "processed line rate", "value": bits / (t * 1e-3) / 1e9, "unit": "Gb/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True,
        "dtype": "f32 chain, bf16 x bf16 -> f32 network", "data": "synthetic (split-step Manakov, seeded)",
        "config": {"workload": "dp-16qam-32gbd-ssfm", "symbols_per_pol": N, "launch_dbm": args.launch_dbm,
                   "spans": fibre.spans, "span_km": fibre.span_km, "train_frames": len(zs),
                   "train_steps": steps, "window": window, "lr": args.lr, "l2": "flushed between timed steps"},
        "plain": {"ber": plain["ber"], "evm": plain["evm"], "bit_errors": plain["bit_errors"],
                  "bits_counted": plain["bits_counted"]},
        "learned": {"ber": learned["ber"], "evm": learned["evm"], "bit_errors": learned["bit_errors"],
                    "bits_counted": learned["bits_counted"]},
        "evm_gain_db": 20 * np.log10(plain["evm"] / learned["evm"]),
        "train": {"ms": train_ms, "tflops": train_tflops, "loss_first": float(losses[:20].mean()),
                  "loss_last": float(losses[-20:].mean()), "train_plain_ber": [s_["ber"] for s_ in train_stats]},
        "roofline": {"kernel": "cnn forward (k_conv_tc: 4 tcgen05 launches, one per layer)",
                     "bound": "tensor", "achieved": fwd_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": fwd_tflops / bf16_peak, "traffic": None,
                     "peak_source": "fallback" if pk.get("fallback") else "measured cuBLAS bf16 burst (MEASURED_PEAKS.json)",
                     "note": "whole forward's algorithmic flops over its time (4 conv launches)"},
        "cnn_ms": tc, "gpu_launches": int(launches), "generate_s": round(gen_s, 1), "clocks": clk.summary(),
    }
    rcv.close()
    return line


def learned_arm(args) -> None:
    print(json.dumps(learned_form(args)))


def cnn_arm(args) -> None:
    """The post-equaliser's inference forward alone (4 tcgen05 launches) on He-initialised weights and
    16QAM-like symbols of 2^20 symbols/pol (or --n-sym): a kernel measurement, not a bench line of the
    chain. HBM algorithmic bytes per DP symbol: 16 in + 128 out (layer 0), 2 x (128 + 128) (hidden
    layers), 128 + 16 + 16 (output layer)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300.learned import PostEqualiser, he_init

    N = args.n_sym or (1 << 20)
    rng = np.random.default_rng(7)
    lv = np.array([-3.0, -1.0, 1.0, 3.0]) / np.sqrt(10.0)
    zc = lv[rng.integers(0, 4, (2, N))] + 1j * lv[rng.integers(0, 4, (2, N))]
    zc = zc + 0.05 * (rng.standard_normal((2, N)) + 1j * rng.standard_normal((2, N)))
    z = torch.from_numpy(zc.astype(np.complex64)).cuda()
    out = torch.empty_like(z)
    pe = PostEqualiser(N, he_init(seed=0))
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        pe.forward(z, out)
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ms = []
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pe.forward(z, out)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    err = pe.error_word()
    pe.close()
    t = sum(ms) / len(ms)
    pk = peaks()
    bf16_peak = pk.get("bf16_tflops", 1900.0)
    tflops = N * CNN_FWD_FLOP / (t * 1e-3) / 1e12
    hbm_bytes = N * ((16 + 128) + 2 * (128 + 128) + (128 + 16 + 16))
    print(json.dumps({
        "metric": "post-equaliser forward", "value": 2 * N / (t * 1e-3) / 1e9, "unit": "GSym/s (DP symbols x 2)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True,
        "dtype": "bf16 x bf16 -> f32", "data": "synthetic",
        "config": {"workload": f"cnn-forward-{N}", "symbols_per_pol": N, "l2": "flushed between timed steps"},
        "roofline": {"kernel": "k_conv_tc x 4 (whole forward)", "bound": "tensor", "achieved": tflops,
                     "peak": bf16_peak, "unit": "TFLOP/s", "frac": tflops / bf16_peak, "traffic": None,
                     "hbm_gbs": hbm_bytes / (t * 1e-3) / 1e9, "hbm_frac": hbm_bytes / (t * 1e-3) / 1e9 / pk.get("hbm_gbs", 6800.0)},
        "error_word": err, "gpu_launches": 4 * args.steps, "clocks": clk.summary()}))


def wl_arm(args) -> None:
    """The widely-linear segmented DD-LMS alone (rx_dd_lms_wl: one launch, one CTA per segment and
    output row) on a 16QAM 32 GBd frame of 2^20 symbols/pol (or --n-sym) with a transmitter IQ
    imbalance (amplitude 0.10, phase skew 0.08 rad): 21 taps, blocks of 128 symbols, segments of
    16 blocks with 4 warm-up blocks. A kernel measurement, not a bench line of the chain.
    Algorithmic FP32 work per DP symbol: 2 rows x (4T complex MACs for the output + 4T for the
    gradient) x 8 flops = 128 T, times 1 + warm-up/segment blocks."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300.receiver import dd_lms_wl
    from synth import LinkParams, generate

    N = args.n_sym or (1 << 20)
    T, Lb, seg, wu, m, mu = args.wl_taps, 128, 16, 4, 4, 1e-3
    th = args.wl_threads
    p = LinkParams(bits_per_sym=m, symbol_rate=32e9, n_sym=N, length=0.0, linewidth=0.0, freq_offset=0.0,
                   snr_db=20.0, jones=False, tx_rrc=False, iq_imbalance=(0.10, 0.08))
    fr = generate(p, SEED)
    xs = fr.samples / np.sqrt(np.mean(np.abs(fr.samples[:, ::2]) ** 2, axis=1, keepdims=True))
    x = torch.from_numpy(np.ascontiguousarray(xs.astype(np.complex64))).cuda()
    h0 = torch.zeros((2, 4, T), dtype=torch.complex64, device="cuda")
    h0[0, 0, T // 2] = 1.0
    h0[1, 1, T // 2] = 1.0
    y = torch.empty((2, N), dtype=torch.complex64, device="cuda")
    ho = torch.empty_like(h0)
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        dd_lms_wl(x, h0, N, Lb, seg, wu, m, mu, mu, y=y, taps_out=ho, threads=th)
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ms = []
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            dd_lms_wl(x, h0, N, Lb, seg, wu, m, mu, mu, y=y, taps_out=ho, threads=th)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    t = sum(ms) / len(ms)
    yc = y[:, 8192:].cpu().numpy()
    psi = np.angle(-np.sum(yc ** 4, axis=-1, keepdims=True)) / 4
    u = yc * np.exp(-1j * psi)
    L = 1 << (m // 2)
    a_l = 1.0 / np.sqrt(2.0 * (L * L - 1) / 3.0)
    dec = lambda v: (np.clip(np.round((v / a_l + (L - 1)) / 2), 0, L - 1) * 2 - (L - 1)) * a_l
    evm_db = 10 * np.log10(np.mean(np.abs(u - dec(u.real) - 1j * dec(u.imag)) ** 2))
    pk = dict(peaks(), **measure_fp32_peak(rx, stream.cuda_stream))
    flop_peak, _, _, peak_note = fp32_peak(pk)
    peak = flop_peak / 1e12
    flops = N * (1 + wu / seg) * 128 * T
    nseg = (N + seg * Lb - 1) // (seg * Lb)
    achieved = flops / (t * 1e-3) / 1e12
    print(json.dumps({
        "metric": "widely-linear DD-LMS line rate", "value": 2 * m * N / (t * 1e-3) / 1e9, "unit": "Gb/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True,
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"wl-dd-lms-16qam-{N}", "symbols_per_pol": N, "taps": T, "block": Lb, "threads": th,
                   "seg_blocks": seg, "warmup_blocks": wu, "l2": "flushed between timed steps (512 MiB write)"},
        "roofline": {"kernel": wl_kernel_name(T, Lb, th), "bound": "alu", "achieved": achieved, "peak": peak,
                     "unit": "TFLOP/s", "frac": achieved / peak, "traffic": _traffic("wl") if (N, T, th) == (1 << 20, 21, 0) else None,
                     "algorithmic_flops": flops, "ctas": 2 * nseg, "peak_note": "FP32 FMA pipes, " + peak_note},
        "evm_db_after_8192_symbols": float(evm_db), "gpu_launches": args.steps, "clocks": clk.summary(),
        "cpu_baseline": None if args.no_cpu_baseline else wl_cpu_baseline(T)}))


def wl_kernel_name(T: int, Lb: int, threads: int) -> str:
    """The kernel rx_dd_lms_wl launches for this shape (compiled shapes: T 15/21/31, blocks of 128)."""
    if T in (15, 21, 31) and Lb == 128 and threads in (0, 128, 256):
        return f"k_lms_fast<{threads or 128}, {T}, {Lb}, widely linear>"
    return f"k_lms<{threads or 256}, widely linear> (generic)"


WL_CPU_SAMPLE = 1 << 20


def wl_oracle_worker(n_sym: int, reps: int, T: int = 21) -> dict:
    """The oracle's widely-linear segmented DD-LMS on the first n_sym symbols of the wl frame."""
    import numpy as np

    from oracle import mimo
    from synth import LinkParams, generate
    p = LinkParams(bits_per_sym=4, symbol_rate=32e9, n_sym=n_sym, length=0.0, linewidth=0.0, freq_offset=0.0,
                   snr_db=20.0, jones=False, tx_rrc=False, iq_imbalance=(0.10, 0.08))
    fr = generate(p, SEED)
    x = fr.samples / np.sqrt(np.mean(np.abs(fr.samples[:, ::2]) ** 2, axis=1, keepdims=True))
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        mimo.dd_lms_wl(x, mimo.wl_identity_taps(T), n_sym, 128, 16, 4, 4, 1e-3, 1e-3)
        times.append(time.perf_counter() - t0)
    return dict(times=times, bits=2 * 4 * n_sym)


def wl_cpu_baseline(T: int = 21, reps: int = 3) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.wl_oracle_worker(%d, %d, %d)))" % (ROOT, WL_CPU_SAMPLE, reps, T))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode:
        raise RuntimeError(r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    t = statistics.median(res["times"])
    return {"value": res["bits"] / t / 1e9, "unit": "Gb/s", "cores": 1, "kind": "oracle",
            "sample": f"the wl frame, {WL_CPU_SAMPLE} symbols/pol, {T} taps, widely-linear segmented "
                      f"DD-LMS in FP64 NumPy, single thread, median of {reps}"}


def kk_arm(args) -> None:
    """The Kramers-Kronig front end alone (rx_kk_process: k_kk_phase + k_kk_mf, N = 1024) on the paper's
    buffer of 2^22 12-bit samples (or --n-sym symbols x 4): 16QAM at 1 GBd, 4 samples/symbol, 1 %
    roll-off, tone 0.547 GHz below the signal, 11 dB CSPR, 20 dB SNR. A kernel measurement, not a bench
    line of the chain. Algorithmic HBM bytes per input sample: 2 (code) + 8 (field out) in the first
    pass, 8 (field in) + 4 (half an output sample) in the second; FP32 FFT work 5 N log2 N per
    N-point transform: 2 transforms of N per N/2 samples in the first pass, one of N and one of N/2 in
    the second."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300.receiver import KKFrontEnd
    from synth.kk import KKLink, generate_kk

    n_sym = args.n_sym or (1 << 20)
    N = 1024
    p = KKLink(bits_per_sym=4, n_sym=n_sym, cspr_db=11.0, snr_db=20.0)
    fr = generate_kk(p, SEED)
    S = 4 * n_sym
    fe = KKFrontEnd(N, p.tone_offset / p.fs, p.rolloff, fr.scale, fr.dc, 1e-6)
    codes = torch.from_numpy(fr.codes.view(np.int16)).cuda()
    field = torch.empty(S, dtype=torch.complex64, device="cuda")
    out = torch.empty(S // 2, dtype=torch.complex64, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        fe.process(codes, field, out)
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ms = []
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fe.process(codes, field, out)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    fe.close()
    t = sum(ms) / len(ms)
    ys = out[::2].cpu().numpy()[256:-256]
    s = fr.symbols[256:-256]
    L = 4
    a_l = 1.0 / np.sqrt(2.0 * (L * L - 1) / 3.0)
    dec = lambda v: (np.clip(np.round((v / a_l + (L - 1)) / 2), 0, L - 1) * 2 - (L - 1)) * a_l
    evm_db = 10 * np.log10(np.mean(np.abs(ys - s) ** 2))
    ser = float(np.mean((dec(ys.real) != dec(s.real)) | (dec(ys.imag) != dec(s.imag))))
    pk = peaks()
    hbm_bytes = S * (2 + 8 + 8 + 4)
    fft_flops = (S / (N / 2)) * (2 * 5 * N * 10 + 5 * N * 10 + 5 * (N // 2) * 9)
    flop_peak = fp32_peak(dict(pk, **measure_fp32_peak(rx, torch.cuda.current_stream().cuda_stream)))[0]
    hbm_gbs = hbm_bytes / (t * 1e-3) / 1e9
    tflops = fft_flops / (t * 1e-3) / 1e12
    print(json.dumps({
        "metric": "KK front-end sample rate", "value": S / (t * 1e-3) / 1e9, "unit": "GSa/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic", "line_rate_gbps": 4 * n_sym / (t * 1e-3) / 1e9,
        "paper_realtime_gsa_s": 4.0,
        "config": {"workload": f"kk-16qam-1gbd-{S}", "samples": S, "fft": N, "sps_in": 4, "sps_out": 2,
                   "cspr_db": 11.0, "l2": "flushed between timed steps (512 MiB write)"},
        "roofline": {"kernel": "k_kk_phase + k_kk_mf (whole front end)", "bound": "hbm", "achieved": hbm_gbs,
                     "peak": pk.get("hbm_gbs", 6800.0), "unit": "GB/s", "frac": hbm_gbs / pk.get("hbm_gbs", 6800.0),
                     "traffic": None, "algorithmic_bytes": hbm_bytes, "fft_tflops": tflops,
                     "fft_frac_of_fp32_peak": tflops / (flop_peak / 1e12)},
        "evm_db": float(evm_db), "symbol_error_rate": ser, "gpu_launches": 2 * args.steps,
        "clocks": clk.summary(), "cpu_baseline": None if args.no_cpu_baseline else kk_cpu_baseline(n_sym)}))


def ingest_arm(args) -> None:
    """Real-time ingest emulation (rx_ingest_run): the digitiser delivers 2^22-sample 12-bit buffers at
    4 GSa/s (one every 1.049 ms); each accepted buffer is copied in, joined to its predecessor, run
    through the KK front end and its 2^21 output samples copied back to host memory. --steps buffers
    (default 20 -> 500 buffers, 0.52 s) per run, for 1, 2 and 5 streams; a buffer that finds every
    stream busy is dropped. The paper's condition: mean buffer time below 1.049 ms x streams."""
    import numpy as np

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300.receiver import KKFrontEnd
    from synth.kk import KKLink, generate_kk

    S = 1 << 22
    nbuf = max(1, args.steps) * 25
    p = KKLink(bits_per_sym=4, n_sym=S // 4, cspr_db=11.0, snr_db=20.0)
    fr = generate_kk(p, SEED)
    fe = KKFrontEnd(1024, p.tone_offset / p.fs, p.rolloff, fr.scale, fr.dc, 1e-6)
    fe.ingest(fr.codes, S, 4e9, 2, max(3, args.warmup))            # warm-up run
    runs = {}
    with ClockSampler(0) as clk:
        for ns in (1, 2, 5):
            st, _ = fe.ingest(fr.codes, S, 4e9, ns, nbuf)
            runs[str(ns)] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in st.items()}
    fe.close()
    one = runs["1"]
    print(json.dumps({
        "metric": "ingest buffers dropped at 4 GSa/s (1 stream)", "value": one["dropped"], "unit": "buffers",
        "n_gpus": 1, "steps": nbuf, "warmup": max(3, args.warmup), "higher_is_better": False,
        "mean_latency_ms_1_stream": one["mean_latency_ms"], "buffer_period_ms": one["buffer_period_ms"],
        "dtype": "f32", "data": "synthetic",
        "config": {"workload": "ingest-kk-16qam-4gsa", "buffer_samples": S, "sample_rate_gsa_s": 4.0,
                   "buffers_per_run": nbuf, "streams": [1, 2, 5]},
        "runs": runs, "gpu_launches": 2 * sum(r["processed"] for r in runs.values()), "clocks": clk.summary()}))


def pam_arm(args) -> None:
    """The IM/DD PAM-4 chain with FD clock recovery (rx_pam_process, 8 launches: clock products,
    105-block averages and phases, winding scan and offsets, correction + variable-rate extraction,
    mean, deviation and its final sum, decision)
    on the paper's buffer of 2^22 12-bit samples at 2 samples/symbol (2 GBd PAM-4, 50 % roll-off, a
    25 ppm receiver clock offset, 20 dB SNR). Line rate: output symbols x 2 bits per buffer time.
    Algorithmic HBM bytes per input sample: 2 (codes, read by two passes: 4) + 4 (y written, read
    twice, 1 output per 2 samples: 6) + 0.5 (levels)."""
    import numpy as np
    import torch

    import __graft_entry__
    __graft_entry__.build()
    from paper_2011_13695_gb300.receiver import PAMReceiver
    from synth.pam import PAMLink, generate_pam

    S = args.n_sym * 2 if args.n_sym else (1 << 22)
    p = PAMLink(levels=4, n_samp=S, clock_ppm=25.0, timing=0.2, snr_db=20.0)
    fr = generate_pam(p, SEED)
    pr = PAMReceiver(1024, 4, p.rolloff, fr.scale, fr.dc, S)
    codes = torch.from_numpy(fr.codes.view(np.int16)).cuda()
    cap = pr.capacity(S)
    y = torch.empty(cap, dtype=torch.float32, device="cuda")
    lev = torch.empty(cap, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    for _ in range(args.warmup):
        pr.process(codes, y, lev)
    torch.cuda.synchronize()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    ms = []
    with ClockSampler(0) as clk:
        for i in range(args.steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            _, _, n_out = pr.process(codes, y, lev)
            b.record(stream)
            torch.cuda.synchronize()
            ms.append(a.elapsed_time(b))
    n = int(n_out.item())
    got = lev[:n].cpu().numpy().astype(np.int64)
    pr.close()
    tx = (fr.symbols[fr.first:fr.first + n] + 3) // 2
    E = 60 * 256
    ser = float(np.mean(got[E:-E] != tx[E:-E]))
    t = sum(ms) / len(ms)
    pk = peaks()
    hbm_bytes = S * (4 + 6 + 0.5)
    print(json.dumps({
        "metric": "PAM-4 chain line rate", "value": 2 * n / (t * 1e-3) / 1e9, "unit": "Gb/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "dtype": "f32",
        "data": "synthetic", "sample_rate_gsa_s": S / (t * 1e-3) / 1e9, "paper_realtime_gsa_s": 4.0,
        "config": {"workload": f"pam4-2gbd-{S}", "samples": S, "fft": 1024, "clock_ppm": 25.0,
                   "l2": "flushed between timed steps (512 MiB write)"},
        "roofline": {"kernel": "rx_pam_process (8 launches)", "bound": "hbm",
                     "achieved": hbm_bytes / (t * 1e-3) / 1e9, "peak": pk.get("hbm_gbs", 6800.0), "unit": "GB/s",
                     "frac": hbm_bytes / (t * 1e-3) / 1e9 / pk.get("hbm_gbs", 6800.0), "traffic": None},
        "symbol_error_rate_interior": ser, "outputs": n, "gpu_launches": 8 * args.steps,
        "clocks": clk.summary(), "cpu_baseline": None if args.no_cpu_baseline else pam_cpu_baseline(S)}))


def pam_oracle_worker(n_samp: int, reps: int) -> dict:
    """The oracle's PAM chain on the pam workload's buffer."""
    from oracle import pam
    from synth.pam import PAMLink, generate_pam
    p = PAMLink(levels=4, n_samp=n_samp, clock_ppm=25.0, timing=0.2, snr_db=20.0)
    fr = generate_pam(p, SEED)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        pam.pam_receive(fr.codes, fr.scale, fr.dc, 4, p.rolloff, 1024)
        times.append(time.perf_counter() - t0)
    return dict(times=times, samples=n_samp)


def pam_cpu_baseline(n_samp: int, reps: int = 3) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.pam_oracle_worker(%d, %d)))" % (ROOT, n_samp, reps))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode:
        raise RuntimeError(r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    t = statistics.median(res["times"])
    return {"value": res["samples"] / t / 1e9, "unit": "GSa/s", "cores": 1, "kind": "oracle",
            "sample": f"the pam buffer, {res['samples']} samples, Steps 1-9 in FP64 NumPy, single thread, "
                      f"median of {reps}"}


def kk_oracle_worker(n_sym: int, reps: int) -> dict:
    """The oracle's KK front end on the kk workload's buffer."""
    from oracle import kk
    from synth.kk import KKLink, generate_kk
    p = KKLink(bits_per_sym=4, n_sym=n_sym, cspr_db=11.0, snr_db=20.0)
    fr = generate_kk(p, SEED)
    times = []
    for _ in range(reps):
        t0 = time.perf_counter()
        kk.kk_receive(fr.codes, fr.scale, fr.dc, 1e-6, p.tone_offset / p.fs, p.rolloff, 1024)
        times.append(time.perf_counter() - t0)
    return dict(times=times, samples=4 * n_sym)


def kk_cpu_baseline(n_sym: int, reps: int = 3) -> dict:
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               NUMEXPR_NUM_THREADS="1", CUDA_VISIBLE_DEVICES="")
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.kk_oracle_worker(%d, %d)))" % (ROOT, n_sym, reps))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=1800)
    if r.returncode:
        raise RuntimeError(r.stderr[-2000:])
    res = json.loads(r.stdout.strip().splitlines()[-1])
    t = statistics.median(res["times"])
    return {"value": res["samples"] / t / 1e9, "unit": "GSa/s", "cores": 1, "kind": "oracle",
            "sample": f"the kk buffer, {res['samples']} samples, Steps 1-8 in FP64 NumPy, single thread, "
                      f"median of {reps}"}


def main():
    args = parse()
    if args.impl == "ours" and args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # started without torchrun: one replica rank per GPU, as torchrun would start them
        spawn_ranks(args.gpus, dispatch, args)
        return
    dispatch(args)


def dispatch(args) -> None:
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "stream":
        stream_arm(args)
    elif args.workload == "forms":
        print(json.dumps(other_forms(args)))
    elif args.workload == "batch":
        batch_arm(args)
    elif args.workload == "inflight":
        print(json.dumps(inflight_form(args.frames, args.steps, args.warmup)))
    elif args.workload == "learned":
        learned_arm(args)
    elif args.workload == "cnn":
        cnn_arm(args)
    elif args.workload == "wl":
        wl_arm(args)
    elif args.workload == "kk":
        kk_arm(args)
    elif args.workload == "ingest":
        ingest_arm(args)
    elif args.workload == "pam":
        pam_arm(args)
    else:
        our_arm(args)


if __name__ == "__main__":
    main()
