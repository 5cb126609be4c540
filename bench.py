#!/usr/bin/env python3
"""Throughput of the bit-packed ASEP / KPZ engine on one GB300 (or N replicas).

Workload (the growth-regime batch of the paper's KPZ study, sec. 2.2, at the
size the headline is quoted on): one ring of L = 2^17 sites per sample (4096
uint32 words, resident in shared memory), ASEP with p = 0.75, q = 0.25, flat
1010... start, 2^14 Monte Carlo sweeps with W^2 recorded at the log-spaced
times of Eq. (sampling), 256 independent samples in one launch, two-phase
Poisson-domain schedule with D = 256.

One step = re-draw the initial state + 2^14 sweeps of all samples (with the
fused height / W^2 recording).  The metric is site-update attempts per second
(L attempts per sample per sweep).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

--impl reference times the CPU oracle (plain C replay of the same schedule)
on the host cores on a bounded sample of the same workload.
Under torchrun (N > 1) every rank runs an independent replica on its own
sample range (no data-path collective); the timed region is bracketed by
barriers and the max over ranks is taken.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_SITES = 1 << 17
DOMAIN = 256
SAMPLES = 256
N_MCS = 1 << 14
P_RATE, Q_RATE = 0.75, 0.25
SEED = 1
REF_STEP_S = 5.0  # CPU seconds per timed step of the reference arm
# Algorithmic int32 lane operations per attempt of the domain kernel: a
# quarter of one Philox4x32-10 call (10 rounds x [2 wide multiplies + 2
# three-input XORs] = 40) plus the update (slot and row decode 2, address 1,
# load 1, straddle test 1, pattern extract 2, threshold select 2, masked
# compare 2, flip mask and xor 2, store 1) = 10 + 14.
OPS_PER_ATTEMPT = 24
# The same count for the two-sub-lattice SCA kernel, per attempt = per bond of
# a 32-bond group and phase: K random planes, each a quarter of one Philox
# call (10 ops) and three comparator ops (threshold mask, less-than, equal),
# plus 12 ops of pattern test and flips per group: (13 K + 12) / 32, with
# K = 2 planes for p = 0.75, q = 0.25.
SCA_PLANES = 2
SCA_OPS_PER_ATTEMPT = (13 * SCA_PLANES + 12) / 32
SMS, LANES_PER_SM = 152, 128  # GB300: 152 SMs x 4 schedulers x 32 lanes issue per clock

WORKLOAD_NAME = ("growth regime, batched: L=2^17 ring (4096 u32 words, shared-memory resident), ASEP p=0.75 q=0.25, "
                 "flat start, 2^14 MCS, W^2 at log-spaced times, 256 samples in one launch")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), f"asep_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self) -> dict | None:
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
        sms, maxes, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sms.append(float(parts[1]))
                    maxes.append(float(parts[2]))
                except ValueError:
                    continue
                for n, v in zip(names, parts[5:9]):
                    if v.lower().startswith("active"):
                        reasons.add(n)
        if not sms:
            return None
        return {"sm_mhz": statistics.median(sms), "sm_max_mhz": max(maxes), "reasons": sorted(reasons),
                "samples": len(sms)}


KERNEL_SOURCES = {
    "domain": ("asep_kernels.cu", "asep_resident.cuh", "asep_domain.cuh", "asep_device.cuh", "asep_internal.h"),
    "domain_bal": ("asep_balance.cu", "asep_resident.cuh", "asep_domain.cuh", "asep_device.cuh", "asep_internal.h"),
    "sca": ("asep_sca.cu", "asep_device.cuh", "asep_internal.h"),
    "sca_stream": ("asep_sca.cu", "asep_device.cuh", "asep_internal.h"),
    "stream": ("asep_stream.cu", "asep_domain.cuh", "asep_device.cuh", "asep_internal.h"),
    "serial": ("asep_serial.cu", "asep_device.cuh", "asep_internal.h"),
}
TRAFFIC_FILES = {
    "domain": "k_domain_growth_regime_traffic.txt",
    "domain_bal": "k_domain_bal_growth_regime_traffic.txt",
    "sca": "k_sca_growth_regime_traffic.txt",
    "sca_stream": "k_sca_stream_large_rings_traffic.txt",
    "stream": "k_stream_large_rings_traffic.txt",
    "serial": "k_serial_plain_tasep_traffic.txt",
}


def kernel_source_digest(kernel: str = "domain") -> str:
    """sha256 prefix over the source files a kernel is compiled from."""
    import hashlib

    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1012_0385_gb300", "csrc")
    for name in KERNEL_SOURCES[kernel]:
        h.update(open(os.path.join(csrc, name), "rb").read())
    return h.hexdigest()[:16]


def _traffic_from_profile(kernel: str = "domain"):
    """DRAM bytes per launch of the kernel from the committed ncu summary, if
    it was taken on the current kernel sources."""
    prof = os.path.join(ROOT, "profiles", TRAFFIC_FILES[kernel])
    try:
        digest = kernel_source_digest(kernel)
        kv = dict(line.strip().split("=", 1) for line in open(prof) if "=" in line)
        if kv.get("kernel_source_sha256_16") == digest:
            return float(kv["dram_bytes_per_launch"])
    except Exception:
        pass
    return None


WINDOW_KERNELS = ["serial", "domain", "domain", "domain", "sca", "sca", "stream", "sca_stream"]
COUNTS_FILE = "window_kernels_counts.txt"


def _inst_counts() -> dict:
    """Thread instructions per attempt of the benchmarked kernels, from the
    committed ncu summary: name ("window<i>", "headline_domain",
    "headline_domain_bal") -> value, for kernels whose sources are unchanged
    since the counts were taken."""
    out = {}
    try:
        for line in open(os.path.join(ROOT, "profiles", COUNTS_FILE)):
            if line.startswith("#") or "=" not in line:
                continue
            kv = dict(x.split("=", 1) for x in line.split())
            if kv.get("kernel_source_sha256_16") == kernel_source_digest(kv["family"]):
                out[kv["name"]] = float(kv["inst_per_attempt"])
    except Exception:
        pass
    return out


def _smem_counts() -> dict:
    """Shared-memory wavefronts per attempt of the benchmarked kernels (ncu
    l1tex__data_pipe_lsu_wavefronts_mem_shared.sum / attempts), same source
    and digest rule as _inst_counts."""
    out = {}
    try:
        for line in open(os.path.join(ROOT, "profiles", COUNTS_FILE)):
            if line.startswith("#") or "=" not in line:
                continue
            kv = dict(x.split("=", 1) for x in line.split())
            if kv.get("kernel_source_sha256_16") == kernel_source_digest(kv["family"]) and \
                    "smem_wavefronts_per_attempt" in kv:
                out[kv["name"]] = float(kv["smem_wavefronts_per_attempt"])
    except Exception:
        pass
    return out


def _smem_fraction(rate: float, name: str, max_mhz: float):
    """Shared-memory bandwidth the kernel uses: measured wavefronts per
    attempt x attempts/s, over one wavefront (128 bytes) per SM and clock;
    None without a count for the current sources."""
    wpa = _smem_counts().get(name)
    if wpa is None:
        return None
    peak = SMS * max_mhz * 1e6
    return {"wavefronts_per_attempt": wpa, "achieved_wavefronts_per_s": rate * wpa, "peak_wavefronts_per_s": peak,
            "frac": rate * wpa / peak, "peak_basis": "152 SMs x 1 wavefront (128 B) per clock x max SM clock",
            "source": "profiles/" + COUNTS_FILE}


def _window_counts() -> dict:
    """Window index -> thread instructions per attempt (see _inst_counts)."""
    return {int(k[len("window"):]): v for k, v in _inst_counts().items() if k.startswith("window")}


def cpu_oracle_sample(target_s: float, n_mcs_cap: int = N_MCS):
    """Time the CPU oracle (whole path: init, sweeps, heights at the log
    times) on `cores` samples of the workload, sized to about target_s."""
    import oracle

    cores = os.cpu_count() or 1
    th = oracle.threshold
    P = oracle.Params(L=L_SITES, D=DOMAIN, samples_per_real=SAMPLES, p_thr=th(P_RATE), q_thr=th(Q_RATE), seed=SEED)
    k = min(cores, SAMPLES)
    oracle.build()
    # calibrate on the difference of an 8- and a 40-sweep run (start-up costs cancel)
    t0 = time.perf_counter()
    oracle.run(P, 8, [0], threads=cores, samples=range(k))
    t1 = time.perf_counter()
    oracle.run(P, 40, [0], threads=cores, samples=range(k))
    t2 = time.perf_counter()
    rate = k * L_SITES * 32 / max(1e-6, (t2 - t1) - (t1 - t0))
    n = int(max(8, min(n_mcs_cap, target_s * rate / (k * L_SITES))))
    from paper_1012_0385_gb300.sampling import log_times

    t0 = time.perf_counter()
    oracle.run(P, n, [t for t in log_times(N_MCS) if t <= n], threads=cores, samples=range(k))
    dt = time.perf_counter() - t0
    return {"value": k * L_SITES * n / dt, "unit": "attempts/s", "cores": cores, "kind": "oracle",
            "value_per_core": k * L_SITES * n / dt / cores, "seconds": dt, "attempts": k * L_SITES * n,
            "sample": f"{k} of 256 samples x {n} of 2^14 sweeps (init + sweeps + W^2 at the log times), "
                      f"{dt:.1f} s on {cores} host threads"}


def cpu_baselines_by_config(seconds_each: float = 2.5):
    """The oracle's two programs on the host cores for configurations 0-3:
    the schedule replay (the GPU path's own schedule, bit-identical to it:
    serial RSU for configuration 0, the domain schedule for 1-3) and the
    independent serial RSU reference (its own generator).  Configuration 0
    runs in full (8 samples x 10^4 sweeps); the others on a bounded sample:
    the first `cores` samples over as many sweeps of their window as fit
    about `seconds_each` seconds, from the flat or random start.  One thread
    per sample."""
    import oracle

    cores = os.cpu_count() or 1
    th = oracle.threshold
    oracle.build()
    cfgs = [
        ("0: plain TASEP, L=4096, 8 samples, 10^4 MCS", 10_000, 8,
         dict(L=4096, schedule=oracle.SCHED_SERIAL, samples_per_real=8, p_thr=oracle.ALWAYS, q_thr=0, seed=1)),
        ("1: growth regime, L=2^17, ASEP p=0.75 q=0.25 (256 samples, 2^14 MCS)", 1 << 14, 256,
         dict(L=1 << 17, D=256, samples_per_real=min(cores, 256), p_thr=th(0.75), q_thr=th(0.25), seed=1)),
        ("2: bimodal disorder, L=2^16, Q=0.1, p_slow=0.3 (64 x 4 samples, 10^4-MCS window)", 10_000, 256,
         dict(L=1 << 16, D=256, n_realizations=max(1, min(cores, 256) // 4), samples_per_real=4,
              p_thr=oracle.ALWAYS, q_thr=0, dis_kind=oracle.DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3),
              dis_seed=2, seed=1)),
        ("3: two lanes, 2 x L=2^16, turning 0.05, omega 0.1, D=128 (128 samples, 10^4-MCS window)", 10_000, 128,
         dict(model=oracle.MODEL_TWO_LANE, L=1 << 16, D=128, samples_per_real=min(cores, 128), p_thr=oracle.ALWAYS,
              q_thr=oracle.ALWAYS, dis_kind=oracle.DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1), dis_seed=3,
              init_kind=oracle.INIT_BERNOULLI_HALF, init_seed=4, seed=1)),
    ]
    rows = []
    for name, window, s_full, kw in cfgs:
        P = oracle.Params(**kw)
        mask = oracle.disorder(P)
        for program in ("replay", "serial reference"):
            def run(n, st):
                if program == "replay":
                    oracle.replay(P, st, 0, n, mask=mask, threads=cores)
                else:
                    oracle.serial_reference(P, st, n, rng_seeds=[17 + s for s in range(P.S)], mask=mask,
                                            threads=cores)

            st = oracle.init_state(P)
            t0 = time.perf_counter()
            run(1, st)
            per_sweep = max(1e-6, time.perf_counter() - t0)
            n = window if P.S == s_full else int(max(2, min(window, seconds_each / per_sweep)))
            st = oracle.init_state(P)
            t0 = time.perf_counter()
            run(n, st)
            dt = time.perf_counter() - t0
            attempts = P.S * P.L * P.planes * n
            rows.append({"config": name, "program": program, "samples": P.S, "sweeps": n,
                         "attempts_per_s": attempts / dt, "attempts_per_s_per_core": attempts / dt / min(cores, P.S),
                         "threads": min(cores, P.S), "seconds": dt,
                         "sample": "full run" if (P.S == s_full and n == window) else
                         f"{P.S} of {s_full} samples x {n} of {window} sweeps"})
    return rows


def _issue_fraction(rate: float, name: str, peak_ops: float):
    """Issue slots the kernel fills: measured thread instructions per attempt
    (ncu) x attempts/s, over 152 SMs x 128 lanes x clock; None without a
    count for the current sources."""
    ipa = _inst_counts().get(name)
    if ipa is None:
        return None
    return {"inst_per_attempt": ipa, "achieved_tops": rate * ipa / 1e12, "peak_tops": peak_ops / 1e12,
            "frac": rate * ipa / peak_ops, "source": "profiles/" + COUNTS_FILE}


def workload_config(world: int) -> dict:
    """The benchmarked workload, identical in both arms' JSON lines."""
    from paper_1012_0385_gb300.sampling import log_times

    return {"workload": WORKLOAD_NAME, "L": L_SITES, "samples_per_gpu": SAMPLES, "n_mcs": N_MCS,
            "sample_times": len(log_times(N_MCS)), "domain_sites": DOMAIN,
            "schedule": "two-phase Poisson-domain RSU", "rates": {"p": P_RATE, "q": Q_RATE},
            "observables": "W^2 at the log times (hop counters off)",
            "l2": "flushed between steps (256 MB write outside the timed region)",
            "parallelism": f"replicas x{world} (disjoint sample ranges)"}


def run_reference(args):
    """The oracle as it stands, on the host cores: each timed step is one
    bounded sample of the workload (REF_STEP_S seconds of CPU work: a subset
    of the samples over a prefix of the sweeps, whole path), and the rate is
    the attempts those steps made over their time."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    for _ in range(args.warmup):
        cpu_oracle_sample(0.5)
    runs = [cpu_oracle_sample(REF_STEP_S) for _ in range(args.steps)]
    secs = [r["seconds"] for r in runs]
    value = sum(r["attempts"] for r in runs) / sum(secs)
    cores = runs[-1]["cores"]
    line = {"metric": "site-update attempts/s", "value": value, "unit": "attempts/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * statistics.mean(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "impl": "reference", "config": workload_config(args.gpus),
            "cpu_baseline": {"value": value, "unit": "attempts/s", "cores": cores, "kind": "oracle",
                             "value_per_core": value / cores,
                             "sample": "each step: " + runs[-1]["sample"] + " (the oracle's schedule replay)"},
            "e2e": {"value": value, "unit": "attempts/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch

    from paper_1012_0385_gb300 import asep as A
    from paper_1012_0385_gb300 import replicas
    from paper_1012_0385_gb300.sampling import log_times

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()

    th = A.asep_threshold
    times = log_times(N_MCS)
    first, count = replicas.sample_range(rank, world, SAMPLES)

    def params():
        return A.make_params(L=L_SITES, domain_sites=DOMAIN, samples_per_real=count, first_sample=first,
                             p_thr=th(P_RATE), q_thr=th(Q_RATE), seed=SEED, flags=A.ASEP_FLAG_NO_HOP_COUNTS)

    stream = torch.cuda.current_stream()
    ctx = A.asep_create(params(), sample_times=times)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")  # > 129 MB L2
    attempts_per_step = L_SITES * SAMPLES * N_MCS
    plan, tune_table = None, None
    if not args.no_autotune:
        from paper_1012_0385_gb300.autotune import autotune

        plan, tune_table = autotune(ctx, probe_sweeps=64)

    for w in range(args.warmup):
        A.asep_reset(ctx, seed=1000 + w)
        A.asep_sweep(ctx, N_MCS)
    torch.cuda.synchronize()

    launches0 = A.asep_get_info(ctx)["kernel_launches"]
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    step_ms, kern_ms = [], []
    for k in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        barrier()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        A.asep_reset(ctx, seed=SEED + k)
        e1.record(stream)
        A.asep_sweep(ctx, N_MCS)
        e2.record(stream)
        torch.cuda.synchronize()
        barrier()
        step_ms.append(e0.elapsed_time(e2))
        kern_ms.append(e1.elapsed_time(e2))
    clk = clocks.stop()
    launches = A.asep_get_info(ctx)["kernel_launches"] - launches0
    # sanity: the last step's width table is finite and starts at W^2 = 1/4
    _, _, w2 = A.asep_width(ctx)
    assert w2.shape[0] == len(times) and abs(w2[0].mean() - 0.25) < 1e-12 and w2[-1].mean() > 1.0
    A.asep_destroy(ctx)

    total_ms, kernel_ms = replicas.max_over_ranks([sum(step_ms), statistics.mean(kern_ms)], dist, device="cuda")
    value = replicas.throughput(attempts_per_step, args.steps, world, total_ms)

    # end to end through the C ABI with host buffers: create (host params and
    # sample times in), sweeps, W(t) table out, destroy
    e2e_steps = max(1, min(args.steps, 3))
    h2d = d2h = 0
    e2e_s = []
    for k in range(e2e_steps):
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        c = A.asep_create(params(), sample_times=times)
        if plan:  # the tuned plan, as a user applies a cached one
            A.asep_set_plan(c, plan.cluster, plan.samples_per_group if plan.cluster in (1, 32) else 0)
            A.asep_set_balance(c, plan.balance)
            A.asep_set_launch_sweeps(c, plan.launch_sweeps)
        A.asep_sweep(c, N_MCS)
        sh, sh2, w2 = A.asep_width(c)
        A.asep_destroy(c)
        torch.cuda.synchronize()
        e2e_s.append(time.perf_counter() - t0)
        h2d = 8 * len(times) + 4 * len(A.asep_poisson_table(DOMAIN)[1])
        d2h = sh.nbytes + sh2.nbytes
    (e2e_ms,) = replicas.max_over_ranks([1000.0 * statistics.mean(e2e_s)], dist, device="cuda")
    e2e_value = replicas.throughput(attempts_per_step, 1, world, e2e_ms)

    # the random stream alone: Philox4x32-10 calls/s with no lattice memory
    sink = torch.empty(152 * 8 * 256, dtype=torch.int32, device="cuda")
    A.asep_philox_bench(152 * 8, 256, 1 << 12, sink.data_ptr(), stream.cuda_stream)
    ph_ms = A.asep_philox_bench(152 * 8, 256, 1 << 14, sink.data_ptr(), stream.cuda_stream)
    philox_calls_s = 152 * 8 * 256 * (1 << 14) / (ph_ms / 1000.0)
    # the same stream driving the plain-ring bit operations on register-held
    # word pairs (no lattice memory): at full occupancy, and in the kernel's
    # own launch shape (one thread per column of every sample)
    rb_sink = torch.empty(2 * 152 * 8 * 256, dtype=torch.int32, device="cuda")
    pt, qt = th(P_RATE), th(Q_RATE)
    A.asep_attempt_bench(152 * 8, 256, 1 << 10, pt, qt, rb_sink.data_ptr(), stream.cuda_stream)
    rb_ms = A.asep_attempt_bench(152 * 8, 256, 1 << 13, pt, qt, rb_sink.data_ptr(), stream.cuda_stream)
    rb_attempts_s = 4 * 152 * 8 * 256 * (1 << 13) / (rb_ms / 1000.0)
    n_cols = SAMPLES * (L_SITES // (2 * DOMAIN))
    rbk_ms = A.asep_attempt_bench(max(1, n_cols // 256), 256, 1 << 13, pt, qt, rb_sink.data_ptr(), stream.cuda_stream)
    rbk_attempts_s = 4 * max(1, n_cols // 256) * 256 * (1 << 13) / (rbk_ms / 1000.0)

    if rank == 0:
        peaks = _peaks()
        max_mhz = float(peaks.get("sm_max_mhz", 2070.0))
        peak_ops = SMS * LANES_PER_SM * max_mhz * 1e6
        achieved_ops = L_SITES * SAMPLES * N_MCS / (kernel_ms / 1000.0) * OPS_PER_ATTEMPT
        headline_family = ("stream" if plan and plan.cluster == 32 else
                           "domain_bal" if plan and plan.balance else "domain")
        line = {
            "metric": "site-update attempts/s", "value": value, "unit": "attempts/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(world),
            "plan": ({"cluster": plan.cluster,
                      ("tile_columns" if plan.cluster == 32 else "samples_per_group"): plan.samples_per_group,
                      "balance_chunk_sweeps": plan.balance or "off",
                      "launch_sweeps": plan.launch_sweeps or "auto"} if plan else "default"),
            "roofline": {"bound": "alu", "achieved": achieved_ops / 1e12, "peak": peak_ops / 1e12,
                         "unit": "Tops/s", "frac": achieved_ops / peak_ops,
                         "traffic": _traffic_from_profile(headline_family),
                         "kernel": {"domain_bal": "k_domain_bal<ring> (balanced launch)",
                                    "stream": "k_stream<ring> (streamed tiles)"}.get(headline_family,
                                                                                      "k_domain<ring>"),
                         "kernel_ms": kernel_ms,
                         "ops_per_attempt": OPS_PER_ATTEMPT,
                         "peak_basis": f"{SMS} SMs x {LANES_PER_SM} int32 lanes/clk x {max_mhz:.0f} MHz (issue)",
                         "philox_only_attempts_per_s": 4 * philox_calls_s,
                         "rng_bitop_only_attempts_per_s": rb_attempts_s,
                         "rng_bitop_only_at_kernel_shape_attempts_per_s": rbk_attempts_s,
                         "frac_of_rng_bitop_only": value / rb_attempts_s},
            "issue": (_issue_fraction(value, "headline_" + headline_family, peak_ops)
                      if headline_family != "stream" else None),
            "smem": (_smem_fraction(value, "headline_" + headline_family, max_mhz)
                     if headline_family != "stream" else None),
            "e2e": {"value": e2e_value, "unit": "attempts/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": int(launches),
            "clocks": clk,
        }
        if tune_table:
            line["autotune"] = [{k: v for k, v in r.items() if k != "requested"} for r in tune_table]
            line["autotune_batch"] = batch_mode_table()
        if not args.no_workloads and world == 1:
            line["sca"] = sca_growth(max(1, min(args.steps, 5)), peak_ops)
            line["workloads"] = other_workloads(tune=not args.no_autotune, peak_ops=peak_ops, rng_bitop=rb_attempts_s)
        if not args.no_serving and world == 1:
            line["serving"] = serving_comparison(capacity=value)
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_oracle_sample(args.cpu_seconds)
            line["cpu_baseline"]["by_config"] = cpu_baselines_by_config()
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def batch_mode_table(n_contexts: int = 64, step_sweeps: int = 8, steps: int = 50):
    """The batch knob of the autotuner on small jobs, where launch overhead
    matters: 64 contexts of the served mix's small end (L in [2^10, 2^14],
    1-16 samples, the four families) advanced in steps of 8 sweeps, eager
    persistent launches against one captured CUDA graph replayed per step
    (bit-identical lattices required)."""
    from paper_1012_0385_gb300 import asep as A
    from paper_1012_0385_gb300 import autotune, serve

    jobs = serve.make_trace(n_contexts, seed=7, rate_hz=1.0, L_range=(1 << 10, 1 << 14), samples_range=(1, 16),
                            n_mcs_range=(100, 100))

    def make():
        return [A.asep_create(j.params(), sample_times=[]) for j in jobs]

    mode, rows = autotune.tune_batch_mode(make, [step_sweeps] * n_contexts, steps=steps)
    return {"choice": mode, "contexts": n_contexts, "step_sweeps": step_sweeps, "rows": rows}


def sca_growth(steps: int, peak_ops: float):
    """The benchmarked workload under the paper's own schedule, the
    two-sub-lattice SCA (k_sca): same rings, rates, sweeps and sample times,
    re-drawn initial state + 2^14 sweeps per step, device-timed."""
    import torch

    from paper_1012_0385_gb300 import asep as A
    from paper_1012_0385_gb300.sampling import log_times

    th = A.asep_threshold
    prm = A.make_params(L=L_SITES, schedule=A.ASEP_SCHED_SCA, samples_per_real=SAMPLES, p_thr=th(P_RATE),
                        q_thr=th(Q_RATE), seed=SEED, flags=A.ASEP_FLAG_NO_HOP_COUNTS)
    stream = torch.cuda.current_stream()
    with A.asep_create(prm, sample_times=log_times(N_MCS)) as ctx:
        A.asep_sweep(ctx, 256)  # warm-up
        ms = []
        for k in range(steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            A.asep_reset(ctx, seed=SEED + k)
            A.asep_sweep(ctx, N_MCS)
            e1.record(stream)
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        info = A.asep_get_info(ctx)
    t = statistics.mean(ms)
    rate = L_SITES * SAMPLES * N_MCS / (t / 1000.0)
    achieved = rate * SCA_OPS_PER_ATTEMPT
    return {"workload": "the same growth-regime workload under the paper's two-sub-lattice SCA schedule "
                        "(even bonds, then odd bonds, one attempt per bond per sweep)",
            "attempts_per_s": rate, "ms_per_step": t, "steps": steps, "kernel": "k_sca",
            "threads_per_cta": info["threads"],
            "roofline": {"bound": "alu", "achieved": achieved / 1e12, "peak": peak_ops / 1e12, "unit": "Tops/s",
                         "frac": achieved / peak_ops, "ops_per_attempt": SCA_OPS_PER_ATTEMPT,
                         "traffic": _traffic_from_profile("sca")}}


def window_cases():
    """(name, parameters, sample times, lanes) of the windows of the other
    configurations (see other_workloads)."""
    from paper_1012_0385_gb300 import asep as A
    from paper_1012_0385_gb300.sampling import every, log_times

    th = A.asep_threshold
    win = 10_000
    lt = log_times(win) + ([win] if log_times(win)[-1] != win else [])
    t0 = min(t for t in lt if t >= win // 2)
    cases = [
        ("plain TASEP, serial RSU: L=4096, p=1 q=0, flat, 10^4 MCS, 8 samples, snapshots every 100",
         dict(L=4096, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=8, p_thr=A.ASEP_ALWAYS, q_thr=0, seed=1),
         every(100, win), 1),
        ("plain TASEP, domain schedule D=256: L=4096, p=1 q=0, flat, 10^4 MCS, 8 samples, snapshots every 100",
         dict(L=4096, domain_sites=256, samples_per_real=8, p_thr=A.ASEP_ALWAYS, q_thr=0, seed=1), every(100, win), 1),
        ("quenched bimodal disorder: L=2^16, p_i=1 or 0.3 (Q=0.1), q=0, 64 realizations x 4 samples, "
         "10^4-MCS window, log times",
         dict(L=1 << 16, domain_sites=256, n_realizations=64, samples_per_real=4, p_thr=A.ASEP_ALWAYS, q_thr=0,
              dis_kind=A.ASEP_DIS_BIMODAL, dis_a_thr=th(0.1), dis_b_thr=th(0.3), dis_seed=2, seed=1), lt, 1),
        ("two lanes: 2 x L=2^16, rate 1 both lanes, turning density 0.05, omega 0.1, Bernoulli(1/2) start, "
         "128 samples, 10^4-MCS window, currents + profile + autocorrelation, D=128 (256 bonds per domain)",
         dict(model=A.ASEP_MODEL_TWO_LANE, L=1 << 16, domain_sites=128, samples_per_real=128,
              p_thr=A.ASEP_ALWAYS, q_thr=A.ASEP_ALWAYS, dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05),
              dis_b_thr=th(0.1), dis_seed=3, init_kind=A.ASEP_INIT_BERNOULLI_HALF, init_seed=4, seed=1,
              flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=t0), lt, 2),
        ("two lanes, the paper's SCA sequence (even bonds, A->B, odd bonds, B->A) with its in-lane rate 0.5: "
         "2 x L=2^16, turning density 0.05, omega 0.1, Bernoulli(1/2) start, 128 samples, 10^4-MCS window",
         dict(model=A.ASEP_MODEL_TWO_LANE, L=1 << 16, schedule=A.ASEP_SCHED_SCA, samples_per_real=128,
              p_thr=th(0.5), q_thr=th(0.5), dis_kind=A.ASEP_DIS_TURNING, dis_a_thr=th(0.05), dis_b_thr=th(0.1),
              dis_seed=3, init_kind=A.ASEP_INIT_BERNOULLI_HALF, init_seed=4, seed=1,
              flags=A.ASEP_FLAG_PROFILE | A.ASEP_FLAG_AUTOCORR, autocorr_t0=t0), lt, 2),
        ("Q-SSEP (the paper's quenched SSEP, SCA schedule, its p=0.8): L=2^16, p=q=0.8, independent slow classes "
         "for right and left hops (Q=0.5 each, r=0.2), 256 realizations, 10^4-MCS window, log times",
         dict(L=1 << 16, schedule=A.ASEP_SCHED_SCA, n_realizations=256, samples_per_real=1, p_thr=th(0.8),
              q_thr=th(0.8), dis_kind=A.ASEP_DIS_BIMODAL_PQ, dis_a_thr=th(0.5), dis_b_thr=th(0.16),
              dis_c_thr=th(0.16), dis_seed=2, seed=1), lt, 1),
        ("streamed tier: L=2^24 rings (beyond a 16-CTA cluster; lattice in HBM, tiles through shared memory), "
         "ASEP p=0.75 q=0.25, 16 samples, 200-MCS window",
         dict(L=1 << 24, domain_sites=256, samples_per_real=16, p_thr=th(0.75), q_thr=th(0.25), seed=1,
              flags=A.ASEP_FLAG_NO_HOP_COUNTS), [200], 1),
        ("streamed SCA: L=2^28 rings (the paper's one-large-sample-per-GPU mode; lattice in HBM, a thread per "
         "8 words, one launch per phase), ASEP p=0.75 q=0.25, 8 samples (256 MB, beyond L2), 200-MCS window",
         dict(L=1 << 28, schedule=A.ASEP_SCHED_SCA, samples_per_real=8, p_thr=th(0.75), q_thr=th(0.25), seed=1,
              flags=A.ASEP_FLAG_NO_HOP_COUNTS), [200], 1),
    ]
    return cases


def other_workloads(tune: bool = True, peak_ops: float | None = None, rng_bitop: float | None = None):
    """Device-timed windows of the other configurations of the study (one
    run each after a warm-up launch, CUDA events on the launching stream):
    plain TASEP under serial RSU and under the domain schedule (full 10^4
    sweeps, snapshots every 100), quenched bimodal disorder and the two-lane
    model with turning sites (10^4-sweep windows of their 10^7 / 10^6 sweep
    runs, log-spaced sample times, two-lane currents, profile and
    autocorrelation on), the latter also under the paper's two-lane SCA; the
    paper's quenched SSEP (independent slow classes for both directions); and
    the two streamed modes (domain schedule and SCA) on rings far beyond
    shared memory.  Resident domain-schedule windows first take the
    autotuner's plan (bit-exactness guarded; `tune`)."""
    import torch

    from paper_1012_0385_gb300 import asep as A
    from paper_1012_0385_gb300.sampling import every, log_times

    cases = window_cases()
    counts = _window_counts()
    stream = torch.cuda.current_stream()
    out = []
    for wi, (name, kw, times, lanes) in enumerate(cases):
        with A.asep_create(A.make_params(**kw), sample_times=times) as ctx:
            tuned = None
            if tune and kw.get("schedule", A.ASEP_SCHED_DOMAIN) == A.ASEP_SCHED_DOMAIN:
                from paper_1012_0385_gb300.autotune import autotune

                choice, _ = autotune(ctx, probe_sweeps=16)
                tuned = {"cluster": choice.cluster, ("tile_columns" if choice.cluster == 32 else "samples_per_group"):
                         choice.samples_per_group,
                         "balance_chunk_sweeps": choice.balance or "off",
                         "launch_sweeps": choice.launch_sweeps or "auto", "autotuned": True}
            A.asep_reset(ctx, seed=kw["seed"], init_seed=kw.get("init_seed", 0))
            A.asep_sweep(ctx, 8)  # warm-up launch
            A.asep_reset(ctx, seed=kw["seed"], init_seed=kw.get("init_seed", 0))
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            n_sweeps = max(times) if times else win
            A.asep_sweep(ctx, n_sweeps)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            info = A.asep_get_info(ctx)
            attempts = lanes * kw["L"] * info["S"] * n_sweeps
            row = {"workload": name, "attempts": attempts, "ms": ms, "attempts_per_s": attempts / (ms / 1e3),
                   "kernel": ("k_serial" if kw.get("schedule") == A.ASEP_SCHED_SERIAL
                              else ("k_sca_stream" if info["cluster"] == 32 else "k_sca")
                              if kw.get("schedule") == A.ASEP_SCHED_SCA
                              else "k_stream" if info["cluster"] == 32
                              else "k_cluster" if info["cluster"] > 1 else "k_domain"),
                   "samples_per_group": info["samples_per_group"]}
            if tuned:
                row["plan"] = tuned
            # issue-slot roofline: measured instructions per attempt x attempts/s over the SMs' issue rate
            if peak_ops and wi in counts:
                ach = row["attempts_per_s"] * counts[wi]
                row["roofline"] = {"bound": "alu", "unit": "Tops/s", "achieved": ach / 1e12, "peak": peak_ops / 1e12,
                                   "frac": ach / peak_ops, "inst_per_attempt": counts[wi],
                                   "basis": "thread instructions per attempt (ncu, profiles/" + COUNTS_FILE +
                                            ") x attempts/s, over 152 SMs x 128 lanes x clock"}
                if rng_bitop and WINDOW_KERNELS[wi] in ("serial", "domain", "stream"):
                    row["roofline"]["frac_of_rng_bitop_only"] = row["attempts_per_s"] / rng_bitop
                sm = _smem_fraction(row["attempts_per_s"], f"window{wi}", peak_ops / (SMS * LANES_PER_SM * 1e6))
                if sm:  # shared-memory bandwidth: wavefronts per attempt (ncu) x attempts/s over 1 per SM and clock
                    row["roofline"]["smem_frac"] = sm["frac"]
                    row["roofline"]["smem_wavefronts_per_attempt"] = sm["wavefronts_per_attempt"]
            if info["cluster"] == 32:
                # streamed: each phase reads and writes every lattice word once (4 x L/8 bytes per plane
                # and sweep); the whole window, launch gaps and records included, against measured HBM
                alg = 4 * (kw["L"] // 8) * lanes * info["S"] * n_sweeps
                gbs = alg / (ms / 1e3) / 1e9
                measured = _peaks().get("hbm_gbs")
                peak = measured or 6800.0
                row["hbm"] = {"algorithmic_bytes": alg, "achieved_gbs": gbs, "peak_gbs": peak, "frac": gbs / peak,
                              "peak_basis": "of measured copy bandwidth" if measured else "of fallback 6.8 TB/s"}
                if kw.get("schedule") == A.ASEP_SCHED_SCA:
                    row["hbm"]["traffic_per_launch"] = _traffic_from_profile("sca_stream")
            out.append(row)
    return out


def serving_comparison(capacity: float, n_jobs: int = 500, seed: int = 2026, load: float = 0.4,
                       n_burst: int = 200, burst_seed: int = 77):
    """The served ensemble mix (configuration 4) in a time-scaled reading,
    replayed with continuous batching (admission by the library's device- and
    shared-memory plan, up to 10^4 jobs in flight, age-weighted quanta) and
    with one launch per job, on the same GPU; results bit-identical between
    the two.  Jobs are drawn from the four workload families (plain TASEP,
    ASEP growth, bimodal disorder, two lanes) with L log-uniform in [2^10,
    2^22] (the mix's full range; L above ~2^19 runs on thread-block
    clusters), 1-256 samples and n_mcs log-uniform in [5, 5000] (the mix's
    10^3-10^6 divided by 200, so that both modes finish in minutes).  Two
    regimes: `latency` -- n_jobs Poisson arrivals offering 40 % of the
    headline kernel's rate (about 80 % of what the batched server sustains on
    this mix: two-lane, disordered and cluster-tier jobs run slower than the
    benchmarked ring), where throughput follows the arrivals and the
    latencies differ; `capacity` -- n_burst jobs arriving at once, where the
    makespan measures each mode's throughput."""
    from paper_1012_0385_gb300 import serve

    def trace(n, sd, at_zero):
        t = serve.make_trace(n, seed=sd, rate_hz=1.0, L_range=(1 << 10, 1 << 22), samples_range=(1, 256),
                             n_mcs_range=(5, 5000), load=load, capacity=capacity)
        if at_zero:
            for j in t:
                j.arrival = 0.0
        return t

    out = {}
    for regime, n, sd, at_zero in (("latency", n_jobs, seed, False), ("capacity", n_burst, burst_seed, True)):
        batched_jobs, plain_jobs = trace(n, sd, at_zero), trace(n, sd, at_zero)
        batched = serve.serve_batched(batched_jobs, quantum_s=0.02)
        plain = serve.serve_plain(plain_jobs)
        same = all(np.array_equal(a.result[k], b.result[k]) for a, b in zip(batched_jobs, plain_jobs)
                   for k in ("sum_h", "sum_h2", "counters"))
        desc = (f"{n} jobs arriving together" if at_zero else
                f"{n} jobs, Poisson ~{n / max(j.arrival for j in batched_jobs):.2f} Hz (offered load {load:g} of "
                f"{capacity:.3g} attempts/s)")
        out[regime] = {
            "trace": desc + ", kinds tasep/asep/bimodal/two_lane, L log-uniform [2^10, 2^22], samples "
                            "log-uniform [1, 256], n_mcs log-uniform [5, 5000] (the configuration's [10^3, 10^6] / 200)",
            "batched": batched, "plain": plain, "results_identical": bool(same),
            "throughput_ratio": batched["throughput_attempts_per_s"] / plain["throughput_attempts_per_s"],
            "p50_ratio": batched["p50_latency_s"] / plain["p50_latency_s"],
            "p99_ratio": batched["p99_latency_s"] / plain["p99_latency_s"]}
    return out


def profile_case(schedule: str = "domain"):
    """Short untimed runs of one kernel each, for ncu:
    "domain"      the benchmarked configuration, 64 sweeps in one launch of
                  k_domain (one record, at the end; the kernel reads and
                  writes each lattice once per launch, so its DRAM traffic per
                  launch is that of a full step);
    "domain_bal"  the same as a balanced launch (k_domain_bal), 512 sweeps in
                  chunks of 32: the groups move between SMs 16 times;
    "sca"         the same workload under the two-sub-lattice SCA (k_sca);
    "sca_stream"  two sweeps (four launches, one per phase) of the streamed
                  SCA on 8 rings of 2^28 sites (256 MB);
    "stream"      two sweeps (four launches) of the streamed domain tier
                  (k_stream) on 16 rings of 2^24 sites (32 MB), the bench's
                  streamed window;
    "serial"      1000 sweeps of the serial schedule on the plain-TASEP
                  configuration (L = 4096, 8 samples; its automatic plan, one
                  CTA per sample running each sweep in dependency rounds);
    "window<i>"   window i of window_cases(), 32 sweeps (streamed: 2);
    "attempt_bench" the RNG + bit-op microbenchmark at full occupancy
                  (152 x 8 CTAs of 256 threads, 4096 Philox calls each), the
                  measured roof of the domain schedule."""
    import torch

    from paper_1012_0385_gb300 import asep as A

    th = A.asep_threshold
    if schedule == "attempt_bench":
        sink = torch.empty(2 * 152 * 8 * 256, dtype=torch.int32, device="cuda")
        ms = A.asep_attempt_bench(152 * 8, 256, 1 << 12, th(P_RATE), th(Q_RATE), sink.data_ptr(),
                                  torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
        print(f"profile case done: attempt_bench {152 * 8 * 256 * 4 * (1 << 12) / (ms / 1e3):.3e} attempts/s",
              flush=True)
        return 0
    if schedule.startswith("window"):
        # one window of the other configurations, briefly: 32 sweeps (streamed ones 2), one record at the end
        name, kw, times, lanes = window_cases()[int(schedule[len("window"):])]
        kw = dict(kw)
        n = 2 if kw["L"] >= 1 << 24 else 32
        if kw.get("flags", 0) & A.ASEP_FLAG_AUTOCORR:
            kw["autocorr_t0"] = n
        with A.asep_create(A.make_params(**kw), sample_times=[n]) as ctx:
            A.asep_sweep(ctx, n)
            A.asep_sync(ctx)
            info = A.asep_get_info(ctx)
        torch.cuda.synchronize()
        print(f"profile case done: {name}; attempts {lanes * kw['L'] * info['S'] * n} in {n} sweeps", flush=True)
        return 0
    if schedule in ("sca_stream", "stream", "serial"):
        if schedule == "sca_stream":
            prm = A.make_params(L=1 << 28, schedule=A.ASEP_SCHED_SCA, samples_per_real=8, p_thr=th(P_RATE),
                                q_thr=th(Q_RATE), seed=SEED, flags=A.ASEP_FLAG_NO_HOP_COUNTS)
            n = 2
        elif schedule == "stream":
            prm = A.make_params(L=1 << 24, domain_sites=256, samples_per_real=16, p_thr=th(P_RATE), q_thr=th(Q_RATE),
                                seed=SEED, flags=A.ASEP_FLAG_NO_HOP_COUNTS)
            n = 2
        else:
            prm = A.make_params(L=4096, schedule=A.ASEP_SCHED_SERIAL, samples_per_real=8, p_thr=A.ASEP_ALWAYS,
                                q_thr=0, seed=SEED)
            n = 1000
        with A.asep_create(prm, sample_times=[]) as ctx:
            A.asep_sweep(ctx, n)
            A.asep_sync(ctx)
        torch.cuda.synchronize()
        print("profile case done", flush=True)
        return 0
    sched = A.ASEP_SCHED_SCA if schedule == "sca" else A.ASEP_SCHED_DOMAIN
    prm = A.make_params(L=L_SITES, domain_sites=DOMAIN, samples_per_real=SAMPLES, p_thr=th(P_RATE),
                        q_thr=th(Q_RATE), seed=SEED, flags=A.ASEP_FLAG_NO_HOP_COUNTS, schedule=sched)
    n = 512 if schedule == "domain_bal" else 64
    # one record, at the end: the full run records 131 times in 2^14 sweeps
    with A.asep_create(prm, sample_times=[n]) as ctx:
        if schedule == "domain_bal":
            A.asep_set_balance(ctx, 32)
        A.asep_sweep(ctx, n)
        A.asep_sync(ctx)
    torch.cuda.synchronize()
    print("profile case done", flush=True)
    return 0


def main():
    global DOMAIN
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-serving", action="store_true", help="skip the served-mix comparison")
    ap.add_argument("--no-workloads", action="store_true", help="skip the windows of the other configurations")
    ap.add_argument("--no-autotune", action="store_true", help="keep the automatic launch plan")
    ap.add_argument("--domain", type=int, default=DOMAIN, help="domain sites D of the schedule (default 256)")
    ap.add_argument("--profile-case", nargs="?", const="domain",
                    choices=["domain", "domain_bal", "sca", "sca_stream", "stream", "serial", "attempt_bench"] +
                    [f"window{i}" for i in range(8)],
                    help="a short untimed run of one kernel for ncu (see profile_case)")
    args = ap.parse_args()
    if args.profile_case:
        return profile_case(args.profile_case)
    if args.warmup < 3:
        args.warmup = 3
    DOMAIN = args.domain
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
