#!/usr/bin/env python
"""Benchmark of exact mod-p Gauss-Jordan elimination to RREF on GB300.

Headline workload: the dense 32768 x 33024 system over F_p, p = 2^31 - 1
(A 32768 x 32768 plus 256 right-hand-side columns, uniform residues, full
rank), reduced in place by linac_rref.  One step = one complete RREF.
Metric: field multiply-adds per second, counted as the Gauss-Jordan work
W = sum over pivots t of (m - 1) * (n - c_t - 1), the multiply-adds the
paper's column-by-column elimination performs (section 3.2), whatever the
blocking.

Timing: W >= 3 untimed warm-up steps, then K timed steps bracketed by a
barrier and torch.cuda.synchronize(); every step restores the pristine input
with a full device copy (4.3 GB, larger than L2) outside its CUDA events, so
each timed elimination starts from cold L2.  With --gpus N under torchrun
every rank reduces its own copy (replicas; the elimination of one matrix
does not shard) and value = total work / max rank time.

Also reported: the dominant kernel's roofline (CUDA events around each of
its launches, on the launch stream), the e2e rate through the public API
with host buffers (pinned H2D, RREF, D2H each step), the CPU oracle on a
bounded sample of the same workload, the u8-limb tensor path beside the
plain path, the batched workload (systems/s), the shared-pattern batch, the
construction leg and the uint64 leg (RREF of 8192 x 8448 at p = 2^64 - 59).

--impl reference times the CPU oracle alone (rank 0), on bounded samples of
the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "mod-p MACs/s for RREF at n=32768 (tensor vs plain path); batched systems/s"
UNIT = "field MAC/s"
P31 = 2**31 - 1
# 64-bit-accumulating integer multiply-adds (mad.wide.s32) per SM per clock:
# 4 schedulers x a 16-lane multiply pipe, two passes per wide multiply-add
# (ncu: ~4 pipe cycles per 32-thread warp instruction on GB300)
IMAD_WIDE_PER_SM_CLK = 32
# DRAM bytes moved by the batched kernels per byte of the batch's matrices
# (ncu: 1.627 + 1.875 GB and 0.024 + 0.0002 GB read + written by the two
# launches of the 2000-system uneven batch, whose matrices hold 0.385 GB;
# summary in profiles/batched_uneven_bucket512.md)
BATCHED_DRAM_PER_MATRIX_BYTE = 3.358e9 / 0.3854e9

# DRAM bytes per output of the update kernels from one ncu capture each
# (dram__bytes_read.sum + dram__bytes_write.sum of one panel's update in the
# 8192 x 8448 elimination, divided by its outputs; summaries in
# profiles/update_plain_rref_8192x8448.md and
# profiles/update_hybrid_rref_8192x8448.md), valid while the kernel's sources
# hash to the recorded fingerprint; the traffic is reported as null otherwise
_CSRC = "paper_2605_25863_gb300/csrc/"
UPDATE_TRAFFIC = {
    "update_plain": {"bytes_per_output": 478.12e6 / (8192 * 8192), "sha": "4401ada011c488ff",
                     "files": [_CSRC + f for f in ("update_plain.cu", "update_tiles.cuh", "update.cuh",
                                                    "linac_device.cuh")]},
    "update_hybrid": {"bytes_per_output": 504.68e6 / (8192 * 8192), "sha": "76956f08df59e200",
                      "files": [_CSRC + f for f in ("update_hybrid.cu", "update_tiles.cuh", "update.cuh",
                                                     "linac_device.cuh")]},
}


def parse():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--m", type=int, default=32768, help="rows (= unknowns) of the dense system")
    ap.add_argument("--rhs", type=int, default=256, help="right-hand-side columns")
    ap.add_argument("--nb", type=int, default=128, help="panel width")
    ap.add_argument("--path", default="auto", choices=["auto", "plain", "limb", "crt", "hybrid"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="CPU oracle sample budget")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the CPU oracle, path comparison and batched legs")
    ap.add_argument("--batch-count", type=int, default=10000)
    ap.add_argument("--only", choices=["all", "batched", "construction", "dense64"], default="all",
                    help="batched / construction: run that workload alone (a profiling aid; prints its own line)")
    ap.add_argument("--m64", type=int, default=8192, help="unknowns of the uint64 leg's system")
    ap.add_argument("--widths", default="",
                    help="comma-separated panel widths per size bucket for the batched legs (default: autotune)")
    ap.add_argument("--measure-peaks", action="store_true",
                    help="print the measured integer pipe rates (roofline denominators) and exit")
    return ap.parse_args()


def gj_work(m: int, n: int, pivots) -> int:
    """Field multiply-adds of Gauss-Jordan elimination: sum_t (m-1)(n-c_t-1)."""
    piv = np.asarray(pivots, dtype=np.int64)
    return int(((m - 1) * (n - piv - 1)).sum())


def update_work(m: int, n: int, pivots, nb: int) -> int:
    """Useful multiply-adds of the blocked trailing updates: per panel starting
    at c0 with k pivots, (m - k) rows x (n - c0) columns x k."""
    piv = np.asarray(pivots, dtype=np.int64)
    total = 0
    for c0 in range(0, n, nb):
        k = int(((piv >= c0) & (piv < c0 + nb)).sum())
        total += (m - k) * (n - c0) * k
    return total


def replica_rate(local_ms: float, local_work: float, world: int, device) -> tuple[float, float]:
    """Whole-job rate of N independent replicas (weak scaling): every rank did
    the same work; the job took as long as the slowest rank, so the time is
    the maximum over ranks (an all-reduce on the process group when world > 1)
    and the rate is world x work / that time.  Returns (rate, max_ms)."""
    max_ms = local_ms
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([local_ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        max_ms = float(t.item())
    return world * local_work / (max_ms / 1000.0), max_ms


def device_sms_and_max_clock(dev) -> tuple[int, float, str]:
    """SM count (CUDA device properties) and maximum SM clock in MHz
    (nvidia-smi clocks.max.sm) of the benchmarked device."""
    import torch
    props = torch.cuda.get_device_properties(dev)
    sms = int(props.multi_processor_count)
    uuid = getattr(props, "uuid", None)
    cmd = ["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits"]
    if uuid:
        cmd.insert(1, f"--id=GPU-{uuid}")
    try:
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=30).stdout.strip().splitlines()
        return sms, float(out[0]), "nvidia-smi clocks.max.sm"
    except Exception as e:   # no nvidia-smi: the clock rate CUDA reports
        clk = getattr(props, "clock_rate", 0) / 1000.0
        if clk <= 0:
            raise RuntimeError(f"cannot read the maximum SM clock: {e}")
        return sms, clk, "CUDA device clock rate"


def src_sha(files) -> str:
    import hashlib
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def update_outputs(m: int, n: int, nb: int) -> int:
    """Outputs written by the trailing updates of one elimination: m rows x
    (n - c0) columns per panel start c0 (a panel without pivots launches no
    update; the bench matrix has full rank)."""
    return sum(m * (n - c0) for c0 in range(0, min(m, n), nb))


def workload_name(m, n, rhs):
    return (f"dense RREF over F_p, p = 2^31 - 1: {m} x {n} (A {m} x {m} plus {rhs} right-hand "
            f"sides), uniform residues, full rank")


def fold_of(p: int) -> int:
    c32 = (1 << 32) % p
    half = (p - 1) // 2
    amax = max(((1 << 31) - 1) * c32 + (1 << 32) - 1, (1 << 31) * c32)
    f = ((1 << 63) - 1 - amax) // (half * half)
    return 16 if f >= 16 else (8 if f >= 8 else 4)


# ---------------------------------------------------------------------------
# clocks during the timed region

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.lines: list[str] = []
        self.err = None
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
            if gpu_id:
                cmd.insert(1, f"--id={gpu_id}")
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception as e:  # nvidia-smi missing
            self.proc = None
            self.err = str(e)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"error": self.err}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"error": "no samples", "samples": len(self.lines)}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm), "sm_mhz_min": min(sm)}


# ---------------------------------------------------------------------------
# CPU oracle on a bounded sample of the workload

def cpu_oracle_sample(M: np.ndarray, p: int, budget_s: float, cores: int):
    """Time the oracle on the first P pivot steps of M (P sized to the
    budget).  Returns (rate, seconds, P, macs)."""
    import oracle
    m, n = M.shape
    t0 = time.perf_counter()
    _, r, piv, _ = oracle.rref(M, p, max_pivots=1, nthreads=cores)
    t1 = time.perf_counter() - t0
    P = max(1, min(m, int(budget_s / max(t1, 1e-3))))
    t0 = time.perf_counter()
    _, r, piv, _ = oracle.rref(M, p, max_pivots=P, nthreads=cores)
    dt = time.perf_counter() - t0
    macs = gj_work(m, n, piv)
    return macs / dt, dt, int(r), macs


def host_matrix(m: int, n: int, p: int, seed: int = 5) -> np.ndarray:
    from paper_2605_25863_gb300 import synth
    import torch
    t = synth.uniform_torch(m, n, p, synth.stream_key(seed, "large_dense"), device="cpu")
    return t.numpy().view(np.uint32)


# ---------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    m, n = args.m, args.m + args.rhs
    cores = os.cpu_count() or 1
    M = host_matrix(m, n, P31)
    steps, warm = args.steps, args.warmup
    per_step = max(2.0, 120.0 / max(1, steps + warm))
    for _ in range(warm):
        cpu_oracle_sample(M, P31, per_step, cores)
    rates, secs, samples = [], [], []
    for _ in range(steps):
        rate, dt, P, macs = cpu_oracle_sample(M, P31, per_step, cores)
        rates.append(rate)
        secs.append(dt)
        samples.append(P)
    value = float(sum(r * s for r, s in zip(rates, secs)) / sum(secs))
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": steps, "warmup": warm, "ms_per_step": 1000.0 * sum(secs) / steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": workload_name(m, n, args.rhs), "m": m, "n": n, "p": P31},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"first {samples} pivot steps (of {m}) of the {m} x {n} elimination "
                                   f"per step, {cores} threads"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args):
    import torch
    import torch.distributed as dist

    import __graft_entry__
    __graft_entry__.build()
    from paper_2605_25863_gb300 import linac, synth

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    if args.only == "batched":
        print(json.dumps({"batched": batched_leg(args, linac, synth, dev, stream)}), flush=True)
        return 0
    # pinned staging buffers of the e2e leg, allocated once at start-up as an
    # application would (4.3 GB transfers through pinned buffers allocated
    # later in the process were measured up to 10x slower)
    staging = None
    if rank == 0 and not args.no_extras and args.only == "all":
        staging = (torch.empty((args.m, args.m + args.rhs), dtype=torch.int32, pin_memory=True),
                   torch.empty((args.m, args.m + args.rhs), dtype=torch.int32, pin_memory=True))
    if args.only == "construction":
        print(json.dumps({"construction": construction_leg(args, linac, synth, dev)}), flush=True)
        return 0
    if args.only == "dense64":
        print(json.dumps({"dense64": dense64_leg(args, linac, synth, dev)}), flush=True)
        return 0

    m, rhs = args.m, args.rhs
    n = m + rhs
    p = P31
    nb = args.nb
    key = synth.stream_key(5, "large_dense")
    pristine = synth.uniform_torch(m, n, p, key, device=dev)          # int32 view of the residues
    work = torch.empty_like(pristine)

    def step(path=args.path):
        work.copy_(pristine)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        r, piv = linac.linac_rref(work, p, nb=nb, path=path)
        e1.record(stream)
        return e0, e1, r, piv

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)
    sampler = ClockSampler(f"GPU-{uuid}" if uuid else None)
    linac.linac_profile_reset()
    linac.linac_profile_enable(True)
    launches0 = linac.linac_launch_count()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("bench_timed")     # ncu --nvtx --nvtx-include "bench_timed/"
    events = [step() for _ in range(args.steps)]
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    if world > 1:
        dist.barrier()
    launches = linac.linac_launch_count() - launches0
    clocks = sampler.stop()
    linac.linac_profile_enable(False)
    prof = linac.linac_profile_read()

    step_ms = [a.elapsed_time(b) for a, b, _, _ in events]
    rank_v = int(events[-1][2].item())
    piv = events[-1][3].cpu().numpy()[:rank_v]
    ok = rank_v == m and np.array_equal(piv, np.arange(m))
    content = content_check(linac, pristine, work, m, p) if ok else {"checked": False}
    ok = ok and content.get("identity_block", False) and content.get("freivalds", False)
    work_macs = gj_work(m, n, piv)
    value, tot_ms = replica_rate(sum(step_ms), work_macs * args.steps, world, dev)

    # dominant kernel: the trailing update
    # the update kernel that ran (LINAC_PATH_AUTO picks by size): the update
    # class with the largest timed share
    upd_name = max((k for k in prof if k.startswith("update")), key=lambda k: prof[k][1], default="update_plain")
    upd_launches, upd_ms = prof.get(upd_name, (0, 0.0))
    upd_macs = update_work(m, n, piv, nb) * args.steps
    fold = fold_of(p)
    shift_fold = bin((1 << 32) % p).count("1") <= 3       # folds run on the ALU pipe
    imad_per_mac = 1.0 if shift_fold else 1.0 + 2.0 / fold
    achieved = upd_macs / (upd_ms / 1000.0) if upd_ms else 0.0
    traffic = None
    tr = UPDATE_TRAFFIC.get(upd_name)
    if tr and tr["bytes_per_output"] and upd_launches and src_sha(tr["files"]) == tr["sha"]:
        traffic = tr["bytes_per_output"] * update_outputs(m, n, nb) * args.steps / upd_launches
    sms, sm_max_mhz, clk_src = device_sms_and_max_clock(dev)
    peak = sms * IMAD_WIDE_PER_SM_CLK * sm_max_mhz * 1e6 / imad_per_mac
    rates = imma_peak()
    s8_peak, u8_peak = rates["imma_s8_mac_per_s"], rates["imma_u8_mac_per_s"]
    # what the two pipes deliver together: in the probe's mixed block each
    # group keeps only a fraction of its solo rate (time alone / time together)
    fi = rates["coissue_imad_only_ms"] / rates["coissue_both_ms"]
    ft = rates["coissue_imma_only_ms"] / rates["coissue_both_ms"]
    coissue = rates["imad_wide_per_s"] / imad_per_mac * fi + s8_peak / PATH_NARROW["crt"] * ft
    peaks = {"plain": peak, "plain_basis": f"{sms} SMs x {IMAD_WIDE_PER_SM_CLK} mad.wide.s32/clk x "
                                           f"{sm_max_mhz:.0f} MHz / {imad_per_mac:.3f} per field MAC",
             "imma_s8": s8_peak, "imma_u8": u8_peak, "coissue": coissue,
             "coissue_basis": f"measured mad.wide.s32 rate x {fi:.2f} + measured s8 mma.sync rate / 9 x {ft:.2f} "
                              f"(fractions of each pipe's solo rate kept when 8 warps of each run in one block, "
                              f"probes/int_rates.cu)"}
    if upd_name == "update_plain":
        roof = {"kernel": upd_name, "bound": "alu", "achieved": achieved / 1e12,
                "peak": peak / 1e12, "unit": "Tfield-MAC/s", "frac": achieved / peak if peak else None,
                "traffic": traffic,
                "traffic_basis": "ncu DRAM bytes per output of the 8192 x 8448 capture x outputs per launch"
                                 if traffic is not None else "kernel changed since the ncu capture",
                "peak_basis": f"{sms} SMs x {IMAD_WIDE_PER_SM_CLK} mad.wide.s32/clk x {sm_max_mhz:.0f} MHz"
                              f" ({clk_src})"
                              f" / {imad_per_mac:.3f} per field MAC"
                              f" ({'folds on the ALU pipe' if shift_fold else f'fold every {fold} on the multiply pipe'})",
                "avg_launch_ms": upd_ms / max(1, upd_launches), "launches": upd_launches}
    elif upd_name == "update_hybrid":   # both pipes at once
        both = peak + s8_peak / PATH_NARROW["crt"]
        co = peaks["coissue"]
        roof = {"kernel": upd_name, "bound": "alu", "achieved": achieved / 1e12, "peak": both / 1e12,
                "unit": "Tfield-MAC/s", "frac": achieved / both, "traffic": traffic,
                "traffic_basis": "ncu DRAM bytes per output of the 8192 x 8448 capture x outputs per launch"
                                 if traffic is not None else "kernel changed since the ncu capture",
                "peak_basis": "multiply-pipe peak + measured s8 mma.sync rate / 9: both pipes at full rate at "
                              "once, which this chip does not sustain (coissue_ceiling)",
                "coissue_ceiling": {"value": co / 1e12, "frac": achieved / co, "basis": peaks["coissue_basis"]},
                "avg_launch_ms": upd_ms / max(1, upd_launches), "launches": upd_launches}
    else:   # integer tensor pipe: narrow products per second against the measured mma.sync rate
        narrow = PATH_NARROW[args.path]
        tpeak = u8_peak if args.path == "limb" else s8_peak
        roof = {"kernel": upd_name, "bound": "tensor", "achieved": achieved * narrow / 1e12,
                "peak": tpeak / 1e12, "unit": "T narrow-MAC/s", "frac": achieved * narrow / tpeak,
                "traffic": None, "traffic_basis": "not captured for this path",
                "peak_basis": "measured mma.sync m16n8k32 rate (probes/int_rates.cu)",
                "avg_launch_ms": upd_ms / max(1, upd_launches), "launches": upd_launches}
    kernel_times = {k: {"launches": v[0], "total_ms": round(v[1], 3),
                        "share": round(v[1] / max(1e-9, sum(x[1] for x in prof.values())), 4)}
                    for k, v in sorted(prof.items(), key=lambda kv: -kv[1][1])}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tot_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": workload_name(m, n, rhs), "m": m, "n": n, "p": p, "nb": nb,
                   "path": args.path, "parallelism": "replicas" if world > 1 else "single",
                   "l2": "input 4.3 GB > L2, restored by a full device copy before every step"
                         if m == 32768 else "input restored by a full device copy before every step"},
        "roofline": roof,
        "gpu_launches": int(launches),
        "clocks": clocks,
        "correct": bool(ok),
        "correct_checks": content,
        "wall_s_timed": t_wall,
        "kernel_times": kernel_times,
    }

    if rank == 0 and not args.no_extras:
        line["e2e"] = e2e_leg(args, linac, synth, pristine, work, m, n, p, nb, stream, staging)
        line["paths"] = path_leg(args, linac, pristine, work, m, n, p, nb, stream, peaks)
        line["dense_4096"] = dense_4096_leg(args, linac, synth, dev, stream, peaks)
        line["dense_256"] = dense_256_leg(args, linac, synth, dev)
        if world == 1:
            line["cpu_baseline"] = cpu_leg(args, pristine, m, n, p)
        line["batched"] = batched_leg(args, linac, synth, dev, stream)
        line["shared_pattern"] = shared_leg(args, linac, synth, dev, stream)
        line["construction"] = construction_leg(args, linac, synth, dev)
        line["dense64"] = dense64_leg(args, linac, synth, dev)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def content_check(linac, pristine, work, m, p, trials=2):
    """The reduced matrix, beyond rank and pivots: its left block is exactly
    the identity ([A | B] reduces to [I | X], section 5.2), and A X = B mod p
    by Freivalds' test, A (X v) = B v for random v (a wrong X passes a trial
    with probability <= 1/p), with the products on linac_matmul."""
    import torch
    dev = work.device
    eye_ok = True
    for r0 in range(0, m, 4096):
        blk = work[r0:r0 + 4096, :m]
        nz = int(torch.count_nonzero(blk).item())
        diag = blk[torch.arange(blk.shape[0], device=dev), torch.arange(r0, r0 + blk.shape[0], device=dev)]
        eye_ok &= nz == blk.shape[0] and bool((diag == 1).all().item())
    rhs = work.shape[1] - m
    g = np.random.default_rng(2026)
    v = linac.to_device(g.integers(0, p, size=(rhs, trials), dtype=np.int64).astype(np.uint32), dev)
    xv = linac.linac_matmul(work[:, m:], v, p)
    lhs = linac.linac_matmul(pristine[:, :m], xv, p)
    bv = linac.linac_matmul(pristine[:, m:], v, p)
    torch.cuda.synchronize()
    return {"checked": True, "identity_block": bool(eye_ok), "freivalds": bool(torch.equal(lhs, bv)),
            "freivalds_trials": trials}


def e2e_leg(args, linac, synth, pristine, work, m, n, p, nb, stream, staging=None):
    """Through the public API with host buffers: linac_rref_host on the
    matrix in pinned host memory, which copies it to the device, reduces it
    and copies the RREF, rank and pivots back, every step (host wall clock
    around the call and the stream synchronisation).  The pinned input is
    restored from a pinned pristine copy before each step, outside the
    timed region."""
    import torch
    if staging is not None:
        host_src, host_io = staging
    else:
        host_src = torch.empty(pristine.shape, dtype=torch.int32, pin_memory=True)
        host_io = torch.empty_like(host_src, pin_memory=True)
    host_src.copy_(pristine)
    rank = torch.zeros(1, dtype=torch.int32, pin_memory=True)
    piv = torch.full((m,), -1, dtype=torch.int32, pin_memory=True)
    steps = max(1, min(args.steps, 3))
    times, parts = [], []
    for it in range(steps + 2):
        host_io.copy_(host_src)
        profiled = it == steps + 1   # one extra call with per-kernel events, for the split
        if profiled:
            linac.linac_profile_reset()
            linac.linac_profile_enable(True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        linac.linac_rref_host(host_io, p, rank=rank, pivots=piv, stream=stream)
        stream.synchronize()
        dt = time.perf_counter() - t0
        if profiled:
            linac.linac_profile_enable(False)
            parts.append(linac.linac_profile_read().get("host_copy", (0, 0.0))[1])
        elif it:   # the first call is the warm-up (it allocates the scratch)
            times.append(dt)
    rk = int(rank.item())
    ok = rk == m and np.array_equal(piv.numpy(), np.arange(m))
    # the reduced matrix that came back agrees with the device elimination
    ok = ok and torch.equal(host_io[:4096], work[:4096].cpu())
    macs = gj_work(m, n, np.arange(rk))
    nbytes = host_io.numel() * 4
    dt = statistics.median(times)
    return {"value": macs / dt, "unit": UNIT, "h2d_bytes_per_step": nbytes,
            "d2h_bytes_per_step": nbytes + 4 + 4 * m, "steps": steps, "warmup": 1,
            "ms_per_step": 1000 * dt, "correct": bool(ok),
            "api": "linac_rref_host (pinned host matrix; transfers by SM copies inside the call)",
            "parts_ms": {"copies_in_and_out": parts[0], "rest": 1000 * dt - parts[0]}}


def imma_peak():
    """Measured integer pipe rates of this device (probes/int_rates.cu): the
    s8 and u8 mma.sync multiply-adds per second (the tensor pipe's roofline),
    mad.wide.s32 per second, and the co-issue timings."""
    from paper_2605_25863_gb300 import probes
    return probes.measure_int_rates()


PATH_KERNEL = {"plain": "update_plain", "limb": "update_limb", "crt": "update_crt", "hybrid": "update_hybrid"}
# narrow multiply-adds per field multiply-add: u8 limb products (4 x 4) and
# s8 residue products (nine moduli)
PATH_NARROW = {"limb": 16, "crt": 9}


def time_paths(linac, pristine, work, m, n, p, nb, stream, paths, peaks, reps=2):
    """One timed elimination per update path (after reps - 1 warm-ups):
    field MAC/s of the whole elimination and of its update kernel, the
    latter against the path's roofline (plain: the multiply pipe's
    mad.wide.s32 rate; limb, crt: the measured tensor-pipe rate of their
    narrow products)."""
    import torch
    out = {}
    for path in paths:
        try:
            for it in range(reps):
                work.copy_(pristine)
                linac.linac_profile_reset()
                linac.linac_profile_enable(True)
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                r, piv = linac.linac_rref(work, p, nb=nb, path=path)
                e1.record(stream)
                torch.cuda.synchronize()
                linac.linac_profile_enable(False)
            prof = linac.linac_profile_read()
            ms = e0.elapsed_time(e1)
            rk = int(r.item())
            pv = piv.cpu().numpy()[:rk]
            macs = gj_work(m, n, pv)
            kl, kms = prof.get(PATH_KERNEL[path], (0, 0.0))
            umacs = update_work(m, n, pv, nb)
            rate = umacs / (kms / 1e3) if kms else 0.0
            entry = {"value": macs / (ms / 1000.0), "ms": ms, "rank": rk,
                     "update_kernel": PATH_KERNEL[path], "update_ms": kms, "update_field_macs_per_s": rate}
            if path == "plain":
                entry["roofline"] = {"bound": "alu", "peak": peaks["plain"], "frac": rate / peaks["plain"],
                                     "unit": "field MAC/s", "basis": peaks["plain_basis"]}
            elif path == "hybrid":
                both = peaks["plain"] + peaks["imma_s8"] / PATH_NARROW["crt"]
                entry["roofline"] = {"bound": "alu+tensor", "peak": both, "frac": rate / both, "unit": "field MAC/s",
                                     "basis": "multiply-pipe peak + measured s8 mma.sync rate / 9 (both pipes "
                                              "at full rate at once, which this chip does not sustain)",
                                     "coissue_ceiling": peaks["coissue"], "coissue_frac": rate / peaks["coissue"]}
            else:
                narrow = PATH_NARROW[path]
                pk = peaks["imma_u8"] if path == "limb" else peaks["imma_s8"]
                entry["roofline"] = {"bound": "tensor", "achieved": rate * narrow, "peak": pk,
                                     "frac": rate * narrow / pk, "unit": "narrow MAC/s",
                                     "basis": f"{narrow} {'u8' if path == 'limb' else 's8'} products per field "
                                              f"MAC x update rate / measured mma.sync m16n8k32 rate"}
            out[path] = entry
        except Exception as e:  # a path that is not available reports why
            out[path] = {"error": str(e)}
    return out


def path_leg(args, linac, pristine, work, m, n, p, nb, stream, peaks):
    """Plain CUDA-core update vs the multi-modular (CRT, nine s8 residue
    GEMMs) and u8-limb integer-tensor updates on the headline workload."""
    out = time_paths(linac, pristine, work, m, n, p, nb, stream, ("plain", "crt", "hybrid", "limb"), peaks)
    for path in ("crt", "hybrid", "limb"):
        if "value" in out.get("plain", {}) and "value" in out.get(path, {}):
            out[f"{path}_over_plain"] = out[path]["value"] / out["plain"]["value"]
    return out


def dense_4096_leg(args, linac, synth, dev, stream, peaks):
    """The 4096 x 4160 system with 64 rows replaced by combinations of others
    (rank 4032): each update path, elimination time and update-kernel
    roofline; checked: rank 4032 and pivots 0..4031."""
    import torch
    M, _ = synth.rank_deficient()
    m, n = M.shape
    pristine = linac.to_device(M, dev)
    work = linac.padded(m, n, dev)
    out = time_paths(linac, pristine, work, m, n, P31, 128, stream, ("plain", "crt", "hybrid", "limb"), peaks, reps=3)
    for path, e in out.items():
        if "rank" in e:
            e["correct"] = e["rank"] == 4032
    out["workload"] = "dense RREF 4096 x 4160, p = 2^31 - 1, 64 rows replaced by combinations (rank 4032)"
    return out


def dense_256_leg(args, linac, synth, dev):
    """The 256 x 256 system with one right-hand side: [A | b] reduced by
    linac_rref (one call captured in a CUDA graph, replayed), latency per
    system; and 1000 such systems in one linac_rref_batched call."""
    import torch
    S = synth.dense_system(n=256, k=1, p=P31, seed=1)
    pristine = linac.to_device(S, dev)
    A = linac.padded(256, 257, dev)
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        rank = torch.zeros(1, dtype=torch.int32, device=dev)
        piv = torch.full((256,), -1, dtype=torch.int32, device=dev)
        lib = linac.lib()
        ptr, mm, nn, ld = linac._matrix(A, "A")

        def call():
            A.copy_(pristine)
            code = lib.linac_rref(ptr, mm, nn, ld, P31, rank.data_ptr(), piv.data_ptr(), s.cuda_stream)
            if code != 0:
                raise linac.LinacError(code, "linac_rref")
        call()
    s.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        call()
    reps = 200
    with torch.cuda.stream(s):
        for _ in range(10):
            g.replay()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            g.replay()
        e1.record(s)
    s.synchronize()
    us = e0.elapsed_time(e1) * 1e3 / reps
    R = A.cpu().numpy().view(np.uint32)
    ok = int(rank.item()) == 256 and np.array_equal(R[:, :256], np.eye(256, dtype=np.uint32))
    # many copies through the batched entry point (independent systems)
    count = 1000
    systems = [synth.dense_system(n=256, k=1, p=P31, seed=1 + i) for i in range(count)]
    B = synth._pack(systems, P31, [256] * count, [0] * count)
    g2, gs, data, data0, (ranks, pv, poff, st) = _batched_graph(linac, B, dev, 0)
    ms = _time_graph(g2, data, data0, gs, 3)
    okb = bool((ranks[:count].cpu().numpy() == 256).all())
    W = gj_work(256, 257, np.arange(256))
    return {"workload": "dense RREF of [A | b], A 256 x 256 uniform, p = 2^31 - 1", "us_per_system": us,
            "systems_per_s": 1e6 / us, "field_macs_per_s": W / (us * 1e-6), "correct": bool(ok),
            "launch": "linac_rref captured in a CUDA graph, replayed (input restored inside the graph)",
            "batched": {"systems": count, "ms": ms, "systems_per_s": count / (ms / 1e3), "ranks_ok": okb,
                        "launch": "linac_rref_batched in a CUDA graph"}}


def cpu_leg(args, pristine, m, n, p):
    cores = os.cpu_count() or 1
    M = pristine.cpu().numpy().view(np.uint32)
    rate, dt, P, macs = cpu_oracle_sample(M, p, args.cpu_seconds, cores)
    return {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"first {P} pivot steps (of {m}) of the same {m} x {n} elimination "
                      f"({macs:.3e} field MACs, {dt:.1f} s, {cores} threads)"}


def _batched_graph(linac, B, dev, flags):
    """Device copies of a packed batch, one eager call (creates the library's
    scratch), then the call captured into a CUDA graph on a side stream (the
    default stream cannot be captured).  Returns (graph, stream, data,
    pristine data, outputs)."""
    import torch
    stream = torch.cuda.Stream()
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    data0 = t(B.data.view(np.int32))
    offs, mm, nn, ld, ns = t(B.offsets), t(B.m), t(B.n), t(B.ld), t(B.nA)
    max_m, max_n = int(B.m.max()), int(B.n.max())
    with torch.cuda.stream(stream):
        data = data0.clone()
        outs = linac.batched_outputs(mm, nn, ns)
        call = lambda: linac.linac_rref_batched_into(data, offs, mm, nn, ld, B.p, *outs, max_m=max_m,
                                                     max_n=max_n, nsearch=ns, flags=flags)
        call()
    stream.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=stream):
        call()
    return g, stream, data, data0, outs


def _time_graph(g, data, data0, stream, reps):
    """Median CUDA-event time of graph replays on restored inputs."""
    import torch
    times = []
    with torch.cuda.stream(stream):
        for it in range(reps + 1):
            data.copy_(data0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g.replay()
            e1.record(stream)
            stream.synchronize()
            if it:
                times.append(e0.elapsed_time(e1))
    return statistics.median(times)


def batched_widths(args, linac, p):
    """Panel widths per size bucket: --widths, else the autotuner (once per
    process, untimed)."""
    if args.widths:
        linac.linac_batched_set_panel_widths([int(w) for w in args.widths.split(",")])
        return linac.linac_batched_panel_widths()
    return linac.linac_batched_tune(p)


def batched_leg(args, linac, synth, dev, stream):
    """10,000 uneven systems [A | B] (n log-uniform in [32, 512], 4 RHS, 10 %
    rank-deficient): the whole linac_rref_batched call captured once into a
    CUDA graph, one graph replay per step."""
    B = synth.batched_uneven(count=args.batch_count)
    widths = batched_widths(args, linac, B.p)
    g, gs, data, data0, (ranks, piv, poff, st) = _batched_graph(linac, B, dev, 0)
    ms = _time_graph(g, data, data0, gs, 3)
    rk = ranks[:B.count].cpu().numpy()
    ok = bool((rk == B.nA - B.deficiency).all())
    macs = sum((int(B.m[s]) - 1) * (int(B.n[s]) * int(rk[s]) - int(rk[s]) * (int(rk[s]) + 1) // 2)
               for s in range(B.count))
    rate = macs / (ms / 1000.0)
    peak = batched_peak(dev, B.p)
    words = int((B.m.astype(np.int64) * B.ld.astype(np.int64)).sum())
    return {"systems": B.count, "systems_per_s": B.count / (ms / 1000.0), "ms": ms, "panel_widths": widths,
            "field_macs_per_s_approx": rate, "ranks_ok": ok, "launch": "cuda_graph",
            "roofline": {"bound": "alu", "achieved": rate, "peak": peak["value"], "frac": rate / peak["value"],
                         "unit": "field MAC/s", "basis": peak["basis"],
                         "dram_bytes_per_system": BATCHED_DRAM_PER_MATRIX_BYTE * words * 4 / B.count,
                         "one_read_and_write_bytes_per_system": 2 * words * 4 / B.count,
                         "dram_basis": "ncu DRAM bytes of the 2000-system capture per byte of its matrices "
                                       "(profiles/batched_uneven_bucket512.md) x this batch's matrix bytes"},
            "workload": "batched uneven [A|B], n log-uniform [32,512], 4 RHS, p = 2^31 - 19"}


def batched_peak(dev, p):
    """The multiply-pipe roofline of the batched kernel for prime p: one
    mad.wide.s32 per field MAC plus its folds (on the multiply pipe unless
    2^32 mod p is a single power of two, the batched kernel's rule)."""
    sms, mhz, src = device_sms_and_max_clock(dev)
    c32 = (1 << 32) % p
    single = c32 & (c32 - 1) == 0
    fold = fold_of(p)
    per = 1.0 if single else 1.0 + 2.0 / fold
    return {"value": sms * IMAD_WIDE_PER_SM_CLK * mhz * 1e6 / per,
            "basis": f"{sms} SMs x {IMAD_WIDE_PER_SM_CLK} mad.wide.s32/clk x {mhz:.0f} MHz / {per:.3f} per field MAC"
                     f" ({'shift fold' if single else f'fold every {fold} on the multiply pipe'})"}


def shared_leg(args, linac, synth, dev, stream):
    """4096 evaluations of a 384 x 400 block-banded polynomial template, with
    and without the shared pivot pattern (each call captured in a CUDA graph)."""
    B = synth.shared_pattern(count=4096)
    widths = batched_widths(args, linac, B.p)
    out = {}
    for name, flags in (("search", 0), ("shared_pattern", linac.LINAC_SHARED_PATTERN)):
        g, gs, data, data0, (ranks, piv, poff, st) = _batched_graph(linac, B, dev, flags)
        ms = _time_graph(g, data, data0, gs, 2)
        out[name] = {"systems_per_s": B.count / (ms / 1000.0), "ms": ms,
                     "ranks_ok": bool((ranks[:B.count].cpu().numpy() == 384).all())}
        del g
    out["speedup"] = out["search"]["ms"] / out["shared_pattern"]["ms"]
    out["panel_widths"] = widths
    out["launch"] = "cuda_graph"
    return out


def dense64_leg(args, linac, synth, dev):
    """uint64 residues (paper section 2.3: primes that do not fit 32 bits):
    RREF of [A | B], A m64 x m64 uniform (default 8192), 256 right-hand sides,
    p = 2^64 - 59 (the largest prime below 2^64).  The default input (577 MB)
    is larger than L2 and is restored from a pristine copy outside the timed
    region.  Checked: rank m64, pivots 0..m64-1, and A X = B on sampled
    entries in exact integers."""
    import torch
    p = 2**64 - 59
    m, rhs = args.m64, 256
    n = m + rhs
    M = synth.uniform64((m, n), p, synth.stream_key(64, "dense64"))
    pristine = linac.to_device64(M)
    A = pristine.clone()
    times = []
    for it in range(4):
        A.copy_(pristine)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        rank, piv = linac.linac_rref64(A, p)
        e1.record()
        torch.cuda.synchronize()
        if it:
            times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    R = linac.host64(A)
    ok = int(rank.item()) == m and np.array_equal(piv.cpu().numpy(), np.arange(m))
    for i, c in ((0, 0), (m // 2 + 1, 131), (m - 1, rhs - 1)):
        row = [int(v) for v in M[i, :m]]
        x = [int(v) for v in R[:m, m + c]]
        ok = ok and sum(a * b for a, b in zip(row, x)) % p == int(M[i, m + c])
    W = sum((m - 1) * (n - t - 1) for t in range(m))
    return {"workload": f"RREF {m} x {n} ({rhs} RHS), p = 2^64 - 59, uint64", "ms": ms,
            "value": W / (ms / 1e3), "unit": "field MAC/s", "correct": bool(ok), "timed_runs": len(times)}


def construction_leg(args, linac, synth, dev):
    """Systems built on the device (paper section 3.3).

    (a) linac_load_matrix at the paper's largest construction size, n = 20000
        points x 20000 monomials of degree 8 over 64 basis variables (the
        paper reports 2.6 s on an RTX 4070 Laptop GPU for n = 2 x 10^4).
    (b) the shared-pattern workload end to end: monomial values of 4096 points
        (load_matrix), the 384 x 400 template's coefficients applied to them
        (linac_matmul), and the shared-pattern RREF of the 4096 systems, all
        captured in one CUDA graph."""
    import torch
    out = {}
    p = P31
    # (a)
    n, nb, d = 20000, 64, 8
    bases = torch.from_numpy(synth.uniform((n, nb), p, synth.stream_key(20, "lm_bases")).view(np.int32)).to(dev)
    g = np.random.default_rng(20)
    lind = torch.from_numpy(g.integers(0, nb, size=(n, d), dtype=np.int64).astype(np.int32)).to(dev)
    A = linac.padded(n, n, dev)
    times = []
    for it in range(4):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record()
        linac.linac_load_matrix(bases, lind, p, out=A)
        e1.record()
        torch.cuda.synchronize()
        if it:
            times.append(e0.elapsed_time(e1))
    ms = statistics.median(times)
    out["load_matrix"] = {"rows": n, "cols": n, "degree": d, "basis": nb, "ms": ms,
                          "entries_per_s": n * n / (ms / 1e3), "modmul_per_s": n * n * d / (ms / 1e3),
                          "write_gbs": n * n * 4 / (ms / 1e3) / 1e9, "paper_context": "2.6 s, RTX 4070 Laptop, n = 2e4"}
    del A
    # (b)
    mask, coefs, mons = synth.shared_pattern_template()
    count = 4096
    rows, cols = mask.shape
    pts = synth.uniform((count, 2), p, synth.stream_key(4, "sp_points"))
    Cd = np.zeros((len(mons), rows * cols), dtype=np.uint32)
    Cd[:, np.flatnonzero(mask.ravel())] = coefs.T
    deg = max(a + b for a, b in mons)
    li = np.zeros((len(mons), deg), dtype=np.int32)
    for u, (a, b) in enumerate(mons):
        idx = [1] * a + [2] * b
        li[u, :len(idx)] = idx
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    bases2 = t(np.concatenate([np.ones((count, 1), dtype=np.uint32), pts], axis=1).view(np.int32))
    lind2 = t(li)
    Cdev = t(Cd.view(np.int32))
    V = linac.padded(count, len(mons), dev)
    data2 = linac.padded(count, rows * cols, dev)
    flat = data2.view(-1)
    offs = torch.arange(count, dtype=torch.int64, device=dev) * (rows * cols)
    mm = torch.full((count,), rows, dtype=torch.int32, device=dev)
    nn = torch.full((count,), cols, dtype=torch.int32, device=dev)
    ns = torch.full((count,), cols - 16, dtype=torch.int32, device=dev)
    s2 = torch.cuda.Stream()
    with torch.cuda.stream(s2):
        outs = linac.batched_outputs(mm, nn, ns)

        def build_and_reduce():
            linac.linac_load_matrix(bases2, lind2, p, out=V, stream=s2)
            linac.linac_matmul(V, Cdev, p, out=data2, stream=s2)
            linac.linac_rref_batched_into(flat, offs, mm, nn, nn, p, *outs, max_m=rows, max_n=cols, nsearch=ns,
                                          flags=linac.LINAC_SHARED_PATTERN, stream=s2)
        build_and_reduce()
    s2.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=s2):
        build_and_reduce()
    times, tb = [], []
    with torch.cuda.stream(s2):
        for it in range(4):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e2 = torch.cuda.Event(enable_timing=True)
            e0.record(s2)
            graph.replay()
            e1.record(s2)
            # construction alone, eagerly, for its share
            linac.linac_load_matrix(bases2, lind2, p, out=V, stream=s2)
            linac.linac_matmul(V, Cdev, p, out=data2, stream=s2)
            e2.record(s2)
            s2.synchronize()
            if it:
                times.append(e0.elapsed_time(e1))
                tb.append(e1.elapsed_time(e2))
    ms2, msb = statistics.median(times), statistics.median(tb)
    ranks = outs[0][:count].cpu().numpy()
    out["template_pipeline"] = {
        "systems": count, "ms": ms2, "systems_per_s": count / (ms2 / 1e3), "construction_ms": msb,
        "construction_share": msb / ms2, "ranks_ok": bool((ranks == rows).all()), "launch": "cuda_graph",
        "workload": "4096 evaluations of a 384 x 400 block-banded template of bivariate polynomials "
                    "(degree <= 4, 16 RHS), built on the device and reduced with the shared pattern"}
    return out


def main():
    args = parse()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps; the number is not a valid bench value", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.measure_peaks:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        from paper_2605_25863_gb300 import probes
        r = probes.measure_int_rates()
        r["imad_per_sm_per_clk"] = r["imad_wide_per_s"] / (r["sm_count"] * r["sm_clock_khz"] * 1e3)
        r["device"] = torch.cuda.get_device_name(0)
        print(json.dumps(r))
        return 0
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
