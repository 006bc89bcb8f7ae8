#!/usr/bin/env python
"""Throughput of the CKKS homomorphic linear transformation on one GB300.

Workload (one "step" = one LT, the whole hot path): N = 2^16 ring, one
ciphertext at the top level (24 Q limbs: 55b + 23x40b), 4 special 60-bit
primes, dnum 6 (alpha 4, beta 6), a 2^15 x 2^15 matrix with 256 consecutive
nonzero diagonals, evaluated by triple-hoisted BSGS (Algorithm 2) with the
library's split.  Keys, diagonals and the ciphertext are uniform residues
drawn on the device (the work does not depend on the values); the keys and
the diagonals (6+ GB) stay resident and are far larger than L2, so no flush
is needed between steps.

Prints one JSON line (rank 0):
  value      LT/s over all ranks with inputs resident in HBM (device events)
  e2e        LT/s through the C ABI with the ciphertext copied from pinned
             host memory and the result copied back inside each step
  roofline   the dominant kernel's algorithmic bytes / its live event-timed
             duration, against the measured HBM copy bandwidth
  alu_roofline  per kernel class, its counted multiply-accumulates and NTT
             butterflies at the rates of a live register-only probe of the
             same arithmetic, over its measured time
  cpu_baseline  the CPU oracle timed on this host on one LT of the workload

--impl reference times the CPU oracle alone (the reference arm).
Multi-GPU: under torchrun each rank runs its own replica of the workload
(independent LTs; no collective on the data path): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "encrypted LT/s and ms per LT at N=2^16 (bit-exact), % of HBM roofline; p50/p99"
PARAMS = "n16"
D = 256
LEVEL = 24
SEED = 1


def parse():
    ap = argparse.ArgumentParser(description="Throughput of the CKKS linear transformation; prints one JSON line.")
    ap.add_argument("--gpus", type=int, default=1, help="GPUs (one rank each under torchrun; replicas, weak scaling)")
    ap.add_argument("--steps", type=int, default=200, help="timed steps")
    ap.add_argument("--warmup", type=int, default=5, help="untimed warm-up steps (at least 3 are run)")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"],
                    help="reference: the CPU oracle on this host's cores")
    ap.add_argument("--algo", default="th", choices=["th", "dh", "bsgs", "diag"],
                    help="TH-BSGS (Alg. 2), DH-BSGS (Alg. 1), BSGS (Eq. 5) or the diagonal method")
    ap.add_argument("--split", default="", help="e.g. 4,8,8 (default: the library's choice)")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="skip timing the CPU oracle")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end run with host copies")
    ap.add_argument("--diags", type=int, default=256, help="number of diagonals (256 = the benchmark workload)")
    ap.add_argument("--level", type=int, default=24, help="ciphertext level (24 = the benchmark workload)")
    ap.add_argument("--workload", default="single",
                    choices=["single", "batched", "uneven", "serving", "paper-a", "paper-b", "cts", "stc", "steps"],
                    help="single: one LT per step (the headline); batched: 64 ciphertexts at levels "
                         "{8,16,24} and one shared 256-diagonal matrix per step; uneven: 128 LTs over 20 "
                         "(diagonals, stride) shapes per step; serving: Poisson arrivals of LT requests "
                         "through the continuous-batching server; paper-a / paper-b: the paper's Set-A / "
                         "Set-B dense LTs; cts / stc: CoeffToSlot / SlotToCoeff chains at N=2^16; steps: "
                         "the key-switching steps one at a time")
    ap.add_argument("--duration", type=float, default=60.0, help="serving: seconds of arrivals")
    ap.add_argument("--rate", type=float, default=200.0, help="serving: requests per second")
    return ap.parse_args()


# ----------------------------------------------------------------------------- distributed
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None
        if self.world > 1:
            import torch
            import torch.distributed as dist
            backend = "nccl" if torch.cuda.is_available() else "gloo"
            if backend == "nccl":
                torch.cuda.set_device(self.local)
            dist.init_process_group(backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if torch.cuda.is_available() else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


def shard(total: int, world: int, rank: int) -> range:
    """Units of work of one rank when `total` independent units are split."""
    per, extra = divmod(total, world)
    start = rank * per + min(rank, extra)
    return range(start, start + per + (1 if rank < extra else 0))


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=2)
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
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- byte model
def algorithmic_bytes(cls: str, split, level: int, k: int, beta: int, n_diag: int, N: int,
                      outer_rotated: int | None = None) -> tuple:
    """(bytes, launches) per LT of one kernel class in the TH/DH schedule: the
    compulsory words the class must read, 8 bytes each -- the diagonals and
    the switching keys it streams (the per-LT byte formula's D (l+k) and
    K 2 beta (l+k) terms).  Intermediates (digits, baby pairs, partial sums)
    are not algorithmic bytes; the ncu traffic shows what they add.
    outer_rotated: how many outer amounts are nonzero (n3 - 1 for consecutive
    offsets from 0; up to n3 with a base)."""
    n1, n2, n3 = split
    n_out = n3 - 1 if outer_rotated is None else outer_rotated
    ext = level + k
    limb = 8 * N
    if cls == "diag_mac":
        limbs = n_diag * ext                                   # diagonals
        limbs += (n2 - 1) * 2 * beta * ext                      # middle-layer keys
        return limbs * limb, 1
    if cls == "ks_inner":
        return ((n1 - 1) + n_out) * 2 * beta * ext * limb, (n1 - 1) + n_out   # inner- and outer-layer keys
    return None, None


def algorithmic_bytes_for(algo: str, cls: str, split, level: int, k: int, beta: int, n_diag: int, N: int,
                          dh_fused: bool = False) -> tuple:
    """algorithmic_bytes for any algorithm: DH(n1, n2) runs as TH(n1, 1, n2), or
    as TH(1, n1, n2) with its baby steps fused into K6 (dh_fused), and the
    diagonal method as TH(1, D, 1); BSGS multiplies over Q only (K6 without the
    P limbs or a middle layer) and switches keys once per rotation."""
    if algo == "dh":
        th = (1, split[0], split[1]) if dh_fused else (split[0], 1, split[1])
        return algorithmic_bytes(cls, th, level, k, beta, n_diag, N)
    if algo == "diag":
        return algorithmic_bytes(cls, (1, n_diag, 1), level, k, beta, n_diag, N)
    if algo == "bsgs":
        n1, n2 = split[0], split[1]
        limb, ext = 8 * N, level + k
        if cls == "diag_mac":
            return limb * n_diag * level, 1
        if cls == "ks_inner":
            rots = (n1 - 1) + (n2 - 1)
            return rots * limb * 2 * beta * ext, rots
        return None, None
    return algorithmic_bytes(cls, split, level, k, beta, n_diag, N)


def alu_roofline(binding, device: int, shares: dict, work: dict, dominant: str, dom_time: tuple,
                 dom_work: tuple) -> dict:
    """Integer-ALU roofline of every kernel class that does counted work:
    frac = (its 128-bit multiply-accumulates at the probed MAC rate + its NTT
    butterflies at the probed butterfly rate) / its measured device time.
    The rates come from the library's register-only probe of the same
    arithmetic, run here, after the timed region.  The dominant kernel uses
    its timed-region launches, the others the warm-up launches."""
    mac_rate, bfly_rate = binding.probe_int_rates(device)
    kernels = {}
    for c, (ms, n) in shares.items():
        macs, bfly = work[c]
        if c == dominant and dom_time[1]:
            (ms, n), (macs, bfly) = dom_time, dom_work
        if not n or not ms or (macs == 0 and bfly == 0):
            continue
        ideal_s = macs / mac_rate + bfly / bfly_rate
        kernels[c] = {"macs_per_launch": int(macs / n), "butterflies_per_launch": int(bfly / n),
                      "ms_per_launch": round(ms / n, 4), "frac": round(ideal_s / (ms / 1e3), 4)}
    return {"bound": "alu", "unit": "fraction of the probed integer rate",
            "peak": {"macs_per_s": round(mac_rate, -6), "butterflies_per_s": round(bfly_rate, -6)},
            "peak_source": "register-only probe of the library's own 128-bit multiply-accumulate and growing "
                           "NTT butterfly, run live on this GPU (ckks_probe_int_rates)",
            "kernels": kernels}


def lt_compulsory_bytes(split, level: int, k: int, beta: int, n_diag: int, N: int) -> int:
    """Compulsory bytes of one LT: diagonals, distinct keys, ciphertext in and out."""
    n1, n2, n3 = split
    keys = (n1 - 1) + (n2 - 1) + (n3 - 1)
    ext = level + k
    return 8 * N * (n_diag * ext + keys * 2 * beta * ext + 2 * level + 2 * (level - 1))


def source_digest(paths) -> str:
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_peaks() -> dict:
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def ncu_traffic(cls: str):
    """dram bytes per launch of `cls` from the committed ncu summary, or None
    when the kernel's sources changed since it was captured."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f).get(cls)
    except (OSError, ValueError):
        return None
    if not rec:
        return None
    if rec.get("source_digest") != source_digest(rec.get("sources", [])):
        return None
    return rec.get("dram_bytes_per_launch")


# ----------------------------------------------------------------------------- CPU oracle
def oracle_problem_from_device(ps, g, split, keys_t, diags_t, ct_t):
    import numpy as np
    from paper_2605_17222_gb300 import binding
    keys = {r: binding.to_host(t).reshape(g.beta_max, 2, ps.L + ps.k, ps.n) for r, t in keys_t.items()}
    diags = binding.to_host(diags_t)
    ct = binding.to_host(ct_t)
    return keys, np.ascontiguousarray(diags), (np.ascontiguousarray(ct[0]), np.ascontiguousarray(ct[1]))


def time_oracle(ps, algo, split, keys, diags, ct, budget_s: float, max_steps: int, warmup: int = 0,
                warmup_budget_s: float = 0.0):
    """Times full oracle LTs until `max_steps` or `budget_s` (at least one),
    after up to `warmup` untimed LTs that stop early once `warmup_budget_s` is
    spent.  Returns (times, warm-up LTs run, the last LT's output [2][level-1][N])."""
    from oracle import lt as olt
    from oracle.ckks import Ctx
    octx = Ctx(ps)
    w_start, warm = time.perf_counter(), 0
    while warm < warmup and (warm == 0 or time.perf_counter() - w_start < warmup_budget_s):
        olt.run(octx, algo, ct, diags, keys, split if algo != "diag" else None)
        warm += 1
    times, out = [], None
    t_start = time.perf_counter()
    while len(times) < max(1, max_steps):
        t0 = time.perf_counter()
        out, _ = olt.run(octx, algo, ct, diags, keys, split if algo != "diag" else None)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start + times[-1] > budget_s:
            break
    return times, warm, out


def parity_with_oracle(got, want) -> dict:
    """Word-for-word comparison of the GPU's output residues with the oracle's."""
    import numpy as np
    want = np.stack(want)
    if got.shape != want.shape:
        return {"parity": "mismatch", "detail": f"shape {list(got.shape)} vs {list(want.shape)}"}
    diff = np.argwhere(got != want)
    if diff.size == 0:
        return {"parity": "bit-exact", "words": int(got.size)}
    i = tuple(int(v) for v in diff[0])
    return {"parity": "mismatch", "words": int(got.size), "differing": int(len(diff)), "first_index": list(i),
            "gpu": int(got[i]), "oracle": int(want[i])}


def cores_used() -> int:
    n = os.environ.get("OMP_NUM_THREADS")
    return int(n) if n else (len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else os.cpu_count())


# ----------------------------------------------------------------------------- end to end
def e2e_pipelined(g, compute, hin, n_out: int, level_in: int, level_out: int, steps: int, dist) -> float:
    """Milliseconds for `steps` end-to-end steps through the C ABI: every step
    copies its input from pinned host memory to the device and its result back
    to pinned host memory.  Device ciphertexts are double-buffered: the upload
    of step i+1's input and the download of step i's result run on a copy
    stream while step i+1 / i computes, so the copies hide behind the LTs.
    `compute(d_in, d_out, stream)` queues one step on `stream`."""
    import numpy as np
    import torch
    sc, sx = torch.cuda.Stream(), torch.cuda.Stream()
    d_in = [g.ct_create(level_in) for _ in range(2)]
    d_out = [g.ct_create(level_out) for _ in range(2)]
    h_out = [torch.empty(n_out, dtype=torch.int64, pin_memory=True) for _ in range(2)]
    hout = [h.numpy().view(np.uint64) for h in h_out]

    def run(n):
        ev = [[torch.cuda.Event() for _ in range(2)] for _ in range(3)]
        in_ready, done, copied = ev
        sx.wait_stream(sc)
        g.h2d_async(d_in[0], hin, stream=sx)
        in_ready[0].record(sx)
        for i in range(n):
            b = i % 2
            sc.wait_event(in_ready[b])
            if i >= 2:
                sc.wait_event(copied[b])  # d_out[b]'s previous result is on the host
            compute(d_in[b], d_out[b], sc)
            done[b].record(sc)
            if i + 1 < n:
                nb = (i + 1) % 2
                if i >= 1:
                    sx.wait_event(done[nb])  # d_in[nb] was consumed by step i-1
                g.h2d_async(d_in[nb], hin, stream=sx)
                in_ready[nb].record(sx)
            sx.wait_event(done[b])
            g.d2h_async(d_out[b], hout[b], stream=sx)
            copied[b].record(sx)
        sc.wait_stream(sx)

    run(2)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    torch.cuda.synchronize()
    e0.record(sc)
    run(steps)
    e1.record(sc)
    torch.cuda.synchronize()
    dist.barrier()
    return dist.max(e0.elapsed_time(e1))


# ----------------------------------------------------------------------------- main arms
def make_inputs(g, ps, splits, algo, device):
    import torch
    from paper_2605_17222_gb300 import synth
    N = ps.n
    rots = sorted({r for sp in splits for r in g.required_rotations(algo, sp if algo != "diag" else None, D, 1)})
    keys_t = {}
    for r in rots:
        t = synth.uniform_mod_device(SEED, f"key/{r}", ps.moduli, N, count=2 * g.beta_max, device=device)
        g.upload_rotation_key_device(r, t)
        keys_t[r] = t
    top = list(ps.q) + list(ps.p)
    diags_t = synth.uniform_mod_device(SEED, "diag", top, N, count=D, device=device)
    f = g.upload_diagonals_device(diags_t, stride=1, level=ps.L)
    ct_t = synth.uniform_mod_device(SEED, "ct", list(ps.q[:LEVEL]), N, count=2, device=device)
    torch.cuda.synchronize()
    return rots, keys_t, diags_t, f, ct_t


def run_ours(args, dist: Dist):
    global D, LEVEL
    D, LEVEL = args.diags, args.level
    import numpy as np
    import torch
    from paper_2605_17222_gb300 import binding, synth
    device = f"cuda:{dist.local}"
    torch.cuda.set_device(dist.local)
    ps = synth.param_set(PARAMS)
    g = binding.Context.from_params(ps, device=dist.local)
    algo = args.algo
    tuned_ms = None
    if args.split:
        split = tuple(int(x) for x in args.split.split(","))
        split3 = tuple(split) + (1,) * (3 - len(split))
        rots, keys_t, diags_t, f, ct_t = make_inputs(g, ps, [split3], algo, device)
        ct = g.ct_wrap(ct_t, LEVEL)
    else:
        # the library's autotuner: keys for the cost model's best candidates, each timed once here
        cands = [g.choose_split(algo, LEVEL, D)] if algo == "diag" else g.candidate_splits(algo, LEVEL, D, 6)
        rots, keys_t, diags_t, f, ct_t = make_inputs(g, ps, cands, algo, device)
        ct = g.ct_wrap(ct_t, LEVEL)
        if algo == "diag":
            split3 = (1, D, 1)
        else:
            split3, tuned_ms = g.autotune(algo, ct, f, len(cands))
    out = g.ct_empty(LEVEL - 1)
    keep_host_copy = not args.no_cpu_baseline and dist.rank == 0 and dist.world == 1
    if not keep_host_copy:  # the library holds its own copies
        keys_t, diags_t = None, None
        torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    beta = g.beta(LEVEL)

    # warm-up; the warm-up steps after the first also rank the kernel classes by
    # device time (the first LT of a process loads each kernel's module, and
    # that host time would land between a class's events)
    g.lt_eval(ct, f, algo, split3, out=out)
    torch.cuda.synchronize()
    for c in binding.KERNEL_CLASSES:
        binding.profile_enable(c, True)
    binding.profile_reset()
    for _ in range(max(3, args.warmup) - 1):
        g.lt_eval(ct, f, algo, split3, out=out)
    torch.cuda.synchronize()
    shares = {c: binding.profile_read(c) for c in binding.KERNEL_CLASSES}
    work = {c: binding.profile_work(c) for c in binding.KERNEL_CLASSES}
    for c in binding.KERNEL_CLASSES:
        binding.profile_enable(c, False)
    tot = sum(v[0] for v in shares.values()) or 1.0
    dominant = max(shares, key=lambda c: shares[c][0])
    if dominant not in ("diag_mac", "ks_inner"):
        # the roofline below is defined for the HBM-streaming kernels
        dominant = max(("diag_mac", "ks_inner"), key=lambda c: shares[c][0])

    clocks = ClockSampler(dist.local)
    clocks.start()
    time.sleep(0.3)
    # ---------------------------------------------------------------- timed: device-resident inputs
    binding.profile_reset()
    binding.profile_enable(dominant, True)
    l0 = binding.kernel_launches()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    dist.barrier()
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(args.steps):
        if i == 0:  # marks one LT's launches for profilers (ncu --nvtx --nvtx-include "timed_lt/")
            torch.cuda.nvtx.range_push("timed_lt")
        g.lt_eval(ct, f, algo, split3, out=out)
        if i == 0:
            torch.cuda.nvtx.range_pop()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    launches = binding.kernel_launches() - l0
    dom_ms, dom_n = binding.profile_read(dominant)
    dom_work = binding.profile_work(dominant)
    binding.profile_enable(dominant, False)
    step_ms = [evs[i].elapsed_time(evs[i + 1]) for i in range(args.steps)]
    total_ms = evs[0].elapsed_time(evs[-1])
    # ---------------------------------------------------------------- timed: end to end through the C ABI
    e2e = None
    if not args.no_e2e:
        n_in, n_out = 2 * LEVEL * ps.n, 2 * (LEVEL - 1) * ps.n
        h_in = torch.empty(n_in, dtype=torch.int64, pin_memory=True)
        h_in.copy_(ct_t.reshape(-1).cpu())
        hin = h_in.numpy().view(np.uint64)
        e2e_steps = max(2, args.steps // 2)
        e2e_ms = e2e_pipelined(g, lambda di, do, st: g.lt_eval(di, f, algo, split3, out=do, stream=st), hin, n_out,
                               LEVEL, LEVEL - 1, e2e_steps, dist)
        e2e = {"value": round(dist.world * e2e_steps / (e2e_ms / 1e3), 3), "unit": "LT/s",
               "h2d_bytes_per_step": n_in * 8, "d2h_bytes_per_step": n_out * 8,
               "ms_per_step": round(e2e_ms / e2e_steps, 4),
               "copies": "double-buffered on a copy stream, overlapping the previous/next step's LT"}
    clk = clocks.stop()

    max_ms = dist.max(total_ms)
    value = dist.world * args.steps / (max_ms / 1e3)
    srt = sorted(step_ms)
    p50 = srt[len(srt) // 2]
    p99 = srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))]
    # ---------------------------------------------------------------- roofline of the dominant kernel
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs")
    peak_src = "measured" if peak else "fallback"
    peak = peak or 6800.0
    dh_sched = g.dh_schedule(f, LEVEL, split3) if algo == "dh" else None
    tile = g.tuned_tile(algo, f, LEVEL) if tuned_ms is not None else None
    b_lt, n_lt = algorithmic_bytes_for(algo, dominant, split3, LEVEL, ps.k, beta, D, ps.n, dh_sched == "fused")
    roof = None
    if b_lt and dom_n:
        per_launch = b_lt / n_lt
        avg_s = dom_ms / dom_n / 1e3
        ach = per_launch / avg_s / 1e9
        roof = {"kernel": dominant, "bound": "hbm", "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "traffic": ncu_traffic(dominant),
                "algorithmic_bytes_per_launch": int(per_launch), "avg_launch_ms": round(avg_s * 1e3, 4),
                "peak_source": f"{peak_src} HBM copy bandwidth"}
    lt_bytes = lt_compulsory_bytes(split3, LEVEL, ps.k, beta, D, ps.n) if algo in ("th", "dh") else None
    result = {
        "metric": METRIC, "value": round(value, 3), "unit": "LT/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(max_ms / args.steps, 4),
        "p50_ms": round(p50, 4), "p99_ms": round(p99, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (uniform residues drawn on the device; seeded)",
        "config": {"workload": f"single LT: N=2^16, level {LEVEL} (Q = 55b + 23x40b), 4x60b special primes, "
                               f"dnum 6, {D} consecutive diagonals, one ciphertext at the top level",
                   "algo": algo, "split": list(split3), "parallelism": f"replicas x{dist.world}",
                   **({"dh_schedule": dh_sched} if dh_sched else {}),
                   **({"k6_tile": {"outer_per_cta": tile[0] or "default", "positions_per_cta": tile[1] or "default"}}
                      if tile else {}),
                   "split_choice": ("given" if args.split else "the diagonal method has one split" if tuned_ms is None
                                    else f"autotuned over the cost model's best candidates ({tuned_ms:.3f} ms "
                                         f"when measured)"),
                   "l2": "inputs larger than L2 (keys + diagonals resident, > 6 GB per step); no flush"},
        "hbm_roofline_lt": (None if lt_bytes is None else {
            "compulsory_bytes": lt_bytes, "achieved_gbs": round(lt_bytes / (max_ms / args.steps / 1e3) / 1e9, 1),
            "frac": round(lt_bytes / (max_ms / args.steps / 1e3) / 1e9 / peak, 4)}),
        "roofline": roof,
        "alu_roofline": alu_roofline(binding, dist.local, shares, work, dominant, (dom_ms, dom_n), dom_work),
        "kernel_shares": {c: round(v[0] / tot, 4) for c, v in shares.items()},
        "e2e": e2e,
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    # ---------------------------------------------------------------- CPU oracle baseline
    if not args.no_cpu_baseline and dist.rank == 0 and dist.world == 1:
        keys, diags, cth = oracle_problem_from_device(ps, g, split3, keys_t, diags_t, ct_t)
        times, _, want = time_oracle(ps, algo, split3, keys, diags, cth, budget_s=30.0, max_steps=1)
        # the timed split's GPU output (every timed LT wrote the same residues into `out`)
        # against the oracle's on the same inputs
        result["parity"] = dict(parity_with_oracle(out.numpy(), want),
                                against=f"CPU oracle, same inputs and split {list(split3)}")
        result["cpu_baseline"] = {
            "value": round(len(times) / sum(times), 5), "unit": "LT/s", "cores": cores_used(), "kind": "oracle",
            "sample": f"{len(times)} full LT(s) of this workload ({algo}, split {list(split3)}) on the same "
                      f"uniform inputs copied to the host; {sum(times):.1f} s"}
    return result


def run_batched(args, dist: Dist):
    """64 ciphertexts at N=2^16 with levels drawn from {8, 16, 24} (seed 2), all
    multiplied by one shared 256-diagonal matrix: one recorded lt_eval_batch per
    step, against the same 64 LTs as sequential lt_eval calls."""
    import numpy as np
    import torch
    from paper_2605_17222_gb300 import binding, synth
    device = f"cuda:{dist.local}"
    torch.cuda.set_device(dist.local)
    ps = synth.param_set(PARAMS)
    g = binding.Context.from_params(ps, device=dist.local)
    n_ct = 64
    levels = [int(v) for v in np.random.default_rng(2).choice([8, 16, 24], n_ct)]
    lvs = sorted(set(levels))
    # keys for the cost model's best candidates at every level; the library's
    # autotuners then pick one split per level for single LTs and one for the batch
    cands = {lv: g.candidate_splits("th", lv, D, 6) for lv in lvs}
    rots = sorted({r for lv in lvs for sp in cands[lv] for r in g.required_rotations("th", sp, D, 1)})
    for r in rots:
        t = synth.uniform_mod_device(SEED, f"key/{r}", ps.moduli, ps.n, count=2 * g.beta_max, device=device)
        g.upload_rotation_key_device(r, t)
        del t
    top = list(ps.q) + list(ps.p)
    dt = synth.uniform_mod_device(SEED, "diag", top, ps.n, count=D, device=device)
    f = g.upload_diagonals_device(dt, stride=1, level=ps.L)
    del dt
    cts = [g.ct_wrap(synth.uniform_mod_device(SEED + 1 + n, f"ct/{n}", list(ps.q[:lv]), ps.n, count=2,
                                              device=device), lv) for n, lv in enumerate(levels)]
    outs = [g.ct_empty(lv - 1) for lv in levels]
    single = {lv: g.autotune("th", next(c for c in cts if c.level == lv), f, len(cands[lv]))[0] for lv in lvs}
    splits = {lv: g.autotune_batch("th", [c for c in cts if c.level == lv], f, len(cands[lv]))[0] for lv in lvs}
    sp_list = [splits[lv] for lv in levels]
    seq_list = [single[lv] for lv in levels]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dist.barrier()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        return dist.max(e0.elapsed_time(e1))

    def sequential():
        for c, o, sp in zip(cts, outs, seq_list):
            g.lt_eval(c, f, "th", sp, out=o)

    rec = g.lt_graph(cts, [f] * n_ct, algos=["th"] * n_ct, splits=sp_list, outs=outs)
    steps = max(1, args.steps)
    clocks = ClockSampler(dist.local)
    clocks.start()
    ms_graph = timed(lambda: rec.launch(), steps)
    ms_batch = timed(lambda: g.lt_eval_batch(cts, [f] * n_ct, algos=["th"] * n_ct, splits=sp_list, outs=outs),
                     steps)
    ms_seq = timed(sequential, steps)
    clk = clocks.stop()
    rec.close()
    # integer-ALU roofline of one batch step, untimed: profiled lt_eval_batch (a graph replay makes no
    # host launches to bracket); the lanes' kernels overlap, so a launch's event time includes time it
    # shares with other lanes and the fractions are lower bounds
    for c in binding.KERNEL_CLASSES:
        binding.profile_enable(c, True)
    binding.profile_reset()
    g.lt_eval_batch(cts, [f] * n_ct, algos=["th"] * n_ct, splits=sp_list, outs=outs)
    torch.cuda.synchronize()
    shares_b = {c: binding.profile_read(c) for c in binding.KERNEL_CLASSES}
    work_b = {c: binding.profile_work(c) for c in binding.KERNEL_CLASSES}
    for c in binding.KERNEL_CLASSES:
        binding.profile_enable(c, False)
    alu = alu_roofline(binding, dist.local, shares_b, work_b, "", (0.0, 0), (0.0, 0.0))
    # compulsory bytes of one step: diagonals and keys once per level used, every ciphertext in and out
    limb = 8 * ps.n
    comp = 0
    for lv, sp in splits.items():
        beta = g.beta(lv)
        ext = lv + ps.k
        keys = (sp[0] - 1) + (sp[1] - 1) + (sp[2] - 1)
        comp += limb * (D * ext + keys * 2 * beta * ext)
    comp += sum(limb * (2 * lv + 2 * (lv - 1)) for lv in levels)
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    val = dist.world * n_ct * steps / (ms_graph / 1e3)
    return {
        "metric": METRIC, "value": round(val, 3), "unit": "LT/s", "n_gpus": dist.world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": round(ms_graph / steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (uniform residues drawn on the device; seeded)",
        "config": {"workload": f"batched: {n_ct} ciphertexts, N=2^16, levels from {{8,16,24}} (seed 2), one shared "
                               f"{D}-diagonal matrix; one recorded lt_eval_batch per step",
                   "levels": {str(lv): levels.count(lv) for lv in sorted(set(levels))},
                   "splits": {str(lv): list(sp) for lv, sp in splits.items()},
                   "split_choice": "per level: lt_autotune_batch over the level's ciphertexts (batch) and "
                                   "lt_autotune on one of them (sequential), over the cost model's 6 best",
                   "sequential_splits": {str(lv): list(sp) for lv, sp in single.items()},
                   "l2": "inputs larger than L2; no flush"},
        "batched_graph_lt_per_s": round(val, 3),
        "batched_call_lt_per_s": round(dist.world * n_ct * steps / (ms_batch / 1e3), 3),
        "sequential_lt_per_s": round(dist.world * n_ct * steps / (ms_seq / 1e3), 3),
        "speedup_vs_sequential": round(ms_seq / ms_graph, 3),
        "hbm_roofline_batch": {"compulsory_bytes": comp,
                               "frac": round(comp / (ms_graph / steps / 1e3) / 1e9 / peak, 4)},
        "alu_roofline_batch": alu,
        "clocks": clk,
    }


def run_uneven(args, dist: Dist):
    """128 LTs per step at N = 2^16: diagonal counts from {16, 64, 256, 1024},
    offsets consecutive or strided by 2^k (k = 1..4, D 2^k <= N/2), levels
    uniform in 6..24 (seed 3); one matrix per distinct (D, stride) shape shared
    by the LTs of that shape; one split per (shape, level), picked by the
    measuring autotuner among the cost model's best candidates; one recorded
    lt_eval_batch per step against 128 sequential lt_eval calls."""
    import numpy as np
    import torch
    from paper_2605_17222_gb300 import binding, synth
    device = f"cuda:{dist.local}"
    torch.cuda.set_device(dist.local)
    ps = synth.param_set(PARAMS)
    g = binding.Context.from_params(ps, device=dist.local)
    rng = np.random.default_rng(3)
    n_lt = 128
    items = []
    for _ in range(n_lt):
        d = int(rng.choice([16, 64, 256, 1024]))
        ks = [k for k in range(1, 5) if d * (1 << k) <= ps.n // 2]
        stride = 1 if rng.random() < 0.5 or not ks else 1 << int(rng.choice(ks))
        items.append((d, stride, int(rng.integers(6, 25))))
    shapes = sorted({(d, st) for d, st, _ in items})
    combos = sorted({(d, st, lv) for d, st, lv in items})
    # keys for the cost model's best candidates of every (shape, level) present,
    # as many candidates as keep the key set within 300 keys (176 MB each)
    for ncand in (3, 2, 1):
        cands = {c: g.candidate_splits("th", c[2], c[0], ncand) for c in combos}
        rots = sorted({r for (d, st, lv), cs in cands.items() for sp in cs
                       for r in g.required_rotations("th", sp, d, st)})
        if len(rots) <= 300:
            break
    for r in rots:
        t = synth.uniform_mod_device(SEED, f"key/{r}", ps.moduli, ps.n, count=2 * g.beta_max, device=device)
        g.upload_rotation_key_device(r, t)
        del t
    top = list(ps.q) + list(ps.p)
    mats = {}
    for (d, st) in shapes:
        t = synth.uniform_mod_device(SEED, f"diag/{d}/{st}", top, ps.n, count=d, device=device)
        mats[(d, st)] = g.upload_diagonals_device(t, stride=st, level=ps.L)
        del t
    torch.cuda.empty_cache()
    cts = [g.ct_wrap(synth.uniform_mod_device(SEED + 10 + n, f"ct/{n}", list(ps.q[:lv]), ps.n, count=2,
                                              device=device), lv) for n, (_, _, lv) in enumerate(items)]
    outs = [g.ct_empty(lv - 1) for (_, _, lv) in items]
    fs = [mats[(d, st)] for d, st, _ in items]
    # the measuring autotuner, per (shape, level): times the candidates on one of the LTs
    split_of = {}
    for (d, st, lv), cs in cands.items():
        sample = next(c for c, it in zip(cts, items) if it == (d, st, lv))
        split_of[(d, st, lv)] = g.autotune("th", sample, mats[(d, st)], len(cs))[0] if len(cs) > 1 else cs[0]
    sps = [split_of[it] for it in items]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()

    def timed(fn, steps):
        for _ in range(max(3, args.warmup)):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        dist.barrier()
        e0.record(stream)
        for _ in range(steps):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        dist.barrier()
        return dist.max(e0.elapsed_time(e1))

    def sequential():
        for c, o, f, sp in zip(cts, outs, fs, sps):
            g.lt_eval(c, f, "th", sp, out=o)

    rec = g.lt_graph(cts, fs, algos=["th"] * n_lt, splits=sps, outs=outs)
    steps = max(1, min(args.steps, 20))
    clocks = ClockSampler(dist.local)
    clocks.start()
    ms_graph = timed(lambda: rec.launch(), steps)
    ms_seq = timed(sequential, steps)
    clk = clocks.stop()
    rec.close()
    val = dist.world * n_lt * steps / (ms_graph / 1e3)
    return {
        "metric": METRIC, "value": round(val, 3), "unit": "LT/s", "n_gpus": dist.world, "steps": steps,
        "warmup": args.warmup, "ms_per_step": round(ms_graph / steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (uniform residues drawn on the device; seeded)",
        "config": {"workload": f"uneven batch: {n_lt} LTs, N=2^16, D from {{16,64,256,1024}}, consecutive or "
                               f"2^k-strided offsets, levels 6..24 (seed 3), one matrix per (D, stride) shape; one "
                               f"recorded lt_eval_batch per step",
                   "splits": {f"{d}/{st}@{lv}": list(sp) for (d, st, lv), sp in sorted(split_of.items())},
                   "split_choice": f"lt_autotune per (shape, level) over the cost model's {ncand} best "
                                   f"({len(rots)} keys resident)",
                   "keys": len(rots)},
        "sequential_lt_per_s": round(dist.world * n_lt * steps / (ms_seq / 1e3), 3),
        "speedup_vs_sequential": round(ms_seq / ms_graph, 3),
        "clocks": clk,
    }


PAPER_SHAPES = {
    # the paper's parameter sets (Table "HE parameters") with its min-compute splits (Table of
    # algorithmic/hardware parameters) and its FPGA latency for TH-BSGS (Table of resources and latency)
    "paper-a": dict(params="setA", n_diag=4096, split=(16, 16, 16), fpga_ms=19.44),
    "paper-b": dict(params="setB", n_diag=16384, split=(32, 16, 32), fpga_ms=726.59),
}


def fpga_offchip(params: str) -> dict:
    """The paper's data-path off-chip model at its own knobs (Sec. IV formulas),
    next to the total its resource table prints; units of 2^30 bytes, 54-bit words."""
    from paper_2605_17222_gb300 import memory_model as mm
    shape, knobs, printed = mm.PAPER_SETS[{"setA": "Set-A", "setB": "Set-B"}[params]]
    by = mm.offchip_by_category(shape, knobs)
    return {"model": round(mm.paper_units(sum(by.values())), 3), "printed": printed, "unit": "2^30 bytes (54-bit words)",
            "by_category": {c: round(mm.paper_units(v), 3) for c, v in by.items()}}


def run_paper_shape(args, dist: Dist):
    """One dense LT (n = N/2 nonzero diagonals) with the paper's parameter set
    and split, timed like the headline workload."""
    import torch
    from paper_2605_17222_gb300 import binding, synth
    cfg = PAPER_SHAPES[args.workload]
    device = f"cuda:{dist.local}"
    torch.cuda.set_device(dist.local)
    ps = synth.param_set(cfg["params"])
    g = binding.Context.from_params(ps, device=dist.local)
    split, Dn, lvl = cfg["split"], cfg["n_diag"], ps.L
    for r in g.required_rotations("th", split, Dn, 1):
        t = synth.uniform_mod_device(SEED, f"key/{r}", ps.moduli, ps.n, count=2 * g.beta_max, device=device)
        g.upload_rotation_key_device(r, t)
        del t
    f = g.diags_create(Dn, 1, lvl)
    top = list(ps.q) + list(ps.p)
    chunk = 256
    for first in range(0, Dn, chunk):
        t = synth.uniform_mod_device(SEED + first, "diag", top, ps.n, count=min(chunk, Dn - first), device=device)
        g.diags_write(f, first, t)
        torch.cuda.synchronize()
        del t
    torch.cuda.empty_cache()
    ct = g.ct_wrap(synth.uniform_mod_device(SEED, "ct", list(ps.q[:lvl]), ps.n, count=2, device=device), lvl)
    out = g.ct_empty(lvl - 1)
    stream = torch.cuda.current_stream()
    # the measuring autotuner over the splits whose keys are resident (the paper's), then the
    # diagonal kernel's tile for it
    tuned_split, tuned_ms = g.autotune("th", ct, f, 4)
    tile = g.tuned_tile("th", f, lvl)
    for _ in range(max(3, args.warmup)):
        g.lt_eval(ct, f, "th", split, out=out)
    steps = max(1, min(args.steps, 50))
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    clocks = ClockSampler(dist.local)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(steps):
        if i == 0:  # one LT's launches for profilers (ncu --nvtx --nvtx-include "timed_lt/")
            torch.cuda.nvtx.range_push("timed_lt")
        g.lt_eval(ct, f, "th", split, out=out)
        if i == 0:
            torch.cuda.nvtx.range_pop()
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    clk = clocks.stop()
    step_ms = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(steps))
    total = dist.max(evs[0].elapsed_time(evs[-1]))
    limb = 8 * ps.n
    ext = lvl + ps.k
    keys = split[0] + split[1] + split[2] - 3
    comp = limb * (Dn * ext + keys * 2 * g.beta(lvl) * ext + 2 * lvl + 2 * (lvl - 1))
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    ms = total / steps
    return {
        "metric": METRIC, "value": round(dist.world * steps / (total / 1e3), 3), "unit": "LT/s",
        "n_gpus": dist.world, "steps": steps, "warmup": args.warmup, "ms_per_step": round(ms, 4),
        "p50_ms": round(step_ms[len(step_ms) // 2], 4), "p99_ms": round(step_ms[-1], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (uniform residues drawn on the device; seeded)",
        "config": {"workload": f"dense LT with the paper's {cfg['params']}: N=2^{ps.log_n}, L+1={ps.L}, "
                               f"alpha={ps.alpha}, beta={g.beta(lvl)}, n={Dn}, split {split}",
                   "split": list(split), "autotuned": {"split": list(tuned_split), "ms": round(tuned_ms, 4),
                                                        "k6_tile": list(tile) if tile else None}},
        "paper_fpga_ms_context": cfg["fpga_ms"],
        "paper_fpga_offchip": fpga_offchip(cfg["params"]),
        "hbm_roofline_lt": {"compulsory_bytes": comp, "frac": round(comp / (ms / 1e3) / 1e9 / peak, 4)},
        "clocks": clk,
    }


def chain_shapes(kind: str, log_slots: int, radices) -> list:
    """(offset0, stride, D) of each stage of a factored slot DFT, first applied
    first.  A group of r butterfly stages S_t .. S_{t+r-1} has its diagonals at
    the multiples of 2^(t-1) from -(2^r - 1) 2^(t-1) to +(2^r - 1) 2^(t-1),
    2^(r+1) - 1 of them, padded to 2^(r+1); the group that ends at the last
    stage covers every multiple, 2^r from offset 0.  SlotToCoeff applies the
    groups from S_1 up, CoeffToSlot (the inverses) from the last stage down."""
    out, t = [], 1
    for r in radices:
        h = 1 << (t - 1)
        if t + r - 1 == log_slots:
            out.append((0, h, 1 << r))
        else:
            out.append((-((1 << r) - 1) * h, h, 1 << (r + 1)))
        t += r
    if t - 1 != log_slots:
        raise ValueError("radices must sum to log2(N/2)")
    return out if kind == "stc" else out[::-1]


def run_chain(args, dist: Dist):
    """One CoeffToSlot (or SlotToCoeff) transform per step: a chain of three
    LTs (radices 5, 5, 5) from level 24 to 21 at N = 2^16, through
    lt_eval_chain, each stage with its autotuned TH-BSGS split."""
    import numpy as np
    import torch
    from paper_2605_17222_gb300 import binding, synth
    kind = args.workload
    device = f"cuda:{dist.local}"
    torch.cuda.set_device(dist.local)
    ps = synth.param_set(PARAMS)
    g = binding.Context.from_params(ps, device=dist.local)
    N, lvl0 = ps.n, LEVEL
    radices = (5, 5, 5)
    shapes = chain_shapes(kind, ps.log_n - 1, radices)
    top = list(ps.q) + list(ps.p)
    fs, cands = [], []
    for i, (off0, stride, Dn) in enumerate(shapes):
        t = synth.uniform_mod_device(SEED + 100 * i, f"chain/diag/{i}", top, N, count=Dn, device=device)
        fs.append(g.upload_diagonals_device(t, stride=stride, level=ps.L, offset0=off0))
        del t
        cands.append(g.candidate_splits("th", lvl0 - i, Dn, 4))
    keys_t = {}
    for i, (off0, stride, Dn) in enumerate(shapes):
        for sp in cands[i]:
            for r in g.required_rotations("th", sp, Dn, stride, offset0=off0):
                if r not in keys_t:
                    keys_t[r] = synth.uniform_mod_device(SEED, f"key/{r}", ps.moduli, N, count=2 * g.beta_max,
                                                         device=device)
                    g.upload_rotation_key_device(r, keys_t[r])
    splits = []
    for i, f in enumerate(fs):
        sample = g.ct_wrap(synth.uniform_mod_device(SEED + i, "chain/sample", list(ps.q[:lvl0 - i]), N, count=2,
                                                    device=device), lvl0 - i)
        sp, _ = g.autotune("th", sample, f, len(cands[i]))
        splits.append(sp)
    ct_t = synth.uniform_mod_device(SEED, "chain/ct", list(ps.q[:lvl0]), N, count=2, device=device)
    ct = g.ct_wrap(ct_t, lvl0)
    nst = len(shapes)
    out = g.ct_empty(lvl0 - nst)
    keep_host = not args.no_cpu_baseline and dist.rank == 0 and dist.world == 1
    used = set()
    for (off0, stride, Dn), sp in zip(shapes, splits):
        used |= set(g.required_rotations("th", sp, Dn, stride, offset0=off0))
    keys_t = {r: t for r, t in keys_t.items() if r in used} if keep_host else {}
    torch.cuda.empty_cache()
    stream = torch.cuda.current_stream()
    for c in binding.KERNEL_CLASSES:
        binding.profile_enable(c, True)
    binding.profile_reset()
    for _ in range(max(3, args.warmup)):
        g.lt_eval_chain(ct, fs, out=out)
    torch.cuda.synchronize()
    shares = {c: binding.profile_read(c) for c in binding.KERNEL_CLASSES}
    for c in binding.KERNEL_CLASSES:
        binding.profile_enable(c, False)
    tot = sum(v[0] for v in shares.values()) or 1.0
    dominant = max(("diag_mac", "ks_inner"), key=lambda c: shares[c][0])
    clocks = ClockSampler(dist.local)
    clocks.start()
    time.sleep(0.3)
    binding.profile_reset()
    binding.profile_enable(dominant, True)
    l0 = binding.kernel_launches()
    steps = max(1, args.steps)
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
    dist.barrier()
    torch.cuda.synchronize()
    evs[0].record(stream)
    for i in range(steps):
        g.lt_eval_chain(ct, fs, out=out)
        evs[i + 1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    launches = binding.kernel_launches() - l0
    dom_ms, dom_n = binding.profile_read(dominant)
    binding.profile_enable(dominant, False)
    step_ms = sorted(evs[i].elapsed_time(evs[i + 1]) for i in range(steps))
    total_ms = dist.max(evs[0].elapsed_time(evs[-1]))
    # the same transform recorded once (lt_graph_begin/end) and replayed
    rs = torch.cuda.Stream()
    g.lt_eval_chain(ct, fs, out=out, stream=rs)
    rs.synchronize()
    g.graph_begin(rs)
    g.lt_eval_chain(ct, fs, out=out, stream=rs)
    rec = g.graph_end(rs, keep=(ct, out, fs))
    for _ in range(3):
        rec.launch(rs)
    rs.synchronize()
    g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    dist.barrier()
    g0.record(rs)
    for _ in range(steps):
        rec.launch(rs)
    g1.record(rs)
    torch.cuda.synchronize()
    dist.barrier()
    graph_ms = dist.max(g0.elapsed_time(g1))
    rec.close()
    # end to end through the C ABI: host ciphertext in, host result out, every step
    n_in, n_out = 2 * lvl0 * N, 2 * (lvl0 - nst) * N
    h_in = torch.empty(n_in, dtype=torch.int64, pin_memory=True)
    h_in.copy_(ct_t.reshape(-1).cpu())
    hin = h_in.numpy().view(np.uint64)
    e2e_steps = max(2, steps // 2)
    e2e_ms = e2e_pipelined(g, lambda di, do, st: g.lt_eval_chain(di, fs, out=do, stream=st), hin, n_out, lvl0,
                           lvl0 - nst, e2e_steps, dist)
    clk = clocks.stop()
    # roofline of the dominant kernel: its algorithmic bytes summed over the stages
    peaks = measured_peaks()
    peak = peaks.get("hbm_gbs", 6800.0)
    per_chain, per_chain_launches = 0, 0
    for i, ((off0, stride, Dn), sp) in enumerate(zip(shapes, splits)):
        amounts = [(off0 + stride * sp[0] * sp[1] * kk) % (N // 2) for kk in range(sp[2])]
        b, n = algorithmic_bytes(dominant, sp, lvl0 - i, ps.k, g.beta(lvl0 - i), Dn, N,
                                 outer_rotated=sum(1 for a in amounts if a))
        per_chain += b
        per_chain_launches += n
    ach = per_chain * steps / (dom_ms / 1e3) / 1e9 if dom_ms else None
    unit = "CoeffToSlot/s" if kind == "cts" else "SlotToCoeff/s"
    res = {
        "metric": f"{'CoeffToSlot' if kind == 'cts' else 'SlotToCoeff'} transforms/s at N=2^16 (3 levels, "
                  f"bit-exact TH-BSGS chain)",
        "value": round(dist.world * steps / (total_ms / 1e3), 3), "unit": unit, "n_gpus": dist.world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(total_ms / steps, 4),
        "p50_ms": round(step_ms[len(step_ms) // 2], 4), "p99_ms": round(step_ms[-1], 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u64",
        "data": "synthetic (uniform residues drawn on the device; seeded)",
        "config": {"workload": f"{kind}: factored slot DFT at N=2^16, level {lvl0} -> {lvl0 - nst}, radices "
                               f"{list(radices)}, stages (offset0, stride, D) {shapes}",
                   "splits": [list(s) for s in splits], "parallelism": f"replicas x{dist.world}",
                   "l2": "diagonals + keys resident, several GB per step > L2; no flush"},
        "lt_per_s": round(dist.world * steps * nst / (total_ms / 1e3), 3),
        "recorded_graph_per_s": round(dist.world * steps / (graph_ms / 1e3), 3),
        "roofline": {"kernel": dominant, "bound": "hbm", "achieved": round(ach, 1) if ach else None, "peak": peak,
                     "unit": "GB/s", "frac": round(ach / peak, 4) if ach else None, "traffic": None,
                     "algorithmic_bytes_per_chain": int(per_chain),
                     "avg_launch_ms": round(dom_ms / dom_n, 4) if dom_n else None,
                     "peak_source": "measured HBM copy bandwidth" if "hbm_gbs" in peaks else "fallback"},
        "kernel_shares": {c: round(v[0] / tot, 4) for c, v in shares.items()},
        "e2e": {"value": round(dist.world * e2e_steps / (e2e_ms / 1e3), 3), "unit": unit,
                "h2d_bytes_per_step": n_in * 8, "d2h_bytes_per_step": n_out * 8,
                "ms_per_step": round(e2e_ms / e2e_steps, 4)},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if keep_host:
        t0 = time.perf_counter()
        from oracle import lt as olt
        from oracle.ckks import Ctx
        keys = {r: binding.to_host(t).reshape(g.beta_max, 2, ps.L + ps.k, N) for r, t in keys_t.items()}
        stages = []
        for i, ((off0, stride, Dn), sp) in enumerate(zip(shapes, splits)):
            dt = synth.uniform_mod_device(SEED + 100 * i, f"chain/diag/{i}", top, N, count=Dn, device=device)
            stages.append((np.ascontiguousarray(binding.to_host(dt)), "th", sp, stride, off0))
            del dt
        cth = binding.to_host(ct_t)
        octx = Ctx(ps)
        t1 = time.perf_counter()
        olt.lt_chain(octx, (np.ascontiguousarray(cth[0]), np.ascontiguousarray(cth[1])), stages, keys)
        cpu_s = time.perf_counter() - t1
        res["cpu_baseline"] = {"value": round(1.0 / cpu_s, 5), "unit": unit, "cores": cores_used(), "kind": "oracle",
                               "sample": f"one full oracle chain ({nst} LTs) of the workload, "
                                         f"{cpu_s:.1f} s (setup {t1 - t0:.1f} s untimed)"}
    return res


def run_steps(args, dist: Dist):
    """The key-switching steps on their own at N = 2^16, level 24 (no LT):
    Decompose of a ciphertext's c1 (144 limbs of forward NTT with the basis
    conversion fused into the column pass, 24 limbs of inverse NTT) and the
    forward NTT of a 28-limb extended polynomial, each timed over `steps`
    calls with CUDA events, with the library's per-class kernel times.  The
    device holds a few hundred MB, which keeps ncu captures of the NTT
    passes small."""
    import torch
    from paper_2605_17222_gb300 import binding, synth
    device = f"cuda:{dist.local}"
    torch.cuda.set_device(dist.local)
    ps = synth.param_set(PARAMS)
    g = binding.Context.from_params(ps, device=dist.local)
    N, L, K = ps.n, LEVEL, ps.k
    cs = synth.uniform_mod_device(SEED, "steps/c", list(ps.q[:L]), N, count=8, device=device)
    digs = [torch.empty((g.beta(L), L + K, N), dtype=torch.int64, device=device) for _ in range(8)]
    ext = synth.uniform_mod_device(SEED, "steps/ext", list(ps.q[:L]) + list(ps.p), N, count=8, device=device)
    steps = max(1, args.steps)
    for i in range(max(3, args.warmup)):
        g.decompose(cs[i % 8], L, digits=digs[i % 8])
        g.ntt(ext[i % 8], L, True, False)
    torch.cuda.synchronize()
    res = {"metric": "key-switching steps at N=2^16, level 24 (us per call)", "unit": "us", "steps": steps,
           "warmup": args.warmup, "n_gpus": 1, "higher_is_better": False, "dtype": "u64",
           "data": "synthetic (uniform residues drawn on the device; seeded)",
           "config": {"workload": "steps: Decompose of c1 at level 24 (alpha 4, beta 6, k 4), forward NTT of a "
                                  "28-limb extended polynomial"}}
    for name, fn in [("decompose", lambda i: g.decompose(cs[i % 8], L, digits=digs[i % 8])),
                     ("ntt_fwd_ext", lambda i: g.ntt(ext[i % 8], L, True, False))]:
        for c in binding.KERNEL_CLASSES:
            binding.profile_enable(c, True)
        binding.profile_reset()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for i in range(steps):
            fn(i)
        e1.record()
        torch.cuda.synchronize()
        per = {c: binding.profile_read(c) for c in binding.KERNEL_CLASSES}
        for c in binding.KERNEL_CLASSES:
            binding.profile_enable(c, False)
        res[name] = {"us_per_call": round(e0.elapsed_time(e1) * 1e3 / steps, 2),
                     "kernels_us_per_call": {c: round(ms * 1e3 / steps, 2) for c, (ms, n) in per.items() if n}}
    return res


def run_serving(args, dist: Dist):
    """Poisson arrivals (rate, duration; seed 4) of single-LT requests, each with
    N from {2^15, 2^16}, 32..512 diagonals (powers of two) and a level of
    6..24 (6..16 at N = 2^15); keys and matrices resident; admission under a
    150 GB HBM budget; continuous batching over 4 streams."""
    import numpy as np
    import torch
    from paper_2605_17222_gb300 import binding, synth
    from paper_2605_17222_gb300.serving import LtServer, Request, percentile, run_open_loop
    device = f"cuda:{dist.local}"
    torch.cuda.set_device(dist.local)
    rng = np.random.default_rng(4 + dist.rank)
    sizes = [32, 64, 128, 256, 512]
    sets = {16: synth.param_set("n16"), 15: synth.param_set("n15")}
    lv_range = {16: (6, 24), 15: (6, 16)}
    ctxs, mats, pools, resident = {}, {}, {}, 0
    for ln, ps in sets.items():
        g = binding.Context.from_params(ps, device=dist.local)
        ctxs[ln] = g
        lo, hi = lv_range[ln]
        rots = set()
        for d in sizes:
            for lv in range(lo, hi + 1):
                rots |= set(g.required_rotations("th", g.choose_split("th", lv, d), d, 1))
        for r in sorted(rots):
            t = synth.uniform_mod_device(SEED, f"key/{ln}/{r}", ps.moduli, ps.n, count=2 * g.beta_max, device=device)
            g.upload_rotation_key_device(r, t)
            resident += t.numel() * 8
            del t
        top = list(ps.q) + list(ps.p)
        for d in sizes:
            t = synth.uniform_mod_device(SEED, f"diag/{ln}/{d}", top, ps.n, count=d, device=device)
            mats[(ln, d)] = g.upload_diagonals_device(t, stride=1, level=ps.L)
            resident += t.numel() * 8
            del t
        for lv in range(lo, hi + 1):
            pools[(ln, lv)] = [g.ct_wrap(synth.uniform_mod_device(SEED + c, f"ct/{ln}/{lv}/{c}", list(ps.q[:lv]),
                                                                  ps.n, count=2, device=device), lv)
                               for c in range(2)]
    torch.cuda.synchronize()
    n_req = int(args.rate * args.duration)
    arrivals = np.cumsum(rng.exponential(1.0 / args.rate, n_req)).tolist()
    specs = []
    for i in range(n_req):
        ln = int(rng.choice([15, 16]))
        lo, hi = lv_range[ln]
        specs.append((ln, int(rng.choice(sizes)), int(rng.integers(lo, hi + 1))))

    def make_request(i, t_arr):
        ln, d, lv = specs[i]
        return Request(i, ln, mats[(ln, d)], pools[(ln, lv)][i % 2], t_arr)

    srv = LtServer(ctxs, hbm_budget=150e9, resident_bytes=resident, streams=4, max_batch=16)
    # warm-up: one request of every (context, level, matrix) shape sets up tables and kernel attributes
    for ln in sets:
        lo, hi = lv_range[ln]
        for lv in range(lo, hi + 1):
            for d in sizes:
                srv.submit(Request(-1, ln, mats[(ln, d)], pools[(ln, lv)][0], time.perf_counter()))
    srv.drain(timeout_s=600)
    srv.stats = type(srv.stats)()
    srv.completed = []
    clocks = ClockSampler(dist.local)
    clocks.start()
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    run_open_loop(srv, arrivals, make_request)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    dist.barrier()
    clk = clocks.stop()
    lat = srv.stats.latencies
    done = dist.world * srv.stats.completed
    wall_max = dist.max(wall)
    # the plain form on the identical request list: one lt_eval after another on
    # one stream, each with the split the server used for its shape
    outs = {key: ctxs[key[0]].ct_empty(key[1] - 1) for key in pools}
    splits = {(ln, d, lv): ctxs[ln].choose_split("th", lv, d) for ln, d, lv in set(specs)}
    torch.cuda.synchronize()
    t_seq = time.perf_counter()
    for i, (ln, d, lv) in enumerate(specs):
        ctxs[ln].lt_eval(pools[(ln, lv)][i % 2], mats[(ln, d)], "th", splits[(ln, d, lv)], out=outs[(ln, lv)])
    torch.cuda.synchronize()
    seq_s = dist.max(time.perf_counter() - t_seq)
    return {
        "metric": METRIC, "value": round(done / wall_max, 3), "unit": "LT/s", "n_gpus": dist.world,
        "steps": srv.stats.completed, "warmup": 1, "ms_per_step": None, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u64", "data": "synthetic (uniform residues drawn on the device; seeded)",
        "config": {"workload": f"serving: Poisson arrivals {args.rate:g} req/s for {args.duration:g} s (seed 4), "
                               f"N in {{2^15, 2^16}}, {sizes[0]}..{sizes[-1]} diagonals, levels 6..24 (6..16 at "
                               f"2^15), keys and matrices resident, 150 GB admission budget, 4 streams",
                   "resident_bytes": resident},
        "p50_ms": round(1e3 * percentile(lat, 50), 3), "p99_ms": round(1e3 * percentile(lat, 99), 3),
        "mean_ms": round(1e3 * float(np.mean(lat)), 3) if lat else None,
        "offered_rate": args.rate, "completed": srv.stats.completed, "wall_s": round(wall_max, 3),
        "batches": srv.stats.batches, "mean_batch": round(srv.stats.completed / max(1, srv.stats.batches), 2),
        "admission_waits": srv.stats.admission_waits, "max_inflight_scratch_bytes": srv.stats.max_inflight_bytes,
        "sequential": {"value": round(dist.world * len(specs) / seq_s, 3), "unit": "LT/s", "wall_s": round(seq_s, 3),
                       "how": "the same request list as back-to-back lt_eval calls on one stream (no batching, "
                              "no arrival gaps): the plain single-ciphertext form's capacity"},
        "served_over_sequential": round((done / wall_max) / (dist.world * len(specs) / seq_s), 3),
        "clocks": clk,
    }


def run_reference(args, dist: Dist):
    """The CPU oracle as the reference arm, on this host's cores."""
    global D, LEVEL
    D, LEVEL = args.diags, args.level
    if dist.rank != 0:
        return None
    import numpy as np
    from paper_2605_17222_gb300 import synth
    ps = synth.param_set(PARAMS)
    split = tuple(int(x) for x in args.split.split(",")) if args.split else (4, 8, 8)
    split3 = tuple(split) + (1,) * (3 - len(split))
    N = ps.n
    alpha = -(-ps.L // ps.dnum)
    beta_max = -(-ps.L // alpha)
    top = list(ps.q) + list(ps.p)
    from oracle import lt as olt
    rots = olt.rotation_set(args.algo, D, split3 if args.algo != "diag" else None, 1, N // 2)
    keys = {r: synth.uniform_mod(SEED, f"key/{r}", top * (2 * beta_max), N).reshape(beta_max, 2, len(top), N)
            for r in rots}
    diags = np.stack([synth.uniform_mod(SEED, f"diag/{t}", top, N) for t in range(D)])
    ct = (synth.uniform_mod(SEED, "ct0", ps.q[:LEVEL], N), synth.uniform_mod(SEED, "ct1", ps.q[:LEVEL], N))
    budget, warm_budget = 150.0, 40.0
    times, warm, _ = time_oracle(ps, args.algo, split3, keys, diags, ct, budget_s=budget, max_steps=args.steps,
                              warmup=args.warmup, warmup_budget_s=warm_budget)
    total = sum(times)
    v = len(times) / total
    return {
        "metric": METRIC, "value": round(v, 5), "unit": "LT/s", "n_gpus": dist.world, "steps": len(times),
        "warmup": warm, "ms_per_step": round(1e3 * total / len(times), 1), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic (uniform residues, seeded)",
        "config": {"workload": f"single LT: N=2^16, level {LEVEL} (Q = 55b + 23x40b), 4x60b special primes, "
                               f"dnum 6, {D} consecutive diagonals, one ciphertext at the top level",
                   "algo": args.algo, "split": list(split3), "parallelism": "cpu",
                   "split_choice": "given" if args.split else "(4,8,8): the oracle's cheapest TH split at this D "
                                                              "(fewest key inner products)"},
        "impl": "reference",
        "cpu_baseline": {"value": round(v, 5), "unit": "LT/s", "cores": cores_used(), "kind": "oracle",
                         "sample": f"{len(times)} full oracle LT(s) of the workload after {warm} untimed "
                                   f"warm-up LT(s) (budgets {warm_budget:.0f} s warm-up, {budget:.0f} s timed "
                                   f"cap the {args.warmup} + {args.steps} requested)"},
        "e2e": {"value": round(v, 5), "unit": "LT/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main():
    args = parse()
    dist = Dist()
    try:
        if args.impl == "reference":
            res = run_reference(args, dist)
        elif args.workload == "batched":
            res = run_batched(args, dist)
        elif args.workload == "serving":
            res = run_serving(args, dist)
        elif args.workload == "uneven":
            res = run_uneven(args, dist)
        elif args.workload in PAPER_SHAPES:
            res = run_paper_shape(args, dist)
        elif args.workload in ("cts", "stc"):
            res = run_chain(args, dist)
        elif args.workload == "steps":
            res = run_steps(args, dist)
        else:
            res = run_ours(args, dist)
        if dist.rank == 0 and res is not None:
            print(json.dumps(res), flush=True)
    finally:
        dist.close()


if __name__ == "__main__":
    main()
