"""Benchmark: certified minimum distance on one GB300 (or N GPUs).

One step certifies d of the headline code once, the whole hot path (every
pass of the Brouwer-Zimmermann search, Sec. 3.1 Alg. 6, on the device).
Default workload: the F_3 [80,40] random systematic code (PCG64 seed 2),
the largest single-code configuration.

value     codewords/s of the device search with the code's tables already
          resident in HBM (CUDA events around each step, on the search's
          stream; L2 flushed between steps with a 256 MiB memset outside the
          timed windows).
e2e       the same metric through fpcode_min_distance() from a pinned host
          matrix: host preparation, H2D, search, D2H read-back of the result.
roofline  the enumeration kernel against the POPC issue ceiling of the SMs:
          the rate fpcode_int_peaks() measures (POPC lanes per clock per SM)
          x SMs x the median SM clock sampled during the timed region.
cpu_baseline  the CPU oracle (test infrastructure) on the same code, all
          host cores.

The default line also carries the other configurations at their stated
sizes, each measured in the same run:
  f7_n40_k20  the F_7 [40,20] code (PCG64 seed 1): certified search time,
              codewords/s, roofline fraction, and one long pass alone;
  batch512    512 random codes (p in {3,7}, n in 24..64, PCG64 seed 3) in
              persistent launches (fpcode_min_distance_batch) against one
              launch per code, codes/s from host matrices, per-code budget
              --budget codewords;
  serve       10 000 codes (p in {3,5,7}, n in 20..72, PCG64 seed 4)
              arriving as a Poisson process at 200 requests/s, served with
              continuous batching (fpcode_serve_*): codes/s and latency from
              arrival to result (p50, p90, p99, max).

Further workloads have their own line (--workload): the single-pass probes,
the additions benchmark of Sec. 5.1, and each extra above alone.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W]
                       [--impl ours|reference] [--workload NAME]
                       [--budget B] [--requests R] [--no-extras]
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

WORKLOADS = {
    "f3_n80_k40": "F_3 [80,40] random systematic code G=[I|A], A uniform, PCG64 seed 2",
    "f7_n40_k20": "F_7 [40,20] random systematic code G=[I|A], A uniform, PCG64 seed 1",
    "f3_n30_k15": "F_3 [30,15] random systematic code G=[I|A], A uniform, PCG64 seed 0",
    "additions_f3": "10 000 pairs of F_3 vectors of 512 symbols added 10 000 times (Sec. 5.1 workload)",
    "additions_f7": "10 000 pairs of F_7 vectors of 512 symbols added 10 000 times (Sec. 5.1 workload)",
    "probe_f3_n80_k40_g8": "one pass (g=8, Gamma_1) of the F_3 [80,40] code alone, termination off, U seeded at d: "
                           "C(40,8) 2^7 = 9 843 799 680 codewords",
    "probe_f7_n40_k20_g7": "one pass (g=7, Gamma_1) of the F_7 [40,20] code alone, termination off, U seeded at d: "
                           "C(20,7) 6^6 = 3 616 773 120 codewords",
    "f3_n80_k40_split": "the F_3 [80,40] search (PCG64 seed 2) split over the ranks: every pass's tasks in contiguous "
                        "ranges, one allreduce-min of the 8-byte packed key per pass before its termination test",
    "batch512": "512 random codes, p in {3,7}, n in {24,...,64}, k = round(r n), r ~ U[1/3,2/3], PCG64 seed 3",
    "serve": "Poisson arrivals (200/s) of 10 000 random codes, p in {3,5,7}, n ~ U[20,72], k ~ U[n/3,2n/3], "
             "PCG64 seed 4",
}
PROBES = {"probe_f3_n80_k40_g8": ("f3_n80_k40", 8), "probe_f7_n40_k20_g7": ("f7_n40_k20", 7)}
ADDITIONS = {"additions_f3": 3, "additions_f7": 7}
FLUSH_BYTES = 256 << 20

# DRAM bytes of one bz_kernel launch per workload, from one ncu capture of
# that workload (dram__bytes_read.sum + dram__bytes_write.sum, summarised
# under profiles/).  Reported only while the kernel sources hash to the
# version that was profiled; any later change of their code reports null
# (the hash skips comments and blank lines).
KERNEL_SOURCES = ["fp_kernel.cuh", "fp_enum.cuh", "fp_bitslice.cuh", "fp_types.h"]
_SHA_PROFILED = "8780d0da516689b5a57dcd3df7282efb232c48e9f0263d9e0ea74675ba62254a"
PROFILED_TRAFFIC: dict = {  # profiles/bz_kernel_*.md (the command of each capture is there)
    "f3_n80_k40": {"bytes": 5725952 + 0, "sources_sha256": _SHA_PROFILED},
    "probe_f3_n80_k40_g8": {"bytes": 5715712 + 0, "sources_sha256": _SHA_PROFILED},
    "f7_n40_k20": {"bytes": 9477376 + 256, "sources_sha256": _SHA_PROFILED},
    "probe_f7_n40_k20_g7": {"bytes": 7579136 + 29952, "sources_sha256": _SHA_PROFILED},
}


def code_of(text: str) -> str:
    """C++ source without comments, trailing blanks and blank lines."""
    import re

    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    lines = (re.sub(r"//.*$", "", ln).rstrip() for ln in text.splitlines())
    return "\n".join(ln for ln in lines if ln)


def kernel_sources_sha256() -> str:
    import hashlib

    h = hashlib.sha256()
    root = os.path.join(ROOT, "paper_2603_29942_gb300", "csrc")
    for f in KERNEL_SOURCES:
        with open(os.path.join(root, f), encoding="utf-8") as fh:
            h.update(code_of(fh.read()).encode())
    return h.hexdigest()


def profiled_traffic(workload: str):
    rec = PROFILED_TRAFFIC.get(workload)
    if rec and rec["sources_sha256"] == kernel_sources_sha256():
        return rec["bytes"]
    return None


# ----------------------------------------------------------- processes ----

def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def dist_init(world: int, local: int, backend: str = "nccl") -> None:
    """One process per GPU (torchrun); nothing to do for a single rank."""
    if world <= 1:
        return
    import torch
    import torch.distributed as dist

    if dist.is_initialized():
        return
    if backend == "nccl":
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        dist.init_process_group(backend)


def shard(n: int, rank: int, world: int) -> range:
    """The contiguous block of n independent units (codes) rank `rank` of
    `world` takes: n split evenly, the first n % world ranks one more."""
    base, extra = divmod(n, world)
    lo = rank * base + min(rank, extra)
    return range(lo, lo + base + (1 if rank < extra else 0))


def _reduce(x: float, world: int, op: str) -> float:
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    dev = torch.device("cuda") if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM if op == "sum" else dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(x: float, world: int) -> float:
    """The total of a per-rank count over all ranks."""
    return _reduce(x, world, "sum")


def max_over_ranks(x: float, world: int) -> float:
    """The largest value over all ranks (a job takes as long as its slowest
    rank); barrier semantics come with the collective."""
    return _reduce(x, world, "max")


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        time.sleep(0.3)
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        """Median SM clock over the samples taken under load (power above the
        idle floor or clock above a quarter of the maximum), the maximum clock,
        and every throttle reason seen."""
        rows, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((float(parts[1]), float(parts[3])))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        loaded = [c for c, _p in rows if c > 0.25 * mx] if mx else []
        mhz = loaded or [c for c, _p in rows]
        return {"sm_mhz": statistics.median(mhz) if mhz else None, "sm_max_mhz": mx or None,
                "reasons": sorted(reasons), "samples": len(rows), "samples_under_load": len(loaded)}


# ------------------------------------------------------------- CPU arms ----

def cpu_baseline(code) -> dict:
    """The oracle as it stands, on every host core, on the same code."""
    import oracle

    threads = os.cpu_count() or 1
    t0 = time.perf_counter()
    r = oracle.bz(code, threads=threads)
    dt = time.perf_counter() - t0
    return {"value": r.evaluated / dt, "unit": "codewords/s", "cores": threads, "kind": "oracle",
            "sample": f"full certified search of the same code ({r.evaluated} codewords, d={r.d}) in {dt:.2f} s",
            "d": r.d, "seconds": dt}


def single_config(name: str, d=None) -> dict:
    """The config dict of a single-code workload, the same in both arms."""
    cfg = {"workload": name, "description": WORKLOADS[name], "l2": "flushed between timed steps (256 MiB memset)",
           "parallelism": "single GPU"}
    if d is not None:
        cfg["d"] = d
    return cfg


def run_reference(args, code, rank: int, world: int):
    """Reference arm: the CPU oracle on the host cores, same metric and config
    (rank 0 only; the other ranks exit without work)."""
    if rank != 0:
        return
    import oracle

    threads = os.cpu_count() or 1
    for _ in range(args.warmup):
        oracle.bz(code, threads=threads)
    times, ev = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        r = oracle.bz(code, threads=threads)
        times.append(time.perf_counter() - t0)
        ev = r.evaluated
    total = sum(times)
    value = ev * args.steps / total
    cfg = single_config(args.workload, r.d)
    cfg["parallelism"] = "replicas" if world > 1 else "single GPU"
    line = {
        "impl": "reference", "metric": "codewords_per_s", "value": value, "unit": "codewords/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
        "config": cfg,
        "cpu_baseline": {"value": value, "unit": "codewords/s", "cores": threads, "kind": "oracle",
                         "sample": f"full certified search of the same code per step ({ev} codewords)"},
        "e2e": {"value": value, "unit": "codewords/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# -------------------------------------------------------------- the GPU ----

def _cuda(local):
    import torch

    torch.cuda.set_device(local)
    from paper_2603_29942_gb300 import _binding as B
    from paper_2603_29942_gb300 import build as _b

    _b.build()
    B.lib()
    return torch, B


def popc_peak(B, stream, sm_mhz, sms) -> dict:
    """The POPC ceiling: lanes per clock per SM measured by fpcode_int_peaks
    (independent chains on every SM) x SMs x the SM clock sampled under load
    (the microbenchmark's own clock if none was sampled)."""
    rates = B.fpcode_int_peaks(stream)
    mhz = sm_mhz or rates["sm_mhz"]
    per_clk = rates["popc_per_clk_sm"]
    return {"tpopc_s": per_clk * sms * mhz * 1e6 / 1e12, "popc_per_clk_sm": per_clk,
            "lop3_per_clk_sm": rates["lop3_per_clk_sm"], "sm_mhz": mhz, "sms": sms,
            "basis": f"fpcode_int_peaks: {per_clk:.2f} POPC/clk/SM x {sms} SMs x {mhz:.0f} MHz (median under load)"}


def time_search(torch, B, prep, stream, steps, warmup, flush, want_d=None):
    """Device-timed certified searches on resident tables: CUDA events on the
    search's stream around each enqueue, L2 flushed outside the windows.
    Returns (event ms per step, kernel ms per step, last result)."""
    for _ in range(warmup):
        B.fpcode_search_enqueue(prep, stream)
        res = B.fpcode_search_finish(prep, stream, want_witness=False)
    assert res.status == B.OK and (want_d is None or res.d == want_d)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kern = []
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(i & 0xFF)  # L2 flush, outside the timed window
            evs[i][0].record(stream)
            B.fpcode_search_enqueue(prep, stream)
            evs[i][1].record(stream)
            r = B.fpcode_search_finish(prep, stream, want_witness=(i == steps - 1))
            assert r.status == B.OK and r.d == res.d
            kern.append(r.t_kernel_ms)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs], kern, r


def time_pass(torch, B, pr, idx, d, stream, steps, warmup, flush):
    """Time pass `idx` of prepared code `pr` alone (U seeded at d), L2
    flushed between steps.  Returns (total event ms, mean kernel ms, least
    weight found in the pass)."""
    g, size = B.fpcode_prepared_passes(pr)[idx][0], B.fpcode_prepared_passes(pr)[idx][5]
    probe = B.fpcode_prepared_single_pass(pr, idx, d)
    B.fpcode_prepared_upload(probe, stream)
    for _ in range(warmup):
        B.fpcode_search_enqueue(probe, stream)
        r = B.fpcode_search_finish(probe, stream, want_witness=False)
    assert r.counts[g] == size
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    kern = []
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for i in range(steps):
            flush.fill_(i & 0xFF)
            evs[i][0].record(stream)
            B.fpcode_search_enqueue(probe, stream)
            evs[i][1].record(stream)
            r = B.fpcode_search_finish(probe, stream, want_witness=False)
            assert r.counts[g] == size
            kern.append(r.t_kernel_ms)
    torch.cuda.synchronize()
    return sum(a.elapsed_time(b) for a, b in evs), statistics.mean(kern), r.U


def probe_prepare(B, code):
    """The code prepared for a single-pass probe: the full schedule, with the
    leaf form the library's own rule gives a search of the timed pass's size
    (pair leaves from 10^8 codewords on, where they fit)."""
    return B.fpcode_prepare(code.p, code.n, code.k, code.G, B.fpcode_opts_default(budget=0, pair_leaves=1))


def probe_line(torch, B, code, name, g, d, stream, flush, peak_t, steps=5, warmup=3) -> dict:
    """The kernel's steady state: one long pass of fixed, closed-form size
    alone, termination off, U seeded at d (the threshold a certified search
    has at that level)."""
    pr = probe_prepare(B, code)
    passes = B.fpcode_prepared_passes(pr)
    idx = next(i for i, x in enumerate(passes) if x[0] == g and x[1] == 0)
    size = passes[idx][5]
    t_ms, k_ms, least = time_pass(torch, B, pr, idx, d, stream, steps, warmup, flush)
    W = max(1, -(-(code.n - code.k) // 32))
    ach = size * W / (k_ms * 1e-3) / 1e12
    return {"bound": "alu", "achieved": ach, "peak": peak_t, "unit": "Tpopc/s", "frac": ach / peak_t,
            "traffic": profiled_traffic(name), "pass": [g, 0], "codewords": size, "kernel_ms": k_ms, "workload": name,
            "leaf_form": "pair" if B.fpcode_test_pair_mode(pr) else "one-row", "least_weight_in_pass": least,
            "note": "the same kernel on one pass of fixed size alone, termination off, U seeded at d"}


def single_code(args, torch, B, name, stream, flush, world, clk_need=True):
    """One certified single-code workload: device-timed steps and the kernel
    time of each.  Returns a dict of the measurements."""
    from paper_2603_29942_gb300 import inputs

    code = inputs.single(name)
    prep = B.fpcode_prepare(code.p, code.n, code.k, code.G)
    B.fpcode_prepared_upload(prep, stream)
    steps_ms, kern, r = time_search(torch, B, prep, stream, args.steps, args.warmup, flush)
    W = max(1, -(-(code.n - code.k) // 32))
    return {"code": code, "prep": prep, "res": r, "steps_ms": steps_ms, "kern_ms": kern, "W": W,
            "codewords": r.enumerated, "counts_total": sum(r.counts),
            "leaf_form": "pair" if B.fpcode_test_pair_mode(prep) else "one-row"}


def e2e_line(torch, B, code, prep, stream, steps, world, counts_total):
    """The same metric through the public call from a pinned host matrix:
    preparation, H2D of the tables, search, D2H of the result each step."""
    h2d, d2h = B.fpcode_prepared_bytes(prep)
    G_host = torch.from_numpy(code.G.copy()).pin_memory().numpy()
    for _ in range(3):
        B.fpcode_min_distance(code.p, code.n, code.k, G_host, stream)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        d, _w = B.fpcode_min_distance(code.p, code.n, code.k, G_host, stream)
    e2e_s = time.perf_counter() - t0
    return {"value": world * counts_total * steps / e2e_s, "unit": "codewords/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s / steps, "d": d}


def batch_measure(args, torch, B, rank, world) -> dict:
    """512 codes: persistent batched launches vs one launch per code, end to
    end from host matrices, the same per-code budget."""
    from paper_2603_29942_gb300 import inputs

    all_codes = inputs.batch_codes(512)
    codes = [all_codes[i] for i in shard(len(all_codes), rank, world)]  # codes are independent: no exchange
    budget = int(args.budget)
    budgets = [budget] * len(codes)
    stream = torch.cuda.Stream()
    # launch settings chosen by measurement on this GPU (outside the timed region)
    tuning = B.fpcode_autotune_batch(codes, stream, budgets=budgets, reps=2)
    opts = tuning.pop("opts")
    for _ in range(2):
        res = B.fpcode_min_distance_batch(codes, stream, opts=opts, budgets=budgets, want_witness=False)
    torch.cuda.synchronize()
    max_over_ranks(0.0, world)  # barrier
    reps = 3
    t0 = time.perf_counter()
    for _ in range(reps):
        res = B.fpcode_min_distance_batch(codes, stream, opts=opts, budgets=budgets, want_witness=True)
    torch.cuda.synchronize()
    t_batch = max_over_ranks((time.perf_counter() - t0) / reps, world)
    launches = sorted({r.launch for r in res})
    kernel_ms = sum(next(r.t_kernel_ms for r in res if r.launch == L) for L in launches)
    # one launch per code, with the task plan of a single code (min_steps 8)
    one = B.fpcode_opts_default(min_steps=8)
    for c in codes[:8]:
        B.fpcode_min_distance_batch([c], stream, opts=one, budgets=[budget], want_witness=True)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for c in codes:
        B.fpcode_min_distance_batch([c], stream, opts=one, budgets=[budget], want_witness=True)
    torch.cuda.synchronize()
    t_single = max_over_ranks(time.perf_counter() - t0, world)
    certified = int(sum_over_ranks(sum(r.status == B.OK for r in res), world))
    work = int(sum_over_ranks(sum(r.enumerated for r in res), world))
    return {"codes_per_s": len(all_codes) / t_batch, "ms_per_batch": 1e3 * t_batch, "budget_per_code": budget,
            "certified": certified, "budget_limited": len(all_codes) - certified, "codewords": work,
            "kernel_ms": kernel_ms, "launches_per_batch": len(launches),
            "per_code": {"codes_per_s": len(all_codes) / t_single, "ms_total": 1e3 * t_single,
                         "form": "fpcode_min_distance_batch on one code at a time (one launch per code, "
                                 "single-code task plan)"},
            "batched_over_per_code": t_single / t_batch,
            "tuning": tuning,
            "timing": "end to end from host matrices (host preparation on all cores, H2D, launches, D2H), "
                      f"mean of {reps} batches",
            "shard": "the 512 codes split into contiguous blocks, one per rank" if world > 1 else "one GPU"}


def serve_measure(args, torch, B, n_req=None) -> dict:
    """Continuous batching of Poisson arrivals; latency from arrival to result."""
    from paper_2603_29942_gb300 import inputs

    codes, arrivals = inputs.serve_codes()
    n_req = min(n_req or args.requests, len(codes))
    codes, arrivals = codes[:n_req], arrivals[:n_req]
    budget = int(args.budget)
    stream = torch.cuda.Stream()
    srv = B.fpcode_serve_create(B.fpcode_serve_opts_default(slots=128), stream)
    for c in codes[:8]:  # warm-up: a few codes through the server
        B.fpcode_serve_submit(srv, c, budget=budget)
    B.fpcode_serve_drain(srv)
    B.fpcode_serve_poll(srv)
    relaunch0 = B.fpcode_serve_launches(srv)
    pending = list(range(n_req))
    ticket_of, done_at, results = {}, {}, {}
    t0 = time.perf_counter()
    while len(done_at) < n_req:
        now = time.perf_counter() - t0
        while pending and arrivals[pending[0]] <= now:
            i = pending[0]
            t = B.fpcode_serve_submit(srv, codes[i], budget=budget)
            if t is None:
                break  # no slot or memory free: the request waits (its latency runs)
            ticket_of[t] = i
            pending.pop(0)
        for t, r in B.fpcode_serve_poll(srv, want_witness=False):
            i = ticket_of.pop(t)
            done_at[i] = time.perf_counter() - t0
            results[i] = r
        if not pending and not ticket_of:
            break
        time.sleep(0.00005)  # the client's poll interval (50 us)
    elapsed = time.perf_counter() - t0
    launches = B.fpcode_serve_launches(srv) - relaunch0
    B.fpcode_serve_destroy(srv)
    lat = sorted((done_at[i] - arrivals[i]) * 1e3 for i in done_at)
    pct = lambda q: lat[min(len(lat) - 1, int(q * len(lat)))]
    return {"codes_per_s": n_req / elapsed, "requests": n_req, "seconds": elapsed, "budget_per_code": budget,
            "certified": sum(r.status == B.OK for r in results.values()), "arrival_span_s": float(arrivals[-1]),
            "latency_ms": {"p50": pct(0.50), "p90": pct(0.90), "p99": pct(0.99), "max": lat[-1]},
            "gpu_launches": launches}


# ------------------------------------------------------------ workloads ----

def run_default(args, rank, world, local):
    """The headline single code, with the other configurations as extra keys."""
    from paper_2603_29942_gb300 import inputs

    code = inputs.single(args.workload)
    if args.impl == "reference":
        return run_reference(args, code, rank, world)
    torch, B = _cuda(local)
    dist_init(world, local)
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    sms = torch.cuda.get_device_properties(local).multi_processor_count

    # --- value: device search on resident tables (the timed region) ---
    if world > 1:
        torch.distributed.barrier()
    with ClockSampler(local) as clk:
        head = single_code(args, torch, B, args.workload, stream, flush, world)
        if world > 1:
            torch.distributed.barrier()
    clocks = clk.summary()
    t_ms = max_over_ranks(sum(head["steps_ms"]), world)
    value = world * head["codewords"] * args.steps / (t_ms * 1e-3)
    e2e = e2e_line(torch, B, head["code"], head["prep"], stream, args.steps, world, head["counts_total"])

    # --- roofline of the enumeration kernel (peak measured, at the sampled clock) ---
    peak = popc_peak(B, stream, clocks["sm_mhz"], sms)
    kern_ms = statistics.mean(head["kern_ms"])
    W = head["W"]
    ach = head["codewords"] * W / (kern_ms * 1e-3) / 1e12
    roof = {"bound": "alu", "achieved": ach, "peak": peak["tpopc_s"], "unit": "Tpopc/s", "frac": ach / peak["tpopc_s"],
            "traffic": profiled_traffic(args.workload), "kernel": "bz_kernel", "ops_per_codeword": W,
            "kernel_ms": kern_ms, "peak_basis": peak["basis"], "peak_of": "measured",
            "leaf_form": head["leaf_form"]}
    probe_of = {v[0]: (k, v[1]) for k, v in PROBES.items()}
    roof_probe = None
    if args.workload in probe_of:
        pname, pg = probe_of[args.workload]
        roof_probe = probe_line(torch, B, head["code"], pname, pg, head["res"].d, stream, flush, peak["tpopc_s"])

    line = {
        "metric": "codewords_per_s", "value": value, "unit": "codewords/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": single_config(args.workload, head["res"].d) | {
            "parallelism": "replicas" if world > 1 else "single GPU"},
        "time_to_certified_d_ms": t_ms / args.steps, "codewords_per_step": head["codewords"],
        "schedule_codewords": head["counts_total"],
        "roofline": roof, "roofline_pass_probe": roof_probe, "e2e": e2e,
        "gpu_launches": args.steps, "clocks": clocks,
    }

    # --- the other configurations, each at its stated size ---
    if not args.no_extras:
        extras = {}
        name7 = "f7_n40_k20"
        if args.workload != name7:
            f7 = single_code(args, torch, B, name7, stream, flush, world)
            k7 = statistics.mean(f7["kern_ms"])
            t7 = max_over_ranks(sum(f7["steps_ms"]), world) / args.steps
            a7 = f7["codewords"] * f7["W"] / (k7 * 1e-3) / 1e12
            extras[name7] = {
                "d": f7["res"].d, "time_to_certified_d_ms": t7, "kernel_ms": k7,
                "codewords_per_step": f7["codewords"], "codewords_per_s": world * f7["codewords"] / (t7 * 1e-3),
                "roofline": {"bound": "alu", "achieved": a7, "peak": peak["tpopc_s"], "unit": "Tpopc/s",
                             "frac": a7 / peak["tpopc_s"], "traffic": profiled_traffic(name7),
                             "ops_per_codeword": f7["W"], "leaf_form": f7["leaf_form"]},
                "roofline_pass_probe": probe_line(torch, B, f7["code"], "probe_f7_n40_k20_g7", 7, f7["res"].d, stream,
                                                  flush, peak["tpopc_s"]),
                "gpu_launches": args.steps}
        extras["batch512"] = batch_measure(args, torch, B, rank, world)
        if rank == 0:
            extras["serve"] = serve_measure(args, torch, B)
        line["extras"] = extras
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(head["code"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_probe(args, rank, world, local):
    """Kernel efficiency on one pass of fixed, closed-form size (no early
    termination): the pass runs alone, every task to the end, with the record
    threshold a certified search has at that level (U = d)."""
    from paper_2603_29942_gb300 import inputs

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle is timed on the certified "
                              "single-code searches; a single pass has no reference arm"}))
        return
    from paper_2603_29942_gb300 import inputs

    torch, B = _cuda(local)
    name, g = PROBES[args.workload]
    code = inputs.single(name)
    stream = torch.cuda.Stream()
    flush = torch.empty(FLUSH_BYTES, dtype=torch.uint8, device="cuda")
    d = B.fpcode_min_distance_ex(B.fpcode_prepare(code.p, code.n, code.k, code.G), stream).d
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    with ClockSampler(local) as clk:
        pr = probe_prepare(B, code)
        passes = B.fpcode_prepared_passes(pr)
        idx = next(i for i, x in enumerate(passes) if x[0] == g and x[1] == 0)
        size = passes[idx][5]
        t_ms, kern_ms, least = time_pass(torch, B, pr, idx, d, stream, args.steps, args.warmup, flush)
    clocks = clk.summary()
    peak = popc_peak(B, stream, clocks["sm_mhz"], sms)
    W = max(1, -(-(code.n - code.k) // 32))
    achieved = size * W / (kern_ms * 1e-3) / 1e12
    line = {
        "metric": "codewords_per_s", "value": world * size * args.steps / (t_ms * 1e-3), "unit": "codewords/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "pass": [g, 0],
                   "codewords_per_step": size, "u_seed": d, "least_weight_in_pass": least,
                   "l2": "flushed between timed steps (256 MiB memset)", "parallelism": "single GPU"},
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak["tpopc_s"], "unit": "Tpopc/s",
                     "frac": achieved / peak["tpopc_s"], "traffic": profiled_traffic(args.workload),
                     "kernel": "bz_kernel", "ops_per_codeword": W, "peak_basis": peak["basis"], "peak_of": "measured"},
        "gpu_launches": args.steps,
        "clocks": clocks,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_batch(args, rank, world, local):
    """512 codes: persistent batched launches vs one launch per code."""
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle is timed on the single-code "
                              "workloads only; batch512 has no reference arm"}))
        return
    torch, B = _cuda(local)
    dist_init(world, local)
    with ClockSampler(local) as clk:
        b = batch_measure(args, torch, B, rank, world)
    line = {
        "metric": "codes_per_s", "value": b["codes_per_s"], "unit": "codes/s", "n_gpus": world, "steps": 3,
        "warmup": 2, "ms_per_step": b["ms_per_batch"], "higher_is_better": True,
        "scaling": "strong" if world > 1 else "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "batch512", "description": WORKLOADS["batch512"]},
        "batch512": b, "batched_over_per_code": b["batched_over_per_code"],
        "gpu_launches": 3 * b["launches_per_batch"], "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)


def run_serve(args, rank, world, local):
    """Continuous batching of Poisson arrivals; latency from arrival to result."""
    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle is timed on the single-code "
                              "workloads only; serve has no reference arm"}))
        return
    if rank != 0:
        return  # one request stream, served by one GPU (the other ranks hold none)
    torch, B = _cuda(local)
    with ClockSampler(local) as clk:
        s = serve_measure(args, torch, B)
    line = {
        "metric": "codes_per_s", "value": s["codes_per_s"], "unit": "codes/s", "n_gpus": 1,
        "steps": 1, "warmup": 1, "ms_per_step": 1e3 * s["seconds"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": "serve", "description": WORKLOADS["serve"], "requests": s["requests"],
                   "budget_per_code": s["budget_per_code"]},
        "serve": s, "latency_ms": s["latency_ms"], "gpu_launches": s["gpu_launches"], "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def run_split(args, rank, world, local):
    """One search split over the ranks (paper_2603_29942_gb300.shard): each
    pass's tasks in contiguous ranges, one allreduce-min of the packed key per
    pass (NCCL).  Strong scaling: the work of one search over all ranks."""
    from paper_2603_29942_gb300 import inputs, shard

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle is timed on the single-code "
                              "workloads; the split search has no reference arm"}))
        return
    torch, B = _cuda(local)
    dist_init(world, local)
    code = inputs.single("f3_n80_k40")
    stream = torch.cuda.Stream()
    device = torch.device("cuda", local) if world > 1 else None
    ref = B.fpcode_min_distance_ex(B.fpcode_prepare(code.p, code.n, code.k, code.G), stream)
    mn, sm = shard.torch_reducers(device) if world > 1 else ((lambda x: x), (lambda x: x))
    prep = B.fpcode_prepare(code.p, code.n, code.k, code.G)
    B.fpcode_prepared_upload(prep, stream)
    sched = B.fpcode_prepared_schedule(prep)
    gpu = shard.GpuSlices(B, prep, stream)

    def one():
        return shard.split_search(sched, n=code.n, k=code.k, per_round_check=False, complete=True, rank=rank,
                                  world=world, search_slice=gpu, min_over_ranks=mn, sum_over_ranks=sm)

    for _ in range(args.warmup):
        r = one()
    assert r.d == ref.d and r.counts == ref.counts
    max_over_ranks(0.0, world)
    with ClockSampler(local) as clk:
        t0 = time.perf_counter()
        for _ in range(args.steps):
            r = one()
        torch.cuda.synchronize()
        dt = max_over_ranks(time.perf_counter() - t0, world)
    line = {
        "metric": "codewords_per_s", "value": sum(r.counts) * args.steps / dt, "unit": "codewords/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "description": WORKLOADS[args.workload], "d": r.d,
                   "passes": r.npasses, "parallelism": f"one search split over {world} rank(s)",
                   "timing": "host clock around whole searches (per pass: slice upload, search, read-back, allreduce)"},
        "gpu_launches": args.steps * r.npasses, "clocks": clk.summary(),
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def run_additions(args, rank, world, local):
    """The additions benchmark of Sec. 5.1 on the GPU: two sets of 10 000
    vectors of 512 symbols added pairwise 10 000 times (a dependent chain),
    bit-sliced against one symbol per byte."""
    import numpy as np

    if args.impl == "reference":
        if rank == 0:
            print(json.dumps({"impl": "reference", "unavailable": "the CPU oracle is timed on the certified "
                              "single-code searches; the additions benchmark has no reference arm"}))
        return
    if rank != 0:
        return
    torch, B = _cuda(local)
    p = ADDITIONS[args.workload]
    nvec, nsym, reps = 10_000, 512, 10_000
    rng = np.random.default_rng(5)
    a = rng.integers(0, p, size=(nvec, nsym), dtype=np.uint8)
    b = rng.integers(0, p, size=(nvec, nsym), dtype=np.uint8)
    want = ((a.astype(np.int64) + reps * b.astype(np.int64)) % p).astype(np.uint8)
    rates, times = {}, {}
    steps = max(1, min(args.steps, 5))
    with ClockSampler(local) as clk:
        for form, sliced in (("sliced", True), ("bytes", False)):
            B.fpcode_bench_additions(p, a[:64], b[:64], 10, sliced)  # warm-up
            ms = []
            for _ in range(steps):
                out, t = B.fpcode_bench_additions(p, a, b, reps, sliced)
                assert np.array_equal(out, want)
                ms.append(t)
            times[form] = statistics.median(ms)
            rates[form] = nvec * nsym * reps / (times[form] * 1e-3)
    line = {
        "metric": "symbol_additions_per_s", "value": rates["sliced"], "unit": "symbol additions/s", "n_gpus": 1,
        "steps": steps, "warmup": 1, "ms_per_step": times["sliced"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": args.workload, "p": p, "vectors": nvec, "symbols": nsym, "repetitions": reps,
                   "form": "bit-sliced natural encoding, 32 symbols per word and slice; repetitions chained",
                   "bytes_form_ms": times["bytes"], "bytes_form_symbol_additions_per_s": rates["bytes"],
                   "sliced_over_bytes": times["bytes"] / times["sliced"], "checked": "a + reps*b mod p, every symbol"},
        "gpu_launches": 2 * steps,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="f3_n80_k40", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="leave the other configurations out of the default line")
    ap.add_argument("--budget", type=float, default=1e8, help="per-code budget (batch512, serve)")
    ap.add_argument("--requests", type=int, default=10000, help="requests served (serve)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)

    rank, world, local = dist_env()
    if args.workload == "batch512":
        return run_batch(args, rank, world, local)
    if args.workload in PROBES:
        return run_probe(args, rank, world, local)
    if args.workload in ADDITIONS:
        return run_additions(args, rank, world, local)
    if args.workload == "serve":
        return run_serve(args, rank, world, local)
    if args.workload == "f3_n80_k40_split":
        return run_split(args, rank, world, local)
    return run_default(args, rank, world, local)


if __name__ == "__main__":
    main()
