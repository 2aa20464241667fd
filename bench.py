"""Benchmark: exact stabilizer-term sums on GB300.

One step = one full exact amplitude of the large workload (n = 50 qubits,
2000 gates with 80 T gates, seeded random output bitstring): the compiled
scalar's inner table (the sum over its inner parameters, built on the GPU)
and the Gray-code walk over all of its outer parameters, result on the
device (value, amplitudes/s), or one request through the public host API
from the scalar's table bytes to the exact result on the host (e2e).  The
circuit is reduced to the scalar once, before timing.  Secondary lines: the
medium workload (n = 20, 600 gates, 40 T), the unsplit n = 50 / T = 50 sum
(k = 37), a batch of 512 circuits, Poisson-arrival serving, the paper's
parametric use, and the integer-throughput microbenchmark.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  With N > 1 (torchrun) every rank sums its own
copy of the workload: independent amplitudes, no collective on the data path
(weak scaling); the timed region is bracketed by barriers and the slowest
rank's time is used.
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

METRIC = "exact stabilizer terms/sec and amplitudes/sec (fraction of INT roofline)"
ISSUE_LANES_PER_SM_CLK = 4 * 32       # 4 schedulers x 1 warp-instruction x 32 lanes per clock
LARGE_TABLES = os.path.join(ROOT, "zxp_inputs", "tables", "large_n50_g2000_t80_seed0.zxps")


class ClockSampler:
    """nvidia-smi samples during the timed region (clocks, throttle reasons)."""
    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "20"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 8:
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if "Active" in r[4 + i]
                          and "Not" not in r[4 + i]})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


# the sources that decide a profiled kernel's code and the tables it reads
# from a scalar (the scalar itself is pinned by the digest of its table
# bytes, scalar_sha256)
KERNEL_SOURCES = ("sum_kernel.cuh", "kernel_core.cuh", "kernel.cu", "kernel_count.cu", "zring.h",
                  "plan.h", "plan.cpp")
INNER_SOURCES = ("inner.cu", "zring.h", "plan.h", "plan.cpp")


def kernel_source_sha(sources=KERNEL_SOURCES) -> str:
    """Hash of the sources that decide the sum kernel's code and tables
    (or, with INNER_SOURCES, the inner table's)."""
    h = hashlib.sha256()
    for f in sources:
        h.update(open(os.path.join(ROOT, "paper_2403_06777_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def tables_sha(*blobs: bytes) -> str:
    """Digest of the table bytes of the scalars a profile ran on."""
    h = hashlib.sha256()
    for b in blobs:
        h.update(b)
    return h.hexdigest()


def profile_fields(kernel_src_sha: str, name: str = "sum_kernel_medium.txt", scalar_sha: str | None = None):
    """Fields of a committed ncu summary, if it was taken on the current
    kernel sources and (scalar_sha) on the same scalar (else None)."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    fields = {}
    for line in open(path):
        if ":" in line:
            k, v = line.split(":", 1)
            fields[k.strip()] = v.strip()
    if fields.get("kernel_source_sha256") != kernel_src_sha:
        return None
    if scalar_sha is not None and fields.get("scalar_sha256") != scalar_sha:
        return None
    return fields


def profile_number(fields, key):
    try:
        return float(fields[key].split()[0]) if fields else None
    except (KeyError, ValueError, IndexError):
        return None


def cpu_baseline(blob: bytes, terms_per_amp: int, seconds: float = 10.0):
    """The oracle as it stands, on the host cores: all threads and one
    thread, each on a bounded sample of the same scalar (whole outer terms,
    every inner value of each), scaled to amplitudes/s by the stabilizer
    terms of one amplitude."""
    import oracle
    cores = os.cpu_count() or 1
    inner = terms_per_amp >> oracle.outer_k(blob)

    def rate(threads, budget):
        n = 1
        while True:
            t = time.perf_counter()
            oracle.ps_sum(blob, 0, n, nthreads=threads)
            dt = time.perf_counter() - t
            if dt >= budget * 0.6 or n >= (1 << oracle.outer_k(blob)):
                return n * inner / dt, n, dt
            n *= max(2, min(64, int(budget / max(dt, 1e-4))))
            n = min(n, 1 << oracle.outer_k(blob))

    v_all, n_all, dt_all = rate(cores, seconds)
    v_one, n_one, dt_one = rate(1, seconds / 3)
    return {"value": v_all / terms_per_amp, "unit": "amplitudes/s", "cores": cores, "kind": "oracle",
            "stabilizer_terms_per_s": v_all,
            "single_thread": {"value": v_one / terms_per_amp, "unit": "amplitudes/s",
                              "stabilizer_terms_per_s": v_one, "cores": 1,
                              "sample": f"{n_one} outer terms x {inner} inner values, {dt_one:.1f} s"},
            "sample": f"outer Gray-index range [0, {n_all}) of the same scalar, every one of the "
                      f"{inner} inner values of each ({n_all * inner} stabilizer terms), {dt_all:.1f} s "
                      f"on {cores} host threads; amplitudes/s = stabilizer terms/s / {terms_per_amp}"}


SERVE_MAX_K = 38


def serve_run(Z, ctx, reqs, policy, max_k, **opts):
    """Replay the arrivals against one server (zxp_server_opts fields in
    opts); per-request latency is the library's own submit-to-value time."""
    srv = Z.zxp_server_create(ctx, policy=policy, max_k=max_k, **opts)
    warm = [Z.zxp_server_submit(srv, r["gb"], r["n"], r["bits"], marg_mask=r["mask"],
                                kind=r["kind"]) for r in reqs[:16]]
    for t in warm:
        Z.zxp_server_poll(srv, t, -1)
    tickets = []
    t0 = time.perf_counter()
    for r in reqs:
        target = t0 + r["t"]
        while True:
            now = time.perf_counter()
            if now >= target:
                break
            if target - now > 6e-4:
                time.sleep(target - now - 5e-4)
        tickets.append(Z.zxp_server_submit(srv, r["gb"], r["n"], r["bits"],
                                           marg_mask=r["mask"], kind=r["kind"]))
    res = [Z.zxp_server_poll(srv, t, -1) for t in tickets]
    st = Z.zxp_server_stats(srv)
    srv.close()
    ok = [(v, tm) for rc, v, tm in res if rc == Z.ZXP_OK]
    lat = sorted((tm["done_us"] - tm["submit_us"]) / 1e3 for _, tm in ok)
    span_s = (max(tm["done_us"] for _, tm in ok) - min(tm["submit_us"] for _, tm in ok)) / 1e6

    def pct(q):
        return lat[min(len(lat) - 1, int(q * len(lat)))]

    out = {"p50_ms": pct(0.50), "p90_ms": pct(0.90), "p99_ms": pct(0.99), "max_ms": lat[-1],
           "amplitudes_per_s": len(ok) / span_s, "completed": len(ok),
           "rejected_k": sum(1 for rc, _, _ in res if rc == Z.ZXP_ETOOBIG),
           "other_errors": sum(1 for rc, _, _ in res if rc not in (Z.ZXP_OK, Z.ZXP_ETOOBIG)),
           "steps": st["steps"], "launches": st["launches"],
           "terms": st["terms"], "device_busy_ms": st["device_busy_us"] / 1e3,
           "peak_active": st["peak_active"]}
    return out, [v for rc, v, _ in res]


SERVE_P99_SLO_MS = 20.0
SERVE_SWEEP_HZ = (2000.0, 5000.0, 10000.0, 20000.0, 50000.0)


def serve_bench(Z, ctx, zi, n_req: int, rate_hz: float, max_k: int, sweep=SERVE_SWEEP_HZ):
    reqs = zi.serve_requests(0, n_req, rate_hz)
    for r in reqs:
        r["gb"] = zi.pack_gates(r["gates"])
    # one untimed pass of each policy over the whole mix: the first launch of
    # every kernel variant loads its code (lazy module loading), which would
    # otherwise land inside the first measured steps
    serve_run(Z, ctx, reqs, Z.ZXP_SERVE_BATCHED, max_k)
    serve_run(Z, ctx, reqs, Z.ZXP_SERVE_PLAIN, max_k)
    batched, vb = serve_run(Z, ctx, reqs, Z.ZXP_SERVE_BATCHED, max_k)
    plain, vp = serve_run(Z, ctx, reqs, Z.ZXP_SERVE_PLAIN, max_k)
    assert vb == vp, "served values differ between policies"
    # arrival-rate sweep: the same request mix offered faster; a policy keeps
    # up at a rate when it completes within 10 % of the offered rate with p99
    # under the SLO; the knee is the highest such rate of the sweep
    rows, knee = [], {}
    for hz in sweep:
        rq = zi.serve_requests(0, n_req, hz)
        for r in rq:
            r["gb"] = zi.pack_gates(r["gates"])
        row = {"offered_hz": hz}
        for name, pol in (("batched", Z.ZXP_SERVE_BATCHED), ("plain", Z.ZXP_SERVE_PLAIN)):
            o, _ = serve_run(Z, ctx, rq, pol, max_k)
            ok = o["amplitudes_per_s"] >= 0.9 * hz and o["p99_ms"] <= SERVE_P99_SLO_MS
            row[name] = {"amplitudes_per_s": o["amplitudes_per_s"], "p50_ms": o["p50_ms"],
                         "p99_ms": o["p99_ms"], "device_busy_ms": o["device_busy_ms"], "keeps_up": ok}
            if ok:
                knee[name] = max(knee.get(name, 0.0), hz)
        rows.append(row)
    return {"workload": f"{n_req} requests, Poisson {rate_hz:.0f}/s, seed 0: amplitude and "
                        "single-qubit doubled-marginal, n~U[10,50], T~U[10,70]",
            "admission_max_k": max_k, "batched": batched,
            "plain_one_scalar_per_launch": plain,
            "device_busy_batched_over_plain": batched["device_busy_ms"] / plain["device_busy_ms"],
            "p99_plain_over_batched": plain["p99_ms"] / batched["p99_ms"],
            "sweep": rows, "p99_slo_ms": SERVE_P99_SLO_MS,
            "knee_hz": {"batched": knee.get("batched"), "plain": knee.get("plain")}}


def param_bench(Z, ctx, zi, n_values=(1, 4, 16, 64, 256, 1024), seed=0):
    """The paper's own use: one parametric reduction of the medium circuit
    (all 20 output bits parameters), N random bitstrings bound and evaluated
    through the server, against N fixed-bit compiles through the same server.
    S_N = T_plain(N) / T_param(N); T_param includes the one reduction."""
    import random
    w = zi.workload_medium(seed)
    t0 = time.perf_counter()
    ps = Z.zxp_compile_param(w.gates, w.n, [0] * w.n, list(range(w.n)))
    t_reduce = time.perf_counter() - t0
    gb = zi.pack_gates(w.gates)
    rng = random.Random(1234)
    srv = Z.zxp_server_create(ctx)
    # warm-up: kernels' first launches, worker threads
    for t in [Z.zxp_server_submit_bind(srv, ps, 0), Z.zxp_server_submit(srv, gb, w.n, [0] * w.n)]:
        Z.zxp_server_poll(srv, t, -1)
    rows = []
    for N in n_values:
        bs = [rng.getrandbits(w.n) for _ in range(N)]
        t0 = time.perf_counter()
        tk = [Z.zxp_server_submit_bind(srv, ps, b) for b in bs]
        vp = [Z.zxp_server_poll(srv, t, -1)[1] for t in tk]
        t_param = t_reduce + (time.perf_counter() - t0)
        t0 = time.perf_counter()
        tk = [Z.zxp_server_submit(srv, gb, w.n, [(b >> q) & 1 for q in range(w.n)]) for b in bs]
        vc = [Z.zxp_server_poll(srv, t, -1)[1] for t in tk]
        t_plain = time.perf_counter() - t0
        assert vp == vc, "bound and fixed-bit values differ"
        rows.append({"N": N, "param_s": t_param, "plain_s": t_plain, "S_N": t_plain / t_param})
    srv.close()
    # the same plain path with one compile thread (the paper's baseline reduces
    # each bitstring on one core); the parametric path's binding is cheap
    # enough that its thread count does not matter
    srv1 = Z.zxp_server_create(ctx, compile_threads=1)
    one = []
    for N in (16, 128):
        bs = [rng.getrandbits(w.n) for _ in range(N)]
        t0 = time.perf_counter()
        tk = [Z.zxp_server_submit(srv1, gb, w.n, [(b >> q) & 1 for q in range(w.n)]) for b in bs]
        for t in tk:
            Z.zxp_server_poll(srv1, t, -1)
        one.append((N, time.perf_counter() - t0))
    srv1.close()
    plain1_per_eval = (one[1][1] - one[0][1]) / (one[1][0] - one[0][0])
    # terminal speedup: ratio of the marginal per-evaluation costs of the two
    # largest N; inflection: the N where S_N reaches half of it (log interpolation)
    a, b = rows[-2], rows[-1]
    s_inf = (b["plain_s"] - a["plain_s"]) / max(1e-9, b["param_s"] - a["param_s"])
    n_inf = None
    for r0, r1 in zip(rows, rows[1:]):
        if r0["S_N"] < s_inf / 2 <= r1["S_N"]:
            import math
            f = (s_inf / 2 - r0["S_N"]) / (r1["S_N"] - r0["S_N"])
            n_inf = math.exp(math.log(r0["N"]) + f * (math.log(r1["N"]) - math.log(r0["N"])))
    if n_inf is None and rows[0]["S_N"] >= s_inf / 2:
        n_inf = rows[0]["N"]
    info = Z.zxp_pscalar_info(ps)
    return {"workload": f"{w.name} seed={seed}: all {w.n} output bits parameters, random bitstrings",
            "k_param": info["k"], "k_fixed": Z.zxp_scalar_info(Z.zxp_compile(w.gates, w.n, w.out_bits))["k"],
            "reduce_ms": t_reduce * 1e3, "rows": rows, "S_inf": s_inf, "N_inflec": n_inf,
            "param_ms_per_eval": 1e3 * (b["param_s"] - a["param_s"]) / (b["N"] - a["N"]),
            "plain_ms_per_eval": 1e3 * (b["plain_s"] - a["plain_s"]) / (b["N"] - a["N"]),
            "plain_1thread_ms_per_eval": plain1_per_eval * 1e3,
            "S_inf_vs_1thread": plain1_per_eval / ((b["param_s"] - a["param_s"]) / (b["N"] - a["N"])),
            "plain": "fixed-bit compile of each bitstring on the server's compile workers "
                     "(all host threads; 1thread: one worker), same GPU path"}


def free_port() -> int:
    import socket
    with socket.socket() as so:
        so.bind(("127.0.0.1", 0))
        return so.getsockname()[1]


def setup_dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """The oracle on the host cores on the headline workload's scalar (the
    committed table bytes of the compiled large circuit): each step sums a
    bounded sample of whole outer terms, every inner value of each, and the
    rate is scaled to amplitudes/s by the stabilizer terms of one amplitude."""
    if rank != 0:
        return
    import oracle
    blob = open(LARGE_TABLES, "rb").read()
    k = int.from_bytes(blob[8:12], "little")
    ko = oracle.outer_k(blob)
    inner = 1 << (k - ko)
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    oracle.ps_sum(blob, 0, 1, nthreads=cores)
    per_outer = time.perf_counter() - t
    total_budget = 150.0
    n = max(1, int(total_budget / max(1, args.steps + args.warmup) / per_outer))
    for i in range(args.warmup):
        oracle.ps_sum(blob, 0, n, nthreads=cores)
    t = time.perf_counter()
    for i in range(args.steps):
        first = (i * n) % ((1 << ko) - n + 1)
        oracle.ps_sum(blob, first, n, nthreads=cores)
    dt = time.perf_counter() - t
    stab = n * inner * args.steps / dt
    v = stab / (1 << k)
    sample = (f"{n} outer terms x {inner} inner values ({n * inner} of the 2^{k} stabilizer terms "
              f"of one amplitude) per step; amplitudes/s = stabilizer terms/s / 2^{k}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "amplitudes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int128",
        "data": "synthetic",
        "config": {"workload": "large n=50 G=2000 t=80 seed=0: one exact amplitude per step",
                   "k": ko, "k_inner": k - ko, "stabilizer_terms_per_amplitude": 1 << k,
                   "sample": sample},
        "stabilizer_terms_per_s": stab,
        "cpu_baseline": {"value": v, "unit": "amplitudes/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def inner_launches(k_inner: int) -> int:
    """Launches that build an inner table of 32-byte entries (inner.cu):
    the term kernel with the low 11 bits, then passes of at most 11 bits."""
    return 1 + (max(k_inner - 11, 0) + 10) // 11


def inner_roofline(inner_bits: int, k_inner: int, seconds: float, prof):
    """HBM roofline of the inner table: every pass reads and writes the
    table once, the term kernel writes it once (32 bytes per entry)."""
    table = 32 << inner_bits
    passes = inner_launches(k_inner) - 1
    alg = table * (1 + 2 * passes)
    peak = measured_peaks().get("hbm_gbs")
    ach = alg / seconds / 1e9
    return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
            "frac": None if not peak else ach / peak, "algorithmic_bytes": alg,
            "traffic": profile_number(prof, "dram_bytes_per_step"),
            "table_bytes": table, "passes": passes,
            "peak_basis": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
            "source": "profiles/inner_table_large80.txt"}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def issue_peak(torch, dev: int, sm_max_mhz):
    """Integer issue peak (thread instructions/s): SMs x 4 warp-instructions
    per clock x 32 lanes x the SM clock (the maximum that nvidia-smi reports,
    else the device attribute)."""
    props = torch.cuda.get_device_properties(dev)
    sms = props.multi_processor_count
    mhz = sm_max_mhz or getattr(props, "clock_rate", 0) / 1e3 or 2070.0
    return sms * ISSUE_LANES_PER_SM_CLK * mhz * 1e6, sms, mhz


def roofline_from_profile(prof, terms, seconds, peak, source):
    """Issue roofline of a sum-kernel launch from its committed ncu summary:
    measured thread instructions per term x terms / event time / issue peak,
    with the ALU pipe's share of cycles and the DRAM bytes beside it."""
    ipt = profile_number(prof, "instructions_per_term")
    ach = None if ipt is None else ipt * terms / seconds
    return {"bound": "alu", "achieved": None if ach is None else ach / 1e12, "peak": peak / 1e12,
            "unit": "T thread-instr/s", "frac": None if ach is None else ach / peak,
            "traffic": profile_number(prof, "dram_bytes_per_launch"),
            "instructions_per_term": ipt,
            "alu_pipe_frac": profile_number(prof, "alu_pipe_frac"),
            "issue_active_frac": profile_number(prof, "issue_active_frac"),
            "peak_basis": "SMs x 4 warp-instructions/clk x 32 lanes x max SM clock",
            "source": source}


def timed_amplitude(torch, Z, ctx, s, stream, out, flush, steps, sampler_dev):
    """steps full amplitudes of s (inner table, then the whole outer range),
    L2 flushed before each; returns per-step (inner ms, walk ms) and clocks."""
    info = Z.zxp_scalar_info(s)
    terms = 1 << info["k"]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(steps)]
    torch.cuda.synchronize()
    with ClockSampler(sampler_dev) as clk:
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            Z.zxp_inner_sum(ctx, s)
            ev[i][1].record(stream)
            Z.zxp_eval_device(ctx, s, 0, terms, out.data_ptr())
            ev[i][2].record(stream)
        torch.cuda.synchronize()
    inner = [e[0].elapsed_time(e[1]) for e in ev]
    walk = [e[1].elapsed_time(e[2]) for e in ev]
    return inner, walk, clk.summary()


def timed_sharded(torch, Z, dist, ctx, s, stream, flush, steps, world, rank, sampler_dev, ref):
    """steps amplitudes of s, each one sharded over the ranks: every rank
    builds the inner table and walks its share of the outer range
    (dist.shard_range), and the 40-byte raw partials are all-gathered over
    NCCL on the stream (no peer memory in any kernel); returns per-step
    (inner, walk, all-gather) ms and the clocks, after checking that the
    combined last step equals the reference amplitude exactly."""
    from paper_2403_06777_gb300 import dist as zd
    k = Z.zxp_scalar_info(s)["k"]
    first, count = zd.shard_range(k, world, rank)
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    gathered = [torch.empty_like(out) for _ in range(world)]
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(4)] for _ in range(steps)]
    torch.cuda.synchronize()
    dist.barrier()
    with ClockSampler(sampler_dev) as clk:
        for i in range(steps):
            flush.zero_()
            ev[i][0].record(stream)
            Z.zxp_inner_sum(ctx, s)
            ev[i][1].record(stream)
            Z.zxp_eval_device(ctx, s, first, count, out.data_ptr())
            ev[i][2].record(stream)
            dist.all_gather(gathered, out)
            ev[i][3].record(stream)
        torch.cuda.synchronize()
    parts = []
    for g in gathered:
        v = g.tolist()
        parts.append((v[0], v[1], v[2], v[3], v[4] & 0xFFFFFFFF))
    got = Z.zxp_zomega_canon(zd.combine(parts))
    assert got == ref, (got, ref)
    return ([e[0].elapsed_time(e[1]) for e in ev], [e[1].elapsed_time(e[2]) for e in ev],
            [e[2].elapsed_time(e[3]) for e in ev], clk.summary())


def sharded_requests(torch, Z, dist, blob, ctx, n, world, rank, ref):
    """n sharded amplitudes through the public host API; returns seconds per
    amplitude (max over ranks)."""
    from paper_2403_06777_gb300 import dist as zd
    dev = torch.device("cuda", torch.cuda.current_device())
    dist.barrier()
    t = time.perf_counter()
    for _ in range(n):
        s = Z.zxp_scalar_from_tables(blob)
        k = Z.zxp_scalar_info(s)["k"]
        first, count = zd.shard_range(k, world, rank)
        part = Z.zxp_eval(ctx, s, first, count)
        mine = torch.tensor([zd._i64(v) for v in part], dtype=torch.int64).to(dev)
        out = [torch.empty_like(mine) for _ in range(world)]
        dist.all_gather(out, mine)
        got = Z.zxp_zomega_canon(zd.combine([tuple(int(x) for x in o.cpu().tolist()) for o in out]))
        assert got == ref, (got, ref)
    sec = torch.tensor([(time.perf_counter() - t) / n], dtype=torch.float64, device=dev)
    dist.all_reduce(sec, op=dist.ReduceOp.MAX)
    return float(sec.item())


def stream_requests(Z, ctx, blob, n, depth=2):
    """n requests of the scalar with table bytes `blob` through the public
    host API (zxp_submit_tables, zxp_poll), `depth` in flight; returns the
    seconds per request and the results."""
    from collections import deque
    q, got = deque(), []
    t = time.perf_counter()
    for i in range(n + depth):
        if i < n:
            q.append(Z.zxp_submit_tables(ctx, blob))
        if len(q) > depth or (i >= n and q):
            got.append(Z.zxp_poll(ctx, q.popleft(), -1))
    return (time.perf_counter() - t) / n, got


PROFILE_CASES = ("large80", "large80_1g", "inner", "medium", "large37", "peak", "synth36")

# the k = 36 stand-in: synthetic tables with the statistics of compiled
# scalars of k 34-40 (n = 40-50, 1500-2000 gates, T 50-55, 23 scalars:
# 48 linear, 36 quadratic, 10 odd node rows, mask densities 0.10 / 0.14 /
# 0.16, about 0.13 over all masks), drawn order and relabelled
SYNTH36 = dict(seed=3601, k=36, n_lin=48, n_quad=36, n_node=10, odd_nodes_only=True, density=0.13)


def synth36_scalars(Z, zi):
    p = dict(SYNTH36)
    ps = zi.synthetic_ps(p.pop("seed"), p.pop("k"), **p)
    s = Z.zxp_scalar_from_tables(ps.pack())
    return s, Z.zxp_scalar_reorder(s)


def run_profile_case(case: str):
    """A short, fixed launch sequence of one kernel, for capturing it under
    ncu on a small case (--profile):
      large80  the large workload's amplitude (inner table, then the walk over
               all 2^k outer terms), then one walk over 2^28 terms
      large80_1g the same, then one walk over 2^30 terms
      inner    the large workload's amplitude, then its inner table again
      medium   three amplitudes of the medium workload
      large37  one 2^30-term launch of the unsplit n=50 / T=50 scalar (k = 37)
      peak     the integer microbenchmark, every kind once
      synth36  one 2^32-term launch of the k = 36 stand-in, drawn order, then
               relabelled"""
    import torch
    import paper_2403_06777_gb300 as Z
    import zxp_inputs as zi
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = Z.zxp_ctx_create(0, stream.cuda_stream)
    rec = {"profile": case}
    if case in ("large80", "large80_1g", "inner"):
        w = zi.workload_large(0)
        s = Z.zxp_compile(w.gates, w.n, w.out_bits)
        rec["amplitude"] = Z.zxp_amplitude(ctx, s)
        if case == "large80":
            rec["partial"] = Z.zxp_eval(ctx, s, 0, 1 << 28)
        elif case == "large80_1g":
            rec["partial"] = Z.zxp_eval(ctx, s, 0, 1 << 30)
        else:
            Z.zxp_inner_sum(ctx, s)
        rec["info"] = Z.zxp_scalar_info(s)
    elif case == "medium":
        w = zi.workload_medium(0)
        s = Z.zxp_compile(w.gates, w.n, w.out_bits)
        rec["amplitude"] = [Z.zxp_amplitude(ctx, s) for _ in range(3)][-1]
        rec["info"] = Z.zxp_scalar_info(s)
    elif case == "large37":
        w = zi.workload_large_t50(0)
        s = Z.zxp_compile(w.gates, w.n, w.out_bits, split=False)
        rec["partial"] = Z.zxp_eval(ctx, s, 0, 1 << 30)
        rec["info"] = Z.zxp_scalar_info(s)
    elif case == "synth36":
        raw, re = synth36_scalars(Z, zi)
        rec["variants"] = [raw.info["kernel_variant"], re.info["kernel_variant"]]
        rec["partials"] = [Z.zxp_eval(ctx, raw, 0, 1 << 32), Z.zxp_eval(ctx, re, 0, 1 << 32)]
    else:
        rec["int_peak"] = {kind: Z.zxp_int_peak(ctx, kind) for kind in range(5)}
    torch.cuda.synchronize()
    ctx.close()
    print(json.dumps(rec))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shard", action="store_true",
                    help="strong scaling: every amplitude's outer range split over the ranks")
    ap.add_argument("--profile", choices=PROFILE_CASES, help="run one kernel's short launch sequence")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = setup_dist()
    if args.profile:
        run_profile_case(args.profile)
        return

    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import paper_2403_06777_gb300 as Z
    import zxp_inputs as zi

    torch.cuda.set_device(local)
    dist = None
    if world > 1 or args.shard:
        import torch.distributed as dist
        if world == 1:   # one rank of its own (the sharded path with N = 1)
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            os.environ.setdefault("MASTER_PORT", str(free_port()))
            os.environ.setdefault("RANK", "0")
            os.environ.setdefault("WORLD_SIZE", "1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # a dedicated stream: the library launches on it and the CUDA events are
    # recorded on it (torch's legacy default stream has handle 0, which the
    # C ABI reads as "create your own stream")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = Z.zxp_ctx_create(local, stream.cuda_stream)
    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    # ---- headline: the large workload, one exact amplitude per step --------
    w = zi.workload_large(args.seed)
    t0 = time.perf_counter()
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    compile_ms = (time.perf_counter() - t0) * 1e3
    info = Z.zxp_scalar_info(s)
    k, ki = info["k"], info["k_inner"]
    terms = 1 << k
    stab_terms = 1 << (k + ki)
    blob = Z.zxp_scalar_to_tables(s)
    ref = Z.zxp_amplitude(ctx, s)
    for _ in range(args.warmup):
        Z.zxp_inner_sum(ctx, s)
        Z.zxp_eval_device(ctx, s, 0, terms, out.data_ptr())
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    wall0 = time.perf_counter()
    gather_ms = []
    walked = terms   # outer terms one rank walks per step
    if args.shard:
        from paper_2403_06777_gb300 import dist as zd
        walked = zd.shard_range(k, world, rank)[1]
        inner_ms, walk_ms, gather_ms, clocks = timed_sharded(torch, Z, dist, ctx, s, stream, flush, args.steps,
                                                             world, rank, local, ref)
    else:
        inner_ms, walk_ms, clocks = timed_amplitude(torch, Z, ctx, s, stream, out, flush, args.steps, local)
    wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    if not args.shard:
        # the device result of the last step must be the exact amplitude
        r = out.tolist()
        got = Z.zxp_zomega_canon((r[0], r[1], r[2], r[3], r[4] & 0xFFFFFFFF))
        assert got == ref, (got, ref)
    step_ms = sum(inner_ms) + sum(walk_ms) + sum(gather_ms)
    t_rank = torch.tensor([step_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t_rank, op=dist.ReduceOp.MAX)
    step_ms = float(t_rank.item())
    sec = step_ms / 1e3
    # replicas: every rank one amplitude per step; sharded: one per step in all
    value = args.steps / sec if args.shard else args.steps * world / sec
    walk_s = statistics.median(walk_ms) / 1e3
    inner_s = statistics.median(inner_ms) / 1e3

    # e2e: the public host API, one request per step: the scalar's table
    # bytes (host) are submitted (zxp_submit_tables: the scalar is built on
    # the host, its tables copied from pinned staging, the inner table built
    # and the walk launched on the device) and polled (the 40-byte result the
    # kernel wrote into pinned host memory); two requests in flight.  Every
    # result is checked after the timed loop.
    E2E_DEPTH = 2
    e2e_steps = max(20, args.steps)
    if args.shard:
        # sharded, through the public API: the scalar from its table bytes
        # (host), this rank's range summed to a host result (zxp_eval), the
        # 40-byte partials exchanged over NCCL and combined on the host
        e2e_sec = sharded_requests(torch, Z, dist, blob, ctx, e2e_steps, world, rank, ref)
        E2E_DEPTH = 1
    else:
        stream_requests(Z, ctx, blob, 3, E2E_DEPTH)
        torch.cuda.synchronize()
        e2e_sec, got = stream_requests(Z, ctx, blob, e2e_steps, E2E_DEPTH)
        bad = sum(Z.zxp_zomega_canon(x) != ref for x in got)
        assert bad == 0 and len(got) == e2e_steps, (bad, len(got))

    # ---- integer microbenchmark (the measured peak beside the issue peak) ----
    int_peak = None
    if rank == 0:
        int_peak = {}
        for kind, name in enumerate(("lop3", "add", "popc", "mad", "lop3_mad")):
            v, ms = Z.zxp_int_peak(ctx, kind)
            int_peak[name] = {"thread_instr_per_s": v, "ms": ms}

    # ---- medium workload: one launch per amplitude ---------------------------
    medium = None
    if rank == 0 and not os.environ.get("ZXP_BENCH_SKIP_MEDIUM"):
        wm = zi.workload_medium(args.seed)
        sm_ = Z.zxp_compile(wm.gates, wm.n, wm.out_bits)
        im = Z.zxp_scalar_info(sm_)
        nm = 1 << im["k"]
        refm = Z.zxp_amplitude(ctx, sm_)
        for _ in range(20):
            Z.zxp_eval_device(ctx, sm_, 0, nm, out.data_ptr())
        steps_m = 2000
        st_ = [torch.cuda.Event(enable_timing=True) for _ in range(steps_m)]
        sp_ = [torch.cuda.Event(enable_timing=True) for _ in range(steps_m)]
        torch.cuda.synchronize()
        for i in range(steps_m):
            flush.zero_()
            st_[i].record(stream)
            Z.zxp_eval_device(ctx, sm_, 0, nm, out.data_ptr())
            sp_[i].record(stream)
        torch.cuda.synchronize()
        ms_m = sum(a.elapsed_time(b) for a, b in zip(st_, sp_)) / steps_m
        r = out.tolist()
        assert Z.zxp_zomega_canon((r[0], r[1], r[2], r[3], r[4] & 0xFFFFFFFF)) == refm
        blob_m = Z.zxp_scalar_to_tables(sm_)
        e2e_m, gm = stream_requests(Z, ctx, blob_m, 2000)
        assert all(Z.zxp_zomega_canon(x) == refm for x in gm)
        peak_m, _, _ = issue_peak(torch, local, clocks.get("sm_max_mhz"))
        medium = {"workload": f"{wm.name} seed={args.seed}: one exact amplitude per step, L2 flushed",
                  "k": im["k"], "terms": nm, "ms_per_amplitude": ms_m,
                  "amplitudes_per_s": 1e3 / ms_m, "terms_per_s": nm / (ms_m / 1e3),
                  "kernel_variant": im["kernel_variant"],
                  "e2e": {"amplitudes_per_s": 1 / e2e_m, "us_per_request": e2e_m * 1e6,
                          "h2d_bytes_per_step": im["upload_bytes"], "d2h_bytes_per_step": 40,
                          "requests_in_flight": 2},
                  "roofline": roofline_from_profile(profile_fields(kernel_source_sha(), "sum_kernel_medium.txt",
                                                                  tables_sha(blob_m)),
                                                    nm, ms_m / 1e3, peak_m, "profiles/sum_kernel_medium.txt")}

    # ---- the k = 36 stand-in with compiled statistics, drawn and relabelled ---
    synth = None
    if rank == 0 and not os.environ.get("ZXP_BENCH_SKIP_LARGE"):
        raw, re = synth36_scalars(Z, zi)
        sprof = profile_fields(kernel_source_sha(), "sum_kernel_synthetic36.txt",
                               tables_sha(Z.zxp_scalar_to_tables(raw), Z.zxp_scalar_to_tables(re)))
        synth = {"workload": "synthetic k=36 tables with compiled k 34-40 statistics " + json.dumps(SYNTH36)}
        for tag, sc, n in (("drawn_order", raw, 1 << 34), ("relabelled", re, 1 << 36)):
            Z.zxp_eval_device(ctx, sc, 0, 1 << 24, out.data_ptr())
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            Z.zxp_eval_device(ctx, sc, 0, n, out.data_ptr())
            b.record(stream)
            torch.cuda.synchronize()
            ms = a.elapsed_time(b)
            synth[tag] = {"kernel_variant": sc.info["kernel_variant"], "terms": n, "ms": ms,
                          "terms_per_s": n / (ms / 1e3),
                          "instructions_per_term": profile_number(sprof, "instructions_per_term_" + tag)}
        # relabelling keeps the sum: the full sum of both orders
        synth["same_full_sum"] = Z.zxp_zomega_canon(Z.zxp_eval(ctx, raw)) == Z.zxp_zomega_canon(Z.zxp_eval(ctx, re))
        assert synth["same_full_sum"]

    # ---- the unsplit sum kernel at k = 37 (n = 50, 2000 gates, T = 50) -------
    unsplit = None
    if rank == 0 and not os.environ.get("ZXP_BENCH_SKIP_LARGE"):
        wl = zi.workload_large_t50(0)
        sl = Z.zxp_compile(wl.gates, wl.n, wl.out_bits, split=False)
        il = Z.zxp_scalar_info(sl)
        nl = 1 << il["k"]
        Z.zxp_eval_device(ctx, sl, 0, min(nl, 1 << 30), out.data_ptr())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with ClockSampler(local) as clkl:
            a.record(stream)
            Z.zxp_eval_device(ctx, sl, 0, nl, out.data_ptr())
            b.record(stream)
            torch.cuda.synchronize()
        msl = a.elapsed_time(b)
        peak_l, _, _ = issue_peak(torch, local, clkl.summary().get("sm_max_mhz"))
        unsplit = {"workload": f"{wl.name} seed=0 without the split: one exact amplitude, one launch",
                   "k": il["k"], "terms": nl, "ms": msl, "terms_per_s": nl / (msl / 1e3),
                   "kernel_variant": il["kernel_variant"],
                   "roofline": roofline_from_profile(profile_fields(kernel_source_sha(), "sum_kernel_large37.txt",
                                                                   tables_sha(Z.zxp_scalar_to_tables(sl))),
                                                     nl, msl / 1e3, peak_l, "profiles/sum_kernel_large37.txt"),
                   "clocks": clkl.summary()}

    # batched workload: 512 circuits (n ~ U[10,40], T ~ U[20,60]), one
    # amplitude each: one launch per scalar vs one tuned, graph-captured batch
    batch = None
    if rank == 0 and not os.environ.get("ZXP_BENCH_SKIP_BATCH"):
        items = [zi.workload_batch_item(i) for i in range(512)]
        scal = [Z.zxp_compile(it.gates, it.n, it.out_bits) for it in items]
        ks = [Z.zxp_scalar_info(x)["k"] for x in scal]
        outs = torch.zeros(len(scal), 5, dtype=torch.int64, device="cuda")

        def plain():
            for j, x in enumerate(scal):
                Z.zxp_eval_device(ctx, x, 0, 1 << ks[j], outs[j].data_ptr())

        plain()
        a, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        a.record(stream)
        for _ in range(reps):
            plain()
        b2.record(stream)
        torch.cuda.synchronize()
        plain_ms = a.elapsed_time(b2) / reps
        t0b = time.perf_counter()
        bt = Z.zxp_batch_create(ctx, scal)
        create_ms = (time.perf_counter() - t0b) * 1e3
        res = Z.zxp_batch_run(bt)
        want = [tuple(v[:4]) + (v[4] & 0xFFFFFFFF,) for v in outs.tolist()]
        assert [tuple(r) for r in res] == want
        a.record(stream)
        for _ in range(reps):
            Z.zxp_batch_run(bt)
        b2.record(stream)
        torch.cuda.synchronize()
        batch_ms = a.elapsed_time(b2) / reps
        binfo = Z.zxp_batch_info(bt)
        batch = {"workload": "512 circuits, seeds 0-511, n~U[10,40], T~U[20,60], one amplitude each",
                 "k_min": min(ks), "k_max": max(ks), "total_terms": sum(1 << x for x in ks),
                 "plain_ms": plain_ms, "batch_ms": batch_ms,
                 "plain_amplitudes_per_s": len(scal) / (plain_ms / 1e3),
                 "batch_amplitudes_per_s": len(scal) / (batch_ms / 1e3),
                 "batch_terms_per_s": sum(1 << x for x in ks) / (batch_ms / 1e3),
                 "batch_create_ms": create_ms,
                 "tuned": {"threads": binfo["threads"], "chunk_log2": binfo["chunk_log2"],
                           "groups": binfo["n_groups"], "chunks": binfo["n_chunks"],
                           "candidates": binfo["candidates"]}}
        bt.close()

    # serving: Poisson arrivals of amplitude and doubled-marginal requests;
    # the server with continuous batching vs the same server evaluating one
    # scalar per launch in arrival order
    serving = None
    if rank == 0 and not os.environ.get("ZXP_BENCH_SKIP_SERVE"):
        serving = serve_bench(Z, ctx, zi, n_req=2000, rate_hz=2000.0, max_k=SERVE_MAX_K)

    param = None
    if rank == 0 and not os.environ.get("ZXP_BENCH_SKIP_PARAM"):
        param = param_bench(Z, ctx, zi)

    if rank != 0:
        if dist:
            dist.destroy_process_group()
        return

    peak, sms, mhz = issue_peak(torch, local, clocks.get("sm_max_mhz"))
    sha = kernel_source_sha()
    prof = profile_fields(sha, "sum_kernel_large80.txt", tables_sha(blob))
    roof = roofline_from_profile(prof, walked, walk_s, peak, "profiles/sum_kernel_large80.txt")
    roof["sms"] = sms
    roof["sm_max_mhz"] = mhz
    if int_peak:
        mix = int_peak["lop3_mad"]["thread_instr_per_s"]
        roof["measured_int_peak"] = {"lop3_mad_thread_instr_per_s": mix,
                                     "frac": None if roof["achieved"] is None else roof["achieved"] * 1e12 / mix,
                                     "basis": "integer microbenchmark (zxp_int_peak kind 4): logic and "
                                              "multiply-add chains in turn on a full grid"}
    launches_per_step = (inner_launches(ki) + 1) if ki else 1
    iprof = profile_fields(kernel_source_sha(INNER_SOURCES), "inner_table_large80.txt", tables_sha(blob))

    line = {
        "metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_ms / args.steps,
        "higher_is_better": True, "scaling": "strong" if args.shard else "weak", "vs_baseline": None,
        "dtype": "int64", "data": "synthetic",
        "config": {"workload": f"{w.name} seed={args.seed}: one exact amplitude per step "
                               "(inner table + Gray-code walk over the outer parameters)",
                   "k": k, "k_inner": ki, "inner_bits": info["inner_bits"],
                   "walked_terms_per_step": terms, "stabilizer_terms_per_step": stab_terms,
                   "t_count": info["t_count"], "kernel_variant": info["kernel_variant"],
                   "compile_ms": compile_ms, "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": (f"dp{world}: every amplitude's outer range sharded over the ranks, "
                                   "40-byte partials all-gathered (NCCL)") if args.shard
                                  else f"replicas x{world}"},
        "ms_inner_table": inner_s * 1e3, "ms_walk": walk_s * 1e3,
        "terms_per_s": walked / walk_s,
        "stabilizer_terms_per_s": stab_terms * value,
        "ms_allgather": statistics.median(gather_ms) if gather_ms else None,
        "roofline": roof,
        "inner_roofline": inner_roofline(info["inner_bits"], ki, inner_s, iprof) if ki else None,
        "e2e": {"value": 1 / e2e_sec, "unit": "amplitudes/s",
                "h2d_bytes_per_step": info["upload_bytes"], "d2h_bytes_per_step": 40,
                "requests_in_flight": E2E_DEPTH, "steps": e2e_steps},
        "clocks": clocks,
        "gpu_launches": launches_per_step * args.steps,
        "wall_s_timed_region": wall,
        "int_peak": int_peak,
    }
    if medium:
        line["medium"] = medium
    if unsplit:
        line["unsplit_k37"] = unsplit
    if synth:
        line["synthetic_k36"] = synth
    if batch:
        line["batch"] = batch
    if serving:
        line["serving"] = serving
    if param:
        line["parametric"] = param
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(blob, stab_terms)
    print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
