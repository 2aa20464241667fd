"""Benchmark: exact stabilizer-term sums on GB300.

One step = one full exact amplitude of the medium workload (n = 20 qubits,
600 gates with 40 T gates, seeded random output bitstring): the sum of all
2^k terms of its compiled parametric scalar on the GPU, result on the device
(value), or one request through the public host API from the scalar's table
bytes to the exact result on the host, two requests in flight (e2e).  The
circuit is reduced to the scalar once, before timing.

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
SM_COUNT_GB300 = 152
ISSUE_LANES_PER_SM_CLK = 4 * 32       # 4 schedulers x 1 warp-instruction x 32 lanes


def alg_ops_per_term(node_words: int, other_words: int, n_pairs: int) -> int:
    """Integer operations the method needs per term, counted from the steps
    of one term: Gray step (ctz, flip XORs, quadratic bit), node count, linear
    phase planes, zero test, table fetch and the four 64-bit adds.  Up to
    two phase-pair factors are folded into the table index (2 operations);
    beyond that each is a Z[w] product (16 64-bit multiply-adds)."""
    nw = node_words + other_words
    ops = 2 + nw + 4                 # ctz + loop, flip XORs, quadratic update
    ops += 2 * node_words            # popc + add per node word
    ops += 4 * other_words           # (and + popc) x 2 linear planes
    ops += nw + 1                    # plane 2: and-xor per word, popc
    ops += other_words               # zero test
    ops += 4 + 3 + 8                 # J, table address + load, 4 x 64-bit add
    ops += 40 * n_pairs if n_pairs > 2 else (2 if n_pairs else 0)
    return ops


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


KERNEL_SOURCES = ("sum_kernel.cuh", "kernel_core.cuh", "kernel.cu", "kernel_count.cu", "zring.h",
                  "plan.cpp")


def kernel_source_sha() -> str:
    """Hash of the sources that decide the sum kernel's code and tables."""
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        h.update(open(os.path.join(ROOT, "paper_2403_06777_gb300", "csrc", f), "rb").read())
    return h.hexdigest()


def profile_fields(kernel_src_sha: str, name: str = "sum_kernel_medium.txt"):
    """Fields of a committed ncu summary, if it was taken on the current
    kernel sources (else None)."""
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
    return fields


def profile_number(fields, key):
    try:
        return float(fields[key].split()[0]) if fields else None
    except (KeyError, ValueError, IndexError):
        return None


def cpu_baseline(blob: bytes, k: int, seconds: float = 10.0):
    import oracle
    cores = os.cpu_count() or 1
    n = 1 << 14
    t = time.perf_counter()
    oracle.ps_sum(blob, 0, min(n, 1 << k), nthreads=cores)
    dt = max(time.perf_counter() - t, 1e-6)
    target = int(n * seconds / dt)
    n = 1 << max(10, min(k, target.bit_length() - 1))
    t = time.perf_counter()
    oracle.ps_sum(blob, 0, n, nthreads=cores)
    dt = time.perf_counter() - t
    return {"value": n / dt, "unit": "terms/s", "cores": cores, "kind": "oracle",
            "sample": f"Gray-index range [0, 2^{n.bit_length() - 1}) of the same scalar, "
                      f"{dt:.1f} s on {cores} host threads"}


SERVE_MAX_K = 38


def serve_run(Z, ctx, reqs, policy, max_k):
    """Replay the arrivals against one server; per-request latency is the
    library's own submit-to-value time."""
    srv = Z.zxp_server_create(ctx, policy=policy, max_k=max_k)
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


def serve_bench(Z, ctx, zi, n_req: int, rate_hz: float, max_k: int):
    reqs = zi.serve_requests(0, n_req, rate_hz)
    for r in reqs:
        r["gb"] = zi.pack_gates(r["gates"])
    batched, vb = serve_run(Z, ctx, reqs, Z.ZXP_SERVE_BATCHED, max_k)
    plain, vp = serve_run(Z, ctx, reqs, Z.ZXP_SERVE_PLAIN, max_k)
    assert vb == vp, "served values differ between policies"
    return {"workload": f"{n_req} requests, Poisson {rate_hz:.0f}/s, seed 0: amplitude and "
                        "single-qubit doubled-marginal, n~U[10,50], T~U[10,70]",
            "admission_max_k": max_k, "batched": batched,
            "plain_one_scalar_per_launch": plain,
            "p99_plain_over_batched": plain["p99_ms"] / batched["p99_ms"]}


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


def setup_dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def run_reference(args, world, rank):
    """The oracle on the host cores, bounded sample per step."""
    if rank != 0:
        return
    import oracle
    import paper_2403_06777_gb300 as Z
    import zxp_inputs as zi
    w = zi.workload_medium(args.seed)
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    blob = Z.zxp_scalar_to_tables(s)
    k = Z.zxp_scalar_info(s)["k"]
    cores = os.cpu_count() or 1
    t = time.perf_counter()
    oracle.ps_sum(blob, 0, 1 << 12, nthreads=cores)
    per_term = (time.perf_counter() - t) / (1 << 12)
    total_budget = 150.0
    n = 1 << max(8, min(k, int(total_budget / max(1, args.steps + args.warmup) / per_term).bit_length() - 1))
    for i in range(args.warmup):
        oracle.ps_sum(blob, 0, n, nthreads=cores)
    t = time.perf_counter()
    for i in range(args.steps):
        first = (i * n) % ((1 << k) - n + 1)
        oracle.ps_sum(blob, first, n, nthreads=cores)
    dt = time.perf_counter() - t
    v = n * args.steps / dt
    sample = f"{n} terms (2^{n.bit_length() - 1}) of the 2^{k}-term scalar per step"
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "terms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int128",
        "data": "synthetic",
        "config": {"workload": f"{w.name} seed={args.seed}: one exact amplitude per step", "k": k,
                   "terms_per_step": n, "sample": sample},
        "cpu_baseline": {"value": v, "unit": "terms/s", "cores": cores, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "terms/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    world, rank, local = setup_dist()

    if args.impl == "reference":
        run_reference(args, world, rank)
        return

    import torch
    import paper_2403_06777_gb300 as Z
    import zxp_inputs as zi

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # a dedicated stream: the library launches on it and the CUDA events are
    # recorded on it (torch's legacy default stream has handle 0, which the
    # C ABI reads as "create your own stream")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx = Z.zxp_ctx_create(local, stream.cuda_stream)

    w = zi.workload_medium(args.seed)
    t0 = time.perf_counter()
    s = Z.zxp_compile(w.gates, w.n, w.out_bits)
    compile_ms = (time.perf_counter() - t0) * 1e3
    info = Z.zxp_scalar_info(s)
    k = info["k"]
    terms = 1 << k
    blob = Z.zxp_scalar_to_tables(s)

    out = torch.zeros(5, dtype=torch.int64, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")   # > 129 MB L2

    for _ in range(args.warmup):
        Z.zxp_eval_device(ctx, s, 0, terms, out.data_ptr())
    torch.cuda.synchronize()
    ref = Z.zxp_amplitude(ctx, s)

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    stops = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()                           # L2 flushed between timed steps
            starts[i].record(stream)
            Z.zxp_eval_device(ctx, s, 0, terms, out.data_ptr())
            stops[i].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - wall0
    if dist:
        dist.barrier()
    kernel_ms = sum(a.elapsed_time(b) for a, b in zip(starts, stops))
    # the device result of the last step must be the exact amplitude
    r = out.tolist()
    got = Z.zxp_zomega_canon((r[0], r[1], r[2], r[3], r[4] & 0xFFFFFFFF))
    assert got == ref, (got, ref)
    t_rank = torch.tensor([kernel_ms], dtype=torch.float64, device="cuda")
    if dist:
        dist.all_reduce(t_rank, op=dist.ReduceOp.MAX)
    kernel_ms = float(t_rank.item())
    sec = kernel_ms / 1e3
    value = terms * args.steps * world / sec
    amps = args.steps * world / sec
    per_launch_s = sec / args.steps

    # e2e: the public host API, one request per step: the tables (host
    # bytes) are submitted (zxp_submit_tables: the scalar is built on the
    # host, its tables copied from pinned staging, the kernel launched) and
    # polled (the 40-byte result the kernel wrote into pinned host memory);
    # up to E2E_DEPTH requests are in flight, as a client streaming requests
    # runs them.  Every result is checked against the exact amplitude after
    # the timed loop.  The latency of one blocking request (nothing else in
    # flight) is reported beside it.
    E2E_DEPTH = 2
    e2e_steps = max(200, 10 * args.steps)
    from collections import deque
    torch.cuda.synchronize()
    q = deque()
    got = []
    t = time.perf_counter()
    for i in range(e2e_steps + E2E_DEPTH):
        if i < e2e_steps:
            q.append(Z.zxp_submit_tables(ctx, blob))
        if len(q) > E2E_DEPTH or (i >= e2e_steps and q):
            got.append(Z.zxp_poll(ctx, q.popleft(), -1))
    e2e_sec = (time.perf_counter() - t) / e2e_steps
    bad = sum(Z.zxp_zomega_canon(r) != ref for r in got)
    assert bad == 0 and len(got) == e2e_steps, (bad, len(got))
    lat = []
    for _ in range(100):
        t = time.perf_counter()
        s2 = Z.zxp_scalar_from_tables(blob)
        Z.zxp_amplitude(ctx, s2)
        s2.free()
        lat.append(time.perf_counter() - t)
    lat.sort()
    latency_us = lat[len(lat) // 2] * 1e6
    table_bytes = info["device_bytes"]

    # large scalar: k = 36 synthetic tables with compiled statistics (the
    # compiled n = 50 / t = 80 circuit needs k ~ 50, out of reach)
    large = None
    if rank == 0 and not os.environ.get("ZXP_BENCH_SKIP_LARGE"):
        # row counts of the compiled n = 50 / t = 80 circuit (seed 0: 59 linear,
        # 47 quadratic, 13 odd-node and 1 phase-pair rows at k = 50), at k = 36
        ps36 = zi.synthetic_ps(36, 36, n_lin=59, n_quad=36, n_node=13, n_pair=1,
                               odd_nodes_only=True, density=0.12)
        s36 = Z.zxp_scalar_from_tables(ps36.pack())
        i36 = Z.zxp_scalar_info(s36)
        Z.zxp_eval_device(ctx, s36, 0, 1 << 30, out.data_ptr())
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        with ClockSampler(local) as clk36:
            a.record(stream)
            Z.zxp_eval_device(ctx, s36, 0, 1 << 36, out.data_ptr())
            b.record(stream)
            torch.cuda.synchronize()
        ms36 = a.elapsed_time(b)
        ops36 = alg_ops_per_term(i36["node_words"], i36["other_words"], i36["n_pair"])
        ach36 = ops36 * (1 << 36) / (ms36 / 1e3) / 1e9
        peak = SM_COUNT_GB300 * ISSUE_LANES_PER_SM_CLK * 2070e6 / 1e9
        prof_s = profile_fields(kernel_source_sha(), "sum_kernel_synthetic36.txt")
        ipt_s = profile_number(prof_s, "instructions_per_term")
        iss_s = None if ipt_s is None else ipt_s * (1 << 36) / (ms36 / 1e3) / 1e9
        large = {"workload": "synthetic k=36 (59 linear, 36 quadratic, 13 odd-node, 1 phase-pair rows)",
                 "terms": 1 << 36, "ms": ms36, "terms_per_s": (1 << 36) / (ms36 / 1e3),
                 "node_words": i36["node_words"], "other_words": i36["other_words"],
                 "kernel_variant": i36["kernel_variant"],
                 "roofline": {"bound": "alu", "achieved": ach36, "peak": peak, "unit": "Gop/s",
                              "frac": ach36 / peak, "ops_per_term": ops36,
                              "traffic": profile_number(prof_s, "dram_bytes_per_launch"),
                              "issue": {"instructions_per_term": ipt_s, "achieved": iss_s,
                                        "frac": None if iss_s is None else iss_s / peak,
                                        "source": "thread instructions per term of the committed "
                                                  "ncu capture (profiles/sum_kernel_synthetic36.txt)"}},
                 "clocks": clk36.summary()}

    # large compiled circuit: n = 50, 2000 gates at T-count 50 (k = 37), the
    # full exact sum in one launch
    large_c = None
    if rank == 0 and not os.environ.get("ZXP_BENCH_SKIP_LARGE"):
        wl = zi.workload_large_t50(0)
        sl = Z.zxp_compile(wl.gates, wl.n, wl.out_bits)
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
        opsl = alg_ops_per_term(il["node_words"], il["other_words"], il["n_pair"])
        achl = opsl * nl / (msl / 1e3) / 1e9
        peak = SM_COUNT_GB300 * ISSUE_LANES_PER_SM_CLK * 2070e6 / 1e9
        prof_l = profile_fields(kernel_source_sha(), "sum_kernel_large37.txt")
        ipt_l = profile_number(prof_l, "instructions_per_term")
        iss_l = None if ipt_l is None else ipt_l * nl / (msl / 1e3) / 1e9
        large_c = {"workload": f"{wl.name} seed=0: one exact amplitude", "k": il["k"], "terms": nl,
                   "ms": msl, "terms_per_s": nl / (msl / 1e3), "kernel_variant": il["kernel_variant"],
                   "roofline": {"bound": "alu", "achieved": achl, "peak": peak, "unit": "Gop/s",
                                "frac": achl / peak, "ops_per_term": opsl,
                                "traffic": profile_number(prof_l, "dram_bytes_per_launch"),
                                "issue": {"instructions_per_term": ipt_l, "achieved": iss_l,
                                          "frac": None if iss_l is None else iss_l / peak,
                                          "source": "thread instructions per term of the committed "
                                                    "ncu capture (profiles/sum_kernel_large37.txt)"}},
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

    # serving: Poisson arrivals (2000 req/s) of amplitude and doubled-marginal
    # requests; the server with continuous batching vs the same server
    # evaluating one scalar per launch in arrival order
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

    clocks = clk.summary()
    ops = alg_ops_per_term(info["node_words"], info["other_words"], info["n_pair"])
    f_hz = 2070e6
    peak = SM_COUNT_GB300 * ISSUE_LANES_PER_SM_CLK * f_hz / 1e9          # Gop/s
    achieved = ops * terms / per_launch_s / 1e9
    sha = kernel_source_sha()
    prof = profile_fields(sha)
    traffic = profile_number(prof, "dram_bytes_per_launch")
    ipt = profile_number(prof, "instructions_per_term")

    line = {
        "metric": METRIC, "value": value, "unit": "terms/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": kernel_ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
        "data": "synthetic",
        "config": {"workload": f"{w.name} seed={args.seed}: one exact amplitude per step",
                   "k": k, "terms_per_step": terms, "t_count": info["t_count"],
                   "compile_ms": compile_ms, "l2": "flushed (256 MB write) between timed steps",
                   "parallelism": f"replicas x{world}"},
        "amplitudes_per_s": amps,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gop/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "ops_per_term": ops,
                     "peak_basis": "issue: 152 SM x 4 warp-instr/clk x 32 lanes x 2070 MHz",
                     "issue": {"instructions_per_term": ipt,
                               "achieved": None if ipt is None else ipt * terms / per_launch_s / 1e9,
                               "frac": None if ipt is None else ipt * terms / per_launch_s / 1e9 / peak,
                               "source": "thread instructions per term of the committed ncu capture"},
                     "note": "ops_per_term counts the per-term method (ctz, flips, popcount planes, "
                             "table fetch, 64-bit adds); the block lookup shares work across 8 terms, "
                             "so the kernel executes fewer instructions per term (issue)"},
        "e2e": {"value": terms / e2e_sec, "unit": "terms/s", "amplitudes_per_s": 1 / e2e_sec,
                "h2d_bytes_per_step": table_bytes, "d2h_bytes_per_step": 40,
                "requests_in_flight": E2E_DEPTH, "steps": e2e_steps,
                "blocking_latency_us": latency_us},
        "clocks": clocks,
        "gpu_launches": args.steps,
        "wall_s_timed_region": wall,
    }
    if large:
        line["large"] = large
    if large_c:
        line["large_compiled"] = large_c
    if batch:
        line["batch"] = batch
    if serving:
        line["serving"] = serving
    if param:
        line["parametric"] = param
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(blob, k)
    print(json.dumps(line))
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
