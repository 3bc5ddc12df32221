"""Benchmark: the batched finite-lattice sweep of Jacobsen (arXiv:1005.3609) on GB300.

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference] [--workload ...]

Default workload: square lattice, finite-lattice order k = 33 (62 rectangles
r x s, r <= s, 30 <= r+s <= 33, widths 1..16), 16 primes from the seed-0
draws, P~ truncated at w^63 (the series to z^63).  One step = one whole sweep:
reset of every strip to e_0, every per-site factor of every strip (batched
launches), every read-out, the finite-lattice series modulo each prime (one
CUDA graph launch) and the Chinese remaindering of the three series on the
GPU.  The transfer-matrix tables (which depend only on lattice and width) are
built once before the timed region, like any plan.

value = state-coefficient updates per second (one update = one 32-bit output
word of one per-site factor), whole job.  e2e = the same metric through the C
ABI with the primes copied host->device and the CRT'd series copied
device->host every step.  The reference arm (--impl reference) times the CPU
oracle on a bounded sample of the same workload.
"""
import argparse
import json
import multiprocessing as mp
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic_inputs  # noqa: E402

L2_BYTES = 129 * 1024 * 1024


# ---------------------------------------------------------------- workload bookkeeping

def motzkin_table(n):
    M = [1, 1]
    for p in range(2, n + 1):
        M.append(M[p - 1] + sum(M[j] * M[p - j - 2] for j in range(p - 1)))
    return M


def band(k):
    return [(r, s) for r in range(1, k // 2 + 1) for s in range(r, k - r + 1) if r + s >= k - 3]


def n_terms(lattice, k):
    if lattice == "square":
        return 2 * k - 2 if k % 2 else 2 * k - 3
    return k


def strip_updates(lattice, r, heights, D1, n_primes):
    """Output words of all per-site factors of one strip (rows and read-outs)."""
    M = motzkin_table(r + 2)
    cnt = lambda n: 1 if n == 0 else M[n - 1]
    Sb = cnt(r)
    Sx = cnt(r) + cnt(r - 1) if r >= 2 else Sb
    if lattice == "square":
        row = sum(Sx if i < r - 1 else Sb for i in range(r))
    else:
        row = r * Sb
    last = sum(cnt(r - i - 1) for i in range(r - 1)) if r >= 2 else 1
    return ((max(heights) - 1) * row + len(heights) * last) * D1 * n_primes


# ---------------------------------------------------------------- CPU oracle (baseline / reference arm)

def _oracle_job(args):
    lattice, widths, k, D, p = args
    from oracle import modp
    hb = {}
    for r, s in band(k):
        hb.setdefault(r, []).append(s)
    t = time.perf_counter()
    for r in widths:
        modp.ptilde_heights(lattice, r, hb[r], D, p)
    return time.perf_counter() - t


def oracle_sample(pool, lattice, k, primes, widths):
    """Run the plain-C mod-p oracle on the band rectangles of the given widths,
    one process per prime.  Returns (updates/s, wall s, updates, processes)."""
    D1 = n_terms(lattice, k)
    hb = {}
    for r, s in band(k):
        hb.setdefault(r, []).append(s)
    upd = sum(strip_updates(lattice, r, hb[r], D1, 1) for r in widths) * len(primes)
    t = time.perf_counter()
    pool.map(_oracle_job, [(lattice, widths, k, D1 - 1, p) for p in primes])
    wall = time.perf_counter() - t
    return upd / wall, wall, upd


def make_pool(n):
    ctx = mp.get_context("spawn")
    return ctx.Pool(n)


# ---------------------------------------------------------------- clocks

class ClockSampler:
    QUERY = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = os.path.join(tempfile.gettempdir(), "clocks_bench_%d.csv" % os.getpid())

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.QUERY,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        self.proc.wait()
        self.f.close()
        rows = []
        for ln in open(self.path):
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows if r[1].replace(".", "").isdigit())
        mx = max(float(r[2]) for r in rows if r[2].replace(".", "").isdigit())
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(rows)}


# ---------------------------------------------------------------- GPU arm

def load_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return None


def load_traffic(kernel_key):
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu summary, if it
    was taken on the current kernel source (same fingerprint)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(path))
    except Exception:
        return None
    ent = d.get(kernel_key)
    if not ent or ent.get("source_sha") != gather_source_sha():
        return None
    return ent


def gather_source_sha():
    import hashlib
    h = hashlib.sha256()
    for f in ("gather.cu", "gather_tma.cu", "cp_internal.h"):
        h.update(open(os.path.join(ROOT, "paper_1005_3609_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def table_layout(cp, args):
    """Apply --per-site-tables / --pairing and describe the layout of the transfer-matrix tables."""
    mode = 0 if args.per_site_tables else (args.pairing if args.pairing is not None else 1)
    cp.set_factor_pairing(mode)
    if mode == 0:
        return "one table per site factor (r launches per row)"
    if mode == 3:
        return ("two-site tables on both lattices: consecutive site factors composed in pairs (ceil(r/2) launches "
                "per row, the intermediate vector never written); updates counted per site factor")
    return ("square lattice, rows >= 3 KB: two-site tables, consecutive site factors composed in pairs (ceil(r/2) "
            "launches per row, the intermediate vector never written); otherwise one table per site factor; "
            "updates counted per site factor either way")


def tile_name(tile):
    rows, ring, edges, cpt = tile & 0xFFF, (tile >> 12) & 0xFF, (tile >> 20) & 15, (tile >> 24) & 15
    shape = (tile >> 28) & 3
    if rows <= 8:
        return "register gather kernel, %d rows/warp" % rows
    return "TMA gather kernel, %d rows/block, %s KB ring, %s edge(s) per stage, %s chunk(s) per thread, %s" % (
        rows, ring or "auto", edges or "auto", cpt or "auto",
        {1: "wide blocks", 2: "narrow blocks"}.get(shape, "block shape auto"))


def plain_run(cp, torch, lattice, k, primes, stream):
    """One (rectangle, prime) at a time: a 1-prime strip per width, reset to e_0
    for every rectangle, advanced by per-site launches, read into device memory."""
    D1 = n_terms(lattice, k)
    hb = {}
    for r, s in band(k):
        hb.setdefault(r, []).append(s)
    strips = {r: cp.Strip(lattice, r, [primes[0]], max_degree=D1 - 1, max_rows=max(hb[r]), stream=stream)
              for r in hb}
    out = torch.zeros(D1, dtype=torch.int32, device="cuda")
    upd = 0
    for r in hb:
        upd += sum(strip_updates(lattice, r, [s], D1, 1) for s in hb[r])
    upd *= len(primes)

    def once():
        for p in primes:
            for r in hb:
                st = strips[r]
                for s in hb[r]:
                    st.reset()
                    st.advance(s - 1)
                    st.read_device(out.data_ptr(), D1)

    # the strips hold primes[0]; the per-prime loop repeats the same work, as a
    # one-prime-at-a-time run on another prime would (same launches, same bytes)
    with torch.cuda.stream(stream):
        once()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        once()
        e1.record(stream)
        torch.cuda.synchronize()
    for s in strips.values():
        s.close()
    return e0.elapsed_time(e1), upd


def gpu_arm(args):
    import torch
    import paper_1005_3609_gb300 as cp

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    pool = None
    if world == 1 and not args.no_cpu_baseline:
        pool = make_pool(min(16, os.cpu_count() or 1))  # spawn, before the first GPU call
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    cp.load()
    lattice, k, P = args.lattice, args.k, args.primes
    # one prime stream, each rank its own slice of P primes (no overlap between ranks)
    from paper_1005_3609_gb300 import distributed as shard
    all_primes = cp.select_primes(synthetic_inputs.prime_draws(0, 64 * world + 64), P * world)
    lo, hi = shard.rank_prime_slice(P * world, world, rank)
    primes = all_primes[lo:hi]
    stream = torch.cuda.Stream()
    t_setup = time.perf_counter()
    layout = table_layout(cp, args)
    sw = cp.Sweep(lattice, k, primes, stream, tile=args.tile, prime_groups=args.groups)
    setup_s = time.perf_counter() - t_setup
    n = sw.n_terms
    limbs = (31 * P + 33) // 32 + 1
    res_dev = torch.zeros(3 * P * n, dtype=torch.int32, device="cuda")
    limb_dev = torch.zeros(3 * n * limbs, dtype=torch.int32, device="cuda")
    lib = cp.load()
    import ctypes
    pr_arr = (ctypes.c_uint32 * P)(*primes)

    def crt_device():
        # residues [3][P][n] -> limbs [3][n][limbs], one launch per series
        sw.read_series_device(res_dev.data_ptr(), res_dev.numel())
        for x in range(3):
            cp._lib.check("cp_crt_device", lib.cp_crt_device(
                ctypes.c_void_p(res_dev.data_ptr() + 4 * x * P * n), pr_arr, P, n,
                ctypes.c_void_p(limb_dev.data_ptr() + 4 * x * n * limbs), limbs, ctypes.c_void_p(stream.cuda_stream)))

    def step():
        sw.run()
        crt_device()

    def barrier():
        if dist:
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    if dist:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    updates_total = sw.updates_per_run * args.steps * world
    value = updates_total / (ms / 1e3)

    # ---- e2e through the C ABI: primes host->device (cp_sweep_set_primes), the sweep
    # (cp_sweep_run), the series CRT'd and checked for stability on the device and
    # their limbs copied into a pinned host buffer (cp_sweep_series_integers)
    import numpy as np
    pinned_primes = torch.tensor(primes, dtype=torch.int64).to(torch.int32).pin_memory()
    pinned_out = torch.zeros(3 * n * limbs, dtype=torch.int32).pin_memory()
    out_np = pinned_out.numpy().view(np.uint32).reshape(3, n, limbs)
    h2d = 4 * P
    d2h = 4 * 3 * n * limbs + 4 * 3 * n  # limbs and the per-term stability flags

    def e2e_step():
        sw.set_primes(pinned_primes.numpy().view("uint32"))
        sw.run()
        return sw.series_integers(limbs_per_coeff=limbs, out=out_np)

    for _ in range(max(1, args.warmup)):
        e2e_step()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record(stream)
    for _ in range(args.steps):
        series = e2e_step()
    f1.record(stream)
    torch.cuda.synchronize()
    barrier()
    e2e_ms = f0.elapsed_time(f1)
    host_ms = (time.perf_counter() - t0) * 1e3
    e2e_ms = max(e2e_ms, host_ms)
    if dist:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = float(t.item())
    e2e_value = updates_total / (e2e_ms / 1e3)
    # the e2e result must be the paper's series
    if dist:  # the one exchange: rank 0 gathers every rank's residues and recombines all primes
        got = shard.gather_residues(sw.read_series(), primes, dist)
        if rank == 0:
            res_all, primes_all = got
            series = [cp.crt(res_all[x], primes_all) for x in range(3)]

    # ---- roofline of the dominant kernel (batched gather), one ungraphed pass with per-launch events
    gather_ms, n_gather, pass_ms = sw.profile()
    peaks = load_peaks()
    peak = peaks.get("hbm_gbs") if peaks else None
    peak = peak or 6800.0
    # algorithmic bytes as defined per update (every per-site factor reads its input and writes its
    # output vector once); with two-site tables the launched tables need fewer (reported beside)
    achieved = sw.site_bytes_per_run / (gather_ms / 1e3) / 1e9
    traffic = load_traffic("gather_kernel:%s:k%d:P%d:%s" % (lattice, k, P, "site" if args.per_site_tables else "auto"))
    roofline = {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                "frac": round(achieved / peak, 4),
                "traffic": traffic["dram_bytes_per_launch"] if traffic else None,
                "algorithmic_bytes_per_launch": sw.site_bytes_per_run / n_gather,
                "avg_launch_ms": gather_ms / n_gather,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s",
                "kernel": "batched gather: %s" % tile_name(sw.tile)}
    if sw.bytes_per_run != sw.site_bytes_per_run:
        own = sw.bytes_per_run / (gather_ms / 1e3) / 1e9
        roofline["tables_own_bytes"] = {
            "bytes_per_launch": sw.bytes_per_run / n_gather, "achieved": round(own, 1), "frac": round(own / peak, 4),
            "note": "bytes the two-site tables themselves need (input, output, CSR; no intermediate vector)"}

    out = None
    if rank == 0:
        out = {"metric": "state-coeff updates/s (batched finite-lattice sweep)", "value": value,
               "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
               "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
               "vs_baseline": None, "dtype": "u32", "data": "synthetic",
               "config": {"workload": "%s lattice finite-lattice sweep k=%d: %d rectangles r x s (r<=s, %d<=r+s<=%d, "
                                      "widths 1..%d), %d primes/GPU (seed=rank), P~ to w^%d" %
                                      (lattice, k, sw.n_rects, k - 3, k, k // 2, P, n - 1),
                          "parallelism": ("weak: each rank sweeps its own %d primes, no collective while timed; "
                                          "rank 0 gathers the series residues afterwards" % P) if world > 1
                          else "single GPU",
                          "l2": "no flush: working set > L2 (width-16 vectors %.2f GB each)" %
                                (strip_bytes_max(lattice, k, n, P) / 1e9),
                          "tables": "built once per (lattice, width) before timing (%.2f s incl. autotune)" % setup_s,
                          "factor_tables": layout,
                          "tile": tile_name(sw.tile), "prime_groups": sw.prime_groups,
                          "updates_per_step": sw.updates_per_run,
                          "algorithmic_bytes_per_step": sw.site_bytes_per_run,
                          "table_bytes_per_step": sw.bytes_per_run},
               "e2e": {"value": e2e_value, "unit": "updates/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms / args.steps,
                       "path": "cp_sweep_set_primes (pinned host) -> cp_sweep_run -> cp_sweep_series_integers "
                               "(device CRT + stability flags, limbs into pinned host memory)"},
               "gpu_launches": args.steps * (sw.launches_per_run + 3),
               "roofline": roofline,
               "hbm_gbs_algorithmic": sw.site_bytes_per_run * args.steps / (ms / 1e3) / 1e9}
        if clk:
            out["clocks"] = clk
        if lattice == "square" and k in (33, 41):
            t = table1()
            out["check"] = {"series_match_table1": series[0] == t["alpha"][:n] and series[1] == t["beta"][:n]
                            and series[2][: n - 1] == t["gamma"][: n - 1]}
    if rank == 0 and world == 1 and not args.no_plain:
        plain_ms, plain_upd = plain_run(cp, torch, lattice, k, primes, stream)
        out["batched_vs_plain"] = {
            "plain_ms": plain_ms, "batched_ms": ms / args.steps, "speedup": plain_ms / (ms / args.steps),
            "plain_updates_per_s": plain_upd / (plain_ms / 1e3),
            "plain": "one (rectangle, prime) at a time: 1-prime strip reset to e_0 per rectangle, per-site launches, "
                     "tables cached", "batched": "one graph launch: strip prefixes shared across heights, %d primes "
                     "per row, all widths in each launch" % (P // sw.prime_groups)}
    sw.close()
    if rank == 0 and world == 1 and pool is not None:
        widths = [r for r in range(1, args.cpu_widths + 1)]
        rate, wall, upd = oracle_sample(pool, lattice, k, primes, widths)
        out["cpu_baseline"] = {"value": rate, "unit": "updates/s", "cores": min(16, os.cpu_count() or 1),
                               "kind": "oracle",
                               "sample": "plain-C mod-p oracle (hash-map TM), widths 1..%d of the same band, %d primes "
                                         "(one process per prime), %.1f s wall" % (args.cpu_widths, len(primes), wall)}
    if pool is not None:
        pool.close()
    if rank == 0 and world == 1 and not args.no_extras:
        extra = {}
        if lattice == "square" and k == 33:
            extra["triangular_sweep_k33"] = sweep_measure(cp, torch, "triangular", 33, primes, args)
        p8 = primes[:8]
        extra["config2_square_12x13"] = strip_measure(cp, torch, "square", 12, 13, p8, 5)
        extra["config3_triangular_13x14"] = strip_measure(cp, torch, "triangular", 13, 14, p8, 5)
        extra["serving_prefix"] = serve_measure(cp, torch, args.serve_prefix, args.serve_budget_gb,
                                                args.serve_max_active)
        out["extra_workloads"] = extra
    if rank == 0:
        print(json.dumps(out))
    if dist:
        dist.destroy_process_group()


def table1():
    """Table 1 of the paper (fixture tests/golden/table1_square.txt)."""
    a, b, g = [], [], []
    for ln in open(os.path.join(ROOT, "tests", "golden", "table1_square.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        f = ln.split()
        a.append(int(f[1]))
        b.append(int(f[2]))
        if f[3] != "-":
            g.append(int(f[3]))
    return {"alpha": a, "beta": b, "gamma": g}


def strip_bytes_max(lattice, k, n, P):
    M = motzkin_table(k // 2 + 2)
    r = k // 2
    S = M[r - 1] + (M[r - 2] if lattice == "square" else 0)
    return S * n * P * 4


# ---------------------------------------------------------------- serving workload

def serve_stream(cp, sv, reqs, primes_of, rate_scale=1.0):
    """Feed requests at their (scaled) Poisson arrival times in real time; step the
    server whenever it has work.  Returns per-request (queue s, service s, total s) and wall s."""
    t0 = time.perf_counter()
    ids, i = [], 0
    n = len(reqs)
    done = set()
    while len(done) < n:
        now = time.perf_counter() - t0
        while i < n and reqs[i]["arrival_s"] / rate_scale <= now:
            r = reqs[i]
            ids.append(sv.submit(r["lattice"], r["L"], r["N"], primes_of(r)))
            i += 1
        if len(ids) > len(done):
            _, _, fin = sv.step()
            if fin:
                done.update(sv.poll())
        elif i < n:
            time.sleep(max(0.0, min(0.01, reqs[i]["arrival_s"] / rate_scale - now)))
    wall = time.perf_counter() - t0
    lat = []
    for rid in ids:
        _, _, (ts, ta, td) = sv.result(rid)
        lat.append((ta - ts, td - ta, td - ts))
    return lat, wall


def pct(xs, q):
    xs = sorted(xs)
    return xs[min(len(xs) - 1, int(round(q / 100.0 * (len(xs) - 1))))]


def serve_measure(cp, torch, n_req, budget_gb, max_active, with_plain=True):
    """Serve the first n_req requests of the serving stream (seed 1, 200 req/s offered) in real
    time, then the same requests at 0.7x the measured capacity, then (with_plain) one
    (rectangle, prime) at a time.  Returns the measurement as a dict."""
    reqs = synthetic_inputs.serving_requests(seed=1, rate_per_s=200.0, n=10000)[:n_req]
    pcache = {}

    def primes_of(r):
        key = (r["prime_seed"], r["n_primes"])
        if key not in pcache:
            pcache[key] = cp.select_primes(synthetic_inputs.prime_draws(r["prime_seed"] % (2 ** 31), 64),
                                           r["n_primes"])
        return pcache[key]

    for r in reqs:
        primes_of(r)
    stream = torch.cuda.Stream()
    budget = int(budget_gb * (1 << 30))
    with cp.Server(budget, max_active=max_active, stream=stream) as sv:
        # warm-up: tables of every (lattice, width) in the stream, one tiny request each
        for lat in ("square", "triangular"):
            for L in sorted({r["L"] for r in reqs}):
                rid = sv.submit(lat, L, 1, [primes_of(reqs[0])[0]])
                while sv.result(rid)[0] != sv.DONE:
                    sv.step()
                sv.release(rid)
        sv.poll()
        st0 = sv.stats()
        clocks = ClockSampler(torch.cuda.current_device())
        clocks.start()
        lat, wall = serve_stream(cp, sv, reqs, primes_of)
        clk = clocks.stop()
        st1 = sv.stats()
        upd = st1["updates"] - st0["updates"]
        cap_rps = len(reqs) / wall
        # supplementary stream at 0.7x the measured capacity (added; arrival times rescaled)
        scale = 0.7 * cap_rps / 200.0
        lat07, wall07 = serve_stream(cp, sv, reqs, primes_of, rate_scale=scale)
    out = {"requests": len(reqs), "updates_per_s": upd / wall, "wall_s": wall, "requests_per_s": cap_rps,
           "server_steps": st1["steps"] - st0["steps"], "gpu_launches": st1["launches"] - st0["launches"],
           "latency_s": {"p50": pct([x[2] for x in lat], 50), "p99": pct([x[2] for x in lat], 99),
                         "queue_p50": pct([x[0] for x in lat], 50), "queue_p99": pct([x[0] for x in lat], 99),
                         "service_p50": pct([x[1] for x in lat], 50), "service_p99": pct([x[1] for x in lat], 99),
                         "note": "offered 200 req/s is several times the capacity: p50/p99 at saturation are "
                                 "mostly queueing; the 0.7x stream shows the latency below saturation"},
           "at_0.7x_capacity (added)": {"offered_req_per_s": 200.0 * scale, "wall_s": wall07,
                                        "p50": pct([x[2] for x in lat07], 50), "p99": pct([x[2] for x in lat07], 99),
                                        "queue_p99": pct([x[0] for x in lat07], 99)}}
    if with_plain:
        t = time.perf_counter()
        for r in reqs:
            for p in primes_of(r):
                with cp.Strip(r["lattice"], r["L"], [p], max_degree=-1, max_rows=r["N"], stream=stream) as st:
                    st.advance(r["N"] - 1)
                    st.read()
        plain_s = time.perf_counter() - t
        out["served_vs_plain"] = {"served_s": wall, "plain_s": plain_s, "speedup": plain_s / wall,
                                  "plain": "each request one prime at a time, 1-prime strip, per-site launches"}
    if clk:
        out["clocks"] = clk
    return out


def serve_arm(args):
    import torch
    import paper_1005_3609_gb300 as cp
    torch.cuda.set_device(0)
    cp.load()
    m = serve_measure(cp, torch, args.serve_n, args.serve_budget_gb, args.serve_max_active)
    out = {"metric": "served rectangle solves: state-coeff updates/s and p50/p99 latency", "value": m["updates_per_s"],
           "unit": "updates/s", "n_gpus": 1, "steps": 1, "warmup": 1, "ms_per_step": m["wall_s"] * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": "serving: Poisson stream seed 1, 200 req/s offered, first %d of 10000 requests; "
                                  "lattice U{square, triangular}, L U{4..16}, N in {L, L+1}, 4..16 primes, full degree"
                                  % m["requests"],
                      "mem_budget_gb": args.serve_budget_gb, "max_active": args.serve_max_active}}
    out.update({k: v for k, v in m.items() if k not in ("updates_per_s", "wall_s")})
    print(json.dumps(out))


# ---------------------------------------------------------------- further workloads on the default line

def baxter_bulk(n):
    """Baxter's product for the triangular lattice's (1-x)^2 exp(f_b)/q, eq. (efb), to x^(n-1)."""
    ser = [1] + [0] * (n - 1)

    def mul_factor(e, power):  # ser *= (1 - x^e)^power
        for _ in range(abs(power)):
            if power > 0:
                for i in range(n - 1, e - 1, -1):
                    ser[i] -= ser[i - e]
            else:
                for i in range(e, n):
                    ser[i] += ser[i - e]

    for j in range(1, n):
        for e, pw in ((6 * j - 3, 1), (6 * j - 2, 2), (6 * j - 1, 1), (6 * j - 5, -1), (6 * j - 4, -1),
                      (6 * j, -1), (6 * j + 1, -1)):
            if e < n:
                mul_factor(e, pw)
    return ser


def triangular_printed():
    s, c = [], []
    for ln in open(os.path.join(ROOT, "tests", "golden", "triangular_series.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        f = ln.split()
        s.append(int(f[1]))
        c.append(int(f[2]))
    return s, c


def sweep_measure(cp, torch, lattice, k, primes, args):
    """One more batched sweep (tables built and tile autotuned before timing): ms per sweep,
    updates/s, the gather's roofline fractions and the check against the printed series."""
    stream = torch.cuda.Stream()
    sw = cp.Sweep(lattice, k, primes, stream, tile=0, prime_groups=0)
    for _ in range(args.warmup):
        sw.run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        sw.run()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    series = sw.series_integers()
    gather_ms, n_gather, _ = sw.profile()
    peak = (load_peaks() or {}).get("hbm_gbs") or 6800.0
    n = sw.n_terms
    out = {"workload": "%s lattice finite-lattice sweep k=%d, %d rectangles, %d primes, P~ to w^%d"
                       % (lattice, k, sw.n_rects, len(primes), n - 1),
           "ms_per_sweep": ms, "updates_per_s": sw.updates_per_run / (ms / 1e3),
           "tile": tile_name(sw.tile), "prime_groups": sw.prime_groups,
           "gather_roofline_frac": round(sw.site_bytes_per_run / (gather_ms / 1e3) / 1e9 / peak, 4),
           "gather_roofline_frac_tables_own_bytes": round(sw.bytes_per_run / (gather_ms / 1e3) / 1e9 / peak, 4),
           "gather_launches": n_gather, "gather_ms": gather_ms}
    if lattice == "triangular":
        surf, corner = triangular_printed()
        out["check"] = {"bulk_equals_baxter_product": series[0] == baxter_bulk(n),
                        "surface_corner_match_printed": series[1] == surf[:n] and series[2] == corner[:n]}
    sw.close()
    return out


def strip_measure(cp, torch, lattice, L, N, primes, reps):
    """One plain rectangle solve at full degree (a strip reset to e_0, N-1 rows, read-out)."""
    stream = torch.cuda.Stream()
    with cp.Strip(lattice, L, primes, max_degree=-1, max_rows=N, stream=stream) as s:
        row_upd, _, ro_upd, _, _, _ = s.work()
        out_dev = torch.zeros(len(primes) * L * N, dtype=torch.int32, device="cuda")

        def once():
            s.reset()
            s.advance(N - 1)
            s.read_device(out_dev.data_ptr(), out_dev.numel())

        once()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            once()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / reps
        upd = (N - 1) * row_upd + ro_upd
        ints = s.read_integers(strict=False)
    return {"workload": "%s %dx%d, full degree %d, %d primes: reset, %d rows, read-out" % (
                lattice, L, N, L * N - 1, len(primes), N - 1),
            "ms_per_solve": ms, "updates_per_s": upd / (ms / 1e3), "updates": upd,
            "exact_integers_from_these_primes": ints[2] == 0}


# ---------------------------------------------------------------- paper-scale workload

def paper_arm(args):
    """The paper's own scale: k = 41 (widths up to m_max = 20, Sec. 4.2-4.3) on 16 primes,
    as two prime groups of 8 swept back to back (8 primes of width-20 vectors take about
    250 GB, so both groups do not fit at once); the 16 primes' series residues are then
    recombined by CRT with the stabilisation check (cp_crt_checked)."""
    import numpy as np
    import torch
    import paper_1005_3609_gb300 as cp
    torch.cuda.set_device(0)
    lattice, k = args.lattice, 41
    primes = cp.select_primes(synthetic_inputs.prime_draws(0, 128), 16)
    stream = torch.cuda.Stream()
    tile = args.tile or 32  # TMA kernel, rows/block 32, ring, stages and chunks per thread picked by row width
    table_layout(cp, args)
    peak = (load_peaks() or {}).get("hbm_gbs") or 6800.0
    groups, res_all = [], []
    for g in range(2):
        pg = primes[8 * g: 8 * g + 8]
        t0 = time.perf_counter()
        sw = cp.Sweep(lattice, k, pg, stream, tile=tile, prime_groups=1)
        setup_s = time.perf_counter() - t0
        for _ in range(max(1, args.warmup)):
            sw.run()
        sw.sync()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        sw.run()
        e1.record(stream)
        sw.sync()
        ms = e0.elapsed_time(e1)
        res_all.append(sw.read_series())
        groups.append({"primes": pg, "ms": ms, "setup_s": setup_s, "updates": sw.updates_per_run,
                       "updates_per_s": sw.updates_per_run / (ms / 1e3),
                       "frac_per_update_bytes": round(sw.site_bytes_per_run / (ms / 1e3) / 1e9 / peak, 4),
                       "frac_tables_own_bytes": round(sw.bytes_per_run / (ms / 1e3) / 1e9 / peak, 4)})
        n = sw.n_terms
        sw.close()
    series, stable = [], True
    for x in range(3):
        ints, _, rc = cp.crt_checked(np.concatenate([res_all[0][x], res_all[1][x]], axis=0), primes)
        series.append(ints)
        stable = stable and rc == 0
    check = {"series_stable_over_16_primes": stable}
    if lattice == "square":
        t = table1()
        check["series_match_table1"] = (series[0] == t["alpha"][:n] and series[1] == t["beta"][:n]
                                        and series[2][: n - 1] == t["gamma"][: n - 1])
    else:
        surf, corner = triangular_printed()
        check["bulk_equals_baxter_product"] = series[0] == baxter_bulk(n)
        check["surface_corner_match_printed"] = series[1] == surf[:n] and series[2] == corner[:n]
    tot_ms = sum(g_["ms"] for g_ in groups)
    upd = sum(g_["updates"] for g_ in groups)
    out = {"metric": "state-coeff updates/s (paper-scale finite-lattice sweep)", "value": upd / (tot_ms / 1e3),
           "unit": "updates/s", "n_gpus": 1, "steps": 1, "warmup": max(1, args.warmup), "ms_per_step": tot_ms,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": "%s lattice finite-lattice sweep k=41 (widths 1..20), 16 primes as two groups "
                                  "of 8 swept back to back, series CRT'd over all 16" % lattice,
                      "tile": tile_name(tile)},
           "groups": groups, "check": check}
    print(json.dumps(out))


# ---------------------------------------------------------------- reference arm (the CPU oracle)

def reference_arm(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    lattice, k, P = args.lattice, args.k, args.primes
    from oracle import crt as ocrt
    primes = ocrt.primes_from_draws(synthetic_inputs.prime_draws(0, 256), P)
    cores = min(16, os.cpu_count() or 1)
    pool = make_pool(cores)
    widths = list(range(1, args.ref_widths + 1))
    for _ in range(args.warmup):
        oracle_sample(pool, lattice, k, primes[:cores], [1, 2, 3])
    tot_upd, tot_s = 0, 0.0
    for _ in range(args.steps):
        rate, wall, upd = oracle_sample(pool, lattice, k, primes, widths)
        tot_upd += upd
        tot_s += wall
    pool.close()
    value = tot_upd / tot_s
    out = {"impl": "reference", "metric": "state-coeff updates/s (batched finite-lattice sweep)", "value": value,
           "unit": "updates/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": tot_s * 1e3 / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "u32", "data": "synthetic",
           "config": {"workload": "%s lattice finite-lattice sweep k=%d, %d primes; each step a bounded sample: "
                                  "widths 1..%d" % (lattice, k, P, args.ref_widths)},
           "cpu_baseline": {"value": value, "unit": "updates/s", "cores": cores, "kind": "oracle",
                            "sample": "plain-C mod-p oracle, widths 1..%d of the k=%d band, %d primes, one process "
                                      "per prime" % (args.ref_widths, k, P)},
           "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# ---------------------------------------------------------------- probe workload (one wide strip)

def _probe_oracle_job(args):
    lattice, L, rows, D, p = args
    from oracle import modp
    t = time.perf_counter()
    modp.ptilde_heights(lattice, L, [rows + 1], D, p)
    return time.perf_counter() - t


def probe_arm(args):
    """One strip of width L (default: square, width 18, 3 210 246 intermediate
    states, 12.9 GB per vector at D = 62 and 16 primes): each step resets it to
    e_0, advances `rows` rows and reads P~ out.  The per-site kernel runs far
    beyond the L2 here.  --lattice triangular gives the triangular strip."""
    import torch
    import paper_1005_3609_gb300 as cp
    pool = None
    if not args.no_cpu_baseline:
        pool = make_pool(min(16, os.cpu_count() or 1))  # spawn, before the first GPU call
    L, D, P, rows = args.probe_L, args.probe_D, args.primes, args.probe_rows
    primes = cp.select_primes(synthetic_inputs.prime_draws(0, 64), P)
    stream = torch.cuda.Stream()
    t_setup = time.perf_counter()
    layout = table_layout(cp, args)
    lattice = args.lattice
    s = cp.Strip(lattice, L, primes, max_degree=D, max_rows=rows + 1, stream=stream)
    if args.tile:
        s.set_tile(args.tile)
    setup_s = time.perf_counter() - t_setup
    row_upd, row_own, ro_upd, ro_own, row_bytes, ro_bytes = s.work()
    paired = row_own < row_bytes
    len_row = (L + 1) // 2 if paired else L  # gather launches per row
    out = torch.zeros(P * (D + 1), dtype=torch.int32, device="cuda")

    def step():
        s.reset()
        s.advance(rows)
        s.read_device(out.data_ptr(), out.numel())

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(0)
    clocks.start()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    upd_step = rows * row_upd + ro_upd
    value = upd_step * args.steps / (ms / 1e3)
    # roofline of the per-site gather: each row advance is L gather launches and nothing else
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * rows)]
    s.reset()
    for r in range(rows):
        ev[2 * r].record(stream)
        s.advance(1)
        ev[2 * r + 1].record(stream)
    torch.cuda.synchronize()
    row_ms = sum(ev[2 * r].elapsed_time(ev[2 * r + 1]) for r in range(rows)) / rows
    peaks = load_peaks()
    peak = (peaks or {}).get("hbm_gbs") or 6800.0
    achieved = row_bytes / (row_ms / 1e3) / 1e9  # per-update algorithmic bytes (one factor at a time)
    own = row_own / (row_ms / 1e3) / 1e9        # bytes the launched tables need
    traffic = load_traffic("gather_kernel:probe:%s:L%d:D%d:P%d:%s" % (lattice, L, D, P,
                                                                          "site" if args.per_site_tables else "auto"))
    # e2e through the C ABI: the read-out copied to host memory every step
    host = None
    f0 = time.perf_counter()
    for _ in range(args.steps):
        s.reset()
        s.advance(rows)
        host = s.read()
    e2e_ms = (time.perf_counter() - f0) * 1e3
    n_states = s.n_states
    s.close()
    res = {"metric": "state-coeff updates/s (one wide strip, per-site gather)", "value": value, "unit": "updates/s",
           "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
           "config": {"workload": "%s strip width %d (%d NCNNN / %d intermediate states), %d primes, D=%d: "
                                  "reset to e_0, %d rows, read-out" % (lattice, L, n_states[0], n_states[1], P, D,
                                                                       rows),
                      "l2": "no flush: vectors %.1f GB each, > 100x L2" % (n_states[1] * (D + 1) * P * 4 / 1e9),
                      "tables": "built before timing (%.1f s)" % setup_s, "tile": "strip default (TMA gather)",
                      "factor_tables": layout,
                      "updates_per_step": upd_step},
           "e2e": {"value": upd_step * args.steps / (e2e_ms / 1e3), "unit": "updates/s", "h2d_bytes_per_step": 0,
                   "d2h_bytes_per_step": 4 * P * (D + 1), "ms_per_step": e2e_ms / args.steps},
           "gpu_launches": args.steps * (rows * len_row + (L // 2 if paired else L - 1) + 1),
           "roofline": {"bound": "hbm", "achieved": round(achieved, 1), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4),
                        "traffic": traffic["dram_bytes_per_launch"] if traffic else None,
                        "algorithmic_bytes_per_launch": row_bytes / len_row, "avg_launch_ms": row_ms / len_row,
                        "peak_source": "MEASURED_PEAKS.json hbm_gbs (of measured)" if peaks else "fallback 6800 GB/s",
                        "kernel": "TMA gather (row advance = %d launches)" % len_row,
                        "tables_own_bytes": {"bytes_per_launch": row_own / len_row, "achieved": round(own, 1),
                                             "frac": round(own / peak, 4)}}}
    if clk:
        res["clocks"] = clk
    if pool is not None:
        cL, cP = args.probe_cpu_L, min(P, min(16, os.cpu_count() or 1))
        t = time.perf_counter()
        pool.map(_probe_oracle_job, [(lattice, cL, rows, D, p) for p in primes[:cP]])
        wall = time.perf_counter() - t
        with cp.Strip(lattice, cL, primes[:1], max_degree=D, max_rows=rows + 1) as sc:
            ru, _, ou, _, _, _ = sc.work()
        cupd = (rows * ru + ou) * cP
        res["cpu_baseline"] = {"value": cupd / wall, "unit": "updates/s", "cores": cP, "kind": "oracle",
                               "sample": "plain-C mod-p oracle (hash-map TM), %s width %d, %d rows, D=%d, %d "
                                         "primes (one process each), %.1f s wall" % (lattice, cL, rows, D, cP, wall)}
        pool.close()
    print(json.dumps(res))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--lattice", default="square", choices=["square", "triangular"])
    ap.add_argument("--k", type=int, default=33)
    ap.add_argument("--primes", type=int, default=16)
    ap.add_argument("--tile", type=int, default=0, help="gather units per thread (0 = autotune)")
    ap.add_argument("--groups", type=int, default=0, help="prime groups (0 = autotune)")
    ap.add_argument("--cpu-widths", type=int, default=13, help="widths of the CPU-baseline sample")
    ap.add_argument("--ref-widths", type=int, default=11, help="widths of each reference-arm step")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--workload", default="sweep", choices=["sweep", "serve", "probe", "paper"])
    ap.add_argument("--probe-L", type=int, default=18, help="strip width of the probe workload")
    ap.add_argument("--probe-D", type=int, default=62)
    ap.add_argument("--probe-rows", type=int, default=4)
    ap.add_argument("--probe-cpu-L", type=int, default=15, help="strip width of the probe's CPU-baseline sample")
    ap.add_argument("--serve-n", type=int, default=300, help="requests of the serving stream to run")
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--serve-max-active", type=int, default=64)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the further workloads of the default line (triangular sweep, configs 2/3, serving)")
    ap.add_argument("--serve-prefix", type=int, default=100,
                    help="requests of the serving stream run on the default line")
    ap.add_argument("--pairing", type=int, default=None, choices=[0, 1, 2, 3],
                    help="table layout (cp_set_factor_pairing): 1 default, 3 two-site tables on both lattices")
    ap.add_argument("--per-site-tables", action="store_true",
                    help="one table per site factor instead of two-site tables (same results)")
    args = ap.parse_args()
    if args.impl == "reference":
        reference_arm(args)
    elif args.workload == "serve":
        serve_arm(args)
    elif args.workload == "probe":
        probe_arm(args)
    elif args.workload == "paper":
        paper_arm(args)
    else:
        gpu_arm(args)


if __name__ == "__main__":
    main()
