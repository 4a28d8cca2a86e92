"""Benchmark: least-squares solves per second on the largest single-GPU
configuration, a dense 5,000,000 x 2000 FP64 problem (80 GB; singular values
geometric 1..1e-8; b = A x_true + 1e-6 g/||g||), sparse sign sketch d = 8000,
zeta = 8, LSQR tolerance 1e-12, at backward error <= 1e-10.  The headline is
the plain FP64 form; the mixed form (sketch terms added in FP32 chunk sums) runs on
the same A and b beside it, and the 2,000,000 x 500 coherent-row problem
(d = 2000) is reported as an extra key.

One step = one full solve (sketch + preconditioner + LSQR + accuracy pass)
through the library's C ABI.  Prints one JSON line.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
                  [--config 0|1|2|3|4] [--prec fp64|mixed] [--native]

Under torchrun (N > 1) every rank solves its own copy of the problem on its
own GPU (the path does not shard in this build: replicas only); the value is
the solves of all ranks divided by the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_BYTES = 129 * 1024 * 1024


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix=f"clocks_gpu{self.gpu}_", suffix=".csv")
            self.f = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:  # no nvidia-smi: no clock record
            self.proc = None
            if getattr(self, "f", None):
                self.f.close()
            if self.path:
                try:
                    os.unlink(self.path)
                except OSError:
                    pass

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        try:
            os.unlink(self.path)
        except OSError:
            pass
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def max_over_ranks(x, device):
    """x from every rank -> the largest (barrier first); x itself on one rank."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.barrier()
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def make_problem(config, device, m=None, n=None, cond=1e10, coherent=0.01):
    from paper_2506_03070_gb300 import synth
    if m and n:
        p = synth.dense_problem(m, n, cond, resid_norm=1e-6, coherent_frac=coherent, seed=10, device=device)
        tag = "_coherent" if coherent > 0 else ""
        p.update(d=4 * n, zeta=8, tol=1e-12, seed_sketch=43, name=f"dense_{m}x{n}_cond{cond:.0e}{tag}")
        return p
    if config == 0:
        p = synth.config0(device=device)
    else:
        p = synth.config1(device=device)
    return p


def _workload(p, prec):
    A = p["A"]
    m, n = A.shape
    return {"workload": p["name"] + f"_d{p['d']}_zeta{p['zeta']}_tol{p['tol']:g}", "m": m, "n": n, "d": p["d"],
            "zeta": p["zeta"], "tol": p["tol"], "prec": prec,
            "l2_policy": "inputs larger than L2 (A alone is %.1f GB vs 129 MB L2)" % (8 * m * n / 1e9)
            if 8 * m * n > L2_BYTES else "inputs fit in L2 (small config)"}


# DRAM traffic / algorithmic bytes of the double-float LSQR kernels, each from
# one ncu capture of a whole launch (init pass, all iterations, accuracy pass):
#   k_lsqr_df<8>, 1e6 x 500, 35 iterations: 161.64 GB measured / 148.73 GB
#     algorithmic (profiles/lsqr_df_1000000x500.md)
#   k_lsqr_dfp<4>, 250,000 x 2000, 36 iterations: 166.53 GB / 154.46 GB
#     (profiles/lsqr_dfp_250000x2000.md)
# The excess is mostly the float-pair image the first pass writes (8mn, 2.7%),
# which the algorithmic count leaves out.  Every term of both counts is linear
# in the rows and the passes, so a launch on another problem of the same kernel
# moves ratio x its algorithmic bytes.
LSQR_DF_TRAFFIC_RATIO = 161.64 / 148.73
LSQR_DFP_TRAFFIC_RATIO = 166.53 / 154.46


def lsqr_algorithmic_bytes(m, n, iters):
    """Bytes the LSQR kernel must move per launch: per LSQR iteration one read
    of A (8mn), u read+write (16m) and M, M^T (16n^2); plus the initial
    residual pass and the accuracy pass (each 8mn + 16m)."""
    return iters * (8.0 * m * n + 16.0 * m + 16.0 * n * n) + 2 * (8.0 * m * n + 16.0 * m)


def host_cores():
    """Threads this process may run on (sched_getaffinity)."""
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:  # pragma: no cover
        return os.cpu_count() or 1


def cpu_oracle_estimate(A_host, b_host, d, zeta, seed, tol, iters, rows=100_000, lsqr_iters=3, qr_cache=None):
    """Time the oracle on a bounded sample of the workload and scale to one
    full solve: sketch and LSQR passes are linear in m (timed on the first
    `rows` rows and scaled by m/rows); the QR + inverse of the d x (n+1)
    sketch is timed at full size (once, when qr_cache holds it); LSQR is timed
    for `lsqr_iters` iterations and scaled to `iters` (+2 passes for the
    initial residual and the check)."""
    import numpy as np

    import oracle
    m, n = A_host.shape
    rows = min(rows, m)
    As = np.ascontiguousarray(A_host[:rows])
    bs = np.ascontiguousarray(b_host[:rows])
    t0 = time.perf_counter()
    Y = oracle.sketch_apply(As, bs, d, zeta, seed)
    t_sketch = (time.perf_counter() - t0) * (m / rows)
    if qr_cache is not None and "t_qr" in qr_cache:
        t_qr, R = qr_cache["t_qr"], qr_cache["R"]
    else:
        t0 = time.perf_counter()
        R, _, _ = oracle.householder_qr(Y)
        oracle.tri_inverse(R[:n, :n])
        t_qr = time.perf_counter() - t0
        if qr_cache is not None:
            qr_cache.update(t_qr=t_qr, R=R)
    M = oracle.tri_inverse(R[:n, :n])
    x0 = M @ R[:n, n]
    t0 = time.perf_counter()
    oracle.lsqr(As, bs, M, x0, 0.0, lsqr_iters)
    t_l = time.perf_counter() - t0
    # lsqr(maxit=k) = 1 residual pass + k iterations (2 passes each)
    per_pass = t_l / (1 + 2 * lsqr_iters) * (m / rows)
    t_total = t_sketch + t_qr + per_pass * (1 + 2 * iters + 1)
    return {"t_solve_s": t_total, "t_sketch_s": t_sketch, "t_qr_s": t_qr, "t_pass_s": per_pass,
            "sample": f"first {rows} of {m} rows: oracle sketch and {lsqr_iters} LSQR iterations timed and scaled "
                      f"by m/rows; QR+inverse of the full {d}x{n + 1} sketch timed"
                      f"{' once per process' if qr_cache is not None else ''}; LSQR scaled to {iters} "
                      f"iterations + 2 passes"}


# ---------------------------------------------------------------------------
# The headline configuration: 5e6 x 2000 (80 GB), plain and mixed forms.
# ---------------------------------------------------------------------------
C2 = {"m": 5_000_000, "n": 2000, "cond": 1e8, "d": 8000, "zeta": 8, "tol": 1e-12, "seed": 20, "sketch_seed": 7}


def c2_config(m, n, cond, d, zeta, tol):
    """The config dict both arms print (identical keys and values)."""
    return {"workload": f"dense_{m}x{n}_cond{cond:.0e}_d{d}_zeta{zeta}_tol{tol:g}",
            "m": m, "n": n, "d": d, "zeta": zeta, "tol": tol,
            "construction": "A = (G/sqrt(m)) diag(s) H1 H2 built in place, s geometric 1..1/cond; "
                            "b = A x_true + 1e-6 g/||g||",
            "l2_policy": "inputs larger than L2 (A is %.0f GB vs 129 MB L2)" % (8 * m * n / 1e9)}


def c2_shape(args):
    m, n = args.m or C2["m"], args.n or C2["n"]
    cond = args.cond if args.cond != 1e10 else C2["cond"]
    return m, n, cond, 4 * n, C2["zeta"], C2["tol"]


def run_reference(args):
    """The reference arm: the CPU oracle (OpenMP build, all host cores) on a
    bounded sample of this arm's workload (the headline by default), each step
    re-timing the sample's sketch and LSQR passes (the QR of the full-size
    sketch is timed once per process)."""
    world, rank, local = _dist()
    if rank != 0:
        return
    import torch

    import oracle
    from paper_2506_03070_gb300 import synth
    cores = host_cores()
    oracle.use_parallel(cores)
    dev = "cuda" if torch.cuda.is_available() else "cpu"
    if args.config in (0, 1):
        p = make_problem(args.config, dev if args.config == 1 else "cpu")
        m, n = p["A"].shape
        d, zeta, tol, seed = p["d"], p["zeta"], p["tol"], p["seed_sketch"]
        rows = min(m, 60_000)
        Ah, bh = p["A"][:rows].cpu().numpy(), p["b"][:rows].cpu().numpy()
        config = _workload(p, "fp64")
    else:
        m, n, cond, d, zeta, tol = c2_shape(args)
        seed = C2["sketch_seed"]
        rows = min(m, 20_000)
        p = synth.large_problem(m, n, cond, seed=C2["seed"], device=dev, rows=rows)
        Ah, bh = p["A"].cpu().numpy(), p["b"].cpu().numpy()
        config = c2_config(m, n, cond, d, zeta, tol)
    del p
    iters_est = oracle.default_maxit(n, d, tol) // 10  # rate estimate of Sec. 4.3
    cache = {}
    times = []
    info = None
    for step in range(args.warmup + args.steps):
        info = cpu_oracle_estimate(_Scaled(Ah, m), bh, d, zeta, seed, tol, iters_est, rows=rows, lsqr_iters=2,
                                   qr_cache=cache)
        if step >= args.warmup:
            times.append(info["t_solve_s"])
    t = statistics.mean(times)
    val = 1.0 / t
    sample = info["sample"] + f" ({'device-generated rows, copied to host' if dev == 'cuda' else 'host-generated'})"
    line = {"metric": "ls_solves_per_sec", "value": val, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config, "impl": "reference",
            "cpu_baseline": {"kind": "oracle", "value": val, "unit": "solves/s", "cores": cores, "sample": sample},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


class _Scaled:
    """A row-sample of an m-row matrix that reports the full row count."""

    def __init__(self, sample, m):
        self.sample, self.m = sample, m
        self.shape = (m, sample.shape[1])

    def __getitem__(self, key):
        return self.sample[key]


def make_batch(count, device, seed=2024, m_lo=2000, m_hi=50000, n_lo=16, n_hi=128):
    """Config 3: independent problems, m ~ U[m_lo, m_hi], n ~ U[n_lo, n_hi],
    log10 cond ~ U[2, 10], d = 4n, zeta = 8 (cheap construction of synth)."""
    import numpy as np

    from paper_2506_03070_gb300 import synth
    rng = np.random.default_rng(seed)
    probs = []
    for k in range(count):
        m = int(rng.integers(m_lo, m_hi + 1))
        n = int(rng.integers(n_lo, n_hi + 1))
        cond = float(10.0 ** rng.uniform(2, 10))
        p = synth.batched_problem(m, n, cond, seed=seed * 100003 + k, device=device)
        probs.append({"A": p["A"], "b": p["b"], "d": 4 * n, "zeta": 8, "seed": k})
    return probs


def run_batch(args):
    import torch

    import paper_2506_03070_gb300 as P
    import __graft_entry__
    __graft_entry__.build()
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    ctx = P.Context(local)
    probs = make_batch(args.batch, f"cuda:{local}")
    elems = sum(p["A"].numel() for p in probs)
    stream = torch.cuda.current_stream()
    flags = P.FLAG_AUTOTUNE
    for _ in range(args.warmup):
        xs, res = ctx.lsq_solve_batch(probs, tol=1e-12, flags=flags, stream=stream)
    times = []
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xs, res = ctx.lsq_solve_batch(probs, tol=1e-12, flags=flags, stream=stream)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    clocks = sampler.stop()
    import oracle
    worst = 0.0
    for k in range(0, len(probs), max(1, len(probs) // 16)):
        worst = max(worst, oracle.backward_error_kw(probs[k]["A"], probs[k]["b"], xs[k]))
    iters = [r["iters"] for r in res]
    t = statistics.mean(times)
    passes = sum(r["iters"] + 2 for r in res)
    # bytes: every pass reads each problem's A (8 B/entry) once
    abytes = sum(p["A"].numel() * 8 * (r["iters"] + 2) for p, r in zip(probs, res))
    peaks, peak_src = _peaks()
    line = {"metric": "ls_solves_per_sec", "value": len(probs) / (t / 1e3), "unit": "solves/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batched_{len(probs)}_m2000-50000_n16-128_cond1e2-1e10_d4n_zeta8_tol1e-12",
                       "problems": len(probs), "total_A_GB": elems * 8 / 1e9},
            "lsqr_iters_mean": statistics.mean(iters), "lsqr_iters_max": max(iters),
            "pass_shapes": [ctx.lsq_batch_shape_get(k) for k in range(4)],
            "hbm_gbs_A_stream": abytes / (t / 1e3) / 1e9, "hbm_peak_gbs": float(peaks["hbm_gbs"]),
            "accuracy": {"backward_error_kw_max_sampled": worst,
                         "statuses": sorted(set(r["status"] for r in res))},
            "clocks": clocks}
    print(json.dumps(line))


def make_bank(count, bank_bytes, device, seed=4040, m_lo=1e4, m_hi=2e6, n_lo=32, n_hi=1000):
    """Serving workload bodies: `count` problems whose (m, n, cond) form a
    Latin hypercube over log-uniform m in [m_lo, m_hi], n in [n_lo, n_hi] and
    cond in [1e2, 1e10] (cheap construction of synth, d = 4n, zeta = 8),
    trimmed from the largest down until the bodies fit in bank_bytes."""
    import math

    import numpy as np

    from paper_2506_03070_gb300 import synth
    rng = np.random.default_rng(seed)
    strata = [rng.permutation(count) for _ in range(3)]
    specs = []
    for k in range(count):
        q = [(strata[a][k] + rng.uniform()) / count for a in range(3)]
        m = int(round(math.exp(math.log(m_lo) + q[0] * (math.log(m_hi) - math.log(m_lo)))))
        n = int(round(math.exp(math.log(n_lo) + q[1] * (math.log(n_hi) - math.log(n_lo)))))
        cond = 10.0 ** (2 + 8 * q[2])
        specs.append((m, n, cond))
    while sum(8 * m * n for m, n, _ in specs) > bank_bytes:
        specs.remove(max(specs, key=lambda s: s[0] * s[1]))
    import torch
    bank = []
    for k, (m, n, cond) in enumerate(specs):
        p = synth.batched_problem(m, n, cond, seed=seed * 1009 + k, device=device)
        bank.append({"A": p["A"], "b": p["b"], "m": m, "n": n, "d": 4 * n})
        del p
    torch.cuda.empty_cache()
    return bank


def _oracle_cost_model():
    """Oracle seconds per request from unit costs timed on one bounded
    problem (20000 x 200, d = 800): sketch per entry of [A|b], Householder QR
    per flop 2 d (n+1)^2, one LSQR pass per entry of A."""
    import numpy as np

    import oracle
    oracle.use_parallel(host_cores())
    from paper_2506_03070_gb300 import synth
    m, n, d = 20000, 200, 800
    p = synth.batched_problem(m, n, 1e6, seed=3, device="cpu")
    A, b = p["A"].numpy(), p["b"].numpy()
    t0 = time.perf_counter()
    Y = oracle.sketch_apply(A, b, d, 8, 1)
    t_sk = time.perf_counter() - t0
    t0 = time.perf_counter()
    R, _, _ = oracle.householder_qr(Y)
    M = oracle.tri_inverse(R[:n, :n])
    t_qr = time.perf_counter() - t0
    t0 = time.perf_counter()
    oracle.lsqr(A, b, M, M @ R[:n, n], 0.0, 3)
    t_l = time.perf_counter() - t0
    return {"sketch_per_entry": t_sk / (m * (n + 1)), "qr_per_flop": t_qr / (2.0 * d * (n + 1) ** 2),
            "pass_per_entry": t_l / (1 + 2 * 3) / (m * n),
            "sample": "oracle timed on one 20000x200 problem (sketch d=800, QR+inverse, 3 LSQR iterations); "
                      "per-request time = sketch + QR + (2 iters + 2) passes from those unit costs"}


def run_serve(args):
    """Config 4: Poisson arrivals of least-squares problems through
    lsq_submit / lsq_poll.  Latency runs from each request's scheduled
    arrival to the library's completion time stamp."""
    import numpy as np
    import torch

    import paper_2506_03070_gb300 as P
    import __graft_entry__
    __graft_entry__.build()
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = f"cuda:{local}"
    bank = make_bank(args.bank_count, int(args.bank_gb * 1e9), dev)
    ctx = P.Context(local)
    ctx.lsq_serve_config(arena_bytes=int(args.arena_gb * 1e9), cta_bytes=args.cta_mb * 2.0 ** 20,
                         max_group=args.max_group)
    # the autotuner picks the small-problem (n <= 256) pass shapes, once per
    # n-range, on small synthetic problems (untimed)
    from paper_2506_03070_gb300 import synth
    small = []
    for j, n in enumerate((24, 48, 100, 200)):
        for rep in range(4):
            p = synth.batched_problem(20000, n, 1e4, seed=900 + 10 * j + rep, device=dev)
            small.append(dict(A=p["A"], b=p["b"], d=4 * n, seed=1))
    ctx.lsq_solve_batch(small, tol=1e-12, flags=P.FLAG_AUTOTUNE)
    del small
    rng = np.random.default_rng(args.serve_seed)

    def stream_run(nreq, rate, tag):
        body = rng.integers(0, len(bank), nreq)
        gaps = rng.exponential(1.0 / rate, nreq)
        arrive = np.cumsum(gaps) - gaps[0]
        xs = [torch.empty(bank[k]["n"], dtype=torch.float64, device=dev) for k in body]
        torch.cuda.synchronize()
        out = [None] * nreq
        open_t = {}
        t0 = time.monotonic() + 0.05
        nxt = 0
        ndone = 0
        while ndone < nreq:
            now = time.monotonic()
            while nxt < nreq and t0 + arrive[nxt] <= now:
                bk = bank[body[nxt]]
                open_t[nxt] = ctx.lsq_submit(bk["A"], bk["b"], bk["d"], seed=nxt + 1, tol=1e-12, x=xs[nxt])
                nxt += 1
            for i in list(open_t)[:256]:
                r = ctx.lsq_poll(open_t[i])
                if r is not None:
                    out[i] = r
                    del open_t[i]
                    ndone += 1
            if not open_t:
                time.sleep(min(1e-4, max(0.0, t0 + arrive[nxt] - time.monotonic()) if nxt < nreq else 1e-4))
        lat = np.array([out[i][2]["t_done_s"] - (t0 + arrive[i]) for i in range(nreq)]) * 1e3
        t_end = max(out[i][2]["t_done_s"] for i in range(nreq))
        span = t_end - t0
        statuses = sorted(set(int(o[0]) for o in out))
        abytes = sum(8.0 * bank[body[i]]["m"] * bank[body[i]]["n"] * (out[i][2]["iters"] + 2) for i in range(nreq))
        # accuracy on a sample (outside the timed region)
        import oracle
        worst = 0.0
        for i in range(0, nreq, max(1, nreq // 12)):
            bk = bank[body[i]]
            if 8 * bk["m"] * bk["n"] <= 2e9:  # the check itself needs a copy of A
                worst = max(worst, oracle.backward_error_kw(bk["A"], bk["b"], out[i][1]))
        groups = [o[2]["group_blocks"] for o in out]
        # block-time per phase (group size x device duration) as a share of
        # all resident blocks over the run's span
        grid = ctx.lsq_serve_stats()["grid_blocks"]
        share = {}
        for key in ("t_group_wait_ms", "t_sketch_ms", "t_precond_ms", "t_lsqr_ms"):
            share[key.replace("t_", "").replace("_ms", "")] = sum(o[2]["group_blocks"] * o[2][key] for o in out) \
                / 1e3 / (grid * span)
        return {"tag": tag, "requests": nreq, "rate_per_s": rate, "solves_per_s": nreq / span, "span_s": span,
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                               "mean": float(lat.mean()), "max": float(lat.max())},
                "hbm_gbs_A_stream": abytes / span / 1e9, "statuses": statuses,
                "backward_error_kw_max_sampled": worst,
                "group_blocks": {"min": min(groups), "median": float(np.median(groups)), "max": max(groups)},
                "block_time_share": share,
                "lsqr_iters_mean": float(np.mean([o[2]["iters"] for o in out])), "body": body}

    # warm-up: a few requests through the server
    warm = stream_run(min(32, args.requests), args.rate, "warmup")
    launches0 = ctx.lsq_serve_stats()["server_launches"]
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    sat = stream_run(args.requests, args.rate, "saturated")
    clocks = sampler.stop()
    stats = ctx.lsq_serve_stats()
    launches = stats["server_launches"] - launches0
    sub = stream_run(args.sub_requests, args.sub_rate, "sub_saturation") if args.sub_requests > 0 else None
    # sequential plain solves (whole-GPU lsq_solve, one problem at a time) on
    # the same request mix, a bounded sample
    seq_idx = sat["body"][: args.seq_sample]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for j, k in enumerate(seq_idx):
        bk = bank[k]
        ctx.lsq_solve(bk["A"], bk["b"], bk["d"], seed=j + 1, tol=1e-12)
    t_seq = time.perf_counter() - t0
    seq_rate = len(seq_idx) / t_seq
    peaks, peak_src = _peaks()
    peak = float(peaks["hbm_gbs"])
    for r in (warm, sat, sub):
        if r is not None:
            r.pop("body", None)
    line = {"metric": "ls_solves_per_sec", "value": sat["solves_per_s"], "unit": "solves/s", "n_gpus": 1,
            "steps": args.requests, "warmup": warm["requests"], "ms_per_step": 1e3 / sat["solves_per_s"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"serving_poisson{args.rate:g}_{args.requests}req_m1e4-2e6_n32-1000"
                                   f"_cond1e2-1e10_d4n_zeta8_tol1e-12",
                       "bank_bodies": len(bank), "bank_GB": sum(8 * b["m"] * b["n"] for b in bank) / 1e9,
                       "arena_GB": args.arena_gb,
                       "l2_policy": "inputs larger than L2 (bodies up to %.1f GB)" %
                                    (max(8 * b["m"] * b["n"] for b in bank) / 1e9)},
            "latency_ms": sat["latency_ms"],
            "roofline": {"bound": "hbm", "kernel": "k_serve", "achieved": sat["hbm_gbs_A_stream"], "peak": peak,
                         "unit": "GB/s", "frac": sat["hbm_gbs_A_stream"] / peak, "traffic": None,
                         "peak_source": f"{peak_src} hbm_gbs", "note": "A-stream bytes (8mn per pass) / wall span"},
            "gpu_launches": launches,
            "saturated": sat, "sub_saturation": sub,
            "sequential_plain_solves": {"solves_per_s": seq_rate, "sample": len(seq_idx),
                                        "serving_over_sequential": sat["solves_per_s"] / seq_rate},
            "serve_stats": stats, "pass_shapes": [ctx.lsq_batch_shape_get(k) for k in range(4)], "clocks": clocks}
    if not args.no_cpu_baseline:
        cm = _oracle_cost_model()
        tot = 0.0
        for k in seq_idx:
            bk = bank[k]
            m, n, d = bk["m"], bk["n"], bk["d"]
            it = 2 * (10 * math.ceil(math.log(1e-12) / math.log(math.sqrt(n / d)))) // 10
            tot += (cm["sketch_per_entry"] * m * (n + 1) + cm["qr_per_flop"] * 2.0 * d * (n + 1) ** 2
                    + cm["pass_per_entry"] * m * n * (2 * it + 2))
        line["cpu_baseline"] = {"value": len(seq_idx) / tot, "unit": "solves/s", "cores": host_cores(),
                                "kind": "oracle",
                                "sample": cm["sample"] + f"; applied to the first {len(seq_idx)} requests "
                                          "(an extrapolation)"}
    print(json.dumps(line))
    ctx.close()


def _mem_available_bytes():
    try:
        for line in open("/proc/meminfo"):
            if line.startswith("MemAvailable:"):
                return int(line.split()[1]) * 1024
    except OSError:
        pass
    return 0


def sketch_slabs(d, ncol):
    """Launches of the FP64 sketch: one per column slab of at most 48e6 bytes
    of Y (a multiple of 32 columns), as the library splits it."""
    w = max(32, int(48e6 / (d * 8.0)) // 32 * 32)
    return 1 if w >= ncol else -(-ncol // w)


def launches_per_solve(n, d, prec, blocked):
    """Kernels of this library one lsq_solve launches: sketch (FP64: one per
    column slab; the mixed form: the chunk-sum kernel and the pair-to-FP64
    pass), column-major copy, QR (unblocked: 1 kernel; blocked, per 64-column
    panel of the n columns: the panel kernel, four slicing kernels, three
    tensor-core GEMMs and T -- the b column always leaves a trailing update),
    R extraction, R^T, inverse, transpose, x0, and the LSQR kernel (with the
    accuracy pass).  Checked against the ncu launch list of the default bench
    line (298 per plain solve, 297 per mixed one at 5e6 x 2000)."""
    qr = 9 * ((n + 63) // 64) if blocked else 1
    sketch = 2 if prec == 1 else sketch_slabs(d, n + 1)
    return sketch + 1 + qr + 5 + 1


def run_headline(args):
    """The largest single-GPU configuration (5e6 x 2000, 80 GB): the plain FP64
    form is the headline value; the mixed form solves the same A and b."""
    import numpy as np
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_03070_gb300 as P
    from paper_2506_03070_gb300 import synth

    m, n, cond, d, zeta, tol = c2_shape(args)
    dev = f"cuda:{local}"
    p = synth.large_problem(m, n, cond, seed=C2["seed"], device=dev)
    A, b = p["A"], p["b"]
    del p
    torch.cuda.synchronize()
    ctx = P.Context(local)
    stream = torch.cuda.current_stream()
    flags = P.FLAG_TIMING

    def solve(prec):
        return ctx.lsq_solve(A, b, d, zeta=zeta, seed=C2["sketch_seed"], tol=tol, prec=prec, flags=flags,
                             stream=stream)

    for _ in range(args.warmup):
        x, info = solve(P.PREC_FP64)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, infos = [], []
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = solve(P.PREC_FP64)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        infos.append(info)
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(total_ms, dev)
    value = world * args.steps / (t_max / 1e3)
    xp = x.clone()

    # the mixed form on the same A and b (extra key; fewer timed solves)
    km = max(1, min(args.steps, 5))
    for _ in range(min(args.warmup, 2)):
        xm, im = solve(P.PREC_MIXED)
    mixed_ms, minfos = [], []
    for _ in range(km):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xm, im = solve(P.PREC_MIXED)
        e1.record(stream)
        e1.synchronize()
        mixed_ms.append(e0.elapsed_time(e1))
        minfos.append(im)
    bn = float(torch.linalg.vector_norm(b))
    dist_mp = float(torch.linalg.vector_norm(A @ (xm - xp))) / bn
    # accuracy of the mixed solution by the same FP64 pass
    chk_m = ctx.lsq_check(A, b, xm)

    # the plain solve with every LSQR pass on the FP64 pipe (LSQ_FLAG_NATIVE_FP64;
    # extra key, one warm-up and one timed solve)
    native = None
    if not args.no_native:
        def solve_native():
            return ctx.lsq_solve(A, b, d, zeta=zeta, seed=C2["sketch_seed"], tol=tol, prec=P.PREC_FP64,
                                 flags=flags | P.FLAG_NATIVE_FP64, stream=stream)
        solve_native()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        xn, inn = solve_native()
        e1.record(stream)
        e1.synchronize()
        nat_ms = e0.elapsed_time(e1)
        t_ln = inn["t_lsqr_ms"]
        native = {"solves_per_s": 1e3 / nat_ms, "ms_per_solve": nat_ms, "steps": 1, "lsqr_iters": inn["iters"],
                  "phases_ms": {"sketch": inn["t_sketch_ms"], "precond": inn["t_precond_ms"],
                                "lsqr_and_check": t_ln, "check": inn["t_check_ms"]},
                  "lsqr_gbs_algorithmic": lsqr_algorithmic_bytes(m, n, inn["iters"]) / (t_ln / 1e3) / 1e9,
                  "rel_residual_distance_to_plain": float(torch.linalg.vector_norm(A @ (xn - xp))) / bn,
                  "backward_error_pre": inn["backward_error_pre"], "status": inn["status"],
                  "dtype": "LSQR passes in native FP64 (FP64 pipe, two FMA per entry); sketch and QR as plain"}
        del xn

    peaks, peak_src = _peaks()
    peak = float(peaks["hbm_gbs"])
    it = statistics.mean(i["iters"] for i in infos)
    t_lsqr = statistics.mean(i["t_lsqr_ms"] for i in infos)
    t_check = statistics.mean(i["t_check_ms"] for i in infos)
    alg = lsqr_algorithmic_bytes(m, n, it)
    achieved = alg / (t_lsqr / 1e3) / 1e9
    alg_iter = it * (8.0 * m * n + 16.0 * m + 16.0 * n * n) + (8.0 * m * n + 16.0 * m)
    achieved_iter = alg_iter / ((t_lsqr - t_check) / 1e3) / 1e9 if t_lsqr > t_check else None
    sketch_ms = statistics.mean(i["t_sketch_ms"] for i in infos)
    precond_ms = statistics.mean(i["t_precond_ms"] for i in infos)
    blocked = 8 * d * (n + 1) >= (32 << 20)
    per_solve = launches_per_solve(n, d, 0, blocked)

    def phase(ii):
        return {"sketch": statistics.mean(i["t_sketch_ms"] for i in ii),
                "precond": statistics.mean(i["t_precond_ms"] for i in ii),
                "lsqr_and_check": statistics.mean(i["t_lsqr_ms"] for i in ii),
                "check": statistics.mean(i["t_check_ms"] for i in ii)}

    mixed_val = 1e3 / statistics.mean(mixed_ms)
    line = {
        "metric": "ls_solves_per_sec", "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": c2_config(m, n, cond, d, zeta, tol),
        "lsqr_arith": "df47 (A as float pairs of its top 47 bits, pair sums; FP64 recurrences; native FP64 check)",
        "roofline": {"bound": "hbm", "kernel": "k_lsqr_dfp<4> (LSQR + accuracy pass, one launch per solve)",
                     "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": LSQR_DFP_TRAFFIC_RATIO * alg,
                     "traffic_source": "ncu capture ratio (profiles/lsqr_dfp_250000x2000.md, 250,000 x 2000) x this "
                                       "launch's algorithmic bytes: both scale with rows x passes",
                     "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json, of measured)",
                     "algorithmic_bytes_per_launch": alg,
                     "achieved_excluding_check": achieved_iter,
                     "check_pass_ms": t_check,
                     "check_pass_gbs": (8.0 * m * n + 16.0 * m) / (t_check / 1e3) / 1e9 if t_check > 0 else None},
        "gpu_launches": per_solve * args.steps,
        "latency_ms": {"p50": statistics.median(step_ms),
                       "p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
        "phases_ms": {"sketch": sketch_ms, "precond": precond_ms, "lsqr_and_check": t_lsqr, "check": t_check},
        "sketch_gbs": (8.0 * m * (n + 1) + 8.0 * d * (n + 1)) / (sketch_ms / 1e3) / 1e9,
        "lsqr_iters": it,
        "accuracy": {"backward_error_ne": infos[-1]["backward_error_ne"],
                     "backward_error_pre": infos[-1]["backward_error_pre"],
                     "gate_bound": min(infos[-1]["backward_error_ne"], infos[-1]["backward_error_pre"]),
                     "note": "FP64 accuracy pass on the device: Stewart's bound ||A^T r||/(||A||_F ||r||) and "
                             "||M^T A^T r||/(||A||_F ||x||) (bounds the Karlson-Walden estimate up to the "
                             "sketch distortion); the oracle's KW needs a QR of [||x|| A; ||r|| I] (80 GB)"},
        "mixed": {"solves_per_s": mixed_val, "ms_per_solve": statistics.mean(mixed_ms), "steps": km,
                  "lsqr_iters": statistics.mean(i["iters"] for i in minfos), "phases_ms": phase(minfos),
                  "precond_fallback": minfos[-1]["precond_fallback"], "status": minfos[-1]["status"],
                  "mixed_over_plain": mixed_val / value * world,
                  "rel_residual_distance_to_plain": dist_mp,
                  "backward_error_ne": chk_m["backward_error_ne"], "backward_error_pre": minfos[-1][
                      "backward_error_pre"],
                  "dtype": "sketch: terms added in FP32 (chunk sums of ~16 terms per entry, combined in FP64); QR: FP64 (tcgen05 trailing updates, FP32 accumulation); LSQR: df47 + FP64 recurrences"},
        "clocks": clocks,
    }
    if native is not None:
        line["native_fp64"] = native

    # e2e: host (pinned) A, b through the same C ABI, copies inside the timed region
    e2e = None
    need = 8 * m * n + 8 * m
    if not args.no_e2e and _mem_available_bytes() > 1.25 * need:
        try:
            Ah = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
            bh = torch.empty((m,), dtype=torch.float64, pin_memory=True)
            Ah.copy_(A)
            bh.copy_(b)
            Anp, bnp = Ah.numpy(), bh.numpy()
            xh = np.empty(n, dtype=np.float64)
            ctx.lsq_solve(Anp, bnp, d, zeta=zeta, seed=C2["sketch_seed"], tol=tol, flags=flags, x=xh)
            k2 = max(1, min(args.steps, 3))
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(k2):
                ctx.lsq_solve(Anp, bnp, d, zeta=zeta, seed=C2["sketch_seed"], tol=tol, flags=flags, x=xh)
            t_e2e = time.perf_counter() - t0
            e2e = {"value": world * k2 / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": 8 * m * n + 8 * m,
                   "d2h_bytes_per_step": 8 * n + 4096, "steps": k2}
            del Ah, bh, Anp, bnp
        except Exception as exc:  # pinned allocation of the whole problem refused
            e2e = {"value": None, "unit": "solves/s", "h2d_bytes_per_step": need, "d2h_bytes_per_step": 8 * n,
                   "unavailable": f"{type(exc).__name__}: {exc}"[:200]}
    elif not args.no_e2e:
        e2e = {"value": None, "unit": "solves/s", "h2d_bytes_per_step": need, "d2h_bytes_per_step": 8 * n,
               "unavailable": f"host memory available ({_mem_available_bytes() / 1e9:.0f} GB) below the pinned "
                              f"copy of A and b ({need / 1e9:.0f} GB)"}
    line["e2e"] = e2e

    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle
        cores = host_cores()
        oracle.use_parallel(cores)
        rows = min(m, 20_000)
        Ah2 = A[:rows].cpu().numpy()
        bh2 = b[:rows].cpu().numpy()
        est = cpu_oracle_estimate(_Scaled(Ah2, m), bh2, d, zeta, C2["sketch_seed"], tol, int(round(it)), rows=rows,
                                  lsqr_iters=2)
        line["cpu_baseline"] = {"value": 1.0 / est["t_solve_s"], "unit": "solves/s", "cores": cores,
                                "kind": "oracle", "sample": est["sample"] + " (OpenMP build, -O3 -fopenmp)"}
    del A, b, x, xp, xm
    ctx.close()
    torch.cuda.empty_cache()

    if rank == 0 and world == 1 and not args.no_c1:
        # the 2,000,000 x 500 coherent-row configuration as an extra key
        import copy
        a1 = copy.copy(args)
        a1.config, a1.m, a1.n, a1.cond, a1.steps, a1.warmup = 1, 0, 0, 1e10, min(args.steps, 5), min(args.warmup, 3)
        a1.no_e2e, a1.no_cpu_baseline = True, True
        c1 = run_gpu(a1, emit=False)
        line["c1"] = {k: c1[k] for k in ("value", "ms_per_step", "config", "roofline", "phases_ms", "lsqr_iters",
                                         "accuracy", "auto_d", "hbm", "sketch_gbs") if k in c1}
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def run_sparse(args):
    """The paper's 5e5_500_sparse workload (Sec. 4.1): 500,000 x 500, entries
    nonzero with probability 1/100, random signs; d = 2000, zeta = 8."""
    import torch

    import paper_2506_03070_gb300 as P
    import __graft_entry__
    __graft_entry__.build()
    from paper_2506_03070_gb300 import synth
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    m, n, d = args.m or 500_000, args.n or 500, 2000
    p = synth.sparse_sign_problem(m, n, 0.01, seed=55, device=f"cuda:{local}")
    ctx = P.Context(local)
    stream = torch.cuda.current_stream()
    nnz = p["values"].numel()

    def solve():
        return ctx.lsq_solve_csr(p["row_ptr"], p["col_idx"], p["values"], p["b"], n, d, seed=8, tol=1e-12,
                                 flags=P.FLAG_TIMING, stream=stream)

    for _ in range(args.warmup):
        x, info = solve()
    ms = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = solve()
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    import oracle
    A = synth.csr_to_dense(p)
    bwd = oracle.backward_error_kw(A, p["b"], x)
    del A
    t = statistics.mean(ms)
    # bytes per pass: values (8) + column indices (4) per nonzero, row offsets and u (8 + 16 per row)
    pass_bytes = 12.0 * nnz + 24.0 * m
    it = info["iters"]
    lsqr_gbs = pass_bytes * (it + 2) / (info["t_lsqr_ms"] / 1e3) / 1e9
    peaks, peak_src = _peaks()
    line = {"metric": "ls_solves_per_sec", "value": 1e3 / t, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"sparse_sign_{m}x{n}_p0.01_d{d}_zeta8_tol1e-12", "nnz": nnz},
            "phases_ms": {"sketch": info["t_sketch_ms"], "precond": info["t_precond_ms"],
                          "lsqr_and_check": info["t_lsqr_ms"]},
            "lsqr_iters": it, "lsqr_pass_gbs": lsqr_gbs, "hbm_peak_gbs": float(peaks["hbm_gbs"]),
            "accuracy": {"backward_error_kw": bwd}}
    print(json.dumps(line))
    ctx.close()


def run_gpu(args, emit=True):
    """Configs 0 and 1 (one problem per rank).  Returns the JSON line (and
    prints it when emit)."""
    import numpy as np
    import torch

    world, rank, local = _dist()
    torch.cuda.set_device(local)
    if world > 1 and emit:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_2506_03070_gb300 as P

    ctx = P.Context(local)
    p = make_problem(args.config, f"cuda:{local}", args.m, args.n, args.cond, args.coherent)
    A, b = p["A"], p["b"]
    m, n = A.shape
    d, zeta, tol, seed = p["d"], p["zeta"], p["tol"], p["seed_sketch"]
    prec = 0 if args.prec == "fp64" else 1
    flags = P.FLAG_TIMING | (P.FLAG_NATIVE_FP64 if args.native else 0)
    stream = torch.cuda.current_stream()

    def solve():
        return ctx.lsq_solve(A, b, d, zeta=zeta, seed=seed, tol=tol, prec=prec, flags=flags, stream=stream)

    for _ in range(args.warmup):
        x, info = solve()
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, lsqr_ms, sketch_ms, precond_ms, iters = [], [], [], [], []
    torch.cuda.synchronize()
    ev0.record(stream)
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        x, info = solve()
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        lsqr_ms.append(info["t_lsqr_ms"])
        sketch_ms.append(info["t_sketch_ms"])
        precond_ms.append(info["t_precond_ms"])
        iters.append(info["iters"])
    ev1.record(stream)
    torch.cuda.synchronize()
    clocks = sampler.stop()
    total_ms = ev0.elapsed_time(ev1)
    t_max = max_over_ranks(total_ms, f"cuda:{local}")
    value = world * args.steps / (t_max / 1e3)

    # accuracy of the last solution (outside the timed region)
    import oracle
    bwd = oracle.backward_error_kw(A, b, x)
    xt = p["x_true"]
    fwd_res = float(torch.linalg.vector_norm(A @ (x - xt)) / torch.linalg.vector_norm(b))

    # e2e: host (pinned) A, b through the same C ABI, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        Ah = torch.empty((m, n), dtype=torch.float64, pin_memory=True)
        Ah.copy_(A)
        bh = torch.empty((m,), dtype=torch.float64, pin_memory=True)
        bh.copy_(b)
        Anp, bnp = Ah.numpy(), bh.numpy()
        xh = np.empty(n, dtype=np.float64)
        ctx.lsq_solve(Anp, bnp, d, zeta=zeta, seed=seed, tol=tol, prec=prec, flags=flags, x=xh)
        k2 = max(1, min(args.steps, 3))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(k2):
            ctx.lsq_solve(Anp, bnp, d, zeta=zeta, seed=seed, tol=tol, prec=prec, flags=flags, x=xh)
        t_e2e = time.perf_counter() - t0
        e2e = {"value": world * k2 / t_e2e, "unit": "solves/s", "h2d_bytes_per_step": 8 * m * n + 8 * m,
               "d2h_bytes_per_step": 8 * n + 4096, "steps": k2}
        del Ah, bh

    peaks, peak_src = _peaks()
    it_mean = statistics.mean(iters)
    lsqr_avg_ms = statistics.mean(lsqr_ms)
    alg_bytes = lsqr_algorithmic_bytes(m, n, it_mean)
    achieved = alg_bytes / (lsqr_avg_ms / 1e3) / 1e9
    peak = float(peaks["hbm_gbs"])
    sketch_bytes = 8.0 * m * (n + 1) + 8.0 * d * (n + 1)
    line = {
        "metric": "ls_solves_per_sec", "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _workload(p, args.prec),
        "roofline": {"bound": "hbm", "kernel": (("k_lsqr_native_wide" if n > 512 else "k_lsqr_native") if args.native
                                                else ("k_lsqr_dfp" if n > 512 else "k_lsqr_df")),
                     "achieved": achieved, "peak": peak,
                     "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None if args.native else (LSQR_DFP_TRAFFIC_RATIO if n > 512 else LSQR_DF_TRAFFIC_RATIO)
                     * alg_bytes,
                     "traffic_source": "ncu capture ratio x this launch's algorithmic bytes ("
                     + ("profiles/lsqr_dfp_250000x2000.md" if n > 512 else "profiles/lsqr_df_1000000x500.md") + ")",
                     "peak_source": f"{peak_src} hbm_gbs (MEASURED_PEAKS.json)" if peak_src == "measured"
                     else "fallback 6.8 TB/s"},
        "gpu_launches": 8 * args.steps,
        "latency_ms": {"p50": statistics.median(step_ms),
                       "p99": sorted(step_ms)[min(len(step_ms) - 1, int(0.99 * len(step_ms)))]},
        "phases_ms": {"sketch": statistics.mean(sketch_ms), "precond": statistics.mean(precond_ms),
                      "lsqr_and_check": lsqr_avg_ms},
        "sketch_gbs": sketch_bytes / (statistics.mean(sketch_ms) / 1e3) / 1e9,
        "lsqr_iters": it_mean,
        "accuracy": {"backward_error_kw": bwd, "backward_error_ne": info["backward_error_ne"],
                     "rel_residual_distance_to_x_true": fwd_res},
        "clocks": clocks,
        "e2e": e2e,
    }
    if rank == 0 and world == 1 and not args.no_auto_d:
        # the same A and b with the embedding dimension chosen by lsq_choose_d
        # (Sec. 4.3 balance with this GPU's measured constants); the headline
        # value above keeps the configuration's d
        d_auto = ctx.lsq_choose_d(m, n, tol)
        for _ in range(2):
            xa, ia = ctx.lsq_solve(A, b, 0, zeta=zeta, seed=seed, tol=tol, prec=prec, flags=flags, stream=stream)
        ms_a = []
        for _ in range(max(1, min(args.steps, 3))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            xa, ia = ctx.lsq_solve(A, b, 0, zeta=zeta, seed=seed, tol=tol, prec=prec, flags=flags, stream=stream)
            e1.record(stream)
            e1.synchronize()
            ms_a.append(e0.elapsed_time(e1))
        line["auto_d"] = {"d": ia["d_used"], "chosen": d_auto, "solves_per_s": 1e3 / statistics.mean(ms_a),
                          "ms_per_solve": statistics.mean(ms_a), "lsqr_iters": ia["iters"],
                          "phases_ms": {"sketch": ia["t_sketch_ms"], "precond": ia["t_precond_ms"],
                                        "lsqr_and_check": ia["t_lsqr_ms"]},
                          "backward_error_kw": oracle.backward_error_kw(A, b, xa)}
    if rank == 0 and world == 1 and not args.no_auto_d:
        # the same problem solved with heavy-ball momentum (Algorithm 6) instead of LSQR
        for _ in range(2):
            xh, ih = ctx.lsq_solve(A, b, d, zeta=zeta, seed=seed, tol=tol, prec=prec, flags=flags | P.FLAG_HBM,
                                   stream=stream, allow_noconv=True)
        ms_h = []
        for _ in range(max(1, min(args.steps, 3))):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            xh, ih = ctx.lsq_solve(A, b, d, zeta=zeta, seed=seed, tol=tol, prec=prec, flags=flags | P.FLAG_HBM,
                                   stream=stream, allow_noconv=True)
            e1.record(stream)
            e1.synchronize()
            ms_h.append(e0.elapsed_time(e1))
        line["hbm"] = {"solves_per_s": 1e3 / statistics.mean(ms_h), "ms_per_solve": statistics.mean(ms_h),
                       "iters": ih["iters"], "status": ih["status"], "stop": ih["stop"],
                       "lsqr_phase_ms": ih["t_lsqr_ms"], "backward_error_kw": oracle.backward_error_kw(A, b, xh)}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        import oracle as orc
        cores = host_cores()
        orc.use_parallel(cores)
        rows = 100_000 if m > 100_000 else m
        Ah2 = A[:rows].cpu().numpy()
        bh2 = b[:rows].cpu().numpy()
        est = cpu_oracle_estimate(_Scaled(Ah2, m), bh2, d, zeta, seed, tol, int(round(it_mean)), rows=rows,
                                  lsqr_iters=2)
        line["cpu_baseline"] = {"value": 1.0 / est["t_solve_s"], "unit": "solves/s", "cores": cores, "kind": "oracle",
                                "sample": est["sample"] + " (OpenMP build, -O3 -fopenmp)"}
        # the same estimate on one thread (C0 and C1)
        orc.set_threads(1)
        est1 = cpu_oracle_estimate(_Scaled(Ah2, m), bh2, d, zeta, seed, tol, int(round(it_mean)), rows=rows,
                                   lsqr_iters=2)
        orc.set_threads(cores)
        line["cpu_baseline"]["value_1_thread"] = 1.0 / est1["t_solve_s"]
    if rank == 0 and emit:
        print(json.dumps(line))
    if world > 1 and emit:
        torch.distributed.destroy_process_group()
    ctx.close()
    return line


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=2, choices=[0, 1, 2, 3, 4],
                    help="2 (default): the 5e6 x 2000 headline with plain and mixed forms; 1: 2e6 x 500; "
                         "0: 20000 x 200; 3: batched; 4: serving")
    ap.add_argument("--requests", type=int, default=10000, help="serving: requests in the Poisson stream")
    ap.add_argument("--rate", type=float, default=2000.0, help="serving: mean arrival rate (1/s)")
    ap.add_argument("--sub-requests", type=int, default=1000, help="serving: requests of the extra sub-saturation run")
    ap.add_argument("--sub-rate", type=float, default=150.0, help="serving: arrival rate of the extra run")
    ap.add_argument("--bank-count", type=int, default=64, help="serving: problem bodies (Latin hypercube)")
    ap.add_argument("--bank-gb", type=float, default=60.0, help="serving: device memory for problem bodies")
    ap.add_argument("--arena-gb", type=float, default=150.0, help="serving: HBM budget for admitted requests")
    ap.add_argument("--seq-sample", type=int, default=100, help="serving: requests timed as sequential solves")
    ap.add_argument("--serve-seed", type=int, default=7)
    ap.add_argument("--cta-mb", type=float, default=0.0, help="serving: MiB of A per block of a group (0: default)")
    ap.add_argument("--max-group", type=int, default=0, help="serving: most blocks per request (0: default)")
    ap.add_argument("--batch", type=int, default=4096, help="problems in the batched config")
    ap.add_argument("--prec", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--no-native", action="store_true", help="skip the native-FP64 LSQR solve of the headline")
    ap.add_argument("--native", action="store_true", help="LSQR matvecs on the native FP64 pipe")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--m", type=int, default=0, help="custom problem rows (profiling runs)")
    ap.add_argument("--cond", type=float, default=1e10, help="condition number of a custom problem")
    ap.add_argument("--coherent", type=float, default=0.01, help="fraction of rows scaled x1e4 (custom problem)")
    ap.add_argument("--n", type=int, default=0, help="custom problem columns (profiling runs)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-auto-d", action="store_true", help="skip the extra solve with the chosen embedding dimension")
    ap.add_argument("--sparse", action="store_true", help="the paper's 5e5_500_sparse workload (CSR path)")
    ap.add_argument("--no-c1", action="store_true", help="headline: skip the extra 2e6 x 500 solves")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.config == 2 and not args.sparse:
        run_headline(args)
    elif args.config == 3:
        run_batch(args)
    elif args.config == 4:
        run_serve(args)
    elif args.sparse:
        run_sparse(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
