#!/usr/bin/env python3
"""Benchmark: space-time DOF/s of MGRIT at a 1e-10 relative residual.

Workload (one "step" = one complete solve to tol 1e-10): ERK3+U3 on periodic
[-1, 1), nx = 4096, nt = 16384, c = 0.85 * 1.62589 (85% of Table 1's limit),
u0 = random Fourier field (modes 1..64, N(0,1)/k^2, seed 2), zero initial
iterate, V-cycle with 4 levels and m = 8, least-squares Psi on every level,
FP32 second F-relaxation with FP64 residual / coarse solve / test.  Also timed
on the same GPU: the FP64 variant, two-level m = 8, and plain FP64
sequential time stepping.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  Multi-GPU runs are independent replicas
(the solve has no data-parallel exchange on one box): value = total DOF of all
ranks / max-over-ranks time.  Its roofline object is for the level-1 FCF in
the form the autotuner picked: the stencil form against the FP64 FMA peak, the
Fourier-space form against the FP64 pipe's issue rate times that form's flops
per operation (fourier_fcf_work).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

NX, NT, P, M, LEVELS = 4096, 16384, 3, 8, 4
CMAX3 = 1.62589
CFL = 0.85 * CMAX3
TOL = 1e-10
METRIC = "space-time DOF/s at 1e-10 rel. residual vs GPU seq. stepping; p50/p99 latency"
# FP64 peak from unit counts and clocks: 152 SMs x 2 DFMA/clk/SM x 2 flop x 2.070 GHz
FP64_PEAK_TFLOPS = 152 * 4 * 2.070e9 / 1e12
# the FP64 pipe's issue rate: 152 SMs x 2 operations (add, mul, fma, conversion) per clock x 2.070 GHz
FP64_OPS_PEAK = 152 * 2 * 2.070e9


def fourier_fcf_work(nx):
    """FP64 operations and flops per interval of the level-1 FCF's FP64 pass in
    Fourier space (Phi^m c_{j-1} by a half-length complex FFT of the slab):
    forward and inverse radix-4 passes of h/4 butterflies (eight complex
    additions each, and three complex products, 2 mul + 2 fma = 6 flops each,
    where the twiddles are not 1), a radix-2 pass of span 1 (two complex
    additions per butterfly) when log2 h is odd, 32 operations (40 flops) per
    mode pair of the split / symbol product / recombination, and per point the
    subtraction rho = c' - c and its rounding to FP32."""
    h = nx // 2
    logh = h.bit_length() - 1
    ops = flops = 0
    q = h // 4
    while q >= 1:
        nontrivial = (h // 4) * (q - 1) // q
        ops += 2 * (16 * (h // 4) + 12 * nontrivial)
        flops += 2 * (16 * (h // 4) + 18 * nontrivial)
        q //= 4
    if logh % 2:
        ops += 2 * 4 * (h // 2)
        flops += 2 * 4 * (h // 2)
    pairs = h // 2 + 1
    return ops + 32 * pairs + 2 * nx, flops + 40 * pairs + nx


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


# --------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi samples during the timed region (median SM clock, reasons)."""
    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, dev):
        self.dev, self.samples, self.proc = dev, [], None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.samples)}


# --------------------------------------------------------- oracle (CPU)

CPU_NT_SAMPLE = 1024     # the oracle's sample of the horizon (the first 1/16)


def oracle_sample(nt_sample=CPU_NT_SAMPLE, repeats=1):
    """Oracle FCF-MGRIT on the headline's scheme, CFL, u0, tolerance and
    hierarchy shape over the first nt_sample steps of the horizon (one
    thread); returns (DOF/s, seconds, iterations).  Psi setup excluded."""
    from oracle import mgrit as omg
    from oracle import psi as opsi
    from oracle import stepping
    u0 = workloads.fourier_field(NX)
    st = stepping.FineStep("ERK", P, CFL, NX)
    ops = opsi.build_hierarchy("ERK", P, CFL, NX, nt_sample, M, LEVELS, rule="auto")
    lev = omg.make_levels(st, M, [o.diag for o in ops])
    dt, it = 0.0, 0
    for _ in range(repeats):
        U = omg.zero_iterate(u0, nt_sample)
        t0 = time.perf_counter()
        it, _ = omg.solve(lev, U, tol=TOL)
        dt += time.perf_counter() - t0
    return NX * nt_sample * repeats / dt, dt, it


def _oracle_worker(args):
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    if args[0] == 0:                          # warm-up: imports only
        from oracle import mgrit  # noqa: F401
        return None
    return oracle_sample(*args)


def oracle_all_cores(nt_sample=CPU_NT_SAMPLE, repeats=2):
    """The same oracle solves run concurrently, one process (one thread) per
    host core (spawned, so no CUDA state is inherited): aggregate DOF/s of
    the host.  Returns (DOF/s, processes, wall seconds)."""
    import multiprocessing as mp
    n = os.cpu_count() or 1
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(n) as pool:
            pool.map(_oracle_worker, [(0, 1)] * n)             # imports outside the timing
            t0 = time.perf_counter()
            res = pool.map(_oracle_worker, [(nt_sample, repeats)] * n)
            wall = time.perf_counter() - t0
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return NX * nt_sample * repeats * len(res) / wall, n, wall


SUBSET_MAX_DOF = 2 ** 21  # the batch subset's solves the oracle leg takes (24 solves, seconds on 16 cores)


def _oracle_mix_worker(spec):
    """One solve of the uneven batch by the oracle: two-level FCF-MGRIT in FP64
    from the zero iterate to 1e-10 (Section 2.2), its Psi fitted as the server
    fits it (auto width for ERK, the threshold rule for SDIRK); returns the
    final time level, the iteration count and the seconds (Psi fit
    included, as in the batch's timing)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    from oracle import mgrit as omg
    from oracle import psi as opsi
    from oracle import stepping
    fam, p, nx, nt, m = spec["family"], spec["p"], spec["nx"], spec["nt"], spec["m"]
    c = 4.0 if fam == "SDIRK" else 0.85 * CMAX_TABLE1[p]
    t0 = time.perf_counter()
    st = stepping.FineStep(fam, p, c, nx)
    ops = opsi.build_hierarchy(fam, p, c, nx, nt, m, 2, rule="threshold" if fam == "SDIRK" else "auto")
    U = omg.zero_iterate(workloads.fourier_field(nx, seed=spec["field_seed"]), nt)
    it, _ = omg.solve(omg.make_levels(st, m, [o.diag for o in ops]), U, tol=TOL, max_iter=80)
    return U[-1].copy(), it, time.perf_counter() - t0


def batch_subset_vs_oracle(capi, batch_dof, batch_wall_s, headline_oracle_all_cores):
    """The solves of the seeded 64-solve subset of the uneven batch (its first
    64) with nx*nt <= SUBSET_MAX_DOF: timed in the oracle on all host cores
    at once (spawned processes, one thread each), and through the server in
    MIXED as the batch runs them; per result, the relative L2 error of the
    final time level against the oracle's.  The oracle's batch time is
    extrapolated from the sample's DOF/s; small solves cost the oracle more
    per DOF (per-step interpreter overhead), so the headline sample's rate
    (nx = 4096) is given as the other bound."""
    import multiprocessing as mp
    specs = [s for s in workloads.batch_specs(64) if s["nx"] * s["nt"] <= SUBSET_MAX_DOF]
    dof = sum(s["nx"] * s["nt"] for s in specs)
    n = os.cpu_count() or 1
    env = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in env:
        os.environ[k] = "1"
    try:
        with mp.get_context("spawn").Pool(n) as pool:
            pool.map(_oracle_worker, [(0, 1)] * n)  # imports outside the timing
            t0 = time.perf_counter()
            ref = pool.map(_oracle_mix_worker, specs, chunksize=1)
            wall = time.perf_counter() - t0
    finally:
        for k, v in env.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    srv = capi.mgrit_server_create(150e9)
    errs, dits = [], []
    try:
        tickets = [capi.mgrit_submit(srv, *mix_request(capi, s, TOL, capi.PREC_MIXED)) for s in specs]
        for s, t, (fin_o, it_o, _) in zip(specs, tickets, ref):
            fin = np.zeros(s["nx"])
            while True:
                st, r = capi.mgrit_poll(srv, t, fin)
                if st != capi.MGRIT_PENDING:
                    break
                time.sleep(0.001)
            errs.append(float(np.linalg.norm(fin - fin_o) / np.linalg.norm(fin_o)) if st == 0 else float("inf"))
            dits.append(r.iterations - it_o)
    finally:
        capi.mgrit_server_destroy(srv)
    rate_all = dof / wall
    return {"solves": len(specs), "dof": dof, "cores": n,
            "sample": f"the {len(specs)} solves with nx*nt <= {SUBSET_MAX_DOF} of the batch's first 64 (seed 4)",
            "oracle_wall_s": wall, "oracle_dof_per_s_all_cores": rate_all,
            "oracle_dof_per_s_one_thread": dof / sum(x[2] for x in ref),
            "extrapolated_oracle_batch_s": {"subset_rate": batch_dof / rate_all,
                                            "headline_sample_rate": batch_dof / headline_oracle_all_cores},
            "gpu_batch_s": batch_wall_s,
            "err_vs_oracle": {"max": max(errs), "median": float(np.median(errs)),
                              "per_result": [float(f"{e:.3g}") for e in errs]},
            "iterations_minus_oracle": [min(dits), max(dits)]}


def cpu_sample_text(nt_sample=CPU_NT_SAMPLE):
    return (f"oracle (numpy FP64) V-cycle L=4 m=8 FCF-MGRIT on nx=4096, nt={nt_sample} (the first "
            f"{nt_sample}/16384 of the horizon), same scheme, CFL, u0 and tol; Psi setup excluded")


def run_reference(args, rank, world):
    """The oracle as the reference arm: each step one single-thread oracle
    solve of the CPU sample (the sample cpu_baseline's one-thread figure
    uses)."""
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample()
    secs = [oracle_sample()[1] for _ in range(args.steps)]
    value = NX * CPU_NT_SAMPLE * len(secs) / sum(secs)
    sample = cpu_sample_text() + "; one thread"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "DOF/s", "cores": 1, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "DOF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def oracle_sequential_cpoints():
    """The plain definition at full size: the oracle's sequential stepping
    u^{n+1} = Phi u^n of the headline problem (Eq. 3), at the C-points."""
    from oracle import stepping
    st = stepping.FineStep("ERK", P, CFL, NX)
    u = workloads.fourier_field(NX)
    out = np.empty((NT // M + 1, NX))
    out[0] = u
    for n in range(1, NT + 1):
        u = st(u)
        if n % M == 0:
            out[n // M] = u
    return out


# ------------------------------------------------------------- GPU arm

def fcf_traffic_from_profile(fourier=False):
    """Per-launch DRAM bytes of the level-1 FCF kernel (stencil or Fourier
    form) from the committed ncu summary, if it was taken on the current
    kernels source; else None."""
    name = "fcf_fourier_kernel_erk3u3_4096.md" if fourier else "fcf_kernel_erk3u3_4096.md"
    path = os.path.join(ROOT, "profiles", name)
    src = os.path.join(ROOT, "paper_1910_03726_gb300", "csrc", "kernels.cu")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    m1 = re.search(r"kernels\.cu sha256\[:16\]:\s*([0-9a-f]{16})", text)
    m2 = re.search(r"traffic_bytes_per_full_launch:\s*([0-9.eE+]+)", text)
    if not (m1 and m2) or m1.group(1) != h:
        return None
    return float(m2.group(1))


CMAX_TABLE1 = {1: 1.0, 2: 0.5, 3: 1.62589, 4: 1.04449, 5: 1.96583}   # Table 1 CFL limits (ERK_p+U_p)


def mix_request(capi, s, tol, precision):
    """Problem, options and u0 of one solve of the uneven batch / serving mix:
    ERK at 85% of Table 1's limit with the auto-width Psi, SDIRK at c = 4 with
    the threshold Psi; two-level, final time level returned."""
    fam, p = s["family"], s["p"]
    c = 4.0 if fam == "SDIRK" else 0.85 * CMAX_TABLE1[p]
    prob = capi.problem(s["nx"], s["nt"], fam, p, p, c)
    opts = capi.mgrit_opts_default(m=s["m"], levels=2, precision=precision, tol=tol, output=capi.OUT_FINAL,
                                   max_iter=80, psi_rule=capi.PSI_THRESHOLD if fam == "SDIRK" else capi.PSI_AUTO)
    return prob, opts, workloads.fourier_field(s["nx"], seed=s["field_seed"])


def run_server(capi, reqs, times, budget):
    """Submit reqs[i] at times[i] seconds (None: all at once), wait for all.
    Returns wall seconds from the first submission to the last completion,
    per-request latencies (seconds, measured inside the library from submit to
    completion) and results."""
    srv = capi.mgrit_server_create(budget)
    tickets = []
    stats = None
    try:
        t0 = time.perf_counter()
        for i, (prob, opts, u0) in enumerate(reqs):
            if times is not None:
                wait = t0 + times[i] - time.perf_counter()
                if wait > 0:
                    time.sleep(wait)
            tickets.append(capi.mgrit_submit(srv, prob, opts, u0))
        pending = dict(enumerate(tickets))
        results = [None] * len(tickets)
        while pending:
            for i in list(pending):
                st, r = capi.mgrit_poll(srv, pending[i])
                if st != capi.MGRIT_PENDING:
                    results[i] = (st, r)
                    del pending[i]
            if pending:
                time.sleep(0.001)
        wall = time.perf_counter() - t0
        stats = capi.mgrit_server_stats(srv)
    finally:
        capi.mgrit_server_destroy(srv)
    lat = [r.solve_s for st, r in results]
    return wall, lat, results, stats


def batch_variant(capi, count, stream):
    """Uneven batch of independent solves through the continuous-batching
    server (all submitted at once; FP32 F-relaxation, FP64 residual), against
    a sample of the same solves run alone in plain FP64 and by sequential
    stepping on the same GPU."""
    specs = workloads.batch_specs(count)
    reqs = [mix_request(capi, s, TOL, capi.PREC_MIXED) for s in specs]
    dof = sum(s["nx"] * s["nt"] for s in specs)
    wall, lat, results, stats = run_server(capi, reqs, None, 150e9)
    ok = sum(1 for st, r in results if st == 0 and r.converged)
    its = [r.iterations for st, r in results]
    sample = specs[:32]
    t_fp64 = t_seq = t_setup = 0.0
    dof_s = 0
    import torch
    for s in sample:
        prob, opts, u0 = mix_request(capi, s, TOL, capi.PREC_FP64)
        h = capi.mgrit_setup(prob, opts, stream=stream)
        try:
            capi.mgrit_solve(h, u0, None)
            r, _ = capi.mgrit_solve(h, u0, None)
            t_fp64 += r.solve_s
            t_setup += r.setup_s
            fin = torch.empty(s["nx"], dtype=torch.float64, device="cuda")
            t_seq += capi.mgrit_sequential(h, u0, fin)
        finally:
            capi.mgrit_destroy(h)
        dof_s += s["nx"] * s["nt"]
    return {"solves": count, "converged": ok, "dof": dof, "wall_s": wall, "dof_per_s": dof / wall,
            "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)), "p99": 1e3 * float(np.percentile(lat, 99))},
            "iterations_mean": float(np.mean(its)),
            "plain_fp64_alone_dof_per_s": dof_s / t_fp64, "gpu_sequential_dof_per_s": dof_s / t_seq,
            "plain_fp64_alone_with_setup_dof_per_s": dof_s / (t_fp64 + t_setup),
            "baseline_sample": f"first {len(sample)} solves of the batch, each alone: solve time (and solve plus "
                               f"set-up: Psi fit, allocation, autotuning)", "budget_bytes": 150e9,
            "batch_timing": "wall from the first submission to the last completion (admission and the Psi fits, "
                            "done by planner threads as requests arrive, included)",
            "mix": "nx 256..4096, nt 1024..16384, p 1..5, ERK or SDIRK, m 4/8/16 (seed 4), two-level, tol 1e-10",
            "server_stats": stats}


def fifo_latencies(times, service):
    """Completion minus arrival of requests served one at a time in arrival
    order (a queue in front of a single solver)."""
    done, lat = 0.0, []
    for a, s in zip(times, service):
        done = max(done, a) + s
        lat.append(done - a)
    return lat


def alone_service_times(capi, reqs, stream, keys=None, cache=None):
    """Per request, measured alone on the GPU: plain FP64 MGRIT (set-up -- Psi
    fit, allocation, autotuning -- plus the solve) and sequential stepping.
    With keys and a cache dict, a request whose key (scheme, order, nx, nt, m,
    tolerance) was measured before reuses that measurement: such requests
    differ in u0 only."""
    import torch
    fp64, seq = [], []
    for i, (prob, opts, u0) in enumerate(reqs):
        key = keys[i] if keys is not None else None
        if key is not None and key in cache:
            fp64.append(cache[key][0])
            seq.append(cache[key][1])
            continue
        o = capi.MgritOpts.from_buffer_copy(opts)
        o.precision = capi.PREC_FP64
        t0 = time.perf_counter()
        h = capi.mgrit_setup(prob, o, stream=stream)
        try:
            capi.mgrit_solve(h, u0, None, allow_not_converged=True)
            torch.cuda.synchronize()
            fp64.append(time.perf_counter() - t0)
            fin = torch.empty(prob.nx, dtype=torch.float64, device="cuda")
            seq.append(capi.mgrit_sequential(h, u0, fin))
        finally:
            capi.mgrit_destroy(h)
        if key is not None:
            cache[key] = (fp64[-1], seq[-1])
    return fp64, seq


SERVE_MEASURE_EACH = 1024  # above this many requests, service times are measured once per key


def serving_variant(capi, rates, count, stream=None, baselines=True):
    """Poisson arrivals of the batch mix with a 1e-8 or 1e-10 tolerance drawn
    per request; latency from submission to completion.  Baselines under the
    same arrival stream: a FIFO queue in front of one plain-FP64 MGRIT solver
    (each request set up and solved alone) and in front of GPU sequential
    stepping, with service times measured per request on the same GPU and the
    queue replayed on them.  Above SERVE_MEASURE_EACH requests a service time
    is measured once per (scheme, order, nx, nt, m, tolerance) and shared by
    all requests and rates with that key."""
    out = {}
    cache = {} if count > SERVE_MEASURE_EACH else None
    for rate in rates:
        times, tols = workloads.arrivals(rate, count)
        specs = workloads.batch_specs(count, seed=workloads.SEED_ARRIVALS * 7 + int(rate))
        reqs = [mix_request(capi, s, float(t), capi.PREC_MIXED) for s, t in zip(specs, tols)]
        dof = sum(s["nx"] * s["nt"] for s in specs)
        wall, lat, results, stats = run_server(capi, reqs, times, 150e9)
        ok = sum(1 for st, r in results if st == 0 and r.converged)
        row = {"requests": count, "converged": ok, "wall_s": wall, "dof_per_s": dof / wall,
               "latency_ms": {"p50": 1e3 * float(np.percentile(lat, 50)),
                              "p99": 1e3 * float(np.percentile(lat, 99))},
               "server_stats": stats}
        if baselines:
            keys = None if cache is None else [(s["family"], s["p"], s["nx"], s["nt"], s["m"], float(t))
                                               for s, t in zip(specs, tols)]
            fp64, seq = alone_service_times(capi, reqs, stream, keys, cache)
            row["service_times"] = ("measured per request" if cache is None else
                                    f"measured once per key: {len(cache)} keys so far")
            for name, svc in (("fifo_plain_fp64", fp64), ("fifo_gpu_sequential", seq)):
                fl = fifo_latencies(list(times), svc)
                span = max(max(times) + 0.0, 0.0)
                end = max(a + l for a, l in zip(times, fl))
                row[name] = {"latency_ms": {"p50": 1e3 * float(np.percentile(fl, 50)),
                                            "p99": 1e3 * float(np.percentile(fl, 99))},
                             "dof_per_s": dof / max(end - float(times[0]), 1e-9), "busy_s": float(sum(svc)),
                             "arrival_span_s": span}
        out[f"{rate:g}/s"] = row
    return out


def sdirk_variant(capi, stream, K, flags=0):
    """SDIRK3+U5, nx = 8192, nt = 8192, c = 4, two-level m = 16, threshold
    Psi, wave-packet u0 (seed 3): MIXED, FP64 and sequential stepping."""
    import torch
    nx = nt = 8192
    u0 = torch.tensor(workloads.wave_packet(nx), device="cuda")
    prob = capi.problem(nx, nt, "SDIRK", 3, 5, 4.0)
    res = {}
    for name, prec in (("mixed", capi.PREC_MIXED), ("fp64", capi.PREC_FP64)):
        o = capi.mgrit_opts_default(m=16, levels=2, precision=prec, tol=TOL, output=capi.OUT_FINAL,
                                    psi_rule=capi.PSI_THRESHOLD, max_iter=50, flags=flags)
        h = capi.mgrit_setup(prob, o, stream=stream)
        try:
            capi.mgrit_solve(h, u0, None)
            ts = []
            for _ in range(K):
                r, _ = capi.mgrit_solve(h, u0, None)
                ts.append(r.solve_s)
            res[name] = {"dof_per_s": nx * nt / statistics.median(ts), "ms": 1e3 * statistics.median(ts),
                         "iterations": r.iterations, "rel_residual": r.rel_residual}
            if name == "fp64":
                fin = torch.empty(nx, dtype=torch.float64, device="cuda")
                s = capi.mgrit_sequential(h, u0, fin)
                res["gpu_sequential_fp64"] = {"dof_per_s": nx * nt / s, "ms": 1e3 * s}
        finally:
            capi.mgrit_destroy(h)
    res["workload"] = "SDIRK3+U5 8192x8192 c=4, two-level m=16, threshold Psi, wave packet u0 (seed 3), tol 1e-10"
    return res


TABLE4_MAX = {1: (16384, 7, (6, 7, 7, 7, 7, 7)), 3: (8192, 6, (6, 7, 7, 8, 8)), 5: (8192, 6, (3, 4, 5, 5, 5))}


def paper_parallel_variant(capi, stream):
    """The paper's parallel runs (Section 5): ERKp+Up, p = 1, 3, 5, on
    2^12 x (2^14, 2^13, 2^13) with V-cycles, m = 4 and the most levels of
    Table 4 (7, 6, 6); MIXED and FP64 against GPU sequential stepping (the
    paper's speed-up metric), iterations beside Table 4's (random initial
    iterate there, zero here)."""
    import torch
    out = {}
    for p, (nt, L, t4) in TABLE4_MAX.items():
        nx = 4096
        prob = capi.problem(nx, nt, "ERK", p, p, 0.85 * CMAX_TABLE1[p])
        u0 = torch.tensor(workloads.fourier_field(nx), device="cuda")
        row = {"nx": nx, "nt": nt, "levels": L, "m": 4, "table4_iterations": t4[L - 2]}
        for name, prec in (("mixed", capi.PREC_MIXED), ("fp64", capi.PREC_FP64)):
            o = capi.mgrit_opts_default(m=4, levels=L, precision=prec, tol=TOL, output=capi.OUT_FINAL, max_iter=50,
                                        min_coarse=4)
            h = capi.mgrit_setup(prob, o, stream=stream)
            try:
                capi.mgrit_solve(h, u0, None)
                ts = []
                for _ in range(3):
                    r, _ = capi.mgrit_solve(h, u0, None)
                    ts.append(r.solve_s)
                row[name] = {"ms": 1e3 * statistics.median(ts), "dof_per_s": nx * nt / statistics.median(ts),
                             "iterations": r.iterations, "op_complexity": r.op_complexity}
                if name == "fp64":
                    fin = torch.empty(nx, dtype=torch.float64, device="cuda")
                    sq = capi.mgrit_sequential(h, u0, fin)
                    row["gpu_sequential_ms"] = 1e3 * sq
            finally:
                capi.mgrit_destroy(h)
        row["speedup_vs_gpu_sequential"] = row["gpu_sequential_ms"] / row["mixed"]["ms"]
        out[f"ERK{p}+U{p}"] = row
    return out


# Table 5's largest grids (inflow/outflow, Section 4.5): p -> (nt, most levels, V-cycle counts L = 2..)
TABLE5_MAX = {1: (16384, 7, (6, 7, 7, 7, 7, 7)), 3: (8192, 6, (6, 7, 7, 7, 7)), 5: (8192, 6, (5, 5, 5, 5, 5))}


def inflow_variant(capi, stream):
    """Inflow/outflow boundaries (Section 4.5, Table 5's 2^12 grids): ERKp+Up,
    p = 1, 3, 5, V-cycles with m = 4 and the most levels Table 5 lists; MIXED
    and FP64 solves beside the same configuration with periodic boundaries
    (the cost of the boundary rows) and GPU sequential stepping of the closed
    problem; iterations beside Table 5's (random initial iterate there, zero
    here)."""
    import torch
    out = {}
    for p, (nt, L, t5) in TABLE5_MAX.items():
        nx = 4096
        c = 0.85 * CMAX_TABLE1[p]
        u0 = torch.tensor(workloads.fourier_field(nx), device="cuda")
        row = {"nx": nx, "nt": nt, "levels": L, "m": 4, "table5_iterations": t5[L - 2]}
        for bc in ("inflow", "periodic"):
            prob = capi.problem(nx, nt, "ERK", p, p, c, boundary=bc)
            for name, prec in (("mixed", capi.PREC_MIXED), ("fp64", capi.PREC_FP64)):
                if bc == "periodic" and name == "fp64":
                    continue
                o = capi.mgrit_opts_default(m=4, levels=L, precision=prec, tol=TOL, output=capi.OUT_FINAL,
                                            max_iter=50, min_coarse=4)
                h = capi.mgrit_setup(prob, o, stream=stream)
                try:
                    capi.mgrit_solve(h, u0, None)
                    ts = []
                    for _ in range(3):
                        r, _ = capi.mgrit_solve(h, u0, None)
                        ts.append(r.solve_s)
                    key = name if bc == "inflow" else f"periodic_{name}"
                    row[key] = {"ms": 1e3 * statistics.median(ts), "dof_per_s": nx * nt / statistics.median(ts),
                                "iterations": r.iterations}
                    if bc == "inflow" and name == "fp64":
                        fin = torch.empty(nx, dtype=torch.float64, device="cuda")
                        row["gpu_sequential_ms"] = 1e3 * capi.mgrit_sequential(h, u0, fin)
                finally:
                    capi.mgrit_destroy(h)
        row["speedup_vs_gpu_sequential"] = row["gpu_sequential_ms"] / row["mixed"]["ms"]
        row["cost_vs_periodic"] = row["mixed"]["ms"] / row["periodic_mixed"]["ms"]
        out[f"ERK{p}+U{p}"] = row
    return out


def measured_hbm_gbs():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        return float(json.load(open(path))["hbm_gbs"]), "measured (MEASURED_PEAKS.json hbm_gbs)"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback 6.8 TB/s"


def hbm_variant(capi, stream, steps=3):
    """The memory-bound instance of the level-1 FCF: ERK1+U1 with m = 4
    (collapsed Phi^4: 5 taps) on 4096 x 16384, V-cycle L = 4.  In MIXED_DF
    both passes run on the FP32 pipes, so the kernel is bound by HBM: per
    launch it must read every C-point slab once (FP64), write every new
    C-point (FP64) and every residual slab (FP32), 20 B per point and
    interval.  CUDA events around back-to-back sweeps of mgrit_relax (one
    FCF launch each, queued without host gaps) on the converged iterate; the
    algorithmic bytes per launch over the time per launch, against the
    measured copy bandwidth.  MIXED (FP64 first pass) alongside: FP64-bound
    there (0.37 flop/B against a 0.18 flop/B ridge)."""
    import torch
    nx, nt, m, L = 4096, 16384, 4, 4
    peak, src = measured_hbm_gbs()
    prob = capi.problem(nx, nt, "ERK", 1, 1, 0.85)
    u0 = torch.tensor(workloads.fourier_field(nx), device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    N1 = nt // m
    out = {"nx": nx, "nt": nt, "m": m, "levels": L, "peak_gbs": peak, "peak_source": src,
           "bytes_per_launch": N1 * nx * 20}
    sweeps = 40
    for name, prec in (("mixed_df", capi.PREC_MIXED_DF), ("mixed", capi.PREC_MIXED)):
        o = capi.mgrit_opts_default(m=m, levels=L, precision=prec, tol=TOL, output=capi.OUT_FINAL)
        h = capi.mgrit_setup(prob, o, stream=stream)
        try:
            r, _ = capi.mgrit_solve(h, u0, None)
            capi.mgrit_relax(h, 3)
            per = []
            for _ in range(steps):
                flush.zero_()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(torch.cuda.current_stream())
                capi.mgrit_relax(h, sweeps)          # back-to-back FCF launches, one norm at the end
                e1.record(torch.cuda.current_stream())
                torch.cuda.synchronize()
                per.append(e0.elapsed_time(e1) / sweeps)
            ms = statistics.median(per)
            gbs = out["bytes_per_launch"] / (ms * 1e-3) / 1e9
            out[name] = {"fcf_launch_ms": ms, "achieved_gbs": gbs, "frac_of_hbm_peak": gbs / peak,
                         "iterations": r.iterations, "shape": [r.fine_tile, r.fine_threads, r.fine_collapsed, r.fine_fourier],
                         "timing": f"CUDA events around {sweeps} back-to-back sweeps (mgrit_relax) on the "
                                   f"converged iterate, median of {steps}; L2 flushed before each group"}
        finally:
            capi.mgrit_destroy(h)
    return out


def hbm_summary(h):
    """The HBM-roofline fraction of the level-1 FCF on its memory-bound
    instance (from hbm_variant), or None when that variant did not run."""
    if not isinstance(h, dict) or "mixed_df" not in h:
        return None
    d = h["mixed_df"]
    return {"instance": f"ERK1+U1 nx={h['nx']} nt={h['nt']} m={h['m']}, MIXED_DF (float-float C-points)",
            "achieved": d["achieved_gbs"], "peak": h["peak_gbs"], "unit": "GB/s", "frac": d["frac_of_hbm_peak"],
            "bytes_per_launch": h["bytes_per_launch"], "launch_ms": d["fcf_launch_ms"],
            "peak_source": h["peak_source"],
            "mixed_fp64_first_pass_frac": h.get("mixed", {}).get("frac_of_hbm_peak")}


def exact_cpoints(nx, nt, m, c, device):
    """Exact solution of Eq. 1 (alpha = 1) at the C-points t_j = j m dt for the
    Fourier-field initial condition: u0(x - t) as a product of the per-time
    mode amplitudes and the spatial modes (angle addition), on the device."""
    import torch
    a, b = workloads.fourier_coefficients()
    K = len(a)
    k = torch.arange(1, K + 1, dtype=torch.float64, device=device)
    x = torch.tensor(workloads.grid(nx), device=device)
    t = torch.arange(0, nt + 1, m, dtype=torch.float64, device=device) * (c * 2.0 / nx)
    ak = torch.tensor(a, device=device) / k ** 2
    bk = torch.tensor(b, device=device) / k ** 2
    ct, st = torch.cos(torch.pi * t[:, None] * k), torch.sin(torch.pi * t[:, None] * k)
    A = ak * ct - bk * st                    # coefficient of cos(k pi x) at time t
    B = ak * st + bk * ct                    # coefficient of sin(k pi x)
    return A @ torch.cos(torch.pi * k[:, None] * x) + B @ torch.sin(torch.pi * k[:, None] * x)


def disc_error_variant(capi, stream):
    """Time to discretization-error accuracy (Section 5's second stopping
    criterion): the fewest MGRIT iterations whose C-points are within 1% of
    sequential stepping's own error against the exact solution, on the
    paper's parallel configurations (MIXED, V-cycles, m = 4), against GPU
    sequential stepping."""
    import torch
    out = {}
    for p, (nt, L, _) in TABLE4_MAX.items():
        nx, m = 4096, 4
        c = 0.85 * CMAX_TABLE1[p]
        prob = capi.problem(nx, nt, "ERK", p, p, c)
        u0 = torch.tensor(workloads.fourier_field(nx), device="cuda")
        ex = exact_cpoints(nx, nt, m, c, "cuda")
        nrm = float(torch.linalg.norm(ex))
        seq = torch.empty((nt // m + 1, nx), dtype=torch.float64, device="cuda")
        hs = capi.mgrit_setup(prob, capi.mgrit_opts_default(m=m, levels=L, min_coarse=4), stream=stream)
        capi.mgrit_sequential(hs, u0, seq)
        seq_s = capi.mgrit_sequential(hs, u0, seq)
        capi.mgrit_destroy(hs)
        e_d = float(torch.linalg.norm(seq - ex)) / nrm
        row = {"discretization_error_rel": e_d, "gpu_sequential_ms": 1e3 * seq_s}
        cp = torch.empty_like(seq)
        for k in range(1, 30):
            o = capi.mgrit_opts_default(m=m, levels=L, precision=capi.PREC_MIXED, tol=TOL, max_iter=k, min_coarse=4)
            h = capi.mgrit_setup(prob, o, stream=stream)
            try:
                capi.mgrit_solve(h, u0, cp, allow_not_converged=True)
                err = float(torch.linalg.norm(cp - ex)) / nrm
                if err <= 1.01 * e_d:
                    ts = []
                    for _ in range(3):
                        r, _ = capi.mgrit_solve(h, u0, None, allow_not_converged=True)
                        ts.append(r.solve_s)
                    row.update({"iterations": k, "error_rel": err, "ms": 1e3 * statistics.median(ts),
                                "dof_per_s": nx * nt / statistics.median(ts),
                                "speedup_vs_gpu_sequential": seq_s / statistics.median(ts)})
                    break
            finally:
                capi.mgrit_destroy(h)
        out[f"ERK{p}+U{p}"] = row
    return out


def replica_max(total_ms, world, device="cuda"):
    """Max over ranks of each rank's timed total (ms); one all-reduce when the
    job runs N > 1 independent replicas (torchrun, NCCL on GPUs, gloo on CPU)."""
    if world <= 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(total_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replicas_value(world, dof_per_step, steps, max_total_ms):
    """Whole-job throughput: the DOF of all ranks' timed steps over the slowest
    rank's time (weak scaling: each replica solves the full problem)."""
    return world * dof_per_step * steps / (max_total_ms * 1e-3)


def pct(xs, q):
    return float(np.percentile(np.asarray(xs), q)) if len(xs) else None


def compact_summary(extra):
    """The variants' headline figures, small enough for the bench line."""
    out = {}
    g = extra.get("gpu_sequential_fp64")
    if g:
        out["gpu_sequential_dof_per_s"] = g["dof_per_s"]
        out["speedup_vs_gpu_sequential"] = extra.get("speedup_vs_gpu_sequential")
    for key, name in (("fp64_vcycle_L4_m8", "plain_fp64_mgrit_dof_per_s"),
                      ("mixed_df_vcycle_L4_m8", "mixed_df_dof_per_s")):
        if key in extra:
            out[name] = extra[key]["dof_per_s"]
    b = extra.get("batch_uneven")
    if b:
        out["batch_4096"] = {"dof_per_s": b["dof_per_s"], "plain_fp64_alone": b["plain_fp64_alone_dof_per_s"],
                             "plain_fp64_alone_with_setup": b["plain_fp64_alone_with_setup_dof_per_s"],
                             "gpu_seq_alone": b["gpu_sequential_dof_per_s"], "p50_ms": b["latency_ms"]["p50"],
                             "p99_ms": b["latency_ms"]["p99"], "converged": b["converged"]}
    sv = extra.get("serving_poisson")
    if sv:
        def trio(v):
            return [round(v["latency_ms"]["p50"], 1), round(v["latency_ms"]["p99"], 1), float("%.4g" % v["dof_per_s"])]
        out["serving"] = {k: {"batched": trio(v), **({"fifo_fp64": trio(v["fifo_plain_fp64"]),
                                                      "fifo_seq": trio(v["fifo_gpu_sequential"])}
                                                     if "fifo_plain_fp64" in v else {})} for k, v in sv.items()}
        out["serving_fields"] = "[p50 ms, p99 ms, DOF/s]; fifo_*: one solver in arrival order, service measured alone"
    bs = extra.get("batch_subset_vs_oracle")
    if bs:
        ex = bs["extrapolated_oracle_batch_s"]
        out["batch_subset_vs_oracle"] = {"solves": bs["solves"], "err_max": float("%.3g" % bs["err_vs_oracle"]["max"]),
                                         "iterations_minus_oracle": bs["iterations_minus_oracle"],
                                         "oracle_batch_s_extrapolated": [round(ex["subset_rate"]),
                                                                         round(ex["headline_sample_rate"])],
                                         "gpu_batch_s": round(bs["gpu_batch_s"], 2)}
    sd = extra.get("sdirk3_u5_8192")
    if sd:
        out["sdirk3_u5_8192_ms"] = {"mixed": sd["mixed"]["ms"], "fp64": sd["fp64"]["ms"],
                                    "gpu_seq": sd["gpu_sequential_fp64"]["ms"]}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-variants", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "mixed_df"],
                    help="arithmetic of the headline solve")
    ap.add_argument("--batch", type=int, default=4096, help="solves in the uneven batch (0: skip)")
    ap.add_argument("--serve", type=int, default=400, help="requests per arrival rate (0: skip)")
    ap.add_argument("--only", choices=["sdirk", "batch", "serve", "inflow", "hbm"],
                    help="run just this variant and print its JSON (no headline line)")
    ap.add_argument("--host-loop", action="store_true",
                    help="with --only sdirk: drive cycles from the host (kernels visible to ncu)")
    ap.add_argument("--variants-out", default="",
                    help="file for the full variant record (written when its folder exists; default none)")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)
    rank, world, local = dist_env()

    if args.impl == "reference":
        run_reference(args, rank, world)
        return

    import torch
    import torch.distributed as dist
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1910_03726_gb300 import build
    if rank == 0:
        build.build()
    if world > 1:
        dist.barrier()
    from paper_1910_03726_gb300 import capi

    stream = torch.cuda.current_stream()
    sp = int(stream.cuda_stream)
    if args.only:
        run = {"sdirk": lambda: sdirk_variant(capi, sp, args.steps,
                                              capi.FLAG_HOST_LOOP if args.host_loop else 0),
               "batch": lambda: batch_variant(capi, args.batch, sp),
               "serve": lambda: serving_variant(capi, (100, 1000, 3000, 10000), args.serve, sp),
               "inflow": lambda: inflow_variant(capi, sp),
               "hbm": lambda: hbm_variant(capi, sp)}[args.only]
        print(json.dumps({args.only: run()}), flush=True)
        return
    u0_np = workloads.fourier_field(NX)
    u0 = torch.tensor(u0_np, device="cuda")
    N1 = NT // M
    out = torch.empty((N1 + 1, NX), dtype=torch.float64, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")  # > 129 MB L2
    prob = capi.problem(NX, NT, "ERK", P, P, CFL)

    def make(levels, m, precision, flags=0, cycle=0, relax=0):
        o = capi.mgrit_opts_default(m=m, levels=levels, precision=precision, tol=TOL, output=capi.OUT_CPOINTS,
                                    flags=flags, max_iter=100, cycle=cycle, relax=relax)
        return capi.mgrit_setup(prob, o, stream=sp)

    def timed_solves(h, K, W, queued=True):
        """K solves of u0, each bracketed by CUDA events on the solve stream
        with the L2 flushed before it.  Queued: all K are enqueued
        (mgrit_solve_async) before the first wait, so host-side delays cannot
        leave the GPU idle inside a bracket; otherwise one mgrit_solve at a
        time (the host loop of the kernel-timing pass)."""
        for _ in range(W):
            capi.mgrit_solve(h, u0, out)
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        e0 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        e1 = [torch.cuda.Event(enable_timing=True) for _ in range(K)]
        results = []
        for k0 in range(0, K, capi.MAX_INFLIGHT):
            ks = range(k0, min(K, k0 + capi.MAX_INFLIGHT))
            for k in ks:
                flush.zero_()                       # evict L2 between steps
                e0[k].record(stream)
                if queued:
                    capi.mgrit_solve_async(h, u0, out)
                else:
                    results.append(capi.mgrit_solve(h, u0, out)[0])
                e1[k].record(stream)
            if queued:
                results += [capi.mgrit_solve_wait(h)[0] for _ in ks]
        torch.cuda.synchronize()
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()
        lat = [a.elapsed_time(b) for a, b in zip(e0, e1)]
        return lat, replica_max(sum(lat), world), results

    clocks = ClockSampler(local)
    head_prec = {"fp64": capi.PREC_FP64, "mixed": capi.PREC_MIXED, "mixed_df": capi.PREC_MIXED_DF}[args.precision]
    # ---- headline: V-cycle L=4, m=8, each solve one CUDA-graph launch, queued
    h = make(LEVELS, M, head_prec)
    clocks.start()
    lat, total, results = timed_solves(h, args.steps, args.warmup)
    clk = clocks.stop()
    res0 = results[-1]
    value = replicas_value(world, NX * NT, args.steps, total)
    launches = sum(r.launches for r in results)
    head_cpoints = out.cpu().numpy()
    # ---- e2e through the C ABI with host buffers (u0 in, C-points out), in
    # pinned host memory
    u0_host = torch.tensor(u0_np).pin_memory()
    out_host = torch.empty((N1 + 1, NX), dtype=torch.float64).pin_memory()
    capi.mgrit_solve(h, u0_host, out_host)
    torch.cuda.synchronize()
    e2e_t = []
    for _ in range(max(3, args.steps // 2)):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        capi.mgrit_solve(h, u0_host, out_host)
        e2e_t.append(time.perf_counter() - t0)
    e2e_value = world * NX * NT * len(e2e_t) / sum(e2e_t)
    capi.mgrit_destroy(h)
    # ---- roofline pass: the same solves driven cycle by cycle from the host
    # with CUDA events around every kernel (identical kernels and shapes)
    hp = make(LEVELS, M, head_prec, flags=capi.FLAG_TIME_KERNELS)
    p_lat, p_total, p_results = timed_solves(hp, args.steps, args.warmup, queued=False)
    capi.mgrit_destroy(hp)
    fcf_ms = sum(r.kernel_ms[0] for r in p_results)
    fcf_n = sum(r.kernel_count[0] for r in p_results)
    phi_off = capi.mgrit_phi_taps(prob)[0]
    nnz_phi = len(phi_off)
    fourier = bool(p_results[-1].fine_fourier)
    peak64 = FP64_PEAK_TFLOPS
    peak_src = "152 SM x 4 FP64 flop/clk x 2.07 GHz"
    if fourier:                                  # FP64 pass in Fourier space
        ops_i, flops_i = fourier_fcf_work(NX)
        flops64 = N1 * flops_i
        # the pipe issues one add, mul, fma or conversion per lane-slot: the
        # peak of this operation mix is the issue rate x its flops per operation
        peak64 = FP64_OPS_PEAK * flops_i / ops_i / 1e12
        peak_src = (f"152 SM x 2 FP64 ops/clk x 2.07 GHz x {flops_i / ops_i:.4f} flop/op "
                    f"(the Fourier form's {ops_i / NX:.2f} ops, {flops_i / NX:.2f} flops per point)")
    elif p_results[-1].fine_collapsed:           # one application of Phi^m per pass
        flops64 = N1 * NX * 2 * (M * (max(phi_off) - min(phi_off)) + 1)
    else:                                        # m applications of Phi per pass
        flops64 = N1 * M * NX * 2 * nnz_phi
    # the first FCF of a solve starts from the zero iterate: only interval 1
    # holds nonzero data (the kernels skip Phi^m of zero slabs), so its
    # algorithmic work is 1/N1 of a full launch; its time stays in the total
    full_equiv = fcf_n - len(p_results) + len(p_results) / N1
    fcf_avg_s = fcf_ms / max(1e-9, full_equiv) * 1e-3
    achieved = flops64 / fcf_avg_s / 1e12 if fcf_avg_s > 0 else None
    tot_ms = max(1e-9, sum(sum(r.kernel_ms) for r in p_results))
    kernel_share = {capi.KERNEL_KINDS[i]: round(sum(r.kernel_ms[i] for r in p_results) / tot_ms, 4)
                    for i in range(capi.K_KINDS)}
    extra = {"kernel_time_share": kernel_share,
             "host_loop_with_kernel_events": {"dof_per_s": world * NX * NT * args.steps / (p_total * 1e-3),
                                              "ms": p_total / args.steps},
             "latency_ms_all": [round(x, 4) for x in lat]}
    if not args.no_variants:
        ks = max(3, args.steps // 2)
        for name, (lv, m, prec, cyc, rlx) in {
                "mixed_df_vcycle_L4_m8": (4, 8, capi.PREC_MIXED_DF, 0, 0),
                "fp64_vcycle_L4_m8": (4, 8, capi.PREC_FP64, 0, 0),
                "mixed_fcycle_L4_m8": (4, 8, capi.PREC_MIXED, 1, 0),
                "mixed_two_level_m8": (2, 8, capi.PREC_MIXED, 0, 0),
                "fp64_two_level_m8": (2, 8, capi.PREC_FP64, 0, 0),
                "mixed_parareal_two_level_m8": (2, 8, capi.PREC_MIXED, 0, 1),
                "mixed_f_relax_vcycle_L4_m8": (4, 8, capi.PREC_MIXED, 0, 1)}.items():
            hv = make(lv, m, prec, cycle=cyc, relax=rlx)
            lv_lat, lv_total, lv_res = timed_solves(hv, ks, 1)
            extra[name] = {"dof_per_s": NX * NT * ks / (lv_total * 1e-3), "ms": lv_total / ks,
                           "iterations": lv_res[-1].iterations, "rel_residual": lv_res[-1].rel_residual}
            capi.mgrit_destroy(hv)
        # plain FP64 sequential stepping on the GPU (one thread-block cluster)
        hs = make(2, M, capi.PREC_FP64)
        fin = torch.empty((N1 + 1, NX), dtype=torch.float64, device="cuda")
        capi.mgrit_sequential(hs, u0, fin)
        torch.cuda.synchronize()
        sl = []
        for _ in range(3):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            capi.mgrit_sequential(hs, u0, fin)
            b.record(stream)
            torch.cuda.synchronize()
            sl.append(a.elapsed_time(b))
        seq_ms = statistics.median(sl)
        extra["gpu_sequential_fp64"] = {"dof_per_s": NX * NT / (seq_ms * 1e-3), "ms": seq_ms}
        extra["speedup_vs_gpu_sequential"] = seq_ms / statistics.median(lat)
        extra["rel_l2_vs_gpu_fp64_sequential"] = float(np.linalg.norm(head_cpoints - fin.cpu().numpy())
                                                       / np.linalg.norm(fin.cpu().numpy()))
        capi.mgrit_destroy(hs)
        extra["sdirk3_u5_8192"] = sdirk_variant(capi, sp, 3)
        extra["paper_parallel_configs"] = paper_parallel_variant(capi, sp)
        extra["paper_configs_to_discretization_error"] = disc_error_variant(capi, sp)
        extra["inflow_outflow_table5_configs"] = inflow_variant(capi, sp)
        extra["hbm_bound_erk1_m4"] = hbm_variant(capi, sp)
        if args.batch > 0:
            extra["batch_uneven"] = batch_variant(capi, args.batch, sp)
        if args.serve > 0:
            extra["serving_poisson"] = serving_variant(capi, (100, 1000, 3000, 10000), args.serve, sp)

    line = None
    if rank == 0:
        cpu = None
        err_oracle = None
        if not args.no_cpu and world == 1:
            # the headline result against the plain definition at full size
            t_seq = time.perf_counter()
            ref = oracle_sequential_cpoints()
            t_seq = time.perf_counter() - t_seq
            err_oracle = float(np.linalg.norm(head_cpoints - ref) / np.linalg.norm(ref))
            v1, s1, it1 = oracle_sample(repeats=3)
            va, nproc, wall = oracle_all_cores()
            cpu = {"value": va, "unit": "DOF/s", "cores": nproc, "kind": "oracle",
                   "sample": f"oracle V(L=4,m=8) on nx=4096 nt={CPU_NT_SAMPLE}, {nproc} concurrent 1-thread "
                             f"solves, {wall:.1f} s", "one_thread_value": v1,
                   "sequential_one_thread_value": NX * NT / t_seq,
                   "sequential_sample": f"oracle sequential stepping (Eq. 3), full {NX}x{NT}, one thread, "
                                        f"{t_seq:.1f} s"}
            bu = extra.get("batch_uneven")
            if bu is not None:
                extra["batch_subset_vs_oracle"] = batch_subset_vs_oracle(capi, bu["dof"], bu["wall_s"], va)
        hb = hbm_summary(extra.get("hbm_bound_erk1_m4"))
        line = {
            "metric": METRIC, "value": value, "unit": "DOF/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "fp64+fp32", "data": "synthetic",
            "gpu_launches": launches,
            "config": {"workload": "ERK3+U3 4096x16384 c=.85cmax, V(L=4,m=8), LSQ Psi, FP32 relax/FP64 residual, "
                                   "tol 1e-10", "parallelism": f"replicas x{world}", "l2": "flushed per step",
                       "timing": "events per queued solve"},
            "e2e": {"value": e2e_value, "unit": "DOF/s", "h2d_bytes_per_step": NX * 8,
                    "d2h_bytes_per_step": (N1 + 1) * NX * 8},
            "clocks": clk, "cpu_baseline": cpu,
            "roofline": {"bound": "alu",
                         "kernel": ("fcf_fourier_kernel level 1 (FP64 pass in Fourier space)" if fourier
                                    else "fcf_kernel level 1"),
                         "achieved": achieved, "peak": peak64, "unit": "TFLOP/s",
                         "frac": (achieved / peak64) if achieved else None,
                         "traffic": fcf_traffic_from_profile(fourier), "peak_source": peak_src,
                         "launch_ms": fcf_avg_s * 1e3},
            "hbm_roofline_fcf": ({"frac": hb["frac"], "achieved": hb["achieved"], "peak": hb["peak"],
                                  "unit": "GB/s", "instance": "ERK1 m=4 MIXED_DF",
                                  "mixed_frac": hb["mixed_fp64_first_pass_frac"]} if hb else None),
            "iterations": res0.iterations, "rel_residual": res0.rel_residual,
            "err_vs_oracle_sequential": err_oracle,
            "latency_ms": {"min": min(lat), "p50": pct(lat, 50), "p99": pct(lat, 99), "max": max(lat)},
            "summary": compact_summary(extra),
        }
        try:
            if args.variants_out and os.path.isdir(os.path.dirname(os.path.abspath(args.variants_out))):
                with open(args.variants_out, "w") as f:
                    json.dump({"line": line, "variants": extra}, f, indent=1)
        except OSError:
            pass
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
