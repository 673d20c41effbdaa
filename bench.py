#!/usr/bin/env python
"""Benchmark: excitation states converged per second on one GB300 (or N replicas).

One step is the whole hot path on the medium response workload (n_occ=60,
n_vir=400, n_aux=2000, ris n_aux=360): a Casida solve for the 10 lowest states
and the polarizability alpha(omega) for 3 dipoles at omega = 0, 0.05, 0.1 Ha,
both with the rid preconditioner to a residual of 1e-5, MIXED precision (exact
products as BF16 hi+lo on the tcgen05 tensor cores, FP32 accumulation; ris
inner solves with FP32 vectors on the BF16 ris factors; FP64 outer subspace
algebra; FP32 re-certification of the converged residuals).

value: states converged per second (10 per step x steps x ranks / max time),
device-timed with CUDA events on the solver's stream, factors resident in HBM;
p50/p99 over the per-step times (30 steps by default).
e2e:   the same through the C ABI with host (pinned) inputs: tddft_create
       (host->device copy and conversion of every factor) + the two solves
       with host outputs + tddft_destroy, every step.
plain: the same step in the plain FP64 form on the same GPU (FP64 factors,
       vectors and inner solves, SIMT contractions), for mixed vs plain.
Inputs (the FP32/BF16 factors, 2.8 GB) are larger than L2, so no L2 flush is
added between steps.

serving: an open-loop Poisson stream of TDA / Casida / polarizability requests
       of random sizes through the server API (each request brings its own
       device-resident problem), p50/p99 latency and states/s (--serve-*).
batched: 256 small independent TDA solves queued at once on the server
       (solves/s; --batch*).

Multi-GPU: one independent replica per GPU (the path does not shard on one
box), launched under torch.distributed.run; rank 0 prints one JSON line.

--impl reference times the CPU oracle (FP64, NumPy) on a bounded sample of the
same workload and prints the same line with "impl": "reference".
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

WORKLOAD = "rpa_polar_medium"
N_STATES = 10
METRIC = "states converged/s at ||r||<=1e-5 (Casida, rid, mixed) + alpha(omega) per step"
UNIT = "states/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tensor-cores", type=int, default=-1, help="1/0 (default 1: tcgen05 exchange)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--kernel-breakdown", action="store_true",
                    help="run one warm step under the CUDA activity profiler and print per-kernel totals")
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="steps of the plain FP64 form timed for the mixed-vs-plain comparison (0: skip)")
    ap.add_argument("--precond", default="rid", choices=["rid", "diag"])
    ap.add_argument("--serve-seconds", type=float, default=10.0,
                    help="length of the served request stream (0: no serving measurement)")
    ap.add_argument("--serve-rate", type=float, default=30.0, help="Poisson arrival rate, requests/s")
    ap.add_argument("--serve-max-occ", type=int, default=40, help="largest n_occ of a served request")
    ap.add_argument("--serve-slots", type=int, default=16, help="requests running at once")
    ap.add_argument("--batch", type=int, default=256, help="independent small TDA solves queued at once (0: none)")
    ap.add_argument("--batch-slots", type=int, default=16)
    ap.add_argument("--serve-budget-gb", type=float, default=150.0)
    ap.add_argument("--apply-only", type=int, default=0, metavar="K",
                    help="time K exact pair products ((A+B)X, (A-B)X) of 2*n_states device vectors "
                         "and exit (a short program for kernel profiling)")
    return ap.parse_args()


def max_over_ranks(x, world):
    """The largest x over the ranks (a time: the job ends with its slowest replica)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, world, max_ms):
    """Whole-job throughput of `world` replicas that each processed units_per_rank
    units, over the slowest replica's time (ms)."""
    return units_per_rank * world / (max_ms / 1e3)


def dist_env():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.idx = gpu_index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(gpu_index), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        rows = [r.split(",") for r in self.f.read().strip().splitlines() if r.count(",") >= 8]
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows]
        mx = max(float(r[2]) for r in rows)
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip() == "Active"})
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": reasons,
                "samples": len(rows)}


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0,
                "sm_max_mhz": 2070.0}, "fallback"


def golden():
    with open(os.path.join(ROOT, "tests", "golden", WORKLOAD + ".json")) as f:
        return json.load(f)


def oracle_sample(seconds_budget=20.0):
    """Time the oracle's exact and ris pair products on the workload's inputs and
    scale them by the oracle's own product counts for one step (RPA + polar).
    Returns (step_seconds, description, cores)."""
    import numpy as np
    from oracle import operators as O
    from synth.generator import make_config

    p = make_config(WORKLOAD)
    op, T = O.exact_operator(p), O.ris_operator(p)
    g = golden()
    X = np.random.default_rng(0).standard_normal((2, p.n_ov))
    t0 = time.perf_counter()
    n_ex = 0
    while True:
        op.apb_amb(X)
        n_ex += 2
        if time.perf_counter() - t0 > 0.7 * seconds_budget or n_ex >= 32:
            break
    t_ex = (time.perf_counter() - t0) / n_ex
    Xr = np.random.default_rng(1).standard_normal((16, p.n_ov))
    t0 = time.perf_counter()
    T.apb_amb(Xr)
    t_ris = (time.perf_counter() - t0) / 16
    n_mv = g["rpa"]["n_mv"] + g["polar"]["n_mv"]
    n_ris = g["rpa"]["n_ris_mv"] + g["polar"]["n_ris_mv"]
    step = t_ex * n_mv + t_ris * n_ris
    desc = ("%d oracle (A+B, A-B) products + 16 ris pair products at the full workload size, "
            "scaled by the oracle's own counts for one step (%d exact, %d ris vectors)" % (n_ex, n_mv, n_ris))
    return step, desc, os.cpu_count()


def reference_arm(args, rank, world):
    if rank != 0:
        return
    steps = []
    desc = cores = None
    for _ in range(args.warmup):
        pass  # the oracle has nothing to warm up
    for _ in range(args.steps):
        s, desc, cores = oracle_sample(seconds_budget=max(5.0, 60.0 / max(args.steps, 1)))
        steps.append(s)
    step = statistics.mean(steps)
    value = N_STATES / step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle (NumPy)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def our_arm(args, rank, world, local):
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as ge
    ge.build()
    from paper_2404_17133_gb300 import api
    from synth.generator import CONFIGS, dipoles, make_config

    cfg = CONFIGS[WORKLOAD]
    p = make_config(WORKLOAD)
    mu = dipoles(cfg["mu_seed"], cfg["n_dip"], p.n_ov)
    omegas = list(cfg["omegas"])
    tc = args.tensor_cores
    if tc < 0:
        tc = 1
    stream = torch.cuda.current_stream()
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32))
    kidx = p.ris_K_index
    host = {"eo": torch.from_numpy(p.eps_occ.copy()), "ev": torch.from_numpy(p.eps_vir.copy()),
            "oo": f32(p.L_oo), "ov": f32(p.L_ov), "vv": f32(p.L_vv), "roo": f32(p.Lr_oo[kidx]),
            "rov": f32(p.Lr_ov), "rvv": f32(p.Lr_vv[kidx]), "k": torch.from_numpy(kidx.copy())}
    dev = {k: v.cuda() for k, v in host.items()}
    pinned = {k: v.pin_memory() for k, v in host.items()}
    h2d_bytes = sum(v.numel() * v.element_size() for v in host.values()) + mu.nbytes + 8 * len(omegas)
    d2h_bytes = 8 * (2 * N_STATES + len(omegas) * cfg["n_dip"] ** 2)

    def make_solver(src, stream_ptr):
        return api.Solver(p.n_occ, p.n_vir, src["eo"], src["ev"], src["oo"], src["ov"], src["vv"],
                          src["roo"], src["rov"], src["rvv"], src["k"], a_x=p.a_x,
                          coulomb_factor=p.coulomb_factor, t_cut_ha=p.t_cut_ha, precisions=2,
                          dtype=api.F32, stream=stream_ptr)

    pc = api.RID if args.precond == "rid" else api.DIAG
    o_rpa = api.default_opts(n_states=N_STATES, precond=pc, precision=api.MIXED, tensor_cores=tc)
    o_pol = api.default_opts(precond=pc, precision=api.MIXED, tensor_cores=tc)
    solver = make_solver(dev, stream.cuda_stream)
    if args.apply_only > 0:
        apply_only(args, api, solver, p, tc, stream)
        solver.close()
        return
    if args.kernel_breakdown:
        kernel_breakdown(solver, o_rpa, o_pol, mu, omegas)
        solver.close()
        return

    def step(s):
        a = s.solve_rpa(o_rpa, want_vectors=False)
        b = s.solve_polar(o_pol, mu, omegas)
        return a, b

    for _ in range(max(args.warmup, 0)):
        step(solver)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    solver.profile(True)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps + 1)]
    ev[0].record(stream)
    launches = 0
    results = []
    for i in range(args.steps):
        a, b = step(solver)
        ev[i + 1].record(stream)
        launches += a["stats"]["gpu_launches"] + b["stats"]["gpu_launches"]
        results.append((a, b))
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    prof = solver.profile_read(0 if tc else 1)
    rec_ms, rec_fl, rec_by = solver.profile_records(0 if tc else 1)
    solver.profile(False)
    clk = clocks.stop() if clocks else None
    per_step = [ev[i].elapsed_time(ev[i + 1]) for i in range(args.steps)]
    total_ms = ev[0].elapsed_time(ev[-1])
    total_ms = max_over_ranks(total_ms, world)
    value = replica_throughput(N_STATES * args.steps, world, total_ms)
    a, b = results[-1]
    conv = all(r["status"] == api.OK for pair in results for r in pair)

    # ---- end to end through the C ABI with pinned host inputs and host outputs
    e2e_ms = []
    for _ in range(0 if args.no_e2e else max(args.e2e_steps, 1)):
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        s2 = make_solver(pinned, stream.cuda_stream)
        step(s2)
        s2.close()
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms.append(e0.elapsed_time(e1))
    e2e_t = statistics.mean(e2e_ms) if e2e_ms else float("nan")

    # ---- the plain FP64 form of the same step (FP64 inputs, FP64 everywhere, SIMT)
    plain = None
    if args.plain_steps > 0 and rank == 0:
        f64 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()
        sp = api.Solver(p.n_occ, p.n_vir, dev["eo"], dev["ev"], f64(p.L_oo), f64(p.L_ov), f64(p.L_vv),
                        f64(p.Lr_oo[kidx]), f64(p.Lr_ov), f64(p.Lr_vv[kidx]), dev["k"], a_x=p.a_x,
                        coulomb_factor=p.coulomb_factor, t_cut_ha=p.t_cut_ha, precisions=1, dtype=api.F64,
                        stream=stream.cuda_stream)
        o_rpa_p = api.default_opts(n_states=N_STATES, precond=pc, precision=api.PLAIN)
        o_pol_p = api.default_opts(precond=pc, precision=api.PLAIN)
        pms, pit = [], []
        for _ in range(args.plain_steps):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ra = sp.solve_rpa(o_rpa_p, want_vectors=False)
            rb = sp.solve_polar(o_pol_p, mu, omegas)
            e1.record(stream)
            torch.cuda.synchronize()
            pms.append(e0.elapsed_time(e1))
            pit.append((ra["stats"]["n_iter"], rb["stats"]["n_iter"]))
        sp.close()
        pm = statistics.mean(pms)
        plain = {"value": N_STATES / (pm / 1e3), "unit": UNIT, "ms_per_step": pm, "steps": args.plain_steps,
                 "dtype": "f64", "rpa_n_iter": pit[-1][0], "polar_n_iter": pit[-1][1],
                 "max_abs_omega_diff_vs_mixed": float(np.max(np.abs(np.asarray(ra["omega"]) -
                                                                    np.asarray(results[-1][0]["omega"])))),
                 "note": "same step in the plain form: FP64 factors and vectors, SIMT contractions, "
                         "FP64 inner solves; warm kernels, one step"}
    e2e_t = max_over_ranks(e2e_t, world)
    if rank != 0:
        solver.close()
        return
    peaks, src = load_peaks()
    kernel_ms = prof["ms"] / max(prof["launches"], 1)
    flops_launch = prof["flops"] / max(prof["launches"], 1)
    achieved = flops_launch / (kernel_ms * 1e-3) / 1e12 if prof["launches"] else 0.0
    if tc:
        peak = peaks["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "unit": "TFLOP/s", "peak_kind": "bf16 sustained, " + src,
                "note": "algorithmic flops 2*M*N*K; the hi+lo split issues 3 BF16 products per flop"}
    else:
        sm = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s",
                "peak_kind": "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x %.0f MHz" % sm}
    # per-launch roofline: the launch's attainable time is the larger of its
    # tensor time (tcgen05: three BF16 products per algorithmic flop for the
    # hi+lo exact factors) and its HBM time (algorithmic bytes at the measured
    # copy bandwidth); small trial blocks make a launch HBM-bound
    if rec_ms.size:
        per_flop = 3.0 if tc else 1.0
        t_ten = rec_fl * per_flop / (peak * 1e12) * 1e3
        t_hbm = rec_by / (peaks["hbm_gbs"] * 1e9) * 1e3
        t_att = np.maximum(t_ten, t_hbm)
        roof.update({
            "attainable_frac": float(t_att.sum() / rec_ms.sum()),
            "hbm_bound_time_share": float(rec_ms[t_hbm > t_ten].sum() / rec_ms.sum()),
            "achieved_hbm_gbs": float(rec_by.sum() / rec_ms.sum() / 1e6),
            "algorithmic_bytes_per_launch": float(rec_by.mean()),
            "attainable_note": "per launch max(%g BF16 products per flop at the tensor peak, algorithmic bytes "
                               "at hbm_gbs %.0f); attainable_frac = sum of those / sum of measured times"
                               % (per_flop, peaks["hbm_gbs"])})
    roof.update({"achieved": achieved, "peak": peak, "frac": achieved / peak if peak else None,
                 "traffic": None, "kernel": "exchange K1 contraction sum_(P,a) Z L_vv",
                 "launches": prof["launches"], "ms_per_launch": kernel_ms,
                 "share_of_step": prof["ms"] / total_ms if total_ms else None})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (tensor: bf16x3) + fp64 subspace",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_occ": p.n_occ, "n_vir": p.n_vir, "n_aux": p.n_aux,
                       "n_aux_ris": p.n_ris, "n_states": N_STATES, "n_dip": cfg["n_dip"],
                       "omegas": omegas, "precond": args.precond, "tensor_cores": bool(tc),
                       "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (2.8 GB resident factors), no flush"},
            "p50_ms": statistics.median(per_step),
            "p99_ms": sorted(per_step)[min(len(per_step) - 1, int(0.99 * len(per_step)))],
            "converged": conv,
            "rpa": {"omega": list(map(float, a["omega"])), "n_iter": a["stats"]["n_iter"],
                    "n_matvec": a["stats"]["n_matvec"], "n_ris_matvec": a["stats"]["n_ris_matvec"],
                    "max_resid": a["stats"]["max_resid"],
                    "max_resid_certified": a["stats"]["max_resid_certified"],
                    "t_precond_share": a["stats"]["t_precond_s"] / max(a["stats"]["t_total_s"], 1e-12)},
            "polar": {"n_iter": b["stats"]["n_iter"], "n_matvec": b["stats"]["n_matvec"],
                      "alpha_static_diag": [float(b["alpha"][0][i][i]) for i in range(cfg["n_dip"])]},
            "roofline": roof,
            "plain": plain,
            "speedup_vs_plain": (plain["ms_per_step"] / (total_ms / args.steps)) if plain else None,
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": {"value": N_STATES * world / (e2e_t / 1e3), "unit": UNIT, "ms_per_step": e2e_t,
                    "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": int(d2h_bytes)}}
    if args.serve_seconds > 0 and world == 1:
        try:
            line["serving"] = serving(args, api, torch)
        except Exception as e:   # the served stream is reported, not required for the line
            line["serving"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if args.batch > 0 and world == 1:
        try:
            line["batched"] = batched(args, api, torch)
        except Exception as e:
            line["batched"] = {"error": "%s: %s" % (type(e).__name__, e)}
        try:
            line["batched_tc"] = batched(args, api, torch, tc=1)
        except Exception as e:
            line["batched_tc"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if not args.no_cpu_baseline and world == 1:
        step_s, desc, cores = oracle_sample()
        line["cpu_baseline"] = {"value": N_STATES / step_s, "unit": UNIT, "cores": cores,
                                "kind": "oracle", "sample": desc}
    print(json.dumps(line), flush=True)
    solver.close()
    if world > 1:
        torch.distributed.destroy_process_group()


def _run_stream(api, reqs, arrivals, slots, budget_gb, warm_kw):
    """Submit reqs[i] = (kind, opts, create_kw, mu, omegas) at arrivals[i] seconds
    (open loop) to a server; returns the finished (request index, result) pairs,
    the server's state and the number left unfinished."""
    from synth.generator import dipoles

    srv = api.Server(hbm_budget_gb=budget_gb, max_active=slots)
    try:
        # warm-up: one request of each kind on a small problem (untimed)
        ws = [srv.submit(k, api.default_opts(n_states=5, precond=api.RID, precision=api.MIXED, tensor_cores=1),
                         create_kw=dict(warm_kw, precisions=2, dtype=api.F32),
                         mu=dipoles(1, 3, warm_kw["n_occ"] * warm_kw["n_vir"]) if k == 2 else None,
                         omegas=[0.0, 0.05] if k == 2 else None) for k in (0, 1, 2)]
        for t in ws:
            while srv.poll(t, timeout_ms=100) is None:
                pass
        done, pending = [], {}
        t0 = time.perf_counter()
        i, n = 0, len(reqs)
        limit = float(arrivals[-1]) + 300.0 if n else 0.0
        while i < n or pending:
            now = time.perf_counter() - t0
            while i < n and arrivals[i] <= now:
                kind, o, kw, mu, om = reqs[i]
                t = srv.submit(kind, o, create_kw=dict(kw, precisions=2, dtype=api.F32), mu=mu, omegas=om)
                pending[t] = i
                i += 1
            for t in list(pending):
                r = srv.poll(t, timeout_ms=0)
                if r is not None:
                    done.append((pending.pop(t), r))
            if now > limit:
                break
            time.sleep(0.001)
        info = srv.info()
    finally:
        srv.close()
    return done, info, len(pending)


def _stream_report(api, reqs, done, info, unfinished):
    pct = lambda v, q: v[min(len(v) - 1, int(q * len(v)))]
    lat = sorted(r["latency_s"] * 1e3 for _, r in done)
    wait = sorted((r["t_start_s"] - r["t_submit_s"]) * 1e3 for _, r in done)
    span = max(r["t_end_s"] for _, r in done) - min(r["t_submit_s"] for _, r in done)
    ok = [(i, r) for i, r in done if r["status"] == api.OK]
    states = sum(reqs[i][1].n_states for i, r in ok if reqs[i][0] in (0, 1))
    starts = sorted(r["t_start_s"] for _, r in done)
    most = max(sum(1 for _, q in done if q["t_start_s"] <= t < q["t_end_s"]) for t in starts)
    by_kind = {}
    for i, r in done:
        by_kind.setdefault(reqs[i][0], []).append(r["latency_s"] * 1e3)
    return {"requests": len(reqs), "finished": len(done), "ok": len(ok),
            "noconv": sum(1 for _, r in done if r["status"] == api.ERR_NOCONV),
            "errors": sum(1 for _, r in done if r["status"] not in (api.OK, api.ERR_NOCONV)),
            "unfinished": unfinished, "span_s": span, "states_per_s": states / span,
            "solves_per_s": len(ok) / span, "p50_ms": pct(lat, 0.50), "p99_ms": pct(lat, 0.99),
            "queue_wait_p50_ms": pct(wait, 0.50), "queue_wait_p99_ms": pct(wait, 0.99),
            "p50_ms_by_kind": {("tda", "casida", "polar")[k]: statistics.median(v) for k, v in by_kind.items()},
            "max_concurrent": most, "budget_gb": info["budget_bytes"] / 1e9,
            "peak_charge_gb": info["peak_in_use_bytes"] / 1e9,
            "pool_high_gb": (info["pool_high_bytes"] - info["pool_used_at_create_bytes"]) / 1e9}


def serving(args, api, torch):
    """Open-loop served stream: Poisson arrivals of TDA (60 %), Casida (25 %) and
    polarizability (15 %, 3 dipoles, 1-4 frequencies) requests of random sizes
    (n_occ log-uniform, n_vir = n_occ x U{4..9}, n_aux = 5 n_mo, ris n_aux =
    9 ceil(n_occ/2), 5-20 states), each bringing its own FP32 device-resident
    problem, MIXED precision with tcgen05 products and rid; admitted by the
    server's HBM budget with a fixed number of slots.  Latency = finish - submit
    (server clock); throughput over the whole stream, first submit to last finish."""
    from synth.device import problem_kw, serving_mix
    from synth.generator import dipoles

    rng = np.random.default_rng(2404)
    gaps = rng.exponential(1.0 / args.serve_rate, size=int(args.serve_rate * args.serve_seconds * 3) + 16)
    arrivals = np.cumsum(gaps)
    arrivals = arrivals[arrivals < args.serve_seconds]
    n_req = int(arrivals.size)
    mix = serving_mix(2404, n_req, max_occ=args.serve_max_occ)
    n_pool = min(48, n_req)
    pool = [problem_kw(1000 + i, m["n_occ"], m["n_vir"], m["n_aux"], m["n_ris"]) for i, m in
            enumerate(mix[:n_pool])]
    torch.cuda.synchronize()
    freqs = [0.0, 0.05, 0.1, 0.15]
    reqs = []
    for i, m in enumerate(mix):
        kw = pool[i % n_pool]
        ov = kw["n_occ"] * kw["n_vir"]
        kind = m["kind"]
        if kind == 2:
            o = api.default_opts(precond=api.RID, precision=api.MIXED, tensor_cores=1)
            reqs.append((kind, o, kw, dipoles(5000 + i, 3, ov), freqs[:m["n_freq"]]))
        else:
            o = api.default_opts(n_states=min(m["n_states"], ov), precond=api.RID, precision=api.MIXED,
                                 tensor_cores=1)
            reqs.append((kind, o, kw, None, None))
    warm = min(pool, key=lambda k: k["n_occ"] * k["n_vir"])
    done, info, left = _run_stream(api, reqs, arrivals, args.serve_slots, args.serve_budget_gb, warm)
    if not done:
        return {"error": "no request finished"}
    out = _stream_report(api, reqs, done, info, left)
    out.update({"offered_rate_req_s": args.serve_rate, "seconds": args.serve_seconds, "slots": args.serve_slots,
                "n_occ_range": [10, args.serve_max_occ], "distinct_problems": n_pool,
                "note": "each request creates its context from FP32 device arrays (MIXED copies only), "
                        "solves, destroys it; MIXED + tcgen05 + rid; latency = finish - submit"})
    return out


def batched(args, api, torch, tc=0):
    """Many small independent TDA solves submitted together: n_occ ~ U{8..64},
    n_vir = n_occ x U{4..8}, n_aux = 5 n_mo, ris n_aux = 9 ceil(n_occ/2), 5-10
    states, MIXED (FP32 outer products on the SIMT path, or with tc the BF16
    hi+lo tcgen05 products; BF16 ris), rid; all queued at time 0 on a server
    with --batch-slots slots (concurrent streams, not one persistent kernel).
    Throughput = solves / (first submit to last finish)."""
    from synth.device import problem_kw

    g = np.random.Generator(np.random.Philox(key=np.array([2405, 1], dtype=np.uint64)))
    n = args.batch
    sizes = []
    for _ in range(n):
        no = int(g.integers(8, 65))
        nv = no * int(g.integers(4, 9))
        sizes.append((no, nv, 5 * (no + nv), 9 * ((no + 1) // 2), int(g.integers(5, 11))))
    n_pool = min(64, n)
    pool = [problem_kw(3000 + i, *sizes[i][:4]) for i in range(n_pool)]
    torch.cuda.synchronize()
    reqs = []
    for i in range(n):
        kw = pool[i % n_pool]
        o = api.default_opts(n_states=sizes[i % n_pool][4], precond=api.RID, precision=api.MIXED,
                             tensor_cores=tc)
        reqs.append((0, o, kw, None, None))
    warm = min(pool, key=lambda k: k["n_occ"] * k["n_vir"])
    done, info, left = _run_stream(api, reqs, np.zeros(n), args.batch_slots, args.serve_budget_gb, warm)
    if not done:
        return {"error": "no request finished"}
    out = _stream_report(api, reqs, done, info, left)
    out.update({"slots": args.batch_slots, "distinct_problems": n_pool,
                "note": "TDA solves queued at once, each creating its context from FP32 device arrays; "
                        "MIXED, %s outer products, BF16 ris, rid"
                        % ("BF16 hi+lo tcgen05" if tc else "FP32 SIMT")})
    return out


def apply_only(args, api, solver, p, tc, stream):
    """K exact pair products on 2*n_states device vectors, each timed with CUDA events."""
    import torch
    X = torch.from_numpy(np.random.default_rng(7).standard_normal((2 * N_STATES, p.n_ov))).cuda()
    ms = []
    for _ in range(args.apply_only):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.apply(1, X, precision=api.MIXED, tensor_cores=bool(tc))
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"apply_only": args.apply_only, "m": 2 * N_STATES, "ms": ms,
                      "workload": WORKLOAD, "tensor_cores": bool(tc)}), flush=True)


def kernel_breakdown(solver, o_rpa, o_pol, mu, omegas):
    """One warm step under the CUDA activity profiler (CUPTI): every kernel and
    copy with its device time; printed as one JSON line."""
    import collections
    import re
    import torch
    from torch.profiler import ProfilerActivity, profile

    def step():
        solver.solve_rpa(o_rpa, want_vectors=False)
        solver.solve_polar(o_pol, mu, omegas)

    step()
    torch.cuda.synchronize()
    with profile(activities=[ProfilerActivity.CUDA]) as prof:
        t0 = time.perf_counter()
        step()
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    ev = [e for e in prof.events() if e.device_type == torch.autograd.DeviceType.CUDA]
    tot, cnt = collections.defaultdict(float), collections.Counter()
    span0, span1 = float("inf"), 0.0
    for e in ev:
        nm = e.name.replace("(anonymous namespace)::", "").replace("void ", "").replace("tddft::", "")
        nm = re.sub(r"\(.*", "", nm)
        tot[nm] += e.time_range.elapsed_us()
        cnt[nm] += 1
        span0, span1 = min(span0, e.time_range.start), max(span1, e.time_range.end)
    busy = sum(tot.values())
    rows = [{"kernel": k, "launches": cnt[k], "ms": round(v / 1e3, 3), "share": round(v / busy, 4)}
            for k, v in sorted(tot.items(), key=lambda x: -x[1])]
    print(json.dumps({"kernel_breakdown": rows, "busy_ms": busy / 1e3, "span_ms": (span1 - span0) / 1e3,
                      "first_start_ms": span0 / 1e3, "last_end_ms": span1 / 1e3, "events": len(ev),
                      "wall_ms": wall * 1e3, "workload": WORKLOAD}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    our_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
