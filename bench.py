#!/usr/bin/env python
"""Benchmark: excitation states converged per second on one GB300 (or N replicas).

One step is the whole hot path on the large mixed workload (n_occ=150,
n_vir=1350, ov=202,500, exact n_aux=6000, ris n_aux=1350): a TDA solve and a
Casida solve for the 20 lowest states each, with the rid preconditioner to a
residual of 1e-5, MIXED precision (exact products on the tcgen05 tensor cores
with every operand scaled by a power of two and split into FP16 hi + lo, FP32
accumulation: FP32-accurate products; ris inner solves with FP32 vectors on the
BF16 ris factors; FP64 outer subspace algebra; the converged residuals
recomputed from fresh products).  40 converged states per step.

value: states converged per second (40 per step x steps x ranks / max time),
device-timed with CUDA events on the solver's stream, factors resident in HBM;
p50/p99 over the per-step times.
e2e:   the same through the C ABI with host (pinned) inputs: tddft_create
       (host->device copy and conversion of every factor, 56 GB) + the two
       solves with host outputs + tddft_destroy, every step.
medium: the medium workload (n_occ=60, n_vir=400, n_aux=2000) as context:
       Casida (10 states) + alpha(omega) per step, MIXED, and the same step in
       the plain FP64 form (the plain form of the large step would take most
       of an hour on GB300's FP64 units).
Inputs (the resident factor copies, ~100 GB) are far larger than L2, so no L2
flush is added between steps.

serving: an open-loop Poisson stream of TDA / Casida / polarizability requests
       of random sizes through the server API (each request brings its own
       device-resident problem), p50/p99 latency and states/s (--serve-*).
batched: 256 small independent TDA solves queued at once on the server
       (solves/s; --batch*).

Multi-GPU: one independent replica per GPU (the path does not shard on one
box), launched under torch.distributed.run; rank 0 prints one JSON line.

--impl reference times the CPU oracle (FP64, NumPy) on a bounded sample of the
same workload (the exact and ris products of a few vectors over a few
auxiliary rows, scaled to all rows and to the products one step makes) and
prints the same line with "impl": "reference".
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

WORKLOAD = "large_mixed"
N_STATES = 20
STATES_PER_STEP = 2 * N_STATES          # TDA + Casida
METRIC = "states converged/s at ||r||<=1e-5 (TDA + Casida, 20 states each, rid, mixed)"
UNIT = "states/s"
MEDIUM = "rpa_polar_medium"
MEDIUM_STATES = 10
# Exact and ris products one step of the large workload makes (TDA vectors,
# Casida pair vectors), as the mixed GPU solve counted them on GB300; the
# oracle cannot run the Davidson iteration at this size (108 GB of FP64
# factors), so its step time is its per-vector product time scaled by these.
LARGE_COUNTS = {"tda_mv": 107, "tda_ris_mv": 751, "rpa_mv": 535, "rpa_ris_mv": 2009}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--tensor-cores", type=int, default=-1, help="1/0 (default 1: tcgen05 exchange)")
    ap.add_argument("--e2e-steps", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-diag", action="store_true", help="skip the diag-preconditioner iteration counts")
    ap.add_argument("--kernel-breakdown", action="store_true",
                    help="run one warm step under the CUDA activity profiler and print per-kernel totals")
    ap.add_argument("--medium-steps", type=int, default=5,
                    help="steps of the medium workload (0: skip the medium object)")
    ap.add_argument("--plain-steps", type=int, default=1,
                    help="steps of the medium workload's plain FP64 form (mixed vs plain; 0: skip)")
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
    ap.add_argument("--workload", default=WORKLOAD, help="workload of --apply-only / --kernel-breakdown")
    ap.add_argument("--oracle-sample", type=int, default=0, metavar="THREADS", help=argparse.SUPPRESS)
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
    with open(os.path.join(ROOT, "tests", "golden", MEDIUM + ".json")) as f:
        return json.load(f)


# ---------------------------------------------------------------------------
# CPU oracle samples (the reference arm and cpu_baseline)

def _oracle_sample_worker(seconds_budget):
    """In a fresh process with the BLAS thread count of its environment: the
    oracle's FP64 TDA product, pair product ((A+B)X, (A-B)X) and the ris
    products of the large workload on a few auxiliary rows, as seconds per
    vector over all rows.  Prints one JSON line."""
    import types
    from oracle import operators as O
    from synth.generator import config_meta, factor_rows, ris_rows

    meta = config_meta(WORKLOAD)
    no, nv, na, nr = meta["n_occ"], meta["n_vir"], meta["n_aux"], meta["n_ris"]
    rows, m = 8, 2
    oo, ov, vv = factor_rows(WORKLOAD, 0, rows)
    X = np.random.default_rng(0).standard_normal((m, no * nv))
    op = O.Operator(meta["eps_occ"], meta["eps_vir"], ov, oo, ov, vv, meta["a_x"], meta["coulomb_factor"])
    t0 = time.perf_counter()
    n = 0
    while True:
        op.apb_amb(X)
        n += 1
        if time.perf_counter() - t0 > 0.4 * seconds_budget:
            break
    t_pair = (time.perf_counter() - t0) / n / m * (na / rows)
    t0 = time.perf_counter()
    op.tda(X)
    t_tda = (time.perf_counter() - t0) / m * (na / rows)
    roo, rov, rvv = ris_rows(WORKLOAD, 0, 9)
    pr = types.SimpleNamespace(eps_occ=meta["eps_occ"], eps_vir=meta["eps_vir"], Lr_oo=roo, Lr_ov=rov,
                               Lr_vv=rvv, ris_K_index=np.array([0], dtype=np.int32), a_x=meta["a_x"],
                               coulomb_factor=meta["coulomb_factor"], t_cut_ha=meta["t_cut_ha"])
    T = O.ris_operator(pr)
    t0 = time.perf_counter()
    T.apb_amb(X)
    t_rpair = (time.perf_counter() - t0) / m * (nr / 9)
    t0 = time.perf_counter()
    T.tda(X)
    t_rtda = (time.perf_counter() - t0) / m * (nr / 9)
    print(json.dumps({"t_pair": t_pair, "t_tda": t_tda, "t_ris_pair": t_rpair, "t_ris_tda": t_rtda,
                      "rows": rows, "vectors": m, "threads": os.environ.get("OPENBLAS_NUM_THREADS")}))


def oracle_sample(threads=None, seconds_budget=8.0):
    """Run _oracle_sample_worker in a fresh interpreter (its own BLAS thread
    count: `threads`, or the library default) and return its timings."""
    env = dict(os.environ)
    for v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
        if threads:
            env[v] = str(threads)
        else:
            env.pop(v, None)
    code = "import bench; bench._oracle_sample_worker(%r)" % seconds_budget
    r = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=600)
    if r.returncode != 0:
        raise RuntimeError("oracle sample failed: " + r.stderr[-500:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def oracle_step_seconds(t, counts):
    """Seconds of one large step on the oracle: per-vector product times times
    the products a step makes (TDA: A X and T X; Casida: pair products)."""
    return (t["t_tda"] * counts["tda_mv"] + t["t_ris_tda"] * counts["tda_ris_mv"] +
            t["t_pair"] * counts["rpa_mv"] + t["t_ris_pair"] * counts["rpa_ris_mv"])


def sample_note(t, counts):
    return ("extrapolation: the oracle's FP64 TDA and pair products of %d vectors over %d of the 6000 "
            "exact rows (and the ris products over 9 of the 1350 ris rows), scaled to all rows and to "
            "the products of one step (%d TDA and %d Casida exact vectors, %d + %d ris vectors, as the "
            "GPU solve counted them; the oracle cannot run this Davidson: 108 GB of FP64 factors); "
            "BLAS threads: %s" % (t["vectors"], t["rows"], counts["tda_mv"], counts["rpa_mv"],
                                  counts["tda_ris_mv"], counts["rpa_ris_mv"], t["threads"] or "default"))


def reference_arm(args, rank, world):
    if rank != 0:
        return
    steps = []
    t = None
    budget = max(2.0, min(8.0, 150.0 / max(args.steps + args.warmup, 1)))
    for _ in range(args.warmup):
        oracle_sample(seconds_budget=budget)
    for _ in range(args.steps):
        t = oracle_sample(seconds_budget=budget)
        steps.append(oracle_step_seconds(t, LARGE_COUNTS))
    step = statistics.mean(steps)
    value = STATES_PER_STEP / step
    cores = os.cpu_count()
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "impl": "FP64 CPU oracle (NumPy)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample_note(t, LARGE_COUNTS)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# the GPU arm

def load_large(api, torch, stream_ptr, pinned_copy=False):
    """The large workload's factors drawn chunk-wise on the host into FP32
    device tensors (synth/chunked.py), a MIXED-only context created from them
    and the staging tensors released; with pinned_copy, also a pinned host
    copy of the inputs for the end-to-end measurement."""
    from synth import chunked
    from synth.generator import config_meta

    meta = config_meta(WORKLOAD)
    no, nv, na, nr = meta["n_occ"], meta["n_vir"], meta["n_aux"], meta["n_ris"]
    kidx = meta["ris_K_index"]
    t0 = time.time()
    dev = (torch.empty(na, no, no, device="cuda"), torch.empty(na, no, nv, device="cuda"),
           torch.empty(na, nv, nv, device="cuda"))
    chunked.load_exact(WORKLOAD, meta, dev)
    rdev = (torch.empty(kidx.size, no, no, device="cuda"), torch.empty(nr, no, nv, device="cuda"),
            torch.empty(kidx.size, nv, nv, device="cuda"))
    chunked.load_ris(WORKLOAD, meta, rdev)
    small = {"eo": torch.from_numpy(meta["eps_occ"].copy()), "ev": torch.from_numpy(meta["eps_vir"].copy()),
             "k": torch.from_numpy(kidx.copy())}
    t_load = time.time() - t0
    arrays = {"oo": dev[0], "ov": dev[1], "vv": dev[2], "roo": rdev[0], "rov": rdev[1], "rvv": rdev[2]}
    host = None
    if pinned_copy:
        host = {k: torch.empty(v.shape, dtype=v.dtype, pin_memory=True) for k, v in arrays.items()}
        for k, v in arrays.items():
            host[k].copy_(v)
        host.update({k: v.pin_memory() for k, v in small.items()})
    src = dict(arrays)
    src.update({k: v.cuda() for k, v in small.items()})
    solver = make_solver(api, meta, src, stream_ptr)
    torch.cuda.synchronize()
    del dev, rdev, arrays, src
    torch.cuda.empty_cache()
    return solver, meta, host, t_load


def make_solver(api, meta, src, stream_ptr):
    return api.Solver(meta["n_occ"], meta["n_vir"], src["eo"], src["ev"], src["oo"], src["ov"], src["vv"],
                      src["roo"], src["rov"], src["rvv"], src["k"], a_x=meta["a_x"],
                      coulomb_factor=meta["coulomb_factor"], t_cut_ha=meta["t_cut_ha"], precisions=2,
                      dtype=api.F32, stream=stream_ptr)


def our_arm(args, rank, world, local):
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__ as ge
    ge.build()
    from paper_2404_17133_gb300 import api

    tc = 1 if args.tensor_cores < 0 else args.tensor_cores
    stream = torch.cuda.current_stream()
    if args.apply_only > 0 or args.kernel_breakdown:
        solver, p = small_solver(args, api, torch, stream)
        if args.apply_only > 0:
            apply_only(args, api, solver, p, tc, stream)
        else:
            kernel_breakdown(args, api, solver, tc)
        solver.close()
        return
    want_e2e = not args.no_e2e and rank == 0
    solver, meta, host, t_load = load_large(api, torch, stream.cuda_stream, pinned_copy=want_e2e)
    h2d_bytes = sum(v.numel() * v.element_size() for v in host.values()) if host else 0
    d2h_bytes = 8 * (2 * N_STATES + 2 * N_STATES)     # energies and residual norms of both solves
    pc = api.RID if args.precond == "rid" else api.DIAG
    o = api.default_opts(n_states=N_STATES, precond=pc, precision=api.MIXED, tensor_cores=tc)

    def step(s):
        a = s.solve_tda(o, want_vectors=False)
        b = s.solve_rpa(o, want_vectors=False)
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
    value = replica_throughput(STATES_PER_STEP * args.steps, world, total_ms)
    a, b = results[-1]
    conv = all(r["status"] == api.OK for pair in results for r in pair)
    counts = {"tda_mv": a["stats"]["n_matvec"], "tda_ris_mv": a["stats"]["n_ris_matvec"],
              "rpa_mv": b["stats"]["n_matvec"], "rpa_ris_mv": b["stats"]["n_ris_matvec"]}

    diag = None
    if not args.no_diag and rank == 0:
        od = api.default_opts(n_states=N_STATES, precond=api.DIAG, precision=api.MIXED, tensor_cores=tc)
        da, db = solver.solve_tda(od, want_vectors=False), solver.solve_rpa(od, want_vectors=False)
        diag = {"tda_n_iter": da["stats"]["n_iter"], "rpa_n_iter": db["stats"]["n_iter"],
                "tda_s": da["stats"]["t_total_s"], "rpa_s": db["stats"]["t_total_s"],
                "converged": da["status"] == api.OK and db["status"] == api.OK,
                "max_abs_omega_diff_vs_rid": float(max(np.max(np.abs(da["omega"] - a["omega"])),
                                                       np.max(np.abs(db["omega"] - b["omega"]))))}
    peaks, src = load_peaks()
    roof = roofline(prof, rec_ms, rec_fl, rec_by, peaks, src, tc, clk, total_ms)

    # ---- end to end through the C ABI with pinned host inputs and host outputs
    e2e_ms = []
    if want_e2e:
        solver.close()
        solver = None
        torch.cuda.empty_cache()
        for _ in range(max(args.e2e_steps, 1)):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            s2 = make_solver(api, meta, host, stream.cuda_stream)
            step(s2)
            s2.close()
            e1.record(stream)
            torch.cuda.synchronize()
            e2e_ms.append(e0.elapsed_time(e1))
        host = None
    e2e_t = statistics.mean(e2e_ms) if e2e_ms else float("nan")
    e2e_t = max_over_ranks(e2e_t, world)
    if solver is not None:
        solver.close()
        solver = None
    torch.cuda.empty_cache()
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32 (tensor: fp16 hi+lo x3) + fp64 subspace",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n_occ": meta["n_occ"], "n_vir": meta["n_vir"],
                       "n_aux": meta["n_aux"], "n_aux_ris": meta["n_ris"], "n_states": N_STATES,
                       "solves_per_step": ["tda", "casida"], "precond": args.precond,
                       "tensor_cores": bool(tc), "parallelism": "replicas" if world > 1 else "single",
                       "l2": "inputs larger than L2 (~100 GB resident factor copies), no flush"},
            "p50_ms": statistics.median(per_step),
            "p99_ms": sorted(per_step)[min(len(per_step) - 1, int(0.99 * len(per_step)))],
            "converged": conv, "load_s": t_load,
            "tda": {"omega0": float(a["omega"][0]), "n_iter": a["stats"]["n_iter"],
                    "n_matvec": a["stats"]["n_matvec"], "n_ris_matvec": a["stats"]["n_ris_matvec"],
                    "max_resid_certified": a["stats"]["max_resid_certified"], "s": a["stats"]["t_total_s"],
                    "exact_product_s": a["stats"]["t_matvec_s"], "precond_s": a["stats"]["t_precond_s"]},
            "rpa": {"omega0": float(b["omega"][0]), "n_iter": b["stats"]["n_iter"],
                    "n_matvec": b["stats"]["n_matvec"], "n_ris_matvec": b["stats"]["n_ris_matvec"],
                    "max_resid_certified": b["stats"]["max_resid_certified"], "s": b["stats"]["t_total_s"],
                    "exact_product_s": b["stats"]["t_matvec_s"], "precond_s": b["stats"]["t_precond_s"]},
            "diag": diag,
            "roofline": roof,
            "gpu_launches": launches,
            "clocks": clk,
            "e2e": {"value": STATES_PER_STEP * world / (e2e_t / 1e3) if e2e_ms else None, "unit": UNIT,
                    "ms_per_step": e2e_t if e2e_ms else None,
                    "h2d_bytes_per_step": int(h2d_bytes), "d2h_bytes_per_step": int(d2h_bytes)}}
    if args.medium_steps > 0 and world == 1:
        try:
            line["medium"] = medium(args, api, torch, stream, tc)
        except Exception as e:
            line["medium"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if args.serve_seconds > 0 and world == 1:
        try:
            line["serving"] = serving(args, api, torch)
        except Exception as e:   # the served stream is reported, not required for the line
            line["serving"] = {"error": "%s: %s" % (type(e).__name__, e)}
    if args.batch > 0 and world == 1:
        try:
            line["batched_lockstep"] = batched_lockstep(args, api, torch)
        except Exception as e:
            line["batched_lockstep"] = {"error": "%s: %s" % (type(e).__name__, e)}
        for key, t in (("batched", 0), ("batched_tc", 1)):
            try:
                line[key] = batched(args, api, torch, tc=t)
            except Exception as e:
                line[key] = {"error": "%s: %s" % (type(e).__name__, e)}
    if not args.no_cpu_baseline and world == 1:
        try:
            tm = oracle_sample()
            t1 = oracle_sample(threads=1)
            step_s = oracle_step_seconds(tm, counts)
            line["cpu_baseline"] = {"value": STATES_PER_STEP / step_s, "unit": UNIT, "cores": os.cpu_count(),
                                    "kind": "oracle", "sample": sample_note(tm, counts),
                                    "single_thread_value": STATES_PER_STEP / oracle_step_seconds(t1, counts)}
        except Exception as e:
            line["cpu_baseline"] = {"error": "%s: %s" % (type(e).__name__, e)}
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# DRAM traffic of the K1 contraction from one ncu capture of the full-size
# launch (dram__bytes_read.sum + dram__bytes_write.sum, 1 pass, two launches of
# m = 40 trial vectors over a 132-row P-chunk of the large workload, under
# `bench.py --apply-only 3`): 9.85 GB per launch against 5.30 GB of
# algorithmic bytes.  The bench's launches (m = 20..40) are reported at the
# same ratio of their own algorithmic bytes.
K1_TRAFFIC_PER_ALGORITHMIC_BYTE = 9.85e9 / 5.30e9


def roofline(prof, rec_ms, rec_fl, rec_by, peaks, src, tc, clk, total_ms):
    """Roofline object of the dominant kernel (the K1 exchange contraction)."""
    kernel_ms = prof["ms"] / max(prof["launches"], 1)
    flops_launch = prof["flops"] / max(prof["launches"], 1)
    achieved = flops_launch / (kernel_ms * 1e-3) / 1e12 if prof["launches"] else 0.0
    if tc:
        # FP16 and BF16 run at the same dense tensor rate (nominal ratio 1)
        peak = peaks["bf16_tflops_sustained"]
        roof = {"bound": "tensor", "unit": "TFLOP/s",
                "peak_kind": "fp16 dense = bf16 sustained (nominal ratio 1), " + src,
                "note": "algorithmic flops 2*M*N*K; the hi+lo split issues 3 FP16 products per flop, "
                        "so frac <= 1/3 (mma_pipe_frac = 3 x frac)"}
    else:
        sm = (clk or {}).get("sm_max_mhz") or peaks.get("sm_max_mhz", 2070.0)
        peak = 152 * 128 * 2 * sm * 1e6 / 1e12
        roof = {"bound": "alu", "unit": "TFLOP/s",
                "peak_kind": "FP32 FFMA: 152 SMs x 128 lanes x 2 flop x %.0f MHz" % sm}
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
            "attainable_note": "per launch max(%g FP16 products per flop at the tensor peak, algorithmic bytes "
                               "at hbm_gbs %.0f); attainable_frac = sum of those / sum of measured times"
                               % (per_flop, peaks["hbm_gbs"])})
    traffic = None
    if tc and rec_by.size:
        traffic = float(rec_by.mean()) * K1_TRAFFIC_PER_ALGORITHMIC_BYTE
        roof["traffic_note"] = ("bytes per launch: the measured DRAM/algorithmic ratio of the full-size ncu "
                                "capture (%.2f) times this run's mean algorithmic bytes per launch"
                                % K1_TRAFFIC_PER_ALGORITHMIC_BYTE)
    roof.update({"achieved": achieved, "peak": peak, "frac": achieved / peak if peak else None,
                 "mma_pipe_frac": 3.0 * achieved / peak if (peak and tc) else None,
                 "traffic": traffic, "kernel": "exchange K1 contraction sum_(P,a) Z L_vv",
                 "launches": prof["launches"], "ms_per_launch": kernel_ms,
                 "share_of_step": prof["ms"] / total_ms if total_ms else None})
    return roof


def medium(args, api, torch, stream, tc):
    """Context object: the medium workload's step (Casida, 10 states, + alpha at
    3 frequencies, rid, MIXED) and the same step in the plain FP64 form."""
    from synth.generator import CONFIGS, dipoles, make_config

    cfg = CONFIGS[MEDIUM]
    p = make_config(MEDIUM)
    mu = dipoles(cfg["mu_seed"], cfg["n_dip"], p.n_ov)
    omegas = list(cfg["omegas"])
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    kidx = p.ris_K_index
    eo, ev, k = (torch.from_numpy(p.eps_occ.copy()).cuda(), torch.from_numpy(p.eps_vir.copy()).cuda(),
                 torch.from_numpy(kidx.copy()).cuda())
    s = api.Solver(p.n_occ, p.n_vir, eo, ev, f32(p.L_oo), f32(p.L_ov), f32(p.L_vv), f32(p.Lr_oo[kidx]),
                   f32(p.Lr_ov), f32(p.Lr_vv[kidx]), k, a_x=p.a_x, coulomb_factor=p.coulomb_factor,
                   t_cut_ha=p.t_cut_ha, precisions=2, dtype=api.F32, stream=stream.cuda_stream)
    o_rpa = api.default_opts(n_states=MEDIUM_STATES, precond=api.RID, precision=api.MIXED, tensor_cores=tc)
    o_pol = api.default_opts(precond=api.RID, precision=api.MIXED, tensor_cores=tc)

    def step(sv):
        return sv.solve_rpa(o_rpa, want_vectors=False), sv.solve_polar(o_pol, mu, omegas)

    try:
        for _ in range(2):
            step(s)
        torch.cuda.synchronize()
        ev_ = [torch.cuda.Event(enable_timing=True) for _ in range(args.medium_steps + 1)]
        ev_[0].record(stream)
        for i in range(args.medium_steps):
            a, b = step(s)
            ev_[i + 1].record(stream)
        torch.cuda.synchronize()
    finally:
        s.close()
    per = [ev_[i].elapsed_time(ev_[i + 1]) for i in range(args.medium_steps)]
    ms = ev_[0].elapsed_time(ev_[-1]) / args.medium_steps
    out = {"workload": MEDIUM, "value": MEDIUM_STATES / (ms / 1e3), "unit": UNIT, "ms_per_step": ms,
           "p50_ms": statistics.median(per), "steps": args.medium_steps,
           "rpa_n_iter": a["stats"]["n_iter"], "polar_n_iter": b["stats"]["n_iter"],
           "oracle_rpa_n_iter": golden()["rpa"]["n_iter"],
           "max_resid_certified": a["stats"]["max_resid_certified"]}
    if args.plain_steps > 0:
        f64 = lambda a_: torch.from_numpy(np.ascontiguousarray(a_, dtype=np.float64)).cuda()
        sp = api.Solver(p.n_occ, p.n_vir, eo, ev, f64(p.L_oo), f64(p.L_ov), f64(p.L_vv), f64(p.Lr_oo[kidx]),
                        f64(p.Lr_ov), f64(p.Lr_vv[kidx]), k, a_x=p.a_x, coulomb_factor=p.coulomb_factor,
                        t_cut_ha=p.t_cut_ha, precisions=1, dtype=api.F64, stream=stream.cuda_stream)
        o_rpa_p = api.default_opts(n_states=MEDIUM_STATES, precond=api.RID, precision=api.PLAIN)
        o_pol_p = api.default_opts(precond=api.RID, precision=api.PLAIN)
        pms = []
        try:
            for _ in range(args.plain_steps):
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                ra = sp.solve_rpa(o_rpa_p, want_vectors=False)
                rb = sp.solve_polar(o_pol_p, mu, omegas)
                e1.record(stream)
                torch.cuda.synchronize()
                pms.append(e0.elapsed_time(e1))
        finally:
            sp.close()
        pm = statistics.mean(pms)
        out["plain"] = {"value": MEDIUM_STATES / (pm / 1e3), "unit": UNIT, "ms_per_step": pm,
                        "steps": args.plain_steps, "dtype": "f64", "rpa_n_iter": ra["stats"]["n_iter"],
                        "polar_n_iter": rb["stats"]["n_iter"],
                        "max_abs_omega_diff_vs_mixed": float(np.max(np.abs(ra["omega"] - a["omega"])))}
        out["speedup_vs_plain"] = pm / ms
    return out


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
    states, MIXED (FP32 outer products on the SIMT path, or with tc the FP16
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
                        % ("FP16 hi+lo tcgen05" if tc else "FP32 SIMT")})
    return out


def small_solver(args, api, torch, stream):
    """A MIXED context for --apply-only / --kernel-breakdown on args.workload."""
    if args.workload == WORKLOAD:
        solver, meta, _, _ = load_large(api, torch, stream.cuda_stream)
        return solver, meta
    from synth.generator import make_config
    p = make_config(args.workload)
    f32 = lambda a: torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()
    kidx = p.ris_K_index
    s = api.Solver(p.n_occ, p.n_vir, torch.from_numpy(p.eps_occ.copy()).cuda(),
                   torch.from_numpy(p.eps_vir.copy()).cuda(), f32(p.L_oo), f32(p.L_ov), f32(p.L_vv),
                   f32(p.Lr_oo[kidx]), f32(p.Lr_ov), f32(p.Lr_vv[kidx]), torch.from_numpy(kidx.copy()).cuda(),
                   a_x=p.a_x, coulomb_factor=p.coulomb_factor, t_cut_ha=p.t_cut_ha, precisions=2,
                   dtype=api.F32, stream=stream.cuda_stream)
    return s, {"n_occ": p.n_occ, "n_vir": p.n_vir}


def batched_lockstep(args, api, torch):
    """The batched workload as one lockstep batch (tddft_solve_tda_batch): the
    same 256 TDA solves as `batched` (n_occ ~ U{8..64}, n_vir = n_occ x U{4..8},
    n_aux = 5 n_mo, ris n_aux = 9 ceil(n_occ/2), 5-10 states, rid, FP32 outer
    products, BF16 ris) on 64 distinct resident problems, advanced together;
    grouped launches, captured operator graph, autotuned tiles.  Every solve
    finishes when the batch does, so its latency is the batch time."""
    from synth.device import problem_kw

    g = np.random.Generator(np.random.Philox(key=np.array([2405, 1], dtype=np.uint64)))
    n = args.batch
    sizes = []
    for _ in range(n):
        no = int(g.integers(8, 65))
        nv = no * int(g.integers(4, 9))
        sizes.append((no, nv, 5 * (no + nv), 9 * ((no + 1) // 2), int(g.integers(5, 11))))
    n_pool = min(64, n)
    solvers = []
    try:
        for i in range(n_pool):
            kw = problem_kw(3000 + i, *sizes[i][:4])
            solvers.append(api.Solver(**kw, precisions=2, dtype=api.F32))
            del kw
        torch.cuda.synchronize()
        entries = [solvers[i % n_pool] for i in range(n)]
        opts = [api.default_opts(n_states=sizes[i % n_pool][4], precond=api.RID, precision=api.MIXED)
                for i in range(n)]
        api.solve_tda_batch(entries[:8], opts[:8])      # warm-up (kernel loading)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, res, info = api.solve_tda_batch(entries, opts)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
    finally:
        for sv in solvers:
            sv.close()
    ok = sum(1 for r in res if r["stats"]["converged"])
    states = sum(len(r["omega"]) for r in res if r["stats"]["converged"])
    return {"solves": n, "converged": ok, "seconds": wall, "solves_per_s": ok / wall, "states_per_s": states / wall,
            "p50_ms": wall * 1e3, "p99_ms": wall * 1e3, "distinct_problems": n_pool,
            "outer_iterations": info["outer_iterations"], "launches": info["launches"],
            "graph_replays": info["graph_launches"], "graph_nodes": info["graph_nodes"],
            "autotune_ms": info["autotune_ms"], "tile_variant": info["variant"],
            "note": "one lockstep batch; every solve completes with the batch, so p50 = p99 = batch time"}


def apply_only(args, api, solver, meta, tc, stream):
    """K exact pair products on 2*n_states device vectors, each timed with CUDA events."""
    import torch
    from synth.generator import CONFIGS
    m = 2 * CONFIGS[args.workload]["n_states"]
    X = torch.from_numpy(np.random.default_rng(7).standard_normal((m, meta["n_occ"] * meta["n_vir"]))).cuda()
    ms = []
    for _ in range(args.apply_only):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        solver.apply(1, X, precision=api.MIXED, tensor_cores=bool(tc))
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    print(json.dumps({"apply_only": args.apply_only, "m": m, "ms": ms,
                      "workload": args.workload, "tensor_cores": bool(tc)}), flush=True)


def kernel_breakdown(args, api, solver, tc):
    """One warm step under the CUDA activity profiler (CUPTI): every kernel and
    copy with its device time; printed as one JSON line."""
    import collections
    import re
    import torch
    from torch.profiler import ProfilerActivity, profile
    from synth.generator import CONFIGS, dipoles

    if args.workload == WORKLOAD:
        o = api.default_opts(n_states=N_STATES, precond=api.RID, precision=api.MIXED, tensor_cores=tc)

        def step():
            solver.solve_tda(o, want_vectors=False)
            solver.solve_rpa(o, want_vectors=False)
    else:
        cfg = CONFIGS[args.workload]
        mu = dipoles(cfg["mu_seed"], cfg.get("n_dip", 3), solver.n_ov)
        o_rpa = api.default_opts(n_states=cfg["n_states"], precond=api.RID, precision=api.MIXED, tensor_cores=tc)
        o_pol = api.default_opts(precond=api.RID, precision=api.MIXED, tensor_cores=tc)

        def step():
            solver.solve_rpa(o_rpa, want_vectors=False)
            solver.solve_polar(o_pol, mu, list(cfg.get("omegas", (0.0,))))

    step()
    torch.cuda.synchronize()
    # a first activity session in a process has returned no records of this
    # library's launches; one short session on a torch kernel comes first
    with profile(activities=[ProfilerActivity.CUDA]):
        torch.zeros(1, device="cuda").add_(1.0)
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
                      "events": len(ev), "wall_ms": wall * 1e3, "workload": args.workload}), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    our_arm(args, rank, world, local)


if __name__ == "__main__":
    main()
