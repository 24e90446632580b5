"""Benchmark of the restarted-PDHG hot path on one B300 (or N independent replicas).

Workload (default): the large planted sparse LP -- n = 2e6 columns, m = 1e6 rows (40 %
equalities), nnz ~ 2e7 with Zipf(1.5) row lengths, values +-10^U(-3,3), mixed bounds,
Ruiz + Pock-Chambolle scaling (lpgen.planted_zipf, seed 0 + rank).

A step is one check interval: check_every (64) PDHG iterations -- each one the fused
K'y SpMV + primal step kernel and the fused K x SpMV + dual step kernel -- followed by
the restart/termination check (three SpMVs, the KKT and duality-gap reductions, the
restart decision and the restart).  `value` is PDHG iterations per second of the whole
job (all ranks), timed with CUDA events on the current stream around one pdlp_solve of
steps * 64 iterations (tolerance 0, so every step runs), inputs resident in HBM.

    python bench.py [--steps K] [--warmup W] [--impl ours|reference] [--workload large|small]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time-to-1e-4 KKT & PDHG iter/s (HBM GB/s vs peak); batched & warm-start vs plain"
CHECK_EVERY = 64


def aggregate_ranks(ms_local, units_local, world, dist_mod=None):
    """Whole-job timing of replicas: the slowest rank's time (max over ranks) and the
    units of all ranks (each rank does the same number) divided by it, per second."""
    ms = float(ms_local)
    if dist_mod is not None and world > 1:
        import torch
        dev = "cuda" if dist_mod.get_backend() == "nccl" else "cpu"
        t = torch.tensor([ms], dtype=torch.float64, device=dev)
        dist_mod.all_reduce(t, op=dist_mod.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_local / (ms * 1e-3)


def workload(name, rank):
    import lpgen
    if name == "large":
        lp = lpgen.planted_zipf(seed=rank, n=2_000_000, m=1_000_000, nnz=20_000_000)
        desc = ("planted sparse LP, n=2e6, m=1e6 (m1=4e5), nnz~2e7, Zipf(1.5) row lengths capped 1e4, "
                "values +-10^U(-3,3), bounds 25% free / 50% [0,U(1,100)] / 25% [0,inf), "
                "Ruiz(10)+Pock-Chambolle scaling")
    elif name == "medium":
        lp = lpgen.planted_zipf(seed=rank, n=500_000, m=250_000, nnz=5_000_000)
        desc = ("planted sparse LP, n=5e5, m=2.5e5, nnz~5e6, the large recipe at a quarter of the size, "
                "Ruiz(10)+Pock-Chambolle scaling")
    elif name == "small":
        lp = lpgen.planted_small(seed=rank)
        desc = "planted LP m1=200, m2=300, n=1000, nnz=5000, N(0,1) values"
    else:
        raise SystemExit(f"unknown workload {name}")
    return lp, desc


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6400.0}, "fallback"


def kernel_bytes(lp):
    """Algorithmic bytes per launch of the two fused iteration kernels (unique-bytes model:
    FP64 values, int32 indices, each array touched once, the gathered vector once)."""
    nnz, m, n = lp["val"].shape[0], lp["m"], lp["n"]
    primal = 12 * nnz + 4 * (n + 1) + 8 * m + 56 * n   # K' CSR, y gather, x c l u sx read, x sx written
    dual = 12 * nnz + 4 * (m + 1) + 8 * n + 56 * m     # K CSR, x gather, y q Kx sy read, y Kx sy written
    return primal, dual


def stored_traffic(kernel, workload_name):
    """DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from the
    committed ncu summary profiles/ncu_traffic.txt, if it was taken on the current
    kernel source and this workload; else None.  Format: `key = value` lines
    (source_sha, workload) and `kernel <name> = <bytes per launch>` lines."""
    path = os.path.join(ROOT, "profiles", "ncu_traffic.txt")
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return None
    rec, kern = {}, {}
    for ln in lines:
        if "=" not in ln or ln.lstrip().startswith("#"):
            continue
        key, val = (t.strip() for t in ln.split("=", 1))
        if key.startswith("kernel "):
            kern[key[len("kernel "):].strip()] = float(val)
        else:
            rec[key] = val
    src = os.path.join(ROOT, "paper_2312_14832_b300", "csrc", "kernels.cuh")
    h = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec.get("source_sha") != h or rec.get("workload") != workload_name:
        return None
    return kern.get(kernel)


class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi during the timed region."""

    def __init__(self, dev):
        self.p = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(dev)
            sel = f"{pr.pci_domain_id:08X}:{pr.pci_bus_id:02X}:{pr.pci_device_id:02X}.0"
        except Exception:
            sel = str(dev)
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", sel, f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
            out, _ = self.p.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [v.strip() for v in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "samples": len(sm),
                "reasons": sorted(reasons)}


def time_to_tol_small(pk, seed=0):
    """Cold-start time to 1e-4 and 1e-8 relative KKT on the small planted LP (m1=200,
    m2=300, n=1000, nnz=5000): GPU (device time of pdlp_solve, CUDA events; the automatic
    engine is the persistent one for this LP, engine 1 the kernels launched per
    iteration), the batched solver with one LP, and the CPU oracle (wall time of the
    whole oracle solve, single thread)."""
    import lpgen
    import oracle
    lp = lpgen.planted_small(seed)
    out = {}
    # the persistent single-CTA path (a batch of one LP): no kernel launches per iteration
    with pk.BatchSolver.from_lps([lp]) as b:
        b.solve(tol=1e-4, want_points=False)
        for tol in (1e-4, 1e-8):
            t0 = time.perf_counter()
            r = b.solve(tol=tol, want_points=False)[0]
            wall = time.perf_counter() - t0
            out[f"persistent_{tol:.0e}"] = {"gpu_s": r["device_ms"] * 1e-3, "gpu_wall_s": wall, "iters": r["iters"],
                                            "rel_obj_err_vs_planted": abs(r["primal_obj"] - lp["obj_star"]) /
                                            abs(lp["obj_star"])}
    with pk.Solver.from_lp(lp) as s:
        s.solve(tol=1e-4, want_point=False, engine=1)   # warm-up (graph capture)
        for tol in (1e-4, 1e-8):
            rk = s.solve(tol=tol, want_point=False, engine=1)
            out[f"kernels_{tol:.0e}"] = {"gpu_s": rk["device_ms"] * 1e-3, "gpu_wall_s": rk["solve_s"],
                                         "iters": rk["iters"], "note": "engine 1: kernels launched per iteration"}
            r = s.solve(tol=tol, want_point=False)
            t0 = time.perf_counter()
            ref = oracle.solve(lp, tol=tol)
            cpu = time.perf_counter() - t0
            out[f"{tol:.0e}"] = {
                "gpu_s": r["device_ms"] * 1e-3, "gpu_wall_s": r["solve_s"], "iters": r["iters"],
                "oracle_iters": int(ref["iters"]), "oracle_s": cpu, "speedup": cpu / max(r["solve_s"], 1e-9),
                "rel_obj_err_vs_planted": abs(r["primal_obj"] - lp["obj_star"]) / abs(lp["obj_star"]),
                "rel_obj_diff_vs_oracle": abs(r["primal_obj"] - ref["primal_obj"]) / abs(ref["primal_obj"])}
    return out


def gather_ceiling(nnz, nx):
    """Runs the committed stream/gather microbenchmark (csrc/gather_ceiling.cu) for the
    workload's nnz and gathered-vector length."""
    from paper_2312_14832_b300 import build as pkbuild
    try:
        out = subprocess.check_output([pkbuild.build_ceiling(), str(int(nnz)), str(int(nx))], timeout=120)
        return json.loads(out.decode().strip().splitlines()[-1])
    except Exception as e:  # the bench line still prints without it
        return {"error": str(e)[:200]}


def cpu_info():
    """Threads available to this process and the host CPU's model name."""
    model = None
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.startswith("model name"):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    try:
        cores = len(os.sched_getaffinity(0))
    except AttributeError:
        cores = os.cpu_count() or 1
    return cores, model


def cpu_baseline(lp, seconds=12.0):
    """The oracle's PDHG step on the same LP: on every host core (oracle.ThreadedStep,
    the same arithmetic split over threads, bit-identical to the serial step) for about
    two thirds of `seconds`, and single-threaded (oracle.pdhg_step) for the rest."""
    import oracle
    cores, model = cpu_info()
    x0 = np.clip(np.zeros(lp["n"]), lp["l"], lp["u"])
    y0 = np.zeros(lp["m"])
    # all cores
    T = oracle.ThreadedStep(lp, cores)
    x, y = x0.copy(), y0.copy()
    T.step(x, y, 1e-3, 1.0)                      # untimed: pages the arrays in
    steps, t0 = 0, time.perf_counter()
    while True:
        T.step(x, y, 1e-3, 1.0)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds * 2 / 3 or steps >= 2000:
            break
    par = {"value": steps / el, "steps": steps, "s": el}
    # one thread
    x, y = x0.copy(), y0.copy()
    steps1, t0 = 0, time.perf_counter()
    while True:
        x, y = oracle.pdhg_step(lp, x, y, 1e-3, 1.0)
        steps1 += 1
        el1 = time.perf_counter() - t0
        if el1 >= seconds / 3 or steps1 >= 200:
            break
    return {"value": par["value"], "unit": "PDHG iter/s", "cores": cores, "kind": "oracle", "cpu_model": model,
            "sample": f"{par['steps']} oracle PDHG steps (K'y, primal step, K(2x+-x), dual step; "
                      f"orc_pdhg_step_par on {cores} threads) on the full workload, {par['s']:.1f} s",
            "single_thread": {"value": steps1 / el1, "unit": "PDHG iter/s", "cores": 1,
                              "sample": f"{steps1} orc_pdhg_step steps, {el1:.1f} s"}}


_FP64_PEAK = None


def fp64_peak():
    """FP64 FMA lane-operations/s of this GPU, measured by the committed microbenchmark
    (csrc/fp64_peak.cu) once per process: the arithmetic roof of the FP64 kernels."""
    global _FP64_PEAK
    if _FP64_PEAK is None:
        from paper_2312_14832_b300 import build as pkbuild
        try:
            out = subprocess.check_output([pkbuild.build_fp64_peak()], timeout=120)
            _FP64_PEAK = json.loads(out.decode().strip().splitlines()[-1])
        except Exception as e:
            _FP64_PEAK = {"error": str(e)[:200]}
    return _FP64_PEAK


def fp64_roofline(achieved, note):
    pk_ = fp64_peak()
    peak = pk_.get("fma_per_s")
    return {"bound": "alu", "unit": "FMA/s", "achieved": achieved, "peak": peak,
            "frac": achieved / peak if peak else None, "peak_kind": "measured by csrc/fp64_peak.cu in this run",
            "probe": pk_, "note": note}


def bench_batched(args):
    """Batched workload: `count` independent planted LPs (lpgen.batch_planted, seed 0),
    n ~ U(50, 5000), m ~ U(0.3, 0.8) n, density U(0.5%, 5%), N(0,1) values; solved to
    1e-4 relative KKT by one persistent launch, against the same LPs solved one after
    the other by the single-LP solver (a sample of them, scaled to the full count)."""
    import torch
    import lpgen
    import paper_2312_14832_b300 as pk
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    lps = lpgen.batch_planted(args.count, seed=0)
    gen_s = time.perf_counter() - t0
    nnz = [int(lp["val"].shape[0]) for lp in lps]
    t0 = time.perf_counter()
    b = pk.BatchSolver.from_lps(lps, scaling=args.batch_scaling)
    setup_s = time.perf_counter() - t0
    b.solve(tol=1e-4, max_iter=64, want_points=False, batch_tune=1)      # warm-up launch
    clk = Clocks(0)
    # the team-size rule alone, then the first solve with the online autotuner (its
    # timed slices are part of the solve and of its time), then a solve that keeps the
    # tuned choice (one CUDA graph holding the persistent launch)
    res_rule = b.solve(tol=1e-4, max_iter=args.batch_max_iter, want_points=False, batch_tune=1)
    inf_rule = b.info()
    res_first = b.solve(tol=1e-4, max_iter=args.batch_max_iter, want_points=False)
    inf_tuned = b.info()
    res = b.solve(tol=1e-4, max_iter=args.batch_max_iter, want_points=False)
    res_again = res
    k = inf_tuned["batch_tuned"]
    tuning = {"rule": {"device_s": res_rule[0]["device_ms"] * 1e-3, "team": inf_rule["batch_team"],
                       "resident": inf_rule["batch_resident"]},
              "tuned_first_solve": {"device_s": res_first[0]["device_ms"] * 1e-3, "launches": res_first[0]["launches"],
                                    "note": "the online autotuner's timed slices are this solve's own iterations"},
              "candidates": [{"team": inf_tuned["tune_team"][i], "resident": inf_tuned["tune_resident"][i],
                              "stored_gbs": inf_tuned["tune_gbs"][i]} for i in range(min(k, 8))],
              "kept": {"team": inf_tuned["batch_team"], "resident": inf_tuned["batch_resident"]},
              "tuned_again": {"device_s": res_again[0]["device_ms"] * 1e-3, "launches": res_again[0]["launches"]},
              "same_iteration_counts": all(a["iters"] == c["iters"] == d["iters"]
                                           for a, c, d in zip(res, res_rule, res_first)),
              "max_rel_obj_diff_vs_rule": max(abs(a["primal_obj"] - c["primal_obj"]) / (1 + abs(c["primal_obj"]))
                                              for a, c in zip(res, res_rule))}
    one_launch_s = res[0]["device_ms"] * 1e-3
    two_stage = None
    if args.batch_tail > 0:
        # the same solve in two stages: LPs past batch_tail iterations continue on teams
        res2 = b.solve(tol=1e-4, max_iter=args.batch_max_iter, want_points=False, batch_tail_iters=args.batch_tail)
        inf = b.info()
        same = all(r1["iters"] == r2["iters"] for r1, r2 in zip(res, res2))
        two_stage = {"device_s": res2[0]["device_ms"] * 1e-3, "tail_iters": args.batch_tail,
                     "resumed": inf["batch_resumed"], "second_stage_team": inf["batch_team"],
                     "same_iteration_counts": same,
                     "max_rel_obj_diff": max(abs(r1["primal_obj"] - r2["primal_obj"]) / (1 + abs(r1["primal_obj"]))
                                             for r1, r2 in zip(res, res2))}
        if res2[0]["device_ms"] < res[0]["device_ms"]:
            res = res2
    mixed = None
    if args.batch_mixed:
        # FP32 iterations with FP64 checks; unfinished LPs continue in FP64
        bm = pk.BatchSolver.from_lps(lps, scaling=args.batch_scaling, precision=pk.MIXED)
        bm.solve(tol=1e-4, max_iter=64, want_points=False)
        rm = bm.solve(tol=1e-4, max_iter=args.batch_max_iter, want_points=False)
        fp32 = np.array([r["fp32_iters"] for r in rm])
        itm = np.array([r["iters"] for r in rm])
        mixed = {"device_s": rm[0]["device_ms"] * 1e-3, "lps_per_s": args.count / (rm[0]["device_ms"] * 1e-3),
                 "optimal": int(sum(r["status"] == 0 for r in rm)), "iters_mean": float(itm.mean()),
                 "fp32_iter_share": float(fp32.sum() / max(itm.sum(), 1)),
                 "continued_in_fp64": bm.info()["batch_resumed"],
                 "max_rel_obj_diff_vs_fp64": max(abs(a["primal_obj"] - c["primal_obj"]) / (1 + abs(a["primal_obj"]))
                                                 for a, c in zip(res, rm) if a["status"] == 0 and c["status"] == 0),
                 "max_rel_error_of_optimal": max(max(r["rel_primal"], r["rel_dual"], r["rel_gap"])
                                                 for r in rm if r["status"] == 0)}
        bm.close()
    clocks = clk.stop()
    dev_s = res[0]["device_ms"] * 1e-3
    iters = np.array([r["iters"] for r in res])
    status = np.array([r["status"] for r in res])
    fma = float(np.sum(2.0 * np.array(nnz) * iters))
    slow = int(np.argmax(iters))
    tail = {"iters_p50": float(np.percentile(iters, 50)), "iters_p99": float(np.percentile(iters, 99)),
            "slowest_lp": {"index": slow, "iters": int(iters[slow]), "n": int(lps[slow]["n"]),
                           "m": int(lps[slow]["m"]), "nnz": nnz[slow]}}
    b.close()
    # sequential single-LP solves on a sample
    stride = max(1, args.count // args.seq_sample)
    sample = list(range(0, args.count, stride))
    seq_s, seq_it = 0.0, 0
    for i in sample:
        with pk.Solver.from_lp(lps[i], scaling=args.batch_scaling) as s1:
            r1 = s1.solve(tol=1e-4, max_iter=args.batch_max_iter, want_point=False)
        seq_s += r1["solve_s"]
        seq_it += r1["iters"]
    seq_total = seq_s * args.count / len(sample)
    # the CPU oracle (single thread) solving LPs of the same sample to the same tolerance,
    # for about args.cpu_seconds, scaled to the whole batch
    import oracle
    cpu_s, cpu_n, t_cpu = 0.0, 0, time.perf_counter()
    for i in sample:
        if time.perf_counter() - t_cpu > args.cpu_seconds / 2:
            break
        t1 = time.perf_counter()
        oracle.solve(lps[i], tol=1e-4, scaling=args.batch_scaling, max_iter=args.batch_max_iter)
        cpu_s += time.perf_counter() - t1
        cpu_n += 1
    cpu_total = cpu_s * args.count / max(cpu_n, 1)
    # every host core: the oracle's solves of sample LPs run side by side on a thread pool
    # (the C oracle runs without the interpreter lock), LPs per wall second
    from concurrent.futures import ThreadPoolExecutor
    cores, model = cpu_info()
    solve1 = lambda i: oracle.solve(lps[i], tol=1e-4, scaling=args.batch_scaling, max_iter=args.batch_max_iter)
    par_n, t_par = 0, time.perf_counter()
    with ThreadPoolExecutor(max_workers=cores) as ex:
        while time.perf_counter() - t_par < args.cpu_seconds / 2:
            idx = [sample[(par_n + j) % len(sample)] for j in range(cores)]
            list(ex.map(solve1, idx))
            par_n += cores
    par_s = time.perf_counter() - t_par
    best = args.count / dev_s
    variant = "fp64"
    if mixed is not None and mixed["optimal"] >= int(np.sum(status == 0)) and mixed["lps_per_s"] > best:
        best, variant = mixed["lps_per_s"], "fp32 iterations, fp64 checks"
    out = {"metric": METRIC, "value": best, "value_variant": variant, "unit": "LPs/s to 1e-4", "n_gpus": 1,
           "higher_is_better": True, "dtype": "f64", "data": "synthetic", "impl": "ours-batched",
           "config": {"workload": f"{args.count} planted LPs, n~U(50,5000), m~U(0.3,0.8)n, density U(0.5%,5%), "
                                  "N(0,1) values (lpgen.batch_planted seed 0)",
                      "scaling": args.batch_scaling, "total_nnz": int(np.sum(nnz))},
           "batch_device_s": dev_s, "optimal": int(np.sum(status == 0)), "iters_mean": float(iters.mean()),
           "iters_max": int(iters.max()),
           "roofline": fp64_roofline(fma / dev_s, "FP64 FMAs of both SpMVs per iteration"),
           "sequential": {"sample": len(sample), "sample_s": seq_s, "sample_iters": seq_it,
                          "estimated_total_s": seq_total, "lps_per_s": args.count / seq_total},
           "speedup_vs_sequential": seq_total / dev_s, "setup_s": setup_s, "generate_s": gen_s,
           "cpu_baseline": {"value": par_n / par_s, "unit": "LPs/s to 1e-4", "cores": cores, "kind": "oracle",
                            "cpu_model": model,
                            "sample": f"oracle.solve to 1e-4 of {par_n} LPs of the sample, {cores} at a time on a "
                                      f"thread pool, {par_s:.1f} s",
                            "single_thread": {"value": args.count / cpu_total, "unit": "LPs/s to 1e-4", "cores": 1,
                                              "sample": f"oracle.solve to 1e-4 on {cpu_n} LPs of the sample "
                                                        f"({cpu_s:.1f} s), scaled to {args.count} LPs"}},
           "one_launch_device_s": one_launch_s, "tuning": tuning, "two_stage": two_stage, "tail": tail,
           "mixed": mixed,
           "clocks": clocks}
    print(json.dumps(out))


def bench_mcf(args):
    """Mixed precision on the multicommodity-flow LP (lpgen.mcf: 8 commodities, 2e5 nodes,
    1e6 arcs, n = 8e6, m = 2.6e6, nnz = 2.4e7, Ruiz + Pock-Chambolle scaling): PDHG
    iterations/s and time to 1e-4 for FP64 and for MIXED (FP32 iterations, FP64
    checks and refinement) with the +-1 entries stored as sign bits ("mixed", the
    automatic choice) and as FP32 value copies ("mixed_values"), and the relative
    objective difference between FP64 and MIXED."""
    import torch
    import lpgen
    import paper_2312_14832_b300 as pk
    torch.cuda.set_device(0)
    lp = lpgen.mcf(0)
    stream = torch.cuda.current_stream()
    out = {"metric": METRIC, "unit": "PDHG iter/s", "n_gpus": 1, "higher_is_better": True,
           "data": "synthetic", "impl": "ours-mcf",
           "config": {"workload": "multicommodity flow: 8 commodities, 2e5 nodes, 1e6 arcs (with a Hamiltonian "
                                  "cycle), n=8e6, m=2.6e6, nnz=2.4e7, +-1 entries, costs U(1,10), cap U(5,50), "
                                  "planted feasible flow; Ruiz(10)+Pock-Chambolle scaling",
                      "check_every": CHECK_EVERY}}
    iters = args.steps * CHECK_EVERY
    nnz, mn = lp["row_ptr"][-1], lp["m"] + lp["n"]
    # unique bytes of one iteration's two products (values + indices, the vectors each
    # step reads and writes, the gathered vector once): FP64 24 nnz + 68 (m + n); FP32
    # value copies 16 nnz + 32 (m + n); sign bits 8 nnz + 36 (m + n) (D_c^2, D_r^2 read
    # by the steps)
    model = {0: 24.0 * nnz + 68.0 * mn, 1: 16.0 * nnz + 32.0 * mn, 2: 8.0 * nnz + 36.0 * mn}
    variants = (("fp64", pk.FP64, {}), ("mixed", pk.MIXED, {}), ("mixed_values", pk.MIXED, {"mixed_values": 1}))
    for name, prec, extra in variants:
        s = pk.Solver.from_lp(lp, scaling=1, precision=prec, stream=stream.cuda_stream, **extra)
        storage = s.info()["mixed_values"]
        s.solve(tol=0.0, max_iter=max(args.warmup, 1) * CHECK_EVERY, want_point=False,
                mixed_switch_tol=1e-30)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        # tol 0 and a switch tolerance that is never reached: every interval in this precision
        r = s.solve(tol=0.0, max_iter=iters, want_point=False, mixed_switch_tol=1e-30)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        mp, md = s.time_iterations(100)
        rt = s.solve(tol=1e-4, time_limit_s=args.mcf_budget)
        status = ["optimal", "iter_limit", "time_limit", "numerical"]
        out[name] = {"iter_per_s": iters / (ms * 1e-3), "ms_primal": mp, "ms_dual": md,
                     "fp32_storage": ["none (fp64)", "fp32 value copies", "sign bits"][storage],
                     "bytes_per_iter_model": model[storage],
                     "kernels_gbs": model[storage] / ((mp + md) * 1e-3) / 1e9,
                     "fp32_iters_in_timed": r["fp32_iters"],
                     "time_to_1e-4": {"status": status[rt["status"]],
                                      "iters": rt["iters"], "fp32_iters": rt["fp32_iters"],
                                      "device_s": rt["device_ms"] * 1e-3, "primal_obj": rt["primal_obj"],
                                      "rel_primal": rt["rel_primal"], "rel_dual": rt["rel_dual"],
                                      "rel_gap": rt["rel_gap"]}}
        out[name + "_x"] = rt["x"]
        if args.mcf_tol_hi > 0 and name != "mixed_values":
            # high accuracy: in MIXED the FP32 phase hands over to FP64 refinement; the
            # returned point's three relative tests re-evaluated by the FP64 oracle
            import oracle
            hk = {"mixed_switch_tol": args.mcf_switch_tol} if args.mcf_switch_tol > 0 else {}
            rh = s.solve(tol=args.mcf_tol_hi, time_limit_s=args.mcf_budget, **hk)
            orp, ord_, org = oracle.relative_errors(lp, rh["x"], rh["y"])
            out[name][f"time_to_{args.mcf_tol_hi:g}"] = {
                "status": status[rh["status"]], "iters": rh["iters"], "fp32_iters": rh["fp32_iters"],
                "fp32_share": rh["fp32_iters"] / max(rh["iters"], 1), "device_s": rh["device_ms"] * 1e-3,
                "primal_obj": rh["primal_obj"], "rel_errors_solver": [rh["rel_primal"], rh["rel_dual"], rh["rel_gap"]],
                "rel_errors_oracle": [orp, ord_, org], "obj_star": lp.get("obj_star")}
            out[name + "_hi_obj"] = rh["primal_obj"]
        s.close()
    a, b = out["fp64"]["time_to_1e-4"], out["mixed"]["time_to_1e-4"]
    out["mixed_vs_fp64"] = {"iter_speedup": out["mixed"]["iter_per_s"] / out["fp64"]["iter_per_s"],
                            "time_to_1e-4_speedup": a["device_s"] / max(b["device_s"], 1e-9),
                            "rel_obj_diff": abs(a["primal_obj"] - b["primal_obj"]) / abs(a["primal_obj"]),
                            "rel_x_diff": float(np.linalg.norm(out["fp64_x"] - out["mixed_x"]) /
                                                np.linalg.norm(out["fp64_x"]))}
    c = out["mixed_values"]
    out["sign_bits_vs_value_copies"] = {
        "iter_speedup": out["mixed"]["iter_per_s"] / c["iter_per_s"],
        "kernel_speedup": (c["ms_primal"] + c["ms_dual"]) / (out["mixed"]["ms_primal"] + out["mixed"]["ms_dual"]),
        "time_to_1e-4_speedup": c["time_to_1e-4"]["device_s"] / max(b["device_s"], 1e-9),
        "rel_x_diff": float(np.linalg.norm(out["mixed_values_x"] - out["mixed_x"]) /
                            np.linalg.norm(out["mixed_values_x"]))}
    del out["fp64_x"], out["mixed_x"], out["mixed_values_x"]
    if args.mcf_tol_hi > 0:
        out["mixed_vs_fp64"][f"rel_obj_diff_at_{args.mcf_tol_hi:g}"] = (
            abs(out["fp64_hi_obj"] - out["mixed_hi_obj"]) / abs(out["fp64_hi_obj"]))
        del out["fp64_hi_obj"], out["mixed_hi_obj"]
    base = cpu_baseline(lp, seconds=args.cpu_seconds)
    base["sample"] = base["sample"].replace("full workload", "same LP (FP64)")
    out["cpu_baseline"] = base
    out["value"] = out["mixed"]["iter_per_s"]
    out["dtype"] = "f32 iterations / f64 checks"
    print(json.dumps(out))


def bench_pagerank(args):
    """PageRank-shaped LP of the size of the paper's rand_1m instance (lpgen.pagerank:
    n = 1e6 columns, m = 1e6 + 1 rows, nnz = 8e6, one dense row stored as a wide row),
    Ruiz + Pock-Chambolle scaling: time to 1e-6 relative KKT (the accuracy of the
    paper's large-instance table) with the constant step of Section 2, with the
    adaptive step rule and in mixed precision; PDHG iterations/s; the CPU oracle's time
    per iteration on the same LP (a few iterations, single thread)."""
    import torch
    import lpgen
    import oracle
    import paper_2312_14832_b300 as pk
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    lp = lpgen.pagerank(args.pr_nodes, seed=0)
    gen_s = time.perf_counter() - t0
    stream = torch.cuda.current_stream()
    out = {"metric": METRIC, "unit": "s to 1e-6", "n_gpus": 1, "higher_is_better": False,
           "data": "synthetic", "impl": "ours-pagerank", "dtype": "f64",
           "config": {"workload": f"PageRank LP on a random graph (out-degree 6, damping 0.85), n={lp['n']}, "
                                  f"m={lp['m']}, nnz={len(lp['val'])}; Ruiz(10)+Pock-Chambolle scaling",
                      "tol": 1e-6, "check_every": CHECK_EVERY},
           "paper_context": {"instance": "rand_1m_nodes (m=1,000,001, n=1e6, nnz=7,999,982)",
                             "cuPDLP-C H100 s": 3.56, "note": "different random graph; context only"}}
    runs = (("constant", dict(step_rule=0, precision=pk.FP64)), ("adaptive", dict(step_rule=1, precision=pk.FP64)),
            ("mixed", dict(step_rule=0, precision=pk.MIXED)))
    for name, kw in runs:
        t0 = time.perf_counter()
        s = pk.Solver.from_lp(lp, scaling=1, stream=stream.cuda_stream, **kw)
        setup_s = time.perf_counter() - t0
        s.solve(tol=0.0, max_iter=max(args.warmup, 1) * CHECK_EVERY, want_point=False)   # graph capture
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = args.steps * CHECK_EVERY
        e0.record(stream)
        s.solve(tol=0.0, max_iter=iters, want_point=False, mixed_switch_tol=1e-30)
        e1.record(stream)
        torch.cuda.synchronize()
        ips = iters / (e0.elapsed_time(e1) * 1e-3)
        r = s.solve(tol=1e-6, time_limit_s=args.pr_budget)
        err = float(np.abs(r["x"] - lp["x_star"]).max() / lp["x_star"].max())
        out[name] = {"time_to_1e-6_s": r["device_ms"] * 1e-3, "wall_s": r["solve_s"], "iters": r["iters"],
                     "accepted": r["accepted"], "fp32_iters": r["fp32_iters"], "restarts": r["restarts"],
                     "status": ["optimal", "iter_limit", "time_limit", "numerical"][r["status"]],
                     "rel_errors": [r["rel_primal"], r["rel_dual"], r["rel_gap"]],
                     "max_rel_dev_from_pagerank_vector": err, "iter_per_s": ips, "setup_s": setup_s,
                     "wide_rows_K": s.info()["wide_rows_K"]}
        s.close()
    # the CPU oracle: time per PDHG step on the same LP (scaled problem not needed for a step)
    x = np.zeros(lp["n"])
    y = np.zeros(lp["m"])
    t0 = time.perf_counter()
    k = 0
    while time.perf_counter() - t0 < 10.0:
        x, y = oracle.pdhg_step(lp, x, y, 0.5, 1.0)
        k += 1
    cpu_it_s = (time.perf_counter() - t0) / k
    best = min(out[nm]["time_to_1e-6_s"] for nm, _ in runs if out[nm]["status"] == "optimal")
    out["value"] = best
    out["cpu_baseline"] = {"value": cpu_it_s * out["constant"]["iters"], "unit": "s to 1e-6 (estimated)",
                           "cores": 1, "kind": "oracle",
                           "sample": f"{k} oracle PDHG steps ({cpu_it_s * 1e3:.1f} ms each) x the GPU's "
                                     f"constant-step iteration count"}
    out["generate_s"] = gen_s
    print(json.dumps(out))


def bench_teams(args):
    """Small LPs on the batched persistent kernel with thread-block-cluster teams: the
    small planted LP alone (time to 1e-4 and 1e-8 for teams of 1..16 CTAs, matrix
    slices streamed or resident in shared memory; best of 3 launches), and 64 planted
    LPs with n ~ U(2000, 5000).  --fixed-iters N instead runs one launch of N iterations
    of the small LP (team --team-one, resident slices), for profiler captures."""
    import torch
    import lpgen
    import paper_2312_14832_b300 as pk
    torch.cuda.set_device(0)
    lp = lpgen.planted_small(0)
    if args.fixed_iters > 0:
        with pk.BatchSolver.from_lps([lp]) as b:
            r = b.solve(tol=0.0, max_iter=args.fixed_iters, want_points=False, cluster_ctas=args.team_one,
                        resident=2)[0]
        print(json.dumps({"impl": "ours-teams-fixed", "iters": r["iters"], "device_ms": r["device_ms"],
                          "team": args.team_one}))
        return
    out = {"metric": METRIC, "unit": "ms to 1e-4 (small planted LP)", "n_gpus": 1, "higher_is_better": False,
           "data": "synthetic", "impl": "ours-teams", "dtype": "f64",
           "config": {"workload": "small planted LP (m1=200, m2=300, n=1000, nnz=5000), one LP per launch; "
                                  "64 planted LPs n~U(2000,5000)"}}
    small = {}
    with pk.BatchSolver.from_lps([lp]) as b:
        for team in (1, 2, 4, 8, 16, 0):
            for res in (1, 2):
                b.solve(tol=1e-4, want_points=False, cluster_ctas=team, resident=res)
                row = {}
                for tol in (1e-4, 1e-8):
                    best = None
                    for _ in range(3):
                        r = b.solve(tol=tol, want_points=False, cluster_ctas=team, resident=res)[0]
                        best = r["device_ms"] if best is None else min(best, r["device_ms"])
                    row[f"{tol:.0e}"] = {"ms": best, "iters": r["iters"], "us_per_iter": 1e3 * best / r["iters"]}
                inf = b.info()
                row["team"], row["resident"] = inf["batch_team"], inf["batch_resident"]
                small[f"team={team} resident={res}"] = row
    out["small"] = small
    lps = lpgen.batch_planted(64, seed=11, n_lo=2000, n_hi=5000)
    med = {}
    with pk.BatchSolver.from_lps(lps) as b:
        for team in (1, 2, 4, 8, 0):
            r = b.solve(tol=1e-4, want_points=False, cluster_ctas=team)
            med[f"team={team}"] = {"ms": r[0]["device_ms"], "team": b.info()["batch_team"],
                                   "iters_max": max(x["iters"] for x in r)}
    out["medium64"] = med
    out["value"] = min(v["1e-04"]["ms"] for v in small.values())
    import oracle
    t0, k = time.perf_counter(), 0
    while k < 3 or time.perf_counter() - t0 < min(args.cpu_seconds, 5.0):
        ro = oracle.solve(lp, tol=1e-4)
        k += 1
    out["cpu_baseline"] = {"value": (time.perf_counter() - t0) / k * 1e3, "unit": "ms to 1e-4 (small planted LP)",
                           "cores": 1, "kind": "oracle",
                           "sample": f"oracle.solve of the small planted LP to 1e-4, {k} runs, {int(ro['iters'])} "
                                     "iterations each"}
    print(json.dumps(out))


def bench_warmstart(args):
    """Learned warm start on a transportation family (lpgen.transport_family(S, D), seed 0):
    solutions of args.ws_train instances (seeds 1..) from the batched solver train the
    3-layer width-1024 BF16 MLP on the device; held-out seeds 100001.. are solved cold and
    warm-started (KKT fallback) to 1e-4 and 1e-8."""
    import torch
    import lpgen
    from paper_2312_14832_b300 import warmstart as ws
    torch.cuda.set_device(0)
    fam = lpgen.transport_family(args.ws_supplies, args.ws_demands, seed=0)
    t0 = time.perf_counter()
    train = [lpgen.transport_instance(fam, s) for s in range(1, args.ws_train + 1)]
    held = [lpgen.transport_instance(fam, s) for s in range(100001, 100001 + args.ws_heldout)]
    gen_s = time.perf_counter() - t0
    P = np.array([lp["features"] for lp in train])
    t0 = time.perf_counter()
    fam_params = {"precision": 1} if args.ws_train_mixed else {}
    X, Y, W, its, st, dev = ws.solve_family(train, tol=args.ws_train_tol, chunk=args.ws_chunk, **fam_params)
    data_s = time.perf_counter() - t0
    print(f"training data: {len(train)} LPs in {data_s:.1f} s (device {dev:.1f} s)", file=sys.stderr, flush=True)
    model = ws.WarmStart(P.shape[1], train[0]["n"], train[0]["m"], hidden=1024, max_batch=256, seed=0)
    fit = model.fit(P, X, Y, W, epochs=args.ws_epochs, batch=256, lr=1e-3)
    del X, Y
    print(f"training: {fit['train_device_s']:.1f} s device", file=sys.stderr, flush=True)
    Ph = np.array([lp["features"] for lp in held])
    ev = ws.evaluate(model, held, Ph, tols=tuple(float(t) for t in args.ws_tols.split(",")))
    if args.ws_tols_hi:
        k = min(args.ws_heldout_hi, len(held))
        ev_hi = ws.evaluate(model, held[:k], Ph[:k], tols=tuple(float(t) for t in args.ws_tols_hi.split(",")))
        for key, val in ev_hi.items():
            if key.startswith("1e") or key[0].isdigit():
                ev[key] = dict(val, heldout=k)
    model.close()
    # the CPU oracle, cold, on held-out LPs to 1e-4
    import oracle
    t0, k, it = time.perf_counter(), 0, 0
    while k < len(held) and (k < 2 or time.perf_counter() - t0 < args.cpu_seconds):
        it += int(oracle.solve(held[k], tol=1e-4)["iters"])
        k += 1
    cpu_s = time.perf_counter() - t0
    n_in, hid, n_out = P.shape[1], 1024, train[0]["n"] + train[0]["m"] + 1
    flop_step = 2 * 256 * (n_in * hid + hid * hid + hid * n_out) * 3
    steps = args.ws_epochs * (len(train) // 256)
    out = {"metric": METRIC, "value": ev["1e-04"]["iters_ratio"], "unit": "cold/warm mean iterations to 1e-4",
           "higher_is_better": True, "n_gpus": 1, "data": "synthetic", "impl": "ours-warmstart", "dtype": "bf16 MLP / f64 LP",
           "config": {"workload": f"transportation family {args.ws_supplies} x {args.ws_demands} (n="
                                  f"{train[0]['n']}, m={train[0]['m']}), s,d ~ Gamma(2,50), costs = distance + "
                                  "N(0,0.05); MLP in -> 1024 -> 1024 -> n+m+1 (BF16, tcgen05)",
                      "train": len(train), "heldout": len(held), "epochs": args.ws_epochs,
                      "train_tol": args.ws_train_tol, "train_fp32": bool(args.ws_train_mixed)},
           "evaluation": ev, "train_loss_first_last": [float(fit["losses"][0]), float(fit["losses"][-1])],
           "train_device_s": fit["train_device_s"],
           "cpu_baseline": {"value": cpu_s / k, "unit": "s per held-out LP to 1e-4, cold", "cores": 1,
                            "kind": "oracle", "sample": f"oracle.solve on {k} held-out LPs ({it / k:.0f} "
                                                        "iterations on average)"},
           "train_tflops": flop_step * steps / max(fit["train_device_s"], 1e-9) / 1e12,
           "data_generation": {"solve_device_s": dev, "wall_s": data_s, "mean_iters": float(its.mean()),
                               "optimal": int(np.sum(st == 0)), "generate_s": gen_s}}
    print(json.dumps(out))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large",
                    choices=["large", "medium", "small", "batched", "mcf", "warmstart", "pagerank", "teams"])
    ap.add_argument("--ttt-budget", type=float, default=0.0,
                    help="seconds for a cold time-to-1e-4 solve of the bench workload (0 = skip)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--step-rule", type=int, default=0, choices=[0, 1],
                    help="timed solve: 0 constant step (Section 2), 1 adaptive rule (units: attempts)")
    ap.add_argument("--no-ttt", action="store_true", help="skip the small-LP time-to-tolerance section")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--spmv-stage", type=int, default=0, choices=[0, 1, 2, 3],
                    help="large: how the SpMVs read values and indices (0 = the setup autotuner's choice)")
    ap.add_argument("--cpu-seconds", type=float, default=10.0,
                    help="CPU work of the oracle baseline in the batched and mcf workloads")
    ap.add_argument("--count", type=int, default=4096, help="LPs in the batched workload")
    ap.add_argument("--batch-max-iter", type=int, default=200000)
    ap.add_argument("--batch-scaling", type=int, default=0)
    ap.add_argument("--batch-mixed", type=int, default=1, help="batched: also time the FP32 variant")
    ap.add_argument("--batch-tail", type=int, default=8192,
                    help="batched: also time the two-stage solve (LPs past this many iterations continue on teams)")
    ap.add_argument("--seq-sample", type=int, default=32)
    ap.add_argument("--mcf-budget", type=float, default=60.0, help="seconds per time-to-tolerance solve (mcf)")
    ap.add_argument("--mcf-switch-tol", type=float, default=0.0,
                    help="mcf: MIXED switches to FP64 at this largest relative error in the high-accuracy solve "
                         "(0 = the library default, max(tol, 1e-5))")
    ap.add_argument("--mcf-tol-hi", type=float, default=1e-8,
                    help="mcf: also solve to this tolerance (0 = skip), with the same time budget")
    ap.add_argument("--fixed-iters", type=int, default=0, help="teams: one launch of this many iterations")
    ap.add_argument("--team-one", type=int, default=1, help="teams: CTAs per LP for --fixed-iters")
    ap.add_argument("--pr-nodes", type=int, default=1_000_000)
    ap.add_argument("--pr-budget", type=float, default=60.0, help="seconds per time-to-1e-6 solve (pagerank)")
    ap.add_argument("--ws-train", type=int, default=50000)
    ap.add_argument("--ws-heldout", type=int, default=1000)
    ap.add_argument("--ws-epochs", type=int, default=30)
    ap.add_argument("--ws-train-tol", type=float, default=1e-6)
    ap.add_argument("--ws-train-mixed", type=int, default=0, help="training solves with FP32 iterations")
    ap.add_argument("--ws-chunk", type=int, default=4096, help="LPs per batched launch of the training solves")
    ap.add_argument("--ws-tols", default="1e-4,1e-8")
    ap.add_argument("--ws-tols-hi", default="", help="tolerances evaluated on the first --ws-heldout-hi LPs only")
    ap.add_argument("--ws-heldout-hi", type=int, default=300)
    ap.add_argument("--ws-supplies", type=int, default=40)
    ap.add_argument("--ws-demands", type=int, default=60)
    args = ap.parse_args()
    if args.workload == "batched":
        bench_batched(args)
        return
    if args.workload == "mcf":
        bench_mcf(args)
        return
    if args.workload == "warmstart":
        bench_warmstart(args)
        return
    if args.workload == "pagerank":
        bench_pagerank(args)
        return
    if args.workload == "teams":
        bench_teams(args)
        return

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        # the reference arm is the CPU oracle on every host core, on rank 0 only: one step
        # is one oracle PDHG iteration on the full workload (W untimed, then K timed)
        if rank != 0:
            return
        import oracle
        lp, desc = workload(args.workload, 0)
        cores, model = cpu_info()
        T = oracle.ThreadedStep(lp, cores)
        x = np.clip(np.zeros(lp["n"]), lp["l"], lp["u"])
        y = np.zeros(lp["m"])
        for _ in range(args.warmup):
            T.step(x, y, 1e-3, 1.0)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            T.step(x, y, 1e-3, 1.0)
        el = time.perf_counter() - t0
        rate = args.steps / el
        base = {"value": rate, "unit": "PDHG iter/s", "cores": cores, "kind": "oracle", "cpu_model": model,
                "sample": f"{args.steps} oracle PDHG steps (orc_pdhg_step_par on {cores} threads: K'y, primal "
                          f"step, K(2x+-x), dual step) on the full workload after {args.warmup} untimed, "
                          f"{el:.1f} s"}
        out = {"metric": METRIC, "value": rate, "unit": "PDHG iter/s", "n_gpus": 0,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "impl": "reference",
               "config": {"workload": desc, "check_every": CHECK_EVERY, "step": "1 oracle PDHG iteration",
                          "m": lp["m"], "n": lp["n"], "nnz": int(lp["val"].shape[0])},
               "cpu_baseline": base,
               "e2e": {"value": rate, "unit": "PDHG iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return

    import torch
    import paper_2312_14832_b300 as pk
    from paper_2312_14832_b300 import build as pkbuild
    pkbuild.build()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    lp, desc = workload(args.workload, rank)
    stream = torch.cuda.current_stream()
    s = pk.Solver.from_lp(lp, scaling=1, stream=stream.cuda_stream, spmv_stage=args.spmv_stage)
    info = s.info()
    iters = args.steps * CHECK_EVERY
    s.solve(tol=0.0, max_iter=max(args.warmup, 1) * CHECK_EVERY, want_point=False, step_rule=args.step_rule)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    clk = Clocks(local)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = s.solve(tol=0.0, max_iter=iters, want_point=False, step_rule=args.step_rule)
    e1.record(stream)
    barrier()
    clocks = clk.stop()
    ms, value = aggregate_ranks(e0.elapsed_time(e1), iters, world, dist)

    # dominant kernel, timed live with CUDA events on the solver's stream
    ms_p, ms_d = s.time_iterations(200)
    bp, bd = kernel_bytes(lp)
    pk_, peak_kind = peaks()
    if ms_p >= ms_d:
        kname, kb, kms = "primal (K'y SpMV + primal step)", bp, ms_p
        kkey = "sell_rows_kernel<OpSpmv,EpiPrimal>"
    else:
        kname, kb, kms = "dual (K x SpMV + dual step)", bd, ms_d
        kkey = "sell_rows_kernel<OpSpmv,EpiDual>"
    achieved = kb / (kms * 1e-3) / 1e9
    nnz = int(lp["val"].shape[0])
    ceil = gather_ceiling(nnz, lp["n"] if kms == ms_d else lp["m"])
    roofline = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": pk_["hbm_gbs"],
                "unit": "GB/s", "frac": achieved / pk_["hbm_gbs"], "peak_kind": peak_kind,
                "traffic": stored_traffic(kkey, args.workload),
                "bytes_per_launch": kb, "ms_per_launch": kms,
                "other_kernel_ms": ms_d if kms == ms_p else ms_p,
                "gather": {"gathers_per_launch": nnz, "achieved_per_s": nnz / (kms * 1e-3),
                           "ceiling_per_s": ceil.get("gathers_per_s"),
                           "frac": (nnz / (kms * 1e-3) / ceil["gathers_per_s"]) if "gathers_per_s" in ceil else None,
                           "ceiling_run": ceil},
                "fp64": fp64_roofline(nnz / (kms * 1e-3), "one DFMA per stored nonzero of the product "
                                                         "(the epilogue's FP64 work is not counted)")}
    iter_bytes = info["algorithmic_bytes_per_iter"]
    whole_iter_gbs = iter_bytes * (iters / (ms * 1e-3)) / 1e9

    # time to tolerance: on the small planted LP (GPU and CPU oracle, 1e-4 and 1e-8), and
    # optionally on the bench workload itself (cold start, with a time budget)
    ttt = {} if args.no_ttt else {"small_planted": time_to_tol_small(pk)}
    if args.ttt_budget > 0:
        for name, rule in (("workload_1e-4", 0), ("workload_1e-4_adaptive", 1)):
            rt = s.solve(tol=1e-4, time_limit_s=args.ttt_budget, want_point=False, step_rule=rule)
            ttt[name] = {
                "status": ["optimal", "iter_limit", "time_limit", "numerical"][rt["status"]],
                "iters": rt["iters"], "accepted": rt["accepted"], "restarts": rt["restarts"],
                "device_s": rt["device_ms"] * 1e-3, "wall_s": rt["solve_s"], "rel_primal": rt["rel_primal"],
                "rel_dual": rt["rel_dual"], "rel_gap": rt["rel_gap"], "primal_obj": rt["primal_obj"],
                "obj_star": lp.get("obj_star")}
    s.close()

    # end to end through the public API with host buffers: setup (H2D, layout), solve, D2H
    e2e = None
    if not args.no_e2e:
        barrier()
        t0 = time.perf_counter()
        s2 = pk.Solver.from_lp(lp, scaling=1, spmv_stage=args.spmv_stage)
        r2 = s2.solve(tol=0.0, max_iter=iters)
        _ = (r2["x"], r2["y"])
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        s2.close()
        if dist is not None:
            t = torch.tensor([el], device="cuda")
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            el = float(t.item())
        nnz = lp["val"].shape[0]
        h2d = 8 * (lp["m"] + 1) + 12 * nnz + 8 * (3 * lp["n"] + lp["m"])
        d2h = 8 * (lp["n"] + lp["m"])
        e2e = {"value": world * iters / el, "unit": "PDHG iter/s", "h2d_bytes_per_step": h2d / args.steps,
               "d2h_bytes_per_step": d2h / args.steps, "wall_s": el,
               "note": "setup (host CSR -> device layout, scaling, ||K|| estimate) + solve + result copy"}

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    base = None if args.no_cpu or world > 1 else cpu_baseline(lp)
    out = {"metric": METRIC, "value": value, "unit": "PDHG iter/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": desc, "check_every": CHECK_EVERY,
                      "step": f"{CHECK_EVERY} PDHG iterations + 1 restart/termination check",
                      "l2": "inputs larger than L2 (~0.7 GB touched per iteration)",
                      "parallelism": "replicas only" if world > 1 else "1 GPU",
                      "m": lp["m"], "n": lp["n"], "nnz": int(lp["val"].shape[0])},
           "roofline": roofline,
           "iteration_gbs": whole_iter_gbs, "iteration_frac": whole_iter_gbs / pk_["hbm_gbs"],
           "algorithmic_bytes_per_iter": iter_bytes, "stored_bytes_per_iter": info["stored_bytes_per_iter"],
           "time_to_tol": ttt, "cpu_baseline": base, "e2e": e2e, "gpu_launches": int(r["launches"]),
           "device_ms_library": r["device_ms"], "clocks": clocks,
           "layout": {k: info[k] for k in ("slots_K", "slots_Kt", "tasks_K", "tasks_Kt", "split_chunks_K",
                                           "split_chunks_Kt", "tile_slots_K", "spmv_batch_K", "spmv_stage_K",
                                           "spmv_stage_Kt")},
           "eta": info["eta"], "norm_K": info["norm_K"]}
    print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
