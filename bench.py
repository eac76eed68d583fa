#!/usr/bin/env python3
"""Throughput of the dual sweep (nnz*iters/s) on one GB300, with the
roofline of the sweep kernel, the end-to-end number through the C-ABI with
host buffers, and the FP64 CPU oracle timed beside it.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload precision]
    python bench.py --impl reference ...   # the oracle arm

One step = `--iters` iterations (sweep + accelerated update) of the hot path
on the workload's instance.  Inputs are generated on the host (seeded), then
made resident in HBM before the timed region; the instance (>= 6 GB) is far
larger than L2, so no flush is needed between iterations.
Under torchrun (N > 1) each rank solves its own replica (the single-GPU path
does not exchange data), and `value` is the sum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "nnz·iters/s (% HBM peak); time-to-1e-4 rel. dual gap, learned+BF16 vs plain"
UNIT = "nnz·iters/s"

WORKLOADS = {
    "precision": dict(
        desc="precision form: 80M users x 5,000 items, ~2.0B nnz; degree truncated lognormal (mean 25, max 500), "
             "item popularity ~ rank^-0.8; c = -LogNormal(0,0.5), a = U(0.5,1.5) stored BF16; int32 item idx, "
             "int64 row_ptr; b_j = 0.05 sum_i a_ij; gamma = 1e-3 fixed",
        users=80_000_000, items=5_000, seed=1002, bf16=True, schedule=(1e-3, 1e-3, 0.5, 1 << 30)),
    "production": dict(
        desc="production shape: 20M users x 2,000 items, ~500M nnz; same generators; c, a FP32; "
             "gamma continuation 1e-1 -> 1e-3 halved every 100 iterations",
        users=20_000_000, items=2_000, seed=1001, bf16=False, schedule=(1e-1, 1e-3, 0.5, 100)),
    "families": dict(
        desc="two capacity families (Def. 1): the production shape, 20M users x 2,000 items, ~500M nnz, with a "
             "second coefficient per edge a2 = U(0.1, 2) and b2_j = 0.05 sum_i a2_ij; c, a, a2 stored BF16; "
             "gamma = 1e-3 fixed; the general multi-family sweep",
        users=20_000_000, items=2_000, seed=1001, bf16=True, schedule=(1e-3, 1e-3, 0.5, 1 << 30), families=2),
    "boxcut": dict(
        desc="box cut by a per-user budget ({0 <= x_ij <= 0.5, sum_j x_ij <= 1}): the production shape, 20M users "
             "x 2,000 items, ~500M nnz; c, a stored BF16; gamma = 1e-3 fixed; the box-cut sweep",
        users=20_000_000, items=2_000, seed=1001, bf16=True, schedule=(1e-3, 1e-3, 0.5, 1 << 30),
        kind=3, z=0.5, cut=1.0),
    "appendix": dict(
        desc="the paper's appendix generator (App. A) at the preconditioning experiment's size: 25M requests x "
             "10,000 resources, 0.1% density (nu = 10, ~250M nnz); breadth LogNormal(0,1), K_j ~ Poisson(p_j I nu) "
             "distinct requests; value v_j u_i eps_ij (LogNormal 0.5, 0.5, 0.25) capped at 5, c = -value; "
             "a = s_j value with s_j ~ LogNormal(0,1.5); b_j = rho_j (greedy load + 1e-3), rho_j ~ U[0.5,1]; "
             "c, a FP32; gamma = 1e-2 fixed; row normalization (per-item steps)",
        users=25_000_000, items=10_000, seed=1006, bf16=False, schedule=(1e-2, 1e-2, 0.5, 1 << 30),
        precondition=True, appendix=True, autotune=True),
    "batched": dict(
        desc="batched form: 64 independent instances of the production generators, users log-uniform 1e4-5e6, "
             "items log-uniform 50-2,000, gamma drawn from {1e-1, 1e-2, 1e-3} (fixed per instance); c, a stored "
             "BF16; one sweep launch + one update launch per iteration for all 64, replayed as CUDA graphs; "
             "mapping chosen by the library's tuner",
        n=64, seed=1003, bf16=True),
    "tiny": dict(
        desc="tiny: 10,000 users x 100 items, ~100k nnz, 1+Poisson(9) degree, uniform items, c=-U(0,1), a=1, "
             "b_j = 0.05 deg_j, gamma = 1e-2",
        users=10_000, items=100, seed=1000, bf16=False, schedule=(1e-2, 1e-2, 0.5, 1 << 30)),
}


def config_for(args, world):
    """The `config` object of the JSON line, from the arguments alone, so the
    oracle arm prints the same one as the GPU arm."""
    w = WORKLOADS[args.workload]
    desc = w["desc"] if args.scale == 1.0 else w["desc"] + f" (users scaled x{args.scale})"
    cfg = {"workload": desc, "iters_per_step": args.iters,
           "parallelism": "single GPU" if world == 1 else
           ("replicas" if args.workload == "batched" else
            f"user-sharded over {world} GPUs (each rank {w.get('users', 0):,} users; int64 item sums all-reduced "
            f"every iteration)")}
    if args.workload == "batched":
        cfg.update(instances=w["n"], storage="bf16")
    else:
        cfg.update(users=max(1000, int(round(w["users"] * args.scale))) if args.workload != "tiny" else w["users"],
                   items=w["items"], storage="bf16" if w["bf16"] else "f32")
    cfg["l2"] = ("inputs fit in L2 (tiny case)" if args.workload == "tiny" else
                 "inputs of several GB per iteration >> 129 MB L2 (no flush)")
    return cfg


def recipe_for(name, scale):
    import synth

    w = WORKLOADS[name]
    I = max(1000, int(round(w["users"] * scale)))
    if name == "tiny":
        return synth.recipe_tiny(w["seed"])
    if name in ("production", "families", "boxcut"):
        return synth.recipe_production(I=I, J=w["items"], seed=w["seed"])
    if name == "appendix":
        return synth.recipe_appendix(I=I, J=w["items"], seed=w["seed"])
    return synth.recipe_precision(I=I, J=w["items"], seed=w["seed"])


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


SWEEP_SOURCES = ("sweep.cu", "sweep_multi.cu", "sweep_common.cuh", "dlm_impl.cuh")


def sweep_source_hash(files=SWEEP_SOURCES):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, "paper_2606_07777_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, nnz, users):
    """DRAM bytes per sweep launch from the committed ncu summary, scaled to
    this instance, or None if the kernel changed since it was captured."""
    p = os.path.join(ROOT, "profiles", "sweep_traffic.json")
    if not os.path.exists(p):
        return None
    try:
        with open(p) as f:
            d = json.load(f)
        rec = d.get(workload)
        if not rec or rec.get("source_hash") != sweep_source_hash(tuple(rec.get("files", SWEEP_SOURCES))):
            return None
        return rec["bytes_per_nnz"] * nnz + rec.get("bytes_per_user", 0.0) * users
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_id):
        self.dev_id = dev_id
        self.proc = None

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
            if self.dev_id is not None:
                cmd += ["-i", str(self.dev_id)]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


def gpu_id_for_smi(torch, dev):
    try:
        u = str(torch.cuda.get_device_properties(dev).uuid)
        if u:
            return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        pass
    vis = os.environ.get("CUDA_VISIBLE_DEVICES")
    if vis:
        return vis.split(",")[dev.index or 0]
    return dev.index or 0


def make_instance(recipe, bf16, torch, pinned, threads):
    import numpy as np
    import synth

    def pin_alloc(n, dtype):
        t = torch.empty(int(n), dtype={np.int64: torch.int64, np.int32: torch.int32, np.float32: torch.float32,
                                       np.uint16: torch.int16}[np.dtype(dtype).type], pin_memory=pinned)
        return t.numpy().view(dtype)

    if isinstance(recipe, synth.AppRecipe):
        return synth.generate_appendix(recipe, nthreads=threads, alloc=pin_alloc)
    if bf16:
        inst = synth.generate(recipe, nthreads=threads, alloc=lambda n, dt: pin_alloc(n, dt) if dt != np.float32
                              else np.empty(int(n), dt))
        c16 = pin_alloc(inst.nnz, np.uint16)
        a16 = pin_alloc(inst.nnz, np.uint16)
        synth.round_bf16(inst.c, threads, c16)
        synth.round_bf16(inst.a, threads, a16)
        inst.c32, inst.a32 = inst.c, inst.a  # FP32 values, kept for the error statement
        inst.c, inst.a = c16, a16
    else:
        inst = synth.generate(recipe, nthreads=threads, alloc=pin_alloc)
    return inst


def add_second_family(inst, torch, threads):
    """A second capacity family: a2 = U(0.1, 2) per edge (seeded), b2_j = 0.05
    sum_i a2_ij; inst.a becomes the [nnz, 2] edge-major BF16 pair array and
    inst.b the [2, J] capacities."""
    import numpy as np
    import synth

    a2 = (0.1 + 1.9 * synth.uniforms(1005, 0, 7, inst.nnz)).astype(np.float32)
    b2 = 0.05 * np.bincount(inst.col, weights=synth.bf16_to_f32(synth.round_bf16(a2, threads)).astype(np.float64),
                            minlength=inst.J)
    pair = torch.empty((inst.nnz, 2), dtype=torch.int16, pin_memory=True).numpy().view(np.uint16)
    pair[:, 0] = inst.a
    pair[:, 1] = synth.round_bf16(a2, threads)
    inst.a = pair
    inst.b = np.ascontiguousarray(np.stack([inst.b, b2]))
    inst.c32 = inst.a32 = None


def solve_from_zero(s, torch, target, max_iters, sched=(1e-1, 1e-3, 0.5, 50), gap_every=50, restart=True):
    """Drives a handle from lam = 0 to a certified gap under a continuation
    schedule with row normalization; returns (Stats, seconds)."""
    s.set_schedule(*sched)
    s.set_options(precondition=True, restart=restart, gap_every=gap_every)
    s.set_lambda(torch.zeros(s.dual_dim, dtype=torch.float32, device=s.device))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    st = s.solve(target, max_iters)
    torch.cuda.synchronize()
    return st, time.perf_counter() - t0


def bf16_error_statement(dlm, torch, inst, recipe, threads, gamma=1e-3, target=1e-5, max_iters=4000,
                         sample_frac=2e-3, sample_iters=3000):
    """Error of the BF16-storage form, optimum to optimum.

    Full instance: the BF16 form, the FP32 form and the FP32 form with only c
    rounded to BF16 are each driven from lam = 0 to a certified gap (the
    1e-1 -> gamma continuation, row normalization, adaptive restart).  Rounding
    c alone moves the optimum by at most ||dc||_2 / gamma (the primal optimum
    is the projection of -c / gamma onto a fixed convex set: nonexpansive);
    each solve's own distance to its optimum is at most sqrt(2 gap |g| / gamma)
    on the certified point.  Rounding a changes the feasible set, for which
    only the measured difference is stated.
    Sample: a seeded user sample of the same recipe (capacities from the
    sample) solved by the BF16 form on the GPU and by the FP64 oracle on the
    FP32 values (all host threads), both to the same gap."""
    import numpy as np
    import oracle
    import synth

    dev = torch.device("cuda", torch.cuda.current_device())
    sched = (1e-1, gamma, 0.5, 50)
    c32 = torch.from_numpy(inst.c32).to(dev)
    a32 = torch.from_numpy(inst.a32).to(dev)
    c16 = torch.from_numpy(inst.c.view(np.int16)).to(dev).view(torch.bfloat16)
    a16 = torch.from_numpy(inst.a.view(np.int16)).to(dev).view(torch.bfloat16)
    rp, col, b = (torch.from_numpy(v).to(dev) for v in (inst.row_ptr, inst.col, inst.b))
    forms = {"bf16": (c16, a16, True), "fp32": (c32, a32, False), "fp32_c_rounded": (c16.float(), a32, False)}
    sol = {}
    for name, (c, a, bf) in forms.items():
        h = dlm.Solver(rp, col, c, a, b, inst.J, bf16=bf)
        st, sec = solve_from_zero(h, torch, target, max_iters, sched)
        sol[name] = dict(lam=h.lam().double(), x=h.x(), g=st.dual_obj, gap=st.rel_gap, iters=int(st.iter),
                         seconds=sec, converged=bool(st.converged))
        h.close()
    dc = float(torch.linalg.vector_norm((c16.float() - c32).double()).item())
    tol = {k: math.sqrt(2.0 * max(v["gap"], 0.0) * abs(v["g"]) / gamma) for k, v in sol.items()}

    def diff(u, v):
        dx = (sol[u]["x"] - sol[v]["x"]).double()
        dl = (sol[u]["lam"] - sol[v]["lam"]).abs().max().item()
        return {"x_l2": float(torch.linalg.vector_norm(dx).item()), "x_max_abs": float(dx.abs().max().item()),
                "lam_max_abs_rel": dl / max(float(sol[v]["lam"].abs().max().item()), 1e-30),
                "dual_obj_rel": abs(sol[u]["g"] - sol[v]["g"]) / abs(sol[v]["g"])}

    full = {"gamma": gamma, "target_rel_gap": target,
            "solves": {k: {q: v[q] for q in ("g", "gap", "iters", "seconds", "converged")} for k, v in sol.items()},
            "c_rounding_only": dict(diff("fp32_c_rounded", "fp32"), bound_l2=dc / gamma,
                                    solver_tolerance_l2=tol["fp32_c_rounded"] + tol["fp32"]),
            "bf16_vs_fp32": diff("bf16", "fp32")}
    c_only = full["c_rounding_only"]
    c_only["within_bound"] = c_only["x_l2"] <= c_only["bound_l2"] + c_only["solver_tolerance_l2"]
    del sol, c32, a32, c16, a16, rp, col, b
    torch.cuda.empty_cache()
    # sample: GPU BF16 form against the FP64 oracle on the FP32 values
    ids = synth.sample_users(recipe.I, sample_frac, 4545)
    sub = synth.generate(recipe, ids=ids, nthreads=threads)
    cr, ar = synth.round_bf16(sub.c), synth.round_bf16(sub.a)
    arrs = [torch.from_numpy(v).to(dev) for v in (sub.row_ptr, sub.col)]
    h = dlm.Solver(arrs[0], arrs[1], torch.from_numpy(cr.view(np.int16)).to(dev).view(torch.bfloat16),
                   torch.from_numpy(ar.view(np.int16)).to(dev).view(torch.bfloat16),
                   torch.from_numpy(sub.b).to(dev), sub.J, bf16=True)
    st, sec = solve_from_zero(h, torch, target, sample_iters, sched)
    lam_g = h.lam().cpu().numpy().astype(np.float64)
    x_g = h.x().cpu().numpy().astype(np.float64)
    h.close()
    p = oracle.Problem(sub.row_ptr, sub.col, sub.c.astype(np.float64), sub.a.astype(np.float64), sub.b, sub.J)
    nc = host_cores()
    t0 = time.perf_counter()
    ref = oracle.solve_threads(p, *sched, precondition=True, restart=True, target=target, gap_every=50,
                               max_iters=sample_iters, nthreads=nc)
    t_ref = time.perf_counter() - t0
    x_r = oracle.sweep(p, ref["lam"], gamma)["x"]
    sample = {"users": int(len(ids)), "nnz": int(p.nnz), "gpu_bf16": {"g": st.dual_obj, "gap": st.rel_gap,
                                                                        "iters": int(st.iter),
                                                                        "converged": bool(st.converged)},
              "oracle_fp64": {"g": ref["g"], "gap": ref["rel_gap"], "iters": ref["iters"], "seconds": t_ref,
                              "cores": nc},
              "x_l2": float(np.linalg.norm(x_g - x_r)), "x_max_abs": float(np.abs(x_g - x_r).max()),
              "lam_max_abs_rel": float(np.abs(lam_g - ref["lam"]).max() / max(np.abs(ref["lam"]).max(), 1e-30)),
              "dual_obj_rel": abs(st.dual_obj - ref["g"]) / abs(ref["g"]),
              "bound_c_rounding_l2": float(np.linalg.norm(synth.bf16_to_f32(cr).astype(np.float64) -
                                                          sub.c.astype(np.float64))) / gamma}
    return {"full_instance": full, "vs_fp64_oracle_sample": sample,
            "how": "optimum to optimum: every form solved from lam = 0 to the same certified gap"}


def production_summary(args, dlm, torch, dev, threads):
    """The production shape (20M users x 2,000 items, FP32 values, gamma
    continuation 1e-1 -> 1e-3 halved every 100 iterations): sweep throughput
    over the whole continuation (700 iterations, every sweep timed by CUDA
    events) and the time to a 1e-4 certified gap from lam = 0 (row
    normalization: the items' row norms are about 250x apart)."""
    w = WORKLOADS["production"]
    t0 = time.perf_counter()
    inst = make_instance(recipe_for("production", args.scale), False, torch, False, threads)
    t_gen = time.perf_counter() - t0
    arrs = [torch.from_numpy(v).to(dev) for v in (inst.row_ptr, inst.col, inst.c, inst.a, inst.b)]
    s = dlm.Solver(*arrs, inst.J)
    del arrs
    info = s.info()
    s.set_schedule(*w["schedule"])
    s.step(20)
    s.set_schedule(*w["schedule"])
    torch.cuda.synchronize()
    T = 700
    sw, up, tot = s.step_timed(T)
    peak, _ = load_peaks()
    st, sec = solve_from_zero(s, torch, 1e-4, 20000, sched=w["schedule"], gap_every=25)
    s.close()
    return {"workload": w["desc"], "nnz": info["nnz"], "generate_s": t_gen,
            "throughput": {"value": info["nnz"] * T / (tot / 1000.0), "unit": UNIT, "iters": T,
                           "sweep_us": sw * 1000.0 / T, "update_us": up * 1000.0 / T,
                           "frac": info["bytes_per_iter"] / (sw / 1000.0 / T) / 1e9 / peak},
            "time_to_gap": {"target_rel_gap": 1e-4, "seconds": sec, "iters": int(st.iter), "rel_gap": st.rel_gap,
                            "converged": bool(st.converged), "options": "row normalization, adaptive restart, "
                                                                        "gap check every 25 iterations"}}


def batched_summary(args, dlm, torch, dev, threads, iters=100, steps=2):
    """The batched workload (64 instances, BF16) in brief: the tuner's mapping,
    then `steps` x `iters` iterations with every kernel timed."""
    import numpy as np
    import synth

    w = WORKLOADS["batched"]
    t0 = time.perf_counter()
    recipes = synth.recipe_batch(n=w["n"], seed=w["seed"])
    solvers = []
    for r, g in recipes:
        if args.scale != 1.0:
            r.I = max(1000, int(round(r.I * args.scale)))
        inst = make_instance(r, True, torch, False, threads)
        arrs = [torch.from_numpy(v).to(dev) for v in (inst.row_ptr, inst.col, inst.c.view(np.int16),
                                                      inst.a.view(np.int16), inst.b)]
        s = dlm.Solver(arrs[0], arrs[1], arrs[2].view(torch.bfloat16), arrs[3].view(torch.bfloat16), arrs[4],
                       inst.J, bf16=True)
        s.set_schedule(g)
        solvers.append(s)
        del arrs, inst
    t_setup = time.perf_counter() - t0
    bt = dlm.Batch(solvers)
    chosen, _ = bt.autotune(3)
    bt.step(iters)
    sw = up = tot = 0.0
    for _ in range(steps):
        a_, b_, c_ = bt.step_timed(iters)
        sw, up, tot = sw + a_, up + b_, tot + c_
    infos = [s.info() for s in solvers]
    nnz = sum(i["nnz"] for i in infos)
    bytes_iter = sum(i["bytes_per_iter"] for i in infos)
    status = sorted({x.status for x in bt.stats()})
    bt.close()
    for s in solvers:
        s.close()
    peak, _ = load_peaks()
    T = iters * steps
    return {"workload": w["desc"], "instances": len(solvers), "nnz": nnz, "generate_and_create_s": t_setup,
            "mapping": {k: getattr(chosen, k) for k in ("mapping", "coop_max", "block_threads", "topk")},
            "value": nnz * T / (tot / 1000.0), "unit": UNIT, "sweep_us": sw * 1000.0 / T, "update_us": up * 1000.0 / T,
            "frac": bytes_iter / (sw / 1000.0 / T) / 1e9 / peak, "member_status": status}


def cpu_sample(workload, bf16, frac, seed=4242, threads=0, inst=None):
    """A seeded user sample of the workload, regenerated row by row (the
    appendix instance is drawn resource by resource, so its sample is cut
    from ``inst``), as an FP64 oracle problem (BF16 values widened exactly)."""
    import numpy as np
    import oracle
    import synth

    r = recipe_for(workload, 1.0) if workload != "batched" else None
    if workload == "batched":
        return batch_sample(frac, seed, threads)
    if workload == "appendix":
        if inst is None:
            inst = synth.generate_appendix(r, nthreads=threads)
        inst = synth.subset(inst, synth.sample_users(inst.I, frac, seed))
    elif workload == "tiny":
        inst = synth.generate(r)
    else:
        ids = synth.sample_users(r.I, frac, seed)
        inst = synth.generate(r, ids=ids, nthreads=threads)
    c, a = inst.c, inst.a
    if bf16:
        c = synth.bf16_to_f32(synth.round_bf16(c))
        a = synth.bf16_to_f32(synth.round_bf16(a))
    w = WORKLOADS[workload]
    return oracle.Problem(inst.row_ptr, inst.col, c.astype(np.float64), a.astype(np.float64), inst.b, inst.J,
                          w.get("kind", oracle.SIMPLEX_LE), w.get("z", 1.0),
                          cut=w["cut"] if w.get("cut") is not None else np.inf)


def batch_sample(frac, seed=4242, threads=0):
    """A seeded user sample of every member of the batched workload, as a
    list of (FP64 oracle problem, gamma)."""
    import numpy as np
    import oracle
    import synth

    w = WORKLOADS["batched"]
    out = []
    for k, (r, gamma) in enumerate(synth.recipe_batch(n=w["n"], seed=w["seed"])):
        ids = synth.sample_users(r.I, frac, seed + k)
        if len(ids) == 0:
            continue
        inst = synth.generate(r, ids=ids, nthreads=threads)
        c = synth.bf16_to_f32(synth.round_bf16(inst.c))
        a = synth.bf16_to_f32(synth.round_bf16(inst.a))
        out.append((oracle.Problem(inst.row_ptr, inst.col, c.astype(np.float64), a.astype(np.float64), inst.b,
                                   inst.J), gamma))
    return out


def time_oracle_batch(ps, budget_s, nthreads=1):
    """Oracle iterations over every sampled member, about budget_s seconds in
    total; returns (nnz*iters/s, iters per member, seconds, nnz)."""
    import oracle

    def run(T):
        for p, g in ps:
            if nthreads > 1:
                oracle.fista_threads(p, T, g, nthreads=nthreads)
            else:
                oracle.fista(p, T, g, trajectory=False)

    t0 = time.perf_counter()
    run(1)
    t1 = time.perf_counter() - t0
    iters = max(1, int(budget_s / max(t1, 1e-6)))
    t0 = time.perf_counter()
    run(iters)
    dt = time.perf_counter() - t0
    nnz = sum(p.nnz for p, _ in ps)
    return nnz * iters / dt, iters, dt, nnz


def time_oracle(p, gamma, budget_s, nthreads=1):
    """Oracle iterations on problem p for about budget_s seconds; returns
    (nnz*iters/s, iters, seconds).  nthreads > 1 times the threaded loop
    (the same iteration with the sweep split over host threads)."""
    import oracle

    def run(T):
        if nthreads > 1:
            oracle.fista_threads(p, T, gamma, nthreads=nthreads)
        else:
            oracle.fista(p, T, gamma, trajectory=False)

    t0 = time.perf_counter()
    run(1)
    t1 = time.perf_counter() - t0
    iters = max(1, int(budget_s / max(t1, 1e-6)))
    t0 = time.perf_counter()
    run(iters)
    dt = time.perf_counter() - t0
    return p.nnz * iters / dt, iters, dt


def replica_throughput(units, seconds, dist=None, device=None):
    """Whole-job throughput of independent replicas: the units all ranks
    processed divided by the slowest rank's time (max over ranks).  Returns
    (units per second, max seconds).  Without a process group: this rank's."""
    if dist is None:
        return units / seconds, seconds
    import torch

    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(u.item()) / float(t.item()), float(t.item())


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args, rank, world):
    w = WORKLOADS[args.workload]
    if rank != 0:
        return 0
    frac = args.cpu_frac
    per_step = []
    nc = host_cores()
    if args.workload == "batched":
        ps = batch_sample(frac)
        for k in range(args.warmup + args.steps):
            v, iters, dt, nnz_s = time_oracle_batch(ps, args.ref_step_seconds, nthreads=nc)
            if k >= args.warmup:
                per_step.append((v, iters * nnz_s, dt))
        users = sum(p.I for p, _ in ps)
        desc_n = f"{users} users, {nnz_s} nnz over {len(ps)} members"
    else:
        p = cpu_sample(args.workload, w["bf16"], frac)
        gamma = w["schedule"][1]
        for k in range(args.warmup + args.steps):
            v, iters, dt = time_oracle(p, gamma, args.ref_step_seconds, nthreads=nc)
            if k >= args.warmup:
                per_step.append((v, iters * p.nnz, dt))
        desc_n = f"{p.I} users, {p.nnz} nnz"
    total_nnz_iters = sum(ni for _, ni, _ in per_step)
    total_s = sum(dt for _, _, dt in per_step)
    value = total_nnz_iters / total_s
    sample = (f"{'all' if args.workload == 'tiny' else f'{frac:.2%} seeded user sample'} of the {args.workload} "
              f"workload ({desc_n}), FP64 oracle iterations (sweep split over {nc} threads + accelerated "
              f"update), {per_step[0][1]} nnz-iterations per step")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1000 * total_s / len(per_step), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": config_for(args, world),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": nc, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", choices=list(WORKLOADS), default="precision")
    ap.add_argument("--iters", type=int, default=100, help="iterations per step")
    ap.add_argument("--scale", type=float, default=1.0, help="fraction of the workload's users (smoke runs)")
    ap.add_argument("--threads", type=int, default=0, help="host threads for instance generation")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--cpu-frac", type=float, default=0.01)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--ref-step-seconds", type=float, default=6.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-error-statement", action="store_true")
    ap.add_argument("--autotune", action="store_true", help="let the library's tuner pick the sweep mapping")
    ap.add_argument("--no-time-to-gap", action="store_true", help="skip the recurring-instance time-to-gap run")
    ap.add_argument("--ttg-users", type=int, default=5_000_000)
    ap.add_argument("--ttg-items", type=int, default=1_000)
    ap.add_argument("--ttg-gamma", type=float, default=1e-3)
    ap.add_argument("--ttg-only", action="store_true", help="print only the time-to-gap object (development)")
    ap.add_argument("--no-companions", action="store_true",
                    help="skip the production and batched summaries of the default line")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return run_reference(args, rank, world)

    import numpy as np
    import torch

    import paper_2606_07777_gb300 as dlm

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(v):
        if dist is None:
            return v
        t = torch.tensor([v], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    if args.workload == "batched":
        return run_batched(args, dlm, torch, dev, rank, world, barrier, max_over_ranks, dist)
    if world > 1 and args.workload not in ("tiny", "families", "appendix"):
        return run_sharded(args, dlm, torch, dev, rank, world, barrier, dist)
    if args.ttg_only:
        print(json.dumps(time_to_gap(args, dlm, torch, dev)), flush=True)
        return 0

    w = WORKLOADS[args.workload]
    bf16 = w["bf16"]
    recipe = recipe_for(args.workload, args.scale)
    t_gen = time.perf_counter()
    inst = make_instance(recipe, bf16, torch, True, args.threads)
    if w.get("families", 1) > 1:
        add_second_family(inst, torch, args.threads)
    t_gen = time.perf_counter() - t_gen

    # Device-resident inputs.
    def dev_arrays():
        rp = torch.from_numpy(inst.row_ptr).to(dev, non_blocking=True)
        col = torch.from_numpy(inst.col).to(dev, non_blocking=True)
        if bf16:
            c = torch.from_numpy(inst.c.view(np.int16)).to(dev, non_blocking=True).view(torch.bfloat16)
            a = torch.from_numpy(inst.a.view(np.int16)).to(dev, non_blocking=True).view(torch.bfloat16)
        else:
            c = torch.from_numpy(inst.c).to(dev, non_blocking=True)
            a = torch.from_numpy(inst.a).to(dev, non_blocking=True)
        b = torch.from_numpy(inst.b).to(dev, non_blocking=True)
        torch.cuda.synchronize(dev)
        return rp, col, c, a, b

    dlm.load()
    t_setup = time.perf_counter()
    arrs = dev_arrays()
    kind_args = dict(kind=w.get("kind", 0), z=w.get("z", 1.0), cut=w.get("cut"))
    s = dlm.Solver(*arrs, inst.J, bf16=bf16, **kind_args)
    del arrs
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t_setup
    s.set_schedule(*w["schedule"])
    precond = bool(w.get("precondition", False))
    s.set_options(precondition=precond)
    info = s.info()
    nnz, I, J, bytes_iter = info["nnz"], info["num_users"], info["num_items"], info["bytes_per_iter"]

    for _ in range(args.warmup):
        s.step(args.iters)
    torch.cuda.synchronize(dev)
    tuned = None
    if args.autotune or w.get("autotune"):
        # the library's tuner picks the sweep mapping from the warmed-up state
        # (which it restores); its choice depends on that state, so the default
        # keeps the library's default mapping
        opts, tune_ms = s.autotune(3)
        tuned = {k: opts.as_dict()[k] for k in ("mapping", "coop_max", "block_threads", "topk", "short_rows")}
        tuned["sweep_ms"] = tune_ms

    # ---- timed region: K steps, every kernel bracketed by CUDA events ----
    sampler = ClockSampler(gpu_id_for_smi(torch, dev))
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    sweep_ms = upd_ms = tot_ms = 0.0
    for _ in range(args.steps):
        a_, b_, c_ = s.step_timed(args.iters)
        sweep_ms += a_
        upd_ms += b_
        tot_ms += c_
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    iters_total = args.iters * args.steps
    value, elapsed_s = replica_throughput(nnz * iters_total, tot_ms / 1000.0, dist, dev)

    # Same steps replayed through the captured CUDA graphs (the default path).
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        s.step(args.iters)
    e1.record(st)
    torch.cuda.synchronize(dev)
    graph_ms_per_step = e0.elapsed_time(e1) / args.steps

    # ---- end to end through the C-ABI: host (pinned) inputs -> create ->
    # iterations -> lam back to the host, every step ----
    dual_dim = w.get("families", 1) * J
    lam_host = torch.empty(dual_dim, dtype=torch.float32, pin_memory=True)
    h2d = inst.row_ptr.nbytes + inst.col.nbytes + inst.c.nbytes + inst.a.nbytes + inst.b.nbytes
    # measured before the companion measurements below, whose device arrays
    # and pageable host copies would otherwise share the box with it
    torch.cuda.synchronize(dev)
    torch.cuda.empty_cache()
    e2e_times = []
    create_phases = None
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s2 = dlm.Solver(inst.row_ptr, inst.col, inst.c, inst.a, inst.b, inst.J, bf16=bf16, **kind_args)
        create_phases = s2.setup_seconds()
        s2.set_schedule(*w["schedule"])
        if precond:
            s2.set_options(precondition=True)
        s2.step(args.iters)
        dlm.dlm_get_lambda(s2.h, lam_host, dlm.DLM_MEM_HOST)
        s2.close()
        dt = time.perf_counter() - t0
        if k > 0:  # first call warms the allocator
            e2e_times.append(dt)
    e2e_value = None
    if e2e_times:
        e2e_value, _ = replica_throughput(nnz * args.iters, statistics.mean(e2e_times), dist, dev)

    conv = None
    if w.get("appendix") and not args.no_time_to_gap:
        conv = precondition_convergence(s, dlm, w["schedule"][1])

    bf16_err = None
    if bf16 and not args.no_error_statement and w.get("families", 1) == 1 and args.workload == "precision":
        bf16_err = bf16_error_statement(dlm, torch, inst, recipe, args.threads, gamma=w["schedule"][1])

    # ---- roofline of the dominant kernel (the sweep) ----
    # the tuner may pick the short-row sweep (one launch, another kernel, its own traffic record)
    short_on = bool(tuned is not None and tuned.get("short_rows"))
    traffic = (recorded_traffic(args.workload + ("_short" if short_on else ""), nnz, I) if args.scale == 1.0
               else None)
    peak, peak_kind = load_peaks()
    sweep_s = sweep_ms / 1000.0 / iters_total
    achieved = bytes_iter / sweep_s / 1e9
    # bytes the library's layout streams: 16-bit item indices, the values, a
    # 12-byte header per 32 users
    vsz = 2 if bf16 else 4
    fam = w.get("families", 1)
    layout_bytes = nnz * (2 + (1 + fam) * vsz) + (I + 31) // 32 * 12
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "peak_source": f"{peak_kind} (copy bandwidth, MEASURED_PEAKS.json)"
            if peak_kind == "measured" else "fallback 6.8 TB/s",
            "kernel": ("sweep_multi_kernel" if w.get("families", 1) > 1 else
                       "sweep_boxcut_kernel" if w.get("kind") == 3 else
                       "sweep_short_kernel" if short_on else
                       "sweep_dyn_kernel" if tuned is not None and tuned["mapping"] == 3 else "sweep_kernel"),
            "algorithmic_bytes_per_launch": bytes_iter,
            "layout_bytes_per_launch": layout_bytes,
            "layout_frac": layout_bytes / sweep_s / 1e9 / peak,
            "sweep_share_of_iteration": sweep_ms / tot_ms if tot_ms > 0 else None,
            "sweep_us": sweep_s * 1e6, "update_us": upd_ms * 1000.0 / iters_total}

    cpu = None
    if rank == 0 and not args.no_cpu_baseline and w.get("families", 1) == 1:
        p = cpu_sample(args.workload, bf16, args.cpu_frac, threads=args.threads, inst=inst)
        nc = host_cores()
        v1, it1, dt1 = time_oracle(p, w["schedule"][1], args.cpu_seconds * 0.4)
        vn, itn, dtn = time_oracle(p, w["schedule"][1], args.cpu_seconds * 0.6, nthreads=nc)
        cpu = {"value": vn, "unit": UNIT, "cores": nc, "kind": "oracle", "single_core_value": v1,
               "sample": (f"{'all' if args.workload == 'tiny' else f'{args.cpu_frac:.0%} seeded user sample'} of "
                          f"the workload ({p.I} users, {p.nnz} nnz): {itn} FP64 oracle iterations on {nc} threads "
                          f"in {dtn:.1f} s (sweep split over threads); single-threaded {it1} iterations in "
                          f"{dt1:.1f} s")}

    ttg = None
    if rank == 0 and not args.no_time_to_gap and args.workload == "precision":
        ttg = time_to_gap(args, dlm, torch, dev)
    production = batched = None
    if rank == 0 and not args.no_companions and args.workload == "precision":
        production = production_summary(args, dlm, torch, dev, args.threads)
        batched = batched_summary(args, dlm, torch, dev, args.threads)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_s * 1000.0 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_for(args, world),
        "instance": {"users": I, "items": J, "nnz": nnz, "bytes_per_iter": bytes_iter,
                     "sweep_mapping": tuned if tuned is not None else "default"},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(dual_dim * 4),
                "note": "per step: dlm_create from pinned host arrays (copy + layout), iterations, lam to host",
                "create_seconds_by_phase": create_phases},
        "gpu_launches": 2 * iters_total,
        "clocks": clocks,
        "graph_ms_per_step": graph_ms_per_step,
        "bf16_error": bf16_err,
        "time_to_gap": ttg,
        "production": production,
        "batched": batched,
        "precondition_convergence": conv,
        "setup_s": {"generate": t_gen, "upload_and_create": t_setup},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def precondition_convergence(s, dlm, gamma, target=1e-4, max_iters=6000, gap_every=25):
    """The row-normalization comparison of the preconditioning experiment on
    this instance: from lam = 0, the solve with per-item steps to the target
    certified gap, then the plain step 1/L for the same number of
    iterations."""
    import torch

    out = {"target_rel_gap": target, "gamma": gamma, "gap_every": gap_every}
    for name, pre in (("row_normalized", True), ("plain", False)):
        lam0 = torch.zeros(s.dual_dim, dtype=torch.float32, device="cuda")
        s.set_schedule(gamma)
        s.set_options(precondition=pre, gap_every=gap_every, restart=True)
        s.set_lambda(lam0)
        limit = max_iters if pre else max(out["row_normalized"]["iters"], gap_every)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st = s.solve(target, limit)
        torch.cuda.synchronize()
        out[name] = {"iters": int(st.iter), "seconds": time.perf_counter() - t0, "rel_gap": st.rel_gap,
                     "max_viol": st.max_viol, "reached": bool(st.rel_gap <= target)}
    s.set_options(precondition=True)
    return out


# Continuations a warm start may enter (gamma_0, factor, iterations per
# stage); the cold start always takes the first.
WARM_SCHEDULES = [(1e-1, 0.5, 50), (1e-1, 0.25, 50), (1e-1, 0.5, 25), (1e-1, 0.25, 25), (1e-2, 0.5, 25),
                  (1e-2, 0.25, 25), (None, 1.0, 1 << 30)]


def time_to_gap(args, dlm, torch, dev):
    """Recurring daily instances (users x items of the daily recipe; day t
    from day t-1: 10% of edges' c perturbed by N(0, 0.02), b_j scaled by
    1 + N(0, 0.05), 2% of users churned).  Days 0-20 are solved to a 1e-5
    certified gap for labels.  The warm-start network trains on days 1-17;
    on days 18-20 (held out from the network, before any evaluation day) each
    warm start -- the previous day's dual and the network's prediction --
    picks the continuation (WARM_SCHEDULES: where it enters and how fast it
    descends to gamma_end) with the least mean time to the 1e-4 gap.  On days
    21-30 every start is driven to a 1e-4 certified gap and timed end to end
    (features and prediction included):
      fp32_cold     FP32 values, lam = 0, gamma 1e-1 -> gamma_end halved every
                    50 iterations (the plain method)
      bf16_cold     the same on BF16 values
      fp32_prev     FP32 from the previous day's dual, its chosen continuation
      fp32_learned  FP32 from the network's prediction, its chosen continuation
      bf16_learned  BF16 values + the prediction (the headline)
      fp32_prev_base, fp32_learned_base   both warm starts on the cold
                    start's continuation, for reference
    All forms use row normalization and check the gap every 25 iterations;
    warm starts add the adaptive restart."""
    import numpy as np
    import synth

    g_end, I, J = args.ttg_gamma, args.ttg_users, args.ttg_items
    n_days, n_train, n_select, gap_every = 30, 17, 20, 25
    t_all = time.perf_counter()
    inst = synth.generate(synth.recipe_daily(I=I, J=J, seed=1004), nthreads=args.threads)

    def make(inst, bf16):
        if bf16:
            c = torch.from_numpy(synth.round_bf16(inst.c, args.threads).view(np.int16)).to(dev).view(torch.bfloat16)
            a = torch.from_numpy(synth.round_bf16(inst.a, args.threads).view(np.int16)).to(dev).view(torch.bfloat16)
        else:
            c, a = torch.from_numpy(inst.c).to(dev), torch.from_numpy(inst.a).to(dev)
        rp, col = torch.from_numpy(inst.row_ptr).to(dev), torch.from_numpy(inst.col).to(dev)
        b = torch.from_numpy(inst.b).to(dev)
        s = dlm.Solver(rp, col, c, a, b, inst.J, bf16=bf16)
        del rp, col, c, a, b
        return s

    def run(s, start, sched, d):
        """One timed solve; returns (seconds, Stats)."""
        g0, factor, ips = sched
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        s.set_options(precondition=True, gap_every=gap_every, restart=start != "cold")
        s.set_schedule(g_end if g0 is None else g0, g_end, factor, ips)
        if start == "cold":
            s.set_lambda(zeros)
        elif start == "prev":
            s.set_lambda(labels[d - 1])
        else:
            s.set_lambda(ws.predict(dlm.WarmStart.features(s, labels[d - 1], g_end)))
        st = s.solve(1e-4, 100_000)
        torch.cuda.synchronize(dev)
        return time.perf_counter() - t0, st

    peak, _ = load_peaks()
    base = WARM_SCHEDULES[0]
    chosen = {}
    modes = ["fp32_cold", "bf16_cold", "fp32_prev", "fp32_learned", "bf16_learned", "fp32_prev_base",
             "fp32_learned_base"]
    res = {m: {"seconds": [], "iters": [], "gap": [], "roofline_frac": []} for m in modes}
    select = {st: {k: [] for k in range(len(WARM_SCHEDULES))} for st in ("prev", "learned")}
    labels, feats = {}, {}
    label_gap, label_iters = [], []
    ws, train = None, None
    zeros = torch.zeros(J, dtype=torch.float32, device=dev)
    for d in range(n_days + 1):
        if d > 0:
            inst = synth.next_day(inst, d, seed=1004, nthreads=args.threads)
        s32 = make(inst, False)
        bytes32 = s32.info()["bytes_per_iter"]
        if n_train < d <= n_select:
            # held-out days: every warm start tries every continuation
            for start in ("prev", "learned"):
                for k, sched in enumerate(WARM_SCHEDULES):
                    select[start][k].append(run(s32, start, sched, d)[0])
            if d == n_select:
                for start in ("prev", "learned"):
                    chosen[start] = WARM_SCHEDULES[min(select[start], key=lambda k: np.mean(select[start][k]))]
        if d > n_select:
            s16 = make(inst, True)
            bytes16 = s16.info()["bytes_per_iter"]
            plan = {"fp32_cold": ("cold", base), "bf16_cold": ("cold", base), "fp32_prev": ("prev", chosen["prev"]),
                    "fp32_learned": ("learned", chosen["learned"]), "bf16_learned": ("learned", chosen["learned"]),
                    "fp32_prev_base": ("prev", base), "fp32_learned_base": ("learned", base)}
            for m in modes:
                s, nbytes = (s16, bytes16) if m.startswith("bf16") else (s32, bytes32)
                start, sched = plan[m]
                dt, st = run(s, start, sched, d)
                sweeps = st.iter + st.iter // gap_every + 1 + (1 if start == "learned" else 0)
                res[m]["seconds"].append(dt)
                res[m]["iters"].append(int(st.iter))
                res[m]["gap"].append(float(st.rel_gap))
                res[m]["roofline_frac"].append(sweeps * nbytes / dt / 1e9 / peak)
            s16.close()
        # label: the day solved to 1e-5 from the previous day's dual
        s32.set_options(precondition=True, gap_every=50, restart=True)
        if d == 0:
            s32.set_schedule(1e-1, g_end, 0.5, 50)
            s32.set_lambda(zeros)
        else:
            s32.set_schedule(g_end)
            s32.set_lambda(labels[d - 1])
            if d <= n_train:
                feats[d] = dlm.WarmStart.features(s32, labels[d - 1], g_end)
        st = s32.solve(1e-5, 8_000)
        label_gap.append(float(st.rel_gap))
        label_iters.append(int(st.iter))
        labels[d] = s32.lam()
        s32.close()
        if d == n_train:
            X = torch.cat([feats[k] for k in range(1, n_train + 1)])
            y = torch.cat([labels[k] for k in range(1, n_train + 1)])
            ws = dlm.WarmStart(128, 1)
            t0 = time.perf_counter()
            losses = ws.train(X, y, 300, 1e-3)
            train = {"rows": int(X.shape[0]), "days": f"1-{n_train}", "steps": 300, "lr": 1e-3,
                     "loss_first": float(losses[0]), "loss_last": float(losses[-1]),
                     "seconds": time.perf_counter() - t0}
    fmt = lambda sc: {"gamma_0": g_end if sc[0] is None else sc[0], "factor": sc[1],
                      "iters_per_stage": sc[2] if sc[0] is not None else None}
    out = {"workload": f"recurring daily instances: {I:,} users x {J:,} items (~{I * 25 / 1e6:.0f}M nnz), "
                       f"30 days; network trained on days 1-{n_train}, continuations chosen on days "
                       f"{n_train + 1}-{n_select}, evaluated on days {n_select + 1}-{n_days}",
           "gamma_end": g_end, "target_rel_gap": 1e-4, "gap_every": gap_every, "train": train,
           "labels": {"target": 1e-5, "max_iters": 8000, "worst_gap": max(label_gap),
                      "mean_iters": float(np.mean(label_iters))},
           "continuations": {"candidates": [fmt(sc) for sc in WARM_SCHEDULES],
                             "chosen": {k: fmt(v) for k, v in chosen.items()},
                             "selection_mean_s": {st: [float(np.mean(select[st][k])) for k in range(len(WARM_SCHEDULES))]
                                                  for st in select}},
           "modes": {m: {"mean_s": float(np.mean(v["seconds"])), "mean_iters": float(np.mean(v["iters"])),
                         "mean_roofline_frac": float(np.mean(v["roofline_frac"])), "per_day_s": v["seconds"],
                         "per_day_iters": v["iters"], "max_gap": max(v["gap"])} for m, v in res.items()},
           "seconds_total": time.perf_counter() - t_all}
    M = out["modes"]
    out["headline_speedup_bf16_learned_vs_fp32_cold"] = M["fp32_cold"]["mean_s"] / M["bf16_learned"]["mean_s"]
    out["learned_vs_prev_seconds"] = M["fp32_learned"]["mean_s"] / M["fp32_prev"]["mean_s"]
    out["learned_vs_prev_iters"] = M["fp32_learned"]["mean_iters"] / M["fp32_prev"]["mean_iters"]
    out["bf16_learned_vs_fp32_prev_iters_saved"] = M["fp32_prev"]["mean_iters"] - M["bf16_learned"]["mean_iters"]
    out["oracle_fp32_cold"] = oracle_time_to_gap(args, dlm, torch, dev, g_end, gap_every)
    if ws is not None:
        ws.close()
    return out


def oracle_time_to_gap(args, dlm, torch, dev, g_end, gap_every, frac=0.01):
    """The FP64 oracle's time to the 1e-4 certified gap, FP32 cold start and
    the protocol of fp32_cold (continuation 1e-1 -> gamma_end halved every 50
    iterations, row normalization, a check every gap_every iterations), on a
    seeded user sample of the daily recipe (capacities from the sample), on
    all host threads; the GPU's FP32 cold start on the same sample beside it."""
    import numpy as np
    import oracle
    import synth

    r = synth.recipe_daily(I=args.ttg_users, J=args.ttg_items, seed=1004)
    ids = synth.sample_users(r.I, frac, 5151)
    sub = synth.generate(r, ids=ids, nthreads=args.threads)
    p = oracle.Problem(sub.row_ptr, sub.col, sub.c.astype(np.float64), sub.a.astype(np.float64), sub.b, sub.J)
    sched = (1e-1, g_end, 0.5, 50)
    nc = host_cores()
    t0 = time.perf_counter()
    ref = oracle.solve_threads(p, *sched, precondition=True, target=1e-4, gap_every=gap_every, max_iters=100_000,
                               nthreads=nc)
    t_ref = time.perf_counter() - t0
    arrs = [torch.from_numpy(v).to(dev) for v in (sub.row_ptr, sub.col, sub.c, sub.a, sub.b)]
    s = dlm.Solver(*arrs, sub.J)
    s.set_schedule(*sched)  # warm the graphs and kernels once
    s.step(20)
    st, sec = solve_from_zero(s, torch, 1e-4, 100_000, sched=sched, gap_every=gap_every, restart=False)
    s.close()
    return {"instance": f"daily recipe, {frac:.0%} seeded user sample of day 0 ({len(ids):,} users, {p.nnz:,} nnz)",
            "oracle": {"seconds": t_ref, "iters": ref["iters"], "rel_gap": ref["rel_gap"], "cores": nc,
                       "kind": "oracle (FP64, sweep split over host threads)"},
            "gpu_fp32_cold": {"seconds": sec, "iters": int(st.iter), "rel_gap": st.rel_gap},
            "gpu_speedup": t_ref / sec if sec > 0 else None}


def run_sharded(args, dlm, torch, dev, rank, world, barrier, dist):
    """N > 1 GPUs on one instance, user-sharded (weak scaling: every rank holds
    the workload's users -- rank r the users r I .. (r + 1) I - 1 of an
    instance of N I users over the same items -- and the capacities are those
    of the whole instance).  Each iteration: every rank sweeps its users, the
    int64 fixed-point item sums are all-reduced (NCCL), every rank takes the
    same update.  Timed with CUDA events, barrier and synchronize on both
    sides, the slowest rank's time."""
    import numpy as np
    import synth

    w = WORKLOADS[args.workload]
    bf16 = w["bf16"]
    I = max(1000, int(round(w["users"] * args.scale)))
    r = synth.Recipe(I=I * world, J=w["items"], seed=w["seed"]) if args.workload != "boxcut" else \
        synth.recipe_production(I=I * world, J=w["items"], seed=w["seed"])
    t_gen = time.perf_counter()
    ids = np.arange(rank * I, (rank + 1) * I, dtype=np.int64)
    inst = synth.generate(r, ids=ids, nthreads=args.threads)
    b = torch.from_numpy(inst.b).to(dev)
    dist.all_reduce(b)  # the capacities of the whole instance (0.05 sum over every rank's users)
    t_gen = time.perf_counter() - t_gen
    to = lambda v: torch.from_numpy(v).to(dev)
    if bf16:
        c = to(synth.round_bf16(inst.c, args.threads).view(np.int16)).view(torch.bfloat16)
        a = to(synth.round_bf16(inst.a, args.threads).view(np.int16)).view(torch.bfloat16)
    else:
        c, a = to(inst.c), to(inst.a)
    kind_args = dict(kind=w.get("kind", 0), z=w.get("z", 1.0), cut=w.get("cut"), bf16=bf16)
    t_setup = time.perf_counter()
    s = dlm.ShardedSolver.distributed(to(inst.row_ptr), to(inst.col), c, a, b, inst.J, **kind_args)
    torch.cuda.synchronize(dev)
    t_setup = time.perf_counter() - t_setup
    s.set_schedule(*w["schedule"])
    info = s.info()
    for _ in range(args.warmup):
        s.step(args.iters)
    sampler = ClockSampler(gpu_id_for_smi(torch, dev))
    sampler.start()
    time.sleep(0.3)
    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize(dev)
    e0.record(st)
    for _ in range(args.steps):
        s.step(args.iters)
    e1.record(st)
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    elapsed = e0.elapsed_time(e1) / 1000.0
    units = info["nnz"] * args.iters * args.steps
    value, tmax = replica_throughput(units, elapsed, dist, dev)
    cert = s.stats()
    peak, peak_kind = load_peaks()
    it_s = tmax / (args.iters * args.steps)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": tmax * 1000.0 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_for(args, world),
        "instance": {"users_per_rank": I, "nnz_this_rank": info["nnz"], "items": inst.J,
                     "bytes_per_iter_this_rank": info["bytes_per_iter"]},
        "roofline": {"bound": "hbm", "achieved": info["bytes_per_iter"] / it_s / 1e9, "peak": peak, "unit": "GB/s",
                     "frac": info["bytes_per_iter"] / it_s / 1e9 / peak, "traffic": None,
                     "peak_source": f"{peak_kind} (copy bandwidth)",
                     "kernel": "sweep_kernel + int64 all-reduce + fista_update_kernel (per-iteration time of the "
                               "slowest rank)"},
        "cpu_baseline": None,
        "e2e": {"value": None, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0,
                "note": "not measured in the sharded form"},
        "gpu_launches": 2 * args.iters * args.steps,
        "clocks": clocks,
        "certificate_after_timing": {"rel_gap": cert.rel_gap, "dual_obj": cert.dual_obj, "iter": cert.iter},
        "setup_s": {"generate": t_gen, "shard_setup_and_create": t_setup},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    s.close()
    dist.destroy_process_group()
    return 0


def run_batched(args, dlm, torch, dev, rank, world, barrier, max_over_ranks, dist):
    """The batched workload: 64 handles run as one batch."""
    import numpy as np
    import synth

    w = WORKLOADS["batched"]
    recipes = synth.recipe_batch(n=w["n"], seed=w["seed"])
    if args.scale != 1.0:
        for r, _ in recipes:
            r.I = max(1000, int(round(r.I * args.scale)))
    t_gen = time.perf_counter()
    insts = [(make_instance(r, True, torch, True, args.threads), g) for r, g in recipes]
    for inst, _ in insts:
        inst.c32 = inst.a32 = None  # FP32 copies are only needed for the single-instance error statement
    t_gen = time.perf_counter() - t_gen
    dlm.load()

    def create(inst, on_device):
        if on_device:
            arrs = [torch.from_numpy(v).to(dev, non_blocking=True) for v in
                    (inst.row_ptr, inst.col, inst.c.view(np.int16), inst.a.view(np.int16), inst.b)]
            arrs[2], arrs[3] = arrs[2].view(torch.bfloat16), arrs[3].view(torch.bfloat16)
            s = dlm.Solver(*arrs, inst.J, bf16=True)
            del arrs
        else:
            s = dlm.Solver(inst.row_ptr, inst.col, inst.c, inst.a, inst.b, inst.J, bf16=True)
        return s

    t_setup = time.perf_counter()
    solvers = []
    for inst, g in insts:
        s = create(inst, True)
        s.set_schedule(g)
        solvers.append(s)
    torch.cuda.synchronize(dev)
    bt = dlm.Batch(solvers)
    t_setup = time.perf_counter() - t_setup
    infos = [s.info() for s in solvers]
    nnz = sum(i["nnz"] for i in infos)
    users = sum(i["num_users"] for i in infos)
    bytes_iter = sum(i["bytes_per_iter"] for i in infos)
    # bytes the layout streams: 16-bit item index + two bf16 values per edge,
    # a 12-byte header per 32 users
    layout_bytes = sum(6 * i["nnz"] + (i["num_users"] + 31) // 32 * 12 for i in infos)

    t_tune = time.perf_counter()
    chosen, tune_ms = bt.autotune(3)
    t_tune = time.perf_counter() - t_tune
    for _ in range(args.warmup):
        bt.step(args.iters)
    torch.cuda.synchronize(dev)

    sampler = ClockSampler(gpu_id_for_smi(torch, dev))
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize(dev)
    sweep_ms = upd_ms = tot_ms = 0.0
    for _ in range(args.steps):
        a_, b_, c_ = bt.step_timed(args.iters)
        sweep_ms += a_
        upd_ms += b_
        tot_ms += c_
    torch.cuda.synchronize(dev)
    barrier()
    clocks = sampler.stop()
    iters_total = args.iters * args.steps
    value, elapsed_s = replica_throughput(nnz * iters_total, tot_ms / 1000.0, dist, dev)

    st = torch.cuda.current_stream(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(st)
    for _ in range(args.steps):
        bt.step(args.iters)
    e1.record(st)
    torch.cuda.synchronize(dev)
    graph_ms_per_step = e0.elapsed_time(e1) / args.steps
    stats = bt.stats()
    bt.close()
    for s in solvers:
        s.close()
    del solvers
    torch.cuda.synchronize(dev)

    # end to end: every member created from pinned host arrays, batched, the
    # iterations, every member's lam back to the host
    h2d = sum(i.row_ptr.nbytes + i.col.nbytes + i.c.nbytes + i.a.nbytes + i.b.nbytes for i, _ in insts)
    d2h = sum(4 * i.J for i, _ in insts)
    lam_host = [torch.empty(i.J, dtype=torch.float32, pin_memory=True) for i, _ in insts]
    e2e_times = []
    for k in range(args.e2e_steps + 1 if args.e2e_steps > 0 else 0):
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        ss = []
        for inst, g in insts:
            s = create(inst, False)
            s.set_schedule(g)
            ss.append(s)
        b2 = dlm.Batch(ss)
        b2.set_options(**{f: getattr(chosen, f) for f in ("mapping", "coop_max", "block_threads", "ctas_per_sm",
                                                           "topk")})
        b2.step(args.iters)
        for s, lh in zip(ss, lam_host):
            dlm.dlm_get_lambda(s.h, lh, dlm.DLM_MEM_HOST)
        b2.close()
        for s in ss:
            s.close()
        dt = time.perf_counter() - t0
        if k > 0:
            e2e_times.append(dt)
    e2e_value = None
    if e2e_times:
        e2e_value, _ = replica_throughput(nnz * args.iters, statistics.mean(e2e_times), dist, dev)

    peak, peak_kind = load_peaks()
    sweep_s = sweep_ms / 1000.0 / iters_total
    achieved = bytes_iter / sweep_s / 1e9
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": recorded_traffic("batched", nnz, users) if args.scale == 1.0 else None,
            "peak_source": f"{peak_kind} (copy bandwidth, MEASURED_PEAKS.json)"
            if peak_kind == "measured" else "fallback 6.8 TB/s",
            "kernel": ("sweep_dyn_kernel" if chosen.mapping == 3 else "sweep_kernel") +
                      " (all 64 instances in one launch)",
            "algorithmic_bytes_per_launch": bytes_iter,
            "layout_bytes_per_launch": layout_bytes,
            "layout_frac": layout_bytes / sweep_s / 1e9 / peak,
            "sweep_share_of_iteration": sweep_ms / tot_ms if tot_ms > 0 else None,
            "sweep_us": sweep_s * 1e6, "update_us": upd_ms * 1000.0 / iters_total}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        ps = batch_sample(args.cpu_frac, threads=args.threads)
        nc = host_cores()
        v1, it1, dt1, nnz_s = time_oracle_batch(ps, args.cpu_seconds * 0.4)
        v, iters, dt, nnz_s = time_oracle_batch(ps, args.cpu_seconds * 0.6, nthreads=nc)
        cpu = {"value": v, "unit": UNIT, "cores": nc, "kind": "oracle", "single_core_value": v1,
               "sample": (f"{args.cpu_frac:.0%} seeded user sample of every member ({nnz_s} nnz over {len(ps)} "
                          f"members), {iters} FP64 oracle iterations each on {nc} threads in {dt:.1f} s; "
                          f"single-threaded {it1} iterations in {dt1:.1f} s")}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": elapsed_s * 1000.0 / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": config_for(args, world),
        "instance": {"instances": len(insts), "users": users, "nnz": nnz, "bytes_per_iter": bytes_iter,
                     "mapping": chosen.as_dict(), "tuner_sweep_ms": tune_ms},
        "roofline": roof,
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "note": "per step: 64 x dlm_create from pinned host arrays, batch, iterations, every lam to host"},
        "gpu_launches": 2 * iters_total,
        "clocks": clocks,
        "graph_ms_per_step": graph_ms_per_step,
        "member_status": sorted({x.status for x in stats}),
        "setup_s": {"generate": t_gen, "upload_and_create": t_setup, "autotune": t_tune},
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
