"""Benchmark: batched interior-point solves on one GB300 (or N GPUs, one set per GPU).

Headline workload ("batch320-lifted"): 256 load scenarios of a seeded synthetic 1,000-bus
AC-OPF grid (per-bus load scaling U[0.8, 1.2]) plus 64 seeded grids of 118-2,000 buses, solved
together by the batched LiftedKKT FP64 interior-point method to the 1e-6 scaled KKT tolerance.
One step = set every instance back to its starting point and run sweeps until every instance has
converged or stopped; value = converged instances / step time (symbolic analyses, once per
pattern at batch creation, are reported separately as init_s, like the paper's "init").  The
instance pool (~0.7 GB) is larger than L2, so no flush is needed between steps.

Also reported: the single-problem GPU IPM on a sample of the same instances ("plain"), the
condensed KKT solve kernel at 10,000 buses with its own roofline ("kkt10k"), full single-problem
IPM solves of several grids and forms ("ipm"), and the CPU oracle ("cpu_baseline").

Prints one JSON line (rank 0).  ``--impl reference`` times the CPU oracle on the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "IPM solves/s at 1e-6 KKT tol, plain vs batched/warm-start; factor GB/s"
UNIT = "IPM solves/s"
KKT_UNIT = "KKT solves/s"
FORM_NAMES = {"lifted": "LiftedKKT", "regularized": "dual-regularized condensed (delta_c = 1/gamma, "
               "gamma = 1e6)", "hykkt": "HyKKT (gamma = 1e6)"}


def workload_name(kkt):
    return (f"batch320-{kkt}: 256 load scenarios of a seeded 1,000-bus grid + 64 seeded grids of "
            f"118-2,000 buses, batched {FORM_NAMES[kkt]} FP64 IPM to 1e-6 scaled KKT tolerance")
KKT_WORKLOAD = ("kkt10k-lifted: LiftedKKT condensed KKT solve (condense + supernodal Cholesky + "
                "FP64-refined solve) on a seeded synthetic 10,000-bus grid, Sigma log-uniform "
                "[1e-8,1e8]")
MAX_ITER = 300
# FP64 peak from unit counts: 4 SMSPs x 0.5 FP64 FMA per cycle (one FP64 warp instruction per 64
# cycles, measured) x 2 flops x 152 SMs x 2.07 GHz
FP64_PEAK_TFLOPS = 152 * 4 * 0.5 * 2 * 2.07e9 / 1e12


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def build_inputs(seed=3):
    from synth import config_grid, kkt_point
    g = config_grid("planar10k")
    p = kkt_point(g, seed)
    d = np.concatenate([p["d_g"], p["d_s"]])
    b = np.concatenate([p["r3"], p["r4"]])
    return g, p, d, b


# ------------------------------------------------------------------ oracle (CPU) arm
def oracle_setup():
    from oracle.opf import OPFModel
    from oracle import kkt as K
    g, p, d, b = build_inputs()
    m = OPFModel(g)
    J = m.jacobian(p["x"]).tocsr()
    Wf = m.hessian(p["x"], p["y"], p["z"])
    solver = K.CondensedSolver(Wf, J)
    dw, F, _ = K.inertia_schedule(lambda dw: K.condensed_matrix(Wf, p["sigma_x"], J, d, dw), solver)
    return dict(J=J, Wf=Wf, sigma=p["sigma_x"], d=d, a=p["r1"], b=b, solver=solver, dw=dw)


def oracle_step(o):
    from oracle import kkt as K
    Km = K.condensed_matrix(o["Wf"], o["sigma"], o["J"], o["d"], o["dw"])
    F = o["solver"].factor(Km)
    A = K.aug_matrix(o["Wf"], o["sigma"], o["J"], o["d"], 0, o["dw"])
    dx, dz, hist = K.lifted_solve(F, A, o["J"], o["d"], o["a"], o["b"])
    return hist[-1]


def kkt_cpu_baseline(budget_s=8.0, min_solves=3):
    o = oracle_setup()
    oracle_step(o)  # warm
    t0 = time.perf_counter()
    k = 0
    while k < min_solves or time.perf_counter() - t0 < budget_s:
        oracle_step(o)
        k += 1
        if k >= 200:
            break
    el = time.perf_counter() - t0
    return {"value": k / el, "unit": KKT_UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{k} full KKT solves of the same workload in {el:.1f} s "
                      f"(scipy condensation + plain C up-looking Cholesky + numpy refinement, "
                      f"single thread; host has {os.cpu_count()} cores)"}


def _oracle_solve(grid, kkt="lifted"):
    from oracle.opf import OPFModel
    from oracle import ipm as oipm
    r = oipm.solve(OPFModel(grid), oipm.Options(kkt=kkt, gamma=1e6))
    return r.status == "converged", r.iters


def _oracle_solve_seed(spec):
    """Pool worker (spawned process): rebuild the instance from its seeds and solve it."""
    sys.path.insert(0, ROOT)
    from synth import config_grid, scale_loads, mixed_grid
    kind, seed, kkt = spec
    g = scale_loads(config_grid("planar1k"), seed) if kind == "scen" else mixed_grid(seed)
    return _oracle_solve(g, kkt)


def sample_specs(k, part=0):
    """k instances of the batched workload, alternating scenarios and mixed grids."""
    o = 100000 * part
    out = []
    for i in range(k):
        out.append(("scen", o + 1000 + i // 2) if i % 2 == 0 else ("mixed", o + 2000 + i // 2))
    return out


def batch_cpu_baseline(budget_s=10.0, pool=True, kkt="lifted"):
    """The oracle IPM (plain FP64 CPU, simple sparse LDL^T) on a bounded sample of the batched
    workload: one thread, then (pool) one problem per host core in spawned processes."""
    from synth import config_grid, scale_loads, mixed_grid
    specs = sample_specs(64)
    t0 = time.perf_counter()
    k = conv = 0
    while k < 2 or (time.perf_counter() - t0 < budget_s and k < len(specs)):
        kind, seed = specs[k]
        g = scale_loads(config_grid("planar1k"), seed) if kind == "scen" else mixed_grid(seed)
        ok, _ = _oracle_solve(g, kkt)
        conv += ok
        k += 1
    el = time.perf_counter() - t0
    out = {"value": conv / el, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{k} instances of the batched workload (alternating 1,000-bus scenarios and "
                     f"mixed grids), {conv} converged, {el:.1f} s, one thread; host has "
                     f"{os.cpu_count()} cores"}
    if pool:
        import multiprocessing as mp
        cores = os.cpu_count() or 1
        specs = [(kind, seed, kkt) for kind, seed in sample_specs(2 * cores)]
        ctx = mp.get_context("spawn")
        with ctx.Pool(cores) as P:
            P.map(_oracle_solve_seed, specs[:cores])  # start-up and imports, untimed
            t0 = time.perf_counter()
            res = P.map(_oracle_solve_seed, specs)
            el = time.perf_counter() - t0
        c2 = sum(ok for ok, _ in res)
        out["pool"] = {"value": c2 / el, "unit": UNIT, "cores": cores,
                       "sample": f"{len(specs)} instances, one per core at a time, {c2} converged, "
                                 f"{el:.1f} s"}
    return out


def run_reference(args, rank, world):
    """The oracle on the batched workload: each step solves one instance (cycling through a
    sample of scenarios and mixed grids) with the plain CPU IPM, single thread."""
    if rank != 0:
        return
    from synth import config_grid, scale_loads, mixed_grid
    specs = sample_specs(max(8, args.steps + args.warmup))
    grids = [scale_loads(config_grid("planar1k"), s_) if k_ == "scen" else mixed_grid(s_)
             for k_, s_ in specs]
    for i in range(args.warmup):
        _oracle_solve(grids[i], args.kkt)
    t0 = time.perf_counter()
    conv = 0
    for i in range(args.steps):
        ok, _ = _oracle_solve(grids[args.warmup + i], args.kkt)
        conv += ok
    el = time.perf_counter() - t0
    v = conv / el
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload_name(args.kkt),
                       "parallelism": "one instance per step, one thread"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} instances of the batched workload, "
                                       f"{conv} converged, single thread"},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm
def kkt_measure(args):
    """The condensed KKT solve at 10,000 buses (condense + factor + FP64-refined solve), with the
    FP32-factor variant, its own roofline, e2e and oracle timing (one GPU)."""
    import torch
    import paper_2405_14236_gb300 as cp
    world, rank, local_rank = 1, 0, torch.cuda.current_device()
    stream = torch.cuda.current_stream()
    f64 = dict(dtype=torch.float64, device="cuda")
    g, p, d, b = build_inputs()
    t = lambda a: torch.as_tensor(np.ascontiguousarray(a), **f64)
    opf = cp.Opf(g)
    n, m = g.n, g.m_e + g.m_i
    Jv = torch.zeros(opf.nnzJ, **f64)
    Wv = torch.zeros(opf.nnzW, **f64)
    gg, hh = torch.zeros(g.m_e, **f64), torch.zeros(g.m_i, **f64)
    opf.eval(t(p["x"]), t(p["y"]), t(p["z"]), 1.0, None, None, gg, hh, Jv, Wv)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    S = cp.Symbolic(n, m, opf.J_rowptr, opf.J_colind, opf.W_rowptr, opf.W_colind)
    symbolic_s = time.perf_counter() - t0
    N = cp.Numeric(S)
    sig, dd, a, bb = t(p["sigma_x"]), t(d), t(p["r1"]), t(b)
    info = torch.zeros(1, dtype=torch.int32, device="cuda")
    dw = 0.0
    for k in range(40):
        dw = 0.0 if k == 0 else 1e-4 * 100.0 ** (k - 1)
        cp.ipm_condense(S, N, Wv, sig, Jv, dd, dw)
        cp.ipm_factor(S, N, info)
        if int(info.item()) == -1:
            break
    dx, dz = torch.zeros(n, **f64), torch.zeros(m, **f64)
    eta = torch.zeros(1, **f64)
    steps_t = torch.zeros(1, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def step():
        cp.ipm_condense(S, N, Wv, sig, Jv, dd, dw)
        e1.record(stream)
        cp.ipm_factor(S, N, info)
        e2.record(stream)
        cp.ipm_aug_solve(S, N, Wv, sig, Jv, dd, dw, a, bb, dx, dz, eta, steps_t)

    e0, e1, e2, e3 = (torch.cuda.Event(enable_timing=True) for _ in range(4))
    for _ in range(args.warmup):
        flush.zero_()
        e0.record(stream)
        step()
        e3.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    torch.cuda.synchronize()
    ph = np.zeros((args.steps, 3))
    l0 = cp.launch_count()
    for k in range(args.steps):
        flush.zero_()
        e0.record(stream)
        step()
        e3.record(stream)
        e3.synchronize()
        ph[k] = [e0.elapsed_time(e1), e1.elapsed_time(e2), e2.elapsed_time(e3)]
    launches = cp.launch_count() - l0
    torch.cuda.synchronize()
    ok = int(info.item()) == -1
    eta_v, refine = float(eta.item()), int(steps_t.item())
    # ---- e2e: host buffers, copies inside the timed region
    hW, hJ, hs, hd, ha, hb = (x.cpu().pin_memory() for x in (Wv, Jv, sig, dd, a, bb))
    hdx, hdz = torch.empty(n, dtype=torch.float64).pin_memory(), torch.empty(m, dtype=torch.float64).pin_memory()
    dW, dJ, ds_, ddd, da, db = (torch.empty_like(x) for x in (Wv, Jv, sig, dd, a, bb))
    e_tot = 0.0
    for k in range(max(3, args.steps // 2)):
        flush.zero_()
        e0.record(stream)
        for dst, src in ((dW, hW), (dJ, hJ), (ds_, hs), (ddd, hd), (da, ha), (db, hb)):
            dst.copy_(src, non_blocking=True)
        cp.ipm_condense(S, N, dW, ds_, dJ, ddd, dw)
        cp.ipm_factor(S, N, info)
        cp.ipm_aug_solve(S, N, dW, ds_, dJ, ddd, dw, da, db, dx, dz, eta, steps_t)
        hdx.copy_(dx, non_blocking=True)
        hdz.copy_(dz, non_blocking=True)
        e3.record(stream)
        e3.synchronize()
        e_tot += e0.elapsed_time(e3)
    n_e2e = max(3, args.steps // 2)
    # ---- precision row: FP32 condensation/factor/solves + FP64 preconditioned CG refinement
    fp32 = None
    if not args.no_fp32:
        N32 = cp.Numeric(S, precision=32)
        dx32, dz32 = torch.zeros(n, **f64), torch.zeros(m, **f64)
        dw32 = dw
        for k in range(40):  # the FP32 factor of the shifted matrix may need a larger delta_w
            cp.ipm_condense(S, N32, Wv, sig, Jv, dd, dw32)
            cp.ipm_factor(S, N32, info)
            if int(info.item()) == -1:
                break
            dw32 = max(1e-4, dw32 * 100.0)
        ph32 = []
        st32 = 0
        for k in range(args.warmup + max(3, args.steps // 2)):
            flush.zero_()
            e0.record(stream)
            cp.ipm_condense(S, N32, Wv, sig, Jv, dd, dw32)
            e1.record(stream)
            cp.ipm_factor(S, N32, info)
            e2.record(stream)
            try:
                st32 = cp.ipm_aug_solve(S, N32, Wv, sig, Jv, dd, dw32, a, bb, dx32, dz32, eta, steps_t)
            except Exception as ex:  # reported, not fatal to the FP64 line
                st32 = str(ex)
            e3.record(stream)
            e3.synchronize()
            if k >= args.warmup:
                ph32.append([e0.elapsed_time(e1), e1.elapsed_time(e2), e2.elapsed_time(e3)])
        ph32 = np.array(ph32)
        prec, pcg = cp.ipm_num_info(N32)
        rel = float((dx32 - dx).abs().max().item() / dx.abs().max().item()) if dw32 == dw else None
        fp32 = {"value": len(ph32) / (ph32.sum() / 1e3), "unit": KKT_UNIT,
                "phases_ms": {nm: float(v) for nm, v in zip(["condense", "factor", "solve"],
                                                            ph32.mean(axis=0))},
                "delta_w": dw32, "pcg_iters": pcg, "backward_error": float(eta.item()),
                "status": st32, "dx_rel_diff_vs_fp64": rel}
    clk = clocks.stop()
    h2d = 8 * (opf.nnzW + opf.nnzJ + n + m + n + m)
    d2h = 8 * (n + m)
    step_ms = ph.sum(axis=1)
    t_max = float(step_ms.sum())
    if world > 1:
        tt = torch.tensor([t_max], dtype=torch.float64, device="cuda")
        torch.distributed.all_reduce(tt, op=torch.distributed.ReduceOp.MAX)
        t_max = float(tt.item())
    value = world * args.steps / (t_max / 1e3)
    if rank != 0:
        return
    # ---- roofline of the dominant phase
    hbm, hbm_src = measured_peaks()
    mean = ph.mean(axis=0)
    nnzL = S.nnz_offdiag + n
    nsolves = 1 + refine
    bytes_ = {
        "condense": 8.0 * (opf.nnzJ + m + opf.nnzW + n) + 8.0 * S.nnz_k,
        "factor": 8.0 * (S.nnz_k + nnzL),
        "solve": nsolves * (2 * 8.0 * nnzL + 3 * 8.0 * n) + 8.0 * (2 * opf.nnzJ + 2 * opf.nnzW),
    }
    names = ["condense", "factor", "solve"]
    dom = int(np.argmax(mean))
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            import hashlib
            tr = json.load(open(tfile))
            h = hashlib.sha256(open(os.path.join(ROOT, "paper_2405_14236_gb300", "csrc",
                                                  "numeric.cu"), "rb").read()).hexdigest()[:16]
            if tr.get("numeric_cu_sha") == h and names[dom] in tr.get("bytes_per_step", {}):
                traffic = tr["bytes_per_step"][names[dom]]
        except Exception:
            traffic = None
    ach = bytes_[names[dom]] / (mean[dom] / 1e3) / 1e9
    line = {
        "value": value, "unit": KKT_UNIT, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(step_ms.mean()),
        "config": {"workload": KKT_WORKLOAD, "n": n, "m": m, "nnzJ": opf.nnzJ, "nnzW": opf.nnzW,
                   "nnzK_lower": S.nnz_k, "nnzL": nnzL, "nsuper": S.nsuper,
                   "nlevels": S.nlevels, "factor_flops": S.flops, "delta_w": dw,
                   "l2": "flushed between timed steps (256 MiB write)",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "roofline": {"kernel": names[dom], "bound": "hbm", "achieved": ach, "peak": hbm,
                     "unit": "GB/s", "frac": ach / hbm, "peak_source": hbm_src,
                     "traffic": traffic, "algorithmic_bytes": bytes_[names[dom]]},
        "phases_ms": {nm: float(v) for nm, v in zip(names, mean)},
        "factor": {"GB_s": bytes_["factor"] / (mean[1] / 1e3) / 1e9,
                   "GFLOP_s": S.flops / (mean[1] / 1e3) / 1e9},
        "backward_error": eta_v, "refine_steps": refine, "factor_ok": ok,
        "symbolic_s": symbolic_s,
        "e2e": {"value": n_e2e / (e_tot / 1e3), "unit": KKT_UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "fp32": fp32,
        "clocks": clk,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = kkt_cpu_baseline()
    return line


def aggregate_ranks(t_ms, converged, world, device):
    """Whole-job figures of a run on `world` ranks: the slowest rank's time and the sum of the
    converged instances (each rank solves its own instance set)."""
    if world == 1:
        return t_ms, converged
    import torch
    import torch.distributed as dist
    t = torch.tensor([t_ms], dtype=torch.float64, device=device)
    c = torch.tensor([converged], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), float(c.item())


def batch_form_measure(grids, kkt="regularized", gamma=1e6, steps=3, precision=64, relax=(0, 0)):
    """The headline's instances solved by another batched form: "regularized" (the
    dual-regularized condensed form: equality rows kept, delta_c = 1/gamma) or "hykkt" (CG on
    the Schur complement of K_gamma, Section 3.1); or, with precision 32, LiftedKKT with the FP32
    factor and FP64 refinement (launch shapes autotuned for it, per-sweep kernel times, the share
    of iterations the FP32 factor served)."""
    import torch
    import paper_2405_14236_gb300 as cp
    opfs = [cp.Opf(g) for g in grids]
    B = cp.Batch(opfs, kkt=kkt, gamma=gamma, precision=precision, relax=relax)
    # launch shapes tuned for this form, as for the headline
    tune = B.autotune(sweeps=8)
    best = tune["candidates"][tune["best"]]
    shape = {k: best[k] for k in ("cluster", "threshold", "blocks_per_instance")}
    B.set_timing(True)
    B.run(max_iter=MAX_ITER)
    B.kernel_time()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms, conv, its = [], [], []
    fact_ms = solve_ms = 0.0
    n_sw = it32 = it_all = n64 = 0
    for _ in range(steps):
        torch.cuda.synchronize()
        e0.record(stream)
        B.reset()
        B.run(max_iter=MAX_ITER)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
        r = B.results()
        conv.append(int((r["status"] == 1).sum()))
        its.append(float(r["iters"].mean()))
        kt = B.kernel_time()
        fact_ms += kt["fact_ms"]
        solve_ms += kt["solve_ms"]
        n_sw += kt["sweeps"]
        if precision == 32:
            pr = B.solve_info()
            it32 += int(pr["iters32"].sum())
            it_all += int(r["iters"].sum())
            n64 += int((pr["k64"] >= 0).sum())
    out = {"kkt": kkt, "gamma": gamma, "value": float(np.sum(conv) / (np.sum(ms) / 1e3)),
           "unit": UNIT, "converged_per_step": conv, "iters_mean": float(np.mean(its)),
           "ms_per_step": float(np.mean(ms)), "sweeps": int(r["sweeps"]),
           "launch_shape": shape, "relax": list(relax),
           "kernels_ms_per_sweep": {"factor_both_rounds": fact_ms / max(n_sw, 1),
                                    "solve_first": solve_ms / max(n_sw, 1)}}
    if precision == 32:
        out.update({"precision": "FP32 condensed matrix, factor and triangular solves; FP64 "
                                 "Richardson refinement on the augmented system to 1e-10",
                    "fp32_share_of_iterations": it32 / max(it_all, 1),
                    "instances_gone_fp64_per_step": n64 / steps})
    if kkt == "hykkt":
        out["cg_iters_per_ipm_iter"] = float(r["cg_iters"].sum() / max(1, r["iters"].sum()))
    return out


def recipe_measure(steps=2):
    """The batched LiftedKKT IPM (with the restoration phase) on the workload's shape drawn at the
    stated parameters (synth.recipe_batch: impedances and loads unscaled, ratings 1.2 x base
    flow): how the instances end (converged, locally infeasible, failed line search at a
    feasible point, iteration limit) and the time of a batch."""
    import torch
    import paper_2405_14236_gb300 as cp
    from synth import recipe_batch
    grids = recipe_batch()
    B = cp.Batch([cp.Opf(g) for g in grids])
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        B.reset()
        torch.cuda.synchronize()
        e0.record(stream)
        B.run(max_iter=MAX_ITER)
        e1.record(stream)
        e1.synchronize()
        ms.append(e0.elapsed_time(e1))
    r = B.results()
    names = {1: "converged", 5: "failed line search at a feasible point", 7: "iteration limit",
             8: "locally infeasible (restoration converged with the violation)"}
    counts = {}
    for s in r["status"]:
        k = names.get(int(s), f"status {int(s)}")
        counts[k] = counts.get(k, 0) + 1
    return {"workload": "32 load scenarios of a 1,000-bus grid + 8 grids of 118-2,000 buses at "
                        "the stated parameters (impedances and loads unscaled, ratings 1.2 x base "
                        "flow), batched LiftedKKT FP64 IPM with the restoration phase",
            "instances": len(grids), "status_counts": counts,
            "restoration_phases": int(r["resto_phases"].sum()),
            "iters_mean": float(r["iters"].mean()), "ms_per_batch": float(np.mean(ms)),
            "converged_per_s": float((r["status"] == 1).sum() / (np.mean(ms) / 1e3))}


def plain_measure(grids):
    """Single-problem GPU IPM (ipm_step loop, LiftedKKT FP64) on the given instances, one after
    another; time of the iterations (the per-problem symbolic analysis excluded, as for the
    batch)."""
    import torch
    import paper_2405_14236_gb300 as cp
    conv, t_tot, iters = 0, 0.0, []
    for g in grids:
        st = cp.IpmState(cp.Opf(g), kkt="lifted")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(MAX_ITER + 1):
            info = st.step()
            if info.status != 0:
                break
        t_tot += time.perf_counter() - t0
        conv += info.status == 1
        iters.append(info.k)
    return {"value": conv / t_tot, "unit": UNIT, "instances": len(grids), "converged": int(conv),
            "mean_iters": float(np.mean(iters)),
            "sample": "single-problem GPU IPM (one instance at a time) on alternating "
                      "1,000-bus scenarios and mixed grids of the batched workload"}


def run_gpu(args, rank, world, local_rank):
    import torch
    import paper_2405_14236_gb300 as cp
    from synth import batch_grids
    torch.cuda.set_device(local_rank)
    stream = torch.cuda.current_stream()
    # ---- instances of this GPU: weak scaling (one full set per GPU), or --split: one set split
    # across the GPUs by size (strong scaling; results gathered on the host)
    split = bool(args.split) and world > 1
    if split:
        from paper_2405_14236_gb300.shard import partition_by_cost
        all_grids = batch_grids(args.batch_scen, args.batch_mixed, part=0)
        share = partition_by_cost([2 * g.nb + 2 * g.ng for g in all_grids], world)[rank]
        grids = [all_grids[i] for i in share]
    else:
        grids = batch_grids(args.batch_scen, args.batch_mixed, part=rank)
    opfs = [cp.Opf(g) for g in grids]
    # supernode partition chosen by measurement (outside the timed steps, like the launch shapes)
    relax, sn_tune = (0, 0), None
    if args.relax:
        relax = tuple(int(v) for v in args.relax.split(","))
    elif not args.no_autotune and not args.launch_shape:
        from paper_2405_14236_gb300 import tune
        t0 = time.perf_counter()
        relax, recs = tune.supernode_shapes(opfs, kkt=args.kkt, gamma=1e6)
        sn_tune = {"relax": list(relax), "candidates": recs,
                   "tune_s": time.perf_counter() - t0}
    t0 = time.perf_counter()
    B = cp.Batch(opfs, relax=relax, kkt=args.kkt, gamma=1e6)
    torch.cuda.synchronize()
    init_s = time.perf_counter() - t0
    # launch shapes chosen by measurement (outside the timed steps, like the symbolic analyses)
    shape, autotune_s = None, 0.0
    if args.launch_shape:
        # a fixed launch shape (profiling): cluster size, "big" threshold numerator, denominator
        cl, num, den = (int(v) for v in args.launch_shape.split(","))
        nbig = B.set_shape(cl, num, den, 0)
        shape = {"cluster": cl, "threshold": num / den if den else None, "big_instances": nbig,
                 "fixed": True}
    elif not args.no_autotune:
        t0 = time.perf_counter()
        tune = B.autotune(sweeps=8)
        autotune_s = time.perf_counter() - t0
        best = tune["candidates"][tune["best"]]
        shape = {k: best[k] for k in ("cluster", "threshold", "blocks_per_instance")}
        shape["candidates"] = len(tune["candidates"])
    info = B.info()
    B.set_timing(True)
    for _ in range(args.warmup):
        B.reset()
        B.run(max_iter=MAX_ITER)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    clocks = ClockSampler(local_rank)
    clocks.start()
    time.sleep(0.3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step_ms, conv, iters_mean, iters_max, sweeps = [], [], [], [], []
    stopped, resto_phases, resto_iters = {}, [], []
    ks = {"solves": 0, "above": 0, "eta_max": 0.0}
    fact_ms = solve_ms = 0.0
    n_sw = 0
    nfac = 0
    w = B.work()
    fl_inst = w["factor_flops"] + w["condense_flops"]
    fl_tot = by_tot = 0.0
    l0 = cp.launch_count()
    for _ in range(args.steps):
        torch.cuda.synchronize()
        e0.record(stream)
        B.reset()
        B.run(max_iter=MAX_ITER)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
        r = B.results()
        kt = B.kernel_time()
        fact_ms += kt["fact_ms"]
        solve_ms += kt["solve_ms"]
        n_sw += kt["sweeps"]
        nfac += int(r["n_factor"].sum())
        fl_tot += float(np.sum(fl_inst * r["n_factor"]))
        by_tot += float(np.sum(w["bytes"] * r["n_factor"]))
        conv.append(int((r["status"] == 1).sum()))
        for code in r["status"][r["status"] != 1]:
            stopped[int(code)] = stopped.get(int(code), 0) + 1
        si = B.solve_info()
        for k in ("solves", "above"):
            ks[k] += int(si[k].sum())
        ks["eta_max"] = max(ks["eta_max"], float(si["eta_max"].max()))
        resto_phases.append(int(r["resto_phases"].sum()))
        resto_iters.append(int(r["resto_iters"].sum()))
        iters_mean.append(float(r["iters"].mean()))
        iters_max.append(int(r["iters"].max()))
        sweeps.append(int(r["sweeps"]))
    launches = cp.launch_count() - l0
    clk = clocks.stop()
    t_tot, tot_conv = aggregate_ranks(float(np.sum(step_ms)), float(np.sum(conv)), world, "cuda")
    value = tot_conv / (t_tot / 1e3)
    gathered = None
    if split:
        from paper_2405_14236_gb300.shard import gather_results
        r = B.results()
        gathered = gather_results({"status": r["status"], "obj": r["obj"]}, share,
                                  len(all_grids), world)
    # ---- e2e through the public API with host data: new loads for every scenario from host
    # memory, solve, every x back to host memory
    host_pd = [np.ascontiguousarray(g.pd, dtype=np.float64) for g in grids]
    host_qd = [np.ascontiguousarray(g.qd, dtype=np.float64) for g in grids]
    x_host = np.zeros(sum(o.n for o in opfs))
    n_e2e = max(2, args.steps // 3)
    e_ms, e_conv = 0.0, 0
    B.set_timing(False)
    for _ in range(n_e2e):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for o, pd, qd in zip(opfs, host_pd, host_qd):
            o.set_loads(pd, qd)
        B.reset()
        B.run(max_iter=MAX_ITER)
        B.x_all(x_host)
        e_ms += 1e3 * (time.perf_counter() - t0)
        e_conv += int((B.results()["status"] == 1).sum())
    h2d = int(sum(16 * g.nb for g in grids))
    d2h = int(8 * x_host.size)
    if rank != 0:
        return
    # ---- roofline of the dominant kernel: fused condensation + factorization (FP64 arithmetic,
    # latency-bound on these small supernodes): algorithmic FP64 flops per launch / its duration
    flops_all = float(np.sum(fl_inst))
    bytes_all = float(np.sum(w["bytes"]))
    # every factorization of every instance over the timed steps against the summed duration of
    # the factorization launches (two per sweep)
    launches_fact = 2 * max(n_sw, 1)
    fact_avg_ms = fact_ms / launches_fact
    ach_tf = fl_tot / (fact_ms / 1e3) / 1e12
    fl_per_fact = fl_tot
    by_per_fact = by_tot
    traffic = None
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    if os.path.exists(tfile):
        try:
            import hashlib
            tr = json.load(open(tfile))
            h = hashlib.sha256(open(os.path.join(ROOT, "paper_2405_14236_gb300", "csrc",
                                                  "batch.cu"), "rb").read()).hexdigest()[:16]
            if tr.get("batch_cu_sha") == h and tr.get("k_b_fact_inst_traffic_over_algorithmic"):
                # measured DRAM bytes / algorithmic bytes of a 40-instance launch, scaled to this
                # launch's algorithmic bytes (traffic grows with the instances factored)
                traffic = tr["k_b_fact_inst_traffic_over_algorithmic"] * by_per_fact / launches_fact
        except Exception:
            traffic = None
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": float(np.mean(step_ms)), "higher_is_better": True,
        "scaling": "strong" if split else "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args.kkt),
                   "instances": len(all_grids) if split else len(grids),
                   "patterns": info["patterns"],
                   "tol": 1e-6, "max_iter": MAX_ITER, "pool_bytes": info["device_bytes"],
                   "l2": "not flushed: the instance pool (%.2f GB) exceeds L2"
                         % (info["device_bytes"] / 1e9),
                   "parallelism": (f"split{world}: one instance set split by size across "
                                   "the GPUs" if split else
                                   f"dp{world}: one instance set per GPU" if world > 1
                                   else "single GPU")},
        "converged_per_step": conv, "instances_per_step": len(grids) * world if not split
        else len(all_grids),
        "gathered_converged": None if gathered is None else int((gathered["status"] == 1).sum()),
        "iters_mean": float(np.mean(iters_mean)),
        "iters_max": iters_max, "sweeps_per_step": sweeps,
        # statuses of the instances that did not converge, over all timed steps; feasibility
        # restoration phases entered and their iterations, per step
        "stopped_status_counts": {str(k): v for k, v in sorted(stopped.items())},
        "restoration": {"phases_per_step": resto_phases, "iters_per_step": resto_iters},
        # every KKT solve of the timed steps by the library's own backward error of the augmented
        # system: how many ended above 1e-10 after the refinement (the ill-conditioning of K_tau,
        # Sec. 3.2, in the middle iterations of LiftedKKT)
        "kkt_solves": {"per_step": ks["solves"] / args.steps,
                       "above_1e-10_share": ks["above"] / max(ks["solves"], 1),
                       "eta_max": ks["eta_max"]},
        "launches_per_sweep": B.info()["launches_per_sweep"], "init_s": init_s,
        "launch_shape": shape, "autotune_s": autotune_s, "supernode_shape": sn_tune,
        "roofline": {"kernel": "k_b_fact_inst (condensation + factorization, every instance)",
                     "bound": "alu", "achieved": ach_tf, "peak": FP64_PEAK_TFLOPS,
                     "unit": "TFLOP/s", "frac": ach_tf / FP64_PEAK_TFLOPS,
                     "peak_source": "FP64 from unit counts and the 2070 MHz clock",
                     "traffic": traffic,
                     "algorithmic_flops_per_launch": fl_per_fact / launches_fact,
                     "algorithmic_bytes_per_launch": by_per_fact / launches_fact,
                     "avg_launch_ms": fact_avg_ms, "factorizations": nfac},
        "kernels_ms_per_sweep": {"factor_both_rounds": fact_ms / max(n_sw, 1),
                                 "solve_first": solve_ms / max(n_sw, 1)},
        "factor": {"GB_s": by_tot / (fact_ms / 1e3) / 1e9,
                   "work_per_batch_factorization": {"flops": flops_all, "bytes": bytes_all}},
        "e2e": {"value": e_conv / (e_ms / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if not args.no_plain:
        ns = args.batch_scen
        line["plain"] = plain_measure([grids[i // 2] if i % 2 == 0 or ns == len(grids)
                                       else grids[ns + i // 2] for i in range(4)])
        line["plain"]["batched_speedup"] = value / line["plain"]["value"]
    if not args.no_fp32:
        line["batch_fp32"] = batch_form_measure(grids, kkt="lifted", precision=32, relax=relax)
    if not args.no_forms:
        # the other batched KKT forms on the same instances
        for form in ("lifted", "regularized", "hykkt"):
            if form != args.kkt:
                line[f"batch_{form}"] = batch_form_measure(grids, kkt=form, relax=relax)
    if not args.no_forms:
        line["batch_recipe"] = recipe_measure()
    if not args.no_warm:
        # LiftedKKT: a learned start from 640 points did not reduce the dual-regularized form's
        # iterations (37.7 vs 37.6 on 32 held-out scenarios), it cuts LiftedKKT's by ~40 %
        line["warm"] = warm_measure(kkt="lifted")
        if "plain" in line:
            line["warm"]["vs_plain"] = line["warm"]["warm"]["value"] / line["plain"]["value"]
    if not args.no_kkt:
        line["kkt10k"] = kkt_measure(args)
    if not args.no_ipm:
        line["ipm"] = ipm_measure()
        line["sweeps"] = sweep_measure()
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = cb = batch_cpu_baseline(kkt=args.kkt)
        # the oracle on all host cores next to the one-thread figure: context for the ratio
        line["vs_cpu"] = {"one_thread": value / cb["value"],
                          "all_cores": value / cb["pool"]["value"] if "pool" in cb else None,
                          "all_cores_n": cb.get("pool", {}).get("cores")}
        if "ipm" in line:
            cb["ipm"] = ipm_cpu_baseline(line["ipm"])
    print(json.dumps(line), flush=True)


def warm_measure(steps=6000, n_train=20000, n_test=1024, kkt="lifted"):
    """Learned warm start on load scenarios of the 1,000-bus grid: training points from the
    batched IPM at tolerance 1e-2 (seeds 10000..), the network trained by the library's own
    kernels, then held-out scenarios (seeds 30000..) solved to 1e-6 by the batched IPM from
    the cold start and from the predicted start (the prediction is inside the timed region)."""
    import torch
    import paper_2405_14236_gb300 as cp
    from paper_2405_14236_gb300 import warm
    from synth import config_grid, scale_loads
    base = config_grid("planar1k")
    train = [scale_loads(base, 10000 + k) for k in range(n_train)]
    test = [scale_loads(base, 30000 + k) for k in range(n_test)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    T, ok = warm.collect(train, tol=1e-2, kkt=kkt)
    torch.cuda.synchronize()
    t_collect = time.perf_counter() - t0
    keep = np.nonzero(ok)[0]
    X = warm.input_rows([train[i] for i in keep])
    Tk = T[torch.as_tensor(keep, device="cuda")].contiguous()
    del T
    t0 = time.perf_counter()
    model, losses = warm.train(X, Tk, steps=steps, batch=256, lr=1e-3, log_every=steps // 4)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del Tk
    opfs = [cp.Opf(g) for g in test]
    B = cp.Batch(opfs, kkt=kkt, gamma=1e6)
    Xt = warm.input_rows(test)
    B.run(max_iter=MAX_ITER)  # capture and warm-up
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    rec = {}
    for mode in ("cold", "warm"):
        ms, conv, its, itmax, used = [], [], [], [], 1.0
        for _ in range(3):
            torch.cuda.synchronize()
            e0.record(stream)
            B.reset()
            if mode == "warm":
                used = float(model.start(B, Xt).mean())
            B.run(max_iter=MAX_ITER)
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
            r = B.results()
            conv.append(int((r["status"] == 1).sum()))
            its.append(float(r["iters"].mean()))
            itmax.append(int(r["iters"].max()))
        rec[mode] = {"value": float(np.sum(conv) / (np.sum(ms) / 1e3)), "unit": UNIT,
                     "ms_per_batch": float(np.mean(ms)), "converged": conv,
                     "iters_mean": float(np.mean(its)), "iters_max": itmax, "obj": r["obj"].copy(),
                     "status": r["status"].copy()}
        if mode == "warm":
            rec[mode]["prediction_used"] = used
    # objectives compared over the instances that converged in both runs (the last run of each)
    ok = (rec["cold"]["status"] == 1) & (rec["warm"]["status"] == 1)
    oc, ow = rec["cold"]["obj"][ok], rec["warm"]["obj"][ok]
    rel = np.abs(ow - oc) / np.abs(oc)
    objrel = float(rel.max()) if ok.any() else None
    n_other = int((rel > 1e-6).sum())   # instances whose warm solve found another optimum
    for m in rec.values():
        del m["obj"]
        del m["status"]
    return {"workload": f"{n_test} held-out load scenarios of the 1,000-bus grid (seeds 30000..), "
                        f"batched {FORM_NAMES[kkt]} FP64 IPM to 1e-6",
            "cold": rec["cold"], "warm": rec["warm"],
            "speedup": rec["warm"]["value"] / rec["cold"]["value"],
            "obj_rel_diff_max": objrel, "obj_compared": int(ok.sum()),
            "distinct_optima": n_other,
            "training": {"points": int(len(keep)), "point_tolerance": 1e-2, "collect_s": t_collect,
                         "steps": steps, "batch": 256, "train_s": t_train,
                         "loss": losses, "net": [int(X.shape[1]), *warm.HIDDEN, int(model.tmean.shape[0])],
                         "params": int(model.net.nparams), "dtype": "bf16 weights, fp32 accumulate"}}


def sweep_measure():
    """gamma and tolerance sweeps on the 1,000-bus grid (the paper's experiments on gamma and on
    epsilon_tol): single-problem GPU IPM status, iterations, CG iterations, time, objective and
    the largest equality violation of the result."""
    import torch
    import paper_2405_14236_gb300 as cp
    from synth import config_grid
    from oracle.opf import OPFModel
    g = config_grid("planar1k")
    opf = cp.Opf(g)
    model = OPFModel(g)

    def run(**kw):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        r = cp.ipm_solve_opf(opf, max_iter=MAX_ITER, **kw)
        el = time.perf_counter() - t0
        gx, _ = model.cons(r["x"])
        return {"status": int(r["status"]), "iters": int(r["iters"]), "s": el,
                "cg_iters": int(sum(h["cg_iters"] for h in r["history"])),
                "gamma_last": float(r["history"][-1]["gamma"]), "obj": float(r["obj"]),
                "max_abs_g": float(np.abs(gx).max())}
    out = {"grid": "planar1k (1,000 buses)", "hykkt_gamma": {}, "regularized_gamma": {},
           "lifted_tol": {}}
    for gam in (1e4, 1e5, 1e6, 1e7, 1e8, 0.0):
        out["hykkt_gamma"]["auto" if gam == 0 else f"{gam:g}"] = run(kkt="hykkt", gamma=gam)
    for gam in (1e4, 1e6, 1e8, 0.0):
        out["regularized_gamma"]["auto" if gam == 0 else f"{gam:g}"] = run(kkt="regularized", gamma=gam)
    for tol in (1e-4, 1e-5, 1e-6, 1e-7, 1e-8):
        out["lifted_tol"][f"{tol:g}"] = run(kkt="lifted", tol=tol)
    return out


def ipm_measure():
    """Full IPM solves to the 1e-6 scaled KKT tolerance on the GPU (ipm_step loop); the oracle's
    time on the 1,000-bus problem is part of the CPU baseline (ipm_cpu_baseline)."""
    import torch
    import paper_2405_14236_gb300 as cp
    from synth import config_grid
    out = {}
    cases = [("planar1k", "lifted", 64), ("planar1k", "hykkt", 64), ("planar10k", "hykkt", 64),
             ("planar10k", "lifted", 64), ("planar1k", "lifted", 32), ("planar10k", "hykkt", 32),
             ("planar80k", "lifted", 64), ("planar80k", "hykkt", 32),
             ("planar10k-flow", "hykkt", 64), ("planar10k-flow", "lifted", 64),
             # the branch-flow formulation at 80,000 buses: n = 608,000 and m = 784,001, the size
             # of the paper's largest instance (78484epigrids: n = 674,562, m = 1,039,062)
             ("planar80k-flow", "hykkt", 64), ("planar80k-flow", "regularized", 64)]
    warm = cp.ipm_solve_opf(cp.Opf(config_grid("ring30")), kkt="hykkt")
    del warm
    for name, kkt, prec in cases:
        # "-flow": the flow-variable formulation (the shape of the paper's instances)
        g = config_grid(name.replace("-flow", ""))
        opf = cp.Opf(g, form="flow" if name.endswith("-flow") else "compact")
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        # the 80,000-bus cases are the large configuration: gamma = 1e7 (and, compact HyKKT, the
        # FP32 factor requested)
        gam = 1e7 if name.startswith("planar80k") else 1e6
        sizes = {"n": opf.n, "m_e": opf.m_e, "m_i": opf.m_i}
        st = cp.IpmState(opf, kkt=kkt, gamma=gam, precision=prec)
        torch.cuda.synchronize()
        t_init = time.perf_counter() - t0
        t0 = time.perf_counter()
        hist = []
        for _ in range(3001):
            info = st.step()
            hist.append(info)
            if info.status != 0:
                break
        t_solve = time.perf_counter() - t0
        rec = {"status": "converged" if hist[-1].status == 1 else f"status {hist[-1].status}",
               "iters": hist[-1].k, "obj": st.objective(), "init_s": t_init, "solve_s": t_solve,
               "ms_per_iter": 1e3 * t_solve / max(hist[-1].k, 1),
               "ipm_solves_per_s": 1.0 / t_solve,
               "factorizations": int(sum(h.n_factor for h in hist)),
               "cg_iters": int(sum(h.cg_iters for h in hist)),
               "fp32_iters": int(sum(1 for h in hist if h.precision == 32)), "gamma": gam,
               **sizes}
        if name.startswith("planar80k"):
            # per iteration: factor precision, delta_w and the backward error of the augmented
            # system that the library computed for the step's KKT solve (every one of these solves
            # is checked against the oracle's own evaluation in the GPU tests at this size)
            rec["per_iteration"] = [{"k": h.k, "precision": h.precision, "eta": h.eta,
                                     "delta_w": h.delta_w, "cg": h.cg_iters} for h in hist
                                    if h.status == 0]
        out[f"{name}-{kkt}" + ("-fp32" if prec == 32 else "")] = rec
    return out


def ipm_cpu_baseline(ipm):
    """The oracle IPM (one thread) on the 1,000-bus grid of the single-problem GPU legs, both
    forms, beside those legs' GPU solves (part of the CPU baseline)."""
    from synth import config_grid
    from oracle.opf import OPFModel
    from oracle import ipm as oipm
    out = {}
    for kkt in ("lifted", "hykkt"):
        t0 = time.perf_counter()
        r = oipm.solve(OPFModel(config_grid("planar1k")), oipm.Options(kkt=kkt, gamma=1e6))
        el = time.perf_counter() - t0
        rec = {"ipm_solves_per_s": 1.0 / el, "iters": r.iters, "obj": r.obj, "cores": 1,
               "status": r.status}
        gpu = ipm.get(f"planar1k-{kkt}")
        if gpu is not None:
            rec["gpu_obj_rel_diff"] = abs(gpu["obj"] - r.obj) / abs(r.obj)
        out[f"planar1k-{kkt}"] = rec
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-ipm", action="store_true", help="skip the full-IPM measurement")
    ap.add_argument("--no-fp32", action="store_true", help="skip the FP32-factor variant")
    ap.add_argument("--no-kkt", action="store_true", help="skip the 10k KKT-solve kernel line")
    ap.add_argument("--no-plain", action="store_true", help="skip the single-problem GPU IPM")
    ap.add_argument("--no-warm", action="store_true", help="skip the learned warm start")
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the default launch shapes of the batched kernels")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the other batched KKT forms (dual-regularized, HyKKT)")
    ap.add_argument("--kkt-only", action="store_true",
                    help="print only the 10k-bus KKT-solve leg (profiling)")
    ap.add_argument("--batch-scen", type=int, default=256,
                    help="load scenarios of the 1,000-bus grid in the batch (profiling: fewer)")
    ap.add_argument("--batch-mixed", type=int, default=64,
                    help="mixed grids of 118-2,000 buses in the batch (profiling: fewer)")
    ap.add_argument("--launch-shape", default="",
                    help="CL,NUM,DEN: fixed launch shape (clusters of CL blocks for instances above "
                         "NUM/DEN times the median supernode count) instead of the autotuner")
    ap.add_argument("--kkt", default="regularized", choices=["lifted", "regularized", "hykkt"],
                    help="KKT form of the headline batch (and of the oracle in the reference arm); "
                         "default: the dual-regularized condensed form, the fastest of the three "
                         "on this workload")
    ap.add_argument("--relax", default="",
                    help="W,DEN: fixed supernode relaxation (profiling) instead of the tuned one")
    ap.add_argument("--split", action="store_true",
                    help="N > 1: split one instance set across the GPUs by size (strong scaling) "
                         "instead of one set per GPU")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if args.kkt_only:
        print(json.dumps(kkt_measure(args)), flush=True)
        return
    if world > 1:
        import torch
        torch.cuda.set_device(local_rank)
        torch.distributed.init_process_group("nccl")
    run_gpu(args, rank, world, local_rank)
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
