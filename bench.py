"""Benchmark: BP3 (scalar Poisson, Gauss-Legendre q = p+2) FP64 Jacobi-PCG on
perturbed brick meshes of the unit cube, orders p = 1..8 (section
"Benchmarks"; throughput metric of the libCEED BP3 figures: DOFs x CG
iterations / s).

One step = for every order p in the sweep, a fixed number of graph-captured
Jacobi-PCG iterations (apply + vector updates + reductions, the whole hot
path) on that order's mesh of about --dofs global nodes.  `value` is the
aggregate GDOF/s = sum_p N_p * iterations / time, with every input resident
in HBM; `e2e` repeats it through the public API with the right-hand sides
copied from pinned host memory and the solutions copied back every step.

`--impl reference` times the FP64 CPU oracle (test infrastructure) on a
bounded sample of the same workload on the host cores.
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import fem_inputs  # noqa: E402

METRIC = "BP3 FP64 Jacobi-PCG throughput (DOFs x CG iterations / s), p=1..8 sweep"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--dofs", type=float, default=5e7)
    ap.add_argument("--orders", default="1-8")
    ap.add_argument("--iters", type=int, default=10, help="CG iterations per order per step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-graph", action="store_true",
                    help="host-driven CG loop (same kernels; for profilers)")
    ap.add_argument("--tts-dofs", type=float, default=1e7,
                    help="size of the time-to-1e-10 comparison (0 = skip)")
    ap.add_argument("--tts-order", type=int, default=4)
    ap.add_argument("--sections", default="bp56,suite,nsweep,batched,learned",
                    help="extra measured configurations: bp56, suite, nsweep, batched, learned"
                         " (comma list)")
    ap.add_argument("--bp56-n", type=int, default=44, help="elements per direction, BP5/BP6 p=7")
    ap.add_argument("--suite-order", type=int, default=4, help="order of the BP1-BP6 suite section")
    ap.add_argument("--suite-dofs", type=float, default=8e6, help="nodes of the BP1-BP6 suite mesh")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--learned-n", type=int, default=64, help="elements per direction, kappa BP3 p=4")
    ap.add_argument("--profile", default=None,
                    help="only time the apply of one operator, e.g. BP5:7:f32 (problem:order:prec"
                         "[:launch choice])"
                         " on a mesh of --dofs nodes, or PMG:4:f32 for p-multigrid V-cycles,"
                         " BATCH:256:8 for the persistent batch kernel;"
                         " for profilers")
    return ap.parse_args()


def orders(spec):
    if "-" in spec:
        a, b = spec.split("-")
        return list(range(int(a), int(b) + 1))
    return [int(s) for s in spec.split(",")]


def workload(args):
    ps = orders(args.orders)
    return [(p, fem_inputs.bp3_mesh_n(args.dofs, p)) for p in ps]


def algorithmic(p, n):
    """Per apply of BP3 (q = p+2): FP64 bytes that must move and flops."""
    P, q = p + 1, p + 2
    E = n ** 3
    N = (p * n + 1) ** 3
    bytes_ = 8 * N + 8 * N + 4 * E * P ** 3 + 8 * E * q ** 3 * 6
    flops = E * (2 * (2 * (q * P ** 3 + q * q * P * P + q ** 3 * P) + 6 * q ** 4) + 18 * q ** 3)
    return N, E, bytes_, flops


STENCIL_ORDERS = (1,)   # FP64 default body: the assembled 27-point stencil
ELMAT_ORDERS = (2,)     # FP64 default body: assembled element matrices


def stencil_bytes(N):
    """The assembled stencil: 26 double-word off-diagonal coefficients per
    row (the diagonal is implied by the zero row sums), x and y."""
    return 208 * N + 16 * N


def elmat_bytes(N, E, P3):
    return 16 * N + 4 * E * P3 + 8 * E * P3 * (P3 + 1) // 2


def body_algorithmic(p, n):
    """Per FP64 BP3 apply with the default body: bytes that must move and
    flops it executes (FMA = 2).  p >= 3, sum factorization: algorithmic().
    p = 2, element matrices: 16N (x, y) + 4 E P^3 (indices) + 8 E P^3
    (P^3 + 1) / 2 (the packed upper triangle of K_e), and 2 (P^3)^2 flops
    per element for y_e = K_e x_e (each off-diagonal entry used twice) plus
    2 P^3 for x.y.  p = 1, the assembled stencil of a lattice mesh: 208N
    (26 off-diagonal coefficients a row) + 16N (x, y), 26 differences and
    26 FMAs plus x.y: 3 * 26 + 2 flops a row."""
    N, E, by, fl = algorithmic(p, n)
    if p in STENCIL_ORDERS:
        by = stencil_bytes(N)
        fl = N * (3 * 26 + 2)
    elif p in ELMAT_ORDERS:
        P3 = (p + 1) ** 3
        by = elmat_bytes(N, E, P3)
        fl = E * (2 * P3 * P3 + 2 * P3)
    return N, E, by, fl


class Clocks:
    """nvidia-smi sampler during the timed region."""

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        self.proc = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        dev = os.environ.get("CUDA_VISIBLE_DEVICES", "0").split(",")[0]
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", dev, "--query-gpu=" + q, "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.f.flush(); self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# DRAM bytes of one FP64 BP3 apply per order, from one ncu capture
# (dram__bytes_read.sum, dram__bytes_write.sum) of `bench.py --profile
# BP3:<p>:f64 --dofs 4e6` on a B300: (E, N, read, write) of the captured mesh,
# with the default (double-word) body (at p = 1 both kernels of one apply:
# the split of x and the stencil).  The ratio to that body's algorithmic bytes
# (body_algorithmic) is steady across sizes (the bytes are qdata or element
# matrices, indices and the two vectors, all proportional to the mesh), so
# the full-size traffic is that ratio times the full-size algorithmic bytes.
APPLY_F64_DRAM = {
    1: (3944312, 4019679, 948003328, 5165312),
    2: (493039, 4019679, 1690484736, 74309632),
    3: (148877, 4096000, 1001539584, 34050816),
    4: (59319, 3869893, 711564288, 31769088),
    5: (32768, 4173281, 670284544, 32340992),
    6: (17576, 3869893, 617505792, 29090560),
    7: (12167, 4251528, 518869248, 29997824),
    8: (8000, 4173281, 494480128, 157703680),
}


def dram_ratio(p):
    """Measured DRAM bytes over the default body's algorithmic bytes, or None
    when no capture of the current body exists."""
    if APPLY_F64_DRAM.get(p) is None:
        return None
    E, N, rd, wr = APPLY_F64_DRAM[p]
    P, q = p + 1, p + 2
    if p in STENCIL_ORDERS:
        alg = stencil_bytes(N)
    elif p in ELMAT_ORDERS:
        alg = elmat_bytes(N, E, P ** 3)
    else:
        alg = 16 * N + 4 * E * P ** 3 + 48 * E * q ** 3
    return (rd + wr) / alg


def cpu_baseline(work, iters, seconds, seed=0):
    """Oracle (brute-force FP64 apply, as it stands) on a bounded sample of
    elements of every order's mesh; extrapolated to the step's DOF-iterations."""
    import oracle
    cores = len(os.sched_getaffinity(0))
    total_dof_it, total_t, sample = 0.0, 0.0, []
    per = seconds / len(work)
    for p, n in work:
        N, E, _, _ = algorithmic(p, n)
        # a small mesh of the same order and element shape; time elements until `per` s
        m = fem_inputs.box_mesh(min(n, 6), p, perturb=0.1, seed=seed)
        op = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, p + 2, nthreads=cores)
        x = fem_inputs.rhs_uniform(m["N"], None, seed=seed)
        ne, t = 0, 0.0
        chunk = m["E"]
        while t < per:
            t0 = time.perf_counter()
            op.apply(x)
            t += time.perf_counter() - t0
            ne += chunk
        t_elem = t / ne
        total_t += t_elem * E * iters
        total_dof_it += N * iters
        sample.append("p=%d: %d elements in %.1fs" % (p, ne, t))
    # the same oracle with its element matrices computed once and kept
    # (batched dense products): the rate where they fit in memory
    cached_t, cached_dof_it = 0.0, 0.0
    for p, n in work:
        if p > 6:
            continue
        N, E, _, _ = algorithmic(p, n)
        m = fem_inputs.box_mesh(3, p, perturb=0.1, seed=seed)
        op = oracle.Operator(m, oracle.DIFFUSION, oracle.GAUSS, p + 2, nthreads=cores)
        K = np.stack([op.element_matrix(e) for e in range(m["E"])])
        en = m["elem_nodes"]
        x = fem_inputs.rhs_uniform(m["N"], None, seed=seed)
        reps, t = 0, 0.0
        while t < min(1.0, per):
            t0 = time.perf_counter()
            y = np.zeros(m["N"])
            np.add.at(y, en, np.matmul(K, x[en][..., None])[..., 0])
            t += time.perf_counter() - t0
            reps += 1
        cached_t += t / (reps * m["E"]) * E * iters
        cached_dof_it += N * iters
    model = "unknown"
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                model = line.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    return {"value": total_dof_it / total_t / 1e9, "unit": "GDOF/s", "cores": cores,
            "kind": "oracle", "cpu_model": model,
            "cached_element_matrices_gdofs": (cached_dof_it / cached_t / 1e9) if cached_t else None,
            "sample": "; ".join(sample) +
            " (brute-force element apply, extrapolated to every element x iterations;"
            " cached_element_matrices_gdofs: the same with stored K_e, p <= 6)"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    work = workload(args)
    base = cpu_baseline(work, args.iters, max(2.0, args.cpu_seconds / 3))
    steps = []
    for s in range(args.warmup + args.steps):
        b = cpu_baseline(work, args.iters, max(1.0, args.cpu_seconds / 5), seed=s)
        if s >= args.warmup:
            steps.append(b["value"])
    val = float(np.median(steps))
    N_tot = sum(algorithmic(p, n)[0] for p, n in work)
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GDOF/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": N_tot * args.iters / (val * 1e9) * 1e3,
            "extrapolated": True,
            "extrapolation_note": "value and ms_per_step are extrapolated, not timed over a whole"
                                  " step: each step times the oracle's brute-force element apply"
                                  " on a bounded sample of every order's elements (the sample"
                                  " field) and scales that rate to the step's DOF-iterations;"
                                  " a whole step would take hours on the host",
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, work),
            "cpu_baseline": dict(base, value=val),
            "e2e": {"value": val, "unit": "GDOF/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


def time_to_solution(fem, torch, args):
    """BP3 at one order: wall time to ||b - A x|| <= 1e-10 ||b|| (true FP64
    residual) for plain FP64 Jacobi-PCG, for FP32 inner PCG + FP64 iterative
    refinement, and for flexible CG with a p-multigrid V-cycle (orders p,
    p/2, ..., 1 on the same elements; V-cycle in FP64 or FP32; the FP32
    V-cycle also inside FP32 flexible CG with FP64 refinement), same mesh,
    same right-hand side, same GPU.  The multigrid set-up (coarse operators,
    lmax estimates) is timed separately."""
    p = args.tts_order
    n = fem_inputs.bp3_mesh_n(args.tts_dofs, p)
    orders = [p]
    while orders[-1] > 1:
        orders.append(max(1, orders[-1] // 2))
    meshes = [fem_inputs.box_mesh(n, q, perturb=0.1, seed=300 + p) for q in orders]
    m = meshes[0]
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, "BP3", prec=fem.F32)
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=400 + p)).cuda()
    out = {"problem": "BP3 p=%d n=%d N=%d" % (p, n, m["N"]), "rtol": 1e-10,
           "pmg_orders": orders}
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    # coarse levels rediscretized with Gauss q = p + 1 (exact for affine
    # bricks; 7 % faster V-cycles than q = p + 2 at the same iteration count)
    coarse = [fem.Operator(fem.Mesh(mm), fem.DIFFUSION, fem.GAUSS, mm["p"] + 1, prec=fem.F32)
              for mm in meshes[1:]]
    pmg = {"fp64_pmg_fcg": fem.Pmg([op] + coarse, prec=fem.F64),
           "fp32_pmg_fcg": fem.Pmg([op] + coarse, prec=fem.F32)}
    torch.cuda.synchronize()
    out["pmg_setup_seconds"] = time.perf_counter() - t0
    del meshes, m
    res = {}
    for name in ("fp64_pcg", "fp32_refined", "fp64_pmg_fcg", "fp32_pmg_fcg", "fp32_pmg_refined_fcg"):
        best = None
        for rep in range(2):  # first run builds the graphs
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if name == "fp64_pcg":
                st = op.cg(b, x, precond=fem.PC_JACOBI, rtol=1e-10, maxit=100000)
            elif name == "fp32_refined":
                st = op.solve_refined(b, x, rtol=1e-10, inner_rtol=0.1)
            elif name == "fp32_pmg_refined_fcg":
                # FP32 flexible CG around the FP32 V-cycle inside FP64
                # refinement: the FP64 apply once per refinement step
                st = pmg["fp32_pmg_fcg"].solve_refined(b, x, rtol=1e-10, inner_rtol=1e-6)
            else:
                st = pmg[name].solve(b, x, rtol=1e-10)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            best = t if best is None else min(best, t)
        # true FP64 residual of the returned x, by the FP64 apply
        y = op.apply(x)
        r = (b - y)
        r[torch.from_numpy(gm.dirichlet.astype(bool)).cuda()] = 0.0
        true_rel = (torch.linalg.norm(r) / torch.linalg.norm(b)).item()
        res[name] = {"seconds": best, "iterations": st["iterations"], "outer": st["outer"],
                     "status": st["status"], "true_rel_residual": true_rel}
    res["speedup_refined_vs_fp64"] = res["fp64_pcg"]["seconds"] / res["fp32_refined"]["seconds"]
    res["speedup_fp32_pmg_vs_fp64"] = res["fp64_pcg"]["seconds"] / res["fp32_pmg_fcg"]["seconds"]
    res["speedup_fp32_pmg_refined_vs_fp64"] = (res["fp64_pcg"]["seconds"] /
                                               res["fp32_pmg_refined_fcg"]["seconds"])
    out.update(res)
    return out


def _events():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _time_apply(torch, fn, reps=5, warm=3):
    for _ in range(warm):
        fn()
    a0, a1 = _events()
    a0.record()
    for _ in range(reps):
        fn()
    a1.record()
    torch.cuda.synchronize()
    return a0.elapsed_time(a1) / reps * 1e-3


def section_bp56(fem, torch, args):
    """BP5 (scalar) and BP6 (3 components) diffusion, Gauss-Lobatto q=p+1,
    p=7: FP64 and FP32 apply throughput with the FP32 kernel's HBM roofline,
    FP32 apply error against the FP64 oracle on sampled rows, and the time to
    a 1e-10 FP64 residual of plain FP64 PCG vs FP32 PCG + FP64 refinement."""
    import oracle
    p, n = 7, args.bp56_n
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=500)
    gm = fem.Mesh(m)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs", 6400.0)
    out = {"mesh": "p=7 n=%d N=%d per component" % (n, m["N"])}
    rows = np.random.default_rng(5).choice(m["N"], 200, replace=False)
    rows = rows[m["dirichlet"][rows] == 0]
    ptr, rel_el = fem_inputs.elements_of_nodes(m, rows)
    orc = oracle.Operator(m, oracle.DIFFUSION, oracle.LOBATTO, p + 1)
    for name in ("BP5", "BP6"):
        op = fem.Operator.bake_off(gm, name, prec=fem.F32)
        nc = op.ncomp
        N, E = m["N"], m["E"]
        x = torch.from_numpy(np.random.default_rng(1).uniform(-1, 1, nc * N)).cuda()
        y = torch.empty_like(x)
        x32, y32 = x.float(), torch.empty(nc * N, dtype=torch.float32, device="cuda")
        t64 = _time_apply(torch, lambda: op.apply(x, y))
        t32 = _time_apply(torch, lambda: op.apply_f32(x32, y32))
        P, q = p + 1, p + 1
        by64 = nc * 16 * N + 4 * E * P ** 3 + 48 * E * q ** 3
        by32 = nc * 8 * N + 4 * E * P ** 3 + 24 * E * q ** 3
        fl = nc * E * (12 * P ** 4 + 18 * P ** 3)
        # sampled-row error of the FP32 apply (component 0) against the oracle
        ys = y32[:N].double().cpu().numpy()[rows]
        yr = orc.apply_rows(x[:N].cpu().numpy(), rows, ptr, rel_el)
        err32 = float(np.linalg.norm(ys - yr) / np.linalg.norm(yr))
        b = torch.from_numpy(fem_inputs.rhs_uniform(N, m["dirichlet"], seed=600, ncomp=nc)).cuda()
        tts = {}
        for meth in ("fp64_pcg", "fp32_refined"):
            best = None
            for _ in range(2):
                xs = torch.zeros_like(b)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = (op.cg(b, xs, rtol=1e-10) if meth == "fp64_pcg"
                      else op.solve_refined(b, xs, rtol=1e-10, inner_rtol=0.1))
                torch.cuda.synchronize()
                t = time.perf_counter() - t0
                best = t if best is None else min(best, t)
            r = op.residual(b, xs)
            tts[meth] = {"seconds": best, "iterations": st["iterations"],
                         "true_rel_residual": (torch.linalg.norm(r) / torch.linalg.norm(b)).item()}
        out[name] = {
            "dofs": nc * N,
            "apply_f64": {"ms": t64 * 1e3, "gdofs": nc * N / t64 / 1e9, "tflops": fl / t64 / 1e12},
            "apply_f32": {"ms": t32 * 1e3, "gdofs": nc * N / t32 / 1e9,
                          "hbm_gbs": by32 / t32 / 1e9, "hbm_frac_of_measured": by32 / t32 / 1e9 / hbm,
                          "algorithmic_bytes": by32, "tflops": fl / t32 / 1e12},
            "apply_f32_rel_error_vs_oracle": err32,
            "time_to_1e-10": tts,
            "speedup_refined_vs_fp64": tts["fp64_pcg"]["seconds"] / tts["fp32_refined"]["seconds"]}
        del op, x, y, x32, y32, b
    return out


def section_nsweep(fem, torch, args):
    """Throughput against problem size (the paper's throughput-vs-time plots
    of the BP3 runs): FP64 Jacobi-PCG iterations (graph-captured, 20 per
    measurement) on BP3 meshes of 1e4 .. 3e7 DOFs at p = 2, 4, 8; per size
    the time per iteration and DOFs x iterations / s, and per order n_0.8,
    the smallest size reaching 80 % of that order's best rate."""
    out = {}
    targets = [1e4, 3e4, 1e5, 3e5, 1e6, 3e6, 1e7, 3e7]
    iters = 20
    for p in (2, 4, 8):
        rows = []
        for t in targets:
            n = max(1, fem_inputs.bp3_mesh_n(t, p))
            m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=710 + p)
            op = fem.Operator.bake_off(fem.Mesh(m), "BP3")
            b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=711)).cuda()
            x = torch.zeros_like(b)
            op.cg(b, x, precond=fem.PC_JACOBI, maxit=iters, rtol=0.0,
                  zero_guess=True)   # builds the graph
            best = None
            for _ in range(3):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                st = op.cg(b, x, precond=fem.PC_JACOBI, maxit=iters, rtol=0.0, zero_guess=True)
                torch.cuda.synchronize()
                dt = time.perf_counter() - t0
                best = dt if best is None else min(best, dt)
            rows.append({"dofs": m["N"], "seconds_per_iteration": best / st["iterations"],
                         "gdofs": m["N"] * st["iterations"] / best / 1e9})
            del op, m, b, x
        peak = max(r["gdofs"] for r in rows)
        n08 = min((r["dofs"] for r in rows if r["gdofs"] >= 0.8 * peak), default=None)
        out["p%d" % p] = {"points": rows, "best_gdofs": peak, "n_0.8_dofs": n08}
    return out


def section_suite(fem, torch, args):
    """All six bake-off problems (BP1/BP2 mass, BP3/BP4 diffusion with Gauss
    q = p+2, BP5/BP6 diffusion on the Gauss-Lobatto points; odd = scalar,
    even = 3 components) on one mesh at one order: FP64 and FP32 apply
    throughput and the FP64 CG iteration rate (graph-captured, 20 iterations;
    no preconditioner for the mass problems, Jacobi for the others)."""
    p = args.suite_order
    n = fem_inputs.bp3_mesh_n(args.suite_dofs, p)
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=700)
    gm = fem.Mesh(m)
    N, E = m["N"], m["E"]
    hbm = measured_peaks().get("hbm_gbs", 6400.0)
    out = {"mesh": "p=%d n=%d N=%d nodes" % (p, n, N)}
    iters = 20
    for name in ("BP1", "BP2", "BP3", "BP4", "BP5", "BP6"):
        kind, nc, quad, dq = fem.BAKE_OFF[name]
        op = fem.Operator.bake_off(gm, name, prec=fem.F32)
        P, q = p + 1, p + dq
        nd = 1 if kind == fem.MASS else 6
        x = torch.from_numpy(np.random.default_rng(2).uniform(-1, 1, nc * N)).cuda()
        y = torch.empty_like(x)
        x32, y32 = x.float(), torch.empty(nc * N, dtype=torch.float32, device="cuda")
        t64 = _time_apply(torch, lambda: op.apply(x, y))
        t32 = _time_apply(torch, lambda: op.apply_f32(x32, y32))
        by64 = nc * 16 * N + 4 * E * P ** 3 + 8 * nd * E * q ** 3
        by32 = nc * 8 * N + 4 * E * P ** 3 + 4 * nd * E * q ** 3
        b = torch.from_numpy(fem_inputs.rhs_uniform(N, m["dirichlet"], seed=701, ncomp=nc)).cuda()
        pc = fem.PC_NONE if kind == fem.MASS else fem.PC_JACOBI
        xs = torch.zeros_like(b)
        op.cg(b, xs, precond=pc, maxit=iters, rtol=0.0)   # builds the graph
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        xs.zero_()
        st = op.cg(b, xs, precond=pc, maxit=iters, rtol=0.0)
        torch.cuda.synchronize()
        tcg = time.perf_counter() - t0
        out[name] = {"dofs": nc * N, "q": q,
                     "apply_f64": {"ms": t64 * 1e3, "gdofs": nc * N / t64 / 1e9,
                                   "hbm_gbs": by64 / t64 / 1e9},
                     "apply_f32": {"ms": t32 * 1e3, "gdofs": nc * N / t32 / 1e9,
                                   "hbm_gbs": by32 / t32 / 1e9,
                                   "hbm_frac_of_measured": by32 / t32 / 1e9 / hbm},
                     "cg_f64_gdofs_per_iteration": nc * N * st["iterations"] / tcg / 1e9}
        del op, x, y, x32, y32, b, xs
    return out


def _batched_mix(fem, torch, specs):
    """One batch of independent BP3 problems: FP32 operators with FP64
    refinement; problems of at least 2^21 unknowns solved alone with their
    order-specialized kernels, the inner iterations of all others in one
    persistent kernel per outer step (autotuned block shape); vs the same
    problems solved one after another with fem_solve_refined (graphs warmed
    first)."""
    probs = []
    for s_ in specs:
        m = fem_inputs.box_mesh(s_["n"], s_["p"], perturb=0.1, seed=s_["mesh_seed"])
        gm = fem.Mesh(m)
        op = fem.Operator.bake_off(gm, "BP3", prec=fem.F32)
        b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"],
                                                    seed=s_["rhs_seed"])).cuda()
        probs.append((gm, op, b))
    batch = fem.Batch([q[1] for q in probs])
    bs = [q[2] for q in probs]
    t0 = time.perf_counter()
    tune = batch.autotune(bs, [torch.zeros_like(b) for b in bs], iters=10)
    t_tune = time.perf_counter() - t0
    res = None
    best = None
    for _ in range(2):
        xs = [torch.zeros_like(b) for b in bs]
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = batch.solve(bs, xs, rtol=1e-10, inner_rtol=0.1)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        best = t if best is None else min(best, t)
    worst = max(r["true_rel"] for r in res)
    dof_it = sum(q[1].N * r["iterations"] for q, r in zip(probs, res))
    seq = 0.0
    for gm, op, b in probs:
        x = torch.zeros_like(b)
        op.solve_refined(b, x, rtol=1e-10, inner_rtol=0.1)  # warm graphs
        x.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        op.solve_refined(b, x, rtol=1e-10, inner_rtol=0.1)
        torch.cuda.synchronize()
        seq += time.perf_counter() - t0
    return {"problems": len(probs), "total_dofs": sum(q[1].N for q in probs),
            "orders": sorted(set(s_["p"] for s_ in specs)),
            "sizes_n": [min(s_["n"] for s_ in specs), max(s_["n"] for s_ in specs)],
            "seconds": best, "gdofs_per_cg_iteration": dof_it / best / 1e9,
            "max_true_rel_residual": worst, "all_converged": all(r["status"] == "FEM_OK" for r in res),
            "autotune": dict(tune, seconds=t_tune),
            "solo_dofs": batch.solo_dofs, "solo_problems": len(batch.solo),
            "solo_share_of_dofs": sum(probs[i][1].N for i in batch.solo) / sum(q[1].N for q in probs),
            "sequential_refined_seconds": seq, "speedup_vs_sequential": seq / best}


def section_batched(fem, torch, args):
    """Two batches: the bake-off mix (64 BP3 problems, n in 4..32, p in 2..8,
    seed 7: total work dominated by a few large high-order problems) and a
    small-problem mix (256 problems, n in 2..8, p in 1..4, seed 8: each
    solve alone is bound by launch and iteration latency)."""
    return {"bake_off_mix": _batched_mix(fem, torch, fem_inputs.batch_problems(args.batch_count, seed=7)),
            "small_mix": _batched_mix(fem, torch, fem_inputs.batch_problems(
                4 * args.batch_count, seed=8, nmin=2, nmax=8, pmin=1, pmax=4))}


def section_learned(fem, torch, args):
    """BP3 with kappa(x) = exp(Gaussian random field, l = 0.1, sigma = 1),
    p=4, n^3 hexes: train the per-element network on Jacobi-PCG
    residual/error pairs (GPU kernels), calibrate its weight, then time to a
    1e-10 FP64 residual: plain FP64 Jacobi-PCG, FP32+FP64-refinement
    Jacobi-PCG, and FP32 flexible CG with the learned preconditioner inside
    FP64 refinement."""
    p, n = 4, args.learned_n
    rff = fem_inputs.rff_params(1024, 0.1, seed=77)
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=78)
    gm = fem.Mesh(m)
    t0 = time.perf_counter()
    op = fem.Operator.bake_off(gm, "BP3", prec=fem.F32, rff=rff)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    P3 = (p + 1) ** 3
    n_in, n_h, n_out = 160, 256, 128
    net = fem.Mlp(n_in, n_h, n_out, fem_inputs.mlp_init(n_in, n_h, n_out, seed=79), mode=0)
    pc = fem.Precond(op, net)
    ks = (5, 20, 80)
    nrhs = 2
    E = m["E"]
    X = torch.zeros(nrhs * len(ks) * E, n_in, dtype=torch.bfloat16, device="cuda")
    T = torch.zeros(nrhs * len(ks) * E, n_out, dtype=torch.float32, device="cuda")
    t0 = time.perf_counter()
    r0 = 0
    for j in range(nrhs):
        b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=800 + j)).cuda()
        xs = torch.zeros_like(b)
        op.solve_refined(b, xs, rtol=1e-11, inner_rtol=1e-5)
        for k in ks:
            xk = torch.zeros_like(b)
            op.cg(b, xk, maxit=k, rtol=0.0)
            pc.samples(b, xs, xk, X[r0:r0 + E], T[r0:r0 + E])
            r0 += E
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    t0 = time.perf_counter()
    # the network learns e_e / (s ||r_e||): targets normalized by their RMS s
    # (the raw targets are of order 1e4), trained until the loss stops falling
    t_scale = torch.sqrt(torch.mean(T[:, :P3].double() ** 2)).item()
    T /= t_scale
    losses = net.train_plateau(X, T, P3, max_epochs=200, chunk=4, rel_tol=0.01, batch=4096,
                               lr=1e-3, seed=1)
    t_train = time.perf_counter() - t0
    del X, T
    bval = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=898)).cuda()
    gamma = pc.calibrate(bval, gammas=[t_scale * g for g in (2.0, 1.0, 0.5, 0.25, 0.1)] + [0.0],
                         probe_iters=64)
    b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=899)).cuda()
    res = {}
    for meth in ("fp64_jacobi_pcg", "fp32_refined_jacobi", "fp32_refined_learned_fcg",
                 "fp32_refined_jacobi_fcg"):
        best = None
        for _ in range(2):
            x = torch.zeros_like(b)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if meth == "fp64_jacobi_pcg":
                st = op.cg(b, x, rtol=1e-10)
            elif meth == "fp32_refined_jacobi":
                st = op.solve_refined(b, x, rtol=1e-10, inner_rtol=0.1)
            elif meth == "fp32_refined_learned_fcg":
                st = pc.fcg(b, x, rtol=1e-10)
            else:
                st = fem.Precond(op, None).fcg(b, x, rtol=1e-10)
            torch.cuda.synchronize()
            t = time.perf_counter() - t0
            best = t if best is None else min(best, t)
        r = op.residual(b, x)
        res[meth] = {"seconds": best, "iterations": st["iterations"],
                     "fallback": st.get("fallback", 0),
                     "true_rel_residual": (torch.linalg.norm(r) / torch.linalg.norm(b)).item()}
    return {"problem": "kappa BP3 p=%d n=%d N=%d" % (p, n, m["N"]), "setup_seconds": t_setup,
            "training": {"samples": nrhs * len(ks) * E, "data_seconds": t_data,
                         "train_seconds": t_train, "epochs": len(losses),
                         "target_scale": t_scale,
                         "loss_first_epoch": float(losses[0]), "loss_last_epoch": float(losses[-1]),
                         "loss_every_10_epochs": [float(v) for v in losses[::10]],
                         "loss_of_zero_prediction": float(P3),
                         "loss_note": "mean over rows of the squared error summed over the P^3"
                                      " outputs, targets normalized to unit RMS (predicting zero"
                                      " scores P^3); training stops when 4 epochs gain < 1 %"
                                      " or after 200 epochs",
                         "calibrated_gamma": gamma,
                         "calibrated_gamma_over_scale": gamma / t_scale},
            "time_to_1e-10": res,
            "learned_vs_fp64_speedup": res["fp64_jacobi_pcg"]["seconds"] / res["fp32_refined_learned_fcg"]["seconds"],
            "learned_vs_jacobi_fcg_iterations": res["fp32_refined_jacobi_fcg"]["iterations"] / max(1, res["fp32_refined_learned_fcg"]["iterations"])}


def config(args, work):
    return {"workload": "BP3 FP64 Jacobi-PCG, Gauss-Legendre q=p+2, perturbed unit-cube "
                        "brick meshes of about %.0e DOFs per order" % args.dofs,
            "orders": [p for p, _ in work], "elements_per_dim": [n for _, n in work],
            "dofs": [algorithmic(p, n)[0] for p, n in work],
            "cg_iterations_per_order": args.iters, "parallelism": "replicas",
            "l2": "inputs larger than L2 (no flush needed)"}


def run_profile(args):
    """Apply of one operator, --warmup + --steps launches, timed with events."""
    import torch
    from paper_2109_04996_b300 import build as fembuild
    fembuild.build()
    import paper_2109_04996_b300 as fem
    if args.profile.startswith("MLP:"):
        # forward of the per-element network on `rows` element rows (the
        # learned preconditioner's inference): MLP:n_in:n_h:n_out:rows
        n_in, n_h, n_out, rows = (int(v) for v in args.profile.split(":")[1:])
        net = fem.Mlp(n_in, n_h, n_out, fem_inputs.mlp_init(n_in, n_h, n_out, seed=1), mode=0)
        X = torch.from_numpy(np.random.default_rng(0).normal(0, 1, (rows, n_in))).to(
            net.input_dtype).cuda()
        for _ in range(args.warmup):
            net.forward(X)
        e0, e1 = _events()
        e0.record()
        for _ in range(args.steps):
            net.forward(X)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        flops = 2.0 * rows * (n_in * n_h + n_h * n_h + n_h * n_out)
        print(json.dumps({"profile": args.profile, "ms_per_forward": ms,
                          "tflops": flops / ms / 1e9}))
        return
    if args.profile.startswith("BATCH:"):
        # the persistent batch kernel on the small-problem mix (count problems,
        # n in 2..8, p in 1..4, seed): the autotuner launches it from the host,
        # once per shape (block size 128, 256, 512 x blocks per SM 1, 2, max),
        # each launch running --steps inner iterations of every problem
        count, seed = (int(v) for v in args.profile.split(":")[1:])
        specs = fem_inputs.batch_problems(count, seed=seed, nmin=2, nmax=8, pmin=1, pmax=4)
        ops, bs = [], []
        for s_ in specs:
            m = fem_inputs.box_mesh(s_["n"], s_["p"], perturb=0.1, seed=s_["mesh_seed"])
            ops.append(fem.Operator.bake_off(fem.Mesh(m), "BP3", prec=fem.F32))
            bs.append(torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"],
                                                              seed=s_["rhs_seed"])).cuda())
        batch = fem.Batch(ops)
        r = batch.autotune(bs, [torch.zeros_like(b) for b in bs], iters=args.steps)
        print(json.dumps({"profile": args.profile, "problems": count,
                          "dofs": sum(o.n for o in ops), "tune": r}))
        return
    fields = args.profile.split(":")
    name, p, prec = fields[:3]
    choice = int(fields[3]) if len(fields) > 3 else None   # launch choice (default: the operator's)
    p = int(p)
    n = fem_inputs.bp3_mesh_n(args.dofs, p)
    if name == "PMG":
        # one p-multigrid V-cycle (BP3 levels p, p/2, ..., 1) per step
        orders = [p]
        while orders[-1] > 1:
            orders.append(max(1, orders[-1] // 2))
        meshes = [fem_inputs.box_mesh(n, q, perturb=0.1, seed=900) for q in orders]
        ops = [fem.Operator(fem.Mesh(mm), fem.DIFFUSION, fem.GAUSS, mm["p"] + (2 if l == 0 else 1),
                            prec=fem.F32) for l, mm in enumerate(meshes)]
        pm = fem.Pmg(ops, prec=fem.F32 if prec == "f32" else fem.F64)
        N = meshes[0]["N"]
        r = torch.from_numpy(np.where(meshes[0]["dirichlet"] == 0,
                                      np.random.default_rng(0).uniform(-1, 1, N), 0.0)).cuda()
        for _ in range(args.warmup):
            pm.vcycle(r)
        e0, e1 = _events()
        e0.record()
        for _ in range(args.steps):
            pm.vcycle(r)
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        print(json.dumps({"profile": args.profile, "N": N, "E": meshes[0]["E"], "n": n,
                          "orders": orders, "ms_per_vcycle": ms}))
        return
    m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=900)
    gm = fem.Mesh(m)
    op = fem.Operator.bake_off(gm, name, prec=fem.F32)
    if choice is not None:
        op.set_launch_shape(fem.F32 if prec == "f32" else fem.F64, choice, 0)
    nc = op.ncomp
    x = torch.from_numpy(np.random.default_rng(0).uniform(-1, 1, nc * m["N"])).cuda()
    if prec == "f32":
        x = x.float()
        fn = lambda y: op.apply_f32(x, y)
    else:
        fn = lambda y: op.apply(x, y)
    y = torch.empty_like(x)
    for _ in range(args.warmup):
        fn(y)
    e0, e1 = _events()
    e0.record()
    for _ in range(args.steps):
        fn(y)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    print(json.dumps({"profile": args.profile, "N": m["N"], "E": m["E"], "n": n,
                      "ms_per_apply": ms, "gdofs": nc * m["N"] / ms / 1e6}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.profile:
        run_profile(args)
        return
    import torch
    import torch.distributed as dist
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    from paper_2109_04996_b300 import build as fembuild
    if world == 1 or local == 0:
        fembuild.build()      # one rank per node builds (when stale), the others wait
    if world > 1:
        dist.barrier()
    import paper_2109_04996_b300 as fem

    work = workload(args)
    stream = torch.cuda.current_stream()
    ops = []
    for p, n in work:
        m = fem_inputs.box_mesh(n, p, perturb=0.1, seed=100 + p)
        gm = fem.Mesh(m, stream=stream)
        op = fem.Operator.bake_off(gm, "BP3")
        b = torch.from_numpy(fem_inputs.rhs_uniform(m["N"], m["dirichlet"], seed=200 + p)).cuda()
        x = torch.zeros_like(b)
        ops.append((p, n, gm, op, b, x))
        del m
    torch.cuda.synchronize()

    def step():
        for p, n, gm, op, b, x in ops:
            # x0 = 0 (the initial residual is b, no apply spent on it)
            st = op.cg(b, x, precond=fem.PC_JACOBI, maxit=args.iters, rtol=0.0,
                       use_graph=not args.no_graph, zero_guess=True)
            assert st["iterations"] == args.iters, st

    for _ in range(args.warmup):
        step()
    clk = Clocks()
    clk.start()
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    if world > 1:
        t = torch.tensor([ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = t.item()
        dist.barrier()
    clocks = clk.stop()
    dof_it = sum(algorithmic(p, n)[0] for p, n in work) * args.iters
    value = dof_it * world / (ms * 1e-3) / 1e9

    # end to end through the public API: pinned host RHS in, solution out, every step
    hb = [torch.empty(b.numel(), dtype=torch.float64, pin_memory=True).copy_(b.cpu())
          for (_, _, _, _, b, _) in ops]
    hx = [torch.empty(b.numel(), dtype=torch.float64, pin_memory=True)
          for (_, _, _, _, b, _) in ops]

    # the copies run on their own stream: order k+1's right-hand side goes
    # in and order k-1's solution comes out while order k solves (every copy
    # stays inside the timed region)
    cstream = torch.cuda.Stream()
    ev_in = [torch.cuda.Event() for _ in ops]
    ev_out = [torch.cuda.Event() for _ in ops]

    def put_rhs(k):
        with torch.cuda.stream(cstream):
            ops[k][4].copy_(hb[k], non_blocking=True)
            ev_in[k].record(cstream)

    def step_e2e():
        put_rhs(0)
        for k, (p, n, gm, op, b, x) in enumerate(ops):
            stream.wait_event(ev_in[k])
            if k + 1 < len(ops):
                put_rhs(k + 1)
            op.cg(b, x, precond=fem.PC_JACOBI, maxit=args.iters, rtol=0.0, use_graph=True,
                  zero_guess=True)
            ev_out[k].record(stream)
            with torch.cuda.stream(cstream):
                cstream.wait_event(ev_out[k])
                hx[k].copy_(x, non_blocking=True)
        cstream.synchronize()
        stream.synchronize()

    step_e2e()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step_e2e()
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    if world > 1:
        t = torch.tensor([e2e_ms], device="cuda")
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_ms = t.item()
    h2d = sum(8 * b.numel() for (_, _, _, _, b, _) in ops)

    # dominant kernel: the fused apply, timed per launch with events on its stream
    per_p = []
    tot_time, tot_flop, tot_bytes, tot_traffic, tot_exec = 0.0, 0.0, 0.0, 0.0, 0.0
    for p, n, gm, op, b, x in ops:
        y = torch.empty_like(x)
        for _ in range(3):
            op.apply(b, y)
        a0, a1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        a0.record(stream)
        for _ in range(reps):
            op.apply(b, y)
        a1.record(stream)
        torch.cuda.synchronize()
        t_apply = a0.elapsed_time(a1) / reps * 1e-3
        N, E, by, fl = body_algorithmic(p, n)
        _, _, _, fl_sf = algorithmic(p, n)
        per_p.append({"p": p, "N": N, "apply_ms": t_apply * 1e3,
                      "apply_gdofs": N / t_apply / 1e9,
                      "body": ("double-word assembled 27-point stencil" if p in STENCIL_ORDERS
                               else "double-word element matrices" if p in ELMAT_ORDERS
                               else "double-word sum factorization"),
                      "apply_hbm_gbs": by / t_apply / 1e9,
                      "operator_tflops": fl / t_apply / 1e12,
                      "sum_factorization_flops_tflops": fl_sf / t_apply / 1e12})
        tot_time += t_apply; tot_flop += fl_sf; tot_bytes += by
        tot_exec += fl
        r = dram_ratio(p)
        tot_traffic = None if (r is None or tot_traffic is None) else tot_traffic + r * by
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs", 6400.0)
    achieved = tot_bytes / tot_time / 1e9
    sf_orders = [d for d in per_p if d["p"] >= 3]
    sf_bytes = sum(body_algorithmic(d["p"], dict((p, n) for p, n in work)[d["p"]])[2] for d in sf_orders)
    sf_time = sum(d["apply_ms"] for d in sf_orders) * 1e-3
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak, "traffic": tot_traffic,
                "traffic_note": "DRAM bytes of one sweep (one FP64 apply per order), ncu counters"
                                " of a 4e6-DOF capture per order scaled by algorithmic bytes;"
                                " null when no capture of the current bodies exists",
                "algorithmic_bytes": tot_bytes,
                "achieved_note": "algorithmic bytes of one FP64 apply per order (x, y, element"
                                 " indices, qdata -- or the packed element matrices at p = 2, the"
                                 " stencil coefficients at p = 1)"
                                 " over the summed event-timed apply durations",
                "sum_factorized_orders_frac": (sf_bytes / sf_time / 1e9 / hbm_peak
                                               if sf_time > 0 else None),
                "operator_tflops": tot_exec / tot_time / 1e12,
                "sum_factorization_flops_tflops": tot_flop / tot_time / 1e12,
                "kernel": "FP64-accurate fused apply in double-word arithmetic on the FP32 pipe"
                          " (assembled stencil p=1, element-matrix body p=2, line body p>=3), all orders",
                "peak_source": "HBM copy bandwidth of measured (MEASURED_PEAKS.json)"}
    line = {"metric": METRIC, "value": value, "unit": "GDOF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": config(args, work),
            "e2e": {"value": dof_it * world / (e2e_ms * 1e-3) / 1e9, "unit": "GDOF/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": h2d},
            # per order: prepare + init, then per iteration the apply (two
            # kernels for the p = 1 stencil: the split of x and the stencil,
            # one otherwise), update and direction, in passes of 4 (kernels
            # after the last iteration return at once)
            "gpu_launches": sum(2 + (4 if p in STENCIL_ORDERS else 3) * 4 * ((args.iters + 3) // 4)
                                for p, _ in work) * args.steps,
            "roofline": roofline, "clocks": clocks, "per_order": per_p}
    del ops
    # the untimed single-GPU sections run at N = 1 only (a multi-rank run is
    # the replicated headline sweep)
    if args.tts_dofs > 0 and world == 1:
        line["time_to_solution"] = time_to_solution(fem, torch, args)
    secs = [t for t in args.sections.split(",") if t] if world == 1 else []
    if "bp56" in secs:
        line["bp5_bp6"] = section_bp56(fem, torch, args)
    if "suite" in secs:
        line["bp_suite"] = section_suite(fem, torch, args)
    if "nsweep" in secs:
        line["size_sweep"] = section_nsweep(fem, torch, args)
    if "batched" in secs:
        line["batched"] = section_batched(fem, torch, args)
    if "learned" in secs:
        line["learned"] = section_learned(fem, torch, args)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(work, args.iters, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
