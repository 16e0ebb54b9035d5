"""Benchmark: time to ||F(u)||_2 < 1e-8 and subdomain Newton steps/s, FP64 plain vs chosen form.

Workload (default): compressible Neo-Hooke (Eq. 2, plane, E = 210, nu = 0.3) on 2048 x 2048 Q1
cells (8.4M dofs), left edge clamped, vertical dead-load traction on the right edge ramped over
5 load steps, 4096 subdomains from the seeded uneven brick partition (+-15 % per side, seed
2410), overlap 2, RGDSW coarse space (23,376 coarse dofs), hybrid two-level coupling (Eq. 11),
zero initial guess.  One step = one complete solve from u = 0 through the 5 load steps to
||F|| < 1e-8: coarse Newton, one persistent batched local-Newton launch per outer iteration,
exact tangent inside GMRES, outer Newton update -- every step of the hot path on the device.
The chosen form uses FP32 local band factors and FP32 tiled coarse factors (tensor-core trailing
products) with FP64 iterative refinement; the plain form factors in FP64.  Setup (maps, coarse
basis) runs once before the timed region and is reported separately.  ``--workload c2`` runs the
1024 x 1024 nonlinear diffusion problem (Eq. 1) instead.

The line printed by rank 0 is the JSON contract of this repository: value = whole-job full
subdomain Newton steps per second (a step = one local Newton iteration with Jacobian assembly,
band factorization, solve and line search; chord steps on stored factors are reported apart),
roofline of the dominant kernel, e2e through host buffers, err_vs_oracle, and cpu_baseline = the
FP64 oracle on a bounded sample on every host core.  ``--impl reference`` times the oracle itself.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "time to ||F||<1e-8 and subdomain Newton steps/s: plain FP64 vs chosen form"
UNIT = "subdomain Newton steps/s"


def workload(name: str, seed: int = 0):
    """The named workload; `seed` (Neo-Hooke workloads) replaces the brick partition's seed."""
    from paper_2410_24138_gb300 import inputs as I
    seed = seed or I.PARTITION_SEED
    if name == "c2":
        return I.diffusion_c2(), "diffusion 1024x1024 P1 (1.05M dofs), 1024 uneven subdomains, overlap 2"
    if name == "c1":
        return I.diffusion_c1(), "diffusion 64x64 P1, 4x4 subdomains, overlap 1"
    if name == "c3":
        return I.neohooke_c3(seed=seed), "Neo-Hooke 512x512 Q1 (0.5M dofs), 256 uneven subdomains, overlap 2, 5 load steps"
    if name == "c4":
        return I.diffusion_c4(1), "log-normal diffusion 512x512 P1 (263k dofs), 256 uneven subdomains, overlap 2"
    if name == "c5":
        return I.neohooke_c5(seed=seed), ("Neo-Hooke 2048x2048 Q1 (8.4M dofs), 4096 uneven subdomains, overlap 2, "
                                          "5 load steps")
    raise SystemExit(f"unknown workload {name}")


DEFAULT_STEPS = {"c1": 10, "c2": 10, "c3": 5, "c4": 10, "c5": 3, "beam": 1}
WORKLOAD_NAME = ["c5"]  # the workload of this run (the key of the ncu traffic table)


# ----------------------------------------------------------------------------------------------
# CPU baseline: the oracle, as it stands, on a bounded sample of the same workload, on every core
# ----------------------------------------------------------------------------------------------
def sample_state(p) -> np.ndarray:
    """The point at which the CPU baseline solves local problems: u = 0 for Eq. 1 (the source acts
    everywhere), and for Eq. 2 the smooth bending state u_y = -0.02 x^2 (zero on the clamped edge),
    so that every subdomain has a nonlinear local problem to solve, not only those at the loaded
    edge."""
    u = np.zeros(p.n_nodes * p.ndof)
    if p.ndof == 2:
        u[1::2] = -0.02 * p.xy[:, 0] ** 2
    return u


def _oracle_worker(task):
    """One process of the CPU baseline: local Newton solves of the first load step at the sample
    state for its subdomains until ``budget_s`` seconds of solving; returns (steps, subdomains, s)."""
    name, subs, budget_s = task
    from oracle import schwarz as S
    p, _ = workload(name)
    load = 1.0 / max(1, p.load_steps)
    u = sample_state(p)
    steps, done, dt = 0, 0, 0.0
    for c0 in range(0, len(subs), 16):  # chunks amortise the oracle's per-construction mesh pass
        sw = S.Schwarz(p, S.Options(coupling=S.ONE_LEVEL), with_coarse=False, which=subs[c0:c0 + 16])
        t0 = time.perf_counter()
        for lp in sw.locals:
            _, its, _, _, _ = lp.solve_newton(u, u[lp.sub.dofs], sw.opts, load)
            steps += its
            done += 1
        dt += time.perf_counter() - t0
        if dt > budget_s:
            break
    return steps, done, dt


def oracle_sample(name: str, budget_s: float = 20.0, cores: int = 0):
    """The oracle's local solves on ``cores`` processes (0: every host core), each over its own
    seeded random share of the subdomains for about ``budget_s`` seconds of solving.  Returns
    (steps/s summed over the processes, steps, subdomains, seconds per process, processes)."""
    import multiprocessing as mp
    p, _ = workload(name)
    cores = cores or os.cpu_count() or 1
    order = np.random.default_rng(0).permutation(p.n_sub).tolist()
    tasks = [(name, order[k::cores], budget_s) for k in range(cores)]
    saved = {k: os.environ.get(k) for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for k in saved:
        os.environ[k] = "1"  # one thread per process: the processes are the parallelism
    try:
        with mp.get_context("spawn").Pool(cores) as pool:
            res = pool.map(_oracle_worker, tasks)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    rate = sum(st / dt for st, _, dt in res if dt > 0)
    return rate, sum(r[0] for r in res), sum(r[1] for r in res), max(r[2] for r in res), cores


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    for _ in range(args.warmup):
        oracle_sample(args.workload, budget_s=1.0)
    rates, total_steps, total_time, subs, cores = [], 0, 0.0, 0, 1
    for _ in range(args.steps):
        r, st, sd, dt, cores = oracle_sample(args.workload, budget_s=args.ref_budget)
        rates.append(r)
        total_steps += st
        total_time += dt
        subs += sd
    value = statistics.mean(rates)
    _, desc = workload(args.workload)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_time / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"{subs} subdomain local Newton solves at the first load step's sample "
                                       f"state (u = 0 for Eq. 1, bending u_y = -0.02 x^2 for Eq. 2) on {cores} "
                                       f"processes over {args.steps} steps, {total_steps} subdomain Newton steps"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
            # the timed region starts once the sampler is producing lines
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.01)
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------------------------
def run_c4(args):
    """Learned-guess workload (log-normal diffusion, 512 x 512 P1, 256 bricks, overlap 2): harvest
    (features, converged local state) pairs from the method's own solves over training fields,
    train the network on the GPU (BF16 tensor-core GEMMs, FP32 master weights, Adam), then time
    held-out solves with and without the guess on the same context (coefficients swapped with
    nls_set_coefficients).  The timed region is the solves only; training is reported apart."""
    import torch
    from paper_2410_24138_gb300 import build, nls, inputs as I
    build.build()
    n, per = 512, 16
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    base = I.diffusion_c4(1, n=n, per_side=per)
    s = nls.Solver(device=0, stream=stream)
    s.set_problem(base)
    s.set_coarse(nls.COARSE_RGDSW)
    s.set_options(coupling=nls.COUPLING["hybrid"], local_precision=nls.PREC_FP32_IR,
                  coarse_precision=nls.PREC_FP32_IR, autotune=1)
    t0 = time.perf_counter()
    s.setup()
    setup_s = time.perf_counter() - t0
    sizes = s.sizes()
    net = nls.GuessNet(h1=512, h2=512, seed=11, capacity=args.c4_pairs + 4096)
    nls.attach_guess(s, net, nls.GUESS_HARVEST)
    t0 = time.perf_counter()
    seed, harvest_solves = 1, 0
    while net.pairs() < args.c4_pairs:
        s.set_coefficients(*I.c4_elem_coefficients(seed, n))
        u, rep = s.solve()
        seed += 1
        harvest_solves += 1
    harvest_s = time.perf_counter() - t0
    t0 = time.perf_counter()
    losses = net.train(steps=args.c4_train_steps, batch=256, lr=1e-3, seed=5)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float64, device="cuda")
    res = {"plain": [], "guess": [], "guess_first_outer": []}
    accepted = proposed = 0
    counts = {}
    launches = 0
    test_seeds = list(range(1001, 1001 + args.steps))
    for mode in ("plain", "guess", "guess_first_outer"):
        flags = nls.GUESS_USE | (nls.GUESS_FIRST_OUTER if mode == "guess_first_outer" else 0)
        nls.attach_guess(s, None if mode == "plain" else net, flags)
        if mode != "plain":
            nls.set_guess_smoothing(s, args.c4_sweeps, 0.8)
        for i, sd in enumerate([1001, 1002, 1003] + test_seeds):  # the first three warm up
            s.set_coefficients(*I.c4_elem_coefficients(sd, n))
            flush_buf.add_(1.0)
            u = torch.zeros(sizes.n_dofs, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            u, rep = s.solve(u)
            e1.record()
            e1.synchronize()
            if mode != "plain":
                p_, a_ = nls.guess_counts(s)
            if i >= 3:
                res[mode].append((e0.elapsed_time(e1), rep.subdomain_newton_steps - rep.local_chord_steps,
                                  rep.outer_iterations, rep.final_residual, rep.local_chord_steps,
                                  rep.subdomain_newton_steps))
                if mode == "guess_first_outer":
                    launches += rep.kernel_launches
                if mode != "plain":
                    pc, ac = counts.get(mode, (0, 0))
                    counts[mode] = (pc + p_, ac + a_)
                if mode == "guess":
                    proposed += p_
                    accepted += a_
    ms_plain = sum(r[0] for r in res["plain"])
    ms_guess = sum(r[0] for r in res["guess"])
    ms_first = sum(r[0] for r in res["guess_first_outer"])
    st_plain = sum(r[1] for r in res["plain"])
    st_guess = sum(r[1] for r in res["guess"])
    line = {
        "metric": METRIC, "value": sum(r[5] for r in res["guess_first_outer"]) / (ms_first * 1e-3), "unit": UNIT,
        "n_gpus": 1, "steps": args.steps,
        "warmup": 3, "ms_per_step": ms_first / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32 (bf16 network training)", "data": "synthetic",
        "config": {"workload": "log-normal diffusion 512x512 P1 (263k dofs), 256 uneven subdomains, overlap 2; "
                               "learned initial guess proposed at the first outer iteration of every solve",
                   "coupling": "hybrid",
                   "l2": "512 MB buffer written between steps", "setup_s": setup_s,
                   "n_dofs": sizes.n_dofs, "n_sub": sizes.n_sub, "coarse_dofs": sizes.n_coarse_dofs},
        "guess": {"pairs": net.pairs(), "harvest_solves": harvest_solves, "harvest_s": harvest_s,
                  "train_steps": args.c4_train_steps, "train_s": train_s,
                  "loss_first50": float(losses[:50].mean()), "loss_last50": float(losses[-50:].mean()),
                  "proposed": proposed, "accepted": accepted, "smoothing_sweeps": args.c4_sweeps},
        "held_out": {"solves": args.steps,
                     "time_to_solution_ms": {"plain": ms_plain / args.steps, "guess": ms_guess / args.steps},
                     "full_newton_steps": {"plain": st_plain, "guess": st_guess},
                     "local_chord_steps": {"plain": sum(r[4] for r in res["plain"]),
                                           "guess": sum(r[4] for r in res["guess"])},
                     "outer_iterations": {"plain": [r[2] for r in res["plain"]], "guess": [r[2] for r in res["guess"]]},
                     "max_final_residual": max(r[3] for r in res["plain"] + res["guess"])},
        "held_out_first_outer_only": {
            "time_to_solution_ms": sum(r[0] for r in res["guess_first_outer"]) / args.steps,
            "full_newton_steps": sum(r[1] for r in res["guess_first_outer"]),
            "local_chord_steps": sum(r[4] for r in res["guess_first_outer"]),
            "proposed_accepted": counts.get("guess_first_outer"),
            "max_final_residual": max(r[3] for r in res["guess_first_outer"])},
        "tuning": s.tuning(),
        "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def run_beam(args):
    """The beam of Section 1 and Fig. 2's robustness experiment: Neo-Hooke (E = 210, nu = 0.3), 5 x 1,
    clamped at both ends, under a volume force f_x across the beam (laid out along y, see
    inputs.beam_problem).  For every force, one solve from u = 0 (no load steps) with the
    two-level additive and hybrid couplings in the chosen form (FP32 factors + FP64 refinement,
    autotuned CTAs, graph-replayed GMRES iterations); GMRES stops after 100 iterations per linear
    solve, as in Section 3.  One untimed solve at the smallest force per coupling warms up (and
    tunes).  Reports which forces converged (||F|| < 1e-8 within 30 outer iterations), the outer
    and GMRES iterations and the time to solution; the value is the largest force the hybrid
    coupling solved."""
    import torch
    from paper_2410_24138_gb300 import build, nls, inputs as I
    build.build()
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream().cuda_stream
    forces = [float(x) for x in args.beam_forces.split(",")]
    p = I.beam_problem(args.beam_m, args.beam_px, args.beam_py, 1.0)
    unit_force = p.f_vol.copy()
    rows, setup = [], {}
    sizes = None
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float64, device="cuda")
    launches = 0
    for coupling in ("hybrid", "add"):
        s = nls.Solver(device=0, stream=stream)
        s.set_problem(p)
        s.set_coarse(nls.COARSE_RGDSW)
        s.set_options(coupling=nls.COUPLING[coupling], load_steps=1, local_precision=nls.PREC_FP32_IR,
                      coarse_precision=nls.PREC_FP32_IR, autotune=1, gmres_maxit=100,
                      coarse_rebuild=1 if args.coarse_rebuild else 0)
        t0 = time.perf_counter()
        s.setup()
        setup[coupling] = time.perf_counter() - t0
        sizes = s.sizes()
        for i, f in enumerate([forces[0]] + forces):
            s.set_volume_force(f * unit_force)
            flush_buf.add_(1.0)
            u = torch.zeros(sizes.n_dofs, dtype=torch.float64, device="cuda")
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            try:
                u, rep = s.solve(u)
                err = None
            except nls.NLSError as ex:
                rep, err = None, str(ex)
            e1.record()
            e1.synchronize()
            if i == 0:
                continue
            ok = rep is not None and rep.status == 0 and rep.final_residual < 1e-8
            if rep is not None:
                launches += rep.kernel_launches
            rows.append({"coupling": coupling, "f_x": f, "converged": bool(ok),
                         "status": None if rep is None else rep.status,
                         "outer": None if rep is None else rep.outer_iterations,
                         "gmres": None if rep is None else rep.gmres_iterations,
                         "local_steps": None if rep is None else rep.subdomain_newton_steps,
                         "local_failures": None if rep is None else rep.local_failures,
                         "final_residual": None if rep is None else rep.final_residual,
                         "time_s": e0.elapsed_time(e1) * 1e-3, "error": err})
        s.close()
    best = {c: max([r["f_x"] for r in rows if r["coupling"] == c and r["converged"]], default=None)
            for c in ("hybrid", "add")}
    conv = [r for r in rows if r["converged"]]
    line = {
        "metric": "largest volume force solved from u = 0 (hybrid coupling)", "value": best["hybrid"],
        "unit": "f_x (GN/m^3 with E in GPa)", "n_gpus": 1, "steps": len(forces), "warmup": 1,
        "ms_per_step": (sum(r["time_s"] for r in conv) / max(1, len(conv))) * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
        "config": {"workload": f"Neo-Hooke beam 5 x 1 (Section 1), {p.conn.shape[0]} Q1 cells "
                               f"({sizes.n_dofs} dofs), {sizes.n_sub} uneven subdomains, overlap 2, clamped ends, "
                               "volume force, no load steps, GMRES max 100"
                               + (", coarse basis rebuilt at every outer iterate" if args.coarse_rebuild else ""),
                   "setup_s": setup, "n_dofs": sizes.n_dofs, "n_sub": sizes.n_sub,
                   "coarse_dofs": sizes.n_coarse_dofs, "max_local_dofs": sizes.max_local_dofs,
                   "max_half_band": sizes.max_half_band, "coarse_half_band": sizes.coarse_half_band,
                   "l2": "512 MB buffer written between solves"},
        "largest_force_solved": best, "sweep": rows, "gpu_launches": launches,
    }
    print(json.dumps(line), flush=True)


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def timed_solves(torch, solver, n_dofs, steps, flush_buf):
    """Device-resident solves from u = 0; returns per-step ms, total subdomain Newton steps, reports."""
    stream = torch.cuda.current_stream()
    times, reps = [], []
    for _ in range(steps):
        flush_buf.add_(1.0)  # write 512 MB > L2 between steps
        u = torch.zeros(n_dofs, dtype=torch.float64, device="cuda")
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        u, rep = solver.solve(u)
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
        reps.append(rep)
    return times, reps


def replica_throughput(torch, dist, world, total_ms, units, device):
    """Whole-job throughput of ``world`` independent replicas (one per GPU, no exchange on the data
    path): the units all ranks processed divided by the slowest rank's time.  Returns (units per
    second, max ms, summed units); a plain division for one process."""
    ms_t = torch.tensor([float(total_ms)], device=device, dtype=torch.float64)
    st_t = torch.tensor([float(units)], device=device, dtype=torch.float64)
    if world > 1:
        dist.all_reduce(ms_t, op=dist.ReduceOp.MAX)
        dist.all_reduce(st_t, op=dist.ReduceOp.SUM)
    return st_t.item() / (ms_t.item() * 1e-3), ms_t.item(), st_t.item()


def err_vs_oracle(p, u: np.ndarray, samples: int = 6) -> dict:
    """Error of a converged solution against the FP64 oracle, computed outside the timed region.
    Always: the oracle's own FP64 evaluation of ||F(u)||_2 at the final load.  Diffusion meshes up
    to about 1M dofs: the relative l2 distance to the oracle's plain global Newton solution of
    F(u) = 0 (sparse direct FP64 solves, driven to ||F|| < 1e-11).  Larger or elasticity meshes:
    for seeded sampled subdomains, the oracle's local solve of Eq. 4 at the returned u (tight
    tolerances); a solution of F(u) = 0 is a fixed point of every local solve, so the relative
    change of R_i u bounds how far u is from the oracle's local solutions."""
    from oracle import fem, schwarz as S
    F = fem.global_residual(fem.Model(p), u, 1.0)
    out = {"oracle_residual": float(np.linalg.norm(F))}
    t0 = time.perf_counter()
    if p.law == 1 and p.n_nodes * p.ndof <= 1_100_000:
        us, _ = S.plain_newton(p, tol=1e-11, load_steps=p.load_steps)
        out.update(kind="global: the oracle's plain Newton solution (sparse direct FP64) on the same mesh",
                   rel_l2=float(np.linalg.norm(u - us) / np.linalg.norm(us)))
    else:
        rng = np.random.default_rng(2410)
        pick = sorted({0, p.n_sub // 2, p.n_sub - 1, *rng.choice(p.n_sub, samples - 3, replace=False).tolist()})
        opts = S.Options(coupling=S.ONE_LEVEL, inner_rtol=1e-12, inner_atol=1e-13)
        sw = S.Schwarz(p, opts, with_coarse=False, which=pick)
        errs = []
        for lp in sw.locals:
            ru = u[lp.sub.dofs]
            w, _, _, _, _ = lp.solve_newton(u, ru, opts, 1.0)
            errs.append(float(np.linalg.norm(w - ru) / max(np.linalg.norm(ru), 1e-300)))
        out.update(kind="sampled: the oracle's local solves (Eq. 4) at the returned u; relative change of R_i u",
                   subdomains=pick, rel_l2_max=max(errs), rel_l2=errs)
    out["oracle_s"] = time.perf_counter() - t0
    return out


def run_gpu(args):
    import torch
    import torch.distributed as dist
    from paper_2410_24138_gb300 import build, nls

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    build.build()
    p, desc = workload(args.workload)
    steps = args.steps
    stream = torch.cuda.current_stream().cuda_stream
    flush_buf = torch.zeros(64 * 1024 * 1024, dtype=torch.float64, device="cuda")
    coupling = "hybrid" if p.n_sub > 1 else "one"

    def make(precision, prob=None):
        s = nls.Solver(device=local, stream=stream)
        s.set_problem(prob if prob is not None else p)
        s.set_coarse(nls.COARSE_RGDSW if coupling != "one" else nls.COARSE_NONE)
        prec = nls.PREC_FP32_IR if precision == "fp32" else nls.PREC_FP64
        s.set_options(coupling=nls.COUPLING[coupling], load_steps=p.load_steps, local_precision=prec,
                      coarse_precision=prec, autotune=1)
        t0 = time.perf_counter()
        s.setup()
        return s, time.perf_counter() - t0

    chosen, setup_s = make("fp32")
    sizes = chosen.sizes()
    n_dofs = sizes.n_dofs
    timed_solves(torch, chosen, n_dofs, args.warmup, flush_buf)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("bench:timed")  # the range a profiler's launch list selects
    times, reps = timed_solves(torch, chosen, n_dofs, steps, flush_buf)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    total_ms = sum(times)
    # the metric counts full local Newton steps (Jacobian assembly, band factorization, solve,
    # line search); steps taken with stored factors (chord steps) are reported apart
    full_steps = sum(r.subdomain_newton_steps - r.local_chord_steps for r in reps)
    value, _, _ = replica_throughput(torch, dist, world, total_ms, full_steps, "cuda")
    rep0 = reps[-1]
    u_final = None

    # per-kernel timing of one more solve on the same context (CUDA events on the launching
    # stream; graphs are off while profiling), outside the timed region
    chosen.set_options(profile_kernels=1)
    chosen.reset_kernel_stats()
    ptimes, preps = timed_solves(torch, chosen, n_dofs, 1, flush_buf)
    kstats_all = chosen.kernel_stats()
    chosen.set_options(profile_kernels=0)
    phases = {k[6:]: round(v[1], 3) for k, v in kstats_all.items() if k.startswith("phase:")}
    kstats = {k: v for k, v in kstats_all.items() if not k.startswith("phase:")}

    # end to end through the C ABI with host buffers (pinned), copies inside the timed region
    host_u = torch.zeros(n_dofs, dtype=torch.float64).pin_memory()
    e2e_steps, e2e_ms = 0, 0.0
    for _ in range(steps):
        flush_buf.add_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hu = host_u.numpy()
        hu[:] = 0.0
        hu, rep = chosen.solve(hu)
        e2e_ms += (time.perf_counter() - t0) * 1e3
        e2e_steps += rep.subdomain_newton_steps - rep.local_chord_steps
    e2e_value = e2e_steps / (e2e_ms * 1e-3)
    u_final = np.array(hu, copy=True)
    tuning = chosen.tuning()
    chosen.close()

    # plain FP64 form on the same mesh
    plain, plain_setup = make("fp64")
    timed_solves(torch, plain, n_dofs, 1, flush_buf)
    p_times, p_reps = timed_solves(torch, plain, n_dofs, max(1, min(steps, 2)), flush_buf)
    plain_full = sum(r.subdomain_newton_steps - r.local_chord_steps for r in p_reps)
    plain_rate = plain_full / (sum(p_times) * 1e-3)
    plain.close()

    # the learned displacement guess (Eq. 2), trained on a held-out partition
    guess = None
    if p.ndof == 2 and world == 1 and not args.no_guess:
        guess = displacement_guess_leg(torch, nls, args, make, n_dofs, steps, flush_buf,
                                       statistics.median(times), statistics.median(p_times))

    # roofline of the dominant kernel
    peaks, peak_kind = measured_peaks()
    dom_name, (dom_launches, dom_ms) = max(kstats.items(), key=lambda kv: kv[1][1])
    total_prof_ms = sum(v[1] for v in kstats.values())
    # factorizations per launch: one per full local Newton step plus the tangent's
    steps_per_launch = ((preps[-1].subdomain_newton_steps - preps[-1].local_chord_steps)
                        / max(1, preps[-1].outer_iterations))
    split = any(k.startswith("k_local_factor") for k in kstats)
    roof = roofline_for(dom_name, dom_launches, dom_ms, sizes, peaks, peak_kind, steps_per_launch, split)
    roof_top = [roofline_for(k, v[0], v[1], sizes, peaks, peak_kind, steps_per_launch, split)
                for k, v in sorted(kstats.items(), key=lambda kv: -kv[1][1])[:5]]
    coarse_tc = {k: v for k, v in kstats.items() if k.startswith("k_tlu") or k.startswith("k_tile")}
    roof_tensor = [roofline_for(k, v[0], v[1], sizes, peaks, peak_kind) for k, v in kstats.items()
                   if k.startswith("k_tlu_update_tc") or k.startswith("k_tile_solve_products")]

    if rank == 0:
        err = err_vs_oracle(p, u_final) if not args.no_oracle_err else None
        cpu = None
        if world == 1 and not args.no_cpu_baseline:
            r, st, sd, dt, cores = oracle_sample(args.workload, budget_s=args.ref_budget)
            cpu = {"value": r, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": f"{sd} subdomain local Newton solves at the first load step's sample state (u = 0 "
                             f"for Eq. 1, bending u_y = -0.02 x^2 for Eq. 2), {st} subdomain Newton steps, {cores} "
                             f"processes of {dt:.1f} s each (numpy/scipy FP64, one thread per process)"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": steps,
            "warmup": args.warmup, "ms_per_step": total_ms / steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64+f32", "data": "synthetic",
            "config": {"workload": desc, "coupling": coupling,
                       "precision": "FP32 local band factors and FP32 tiled coarse factors + FP64 iterative "
                                    "refinement; FP64 residuals, GMRES, coarse matrix",
                       "l2": "512 MB buffer written between steps; working set > L2",
                       "parallelism": "replicas" if world > 1 else "single GPU", "setup_s": setup_s,
                       "n_dofs": n_dofs, "n_sub": sizes.n_sub, "coarse_dofs": sizes.n_coarse_dofs,
                       "max_local_dofs": sizes.max_local_dofs, "max_half_band": sizes.max_half_band,
                       "coarse_half_band": sizes.coarse_half_band},
            "time_to_solution_s": {"chosen": statistics.median(times) * 1e-3,
                                   "plain_fp64": statistics.median(p_times) * 1e-3},
            "full_newton_steps_per_s": {"chosen": value / world, "plain_fp64": plain_rate},
            "speedup_chosen_vs_plain": statistics.median(p_times) / statistics.median(times),
            "iterations": {"outer": rep0.outer_iterations, "gmres": rep0.gmres_iterations,
                           "full_newton_steps": rep0.subdomain_newton_steps - rep0.local_chord_steps,
                           "chord_steps": rep0.local_chord_steps,
                           "coarse_newton_steps": rep0.coarse_newton_steps,
                           "final_residual": rep0.final_residual, "local_failures": rep0.local_failures},
            "plain_iterations": {"outer": p_reps[-1].outer_iterations, "gmres": p_reps[-1].gmres_iterations,
                                 "full_newton_steps": p_reps[-1].subdomain_newton_steps - p_reps[-1].local_chord_steps,
                                 "final_residual": p_reps[-1].final_residual},
            "phases_s": {"inner": rep0.time_inner_s, "coarse": rep0.time_coarse_s, "gmres": rep0.time_gmres_s,
                         "other": rep0.time_other_s},
            "local_newton_phases_cta_ms": phases,
            "kernels_ms": {k: [v[0], round(v[1], 3), round(100.0 * v[1] / total_prof_ms, 1)] for k, v in
                           sorted(kstats.items(), key=lambda kv: -kv[1][1])[:10]},
            "coarse_factor_kernels_ms": {k: [v[0], round(v[1], 3)] for k, v in coarse_tc.items()},
            "roofline": roof,
            "roofline_top": roof_top,
            "roofline_tensor": roof_tensor,
            "tuning": tuning,
            "err_vs_oracle": err,
            "learned_guess": guess,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 8 * n_dofs, "d2h_bytes_per_step": 8 * n_dofs},
            "gpu_launches": int(sum(r.kernel_launches for r in reps)),
            "clocks": clk,
            "cpu_baseline": cpu,
            "wall_s": t_wall,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


def displacement_guess_leg(torch, nls, args, make, n_dofs, steps, flush_buf, chosen_ms, plain_ms):
    """The learned initial guess on a Neo-Hooke workload: harvest (features, converged local state)
    pairs from one chosen-form solve of the same mesh on a held-out partition (the brick
    generator's next seed), train the displacement network on the GPU (BF16 tensor-core GEMMs,
    FP32 master weights, Adam), then time the chosen form with the guess on the benchmark's own
    partition (outside the headline's timed region; reported beside it)."""
    from paper_2410_24138_gb300 import inputs as I
    hp, _ = workload(args.workload, seed=I.PARTITION_SEED + 1)
    h, _ = make("fp32", hp)
    net = nls.GuessNet(h1=512, h2=512, seed=11, capacity=hp.n_sub * 24, kind=nls.GUESS_KIND_DISPLACEMENT)
    nls.attach_guess(h, net, nls.GUESS_HARVEST)
    t0 = time.perf_counter()
    h.solve()
    torch.cuda.synchronize()
    harvest_s = time.perf_counter() - t0
    pairs = net.pairs()
    h.close()
    t0 = time.perf_counter()
    losses = net.train(steps=args.guess_train_steps, batch=256, lr=1e-3, seed=5)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    mode = nls.GUESS_USE | (nls.GUESS_FIRST_OUTER if args.guess_mode == "first" else 0)
    s, _ = make("fp32")
    nls.attach_guess(s, net, mode)
    timed_solves(torch, s, n_dofs, 1, flush_buf)  # warm-up and autotuning
    nls.guess_counts(s)
    g_times, g_reps = timed_solves(torch, s, n_dofs, steps, flush_buf)
    proposed, accepted = nls.guess_counts(s)
    s.close()
    net.close()
    r = g_reps[-1]
    g_ms = statistics.median(g_times)
    return {"kind": "displacement (Eq. 2)", "mode": "first outer iteration of every load step"
            if args.guess_mode == "first" else "every outer iteration",
            "harvest": {"partition_seed": I.PARTITION_SEED + 1, "pairs": pairs, "solve_s": harvest_s},
            "train": {"steps": args.guess_train_steps, "batch": 256, "s": train_s,
                      "loss_first50": float(losses[:50].mean()), "loss_last50": float(losses[-50:].mean())},
            "time_to_solution_s": {"chosen_with_guess": g_ms * 1e-3, "chosen": chosen_ms * 1e-3,
                                   "plain_fp64": plain_ms * 1e-3},
            "speedup_with_guess_vs_plain": plain_ms / g_ms, "speedup_with_guess_vs_chosen": chosen_ms / g_ms,
            "iterations": {"outer": r.outer_iterations, "gmres": r.gmres_iterations,
                           "full_newton_steps": r.subdomain_newton_steps - r.local_chord_steps,
                           "chord_steps": r.local_chord_steps, "final_residual": r.final_residual},
            "proposed": proposed // steps, "accepted": accepted // steps}


# FP32 FMA peak of the GB300 derived from its unit counts and clock: 152 SMs x 128 FP32 lanes
# x 2 flops per FMA x 2.07 GHz (maximum SM clock).
SMS, FP32_LANES_PER_SM = 152, 128


def fp32_peak_tflops(peaks):
    mhz = peaks.get("sm_max_mhz", 2070.0)
    return SMS * FP32_LANES_PER_SM * 2 * mhz * 1e6 / 1e12


# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of one launch, from the ncu captures
# summarised in profiles/ (keyed by workload and kernel); a kernel changed since its capture has no
# entry.  k_local_apply was captured on the 512^2 Neo-Hooke workload (1.523 GB per launch); on the
# 2048^2 one (same subdomain size, 16x the subdomains) it is scaled by the ratio of the algorithmic
# bytes per launch (8.28 / 0.5126 GB).
NCU_TRAFFIC_BYTES = {
    ("c3", "k_local_apply<float>"): 1.523e9,
    ("c5", "k_local_apply<float>"): 1.523e9 * 8.2796e9 / 0.5126e9,
}


def roofline_for(name, launches, ms, sizes, peaks, peak_kind, steps_per_launch=None, split_factor=False):
    """Achieved algorithmic bandwidth (or ALU rate) of a kernel per launch.  split_factor: the
    refactorisation at the converged states ran in k_local_factor, not in k_local_newton."""
    avg_s = ms * 1e-3 / max(1, launches)
    if "local_factor" in name:
        # one band LU of every subdomain per launch (the packing is not counted)
        flops = sizes.lu_flops
        peak = fp32_peak_tflops(peaks)
        ach = flops / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "algorithmic_flops_per_launch": flops,
                "avg_launch_ms": avg_s * 1e3,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
    if "local_newton" in name and steps_per_launch is not None:
        # factorizations: one per full local Newton step plus (unless split off) the
        # refactorization at the converged state of every subdomain; one pair of triangular
        # solves per full Newton step
        per_sub_steps = steps_per_launch / sizes.n_sub
        flops = sizes.lu_flops * (per_sub_steps + (0.0 if split_factor else 1.0)) + sizes.solve_flops * per_sub_steps
        peak = fp32_peak_tflops(peaks)
        ach = flops / avg_s / 1e12
        return {"kernel": name, "bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": NCU_TRAFFIC_BYTES.get((WORKLOAD_NAME[0], name)), "algorithmic_flops_per_launch": flops,
                "avg_launch_ms": avg_s * 1e3,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 x max SM clock"}
    if "local_apply" in name:
        fb = sizes.factor_bytes
        # algorithmic bytes of one tangent application: every subdomain's band factors read once
        # (sum_i n_i (2 b_i + 1) entries), its local Jacobian (value + column index, 12 bytes per
        # nonzero) and three global vectors (input, the term added, output)
        alg = sizes.total_factor_entries * fb + sizes.total_local_nnz * 12 + 3 * sizes.n_dofs * 8
        packed = sizes.total_solve_entries * fb
        peak = peaks["hbm_gbs"]
        return {"kernel": name, "bound": "hbm", "achieved": alg / avg_s / 1e9, "peak": peak, "unit": "GB/s",
                "frac": alg / avg_s / 1e9 / peak, "traffic": NCU_TRAFFIC_BYTES.get((WORKLOAD_NAME[0], name)),
                "algorithmic_bytes_per_launch": alg,
                "stored_operand_bytes_per_launch": packed + sizes.total_local_nnz * 12 + 3 * sizes.n_dofs * 8,
                "operand_format_overhead": packed / max(1, sizes.total_factor_entries * fb),
                "avg_launch_ms": avg_s * 1e3, "peak_source": peak_kind}
    if name.startswith("k_tlu_update_tc") or name.startswith("k_tile_solve_products"):
        # tensor-core tile products: three TF32 MMA passes (hi*hi, hi*lo, lo*hi) of 128 x 128 x 128
        # per tile (the executed tensor flops; the algorithmic product is a third of them); peak =
        # the measured sustained BF16 peak (the kernels run inside a seconds-long solve) times the
        # nominal TF32 / BF16 ratio (1.1 / 2.25)
        NT, TB = -(-sizes.n_coarse_dofs // 128), max(1, -(-sizes.coarse_half_band // 128))
        if name.startswith("k_tlu_update_tc"):
            tiles = sum(min(TB, NT - 1 - k) ** 2 for k in range(NT - 1)) / max(1, NT - 1)
        else:
            tiles = sum(1 for t in range(NT) for k in range(1, TB + 1) if t - k >= 0) + \
                sum(1 for t in range(NT) for k in range(1, TB + 1) if t + k < NT)
        flops = 3 * 2 * 128 ** 3 * tiles
        sustained = "bf16_tflops_sustained" in peaks
        peak = peaks["bf16_tflops_sustained" if sustained else "bf16_tflops"] * 1.1 / 2.25
        ach = flops / avg_s / 1e12
        return {"kernel": name, "bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                "frac": ach / peak, "traffic": None, "tf32_flops_per_launch": flops, "avg_launch_ms": avg_s * 1e3,
                "peak_source": f"{peak_kind} {'sustained ' if sustained else ''}bf16 x nominal tf32/bf16 (1.1/2.25)"}
    if name == "k_tile_solve":
        # forward and backward tile-row sweeps of the cluster solve: every tile of the factors read
        # once per solve (L_tt^-1 M_tk / U_tt^-1 N_tk, (TB + 1) 128 x 128 FP32 tiles per tile row
        # and sweep); bound by the latency of the 2 N_T dependent steps, reported against HBM
        NT, TB = -(-sizes.n_coarse_dofs // 128), max(1, -(-sizes.coarse_half_band // 128))
        alg = 2 * NT * (TB + 1) * 128 * 128 * 4 + 3 * sizes.n_coarse_dofs * 8
        peak = peaks["hbm_gbs"]
        return {"kernel": name, "bound": "hbm", "achieved": alg / avg_s / 1e9, "peak": peak, "unit": "GB/s",
                "frac": alg / avg_s / 1e9 / peak, "traffic": None, "algorithmic_bytes_per_launch": alg,
                "avg_launch_ms": avg_s * 1e3, "peak_source": peak_kind}
    if "multidot" in name or "multiaxpy" in name or "spmv" in name or "p0" in name:
        return {"kernel": name, "bound": "hbm", "achieved": None, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": None, "traffic": None, "avg_launch_ms": avg_s * 1e3, "peak_source": peak_kind}
    return {"kernel": name, "bound": "alu", "achieved": None, "peak": None, "unit": "TFLOP/s", "frac": None,
            "traffic": None, "avg_launch_ms": avg_s * 1e3, "peak_source": peak_kind}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=0, help="timed steps (0: the workload's default)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c5", choices=["c1", "c2", "c3", "c4", "c5", "beam"])
    ap.add_argument("--beam-m", type=int, default=240, help="beam cells across its unit width (5m along it)")
    ap.add_argument("--beam-px", type=int, default=8, help="bricks across the beam")
    ap.add_argument("--beam-py", type=int, default=32, help="bricks along the beam")
    ap.add_argument("--beam-forces", default="4,5,6,7,7.5,8,9,10")
    ap.add_argument("--coarse-rebuild", action="store_true", help="beam: rebuild the coarse basis at every outer iterate")
    ap.add_argument("--c4-pairs", type=int, default=50000)
    ap.add_argument("--c4-train-steps", type=int, default=4000)
    ap.add_argument("--c4-sweeps", type=int, default=6)
    ap.add_argument("--ref-budget", type=float, default=20.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-oracle-err", action="store_true", help="skip the error report against the oracle")
    ap.add_argument("--no-guess", action="store_true", help="Neo-Hooke workloads: skip the learned-guess leg")
    ap.add_argument("--guess-mode", default="first", choices=["first", "all"],
                    help="propose at the first outer iteration of every load step, or at every one")
    ap.add_argument("--guess-train-steps", type=int, default=4000)
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("at least 3 warm-up steps are required")
    if not args.steps:
        args.steps = DEFAULT_STEPS.get(args.workload, 3)
    WORKLOAD_NAME[0] = args.workload
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "c4":
        run_c4(args)
    elif args.workload == "beam":
        run_beam(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
