#!/usr/bin/env python
"""Benchmark of the DG-SBM hp-multigrid FGMRES solve on GB300.

One step = one FGMRES(30) solve to 1e-8 relative FP64 residual from x = 0 (every row of the
hot path: operator apply, coloured block smoother, transfers, coarse solve, Arnoldi with
two-pass classical Gram-Schmidt) of the 2D p=2 star workload, 512^2 background cells, with the
FP32 V-cycle under FP64 FGMRES.  The FP64-V-cycle solve of the same workload is timed beside
it.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
  python bench.py --profile solve|kernels [--profile-n N]   (fixed launches for ncu, no JSON)

Under torchrun each rank solves its own seeded replica of the workload on its own GPU
(replicas only: no data-path collective); the reported time is the max over ranks.
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

# the oracle arms run on one host core: pin the BLAS thread pools before numpy is first imported
if "--cpu-worker" in sys.argv or "reference" in sys.argv:
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "solve time to 1e-8 rel. residual (FP32/learned vs FP64 V-cycle); apply GB/s"
WORKLOADS = {
    "star2d_p2_n512": lambda seed: W.star2d_p2(512, seed),
    "disk2d_p1_n32": lambda seed: W.disk2d_p1(32, seed),
    "sphere3d_p1_n64": lambda seed: W.sphere3d(64, 1, seed),
    "sphere3d_p2_n64": lambda seed: W.sphere3d(64, 2, seed),
    "ellipsoid3d_p3_n96": lambda seed: W.ellipsoid3d_p3(96, seed),
    "ellipsoid3d_p3_n96_s1": lambda seed: W.ellipsoid3d_p3(96, seed, smooth=1),
}
DESCRIPTION = {
    "star2d_p2_n512": "2D star r(theta)=0.7(1+0.1 sin(5 theta+phi)), 512^2 background cells, Q2 DG-SBM, "
                      "u=exp(x)cos(2y), lambda=0.75, hp-multigrid p2->p1 then h to 8^2, FGMRES(30) tol 1e-8",
    "disk2d_p1_n32": "2D disk r=0.7, 32^2 background cells, Q1 DG-SBM, u=sin(pi x)sin(pi y), lambda>=0.5, "
                     "hp-multigrid h to 4^2, FGMRES(30) tol 1e-8",
    "sphere3d_p1_n64": "3D sphere r=0.7, 64^3 background cells, Q1 DG-SBM, u=sin sin sin, lambda=0.75, "
                       "h-multigrid to 4^3, FGMRES(30) tol 1e-8",
    "sphere3d_p2_n64": "3D sphere r=0.7, 64^3 background cells, Q2 DG-SBM, u=sin sin sin, lambda=0.75, "
                       "hp-multigrid p2->p1 then h to 4^3, FGMRES(30) tol 1e-8",
    "ellipsoid3d_p3_n96": "3D rotated ellipsoid (0.75,0.6,0.5), 96^3 background cells, Q3 DG-SBM, u=sin sin sin, "
                          "lambda=0.75, hp-multigrid p3->p2->p1 then h to 6^3, 2 pre/2 post smoothing steps, "
                          "FGMRES(30) tol 1e-8",
    "ellipsoid3d_p3_n96_s1": "the 96^3 p=3 ellipsoid with 1 pre/1 post smoothing step (stalls without help)",
}
TOL, RESTART, MAX_IT = 1e-8, 30, 300
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


# ----------------------------------------------------------------------------- CPU oracle worker
def cpu_worker(workload: str, seed: int, budget_s: float) -> dict:
    """Times the CPU FP64 oracle (set-up untimed) on the same workload: whole FGMRES(30) solves to
    1e-8 from x = 0, repeated until `budget_s` of solve time is spent (at least one).  Writes the
    oracle's solution and the background cell of every oracle cell to an .npz file (for the error
    of the GPU solutions against the oracle) and returns its path with the timings."""
    import numpy as np
    from oracle import krylov as K
    from oracle import multigrid as MG
    prob = WORKLOADS[workload](seed)
    t0 = time.perf_counter()
    H = MG.Hierarchy(prob)
    F = H.finest
    b = F.disc.rhs()
    setup_s = time.perf_counter() - t0
    times, its, x, info = [], [], None, None
    while not times or sum(times) < budget_s:
        t0 = time.perf_counter()
        x, info = K.fgmres(lambda v: F.A @ v, H.vcycle, b, tol=TOL, m=RESTART, max_it=MAX_IT)
        times.append(time.perf_counter() - t0)
        its.append(info.iterations)
    fd, path = tempfile.mkstemp(suffix=".npz")
    os.close(fd)
    np.savez(path, x=x, active_cells=F.geom.active_cells, nb=F.nb)
    return dict(solve_ms=1e3 * statistics.mean(times), solves=len(times), iterations=its, setup_s=setup_s,
                n_dof=F.N, converged=bool(info.converged), solution=path)


def start_cpu_worker(workload, seed, budget_s):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-worker", workload, str(seed), str(budget_s)]
    return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.PIPE, env=env, cwd=ROOT)


def finish_cpu_worker(proc) -> dict | None:
    out, err = proc.communicate()
    if proc.returncode != 0:
        sys.stderr.write(err.decode(errors="replace")[-2000:])
        return None
    return json.loads(out.decode().strip().splitlines()[-1])


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={gpu_index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=self.file, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        self.proc.wait()
        self.file.seek(0)
        rows = [r.split(",") for r in self.file.read().strip().splitlines() if r.strip()]
        os.unlink(self.file.name)
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                smax = float(r[2])
                for k, name in enumerate(names):
                    if r[5 + k].strip().lower() == "active":
                        reasons.add(name)
            except (ValueError, IndexError):
                continue
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- helpers
def peaks():
    try:
        with open(PEAKS_FILE) as fh:
            d = json.load(fh)
        return d.get("hbm_gbs"), "measured"
    except (OSError, ValueError):
        return 6800.0, "fallback"


def committed_traffic(workload: str, kernel: str):
    """dram__bytes_read.sum + dram__bytes_write.sum per launch of `kernel` on `workload` from the
    committed ncu summary profiles/<kernel instantiation>_<workload>_traffic.txt, e.g.
    k_smooth_cell_2_2_float_star2d_p2_n512_traffic.txt (one line 'traffic_bytes_per_launch <B>'),
    or None when there is none."""
    import re
    name = re.sub(r"[^A-Za-z0-9]+", "_", kernel.split(" ")[0]).strip("_")
    path = os.path.join(ROOT, "profiles", f"{name}_{workload}_traffic.txt")
    try:
        with open(path) as fh:
            for line in fh:
                if line.startswith("traffic_bytes_per_launch"):
                    return int(float(line.split()[1]))
    except OSError:
        pass
    return None


def make_flush(torch):
    """L2 flush between timed launches: a 256 MB write (twice the 126 MB L2), then a 256 MB read of
    a second buffer, which writes the flush's dirty lines back and leaves L2 holding clean lines
    of neither the timed kernel's data nor anything it must write back."""
    wbuf = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")
    rbuf = torch.zeros(64 * 1024 * 1024, dtype=torch.float32, device="cuda")

    def flush():
        wbuf.fill_(1.0)
        rbuf.sum()
    return flush


def event_time(torch, fn, reps, flush=None):
    """Mean device time (ms) of fn() over reps launches on the current stream, after one untimed
    call (first calls allocate work buffers).  Before each start event the stream gets a ~50 us
    device-side sleep, so that the host's time to enqueue fn()'s launches (the Python call and the
    C-ABI entry) is spent while the GPU is still busy and is not counted as kernel time."""
    s = torch.cuda.current_stream()
    fn()
    torch.cuda.synchronize()
    total = 0.0
    for _ in range(reps):
        if flush is not None:
            flush()
        torch.cuda._sleep(100_000)             # ~50 us at 2 GHz: covers the host-side enqueue of fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        fn()
        e1.record(s)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    return total / reps


def reduce_max(value: float, device: str = "cuda") -> float:
    """Max of `value` over the ranks of the default process group (the job's time is the slowest
    rank's); the value itself without a process group or with one rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def timed_solves(torch, solver, b, x, n, flush):
    """n solves from x = 0 after an L2 flush each, CUDA events on the current stream: (ms list,
    info list)."""
    ts, infos = [], []
    for _ in range(n):
        x.zero_()
        flush()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = solver.solve(b, x, tol=TOL, restart=RESTART, max_it=MAX_IT)
        e1.record()
        e1.synchronize()
        ts.append(e0.elapsed_time(e1))
        infos.append(info)
    return ts, infos


def settings(prob) -> dict:
    """The discretisation and solver settings a workload runs with."""
    return {"sigma_F": f"{prob.sigma_face_c} (p_l+1)^2/h_l", "sigma_Gamma": f"{prob.sigma_bnd_c} (p_l+1)^2/h_l",
            "lambda": prob.lam, "active_test": ">=" if prob.lam_inclusive else ">", "alpha": prob.alpha,
            "extension": "u(x~)+d.grad u(x~) (first-order Taylor)" if prob.extension == 0
            else "cell polynomial at x~+d (full order)",
            "pre_smooth": prob.pre_smooth, "post_smooth": prob.post_smooth, "ssor_each": prob.ssor_each,
            "omega": prob.omega, "omega_p3": prob.omega_p3, "coarsest_n": prob.coarsest_n}


def smoother_bytes(w: int, N: int, n_bnd: int, npc: int, n_sface: int, nq: int, dim: int) -> float:
    """Algorithmic bytes of one full block Gauss-Seidel sweep: f read, u read, u written (3wN; the
    neighbours' values are counted once), the boundary cells' dense inverses and the shift vectors
    of the surrogate faces."""
    return 3 * w * N + n_bnd * npc * npc * w + n_sface * nq * dim * w


def apply_bytes(w: int, N: int, n_sface: int, nq: int, dim: int) -> float:
    """Algorithmic bytes of one operator apply: x read, y written, the surrogate-face shift vectors."""
    return 2 * w * N + n_sface * nq * dim * w


def large_mesh_rooflines(torch, S, hbm, flush, reps=10) -> list:
    """FP32 operator and smoother kernels on meshes whose vectors exceed L2, each launch after an L2
    flush: achieved GB/s from the algorithmic bytes, against the measured HBM copy bandwidth."""
    rows = []
    cases = (("star2d p=2 2048^2", W.star2d_p2(2048, 0), 2), ("sphere3d p=2 128^3", W.sphere3d(128, 2, 0), 2),
             ("ellipsoid3d p=3 96^3", W.ellipsoid3d_p3(96, 0), 1),
             # finest levels whose FP32 vectors are one to two times L2 and more
             ("star2d p=2 4096^2", W.star2d_p2(4096, 0), 1), ("sphere3d p=2 192^3", W.sphere3d(192, 2, 0), 1),
             ("ellipsoid3d p=3 128^3", W.ellipsoid3d_p3(128, 0), 1))
    for label, prob, nlev in cases:
        g = S.Solver(prob, "f32")
        L = g.num_levels - 1
        for level in range(L, L - nlev, -1):
            inf = g.info(level)
            N = inf["n_dof"]
            npc = (inf["p"] + 1) ** prob.dim
            nq = (inf["p"] + 1) ** (prob.dim - 1)
            ngrp = prob.dim + 1                  # launches per sweep (colour groups)
            f = torch.rand(N, device="cuda")
            u = torch.rand_like(f)
            y = torch.empty_like(f)
            t_apply = event_time(torch, lambda: g.apply(f, y, level=level), reps, flush)
            t_smooth = event_time(torch, lambda: g.smooth(f, u, level=level), reps, flush) / ngrp
            b_apply = apply_bytes(4, N, inf["n_sface"], nq, prob.dim)
            b_smooth = smoother_bytes(4, N, inf["n_boundary"], npc, inf["n_sface"], nq, prob.dim) / ngrp
            for kern, b, t in (("apply", b_apply, t_apply), ("smoother, mean launch of a sweep", b_smooth, t_smooth)):
                gbs = b / t / 1e6
                rows.append({"workload": label, "level": f"{inf['n']}^{prob.dim} p={inf['p']}", "n_dof": N,
                             "kernel": kern, "bytes": int(b), "ms": round(t, 5), "GB/s": round(gbs, 1),
                             "frac": round(gbs / hbm, 3)})
            del f, u, y
        g.close()
        torch.cuda.empty_cache()
    return rows


def other_workloads(torch, S, flush, n) -> dict:
    """The other benchmark configurations at full size: FP32-V-cycle and FP64-V-cycle solves (n
    timed each after one warm-up), iterations and residuals."""
    out = {}
    for name in ("disk2d_p1_n32", "sphere3d_p1_n64", "sphere3d_p2_n64", "ellipsoid3d_p3_n96"):
        prob = WORKLOADS[name](0)
        res = {"description": DESCRIPTION[name], "settings": settings(prob)}
        for prec in ("f32", "f64"):
            g = S.Solver(prob, prec)
            b = g.rhs()
            x = torch.zeros_like(b)
            timed_solves(torch, g, b, x, 1, flush)
            ts, infos = timed_solves(torch, g, b, x, n, flush)
            res["n_dof"] = b.numel()
            res[prec] = {"ms": round(statistics.mean(ts), 4), "iterations": infos[-1].iterations,
                         "converged": all(i.converged for i in infos),
                         "true_rel_residual": max(i.true_rel_residual for i in infos)}
            g.close()
        res["speedup_fp32_over_fp64_vcycle"] = round(res["f64"]["ms"] / res["f32"]["ms"], 3)
        out[name] = res
        torch.cuda.empty_cache()
    return out


SEED_CONFIGS = ("disk2d_p1_n32", "star2d_p2_n512", "sphere3d_p1_n64", "sphere3d_p2_n64", "ellipsoid3d_p3_n96")


def seed_study(torch, S, flush, seeds=5, n=5) -> dict:
    """Every benchmark configuration over seeds 0..seeds-1 (the seed moves the disk's and the
    sphere's centre, the star's phase and the ellipsoid's rotation): per seed the median of n timed
    solves after two warm-ups, FP32- and FP64-V-cycle; per configuration the median over the seeds,
    the spread (min, max) and the iteration counts per seed."""
    out = {}
    for name in SEED_CONFIGS:
        ms = {"f32": [], "f64": []}
        its = {"f32": [], "f64": []}
        converged = True
        for sd in range(seeds):
            prob = WORKLOADS[name](sd)
            for prec in ("f32", "f64"):
                g = S.Solver(prob, prec)
                b = g.rhs()
                x = torch.zeros_like(b)
                timed_solves(torch, g, b, x, 2, flush)
                ts, infos = timed_solves(torch, g, b, x, n, flush)
                ms[prec].append(statistics.median(ts))
                its[prec].append(infos[-1].iterations)
                converged = converged and all(i.converged for i in infos)
                g.close()
            torch.cuda.empty_cache()
        out[name] = {prec: {"median_ms": round(statistics.median(ms[prec]), 4), "min_ms": round(min(ms[prec]), 4),
                            "max_ms": round(max(ms[prec]), 4), "iterations": its[prec]} for prec in ("f32", "f64")}
        out[name]["converged"] = converged
    return {"seeds": list(range(seeds)), "timed_solves_per_seed": n, "configs": out}


def run_seed_study(args) -> dict:
    import torch
    import paper_2506_12899_gb300 as S
    return {"experiment": "solve time over seeds 0..4 per benchmark configuration",
            **seed_study(torch, S, make_flush(torch))}


def setup_times(S, reps=2) -> dict:
    """Wall time of sbm_setup (host build of every level, device uploads) for the 96^3 p=3 ellipsoid
    with the volume fractions and closest points on the device, and on the host cores."""
    out = {}
    prob = WORKLOADS["ellipsoid3d_p3_n96"](0)
    for label, flag in (("device_geometry", 1), ("host_geometry", -1)):
        ts = []
        for _ in range(reps):
            t0 = time.perf_counter()
            g = S.Solver(prob, "f32", device_geometry=flag)
            ts.append(time.perf_counter() - t0)
            g.close()
        out[label + "_s"] = round(min(ts), 3)
    out["workload"] = "ellipsoid3d_p3_n96"
    return out


def error_vs_oracle(solver, x, path) -> float | None:
    """||x - x_oracle|| / ||x_oracle|| with the oracle's solution from the CPU worker's file, mapped
    from the library's compact layout to the oracle's cell order by background cell index."""
    import numpy as np
    try:
        d = np.load(path)
    except OSError:
        return None
    xo, act, nb = d["x"], d["active_cells"], int(d["nb"])
    n, dim = solver.prob.n, solver.prob.dim
    c = solver.layout()
    lin = c[:, 0].astype(np.int64) + n * c[:, 1].astype(np.int64) + (n * n * c[:, 2].astype(np.int64) if dim == 3 else 0)
    pos = {int(v): i for i, v in enumerate(act)}
    cells = np.array([pos[int(v)] for v in lin])
    xg = x.cpu().numpy().reshape(-1, nb)
    xo = xo.reshape(-1, nb)[cells]
    return float(np.linalg.norm(xg - xo) / np.linalg.norm(xo))


def run_ours(args) -> dict | None:
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cpu_proc = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu_proc = start_cpu_worker(args.workload, 0, args.cpu_budget)   # spawned before any CUDA call
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import paper_2506_12899_gb300 as S

    prob = WORKLOADS[args.workload](rank)
    s32 = S.Solver(prob, "f32")
    s64 = S.Solver(prob, "f64")
    b = s32.rhs()
    x = torch.zeros_like(b)
    N = b.numel()
    flush = make_flush(torch)

    for _ in range(args.warmup):
        timed_solves(torch, s32, b, x, 1, flush)
        timed_solves(torch, s64, b, x, 1, flush)
    # ---- timed region: K FP32-V-cycle solves
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    launches0 = S.kernel_launches()
    times32, infos32 = timed_solves(torch, s32, b, x, args.steps, flush)
    launches = S.kernel_launches() - launches0
    torch.cuda.synchronize()
    clk = clocks.stop()
    if world > 1:
        dist.barrier()
    total_ms = reduce_max(sum(times32), "cuda")
    x32 = x.clone()                              # the last FP32-V-cycle solution
    # ---- FP64 V-cycle solves (the plain variant), same workload
    times64, infos64 = timed_solves(torch, s64, b, x, args.steps, flush)
    x64 = x.clone()
    # FP32-V-cycle solution against the FP64-V-cycle one; both are solved to the same FP64 residual
    err_vs_fp64 = float(torch.linalg.norm(x32 - x64) / torch.linalg.norm(x64))
    # ---- the FP32 V-cycle under FGMRES with the plain FP64 basis and FP64 operator (krylov_basis 1)
    sb1 = S.Solver(prob, "f32", krylov_basis=1)
    timed_solves(torch, sb1, b, x, 1, flush)
    tb1, ib1 = timed_solves(torch, sb1, b, x, args.steps, flush)
    fp64_basis = {"ms": round(statistics.mean(tb1), 4), "iterations": [i.iterations for i in ib1],
                  "converged": all(i.converged for i in ib1),
                  "true_rel_residual": max(i.true_rel_residual for i in ib1),
                  "variant": "FP32 V-cycle, FGMRES(30) with FP64 basis, FP64 Gram-Schmidt and FP64 operator"}
    sb1.close()
    # ---- the same workload with the full-order boundary extension (cell polynomial at x~ + d)
    # instead of the first-order Taylor term, FP32 V-cycle
    full_ext = None
    if prob.extension == 0 and prob.p >= 2:
        sfe = S.Solver(prob.replace(extension=1), "f32")
        bfe = sfe.rhs()
        xfe = torch.zeros_like(bfe)
        timed_solves(torch, sfe, bfe, xfe, 1, flush)
        tf, fe = timed_solves(torch, sfe, bfe, xfe, args.steps, flush)
        full_ext = {"ms": round(statistics.mean(tf), 4), "iterations": [i.iterations for i in fe],
                    "converged": all(i.converged for i in fe),
                    "true_rel_residual": max(i.true_rel_residual for i in fe)}
        sfe.close()
    # ---- learned variant: the boundary-cell MLP trained (untimed) on pairs collected from the
    # stationary V-cycle iteration on this hierarchy, attached with the fallback rule at the
    # plain solve's mean rate per step; the timed solves are otherwise identical
    learned = None
    if not args.no_learned:
        gen = torch.Generator(device="cuda").manual_seed(1000 + rank)
        mlp = S.Mlp(prob.dim, prob.p, 128, seed=rank)
        u0 = (2 * torch.rand((4, N), generator=gen, device="cuda", dtype=torch.float32) - 1).contiguous()
        pairs = s32.collect(mlp, u0, 3)
        rms = mlp.target_scale()                 # train on unit-RMS targets, attach with scale = RMS
        loss = mlp.train(epochs=20, batch=4096, lr=1e-3, seed=rank)
        its_plain = infos32[-1].iterations
        rate = infos32[-1].true_rel_residual ** (1.0 / max(its_plain, 1))
        s32.attach_mlp(mlp, rms, fallback_rate=rate)
        timed_solves(torch, s32, b, x, 1, flush)
        tl, il = timed_solves(torch, s32, b, x, args.steps, flush)
        s32.attach_mlp(None)
        learned = {"ms": round(statistics.mean(tl), 4), "iterations": [i.iterations for i in il],
                   "converged": all(i.converged for i in il), "fallback": [i.learned_fallback for i in il],
                   "train_pairs": pairs, "train_loss_relative_to_target_power": round(loss, 6),
                   "target_rms": rms, "fallback_rate": rate,
                   "mlp": "F-128-128-n_p ReLU, BF16 tensor-core GEMMs, Adam 20 epochs, batch 4096"}
    # ---- end to end through the host-buffer C-ABI call (copies inside the timed region)
    bh = torch.empty(N, dtype=torch.float64, pin_memory=True)
    xh = torch.empty(N, dtype=torch.float64, pin_memory=True)
    bh.copy_(b)
    bnp, xnp = bh.numpy(), xh.numpy()
    s32.solve_host(bnp, xnp, tol=TOL, restart=RESTART, max_it=MAX_IT)
    e2e = []
    for _ in range(args.steps):
        flush()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        s32.solve_host(bnp, xnp, tol=TOL, restart=RESTART, max_it=MAX_IT)
        e2e.append(1e3 * (time.perf_counter() - t0))
    # ---- per-kernel rooflines, each kernel timed alone with CUDA events on the solver's stream
    # after an L2 flush (finest level: FP32 as in the V-cycle; FP64 operator and Gram-Schmidt as in
    # FGMRES).  Algorithmic bytes count every vector once; flops are the method's FMAs x 2.
    info = s32.info()
    nb = (info["p"] + 1) ** prob.dim
    nq = (info["p"] + 1) ** (prob.dim - 1)
    r32 = torch.rand(N, device="cuda", dtype=torch.float32)
    u32 = torch.rand_like(r32)
    y32 = torch.empty_like(r32)
    xr64 = torch.rand(N, device="cuda", dtype=torch.float64)
    y64 = torch.empty_like(xr64)
    nv = 27                                      # Gram-Schmidt width at the last step of the bench solve
    V64 = torch.rand((nv, N), device="cuda", dtype=torch.float64)
    ngrp = prob.dim + 1                          # smoother launches per sweep (colour groups)
    # the p = 1 level on the same mesh (one below the finest), whose smoother is the kernel with
    # the largest share of the solve (three p = 1 levels, two sweeps of d + 1 launches per V-cycle)
    Lp1 = s32.num_levels - 2
    info1 = s32.info(Lp1)
    N1 = info1["n_dof"]
    nb1 = (info1["p"] + 1) ** prob.dim
    nq1 = (info1["p"] + 1) ** (prob.dim - 1)
    r1 = torch.rand(N1, device="cuda", dtype=torch.float32)
    u1 = torch.rand_like(r1)
    t_smooth1 = event_time(torch, lambda: s32.smooth(r1, u1, level=Lp1), 20, flush) / ngrp
    t_apply32 = event_time(torch, lambda: s32.apply(r32, y32), 20, flush)
    t_apply64 = event_time(torch, lambda: s64.apply(xr64, y64), 20, flush)
    t_smooth = event_time(torch, lambda: s32.smooth(r32, u32), 20, flush) / ngrp
    t_dots = event_time(torch, lambda: s64.dots(V64, xr64), 20, flush)
    hbm, src = peaks()
    fp64_tflops = 152 * 2.07e9 * 2 * 2 / 1e12    # SMs x max clock x 2 FP64 FMA/clk/SM x 2 flop
    kernels = {
        # one block Gauss-Seidel sweep moves f, u read, u written (3wN), the dense inverses of the
        # boundary cells and their face data; it takes d + 1 launches (colour groups), and the unit
        # is their mean
        f"k_smooth_cell<{prob.dim},{info1['p'] + 1},float> ({info1['n']}^{prob.dim} p={info1['p']} level, mean launch of a sweep)":
            ("hbm", smoother_bytes(4, N1, info1["n_boundary"], nb1, info1["n_sface"], nq1, prob.dim) / ngrp, t_smooth1),
        f"k_smooth_cell<{prob.dim},{info['p'] + 1},float> (finest level, mean launch of a sweep)":
            ("hbm", smoother_bytes(4, N, info["n_boundary"], nb, info["n_sface"], nq, prob.dim) / ngrp, t_smooth),
        f"k_apply_cell<{prob.dim},{info['p'] + 1},float> (FP32 operator, finest level)":
            ("hbm", apply_bytes(4, N, info["n_sface"], nq, prob.dim), t_apply32),
        f"k_apply<{prob.dim},{info['p'] + 1},double> (FP64 operator, finest level)":
            ("hbm", apply_bytes(8, N, info["n_sface"], nq, prob.dim), t_apply64),
        # sbm_dots: the FP64 multi-vector dot product (the solver's own sweeps run in double-float)
        "k_multi_dot<27> (FP64, sbm_dots)": ("alu", 2 * nv * N, t_dots),
    }
    rooflines = {}
    for k, (bound, amount, t_) in kernels.items():
        if bound == "hbm":
            ach = amount / t_ / 1e6
            rooflines[k] = {"bound": "hbm", "achieved": round(ach, 1), "peak": hbm, "unit": "GB/s",
                            "frac": round(ach / hbm, 3), "bytes_per_launch": int(amount), "ms_per_launch": t_}
        else:
            ach = amount / t_ / 1e9
            rooflines[k] = {"bound": "alu", "achieved": round(ach, 4), "peak": round(fp64_tflops, 4),
                            "unit": "TFLOP/s", "frac": round(ach / fp64_tflops, 3), "flops_per_launch": int(amount),
                            "ms_per_launch": t_, "bytes_per_launch": 8 * (nv + 1) * N}
    dominant = next(iter(kernels))
    roof = dict(rooflines[dominant])
    roof.update(kernel=dominant, peak_source=src, traffic=committed_traffic(args.workload, dominant))
    del r32, u32, y32, xr64, y64, V64, r1, u1
    torch.cuda.empty_cache()
    # ---- the other benchmark configurations, and the kernels on meshes larger than L2
    others = large = setup = seeds = None
    if not args.no_extra:
        others = other_workloads(torch, S, flush, 5)
        large = large_mesh_rooflines(torch, S, hbm, flush)
        setup = setup_times(S)
        seeds = seed_study(torch, S, flush)
    if rank != 0:
        return None
    cpu = finish_cpu_worker(cpu_proc) if cpu_proc is not None else None
    ms32 = total_ms / args.steps
    its32 = [i.iterations for i in infos32]
    out = {
        "metric": METRIC, "value": round(ms32, 4), "unit": "ms", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms32, 4), "step_ms": [round(t, 3) for t in times32],
        "higher_is_better": False, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": args.workload, "description": DESCRIPTION.get(args.workload, args.workload),
                   "n_dof": N, "levels": s32.num_levels,
                   "variant": "FP32 V-cycle; FGMRES(30) with a double-float basis (FP32 pairs, ~48-bit "
                              "significands), Gram-Schmidt and Arnoldi operator on the FP32 pipes; FP64 true residual",
                   "settings": settings(prob),
                   "l2": "flushed (256 MB write, then a 256 MB read of another buffer) before every step", "parallelism": f"replicas x{world}"},
        "iterations": its32, "converged": all(i.converged for i in infos32),
        "true_rel_residual": max(i.true_rel_residual for i in infos32),
        "fp64_vcycle": {"ms": round(statistics.mean(times64), 4), "iterations": [i.iterations for i in infos64],
                        "converged": all(i.converged for i in infos64)},
        "fp64_basis": fp64_basis,
        "rel_l2_error_vs_fp64_vcycle_solution": err_vs_fp64,
        "speedup_fp32_over_fp64_vcycle": round(statistics.mean(times64) / ms32, 3),
        "learned": learned,
        "full_order_extension": full_ext,
        "solves_per_s_total": round(world * args.steps / (total_ms / 1e3), 3),
        "apply_gbs": {"fp32": list(rooflines.values())[2]["achieved"],
                      "fp64": list(rooflines.values())[3]["achieved"]},
        "clocks": clk,
        "e2e": {"value": round(statistics.mean(e2e), 4), "unit": "ms", "h2d_bytes_per_step": 8 * N,
                "d2h_bytes_per_step": 8 * N},
        "gpu_launches": int(launches),
        "roofline": roof,
        "rooflines": rooflines,
        "rooflines_large_meshes": large,
        "other_workloads": others,
        "seed_study": seeds,
        "setup_time": setup,
    }
    if cpu is not None:
        path = cpu["solution"]
        out["rel_l2_error_vs_oracle"] = {"fp32_vcycle": error_vs_oracle(s32, x32, path),
                                         "fp64_vcycle": error_vs_oracle(s32, x64, path),
                                         "oracle_iterations": cpu["iterations"][-1]}
        os.unlink(path)
        out["cpu_baseline"] = {"value": round(cpu["solve_ms"], 1), "unit": "ms", "cores": 1, "kind": "oracle",
                               "sample": f"{cpu['solves']} whole FGMRES(30) solves to 1e-8 of the same workload "
                                         f"by the FP64 oracle on one host core ({cpu['iterations'][-1]} iterations "
                                         f"each), mean; oracle set-up {cpu['setup_s']:.0f} s not timed"}
    return out


def run_profile(args) -> None:
    """Fixed launch sequences for ncu captures (numbers printed under ncu are not bench values).
    solve:   one warm-up and one FP32-V-cycle FGMRES solve of --workload; prints how many of the
             library's kernels the warm-up launched (the ncu skip count) and how many the solve did.
    mlp:     the 3D p=3 MLP (F = 2023, H = 128, O = 64): one forward and one gradient pass on
             --profile-n random rows.
    kernels: 2D p=2 star at --profile-n^2 cells (or the 3D sphere of degree --profile-p, or the
             3D p=3 ellipsoid, at --profile-n^3): one FP32 operator apply and one smoother sweep
             (d+1 colour-group launches) on the level --profile-level below the finest, and one
             V-cycle when that is the finest."""
    import torch
    import paper_2506_12899_gb300 as S
    if args.profile == "mlp":                    # the learned part's GEMMs: one forward and one gradient pass
        mlp = S.Mlp(3, 3, 128, seed=0)
        gen = torch.Generator(device="cuda").manual_seed(0)
        rows = args.profile_n
        X = (2 * torch.rand((rows, mlp.F), generator=gen, device="cuda") - 1).contiguous()
        T = torch.randn((rows, mlp.O), generator=gen, device="cuda").contiguous()
        mlp.forward(X)
        loss, _ = mlp.gradients(X, T)
        torch.cuda.synchronize()
        print("ROWS", rows, "F", mlp.F, "H", mlp.H, "O", mlp.O, "LOSS", loss, flush=True)
        return
    if args.profile == "solve":
        g = S.Solver(WORKLOADS[args.workload](0), "f32", krylov_basis=args.krylov_basis)
        b = g.rhs()
        x = torch.zeros_like(b)
        l0 = S.kernel_launches()
        g.solve(b, x, tol=TOL, restart=RESTART, max_it=MAX_IT)
        l1 = S.kernel_launches()
        x.zero_()
        info = g.solve(b, x, tol=TOL, restart=RESTART, max_it=MAX_IT)
        torch.cuda.synchronize()
        print("WARM_LAUNCHES", l1 - l0, flush=True)
        print("SOLVE_LAUNCHES", S.kernel_launches() - l1, flush=True)
        print("ITERATIONS", info.iterations, "CONVERGED", info.converged, flush=True)
    else:
        prob = {"star2d": lambda: W.star2d_p2(args.profile_n, 0),
                "sphere3d": lambda: W.sphere3d(args.profile_n, args.profile_p, 0),
                "ellipsoid3d": lambda: W.ellipsoid3d_p3(args.profile_n, 0)}[args.profile_shape]()
        g = S.Solver(prob, "f32", tail_max_cells=args.tail_max_cells, tail_cluster_ctas=args.tail_cluster,
                     staged_min_cells=args.staged_min)
        lev = g.num_levels - 1 - args.profile_level
        N = g.info(lev)["n_dof"]
        gen = torch.Generator(device="cuda").manual_seed(0)
        f = torch.rand(N, device="cuda", generator=gen)
        u = torch.rand(N, device="cuda", generator=gen)
        y = torch.empty_like(f)
        g.apply(f, y, level=lev)
        g.smooth(f, u, level=lev)
        if lev == g.num_levels - 1:
            g.vcycle(f, y)
        torch.cuda.synchronize()
        print("N", N, "LEVELS", g.num_levels, "LEVEL", lev, flush=True)


def run_learned_heldout(args) -> dict:
    """a7 on a family of domains: the MLP is trained on pairs collected from the training seeds
    (4 seeded starts x 3 stationary V-cycle steps each), then every held-out domain is solved
    plain, with the learned correction and the fallback rule, and with the correction forced on.
    Reports FGMRES iterations and device times (FP32 V-cycle, FP64 FGMRES, tol 1e-8)."""
    import torch
    import paper_2506_12899_gb300 as S
    dim = 2 if args.family == "star2d" else 3
    make = (lambda sd: W.random_star2d_p3(128, sd)) if dim == 2 else (lambda sd: W.random_ellipsoid3d_p3(32, sd))
    mlp = S.Mlp(dim, 3, 128, seed=0)
    gen = torch.Generator(device="cuda").manual_seed(0)
    t0 = time.perf_counter()
    pairs = 0
    for sd in range(1000, 1000 + args.n_train):
        g = S.Solver(make(sd), "f32")
        u0 = (2 * torch.rand((4, g.n_dof()), generator=gen, device="cuda", dtype=torch.float32) - 1).contiguous()
        pairs += g.collect(mlp, u0, 3)
        g.close()
    collect_s = time.perf_counter() - t0
    rms = mlp.target_scale()                     # unit-RMS targets; the correction is attached with scale = RMS
    t0 = time.perf_counter()
    loss = mlp.train(epochs=20, batch=4096, lr=1e-3, seed=0)
    train_s = time.perf_counter() - t0

    def timed(g, b, x):
        x.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        info = g.solve(b, x, tol=TOL, restart=RESTART, max_it=MAX_IT)
        e1.record()
        e1.synchronize()
        return info, e0.elapsed_time(e1)

    rows = []
    evals = [(sd, make(sd)) for sd in range(2000, 2000 + args.n_eval)]
    if args.eval_workload:
        evals.append((args.eval_workload, WORKLOADS[args.eval_workload](0)))
    for sd, prob_e in evals:
        g = S.Solver(prob_e, "f32")
        b = g.rhs()
        x = torch.zeros_like(b)
        timed(g, b, x)
        plain, tp = timed(g, b, x)
        rate = plain.true_rel_residual ** (1.0 / max(plain.iterations, 1))
        g.attach_mlp(mlp, rms, fallback_rate=rate)
        timed(g, b, x)
        gated, tg = timed(g, b, x)
        g.attach_mlp(mlp, rms, fallback_rate=0.0)
        timed(g, b, x)
        forced, tf = timed(g, b, x)
        g.attach_mlp(None)
        rows.append({"seed": sd, "plain": [plain.iterations, round(tp, 3)],
                     "learned_gated": [gated.iterations, round(tg, 3), gated.learned_fallback, gated.converged],
                     "learned_forced": [forced.iterations, round(tf, 3), forced.converged]})
        g.close()
    extra = [r for r in rows if not isinstance(r["seed"], int)]
    rows = [r for r in rows if isinstance(r["seed"], int)]
    med = lambda k, i: statistics.median(r[k][i] for r in rows) if rows else None
    return {"experiment": f"learned boundary correction, held-out {args.family} p=3", "train_seeds": args.n_train,
            "eval_seeds": args.n_eval, "train_pairs": pairs, "target_rms": rms,
            "train_loss_relative_to_target_power": loss, "collect_s": round(collect_s, 1),
            "train_s": round(train_s, 1),
            "median_iterations": {"plain": med("plain", 0), "learned_gated": med("learned_gated", 0),
                                  "learned_forced": med("learned_forced", 0)},
            "median_ms": {"plain": med("plain", 1), "learned_gated": med("learned_gated", 1),
                          "learned_forced": med("learned_forced", 1)},
            "fallbacks": sum(1 for r in rows if r["learned_gated"][2]), "workload_eval": extra, "rows": rows}


def run_roofline_sweep(args) -> dict:
    """Operator and smoother kernels on meshes whose FP32 vectors exceed L2 (the bench workload's
    fit in L2): CUDA-event time per launch after an L2 flush, algorithmic bytes (every vector
    entry once), achieved GB/s against the measured HBM copy bandwidth."""
    import torch
    import paper_2506_12899_gb300 as S
    hbm, src = peaks()
    rows = large_mesh_rooflines(torch, S, hbm, make_flush(torch))
    return {"experiment": "FP32 operator / smoother roofline sweep (vectors > L2)", "peak_gbs": hbm,
            "peak_source": src, "l2": "flushed (256 MB write, then a 256 MB read of another buffer) before every launch", "rows": rows}


def run_paper_replica(args) -> dict:
    """The paper's unit-disk / unit-sphere study (Sec. 5): [-1.01,1.01]^d with 4*2^level cells,
    kappa > lambda, polynomial boundary extension, u = 2 cos x sin y, FP64 V-cycle, GMRES tolerance
    1e-12 and a cap of 100 iterations, omega = 0.8 at p = 3.  Reports iteration counts per
    (dim, p, lambda, level) for three readings of the paper's solver settings:
      base:       sigma_F = (p+1)^2/h, sigma_Gamma = 5 (p+1)^2/h, one forward sweep before and one
                  reverse sweep after the coarse correction (the cell-wise SSOR split over the V);
      ssor:       the same penalties, a full SSOR step (forward + reverse) before and after;
      sipg_ssor:  full SSOR steps with the interior penalty sigma_F = p(p+1)/h (p^2/h at p >= 2),
                  sigma_Gamma = 5 (p+1)^2/h."""
    import torch
    import paper_2506_12899_gb300 as S
    plan = [(2, 1, range(1, 8)), (3, 1, range(1, 5)), (2, 2, range(1, 7)), (3, 2, range(1, 5)), (2, 3, range(1, 6))]
    readings = {"base": dict(ssor_each=0), "ssor": dict(ssor_each=1), "sipg_ssor": dict(ssor_each=1, sipg=True)}
    rows = []
    for dim, p, levels in plan:
        for lam in (1.0, 0.75, 0.5, 0.25):
            for name, rd in readings.items():
                its = []
                for lev in levels:
                    prob = W.paper_disk(lev, p, lam, dim).replace(ssor_each=rd["ssor_each"])
                    if rd.get("sipg"):
                        cf = (p * (p + 1) if p == 1 else p * p) / (p + 1) ** 2
                        prob = prob.replace(sigma_face_c=cf)
                    if p == 3:
                        prob = prob.replace(omega_p3=0.8)
                    try:
                        g = S.Solver(prob, "f64")
                        b = g.rhs()
                        x = torch.zeros_like(b)
                        info = g.solve(b, x, tol=1e-12, restart=30, max_it=100)
                        its.append(info.iterations if info.converged else 100)
                        g.close()
                    except Exception as e:                # e.g. no active cell on a coarse level
                        its.append(str(e)[:40])
                rows.append({"dim": dim, "p": p, "lambda": lam, "reading": name, "iterations_by_level": its})
    return {"experiment": "paper replica: unit disk/sphere iteration counts (tol 1e-12, cap 100)", "rows": rows}


def run_complex2d(args) -> dict:
    """The complex deformed domain of Sec. 5.4 on the GPU: phi = (1 - 3/4 sin^2(pi x))(x^2 + y^2) - 1/5,
    u = phi + 1, [-1.01,1.01]^2 with 4*2^level cells, lambda in {1, .75, .5, .25}, p = 1..3; FP64
    V-cycle, GMRES tolerance 1e-12 and a cap of 100 iterations; the iteration count and the L2 error
    ||u - u_h|| over the surrogate domain (sbm_l2_error) of each solve."""
    import torch
    import paper_2506_12899_gb300 as S
    rows = []
    for p, levels in ((1, range(1, 8)), (2, range(1, 8)), (3, range(1, 7))):
        for lam in (1.0, 0.75, 0.5, 0.25):
            its, errs = [], []
            for lev in levels:
                prob = W.paper_complex2d(lev, p, lam)
                if p == 3:
                    prob = prob.replace(omega_p3=0.8)
                try:
                    g = S.Solver(prob, "f64")
                    b = g.rhs()
                    x = torch.zeros_like(b)
                    info = g.solve(b, x, tol=1e-12, restart=30, max_it=100)
                    its.append(info.iterations if info.converged else 100)
                    errs.append(float(f"{g.l2_error(x):.4e}"))
                    g.close()
                except Exception as e:
                    its.append(str(e)[:40])
                    errs.append(None)
            rows.append({"p": p, "lambda": lam, "iterations_by_level": its, "l2_error_by_level": errs})
    return {"experiment": "complex deformed 2D domain (Sec. 5.4): iterations (tol 1e-12, cap 100) and L2 errors",
            "rows": rows}


def run_reference(args) -> dict | None:
    """The reference arm: the CPU FP64 oracle on the host cores (no GPU); each step is one whole
    FGMRES(30) solve to 1e-8 from x = 0 (set-up untimed)."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return None
    from oracle import krylov as K
    from oracle import multigrid as MG
    prob = WORKLOADS[args.workload](0)
    H = MG.Hierarchy(prob)
    F = H.finest
    b = F.disc.rhs()
    times, info = [], None
    for k in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        _x, info = K.fgmres(lambda v: F.A @ v, H.vcycle, b, tol=TOL, m=RESTART, max_it=MAX_IT)
        if k >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * statistics.mean(times)
    cores = 1                                    # single-threaded BLAS, scalar Python loops
    return {"impl": "reference", "metric": METRIC, "value": round(ms, 1), "unit": "ms", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms, 1), "higher_is_better": False,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "description": DESCRIPTION.get(args.workload, args.workload),
                       "n_dof": F.N, "settings": settings(prob),
                       "variant": "CPU FP64 oracle: assembled CSR, coloured block GS V-cycle, FGMRES(30)"},
            "iterations": info.iterations, "converged": info.converged,
            "cpu_baseline": {"value": round(ms, 1), "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": f"each step one whole FGMRES(30) solve of the workload to 1e-8 "
                                       f"({info.iterations} iterations); oracle set-up not timed"},
            "e2e": {"value": round(ms, 1), "unit": "ms", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    if len(sys.argv) > 1 and sys.argv[1] == "--cpu-worker":
        workload, seed, budget = sys.argv[2], int(sys.argv[3]), float(sys.argv[4])
        print(json.dumps(cpu_worker(workload, seed, budget)))
        return
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="star2d_p2_n512", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-budget", type=float, default=10.0, help="seconds of whole oracle solves to time")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-correction variant")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the other workloads and the large-mesh rooflines in the bench line")
    ap.add_argument("--profile", choices=["solve", "kernels", "mlp"], help="fixed launches for an ncu capture")
    ap.add_argument("--profile-n", type=int, default=2048, help="cells per direction for --profile kernels")
    ap.add_argument("--profile-shape", default="star2d", choices=["star2d", "sphere3d", "ellipsoid3d"],
                    help="--profile kernels: 2D p=2 star, 3D sphere (degree --profile-p) or 3D p=3 ellipsoid")
    ap.add_argument("--staged-min", type=int, default=0,
                    help="--profile kernels: staged thread-per-cell kernels from this many cells (<0 never)")
    ap.add_argument("--profile-p", type=int, default=2)
    ap.add_argument("--profile-level", type=int, default=0,
                    help="--profile kernels: level below the finest (0: finest, with one V-cycle)")
    ap.add_argument("--tail-max-cells", type=int, default=0, help="--profile kernels: cluster-tail cut-off")
    ap.add_argument("--tail-cluster", type=int, default=0, help="--profile kernels: cluster-tail CTAs")
    ap.add_argument("--krylov-basis", type=int, default=0, choices=[0, 1],
                    help="--profile solve: FGMRES basis storage (0 double-float, 1 FP64)")
    ap.add_argument("--experiment", choices=["learned-heldout", "roofline-sweep", "paper-replica", "complex2d", "seeds"],
                    help="a7 on held-out domains, or the large-mesh roofline sweep (no bench line)")
    ap.add_argument("--family", default="star2d", choices=["star2d", "ellipsoid3d"])
    ap.add_argument("--n-train", type=int, default=256)
    ap.add_argument("--n-eval", type=int, default=32)
    ap.add_argument("--eval-workload", choices=sorted(WORKLOADS), help="also evaluate the trained MLP on this workload")
    args = ap.parse_args()
    if args.experiment:
        run = {"learned-heldout": run_learned_heldout, "roofline-sweep": run_roofline_sweep,
               "paper-replica": run_paper_replica, "complex2d": run_complex2d,
               "seeds": run_seed_study}[args.experiment]
        print(json.dumps(run(args)))
        return
    if args.profile:
        run_profile(args)
        return
    out = run_reference(args) if args.impl == "reference" else run_ours(args)
    if out is not None:
        print(json.dumps(out))
    if int(os.environ.get("WORLD_SIZE", "1")) > 1 and args.impl == "ours":
        import torch.distributed as dist
        if dist.is_initialized():
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
