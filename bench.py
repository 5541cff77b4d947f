"""Benchmark: Newton iterations per second of the implicit octree GIMP MPM load
step on one GB300, FP32+refinement vs FP64, with the HBM roofline of the
dominant kernel.

A step is one quasi-static load step of the indentation workload: rebuild of
the adapted octree, GIMP split, discrete GIMP basis, block pattern and ghost
matrix, then Newton-Raphson (assembly, Krylov solve, line search) to a 1e-8
residual, then the point update.  value = Newton iterations / second over the
timed steps of the mixed-precision path; the FP64 path is timed on the same
steps.  Multi-GPU runs are independent replicas (the path has no data-parallel
exchange at this level), so scaling is weak.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "indent"
SOLVER = 3
CPU_SAMPLE = dict(depth_min=4, depth_max=5, dx_region=2.0 / 32,
                  points=dict(spacing=1.0 / 32, jitter=1.0 / 128))
PROF_NAMES = ["pcg_update", "pcg_spmv", "tangent_rows", "constitutive", "kinematics", "force",
              "basis", "residual_rows", "contact", "bicgstab_spmv", "refine_residual", "pattern",
              "multigrid_vcycle", "multigrid_setup"]
NPROF = len(PROF_NAMES)
METRIC = "Newton iters/s at ~1M DOF: FP32+refine vs FP64 (1e-8 residual); HBM roofline %"


def args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--method", type=int, default=SOLVER,
                    help="Krylov method of mpm_solve_params (1 block-Jacobi PCG, 3 multigrid PCG)")
    ap.add_argument("--inner-tol", type=float, default=1e-4,
                    help="mixed precision: relative target of each FP32 inner solve")
    ap.add_argument("--mg-reuse", type=int, default=1,
                    help="method 3: keep the coarse operators across the Newton iterations of a step")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return p["hbm_gbs"], "measured"
    except Exception:
        return 6800.0, "fallback"


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", delete=False, suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(index), "--query-gpu=" + q,
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as f:
            for line in f:
                v = [x.strip() for x in line.split(",")]
                if len(v) >= 9:
                    rows.append(v)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_sample_cfg(workload):
    from paper_2606_09275_gb300 import inputs
    return inputs.workload(workload, **CPU_SAMPLE)


def run_oracle_sample(workload, nsteps):
    """The oracle as it stands, on a bounded sample of the same workload recipe."""
    import oracle
    from paper_2606_09275_gb300 import inputs
    cfg = cpu_sample_cfg(workload)
    pts = inputs.make_points(cfg)
    m = oracle.Model(cfg, pts)
    its, t0 = 0, time.perf_counter()
    dof = 0
    for n in range(1, nsteps + 1):
        m.set_body_z(inputs.body_z(cfg, n))
        st = m.step(load=1.0, tol=cfg["newton_tol"], lin_tol=cfg["lin_tol"],
                    lin_maxit=cfg["lin_maxit"])
        if st["status"]:
            raise RuntimeError("oracle sample step failed: %d" % st["status"])
        its += st["newton_its"]
        dof = 3 * m.counts()["ndof"]
    dt = time.perf_counter() - t0
    sample = ("oracle load steps 1-%d of the %s recipe at depth %d->%d (%d points, %d DOF), "
              "one host thread" % (nsteps, workload, cfg["depth_min"], cfg["depth_max"],
                                   m.counts()["npts"], dof))
    return its / dt, dt, sample, its


def reference_main(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps = max(1, a.steps)
    # warm-up: the first load step of the sample (untimed)
    run_oracle_sample(a.workload, 1)
    v, dt, sample, its = run_oracle_sample(a.workload, steps)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Newton it/s",
            "n_gpus": a.gpus, "steps": steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": a.workload + " (bounded CPU sample)", "sample": sample},
            "cpu_baseline": {"value": v, "unit": "Newton it/s", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": v, "unit": "Newton it/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def spmv_bytes(nnzb, nd, mixed):
    """Algorithmic bytes of one fused PCG SpMV launch: matrix values and column
    indices once, row pointers, and z, p, q (p and q read and written)."""
    w = 4 if mixed else 8
    return nnzb * (9 * w + 4) + 4 * (nd + 1) + 5 * 3 * nd * w


def traffic_record(kernel):
    """ncu DRAM bytes per launch of the kernel, if captured for the current source."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    r = rec.get(kernel)
    if not r:
        return None
    with open(os.path.join(ROOT, r["source"])) as f:
        src = f.read()
    txt = ""
    for name in r["kernels"]:
        i = src.find("__global__ void " + name)
        if i < 0:
            return None
        txt += src[i:src.index("\n}\n", i) + 3]
    if hashlib.sha256(txt.encode()).hexdigest()[:16] != r["source_sha"]:
        return None  # the kernel changed since the counters were taken
    return r


def replica_totals(its, ms, world, dev):
    """Whole-job totals of N independent replicas (one per rank): the Newton
    iterations summed over the ranks and the time of the slowest rank."""
    if world == 1:
        return its, ms
    import torch
    import torch.distributed as dist
    t_its = torch.tensor([float(its)], dtype=torch.float64, device=dev)
    t_ms = torch.tensor([float(ms)], dtype=torch.float64, device=dev)
    dist.all_reduce(t_its, op=dist.ReduceOp.SUM)
    dist.all_reduce(t_ms, op=dist.ReduceOp.MAX)
    return int(round(t_its.item())), float(t_ms.item())


def adjoint_leg(dev, method):
    """Cost of the discrete adjoint against the forward run it differentiates:
    the punch at depth 3 -> 5 with lognormal E, 20 load steps, FP64, gradient
    of the final vertical punch reaction in every point's E and yield stress."""
    import torch

    from paper_2606_09275_gb300 import autodiff, inputs, mpm
    cfg = inputs.workload("adjoint")
    pts = inputs.make_points(cfg)
    ctx = mpm.Context()
    path = autodiff.LoadPath(ctx, cfg, pts, cfg["nsteps"], tol=cfg["newton_tol"],
                             lin_tol=cfg["lin_tol"], lin_maxit=cfg["lin_maxit"], method=method,
                             mg_reuse=1)
    E = torch.tensor(pts["E"], device=dev)
    ys = torch.tensor(pts["ys"], device=dev)
    path.run(E, ys, keep=False)  # warm-up (allocations, module load)
    stream = torch.cuda.current_stream()
    e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
    e[0].record(stream)
    _, _, st_plain = path.run(E, ys, keep=False)
    e[1].record(stream)
    _, ckpts, _ = path.run(E, ys, keep=True)
    e[2].record(stream)
    dE, dys, ast = path.gradient(ckpts, (0.0, 0.0, 1.0))
    e[3].record(stream)
    torch.cuda.synchronize()
    n = cfg["nsteps"]
    fwd, fwd_ck, adj = (e[0].elapsed_time(e[1]), e[1].elapsed_time(e[2]), e[2].elapsed_time(e[3]))
    ctx.close()
    return {"workload": "adjoint: flat punch into a von Mises block 1x1x0.5 m, depth 3 -> 5, "
                        "lognormal E (sigma 0.2), %d load steps, FP64, d(reaction_z)/d(E, ys)" % n,
            "points_last_step": st_plain[-1]["npts"], "dof_last_step": st_plain[-1]["ndof"],
            "forward_ms_per_step": round(fwd / n, 3),
            "forward_with_checkpoints_ms_per_step": round(fwd_ck / n, 3),
            "adjoint_ms_per_step": round(adj / n, 3),
            "adjoint_over_forward": round(adj / fwd, 3),
            "adjoint_resolve_ms_per_step": round(ast["ms_forward"] / n, 3),
            "adjoint_backward_ms_per_step": round(ast["ms_backward"] / n, 3),
            "adjoint_krylov_its": ast["lin_its"], "krylov_method": method,
            "forward_krylov_its": int(sum(s["lin_its"] for s in st_plain))}


def gpu_main(a):
    import torch
    import torch.distributed as dist

    from paper_2606_09275_gb300 import inputs, mpm

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    cfg = inputs.workload(a.workload)
    pts0 = inputs.make_points(cfg)
    P0 = len(pts0["x"])
    cap = 2 * P0
    W, K = a.warmup, a.steps
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def arm(precision, profile=False, e2e=False):
        ctx = mpm.Context()
        P = mpm.Points(pts0, capacity=cap, device=dev)
        host = None
        if e2e:
            host = {k: torch.empty_like(t, device="cpu").pin_memory() for k, t in P.t.items()}
            for k in host:
                host[k].copy_(P.t[k])
        step_kw = dict(load=1.0, tol=cfg["newton_tol"], maxit=cfg["newton_maxit"],
                       lin_tol=cfg["lin_tol"], lin_maxit=cfg["lin_maxit"], precision=precision,
                       method=a.method, mg_reuse=a.mg_reuse, inner_tol=a.inner_tol)
        for n in range(1, W + 1):
            mpm.step(ctx, cfg, P, body_z=inputs.body_z(cfg, n), **step_kw)
        if e2e:
            for k in host:
                host[k].copy_(P.t[k])
        barrier()
        clk = Clocks(local) if (rank == 0 and not e2e) else None
        if profile:
            mpm.lib().mpm_profile(ctx.h, 1)
        nl0 = mpm.C.c_longlong(0)
        mpm.lib().mpm_launch_count(ctx.h, mpm.C.byref(nl0))
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        its, stats, h2d, d2h = 0, [], 0, 0
        ev0.record(stream)
        for n in range(W + 1, W + K + 1):
            if e2e:
                cnt = P.count
                for k, t in P.t.items():
                    t[:cnt].copy_(host[k][:cnt], non_blocking=True)
                    h2d += host[k][:cnt].numel() * 8
            st = mpm.step(ctx, cfg, P, body_z=inputs.body_z(cfg, n), **step_kw)
            its += st["newton_its"]
            stats.append(st)
            if e2e:
                cnt = P.count
                for k, t in P.t.items():
                    host[k][:cnt].copy_(t[:cnt], non_blocking=True)
                    d2h += t[:cnt].numel() * 8
        ev1.record(stream)
        torch.cuda.synchronize()
        ms = ev0.elapsed_time(ev1)
        nl1 = mpm.C.c_longlong(0)
        mpm.lib().mpm_launch_count(ctx.h, mpm.C.byref(nl1))
        prof = None
        if profile:
            L = (mpm.C.c_longlong * NPROF)()
            T = (mpm.C.c_double * NPROF)()
            mpm.lib().mpm_profile_read(ctx.h, L, T)
            mpm.lib().mpm_profile(ctx.h, 0)
            prof = {"launches": list(L), "ms": list(T)}
        clocks = clk.stop() if clk else None
        barrier()
        its_all, ms = replica_totals(its, ms, world, dev)
        ctx.close()
        return dict(ms=ms, its=its, its_all=its_all, stats=stats, prof=prof, clocks=clocks,
                    launches=nl1.value - nl0.value, h2d=h2d // max(K, 1), d2h=d2h // max(K, 1))

    mixed = arm(mpm.MIXED, profile=True)
    fp64 = None if a.no_fp64 else arm(mpm.FP64)
    e2e = None if a.no_e2e else arm(mpm.MIXED, e2e=True)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    value = mixed["its_all"] / (mixed["ms"] * 1e-3)
    last = mixed["stats"][-1]
    nnzb = np.mean([s["nnzb"] for s in mixed["stats"]])
    nd = np.mean([s["ndof"] for s in mixed["stats"]]) / 3.0
    names = PROF_NAMES
    prof = mixed["prof"]
    kern = {n: {"launches": prof["launches"][i], "ms": round(prof["ms"][i], 3)}
            for i, n in enumerate(names) if prof["launches"][i]}
    dom = max(kern, key=lambda n: kern[n]["ms"])
    peak, peak_src = peaks()
    i_spmv = names.index("pcg_spmv")
    roof = None
    if prof["launches"][i_spmv]:
        avg_ms = prof["ms"][i_spmv] / prof["launches"][i_spmv]
        B = spmv_bytes(nnzb, nd, True)
        ach = B / (avg_ms * 1e-3) / 1e9
        tr = traffic_record("k_pcg_b<float,float>")
        roof = {"kernel": "k_pcg_b<float,float> (PCG SpMV, FP32 3x3 BSR)", "bound": "hbm",
                "achieved": round(ach, 1), "peak": peak, "unit": "GB/s",
                "frac": round(ach / peak, 4), "peak_source": peak_src,
                "traffic": (round(tr["bytes_per_launch"] * B / tr["alg_bytes_per_launch"])
                            if tr else None),
                "algorithmic_bytes_per_launch": int(B), "avg_launch_ms": round(avg_ms, 5),
                "dominant_kernel_by_time": dom}
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "Newton it/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": round(mixed["ms"] / K, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (FP32 tangent and inner PCG; FP64 residual, dF, return map, refinement)",
        "data": "synthetic",
        "config": {"workload": "%s: flat punch (r 0.1 m) into a von Mises block 1x1x0.875 m, "
                               "octree depth 6 refined to 7 at the punch, jittered 2x2x2 points "
                               "per cell" % a.workload,
                   "points": last["npts"], "dof": last["ndof"], "nnzb": last["nnzb"],
                   "newton_tol": cfg["newton_tol"], "krylov_tol": cfg["lin_tol"],
                   "krylov": {1: "block-Jacobi PCG", 3: "multigrid-preconditioned PCG"}.get(
                       a.method, "method %d" % a.method),
                   "mixed_inner_tol": a.inner_tol, "mg_reuse": a.mg_reuse,
                   "step": "one load step: mesh rebuild + Newton to 1e-8 + point update",
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (stiffness %.2f GB FP32)" % (nnzb * 40 / 1e9)},
        "newton_its": mixed["its"], "krylov_its": sum(s["lin_its"] for s in mixed["stats"]),
        "solver_only": {
            "value": round(mixed["its_all"] / (1e-3 * sum(
                s["ms_assemble"] + s["ms_solve"] for s in mixed["stats"])), 4),
            "unit": "Newton it/s", "what": "assembly + Krylov solve + line search, rebuild and "
                                          "point update excluded"},
        "kernels": kern,
        "gpu_launches": mixed["launches"],
    }
    if fp64:
        v64 = fp64["its_all"] / (fp64["ms"] * 1e-3)
        line["fp64"] = {"value": round(v64, 4), "unit": "Newton it/s",
                        "ms_per_step": round(fp64["ms"] / K, 2), "newton_its": fp64["its"],
                        "krylov_its": sum(s["lin_its"] for s in fp64["stats"])}
        line["mixed_speedup_vs_fp64"] = round(value / v64, 3)
        line["mixed_time_per_step_speedup_vs_fp64"] = round(fp64["ms"] / mixed["ms"], 3)
        ev = lambda arm: [(s["npts"], s["ndof"], s["nnzb"]) for s in arm["stats"]]
        line["events_match_fp64"] = ev(mixed) == ev(fp64)
        line["reaction_mixed_vs_fp64_rel"] = float(
            abs(mixed["stats"][-1]["reaction"][2] - fp64["stats"][-1]["reaction"][2]) /
            abs(fp64["stats"][-1]["reaction"][2]))
    if e2e:
        line["e2e"] = {"value": round(e2e["its_all"] / (e2e["ms"] * 1e-3), 4),
                       "unit": "Newton it/s", "h2d_bytes_per_step": int(e2e["h2d"]),
                       "d2h_bytes_per_step": int(e2e["d2h"])}
    if roof:
        line["roofline"] = roof
    if mixed["clocks"]:
        line["clocks"] = mixed["clocks"]
    if not a.no_adjoint:
        # the adjoint workload is small (about a thousand dofs): block-Jacobi PCG
        line["adjoint"] = adjoint_leg(dev, 1)
    if not a.no_cpu and world >= 1:
        v, dt, sample, its = run_oracle_sample(a.workload, 1)
        line["cpu_baseline"] = {"value": round(v, 5), "unit": "Newton it/s", "cores": 1,
                                "kind": "oracle", "sample": sample}
    print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def main():
    a = args()
    if a.impl == "reference":
        return reference_main(a)
    return gpu_main(a)


if __name__ == "__main__":
    sys.exit(main())
