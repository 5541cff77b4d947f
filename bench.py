"""Benchmark: Newton iterations per second of the implicit octree GIMP MPM load
step on one GB300, FP32+refinement vs FP64, with the HBM and FP64 rooflines of
the dominant kernels.

A step is one quasi-static load step: rebuild of the adapted octree, GIMP
split, discrete GIMP basis, block pattern and ghost matrix, then
Newton-Raphson (assembly, Krylov solve, line search) to a 1e-8 residual, then
the point update.  value = Newton iterations / second over the timed steps of
the mixed-precision path on the headline workload (`indent`, the punch at
~0.75 M unknowns); the FP64 path is timed on the same steps and the two are
compared step by step (events and reactions).  The ~1 M-DOF Drucker-Prager
cone (`cone_1m`, non-symmetric tangent, multigrid BiCGStab) is timed beside it.
Further keys: the discrete adjoint's cost against the forward run it
differentiates, 20 load steps of the punch at depth 3 -> 5 with about 70 k
points (`adjoint`) and with 9.5 k (`adjoint_small`); Newmark time steps of the
rolling sphere with a free rigid body (`rolling_sphere`).  Multi-GPU runs are independent replicas (the path has no data-parallel
exchange at this level), so scaling is weak.

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]
"""
import argparse
import hashlib
import json
import math
import multiprocessing as mp
import os
import platform
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "indent"
CONE = "cone_1m"
SOLVER = 3
CPU_SAMPLE = dict(depth_min=4, depth_max=5, dx_region=2.0 / 32,
                  points=dict(spacing=1.0 / 32, jitter=1.0 / 128))
PROF_NAMES = ["pcg_update", "pcg_spmv", "tangent_rows", "constitutive", "kinematics", "grad_x",
              "basis", "residual_rows", "contact", "bicgstab_spmv", "refine_residual", "pattern",
              "vcycle_coarse", "mg_setup", "vcycle_fine", "vcycle_level1", "mg_galerkin"]
NPROF = len(PROF_NAMES)
VCYCLE = ("vcycle_coarse", "vcycle_fine", "vcycle_level1")
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
    ap.add_argument("--no-cone", action="store_true")
    ap.add_argument("--cone-steps", type=int, default=3)
    ap.add_argument("--cone-warmup", type=int, default=3)
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-dynamics", action="store_true")
    ap.add_argument("--no-tight", action="store_true",
                    help="skip the mixed-vs-FP64 comparison at a 1e-10 Newton residual")
    ap.add_argument("--method", type=int, default=SOLVER,
                    help="Krylov method of mpm_solve_params (1 block-Jacobi PCG, 3 multigrid PCG)")
    ap.add_argument("--inner-tol", type=float, default=1e-4,
                    help="mixed precision: relative target of each FP32 inner solve")
    ap.add_argument("--mg-reuse", type=int, default=1,
                    help="method 3: keep the coarse operators across the Newton iterations of a step")
    ap.add_argument("--cpu-procs", type=int, default=0,
                    help="oracle processes of the CPU baseline (0: every host core)")
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


# ----------------------------------------------------------------- CPU baseline (the oracle)

def cpu_sample_cfg(workload):
    from paper_2606_09275_gb300 import inputs
    return inputs.workload(workload, **CPU_SAMPLE)


def run_oracle_sample(workload, nsteps, sample=None):
    """The oracle as it stands, on a bounded sample of the same workload recipe
    (one host thread).  Returns (Newton its, seconds, description, DOF)."""
    import oracle
    from paper_2606_09275_gb300 import inputs
    if sample is not None:
        cfg = inputs.workload(workload, **sample)
    else:
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
    desc = ("oracle load steps 1-%d of the %s recipe at depth %d->%d (%d points, %d DOF)" %
            (nsteps, workload, cfg["depth_min"], cfg["depth_max"], m.counts()["npts"], dof))
    return its, dt, desc, dof


def _oracle_worker(a):
    return run_oracle_sample(*a)


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    return platform.processor() or platform.machine()


def cpu_baseline(workload, nsteps, procs):
    """The oracle on every host core: `procs` independent copies of the sample
    (spawned processes, one thread each), throughput = their Newton iterations
    / wall time.  Returns the cpu_baseline object."""
    procs = procs or os.cpu_count() or 1
    t0 = time.perf_counter()
    if procs == 1:
        res = [run_oracle_sample(workload, nsteps)]
    else:
        with mp.get_context("spawn").Pool(procs) as pool:
            res = pool.map(_oracle_worker, [(workload, nsteps)] * procs)
    wall = time.perf_counter() - t0
    its = sum(r[0] for r in res)
    v = its / wall
    dof = res[0][3]
    return {"value": round(v, 5), "unit": "Newton it/s", "cores": procs, "kind": "oracle",
            "sample": "%s; %d independent copies, one per host core, in parallel" % (res[0][2], procs)
            if procs > 1 else res[0][2] + ", one host thread",
            "cpu_model": cpu_model(), "nproc": os.cpu_count(),
            "dof": dof, "dof_newton_its_per_s": round(v * dof, 1),
            "single_copy_newton_its_per_s": round(res[0][0] / res[0][1], 5),
            "wall_s": round(wall, 2)}


def reference_main(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    steps = max(1, a.steps)
    procs = a.cpu_procs or os.cpu_count() or 1
    run_oracle_sample(a.workload, 1)  # warm-up (untimed)
    t0 = time.perf_counter()
    its, desc, dof = 0, None, 0
    for _ in range(steps):
        cb = cpu_baseline(a.workload, 1, procs)
        its += cb["value"] * cb["wall_s"]
        desc, dof = cb["sample"], cb["dof"]
    dt = time.perf_counter() - t0
    v = its / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "Newton it/s",
            "n_gpus": a.gpus, "steps": steps, "warmup": a.warmup,
            "ms_per_step": 1e3 * dt / steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": a.workload + " (bounded CPU sample)", "sample": desc},
            "cpu_baseline": {"value": v, "unit": "Newton it/s", "cores": procs, "kind": "oracle",
                             "sample": desc, "cpu_model": cpu_model(), "nproc": os.cpu_count(),
                             "dof": dof, "dof_newton_its_per_s": v * dof},
            "e2e": {"value": v, "unit": "Newton it/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ----------------------------------------------------------------- byte and flop models

# ALU and shared-memory ceilings derived from GB300's unit counts and clock
# (152 SMs at 2070 MHz; 128 FP32 lanes and 128 bytes per clock of shared
# memory per SM)
FP32_PEAK = 152 * 128 * 2 * 2.07e9
FP32_PEAK_NOTE = "152 SMs x 128 FP32 lanes x 2 flop x 2.07 GHz = 80.5 TFLOP/s (derived, not measured)"
SMEM_PEAK = 152 * 128 * 2.07e9
SMEM_PEAK_NOTE = "152 SMs x 128 B/clock x 2.07 GHz = 40.3 TB/s (derived, not measured)"


def spmv_bytes(nnzb, nd, mixed):
    """Algorithmic bytes of one fused PCG SpMV launch: matrix values and column
    indices once, row pointers, and z, p, q (p and q read and written)."""
    w = 4 if mixed else 8
    return nnzb * (9 * w + 4) + 4 * (nd + 1) + 5 * 3 * nd * w


def kernel_models(s, mixed=True):
    """Per-launch algorithmic bytes (and FP64 flops) of the dominant kernels
    from the step's sizes: s = step stats (npts, ndof (dof nodes), nnzb,
    nsrc, nslot, mg_rows1, mg_stencil1)."""
    P, nd, nnzb, nsrc, nslot = s["npts"], s["ndof"], s["nnzb"], s["nsrc"], s["nslot"]
    w = 4 if mixed else 8
    m = {}
    m["pcg_spmv"] = dict(kernel="k_pcg_b<float,float>", what="PCG SpMV fused with p, q and p.q (FP32)",
                         bytes=spmv_bytes(nnzb, nd, mixed), bound="hbm")
    # both fine-level V-cycle kernels: the FP16 copy of K and its columns once,
    # x, b and the output (and the smoother's 3x3 inverses in MODE 1): 72 B/row
    m["vcycle_fine"] = dict(kernel="k_mg_fine<float,0|1,__half>",
                            what="V-cycle fine-level residual / smoothing over the FP16 copy of K",
                            bytes=nnzb * (9 * 2 + 4) + 4 * (nd + 1) + 72 * nd, bound="hbm")
    if s.get("mg_rows1"):
        r1, S1 = s["mg_rows1"], s["mg_stencil1"]
        m["vcycle_level1"] = dict(kernel="k_mg_lvl<float,0|1> (level 1)",
                                  what="V-cycle level-1 residual / smoothing, operator stored per "
                                       "stencil offset (FP32)", bytes=r1 * (S1 * 36 + 72), bound="hbm")
    # tangent rows, per Newton iteration (its two launches together): the
    # 81-entry tangents, grad_x S and support indices, the source keys, V0,
    # ghost coefficients and columns in; the sliced K out
    # and its arithmetic: 27 FMA per (source, column) pair, npair = sum of the
    # squared support sizes, plus the 27 terms of each source (81 FMA + 27
    # multiplications); its accumulators take 9 shared-memory read-modify-writes
    # per pair (72 bytes in FP32)
    npair = s.get("npair") or 0
    m["tangent_rows"] = dict(kernel="k_tangent_rows<float> (both passes)",
                             what="row-gather tangent assembly, per Newton iteration",
                             bytes=P * (81 * w + 8) + nsrc * (3 * w + 4 + 8) + nnzb * 12 + nslot * 9 * w,
                             fp32_flops=54.0 * npair + 189.0 * nsrc, smem_bytes=2.0 * 9 * w * npair,
                             bound="latency", per="newton_it")
    # internal-force gather + residual rows: FP64, 9 FMA per (point, support)
    m["residual_rows"] = dict(kernel="k_residual_rows", what="internal-force gather + residual (FP64)",
                              bytes=nsrc * (8 + 24) + P * 96 + nnzb * 12 + nd * 96,
                              flops=18.0 * nsrc + 6.0 * nnzb, bound="fp64")
    m["kinematics"] = dict(kernel="k_kinematics", what="dF = I + sum du (x) grad S (FP64)",
                           bytes=nsrc * (4 + 24 + 24) + P * 72, flops=18.0 * nsrc, bound="fp64")
    return m


def roofline_entries(prof, s, hbm_peak, fp64_peak, mixed=True):
    """Roofline objects from the profiled launches (CUDA events on the
    launching stream): achieved = algorithmic bytes (or flops) / average launch
    time; frac against the measured peaks."""
    out = {}
    models = kernel_models(s, mixed)
    newton = max(prof.get("newton_its", 0), 1)
    for name, mdl in models.items():
        k = PROF_NAMES.index(name)
        nl, ms = prof["launches"][k], prof["ms"][k]
        if not nl:
            continue
        per = ms / (newton if mdl.get("per") == "newton_it" else nl)
        e = {"kernel": mdl["kernel"], "what": mdl["what"], "bound": mdl["bound"],
             "avg_ms": round(per, 5), "launches": nl, "total_ms": round(ms, 3),
             "algorithmic_bytes": int(mdl["bytes"]),
             "achieved_gbs": round(mdl["bytes"] / (per * 1e-3) / 1e9, 1),
             "hbm_frac": round(mdl["bytes"] / (per * 1e-3) / 1e9 / hbm_peak, 4)}
        if "flops" in mdl and fp64_peak:
            f = mdl["flops"] / (per * 1e-3)
            e.update(fp64_flops=int(mdl["flops"]), achieved_fp64_tflops=round(f / 1e12, 4),
                     fp64_frac=round(f / fp64_peak, 4))
        if mdl.get("fp32_flops"):
            f = mdl["fp32_flops"] / (per * 1e-3)
            e.update(fp32_flops=int(mdl["fp32_flops"]), achieved_fp32_tflops=round(f / 1e12, 3),
                     fp32_frac=round(f / FP32_PEAK, 4), fp32_peak_note=FP32_PEAK_NOTE,
                     smem_bytes=int(mdl["smem_bytes"]),
                     smem_frac=round(mdl["smem_bytes"] / (per * 1e-3) / SMEM_PEAK, 4),
                     smem_peak_note=SMEM_PEAK_NOTE)
        if mdl.get("per"):
            e["per"] = mdl["per"]
        out[name] = e
    return out


def source_hash(parts):
    """Hash of the text of the named functions ([file, function name] pairs):
    the kernel and the device helpers it calls."""
    txt = ""
    for path, name in parts:
        with open(os.path.join(ROOT, path)) as f:
            src = f.read()
        i = src.find(" " + name + "(")
        if i < 0:
            return None
        i = src.rfind("\n", 0, i) + 1
        txt += src[i:src.index("\n}\n", i) + 3]
    return hashlib.sha256(txt.encode()).hexdigest()[:16]


def traffic_record(kernel):
    """ncu DRAM bytes per launch of the kernel, if captured for the current
    source (the record's "parts" and their hash)."""
    try:
        with open(os.path.join(ROOT, "profiles", "ncu_traffic.json")) as f:
            rec = json.load(f)
    except Exception:
        return None
    r = rec.get(kernel)
    if not r or "parts" not in r:
        return None
    if source_hash(r["parts"]) != r["source_sha"]:
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


def adjoint_leg(dev, method, name="adjoint"):
    """Cost of the discrete adjoint against the forward run it differentiates:
    the punch at depth 3 -> 5 with lognormal E, 20 load steps, FP64, gradient
    of the final vertical punch reaction in every point's E and yield stress;
    `name` picks the point lattice ("adjoint": spacing 1/16, "adjoint_60k":
    spacing 1/48)."""
    import torch

    from paper_2606_09275_gb300 import autodiff, inputs, mpm
    cfg = inputs.workload(name)
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
    return {"workload": "%s: flat punch into a von Mises block 1x1x0.5 m, depth 3 -> 5, "
                        "lognormal E (sigma 0.2), %d load steps, FP64, d(reaction_z)/d(E, ys)"
                        % (name, n),
            "points_first_step": st_plain[0]["npts"], "initial_points": len(pts["x"]),
            "points_last_step": st_plain[-1]["npts"], "dof_last_step": 3 * st_plain[-1]["ndof"],
            "forward_ms_per_step": round(fwd / n, 3),
            "forward_with_checkpoints_ms_per_step": round(fwd_ck / n, 3),
            "adjoint_ms_per_step": round(adj / n, 3),
            "adjoint_over_forward": round(adj / fwd, 3),
            "adjoint_resolve_ms_per_step": round(ast["ms_forward"] / n, 3),
            "adjoint_backward_ms_per_step": round(ast["ms_backward"] / n, 3),
            "adjoint_krylov_its": ast["lin_its"], "krylov_method": method,
            "forward_krylov_its": int(sum(s["lin_its"] for s in st_plain))}


def dynamics_leg(dev, nwarm=3, nsteps=12):
    """Newmark time steps with a free rigid body (Sec. 2.4, 2.3): the rolling
    sphere of Sec. 6.3 (mu = 1, the sticking regime), FP64 and mixed, timed
    over `nsteps` time steps after `nwarm`, and the distance travelled against
    the paper's closed form 5 g t^2 sin(theta) / 14."""
    import torch

    from paper_2606_09275_gb300 import inputs, mpm
    cfg = inputs.workload("rolling_sphere", mu=1.0)
    out = {"workload": "rolling_sphere: rigid sphere (d 2 m, 1e4 kg, J 4000 kg m2) rolling on a "
                       "stiff slab under gravity tilted 45 degrees, mu = 1 (sticking), Newmark "
                       "gamma 1 beta 1/2, dt %.3g s, the sphere free in x, z and about y "
                       "(Schur elimination: 1 + 3 solves per Newton iteration)" % cfg["dt"],
           "timed_steps": "time steps %d-%d after %d warm-up steps" % (nwarm + 1, nwarm + nsteps, nwarm)}
    for prec, name in ((mpm.FP64, "fp64"), (mpm.MIXED, "mixed")):
        pts = inputs.make_points(cfg)
        ctx = mpm.Context()
        P = mpm.Points(pts, capacity=64 * len(pts["x"]), velocity=True)
        state = mpm.body_start(cfg)
        lin_tol = cfg["lin_tol"]
        run = lambda: mpm.step(ctx, cfg, P, load=1.0, tol=cfg["newton_tol"], maxit=40,
                               lin_tol=lin_tol, lin_maxit=cfg["lin_maxit"], precision=prec,
                               inner_tol=1e-4, dt=cfg["dt"], body_state=state)
        for _ in range(nwarm):
            run()
        stream = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        sts = [run() for _ in range(nsteps)]
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        its = sum(st["newton_its"] for st in sts)
        t = (nwarm + nsteps) * cfg["dt"]
        d = float(state["pose"][0] - cfg["body"]["cx"])
        ana = 5.0 * 9.81 * t * t * math.sin(math.pi / 4) / 14.0
        out[name] = {"time_steps_per_s": round(nsteps / (ms * 1e-3), 3),
                     "newton_its_per_s": round(its / (ms * 1e-3), 3), "ms_per_step": round(ms / nsteps, 3),
                     "newton_its": its, "krylov_its": int(sum(st["lin_its"] for st in sts)),
                     "points": sts[-1]["npts"], "dof": 3 * sts[-1]["ndof"],
                     "distance_m": round(d, 6), "closed_form_m": round(ana, 6),
                     "distance_rel_err": round(abs(d - ana) / ana, 5),
                     "rolling_theta_r_over_distance": round(float(state["theta"][1]) * cfg["body"]["r"] / d, 5)}
        ctx.close()
    return out


def compare_arms(mixed, fp64):
    """Step-by-step comparison of the mixed and FP64 runs from the same
    initial state (warm-up steps included): discrete events (points after
    splits, dofs, blocks) and the vertical reaction."""
    ev = lambda s: (s["npts"], s["ndof"], s["nnzb"])
    steps, first = [], None
    for n, (a, b) in enumerate(zip(mixed["all_stats"], fp64["all_stats"]), 1):
        rel = abs(a["reaction"][2] - b["reaction"][2]) / max(abs(b["reaction"][2]), 1e-300)
        same = ev(a) == ev(b)
        if not same and first is None:
            first = n
        steps.append({"step": n, "events_match": same, "reaction_rel": float(rel),
                      "newton_its": [a["newton_its"], b["newton_its"]],
                      "line_search_eta": [list(map(float, a["eta_hist"])), list(map(float, b["eta_hist"]))]})
    before = [s["reaction_rel"] for s in steps if first is None or s["step"] < first]
    return {"events_match_fp64": first is None, "first_event_divergence_step": first,
            "reaction_mixed_vs_fp64_rel_max_before_divergence": max(before) if before else None,
            "per_step": steps}


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
    stream = torch.cuda.current_stream()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    def arm(workload, precision, W, K, method, profile=False, e2e=False, clocks=False, tol=None,
            lin_tol=None):
        cfg = inputs.workload(workload)
        pts0 = inputs.make_points(cfg)
        ctx = mpm.Context()
        P = mpm.Points(pts0, capacity=cfg.get("cap_factor", 2) * len(pts0["x"]), device=dev)
        host = None
        if e2e:
            host = {k: torch.empty_like(t, device="cpu").pin_memory() for k, t in P.t.items()}
            for k in host:
                host[k].copy_(P.t[k])
        step_kw = dict(load=1.0, tol=tol or cfg["newton_tol"], maxit=cfg["newton_maxit"],
                       lin_tol=lin_tol or cfg["lin_tol"], lin_maxit=cfg["lin_maxit"], precision=precision,
                       method=method, mg_reuse=a.mg_reuse, inner_tol=a.inner_tol)
        all_stats = []
        for n in range(1, W + 1):
            all_stats.append(mpm.step(ctx, cfg, P, body_z=inputs.body_z(cfg, n), **step_kw))
        if e2e:
            for k in host:
                host[k].copy_(P.t[k])
        barrier()
        clk = Clocks(local) if (rank == 0 and clocks) else None
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
            prof = {"launches": list(L), "ms": list(T), "newton_its": its}
        clk_out = clk.stop() if clk else None
        barrier()
        its_all, ms = replica_totals(its, ms, world, dev)
        ctx.close()
        del P
        torch.cuda.empty_cache()
        return dict(cfg=cfg, ms=ms, its=its, its_all=its_all, stats=stats,
                    all_stats=all_stats + stats, prof=prof, clocks=clk_out,
                    launches=nl1.value - nl0.value, h2d=h2d // max(K, 1), d2h=d2h // max(K, 1))

    W, K = a.warmup, a.steps
    hbm_peak, peak_src = peaks()
    pctx = mpm.Context()
    fp64_flops, fp64_ms = mpm.fp64_peak(pctx, 1.0)
    pctx.close()

    # headline: mixed precision, no per-launch events in the timed region
    mixed = arm(a.workload, mpm.MIXED, W, K, a.method, clocks=True)
    fp64 = None if a.no_fp64 else arm(a.workload, mpm.FP64, W, K, a.method)
    # per-kernel times: a separate profiled run of the same steps
    profd = arm(a.workload, mpm.MIXED, W, K, a.method, profile=True)
    e2e = None if a.no_e2e else arm(a.workload, mpm.MIXED, W, K, a.method, e2e=True)
    cone = cone64 = None
    if not a.no_cone:
        cone = arm(CONE, mpm.MIXED, a.cone_warmup, a.cone_steps, 3, profile=True)
        if not a.no_fp64:
            cone64 = arm(CONE, mpm.FP64, a.cone_warmup, a.cone_steps, 3)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return 0

    value = mixed["its_all"] / (mixed["ms"] * 1e-3)
    last = mixed["stats"][-1]
    prof = profd["prof"]
    kern = {n: {"launches": prof["launches"][i], "ms": round(prof["ms"][i], 3)}
            for i, n in enumerate(PROF_NAMES) if prof["launches"][i]}
    vms = sum(kern[n]["ms"] for n in VCYCLE if n in kern)
    dom_class = max(list(kern) + ["vcycle (all)"],
                    key=lambda n: vms if n == "vcycle (all)" else kern[n]["ms"])
    roofs = roofline_entries(prof, profd["stats"][-1], hbm_peak, fp64_flops, True)
    hbm_roofs = {n: r for n, r in roofs.items() if r["bound"] == "hbm" and r.get("per") is None}
    top = max(hbm_roofs, key=lambda n: hbm_roofs[n]["total_ms"])
    t = hbm_roofs[top]
    tr = traffic_record(t["kernel"])
    roof = {"kernel": t["kernel"], "bound": "hbm", "achieved": t["achieved_gbs"], "peak": hbm_peak,
            "unit": "GB/s", "frac": t["hbm_frac"], "peak_source": peak_src,
            "traffic": (round(tr["bytes_per_launch"] * t["algorithmic_bytes"] /
                              tr["alg_bytes_per_launch"]) if tr else None),
            "algorithmic_bytes_per_launch": t["algorithmic_bytes"], "avg_launch_ms": t["avg_ms"],
            "why_this_kernel": "the HBM-bound kernel with the largest total time in the profiled "
                               "steps; per-kernel entries in `rooflines`",
            "dominant_class_by_time": dom_class}
    nodes = int(last["ndof"])
    line = {
        "metric": METRIC, "value": round(value, 4), "unit": "Newton it/s", "n_gpus": world,
        "steps": K, "warmup": W, "ms_per_step": round(mixed["ms"] / K, 2),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64 (FP32 tangent and inner PCG; FP64 residual, dF, return map, refinement)",
        "data": "synthetic",
        "config": {"workload": "%s: flat punch (r 0.1 m) into a von Mises block 1x1x0.875 m, "
                               "octree depth 6 refined to 7 at the punch, jittered 2x2x2 points "
                               "per cell" % a.workload,
                   "points": last["npts"], "dof": 3 * nodes, "nodes": nodes, "nnzb": last["nnzb"],
                   "newton_tol": mixed["cfg"]["newton_tol"], "krylov_tol": mixed["cfg"]["lin_tol"],
                   "krylov": {1: "block-Jacobi PCG", 3: "multigrid-preconditioned PCG"}.get(
                       a.method, "method %d" % a.method),
                   "mixed_inner_tol": a.inner_tol, "mg_reuse": a.mg_reuse,
                   "step": "one load step: mesh rebuild + Newton to 1e-8 + point update",
                   "timed_steps": "load steps %d-%d after %d warm-up steps" % (W + 1, W + K, W),
                   "parallelism": "replicas" if world > 1 else "1 GPU",
                   "l2": "inputs larger than L2 (stiffness %.2f GB FP32)" % (last["nnzb"] * 40 / 1e9)},
        "newton_its": mixed["its"], "krylov_its": sum(s["lin_its"] for s in mixed["stats"]),
        "dof_newton_its_per_s": round(value * 3 * nodes, 1),
        "solver_only": {
            "value": round(mixed["its_all"] / (1e-3 * sum(
                s["ms_assemble"] + s["ms_solve"] for s in mixed["stats"])), 4),
            "unit": "Newton it/s", "what": "assembly + Krylov solve + line search, rebuild and "
                                          "point update excluded"},
        "kernels": kern,
        "kernels_note": "per-class CUDA-event totals of a separate profiled run of the same steps "
                        "(%d Newton iterations)" % profd["its"],
        "gpu_launches": mixed["launches"],
        "fp64_peak": {"value": round(fp64_flops / 1e12, 4), "unit": "TFLOP/s",
                      "how": "mpm_fp64_peak: 8 independent FMA chains per thread on every SM, "
                             "CUDA events, %.0f ms" % fp64_ms},
    }
    if fp64:
        v64 = fp64["its_all"] / (fp64["ms"] * 1e-3)
        line["fp64"] = {"value": round(v64, 4), "unit": "Newton it/s",
                        "ms_per_step": round(fp64["ms"] / K, 2), "newton_its": fp64["its"],
                        "krylov_its": sum(s["lin_its"] for s in fp64["stats"])}
        line["mixed_speedup_vs_fp64"] = round(value / v64, 3)
        line["mixed_time_per_step_speedup_vs_fp64"] = round(fp64["ms"] / mixed["ms"], 3)
        line["mixed_vs_fp64"] = compare_arms(mixed, fp64)
        line["events_match_fp64"] = line["mixed_vs_fp64"]["events_match_fp64"]
        line["reaction_mixed_vs_fp64_rel"] = float(
            abs(mixed["stats"][-1]["reaction"][2] - fp64["stats"][-1]["reaction"][2]) /
            abs(fp64["stats"][-1]["reaction"][2]))
    if e2e:
        line["e2e"] = {"value": round(e2e["its_all"] / (e2e["ms"] * 1e-3), 4),
                       "unit": "Newton it/s", "h2d_bytes_per_step": int(e2e["h2d"]),
                       "d2h_bytes_per_step": int(e2e["d2h"])}
    line["roofline"] = roof
    line["rooflines"] = roofs
    if mixed["clocks"]:
        line["clocks"] = mixed["clocks"]
    if cone:
        cl = cone["stats"][-1]
        cv = cone["its_all"] / (cone["ms"] * 1e-3)
        cn = int(cl["ndof"])
        cp = cone["prof"]
        ent = {"workload": "%s: 60-degree cone (r 0.018 m) into a Drucker-Prager layer "
                           "1x1x1.2 m (c 5 kPa, phi 30, psi 0), non-symmetric tangent" % CONE,
               "value": round(cv, 4), "unit": "Newton it/s", "dtype": "f32+f64",
               "points": cl["npts"], "dof": 3 * cn, "nodes": cn, "nnzb": cl["nnzb"],
               "krylov": "multigrid-preconditioned BiCGStab",
               "timed_steps": "load steps %d-%d after %d warm-up steps" % (
                   a.cone_warmup + 1, a.cone_warmup + a.cone_steps, a.cone_warmup),
               "ms_per_step": round(cone["ms"] / a.cone_steps, 2), "newton_its": cone["its"],
               "krylov_its": sum(s["lin_its"] for s in cone["stats"]),
               "dof_newton_its_per_s": round(cv * 3 * cn, 1),
               "kernels": {n: {"launches": cp["launches"][i], "ms": round(cp["ms"][i], 3)}
                           for i, n in enumerate(PROF_NAMES) if cp["launches"][i]},
               "kernels_note": "per-launch CUDA events on in this run (adds about 1 us per launch)"}
        try:
            # the BiCGStab SpMV (FP32 K, FP32 vectors padded to 4 components):
            # values and columns once, x, y and the dot's second vector per row
            ib = PROF_NAMES.index("bicgstab_spmv")
            nlb, msb = cp["launches"][ib], cp["ms"][ib]
            if nlb:
                perb = msb / nlb
                byb = cl["nnzb"] * (9 * 4 + 4) + 48 * cn
                gbs = byb / (perb * 1e-3) / 1e9
                ent["roofline_bicgstab_spmv"] = {
                    "kernel": "k_spmv_dot<float,float>", "bound": "hbm", "avg_ms": round(perb, 5),
                    "launches": nlb, "algorithmic_bytes": int(byb), "achieved_gbs": round(gbs, 1),
                    "hbm_frac": round(gbs / hbm_peak, 4),
                    "note": "average over every launch of the class, including the few that "
                            "return at once after convergence"}
        except Exception as ex:  # a report field only: never lose the line for it
            ent["roofline_bicgstab_spmv"] = {"error": str(ex)[:120]}
        if cone64:
            c64 = cone64["its_all"] / (cone64["ms"] * 1e-3)
            ent["fp64"] = {"value": round(c64, 4), "unit": "Newton it/s",
                           "ms_per_step": round(cone64["ms"] / a.cone_steps, 2),
                           "newton_its": cone64["its"],
                           "krylov_its": sum(s["lin_its"] for s in cone64["stats"])}
            ent["mixed_speedup_vs_fp64"] = round(cv / c64, 3)
            ent["mixed_vs_fp64"] = compare_arms(cone, cone64)
        line["cone_1m"] = ent
    if fp64 and not a.no_tight:
        # the same steps with Newton and Krylov at 1e-10: at 1e-8 the reaction of
        # this perfectly plastic problem is fixed only to about 1e-4 by the
        # residual (two FP64 runs stopped at 1e-8 and 1e-10 differ as much), so
        # the precision pattern is compared where the residual fixes the solution
        tm = arm(a.workload, mpm.MIXED, W, K, a.method, tol=1e-10, lin_tol=1e-10)
        t64 = arm(a.workload, mpm.FP64, W, K, a.method, tol=1e-10, lin_tol=1e-10)
        cmp = compare_arms(tm, t64)
        e64 = compare_arms(fp64, t64)
        line["mixed_vs_fp64_at_1e-10"] = {
            "newton_tol": 1e-10, "krylov_tol": 1e-10,
            "steps": "load steps 1-%d" % (W + K),
            "events_match_fp64": cmp["events_match_fp64"],
            "first_event_divergence_step": cmp["first_event_divergence_step"],
            "reaction_mixed_vs_fp64_rel_max_before_divergence":
                cmp["reaction_mixed_vs_fp64_rel_max_before_divergence"],
            "fp64_at_1e-8_vs_fp64_at_1e-10_rel_max_before_divergence":
                e64["reaction_mixed_vs_fp64_rel_max_before_divergence"],
            "fp64_at_1e-8_vs_1e-10_first_event_divergence_step": e64["first_event_divergence_step"],
            "per_step_reaction_rel": [s_["reaction_rel"] for s_ in cmp["per_step"]]}
    if not a.no_adjoint:
        # the adjoint workloads are small (about a thousand nodes): block-Jacobi
        # PCG; "adjoint" at about 67 k points, "adjoint_small" on the 2,048-point
        # lattice of the 32-point finite-difference test
        for key, name in (("adjoint", "adjoint_60k"), ("adjoint_small", "adjoint")):
            try:
                line[key] = adjoint_leg(dev, 1, name)
            except Exception as ex:  # recorded in the line; the other legs still run
                line[key] = {"workload": name, "error": "%s: %s" % (type(ex).__name__, ex)}
    if not a.no_dynamics:
        line["rolling_sphere"] = dynamics_leg(dev)
    if not a.no_cpu:
        cb = cpu_baseline(a.workload, 1, a.cpu_procs)
        line["cpu_baseline"] = cb
        line["cpu_baseline_note"] = ("DOF x Newton it/s compares the GPU line (%.3g) with the "
                                     "oracle sample (%.3g) across their sizes" %
                                     (line["dof_newton_its_per_s"], cb["dof_newton_its_per_s"]))
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
