"""Krylov solves preconditioned by the geometric multigrid V-cycle (solve
method 3: PCG for symmetric tangents, BiCGStab for the non-associated
Drucker-Prager one), through the C ABI, against the oracle's dense LU and
against the load steps of the oracle.  The preconditioner changes how the
Krylov solve gets to the tolerance, not the solution: the same FP64 and
mixed-precision bars apply as for block Jacobi."""
import numpy as np
import pytest

import oracle
from paper_2606_09275_gb300 import inputs

from test_gpu_parity import CASES, both

pytestmark = pytest.mark.gpu

MG = 3


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2606_09275_gb300 import mpm
    assert torch.cuda.is_available()
    ctx = mpm.Context()
    return mpm, ctx, torch


# (the jittered hanging-node case is left out: its contact tangent has a
# negative eigenvalue at this pose, where no conjugate-gradient method applies)
@pytest.mark.parametrize("case", ["tiny_punch", "punch_d3_6", "column_d3"])
def test_multigrid_pcg_matches_oracle_lu(gpu, case):
    mpm, ctx, torch = gpu
    cfg, bz = CASES[case]()
    om, mesh, P = both(gpu, cfg, bz)
    nd = om.counts()["ndof"]
    # the tangent at the start of the step (symmetric positive definite)
    du = np.zeros(3 * nd)
    o = om.assemble(du)
    xo, _ = om.solve(o["K"], -o["R"], tol=1e-14)
    g = mpm.assemble(ctx, mesh, cfg, torch.tensor(du, device="cuda"), body_z=bz)
    x, st = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-13, maxit=5000, method=MG)
    assert st["status"] == 0 and st["relres"] <= 1e-13
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-9 * np.abs(xo).max()
    xb, sb = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-13, maxit=50000, method=1)
    print("%s: %d dofs, multigrid PCG %d iterations, block-Jacobi PCG %d" % (
        case, nd, st["iterations"], sb["iterations"]))
    # mixed: FP32 V-cycle and inner PCG inside FP64 refinement
    gm = mpm.assemble(ctx, mesh, cfg, torch.tensor(du, device="cuda"), precision=1, body_z=bz)
    xm, sm = mpm.solve(ctx, mesh, cfg, gm["K"], -gm["R"], precision=1, tol=1e-10, maxit=5000,
                       method=MG)
    assert sm["status"] == 0 and sm["refinements"] >= 1
    assert np.max(np.abs(xm.cpu().numpy() - xo)) <= 1e-5 * np.abs(xo).max()


def test_multigrid_needs_far_fewer_iterations_at_scale(gpu):
    # indentation one level below the benchmark (33,600 dofs): the block-Jacobi
    # count grows with the mesh, the multigrid count does not
    mpm, ctx, torch = gpu
    cfg = inputs.workload("indent_small")
    pts = inputs.make_points(cfg)
    P = mpm.Points(pts, capacity=2 * len(pts["x"]))
    bz = inputs.body_z(cfg, 1)
    mesh = mpm.octree_build(ctx, cfg, P, body_z=bz)
    nd = mesh.info()["ndof"]
    zero = torch.zeros(3 * nd, dtype=torch.float64, device="cuda")
    for prec in (0, 1):
        g = mpm.assemble(ctx, mesh, cfg, zero, body_z=bz, precision=prec)
        xb, sb = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-8, maxit=50000, method=1,
                           precision=prec)
        xm, sm = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-8, maxit=5000, method=MG,
                           precision=prec)
        assert sm["status"] == 0 and sb["status"] == 0
        assert sm["iterations"] * 4 <= sb["iterations"], (prec, sm, sb)
        xb, xm = xb.cpu().numpy(), xm.cpu().numpy()
        assert np.max(np.abs(xm - xb)) <= 1e-6 * np.abs(xb).max()
        # reusing the coarse operators of the same K gives the same solve (up to
        # the summation order of the dot products)
        xr, sr = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-8, maxit=5000, method=MG,
                           precision=prec, mg_reuse=1)
        assert abs(sr["iterations"] - sm["iterations"]) <= 1
        assert np.max(np.abs(xr.cpu().numpy() - xm)) <= 1e-7 * np.abs(xm).max()
    # levels: depths down to 1, each coarser grid with fewer rows
    lv = mesh.export("mg_levels")
    lv = lv[lv[:, 0] > 0]
    print("multigrid levels (depth, rows, radius, stencil):", lv.tolist())
    assert list(lv[:, 0]) == list(range(lv[0, 0], 0, -1))
    assert np.all(np.diff(lv[:, 1]) < 0) and lv[0, 1] * 4 <= nd


@pytest.mark.parametrize("reuse", [0, 1])
def test_multigrid_punch_steps_match_oracle(gpu, reuse):
    mpm, ctx, torch = gpu
    cfg = inputs.workload("punch")
    pts = inputs.make_points(cfg)
    om = oracle.Model(cfg, pts)
    P = mpm.Points(pts, capacity=64 * len(pts["x"]))
    Pm = mpm.Points(pts, capacity=64 * len(pts["x"]))
    for n in range(1, 4):
        bz = inputs.body_z(cfg, n)
        om.set_body_z(bz)
        so = om.step(load=1.0, tol=1e-12, lin_tol=1e-13)
        sg = mpm.step(ctx, cfg, P, body_z=bz, tol=1e-12, lin_tol=1e-13, lin_maxit=20000, method=MG,
                      mg_reuse=reuse)
        sm = mpm.step(ctx, cfg, Pm, body_z=bz, tol=1e-8, lin_tol=1e-8, lin_maxit=20000, method=MG,
                      precision=1, mg_reuse=reuse)
        assert so["status"] == 0 and sg["status"] == 0 and sm["status"] == 0
        assert abs(sg["reaction"][2] - so["reaction"][2]) <= 1e-9 * abs(so["reaction"][2])
        assert abs(sm["reaction"][2] - so["reaction"][2]) <= 1e-6 * abs(so["reaction"][2])
    po, pg = om.points(), P.numpy()
    assert np.max(np.abs(pg["x"] - po["x"])) <= 1e-9 * 0.1 * 3 / 50


@pytest.mark.parametrize("precision", [0, 1])
def test_multigrid_bicgstab_on_the_drucker_prager_tangent(gpu, precision):
    # non-associated Drucker-Prager (psi != phi), plastic increment: the
    # tangent is not symmetric, so method 3 runs BiCGStab with the V-cycle
    mpm, ctx, torch = gpu
    cfg, bz = CASES["cone_d4_8"]()
    om, mesh, P = both(gpu, cfg, bz)
    nd = om.counts()["ndof"]
    rng = np.random.default_rng(8)
    du = 1e-4 * rng.standard_normal(3 * nd)
    bcm = om.bcmask()
    du[[bool((bcm[i // 3] >> (i % 3)) & 1) for i in range(3 * nd)]] = 0.0
    o = om.assemble(du)
    xo, _ = om.solve(o["K"], -o["R"], tol=1e-14)
    g = mpm.assemble(ctx, mesh, cfg, torch.tensor(du, device="cuda"), body_z=bz, precision=precision)
    tol = 1e-11 if precision == 0 else 1e-9
    x, st = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=tol, maxit=5000, method=MG,
                      precision=precision)
    assert st["status"] == 0 and st["relres"] <= tol
    bar = 1e-8 if precision == 0 else 1e-5
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= bar * np.abs(xo).max()
    xb, sb = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=tol, maxit=50000, method=2,
                       precision=precision)
    assert sb["status"] == 0
    print("cone (precision %d): %d dofs, multigrid BiCGStab %d iterations, block-Jacobi %d" % (
        precision, nd, st["iterations"], sb["iterations"]))
    assert st["iterations"] < sb["iterations"]


def test_multigrid_bicgstab_cone_steps_match_oracle(gpu):
    # two load steps of the cone into the Drucker-Prager layer, Newton on the
    # non-symmetric tangent with multigrid BiCGStab, FP64 and mixed
    mpm, ctx, torch = gpu
    cfg = inputs.workload("cone")
    pts = inputs.make_points(cfg)
    om = oracle.Model(cfg, pts)
    P = mpm.Points(pts, capacity=64 * len(pts["x"]))
    Pm = mpm.Points(pts, capacity=64 * len(pts["x"]))
    for n in range(1, 3):
        bz = inputs.body_z(cfg, n)
        om.set_body_z(bz)
        load = inputs.load_factor(cfg, n)
        so = om.step(load=load, tol=1e-10, lin_tol=1e-11)
        sg = mpm.step(ctx, cfg, P, body_z=bz, load=load, tol=1e-10, lin_tol=1e-11,
                      lin_maxit=20000, method=MG, mg_reuse=1)
        sm = mpm.step(ctx, cfg, Pm, body_z=bz, load=load, tol=1e-8, lin_tol=1e-8,
                      lin_maxit=20000, method=MG, mg_reuse=1, precision=1)
        assert so["status"] == 0 and sg["status"] == 0 and sm["status"] == 0
        ra = so["reaction"][2]
        assert abs(sg["reaction"][2] - ra) <= 1e-8 * abs(ra)
        assert abs(sm["reaction"][2] - ra) <= 1e-6 * abs(ra)
