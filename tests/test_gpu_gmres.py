"""Restarted GMRES(30) with the block-Jacobi preconditioner (solve method 4;
Sec. 6.4 names GMRES with a Jacobi preconditioner as the iterative route for
the CPT's linear solves), through the C ABI, against the FP64 oracle's LU.

* Linear solves of the non-symmetric Drucker-Prager tangent (plastic
  increment under the cone) and of the symmetric punch tangent: FP64 to
  1e-11 (solution within 1e-8 of the LU's), and the mixed path (FP32 GMRES
  inside FP64 refinement) to the same FP64 target.
* Load steps of the punch with Coulomb friction solved by GMRES: reaction,
  positions, F and b_e within 1e-9 of the oracle's.
"""
import numpy as np
import pytest

import oracle
from paper_2606_09275_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2606_09275_gb300 import mpm
    assert torch.cuda.is_available()
    ctx = mpm.Context()
    yield mpm, ctx, torch
    ctx.close()


def free_mask(bcm):
    return np.array([[not (m >> d) & 1 for d in range(3)] for m in bcm]).ravel()


def both(gpu, cfg, bz):
    mpm, ctx, torch = gpu
    pts = inputs.make_points(cfg)
    om = oracle.Model(cfg, pts, body_z=bz)
    om.build()
    P = mpm.Points(pts, capacity=64 * len(pts["x"]))
    mesh = mpm.octree_build(ctx, cfg, P, body_z=bz)
    return om, mesh


@pytest.mark.parametrize("case", ["cone", "punch"])
def test_gmres_solution_matches_oracle(gpu, case):
    mpm, ctx, torch = gpu
    cfg = inputs.workload(case)
    bz = inputs.body_z(cfg, 1)
    om, mesh = both(gpu, cfg, bz)
    nd = om.counts()["ndof"]
    rng = np.random.default_rng(8)
    du = 1e-4 * rng.standard_normal(3 * nd)
    du[~free_mask(om.bcmask())] = 0.0
    o = om.assemble(du)
    xo, _ = om.solve(o["K"], -o["R"], tol=1e-13)
    g = mpm.assemble(ctx, mesh, cfg, torch.tensor(du, device="cuda"), body_z=bz)
    x, st = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-11, maxit=50000, method=4)
    assert st["status"] == 0 and st["relres"] <= 1e-11, st
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-8 * np.abs(xo).max()
    # mixed: FP32 GMRES inside FP64 refinement
    gm = mpm.assemble(ctx, mesh, cfg, torch.tensor(du, device="cuda"), precision=1, body_z=bz)
    xm, sm = mpm.solve(ctx, mesh, cfg, gm["K"], -gm["R"], precision=1, tol=1e-10, maxit=50000,
                       method=4, inner_tol=1e-4)
    assert sm["status"] == 0 and sm["refinements"] >= 1, sm
    assert np.max(np.abs(xm.cpu().numpy() - xo)) <= 1e-5 * np.abs(xo).max()


def test_friction_punch_steps_with_gmres_match_oracle(gpu):
    mpm, ctx, torch = gpu
    cfg = inputs.workload("punch", mu=0.3)
    pts = inputs.make_points(cfg)
    om = oracle.Model(cfg, pts)
    P = mpm.Points(pts, capacity=64 * len(pts["x"]))
    for n in range(1, 3):
        bz = inputs.body_z(cfg, n)
        om.set_body_z(bz)
        so = om.step(load=1.0, tol=1e-12, lin_tol=1e-13)
        sg = mpm.step(ctx, cfg, P, body_z=bz, load=1.0, tol=1e-12, lin_tol=1e-13,
                      lin_maxit=200000, method=4, check=False)
        assert so["status"] == 0 and sg["status"] == 0, (sg["res_hist"], ctx.error())
        assert np.max(np.abs(sg["reaction"] - so["reaction"])) <= 1e-9 * abs(so["reaction"][2])
    po, pg = om.points(), P.numpy()
    assert np.max(np.abs(pg["x"] - po["x"])) <= 1e-9 * 0.1 * 2 / 50
    for k in ("F", "be", "lp"):
        assert np.max(np.abs(pg[k] - po[k])) <= 1e-9 * max(1.0, np.abs(po[k]).max()), k
