"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Integer and index results (octree, nodes, hanging constraints, supports,
pattern, ghost faces, masks) must be identical; floating-point results are
compared element by element at the tolerance of the FP64 target (1e-9 relative
to the largest entry unless stated)."""
import math

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
    return mpm, ctx, torch


def tiny_cfg(**over):
    pts = dict(spacing=0.25, jitter=0.02, seed=9)
    pts.update(over.pop("points", {}))
    c = inputs.workload("punch", depth_min=1, depth_max=3, dx_region=0.15,
                        body=dict(cx=0.3, cy=0.4, z0=0.5, r=0.1), points=pts)
    c.update(over)
    return c


def sphere_cfg():
    c = tiny_cfg(mu=0.2)
    c["body"] = dict(kind=3, cx=0.31, cy=0.42, z0=0.73, r=0.25, alpha=0.0, dz=-0.002,
                     step_d=(0.003, 0.0, -0.002), mesh=inputs.sphere_mesh(0.25, 10, 12))
    return c


CASES = {
    "tiny_punch": lambda: (tiny_cfg(), 0.49),
    "column_d3": lambda: (inputs.workload("column"), None),
    "punch_d3_6": lambda: (inputs.workload("punch"), inputs.body_z(inputs.workload("punch"), 1)),
    "cone_d4_8": lambda: (inputs.workload("cone"), inputs.body_z(inputs.workload("cone"), 1)),
    "jitter_hang": lambda: (tiny_cfg(depth_min=2, depth_max=4, dx_region=0.1,
                                     points=dict(spacing=0.125, jitter=0.03, seed=5)), 0.47),
    # Coulomb friction (Sec. 2.3, mu = 0.3 as in the paper's CPT and anchor
    # runs) with the body also moving sideways over the step: stick and slip
    "friction_punch": lambda: (dict(tiny_cfg(mu=0.3), body=dict(
        tiny_cfg()["body"], step_d=(0.003, -0.001, -0.01))), 0.49),
    # a closed triangulated body (Sec. 2.3's faceted rigid bodies): a coarse
    # sphere pressed into the block, with friction and a sideways motion
    "sphere_mesh": lambda: (sphere_cfg(), None),
    # the CPT material (Sec. 6.4): the Willam-Warnke cone, plastic, under the cone
    "cone_ww": lambda: (inputs.workload("cone", model=3, phi=math.radians(32.0),
                                        psi=math.radians(2.0)),
                        inputs.body_z(inputs.workload("cone"), 1)),
    # the benchmark's recipe one level coarser: 239 k points, 101 k unknowns,
    # 3.6 M blocks, rows up to 171 blocks (the tangent's long-row pass)
    "indent_small": lambda: (inputs.workload("indent_small"),
                             inputs.body_z(inputs.workload("indent_small"), 1)),
}


def both(gpu, cfg, bz, nosplit=False, capacity=None):
    mpm, ctx, torch = gpu
    pts = inputs.make_points(cfg)
    om = oracle.Model(cfg, pts, body_z=bz)
    om.build(nosplit=nosplit)
    P = mpm.Points(pts, capacity=capacity or 64 * len(pts["x"]))
    mesh = mpm.octree_build(ctx, cfg, P, body_z=bz, nosplit=nosplit)
    return om, mesh, P


@pytest.mark.parametrize("case", list(CASES))
def test_mesh_build_matches_oracle(gpu, case):
    cfg, bz = CASES[case]()
    om, mesh, P = both(gpu, cfg, bz)
    oc = om.counts()
    gi = mesh.info()
    for k in ("nleaf", "nnode", "nhang", "ndof", "nnzb", "nghost", "npts", "maxs"):
        assert gi[k] == oc[k], (k, gi[k], oc[k])
    lev, anc = om.tree()
    assert np.array_equal(mesh.export("leaf_level"), lev)
    assert np.array_equal(mesh.export("leaf_anchor"), anc)
    nd = om.nodes()
    assert np.array_equal(mesh.export("node_coord"), nd["coord"])
    assert np.array_equal(mesh.export("node_hang"), nd["hang"])
    assert np.array_equal(mesh.export("node_dof"), nd["dof"])
    assert np.array_equal(mesh.export("cptr"), nd["cptr"])
    assert np.array_equal(mesh.export("cidx"), nd["cidx"])
    assert np.array_equal(mesh.export("cw"), nd["cw"])
    # split points are identical, bit for bit
    po, pg = om.points(), P.numpy()
    for k in po:
        assert np.array_equal(po[k], pg[k]), k
    nsup, sidx, S, dS = om.support()
    gns = mesh.export("nsup")
    assert np.array_equal(gns, nsup)
    gsi, gS, gdS = mesh.export("sidx"), mesh.export("S"), mesh.export("dS")
    mask = np.arange(64)[None, :] < nsup[:, None]
    assert np.array_equal(np.where(mask, gsi, -1), np.where(mask, sidx, -1))
    assert np.max(np.abs(np.where(mask, gS - S, 0))) < 1e-13
    scale = (1 << cfg["depth_max"]) / cfg["L"]
    assert np.max(np.abs(np.where(mask[..., None], gdS - dS, 0))) < 1e-13 * scale
    rp, col = om.pattern()
    assert np.array_equal(mesh.export("row_ptr"), rp)
    assert np.array_equal(mesh.export("col"), col)
    assert np.array_equal(mesh.export("bcmask"), om.bcmask())
    faces, pop = om.ghost_faces()
    assert np.array_equal(mesh.export("populated"), pop)
    assert np.array_equal(mesh.export("ghost_faces"), faces)
    kg = om.ghost()
    if len(kg):
        assert np.max(np.abs(mesh.export("ghost") - kg)) <= 1e-12 * max(np.abs(kg).max(), 1e-300)


def free_mask(bcmask):
    return np.array([[not (m >> c) & 1 for c in range(3)] for m in bcmask]).ravel()


@pytest.mark.parametrize("case", ["tiny_punch", "punch_d3_6", "cone_d4_8", "jitter_hang",
                                  "friction_punch", "sphere_mesh", "cone_ww", "indent_small"])
@pytest.mark.parametrize("precision", [0, 1])
def test_assembly_matches_oracle(gpu, case, precision):
    mpm, ctx, torch = gpu
    cfg, bz = CASES[case]()
    if case == "tiny_punch":
        cfg["points"]["ys"] = 2e4  # plastic at this increment
    om, mesh, P = both(gpu, cfg, bz)
    nd = om.counts()["ndof"]
    rng = np.random.default_rng(3)
    du = 2e-4 * rng.standard_normal(3 * nd)
    bcm = om.bcmask()
    fr = free_mask(bcm)
    du[~fr] = 0.0
    o = om.assemble(du, load=1.0)
    g = mpm.assemble(ctx, mesh, cfg, torch.tensor(du, device="cuda"), load=1.0,
                     precision=precision, body_z=bz)
    R = g["R"].cpu().numpy()
    scale = np.abs(o["R"]).max()
    assert np.max(np.abs(R - o["R"])) <= 1e-10 * scale
    assert np.allclose(g["reaction"], o["reaction"], rtol=1e-10, atol=1e-10 * scale)
    fi = np.linalg.norm(o["fint"])
    assert abs(g["fint_norm"] - fi) <= 1e-10 * fi
    rp, col = om.pattern()
    Kg = mpm.blocks(ctx, mesh, g["K"], precision)
    Ko = o["K"]
    row = np.repeat(np.arange(nd), np.diff(rp))
    fm = fr.reshape(-1, 3)
    keep = fm[row][:, :, None] & fm[col][:, None, :]
    tol = (1e-10 if precision == 0 else 2e-6) * np.abs(Ko).max()
    assert np.max(np.abs(np.where(keep, Kg - Ko, 0))) <= tol
    # Dirichlet entries: identity on the diagonal, zero elsewhere
    diag = (row == col)[:, None, None] & np.eye(3, dtype=bool)[None]
    assert np.all(np.where(~keep & diag, Kg, 1.0) == 1.0)
    assert np.all(np.where(~keep & ~diag, Kg, 0.0) == 0.0)


@pytest.mark.parametrize("case", ["tiny_punch", "punch_d3_6"])
def test_krylov_solution_matches_oracle(gpu, case):
    mpm, ctx, torch = gpu
    cfg, bz = CASES[case]()
    om, mesh, P = both(gpu, cfg, bz)
    nd = om.counts()["ndof"]
    o = om.assemble(np.zeros(3 * nd))
    xo, _ = om.solve(o["K"], -o["R"], tol=1e-14)
    g = mpm.assemble(ctx, mesh, cfg, torch.zeros(3 * nd, dtype=torch.float64, device="cuda"),
                     body_z=bz)
    x, st = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-13, maxit=50000)
    assert st["status"] == 0 and st["relres"] <= 1e-13
    xg = x.cpu().numpy()
    assert np.max(np.abs(xg - xo)) <= 1e-9 * np.abs(xo).max()
    # mixed: FP32 inner solves inside FP64 refinement reach the same FP64 target
    gm = mpm.assemble(ctx, mesh, cfg, torch.zeros(3 * nd, dtype=torch.float64, device="cuda"),
                      precision=1, body_z=bz)
    xm, sm = mpm.solve(ctx, mesh, cfg, gm["K"], -gm["R"], precision=1, tol=1e-10, maxit=50000)
    assert sm["status"] == 0 and sm["refinements"] >= 1
    # the FP32 tangent differs from the FP64 one by rounding: agreement ~1e-6
    assert np.max(np.abs(xm.cpu().numpy() - xo)) <= 1e-5 * np.abs(xo).max()


@pytest.mark.parametrize("method", [0, 2])
def test_bicgstab_solution_matches_oracle(gpu, method):
    # Drucker-Prager with psi != phi: non-symmetric tangent, plastic increment
    mpm, ctx, torch = gpu
    cfg, bz = CASES["cone_d4_8"]()
    om, mesh, P = both(gpu, cfg, bz)
    nd = om.counts()["ndof"]
    rng = np.random.default_rng(8)
    du = 1e-4 * rng.standard_normal(3 * nd)
    du[~free_mask(om.bcmask())] = 0.0
    o = om.assemble(du)
    xo, _ = om.solve(o["K"], -o["R"], tol=1e-13)
    g = mpm.assemble(ctx, mesh, cfg, torch.tensor(du, device="cuda"), body_z=bz)
    x, st = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-11, maxit=50000, method=method)
    assert st["status"] == 0 and st["relres"] <= 1e-11
    assert np.max(np.abs(x.cpu().numpy() - xo)) <= 1e-8 * np.abs(xo).max()


def run_steps(gpu, cfg, nsteps, precision=0, tol=1e-12, lin_tol=1e-13):
    mpm, ctx, torch = gpu
    pts = inputs.make_points(cfg)
    om = oracle.Model(cfg, pts)
    P = mpm.Points(pts, capacity=64 * len(pts["x"]))
    hist_o, hist_g = [], []
    for n in range(1, nsteps + 1):
        bz = inputs.body_z(cfg, n) if cfg.get("body") else None
        if bz is not None:
            om.set_body_z(bz)
        so = om.step(load=inputs.load_factor(cfg, n), tol=tol, lin_tol=min(lin_tol, 1e-13))
        sg = mpm.step(ctx, cfg, P, body_z=bz, load=inputs.load_factor(cfg, n), tol=tol,
                      lin_tol=lin_tol, precision=precision, lin_maxit=100000, check=False)
        assert so["status"] == 0, (n, so["res_hist"])
        assert sg["status"] == 0, (n, sg["res_hist"], ctx.error())
        hist_o.append(so)
        hist_g.append(sg)
    return om, P, hist_o, hist_g


def test_column_steps_match_oracle_fp64(gpu):
    cfg = inputs.workload("column")
    om, P, ho, hg = run_steps(gpu, cfg, cfg["nsteps"])
    po, pg = om.points(), P.numpy()
    disp_o = po["x"] - inputs.make_points(cfg)["x"]
    disp_g = pg["x"] - inputs.make_points(cfg)["x"]
    assert np.max(np.abs(disp_g - disp_o)) <= 1e-9 * np.abs(disp_o).max()
    for k in ("F", "be", "lp"):
        assert np.max(np.abs(pg[k] - po[k])) <= 1e-9 * max(1.0, np.abs(po[k]).max())
    for a, b in zip(ho, hg):
        assert a["newton_its"] == b["newton_its"]


def test_punch_steps_match_oracle_fp64(gpu):
    cfg = inputs.workload("punch")
    om, P, ho, hg = run_steps(gpu, cfg, 3)
    for a, b in zip(ho, hg):
        assert abs(b["reaction"][2] - a["reaction"][2]) <= 1e-9 * abs(a["reaction"][2])
    po, pg = om.points(), P.numpy()
    x0 = po["x"]
    assert pg["x"].shape == x0.shape
    d = np.max(np.abs(pg["x"] - po["x"]))
    assert d <= 1e-9 * 0.1 * 3 / 50
    for k in ("F", "be", "lp"):
        assert np.max(np.abs(pg[k] - po[k])) <= 1e-9 * max(1.0, np.abs(po[k]).max()), k


def test_punch_steps_with_friction_match_oracle_fp64(gpu):
    # Coulomb friction mu = 0.3 (non-symmetric tangent: BiCGStab on both sides)
    cfg = inputs.workload("punch", mu=0.3)
    om, P, ho, hg = run_steps(gpu, cfg, 3)
    for a, b in zip(ho, hg):
        assert np.max(np.abs(b["reaction"] - a["reaction"])) <= 1e-9 * abs(a["reaction"][2])
    po, pg = om.points(), P.numpy()
    assert np.max(np.abs(pg["x"] - po["x"])) <= 1e-9 * 0.1 * 3 / 50
    for k in ("F", "be", "lp"):
        assert np.max(np.abs(pg[k] - po[k])) <= 1e-9 * max(1.0, np.abs(po[k]).max()), k
    # friction changes the load step against the frictionless run
    om0, P0, ho0, hg0 = run_steps(gpu, inputs.workload("punch"), 1)
    assert abs(hg[0]["reaction"][2] - hg0[0]["reaction"][2]) > 1e-6 * abs(hg0[0]["reaction"][2])


def test_triangulated_punch_steps_with_friction_match_oracle_fp64(gpu):
    # the flat punch as a closed 64-sided prism of triangles, mu = 0.3; the
    # polygon turned by half a side, so that no lattice corner lies on a
    # bisector between two wall faces (where the nearest face, and so the
    # contact normal, jumps, and a tie in the distance decides it)
    cfg = inputs.workload("punch", mu=0.3)
    cfg["body"] = dict(cfg["body"], kind=3, mesh=inputs.cylinder_mesh(0.1, 0.6, 64, phase=0.5))
    om, P, ho, hg = run_steps(gpu, cfg, 2)
    for a, b in zip(ho, hg):
        assert np.max(np.abs(b["reaction"] - a["reaction"])) <= 1e-9 * abs(a["reaction"][2])
    po, pg = om.points(), P.numpy()
    assert np.max(np.abs(pg["x"] - po["x"])) <= 1e-9 * 0.1 * 2 / 50
    for k in ("F", "be", "lp"):
        assert np.max(np.abs(pg[k] - po[k])) <= 1e-9 * max(1.0, np.abs(po[k]).max()), k


def test_cpt_willam_warnke_steps_match_oracle_fp64(gpu):
    # Sec. 6.4's CPT on a coarse quarter domain: the Willam-Warnke cone,
    # E50 by depth, self-weight ramped over 5 steps, the cone with friction
    # 0.3 in contact from step 3 on; five load steps, FP64, against the oracle
    cfg = inputs.workload("cpt", depth_min=4, depth_max=7, dx_region=2 * 25.6 / 128,
                          points=dict(spacing=0.8))
    om, P, ho, hg = run_steps(gpu, cfg, 5)
    assert abs(ho[-1]["reaction"][2]) > 0
    for a, b in zip(ho, hg):
        assert np.max(np.abs(b["reaction"] - a["reaction"])) <= 1e-9 * max(abs(a["reaction"][2]), 1.0)
    po, pg = om.points(), P.numpy()
    assert pg["x"].shape == po["x"].shape
    assert np.max(np.abs(pg["x"] - po["x"])) <= 1e-9 * 0.1
    for k in ("F", "be", "lp"):
        assert np.max(np.abs(pg[k] - po[k])) <= 1e-9 * max(1.0, np.abs(po[k]).max()), k


def test_punch_steps_mixed_precision_within_1e6(gpu):
    cfg = inputs.workload("punch")
    om, P, ho, hg = run_steps(gpu, cfg, 3, precision=1, tol=1e-8, lin_tol=1e-8)
    for a, b in zip(ho, hg):
        assert abs(b["reaction"][2] - a["reaction"][2]) <= 1e-6 * abs(a["reaction"][2])


def test_cone_drucker_prager_step_matches_oracle(gpu):
    # non-associated Drucker-Prager (BiCGStab) with the cone in contact: the
    # reactions and every point array at 1e-9 after two load steps.  Newton
    # to 2e-10: the oracle's own FP64 residual of this case stops falling at
    # 5e-11 to 8e-11 of |f| (rounding under the cone tip, where the penalty
    # stiffness is largest), after the quadratic drop 4e-7 -> 1e-10 of
    # iteration 6 in both load steps
    cfg = inputs.workload("cone")
    om, P, ho, hg = run_steps(gpu, cfg, 2, tol=2e-10, lin_tol=1e-13)
    for a, b in zip(ho, hg):
        ra, rb = a["reaction"][2], b["reaction"][2]
        assert abs(rb - ra) <= 1e-9 * abs(ra)
    po, pg = om.points(), P.numpy()
    assert pg["x"].shape == po["x"].shape
    x0 = inputs.make_points(cfg)["x"]
    du_o = po["x"][:len(x0)] - x0
    assert np.max(np.abs(pg["x"] - po["x"])) <= 1e-9 * max(np.abs(du_o).max(), 1e-12)
    for k in ("F", "be", "lp"):
        assert np.max(np.abs(pg[k] - po[k])) <= 1e-9 * max(1.0, np.abs(po[k]).max()), k


# ---------------------------------------------------------------- edge cases

def test_single_point_and_capacity_error(gpu):
    mpm, ctx, torch = gpu
    cfg = inputs.workload("column", depth_min=1, depth_max=1, contact=0,
                          points=dict(lo=(0.4, 0.4, 0.0), hi=(0.8, 0.8, 0.4), spacing=0.4))
    pts = inputs.make_points(cfg)
    # capacity 1: the split needs 8 points
    P = mpm.Points(pts, capacity=1)
    with pytest.raises(mpm.MPMError) as e:
        mpm.octree_build(ctx, cfg, P)
    assert e.value.code == 7
    # the context is still usable
    P = mpm.Points(pts, capacity=8)
    mesh = mpm.octree_build(ctx, cfg, P)
    assert mesh.info()["npts"] == 8
    om = oracle.Model(cfg, pts)
    om.build()
    assert np.array_equal(P.numpy()["x"], om.points()["x"])


def test_domain_outside_cube_is_reported(gpu):
    mpm, ctx, torch = gpu
    cfg = inputs.workload("column", depth_min=2, depth_max=2)
    pts = inputs.make_points(cfg)
    pts["x"][0] = [2.0, 2.0, 2.0]
    P = mpm.Points(pts)
    with pytest.raises(mpm.MPMError) as e:
        mpm.octree_build(ctx, cfg, P)
    assert e.value.code == 9
    P = mpm.Points(inputs.make_points(cfg))
    assert mpm.octree_build(ctx, cfg, P).info()["npts"] == len(pts["x"])


def test_bad_arguments_return_status(gpu):
    mpm, ctx, torch = gpu
    cfg = inputs.workload("column", depth_min=2, depth_max=1)
    P = mpm.Points(inputs.make_points(inputs.workload("column")))
    with pytest.raises(mpm.MPMError) as e:
        mpm.octree_build(ctx, cfg, P)
    assert e.value.code == 1


def test_krylov_cap_reports_status(gpu):
    # fault injection on the host side: an iteration cap of 1 must come back as
    # ERR_KRYLOV with the context left usable
    mpm, ctx, torch = gpu
    cfg, bz = CASES["punch_d3_6"]()
    om, mesh, P = both(gpu, cfg, bz)
    nd = mesh.info()["ndof"]
    g = mpm.assemble(ctx, mesh, cfg, torch.zeros(3 * nd, dtype=torch.float64, device="cuda"),
                     body_z=bz)
    with pytest.raises(mpm.MPMError) as e:
        mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-12, maxit=1)
    assert e.value.code == 4
    x, st = mpm.solve(ctx, mesh, cfg, g["K"], -g["R"], tol=1e-10, maxit=50000)
    assert st["status"] == 0


def test_nan_point_state_is_reported(gpu):
    mpm, ctx, torch = gpu
    cfg = inputs.workload("column")
    pts = inputs.make_points(cfg)
    pts["be"][5] = [np.nan] * 6
    om = oracle.Model(cfg, inputs.make_points(cfg))
    P = mpm.Points(pts)
    mesh = mpm.octree_build(ctx, cfg, P)
    nd = mesh.info()["ndof"]
    with pytest.raises(mpm.MPMError) as e:
        mpm.assemble(ctx, mesh, cfg, torch.zeros(3 * nd, dtype=torch.float64, device="cuda"))
    assert e.value.code == 5
