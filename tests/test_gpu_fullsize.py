"""Checks at the size the benchmark times (the indentation workload: about
1.87 M points, 248 k dofs, 28 M 3x3 blocks), where the oracle is too slow to
rebuild the whole mesh: properties that hold at any size, checked on every
point or on seeded samples, and FP64 residuals recomputed on the host.

* discrete GIMP basis (Eq. GIMP numerical): partition of unity, zero gradient
  sum and linear completeness of S and grad S on every point whose domain lies
  inside the cube;
* stiffness: block symmetry on sampled blocks; rigid translations in the
  kernel of the internal-force tangent on sampled rows away from contact and
  Dirichlet planes;
* Krylov: the multigrid PCG solution's relative residual recomputed in FP64
  from the exported blocks, FP64 and mixed;
* one load step: mixed precision against FP64 on the same initial state.
"""
import numpy as np
import pytest

from paper_2606_09275_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def big():
    import torch
    from paper_2606_09275_gb300 import mpm
    assert torch.cuda.is_available()
    ctx = mpm.Context()
    cfg = inputs.workload("indent")
    pts = inputs.make_points(cfg)
    P = mpm.Points(pts, capacity=2 * len(pts["x"]))
    bz = inputs.body_z(cfg, 1)
    mesh = mpm.octree_build(ctx, cfg, P, body_z=bz)
    return dict(mpm=mpm, ctx=ctx, torch=torch, cfg=cfg, pts=pts, P=P, bz=bz, mesh=mesh)


def dof_positions(mesh, cfg):
    coord = mesh.export("node_coord").astype(np.float64)
    ndof = mesh.info()["ndof"]
    nd = mesh.export("node_dof")
    pos = np.zeros((ndof, 3))
    sel = nd >= 0
    pos[nd[sel]] = coord[sel] * cfg["L"] / (1 << cfg["depth_max"])
    return pos


def test_basis_partition_and_linear_completeness_on_every_point(big):
    mesh, cfg = big["mesh"], big["cfg"]
    info = mesh.info()
    assert info["ndof"] > 200000 and info["npts"] > 1800000
    nsup = mesh.export("nsup")
    sidx = mesh.export("sidx")
    S = mesh.export("S")
    dS = mesh.export("dS")
    pts = big["P"].numpy()
    x, lp = pts["x"], pts["lp"]
    inside = np.all((x - lp > 1e-9) & (x + lp < cfg["L"] - 1e-9), axis=1)
    assert inside.mean() > 0.8
    valid = np.arange(64)[None, :] < nsup[:, None]
    pos = dof_positions(mesh, cfg)
    Sv = np.where(valid, S, 0.0)[inside]
    dSv = np.where(valid[..., None], dS, 0.0)[inside]
    xv = pos[np.where(valid, sidx, 0)][inside]
    assert np.max(np.abs(Sv.sum(1) - 1.0)) < 1e-12
    gscale = (1 << cfg["depth_max"]) / cfg["L"]
    assert np.max(np.abs(dSv.sum(1))) < 1e-11 * gscale
    # (domain bounds within 1e-9 grid units of a grid plane are snapped onto it)
    assert np.max(np.abs(np.einsum("pk,pkd->pd", Sv, xv) - x[inside])) < 1e-10 * cfg["L"]
    grad_x = np.einsum("pke,pkd->ped", dSv, xv)
    assert np.max(np.abs(grad_x - np.eye(3)[None])) < 1e-10


def blocks_and_pattern(big, precision):
    mpm, ctx, torch, mesh, cfg = big["mpm"], big["ctx"], big["torch"], big["mesh"], big["cfg"]
    nd = mesh.info()["ndof"]
    g = mpm.assemble(ctx, mesh, cfg, torch.zeros(3 * nd, dtype=torch.float64, device="cuda"),
                     precision=precision, body_z=big["bz"])
    Kb = mpm.blocks(ctx, mesh, g["K"], precision)
    return g, Kb, mesh.export("row_ptr"), mesh.export("col")


def test_stiffness_symmetry_and_rigid_translations(big):
    mesh = big["mesh"]
    g, Kb, rp, col = blocks_and_pattern(big, 0)
    nd = len(rp) - 1
    rng = np.random.default_rng(5)
    del g
    row = np.repeat(np.arange(nd), np.diff(rp))
    pick = rng.choice(len(col), size=20000, replace=False)
    scale = np.abs(Kb).max()
    for s in pick:
        r, c = row[s], col[s]
        t = rp[c] + np.searchsorted(col[rp[c]:rp[c + 1]], r)
        assert col[t] == r
        assert np.max(np.abs(Kb[s] - Kb[t].T)) <= 1e-11 * scale
    # rigid translations lie in the kernel of the internal-force and ghost
    # tangents: rows of free dofs, all of whose columns are free, away from
    # the punch (the contact stiffness does not vanish on translations)
    mask = mesh.export("bcmask")
    pos = dof_positions(mesh, big["cfg"])
    body = big["cfg"]["body"]
    far = (np.hypot(pos[:, 0] - body["cx"], pos[:, 1] - body["cy"]) > body["r"] + 0.05) | \
          (pos[:, 2] < big["bz"] - 0.05)
    cand = np.flatnonzero((mask == 0) & far)
    rows = rng.choice(cand, size=5000, replace=False)
    checked = 0
    for r in rows:
        cols = col[rp[r]:rp[r + 1]]
        if (mask[cols] != 0).any():
            continue
        blk = Kb[rp[r]:rp[r + 1]]
        assert np.max(np.abs(blk.sum(0))) <= 1e-9 * np.abs(blk).max(), r
        checked += 1
    assert checked > 1000


@pytest.mark.parametrize("precision", [0, 1])
def test_multigrid_solution_residual_in_fp64(big, precision):
    import scipy.sparse as sp
    mpm, ctx, mesh, cfg = big["mpm"], big["ctx"], big["mesh"], big["cfg"]
    g, Kb, rp, col = blocks_and_pattern(big, precision)
    nd = len(rp) - 1
    b = -g["R"]
    x, st = mpm.solve(ctx, mesh, cfg, g["K"], b, precision=precision, tol=1e-8, maxit=20000,
                      method=3, inner_tol=1e-4)
    assert st["status"] == 0
    K = sp.bsr_matrix((Kb, col, rp), shape=(3 * nd, 3 * nd))
    mask = mesh.export("bcmask")
    free = np.array([[not (m >> c) & 1 for c in range(3)] for m in mask]).ravel()
    bh = b.cpu().numpy() * free
    r = bh - K @ x.cpu().numpy()
    rel = np.linalg.norm(r[free]) / np.linalg.norm(bh)
    # the residual of the exported matrix (FP32 values for the mixed path, whose
    # refinement residual is accumulated in double-float) meets the tolerance
    assert rel <= 1.2e-8, rel


def test_first_load_step_mixed_against_fp64(big):
    mpm, ctx, cfg, pts = big["mpm"], big["ctx"], big["cfg"], big["pts"]
    out = {}
    for prec in (0, 1):
        P = mpm.Points(pts, capacity=2 * len(pts["x"]))
        out[prec] = mpm.step(ctx, cfg, P, body_z=inputs.body_z(cfg, 1), tol=1e-8, lin_tol=1e-8,
                             lin_maxit=20000, precision=prec, method=3, mg_reuse=1,
                             inner_tol=1e-4)
    a, b = out[0], out[1]
    assert (a["npts"], a["ndof"], a["nnzb"]) == (b["npts"], b["ndof"], b["nnzb"])
    rel = abs(b["reaction"][2] - a["reaction"][2]) / abs(a["reaction"][2])
    print("first step reaction: FP64 %.9e, mixed %.9e, relative difference %.2e" % (
        a["reaction"][2], b["reaction"][2], rel))
    assert rel <= 1e-6
