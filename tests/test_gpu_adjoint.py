"""The adjoint of the load steps (mpm_adjoint, through the C ABI and the
torch.autograd.Function) against central finite differences of the forward
run: of the CUDA forward on 32 seeded random points, and of the oracle's
forward on a few points.

The workload is the punch on a von Mises block (depth 2 -> 4, 8 x 8 x 4
points, lognormal E), three load steps; the functional is the vertical
reaction on the punch at the end of the last step.  Finite differences take
a relative step of 1e-4 with Newton converged to 1e-12; the discrete events
(splits, supports, pattern) are checked to be the same in the perturbed runs.
"""
import numpy as np
import pytest

import oracle
from paper_2606_09275_gb300 import inputs

pytestmark = pytest.mark.gpu

NSTEPS = 3
REL = 1e-4
W = (0.0, 0.0, 1.0)


def adj_cfg(**over):
    c = inputs.workload("adjoint", depth_min=2, depth_max=4, dx_region=2.0 / 16,
                        points=dict(spacing=1.0 / 8, E_sigma=0.2, seed=3, jitter=0.0))
    c.update(over)
    return c


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2606_09275_gb300 import autodiff, mpm
    assert torch.cuda.is_available()
    ctx = mpm.Context()
    return mpm, autodiff, ctx, torch


@pytest.fixture(scope="module")
def problem(gpu):
    mpm, autodiff, ctx, torch = gpu
    cfg = adj_cfg()
    pts = inputs.make_points(cfg)
    path = autodiff.LoadPath(ctx, cfg, pts, NSTEPS)
    E = torch.tensor(pts["E"], device="cuda")
    ys = torch.tensor(pts["ys"], device="cuda")
    reaction, ckpts, stats = path.run(E, ys)
    dE, dys, st = path.gradient(ckpts, W)
    return dict(cfg=cfg, pts=pts, path=path, E=E, ys=ys, reaction=reaction.numpy(), stats=stats,
                dE=dE.cpu().numpy(), dys=dys.cpu().numpy(), adj_stats=st)


def events(stats):
    return [(s["npts"], s["ndof"], s["nnzb"]) for s in stats]


def gpu_fd(problem, torch, which, p):
    """Central difference of the vertical reaction in E_p or ys_p."""
    path = problem["path"]
    vals = []
    for sgn in (1.0, -1.0):
        E, ys = problem["E"].clone(), problem["ys"].clone()
        t = E if which == "E" else ys
        h = REL * float(t[p])
        t[p] += sgn * h
        r, _, st = path.run(E, ys, keep=False)
        assert events(st) == events(problem["stats"]), "perturbation changed a discrete event"
        vals.append(float(np.dot(W, r.numpy())))
    return (vals[0] - vals[1]) / (2.0 * h)


def test_adjoint_reaction_is_the_forward_reaction(problem):
    r_fwd = problem["reaction"]
    r_adj = problem["adj_stats"]["reaction"]
    assert np.allclose(r_adj, r_fwd, rtol=1e-9, atol=1e-12 * np.abs(r_fwd).max())
    # the punch pushes down: the reaction on it points up
    assert r_fwd[2] > 0.0
    assert problem["adj_stats"]["lin_its"] > 0


def test_adjoint_matches_gpu_fd_on_32_random_points(gpu, problem):
    mpm, autodiff, ctx, torch = gpu
    dE = problem["dE"]
    scale = np.abs(dE).max()
    assert scale > 0.0
    rng = np.random.default_rng(11)
    # random points among those the reaction depends on (above 1e-3 of the largest)
    live = np.flatnonzero(np.abs(dE) > 1e-3 * scale)
    assert len(live) >= 32
    pick = rng.choice(live, size=32, replace=False)
    worst = 0.0
    for p in pick:
        fd = gpu_fd(problem, torch, "E", int(p))
        err = abs(fd - dE[p]) / (abs(fd) + 1e-3 * scale)
        worst = max(worst, err)
        assert err <= 2e-5, (int(p), fd, dE[p])
    print("adjoint vs GPU FD in E: worst relative error %.2e" % worst)


def test_adjoint_yield_stress_matches_gpu_fd(gpu, problem):
    mpm, autodiff, ctx, torch = gpu
    dys = problem["dys"]
    scale = np.abs(dys).max()
    assert scale > 0.0, "no plastic point in the workload"
    order = np.argsort(-np.abs(dys))
    rng = np.random.default_rng(12)
    pick = list(order[:4]) + list(rng.choice(order[4:40], size=4, replace=False))
    for p in pick:
        fd = gpu_fd(problem, torch, "ys", int(p))
        err = abs(fd - dys[p]) / (abs(fd) + 1e-3 * scale)
        assert err <= 2e-5, (int(p), fd, dys[p])


def oracle_reaction(cfg, pts):
    om = oracle.Model(cfg, pts)
    hist = []
    for n in range(1, NSTEPS + 1):
        om.set_body_z(inputs.body_z(cfg, n))
        s = om.step(load=inputs.load_factor(cfg, n), tol=1e-12, lin_tol=1e-13)
        assert s["status"] == 0
        hist.append(om.counts()["npts"])
    return float(np.dot(W, s["reaction"])), hist


def test_adjoint_matches_oracle_fd(problem):
    cfg, pts = problem["cfg"], problem["pts"]
    dE, dys = problem["dE"], problem["dys"]
    r0, ev0 = oracle_reaction(cfg, pts)
    assert abs(r0 - np.dot(W, problem["reaction"])) <= 1e-9 * abs(r0)
    cases = [("E", int(np.argmax(np.abs(dE)))), ("E", int(np.argsort(-np.abs(dE))[7])),
             ("ys", int(np.argmax(np.abs(dys))))]
    for which, p in cases:
        vals = []
        for sgn in (1.0, -1.0):
            q = {k: v.copy() for k, v in pts.items()}
            h = REL * q[which][p]
            q[which][p] += sgn * h
            r, ev = oracle_reaction(cfg, q)
            assert ev == ev0
            vals.append(r)
        fd = (vals[0] - vals[1]) / (2.0 * h)
        ref = dE if which == "E" else dys
        assert abs(fd - ref[p]) <= 2e-4 * abs(fd) + 1e-6 * np.abs(ref).max(), (which, p, fd, ref[p])


def test_autograd_function_and_linearity_in_w(gpu, problem):
    mpm, autodiff, ctx, torch = gpu
    path = problem["path"]
    E = problem["E"].clone().requires_grad_(True)
    ys = problem["ys"].clone().requires_grad_(True)
    r = autodiff.reaction(path, E, ys)
    w = torch.tensor([0.3, -0.2, 1.5], dtype=torch.float64)
    (r * w).sum().backward()
    # the same through the C ABI, one reaction component at a time
    _, ckpts, _ = path.run(problem["E"], problem["ys"])
    parts = [path.gradient(ckpts, np.eye(3)[d]) for d in range(3)]
    gE = sum(float(w[d]) * parts[d][0].cpu().numpy() for d in range(3))
    gy = sum(float(w[d]) * parts[d][1].cpu().numpy() for d in range(3))
    aE, ay = E.grad.cpu().numpy(), ys.grad.cpu().numpy()
    assert np.max(np.abs(aE - gE)) <= 1e-9 * np.abs(gE).max()
    assert np.max(np.abs(ay - gy)) <= 1e-9 * max(np.abs(gy).max(), 1e-300)
    assert np.allclose(parts[2][0].cpu().numpy(), problem["dE"], rtol=1e-9,
                       atol=1e-12 * np.abs(problem["dE"]).max())


def test_adjoint_rejects_the_non_symmetric_model(gpu):
    mpm, autodiff, ctx, torch = gpu
    cfg = adj_cfg(model=2, phi=0.5, psi=0.0)
    pts = inputs.make_points(cfg)
    P = mpm.Points(pts, capacity=64 * len(pts["x"]))
    with pytest.raises(mpm.MPMError) as e:
        mpm.adjoint(ctx, cfg, [(P, inputs.body_z(cfg, 1), 1.0)], W)
    assert e.value.code == 1


def test_adjoint_with_multigrid_pcg_matches(gpu, problem):
    # the same gradient when forward and adjoint solves use the multigrid PCG
    mpm, autodiff, ctx, torch = gpu
    path = autodiff.LoadPath(ctx, problem["cfg"], problem["pts"], NSTEPS, method=3, mg_reuse=1)
    r, ck, _ = path.run(problem["E"], problem["ys"])
    dE, dys, _ = path.gradient(ck, W)
    dE, dys = dE.cpu().numpy(), dys.cpu().numpy()
    assert np.allclose(r.numpy(), problem["reaction"], rtol=1e-9)
    assert np.max(np.abs(dE - problem["dE"])) <= 1e-7 * np.abs(problem["dE"]).max()
    assert np.max(np.abs(dys - problem["dys"])) <= 1e-7 * np.abs(problem["dys"]).max()


def test_adjoint_from_stored_increments_equals_resolve(gpu, problem):
    # checkpoints with the forward's converged increments (no Newton re-solve in
    # the reverse pass) give the gradient of the re-solving adjoint
    mpm, autodiff, ctx, torch = gpu
    path = autodiff.LoadPath(ctx, problem["cfg"], problem["pts"], NSTEPS, store_increments=False)
    _, ck, _ = path.run(problem["E"], problem["ys"])
    assert all(len(c) == 3 for c in ck)
    dE, dys, st = path.gradient(ck, W)
    dE, dys = dE.cpu().numpy(), dys.cpu().numpy()
    assert np.max(np.abs(dE - problem["dE"])) <= 1e-8 * np.abs(problem["dE"]).max()
    assert np.max(np.abs(dys - problem["dys"])) <= 1e-8 * np.abs(problem["dys"]).max()
    assert st["ms_forward"] > problem["adj_stats"]["ms_forward"]
