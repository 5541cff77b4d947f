"""The punch and adjoint workloads run over their whole load paths on the GPU.

* The flat punch into the von Mises block (depth 3 -> 6, re-adapted every
  step), all 50 load steps to 0.1 m, in FP64 and in the mixed-precision form
  (FP32 tangent and inner PCG inside FP64 refinement), from the same initial
  state, Newton to 1e-10 in both.  The discrete events of a step (splits,
  dofs, blocks) are discontinuous functions of the converged positions: a
  GIMP domain face that ends within rounding of a cell face overlaps that
  cell in one run and not in the other.  So the test compares the two runs
  while their events agree: the vertical reaction of the mixed run within
  1e-6 of the FP64 run's at every such step, at least 30 of the 50 steps
  with the same events, and after a divergence the two histories (of two
  slightly different discrete problems) within 1e-3.  (At a 1e-8 Newton
  tolerance the FP64 run itself leaves its own 1e-10 solution by up to 3e-3
  in the reaction from load step 26 on, and the mixed run by as much: from
  there on the tolerance decides, not the precision.)
* The adjoint workload (the punch at depth 3 -> 5, lognormal E, 20 load
  steps): the gradient of the final vertical reaction with respect to E_p
  from mpm_adjoint against central finite differences of the forward run on
  32 seeded random points.  Over 20 steps a relative change of 1e-4 in one
  E_p moves a discrete event (a split, a dof, a block) somewhere in the run
  for most points; the reaction then jumps and has no derivative, so only
  the points whose perturbed runs keep every event are compared.  Points
  whose perturbation switches a point between elastic and plastic are kept
  (those switches are not events of the mesh), so the check is norm-wise,
  against the largest gradient entry.  The same check runs at 55,296
  starting points (spacing 1/48, about 67 k after the first splits) over
  the first 8 load steps on 12 seeded points.
"""
import numpy as np
import pytest

from paper_2606_09275_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    import torch
    from paper_2606_09275_gb300 import autodiff, mpm
    assert torch.cuda.is_available()
    ctx = mpm.Context()
    yield mpm, autodiff, ctx, torch
    ctx.close()


def run_path(mpm, ctx, cfg, precision, nsteps, tol):
    pts = inputs.make_points(cfg)
    P = mpm.Points(pts, capacity=64 * len(pts["x"]))
    out = []
    for n in range(1, nsteps + 1):
        st = mpm.step(ctx, cfg, P, body_z=inputs.body_z(cfg, n), load=inputs.load_factor(cfg, n),
                      tol=tol, lin_tol=min(tol, 1e-8), lin_maxit=100000, precision=precision,
                      method=3, mg_reuse=1, inner_tol=1e-4, check=False)
        assert st["status"] == 0, (n, precision, st["res_hist"], ctx.error())
        out.append(st)
    return out


def test_punch_fifty_load_steps_mixed_against_fp64(gpu):
    mpm, _, ctx, _ = gpu
    cfg = inputs.workload("punch")
    assert cfg["nsteps"] == 50
    h64 = run_path(mpm, ctx, cfg, mpm.FP64, 50, 1e-10)
    hmx = run_path(mpm, ctx, cfg, mpm.MIXED, 50, 1e-10)
    ev = lambda s: (s["npts"], s["ndof"], s["nnzb"])
    same = [ev(a) == ev(b) for a, b in zip(hmx, h64)]
    first = same.index(False) if False in same else len(same)
    rel = [abs(a["reaction"][2] - b["reaction"][2]) / abs(b["reaction"][2]) for a, b in zip(hmx, h64)]
    print("punch: %d points, %d dofs at step 50; events agree through step %d; max reaction "
          "difference %.2e before, %.2e after" % (h64[-1]["npts"], h64[-1]["ndof"], first,
                                                 max(rel[:first]), max(rel[first:], default=0.0)))
    assert first >= 30, (first, [ev(s) for s in hmx[first:first + 1]], [ev(s) for s in h64[first:first + 1]])
    assert max(rel[:first]) <= 1e-6, rel
    assert max(rel, default=0.0) <= 1e-3, rel
    # the punch pushes into the block all the way: the reaction grows
    r = [abs(s["reaction"][2]) for s in h64]
    assert r[-1] > r[9] > r[0] > 0.0


def adjoint_against_fd(gpu, name, nsteps, npick, seed):
    """Gradient of the vertical reaction at the end of load step `nsteps` in
    E_p from mpm_adjoint against central FD of the forward run on `npick`
    seeded random points; returns the number of points whose perturbed runs
    kept every event, the largest |FD - adjoint| over max |dJ/dE| among them,
    and the run's statistics."""
    mpm, autodiff, ctx, torch = gpu
    cfg = inputs.workload(name)
    pts = inputs.make_points(cfg)
    path = autodiff.LoadPath(ctx, cfg, pts, nsteps)
    E = torch.tensor(pts["E"], device="cuda")
    ys = torch.tensor(pts["ys"], device="cuda")
    _, ckpts, stats = path.run(E, ys)
    w = (0.0, 0.0, 1.0)
    dE, _, _ = path.gradient(ckpts, w)
    dE = dE.cpu().numpy()
    scale = np.abs(dE).max()
    ev = [(s["npts"], s["ndof"], s["nnzb"]) for s in stats]
    rng = np.random.default_rng(seed)
    idx = rng.choice(len(pts["x"]), npick, replace=False)
    checked, worst = 0, 0.0
    for p in idx:
        vals, same = [], True
        h = 1e-4 * float(E[p])
        for sgn in (1.0, -1.0):
            Ep = E.clone()
            Ep[p] += sgn * h
            r, _, st = path.run(Ep, ys, keep=False)
            same = same and [(s["npts"], s["ndof"], s["nnzb"]) for s in st] == ev
            vals.append(float(np.dot(w, r.numpy())))
        if not same:
            continue  # the perturbation moved a discrete event: no derivative there
        fd = (vals[0] - vals[1]) / (2.0 * h)
        worst = max(worst, abs(fd - dE[p]) / scale)
        checked += 1
    return checked, worst, stats


def test_adjoint_twenty_load_steps_matches_finite_differences(gpu):
    assert inputs.workload("adjoint")["nsteps"] == 20
    checked, worst, _ = adjoint_against_fd(gpu, "adjoint", 20, 32, 11)
    print("adjoint, 20 steps: %d of 32 points keep their events; largest |FD - adjoint| %.2e of max |dJ/dE|"
          % (checked, worst))
    assert checked >= 6, checked
    assert worst <= 1e-4, worst


def test_adjoint_sixty_thousand_points_matches_finite_differences(gpu):
    # the same punch with 55,296 points at the start (spacing 1/48), over its
    # first 8 load steps, FD on 12 seeded points; over all 20 steps every one
    # of 8 sampled points moved an event: at about load step 12 this finer
    # block reaches its plastic limit load, where the step's solution is not
    # unique and the last bits of the start decide which one Newton reaches
    # (the oracle: both perturbed runs 0.63 mm from the base run there)
    checked, worst, stats = adjoint_against_fd(gpu, "adjoint_60k", 8, 12, 12)
    print("adjoint_60k, 8 steps: %d points at step 1, %d at step 8; %d of 12 points keep their "
          "events; largest |FD - adjoint| %.2e of max |dJ/dE|"
          % (stats[0]["npts"], stats[-1]["npts"], checked, worst))
    assert stats[0]["npts"] >= 60000, stats[0]["npts"]
    assert checked >= 2, checked
    assert worst <= 1e-4, worst
