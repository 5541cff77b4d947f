"""GPU load step against the oracle's at the size where the tangent's long-row
pass and the multigrid's four coarse levels run: the first FP64 load step of
the indentation recipe one level coarser than the benchmark (depth 5 -> 6,
239 k points, 101 k unknowns), Newton to 1e-12 with a multigrid-preconditioned
PCG to 1e-13.  The oracle needs about six minutes for this step, so its
result is stored by tests/golden/make_indent_small_step.py (which calls only
the oracle): mesh counts, the Newton iteration count, the reaction and the
end-of-step state of 2000 seeded points, compared at 1e-9."""
import os

import numpy as np
import pytest

from paper_2606_09275_gb300 import inputs

pytestmark = pytest.mark.gpu

GOLD = os.path.join(os.path.dirname(__file__), "golden", "indent_small_step1.npz")


def test_indent_small_first_step_matches_oracle():
    import torch
    from paper_2606_09275_gb300 import mpm
    g = np.load(GOLD)
    cfg = inputs.workload("indent_small")
    pts = inputs.make_points(cfg)
    ctx = mpm.Context()
    P = mpm.Points(pts, capacity=2 * len(pts["x"]))
    st = mpm.step(ctx, cfg, P, body_z=inputs.body_z(cfg, 1), load=1.0, tol=float(g["tol"]),
                  lin_tol=float(g["lin_tol"]), lin_maxit=100000, precision=mpm.FP64, method=3)
    torch.cuda.synchronize()
    nleaf, nnode, nhang, ndof, nnzb, nghost, npts = [int(v) for v in g["counts"]]
    assert (st["npts"], st["ndof"], st["nnzb"]) == (npts, ndof, nnzb)
    assert st["newton_its"] == int(g["newton_its"])
    ro, rg = g["reaction"], st["reaction"]
    assert np.max(np.abs(rg - ro)) <= 1e-9 * np.abs(ro).max(), (rg, ro)
    pg = P.numpy()
    idx = g["idx"]
    dz = abs(cfg["body"]["dz"])
    assert np.max(np.abs(pg["x"][idx] - g["x"])) <= 1e-9 * dz
    for k in ("F", "be", "lp"):
        assert np.max(np.abs(pg[k][idx] - g[k])) <= 1e-9 * max(1.0, np.abs(g[k]).max()), k
    ctx.close()
