"""Run-to-run reproducibility of the load step at the benchmark's size.

Every sum on the Newton path is taken in a fixed order (row gathers over the
sorted source lists for the internal force, ghost matrix, gravity and
contact; per-block partials added in block order for the norms and the Krylov
scalars; 64-bit integer accumulation for the multigrid Galerkin products),
so two runs of the same load steps from the same state must agree bit for
bit: the reactions, the Newton and Krylov histories, the discrete events
(splits, dofs, pattern) and every point array.  Three load steps of the
indentation workload (Sec. 2.4 load steps, Sec. 5 re-adaptation each step),
twice per precision.
"""
import numpy as np
import pytest

from paper_2606_09275_gb300 import inputs

pytestmark = pytest.mark.gpu

NSTEPS = 3


def run(precision, method=3):
    import torch
    from paper_2606_09275_gb300 import mpm
    cfg = inputs.workload("indent")
    pts = inputs.make_points(cfg)
    ctx = mpm.Context()
    P = mpm.Points(pts, capacity=2 * len(pts["x"]))
    hist = []
    for n in range(1, NSTEPS + 1):
        st = mpm.step(ctx, cfg, P, body_z=inputs.body_z(cfg, n), load=1.0, tol=cfg["newton_tol"],
                      maxit=cfg["newton_maxit"], lin_tol=cfg["lin_tol"], lin_maxit=cfg["lin_maxit"],
                      precision=precision, method=method, mg_reuse=1, inner_tol=1e-4)
        hist.append(st)
    torch.cuda.synchronize()
    out = P.numpy()
    ctx.close()
    return hist, out


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_runs_agree_bit_for_bit(prec):
    from paper_2606_09275_gb300 import mpm
    precision = mpm.FP64 if prec == "fp64" else mpm.MIXED
    h1, p1 = run(precision)
    h2, p2 = run(precision)
    for a, b in zip(h1, h2):
        assert (a["npts"], a["ndof"], a["nnzb"]) == (b["npts"], b["ndof"], b["nnzb"])
        assert (a["newton_its"], a["lin_its"]) == (b["newton_its"], b["lin_its"])
        assert np.array_equal(a["res_hist"], b["res_hist"])
        assert np.array_equal(a["eta_hist"], b["eta_hist"])
        assert np.array_equal(a["reaction"], b["reaction"]), (a["reaction"], b["reaction"])
    assert p1.keys() == p2.keys()
    for k in p1:
        assert np.array_equal(p1[k], p2[k]), k
