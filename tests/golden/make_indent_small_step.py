"""Writes indent_small_step1.npz: the oracle's first load step of the
indentation recipe one level coarser than the benchmark (depth 5 -> 6,
about 239 k points and 101 k unknowns), for the GPU parity test at the size
where the tangent's long-row pass and the multigrid's four coarse levels run.

Only the oracle is called.  Stored: the mesh counts, the Newton history, the
reaction, and the end-of-step state of 2000 seeded points (x, F, b_e, l_p).

  python tests/golden/make_indent_small_step.py     (about 6 minutes, one core)
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2606_09275_gb300 import inputs  # noqa: E402

TOL, LIN_TOL, NSAMPLE = 1e-12, 1e-13, 2000


def main():
    cfg = inputs.workload("indent_small")
    pts = inputs.make_points(cfg)
    m = oracle.Model(cfg, pts, body_z=inputs.body_z(cfg, 1))
    st = m.step(load=1.0, tol=TOL, maxit=30, lin_tol=LIN_TOL, lin_maxit=200000)
    assert st["status"] == 0, st
    c = m.counts()
    po = m.points()
    P = len(po["x"])
    idx = np.sort(np.random.default_rng(0).choice(P, size=min(NSAMPLE, P), replace=False))
    np.savez_compressed(
        os.path.join(HERE, "indent_small_step1.npz"),
        counts=np.array([c["nleaf"], c["nnode"], c["nhang"], c["ndof"], c["nnzb"], c["nghost"],
                         c["npts"]]),
        newton_its=st["newton_its"], res_hist=np.array(st["res_hist"]),
        reaction=np.array(st["reaction"]), idx=idx,
        x=po["x"][idx], F=po["F"][idx], be=po["be"][idx], lp=po["lp"][idx],
        tol=TOL, lin_tol=LIN_TOL)


if __name__ == "__main__":
    main()
