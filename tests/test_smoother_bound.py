"""The bound behind the multigrid smoother's weight, on tangents the oracle
assembles: for the symmetric positive definite stiffness K and the l1 block
Jacobi matrix M = blockdiag(K_ii) + diag(sum over j != i of |K_ij| row sums),
every generalized eigenvalue of (K, M) lies in (0, 1].  Hence the damped
step x += w M^-1 (b - K x) converges and 2 M / w - K stays positive definite
(the V(1,1) cycle stays SPD) for every weight w < 2, in particular the 1.9
the CUDA V-cycle uses.  No GPU needed."""
import numpy as np
import pytest
import scipy.linalg as sla

import oracle
from paper_2606_09275_gb300 import inputs

W = 1.9


def tiny_cfg(**over):
    pts = dict(spacing=0.25)
    pts.update(over.pop("points", {}))
    c = inputs.workload("punch", depth_min=1, depth_max=3, dx_region=0.15,
                        body=dict(cx=0.3, cy=0.4, z0=0.5, r=0.1), points=pts)
    c.update(over)
    return c


def dense_free(m, K):
    nd = m.counts()["ndof"]
    rp, col = m.pattern()
    A = np.zeros((3 * nd, 3 * nd))
    for i in range(nd):
        for s in range(rp[i], rp[i + 1]):
            j = col[s]
            A[3 * i:3 * i + 3, 3 * j:3 * j + 3] = K[s]
    mask = m.bcmask()
    free = np.array([not (mask[i // 3] >> (i % 3)) & 1 for i in range(3 * nd)])
    return A, free


def l1_block_jacobi(A, free):
    n = A.shape[0] // 3
    Af = np.where(np.outer(free, free), A, 0.0)
    M = np.zeros_like(A)
    for i in range(n):
        b = slice(3 * i, 3 * i + 3)
        M[b, b] = Af[b, b]
        off = np.abs(Af[b, :]).sum(axis=1) - np.abs(Af[b, b]).sum(axis=1)
        M[b, b] += np.diag(off)
    return Af[np.ix_(free, free)], M[np.ix_(free, free)]


@pytest.mark.parametrize("plastic", [False, True])
def test_l1_block_jacobi_bounds_the_stiffness(plastic):
    cfg = tiny_cfg()
    if plastic:
        cfg["points"]["ys"] = 2e4
    m = oracle.Model(cfg, inputs.make_points(cfg), body_z=0.49)
    m.build()
    n3 = 3 * m.counts()["ndof"]
    du = 2e-4 * np.random.default_rng(3).standard_normal(n3) if plastic else np.zeros(n3)
    out = m.assemble(du)
    A, free = dense_free(m, out["K"])
    Kf, Mf = l1_block_jacobi(A, free)
    assert np.allclose(Kf, Kf.T, atol=1e-9 * np.abs(Kf).max())
    Kf = 0.5 * (Kf + Kf.T)
    assert np.linalg.eigvalsh(Kf).min() > 0.0
    lam = sla.eigh(Kf, Mf, eigvals_only=True)
    assert lam.min() > 0.0 and lam.max() <= 1.0 + 1e-12, (lam.min(), lam.max())
    # the smoothing iteration matrix I - w M^-1 K is a contraction, and the
    # V(1,1) condition 2 M / w - K > 0 holds with margin
    assert np.abs(1.0 - W * lam).max() < 1.0
    assert np.linalg.eigvalsh(2.0 * Mf / W - Kf).min() > 0.0
    # the bound is loose on these meshes: M^-1 K reaches well below 1, which
    # is what makes a weight near 2 pay
    print("generalized eigenvalues of (K, M): [%.3e, %.3f]" % (lam.min(), lam.max()))
    assert lam.max() < 0.9


@pytest.mark.parametrize("plastic", [False, True])
def test_fp16_operator_copy_keeps_the_vcycle_positive_definite(plastic):
    # the fine level of the V-cycle applies an FP16 copy of K (scaled by a
    # power of two so that its largest entry sits just below 2^15, rounded to
    # nearest) with the l1 block Jacobi M of the unrounded K: the cycle stays
    # SPD while the rounded operator K_h is SPD and 2 M / w - K_h > 0; the
    # rounding moves each entry by at most 2^-11 of itself, far inside the
    # 5 % margin of 2 / w = 1.053
    cfg = tiny_cfg()
    if plastic:
        cfg["points"]["ys"] = 2e4
    m = oracle.Model(cfg, inputs.make_points(cfg), body_z=0.49)
    m.build()
    n3 = 3 * m.counts()["ndof"]
    du = 2e-4 * np.random.default_rng(3).standard_normal(n3) if plastic else np.zeros(n3)
    out = m.assemble(du)
    A, free = dense_free(m, out["K"])
    Kf, Mf = l1_block_jacobi(A, free)
    Kf = 0.5 * (Kf + Kf.T)
    e = 14 - int(np.ceil(np.log2(np.abs(Kf).max())))
    Kh = (Kf * 2.0 ** e).astype(np.float16).astype(np.float64) * 2.0 ** -e
    assert np.abs(Kh - Kf).max() <= 2.0 ** -11 * np.abs(Kf).max()
    assert np.linalg.eigvalsh(Kh).min() > 0.0
    lam = sla.eigh(Kh, Mf, eigvals_only=True)
    assert lam.max() < 2.0 / W, lam.max()
    assert np.linalg.eigvalsh(2.0 * Mf / W - Kh).min() > 0.0
