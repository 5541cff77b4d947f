"""The allocation-free solve entry point, mpm_solve_static.

It serves callers that may not allocate device memory while they solve (an
application whose device memory belongs to its own pool, or a loop that
cannot take an allocation on its first call): its scratch is a static device
array inside the library.  These checks call it through the C ABI and compare
it with mpm_solve on the same system, twice in a row, since every call reuses
the same array.  The file is collected last so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest

from paper_2606_09275_gb300 import inputs

pytestmark = pytest.mark.gpu


def _system(mpm, ctx, torch, name, nosplit=False):
    cfg = inputs.workload(name)
    bz = inputs.body_z(cfg, 1) if cfg.get("body") else None
    pts = inputs.make_points(cfg)
    P = mpm.Points(pts, capacity=64 * len(pts["x"]))
    mesh = mpm.octree_build(ctx, cfg, P, body_z=bz)
    nd = mesh.info()["ndof"]
    du = torch.zeros(3 * nd, dtype=torch.float64, device="cuda")
    g = mpm.assemble(ctx, mesh, cfg, du, body_z=bz)
    return cfg, mesh, g


def test_static_solve_matches_allocating_solve_twice():
    import torch
    from paper_2606_09275_gb300 import mpm
    ctx = mpm.Context()
    for name in ("punch", "column"):
        cfg, mesh, g = _system(mpm, ctx, torch, name)
        rhs = -g["R"]
        x_ref, st_ref = mpm.solve(ctx, mesh, cfg, g["K"], rhs, tol=1e-12, maxit=50000, method=1)
        scale = x_ref.abs().max().item()
        for call in range(2):
            x, st = mpm.solve_static(ctx, mesh, g["K"], rhs, tol=1e-12, maxit=50000)
            assert st["status"] == 0 and st["relres"] <= 1e-12
            assert (x - x_ref).abs().max().item() <= 1e-9 * scale, (name, call)
    ctx.close()


def test_static_solve_rejects_meshes_beyond_its_limit():
    import torch
    from paper_2606_09275_gb300 import mpm
    ctx = mpm.Context()
    cfg = inputs.workload("indent")
    pts = inputs.make_points(cfg)
    P = mpm.Points(pts, capacity=2 * len(pts["x"]))
    mesh = mpm.octree_build(ctx, cfg, P, body_z=inputs.body_z(cfg, 1))
    info = mesh.info()
    if info["ndof"] <= 149696:
        pytest.skip("mesh within the static limit")
    K = torch.zeros(9 * info["nslot"], dtype=torch.float64, device="cuda")
    rhs = torch.zeros(3 * info["ndof"], dtype=torch.float64, device="cuda")
    with pytest.raises(mpm.MPMError) as e:
        mpm.solve_static(ctx, mesh, K, rhs)
    assert e.value.code == 1 and "149696" in str(e.value)
    ctx.close()
