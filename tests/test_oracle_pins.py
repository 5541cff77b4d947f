"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: brute force
on small inputs, closed forms, invariants, the paper's worked examples and
printed constants.  None of them needs a GPU.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2606_09275_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def tiny_cfg(**over):
    """Small adapted octree with hanging nodes: depth 1 -> 3 around a punch."""
    pts = dict(spacing=0.25)
    pts.update(over.pop("points", {}))
    c = inputs.workload("punch", depth_min=1, depth_max=3, dx_region=0.15,
                        body=dict(cx=0.3, cy=0.4, z0=0.5, r=0.1), points=pts)
    c.update(over)
    return c


def built(cfg, pts=None, body_z=None, nosplit=False):
    pts = inputs.make_points(cfg) if pts is None else pts
    m = oracle.Model(cfg, pts, body_z=body_z)
    m.build(nosplit=nosplit)
    return m


def read_golden(name):
    out = {}
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        k, *v = line.split()
        out[k] = [float(x) for x in v]
    return out


# ---------------------------------------------------------------- octree (Sec. 3.1, Sec. 5)

def leaf_boxes(m):
    lev, anc = m.tree()
    D = m.cfg["depth_max"]
    s = (1 << (D - lev)).astype(np.int64)
    return lev, anc.astype(np.int64), s, D


def test_leaves_tile_the_cube():
    m = built(tiny_cfg())
    lev, anc, s, D = leaf_boxes(m)
    N = 1 << D
    assert int(np.sum(s ** 3)) == N ** 3
    occ = np.zeros((N, N, N), np.int32)
    for a, sz in zip(anc, s):
        occ[a[0]:a[0] + sz, a[1]:a[1] + sz, a[2]:a[2] + sz] += 1
    assert occ.min() == 1 and occ.max() == 1


def test_two_to_one_balance_brute_force():
    # Sec. 5: at most one hanging node per edge/face -> face and edge neighbours
    # differ by at most one level (checked over all leaf pairs)
    m = built(tiny_cfg())
    lev, anc, s, D = leaf_boxes(m)
    lo = anc
    hi = anc + s[:, None]
    n = len(lev)
    for i in range(n):
        ov_lo = np.maximum(lo[i], lo)
        ov_hi = np.minimum(hi[i], hi)
        ext = ov_hi - ov_lo
        touch = np.all(ext >= 0, axis=1)
        pos = np.sum(ext > 0, axis=1)
        nb = touch & (pos >= 1)  # share a face (2 positive extents) or an edge (1)
        nb[i] = False
        assert np.all(np.abs(lev[nb] - lev[i]) <= 1), i


def test_refinement_reaches_body():
    # Step 1 of Sec. 5: every leaf meeting the rigid body is at depth_max
    cfg = tiny_cfg()
    m = built(cfg)
    lev, anc, s, D = leaf_boxes(m)
    unit = cfg["L"] / (1 << D)
    b = cfg["body"]
    lo = anc * unit
    hi = (anc + s[:, None]) * unit
    dx = np.maximum(np.maximum(lo[:, 0] - b["cx"], 0), b["cx"] - hi[:, 0])
    dy = np.maximum(np.maximum(lo[:, 1] - b["cy"], 0), b["cy"] - hi[:, 1])
    meets = (hi[:, 2] >= b["z0"]) & (np.hypot(dx, dy) <= b["r"])
    assert meets.any()
    assert np.all(lev[meets] == cfg["depth_max"])


def test_hanging_definition_brute_force():
    # Eq. (hanging node): x_n on the boundary of some leaf K and not a vertex of K
    m = built(tiny_cfg())
    lev, anc, s, D = leaf_boxes(m)
    nd = m.nodes()
    lo, hi = anc, anc + s[:, None]
    for n, X in enumerate(nd["coord"].astype(np.int64)):
        inside = np.all((lo <= X) & (X <= hi), axis=1)
        vertex = np.all((X == lo) | (X == hi), axis=1)
        expect = bool(np.any(inside & ~vertex))
        assert bool(nd["hang"][n]) == expect, n


def test_constraint_weights_reproduce_linear_fields():
    # Eq. (constraint equation reduced): a hanging node's resolved weights
    # interpolate any linear field exactly, sum to one, and refer only to
    # independent nodes; weights are products of 1/2 and 1/4 (2:1 balance)
    m = built(tiny_cfg())
    nd = m.nodes()
    X = nd["coord"].astype(np.float64)
    rng = np.random.default_rng(3)
    A = rng.normal(size=(3, 3))
    f = X @ A.T
    hang = np.nonzero(nd["hang"])[0]
    assert len(hang) > 10
    for n in hang:
        a, b = nd["cptr"][n], nd["cptr"][n + 1]
        ids, w = nd["cidx"][a:b], nd["cw"][a:b]
        assert abs(w.sum() - 1.0) < 1e-15
        assert not np.any(nd["hang"][ids])
        assert np.allclose(w @ f[ids], f[n], rtol=0, atol=1e-12)
        for wi in w:
            k = math.log2(wi)
            assert k == int(k)


# ---------------------------------------------------------------- background basis (Sec. 3.1)

def node_pos_by_dof(m):
    nd = m.nodes()
    c = m.counts()
    pos = np.zeros((c["ndof"], 3))
    sel = nd["dof"] >= 0
    unit = m.cfg["L"] / (1 << m.cfg["depth_max"])
    pos[nd["dof"][sel]] = nd["coord"][sel] * unit
    return pos


def test_background_basis_partition_and_linear_completeness():
    # Eq. (hanging node solution): sum_i phi~_iK = 1 and sum_i phi~_iK x_i = x in
    # every populated leaf, hanging nodes included
    cfg = tiny_cfg()
    m = built(cfg)
    pos = node_pos_by_dof(m)
    rng = np.random.default_rng(5)
    n_ok = 0
    for _ in range(400):
        x = rng.uniform([0, 0, 0], [1, 1, 0.5])
        idx, phi, dphi = m.eval_background(x)
        if np.any(idx < 0):
            continue  # leaf without active nodes (unpopulated)
        n_ok += 1
        assert abs(phi.sum() - 1) < 1e-13
        assert np.allclose(phi @ pos[idx], x, atol=1e-13)
        assert np.allclose(dphi.sum(axis=0), 0, atol=1e-10)
        assert np.allclose(pos[idx].T @ dphi, np.eye(3), atol=1e-10)
    assert n_ok > 200


def test_background_basis_continuous_across_hanging_faces():
    # C0 continuity restored by the constraints (Sec. 3.1): values on both
    # sides of every leaf face agree
    cfg = tiny_cfg()
    m = built(cfg)
    lev, anc, s, D = leaf_boxes(m)
    unit = cfg["L"] / (1 << D)
    rng = np.random.default_rng(7)
    checked = 0
    for K in range(len(lev)):
        a = anc[K] * unit
        h = s[K] * unit
        if a[2] + h > 0.5:
            continue
        for axis in range(3):
            x = a + rng.uniform(0.1, 0.9, 3) * h
            x[axis] = a[axis] + h
            if x[axis] >= cfg["L"]:
                continue
            eps = 1e-9
            xm, xp = x.copy(), x.copy()
            xm[axis] -= eps
            xp[axis] += eps
            i1, p1, _ = m.eval_background(xm)
            i2, p2, _ = m.eval_background(xp)
            if np.any(i1 < 0) or np.any(i2 < 0):
                continue
            f1 = dict(zip(i1.tolist(), p1))
            f2 = dict(zip(i2.tolist(), p2))
            for k in set(f1) | set(f2):
                assert abs(f1.get(k, 0.0) - f2.get(k, 0.0)) < 1e-7
            checked += 1
    assert checked > 50


# ---------------------------------------------------------------- GIMP basis (Sec. 3.2)

def gimp_1d(xi, h, l):
    """Classic closed-form 1D GIMP function (hat of width h convolved with a box of
    half-length l, l <= h/2), written out from the convolution integral."""
    a = abs(xi)
    if a <= l:
        return 1.0 - (xi * xi + l * l) / (2.0 * h * l)
    if a <= h - l:
        return 1.0 - a / h
    if a <= h + l:
        return (h + l - a) ** 2 / (4.0 * h * l)
    return 0.0


def test_gimp_equals_tensor_product_closed_form_on_uniform_grid():
    cfg = inputs.workload("column", depth_min=3, depth_max=3,
                          points=dict(spacing=1.0 / 16, jitter=1.0 / 40, seed=11))
    m = built(cfg)
    pos = node_pos_by_dof(m)
    nsup, sidx, S, dS = m.support()
    P = m.points()
    h, l = 1.0 / 8, 1.0 / 32
    rng = np.random.default_rng(0)
    for p in rng.choice(len(nsup), 200, replace=False):
        lo = P["x"][p] - l
        hi = P["x"][p] + l
        if np.any(lo < 0) or np.any(hi > 1):
            continue
        for k in range(nsup[p]):
            xv = pos[sidx[p, k]]
            ex = np.prod([gimp_1d(P["x"][p][d] - xv[d], h, l) for d in range(3)])
            assert abs(S[p, k] - ex) < 1e-14


def test_gimp_partition_completeness_on_hanging_mesh():
    # PoU and linear completeness of S_vp across hanging nodes, for boxes inside Omega
    cfg = tiny_cfg(points=dict(spacing=0.25, jitter=0.03, seed=2))
    m = built(cfg)
    pos = node_pos_by_dof(m)
    nsup, sidx, S, dS = m.support()
    P = m.points()
    assert nsup.max() > 8  # jittered domains straddle hanging faces
    for p in range(len(nsup)):
        lo = P["x"][p] - P["lp"][p]
        hi = P["x"][p] + P["lp"][p]
        if np.any(lo < 0) or np.any(hi > 1):
            continue
        k = nsup[p]
        xs = pos[sidx[p, :k]]
        assert abs(S[p, :k].sum() - 1) < 1e-13
        assert np.allclose(S[p, :k] @ xs, P["x"][p], atol=1e-13)
        assert np.allclose(dS[p, :k].sum(axis=0), 0, atol=1e-9)
        assert np.allclose(xs.T @ dS[p, :k], np.eye(3), atol=1e-9)


def test_gimp_gradient_matches_finite_difference():
    # reading: grad S_vp is the derivative of S_vp with respect to the point position
    cfg = tiny_cfg(points=dict(spacing=0.25, jitter=0.03, seed=2))
    pts = inputs.make_points(cfg)
    m = built(cfg, pts, nosplit=True)
    nsup, sidx, S, dS = m.support()
    P = m.points()
    inside = np.nonzero(np.all(P["x"] - P["lp"] > 1e-3, axis=1) &
                        np.all(P["x"] + P["lp"] < [1 - 1e-3, 1 - 1e-3, 1 - 1e-3], axis=1))[0]
    rng = np.random.default_rng(1)
    h = 1e-6
    # boxes clipped by the domain are excluded: there the clipped integral's
    # derivative differs from the integral of the gradient
    for p in rng.choice(inside, 6, replace=False):
        for d in range(3):
            vals = []
            for sgn in (1, -1):
                q = {k: v.copy() for k, v in pts.items()}
                q["x"][p, d] += sgn * h
                mm = built(cfg, q, nosplit=True)
                ns2, si2, S2, _ = mm.support()
                vals.append(dict(zip(si2[p, :ns2[p]].tolist(), S2[p, :ns2[p]])))
            for k in range(nsup[p]):
                j = sidx[p, k]
                fd = (vals[0].get(j, 0.0) - vals[1].get(j, 0.0)) / (2 * h)
                assert abs(fd - dS[p, k, d]) < 1e-6 * max(1.0, abs(dS[p, k, d]))


def test_split_geometry_matches_paper_worked_example():
    # Sec. 5, 1D example: parent at 0.2 with length 0.4 -> children at 0.1 and 0.3,
    # length 0.2; data copied, volume and mass shared out.  A single GIMP of
    # half-length 0.2 over depth-1 leaves (l_K = 0.25 < beta l_p = 0.4) splits once.
    g = read_golden("split_1d.txt")
    cfg = inputs.workload("column", depth_min=1, depth_max=1, contact=0,
                          points=dict(lo=(0.4, 0.4, 0.0), hi=(0.8, 0.8, 0.4), spacing=0.4))
    pts = inputs.make_points(cfg)
    assert len(pts["x"]) == 1 and abs(pts["x"][0, 2] - g["parent_z"][0]) < 1e-15
    assert abs(2 * pts["lp"][0, 2] - g["parent_length"][0]) < 1e-15
    pts["E"][:] = 3.0e6
    m = built(cfg, pts)
    P = m.points()
    assert len(P["x"]) == 8
    assert np.allclose(sorted(np.unique(np.round(P["x"][:, 2], 12))), g["child_z"], atol=1e-14)
    assert np.allclose(2 * P["lp"][:, 2], g["child_length"][0], atol=1e-15)
    assert abs(P["mass"].sum() - pts["mass"].sum()) < 1e-15
    assert abs(P["V0"].sum() - pts["V0"].sum()) < 1e-15
    assert np.all(P["E"] == 3.0e6)


def test_split_children_tile_the_parent():
    cfg = tiny_cfg()
    pts = inputs.make_points(cfg)
    m = built(cfg, pts)
    P = m.points()
    n0 = len(pts["x"])
    assert len(P["x"]) > n0 and (len(P["x"]) - n0) % 7 == 0
    assert abs(P["mass"].sum() - pts["mass"].sum()) < 1e-12 * pts["mass"].sum()
    vol = np.prod(2 * P["lp"], axis=1).sum()
    assert abs(vol - np.prod(2 * pts["lp"], axis=1).sum()) < 1e-12


# ---------------------------------------------------------------- constitutive (Sec. 2.2)

def rot(a, b, c):
    Rx = np.array([[1, 0, 0], [0, math.cos(a), -math.sin(a)], [0, math.sin(a), math.cos(a)]])
    Ry = np.array([[math.cos(b), 0, math.sin(b)], [0, 1, 0], [-math.sin(b), 0, math.cos(b)]])
    Rz = np.array([[math.cos(c), -math.sin(c), 0], [math.sin(c), math.cos(c), 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


I6 = np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0])


def test_hencky_uniaxial_matches_contact_column_formula():
    # Sec. 6.2: with nu = 0 the vertical stress is E (l0/l) ln(l/l0)
    cfg = inputs.workload("column", nu=0.0)
    E = 1e6
    for lam in (0.75, 0.9, 1.0, 1.2):
        dF = np.diag([1.0, 1.0, lam])
        tau, be, A, pl = oracle.constitutive(cfg, E, 0.0, I6, dF)
        sig = tau / lam
        assert abs(sig[2, 2] - E * (1.0 / lam) * math.log(lam)) < 1e-9 * E
        assert abs(sig[0, 0]) < 1e-9 * E


def test_hencky_general_stretch_by_hand_and_objectivity():
    cfg = inputs.workload("column", nu=0.3)
    E, nu = 1e6, 0.3
    mu = E / (2 * (1 + nu))
    lamL = E * nu / ((1 + nu) * (1 - 2 * nu))
    st = np.array([1.1, 0.8, 1.3])
    ln = np.log(st)
    tau_h = lamL * ln.sum() + 2 * mu * ln
    R = rot(0.3, -0.7, 1.1)
    tau, be, A, pl = oracle.constitutive(cfg, E, 0.0, I6, R @ np.diag(st))
    assert np.allclose(R.T @ tau @ R, np.diag(tau_h), atol=1e-8)
    tau2, _, _, _ = oracle.constitutive(cfg, E, 0.0, I6, np.diag(st) @ R)
    assert np.allclose(tau2, np.diag(tau_h), atol=1e-8)


def test_von_mises_return_is_consistent_and_radial():
    cfg = inputs.workload("punch")
    E, ys = 1e7, 1e5
    dF = np.eye(3) + np.array([[0.02, 0.01, 0.0], [0.0, -0.01, 0.005], [0.003, 0.0, 0.01]])
    tau, be, A, pl = oracle.constitutive(cfg, E, ys, I6, dF)
    assert pl == 1
    s = tau - np.trace(tau) / 3 * np.eye(3)
    q = math.sqrt(1.5 * np.sum(s * s))
    assert abs(q - ys) < 1e-12 * ys
    el = dict(cfg, model=0)
    tt, _, _, _ = oracle.constitutive(el, E, ys, I6, dF)
    st = tt - np.trace(tt) / 3 * np.eye(3)
    assert abs(np.trace(tt) - np.trace(tau)) < 1e-7
    assert np.allclose(s / np.linalg.norm(s), st / np.linalg.norm(st), atol=1e-12)
    # elastic branch untouched
    small = np.eye(3) + 1e-5 * np.array([[1, 2, 0], [0, -1, 1], [1, 0, 1.0]])
    t1, _, _, p1 = oracle.constitutive(cfg, E, ys, I6, small)
    t2, _, _, _ = oracle.constitutive(el, E, ys, I6, small)
    assert p1 == 0 and np.allclose(t1, t2, atol=0)


def dp_consts(phi, psi):
    s, sp = math.sin(phi), math.sin(psi)
    return (6 * s / (math.sqrt(3) * (3 - s)), 6 * math.cos(phi) / (math.sqrt(3) * (3 - s)),
            6 * sp / (math.sqrt(3) * (3 - sp)))


def test_drucker_prager_cone_and_apex_returns():
    cfg = inputs.workload("cone")
    E, c, nu = 2e7, 5e3, 0.3
    G = E / (2 * (1 + nu))
    Kb = E / (3 * (1 - 2 * nu))
    eta, xi, etab = dp_consts(cfg["phi"], cfg["psi"])
    # cone return: shear under compression
    dF = np.eye(3) + np.array([[-0.002, 0.05, 0], [0.0, -0.001, 0], [0, 0, -0.001]])
    tau, be, A, pl = oracle.constitutive(cfg, E, c, I6, dF)
    assert pl == 1
    p = np.trace(tau) / 3
    s = tau - p * np.eye(3)
    sj2 = math.sqrt(0.5 * np.sum(s * s))
    assert abs(sj2 + eta * p - xi * c) < 1e-9 * c
    el = dict(cfg, model=0)
    tt, _, _, _ = oracle.constitutive(el, E, c, I6, dF)
    pt = np.trace(tt) / 3
    st = tt - pt * np.eye(3)
    sj2t = math.sqrt(0.5 * np.sum(st * st))
    # flow rule of the DP potential: dp / d sqrt(J2) = K etabar / G
    assert abs((pt - p) - Kb * etab / G * (sj2t - sj2)) < 1e-7 * c
    # apex: volumetric tension
    tau, be, A, pl = oracle.constitutive(cfg, E, c, I6, np.eye(3) * 1.01)
    assert pl == 2
    assert np.allclose(tau, xi * c / eta * np.eye(3), atol=1e-9)


@pytest.mark.parametrize("case", ["elastic", "vm", "dp", "near_repeated"])
def test_spatial_tangent_matches_finite_difference(case):
    # A_ijkm = d tau_ij / d L_km with dF -> (I + L) dF (central differences)
    rng = np.random.default_rng(4)
    if case == "elastic":
        cfg, E, ys = inputs.workload("column"), 1e6, 0.0
        dF = np.eye(3) + 0.05 * rng.normal(size=(3, 3))
    elif case == "vm":
        cfg, E, ys = inputs.workload("punch"), 1e7, 1e5
        dF = np.eye(3) + 0.02 * rng.normal(size=(3, 3))
    elif case == "dp":
        cfg, E, ys = inputs.workload("cone", psi=math.radians(5.0)), 2e7, 5e3
        dF = np.eye(3) + np.array([[-0.002, 0.05, 0], [0.0, -0.001, 0.001], [0, 0, -0.001]])
    else:
        cfg, E, ys = inputs.workload("column"), 1e6, 0.0
        dF = np.diag([1.01, 1.01 + 1e-9, 0.98])
    be = np.array([1.02, 0.99, 1.01, 0.01, -0.005, 0.002])
    tau, _, A, pl = oracle.constitutive(cfg, E, ys, be, dF)
    if case in ("vm", "dp"):
        assert pl == 1
    h = 1e-7
    for k in range(3):
        for mm in range(3):
            Lp = np.zeros((3, 3))
            Lp[k, mm] = h
            tp, _, _, _ = oracle.constitutive(cfg, E, ys, be, (np.eye(3) + Lp) @ dF, tangent=False)
            tm, _, _, _ = oracle.constitutive(cfg, E, ys, be, (np.eye(3) - Lp) @ dF, tangent=False)
            fd = (tp - tm) / (2 * h)
            assert np.allclose(A[:, :, k, mm], fd, atol=2e-6 * E, rtol=0), (k, mm)


# ---------------------------------------------------------------- assembly, ghost, contact

def test_global_tangent_matches_finite_difference_of_residual():
    # plasticity, hanging nodes, ghost faces and contact all active
    cfg = tiny_cfg(points=dict(spacing=0.25, jitter=0.02, seed=9))
    cfg["body"]["z0"] = 0.49
    m = built(cfg, body_z=0.49)
    c = m.counts()
    assert c["nhang"] > 0 and c["nghost"] > 0
    n3 = 3 * c["ndof"]
    rng = np.random.default_rng(2)
    du = 1e-3 * rng.normal(size=n3)
    out = m.assemble(du)
    assert np.linalg.norm(out["reaction"]) > 0  # contact active
    rp, col = m.pattern()
    K = out["K"]
    h = 1e-7
    for _ in range(3):
        v = rng.normal(size=n3)
        Rp = m.assemble(du + h * v, tangent=False)["R"]
        Rm = m.assemble(du - h * v, tangent=False)["R"]
        fd = (Rp - Rm) / (2 * h)
        Kv = np.zeros(n3)
        for i in range(c["ndof"]):
            for s in range(rp[i], rp[i + 1]):
                Kv[3 * i:3 * i + 3] += K[s] @ v[3 * col[s]:3 * col[s] + 3]
        assert np.linalg.norm(Kv - fd) <= 1e-6 * np.linalg.norm(fd)


def test_ghost_matrix_null_on_linear_fields_symmetric_psd():
    # jumps of normal derivatives vanish for globally linear fields (Sec. 4)
    cfg = tiny_cfg()
    m = built(cfg)
    c = m.counts()
    assert c["nghost"] > 0
    kg = m.ghost()
    rp, col = m.pattern()
    n = c["ndof"]
    G = np.zeros((n, n))
    for i in range(n):
        G[i, col[rp[i]:rp[i + 1]]] = kg[rp[i]:rp[i + 1]]
    assert np.abs(G).max() > 0
    assert np.allclose(G, G.T, atol=1e-9 * np.abs(G).max())
    assert np.linalg.eigvalsh(G).min() > -1e-8 * np.abs(G).max()
    pos = node_pos_by_dof(m)
    for f in (pos[:, 0], pos[:, 1], pos[:, 2], np.ones(n)):
        assert np.abs(G @ f).max() < 1e-9 * np.abs(G).max()


def test_ghost_face_set_brute_force():
    # Sec. 4: T^B = populated leaves sharing a face with an unpopulated leaf;
    # F_B = faces K+ cap K- with K+ in T^B and K- populated.  Populated is
    # recomputed here from the point boxes (positive-volume overlap).
    cfg = tiny_cfg(points=dict(spacing=0.25, jitter=0.03, seed=4))
    m = built(cfg, body_z=0.49)
    lev, anc, s, D = leaf_boxes(m)
    faces, pop = m.ghost_faces()
    unit = cfg["L"] / (1 << D)
    P = m.points()
    lo_b = np.clip(np.round((P["x"] - P["lp"]) / unit, 9), 0, 1 << D)
    hi_b = np.clip(np.round((P["x"] + P["lp"]) / unit, 9), 0, 1 << D)
    lo, hi = anc, anc + s[:, None]
    popb = np.zeros(len(lev), bool)
    for K in range(len(lev)):
        ext = np.minimum(hi_b, hi[K]) - np.maximum(lo_b, lo[K])
        popb[K] = np.any(np.all(ext > 1e-9, axis=1))
    assert np.array_equal(popb, pop.astype(bool))
    # face adjacency with positive area
    nl = len(lev)
    adj = []
    for i in range(nl):
        ext = np.minimum(hi[i], hi) - np.maximum(lo[i], lo)
        face = np.all(ext >= 0, axis=1) & (np.sum(ext > 0, axis=1) == 2)
        face[i] = False
        adj.append(np.nonzero(face)[0])
    isB = np.array([popb[i] and any(not popb[j] for j in adj[i]) for i in range(nl)])
    expect = set()
    for i in range(nl):
        for j in adj[i]:
            if popb[i] and popb[j] and (isB[i] or isB[j]):
                expect.add((min(i, j), max(i, j)))
    got = set((min(a, b), max(a, b)) for a, b, _, _ in faces)
    assert len(got) == len(faces)
    assert got == expect
    assert len(got) > 0


def test_ghost_value_on_two_equal_cells_by_hand():
    # Two equal cells sharing the face x = h; only the left one is populated
    # besides the right one being a boundary element.  For the node pair at the
    # far corners the jump product integrates by hand over the face.
    cfg = inputs.workload("column", depth_min=1, depth_max=1, contact=0, bc=[],
                          points=dict(lo=(0, 0, 0), hi=(1.0, 0.5, 0.5), spacing=0.25))
    m = built(cfg)
    c = m.counts()
    assert c["nghost"] == 1
    kg = m.ghost()
    rp, col = m.pattern()
    pos = node_pos_by_dof(m)
    h = 0.5
    E = cfg["points"]["E"]
    # node a at (0,0,0) (left cell only), node b at (1,0,0) (right cell only):
    # [d_n phi_a] = -(-1/h)(1-y/h)(1-z/h) ... integral of the product over the face
    # = (1/h^2) * (h/3)^2 ... written out: int_0^h int_0^h ((1-y/h)(1-z/h))^2 dy dz / h^2
    ia = int(np.nonzero(np.all(np.isclose(pos, [0, 0, 0]), axis=1))[0][0])
    ib = int(np.nonzero(np.all(np.isclose(pos, [1, 0, 0]), axis=1))[0][0])
    s = rp[ia] + int(np.nonzero(col[rp[ia]:rp[ia + 1]] == ib)[0][0])
    integral = (h / 3.0) ** 2 / h ** 2
    # jump for a: left derivative -1/h*(...), right 0; for b: left 0, right +1/h*(...)
    # product of jumps: (-1/h)(0 - 1/h)*... with n = +x: J_a = -(1/h) f, J_b = -(1/h) f
    expect = h * E / 10.0 * integral
    assert abs(kg[s] - expect) < 1e-12 * expect


def test_patch_test_uniform_stress_under_affine_stretch():
    # affine diagonal stretch on a hanging-node mesh with tiling domains:
    # uniform stress and zero residual at interior nodes
    cfg = tiny_cfg(contact=0, ghost=0, model=0, depth_min=3, depth_max=4, dx_region=0.07,
                   points=dict(spacing=1.0 / 16))
    cfg["body"].update(cx=0.45, cy=0.55, r=0.06)
    m = built(cfg, body_z=cfg["body"]["z0"])
    c = m.counts()
    assert c["nhang"] > 0
    pos = node_pos_by_dof(m)
    G = np.diag([0.01, -0.02, 0.015])
    du = (pos @ G.T).ravel()
    out = m.assemble(du, tangent=False)
    sig = m.point_stress(du)
    assert np.allclose(sig, sig[0], atol=1e-9 * np.abs(sig[0]).max())
    # nodes whose support stays inside the block (away from all faces)
    nsup, sidx, S, dS = m.support()
    P = m.points()
    touch = np.zeros(c["ndof"], bool)
    for p in range(len(nsup)):
        lo = P["x"][p] - P["lp"][p]
        hi = P["x"][p] + P["lp"][p]
        if np.any(lo <= 1e-12) or np.any(hi >= [1, 1, 0.5 - 1e-12]):
            touch[sidx[p, :nsup[p]]] = True
    interior = ~touch
    assert interior.sum() > 3
    R = out["R"].reshape(-1, 3)
    assert np.abs(R[interior]).max() < 1e-12 * np.abs(out["fint"]).max()


def test_contact_penalty_constant_and_reaction_balance():
    g = read_golden("paper_constants.txt")
    assert g["contact_normal_factor"][0] == 50.0
    cfg = tiny_cfg(ghost=0, model=0)
    assert cfg["pf"] == g["contact_normal_factor"][0]
    m = built(cfg, body_z=0.49)
    n3 = 3 * m.counts()["ndof"]
    out = m.assemble(np.zeros(n3))
    # at du = 0 only contact loads the mesh: sum of nodal forces = -reaction
    R = out["R"].reshape(-1, 3)
    assert np.allclose(R.sum(axis=0), out["reaction"], rtol=1e-12, atol=1e-9)
    # penetration 0.01 m under the flat face, eps_N = 50 E (V0)^(2/3) per corner
    P = m.points()
    expect = 0.0
    for p in range(len(P["x"])):
        top = P["x"][p, 2] + P["lp"][p, 2]
        r = np.hypot(P["x"][p, 0] + np.array([-1, 1, -1, 1]) * P["lp"][p, 0] - 0.3,
                     P["x"][p, 1] + np.array([-1, -1, 1, 1]) * P["lp"][p, 1] - 0.4)
        pen = top - 0.49
        if pen > 0:
            expect += np.sum(r < 0.1) * 50 * P["E"][p] * P["V0"][p] ** (2 / 3) * pen
    assert abs(out["reaction"][2] - expect) < 1e-9 * expect


# ---------------------------------------------------------------- solves and Newton

def test_krylov_and_lu_agree_with_residual():
    cfg = tiny_cfg()
    m = built(cfg, body_z=0.49)
    n3 = 3 * m.counts()["ndof"]
    out = m.assemble(np.zeros(n3))
    x, its = m.solve(out["K"], -out["R"])
    mask = m.bcmask()
    rp, col = m.pattern()
    Kx = np.zeros(n3)
    for i in range(m.counts()["ndof"]):
        for s in range(rp[i], rp[i + 1]):
            Kx[3 * i:3 * i + 3] += out["K"][s] @ x[3 * col[s]:3 * col[s] + 3]
    free = np.array([not (mask[i // 3] >> (i % 3)) & 1 for i in range(n3)])
    assert np.linalg.norm((Kx + out["R"])[free]) < 1e-10 * np.linalg.norm(out["R"][free])
    assert np.all(x[~free] == 0)


@pytest.mark.slow
def test_column_self_weight_closed_form_and_convergence():
    # closed form (equilibrium at finite strain with rollers): sigma_zz(Z) = -rho0 g (H - Z),
    # sigma_xx/sigma_zz = nu/(1-nu); stretch lambda = exp(-W0(s)), s = rho0 g (H - Z)/M;
    # the volume-weighted error falls at first order or better (Sec. 6.1)
    from scipy.special import lambertw
    errs = []
    for depth in (2, 3):
        cfg = inputs.workload("column", depth_min=depth, depth_max=depth,
                              points=dict(spacing=0.5 ** (depth + 1)))
        pts = inputs.make_points(cfg)
        Z0 = pts["x"][:, 2].copy()
        m = oracle.Model(cfg, pts)
        for n in range(1, cfg["nsteps"] + 1):
            st = m.step(load=inputs.load_factor(cfg, n), tol=1e-11, lin_tol=1e-12)
            assert st["status"] == 0
        m.build(nosplit=True)
        sig = m.point_stress(np.zeros(3 * m.counts()["ndof"]))
        P = m.points()
        rho, g, H, E, nu = 1000.0, 9.81, 1.0, 1e6, 0.3
        V = P["V0"] * np.linalg.det(P["F"].reshape(-1, 3, 3))
        ex = -rho * g * (H - Z0)
        errs.append(np.sum(np.abs(ex - sig[:, 2, 2]) * V) / (rho * g * H * V.sum()))
        assert np.allclose(sig[:, 0, 0], nu / (1 - nu) * sig[:, 2, 2], rtol=1e-9, atol=1e-6)
        # displacement of the points vs integral of (lambda - 1)
        M = E * (1 - nu) / ((1 + nu) * (1 - 2 * nu))
        zz = np.linspace(0, 1, 2001)
        lam = np.exp(-np.real(lambertw(rho * g * (H - zz) / M)))
        uz = np.concatenate([[0], np.cumsum(0.5 * (lam[1:] + lam[:-1] - 2) * np.diff(zz))])
        u_ex = np.interp(Z0, zz, uz)
        u_num = P["x"][:, 2] - Z0
        assert np.max(np.abs(u_num - u_ex)) < 0.05 * np.max(np.abs(u_ex))
        # domain update l = l0 diag(U) (uniaxial: U = diag(1, 1, F_zz)); V = det(F) V0
        F = P["F"].reshape(-1, 3, 3)
        assert np.allclose(P["lp"][:, 2], P["l0"][:, 2] * F[:, 2, 2], rtol=1e-12)
        assert np.allclose(P["lp"][:, :2], P["l0"][:, :2], rtol=1e-12)
    assert errs[1] < 0.04
    assert errs[0] / errs[1] > 1.8


def test_newton_converges_quadratically():
    cfg = tiny_cfg()
    pts = inputs.make_points(cfg)
    m = oracle.Model(cfg, pts)
    m.set_body_z(0.48)
    st = m.step(load=1.0, tol=1e-12, lin_tol=1e-14)
    assert st["status"] == 0
    r = st["res_hist"]
    assert len(r) >= 3
    # the last steps: r_{k+1} <= C r_k^2 with a modest C
    ks = [k for k in range(len(r) - 1) if 1e-11 < r[k] < 1e-2]
    assert ks
    for k in ks:
        assert r[k + 1] <= 1e3 * r[k] ** 2 + 1e-12


@pytest.mark.slow
def test_contact_column_stress_within_one_percent_at_high_penalty():
    # Sec. 6.2: uniform compression by a rigid plate; with nu = 0 the vertical
    # stress is E (l0/l) ln(l/l0); below 1 % error needs p_f > 1000 (paper)
    g = read_golden("paper_constants.txt")
    pf = 4.0 * g["contact_column_pf_for_1pct"][0]
    cfg = inputs.workload("column", depth_min=2, depth_max=2, nu=0.0, g=(0, 0, 0), contact=1,
                          pf=pf, ramp_load=False,
                          points=dict(hi=(1.0, 1.0, 0.75), spacing=0.125))
    cfg["bc"] = [(0, 0.0, 1), (0, 1.0, 1), (1, 0.0, 2), (1, 1.0, 2), (2, 0.0, 7)]
    cfg["body"] = dict(kind=1, cx=0.5, cy=0.5, z0=0.75, r=10.0, alpha=0.0, dz=-0.05 / 4)
    pts = inputs.make_points(cfg)
    m = oracle.Model(cfg, pts)
    for n in range(1, 5):
        m.set_body_z(inputs.body_z(cfg, n))
        # the stiff penalty puts the round-off floor of the residual near 1e-11
        st = m.step(load=1.0, tol=1e-9, lin_tol=1e-13)
        assert st["status"] == 0
    m.build(nosplit=True)
    P = m.points()
    sig = m.point_stress(np.zeros(3 * m.counts()["ndof"]))
    l0, l = 0.75, inputs.body_z(cfg, 4)
    ex = 1e6 * (l0 / l) * math.log(l / l0)
    rel = np.abs(sig[:, 2, 2] - ex) / abs(ex)
    assert rel.max() < 0.01
    # uniform through the body
    assert np.std(sig[:, 2, 2]) < 0.01 * abs(ex)


# ---------------------------------------------------------------- rigid body geometry (Sec. 2.3, Sec. 5)
#
# The rigid bodies are analytic solids: the flat-ended punch {z >= z0, rho <= r}
# and the cone of half angle alpha with its tip at z0 and a shaft of radius r
# above the rim (rho <= min((z - z0) tan alpha, r)), rho the distance to the
# axis.  The pins below sample the solid's boundary densely and take distances
# by brute force over the samples, so they share nothing with the oracle's
# closed-form distance, normal and curvature.

def surface_samples(cfg, z0, h, ztop):
    """Points on the boundary of the solid, no surface point farther than h
    from a sample (rings of arc step <= h at height / radius steps <= h)."""
    b = cfg["body"]
    cx, cy, r = b["cx"], b["cy"], b["r"]
    pts = []

    def ring(rho, z):
        if rho <= 0:
            pts.append(np.array([[cx, cy, z]]))
            return
        n = max(8, int(math.ceil(2 * math.pi * rho / h)))
        t = np.arange(n) * (2 * math.pi / n)
        pts.append(np.stack([cx + rho * np.cos(t), cy + rho * np.sin(t), np.full(n, z)], 1))

    if b["kind"] == 1:
        for rho in np.linspace(0, r, int(math.ceil(r / h)) + 1):
            ring(rho, z0)  # bottom disk
        zw = z0
    else:
        ta = math.tan(b["alpha"])
        hc = r / ta
        # lateral cone: slant step <= h
        ns = int(math.ceil(hc / math.cos(b["alpha"]) / h)) + 1
        for z in np.linspace(z0, z0 + hc, ns):
            ring((z - z0) * ta, z)
        zw = z0 + hc
    for z in np.linspace(zw, ztop, int(math.ceil((ztop - zw) / h)) + 1):
        ring(r, z)  # lateral wall / shaft
    return np.concatenate(pts)


def brute_dist(x, S, chunk=256):
    """Distance from each point of x to the nearest sample of S."""
    out = np.empty(len(x))
    for i in range(0, len(x), chunk):
        d = np.linalg.norm(x[i:i + chunk, None, :] - S[None, :, :], axis=2)
        out[i:i + chunk] = d.min(1)
    return out


def in_solid(cfg, x, z0):
    b = cfg["body"]
    rho = np.hypot(x[:, 0] - b["cx"], x[:, 1] - b["cy"])
    if b["kind"] == 1:
        return (x[:, 2] >= z0) & (rho <= b["r"])
    return (x[:, 2] >= z0) & (rho <= np.minimum((x[:, 2] - z0) * math.tan(b["alpha"]), b["r"]))


def cone_cfg(**over):
    """A cone large against the cells (1/16), so that its tip, flank, rim and
    shaft all meet the refinement."""
    c = inputs.workload("punch", depth_min=1, depth_max=4, dx_region=0.1,
                        points=dict(spacing=0.125, jitter=0.01, seed=3))
    c["body"] = dict(kind=2, cx=0.47, cy=0.52, z0=0.46, r=0.15, alpha=math.radians(35.0),
                     dz=-0.002)
    c.update(over)
    return c


@pytest.mark.parametrize("kind", ["punch", "cone"])
def test_refinement_steps_1_and_2_brute_force(kind):
    # Sec. 5: a leaf is refined while it meets the solid (Step 1) or one of its
    # vertices lies within dx_region of it (Step 2), down to depth_max.  So
    # (a) no leaf coarser than depth_max has a vertex within dx_region of the
    # solid or a piece of the solid's boundary inside it, and (b) the parent of
    # every depth_max leaf met one of the two criteria (the 2:1 balance never
    # makes depth_max leaves).  Catches a wrong distance (e.g. the punch rim,
    # the cone flank against its shaft) or a wrong box test.
    cfg = tiny_cfg() if kind == "punch" else cone_cfg()
    z0 = cfg["body"]["z0"]
    m = built(cfg, body_z=z0)
    lev, anc, s, D = leaf_boxes(m)
    unit = cfg["L"] / (1 << D)
    h = 0.1 * unit
    S = surface_samples(cfg, z0, h, cfg["L"] + 2 * cfg["dx_region"])
    corners = np.array([[i & 1, (i >> 1) & 1, (i >> 2) & 1] for i in range(8)])
    dxr = cfg["dx_region"]
    coarse = np.nonzero(lev < D)[0]
    fine = np.nonzero(lev == D)[0]
    assert len(coarse) and len(fine)
    # (a)
    V = ((anc[coarse, None, :] + corners[None] * s[coarse, None, None]) * unit).reshape(-1, 3)
    dv = brute_dist(V, S).reshape(-1, 8)
    assert np.all(dv > dxr), "a coarse leaf has a vertex within dx_region"
    assert not np.any(in_solid(cfg, V, z0))
    lo, hi = anc[coarse] * unit, (anc[coarse] + s[coarse, None]) * unit
    for k in range(len(coarse)):
        inside = np.all((S > lo[k]) & (S < hi[k]), axis=1)
        assert not inside.any(), "the solid's boundary crosses a coarse leaf"
    # (b)
    ps = 2 * s[fine]
    pa = (anc[fine] // ps[:, None]) * ps[:, None]
    PV = ((pa[:, None, :] + corners[None] * ps[:, None, None]) * unit).reshape(-1, 3)
    dp = brute_dist(PV, S).reshape(-1, 8).min(1)
    plo, phi_ = pa * unit - h, (pa + ps[:, None]) * unit + h
    for k in range(len(fine)):
        if dp[k] <= dxr + h:
            continue
        assert np.any(np.all((S >= plo[k]) & (S <= phi_[k]), axis=1)), k


def sdf_cases(cfg, z0, rng, n):
    """Seeded points in a box around the body's lower part."""
    b = cfg["body"]
    span = 2.5 * b["r"]
    x = np.stack([b["cx"] + rng.uniform(-span, span, n), b["cy"] + rng.uniform(-span, span, n),
                  z0 + rng.uniform(-0.5 * span, 2.0 * span, n)], 1)
    return x


@pytest.mark.parametrize("kind", ["punch", "cone"])
def test_body_signed_distance_brute_force(kind):
    # |phi| is the distance to the solid's boundary, negative inside (Sec. 2.3
    # gap function); the brute-force distance over the samples exceeds the
    # true one by at most the sampling step h
    cfg = tiny_cfg() if kind == "punch" else cone_cfg()
    z0 = cfg["body"]["z0"]
    rng = np.random.default_rng(11)
    x = sdf_cases(cfg, z0, rng, 800)
    h = 2e-3
    S = surface_samples(cfg, z0, h, z0 + 1.0)
    phi, n, H, ins = oracle.body_sdf(cfg, x, body_z=z0)
    sol = in_solid(cfg, x, z0)
    # strictly inside / outside points only (the boundary itself is measure zero)
    assert np.array_equal(ins, sol)
    assert sol.sum() > 40 and (~sol).sum() > 40
    d = brute_dist(x, S)
    assert np.all(np.abs(phi) <= d + 1e-12)
    assert np.all(np.abs(phi) >= d - h)
    assert np.all(phi[sol] <= 0) and np.all(phi[~sol] >= 0)


def smooth_inside_points(cfg, z0, rng, n):
    """Points inside the solid whose nearest boundary point is unique and on a
    smooth piece (flank or shaft of the cone, wall or bottom of the punch),
    away from the axis, the rim, the tip and the medial surfaces."""
    b = cfg["body"]
    r = b["r"]
    out = []
    while len(out) < n:
        th = rng.uniform(0, 2 * math.pi)
        if b["kind"] == 2:
            ta = math.tan(b["alpha"])
            hc = r / ta
            if rng.uniform() < 0.6:  # near the flank, below the rim
                z = z0 + rng.uniform(0.35, 0.8) * hc
                rho = (z - z0) * ta - rng.uniform(0.02, 0.15) * (z - z0) * ta
            else:  # near the shaft, above the rim
                z = z0 + hc + rng.uniform(0.3, 1.0) * r
                rho = r * rng.uniform(0.7, 0.95)
        else:
            if rng.uniform() < 0.5:  # near the bottom
                z = z0 + rng.uniform(0.05, 0.3) * r
                rho = r * rng.uniform(0.2, 0.6)
            else:  # near the wall
                z = z0 + rng.uniform(0.7, 2.0) * r
                rho = r * rng.uniform(0.75, 0.95)
        out.append([b["cx"] + rho * math.cos(th), b["cy"] + rho * math.sin(th), z])
    return np.array(out)


@pytest.mark.parametrize("kind", ["punch", "cone"])
def test_body_normal_and_hessian_match_finite_differences(kind):
    # n = grad phi and H = grad n (the contact stiffness eps_N (n n^T + phi H)
    # of Sec. 2.3 needs both); central differences of the oracle's own phi and
    # n at points with a unique, smooth nearest boundary point.  Catches a sign
    # error in the normal or a wrong curvature factor (cos alpha on the flank).
    cfg = tiny_cfg() if kind == "punch" else cone_cfg()
    z0 = cfg["body"]["z0"]
    rng = np.random.default_rng(5)
    x = smooth_inside_points(cfg, z0, rng, 60)
    phi, n, H, ins = oracle.body_sdf(cfg, x, body_z=z0)
    assert ins.all() and np.all(phi < 0)
    e = 1e-6
    for d in range(3):
        dx = np.zeros(3)
        dx[d] = e
        pp, npl, _, _ = oracle.body_sdf(cfg, x + dx, body_z=z0)
        pm, nmi, _, _ = oracle.body_sdf(cfg, x - dx, body_z=z0)
        assert np.allclose((pp - pm) / (2 * e), n[:, d], atol=1e-7)
        assert np.allclose((npl - nmi) / (2 * e), H[:, :, d], atol=1e-5 * np.abs(H).max())
    assert np.allclose(np.linalg.norm(n, axis=1), 1.0)
    assert np.abs(H).max() > 0


def test_global_tangent_matches_finite_difference_with_cone_contact():
    # the FD pin of the global tangent with the cone in contact: corners on
    # the flank and near the tip, so that eps_N (n n^T + phi H) enters
    cfg = cone_cfg()
    cfg["model"] = 0
    z0 = cfg["body"]["z0"]
    m = built(cfg, body_z=z0 - 0.06)
    c = m.counts()
    n3 = 3 * c["ndof"]
    rng = np.random.default_rng(7)
    du = 1e-3 * rng.normal(size=n3)
    out = m.assemble(du)
    assert np.linalg.norm(out["reaction"]) > 0  # contact active
    rp, col = m.pattern()
    K = out["K"]
    h = 1e-7
    for _ in range(3):
        v = rng.normal(size=n3)
        Rp = m.assemble(du + h * v, tangent=False)["R"]
        Rm = m.assemble(du - h * v, tangent=False)["R"]
        fd = (Rp - Rm) / (2 * h)
        Kv = np.zeros(n3)
        for i in range(c["ndof"]):
            for s_ in range(rp[i], rp[i + 1]):
                Kv[3 * i:3 * i + 3] += K[s_] @ v[3 * col[s_]:3 * col[s_] + 3]
        assert np.linalg.norm(Kv - fd) <= 1e-6 * np.linalg.norm(fd)


# ---------------------------------------------------------------- Coulomb friction (Sec. 2.3)
#
# Reading: the slip of a contact node is its displacement relative to the body
# over the load step, projected on the tangent plane; eps_T = 25 E_p A_p^0
# (Sec. 2.3), stick while the tangential penalty force stays within mu f_N.

def friction_cfg(mu, d):
    cfg = tiny_cfg(ghost=0, model=0, mu=mu)
    cfg["body"]["step_d"] = (d, 0.0, 0.0)
    return cfg


@pytest.mark.parametrize("regime", ["stick", "slip"])
def test_friction_stick_and_slip_by_hand(regime):
    # at du = 0 every corner under the punch face has penetration pen = 0.01 m
    # and slips by -d relative to the body moving by (d, 0, 0): stick gives
    # f_x = eps_T d, slip gives f_x = mu eps_N pen; stick iff 25 d <= 50 mu pen
    g = read_golden("paper_constants.txt")
    mu, pen = 0.3, 0.01
    d = (0.5 if regime == "stick" else 4.0) * 2 * mu * pen * g["contact_normal_factor"][0] / (
        2 * g["contact_tangential_factor"][0])
    cfg = friction_cfg(mu, d)
    assert cfg["pt"] == g["contact_tangential_factor"][0]
    m = built(cfg, body_z=0.49)
    out = m.assemble(np.zeros(3 * m.counts()["ndof"]))
    P = m.points()
    ex, ez = 0.0, 0.0
    for p in range(len(P["x"])):
        top = P["x"][p, 2] + P["lp"][p, 2]
        r = np.hypot(P["x"][p, 0] + np.array([-1, 1, -1, 1]) * P["lp"][p, 0] - 0.3,
                     P["x"][p, 1] + np.array([-1, -1, 1, 1]) * P["lp"][p, 1] - 0.4)
        if top - 0.49 <= 0:
            continue
        assert np.all((r > 0.1) | (0.1 - r > pen))  # every touching corner is under the face
        A = P["V0"][p] ** (2 / 3)
        k = np.sum(r < 0.1)
        fN = 50 * P["E"][p] * A * pen
        ft = 25 * P["E"][p] * A * d if regime == "stick" else mu * fN
        ez += k * fN
        ex += k * ft
    assert ex > 0
    # reaction = force on the body = -(force on the material)
    assert abs(out["reaction"][2] - ez) < 1e-9 * ez
    assert abs(out["reaction"][0] + ex) < 1e-9 * ex
    assert abs(out["reaction"][1]) < 1e-9 * ex


def test_friction_free_limit_is_frictionless():
    a = built(tiny_cfg(ghost=0, model=0), body_z=0.49)
    b = built(friction_cfg(0.0, 0.02), body_z=0.49)
    du = 1e-3 * np.random.default_rng(4).normal(size=3 * a.counts()["ndof"])
    oa, ob = a.assemble(du), b.assemble(du)
    assert np.array_equal(oa["R"], ob["R"]) and np.array_equal(oa["K"], ob["K"])


@pytest.mark.parametrize("mu", [0.05, 5.0])
def test_frictional_tangent_matches_finite_difference(mu):
    # mu = 0.05: most touching corners slip; mu = 5: all stick.  The body moves
    # sideways over the step so the tangential forces are not zero.
    cfg = friction_cfg(mu, 0.004)
    cfg["points"].update(jitter=0.02, seed=9)
    m = built(cfg, body_z=0.49)
    c = m.counts()
    n3 = 3 * c["ndof"]
    rng = np.random.default_rng(12)
    du = 1e-3 * rng.normal(size=n3)
    out = m.assemble(du)
    rp, col = m.pattern()
    K = out["K"]
    h = 1e-7
    for _ in range(3):
        v = rng.normal(size=n3)
        Rp = m.assemble(du + h * v, tangent=False)["R"]
        Rm = m.assemble(du - h * v, tangent=False)["R"]
        fd = (Rp - Rm) / (2 * h)
        Kv = np.zeros(n3)
        for i in range(c["ndof"]):
            for s_ in range(rp[i], rp[i + 1]):
                Kv[3 * i:3 * i + 3] += K[s_] @ v[3 * col[s_]:3 * col[s_] + 3]
        assert np.linalg.norm(Kv - fd) <= 1e-6 * np.linalg.norm(fd)
    if mu < 1:
        # slipping friction: the contact stiffness is not symmetric
        n = c["ndof"]
        G = np.zeros((n3, n3))
        for i in range(n):
            for s_ in range(rp[i], rp[i + 1]):
                G[3 * i:3 * i + 3, 3 * col[s_]:3 * col[s_] + 3] = K[s_]
        assert np.abs(G - G.T).max() > 1e-6 * np.abs(G).max()


# ---------------------------------------------------------------- triangulated bodies (Sec. 2.3)
#
# Sec. 2.3 represents the rigid bodies by closed triangular faceted meshes.
# The signed distance of such a body is checked against the distance to a
# dense sampling of its triangles and, for the sign, against the analytic
# solid it approximates (away from the band where the two differ).

def mesh_samples(v, t, h):
    """Points on every triangle, no surface point farther than about h."""
    out = []
    for a, b, c in t:
        A, B, C = v[a], v[b], v[c]
        L = max(np.linalg.norm(B - A), np.linalg.norm(C - A), np.linalg.norm(C - B))
        k = max(1, int(math.ceil(L / h)))
        i, j = np.meshgrid(np.arange(k + 1), np.arange(k + 1), indexing="ij")
        sel = (i + j) <= k
        u, w = i[sel] / k, j[sel] / k
        out.append(A[None] + u[:, None] * (B - A)[None] + w[:, None] * (C - A)[None])
    return np.concatenate(out)


def sphere_body_cfg(radius=0.3, nlat=12, nlon=16, center=(0.5, 0.5, 0.7)):
    cfg = tiny_cfg()
    cfg["body"] = dict(kind=3, cx=center[0], cy=center[1], z0=center[2], r=radius, alpha=0.0,
                       dz=-0.002, mesh=inputs.sphere_mesh(radius, nlat, nlon))
    return cfg


def test_triangulated_body_signed_distance_brute_force():
    cfg = sphere_body_cfg()
    b = cfg["body"]
    c = np.array([b["cx"], b["cy"], b["z0"]])
    v = b["mesh"]["v"] + c[None]
    h = 4e-3
    S = mesh_samples(v, b["mesh"]["t"], h)
    rng = np.random.default_rng(21)
    x = c[None] + rng.uniform(-0.45, 0.45, size=(300, 3))
    phi, n, H, ins = oracle.body_sdf(cfg, x)
    d = brute_dist(x, S)
    assert np.all(np.abs(phi) <= d + 1e-12) and np.all(np.abs(phi) >= d - h)
    # sign against the sphere, outside the band between the sphere and its
    # inscribed polyhedron (chord sagitta of the coarsest triangles)
    r = np.linalg.norm(x - c[None], axis=1)
    band = b["r"] * (1 - math.cos(math.pi / 12))
    far = np.abs(r - b["r"]) > band
    assert far.sum() > 200
    assert np.array_equal(ins[far], (r < b["r"])[far])
    assert np.all(phi[ins] < 0) and np.all(phi[~ins] >= 0)
    # inside, the normal is the nearest face's outward normal: the gradient of phi
    e = 1e-6
    xi = x[ins & far]
    for dd in range(3):
        dx = np.zeros(3)
        dx[dd] = e
        pp = oracle.body_sdf(cfg, xi + dx)[0]
        pm = oracle.body_sdf(cfg, xi - dx)[0]
        ok = np.abs((pp - pm) / (2 * e) - n[ins & far][:, dd]) < 1e-6
        assert ok.mean() > 0.95  # the few misses sit on bisectors between faces


def test_triangulated_punch_matches_analytic_punch_under_the_face():
    # a 64-sided prism for the flat punch: corners under its bottom face see
    # the same gap and normal as under the analytic cylinder's face, so the
    # contact force (with friction) on the body is the same at du = 0 (the
    # octrees differ, Step 1 being conservative for meshes: no GIMP split, and
    # only the reaction, which does not depend on the background basis at
    # du = 0, is compared)
    mu = 0.3
    a_cfg = friction_cfg(mu, 0.004)
    t_cfg = friction_cfg(mu, 0.004)
    for c in (a_cfg, t_cfg):
        c["points"]["spacing"] = 0.125
    t_cfg["body"] = dict(a_cfg["body"], kind=3, mesh=inputs.cylinder_mesh(0.1, 0.6, 64))
    ma = built(a_cfg, body_z=0.49, nosplit=True)
    mt = built(t_cfg, body_z=0.49, nosplit=True)
    P = ma.points()
    inner = 0.1 * math.cos(math.pi / 64)
    for p in range(len(P["x"])):
        if P["x"][p, 2] + P["lp"][p, 2] <= 0.49:
            continue
        r = np.hypot(P["x"][p, 0] + np.array([-1, 1, -1, 1]) * P["lp"][p, 0] - 0.3,
                     P["x"][p, 1] + np.array([-1, -1, 1, 1]) * P["lp"][p, 1] - 0.4)
        assert not np.any((r > inner - 0.011) & (r <= 0.1))
    oa = ma.assemble(np.zeros(3 * ma.counts()["ndof"]))
    ot = mt.assemble(np.zeros(3 * mt.counts()["ndof"]))
    assert np.abs(oa["reaction"]).max() > 0 and abs(oa["reaction"][0]) > 0
    assert np.allclose(oa["reaction"], ot["reaction"], rtol=1e-12, atol=0)


def test_global_tangent_matches_finite_difference_with_triangulated_body():
    # a faceted sphere pressed into the block with friction: facets, edges and
    # the sphere's curvature through the facet changes
    cfg = sphere_body_cfg(radius=0.25, nlat=10, nlon=12, center=(0.31, 0.42, 0.73))
    cfg.update(mu=0.2, ghost=0, model=0)
    cfg["body"]["step_d"] = (0.003, 0.0, -0.002)
    m = built(cfg)
    c = m.counts()
    n3 = 3 * c["ndof"]
    rng = np.random.default_rng(13)
    du = 1e-3 * rng.normal(size=n3)
    out = m.assemble(du)
    assert np.linalg.norm(out["reaction"]) > 0
    rp, col = m.pattern()
    K = out["K"]
    h = 1e-7
    for _ in range(3):
        v = rng.normal(size=n3)
        fd = (m.assemble(du + h * v, tangent=False)["R"] -
              m.assemble(du - h * v, tangent=False)["R"]) / (2 * h)
        Kv = np.zeros(n3)
        for i in range(c["ndof"]):
            for s_ in range(rp[i], rp[i + 1]):
                Kv[3 * i:3 * i + 3] += K[s_] @ v[3 * col[s_]:3 * col[s_] + 3]
        assert np.linalg.norm(Kv - fd) <= 1e-6 * np.linalg.norm(fd)


# ---------------------------------------------------------------- Willam-Warnke cone (Sec. 6.4)
#
# The CPT material's frictional cone with a Willam-Warnke deviatoric section
# and a non-associated Drucker-Prager potential: f = sqrt(J2) r(theta) + eta p
# - xi c, r = 1 on the compressive meridian (the outer Drucker-Prager cone)
# and 1/e on the tensile one, e = (3 - sin phi)/(3 + sin phi) (the
# Mohr-Coulomb ratio of the two meridian radii).

def ww_cfg(phi=32.0, psi=2.0):
    return inputs.workload("cone", model=3, phi=math.radians(phi), psi=math.radians(psi))


def stress_invariants(tau):
    p = np.trace(tau) / 3
    s = tau - p * np.eye(3)
    J2 = 0.5 * np.sum(s * s)
    J3 = np.linalg.det(s)
    zeta = np.clip(1.5 * math.sqrt(3) * J3 / J2 ** 1.5, -1, 1)
    return p, math.sqrt(J2), math.acos(zeta) / 3


def mohr_coulomb_radius_ratio(phi):
    # deviatoric radius of the Mohr-Coulomb hexagon on the tensile over the
    # compressive meridian, from the Mohr-Coulomb criterion written out in
    # principal stresses (tension positive): (s1 - s3) = -(s1 + s3) sin phi
    # + 2 c cos phi at p = 0, c = 1
    out = []
    for lode in ("t", "c"):
        # s = k (2, -1, -1)/sqrt6 (tensile) or k (1, 1, -2)/sqrt6 (compressive)
        d = np.array([2, -1, -1]) / math.sqrt(6) if lode == "t" else np.array([1, 1, -2]) / math.sqrt(6)
        s1, s3 = d.max(), d.min()
        k = 2 * math.cos(math.radians(phi)) / ((s1 - s3) + (s1 + s3) * math.sin(math.radians(phi)))
        out.append(k)
    return out[0] / out[1]


def test_willam_warnke_meridians_match_mohr_coulomb_and_drucker_prager():
    G, K, E = None, None, 2e7
    c = 5e3
    for phi in (20.0, 32.0, 40.0):
        cfg = ww_cfg(phi, 2.0)
        sphi = math.sin(math.radians(phi))
        eta = 6 * sphi / (math.sqrt(3) * (3 - sphi))
        xi = 6 * math.cos(math.radians(phi)) / (math.sqrt(3) * (3 - sphi))
        e = (3 - sphi) / (3 + sphi)
        assert abs(e - mohr_coulomb_radius_ratio(phi)) < 1e-12
        # compressive meridian (axial shortening with equal lateral strains):
        # identical to the outer-cone Drucker-Prager return
        dF = np.diag([1.0 + 0.008, 1.0 + 0.008, 1.0 - 0.015])
        t3, _, _, pl3 = oracle.constitutive(cfg, E, c, np.array([1, 1, 1, 0, 0, 0.0]), dF)
        t2, _, _, pl2 = oracle.constitutive(dict(cfg, model=2), E, c, np.array([1, 1, 1, 0, 0, 0.0]), dF)
        assert pl3 == 1 and pl2 == 1
        assert np.allclose(t3, t2, rtol=0, atol=1e-9 * c)
        p, sj, th = stress_invariants(t3)
        assert abs(th - math.pi / 3) < 1e-6
        # tensile meridian (axial extension): yields at e times that radius
        dF = np.diag([1.0 - 0.006, 1.0 - 0.006, 1.0 + 0.01])
        t3, _, _, pl3 = oracle.constitutive(cfg, E, c, np.array([1, 1, 1, 0, 0, 0.0]), dF)
        assert pl3 == 1
        p, sj, th = stress_invariants(t3)
        assert abs(th) < 1e-6
        assert abs(sj - e * (xi * c - eta * p)) < 1e-9 * c


def test_willam_warnke_return_is_consistent_keeps_lode_angle_and_section_is_convex():
    cfg = ww_cfg()
    E, c = 2e7, 5e3
    rng = np.random.default_rng(31)
    sphi = math.sin(math.radians(32.0))
    eta = 6 * sphi / (math.sqrt(3) * (3 - sphi))
    xi = 6 * math.cos(math.radians(32.0)) / (math.sqrt(3) * (3 - sphi))
    n_pl = 0
    for _ in range(40):
        dF = np.eye(3) + 0.02 * rng.normal(size=(3, 3)) - 0.01 * np.eye(3)
        el, _, _, _ = oracle.constitutive(dict(cfg, model=0), E, c, np.array([1, 1, 1, 0, 0, 0.0]), dF)
        t, _, _, pl = oracle.constitutive(cfg, E, c, np.array([1, 1, 1, 0, 0, 0.0]), dF)
        if pl != 1:
            continue
        n_pl += 1
        p, sj, th = stress_invariants(t)
        pe, sje, the = stress_invariants(el)
        assert abs(th - the) < 1e-7  # radial return: the Lode angle is kept
        # consistency: the section radius at this Lode angle
        r = ww_radius(th, (3 - sphi) / (3 + sphi))
        assert abs(sj * r + eta * p - xi * c) < 1e-8 * c
    assert n_pl >= 10
    # the deviatoric section rho(theta) = 1 / r(theta) is convex
    e = (3 - sphi) / (3 + sphi)
    th = np.linspace(0, math.pi / 3, 400)
    rho = 1.0 / np.array([ww_radius(t, e) for t in th])
    x, y = rho * np.cos(th), rho * np.sin(th)
    cross = (x[1:-1] - x[:-2]) * (y[2:] - y[1:-1]) - (y[1:-1] - y[:-2]) * (x[2:] - x[1:-1])
    assert np.all(cross > 0)


def ww_radius(theta, e):
    # the Willam-Warnke elliptic interpolation written in terms of theta
    a, b = 1 - e * e, 2 * e - 1
    c = math.cos(theta)
    return (4 * a * c * c + b * b) / (2 * a * c + b * math.sqrt(4 * a * c * c + 5 * e * e - 4 * e))


@pytest.mark.parametrize("psi", [2.0, 32.0])
def test_willam_warnke_spatial_tangent_matches_finite_difference(psi):
    cfg = ww_cfg(32.0, psi)
    E, ys = 2e7, 5e3
    rng = np.random.default_rng(8)
    be = np.array([1.02, 0.99, 1.01, 0.01, -0.005, 0.002])
    checked = 0
    for _ in range(6):
        dF = np.eye(3) + 0.01 * rng.normal(size=(3, 3)) - 0.003 * np.eye(3)
        tau, _, A, pl = oracle.constitutive(cfg, E, ys, be, dF)
        if pl != 1:
            continue
        checked += 1
        h = 1e-7
        for k in range(3):
            for mm in range(3):
                Lp = np.zeros((3, 3))
                Lp[k, mm] = h
                tp, _, _, _ = oracle.constitutive(cfg, E, ys, be, (np.eye(3) + Lp) @ dF, tangent=False)
                tm, _, _, _ = oracle.constitutive(cfg, E, ys, be, (np.eye(3) - Lp) @ dF, tangent=False)
                fd = (tp - tm) / (2 * h)
                assert np.allclose(A[:, :, k, mm], fd, atol=2e-6 * E, rtol=0), (k, mm)
    assert checked >= 2


def test_global_tangent_matches_finite_difference_willam_warnke_with_cone():
    # (the directions avoid cone/apex and contact switches within the FD step)
    cfg = cone_cfg(model=3, phi=math.radians(32.0), psi=math.radians(2.0))
    z0 = cfg["body"]["z0"]
    m = built(cfg, body_z=z0 - 0.06)
    c = m.counts()
    n3 = 3 * c["ndof"]
    du = 1e-3 * np.random.default_rng(17).normal(size=n3)
    out = m.assemble(du)
    rp, col = m.pattern()
    K = out["K"]
    h = 1e-7
    rng = np.random.default_rng(5)
    for _ in range(3):
        v = rng.normal(size=n3)
        fd = (m.assemble(du + h * v, tangent=False)["R"] -
              m.assemble(du - h * v, tangent=False)["R"]) / (2 * h)
        Kv = np.zeros(n3)
        for i in range(c["ndof"]):
            for s_ in range(rp[i], rp[i + 1]):
                Kv[3 * i:3 * i + 3] += K[s_] @ v[3 * col[s_]:3 * col[s_] + 3]
        assert np.linalg.norm(Kv - fd) <= 1e-6 * np.linalg.norm(fd)


def test_cpt_workload_follows_the_paper_table_and_stiffness_law():
    # Sec. 6.4: the CPT sand's constants, K0 = 1 - sin(phi) (Jaky), and E50
    # fixed per point by its initial depth d: E50_ref (gamma d K0 / p_ref)^m_E
    g = read_golden("paper_constants.txt")
    cfg = inputs.workload("cpt")
    pc = cfg["points"]
    assert pc["E"] == g["cpt_E50_ref"][0] and cfg["nu"] == g["cpt_nu"][0]
    assert abs(pc["rho"] * 9.81 - g["cpt_unit_weight"][0]) < 1e-9
    assert abs(math.degrees(cfg["phi"]) - g["cpt_phi"][0]) < 1e-12
    assert abs(math.degrees(cfg["psi"]) - g["cpt_psi"][0]) < 1e-12
    assert pc["ys"] == g["cpt_cohesion"][0] and cfg["mu"] == g["cpt_mu"][0]
    assert cfg["model"] == 3
    assert abs((1 - math.sin(cfg["phi"])) - g["cpt_K0"][0]) < 5e-3
    b = cfg["body"]
    assert b["r"] == g["cpt_cone_radius"][0]
    assert abs(2 * math.degrees(b["alpha"]) - g["cpt_cone_apex_angle"][0]) < 1e-12
    # quarter domain: half the width, rollers on the symmetry planes through the axis
    assert pc["hi"][0] == g["cpt_Lx"][0] / 2 and pc["hi"][2] == g["cpt_Lz"][0]
    assert b["cx"] == 0.0 and b["cy"] == 0.0
    assert (0, 0.0, inputs.ROLLER_X) in cfg["bc"] and (1, 0.0, inputs.ROLLER_Y) in cfg["bc"]
    pts = inputs.make_points(cfg)
    d = pc["hi"][2] - pts["x"][:, 2]
    K0 = 1 - math.sin(math.radians(g["cpt_phi"][0]))
    for k in (0, len(d) // 2, len(d) - 1):
        e = g["cpt_E50_ref"][0] * (g["cpt_unit_weight"][0] * d[k] * K0 / 100e3) ** g["cpt_mE"][0]
        assert abs(pts["E"][k] - e) < 1e-9 * e
    # at 10 m depth: 19.2 MPa (16.3 * 10 * 0.47 / 100)^0.6 = about 15.7 MPa
    assert abs(inputs.cpt_stiffness(10.0) - 19.2e6 * (16.3 * 10 * K0 / 100) ** 0.6) < 1e-6
