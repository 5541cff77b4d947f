"""Pins of the oracle's time steps (Sec. 2.4: Newmark with gamma = 1,
beta = 1/2) and of the free rigid body coupled by contact (Sec. 2.3, 2.4),
checked against what the mechanics fixes, not against the oracle itself.

* A block in free fall (no support, no body): Newmark integrates a constant
  acceleration exactly, so every point follows x0 + g t^2 / 2 with velocity
  g t to rounding, and stays unstrained.  A wrong beta or gamma, a dropped
  mass or a wrong sign of the inertia term all break this.
* A free rigid body in free fall: the same parabola for the body, no rotation.
* A free elastic block with a non-uniform initial velocity and no external
  force conserves its linear momentum sum_p m_p v_p (the basis is a
  partition of unity, the internal force and the ghost term sum to zero over
  the nodes); a wrong velocity update or a mass missing from the inertia
  shows here.
* Directional central differences of the material and body residuals
  (R, Rb) against the bordered Jacobian (K, dR/dq, dRb/du, dRb/dq) with
  the sphere in frictional contact, some nodes sticking and some slipping,
  and a non-zero body rotation: catches a wrong sign or a missing term in the
  coupling blocks (the lever arm, [f]x, [q_R]x).
* The rolling sphere of Sec. 6.3 against the paper's closed form of the
  distance travelled (stick: 5 g t^2 sin(theta) / 14; slip:
  g t^2 (sin(theta) - mu cos(theta)) / 2), in the three regimes the paper's
  friction coefficients span: mu = 1 sticks (the sphere rolls, theta R = d),
  mu = 0.1 slips (its spin follows the friction torque), mu = 0 slides
  without turning.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2606_09275_gb300 import inputs


def free_block_cfg(**over):
    c = inputs.workload("column", contact=0, ramp_load=False, model=0, nu=0.3, bc=[], dt=0.01,
                        g=(0.0, 0.0, 0.0))
    c.update(L=1.0, depth_min=3, depth_max=3)
    c["points"].update(lo=(0.25, 0.25, 0.25), hi=(0.75, 0.75, 0.75), spacing=1.0 / 16, E=1e6)
    c.update(over)
    return c


def test_free_fall_of_a_block_follows_the_parabola():
    g = np.array([1.0, -2.0, -9.81])
    cfg = free_block_cfg(g=tuple(g))
    pts = inputs.make_points(cfg)
    m = oracle.Model(cfg, pts)
    x0 = pts["x"].copy()
    dt = cfg["dt"]
    for n in range(1, 5):
        st = m.step(load=1.0, tol=1e-11, lin_tol=1e-14)
        assert st["status"] == 0
        t = n * dt
        p = m.points()
        # a wrong beta, gamma or inertia sign moves these by O(g dt^2)
        assert np.abs(p["x"] - (x0 + 0.5 * g * t * t)).max() <= 1e-12
        assert np.abs(m.velocity() - g * t).max() <= 1e-11
        assert np.abs(p["F"] - np.eye(3).ravel()).max() <= 1e-12


def test_free_fall_of_a_free_body_follows_the_parabola():
    # the sphere above the block, out of contact: only its own equations move it
    g = np.array([0.5, 0.0, -9.81])
    cfg = free_block_cfg(g=tuple(g), contact=1, dx_region=0.0, depth_max=3,
                         body=dict(kind=4, cx=0.5, cy=0.5, z0=0.95, r=0.1, dz=0.0,
                                   step_d=(0.0, 0.0, 0.0), free=63, mass=3.0, inertia=0.2,
                                   v=(0.0, 0.0, 0.0), w=(0.0, 0.0, 0.0)))
    cfg["points"].update(lo=(0.25, 0.25, 0.0), hi=(0.75, 0.75, 0.25))
    m = oracle.Model(cfg, inputs.make_points(cfg))
    for n in range(1, 4):
        st = m.step(load=1.0, tol=1e-11, lin_tol=1e-14)
        assert st["status"] == 0
        b = m.body_state()
        t = n * cfg["dt"]
        X = np.array([0.5, 0.5, 0.95]) + 0.5 * g * t * t
        assert np.abs(b["pose"] - X).max() <= 1e-12
        assert np.abs(b["v"] - g * t).max() <= 1e-11
        assert np.abs(b["w"]).max() == 0.0 and np.abs(b["theta"]).max() == 0.0
        assert np.abs(st["reaction"]).max() == 0.0


def test_free_elastic_block_conserves_linear_momentum():
    cfg = free_block_cfg()
    pts = inputs.make_points(cfg)
    m = oracle.Model(cfg, pts)
    x = pts["x"] - 0.5
    # rigid spin + a shear + a stretch: non-uniform, so the block deforms
    v = np.cross(np.array([0.0, 0.0, 2.0]), x) + np.stack(
        [0.5 * x[:, 2], 0.0 * x[:, 0], -0.8 * x[:, 2] + 0.3], axis=1)
    m.set_velocity(v)
    mass = pts["mass"]
    p0 = (mass[:, None] * v).sum(axis=0)
    scale = (mass[:, None] * np.abs(v)).sum()
    for _ in range(3):
        st = m.step(load=1.0, tol=1e-11, lin_tol=1e-14)
        assert st["status"] == 0
        vn = m.velocity()
        mn = m.points()["mass"]
        p1 = (mn[:, None] * vn).sum(axis=0)
        assert np.abs(p1 - p0).max() <= 1e-10 * scale, (p0, p1)
    # and the block did deform (the test is not a rigid translation)
    assert np.abs(m.points()["F"] - np.eye(3).ravel()).max() > 1e-4


def _contact_state(mu):
    """A rolling-sphere mesh with the sphere pressed into the slab, a nodal
    increment with a tangential part and a body increment that turns it."""
    cfg = inputs.workload("rolling_sphere", mu=mu)
    cfg["body"]["free"] = 63
    cfg["body"]["z0"] = 2.0 - 0.004
    cfg["body"]["v"] = (0.3, 0.0, -0.1)
    cfg["body"]["w"] = (0.0, 0.2, 0.0)
    pts = inputs.make_points(cfg)
    m = oracle.Model(cfg, pts)
    m.build()
    rng = np.random.default_rng(5)
    n3 = 3 * m.counts()["ndof"]
    du = 1e-4 * rng.standard_normal(n3)
    q = np.array([2e-3, -1e-4, -5e-4, 1e-4, 1.5e-3, -2e-4])
    return m, du, q


def _apply(m, out, v, w):
    """(K v + dR/dq w, dRb/du v + dRb/dq w) from the assembled blocks."""
    rp, col = m.pattern()
    K = out["K"]
    n = len(rp) - 1
    Kv = np.zeros(3 * n)
    for i in range(n):
        for s in range(rp[i], rp[i + 1]):
            Kv[3 * i:3 * i + 3] += K[s] @ v[3 * col[s]:3 * col[s] + 3]
    return Kv + out["Kgb"].T @ w, out["Kbg"] @ v + out["Kbb"] @ w


@pytest.mark.parametrize("mu", [0.0, 0.05, 0.3, 3.0])
def test_bordered_jacobian_matches_central_differences(mu):
    m, du, q = _contact_state(mu)
    out = m.assemble_body(du, q)
    assert np.abs(out["Rb"]).max() > 0.0 and np.abs(out["Kgb"]).max() > 0.0
    rng = np.random.default_rng(7)
    n3 = len(du)
    dirs = [(rng.standard_normal(n3), np.zeros(6))]
    dirs += [(np.zeros(n3), np.eye(6)[j]) for j in range(6)]
    dirs += [(rng.standard_normal(n3), rng.standard_normal(6))]
    Rscale = max(np.abs(out["R"]).max(), 1.0)
    Bscale = max(np.abs(out["Rb"]).max(), 1.0)
    for v, w in dirs:
        v = v * 1e-4 / max(np.abs(v).max(), 1e-300)
        w = w * 1e-4
        h = 1e-4
        a = m.assemble_body(du + h * v, q + h * w, tangent=False)
        b = m.assemble_body(du - h * v, q - h * w, tangent=False)
        fdR = (a["R"] - b["R"]) / (2 * h)
        fdB = (a["Rb"] - b["Rb"]) / (2 * h)
        JR, JB = _apply(m, out, v, w)
        # every direction moves the residuals measurably
        assert np.abs(fdR).max() + np.abs(fdB).max() > 1e-6 * (Rscale + Bscale)
        assert np.abs(JR - fdR).max() <= 1e-6 * max(np.abs(fdR).max(), 1e-3 * Rscale), (mu, w)
        assert np.abs(JB - fdB).max() <= 1e-6 * max(np.abs(fdB).max(), 1e-3 * Bscale), (mu, w)


@pytest.mark.parametrize("mu,regime", [(1.0, "stick"), (0.1, "slip"), (0.0, "slide")])
def test_rolling_sphere_matches_the_closed_form(mu, regime):
    cfg = inputs.workload("rolling_sphere", mu=mu)
    m = oracle.Model(cfg, inputs.make_points(cfg))
    g, th, dt = 9.81, math.pi / 4, cfg["dt"]
    x0 = m.body_state()["pose"][0]
    nsteps = 10
    for _ in range(nsteps):
        st = m.step(load=1.0, tol=1e-10, maxit=40, lin_tol=1e-12)
        assert st["status"] == 0
    t = nsteps * dt
    b = m.body_state()
    d = b["pose"][0] - x0
    if regime == "stick":
        assert math.tan(th) <= 3.5 * mu
        ana = 5.0 * g * t * t * math.sin(th) / 14.0
        # rolling without slip: the rotation about y times the radius is the distance
        assert abs(b["theta"][1] * cfg["body"]["r"] - d) <= 0.05 * d
    else:
        assert math.tan(th) > 3.5 * mu
        ana = 0.5 * g * t * t * (math.sin(th) - mu * math.cos(th))
        # the friction torque mu N r spins the sphere up: theta = mu N r t^2 / (2 J)
        N = cfg["body"]["mass"] * g * math.cos(th)
        spin = mu * N * cfg["body"]["r"] * t * t / (2.0 * cfg["body"]["inertia"])
        assert abs(b["theta"][1] - spin) <= 0.05 * spin + 1e-9
    # the three regimes differ by 11 % and more at this time
    assert abs(d - ana) <= 0.02 * ana, (regime, d, ana)
