"""Seeded synthetic inputs shared by the GPU path, the oracle and the benchmark.

This module holds none of the method's arithmetic.  It only
  * places material points on a regular lattice inside a block (optionally
    jittered with a seeded uniform offset) and gives them their material
    constants (optionally a seeded lognormal Young's modulus), and
  * states the parameter sets of the workloads: domain cube, refinement depths,
    Dirichlet planes, rigid body and its motion, material, load schedule.

Point arrays (all float64, C order):
  x (P,3) centre, lp (P,3) current half-lengths, l0 (P,3) reference
  half-lengths, F (P,9) row-major deformation gradient, be (P,6) elastic left
  Cauchy-Green tensor as (xx, yy, zz, xy, yz, xz), V0 (P,) reference volume,
  mass (P,), E (P,) Young's modulus, ys (P,) yield stress (von Mises) or
  cohesion (Drucker-Prager).
"""
import copy
import math

import numpy as np

# roller planes: (axis, position, fixed-component mask); mask bit d = component d
ROLLER_X, ROLLER_Y, ROLLER_Z, FIXED = 1, 2, 4, 7


def lattice_points(lo, hi, spacing, rho, E, ys, jitter=0.0, seed=0, E_sigma=0.0):
    """Material points on a lattice of the given spacing filling [lo, hi].

    Each point's domain is the lattice cell (half-length spacing/2).  With
    jitter > 0 every centre is moved by U(-jitter, jitter) per axis (seeded).
    With E_sigma > 0 the modulus is lognormal around E (seeded, seed + 1).
    """
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    n = [int(round((hi[d] - lo[d]) / spacing)) for d in range(3)]
    iz, iy, ix = np.meshgrid(np.arange(n[2]), np.arange(n[1]), np.arange(n[0]), indexing="ij")
    idx = np.stack([ix.ravel(), iy.ravel(), iz.ravel()], axis=1).astype(np.float64)
    x = lo[None, :] + (idx + 0.5) * spacing
    P = x.shape[0]
    if jitter > 0.0:
        rng = np.random.default_rng(seed)
        x = x + rng.uniform(-jitter, jitter, size=(P, 3))
    half = 0.5 * spacing
    pts = {
        "x": np.ascontiguousarray(x),
        "lp": np.full((P, 3), half),
        "l0": np.full((P, 3), half),
        "F": np.tile(np.eye(3).ravel(), (P, 1)),
        "be": np.tile(np.array([1.0, 1.0, 1.0, 0.0, 0.0, 0.0]), (P, 1)),
        "V0": np.full(P, spacing ** 3),
        "mass": np.full(P, rho * spacing ** 3),
        "E": np.full(P, float(E)),
        "ys": np.full(P, float(ys)),
    }
    if E_sigma > 0.0:
        rng = np.random.default_rng(seed + 1)
        pts["E"] = np.exp(rng.normal(math.log(E), E_sigma, size=P))
    return pts


def cpt_stiffness(depth, E_ref=19.2e6, gamma=16.3e3, phi=math.radians(32.0), m_E=0.6,
                  p_ref=100e3):
    """E50 of the CPT sand (Sec. 6.4): E_ref (sigma_v K0 / p_ref)^m_E with
    sigma_v = gamma d (d the initial depth of the point centre, gamma the unit
    weight) and K0 = 1 - sin(phi); p_ref, which the paper does not state, is
    taken as the usual 100 kPa."""
    K0 = 1.0 - math.sin(phi)
    return E_ref * (gamma * np.asarray(depth) * K0 / p_ref) ** m_E


def make_points(cfg):
    pc = cfg["points"]
    pts = lattice_points(pc["lo"], pc["hi"], pc["spacing"], pc["rho"], pc["E"], pc["ys"],
                         jitter=pc.get("jitter", 0.0), seed=pc.get("seed", 0),
                         E_sigma=pc.get("E_sigma", 0.0))
    if cfg.get("cpt"):
        # fixed by each point's initial depth below the block top
        pts["E"] = cpt_stiffness(pc["hi"][2] - pts["x"][:, 2], E_ref=pc["E"],
                                 gamma=pc["rho"] * 9.81, phi=cfg["phi"])
    return pts


def sphere_mesh(radius, nlat=40, nlon=40):
    """Closed triangulated sphere on a latitude-longitude grid (the smallest
    triangles at the poles): nlat bands, nlon sectors, 2 nlon (nlat - 1)
    triangles (3120 for 40 x 40), counter-clockwise seen from outside, centred
    on the origin."""
    th = np.pi * np.arange(1, nlat) / nlat
    ph = 2 * np.pi * np.arange(nlon) / nlon
    v = [[0.0, 0.0, radius]]
    for t in th:
        for p in ph:
            v.append([radius * math.sin(t) * math.cos(p), radius * math.sin(t) * math.sin(p),
                      radius * math.cos(t)])
    v.append([0.0, 0.0, -radius])
    south = len(v) - 1
    ring = lambda i, j: 1 + i * nlon + (j % nlon)
    tri = []
    for j in range(nlon):
        tri.append([0, ring(0, j), ring(0, j + 1)])
    for i in range(nlat - 2):
        for j in range(nlon):
            a, b, c, d = ring(i, j), ring(i, j + 1), ring(i + 1, j), ring(i + 1, j + 1)
            tri.append([a, c, d])
            tri.append([a, d, b])
    for j in range(nlon):
        tri.append([south, ring(nlat - 2, j + 1), ring(nlat - 2, j)])
    return dict(v=np.array(v), t=np.array(tri, dtype=np.int32))


def cylinder_mesh(radius, height, nside=64, phase=0.0):
    """Closed triangulated flat-ended cylinder (a prism of nside sides) with
    its bottom face at z = 0 centred on the axis, counter-clockwise seen from
    outside; the polygon's vertices at angles (k + phase) 2 pi / nside."""
    ph = 2 * np.pi * (np.arange(nside) + phase) / nside
    v = [[0.0, 0.0, 0.0], [0.0, 0.0, height]]
    for z in (0.0, height):
        for p in ph:
            v.append([radius * math.cos(p), radius * math.sin(p), z])
    lo = lambda j: 2 + (j % nside)
    hi = lambda j: 2 + nside + (j % nside)
    tri = []
    for j in range(nside):
        tri.append([0, lo(j + 1), lo(j)])        # bottom, normal -z
        tri.append([1, hi(j), hi(j + 1)])        # top, normal +z
        tri.append([lo(j), lo(j + 1), hi(j + 1)])
        tri.append([lo(j), hi(j + 1), hi(j)])
    return dict(v=np.array(v), t=np.array(tri, dtype=np.int32))


def body_z(cfg, step):
    """Vertical position of the rigid body at the end of load step `step` (1-based)."""
    b = cfg["body"]
    return b["z0"] + step * b["dz"]


def load_factor(cfg, step):
    if cfg.get("ramp_steps"):
        return min(1.0, step / cfg["ramp_steps"])
    return step / cfg["nsteps"] if cfg.get("ramp_load", False) else 1.0


def _block_rollers(x1, y1, fixed_base=True):
    return [(0, 0.0, ROLLER_X), (0, x1, ROLLER_X), (1, 0.0, ROLLER_Y), (1, y1, ROLLER_Y),
            (2, 0.0, FIXED if fixed_base else ROLLER_Z)]


_BASE = dict(beta=2.0, nu=0.3, phi=0.0, psi=0.0, g=(0.0, 0.0, 0.0), kappa=10.0, pf=50.0, pt=25.0,
             mu=0.0,
             ghost=1, contact=1, body=None, dx_region=0.0, ramp_load=False,
             newton_tol=1e-8, newton_maxit=30, lin_tol=1e-8, lin_maxit=20000)


def workload(name, **over):
    """Parameter set of a named workload (a fresh dict; keyword overrides win)."""
    c = copy.deepcopy(_BASE)
    if name == "column":
        # elastic column under self-weight, unit cube, uniform depth 3, 2x2x2 points
        # per cell, gravity ramped over 10 load steps, roller sides, fixed base
        c.update(L=1.0, depth_min=3, depth_max=3, bc=_block_rollers(1.0, 1.0), model=0,
                 g=(0.0, 0.0, -9.81), nsteps=10, ramp_load=True, contact=0,
                 points=dict(lo=(0, 0, 0), hi=(1, 1, 1), spacing=1.0 / 16, rho=1000.0,
                             E=1e6, ys=0.0))
    elif name == "punch":
        # flat-ended cylindrical punch (r = 0.1 m) into a 1 x 1 x 0.5 m von Mises
        # block, depth 3 far field refined to depth 6 within 2 finest cells of the
        # punch, 50 load steps to 0.1 m
        c.update(L=1.0, depth_min=3, depth_max=6, bc=_block_rollers(1.0, 1.0), model=1,
                 body=dict(kind=1, cx=0.5, cy=0.5, z0=0.5, r=0.1, alpha=0.0, dz=-0.1 / 50),
                 dx_region=2.0 / 64, nsteps=50,
                 points=dict(lo=(0, 0, 0), hi=(1, 1, 0.5), spacing=1.0 / 16, rho=1000.0,
                             E=1e7, ys=1e5))
    elif name == "cone":
        # 60-degree cone (base diameter 0.036 m) pushed 0.3 m into a 1 x 1 x 1.2 m
        # Drucker-Prager layer; the cube [0,1.6]^3 at depth 4 (0.1 m cells) keeps
        # the layer faces on cell faces; refined to depth 8 at the cone.  Centres
        # jittered by U(-h/8, h/8) so that no domain corner sits on the cone axis
        c.update(L=1.6, depth_min=4, depth_max=8, bc=_block_rollers(1.0, 1.0), model=2,
                 phi=math.radians(30.0), psi=0.0,
                 body=dict(kind=2, cx=0.5, cy=0.5, z0=1.2, r=0.018, alpha=math.radians(30.0),
                           dz=-0.3 / 200),
                 dx_region=2.0 * 1.6 / 256, nsteps=200,
                 points=dict(lo=(0, 0, 0), hi=(1, 1, 1.2), spacing=0.05, rho=1000.0,
                             E=2e7, ys=5e3, jitter=0.0125, seed=0))
    elif name == "cpt":
        # the cone penetration test of Sec. 6.4 on a quarter domain (symmetry
        # planes x = 0 and y = 0 through the cone axis): the CPT sand of the
        # material table (E50_ref 19.2 MPa, unit weight 16.3 kN/m3, nu 0.25,
        # phi 32, psi 2, c 0.3 kPa, K0 0.47, m_E 0.6) as the Willam-Warnke cone
        # (model 3), E fixed per point by its initial depth (cpt_stiffness),
        # self-weight (ramped over the first 5 load steps, while the cone
        # approaches), a 60-degree cone of radius 0.4 m with friction 0.3; the
        # block 6.4 x 6.4 x 24.6 m in a 25.6 m cube, 1.6 m cells refined to
        # 0.1 m within 0.2 m of the cone
        c.update(L=25.6, depth_min=4, depth_max=8, bc=_block_rollers(6.4, 6.4), model=3,
                 nu=0.25, phi=math.radians(32.0), psi=math.radians(2.0), mu=0.3,
                 g=(0.0, 0.0, -9.81), dx_region=0.2, nsteps=300, cpt=True, ramp_steps=5,
                 body=dict(kind=2, cx=0.0, cy=0.0, z0=24.6 + 0.135, r=0.4,
                           alpha=math.radians(30.0), dz=-0.025),
                 points=dict(lo=(0, 0, 0), hi=(6.4, 6.4, 24.6), spacing=0.8,
                             rho=16.3e3 / 9.81, E=19.2e6, ys=300.0, jitter=0.1, seed=0))
    elif name == "adjoint":
        # the punch at depth 3 to 5, 20 load steps, lognormal E (sigma 0.2);
        # centres jittered by U(-h/8, h/8) as in the indentation recipes, so
        # that no domain face starts on a cell plane (there the far field's
        # tiny displacements decide whether a cell is populated, and the
        # discrete events of a run flip under any perturbation of the input)
        c.update(L=1.0, depth_min=3, depth_max=5, bc=_block_rollers(1.0, 1.0), model=1,
                 body=dict(kind=1, cx=0.5, cy=0.5, z0=0.5, r=0.1, alpha=0.0, dz=-0.1 / 50),
                 dx_region=2.0 / 32, nsteps=20,
                 points=dict(lo=(0, 0, 0), hi=(1, 1, 0.5), spacing=1.0 / 16, rho=1000.0,
                             E=1e7, ys=1e5, E_sigma=0.2, seed=0, jitter=1.0 / 128))
    elif name == "adjoint_60k":
        # the same punch and mesh with the points three times finer per axis
        # (spacing 1/48, 6x6x6 per depth-3 cell, jitter U(-h/8, h/8)): 55,296
        # points at the start, about 67 k after the first step's splits
        c = workload("adjoint")
        c["points"].update(spacing=1.0 / 48, jitter=1.0 / 384)
    elif name == "cone_1m":
        # the cone of "cone" at the ~1M-DOF scale: the same Drucker-Prager layer
        # and cone on a depth-6 far field (0.025 m cells, 2x2x2 points per cell,
        # jittered by U(-h/8, h/8)) refined to depth 8 (6.25 mm) within a wider
        # region around the cone (0.3 m), so that the adapted mesh has about a
        # million unknowns; the GIMP split grows the points about 4.8 times
        # (cap_factor: the point capacity to allocate, in initial points)
        c.update(L=1.6, depth_min=6, depth_max=8, bc=_block_rollers(1.0, 1.0), model=2,
                 phi=math.radians(30.0), psi=0.0,
                 body=dict(kind=2, cx=0.5, cy=0.5, z0=1.2, r=0.018, alpha=math.radians(30.0),
                           dz=-0.3 / 200),
                 dx_region=0.3, nsteps=200, cap_factor=6,
                 points=dict(lo=(0, 0, 0), hi=(1, 1, 1.2), spacing=0.0125, rho=1000.0,
                             E=2e7, ys=5e3, jitter=0.0125 / 4, seed=0))
    elif name == "indent":
        # indentation at the ~1M-DOF scale: the punch physics of "punch" on a depth 6
        # far field (2x2x2 jittered points per cell, U(-h/8, h/8)) refined to depth
        # 7 at the punch; block 1 x 1 x 0.875 m under the cube top
        c.update(L=1.0, depth_min=6, depth_max=7, bc=_block_rollers(1.0, 1.0), model=1,
                 body=dict(kind=1, cx=0.5, cy=0.5, z0=0.875, r=0.1, alpha=0.0, dz=-0.1 / 50),
                 dx_region=2.0 / 128, nsteps=50,
                 points=dict(lo=(0, 0, 0), hi=(1, 1, 0.875), spacing=1.0 / 128, rho=1000.0,
                             E=1e7, ys=1e5, jitter=1.0 / 512, seed=0))
    elif name == "rolling_sphere":
        # the rigid sphere rolling down a 45-degree slope of Sec. 6.3, shortened:
        # sphere of diameter 2 m, mass 1e4 kg, rotational inertia 4000 kg m2
        # (the analytic sphere), on a stiff elastic slab (E 1e9 Pa, nu 0;
        # density 2000 kg/m3, which the paper does not state) 4 x 1 x 1 m in
        # a 4 m cube, 0.5 m cells refined to 0.125 m within 0.25 m of the
        # sphere; the slope is the slab's top face under the tilted gravity
        # 9.81 (1/sqrt 2, 0, -1/sqrt 2); the sphere starts at rest touching the
        # slab; Newmark time steps of 0.01 s; the sphere is free to translate
        # in x and z and to rotate about y (the motion stays in that plane by
        # symmetry); rollers on the slab's sides, its base fixed
        gs = 9.81 / math.sqrt(2.0)
        c.update(L=4.0, depth_min=3, depth_max=5, bc=_block_rollers(4.0, 1.0), model=0, nu=0.0,
                 g=(gs, 0.0, -gs), dt=0.01, nsteps=40, mu=1.0, dx_region=0.25,
                 body=dict(kind=4, cx=1.0, cy=0.5, z0=2.0, r=1.0, dz=0.0, step_d=(0.0, 0.0, 0.0),
                           free=1 | 4 | 16, mass=1e4, inertia=4000.0),
                 points=dict(lo=(0, 0, 0), hi=(4, 1, 1), spacing=0.25, rho=2000.0,
                             E=1e9, ys=0.0))
    elif name == "indent_small":
        # the indentation recipe one level coarser (depth 5 -> 6): stiffness larger
        # than L2 but a few GB on the device, for detailed profiles
        c.update(L=1.0, depth_min=5, depth_max=6, bc=_block_rollers(1.0, 1.0), model=1,
                 body=dict(kind=1, cx=0.5, cy=0.5, z0=0.875, r=0.1, alpha=0.0, dz=-0.1 / 50),
                 dx_region=2.0 / 64, nsteps=50,
                 points=dict(lo=(0, 0, 0), hi=(1, 1, 0.875), spacing=1.0 / 64, rho=1000.0,
                             E=1e7, ys=1e5, jitter=1.0 / 256, seed=0))
    else:
        raise KeyError(name)
    for k, v in over.items():
        if k == "points":
            c["points"].update(v)
        elif k == "body" and v is not None and c["body"] is not None:
            c["body"].update(v)
        else:
            c[k] = v
    return c
