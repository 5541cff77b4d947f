"""Python wrapper of the FP64 CPU oracle (ctypes over oracle/liboracle.so).

TEST INFRASTRUCTURE ONLY: the test-suite, the smoke check and the CPU-baseline
and reference legs of the benchmark use it; the product path never imports it.  It shares no
code with the CUDA library; inputs come from the seeded generators in
paper_2606_09275_gb300.inputs, passed in as plain arrays and dicts.
"""
import ctypes as C
import os

import numpy as np

from . import build as _build

MAXS = 64
_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp = C.c_void_p
        L.o_create.restype = vp
        L.o_create.argtypes = [C.POINTER(Params)]
        L.o_free.argtypes = [vp]
        L.o_set_points.argtypes = [vp, C.c_int] + [vp] * 9
        L.o_get_points.argtypes = [vp] + [vp] * 9
        L.o_set_body_z.argtypes = [vp, C.c_double]
        L.o_build.argtypes = [vp, C.c_int]
        L.o_counts_get.argtypes = [vp, C.POINTER(Counts)]
        L.o_export_tree.argtypes = [vp, vp, vp]
        L.o_export_nodes.argtypes = [vp] + [vp] * 6
        L.o_export_support.argtypes = [vp] + [vp] * 4
        L.o_export_pattern.argtypes = [vp, vp, vp]
        L.o_export_ghost.argtypes = [vp, vp]
        L.o_export_bcmask.argtypes = [vp, vp]
        L.o_export_ghost_faces.argtypes = [vp, vp, vp]
        L.o_eval_background.argtypes = [vp, vp, vp, vp, vp, vp]
        L.o_assemble.argtypes = [vp, vp, C.c_double, vp, vp, vp, vp]
        L.o_solve.argtypes = [vp, vp, vp, vp, C.c_double, C.c_int, vp]
        L.o_step.argtypes = [vp, C.POINTER(StepParams), C.POINTER(StepStats)]
        L.o_constitutive.argtypes = [C.POINTER(Params), C.c_double, C.c_double, vp, vp, vp, vp,
                                     vp, vp]
        L.o_eig_sym3.argtypes = [vp, vp, vp]
        L.o_point_stress.argtypes = [vp, vp, vp]
        L.o_body_sdf.argtypes = [C.POINTER(Params), vp, vp, vp, vp]
        L.o_assemble_body.argtypes = [vp, vp, vp, C.c_double] + [vp] * 8
        L.o_set_velocity.argtypes = [vp, vp]
        L.o_get_velocity.argtypes = [vp, vp]
        L.o_get_body.argtypes = [vp, vp, vp, vp, vp]
        _lib = L
    return _lib


class Params(C.Structure):
    _fields_ = [("L", C.c_double), ("depth_min", C.c_int), ("depth_max", C.c_int),
                ("nbc", C.c_int), ("bc_axis", C.c_int * 8), ("bc_pos", C.c_double * 8),
                ("bc_mask", C.c_int * 8),
                ("body_kind", C.c_int), ("body_cx", C.c_double), ("body_cy", C.c_double),
                ("body_z", C.c_double), ("body_r", C.c_double), ("body_alpha", C.c_double),
                ("dx_region", C.c_double), ("beta", C.c_double),
                ("model", C.c_int), ("nu", C.c_double), ("phi", C.c_double), ("psi", C.c_double),
                ("g", C.c_double * 3), ("kappa", C.c_double), ("pf", C.c_double),
                ("ghost_on", C.c_int), ("contact_on", C.c_int),
                ("mu", C.c_double), ("pt", C.c_double), ("body_d", C.c_double * 3),
                ("ntri", C.c_int), ("nvert", C.c_int), ("tri_v", C.c_void_p),
                ("tri_t", C.c_void_p), ("dt", C.c_double), ("body_free", C.c_int),
                ("body_mass", C.c_double), ("body_inertia", C.c_double),
                ("body_v", C.c_double * 3), ("body_w", C.c_double * 3)]


class Counts(C.Structure):
    _fields_ = [(n, C.c_int) for n in
                ("nleaf", "nnode", "nhang", "ndof", "nnzb", "nghost", "npts", "maxs")]


class StepParams(C.Structure):
    _fields_ = [("load", C.c_double), ("tol", C.c_double), ("maxit", C.c_int),
                ("lin_tol", C.c_double), ("lin_maxit", C.c_int)]


class StepStats(C.Structure):
    _fields_ = [("newton_its", C.c_int), ("lin_its_total", C.c_int), ("status", C.c_int),
                ("res_hist", C.c_double * 64), ("reaction", C.c_double * 3),
                ("eta_hist", C.c_double * 64), ("body_q", C.c_double * 6)]


def params_from_cfg(cfg, body_z=None):
    p = Params()
    p.L = cfg["L"]
    p.depth_min = cfg["depth_min"]
    p.depth_max = cfg["depth_max"]
    p.nbc = len(cfg["bc"])
    for i, (ax, pos, mask) in enumerate(cfg["bc"]):
        p.bc_axis[i] = ax
        p.bc_pos[i] = pos
        p.bc_mask[i] = mask
    b = cfg.get("body")
    if b:
        p.body_kind = b["kind"]
        p.body_cx, p.body_cy = b["cx"], b["cy"]
        p.body_z = b["z0"] if body_z is None else body_z
        p.body_r, p.body_alpha = b["r"], b.get("alpha", 0.0)
    p.dx_region = cfg.get("dx_region", 0.0)
    p.beta = cfg.get("beta", 2.0)
    p.model = cfg["model"]
    p.nu, p.phi, p.psi = cfg["nu"], cfg.get("phi", 0.0), cfg.get("psi", 0.0)
    for d in range(3):
        p.g[d] = cfg["g"][d]
    p.kappa, p.pf = cfg.get("kappa", 10.0), cfg.get("pf", 50.0)
    p.ghost_on, p.contact_on = int(cfg.get("ghost", 1)), int(cfg.get("contact", 1))
    p.mu, p.pt = cfg.get("mu", 0.0), cfg.get("pt", 25.0)
    p.dt = cfg.get("dt", 0.0)
    if b:
        d = b.get("step_d", (0.0, 0.0, b.get("dz", 0.0)))
        for k in range(3):
            p.body_d[k] = d[k]
        # a free body (time steps only): free components, mass, rotational
        # inertia and its velocities at the start
        p.body_free = int(b.get("free", 0))
        p.body_mass, p.body_inertia = b.get("mass", 0.0), b.get("inertia", 0.0)
        for k in range(3):
            p.body_v[k] = b.get("v", (0.0, 0.0, 0.0))[k]
            p.body_w[k] = b.get("w", (0.0, 0.0, 0.0))[k]
        if b["kind"] == 3:
            # the triangulated surface: host arrays kept alive by the struct
            v = np.ascontiguousarray(b["mesh"]["v"], dtype=np.float64)
            t = np.ascontiguousarray(b["mesh"]["t"], dtype=np.int32)
            p._keep = (v, t)
            p.nvert, p.ntri = len(v), len(t)
            p.tri_v, p.tri_t = v.ctypes.data, t.ctypes.data
    return p


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


_PT_KEYS = ("x", "lp", "l0", "F", "be", "V0", "mass", "E", "ys")
_PT_W = {"x": 3, "lp": 3, "l0": 3, "F": 9, "be": 6, "V0": 1, "mass": 1, "E": 1, "ys": 1}


class Model:
    """One oracle model: parameters, material points and the current mesh."""

    def __init__(self, cfg, points=None, body_z=None):
        self.cfg = cfg
        self.params = params_from_cfg(cfg, body_z)
        self.h = lib().o_create(C.byref(self.params))
        if points is not None:
            self.set_points(points)

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.o_free(self.h)
            self.h = None

    def set_points(self, pts):
        arrs = [np.ascontiguousarray(pts[k], dtype=np.float64) for k in _PT_KEYS]
        self._keep = arrs
        n = arrs[0].shape[0]
        lib().o_set_points(self.h, n, *[_ptr(a) for a in arrs])

    def set_body_z(self, z):
        lib().o_set_body_z(self.h, z)

    def set_velocity(self, v):
        v = np.ascontiguousarray(v, dtype=np.float64).reshape(-1, 3)
        assert len(v) == self.counts()["npts"] or len(v) == self._keep[0].shape[0]
        lib().o_set_velocity(self.h, _ptr(v))

    def velocity(self):
        n = self.counts()["npts"]
        v = np.zeros((n, 3))
        lib().o_get_velocity(self.h, _ptr(v))
        return v

    def body_state(self):
        out = [np.zeros(3) for _ in range(4)]
        lib().o_get_body(self.h, *[_ptr(a) for a in out])
        return dict(pose=out[0], v=out[1], w=out[2], theta=out[3])

    def assemble_body(self, du, q, load=1.0, tangent=True):
        """Residual and Jacobian of the material and the rigid body's
        equations at the increments (du, q): R, K (blocks), Rb (6), Kbb (6x6),
        Kgb (6, 3 ndof) = dR/dq, Kbg (6, 3 ndof) = dRb/du."""
        c = self.counts()
        n3 = 3 * c["ndof"]
        du = np.ascontiguousarray(du, dtype=np.float64).reshape(n3)
        q = np.ascontiguousarray(q, dtype=np.float64).reshape(6)
        R = np.zeros(n3)
        fi = np.zeros(n3 + 2)
        K = np.zeros((max(c["nnzb"], 1), 3, 3)) if tangent else None
        reac, Rb, Kbb = np.zeros(3), np.zeros(6), np.zeros((6, 6))
        Kgb, Kbg = np.zeros((6, n3)), np.zeros((6, n3))
        st = lib().o_assemble_body(self.h, _ptr(du), _ptr(q), load, _ptr(R),
                                   _ptr(K) if tangent else None, _ptr(fi), _ptr(reac), _ptr(Rb),
                                   _ptr(Kbb), _ptr(Kgb), _ptr(Kbg))
        if st:
            raise RuntimeError("oracle assemble status %d" % st)
        return dict(R=R, K=K[: c["nnzb"]] if tangent else None, fint=fi[:n3], fextc_norm=fi[n3],
                    finert_norm=fi[n3 + 1], reaction=reac, Rb=Rb, Kbb=Kbb, Kgb=Kgb, Kbg=Kbg)

    def counts(self):
        c = Counts()
        lib().o_counts_get(self.h, C.byref(c))
        return {n: getattr(c, n) for n, _ in Counts._fields_}

    def points(self):
        n = self.counts()["npts"]
        out = {k: np.zeros((n, _PT_W[k])) if _PT_W[k] > 1 else np.zeros(n) for k in _PT_KEYS}
        lib().o_get_points(self.h, *[_ptr(out[k]) for k in _PT_KEYS])
        return out

    def build(self, nosplit=False):
        st = lib().o_build(self.h, int(nosplit))
        if st:
            raise RuntimeError("oracle build failed with status %d" % st)
        return self.counts()

    def tree(self):
        c = self.counts()
        lev = np.zeros(c["nleaf"], np.int32)
        anc = np.zeros((c["nleaf"], 3), np.int32)
        lib().o_export_tree(self.h, _ptr(lev), _ptr(anc))
        return lev, anc

    def nodes(self):
        c = self.counts()
        n = c["nnode"]
        coord = np.zeros((n, 3), np.int32)
        hang = np.zeros(n, np.int32)
        dof = np.zeros(n, np.int32)
        cptr = np.zeros(n + 1, np.int32)
        # constraint lists: at most 16 per node
        cidx = np.zeros(16 * n + 1, np.int32)
        cw = np.zeros(16 * n + 1)
        lib().o_export_nodes(self.h, _ptr(coord), _ptr(hang), _ptr(dof), _ptr(cptr), _ptr(cidx),
                             _ptr(cw))
        m = cptr[-1]
        return dict(coord=coord, hang=hang, dof=dof, cptr=cptr, cidx=cidx[:m].copy(),
                    cw=cw[:m].copy())

    def support(self):
        n = self.counts()["npts"]
        nsup = np.zeros(n, np.int32)
        sidx = np.zeros((n, MAXS), np.int32)
        S = np.zeros((n, MAXS))
        dS = np.zeros((n, MAXS, 3))
        lib().o_export_support(self.h, _ptr(nsup), _ptr(sidx), _ptr(S), _ptr(dS))
        return nsup, sidx, S, dS

    def pattern(self):
        c = self.counts()
        rp = np.zeros(c["ndof"] + 1, np.int32)
        col = np.zeros(max(c["nnzb"], 1), np.int32)
        lib().o_export_pattern(self.h, _ptr(rp), _ptr(col))
        return rp, col[: c["nnzb"]]

    def ghost(self):
        c = self.counts()
        kg = np.zeros(max(c["nnzb"], 1))
        lib().o_export_ghost(self.h, _ptr(kg))
        return kg[: c["nnzb"]]

    def ghost_faces(self):
        c = self.counts()
        f = np.zeros((max(c["nghost"], 1), 4), np.int32)
        pop = np.zeros(c["nleaf"], np.int32)
        lib().o_export_ghost_faces(self.h, _ptr(f), _ptr(pop))
        return f[: c["nghost"]], pop

    def bcmask(self):
        c = self.counts()
        m = np.zeros(max(c["ndof"], 1), np.int32)
        lib().o_export_bcmask(self.h, _ptr(m))
        return m[: c["ndof"]]

    def eval_background(self, x):
        idx = np.zeros(MAXS, np.int32)
        phi = np.zeros(MAXS)
        dphi = np.zeros((MAXS, 3))
        n = C.c_int(0)
        xx = np.ascontiguousarray(x, dtype=np.float64)
        st = lib().o_eval_background(self.h, _ptr(xx), C.byref(n), _ptr(idx), _ptr(phi),
                                     _ptr(dphi))
        if st:
            raise RuntimeError("eval_background status %d" % st)
        k = n.value
        return idx[:k].copy(), phi[:k].copy(), dphi[:k].copy()

    def assemble(self, du, load=1.0, tangent=True):
        c = self.counts()
        n3 = 3 * c["ndof"]
        du = np.ascontiguousarray(du, dtype=np.float64).reshape(n3)
        R = np.zeros(n3)
        fi = np.zeros(n3 + 2)
        K = np.zeros((max(c["nnzb"], 1), 3, 3)) if tangent else None
        reac = np.zeros(3)
        st = lib().o_assemble(self.h, _ptr(du), load, _ptr(R), _ptr(K) if tangent else None,
                              _ptr(fi), _ptr(reac))
        if st:
            raise RuntimeError("oracle assemble status %d" % st)
        return dict(R=R, K=K[: c["nnzb"]] if tangent else None, fint=fi[:n3], fextc_norm=fi[n3],
                    reaction=reac)

    def solve(self, K, b, tol=1e-13, maxit=100000):
        c = self.counts()
        n3 = 3 * c["ndof"]
        K = np.ascontiguousarray(K, dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        x = np.zeros(n3)
        its = C.c_int(0)
        st = lib().o_solve(self.h, _ptr(K), _ptr(b), _ptr(x), tol, maxit, C.byref(its))
        if st:
            raise RuntimeError("oracle solve status %d" % st)
        return x, its.value

    def point_stress(self, du):
        n = self.counts()["npts"]
        sig = np.zeros((n, 3, 3))
        du = np.ascontiguousarray(du, dtype=np.float64)
        st = lib().o_point_stress(self.h, _ptr(du), _ptr(sig))
        if st:
            raise RuntimeError("oracle stress status %d" % st)
        return sig

    def step(self, load=1.0, tol=1e-12, maxit=30, lin_tol=1e-13, lin_maxit=100000):
        sp = StepParams(load, tol, maxit, lin_tol, lin_maxit)
        ss = StepStats()
        lib().o_step(self.h, C.byref(sp), C.byref(ss))
        nh = ss.newton_its + 1
        if ss.status:  # the whole history of a step that did not converge
            h = np.array(ss.res_hist[: min(maxit + 1, 64)])
            nh = int(np.max(np.nonzero(h)[0], initial=0)) + 1
        return dict(status=ss.status, newton_its=ss.newton_its, lin_its=ss.lin_its_total,
                    res_hist=np.array(ss.res_hist[:nh]),
                    eta_hist=np.array(ss.eta_hist[: ss.newton_its]),
                    reaction=np.array(ss.reaction[:]), body_q=np.array(ss.body_q[:]))


def constitutive(cfg, E, ys, be_n, dF, tangent=True):
    """Per-point Hencky + return map update; returns tau (3x3), b_e (6), A (81) and the
    plastic flag (0 elastic, 1 return, 2 apex)."""
    p = params_from_cfg(cfg)
    be = np.ascontiguousarray(be_n, dtype=np.float64)
    dFa = np.ascontiguousarray(dF, dtype=np.float64).reshape(9)
    tau = np.zeros(9)
    ben = np.zeros(6)
    A = np.zeros(81)
    pl = C.c_int(0)
    st = lib().o_constitutive(C.byref(p), E, ys, _ptr(be), _ptr(dFa), _ptr(tau), _ptr(ben),
                              _ptr(A) if tangent else None, C.byref(pl))
    if st:
        raise RuntimeError("constitutive status %d" % st)
    return tau.reshape(3, 3), ben, A.reshape(3, 3, 3, 3), pl.value


def eig_sym3(a):
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(9)
    lam = np.zeros(3)
    Q = np.zeros(9)
    lib().o_eig_sym3(_ptr(a), _ptr(lam), _ptr(Q))
    return lam, Q.reshape(3, 3)


def body_sdf(cfg, x, body_z=None):
    """Signed distance of the rigid body at points x (n, 3): (phi, n, H, inside)."""
    p = params_from_cfg(cfg, body_z)
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    k = len(x)
    phi, nv, H = np.zeros(k), np.zeros((k, 3)), np.zeros((k, 3, 3))
    ins = np.zeros(k, dtype=bool)
    f, nn, hh = C.c_double(), np.zeros(3), np.zeros(9)
    for i in range(k):
        xi = np.ascontiguousarray(x[i])
        ins[i] = bool(lib().o_body_sdf(C.byref(p), _ptr(xi), C.cast(C.byref(f), C.c_void_p),
                                       _ptr(nn), _ptr(hh)))
        phi[i], nv[i], H[i] = f.value, nn, hh.reshape(3, 3)
    return phi, nv, H, ins

