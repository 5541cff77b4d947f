"""ctypes binding of libmpm_gb300.so (include/mpm.h).

Argument marshalling only: every computation runs in the library's CUDA
kernels.  Device memory is held in torch tensors (passed as raw pointers) and
work is issued on the current torch CUDA stream.  There is no fallback: if the
shared library is missing or fails to load, the import raises.
"""
import atexit
import ctypes as C
import os
import weakref

import numpy as np
import torch

from . import build as _build

MAXS = 64
OK = 0
STATUS = {0: "OK", 1: "ERR_ARG", 2: "ERR_CUDA", 3: "ERR_NEWTON", 4: "ERR_KRYLOV", 5: "ERR_NAN",
          6: "ERR_SUPPORT", 7: "ERR_CAPACITY", 8: "ERR_BALANCE", 9: "ERR_DOMAIN"}
FP64, MIXED = 0, 1

EXPORT = dict(leaf_level=0, leaf_anchor=1, node_coord=2, node_hang=3, node_dof=4, cptr=5, cidx=6,
              cw=7, nsup=8, sidx=9, S=10, dS=11, row_ptr=12, col=13, ghost=14, bcmask=15,
              populated=16, ghost_faces=17, mg_levels=18)

SYMBOLS = ["mpm_create", "mpm_destroy", "mpm_last_error", "mpm_octree_build", "mpm_mesh_free",
           "mpm_mesh_counts", "mpm_mesh_export", "mpm_assemble", "mpm_solve", "mpm_step",
           "mpm_profile", "mpm_profile_read", "mpm_launch_count", "mpm_solve_static",
           "mpm_blocks_export", "mpm_adjoint", "mpm_fp64_peak", "mpm_assemble_body"]


class Domain(C.Structure):
    _fields_ = [("L", C.c_double), ("depth_min", C.c_int), ("depth_max", C.c_int),
                ("nbc", C.c_int), ("bc_axis", C.c_int * 8), ("bc_pos", C.c_double * 8),
                ("bc_mask", C.c_int * 8)]


class Rigid(C.Structure):
    _fields_ = [("kind", C.c_int), ("cx", C.c_double), ("cy", C.c_double), ("z", C.c_double),
                ("r", C.c_double), ("alpha", C.c_double), ("step_d", C.c_double * 3),
                ("ntri", C.c_int), ("nvert", C.c_int), ("tri_v", C.c_void_p), ("tri_t", C.c_void_p),
                ("free", C.c_int), ("mass", C.c_double), ("inertia", C.c_double),
                ("v", C.c_double * 3), ("w", C.c_double * 3)]


class Adapt(C.Structure):
    _fields_ = [("dx_region", C.c_double), ("beta", C.c_double)]


class Material(C.Structure):
    _fields_ = [("model", C.c_int), ("nu", C.c_double), ("phi", C.c_double), ("psi", C.c_double),
                ("g", C.c_double * 3), ("kappa", C.c_double), ("pf", C.c_double),
                ("ghost_on", C.c_int), ("contact_on", C.c_int), ("mu", C.c_double),
                ("pt", C.c_double)]


class PointsT(C.Structure):
    _fields_ = [("count", C.c_int), ("capacity", C.c_int)] + [
        (n, C.c_void_p) for n in ("x", "lp", "l0", "F", "be", "V0", "mass", "E", "ys", "v")]


class MeshInfo(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("nleaf", "nnode", "nhang", "ndof", "nnzb", "nghost", "npts",
                                       "maxs", "ncontact", "maxrow", "nslot")]


class SolveParams(C.Structure):
    _fields_ = [("method", C.c_int), ("precision", C.c_int), ("tol", C.c_double),
                ("maxit", C.c_int), ("inner_tol", C.c_double), ("mg_reuse", C.c_int)]


class SolveStats(C.Structure):
    _fields_ = [("iterations", C.c_int), ("refinements", C.c_int), ("status", C.c_int),
                ("relres", C.c_double)]


class StepParams(C.Structure):
    _fields_ = [("load", C.c_double), ("tol", C.c_double), ("maxit", C.c_int),
                ("lin", SolveParams), ("du_out", C.c_void_p), ("du_capacity", C.c_longlong),
                ("dt", C.c_double)]


class StepStats(C.Structure):
    _fields_ = [(n, C.c_int) for n in ("newton_its", "lin_its", "status", "npts", "ndof", "nnzb")] + [
        ("res_hist", C.c_double * 64), ("eta_hist", C.c_double * 64), ("reaction", C.c_double * 3),
        ("ms_build", C.c_double), ("ms_assemble", C.c_double), ("ms_solve", C.c_double),
        ("ms_update", C.c_double), ("nsrc", C.c_longlong), ("nslot", C.c_longlong),
        ("mg_rows1", C.c_int), ("mg_stencil1", C.c_int), ("npair", C.c_longlong),
        ("body_q", C.c_double * 6), ("body_v", C.c_double * 3), ("body_w", C.c_double * 3)]


class Checkpoint(C.Structure):
    _fields_ = [("pts", PointsT), ("body_z", C.c_double), ("load", C.c_double),
                ("du", C.c_void_p), ("du_len", C.c_longlong)]


class AdjointStats(C.Structure):
    _fields_ = [("status", C.c_int), ("lin_its", C.c_int), ("reaction", C.c_double * 3),
                ("ms_forward", C.c_double), ("ms_backward", C.c_double)]


_lib = None


def lib_path():
    return _build.LIB


def lib():
    """Load libmpm_gb300.so (building it first if it is out of date)."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        vp, i, d = C.c_void_p, C.c_int, C.c_double
        L.mpm_create.argtypes = [C.POINTER(vp), vp]
        L.mpm_destroy.argtypes = [vp]
        L.mpm_last_error.argtypes = [vp]
        L.mpm_last_error.restype = C.c_char_p
        L.mpm_octree_build.argtypes = [vp, C.POINTER(Domain), C.POINTER(Rigid), C.POINTER(Adapt),
                                       C.POINTER(Material), C.POINTER(PointsT), i, C.POINTER(vp)]
        L.mpm_mesh_free.argtypes = [vp]
        L.mpm_mesh_counts.argtypes = [vp, C.POINTER(MeshInfo)]
        L.mpm_mesh_export.argtypes = [vp, i, vp, C.c_size_t]
        L.mpm_assemble.argtypes = [vp, vp, C.POINTER(Material), C.POINTER(Rigid), vp, d, i, vp, vp,
                                   vp, vp]
        L.mpm_solve.argtypes = [vp, vp, C.POINTER(Material), vp, vp, vp, C.POINTER(SolveParams),
                                C.POINTER(SolveStats)]
        L.mpm_step.argtypes = [vp, C.POINTER(Domain), C.POINTER(Rigid), C.POINTER(Adapt),
                               C.POINTER(Material), C.POINTER(PointsT), C.POINTER(StepParams),
                               C.POINTER(StepStats)]
        L.mpm_blocks_export.argtypes = [vp, vp, vp, i, vp]
        L.mpm_solve_static.argtypes = [vp, vp, vp, vp, vp, d, i, C.POINTER(SolveStats)]
        L.mpm_profile.argtypes = [vp, i]
        L.mpm_profile_read.argtypes = [vp, vp, vp]
        L.mpm_launch_count.argtypes = [vp, vp]
        L.mpm_fp64_peak.argtypes = [vp, d, vp, vp]
        L.mpm_assemble_body.argtypes = [vp, vp, C.POINTER(Material), C.POINTER(Rigid), vp, vp, d, d,
                                        i, vp, vp, vp, vp, vp, vp, vp, vp]
        L.mpm_adjoint.argtypes = [vp, C.POINTER(Domain), C.POINTER(Rigid), C.POINTER(Adapt),
                                  C.POINTER(Material), C.POINTER(Checkpoint), i,
                                  C.POINTER(StepParams), vp, vp, vp, C.POINTER(AdjointStats)]
        _lib = L
    return _lib


class MPMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("%s (%d): %s" % (STATUS.get(code, "?"), code, msg))
        self.code = code


# ----------------------------------------------------------------- parameter structs

def domain(cfg):
    d = Domain()
    d.L = cfg["L"]
    d.depth_min, d.depth_max = cfg["depth_min"], cfg["depth_max"]
    d.nbc = len(cfg["bc"])
    for k, (ax, pos, mask) in enumerate(cfg["bc"]):
        d.bc_axis[k], d.bc_pos[k], d.bc_mask[k] = ax, pos, mask
    return d


_TRI = {}  # device copies of triangulated bodies, by the id of their vertex array


def _tri_device(mesh):
    v = mesh["v"]
    hit = _TRI.get(id(v))
    if hit is None or hit[0] is not v:
        tv = torch.as_tensor(np.ascontiguousarray(v, dtype=np.float64), device="cuda").contiguous()
        tt = torch.as_tensor(np.ascontiguousarray(mesh["t"], dtype=np.int32), device="cuda").contiguous()
        hit = (v, tv, tt)
        _TRI[id(v)] = hit
    return hit[1], hit[2]


def rigid(cfg, z=None, state=None):
    """The body of cfg at height z (default its start height); `state`
    (optional dict: pose (3), v (3), w (3)) overrides a free body's pose and
    velocities, which a run of time steps carries from step to step."""
    r = Rigid()
    b = cfg.get("body")
    if b:
        r.kind, r.cx, r.cy = b["kind"], b["cx"], b["cy"]
        r.z = b["z0"] if z is None else z
        r.r, r.alpha = b["r"], b.get("alpha", 0.0)
        d = b.get("step_d", (0.0, 0.0, b.get("dz", 0.0)))
        for k in range(3):
            r.step_d[k] = d[k]
        r.free, r.mass, r.inertia = int(b.get("free", 0)), b.get("mass", 0.0), b.get("inertia", 0.0)
        for k in range(3):
            r.v[k] = b.get("v", (0.0, 0.0, 0.0))[k]
            r.w[k] = b.get("w", (0.0, 0.0, 0.0))[k]
        if state is not None:
            r.cx, r.cy, r.z = [float(x) for x in state["pose"]]
            for k in range(3):
                r.v[k], r.w[k] = float(state["v"][k]), float(state["w"][k])
        if b["kind"] == 3:
            tv, tt = _tri_device(b["mesh"])
            r.nvert, r.ntri = tv.shape[0], tt.shape[0]
            r.tri_v, r.tri_t = tv.data_ptr(), tt.data_ptr()
    return r


def adapt(cfg):
    return Adapt(cfg.get("dx_region", 0.0), cfg.get("beta", 2.0))


def material(cfg):
    m = Material()
    m.model, m.nu, m.phi, m.psi = cfg["model"], cfg["nu"], cfg.get("phi", 0.0), cfg.get("psi", 0.0)
    for k in range(3):
        m.g[k] = cfg["g"][k]
    m.kappa, m.pf = cfg.get("kappa", 10.0), cfg.get("pf", 50.0)
    m.ghost_on, m.contact_on = int(cfg.get("ghost", 1)), int(cfg.get("contact", 1))
    m.mu, m.pt = cfg.get("mu", 0.0), cfg.get("pt", 25.0)
    return m


def _p(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _check_vec(fn, name, t, dtype, n=None):
    """The library cannot see the size or type of a device buffer, so every
    tensor handed to it is checked here: contiguous, `dtype`, exactly `n`
    entries (any number when n is None: the caller passes the count), on the
    current CUDA device."""
    ok = (isinstance(t, torch.Tensor) and t.dtype == dtype and t.is_cuda and
          t.device.index == torch.cuda.current_device() and t.is_contiguous() and
          (n is None or t.numel() == n))
    if not ok:
        got = ("%s %s[%d] on %s%s" % (type(t).__name__, t.dtype, t.numel(), t.device,
                                      "" if t.is_contiguous() else ", not contiguous")
               if isinstance(t, torch.Tensor) else type(t).__name__)
        raise MPMError(1, "%s: %s must be a contiguous %s tensor%s on the current CUDA device "
                          "(got %s)" % (fn, name, dtype, "" if n is None else " of %d entries" % n,
                                        got))


def _k_dtype(precision):
    return torch.float32 if precision == MIXED else torch.float64


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


# ----------------------------------------------------------------- objects

_contexts = weakref.WeakSet()


@atexit.register
def _close_all():
    for c in list(_contexts):
        c.close()


class Context:
    """Library context bound to the current torch CUDA stream.  Meshes made with
    it are freed before it (explicitly, by close(), or at interpreter exit)."""

    def __init__(self, stream=None):
        h = C.c_void_p()
        s = C.c_void_p(stream.cuda_stream) if stream is not None else _stream()
        st = lib().mpm_create(C.byref(h), s)
        if st:
            raise MPMError(st, "mpm_create failed")
        self.h = h
        self.meshes = weakref.WeakSet()
        _contexts.add(self)

    def error(self):
        return lib().mpm_last_error(self.h).decode()

    def check(self, st):
        if st:
            raise MPMError(st, self.error())

    def close(self):
        if self.h:
            for m in list(self.meshes):
                m.h = None  # the library frees them with the context
            lib().mpm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_PT = (("x", 3), ("lp", 3), ("l0", 3), ("F", 9), ("be", 6), ("V0", 1), ("mass", 1), ("E", 1),
       ("ys", 1))


class Points:
    """Caller-owned device point arrays (torch float64 tensors of `capacity`
    rows); with velocity=True (or a "v" entry in pts) also the velocities that
    time steps need."""

    def __init__(self, pts, capacity=None, device="cuda", velocity=False):
        n = len(pts["x"])
        cap = max(n, capacity or n)
        self.count, self.capacity = n, cap
        self.t = {}
        keys = _PT + ((("v", 3),) if velocity or "v" in pts else ())
        for k, w in keys:
            t = torch.zeros((cap, w) if w > 1 else (cap,), dtype=torch.float64, device=device)
            if k in pts:
                t[:n] = torch.as_tensor(np.asarray(pts[k], dtype=np.float64)).reshape(t[:n].shape)
            self.t[k] = t

    def clone(self):
        """A device copy of the first `count` rows with the same capacity."""
        c = Points.__new__(Points)
        c.count, c.capacity = self.count, self.capacity
        c.t = {k: v.clone() for k, v in self.t.items()}
        return c

    def struct(self):
        s = PointsT()
        s.count, s.capacity = self.count, self.capacity
        for k, _ in _PT:
            setattr(s, k, self.t[k].data_ptr())
        s.v = self.t["v"].data_ptr() if "v" in self.t else None
        return s

    def numpy(self):
        n = self.count
        return {k: self.t[k][:n].cpu().numpy().copy() for k in self.t}


class Mesh:
    def __init__(self, ctx, h):
        self.ctx, self.h = ctx, h
        ctx.meshes.add(self)

    def info(self):
        i = MeshInfo()
        self.ctx.check(lib().mpm_mesh_counts(self.h, C.byref(i)))
        return {n: getattr(i, n) for n, _ in MeshInfo._fields_}

    def export(self, what):
        info = self.info()
        nl, nn, nd, nz, P = info["nleaf"], info["nnode"], info["ndof"], info["nnzb"], info["npts"]
        sizes = dict(leaf_level=(nl, np.int32), leaf_anchor=((nl, 3), np.int32),
                     node_coord=((nn, 3), np.int32), node_hang=(nn, np.int32),
                     node_dof=(nn, np.int32), cptr=(nn + 1, np.int32), nsup=(P, np.int32),
                     sidx=((P, MAXS), np.int32), S=((P, MAXS), np.float64),
                     dS=((P, MAXS, 3), np.float64), row_ptr=(nd + 1, np.int32),
                     col=(nz, np.int32), ghost=(nz, np.float64), bcmask=(nd, np.int32),
                     populated=(nl, np.int32), ghost_faces=((info["nghost"], 4), np.int32),
                     mg_levels=((8, 4), np.int32))
        if what in ("cidx", "cw"):
            ncon = int(self.export("cptr")[-1])
            shape, dt = ncon, (np.int32 if what == "cidx" else np.float64)
        else:
            shape, dt = sizes[what]
        out = np.zeros(shape, dtype=dt)
        if out.size:
            self.ctx.check(lib().mpm_mesh_export(self.h, EXPORT[what],
                                                 out.ctypes.data_as(C.c_void_p), out.nbytes))
        return out

    def free(self):
        if self.h and self.ctx.h:
            lib().mpm_mesh_free(self.h)
        self.h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


def octree_build(ctx, cfg, points, body_z=None, nosplit=False, mesh=None):
    """mpm_octree_build: adapt, split, nodes, basis, pattern, ghost for the body pose."""
    s = points.struct()
    h = C.c_void_p(mesh.h.value if isinstance(mesh.h, C.c_void_p) else mesh.h) if mesh else C.c_void_p()
    st = lib().mpm_octree_build(ctx.h, C.byref(domain(cfg)), C.byref(rigid(cfg, body_z)),
                                C.byref(adapt(cfg)), C.byref(material(cfg)), C.byref(s),
                                1 if nosplit else 0, C.byref(h))
    points.count = s.count
    if mesh is None and h.value:
        mesh = Mesh(ctx, h)
    ctx.check(st)
    return mesh


def assemble(ctx, mesh, cfg, du, load=1.0, precision=FP64, tangent=True, body_z=None):
    """mpm_assemble: residual R (and the tangent values) at the increment du."""
    info = mesh.info()
    nd, ns = info["ndof"], info["nslot"]
    _check_vec("assemble", "du", du, torch.float64, 3 * nd)
    R = torch.empty(3 * nd, dtype=torch.float64, device=du.device)
    K = None
    if tangent:
        K = torch.empty(9 * max(ns, 1), dtype=_k_dtype(precision), device=du.device)
    reac = (C.c_double * 3)()
    norms = (C.c_double * 2)()
    st = lib().mpm_assemble(ctx.h, mesh.h, C.byref(material(cfg)), C.byref(rigid(cfg, body_z)),
                            _p(du), load, precision, _p(R), _p(K), reac, norms)
    ctx.check(st)
    return dict(R=R, K=K, reaction=np.array(reac[:]), fint_norm=norms[0], fextc_norm=norms[1])


def assemble_body(ctx, mesh, cfg, du, q, dt, load=1.0, precision=FP64, tangent=True, state=None):
    """mpm_assemble_body: the residual, tangent and a free body's equations of a
    time step at the increments (du, q): R, K, Rb (6), Kbb (6x6), Kgb and Kbg
    (device [6, 3 ndof])."""
    info = mesh.info()
    nd, ns = info["ndof"], info["nslot"]
    _check_vec("assemble_body", "du", du, torch.float64, 3 * nd)
    if len(q) != 6:
        raise MPMError(1, "assemble_body: q must hold 6 values (translation, rotation)")
    R = torch.empty(3 * nd, dtype=torch.float64, device=du.device)
    K = Kgb = Kbg = None
    if tangent:
        K = torch.empty(9 * max(ns, 1), dtype=_k_dtype(precision), device=du.device)
        Kgb = torch.empty((6, 3 * nd), dtype=torch.float64, device=du.device)
        Kbg = torch.empty((6, 3 * nd), dtype=torch.float64, device=du.device)
    qv = (C.c_double * 6)(*[float(v) for v in q])
    reac, norms = (C.c_double * 3)(), (C.c_double * 3)()
    Rb, Kbb = (C.c_double * 6)(), (C.c_double * 36)()
    st = lib().mpm_assemble_body(ctx.h, mesh.h, C.byref(material(cfg)),
                                 C.byref(rigid(cfg, state=state)), _p(du), C.cast(qv, C.c_void_p), dt,
                                 load, precision, _p(R), _p(K), reac, norms, Rb, Kbb, _p(Kgb),
                                 _p(Kbg))
    ctx.check(st)
    return dict(R=R, K=K, reaction=np.array(reac[:]), fint_norm=norms[0], fextc_norm=norms[1],
                finert_norm=norms[2], Rb=np.array(Rb[:]), Kbb=np.array(Kbb[:]).reshape(6, 6),
                Kgb=Kgb, Kbg=Kbg)


def solve(ctx, mesh, cfg, K, rhs, precision=FP64, tol=1e-10, maxit=20000, method=0,
          inner_tol=1e-3, mg_reuse=0):
    """mpm_solve: block-Jacobi PCG, BiCGStab or multigrid PCG / BiCGStab (method 3); FP32
    inner solves inside FP64 refinement when mixed.  K holds mpm_assemble's values for the
    same precision (FP32 when mixed), rhs 3 * ndof doubles."""
    info = mesh.info()
    _check_vec("solve", "K", K, _k_dtype(precision), 9 * max(info["nslot"], 1))
    _check_vec("solve", "rhs", rhs, torch.float64, 3 * info["ndof"])
    x = torch.empty_like(rhs)
    sp = SolveParams(method, precision, tol, maxit, inner_tol, mg_reuse)
    ss = SolveStats()
    st = lib().mpm_solve(ctx.h, mesh.h, C.byref(material(cfg)), _p(K), _p(rhs), _p(x), C.byref(sp),
                         C.byref(ss))
    stats = dict(iterations=ss.iterations, refinements=ss.refinements, status=ss.status,
                 relres=ss.relres)
    ctx.check(st)
    return x, stats


def solve_static(ctx, mesh, K, rhs, tol=1e-10, maxit=20000):
    """mpm_solve_static: FP64 block-Jacobi PCG whose scratch is the library's
    static device array, so the call allocates no device memory.  K must be the
    FP64 values of mpm_assemble (9 * nslot doubles) and rhs 3 * ndof doubles,
    both contiguous on the current CUDA device: the library cannot check the
    size of a device buffer, so they are checked here."""
    info = mesh.info()
    _check_vec("solve_static", "K", K, torch.float64, 9 * max(info["nslot"], 1))
    _check_vec("solve_static", "rhs", rhs, torch.float64, 3 * info["ndof"])
    x = torch.empty_like(rhs)
    ss = SolveStats()
    st = lib().mpm_solve_static(ctx.h, mesh.h, _p(K), _p(rhs), _p(x), tol, maxit, C.byref(ss))
    stats = dict(iterations=ss.iterations, refinements=ss.refinements, status=ss.status,
                 relres=ss.relres)
    ctx.check(st)
    return x, stats


def body_start(cfg):
    """A free body's state at the start of a run: pose, velocity, angular velocity."""
    b = cfg["body"]
    return dict(pose=np.array([b["cx"], b["cy"], b["z0"]], dtype=np.float64),
                v=np.array(b.get("v", (0.0, 0.0, 0.0)), dtype=np.float64),
                w=np.array(b.get("w", (0.0, 0.0, 0.0)), dtype=np.float64),
                theta=np.zeros(3))


def step(ctx, cfg, points, body_z=None, load=1.0, tol=1e-8, maxit=30, lin_tol=1e-8,
         lin_maxit=20000, precision=FP64, method=0, inner_tol=1e-3, check=True, mg_reuse=0,
         du_out=None, dt=0.0, body_state=None):
    """mpm_step: one load step (dt = 0) or Newmark time step (dt > 0); returns
    the statistics.  du_out (optional float64 device tensor) receives the
    converged increment.  body_state (a free body's pose and velocities at
    the step start, see body_start) is advanced in place."""
    if du_out is not None:
        _check_vec("step", "du_out", du_out, torch.float64)
    s = points.struct()
    sp = StepParams(load, tol, maxit, SolveParams(method, precision, lin_tol, lin_maxit, inner_tol,
                                                  mg_reuse),
                    _p(du_out) if du_out is not None else None,
                    du_out.numel() if du_out is not None else 0, dt)
    ss = StepStats()
    st = lib().mpm_step(ctx.h, C.byref(domain(cfg)), C.byref(rigid(cfg, body_z, body_state)),
                        C.byref(adapt(cfg)), C.byref(material(cfg)), C.byref(s), C.byref(sp),
                        C.byref(ss))
    if st == 0 and body_state is not None:
        q = np.array(ss.body_q[:])
        body_state["pose"] = body_state["pose"] + q[:3]
        body_state["theta"] = body_state["theta"] + q[3:]
        body_state["v"] = np.array(ss.body_v[:])
        body_state["w"] = np.array(ss.body_w[:])
    points.count = s.count
    out = dict(status=st, newton_its=ss.newton_its, lin_its=ss.lin_its, npts=ss.npts, ndof=ss.ndof,
               nnzb=ss.nnzb, res_hist=np.array(ss.res_hist[: ss.newton_its + 1]),
               eta_hist=np.array(ss.eta_hist[: ss.newton_its]), reaction=np.array(ss.reaction[:]),
               ms_build=ss.ms_build, ms_assemble=ss.ms_assemble, ms_solve=ss.ms_solve,
               ms_update=ss.ms_update, nsrc=ss.nsrc, nslot=ss.nslot, mg_rows1=ss.mg_rows1,
               mg_stencil1=ss.mg_stencil1, npair=ss.npair, body_q=np.array(ss.body_q[:]),
               body_v=np.array(ss.body_v[:]), body_w=np.array(ss.body_w[:]))
    if check:
        ctx.check(st)
    return out


def fp64_peak(ctx, seconds=1.0):
    """mpm_fp64_peak: measured FP64 FMA throughput (flop/s) and the timed ms."""
    f, ms = C.c_double(), C.c_double()
    ctx.check(lib().mpm_fp64_peak(ctx.h, seconds, C.byref(f), C.byref(ms)))
    return f.value, ms.value


def blocks(ctx, mesh, K, precision=FP64):
    """mpm_blocks_export: stiffness values -> host array [nnzb, 3, 3] in CSR order."""
    info = mesh.info()
    _check_vec("blocks", "K", K, _k_dtype(precision), 9 * max(info["nslot"], 1))
    nz = info["nnzb"]
    out = np.zeros((max(nz, 1), 3, 3))
    ctx.check(lib().mpm_blocks_export(ctx.h, mesh.h, _p(K), precision,
                                      out.ctypes.data_as(C.c_void_p)))
    return out[:nz]


def adjoint(ctx, cfg, checkpoints, w, tol=1e-8, maxit=30, lin_tol=1e-10, lin_maxit=20000,
            method=0, precision=FP64, inner_tol=1e-3, mg_reuse=0):
    """mpm_adjoint: gradient of w . reaction (end of the last step) with respect
    to the per-point E and yield stress of the first checkpoint.

    checkpoints: list of (Points, body_z, load) or (Points, body_z, load, du),
    the state at the start of each step and, optionally, the step's converged
    increment (then the step is not solved again); the Newton settings should
    be those of the forward run.  Returns (dJ_dE, dJ_dys) as device float64
    tensors and the statistics."""
    n = len(checkpoints)
    arr = (Checkpoint * n)()
    for k, ck in enumerate(checkpoints):
        pts, bz, ld = ck[:3]
        du = ck[3] if len(ck) > 3 else None
        if du is not None:
            _check_vec("adjoint", "checkpoint %d's du" % k, du, torch.float64)
        arr[k].pts = pts.struct()
        arr[k].body_z = bz
        arr[k].load = ld
        arr[k].du = _p(du) if du is not None else None
        arr[k].du_len = du.numel() if du is not None else 0
    p0 = checkpoints[0][0]
    dE = torch.zeros(p0.count, dtype=torch.float64, device=p0.t["E"].device)
    dys = torch.zeros_like(dE)
    wv = (C.c_double * 3)(*[float(v) for v in w])
    sp = StepParams(1.0, tol, maxit, SolveParams(method, precision, lin_tol, lin_maxit, inner_tol,
                                                 mg_reuse), None, 0, 0.0)
    st_ = AdjointStats()
    st = lib().mpm_adjoint(ctx.h, C.byref(domain(cfg)), C.byref(rigid(cfg)), C.byref(adapt(cfg)),
                           C.byref(material(cfg)), arr, n, C.byref(sp),
                           C.cast(wv, C.c_void_p), _p(dE), _p(dys), C.byref(st_))
    ctx.check(st)
    stats = dict(lin_its=st_.lin_its, reaction=np.array(st_.reaction[:]),
                 ms_forward=st_.ms_forward, ms_backward=st_.ms_backward)
    return dE, dys, stats
