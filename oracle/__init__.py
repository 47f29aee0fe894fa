"""CPU oracle for the moving-grid hybrid LBM -- TEST INFRASTRUCTURE ONLY.

Plain serial FP64 C (``hlbm_oracle.c``) behind a ctypes wrapper.  Only the
tests, the smoke check and the benchmark's CPU-baseline / reference arm may
import this package; the product path (``paper_2006_13631_gb300``) never does.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hlbm_oracle.c")
_LIB = os.path.join(_HERE, "_build", "libhlbm_oracle.so")

DISC, INTERP, UNUSED = 0, 1, 2
MAX_LEVELS = 4


_LIB_OMP = os.path.join(_HERE, "_build", "libhlbm_oracle_omp.so")


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile the oracle with gcc (-ffp-contract=off): serial, or with
    OpenMP over the node loops (the CPU baseline; the same results)."""
    out = _LIB_OMP if openmp else _LIB
    os.makedirs(os.path.dirname(out), exist_ok=True)
    if force or not os.path.exists(out) or os.path.getmtime(out) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "hlbm_oracle.h"))):
        tmp = out + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-std=c11", "-O2", "-ffp-contract=off", "-fPIC", "-shared"] +
                              (["-fopenmp"] if openmp else []) + ["-o", tmp, _SRC, "-lm"])
        os.replace(tmp, out)
    return out


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int), ("bc_x", C.c_int), ("bc_y", C.c_int),
        ("rho0", C.c_double), ("rho_init", C.POINTER(C.c_double)),
        ("u0x", C.c_double), ("u0y", C.c_double),
        ("ux_init", C.POINTER(C.c_double)), ("uy_init", C.POINTER(C.c_double)), ("tau_s", C.c_double),
        ("L", C.c_double), ("T", C.c_double), ("xc", C.c_double), ("yc", C.c_double),
        ("delta_f", C.c_double),
        ("n_nodes", C.c_int), ("n_tris", C.c_int),
        ("xy", C.POINTER(C.c_double)), ("tri", C.POINTER(C.c_int32)), ("kind", C.POINTER(C.c_int8)),
        ("n_sub", C.c_int), ("lumped", C.c_int), ("motion", C.c_int),
        ("A", C.c_double), ("omega", C.c_double), ("vx", C.c_double), ("vy", C.c_double),
        ("outer_fv", C.c_int),
        ("mass", C.c_double), ("stiffness", C.c_double), ("damping", C.c_double), ("y0", C.c_double),
        ("v0", C.c_double),
        ("n_levels", C.c_int), ("lv_nx", C.c_int * MAX_LEVELS), ("lv_ny", C.c_int * MAX_LEVELS),
        ("lv_ox", C.c_int * MAX_LEVELS), ("lv_oy", C.c_int * MAX_LEVELS),
        ("lv_rho", C.POINTER(C.c_double) * MAX_LEVELS), ("lv_ux", C.POINTER(C.c_double) * MAX_LEVELS),
        ("lv_uy", C.POINTER(C.c_double) * MAX_LEVELS),
        ("sponge_rows", C.c_int), ("sponge_sigma", C.c_double),
    ]


_lib = None
_lib_omp = None


def lib():
    """The serial oracle (what the tests use)."""
    global _lib
    if _lib is None:
        _lib = _declare(C.CDLL(build()))
    return _lib


def lib_omp():
    """The same source built with OpenMP over its node loops (CPU baseline);
    the threads follow OMP_NUM_THREADS, else every host core."""
    global _lib_omp
    if _lib_omp is None:
        _lib_omp = _declare(C.CDLL(build(openmp=True)))
    return _lib_omp


def _declare(L):
    if True:
        P = C.c_void_p
        dp = C.POINTER(C.c_double)
        ip = C.POINTER(C.c_int32)
        L.orc_create.restype = P
        L.orc_create.argtypes = [C.POINTER(_Params)]
        L.orc_destroy.argtypes = [P]
        L.orc_step.argtypes = [P, C.c_int64]
        L.orc_status.argtypes = [P]
        L.orc_time.argtypes = [P]
        L.orc_time.restype = C.c_int64
        for name in ("orc_struct_f", "orc_patch_f"):
            getattr(L, name).argtypes = [P, dp]
        for name in ("orc_struct_macro", "orc_patch_macro"):
            getattr(L, name).argtypes = [P, dp, dp, dp]
        L.orc_level_macro.argtypes = [P, C.c_int, dp, dp, dp]
        L.orc_struct_class.argtypes = [P, C.POINTER(C.c_int8)]
        L.orc_classify_at.argtypes = [P, C.c_int64, C.POINTER(C.c_int8)]
        L.orc_relocate_at.argtypes = [P, C.c_int64, ip, ip]
        L.orc_refill_record.argtypes = [P, ip, ip]
        L.orc_force.argtypes = [P, dp, dp]
        L.orc_gamma.argtypes = [P, C.c_double, C.c_double, dp, dp, dp]
        L.orc_feq.argtypes = [C.c_double, C.c_double, C.c_double, dp]
        L.orc_locate.argtypes = [P, C.c_double, C.c_double, dp]
        L.orc_fv_nnz.argtypes = [P]
        L.orc_fv_coeffs.argtypes = [P, ip, ip, dp, dp, dp, dp]
        L.orc_n_wall_segments.argtypes = [P]
        L.orc_motion_history.argtypes = [P, C.c_int64, dp, dp]
        L.orc_outer_fv.argtypes = [C.c_int, dp, C.c_int, ip, C.POINTER(C.c_int8), C.c_double, C.c_double, C.c_int,
                                   dp, dp, dp]
        L.orc_sine_fit.argtypes = [dp, C.c_int64, C.c_int64, C.c_double, dp, dp, dp]
        L.orc_theta.argtypes = [dp, C.c_int64, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.c_double, dp, dp, dp]
        L.orc_fv_periodic.argtypes = [C.c_int, dp, C.c_int, ip, C.c_double, C.c_double, C.c_double,
                                      C.c_double, C.c_int, C.c_int, dp]
        L.orc_lbgk.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_double, C.c_int, C.c_double, C.c_int, dp]
    return L


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a):
    return a.ctypes.data_as(C.POINTER(C.c_int32))


def feq(rho, ux, uy):
    out = np.zeros(9)
    lib().orc_feq(rho, ux, uy, _dp(out))
    return out


def sine_fit(F, t0, t1, omega):
    F = np.ascontiguousarray(F, dtype=np.float64)
    a, b, r = C.c_double(), C.c_double(), C.c_double()
    lib().orc_sine_fit(_dp(F), t0, t1, omega, C.byref(a), C.byref(b), C.byref(r))
    return a.value, b.value, r.value


def theta(F, rho0, omega, L, A, discard=1.0, fit=3.0):
    """Theta = F-hat / ((pi/4) rho0 w^2 L^2 A) of a force history F[t], t = 0..n-1,
    fitted over [discard, discard + fit] periods (Sec. 2.1)."""
    F = np.ascontiguousarray(F, dtype=np.float64)
    re, im, r = C.c_double(), C.c_double(), C.c_double()
    rc = lib().orc_theta(_dp(F), len(F), rho0, omega, L, A, discard, fit, C.byref(re), C.byref(im), C.byref(r))
    if rc != 0:
        raise ValueError(f"orc_theta failed ({rc})")
    return complex(re.value, im.value), r.value


def fv_periodic(xy, tri, period_x, period_y, tau_u, dt_u, n_iter, f9, lumped=0):
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    f = np.ascontiguousarray(f9, dtype=np.float64).copy()
    lib().orc_fv_periodic(xy.shape[0], _dp(xy), tri.shape[0], _ip(tri), period_x, period_y, tau_u, dt_u,
                          lumped, n_iter, _dp(f))
    return f


def outer_fv(xy, tri, kind, tau_u, dt_u, fin, dstar, lumped=0):
    """R10 alone: the full eq. postcollision2_u value of every outer node
    (other rows of the result are zero)."""
    xy = np.ascontiguousarray(xy, dtype=np.float64)
    tri = np.ascontiguousarray(tri, dtype=np.int32)
    kind = np.ascontiguousarray(kind, dtype=np.int8)
    fin = np.ascontiguousarray(fin, dtype=np.float64)
    dstar = np.ascontiguousarray(dstar, dtype=np.float64)
    out = np.zeros_like(fin)
    lib().orc_outer_fv(xy.shape[0], _dp(xy), tri.shape[0], _ip(tri), kind.ctypes.data_as(C.POINTER(C.c_int8)),
                       tau_u, dt_u, lumped, _dp(fin), _dp(dstar), _dp(out))
    return out


def theta_fd_gradient(w, nsteps, discard=1.0, fit=3.0, rel_step=1e-4, mesh=None, rho_init=None):
    """Theta of workload w and d(Re, Im Theta)/d(A, omega, tau_s) by central
    differences: seven oracle runs (the base point and each parameter moved by
    -/+ rel_step of its value), each fitted (Sec. 2.1) over the same steps
    [ceil(discard T), floor((discard + fit) T)] of the base period, with its
    own omega and A.  Returns (theta complex, grad [3] complex)."""
    import copy

    mesh = mesh if mesh is not None else w.mesh()
    rho = rho_init if rho_init is not None else w.rho_init()
    base = (w.A, w.omega, w.tau_s)
    steps = [rel_step * abs(v) for v in base]
    Tp = 2.0 * math.pi / w.omega
    t0, t1 = int(math.ceil(discard * Tp)), int(math.floor((discard + fit) * Tp))
    th = []
    for i in range(7):
        v = copy.copy(w)
        if i > 0:
            k, sgn = (i - 1) // 2, (-1.0 if i % 2 == 1 else 1.0)
            if k == 0:
                v.A = w.A + sgn * steps[0]
            elif k == 1:
                v.omega = w.omega + sgn * steps[1]
            else:
                v.tau_s = w.tau_s + sgn * steps[2]
        o = Oracle(v, mesh=mesh, rho_init=rho)
        o.step(nsteps)
        _, fy = o.force()
        a, b, _ = sine_fit(fy, t0, t1, v.omega)
        N = 0.25 * math.pi * v.rho0 * v.omega ** 2 * v.L ** 2 * v.A
        th.append(complex(a / N, b / N))
    grad = np.array([(th[2 + 2 * k] - th[1 + 2 * k]) / (2.0 * steps[k]) for k in range(3)])
    return th[0], grad


def theta_tangent(w, nsteps, discard=1.0, fit=3.0, rel_step=1e-6, mesh=None, rho_init=None):
    """The FP64 tangent of Theta in (A, omega, tau_s) along the oracle's branch
    of decisions: for each parameter, two oracle runs at -/+ rel_step of its
    value, stepped in lockstep, must take the same decisions at every step
    (lattice node classes and refill types; a donor triangle may differ only
    where the moved node lies on an edge shared by both, where the
    interpolated value is the same); Theta of each is fitted
    over the base window as in theta_fd_gradient, and the central quotient is
    then the derivative of the map the method is smooth on between decisions,
    to O(rel_step^2) (at 1e-6 relative the truncation and FP64 rounding are
    both far below 1e-6 of the result).  Raises ValueError when a decision
    differs, naming the parameter and step.  Returns (grad [3] complex, the
    number of node-steps whose donor triangles differed at such ties)."""
    import copy

    mesh = mesh if mesh is not None else w.mesh()
    rho = rho_init if rho_init is not None else w.rho_init()
    base = (w.A, w.omega, w.tau_s)
    Tp = 2.0 * math.pi / w.omega
    t0, t1 = int(math.ceil(discard * Tp)), int(math.floor((discard + fit) * Tp))
    grad = []
    ties = 0
    for k, name in enumerate(("A", "omega", "tau_s")):
        h = rel_step * abs(base[k])
        runs = []
        for sgn in (-1.0, 1.0):
            v = copy.copy(w)
            setattr(v, name, base[k] + sgn * h)
            runs.append((v, Oracle(v, mesh=mesh, rho_init=rho)))
        for t in range(nsteps):
            for _, o in runs:
                o.step(1)
            (_, om), (_, op) = runs
            if not np.array_equal(om.struct_class(), op.struct_class()):
                raise ValueError(f"{name}: node classes differ at step {t + 1}")
            tm, dm = om.refill_record()
            tp, dp = op.refill_record()
            if not np.array_equal(tm, tp):
                raise ValueError(f"{name}: refill types differ at step {t + 1}")
            # a node moved onto an edge may take either triangle: the linear
            # interpolants agree there, so the value does not jump
            ties += int((dm != dp).sum())
        th = []
        for v, o in runs:
            _, fy = o.force()
            a, b, _ = sine_fit(fy, t0, t1, v.omega)
            N = 0.25 * math.pi * v.rho0 * v.omega ** 2 * v.L ** 2 * v.A
            th.append(complex(a / N, b / N))
        grad.append((th[1] - th[0]) / (2.0 * h))
    return np.array(grad), ties


def theta_semi_analytic(beta, eps):
    """eq. hydro_tot with eq. hydro_gamma and eq. hydro_delta (Sec. 2.1):
    Theta = 1.02 + 2.45 beta^-1/2 - i (2.49 beta^-1/2 + 0.879 beta^3/4 eps^2)."""
    beta = np.asarray(beta, dtype=np.float64)
    eps = np.asarray(eps, dtype=np.float64)
    return 1.02 + 2.45 * beta ** -0.5 - 1j * (2.49 * beta ** -0.5 + 0.879 * beta ** 0.75 * eps ** 2)


def lbgk(f9, bc_x, bc_y, tau_s, n_iter, sponge_rows=0, sponge_sigma=0.0):
    """n_iter collide-and-stream steps of the plain lattice (Sec. 3, eq. LBE;
    Sec. 5 boundaries; R13's absorbing layer when sponge_rows > 0, rho0 = 1)."""
    f = np.ascontiguousarray(f9, dtype=np.float64).copy()
    _, ny, nx = f.shape
    lib().orc_lbgk(nx, ny, bc_x, bc_y, tau_s, int(sponge_rows), float(sponge_sigma), n_iter, _dp(f))
    return f


class Oracle:
    """Serial FP64 MG-HLBM run for one workload (see ``inputs.Workload``)."""

    def __init__(self, w, mesh=None, rho_init=None, u_init=None, level_u_init=None, level_rho_init=None,
                 openmp=False):
        self.w = w
        self._L = lib_omp() if openmp else lib()
        self.mesh = mesh if mesh is not None else w.mesh()
        rho = rho_init if rho_init is not None else w.rho_init()
        self._keep = [np.ascontiguousarray(rho, dtype=np.float64),
                      np.ascontiguousarray(self.mesh.xy, dtype=np.float64),
                      np.ascontiguousarray(self.mesh.tri, dtype=np.int32),
                      np.ascontiguousarray(self.mesh.kind, dtype=np.int8)]
        p = _Params()
        p.nx, p.ny, p.bc_x, p.bc_y = w.nx, w.ny, w.bc_x, w.bc_y
        p.rho0 = w.rho0
        p.rho_init = _dp(self._keep[0])
        p.u0x, p.u0y = w.u0x, w.u0y
        if u_init is not None:
            self._keep += [np.ascontiguousarray(u_init[0], dtype=np.float64),
                           np.ascontiguousarray(u_init[1], dtype=np.float64)]
            p.ux_init, p.uy_init = _dp(self._keep[-2]), _dp(self._keep[-1])
        p.tau_s = w.tau_s
        p.L, p.T, p.xc, p.yc, p.delta_f = w.L, w.T, w.xc, w.yc, w.delta_f
        p.n_nodes, p.n_tris = self.mesh.n_nodes, self.mesh.n_tris
        p.xy = _dp(self._keep[1])
        p.tri = _ip(self._keep[2])
        p.kind = self._keep[3].ctypes.data_as(C.POINTER(C.c_int8))
        p.n_sub, p.lumped, p.motion = w.n_sub, w.lumped, w.motion
        p.outer_fv = int(getattr(w, "outer_fv", 0))
        p.sponge_rows = int(getattr(w, "sponge_rows", 0))
        p.sponge_sigma = float(getattr(w, "sponge_sigma", 0.0))
        p.mass, p.stiffness, p.damping = float(w.mass), float(w.stiffness), float(w.damping)
        p.y0, p.v0 = float(w.y0), float(w.v0)
        p.A, p.omega, p.vx, p.vy = w.A, w.omega, w.vx, w.vy
        levels = list(getattr(w, "levels", []))
        if len(levels) > MAX_LEVELS:
            raise ValueError(f"at most {MAX_LEVELS} coarser levels")
        p.n_levels = len(levels)
        for k, (nx, ny, ox, oy) in enumerate(levels):
            p.lv_nx[k], p.lv_ny[k], p.lv_ox[k], p.lv_oy[k] = nx, ny, ox, oy
            if level_u_init is not None and level_u_init[k] is not None:
                self._keep += [np.ascontiguousarray(level_u_init[k][0], dtype=np.float64),
                               np.ascontiguousarray(level_u_init[k][1], dtype=np.float64)]
                p.lv_ux[k], p.lv_uy[k] = _dp(self._keep[-2]), _dp(self._keep[-1])
            if level_rho_init is not None and level_rho_init[k] is not None:
                self._keep.append(np.ascontiguousarray(level_rho_init[k], dtype=np.float64))
                p.lv_rho[k] = _dp(self._keep[-1])
        self._h = self._L.orc_create(C.byref(p))
        self.n = self.mesh.n_nodes

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            self._L.orc_destroy(h)
            self._h = None

    def step(self, nsteps=1):
        return self._L.orc_step(self._h, nsteps)

    @property
    def status(self):
        return self._L.orc_status(self._h)

    @property
    def time(self):
        return self._L.orc_time(self._h)

    def struct_f(self):
        out = np.empty((9, self.w.ny, self.w.nx))
        self._L.orc_struct_f(self._h, _dp(out))
        return out

    def struct_macro(self):
        r, ux, uy = (np.empty((self.w.ny, self.w.nx)) for _ in range(3))
        self._L.orc_struct_macro(self._h, _dp(r), _dp(ux), _dp(uy))
        return r, ux, uy

    def level_macro(self, k=1):
        """rho, ux, uy of coarser level k (1..len(w.levels)) at its current time (R12)."""
        nx, ny = self.w.levels[k - 1][:2]
        r, ux, uy = (np.empty((ny, nx)) for _ in range(3))
        self._L.orc_level_macro(self._h, int(k), _dp(r), _dp(ux), _dp(uy))
        return r, ux, uy

    def struct_class(self):
        out = np.empty((self.w.ny, self.w.nx), dtype=np.int8)
        self._L.orc_struct_class(self._h, out.ctypes.data_as(C.POINTER(C.c_int8)))
        return out

    def classify_at(self, t):
        out = np.empty((self.w.ny, self.w.nx), dtype=np.int8)
        self._L.orc_classify_at(self._h, t, out.ctypes.data_as(C.POINTER(C.c_int8)))
        return out

    def relocate_at(self, t):
        ty, d = np.empty(self.n, np.int32), np.empty(self.n, np.int32)
        self._L.orc_relocate_at(self._h, t, _ip(ty), _ip(d))
        return ty, d

    def patch_f(self):
        out = np.empty((self.n, 9))
        self._L.orc_patch_f(self._h, _dp(out))
        return out

    def patch_macro(self):
        r, ux, uy = (np.empty(self.n) for _ in range(3))
        self._L.orc_patch_macro(self._h, _dp(r), _dp(ux), _dp(uy))
        return r, ux, uy

    def refill_record(self):
        t, d = np.empty(self.n, np.int32), np.empty(self.n, np.int32)
        self._L.orc_refill_record(self._h, _ip(t), _ip(d))
        return t, d

    def force(self):
        n = self.time + 1
        fx, fy = np.empty(n), np.empty(n)
        self._L.orc_force(self._h, _dp(fx), _dp(fy))
        return fx, fy

    def motion(self):
        """(y, v) of the lamina at integer times 0..t."""
        n = self.time + 1
        y, v = np.empty(n), np.empty(n)
        self._L.orc_motion_history(self._h, n, _dp(y), _dp(v))
        return y, v

    def gamma(self, discard=1.0, fit=3.0):
        re, im, r = C.c_double(), C.c_double(), C.c_double()
        rc = self._L.orc_gamma(self._h, discard, fit, C.byref(re), C.byref(im), C.byref(r))
        if rc != 0:
            raise ValueError(f"orc_gamma failed ({rc})")
        return re.value, im.value, r.value

    def locate(self, qx, qy):
        lam = np.zeros(3)
        k = self._L.orc_locate(self._h, qx, qy, _dp(lam))
        return k, lam

    def fv_coeffs(self):
        nnz = self._L.orc_fv_nnz(self._h)
        rp = np.empty(self.n + 1, np.int32)
        col = np.empty(nnz, np.int32)
        gx, gy, cc = np.empty(nnz), np.empty(nnz), np.empty(nnz)
        vol = np.empty(self.n)
        self._L.orc_fv_coeffs(self._h, _ip(rp), _ip(col), _dp(gx), _dp(gy), _dp(cc), _dp(vol))
        return rp, col, gx, gy, cc, vol

    @property
    def n_wall_segments(self):
        return self._L.orc_n_wall_segments(self._h)
