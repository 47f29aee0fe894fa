"""Python binding of the C ABI (include/hlbm.h).

The functions below carry the C names and only marshal arguments; every
step of the solver runs in the CUDA library.  PyTorch supplies device memory
(its caching allocator is installed as the library's allocator) and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import _native as N

_callbacks = None


class HLBMError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"hlbm error {code}: {msg}")
        self.code = code


def _check(rc: int, h=None):
    if rc != N.HLBM_OK:
        lib = N.load()
        msg = lib.hlbm_last_error(h).decode() if lib.hlbm_last_error(h) else ""
        raise HLBMError(rc, msg)


def use_torch_allocator():
    """Route the library's device allocations through torch's caching allocator.

    Installed once per process: every solver keeps the callbacks it was created
    with, so they must outlive all solvers (a second install would free the
    first pair under solvers still holding them)."""
    global _callbacks
    if _callbacks is not None:
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(), int(stream or 0))
        except Exception:  # allocation failure is reported to the library as NULL
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _callbacks = (N.ALLOC_FN(_alloc), N.FREE_FN(_free))
    _check(N.load().hlbm_set_allocator(_callbacks[0], _callbacks[1], None))


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double)) if a is not None else None


def _structs(grid: dict, patch: dict, motion: dict):
    """ctypes structs of the inputs and the host arrays they point to, which
    the caller keeps alive for the duration of the call."""
    keep = []

    def arr(x, dt):
        if x is None:
            return None
        a = np.ascontiguousarray(x, dtype=dt)
        keep.append(a)
        return a

    g = N.hlbm_grid_t()
    g.nx, g.ny = int(grid["nx"]), int(grid["ny"])
    g.bc_x, g.bc_y = int(grid.get("bc_x", N.HLBM_BC_WALL)), int(grid.get("bc_y", N.HLBM_BC_OUTFLOW))
    dt = grid.get("dtype", "f32")
    g.dtype = {"f64": N.HLBM_F64, "f32": N.HLBM_F32, "f16": N.HLBM_F16, "bf16": N.HLBM_BF16}.get(dt, dt)
    g.rho0 = float(grid.get("rho0", 1.0))
    g.u0x, g.u0y = float(grid.get("u0x", 0.0)), float(grid.get("u0y", 0.0))
    g.rho_init = _dp(arr(grid.get("rho_init"), np.float64))
    g.ux_init = _dp(arr(grid.get("ux_init"), np.float64))
    g.uy_init = _dp(arr(grid.get("uy_init"), np.float64))
    g.sponge_rows, g.sponge_sigma = int(grid.get("sponge_rows", 0)), float(grid.get("sponge_sigma", 0.0))
    levels = grid.get("levels") or []
    g.n_levels = len(levels)
    if levels:
        lv = (N.hlbm_level_t * len(levels))()
        keep.append(lv)
        for k, L in enumerate(levels):
            lv[k].nx, lv[k].ny, lv[k].ox, lv[k].oy = int(L["nx"]), int(L["ny"]), int(L["ox"]), int(L["oy"])
            lv[k].rho_init = _dp(arr(L.get("rho_init"), np.float64))
            lv[k].ux_init = _dp(arr(L.get("ux_init"), np.float64))
            lv[k].uy_init = _dp(arr(L.get("uy_init"), np.float64))
        g.levels = C.cast(lv, C.POINTER(N.hlbm_level_t))
    p = N.hlbm_patch_t()
    xy, tri, kind = arr(patch["xy"], np.float64), arr(patch["tri"], np.int32), arr(patch["kind"], np.int8)
    p.n_nodes, p.n_tris = xy.shape[0], tri.shape[0]
    p.xy = _dp(xy)
    p.tri = tri.ctypes.data_as(C.POINTER(C.c_int32))
    p.kind = kind.ctypes.data_as(C.POINTER(C.c_int8))
    p.lamina_L, p.lamina_T = float(patch["lamina_L"]), float(patch["lamina_T"])
    p.x_c, p.y_c = float(patch["x_c"]), float(patch["y_c"])
    p.delta_f = float(patch["delta_f"])
    p.n_sub, p.lumped = int(patch["n_sub"]), int(patch.get("lumped", 0))
    p.outer_fv = int(patch.get("outer_fv", 0))
    p.fv_kernel = int(patch.get("fv_kernel", 0))
    m = N.hlbm_motion_t()
    m.kind = int(motion.get("kind", N.HLBM_MOTION_STATIC))
    m.A, m.omega = float(motion.get("A", 0.0)), float(motion.get("omega", 0.0))
    m.vx, m.vy = float(motion.get("vx", 0.0)), float(motion.get("vy", 0.0))
    m.mass = float(motion.get("mass", 1.0))
    m.stiffness, m.damping = float(motion.get("stiffness", 0.0)), float(motion.get("damping", 0.0))
    m.y0, m.v0 = float(motion.get("y0", 0.0)), float(motion.get("v0", 0.0))
    return g, p, m, keep


def hlbm_create(grid: dict, patch: dict, tau_s: float, motion: dict, cuda_stream: int = 0):
    """grid: nx, ny, bc_x, bc_y, dtype ('f64'|'f32'|'f16'|'bf16'), rho0, u0x, u0y, rho_init, ux_init, uy_init,
    and levels: a list of dicts nx, ny, ox, oy, rho_init, ux_init, uy_init (coarser levels, finest first)
    patch: xy [n,2], tri [m,3], kind [n], lamina_L, lamina_T, x_c, y_c, delta_f, n_sub, lumped, outer_fv, fv_kernel
    motion: kind, A, omega, vx, vy, mass, stiffness, damping, y0, v0.  Returns an opaque handle."""
    g, p, m, keep = _structs(grid, patch, motion)
    h = C.c_void_p()
    _check(N.load().hlbm_create(C.byref(g), C.byref(p), float(tau_s), C.byref(m), C.c_void_p(cuda_stream or None),
                                C.byref(h)))
    return h


def hlbm_theta_gradient(grid: dict, patch: dict, tau_s: float, motion: dict, nsteps: int, discard=1.0, fit=3.0,
                        rel_step=1e-4, cuda_stream: int = 0):
    """Theta and d(Re, Im Theta)/d(A, omega, tau_s) by central differences over
    seven solvers stepped as one sweep.  Returns (theta complex, grad [3]
    complex, device ms of the solves)."""
    g, p, m, keep = _structs(grid, patch, motion)
    th, gr, ms = np.zeros(2), np.zeros(6), np.zeros(1)
    _check(N.load().hlbm_theta_gradient(C.byref(g), C.byref(p), float(tau_s), C.byref(m), int(nsteps), float(discard),
                                        float(fit), float(rel_step), C.c_void_p(cuda_stream or None), _dp(th), _dp(gr),
                                        _dp(ms)))
    return complex(th[0], th[1]), gr[0::2] + 1j * gr[1::2], float(ms[0])


def hlbm_theta_adjoint(grid: dict, patch: dict, tau_s: float, motion: dict, nsteps: int, discard=1.0, fit=3.0,
                       w_re=1.0, w_im=0.0, checkpoint_every=256, cuda_stream: int = 0):
    """Theta and the gradient of L = w_re Re Theta + w_im Im Theta in
    (A, omega, tau_s) by the adjoint of the discrete step.  Returns
    (theta complex, grad [3] real, forward ms, reverse ms)."""
    g, p, m, keep = _structs(grid, patch, motion)
    th, gr, fw, bw = np.zeros(2), np.zeros(3), np.zeros(1), np.zeros(1)
    _check(N.load().hlbm_theta_adjoint(C.byref(g), C.byref(p), float(tau_s), C.byref(m), int(nsteps), float(discard),
                                       float(fit), float(w_re), float(w_im), int(checkpoint_every),
                                       C.c_void_p(cuda_stream or None), _dp(th), _dp(gr), _dp(fw), _dp(bw)))
    return complex(th[0], th[1]), gr.copy(), float(fw[0]), float(bw[0])


def theta_function(w, nsteps: int, discard=1.0, fit=3.0, checkpoint_every=256, mesh=None, rho_init=None,
                   cuda_stream: int = 0):
    """A differentiable Theta(A, omega, tau_s) of workload w (HARMONIC motion):
    returns f(params) -> tensor (Re, Im), params a float64 tensor (A, omega,
    tau_s) with requires_grad.  The forward pass steps one solver and fits
    Theta (Sec. 2.1); the backward pass runs the adjoint of the discrete step
    (hlbm_theta_adjoint) with the incoming gradient as the weights of Re and
    Im.  Everything runs in the CUDA library; torch only carries the values."""
    import torch

    mesh = mesh if mesh is not None else w.mesh()
    rho_init = rho_init if rho_init is not None else w.rho_init()

    def inputs_at(params):
        A, om, tau = (float(x) for x in params)
        ww = type(w)(**{k: getattr(w, k) for k in w.__dataclass_fields__})
        ww.A, ww.omega, ww.tau_s = A, om, tau
        grid, patch, motion = workload_inputs(ww, mesh, rho_init)
        return grid, patch, motion, tau

    class _Theta(torch.autograd.Function):
        @staticmethod
        def forward(ctx, params):
            grid, patch, motion, tau = inputs_at(params.detach().cpu())
            h = hlbm_create(grid, patch, tau, motion, cuda_stream)
            try:
                hlbm_step(h, nsteps)
                re, im, _ = hlbm_gamma_window(h, motion["omega"], discard, fit)
            finally:
                hlbm_destroy(h)
            ctx.save_for_backward(params)
            return torch.tensor([re, im], dtype=torch.float64, device=params.device)

        @staticmethod
        def backward(ctx, grad_out):
            (params,) = ctx.saved_tensors
            grid, patch, motion, tau = inputs_at(params.detach().cpu())
            go = grad_out.detach().cpu().double()
            _, gr, _, _ = hlbm_theta_adjoint(grid, patch, tau, motion, nsteps, discard, fit, float(go[0]),
                                             float(go[1]), checkpoint_every, cuda_stream)
            return torch.tensor(gr, dtype=torch.float64, device=params.device)

    return _Theta.apply


def hlbm_gamma_window(h, omega: float, discard: float, fit: float):
    """Theta over [discard, discard + fit] periods of the solver's force history."""
    re, im, rms = C.c_double(), C.c_double(), C.c_double()
    _check(N.load().hlbm_gamma(h, float(discard), float(fit), C.byref(re), C.byref(im), C.byref(rms)), h)
    return re.value, im.value, rms.value


def hlbm_step(h, nsteps: int):
    _check(N.load().hlbm_step(h, int(nsteps)), h)


def hlbm_force(h, first: int, count: int):
    fx, fy = np.empty(count), np.empty(count)
    _check(N.load().hlbm_force(h, int(first), int(count), _dp(fx), _dp(fy)), h)
    return fx, fy


def hlbm_gamma(h, discard_periods: float = 1.0, fit_periods: float = 3.0):
    re, im, rms = C.c_double(), C.c_double(), C.c_double()
    _check(N.load().hlbm_gamma(h, discard_periods, fit_periods, C.byref(re), C.byref(im), C.byref(rms)), h)
    return re.value, im.value, rms.value


def hlbm_info(h):
    info = N.hlbm_info_t()
    _check(N.load().hlbm_info(h, C.byref(info)), h)
    return {k: getattr(info, k) for k, _ in N.hlbm_info_t._fields_}


def hlbm_get_fields(h, nx: int, ny: int, n_nodes: int):
    out = [np.empty((ny, nx)) for _ in range(3)] + [np.empty(n_nodes) for _ in range(3)]
    _check(N.load().hlbm_get_fields(h, *[_dp(o) for o in out]), h)
    return out


def hlbm_get_level_fields(h, level: int, nx: int, ny: int):
    out = [np.empty((ny, nx)) for _ in range(3)]
    _check(N.load().hlbm_get_level_fields(h, int(level), *[_dp(o) for o in out]), h)
    return out


def hlbm_get_class(h, nx: int, ny: int):
    out = np.empty((ny, nx), dtype=np.int8)
    _check(N.load().hlbm_get_class(h, out.ctypes.data_as(C.POINTER(C.c_int8))), h)
    return out


def hlbm_get_refill(h, n_nodes: int):
    t, d = np.empty(n_nodes, np.int32), np.empty(n_nodes, np.int32)
    _check(N.load().hlbm_get_refill(h, t.ctypes.data_as(C.POINTER(C.c_int32)),
                                    d.ctypes.data_as(C.POINTER(C.c_int32))), h)
    return t, d


def hlbm_get_patch_f(h, n_nodes: int):
    out = np.empty((n_nodes, 9))
    _check(N.load().hlbm_get_patch_f(h, _dp(out)), h)
    return out


def hlbm_get_fv(h, n_nodes: int, nnz: int):
    rp, col = np.empty(n_nodes + 1, np.int32), np.empty(nnz, np.int32)
    gx, gy, cc = np.empty(nnz), np.empty(nnz), np.empty(nnz)
    _check(N.load().hlbm_get_fv(h, rp.ctypes.data_as(C.POINTER(C.c_int32)), col.ctypes.data_as(C.POINTER(C.c_int32)),
                                _dp(gx), _dp(gy), _dp(cc)), h)
    return rp, col, gx, gy, cc


def hlbm_status(h) -> int:
    v = C.c_uint32()
    _check(N.load().hlbm_status(h, C.byref(v)), h)
    return v.value


def hlbm_set_fv_depth(h, depth: int):
    _check(N.load().hlbm_set_fv_depth(h, int(depth)), h)


def hlbm_set_overlap(h, enable: bool = True):
    _check(N.load().hlbm_set_overlap(h, int(bool(enable))), h)


def hlbm_set_overlap_share(h, share: float):
    _check(N.load().hlbm_set_overlap_share(h, float(share)), h)


def hlbm_clear_status(h):
    _check(N.load().hlbm_clear_status(h), h)


def hlbm_inject_fault(h, kind: int, arg: int):
    _check(N.load().hlbm_inject_fault(h, int(kind), int(arg)), h)


def hlbm_profile(h, enable: bool):
    _check(N.load().hlbm_profile(h, 1 if enable else 0), h)


def hlbm_profile_read(h):
    ms = np.zeros(len(N.PHASES))
    launches = np.zeros(len(N.PHASES), dtype=np.int64)
    _check(N.load().hlbm_profile_read(h, _dp(ms), launches.ctypes.data_as(C.POINTER(C.c_int64))), h)
    return {p: (float(ms[k]), int(launches[k])) for k, p in enumerate(N.PHASES)}


def hlbm_fit_static(samples_ptr: int, stride: int, t0: int, t1: int, omega: float, cuda_stream: int = 0):
    """Sine fit of device samples without any device allocation (see include/hlbm.h).
    samples_ptr: device address of the samples.  Returns (a, b, rms)."""
    a, b, rms = C.c_double(), C.c_double(), C.c_double()
    rc = N.load().hlbm_fit_static(C.c_void_p(samples_ptr), int(stride), int(t0), int(t1), float(omega),
                                  C.c_void_p(cuda_stream or None), C.byref(a), C.byref(b), C.byref(rms))
    if rc != N.HLBM_OK:
        raise HLBMError(rc, "hlbm_fit_static failed")
    return a.value, b.value, rms.value


def hlbm_destroy(h):
    if h:
        N.load().hlbm_destroy(h)


def hlbm_save(h, path: str):
    _check(N.load().hlbm_save(h, os.fsencode(path)), h)


def hlbm_load(h, path: str):
    _check(N.load().hlbm_load(h, os.fsencode(path)), h)


def workload_inputs(w, mesh=None, rho_init=None, u_init=None, level_u_init=None, level_rho_init=None):
    """(grid, patch, motion) dicts of hlbm_create from a workload description
    (an object with the attributes of ``inputs.Workload``)."""
    mesh = mesh if mesh is not None else w.mesh()
    rho = rho_init if rho_init is not None else w.rho_init()
    grid = dict(nx=w.nx, ny=w.ny, bc_x=w.bc_x, bc_y=w.bc_y, dtype=w.dtype, rho0=w.rho0, u0x=w.u0x,
                u0y=w.u0y, rho_init=rho, sponge_rows=getattr(w, "sponge_rows", 0),
                sponge_sigma=getattr(w, "sponge_sigma", 0.0),
                ux_init=None if u_init is None else u_init[0], uy_init=None if u_init is None else u_init[1])
    levels = list(getattr(w, "levels", []))
    if levels:
        grid["levels"] = [dict(nx=nx, ny=ny, ox=ox, oy=oy,
                               rho_init=None if level_rho_init is None else level_rho_init[k],
                               ux_init=None if level_u_init is None or level_u_init[k] is None else level_u_init[k][0],
                               uy_init=None if level_u_init is None or level_u_init[k] is None else level_u_init[k][1])
                          for k, (nx, ny, ox, oy) in enumerate(levels)]
    patch = dict(xy=mesh.xy, tri=mesh.tri, kind=mesh.kind, lamina_L=w.L, lamina_T=w.T,
                 x_c=w.xc, y_c=w.yc, delta_f=w.delta_f, n_sub=w.n_sub, lumped=w.lumped,
                 outer_fv=getattr(w, "outer_fv", 0), fv_kernel=getattr(w, "fv_kernel", 0))
    motion = dict(kind=w.motion, A=w.A, omega=w.omega, vx=w.vx, vy=w.vy, mass=getattr(w, "mass", 1.0),
                  stiffness=getattr(w, "stiffness", 0.0), damping=getattr(w, "damping", 0.0),
                  y0=getattr(w, "y0", 0.0), v0=getattr(w, "v0", 0.0))
    return grid, patch, motion


class Solver:
    """Convenience owner of one hlbm handle built from a workload description
    (an object with the attributes of ``inputs.Workload``)."""

    def __init__(self, w, mesh=None, rho_init=None, u_init=None, stream: int | None = None, level_u_init=None,
                 level_rho_init=None):
        import torch

        if not torch.cuda.is_available():
            raise RuntimeError("a CUDA device is required")
        if _callbacks is None:
            use_torch_allocator()
        self.w = w
        self.mesh = mesh if mesh is not None else w.mesh()
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        grid, patch, motion = workload_inputs(w, self.mesh, rho_init, u_init, level_u_init, level_rho_init)
        self.h = hlbm_create(grid, patch, w.tau_s, motion, self.stream)
        self.n = self.mesh.n_nodes

    def close(self):
        if getattr(self, "h", None):
            hlbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, nsteps: int = 1):
        hlbm_step(self.h, nsteps)

    def save(self, path: str):
        hlbm_save(self.h, path)

    def load(self, path: str):
        hlbm_load(self.h, path)

    def info(self):
        return hlbm_info(self.h)

    @property
    def time(self):
        return self.info()["time"]

    def force(self):
        t = self.time
        return hlbm_force(self.h, 0, t + 1)

    def gamma(self, discard=1.0, fit=3.0):
        return hlbm_gamma(self.h, discard, fit)

    def fields(self):
        return hlbm_get_fields(self.h, self.w.nx, self.w.ny, self.n)

    def struct_macro(self):
        return tuple(self.fields()[:3])

    def level_macro(self, k: int = 1):
        """rho, ux, uy of coarser level k (1..len(w.levels)) at its current time."""
        nx, ny = self.w.levels[k - 1][:2]
        return tuple(hlbm_get_level_fields(self.h, k, nx, ny))

    def patch_macro(self):
        return tuple(self.fields()[3:])

    def struct_class(self):
        return hlbm_get_class(self.h, self.w.nx, self.w.ny)

    def refill_record(self):
        return hlbm_get_refill(self.h, self.n)

    def patch_f(self):
        return hlbm_get_patch_f(self.h, self.n)

    def fv_coeffs(self):
        return hlbm_get_fv(self.h, self.n, self.info()["nnz"])

    @property
    def status(self):
        return hlbm_status(self.h)

    def profile(self, enable: bool = True):
        hlbm_profile(self.h, enable)

    def profile_read(self):
        return hlbm_profile_read(self.h)


class Sweep:
    """Independent solvers stepped together (hlbm_sweep_*): each instance's
    lattice part on its own stream, the FV sub-steps one instance after
    another on a shared stream.  The solvers stay owned by the caller."""

    def __init__(self, solvers, stream: int | None = None):
        import torch

        self.solvers = list(solvers)
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        arr = (C.c_void_p * len(self.solvers))(*[s.h.value for s in self.solvers])
        self.h = C.c_void_p()
        rc = N.load().hlbm_sweep_create(len(self.solvers), arr, C.c_void_p(self.stream or None), C.byref(self.h))
        if rc != N.HLBM_OK:
            raise HLBMError(rc, "hlbm_sweep_create failed")

    def _check(self, rc):
        if rc != N.HLBM_OK:
            raise HLBMError(rc, N.load().hlbm_sweep_last_error(self.h).decode())

    def step(self, nsteps: int = 1):
        self._check(N.load().hlbm_sweep_step(self.h, int(nsteps)))

    def tune(self, trial_steps: int = 2):
        out = (C.c_int32 * len(self.solvers))()
        self._check(N.load().hlbm_sweep_tune(self.h, int(trial_steps), out))
        return list(out)

    def pack(self, enable: bool = True):
        """Share FV launches between solvers (hlbm_sweep_pack); returns the number of packs."""
        out = C.c_int32()
        self._check(N.load().hlbm_sweep_pack(self.h, int(bool(enable)), C.byref(out)))
        return out.value

    def fv_time(self, nsteps: int = 1):
        out = np.zeros(len(self.solvers))
        self._check(N.load().hlbm_sweep_fv_time(self.h, int(nsteps), _dp(out)))
        return out

    def close(self):
        if getattr(self, "h", None):
            N.load().hlbm_sweep_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
