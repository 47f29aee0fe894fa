"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module generates problem inputs only -- lamina geometry, body-fitted
triangular patch meshes, initial density fields and the parameter sets of the
named workloads.  It holds none of the method's arithmetic (no equilibrium, no
streaming, no interpolation, no finite-volume coefficients): both the CUDA
library and the CPU oracle receive these arrays and derive everything else on
their own.

Problem parameters follow Sec. 2 of the paper: a rigid lamina of chord L and
thickness T oscillating as y(t) = A sin(wt); eps = A/L, KC = 2*pi*eps,
beta = w L^2 / (2 pi nu), Re = 2 pi beta eps.  Lattice units: dx = dt = 1,
rho0 = 1, c_s^2 = 1/3 (Sec. 3).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, asdict

import numpy as np

# motion kinds (shared enum values with the C-ABI header)
MOTION_STATIC = 0
MOTION_HARMONIC = 1
MOTION_UNIFORM = 2
MOTION_INDUCED = 3
MOTION_HARMONIC_X = 4  # the lamina moves along its chord, x(t) = A sin(w t) (Stokes-layer test case)
# boundary kinds for the Cartesian domain sides
BC_WALL = 0
BC_OUTFLOW = 1
BC_PERIODIC = 2
# node kinds of the patch mesh (Sec. 4: interior = discretization,
# outer boundary = interpolation, wall = lamina surface)
KIND_INTERIOR = 0
KIND_OUTER = 1
KIND_WALL = 2


# --------------------------------------------------------------------------
# seeded noise: SplitMix64 (Steele, Lea, Flood 2014), vectorised
# --------------------------------------------------------------------------
_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(seed: int, index: np.ndarray) -> np.ndarray:
    """SplitMix64 output for state = seed + (index+1)*golden_gamma (mod 2^64)."""
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + (index.astype(np.uint64) + np.uint64(1)) * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return z


def uniform01(seed: int, n: int) -> np.ndarray:
    """n doubles in [0, 1): top 53 bits of SplitMix64 times 2^-53."""
    z = splitmix64(seed, np.arange(n, dtype=np.uint64))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def initial_density(nx: int, ny: int, rho0: float, noise_amp: float, seed: int) -> np.ndarray:
    """rho(x, 0) = rho0 + noise_amp * (2U - 1), U ~ SplitMix64(seed, node index).

    Row-major [ny][nx] float64.  The flow starts at rest (u = 0)."""
    if noise_amp == 0.0:
        return np.full((ny, nx), rho0, dtype=np.float64)
    u = uniform01(seed, nx * ny).reshape(ny, nx)
    return rho0 + noise_amp * (2.0 * u - 1.0)


# --------------------------------------------------------------------------
# body-fitted O-ring mesh around the lamina rectangle
# --------------------------------------------------------------------------
def layer_offsets(n_layers: int, h1: float, d_out: float) -> np.ndarray:
    """Offsets d_0 = 0 < d_1 = h1 < ... < d_{n-1} = d_out, geometric growth."""
    m = n_layers - 1
    if m < 1:
        raise ValueError("need at least two layers")
    if m == 1:
        return np.array([0.0, d_out])
    if abs(h1 * m - d_out) < 1e-12 * d_out:
        return np.linspace(0.0, d_out, n_layers)

    def total(r):
        return h1 * m if abs(r - 1.0) < 1e-14 else h1 * (r ** m - 1.0) / (r - 1.0)

    lo, hi = (1e-6, 1.0) if h1 * m > d_out else (1.0, 4.0)
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if total(mid) > d_out:
            hi = mid
        else:
            lo = mid
    r = 0.5 * (lo + hi)
    d = np.concatenate([[0.0], h1 * np.cumsum(r ** np.arange(m))])
    d[-1] = d_out
    return d


@dataclass
class PatchMesh:
    xy: np.ndarray        # [n_nodes, 2] float64, body frame (origin = lamina centre)
    tri: np.ndarray       # [n_tris, 3] int32, counter-clockwise
    kind: np.ndarray      # [n_nodes] int8 (KIND_*)
    layer: np.ndarray     # [n_nodes] int32 (0 = wall layer)

    @property
    def n_nodes(self) -> int:
        return int(self.xy.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tri.shape[0])


def _layer_nodes(a, b, d, n_L, n_T, n_c, Q):
    """Nodes of the closed curve at offset d from the rectangle [-a,a]x[-b,b],
    counter-clockwise, with an unrolled key used to zip neighbouring layers.

    Sides (bottom, right, top, left) keep n_L / n_T segments; each rounded
    corner carries n_c arc segments.  At d == 0 the four corners are single
    nodes."""
    sides = [  # start point of the side on the rectangle, direction, outward normal, length, segments
        ((-a, -b), (1.0, 0.0), (0.0, -1.0), 2 * a, n_L),
        ((a, -b), (0.0, 1.0), (1.0, 0.0), 2 * b, n_T),
        ((a, b), (-1.0, 0.0), (0.0, 1.0), 2 * a, n_L),
        ((-a, b), (0.0, -1.0), (-1.0, 0.0), 2 * b, n_T),
    ]
    corners = [(a, -b, -0.5 * math.pi), (a, b, 0.0), (-a, b, 0.5 * math.pi), (-a, -b, math.pi)]
    pts, keys = [], []
    u0 = 0.0
    for s, (p0, t, nrm, length, nseg) in enumerate(sides):
        if d == 0.0:
            # corner node shared with the previous side: key in the middle of
            # the previous corner's range
            for k in range(nseg):
                if k == 0:
                    pts.append(p0)
                    keys.append(u0 - 0.5 * Q if s > 0 else 4 * Q + 4 * a + 4 * b - 0.5 * Q)
                else:
                    pts.append((p0[0] + t[0] * length * k / nseg, p0[1] + t[1] * length * k / nseg))
                    keys.append(u0 + length * k / nseg)
        else:
            for k in range(nseg + 1):
                s_k = length * k / nseg if nseg > 0 else 0.0
                pts.append((p0[0] + t[0] * s_k + d * nrm[0], p0[1] + t[1] * s_k + d * nrm[1]))
                keys.append(u0 + s_k)
        u0 += length
        if d > 0.0:
            cx, cy, th0 = corners[s]
            for m in range(1, n_c):
                th = th0 + 0.5 * math.pi * m / n_c
                pts.append((cx + d * math.cos(th), cy + d * math.sin(th)))
                keys.append(u0 + Q * m / n_c)
        u0 += Q
    pts = np.asarray(pts, dtype=np.float64)
    keys = np.asarray(keys, dtype=np.float64)
    order = np.argsort(keys, kind="stable")
    return pts[order], keys[order], u0


def _zip_layers(inner_idx, inner_key, outer_idx, outer_key, period):
    """Triangulate the ring between two closed node sequences sorted by key.

    Walks both sequences together, always advancing the one whose next node
    has the smaller key (ties advance the inner one)."""
    ni, no = len(inner_idx), len(outer_idx)
    tris = []
    if ni == 1:
        for o in range(no):
            tris.append((inner_idx[0], outer_idx[o], outer_idx[(o + 1) % no]))
        return tris
    o0 = int(np.argmin(np.abs(outer_key - inner_key[0])))
    orot = np.concatenate([outer_idx[o0:], outer_idx[:o0]])
    ko = np.concatenate([outer_key[o0:], outer_key[:o0] + period])
    ko = np.concatenate([ko, [ko[0] + period]])
    ki = np.concatenate([inner_key, [inner_key[0] + period]])
    i = o = 0
    while i < ni or o < no:
        if o == no or (i < ni and ki[i + 1] <= ko[o + 1]):
            tris.append((inner_idx[i % ni], orot[o % no], inner_idx[(i + 1) % ni]))
            i += 1
        else:
            tris.append((inner_idx[i % ni], orot[o % no], orot[(o + 1) % no]))
            o += 1
    return tris


def lamina_mesh(L: float, T: float, n_L: int, n_T: int, n_layers: int, h1: float, d_out: float,
                arc_ratio: float = 1.0) -> PatchMesh:
    """O-ring triangular mesh around the rectangle L x T (Sec. 2, Sec. 4).

    Layer 0 is the lamina surface (wall nodes), the last layer the outer
    boundary (interpolation nodes), the rest interior (discretization) nodes.
    Layer j lies at offset d_j (rounded-rectangle offset curve).  Straight
    sides keep n_L / n_T segments on every layer; each corner arc of layer j
    gets about (pi/2) d_j / (arc_ratio * (d_j - d_{j-1})) segments.  With
    L = T = 0 the mesh is a filled disk (a centre node, no wall)."""
    d = layer_offsets(n_layers, h1, d_out)
    a, b = 0.5 * L, 0.5 * T
    disk = (L == 0.0 and T == 0.0)
    if disk:
        n_L = n_T = 0
    Q = 0.5 * math.pi * d_out  # unrolled key length given to each corner
    xy_parts, kind_parts, layer_parts, tris = [], [], [], []
    prev = None
    base = 0
    for j, dj in enumerate(d):
        if j == 0:
            if disk:
                pts, keys = np.zeros((1, 2)), np.zeros(1)
            else:
                pts, keys, period = _layer_nodes(a, b, 0.0, n_L, n_T, 0, Q)
        else:
            dr = dj - d[j - 1]
            n_c = max(1, int(round(0.5 * math.pi * dj / (arc_ratio * dr))))
            if disk:
                n_c = max(n_c, 2)
            pts, keys, period = _layer_nodes(a, b, dj, n_L, n_T, n_c, Q)
        n = len(pts)
        idx = np.arange(base, base + n)
        if j == 0:
            k = KIND_INTERIOR if disk else KIND_WALL
        elif j == len(d) - 1:
            k = KIND_OUTER
        else:
            k = KIND_INTERIOR
        xy_parts.append(pts)
        kind_parts.append(np.full(n, k, dtype=np.int8))
        layer_parts.append(np.full(n, j, dtype=np.int32))
        if prev is not None:
            per = 4 * Q + 4 * a + 4 * b
            tris += _zip_layers(prev[0], prev[1], idx, keys, per)
        prev = (idx, keys)
        base += n
    xy = np.concatenate(xy_parts)
    tri = np.asarray(tris, dtype=np.int32)
    # orient counter-clockwise
    p0, p1, p2 = xy[tri[:, 0]], xy[tri[:, 1]], xy[tri[:, 2]]
    area2 = (p1[:, 0] - p0[:, 0]) * (p2[:, 1] - p0[:, 1]) - (p2[:, 0] - p0[:, 0]) * (p1[:, 1] - p0[:, 1])
    neg = area2 < 0
    tri[neg] = tri[neg][:, [0, 2, 1]]
    return PatchMesh(xy=xy, tri=tri, kind=np.concatenate(kind_parts), layer=np.concatenate(layer_parts))


# --------------------------------------------------------------------------
# workloads
# --------------------------------------------------------------------------
@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    L: float                 # lamina chord (lattice units)
    T: float                 # lamina thickness
    xc: float                # lamina centre at t = 0
    yc: float
    tau_s: float             # structured relaxation time
    n_sub: int               # FV sub-steps per structured step (dt_s = n dt_u)
    motion: int              # MOTION_*
    A: float = 0.0
    omega: float = 0.0
    vx: float = 0.0
    vy: float = 0.0
    delta_f: float = 2.0     # fictitious-curve offset from the lamina
    bc_x: int = BC_WALL
    bc_y: int = BC_OUTFLOW
    dtype: str = "f64"
    steps: int = 0
    rho0: float = 1.0
    noise_amp: float = 0.0
    seed: int = 0
    u0x: float = 0.0         # initial uniform velocity (tests only; 0 in the paper's setup)
    u0y: float = 0.0
    lumped: int = 0          # 1: lumped collision matrix C = identity
    outer_fv: int = 0        # 1: outer nodes take eq. 182 with its FV sums
    fv_kernel: int = 0       # CUDA FV kernel: 0 automatic, 1 global, 2 shared-memory, 3 tensor-memory, 4 deep tiles
    # INDUCED motion: m y'' + c y' + k y = F_y (per unit length), y(0) = y0, y'(0) = v0
    mass: float = 1.0
    stiffness: float = 0.0
    damping: float = 0.0
    y0: float = 0.0
    v0: float = 0.0
    # nested lattice levels: entry k-1 = (nx, ny, ox, oy) of level k, a lattice
    # of twice the spacing of level k-1 (level 0 is the nx x ny lattice) that
    # holds level k-1's node (0, 0) at its node (ox, oy); every level inside
    # another has odd sizes, and bc_x, bc_y belong to the coarsest
    levels: list = field(default_factory=list)
    # absorbing layer along the outflow sides of the lattice carrying the
    # domain boundary (the coarsest level): rows deep, strength at the
    # boundary row; 0 rows = the plain zero-gradient outflow
    sponge_rows: int = 0
    sponge_sigma: float = 0.0
    mesh_args: dict = field(default_factory=dict)

    def mesh(self) -> PatchMesh:
        return lamina_mesh(self.L, self.T, **self.mesh_args)

    def rho_init(self) -> np.ndarray:
        return initial_density(self.nx, self.ny, self.rho0, self.noise_amp, self.seed)

    @property
    def period(self) -> float:
        return 2.0 * math.pi / self.omega if self.omega > 0 else float("inf")

    def as_dict(self) -> dict:
        return asdict(self)


def harmonic_params(L: float, KC: float, beta: float, tau: float | None = None, vmax: float = 0.025):
    """(A, omega, tau_s) for a lamina of chord L at (KC, beta) (Sec. 2).

    With tau given: nu = (tau - 1/2)/3, omega = 2 pi nu beta / L^2.
    Otherwise the peak lamina speed A omega is fixed to vmax (the paper's
    value, Sec. 5): omega = 2 pi vmax / (KC L), nu = vmax L / (KC beta)."""
    A = KC * L / (2.0 * math.pi)
    if tau is not None:
        nu = (tau - 0.5) / 3.0
        omega = 2.0 * math.pi * nu * beta / (L * L)
    else:
        omega = 2.0 * math.pi * vmax / (KC * L)
        nu = vmax * L / (KC * beta)
        tau = 0.5 + 3.0 * nu
    return A, omega, tau


# the (beta, eps) points of the paper's parametric study (Sec. 2): eps in
# {0.02, 0.03, 0.04, 0.05, 0.075, 0.1}, beta in {20, ..., 300}, the pairs
# inside its harmonic-response limit (eq. betalimit)
PAPER_BETAS = (20.0, 50.0, 100.0, 150.0, 200.0, 250.0, 300.0)
PAPER_EPS = (0.02, 0.03, 0.04, 0.05, 0.075, 0.1)


def paper_points():
    return [(b, e) for b in PAPER_BETAS for e in PAPER_EPS if b < 2.6 * e ** -1.6]


def paper_point_workload(beta: float, eps: float, L: float = 32.0, tau_max: float = 0.8) -> Workload:
    """The validation case at (beta, eps) with chord L (domain 5L, thickness
    L/100, FP64), with the peak lamina speed lowered from 0.02 where needed
    to keep tau_s <= tau_max (small beta and eps otherwise give tau_s > 1,
    where the coupled scheme is unstable under these readings)."""
    KC = 2.0 * math.pi * eps
    nu_max = (tau_max - 0.5) / 3.0
    vmax = min(0.02, nu_max * KC * beta / L)
    A, om, tau = harmonic_params(L, KC, beta, vmax=vmax)
    n = int(5 * L)
    w = Workload(f"paper-{beta:g}-{eps:g}-{L:g}", n, n, L, L / 100.0, 0.5 * n + 0.3, 0.5 * n + 0.2, tau, 50,
                 MOTION_HARMONIC, A=A, omega=om, delta_f=2.0, dtype="f64",
                 mesh_args=dict(n_L=int(2 * L), n_T=2, n_layers=14, h1=0.2, d_out=4.0))
    w.n_sub = stable_substeps(w.mesh(), tau - 0.5, minimum=50)
    w.steps = int(math.floor(4 * w.period)) + 1
    return w


def paper_point_levels_workload(beta: float, eps: float, L: float = 800.0, dtype: str = "f32",
                                tau_max: float = 0.8) -> Workload:
    """The validation case at (beta, eps) on the paper's four structured
    levels (Sec. 5: chord 800, domain 5L x 5L, tau at the finest level at
    most 0.8): boxes of spacing 1, 2 and 4 centred on the lamina, about
    1.25L x 0.5L, 2L x L and 3L x 2L, inside a lattice of spacing 8 over
    the whole domain.  Physics and patch as paper_point_workload."""
    w = paper_point_workload(beta, eps, L, tau_max)
    w.name = f"paper-levels4-{beta:g}-{eps:g}-{L:g}"
    w.dtype = dtype
    odd = lambda v: int(v) // 2 * 2 + 1
    sizes = [(odd(1.25 * L), odd(0.5 * L)), (odd(2.0 * L / 2), odd(1.0 * L / 2)), (odd(3.0 * L / 4), odd(2.0 * L / 4)),
             (int(round(5 * L / 8)), int(round(5 * L / 8)))]
    centre = (2.5 * L + 0.3, 2.5 * L + 0.2)
    # physical position (finest units) of node 0 of each level, the coarsest
    # at 0 and each finer one centred, on a node of the level around it
    origin = [(0.0, 0.0)] * 4
    for k in (2, 1, 0):
        ox = [int(round((centre[c] - (sizes[k][c] - 1) * 2 ** k / 2 - origin[k + 1][c]) / 2 ** (k + 1)))
              for c in (0, 1)]
        origin[k] = tuple(origin[k + 1][c] + ox[c] * 2 ** (k + 1) for c in (0, 1))
        sizes[k] = sizes[k] + tuple(ox)
    w.nx, w.ny = sizes[0][0], sizes[0][1]
    w.xc, w.yc = centre[0] - origin[0][0], centre[1] - origin[0][1]
    w.levels = [(sizes[1][0], sizes[1][1], sizes[0][2], sizes[0][3]),
                (sizes[2][0], sizes[2][1], sizes[1][2], sizes[1][3]),
                (sizes[3][0], sizes[3][1], sizes[2][2], sizes[2][3])]
    return w


def workload(name: str) -> Workload:
    """Named synthetic workloads (sizes of the paper's lamina problem)."""
    if name == "lamina-256-f64":
        # 256^2 lattice, chord 20, thickness chord/50, tau 0.6, beta 500,
        # KC 0.25, ~3k-node patch, 4 periods, FP64
        A, om, tau = harmonic_params(20.0, 0.25, 500.0, tau=0.6)
        w = Workload(name, 256, 256, 20.0, 0.4, 128.3, 128.2, tau, 50, MOTION_HARMONIC, A=A, omega=om,
                     delta_f=2.0, dtype="f64",
                     mesh_args=dict(n_L=78, n_T=2, n_layers=15, h1=0.25, d_out=4.0))
        w.steps = int(round(4 * w.period))
        return w
    if name == "lamina-4096-f32":
        # 4096^2 lattice, chord 128, thickness chord/50, KC 1, beta 1000,
        # tau from beta at peak speed 0.025, ~200k-node patch, FP32,
        # density 1 +/- 1e-6 noise
        A, om, tau = harmonic_params(128.0, 1.0, 1000.0)
        w = Workload(name, 4096, 4096, 128.0, 2.56, 2048.3, 2048.2, tau, 64, MOTION_HARMONIC, A=A, omega=om,
                     delta_f=3.0, dtype="f32", noise_amp=1e-6, seed=0,
                     mesh_args=dict(n_L=835, n_T=10, n_layers=100, h1=0.1, d_out=10.0))
        w.steps = int(round(20 * w.period))
        return w
    if name == "lamina-small-f32":
        # small FP32 parity case: ragged lattice 203x157, chord 24
        A, om, tau = harmonic_params(24.0, 0.5, 100.0, vmax=0.025)
        w = Workload(name, 203, 157, 24.0, 0.48, 101.3, 78.2, tau, 24, MOTION_HARMONIC, A=A, omega=om,
                     delta_f=2.0, dtype="f32", noise_amp=1e-6, seed=7,
                     mesh_args=dict(n_L=60, n_T=2, n_layers=12, h1=0.2, d_out=4.0))
        w.steps = 200
        return w
    if name == "lamina-1024-gradient":
        # the gradient case: 1024^2, chord 32, thickness chord/50, KC 0.5, beta 800,
        # peak speed 0.025 (tau_s 0.506), n = 96, FP32, 4 periods (2560 steps)
        A, om, tau = harmonic_params(32.0, 0.5, 800.0, vmax=0.025)
        w = Workload(name, 1024, 1024, 32.0, 0.64, 512.3, 512.2, tau, 96, MOTION_HARMONIC, A=A, omega=om,
                     delta_f=2.0, dtype="f32",
                     mesh_args=dict(n_L=64, n_T=2, n_layers=15, h1=0.25, d_out=4.0))
        w.steps = int(round(4 * w.period))
        return w
    if name == "lamina-small-f64":
        w = workload("lamina-small-f32")
        w.name, w.dtype = name, "f64"
        return w
    if name.startswith("lamina-small-refined-"):
        # the small case's 203x157 lattice as a fine box inside a 204x160
        # coarse lattice of twice the spacing (box at coarse node (51, 40))
        w = workload("lamina-small-f32")
        w.name, w.dtype = name, name.split("-")[-1]
        w.levels = [(204, 160, 51, 40)]
        return w
    if name.startswith("lamina-small-levels3-"):
        # the small case's lattice inside two coarser levels (spacings 2, 4)
        w = workload("lamina-small-f32")
        w.name, w.dtype = name, name.split("-")[-1]
        w.levels = [(211, 167, 52, 43), (216, 176, 53, 44)]
        return w
    if name == "lamina-4096-levels4-f32":
        # the 4096^2 workload's domain and lamina on the paper's four levels
        # (Sec. 5): 513^2 boxes of spacing 1, 2, 4 (4, 8, 16 chords wide) and
        # a 512^2 lattice of spacing 8 over the whole domain; the lamina
        # centre is at (2048.3, 2048.2) of the whole domain
        w = workload("lamina-4096-f32")
        w.name = name
        w.nx = w.ny = 513
        w.xc, w.yc = 256.3, 256.2
        w.levels = [(513, 513, 128, 128), (513, 513, 128, 128), (512, 512, 128, 128)]
        return w
    if name == "lamina-4096-refined-f32":
        # the 4096^2 workload's domain and lamina on two levels: a 2048^2
        # coarse lattice of spacing 2 with a 1025^2 fine box (8 chords wide)
        # around the lamina; the lamina centre is at (2048.3, 2048.2) in
        # fine units of the whole domain, as in the uniform lattice
        w = workload("lamina-4096-f32")
        w.name = name
        w.nx = w.ny = 1025
        w.xc, w.yc = 512.3, 512.2
        w.levels = [(2048, 2048, 768, 768)]
        return w
    if name.startswith("lamina-1024-levels4-"):
        # the 1024^2 workload's domain on four levels: 129^2 boxes of spacing
        # 1, 2, 4 (4, 8, 16 chords) and a 128^2 lattice of spacing 8
        w = workload("lamina-1024-" + name.split("-")[-1])
        w.name = name
        w.nx = w.ny = 129
        w.xc, w.yc = 64.3, 64.2
        w.levels = [(129, 129, 32, 32), (129, 129, 32, 32), (128, 128, 32, 32)]
        return w
    if name.startswith("lamina-1024-refined-"):
        # the 1024^2 workload's domain on two levels: a 512^2 coarse lattice
        # of spacing 2 with a 257^2 fine box (8 chords wide) around the lamina
        w = workload("lamina-1024-" + name.split("-")[-1])
        w.name = name
        w.nx = w.ny = 257
        w.xc, w.yc = 128.3, 128.2
        w.levels = [(512, 512, 192, 192)]
        return w
    if name.startswith("lamina-1024-"):
        # the physics of the 256^2 FP64 workload (tau 0.6, beta 500, KC 0.25) at
        # 1024^2 with chord 32, thickness chord/50, 4 periods; the suffix names
        # the population storage (f64, f32, f16, bf16)
        dtype = name.split("-")[-1]
        A, om, tau = harmonic_params(32.0, 0.25, 500.0, tau=0.6)
        w = Workload(name, 1024, 1024, 32.0, 0.64, 512.3, 512.2, tau, 50, MOTION_HARMONIC, A=A, omega=om,
                     delta_f=2.0, dtype=dtype,
                     mesh_args=dict(n_L=64, n_T=2, n_layers=15, h1=0.25, d_out=4.0))
        w.steps = int(round(4 * w.period))
        return w
    if name.startswith("validation-"):
        # paper point (beta, eps) at chord L, domain 5L x 5L (Sec. 5)
        # name: validation-<beta>-<eps>-<L>
        _, beta, eps, L = name.split("-")
        beta, eps, L = float(beta), float(eps), float(L)
        KC = 2.0 * math.pi * eps
        A, om, tau = harmonic_params(L, KC, beta, vmax=0.02)
        n = int(5 * L)
        w = Workload(name, n, n, L, L / 100.0, 0.5 * n + 0.3, 0.5 * n + 0.2, tau, 50, MOTION_HARMONIC,
                     A=A, omega=om, delta_f=2.0, dtype="f64",
                     mesh_args=dict(n_L=int(2 * L), n_T=2, n_layers=14, h1=0.2, d_out=4.0))
        w.n_sub = stable_substeps(w.mesh(), tau - 0.5, minimum=50)
        w.steps = int(math.floor(4 * w.period)) + 1
        return w
    raise KeyError(name)


def min_edge(mesh: PatchMesh) -> float:
    e = np.concatenate([mesh.tri[:, [0, 1]], mesh.tri[:, [1, 2]], mesh.tri[:, [2, 0]]])
    return float(np.linalg.norm(mesh.xy[e[:, 0]] - mesh.xy[e[:, 1]], axis=1).min())


def stable_substeps(mesh: PatchMesh, tau_u: float, minimum: int = 1) -> int:
    """Sub-steps n with dt_u = 1/n below 2 tau_u (Sec. 7) and, with a factor 3
    of margin, below the diffusive limit h^2 / (|c|^2 tau_u) of the explicit
    central-flux FV update on the smallest edge h (|c|^2 = 2, diagonal
    velocities)."""
    h = min_edge(mesh)
    n = max(minimum, int(math.ceil(1.0 / (1.9 * tau_u))), int(math.ceil(3.0 * 2.0 * tau_u / (h * h))))
    return n


def derived(w: Workload) -> dict:
    """Dimensionless groups of Sec. 2 for a harmonic workload."""
    nu = (w.tau_s - 0.5) / 3.0
    eps = w.A / w.L
    beta = w.omega * w.L ** 2 / (2.0 * math.pi * nu) if nu > 0 else float("nan")
    return dict(nu=nu, eps=eps, KC=2 * math.pi * eps, beta=beta, Re=2 * math.pi * beta * eps,
                vmax=w.A * w.omega, tau_u=w.tau_s - 0.5, period=w.period)


def periodic_mesh(nx: int, ny: int, Lx: float, Ly: float, jitter: float = 0.15, seed: int = 1):
    """Doubly periodic triangulation of [0,Lx) x [0,Ly): an nx x ny node grid
    with seeded jitter (fraction of the spacing) and seeded diagonal
    directions.  Returns (xy [n,2], tri [2 nx ny, 3]) with counter-clockwise
    triangles; node (i, j) has index j*nx + i."""
    hx, hy = Lx / nx, Ly / ny
    u = uniform01(seed, 2 * nx * ny + nx * ny).reshape(-1)
    jx = (2.0 * u[: nx * ny] - 1.0) * jitter * hx
    jy = (2.0 * u[nx * ny: 2 * nx * ny] - 1.0) * jitter * hy
    flip = u[2 * nx * ny:] < 0.5
    ii, jj = np.meshgrid(np.arange(nx), np.arange(ny))
    xy = np.stack([(ii.ravel() + 0.5) * hx + jx, (jj.ravel() + 0.5) * hy + jy], axis=1)
    tris = []
    for j in range(ny):
        for i in range(nx):
            a = j * nx + i
            b = j * nx + (i + 1) % nx
            c = ((j + 1) % ny) * nx + (i + 1) % nx
            d = ((j + 1) % ny) * nx + i
            if flip[j * nx + i]:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    return xy, np.asarray(tris, dtype=np.int32)


def sweep_workloads(vmax: float = 0.025):
    """The parametric KC/beta study as 64 independent instances: KC at 8
    log-spaced values in [0.1, 5], beta at 8 log-spaced values in [100, 5000]
    (the paper's study spans beta 20-300 and eps 0.02-0.1, Sec. 2).  Chord
    L = 16 * 2^round(2 log(beta/100) / log 50) in {16, 32, 64}, lattice 32 L,
    thickness L/50, tau from beta at peak speed vmax.  The patch has about
    10k (L 16) to 100k (L 64) nodes, log-interpolated in L; the number of FV
    sub-steps is the smallest stable one (Sec. 7 and the diffusive limit).
    Instances with tau < 0.505 or Re > 2000 are flagged throughput-only."""
    out = []
    for i in range(8):
        kc = 0.1 * 50.0 ** (i / 7.0)
        for j in range(8):
            beta = 100.0 * 50.0 ** (j / 7.0)
            L = 16.0 * 2 ** round(2.0 * math.log(beta / 100.0) / math.log(50.0))
            A, om, tau = harmonic_params(L, kc, beta, vmax=vmax)
            n = int(32 * L)
            target = 10000.0 * (L / 16.0) ** (math.log(10.0) / math.log(4.0))
            s = math.sqrt(8.0 * L / target)  # node spacing giving about `target` nodes
            layers = max(6, int(round(4.0 / s)) + 1)
            w = Workload(f"sweep-kc{kc:.3g}-beta{beta:.4g}", n, n, L, L / 50.0, 0.5 * n + 0.3, 0.5 * n + 0.2, tau, 8,
                         MOTION_HARMONIC, A=A, omega=om, delta_f=2.0, dtype="f32",
                         mesh_args=dict(n_L=max(8, int(round(L / s))), n_T=max(2, int(round(L / 50.0 / s))),
                                        n_layers=layers, h1=4.0 / (layers - 1), d_out=4.0))
            w.n_sub = stable_substeps(w.mesh(), tau - 0.5, minimum=8)
            w.steps = 1000
            re = 2.0 * math.pi * beta * A / L
            w.throughput_only = tau < 0.505 or re > 2000.0
            out.append(w)
    return out
