// Device-side definitions shared by the solver's translation units.
//
// Populations are stored as deviations from the rest equilibrium,
// f'_i = f_i - w_i rho0, in the storage type T (float or double); the
// arithmetic runs in T as well.  Geometric decisions (node classes, donor
// triangles and cells) are taken in FP64 with explicitly rounded operations
// (__dadd_rn, __dmul_rn, ...) so that they never depend on FMA contraction.
#pragma once
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "hlbm.h"

namespace hk {

// ---------------------------------------------------------------- D2Q9
// Sec. 3: D2Q9 lattice, c_s^2 = 1/3.
__host__ __device__ __forceinline__ constexpr int cx_of(int i) {
    return (i == 1 || i == 5 || i == 8) ? 1 : (i == 3 || i == 6 || i == 7) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int cy_of(int i) {
    return (i == 2 || i == 5 || i == 6) ? 1 : (i == 4 || i == 7 || i == 8) ? -1 : 0;
}
__host__ __device__ __forceinline__ constexpr int opp_of(int i) {
    return i == 0 ? 0 : (i <= 4 ? ((i + 1) % 4) + 1 : ((i - 3) % 4) + 5);
}
template <typename T>
__host__ __device__ __forceinline__ constexpr T w_of(int i) {
    return i == 0 ? T(4) / T(9) : (i <= 4 ? T(1) / T(9) : T(1) / T(36));
}

// Explicitly rounded operations: the compiler contracts a * b + c into a
// fused multiply-add at its discretion, and its choice may differ between
// kernels that inline the same helper; these leave it none, so that a
// helper gives the same bits in every kernel that calls it.
__device__ __forceinline__ float add_rn(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double add_rn(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float sub_rn(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double sub_rn(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float fma_rn(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double fma_rn(double a, double b, double c) { return __fma_rn(a, b, c); }

// Sums over c_i without the zero terms.  IEEE arithmetic does not let the
// compiler drop 0 * x (x may be infinite or NaN), so the components of c_i
// are applied by selection: acc + c_ix v, acc + c_iy v and c_i . (x, y)
// give the same numbers as the products by 0 and +-1 (up to the sign of a
// zero) in fewer instructions.  i is a compile-time constant wherever these
// are called in unrolled loops, so the selections fold away.
template <typename T>
__device__ __forceinline__ T add_cx(int i, T acc, T v) {
    return cx_of(i) > 0 ? add_rn(acc, v) : (cx_of(i) < 0 ? sub_rn(acc, v) : acc);
}
template <typename T>
__device__ __forceinline__ T add_cy(int i, T acc, T v) {
    return cy_of(i) > 0 ? add_rn(acc, v) : (cy_of(i) < 0 ? sub_rn(acc, v) : acc);
}
template <typename T>
__device__ __forceinline__ T cdot(int i, T x, T y) {
    if (cx_of(i) == 0) return cy_of(i) == 0 ? T(0) : (cy_of(i) > 0 ? y : -y);
    const T ax = cx_of(i) > 0 ? x : -x;
    return cy_of(i) == 0 ? ax : (cy_of(i) > 0 ? add_rn(ax, y) : sub_rn(ax, y));
}

enum : int8_t { CLS_DISC = 0, CLS_INTERP = 1, CLS_UNUSED = 2 };

// Polls of a neighbour tile's progress counter before an FV wait gives up
// (with the kernels' short sleeps between polls: well under a second), sets
// HLBM_ST_SYNC_TIMEOUT and the abort flag, and returns.
constexpr long kSpinLimit = 1L << 23;

// patch node record: f'[9], q[6], pad
constexpr int kRec = 16;

// FV matrix entry of row P: column k, g_Pk and C_Pk (S_ik = c_i . g_Pk)
template <typename T>
struct alignas(4 * sizeof(T)) Coef {
    int32_t col;
    T gx, gy, c;
};
template <>
struct alignas(32) Coef<double> {
    int32_t col;
    int32_t pad;
    double gx, gy, c;
};

// Moments of a deviation set: drho = sum f' (= rho - rho0, kept as its own
// number so that small density changes are not rounded against rho0),
// rho = rho0 + drho, u = (sum f' c) / rho.
template <typename T>
__device__ __forceinline__ void moments_dev(const T (&f)[9], T rho0, T& drho, T& rho, T& ux, T& uy) {
    T r = T(0), jx = T(0), jy = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        r = add_rn(r, f[i]);
        jx = add_cx(i, jx, f[i]);
        jy = add_cy(i, jy, f[i]);
    }
    drho = r;
    rho = add_rn(rho0, r);
    T inv = T(1) / rho;
    ux = mul_rn(jx, inv);
    uy = mul_rn(jy, inv);
}

// Eq. local_eq minus w_i rho0:
// f_i^eq - w_i rho0 = w_i (drho + rho (3 c.u + 4.5 (c.u)^2 - 1.5 u^2))
template <typename T>
__device__ __forceinline__ T feq_dev(int i, T drho, T rho, T ux, T uy) {
    T cu = cdot(i, ux, uy);
    T usq = ux * ux + uy * uy;
    return w_of<T>(i) * (drho + rho * (T(3) * cu + T(4.5) * cu * cu - T(1.5) * usq));
}

// BGK relaxation of a deviation set (eq. LBE's collision with tau_s):
// out_i = f_i - omega (f_i - f_i^eq), with f_i^eq - w_i rho0 = w_i (G +- H)
// for the pair i, opp(i) (c_opp = -c_i): G = drho + rho (4.5 (c.u)^2 -
// 1.5 u^2), H = 3 rho c.u.  The same numbers as feq_dev up to rounding, in
// fewer operations; the relaxation keeps the form that rounds only the
// small non-equilibrium part.  rho0 may be given scaled by a power of two
// together with f.  Explicitly rounded: the lattice is collided by more
// than one kernel, which must agree bit for bit.
template <typename T>
__device__ __forceinline__ void bgk_dev(const T (&f)[9], T rho0, T omega, T (&out)[9]) {
    T dr, r, ux, uy;
    moments_dev(f, rho0, dr, r, ux, uy);
    const T q = mul_rn(T(-1.5), fma_rn(ux, ux, mul_rn(uy, uy)));
    out[0] = fma_rn(-omega, sub_rn(f[0], mul_rn(w_of<T>(0), fma_rn(r, q, dr))), f[0]);
#pragma unroll
    for (int i = 1; i < 9; ++i) {
        if (opp_of(i) < i) continue;  // each pair once, from its lower index
        const int j = opp_of(i);
        const T cu = cdot(i, ux, uy);
        const T G = fma_rn(r, fma_rn(mul_rn(T(4.5), cu), cu, q), dr);
        const T H = mul_rn(r, mul_rn(T(3), cu));
        out[i] = fma_rn(-omega, sub_rn(f[i], mul_rn(w_of<T>(i), add_rn(G, H))), f[i]);
        out[j] = fma_rn(-omega, sub_rn(f[j], mul_rn(w_of<T>(j), sub_rn(G, H))), f[j]);
    }
}

// ---------------------------------------------------------------- layout
struct StepArgs {
    int64_t t;      // time at the start of the step
    double cx, cy;  // lamina centre at y(t)
    double dX, dY;  // displacement of the patch from t-1 to t
    int bx0, by0;   // window of this step (class and new state)
    int pbx0, pby0; // window of the previous step (previous class and state)
    int first;      // 1 at t == 0
    double v0, v1;  // INDUCED motion: lamina velocity at t and t+1
};

// The next lattice step's stream-collide outside a rectangle, run by the
// spare warps of the FV kernel while the FV sub-steps of this step run:
// the nodes outside [ex0, ex1) x [ey0, ey1) (the next step's window with the
// pull margin; ex0, ex1 multiples of 4) pull from src (the post-collision
// state at t+1, written by this step's stream-collide) and write dst, in
// chunks of 64 consecutive nodes of a row taken from the counter *next.
template <typename T>
struct FarArgs {
    const T* src;
    T* dst;
    int ex0, ey0, ex1, ey1;
    int n_seg;      // chunks per row
    int n_chunks;   // 0: no lattice work
    unsigned* next; // zero at the launch
};

template <typename T>
struct Dev {
    // lattice
    int nx, ny, pitch;
    int64_t plane; // pitch * ny
    int bc_x, bc_y;
    int sponge_rows;     // absorbing layer along this lattice's outflow sides (0: none)
    double sponge_sigma;
    T* fA;         // post-collision populations read by this step [9][plane]
    T* fB;         // written by this step
    int store;     // lattice storage: 0 as T, HLBM_F16 or HLBM_BF16 (pointers then hold that type)
    float fscale, finv;  // FP16 storage holds fscale * f'
    // lattice window that follows the patch
    int bw, bh;
    int64_t bplane; // bw * bh
    int8_t* cls_cur;
    const int8_t* cls_prev;
    T* sbox_new;        // pre-collision state at t+1 in the window [9][bplane]
    const T* sbox_old;  // pre-collision state at t in the previous window
    // lamina / fictitious curve
    double half_L, half_T, df2;
    // patch mesh
    int n, ntri, nnz, n_outer, nseg;
    const double* xy;      // [n][2]
    const int8_t* kind;    // [n]
    const int32_t* tri;    // [ntri][3]
    const double* trigeo;  // [ntri][8]: ax ay x1 y1 x2 y2 det pad
    const float* trigrad;  // [ntri][6]: gradients of the three barycentric coordinates
    const int32_t* bstart; // point-location bins (CSR)
    const int32_t* bitems;
    double gbx0, gby0, gbh;
    int gnbx, gnby;
    const int32_t* tstart;  // node -> incident triangles (CSR)
    const int32_t* tlist;
    const int32_t* row_ptr; // FV rows, pivot first
    double* fcontrib;       // per-segment force contributions [nseg][2]
    const int32_t* col;
    const Coef<T>* coef;    // per CSR entry: column, g_Pk (x, y), C_Pk
    // persistent FV kernel: node tiles, neighbour tiles, progress counters
    int n_tiles;
    const int32_t* tile_start;
    const int32_t* tile_nb_ptr;
    const int32_t* tile_nb;
    unsigned long long* progress;
    unsigned* abort_flag;
    long spin_limit;   // polls of a neighbour's counter before the wait gives up
    int stall_tile;    // fault injection: this tile never releases its counter (-1: none)
    // deep tiles (HLBM_FV_DEEP): each tile holds its own nodes and deep_k
    // layers of ghost nodes as local slots and exchanges records with its
    // neighbour tiles once every deep_k sub-steps (see k_fv_deep)
    int deep_k;
    int deep_slot_cap;          // most slots of a tile (own nodes and every ghost layer)
    int deep_ocap;              // most outer nodes among a tile's slots
    const int32_t* deep_ptr;    // [n_tiles + 1]: first slot of each tile in the slot arrays
    const int32_t* deep_cnt;    // [n_tiles][kDeepCnt]: n_a, n_own, n_slot, then the slots computed at block sub-step s
    const int32_t* deep_gid;    // per slot: node id
    const int8_t* deep_send;    // per slot: an own node that other tiles hold as a ghost
    const int32_t* deep_optr;   // [n_tiles + 1]: the tile's outer slots in deep_oslot
    const uint16_t* deep_oslot;
    const int32_t* deep_rptr;   // [n_tiles + 1]: first computed slot of each tile in deep_rows
    const uint32_t* deep_rows;  // per computed slot: its FV row as stored in tensor memory
    // shared-memory tiles: halo node lists, ELL matrices with tile-local
    // columns (own nodes first, then halo), and the nodes other tiles read
    int ell_width;            // entries per row (rows padded)
    int tile_cap, halo_cap;   // largest tile and halo
    const int32_t* halo_ptr;  // [n_tiles + 1]
    const int32_t* halo_ids;  // global node ids
    const Coef<T>* ell;       // tile k: entry (row r, slot j) at ell_width*p0 + j*(p1-p0) + r
    const int8_t* send;       // [n] 1 if some other tile reads the node
    const uint16_t* tile_order; // per tile: local node order, nodes reading no halo first
    const int32_t* tile_interior; // per tile: number of nodes reading no halo
    const int32_t* tile_outer_ptr; // per tile: its outer nodes (CSR over tiles)
    const uint16_t* tile_outer_r;  // tile-local index of each
    int tile_ocap;                 // most outer nodes in one tile
    const int32_t* outer;  // outer node ids [n_outer]
    const int32_t* outer_of; // node -> outer index, -1 elsewhere
    const int32_t* seg_a;  // wall segments
    const int32_t* seg_b;
    const double* seg_n;   // [nseg][2] body-outward normal times length
    // patch state, ping-pong, one record of kRec values per node:
    // f'[0..8] and the moment terms q[0..5] of the equilibrium (see q_of)
    const T* fu_in;
    T* fu_out;
    T* snap;               // outer-node feed [2][12][n_outer]
    int32_t* rtype;
    int32_t* rdonor;
    double* force;         // [cap][2]
    unsigned* status;
    // physics
    T rho0, tau_s, tau_u, inv_tau_u, dt_u, k178, kneq;
    int n_sub;
    int outer_fv;  // outer nodes: 1 adds the FV sums of eq. postcollision2_u
    int motion;
    double A, omega, vx, vy;
};

// ---------------------------------------------------------------- lattice storage
// Element access of lattice storage S holding T values.  ld / st convert
// (FP16 holds fscale * f', fscale = 1024); the raw forms rd / wr2 skip the
// scale: kRawScale is the factor between raw and true values, a power of
// two, so arithmetic on raw values with rho0 scaled by it gives the true
// results scaled exactly.  wr2 writes elements k and k + 1 (k even).
template <typename T, typename S>
struct Store {
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ T ld(const S* p, int64_t i, float) { return p[i]; }
    static __device__ __forceinline__ void st(S* p, int64_t i, T v, float) { p[i] = v; }
    static __device__ __forceinline__ T rd(const S* p, int k) { return p[k]; }
    static __device__ __forceinline__ void wr2(S* p, int k, T a, T b) {
        p[k] = a;
        p[k + 1] = b;
    }
};
template <>
struct Store<float, __half> {
    static constexpr bool kScaled = true;
    static __device__ __forceinline__ float ld(const __half* p, int64_t i, float inv) {
        return __half2float(p[i]) * inv;
    }
    static __device__ __forceinline__ void st(__half* p, int64_t i, float v, float scale) {
        p[i] = __float2half_rn(v * scale);
    }
    static __device__ __forceinline__ float rd(const __half* p, int k) { return __half2float(p[k]); }
    static __device__ __forceinline__ void wr2(__half* p, int k, float a, float b) {
        *reinterpret_cast<__half2*>(p + k) = __floats2half2_rn(a, b);
    }
};
template <>
struct Store<float, __nv_bfloat16> {
    static constexpr bool kScaled = false;
    static __device__ __forceinline__ float ld(const __nv_bfloat16* p, int64_t i, float) {
        return __bfloat162float(p[i]);
    }
    static __device__ __forceinline__ void st(__nv_bfloat16* p, int64_t i, float v, float) {
        p[i] = __float2bfloat16_rn(v);
    }
    static __device__ __forceinline__ float rd(const __nv_bfloat16* p, int k) { return __bfloat162float(p[k]); }
    static __device__ __forceinline__ void wr2(__nv_bfloat16* p, int k, float a, float b) {
        *reinterpret_cast<__nv_bfloat162*>(p + k) = __floats2bfloat162_rn(a, b);
    }
};

// The non-reflecting outflow reading of Sec. 5: the factor 1 - s(d) by which
// the post-collision deviations of node (x, y) are damped, d its distance in
// rows from the nearest outflow side, s(d) = sigma ((N - d)/N)^2; 1 outside
// the layer (and on lattices without one).  Computed in FP64 in the order
// the oracle writes it.
template <typename T>
__device__ __forceinline__ T sponge_keep(const Dev<T>& d, int x, int y) {
    const int rows = d.sponge_rows;
    int dist = rows;
    if (d.bc_y == HLBM_BC_OUTFLOW) dist = min(dist, min(y, d.ny - 1 - y));
    if (d.bc_x == HLBM_BC_OUTFLOW) dist = min(dist, min(x, d.nx - 1 - x));
    if (dist >= rows) return T(1);
    const double t = __ddiv_rn((double)(rows - dist), (double)rows);
    return T(__dsub_rn(1.0, __dmul_rn(__dmul_rn(d.sponge_sigma, t), t)));
}

// Pull of population i at lattice node (x, y) from buffer A with the Sec. 5
// boundaries: half-way bounce-back walls (taking precedence at corners),
// zero-gradient outflow, or periodic wrap.
template <typename T, typename S>
__device__ __forceinline__ T pull_edge(const Dev<T>& d, const S* A, int x, int y, int i) {
    int sx = x - cx_of(i), sy = y - cy_of(i);
    if (sx < 0 || sx >= d.nx) {
        if (d.bc_x == HLBM_BC_PERIODIC)
            sx = (sx + d.nx) % d.nx;
        else if (d.bc_x == HLBM_BC_WALL)
            return Store<T, S>::ld(A, opp_of(i) * d.plane + (int64_t)y * d.pitch + x, d.finv);
        else
            sx = x;
    }
    if (sy < 0 || sy >= d.ny) {
        if (d.bc_y == HLBM_BC_PERIODIC)
            sy = (sy + d.ny) % d.ny;
        else if (d.bc_y == HLBM_BC_WALL)
            return Store<T, S>::ld(A, opp_of(i) * d.plane + (int64_t)y * d.pitch + x, d.finv);
        else
            sy = y;
    }
    return Store<T, S>::ld(A, i * d.plane + (int64_t)sy * d.pitch + sx, d.finv);
}

// ---------------------------------------------------------------- geometry
// Barycentric coordinates of q in triangle k (precomputed ax ay x1 y1 x2 y2 det).
__device__ __forceinline__ void bary_rn(const double* g, double qx, double qy, double& la,
                                        double& lb, double& lc) {
    double px = __dsub_rn(qx, g[0]);
    double py = __dsub_rn(qy, g[1]);
    double x1 = g[2], y1 = g[3], x2 = g[4], y2 = g[5], det = g[6];
    lb = __ddiv_rn(__dsub_rn(__dmul_rn(px, y2), __dmul_rn(x2, py)), det);
    lc = __ddiv_rn(__dsub_rn(__dmul_rn(x1, py), __dmul_rn(px, y1)), det);
    la = __dsub_rn(__dsub_rn(1.0, lb), lc);
}

// Triangle of the body-frame mesh containing q: the candidate with the
// largest smallest barycentric coordinate (>= -1e-12), ties to the lowest
// index; -1 if none.
template <typename T>
__device__ __forceinline__ int locate_dev(const Dev<T>& d, double qx, double qy, double lam[3]) {
    int bi = (int)floor(__ddiv_rn(__dsub_rn(qx, d.gbx0), d.gbh));
    int bj = (int)floor(__ddiv_rn(__dsub_rn(qy, d.gby0), d.gbh));
    if (bi < 0 || bj < 0 || bi >= d.gnbx || bj >= d.gnby) return -1;
    int b = bj * d.gnbx + bi;
    int best = -1;
    double best_min = -1.0e300;
    for (int e = d.bstart[b]; e < d.bstart[b + 1]; ++e) {
        int k = d.bitems[e];
        // FP32 estimate from vertex a: lambda = (1, 0, 0) + grad lambda . (q - a).
        // Its error (a few 1e-6 for any triangle of the bin) is far below the
        // -1e-3 under which a triangle is skipped, so every triangle the exact
        // test below would accept (smallest coordinate >= -1e-12) gets it.
        {
            const double* g = d.trigeo + 8 * (int64_t)k;
            const float* gr = d.trigrad + 6 * (int64_t)k;
            const float px = float(__dsub_rn(qx, g[0])), py = float(__dsub_rn(qy, g[1]));
            const float e0 = 1.0f + fmaf(gr[0], px, gr[1] * py);
            const float e1 = fmaf(gr[2], px, gr[3] * py);
            const float e2 = fmaf(gr[4], px, gr[5] * py);
            if (fminf(e0, fminf(e1, e2)) < -1e-3f) continue;
        }
        double la, lb, lc;
        bary_rn(d.trigeo + 8 * (int64_t)k, qx, qy, la, lb, lc);
        double mn = la < lb ? la : lb;
        if (lc < mn) mn = lc;
        if (mn >= -1e-12 && mn > best_min) {
            best = k;
            best_min = mn;
            lam[0] = la;
            lam[1] = lb;
            lam[2] = lc;
        }
    }
    return best;
}

// locate_dev for the relocated position q of patch node P.  The triangles
// around P (its star) are searched first with the same rule as locate_dev.
// If the best of them holds q with P's own coordinate above 1e-6, q lies
// inside the star away from its outer boundary, where no triangle outside
// the star can come within the 1e-12 tolerance (triangles do not overlap);
// that triangle is then the answer of the full search as well, with the
// same coordinates.  Otherwise the full search runs.
// locate_dev with the candidates of the bin spread over the lanes of a warp
// (all 32 lanes call it with the same point): the same exact test, and the
// same choice (largest smallest coordinate, ties to the earliest candidate,
// i.e. the lowest triangle index).  Every lane returns the result.
template <typename T>
__device__ __forceinline__ int locate_warp(const Dev<T>& d, double qx, double qy, double lam[3]) {
    const int lane = threadIdx.x & 31;
    int bi = (int)floor(__ddiv_rn(__dsub_rn(qx, d.gbx0), d.gbh));
    int bj = (int)floor(__ddiv_rn(__dsub_rn(qy, d.gby0), d.gbh));
    if (bi < 0 || bj < 0 || bi >= d.gnbx || bj >= d.gnby) return -1;
    const int b = bj * d.gnbx + bi;
    int best_e = 0x7fffffff, best = -1;
    double best_min = -1.0e300, l0 = 0, l1 = 0, l2 = 0;
    for (int e = d.bstart[b] + lane; e < d.bstart[b + 1]; e += 32) {
        const int k = d.bitems[e];
        const double* g = d.trigeo + 8 * (int64_t)k;
        const float* gr = d.trigrad + 6 * (int64_t)k;
        const float px = float(__dsub_rn(qx, g[0])), py = float(__dsub_rn(qy, g[1]));
        const float e0 = 1.0f + fmaf(gr[0], px, gr[1] * py);
        const float e1 = fmaf(gr[2], px, gr[3] * py);
        const float e2 = fmaf(gr[4], px, gr[5] * py);
        if (fminf(e0, fminf(e1, e2)) < -1e-3f) continue;  // as in locate_dev
        double la, lb, lc;
        bary_rn(g, qx, qy, la, lb, lc);
        double mn = la < lb ? la : lb;
        if (lc < mn) mn = lc;
        if (mn >= -1e-12 && mn > best_min) {  // lanes see their candidates in increasing e
            best_min = mn;
            best_e = e;
            best = k;
            l0 = la;
            l1 = lb;
            l2 = lc;
        }
    }
    for (int off = 16; off > 0; off >>= 1) {
        const double om = __shfl_xor_sync(0xffffffffu, best_min, off);
        const int oe = __shfl_xor_sync(0xffffffffu, best_e, off);
        const int ok = __shfl_xor_sync(0xffffffffu, best, off);
        const double o0 = __shfl_xor_sync(0xffffffffu, l0, off);
        const double o1 = __shfl_xor_sync(0xffffffffu, l1, off);
        const double o2 = __shfl_xor_sync(0xffffffffu, l2, off);
        if (om > best_min || (om == best_min && oe < best_e)) {
            best_min = om;
            best_e = oe;
            best = ok;
            l0 = o0;
            l1 = o1;
            l2 = o2;
        }
    }
    lam[0] = l0;
    lam[1] = l1;
    lam[2] = l2;
    return best;
}

template <typename T>
__device__ __forceinline__ int locate_from_node(const Dev<T>& d, int P, double qx, double qy, double lam[3]) {
    int best = -1, best_slot = 0;
    double best_min = -1.0e300;
    // q = x_P + (dx, dy): an FP32 estimate of the coordinates, lambda_j =
    // [j == P] + grad lambda_j . (dx, dy), discards triangles clearly not
    // holding q (estimate below -1e-5, far beyond its ~1e-7 error); the
    // others take the exact FP64 test
    const float dx = float(__dsub_rn(qx, d.xy[2 * P])), dy = float(__dsub_rn(qy, d.xy[2 * P + 1]));
    if constexpr (sizeof(T) == 4) {
        // FP32 populations: when a single star triangle survives the estimate
        // and holds q clearly inside (every estimate above 1e-5), the exact
        // test can only accept it, so its decision is taken without FP64;
        // the estimates serve as the (FP32) interpolation weights
        int count = 0, k1 = -1, slot1 = 0;
        float m1 = 0.f, est[3] = {0.f, 0.f, 0.f};
        for (int i = d.tstart[P]; i < d.tstart[P + 1] && count < 2; ++i) {
            const int k = d.tlist[i];
            const int32_t* v = d.tri + 3 * k;
            const int slot = v[0] == P ? 0 : (v[1] == P ? 1 : 2);
            const float* gr = d.trigrad + 6 * (int64_t)k;
            const float l0 = fmaf(gr[0], dx, gr[1] * dy) + (slot == 0 ? 1.0f : 0.0f);
            const float l1 = fmaf(gr[2], dx, gr[3] * dy) + (slot == 1 ? 1.0f : 0.0f);
            const float l2 = fmaf(gr[4], dx, gr[5] * dy) + (slot == 2 ? 1.0f : 0.0f);
            const float mn = fminf(l0, fminf(l1, l2));
            if (mn < -1e-5f) continue;
            if (++count == 1) {
                k1 = k;
                slot1 = slot;
                m1 = mn;
                est[0] = l0;
                est[1] = l1;
                est[2] = l2;
            }
        }
        if (count == 1 && m1 > 1e-5f && est[slot1] > 1e-5f) {
            lam[0] = est[0];
            lam[1] = est[1];
            lam[2] = est[2];
            return k1;
        }
    }
    for (int e = d.tstart[P]; e < d.tstart[P + 1]; ++e) {
        int k = d.tlist[e];
        const int32_t* v = d.tri + 3 * k;
        const int slot = v[0] == P ? 0 : (v[1] == P ? 1 : 2);
        const float* gr = d.trigrad + 6 * (int64_t)k;
        float l0 = fmaf(gr[0], dx, gr[1] * dy) + (slot == 0 ? 1.0f : 0.0f);
        float l1 = fmaf(gr[2], dx, gr[3] * dy) + (slot == 1 ? 1.0f : 0.0f);
        float l2 = fmaf(gr[4], dx, gr[5] * dy) + (slot == 2 ? 1.0f : 0.0f);
        if (fminf(l0, fminf(l1, l2)) < -1e-5f) continue;
        double la, lb, lc;
        bary_rn(d.trigeo + 8 * (int64_t)k, qx, qy, la, lb, lc);
        double mn = la < lb ? la : lb;
        if (lc < mn) mn = lc;
        if (mn >= -1e-12 && mn > best_min) {
            best = k;
            best_min = mn;
            lam[0] = la;
            lam[1] = lb;
            lam[2] = lc;
            best_slot = slot;
        }
    }
    if (best >= 0 && lam[best_slot] > 1e-6) return best;
    return locate_dev(d, qx, qy, lam);
}

// Inside the fictitious curve: squared distance to the lamina rectangle
// below delta_f^2 (Sec. 4).
template <typename T>
__device__ __forceinline__ bool inside_curve(const Dev<T>& d, int x, int y, double cx, double cy) {
    double qx = __dsub_rn(fabs(__dsub_rn((double)x, cx)), d.half_L);
    double qy = __dsub_rn(fabs(__dsub_rn((double)y, cy)), d.half_T);
    if (qx < 0.0) qx = 0.0;
    if (qy < 0.0) qy = 0.0;
    return __dadd_rn(__dmul_rn(qx, qx), __dmul_rn(qy, qy)) < d.df2;
}

// ------------------------------------------------------- nested levels
// The coupling of a lattice level with the next coarser one: the coarser
// level's sizes and the layout of its population buffers ([9][plane] with
// row pitch `pitch`, same storage type as every level), its node under the
// finer level's node (0, 0), and the rescaling of post-collision f^neq from
// coarse to fine (acf) and fine to coarse (afc).
struct Refine {
    int nxc, nyc, pitch;
    int64_t plane;
    int ox, oy;
    double acf, afc;
};

// ---------------------------------------------------------------- launchers
template <typename T> void launch_init_struct(const Dev<T>& d, const double* rho, const double* ux,
                                              const double* uy, double u0x, double u0y,
                                              cudaStream_t s);
template <typename T> void launch_init_box(const Dev<T>& d, int bx0, int by0, const double* rho,
                                           const double* ux, const double* uy, double u0x,
                                           double u0y, cudaStream_t s);
template <typename T> void launch_classify(const Dev<T>& d, const StepArgs& a, cudaStream_t s);
template <typename T> void launch_fill(const Dev<T>& d, const StepArgs& a, cudaStream_t s);
template <typename T> void launch_stream_collide(const Dev<T>& d, const StepArgs& a, cudaStream_t s);
template <typename T>
void launch_stream_collide_rect(const Dev<T>& d, const StepArgs& a, int x0, int y0, int x1, int y1, cudaStream_t s);
template <typename T> int launch_sponge(const Dev<T>& d, cudaStream_t s);
template <typename T> void launch_struct_macro(const Dev<T>& d, double* rho, double* ux, double* uy,
                                               cudaStream_t s);
// One coupling launch: the fine ring (into ring_dst) from coarse buffer c0
// (c1 = NULL) or the mean of c0 and c1; when rsrc is set, also the coarse
// nodes strictly inside the box (into rdst) from fine buffer rsrc, with the
// classes of the window at (bx0, by0).
struct Couple {
    const void* c0;
    const void* c1;
    void* ring_dst;
    const void* rsrc;
    void* rdst;
    int bx0, by0;
};
template <typename T> void launch_couple(const Dev<T>& d, const Refine& r, const Couple& c, cudaStream_t s);
template <typename T> void launch_fv_coeffs(const Dev<T>& d, int lumped, Coef<T>* coef, cudaStream_t s);
template <typename T> void launch_patch_init(const Dev<T>& d, const StepArgs& a, cudaStream_t s);
template <typename T> void launch_refill(const Dev<T>& d, const StepArgs& a, cudaStream_t s);
template <typename T> void launch_feed(const Dev<T>& d, const StepArgs& a, cudaStream_t s);
template <typename T> int fv_tile_capacity();
template <typename T> cudaError_t launch_fv_persistent(const Dev<T>& d, const StepArgs& a, cudaStream_t s);
template <typename T> size_t fv_smem_bytes(int tile_cap, int halo_cap, int roff, int n_sub, int ocap);
template <typename T> int fv_tile_max();  // nodes per tile of the shared-memory FV kernel
template <typename T> void launch_build_ell(const Coef<T>* coef, const int32_t* src, const int32_t* col, Coef<T>* ell,
                                            int64_t count, cudaStream_t s);
template <typename T> int fv_smem_tile_capacity(size_t smem);
template <typename T> cudaError_t launch_fv_smem(const Dev<T>& d, const StepArgs& a, cudaStream_t s);
// deep tiles (temporal blocking): rows with at most 7 off-diagonal entries, Dirichlet outer nodes
constexpr int kTmemMaxEntries = 7;  // off-diagonal entries a row may have in the TMEM and deep kernels
constexpr int kDeepMaxK = 4;  // most sub-steps between exchanges
constexpr int kDeepCnt = 3 + kDeepMaxK;
template <typename T> int fv_deep_tmem_slots();          // computed slots a tile may have
template <typename T> int fv_deep_row_words();           // words of one row image
template <typename T> size_t fv_deep_smem_bytes(int slot_cap, int n_sub, int ocap);
template <typename T> int fv_deep_tile_capacity(size_t smem);
template <typename T>
cudaError_t launch_fv_deep(const Dev<T>& d, const StepArgs& a, const FarArgs<T>* far, cudaStream_t s);
// row images of the computed slots from the CSR matrices: slot i takes row
// gid[i] with its off-diagonal entries' columns mapped to local slots lcol[i * 7 + j]
template <typename T> void launch_build_deep_rows(const Dev<T>& d, const int32_t* gid, const int32_t* lcol,
                                                  int64_t count, uint32_t* rows, cudaStream_t s);
// tensor-memory FV kernel: rows with at most 7 off-diagonal entries, Dirichlet outer nodes
template <typename T> size_t fv_tmem_smem_bytes(int tile_cap, int halo_cap, int n_sub, int ocap);
template <typename T> int fv_tmem_tile_capacity(size_t smem);
template <typename T> cudaError_t launch_fv_tmem(const Dev<T>& d, const StepArgs& a, cudaStream_t s);
// several solvers' FV sub-steps in one launch of the tensor-memory kernel
constexpr int kFvPackMax = 16;
template <typename T>
struct FvPack {
    int n;                   // items
    int block0[kFvPackMax];  // first block of each item (its tile 0)
    Dev<T> d[kFvPackMax];
    StepArgs a[kFvPackMax];
    T* g0[kFvPackMax];       // record buffers: sub-step m reads g0 when m is even
    T* g1[kFvPackMax];
};
template <typename T> cudaError_t launch_fv_tmem_pack(const FvPack<T>& pk, int blocks, size_t smem, cudaStream_t s);
template <typename T> void launch_force(const Dev<T>& d, int64_t t_out, cudaStream_t s);  // 2 launches
template <typename T> void launch_patch_macro(const Dev<T>& d, double* rho, double* ux, double* uy,
                                              double* f9, cudaStream_t s);
void launch_gamma_sums(const double* force, int64_t t0, int64_t t1, double omega, double* out,
                       cudaStream_t s);
// adjoint of one lattice step (decisions held fixed); adjoints in the
// population type T, parameter sums (par, lY, lV) in FP64
template <typename T> void launch_adj_force(const Dev<T>& d, double lamF, T* lP, cudaStream_t s);
template <typename T> cudaError_t launch_adj_fv(const Dev<T>& d, const StepArgs& a, T* sub, const T* lPn, T* x0,
                                                T* x1, T* psi, const int32_t* tpos, T* lsnap, double* par,
                                                double* lV, T* lPm, cudaStream_t s);
template <typename T> void launch_adj_feed(const Dev<T>& d, const StepArgs& a, const T* lsnap, T* lSo, T* lSn,
                                           double* lY, cudaStream_t s);
template <typename T> void launch_adj_stream(const Dev<T>& d, const StepArgs& a, const T* lfB, const T* lSn, T* lfA,
                                             double* par, cudaStream_t s);
template <typename T> void launch_adj_fill(const Dev<T>& d, const StepArgs& a, T* lfA, T* lP, double* par, double* lY,
                                           cudaStream_t s);
template <typename T> void launch_adj_refill(const Dev<T>& d, const StepArgs& a, const T* lPm, T* lP0, T* lSo,
                                             double* par, double* lY, cudaStream_t s);
void launch_gamma_resid(const double* force, int64_t t0, int64_t t1, double omega, double a,
                        double b, double* out, cudaStream_t s);

}  // namespace hk
