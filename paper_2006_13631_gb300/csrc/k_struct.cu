// Cartesian-lattice kernels: initial state, node classification (Sec. 4),
// the eq. postcollision2_s feed of interpolation nodes, and the fused pull
// stream-collide of eq. LBE with the Sec. 5 boundaries.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "hlbm_dev.cuh"

namespace hk {

// Lattice storage.  S = T stores f' as is; __half stores fscale * f' (a
// power of two, so the scaling is exact), __nv_bfloat16 stores f'.  The
// arithmetic always runs in T.
// call f.template operator()<S>() with the lattice storage type of d
template <typename T, typename F>
void with_store(const Dev<T>& d, F&& f) {
    if constexpr (sizeof(T) == 4) {
        if (d.store == HLBM_F16) return f.template operator()<__half>();
        if (d.store == HLBM_BF16) return f.template operator()<__nv_bfloat16>();
    }
    f.template operator()<T>();
}

// ------------------------------------------------------------------ init
template <typename T, typename S>
__global__ void k_init_struct(Dev<T> d, const double* rho, const double* ux, const double* uy, double u0x,
                              double u0y) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= d.nx) return;
    int64_t g = (int64_t)y * d.nx + x;
    double r = rho ? rho[g] : double(d.rho0);
    T dr = T(r - double(d.rho0)), rr = T(r);
    T vx = ux ? T(ux[g]) : T(u0x);
    T vy = uy ? T(uy[g]) : T(u0y);
    int64_t s = (int64_t)y * d.pitch + x;
    S* A = reinterpret_cast<S*>(d.fA);
    S* B = reinterpret_cast<S*>(d.fB);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        T v = feq_dev<T>(i, dr, rr, vx, vy);
        Store<T, S>::st(A, i * d.plane + s, v, d.fscale);
        Store<T, S>::st(B, i * d.plane + s, v, d.fscale);
    }
}

template <typename T>
void launch_init_struct(const Dev<T>& d, const double* rho, const double* ux, const double* uy, double u0x,
                        double u0y, cudaStream_t s) {
    dim3 grid((d.nx + 255) / 256, d.ny);
    with_store(d, [&]<typename S>() { k_init_struct<T, S><<<grid, 256, 0, s>>>(d, rho, ux, uy, u0x, u0y); });
}

// pre-collision state at t = 0 inside a window: the initial equilibrium
template <typename T>
__global__ void k_init_box(Dev<T> d, int bx0, int by0, const double* rho, const double* ux, const double* uy,
                           double u0x, double u0y) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= d.bplane) return;
    int x = bx0 + (int)(b % d.bw), y = by0 + (int)(b / d.bw);
    int64_t g = (int64_t)y * d.nx + x;
    double r = rho ? rho[g] : double(d.rho0);
    T dr = T(r - double(d.rho0)), rr = T(r);
    T vx = ux ? T(ux[g]) : T(u0x);
    T vy = uy ? T(uy[g]) : T(u0y);
#pragma unroll
    for (int i = 0; i < 9; ++i) d.sbox_new[i * d.bplane + b] = feq_dev<T>(i, dr, rr, vx, vy);
}

template <typename T>
void launch_init_box(const Dev<T>& d, int bx0, int by0, const double* rho, const double* ux, const double* uy,
                     double u0x, double u0y, cudaStream_t s) {
    k_init_box<T><<<(unsigned)((d.bplane + 255) / 256), 256, 0, s>>>(d, bx0, by0, rho, ux, uy, u0x, u0y);
}

// ------------------------------------------------------- classification
// Sec. 4: discretization outside the fictitious curve, unused inside;
// unused nodes with a discretization node among their 8 lattice
// neighbours are interpolation nodes.  Evaluated on the window that
// follows the patch; every node outside it is a discretization node.
template <typename T>
__global__ void k_classify(Dev<T> d, StepArgs a) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (b >= d.bplane) return;
    int x = a.bx0 + (int)(b % d.bw), y = a.by0 + (int)(b / d.bw);
    int8_t c = CLS_DISC;
    if (inside_curve(d, x, y, a.cx, a.cy)) {
        c = CLS_UNUSED;
#pragma unroll
        for (int i = 1; i < 9; ++i) {
            int xx = x + cx_of(i), yy = y + cy_of(i);
            if (xx < 0 || yy < 0 || xx >= d.nx || yy >= d.ny) continue;
            if (!inside_curve(d, xx, yy, a.cx, a.cy)) {
                c = CLS_INTERP;
                break;
            }
        }
    }
    d.cls_cur[b] = c;
}

template <typename T>
void launch_classify(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    k_classify<T><<<(unsigned)((d.bplane + 127) / 128), 128, 0, s>>>(d, a);
}

// -------------------------------------------- eq. postcollision2_s feed
// Post-collision populations of lattice interpolation nodes (and of nodes
// that just became discretization nodes) from the patch at time t:
// f~ = f^eq,u + 2(tau_s - 1)/(2 tau_s - 1) f^neq,u, with rho, u and f^neq
// barycentric over the enclosing patch triangle.
template <typename T, typename S>
__global__ void k_fill(Dev<T> d, StepArgs a) {
    // one warp per window node: the warp's lanes share the point location
    S* A = reinterpret_cast<S*>(d.fA);
    const int lane = threadIdx.x & 31;
    int64_t b = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    if (b >= d.bplane) return;
    int8_t c = d.cls_cur[b];
    if (c == CLS_UNUSED) return;
    int x = a.bx0 + (int)(b % d.bw), y = a.by0 + (int)(b / d.bw);
    if (c == CLS_DISC) {
        int8_t prev = CLS_DISC;
        if (!a.first) {
            unsigned px = (unsigned)(x - a.pbx0), py = (unsigned)(y - a.pby0);
            if (px < (unsigned)d.bw && py < (unsigned)d.bh) prev = d.cls_prev[(int64_t)py * d.bw + px];
        }
        if (prev == CLS_DISC) return;
        if (prev == CLS_UNUSED && lane == 0) atomicOr(d.status, HLBM_ST_UNUSED_TO_DISC);
    }
    int64_t s = (int64_t)y * d.pitch + x;
    double lam[3];
    int k = locate_warp(d, __dsub_rn((double)x, a.cx), __dsub_rn((double)y, a.cy), lam);
    if (k < 0) {
        if (lane == 0) atomicOr(d.status, HLBM_ST_FILL_NOT_LOCATED);
        if (lane < 9) Store<T, S>::st(A, lane * d.plane + s, T(0), d.fscale);
        return;
    }
    T st[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) st[j] = T(0);
    for (int j = 0; j < 3; ++j) {
        int v = d.tri[3 * k + j];
        T f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = d.fu_in[(int64_t)kRec * v + i];
        T dr, r, ux, uy;
        moments_dev(f, d.rho0, dr, r, ux, uy);
        T l = T(lam[j]);
        st[0] += l * dr;
        st[1] += l * ux;
        st[2] += l * uy;
#pragma unroll
        for (int i = 0; i < 9; ++i) st[3 + i] += l * (f[i] - feq_dev<T>(i, dr, r, ux, uy));
    }
    const T rr = d.rho0 + st[0];
#pragma unroll
    for (int i = 0; i < 9; ++i)
        if (lane == i)
            Store<T, S>::st(A, i * d.plane + s, feq_dev<T>(i, st[0], rr, st[1], st[2]) + d.k178 * st[3 + i], d.fscale);
}

template <typename T>
void launch_fill(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    with_store(d, [&]<typename S>() { k_fill<T, S><<<(unsigned)((d.bplane * 32 + 127) / 128), 128, 0, s>>>(d, a); });
}

// ------------------------------------------------------ stream-collide
// Pull form of eq. LBE: f_i(x, t+1) = f~_i(x - c_i, t), then BGK relaxation
// with tau_s (pull_edge: the Sec. 5 boundaries).
// One lattice node: pull (or take the given pulled values), BGK, store.
template <typename T, typename S>
__device__ __forceinline__ void collide_store(const Dev<T>& d, const StepArgs& a, int x, int y, T (&f)[9]) {
    unsigned rx = (unsigned)(x - a.bx0), ry = (unsigned)(y - a.by0);
    bool inbox = rx < (unsigned)d.bw && ry < (unsigned)d.bh;
    int64_t b = (int64_t)ry * d.bw + rx;
    if (inbox && d.cls_cur[b] != CLS_DISC) return;
    int64_t s = (int64_t)y * d.pitch + x;
    S* __restrict__ B = reinterpret_cast<S*>(d.fB);
    T o[9];
    bgk_dev(f, d.rho0, T(1) / d.tau_s, o);
#pragma unroll
    for (int i = 0; i < 9; ++i) Store<T, S>::st(B, i * d.plane + s, o[i], d.fscale);
    if (inbox) {
#pragma unroll
        for (int i = 0; i < 9; ++i) d.sbox_new[i * d.bplane + b] = f[i];
    }
}

// a vector of consecutive storage elements: 4 nodes (16 bytes) for FP32,
// 2 (16 bytes) for FP64, 4 (8 bytes) for FP16 / BF16.  Measured on the
// 4096^2 lattice, 8-node 16-byte vectors for the 2-byte types reach 0.57 of
// the copy bandwidth against 0.77 for these: a thread then computes 8 nodes
// between its loads, with fewer threads resident to cover the latency.
template <typename S>
struct alignas(sizeof(S) == 2 ? 8 : 16) Pack {
    static constexpr int N = sizeof(S) == 2 ? 4 : 16 / (int)sizeof(S);
    S v[N];
};

template <typename S>
__device__ __forceinline__ S shfl_up1(S v) {
    if constexpr (sizeof(S) == 2) {
        unsigned short u;
        memcpy(&u, &v, 2);
        u = (unsigned short)__shfl_up_sync(0xffffffffu, (unsigned)u, 1);
        memcpy(&v, &u, 2);
        return v;
    } else {
        return __shfl_up_sync(0xffffffffu, v, 1);
    }
}
template <typename S>
__device__ __forceinline__ S shfl_down1(S v) {
    if constexpr (sizeof(S) == 2) {
        unsigned short u;
        memcpy(&u, &v, 2);
        u = (unsigned short)__shfl_down_sync(0xffffffffu, (unsigned)u, 1);
        memcpy(&v, &u, 2);
        return v;
    } else {
        return __shfl_down_sync(0xffffffffu, v, 1);
    }
}

// resident blocks per SM the register budget of k_stream_collide aims at
template <typename S>
constexpr int kStreamBlocks = sizeof(S) == 2 ? 8 : 6;

// Pull form of eq. LBE: f_i(x, t+1) = f~_i(x - c_i, t), then BGK relaxation
// with tau_s.  Each thread owns the V consecutive nodes of one vector of a
// row (Pack<S>) and reads each population as one vector load from row
// y - c_iy; the x - c_ix shift comes from the neighbouring lane (warp
// shuffle), and the first and last lane of a warp load the one element
// beyond their vector.  The nine vectors stay in storage form and are
// converted node by node (FP16 and BF16 at 64 registers, 8 blocks per SM).
// Nodes on the lattice edge take the scalar path with the Sec. 5 boundaries
// (half-way bounce-back walls taking precedence at corners, zero-gradient
// outflow, or periodic wrap).  Every lane runs the vector loads and shuffles
// (rows and columns clamped into the buffer); only the nodes of lanes whose
// whole vector is interior use their results.  The launch covers the
// columns [rx0, rx1) of the rows ry0 + blockIdx.y (rx0 a multiple of V).
template <typename T, typename S>
__global__ void __launch_bounds__(128, kStreamBlocks<S>)
    k_stream_collide(Dev<T> d, StepArgs a, int rx0, int ry0, int rx1) {
    constexpr int V = Pack<S>::N;
    const int lane = threadIdx.x & 31;
    const int x0 = rx0 + (blockIdx.x * blockDim.x + threadIdx.x) * V;
    const int y = ry0 + blockIdx.y;
    const S* __restrict__ A = reinterpret_cast<const S*>(d.fA);
    const bool interior = x0 >= 1 && x0 + V <= d.nx - 1 && x0 + V <= rx1 && y >= 1 && y <= d.ny - 2;
    Pack<S> p[9];
    S edge[9];  // c_ix = +1: the element left of the vector; -1: the one right of it
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sy = y - cy_of(i);
        sy = sy < 0 ? 0 : (sy >= d.ny ? d.ny - 1 : sy);
        const int64_t row = i * d.plane + (int64_t)sy * d.pitch;
        const int xv = x0 < d.pitch ? x0 : d.pitch - V;
        p[i] = *reinterpret_cast<const Pack<S>*>(A + row + xv);
        if (cx_of(i) == 1) {
            edge[i] = shfl_up1(p[i].v[V - 1]);
            if (lane == 0) edge[i] = A[row + (xv > 0 ? xv - 1 : 0)];
        } else if (cx_of(i) == -1) {
            edge[i] = shfl_down1(p[i].v[0]);
            if (lane == 31) edge[i] = A[row + (xv + V < d.pitch ? xv + V : d.pitch - 1)];
        }
    }
    if (interior) {
        // BGK for all V nodes, two at a time on raw storage values, one
        // vector store per population.  Values written at nodes that are
        // not discretization nodes are never read: interpolation and newly
        // uncovered nodes are overwritten by eq. 178 before the next pull,
        // unused nodes are never pulled from.
        using St = Store<T, S>;
        S* __restrict__ B = reinterpret_cast<S*>(d.fB);
        const T omega = T(1) / d.tau_s;
        const T raw = St::kScaled ? T(d.fscale) : T(1);  // raw value = raw * f'
        const T rho0r = d.rho0 * raw;
        const unsigned ry = (unsigned)(y - a.by0);
        const bool row_in_window = ry < (unsigned)d.bh;
        Pack<S> out[9];
#pragma unroll
        for (int k = 0; k < V; k += 2) {
            T o[2][9];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                // node x0 + k + h pulls x0 + k + h - c_ix
                const int kk = k + h;
                T f[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    if (cx_of(i) == 0)
                        f[i] = St::rd(p[i].v, kk);
                    else if (cx_of(i) == 1)
                        f[i] = kk == 0 ? St::rd(&edge[i], 0) : St::rd(p[i].v, kk - 1);
                    else
                        f[i] = kk == V - 1 ? St::rd(&edge[i], 0) : St::rd(p[i].v, kk + 1);
                }
                bgk_dev(f, rho0r, omega, o[h]);
                // the pre-collision state of discretization nodes in the window
                if (row_in_window) {
                    const unsigned rx = (unsigned)(x0 + kk - a.bx0);
                    if (rx < (unsigned)d.bw) {
                        const int64_t b = (int64_t)ry * d.bw + rx;
                        if (d.cls_cur[b] == CLS_DISC) {
#pragma unroll
                            for (int i = 0; i < 9; ++i)
                                d.sbox_new[i * d.bplane + b] = St::kScaled ? f[i] * T(d.finv) : f[i];
                        }
                    }
                }
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) St::wr2(out[i].v, k, o[0][i], o[1][i]);
        }
        const int64_t s0 = (int64_t)y * d.pitch + x0;
#pragma unroll
        for (int i = 0; i < 9; ++i) *reinterpret_cast<Pack<S>*>(B + i * d.plane + s0) = out[i];
    } else {
        for (int k = 0; k < V; ++k) {
            const int x = x0 + k;
            if (x >= d.nx || x >= rx1) break;
            T g[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = pull_edge<T, S>(d, A, x, y, i);
            collide_store<T, S>(d, a, x, y, g);
        }
    }
}

template <typename T>
void launch_stream_collide(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    launch_stream_collide_rect(d, a, 0, 0, d.nx, d.ny, s);
}

// The absorbing layer (non-reflecting outflow reading of Sec. 5) on the
// post-collision populations stream-collide has just written to fB: the
// nodes of [x0, x1) x [y0, y1) within sponge_rows of an outflow side are
// damped towards the rest state (their deviations times 1 - s(d)).  Run
// right after stream-collide, before anything reads fB, it gives the values
// of a damping inside the collision.
template <typename T, typename S>
__global__ void k_sponge(Dev<T> d, int x0, int y0, int x1, int y1) {
    const int x = x0 + blockIdx.x * blockDim.x + threadIdx.x, y = y0 + blockIdx.y;
    if (x >= x1 || y >= y1) return;
    const T keep = sponge_keep(d, x, y);
    if (keep == T(1)) return;
    S* B = reinterpret_cast<S*>(d.fB);
    const int64_t s = (int64_t)y * d.pitch + x;
#pragma unroll
    for (int i = 0; i < 9; ++i)
        Store<T, S>::st(B, i * d.plane + s, mul_rn(keep, Store<T, S>::ld(B, i * d.plane + s, d.finv)), d.fscale);
}

// the layer's rows along the y sides (whole rows), then its columns along the
// x sides between them, so that every node is damped once; returns launches
template <typename T>
int launch_sponge(const Dev<T>& d, cudaStream_t s) {
    const int N = d.sponge_rows;
    if (N <= 0 || d.sponge_sigma == 0.0) return 0;
    int n = 0;
    auto rect = [&](int x0, int y0, int x1, int y1) {
        if (x1 <= x0 || y1 <= y0) return;
        dim3 grid((x1 - x0 + 127) / 128, y1 - y0);
        with_store(d, [&]<typename S>() { k_sponge<T, S><<<grid, 128, 0, s>>>(d, x0, y0, x1, y1); });
        ++n;
    };
    int ya = 0, yb = d.ny;
    if (d.bc_y == HLBM_BC_OUTFLOW) {
        rect(0, 0, d.nx, N);
        rect(0, d.ny - N, d.nx, d.ny);
        ya = N;
        yb = d.ny - N;
    }
    if (d.bc_x == HLBM_BC_OUTFLOW) {
        rect(0, ya, N, yb);
        rect(d.nx - N, ya, d.nx, yb);
    }
    return n;
}

// the nodes of [x0, x1) x [y0, y1) (x0 a multiple of 4)
template <typename T>
void launch_stream_collide_rect(const Dev<T>& d, const StepArgs& a, int x0, int y0, int x1, int y1, cudaStream_t s) {
    if (x1 <= x0 || y1 <= y0) return;
    with_store(d, [&]<typename S>() {
        constexpr int V = Pack<S>::N;
        const int threads_x = (x1 - x0 + V - 1) / V;
        dim3 grid((threads_x + 127) / 128, y1 - y0);
        k_stream_collide<T, S><<<grid, 128, 0, s>>>(d, a, x0, y0, x1);
    });
}

// ------------------------------------------------------------- readback
template <typename T, typename S>
__global__ void k_struct_macro(Dev<T> d, double* rho, double* ux, double* uy) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= d.nx) return;
    int64_t s = (int64_t)y * d.pitch + x;
    const S* A = reinterpret_cast<const S*>(d.fA);
    T f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = Store<T, S>::ld(A, i * d.plane + s, d.finv);
    // the buffer holds post-collision populations, whose moments are those of
    // the state (BGK conserves them) except inside the absorbing layer, where
    // the layer scaled the deviations by keep: undo it for the moments
    if (d.sponge_rows > 0) {
        const T keep = sponge_keep(d, x, y);
        if (keep != T(1)) {
#pragma unroll
            for (int i = 0; i < 9; ++i) f[i] = f[i] / keep;
        }
    }
    T dr, r, vx, vy;
    moments_dev(f, d.rho0, dr, r, vx, vy);
    int64_t g = (int64_t)y * d.nx + x;
    rho[g] = double(d.rho0) + double(dr);
    ux[g] = double(vx);
    uy[g] = double(vy);
}

template <typename T>
void launch_struct_macro(const Dev<T>& d, double* rho, double* ux, double* uy, cudaStream_t s) {
    dim3 grid((d.nx + 255) / 256, d.ny);
    with_store(d, [&]<typename S>() { k_struct_macro<T, S><<<grid, 256, 0, s>>>(d, rho, ux, uy); });
}

// ------------------------------------------------------- nested levels
// Each pair of adjacent levels (Sec. 5 refinement levels): the finer one is
// a box inside the coarser, which has twice the spacing and time step and
// tau_c - 1/2 = (tau_f - 1/2)/2.  Post-collision non-equilibrium parts
// scale as (tau - 1) dx: f^neq_c = 2 (tau_c - 1)/(tau_f - 1) f^neq_f.

// One launch couples the levels after a fine stream-collide:
//  - blocks [0, ring_blocks): the fine box's outermost ring (x = 0, nx-1 or
//    y = 0, ny-1) takes the post-collision ghost f^eq(rho, u) + acf f^neq,
//    with rho, u, f^neq of the coarse lattice at the node: the coarse node
//    itself at even positions, the cubic midpoint rule (-1, 9, 9, -1)/16
//    along the box edge at odd ones; from coarse buffer c0 alone, or the
//    mean of c0 and c1 (odd fine times).  Four lanes share a ring node, one
//    per stencil point, and combine their sums with two shuffles.
//  - the other blocks (only when rsrc is set): the coarse nodes strictly
//    inside the box take the post-collision state of the fine node under
//    them, f^eq + afc f^neq; nodes over a fine node that the last step did
//    not compute (class in the window at (bx0, by0)) take f^eq(rho0, 0),
//    i.e. zero deviations.
// The ring reads coarse nodes on or outside the box's footprint and the
// restriction writes only nodes strictly inside it, so the two never touch
// the same coarse node.
template <typename T, typename S>
__global__ void __launch_bounds__(128) k_couple(Dev<T> d, Refine r, Couple c, int ring_blocks) {
    if ((int)blockIdx.x < ring_blocks) {
        const int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
        const int lane4 = threadIdx.x & 3;
        const int64_t k = g >> 2;
        const int nring = 2 * d.nx + 2 * (d.ny - 2);
        const bool live = k < nring;
        int x = 0, y = 0;
        if (k < d.nx) {
            x = (int)k;
        } else if (k < 2 * d.nx) {
            x = (int)k - d.nx;
            y = d.ny - 1;
        } else if (k < 2 * d.nx + d.ny - 2) {
            y = 1 + (int)k - 2 * d.nx;
        } else {
            x = d.nx - 1;
            y = 1 + (int)k - 2 * d.nx - (d.ny - 2);
        }
        // the stencil runs along the edge: x on the bottom and top rows
        // (corners included), y on the side columns; the fine coordinate
        // across the edge is even (nx, ny odd), i.e. on a coarse line
        const bool along_x = (y == 0 || y == d.ny - 1);
        const int X = 2 * r.ox + x, Y = 2 * r.oy + y;
        const int P = along_x ? X : Y;
        int I = X >> 1, J = Y >> 1;
        T w = T(0);
        if ((P & 1) == 0) {
            w = lane4 == 0 ? T(1) : T(0);
        } else {
            const int p = ((P - 1) >> 1) - 1 + lane4;
            if (along_x)
                I = p;
            else
                J = p;
            w = (lane4 == 0 || lane4 == 3) ? T(-1.0 / 16.0) : T(9.0 / 16.0);
        }
        T acc[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) acc[j] = T(0);
        if (live && w != T(0)) {
            const int nb = c.c1 ? 2 : 1;
            const T wq = nb == 2 ? w * T(0.5) : w;
            const int64_t sc = (int64_t)J * r.pitch + I;
            for (int q = 0; q < nb; ++q) {
                const S* src = reinterpret_cast<const S*>(q == 0 ? c.c0 : c.c1);
                T f[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) f[i] = Store<T, S>::ld(src, i * r.plane + sc, d.finv);
                T dr, rr, vx, vy;
                moments_dev(f, d.rho0, dr, rr, vx, vy);
                acc[0] += wq * dr;
                acc[1] += wq * vx;
                acc[2] += wq * vy;
#pragma unroll
                for (int i = 0; i < 9; ++i) acc[3 + i] += wq * (f[i] - feq_dev<T>(i, dr, rr, vx, vy));
            }
        }
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], 1);
            acc[j] += __shfl_xor_sync(0xffffffffu, acc[j], 2);
        }
        if (!live) return;
        const T rr = d.rho0 + acc[0], acf = T(r.acf);
        S* dst = reinterpret_cast<S*>(c.ring_dst);
        const int64_t s = (int64_t)y * d.pitch + x;
        for (int i = lane4; i < 9; i += 4)
            Store<T, S>::st(dst, i * d.plane + s, feq_dev<T>(i, acc[0], rr, acc[1], acc[2]) + acf * acc[3 + i],
                            d.fscale);
        return;
    }
    const int niw = (d.nx - 1) / 2 - 1, njw = (d.ny - 1) / 2 - 1;
    const int64_t k = ((int64_t)blockIdx.x - ring_blocks) * blockDim.x + threadIdx.x;
    if (k >= (int64_t)niw * njw) return;
    const int ii = (int)(k % niw) + 1, jj = (int)(k / niw) + 1;
    const int x = 2 * ii, y = 2 * jj;
    const int64_t sc = (int64_t)(r.oy + jj) * r.pitch + (r.ox + ii);
    S* dst = reinterpret_cast<S*>(c.rdst);
    const unsigned rx = (unsigned)(x - c.bx0), ry = (unsigned)(y - c.by0);
    if (rx < (unsigned)d.bw && ry < (unsigned)d.bh && d.cls_cur[(int64_t)ry * d.bw + rx] != CLS_DISC) {
#pragma unroll
        for (int i = 0; i < 9; ++i) Store<T, S>::st(dst, i * r.plane + sc, T(0), d.fscale);
        return;
    }
    const S* src = reinterpret_cast<const S*>(c.rsrc);
    const int64_t s = (int64_t)y * d.pitch + x;
    T f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = Store<T, S>::ld(src, i * d.plane + s, d.finv);
    T dr, rr, vx, vy;
    moments_dev(f, d.rho0, dr, rr, vx, vy);
    const T afc = T(r.afc);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const T eq = feq_dev<T>(i, dr, rr, vx, vy);
        Store<T, S>::st(dst, i * r.plane + sc, eq + afc * (f[i] - eq), d.fscale);
    }
}

template <typename T>
void launch_couple(const Dev<T>& d, const Refine& r, const Couple& c, cudaStream_t s) {
    const int64_t nring = 2 * (int64_t)d.nx + 2 * (d.ny - 2);
    const int ring_blocks = (int)((4 * nring + 127) / 128);
    const int64_t ninner = c.rsrc ? (int64_t)((d.nx - 1) / 2 - 1) * ((d.ny - 1) / 2 - 1) : 0;
    const int blocks = ring_blocks + (int)((ninner + 127) / 128);
    with_store(d, [&]<typename S>() { k_couple<T, S><<<blocks, 128, 0, s>>>(d, r, c, ring_blocks); });
}

#define HLBM_INST(T)                                                                                     \
    template void launch_init_struct<T>(const Dev<T>&, const double*, const double*, const double*, double, \
                                        double, cudaStream_t);                                          \
    template void launch_init_box<T>(const Dev<T>&, int, int, const double*, const double*, const double*, \
                                     double, double, cudaStream_t);                                     \
    template void launch_classify<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                      \
    template void launch_fill<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                          \
    template void launch_stream_collide<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                \
    template void launch_stream_collide_rect<T>(const Dev<T>&, const StepArgs&, int, int, int, int, cudaStream_t); \
    template int launch_sponge<T>(const Dev<T>&, cudaStream_t);                                           \
    template void launch_struct_macro<T>(const Dev<T>&, double*, double*, double*, cudaStream_t);        \
    template void launch_couple<T>(const Dev<T>&, const Refine&, const Couple&, cudaStream_t);
HLBM_INST(float)
HLBM_INST(double)

}  // namespace hk
