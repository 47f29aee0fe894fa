// Cartesian-lattice kernels: initial state, node classification (Sec. 4),
// the eq. postcollision2_s feed of interpolation nodes, and the fused pull
// stream-collide of eq. LBE with the Sec. 5 boundaries.
#include "hlbm_dev.cuh"

namespace hk {

// ------------------------------------------------------------------ init
template <typename T>
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
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        T v = feq_dev<T>(i, dr, rr, vx, vy);
        d.fA[i * d.plane + s] = v;
        d.fB[i * d.plane + s] = v;
    }
}

template <typename T>
void launch_init_struct(const Dev<T>& d, const double* rho, const double* ux, const double* uy, double u0x,
                        double u0y, cudaStream_t s) {
    dim3 grid((d.nx + 255) / 256, d.ny);
    k_init_struct<T><<<grid, 256, 0, s>>>(d, rho, ux, uy, u0x, u0y);
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
template <typename T>
__global__ void k_fill(Dev<T> d, StepArgs a) {
    int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
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
        if (prev == CLS_UNUSED) atomicOr(d.status, HLBM_ST_UNUSED_TO_DISC);
    }
    int64_t s = (int64_t)y * d.pitch + x;
    double lam[3];
    int k = locate_dev(d, __dsub_rn((double)x, a.cx), __dsub_rn((double)y, a.cy), lam);
    if (k < 0) {
        atomicOr(d.status, HLBM_ST_FILL_NOT_LOCATED);
#pragma unroll
        for (int i = 0; i < 9; ++i) d.fA[i * d.plane + s] = T(0);
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
        d.fA[i * d.plane + s] = feq_dev<T>(i, st[0], rr, st[1], st[2]) + d.k178 * st[3 + i];
}

template <typename T>
void launch_fill(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    k_fill<T><<<(unsigned)((d.bplane + 127) / 128), 128, 0, s>>>(d, a);
}

// ------------------------------------------------------ stream-collide
// Pull form of eq. LBE: f_i(x, t+1) = f~_i(x - c_i, t), then BGK relaxation
// with tau_s.  Boundaries (Sec. 5): half-way bounce-back walls (taking
// precedence at corners), zero-gradient outflow, or periodic wrap.
template <typename T>
__device__ __forceinline__ T pull_edge(const Dev<T>& d, int x, int y, int i) {
    int sx = x - cx_of(i), sy = y - cy_of(i);
    if (sx < 0 || sx >= d.nx) {
        if (d.bc_x == HLBM_BC_PERIODIC)
            sx = (sx + d.nx) % d.nx;
        else if (d.bc_x == HLBM_BC_WALL)
            return d.fA[opp_of(i) * d.plane + (int64_t)y * d.pitch + x];
        else
            sx = x;
    }
    if (sy < 0 || sy >= d.ny) {
        if (d.bc_y == HLBM_BC_PERIODIC)
            sy = (sy + d.ny) % d.ny;
        else if (d.bc_y == HLBM_BC_WALL)
            return d.fA[opp_of(i) * d.plane + (int64_t)y * d.pitch + x];
        else
            sy = y;
    }
    return d.fA[i * d.plane + (int64_t)sy * d.pitch + sx];
}

template <typename T>
__global__ void __launch_bounds__(256) k_stream_collide(Dev<T> d, StepArgs a) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= d.nx) return;
    unsigned rx = (unsigned)(x - a.bx0), ry = (unsigned)(y - a.by0);
    bool inbox = rx < (unsigned)d.bw && ry < (unsigned)d.bh;
    int64_t b = (int64_t)ry * d.bw + rx;
    if (inbox && d.cls_cur[b] != CLS_DISC) return;
    int64_t s = (int64_t)y * d.pitch + x;
    T f[9];
    if (x > 0 && y > 0 && x < d.nx - 1 && y < d.ny - 1) {
        const T* __restrict__ A = d.fA;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = __ldg(A + i * d.plane + s - cy_of(i) * d.pitch - cx_of(i));
    } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = pull_edge(d, x, y, i);
    }
    T dr, r, ux, uy;
    moments_dev(f, d.rho0, dr, r, ux, uy);
    T omega = T(1) / d.tau_s;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        T fe = feq_dev<T>(i, dr, r, ux, uy);
        d.fB[i * d.plane + s] = f[i] - omega * (f[i] - fe);
    }
    if (inbox) {
#pragma unroll
        for (int i = 0; i < 9; ++i) d.sbox_new[i * d.bplane + b] = f[i];
    }
}

template <typename T>
void launch_stream_collide(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    dim3 grid((d.nx + 255) / 256, d.ny);
    k_stream_collide<T><<<grid, 256, 0, s>>>(d, a);
}

// ------------------------------------------------------------- readback
template <typename T>
__global__ void k_struct_macro(Dev<T> d, double* rho, double* ux, double* uy) {
    int x = blockIdx.x * blockDim.x + threadIdx.x;
    int y = blockIdx.y;
    if (x >= d.nx) return;
    int64_t s = (int64_t)y * d.pitch + x;
    T f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = d.fA[i * d.plane + s];
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
    k_struct_macro<T><<<grid, 256, 0, s>>>(d, rho, ux, uy);
}

#define HLBM_INST(T)                                                                                     \
    template void launch_init_struct<T>(const Dev<T>&, const double*, const double*, const double*, double, \
                                        double, cudaStream_t);                                          \
    template void launch_init_box<T>(const Dev<T>&, int, int, const double*, const double*, const double*, \
                                     double, double, cudaStream_t);                                     \
    template void launch_classify<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                      \
    template void launch_fill<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                          \
    template void launch_stream_collide<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                \
    template void launch_struct_macro<T>(const Dev<T>&, double*, double*, double*, cudaStream_t);
HLBM_INST(float)
HLBM_INST(double)

}  // namespace hk
