// Patch kernels: FV matrices of eq. ulbe, the refill procedure of Sec. 4,
// the outer-node feed of eq. postcollision2_u, the FV sub-step, the force on
// the lamina and the reductions of the hydrodynamic-function fit (Sec. 2.1).
#include "hlbm_dev.cuh"

namespace hk {

constexpr int kMaxRow = 64;

// ------------------------------------------------------ FV matrices
// Cell-vertex FV on median-dual control volumes with f linear on each
// triangle.  Per node P (V_P = sum_T |T|/3):
//   g_Pk = -(1/V_P) sum_{T ni P,k} (|T|/3) grad phi_k|_T   (the boundary flux
//          of CV(P), by the gradient theorem), S_ik = c_i . g_Pk;
//   C_Pk = (1/V_P) sum_{T ni P,k} |T| (11/54 if k = P else 7/108)
//          (integral of phi_k over CV(P)), or the identity when lumped.
template <typename T>
__global__ void k_fv_coeffs(Dev<T> d, const int32_t* tstart, const int32_t* tlist, int lumped, T* gx_out,
                            T* gy_out, T* cc_out) {
    int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.n) return;
    int r0 = d.row_ptr[P], r1 = d.row_ptr[P + 1];
    double gx[kMaxRow], gy[kMaxRow], cc[kMaxRow];
    for (int e = 0; e < r1 - r0; ++e) gx[e] = gy[e] = cc[e] = 0.0;
    double V = 0.0;
    for (int e = tstart[P]; e < tstart[P + 1]; ++e) {
        const int32_t* v = d.tri + 3 * tlist[e];
        double x0 = d.xy[2 * v[0]], y0 = d.xy[2 * v[0] + 1];
        double x1 = d.xy[2 * v[1]], y1 = d.xy[2 * v[1] + 1];
        double x2 = d.xy[2 * v[2]], y2 = d.xy[2 * v[2] + 1];
        double A2 = (x1 - x0) * (y2 - y0) - (x2 - x0) * (y1 - y0);
        double area = 0.5 * fabs(A2);
        V += area / 3.0;
        double X[3] = {x0, x1, x2}, Y[3] = {y0, y1, y2};
        for (int a = 0; a < 3; ++a) {
            int b = (a + 1) % 3, c = (a + 2) % 3;
            double grx = (Y[b] - Y[c]) / A2, gry = (X[c] - X[b]) / A2;
            int pos = -1;
            for (int q = r0; q < r1; ++q)
                if (d.col[q] == v[a]) pos = q - r0;
            if (pos < 0) continue;
            gx[pos] -= area / 3.0 * grx;
            gy[pos] -= area / 3.0 * gry;
            cc[pos] += area * (v[a] == P ? 11.0 / 54.0 : 7.0 / 108.0);
        }
    }
    for (int e = 0; e < r1 - r0; ++e) {
        gx_out[r0 + e] = T(gx[e] / V);
        gy_out[r0 + e] = T(gy[e] / V);
        cc_out[r0 + e] = lumped ? T(d.col[r0 + e] == P ? 1 : 0) : T(cc[e] / V);
    }
}

template <typename T>
void launch_fv_coeffs(const Dev<T>& d, const int32_t* tstart, const int32_t* tlist, int lumped, T* gx, T* gy,
                      T* cc, cudaStream_t s) {
    k_fv_coeffs<T><<<(d.n + 127) / 128, 128, 0, s>>>(d, tstart, tlist, lumped, gx, gy, cc);
}

// ------------------------------------------------ bilinear from lattice
// Sec. 4 (type 1): bilinear Lagrange interpolation of rho, u and f^neq over
// the four lattice nodes of the cell enclosing (wx, wy).  The lattice state
// is read from a window (origin ox, oy) of pre-collision populations; with
// cls given, the four donors must be discretization nodes.
template <typename T>
__device__ __forceinline__ void bilinear_state(const Dev<T>& d, const T* box, int ox, int oy, const int8_t* cls,
                                               double wx, double wy, T st[12], int& cell) {
    double fx0 = floor(wx), fy0 = floor(wy);
    int ix = (int)fx0, iy = (int)fy0;
    double ax = __dsub_rn(wx, fx0), ay = __dsub_rn(wy, fy0);
    T w4[4] = {T((1.0 - ax) * (1.0 - ay)), T(ax * (1.0 - ay)), T((1.0 - ax) * ay), T(ax * ay)};
    cell = iy * d.nx + ix;
#pragma unroll
    for (int j = 0; j < 12; ++j) st[j] = T(0);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        int bx = ix + (q & 1) - ox, by = iy + (q >> 1) - oy;
        if ((unsigned)bx >= (unsigned)d.bw || (unsigned)by >= (unsigned)d.bh) {
            atomicOr(d.status, HLBM_ST_DONOR_NOT_COMPUTED);
            continue;
        }
        int64_t b = (int64_t)by * d.bw + bx;
        if (cls && cls[b] != CLS_DISC) atomicOr(d.status, HLBM_ST_DONOR_NOT_COMPUTED);
        T f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = box[i * d.bplane + b];
        T dr, r, ux, uy;
        moments_dev(f, d.rho0, dr, r, ux, uy);
        st[0] += w4[q] * dr;
        st[1] += w4[q] * ux;
        st[2] += w4[q] * uy;
#pragma unroll
        for (int i = 0; i < 9; ++i) st[3 + i] += w4[q] * (f[i] - feq_dev<T>(i, dr, r, ux, uy));
    }
}

// eq. continuity_stresses: f = f^eq(rho, u) + (1 - 1/(2 tau_s)) f^neq,s;
// st = (drho, ux, uy, f^neq[9])
template <typename T>
__device__ __forceinline__ T f_from_state(const Dev<T>& d, const T st[12], int i) {
    return feq_dev<T>(i, st[0], d.rho0 + st[0], st[1], st[2]) + d.kneq * st[3 + i];
}

// initial patch: every node by the type-1 rule from the initial lattice state
template <typename T>
__global__ void k_patch_init(Dev<T> d, StepArgs a) {
    int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.n) return;
    T st[12];
    int cell;
    bilinear_state(d, d.sbox_old, a.pbx0, a.pby0, (const int8_t*)nullptr, __dadd_rn(a.cx, d.xy[2 * P]),
                   __dadd_rn(a.cy, d.xy[2 * P + 1]), st, cell);
#pragma unroll
    for (int i = 0; i < 9; ++i) d.fu_out[i * (int64_t)d.n + P] = f_from_state(d, st, i);
}

template <typename T>
void launch_patch_init(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    k_patch_init<T><<<(d.n + 127) / 128, 128, 0, s>>>(d, a);
}

// ------------------------------------------------------------ refill
// Sec. 4 at the start of step t: each non-wall node, moved by (dX, dY), is
// located in the previous configuration: type 3 (inside a triangle:
// barycentric f), type 2 (inside the body: keep f), type 1 (outside the
// patch: bilinear from the lattice state at t).  Wall nodes keep f and rho.
template <typename T>
__global__ void k_refill(Dev<T> d, StepArgs a) {
    int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.n) return;
    const int64_t n = d.n;
    if (d.kind[P] == HLBM_NODE_WALL) {
#pragma unroll
        for (int i = 0; i < 9; ++i) d.fu_out[i * n + P] = d.fu_in[i * n + P];
        d.rtype[P] = 0;
        d.rdonor[P] = -1;
        return;
    }
    double qx = __dadd_rn(d.xy[2 * P], a.dX), qy = __dadd_rn(d.xy[2 * P + 1], a.dY);
    double lam[3];
    int k = locate_from_node(d, P, qx, qy, lam);
    if (k >= 0) {
        const int32_t* v = d.tri + 3 * k;
        T l0 = T(lam[0]), l1 = T(lam[1]), l2 = T(lam[2]);
#pragma unroll
        for (int i = 0; i < 9; ++i)
            d.fu_out[i * n + P] = l0 * d.fu_in[i * n + v[0]] + l1 * d.fu_in[i * n + v[1]] + l2 * d.fu_in[i * n + v[2]];
        d.rtype[P] = 3;
        d.rdonor[P] = k;
    } else if (fabs(qx) <= d.half_L && fabs(qy) <= d.half_T) {
#pragma unroll
        for (int i = 0; i < 9; ++i) d.fu_out[i * n + P] = d.fu_in[i * n + P];
        d.rtype[P] = 2;
        d.rdonor[P] = -1;
    } else {
        T st[12];
        int cell;
        bilinear_state(d, d.sbox_old, a.pbx0, a.pby0, d.cls_prev, __dadd_rn(a.cx, d.xy[2 * P]),
                       __dadd_rn(a.cy, d.xy[2 * P + 1]), st, cell);
#pragma unroll
        for (int i = 0; i < 9; ++i) d.fu_out[i * n + P] = f_from_state(d, st, i);
        d.rtype[P] = 1;
        d.rdonor[P] = cell;
    }
}

template <typename T>
void launch_refill(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    k_refill<T><<<(d.n + 127) / 128, 128, 0, s>>>(d, a);
}

// ------------------------------------------------- outer-node feed
// Lattice state at t (previous window) and t+1 (this step's window),
// bilinear at the outer nodes: snap[0] and snap[1], 12 values each.
template <typename T>
__global__ void k_feed(Dev<T> d, StepArgs a) {
    int o = blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= d.n_outer) return;
    int P = d.outer[o];
    double wx = __dadd_rn(a.cx, d.xy[2 * P]), wy = __dadd_rn(a.cy, d.xy[2 * P + 1]);
    T s0[12], s1[12];
    int cell;
    bilinear_state(d, d.sbox_old, a.pbx0, a.pby0, d.cls_prev, wx, wy, s0, cell);
    bilinear_state(d, (const T*)d.sbox_new, a.bx0, a.by0, (const int8_t*)d.cls_cur, wx, wy, s1, cell);
    const int64_t no = d.n_outer;
#pragma unroll
    for (int j = 0; j < 12; ++j) {
        d.snap[j * no + o] = s0[j];
        d.snap[(12 + j) * no + o] = s1[j];
    }
}

template <typename T>
void launch_feed(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    if (d.n_outer) k_feed<T><<<(d.n_outer + 127) / 128, 128, 0, s>>>(d, a);
}

// ----------------------------------------------------------- FV step
// One explicit step of eq. ulbe on interior and wall nodes:
//   f_P += dt_u sum_k [ (c_i . g_Pk) f_k - (C_Pk / tau_u) (f_k - f_k^eq) ]
// (deviations drop out of the streaming sum because sum_k g_Pk = 0);
// wall nodes then take the lamina velocity: f += f^eq(rho, U) - f^eq(rho, u).
// Outer nodes take the lattice state, linear in time at theta = (m+1)/n:
//   f = f^eq(rho, u) + (1 - 1/(2 tau_s)) f^neq  (eq. postcollision2_u).
template <typename T>
__global__ void __launch_bounds__(128) k_fv_substep(Dev<T> d, StepArgs a, int m) {
    int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.n) return;
    const int64_t n = d.n;
    int8_t kind = d.kind[P];
    if (kind == HLBM_NODE_OUTER) {
        int o = d.outer_of[P];
        const int64_t no = d.n_outer;
        T th = T(m + 1) / T(d.n_sub);
        T st[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) st[j] = (T(1) - th) * d.snap[j * no + o] + th * d.snap[(12 + j) * no + o];
#pragma unroll
        for (int i = 0; i < 9; ++i) d.fu_out[i * n + P] = f_from_state(d, st, i);
        return;
    }
    T acc[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) acc[i] = T(0);
    T inv_tau = T(1) / d.tau_u;
    for (int e = d.row_ptr[P]; e < d.row_ptr[P + 1]; ++e) {
        int k = d.col[e];
        T f[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = d.fu_in[i * n + k];
        T dr, r, ux, uy;
        moments_dev(f, d.rho0, dr, r, ux, uy);
        T gxe = d.gx[e], gye = d.gy[e], ce = d.cc[e] * inv_tau;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            T S = T(cx_of(i)) * gxe + T(cy_of(i)) * gye;
            acc[i] += S * f[i] - ce * (f[i] - feq_dev<T>(i, dr, r, ux, uy));
        }
    }
    T fn[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) fn[i] = d.fu_in[i * n + P] + d.dt_u * acc[i];
    if (kind == HLBM_NODE_WALL) {
        double time = double(a.t) + double(m + 1) / double(d.n_sub);
        T U = T(0), V = T(0);
        if (d.motion == HLBM_MOTION_HARMONIC) {
            V = T(d.A * d.omega * cos(d.omega * time));
        } else if (d.motion == HLBM_MOTION_UNIFORM) {
            U = T(d.vx);
            V = T(d.vy);
        }
        T dr, r, ux, uy;
        moments_dev(fn, d.rho0, dr, r, ux, uy);
#pragma unroll
        for (int i = 0; i < 9; ++i) fn[i] += feq_dev<T>(i, dr, r, U, V) - feq_dev<T>(i, dr, r, ux, uy);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) d.fu_out[i * n + P] = fn[i];
}

template <typename T>
void launch_fv_substep(const Dev<T>& d, const StepArgs& a, int m, cudaStream_t s) {
    k_fv_substep<T><<<(d.n + 127) / 128, 128, 0, s>>>(d, a, m);
}

// ------------------------------------------------------------- force
// Stress at wall nodes, sigma = -(rho - rho0) c_s^2 I - sum_i f^neq_i c_i c_i,
// integrated by the trapezoid rule over the wall segments with the body's
// outward normal (force of the fluid on the lamina, per unit length).
// One block, fixed-order tree reduction: the result does not depend on
// scheduling.
template <typename T>
__device__ void wall_stress(const Dev<T>& d, int P, double s[3]) {
    T f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = d.fu_in[i * (int64_t)d.n + P];
    T dr, r, ux, uy;
    moments_dev(f, d.rho0, dr, r, ux, uy);
    double pxx = 0, pxy = 0, pyy = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        double fneq = double(f[i] - feq_dev<T>(i, dr, r, ux, uy));
        pxx += fneq * (cx_of(i) * cx_of(i));
        pxy += fneq * (cx_of(i) * cy_of(i));
        pyy += fneq * (cy_of(i) * cy_of(i));
    }
    double p = double(dr) / 3.0;
    s[0] = -p - pxx;
    s[1] = -pxy;
    s[2] = -p - pyy;
}

template <typename T>
__global__ void __launch_bounds__(128) k_force_segments(Dev<T> d) {
    int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.nseg) return;
    double sa[3], sb[3];
    wall_stress(d, d.seg_a[k], sa);
    wall_stress(d, d.seg_b[k], sb);
    double nx = d.seg_n[2 * k], ny = d.seg_n[2 * k + 1];
    d.fcontrib[2 * k] = 0.5 * ((sa[0] + sb[0]) * nx + (sa[1] + sb[1]) * ny);
    d.fcontrib[2 * k + 1] = 0.5 * ((sa[1] + sb[1]) * nx + (sa[2] + sb[2]) * ny);
}

// fixed-order sum of the segment contributions (independent of scheduling)
__global__ void __launch_bounds__(512) k_force_sum(const double* contrib, int nseg, double* force, int64_t t_out,
                                                  unsigned* status) {
    __shared__ double sx[512], sy[512];
    double fx = 0.0, fy = 0.0;
    for (int k = threadIdx.x; k < nseg; k += blockDim.x) {
        fx += contrib[2 * k];
        fy += contrib[2 * k + 1];
    }
    sx[threadIdx.x] = fx;
    sy[threadIdx.x] = fy;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) {
            sx[threadIdx.x] += sx[threadIdx.x + w];
            sy[threadIdx.x] += sy[threadIdx.x + w];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        force[2 * t_out] = sx[0];
        force[2 * t_out + 1] = sy[0];
        if (!isfinite(sx[0]) || !isfinite(sy[0])) atomicOr(status, HLBM_ST_NONFINITE);
    }
}

template <typename T>
void launch_force(const Dev<T>& d, int64_t t_out, cudaStream_t s) {
    if (d.nseg > 0) k_force_segments<T><<<(d.nseg + 127) / 128, 128, 0, s>>>(d);
    k_force_sum<<<1, 512, 0, s>>>(d.fcontrib, d.nseg, d.force, t_out, d.status);
}

// ---------------------------------------------------------- readback
template <typename T>
__global__ void k_patch_macro(Dev<T> d, double* rho, double* ux, double* uy, double* f9) {
    int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.n) return;
    T f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = d.fu_in[i * (int64_t)d.n + P];
    T dr, r, vx, vy;
    moments_dev(f, d.rho0, dr, r, vx, vy);
    if (rho) rho[P] = double(d.rho0) + double(dr);
    if (ux) ux[P] = double(vx);
    if (uy) uy[P] = double(vy);
    if (f9) {
#pragma unroll
        for (int i = 0; i < 9; ++i) f9[9 * (int64_t)P + i] = double(f[i]) + double(w_of<T>(i)) * double(d.rho0);
    }
}

template <typename T>
void launch_patch_macro(const Dev<T>& d, double* rho, double* ux, double* uy, double* f9, cudaStream_t s) {
    k_patch_macro<T><<<(d.n + 127) / 128, 128, 0, s>>>(d, rho, ux, uy, f9);
}

// ------------------------------------------- hydrodynamic function fit
// Sums of the normal equations of F_y(t) = a sin(w t) + b cos(w t).
__global__ void __launch_bounds__(512) k_gamma_sums(const double* force, int64_t t0, int64_t t1, double omega,
                                                    double* out) {
    __shared__ double sh[5][512];
    double acc[5] = {0, 0, 0, 0, 0};
    for (int64_t t = t0 + threadIdx.x; t <= t1; t += blockDim.x) {
        double s, c;
        sincos(omega * (double)t, &s, &c);
        double F = force[2 * t + 1];
        acc[0] += s * s;
        acc[1] += s * c;
        acc[2] += c * c;
        acc[3] += F * s;
        acc[4] += F * c;
    }
    for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] = acc[j];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int j = 0; j < 5; ++j) sh[j][threadIdx.x] += sh[j][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = sh[threadIdx.x][0];
}

__global__ void __launch_bounds__(512) k_gamma_resid(const double* force, int64_t t0, int64_t t1, double omega,
                                                     double a, double b, double* out) {
    __shared__ double sh[512];
    double acc = 0.0;
    for (int64_t t = t0 + threadIdx.x; t <= t1; t += blockDim.x) {
        double s, c;
        sincos(omega * (double)t, &s, &c);
        double e = force[2 * t + 1] - (a * s + b * c);
        acc += e * e;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) out[0] = sh[0];
}

void launch_gamma_sums(const double* force, int64_t t0, int64_t t1, double omega, double* out, cudaStream_t s) {
    k_gamma_sums<<<1, 512, 0, s>>>(force, t0, t1, omega, out);
}

void launch_gamma_resid(const double* force, int64_t t0, int64_t t1, double omega, double a, double b,
                        double* out, cudaStream_t s) {
    k_gamma_resid<<<1, 512, 0, s>>>(force, t0, t1, omega, a, b, out);
}

#define HLBM_INST(T)                                                                                        \
    template void launch_fv_coeffs<T>(const Dev<T>&, const int32_t*, const int32_t*, int, T*, T*, T*,         \
                                      cudaStream_t);                                                        \
    template void launch_patch_init<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                         \
    template void launch_refill<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                             \
    template void launch_feed<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                               \
    template void launch_fv_substep<T>(const Dev<T>&, const StepArgs&, int, cudaStream_t);                   \
    template void launch_force<T>(const Dev<T>&, int64_t, cudaStream_t);                                      \
    template void launch_patch_macro<T>(const Dev<T>&, double*, double*, double*, double*, cudaStream_t);
HLBM_INST(float)
HLBM_INST(double)

}  // namespace hk
