// Patch kernels: FV matrices of eq. ulbe, the refill procedure of Sec. 4,
// the outer-node feed of eq. postcollision2_u, the n FV sub-steps of one
// lattice step (one persistent cooperative kernel), the force on the lamina
// and the reductions of the hydrodynamic-function fit (Sec. 2.1).
//
// Patch state: one record of kRec values per node, f'[0..8] (deviation from
// w_i rho0) followed by the quadratic equilibrium terms z[0..2] (z_of).
#include <cooperative_groups.h>

#include <algorithm>

#include "hlbm_dev.cuh"

namespace hk {

constexpr int kMaxRow = 64;

// Patch record: f'[0..8] and the quadratic equilibrium terms
// z = (jx^2 / rho, jx jy / rho, jy^2 / rho) at [9..11].  With j = sum_i c_i f'_i
// and drho = sum_i f'_i,
//   f_i^eq - w_i rho0 = w_i (drho - 1.5 (z0 + z2) + 3 c_i.j + 4.5 (cx^2 z0 + 2 cx cy z1 + cy^2 z2)),
// linear in (drho, j, z).  For sum_k C_Pk f^eq(P_k) the drho and j parts
// are sums of Cf_i = sum_k C_Pk f'_k,i, so only z has to be carried.
template <typename T>
__device__ __forceinline__ void z_of(const T (&f)[9], T rho0, T (&z)[3]) {
    T dr = T(0), jx = T(0), jy = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        dr += f[i];
        jx = add_cx(i, jx, f[i]);
        jy = add_cy(i, jy, f[i]);
    }
    T inv = T(1) / (rho0 + dr);
    z[0] = jx * jx * inv;
    z[1] = jx * jy * inv;
    z[2] = jy * jy * inv;
}

// sum_k C_Pk (f^eq_k,i - w_i rho0) from Cf_i and Z = sum_k C_Pk z_k
template <typename T>
__device__ __forceinline__ void ceq_of(const T (&Cf)[9], const T (&Z)[3], T (&ceq)[9]) {
    T dr = T(0), jx = T(0), jy = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        dr += Cf[i];
        jx = add_cx(i, jx, Cf[i]);
        jy = add_cy(i, jy, Cf[i]);
    }
    const T q0 = dr - T(1.5) * (Z[0] + Z[2]);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        // (c_i . j) and c_i c_i : Z, i.e. Z0, Z2 or Z0 +- 2 Z1 + Z2
        const T quad = cx_of(i) == 0 ? (cy_of(i) == 0 ? T(0) : Z[2])
                                     : (cy_of(i) == 0 ? Z[0]
                                                      : (cx_of(i) * cy_of(i) > 0 ? Z[0] + T(2) * Z[1]
                                                                                 : Z[0] - T(2) * Z[1]) + Z[2]);
        ceq[i] = w_of<T>(i) * (q0 + T(3) * cdot(i, jx, jy) + T(4.5) * quad);
    }
}

template <typename T>
__device__ __forceinline__ void load_f(const T* rec, T (&f)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = rec[i];
}

template <typename T>
__device__ __forceinline__ void store_rec(T* rec, const T (&f)[9], T rho0) {
    T z[3];
    z_of(f, rho0, z);
#pragma unroll
    for (int i = 0; i < 9; ++i) rec[i] = f[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) rec[9 + j] = z[j];
#pragma unroll
    for (int j = 12; j < kRec; ++j) rec[j] = T(0);
}

// ------------------------------------------------------ FV matrices
// Cell-vertex FV on median-dual control volumes with f linear on each
// triangle.  Per node P (V_P = sum_T |T|/3):
//   g_Pk = -(1/V_P) sum_{T ni P,k} (|T|/3) grad phi_k|_T   (the boundary flux
//          of CV(P), by the gradient theorem), S_ik = c_i . g_Pk;
//   C_Pk = (1/V_P) sum_{T ni P,k} |T| (11/54 if k = P else 7/108)
//          (integral of phi_k over CV(P)), or the identity when lumped.
template <typename T>
__global__ void k_fv_coeffs(Dev<T> d, int lumped, Coef<T>* coef) {
    int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.n) return;
    int r0 = d.row_ptr[P], r1 = d.row_ptr[P + 1];
    double gx[kMaxRow], gy[kMaxRow], cc[kMaxRow];
    for (int e = 0; e < r1 - r0; ++e) gx[e] = gy[e] = cc[e] = 0.0;
    double V = 0.0;
    for (int e = d.tstart[P]; e < d.tstart[P + 1]; ++e) {
        const int32_t* v = d.tri + 3 * d.tlist[e];
        double X[3], Y[3];
        for (int j = 0; j < 3; ++j) {
            X[j] = d.xy[2 * v[j]];
            Y[j] = d.xy[2 * v[j] + 1];
        }
        double A2 = (X[1] - X[0]) * (Y[2] - Y[0]) - (X[2] - X[0]) * (Y[1] - Y[0]);
        double area = 0.5 * fabs(A2);
        V += area / 3.0;
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
        Coef<T> c;
        c.col = d.col[r0 + e];
        c.gx = T(gx[e] / V);
        c.gy = T(gy[e] / V);
        c.c = lumped ? T(c.col == P ? 1 : 0) : T(cc[e] / V);
        coef[r0 + e] = c;
    }
}

template <typename T>
void launch_fv_coeffs(const Dev<T>& d, int lumped, Coef<T>* coef, cudaStream_t s) {
    k_fv_coeffs<T><<<(d.n + 127) / 128, 128, 0, s>>>(d, lumped, coef);
}

// ------------------------------------------------ bilinear from lattice
// Sec. 4 (type 1): bilinear Lagrange interpolation of rho, u and f^neq over
// the four lattice nodes of the cell enclosing (wx, wy).  The lattice state
// is read from a window (origin ox, oy) of pre-collision populations; with
// cls given, the four donors must be discretization nodes.
// st = (drho, ux, uy, f^neq[9]).
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

// eq. continuity_stresses: f = f^eq(rho, u) + (1 - 1/(2 tau_s)) f^neq,s
template <typename T>
__device__ __forceinline__ void f_from_state(const Dev<T>& d, const T st[12], T (&f)[9]) {
    const T r = d.rho0 + st[0];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = feq_dev<T>(i, st[0], r, st[1], st[2]) + d.kneq * st[3 + i];
}

// initial patch: every node by the type-1 rule from the initial lattice state
template <typename T>
__global__ void k_patch_init(Dev<T> d, StepArgs a) {
    int P = blockIdx.x * blockDim.x + threadIdx.x;
    if (P >= d.n) return;
    T st[12], f[9];
    int cell;
    bilinear_state(d, d.sbox_old, a.pbx0, a.pby0, (const int8_t*)nullptr, __dadd_rn(a.cx, d.xy[2 * P]),
                   __dadd_rn(a.cy, d.xy[2 * P + 1]), st, cell);
    f_from_state(d, st, f);
    store_rec(d.fu_out + (int64_t)kRec * P, f, d.rho0);
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
    const T* in = d.fu_in;
    T* out = d.fu_out + (int64_t)kRec * P;
    if (d.kind[P] == HLBM_NODE_WALL) {
#pragma unroll
        for (int j = 0; j < kRec; ++j) out[j] = in[(int64_t)kRec * P + j];
        d.rtype[P] = 0;
        d.rdonor[P] = -1;
        return;
    }
    double qx = __dadd_rn(d.xy[2 * P], a.dX), qy = __dadd_rn(d.xy[2 * P + 1], a.dY);
    double lam[3];
    int k = locate_from_node(d, P, qx, qy, lam);
    T f[9];
    if (k >= 0) {
        const int32_t* v = d.tri + 3 * k;
        T l0 = T(lam[0]), l1 = T(lam[1]), l2 = T(lam[2]);
        const T *a0 = in + (int64_t)kRec * v[0], *a1 = in + (int64_t)kRec * v[1], *a2 = in + (int64_t)kRec * v[2];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = l0 * a0[i] + l1 * a1[i] + l2 * a2[i];
        d.rtype[P] = 3;
        d.rdonor[P] = k;
    } else if (fabs(qx) <= d.half_L && fabs(qy) <= d.half_T) {
        load_f(in + (int64_t)kRec * P, f);
        d.rtype[P] = 2;
        d.rdonor[P] = -1;
    } else {
        T st[12];
        int cell;
        bilinear_state(d, d.sbox_old, a.pbx0, a.pby0, d.cls_prev, __dadd_rn(a.cx, d.xy[2 * P]),
                       __dadd_rn(a.cy, d.xy[2 * P + 1]), st, cell);
        f_from_state(d, st, f);
        d.rtype[P] = 1;
        d.rdonor[P] = cell;
    }
    store_rec(out, f, d.rho0);
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

// ----------------------------------------------------------- FV steps
// n explicit steps of eq. ulbe on interior and wall nodes,
//   f_P += dt_u sum_k [ (c_i . g_Pk) f_k - (C_Pk / tau_u) (f_k - f_k^eq) ],
// evaluated as dt_u [ S_i - (Cf_i - f^eq_i(Q)) / tau_u ]
// with S_i = sum_{k != P} (c_i . g_Pk) (f'_k,i - f'_P,i),
// Cf_i = sum_k C_Pk f'_k,i, Q = sum_k C_Pk q_k (the deviations drop out of
// the streaming sum because sum_k g_Pk = 0).
// Wall nodes then take the lamina velocity: f += f^eq(rho, U) - f^eq(rho, u).
// Outer nodes take the lattice state, linear in time at theta = (m+1)/n:
//   f = f^eq(rho, u) + (1 - 1/(2 tau_s)) f^neq   (eq. postcollision2_u).
// The FV update of one node (eq. ulbe), shared by both FV kernels so that
// the result of a node does not depend on the kernel or the tiling: the
// off-diagonal entries k != P in row order, then the pivot.  With the
// exact zero row sum g_PP = -sum_k g_Pk the streaming sums are written
// S_i = sum_{k != P} (c_i . g_Pk) (f_k,i - f_P,i): the same number in exact
// arithmetic, but the differences are small next to f_k, so that in FP32 the
// products no longer round at the scale of |g| |f| (|g| ~ 1/h, h down to 0.1
// at the wall).  c_i . g_Pk is gx, gy, gx + gy or gx - gy up to its sign.
template <typename T>
struct FvAcc {
    T S[9], Cf[9], Z[3];  // S[0] stays 0 (c_0 = 0)
};

template <typename T>
__device__ __forceinline__ void fv_acc_init(FvAcc<T>& a) {
#pragma unroll
    for (int i = 0; i < 9; ++i) a.S[i] = a.Cf[i] = T(0);
#pragma unroll
    for (int j = 0; j < 3; ++j) a.Z[j] = T(0);
}

// entry (g_Pk, C_Pk) of row P with the neighbour's state f, z; fP is the
// pivot's state
template <typename T>
__device__ __forceinline__ void fv_acc_entry(FvAcc<T>& a, T gx, T gy, T c, const T (&f)[9], const T (&z)[3],
                                             const T (&fP)[9]) {
    const T gp = gx + gy, gm = gx - gy;
    a.S[1] += gx * (f[1] - fP[1]);
    a.S[2] += gy * (f[2] - fP[2]);
    a.S[3] -= gx * (f[3] - fP[3]);
    a.S[4] -= gy * (f[4] - fP[4]);
    a.S[5] += gp * (f[5] - fP[5]);
    a.S[6] -= gm * (f[6] - fP[6]);
    a.S[7] -= gp * (f[7] - fP[7]);
    a.S[8] += gm * (f[8] - fP[8]);
#pragma unroll
    for (int i = 0; i < 9; ++i) a.Cf[i] += c * f[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) a.Z[k] += c * z[k];
}

// The update of eq. ulbe from the sums.  The collision sums Cf_i - ceq_i
// carry no mass and no momentum in exact arithmetic (ceq is built from the
// moments of Cf); their rounding residues m0 = sum_i n_i, m = sum_i c_i n_i
// are removed by subtracting w_i (m0 + 3 c_i.m), which leaves exact values
// unchanged and stops the residues from acting, sub-step after sub-step, as
// spurious sources of mass and momentum.
template <typename T>
__device__ __forceinline__ void fv_acc_finish(const Dev<T>& d, FvAcc<T>& a, T cP, const T (&fP)[9], const T (&zP)[3],
                                              T (&fn)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) a.Cf[i] += cP * fP[i];
#pragma unroll
    for (int k = 0; k < 3; ++k) a.Z[k] += cP * zP[k];
    T ceq[9];
    ceq_of(a.Cf, a.Z, ceq);
    T nq[9], m0 = T(0), mx = T(0), my = T(0);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        nq[i] = a.Cf[i] - ceq[i];
        m0 += nq[i];
        mx = add_cx(i, mx, nq[i]);
        my = add_cy(i, my, nq[i]);
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        nq[i] -= w_of<T>(i) * (m0 + T(3) * cdot(i, mx, my));
        fn[i] = fP[i] + d.dt_u * (a.S[i] - nq[i] * d.inv_tau_u);
    }
}

// wall nodes: impose the lamina velocity, keep the non-equilibrium part
template <typename T>
__device__ __forceinline__ void fv_wall(const Dev<T>& d, T U, T V, T (&fn)[9]) {
    T dr, rr, ux, uy;
    moments_dev(fn, d.rho0, dr, rr, ux, uy);
#pragma unroll
    for (int i = 0; i < 9; ++i) fn[i] += feq_dev<T>(i, dr, rr, U, V) - feq_dev<T>(i, dr, rr, ux, uy);
}

// outer nodes: the lattice state interpolated linearly in time (eq. 182,
// Dirichlet reading); sn[j * stride], j < 12, is the state at t and
// sn[(12 + j) * stride] the one at t + 1
template <typename T>
__device__ __forceinline__ void fv_outer_from(const Dev<T>& d, const T* sn, int64_t stride, int m, T (&fn)[9]) {
    const T th = T(m + 1) / T(d.n_sub);
    T st[12];
#pragma unroll
    for (int j = 0; j < 12; ++j) st[j] = (T(1) - th) * sn[j * stride] + th * sn[(12 + j) * stride];
    f_from_state(d, st, fn);
}

template <typename T>
__device__ __forceinline__ void fv_outer(const Dev<T>& d, int P, int m, T (&fn)[9]) {
    fv_outer_from(d, d.snap + d.outer_of[P], (int64_t)d.n_outer, m, fn);
}

template <typename T>
__device__ __forceinline__ void fv_node(const Dev<T>& d, const T* __restrict__ in, T* __restrict__ out, int P,
                                        int m, T U, T V) {
    const int8_t kind = d.kind[P];
    T fn[9];
    if (kind == HLBM_NODE_OUTER) {
        fv_outer(d, P, m, fn);
        if (d.outer_fv) {
            // eq. postcollision2_u with its FV sums: interpolated values at
            // interpolation nodes (this one included), patch values elsewhere
            FvAcc<T> acc;
            fv_acc_init(acc);
            const int r0 = d.row_ptr[P], r1 = d.row_ptr[P + 1];
            for (int e = r0 + 1; e < r1; ++e) {
                const Coef<T> c = d.coef[e];
                T f[9], z[3];
                if (d.kind[c.col] == HLBM_NODE_OUTER) {
                    fv_outer(d, c.col, m, f);
                    z_of(f, d.rho0, z);
                } else {
                    const T* rec = in + (int64_t)kRec * c.col;
#pragma unroll
                    for (int i = 0; i < 9; ++i) f[i] = rec[i];
#pragma unroll
                    for (int j = 0; j < 3; ++j) z[j] = rec[9 + j];
                }
                fv_acc_entry(acc, c.gx, c.gy, c.c, f, z, fn);
            }
            T fP[9], zP[3];
#pragma unroll
            for (int i = 0; i < 9; ++i) fP[i] = fn[i];
            z_of(fP, d.rho0, zP);
            fv_acc_finish(d, acc, d.coef[r0].c, fP, zP, fn);
        }
        store_rec(out + (int64_t)kRec * P, fn, d.rho0);
        return;
    }
    T fP[9], zP[3];
    const T* own = in + (int64_t)kRec * P;
#pragma unroll
    for (int i = 0; i < 9; ++i) fP[i] = own[i];
#pragma unroll
    for (int j = 0; j < 3; ++j) zP[j] = own[9 + j];
    FvAcc<T> acc;
    fv_acc_init(acc);
    const int r0 = d.row_ptr[P], r1 = d.row_ptr[P + 1];
    for (int e = r0 + 1; e < r1; ++e) {
        const Coef<T> c = d.coef[e];
        T f[9], z[3];
        const T* rec = in + (int64_t)kRec * c.col;
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = rec[i];
#pragma unroll
        for (int j = 0; j < 3; ++j) z[j] = rec[9 + j];
        fv_acc_entry(acc, c.gx, c.gy, c.c, f, z, fP);
    }
    fv_acc_finish(d, acc, d.coef[r0].c, fP, zP, fn);
    if (kind == HLBM_NODE_WALL) fv_wall(d, U, V, fn);
    store_rec(out + (int64_t)kRec * P, fn, d.rho0);
}

__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// 16-byte global -> shared copy that bypasses L1; completed by cp_async_wait_all
__device__ __forceinline__ void cp_async16(void* smem_dst, const void* gmem_src) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst), "l"(gmem_src) : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

constexpr int kFvThreads = 256;

// Lamina velocity at the end of sub-step m, t + (m+1)/n (the wall nodes'
// Dirichlet value, eq. 182); INDUCED motion interpolates v(t) -> v(t+1).
template <typename T>
__device__ __forceinline__ void wall_velocity(const Dev<T>& d, const StepArgs& a, int m, T& U, T& V) {
    const double time = double(a.t) + double(m + 1) / double(d.n_sub);
    U = T(0);
    V = T(0);
    if (d.motion == HLBM_MOTION_HARMONIC) {
        V = T(d.A * d.omega * cos(d.omega * time));
    } else if (d.motion == HLBM_MOTION_UNIFORM) {
        U = T(d.vx);
        V = T(d.vy);
    } else if (d.motion == HLBM_MOTION_INDUCED) {
        V = T(a.v0 + double(m + 1) / double(d.n_sub) * (a.v1 - a.v0));
    }
}

// All n sub-steps of one lattice step in one cooperative launch.  Block b
// owns the node tile [tile_start[b], tile_start[b+1]) (nodes are numbered
// along a Morton curve, so tiles are compact).  Before sub-step m a block
// waits only for the tiles that own columns of its rows to finish sub-step
// m-1 (monotone progress counters, acquire/release); that also guarantees
// they are done reading the buffer it is about to overwrite.  Sub-step m
// reads record buffer m%2 and writes buffer (m+1)%2.  Every wait is
// bounded: on timeout the block raises HLBM_ST_SYNC_TIMEOUT and the abort
// flag, and every block returns.
template <typename T>
__global__ void __launch_bounds__(kFvThreads) k_fv_steps(Dev<T> d, StepArgs a, const T* buf0, T* buf1) {
    __shared__ int abort_sh;
    const int tile = blockIdx.x;
    const int p0 = d.tile_start[tile], p1 = d.tile_start[tile + 1];
    if (threadIdx.x == 0) abort_sh = 0;
    const unsigned long long base = (unsigned long long)a.t * (unsigned long long)d.n_sub;
    const int nb0 = d.tile_nb_ptr[tile], nb1 = d.tile_nb_ptr[tile + 1];
    __syncthreads();
    for (int m = 0; m < d.n_sub; ++m) {
        if (m > 0 && threadIdx.x < 32) {
            bool ok = true;
            for (int e = nb0 + (int)threadIdx.x; e < nb1 && ok; e += 32) {
                const unsigned long long* pc = d.progress + d.tile_nb[e];
                long spins = 0;
                while (ld_acquire(pc) < base + m) {
                    if (*(volatile unsigned*)d.abort_flag) {
                        ok = false;
                        break;
                    }
                    if (++spins > d.spin_limit) {
                        atomicOr(d.status, HLBM_ST_SYNC_TIMEOUT);
                        atomicExch(d.abort_flag, 1u);
                        ok = false;
                        break;
                    }
                    __nanosleep(128);
                }
            }
            __threadfence();
            ok = __all_sync(0xffffffffu, ok);
            if (threadIdx.x == 0 && !ok) abort_sh = 1;
        }
        __syncthreads();
        if (abort_sh) return;
        const T* in = (m & 1) ? (const T*)buf1 : buf0;
        T* out = (m & 1) ? (T*)buf0 : buf1;
        T U, V;
        wall_velocity(d, a, m, U, V);
        for (int P = p0 + threadIdx.x; P < p1; P += blockDim.x) fv_node(d, in, out, P, m, U, V);
        __syncthreads();
        if (threadIdx.x == 0 && tile != d.stall_tile) {
            __threadfence();
            st_release(d.progress + tile, base + m + 1);
        }
    }
}

template <typename T>
int fv_tile_capacity() {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_fv_steps<T>, kFvThreads, 0);
    return sms * per;
}

template <typename T>
cudaError_t launch_fv_persistent(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    Dev<T> dd = d;
    StepArgs aa = a;
    const T* b0 = d.fu_in;
    T* b1 = d.fu_out;
    void* args[] = {&dd, &aa, &b0, &b1};
    return cudaLaunchCooperativeKernel((const void*)k_fv_steps<T>, dim3(d.n_tiles), dim3(kFvThreads), args, 0, s);
}

// Shared-memory variant of k_fv_steps: one block per SM and everything its
// inner loop reads in shared memory.  Block b holds, for its tile of nodes:
//   - the records (f', z; 12 values) of its own nodes, updated in place:
//     the new values of a thread's nodes wait in registers until every read
//     of the old ones is done,
//   - the records of its halo (the nodes of other tiles its rows read),
//     reloaded each sub-step,
//   - the off-diagonal FV entries in ELL form (tile-local column, g_Pk,
//     C_Pk) and per node C_PP; the pivot g_PP is minus the sum of the
//     off-diagonal g_Pk (the rows of g sum to zero),
//   - node kinds, which nodes other tiles read, and a node order with the
//     nodes that read no halo first.
// A sub-step first updates the nodes that read no halo, then waits for the
// neighbour tiles, loads the halo and updates the rest, so the exchange
// overlaps the first part.  Only nodes read by other tiles are written to
// global memory each sub-step, into record buffer (m+1)%2; the final state
// of every node goes to buffer n%2.
// threads per block and own nodes per thread (tile_n <= kSlots * threads):
// FP32 1024 x 2 fits 64 registers per thread; FP64 512 x 1
template <typename T>
constexpr int kSmemThreads = sizeof(T) == 4 ? 1024 : 512;
template <typename T>
constexpr int kSlots = sizeof(T) == 4 ? 2 : 1;
constexpr int kSR = 12;  // values per record in shared memory
constexpr int kSnap = 24;  // outer-node feed values (12 at t, 12 at t + 1)

template <typename T>
int fv_tile_max() {
    return kSlots<T> * kSmemThreads<T>;
}

struct TileSmem {
    size_t own, halo, ecol, ecoef, cpp, order, kind, send, hid, uv, omap, osnap, cnt, total;
};

template <typename T>
__host__ __device__ inline TileSmem tile_smem_layout(int cap, int hcap, int roff, int n_sub, int ocap) {
    auto up = [](size_t x) { return (x + 15) / 16 * 16; };
    TileSmem L;
    size_t o = 0;
    L.own = o;
    o = up(o + sizeof(T) * kSR * (size_t)cap);
    L.halo = o;
    o = up(o + sizeof(T) * kSR * (size_t)hcap);
    L.ecoef = o;
    o = up(o + sizeof(T) * 3 * (size_t)roff * cap);
    L.cpp = o;
    o = up(o + sizeof(T) * (size_t)cap);
    L.uv = o;
    o = up(o + sizeof(T) * 2 * (size_t)n_sub);
    L.osnap = o;
    o = up(o + sizeof(T) * kSnap * (size_t)ocap);
    L.hid = o;
    o = up(o + sizeof(int32_t) * (size_t)hcap);
    L.ecol = o;
    o = up(o + sizeof(uint16_t) * (size_t)roff * cap);
    L.order = o;
    o = up(o + sizeof(uint16_t) * (size_t)cap);
    L.kind = o;
    o = up(o + (size_t)cap);
    L.send = o;
    o = up(o + (size_t)cap);
    L.omap = o;
    o = up(o + sizeof(int16_t) * (size_t)cap);
    L.cnt = o;
    o = up(o + (size_t)cap);
    L.total = o;
    return L;
}

template <typename T>
size_t fv_smem_bytes(int tile_cap, int halo_cap, int roff, int n_sub, int ocap) {
    return tile_smem_layout<T>(tile_cap, halo_cap, roff, n_sub, ocap).total;
}

// 16-byte (float) or 2 x 16-byte (double) vector load and store
template <typename T>
struct Vec4 {
    T x, y, z, w;
};
template <typename T>
__device__ __forceinline__ Vec4<T> ld4(const T* p) {
    Vec4<T> v;
    if constexpr (sizeof(T) == 4) {
        const float4 a4 = *reinterpret_cast<const float4*>(p);
        v.x = a4.x, v.y = a4.y, v.z = a4.z, v.w = a4.w;
    } else {
        const double2 a2 = *reinterpret_cast<const double2*>(p);
        const double2 b2 = *reinterpret_cast<const double2*>(p + 2);
        v.x = a2.x, v.y = a2.y, v.z = b2.x, v.w = b2.y;
    }
    return v;
}
template <typename T>
__device__ __forceinline__ void st4(T* p, T x, T y, T z, T w) {
    if constexpr (sizeof(T) == 4) {
        *reinterpret_cast<float4*>(p) = make_float4(x, y, z, w);
    } else {
        *reinterpret_cast<double2*>(p) = make_double2(x, y);
        *reinterpret_cast<double2*>(p + 2) = make_double2(z, w);
    }
}

template <typename T>
__device__ __forceinline__ void read_rec12(const T* r, T (&f)[9], T (&z)[3]) {
    const Vec4<T> a = ld4(r), b = ld4(r + 4), c = ld4(r + 8);
    f[0] = a.x, f[1] = a.y, f[2] = a.z, f[3] = a.w;
    f[4] = b.x, f[5] = b.y, f[6] = b.z, f[7] = b.w;
    f[8] = c.x, z[0] = c.y, z[1] = c.z, z[2] = c.w;
}

// f'[0..8] of a record, and its z terms on their own (the pivot of a row is
// read before its entries for the gradient differences, its z only at the end)
template <typename T>
__device__ __forceinline__ void read_rec9(const T* r, T (&f)[9]) {
    const Vec4<T> a = ld4(r), b = ld4(r + 4);
    f[0] = a.x, f[1] = a.y, f[2] = a.z, f[3] = a.w;
    f[4] = b.x, f[5] = b.y, f[6] = b.z, f[7] = b.w;
    f[8] = r[8];
}
template <typename T>
__device__ __forceinline__ void read_z3(const T* r, T (&z)[3]) {
    z[0] = r[9], z[1] = r[10], z[2] = r[11];
}

template <typename T>
__device__ __forceinline__ void fv_node_tile(const Dev<T>& d, const unsigned char* sm, const TileSmem& L, int r,
                                             T (&fn)[9]) {
    const int cap = d.tile_cap, roff = d.ell_width - 1;
    const T* own = reinterpret_cast<const T*>(sm + L.own);
    const T* halo = reinterpret_cast<const T*>(sm + L.halo) - (size_t)kSR * cap;
    const T* ec = reinterpret_cast<const T*>(sm + L.ecoef);
    const uint16_t* ecol = reinterpret_cast<const uint16_t*>(sm + L.ecol);
    T fP[9], zP[3];
    read_rec9(own + (size_t)kSR * r, fP);
    FvAcc<T> acc;
    fv_acc_init(acc);
    const int ne = reinterpret_cast<const uint8_t*>(sm + L.cnt)[r];  // off-diagonal entries of the row
    for (int j = 0; j < ne; ++j) {
        const int e = j * cap + r;
        const int col = ecol[e];
        T f[9], z[3];
        read_rec12((col < cap ? own : halo) + (size_t)kSR * col, f, z);
        fv_acc_entry(acc, ec[e], ec[(roff + j) * cap + r], ec[(2 * roff + j) * cap + r], f, z, fP);
    }
    read_z3(own + (size_t)kSR * r, zP);
    fv_acc_finish(d, acc, reinterpret_cast<const T*>(sm + L.cpp)[r], fP, zP, fn);
}

// eq. postcollision2_u with its FV sums at the outer node in slot r, whose
// interpolated value fn holds on entry: the starred values are the
// interpolated ones at interpolation nodes (own ones from the staged feed,
// halo ones from global memory) and the patch records elsewhere
template <typename T>
__device__ __noinline__ void fv_outer_sums_tile(const Dev<T>& d, const unsigned char* sm, const TileSmem& L, int r,
                                                int m, T (&fn)[9]) {
    const int cap = d.tile_cap, roff = d.ell_width - 1;
    const T* own = reinterpret_cast<const T*>(sm + L.own);
    const T* halo = reinterpret_cast<const T*>(sm + L.halo);
    const T* ec = reinterpret_cast<const T*>(sm + L.ecoef);
    const uint16_t* ecol = reinterpret_cast<const uint16_t*>(sm + L.ecol);
    const int8_t* kd = reinterpret_cast<const int8_t*>(sm + L.kind);
    const int16_t* om = reinterpret_cast<const int16_t*>(sm + L.omap);
    const T* osn = reinterpret_cast<const T*>(sm + L.osnap);
    const int32_t* hid = reinterpret_cast<const int32_t*>(sm + L.hid);
    FvAcc<T> acc;
    fv_acc_init(acc);
    const int ne = reinterpret_cast<const uint8_t*>(sm + L.cnt)[r];
    for (int j = 0; j < ne; ++j) {
        const int e = j * cap + r;
        const int col = ecol[e];
        T f[9], z[3];
        if (col < cap) {
            if (kd[col] == HLBM_NODE_OUTER) {
                fv_outer_from(d, osn + kSnap * om[col], 1, m, f);
                z_of(f, d.rho0, z);
            } else {
                read_rec12(own + (size_t)kSR * col, f, z);
            }
        } else {
            const int g = hid[col - cap];
            if (d.kind[g] == HLBM_NODE_OUTER) {
                fv_outer(d, g, m, f);
                z_of(f, d.rho0, z);
            } else {
                read_rec12(halo + (size_t)kSR * (col - cap), f, z);
            }
        }
        fv_acc_entry(acc, ec[e], ec[(roff + j) * cap + r], ec[(2 * roff + j) * cap + r], f, z, fn);
    }
    T fP[9], zP[3];
#pragma unroll
    for (int i = 0; i < 9; ++i) fP[i] = fn[i];
    z_of(fP, d.rho0, zP);
    fv_acc_finish(d, acc, reinterpret_cast<const T*>(sm + L.cpp)[r], fP, zP, fn);
}

template <typename T, bool kOuterFv>
__device__ __forceinline__ void fv_update_slot(const Dev<T>& d, const unsigned char* sm, const TileSmem& L, int r, int m,
                                               T (&fn)[9]) {
    const int8_t kind = reinterpret_cast<const int8_t*>(sm + L.kind)[r];
    if (kind == HLBM_NODE_OUTER) {
        const int q = reinterpret_cast<const int16_t*>(sm + L.omap)[r];
        fv_outer_from(d, reinterpret_cast<const T*>(sm + L.osnap) + kSnap * q, 1, m, fn);
        if constexpr (kOuterFv) fv_outer_sums_tile(d, sm, L, r, m, fn);
        return;
    }
    fv_node_tile(d, sm, L, r, fn);
    if (kind == HLBM_NODE_WALL) {
        const T* uv = reinterpret_cast<const T*>(sm + L.uv);
        fv_wall(d, uv[m], uv[d.n_sub + m], fn);
    }
}

template <typename T, bool kOuterFv>
__global__ void __launch_bounds__(kSmemThreads<T>, 1) k_fv_tiles(Dev<T> d, StepArgs a, T* g0, T* g1) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int abort_sh;
    const int cap = d.tile_cap, hcap = d.halo_cap, roff = d.ell_width - 1;
    const TileSmem L = tile_smem_layout<T>(cap, hcap, roff, d.n_sub, d.tile_ocap);
    T* own = reinterpret_cast<T*>(sm + L.own);
    T* halo = reinterpret_cast<T*>(sm + L.halo);
    T* uv = reinterpret_cast<T*>(sm + L.uv);
    int32_t* hid = reinterpret_cast<int32_t*>(sm + L.hid);
    const uint16_t* order = reinterpret_cast<const uint16_t*>(sm + L.order);
    const int8_t* send = reinterpret_cast<const int8_t*>(sm + L.send);
    const int tile = blockIdx.x;
    const int p0 = d.tile_start[tile], p1 = d.tile_start[tile + 1], tile_n = p1 - p0;
    const int h0 = d.halo_ptr[tile], halo_n = d.halo_ptr[tile + 1] - h0;
    const int tid = threadIdx.x, nt = blockDim.x;
    // nodes updated before the halo arrives: the interior ones, but only as
    // many as fill whole rounds of the block, so that the rest (boundary
    // nodes and the remainder) take exactly one more round
    const int rounds = (tile_n + nt - 1) / nt;
    const int n_int = min(d.tile_interior[tile], (rounds - 1) * nt);
    // ---- tile set-up: wall velocity per sub-step, own records (buffer 0),
    // matrices, kinds, send flags, node order, halo ids
    for (int m = tid; m < d.n_sub; m += nt) wall_velocity(d, a, m, uv[m], uv[d.n_sub + m]);
    for (int x = tid; x < 3 * tile_n; x += nt) {
        const int sl = x / 3, c = x - 3 * sl;
        const Vec4<T> v = ld4(g0 + (int64_t)kRec * (p0 + d.tile_order[p0 + sl]) + 4 * c);
        st4(own + (size_t)kSR * sl + 4 * c, v.x, v.y, v.z, v.w);
    }
    {
        const Coef<T>* ell = d.ell + (int64_t)d.ell_width * p0;
        T* ec = reinterpret_cast<T*>(sm + L.ecoef);
        uint16_t* ecol = reinterpret_cast<uint16_t*>(sm + L.ecol);
        T* cpp = reinterpret_cast<T*>(sm + L.cpp);
        for (int x = tid; x < d.ell_width * tile_n; x += nt) {
            const int j = x / tile_n, r = x - j * tile_n;
            const Coef<T> c = ell[x];
            if (j == 0) {
                cpp[r] = c.c;
            } else {
                const int e = (j - 1) * cap + r;
                ecol[e] = (uint16_t)c.col;
                ec[e] = c.gx;
                ec[(roff + j - 1) * cap + r] = c.gy;
                ec[(2 * roff + j - 1) * cap + r] = c.c;
            }
        }
        int8_t* kd = reinterpret_cast<int8_t*>(sm + L.kind);
        int8_t* sd = reinterpret_cast<int8_t*>(sm + L.send);
        uint16_t* od = reinterpret_cast<uint16_t*>(sm + L.order);
        uint8_t* cn = reinterpret_cast<uint8_t*>(sm + L.cnt);
        for (int sl = tid; sl < tile_n; sl += nt) {
            const int r = d.tile_order[p0 + sl];
            kd[sl] = d.kind[p0 + r];
            sd[sl] = d.send[p0 + r];
            od[sl] = (uint16_t)r;
            cn[sl] = (uint8_t)(d.row_ptr[p0 + r + 1] - d.row_ptr[p0 + r] - 1);
        }
        for (int h = tid; h < halo_n; h += nt) hid[h] = d.halo_ids[h0 + h];
        // the outer nodes' feed (written by k_feed before this launch)
        const int o0 = d.tile_outer_ptr[tile], on = d.tile_outer_ptr[tile + 1] - o0;
        int16_t* om = reinterpret_cast<int16_t*>(sm + L.omap);
        T* osn = reinterpret_cast<T*>(sm + L.osnap);
        for (int q = tid; q < on; q += nt) om[d.tile_outer_r[o0 + q]] = (int16_t)q;
        const int64_t no = d.n_outer;
        for (int x = tid; x < kSnap * on; x += nt) {
            const int q = x / kSnap, j = x - kSnap * q;
            osn[x] = d.snap[j * no + d.outer_of[p0 + d.tile_order[p0 + d.tile_outer_r[o0 + q]]]];
        }
    }
    if (tid == 0) abort_sh = 0;
    __syncthreads();
    const unsigned long long base = (unsigned long long)a.t * (unsigned long long)d.n_sub;
    const int nb0 = d.tile_nb_ptr[tile], nb1 = d.tile_nb_ptr[tile + 1];
    for (int m = 0; m < d.n_sub; ++m) {
        T fn[kSlots<T>][9];
        // nodes that read no halo
#pragma unroll
        for (int s = 0; s < kSlots<T>; ++s) {
            const int x = tid + s * nt;
            if (x < n_int) fv_update_slot<T, kOuterFv>(d, sm, L, x, m, fn[s]);
        }
        // warp 0: wait for the neighbour tiles to publish state m (lane l
        // acquires the counters l, l + 32, ...; the warp barrier then orders
        // every lane's later reads after all of them), then copy the halo
        // records into shared memory asynchronously while the other warps
        // still update their nodes
        if (tid < 32) {
            bool ok = true;
            if (m > 0) {
                for (int e = nb0 + tid; e < nb1 && ok; e += 32) {
                    const unsigned long long* pc = d.progress + d.tile_nb[e];
                    long spins = 0;
                    while (ld_acquire(pc) < base + m) {
                        if (*(volatile unsigned*)d.abort_flag) {
                            ok = false;
                            break;
                        }
                        if (++spins > d.spin_limit) {
                            atomicOr(d.status, HLBM_ST_SYNC_TIMEOUT);
                            atomicExch(d.abort_flag, 1u);
                            ok = false;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
            }
            __syncwarp();
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                const T* gin = (m & 1) ? g1 : g0;
                constexpr int kChunks = kSR * (int)sizeof(T) / 16;  // 16-byte pieces of a record
                for (int x = tid; x < kChunks * halo_n; x += 32) {
                    const int h = x / kChunks, c = x - kChunks * h;
                    cp_async16(reinterpret_cast<unsigned char*>(halo) + (size_t)h * kSR * sizeof(T) + 16 * c,
                               reinterpret_cast<const unsigned char*>(gin + (int64_t)kRec * hid[h]) + 16 * c);
                }
            }
            cp_async_wait_all();
            if (tid == 0 && !ok) abort_sh = 1;
        }
        __syncthreads();
        if (abort_sh) return;
        // nodes that read the halo
#pragma unroll
        for (int s = 0; s < kSlots<T>; ++s) {
            const int x = tid + s * nt;
            if (x >= n_int && x < tile_n) fv_update_slot<T, kOuterFv>(d, sm, L, x, m, fn[s]);
        }
        __syncthreads();
        // publish state m+1
        T* gout = (m & 1) ? g0 : g1;
        const bool last = (m == d.n_sub - 1);
#pragma unroll
        for (int s = 0; s < kSlots<T>; ++s) {
            const int x = tid + s * nt;
            if (x < tile_n) {
                T z[3];
                z_of(fn[s], d.rho0, z);
                T* o = own + (size_t)kSR * x;
                st4(o, fn[s][0], fn[s][1], fn[s][2], fn[s][3]);
                st4(o + 4, fn[s][4], fn[s][5], fn[s][6], fn[s][7]);
                st4(o + 8, fn[s][8], z[0], z[1], z[2]);
                if (last || send[x]) {
                    T* rec = gout + (int64_t)kRec * (p0 + order[x]);
                    st4(rec, fn[s][0], fn[s][1], fn[s][2], fn[s][3]);
                    st4(rec + 4, fn[s][4], fn[s][5], fn[s][6], fn[s][7]);
                    st4(rec + 8, fn[s][8], z[0], z[1], z[2]);
                }
            }
        }
        __syncthreads();
        if (tid == 0 && tile != d.stall_tile) {
            __threadfence();
            st_release(d.progress + tile, base + m + 1);
        }
    }
}

// ---------------------------------------------------------------------------
// Tensor-memory variant of k_fv_tiles.  Each thread's own FV rows (per
// off-diagonal entry g_Pk, C_Pk and the tile-local column; C_PP and the
// entry count) live in tensor memory (TMEM), which a thread reads from its
// own lane with tcgen05.ld.  That frees the shared memory the coefficients
// took, so the records are double-buffered: sub-step m reads buffer m%2 and
// each thread writes its nodes' new records into the other buffer as soon
// as they are computed.  A sub-step then needs two block barriers (halo in,
// sub-step done) and no separate publish pass.
//
// TMEM: the block allocates all 512 columns.  Warp w reads lanes
// 32 (w % 4) .. 32 (w % 4) + 31 (one per thread) and its own column range
// kTmemCols<T> * (w / 4) .. + kTmemCols<T>: one slot of kTmemSlotWords<T>
// words per node the thread updates.
template <typename T>
constexpr int kTmemEntryWords = sizeof(T) == 4 ? 4 : 8;  // gx, gy, c, col (FP64: 2 words each, col, pad)
template <typename T>
constexpr int kTmemSlotWords = sizeof(T) == 4 ? 32 : 64;
template <typename T>
constexpr int kTmemCols = kSlots<T> * kTmemSlotWords<T>;
static_assert(1024 / 32 / 4 * kTmemCols<float> == 512, "TMEM columns (FP32)");
static_assert(512 / 32 / 4 * kTmemCols<double> <= 512, "TMEM columns (FP64)");

__device__ __forceinline__ void tmem_alloc_512(uint32_t* smem_dst) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(smem_dst);
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(dst) : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_512(uint32_t taddr) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(taddr) : "memory");
}
__device__ __forceinline__ void tmem_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
// 4 words from this thread's lane, columns taddr .. taddr + 3; complete on return
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, uint32_t (&v)[4]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t (&v)[8]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_st4(uint32_t taddr, uint32_t a, uint32_t b, uint32_t c, uint32_t e) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1, %2, %3, %4};" ::"r"(taddr), "r"(a), "r"(b),
                 "r"(c), "r"(e)
                 : "memory");
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

template <typename T>
__device__ __forceinline__ uint32_t lo_word(T v) {
    if constexpr (sizeof(T) == 4)
        return __float_as_uint(v);
    else
        return (uint32_t)__double2loint(v);
}
template <typename T>
__device__ __forceinline__ uint32_t hi_word(T v) {
    if constexpr (sizeof(T) == 4)
        return 0u;
    else
        return (uint32_t)__double2hiint(v);
}
template <typename T>
__device__ __forceinline__ T from_words(uint32_t lo, uint32_t hi) {
    if constexpr (sizeof(T) == 4)
        return __uint_as_float(lo);
    else
        return __hiloint2double((int)hi, (int)lo);
}

// one FV entry of the thread's slot: (g_x, g_y, C, column)
template <typename T>
__device__ __forceinline__ void tmem_entry(uint32_t taddr, T& gx, T& gy, T& c, int& col) {
    if constexpr (sizeof(T) == 4) {
        uint32_t v[4];
        tmem_ld4(taddr, v);
        gx = from_words<T>(v[0], 0);
        gy = from_words<T>(v[1], 0);
        c = from_words<T>(v[2], 0);
        col = (int)v[3];
    } else {
        uint32_t v[8];
        tmem_ld8(taddr, v);
        gx = from_words<T>(v[0], v[1]);
        gy = from_words<T>(v[2], v[3]);
        c = from_words<T>(v[4], v[5]);
        col = (int)v[6];
    }
}

struct TmemSmem {
    size_t own0, own1, halo, uv, osnap, hid, order, kind, send, omap, total;
};

template <typename T>
__host__ __device__ inline TmemSmem tmem_smem_layout(int cap, int hcap, int n_sub, int ocap) {
    auto up = [](size_t x) { return (x + 15) / 16 * 16; };
    TmemSmem L;
    size_t o = 0;
    L.own0 = o;
    o = up(o + sizeof(T) * kSR * (size_t)cap);
    L.own1 = o;
    o = up(o + sizeof(T) * kSR * (size_t)cap);
    L.halo = o;
    o = up(o + sizeof(T) * kSR * (size_t)hcap);
    L.uv = o;
    o = up(o + sizeof(T) * 2 * (size_t)n_sub);
    L.osnap = o;
    o = up(o + sizeof(T) * kSnap * (size_t)ocap);
    L.hid = o;
    o = up(o + sizeof(int32_t) * (size_t)hcap);
    L.order = o;
    o = up(o + sizeof(uint16_t) * (size_t)cap);
    L.kind = o;
    o = up(o + (size_t)cap);
    L.send = o;
    o = up(o + (size_t)cap);
    L.omap = o;
    o = up(o + sizeof(int16_t) * (size_t)cap);
    L.total = o;
    return L;
}

template <typename T>
size_t fv_tmem_smem_bytes(int tile_cap, int halo_cap, int n_sub, int ocap) {
    return tmem_smem_layout<T>(tile_cap, halo_cap, n_sub, ocap).total;
}

// The update of the node in slot r of a warp-uniform call (lanes with
// valid = false take part in the TMEM loads only) and its write into the
// next record buffer and, when other tiles read it or on the last
// sub-step, into global buffer gout.
template <typename T>
__device__ __forceinline__ void fv_tmem_node(const Dev<T>& d, const unsigned char* sm, const TmemSmem& L,
                                             const T* cur, T* nxt, uint32_t tslot, bool valid, int r, int m, T* gout,
                                             bool last, int p0) {
    const int cap = d.tile_cap;
    const int8_t kind = valid ? reinterpret_cast<const int8_t*>(sm + L.kind)[r] : (int8_t)HLBM_NODE_OUTER;
    uint32_t hdr[4];
    tmem_ld4(tslot + kTmemMaxEntries * kTmemEntryWords<T>, hdr);
    const T cP = from_words<T>(hdr[0], hdr[1]);
    const int ne = (valid && kind != HLBM_NODE_OUTER) ? (int)hdr[2] : 0;
    const int nem = __reduce_max_sync(0xffffffffu, (unsigned)ne);
    T fn[9];
    T fP[9] = {};
    if (valid && kind != HLBM_NODE_OUTER) read_rec9(cur + (size_t)kSR * r, fP);
    FvAcc<T> acc;
    fv_acc_init(acc);
    const T* halo = reinterpret_cast<const T*>(sm + L.halo) - (size_t)kSR * cap;
#pragma unroll
    for (int j = 0; j < kTmemMaxEntries; ++j) {
        if (j >= nem) break;
        T gx, gy, c;
        int col;
        tmem_entry<T>(tslot + j * kTmemEntryWords<T>, gx, gy, c, col);
        if (j < ne) {
            T f[9], z[3];
            read_rec12((col < cap ? cur : halo) + (size_t)kSR * col, f, z);
            fv_acc_entry(acc, gx, gy, c, f, z, fP);
        }
    }
    if (!valid) return;
    if (kind == HLBM_NODE_OUTER) {
        const int q = reinterpret_cast<const int16_t*>(sm + L.omap)[r];
        fv_outer_from(d, reinterpret_cast<const T*>(sm + L.osnap) + kSnap * q, 1, m, fn);
    } else {
        T zP[3];
        read_z3(cur + (size_t)kSR * r, zP);
        fv_acc_finish(d, acc, cP, fP, zP, fn);
        if (kind == HLBM_NODE_WALL) {
            const T* uv = reinterpret_cast<const T*>(sm + L.uv);
            fv_wall(d, uv[m], uv[d.n_sub + m], fn);
        }
    }
    T z[3];
    z_of(fn, d.rho0, z);
    T* o = nxt + (size_t)kSR * r;
    st4(o, fn[0], fn[1], fn[2], fn[3]);
    st4(o + 4, fn[4], fn[5], fn[6], fn[7]);
    st4(o + 8, fn[8], z[0], z[1], z[2]);
    if (last || reinterpret_cast<const int8_t*>(sm + L.send)[r]) {
        T* rec = gout + (int64_t)kRec * (p0 + reinterpret_cast<const uint16_t*>(sm + L.order)[r]);
        st4(rec, fn[0], fn[1], fn[2], fn[3]);
        st4(rec + 4, fn[4], fn[5], fn[6], fn[7]);
        st4(rec + 8, fn[8], z[0], z[1], z[2]);
    }
}

// The body of the tensor-memory FV kernel for tile `tile` of the solver d
// (one block); k_fv_tmem runs one solver, k_fv_tmem_pack several.
template <typename T>
__device__ __forceinline__ void fv_tmem_body(const Dev<T>& d, const StepArgs& a, T* g0, T* g1, const int tile,
                                             unsigned char* sm, int& abort_sh, uint32_t& tmem_base_sh) {
    const int cap = d.tile_cap, hcap = d.halo_cap;
    const TmemSmem L = tmem_smem_layout<T>(cap, hcap, d.n_sub, d.tile_ocap);
    T* own0 = reinterpret_cast<T*>(sm + L.own0);
    T* own1 = reinterpret_cast<T*>(sm + L.own1);
    T* halo = reinterpret_cast<T*>(sm + L.halo);
    T* uv = reinterpret_cast<T*>(sm + L.uv);
    int32_t* hid = reinterpret_cast<int32_t*>(sm + L.hid);
    const int p0 = d.tile_start[tile], p1 = d.tile_start[tile + 1], tile_n = p1 - p0;
    const int h0 = d.halo_ptr[tile], halo_n = d.halo_ptr[tile + 1] - h0;
    const int tid = threadIdx.x, nt = blockDim.x, warp = tid >> 5;
    const int rounds = (tile_n + nt - 1) / nt;
    const int n_int = min(d.tile_interior[tile], (rounds - 1) * nt);
    // ---- TMEM for the block
    if (warp == 0) tmem_alloc_512(&tmem_base_sh);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tbase = tmem_base_sh;
    const uint32_t twarp = tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(kTmemCols<T> * (warp >> 2));
    // ---- set-up: wall velocity, records (buffer 0), kinds, flags, order, halo ids, outer feed
    for (int m = tid; m < d.n_sub; m += nt) wall_velocity(d, a, m, uv[m], uv[d.n_sub + m]);
    for (int x = tid; x < 3 * tile_n; x += nt) {
        const int sl = x / 3, c = x - 3 * sl;
        const Vec4<T> v = ld4(g0 + (int64_t)kRec * (p0 + d.tile_order[p0 + sl]) + 4 * c);
        st4(own0 + (size_t)kSR * sl + 4 * c, v.x, v.y, v.z, v.w);
    }
    {
        int8_t* kd = reinterpret_cast<int8_t*>(sm + L.kind);
        int8_t* sd = reinterpret_cast<int8_t*>(sm + L.send);
        uint16_t* od = reinterpret_cast<uint16_t*>(sm + L.order);
        for (int sl = tid; sl < tile_n; sl += nt) {
            const int r = d.tile_order[p0 + sl];
            kd[sl] = d.kind[p0 + r];
            sd[sl] = d.send[p0 + r];
            od[sl] = (uint16_t)r;
        }
        for (int h = tid; h < halo_n; h += nt) hid[h] = d.halo_ids[h0 + h];
        const int o0 = d.tile_outer_ptr[tile], on = d.tile_outer_ptr[tile + 1] - o0;
        int16_t* om = reinterpret_cast<int16_t*>(sm + L.omap);
        T* osn = reinterpret_cast<T*>(sm + L.osnap);
        for (int q = tid; q < on; q += nt) om[d.tile_outer_r[o0 + q]] = (int16_t)q;
        const int64_t no = d.n_outer;
        for (int x = tid; x < kSnap * on; x += nt) {
            const int q = x / kSnap, j = x - kSnap * q;
            osn[x] = d.snap[j * no + d.outer_of[p0 + d.tile_order[p0 + d.tile_outer_r[o0 + q]]]];
        }
        // this thread's rows into its TMEM slots (every lane stores; lanes
        // without a node store zeros)
        const Coef<T>* ell = d.ell + (int64_t)d.ell_width * p0;
#pragma unroll
        for (int s = 0; s < kSlots<T>; ++s) {
            const int x = tid + s * nt;
            const bool have = x < tile_n;
            const uint32_t tslot = twarp + (uint32_t)(s * kTmemSlotWords<T>);
            const int q = have ? p0 + d.tile_order[p0 + x] : 0;
            const int ne = have ? d.row_ptr[q + 1] - d.row_ptr[q] - 1 : 0;
            for (int j = 0; j < kTmemMaxEntries; ++j) {
                Coef<T> c{};
                c.col = x;
                c.gx = c.gy = c.c = T(0);
                if (have && j < ne) c = ell[(int64_t)(j + 1) * tile_n + x];
                const uint32_t t = tslot + (uint32_t)(j * kTmemEntryWords<T>);
                if constexpr (sizeof(T) == 4) {
                    tmem_st4(t, lo_word(c.gx), lo_word(c.gy), lo_word(c.c), (uint32_t)c.col);
                } else {
                    tmem_st4(t, lo_word(c.gx), hi_word(c.gx), lo_word(c.gy), hi_word(c.gy));
                    tmem_st4(t + 4, lo_word(c.c), hi_word(c.c), (uint32_t)c.col, 0u);
                }
            }
            const T cP = have ? ell[x].c : T(0);
            tmem_st4(tslot + kTmemMaxEntries * kTmemEntryWords<T>, lo_word(cP), hi_word(cP), (uint32_t)ne, 0u);
        }
        tmem_wait_st();
    }
    if (tid == 0) abort_sh = 0;
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned long long base = (unsigned long long)a.t * (unsigned long long)d.n_sub;
    const int nb0 = d.tile_nb_ptr[tile], nb1 = d.tile_nb_ptr[tile + 1];
    for (int m = 0; m < d.n_sub; ++m) {
        const T* cur = (m & 1) ? own1 : own0;
        T* nxt = (m & 1) ? own0 : own1;
        T* gout = (m & 1) ? g0 : g1;
        const bool last = (m == d.n_sub - 1);
        // nodes that read no halo (warp-uniform calls)
#pragma unroll
        for (int s = 0; s < kSlots<T>; ++s) {
            const int x = tid + s * nt;
            const bool v = x < n_int;
            if (__any_sync(0xffffffffu, v))
                fv_tmem_node(d, sm, L, cur, nxt, twarp + (uint32_t)(s * kTmemSlotWords<T>), v, x, m, gout, last,
                             p0);
        }
        // warp 0: neighbour wait and halo copy, as in k_fv_tiles
        if (warp == 0) {
            bool ok = true;
            if (m > 0) {
                for (int e = nb0 + tid; e < nb1 && ok; e += 32) {
                    const unsigned long long* pc = d.progress + d.tile_nb[e];
                    long spins = 0;
                    while (ld_acquire(pc) < base + m) {
                        if (*(volatile unsigned*)d.abort_flag) {
                            ok = false;
                            break;
                        }
                        if (++spins > d.spin_limit) {
                            atomicOr(d.status, HLBM_ST_SYNC_TIMEOUT);
                            atomicExch(d.abort_flag, 1u);
                            ok = false;
                            break;
                        }
                        __nanosleep(32);
                    }
                }
            }
            __syncwarp();
            ok = __all_sync(0xffffffffu, ok);
            if (ok) {
                const T* gin = (m & 1) ? g1 : g0;
                constexpr int kChunks = kSR * (int)sizeof(T) / 16;
                for (int x = tid; x < kChunks * halo_n; x += 32) {
                    const int h = x / kChunks, c = x - kChunks * h;
                    cp_async16(reinterpret_cast<unsigned char*>(halo) + (size_t)h * kSR * sizeof(T) + 16 * c,
                               reinterpret_cast<const unsigned char*>(gin + (int64_t)kRec * hid[h]) + 16 * c);
                }
            }
            cp_async_wait_all();
            if (tid == 0 && !ok) abort_sh = 1;
        }
        __syncthreads();
        if (abort_sh) break;
        // nodes that read the halo
#pragma unroll
        for (int s = 0; s < kSlots<T>; ++s) {
            const int x = tid + s * nt;
            const bool v = x >= n_int && x < tile_n;
            if (__any_sync(0xffffffffu, v))
                fv_tmem_node(d, sm, L, cur, nxt, twarp + (uint32_t)(s * kTmemSlotWords<T>), v, x, m, gout, last,
                             p0);
        }
        __syncthreads();
        if (tid == 0 && tile != d.stall_tile) {
            __threadfence();
            st_release(d.progress + tile, base + m + 1);
        }
    }
    // ---- release TMEM (also after an abort: every warp is past its last tcgen05.ld)
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc_512(tbase);
}

template <typename T>
__global__ void __launch_bounds__(kSmemThreads<T>, 1) k_fv_tmem(Dev<T> d, StepArgs a, T* g0, T* g1) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int abort_sh;
    __shared__ uint32_t tmem_base_sh;
    fv_tmem_body<T>(d, a, g0, g1, blockIdx.x, sm, abort_sh, tmem_base_sh);
}

// Several solvers' FV sub-steps in one cooperative launch: block b runs
// tile b - block0 of the item whose range [block0, next block0) holds b.
// Each item keeps its own tables, counters, sub-step count and buffers;
// items only share the GPU.
template <typename T>
__global__ void __launch_bounds__(kSmemThreads<T>, 1) k_fv_tmem_pack(const __grid_constant__ FvPack<T> pk) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int abort_sh;
    __shared__ uint32_t tmem_base_sh;
    int i = 0;
    while (i + 1 < pk.n && pk.block0[i + 1] <= (int)blockIdx.x) ++i;
    fv_tmem_body<T>(pk.d[i], pk.a[i], pk.g0[i], pk.g1[i], (int)blockIdx.x - pk.block0[i], sm, abort_sh,
                    tmem_base_sh);
}

template <typename T>
cudaError_t launch_fv_tmem_pack(const FvPack<T>& pk, int blocks, size_t smem, cudaStream_t s) {
    FvPack<T> p = pk;
    void* args[] = {&p};
    return cudaLaunchCooperativeKernel((const void*)k_fv_tmem_pack<T>, dim3(blocks), dim3(kSmemThreads<T>), args,
                                       smem, s);
}

template <typename T>
int fv_tmem_tile_capacity(size_t smem) {
    if (smem == 0) return 0;
    int dev = 0, sms = 0, per = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // each block allocates all 512 TMEM columns of its SM, so a second block
    // on the same SM would wait for the first: only run where one fits
    for (const void* fn : {(const void*)k_fv_tmem<T>, (const void*)k_fv_tmem_pack<T>}) {
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const int limit = maxsm - (int)fa.sharedSizeBytes;
        if (smem > (size_t)limit) return 0;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kSmemThreads<T>, smem);
        if (per != 1) return 0;
    }
    return sms;
}

template <typename T>
cudaError_t launch_fv_tmem(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    Dev<T> dd = d;
    StepArgs aa = a;
    T* b0 = (T*)d.fu_in;
    T* b1 = d.fu_out;
    void* args[] = {&dd, &aa, &b0, &b1};
    size_t smem = fv_tmem_smem_bytes<T>(d.tile_cap, d.halo_cap, d.n_sub, d.tile_ocap);
    return cudaLaunchCooperativeKernel((const void*)k_fv_tmem<T>, dim3(d.n_tiles), dim3(kSmemThreads<T>), args, smem,
                                       s);
}

// ---------------------------------------------------------------------------
// Deep tiles: the FV sub-steps with one exchange between tiles every K
// sub-steps (temporal blocking).  A tile holds, as local "slots", its own
// nodes and K layers of ghost nodes around them: layer j holds the nodes
// that the updates of layer j-1 read and that are not in earlier layers
// (outer nodes read nothing).  Sub-step s of a block of K recomputes the
// own nodes and ghost layers 1 .. K-1-s from the tile's own data, so the
// tile needs its neighbours' records only once per block: the own nodes
// other tiles hold as ghosts are written to the global record buffer at the
// end of a block, the tile releases its progress counter, and at the start
// of the next block each tile fetches its ghost layers after acquiring its
// neighbour tiles' counters.  Meanwhile the threads update the own nodes
// whose rows read only own nodes (slots [0, n_a)); then one block barrier
// per sub-step.  The arithmetic of a node is that of the other FV kernels
// (fv_acc_*, same entry order), so the results are the same bit for bit.
//
// Slots: own nodes (those reading only own nodes first), then the ghost
// layers in order.  Records of all slots are double-buffered in shared
// memory; the FV rows of the computed slots live in tensor memory, one row
// image per slot (header cP, ne, then per off-diagonal entry gx, gy, C and
// the local slot of the column; FP64 values take two words).  Slot x is
// updated by thread x % kDeepThreads, which reads its row image from its
// own TMEM lane: FP32 runs 768 FV threads of two slots and loads a row
// entry by entry (64 registers), FP64 512 threads of two slots that load a
// row in two halves.  The FP32 block has 256 more threads (8 warps) that run
// the next lattice step's stream-collide away from the patch (FarArgs)
// while the FV warps step the patch: the FV work is latency-bound and the
// lattice work bandwidth-bound, so they share the SM.  On the 4096^2
// workload 768 FV threads of exactly two slots each also beat 1024 of one
// or two (0.416 against 0.423 ms per step).
template <typename T>
constexpr int kDeepThreads = sizeof(T) == 4 ? 1024 : 512;  // block size
template <typename T>
constexpr int kDeepFv = sizeof(T) == 4 ? 768 : 512;  // FV threads: warps 0 .. kDeepFv / 32 - 1
template <typename T>
constexpr int kDeepSlotWords = sizeof(T) == 4 ? 32 : 64;  // TMEM columns of one slot
template <typename T>
constexpr int kDeepGroups = 2;  // slots per FV thread
template <typename T>
constexpr int kDeepHalf = kDeepSlotWords<T> / 2;  // words per tcgen05.ld of a row
template <typename T>
constexpr int kDeepEntryWords = sizeof(T) == 4 ? 4 : 8;
static_assert(kDeepSlotWords<float> * (kDeepGroups<float> * kDeepFv<float> / 128) <= 512 &&
                  kDeepSlotWords<double> * (kDeepGroups<double> * kDeepFv<double> / 128) <= 512,
              "row images of all slots within the 512 TMEM columns");
static_assert(1 + kTmemMaxEntries <= 8, "row image: header and 7 entries");

template <typename T>
int fv_deep_tmem_slots() {
    return kDeepGroups<T> * kDeepFv<T>;
}
template <typename T>
int fv_deep_row_words() {
    return kDeepSlotWords<T>;
}

struct DeepSmem {
    size_t buf0, buf1, uv, osnap, gid, kind, send, omap, total;
};

template <typename T>
__host__ __device__ inline DeepSmem deep_smem_layout(int cap, int n_sub, int ocap) {
    auto up = [](size_t x) { return (x + 15) / 16 * 16; };
    DeepSmem L;
    size_t o = 0;
    L.buf0 = o;
    o = up(o + sizeof(T) * kSR * (size_t)cap);
    L.buf1 = o;
    o = up(o + sizeof(T) * kSR * (size_t)cap);
    L.uv = o;
    o = up(o + sizeof(T) * 2 * (size_t)n_sub);
    L.osnap = o;
    o = up(o + sizeof(T) * kSnap * (size_t)ocap);
    L.gid = o;
    o = up(o + sizeof(int32_t) * (size_t)cap);
    L.kind = o;
    o = up(o + (size_t)cap);
    L.send = o;
    o = up(o + (size_t)cap);
    L.omap = o;
    o = up(o + sizeof(int16_t) * (size_t)cap);
    L.total = o;
    return L;
}

template <typename T>
size_t fv_deep_smem_bytes(int slot_cap, int n_sub, int ocap) {
    return deep_smem_layout<T>(slot_cap, n_sub, ocap).total;
}

// 16 or 32 words of this thread's TMEM lane, complete on return
template <int N>
__device__ __forceinline__ void tmem_ldn(uint32_t taddr, uint32_t (&v)[N]) {
    if constexpr (N == 16) {
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15}, [%16];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr)
            : "memory");
    } else {
        static_assert(N == 32, "x16 or x32");
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, "
            "%14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n\t"
            "tcgen05.wait::ld.sync.aligned;"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
              "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]),
              "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]),
              "=r"(v[30]), "=r"(v[31])
            : "r"(taddr)
            : "memory");
    }
}

// entry (gx, gy, C, column) at word w of a row image half
template <typename T, int N>
__device__ __forceinline__ void deep_entry(const uint32_t (&v)[N], int w, T& gx, T& gy, T& c, int& col) {
    if constexpr (sizeof(T) == 4) {
        gx = __uint_as_float(v[w]);
        gy = __uint_as_float(v[w + 1]);
        c = __uint_as_float(v[w + 2]);
        col = (int)v[w + 3];
    } else {
        gx = from_words<T>(v[w], v[w + 1]);
        gy = from_words<T>(v[w + 2], v[w + 3]);
        c = from_words<T>(v[w + 4], v[w + 5]);
        col = (int)v[w + 6];
    }
}

// The update of slot x (warp-uniform call: lanes with valid = false take
// part in the TMEM loads only), written into the next record buffer and,
// when out is set, into the global record of its node.  Both halves of the
// row image are loaded by every lane of the warp at points where the warp
// is converged (tcgen05.ld is .sync.aligned); only the arithmetic between
// them is predicated.
template <typename T>
__device__ __forceinline__ void deep_node(const Dev<T>& d, const unsigned char* sm, const DeepSmem& L, const T* cur,
                                          T* nxt, uint32_t tslot, bool valid, int x, int m, T* gout, bool out) {
    constexpr int EW = kDeepEntryWords<T>;
    const int8_t kind = valid ? reinterpret_cast<const int8_t*>(sm + L.kind)[x] : (int8_t)HLBM_NODE_OUTER;
    T fP[9] = {};
    if (valid && kind != HLBM_NODE_OUTER) read_rec9(cur + (size_t)kSR * x, fP);
    FvAcc<T> acc;
    fv_acc_init(acc);
    T cP;
    if constexpr (sizeof(T) == 4) {
        // header, then the entries one by one up to the warp's longest row
        uint32_t hdr[4];
        tmem_ld4(tslot, hdr);
        cP = __uint_as_float(hdr[0]);
        const int ne = kind != HLBM_NODE_OUTER ? (int)hdr[1] : 0;
        const int nem = (int)__reduce_max_sync(0xffffffffu, (unsigned)ne);
        // two entries per tensor-memory load (one wait for both; entry 7 of
        // the last pair reads the next columns, which no row uses)
#pragma unroll
        for (int j = 0; j < kTmemMaxEntries; j += 2) {
            if (j >= nem) break;
            uint32_t e[8];
            tmem_ld8(tslot + EW * (j + 1), e);
            if (j < ne) {
                T f[9], z[3];
                read_rec12(cur + (size_t)kSR * (int)e[3], f, z);
                fv_acc_entry(acc, __uint_as_float(e[0]), __uint_as_float(e[1]), __uint_as_float(e[2]), f, z, fP);
            }
            if (j + 1 < ne) {
                T f[9], z[3];
                read_rec12(cur + (size_t)kSR * (int)e[7], f, z);
                fv_acc_entry(acc, __uint_as_float(e[4]), __uint_as_float(e[5]), __uint_as_float(e[6]), f, z, fP);
            }
        }
    } else {
        constexpr int H = kDeepHalf<T>;
        constexpr int E0 = H / EW - 1;  // entries in the first half (after the header)
        uint32_t v[H];
        tmem_ldn<H>(tslot, v);
        cP = from_words<T>(v[0], v[1]);
        const int ne = kind != HLBM_NODE_OUTER ? (int)v[2] : 0;
#pragma unroll
        for (int j = 0; j < E0; ++j) {
            if (j < ne) {
                T gx, gy, c;
                int col;
                deep_entry<T, H>(v, EW * (j + 1), gx, gy, c, col);
                T f[9], z[3];
                read_rec12(cur + (size_t)kSR * col, f, z);
                fv_acc_entry(acc, gx, gy, c, f, z, fP);
            }
        }
        __syncwarp();
        tmem_ldn<H>(tslot + H, v);  // entries E0 .. 6
#pragma unroll
        for (int j = E0; j < kTmemMaxEntries; ++j) {
            if (j < ne) {
                T gx, gy, c;
                int col;
                deep_entry<T, H>(v, EW * (j - E0), gx, gy, c, col);
                T f[9], z[3];
                read_rec12(cur + (size_t)kSR * col, f, z);
                fv_acc_entry(acc, gx, gy, c, f, z, fP);
            }
        }
    }
    if (!valid) return;
    T fn[9];
    if (kind == HLBM_NODE_OUTER) {
        const int q = reinterpret_cast<const int16_t*>(sm + L.omap)[x];
        fv_outer_from(d, reinterpret_cast<const T*>(sm + L.osnap) + kSnap * q, 1, m, fn);
    } else {
        T zP[3];
        read_z3(cur + (size_t)kSR * x, zP);
        fv_acc_finish(d, acc, cP, fP, zP, fn);
        if (kind == HLBM_NODE_WALL) {
            const T* uv = reinterpret_cast<const T*>(sm + L.uv);
            fv_wall(d, uv[m], uv[d.n_sub + m], fn);
        }
    }
    T z[3];
    z_of(fn, d.rho0, z);
    T* o = nxt + (size_t)kSR * x;
    st4(o, fn[0], fn[1], fn[2], fn[3]);
    st4(o + 4, fn[4], fn[5], fn[6], fn[7]);
    st4(o + 8, fn[8], z[0], z[1], z[2]);
    if (out) {
        T* rec = gout + (int64_t)kRec * reinterpret_cast<const int32_t*>(sm + L.gid)[x];
        st4(rec, fn[0], fn[1], fn[2], fn[3]);
        st4(rec + 4, fn[4], fn[5], fn[6], fn[7]);
        st4(rec + 8, fn[8], z[0], z[1], z[2]);
    }
}

// One chunk of the next lattice step's stream-collide (FarArgs, FP32
// storage) on the lattice warps: row y = c / n_seg, nodes [64 seg,
// 64 seg + 64), two per lane.  The pull and BGK arithmetic of a node is that
// of k_stream_collide (the same pulled values through bgk_dev; edge nodes
// through pull_edge), so the results are the same bits.  Every lane of the
// warp takes part in the loads and shuffles; only lanes whose nodes lie
// outside the rectangle store.  (Staging the rows in shared memory with
// cp.async, two chunks per warp, measured slower: the FV tile leaves about
// 50 KB of shared memory, too little to keep more loads in flight.)
__device__ __forceinline__ void far_chunk(const Dev<float>& d, const FarArgs<float>& far, int c, int lane) {
    const int y = c / far.n_seg, seg = c - y * far.n_seg;
    const int x0 = 64 * seg + 2 * lane;
    const bool rows_out = y < far.ey0 || y >= far.ey1;
    if (!rows_out && 64 * seg >= far.ex0 && 64 * seg + 64 <= far.ex1) return;  // the whole chunk inside
    const bool mine = x0 < d.nx && (rows_out || x0 < far.ex0 || x0 >= far.ex1);
    const bool interior = x0 >= 1 && x0 + 2 <= d.nx - 1 && y >= 1 && y <= d.ny - 2;
    const float* __restrict__ A = far.src;
    float* __restrict__ B = far.dst;
    const float omega = 1.0f / d.tau_s;
    float2 p[9];
    float edge[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int sy = y - cy_of(i);
        sy = sy < 0 ? 0 : (sy >= d.ny ? d.ny - 1 : sy);
        const int64_t row = i * d.plane + (int64_t)sy * d.pitch;
        const int xv = x0 < d.pitch ? x0 : d.pitch - 2;
        p[i] = *reinterpret_cast<const float2*>(A + row + xv);
        if (cx_of(i) == 1) {
            edge[i] = __shfl_up_sync(0xffffffffu, p[i].y, 1);
            if (lane == 0) edge[i] = A[row + (xv > 0 ? xv - 1 : 0)];
        } else if (cx_of(i) == -1) {
            edge[i] = __shfl_down_sync(0xffffffffu, p[i].x, 1);
            if (lane == 31) edge[i] = A[row + (xv + 2 < d.pitch ? xv + 2 : d.pitch - 1)];
        }
    }
    if (!mine) return;
    if (interior) {
        float f[9], o0[9], o1[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = cx_of(i) == 0 ? p[i].x : (cx_of(i) == 1 ? edge[i] : p[i].y);
        bgk_dev(f, d.rho0, omega, o0);
#pragma unroll
        for (int i = 0; i < 9; ++i) f[i] = cx_of(i) == 0 ? p[i].y : (cx_of(i) == 1 ? p[i].x : edge[i]);
        bgk_dev(f, d.rho0, omega, o1);
        const int64_t s0 = (int64_t)y * d.pitch + x0;
#pragma unroll
        for (int i = 0; i < 9; ++i) *reinterpret_cast<float2*>(B + i * d.plane + s0) = make_float2(o0[i], o1[i]);
    } else {
        for (int k = 0; k < 2; ++k) {
            const int x = x0 + k;
            if (x >= d.nx) break;
            float g[9], o[9];
#pragma unroll
            for (int i = 0; i < 9; ++i) g[i] = pull_edge<float, float>(d, A, x, y, i);
            bgk_dev(g, d.rho0, omega, o);
#pragma unroll
            for (int i = 0; i < 9; ++i) B[i * d.plane + (int64_t)y * d.pitch + x] = o[i];
        }
    }
}

// the FV warps' barrier (named barrier 1; the lattice warps never join it)
template <int N>
__device__ __forceinline__ void fv_bar() {
    asm volatile("bar.sync 1, %0;" ::"n"(N) : "memory");
}

template <typename T>
__global__ void __launch_bounds__(kDeepThreads<T>, 1) k_fv_deep(Dev<T> d, StepArgs a, T* g0, T* g1, FarArgs<T> far) {
    extern __shared__ __align__(16) unsigned char sm[];
    __shared__ int abort_sh;
    __shared__ uint32_t tmem_base_sh;
    constexpr int NT = kDeepFv<T>, BT = kDeepThreads<T>, G = kDeepGroups<T>, SW = kDeepSlotWords<T>;
    const int tile = blockIdx.x, tid = threadIdx.x, warp = tid >> 5;
    const int s0 = d.deep_ptr[tile];
    const int32_t* cnt = d.deep_cnt + kDeepCnt * tile;
    const int n_a = cnt[0], n_own = cnt[1], n_slot = cnt[2];
    const int K = d.deep_k;
    const DeepSmem L = deep_smem_layout<T>(d.deep_slot_cap, d.n_sub, d.deep_ocap);
    T* buf0 = reinterpret_cast<T*>(sm + L.buf0);
    T* buf1 = reinterpret_cast<T*>(sm + L.buf1);
    T* uv = reinterpret_cast<T*>(sm + L.uv);
    int32_t* gid = reinterpret_cast<int32_t*>(sm + L.gid);
    int8_t* kd = reinterpret_cast<int8_t*>(sm + L.kind);
    int8_t* sd = reinterpret_cast<int8_t*>(sm + L.send);
    int16_t* om = reinterpret_cast<int16_t*>(sm + L.omap);
    // ---- tensor memory: all 512 columns; warp w reads lanes 32 (w % 4) ..
    // and, for its slot group j, the columns SW (j NT / 128 + w / 4) ..
    if (warp == 0) tmem_alloc_512(&tmem_base_sh);
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const uint32_t tbase = tmem_base_sh;
    auto tslot_of = [&](int j) {
        return tbase + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)(SW * (j * (NT / 128) + (warp >> 2)));
    };
    // ---- set-up: wall velocity per sub-step, slot tables, records of every
    // slot at sub-step 0, the outer nodes' feed, the row images
    for (int m = tid; m < d.n_sub; m += BT) wall_velocity(d, a, m, uv[m], uv[d.n_sub + m]);
    for (int x = tid; x < n_slot; x += BT) {
        const int g = d.deep_gid[s0 + x];
        gid[x] = g;
        kd[x] = d.kind[g];
        sd[x] = d.deep_send[s0 + x];
        om[x] = -1;
    }
    __syncthreads();
    for (int x = tid; x < 3 * n_slot; x += BT) {
        const int sl = x / 3, c = x - 3 * sl;
        const Vec4<T> v = ld4(g0 + (int64_t)kRec * gid[sl] + 4 * c);
        st4(buf0 + (size_t)kSR * sl + 4 * c, v.x, v.y, v.z, v.w);
    }
    {
        const int o0 = d.deep_optr[tile], on = d.deep_optr[tile + 1] - o0;
        T* osn = reinterpret_cast<T*>(sm + L.osnap);
        for (int q = tid; q < on; q += BT) om[d.deep_oslot[o0 + q]] = (int16_t)q;
        const int64_t no = d.n_outer;
        for (int x = tid; x < kSnap * on; x += BT) {
            const int q = x / kSnap, j = x - kSnap * q;
            osn[x] = d.snap[j * no + d.outer_of[gid[d.deep_oslot[o0 + q]]]];
        }
        // row images of the computed slots (lanes without one store zeros;
        // FV warps only)
        const int n_comp = cnt[3];
        const uint4* rows = reinterpret_cast<const uint4*>(d.deep_rows) + (int64_t)(SW / 4) * d.deep_rptr[tile];
#pragma unroll 1
        for (int j = 0; j < G && tid < NT; ++j) {
            const int x = j * NT + tid;
            const bool have = x < n_comp;
            const uint32_t ts = tslot_of(j);
#pragma unroll 1
            for (int w4 = 0; w4 < SW / 4; ++w4) {
                uint4 u = make_uint4(0u, 0u, 0u, 0u);
                if (have) u = rows[(int64_t)(SW / 4) * x + w4];
                tmem_st4(ts + 4 * w4, u.x, u.y, u.z, u.w);
            }
        }
        tmem_wait_st();
    }
    if (tid == 0) abort_sh = 0;
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    const unsigned long long base = (unsigned long long)a.t * (unsigned long long)d.n_sub;
    if (tid < NT) {
        const int nb0 = d.tile_nb_ptr[tile], nb1 = d.tile_nb_ptr[tile + 1];
        int m = 0;
        bool aborted = false;
        for (int b = 0; m < d.n_sub && !aborted; ++b) {
            const int kb = min(K, d.n_sub - m);
            const bool final_block = (m + kb == d.n_sub);
            T* gout = (b & 1) ? g0 : g1;  // the state at the end of block b is exchange b + 1
            for (int s = 0; s < kb; ++s, ++m) {
                T* cur = (m & 1) ? buf1 : buf0;
                T* nxt = (m & 1) ? buf0 : buf1;
                const bool last = (s == kb - 1);
                const int cs = cnt[3 + s];
                int lo = 0;
                if (s == 0 && b > 0) {
                    // own nodes that read only own nodes, while warp 0 waits for
                    // the neighbour tiles' exchange b and copies the ghost layers
    #pragma unroll
                    for (int j = 0; j < G; ++j) {
                        const int x = j * NT + tid;
                        const bool v = x < n_a;
                        if (__any_sync(0xffffffffu, v))
                            deep_node(d, sm, L, cur, nxt, tslot_of(j), v, x, m, gout, false);
                    }
                    if (warp == 0) {
                        bool ok = true;
                        for (int e = nb0 + tid; e < nb1 && ok; e += 32) {
                            const unsigned long long* pc = d.progress + d.tile_nb[e];
                            long spins = 0;
                            while (ld_acquire(pc) < base + m) {
                                if (*(volatile unsigned*)d.abort_flag) {
                                    ok = false;
                                    break;
                                }
                                if (++spins > d.spin_limit) {
                                    atomicOr(d.status, HLBM_ST_SYNC_TIMEOUT);
                                    atomicExch(d.abort_flag, 1u);
                                    ok = false;
                                    break;
                                }
                                __nanosleep(32);
                            }
                        }
                        __syncwarp();
                        ok = __all_sync(0xffffffffu, ok);
                        if (ok) {
                            const T* gin = (b & 1) ? g1 : g0;
                            constexpr int kChunks = kSR * (int)sizeof(T) / 16;
                            for (int x = tid; x < kChunks * (n_slot - n_own); x += 32) {
                                const int hs = x / kChunks, c = x - kChunks * hs;
                                const int sl = n_own + hs;
                                cp_async16(reinterpret_cast<unsigned char*>(cur + (size_t)kSR * sl) + 16 * c,
                                           reinterpret_cast<const unsigned char*>(gin + (int64_t)kRec * gid[sl]) + 16 * c);
                            }
                        }
                        cp_async_wait_all();
                        if (tid == 0 && !ok) abort_sh = 1;
                    }
                    fv_bar<NT>();
                    if (abort_sh) {
                        aborted = true;
                        break;
                    }
                    // a block of one sub-step ends here: the records of those nodes go
                    // to the exchange buffer only now, after the neighbours' counters
                    // were acquired (a neighbour may still have been reading that
                    // buffer's previous contents, two exchanges back, before)
                    if (last) {
                        for (int x = tid; x < n_a; x += NT) {
                            if (!final_block && !sd[x]) continue;
                            const T* r = nxt + (size_t)kSR * x;
                            T* rec = gout + (int64_t)kRec * gid[x];
                            const Vec4<T> a0 = ld4(r), a1 = ld4(r + 4), a2 = ld4(r + 8);
                            st4(rec, a0.x, a0.y, a0.z, a0.w);
                            st4(rec + 4, a1.x, a1.y, a1.z, a1.w);
                            st4(rec + 8, a2.x, a2.y, a2.z, a2.w);
                        }
                    }
                    lo = n_a;
                }
    #pragma unroll
                for (int j = 0; j < G; ++j) {
                    const int x = j * NT + tid;
                    const bool v = x >= lo && x < cs;
                    if (__any_sync(0xffffffffu, v))
                        deep_node(d, sm, L, cur, nxt, tslot_of(j), v, x, m, gout,
                                  last && x < n_own && (final_block || sd[x]));
                }
                fv_bar<NT>();
            }
            if (!aborted && !final_block && tid == 0 && tile != d.stall_tile) {
                __threadfence();
                st_release(d.progress + tile, base + m);
            }
        }
    } else if constexpr (sizeof(T) == 4) {
        // lattice warps: chunks of the next step's stream-collide until none is left
        const int lane = tid & 31;
        for (; far.n_chunks > 0;) {
            int c = 0;
            if (lane == 0) c = (int)atomicAdd(far.next, 1u);
            c = __shfl_sync(0xffffffffu, c, 0);
            if (c >= far.n_chunks) break;
            far_chunk(d, far, c, lane);
        }
    }
    // ---- release TMEM (also after an abort: every warp is past its last tcgen05.ld)
    tmem_fence_before();
    __syncthreads();
    tmem_fence_after();
    if (warp == 0) tmem_dealloc_512(tbase);
}

template <typename T>
int fv_deep_tile_capacity(size_t smem) {
    if (smem == 0) return 0;
    int dev = 0, sms = 0, per = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, (const void*)k_fv_deep<T>) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const int limit = maxsm - (int)fa.sharedSizeBytes;
    if (smem > (size_t)limit) return 0;
    if (cudaFuncSetAttribute((const void*)k_fv_deep<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) !=
        cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    // each block allocates all 512 TMEM columns: only one block per SM
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_fv_deep<T>, kDeepThreads<T>, smem);
    return per == 1 ? sms : 0;
}

template <typename T>
cudaError_t launch_fv_deep(const Dev<T>& d, const StepArgs& a, const FarArgs<T>* far, cudaStream_t s) {
    Dev<T> dd = d;
    StepArgs aa = a;
    T* b0 = (T*)d.fu_in;
    T* b1 = d.fu_out;
    FarArgs<T> fa{};
    if (far && sizeof(T) == 4) fa = *far;
    void* args[] = {&dd, &aa, &b0, &b1, &fa};
    const size_t smem = fv_deep_smem_bytes<T>(d.deep_slot_cap, d.n_sub, d.deep_ocap);
    return cudaLaunchCooperativeKernel((const void*)k_fv_deep<T>, dim3(d.n_tiles), dim3(kDeepThreads<T>), args, smem,
                                       s);
}

// Row image of computed slot i: header (C_PP, entry count), then the
// off-diagonal entries of row gid[i] in row order with their local columns.
template <typename T>
__global__ void k_build_deep_rows(Dev<T> d, const int32_t* gid, const int32_t* lcol, int64_t count,
                                  uint32_t* rows) {
    const int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    constexpr int SW = kDeepSlotWords<T>, EW = kDeepEntryWords<T>;
    uint32_t* r = rows + (int64_t)SW * i;
    for (int w = 0; w < SW; ++w) r[w] = 0u;
    const int P = gid[i];
    const int r0 = d.row_ptr[P], ne = d.row_ptr[P + 1] - r0 - 1;
    const T cP = d.coef[r0].c;
    r[0] = lo_word(cP);
    if constexpr (sizeof(T) == 4) {
        r[1] = (uint32_t)ne;
    } else {
        r[1] = hi_word(cP);
        r[2] = (uint32_t)ne;
    }
    for (int j = 0; j < ne && j < kTmemMaxEntries; ++j) {
        const Coef<T> c = d.coef[r0 + 1 + j];
        uint32_t* e = r + EW * (j + 1);
        e[0] = lo_word(c.gx);
        if constexpr (sizeof(T) == 4) {
            e[1] = lo_word(c.gy);
            e[2] = lo_word(c.c);
            e[3] = (uint32_t)lcol[(int64_t)kTmemMaxEntries * i + j];
        } else {
            e[1] = hi_word(c.gx);
            e[2] = lo_word(c.gy);
            e[3] = hi_word(c.gy);
            e[4] = lo_word(c.c);
            e[5] = hi_word(c.c);
            e[6] = (uint32_t)lcol[(int64_t)kTmemMaxEntries * i + j];
        }
    }
}

template <typename T>
void launch_build_deep_rows(const Dev<T>& d, const int32_t* gid, const int32_t* lcol, int64_t count, uint32_t* rows,
                            cudaStream_t s) {
    if (count > 0) k_build_deep_rows<T><<<(unsigned)((count + 127) / 128), 128, 0, s>>>(d, gid, lcol, count, rows);
}

// ELL copy of the FV matrices for the shared-memory kernel: entry i takes
// CSR entry src[i] with tile-local column col[i] (src -1: padding, zero)
template <typename T>
__global__ void k_build_ell(const Coef<T>* coef, const int32_t* src, const int32_t* col, Coef<T>* ell, int64_t count) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= count) return;
    Coef<T> c;
    c.col = col[i];
    c.gx = c.gy = c.c = T(0);
    if (src[i] >= 0) {
        const Coef<T> s = coef[src[i]];
        c.gx = s.gx;
        c.gy = s.gy;
        c.c = s.c;
    }
    ell[i] = c;
}

template <typename T>
void launch_build_ell(const Coef<T>* coef, const int32_t* src, const int32_t* col, Coef<T>* ell, int64_t count,
                      cudaStream_t s) {
    k_build_ell<T><<<(unsigned)((count + 255) / 256), 256, 0, s>>>(coef, src, col, ell, count);
}

template <typename T>
int fv_smem_tile_capacity(size_t smem) {
    if (smem == 0) return 0;
    int dev = 0, sms = 0, per = 0, maxsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    // the opt-in maximum less the kernel's static shared memory, so that
    // solvers with different tile sizes can all launch; residency follows
    // from the bytes each launch asks for
    int cap = 1 << 30;
    for (const void* fn : {(const void*)k_fv_tiles<T, false>, (const void*)k_fv_tiles<T, true>}) {
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const int limit = maxsm - (int)fa.sharedSizeBytes;
        if (smem > (size_t)limit) return 0;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, limit) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, kSmemThreads<T>, smem);
        cap = std::min(cap, sms * per);
    }
    return cap;
}

template <typename T>
cudaError_t launch_fv_smem(const Dev<T>& d, const StepArgs& a, cudaStream_t s) {
    Dev<T> dd = d;
    StepArgs aa = a;
    T* b0 = (T*)d.fu_in;
    T* b1 = d.fu_out;
    void* args[] = {&dd, &aa, &b0, &b1};
    size_t smem = fv_smem_bytes<T>(d.tile_cap, d.halo_cap, d.ell_width - 1, d.n_sub, d.tile_ocap);
    const void* fn = d.outer_fv ? (const void*)k_fv_tiles<T, true> : (const void*)k_fv_tiles<T, false>;
    return cudaLaunchCooperativeKernel(fn, dim3(d.n_tiles), dim3(kSmemThreads<T>), args, smem, s);
}

// ------------------------------------------------------------- force
// Stress at wall nodes, sigma = -(rho - rho0) c_s^2 I - sum_i f^neq_i c_i c_i,
// integrated by the trapezoid rule over the wall segments with the body's
// outward normal (force of the fluid on the lamina, per unit length).
template <typename T>
__device__ void wall_stress(const Dev<T>& d, int P, double s[3]) {
    T f[9];
    load_f(d.fu_in + (int64_t)kRec * P, f);
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
    load_f(d.fu_in + (int64_t)kRec * P, f);
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

// ------------------------------------------------------------ adjoint
// Reverse mode of one lattice step, with every decision of the forward step
// held fixed (node classes, refill types, donor cells and triangles: the map
// is smooth in the states and parameters between decisions).  All adjoints
// are FP64.  Notation: for a deviation set f (f_i = f'_i), rho = rho0 + dr,
// u = j / rho; the equilibrium's derivatives are
//   d feq_i / d dr |_u = A_i = w_i (1 + 3 c.u + 4.5 (c.u)^2 - 1.5 u^2),
//   d feq_i / d u      = B_i = w_i rho (3 c_i + 9 (c.u) c_i - 3 u),
// so that d feq_i / d f_j = A_i + B_i . (c_j - u) / rho, and the transpose
// product is (J^T l)_j = a + b . (c_j - u) / rho with a = sum_i l_i A_i,
// b = sum_i l_i B_i.
template <typename R>
__device__ __forceinline__ void feq_ab(int i, R rho, R ux, R uy, R& A, R& Bx, R& By) {
    const R w = w_of<R>(i), cx = R(cx_of(i)), cy = R(cy_of(i));
    const R cu = cx * ux + cy * uy, usq = ux * ux + uy * uy;
    A = w * (R(1) + R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq);
    Bx = w * rho * (R(3) * cx + R(9) * cu * cx - R(3) * ux);
    By = w * rho * (R(3) * cy + R(9) * cu * cy - R(3) * uy);
}

template <typename R>
__device__ __forceinline__ void mom_d(const R (&f)[9], R rho0, R& dr, R& rho, R& ux, R& uy) {
    R r = 0, jx = 0, jy = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        r += f[i];
        jx += R(cx_of(i)) * f[i];
        jy += R(cy_of(i)) * f[i];
    }
    dr = r;
    rho = rho0 + r;
    ux = jx / rho;
    uy = jy / rho;
}

template <typename R>
__device__ __forceinline__ R feq_d(int i, R dr, R rho, R ux, R uy) {
    const R cu = R(cx_of(i)) * ux + R(cy_of(i)) * uy, usq = ux * ux + uy * uy;
    return w_of<R>(i) * (dr + rho * (R(3) * cu + R(4.5) * cu * cu - R(1.5) * usq));
}

// out += scale * J_feq(f)^T lam, J at the moments (dr, rho, u) of f
template <typename R>
__device__ __forceinline__ void jfeqT_add(R rho, R ux, R uy, const R (&lam)[9], R scale, R (&out)[9]) {
    R a = 0, bx = 0, by = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        R A, Bx, By;
        feq_ab(i, rho, ux, uy, A, Bx, By);
        a += lam[i] * A;
        bx += lam[i] * Bx;
        by += lam[i] * By;
    }
#pragma unroll
    for (int j = 0; j < 9; ++j) out[j] += scale * (a + (bx * (R(cx_of(j)) - ux) + by * (R(cy_of(j)) - uy)) / rho);
}

// the interpolated state s(f) = (dr, ux, uy, f^neq[9]) of a deviation set
template <typename R>
__device__ __forceinline__ void state_d(const R (&f)[9], R rho0, R (&st)[12]) {
    R dr, rho, ux, uy;
    mom_d(f, rho0, dr, rho, ux, uy);
    st[0] = dr;
    st[1] = ux;
    st[2] = uy;
#pragma unroll
    for (int i = 0; i < 9; ++i) st[3 + i] = f[i] - feq_d(i, dr, rho, ux, uy);
}

// out += scale * (d s / d f)^T ls
template <typename R>
__device__ __forceinline__ void stateT_add(const R (&f)[9], R rho0, const R (&ls)[12], R scale, R (&out)[9]) {
    R dr, rho, ux, uy;
    mom_d(f, rho0, dr, rho, ux, uy);
    R ln[9];
#pragma unroll
    for (int j = 0; j < 9; ++j) {
        ln[j] = ls[3 + j];
        out[j] += scale * (ls[0] + (ls[1] * (R(cx_of(j)) - ux) + ls[2] * (R(cy_of(j)) - uy)) / rho + ls[3 + j]);
    }
    jfeqT_add(rho, ux, uy, ln, -scale, out);
}

// f = f^eq(st) + k f^neq(st) (eq. continuity_stresses with k = 1 - 1/(2 tau_s),
// eq. postcollision2_s with k = 2 (tau_s - 1)/(2 tau_s - 1)): ls = (d f / d st)^T lf,
// lk += d f / d k . lf
template <typename R>
__device__ __forceinline__ void ffsT(const R (&st)[12], R rho0, R k, const R (&lf)[9], R (&ls)[12], double& lk) {
    const R rho = rho0 + st[0];
    R a = 0, bx = 0, by = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        R A, Bx, By;
        feq_ab(i, rho, st[1], st[2], A, Bx, By);
        a += lf[i] * A;
        bx += lf[i] * Bx;
        by += lf[i] * By;
        ls[3 + i] = k * lf[i];
        lk += lf[i] * st[3 + i];
    }
    ls[0] = a;
    ls[1] = bx;
    ls[2] = by;
}

template <typename T>
__device__ __forceinline__ void load_d(const T* p, T (&f)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = p[i];
}

// sum over the warp, one atomic per warp (every lane of the warp must call)
__device__ __forceinline__ void warp_atomic_add(double* dst, double v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if ((threadIdx.x & 31) == 0 && v != 0.0) atomicAdd(dst, v);
}

template <typename R>
__device__ __forceinline__ void atomic_add9(R* dst, const R (&v)[9]) {
#pragma unroll
    for (int i = 0; i < 9; ++i)
        if (v[i] != R(0)) atomicAdd(dst + i, v[i]);
}

// the window node of lattice cell corner q (0..3) for the bilinear stencil
// at (wx, wy), its weight and the weight's derivative in wy; false when the
// corner is outside the window (the forward skipped it)
template <typename T>
__device__ __forceinline__ bool bilinear_corner(const Dev<T>& d, int ox, int oy, double wx, double wy, int q,
                                                int64_t& b, double& w, double& dwy) {
    const double fx0 = floor(wx), fy0 = floor(wy);
    const int ix = (int)fx0, iy = (int)fy0;
    const double ax = __dsub_rn(wx, fx0), ay = __dsub_rn(wy, fy0);
    const double wxq = (q & 1) ? ax : 1.0 - ax, wyq = (q >> 1) ? ay : 1.0 - ay;
    w = wxq * wyq;
    dwy = (q >> 1) ? wxq : -wxq;
    const int bx = ix + (q & 1) - ox, by = iy + (q >> 1) - oy;
    if ((unsigned)bx >= (unsigned)d.bw || (unsigned)by >= (unsigned)d.bh) return false;
    b = (int64_t)by * d.bw + bx;
    return true;
}

// derivatives of the barycentric coordinates of triangle k in q_y
__device__ __forceinline__ void bary_dqy(const double* g, double (&dl)[3]) {  // FP64 geometry
    const double x1 = g[2], x2 = g[4], det = g[6];
    dl[1] = -x2 / det;
    dl[2] = x1 / det;
    dl[0] = -dl[1] - dl[2];
}

// Adjoint of F_y at t+1 (lamF = dJ/dF_y(t+1)) into the patch state that the
// force was computed from (d.fu_in): sigma_xy = -sum f^neq c_x c_y,
// sigma_yy = -dr/3 - sum f^neq c_y^2, F_y = sum_seg (sigma_xy n_x + sigma_yy n_y)
// at the mean of its two nodes.
template <typename T>
__global__ void k_adj_force(Dev<T> d, double lamF, T* lP) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= d.nseg) return;
    const T nx = T(d.seg_n[2 * k]), ny = T(d.seg_n[2 * k + 1]);
    const T lxy = 0.5 * nx * lamF, lyy = 0.5 * ny * lamF;
    for (int e = 0; e < 2; ++e) {
        const int P = e == 0 ? d.seg_a[k] : d.seg_b[k];
        T f[9], dr, rho, ux, uy;
        load_d(d.fu_in + (int64_t)kRec * P, f);
        mom_d(f, T(d.rho0), dr, rho, ux, uy);
        T ln[9], out[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            ln[i] = -(lxy * cx_of(i) * cy_of(i) + lyy * cy_of(i) * cy_of(i));
            out[i] = -lyy / 3.0 + ln[i];
        }
        jfeqT_add(rho, ux, uy, ln, T(-1), out);
        atomic_add9(lP + 9 * (int64_t)P, out);
    }
}

// The FV update of a regular node P from state `in`: the updated
// populations fv and the collision sums Cf_i - ceq_i (eq. ulbe).
template <typename T>
__device__ __forceinline__ void fv_update_d(const Dev<T>& d, const T* in, int P, T (&fv)[9], T (&cneq)[9]) {
    const T rho0 = T(d.rho0);
    T S[9], Cf[9], Z[3] = {0, 0, 0}, gpx = 0, gpy = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) S[i] = Cf[i] = 0.0;
    const int r0 = d.row_ptr[P], r1 = d.row_ptr[P + 1];
    for (int e = r0 + 1; e < r1; ++e) {
        const Coef<T> c = d.coef[e];
        T f[9], zz[3];
        load_d(in + (int64_t)kRec * c.col, f);
        T dr, rho, ux, uy;
        mom_d(f, rho0, dr, rho, ux, uy);
        zz[0] = ux * ux * rho;
        zz[1] = ux * uy * rho;
        zz[2] = uy * uy * rho;
        const T gx = T(c.gx), gy = T(c.gy), cc = T(c.c);
        gpx -= gx;
        gpy -= gy;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            S[i] += (cx_of(i) * gx + cy_of(i) * gy) * f[i];
            Cf[i] += cc * f[i];
        }
#pragma unroll
        for (int j = 0; j < 3; ++j) Z[j] += cc * zz[j];
    }
    T fP[9];
    load_d(in + (int64_t)kRec * P, fP);
    {
        T dr, rho, ux, uy;
        mom_d(fP, rho0, dr, rho, ux, uy);
        const T cc = T(d.coef[r0].c);
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            S[i] += (cx_of(i) * gpx + cy_of(i) * gpy) * fP[i];
            Cf[i] += cc * fP[i];
        }
        Z[0] += cc * ux * ux * rho;
        Z[1] += cc * ux * uy * rho;
        Z[2] += cc * uy * uy * rho;
    }
    // sum_k C (f^eq_k) from the linear parts Cf and the quadratic ones Z
    T dr = 0, jx = 0, jy = 0;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        dr += Cf[i];
        jx += cx_of(i) * Cf[i];
        jy += cy_of(i) * Cf[i];
    }
    const T q0 = dr - 1.5 * (Z[0] + Z[2]);
    const T inv = T(d.inv_tau_u), dt = T(d.dt_u);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        const T cx = cx_of(i), cy = cy_of(i);
        const T ceq = w_of<T>(i) * (q0 + 3.0 * (cx * jx + cy * jy) +
                                              4.5 * (cx * cx * Z[0] + 2.0 * cx * cy * Z[1] + cy * cy * Z[2]));
        cneq[i] = Cf[i] - ceq;
        fv[i] = fP[i] + dt * (S[i] - inv * cneq[i]);
    }
}

// Reverse of sub-step m, first pass at node P: psi_P, the adjoint of its
// FV update (through the wall rule at wall nodes), the outer nodes' feed
// adjoint, and the parameter terms (1/tau_u, kneq, wall velocity) added to
// the caller's sums.
template <typename T>
__device__ __forceinline__ void adj_psi_node(const Dev<T>& d, const StepArgs& a, const T* in, int m, const T* lnext,
                                             T* psi, T* lsnap, int P, T& l_inv, double& l_kneq, T& l_v) {
    const int8_t kind = d.kind[P];
    T lam[9], ps[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) lam[i] = lnext[9 * (int64_t)P + i];
    if (kind == HLBM_NODE_OUTER) {
        const int64_t no = d.n_outer;
        const int o = d.outer_of[P];
        const T th = T(m + 1) / T(d.n_sub);
        T st[12], ls[12];
#pragma unroll
        for (int j = 0; j < 12; ++j) st[j] = (T(1) - th) * T(d.snap[j * no + o]) + th * T(d.snap[(12 + j) * no + o]);
        ffsT(st, T(d.rho0), T(d.kneq), lam, ls, l_kneq);
#pragma unroll
        for (int j = 0; j < 12; ++j) {
            lsnap[j * no + o] += (T(1) - th) * ls[j];
            lsnap[(12 + j) * no + o] += th * ls[j];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i) ps[i] = T(0);
    } else {
        T fv[9], cneq[9];
        fv_update_d(d, in, P, fv, cneq);
#pragma unroll
        for (int i = 0; i < 9; ++i) ps[i] = lam[i];
        if (kind == HLBM_NODE_WALL) {
            // g(f) = f + f^eq(rho, U) - f^eq(rho, u(f))
            T U, V;
            wall_velocity(d, a, m, U, V);
            T dr, rho, ux, uy;
            mom_d(fv, T(d.rho0), dr, rho, ux, uy);
            T aU = T(0);
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                T A, Bx, By;
                feq_ab(i, rho, U, V, A, Bx, By);
                aU += lam[i] * A;
                l_v += lam[i] * By;
            }
#pragma unroll
            for (int i = 0; i < 9; ++i) ps[i] += aU;
            jfeqT_add(rho, ux, uy, lam, T(-1), ps);
        }
        const T dt = T(d.dt_u);
#pragma unroll
        for (int i = 0; i < 9; ++i) l_inv -= dt * ps[i] * cneq[i];
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) psi[9 * (int64_t)P + i] = ps[i];
}

// Reverse of sub-step m, second pass at node k: the adjoint of its state
// before the sub-step, gathered from the rows that read it (k itself and its
// neighbours; tpos gives row P's entry of column k).
template <typename T>
__device__ __forceinline__ void adj_gather_node(const Dev<T>& d, const T* in, const T* psi, const int32_t* tpos,
                                                T* lcur, int k) {
    const T dt = T(d.dt_u), inv = T(d.inv_tau_u);
    T out[9], Lc[9];
    const bool regular = d.kind[k] != HLBM_NODE_OUTER;
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        out[i] = regular ? psi[9 * (int64_t)k + i] : T(0);
        Lc[i] = T(0);
    }
    const int r0 = d.row_ptr[k], r1 = d.row_ptr[k + 1];
    for (int e = r0; e < r1; ++e) {
        const int P = e == r0 ? k : d.coef[e].col;
        if (d.kind[P] == HLBM_NODE_OUTER) continue;
        T gx, gy, cc;
        if (P == k) {
            gx = gy = T(0);
            for (int q = r0 + 1; q < r1; ++q) {
                gx -= d.coef[q].gx;
                gy -= d.coef[q].gy;
            }
            cc = d.coef[r0].c;
        } else {
            const Coef<T> c = d.coef[tpos[e]];
            gx = c.gx;
            gy = c.gy;
            cc = c.c;
        }
        const T* pp = psi + 9 * (int64_t)P;
#pragma unroll
        for (int j = 0; j < 9; ++j) {
            out[j] += dt * ((T(cx_of(j)) * gx + T(cy_of(j)) * gy) - inv * cc) * pp[j];
            Lc[j] += cc * pp[j];
        }
    }
    T f[9], dr, rho, ux, uy;
    load_d(in + (int64_t)kRec * k, f);
    mom_d(f, T(d.rho0), dr, rho, ux, uy);
    jfeqT_add(rho, ux, uy, Lc, dt * inv, out);
#pragma unroll
    for (int j = 0; j < 9; ++j) lcur[9 * (int64_t)k + j] = out[j];
}

// The FV part of one step's reverse in one cooperative launch: the n
// sub-steps forward again from sub[0] (every state kept in sub), then their
// reverse from lPn (the adjoint of the patch after them) to lPm (before
// them), with grid-wide barriers between the passes.  Every thread runs the
// same number of node iterations, so the warp sums stay convergent.
template <typename T>
__global__ void __launch_bounds__(128) k_adj_fv_all(Dev<T> d, StepArgs a, T* sub, const T* lPn, T* x0, T* x1,
                                                    T* psi, const int32_t* tpos, T* lsnap, double* par, double* lV,
                                                    T* lPm) {
    namespace cg = cooperative_groups;
    cg::grid_group grid = cg::this_grid();
    const int n = d.n, ns = d.n_sub;
    const int nth = gridDim.x * blockDim.x, gtid = blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t rec = (int64_t)kRec * n;
    for (int m = 0; m < ns; ++m) {
        T U, V;
        wall_velocity(d, a, m, U, V);
        for (int P = gtid; P < n; P += nth) fv_node(d, sub + m * rec, sub + (m + 1) * rec, P, m, U, V);
        grid.sync();
    }
    T l_inv = T(0);
    double l_kneq = 0.0;
    const T* lnext = lPn;
    for (int m = ns - 1; m >= 0; --m) {
        const T* in = sub + m * rec;
        T l_v = T(0);
        for (int base = 0; base < n; base += nth) {
            const int P = base + gtid;
            if (P < n) adj_psi_node(d, a, in, m, lnext, psi, lsnap, P, l_inv, l_kneq, l_v);
        }
        warp_atomic_add(lV + (int64_t)a.t * ns + m, double(l_v));
        grid.sync();
        T* lcur = (m & 1) ? x1 : x0;
        for (int k = gtid; k < n; k += nth) adj_gather_node(d, in, psi, tpos, lcur, k);
        grid.sync();
        lnext = lcur;
    }
    for (int64_t i = gtid; i < 9 * (int64_t)n; i += nth) lPm[i] = lnext[i];
    warp_atomic_add(par + 1, double(l_inv));
    warp_atomic_add(par + 3, l_kneq);
}

// Reverse of the outer nodes' feed: snap[0] bilinear from the window state
// at t (previous window), snap[1] from the one at t+1; positions at y(t).
template <typename T>
__global__ void k_adj_feed(Dev<T> d, StepArgs a, const T* lsnap, T* lSo, T* lSn, double* lY) {
    const int o = blockIdx.x * blockDim.x + threadIdx.x;
    double gy = 0.0;
    if (o < d.n_outer) {
        const int P = d.outer[o];
        const double wx = __dadd_rn(a.cx, d.xy[2 * P]), wy = __dadd_rn(a.cy, d.xy[2 * P + 1]);
        const int64_t no = d.n_outer;
        for (int side = 0; side < 2; ++side) {
            const T* box = side == 0 ? d.sbox_old : (const T*)d.sbox_new;
            const int ox = side == 0 ? a.pbx0 : a.bx0, oy = side == 0 ? a.pby0 : a.by0;
            T* lS = side == 0 ? lSo : lSn;
            T ls[12];
#pragma unroll
            for (int j = 0; j < 12; ++j) ls[j] = lsnap[(12 * side + j) * no + o];
            for (int q = 0; q < 4; ++q) {
                int64_t b;
                double w, dw;
                if (!bilinear_corner(d, ox, oy, wx, wy, q, b, w, dw)) continue;
                T f[9], st[12], out[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    f[i] = T(box[i * d.bplane + b]);
                    out[i] = 0.0;
                }
                state_d(f, T(d.rho0), st);
                stateT_add(f, T(d.rho0), ls, T(w), out);
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (out[i] != 0.0) atomicAdd(lS + i * d.bplane + b, out[i]);
                T dot = 0.0;
#pragma unroll
                for (int j = 0; j < 12; ++j) dot += ls[j] * st[j];
                gy += dw * double(dot);
            }
        }
    }
    warp_atomic_add(lY + a.t, gy);
}

// source element of population i pulled by node (x, y) (the boundary rules
// of the stream-collide: bounce-back walls, zero-gradient outflow, periodic)
template <typename T>
__device__ __forceinline__ int64_t pull_src(const Dev<T>& d, int x, int y, int i) {
    int sx = x - cx_of(i), sy = y - cy_of(i);
    if (sx < 0 || sx >= d.nx) {
        if (d.bc_x == HLBM_BC_PERIODIC)
            sx = (sx + d.nx) % d.nx;
        else if (d.bc_x == HLBM_BC_WALL)
            return opp_of(i) * d.plane + (int64_t)y * d.pitch + x;
        else
            sx = x;
    }
    if (sy < 0 || sy >= d.ny) {
        if (d.bc_y == HLBM_BC_PERIODIC)
            sy = (sy + d.ny) % d.ny;
        else if (d.bc_y == HLBM_BC_WALL)
            return opp_of(i) * d.plane + (int64_t)y * d.pitch + x;
        else
            sy = y;
    }
    return i * d.plane + (int64_t)sy * d.pitch + sx;
}

// Reverse of the stream-collide (pull, BGK with 1/tau_s) at every node it
// wrote (discretization nodes), plus the window state it wrote (lSn).
template <typename T>
__global__ void k_adj_stream(Dev<T> d, StepArgs a, const T* lfB, const T* lSn, T* lfA, double* par) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
    T l_om = 0;
    bool active = x < d.nx;
    int64_t b = -1;
    if (active) {
        const unsigned rx = (unsigned)(x - a.bx0), ry = (unsigned)(y - a.by0);
        if (rx < (unsigned)d.bw && ry < (unsigned)d.bh) {
            b = (int64_t)ry * d.bw + rx;
            active = d.cls_cur[b] == CLS_DISC;
        }
    }
    if (active) {
        const T* A = d.fA;
        T f[9];
        int64_t src[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            src[i] = pull_src(d, x, y, i);
            f[i] = T(A[src[i]]);
        }
        T dr, rho, ux, uy;
        mom_d(f, T(d.rho0), dr, rho, ux, uy);
        const T om = 1.0 / T(d.tau_s);
        const int64_t s = (int64_t)y * d.pitch + x;
        T lam[9], mu[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            lam[i] = lfB[i * d.plane + s];
            mu[i] = (1.0 - om) * lam[i];
            l_om -= lam[i] * (f[i] - feq_d(i, dr, rho, ux, uy));
        }
        jfeqT_add(rho, ux, uy, lam, om, mu);
        if (b >= 0) {
#pragma unroll
            for (int i = 0; i < 9; ++i) mu[i] += lSn[i * d.bplane + b];
        }
#pragma unroll
        for (int i = 0; i < 9; ++i)
            if (mu[i] != 0.0) atomicAdd(lfA + src[i], mu[i]);
    }
    warp_atomic_add(par + 0, l_om);
}

// Reverse of the eq. postcollision2_s fill: the adjoint of the populations
// it wrote goes to the patch state it interpolated (and is consumed).
template <typename T>
__global__ void k_adj_fill(Dev<T> d, StepArgs a, T* lfA, T* lP, double* par, double* lY) {
    const int64_t b = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    double l_k = 0.0, gy = 0.0;
    bool fill = false;
    int x = 0, y = 0;
    if (b < d.bplane) {
        const int8_t c = d.cls_cur[b];
        x = a.bx0 + (int)(b % d.bw);
        y = a.by0 + (int)(b / d.bw);
        if (c == CLS_INTERP) {
            fill = true;
        } else if (c == CLS_DISC && !a.first) {
            const unsigned px = (unsigned)(x - a.pbx0), py = (unsigned)(y - a.pby0);
            const int8_t prev = (px < (unsigned)d.bw && py < (unsigned)d.bh) ? d.cls_prev[(int64_t)py * d.bw + px]
                                                                             : (int8_t)CLS_DISC;
            fill = prev != CLS_DISC;
        }
    }
    if (fill) {
        const int64_t s = (int64_t)y * d.pitch + x;
        T lp[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            lp[i] = lfA[i * d.plane + s];
            lfA[i * d.plane + s] = 0.0;
        }
        double lam[3];
        const double qx = __dsub_rn((double)x, a.cx), qy = __dsub_rn((double)y, a.cy);
        const int k = locate_dev(d, qx, qy, lam);
        if (k >= 0) {
            const T rho0 = T(d.rho0);
            T fv[3][9], sv[3][12], st[12];
#pragma unroll
            for (int j = 0; j < 12; ++j) st[j] = 0.0;
            for (int q = 0; q < 3; ++q) {
                load_d(d.fu_in + (int64_t)kRec * d.tri[3 * k + q], fv[q]);
                state_d(fv[q], rho0, sv[q]);
#pragma unroll
                for (int j = 0; j < 12; ++j) st[j] += T(lam[q]) * sv[q][j];
            }
            T ls[12];
            ffsT(st, rho0, T(d.k178), lp, ls, l_k);
            double dl[3];
            bary_dqy(d.trigeo + 8 * (int64_t)k, dl);
            for (int q = 0; q < 3; ++q) {
                T out[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) out[i] = 0.0;
                stateT_add(fv[q], rho0, ls, T(lam[q]), out);
                atomic_add9(lP + 9 * (int64_t)d.tri[3 * k + q], out);
                T dot = 0.0;
#pragma unroll
                for (int j = 0; j < 12; ++j) dot += ls[j] * sv[q][j];
                gy -= dl[q] * double(dot);  // q_y = y - c_y
            }
        }
    }
    warp_atomic_add(par + 2, l_k);
    warp_atomic_add(lY + a.t, gy);
}

// Reverse of the refill of Sec. 4 (types 1, 2, 3 and wall nodes) from the
// adjoint lPm of the refilled state into the state before it (lP0) and the
// window state at t (lSo).
template <typename T>
__global__ void k_adj_refill(Dev<T> d, StepArgs a, const T* lPm, T* lP0, T* lSo, double* par,
                             double* lY) {
    const int P = blockIdx.x * blockDim.x + threadIdx.x;
    double l_k = 0.0, gy = 0.0, gdy = 0.0;
    if (P < d.n) {
        T lam[9];
#pragma unroll
        for (int i = 0; i < 9; ++i) lam[i] = lPm[9 * (int64_t)P + i];
        const int type = d.rtype[P];
        const T rho0 = T(d.rho0);
        if (type == 0 || type == 2) {
            atomic_add9(lP0 + 9 * (int64_t)P, lam);
        } else if (type == 3) {
            const int k = d.rdonor[P];
            const double qx = __dadd_rn(d.xy[2 * P], a.dX), qy = __dadd_rn(d.xy[2 * P + 1], a.dY);
            double l0, l1, l2, dl[3];
            bary_rn(d.trigeo + 8 * (int64_t)k, qx, qy, l0, l1, l2);
            bary_dqy(d.trigeo + 8 * (int64_t)k, dl);
            const T lb[3] = {T(l0), T(l1), T(l2)};
            for (int q = 0; q < 3; ++q) {
                const int v = d.tri[3 * k + q];
                T out[9], f[9];
                load_d(d.fu_in + (int64_t)kRec * v, f);
                T dot = 0.0;
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    out[i] = lb[q] * lam[i];
                    dot += lam[i] * f[i];
                }
                atomic_add9(lP0 + 9 * (int64_t)v, out);
                gdy += dl[q] * double(dot);
            }
        } else if (type == 1) {
            const double wx = __dadd_rn(a.cx, d.xy[2 * P]), wy = __dadd_rn(a.cy, d.xy[2 * P + 1]);
            T st[12], fq[4][9], sq[4][12];
            double wq[4], dwq[4];
            int64_t bq[4];
            bool ok[4];
#pragma unroll
            for (int j = 0; j < 12; ++j) st[j] = 0.0;
            for (int q = 0; q < 4; ++q) {
                ok[q] = bilinear_corner(d, a.pbx0, a.pby0, wx, wy, q, bq[q], wq[q], dwq[q]);
                if (!ok[q]) continue;
#pragma unroll
                for (int i = 0; i < 9; ++i) fq[q][i] = T(d.sbox_old[i * d.bplane + bq[q]]);
                state_d(fq[q], rho0, sq[q]);
#pragma unroll
                for (int j = 0; j < 12; ++j) st[j] += T(wq[q]) * sq[q][j];
            }
            T ls[12];
            ffsT(st, rho0, T(d.kneq), lam, ls, l_k);
            for (int q = 0; q < 4; ++q) {
                if (!ok[q]) continue;
                T out[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) out[i] = 0.0;
                stateT_add(fq[q], rho0, ls, T(wq[q]), out);
#pragma unroll
                for (int i = 0; i < 9; ++i)
                    if (out[i] != 0.0) atomicAdd(lSo + i * d.bplane + bq[q], out[i]);
                T dot = 0.0;
#pragma unroll
                for (int j = 0; j < 12; ++j) dot += ls[j] * sq[q][j];
                gy += dwq[q] * double(dot);
            }
        }
    }
    warp_atomic_add(par + 3, l_k);
    warp_atomic_add(lY + a.t, gy + gdy);
    warp_atomic_add(lY + a.t - 1, -gdy);
}

template <typename T>
void launch_adj_force(const Dev<T>& d, double lamF, T* lP, cudaStream_t s) {
    if (d.nseg > 0) k_adj_force<T><<<(d.nseg + 127) / 128, 128, 0, s>>>(d, lamF, lP);
}
template <typename T>
cudaError_t launch_adj_fv(const Dev<T>& d, const StepArgs& a, T* sub, const T* lPn, T* x0, T* x1, T* psi,
                          const int32_t* tpos, T* lsnap, double* par, double* lV, T* lPm, cudaStream_t s) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, (const void*)k_adj_fv_all<T>, 128, 0);
    const int blocks = std::max(1, std::min((d.n + 127) / 128, std::max(per, 1) * sms));
    Dev<T> dd = d;
    StepArgs aa = a;
    void* args[] = {&dd, &aa, &sub, &lPn, &x0, &x1, &psi, &tpos, &lsnap, &par, &lV, &lPm};
    return cudaLaunchCooperativeKernel((const void*)k_adj_fv_all<T>, dim3(blocks), dim3(128), args, 0, s);
}
template <typename T>
void launch_adj_feed(const Dev<T>& d, const StepArgs& a, const T* lsnap, T* lSo, T* lSn, double* lY,
                     cudaStream_t s) {
    if (d.n_outer) k_adj_feed<T><<<(d.n_outer + 127) / 128, 128, 0, s>>>(d, a, lsnap, lSo, lSn, lY);
}
template <typename T>
void launch_adj_stream(const Dev<T>& d, const StepArgs& a, const T* lfB, const T* lSn, T* lfA,
                       double* par, cudaStream_t s) {
    dim3 grid((d.nx + 127) / 128, d.ny);
    k_adj_stream<T><<<grid, 128, 0, s>>>(d, a, lfB, lSn, lfA, par);
}
template <typename T>
void launch_adj_fill(const Dev<T>& d, const StepArgs& a, T* lfA, T* lP, double* par, double* lY,
                     cudaStream_t s) {
    k_adj_fill<T><<<(unsigned)((d.bplane + 127) / 128), 128, 0, s>>>(d, a, lfA, lP, par, lY);
}
template <typename T>
void launch_adj_refill(const Dev<T>& d, const StepArgs& a, const T* lPm, T* lP0, T* lSo, double* par,
                       double* lY, cudaStream_t s) {
    k_adj_refill<T><<<(d.n + 127) / 128, 128, 0, s>>>(d, a, lPm, lP0, lSo, par, lY);
}

#define HLBM_INST(T)                                                                                        \
    template void launch_fv_coeffs<T>(const Dev<T>&, int, Coef<T>*, cudaStream_t);                          \
    template void launch_patch_init<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                         \
    template void launch_refill<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                             \
    template void launch_feed<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                               \
    template int fv_tile_capacity<T>();                                                                       \
    template cudaError_t launch_fv_persistent<T>(const Dev<T>&, const StepArgs&, cudaStream_t);               \
    template size_t fv_smem_bytes<T>(int, int, int, int, int);                                                     \
    template int fv_tile_max<T>();                                                                            \
    template void launch_build_ell<T>(const Coef<T>*, const int32_t*, const int32_t*, Coef<T>*, int64_t,       \
                                      cudaStream_t);                                                          \
    template int fv_smem_tile_capacity<T>(size_t);                                                            \
    template cudaError_t launch_fv_smem<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                     \
    template size_t fv_tmem_smem_bytes<T>(int, int, int, int);                                                \
    template int fv_tmem_tile_capacity<T>(size_t);                                                            \
    template cudaError_t launch_fv_tmem<T>(const Dev<T>&, const StepArgs&, cudaStream_t);                     \
    template cudaError_t launch_fv_tmem_pack<T>(const FvPack<T>&, int, size_t, cudaStream_t);                 \
    template int fv_deep_tmem_slots<T>();                                                                     \
    template int fv_deep_row_words<T>();                                                                      \
    template size_t fv_deep_smem_bytes<T>(int, int, int);                                                     \
    template int fv_deep_tile_capacity<T>(size_t);                                                            \
    template cudaError_t launch_fv_deep<T>(const Dev<T>&, const StepArgs&, const FarArgs<T>*, cudaStream_t);  \
    template void launch_build_deep_rows<T>(const Dev<T>&, const int32_t*, const int32_t*, int64_t, uint32_t*, \
                                            cudaStream_t);                                                    \
    template void launch_force<T>(const Dev<T>&, int64_t, cudaStream_t);                                      \
    template void launch_patch_macro<T>(const Dev<T>&, double*, double*, double*, double*, cudaStream_t);    \
    template void launch_adj_force<T>(const Dev<T>&, double, T*, cudaStream_t);                               \
    template cudaError_t launch_adj_fv<T>(const Dev<T>&, const StepArgs&, T*, const T*, T*, T*, T*,            \
                                          const int32_t*, T*, double*, double*, T*, cudaStream_t);            \
    template void launch_adj_feed<T>(const Dev<T>&, const StepArgs&, const T*, T*, T*, double*, cudaStream_t); \
    template void launch_adj_stream<T>(const Dev<T>&, const StepArgs&, const T*, const T*, T*, double*,        \
                                       cudaStream_t);                                                         \
    template void launch_adj_fill<T>(const Dev<T>&, const StepArgs&, T*, T*, double*, double*, cudaStream_t);  \
    template void launch_adj_refill<T>(const Dev<T>&, const StepArgs&, const T*, T*, T*, double*, double*,     \
                                       cudaStream_t);
HLBM_INST(float)
HLBM_INST(double)

}  // namespace hk
