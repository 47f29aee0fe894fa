/* CPU correctness oracle for the moving-grid hybrid lattice Boltzmann method.
 *
 * TEST INFRASTRUCTURE ONLY: plain serial FP64 C.  Each function follows one
 * passage of the paper (Di Ilio et al., "A moving-grid approach for
 * fluid-structure interaction problems with hybrid lattice Boltzmann
 * method"), cited beside it.  Built with -ffp-contract=off so that the
 * geometric decisions (node classes, donor cells and triangles) are the
 * IEEE results of the operations as written.
 *
 * Readings of passages the paper leaves open (restated where used):
 *  R1  S_ik, C_ik (Sec. 3, eq. ulbe): cell-vertex FV on median-dual control
 *      volumes with piecewise-linear f on each triangle; S_ik = c_i . g_Pk
 *      with g_Pk = -(1/V_P) * closed-boundary integral of n phi_k;
 *      C_Pk = (1/V_P) * integral over CV(P) of phi_k (consistent), or
 *      identity (lumped).
 *  R2  Outer patch nodes (eq. postcollision2_u): Dirichlet reading,
 *      f = f^eq(rho, u) + (1 - 1/(2 tau_s)) f^neq with rho, u, f^neq
 *      bilinear from the structured state, linear in time between t and
 *      t+1 at theta = (m+1)/n.
 *  R3  Wall nodes during sub-steps: FV update on the truncated CV, then the
 *      equilibrium part is moved to the wall velocity:
 *      f += f^eq(rho, U) - f^eq(rho, u).
 *  R4  Force: sigma = -(rho - rho0) c_s^2 I - sum_i f^neq_i c_i c_i at wall
 *      nodes, trapezoid rule over the wall segments with the body's outward
 *      normal.
 *  R5  Outflow (Sec. 5): zero-gradient copy of the source row; half-way
 *      bounce-back on walls, which takes precedence at corners.
 *  R6  Step order: refill at the start of step t (patch moved to y(t)),
 *      classification at y(t), eq. 178 feeds the structured interpolation
 *      nodes from the patch at t, structured step t -> t+1, then n FV
 *      sub-steps fed by the structured state at t and t+1.
 *  R7  Interpolations carry rho, u and f^neq; f^eq is rebuilt from the
 *      interpolated rho, u (Sec. 4, type 1 and eq. 178).  Type 3 moves f.
 *  R8  Structured nodes that become discretization nodes take their
 *      post-collision value from eq. 178 on their first step.
 *  R9  Donor triangle = the candidate with the largest smallest barycentric
 *      coordinate, among those with smallest coordinate >= -1e-12; ties go
 *      to the lowest triangle index.  Donor cell = (floor x, floor y).
 *  R10 Full eq. postcollision2_u (outer_fv = 1): the outer node's value is
 *      the R2 value plus dt_u sum_k S_ik f*_k - (dt_u/tau_u) sum_k C_ik
 *      (f*_k - f^eq(f*_k)) over its truncated control volume, where f*_k
 *      is the R2 value of node k at theta = (m+1)/n when k is an outer
 *      (interpolation) node, including k = P, and the patch value at
 *      sub-step m otherwise.  f^eq(f*) of an R2 value is f^eq,s (f^neq,s
 *      carries no mass or momentum), so f* - f^eq(f*) is the starred
 *      non-equilibrium part of the paper.  Regular nodes read an outer
 *      neighbour's stored value, increment included.
 *  R11 INDUCED motion (the paper's outlook, Sec. 7): the lamina is a rigid
 *      body on a spring and damper, m y'' + c y' + k y = F_y, integrated
 *      once per lattice step by symplectic Euler with the force at the
 *      start of the step: v(t+1) = v(t) + (F_y(t) - c v(t) - k y(t))/m,
 *      y(t+1) = y(t) + v(t+1).  The patch sits at y(t) during step t; the
 *      wall velocity at sub-step m is v(t) + theta (v(t+1) - v(t)).
 *  R12 Nested lattice levels (the paper's refinement levels, Sec. 5; the
 *      coupling is not given there): the lattice around the patch is a box
 *      inside a lattice of twice the spacing and twice the time step
 *      (acoustic scaling, same lattice velocities), tau_c - 1/2 =
 *      (tau_s - 1/2)/2 for the same viscosity, which may itself be a box
 *      inside a coarser one, and so on.  Each pair couples as follows.
 *      Non-equilibrium parts scale as tau dx (f^neq = -tau dt D f^eq); for
 *      post-collision populations f^neq_c = 2 (tau_c - 1)/(tau_f - 1)
 *      f^neq_f (tau_f, tau_c != 1).  Per coarse step (fine steps 2T, 2T+1):
 *      the coarse lattice streams and collides T -> T+1; before each fine
 *      step the fine box's outermost ring takes the post-collision
 *      f^eq(rho, u) + f^neq_f rebuilt from the coarse rho, u, f^neq (the
 *      coarse node itself at even positions, the cubic midpoint rule
 *      (-1, 9, 9, -1)/16 along the box edge at odd ones; at odd fine times
 *      the mean of coarse times T and T+1) and is not streamed itself; after
 *      the second fine step the coarse nodes strictly inside the box take
 *      the post-collision state of the fine node they sit on.  Levels step
 *      coarsest first, restrict finest first, and rebuild their rings on
 *      their own clocks.
 *  R13 Non-reflecting outflow, the second reading of Sec. 5's unspecified
 *      outflow (a flag; R5 stays the default): an absorbing layer of N rows
 *      along each outflow side of the lattice that carries the domain
 *      boundary.  At a node d rows from the nearest such side (d < N) the
 *      post-collision populations relax towards the rest state,
 *      f <- w rho0 + (1 - sigma(d)) (f - w rho0), sigma(d) = sigma_max
 *      ((N - d)/N)^2, so that waves leaving the domain are damped before
 *      the zero-gradient copy can reflect them.  Nodes with d >= N are not
 *      touched.
 */
#include "hlbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* D2Q9 lattice, Sec. 3: c_s = 1/sqrt(3)                                     */
/* ------------------------------------------------------------------------ */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0, 1.0 / 9.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const double CS2 = 1.0 / 3.0;
#define ORC_PI 3.14159265358979323846

/* Eq. local_eq: f_i^eq = w_i rho (1 + c.u/cs^2 + (c.u)^2/(2 cs^4) - u^2/(2 cs^2)) */
void orc_feq(double rho, double ux, double uy, double* feq) {
    double usq = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        double cu = CX[i] * ux + CY[i] * uy;
        feq[i] = W[i] * rho * (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - usq / (2.0 * CS2));
    }
}

/* rho and u: the first two moments of f (Sec. 3) */
static void moments(const double* f, double* rho, double* ux, double* uy) {
    double r = 0.0, jx = 0.0, jy = 0.0;
    for (int i = 0; i < 9; ++i) {
        r += f[i];
        jx += CX[i] * f[i];
        jy += CY[i] * f[i];
    }
    *rho = r;
    *ux = jx / r;
    *uy = jy / r;
}

/* rho, u and f^neq = f - f^eq(rho, u) of one node */
static void state_of(const double* f, double* rho, double* ux, double* uy, double* fneq) {
    double feq[9];
    moments(f, rho, ux, uy);
    orc_feq(*rho, *ux, *uy, feq);
    for (int i = 0; i < 9; ++i) fneq[i] = f[i] - feq[i];
}

/* ------------------------------------------------------------------------ */
/* oracle state                                                              */
/* ------------------------------------------------------------------------ */
/* R12: one coarser lattice level, post-collision populations [9][ny][nx];
 * f[cur] at the level's current time */
typedef struct {
    int nx, ny, ox, oy;
    int64_t N;
    double* f[2];
    int cur;
} orc_level_t;

struct orc {
    orc_params_t p;
    double* xy;
    int32_t* tri;
    int8_t* kind;
    int64_t N;
    double* fs[2]; /* structured pre-collision state [9][ny][nx] */
    int cur;
    double* fpost; /* structured post-collision scratch */
    int8_t* cls_prev;
    int8_t* cls_cur;
    double* fu[2]; /* patch state [n][9] */
    int ucur;
    double* feq_u; /* per-node equilibrium scratch [n][9] */
    /* FV coefficients, CSR by node, pivot first (R1) */
    int32_t *row_ptr, *col;
    double *gx, *gy, *cc, *vol;
    /* wall segments (R4): end nodes and body-outward normal scaled by length */
    int nseg;
    int32_t *seg_a, *seg_b;
    double *seg_nx, *seg_ny;
    /* point-location bins over the body-frame mesh */
    double bx0, by0, bh;
    int nbx, nby;
    int32_t *bstart, *bitems;
    /* outer-node feed: rho, ux, uy, fneq[9] at t and t+1 (R2) */
    double *snap0, *snap1;
    double* dstar; /* R2 values of the outer nodes at the current sub-step [n][9] */
    int32_t *rtype, *rdonor;
    double *Fx, *Fy;
    int64_t hcap;
    int64_t t;
    double Xprev, Yprev;
    double *Yh, *Vh; /* INDUCED motion: y and v at integer times (R11) */
    orc_level_t lv[ORC_MAX_LEVELS]; /* R12: coarser levels 1..n_levels */
    int64_t mcap;
    int status;
};

/* lamina position at time t (Sec. 2: y(t) = A sin(w t)); HARMONIC_X moves
 * the lamina along its own chord, x(t) = A sin(w t) (Stokes' second problem
 * for the two long faces: a test case, not the paper's motion) */
static void motion_pos(const orc_params_t* p, int64_t t, double* X, double* Y) {
    double tt = (double)t;
    if (p->motion == ORC_MOTION_HARMONIC) {
        *X = 0.0;
        *Y = p->A * sin(p->omega * tt);
    } else if (p->motion == ORC_MOTION_HARMONIC_X) {
        *X = p->A * sin(p->omega * tt);
        *Y = 0.0;
    } else if (p->motion == ORC_MOTION_UNIFORM) {
        *X = p->vx * tt;
        *Y = p->vy * tt;
    } else {
        *X = 0.0;
        *Y = 0.0;
    }
}

/* lamina velocity at (fractional) time */
static void motion_vel(const orc_params_t* p, double time, double* U, double* V) {
    if (p->motion == ORC_MOTION_HARMONIC) {
        *U = 0.0;
        *V = p->A * p->omega * cos(p->omega * time);
    } else if (p->motion == ORC_MOTION_HARMONIC_X) {
        *U = p->A * p->omega * cos(p->omega * time);
        *V = 0.0;
    } else if (p->motion == ORC_MOTION_UNIFORM) {
        *U = p->vx;
        *V = p->vy;
    } else {
        *U = 0.0;
        *V = 0.0;
    }
}

/* position at integer time t; INDUCED motion reads the history (R11) */
static void lamina_pos(const orc_t* o, int64_t t, double* X, double* Y) {
    if (o->p.motion == ORC_MOTION_INDUCED) {
        *X = 0.0;
        *Y = o->Yh[t];
    } else {
        motion_pos(&o->p, t, X, Y);
    }
}

/* ------------------------------------------------------------------------ */
/* barycentric coordinates and point location (Sec. 4, type 3; R9)           */
/* ------------------------------------------------------------------------ */
static void bary(double ax, double ay, double bx, double by, double cx, double cy, double qx,
                 double qy, double* l) {
    double x1 = bx - ax, y1 = by - ay, x2 = cx - ax, y2 = cy - ay;
    double det = x1 * y2 - x2 * y1;
    double px = qx - ax, py = qy - ay;
    double lb = (px * y2 - x2 * py) / det;
    double lc = (x1 * py - px * y1) / det;
    l[0] = (1.0 - lb) - lc;
    l[1] = lb;
    l[2] = lc;
}

static void bins_build(orc_t* o) {
    const double* xy = o->xy;
    int n = o->p.n_nodes, nt = o->p.n_tris;
    double xmin = xy[0], xmax = xy[0], ymin = xy[1], ymax = xy[1], area = 0.0;
    for (int i = 1; i < n; ++i) {
        if (xy[2 * i] < xmin) xmin = xy[2 * i];
        if (xy[2 * i] > xmax) xmax = xy[2 * i];
        if (xy[2 * i + 1] < ymin) ymin = xy[2 * i + 1];
        if (xy[2 * i + 1] > ymax) ymax = xy[2 * i + 1];
    }
    for (int k = 0; k < nt; ++k) {
        const int32_t* v = o->tri + 3 * k;
        double a = (xy[2 * v[1]] - xy[2 * v[0]]) * (xy[2 * v[2] + 1] - xy[2 * v[0] + 1]) -
                   (xy[2 * v[2]] - xy[2 * v[0]]) * (xy[2 * v[1] + 1] - xy[2 * v[0] + 1]);
        area += 0.5 * fabs(a);
    }
    o->bh = 2.0 * sqrt(area / nt);
    o->bx0 = xmin - 1e-6;
    o->by0 = ymin - 1e-6;
    o->nbx = (int)((xmax + 1e-6 - o->bx0) / o->bh) + 1;
    o->nby = (int)((ymax + 1e-6 - o->by0) / o->bh) + 1;
    int64_t nb = (int64_t)o->nbx * o->nby;
    int32_t* cnt = calloc(nb + 1, sizeof(int32_t));
    for (int pass = 0; pass < 2; ++pass) {
        for (int k = 0; k < nt; ++k) {
            const int32_t* v = o->tri + 3 * k;
            double lo_x = xy[2 * v[0]], hi_x = lo_x, lo_y = xy[2 * v[0] + 1], hi_y = lo_y;
            for (int j = 1; j < 3; ++j) {
                double x = xy[2 * v[j]], y = xy[2 * v[j] + 1];
                if (x < lo_x) lo_x = x;
                if (x > hi_x) hi_x = x;
                if (y < lo_y) lo_y = y;
                if (y > hi_y) hi_y = y;
            }
            int i0 = (int)floor((lo_x - 1e-9 - o->bx0) / o->bh);
            int i1 = (int)floor((hi_x + 1e-9 - o->bx0) / o->bh);
            int j0 = (int)floor((lo_y - 1e-9 - o->by0) / o->bh);
            int j1 = (int)floor((hi_y + 1e-9 - o->by0) / o->bh);
            if (i0 < 0) i0 = 0;
            if (j0 < 0) j0 = 0;
            if (i1 >= o->nbx) i1 = o->nbx - 1;
            if (j1 >= o->nby) j1 = o->nby - 1;
            for (int bj = j0; bj <= j1; ++bj)
                for (int bi = i0; bi <= i1; ++bi) {
                    int64_t b = (int64_t)bj * o->nbx + bi;
                    if (pass == 0)
                        cnt[b + 1]++;
                    else
                        o->bitems[o->bstart[b] + cnt[b]++] = k;
                }
        }
        if (pass == 0) {
            o->bstart = malloc((nb + 1) * sizeof(int32_t));
            o->bstart[0] = 0;
            for (int64_t b = 0; b < nb; ++b) o->bstart[b + 1] = o->bstart[b] + cnt[b + 1];
            o->bitems = malloc((size_t)(o->bstart[nb] + 1) * sizeof(int32_t));
            memset(cnt, 0, (nb + 1) * sizeof(int32_t));
        }
    }
    free(cnt);
}

/* Triangle of the body-frame mesh containing (qx, qy), or -1 (R9). */
static int locate(const orc_t* o, double qx, double qy, double* lam) {
    int bi = (int)floor((qx - o->bx0) / o->bh);
    int bj = (int)floor((qy - o->by0) / o->bh);
    if (bi < 0 || bj < 0 || bi >= o->nbx || bj >= o->nby) return -1;
    int64_t b = (int64_t)bj * o->nbx + bi;
    int best = -1;
    double best_min = -INFINITY;
    for (int32_t e = o->bstart[b]; e < o->bstart[b + 1]; ++e) {
        int k = o->bitems[e];
        const int32_t* v = o->tri + 3 * k;
        double l[3];
        bary(o->xy[2 * v[0]], o->xy[2 * v[0] + 1], o->xy[2 * v[1]], o->xy[2 * v[1] + 1],
             o->xy[2 * v[2]], o->xy[2 * v[2] + 1], qx, qy, l);
        double mn = l[0] < l[1] ? l[0] : l[1];
        if (l[2] < mn) mn = l[2];
        if (mn >= -1e-12 && mn > best_min) {
            best = k;
            best_min = mn;
            lam[0] = l[0];
            lam[1] = l[1];
            lam[2] = l[2];
        }
    }
    return best;
}

int orc_locate(const orc_t* o, double qx, double qy, double* lam3) { return locate(o, qx, qy, lam3); }

/* ------------------------------------------------------------------------ */
/* FV coefficients on median-dual control volumes (Sec. 3, eq. ulbe; R1)     */
/* ------------------------------------------------------------------------ */
typedef struct {
    int32_t *row_ptr, *col;
    double *gx, *gy, *cc, *vol;
} fv_coeffs_t;

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/* period_x/y > 0: coordinates of neighbours are taken as the minimum image */
static void build_fv(int n, const double* xy, int nt, const int32_t* tri, double period_x,
                     double period_y, int lumped, fv_coeffs_t* out) {
    /* node -> incident triangles */
    int32_t* tstart = calloc(n + 1, sizeof(int32_t));
    for (int k = 0; k < nt; ++k)
        for (int j = 0; j < 3; ++j) tstart[tri[3 * k + j] + 1]++;
    for (int i = 0; i < n; ++i) tstart[i + 1] += tstart[i];
    int32_t* tlist = malloc((size_t)tstart[n] * sizeof(int32_t));
    int32_t* fillc = calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    for (int k = 0; k < nt; ++k)
        for (int j = 0; j < 3; ++j) {
            int v = tri[3 * k + j];
            tlist[tstart[v] + fillc[v]++] = k;
        }
    free(fillc);
    /* neighbour rows: pivot first, then the other vertices ascending */
    int32_t* row_ptr = malloc((n + 1) * sizeof(int32_t));
    int32_t* tmp = malloc(64 * sizeof(int32_t));
    int cap = 64;
    int32_t* col = NULL;
    int nnz = 0, colcap = 0;
    row_ptr[0] = 0;
    for (int P = 0; P < n; ++P) {
        int m = 0;
        for (int e = tstart[P]; e < tstart[P + 1]; ++e)
            for (int j = 0; j < 3; ++j) {
                int v = tri[3 * tlist[e] + j];
                if (v == P) continue;
                if (m == cap) {
                    cap *= 2;
                    tmp = realloc(tmp, cap * sizeof(int32_t));
                }
                tmp[m++] = v;
            }
        qsort(tmp, m, sizeof(int32_t), cmp_i32);
        int u = 0;
        for (int j = 0; j < m; ++j)
            if (u == 0 || tmp[j] != tmp[u - 1]) tmp[u++] = tmp[j];
        if (nnz + u + 1 > colcap) {
            colcap = 2 * (nnz + u + 1) + 1024;
            col = realloc(col, colcap * sizeof(int32_t));
        }
        col[nnz++] = P;
        for (int j = 0; j < u; ++j) col[nnz++] = tmp[j];
        row_ptr[P + 1] = nnz;
    }
    free(tmp);
    double* gx = calloc(nnz, sizeof(double));
    double* gy = calloc(nnz, sizeof(double));
    double* cc = calloc(nnz, sizeof(double));
    double* vol = calloc(n, sizeof(double));
    for (int P = 0; P < n; ++P) {
        double px = xy[2 * P], py = xy[2 * P + 1];
        double V = 0.0;
        for (int e = tstart[P]; e < tstart[P + 1]; ++e) {
            const int32_t* v = tri + 3 * tlist[e];
            /* rotate so that the pivot comes first, keeping the cyclic order */
            int r = (v[0] == P) ? 0 : (v[1] == P) ? 1 : 2;
            int iq = v[(r + 1) % 3], ir = v[(r + 2) % 3];
            double qx = xy[2 * iq], qy = xy[2 * iq + 1], rx = xy[2 * ir], ry = xy[2 * ir + 1];
            if (period_x > 0) {
                qx -= period_x * round((qx - px) / period_x);
                rx -= period_x * round((rx - px) / period_x);
            }
            if (period_y > 0) {
                qy -= period_y * round((qy - py) / period_y);
                ry -= period_y * round((ry - py) / period_y);
            }
            double tri_area2 = (qx - px) * (ry - py) - (rx - px) * (qy - py);
            double s = tri_area2 > 0 ? 1.0 : -1.0;
            /* sub-region of CV(P) in this triangle: P -> M_PQ -> G -> M_PR */
            double X[4] = {px, 0.5 * (px + qx), (px + qx + rx) / 3.0, 0.5 * (px + rx)};
            double Y[4] = {py, 0.5 * (py + qy), (py + qy + ry) / 3.0, 0.5 * (py + ry)};
            int32_t ids[3] = {P, iq, ir};
            /* boundary flux: outward normal times length, phi_k at the edge midpoint */
            for (int j = 0; j < 4; ++j) {
                double ax = X[j], ay = Y[j], bx = X[(j + 1) % 4], by = Y[(j + 1) % 4];
                double nx = s * (by - ay), ny = -s * (bx - ax);
                double l[3];
                bary(px, py, qx, qy, rx, ry, 0.5 * (ax + bx), 0.5 * (ay + by), l);
                for (int a = 0; a < 3; ++a)
                    for (int c = row_ptr[P]; c < row_ptr[P + 1]; ++c)
                        if (col[c] == ids[a]) {
                            gx[c] += nx * l[a];
                            gy[c] += ny * l[a];
                        }
            }
            /* volume integral of phi_k: two sub-triangles, vertex rule */
            int sub[2][3] = {{0, 1, 2}, {0, 2, 3}};
            for (int h = 0; h < 2; ++h) {
                double ax = X[sub[h][0]], ay = Y[sub[h][0]];
                double bx = X[sub[h][1]], by = Y[sub[h][1]];
                double cx = X[sub[h][2]], cy = Y[sub[h][2]];
                double area = 0.5 * fabs((bx - ax) * (cy - ay) - (cx - ax) * (by - ay));
                V += area;
                double la[3], lb[3], lc[3];
                bary(px, py, qx, qy, rx, ry, ax, ay, la);
                bary(px, py, qx, qy, rx, ry, bx, by, lb);
                bary(px, py, qx, qy, rx, ry, cx, cy, lc);
                for (int a = 0; a < 3; ++a)
                    for (int c = row_ptr[P]; c < row_ptr[P + 1]; ++c)
                        if (col[c] == ids[a]) cc[c] += area * (la[a] + lb[a] + lc[a]) / 3.0;
            }
        }
        vol[P] = V;
        for (int c = row_ptr[P]; c < row_ptr[P + 1]; ++c) {
            gx[c] = -gx[c] / V;
            gy[c] = -gy[c] / V;
            cc[c] = lumped ? (col[c] == P ? 1.0 : 0.0) : cc[c] / V;
        }
    }
    free(tstart);
    free(tlist);
    out->row_ptr = row_ptr;
    out->col = col;
    out->gx = gx;
    out->gy = gy;
    out->cc = cc;
    out->vol = vol;
}

/* One explicit step of eq. ulbe at node P:
 * f_P + dt_u * sum_k [ (c_i . g_Pk) f_k - (C_Pk / tau_u) (f_k - f_k^eq) ] */
static void fv_update_node(int P, const fv_coeffs_t* fc, const double* fin, const double* feq_in,
                           double tau_u, double dt_u, double* fout) {
    double acc[9] = {0};
    for (int e = fc->row_ptr[P]; e < fc->row_ptr[P + 1]; ++e) {
        int k = fc->col[e];
        for (int i = 0; i < 9; ++i) {
            double S = CX[i] * fc->gx[e] + CY[i] * fc->gy[e];
            acc[i] += S * fin[9 * k + i] - fc->cc[e] / tau_u * (fin[9 * k + i] - feq_in[9 * k + i]);
        }
    }
    for (int i = 0; i < 9; ++i) fout[9 * P + i] = fin[9 * P + i] + dt_u * acc[i];
}

int orc_fv_periodic(int n_nodes, const double* xy, int n_tris, const int32_t* tri, double period_x,
                    double period_y, double tau_u, double dt_u, int lumped, int n_iter, double* f9) {
    fv_coeffs_t fc;
    build_fv(n_nodes, xy, n_tris, tri, period_x, period_y, lumped, &fc);
    double* f2 = malloc((size_t)n_nodes * 9 * sizeof(double));
    double* feq = malloc((size_t)n_nodes * 9 * sizeof(double));
    double *a = f9, *b = f2;
    for (int it = 0; it < n_iter; ++it) {
        for (int P = 0; P < n_nodes; ++P) {
            double r, ux, uy;
            moments(a + 9 * P, &r, &ux, &uy);
            orc_feq(r, ux, uy, feq + 9 * P);
        }
        for (int P = 0; P < n_nodes; ++P) fv_update_node(P, &fc, a, feq, tau_u, dt_u, b);
        double* t = a;
        a = b;
        b = t;
    }
    if (a != f9) memcpy(f9, a, (size_t)n_nodes * 9 * sizeof(double));
    free(f2);
    free(feq);
    free(fc.row_ptr);
    free(fc.col);
    free(fc.gx);
    free(fc.gy);
    free(fc.cc);
    free(fc.vol);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* structured LBGK (Sec. 3, eq. LBE) with the Sec. 5 boundaries (R5)         */
/* ------------------------------------------------------------------------ */
static void bgk_collide(const double* f, double tau, double* post) {
    double r, ux, uy, feq[9];
    moments(f, &r, &ux, &uy);
    orc_feq(r, ux, uy, feq);
    for (int i = 0; i < 9; ++i) post[i] = f[i] - (f[i] - feq[i]) / tau;
}

/* R13: the factor 1 - sigma(d) of node (x, y), d its distance in rows from
 * the nearest outflow side; 1 outside the layer */
static double sponge_keep(int nx, int ny, int bcx, int bcy, int rows, double sigma, int x, int y) {
    if (rows <= 0 || sigma == 0.0) return 1.0;
    int d = rows;
    if (bcy == ORC_BC_OUTFLOW) {
        d = y < d ? y : d;
        d = ny - 1 - y < d ? ny - 1 - y : d;
    }
    if (bcx == ORC_BC_OUTFLOW) {
        d = x < d ? x : d;
        d = nx - 1 - x < d ? nx - 1 - x : d;
    }
    if (d >= rows) return 1.0;
    const double t = (double)(rows - d) / (double)rows;
    return 1.0 - sigma * t * t;
}

/* R13 applied to a post-collision set (keep < 1 only inside the layer) */
static void sponge_apply(double keep, double rho0, double* post) {
    if (keep == 1.0) return;
    for (int i = 0; i < 9; ++i) post[i] = W[i] * rho0 + keep * (post[i] - W[i] * rho0);
}

/* f_i(x, y, t+1) from the post-collision field (pull form of eq. LBE).
 * Sets *bad if the source node is not a computed node. */
static double pull(int nx, int ny, int bcx, int bcy, const double* post, int64_t N, int x, int y,
                   int i, const int8_t* cls, int* bad) {
    int sx = x - CX[i], sy = y - CY[i];
    if (sx < 0 || sx >= nx) {
        if (bcx == ORC_BC_PERIODIC)
            sx = (sx + nx) % nx;
        else if (bcx == ORC_BC_WALL)
            return post[OPP[i] * N + (int64_t)y * nx + x];
        else
            sx = x;
    }
    if (sy < 0 || sy >= ny) {
        if (bcy == ORC_BC_PERIODIC)
            sy = (sy + ny) % ny;
        else if (bcy == ORC_BC_WALL)
            return post[OPP[i] * N + (int64_t)y * nx + x];
        else
            sy = y;
    }
    int64_t s = (int64_t)sy * nx + sx;
    if (cls && cls[s] == ORC_UNUSED) *bad = 1;
    return post[i * N + s];
}

/* ------------------------------------------------------------------------ */
/* nested lattice levels (R12)                                               */
/* ------------------------------------------------------------------------ */
/* level 0 is the nx x ny lattice around the patch; level k >= 1 is
 * o->lv[k - 1], with twice the spacing and time step of level k - 1 */
static double tau_level(const orc_t* o, int k) { return 0.5 + ldexp(o->p.tau_s - 0.5, -k); }

static int level_nx(const orc_t* o, int k) { return k == 0 ? o->p.nx : o->lv[k - 1].nx; }
static int level_ny(const orc_t* o, int k) { return k == 0 ? o->p.ny : o->lv[k - 1].ny; }

/* the outermost ring of level k < n_levels takes its values from level k+1 */
static int is_ring_k(const orc_t* o, int k, int x, int y) {
    return k < o->p.n_levels && (x == 0 || y == 0 || x == level_nx(o, k) - 1 || y == level_ny(o, k) - 1);
}
static int is_ring(const orc_t* o, int x, int y) { return is_ring_k(o, 0, x, y); }

/* rho, ux, uy, f^neq of node s of level k >= 1, buffer b */
static void level_state(const orc_t* o, int k, int b, int64_t s, double* st) {
    const orc_level_t* L = &o->lv[k - 1];
    double f[9], fneq[9];
    for (int i = 0; i < 9; ++i) f[i] = L->f[b][i * L->N + s];
    state_of(f, &st[0], &st[1], &st[2], fneq);
    for (int i = 0; i < 9; ++i) st[3 + i] = fneq[i];
}

/* coarse nodes and weights giving a value at fine coordinate X along one
 * axis: the coarse node itself (X even) or the cubic Lagrange midpoint rule
 * over the four nearest coarse nodes (X odd) */
static int axis_weights(int X, int* idx, double* w) {
    if (X % 2 == 0) {
        idx[0] = X / 2;
        w[0] = 1.0;
        return 1;
    }
    const int I0 = (X - 1) / 2;
    const double cw[4] = {-1.0 / 16.0, 9.0 / 16.0, 9.0 / 16.0, -1.0 / 16.0};
    for (int k = 0; k < 4; ++k) {
        idx[k] = I0 - 1 + k;
        w[k] = cw[k];
    }
    return 4;
}

/* post-collision populations of ring node (x, y) of level k at its time tk:
 * rho, u and f^neq of level k+1 at the node's position (cubic along the box
 * edge; at odd tk the mean of level k+1's times tk/2 -/+ 1/2), then
 * f^eq(rho, u) + f^neq rescaled to level k */
static void ghost_post(const orc_t* o, int k, int x, int y, int64_t tk, double* post) {
    const orc_level_t* C = &o->lv[k]; /* level k+1 */
    int I[4], J[4];
    double wi[4], wj[4];
    const int ni = axis_weights(2 * C->ox + x, I, wi);
    const int nj = axis_weights(2 * C->oy + y, J, wj);
    double st[12] = {0};
    const int nb = (tk % 2 == 0) ? 1 : 2;
    const int bufs[2] = {C->cur, 1 - C->cur};
    for (int q = 0; q < nb; ++q)
        for (int c = 0; c < nj; ++c)
            for (int a = 0; a < ni; ++a) {
                double w = wi[a] * wj[c] / nb, sc[12];
                level_state(o, k + 1, bufs[q], (int64_t)J[c] * C->nx + I[a], sc);
                for (int j = 0; j < 12; ++j) st[j] += w * sc[j];
            }
    const double tf = tau_level(o, k), tc = tau_level(o, k + 1);
    const double acf = (tf - 1.0) / (2.0 * (tc - 1.0));
    double feq[9];
    orc_feq(st[0], st[1], st[2], feq);
    for (int i = 0; i < 9; ++i) post[i] = feq[i] + acf * st[3 + i];
}

/* the ring of level k takes its post-collision ghost for its time tk, into
 * the current buffer (level 0: the pre-collision array, whose moments are
 * then the ring's rho and u) */
static void fill_ring(orc_t* o, int k, int64_t tk) {
    const int nx = level_nx(o, k), ny = level_ny(o, k);
    double* dst = k == 0 ? o->fs[o->cur] : o->lv[k - 1].f[o->lv[k - 1].cur];
    const int64_t N = k == 0 ? o->N : o->lv[k - 1].N;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            if (!is_ring_k(o, k, x, y)) continue;
            double post[9];
            ghost_post(o, k, x, y, tk, post);
            for (int i = 0; i < 9; ++i) dst[i * N + (int64_t)y * nx + x] = post[i];
        }
}

/* level k >= 1 streams and collides from f[cur] into f[1 - cur]; the
 * coarsest level has the lattice's boundaries, a finer one zero-gradient
 * edges (its ring is rebuilt afterwards) */
static void level_step(orc_t* o, int k) {
    orc_level_t* L = &o->lv[k - 1];
    const int coarsest = k == o->p.n_levels;
    const int bcx = coarsest ? o->p.bc_x : ORC_BC_OUTFLOW, bcy = coarsest ? o->p.bc_y : ORC_BC_OUTFLOW;
    const double* post = L->f[L->cur];
    double* out = L->f[1 - L->cur];
    const double tc = tau_level(o, k);
    int bad = 0;
    for (int y = 0; y < L->ny; ++y)
        for (int x = 0; x < L->nx; ++x) {
            double f[9], q[9];
            for (int i = 0; i < 9; ++i) f[i] = pull(L->nx, L->ny, bcx, bcy, post, L->N, x, y, i, NULL, &bad);
            bgk_collide(f, tc, q);
            if (coarsest)
                sponge_apply(sponge_keep(L->nx, L->ny, bcx, bcy, o->p.sponge_rows, o->p.sponge_sigma, x, y),
                             o->p.rho0, q);
            for (int i = 0; i < 9; ++i) out[i * L->N + (int64_t)y * L->nx + x] = q[i];
        }
}

/* the nodes of level k+1 strictly inside level k's box take the
 * post-collision state of the level-k node under them, f^eq + f^neq
 * rescaled, into level k+1's buffer b.  Level 0's state is its pre-collision
 * array at an even time, collided; a level-0 node that is not computed
 * (under the lamina) gives f^eq(rho0, 0), which nothing retained reads. */
static void restrict_level(orc_t* o, int k, int b) {
    orc_level_t* C = &o->lv[k];
    const int nx = level_nx(o, k), ny = level_ny(o, k);
    const double tf = tau_level(o, k), tc = tau_level(o, k + 1);
    const double afc = 2.0 * (tc - 1.0) / (tf - 1.0);
    for (int J = C->oy + 1; J < C->oy + (ny - 1) / 2; ++J)
        for (int I = C->ox + 1; I < C->ox + (nx - 1) / 2; ++I) {
            const int x = 2 * (I - C->ox), y = 2 * (J - C->oy);
            const int64_t sc = (int64_t)J * C->nx + I;
            double post[9];
            if (k == 0) {
                const int64_t s = (int64_t)y * nx + x;
                if (o->cls_cur[s] == ORC_DISC) {
                    double f[9];
                    for (int i = 0; i < 9; ++i) f[i] = o->fs[o->cur][i * o->N + s];
                    bgk_collide(f, tf, post);
                } else {
                    orc_feq(o->p.rho0, 0.0, 0.0, post);
                }
            } else {
                const orc_level_t* F = &o->lv[k - 1];
                const int64_t s = (int64_t)y * F->nx + x;
                for (int i = 0; i < 9; ++i) post[i] = F->f[F->cur][i * F->N + s];
            }
            double r, ux, uy, fneq[9], feq[9];
            state_of(post, &r, &ux, &uy, fneq);
            orc_feq(r, ux, uy, feq);
            for (int i = 0; i < 9; ++i) C->f[b][i * C->N + sc] = feq[i] + afc * fneq[i];
        }
}

void orc_level_macro(const orc_t* o, int k, double* rho, double* ux, double* uy) {
    const orc_level_t* L = &o->lv[k - 1];
    for (int64_t s = 0; s < L->N; ++s) {
        double st[12];
        level_state(o, k, L->cur, s, st);
        rho[s] = st[0];
        ux[s] = st[1];
        uy[s] = st[2];
    }
}

int orc_lbgk(int nx, int ny, int bc_x, int bc_y, double tau_s, int sponge_rows, double sponge_sigma, int n_iter,
             double* f9) {
    int64_t N = (int64_t)nx * ny;
    double* post = malloc((size_t)N * 9 * sizeof(double));
    int bad = 0;
    for (int it = 0; it < n_iter; ++it) {
        for (int64_t s = 0; s < N; ++s) {
            double f[9], q[9];
            for (int i = 0; i < 9; ++i) f[i] = f9[i * N + s];
            bgk_collide(f, tau_s, q);
            /* R13 with rho0 = 1 */
            sponge_apply(sponge_keep(nx, ny, bc_x, bc_y, sponge_rows, sponge_sigma, (int)(s % nx), (int)(s / nx)), 1.0,
                         q);
            for (int i = 0; i < 9; ++i) post[i * N + s] = q[i];
        }
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                for (int i = 0; i < 9; ++i)
                    f9[i * N + (int64_t)y * nx + x] = pull(nx, ny, bc_x, bc_y, post, N, x, y, i, NULL, &bad);
    }
    free(post);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* node classification (Sec. 4)                                              */
/* ------------------------------------------------------------------------ */
/* inside the fictitious curve: the rounded rectangle at offset delta_f */
static int inside_fictitious(const orc_t* o, int x, int y, double cx, double cy) {
    double qx = fabs((double)x - cx) - 0.5 * o->p.L;
    double qy = fabs((double)y - cy) - 0.5 * o->p.T;
    if (qx < 0.0) qx = 0.0;
    if (qy < 0.0) qy = 0.0;
    return qx * qx + qy * qy < o->p.delta_f * o->p.delta_f;
}

/* discretization outside the curve; unused inside; unused nodes with a
 * discretization node among their 8 lattice neighbours are interpolation */
static void classify(orc_t* o, double cx, double cy, int8_t* cls) {
    int nx = o->p.nx, ny = o->p.ny;
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t s = (int64_t)y * nx + x;
            if (!inside_fictitious(o, x, y, cx, cy)) {
                cls[s] = ORC_DISC;
                continue;
            }
            cls[s] = ORC_UNUSED;
            for (int i = 1; i < 9; ++i) {
                int xx = x + CX[i], yy = y + CY[i];
                if (xx < 0 || yy < 0 || xx >= nx || yy >= ny) continue;
                if (!inside_fictitious(o, xx, yy, cx, cy)) {
                    cls[s] = ORC_INTERP;
                    break;
                }
            }
        }
}

/* ------------------------------------------------------------------------ */
/* interpolations (Sec. 4; R7)                                               */
/* ------------------------------------------------------------------------ */
/* bilinear Lagrange interpolation of rho, u, f^neq over the four structured
 * donors of the cell enclosing (wx, wy); cls (if given) must mark them as
 * discretization nodes */
static void bilinear_state(orc_t* o, const double* fs, const int8_t* cls, double wx, double wy,
                           double* st, int32_t* cell) {
    int nx = o->p.nx, ny = o->p.ny;
    double fx0 = floor(wx), fy0 = floor(wy);
    int ix = (int)fx0, iy = (int)fy0;
    double ax = wx - fx0, ay = wy - fy0;
    double w[4] = {(1.0 - ax) * (1.0 - ay), ax * (1.0 - ay), (1.0 - ax) * ay, ax * ay};
    int dxs[4] = {0, 1, 0, 1}, dys[4] = {0, 0, 1, 1};
    for (int j = 0; j < 12; ++j) st[j] = 0.0;
    if (cell) *cell = iy * nx + ix;
    for (int d = 0; d < 4; ++d) {
        int x = ix + dxs[d], y = iy + dys[d];
        if (x < 0 || y < 0 || x >= nx || y >= ny) {
            o->status |= ORC_ERR_DONOR_NOT_COMPUTED;
            continue;
        }
        int64_t s = (int64_t)y * nx + x;
        if (cls && cls[s] != ORC_DISC) o->status |= ORC_ERR_DONOR_NOT_COMPUTED;
        double f[9], r, ux, uy, fneq[9];
        for (int i = 0; i < 9; ++i) f[i] = fs[i * o->N + s];
        state_of(f, &r, &ux, &uy, fneq);
        st[0] += w[d] * r;
        st[1] += w[d] * ux;
        st[2] += w[d] * uy;
        for (int i = 0; i < 9; ++i) st[3 + i] += w[d] * fneq[i];
    }
}

/* Eq. continuity_stresses (type 1): f = f^eq(rho, u) + (1 - 1/(2 tau_s)) f^neq,s */
static void f_from_struct_state(const orc_t* o, const double* st, double* f) {
    double feq[9], k = 1.0 - 1.0 / (2.0 * o->p.tau_s);
    orc_feq(st[0], st[1], st[2], feq);
    for (int i = 0; i < 9; ++i) f[i] = feq[i] + k * st[3 + i];
}

/* ------------------------------------------------------------------------ */
/* refill procedure (Sec. 4)                                                 */
/* ------------------------------------------------------------------------ */
static void refill(orc_t* o, double X0, double Y0, double X1, double Y1) {
    double dX = X1 - X0, dY = Y1 - Y0;
    double cx = o->p.xc + X1, cy = o->p.yc + Y1;
    double a = 0.5 * o->p.L, b = 0.5 * o->p.T;
    const double* fold = o->fu[o->ucur];
    double* fnew = o->fu[1 - o->ucur];
    for (int P = 0; P < o->p.n_nodes; ++P) {
        double* fo = fnew + 9 * P;
        if (o->kind[P] == ORC_KIND_WALL) {
            /* wall nodes keep their own density and distributions; the wall
             * velocity is imposed during the sub-steps (R3) */
            memcpy(fo, fold + 9 * P, 9 * sizeof(double));
            o->rtype[P] = 0;
            o->rdonor[P] = -1;
            continue;
        }
        /* the new node position seen in the previous mesh configuration */
        double qx = o->xy[2 * P] + dX, qy = o->xy[2 * P + 1] + dY;
        double lam[3];
        int k = locate(o, qx, qy, lam);
        if (k >= 0) {
            /* type 3: barycentric interpolation over the enclosing triangle */
            const int32_t* v = o->tri + 3 * k;
            for (int i = 0; i < 9; ++i)
                fo[i] = lam[0] * fold[9 * v[0] + i] + lam[1] * fold[9 * v[1] + i] +
                        lam[2] * fold[9 * v[2] + i];
            o->rtype[P] = 3;
            o->rdonor[P] = k;
        } else if (fabs(qx) <= a && fabs(qy) <= b) {
            /* type 2: inside the body, keep the node's previous values */
            memcpy(fo, fold + 9 * P, 9 * sizeof(double));
            o->rtype[P] = 2;
            o->rdonor[P] = -1;
        } else {
            /* type 1: bilinear from the structured state at time t */
            double st[12];
            int32_t cell;
            bilinear_state(o, o->fs[o->cur], o->cls_prev, cx + o->xy[2 * P], cy + o->xy[2 * P + 1], st,
                           &cell);
            f_from_struct_state(o, st, fo);
            o->rtype[P] = 1;
            o->rdonor[P] = cell;
        }
    }
    o->ucur = 1 - o->ucur;
}

/* ------------------------------------------------------------------------ */
/* eq. postcollision2_s at structured interpolation nodes                    */
/* ------------------------------------------------------------------------ */
static void post_from_patch(orc_t* o, int x, int y, double cx, double cy, double* post) {
    double qx = (double)x - cx, qy = (double)y - cy;
    double lam[3];
    int k = locate(o, qx, qy, lam);
    if (k < 0) {
#pragma omp atomic
        o->status |= ORC_ERR_FILL_NOT_LOCATED;
        orc_feq(o->p.rho0, 0.0, 0.0, post);
        return;
    }
    const int32_t* v = o->tri + 3 * k;
    double st[12] = {0};
    for (int j = 0; j < 3; ++j) {
        double r, ux, uy, fneq[9];
        state_of(o->fu[o->ucur] + 9 * v[j], &r, &ux, &uy, fneq);
        st[0] += lam[j] * r;
        st[1] += lam[j] * ux;
        st[2] += lam[j] * uy;
        for (int i = 0; i < 9; ++i) st[3 + i] += lam[j] * fneq[i];
    }
    double feq[9], ts = o->p.tau_s;
    double k178 = 2.0 * (ts - 1.0) / (2.0 * ts - 1.0);
    orc_feq(st[0], st[1], st[2], feq);
    for (int i = 0; i < 9; ++i) post[i] = feq[i] + k178 * st[3 + i];
}

static void structured_step(orc_t* o, double cx, double cy) {
    int nx = o->p.nx, ny = o->p.ny;
    int64_t N = o->N;
    const double* f = o->fs[o->cur];
    double* fn = o->fs[1 - o->cur];
    /* every node's update reads only the previous state: the loops may run
     * in parallel (OpenMP build of the CPU baseline), with the same results */
#pragma omp parallel for schedule(static)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t s = (int64_t)y * nx + x;
            int8_t c = o->cls_cur[s];
            if (c == ORC_UNUSED) continue;
            double post[9];
            if (is_ring(o, x, y)) {
                for (int i = 0; i < 9; ++i) post[i] = f[i * N + s]; /* R12: the ring holds its ghost */
            } else if (c == ORC_INTERP || o->cls_prev[s] != ORC_DISC) {
                if (c == ORC_DISC && o->cls_prev[s] == ORC_UNUSED) {
#pragma omp atomic
                    o->status |= ORC_ERR_UNUSED_TO_DISC;
                }
                post_from_patch(o, x, y, cx, cy, post);
            } else {
                double fl[9];
                for (int i = 0; i < 9; ++i) fl[i] = f[i * N + s];
                bgk_collide(fl, o->p.tau_s, post);
                if (o->p.n_levels == 0)
                    sponge_apply(sponge_keep(nx, ny, o->p.bc_x, o->p.bc_y, o->p.sponge_rows, o->p.sponge_sigma, x, y),
                                 o->p.rho0, post);
            }
            for (int i = 0; i < 9; ++i) o->fpost[i * N + s] = post[i];
        }
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(| : bad)
    for (int y = 0; y < ny; ++y)
        for (int x = 0; x < nx; ++x) {
            int64_t s = (int64_t)y * nx + x;
            if (o->cls_cur[s] != ORC_DISC || is_ring(o, x, y)) continue;
            for (int i = 0; i < 9; ++i)
                fn[i * N + s] = pull(nx, ny, o->p.bc_x, o->p.bc_y, o->fpost, N, x, y, i, o->cls_cur, &bad);
        }
    if (bad) o->status |= ORC_ERR_PULL_SOURCE;
}

/* ------------------------------------------------------------------------ */
/* FV sub-steps on the patch (Sec. 3: eq. ulbe n times per structured step)  */
/* ------------------------------------------------------------------------ */
static void feed_snapshots(orc_t* o, double cx, double cy) {
    for (int P = 0; P < o->p.n_nodes; ++P) {
        if (o->kind[P] != ORC_KIND_OUTER) continue;
        double wx = cx + o->xy[2 * P], wy = cy + o->xy[2 * P + 1];
        bilinear_state(o, o->fs[o->cur], o->cls_prev, wx, wy, o->snap0 + 12 * P, NULL);
        bilinear_state(o, o->fs[1 - o->cur], o->cls_cur, wx, wy, o->snap1 + 12 * P, NULL);
    }
}

/* R10: eq. postcollision2_u with its FV sums at the outer node P; dstar
 * holds the R2 values of the outer nodes at the new sub-step, fin the patch
 * state at sub-step m */
static void outer_fv_update(int P, const fv_coeffs_t* fc, const int8_t* kind, const double* dstar,
                            const double* fin, double tau_u, double dt_u, double* fout) {
    double acc[9] = {0};
    for (int e = fc->row_ptr[P]; e < fc->row_ptr[P + 1]; ++e) {
        int k = fc->col[e];
        const double* fk = kind[k] == ORC_KIND_OUTER ? dstar + 9 * k : fin + 9 * k;
        double r, ux, uy, feq[9];
        moments(fk, &r, &ux, &uy);
        orc_feq(r, ux, uy, feq);
        for (int i = 0; i < 9; ++i) {
            double S = CX[i] * fc->gx[e] + CY[i] * fc->gy[e];
            acc[i] += S * fk[i] - fc->cc[e] / tau_u * (fk[i] - feq[i]);
        }
    }
    for (int i = 0; i < 9; ++i) fout[9 * P + i] = dstar[9 * P + i] + dt_u * acc[i];
}

int orc_outer_fv(int n_nodes, const double* xy, int n_tris, const int32_t* tri, const int8_t* kind,
                 double tau_u, double dt_u, int lumped, const double* fin, const double* dstar, double* fout) {
    fv_coeffs_t fc;
    build_fv(n_nodes, xy, n_tris, tri, 0.0, 0.0, lumped, &fc);
    for (int P = 0; P < n_nodes; ++P)
        if (kind[P] == ORC_KIND_OUTER) outer_fv_update(P, &fc, kind, dstar, fin, tau_u, dt_u, fout);
    free(fc.row_ptr);
    free(fc.col);
    free(fc.gx);
    free(fc.gy);
    free(fc.cc);
    free(fc.vol);
    return 0;
}

static void fv_substeps(orc_t* o, int64_t t) {
    int n = o->p.n_sub, nn = o->p.n_nodes;
    double dtu = 1.0 / n, tau_u = o->p.tau_s - 0.5;
    fv_coeffs_t fc = {o->row_ptr, o->col, o->gx, o->gy, o->cc, o->vol};
    for (int m = 0; m < n; ++m) {
        double theta = (double)(m + 1) / (double)n;
        double U, V;
        if (o->p.motion == ORC_MOTION_INDUCED) {
            U = 0.0;
            V = o->Vh[t] + theta * (o->Vh[t + 1] - o->Vh[t]);
        } else {
            motion_vel(&o->p, (double)t + theta, &U, &V);
        }
        const double* fin = o->fu[o->ucur];
        double* fout = o->fu[1 - o->ucur];
#pragma omp parallel for schedule(static)
        for (int P = 0; P < nn; ++P) {
            double r, ux, uy;
            moments(fin + 9 * P, &r, &ux, &uy);
            orc_feq(r, ux, uy, o->feq_u + 9 * P);
        }
        /* interpolation (outer) nodes: structured state, linear in time (R2) */
#pragma omp parallel for schedule(static)
        for (int P = 0; P < nn; ++P) {
            if (o->kind[P] != ORC_KIND_OUTER) continue;
            double st[12];
            const double *s0 = o->snap0 + 12 * P, *s1 = o->snap1 + 12 * P;
            for (int j = 0; j < 12; ++j) st[j] = (1.0 - theta) * s0[j] + theta * s1[j];
            f_from_struct_state(o, st, o->dstar + 9 * P);
        }
#pragma omp parallel for schedule(static)
        for (int P = 0; P < nn; ++P) {
            if (o->kind[P] == ORC_KIND_OUTER) {
                if (o->p.outer_fv)
                    outer_fv_update(P, &fc, o->kind, o->dstar, fin, tau_u, dtu, fout);
                else
                    memcpy(fout + 9 * P, o->dstar + 9 * P, 9 * sizeof(double));
                continue;
            }
            fv_update_node(P, &fc, fin, o->feq_u, tau_u, dtu, fout);
            if (o->kind[P] == ORC_KIND_WALL) {
                /* no-slip wall moving with the lamina (R3) */
                double r, ux, uy, fa[9], fb[9];
                moments(fout + 9 * P, &r, &ux, &uy);
                orc_feq(r, U, V, fa);
                orc_feq(r, ux, uy, fb);
                for (int i = 0; i < 9; ++i) fout[9 * P + i] += fa[i] - fb[i];
            }
        }
        o->ucur = 1 - o->ucur;
    }
}

/* ------------------------------------------------------------------------ */
/* force on the lamina (Sec. 2.1; R4)                                        */
/* ------------------------------------------------------------------------ */
static void wall_stress(const orc_t* o, const double* f, double* s) {
    double r, ux, uy, fneq[9];
    state_of(f, &r, &ux, &uy, fneq);
    double pxx = 0, pxy = 0, pyy = 0;
    for (int i = 0; i < 9; ++i) {
        pxx += fneq[i] * CX[i] * CX[i];
        pxy += fneq[i] * CX[i] * CY[i];
        pyy += fneq[i] * CY[i] * CY[i];
    }
    double p = (r - o->p.rho0) * CS2;
    s[0] = -p - pxx;
    s[1] = -pxy;
    s[2] = -p - pyy;
}

static void compute_force(orc_t* o, double* Fx, double* Fy) {
    const double* f = o->fu[o->ucur];
    double fx = 0.0, fy = 0.0;
    for (int k = 0; k < o->nseg; ++k) {
        double sa[3], sb[3];
        wall_stress(o, f + 9 * o->seg_a[k], sa);
        wall_stress(o, f + 9 * o->seg_b[k], sb);
        double nx = o->seg_nx[k], ny = o->seg_ny[k];
        fx += 0.5 * ((sa[0] + sb[0]) * nx + (sa[1] + sb[1]) * ny);
        fy += 0.5 * ((sa[1] + sb[1]) * nx + (sa[2] + sb[2]) * ny);
    }
    if (!isfinite(fx) || !isfinite(fy)) o->status |= ORC_ERR_NONFINITE;
    *Fx = fx;
    *Fy = fy;
}

/* wall segments: mesh-boundary edges joining two wall nodes; the normal
 * points away from the body, i.e. towards the triangle's third vertex */
static void build_wall_segments(orc_t* o) {
    int n = o->p.n_nodes, nt = o->p.n_tris;
    int32_t* tstart = calloc(n + 1, sizeof(int32_t));
    for (int k = 0; k < nt; ++k)
        for (int j = 0; j < 3; ++j) tstart[o->tri[3 * k + j] + 1]++;
    for (int i = 0; i < n; ++i) tstart[i + 1] += tstart[i];
    int32_t* tlist = malloc((size_t)tstart[n] * sizeof(int32_t));
    int32_t* fillc = calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    for (int k = 0; k < nt; ++k)
        for (int j = 0; j < 3; ++j) {
            int v = o->tri[3 * k + j];
            tlist[tstart[v] + fillc[v]++] = k;
        }
    free(fillc);
    int cap = 1024;
    o->seg_a = malloc(cap * sizeof(int32_t));
    o->seg_b = malloc(cap * sizeof(int32_t));
    o->seg_nx = malloc(cap * sizeof(double));
    o->seg_ny = malloc(cap * sizeof(double));
    o->nseg = 0;
    for (int k = 0; k < nt; ++k)
        for (int j = 0; j < 3; ++j) {
            int a = o->tri[3 * k + j], b = o->tri[3 * k + (j + 1) % 3], c = o->tri[3 * k + (j + 2) % 3];
            if (o->kind[a] != ORC_KIND_WALL || o->kind[b] != ORC_KIND_WALL) continue;
            int shared = 0;
            for (int e = tstart[a]; e < tstart[a + 1]; ++e) {
                int k2 = tlist[e];
                if (k2 == k) continue;
                const int32_t* v = o->tri + 3 * k2;
                if (v[0] == b || v[1] == b || v[2] == b) shared = 1;
            }
            if (shared) continue;
            double ex = o->xy[2 * b] - o->xy[2 * a], ey = o->xy[2 * b + 1] - o->xy[2 * a + 1];
            double nx = ey, ny = -ex;
            double tx = o->xy[2 * c] - o->xy[2 * a], ty = o->xy[2 * c + 1] - o->xy[2 * a + 1];
            if (nx * tx + ny * ty < 0) {
                nx = -nx;
                ny = -ny;
            }
            if (o->nseg == cap) {
                cap *= 2;
                o->seg_a = realloc(o->seg_a, cap * sizeof(int32_t));
                o->seg_b = realloc(o->seg_b, cap * sizeof(int32_t));
                o->seg_nx = realloc(o->seg_nx, cap * sizeof(double));
                o->seg_ny = realloc(o->seg_ny, cap * sizeof(double));
            }
            o->seg_a[o->nseg] = a;
            o->seg_b[o->nseg] = b;
            o->seg_nx[o->nseg] = nx;
            o->seg_ny[o->nseg] = ny;
            o->nseg++;
        }
    free(tstart);
    free(tlist);
}

int orc_n_wall_segments(const orc_t* o) { return o->nseg; }

/* ------------------------------------------------------------------------ */
/* hydrodynamic function (Sec. 2.1, eq. force_phasor)                        */
/* ------------------------------------------------------------------------ */
/* least squares of F(t) = F0 sin(w t + phi) = a sin(w t) + b cos(w t) */
void orc_sine_fit(const double* F, int64_t t0, int64_t t1, double omega, double* a, double* b,
                  double* rms) {
    double ss = 0, sc = 0, cc = 0, fs = 0, fc = 0;
    for (int64_t t = t0; t <= t1; ++t) {
        double s = sin(omega * (double)t), c = cos(omega * (double)t);
        ss += s * s;
        sc += s * c;
        cc += c * c;
        fs += F[t] * s;
        fc += F[t] * c;
    }
    double det = ss * cc - sc * sc;
    *a = (fs * cc - fc * sc) / det;
    *b = (fc * ss - fs * sc) / det;
    double r2 = 0;
    for (int64_t t = t0; t <= t1; ++t) {
        double e = F[t] - (*a * sin(omega * (double)t) + *b * cos(omega * (double)t));
        r2 += e * e;
    }
    *rms = sqrt(r2 / (double)(t1 - t0 + 1));
}

/* Theta of a force history F[0..n-1] (eq. force_phasor): the sine fit over
 * t in [ceil(discard T), floor((discard + fit) T)], T = 2 pi / w, gives
 * F-hat = F0 e^{i phi} = a + i b, and F-hat = (pi/4) rho w^2 L^2 Theta A. */
int orc_theta(const double* F, int64_t n, double rho0, double omega, double L, double A, double discard_periods,
              double fit_periods, double* re, double* im, double* rms) {
    if (omega <= 0) return -1;
    double Tp = 2.0 * ORC_PI / omega;
    int64_t t0 = (int64_t)ceil(discard_periods * Tp);
    int64_t t1 = (int64_t)floor((discard_periods + fit_periods) * Tp);
    if (t1 >= n || t1 <= t0) return -2;
    double a, b;
    orc_sine_fit(F, t0, t1, omega, &a, &b, rms);
    double N = 0.25 * ORC_PI * rho0 * omega * omega * L * L * A;
    *re = a / N;
    *im = b / N;
    *rms /= N;
    return 0;
}

int orc_gamma(const orc_t* o, double discard_periods, double fit_periods, double* re, double* im,
              double* rms) {
    if (o->p.motion != ORC_MOTION_HARMONIC) return -1;
    return orc_theta(o->Fy, o->t + 1, o->p.rho0, o->p.omega, o->p.L, o->p.A, discard_periods, fit_periods, re, im,
                     rms);
}

/* ------------------------------------------------------------------------ */
/* lifecycle                                                                 */
/* ------------------------------------------------------------------------ */
static void record_force(orc_t* o) {
    if (o->t + 1 > o->hcap) {
        o->hcap = 2 * (o->t + 1) + 1024;
        o->Fx = realloc(o->Fx, o->hcap * sizeof(double));
        o->Fy = realloc(o->Fy, o->hcap * sizeof(double));
    }
    compute_force(o, &o->Fx[o->t], &o->Fy[o->t]);
}

orc_t* orc_create(const orc_params_t* p) {
    orc_t* o = calloc(1, sizeof(orc_t));
    o->p = *p;
    int n = p->n_nodes, nt = p->n_tris;
    o->xy = malloc((size_t)n * 2 * sizeof(double));
    memcpy(o->xy, p->xy, (size_t)n * 2 * sizeof(double));
    o->tri = malloc((size_t)nt * 3 * sizeof(int32_t));
    memcpy(o->tri, p->tri, (size_t)nt * 3 * sizeof(int32_t));
    o->kind = malloc(n);
    memcpy(o->kind, p->kind, n);
    o->p.xy = o->xy;
    o->p.tri = o->tri;
    o->p.kind = o->kind;
    o->p.rho_init = NULL;
    o->p.ux_init = NULL;
    o->p.uy_init = NULL;
    o->N = (int64_t)p->nx * p->ny;
    for (int b = 0; b < 2; ++b) o->fs[b] = malloc((size_t)o->N * 9 * sizeof(double));
    o->fpost = malloc((size_t)o->N * 9 * sizeof(double));
    o->cls_prev = malloc(o->N);
    o->cls_cur = malloc(o->N);
    for (int b = 0; b < 2; ++b) o->fu[b] = calloc((size_t)n * 9, sizeof(double));
    o->feq_u = malloc((size_t)n * 9 * sizeof(double));
    o->snap0 = calloc((size_t)n * 12, sizeof(double));
    o->snap1 = calloc((size_t)n * 12, sizeof(double));
    o->dstar = calloc((size_t)n * 9, sizeof(double));
    o->rtype = calloc(n, sizeof(int32_t));
    o->rdonor = malloc(n * sizeof(int32_t));
    for (int i = 0; i < n; ++i) o->rdonor[i] = -1;
    fv_coeffs_t fc;
    build_fv(n, o->xy, nt, o->tri, 0.0, 0.0, p->lumped, &fc);
    o->row_ptr = fc.row_ptr;
    o->col = fc.col;
    o->gx = fc.gx;
    o->gy = fc.gy;
    o->cc = fc.cc;
    o->vol = fc.vol;
    build_wall_segments(o);
    bins_build(o);
    /* initial state: equilibrium at rho_init and the initial velocity */
    for (int64_t s = 0; s < o->N; ++s) {
        double feq[9];
        orc_feq(p->rho_init ? p->rho_init[s] : p->rho0, p->ux_init ? p->ux_init[s] : p->u0x,
                p->uy_init ? p->uy_init[s] : p->u0y, feq);
        for (int i = 0; i < 9; ++i) o->fs[0][i * o->N + s] = feq[i];
    }
    o->cur = 0;
    o->mcap = 1024;
    o->Yh = calloc((size_t)o->mcap, sizeof(double));
    o->Vh = calloc((size_t)o->mcap, sizeof(double));
    o->Yh[0] = p->motion == ORC_MOTION_INDUCED ? p->y0 : 0.0;
    o->Vh[0] = p->motion == ORC_MOTION_INDUCED ? p->v0 : 0.0;
    double X, Y;
    lamina_pos(o, 0, &X, &Y);
    double cx = p->xc + X, cy = p->yc + Y;
    classify(o, cx, cy, o->cls_cur);
    memcpy(o->cls_prev, o->cls_cur, o->N);
    /* the patch starts from the structured field, by the type-1 rule */
    for (int P = 0; P < n; ++P) {
        double st[12];
        bilinear_state(o, o->fs[0], NULL, cx + o->xy[2 * P], cy + o->xy[2 * P + 1], st, NULL);
        f_from_struct_state(o, st, o->fu[0] + 9 * P);
    }
    o->ucur = 0;
    o->t = 0;
    o->Xprev = X;
    o->Yprev = Y;
    /* R12: coarser levels at equilibrium, then each restricted from the one
     * inside it (finest first) and every ring rebuilt */
    for (int k = 1; k <= p->n_levels; ++k) {
        orc_level_t* L = &o->lv[k - 1];
        L->nx = p->lv_nx[k - 1];
        L->ny = p->lv_ny[k - 1];
        L->ox = p->lv_ox[k - 1];
        L->oy = p->lv_oy[k - 1];
        L->N = (int64_t)L->nx * L->ny;
        for (int b = 0; b < 2; ++b) L->f[b] = calloc((size_t)L->N * 9, sizeof(double));
        for (int64_t sc = 0; sc < L->N; ++sc) {
            double feq[9];
            orc_feq(p->lv_rho[k - 1] ? p->lv_rho[k - 1][sc] : p->rho0, p->lv_ux[k - 1] ? p->lv_ux[k - 1][sc] : p->u0x,
                    p->lv_uy[k - 1] ? p->lv_uy[k - 1][sc] : p->u0y, feq);
            for (int i = 0; i < 9; ++i) L->f[0][i * L->N + sc] = feq[i];
        }
        L->cur = 0;
        o->p.lv_rho[k - 1] = NULL;
        o->p.lv_ux[k - 1] = NULL;
        o->p.lv_uy[k - 1] = NULL;
    }
    for (int k = 0; k < p->n_levels; ++k) restrict_level(o, k, 0);
    for (int k = 0; k < p->n_levels; ++k) fill_ring(o, k, 0);
    record_force(o);
    return o;
}

int orc_step(orc_t* o, int64_t nsteps) {
    for (int64_t s = 0; s < nsteps; ++s) {
        int64_t t = o->t;
        if (o->p.motion == ORC_MOTION_INDUCED) {
            /* R11: one symplectic Euler step with the force at t */
            if (t + 2 > o->mcap) {
                o->mcap = 2 * (t + 2) + 1024;
                o->Yh = realloc(o->Yh, (size_t)o->mcap * sizeof(double));
                o->Vh = realloc(o->Vh, (size_t)o->mcap * sizeof(double));
            }
            const orc_params_t* q = &o->p;
            double a = (o->Fy[t] - q->damping * o->Vh[t] - q->stiffness * o->Yh[t]) / q->mass;
            o->Vh[t + 1] = o->Vh[t] + a;
            o->Yh[t + 1] = o->Yh[t] + o->Vh[t + 1];
            if (!(fabs(o->Vh[t + 1]) < 1.0)) o->status |= ORC_ERR_FAST_MOTION;
        }
        /* R12: every level whose step starts now, coarsest first */
        for (int k = o->p.n_levels; k >= 1; --k)
            if (t % ((int64_t)1 << k) == 0) level_step(o, k);
        double X, Y;
        lamina_pos(o, t, &X, &Y);
        double cx = o->p.xc + X, cy = o->p.yc + Y;
        if (t > 0) {
            refill(o, o->Xprev, o->Yprev, X, Y);
            classify(o, cx, cy, o->cls_cur);
        }
        structured_step(o, cx, cy);
        feed_snapshots(o, cx, cy);
        fv_substeps(o, t);
        o->cur = 1 - o->cur;
        memcpy(o->cls_prev, o->cls_cur, o->N);
        o->Xprev = X;
        o->Yprev = Y;
        o->t = t + 1;
        record_force(o);
        /* R12: restriction onto every level that level k has caught up with
         * (finest first), then the rings of the levels that just stepped */
        for (int k = 0; k < o->p.n_levels; ++k)
            if (o->t % ((int64_t)1 << (k + 1)) == 0) {
                restrict_level(o, k, 1 - o->lv[k].cur);
                o->lv[k].cur = 1 - o->lv[k].cur;
            }
        for (int k = 0; k < o->p.n_levels; ++k)
            if (o->t % ((int64_t)1 << k) == 0) fill_ring(o, k, o->t >> k);
    }
    return o->status;
}

void orc_motion_history(const orc_t* o, int64_t count, double* y, double* v) {
    for (int64_t t = 0; t < count; ++t) {
        double X, Y, U = 0.0, V = 0.0;
        lamina_pos(o, t, &X, &Y);
        if (o->p.motion == ORC_MOTION_INDUCED)
            V = o->Vh[t];
        else
            motion_vel(&o->p, (double)t, &U, &V);
        y[t] = Y;
        v[t] = V;
    }
}

/* geometry only, for any time t >= 1 without advancing the run: the node
 * classes of step t and the refill types and donors of the relocation
 * t-1 -> t (Sec. 4) */
void orc_classify_at(orc_t* o, int64_t t, int8_t* cls) {
    double X, Y;
    lamina_pos(o, t, &X, &Y);
    classify(o, o->p.xc + X, o->p.yc + Y, cls);
}

void orc_relocate_at(const orc_t* o, int64_t t, int32_t* type, int32_t* donor) {
    double X0, Y0, X1, Y1;
    lamina_pos(o, t - 1, &X0, &Y0);
    lamina_pos(o, t, &X1, &Y1);
    double dX = X1 - X0, dY = Y1 - Y0;
    double cx = o->p.xc + X1, cy = o->p.yc + Y1;
    double a = 0.5 * o->p.L, b = 0.5 * o->p.T;
    for (int P = 0; P < o->p.n_nodes; ++P) {
        if (o->kind[P] == ORC_KIND_WALL) {
            type[P] = 0;
            donor[P] = -1;
            continue;
        }
        double qx = o->xy[2 * P] + dX, qy = o->xy[2 * P + 1] + dY;
        double lam[3];
        int k = locate(o, qx, qy, lam);
        if (k >= 0) {
            type[P] = 3;
            donor[P] = k;
        } else if (fabs(qx) <= a && fabs(qy) <= b) {
            type[P] = 2;
            donor[P] = -1;
        } else {
            double wx = cx + o->xy[2 * P], wy = cy + o->xy[2 * P + 1];
            type[P] = 1;
            donor[P] = (int)floor(wy) * o->p.nx + (int)floor(wx);
        }
    }
}

int orc_status(const orc_t* o) { return o->status; }
int64_t orc_time(const orc_t* o) { return o->t; }

void orc_struct_f(const orc_t* o, double* f9) {
    memcpy(f9, o->fs[o->cur], (size_t)o->N * 9 * sizeof(double));
}

void orc_struct_macro(const orc_t* o, double* rho, double* ux, double* uy) {
    for (int64_t s = 0; s < o->N; ++s) {
        double f[9];
        for (int i = 0; i < 9; ++i) f[i] = o->fs[o->cur][i * o->N + s];
        moments(f, rho + s, ux + s, uy + s);
    }
}

void orc_struct_class(const orc_t* o, int8_t* cls) { memcpy(cls, o->cls_cur, o->N); }

void orc_patch_f(const orc_t* o, double* f9) {
    memcpy(f9, o->fu[o->ucur], (size_t)o->p.n_nodes * 9 * sizeof(double));
}

void orc_patch_macro(const orc_t* o, double* rho, double* ux, double* uy) {
    for (int P = 0; P < o->p.n_nodes; ++P) moments(o->fu[o->ucur] + 9 * P, rho + P, ux + P, uy + P);
}

void orc_refill_record(const orc_t* o, int32_t* type, int32_t* donor) {
    memcpy(type, o->rtype, o->p.n_nodes * sizeof(int32_t));
    memcpy(donor, o->rdonor, o->p.n_nodes * sizeof(int32_t));
}

void orc_force(const orc_t* o, double* fx, double* fy) {
    memcpy(fx, o->Fx, (size_t)(o->t + 1) * sizeof(double));
    memcpy(fy, o->Fy, (size_t)(o->t + 1) * sizeof(double));
}

int orc_fv_nnz(const orc_t* o) { return o->row_ptr[o->p.n_nodes]; }

void orc_fv_coeffs(const orc_t* o, int32_t* row_ptr, int32_t* col, double* gx, double* gy, double* cc,
                   double* vol) {
    int n = o->p.n_nodes, nnz = o->row_ptr[n];
    memcpy(row_ptr, o->row_ptr, (n + 1) * sizeof(int32_t));
    memcpy(col, o->col, nnz * sizeof(int32_t));
    memcpy(gx, o->gx, nnz * sizeof(double));
    memcpy(gy, o->gy, nnz * sizeof(double));
    memcpy(cc, o->cc, nnz * sizeof(double));
    memcpy(vol, o->vol, n * sizeof(double));
}

void orc_destroy(orc_t* o) {
    if (!o) return;
    free(o->xy);
    free(o->tri);
    free(o->kind);
    free(o->fs[0]);
    free(o->fs[1]);
    free(o->fpost);
    free(o->cls_prev);
    free(o->cls_cur);
    free(o->fu[0]);
    free(o->fu[1]);
    free(o->feq_u);
    free(o->row_ptr);
    free(o->col);
    free(o->gx);
    free(o->gy);
    free(o->cc);
    free(o->vol);
    free(o->seg_a);
    free(o->seg_b);
    free(o->seg_nx);
    free(o->seg_ny);
    free(o->bstart);
    free(o->bitems);
    free(o->Yh);
    free(o->Vh);
    for (int k = 0; k < o->p.n_levels; ++k) {
        free(o->lv[k].f[0]);
        free(o->lv[k].f[1]);
    }
    free(o->snap0);
    free(o->snap1);
    free(o->dstar);
    free(o->rtype);
    free(o->rdonor);
    free(o->Fx);
    free(o->Fy);
    free(o);
}
