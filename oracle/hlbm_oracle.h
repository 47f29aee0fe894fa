/* CPU correctness oracle for the moving-grid hybrid lattice Boltzmann method.
 *
 * TEST INFRASTRUCTURE ONLY.  Plain serial FP64 C, written for readability, not
 * speed.  Only the tests, the smoke check and the benchmark's CPU-baseline arm
 * may load it; the product library never does, and the two share no code.
 *
 * Paper: Di Ilio, Chiappini, Ubertini, Bella, Succi, "A moving-grid approach
 * for fluid-structure interaction problems with hybrid lattice Boltzmann
 * method" (Sec. 2 problem statement, Sec. 3 HLBM, Sec. 4 refill procedure,
 * Sec. 5 numerical setup).  Readings of passages the paper leaves open are
 * listed in the repository's design notes and restated beside the code.
 */
#ifndef HLBM_ORACLE_H
#define HLBM_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_BC_WALL = 0, ORC_BC_OUTFLOW = 1, ORC_BC_PERIODIC = 2 };
enum { ORC_MOTION_STATIC = 0, ORC_MOTION_HARMONIC = 1, ORC_MOTION_UNIFORM = 2, ORC_MOTION_INDUCED = 3,
       ORC_MOTION_HARMONIC_X = 4 };
enum { ORC_KIND_INTERIOR = 0, ORC_KIND_OUTER = 1, ORC_KIND_WALL = 2 };
enum { ORC_DISC = 0, ORC_INTERP = 1, ORC_UNUSED = 2 };
enum { ORC_MAX_LEVELS = 4 };
/* status bits */
enum {
    ORC_ERR_FILL_NOT_LOCATED = 1,   /* eq. 178 node outside the patch          */
    ORC_ERR_DONOR_NOT_COMPUTED = 2, /* bilinear donor not a computed node      */
    ORC_ERR_PULL_SOURCE = 4,        /* streaming source is an unused node      */
    ORC_ERR_NONFINITE = 8,          /* NaN / Inf in the force                   */
    ORC_ERR_UNUSED_TO_DISC = 16,    /* node jumped unused -> disc in one step  */
    ORC_ERR_FAST_MOTION = 64        /* INDUCED lamina moved >= 1 per step       */
};

typedef struct {
    int nx, ny, bc_x, bc_y;
    double rho0;
    const double* rho_init; /* [ny*nx] row-major, or NULL for rho0 everywhere */
    double u0x, u0y;        /* initial uniform velocity                        */
    const double* ux_init;  /* [ny*nx] initial velocity field, or NULL for u0   */
    const double* uy_init;
    double tau_s;           /* structured relaxation time                      */
    double L, T, xc, yc;    /* lamina rectangle and its centre at t = 0         */
    double delta_f;         /* fictitious-curve offset                          */
    int n_nodes, n_tris;
    const double* xy;       /* [n_nodes*2] body frame                          */
    const int32_t* tri;     /* [n_tris*3]                                      */
    const int8_t* kind;     /* [n_nodes]                                       */
    int n_sub;              /* FV sub-steps per structured step                 */
    int lumped;             /* 1: C = identity                                  */
    int motion;
    double A, omega, vx, vy;
    int outer_fv;           /* 1: outer nodes take eq. 182 with its FV sums (R10) */
    /* INDUCED motion (R11): m y'' + c y' + k y = F_y, y(0) = y0, y'(0) = v0 */
    double mass, stiffness, damping, y0, v0;
    /* nested lattice levels (R12): n_levels coarser lattices around the
     * nx x ny lattice.  Level k (1..n_levels) has twice the spacing and time
     * step of level k-1, lv_nx[k-1] x lv_ny[k-1] nodes, and holds node (0, 0)
     * of level k-1 at its node (lv_ox[k-1], lv_oy[k-1]); every level inside
     * another has odd sizes.  bc_x, bc_y apply to the coarsest level.  Level
     * k starts at equilibrium with the density lv_rho[k-1] and the velocity
     * lv_ux[k-1], lv_uy[k-1] ([ny*nx] each, or NULL for rho0 and u0). */
    int n_levels;
    int lv_nx[ORC_MAX_LEVELS], lv_ny[ORC_MAX_LEVELS], lv_ox[ORC_MAX_LEVELS], lv_oy[ORC_MAX_LEVELS];
    const double* lv_rho[ORC_MAX_LEVELS];
    const double* lv_ux[ORC_MAX_LEVELS];
    const double* lv_uy[ORC_MAX_LEVELS];
    /* R13: absorbing layer next to the outflow sides of the lattice that
     * carries the domain boundary (the coarsest level): sponge_rows > 0
     * rows deep, strength sponge_sigma at the boundary row (0: none) */
    int sponge_rows;
    double sponge_sigma;
} orc_params_t;

typedef struct orc orc_t;

orc_t* orc_create(const orc_params_t* p);
void orc_destroy(orc_t* o);
int orc_step(orc_t* o, int64_t nsteps);
/* lamina position and velocity at integer times 0..t (+1 for the position:
 * INDUCED motion knows y(t+1) once step t has started) */
void orc_motion_history(const orc_t* o, int64_t count, double* y, double* v);
int orc_status(const orc_t* o);
int64_t orc_time(const orc_t* o);

/* structured fields at the current time (pre-collision state) */
void orc_struct_f(const orc_t* o, double* f9);               /* [9][ny][nx] */
void orc_struct_macro(const orc_t* o, double* rho, double* ux, double* uy);
/* R12: rho, u of level k (1..n_levels) [ny_k*nx_k] at its current time
 * (the fine time rounded down to a multiple of 2^k) */
void orc_level_macro(const orc_t* o, int k, double* rho, double* ux, double* uy);
void orc_struct_class(const orc_t* o, int8_t* cls);          /* class of the last step */
/* patch fields at the current time */
void orc_patch_f(const orc_t* o, double* f9);                /* [n][9] */
void orc_patch_macro(const orc_t* o, double* rho, double* ux, double* uy);
/* refill record of the last relocation: type 0 wall, 1/2/3 as in Sec. 4;
 * donor = triangle (type 3), cell index iy*nx+ix (type 1), else -1 */
void orc_refill_record(const orc_t* o, int32_t* type, int32_t* donor);
/* force history F(t), t = 0 .. current time */
void orc_force(const orc_t* o, double* fx, double* fy);
/* hydrodynamic function from the force history (Sec. 2.1) */
int orc_gamma(const orc_t* o, double discard_periods, double fit_periods,
              double* re, double* im, double* rms);
/* the same from a given history F[0..n-1] of the force along the motion */
int orc_theta(const double* F, int64_t n, double rho0, double omega, double L, double A,
              double discard_periods, double fit_periods, double* re, double* im, double* rms);

/* geometry only (no state change): classes of step t, refill record of t-1 -> t */
void orc_classify_at(orc_t* o, int64_t t, int8_t* cls);
void orc_relocate_at(const orc_t* o, int64_t t, int32_t* type, int32_t* donor);

/* building blocks exposed for the pins */
void orc_feq(double rho, double ux, double uy, double* feq9);
int orc_locate(const orc_t* o, double qx, double qy, double* lam3);
int orc_fv_nnz(const orc_t* o);
void orc_fv_coeffs(const orc_t* o, int32_t* row_ptr, int32_t* col, double* gx, double* gy,
                   double* cc, double* vol);
int orc_n_wall_segments(const orc_t* o);
/* least-squares fit F(t_m) = a sin(w t_m) + b cos(w t_m), t_m = t0..t1 */
void orc_sine_fit(const double* F, int64_t t0, int64_t t1, double omega, double* a, double* b,
                  double* rms);

/* FV-LBM on a doubly periodic triangulated mesh (no wall, no outer nodes):
 * n_iter explicit steps of eq. ulbe with time step dt_u.  f9 is [n][9], in/out. */
int orc_fv_periodic(int n_nodes, const double* xy, int n_tris, const int32_t* tri,
                    double period_x, double period_y, double tau_u, double dt_u, int lumped,
                    int n_iter, double* f9);

/* R10 alone: the full eq. postcollision2_u update of every outer node of a
 * mesh (no periodicity) from the patch state fin and the R2 values dstar
 * (both [n][9]); fout [n][9] receives the outer nodes' new values */
int orc_outer_fv(int n_nodes, const double* xy, int n_tris, const int32_t* tri, const int8_t* kind,
                 double tau_u, double dt_u, int lumped, const double* fin, const double* dstar, double* fout);

/* structured LBGK alone (no patch): n_iter steps of eq. LBE on f9 [9][ny][nx] */
int orc_lbgk(int nx, int ny, int bc_x, int bc_y, double tau_s, int sponge_rows, double sponge_sigma, int n_iter,
             double* f9);

#ifdef __cplusplus
}
#endif
#endif
