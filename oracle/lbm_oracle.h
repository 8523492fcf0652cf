/*
 * lbm_oracle.h -- plain FP64 CPU oracle of the B-TriRT melting solver.
 *
 * TEST INFRASTRUCTURE ONLY.  This is the slow, obviously-correct statement of
 * what the GPU sweep computes, written from the paper (Zhao, Wu, Chai, Shi,
 * "Lattice Boltzmann simulations of melting in a rectangular cavity heated
 * locally from below at high Rayleigh number"):
 *   Eq. 1  total-enthalpy energy equation, H = C_p T + f_l L
 *   Eq. 2  block triple-relaxation-time (B-TriRT) collision
 *   Eq. 4  enthalpy equilibrium g_eq
 *   Eq. 5  k1 from the thermal diffusivity
 *   Eq. 6  the anti-numerical-diffusion rule k1 + k2 = 2
 *   Eqs. 7-8  Neumann solution of one-phase melting (Sec. 3.1)
 * plus the readings adopted where the paper is silent (flow solver, buoyancy,
 * solid treatment, wall schemes, unit mapping), each marked "reading" below.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this library.  It shares no source with the CUDA path: it has its own
 * lattice tables, its own parameter struct and its own random generator.
 *
 * Layout of every population array: plane-major, [i][y][x], i = 0..8,
 * index i*ny*nx + y*nx + x, FP64.  Field arrays: [y][x].
 * All functions return 0 on success, a negative code on error.
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_ERR_ARG = -1, ORC_ERR_OOM = -2, ORC_ERR_STATE = -5 };
enum { ORC_CAVITY = 0, ORC_STEFAN = 1 };

typedef struct {
    int problem;            /* ORC_CAVITY or ORC_STEFAN                          */
    double Ra, Pr, Ste, Ma; /* Rayleigh, Prandtl, Stefan, Mach numbers            */
    double strip_center;    /* C: heated-strip centre, fraction of the width      */
    double strip_width;     /* D: heated-strip width, fraction of the width       */
    double k0, k2;          /* g relaxation rates; k2 < 0 selects k2 = 2 - k1     */
    double alpha_override;  /* > 0: thermal diffusivity in lattice units          */
    double k0f, k1f;        /* flow ghost and first-moment rates                  */
    int flow_on;            /* 0: u = 0 and f is not evolved                      */
    double init_amp;        /* amplitude of the seeded perturbation of T          */
    uint64_t seed;          /* seed of the perturbation                           */
} orc_params;

/* Parameters derived from orc_params (lattice units). */
typedef struct {
    double cs2;            /* lattice sound speed squared, 1/3                   */
    double nu, alpha;      /* kinematic viscosity, thermal diffusivity           */
    double gbeta;          /* g*beta of the Boussinesq force                     */
    double k0, k1, k2;     /* g relaxation rates                                 */
    double k0f, k1f, k2f;  /* f relaxation rates                                 */
    double Lh;             /* latent heat                                        */
    double a, b;           /* heated segment [a, b] along the wall, in cells     */
    double Href;           /* reference length (cavity height / Stefan length)   */
    double heated_len;     /* heated length used by the Nusselt number           */
} orc_derived;

typedef struct {
    double step;           /* steps taken                                        */
    double melt_fraction;  /* sum f_l / (nx ny)                                  */
    double H_total;        /* sum H                                              */
    double Q_strip;        /* enthalpy entering through the heated wall, last step */
    double Q_cum;          /* Q_strip summed over all steps taken                */
    double Nu;             /* Q_strip Href / (alpha dT heated_len)               */
    double front_x;        /* sum f_l / ny                                       */
    double max_u;          /* max |u|                                            */
    double nan_flag;       /* 1 if any H or rho is not finite                    */
} orc_diag;

typedef struct orc_state orc_state;

/* ---- per-cell pieces (exposed so the tests can pin them one by one) ---- */
void orc_lattice(int cx[9], int cy[9], double w[9], int opp[9]);
uint64_t orc_splitmix64(uint64_t v);
void orc_invert(double H, double Lh, double *T, double *fl);
void orc_geq(double H, double T, double ux, double uy, double out[9]);
void orc_g_collide(const double g[9], double H, double T, double ux, double uy,
                   double k0, double k1, double k2, double out[9]);
void orc_feq(double rho, double ux, double uy, double out[9]);
void orc_f_collide(const double f[9], double rho, double ux, double uy,
                   double Fx, double Fy, double k0f, double k1f, double k2f,
                   double out[9]);
double orc_stefan_lambda(double Ste);
double orc_neumann_T(double x, double t, double alpha, double lambda,
                     double Th, double Tm);
int orc_derive(int nx, int ny, const orc_params *p, orc_derived *d);

/* ---- whole lattice ---- */
int orc_create(int nx, int ny, const orc_params *p, orc_state **out);
void orc_destroy(orc_state *s);
int orc_set_threads(orc_state *s, int nthreads);
int orc_step(orc_state *s, long long n);
int orc_fields(const orc_state *s, double *H, double *T, double *fl,
               double *ux, double *uy, double *rho);
int orc_diagnostics(const orc_state *s, orc_diag *out);
int orc_get_derived(const orc_state *s, orc_derived *out);
int orc_get_populations(const orc_state *s, double *f, double *g);
int orc_set_populations(orc_state *s, const double *f, const double *g,
                        long long step);
/* One cell of one step, from arbitrary previous post-collision populations
 * fprev/gprev (plane-major, nx*ny per plane) of a lattice with the same sizes
 * and parameters as s.  Writes the cell's new post-collision populations
 * (f_out, g_out), its fields macro = {H, T, fl, ux, uy, rho} and its heated-wall
 * inflow q.  The state s itself is not modified. */
int orc_cell_update(const orc_state *s, const double *fprev, const double *gprev,
                    int x, int y, double f_out[9], double g_out[9],
                    double macro[6], double *q);

#ifdef __cplusplus
}
#endif
#endif
