/*
 * lbm_oracle.c -- plain FP64 CPU oracle of the B-TriRT melting solver.
 *
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.h).  Scalar loops, one cell at a
 * time, in the order the method states its steps.  Built with
 * -O2 -ffp-contract=off -fno-fast-math so that every operation is the FP64
 * operation written here.  OpenMP only splits the cell loop; every sum over
 * cells is taken afterwards in a fixed serial order, so the result does not
 * depend on the thread count.
 *
 * Paper passages followed (Zhao, Wu, Chai, Shi):
 *   Sec. 2, Eq. 1   H = C_p T + f_l L (total enthalpy)
 *   Sec. 2, Eq. 2   B-TriRT evolution with k0, k1, k2 and M1^neq, M2^neq
 *   Sec. 2, Eq. 4   g_eq; D2Q9 weights 4/9, 1/9, 1/36
 *   Sec. 2, Eq. 5   1/k1 = alpha/(c_s^2 dt) + 1/2
 *   Sec. 2, Eq. 6   k1 + k2 = 2
 *   Sec. 3.1, Eqs. 7-8  Neumann solution of one-phase melting
 *   Sec. 3.2        cavity heated locally from below, no-slip adiabatic walls
 * Readings adopted where the paper is silent are marked "reading".
 */
#include "lbm_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* Physical constants of the nondimensional problem (reading: C_p = rho0 = 1,
 * T_m = 0, T_h = 1, so dT = 1). */
static const double CP = 1.0;
static const double RHO0 = 1.0;
static const double TM = 0.0;
static const double TH = 1.0;

/* D2Q9 lattice: velocities, weights (Sec. 2, after Eq. 4) and opposites. */
static const int CX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int CY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const double W[9] = {4.0 / 9.0,  1.0 / 9.0,  1.0 / 9.0,
                            1.0 / 9.0,  1.0 / 9.0,  1.0 / 36.0,
                            1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
/* c_s^2 = c^2/3 with c = dx/dt = 1 (reading: the paper does not state it). */
static const double CS2 = 1.0 / 3.0;

struct orc_state {
    int nx, ny;
    orc_params p;
    orc_derived d;
    double *f, *g;        /* post-collision populations of the current step */
    double *fn, *gn;      /* next step, written by orc_step                  */
    double *H, *T, *fl, *ux, *uy, *rho; /* fields of the current step        */
    double *qcell;        /* per-cell heated-wall inflow of the current step */
    long long step;
    double Q_last, Q_cum;
    int fields_valid;
    int nthreads;
};

void orc_lattice(int cx[9], int cy[9], double w[9], int opp[9])
{
    for (int i = 0; i < 9; ++i) {
        cx[i] = CX[i];
        cy[i] = CY[i];
        w[i] = W[i];
        opp[i] = OPP[i];
    }
}

/* SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014; Vigna's
 * public-domain reference): add the golden-ratio increment, then two
 * xor-shift-multiply rounds and a final xor-shift. */
uint64_t orc_splitmix64(uint64_t v)
{
    uint64_t z = v + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* H -> (T, f_l) for a pure substance with one C_p (Eq. 1: H = C_p T + f_l L).
 * H_s = C_p T_m is the enthalpy of solid at T_m, H_l = H_s + L of liquid. */
void orc_invert(double H, double Lh, double *T, double *fl)
{
    const double Hs = CP * TM;
    const double Hl = Hs + Lh;
    if (H <= Hs) {
        *T = H / CP;
        *fl = 0.0;
    } else if (H >= Hl) {
        *T = TM + (H - Hl) / CP;
        *fl = 1.0;
    } else {
        *T = TM;
        *fl = (H - Hs) / Lh;
    }
}

/* Enthalpy equilibrium, Eq. 4. */
void orc_geq(double H, double T, double ux, double uy, double out[9])
{
    for (int i = 0; i < 9; ++i) {
        if (i == 0) {
            out[0] = H - CP * T + W[0] * CP * T;
        } else {
            const double cu = CX[i] * ux + CY[i] * uy;
            out[i] = W[i] * CP * T * (1.0 + cu / CS2);
        }
    }
}

/* First and second moments of a non-equilibrium part n (after Eq. 2):
 * M1 = sum_j c_j n_j, M2 = sum_j c_j c_j n_j (symmetric: xx, xy, yy). */
static void neq_moments(const double n[9], double M1[2], double M2[3])
{
    M1[0] = M1[1] = 0.0;
    M2[0] = M2[1] = M2[2] = 0.0;
    for (int j = 0; j < 9; ++j) {
        M1[0] += CX[j] * n[j];
        M1[1] += CY[j] * n[j];
        M2[0] += CX[j] * CX[j] * n[j];
        M2[1] += CX[j] * CY[j] * n[j];
        M2[2] += CY[j] * CY[j] * n[j];
    }
}

/* (c_i c_i - c_s^2 I) : X for a symmetric 2x2 tensor X = (xx, xy, yy). */
static double q_contract(int i, const double X[3])
{
    return (CX[i] * CX[i] - CS2) * X[0] + 2.0 * CX[i] * CY[i] * X[1] +
           (CY[i] * CY[i] - CS2) * X[2];
}

/* The block collision operator of Eq. 2 applied to populations p with
 * equilibrium peq: returns p_i - k0 n_i - (k1-k0) w_i c_i.M1/c_s^2
 *                           - (k2-k0) w_i (c_i c_i - c_s^2 I):M2 / (2 c_s^4). */
static void btrirt(const double p[9], const double peq[9], double k0, double k1,
                   double k2, double out[9])
{
    double n[9], M1[2], M2[3];
    for (int i = 0; i < 9; ++i) n[i] = p[i] - peq[i];
    neq_moments(n, M1, M2);
    for (int i = 0; i < 9; ++i) {
        const double cM1 = CX[i] * M1[0] + CY[i] * M1[1];
        out[i] = p[i] - k0 * n[i] - (k1 - k0) * W[i] * cM1 / CS2 -
                 (k2 - k0) * W[i] * q_contract(i, M2) / (2.0 * CS2 * CS2);
    }
}

/* Eq. 2 with the equilibrium of Eq. 4: the enthalpy (g) collision. */
void orc_g_collide(const double g[9], double H, double T, double ux, double uy,
                   double k0, double k1, double k2, double out[9])
{
    double geq[9];
    orc_geq(H, T, ux, uy, geq);
    btrirt(g, geq, k0, k1, k2, out);
}

/* Second-order D2Q9 flow equilibrium (reading: the paper cites its flow
 * model without writing it down). */
void orc_feq(double rho, double ux, double uy, double out[9])
{
    const double uu = ux * ux + uy * uy;
    for (int i = 0; i < 9; ++i) {
        const double cu = CX[i] * ux + CY[i] * uy;
        out[i] = W[i] * rho *
                 (1.0 + cu / CS2 + cu * cu / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Flow collision (reading): the same block operator as Eq. 2 with rates
 * (k0f, k1f, k2f), plus a body-force source whose first moment is
 * (1 - k1f/2) F and whose second moment is (1 - k2f/2)(uF + Fu).  With
 * k0f = k1f = k2f this is BGK with Guo's forcing. */
void orc_f_collide(const double f[9], double rho, double ux, double uy,
                   double Fx, double Fy, double k0f, double k1f, double k2f,
                   double out[9])
{
    double feq[9];
    orc_feq(rho, ux, uy, feq);
    btrirt(f, feq, k0f, k1f, k2f, out);
    const double uF[3] = {2.0 * ux * Fx, ux * Fy + uy * Fx, 2.0 * uy * Fy};
    for (int i = 0; i < 9; ++i) {
        const double cF = CX[i] * Fx + CY[i] * Fy;
        out[i] += W[i] * ((1.0 - 0.5 * k1f) * cF / CS2 +
                          (1.0 - 0.5 * k2f) * q_contract(i, uF) / (2.0 * CS2 * CS2));
    }
}

/* Root of Eq. 8, Ste / (exp(l^2) erf(l)) = l sqrt(pi), by bisection.
 * The left side minus the right side decreases strictly in l > 0. */
double orc_stefan_lambda(double Ste)
{
    if (!(Ste > 0.0)) return NAN;
    const double sqpi = sqrt(3.14159265358979323846);
    double lo = 0.0, hi = 1.0;
    /* F(l) = l sqrt(pi) exp(l^2) erf(l) - Ste increases from -Ste at 0. */
    while (hi * sqpi * exp(hi * hi) * erf(hi) < Ste) hi *= 2.0;
    for (int it = 0; it < 200; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (mid * sqpi * exp(mid * mid) * erf(mid) < Ste)
            lo = mid;
        else
            hi = mid;
        if (hi - lo <= 0.0) break;
    }
    return 0.5 * (lo + hi);
}

/* Temperature of the Neumann solution, Eq. 7; the front is X = 2 l sqrt(a t). */
double orc_neumann_T(double x, double t, double alpha, double lambda, double Th,
                     double Tm)
{
    const double X = 2.0 * lambda * sqrt(alpha * t);
    if (x < X) return Th - (Th - Tm) * erf(x / (2.0 * sqrt(alpha * t))) / erf(lambda);
    return Tm;
}

/* Parameter mapping (reading for the cavity; Eq. 5 for k1, Eq. 6 for k2).
 * Reference length Href = cavity height ny; free-fall velocity U = Ma c_s;
 * nu = U Href sqrt(Pr/Ra), alpha = nu/Pr, g beta = U^2/(dT Href), so that
 * Ra = g beta dT Href^3/(nu alpha) and Pr = nu/alpha.  alpha_override > 0 sets
 * alpha directly (nu = Pr alpha, g beta from Ra). */
int orc_derive(int nx, int ny, const orc_params *p, orc_derived *d)
{
    if (nx < 2 || ny < 2 || !p || !d) return ORC_ERR_ARG;
    if (p->problem != ORC_CAVITY && p->problem != ORC_STEFAN) return ORC_ERR_ARG;
    memset(d, 0, sizeof(*d));
    const double dT = TH - TM;
    d->cs2 = CS2;
    d->Href = (p->problem == ORC_CAVITY) ? (double)ny : (double)nx;
    if (!(p->Ste > 0.0)) return ORC_ERR_ARG;
    if (p->alpha_override < 0.0 || p->alpha_override != p->alpha_override) return ORC_ERR_ARG;
    if (p->alpha_override > 0.0) {
        d->alpha = p->alpha_override;
        d->nu = (p->Pr > 0.0 ? p->Pr : 1.0) * d->alpha;
        d->gbeta = (p->Ra > 0.0)
                       ? p->Ra * d->nu * d->alpha / (dT * d->Href * d->Href * d->Href)
                       : 0.0;
    } else {
        if (!(p->Ra > 0.0) || !(p->Pr > 0.0) || !(p->Ma > 0.0)) return ORC_ERR_ARG;
        const double U = p->Ma * sqrt(CS2);
        d->nu = U * d->Href * sqrt(p->Pr / p->Ra);
        d->alpha = d->nu / p->Pr;
        d->gbeta = U * U / (dT * d->Href);
    }
    /* Eq. 5 with dt = 1. */
    d->k1 = 1.0 / (d->alpha / CS2 + 0.5);
    d->k0 = p->k0;
    d->k2 = (p->k2 < 0.0) ? 2.0 - d->k1 : p->k2; /* Eq. 6 on request */
    d->k0f = p->k0f;
    d->k1f = p->k1f;
    d->k2f = 1.0 / (d->nu / CS2 + 0.5);
    d->Lh = CP * dT / p->Ste;
    if (p->problem == ORC_CAVITY) {
        d->a = nx * (p->strip_center - 0.5 * p->strip_width);
        d->b = nx * (p->strip_center + 0.5 * p->strip_width);
        d->heated_len = d->b - d->a;
    } else {
        d->a = 0.0;
        d->b = 0.0;
        d->heated_len = (double)ny;
    }
    /* Every rate must lie in (0, 2). */
    const double ks[3] = {d->k0, d->k1, d->k2};
    for (int i = 0; i < 3; ++i)
        if (!(ks[i] > 0.0 && ks[i] < 2.0)) return ORC_ERR_ARG;
    if (p->flow_on) {
        const double kf[3] = {d->k0f, d->k1f, d->k2f};
        for (int i = 0; i < 3; ++i)
            if (!(kf[i] > 0.0 && kf[i] < 2.0)) return ORC_ERR_ARG;
    }
    if (p->problem == ORC_CAVITY &&
        !(p->strip_width >= 0.0 && p->strip_center >= 0.0 && p->strip_center <= 1.0))
        return ORC_ERR_ARG;
    return ORC_OK;
}

static size_t plane(const orc_state *s) { return (size_t)s->nx * (size_t)s->ny; }

/* Does the population of direction i arriving at (x, y) from the outside
 * source (sx, sy) cross a heated (Dirichlet T_h) wall?  Reading: cavity, the
 * bottom wall is heated on [a, b] (closed), the crossing abscissa being
 * x + 1/2 - c_ix/2; a corner crossing takes the bottom-wall rule.  Stefan: the
 * left wall x = 0 is heated (Sec. 3.1).  A cavity strip of width 0 heats
 * nothing. */
static int heated_crossing(const orc_state *s, int x, int i, int sx, int sy)
{
    if (s->p.problem == ORC_STEFAN) return sx < 0;
    if (!(s->p.strip_width > 0.0)) return 0; /* width 0: closed adiabatic box */
    if (sy >= 0) return 0;
    const double xc = x + 0.5 - 0.5 * CX[i];
    return s->d.a <= xc && xc <= s->d.b;
}

int orc_cell_update(const orc_state *s, const double *fprev, const double *gprev,
                    int x, int y, double f_out[9], double g_out[9],
                    double macro[6], double *q)
{
    if (!s || !gprev || x < 0 || y < 0 || x >= s->nx || y >= s->ny) return ORC_ERR_ARG;
    const int nx = s->nx, ny = s->ny;
    const size_t P = plane(s);
    const int flow = s->p.flow_on && fprev;
    double f[9], g[9];
    double qin = 0.0;

    /* Step 1: pull streaming with the wall rules (reading: half-way
     * bounce-back for f and for g on adiabatic walls, half-way anti-bounce-back
     * for g on a wall held at T_h). */
    for (int i = 0; i < 9; ++i) {
        int sx = x - CX[i];
        int sy = y - CY[i];
        if (s->p.problem == ORC_STEFAN) sy = ((sy % ny) + ny) % ny; /* periodic y */
        const int inside = sx >= 0 && sx < nx && sy >= 0 && sy < ny;
        if (inside) {
            const size_t k = (size_t)i * P + (size_t)sy * nx + sx;
            if (flow) f[i] = fprev[k];
            g[i] = gprev[k];
        } else {
            const size_t ko = (size_t)OPP[i] * P + (size_t)y * nx + x;
            if (flow) f[i] = fprev[ko];
            if (heated_crossing(s, x, i, sx, sy)) {
                g[i] = -gprev[ko] + 2.0 * W[i] * CP * TH;
                qin += 2.0 * W[i] * CP * TH - 2.0 * gprev[ko];
            } else {
                g[i] = gprev[ko];
            }
        }
    }

    /* Step 2: flow moments. */
    double rho = RHO0, jx = 0.0, jy = 0.0;
    if (flow) {
        rho = 0.0;
        for (int i = 0; i < 9; ++i) {
            rho += f[i];
            jx += CX[i] * f[i];
            jy += CY[i] * f[i];
        }
    }

    /* Step 3: enthalpy and its inversion (Eq. 1). */
    double H = 0.0;
    for (int i = 0; i < 9; ++i) H += g[i];
    double T, fl;
    orc_invert(H, s->d.Lh, &T, &fl);

    /* Step 4: Boussinesq force and solid treatment (reading):
     * F = rho0 g beta (T - T_m) y-hat, u* = (j + F/2)/rho, u = f_l u*. */
    double ux = 0.0, uy = 0.0, Fx = 0.0, Fy = 0.0;
    if (flow) {
        Fy = RHO0 * s->d.gbeta * (T - TM);
        ux = fl * (jx + 0.5 * Fx) / rho;
        uy = fl * (jy + 0.5 * Fy) / rho;
    }

    /* Step 5: enthalpy collision, Eq. 2 with Eq. 4. */
    orc_g_collide(g, H, T, ux, uy, s->d.k0, s->d.k1, s->d.k2, g_out);

    /* Step 6: flow collision with forcing (reading). */
    if (flow) {
        orc_f_collide(f, rho, ux, uy, Fx, Fy, s->d.k0f, s->d.k1f, s->d.k2f, f_out);
    } else if (f_out) {
        for (int i = 0; i < 9; ++i) f_out[i] = fprev ? fprev[(size_t)i * P + (size_t)y * nx + x] : W[i];
    }

    if (macro) {
        macro[0] = H;
        macro[1] = T;
        macro[2] = fl;
        macro[3] = ux;
        macro[4] = uy;
        macro[5] = rho;
    }
    if (q) *q = qin;
    return ORC_OK;
}

int orc_create(int nx, int ny, const orc_params *p, orc_state **out)
{
    if (!out) return ORC_ERR_ARG;
    *out = NULL;
    orc_derived d;
    int rc = orc_derive(nx, ny, p, &d);
    if (rc) return rc;
    orc_state *s = (orc_state *)calloc(1, sizeof(orc_state));
    if (!s) return ORC_ERR_OOM;
    s->nx = nx;
    s->ny = ny;
    s->p = *p;
    s->d = d;
    s->nthreads = 1;
    const size_t P = plane(s);
    s->f = (double *)calloc(9 * P, sizeof(double));
    s->g = (double *)calloc(9 * P, sizeof(double));
    s->fn = (double *)calloc(9 * P, sizeof(double));
    s->gn = (double *)calloc(9 * P, sizeof(double));
    s->H = (double *)calloc(P, sizeof(double));
    s->T = (double *)calloc(P, sizeof(double));
    s->fl = (double *)calloc(P, sizeof(double));
    s->ux = (double *)calloc(P, sizeof(double));
    s->uy = (double *)calloc(P, sizeof(double));
    s->rho = (double *)calloc(P, sizeof(double));
    s->qcell = (double *)calloc(P, sizeof(double));
    if (!s->f || !s->g || !s->fn || !s->gn || !s->H || !s->T || !s->fl || !s->ux ||
        !s->uy || !s->rho || !s->qcell) {
        orc_destroy(s);
        return ORC_ERR_OOM;
    }
    /* Initial state (reading of "solid at T_m with a seeded +-amp perturbation
     * of T"): delta = amp (2r - 1), r = (splitmix64(seed xor cell) >> 11) 2^-53,
     * H0 = C_p (T_m + delta); f_i = w_i (rho = 1, u = 0); g_i = g_eq(H0). */
    for (int y = 0; y < ny; ++y) {
        for (int x = 0; x < nx; ++x) {
            const uint64_t cell = (uint64_t)y * (uint64_t)nx + (uint64_t)x;
            const double r = (double)(orc_splitmix64(p->seed ^ cell) >> 11) *
                             (1.0 / 9007199254740992.0);
            const double delta = p->init_amp * (2.0 * r - 1.0);
            const double H0 = CP * (TM + delta);
            double T0, fl0, geq[9];
            orc_invert(H0, d.Lh, &T0, &fl0);
            orc_geq(H0, T0, 0.0, 0.0, geq);
            const size_t c = (size_t)y * nx + x;
            for (int i = 0; i < 9; ++i) {
                s->f[(size_t)i * P + c] = W[i];
                s->g[(size_t)i * P + c] = geq[i];
            }
            s->H[c] = H0;
            s->T[c] = T0;
            s->fl[c] = fl0;
            s->ux[c] = 0.0;
            s->uy[c] = 0.0;
            s->rho[c] = 1.0;
        }
    }
    s->step = 0;
    s->Q_last = 0.0;
    s->Q_cum = 0.0;
    s->fields_valid = 1;
    *out = s;
    return ORC_OK;
}

void orc_destroy(orc_state *s)
{
    if (!s) return;
    free(s->f);
    free(s->g);
    free(s->fn);
    free(s->gn);
    free(s->H);
    free(s->T);
    free(s->fl);
    free(s->ux);
    free(s->uy);
    free(s->rho);
    free(s->qcell);
    free(s);
}

int orc_set_threads(orc_state *s, int nthreads)
{
    if (!s || nthreads < 1) return ORC_ERR_ARG;
    s->nthreads = nthreads;
    return ORC_OK;
}

int orc_step(orc_state *s, long long n)
{
    if (!s || n < 0) return ORC_ERR_ARG;
    const int nx = s->nx, ny = s->ny;
    const size_t P = plane(s);
    for (long long it = 0; it < n; ++it) {
        const long long ncell = (long long)P;
#pragma omp parallel for schedule(static) num_threads(s->nthreads)
        for (long long c = 0; c < ncell; ++c) {
            const int y = (int)(c / nx), x = (int)(c % nx);
            double fo[9], go[9], m[6], q;
            orc_cell_update(s, s->f, s->g, x, y, fo, go, m, &q);
            for (int i = 0; i < 9; ++i) {
                s->fn[(size_t)i * P + c] = fo[i];
                s->gn[(size_t)i * P + c] = go[i];
            }
            s->H[c] = m[0];
            s->T[c] = m[1];
            s->fl[c] = m[2];
            s->ux[c] = m[3];
            s->uy[c] = m[4];
            s->rho[c] = m[5];
            s->qcell[c] = q;
        }
        double Q = 0.0;
        for (size_t c = 0; c < P; ++c) Q += s->qcell[c];
        double *t;
        t = s->f; s->f = s->fn; s->fn = t;
        t = s->g; s->g = s->gn; s->gn = t;
        s->Q_last = Q;
        s->Q_cum += Q;
        s->step += 1;
        s->fields_valid = 1;
    }
    (void)ny;
    return ORC_OK;
}

int orc_fields(const orc_state *s, double *H, double *T, double *fl, double *ux,
               double *uy, double *rho)
{
    if (!s) return ORC_ERR_ARG;
    if (!s->fields_valid) return ORC_ERR_STATE;
    const size_t P = plane(s);
    if (H) memcpy(H, s->H, P * sizeof(double));
    if (T) memcpy(T, s->T, P * sizeof(double));
    if (fl) memcpy(fl, s->fl, P * sizeof(double));
    if (ux) memcpy(ux, s->ux, P * sizeof(double));
    if (uy) memcpy(uy, s->uy, P * sizeof(double));
    if (rho) memcpy(rho, s->rho, P * sizeof(double));
    return ORC_OK;
}

/* Diagnostics of the current step (reading: the paper plots f_l(t) only;
 * Nu is defined from the exact heated-wall inflow). */
int orc_diagnostics(const orc_state *s, orc_diag *o)
{
    if (!s || !o) return ORC_ERR_ARG;
    if (!s->fields_valid) return ORC_ERR_STATE;
    const size_t P = plane(s);
    double sum_fl = 0.0, sum_H = 0.0, umax = 0.0;
    int bad = 0;
    for (size_t c = 0; c < P; ++c) {
        sum_fl += s->fl[c];
        sum_H += s->H[c];
        const double um = sqrt(s->ux[c] * s->ux[c] + s->uy[c] * s->uy[c]);
        if (um > umax) umax = um;
        if (!isfinite(s->H[c]) || !isfinite(s->rho[c])) bad = 1;
    }
    o->step = (double)s->step;
    o->melt_fraction = sum_fl / (double)P;
    o->H_total = sum_H;
    o->Q_strip = s->Q_last;
    o->Q_cum = s->Q_cum;
    o->Nu = (s->d.heated_len > 0.0)
                ? s->Q_last * s->d.Href / (s->d.alpha * RHO0 * CP * (TH - TM) * s->d.heated_len)
                : 0.0;
    o->front_x = sum_fl / (double)s->ny;
    o->max_u = umax;
    o->nan_flag = bad ? 1.0 : 0.0;
    return ORC_OK;
}

int orc_get_derived(const orc_state *s, orc_derived *out)
{
    if (!s || !out) return ORC_ERR_ARG;
    *out = s->d;
    return ORC_OK;
}

int orc_get_populations(const orc_state *s, double *f, double *g)
{
    if (!s) return ORC_ERR_ARG;
    const size_t n = 9 * plane(s);
    if (f) memcpy(f, s->f, n * sizeof(double));
    if (g) memcpy(g, s->g, n * sizeof(double));
    return ORC_OK;
}

int orc_set_populations(orc_state *s, const double *f, const double *g, long long step)
{
    if (!s || !f || !g || step < 0) return ORC_ERR_ARG;
    const size_t n = 9 * plane(s);
    memcpy(s->f, f, n * sizeof(double));
    memcpy(s->g, g, n * sizeof(double));
    s->step = step;
    s->Q_last = 0.0;
    s->Q_cum = 0.0;
    s->fields_valid = 0; /* fields belong to the next step taken */
    return ORC_OK;
}
