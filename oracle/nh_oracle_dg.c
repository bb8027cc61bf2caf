/*
 * nh_oracle_dg.c -- FP64 CPU oracle of the DG-P1 predictor and the LDG
 * correction (the paper's own discretisation, Sec. 3).  TEST INFRASTRUCTURE
 * ONLY; see nh_oracle_dg.h for the layout and the readings taken.
 */
#include "nh_oracle_dg.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ----------------------------------------------------------------- bottom */

/* Positions of the moving parts (the same laws as the finite-volume oracle's
   motions: s0 ln cosh(t/t0) for the mound, the piecewise-quadratic glide of
   the sliding block of Sec. 4.3). */
static void dg_slide_law(const or_dg_params* P, double t, double* s, double* sd, double* sdd)
{
    double z = t / P->t0;
    *s = P->s0 * log(cosh(z));
    *sd = (P->s0 / P->t0) * tanh(z);
    *sdd = (P->s0 / (P->t0 * P->t0)) / (cosh(z) * cosh(z));
}

static void dg_block_law(const or_dg_params* P, double t, double* S, double* Sd, double* Sdd)
{
    double a0 = P->s0, t1 = P->t0, t2 = P->t2, t3 = t2 + t1, ut = a0 * t1;
    double S1 = 0.5 * a0 * t1 * t1;
    if (t <= 0.0) { *S = 0.0; *Sd = 0.0; *Sdd = 0.0; }
    else if (t <= t1) { *S = 0.5 * a0 * t * t; *Sd = a0 * t; *Sdd = a0; }
    else if (t <= t2) { *S = S1 + ut * (t - t1); *Sd = ut; *Sdd = 0.0; }
    else if (t <= t3) {
        *S = S1 + ut * (t - t1) - 0.5 * a0 * (t - t2) * (t - t2);
        *Sd = ut - a0 * (t - t2);
        *Sdd = -a0;
    } else {
        *S = S1 + ut * (t3 - t1) - 0.5 * a0 * (t3 - t2) * (t3 - t2);
        *Sd = 0.0; *Sdd = 0.0;
    }
}

void or_dg_bottom(const or_dg_params* P, double x, double t, double out[6])
{
    double d = P->b0 + P->b1 * (x - P->xl), d_x = P->b1, d_xx = 0.0;
    double d_t = 0.0, d_xt = 0.0, d_tt = 0.0;
    if (P->slide == OR_SLIDE_GAUSS_LNCOSH) {
        double s, sd, sdd;
        dg_slide_law(P, t, &s, &sd, &sdd);
        double L = P->L, xi = (x - P->xc0 - s) / L;
        double m = P->A * exp(-xi * xi);
        d -= m;
        d_x -= m * (-2.0 * xi / L);
        d_xx -= m * (4.0 * xi * xi - 2.0) / (L * L);
        d_t = -m * (2.0 * xi / L) * sd;
        d_xt = m * (2.0 / (L * L)) * (2.0 * xi * xi - 1.0) * sd;
        d_tt = -m * (2.0 / (L * L)) * ((2.0 * xi * xi - 1.0) * sd * sd + xi * L * sdd);
    } else if (P->slide == OR_SLIDE_PLATE_EXP) {
        if (fabs(x - P->xc0) < P->L) {
            double e = exp(-t / P->t0);
            d -= P->A * (1.0 - e);
            d_t = -P->A * e / P->t0;
            d_tt = P->A * e / (P->t0 * P->t0);
        }
    } else if (P->slide == OR_SLIDE_QUARTIC) {
        double S, Sd, Sdd;
        dg_block_law(P, t, &S, &Sd, &Sdd);
        double L = P->L, xi = 2.0 * (x - P->xc0 - S) / L;
        if (fabs(xi) < 1.0) {
            double A = P->A, xi2 = xi * xi, xi3 = xi2 * xi;
            d -= A * (1.0 - xi2 * xi2);
            d_x -= -8.0 * A * xi3 / L;
            d_xx -= -48.0 * A * xi2 / (L * L);
            d_t = -8.0 * A * xi3 * Sd / L;
            d_xt = -48.0 * A * xi2 * Sd / (L * L);
            d_tt = -(8.0 * A / L) * (-6.0 * xi2 * Sd * Sd / L + xi3 * Sdd);
        }
    }
    out[0] = d; out[1] = d_x; out[2] = d_xx; out[3] = d_t; out[4] = d_xt; out[5] = d_tt;
}

static double node_x(const or_dg_params* P, int k)
{
    return P->xl + (k / 2 + (k & 1)) * P->dx;   /* node 2i at xl + i dx, node 2i+1 at xl + (i+1) dx */
}

/* -------------------------------------------------------------- predictor */

/* Hydrostatic flux F(Q) = (hu, hu^2/h + g h^2/2, hu hw / h). */
static void flux(double g, double h, double hu, double hw, double F[3])
{
    double u = hu / h;
    F[0] = hu;
    F[1] = hu * u + 0.5 * g * h * h;
    F[2] = hu * hw / h;
}

/* Rusanov flux between the states QL (left of the interface) and QR
   (Sec. 3.1): the mean of the fluxes minus half the largest wave speed times
   the jump. */
static void rusanov_dg(double g, const double QL[3], const double QR[3], double F[3])
{
    double FL[3], FR[3];
    flux(g, QL[0], QL[1], QL[2], FL);
    flux(g, QR[0], QR[1], QR[2], FR);
    double sL = fabs(QL[1] / QL[0]) + sqrt(g * QL[0]);
    double sR = fabs(QR[1] / QR[0]) + sqrt(g * QR[0]);
    double s = sL > sR ? sL : sR;
    for (int c = 0; c < 3; ++c) F[c] = 0.5 * (FL[c] + FR[c]) - 0.5 * s * (QR[c] - QL[c]);
}

/* Weak form of Sec. 3.1 per element with the P1 nodal basis at the end points:
   M dQ/dt = (volume term) + (interface term) + M S, with
   M = dx/6 [[2,1],[1,2]], volume term_j = sum_k F_k int phi_j' phi_k
   (= -(F_L + F_R)/2 for j = L, +(F_L + F_R)/2 for j = R), interface term
   +F*(left end) for j = L and -F*(right end) for j = R, and the source
   S = (0, g h d_x, 0) interpolated at the nodes.  Walls: the ghost state is
   the node's mirror (h, -hu, hw). */
void or_dg_rhs(const or_dg_params* P, double t, const double* h, const double* hu, const double* hw,
               double* rh, double* rhu, double* rhw)
{
    int ne = P->ne;
    double g = P->g, dx = P->dx;
    double* Fs = malloc(sizeof(double) * 3 * (ne + 1));   /* interface fluxes, interface e at xl + e dx */
    for (int e = 0; e <= ne; ++e) {
        double QL[3], QR[3];
        if (e == 0) {
            int k = 0;
            QR[0] = h[k]; QR[1] = hu[k]; QR[2] = hw[k];
            QL[0] = h[k]; QL[1] = -hu[k]; QL[2] = hw[k];
        } else if (e == ne) {
            int k = 2 * ne - 1;
            QL[0] = h[k]; QL[1] = hu[k]; QL[2] = hw[k];
            QR[0] = h[k]; QR[1] = -hu[k]; QR[2] = hw[k];
        } else {
            int kl = 2 * e - 1, kr = 2 * e;
            QL[0] = h[kl]; QL[1] = hu[kl]; QL[2] = hw[kl];
            QR[0] = h[kr]; QR[1] = hu[kr]; QR[2] = hw[kr];
        }
        rusanov_dg(g, QL, QR, Fs + 3 * e);
    }
    for (int i = 0; i < ne; ++i) {
        int kL = 2 * i, kR = 2 * i + 1;
        double FL[3], FR[3];
        flux(g, h[kL], hu[kL], hw[kL], FL);
        flux(g, h[kR], hu[kR], hw[kR], FR);
        double bL[6], bR[6];
        or_dg_bottom(P, node_x(P, kL), t, bL);
        or_dg_bottom(P, node_x(P, kR), t, bR);
        double rhsL[3], rhsR[3];
        for (int c = 0; c < 3; ++c) {
            rhsL[c] = -0.5 * (FL[c] + FR[c]) + Fs[3 * i + c];
            rhsR[c] = 0.5 * (FL[c] + FR[c]) - Fs[3 * (i + 1) + c];
        }
        /* M^{-1} = (2/dx) [[2, -1], [-1, 2]] */
        double outL[3], outR[3];
        for (int c = 0; c < 3; ++c) {
            outL[c] = (2.0 / dx) * (2.0 * rhsL[c] - rhsR[c]);
            outR[c] = (2.0 / dx) * (-rhsL[c] + 2.0 * rhsR[c]);
        }
        outL[1] += g * h[kL] * bL[1];
        outR[1] += g * h[kR] * bR[1];
        rh[kL] = outL[0]; rhu[kL] = outL[1]; rhw[kL] = outL[2];
        rh[kR] = outR[0]; rhu[kR] = outR[1]; rhw[kR] = outR[2];
    }
    free(Fs);
}

/* Heun: Q* = Q^n + dt H(Q^n, t^n); Q~ = Q^n + dt/2 (H(Q^n, t^n) + H(Q*, t^{n+1})). */
void or_dg_predict(const or_dg_params* P, double t, double dt, const double* h, const double* hu,
                   const double* hw, double* ht, double* hut, double* hwt)
{
    int n = 2 * P->ne;
    double* k1 = malloc(sizeof(double) * 3 * n);
    double* k2 = malloc(sizeof(double) * 3 * n);
    double* qs = malloc(sizeof(double) * 3 * n);
    or_dg_rhs(P, t, h, hu, hw, k1, k1 + n, k1 + 2 * n);
    for (int k = 0; k < n; ++k) {
        qs[k] = h[k] + dt * k1[k];
        qs[n + k] = hu[k] + dt * k1[n + k];
        qs[2 * n + k] = hw[k] + dt * k1[2 * n + k];
    }
    or_dg_rhs(P, t + dt, qs, qs + n, qs + 2 * n, k2, k2 + n, k2 + 2 * n);
    for (int k = 0; k < n; ++k) {
        ht[k] = h[k] + 0.5 * dt * (k1[k] + k2[k]);
        hut[k] = hu[k] + 0.5 * dt * (k1[n + k] + k2[n + k]);
        hwt[k] = hw[k] + 0.5 * dt * (k1[2 * n + k] + k2[2 * n + k]);
    }
    free(k1); free(k2); free(qs);
}

/* ------------------------------------------------------------------- mask */

/* Criterion of Sec. 5.1 on element i: the mean of its two nodal values, the
   P1 slope for the x-derivatives. */
static double dg_criterion(const or_dg_params* P, double t1, const double* ht, const double* hut,
                           const double* hwt, int i)
{
    int kL = 2 * i, kR = 2 * i + 1;
    double bL[6], bR[6];
    or_dg_bottom(P, node_x(P, kL), t1, bL);
    or_dg_bottom(P, node_x(P, kR), t1, bR);
    double etaL = ht[kL] - bL[0], etaR = ht[kR] - bR[0];
    double uL = hut[kL] / ht[kL], uR = hut[kR] / ht[kR];
    double wL = hwt[kL] / ht[kL], wR = hwt[kR] / ht[kR];
    switch (P->crit) {
        case OR_CRIT_ETA_D: return fabs(0.5 * (etaL + etaR) / (0.5 * (bL[0] + bR[0])));
        case OR_CRIT_ETA_X: return fabs((etaR - etaL) / P->dx);
        case OR_CRIT_U: return fabs(0.5 * (uL + uR));
        case OR_CRIT_U_X: return fabs((uR - uL) / P->dx);
        case OR_CRIT_W: return fabs(0.5 * (wL + wR));
        case OR_CRIT_W_X: return fabs((wR - wL) / P->dx);
        default: return 0.0;
    }
}

int or_dg_mask(const or_dg_params* P, double t1, long step, const double* ht, const double* hut,
               const double* hwt, unsigned char* mask)
{
    int ne = P->ne, cnt = 0;
    if (P->crit == OR_CRIT_GLOBAL || (P->first_step_global && step == 0)) {
        for (int i = 0; i < ne; ++i) mask[i] = 1;
        return ne;
    }
    unsigned char* m0 = calloc(ne, 1);
    if (P->crit != OR_CRIT_HYDROSTATIC)
        for (int i = 0; i < ne; ++i) m0[i] = dg_criterion(P, t1, ht, hut, hwt, i) > P->knh;
    for (int i = 0; i < ne; ++i) {
        int on = 0;
        for (int j = i - P->enlarge; j <= i + P->enlarge && !on; ++j)
            if (j >= 0 && j < ne && m0[j]) on = 1;
        mask[i] = (unsigned char)on;
        cnt += on;
    }
    free(m0);
    return cnt;
}

/* -------------------------------------------------------------- assembly */

/* Coefficients of Eqs. 12-13 at node k: s11, s12, f1, s21, s22, f2, and the
   pieces of the correction (Eq. 11): phi, D = 4 + d_x^2, d_x. */
typedef struct {
    double s11, s12, f1, s21, s22, f2, phi, D, d_x;
} node_coef;

static node_coef coef_at(const or_dg_params* P, double t1, double dt, const double* ht, const double* hut,
                         const double* hwt, int i, int k)
{
    int kL = 2 * i, kR = 2 * i + 1;
    double b[6], bL[6], bR[6];
    or_dg_bottom(P, node_x(P, k), t1, b);
    or_dg_bottom(P, node_x(P, kL), t1, bL);
    or_dg_bottom(P, node_x(P, kR), t1, bR);
    double rho = P->rho;
    double h = ht[k], hu = hut[k], hw = hwt[k], u = hu / h;
    double h_x = (ht[kR] - ht[kL]) / P->dx;
    double eta_x = ((ht[kR] - bR[0]) - (ht[kL] - bL[0])) / P->dx;
    double d_x = b[1], d_xx = b[2], d_t = b[3], d_xt = b[4], d_tt = b[5];
    double D = 4.0 + d_x * d_x;
    node_coef c;
    c.phi = rho * h / D * (P->g * d_x * eta_x - d_tt - 2.0 * u * d_xt - u * u * d_xx);   /* Eq. 5 */
    c.s11 = (2.0 * h_x - 3.0 * d_x) / (2.0 * h);                                          /* Eq. 12 */
    c.s12 = rho * D / (4.0 * dt * h);
    c.f1 = D / (4.0 * h) * (c.phi * d_x + rho / dt * hu);
    c.s21 = (3.0 * d_x - 2.0 * h_x) / (2.0 * h);                                          /* Eq. 13 */
    c.s22 = 3.0 * dt / (rho * h);
    c.f2 = -2.0 * d_t - 2.0 * hw / h - d_x * hu / (2.0 * h) - dt * D * c.phi / (2.0 * rho * h);
    c.D = D;
    c.d_x = d_x;
    return c;
}

/* The LDG weak forms of Eqs. 12-13 on element i, tested with phi_L and phi_R
   (the same nodal P1 representation of the products s p, s hu and of f):
     Eq. 12_j: [p* phi_j] - int p phi_j' + int (s11 p + s12 hu) phi_j = int f1 phi_j
     Eq. 13_j: [hu* phi_j] - int hu phi_j' + int (s21 hu + s22 p) phi_j = int f2 phi_j
   with int p phi_L' = -(p_L + p_R)/2, int p phi_R' = (p_L + p_R)/2 and the
   mass matrix dx/6 [[2,1],[1,2]] for the rest.  Fluxes (Eqs. 14-15,
   flip-flop): between marked elements p* = p+ and hu* = hu- + c11 (p- - p+);
   at a sub-domain edge or a wall p* = 0 and the outside hu is the predicted
   one (0 at a wall), p outside = 0. */
void or_dg_assemble(const or_dg_params* P, double t1, double dt, const double* ht, const double* hut,
                    const double* hwt, const unsigned char* mask, double* blk, double* rhs)
{
    int ne = P->ne;
    double dx = P->dx, c11 = P->c11;
    memset(blk, 0, sizeof(double) * 48 * ne);
    memset(rhs, 0, sizeof(double) * 4 * ne);
    enum { PL = 0, PR = 1, UL = 2, UR = 3 };
    for (int i = 0; i < ne; ++i) {
        double* Lb = blk + 48 * i;        /* couplings to element i-1 */
        double* Db = Lb + 16;             /* to itself */
        double* Ub = Lb + 32;             /* to element i+1 */
        double* r = rhs + 4 * i;
        if (!mask[i]) {
            Db[0 * 4 + PL] = 1.0; Db[1 * 4 + PR] = 1.0; Db[2 * 4 + UL] = 1.0; Db[3 * 4 + UR] = 1.0;
            r[2] = hut[2 * i]; r[3] = hut[2 * i + 1];
            continue;
        }
        node_coef cL = coef_at(P, t1, dt, ht, hut, hwt, i, 2 * i);
        node_coef cR = coef_at(P, t1, dt, ht, hut, hwt, i, 2 * i + 1);
        int mlft = (i > 0 && mask[i - 1]), mrgt = (i < ne - 1 && mask[i + 1]);
        double m6 = dx / 6.0;
        /* row 0: Eq. 12 tested with phi_L:  -p*(left) + (p_L + p_R)/2 + mass terms = int f1 phi_L */
        if (mlft) Db[0 * 4 + PL] += -1.0;          /* p*(left) = p_L of this element */
        /* else p*(left) = 0 */
        Db[0 * 4 + PL] += 0.5; Db[0 * 4 + PR] += 0.5;
        Db[0 * 4 + PL] += m6 * 2.0 * cL.s11; Db[0 * 4 + PR] += m6 * cR.s11;
        Db[0 * 4 + UL] += m6 * 2.0 * cL.s12; Db[0 * 4 + UR] += m6 * cR.s12;
        r[0] = m6 * (2.0 * cL.f1 + cR.f1);
        /* row 1: Eq. 12 tested with phi_R:  +p*(right) - (p_L + p_R)/2 + mass terms = int f1 phi_R */
        if (mrgt) Ub[1 * 4 + PL] += 1.0;           /* p*(right) = p_L of element i+1 */
        Db[1 * 4 + PL] += -0.5; Db[1 * 4 + PR] += -0.5;
        Db[1 * 4 + PL] += m6 * cL.s11; Db[1 * 4 + PR] += m6 * 2.0 * cR.s11;
        Db[1 * 4 + UL] += m6 * cL.s12; Db[1 * 4 + UR] += m6 * 2.0 * cR.s12;
        r[1] = m6 * (cL.f1 + 2.0 * cR.f1);
        /* row 2: Eq. 13 tested with phi_L:  -hu*(left) + (hu_L + hu_R)/2 + mass terms = int f2 phi_L,
           hu*(left) = hu- + c11 (p- - p_L) */
        if (mlft) {
            Lb[2 * 4 + UR] += -1.0;                /* hu- = hu_R of element i-1 */
            Lb[2 * 4 + PR] += -c11;                /* p-  = p_R of element i-1 */
        } else {
            double hum = (i > 0) ? hut[2 * i - 1] : 0.0;   /* predicted hu outside, 0 at the wall */
            r[2] += hum;                                   /* -(-hum) moved to the right-hand side */
        }
        Db[2 * 4 + PL] += c11;                     /* -(-c11 p_L) */
        Db[2 * 4 + UL] += 0.5; Db[2 * 4 + UR] += 0.5;
        Db[2 * 4 + UL] += m6 * 2.0 * cL.s21; Db[2 * 4 + UR] += m6 * cR.s21;
        Db[2 * 4 + PL] += m6 * 2.0 * cL.s22; Db[2 * 4 + PR] += m6 * cR.s22;
        r[2] += m6 * (2.0 * cL.f2 + cR.f2);
        /* row 3: Eq. 13 tested with phi_R:  +hu*(right) - (hu_L + hu_R)/2 + mass terms = int f2 phi_R,
           hu*(right) = hu_R + c11 (p_R - p+), p+ = p_L of element i+1 or 0 */
        Db[3 * 4 + UR] += 1.0;
        Db[3 * 4 + PR] += c11;
        if (mrgt) Ub[3 * 4 + PL] += -c11;
        Db[3 * 4 + UL] += -0.5; Db[3 * 4 + UR] += -0.5;
        Db[3 * 4 + UL] += m6 * cL.s21; Db[3 * 4 + UR] += m6 * 2.0 * cR.s21;
        Db[3 * 4 + PL] += m6 * cL.s22; Db[3 * 4 + PR] += m6 * 2.0 * cR.s22;
        r[3] = m6 * (cL.f2 + 2.0 * cR.f2);
    }
}

/* ----------------------------------------------------------------- solve */

/* Gaussian elimination with partial pivoting in band form (Golub & Van Loan):
   n = 4 ne unknowns, lower bandwidth KL = 7 and upper bandwidth KU = 7 of the
   block-tridiagonal matrix; pivoting widens the upper band by KL.  Row r of
   the band holds columns r - KL .. r + KL + KU at index c - r + KL. */
static int band_solve(int ne, const double* blk, const double* rhs, double* x)
{
    enum { KL = 7, KU = 7, W = 2 * KL + KU + 1 };
    int n = 4 * ne;
    double* A = calloc((size_t)n * W, sizeof(double));
    double* b = malloc(sizeof(double) * n);
#define AB(r, c) A[(size_t)(r) * W + ((c) - (r) + KL)]
    for (int i = 0; i < ne; ++i)
        for (int a = 0; a < 4; ++a) {
            int r = 4 * i + a;
            for (int q = 0; q < 3; ++q) {
                int e = i + q - 1;
                if (e < 0 || e >= ne) continue;
                for (int c = 0; c < 4; ++c) {
                    double v = blk[48 * i + 16 * q + 4 * a + c];
                    if (v != 0.0) AB(r, 4 * e + c) = v;
                }
            }
            b[r] = rhs[r];
        }
    int status = OR_OK;
    for (int c = 0; c < n; ++c) {
        int piv = c, last = c + KL < n - 1 ? c + KL : n - 1;
        for (int r = c + 1; r <= last; ++r)
            if (fabs(AB(r, c)) > fabs(AB(piv, c))) piv = r;
        if (AB(piv, c) == 0.0) { status = OR_SINGULAR; break; }
        int jmax = c + KL + KU < n - 1 ? c + KL + KU : n - 1;
        if (piv != c) {
            for (int j = c; j <= jmax; ++j) {
                double tmp = AB(c, j); AB(c, j) = AB(piv, j); AB(piv, j) = tmp;
            }
            double tb = b[c]; b[c] = b[piv]; b[piv] = tb;
        }
        for (int r = c + 1; r <= last; ++r) {
            double f = AB(r, c) / AB(c, c);
            if (f == 0.0) continue;
            for (int j = c; j <= jmax; ++j) AB(r, j) -= f * AB(c, j);
            b[r] -= f * b[c];
        }
    }
    if (status == OR_OK) {
        for (int r = n - 1; r >= 0; --r) {
            double s = b[r];
            int jmax = r + KL + KU < n - 1 ? r + KL + KU : n - 1;
            for (int j = r + 1; j <= jmax; ++j) s -= AB(r, j) * x[j];
            x[r] = s / AB(r, r);
        }
    }
#undef AB
    free(A); free(b);
    return status;
}

/* r = rhs - A x of the block-tridiagonal system; returns ||rhs||^2 in *bb. */
static double dg_residual(int ne, const double* blk, const double* rhs, const double* x, double* r, double* bb)
{
    double rr = 0.0, b2 = 0.0;
    for (int i = 0; i < ne; ++i)
        for (int a = 0; a < 4; ++a) {
            double s = rhs[4 * i + a];
            for (int q = 0; q < 3; ++q) {
                int e = i + q - 1;
                if (e < 0 || e >= ne) continue;
                for (int c = 0; c < 4; ++c) s -= blk[48 * i + 16 * q + 4 * a + c] * x[4 * e + c];
            }
            r[4 * i + a] = s;
            rr += s * s;
            b2 += rhs[4 * i + a] * rhs[4 * i + a];
        }
    *bb = b2;
    return rr;
}

/* The banded elimination, then two steps of iterative refinement (the
   residual in FP64, the correction by the same elimination): the system's
   conditioning amplifies the elimination's rounding (the unscaled penalty c11
   dominates the p-rows over the physical terms), and refinement brings the
   solution back to the accuracy that conditioning allows. */
int or_dg_solve(const or_dg_params* P, const double* blk, const double* rhs, double* x, double* rel_res)
{
    int ne = P->ne, n = 4 * ne;
    int status = band_solve(ne, blk, rhs, x);
    double* r = malloc(sizeof(double) * n);
    double* dx = malloc(sizeof(double) * n);
    double bb = 0.0;
    for (int it = 0; it < 2 && status == OR_OK; ++it) {
        dg_residual(ne, blk, rhs, x, r, &bb);
        status = band_solve(ne, blk, r, dx);
        if (status == OR_OK)
            for (int k = 0; k < n; ++k) x[k] += dx[k];
    }
    if (status == OR_OK && rel_res) {
        double rr = dg_residual(ne, blk, rhs, x, r, &bb);
        *rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    }
    free(r); free(dx);
    return status;
}

/* ------------------------------------------------------------ correction */

/* Eq. 11 on marked elements: hw = hw~ + (dt/rho) (6/D p + d_x/D (h p)_x + phi),
   (h p)_x the element's P1 slope of the nodal h~ p; hu = the LDG unknown;
   h = h~ (Sec. 3.2). */
void or_dg_correct(const or_dg_params* P, double t1, double dt, const unsigned char* mask, const double* x,
                   const double* ht, const double* hut, const double* hwt, double* h, double* hu, double* hw,
                   double* p)
{
    int ne = P->ne;
    for (int i = 0; i < ne; ++i) {
        int kL = 2 * i, kR = 2 * i + 1;
        h[kL] = ht[kL]; h[kR] = ht[kR];
        if (!mask[i]) {
            hu[kL] = hut[kL]; hu[kR] = hut[kR];
            hw[kL] = hwt[kL]; hw[kR] = hwt[kR];
            p[kL] = 0.0; p[kR] = 0.0;
            continue;
        }
        double pL = x[4 * i], pR = x[4 * i + 1];
        double hp_x = (ht[kR] * pR - ht[kL] * pL) / P->dx;
        for (int s = 0; s < 2; ++s) {
            int k = s ? kR : kL;
            double pk = s ? pR : pL;
            node_coef c = coef_at(P, t1, dt, ht, hut, hwt, i, k);
            hw[k] = hwt[k] + dt / P->rho * (6.0 / c.D * pk + c.d_x / c.D * hp_x + c.phi);
            hu[k] = x[4 * i + 2 + s];
            p[k] = pk;
        }
    }
}

int or_dg_step(const or_dg_params* P, double t, long step, double dt, double* h, double* hu, double* hw,
               double* p, unsigned char* mask_out, or_dg_info* info)
{
    int ne = P->ne, n = 2 * ne;
    double* ht = malloc(sizeof(double) * 3 * n);
    double *hut = ht + n, *hwt = ht + 2 * n;
    unsigned char* mask = malloc(ne);
    or_dg_predict(P, t, dt, h, hu, hw, ht, hut, hwt);
    int na = or_dg_mask(P, t + dt, step, ht, hut, hwt, mask);
    double* blk = malloc(sizeof(double) * 48 * ne);
    double* rhs = malloc(sizeof(double) * 4 * ne);
    double* x = calloc(4 * ne, sizeof(double));
    or_dg_assemble(P, t + dt, dt, ht, hut, hwt, mask, blk, rhs);
    double rel = 0.0;
    int status = or_dg_solve(P, blk, rhs, x, &rel);
    if (status == OR_OK) or_dg_correct(P, t + dt, dt, mask, x, ht, hut, hwt, h, hu, hw, p);
    if (mask_out) memcpy(mask_out, mask, ne);
    if (info) { info->n_active = na; info->status = status; info->rel_res = rel; }
    free(ht); free(mask); free(blk); free(rhs); free(x);
    return status;
}
