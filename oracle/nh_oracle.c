/*
 * nh_oracle.c -- plain FP64 CPU oracle (1D) of the locally adaptive
 * non-hydrostatic shallow-water method.  TEST INFRASTRUCTURE ONLY: see
 * nh_oracle.h.  Written for reading, not speed: one loop per formula, whole
 * arrays with ghost cells, no fusion.
 *
 * ---------------------------------------------------------------------------
 * The elliptic equation (derived here from Sec. 3.2, Eqs. 4, 5, 10, 11).
 *
 * Notation: h = h~^{n+1}, d = d^{n+1}, G = d_x^2, D = 4 + G, a = dt / rho and
 * q = h p^nh.  Eq. 5 at the bottom, with (h p)_x = q_x:
 *     P = 6 q / (h D) + d_x q_x / D + phi,
 *     phi = rho h / D (g d_x eta_x - d_tt - 2 u d_xt - u^2 d_xx).
 * Eq. 10:  HU = hu~ - a q_x + a d_x P
 *            = U0 - a (4/D) q_x + (6 a d_x / (h D)) q,   U0 = hu~ + a phi d_x
 * Eq. 11:  HW = hw~ + a P
 * Constraint Eq. 4 at n+1, h (HU)_x + HU (2 d_x - h_x) + 2 HW + 2 h d_t = 0,
 * rewritten as h^2 (HU/h)_x + 2 d_x HU + 2 HW + 2 h d_t = 0 and divided by
 * h^2.  Inserting HU and HW, the q_x terms that are not under the outer
 * derivative carry the factors 6, -8 and +2 (times a d_x / (h^2 D)) and
 * cancel, which leaves the self-adjoint equation
 *     -(K q_x)_x + gamma q = R
 *     K     = 4 a / (h D)
 *     beta  = 6 a d_x / (h^2 D)
 *     gamma = beta_x + 12 a (1 + G) / (h^3 D)
 *     R     = -[ (U0/h)_x + 2 d_x U0 / h^2 + 2 hw~ / h^2 + 2 a phi / h^2
 *                + 2 d_t / h ].
 * Discretisation: conservative three-point form with face coefficients
 * K_{i+1/2} = (K_i + K_{i+1}) / 2, central differences for beta_x, (U0/h)_x,
 * eta_x, u; q = 0 on cells outside the mask and outside a walled domain
 * (zero Dirichlet data, Sec. 3.2 last paragraph and Sec. 5.2).  The matrix is
 * symmetric; it is positive definite when gamma > 0 on every active cell.
 *
 * Ghost cells at a wall: every scalar is mirrored (eta, h, d, w, K even;
 * u, hu, d_x and everything odd in d_x, i.e. beta and U0/h, change sign).
 * ---------------------------------------------------------------------------
 */
#include "nh_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ----------------------------------------------------------------- ghosts */

/* In-domain cell for index j in [-2, nx+1]; *odd = -1 where a wall mirror
   flips the sign of odd quantities, +1 otherwise. */
static int ghost(const or_params* P, int j, double* odd)
{
    int n = P->nx;
    *odd = 1.0;
    if (j >= 0 && j < n) return j;
    if (P->bc == OR_BC_PERIODIC) return ((j % n) + n) % n;
    *odd = -1.0;
    return (j < 0) ? (-1 - j) : (2 * n - 1 - j);
}

/* Is the neighbour j of an active cell a valid unknown?  Returns its index,
   or -1 if it lies outside a walled domain. */
static int inner(const or_params* P, int j)
{
    int n = P->nx;
    if (j >= 0 && j < n) return j;
    if (P->bc == OR_BC_PERIODIC) return ((j % n) + n) % n;
    return -1;
}

/* ----------------------------------------------------------------- bottom */

/* Slide displacement s(t) = s0 ln cosh(t/t0) and its first two derivatives. */
static void slide_law(const or_params* P, double t, double* s, double* sd, double* sdd)
{
    double z = t / P->t0;
    *s = P->s0 * log(cosh(z));
    *sd = (P->s0 / P->t0) * tanh(z);
    *sdd = (P->s0 / (P->t0 * P->t0)) / (cosh(z) * cosh(z));
}

/* The sliding block's position S(t) (Sec. 4.3): S = a0 t^2 / 2 up to t1,
   then S(t1) + ut (t - t1) up to t2, then that minus a0 (t - t2)^2 / 2 up to
   t3, constant after; ut = a0 t1 and t3 = t2 + t1 make S' continuous and
   zero from t3 on.  S(t) = 0 before t = 0. */
static void block_law(const or_params* P, double t, double* S, double* Sd, double* Sdd)
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

/* d(x,t) = d0(x) - m(x,t) for the motions listed in nh_oracle.h.  For the
   mound, xi = (x - xc0 - s(t)) / L and the derivatives of m follow from the
   chain rule with dxi/dx = 1/L and dxi/dt = -s'(t)/L; for the block,
   xi = 2 (x - xc0 - S(t)) / L with dxi/dx = 2/L and dxi/dt = -2 S'(t)/L; the
   plate moves vertically only, and its edges (a jump of the depth) reach the
   method through the depth at cell centres and faces. */
void or_bottom(const or_params* P, const double* d0, int i, double t, double out[6])
{
    double odd;
    int im = ghost(P, i - 1, &odd), ip = ghost(P, i + 1, &odd);
    double dx = P->dx;
    double d = d0[i];
    double d_x = (d0[ip] - d0[im]) / (2.0 * dx);
    double d_xx = (d0[ip] - 2.0 * d0[i] + d0[im]) / (dx * dx);
    double d_t = 0.0, d_xt = 0.0, d_tt = 0.0;
    if (P->slide == OR_SLIDE_GAUSS_LNCOSH) {
        double s, sd, sdd;
        slide_law(P, t, &s, &sd, &sdd);
        double x = P->xl + (i + 0.5) * dx;
        double L = P->L;
        double xi = (x - P->xc0 - s) / L;
        double m = P->A * exp(-xi * xi);
        double m_x = m * (-2.0 * xi / L);
        double m_xx = m * (4.0 * xi * xi - 2.0) / (L * L);
        double m_t = m * (2.0 * xi / L) * sd;
        double m_xt = -m * (2.0 / (L * L)) * (2.0 * xi * xi - 1.0) * sd;
        double m_tt = m * (2.0 / (L * L)) * ((2.0 * xi * xi - 1.0) * sd * sd + xi * L * sdd);
        d -= m; d_x -= m_x; d_xx -= m_xx;
        d_t = -m_t; d_xt = -m_xt; d_tt = -m_tt;
    } else if (P->slide == OR_SLIDE_PLATE_EXP) {
        double x = P->xl + (i + 0.5) * dx;
        if (fabs(x - P->xc0) < P->L) {
            double e = exp(-t / P->t0);
            d -= P->A * (1.0 - e);
            d_t = -P->A * e / P->t0;
            d_tt = P->A * e / (P->t0 * P->t0);
        }
    } else if (P->slide == OR_SLIDE_QUARTIC) {
        double S, Sd, Sdd;
        block_law(P, t, &S, &Sd, &Sdd);
        double x = P->xl + (i + 0.5) * dx;
        double L = P->L;
        double xi = 2.0 * (x - P->xc0 - S) / L;
        if (fabs(xi) < 1.0) {
            double A = P->A, xi2 = xi * xi, xi3 = xi2 * xi;
            double m = A * (1.0 - xi2 * xi2);
            double m_x = -8.0 * A * xi3 / L;
            double m_xx = -48.0 * A * xi2 / (L * L);
            double m_t = 8.0 * A * xi3 * Sd / L;
            double m_xt = 48.0 * A * xi2 * Sd / (L * L);
            double m_tt = (8.0 * A / L) * (-6.0 * xi2 * Sd * Sd / L + xi3 * Sdd);
            d -= m; d_x -= m_x; d_xx -= m_xx;
            d_t = -m_t; d_xt = -m_xt; d_tt = -m_tt;
        }
    }
    out[0] = d; out[1] = d_x; out[2] = d_xx; out[3] = d_t; out[4] = d_xt; out[5] = d_tt;
}

static double depth_at(const or_params* P, const double* d0, int i, double t)
{
    double b[6];
    or_bottom(P, d0, i, t, b);
    return b[0];
}

/* -------------------------------------------------------------- predictor */

static double minmod2(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return (fabs(a) < fabs(b)) ? a : b;
}

/* Limited slope (per cell) from the three values vm, v0, vp. */
static double slope(int limiter, double vm, double v0, double vp)
{
    switch (limiter) {
    case OR_LIM_CENTRAL: return 0.5 * (vp - vm);
    case OR_LIM_MINMOD:  return minmod2(vp - v0, v0 - vm);
    case OR_LIM_MC:      return minmod2(0.5 * (vp - vm), minmod2(2.0 * (vp - v0), 2.0 * (v0 - vm)));
    default:             return 0.0;
    }
}

/* Rusanov (local Lax-Friedrichs) flux of F(Q) = (hu, hu^2 + g h^2/2, huw)
   (Sec. 3.1) between left state (hL,uL,wL) and right state (hR,uR,wR). */
static void rusanov(double g, double hL, double uL, double wL,
                    double hR, double uR, double wR, double F[3])
{
    double FL0 = hL * uL, FL1 = hL * uL * uL + 0.5 * g * hL * hL, FL2 = hL * uL * wL;
    double FR0 = hR * uR, FR1 = hR * uR * uR + 0.5 * g * hR * hR, FR2 = hR * uR * wR;
    double sL = fabs(uL) + sqrt(g * hL), sR = fabs(uR) + sqrt(g * hR);
    double s = (sL > sR) ? sL : sR;
    F[0] = 0.5 * (FL0 + FR0) - 0.5 * s * (hR - hL);
    F[1] = 0.5 * (FL1 + FR1) - 0.5 * s * (hR * uR - hL * uL);
    F[2] = 0.5 * (FL2 + FR2) - 0.5 * s * (hR * wR - hL * wL);
}

/* H(Q) of the hydrostatic equations (Eqs. 1-3 without p^nh terms), source
   S = (0, g h d_x, 0).  Second-order MUSCL reconstruction of eta, u, w with
   the bottom depth taken continuous at faces, d_f = (d_i + d_{i+1}) / 2, so
   that h_f = eta_f + d_f; the source is integrated as
   g * (h_{i-1/2}^+ + h_{i+1/2}^-) / 2 * (d_{i+1/2} - d_{i-1/2}) / dx, which
   balances the flux of g h^2/2 exactly for a lake at rest. */
void or_rhs(const or_params* P, const double* d0, double t,
            const double* h, const double* hu, const double* hw,
            double* rh, double* rhu, double* rhw)
{
    int n = P->nx;
    double g = P->g, dx = P->dx;
    /* extended arrays, index j+2 for cell j in [-2, n+1] */
    double* eta = malloc(sizeof(double) * (n + 4));
    double* u = malloc(sizeof(double) * (n + 4));
    double* w = malloc(sizeof(double) * (n + 4));
    double* d = malloc(sizeof(double) * (n + 4));
    double* se = malloc(sizeof(double) * (n + 4));
    double* su = malloc(sizeof(double) * (n + 4));
    double* sw = malloc(sizeof(double) * (n + 4));
    double* df = malloc(sizeof(double) * (n + 1));
    double (*F)[3] = malloc(sizeof(double[3]) * (n + 1));
    double* hplus = malloc(sizeof(double) * n);   /* cell i at its left face  */
    double* hminus = malloc(sizeof(double) * n);  /* cell i at its right face */

    for (int j = -2; j < n + 2; ++j) {
        double odd;
        int c = ghost(P, j, &odd);
        double dc = depth_at(P, d0, c, t);
        d[j + 2] = dc;
        eta[j + 2] = h[c] - dc;
        u[j + 2] = odd * hu[c] / h[c];
        w[j + 2] = hw[c] / h[c];
    }
    for (int j = -1; j < n + 1; ++j) {
        se[j + 2] = slope(P->limiter, eta[j + 1], eta[j + 2], eta[j + 3]);
        su[j + 2] = slope(P->limiter, u[j + 1], u[j + 2], u[j + 3]);
        sw[j + 2] = slope(P->limiter, w[j + 1], w[j + 2], w[j + 3]);
    }
    /* face k lies between cells k-1 and k */
    for (int k = 0; k <= n; ++k) {
        int L = k - 1, R = k;
        df[k] = 0.5 * (d[L + 2] + d[R + 2]);
        double hL = eta[L + 2] + 0.5 * se[L + 2] + df[k];
        double uL = u[L + 2] + 0.5 * su[L + 2];
        double wL = w[L + 2] + 0.5 * sw[L + 2];
        double hR = eta[R + 2] - 0.5 * se[R + 2] + df[k];
        double uR = u[R + 2] - 0.5 * su[R + 2];
        double wR = w[R + 2] - 0.5 * sw[R + 2];
        rusanov(g, hL, uL, wL, hR, uR, wR, F[k]);
    }
    for (int i = 0; i < n; ++i) {
        hplus[i] = eta[i + 2] - 0.5 * se[i + 2] + df[i];
        hminus[i] = eta[i + 2] + 0.5 * se[i + 2] + df[i + 1];
    }
    for (int i = 0; i < n; ++i) {
        double S = g * 0.5 * (hplus[i] + hminus[i]) * (df[i + 1] - df[i]) / dx;
        rh[i] = -(F[i + 1][0] - F[i][0]) / dx;
        rhu[i] = -(F[i + 1][1] - F[i][1]) / dx + S;
        rhw[i] = -(F[i + 1][2] - F[i][2]) / dx;
    }
    free(eta); free(u); free(w); free(d); free(se); free(su); free(sw);
    free(df); free(F); free(hplus); free(hminus);
}

/* Heun: Q* = Q^n + dt H(Q^n; d^n),  Q~ = Q^n + dt/2 (H(Q^n; d^n) + H(Q*; d^{n+1})). */
void or_predict(const or_params* P, const double* d0, double t, double dt,
                const double* h, const double* hu, const double* hw,
                double* ht, double* hut, double* hwt)
{
    int n = P->nx;
    double* k1h = malloc(sizeof(double) * n);
    double* k1u = malloc(sizeof(double) * n);
    double* k1w = malloc(sizeof(double) * n);
    double* k2h = malloc(sizeof(double) * n);
    double* k2u = malloc(sizeof(double) * n);
    double* k2w = malloc(sizeof(double) * n);
    double* sh = malloc(sizeof(double) * n);
    double* su = malloc(sizeof(double) * n);
    double* sw = malloc(sizeof(double) * n);
    or_rhs(P, d0, t, h, hu, hw, k1h, k1u, k1w);
    for (int i = 0; i < n; ++i) {
        sh[i] = h[i] + dt * k1h[i];
        su[i] = hu[i] + dt * k1u[i];
        sw[i] = hw[i] + dt * k1w[i];
    }
    or_rhs(P, d0, t + dt, sh, su, sw, k2h, k2u, k2w);
    for (int i = 0; i < n; ++i) {
        ht[i] = h[i] + 0.5 * dt * (k1h[i] + k2h[i]);
        hut[i] = hu[i] + 0.5 * dt * (k1u[i] + k2u[i]);
        hwt[i] = hw[i] + 0.5 * dt * (k1w[i] + k2w[i]);
    }
    free(k1h); free(k1u); free(k1w); free(k2h); free(k2u); free(k2w);
    free(sh); free(su); free(sw);
}

/* ---------------------------------------------------------- criterion, mask */

/* Sec. 5.1: |eta/d|, |eta_x|, |u|, |u_x|, |w|, |w_x| of the predicted state;
   x-derivatives by central differences with mirrored / periodic ghosts. */
void or_criterion(const or_params* P, const double* d0, double t,
                  const double* ht, const double* hut, const double* hwt,
                  double* c)
{
    int n = P->nx;
    double dx = P->dx;
    for (int i = 0; i < n; ++i) {
        double om, op;
        int im = ghost(P, i - 1, &om), ip = ghost(P, i + 1, &op);
        double dm = depth_at(P, d0, im, t), di = depth_at(P, d0, i, t), dp = depth_at(P, d0, ip, t);
        double eta_m = ht[im] - dm, eta_i = ht[i] - di, eta_p = ht[ip] - dp;
        double u_m = om * hut[im] / ht[im], u_i = hut[i] / ht[i], u_p = op * hut[ip] / ht[ip];
        double w_m = hwt[im] / ht[im], w_i = hwt[i] / ht[i], w_p = hwt[ip] / ht[ip];
        double v;
        switch (P->crit) {
        case OR_CRIT_ETA_D: v = fabs(eta_i / di); break;
        case OR_CRIT_ETA_X: v = fabs((eta_p - eta_m) / (2.0 * dx)); break;
        case OR_CRIT_U:     v = fabs(u_i); break;
        case OR_CRIT_U_X:   v = fabs((u_p - u_m) / (2.0 * dx)); break;
        case OR_CRIT_W:     v = fabs(w_i); break;
        case OR_CRIT_W_X:   v = fabs((w_p - w_m) / (2.0 * dx)); break;
        default:            v = 0.0; break;
        }
        c[i] = v;
    }
}

/* Cells where the criterion exceeds knh (Sec. 5.1), all cells on the first
   step when first_step_global is set (Sec. 5.1.2), then enlarged by
   `enlarge` cells on each side (Sec. 5.2). */
int or_mask(const or_params* P, const double* d0, double t, long step,
            const double* ht, const double* hut, const double* hwt,
            unsigned char* mask)
{
    int n = P->nx;
    unsigned char* marked = malloc(n);
    if (P->crit == OR_CRIT_GLOBAL || (P->first_step_global && step == 0)) {
        for (int i = 0; i < n; ++i) marked[i] = 1;
    } else if (P->crit == OR_CRIT_HYDROSTATIC) {
        for (int i = 0; i < n; ++i) marked[i] = 0;
    } else {
        double* c = malloc(sizeof(double) * n);
        or_criterion(P, d0, t, ht, hut, hwt, c);
        for (int i = 0; i < n; ++i) marked[i] = (c[i] > P->knh) ? 1 : 0;
        free(c);
    }
    int count = 0;
    for (int i = 0; i < n; ++i) {
        unsigned char m = 0;
        for (int k = -P->enlarge; k <= P->enlarge; ++k) {
            int j = inner(P, i + k);
            if (j >= 0 && marked[j]) m = 1;
        }
        mask[i] = m;
        count += m;
    }
    free(marked);
    return count;
}

/* --------------------------------------------------------------- assembly */

void or_assemble(const or_params* P, const double* d0, double t1, double dt,
                 const double* ht, const double* hut, const double* hwt,
                 double* Kf, double* gam, double* R)
{
    int n = P->nx;
    double dx = P->dx, g = P->g, rho = P->rho;
    double a = dt / rho;
    double* K = malloc(sizeof(double) * n);
    double* beta = malloc(sizeof(double) * n);
    double* V = malloc(sizeof(double) * n);   /* U0 / h */
    double* U0 = malloc(sizeof(double) * n);
    double* phi = malloc(sizeof(double) * n);
    for (int i = 0; i < n; ++i) {
        double b[6], om, op;
        or_bottom(P, d0, i, t1, b);
        int im = ghost(P, i - 1, &om), ip = ghost(P, i + 1, &op);
        double eta_x = ((ht[ip] - depth_at(P, d0, ip, t1)) - (ht[im] - depth_at(P, d0, im, t1))) / (2.0 * dx);
        double h = ht[i], u = hut[i] / h;
        double d_x = b[1], d_xx = b[2], d_xt = b[4], d_tt = b[5];
        double D = 4.0 + d_x * d_x;
        /* Eq. 5: phi = rho h / (4 + d_x^2) (g d_x eta_x - d_tt - 2 u d_xt - u^2 d_xx) */
        phi[i] = rho * h / D * (g * d_x * eta_x - d_tt - 2.0 * u * d_xt - u * u * d_xx);
        K[i] = 4.0 * a / (h * D);
        beta[i] = 6.0 * a * d_x / (h * h * D);
        U0[i] = hut[i] + a * phi[i] * d_x;
        V[i] = U0[i] / h;
    }
    for (int k = 0; k <= n; ++k) {
        double om, op;
        int L = ghost(P, k - 1, &om), Rr = ghost(P, k, &op);
        Kf[k] = 0.5 * (K[L] + K[Rr]);
    }
    for (int i = 0; i < n; ++i) {
        double b[6], om, op;
        or_bottom(P, d0, i, t1, b);
        int im = ghost(P, i - 1, &om), ip = ghost(P, i + 1, &op);
        double h = ht[i];
        double d_x = b[1], d_t = b[3];
        double G = d_x * d_x, D = 4.0 + G;
        double beta_x = (op * beta[ip] - om * beta[im]) / (2.0 * dx);
        double V_x = (op * V[ip] - om * V[im]) / (2.0 * dx);
        gam[i] = beta_x + 12.0 * a * (1.0 + G) / (h * h * h * D);
        R[i] = -(V_x + 2.0 * d_x * U0[i] / (h * h) + 2.0 * hwt[i] / (h * h)
                 + 2.0 * a * phi[i] / (h * h) + 2.0 * d_t / h);
    }
    free(K); free(beta); free(V); free(U0); free(phi);
}

/* (A x)_i = [K_{i-1/2}(x_i - x_{i-1}) + K_{i+1/2}(x_i - x_{i+1})] / dx^2 + gamma_i x_i,
   with x = 0 on inactive cells and outside a walled domain. */
void or_apply(const or_params* P, const unsigned char* mask,
              const double* Kf, const double* gam, const double* x, double* y)
{
    int n = P->nx;
    double idx2 = 1.0 / (P->dx * P->dx);
    for (int i = 0; i < n; ++i) {
        if (!mask[i]) { y[i] = 0.0; continue; }
        int jm = inner(P, i - 1), jp = inner(P, i + 1);
        double xm = (jm >= 0 && mask[jm]) ? x[jm] : 0.0;
        double xp = (jp >= 0 && mask[jp]) ? x[jp] : 0.0;
        y[i] = (Kf[i] * (x[i] - xm) + Kf[i + 1] * (x[i] - xp)) * idx2 + gam[i] * x[i];
    }
}

/* ----------------------------------------------------------------- solvers */

static double dot_masked(int n, const unsigned char* mask, const double* a, const double* b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        if (mask[i]) s += a[i] * b[i];
    return s;
}

/* Conjugate gradients (Hestenes-Stiefel) on the active cells. */
static int solve_cg(const or_params* P, const unsigned char* mask, const double* Kf,
                    const double* gam, const double* R, double* x, or_step_info* info)
{
    int n = P->nx;
    double* r = calloc(n, sizeof(double));
    double* p = calloc(n, sizeof(double));
    double* Ap = calloc(n, sizeof(double));
    for (int i = 0; i < n; ++i) if (!mask[i]) x[i] = 0.0;
    or_apply(P, mask, Kf, gam, x, Ap);
    for (int i = 0; i < n; ++i) r[i] = mask[i] ? R[i] - Ap[i] : 0.0;
    double bnorm = sqrt(dot_masked(n, mask, R, R));
    double rr = dot_masked(n, mask, r, r);
    int it = 0, status = OR_NOT_CONVERGED;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        rr = 0.0; bnorm = 1.0; status = OR_OK;
    } else if (sqrt(rr) <= P->rtol * bnorm) {
        status = OR_OK;
    } else {
        for (int i = 0; i < n; ++i) p[i] = r[i];
        for (it = 1; it <= P->max_iter; ++it) {
            or_apply(P, mask, Kf, gam, p, Ap);
            double alpha = rr / dot_masked(n, mask, p, Ap);
            for (int i = 0; i < n; ++i) if (mask[i]) { x[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; }
            double rr_new = dot_masked(n, mask, r, r);
            if (sqrt(rr_new) <= P->rtol * bnorm) { rr = rr_new; status = OR_OK; break; }
            double beta = rr_new / rr;
            rr = rr_new;
            for (int i = 0; i < n; ++i) if (mask[i]) p[i] = r[i] + beta * p[i];
        }
        if (it > P->max_iter) it = P->max_iter;
    }
    info->iters = it;
    info->rel_res = sqrt(rr) / bnorm;
    info->solver_used = OR_SOLVER_CG;
    free(r); free(p); free(Ap);
    return status;
}

/* BiCGStab (van der Vorst 1992) on the active cells. */
static int solve_bicgstab(const or_params* P, const unsigned char* mask, const double* Kf,
                          const double* gam, const double* R, double* x, or_step_info* info)
{
    int n = P->nx;
    double* r = calloc(n, sizeof(double));
    double* rh = calloc(n, sizeof(double));
    double* p = calloc(n, sizeof(double));
    double* v = calloc(n, sizeof(double));
    double* s = calloc(n, sizeof(double));
    double* tt = calloc(n, sizeof(double));
    for (int i = 0; i < n; ++i) if (!mask[i]) x[i] = 0.0;
    or_apply(P, mask, Kf, gam, x, v);
    for (int i = 0; i < n; ++i) { r[i] = mask[i] ? R[i] - v[i] : 0.0; rh[i] = r[i]; v[i] = 0.0; }
    double bnorm = sqrt(dot_masked(n, mask, R, R));
    double rnorm = sqrt(dot_masked(n, mask, r, r));
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    int it = 0, status = OR_NOT_CONVERGED;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        rnorm = 0.0; bnorm = 1.0; status = OR_OK;
    } else if (rnorm <= P->rtol * bnorm) {
        status = OR_OK;
    } else {
        for (it = 1; it <= P->max_iter; ++it) {
            double rho = dot_masked(n, mask, rh, r);
            double beta = (rho / rho_old) * (alpha / omega);
            for (int i = 0; i < n; ++i) if (mask[i]) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            or_apply(P, mask, Kf, gam, p, v);
            alpha = rho / dot_masked(n, mask, rh, v);
            for (int i = 0; i < n; ++i) if (mask[i]) s[i] = r[i] - alpha * v[i];
            double snorm = sqrt(dot_masked(n, mask, s, s));
            if (snorm <= P->rtol * bnorm) {
                for (int i = 0; i < n; ++i) if (mask[i]) x[i] += alpha * p[i];
                rnorm = snorm; status = OR_OK; break;
            }
            or_apply(P, mask, Kf, gam, s, tt);
            omega = dot_masked(n, mask, tt, s) / dot_masked(n, mask, tt, tt);
            for (int i = 0; i < n; ++i) if (mask[i]) {
                x[i] += alpha * p[i] + omega * s[i];
                r[i] = s[i] - omega * tt[i];
            }
            rnorm = sqrt(dot_masked(n, mask, r, r));
            if (rnorm <= P->rtol * bnorm) { status = OR_OK; break; }
            rho_old = rho;
        }
        if (it > P->max_iter) it = P->max_iter;
    }
    info->iters = it;
    info->rel_res = rnorm / bnorm;
    info->solver_used = OR_SOLVER_BICGSTAB;
    free(r); free(rh); free(p); free(v); free(s); free(tt);
    return status;
}

/* Dense Gaussian elimination with partial pivoting on the active block
   (textbook; tiny grids only).  Column l of the block is A applied to the
   l-th active unit vector. */
static int solve_dense(const or_params* P, const unsigned char* mask, const double* Kf,
                       const double* gam, const double* R, double* x, or_step_info* info)
{
    int n = P->nx, m = 0;
    int* idx = malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) if (mask[i]) idx[m++] = i;
    double* M = calloc((size_t)m * m, sizeof(double));
    double* b = malloc(sizeof(double) * (m > 0 ? m : 1));
    double* e = calloc(n, sizeof(double));
    double* col = calloc(n, sizeof(double));
    for (int l = 0; l < m; ++l) {
        e[idx[l]] = 1.0;
        or_apply(P, mask, Kf, gam, e, col);
        e[idx[l]] = 0.0;
        for (int k = 0; k < m; ++k) M[(size_t)k * m + l] = col[idx[k]];
    }
    for (int k = 0; k < m; ++k) b[k] = R[idx[k]];
    int status = OR_OK;
    for (int c = 0; c < m; ++c) {
        int piv = c;
        for (int r = c + 1; r < m; ++r)
            if (fabs(M[(size_t)r * m + c]) > fabs(M[(size_t)piv * m + c])) piv = r;
        if (M[(size_t)piv * m + c] == 0.0) { status = OR_SINGULAR; break; }
        if (piv != c) {
            for (int l = 0; l < m; ++l) {
                double tmp = M[(size_t)c * m + l];
                M[(size_t)c * m + l] = M[(size_t)piv * m + l];
                M[(size_t)piv * m + l] = tmp;
            }
            double tb = b[c]; b[c] = b[piv]; b[piv] = tb;
        }
        for (int r = c + 1; r < m; ++r) {
            double f = M[(size_t)r * m + c] / M[(size_t)c * m + c];
            for (int l = c; l < m; ++l) M[(size_t)r * m + l] -= f * M[(size_t)c * m + l];
            b[r] -= f * b[c];
        }
    }
    for (int i = 0; i < n; ++i) x[i] = 0.0;
    if (status == OR_OK) {
        for (int k = m - 1; k >= 0; --k) {
            double s = b[k];
            for (int l = k + 1; l < m; ++l) s -= M[(size_t)k * m + l] * x[idx[l]];
            x[idx[k]] = s / M[(size_t)k * m + k];
        }
    }
    info->iters = 1;
    info->rel_res = 0.0;
    info->solver_used = OR_SOLVER_DENSE;
    free(idx); free(M); free(b); free(e); free(col);
    return status;
}

/* Direct solve of the tridiagonal active block: Gaussian elimination with
   partial pivoting in band form (a row interchange gives U a second
   superdiagonal; Golub & Van Loan, band Gaussian elimination with pivoting).
   The three diagonals are read off the operator itself: or_apply on the
   vector that is 1 on every third cell (offset s = 0, 1, 2) gives, in row i,
   the entry of the one column of that colour among i-1, i, i+1.  Inactive
   rows become identity rows (zero right-hand side).  Walls, or a periodic
   grid whose two end cells are not both active (no coupling across the
   wrap); OR_BAD_ARG otherwise. */
static int solve_banded(const or_params* P, const unsigned char* mask, const double* Kf,
                        const double* gam, const double* R, double* x, or_step_info* info)
{
    int n = P->nx;
    if (P->bc == OR_BC_PERIODIC && mask[0] && mask[n - 1]) return OR_BAD_ARG;
    double* lo = calloc(n, sizeof(double));
    double* di = calloc(n, sizeof(double));
    double* up = calloc(n, sizeof(double));
    double* up2 = calloc(n, sizeof(double));
    double* b = calloc(n, sizeof(double));
    double* e = calloc(n, sizeof(double));
    double* y = calloc(n, sizeof(double));
    for (int s = 0; s < 3; ++s) {
        for (int i = 0; i < n; ++i) e[i] = (i % 3 == s) ? 1.0 : 0.0;
        or_apply(P, mask, Kf, gam, e, y);
        for (int i = 0; i < n; ++i) {
            if (!mask[i]) continue;
            if (i % 3 == s) di[i] = y[i];
            else if (i - 1 >= 0 && (i - 1) % 3 == s) lo[i] = y[i];
            else if (i + 1 < n && (i + 1) % 3 == s) up[i] = y[i];
        }
    }
    for (int i = 0; i < n; ++i) {
        if (mask[i]) b[i] = R[i];
        else { lo[i] = 0.0; di[i] = 1.0; up[i] = 0.0; b[i] = 0.0; }
    }
    int status = OR_OK;
    for (int c = 0; c < n; ++c) {
        /* row c holds columns c, c+1, c+2 in di, up, up2; row c+1 holds
           columns c, c+1, c+2 in lo, di, up */
        if (c + 1 < n && fabs(lo[c + 1]) > fabs(di[c])) {
            double r0 = di[c], r1 = up[c];
            di[c] = lo[c + 1]; up[c] = di[c + 1]; up2[c] = up[c + 1];
            lo[c + 1] = r0; di[c + 1] = r1; up[c + 1] = 0.0;
            double tb = b[c]; b[c] = b[c + 1]; b[c + 1] = tb;
        }
        if (di[c] == 0.0) { status = OR_SINGULAR; break; }
        if (c + 1 < n) {
            double f = lo[c + 1] / di[c];
            di[c + 1] -= f * up[c];
            up[c + 1] -= f * up2[c];
            b[c + 1] -= f * b[c];
            lo[c + 1] = 0.0;
        }
    }
    if (status == OR_OK) {
        for (int c = n - 1; c >= 0; --c) {
            double s = b[c];
            if (c + 1 < n) s -= up[c] * x[c + 1];
            if (c + 2 < n) s -= up2[c] * x[c + 2];
            x[c] = s / di[c];
        }
        for (int i = 0; i < n; ++i) if (!mask[i]) x[i] = 0.0;
        or_apply(P, mask, Kf, gam, x, y);
        double rr = 0.0, bb = 0.0;
        for (int i = 0; i < n; ++i)
            if (mask[i]) { rr += (R[i] - y[i]) * (R[i] - y[i]); bb += R[i] * R[i]; }
        info->rel_res = bb > 0.0 ? sqrt(rr / bb) : 0.0;
    } else {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        info->rel_res = 0.0;
    }
    info->iters = 1;
    info->solver_used = OR_SOLVER_BANDED;
    free(lo); free(di); free(up); free(up2); free(b); free(e); free(y);
    return status;
}

int or_solve(const or_params* P, const unsigned char* mask,
             const double* Kf, const double* gam, const double* R,
             double* q, or_step_info* info)
{
    int n = P->nx;
    double gmin = INFINITY;
    int na = 0;
    for (int i = 0; i < n; ++i) if (mask[i]) { ++na; if (gam[i] < gmin) gmin = gam[i]; }
    info->min_gamma = gmin;
    info->n_active = na;
    if (na == 0) {
        for (int i = 0; i < n; ++i) q[i] = 0.0;
        info->iters = 0; info->rel_res = 0.0; info->solver_used = -1;
        return OR_OK;
    }
    int kind = P->solver;
    if (kind == OR_SOLVER_AUTO) kind = (gmin > 0.0) ? OR_SOLVER_CG : OR_SOLVER_BICGSTAB;
    if (kind == OR_SOLVER_CG) return solve_cg(P, mask, Kf, gam, R, q, info);
    if (kind == OR_SOLVER_BICGSTAB) return solve_bicgstab(P, mask, Kf, gam, R, q, info);
    if (kind == OR_SOLVER_DENSE) return solve_dense(P, mask, Kf, gam, R, q, info);
    if (kind == OR_SOLVER_BANDED) return solve_banded(P, mask, Kf, gam, R, q, info);
    return OR_BAD_ARG;
}

/* -------------------------------------------------------------- correction */

/* Eq. 10: (hu - hu~)/dt = -(1/rho) q_x + (d_x/rho) P,
   Eq. 11: (hw - hw~)/dt = P / rho,   P = 6 q/(h D) + d_x q_x / D + phi,
   q_x by central differences with q = 0 off the mask; h = h~ (Sec. 3.2). */
void or_correct(const or_params* P, const double* d0, double t1, double dt,
                const unsigned char* mask, const double* q,
                const double* ht, const double* hut, const double* hwt,
                double* h, double* hu, double* hw)
{
    int n = P->nx;
    double dx = P->dx, g = P->g, rho = P->rho;
    for (int i = 0; i < n; ++i) {
        h[i] = ht[i];
        hu[i] = hut[i];
        hw[i] = hwt[i];
        if (!mask[i]) continue;
        double b[6], om, op;
        or_bottom(P, d0, i, t1, b);
        int im = ghost(P, i - 1, &om), ip = ghost(P, i + 1, &op);
        double eta_x = ((ht[ip] - depth_at(P, d0, ip, t1)) - (ht[im] - depth_at(P, d0, im, t1))) / (2.0 * dx);
        double hh = ht[i], u = hut[i] / hh;
        double d_x = b[1], d_xx = b[2], d_xt = b[4], d_tt = b[5];
        double D = 4.0 + d_x * d_x;
        double phi = rho * hh / D * (g * d_x * eta_x - d_tt - 2.0 * u * d_xt - u * u * d_xx);
        int jm = inner(P, i - 1), jp = inner(P, i + 1);
        double qm = (jm >= 0 && mask[jm]) ? q[jm] : 0.0;
        double qp = (jp >= 0 && mask[jp]) ? q[jp] : 0.0;
        double q_x = (qp - qm) / (2.0 * dx);
        double Pb = 6.0 * q[i] / (hh * D) + d_x * q_x / D + phi;
        hu[i] = hut[i] + dt / rho * (-q_x + d_x * Pb);
        hw[i] = hwt[i] + dt / rho * Pb;
    }
}

/* -------------------------------------------------------------------- step */

int or_step(const or_params* P, const double* d0, double t, long step, double dt,
            double* h, double* hu, double* hw, double* q, unsigned char* mask,
            or_step_info* info)
{
    int n = P->nx;
    if (n < 3 || !(P->dx > 0.0) || !(dt > 0.0)) return OR_BAD_ARG;
    double* ht = malloc(sizeof(double) * n);
    double* hut = malloc(sizeof(double) * n);
    double* hwt = malloc(sizeof(double) * n);
    double* Kf = malloc(sizeof(double) * (n + 1));
    double* gam = malloc(sizeof(double) * n);
    double* R = malloc(sizeof(double) * n);
    unsigned char* m = malloc(n);
    or_step_info loc;
    memset(&loc, 0, sizeof(loc));
    loc.solver_used = -1;
    double t1 = t + dt;

    or_predict(P, d0, t, dt, h, hu, hw, ht, hut, hwt);
    int na = or_mask(P, d0, t1, step, ht, hut, hwt, m);
    int status = OR_OK;
    if (na > 0) {
        or_assemble(P, d0, t1, dt, ht, hut, hwt, Kf, gam, R);
        if (P->guess == OR_GUESS_ZERO)
            for (int i = 0; i < n; ++i) q[i] = 0.0;
        /* previous q on cells active now, zero on newly activated ones */
        for (int i = 0; i < n; ++i) if (!m[i]) q[i] = 0.0;
        status = or_solve(P, m, Kf, gam, R, q, &loc);
        or_correct(P, d0, t1, dt, m, q, ht, hut, hwt, h, hu, hw);
    } else {
        for (int i = 0; i < n; ++i) { h[i] = ht[i]; hu[i] = hut[i]; hw[i] = hwt[i]; q[i] = 0.0; }
        loc.min_gamma = 0.0;
    }
    loc.n_active = na;
    loc.status = status;
    if (mask) memcpy(mask, m, n);
    if (info) *info = loc;
    free(ht); free(hut); free(hwt); free(Kf); free(gam); free(R); free(m);
    return status;
}

int or_run(const or_params* P, const double* d0, double t_start, long step0,
           double dt, long n_steps, double* h, double* hu, double* hw, double* q,
           or_step_info* info, long long* total_iters, long long* total_active)
{
    int first_bad = OR_OK;
    long long it = 0, act = 0;
    or_step_info loc;
    memset(&loc, 0, sizeof(loc));
    for (long s = 0; s < n_steps; ++s) {
        double t = t_start + (double)s * dt;
        int st = or_step(P, d0, t, step0 + s, dt, h, hu, hw, q, NULL, &loc);
        it += loc.iters;
        act += loc.n_active;
        if (st != OR_OK && first_bad == OR_OK) first_bad = st;
    }
    if (info) *info = loc;
    if (total_iters) *total_iters = it;
    if (total_active) *total_active = act;
    return first_bad;
}
