/*
 * nh_oracle2d.c -- plain FP64 CPU oracle of the two-dimensional form of the
 * locally adaptive non-hydrostatic shallow-water method.  TEST
 * INFRASTRUCTURE ONLY: see nh_oracle2d.h.  One loop per formula, no fusion.
 *
 * ---------------------------------------------------------------------------
 * The two-dimensional equations (the paper's model is 1D, Sec. 2; its Sec. 6
 * names the 2D extension as future work).  With U = (hu, hv):
 *   h_t + div U = 0                                              (Eq. 1)
 *   U_t + div(U u) + g h grad(eta) = -(1/rho) grad(h p) + (p_b/rho) grad d
 *   (hw)_t + div(hw u) = p_b / rho
 *   2 hw + U . grad(2 d - h) + 2 h d_t = -h div U                (Eq. 4)
 * and the bottom pressure (Eq. 5 with d_x q_x -> grad d . grad q):
 *   P = p_b/rho scaled as in 1D: P = 6 q/(h D) + grad d . grad q / D + phi,
 *   D = 4 + G, G = |grad d|^2, q = h p,
 *   phi = rho h / D (g grad d . grad eta - d_tt - 2 u . grad d_t - u.(grad grad d) u).
 * Each term is the 1D term with x-derivatives replaced by gradients, so a
 * state and bottom independent of y reproduce the 1D oracle (tested).
 *
 * Projection (Eqs. 10-11), a = dt / rho:
 *   HU = U~ - a grad q + a grad d P = U0 - a M grad q + (6 a grad d/(h D)) q,
 *   U0 = U~ + a phi grad d,   M = I - grad d grad d^T / D,
 *   HW = hw~ + a P.
 * Constraint Eq. 4 at n+1 as h^2 div(HU/h) + 2 grad d . HU + 2 HW + 2 h d_t = 0,
 * divided by h^2.  The grad q terms outside the divergence are
 * (6 - 8 + 2) a grad d . grad q / (h^2 D) = 0 (grad d . M grad q =
 * (4/D) grad d . grad q), as in 1D, which leaves the self-adjoint equation
 *   -div(K grad q) + gamma q = R,
 *   K     = (a/h) M      (K_xx = (a/h)(1 - d_x^2/D), K_yy = (a/h)(1 - d_y^2/D),
 *                         K_xy = -(a/h) d_x d_y / D; in 1D K = 4a/(hD))
 *   beta  = 6 a grad d / (h^2 D)
 *   gamma = div beta + 12 a (1 + G) / (h^3 D)
 *   R     = -[ div(U0/h) + 2 grad d . U0 / h^2 + 2 hw~/h^2 + 2 a phi / h^2 + 2 d_t/h ].
 *
 * Discretisation: K_xx on x-faces and K_yy on y-faces as face averages of
 * the cell values (five-point part, as in 1D); the cross terms
 * -d_x(K_xy d_y q) - d_y(K_xy d_x q) by central differences of cell values,
 * which gives the four diagonal couplings
 *   NE: -(K_xy(E) + K_xy(N)) / (4 dx dy),  SW: -(K_xy(W) + K_xy(S)) / (4 dx dy),
 *   SE: +(K_xy(E) + K_xy(S)) / (4 dx dy),  NW: +(K_xy(W) + K_xy(N)) / (4 dx dy),
 * and a symmetric matrix (the NE coefficient of cell (i, j) equals the SW
 * coefficient of cell (i+1, j+1)).  div beta, div(U0/h), grad eta by central
 * differences.  q = 0 on inactive cells and outside walled sides.
 *
 * Ghost cells at a wall normal to x: every scalar mirrored; quantities odd in
 * x (u, hu, d_x, beta_x, U0_x/h, d_xy, K_xy) change sign.  Likewise in y.
 * ---------------------------------------------------------------------------
 */
#include "nh_oracle2d.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ----------------------------------------------------------------- ghosts */

/* In-domain index along one direction of n cells; *odd = -1 where a wall
   mirror flips quantities odd in that direction. */
static int ghost1(int bc, int n, int i, double* odd)
{
    *odd = 1.0;
    if (i >= 0 && i < n) return i;
    if (bc == OR_BC_PERIODIC) return ((i % n) + n) % n;
    *odd = -1.0;
    return (i < 0) ? (-1 - i) : (2 * n - 1 - i);
}

/* Flat in-domain index of cell (i, j) with the parities of the two mirrors. */
static int ghost2(const or2_params* P, int i, int j, double* ox, double* oy)
{
    int ci = ghost1(P->bcx, P->nx, i, ox);
    int cj = ghost1(P->bcy, P->ny, j, oy);
    return cj * P->nx + ci;
}

/* Flat index of the unknown at (i, j), or -1 outside a walled side. */
static int inner2(const or2_params* P, int i, int j)
{
    if (i < 0 || i >= P->nx) {
        if (P->bcx != OR_BC_PERIODIC) return -1;
        i = ((i % P->nx) + P->nx) % P->nx;
    }
    if (j < 0 || j >= P->ny) {
        if (P->bcy != OR_BC_PERIODIC) return -1;
        j = ((j % P->ny) + P->ny) % P->ny;
    }
    return j * P->nx + i;
}

/* ----------------------------------------------------------------- bottom */

static void slide_law2(const or2_params* P, double t, double* s, double* sd, double* sdd)
{
    double z = t / P->t0;
    *s = P->s0 * log(cosh(z));
    *sd = (P->s0 / P->t0) * tanh(z);
    *sdd = (P->s0 / (P->t0 * P->t0)) / (cosh(z) * cosh(z));
}

/* d = d0 - m, m = A exp(-xi^2 - zeta^2), xi = (x - xc0 - s(t))/Lx,
   zeta = (y - yc0)/Ly; d0's derivatives by central differences (mirrored or
   wrapped neighbours), the mound's analytically (chain rule, dxi/dt = -s'/Lx). */
void or2_bottom(const or2_params* P, const double* d0, int i, int j, double t, double out[10])
{
    double o1, o2;
    double dx = P->dx, dy = P->dy;
    double c = d0[j * P->nx + i];
    double xm = d0[ghost2(P, i - 1, j, &o1, &o2)], xp = d0[ghost2(P, i + 1, j, &o1, &o2)];
    double ym = d0[ghost2(P, i, j - 1, &o1, &o2)], yp = d0[ghost2(P, i, j + 1, &o1, &o2)];
    double mm = d0[ghost2(P, i - 1, j - 1, &o1, &o2)], pm = d0[ghost2(P, i + 1, j - 1, &o1, &o2)];
    double mp = d0[ghost2(P, i - 1, j + 1, &o1, &o2)], pp = d0[ghost2(P, i + 1, j + 1, &o1, &o2)];
    double d = c;
    double d_x = (xp - xm) / (2.0 * dx);
    double d_y = (yp - ym) / (2.0 * dy);
    double d_xx = (xp - 2.0 * c + xm) / (dx * dx);
    double d_yy = (yp - 2.0 * c + ym) / (dy * dy);
    double d_xy = (pp - pm - mp + mm) / (4.0 * dx * dy);
    double d_t = 0.0, d_xt = 0.0, d_yt = 0.0, d_tt = 0.0;
    if (P->slide == OR_SLIDE_GAUSS_LNCOSH) {
        double s, sd, sdd;
        slide_law2(P, t, &s, &sd, &sdd);
        double x = P->x0 + (i + 0.5) * dx, y = P->y0 + (j + 0.5) * dy;
        double Lx = P->Lx, Ly = P->Ly;
        double xi = (x - P->xc0 - s) / Lx, ze = (y - P->yc0) / Ly;
        double m = P->A * exp(-xi * xi - ze * ze);
        double m_x = m * (-2.0 * xi / Lx);
        double m_y = m * (-2.0 * ze / Ly);
        double m_xx = m * (4.0 * xi * xi - 2.0) / (Lx * Lx);
        double m_yy = m * (4.0 * ze * ze - 2.0) / (Ly * Ly);
        double m_xy = m * (4.0 * xi * ze) / (Lx * Ly);
        double m_t = m * (2.0 * xi / Lx) * sd;
        double m_xt = -m * (2.0 / (Lx * Lx)) * (2.0 * xi * xi - 1.0) * sd;
        double m_yt = -m * (4.0 * xi * ze / (Lx * Ly)) * sd;
        double m_tt = m * (2.0 / (Lx * Lx)) * ((2.0 * xi * xi - 1.0) * sd * sd + xi * Lx * sdd);
        d -= m; d_x -= m_x; d_y -= m_y; d_xx -= m_xx; d_yy -= m_yy; d_xy -= m_xy;
        d_t = -m_t; d_xt = -m_xt; d_yt = -m_yt; d_tt = -m_tt;
    }
    out[0] = d; out[1] = d_x; out[2] = d_y; out[3] = d_xx; out[4] = d_yy; out[5] = d_xy;
    out[6] = d_t; out[7] = d_xt; out[8] = d_yt; out[9] = d_tt;
}

static double depth2(const or2_params* P, const double* d0, int i, int j, double t)
{
    double b[10];
    or2_bottom(P, d0, i, j, t, b);
    return b[0];
}

/* -------------------------------------------------------------- predictor */

static double minmod2d(double a, double b)
{
    if (a * b <= 0.0) return 0.0;
    return (fabs(a) < fabs(b)) ? a : b;
}

static double slope2(int limiter, double vm, double v0, double vp)
{
    switch (limiter) {
    case OR_LIM_CENTRAL: return 0.5 * (vp - vm);
    case OR_LIM_MINMOD:  return minmod2d(vp - v0, v0 - vm);
    case OR_LIM_MC:      return minmod2d(0.5 * (vp - vm), minmod2d(2.0 * (vp - v0), 2.0 * (v0 - vm)));
    default:             return 0.0;
    }
}

/* Rusanov flux normal to a face, (hun, hun un + g h^2/2, hun ut, hun w), from
   left / right states (h, un, ut, w): un the normal and ut the tangential
   velocity.  The same flux as the 1D oracle's, with the tangential momentum
   carried like w. */
static void rusanov2(double g, double hL, double nL, double tL, double wL,
                     double hR, double nR, double tR, double wR, double F[4])
{
    double FL0 = hL * nL, FL1 = hL * nL * nL + 0.5 * g * hL * hL, FL2 = hL * nL * tL, FL3 = hL * nL * wL;
    double FR0 = hR * nR, FR1 = hR * nR * nR + 0.5 * g * hR * hR, FR2 = hR * nR * tR, FR3 = hR * nR * wR;
    double sL = fabs(nL) + sqrt(g * hL), sR = fabs(nR) + sqrt(g * hR);
    double s = (sL > sR) ? sL : sR;
    F[0] = 0.5 * (FL0 + FR0) - 0.5 * s * (hR - hL);
    F[1] = 0.5 * (FL1 + FR1) - 0.5 * s * (hR * nR - hL * nL);
    F[2] = 0.5 * (FL2 + FR2) - 0.5 * s * (hR * tR - hL * tL);
    F[3] = 0.5 * (FL3 + FR3) - 0.5 * s * (hR * wR - hL * wL);
}

/* One direction's flux divergence and bottom source, added into r*.  dir 0:
   x (faces between (i-1, j) and (i, j)), dir 1: y.  The same MUSCL
   reconstruction of eta, the normal and tangential velocities and w, with
   the depth continuous at faces, as the 1D oracle's or_rhs. */
static void rhs_dir(const or2_params* P, const double* d0, double t, int dir,
                    const double* h, const double* hu, const double* hv, const double* hw,
                    double* rh, double* rhu, double* rhv, double* rhw)
{
    int nx = P->nx, ny = P->ny;
    int n = dir == 0 ? nx : ny;         /* cells along the line */
    int lines = dir == 0 ? ny : nx;
    double ds = dir == 0 ? P->dx : P->dy, g = P->g;
    double* eta = malloc(sizeof(double) * (n + 4));
    double* un = malloc(sizeof(double) * (n + 4));
    double* ut = malloc(sizeof(double) * (n + 4));
    double* w = malloc(sizeof(double) * (n + 4));
    double* d = malloc(sizeof(double) * (n + 4));
    double* se = malloc(sizeof(double) * (n + 4));
    double* sn = malloc(sizeof(double) * (n + 4));
    double* st = malloc(sizeof(double) * (n + 4));
    double* sw = malloc(sizeof(double) * (n + 4));
    double* df = malloc(sizeof(double) * (n + 1));
    double (*F)[4] = malloc(sizeof(double[4]) * (n + 1));
    for (int l = 0; l < lines; ++l) {
        for (int m = -2; m < n + 2; ++m) {
            double ox, oy;
            int i = dir == 0 ? m : l, j = dir == 0 ? l : m;
            int c = ghost2(P, i, j, &ox, &oy);
            int ci = c % nx, cj = c / nx;
            double dc = depth2(P, d0, ci, cj, t);
            d[m + 2] = dc;
            eta[m + 2] = h[c] - dc;
            double u = ox * hu[c] / h[c], v = oy * hv[c] / h[c];
            un[m + 2] = dir == 0 ? u : v;
            ut[m + 2] = dir == 0 ? v : u;
            w[m + 2] = hw[c] / h[c];
        }
        for (int m = -1; m < n + 1; ++m) {
            se[m + 2] = slope2(P->limiter, eta[m + 1], eta[m + 2], eta[m + 3]);
            sn[m + 2] = slope2(P->limiter, un[m + 1], un[m + 2], un[m + 3]);
            st[m + 2] = slope2(P->limiter, ut[m + 1], ut[m + 2], ut[m + 3]);
            sw[m + 2] = slope2(P->limiter, w[m + 1], w[m + 2], w[m + 3]);
        }
        for (int k = 0; k <= n; ++k) {
            int L = k - 1, Rr = k;
            df[k] = 0.5 * (d[L + 2] + d[Rr + 2]);
            double hL = eta[L + 2] + 0.5 * se[L + 2] + df[k];
            double hR = eta[Rr + 2] - 0.5 * se[Rr + 2] + df[k];
            rusanov2(g, hL, un[L + 2] + 0.5 * sn[L + 2], ut[L + 2] + 0.5 * st[L + 2], w[L + 2] + 0.5 * sw[L + 2],
                     hR, un[Rr + 2] - 0.5 * sn[Rr + 2], ut[Rr + 2] - 0.5 * st[Rr + 2], w[Rr + 2] - 0.5 * sw[Rr + 2],
                     F[k]);
        }
        for (int m = 0; m < n; ++m) {
            int i = dir == 0 ? m : l, j = dir == 0 ? l : m;
            int c = j * nx + i;
            double hplus = eta[m + 2] - 0.5 * se[m + 2] + df[m];
            double hminus = eta[m + 2] + 0.5 * se[m + 2] + df[m + 1];
            double S = g * 0.5 * (hplus + hminus) * (df[m + 1] - df[m]) / ds;
            rh[c] += -(F[m + 1][0] - F[m][0]) / ds;
            double rn = -(F[m + 1][1] - F[m][1]) / ds + S;
            double rt = -(F[m + 1][2] - F[m][2]) / ds;
            if (dir == 0) { rhu[c] += rn; rhv[c] += rt; }
            else          { rhv[c] += rn; rhu[c] += rt; }
            rhw[c] += -(F[m + 1][3] - F[m][3]) / ds;
        }
    }
    free(eta); free(un); free(ut); free(w); free(d); free(se); free(sn); free(st); free(sw);
    free(df); free(F);
}

/* H(Q) of the hydrostatic equations: the x and the y flux divergences and
   bottom sources added. */
void or2_rhs(const or2_params* P, const double* d0, double t,
             const double* h, const double* hu, const double* hv, const double* hw,
             double* rh, double* rhu, double* rhv, double* rhw)
{
    int N = P->nx * P->ny;
    for (int k = 0; k < N; ++k) { rh[k] = 0.0; rhu[k] = 0.0; rhv[k] = 0.0; rhw[k] = 0.0; }
    rhs_dir(P, d0, t, 0, h, hu, hv, hw, rh, rhu, rhv, rhw);
    rhs_dir(P, d0, t, 1, h, hu, hv, hw, rh, rhu, rhv, rhw);
}

/* Heun (Eqs. 8-9), as in 1D. */
void or2_predict(const or2_params* P, const double* d0, double t, double dt,
                 const double* h, const double* hu, const double* hv, const double* hw,
                 double* ht, double* hut, double* hvt, double* hwt)
{
    int N = P->nx * P->ny;
    double* k1 = malloc(sizeof(double) * 4 * N);
    double* k2 = malloc(sizeof(double) * 4 * N);
    double* s = malloc(sizeof(double) * 4 * N);
    or2_rhs(P, d0, t, h, hu, hv, hw, k1, k1 + N, k1 + 2 * N, k1 + 3 * N);
    for (int k = 0; k < N; ++k) {
        s[k] = h[k] + dt * k1[k];
        s[N + k] = hu[k] + dt * k1[N + k];
        s[2 * N + k] = hv[k] + dt * k1[2 * N + k];
        s[3 * N + k] = hw[k] + dt * k1[3 * N + k];
    }
    or2_rhs(P, d0, t + dt, s, s + N, s + 2 * N, s + 3 * N, k2, k2 + N, k2 + 2 * N, k2 + 3 * N);
    for (int k = 0; k < N; ++k) {
        ht[k] = h[k] + 0.5 * dt * (k1[k] + k2[k]);
        hut[k] = hu[k] + 0.5 * dt * (k1[N + k] + k2[N + k]);
        hvt[k] = hv[k] + 0.5 * dt * (k1[2 * N + k] + k2[2 * N + k]);
        hwt[k] = hw[k] + 0.5 * dt * (k1[3 * N + k] + k2[3 * N + k]);
    }
    free(k1); free(k2); free(s);
}

/* ---------------------------------------------------------- criterion, mask */

/* Sec. 5.1 in 2D: |eta/d|, |grad eta|, |u| (speed), |grad u| (Frobenius norm
   of the velocity gradient), |w|, |grad w|; central differences.  With no y
   dependence (v = 0) each reduces to the 1D criterion. */
void or2_criterion(const or2_params* P, const double* d0, double t,
                   const double* ht, const double* hut, const double* hvt, const double* hwt,
                   double* c)
{
    int nx = P->nx, ny = P->ny;
    double dx = P->dx, dy = P->dy;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            double o[4][2];
            int nb[4] = {ghost2(P, i - 1, j, &o[0][0], &o[0][1]), ghost2(P, i + 1, j, &o[1][0], &o[1][1]),
                         ghost2(P, i, j - 1, &o[2][0], &o[2][1]), ghost2(P, i, j + 1, &o[3][0], &o[3][1])};
            double eta[4], u[4], v[4], w[4];
            for (int q = 0; q < 4; ++q) {
                int m = nb[q];
                eta[q] = ht[m] - depth2(P, d0, m % nx, m / nx, t);
                u[q] = o[q][0] * hut[m] / ht[m];
                v[q] = o[q][1] * hvt[m] / ht[m];
                w[q] = hwt[m] / ht[m];
            }
            double dk = depth2(P, d0, i, j, t);
            double eta_k = ht[k] - dk, uk = hut[k] / ht[k], vk = hvt[k] / ht[k], wk = hwt[k] / ht[k];
            double ex = (eta[1] - eta[0]) / (2.0 * dx), ey = (eta[3] - eta[2]) / (2.0 * dy);
            double ux = (u[1] - u[0]) / (2.0 * dx), uy = (u[3] - u[2]) / (2.0 * dy);
            double vx = (v[1] - v[0]) / (2.0 * dx), vy = (v[3] - v[2]) / (2.0 * dy);
            double wx = (w[1] - w[0]) / (2.0 * dx), wy = (w[3] - w[2]) / (2.0 * dy);
            double val;
            switch (P->crit) {
            case OR_CRIT_ETA_D: val = fabs(eta_k / dk); break;
            case OR_CRIT_ETA_X: val = sqrt(ex * ex + ey * ey); break;
            case OR_CRIT_U:     val = sqrt(uk * uk + vk * vk); break;
            case OR_CRIT_U_X:   val = sqrt(ux * ux + uy * uy + vx * vx + vy * vy); break;
            case OR_CRIT_W:     val = fabs(wk); break;
            case OR_CRIT_W_X:   val = sqrt(wx * wx + wy * wy); break;
            default:            val = 0.0; break;
            }
            c[k] = val;
        }
}

/* Marked cells (Sec. 5.1; all cells on the first step with
   first_step_global, Sec. 5.1.2), enlarged to the Moore neighbourhood of
   radius `enlarge` (the 2D form of Sec. 5.2's one cell on each side). */
int or2_mask(const or2_params* P, const double* d0, double t, long step,
             const double* ht, const double* hut, const double* hvt, const double* hwt,
             unsigned char* mask)
{
    int nx = P->nx, ny = P->ny, N = nx * ny;
    unsigned char* marked = malloc(N);
    if (P->crit == OR_CRIT_GLOBAL || (P->first_step_global && step == 0)) {
        for (int k = 0; k < N; ++k) marked[k] = 1;
    } else if (P->crit == OR_CRIT_HYDROSTATIC) {
        for (int k = 0; k < N; ++k) marked[k] = 0;
    } else {
        double* c = malloc(sizeof(double) * N);
        or2_criterion(P, d0, t, ht, hut, hvt, hwt, c);
        for (int k = 0; k < N; ++k) marked[k] = (c[k] > P->knh) ? 1 : 0;
        free(c);
    }
    int count = 0, e = P->enlarge;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            unsigned char m = 0;
            for (int b = -e; b <= e && !m; ++b)
                for (int a = -e; a <= e; ++a) {
                    int q = inner2(P, i + a, j + b);
                    if (q >= 0 && marked[q]) { m = 1; break; }
                }
            mask[j * nx + i] = m;
            count += m;
        }
    free(marked);
    return count;
}

/* --------------------------------------------------------------- assembly */

/* Per-cell quantities of the elliptic equation (see the header comment). */
typedef struct {
    double h, Kxx, Kyy, Kxy, bx, by, Vx, Vy, U0, V0, phi, d_x, d_y, d_t, G, D;
} cellq2;

static cellq2 cell_q2(const or2_params* P, const double* d0, double t1, double a,
                      const double* ht, const double* hut, const double* hvt, int i, int j)
{
    int nx = P->nx;
    double b[10], o1, o2;
    or2_bottom(P, d0, i, j, t1, b);
    int kw = ghost2(P, i - 1, j, &o1, &o2), ke = ghost2(P, i + 1, j, &o1, &o2);
    int ks = ghost2(P, i, j - 1, &o1, &o2), kn = ghost2(P, i, j + 1, &o1, &o2);
    double eta_x = ((ht[ke] - depth2(P, d0, ke % nx, ke / nx, t1)) - (ht[kw] - depth2(P, d0, kw % nx, kw / nx, t1)))
                   / (2.0 * P->dx);
    double eta_y = ((ht[kn] - depth2(P, d0, kn % nx, kn / nx, t1)) - (ht[ks] - depth2(P, d0, ks % nx, ks / nx, t1)))
                   / (2.0 * P->dy);
    int k = j * nx + i;
    cellq2 q;
    q.h = ht[k];
    double u = hut[k] / q.h, v = hvt[k] / q.h;
    q.d_x = b[1]; q.d_y = b[2]; q.d_t = b[6];
    double d_xx = b[3], d_yy = b[4], d_xy = b[5], d_xt = b[7], d_yt = b[8], d_tt = b[9];
    q.G = q.d_x * q.d_x + q.d_y * q.d_y;
    q.D = 4.0 + q.G;
    q.phi = P->rho * q.h / q.D * (P->g * (q.d_x * eta_x + q.d_y * eta_y) - d_tt
                                  - 2.0 * (u * d_xt + v * d_yt)
                                  - (u * u * d_xx + 2.0 * u * v * d_xy + v * v * d_yy));
    q.Kxx = a / q.h * (1.0 - q.d_x * q.d_x / q.D);
    q.Kyy = a / q.h * (1.0 - q.d_y * q.d_y / q.D);
    q.Kxy = -a / q.h * q.d_x * q.d_y / q.D;
    q.bx = 6.0 * a * q.d_x / (q.h * q.h * q.D);
    q.by = 6.0 * a * q.d_y / (q.h * q.h * q.D);
    q.U0 = hut[k] + a * q.phi * q.d_x;
    q.V0 = hvt[k] + a * q.phi * q.d_y;
    q.Vx = q.U0 / q.h;
    q.Vy = q.V0 / q.h;
    return q;
}

/* Quantities of cell (i, j) seen from a neighbour: in-domain or mirrored (odd
   components flipped). */
static cellq2 cell_q2_at(const or2_params* P, const double* d0, double t1, double a,
                         const double* ht, const double* hut, const double* hvt, int i, int j)
{
    double ox, oy;
    int c = ghost2(P, i, j, &ox, &oy);
    cellq2 q = cell_q2(P, d0, t1, a, ht, hut, hvt, c % P->nx, c / P->nx);
    q.Kxy *= ox * oy;
    q.bx *= ox; q.by *= oy;
    q.Vx *= ox; q.Vy *= oy;
    return q;
}

void or2_assemble(const or2_params* P, const double* d0, double t1, double dt,
                  const double* ht, const double* hut, const double* hvt, const double* hwt,
                  double* coef, double* gam, double* R)
{
    int nx = P->nx, ny = P->ny, N = nx * ny;
    double a = dt / P->rho, dx = P->dx, dy = P->dy;
    double idx2 = 1.0 / (dx * dx), idy2 = 1.0 / (dy * dy), ixy = 1.0 / (4.0 * dx * dy);
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            cellq2 c = cell_q2(P, d0, t1, a, ht, hut, hvt, i, j);
            cellq2 W = cell_q2_at(P, d0, t1, a, ht, hut, hvt, i - 1, j);
            cellq2 E = cell_q2_at(P, d0, t1, a, ht, hut, hvt, i + 1, j);
            cellq2 S = cell_q2_at(P, d0, t1, a, ht, hut, hvt, i, j - 1);
            cellq2 Nn = cell_q2_at(P, d0, t1, a, ht, hut, hvt, i, j + 1);
            double Kw = 0.5 * (W.Kxx + c.Kxx), Ke = 0.5 * (c.Kxx + E.Kxx);
            double Ks = 0.5 * (S.Kyy + c.Kyy), Kn = 0.5 * (c.Kyy + Nn.Kyy);
            double div_beta = (E.bx - W.bx) / (2.0 * dx) + (Nn.by - S.by) / (2.0 * dy);
            double div_V = (E.Vx - W.Vx) / (2.0 * dx) + (Nn.Vy - S.Vy) / (2.0 * dy);
            double h = c.h, h2 = h * h;
            gam[k] = div_beta + 12.0 * a * (1.0 + c.G) / (h2 * h * c.D);
            R[k] = -(div_V + 2.0 * (c.d_x * c.U0 + c.d_y * c.V0) / h2 + 2.0 * hwt[k] / h2
                     + 2.0 * a * c.phi / h2 + 2.0 * c.d_t / h);
            coef[OR2_C * N + k] = (Kw + Ke) * idx2 + (Ks + Kn) * idy2 + gam[k];
            coef[OR2_W * N + k] = -Kw * idx2;
            coef[OR2_E * N + k] = -Ke * idx2;
            coef[OR2_S * N + k] = -Ks * idy2;
            coef[OR2_N * N + k] = -Kn * idy2;
            coef[OR2_NE * N + k] = -(E.Kxy + Nn.Kxy) * ixy;
            coef[OR2_SW * N + k] = -(W.Kxy + S.Kxy) * ixy;
            coef[OR2_SE * N + k] = (E.Kxy + S.Kxy) * ixy;
            coef[OR2_NW * N + k] = (W.Kxy + Nn.Kxy) * ixy;
        }
}

/* Neighbour offsets of the coefficients OR2_W .. OR2_NE. */
static const int nb_di[OR2_NCOEF] = {0, -1, 1, 0, 0, -1, 1, -1, 1};
static const int nb_dj[OR2_NCOEF] = {0, 0, 0, -1, 1, -1, -1, 1, 1};

/* (A x)_k = sum over the 9-point row, x = 0 on inactive cells and outside
   walled sides. */
void or2_apply(const or2_params* P, const unsigned char* mask, const double* coef,
               const double* x, double* y)
{
    int nx = P->nx, ny = P->ny, N = nx * ny;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            if (!mask[k]) { y[k] = 0.0; continue; }
            double s = coef[OR2_C * N + k] * x[k];
            for (int m = 1; m < OR2_NCOEF; ++m) {
                int q = inner2(P, i + nb_di[m], j + nb_dj[m]);
                if (q >= 0 && mask[q]) s += coef[m * N + k] * x[q];
            }
            y[k] = s;
        }
}

/* ----------------------------------------------------------------- solvers */

static double dot2(int n, const unsigned char* mask, const double* a, const double* b)
{
    double s = 0.0;
    for (int i = 0; i < n; ++i)
        if (mask[i]) s += a[i] * b[i];
    return s;
}

/* Conjugate gradients (Hestenes-Stiefel), as in 1D. */
static int cg2(const or2_params* P, const unsigned char* mask, const double* coef,
               const double* R, double* x, or_step_info* info)
{
    int n = P->nx * P->ny;
    double* r = calloc(n, sizeof(double));
    double* p = calloc(n, sizeof(double));
    double* Ap = calloc(n, sizeof(double));
    for (int i = 0; i < n; ++i) if (!mask[i]) x[i] = 0.0;
    or2_apply(P, mask, coef, x, Ap);
    for (int i = 0; i < n; ++i) r[i] = mask[i] ? R[i] - Ap[i] : 0.0;
    double bnorm = sqrt(dot2(n, mask, R, R));
    double rr = dot2(n, mask, r, r);
    int it = 0, status = OR_NOT_CONVERGED;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        rr = 0.0; bnorm = 1.0; status = OR_OK;
    } else if (sqrt(rr) <= P->rtol * bnorm) {
        status = OR_OK;
    } else {
        for (int i = 0; i < n; ++i) p[i] = r[i];
        for (it = 1; it <= P->max_iter; ++it) {
            or2_apply(P, mask, coef, p, Ap);
            double alpha = rr / dot2(n, mask, p, Ap);
            for (int i = 0; i < n; ++i) if (mask[i]) { x[i] += alpha * p[i]; r[i] -= alpha * Ap[i]; }
            double rr_new = dot2(n, mask, r, r);
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

/* BiCGStab (van der Vorst 1992), as in 1D. */
static int bicgstab2(const or2_params* P, const unsigned char* mask, const double* coef,
                     const double* R, double* x, or_step_info* info)
{
    int n = P->nx * P->ny;
    double* r = calloc(n, sizeof(double));
    double* rh = calloc(n, sizeof(double));
    double* p = calloc(n, sizeof(double));
    double* v = calloc(n, sizeof(double));
    double* s = calloc(n, sizeof(double));
    double* tt = calloc(n, sizeof(double));
    for (int i = 0; i < n; ++i) if (!mask[i]) x[i] = 0.0;
    or2_apply(P, mask, coef, x, v);
    for (int i = 0; i < n; ++i) { r[i] = mask[i] ? R[i] - v[i] : 0.0; rh[i] = r[i]; v[i] = 0.0; }
    double bnorm = sqrt(dot2(n, mask, R, R));
    double rnorm = sqrt(dot2(n, mask, r, r));
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    int it = 0, status = OR_NOT_CONVERGED;
    if (bnorm == 0.0) {
        for (int i = 0; i < n; ++i) x[i] = 0.0;
        rnorm = 0.0; bnorm = 1.0; status = OR_OK;
    } else if (rnorm <= P->rtol * bnorm) {
        status = OR_OK;
    } else {
        for (it = 1; it <= P->max_iter; ++it) {
            double rho = dot2(n, mask, rh, r);
            double beta = (rho / rho_old) * (alpha / omega);
            for (int i = 0; i < n; ++i) if (mask[i]) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            or2_apply(P, mask, coef, p, v);
            alpha = rho / dot2(n, mask, rh, v);
            for (int i = 0; i < n; ++i) if (mask[i]) s[i] = r[i] - alpha * v[i];
            double snorm = sqrt(dot2(n, mask, s, s));
            if (snorm <= P->rtol * bnorm) {
                for (int i = 0; i < n; ++i) if (mask[i]) x[i] += alpha * p[i];
                rnorm = snorm; status = OR_OK; break;
            }
            or2_apply(P, mask, coef, s, tt);
            omega = dot2(n, mask, tt, s) / dot2(n, mask, tt, tt);
            for (int i = 0; i < n; ++i) if (mask[i]) {
                x[i] += alpha * p[i] + omega * s[i];
                r[i] = s[i] - omega * tt[i];
            }
            rnorm = sqrt(dot2(n, mask, r, r));
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
   (tiny grids only); column l is A applied to the l-th active unit vector. */
static int dense2(const or2_params* P, const unsigned char* mask, const double* coef,
                  const double* R, double* x, or_step_info* info)
{
    int n = P->nx * P->ny, m = 0;
    int* idx = malloc(sizeof(int) * n);
    for (int i = 0; i < n; ++i) if (mask[i]) idx[m++] = i;
    double* M = calloc((size_t)m * m, sizeof(double));
    double* b = malloc(sizeof(double) * (m > 0 ? m : 1));
    double* e = calloc(n, sizeof(double));
    double* col = calloc(n, sizeof(double));
    for (int l = 0; l < m; ++l) {
        e[idx[l]] = 1.0;
        or2_apply(P, mask, coef, e, col);
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

int or2_solve(const or2_params* P, const unsigned char* mask, const double* coef,
              const double* gam, const double* R, double* q, or_step_info* info)
{
    int n = P->nx * P->ny;
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
    if (kind == OR_SOLVER_CG) return cg2(P, mask, coef, R, q, info);
    if (kind == OR_SOLVER_BICGSTAB) return bicgstab2(P, mask, coef, R, q, info);
    if (kind == OR_SOLVER_DENSE) return dense2(P, mask, coef, R, q, info);
    return OR_BAD_ARG;
}

/* -------------------------------------------------------------- correction */

/* Eqs. 10-11 in 2D: U = U~ + a (-grad q + grad d P), hw = hw~ + a P,
   P = 6 q/(h D) + grad d . grad q / D + phi; grad q central with q = 0 off
   the mask and outside walled sides; h = h~ (Sec. 3.2). */
void or2_correct(const or2_params* P, const double* d0, double t1, double dt,
                 const unsigned char* mask, const double* q,
                 const double* ht, const double* hut, const double* hvt, const double* hwt,
                 double* h, double* hu, double* hv, double* hw)
{
    int nx = P->nx, ny = P->ny;
    double a = dt / P->rho;
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            h[k] = ht[k]; hu[k] = hut[k]; hv[k] = hvt[k]; hw[k] = hwt[k];
            if (!mask[k]) continue;
            cellq2 c = cell_q2(P, d0, t1, a, ht, hut, hvt, i, j);
            int w = inner2(P, i - 1, j), e = inner2(P, i + 1, j);
            int s = inner2(P, i, j - 1), n = inner2(P, i, j + 1);
            double qw = (w >= 0 && mask[w]) ? q[w] : 0.0, qe = (e >= 0 && mask[e]) ? q[e] : 0.0;
            double qs = (s >= 0 && mask[s]) ? q[s] : 0.0, qn = (n >= 0 && mask[n]) ? q[n] : 0.0;
            double q_x = (qe - qw) / (2.0 * P->dx), q_y = (qn - qs) / (2.0 * P->dy);
            double Pb = 6.0 * q[k] / (c.h * c.D) + (c.d_x * q_x + c.d_y * q_y) / c.D + c.phi;
            hu[k] = hut[k] + a * (-q_x + c.d_x * Pb);
            hv[k] = hvt[k] + a * (-q_y + c.d_y * Pb);
            hw[k] = hwt[k] + a * Pb;
        }
}

/* -------------------------------------------------------------------- step */

int or2_step(const or2_params* P, const double* d0, double t, long step, double dt,
             double* h, double* hu, double* hv, double* hw, double* q, unsigned char* mask,
             or_step_info* info)
{
    int N = P->nx * P->ny;
    if (P->nx < 3 || P->ny < 3 || !(P->dx > 0.0) || !(P->dy > 0.0) || !(dt > 0.0)) return OR_BAD_ARG;
    double* ht = malloc(sizeof(double) * N);
    double* hut = malloc(sizeof(double) * N);
    double* hvt = malloc(sizeof(double) * N);
    double* hwt = malloc(sizeof(double) * N);
    double* coef = malloc(sizeof(double) * OR2_NCOEF * N);
    double* gam = malloc(sizeof(double) * N);
    double* R = malloc(sizeof(double) * N);
    unsigned char* m = malloc(N);
    or_step_info loc;
    memset(&loc, 0, sizeof(loc));
    loc.solver_used = -1;
    double t1 = t + dt;

    or2_predict(P, d0, t, dt, h, hu, hv, hw, ht, hut, hvt, hwt);
    int na = or2_mask(P, d0, t1, step, ht, hut, hvt, hwt, m);
    int status = OR_OK;
    if (na > 0) {
        or2_assemble(P, d0, t1, dt, ht, hut, hvt, hwt, coef, gam, R);
        if (P->guess == OR_GUESS_ZERO)
            for (int k = 0; k < N; ++k) q[k] = 0.0;
        for (int k = 0; k < N; ++k) if (!m[k]) q[k] = 0.0;
        status = or2_solve(P, m, coef, gam, R, q, &loc);
        or2_correct(P, d0, t1, dt, m, q, ht, hut, hvt, hwt, h, hu, hv, hw);
    } else {
        for (int k = 0; k < N; ++k) { h[k] = ht[k]; hu[k] = hut[k]; hv[k] = hvt[k]; hw[k] = hwt[k]; q[k] = 0.0; }
        loc.min_gamma = 0.0;
    }
    loc.n_active = na;
    loc.status = status;
    if (mask) memcpy(mask, m, N);
    if (info) *info = loc;
    free(ht); free(hut); free(hvt); free(hwt); free(coef); free(gam); free(R); free(m);
    return status;
}

int or2_run(const or2_params* P, const double* d0, double t_start, long step0,
            double dt, long n_steps, double* h, double* hu, double* hv, double* hw, double* q,
            or_step_info* info, long long* total_iters, long long* total_active)
{
    int first_bad = OR_OK;
    long long it = 0, act = 0;
    or_step_info loc;
    memset(&loc, 0, sizeof(loc));
    for (long s = 0; s < n_steps; ++s) {
        int st = or2_step(P, d0, t_start + (double)s * dt, step0 + s, dt, h, hu, hv, hw, q, NULL, &loc);
        it += loc.iters;
        act += loc.n_active;
        if (st != OR_OK && first_bad == OR_OK) first_bad = st;
    }
    if (info) *info = loc;
    if (total_iters) *total_iters = it;
    if (total_active) *total_active = act;
    return first_bad;
}
