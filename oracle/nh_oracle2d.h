/*
 * nh_oracle2d.h -- plain FP64 CPU oracle of the two-dimensional form of the
 * method.  TEST INFRASTRUCTURE ONLY (see nh_oracle.h): only the tests, the
 * smoke check and the benchmark's CPU baseline may call it; it shares no
 * code with the CUDA library.
 *
 * The paper's model is one-dimensional (Sec. 2) and names the 2D extension as
 * future work (Sec. 6).  This oracle generalises Eqs. 1-5 and 10-11 to two
 * horizontal dimensions in the way that reduces exactly to the 1D oracle for
 * a state and bottom that do not depend on y (tested), as derived in
 * nh_oracle2d.c.
 *
 * Layout: cell (i, j), 0 <= i < nx (x fastest), 0 <= j < ny, at k = j nx + i.
 */
#ifndef NH_ORACLE2D_H
#define NH_ORACLE2D_H

#include "nh_oracle.h"

typedef struct {
    int nx, ny;
    int bcx, bcy;             /* OR_BC_WALL or OR_BC_PERIODIC per direction */
    double dx, dy, x0, y0;    /* cell (i, j) centre: (x0 + (i + 1/2) dx, y0 + (j + 1/2) dy) */
    double g, rho;
    int limiter;
    int slide;                /* OR_SLIDE_NONE or OR_SLIDE_GAUSS_LNCOSH */
    double A, Lx, Ly, xc0, yc0, s0, t0;   /* mound A exp(-xi^2 - zeta^2), xi = (x - xc0 - s(t))/Lx,
                                             zeta = (y - yc0)/Ly, s = s0 ln cosh(t/t0) */
    int crit;                 /* OR_CRIT_*; 2D meaning in nh_oracle2d.c */
    double knh;
    int enlarge;              /* Moore neighbourhood of this radius */
    int first_step_global;
    int solver;               /* OR_SOLVER_* */
    double rtol;
    int max_iter;
    int guess;                /* OR_GUESS_* */
} or2_params;

/* 9-point operator rows: for every cell, the coefficient on itself (c[0]) and
   on its neighbours (c[1..8] = W, E, S, N, SW, SE, NW, NE). */
enum { OR2_C, OR2_W, OR2_E, OR2_S, OR2_N, OR2_SW, OR2_SE, OR2_NW, OR2_NE, OR2_NCOEF };

/* d, d_x, d_y, d_xx, d_yy, d_xy, d_t, d_xt, d_yt, d_tt at cell (i, j), time t. */
void or2_bottom(const or2_params* P, const double* d0, int i, int j, double t, double out[10]);

void or2_rhs(const or2_params* P, const double* d0, double t,
             const double* h, const double* hu, const double* hv, const double* hw,
             double* rh, double* rhu, double* rhv, double* rhw);

void or2_predict(const or2_params* P, const double* d0, double t, double dt,
                 const double* h, const double* hu, const double* hv, const double* hw,
                 double* ht, double* hut, double* hvt, double* hwt);

void or2_criterion(const or2_params* P, const double* d0, double t,
                   const double* ht, const double* hut, const double* hvt, const double* hwt,
                   double* c);

int or2_mask(const or2_params* P, const double* d0, double t, long step,
             const double* ht, const double* hut, const double* hvt, const double* hwt,
             unsigned char* mask);

/* coef: OR2_NCOEF arrays of nx*ny (row of cell k in coef[m][k]); gam, R: nx*ny. */
void or2_assemble(const or2_params* P, const double* d0, double t1, double dt,
                  const double* ht, const double* hut, const double* hvt, const double* hwt,
                  double* coef, double* gam, double* R);

void or2_apply(const or2_params* P, const unsigned char* mask, const double* coef,
               const double* x, double* y);

int or2_solve(const or2_params* P, const unsigned char* mask, const double* coef,
              const double* gam, const double* R, double* q, or_step_info* info);

void or2_correct(const or2_params* P, const double* d0, double t1, double dt,
                 const unsigned char* mask, const double* q,
                 const double* ht, const double* hut, const double* hvt, const double* hwt,
                 double* h, double* hu, double* hv, double* hw);

int or2_step(const or2_params* P, const double* d0, double t, long step, double dt,
             double* h, double* hu, double* hv, double* hw, double* q, unsigned char* mask,
             or_step_info* info);

int or2_run(const or2_params* P, const double* d0, double t_start, long step0,
            double dt, long n_steps, double* h, double* hu, double* hv, double* hw, double* q,
            or_step_info* info, long long* total_iters, long long* total_active);

#endif
