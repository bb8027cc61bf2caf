/*
 * nh_oracle.h -- plain FP64 CPU oracle of the locally adaptive non-hydrostatic
 * shallow-water method (Firdaus & Behrens, "Locally Adaptive Non-Hydrostatic
 * Shallow Water Extension for Moving Bottom-Generated Waves").
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * definition that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no source, header, helper or table with the CUDA library.
 *
 * Model (Sec. 2, Eqs. 1-5): unknowns h, hu, hw; fluid depth d(x,t) (bottom at
 * z = -d); thickness h = eta + d; quadratic non-hydrostatic pressure relation.
 * Method per step (Sec. 3): hydrostatic predictor (Sec. 3.1), criterion and
 * mask (Sec. 5.1, enlargement Sec. 5.2), elliptic solve on the masked cells,
 * correction of hu and hw (Sec. 3.2, Eqs. 10-11; h is not corrected).
 *
 * The discretisation is cell-centred finite volume (the paper's DG/LDG form is
 * replaced); the elliptic problem is Eqs. 10-11 + constraint Eq. 4 eliminated to
 * a symmetric scalar equation for q = h~ p^nh (derivation in the .c file).
 *
 * Parity pins (what fixes this code other than itself) live in tests/: the
 * Green-Naghdi solitary wave (Eq. 18), linear dispersion, lake at rest, mass
 * conservation, empty/full mask limits, dense LU on tiny grids, and
 * second-order consistency of the corrected state with Eqs. 4, 11, 12 and 13.
 */
#ifndef NH_ORACLE_H
#define NH_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { OR_BC_WALL = 0, OR_BC_PERIODIC = 1 };
enum { OR_LIM_NONE = 0, OR_LIM_CENTRAL = 1, OR_LIM_MINMOD = 2, OR_LIM_MC = 3 };
/* Bottom motions d(x,t) = d0(x) - m(x,t):
   OR_SLIDE_GAUSS_LNCOSH  m = A exp(-((x - xc0 - s)/L)^2), s = s0 ln cosh(t/t0)
                          (the moving-mound workloads);
   OR_SLIDE_PLATE_EXP     m = A (1 - exp(-t/t0)) for |x - xc0| < L, else 0
                          (the impulsive plate of Sec. 4.2: zeta0 = A, b = L,
                          alpha = 1/t0);
   OR_SLIDE_QUARTIC       m = A (1 - xi^4) for |xi| < 1, xi = 2 (x - xc0 - S(t))/L,
                          else 0, with the piecewise-quadratic law S(t) of the
                          sliding block of Sec. 4.3: acceleration a0 = s0 up to
                          t1 = t0, glide at ut = a0 t1 up to t2, deceleration
                          -a0 up to t3 = t2 + t1, at rest after. */
enum { OR_SLIDE_NONE = 0, OR_SLIDE_GAUSS_LNCOSH = 1, OR_SLIDE_PLATE_EXP = 2, OR_SLIDE_QUARTIC = 3 };
/* Sec. 5.1 criteria; GLOBAL = whole domain (Sec. 4), HYDROSTATIC = no cell */
enum { OR_CRIT_GLOBAL = 0, OR_CRIT_HYDROSTATIC = 1, OR_CRIT_ETA_D = 2,
       OR_CRIT_ETA_X = 3, OR_CRIT_U = 4, OR_CRIT_U_X = 5, OR_CRIT_W = 6,
       OR_CRIT_W_X = 7 };
/* DENSE: Gaussian elimination with partial pivoting on the dense active
   block (tiny grids); BANDED: the same elimination in tridiagonal band form
   (any size; walls, or periodic without an active pair across the wrap). */
enum { OR_SOLVER_AUTO = 0, OR_SOLVER_CG = 1, OR_SOLVER_BICGSTAB = 2,
       OR_SOLVER_DENSE = 3, OR_SOLVER_BANDED = 4 };
enum { OR_GUESS_ZERO = 0, OR_GUESS_PREV = 1 };
enum { OR_OK = 0, OR_NOT_CONVERGED = 1, OR_BAD_ARG = 2, OR_SINGULAR = 3 };

typedef struct {
    int    nx;        /* number of cells, >= 3                              */
    int    bc;        /* OR_BC_*                                            */
    double dx;        /* uniform cell width                                 */
    double xl;        /* left end; cell i spans [xl + i dx, xl + (i+1) dx]  */
    double g;         /* gravity                                            */
    double rho;       /* density                                            */
    int    limiter;   /* OR_LIM_*                                           */
    /* bottom motion (OR_SLIDE_*, see above)                                */
    int    slide;
    double A, L, xc0, s0, t0;
    double t2;        /* OR_SLIDE_QUARTIC: end of the glide (t2 >= t0)       */
    /* adaptivity */
    int    crit;
    double knh;
    int    enlarge;   /* cells added on each side of the marked set          */
    int    first_step_global;
    /* elliptic solve */
    int    solver;
    double rtol;      /* stop when ||r||_2 <= rtol ||R||_2                   */
    int    max_iter;
    int    guess;
} or_params;

typedef struct {
    int    n_active;
    int    iters;
    int    solver_used;  /* OR_SOLVER_CG / BICGSTAB / DENSE, or -1 if none   */
    int    status;       /* OR_OK / OR_NOT_CONVERGED / ...                   */
    double rel_res;      /* final ||r|| / ||R||                              */
    double min_gamma;    /* minimum diagonal reaction term over active cells */
} or_step_info;

/* Bottom and its derivatives at the centre of cell i at time t:
   out = {d, d_x, d_xx, d_t, d_xt, d_tt}. */
void or_bottom(const or_params* P, const double* d0, int i, double t, double out[6]);

/* Semi-discrete hydrostatic operator H(Q) (Sec. 3.1) with the bottom at time t. */
void or_rhs(const or_params* P, const double* d0, double t,
            const double* h, const double* hu, const double* hw,
            double* rh, double* rhu, double* rhw);

/* Heun predictor (Sec. 3.1, Eqs. 8-9): Q^n at t -> Q~^{n+1} at t + dt. */
void or_predict(const or_params* P, const double* d0, double t, double dt,
                const double* h, const double* hu, const double* hw,
                double* ht, double* hut, double* hwt);

/* Criterion value c_i (Sec. 5.1) on the predicted state at time t. */
void or_criterion(const or_params* P, const double* d0, double t,
                  const double* ht, const double* hut, const double* hwt,
                  double* c);

/* Mask: c > knh (or all / none), first-step rule, enlargement; returns count. */
int or_mask(const or_params* P, const double* d0, double t, long step,
            const double* ht, const double* hut, const double* hwt,
            unsigned char* mask);

/* Elliptic coefficients: Kf[nx+1] (face k between cells k-1 and k),
   gam[nx], R[nx] (all cells; only active ones are used). */
void or_assemble(const or_params* P, const double* d0, double t1, double dt,
                 const double* ht, const double* hut, const double* hwt,
                 double* Kf, double* gam, double* R);

/* y = A x on the active cells (x taken as zero off the mask); y = 0 elsewhere. */
void or_apply(const or_params* P, const unsigned char* mask,
              const double* Kf, const double* gam, const double* x, double* y);

/* Solve A q = R on the active cells.  q holds the initial guess on entry. */
int or_solve(const or_params* P, const unsigned char* mask,
             const double* Kf, const double* gam, const double* R,
             double* q, or_step_info* info);

/* Correction (Eqs. 10-11) on the active cells; h is not corrected. */
void or_correct(const or_params* P, const double* d0, double t1, double dt,
                const unsigned char* mask, const double* q,
                const double* ht, const double* hut, const double* hwt,
                double* h, double* hu, double* hw);

/* One full step n -> n+1 in place.  q: pressure unknown q = h p^nh (in: the
   previous step's, used as guess when guess == PREV; out: this step's).
   mask: out, may be NULL. */
int or_step(const or_params* P, const double* d0, double t, long step, double dt,
            double* h, double* hu, double* hw, double* q, unsigned char* mask,
            or_step_info* info);

/* n_steps steps from t = t_start (step counter starts at step0).  Returns the
   first non-OK status, else OR_OK.  info (nullable) receives the last step's. */
int or_run(const or_params* P, const double* d0, double t_start, long step0,
           double dt, long n_steps, double* h, double* hu, double* hw, double* q,
           or_step_info* info, long long* total_iters, long long* total_active);

#ifdef __cplusplus
}
#endif
#endif
