/*
 * nh_oracle_dg.h -- plain FP64 CPU oracle of the paper's own discretisation
 * of the locally adaptive non-hydrostatic method on 1D grids: the
 * discontinuous Galerkin P1 predictor (Sec. 3.1) and the local discontinuous
 * Galerkin (LDG) solve of the mixed (p, hu) elliptic system with the
 * flip-flop flux (Sec. 3.2, Eqs. 12-15), on marked elements (Sec. 5).
 *
 * TEST INFRASTRUCTURE ONLY, like the rest of this directory: the slow,
 * obviously-correct definition that the CUDA library's DG path is checked
 * against.  It shares no source, header, helper or table with the CUDA
 * library.
 *
 * Elements I_i = [xl + i dx, xl + (i+1) dx], i = 0..ne-1, each with two nodal
 * values (the Lagrange basis of P1 at the element's end points): node 2i is
 * the left end, node 2i+1 the right end.  Every per-node array has 2 ne
 * entries.  Bottom: d(x,t) = b0 + b1 (x - xl) - m(x,t) with the moving parts
 * m of nh_oracle.h (Gaussian mound on ln cosh, impulsive plate, sliding
 * block), evaluated with its derivatives at the node positions.  Walls at
 * both ends.
 *
 * Readings of the paper (it prints the weak forms, not every detail):
 *  - fluxes and sources are represented by their nodal values (the P1
 *    interpolant), the mass matrix is exact for P1;
 *  - the bottom's derivatives are analytic at the nodes; h_x and eta_x in the
 *    elliptic coefficients and in phi are the element's P1 slopes;
 *  - the LDG fluxes (Eqs. 14-15) with c12 = 1/2 (flip-flop: p* from the right
 *    element, hu* from the left) and c22 = 0: p* = p+, hu* = hu- + c11 (p- - p+),
 *    c11 = 1/2 as printed; [.] in the hu-flux is read as the jump of hu;
 *  - at a sub-domain edge and at the walls p* = 0 (zero Dirichlet data), the
 *    outside hu is the predicted one (0 at a wall);
 *  - unmarked elements keep the predicted state; hw (Eq. 11) uses the
 *    element's P1 slope of h p;
 *  - the criterion is evaluated on the element (mean of the two nodal values,
 *    P1 slopes for derivatives); enlargement by whole elements (Sec. 5.2).
 */
#ifndef NH_ORACLE_DG_H
#define NH_ORACLE_DG_H

#include "nh_oracle.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
    int    ne;        /* elements, >= 2                                     */
    double dx, xl;    /* element width, left end                            */
    double g, rho;
    double b0, b1;    /* static bottom d0(x) = b0 + b1 (x - xl)             */
    int    slide;     /* OR_SLIDE_*                                         */
    double A, L, xc0, s0, t0, t2;
    int    crit;      /* OR_CRIT_*                                          */
    double knh;
    int    enlarge;   /* elements added on each side                       */
    int    first_step_global;
    double c11;       /* LDG penalty of the hu-flux (the paper: 1/2)        */
} or_dg_params;

typedef struct {
    int    n_active;  /* marked elements                                    */
    int    status;    /* OR_OK / OR_SINGULAR                                */
    double rel_res;   /* ||b - A x|| / ||b|| of the LDG system              */
} or_dg_info;

/* d, d_x, d_xx, d_t, d_xt, d_tt at position x and time t. */
void or_dg_bottom(const or_dg_params* P, double x, double t, double out[6]);

/* Semi-discrete hydrostatic DG operator (Sec. 3.1) at time t, per node. */
void or_dg_rhs(const or_dg_params* P, double t, const double* h, const double* hu, const double* hw,
               double* rh, double* rhu, double* rhw);

/* Heun (Sec. 3.1): Q^n at t -> Q~ at t + dt. */
void or_dg_predict(const or_dg_params* P, double t, double dt, const double* h, const double* hu,
                   const double* hw, double* ht, double* hut, double* hwt);

/* Marked elements (mask[ne]); returns their number. */
int or_dg_mask(const or_dg_params* P, double t1, long step, const double* ht, const double* hut,
               const double* hwt, unsigned char* mask);

/* The LDG system of the marked elements: per element i, rows 4i..4i+3 =
   (Eq. 12 tested with the left / right basis function, Eq. 13 likewise),
   unknowns 4i..4i+3 = (p_L, p_R, hu_L, hu_R).  Unmarked elements get identity
   rows (p = 0, hu = the predicted hu).  blk: per element 48 doubles: the
   4 x 4 couplings to the left element, to itself, to the right element
   (row-major); rhs: 4 per element. */
void or_dg_assemble(const or_dg_params* P, double t1, double dt, const double* ht, const double* hut,
                    const double* hwt, const unsigned char* mask, double* blk, double* rhs);

/* Solve the block-tridiagonal system by banded Gaussian elimination with
   partial pivoting and two steps of iterative refinement; x: 4 ne unknowns;
   rel_res (nullable): ||rhs - A x|| / ||rhs||. */
int or_dg_solve(const or_dg_params* P, const double* blk, const double* rhs, double* x, double* rel_res);

/* Correction (Eqs. 10-11 through the LDG unknowns): h = h~, hu = the LDG hu,
   hw = hw~ + (dt/rho) P on marked elements; p out (0 elsewhere). */
void or_dg_correct(const or_dg_params* P, double t1, double dt, const unsigned char* mask, const double* x,
                   const double* ht, const double* hut, const double* hwt, double* h, double* hu, double* hw,
                   double* p);

/* One step in place; mask (nullable) receives the marked elements. */
int or_dg_step(const or_dg_params* P, double t, long step, double dt, double* h, double* hu, double* hw,
               double* p, unsigned char* mask, or_dg_info* info);

#ifdef __cplusplus
}
#endif
#endif
