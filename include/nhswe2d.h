/* nhswe2d.h -- the method on two-dimensional grids (FP64, or FP32 state).
 *
 * The paper's model is one-dimensional (Sec. 2) and names the extension to
 * two horizontal dimensions as future work (Sec. 6).  These calls run its
 * generalisation in which every x-derivative of Eqs. 1-5 and 10-11 becomes a
 * gradient: a hydrostatic Heun predictor (Eqs. 8-9) with Rusanov fluxes in x
 * and y, the criteria of Sec. 5.1 in their 2D form (|eta/d|, |grad eta|,
 * |u|, |grad u|, |w|, |grad w|), enlargement to the Moore neighbourhood
 * (Sec. 5.2), and the projection (Eqs. 10-11), whose elimination into the
 * constraint (Eq. 4) gives the self-adjoint equation
 *     -div(K grad q) + gamma q = R,  K = (dt/rho)/h (I - grad d grad d^T / D),
 *     D = 4 + |grad d|^2, q = h p,
 * on the marked cells (q = 0 elsewhere and outside walled sides), discretised
 * with a symmetric 9-point stencil and solved by CG preconditioned with an
 * aggregation multigrid V-cycle (or with exact x-line tridiagonal solves).
 * A problem that does not depend on y gives the 1D method's result.
 *
 * Ensembles: one handle may hold n_members grids, each with its own size,
 * spacing, sides, static depth and slide (the drawn-parameter landslide runs
 * of Sec. 4.2 side by side), stepped together with one dt and one criterion
 * and solver setting.  Every kernel of a step covers all members; their
 * Krylov solves share one cooperative launch, and nh2d_run replays the whole
 * step from a captured CUDA graph.  A single grid is the one-member
 * ensemble; the calls without "member" act on member 0 (set_bottom_motion:
 * on all members).
 *
 * Layout: host arrays are nx * ny FP64, row-major with x fastest (cell (i, j)
 * at j * nx + i).  On the device member m's cells sit at m * pitch in every
 * per-cell buffer, pitch = the largest member's cell count rounded up to 256.
 * Device memory is the caller's workspace (nh2d_workspace_bytes /
 * nh2d_ensemble_workspace_bytes, 256-byte aligned, alive until
 * nh2d_destroy); the handle creates one extra (capture) stream and otherwise
 * allocates no device memory.  Calls are ordered on the handle's stream;
 * nh2d_step / nh2d_run synchronise it.  Errors as in nhswe.h: NH_ERR_ARG (bad
 * argument), NH_ERR_CUDA, NH_ERR_NOT_CONVERGED / NH_ERR_NONFINITE (the step
 * is not taken: the state stays at the last accepted step), NH_ERR_TIMEOUT,
 * NH_ERR_STATE (no state set).
 */
#ifndef NHSWE2D_H
#define NHSWE2D_H

#include "nhswe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nh_grid2d nh_grid2d;

typedef struct {
    int    nx, ny;       /* cells; 3 <= nx, ny; nx * ny <= 2^26                  */
    int    bc_x, bc_y;   /* NH_BC_WALL or NH_BC_PERIODIC                         */
    int    limiter;      /* NH_LIM_*                                              */
    double dx, dy;       /* cell size (m)                                        */
    double x0, y0;       /* lower-left corner: cell (i, j) centre at
                            (x0 + (i + 1/2) dx, y0 + (j + 1/2) dy)                */
    double g, rho;       /* gravity (m/s^2), density (kg/m^3)                    */
} nh_grid2d_desc;

/* Moving bottom (Sec. 4.2 form, elliptic mound): d(x, y, t) = d0(x, y) -
   A exp(-((x - xc0 - s(t))/Lx)^2 - ((y - yc0)/Ly)^2), s = s0 ln cosh(t/t0). */
typedef struct {
    int    shape;        /* NH_SLIDE_NONE or NH_SLIDE_GAUSS_LNCOSH */
    double A, Lx, Ly, xc0, yc0, s0, t0;
} nh_slide2d_desc;

/* 0 for an invalid description. */
size_t nh2d_workspace_bytes(const nh_grid2d_desc* desc);

/* 1 <= n_members <= 4096, n_members * pitch <= 2^28; 0 when invalid. */
size_t nh2d_ensemble_workspace_bytes(int n_members, const nh_grid2d_desc* descs);

/* d0_host: static depth d0 (m, > 0), nx * ny values. */
nh_status nh2d_create(const nh_grid2d_desc* desc, const double* d0_host, void* ws, size_t ws_bytes,
                      void* stream, nh_grid2d** out);

/* descs[m], d0_host[m]: member m's grid and static depth. */
nh_status nh2d_create_ensemble(int n_members, const nh_grid2d_desc* descs, const double* const* d0_host,
                               void* ws, size_t ws_bytes, void* stream, nh_grid2d** out);

/* Number of members (0 for NULL). */
int nh2d_members(const nh_grid2d* g);

/* NULL: static bottom.  nh2d_set_bottom_motion sets every member's. */
nh_status nh2d_set_bottom_motion(nh_grid2d* g, const nh_slide2d_desc* slide);
nh_status nh2d_set_member_bottom_motion(nh_grid2d* g, int member, const nh_slide2d_desc* slide);

/* As nh_set_criterion (NH_CRIT_*, k_nh > 0, 0 <= enlarge <= 16). */
nh_status nh2d_set_criterion(nh_grid2d* g, int kind, double k_nh, int enlarge, int first_step_global);

/* rtol: ||R - A q||_2 <= rtol ||R||_2; guess NH_GUESS_ZERO or NH_GUESS_PREV.
   Defaults 1e-12, 20000, NH_GUESS_PREV.  A CG breakdown (indefinite
   operator) is solved again by unpreconditioned BiCGStab. */
nh_status nh2d_set_solver(nh_grid2d* g, double rtol, int max_iter, int guess);

/* Preconditioner of the CG solve: NH_PRECOND_MG (default) or
   NH_PRECOND_LINE.  MG: aggregation multigrid over the bounding box of each
   member's active cells -- coarse cell (I, J) at level l gathers the fine
   cells (i >> l, j >> l) = (I, J), Galerkin coarse operators (sums of the
   children's 9-point rows), one damped-Jacobi sweep (omega 0.7) before and
   after the coarse correction, 7 sweeps on the coarsest level (at most 16
   cells), all in FP32 -- applied once per iteration of the FP64 flexible PCG.
   LINE: exact x-line (tridiagonal) solves by cyclic reduction in FP32.  The
   converged answer is the same (the preconditioner changes the iteration,
   not the solution); members that fall back to BiCGStab (an indefinite
   operator) use the line preconditioner.  Errors: NH_ERR_ARG. */
nh_status nh2d_set_preconditioner(nh_grid2d* g, int kind);

/* NH_FP64 (default) or NH_MIXED_FP64_SOLVE: the state is stored in FP32 as
   zeta = h - d0, hu, hv, hw (so eta = zeta + mound keeps its digits), the
   predictor and the criterion run in FP32, the assembly, the Krylov solve,
   the correction's arithmetic and every reduction stay FP64.  A change
   clears every member's state (set it again before stepping). */
nh_status nh2d_set_precision(nh_grid2d* g, int precision);

/* 1 (default): nh2d_run replays captured graphs when it can (not for a
   first step that is global by request, nor right after a change of dt);
   0: every step is enqueued from the host. */
nh_status nh2d_set_graphs(nh_grid2d* g, int on);

/* As nh_set_wait_budget: spin limit (SM clock cycles, 0 = about one second)
   of the persistent solver's grid barrier; on expiry the step reports
   NH_ERR_TIMEOUT and is not taken. */
nh_status nh2d_set_wait_budget(nh_grid2d* g, long long cycles);

/* h > 0 (m), hu, hv, hw (m^2/s) of member m; sets the whole ensemble's time
   to t and clears member m's warm start.  Steps need every member set. */
nh_status nh2d_set_state(nh_grid2d* g, const double* h, const double* hu, const double* hv,
                         const double* hw, double t);
nh_status nh2d_set_member_state(nh_grid2d* g, int member, const double* h, const double* hu,
                                const double* hv, const double* hw, double t);

/* Replace member m's state with host values (same layout and units as
   nh2d_set_member_state) and keep the time, the step count and the warm
   start: the state a caller hands in between steps.  The copies are ordered
   on the handle's stream and the call does not synchronise it, so the host
   arrays must stay untouched until the next synchronising call (pinned
   memory makes the copies asynchronous).  Values are not checked on the
   host: a non-positive or non-finite thickness fails the next step
   (NH_ERR_NONFINITE).  Errors: NH_ERR_ARG, NH_ERR_STATE (no state set yet),
   NH_ERR_CUDA. */
nh_status nh2d_put_member_state(nh_grid2d* g, int member, const double* h, const double* hu, const double* hv,
                                const double* hw);

/* Any pointer may be NULL.  p_nh: non-hydrostatic pressure of the last step
   (Pa; 0 on cells that were hydrostatic). */
nh_status nh2d_get_state(nh_grid2d* g, double* h, double* hu, double* hv, double* hw, double* p_nh);
nh_status nh2d_get_member_state(nh_grid2d* g, int member, double* h, double* hu, double* hv, double* hw,
                                double* p_nh);

/* Last step's non-hydrostatic mask (nx * ny bytes). */
nh_status nh2d_get_mask(nh_grid2d* g, unsigned char* mask);
nh_status nh2d_get_member_mask(nh_grid2d* g, int member, unsigned char* mask);

/* info (may be NULL): as nh_step_info, summed (n_active, mass) or taken
   worst (iters, rel_res, status) over members; mass = sum(h) dx dy. */
nh_status nh2d_step(nh_grid2d* g, double dt, nh_step_info* info);
nh_status nh2d_run(nh_grid2d* g, double dt, long long n_steps, nh_run_info* info);

/* Member m's figures of the last step (n_active, iters, rel_res, min_gamma,
   solver, status) and the mass sum(h) dx dy of its new state. */
nh_status nh2d_get_member_info(nh_grid2d* g, int member, nh_step_info* info);

/* Tile of the one-launch FP32-state predictor (NH_MIXED_FP64_SOLVE): the
   candidates are 32 x 16, 64 x 8, 32 x 8 and 64 x 16 cells (tile = 0..3).
   By default the first FP32 step times each candidate on the live state and
   keeps the fastest (cached per set of member sizes and limiters).  tile
   0..3 forces a candidate, -2 asks for a new timing at the next step, -1
   only reads; *chosen (may be NULL) receives the candidate in use (-1: not
   chosen yet).  Every candidate gives the same result bit for bit.  Errors:
   NH_ERR_ARG. */
nh_status nh2d_set_tile(nh_grid2d* g, int tile, int* chosen);

/* Kernel classes of nh2d_get_profile. */
enum { NH2_K_KIN = 0, NH2_K_DEPTH, NH2_K_STAGE, NH2_K_MARKS, NH2_K_DILATE, NH2_K_COMPACT, NH2_K_ASSEMBLE,
       NH2_K_MASS, NH2_K_SOLVE_INIT, NH2_K_SOLVE, NH2_K_SUMMARY, NH2_K_CLEAR, NH2_K_CORRECT, NH2_K_COUNT };

/* 1: later steps are enqueued from the host (no graph replay) with a CUDA
   event pair on the handle's stream around every launch, summed per kernel
   class (NH2_K_SOLVE: the whole Krylov solve of a step, NH2_K_COMPACT: the
   four compaction launches); 0: off.  Either call resets the totals. */
nh_status nh2d_set_profiling(nh_grid2d* g, int enable);

/* ms[NH2_K_COUNT]: device milliseconds per class since the last
   nh2d_set_profiling; launches[NH2_K_COUNT]: launches (event pairs) per
   class.  Errors: NH_ERR_ARG. */
nh_status nh2d_get_profile(nh_grid2d* g, double* ms, long long* launches);

/* Number of captured-graph runs nh2d_run has made (-1 for NULL). */
long long nh2d_graph_runs(const nh_grid2d* g);

void nh2d_destroy(nh_grid2d* g);

#ifdef __cplusplus
}
#endif
#endif /* NHSWE2D_H */
