/*
 * nhswe_dg.h -- C ABI of the library's discontinuous Galerkin path: the
 * paper's own discretisation of the locally adaptive non-hydrostatic method
 * on batches of 1D grids (Firdaus & Behrens, Sec. 3).
 *
 * One step (Sec. 3, with the adaptivity of Sec. 5):
 *  1. hydrostatic predictor: DG with the nodal P1 (Lagrange) basis at the
 *     element end points, the Rusanov flux, and Heun's two stages (Sec. 3.1,
 *     Eqs. 6-9);
 *  2. criterion of Sec. 5.1 on each element of the predicted state (mean of
 *     its two nodal values, P1 slopes for the x-derivatives), marked elements
 *     enlarged by `enlarge` whole elements on each side (Sec. 5.2);
 *  3. on the marked elements, the mixed (p, hu) elliptic system of Eqs. 12-13
 *     discretised by LDG with the flip-flop fluxes of Eqs. 14-15:
 *     p* = p+, hu* = hu- + c11 (p- - p+) between marked elements; p* = 0 at
 *     the edge of a marked region and at a wall, the outside hu there being
 *     the predicted one (0 at a wall);
 *  4. correction: hu = the LDG unknown, hw from Eq. 11 with the element's P1
 *     slope of h p, h unchanged; unmarked elements keep the predicted state.
 *
 * How it is solved (the result is the solution of that linear system, up to
 * FP64 rounding): each marked element's two Eq. 12 rows give its hu as an
 * affine function of its own p and of its right neighbour's p (the rows'
 * hu-block is the element's mass matrix weighted by s12 > 0, inverted per
 * element); substituting into the Eq. 13 rows leaves a block-tridiagonal
 * system in p with 2 x 2 blocks, one block row per marked element, which
 * block cyclic reduction solves without pivoting (each level halves the
 * rows; O(marked elements) work per member).
 *
 * Conventions (as in nhswe.h):
 *  - Host arrays are FP64, member-major, two values per element: node 2i is
 *    the left end of element i (x0 + i dx), node 2i+1 its right end
 *    (x0 + (i+1) dx); value (b, k) of a field is at [b * 2 ne + k].
 *  - Device memory is never allocated by the library: it lives in the
 *    caller's workspace (nh_dg_workspace_bytes()), 256-byte aligned, valid
 *    and untouched until nh_dg_destroy().
 *  - All GPU work is ordered on the caller's stream (a cudaStream_t, NULL =
 *    legacy default stream); nh_dg_step, nh_dg_run and the nh_dg_get_* calls
 *    synchronise it.  A handle is used by one host thread at a time.
 *  - Errors are returned as nh_status (nhswe.h).  FP64 throughout; no CPU
 *    fallback: a missing or unusable device is NH_ERR_CUDA.
 *  - Both ends of every member are walls (mirror ghost state h, -hu, hw).
 */
#ifndef NHSWE_DG_H
#define NHSWE_DG_H

#include <stddef.h>

#include "nhswe.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nh_dg nh_dg;   /* opaque, created by nh_dg_create */

typedef struct {
    int    ne;      /* elements per member, 2 <= ne <= 2^20                 */
    int    nbatch;  /* members, >= 1                                        */
    double dx;      /* element width (m), > 0                               */
    double x0;      /* left end of the domain (m)                           */
    double g;       /* gravity (m/s^2), > 0                                 */
    double rho;     /* density (kg/m^3), > 0                                */
    double c11;     /* LDG penalty of the hu-flux, >= 0 (the paper: 1/2)    */
} nh_dg_desc;

/* Bytes of device workspace nh_dg_create needs (0 if desc is invalid). */
size_t nh_dg_workspace_bytes(const nh_dg_desc* desc);

/* Create a handle and upload the static depth.  d0_host: nbatch * 2 ne FP64
   nodal depths d0 > 0 (m); the static part's x-derivative on element i is
   its P1 slope (d0[2i+1] - d0[2i]) / dx, its second derivative 0.  Defaults:
   no bottom motion, criterion GLOBAL with k_nh = 1e-3 and one enlarging
   element, residual check on.  No state: nh_dg_set_state comes first.
   Errors: NH_ERR_ARG (bad descriptor, NULL pointer, non-positive or
   non-finite depth, short or misaligned workspace), NH_ERR_CUDA. */
nh_status nh_dg_create(const nh_dg_desc* desc, const double* d0_host, void* ws, size_t ws_bytes,
                       void* stream, nh_dg** out);

/* Bottom motion per member (nh_slide_desc of nhswe.h; its value and
   derivatives are analytic at the nodes).  slides: nbatch entries, or NULL
   for a static bottom.  Errors: NH_ERR_ARG (non-finite or out-of-range
   parameters). */
nh_status nh_dg_set_bottom_motion(nh_dg* g, const nh_slide_desc* slides);

/* Sec. 5.1-5.2: an element whose criterion value on the predicted state
   exceeds k_nh (strictly) is marked; the set is enlarged by `enlarge`
   elements (0..16) on each side.  kind: NH_CRIT_* of nhswe.h.
   first_step_global != 0 marks every element in the first step after
   nh_dg_set_state.  Errors: NH_ERR_ARG. */
nh_status nh_dg_set_criterion(nh_dg* g, int kind, double k_nh, int enlarge, int first_step_global);

/* check != 0 (the default): every step also forms the residual of the
   block-tridiagonal p-system at the solution and reports, as a backward
   error, max over members of ||r - A p|| / || |r| + |A| |p| || (FP64, 2-norms
   over the member's rows, |.| elementwise) in nh_step_info.rel_res.
   check == 0 skips that pass (rel_res = 0).  Non-finite values in the
   solution are detected either way.  Errors: NH_ERR_ARG. */
nh_status nh_dg_set_check(nh_dg* g, int check);

/* Upload a state at model time t (host FP64, nbatch * 2 ne each): nodal
   h > 0 (m), hu, hw (m^2/s).  Resets the step counter and p.
   Errors: NH_ERR_ARG (NULL, h <= 0 or non-finite), NH_ERR_CUDA. */
nh_status nh_dg_set_state(nh_dg* g, const double* h, const double* hu, const double* hw, double t);

/* Download the state (host FP64, nbatch * 2 ne each; any pointer may be
   NULL): h, hu, hw and p, the non-hydrostatic pressure of the last step at
   the nodes (Pa; 0 on unmarked elements).  Errors: NH_ERR_STATE,
   NH_ERR_CUDA. */
nh_status nh_dg_get_state(nh_dg* g, double* h, double* hu, double* hw, double* p);

/* The last step's marked elements (nbatch * ne bytes, 1 = marked) and
   per-member residuals (nbatch doubles, 0 with the check off); either
   pointer may be NULL.  Errors: NH_ERR_STATE, NH_ERR_CUDA. */
nh_status nh_dg_get_mask(nh_dg* g, unsigned char* mask, double* rel_res);

/* One step of size dt > 0.  A step whose solution holds a non-finite value
   returns NH_ERR_NONFINITE and leaves the state as it was.  info (nullable):
   step, t, n_active (marked elements, all members), n_active_max, iters = 0
   (direct solve), solver = -1, status, rel_res, mass = sum over members and
   elements of dx (h_L + h_R) / 2. */
nh_status nh_dg_step(nh_dg* g, double dt, nh_step_info* info);

/* n_steps steps of size dt, replayed from CUDA graphs captured on first use
   (one per state-buffer parity) with one synchronisation at the end; time,
   step counter and acceptance live on the device.  Stops at the first failing
   step with the last accepted state intact (its status is returned and
   info->last describes it).  info may be NULL. */
nh_status nh_dg_run(nh_dg* g, double dt, long long n_steps, nh_run_info* info);

/* Kernel classes of the DG path (index into nh_dg_get_profile arrays). */
enum { NH_DG_K_KINEMATICS = 0, NH_DG_K_PREDICT = 1, NH_DG_K_MARK = 2, NH_DG_K_COMPACT = 3,
       NH_DG_K_LOCAL = 4, NH_DG_K_FORM = 5, NH_DG_K_REDUCE = 6, NH_DG_K_BACK = 7,
       NH_DG_K_CORRECT = 8, NH_DG_K_FINISH = 9, NH_DG_K_COUNT = 10 };

/* enable != 0: bracket every launch of nh_dg_step with CUDA events and
   accumulate device time per class (nh_dg_run then steps one by one);
   resets the accumulators.  nh_dg_get_profile: NH_DG_K_COUNT entries each
   (nullable): milliseconds and launches since the last nh_dg_set_profiling. */
nh_status nh_dg_set_profiling(nh_dg* g, int enable);
nh_status nh_dg_get_profile(nh_dg* g, double* ms, long long* launches);

/* Release the handle (the workspace stays the caller's). */
void nh_dg_destroy(nh_dg* g);

#ifdef __cplusplus
}
#endif
#endif /* NHSWE_DG_H */
