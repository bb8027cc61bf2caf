/*
 * nhswe.h -- C ABI of the GB300 (sm_103a) locally adaptive non-hydrostatic
 * shallow-water library.
 *
 * The library advances the one-dimensional non-hydrostatic extension of the
 * shallow-water equations with a moving bottom (Firdaus & Behrens, Sec. 2,
 * Eqs. 1-5) by the projection method of Sec. 3: a hydrostatic predictor
 * (Sec. 3.1), a criterion on the predicted state that marks the
 * non-hydrostatic cells (Sec. 5.1, enlarged by whole cells as in Sec. 5.2),
 * an elliptic solve for the non-hydrostatic pressure on the marked cells only
 * (Sec. 3.2, Eqs. 12-13, zero Dirichlet data on the sub-domain boundary), and
 * the backward-Euler correction of hu and hw (Eqs. 10-11; h is not corrected).
 *
 * One handle holds a batch of `nbatch` independent members that share the grid
 * geometry (cell count, spacing, boundary kind) but each have their own static
 * depth, slide motion and state; every kernel processes the whole batch.
 *
 * Conventions for every entry point:
 *  - Host arrays are FP64, member-major: element (b, i) of a field is at
 *    [b * nx + i]; cell i of a member spans [x0 + i dx, x0 + (i+1) dx].
 *  - Device memory is never allocated by the library.  All of it lives in the
 *    caller's workspace (`ws`, `ws_bytes` from nh_workspace_bytes()), which
 *    must stay valid and untouched until nh_destroy().
 *  - All GPU work is ordered on the caller's stream (`stream`, a
 *    cudaStream_t, NULL = legacy default stream).  Calls that return data to
 *    the host (nh_get_*), nh_step and nh_run synchronise that stream.
 *  - Errors are returned as nh_status, never thrown; nh_status_string()
 *    names them.  A handle is used by one host thread at a time.
 *  - The library computes on the GPU only.  There is no CPU fallback; a
 *    missing or unusable device is reported as NH_ERR_CUDA.
 */
#ifndef NHSWE_H
#define NHSWE_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct nh_grid nh_grid;   /* opaque, created by nh_create_grid */

typedef enum {
    NH_OK = 0,
    NH_ERR_ARG = 1,            /* invalid argument or descriptor            */
    NH_ERR_CUDA = 2,           /* a CUDA runtime call failed                */
    NH_ERR_NOT_CONVERGED = 3,  /* Krylov solve hit max_iter; step rolled back */
    NH_ERR_NONFINITE = 4,      /* NaN/Inf in a residual norm; step rolled back */
    NH_ERR_TIMEOUT = 5,        /* a bounded device-side wait gave up        */
    NH_ERR_STATE = 6           /* call out of order (e.g. no state set)     */
} nh_status;

enum { NH_BC_WALL = 0, NH_BC_PERIODIC = 1 };
/* NH_FP64: every field, coefficient, vector and sum in FP64.
   NH_MIXED: state, predictor, coefficients and Krylov vectors in FP32;
   inner products, norms, mass sums and the iterative-refinement residual in
   FP64.
   NH_MIXED_FP64_SOLVE: state, predictor and correction coefficients in
   FP32; the elliptic operator, the Krylov vectors and every sum in FP64 (one
   FP64 Krylov solve per step, no refinement passes). */
enum { NH_FP64 = 0, NH_MIXED = 1, NH_MIXED_FP64_SOLVE = 2 };
/* Slope limiter of the piecewise-linear reconstruction of eta, u, w. */
enum { NH_LIM_NONE = 0, NH_LIM_CENTRAL = 1, NH_LIM_MINMOD = 2, NH_LIM_MC = 3 };
/* Sec. 5.1 criteria.  GLOBAL = every cell (the global model of Sec. 4);
   HYDROSTATIC = no cell (plain SWE). */
enum { NH_CRIT_GLOBAL = 0, NH_CRIT_HYDROSTATIC = 1, NH_CRIT_ETA_D = 2,
       NH_CRIT_ETA_X = 3, NH_CRIT_U = 4, NH_CRIT_U_X = 5, NH_CRIT_W = 6,
       NH_CRIT_W_X = 7 };
/* The discrete operator is symmetric.  AUTO: (preconditioned) CG; a member
   whose CG detects indefiniteness (p.Ap <= 0 or r.z <= 0) is solved again by
   BiCGStab from the warm start.  gamma > 0 on every active cell is sufficient
   for positive definiteness; a few negative gamma cells (e.g. at a kink of
   d0) usually leave the operator definite.  CG / BICGSTAB force one method. */
enum { NH_SOLVER_AUTO = 0, NH_SOLVER_CG = 1, NH_SOLVER_BICGSTAB = 2 };
/* NH_GUESS_CNN: the learned guess of nhswe_cnn.h (needs nh_cnn_attach). */
enum { NH_GUESS_ZERO = 0, NH_GUESS_PREV = 1, NH_GUESS_CNN = 2 };
/* Preconditioner of the CG branch.  NH_PRECOND_LINE: the tridiagonal operator
   restricted to blocks of 8192 consecutive active cells, solved by parallel
   cyclic reduction in FP32 (exact up to FP32 rounding on any active segment
   that fits in one block), inside a flexible (Polak-Ribiere) PCG whose
   vectors, dots and stopping test stay in the handle's precision. */
/* NH_PRECOND_MG (2D grids only, nhswe2d.h): an aggregation multigrid V-cycle
   in FP32 inside the same flexible PCG. */
enum { NH_PRECOND_NONE = 0, NH_PRECOND_LINE = 1, NH_PRECOND_MG = 2 };
enum { NH_SLIDE_NONE = 0, NH_SLIDE_GAUSS_LNCOSH = 1, NH_SLIDE_PLATE_EXP = 2, NH_SLIDE_QUARTIC = 3 };

typedef struct {
    int    dim;        /* 1                                                 */
    int    nx;         /* cells per member, 8 <= nx <= 2^20                  */
    int    nbatch;     /* members, >= 1                                     */
    int    bc;         /* NH_BC_WALL or NH_BC_PERIODIC (both ends)          */
    int    precision;  /* NH_FP64, NH_MIXED or NH_MIXED_FP64_SOLVE          */
    int    limiter;    /* NH_LIM_*                                          */
    double dx;         /* cell width (m), > 0                               */
    double x0;         /* left end of the domain (m)                        */
    double g;          /* gravity (m/s^2), > 0                              */
    double rho;        /* density (kg/m^3), > 0; scales p^nh only           */
} nh_grid_desc;

/* Moving bottom of one member, d(x,t) = d0(x) - m(x,t):
   NH_SLIDE_GAUSS_LNCOSH  m = A exp(-((x - xc0 - s(t))/L)^2), s(t) = s0 ln cosh(t/t0)
                          (a Gaussian mound sliding down-slope);
   NH_SLIDE_PLATE_EXP     m = A (1 - exp(-t/t0)) on |x - xc0| < L, else 0: the
                          impulsively moved plate of Sec. 4.2 (A = zeta0, L = b,
                          t0 = 1/alpha); the plate's edges are a jump of the depth;
   NH_SLIDE_QUARTIC       m = A (1 - xi^4) on |xi| < 1, xi = 2 (x - xc0 - S(t))/L,
                          else 0: the sliding block of Sec. 4.3 (A = H_s, L = L_s)
                          with S = s0 t^2/2 up to t0, then a glide at s0 t0 up to t2,
                          then deceleration -s0 up to t2 + t0, at rest after.
   The static part d0 is sampled per cell; its x-derivatives are central
   differences; the moving part's value and derivatives are analytic. */
typedef struct {
    int    shape;      /* NH_SLIDE_*                                        */
    double A, L, xc0;  /* height (m), width (m, > 0), position (m)          */
    double s0, t0;     /* GAUSS: travel scale (m), time scale (s, > 0);
                          PLATE: s0 unused, t0 = 1/alpha (s, > 0);
                          QUARTIC: acceleration a0 (m/s^2), its duration t1 (s, > 0) */
    double t2;         /* QUARTIC: end of the glide (s, >= t0); else unused  */
} nh_slide_desc;

typedef struct {
    long long step;        /* steps taken since the state was set              */
    double    t;           /* model time after the step (s)                    */
    long long n_active;    /* active (non-hydrostatic) cells, all members      */
    int       n_active_max;/* largest per-member active count                  */
    int       iters;       /* Krylov iterations, maximum over members          */
    int       ir_passes;   /* refinement passes (NH_MIXED), maximum over members */
    int       solver;      /* NH_SOLVER_CG if every solved member finished with
                              CG, NH_SOLVER_BICGSTAB if any used BiCGStab, -1 none */
    int       status;      /* nh_status of the step                             */
    double    rel_res;     /* max over members of ||R - A q|| / ||R||           */
    double    min_gamma;   /* min over active cells of the scaled reaction term */
    double    mass;        /* sum over members and cells of h dx (FP64)         */
} nh_step_info;

typedef struct {
    long long steps;         /* steps completed                                */
    long long iters_total;   /* sum over steps of nh_step_info.iters           */
    long long active_total;  /* sum over steps of nh_step_info.n_active        */
    nh_step_info last;       /* the last step: completed, or the failing one   */
} nh_run_info;

/* Bytes of device workspace nh_create_grid needs for `desc` (0 if invalid). */
size_t nh_workspace_bytes(const nh_grid_desc* desc);

/* Create a handle over the caller's workspace and upload the static depth.
   d0_host: nbatch * nx FP64 depths d0 > 0 (m), member-major.  The workspace
   must be 256-byte aligned and at least nh_workspace_bytes(desc) long.
   The new handle has no state (nh_set_state must come before stepping), no
   bottom motion, criterion GLOBAL with k_nh = 1e-3 and one enlarging cell,
   solver AUTO, rtol 1e-12, max_iter 20000, warm start PREV, ir_max 30,
   inner_rtol 1e-5, and preconditioner NH_PRECOND_LINE.
   Errors: NH_ERR_ARG (bad descriptor, NULL pointer, short or misaligned
   workspace), NH_ERR_CUDA. */
nh_status nh_create_grid(const nh_grid_desc* desc, const double* d0_host,
                         void* ws, size_t ws_bytes, void* stream, nh_grid** out);

/* Ensemble of members with different cell counts (uneven grids) in one
   handle: nx_per_member[b] cells for member b (8 <= nx <= 2^20); desc->nx is
   ignored.  Host arrays of every entry point are then the members
   concatenated: member b occupies [sum_{b'<b} nx_{b'}, sum_{b'<=b} nx_{b'}).
   d0_host likewise.  Every kernel of a step still processes all members in
   one launch; device storage per member is sized for the largest member.
   Errors as nh_create_grid. */
size_t nh_workspace_bytes_ensemble(const nh_grid_desc* desc, const int* nx_per_member);
nh_status nh_create_ensemble(const nh_grid_desc* desc, const int* nx_per_member, const double* d0_host,
                             void* ws, size_t ws_bytes, void* stream, nh_grid** out);

/* Bottom motion per member (nh_slide_desc: the Gaussian mound, and the
   paper's own moving bottoms of Sec. 4.2-4.3).  slides: nbatch entries, or
   NULL for a static bottom.  Errors: NH_ERR_ARG. */
nh_status nh_set_bottom_motion(nh_grid* g, const nh_slide_desc* slides);

/* Adaptivity (Sec. 5.1, 5.2): cells whose criterion value on the predicted
   state exceeds k_nh (strictly) are marked, then the set is enlarged by
   `enlarge` cells on each side (0 <= enlarge <= 16).  first_step_global != 0
   applies the model on every cell in the first step after nh_set_state (the
   rule Sec. 5.1.2 gives for the |w| and |w_x| criteria).  Errors: NH_ERR_ARG. */
nh_status nh_set_criterion(nh_grid* g, int kind, double k_nh, int enlarge,
                           int first_step_global);

/* Elliptic solve on the marked cells (Sec. 3.2).  rtol: stop when
   ||R - A q||_2 <= rtol ||R||_2 per member (FP64 norms).  max_iter >= 1.
   guess: NH_GUESS_PREV starts from the previous step's pressure on cells
   active in both steps (zero elsewhere); NH_GUESS_CNN from the learned
   guess (NH_ERR_STATE unless nh_cnn_attach was called).  NH_MIXED only: ir_max >= 1 outer
   refinement passes with an FP64 residual, each an FP32 Krylov solve to
   inner_rtol (relative to its own right-hand side).  Errors: NH_ERR_ARG. */
nh_status nh_set_solver(nh_grid* g, int kind, double rtol, int max_iter, int guess,
                        int ir_max, double inner_rtol);

/* Preconditioner for members solved by CG (NH_PRECOND_NONE or
   NH_PRECOND_LINE; the default is NH_PRECOND_LINE).  It changes how fast the
   solve converges, not what it converges to.  BiCGStab members are not
   preconditioned.  Errors: NH_ERR_ARG. */
nh_status nh_set_preconditioner(nh_grid* g, int kind);

/* Upload a state (host FP64, nbatch * nx each): h > 0 (m), hu (m^2/s),
   hw (m^2/s) at model time t; the step counter restarts at 0 and the
   previous pressure is cleared.  Errors: NH_ERR_ARG, NH_ERR_CUDA. */
nh_status nh_set_state(nh_grid* g, const double* h, const double* hu, const double* hw,
                       double t);

/* Replace the state in place (host FP64, nbatch * nx each) and keep running:
   model time, step counter and the previous pressure (warm start) are kept.
   This is the upload half of a host-buffer round trip per step.
   Errors: NH_ERR_ARG, NH_ERR_STATE (no state set yet), NH_ERR_CUDA. */
nh_status nh_put_state(nh_grid* g, const double* h, const double* hu, const double* hw);

/* Download the state (host FP64, nbatch * nx each; any pointer may be NULL):
   h, hu, hw, and p_nh = the non-hydrostatic pressure of the last step
   (Pa; zero on cells that were hydrostatic).  Errors: NH_ERR_STATE, NH_ERR_CUDA. */
nh_status nh_get_state(nh_grid* g, double* h, double* hu, double* hw, double* p_nh);

/* Download the last step's non-hydrostatic mask (nbatch * nx bytes, 1 =
   corrected cell) and per-member Krylov iterations / relative residuals
   (nbatch entries each; any pointer may be NULL). */
nh_status nh_get_mask(nh_grid* g, unsigned char* mask, int* iters, double* rel_res);

/* One step of size dt > 0: predictor, criterion and mask, elliptic solve on
   the mask, correction.  On NH_ERR_NOT_CONVERGED, NH_ERR_NONFINITE or
   NH_ERR_TIMEOUT the state is left as it was before the step.  info may be
   NULL. */
nh_status nh_step(nh_grid* g, double dt, nh_step_info* info);

/* n_steps steps of size dt; stops at the first failing step (whose status is
   returned; info->last describes it).  info may be NULL. */
nh_status nh_run(nh_grid* g, double dt, long long n_steps, nh_run_info* info);

/* Predictor tile (cells per CTA: 128, 256 or 512).  By default the first
   nh_step / nh_run of a handle times every candidate on the handle's state
   with CUDA events and keeps the fastest (cached per shape for the process).
   tile != 0 forces a tile; tile == 0 keeps the current choice.  chosen
   (nullable) receives the tile in use, 0 if not chosen yet.
   Errors: NH_ERR_ARG. */
nh_status nh_set_tile(nh_grid* g, int tile, int* chosen);

/* use_graphs != 0 (the default): nh_run captures one FP64 step per
   state-buffer parity as a CUDA graph (on a private capture stream, replayed
   on the handle's stream) and replays it n_steps times with a single
   synchronisation at the end; time and step acceptance live on the device.
   Used when the handle is FP64 with NH_PRECOND_LINE and solver AUTO or CG,
   profiling is off and dt is unchanged.  A step that fails inside a replay
   stops the replay with the last accepted state intact and is redone by the
   step-by-step path.  use_graphs == 0: always step by step. */
nh_status nh_set_run_mode(nh_grid* g, int use_graphs);

/* Spin limit of the persistent solver's grid-wide barrier, in SM clock
   cycles (0: the default, about one second of the device clock).  A barrier
   whose partners do not arrive within the limit makes every CTA of the solve
   return; the step reports NH_ERR_TIMEOUT, is not taken (the state stays at
   the last accepted step) and the handle stays usable.  Drops the captured
   graphs.  Errors: NH_ERR_ARG (cycles < 0). */
nh_status nh_set_wait_budget(nh_grid* g, long long cycles);

/* Kernel classes timed by the profiler (index into nh_get_profile arrays). */
enum { NH_K_KINEMATICS = 0, NH_K_PREDICT = 1, NH_K_COMPACT = 2, NH_K_ASSEMBLE = 3,
       NH_K_SOLVE_INIT = 4, NH_K_PRECOND = 5, NH_K_PCG_A = 6, NH_K_PCG_B = 7,
       NH_K_CG_A = 8, NH_K_CG_B = 9, NH_K_BI_1 = 10, NH_K_BI_2 = 11, NH_K_BI_3 = 12,
       NH_K_SUMMARY = 13, NH_K_CLEAR = 14, NH_K_CORRECT = 15,
       NH_K_PCG_LOOP = 16,   /* all PCG iterations of a solve in one cooperative launch */
       NH_K_CNN = 17,        /* learned guess: history, features, network, guess */
       NH_K_COUNT = 18 };

/* enable != 0: bracket every kernel launch with CUDA events on the handle's
   stream and accumulate per-class device time (read back at the step's own
   synchronisation points); also resets the accumulators.  Launch counts are
   kept whether or not timing is enabled. */
nh_status nh_set_profiling(nh_grid* g, int enable);

/* Per kernel class (NH_K_COUNT entries each, any pointer may be NULL):
   total device milliseconds (0 unless profiling was enabled) and launches
   since the last nh_set_profiling call.  Errors: NH_ERR_ARG. */
nh_status nh_get_profile(nh_grid* g, double* ms, long long* launches);

/* ---- Predictor step without any allocation (the paper has no counterpart:
   this entry point exists for callers that cannot allocate device memory) ----

   Some callers cannot call cudaMalloc or hand the library a workspace: a host
   framework that plans all device memory before it starts, a real-time loop
   that must not block in an allocator, or code that cannot keep a workspace
   alive between calls.  nh_predict_static runs the hydrostatic predictor of
   Sec. 3.1 (Heun, Eqs. 8-9; the same kernel nh_step uses) on the caller's
   device buffers for one member and keeps its scratch in a fixed device array
   inside the library, so it allocates nothing.

   h, hu, hw, d0: device, FP64, nx values each: thickness h > 0 (m), hu, hw
   (m^2/s) at time t, static depth d0 (m).  h_out, hu_out, hw_out: device,
   FP64, nx values: the predicted state at t + dt (no non-hydrostatic
   correction); each output must not alias its input.  slide: host pointer to
   the member's bottom motion, or NULL for a static bottom.  mass: host
   pointer receiving sum(h_out) dx, or NULL; when non-NULL the call
   synchronises `stream`, so mass must be NULL while `stream` is being
   captured (NH_ERR_ARG otherwise).  Geometry arguments as in nh_grid_desc
   (one member); slide values must be finite.
   Limits: 8 <= nx <= NH_STATIC_MAX_CELLS, else NH_ERR_ARG.
   The scratch array (about 2.2 MB) is held by every GPU that loads the
   library until the process exits.  The first call on a device looks up the
   array's device address (cudaGetSymbolAddress) with that device current;
   make that first call before any stream capture.  All calls share the
   array, so calls that overlap on the GPU race; issue them on one stream.
   Errors: NH_ERR_ARG, NH_ERR_CUDA (also returned, with nothing launched,
   when a CUDA error from earlier work is still pending).  With mass == NULL
   the call reports launch errors only; a fault inside its kernels surfaces
   at the caller's next synchronisation of `stream`. */
#define NH_STATIC_MAX_CELLS 262144
nh_status nh_predict_static(const double* h, const double* hu, const double* hw,
                            const double* d0, double* h_out, double* hu_out, double* hw_out,
                            int nx, double dx, double x0, int bc, int limiter, double g,
                            const nh_slide_desc* slide, double t, double dt, double* mass,
                            void* stream);

/* Release the handle (the workspace stays the caller's). */
void nh_destroy(nh_grid* g);

const char* nh_status_string(nh_status s);

#ifdef __cplusplus
}
#endif
#endif /* NHSWE_H */
