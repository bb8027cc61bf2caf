/* nhswe_cnn.h -- the learned initial guess of the elliptic solve.
 *
 * The paper has no counterpart: it solves the non-hydrostatic system of
 * Sec. 3.2 (Eqs. 12-13) with a Krylov method and says nothing of how the
 * iteration is started.  This part starts it from the next pressure unknown
 * extrapolated in time from the method's own recent solutions, corrected by
 * a small convolutional network trained on pairs the method itself
 * produces.  The network cannot change the converged answer: the solve stops
 * on the same residual test (||R - A q|| <= rtol ||R||) whatever its starting
 * point, and a step whose solve fails from the learned start is solved again
 * from the plain warm start (NH_GUESS_PREV).
 *
 * Network: four width-3 convolutions along each member's cells, channels
 * 16 -> 32 -> 32 -> 32 -> 16, ReLU after the first three, zero padding
 * outside the member; the output is channel 0 of the last layer.  BF16
 * operands on the tensor cores, FP32 accumulation, FP32 parameters:
 *   params = per layer l = 0..3: W_l[c_out][3 c_in] then b_l[c_out], where
 *   column k c_in + c of W_l weights input channel c of the cell at offset
 *   k - 1 (k = 0, 1, 2); NH_CNN_PARAMS floats in all.
 *
 * History: psi^n is the pressure unknown of the last step (zero off its
 * active cells), psi^{n-1} and psi^{n-2} the two before.  On a cell where
 * psi^n and psi^{n-1} are both nonzero the first difference is
 * d1 = psi^n - psi^{n-1}; where psi^{n-2} is nonzero as well the second
 * difference is D2 = d1 - (psi^{n-1} - psi^{n-2}) (zero elsewhere, and until
 * the solutions exist).  S1 = max |d1| and S2 = max |D2| over all cells.
 *
 * Features (BF16, NH_CNN_IN per cell, cell-major [nbatch * pitch][16]) for
 * the step n -> n+1:
 *   0: d1 / S1     1: (psi^{n-1} - psi^{n-2}) / S1 where D2 is defined
 *   2: 1 on cells marked for step n+1      3: 1 where psi^n != 0
 *   4: D2 / S2     5: 1 where D2 is defined     6..15: 0 (reserved)
 * Candidates for the start of the solve on a marked cell: (0) psi^n, the
 * plain warm start; (1) the extrapolation psi^n + d1 + D2 (terms that are
 * not defined are dropped: quadratic, linear or none); (2) the extrapolation
 * plus S2 y, y the network's output, where D2 is defined (psi^n alone where
 * S2 y is not finite).  Before each solve the candidates are judged, per
 * member and with the operator of that step, by the energy CG minimises:
 * ||x0 - q||_A^2, q the solution, computed as the difference
 * J(x0) - J(psi^n), J(x) = x.Ax - 2 x.R, from x0 - psi^n and the warm start's
 * residual.  The lowest wins (ties go to the lower number), so the learned
 * start is used only where it is the better one.
 * Target (harvest): what the extrapolation misses,
 * (psi^{n+1} - psi^n - d1 - D2) / S2, on marked cells where D2 is defined.
 *
 * Layouts: "cells" arrays are member-major with a row pitch (`pitch` cells
 * per member, member b's cell i at b * pitch + i); nx_dev[b] (device) holds
 * member b's cell count (<= pitch).  All pointers are device pointers unless
 * stated; the library never frees or keeps them past the call.
 * Errors: NH_ERR_ARG (bad pointer, size or alignment), NH_ERR_CUDA (launch
 * or copy failed), NH_ERR_TIMEOUT (a tensor-core completion wait gave up
 * after about one second: results are incomplete, the context stays usable),
 * NH_ERR_STATE (handle calls made in the wrong order).
 */
#ifndef NHSWE_CNN_H
#define NHSWE_CNN_H

#include "nhswe.h"

#ifdef __cplusplus
extern "C" {
#endif

#define NH_CNN_PARAMS 9328
#define NH_CNN_IN 16

/* ---- standalone network calls (training and evaluation) ---- */

/* y[b * pitch + i] = out_scale * net(feat)[b * pitch + i] for i < nx_dev[b];
   other entries of y are left untouched.  feat: [nbatch * pitch][16] BF16,
   16-byte aligned; pitch % 8 == 0.  status_dev: NULL or a device int set to
   NH_ERR_TIMEOUT if a completion wait gave up (never cleared by the call).
   Asynchronous on `stream`. */
nh_status nh_cnn_forward(const void* feat, const int* nx_dev, int nbatch, int pitch,
                         const float* params, float* y, float out_scale, int* status_dev,
                         void* stream);

/* Scratch bytes nh_cnn_loss_grad needs for nbatch x pitch cells. */
size_t nh_cnn_workspace_bytes(int nbatch, int pitch);

/* Loss L = sum(mask (y - target)^2) / max(1, mask_count) over the cells
   i < nx_dev[b] and its gradient w.r.t. params (FP32, NH_CNN_PARAMS floats,
   overwritten).  target: FP32 cells; mask: bytes (nonzero = counted) cells;
   mask_count: the number of counted cells.  loss: host pointer or NULL.
   ws: 256-byte aligned device scratch of nh_cnn_workspace_bytes bytes.
   Synchronises `stream` (to read the loss and the status). */
nh_status nh_cnn_loss_grad(const void* feat, const int* nx_dev, int nbatch, int pitch,
                           const float* params, const float* target, const unsigned char* mask,
                           long long mask_count, float* grad, double* loss, void* ws,
                           size_t ws_bytes, void* stream);

/* One Adam update (beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected for
   `step` >= 1): params -= lr m_hat / (sqrt(v_hat) + eps); m, v: FP32 moments
   (NH_CNN_PARAMS each, zero before step 1).  Asynchronous on `stream`. */
nh_status nh_cnn_adam(float* params, const float* grad, float* m, float* v, int step, float lr,
                      void* stream);

/* ---- the network inside a solver handle ---- */

/* Device bytes the handle's guess buffers take (history, features, output,
   parameters); 0 on a bad handle. */
size_t nh_cnn_attach_bytes(const nh_grid* g);

/* Give the handle its guess buffers (device, 256-byte aligned, at least
   nh_cnn_attach_bytes; the caller keeps them alive until nh_destroy) and
   start the solution history empty.  Afterwards each step keeps the last
   three solutions, which nh_set_solver(..., NH_GUESS_CNN, ...) and
   nh_cnn_record need.  Synchronises the handle's stream. */
nh_status nh_cnn_attach(nh_grid* g, void* ws, size_t ws_bytes);

/* Copy NH_CNN_PARAMS FP32 parameters (device pointer) into the handle; later
   steps (captured runs included) use them.  Errors: NH_ERR_STATE before
   nh_cnn_attach. */
nh_status nh_cnn_set_params(nh_grid* g, const float* params_dev);

/* record != 0: build the features every step even when the solve does not
   start from the network, so nh_cnn_harvest can collect training pairs from
   the plain method.  Errors: NH_ERR_STATE before nh_cnn_attach. */
nh_status nh_cnn_record(nh_grid* g, int record);

/* Solves started from each candidate since nh_cnn_attach or the last
   nh_set_state, one count per member and step with active cells: counts[0]
   the previous pressure, counts[1] the extrapolation psi^n + d1 + D2,
   counts[2] the extrapolation corrected by the network.  Synchronises the
   handle's stream.  Errors: NH_ERR_STATE before nh_cnn_attach. */
nh_status nh_cnn_choices(nh_grid* g, long long* counts);

/* After a step that built features (record mode or NH_GUESS_CNN): copy that
   step's features (feat_out: [nbatch * pitch][16] BF16), its target
   (target_out: FP32 cells) and its mask (mask_out: bytes, 1 on the cells
   that carry a target; all 0 when S2 was 0, i.e. no sample) into
   the caller's device buffers, and return the target's scale S2 (host, may
   be NULL) and the row pitch (host, may be NULL).  Synchronises the
   handle's stream.
   Errors: NH_ERR_STATE when no features were built. */
nh_status nh_cnn_harvest(nh_grid* g, void* feat_out, float* target_out, unsigned char* mask_out,
                         double* scale, int* pitch);

#ifdef __cplusplus
}
#endif
#endif /* NHSWE_CNN_H */
