// nh_cnn.cuh -- launch interface of the learned-guess kernels (nh_cnn.cu)
// used by the solver handle.  Every function enqueues on `st` and returns the
// launch status; none synchronises.
#pragma once

#include "nh_internal.cuh"
#include "nhswe_cnn.h"

namespace nh {
namespace cnn {

// Device control block of the learned guess (inside the handle's buffers).
struct GuessCtl {
    unsigned long long smax1_bits;  // max |d1| (first differences) as the bits of a non-negative double
    unsigned long long smax2_bits;  // max |D2| (second differences)
    double S1_used, S2_used;        // scales of the features built last
    int v1, v2;                     // psi^{n-1}, psi^{n-2} exist
    int built;                      // features of the last step exist
    int status;                     // NH_ERR_TIMEOUT from a tensor-core wait
    unsigned long long counts[3];   // solves started from: previous pressure, extrapolation, network
};

struct GuessBufs {
    double* h1;        // psi^{n-1}, dense [nb * pitch]
    double* h2;        // psi^{n-2}
    void* feat;        // BF16 [nb * pitch][16]
    float* y;          // network output [nb * pitch]
    double* guess;     // psi^n + d1 + D2 + S2 y, then the judged start, dense [nb * pitch]
    double* base;      // psi^n + d1 + D2 (extrapolation alone), dense [nb * pitch]
    int* choice;       // per member: 0 previous pressure, 1 extrapolation, 2 network
    double* d2;        // D2 of the step being solved, dense [nb * pitch]
    float* params;     // NH_CNN_PARAMS
    GuessCtl* ctl;
};

struct GuessGeo {
    int nb, pitch, wpitch;
    const int* nxv;        // cells per member (device)
    const uint32_t* act;   // mask bits of the step being solved, [nb][wpitch]
    const double* psi;     // psi^n, dense
    const TimeCtl* tc;     // captured runs: stand down after an aborted step
    int sms;
};

// Opt the tensor-core kernels into their shared memory on the current device
// (call outside stream capture).
cudaError_t prepare_device();
// Scale S and the features of the step being solved.
cudaError_t launch_features(const GuessBufs& B, const GuessGeo& G, cudaStream_t st);
// Network output and the guess psi^n + d1 + D2 + S2 y.
cudaError_t launch_guess(const GuessBufs& B, const GuessGeo& G, cudaStream_t st);
// guess = the candidate each member's judge chose (choice[b]).
cudaError_t launch_select(const GuessBufs& B, const GuessGeo& G, cudaStream_t st);
// After an accepted solve, before psi is overwritten: h2 = h1, h1 = psi^n.
cudaError_t launch_shift(const GuessBufs& B, const GuessGeo& G, cudaStream_t st);
// Target (second difference of psi^{n+1} in units of S2) and mask of the last step.
cudaError_t launch_harvest(const GuessBufs& B, const GuessGeo& G, float* target, unsigned char* mask,
                           cudaStream_t st);

}  // namespace cnn
}  // namespace nh
