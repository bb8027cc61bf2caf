// nh_internal.cuh -- device-side building blocks of the 1D library path.
//
// State on the GPU: zeta = h - d0 (deviation of the thickness from the static
// depth), hu, hw.  eta = zeta + m and h = zeta + d0, where m is the moving
// mound (d = d0 - m), so the surface is formed from two small numbers and an
// FP32 state keeps sub-nanometre resolution of eta.
//
// Unknown used on the GPU: psi = (dt / rho) h~ p^nh.  With this scaling the
// elliptic problem of Sec. 3.2 (Eqs. 10-13 with the constraint Eq. 4
// eliminated) reads
//     -(Kc psi_x)_x + gam psi = R,
//     Kc  = 4 / (h D),  D = 4 + d_x^2,
//     gam = beta_x + 12 (1 + d_x^2) / (h^3 D),   beta = 6 d_x / (h^2 D),
//     R   = -[(U0/h)_x + 2 d_x U0 / h^2 + 2 hw~ / h^2 + 2 phi' / h^2 + 2 d_t / h],
//     U0  = hu~ + phi' d_x,
//     phi'= dt h / D (g d_x eta_x - d_tt - 2 u d_xt - u^2 d_xx)   (= dt phi / rho, Eq. 5),
// and the correction (Eqs. 10-11) is
//     P'  = 6 psi / (h D) + d_x psi_x / D + phi',
//     hu  = hu~ - psi_x + d_x P',   hw = hw~ + P',   h = h~.
// rho only rescales the reported pressure p^nh = rho psi / (dt h).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "nhswe.h"

namespace nh {

constexpr int kPredTile = 256;   // default cells per predictor CTA (autotuned: 128, 256, 512)
constexpr int kPredTileMax = 512;
constexpr int kPredTileMin = 128;
constexpr int kPredHalo = 5;     // two Heun stages + one cell for the criterion
constexpr int kChunk = 256;      // active cells per solver work item (= blockDim)
constexpr int kMaxExt = 6;       // extra couplings of a row beyond its list neighbours (2D: S, N, 4 diagonals)
constexpr int kCompactThreads = 1024;
constexpr int kPcrThreads = 1024;     // preconditioner CTA
constexpr int kPcrRows = 8192;        // active cells per preconditioner block (power of 2)
constexpr int kPcrLevels = 13;        // cyclic-reduction levels of a full block
static_assert((1 << kPcrLevels) == kPcrRows, "kPcrLevels = log2(kPcrRows)");

// Beyond xi^2 = 40 the Gaussian mound is below exp(-40) A = 4.3e-18 A: under
// half an ulp (>= 2^-54 d0) of the depth it is subtracted from whenever
// A < 12 d0, so its value and derivative terms are taken as 0 there instead
// of evaluating exp.
constexpr double kMoundCut = 40.0;

// Per-member slide parameters (device copy of nh_slide_desc, FP64).
// Shapes (NH_SLIDE_*): GAUSS_LNCOSH m = A exp(-((x - xc0 - s)/L)^2) with
// s = s0 ln cosh(t/t0); PLATE_EXP m = A s on |x - xc0| < L with the time
// factor s = 1 - exp(-t/t0) (Sec. 4.2); QUARTIC m = A (1 - xi^4) on |xi| < 1,
// xi = 2 (x - xc0 - s)/L, s = S(t) the sliding block's position (Sec. 4.3:
// acceleration s0 up to t0, glide at s0 t0 up to t2, deceleration up to
// t2 + t0, at rest after).
struct Slide {
    double A, L, xc0, s0, t0;
    double iL;    // 1 / L (set on the host with L)
    double t2;    // QUARTIC: end of the glide
    int shape;
    int pad;
};

// s(t), s'(t), s''(t) of a slide (the mound's displacement, the plate's time
// factor or the block's position, see Slide).
__host__ __device__ __forceinline__ void slide_law(const Slide& sl, double t, double* s, double* sd, double* sdd)
{
    *s = 0.0; *sd = 0.0; *sdd = 0.0;
    if (sl.shape == NH_SLIDE_GAUSS_LNCOSH) {
        const double z = t / sl.t0, c = cosh(z);
        *s = sl.s0 * log(c);
        *sd = (sl.s0 / sl.t0) * tanh(z);
        *sdd = (sl.s0 / (sl.t0 * sl.t0)) / (c * c);
    } else if (sl.shape == NH_SLIDE_PLATE_EXP) {
        const double e = exp(-t / sl.t0);
        *s = 1.0 - e;
        *sd = e / sl.t0;
        *sdd = -e / (sl.t0 * sl.t0);
    } else if (sl.shape == NH_SLIDE_QUARTIC) {
        const double a0 = sl.s0, t1 = sl.t0, t2 = sl.t2, t3 = t2 + t1, ut = a0 * t1;
        const double S1 = 0.5 * a0 * t1 * t1;
        if (t <= 0.0) {
        } else if (t <= t1) {
            *s = 0.5 * a0 * t * t; *sd = a0 * t; *sdd = a0;
        } else if (t <= t2) {
            *s = S1 + ut * (t - t1); *sd = ut;
        } else if (t <= t3) {
            *s = S1 + ut * (t - t1) - 0.5 * a0 * (t - t2) * (t - t2);
            *sd = ut - a0 * (t - t2); *sdd = -a0;
        } else {
            *s = S1 + ut * (t3 - t1) - 0.5 * a0 * (t3 - t2) * (t3 - t2);
        }
    }
}

// Per-member slide kinematics at t^n and t^{n+1}: position s and, at t^{n+1},
// its first and second time derivatives.
struct Kin {
    double s_n, s_n1, sd_n1, sdd_n1;
};

// Per-member solver scalars (FP64) and bookkeeping.
struct MState {
    double bnorm2;     // ||R||^2
    double bnorm;      // ||R||
    double rr;         // CG: <r,r>; BiCGStab: rho = <rhat, r>
    double alpha, beta, omega;
    double rel_res;
    double min_gamma;
    double snorm;      // BiCGStab: ||s|| of the current iteration
    double rz;         // PCG: <r, z>
    int status;        // nh_status
    int iters;
    int done;          // 1 once converged / failed
    int kind;          // NH_SOLVER_CG or NH_SOLVER_BICGSTAB
    int zero_sol;      // R == 0: solution is exactly zero
    int s_conv;        // BiCGStab: converged on s this iteration
    int n_active;
    int nchunks;
    int auto_kind;     // AUTO: CG first, BiCGStab if CG detects indefiniteness
    int npb;           // preconditioner blocks
    int ioff;          // first work item (kChunk cells) of this member in the item list
    int poff;          // first preconditioner block of this member in the block list
};

// MState.status value (never returned): CG broke down on an AUTO member,
// which is then solved again by BiCGStab.
constexpr int kStatusFallback = 100;

// Device-side time stepping of a captured run: t^n = t_base + n dt.  A failed
// step sets `abort` (and `fail_step`); the kernels that write the state or the
// pressure then stand down, so the last committed state stays intact.
struct TimeCtl {
    double t_base;
    double dt;
    long long n;          // steps since t_base
    long long done;       // steps committed in this run
    long long iters_total;   // Krylov iterations summed over committed steps
    long long active_total;  // active cells summed over committed steps
    int abort;
    int fail_status;
    int prev_ok;          // psi holds the previous step's solution for this dt
    int pad;
};

// Counters shared by all members (device).
struct Ctl {
    int not_done;      // members still iterating
    int n_cg, n_bicg;  // members per solver kind after set-up
    int ir_pending;    // mixed path: members needing another refinement pass
    int n_fallback;    // AUTO members whose CG broke down in this solve
    int n_items;       // work items (member, chunk of kChunk active cells) this step
    int n_pitems;      // preconditioner blocks (member, kPcrRows active cells) this step
    int timeout;       // a bounded grid barrier gave up (persistent solve)
    unsigned bar_count;         // grid barrier: arrivals
    unsigned bar_gen;           // grid barrier: generation
    int go[2];                  // persistent solve: continue flag per iteration parity
    int max_npb;                // largest number of preconditioner blocks of a member this step
};

__device__ __forceinline__ int resolve(int j, int n, int bc, int* sgn)
{
    // In-domain cell for index j (|j| small beyond the ends); *sgn = -1 when a
    // wall mirror flips odd quantities (u, hu, d_x, ...).
    if (j >= 0 && j < n) { *sgn = 1; return j; }
    if (bc == NH_BC_PERIODIC) { *sgn = 1; int r = j % n; return r < 0 ? r + n : r; }
    *sgn = -1;
    return j < 0 ? (-1 - j) : (2 * n - 1 - j);
}

template <typename T> __device__ __forceinline__ T tabs(T v) { return v < T(0) ? -v : v; }
__device__ __forceinline__ double texp(double v) { return exp(v); }
__device__ __forceinline__ float texp(float v) { return expf(v); }
__device__ __forceinline__ double tsqrt(double v) { return sqrt(v); }
__device__ __forceinline__ float tsqrt(float v) { return sqrtf(v); }
// Gravity-wave speed sqrt(g h) for the Rusanov dissipation coefficient
// s = max(|u| + sqrt(g h)) over a face: s only scales the numerical
// diffusion (the flux stays consistent and conservative for any s), so it is
// taken in FP32 (relative error 6e-8) even on the FP64 path, sparing two
// FP64 square roots per face on GB300's narrow FP64 pipe.
__device__ __forceinline__ double wave_sqrt(double v) { return (double)sqrtf((float)v); }
__device__ __forceinline__ float wave_sqrt(float v) { return sqrtf(v); }


// Height of the moving mound at the centre of cell c (already resolved) at
// displacement s: m = A exp(-xi^2), xi = (x_c - xc0 - s) / L; the depth is
// d = d0 - m.
template <typename T>
__device__ __forceinline__ T mound_at(int c, double x0, double dx, const Slide& sl, double s)
{
    if (sl.shape == NH_SLIDE_GAUSS_LNCOSH) {
        const double xc = x0 + (c + 0.5) * dx;
        const T xi = T((xc - sl.xc0 - s) * sl.iL);
        if (xi * xi > T(kMoundCut)) return T(0);
        return T(sl.A) * texp(-xi * xi);
    }
    if (sl.shape == NH_SLIDE_PLATE_EXP) {
        const double xc = x0 + (c + 0.5) * dx;
        return fabs(xc - sl.xc0) < sl.L ? T(sl.A * s) : T(0);
    }
    if (sl.shape == NH_SLIDE_QUARTIC) {
        const double xc = x0 + (c + 0.5) * dx;
        const double xi = 2.0 * (xc - sl.xc0 - s) / sl.L;
        if (!(fabs(xi) < 1.0)) return T(0);
        const double xi2 = xi * xi;
        return T(sl.A * (1.0 - xi2 * xi2));
    }
    return T(0);
}

template <typename T>
__device__ __forceinline__ T depth_at(const T* __restrict__ d0m, int c, double x0, double dx,
                                      const Slide& sl, double s)
{
    return d0m[c] - mound_at<T>(c, x0, dx, sl, s);
}

template <typename T>
struct Bottom {
    T d, d_x, d_xx, d_t, d_xt, d_tt;
    T m;          // the mound's height (0 without a slide)
};

// Depth and its x/t derivatives at cell i (in the domain) at t^{n+1}: central
// differences of d0 (ghosts mirrored or wrapped), analytic mound terms.
template <typename T>
__device__ __forceinline__ Bottom<T> bottom_full(const T* __restrict__ d0m, int i, int nx, int bc,
                                                 double x0, double dx, const Slide& sl, const Kin& k)
{
    int sg;
    int im = resolve(i - 1, nx, bc, &sg), ip = resolve(i + 1, nx, bc, &sg);
    const T dxT = T(dx);
    Bottom<T> B;
    T a = d0m[im], c = d0m[i], e = d0m[ip];
    B.d = c;
    B.d_x = (e - a) / (T(2) * dxT);
    B.d_xx = (e - T(2) * c + a) / (dxT * dxT);
    const T iL = T(sl.iL), iL2 = iL * iL;
    B.d_t = T(0); B.d_xt = T(0); B.d_tt = T(0); B.m = T(0);
    if (sl.shape == NH_SLIDE_GAUSS_LNCOSH) {
        const T L = T(sl.L);
        double xc = x0 + (i + 0.5) * dx;
        T xi = T((xc - sl.xc0 - k.s_n1) * sl.iL);   // as in mound_at: B.m == mound_at
        T m = xi * xi > T(kMoundCut) ? T(0) : T(sl.A) * texp(-xi * xi);
        T sd = T(k.sd_n1), sdd = T(k.sdd_n1);
        T two_xi2m1 = T(2) * xi * xi - T(1);
        T m_x = m * (T(-2) * xi * iL);
        T m_xx = m * (T(4) * xi * xi - T(2)) * iL2;
        T m_t = m * (T(2) * xi * iL) * sd;
        T m_xt = -m * (T(2) * iL2) * two_xi2m1 * sd;
        T m_tt = m * (T(2) * iL2) * (two_xi2m1 * sd * sd + xi * L * sdd);
        B.d -= m; B.d_x -= m_x; B.d_xx -= m_xx; B.m = m;
        B.d_t = -m_t; B.d_xt = -m_xt; B.d_tt = -m_tt;
    } else if (sl.shape == NH_SLIDE_PLATE_EXP) {
        // vertical motion only; the plate's edges are a jump of the depth
        const double xc = x0 + (i + 0.5) * dx;
        if (fabs(xc - sl.xc0) < sl.L) {
            const T m = T(sl.A * k.s_n1);
            B.d -= m; B.m = m;
            B.d_t = T(-sl.A * k.sd_n1);
            B.d_tt = T(-sl.A * k.sdd_n1);
        }
    } else if (sl.shape == NH_SLIDE_QUARTIC) {
        const double xc = x0 + (i + 0.5) * dx;
        const double xi = 2.0 * (xc - sl.xc0 - k.s_n1) / sl.L;   // as in mound_at
        if (fabs(xi) < 1.0) {
            const double L = sl.L, A = sl.A, Sd = k.sd_n1, Sdd = k.sdd_n1;
            const double xi2 = xi * xi, xi3 = xi2 * xi;
            const double m = A * (1.0 - xi2 * xi2);
            const double m_x = -8.0 * A * xi3 / L;
            const double m_xx = -48.0 * A * xi2 / (L * L);
            const double m_t = 8.0 * A * xi3 * Sd / L;
            const double m_xt = 48.0 * A * xi2 * Sd / (L * L);
            const double m_tt = (8.0 * A / L) * (-6.0 * xi2 * Sd * Sd / L + xi3 * Sdd);
            B.d -= T(m); B.d_x -= T(m_x); B.d_xx -= T(m_xx); B.m = T(m);
            B.d_t = T(-m_t); B.d_xt = T(-m_xt); B.d_tt = T(-m_tt);
        }
    }
    return B;
}

// Reductions ---------------------------------------------------------------

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}
__device__ __forceinline__ double warp_min(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmin(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

// Block-wide sum of NV doubles; result valid in thread 0.  `sh` needs
// NV * 32 doubles.  Ends with __syncthreads() so `sh` can be reused.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV], double* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        double s = warp_sum(v[q]);
        if (lane == 0) sh[q * 32 + wid] = s;
    }
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int q = 0; q < NV; ++q) {
            double s = (lane < nw) ? sh[q * 32 + lane] : 0.0;
            v[q] = warp_sum(s);
        }
    }
    __syncthreads();
}

__device__ __forceinline__ double block_min(double v, double* sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    double s = warp_min(v);
    if (lane == 0) sh[wid] = s;
    __syncthreads();
    if (wid == 0) {
        double t = (lane < nw) ? sh[lane] : INFINITY;
        v = warp_min(t);
    }
    __syncthreads();
    return v;
}

}  // namespace nh
