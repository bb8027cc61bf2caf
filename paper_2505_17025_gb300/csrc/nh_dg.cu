// nh_dg.cu -- the discontinuous Galerkin path (nhswe_dg.h): the paper's own
// discretisation, DG-P1 predictor and LDG mixed (p, hu) solve (Sec. 3.1-3.2),
// on batches of 1D grids with walls at both ends, FP64 throughout.
//
// Per step (one CUDA graph node each; all members in every launch):
//   k_dg_kin      slide position / velocity / acceleration per member at t^n, t^{n+1}
//   k_dg_predict  both Heun stages of Sec. 3.1 in one launch (a tile of
//                 elements plus one halo element per stage in shared memory),
//                 the criterion of Sec. 5.1 per element, mass partial sums
//   k_dg_compact  enlargement by whole elements (Sec. 5.2), list of marked elements
//   k_dg_local    per marked element: Eq. 12-13 coefficients at its nodes; hu as an
//                 affine function of p (Eq. 12 rows, inverted through the element's
//                 s12-weighted mass matrix); the element's own part of the p-system
//   k_dg_form     the left neighbour's part of the p-system (flip-flop coupling)
//   k_cr_reduce   block cyclic reduction of the 2x2-block tridiagonal p-system,
//                 one launch per level while a member has more than kCrSmemRows rows
//   k_cr_small    the remaining levels, top solve and their back-substitution in
//                 shared memory, one CTA per member
//   k_cr_back     back-substitution of the global levels
//   k_dg_correct  hu and hw (Eq. 11), p; residual and finiteness of the solution
//   k_dg_finish   step summary and acceptance (device-side time and counters)
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "nh_internal.cuh"
#include "nhswe_dg.h"

using namespace nh;

namespace {

constexpr int kDgTile = 256;       // elements per predictor CTA (= blockDim)
constexpr int kDgThreads = 256;    // threads of the per-element kernels
constexpr int kCrSmemRows = 512;   // rows a member may still have when k_cr_small takes over
constexpr int kCrSmallThreads = 256;
constexpr int kMaxLevels = 24;
constexpr int kCrSmallRows = 2 * kCrSmemRows + 16;   // rows of every level of a member in k_cr_small
constexpr size_t kCrSmallSmem = (size_t)kCrSmallRows * (14 + 2) * sizeof(double);

// Slide kinematics of one member at t^n and t^{n+1}.
struct DgKin {
    double s_n, sd_n, sdd_n;
    double s_n1, sd_n1, sdd_n1;
};

// Device-side time and step acceptance.  t^n = t0 + n dt.
struct DgTime {
    double t0, dt;
    long long n;          // steps since t0
    long long steps;      // steps since the state was set (first-step-global rule)
    long long done;       // steps committed by this run
    long long active_total;
    int abort;
    int fail_status;
};

// Per-step summary for the host.
struct DgSummary {
    double mass;
    double rel_res;
    long long n_active;
    int n_active_max;
    int status;
};

// The bottom at a node: the static part from the nodal depths (its P1 slope
// on the element), the moving part analytic.
struct NodeBottom {
    double d, d_x, d_xx, d_t, d_xt, d_tt;
};

__device__ __forceinline__ NodeBottom node_bottom(double d0, double d0_slope, double x, const Slide& sl,
                                                  double s, double sd, double sdd)
{
    NodeBottom B;
    B.d = d0; B.d_x = d0_slope; B.d_xx = 0.0; B.d_t = 0.0; B.d_xt = 0.0; B.d_tt = 0.0;
    if (sl.shape == NH_SLIDE_GAUSS_LNCOSH) {
        const double iL = sl.iL, xi = (x - sl.xc0 - s) * iL;
        if (xi * xi > kMoundCut) return B;
        const double m = sl.A * exp(-xi * xi), q = 2.0 * xi * xi - 1.0;
        B.d -= m;
        B.d_x += m * 2.0 * xi * iL;
        B.d_xx -= m * (4.0 * xi * xi - 2.0) * iL * iL;
        B.d_t = -m * 2.0 * xi * iL * sd;
        B.d_xt = m * 2.0 * iL * iL * q * sd;
        B.d_tt = -m * 2.0 * iL * iL * (q * sd * sd + xi * sl.L * sdd);
    } else if (sl.shape == NH_SLIDE_PLATE_EXP) {
        if (fabs(x - sl.xc0) < sl.L) {
            B.d -= sl.A * s;
            B.d_t = -sl.A * sd;
            B.d_tt = -sl.A * sdd;
        }
    } else if (sl.shape == NH_SLIDE_QUARTIC) {
        const double L = sl.L, xi = 2.0 * (x - sl.xc0 - s) / L;
        if (fabs(xi) < 1.0) {
            const double A = sl.A, xi2 = xi * xi, xi3 = xi2 * xi;
            B.d -= A * (1.0 - xi2 * xi2);
            B.d_x += 8.0 * A * xi3 / L;
            B.d_xx += 48.0 * A * xi2 / (L * L);
            B.d_t = -8.0 * A * xi3 * sd / L;
            B.d_xt = -48.0 * A * xi2 * sd / (L * L);
            B.d_tt = -(8.0 * A / L) * (-6.0 * xi2 * sd * sd / L + xi3 * sdd);
        }
    }
    return B;
}

// x-derivative of the depth at a node (the only bottom term of the predictor).
__device__ __forceinline__ double node_dx(double d0_slope, double x, const Slide& sl, double s)
{
    double d_x = d0_slope;
    if (sl.shape == NH_SLIDE_GAUSS_LNCOSH) {
        const double xi = (x - sl.xc0 - s) * sl.iL;
        if (xi * xi <= kMoundCut) d_x += sl.A * exp(-xi * xi) * 2.0 * xi * sl.iL;
    } else if (sl.shape == NH_SLIDE_QUARTIC) {
        const double xi = 2.0 * (x - sl.xc0 - s) / sl.L;
        if (fabs(xi) < 1.0) d_x += 8.0 * sl.A * xi * xi * xi / sl.L;
    }
    return d_x;
}

// Depth at a node (the criterion's eta = h - d).
__device__ __forceinline__ double node_depth(double d0, double x, const Slide& sl, double s)
{
    if (sl.shape == NH_SLIDE_GAUSS_LNCOSH) {
        const double xi = (x - sl.xc0 - s) * sl.iL;
        return xi * xi > kMoundCut ? d0 : d0 - sl.A * exp(-xi * xi);
    }
    if (sl.shape == NH_SLIDE_PLATE_EXP) return fabs(x - sl.xc0) < sl.L ? d0 - sl.A * s : d0;
    if (sl.shape == NH_SLIDE_QUARTIC) {
        const double xi = 2.0 * (x - sl.xc0 - s) / sl.L;
        if (fabs(xi) < 1.0) { const double xi2 = xi * xi; return d0 - sl.A * (1.0 - xi2 * xi2); }
    }
    return d0;
}

__global__ void k_dg_kin(const Slide* __restrict__ sl, DgKin* __restrict__ kin, int nb, const DgTime* __restrict__ tc)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || tc->abort) return;
    const double tn = tc->t0 + (double)tc->n * tc->dt, tn1 = tn + tc->dt;
    DgKin k;
    slide_law(sl[b], tn, &k.s_n, &k.sd_n, &k.sdd_n);
    slide_law(sl[b], tn1, &k.s_n1, &k.sd_n1, &k.sdd_n1);
    kin[b] = k;
}

// ---------------------------------------------------------------- predictor

struct Geo {
    int ne, nb, pn, pe;   // elements, members, node pitch, element pitch
    double dx, x0, g, rho, c11;
};

struct PredArgs {
    Geo G;
    const double *h, *hu, *hw;     // Q^n (node pitch)
    double *ht, *hut, *hwt, *p;    // Q~ and p = 0 (the other state buffer)
    const double* d0;
    const Slide* slide;
    const DgKin* kin;
    uint8_t* marks;                // criterion per element
    double* mass_part;             // per CTA: sum dx (h_L + h_R) / 2 of Q~
    int crit;
    double knh;
    const DgTime* tc;
};

// Nodal flux F(Q) = (hu, hu u + g h^2 / 2, hu hw / h) and the wave speed
// |u| + sqrt(g h) of one node (Sec. 3.1): one reciprocal of h per node.  The
// element's volume term and both Rusanov fluxes touching the node reuse them.
struct NodeFlux {
    double f0, f1, f2, s;
};

__device__ __forceinline__ NodeFlux node_flux(double g, double h, double hu, double hw)
{
    const double ih = 1.0 / h, u = hu * ih;
    NodeFlux F;
    F.f0 = hu;
    F.f1 = hu * u + 0.5 * g * h * h;
    F.f2 = hu * hw * ih;
    F.s = fabs(u) + sqrt(g * h);
    return F;
}

// The predictor tile: elements [e0, e0 + T); stage 1 runs on [e0 - 1, e0 + T]
// and reads Q^n of [e0 - 2, e0 + T + 1].  Shared memory (doubles):
//   q   Q^n nodes of elements e0-2 .. e0+T+1      3 x 2 (T + 4)
//   qs  Q* nodes of elements e0-1 .. e0+T          3 x 2 (T + 2)
//   k1  H(Q^n) of the tile's own elements          3 x 2 T
//   nf  nodal fluxes and speeds of a stage         4 x 2 (T + 4)
//   fi  interface fluxes of a stage                3 x (T + 3)
constexpr int kQN = 2 * (kDgTile + 4), kQSN = 2 * (kDgTile + 2), kIF = kDgTile + 3;
constexpr size_t kPredSmem = sizeof(double) * (3 * kQN + 3 * kQSN + 3 * 2 * kDgTile + 4 * kQN + 3 * kIF + 32);

// One stage's nodal fluxes (nodes [n0, n0 + nn) of the smem array `q` with
// stride `qn`, the first at global node k0), then interface fluxes for the
// interfaces left of elements [ea, eb] (interface e between nodes 2e-1 and
// 2e; walls mirror the end node: (h, -hu, hw)).  Interface e is stored at
// fi[e - ea]; node k of the stage at nf[k - k0].
__device__ __forceinline__ void stage_fluxes(const Geo& G, const double* q, int qn, int k0, int kn, int ea, int eb,
                                             double* nf, double* fi, int tid)
{
    for (int j = tid; j < kn; j += kDgTile) {
        const int k = k0 + j;
        if (k < 0 || k >= 2 * G.ne) continue;
        const NodeFlux F = node_flux(G.g, q[j], q[qn + j], q[2 * qn + j]);
        nf[j] = F.f0; nf[kQN + j] = F.f1; nf[2 * kQN + j] = F.f2; nf[3 * kQN + j] = F.s;
    }
    __syncthreads();
    for (int j = tid; j <= eb - ea; j += kDgTile) {
        const int e = ea + j;
        if (e < 0 || e > G.ne) continue;
        // left state: node 2e-1 (or the mirror of node 0), right state: node 2e (or the mirror of node 2ne-1)
        int kl = 2 * e - 1 - k0, kr = 2 * e - k0;
        double hL, huL, hwL, hR, huR, hwR, FL0, FL1, FL2, FR0, FR1, FR2, sL, sR;
        if (e == 0) kl = kr;
        if (e == G.ne) kr = kl;
        hL = q[kl]; huL = q[qn + kl]; hwL = q[2 * qn + kl];
        hR = q[kr]; huR = q[qn + kr]; hwR = q[2 * qn + kr];
        FL0 = nf[kl]; FL1 = nf[kQN + kl]; FL2 = nf[2 * kQN + kl]; sL = nf[3 * kQN + kl];
        FR0 = nf[kr]; FR1 = nf[kQN + kr]; FR2 = nf[2 * kQN + kr]; sR = nf[3 * kQN + kr];
        if (e == 0) { huL = -huL; FL0 = -FL0; FL2 = -FL2; }
        if (e == G.ne) { huR = -huR; FR0 = -FR0; FR2 = -FR2; }
        const double s = sL > sR ? sL : sR;
        fi[j] = 0.5 * (FL0 + FR0) - 0.5 * s * (hR - hL);
        fi[kIF + j] = 0.5 * (FL1 + FR1) - 0.5 * s * (huR - huL);
        fi[2 * kIF + j] = 0.5 * (FL2 + FR2) - 0.5 * s * (hwR - hwL);
    }
    __syncthreads();
}

// H(Q) of Sec. 3.1 on element e from its nodal fluxes (smem index kk of its
// left node), its interface fluxes (index ii of its left interface) and the
// bottom slopes at its nodes: the weak form with the P1 mass matrix inverted,
// M^{-1} = (2/dx) [[2, -1], [-1, 2]], plus the nodal source g h d_x.
__device__ __forceinline__ void element_rate(const Geo& G, const double* nf, int kk, const double* fi, int ii,
                                             double hL, double hR, double dxL, double dxR, double out[3][2])
{
    const double c = 2.0 / G.dx;
#pragma unroll
    for (int f = 0; f < 3; ++f) {
        const double FL = nf[f * kQN + kk], FR = nf[f * kQN + kk + 1];
        const double rl = -0.5 * (FL + FR) + fi[f * kIF + ii];
        const double rr = 0.5 * (FL + FR) - fi[f * kIF + ii + 1];
        out[f][0] = c * (2.0 * rl - rr);
        out[f][1] = c * (-rl + 2.0 * rr);
    }
    out[1][0] += G.g * hL * dxL;
    out[1][1] += G.g * hR * dxR;
}

__global__ void __launch_bounds__(kDgTile) k_dg_predict(PredArgs a)
{
    extern __shared__ double pred_sm[];
    double* q = pred_sm;                 // [3][kQN]
    double* qs = q + 3 * kQN;            // [3][kQSN]
    double* k1 = qs + 3 * kQSN;          // [3][2T]
    double* nf = k1 + 3 * 2 * kDgTile;   // [4][kQN]
    double* fi = nf + 4 * kQN;           // [3][kIF]
    double* red = fi + 3 * kIF;          // [32]
    const Geo& G = a.G;
    const int b = blockIdx.y, e0 = blockIdx.x * kDgTile, tid = threadIdx.x;
    if (a.tc->abort) return;
    const size_t mb = (size_t)b * G.pn;
    const double dt = a.tc->dt;
    const Slide sl = a.slide[b];
    const DgKin kn = a.kin[b];
    // Q^n of elements e0-2 .. e0+T+1
    const int n0 = 2 * (e0 - 2);
    for (int j = tid; j < kQN; j += kDgTile) {
        const int k = n0 + j;
        if (k >= 0 && k < 2 * G.ne) {
            q[j] = a.h[mb + k]; q[kQN + j] = a.hu[mb + k]; q[2 * kQN + j] = a.hw[mb + k];
        }
    }
    __syncthreads();
    // stage 1 on elements e0-1 .. e0+T: Q* = Q^n + dt H(Q^n, t^n)
    stage_fluxes(G, q, kQN, n0, kQN, e0 - 1, e0 + kDgTile + 1, nf, fi, tid);
    for (int j = tid; j < kDgTile + 2; j += kDgTile) {
        const int e = e0 - 1 + j;
        if (e < 0 || e >= G.ne) continue;
        const int l = 2 * (j + 1);   // e's left node in q / nf
        const double slope = (a.d0[mb + 2 * e + 1] - a.d0[mb + 2 * e]) / G.dx;
        const double xL = G.x0 + e * G.dx, xR = G.x0 + (e + 1) * G.dx;
        double out[3][2];
        element_rate(G, nf, l, fi, j, q[l], q[l + 1], node_dx(slope, xL, sl, kn.s_n), node_dx(slope, xR, sl, kn.s_n),
                     out);
        const int ls = 2 * j;        // e's left node in qs
#pragma unroll
        for (int f = 0; f < 3; ++f) {
            qs[f * kQSN + ls] = q[f * kQN + l] + dt * out[f][0];
            qs[f * kQSN + ls + 1] = q[f * kQN + l + 1] + dt * out[f][1];
        }
        if (j >= 1 && j <= kDgTile) {
#pragma unroll
            for (int f = 0; f < 3; ++f) {
                k1[f * 2 * kDgTile + 2 * (j - 1)] = out[f][0];
                k1[f * 2 * kDgTile + 2 * (j - 1) + 1] = out[f][1];
            }
        }
    }
    __syncthreads();
    // stage 2 on the tile's own elements: Q~ = Q^n + dt/2 (k1 + H(Q*, t^{n+1}))
    stage_fluxes(G, qs, kQSN, 2 * (e0 - 1), kQSN, e0, e0 + kDgTile, nf, fi, tid);
    const int e = e0 + tid;
    double mass = 0.0;
    if (e < G.ne) {
        const int ls = 2 * (tid + 1);   // e's left node in qs / nf
        const double d0L = a.d0[mb + 2 * e], d0R = a.d0[mb + 2 * e + 1];
        const double slope = (d0R - d0L) / G.dx;
        const double xL = G.x0 + e * G.dx, xR = G.x0 + (e + 1) * G.dx;
        double out[3][2];
        element_rate(G, nf, ls, fi, tid, qs[ls], qs[ls + 1], node_dx(slope, xL, sl, kn.s_n1),
                     node_dx(slope, xR, sl, kn.s_n1), out);
        const int lq = 2 * (tid + 2);
        double qt[3][2];
#pragma unroll
        for (int f = 0; f < 3; ++f) {
#pragma unroll
            for (int s = 0; s < 2; ++s)
                qt[f][s] = q[f * kQN + lq + s] + 0.5 * dt * (k1[f * 2 * kDgTile + 2 * tid + s] + out[f][s]);
        }
        const size_t k = mb + 2 * e;
        a.ht[k] = qt[0][0]; a.ht[k + 1] = qt[0][1];
        a.hut[k] = qt[1][0]; a.hut[k + 1] = qt[1][1];
        a.hwt[k] = qt[2][0]; a.hwt[k + 1] = qt[2][1];
        a.p[k] = 0.0; a.p[k + 1] = 0.0;
        mass = G.dx * (0.5 * (qt[0][0] + qt[0][1]));
        // criterion of Sec. 5.1 on the element: the mean of its two nodal
        // values, the P1 slope for x-derivatives
        uint8_t mk = 0;
        if (a.crit == NH_CRIT_GLOBAL) {
            mk = 1;
        } else if (a.crit != NH_CRIT_HYDROSTATIC) {
            const double dL = node_depth(d0L, xL, sl, kn.s_n1), dR = node_depth(d0R, xR, sl, kn.s_n1);
            const double etaL = qt[0][0] - dL, etaR = qt[0][1] - dR;
            double v = 0.0;
            switch (a.crit) {
                case NH_CRIT_ETA_D: v = fabs(0.5 * (etaL + etaR) / (0.5 * (dL + dR))); break;
                case NH_CRIT_ETA_X: v = fabs((etaR - etaL) / G.dx); break;
                case NH_CRIT_U: v = fabs(0.5 * (qt[1][0] / qt[0][0] + qt[1][1] / qt[0][1])); break;
                case NH_CRIT_U_X: v = fabs((qt[1][1] / qt[0][1] - qt[1][0] / qt[0][0]) / G.dx); break;
                case NH_CRIT_W: v = fabs(0.5 * (qt[2][0] / qt[0][0] + qt[2][1] / qt[0][1])); break;
                case NH_CRIT_W_X: v = fabs((qt[2][1] / qt[0][1] - qt[2][0] / qt[0][0]) / G.dx); break;
                default: break;
            }
            mk = v > a.knh ? 1 : 0;
        }
        a.marks[(size_t)b * G.pe + e] = mk;
    }
    // per-CTA mass (summed by k_dg_finish)
    mass = warp_sum(mass);
    if ((tid & 31) == 0) red[tid >> 5] = mass;
    __syncthreads();
    if (tid < 32) {
        double v = tid < kDgTile / 32 ? red[tid] : 0.0;
        v = warp_sum(v);
        if (tid == 0) a.mass_part[(size_t)b * gridDim.x + blockIdx.x] = v;
    }
}

// ------------------------------------------------------------------- mask

// One CTA per member: an element is marked when a raw mark lies within
// `enlarge` elements (or every element, on a first-step-global step); the
// marked elements are listed in order.
__global__ void __launch_bounds__(1024) k_dg_compact(const uint8_t* __restrict__ marks, uint8_t* __restrict__ mask,
                                                     int* __restrict__ act, int* __restrict__ nact, int ne, int pe,
                                                     int enlarge, int first_global, const DgTime* __restrict__ tc)
{
    __shared__ int wsum[32];
    __shared__ int base;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (tc->abort) return;
    const bool all = first_global && tc->steps == 0;
    const uint8_t* mk = marks + (size_t)b * pe;
    if (tid == 0) base = 0;
    __syncthreads();
    for (int c0 = 0; c0 < ne; c0 += 1024) {
        const int i = c0 + tid;
        int on = 0;
        if (i < ne) {
            if (all) on = 1;
            else {
                const int lo = max(0, i - enlarge), hi = min(ne - 1, i + enlarge);
                for (int j = lo; j <= hi && !on; ++j) on = mk[j];
            }
            mask[(size_t)b * pe + i] = (uint8_t)on;
        }
        const unsigned bal = __ballot_sync(0xffffffffu, on);
        if (lane == 0) wsum[wid] = __popc(bal);
        __syncthreads();
        if (wid == 0) {
            int v = wsum[lane], s = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int t = __shfl_up_sync(0xffffffffu, s, o);
                if (lane >= o) s += t;
            }
            wsum[lane] = s - v;   // exclusive prefix of the warps
        }
        __syncthreads();
        if (on) act[(size_t)b * pe + base + wsum[wid] + __popc(bal & ((1u << lane) - 1u))] = i;
        __syncthreads();
        if (tid == 1023) base += wsum[wid] + __popc(bal);   // last warp's prefix + its count
        __syncthreads();
    }
    if (tid == 0) nact[b] = base;
}

// ----------------------------------------------------------- LDG assembly

// Structure-of-arrays planes of the per-element data (element pitch).
enum {
    kA0 = 0, kA1, kB00, kB01, kB10, kB11, kC0, kC1,   // hu_i = a + B p_i + (C0, C1) pL(i+1)
    kC6L, kC6R, kCxL, kCxR, kPhL, kPhR,              // correction: 6/D, d_x/D, phi at both nodes
    kLocalPlanes
};
// The p-system of one level: L (4), D (4), U (4), r (2), row-major 2x2 blocks.
enum { kL00 = 0, kL01, kL10, kL11, kD00, kD01, kD10, kD11, kU00, kU01, kU10, kU11, kR0, kR1, kSysPlanes };

struct LocalArgs {
    Geo G;
    const double *ht, *hut, *hwt, *d0;
    const Slide* slide;
    const DgKin* kin;
    const int *act, *nact;
    double* loc;        // kLocalPlanes planes of nb * pe
    double* sys;        // level-0 system: kSysPlanes planes of nb * pe
    size_t plane;       // nb * pe
    const DgTime* tc;
};

struct NodeCoef {
    double s11, s12, f1, s21, s22, f2, phi, D, d_x;
};

// Coefficients of Eqs. 12-13 at one node of element i (h_x and eta_x the
// element's P1 slopes; the bottom at t^{n+1}).
__device__ __forceinline__ NodeCoef node_coef(double rho, double g, double dt, double h, double hu, double hw,
                                              double h_x, double eta_x, const NodeBottom& B)
{
    NodeCoef c;
    const double u = hu / h;
    c.D = 4.0 + B.d_x * B.d_x;
    c.d_x = B.d_x;
    c.phi = rho * h / c.D * (g * B.d_x * eta_x - B.d_tt - 2.0 * u * B.d_xt - u * u * B.d_xx);
    c.s11 = (2.0 * h_x - 3.0 * B.d_x) / (2.0 * h);
    c.s12 = rho * c.D / (4.0 * dt * h);
    c.f1 = c.D / (4.0 * h) * (c.phi * B.d_x + rho / dt * hu);
    c.s21 = (3.0 * B.d_x - 2.0 * h_x) / (2.0 * h);
    c.s22 = 3.0 * dt / (rho * h);
    c.f2 = -2.0 * B.d_t - 2.0 * hw / h - B.d_x * hu / (2.0 * h) - dt * c.D * c.phi / (2.0 * rho * h);
    return c;
}

__global__ void __launch_bounds__(kDgThreads) k_dg_local(LocalArgs a)
{
    const Geo& G = a.G;
    const int b = blockIdx.y, j = blockIdx.x * kDgThreads + threadIdx.x;
    if (a.tc->abort) return;
    const int n = a.nact[b];
    if (j >= n) return;
    const size_t me = (size_t)b * G.pe, mb = (size_t)b * G.pn;
    const int i = a.act[me + j];
    const int mlft = (j > 0 && a.act[me + j - 1] == i - 1) ? 1 : 0;
    const int mrgt = (j < n - 1 && a.act[me + j + 1] == i + 1) ? 1 : 0;
    const double dt = a.tc->dt, rho = G.rho, c11 = G.c11, dx = G.dx;
    const Slide sl = a.slide[b];
    const DgKin kn = a.kin[b];
    const size_t kL = mb + 2 * i, kR = kL + 1;
    const double hL = a.ht[kL], hR = a.ht[kR];
    const double d0L = a.d0[kL], d0R = a.d0[kR], slope = (d0R - d0L) / dx;
    const double xL = G.x0 + i * dx, xR = G.x0 + (i + 1) * dx;
    const NodeBottom BL = node_bottom(d0L, slope, xL, sl, kn.s_n1, kn.sd_n1, kn.sdd_n1);
    const NodeBottom BR = node_bottom(d0R, slope, xR, sl, kn.s_n1, kn.sd_n1, kn.sdd_n1);
    const double h_x = (hR - hL) / dx, eta_x = ((hR - BR.d) - (hL - BL.d)) / dx;
    const NodeCoef cL = node_coef(rho, G.g, dt, hL, a.hut[kL], a.hwt[kL], h_x, eta_x, BL);
    const NodeCoef cR = node_coef(rho, G.g, dt, hR, a.hut[kR], a.hwt[kR], h_x, eta_x, BR);
    const double m6 = dx / 6.0;
    // Eq. 12 rows: P p_i + Q p_{i+1} + S hu_i = g1, S = m6 [[2 sL, sR], [sL, 2 sR]] (s = s12)
    const double P00 = -(double)mlft + 0.5 + 2.0 * m6 * cL.s11, P01 = 0.5 + m6 * cR.s11;
    const double P10 = -0.5 + m6 * cL.s11, P11 = -0.5 + 2.0 * m6 * cR.s11;
    const double g0 = m6 * (2.0 * cL.f1 + cR.f1), g1 = m6 * (cL.f1 + 2.0 * cR.f1);
    // S^{-1} = 1 / (3 m6) diag(1/sL, 1/sR) [[2, -1], [-1, 2]]
    const double iL = 1.0 / (3.0 * m6 * cL.s12), iR = 1.0 / (3.0 * m6 * cR.s12);
    const double Si00 = 2.0 * iL, Si01 = -iL, Si10 = -iR, Si11 = 2.0 * iR;
    const double A0 = Si00 * g0 + Si01 * g1, A1 = Si10 * g0 + Si11 * g1;
    const double B00 = -(Si00 * P00 + Si01 * P10), B01 = -(Si00 * P01 + Si01 * P11);
    const double B10 = -(Si10 * P00 + Si11 * P10), B11 = -(Si10 * P01 + Si11 * P11);
    const double C0 = mrgt ? -Si01 : 0.0, C1 = mrgt ? -Si11 : 0.0;   // Q = [[0, 0], [mrgt, 0]]
    // Eq. 13 rows: E hu_i + F p_i + (left: -mlft (hu_R(i-1) + c11 p_R(i-1))) + K p_{i+1} = r23
    const double E00 = 0.5 + 2.0 * m6 * cL.s21, E01 = 0.5 + m6 * cR.s21;
    const double E10 = -0.5 + m6 * cL.s21, E11 = 0.5 + 2.0 * m6 * cR.s21;
    const double F00 = c11 + 2.0 * m6 * cL.s22, F01 = m6 * cR.s22;
    const double F10 = m6 * cL.s22, F11 = c11 + 2.0 * m6 * cR.s22;
    double r2 = m6 * (2.0 * cL.f2 + cR.f2);
    const double r3 = m6 * (cL.f2 + 2.0 * cR.f2);
    if (!mlft) r2 += i > 0 ? a.hut[kL - 1] : 0.0;   // outside hu: the predicted one, 0 at the wall
    const size_t o = me + j, P = a.plane;
    double* L = a.loc;
    L[kA0 * P + o] = A0; L[kA1 * P + o] = A1;
    L[kB00 * P + o] = B00; L[kB01 * P + o] = B01; L[kB10 * P + o] = B10; L[kB11 * P + o] = B11;
    L[kC0 * P + o] = C0; L[kC1 * P + o] = C1;
    L[kC6L * P + o] = 6.0 / cL.D; L[kC6R * P + o] = 6.0 / cR.D;
    L[kCxL * P + o] = cL.d_x / cL.D; L[kCxR * P + o] = cR.d_x / cR.D;
    L[kPhL * P + o] = cL.phi; L[kPhR * P + o] = cR.phi;
    // the element's own part of its p-system row: D = E B + F, U = E C + K, r = r23 - E a
    double* Y = a.sys;
    Y[kD00 * P + o] = E00 * B00 + E01 * B10 + F00;
    Y[kD01 * P + o] = E00 * B01 + E01 * B11 + F01;
    Y[kD10 * P + o] = E10 * B00 + E11 * B10 + F10;
    Y[kD11 * P + o] = E10 * B01 + E11 * B11 + F11;
    Y[kU00 * P + o] = E00 * C0 + E01 * C1;
    Y[kU01 * P + o] = 0.0;
    Y[kU10 * P + o] = E10 * C0 + E11 * C1 - (mrgt ? c11 : 0.0);
    Y[kU11 * P + o] = 0.0;
    Y[kR0 * P + o] = r2 - (E00 * A0 + E01 * A1);
    Y[kR1 * P + o] = r3 - (E10 * A0 + E11 * A1);
}

// The left neighbour's part: row 0 of Eq. 13 holds -(hu_R(i-1) + c11 p_R(i-1))
// with hu_R(i-1) = a1 + B10 pL(i-1) + B11 pR(i-1) + C1 pL(i).
__global__ void __launch_bounds__(kDgThreads) k_dg_form(const int* __restrict__ act, const int* __restrict__ nact,
                                                        const double* __restrict__ loc, double* __restrict__ sys,
                                                        int pe, size_t plane, double c11, const DgTime* __restrict__ tc)
{
    const int b = blockIdx.y, j = blockIdx.x * kDgThreads + threadIdx.x;
    if (tc->abort) return;
    if (j >= nact[b]) return;
    const size_t me = (size_t)b * pe, o = me + j, P = plane;
    double l00 = 0.0, l01 = 0.0;
    if (j > 0 && act[me + j - 1] == act[me + j] - 1) {
        const size_t q = o - 1;
        l00 = -loc[kB10 * P + q];
        l01 = -(loc[kB11 * P + q] + c11);
        sys[kD00 * P + o] -= loc[kC1 * P + q];
        sys[kR0 * P + o] += loc[kA1 * P + q];
    }
    sys[kL00 * P + o] = l00; sys[kL01 * P + o] = l01;
    sys[kL10 * P + o] = 0.0; sys[kL11 * P + o] = 0.0;
}

// ------------------------------------------------- block cyclic reduction

struct M2 {
    double a, b, c, d;   // [[a, b], [c, d]]
};
__device__ __forceinline__ M2 m2_mul(const M2& x, const M2& y)
{
    return {x.a * y.a + x.b * y.c, x.a * y.b + x.b * y.d, x.c * y.a + x.d * y.c, x.c * y.b + x.d * y.d};
}
__device__ __forceinline__ M2 m2_inv(const M2& x)
{
    const double id = 1.0 / (x.a * x.d - x.b * x.c);
    return {x.d * id, -x.b * id, -x.c * id, x.a * id};
}
__device__ __forceinline__ M2 m2_sub(const M2& x, const M2& y) { return {x.a - y.a, x.b - y.b, x.c - y.c, x.d - y.d}; }

struct Row {
    M2 L, D, U;
    double r0, r1;
};
static_assert(sizeof(Row) == kSysPlanes * sizeof(double), "Row holds one p-system row");

__device__ __forceinline__ Row load_row(const double* __restrict__ s, size_t P, size_t o)
{
    Row R;
    R.L = {s[kL00 * P + o], s[kL01 * P + o], s[kL10 * P + o], s[kL11 * P + o]};
    R.D = {s[kD00 * P + o], s[kD01 * P + o], s[kD10 * P + o], s[kD11 * P + o]};
    R.U = {s[kU00 * P + o], s[kU01 * P + o], s[kU10 * P + o], s[kU11 * P + o]};
    R.r0 = s[kR0 * P + o]; R.r1 = s[kR1 * P + o];
    return R;
}
__device__ __forceinline__ void store_row(double* __restrict__ s, size_t P, size_t o, const Row& R)
{
    s[kL00 * P + o] = R.L.a; s[kL01 * P + o] = R.L.b; s[kL10 * P + o] = R.L.c; s[kL11 * P + o] = R.L.d;
    s[kD00 * P + o] = R.D.a; s[kD01 * P + o] = R.D.b; s[kD10 * P + o] = R.D.c; s[kD11 * P + o] = R.D.d;
    s[kU00 * P + o] = R.U.a; s[kU01 * P + o] = R.U.b; s[kU10 * P + o] = R.U.c; s[kU11 * P + o] = R.U.d;
    s[kR0 * P + o] = R.r0; s[kR1 * P + o] = R.r1;
}

// One cyclic-reduction step for row i of a level with n rows (neighbours
// i-1 and i+1 eliminated): the new row couples i-2 and i+2.
__device__ __forceinline__ Row cr_combine(const Row& C, const Row* Lf, const Row* Rt)
{
    Row N;
    N.L = {0.0, 0.0, 0.0, 0.0}; N.U = {0.0, 0.0, 0.0, 0.0};
    N.D = C.D; N.r0 = C.r0; N.r1 = C.r1;
    if (Lf) {
        const M2 al = m2_mul(C.L, m2_inv(Lf->D));
        N.L = m2_mul(al, Lf->L);
        N.L = {-N.L.a, -N.L.b, -N.L.c, -N.L.d};
        N.D = m2_sub(N.D, m2_mul(al, Lf->U));
        N.r0 -= al.a * Lf->r0 + al.b * Lf->r1;
        N.r1 -= al.c * Lf->r0 + al.d * Lf->r1;
    }
    if (Rt) {
        const M2 ga = m2_mul(C.U, m2_inv(Rt->D));
        N.U = m2_mul(ga, Rt->U);
        N.U = {-N.U.a, -N.U.b, -N.U.c, -N.U.d};
        N.D = m2_sub(N.D, m2_mul(ga, Rt->L));
        N.r0 -= ga.a * Rt->r0 + ga.b * Rt->r1;
        N.r1 -= ga.c * Rt->r0 + ga.d * Rt->r1;
    }
    return N;
}

// x_i = D^{-1} (r - L x_{i-1} - U x_{i+1}) (absent neighbours as 0).
__device__ __forceinline__ void cr_solve_row(const Row& R, double xl0, double xl1, double xr0, double xr1,
                                             double* x0, double* x1)
{
    const double v0 = R.r0 - (R.L.a * xl0 + R.L.b * xl1) - (R.U.a * xr0 + R.U.b * xr1);
    const double v1 = R.r1 - (R.L.c * xl0 + R.L.d * xl1) - (R.U.c * xr0 + R.U.d * xr1);
    const M2 Di = m2_inv(R.D);
    *x0 = Di.a * v0 + Di.b * v1;
    *x1 = Di.c * v0 + Di.d * v1;
}

// Level l (n_l = ceil(n_0 / 2^l) rows per member, pitch cap) -> level l+1
// (its even rows, pitch cap1).
__global__ void __launch_bounds__(kDgThreads) k_cr_reduce(const double* __restrict__ s, double* __restrict__ s1,
                                                          const int* __restrict__ nact, int lev, int cap, int cap1,
                                                          size_t P, size_t P1, const DgTime* __restrict__ tc)
{
    const int b = blockIdx.y, k = blockIdx.x * kDgThreads + threadIdx.x;
    if (tc->abort) return;
    const int n0 = nact[b];
    if (n0 == 0) return;
    const int n = (int)(((long long)n0 + (1LL << lev) - 1) >> lev);
    if (k >= (n + 1) / 2) return;
    const int i = 2 * k;
    const size_t m = (size_t)b * cap;
    const Row C = load_row(s, P, m + i);
    Row Lf, Rt;
    const bool hl = i > 0, hr = i + 1 < n;
    if (hl) Lf = load_row(s, P, m + i - 1);
    if (hr) Rt = load_row(s, P, m + i + 1);
    store_row(s1, P1, (size_t)b * cap1 + k, cr_combine(C, hl ? &Lf : nullptr, hr ? &Rt : nullptr));
}

// x of level l from x of level l+1: even rows copied, odd rows solved.
__global__ void __launch_bounds__(kDgThreads) k_cr_back(const double* __restrict__ s, double* __restrict__ x,
                                                        const double* __restrict__ x1, const int* __restrict__ nact,
                                                        int lev, int cap, int cap1, size_t P, size_t X, size_t X1,
                                                        const DgTime* __restrict__ tc)
{
    const int b = blockIdx.y, k = blockIdx.x * kDgThreads + threadIdx.x;
    if (tc->abort) return;
    const int n0 = nact[b];
    if (n0 == 0) return;
    const int n = (int)(((long long)n0 + (1LL << lev) - 1) >> lev);
    const int n1 = (n + 1) / 2;
    if (k >= n1) return;
    const size_t m = (size_t)b * cap, m1 = (size_t)b * cap1;
    const double e0 = x1[m1 + k], e1 = x1[X1 + m1 + k];
    x[m + 2 * k] = e0; x[X + m + 2 * k] = e1;
    const int i = 2 * k + 1;
    if (i < n) {
        double r0 = 0.0, r1 = 0.0;
        if (k + 1 < n1) { r0 = x1[m1 + k + 1]; r1 = x1[X1 + m1 + k + 1]; }
        double y0, y1;
        cr_solve_row(load_row(s, P, m + i), e0, e1, r0, r1, &y0, &y1);
        x[m + i] = y0; x[X + m + i] = y1;
    }
}

// The last levels of a member (n_l <= kCrSmemRows rows at level `lev`) in
// shared memory: reduction to one row, its solve, back-substitution; writes
// x of level `lev`.
__global__ void __launch_bounds__(kCrSmallThreads) k_cr_small(const double* __restrict__ s, double* __restrict__ x,
                                                              const int* __restrict__ nact, int lev, int cap,
                                                              size_t P, size_t X, const DgTime* __restrict__ tc)
{
    extern __shared__ double crs_sm[];
    // rows of all levels one after the other (at most 2 n + levels <= kCrSmallRows), then x of each
    Row* rows = reinterpret_cast<Row*>(crs_sm);
    double* xs = crs_sm + (size_t)kCrSmallRows * kSysPlanes;
    const int b = blockIdx.x, tid = threadIdx.x;
    if (tc->abort) return;
    const int n0 = nact[b];
    if (n0 == 0) return;
    const int n = (int)(((long long)n0 + (1LL << lev) - 1) >> lev);
    const size_t m = (size_t)b * cap;
    int off[16], cnt[16], nl = 0;
    {
        int o = 0, c = n;
        while (true) {
            off[nl] = o; cnt[nl] = c; ++nl;
            if (c == 1) break;
            o += c; c = (c + 1) / 2;
        }
    }
    for (int r = tid; r < n; r += kCrSmallThreads) rows[r] = load_row(s, P, m + r);
    __syncthreads();
    for (int q = 0; q + 1 < nl; ++q) {
        const int c = cnt[q], c1 = cnt[q + 1];
        for (int k = tid; k < c1; k += kCrSmallThreads) {
            const int i = 2 * k;
            const Row* R = rows + off[q];
            rows[off[q + 1] + k] = cr_combine(R[i], i > 0 ? &R[i - 1] : nullptr, i + 1 < c ? &R[i + 1] : nullptr);
        }
        __syncthreads();
    }
    if (tid == 0) {
        const int t = off[nl - 1];
        cr_solve_row(rows[t], 0.0, 0.0, 0.0, 0.0, &xs[2 * t], &xs[2 * t + 1]);
    }
    __syncthreads();
    for (int q = nl - 2; q >= 0; --q) {
        const int c = cnt[q], c1 = cnt[q + 1];
        for (int k = tid; k < c1; k += kCrSmallThreads) {
            const double* xu = xs + 2 * off[q + 1];
            double* xq = xs + 2 * off[q];
            const double e0 = xu[2 * k], e1 = xu[2 * k + 1];
            xq[4 * k] = e0; xq[4 * k + 1] = e1;
            const int i = 2 * k + 1;
            if (i < c) {
                double r0 = 0.0, r1 = 0.0;
                if (k + 1 < c1) { r0 = xu[2 * k + 2]; r1 = xu[2 * k + 3]; }
                cr_solve_row(rows[off[q] + i], e0, e1, r0, r1, &xq[2 * i], &xq[2 * i + 1]);
            }
        }
        __syncthreads();
    }
    for (int r = tid; r < n; r += kCrSmallThreads) { x[m + r] = xs[2 * r]; x[X + m + r] = xs[2 * r + 1]; }
}

// ------------------------------------------------------------- correction

struct CorrArgs {
    Geo G;
    const int *act, *nact;
    const double* loc;
    const double* sys;       // level-0 system (residual check)
    const double* x;         // level-0 solution, 2 planes (pL, pR)
    size_t plane;
    const double *ht, *hwt;
    double *hu, *hw, *p;     // corrected in place (the step's output buffer)
    double* res;             // per member: [2 b] = sum |r - A p|^2, [2 b + 1] = sum (|r| + |A| |p|)^2
    int* bad;                // per member: non-finite solution
    int check;
    const DgTime* tc;
};

__global__ void __launch_bounds__(kDgThreads) k_dg_correct(CorrArgs a)
{
    __shared__ double red[2][32];
    __shared__ int badw;
    const Geo& G = a.G;
    const int b = blockIdx.y, j = blockIdx.x * kDgThreads + threadIdx.x, tid = threadIdx.x;
    if (a.tc->abort) return;
    const int n = a.nact[b];
    if (blockIdx.x * kDgThreads >= n) return;   // uniform per CTA
    if (tid == 0) badw = 0;
    double rr = 0.0, bb = 0.0;
    int bad = 0;
    if (j < n) {
        const size_t me = (size_t)b * G.pe, o = me + j, P = a.plane;
        const int i = a.act[o];
        const bool mrgt = j < n - 1 && a.act[o + 1] == i + 1;
        const double pL = a.x[o], pR = a.x[P + o];
        const double pn = mrgt ? a.x[o + 1] : 0.0;
        const double* L = a.loc;
        const double hu0 = L[kA0 * P + o] + L[kB00 * P + o] * pL + L[kB01 * P + o] * pR + L[kC0 * P + o] * pn;
        const double hu1 = L[kA1 * P + o] + L[kB10 * P + o] * pL + L[kB11 * P + o] * pR + L[kC1 * P + o] * pn;
        const size_t kL = (size_t)b * G.pn + 2 * i, kR = kL + 1;
        const double hp_x = (a.ht[kR] * pR - a.ht[kL] * pL) / G.dx;
        const double q = a.tc->dt / G.rho;
        const double hw0 = a.hwt[kL] + q * (L[kC6L * P + o] * pL + L[kCxL * P + o] * hp_x + L[kPhL * P + o]);
        const double hw1 = a.hwt[kR] + q * (L[kC6R * P + o] * pR + L[kCxR * P + o] * hp_x + L[kPhR * P + o]);
        bad = !(isfinite(pL) && isfinite(pR) && isfinite(hu0) && isfinite(hu1) && isfinite(hw0) && isfinite(hw1));
        a.hu[kL] = hu0; a.hu[kR] = hu1;
        a.hw[kL] = hw0; a.hw[kR] = hw1;
        a.p[kL] = pL; a.p[kR] = pR;
        if (a.check) {
            const Row R = load_row(a.sys, P, o);
            const double xl0 = j > 0 ? a.x[o - 1] : 0.0, xl1 = j > 0 ? a.x[P + o - 1] : 0.0;
            const double xr0 = j < n - 1 ? a.x[o + 1] : 0.0, xr1 = j < n - 1 ? a.x[P + o + 1] : 0.0;
            const double v0 = R.r0 - (R.L.a * xl0 + R.L.b * xl1) - (R.D.a * pL + R.D.b * pR) - (R.U.a * xr0 + R.U.b * xr1);
            const double v1 = R.r1 - (R.L.c * xl0 + R.L.d * xl1) - (R.D.c * pL + R.D.d * pR) - (R.U.c * xr0 + R.U.d * xr1);
            // scale of the row: |r| + |A| |p| (the residual is a backward error against it)
            const double w0 = fabs(R.r0) + fabs(R.L.a * xl0) + fabs(R.L.b * xl1) + fabs(R.D.a * pL) + fabs(R.D.b * pR) +
                              fabs(R.U.a * xr0) + fabs(R.U.b * xr1);
            const double w1 = fabs(R.r1) + fabs(R.L.c * xl0) + fabs(R.L.d * xl1) + fabs(R.D.c * pL) + fabs(R.D.d * pR) +
                              fabs(R.U.c * xr0) + fabs(R.U.d * xr1);
            rr = v0 * v0 + v1 * v1;
            bb = w0 * w0 + w1 * w1;
        }
    }
    __syncthreads();
    if (bad) badw = 1;
    if (a.check) {
        rr = warp_sum(rr); bb = warp_sum(bb);
        if ((tid & 31) == 0) { red[0][tid >> 5] = rr; red[1][tid >> 5] = bb; }
    }
    __syncthreads();
    if (tid == 0) {
        if (badw) atomicOr(&a.bad[b], 1);
        if (a.check) {
            double s0 = 0.0, s1 = 0.0;
            for (int w = 0; w < kDgThreads / 32; ++w) { s0 += red[0][w]; s1 += red[1][w]; }
            atomicAdd(&a.res[2 * b], s0);
            atomicAdd(&a.res[2 * b + 1], s1);
        }
    }
}

// Step summary and acceptance; clears the per-member accumulators.
__global__ void __launch_bounds__(256) k_dg_finish(const double* __restrict__ mass_part, int nparts,
                                                   const int* __restrict__ nact, double* __restrict__ res,
                                                   double* __restrict__ rel_out, int* __restrict__ bad, int nb,
                                                   DgSummary* __restrict__ S, DgTime* __restrict__ tc)
{
    __shared__ double shd[64];
    __shared__ long long shl[32];
    __shared__ int shi[64];
    const int tid = threadIdx.x;
    if (tc->abort) return;
    double m = 0.0, rel = 0.0;
    long long na = 0;
    int nmax = 0, anybad = 0;
    for (int q = tid; q < nparts; q += 256) m += mass_part[q];
    for (int b = tid; b < nb; b += 256) {
        const int n = nact[b];
        na += n; nmax = max(nmax, n);
        const double r2 = res[2 * b], b2 = res[2 * b + 1];
        const double rb = b2 > 0.0 ? sqrt(r2 / b2) : 0.0;
        rel_out[b] = rb;
        rel = fmax(rel, rb);
        anybad |= bad[b];
        res[2 * b] = 0.0; res[2 * b + 1] = 0.0; bad[b] = 0;
    }
    m = warp_sum(m);
    double relw = rel;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) relw = fmax(relw, __shfl_xor_sync(0xffffffffu, relw, o));
    long long naw = na;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) naw += __shfl_xor_sync(0xffffffffu, naw, o);
    int nmw = nmax, bw = anybad;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        nmw = max(nmw, __shfl_xor_sync(0xffffffffu, nmw, o));
        bw |= __shfl_xor_sync(0xffffffffu, bw, o);
    }
    if ((tid & 31) == 0) {
        shd[tid >> 5] = m; shd[32 + (tid >> 5)] = relw; shl[tid >> 5] = naw;
        shi[tid >> 5] = nmw; shi[32 + (tid >> 5)] = bw;
    }
    __syncthreads();
    if (tid == 0) {
        double M = 0.0, R = 0.0;
        long long NA = 0;
        int NM = 0, B = 0;
        for (int w = 0; w < 8; ++w) {
            M += shd[w]; R = fmax(R, shd[32 + w]); NA += shl[w]; NM = max(NM, shi[w]); B |= shi[32 + w];
        }
        S->mass = M; S->rel_res = R; S->n_active = NA; S->n_active_max = NM;
        S->status = B ? NH_ERR_NONFINITE : NH_OK;
        if (B) {
            tc->abort = 1;
            tc->fail_status = NH_ERR_NONFINITE;
        } else {
            tc->n += 1; tc->steps += 1; tc->done += 1; tc->active_total += NA;
        }
    }
}

}  // namespace

// ================================================================== host

struct nh_dg {
    nh_dg_desc d;
    int nb, ne, pn, pe;
    cudaStream_t stream = nullptr, cap_stream = nullptr;
    int sm_count = 0;
    double *h[2], *hu[2], *hw[2], *p[2];
    double* d0;
    Slide* slide;
    DgKin* kin;
    uint8_t *marks, *mask;
    int *act, *nact;
    double* loc;
    double* sys[kMaxLevels];
    double* x[kMaxLevels];
    int cap[kMaxLevels];
    int nglob = 0;          // global cyclic-reduction levels (k_cr_reduce launches per step)
    double* mass_part;
    int npart;
    double* res;
    double* rel;
    int* bad;
    DgSummary* summary;
    DgTime* tc;
    // host state
    int cur = 0;
    bool has_state = false;
    double t0 = 0.0, last_dt = 0.0;
    long long n_since = 0, steps = 0;
    int crit = NH_CRIT_GLOBAL, enlarge = 1, first_global = 0, check = 1;
    double knh = 1e-3;
    // graphs
    cudaGraphExec_t graph[2] = {nullptr, nullptr};
    bool graph_valid = false;
    double graph_key[6] = {0, 0, 0, 0, 0, 0};
    // profiling
    bool prof_on = false;
    double prof_ms[NH_DG_K_COUNT];
    long long prof_n[NH_DG_K_COUNT];
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_cls;   // class of each recorded pair
    int ev_used = 0;
};

namespace {

#define CK(call)                                                  \
    do {                                                          \
        cudaError_t e__ = (call);                                 \
        if (e__ != cudaSuccess) { cudaGetLastError(); return NH_ERR_CUDA; } \
    } while (0)

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }
int round_up(int v, int m) { return (v + m - 1) / m * m; }

bool desc_ok(const nh_dg_desc* d)
{
    return d && d->ne >= 2 && d->ne <= (1 << 20) && d->nbatch >= 1 && std::isfinite(d->dx) && d->dx > 0.0 &&
           std::isfinite(d->x0) && std::isfinite(d->g) && d->g > 0.0 && std::isfinite(d->rho) && d->rho > 0.0 &&
           std::isfinite(d->c11) && d->c11 >= 0.0 &&
           (long long)d->nbatch * d->ne <= (1LL << 31) / 4;
}

// Level capacities: level 0 holds the element pitch; level l >= 1 holds
// ceil(ne / 2^l) rows (rounded up to 8); global levels stop once every
// member fits k_cr_small.
int levels(int ne, int pe, int* cap)
{
    cap[0] = pe;
    int l = 0;
    while (((long long)ne + (1LL << l) - 1) >> l > kCrSmemRows) {
        ++l;
        cap[l] = round_up((int)(((long long)ne + (1LL << l) - 1) >> l), 8);
    }
    return l;
}

// Workspace carving (sizes only when base == nullptr).
size_t carve(nh_dg* g, char* base)
{
    size_t off = 0;
    auto take = [&](size_t bytes) -> char* {
        char* p = base ? base + off : nullptr;
        off += align256(bytes);
        return p;
    };
    const size_t nodes = (size_t)g->nb * g->pn, elems = (size_t)g->nb * g->pe;
    for (int s = 0; s < 2; ++s) {
        g->h[s] = (double*)take(nodes * 8); g->hu[s] = (double*)take(nodes * 8);
        g->hw[s] = (double*)take(nodes * 8); g->p[s] = (double*)take(nodes * 8);
    }
    g->d0 = (double*)take(nodes * 8);
    g->slide = (Slide*)take(sizeof(Slide) * g->nb);
    g->kin = (DgKin*)take(sizeof(DgKin) * g->nb);
    g->marks = (uint8_t*)take(elems);
    g->mask = (uint8_t*)take(elems);
    g->act = (int*)take(elems * 4);
    g->nact = (int*)take((size_t)g->nb * 4);
    g->loc = (double*)take(elems * 8 * kLocalPlanes);
    for (int l = 0; l <= g->nglob; ++l) {
        const size_t rows = (size_t)g->nb * g->cap[l];
        g->sys[l] = (double*)take(rows * 8 * kSysPlanes);
        g->x[l] = (double*)take(rows * 8 * 2);
    }
    g->npart = g->nb * ((g->ne + kDgTile - 1) / kDgTile);
    g->mass_part = (double*)take((size_t)g->npart * 8);
    g->res = (double*)take((size_t)g->nb * 16);
    g->rel = (double*)take((size_t)g->nb * 8);
    g->bad = (int*)take((size_t)g->nb * 4);
    g->summary = (DgSummary*)take(sizeof(DgSummary));
    g->tc = (DgTime*)take(sizeof(DgTime));
    return off;
}

void geometry(nh_dg* g, const nh_dg_desc* d)
{
    g->d = *d;
    g->nb = d->nbatch; g->ne = d->ne;
    g->pn = round_up(2 * d->ne, 32);
    g->pe = round_up(d->ne, 32);
    g->nglob = levels(g->ne, g->pe, g->cap);
}

Geo geo(const nh_dg* g)
{
    Geo G;
    G.ne = g->ne; G.nb = g->nb; G.pn = g->pn; G.pe = g->pe;
    G.dx = g->d.dx; G.x0 = g->d.x0; G.g = g->d.g; G.rho = g->d.rho; G.c11 = g->d.c11;
    return G;
}

// Profiling brackets (step-by-step path only).
void prof_mark(nh_dg* g, int cls, cudaStream_t st)
{
    g->prof_n[cls] += 1;
    if (!g->prof_on) return;
    if ((int)g->ev_pool.size() < 2 * (g->ev_used + 1)) {
        cudaEvent_t a, b;
        cudaEventCreate(&a); cudaEventCreate(&b);
        g->ev_pool.push_back(a); g->ev_pool.push_back(b);
    }
    cudaEventRecord(g->ev_pool[2 * g->ev_used], st);
    g->ev_cls.push_back(cls);
}
void prof_done(nh_dg* g, cudaStream_t st)
{
    if (!g->prof_on) return;
    cudaEventRecord(g->ev_pool[2 * g->ev_used + 1], st);
    g->ev_used += 1;
}
void prof_collect(nh_dg* g)
{
    for (int q = 0; q < g->ev_used; ++q) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, g->ev_pool[2 * q], g->ev_pool[2 * q + 1]) == cudaSuccess)
            g->prof_ms[g->ev_cls[q]] += ms;
    }
    g->ev_used = 0;
    g->ev_cls.clear();
    cudaGetLastError();
}

// One step reading state buffer `cur` and writing `cur ^ 1`.  Launches
// 7 + 2 * nglob kernels.
nh_status enqueue_step(nh_dg* g, cudaStream_t st, int cur)
{
    const int nxt = cur ^ 1;
    const Geo G = geo(g);
    const size_t plane = (size_t)g->nb * g->pe;
    prof_mark(g, NH_DG_K_KINEMATICS, st);
    k_dg_kin<<<(g->nb + 127) / 128, 128, 0, st>>>(g->slide, g->kin, g->nb, g->tc);
    prof_done(g, st);
    PredArgs pa;
    pa.G = G;
    pa.h = g->h[cur]; pa.hu = g->hu[cur]; pa.hw = g->hw[cur];
    pa.ht = g->h[nxt]; pa.hut = g->hu[nxt]; pa.hwt = g->hw[nxt]; pa.p = g->p[nxt];
    pa.d0 = g->d0; pa.slide = g->slide; pa.kin = g->kin; pa.marks = g->marks; pa.mass_part = g->mass_part;
    pa.crit = g->crit; pa.knh = g->knh; pa.tc = g->tc;
    prof_mark(g, NH_DG_K_PREDICT, st);
    k_dg_predict<<<dim3((g->ne + kDgTile - 1) / kDgTile, g->nb), kDgTile, kPredSmem, st>>>(pa);
    prof_done(g, st);
    prof_mark(g, NH_DG_K_COMPACT, st);
    k_dg_compact<<<g->nb, 1024, 0, st>>>(g->marks, g->mask, g->act, g->nact, g->ne, g->pe,
                                         g->crit == NH_CRIT_GLOBAL ? 0 : g->enlarge, g->first_global, g->tc);
    prof_done(g, st);
    LocalArgs la;
    la.G = G;
    la.ht = g->h[nxt]; la.hut = g->hu[nxt]; la.hwt = g->hw[nxt]; la.d0 = g->d0;
    la.slide = g->slide; la.kin = g->kin; la.act = g->act; la.nact = g->nact;
    la.loc = g->loc; la.sys = g->sys[0]; la.plane = plane; la.tc = g->tc;
    const dim3 egrid((g->ne + kDgThreads - 1) / kDgThreads, g->nb);
    prof_mark(g, NH_DG_K_LOCAL, st);
    k_dg_local<<<egrid, kDgThreads, 0, st>>>(la);
    prof_done(g, st);
    prof_mark(g, NH_DG_K_FORM, st);
    k_dg_form<<<egrid, kDgThreads, 0, st>>>(g->act, g->nact, g->loc, g->sys[0], g->pe, plane, g->d.c11, g->tc);
    prof_done(g, st);
    for (int l = 0; l < g->nglob; ++l) {
        const int rows1 = (int)(((long long)g->ne + (1LL << (l + 1)) - 1) >> (l + 1));
        prof_mark(g, NH_DG_K_REDUCE, st);
        k_cr_reduce<<<dim3((rows1 + kDgThreads - 1) / kDgThreads, g->nb), kDgThreads, 0, st>>>(
            g->sys[l], g->sys[l + 1], g->nact, l, g->cap[l], g->cap[l + 1], (size_t)g->nb * g->cap[l],
            (size_t)g->nb * g->cap[l + 1], g->tc);
        prof_done(g, st);
    }
    prof_mark(g, NH_DG_K_REDUCE, st);
    k_cr_small<<<g->nb, kCrSmallThreads, kCrSmallSmem, st>>>(g->sys[g->nglob], g->x[g->nglob], g->nact, g->nglob,
                                                             g->cap[g->nglob], (size_t)g->nb * g->cap[g->nglob],
                                                             (size_t)g->nb * g->cap[g->nglob], g->tc);
    prof_done(g, st);
    for (int l = g->nglob - 1; l >= 0; --l) {
        const int rows1 = (int)(((long long)g->ne + (1LL << (l + 1)) - 1) >> (l + 1));
        prof_mark(g, NH_DG_K_BACK, st);
        k_cr_back<<<dim3((rows1 + kDgThreads - 1) / kDgThreads, g->nb), kDgThreads, 0, st>>>(
            g->sys[l], g->x[l], g->x[l + 1], g->nact, l, g->cap[l], g->cap[l + 1], (size_t)g->nb * g->cap[l],
            (size_t)g->nb * g->cap[l], (size_t)g->nb * g->cap[l + 1], g->tc);
        prof_done(g, st);
    }
    CorrArgs ca;
    ca.G = G;
    ca.act = g->act; ca.nact = g->nact; ca.loc = g->loc; ca.sys = g->sys[0]; ca.x = g->x[0]; ca.plane = plane;
    ca.ht = g->h[nxt]; ca.hwt = g->hw[nxt]; ca.hu = g->hu[nxt]; ca.hw = g->hw[nxt]; ca.p = g->p[nxt];
    ca.res = g->res; ca.bad = g->bad; ca.check = g->check; ca.tc = g->tc;
    prof_mark(g, NH_DG_K_CORRECT, st);
    k_dg_correct<<<egrid, kDgThreads, 0, st>>>(ca);
    prof_done(g, st);
    prof_mark(g, NH_DG_K_FINISH, st);
    k_dg_finish<<<1, 256, 0, st>>>(g->mass_part, g->npart, g->nact, g->res, g->rel, g->bad, g->nb, g->summary,
                                   g->tc);
    prof_done(g, st);
    CK(cudaGetLastError());
    return NH_OK;
}

nh_status write_time(nh_dg* g, double dt, cudaStream_t st)
{
    DgTime tc;
    std::memset(&tc, 0, sizeof(tc));
    tc.t0 = g->t0; tc.dt = dt; tc.n = g->n_since; tc.steps = g->steps;
    CK(cudaMemcpyAsync(g->tc, &tc, sizeof(tc), cudaMemcpyHostToDevice, st));
    return NH_OK;
}

// A new dt restarts the device clock at the current time.
void rebase(nh_dg* g, double dt)
{
    if (g->last_dt != dt) {
        g->t0 = g->t0 + (double)g->n_since * g->last_dt;
        g->n_since = 0;
        g->last_dt = dt;
    }
}

void fill_info(const nh_dg* g, const DgSummary& S, nh_step_info* I, int status)
{
    I->step = g->steps;
    I->t = g->t0 + (double)g->n_since * g->last_dt;
    I->n_active = S.n_active; I->n_active_max = S.n_active_max;
    I->iters = 0; I->ir_passes = 0; I->solver = -1;
    I->status = status;
    I->rel_res = S.rel_res;
    I->min_gamma = 0.0;
    I->mass = S.mass;
}

void graph_destroy(nh_dg* g)
{
    for (int q = 0; q < 2; ++q)
        if (g->graph[q]) { cudaGraphExecDestroy(g->graph[q]); g->graph[q] = nullptr; }
    g->graph_valid = false;
}

nh_status graph_prepare(nh_dg* g)
{
    const double key[6] = {(double)g->crit, g->knh, (double)g->enlarge, (double)g->first_global,
                           (double)g->check, 1.0};
    if (g->graph_valid && std::memcmp(key, g->graph_key, sizeof(key)) == 0) return NH_OK;
    graph_destroy(g);
    if (!g->cap_stream) CK(cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking));
    for (int q = 0; q < 2; ++q) {
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
        nh_status rc = enqueue_step(g, g->cap_stream, q);
        cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
        if (rc != NH_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            graph_destroy(g);
            return rc != NH_OK ? rc : NH_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&g->graph[q], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { g->graph[q] = nullptr; graph_destroy(g); cudaGetLastError(); return NH_ERR_CUDA; }
    }
    std::memcpy(g->graph_key, key, sizeof(key));
    g->graph_valid = true;
    return NH_OK;
}

bool finite_all(const double* v, size_t n)
{
    for (size_t i = 0; i < n; ++i)
        if (!std::isfinite(v[i])) return false;
    return true;
}

}  // namespace

extern "C" {

size_t nh_dg_workspace_bytes(const nh_dg_desc* desc)
{
    if (!desc_ok(desc)) return 0;
    nh_dg g;
    geometry(&g, desc);
    return carve(&g, nullptr);
}

nh_status nh_dg_create(const nh_dg_desc* desc, const double* d0_host, void* ws, size_t ws_bytes, void* stream,
                       nh_dg** out)
{
    if (!out) return NH_ERR_ARG;
    *out = nullptr;
    if (!desc_ok(desc) || !d0_host || !ws || ((uintptr_t)ws & 255)) return NH_ERR_ARG;
    const size_t nn = (size_t)desc->nbatch * 2 * desc->ne;
    for (size_t i = 0; i < nn; ++i)
        if (!(std::isfinite(d0_host[i]) && d0_host[i] > 0.0)) return NH_ERR_ARG;
    nh_dg* g = new (std::nothrow) nh_dg;
    if (!g) return NH_ERR_ARG;
    geometry(g, desc);
    if (ws_bytes < carve(g, nullptr)) { delete g; return NH_ERR_ARG; }
    carve(g, (char*)ws);
    g->stream = (cudaStream_t)stream;
    std::memset(g->prof_ms, 0, sizeof(g->prof_ms));
    std::memset(g->prof_n, 0, sizeof(g->prof_n));
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&g->sm_count, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_cr_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kCrSmallSmem);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_dg_predict, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)kPredSmem);
    if (e != cudaSuccess) { cudaGetLastError(); delete g; return NH_ERR_CUDA; }
    cudaStream_t st = g->stream;
    // zero the whole workspace once (padding lanes stay defined)
    e = cudaMemsetAsync(ws, 0, carve(g, (char*)ws), st);
    std::vector<double> tmp((size_t)g->nb * g->pn, 1.0);
    for (int b = 0; b < g->nb; ++b)
        std::memcpy(&tmp[(size_t)b * g->pn], d0_host + (size_t)b * 2 * g->ne, sizeof(double) * 2 * g->ne);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d0, tmp.data(), sizeof(double) * tmp.size(), cudaMemcpyHostToDevice, st);
    std::vector<Slide> sl(g->nb);
    std::memset(sl.data(), 0, sizeof(Slide) * g->nb);
    for (auto& s : sl) { s.shape = NH_SLIDE_NONE; s.L = 1.0; s.iL = 1.0; s.t0 = 1.0; }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->slide, sl.data(), sizeof(Slide) * g->nb, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) { cudaGetLastError(); delete g; return NH_ERR_CUDA; }
    *out = g;
    return NH_OK;
}

nh_status nh_dg_set_bottom_motion(nh_dg* g, const nh_slide_desc* slides)
{
    if (!g) return NH_ERR_ARG;
    std::vector<Slide> sl(g->nb);
    std::memset(sl.data(), 0, sizeof(Slide) * g->nb);
    for (int b = 0; b < g->nb; ++b) {
        Slide& s = sl[b];
        s.shape = NH_SLIDE_NONE; s.L = 1.0; s.iL = 1.0; s.t0 = 1.0;
        if (!slides) continue;
        const nh_slide_desc& d = slides[b];
        if (d.shape < NH_SLIDE_NONE || d.shape > NH_SLIDE_QUARTIC) return NH_ERR_ARG;
        if (d.shape == NH_SLIDE_NONE) continue;
        if (!(std::isfinite(d.A) && std::isfinite(d.L) && d.L > 0.0 && std::isfinite(d.xc0) &&
              std::isfinite(d.s0) && std::isfinite(d.t0) && d.t0 > 0.0))
            return NH_ERR_ARG;
        if (d.shape == NH_SLIDE_QUARTIC && !(std::isfinite(d.t2) && d.t2 >= d.t0)) return NH_ERR_ARG;
        s.shape = d.shape; s.A = d.A; s.L = d.L; s.iL = 1.0 / d.L; s.xc0 = d.xc0; s.s0 = d.s0; s.t0 = d.t0;
        s.t2 = d.t2;
    }
    CK(cudaMemcpyAsync(g->slide, sl.data(), sizeof(Slide) * g->nb, cudaMemcpyHostToDevice, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return NH_OK;
}

nh_status nh_dg_set_criterion(nh_dg* g, int kind, double k_nh, int enlarge, int first_step_global)
{
    if (!g || kind < NH_CRIT_GLOBAL || kind > NH_CRIT_W_X || !std::isfinite(k_nh) || k_nh < 0.0 || enlarge < 0 ||
        enlarge > 16)
        return NH_ERR_ARG;
    g->crit = kind; g->knh = k_nh; g->enlarge = enlarge; g->first_global = first_step_global ? 1 : 0;
    return NH_OK;
}

nh_status nh_dg_set_check(nh_dg* g, int check)
{
    if (!g) return NH_ERR_ARG;
    g->check = check ? 1 : 0;
    return NH_OK;
}

nh_status nh_dg_set_state(nh_dg* g, const double* h, const double* hu, const double* hw, double t)
{
    if (!g || !h || !hu || !hw || !std::isfinite(t)) return NH_ERR_ARG;
    const size_t nn = (size_t)g->nb * 2 * g->ne;
    for (size_t i = 0; i < nn; ++i)
        if (!(std::isfinite(h[i]) && h[i] > 0.0)) return NH_ERR_ARG;
    if (!finite_all(hu, nn) || !finite_all(hw, nn)) return NH_ERR_ARG;
    cudaStream_t st = g->stream;
    const int c = g->cur;
    const double* src[3] = {h, hu, hw};
    double* dst[3] = {g->h[c], g->hu[c], g->hw[c]};
    std::vector<double> tmp((size_t)g->nb * g->pn);
    for (int f = 0; f < 3; ++f) {
        std::fill(tmp.begin(), tmp.end(), f == 0 ? 1.0 : 0.0);
        for (int b = 0; b < g->nb; ++b)
            std::memcpy(&tmp[(size_t)b * g->pn], src[f] + (size_t)b * 2 * g->ne, sizeof(double) * 2 * g->ne);
        CK(cudaMemcpyAsync(dst[f], tmp.data(), sizeof(double) * tmp.size(), cudaMemcpyHostToDevice, st));
        CK(cudaStreamSynchronize(st));
    }
    CK(cudaMemsetAsync(g->p[c], 0, sizeof(double) * g->nb * g->pn, st));
    CK(cudaMemsetAsync(g->mask, 0, (size_t)g->nb * g->pe, st));
    CK(cudaMemsetAsync(g->rel, 0, sizeof(double) * g->nb, st));
    CK(cudaStreamSynchronize(st));
    g->has_state = true;
    g->t0 = t; g->n_since = 0; g->steps = 0; g->last_dt = 0.0;
    return NH_OK;
}

nh_status nh_dg_get_state(nh_dg* g, double* h, double* hu, double* hw, double* p)
{
    if (!g) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    cudaStream_t st = g->stream;
    const int c = g->cur;
    double* dst[4] = {h, hu, hw, p};
    const double* src[4] = {g->h[c], g->hu[c], g->hw[c], g->p[c]};
    std::vector<double> tmp((size_t)g->nb * g->pn);
    for (int f = 0; f < 4; ++f) {
        if (!dst[f]) continue;
        CK(cudaMemcpyAsync(tmp.data(), src[f], sizeof(double) * tmp.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int b = 0; b < g->nb; ++b)
            std::memcpy(dst[f] + (size_t)b * 2 * g->ne, &tmp[(size_t)b * g->pn], sizeof(double) * 2 * g->ne);
    }
    return NH_OK;
}

nh_status nh_dg_get_mask(nh_dg* g, unsigned char* mask, double* rel_res)
{
    if (!g) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    cudaStream_t st = g->stream;
    if (mask) {
        std::vector<uint8_t> tmp((size_t)g->nb * g->pe);
        CK(cudaMemcpyAsync(tmp.data(), g->mask, tmp.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int b = 0; b < g->nb; ++b) std::memcpy(mask + (size_t)b * g->ne, &tmp[(size_t)b * g->pe], g->ne);
    }
    if (rel_res) {
        CK(cudaMemcpyAsync(rel_res, g->rel, sizeof(double) * g->nb, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
    }
    return NH_OK;
}

nh_status nh_dg_step(nh_dg* g, double dt, nh_step_info* info)
{
    if (!g || !std::isfinite(dt) || dt <= 0.0) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    cudaStream_t st = g->stream;
    rebase(g, dt);
    nh_status rc = write_time(g, dt, st);
    if (rc != NH_OK) return rc;
    rc = enqueue_step(g, st, g->cur);
    if (rc != NH_OK) return rc;
    DgSummary S;
    DgTime tc;
    CK(cudaMemcpyAsync(&S, g->summary, sizeof(S), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&tc, g->tc, sizeof(tc), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    prof_collect(g);
    const int status = tc.abort ? tc.fail_status : NH_OK;
    if (status == NH_OK) {
        g->cur ^= 1;
        g->n_since += 1;
        g->steps += 1;
    }
    if (info) fill_info(g, S, info, status);
    return (nh_status)status;
}

nh_status nh_dg_run(nh_dg* g, double dt, long long n_steps, nh_run_info* R)
{
    if (!g || !std::isfinite(dt) || dt <= 0.0 || n_steps < 0) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    nh_run_info tmp;
    if (!R) R = &tmp;
    std::memset(R, 0, sizeof(*R));
    if (n_steps == 0) return NH_OK;
    if (g->prof_on) {
        for (long long k = 0; k < n_steps; ++k) {
            nh_status rc = nh_dg_step(g, dt, &R->last);
            if (rc != NH_OK) return rc;
            R->steps += 1;
            R->active_total += R->last.n_active;
        }
        return NH_OK;
    }
    cudaStream_t st = g->stream;
    rebase(g, dt);
    nh_status rc = graph_prepare(g);
    if (rc != NH_OK) return rc;
    rc = write_time(g, dt, st);
    if (rc != NH_OK) return rc;
    for (long long k = 0; k < n_steps; ++k) CK(cudaGraphLaunch(g->graph[(g->cur + k) & 1], st));
    DgSummary S;
    DgTime tc;
    CK(cudaMemcpyAsync(&S, g->summary, sizeof(S), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&tc, g->tc, sizeof(tc), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const long long done = tc.done;
    // launches per step by class (the criterion runs inside the predictor)
    const long long per_step[NH_DG_K_COUNT] = {1, 1, 0, 1, 1, 1, g->nglob + 1, g->nglob, 1, 1};
    for (int c = 0; c < NH_DG_K_COUNT; ++c) g->prof_n[c] += per_step[c] * (done + (tc.abort ? 1 : 0));
    if (done & 1) g->cur ^= 1;
    g->n_since += done;
    g->steps += done;
    R->steps = done;
    R->active_total = tc.active_total;
    fill_info(g, S, &R->last, tc.abort ? tc.fail_status : NH_OK);
    return tc.abort ? (nh_status)tc.fail_status : NH_OK;
}

nh_status nh_dg_set_profiling(nh_dg* g, int enable)
{
    if (!g) return NH_ERR_ARG;
    g->prof_on = enable != 0;
    std::memset(g->prof_ms, 0, sizeof(g->prof_ms));
    std::memset(g->prof_n, 0, sizeof(g->prof_n));
    return NH_OK;
}

nh_status nh_dg_get_profile(nh_dg* g, double* ms, long long* launches)
{
    if (!g) return NH_ERR_ARG;
    for (int c = 0; c < NH_DG_K_COUNT; ++c) {
        if (ms) ms[c] = g->prof_ms[c];
        if (launches) launches[c] = g->prof_n[c];
    }
    return NH_OK;
}

void nh_dg_destroy(nh_dg* g)
{
    if (!g) return;
    graph_destroy(g);
    for (auto e : g->ev_pool) cudaEventDestroy(e);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
}

}  // extern "C"
