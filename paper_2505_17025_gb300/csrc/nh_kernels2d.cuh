// nh_kernels2d.cuh -- kernels of the two-dimensional grid.
//
// State storage (template parameter TS): FP64 keeps h, hu, hv, hw and the
// depth d; FP32 keeps zeta = h - d0, hu, hv, hw and the mound m = d0 - d, with
// an FP32 copy of d0, so that eta = zeta + m keeps its digits in FP32 (the 1D
// mixed path's representation).  Assembly, Krylov solve and the correction's
// arithmetic stay FP64 in both.
//
//  k2_depth      bottom depth d = d0 - mound (FP64) or the mound (FP32)  (a1)
//  k2_stage      one Heun stage of the hydrostatic predictor: x and y
//                Rusanov fluxes of MUSCL states, well-balanced sources    (a2)
//  k2_marks      criterion of Sec. 5.1 (2D form) on the predicted state  (a3)
//  k2_dilate     Moore enlargement of the marks                          (a3)
//  k2_count / k2_scan / k2_emit   row-major compaction into the active
//                list and the cell -> list-index map                      (a3)
//  k2_assemble   9-point rows of -div(K grad psi) + gamma psi = R        (a4)
//  k2_correct    Eqs. 10-11 in 2D on the active cells                    (a6)
// The Krylov solve (a5) is the 1D members' (nh_kernels1d.cuh): each 2D grid
// of an ensemble is one member holding its active cells in row-major order,
// so the W / E neighbours are the list neighbours (the line preconditioner
// solves x-lines) and S, N and the four diagonal couplings are the solver's
// extra couplings.  Members (grids of their own sizes, spacings, sides and
// slides) sit at b * pitch in every per-cell array; kernels take the member
// from blockIdx.y (or from the work item) and its geometry from geos[b].
//
// The 2D equations generalise the paper's 1D Eqs. 1-5 and 10-11 by replacing
// x-derivatives with gradients; the elimination of the corrected momenta into
// the constraint (Eq. 4) gives -div(K grad q) + gamma q = R with the tensor
// K = (a/h)(I - grad d grad d^T / D), D = 4 + |grad d|^2.  Here psi = a q
// (a = dt / rho), so the stored K, beta and gamma carry no factor a and the
// stored phi is a phi.
#pragma once

#include "nh_kernels1d.cuh"

namespace nh {

struct Geo2 {
    int nx, ny, bcx, bcy, lim;
    double dx, dy, x0, y0, g;
    double idx, idy;   // 1 / dx, 1 / dy
};

// v with the sign of the parity o (+1 or -1): no floating-point multiply.
template <typename T>
__device__ __forceinline__ T flip(int o, T v) { return o < 0 ? -v : v; }

// 2D slide: mound A exp(-xi^2 - zeta^2), xi = (x - xc0 - s)/Lx, zeta = (y - yc0)/Ly.
// Its position s(t) = s0 ln cosh(t / t0) (Sec. 4.2).
struct Slide2 {
    double A, Lx, Ly, xc0, yc0, s0, t0;
    double iLx, iLy;   // 1 / Lx, 1 / Ly
    int shape, pad;
};

// Slide position, velocity and acceleration at one time.
struct Kin2 {
    double s, sd, sdd;
};

// kin[2b] at t^n, kin[2b + 1] at t^{n+1}: s = s0 ln cosh(t/t0),
// s' = (s0/t0) tanh(t/t0), s'' = (s0/t0^2) / cosh^2(t/t0).  Times from the
// arguments, or from the captured run's control block when tc is set.
static __global__ void k2_kin(const Slide2* __restrict__ slides, int nb, double t_n, double t_n1,
                              const TimeCtl* __restrict__ tc, Kin2* kin)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || (tc && tc->abort)) return;
    if (tc) {
        t_n = tc->t_base + (double)tc->n * tc->dt;
        t_n1 = tc->t_base + (double)(tc->n + 1) * tc->dt;
    }
    const Slide2 S = slides[b];
    for (int w = 0; w < 2; ++w) {
        Kin2 k{0.0, 0.0, 0.0};
        if (S.shape == NH_SLIDE_GAUSS_LNCOSH) {
            const double z = (w ? t_n1 : t_n) / S.t0, c = cosh(z);
            k.s = S.s0 * log(c);
            k.sd = (S.s0 / S.t0) * tanh(z);
            k.sdd = (S.s0 / (S.t0 * S.t0)) / (c * c);
        }
        kin[2 * b + w] = k;
    }
}

// In-domain index of i: wrapped (periodic) or mirrored once at a wall; a
// halo cell further out than the grid is wide (a tile's far halo on a tiny
// grid, which no in-domain stencil reaches) is clamped into the grid, so it
// is never read outside the member's slice.
__device__ __forceinline__ int g2_index1(int bc, int n, int i, int* odd)
{
    *odd = 1;
    if (i >= 0 && i < n) return i;
    if (bc == NH_BC_PERIODIC) return ((i % n) + n) % n;
    *odd = -1;
    const int r = (i < 0) ? (-1 - i) : (2 * n - 1 - i);
    return r < 0 ? 0 : (r >= n ? n - 1 : r);
}

// Flat index of the in-domain (mirrored / wrapped) cell of (i, j) and the
// parities of quantities odd in x and in y.
__device__ __forceinline__ int g2_cell(const Geo2& G, int i, int j, int* ox, int* oy)
{
    const int ci = g2_index1(G.bcx, G.nx, i, ox);
    const int cj = g2_index1(G.bcy, G.ny, j, oy);
    return cj * G.nx + ci;
}

// Flat index of the unknown at (i, j), or -1 outside a walled side.
__device__ __forceinline__ int g2_inner(const Geo2& G, int i, int j)
{
    if (i < 0 || i >= G.nx) {
        if (G.bcx != NH_BC_PERIODIC) return -1;
        i = ((i % G.nx) + G.nx) % G.nx;
    }
    if (j < 0 || j >= G.ny) {
        if (G.bcy != NH_BC_PERIODIC) return -1;
        j = ((j % G.ny) + G.ny) % G.ny;
    }
    return j * G.nx + i;
}

// Mound height at cell (i, j) for slide position s; 0 where xi^2 + zeta^2 >
// kMoundCut (below half an ulp of any depth it is subtracted from when
// A < 12 d0, so the depth is the same double).
__device__ __forceinline__ double mound2(const Geo2& G, const Slide2& S, int i, int j, double s)
{
    if (S.shape != NH_SLIDE_GAUSS_LNCOSH) return 0.0;
    const double x = G.x0 + (i + 0.5) * G.dx, y = G.y0 + (j + 0.5) * G.dy;
    const double xi = (x - S.xc0 - s) * S.iLx, ze = (y - S.yc0) * S.iLy;
    const double r2 = xi * xi + ze * ze;
    return r2 > kMoundCut ? 0.0 : S.A * exp(-r2);
}

// d, d_x, d_y, d_xx, d_yy, d_xy, d_t, d_xt, d_yt, d_tt at cell (i, j):
// central differences of d0 (mirrored / wrapped neighbours) and the mound's
// terms by the chain rule (dxi/dt = -s'/Lx).
__device__ __forceinline__ void bottom2(const Geo2& G, const double* __restrict__ d0, const Slide2& S,
                                        const Kin2& K, int i, int j, double out[10])
{
    int o1, o2;
    const double c = d0[j * G.nx + i];
    const double xm = d0[g2_cell(G, i - 1, j, &o1, &o2)], xp = d0[g2_cell(G, i + 1, j, &o1, &o2)];
    const double ym = d0[g2_cell(G, i, j - 1, &o1, &o2)], yp = d0[g2_cell(G, i, j + 1, &o1, &o2)];
    const double mm = d0[g2_cell(G, i - 1, j - 1, &o1, &o2)], pm = d0[g2_cell(G, i + 1, j - 1, &o1, &o2)];
    const double mp = d0[g2_cell(G, i - 1, j + 1, &o1, &o2)], pp = d0[g2_cell(G, i + 1, j + 1, &o1, &o2)];
    // reciprocals of the spacings and slide lengths instead of divisions
    // (GB300's FP64 division is a long instruction sequence)
    const double ix = G.idx, iy = G.idy;
    double d = c;
    double d_x = (xp - xm) * (0.5 * ix), d_y = (yp - ym) * (0.5 * iy);
    double d_xx = (xp - 2.0 * c + xm) * (ix * ix), d_yy = (yp - 2.0 * c + ym) * (iy * iy);
    double d_xy = (pp - pm - mp + mm) * (0.25 * ix * iy);
    double d_t = 0.0, d_xt = 0.0, d_yt = 0.0, d_tt = 0.0;
    if (S.shape == NH_SLIDE_GAUSS_LNCOSH) {
        const double x = G.x0 + (i + 0.5) * G.dx, y = G.y0 + (j + 0.5) * G.dy;
        const double iLx = S.iLx, iLy = S.iLy, sd = K.sd, sdd = K.sdd;
        const double xi = (x - S.xc0 - K.s) * iLx, ze = (y - S.yc0) * iLy;
        const double m = S.A * exp(-xi * xi - ze * ze);
        const double m_x = m * (-2.0 * xi * iLx), m_y = m * (-2.0 * ze * iLy);
        const double m_xx = m * (4.0 * xi * xi - 2.0) * (iLx * iLx);
        const double m_yy = m * (4.0 * ze * ze - 2.0) * (iLy * iLy);
        const double m_xy = m * (4.0 * xi * ze) * (iLx * iLy);
        const double m_t = m * (2.0 * xi * iLx) * sd;
        const double m_xt = -m * (2.0 * iLx * iLx) * (2.0 * xi * xi - 1.0) * sd;
        const double m_yt = -m * (4.0 * xi * ze * iLx * iLy) * sd;
        const double m_tt = m * (2.0 * iLx * iLx) * ((2.0 * xi * xi - 1.0) * sd * sd + xi * S.Lx * sdd);
        d -= m; d_x -= m_x; d_y -= m_y; d_xx -= m_xx; d_yy -= m_yy; d_xy -= m_xy;
        d_t = -m_t; d_xt = -m_xt; d_yt = -m_yt; d_tt = -m_tt;
    }
    out[0] = d; out[1] = d_x; out[2] = d_y; out[3] = d_xx; out[4] = d_yy; out[5] = d_xy;
    out[6] = d_t; out[7] = d_xt; out[8] = d_yt; out[9] = d_tt;
}

// Depth (FP64 storage) or mound (FP32 storage) at t^n (which = 0) or
// t^{n+1} (which = 1).  The FP32 mound measures the offset from the slide's
// centre as an exact integer cell offset plus an FP32 fraction (computed once
// per CTA in FP64), so xi and zeta keep FP32 relative precision however far
// from the origin the slide is; same kMoundCut test as mound2.
template <typename TS>
static __global__ void k2_depth(const Geo2* __restrict__ geos, const Slide2* __restrict__ slides,
                                const Kin2* __restrict__ kin, int which, size_t pitch,
                                const double* __restrict__ d0, TS* dm, const TimeCtl* __restrict__ tc)
{
    if (tc && tc->abort) return;
    const int b = blockIdx.y;
    const Geo2 G = geos[b];
    const Slide2 S = slides[b];
    const double s = kin[2 * b + which].s;
    const size_t mo = (size_t)b * pitch;
    const int N = G.nx * G.ny;
    if constexpr (sizeof(TS) == 8) {
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x)
            dm[mo + c] = d0[mo + c] - mound2(G, S, c % G.nx, c / G.nx, s);
    } else {
        __shared__ int s_ic[2];
        __shared__ float s_f[5];   // fraction x, fraction y, dx / Lx, dy / Ly, A
        if (threadIdx.x == 0) {
            const double cx = (S.xc0 + s - G.x0) * G.idx - 0.5, cy = (S.yc0 - G.y0) * G.idy - 0.5;
            const double fx = floor(cx), fy = floor(cy);
            s_ic[0] = (int)fmax(fmin(fx, 1e9), -1e9); s_ic[1] = (int)fmax(fmin(fy, 1e9), -1e9);
            s_f[0] = (float)(cx - fx); s_f[1] = (float)(cy - fy);
            s_f[2] = (float)(G.dx * S.iLx); s_f[3] = (float)(G.dy * S.iLy); s_f[4] = (float)S.A;
        }
        __syncthreads();
        const bool on = S.shape == NH_SLIDE_GAUSS_LNCOSH;
        for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
            float m = 0.0f;
            if (on) {
                const int i = c % G.nx, j = c / G.nx;
                const float xi = ((float)(i - s_ic[0]) - s_f[0]) * s_f[2];
                const float ze = ((float)(j - s_ic[1]) - s_f[1]) * s_f[3];
                const float r2 = xi * xi + ze * ze;
                if (r2 <= (float)kMoundCut) m = s_f[4] * expf(-r2);
            }
            dm[mo + c] = m;
        }
    }
}

// h, eta and d of cell c from the stored state (see the head of this file).
template <typename TS>
__device__ __forceinline__ void cell_hed(const TS* __restrict__ hz, const TS* __restrict__ dm,
                                         const TS* __restrict__ d0s, size_t c, TS& h, TS& eta, TS& d)
{
    if constexpr (sizeof(TS) == 8) {
        h = hz[c]; d = dm[c]; eta = h - d;
    } else {
        const TS z = hz[c], m = dm[c], dz = d0s[c];
        d = dz - m; eta = z + m; h = z + dz;
    }
}

template <typename T>
__device__ __forceinline__ T slope2(int lim, T vm, T v0, T vp)
{
    return limited_slope(lim, vm, v0, vp);
}

template <typename TS>
struct StageArgs {
    const Geo2* geos;
    size_t pitch;                          // member b's cells at b * pitch in every array
    const TS *h, *hu, *hv, *hw;            // state the rate is evaluated on (h or zeta first)
    const TS* d;                           // depth (FP64) or mound (FP32) at that state's time
    const TS* d0s;                         // FP32 copy of d0 (FP32 storage)
    const TS *h0, *hu0, *hv0, *hw0;        // Q^n
    TS *k1h, *k1u, *k1v, *k1w;             // stage-1 rates (written at stage 1, read at stage 2)
    TS *oh, *ohu, *ohv, *ohw;              // output: Q* (stage 1) or Q~ (stage 2)
    double dt;
    int stage;
    const TimeCtl* tc;                     // captured runs: skip after an aborted step
};

// Predictor stage on a kTX x kTY tile of cells held in shared memory with a
// two-cell halo in x (for the tile's rows) and in y (for its columns):
//  1. every tile and halo cell (mirrored / wrapped by g2_cell, odd parity on
//     the normal velocity) -> eta, u, v, w, d once (one reciprocal of h);
//  2. every x-face and y-face of the tile -> limited slopes of its two cells
//     and the Rusanov flux, once per face, with the normal momentum flux split
//     as F = A + (g/4)(hL^2 + hR^2) and the jump part G = (g/4)(hR + hL)(etaR - etaL);
//  3. every cell -> per direction -(A_r - A_l + G_r + G_l + g hbar sigma_eta)/ds
//     for the normal momentum (hbar = eta + (d_l + d_r)/2, the mean of its two
//     face thicknesses; algebraically the flux difference plus the bottom
//     source g hbar (d_r - d_l)/ds with the depth continuous at faces, and
//     exact for a lake at rest in any precision), flux differences for the
//     rest, then the Heun stage.
constexpr int kTX = 32, kTY = 8;                 // 256 threads, one cell each
constexpr int kHX = kTX + 4, kHY = kTY + 4;      // tile with halo
constexpr int kFX = (kTX + 1) * kTY;             // x-faces of a tile
constexpr int kFY = kTX * (kTY + 1);             // y-faces

// Face between cells L = -1 and R = 0 (e[k * s] is cell k's value): mass flux,
// normal momentum A and G parts, tangential momentum and hw fluxes.
template <typename T>
__device__ __forceinline__ void face_flux(T g, int lim, const T* e, const T* un, const T* ut, const T* w,
                                          const T* d, int s, T F[5])
{
    const T h2 = T(0.5);
    const T seL = slope2(lim, e[-2 * s], e[-s], e[0]), seR = slope2(lim, e[-s], e[0], e[s]);
    const T snL = slope2(lim, un[-2 * s], un[-s], un[0]), snR = slope2(lim, un[-s], un[0], un[s]);
    const T stL = slope2(lim, ut[-2 * s], ut[-s], ut[0]), stR = slope2(lim, ut[-s], ut[0], ut[s]);
    const T swL = slope2(lim, w[-2 * s], w[-s], w[0]), swR = slope2(lim, w[-s], w[0], w[s]);
    const T df = h2 * (d[-s] + d[0]);
    const T eL = e[-s] + h2 * seL, eR = e[0] - h2 * seR;
    const T uL = un[-s] + h2 * snL, uR = un[0] - h2 * snR;
    const T tL = ut[-s] + h2 * stL, tR = ut[0] - h2 * stR;
    const T wL = w[-s] + h2 * swL, wR = w[0] - h2 * swR;
    const T hL = eL + df, hR = eR + df;
    const T qL = hL * uL, qR = hR * uR;
    const T aL = fabs(uL) + wave_sqrt(g * hL), aR = fabs(uR) + wave_sqrt(g * hR);
    const T sp = aL > aR ? aL : aR;
    const T de = eR - eL;
    F[0] = h2 * (qL + qR) - h2 * sp * de;
    F[1] = h2 * (qL * uL + qR * uR) - h2 * sp * (qR - qL);
    F[2] = T(0.25) * g * (hR + hL) * de;
    F[3] = h2 * (qL * tL + qR * tR) - h2 * sp * (hR * tR - hL * tL);
    F[4] = h2 * (qL * wL + qR * wR) - h2 * sp * (hR * wR - hL * wL);
}

template <typename TS>
static __global__ void __launch_bounds__(kTX * kTY) k2_stage(StageArgs<TS> a)
{
    if (a.tc && a.tc->abort) return;
    __shared__ TS s_e[kHY][kHX], s_u[kHY][kHX], s_v[kHY][kHX], s_w[kHY][kHX], s_d[kHY][kHX];
    __shared__ TS s_fx[5][kTY][kTX + 1], s_fy[5][kTY + 1][kTX];
    const int b = blockIdx.y;
    const size_t mo = (size_t)b * a.pitch;
    const Geo2 G = a.geos[b];
    const int tiles_x = (G.nx + kTX - 1) / kTX, tiles = tiles_x * ((G.ny + kTY - 1) / kTY);
    const int tid = threadIdx.x, tx = tid % kTX, ty = tid / kTX;
    const TS* hz = a.h + mo; const TS* hu = a.hu + mo; const TS* hv = a.hv + mo;
    const TS* hw = a.hw + mo; const TS* dm = a.d + mo; const TS* d0s = a.d0s ? a.d0s + mo : nullptr;
    // constants in the storage precision, converted once per CTA
    __shared__ TS s_k[5];
    if (tid == 0) {
        s_k[0] = TS(G.g); s_k[1] = TS(G.idx); s_k[2] = TS(G.idy); s_k[3] = TS(a.dt); s_k[4] = TS(0.5 * a.dt);
    }
    __syncthreads();
    const TS g = s_k[0], idx = s_k[1], idy = s_k[2], h2 = TS(0.5);
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int i0 = (tile % tiles_x) * kTX, j0 = (tile / tiles_x) * kTY;
        // 1. primitives of the tile and its cross-shaped halo
        for (int q = tid; q < kHX * kHY; q += kTX * kTY) {
            const int lx = q % kHX, ly = q / kHX;
            const bool in_x = lx >= 2 && lx < kTX + 2, in_y = ly >= 2 && ly < kTY + 2;
            if (!in_x && !in_y) continue;   // corners: no stencil reaches them
            int ox, oy;
            const int c = g2_cell(G, i0 + lx - 2, j0 + ly - 2, &ox, &oy);
            TS hc, ec, dc;
            cell_hed<TS>(hz, dm, d0s, c, hc, ec, dc);
            const TS rh = TS(1) / hc;
            s_e[ly][lx] = ec;
            s_d[ly][lx] = dc;
            s_u[ly][lx] = flip(ox, hu[c] * rh);
            s_v[ly][lx] = flip(oy, hv[c] * rh);
            s_w[ly][lx] = hw[c] * rh;
        }
        __syncthreads();
        // 2. face fluxes: x-face (fx, r) between cells fx-1 and fx of row r;
        //    y-face (col, fy) between cells fy-1 and fy of column col
        for (int q = tid; q < kFX + kFY; q += kTX * kTY) {
            TS F[5];
            if (q < kFX) {
                const int fx = q % (kTX + 1), r = q / (kTX + 1);
                const int ly = r + 2, lx = fx + 2;
                face_flux<TS>(g, G.lim, &s_e[ly][lx], &s_u[ly][lx], &s_v[ly][lx], &s_w[ly][lx], &s_d[ly][lx], 1, F);
#pragma unroll
                for (int k = 0; k < 5; ++k) s_fx[k][r][fx] = F[k];
            } else {
                const int q2 = q - kFX, col = q2 % kTX, fy = q2 / kTX;
                const int ly = fy + 2, lx = col + 2;
                face_flux<TS>(g, G.lim, &s_e[ly][lx], &s_v[ly][lx], &s_u[ly][lx], &s_w[ly][lx], &s_d[ly][lx], kHX,
                              F);
#pragma unroll
                for (int k = 0; k < 5; ++k) s_fy[k][fy][col] = F[k];
            }
        }
        __syncthreads();
        // 3. rates and the stage
        const int i = i0 + tx, j = j0 + ty;
        if (i < G.nx && j < G.ny) {
            const int lx = tx + 2, ly = ty + 2;
            const TS ec = s_e[ly][lx], dc = s_d[ly][lx];
            const TS sex = slope2(G.lim, s_e[ly][lx - 1], ec, s_e[ly][lx + 1]);
            const TS hbx = ec + h2 * (h2 * (s_d[ly][lx - 1] + dc) + h2 * (dc + s_d[ly][lx + 1]));
            const TS sey = slope2(G.lim, s_e[ly - 1][lx], ec, s_e[ly + 1][lx]);
            const TS hby = ec + h2 * (h2 * (s_d[ly - 1][lx] + dc) + h2 * (dc + s_d[ly + 1][lx]));
            const TS rh = -(s_fx[0][ty][tx + 1] - s_fx[0][ty][tx]) * idx - (s_fy[0][ty + 1][tx] - s_fy[0][ty][tx]) * idy;
            const TS ru = -((s_fx[1][ty][tx + 1] - s_fx[1][ty][tx]) + (s_fx[2][ty][tx + 1] + s_fx[2][ty][tx])
                            + g * hbx * sex) * idx
                          - (s_fy[3][ty + 1][tx] - s_fy[3][ty][tx]) * idy;
            const TS rv = -(s_fx[3][ty][tx + 1] - s_fx[3][ty][tx]) * idx
                          - ((s_fy[1][ty + 1][tx] - s_fy[1][ty][tx]) + (s_fy[2][ty + 1][tx] + s_fy[2][ty][tx])
                             + g * hby * sey) * idy;
            const TS rw = -(s_fx[4][ty][tx + 1] - s_fx[4][ty][tx]) * idx - (s_fy[4][ty + 1][tx] - s_fy[4][ty][tx]) * idy;
            const size_t c = mo + (size_t)j * G.nx + i;
            const TS dt = s_k[3];
            if (a.stage == 1) {
                a.k1h[c] = rh; a.k1u[c] = ru; a.k1v[c] = rv; a.k1w[c] = rw;
                a.oh[c] = a.h0[c] + dt * rh;
                a.ohu[c] = a.hu0[c] + dt * ru;
                a.ohv[c] = a.hv0[c] + dt * rv;
                a.ohw[c] = a.hw0[c] + dt * rw;
            } else {
                const TS hdt = s_k[4];
                a.oh[c] = a.h0[c] + hdt * (a.k1h[c] + rh);
                a.ohu[c] = a.hu0[c] + hdt * (a.k1u[c] + ru);
                a.ohv[c] = a.hv0[c] + hdt * (a.k1v[c] + rv);
                a.ohw[c] = a.hw0[c] + hdt * (a.k1w[c] + rw);
            }
        }
        __syncthreads();
    }
}

// Criterion (Sec. 5.1, 2D form: |eta/d|, |grad eta|, |u|, |grad u|
// (Frobenius), |w|, |grad w|; central differences), strict > k_nh, in the
// storage precision; only the selected criterion's quantities are formed.
template <typename TS>
static __global__ void k2_marks(const Geo2* __restrict__ geos, size_t pitch, const TS* __restrict__ hz,
                                const TS* __restrict__ hu, const TS* __restrict__ hv,
                                const TS* __restrict__ hw, const TS* __restrict__ dm, const TS* __restrict__ d0s,
                                int crit, double knh, unsigned char* marks)
{
    const int b = blockIdx.y;
    const Geo2 G = geos[b];
    const size_t mo = (size_t)b * pitch;
    hz += mo; hu += mo; hv += mo; hw += mo; dm += mo; marks += mo;
    if (d0s) d0s += mo;
    const int N = G.nx * G.ny;
    const TS two_dx = TS(2.0 * G.dx), two_dy = TS(2.0 * G.dy);
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int i = c % G.nx, j = c / G.nx;
        TS val = TS(0);
        TS h, eta, d;
        if (crit == NH_CRIT_ETA_D) {
            cell_hed<TS>(hz, dm, d0s, c, h, eta, d);
            val = fabs(eta / d);
        } else if (crit == NH_CRIT_U) {
            cell_hed<TS>(hz, dm, d0s, c, h, eta, d);
            const TS uk = hu[c] / h, vk = hv[c] / h;
            val = sqrt(uk * uk + vk * vk);
        } else if (crit == NH_CRIT_W) {
            cell_hed<TS>(hz, dm, d0s, c, h, eta, d);
            val = fabs(hw[c] / h);
        } else {   // the gradient criteria: central differences over the four neighbours
            int o[4][2];
            const int nb[4] = {g2_cell(G, i - 1, j, &o[0][0], &o[0][1]), g2_cell(G, i + 1, j, &o[1][0], &o[1][1]),
                               g2_cell(G, i, j - 1, &o[2][0], &o[2][1]), g2_cell(G, i, j + 1, &o[3][0], &o[3][1])};
            TS hq[4], eq[4];
            for (int q = 0; q < 4; ++q) cell_hed<TS>(hz, dm, d0s, nb[q], hq[q], eq[q], d);
            if (crit == NH_CRIT_ETA_X) {
                const TS ex = (eq[1] - eq[0]) / two_dx, ey = (eq[3] - eq[2]) / two_dy;
                val = sqrt(ex * ex + ey * ey);
            } else if (crit == NH_CRIT_U_X) {
                TS u[4], v[4];
                for (int q = 0; q < 4; ++q) {
                    const int m = nb[q];
                    u[q] = flip(o[q][0], hu[m]) / hq[q];
                    v[q] = flip(o[q][1], hv[m]) / hq[q];
                }
                const TS ux = (u[1] - u[0]) / two_dx, uy = (u[3] - u[2]) / two_dy;
                const TS vx = (v[1] - v[0]) / two_dx, vy = (v[3] - v[2]) / two_dy;
                val = sqrt(ux * ux + uy * uy + vx * vx + vy * vy);
            } else if (crit == NH_CRIT_W_X) {
                TS w[4];
                for (int q = 0; q < 4; ++q) w[q] = hw[nb[q]] / hq[q];
                const TS wx = (w[1] - w[0]) / two_dx, wy = (w[3] - w[2]) / two_dy;
                val = sqrt(wx * wx + wy * wy);
            }
        }
        marks[c] = val > TS(knh) ? 1 : 0;
    }
}

// Moore enlargement of radius e (walls stop it, periodic sides wrap).
static __global__ void k2_dilate(const Geo2* __restrict__ geos, size_t pitch, const unsigned char* __restrict__ marks,
                                 int e, unsigned char* act, const TimeCtl* __restrict__ tc)
{
    if (tc && tc->abort) return;
    const int b = blockIdx.y;
    const Geo2 G = geos[b];
    const size_t mo = (size_t)b * pitch;
    marks += mo; act += mo;
    const int N = G.nx * G.ny;
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < N; c += gridDim.x * blockDim.x) {
        const int i = c % G.nx, j = c / G.nx;
        unsigned char m = 0;
        for (int b = -e; b <= e && !m; ++b)
            for (int a2 = -e; a2 <= e; ++a2) {
                const int q = g2_inner(G, i + a2, j + b);
                if (q >= 0 && marks[q]) { m = 1; break; }
            }
        act[c] = m;
    }
}

constexpr int kCompact2 = 1024;   // cells per compaction block

static __global__ void __launch_bounds__(kCompact2) k2_count(const Geo2* __restrict__ geos, size_t pitch,
                                                            const unsigned char* __restrict__ act, int nblk, int* cnt)
{
    __shared__ int s[32];
    const int b = blockIdx.y;
    const int N = geos[b].nx * geos[b].ny;
    act += (size_t)b * pitch;
    cnt += (size_t)b * nblk;
    const int c = blockIdx.x * kCompact2 + threadIdx.x;
    const int v = (c < N && act[c]) ? 1 : 0;
    const int wsum = __popc(__ballot_sync(0xffffffffu, v));
    if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = wsum;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int q = 0; q < kCompact2 / 32; ++q) t += s[q];
        cnt[blockIdx.x] = t;
    }
}

// Exclusive scan of a member's block counts (one CTA per member); the
// member's solver state is reset as the 1D compaction does, with n_active =
// the total.
static __global__ void __launch_bounds__(1024) k2_scan(const int* __restrict__ cnt, int nblk, int* off, int* nact,
                                                       MState* ms, const TimeCtl* __restrict__ tc)
{
    __shared__ int s_w[32];
    __shared__ int s_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int mb = blockIdx.x;   // member
    cnt += (size_t)mb * nblk;
    off += (size_t)mb * nblk;
    nact += mb;
    ms += mb;
    if (tc && tc->abort) {   // captured run after a failed step: park the solver
        if (tid == 0) ms->done = 1;
        return;
    }
    if (tid == 0) s_base = 0;
    __syncthreads();
    for (int b0 = 0; b0 < nblk; b0 += 1024) {
        const int b = b0 + tid;
        const int v = b < nblk ? cnt[b] : 0;
        int incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int x = s_w[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            s_w[lane] = x;
        }
        __syncthreads();
        if (b < nblk) off[b] = s_base + incl - v + (wid > 0 ? s_w[wid - 1] : 0);
        __syncthreads();
        if (tid == 0) s_base += s_w[31];
        __syncthreads();
    }
    if (tid == 0) {
        const int n = s_base;
        *nact = n;
        MState s;
        s.bnorm2 = 0.0; s.bnorm = 0.0; s.rr = 0.0; s.alpha = 1.0; s.beta = 0.0; s.omega = 1.0;
        s.rel_res = 0.0; s.min_gamma = 0.0; s.snorm = 0.0; s.rz = 0.0;
        s.status = NH_OK; s.iters = 0; s.done = (n == 0); s.kind = -1; s.zero_sol = 0;
        s.s_conv = 0; s.n_active = n; s.nchunks = (n + kChunk - 1) / kChunk;
        s.auto_kind = 0; s.npb = (n + kPcrRows - 1) / kPcrRows; s.ioff = 0; s.poff = 0;
        ms[0] = s;
    }
}

// list[k] = k-th active cell in row-major order; inv[c] = k, or -1.
static __global__ void __launch_bounds__(kCompact2) k2_emit(const Geo2* __restrict__ geos, size_t pitch,
                                                           const unsigned char* __restrict__ act, int nblk,
                                                           const int* __restrict__ off, int* list, int* inv,
                                                           const TimeCtl* __restrict__ tc)
{
    if (tc && tc->abort) return;
    __shared__ int s_w[32];
    const int b = blockIdx.y;
    const int N = geos[b].nx * geos[b].ny;
    act += (size_t)b * pitch; list += (size_t)b * pitch; inv += (size_t)b * pitch;
    off += (size_t)b * nblk;
    const int c = blockIdx.x * kCompact2 + threadIdx.x;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const bool v = c < N && act[c];
    const unsigned bal = __ballot_sync(0xffffffffu, v);
    if (lane == 0) s_w[wid] = __popc(bal);
    __syncthreads();
    if (wid == 0) {
        int x = s_w[lane];
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        s_w[lane] = x;   // inclusive
    }
    __syncthreads();
    if (c < N) {
        if (v) {
            const int k = off[blockIdx.x] + (wid > 0 ? s_w[wid - 1] : 0) + __popc(bal & ((1u << lane) - 1u));
            list[k] = c;
            inv[c] = k;
        } else {
            inv[c] = -1;
        }
    }
}

// Per-cell quantities of the elliptic equation (psi form).
struct CellQ2 {
    double h, Kxx, Kyy, Kxy, bx, by, Vx, Vy, U0, V0, phi, d_x, d_y, d_t, G, D;
};

template <typename TS>
struct Asm2Args {
    const Geo2* geos; const Slide2* slides;
    const Kin2* kin;                       // kin[2b + 1]: bottom motion at t^{n+1}
    int nb, pitch, maxch;
    const TS *ht, *hut, *hvt, *hwt;        // Q~ (h or zeta first)
    const double* d0;
    const TS* d1;                          // depth (FP64) or mound (FP32) at t^{n+1}
    double dt;
    const int* list; const int* inv;
    MState* ms;
    double *diag, *offl, *offr, *R;
    int *nbl, *nbr;
    double* ext_c; int* ext_k; size_t ext_stride;   // S, N, SW, SE, NW, NE; stride nb * pitch
    double *c6, *cx, *cy, *phi, *ddx, *ddy;
    double* cq;                            // [kCq][nb * pitch] per-cell fields (k2_cellq); stride ext_stride
    double* part; int* cnt;                // part: [2][nb * maxch]
    int solver;
    const int2* items; const Ctl* ctl;
};

// One member's fields as seen by the assembly (pointers at the member's
// slice); h and eta in FP64 from either storage.
template <typename TS>
struct Mem2 {
    Geo2 G; Slide2 S; Kin2 K;
    const TS *ht, *hut, *hvt, *d1;
    const double* d0;
    double dt;
    __device__ __forceinline__ double h_at(int k) const
    {
        if constexpr (sizeof(TS) == 8) return ht[k];
        else return (double)ht[k] + d0[k];
    }
    __device__ __forceinline__ double eta_at(int k) const
    {
        if constexpr (sizeof(TS) == 8) return ht[k] - d1[k];
        else return (double)ht[k] + (double)d1[k];
    }
};

template <typename TS>
__device__ __forceinline__ CellQ2 cell_q2(const Mem2<TS>& a, int i, int j)
{
    const Geo2& G = a.G;
    double b[10];
    int o1, o2;
    bottom2(G, a.d0, a.S, a.K, i, j, b);
    const int kw = g2_cell(G, i - 1, j, &o1, &o2), ke = g2_cell(G, i + 1, j, &o1, &o2);
    const int ks = g2_cell(G, i, j - 1, &o1, &o2), kn = g2_cell(G, i, j + 1, &o1, &o2);
    const double eta_x = (a.eta_at(ke) - a.eta_at(kw)) * (0.5 * G.idx);
    const double eta_y = (a.eta_at(kn) - a.eta_at(ks)) * (0.5 * G.idy);
    const int k = j * G.nx + i;
    CellQ2 q;
    q.h = a.h_at(k);
    const double rh = 1.0 / q.h;
    const double u = (double)a.hut[k] * rh, v = (double)a.hvt[k] * rh;
    q.d_x = b[1]; q.d_y = b[2]; q.d_t = b[6];
    const double d_xx = b[3], d_yy = b[4], d_xy = b[5], d_xt = b[7], d_yt = b[8], d_tt = b[9];
    q.G = q.d_x * q.d_x + q.d_y * q.d_y;
    q.D = 4.0 + q.G;
    const double rD = 1.0 / q.D;
    q.phi = a.dt * q.h * rD * (G.g * (q.d_x * eta_x + q.d_y * eta_y) - d_tt - 2.0 * (u * d_xt + v * d_yt)
                                - (u * u * d_xx + 2.0 * u * v * d_xy + v * v * d_yy));
    q.Kxx = rh * (1.0 - q.d_x * q.d_x * rD);
    q.Kyy = rh * (1.0 - q.d_y * q.d_y * rD);
    q.Kxy = -rh * q.d_x * q.d_y * rD;
    q.bx = 6.0 * q.d_x * (rh * rh * rD);
    q.by = 6.0 * q.d_y * (rh * rh * rD);
    q.U0 = (double)a.hut[k] + q.phi * q.d_x;
    q.V0 = (double)a.hvt[k] + q.phi * q.d_y;
    q.Vx = q.U0 * rh;
    q.Vy = q.V0 * rh;
    return q;
}

// The fields of a cell that its neighbours' rows use (Kxx, Kyy, Kxy, bx, by,
// Vx, Vy), stored per cell by k2_cellq so each is computed once per step.
constexpr int kCq = 7;

// The same seen from a neighbour: mirrored cells flip their odd components.
template <typename TS>
__device__ __forceinline__ CellQ2 cell_q2_at(const Mem2<TS>& a, int i, int j)
{
    int ox, oy;
    const int c = g2_cell(a.G, i, j, &ox, &oy);
    CellQ2 q = cell_q2(a, c % a.G.nx, c / a.G.nx);
    q.Kxy = flip(ox * oy, q.Kxy);
    q.bx = flip(ox, q.bx); q.by = flip(oy, q.by);
    q.Vx = flip(ox, q.Vx); q.Vy = flip(oy, q.Vy);
    return q;
}

// A neighbour's stored fields (cq: [kCq][nb * pitch], member slice at mo),
// mirrored cells flipping their odd components.
__device__ __forceinline__ CellQ2 cell_q2_stored(const Geo2& G, const double* __restrict__ cq, size_t T, size_t mo,
                                                 int i, int j)
{
    int ox, oy;
    const size_t c = mo + g2_cell(G, i, j, &ox, &oy);
    CellQ2 q;
    q.Kxx = cq[c];
    q.Kyy = cq[T + c];
    q.Kxy = flip(ox * oy, cq[2 * T + c]);
    q.bx = flip(ox, cq[3 * T + c]);
    q.by = flip(oy, cq[4 * T + c]);
    q.Vx = flip(ox, cq[5 * T + c]);
    q.Vy = flip(oy, cq[6 * T + c]);
    return q;
}

__device__ __forceinline__ void cq_store(double* __restrict__ cq, size_t T, size_t c, const CellQ2& q)
{
    cq[c] = q.Kxx; cq[T + c] = q.Kyy; cq[2 * T + c] = q.Kxy; cq[3 * T + c] = q.bx; cq[4 * T + c] = q.by;
    cq[5 * T + c] = q.Vx; cq[6 * T + c] = q.Vy;
}

// Per-cell quantities of every active cell and of each in-domain cell its
// 9-point row reaches in x and y (mirrored or wrapped), stored once so the
// assembly reads neighbours instead of recomputing them.  Two active cells
// may share an inactive neighbour: both write the same values.
template <typename TS>
static __global__ void __launch_bounds__(kChunk) k2_cellq(Asm2Args<TS> a)
{
    const int n_items = a.ctl->n_items;
    const size_t T = a.ext_stride;
    for (int wi = blockIdx.x; wi < n_items; wi += gridDim.x) {
        const int2 itm = a.items[wi];
        const int b = itm.x;
        const int n = a.ms[b].n_active;
        const int k = itm.y * kChunk + threadIdx.x;
        if (k >= n) continue;
        const size_t mo = (size_t)b * a.pitch;
        Mem2<TS> m;
        m.G = a.geos[b]; m.S = a.slides[b]; m.K = a.kin[2 * b + 1];
        m.ht = a.ht + mo; m.hut = a.hut + mo; m.hvt = a.hvt + mo; m.d0 = a.d0 + mo; m.d1 = a.d1 + mo;
        m.dt = a.dt;
        const Geo2& G = m.G;
        const int c = a.list[mo + k];
        const int i = c % G.nx, j = c / G.nx;
        cq_store(a.cq, T, mo + c, cell_q2(m, i, j));
        const int di[4] = {-1, 1, 0, 0}, dj[4] = {0, 0, -1, 1};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            int ox, oy;
            const int cn = g2_cell(G, i + di[q], j + dj[q], &ox, &oy);
            if (a.inv[mo + cn] >= 0) continue;   // active: its own thread stores it
            cq_store(a.cq, T, mo + cn, cell_q2(m, cn % G.nx, cn / G.nx));
        }
    }
}

// Rows of the 9-point operator on the active cells (work items of kChunk
// list entries of one member) and each member's ||R||^2 and min gamma.
template <typename TS>
static __global__ void __launch_bounds__(kChunk) k2_assemble(Asm2Args<TS> a)
{
    __shared__ double red[64];
    const int n_items = a.ctl->n_items;
    for (int wi = blockIdx.x; wi < n_items; wi += gridDim.x) {
        const int2 itm = a.items[wi];
        const int b = itm.x, jj = itm.y;
        const int n = a.ms[b].n_active, nch = a.ms[b].nchunks, ioff = a.ms[b].ioff;
        const size_t mo = (size_t)b * a.pitch;
        Mem2<TS> m;
        m.G = a.geos[b]; m.S = a.slides[b]; m.K = a.kin[2 * b + 1];
        m.ht = a.ht + mo; m.hut = a.hut + mo; m.hvt = a.hvt + mo; m.d0 = a.d0 + mo; m.d1 = a.d1 + mo;
        m.dt = a.dt;
        const Geo2& G = m.G;
        const int* inv = a.inv + mo;
        const double idx2 = G.idx * G.idx, idy2 = G.idy * G.idy, ixy = 0.25 * G.idx * G.idy;
        const int k = jj * kChunk + threadIdx.x;
        double r2 = 0.0, gmin = INFINITY;
        if (k < n) {
            const size_t o = mo + k;
            const int c = a.list[o];
            const int i = c % G.nx, j = c / G.nx;
            const CellQ2 q = cell_q2(m, i, j);
            const size_t T = a.ext_stride;
            const CellQ2 W = cell_q2_stored(G, a.cq, T, mo, i - 1, j), E = cell_q2_stored(G, a.cq, T, mo, i + 1, j);
            const CellQ2 S = cell_q2_stored(G, a.cq, T, mo, i, j - 1), N = cell_q2_stored(G, a.cq, T, mo, i, j + 1);
            const double Kw = 0.5 * (W.Kxx + q.Kxx), Ke = 0.5 * (q.Kxx + E.Kxx);
            const double Ks = 0.5 * (S.Kyy + q.Kyy), Kn = 0.5 * (q.Kyy + N.Kyy);
            const double div_beta = (E.bx - W.bx) * (0.5 * G.idx) + (N.by - S.by) * (0.5 * G.idy);
            const double div_V = (E.Vx - W.Vx) * (0.5 * G.idx) + (N.Vy - S.Vy) * (0.5 * G.idy);
            const double h = q.h, rh = 1.0 / h, rh2 = rh * rh;
            const double gam = div_beta + 12.0 * (1.0 + q.G) * (rh2 * rh) / q.D;
            const double Rk = -(div_V + 2.0 * (q.d_x * q.U0 + q.d_y * q.V0) * rh2 + 2.0 * (double)a.hwt[mo + c] * rh2
                                + 2.0 * q.phi * rh2 + 2.0 * q.d_t * rh);
            const double cW = -Kw * idx2, cE = -Ke * idx2, cS = -Ks * idy2, cN = -Kn * idy2;
            const double cNE = -(E.Kxy + N.Kxy) * ixy, cSW = -(W.Kxy + S.Kxy) * ixy;
            const double cSE = (E.Kxy + S.Kxy) * ixy, cNW = (W.Kxy + N.Kxy) * ixy;
            auto nbk = [&](int di, int dj) {
                const int qc = g2_inner(G, i + di, j + dj);
                return qc >= 0 ? inv[qc] : -1;
            };
            const int kW = nbk(-1, 0), kE = nbk(1, 0);
            const int ke[6] = {nbk(0, -1), nbk(0, 1), nbk(-1, -1), nbk(1, -1), nbk(-1, 1), nbk(1, 1)};
            const double ce[6] = {cS, cN, cSW, cSE, cNW, cNE};
            a.diag[o] = (Kw + Ke) * idx2 + (Ks + Kn) * idy2 + gam;
            a.offl[o] = kW >= 0 ? cW : 0.0;
            a.offr[o] = kE >= 0 ? cE : 0.0;
            a.nbl[o] = kW;
            a.nbr[o] = kE;
            for (int e = 0; e < 6; ++e) {
                a.ext_c[e * a.ext_stride + o] = ke[e] >= 0 ? ce[e] : 0.0;
                a.ext_k[e * a.ext_stride + o] = ke[e];
            }
            a.R[o] = Rk;
            const double rD = 1.0 / q.D;
            a.c6[o] = 6.0 * rh * rD;
            a.cx[o] = q.d_x * rD;
            a.cy[o] = q.d_y * rD;
            a.phi[o] = q.phi;
            a.ddx[o] = q.d_x;
            a.ddy[o] = q.d_y;
            r2 = Rk * Rk;
            gmin = gam;
        }
        double v[1] = {r2};
        block_sum<1>(v, red);
        const double gm = block_min(gmin, red);
        double* P0 = a.part;
        double* P1 = a.part + (size_t)a.nb * a.maxch;
        if (threadIdx.x == 0) { P0[wi] = v[0]; P1[wi] = gm; }
        if (arrive_last(a.cnt, b, nch)) {
            const double bn2 = member_sum(P0 + ioff, nch, red);
            const double gmn = member_min(P1 + ioff, nch, red);
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                s.bnorm2 = bn2;
                s.bnorm = sqrt(bn2);
                s.min_gamma = gmn;
                s.auto_kind = (a.solver == NH_SOLVER_AUTO);
                s.kind = (a.solver == NH_SOLVER_BICGSTAB) ? NH_SOLVER_BICGSTAB : NH_SOLVER_CG;
            }
        }
    }
}

template <typename TS>
struct Corr2Args {
    const Geo2* geos;
    int pitch;
    const int* list;
    const int* nbl; const int* nbr; const int* ext_k; size_t ext_stride;
    const double* x;             // psi on the active cells
    const double *c6, *cx, *cy, *phi, *ddx, *ddy;
    const MState* ms;
    TS *hu, *hv, *hw;            // Q~, corrected in place (FP64 arithmetic)
    double* psi;                 // dense psi (warm start, pressure output)
    const int2* items; const Ctl* ctl;
    const TimeCtl* tc;           // captured runs: skip unless the step was accepted
};

// Eqs. 10-11 in 2D: with psi = a q, P = c6 psi + cx psi_x + cy psi_y + a phi;
// U = U~ - grad psi + grad d P, hw = hw~ + P; psi = 0 off the mask.
template <typename TS>
static __global__ void __launch_bounds__(kChunk) k2_correct(Corr2Args<TS> a)
{
    if (a.tc && a.tc->abort) return;
    const int n_items = a.ctl->n_items;
    for (int wi = blockIdx.x; wi < n_items; wi += gridDim.x) {
        const int2 itm = a.items[wi];
        const int b = itm.x;
        const int k = itm.y * kChunk + threadIdx.x;
        if (k >= a.ms[b].n_active) continue;
        const bool zero = a.ms[b].zero_sol != 0;
        const size_t mo = (size_t)b * a.pitch, o = mo + k;
        const double dx = a.geos[b].dx, dy = a.geos[b].dy;
        const double* x = a.x + mo;
        const int kw = a.nbl[o], ke = a.nbr[o];
        const int ks = a.ext_k[o], kn = a.ext_k[a.ext_stride + o];
        const double ps = zero ? 0.0 : x[k];
        const double pw = (zero || kw < 0) ? 0.0 : x[kw], pe = (zero || ke < 0) ? 0.0 : x[ke];
        const double pss = (zero || ks < 0) ? 0.0 : x[ks], pn = (zero || kn < 0) ? 0.0 : x[kn];
        const double px = (pe - pw) / (2.0 * dx), py = (pn - pss) / (2.0 * dy);
        const double P = a.c6[o] * ps + a.cx[o] * px + a.cy[o] * py + a.phi[o];
        const size_t c = mo + a.list[o];
        a.hu[c] = TS((double)a.hu[c] + (-px + a.ddx[o] * P));
        a.hv[c] = TS((double)a.hv[c] + (-py + a.ddy[o] * P));
        a.hw[c] = TS((double)a.hw[c] + P);
        a.psi[c] = ps;
    }
}

// Block partial sums of h dx dy (FP64; h = zeta + d0 for FP32 storage):
// part[b * gridDim.x + blockIdx.x].
template <typename TS>
static __global__ void __launch_bounds__(256) k2_mass(const Geo2* __restrict__ geos, size_t pitch,
                                                     const TS* __restrict__ hz, const double* __restrict__ d0,
                                                     double* part)
{
    __shared__ double red[32];
    const int b = blockIdx.y;
    const int N = geos[b].nx * geos[b].ny;
    hz += (size_t)b * pitch;
    d0 += (size_t)b * pitch;
    double v[1] = {0.0};
    for (int c = blockIdx.x * 256 + threadIdx.x; c < N; c += gridDim.x * 256) {
        if constexpr (sizeof(TS) == 8) v[0] += hz[c];
        else v[0] += (double)hz[c] + d0[c];
    }
    block_sum<1>(v, red);
    if (threadIdx.x == 0) part[(size_t)b * gridDim.x + blockIdx.x] = v[0] * geos[b].dx * geos[b].dy;
}

// One member's state between FP64 (h, hu, hv, hw) and FP32 storage
// (zeta = h - d0, hu, hv, hw); n cells.
static __global__ void k2_store_f32(int n, const double* __restrict__ d0, const double* __restrict__ h,
                                    const double* __restrict__ hu, const double* __restrict__ hv,
                                    const double* __restrict__ hw, float* z, float* u, float* v, float* w)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        z[c] = (float)(h[c] - d0[c]);
        u[c] = (float)hu[c];
        v[c] = (float)hv[c];
        w[c] = (float)hw[c];
    }
}

static __global__ void k2_load_f32(int n, const double* __restrict__ d0, const float* __restrict__ z,
                                   const float* __restrict__ u, const float* __restrict__ v,
                                   const float* __restrict__ w, double* h, double* hu, double* hv, double* hw)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        h[c] = (double)z[c] + d0[c];
        hu[c] = (double)u[c];
        hv[c] = (double)v[c];
        hw[c] = (double)w[c];
    }
}

static __global__ void k2_to_f32(size_t n, const double* __restrict__ src, float* dst)
{
    for (size_t c = blockIdx.x * (size_t)blockDim.x + threadIdx.x; c < n; c += (size_t)gridDim.x * blockDim.x)
        dst[c] = (float)src[c];
}

}  // namespace nh
