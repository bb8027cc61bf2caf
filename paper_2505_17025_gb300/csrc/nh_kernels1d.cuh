// nh_kernels1d.cuh -- the 1D batched kernels of one time step.
//
//  k_kinematics  slide position / velocity / acceleration per member       (a1)
//  k_predict     both Heun stages of the hydrostatic predictor in one
//                shared-memory halo tile, plus the criterion marks        (a2, a3)
//  k_compact     enlargement and order-preserving compaction of the marked
//                cells into a per-member active list (ballot + block scan) (a3)
//  k_assemble    elliptic coefficients and right-hand side on active cells  (a4)
//  k_*_init / k_cg_* / k_bi_*   Krylov solve on the active cells            (a5)
//  k_clear_prev / k_correct     correction of hu, hw; pressure scatter       (a6)
//
// Layout: every per-cell field of member b lives at [b * pitch + i]; every
// per-active-cell array of member b at [b * pitch + k], k < n_active(b).
#pragma once

#include "nh_internal.cuh"

namespace nh {

struct Geo {
    int nx, nb, pitch, wpitch, bc, lim, ntiles, maxch;
    double dx, x0, g;
};

// ------------------------------------------------------------------ slide

__global__ void k_kinematics(const Slide* __restrict__ sl, Kin* __restrict__ kin, int nb,
                             double t_n, double t_n1)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    Slide s = sl[b];
    Kin k{0.0, 0.0, 0.0, 0.0};
    if (s.shape == NH_SLIDE_GAUSS_LNCOSH) {
        // s(t) = s0 ln cosh(t/t0);  s' = (s0/t0) tanh(t/t0);  s'' = (s0/t0^2) / cosh^2(t/t0)
        double zn = t_n / s.t0, z1 = t_n1 / s.t0;
        k.s_n = s.s0 * log(cosh(zn));
        k.s_n1 = s.s0 * log(cosh(z1));
        k.sd_n1 = (s.s0 / s.t0) * tanh(z1);
        double c1 = cosh(z1);
        k.sdd_n1 = (s.s0 / (s.t0 * s.t0)) / (c1 * c1);
    }
    kin[b] = k;
}

// -------------------------------------------------------------- predictor

template <typename T>
__device__ __forceinline__ T minmod(T a, T b)
{
    if (a * b <= T(0)) return T(0);
    return tabs(a) < tabs(b) ? a : b;
}

template <typename T>
__device__ __forceinline__ T limited_slope(int lim, T vm, T v0, T vp)
{
    switch (lim) {
    case NH_LIM_CENTRAL: return T(0.5) * (vp - vm);
    case NH_LIM_MINMOD:  return minmod(vp - v0, v0 - vm);
    case NH_LIM_MC:      return minmod(T(0.5) * (vp - vm), minmod(T(2) * (vp - v0), T(2) * (v0 - vm)));
    default:             return T(0);
    }
}

// Local Lax-Friedrichs (Rusanov) flux of (hu, hu^2 + g h^2 / 2, huw).
template <typename T>
__device__ __forceinline__ void rusanov(T g, T hL, T uL, T wL, T hR, T uR, T wR,
                                        T& F0, T& F1, T& F2)
{
    const T qL = hL * uL, qR = hR * uR;
    const T aL = tabs(uL) + tsqrt(g * hL), aR = tabs(uR) + tsqrt(g * hR);
    const T s = aL > aR ? aL : aR;
    const T fL = qL * uL + T(0.5) * g * hL * hL;
    const T fR = qR * uR + T(0.5) * g * hR * hR;
    F0 = T(0.5) * (qL + qR) - T(0.5) * s * (hR - hL);
    F1 = T(0.5) * (fL + fR) - T(0.5) * s * (qR - qL);
    F2 = T(0.5) * (qL * wL + qR * wR) - T(0.5) * s * (hR * wR - hL * wL);
}

template <typename T>
struct PredArgs {
    Geo G;
    const T* h; const T* hu; const T* hw;     // Q^n
    T* ht; T* hut; T* hwt;                    // Q~^{n+1}
    const T* d0;
    const Slide* slide; const Kin* kin;
    uint32_t* marks;                          // nb * wpitch words
    double* mass_part;                        // nb * ntiles
    double dt;
    double knh;
    int crit;
    int all_global;                           // mark every cell this step
};

// One CTA = one tile of kPredTile cells of one member.  Q^n is loaded with a
// halo of 5 cells (ghosts mirrored at walls, wrapped when periodic); stage 1
// (bottom at t^n) is evaluated on the tile plus 3 cells each side, stage 2
// (bottom at t^{n+1}) on the tile plus one cell each side, so the criterion's
// central differences need no second pass.  Q~ = Q^n + dt/2 (k1 + k2).
template <typename T>
__global__ void __launch_bounds__(kPredTile) k_predict(PredArgs<T> a)
{
    constexpr int TILE = kPredTile, H = kPredHalo, NL = TILE + 2 * H;
    __shared__ T sh[NL], shu[NL], shw[NL];      // Q^n, later Q~
    __shared__ T se[NL], su[NL], sw[NL];        // stage primitives eta, u, w
    __shared__ T sdn[NL], sdn1[NL];             // depth at t^n, t^{n+1}
    __shared__ T sle[NL], slu[NL], slw[NL];     // limited slopes
    __shared__ T F0[NL], F1[NL], F2[NL];        // face l: between local cells l-1 and l
    __shared__ T k1h[NL], k1u[NL], k1w[NL];     // stage-1 rates
    __shared__ double red[32];

    const Geo& G = a.G;
    const int b = blockIdx.y, i0 = blockIdx.x * TILE, tid = threadIdx.x;
    const size_t mo = (size_t)b * G.pitch;
    const T* __restrict__ Hn = a.h + mo;
    const T* __restrict__ HUn = a.hu + mo;
    const T* __restrict__ HWn = a.hw + mo;
    const T* __restrict__ D0 = a.d0 + mo;
    const Slide sl = a.slide[b];
    const Kin kn = a.kin[b];
    const T g = T(G.g), dx = T(G.dx), dt = T(a.dt), half_dt = T(0.5) * T(a.dt);

    // A: load Q^n and the bottom at both times.  Cells outside [-6, nx+5]
    // feed only outputs outside [-1, nx] and get a benign still state.
    for (int l = tid; l < NL; l += TILE) {
        const int j = i0 - H + l;
        T hv = T(1), huv = T(0), hwv = T(0), dn = T(1), dn1 = T(1);
        if (j >= -6 && j <= G.nx + 5) {
            int sg;
            const int c = resolve(j, G.nx, G.bc, &sg);
            hv = Hn[c];
            huv = sg > 0 ? HUn[c] : -HUn[c];
            hwv = HWn[c];
            dn = depth_at(D0, c, G.x0, G.dx, sl, kn.s_n);
            dn1 = depth_at(D0, c, G.x0, G.dx, sl, kn.s_n1);
        }
        sh[l] = hv; shu[l] = huv; shw[l] = hwv; sdn[l] = dn; sdn1[l] = dn1;
        se[l] = hv - dn; su[l] = huv / hv; sw[l] = hwv / hv;
    }
    __syncthreads();

    // B: stage-1 slopes on local cells [1, NL-1)
    for (int l = tid + 1; l < NL - 1; l += TILE) {
        sle[l] = limited_slope(G.lim, se[l - 1], se[l], se[l + 1]);
        slu[l] = limited_slope(G.lim, su[l - 1], su[l], su[l + 1]);
        slw[l] = limited_slope(G.lim, sw[l - 1], sw[l], sw[l + 1]);
    }
    __syncthreads();

    // C: stage-1 face fluxes on faces [2, NL-1); depth continuous at faces
    for (int f = tid + 2; f < NL - 1; f += TILE) {
        const T df = T(0.5) * (sdn[f - 1] + sdn[f]);
        const T hL = se[f - 1] + T(0.5) * sle[f - 1] + df;
        const T uL = su[f - 1] + T(0.5) * slu[f - 1];
        const T wL = sw[f - 1] + T(0.5) * slw[f - 1];
        const T hR = se[f] - T(0.5) * sle[f] + df;
        const T uR = su[f] - T(0.5) * slu[f];
        const T wR = sw[f] - T(0.5) * slw[f];
        rusanov(g, hL, uL, wL, hR, uR, wR, F0[f], F1[f], F2[f]);
    }
    __syncthreads();

    // D: stage-1 rates and Q* on cells [2, NL-2); Q* stored as primitives
    //    against the bottom at t^{n+1}
    for (int l = tid + 2; l < NL - 2; l += TILE) {
        const T dfl = T(0.5) * (sdn[l - 1] + sdn[l]), dfr = T(0.5) * (sdn[l] + sdn[l + 1]);
        const T hpl = se[l] - T(0.5) * sle[l] + dfl, hmr = se[l] + T(0.5) * sle[l] + dfr;
        const T S = g * T(0.5) * (hpl + hmr) * (dfr - dfl) / dx;
        const T r0 = -(F0[l + 1] - F0[l]) / dx;
        const T r1 = -(F1[l + 1] - F1[l]) / dx + S;
        const T r2 = -(F2[l + 1] - F2[l]) / dx;
        k1h[l] = r0; k1u[l] = r1; k1w[l] = r2;
        const T hs = sh[l] + dt * r0, hus = shu[l] + dt * r1, hws = shw[l] + dt * r2;
        se[l] = hs - sdn1[l]; su[l] = hus / hs; sw[l] = hws / hs;
    }
    __syncthreads();

    // E: stage-2 slopes on [3, NL-3)
    for (int l = tid + 3; l < NL - 3; l += TILE) {
        sle[l] = limited_slope(G.lim, se[l - 1], se[l], se[l + 1]);
        slu[l] = limited_slope(G.lim, su[l - 1], su[l], su[l + 1]);
        slw[l] = limited_slope(G.lim, sw[l - 1], sw[l], sw[l + 1]);
    }
    __syncthreads();

    // F: stage-2 fluxes on faces [4, NL-3)
    for (int f = tid + 4; f < NL - 3; f += TILE) {
        const T df = T(0.5) * (sdn1[f - 1] + sdn1[f]);
        const T hL = se[f - 1] + T(0.5) * sle[f - 1] + df;
        const T uL = su[f - 1] + T(0.5) * slu[f - 1];
        const T wL = sw[f - 1] + T(0.5) * slw[f - 1];
        const T hR = se[f] - T(0.5) * sle[f] + df;
        const T uR = su[f] - T(0.5) * slu[f];
        const T wR = sw[f] - T(0.5) * slw[f];
        rusanov(g, hL, uL, wL, hR, uR, wR, F0[f], F1[f], F2[f]);
    }
    __syncthreads();

    // G: stage-2 rates and Q~ on [4, NL-4) (the tile and one cell each side)
    for (int l = tid + 4; l < NL - 4; l += TILE) {
        const T dfl = T(0.5) * (sdn1[l - 1] + sdn1[l]), dfr = T(0.5) * (sdn1[l] + sdn1[l + 1]);
        const T hpl = se[l] - T(0.5) * sle[l] + dfl, hmr = se[l] + T(0.5) * sle[l] + dfr;
        const T S = g * T(0.5) * (hpl + hmr) * (dfr - dfl) / dx;
        const T r0 = -(F0[l + 1] - F0[l]) / dx;
        const T r1 = -(F1[l + 1] - F1[l]) / dx + S;
        const T r2 = -(F2[l + 1] - F2[l]) / dx;
        const T hn = sh[l] + half_dt * (k1h[l] + r0);
        const T hun = shu[l] + half_dt * (k1u[l] + r1);
        const T hwn = shw[l] + half_dt * (k1w[l] + r2);
        sh[l] = hn; shu[l] = hun; shw[l] = hwn;
        const int j = i0 - H + l;
        if (j >= i0 && j < i0 + TILE && j < G.nx) {
            a.ht[mo + j] = hn; a.hut[mo + j] = hun; a.hwt[mo + j] = hwn;
        }
    }
    __syncthreads();

    // H: criterion (Sec. 5.1) on the tile; marks as one bit per cell
    {
        const int l = tid + H, j = i0 + tid;
        const bool inside = j < G.nx;
        bool mark = false;
        double mass = 0.0;
        if (inside) {
            mass = (double)sh[l];
            if (a.all_global) {
                mark = true;
            } else if (a.crit >= NH_CRIT_ETA_D) {
                const T inv2dx = T(1) / (T(2) * dx);
                T c;
                switch (a.crit) {
                case NH_CRIT_ETA_D: c = tabs((sh[l] - sdn1[l]) / sdn1[l]); break;
                case NH_CRIT_ETA_X: c = tabs(((sh[l + 1] - sdn1[l + 1]) - (sh[l - 1] - sdn1[l - 1])) * inv2dx); break;
                case NH_CRIT_U:     c = tabs(shu[l] / sh[l]); break;
                case NH_CRIT_U_X:   c = tabs((shu[l + 1] / sh[l + 1] - shu[l - 1] / sh[l - 1]) * inv2dx); break;
                case NH_CRIT_W:     c = tabs(shw[l] / sh[l]); break;
                default:            c = tabs((shw[l + 1] / sh[l + 1] - shw[l - 1] / sh[l - 1]) * inv2dx); break;
                }
                mark = (double)c > a.knh;
            }
        }
        const uint32_t word = __ballot_sync(0xffffffffu, mark);
        if ((tid & 31) == 0) a.marks[(size_t)b * G.wpitch + (j >> 5)] = word;
        double v[1] = {mass};
        block_sum<1>(v, red);
        if (tid == 0) a.mass_part[(size_t)b * G.ntiles + blockIdx.x] = v[0];
    }
}

// ------------------------------------------------------------- compaction

struct CompactArgs {
    int nx, pitch, wpitch, bc, enlarge;
    const uint32_t* marks;
    uint32_t* act;       // dilated mask words
    int* list;           // active cells, per member region
    int* nact;           // active count per member
    MState* ms;
    Ctl* ctl;
};

// One CTA per member: marks are staged in shared memory, enlarged by
// `enlarge` cells with word shifts (wrapped explicitly at periodic ends),
// then compacted in cell order: popcount per word, block-wide exclusive scan,
// each thread writes the positions of its set bits.
__global__ void __launch_bounds__(kCompactThreads) k_compact(CompactArgs a)
{
    extern __shared__ uint32_t s_m[];
    __shared__ int s_wsum[32];
    __shared__ int s_base;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int nwarp = blockDim.x >> 5;
    const int nw = (a.nx + 31) >> 5;
    const uint32_t* M = a.marks + (size_t)b * a.wpitch;
    for (int w = tid; w < nw; w += blockDim.x) s_m[w] = M[w];
    if (tid == 0) s_base = 0;
    if (b == 0 && tid == 0) { a.ctl->not_done = 0; a.ctl->n_cg = 0; a.ctl->n_bicg = 0; }
    __syncthreads();
    const int e = a.enlarge;
    int* L = a.list + (size_t)b * a.pitch;
    for (int w0 = 0; w0 < nw; w0 += blockDim.x) {
        const int w = w0 + tid;
        uint32_t word = 0u;
        if (w < nw) {
            const uint32_t m = s_m[w];
            const uint32_t lo = (w > 0) ? s_m[w - 1] : 0u;
            const uint32_t hi = (w + 1 < nw) ? s_m[w + 1] : 0u;
            uint32_t acc = m;
            for (int s = 1; s <= e; ++s)
                acc |= (m << s) | (lo >> (32 - s)) | (m >> s) | (hi << (32 - s));
            const int nvalid = a.nx - 32 * w;
            if (nvalid < 32) acc &= (1u << nvalid) - 1u;
            if (a.bc == NH_BC_PERIODIC && e > 0) {
                const int c0 = 32 * w, c1 = min(32 * w + 32, a.nx);
                for (int i = c0; i < c1; ++i) {
                    if (i >= e && i < a.nx - e) continue;
                    for (int k = -e; k <= e; ++k) {
                        int c = (i + k) % a.nx;
                        if (c < 0) c += a.nx;
                        if ((s_m[c >> 5] >> (c & 31)) & 1u) { acc |= 1u << (i - c0); break; }
                    }
                }
            }
            word = acc;
            a.act[(size_t)b * a.wpitch + w] = word;
        }
        const int cnt = __popc(word);
        int incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_wsum[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int v = (lane < nwarp) ? s_wsum[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, v, o);
                if (lane >= o) v += y;
            }
            s_wsum[lane] = v;
        }
        __syncthreads();
        int off = s_base + incl - cnt + (wid > 0 ? s_wsum[wid - 1] : 0);
        uint32_t wd = word;
        while (wd) {
            const int bit = __ffs(wd) - 1;
            L[off++] = 32 * w + bit;
            wd &= wd - 1u;
        }
        __syncthreads();
        if (tid == 0) s_base += s_wsum[nwarp - 1];
        __syncthreads();
    }
    if (tid == 0) {
        const int n = s_base;
        a.nact[b] = n;
        MState s;
        s.bnorm2 = 0.0; s.bnorm = 0.0; s.rr = 0.0; s.alpha = 1.0; s.beta = 0.0; s.omega = 1.0;
        s.rel_res = 0.0; s.min_gamma = 0.0; s.snorm = 0.0;
        s.status = NH_OK; s.iters = 0; s.done = (n == 0); s.kind = -1; s.zero_sol = 0;
        s.s_conv = 0; s.n_active = n; s.nchunks = (n + kChunk - 1) / kChunk;
        a.ms[b] = s;
    }
}

// -------------------------------------------------- per-member reductions

// After each CTA of a member wrote its partials, the last one to arrive
// (ticket = nchunks - 1) returns true; it then sums the member's partials in a
// fixed order, so the result does not depend on CTA scheduling.
__device__ __forceinline__ bool arrive_last(int* cnt, int b, int total)
{
    __shared__ int s_last;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        const int t = atomicAdd(&cnt[b], 1);
        s_last = (t == total - 1);
        if (s_last) cnt[b] = 0;
    }
    __syncthreads();
    if (s_last) __threadfence();
    return s_last != 0;
}

// Deterministic block-wide sum of part[0..n) (thread 0 gets it).
__device__ __forceinline__ double member_sum(const double* part, int n, double* sh)
{
    double v[1] = {0.0};
    for (int q = threadIdx.x; q < n; q += blockDim.x) v[0] += __ldcg(part + q);
    block_sum<1>(v, sh);
    return v[0];
}
__device__ __forceinline__ double member_min(const double* part, int n, double* sh)
{
    double v = INFINITY;
    for (int q = threadIdx.x; q < n; q += blockDim.x) v = fmin(v, __ldcg(part + q));
    return block_min(v, sh);
}

// --------------------------------------------------------------- assembly

template <typename T>
struct AsmArgs {
    Geo G;
    const T* ht; const T* hut; const T* hwt;
    const T* d0;
    const Slide* slide; const Kin* kin;
    const int* list; const uint32_t* act;
    MState* ms;
    T* diag; T* offl; T* offr; T* R;
    int* nbl; int* nbr;
    T* c6; T* cx; T* phi; T* ddx;            // correction coefficients
    double* part;                            // [2][nb * maxch]
    int* cnt;
    double dt;
    int solver;                              // NH_SOLVER_*
};

template <typename T>
struct CellQ {
    T h, K, beta, U0, V, phi, d_x, D, d_t;
};

// Per-cell quantities of the elliptic equation at an in-domain cell c.
template <typename T>
__device__ __forceinline__ CellQ<T> cell_q(const AsmArgs<T>& a, const T* __restrict__ ht,
                                           const T* __restrict__ hut, const T* __restrict__ D0,
                                           int c, const Slide& sl, const Kin& kn)
{
    const Geo& G = a.G;
    const Bottom<T> B = bottom_full(D0, c, G.nx, G.bc, G.x0, G.dx, sl, kn);
    int sg;
    const int cm = resolve(c - 1, G.nx, G.bc, &sg), cp = resolve(c + 1, G.nx, G.bc, &sg);
    const T etam = ht[cm] - depth_at(D0, cm, G.x0, G.dx, sl, kn.s_n1);
    const T etap = ht[cp] - depth_at(D0, cp, G.x0, G.dx, sl, kn.s_n1);
    const T eta_x = (etap - etam) / (T(2) * T(G.dx));
    CellQ<T> q;
    q.h = ht[c];
    const T u = hut[c] / q.h;
    q.d_x = B.d_x;
    q.d_t = B.d_t;
    q.D = T(4) + B.d_x * B.d_x;
    q.phi = T(a.dt) * q.h / q.D * (T(G.g) * B.d_x * eta_x - B.d_tt - T(2) * u * B.d_xt - u * u * B.d_xx);
    q.K = T(4) / (q.h * q.D);
    q.beta = T(6) * B.d_x / (q.h * q.h * q.D);
    q.U0 = hut[c] + q.phi * B.d_x;
    q.V = q.U0 / q.h;
    return q;
}

__device__ __forceinline__ bool bit_at(const uint32_t* w, int i)
{
    return (w[i >> 5] >> (i & 31)) & 1u;
}

template <typename T>
__global__ void __launch_bounds__(kChunk) k_assemble(AsmArgs<T> a)
{
    __shared__ double red[64];
    const Geo& G = a.G;
    const int tid = threadIdx.x;
    for (int wi = blockIdx.x; wi < G.nb * G.maxch; wi += gridDim.x) {
        const int b = wi / G.maxch, j = wi - b * G.maxch;
        const int n = a.ms[b].n_active;
        const int nch = (n + kChunk - 1) / kChunk;
        if (j >= nch) continue;
        const size_t mo = (size_t)b * G.pitch;
        const T* ht = a.ht + mo; const T* hut = a.hut + mo; const T* hwt = a.hwt + mo;
        const T* D0 = a.d0 + mo;
        const uint32_t* act = a.act + (size_t)b * G.wpitch;
        const Slide sl = a.slide[b];
        const Kin kn = a.kin[b];
        const int k = j * kChunk + tid;
        double r2 = 0.0, gmin = INFINITY;
        if (k < n) {
            const int i = a.list[mo + k];
            int sgm, sgp;
            const int cm = resolve(i - 1, G.nx, G.bc, &sgm), cp = resolve(i + 1, G.nx, G.bc, &sgp);
            const CellQ<T> qi = cell_q(a, ht, hut, D0, i, sl, kn);
            const CellQ<T> qm = cell_q(a, ht, hut, D0, cm, sl, kn);
            const CellQ<T> qp = cell_q(a, ht, hut, D0, cp, sl, kn);
            const T dxT = T(G.dx), idx2 = T(1) / (dxT * dxT);
            const T Kl = T(0.5) * (qm.K + qi.K), Kr = T(0.5) * (qi.K + qp.K);
            const T bm = sgm > 0 ? qm.beta : -qm.beta, bp = sgp > 0 ? qp.beta : -qp.beta;
            const T Vm = sgm > 0 ? qm.V : -qm.V, Vp = sgp > 0 ? qp.V : -qp.V;
            const T h = qi.h, h2 = h * h;
            const T gam = (bp - bm) / (T(2) * dxT) + T(12) * (T(1) + qi.d_x * qi.d_x) / (h2 * h * qi.D);
            const T Rk = -((Vp - Vm) / (T(2) * dxT) + T(2) * qi.d_x * qi.U0 / h2 + T(2) * hwt[i] / h2
                           + T(2) * qi.phi / h2 + T(2) * qi.d_t / h);
            // neighbours inside the active set (zero Dirichlet data outside)
            bool hasl, hasr;
            int kl = -1, kr = -1;
            if (G.bc == NH_BC_PERIODIC) {
                hasl = bit_at(act, cm);
                hasr = bit_at(act, cp);
                if (hasl) kl = (i == 0) ? n - 1 : k - 1;
                if (hasr) kr = (i == G.nx - 1) ? 0 : k + 1;
            } else {
                hasl = (i > 0) && bit_at(act, i - 1);
                hasr = (i < G.nx - 1) && bit_at(act, i + 1);
                if (hasl) kl = k - 1;
                if (hasr) kr = k + 1;
            }
            a.diag[mo + k] = (Kl + Kr) * idx2 + gam;
            a.offl[mo + k] = hasl ? -Kl * idx2 : T(0);
            a.offr[mo + k] = hasr ? -Kr * idx2 : T(0);
            a.R[mo + k] = Rk;
            a.nbl[mo + k] = kl;
            a.nbr[mo + k] = kr;
            a.c6[mo + k] = T(6) / (h * qi.D);
            a.cx[mo + k] = qi.d_x / qi.D;
            a.phi[mo + k] = qi.phi;
            a.ddx[mo + k] = qi.d_x;
            r2 = (double)Rk * (double)Rk;
            gmin = (double)gam;
        }
        double v[1] = {r2};
        block_sum<1>(v, red);
        const double gm = block_min(gmin, red);
        double* P0 = a.part;
        double* P1 = a.part + (size_t)G.nb * G.maxch;
        if (tid == 0) { P0[wi] = v[0]; P1[wi] = gm; }
        if (arrive_last(a.cnt, b, nch)) {
            const double bn2 = member_sum(P0 + (size_t)b * G.maxch, nch, red);
            const double gmn = member_min(P1 + (size_t)b * G.maxch, nch, red);
            if (tid == 0) {
                MState& s = a.ms[b];
                s.bnorm2 = bn2;
                s.bnorm = sqrt(bn2);
                s.min_gamma = gmn;
                int kind = a.solver;
                if (kind == NH_SOLVER_AUTO) kind = (gmn > 0.0) ? NH_SOLVER_CG : NH_SOLVER_BICGSTAB;
                s.kind = kind;
            }
        }
    }
}

// ------------------------------------------------------------ Krylov solve

template <typename T>
struct SolveArgs {
    int nb, pitch, maxch;
    const int* list;
    const T* diag; const T* offl; const T* offr;
    const int* nbl; const int* nbr;
    const T* R;
    const double* psi_prev;    // dense, previous step's pressure unknown
    double guess_scale;        // dt_new / dt_old, or 0 for a zero guess
    T* x; T* r; T* p0; T* p1; T* q; T* rh; T* v0; T* v1; T* s; T* t;
    MState* ms; Ctl* ctl;
    double* part;              // [3][nb * maxch]
    int* cnt;
    double rtol;
    int max_iter;
    int it;
};

template <typename T>
__device__ __forceinline__ T apply_row(const SolveArgs<T>& a, size_t mo, int k, T xk, T xl, T xr)
{
    T y = a.diag[mo + k] * xk;
    y += a.offl[mo + k] * xl;
    y += a.offr[mo + k] * xr;
    return y;
}

// Shared prologue of the solve kernels: loop over (member, chunk) work items.
#define NH_FOR_ITEMS(A)                                                         \
    for (int wi = blockIdx.x; wi < (A).nb * (A).maxch; wi += gridDim.x) {        \
        const int b = wi / (A).maxch, j = wi - b * (A).maxch;                   \
        const int nch = (A).ms[b].nchunks;                                      \
        if (j >= nch) continue;                                                 \
        const int n = (A).ms[b].n_active;                                       \
        const size_t mo = (size_t)b * (A).pitch;                                \
        const int k = j * kChunk + threadIdx.x;                                 \
        const bool in = k < n;

#define NH_END_ITEMS }

// r = R - A x0, x0 = previous pressure (scaled) on active cells.
template <typename T>
__global__ void __launch_bounds__(kChunk) k_solve_init(SolveArgs<T> a)
{
    __shared__ double red[64];
    NH_FOR_ITEMS(a)
        double rr = 0.0;
        if (in) {
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            const double sc = a.guess_scale;
            T x0 = T(0), xl = T(0), xr = T(0);
            if (sc != 0.0) {
                x0 = T(a.psi_prev[mo + a.list[mo + k]] * sc);
                if (kl >= 0) xl = T(a.psi_prev[mo + a.list[mo + kl]] * sc);
                if (kr >= 0) xr = T(a.psi_prev[mo + a.list[mo + kr]] * sc);
            }
            const T rk = a.R[mo + k] - apply_row(a, mo, k, x0, xl, xr);
            a.x[mo + k] = x0;
            a.r[mo + k] = rk;
            a.p0[mo + k] = T(0);
            a.p1[mo + k] = T(0);
            a.rh[mo + k] = rk;
            a.v0[mo + k] = T(0);
            a.v1[mo + k] = T(0);
            rr = (double)rk * (double)rk;
        }
        double v[1] = {rr};
        block_sum<1>(v, red);
        double* P0 = a.part;
        if (threadIdx.x == 0) P0[wi] = v[0];
        if (arrive_last(a.cnt, b, nch)) {
            const double s_rr = member_sum(P0 + (size_t)b * a.maxch, nch, red);
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                s.rr = s_rr;
                if (s.bnorm2 == 0.0) {
                    s.zero_sol = 1; s.done = 1; s.iters = 0; s.rel_res = 0.0;
                } else if (!isfinite(s_rr) || !isfinite(s.bnorm2)) {
                    s.done = 1; s.status = NH_ERR_NONFINITE; s.rel_res = NAN;
                } else if (sqrt(s_rr) <= a.rtol * s.bnorm) {
                    s.done = 1; s.iters = 0; s.rel_res = sqrt(s_rr) / s.bnorm;
                } else {
                    // BiCGStab's first direction: beta = (rho / 1) (1 / 1)
                    s.alpha = 1.0; s.omega = 1.0; s.beta = s_rr;
                    atomicAdd(&a.ctl->not_done, 1);
                    if (s.kind == NH_SOLVER_CG) atomicAdd(&a.ctl->n_cg, 1);
                    else atomicAdd(&a.ctl->n_bicg, 1);
                }
            }
        }
    NH_END_ITEMS
}

template <typename T>
__device__ __forceinline__ void finish_member(MState& s, Ctl* ctl, int status, int iters, double rel)
{
    s.status = status;
    s.iters = iters;
    s.rel_res = rel;
    s.done = 1;
    atomicSub(&ctl->not_done, 1);
}

// CG, first half of iteration it: p = r + beta p_old (neighbours on the fly),
// q = A p, partial <p, q>; last CTA of the member: alpha = rr / <p, q>.
template <typename T>
__global__ void __launch_bounds__(kChunk) k_cg_a(SolveArgs<T> a)
{
    __shared__ double red[64];
    const int it = a.it;
    const T* pold = (it & 1) ? a.p0 : a.p1;
    T* pnew = (it & 1) ? a.p1 : a.p0;
    NH_FOR_ITEMS(a)
        if (a.ms[b].done || a.ms[b].kind != NH_SOLVER_CG) continue;
        const T beta = (it == 1) ? T(0) : T(a.ms[b].beta);
        double pq = 0.0;
        if (in) {
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            const T pk = a.r[mo + k] + beta * pold[mo + k];
            const T pl = kl >= 0 ? a.r[mo + kl] + beta * pold[mo + kl] : T(0);
            const T pr = kr >= 0 ? a.r[mo + kr] + beta * pold[mo + kr] : T(0);
            const T qk = apply_row(a, mo, k, pk, pl, pr);
            pnew[mo + k] = pk;
            a.q[mo + k] = qk;
            pq = (double)pk * (double)qk;
        }
        double v[1] = {pq};
        block_sum<1>(v, red);
        if (threadIdx.x == 0) a.part[wi] = v[0];
        if (arrive_last(a.cnt, b, nch)) {
            const double s_pq = member_sum(a.part + (size_t)b * a.maxch, nch, red);
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                if (!isfinite(s_pq) || s_pq == 0.0) finish_member<T>(s, a.ctl, NH_ERR_NONFINITE, it, NAN);
                else s.alpha = s.rr / s_pq;
            }
        }
    NH_END_ITEMS
}

// CG, second half: x += alpha p, r -= alpha q, partial <r, r>; last CTA:
// convergence test, beta = rr_new / rr.
template <typename T>
__global__ void __launch_bounds__(kChunk) k_cg_b(SolveArgs<T> a)
{
    __shared__ double red[64];
    const int it = a.it;
    const T* p = (it & 1) ? a.p1 : a.p0;
    NH_FOR_ITEMS(a)
        if (a.ms[b].done || a.ms[b].kind != NH_SOLVER_CG) continue;
        const T alpha = T(a.ms[b].alpha);
        double rr = 0.0;
        if (in) {
            const T xk = a.x[mo + k] + alpha * p[mo + k];
            const T rk = a.r[mo + k] - alpha * a.q[mo + k];
            a.x[mo + k] = xk;
            a.r[mo + k] = rk;
            rr = (double)rk * (double)rk;
        }
        double v[1] = {rr};
        block_sum<1>(v, red);
        if (threadIdx.x == 0) a.part[wi] = v[0];
        if (arrive_last(a.cnt, b, nch)) {
            const double s_rr = member_sum(a.part + (size_t)b * a.maxch, nch, red);
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                const double rel = sqrt(s_rr) / s.bnorm;
                if (!isfinite(s_rr)) finish_member<T>(s, a.ctl, NH_ERR_NONFINITE, it, NAN);
                else if (sqrt(s_rr) <= a.rtol * s.bnorm) finish_member<T>(s, a.ctl, NH_OK, it, rel);
                else if (it >= a.max_iter) finish_member<T>(s, a.ctl, NH_ERR_NOT_CONVERGED, it, rel);
                else { s.beta = s_rr / s.rr; s.rr = s_rr; }
            }
        }
    NH_END_ITEMS
}

// BiCGStab step 1: p = r + beta (p_old - omega v_old), v = A p, partial <rh, v>;
// last CTA: alpha = rho / <rh, v>.
template <typename T>
__global__ void __launch_bounds__(kChunk) k_bi_1(SolveArgs<T> a)
{
    __shared__ double red[64];
    const int it = a.it;
    const T* pold = (it & 1) ? a.p0 : a.p1;
    T* pnew = (it & 1) ? a.p1 : a.p0;
    const T* vold = (it & 1) ? a.v0 : a.v1;
    T* vnew = (it & 1) ? a.v1 : a.v0;
    NH_FOR_ITEMS(a)
        if (a.ms[b].done || a.ms[b].kind != NH_SOLVER_BICGSTAB) continue;
        const T beta = T(a.ms[b].beta), omega = T(a.ms[b].omega);
        double rv = 0.0;
        if (in) {
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            const T pk = a.r[mo + k] + beta * (pold[mo + k] - omega * vold[mo + k]);
            const T pl = kl >= 0 ? a.r[mo + kl] + beta * (pold[mo + kl] - omega * vold[mo + kl]) : T(0);
            const T pr = kr >= 0 ? a.r[mo + kr] + beta * (pold[mo + kr] - omega * vold[mo + kr]) : T(0);
            const T vk = apply_row(a, mo, k, pk, pl, pr);
            pnew[mo + k] = pk;
            vnew[mo + k] = vk;
            rv = (double)a.rh[mo + k] * (double)vk;
        }
        double v[1] = {rv};
        block_sum<1>(v, red);
        if (threadIdx.x == 0) a.part[wi] = v[0];
        if (arrive_last(a.cnt, b, nch)) {
            const double s_rv = member_sum(a.part + (size_t)b * a.maxch, nch, red);
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                if (!isfinite(s_rv) || s_rv == 0.0) finish_member<T>(s, a.ctl, NH_ERR_NONFINITE, it, NAN);
                else s.alpha = s.rr / s_rv;
            }
        }
    NH_END_ITEMS
}

// BiCGStab step 2: s = r - alpha v (neighbours on the fly), t = A s;
// partials <t,s>, <t,t>, <s,s>; last CTA: ||s|| test, omega = <t,s>/<t,t>.
template <typename T>
__global__ void __launch_bounds__(kChunk) k_bi_2(SolveArgs<T> a)
{
    __shared__ double red[96];
    const int it = a.it;
    const T* v = (it & 1) ? a.v1 : a.v0;
    const size_t stride = (size_t)a.nb * a.maxch;
    NH_FOR_ITEMS(a)
        if (a.ms[b].done || a.ms[b].kind != NH_SOLVER_BICGSTAB) continue;
        const T alpha = T(a.ms[b].alpha);
        double acc[3] = {0.0, 0.0, 0.0};
        if (in) {
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            const T sk = a.r[mo + k] - alpha * v[mo + k];
            const T sl = kl >= 0 ? a.r[mo + kl] - alpha * v[mo + kl] : T(0);
            const T sr = kr >= 0 ? a.r[mo + kr] - alpha * v[mo + kr] : T(0);
            const T tk = apply_row(a, mo, k, sk, sl, sr);
            a.s[mo + k] = sk;
            a.t[mo + k] = tk;
            acc[0] = (double)tk * (double)sk;
            acc[1] = (double)tk * (double)tk;
            acc[2] = (double)sk * (double)sk;
        }
        block_sum<3>(acc, red);
        if (threadIdx.x == 0) {
            a.part[wi] = acc[0];
            a.part[stride + wi] = acc[1];
            a.part[2 * stride + wi] = acc[2];
        }
        if (arrive_last(a.cnt, b, nch)) {
            const size_t mb = (size_t)b * a.maxch;
            const double ts = member_sum(a.part + mb, nch, red);
            const double tt = member_sum(a.part + stride + mb, nch, red);
            const double ss = member_sum(a.part + 2 * stride + mb, nch, red);
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                s.snorm = sqrt(ss);
                if (!isfinite(ss)) {
                    finish_member<T>(s, a.ctl, NH_ERR_NONFINITE, it, NAN);
                } else if (s.snorm <= a.rtol * s.bnorm) {
                    s.s_conv = 1;
                } else if (!isfinite(tt) || tt == 0.0) {
                    finish_member<T>(s, a.ctl, NH_ERR_NONFINITE, it, NAN);
                } else {
                    s.omega = ts / tt;
                }
            }
        }
    NH_END_ITEMS
}

// BiCGStab step 3: x += alpha p + omega s, r = s - omega t; partials
// <r,r>, <rh,r>; last CTA: ||r|| test, beta = (rho_new / rho)(alpha / omega).
template <typename T>
__global__ void __launch_bounds__(kChunk) k_bi_3(SolveArgs<T> a)
{
    __shared__ double red[64];
    const int it = a.it;
    const T* p = (it & 1) ? a.p1 : a.p0;
    const size_t stride = (size_t)a.nb * a.maxch;
    NH_FOR_ITEMS(a)
        if (a.ms[b].done || a.ms[b].kind != NH_SOLVER_BICGSTAB) continue;
        const T alpha = T(a.ms[b].alpha), omega = T(a.ms[b].omega);
        const bool sconv = a.ms[b].s_conv != 0;
        double acc[2] = {0.0, 0.0};
        if (in) {
            if (sconv) {
                a.x[mo + k] = a.x[mo + k] + alpha * p[mo + k];
            } else {
                const T sk = a.s[mo + k];
                a.x[mo + k] = a.x[mo + k] + alpha * p[mo + k] + omega * sk;
                const T rk = sk - omega * a.t[mo + k];
                a.r[mo + k] = rk;
                acc[0] = (double)rk * (double)rk;
                acc[1] = (double)a.rh[mo + k] * (double)rk;
            }
        }
        block_sum<2>(acc, red);
        if (threadIdx.x == 0) { a.part[wi] = acc[0]; a.part[stride + wi] = acc[1]; }
        if (arrive_last(a.cnt, b, nch)) {
            const size_t mb = (size_t)b * a.maxch;
            const double rr = member_sum(a.part + mb, nch, red);
            const double rhr = member_sum(a.part + stride + mb, nch, red);
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                if (sconv) {
                    finish_member<T>(s, a.ctl, NH_OK, it, s.snorm / s.bnorm);
                } else {
                    const double rn = sqrt(rr);
                    if (!isfinite(rr)) finish_member<T>(s, a.ctl, NH_ERR_NONFINITE, it, NAN);
                    else if (rn <= a.rtol * s.bnorm) finish_member<T>(s, a.ctl, NH_OK, it, rn / s.bnorm);
                    else if (it >= a.max_iter) finish_member<T>(s, a.ctl, NH_ERR_NOT_CONVERGED, it, rn / s.bnorm);
                    else { s.beta = (rhr / s.rr) * (s.alpha / s.omega); s.rr = rhr; }
                }
            }
        }
    NH_END_ITEMS
}

// ------------------------------------------------------------- correction

struct ClearArgs {
    int nb, pitch, maxlist;
    const int* list_prev;
    const int* nact_prev;
    double* psi;
};

// Zero the dense pressure unknown on the previous step's active cells.
__global__ void k_clear_prev(ClearArgs a)
{
    const size_t total = (size_t)a.nb * a.pitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(q / a.pitch), k = (int)(q - (size_t)b * a.pitch);
        if (k < a.nact_prev[b]) a.psi[(size_t)b * a.pitch + a.list_prev[q]] = 0.0;
    }
}

template <typename T>
struct CorrArgs {
    int nb, pitch, maxch;
    double dx;
    const int* list; const int* nbl; const int* nbr;
    const T* x;
    const T* c6; const T* cx; const T* phi; const T* ddx;
    const MState* ms;
    T* hu; T* hw;          // Q~ buffers, corrected in place into Q^{n+1}
    double* psi;           // dense pressure unknown (for the next warm start)
};

// Eqs. 10-11 on the active cells (h is not corrected, Sec. 3.2).
template <typename T>
__global__ void __launch_bounds__(kChunk) k_correct(CorrArgs<T> a)
{
    for (int wi = blockIdx.x; wi < a.nb * a.maxch; wi += gridDim.x) {
        const int b = wi / a.maxch, j = wi - b * a.maxch;
        const MState& s = a.ms[b];
        if (j >= s.nchunks) continue;
        const int n = s.n_active;
        const size_t mo = (size_t)b * a.pitch;
        const int k = j * kChunk + threadIdx.x;
        if (k >= n) continue;
        const bool zero = s.zero_sol != 0;
        const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
        const T ps = zero ? T(0) : a.x[mo + k];
        const T pl = (zero || kl < 0) ? T(0) : a.x[mo + kl];
        const T pr = (zero || kr < 0) ? T(0) : a.x[mo + kr];
        const T ps_x = (pr - pl) / (T(2) * T(a.dx));
        const T P = a.c6[mo + k] * ps + a.cx[mo + k] * ps_x + a.phi[mo + k];
        const int i = a.list[mo + k];
        a.hu[mo + i] = a.hu[mo + i] - ps_x + a.ddx[mo + k] * P;
        a.hw[mo + i] = a.hw[mo + i] + P;
        a.psi[mo + i] = (double)ps;
    }
}

// ------------------------------------------------------------- summaries

struct Summary {
    long long n_active;
    int n_active_max;
    int iters;
    int any_bicg, any_cg;
    int status;
    int pad;
    double rel_res;
    double min_gamma;
    double mass;
};

__global__ void k_summary(const MState* ms, int nb, const double* mass_part, int nparts, double dx,
                          Summary* out)
{
    __shared__ double red[64];
    double m[1] = {0.0};
    for (int q = threadIdx.x; q < nparts; q += blockDim.x) m[0] += mass_part[q];
    block_sum<1>(m, red);
    if (threadIdx.x == 0) {
        Summary S;
        S.n_active = 0; S.n_active_max = 0; S.iters = 0; S.any_bicg = 0; S.any_cg = 0;
        S.status = NH_OK; S.pad = 0; S.rel_res = 0.0; S.min_gamma = INFINITY; S.mass = m[0] * dx;
        for (int b = 0; b < nb; ++b) {
            const MState& s = ms[b];
            S.n_active += s.n_active;
            S.n_active_max = max(S.n_active_max, s.n_active);
            S.iters = max(S.iters, s.iters);
            if (s.n_active > 0) {
                if (s.kind == NH_SOLVER_BICGSTAB) S.any_bicg = 1;
                if (s.kind == NH_SOLVER_CG) S.any_cg = 1;
                S.min_gamma = fmin(S.min_gamma, s.min_gamma);
                if (!(s.rel_res <= S.rel_res)) S.rel_res = s.rel_res;   // keeps NaN
                if (!s.done && S.status == NH_OK) S.status = NH_ERR_NOT_CONVERGED;
            }
            if (s.status != NH_OK && (S.status == NH_OK || s.status == NH_ERR_NONFINITE)) S.status = s.status;
        }
        if (S.n_active == 0) S.min_gamma = 0.0;
        *out = S;
    }
}

}  // namespace nh
