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
    double idx;          // 1 / dx
    double i2dx, idx2;   // 1 / (2 dx), 1 / dx^2
    const int* nxv;      // per-member cell counts (uneven ensembles), or null: all nx
};

__device__ __forceinline__ int member_nx(const Geo& G, int b) { return G.nxv ? G.nxv[b] : G.nx; }

// ------------------------------------------------------------------ slide

static __global__ void k_kinematics(const Slide* __restrict__ sl, Kin* __restrict__ kin, int nb,
                             double t_n, double t_n1)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    const Slide s = sl[b];
    Kin k{0.0, 0.0, 0.0, 0.0};
    double sd_n, sdd_n;
    slide_law(s, t_n, &k.s_n, &sd_n, &sdd_n);
    slide_law(s, t_n1, &k.s_n1, &k.sd_n1, &k.sdd_n1);
    kin[b] = k;
}

// Same from the device time control block (captured runs).
static __global__ void k_kinematics_dev(const Slide* __restrict__ sl, Kin* __restrict__ kin, int nb,
                                        const TimeCtl* __restrict__ tc)
{
    int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb || tc->abort) return;
    const double t_n = tc->t_base + (double)tc->n * tc->dt;
    const double t_n1 = tc->t_base + (double)(tc->n + 1) * tc->dt;
    const Slide s = sl[b];
    Kin k{0.0, 0.0, 0.0, 0.0};
    double sd_n, sdd_n;
    slide_law(s, t_n, &k.s_n, &sd_n, &sdd_n);
    slide_law(s, t_n1, &k.s_n1, &k.sd_n1, &k.sdd_n1);
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

// Local Lax-Friedrichs (Rusanov) flux of (hu, hu^2 + g h^2 / 2, huw) at a face
// with continuous depth d_f, from left / right states (eta, u, w).  The
// momentum flux is returned split as F1 = A1 + (g/4)(hL^2 + hR^2), with the
// convective / dissipative part A1 and the jump part
// G1 = (g/4)(hR + hL)(etaR - etaL) = (g/4)(hR^2 - hL^2); with the cell's own
// face thicknesses h- (right) and h+ (left) the cell update
//   -(F1_r - F1_l)/dx + g hbar (d_r - d_l)/dx
// equals -(A1_r - A1_l + G1_r + G1_l + g hbar (h- - h+ - d_r + d_l))/dx, and
// h- - h+ - d_r + d_l is the eta slope: the lake at rest is exact in any
// precision.
template <typename T>
__device__ __forceinline__ void rusanov(T g, T df, T eL, T uL, T wL, T eR, T uR, T wR,
                                        T& F0, T& A1, T& G1, T& F2)
{
    const T hL = eL + df, hR = eR + df;
    const T qL = hL * uL, qR = hR * uR;
    const T aL = tabs(uL) + wave_sqrt(g * hL), aR = tabs(uR) + wave_sqrt(g * hR);
    const T s = aL > aR ? aL : aR;
    const T de = eR - eL;
    F0 = T(0.5) * (qL + qR) - T(0.5) * s * de;
    A1 = T(0.5) * (qL * uL + qR * uR) - T(0.5) * s * (qR - qL);
    G1 = T(0.25) * g * (hR + hL) * de;
    F2 = T(0.5) * (qL * wL + qR * wR) - T(0.5) * s * (hR * wR - hL * wL);
}

template <typename T>
struct PredArgs {
    Geo G;
    const T* z; const T* hu; const T* hw;     // Q^n (zeta = h - d0)
    T* zt; T* hut; T* hwt;                    // Q~^{n+1}
    const T* d0;
    const Slide* slide; const Kin* kin;
    uint32_t* marks;                          // nb * wpitch words
    double* mass_part;                        // nb * ntiles: sum of zeta~
    double dt;
    double knh;
    int crit;
    int all_global;                           // mark every cell this step
    const TimeCtl* tc;                        // captured runs: stand down after an abort
};

// One CTA = one tile of kPredTile cells of one member.  Q^n is loaded with a
// halo of 5 cells (ghosts mirrored at walls, wrapped when periodic); stage 1
// (bottom at t^n) is evaluated on the tile plus 3 cells each side, stage 2
// (bottom at t^{n+1}) on the tile plus one cell each side, so the criterion's
// central differences need no second pass.  Q~ = Q^n + dt/2 (k1 + k2).
// Shared memory of one predictor tile (19 arrays of TILE + 2 halo cells).
template <typename T, int TILE>
constexpr size_t predict_smem_bytes() { return sizeof(T) * 20 * (TILE + 2 * kPredHalo); }

template <typename T, int TILE>
__global__ void __launch_bounds__(TILE) k_predict(PredArgs<T> a)
{
    constexpr int H = kPredHalo, NL = TILE + 2 * H;
    extern __shared__ __align__(16) unsigned char psm[];
    T* const sm = reinterpret_cast<T*>(psm);
    T* const sz = sm;               // Q^n, later Q~
    T* const shu = sm + NL;
    T* const shw = sm + 2 * NL;
    T* const sd0 = sm + 3 * NL;     // static depth, mound at t^n, t^{n+1}
    T* const smn = sm + 4 * NL;
    T* const smn1 = sm + 5 * NL;
    T* const se = sm + 6 * NL;      // stage primitives eta, u, w
    T* const su = sm + 7 * NL;
    T* const sw = sm + 8 * NL;
    T* const sle = sm + 9 * NL;     // limited slopes
    T* const slu = sm + 10 * NL;
    T* const slw = sm + 11 * NL;
    T* const F0 = sm + 12 * NL;     // face l: between local cells l-1 and l
    T* const A1 = sm + 13 * NL;
    T* const G1 = sm + 14 * NL;
    T* const F2 = sm + 15 * NL;
    T* const k1h = sm + 16 * NL;    // stage-1 rates
    T* const k1u = sm + 17 * NL;
    T* const k1w = sm + 18 * NL;
    T* const sdf = sm + 19 * NL;    // depth at face l of the current stage
    __shared__ double red_mass[TILE];

    const Geo& G = a.G;
    const int b = blockIdx.y, i0 = blockIdx.x * TILE, tid = threadIdx.x;
    if (a.tc && a.tc->abort) return;
    const size_t mo = (size_t)b * G.pitch;
    const T* __restrict__ Zn = a.z + mo;
    const T* __restrict__ HUn = a.hu + mo;
    const T* __restrict__ HWn = a.hw + mo;
    const T* __restrict__ D0 = a.d0 + mo;
    const Slide sl = a.slide[b];
    const Kin kn = a.kin[b];
    const int nxb = member_nx(G, b);
    if (i0 >= nxb) {   // tile beyond this member's cells (uneven ensemble)
        if (tid == 0) a.mass_part[(size_t)b * G.ntiles + blockIdx.x] = 0.0;
        return;
    }

    // A: load Q^n, d0 and the mound at both times.  Cells outside
    // [-6, nx+5] feed only outputs outside [-1, nx]; they get still water.
    // Cells whose mound term is nonzero at t^n or t^{n+1} lie in [s_mlo,
    // s_mhi] (the cut-off of mound_at with a margin, one cell either side);
    // elsewhere the per-cell evaluation is skipped (it would return 0).
    __shared__ int s_mlo, s_mhi;
    __shared__ T s_k[5];   // g, dt, dt/2, 1/dx, k_nh in T, converted once per CTA
    if (tid == 0) {
        s_k[0] = T(G.g); s_k[1] = T(a.dt); s_k[2] = T(0.5) * T(a.dt); s_k[3] = T(G.idx); s_k[4] = T(a.knh);
        int lo = 1, hi = 0;
        if (sl.shape == NH_SLIDE_GAUSS_LNCOSH || sl.shape == NH_SLIDE_PLATE_EXP || sl.shape == NH_SLIDE_QUARTIC) {
            // support of the mound at t^n and t^{n+1}, with a margin
            double lo_x, hi_x;
            if (sl.shape == NH_SLIDE_PLATE_EXP) {
                lo_x = sl.xc0 - 1.0001 * sl.L; hi_x = sl.xc0 + 1.0001 * sl.L;
            } else {
                const double r = sl.shape == NH_SLIDE_QUARTIC ? 0.5001 * sl.L : sqrt(kMoundCut * 1.0001) * sl.L;
                lo_x = sl.xc0 + fmin(kn.s_n, kn.s_n1) - r; hi_x = sl.xc0 + fmax(kn.s_n, kn.s_n1) + r;
            }
            const double ca = (lo_x - G.x0) / G.dx - 0.5;
            const double cb = (hi_x - G.x0) / G.dx - 0.5;
            lo = (int)fmax(floor(ca) - 1.0, -1073741824.0);
            hi = (int)fmin(ceil(cb) + 1.0, 1073741824.0);
        }
        s_mlo = lo; s_mhi = hi;
    }
    __syncthreads();
    const T g = s_k[0], dt = s_k[1], half_dt = s_k[2], idx = s_k[3];
    for (int l = tid; l < NL; l += TILE) {
        const int j = i0 - H + l;
        T zv = T(0), huv = T(0), hwv = T(0), d0v = T(1), mn = T(0), mn1 = T(0);
        if (j >= -6 && j <= nxb + 5) {
            int sg;
            const int c = resolve(j, nxb, G.bc, &sg);
            zv = Zn[c];
            huv = sg > 0 ? HUn[c] : -HUn[c];
            hwv = HWn[c];
            d0v = D0[c];
            if (c >= s_mlo && c <= s_mhi) {
                mn = mound_at<T>(c, G.x0, G.dx, sl, kn.s_n);
                mn1 = mound_at<T>(c, G.x0, G.dx, sl, kn.s_n1);
            }
        }
        const T rh = T(1) / (zv + d0v);
        sz[l] = zv; shu[l] = huv; shw[l] = hwv; sd0[l] = d0v; smn[l] = mn; smn1[l] = mn1;
        se[l] = zv + mn; su[l] = huv * rh; sw[l] = hwv * rh;
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
        const T df = T(0.5) * ((sd0[f - 1] - smn[f - 1]) + (sd0[f] - smn[f]));
        sdf[f] = df;
        rusanov(g, df, se[f - 1] + T(0.5) * sle[f - 1], su[f - 1] + T(0.5) * slu[f - 1],
                sw[f - 1] + T(0.5) * slw[f - 1], se[f] - T(0.5) * sle[f], su[f] - T(0.5) * slu[f],
                sw[f] - T(0.5) * slw[f], F0[f], A1[f], G1[f], F2[f]);
    }
    __syncthreads();

    // D: stage-1 rates and Q* on cells [2, NL-2); Q* stored as primitives
    //    against the bottom at t^{n+1}
    for (int l = tid + 2; l < NL - 2; l += TILE) {
        // mean of the cell's two face thicknesses (eta -+ slope/2 + face depth)
        const T hbar = se[l] + T(0.5) * (sdf[l] + sdf[l + 1]);
        const T r0 = -(F0[l + 1] - F0[l]) * idx;
        const T r1 = -((A1[l + 1] - A1[l]) + (G1[l + 1] + G1[l]) + g * hbar * sle[l]) * idx;
        const T r2 = -(F2[l + 1] - F2[l]) * idx;
        k1h[l] = r0; k1u[l] = r1; k1w[l] = r2;
        const T zs = sz[l] + dt * r0, hus = shu[l] + dt * r1, hws = shw[l] + dt * r2;
        const T rhs = T(1) / (zs + sd0[l]);
        se[l] = zs + smn1[l]; su[l] = hus * rhs; sw[l] = hws * rhs;
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
        const T df = T(0.5) * ((sd0[f - 1] - smn1[f - 1]) + (sd0[f] - smn1[f]));
        sdf[f] = df;
        rusanov(g, df, se[f - 1] + T(0.5) * sle[f - 1], su[f - 1] + T(0.5) * slu[f - 1],
                sw[f - 1] + T(0.5) * slw[f - 1], se[f] - T(0.5) * sle[f], su[f] - T(0.5) * slu[f],
                sw[f] - T(0.5) * slw[f], F0[f], A1[f], G1[f], F2[f]);
    }
    __syncthreads();

    // G: stage-2 rates and Q~ on [4, NL-4) (the tile and one cell each side)
    for (int l = tid + 4; l < NL - 4; l += TILE) {
        const T hbar = se[l] + T(0.5) * (sdf[l] + sdf[l + 1]);
        const T r0 = -(F0[l + 1] - F0[l]) * idx;
        const T r1 = -((A1[l + 1] - A1[l]) + (G1[l + 1] + G1[l]) + g * hbar * sle[l]) * idx;
        const T r2 = -(F2[l + 1] - F2[l]) * idx;
        const T zn = sz[l] + half_dt * (k1h[l] + r0);
        const T hun = shu[l] + half_dt * (k1u[l] + r1);
        const T hwn = shw[l] + half_dt * (k1w[l] + r2);
        sz[l] = zn; shu[l] = hun; shw[l] = hwn;
        const int j = i0 - H + l;
        if (j >= i0 && j < i0 + TILE && j < nxb) {
            a.zt[mo + j] = zn; a.hut[mo + j] = hun; a.hwt[mo + j] = hwn;
        }
    }
    __syncthreads();

    // H: criterion (Sec. 5.1) on the tile; marks as one bit per cell
    {
        const int l = tid + H, j = i0 + tid;
        const bool inside = j < nxb;
        bool mark = false;
        double mass = 0.0;
        if (inside) {
            mass = (double)sz[l];
            if (a.all_global) {
                mark = true;
            } else if (a.crit >= NH_CRIT_ETA_D) {
                const T inv2dx = T(0.5) * idx;
                // eta~ = zeta~ + m, h~ = zeta~ + d0 at l-1, l, l+1
                const T em = sz[l - 1] + smn1[l - 1], ec = sz[l] + smn1[l], ep = sz[l + 1] + smn1[l + 1];
                const T hm = sz[l - 1] + sd0[l - 1], hc = sz[l] + sd0[l], hp = sz[l + 1] + sd0[l + 1];
                T c;
                switch (a.crit) {
                case NH_CRIT_ETA_D: c = tabs(ec / (sd0[l] - smn1[l])); break;
                case NH_CRIT_ETA_X: c = tabs((ep - em) * inv2dx); break;
                case NH_CRIT_U:     c = tabs(shu[l] / hc); break;
                case NH_CRIT_U_X:   c = tabs((shu[l + 1] / hp - shu[l - 1] / hm) * inv2dx); break;
                case NH_CRIT_W:     c = tabs(shw[l] / hc); break;
                default:            c = tabs((shw[l + 1] / hp - shw[l - 1] / hm) * inv2dx); break;
                }
                mark = c > s_k[4];   // strict, in the state precision
            }
        }
        const uint32_t word = __ballot_sync(0xffffffffu, mark);
        if ((tid & 31) == 0) a.marks[(size_t)b * G.wpitch + (j >> 5)] = word;
        // the tile's FP64 mass: one warp adds the cells' values in a fixed
        // order (fewer FP64 operations than a shuffle tree over every lane)
        red_mass[tid] = mass;
        __syncthreads();
        if (tid < 32) {
            double t = 0.0;
            for (int q = tid; q < TILE; q += 32) t += red_mass[q];
            t = warp_sum(t);
            if (tid == 0) a.mass_part[(size_t)b * G.ntiles + blockIdx.x] = t;
        }
    }
}

// ------------------------------------------------------------- compaction

struct CompactArgs {
    int nx, pitch, wpitch, bc, enlarge;
    const int* nxv;      // per-member cell counts, or null
    const TimeCtl* tc;   // captured runs: stand down after an abort (keeps the last list)
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
static __global__ void __launch_bounds__(kCompactThreads) k_compact(CompactArgs a)
{
    extern __shared__ uint32_t s_m[];
    __shared__ int s_wsum[32];
    __shared__ int s_base;
    const int b = blockIdx.x, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    if (a.tc && a.tc->abort) return;
    const int nwarp = blockDim.x >> 5;
    const int nx = a.nxv ? a.nxv[b] : a.nx;
    const int nw = (nx + 31) >> 5;
    const uint32_t* M = a.marks + (size_t)b * a.wpitch;
    for (int w = tid; w < nw; w += blockDim.x) s_m[w] = M[w];
    if (tid == 0) s_base = 0;
    if (b == 0 && tid == 0) {
        a.ctl->not_done = 0; a.ctl->n_cg = 0; a.ctl->n_bicg = 0; a.ctl->n_fallback = 0;
    }
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
            const int nvalid = nx - 32 * w;
            if (nvalid < 32) acc &= (1u << nvalid) - 1u;
            if (a.bc == NH_BC_PERIODIC && e > 0) {
                const int c0 = 32 * w, c1 = min(32 * w + 32, nx);
                for (int i = c0; i < c1; ++i) {
                    if (i >= e && i < nx - e) continue;
                    for (int k = -e; k <= e; ++k) {
                        int c = (i + k) % nx;
                        if (c < 0) c += nx;
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
        s.auto_kind = 0; s.npb = (n + kPcrRows - 1) / kPcrRows; s.ioff = 0; s.poff = 0;
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

// Work lists of the step: item w = (member, chunk of kChunk active cells),
// pitem w = (member, block of kPcrRows active cells), member-major, so each
// member's items are contiguous from ms[b].ioff / ms[b].poff.  One CTA.
static __global__ void __launch_bounds__(1024) k_items(MState* ms, int nb, int2* items, int2* pitems, Ctl* ctl)
{
    __shared__ int s_w[2][32];
    __shared__ int s_base[2];
    __shared__ int s_maxpb;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nwarp = blockDim.x >> 5;
    if (tid == 0) { s_base[0] = 0; s_base[1] = 0; s_maxpb = 0; }
    __syncthreads();
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int b = b0 + tid;
        const int c0 = b < nb ? ms[b].nchunks : 0, c1 = b < nb ? ms[b].npb : 0;
        if (c1 > 1) atomicMax(&s_maxpb, c1);
        int i0 = c0, i1 = c1;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y0 = __shfl_up_sync(0xffffffffu, i0, o), y1 = __shfl_up_sync(0xffffffffu, i1, o);
            if (lane >= o) { i0 += y0; i1 += y1; }
        }
        if (lane == 31) { s_w[0][wid] = i0; s_w[1][wid] = i1; }
        __syncthreads();
        if (wid == 0) {
            int v0 = lane < nwarp ? s_w[0][lane] : 0, v1 = lane < nwarp ? s_w[1][lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y0 = __shfl_up_sync(0xffffffffu, v0, o), y1 = __shfl_up_sync(0xffffffffu, v1, o);
                if (lane >= o) { v0 += y0; v1 += y1; }
            }
            s_w[0][lane] = v0; s_w[1][lane] = v1;
        }
        __syncthreads();
        const int o0 = s_base[0] + i0 - c0 + (wid > 0 ? s_w[0][wid - 1] : 0);
        const int o1 = s_base[1] + i1 - c1 + (wid > 0 ? s_w[1][wid - 1] : 0);
        if (b < nb) {
            ms[b].ioff = o0;
            ms[b].poff = o1;
            for (int j = 0; j < c0; ++j) items[o0 + j] = make_int2(b, j);
            for (int j = 0; j < c1; ++j) pitems[o1 + j] = make_int2(b, j);
        }
        __syncthreads();
        if (tid == 0) { s_base[0] += s_w[0][nwarp - 1]; s_base[1] += s_w[1][nwarp - 1]; }
        __syncthreads();
    }
    if (tid == 0) { ctl->n_items = s_base[0]; ctl->n_pitems = s_base[1]; ctl->max_npb = s_maxpb; }
}

// Deterministic block-wide sum of part[0..n) (thread 0 gets it).
__device__ __forceinline__ double member_sum(const double* part, int n, double* sh)
{
    double v[1] = {0.0};
    for (int q = threadIdx.x; q < n; q += blockDim.x) v[0] += __ldcg(part + q);
    block_sum<1>(v, sh);
    return v[0];
}

// The same for three partial arrays at part, part + stride, part + 2 stride
// in one block reduction (thread 0 gets v[0..2]).
__device__ __forceinline__ void member_sum3(const double* part, size_t stride, int n, double* sh, double (&v)[3])
{
    v[0] = v[1] = v[2] = 0.0;
    for (int q = threadIdx.x; q < n; q += blockDim.x) {
        v[0] += __ldcg(part + q);
        v[1] += __ldcg(part + stride + q);
        v[2] += __ldcg(part + 2 * stride + q);
    }
    block_sum<3>(v, sh);
}
__device__ __forceinline__ double member_min(const double* part, int n, double* sh)
{
    double v = INFINITY;
    for (int q = threadIdx.x; q < n; q += blockDim.x) v = fmin(v, __ldcg(part + q));
    return block_min(v, sh);
}

// --------------------------------------------------------------- assembly

template <typename TS>
struct AsmArgs {
    Geo G;
    const TS* zt; const TS* hut; const TS* hwt;   // Q~ (zeta = h - d0)
    const double* d0;                           // static depth, FP64
    const Slide* slide; const Kin* kin;
    const int* list; const uint32_t* act;
    MState* ms;
    double* diag; double* offl; double* offr; double* R;      // FP64 operator
    float* diag32; float* offl32; float* offr32;              // FP32 copies (mixed)
    int* nbl; int* nbr;
    TS* c6; TS* cx; TS* phi; TS* ddx;           // correction coefficients
    double* part;                               // [2][nb * maxch]
    int* cnt;
    const int2* items; const Ctl* ctl;
    double dt;
    int solver;                                 // NH_SOLVER_*
};

struct CellQ {
    double h, K, beta, U0, V, phi, d_x, D, d_t;
    double rh, rD;   // 1 / h, 1 / D
};

// Per-cell quantities of the elliptic equation at an in-domain cell c, in FP64
// whatever the state precision, from the cell's bottom terms B and the surface
// at its two neighbours.
template <typename TS>
__device__ __forceinline__ CellQ cell_q_from(const AsmArgs<TS>& a, const TS* __restrict__ zt,
                                             const TS* __restrict__ hut, const double* __restrict__ D0,
                                             int c, const Bottom<double>& B, double etam, double etap)
{
    const Geo& G = a.G;
    const double eta_x = (etap - etam) * G.i2dx;
    CellQ q;
    q.h = (double)zt[c] + D0[c];
    q.rh = 1.0 / q.h;   // the two reciprocals of the cell: every quotient below multiplies
    const double u = (double)hut[c] * q.rh;
    q.d_x = B.d_x;
    q.d_t = B.d_t;
    q.D = 4.0 + B.d_x * B.d_x;
    q.rD = 1.0 / q.D;
    q.phi = a.dt * q.h * q.rD * (G.g * B.d_x * eta_x - B.d_tt - 2.0 * u * B.d_xt - u * u * B.d_xx);
    q.K = 4.0 * q.rh * q.rD;
    q.beta = 6.0 * B.d_x * (q.rh * q.rh) * q.rD;
    q.U0 = (double)hut[c] + q.phi * B.d_x;
    q.V = q.U0 * q.rh;
    return q;
}

// The same with the bottom and the neighbours' surface evaluated here.
template <typename TS>
__device__ __forceinline__ CellQ cell_q(const AsmArgs<TS>& a, const TS* __restrict__ zt,
                                        const TS* __restrict__ hut, const double* __restrict__ D0,
                                        int c, int nxb, const Slide& sl, const Kin& kn)
{
    const Geo& G = a.G;
    const Bottom<double> B = bottom_full(D0, c, nxb, G.bc, G.x0, G.dx, sl, kn);
    int sg;
    const int cm = resolve(c - 1, nxb, G.bc, &sg), cp = resolve(c + 1, nxb, G.bc, &sg);
    const double etam = (double)zt[cm] + mound_at<double>(cm, G.x0, G.dx, sl, kn.s_n1);
    const double etap = (double)zt[cp] + mound_at<double>(cp, G.x0, G.dx, sl, kn.s_n1);
    return cell_q_from(a, zt, hut, D0, c, B, etam, etap);
}

__device__ __forceinline__ bool bit_at(const uint32_t* w, int i)
{
    return (w[i >> 5] >> (i & 31)) & 1u;
}

template <typename TS>
__global__ void __launch_bounds__(kChunk) k_assemble(AsmArgs<TS> a)
{
    __shared__ double red[64];
    __shared__ double s_eta[kChunk], s_K[kChunk], s_beta[kChunk], s_V[kChunk];
    __shared__ int s_cell[kChunk];
    __shared__ CellQ s_q[kChunk];
    const Geo& G = a.G;
    const int tid = threadIdx.x;
    const int n_items = a.ctl->n_items;
    for (int wi = blockIdx.x; wi < n_items; wi += gridDim.x) {
        const int2 itm = a.items[wi];
        const int b = itm.x, j = itm.y;
        const int n = a.ms[b].n_active;
        const int nch = a.ms[b].nchunks;
        const int ioff = a.ms[b].ioff;
        const size_t mo = (size_t)b * G.pitch;
        const TS* zt = a.zt + mo; const TS* hut = a.hut + mo; const TS* hwt = a.hwt + mo;
        const double* D0 = a.d0 + mo;
        const uint32_t* act = a.act + (size_t)b * G.wpitch;
        const Slide sl = a.slide[b];
        const Kin kn = a.kin[b];
        const int k = j * kChunk + tid;
        const bool in = k < n;
        const int nxb = member_nx(G, b);
        // phase 1: own cell's bottom terms and surface (shared with the neighbours)
        int i = -1;
        Bottom<double> B;
        if (in) {
            i = a.list[mo + k];
            B = bottom_full(D0, i, nxb, G.bc, G.x0, G.dx, sl, kn);
            s_eta[tid] = (double)zt[i] + B.m;
        }
        s_cell[tid] = i;
        __syncthreads();
        // phase 2: own cell's coefficients; a neighbour that is the adjacent
        // entry of this chunk's list shares its surface, others are evaluated
        const bool left_here = in && tid > 0 && s_cell[tid - 1] == i - 1;
        const bool right_here = in && tid + 1 < kChunk && k + 1 < n && s_cell[tid + 1] == i + 1;
        int sgm = 1, sgp = 1, cm = -1, cp = -1;
        if (in) {
            cm = resolve(i - 1, nxb, G.bc, &sgm);
            cp = resolve(i + 1, nxb, G.bc, &sgp);
            const double etam = left_here ? s_eta[tid - 1]
                                          : (double)zt[cm] + mound_at<double>(cm, G.x0, G.dx, sl, kn.s_n1);
            const double etap = right_here ? s_eta[tid + 1]
                                           : (double)zt[cp] + mound_at<double>(cp, G.x0, G.dx, sl, kn.s_n1);
            const CellQ q = cell_q_from(a, zt, hut, D0, i, B, etam, etap);
            s_K[tid] = q.K; s_beta[tid] = q.beta; s_V[tid] = q.V;
            s_q[tid] = q;
        }
        __syncthreads();
        double r2 = 0.0, gmin = INFINITY;
        if (in) {
            const CellQ qi = s_q[tid];
            CellQ qm, qp;
            if (left_here) { qm.K = s_K[tid - 1]; qm.beta = s_beta[tid - 1]; qm.V = s_V[tid - 1]; }
            else qm = cell_q(a, zt, hut, D0, cm, nxb, sl, kn);
            if (right_here) { qp.K = s_K[tid + 1]; qp.beta = s_beta[tid + 1]; qp.V = s_V[tid + 1]; }
            else qp = cell_q(a, zt, hut, D0, cp, nxb, sl, kn);
            const double idx2 = G.idx2;
            const double Kl = 0.5 * (qm.K + qi.K), Kr = 0.5 * (qi.K + qp.K);
            const double bm = sgm > 0 ? qm.beta : -qm.beta, bp = sgp > 0 ? qp.beta : -qp.beta;
            const double Vm = sgm > 0 ? qm.V : -qm.V, Vp = sgp > 0 ? qp.V : -qp.V;
            const double rh = qi.rh, rh2 = rh * rh;
            const double gam = (bp - bm) * G.i2dx + 12.0 * (1.0 + qi.d_x * qi.d_x) * (rh2 * rh * qi.rD);
            const double Rk = -((Vp - Vm) * G.i2dx + 2.0 * qi.d_x * qi.U0 * rh2 + 2.0 * (double)hwt[i] * rh2
                                + 2.0 * qi.phi * rh2 + 2.0 * qi.d_t * rh);
            // neighbours inside the active set (zero Dirichlet data outside)
            bool hasl, hasr;
            int kl = -1, kr = -1;
            if (G.bc == NH_BC_PERIODIC) {
                hasl = bit_at(act, cm);
                hasr = bit_at(act, cp);
                if (hasl) kl = (i == 0) ? n - 1 : k - 1;
                if (hasr) kr = (i == nxb - 1) ? 0 : k + 1;
            } else {
                hasl = (i > 0) && bit_at(act, i - 1);
                hasr = (i < nxb - 1) && bit_at(act, i + 1);
                if (hasl) kl = k - 1;
                if (hasr) kr = k + 1;
            }
            const double dg = (Kl + Kr) * idx2 + gam;
            const double ol = hasl ? -Kl * idx2 : 0.0;
            const double orr = hasr ? -Kr * idx2 : 0.0;
            a.diag[mo + k] = dg;
            a.offl[mo + k] = ol;
            a.offr[mo + k] = orr;
            a.R[mo + k] = Rk;
            if (a.diag32) {
                a.diag32[mo + k] = (float)dg;
                a.offl32[mo + k] = (float)ol;
                a.offr32[mo + k] = (float)orr;
            }
            a.nbl[mo + k] = kl;
            a.nbr[mo + k] = kr;
            a.c6[mo + k] = TS(6.0 * rh * qi.rD);
            a.cx[mo + k] = TS(qi.d_x * qi.rD);
            a.phi[mo + k] = TS(qi.phi);
            a.ddx[mo + k] = TS(qi.d_x);
            r2 = Rk * Rk;
            gmin = gam;
        }
        double v[1] = {r2};
        block_sum<1>(v, red);
        const double gm = block_min(gmin, red);
        double* P0 = a.part;
        double* P1 = a.part + (size_t)G.nb * G.maxch;
        if (tid == 0) { P0[wi] = v[0]; P1[wi] = gm; }
        if (arrive_last(a.cnt, b, nch)) {
            const double bn2 = member_sum(P0 + ioff, nch, red);
            const double gmn = member_min(P1 + ioff, nch, red);
            if (tid == 0) {
                MState& s = a.ms[b];
                s.bnorm2 = bn2;
                s.bnorm = sqrt(bn2);
                s.min_gamma = gmn;
                // AUTO: the operator is symmetric, so CG; gamma > 0 on every
                // active cell guarantees positive definiteness, otherwise CG's
                // own curvature checks decide and BiCGStab takes over on failure
                s.auto_kind = (a.solver == NH_SOLVER_AUTO);
                s.kind = (a.solver == NH_SOLVER_BICGSTAB) ? NH_SOLVER_BICGSTAB : NH_SOLVER_CG;
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
    T* r1; T* z;               // PCG: second residual buffer, preconditioned residual
    float2* pf;                // line preconditioner: PCR multipliers [kPcrLevels][nb * pitch]
    float* prb;                // line preconditioner: reciprocal final pivots [nb * pitch]
    size_t pf_stride;          // nb * pitch
    // extra couplings of a row beyond its list neighbours (2D grids: S, N and
    // the four diagonals); n_ext = 0 for 1D members
    int n_ext;
    const double* ext_c;       // [n_ext][nb * pitch] coefficients
    const int* ext_k;          // [n_ext][nb * pitch] compact index of the neighbour, or -1
    size_t ext_stride;         // nb * pitch
    int maxpb;                 // preconditioner blocks per member (upper bound)
    const int2* items; const int2* pitems;
    const TimeCtl* tc;         // captured runs: guess scale from tc->prev_ok
    MState* ms; Ctl* ctl;
    double* part;              // [4][nb * maxch]; slot 3: the persistent PCG's <p, q> item partials
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

// Sum of the extra couplings of row k: sum_e c_e v(k_e), v(j) the vector's
// value at compact index j (a callable).
template <typename T, typename F>
__device__ __forceinline__ T ext_terms(const SolveArgs<T>& a, size_t mo, int k, F v)
{
    // all neighbour indices first, then the values: the loads of the
    // couplings overlap instead of forming a chain per coupling
    int jj[kMaxExt];
#pragma unroll
    for (int e = 0; e < kMaxExt; ++e)
        jj[e] = e < a.n_ext ? __ldg(a.ext_k + (size_t)e * a.ext_stride + mo + k) : -1;
    T s = T(0);
#pragma unroll
    for (int e = 0; e < kMaxExt; ++e)
        if (jj[e] >= 0) s += T(__ldg(a.ext_c + (size_t)e * a.ext_stride + mo + k)) * v(jj[e]);
    return s;
}

// Shared prologue of the solve kernels: loop over (member, chunk) work items.
#define NH_FOR_ITEMS(A)                                                         \
    const int n_items_ = (A).ctl->n_items;                                      \
    for (int wi = blockIdx.x; wi < n_items_; wi += gridDim.x) {                 \
        const int2 itm_ = (A).items[wi];                                        \
        const int b = itm_.x, j = itm_.y;                                       \
        const int nch = (A).ms[b].nchunks;                                      \
        const int n = (A).ms[b].n_active;                                       \
        const int ioff = (A).ms[b].ioff;                                        \
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
        if (a.ms[b].done) continue;
        double rr = 0.0;
        if (in) {
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            const double sc = a.tc ? (a.tc->prev_ok && a.guess_scale != 0.0 ? 1.0 : 0.0) : a.guess_scale;
            T x0 = T(0), xl = T(0), xr = T(0);
            if (sc != 0.0) {
                x0 = T(a.psi_prev[mo + a.list[mo + k]] * sc);
                if (kl >= 0) xl = T(a.psi_prev[mo + a.list[mo + kl]] * sc);
                if (kr >= 0) xr = T(a.psi_prev[mo + a.list[mo + kr]] * sc);
            }
            T ax = apply_row(a, mo, k, x0, xl, xr);
            if (a.n_ext && sc != 0.0)
                ax += ext_terms(a, mo, k, [&](int j) { return T(a.psi_prev[mo + a.list[mo + j]] * sc); });
            const T rk = a.R[mo + k] - ax;
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
            const double s_rr = member_sum(P0 + ioff, nch, red);
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

// Candidate initial guesses judged by the energy CG minimises: for a
// symmetric positive definite A with solution x*, ||x - x*||_A^2 =
// J(x) - J(x*), J(x) = x.Ax - 2 x.R.  Against the warm start x0 (cand0) each
// candidate c = 1, 2 differs by dJ_c = d.Ad - 2 d.r0 (d = x_c - x0,
// r0 = R - A x0) = ||e_c||_A^2 - ||e_0||_A^2, summed over each member's active
// cells from the small quantities d and r0 (no cancellation against J).  The
// lowest of {0, dJ_1, dJ_2} wins (ties go to the lower index) and is recorded
// in choice[b] and counts[].  Candidates are scaled like the warm start.
struct JudgeArgs {
    int pitch;
    size_t stride;             // nb * maxch: offset between the partial-sum slots
    const int* list; const int* nbl; const int* nbr;
    const double* diag; const double* offl; const double* offr; const double* R;
    const double* cand0; const double* cand1; const double* cand2;
    double guess_scale;
    const TimeCtl* tc;
    const int2* items; MState* ms; const Ctl* ctl;
    double* part; int* cnt;
    int* choice; unsigned long long* counts;
};

static __global__ void __launch_bounds__(kChunk) k_guess_judge(JudgeArgs a)
{
    __shared__ double red[96];
    if (a.tc && a.tc->abort) return;
    const double sc = a.tc ? (a.tc->prev_ok && a.guess_scale != 0.0 ? 1.0 : 0.0) : a.guess_scale;
    NH_FOR_ITEMS(a)
        double dj[3] = {0.0, 0.0, 0.0};
        if (in) {
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            const size_t i0 = mo + a.list[mo + k];
            const size_t il = kl >= 0 ? mo + a.list[mo + kl] : 0;
            const size_t ir = kr >= 0 ? mo + a.list[mo + kr] : 0;
            const double dg = a.diag[mo + k], ol = a.offl[mo + k], orr = a.offr[mo + k];
            const double x0 = a.cand0[i0] * sc;
            const double x0l = kl >= 0 ? a.cand0[il] * sc : 0.0;
            const double x0r = kr >= 0 ? a.cand0[ir] * sc : 0.0;
            const double r0 = a.R[mo + k] - (dg * x0 + ol * x0l + orr * x0r);
            const double* c[2] = {a.cand1, a.cand2};
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const double d = c[q][i0] * sc - x0;
                const double dl = kl >= 0 ? c[q][il] * sc - x0l : 0.0;
                const double dr = kr >= 0 ? c[q][ir] * sc - x0r : 0.0;
                dj[q + 1] = d * (dg * d + ol * dl + orr * dr) - 2.0 * d * r0;
            }
        }
        block_sum<3>(dj, red);
        if (threadIdx.x == 0) {
            a.part[a.stride + wi] = dj[1];
            a.part[2 * a.stride + wi] = dj[2];
        }
        if (arrive_last(a.cnt, b, nch)) {
            const double s1 = member_sum(a.part + a.stride + ioff, nch, red);
            const double s2 = member_sum(a.part + 2 * a.stride + ioff, nch, red);
            if (threadIdx.x == 0) {
                int best = 0;
                double bv = 0.0;
                if (isfinite(s1) && s1 < bv) { best = 1; bv = s1; }
                if (isfinite(s2) && s2 < bv) { best = 2; bv = s2; }
                a.choice[b] = best;
                atomicAdd(&a.counts[best], 1ull);
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

// CG curvature or preconditioner breakdown: AUTO members hand over to
// BiCGStab (restarted from the warm start); forced CG reports NONFINITE.
template <typename T>
__device__ __forceinline__ void cg_breakdown(MState& s, Ctl* ctl, int it)
{
    if (s.auto_kind && s.kind == NH_SOLVER_CG) {
        s.status = kStatusFallback;
        s.iters = it;
        s.done = 1;
        atomicSub(&ctl->not_done, 1);
        atomicAdd(&ctl->n_fallback, 1);
    } else {
        finish_member<T>(s, ctl, NH_ERR_NONFINITE, it, NAN);
    }
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
            T qk = apply_row(a, mo, k, pk, pl, pr);
            if (a.n_ext) qk += ext_terms(a, mo, k, [&](int j) { return a.r[mo + j] + beta * pold[mo + j]; });
            pnew[mo + k] = pk;
            a.q[mo + k] = qk;
            pq = (double)pk * (double)qk;
        }
        double v[1] = {pq};
        block_sum<1>(v, red);
        if (threadIdx.x == 0) a.part[wi] = v[0];
        if (arrive_last(a.cnt, b, nch)) {
            const double s_pq = member_sum(a.part + ioff, nch, red);
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                if (!isfinite(s_pq) || !(s_pq > 0.0)) cg_breakdown<T>(s, a.ctl, it);
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
            const double s_rr = member_sum(a.part + ioff, nch, red);
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
            T vk = apply_row(a, mo, k, pk, pl, pr);
            if (a.n_ext)
                vk += ext_terms(a, mo, k, [&](int j) { return a.r[mo + j] + beta * (pold[mo + j] - omega * vold[mo + j]); });
            pnew[mo + k] = pk;
            vnew[mo + k] = vk;
            rv = (double)a.rh[mo + k] * (double)vk;
        }
        double v[1] = {rv};
        block_sum<1>(v, red);
        if (threadIdx.x == 0) a.part[wi] = v[0];
        if (arrive_last(a.cnt, b, nch)) {
            const double s_rv = member_sum(a.part + ioff, nch, red);
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
            T tk = apply_row(a, mo, k, sk, sl, sr);
            if (a.n_ext) tk += ext_terms(a, mo, k, [&](int j) { return a.r[mo + j] - alpha * v[mo + j]; });
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
            const size_t mb = ioff;
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
            const size_t mb = ioff;
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


// ------------------------------------------- preconditioned CG (line / PCR)

// Line preconditioner z = M^{-1} r_new.  M is the tridiagonal operator
// restricted to blocks of kPcrRows consecutive active cells (couplings across a
// block edge are dropped; a contiguous active segment inside one block is
// solved exactly), factorised by parallel cyclic reduction in shared memory in
// precision TP.  Partials <z, r_new> and <z, r_old> feed the flexible
// (Polak-Ribiere) beta = (<z, r_new> - <z, r_old>) / <z_old, r_old>, which
// tolerates the rounding of a low-precision preconditioner.  it == 0 is the
// set-up pass after k_solve_init (rz only).
enum { PCR_PCG = 0, PCR_BI_P = 1, PCR_BI_S = 2, PCR_PCG_STEP = 3 };

// Right-hand side of the preconditioner solve for row k, formed element-wise
// and stored: PCG set-up reads r; the fused PCG step first updates
// x += alpha p and r_new = r_old - alpha q; BiCGStab forms p and s.
template <typename T>
__device__ __forceinline__ T pcr_rhs(const SolveArgs<T>& a, int mode, int it, size_t idx,
                                     T beta, T omega, T alpha)
{
    if (mode == PCR_PCG) return a.r[idx];
    if (mode == PCR_PCG_STEP) {
        const T* p = (it & 1) ? a.p1 : a.p0;
        const T* rold = (it & 1) ? a.r : a.r1;
        T* rnew = (it & 1) ? a.r1 : a.r;
        a.x[idx] = a.x[idx] + alpha * p[idx];
        const T rk = rold[idx] - alpha * a.q[idx];
        rnew[idx] = rk;
        return rk;
    }
    if (mode == PCR_BI_P) {
        const T pk = a.r[idx] + beta * (a.p0[idx] - omega * a.v0[idx]);
        a.p0[idx] = pk;
        return pk;
    }
    const T sk = a.r[idx] - alpha * a.v0[idx];
    a.s[idx] = sk;
    return sk;
}

// Parallel cyclic reduction of one block's tridiagonal rows, factor phase:
// at level l (stride s = 2^l) row i is combined with rows i - s and i + s
// using al = -a_i / b_{i-s} and ga = -c_i / b_{i+s} (zero where the row does
// not exist); the multipliers and, at the end, 1 / b_i are stored, since the
// matrix is the same for every preconditioner application of one solve.
// Runs once per solve for every member that still iterates.
template <typename T, typename TP>
__global__ void __launch_bounds__(kPcrThreads) k_pcr_factor(SolveArgs<T> a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TP* sa = reinterpret_cast<TP*>(smem_raw);
    TP* sb = sa + kPcrRows;
    TP* sc = sb + kPcrRows;
    constexpr int RPT = kPcrRows / kPcrThreads;
    const int n_pitems = a.ctl->n_pitems;
    for (int wi = blockIdx.x; wi < n_pitems; wi += gridDim.x) {
        const int2 itm = a.pitems[wi];
        const int b = itm.x, jb = itm.y;
        if (a.ms[b].done) continue;
        const int n = a.ms[b].n_active;
        const size_t mo = (size_t)b * a.pitch;
        const int k0 = jb * kPcrRows;
        const int rows = min(kPcrRows, n - k0);
        for (int i = threadIdx.x; i < rows; i += kPcrThreads) {
            const int k = k0 + i;
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            sa[i] = (i > 0 && kl == k - 1) ? TP(a.offl[mo + k]) : TP(0);
            sc[i] = (i < rows - 1 && kr == k + 1) ? TP(a.offr[mo + k]) : TP(0);
            sb[i] = TP(a.diag[mo + k]);
        }
        __syncthreads();
        int lev = 0;
        for (int st = 1; st < rows; st <<= 1, ++lev) {
            TP na[RPT], nb2[RPT], nc[RPT];
            float2* f = a.pf + (size_t)lev * a.pf_stride + mo + k0;
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                const int i = threadIdx.x + m * kPcrThreads;
                if (i < rows) {
                    const TP ai = sa[i], ci = sc[i];
                    TP a2 = TP(0), c2 = TP(0), b2 = sb[i], al = TP(0), ga = TP(0);
                    if (i - st >= 0) {
                        al = -ai / sb[i - st];
                        a2 = al * sa[i - st]; b2 += al * sc[i - st];
                    }
                    if (i + st < rows) {
                        ga = -ci / sb[i + st];
                        c2 = ga * sc[i + st]; b2 += ga * sa[i + st];
                    }
                    na[m] = a2; nb2[m] = b2; nc[m] = c2;
                    f[i] = make_float2((float)al, (float)ga);
                }
            }
            __syncthreads();
#pragma unroll
            for (int m = 0; m < RPT; ++m) {
                const int i = threadIdx.x + m * kPcrThreads;
                if (i < rows) { sa[i] = na[m]; sb[i] = nb2[m]; sc[i] = nc[m]; }
            }
            __syncthreads();
        }
        for (int i = threadIdx.x; i < rows; i += kPcrThreads) a.prb[mo + k0 + i] = (float)(TP(1) / sb[i]);
        __syncthreads();
    }
}

// Apply phase of the factored reduction to the right-hand side held in s0
// (rows of one block): d_i <- d_i + al d_{i-s} + ga d_{i+s} level by level,
// ping-ponging between s0 and s1 (one barrier per level).  Returns the buffer
// holding the reduced right-hand side; z_i = d_i / b_i = d_i prb_i.
template <typename T, typename TP>
__device__ __forceinline__ TP* pcr_apply(const SolveArgs<T>& a, TP* s0, TP* s1, int rows, size_t base)
{
    constexpr int RPT = kPcrRows / kPcrThreads;
    TP* src = s0;
    TP* dst = s1;
    // the next level's multipliers are fetched before this level's barrier,
    // so their L2 latency overlaps the wait
    float2 fi[RPT];
#pragma unroll
    for (int m = 0; m < RPT; ++m) {
        const int i = threadIdx.x + m * kPcrThreads;
        fi[m] = (i < rows && rows > 1) ? __ldcg(a.pf + base + i) : make_float2(0.f, 0.f);
    }
    int lev = 0;
    for (int st = 1; st < rows; st <<= 1, ++lev) {
        float2 fn[RPT];
        const bool more = (st << 1) < rows;
        const float2* f1 = a.pf + (size_t)(lev + 1) * a.pf_stride + base;
#pragma unroll
        for (int m = 0; m < RPT; ++m) {
            const int i = threadIdx.x + m * kPcrThreads;
            fn[m] = (more && i < rows) ? __ldcg(f1 + i) : make_float2(0.f, 0.f);
            if (i < rows) {
                TP d = src[i];
                if (i - st >= 0) d += TP(fi[m].x) * src[i - st];
                if (i + st < rows) d += TP(fi[m].y) * src[i + st];
                dst[i] = d;
            }
        }
        __syncthreads();
#pragma unroll
        for (int m = 0; m < RPT; ++m) fi[m] = fn[m];
        TP* t = src; src = dst; dst = t;
    }
    return src;
}

// Line preconditioner z = M^{-1} rhs.  M is the tridiagonal operator
// restricted to blocks of kPcrRows consecutive active cells (couplings across a
// block edge are dropped; a contiguous active segment inside one block is
// solved exactly), factorised by parallel cyclic reduction in shared memory in
// precision TP.
//  PCR_PCG      (it = 0) after k_solve_init: z = M^{-1} r, rz = <z, r>.
//  PCR_PCG_STEP (it >= 1) fused second half of PCG iteration it: x += alpha p,
//               r_new = r_old - alpha q, convergence test on ||r_new||, then
//               z = M^{-1} r_new and the flexible (Polak-Ribiere)
//               beta = (<z, r_new> - <z, r_old>) / <z_old, r_old>, which
//               tolerates the rounding of a low-precision preconditioner.
//  PCR_BI_P / PCR_BI_S  BiCGStab's p-hat = M^{-1} p (into p1), s-hat = M^{-1} s
//               (into z) with the ||s|| test.
template <typename T, typename TP>
__global__ void __launch_bounds__(kPcrThreads) k_pcr(SolveArgs<T> a, int mode)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TP* sa = reinterpret_cast<TP*>(smem_raw);   // reduction ping-pong buffers
    TP* sd = sa + kPcrRows;
    __shared__ double red[96];
    const int it = a.it;
    const T* rnew = (mode == PCR_PCG) ? a.r : ((it & 1) ? a.r1 : a.r);
    const T* rold = (it & 1) ? a.r : a.r1;
    const size_t stride = (size_t)a.nb * a.maxch;
    const int want = (mode == PCR_PCG || mode == PCR_PCG_STEP) ? NH_SOLVER_CG : NH_SOLVER_BICGSTAB;
    const int n_pitems = a.ctl->n_pitems;
    for (int wi = blockIdx.x; wi < n_pitems; wi += gridDim.x) {
        const int2 itm = a.pitems[wi];
        const int b = itm.x, jb = itm.y;
        if (a.ms[b].done || a.ms[b].kind != want) continue;
        const int n = a.ms[b].n_active;
        const int npb = a.ms[b].npb;
        const int poff = a.ms[b].poff;
        const size_t mo = (size_t)b * a.pitch;
        const int k0 = jb * kPcrRows;
        const int rows = min(kPcrRows, n - k0);
        const T beta = T(a.ms[b].beta), omega = T(a.ms[b].omega), alpha = T(a.ms[b].alpha);
        double ss = 0.0;
        for (int i = threadIdx.x; i < rows; i += kPcrThreads) {
            const int k = k0 + i;
            const T rhs = pcr_rhs(a, mode, it, mo + k, beta, omega, alpha);
            if (mode == PCR_BI_S || mode == PCR_PCG_STEP) ss += (double)rhs * (double)rhs;
            sd[i] = TP(rhs);
        }
        __syncthreads();
        const TP* red_d = pcr_apply<T, TP>(a, sd, sa, rows, mo + k0);
        double acc[3] = {0.0, 0.0, ss};
        T* out = (mode == PCR_BI_P) ? a.p1 : a.z;
        for (int i = threadIdx.x; i < rows; i += kPcrThreads) {
            const int k = k0 + i;
            const T zk = T(red_d[i] * TP(a.prb[mo + k]));
            out[mo + k] = zk;
            if (mode == PCR_PCG || mode == PCR_PCG_STEP) {
                acc[0] += (double)zk * (double)rnew[mo + k];
                if (mode == PCR_PCG_STEP) acc[1] += (double)zk * (double)rold[mo + k];
            }
        }
        if (mode == PCR_BI_P) { __syncthreads(); continue; }   // no reduction for p-hat
        block_sum<3>(acc, red);
        if (threadIdx.x == 0) {
            a.part[wi] = acc[0]; a.part[stride + wi] = acc[1]; a.part[2 * stride + wi] = acc[2];
        }
        if (!arrive_last(a.cnt, b, npb)) continue;
        if (mode == PCR_BI_S) {
            const double s_ss = member_sum(a.part + 2 * stride + poff, npb, red);
            if (threadIdx.x == 0) {
                MState& st = a.ms[b];
                st.snorm = sqrt(s_ss);
                if (!isfinite(s_ss)) finish_member<T>(st, a.ctl, NH_ERR_NONFINITE, it, NAN);
                else if (st.snorm <= a.rtol * st.bnorm) st.s_conv = 1;
            }
            continue;
        }
        const double zr = member_sum(a.part + poff, npb, red);
        const double zro = member_sum(a.part + stride + poff, npb, red);
        const double rr = member_sum(a.part + 2 * stride + poff, npb, red);
        if (threadIdx.x == 0) {
            MState& st = a.ms[b];
            if (mode == PCR_PCG) {
                if (!isfinite(zr) || !(zr > 0.0)) cg_breakdown<T>(st, a.ctl, it);
                else st.rz = zr;
            } else {
                const double rel = sqrt(rr) / st.bnorm;
                if (!isfinite(rr)) finish_member<T>(st, a.ctl, NH_ERR_NONFINITE, it, NAN);
                else if (sqrt(rr) <= a.rtol * st.bnorm) finish_member<T>(st, a.ctl, NH_OK, it, rel);
                else if (it >= a.max_iter) finish_member<T>(st, a.ctl, NH_ERR_NOT_CONVERGED, it, rel);
                else if (!isfinite(zr) || !(zr > 0.0)) cg_breakdown<T>(st, a.ctl, it);
                else { st.beta = (zr - zro) / st.rz; st.rz = zr; st.rr = rr; }
            }
        }
    }
}

// PCG, first kernel of iteration it: p = z + beta p_old (neighbours on the
// fly), q = A p, partial <p, q>; last CTA: alpha = <r, z> / <p, q>.  The
// neighbours of active cell k are k -/+ 1 except across a periodic wrap, so
// z and p_old are loaded at k -/+ 1 without waiting for the neighbour index.
template <typename T>
__global__ void __launch_bounds__(kChunk) k_pcg_a(SolveArgs<T> a)
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
            const int km = k > 0 ? k - 1 : k, kp = k + 1 < n ? k + 1 : k;
            const T zk = a.z[mo + k], zm = a.z[mo + km], zp = a.z[mo + kp];
            const T ok = pold[mo + k], om = pold[mo + km], op = pold[mo + kp];
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            const T pk = zk + beta * ok;
            T pl = T(0), pr = T(0);
            if (kl == k - 1) pl = zm + beta * om;
            else if (kl >= 0) pl = a.z[mo + kl] + beta * pold[mo + kl];
            if (kr == k + 1) pr = zp + beta * op;
            else if (kr >= 0) pr = a.z[mo + kr] + beta * pold[mo + kr];
            T qk = apply_row(a, mo, k, pk, pl, pr);
            if (a.n_ext) qk += ext_terms(a, mo, k, [&](int j) { return a.z[mo + j] + beta * pold[mo + j]; });
            pnew[mo + k] = pk;
            a.q[mo + k] = qk;
            pq = (double)pk * (double)qk;
        }
        double v[1] = {pq};
        block_sum<1>(v, red);
        if (threadIdx.x == 0) a.part[wi] = v[0];
        if (arrive_last(a.cnt, b, nch)) {
            const double s_pq = member_sum(a.part + ioff, nch, red);
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                if (!isfinite(s_pq) || !(s_pq > 0.0)) cg_breakdown<T>(s, a.ctl, it);
                else s.alpha = s.rz / s_pq;
            }
        }
    NH_END_ITEMS
}



// ------------------------------------------- persistent PCG (one launch)

// Grid-wide barrier for a cooperative launch (all CTAs co-resident).  The
// spin is bounded by `budget` clock cycles: on expiry the CTA records a
// timeout and returns false instead of waiting for ever.  The last CTA to
// arrive runs `last` (a decision every CTA reads after the barrier) before
// releasing the others.
template <typename F>
__device__ __forceinline__ bool grid_barrier(Ctl* ctl, unsigned nblocks, long long budget, F last)
{
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = &ctl->bar_gen;
        const unsigned g = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(&ctl->bar_count, 1u) + 1u;
        int ok = 1;
        if (arrived == nblocks) {
            last();
            ctl->bar_count = 0u;
            __threadfence();
            atomicAdd(&ctl->bar_gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g) {
                if (clock64() - t0 > budget) { ok = 0; atomicExch(&ctl->timeout, 1); break; }
                __nanosleep(64);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Member-local PCG: when no member has more than one preconditioner block,
// a member's whole solve lives in one CTA (its rows are one block), so every
// iteration needs only block barriers and block reductions: no grid barrier,
// no cross-CTA reduction, and members finish independently.  Same algorithm
// and arithmetic as the grid-wide loop below (p = z + beta p_old, q = A p,
// alpha = rz / <p, q>, x and r update, z = M^{-1} r, flexible beta).
template <typename T, typename TP>
__device__ void pcg_member_local(const SolveArgs<T>& a, TP* sa, TP* sd, double* red)
{
    constexpr int kBreakdown = -2;
    __shared__ double s_bc[4];
    const int n_pitems = a.ctl->n_pitems;
    for (int wi = blockIdx.x; wi < n_pitems; wi += gridDim.x) {
        const int b = a.pitems[wi].x;
        MState& st = a.ms[b];
        if (st.done || st.kind != NH_SOLVER_CG) continue;
        const int n = st.n_active;
        const size_t mo = (size_t)b * a.pitch;
        double rz = st.rz, beta = 0.0, rel = 0.0;
        const double bnorm = st.bnorm;
        int status = NH_ERR_NOT_CONVERGED, iters = 0;
        for (int it = 1; it <= a.max_iter; ++it) {
            const T* pold = (it & 1) ? a.p0 : a.p1;
            T* pnew = (it & 1) ? a.p1 : a.p0;
            const T* rold = (it & 1) ? a.r : a.r1;
            T* rnew = (it & 1) ? a.r1 : a.r;
            iters = it;
            for (int k = threadIdx.x; k < n; k += kPcrThreads)
                pnew[mo + k] = a.z[mo + k] + T(beta) * pold[mo + k];
            __syncthreads();
            double v[1] = {0.0};
            for (int k = threadIdx.x; k < n; k += kPcrThreads) {
                const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
                const T pk = pnew[mo + k];
                const T pl = kl >= 0 ? pnew[mo + kl] : T(0);
                const T pr = kr >= 0 ? pnew[mo + kr] : T(0);
                T qk = apply_row(a, mo, k, pk, pl, pr);
                if (a.n_ext) qk += ext_terms(a, mo, k, [&](int j) { return pnew[mo + j]; });
                a.q[mo + k] = qk;
                v[0] += (double)pk * (double)qk;
            }
            block_sum<1>(v, red);
            if (threadIdx.x == 0) s_bc[0] = v[0];
            __syncthreads();
            const double spq = s_bc[0];
            if (!isfinite(spq) || !(spq > 0.0)) { status = kBreakdown; break; }
            const T alpha = T(rz / spq);
            double acc[3] = {0.0, 0.0, 0.0};
            for (int k = threadIdx.x; k < n; k += kPcrThreads) {
                a.x[mo + k] = a.x[mo + k] + alpha * pnew[mo + k];
                const T rk = rold[mo + k] - alpha * a.q[mo + k];
                rnew[mo + k] = rk;
                acc[2] += (double)rk * (double)rk;
                sd[k] = TP(rk);
            }
            __syncthreads();
            const TP* red_d = pcr_apply<T, TP>(a, sd, sa, n, mo);
            for (int k = threadIdx.x; k < n; k += kPcrThreads) {
                const T zk = T(red_d[k] * TP(a.prb[mo + k]));
                a.z[mo + k] = zk;
                acc[0] += (double)zk * (double)rnew[mo + k];
                acc[1] += (double)zk * (double)rold[mo + k];
            }
            block_sum<3>(acc, red);
            if (threadIdx.x == 0) { s_bc[1] = acc[0]; s_bc[2] = acc[1]; s_bc[3] = acc[2]; }
            __syncthreads();
            const double zr = s_bc[1], zro = s_bc[2], rr = s_bc[3];
            if (!isfinite(rr)) { status = NH_ERR_NONFINITE; rel = NAN; break; }
            rel = sqrt(rr) / bnorm;
            if (sqrt(rr) <= a.rtol * bnorm) { status = NH_OK; break; }
            if (it >= a.max_iter) { status = NH_ERR_NOT_CONVERGED; break; }
            if (!isfinite(zr) || !(zr > 0.0)) { status = kBreakdown; break; }
            beta = (zr - zro) / rz;
            rz = zr;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            if (status == kBreakdown) {
                cg_breakdown<T>(st, a.ctl, iters);
            } else {
                st.beta = beta; st.rz = rz;
                finish_member<T>(st, a.ctl, status, iters, rel);
            }
        }
        __syncthreads();
    }
}

// All PCG iterations of one solve in one cooperative launch: per iteration
// phase A (p = z + beta p_old, q = A p, partial <p, q>) and phase B (alpha,
// x, r update, ||r||, line preconditioner, beta), separated by grid barriers.
// Phase A is spread over every CTA in kChunk-row work items (one row per
// thread, kPcrThreads / kChunk items per CTA pass), so a small active set
// still uses the whole GPU; its partials go to the fourth partial slot.
// Phase B works per preconditioner block (kPcrRows active cells, one CTA):
// each block's CTA sums its member's <p, q> partials in a fixed order, so all
// blocks of a member form the same alpha.  Members finish independently; the
// loop ends when no member is left, after max_iter, or when a barrier times
// out (ctl->timeout).
template <typename T, typename TP>
__global__ void __launch_bounds__(kPcrThreads) k_pcg_persistent(SolveArgs<T> a, long long budget)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    TP* sa = reinterpret_cast<TP*>(smem_raw);   // reduction ping-pong buffers
    TP* sd = sa + kPcrRows;
    __shared__ double red[96];
    __shared__ double s_pq;
    __shared__ int s_skip;
    constexpr int kGroups = kPcrThreads / kChunk;
    static_assert(kGroups * kChunk == kPcrThreads, "whole work items per CTA pass");
    const size_t stride = (size_t)a.nb * a.maxch;
    double* part_pq = a.part + 3 * stride;
    const int n_pitems = a.ctl->n_pitems;
    const int n_items = a.ctl->n_items;
    Ctl* ctl = a.ctl;
    const unsigned nblk = gridDim.x;
    if (ctl->max_npb <= 1) {          // the same for every CTA: no grid barrier needed
        pcg_member_local<T, TP>(a, sa, sd, red);
        return;
    }
    const int grp = threadIdx.x / kChunk, lt = threadIdx.x % kChunk;
    for (int it = 1; it <= a.max_iter; ++it) {
        const T* pold = (it & 1) ? a.p0 : a.p1;
        T* pnew = (it & 1) ? a.p1 : a.p0;
        const T* rold = (it & 1) ? a.r : a.r1;
        T* rnew = (it & 1) ? a.r1 : a.r;
        // ---- phase A: kChunk-row items over all CTAs
        for (int u = blockIdx.x; u * kGroups < n_items; u += gridDim.x) {
            const int w = u * kGroups + grp;
            double pq = 0.0;
            bool live = false;
            if (w < n_items) {
                const int2 itm = a.items[w];
                const int b = itm.x;
                if (!a.ms[b].done && a.ms[b].kind == NH_SOLVER_CG) {
                    live = true;
                    const int n = a.ms[b].n_active;
                    const size_t mo = (size_t)b * a.pitch;
                    const int k = itm.y * kChunk + lt;
                    const T beta = (it == 1) ? T(0) : T(a.ms[b].beta);
                    if (k < n) {
                        const int km = k > 0 ? k - 1 : k, kp = k + 1 < n ? k + 1 : k;
                        const T zk = a.z[mo + k], zm = a.z[mo + km], zp = a.z[mo + kp];
                        const T ok = pold[mo + k], om = pold[mo + km], op = pold[mo + kp];
                        const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
                        const T pk = zk + beta * ok;
                        T pl = T(0), pr = T(0);
                        if (kl == k - 1) pl = zm + beta * om;
                        else if (kl >= 0) pl = a.z[mo + kl] + beta * pold[mo + kl];
                        if (kr == k + 1) pr = zp + beta * op;
                        else if (kr >= 0) pr = a.z[mo + kr] + beta * pold[mo + kr];
                        T qk = apply_row(a, mo, k, pk, pl, pr);
                        if (a.n_ext)
                            qk += ext_terms(a, mo, k, [&](int j) { return a.z[mo + j] + beta * pold[mo + j]; });
                        pnew[mo + k] = pk;
                        a.q[mo + k] = qk;
                        pq = (double)pk * (double)qk;
                    }
                }
            }
            // per-item sum in a fixed order: warps, then the item's warps
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) pq += __shfl_down_sync(0xffffffffu, pq, o);
            if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = pq;
            __syncthreads();
            if (lt == 0 && live) {
                double t = 0.0;
                for (int q = 0; q < kChunk / 32; ++q) t += red[grp * (kChunk / 32) + q];
                part_pq[w] = t;
            }
            __syncthreads();
        }
        if (!grid_barrier(ctl, nblk, budget, [] {})) return;
        // ---- phase B: one preconditioner block per CTA
        for (int wi = blockIdx.x; wi < n_pitems; wi += gridDim.x) {
            const int2 itm = a.pitems[wi];
            const int b = itm.x, jb = itm.y;
            if (threadIdx.x == 0) s_skip = a.ms[b].done || a.ms[b].kind != NH_SOLVER_CG;
            __syncthreads();
            if (s_skip) continue;
            const int n = a.ms[b].n_active, npb = a.ms[b].npb, poff = a.ms[b].poff;
            const int nch = a.ms[b].nchunks, ioff = a.ms[b].ioff;
            const double spq0 = member_sum(part_pq + ioff, nch, red);
            if (threadIdx.x == 0) s_pq = spq0;
            __syncthreads();
            const double spq = s_pq;
            if (!isfinite(spq) || !(spq > 0.0)) {   // the same decision in every block of the member
                if (jb == 0 && threadIdx.x == 0) cg_breakdown<T>(a.ms[b], ctl, it);
                __syncthreads();
                continue;
            }
            const size_t mo = (size_t)b * a.pitch;
            const int k0 = jb * kPcrRows, rows = min(kPcrRows, n - k0);
            const T alpha = T(a.ms[b].rz / spq);
            const T* __restrict__ pb = pnew + mo + k0;
            const T* __restrict__ qb = a.q + mo + k0;
            const T* __restrict__ rob = rold + mo + k0;
            T* __restrict__ xb = a.x + mo + k0;
            T* __restrict__ rnb = rnew + mo + k0;
            double ss = 0.0;
#pragma unroll
            for (int m = 0; m < kPcrRows / kPcrThreads; ++m) {
                const int i = threadIdx.x + m * kPcrThreads;
                if (i < rows) {
                    xb[i] = xb[i] + alpha * pb[i];
                    const T rk = rob[i] - alpha * qb[i];
                    rnb[i] = rk;
                    ss += (double)rk * (double)rk;
                    sd[i] = TP(rk);
                }
            }
            __syncthreads();
            const TP* red_d = pcr_apply<T, TP>(a, sd, sa, rows, mo + k0);
            double acc[3] = {0.0, 0.0, ss};
            const float* __restrict__ prb = a.prb + mo + k0;
            T* __restrict__ zb = a.z + mo + k0;
#pragma unroll
            for (int m = 0; m < kPcrRows / kPcrThreads; ++m) {
                const int i = threadIdx.x + m * kPcrThreads;
                if (i < rows) {
                    const T zk = T(red_d[i] * TP(prb[i]));
                    zb[i] = zk;
                    acc[0] += (double)zk * (double)rnb[i];
                    acc[1] += (double)zk * (double)rob[i];
                }
            }
            block_sum<3>(acc, red);
            if (threadIdx.x == 0) {
                a.part[wi] = acc[0]; a.part[stride + wi] = acc[1]; a.part[2 * stride + wi] = acc[2];
            }
            if (arrive_last(a.cnt, b, npb)) {
                double sums[3];
                member_sum3(a.part + poff, stride, npb, red, sums);
                const double zr = sums[0], zro = sums[1], rr = sums[2];
                if (threadIdx.x == 0) {
                    MState& st = a.ms[b];
                    st.alpha = (double)alpha;
                    const double rel = sqrt(rr) / st.bnorm;
                    if (!isfinite(rr)) finish_member<T>(st, ctl, NH_ERR_NONFINITE, it, NAN);
                    else if (sqrt(rr) <= a.rtol * st.bnorm) finish_member<T>(st, ctl, NH_OK, it, rel);
                    else if (it >= a.max_iter) finish_member<T>(st, ctl, NH_ERR_NOT_CONVERGED, it, rel);
                    else if (!isfinite(zr) || !(zr > 0.0)) cg_breakdown<T>(st, ctl, it);
                    else { st.beta = (zr - zro) / st.rz; st.rz = zr; st.rr = rr; }
                }
            }
        }
        const int par = it & 1;
        if (!grid_barrier(ctl, nblk, budget, [ctl, par] {
                ctl->go[par] = (*(volatile int*)&ctl->not_done) > 0;
            }))
            return;
        if (*(volatile int*)&ctl->go[par] == 0) return;
    }
}

// Preconditioned (right) BiCGStab.  Per iteration: k_pcr(PCR_BI_P) forms
// p = r + beta (p - omega v) and p-hat = M^{-1} p; k_pbi_mv(0) v = A p-hat,
// alpha = rho / <rh, v>; k_pcr(PCR_BI_S) forms s = r - alpha v, s-hat =
// M^{-1} s and tests ||s||; k_pbi_mv(1) t = A s-hat, omega = <t,s>/<t,t>;
// k_pbi_upd x += alpha p-hat + omega s-hat, r = s - omega t, tests ||r||.
template <typename T>
__global__ void __launch_bounds__(kChunk) k_pbi_mv(SolveArgs<T> a, int which)
{
    __shared__ double red[64];
    const int it = a.it;
    const T* xin = which == 0 ? a.p1 : a.z;        // p-hat or s-hat
    T* yout = which == 0 ? a.v0 : a.t;             // v or t
    const size_t stride = (size_t)a.nb * a.maxch;
    NH_FOR_ITEMS(a)
        if (a.ms[b].done || a.ms[b].kind != NH_SOLVER_BICGSTAB) continue;
        if (which == 1 && a.ms[b].s_conv) continue;
        double acc[2] = {0.0, 0.0};
        if (in) {
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            const T xk = xin[mo + k];
            const T xl = kl >= 0 ? xin[mo + kl] : T(0);
            const T xr = kr >= 0 ? xin[mo + kr] : T(0);
            T yk = apply_row(a, mo, k, xk, xl, xr);
            if (a.n_ext) yk += ext_terms(a, mo, k, [&](int j) { return xin[mo + j]; });
            yout[mo + k] = yk;
            if (which == 0) {
                acc[0] = (double)a.rh[mo + k] * (double)yk;
            } else {
                const double sk = (double)a.s[mo + k];
                acc[0] = (double)yk * sk;
                acc[1] = (double)yk * (double)yk;
            }
        }
        block_sum<2>(acc, red);
        if (threadIdx.x == 0) { a.part[wi] = acc[0]; a.part[stride + wi] = acc[1]; }
        if (arrive_last(a.cnt, b, nch)) {
            const size_t mb = ioff;
            const double s0 = member_sum(a.part + mb, nch, red);
            const double s1 = which == 1 ? member_sum(a.part + stride + mb, nch, red) : 0.0;
            if (threadIdx.x == 0) {
                MState& s = a.ms[b];
                if (which == 0) {
                    if (!isfinite(s0) || s0 == 0.0) finish_member<T>(s, a.ctl, NH_ERR_NONFINITE, it, NAN);
                    else s.alpha = s.rr / s0;
                } else {
                    if (!isfinite(s1) || s1 == 0.0) finish_member<T>(s, a.ctl, NH_ERR_NONFINITE, it, NAN);
                    else s.omega = s0 / s1;
                }
            }
        }
    NH_END_ITEMS
}

template <typename T>
__global__ void __launch_bounds__(kChunk) k_pbi_upd(SolveArgs<T> a)
{
    __shared__ double red[64];
    const int it = a.it;
    const size_t stride = (size_t)a.nb * a.maxch;
    NH_FOR_ITEMS(a)
        if (a.ms[b].done || a.ms[b].kind != NH_SOLVER_BICGSTAB) continue;
        const T alpha = T(a.ms[b].alpha), omega = T(a.ms[b].omega);
        const bool sconv = a.ms[b].s_conv != 0;
        double acc[2] = {0.0, 0.0};
        if (in) {
            if (sconv) {
                a.x[mo + k] = a.x[mo + k] + alpha * a.p1[mo + k];
            } else {
                a.x[mo + k] = a.x[mo + k] + alpha * a.p1[mo + k] + omega * a.z[mo + k];
                const T rk = a.s[mo + k] - omega * a.t[mo + k];
                a.r[mo + k] = rk;
                acc[0] = (double)rk * (double)rk;
                acc[1] = (double)a.rh[mo + k] * (double)rk;
            }
        }
        block_sum<2>(acc, red);
        if (threadIdx.x == 0) { a.part[wi] = acc[0]; a.part[stride + wi] = acc[1]; }
        if (arrive_last(a.cnt, b, nch)) {
            const size_t mb = ioff;
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

// Members whose CG broke down restart as BiCGStab members.
static __global__ void k_fallback_reset(MState* ms, int nb)
{
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= nb) return;
    MState& s = ms[b];
    if (s.status == kStatusFallback) {
        s.status = NH_OK; s.done = 0; s.kind = NH_SOLVER_BICGSTAB; s.s_conv = 0;
        s.alpha = 1.0; s.beta = 0.0; s.omega = 1.0;
    }
}

// ------------------------------------------------------------- correction

struct ClearArgs {
    int nb, pitch, maxlist;
    const int* list_prev;
    const int* nact_prev;
    double* psi;
    const TimeCtl* tc;
};

// Zero the dense pressure unknown on the previous step's active cells.
static __global__ void k_clear_prev(ClearArgs a)
{
    if (a.tc && a.tc->abort) return;
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
    const double* x;       // psi on active cells (FP64)
    const T* c6; const T* cx; const T* phi; const T* ddx;
    const MState* ms;
    T* hu; T* hw;          // Q~ buffers, corrected in place into Q^{n+1}
    double* psi;           // dense pressure unknown (for the next warm start)
    const int2* items; const Ctl* ctl;
    const TimeCtl* tc;
};

// Eqs. 10-11 on the active cells (h is not corrected, Sec. 3.2).
template <typename T>
__global__ void __launch_bounds__(kChunk) k_correct(CorrArgs<T> a)
{
    if (a.tc && a.tc->abort) return;
    const int n_items = a.ctl->n_items;
    for (int wi = blockIdx.x; wi < n_items; wi += gridDim.x) {
        const int2 itm = a.items[wi];
        const int b = itm.x, j = itm.y;
        const MState& s = a.ms[b];
        const int n = s.n_active;
        const size_t mo = (size_t)b * a.pitch;
        const int k = j * kChunk + threadIdx.x;
        if (k >= n) continue;
        const bool zero = s.zero_sol != 0;
        const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
        const double ps = zero ? 0.0 : a.x[mo + k];
        const double pl = (zero || kl < 0) ? 0.0 : a.x[mo + kl];
        const double pr = (zero || kr < 0) ? 0.0 : a.x[mo + kr];
        const T ps_x = T((pr - pl) / (2.0 * a.dx));
        const T P = a.c6[mo + k] * T(ps) + a.cx[mo + k] * ps_x + a.phi[mo + k];
        const int i = a.list[mo + k];
        a.hu[mo + i] = a.hu[mo + i] - ps_x + a.ddx[mo + k] * P;
        a.hw[mo + i] = a.hw[mo + i] + P;
        a.psi[mo + i] = ps;
    }
}

static __global__ void k_fill(double* __restrict__ a, double v, size_t n)
{
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        a[q] = v;
}

// dst[b * pitch + i] = src[off[b] + i] for i < off[b+1] - off[b]
static __global__ void k_scatter(const double* __restrict__ src, double* __restrict__ dst, int pitch,
                                 const long long* __restrict__ off)
{
    const int b = blockIdx.y;
    const long long o0 = off[b], n = off[b + 1] - o0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[(size_t)b * pitch + i] = src[o0 + i];
}

static __global__ void k_to_float(const double* __restrict__ a, float* __restrict__ b, size_t n)
{
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (size_t)gridDim.x * blockDim.x)
        b[q] = (float)a[q];
}

// zeta = h - d0 from an FP64 host-layout staging array (pitched), and back.
template <typename T>
__global__ void k_state_in(const double* __restrict__ h, const double* __restrict__ hu,
                           const double* __restrict__ hw, const double* __restrict__ d0,
                           T* z, T* tu, T* tw, int nb, int pitch, const long long* __restrict__ off)
{
    // host layout: member b occupies [off[b], off[b+1]) of the concatenated arrays
    const int b = blockIdx.y;
    const long long o0 = off[b], nxb = off[b + 1] - o0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nxb;
         i += (long long)gridDim.x * blockDim.x) {
        const long long q = o0 + i;
        const size_t o = (size_t)b * pitch + i;
        z[o] = T(h[q] - d0[o]);
        tu[o] = T(hu[q]);
        tw[o] = T(hw[q]);
    }
}

template <typename T>
__global__ void k_state_out(const T* __restrict__ z, const T* __restrict__ tu, const T* __restrict__ tw,
                            const double* __restrict__ d0, const double* __restrict__ psi,
                            double* h, double* hu, double* hw, double* p, double rho_over_dt,
                            int nb, int pitch, const long long* __restrict__ off)
{
    const int b = blockIdx.y;
    const long long o0 = off[b], nxb = off[b + 1] - o0;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < nxb;
         i += (long long)gridDim.x * blockDim.x) {
        const long long q = o0 + i;
        const size_t o = (size_t)b * pitch + i;
        const double hh = (double)z[o] + d0[o];
        h[q] = hh;
        hu[q] = (double)tu[o];
        hw[q] = (double)tw[o];
        p[q] = rho_over_dt * psi[o] / hh;
    }
}

// ------------------------------------------------ mixed precision: refinement

// Outer (FP64) iterate of the mixed path.  k_ir_resid computes
// r64 = R - A x64 in FP64 on the active cells (x64 gathered from the previous
// pressure at pass 0), tests ||r64|| <= rtol ||R||, and hands r64 rounded to
// FP32 to the inner FP32 Krylov solve as its right-hand side.
struct IRState {
    double bnorm64;
    double rel;
    int done;
    int passes;
    int status;
    int iters;          // inner Krylov iterations summed over passes
};

struct IRArgs {
    int nb, pitch, maxch;
    const int* list; const int* nbl; const int* nbr;
    const double* diag; const double* offl; const double* offr; const double* R;
    const double* psi_prev; double guess_scale;
    double* x64;
    const float* e32;       // inner solution
    float* rhs32;           // inner right-hand side
    MState* ms; IRState* ir; Ctl* ctl;
    double* part; int* cnt;
    double rtol;
    int pass;               // 0: x64 = warm start; >0: after k_ir_update
    int ir_max;
    const int2* items;
};

static __global__ void __launch_bounds__(kChunk) k_ir_resid(IRArgs a)
{
    __shared__ double red[64];
    const size_t stride = (size_t)a.nb * a.maxch;
    const int n_items = a.ctl->n_items;
    for (int wi = blockIdx.x; wi < n_items; wi += gridDim.x) {
        const int2 itm = a.items[wi];
        const int b = itm.x, j = itm.y;
        const int nch = a.ms[b].nchunks;
        const int ioff = a.ms[b].ioff;
        if (a.pass > 0 && a.ir[b].done) continue;
        const int n = a.ms[b].n_active;
        const size_t mo = (size_t)b * a.pitch;
        const int k = j * kChunk + threadIdx.x;
        double acc[2] = {0.0, 0.0};
        if (k < n) {
            const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
            double xk = 0.0, xl = 0.0, xr = 0.0;
            if (a.pass == 0) {
                const double sc = a.guess_scale;
                if (sc != 0.0) {
                    xk = a.psi_prev[mo + a.list[mo + k]] * sc;
                    if (kl >= 0) xl = a.psi_prev[mo + a.list[mo + kl]] * sc;
                    if (kr >= 0) xr = a.psi_prev[mo + a.list[mo + kr]] * sc;
                }
                a.x64[mo + k] = xk;
            } else {
                xk = a.x64[mo + k];
                if (kl >= 0) xl = a.x64[mo + kl];
                if (kr >= 0) xr = a.x64[mo + kr];
            }
            const double rk = a.R[mo + k] - (a.diag[mo + k] * xk + a.offl[mo + k] * xl + a.offr[mo + k] * xr);
            const float rf = (float)rk;
            a.rhs32[mo + k] = rf;
            acc[0] = rk * rk;
            acc[1] = (double)rf * (double)rf;
        }
        block_sum<2>(acc, red);
        if (threadIdx.x == 0) { a.part[wi] = acc[0]; a.part[stride + wi] = acc[1]; }
        if (arrive_last(a.cnt, b, nch)) {
            const size_t mb = ioff;
            const double rr = member_sum(a.part + mb, nch, red);
            const double rr32 = member_sum(a.part + stride + mb, nch, red);
            if (threadIdx.x == 0) {
                IRState& q = a.ir[b];
                MState& s = a.ms[b];
                if (a.pass == 0) {
                    q.bnorm64 = s.bnorm; q.done = 0; q.passes = 0; q.status = NH_OK; q.iters = 0;
                } else {
                    q.iters += s.iters;
                    if (s.status == NH_ERR_NONFINITE) q.status = NH_ERR_NONFINITE;
                }
                q.passes = a.pass;
                const double rel = q.bnorm64 > 0.0 ? sqrt(rr) / q.bnorm64 : 0.0;
                q.rel = rel;
                bool fin = true;
                if (q.bnorm64 == 0.0) { s.zero_sol = 1; q.rel = 0.0; }
                else if (q.status != NH_OK) { }
                else if (!isfinite(rr)) q.status = NH_ERR_NONFINITE;
                else if (sqrt(rr) <= a.rtol * q.bnorm64) { }
                else if (a.pass >= a.ir_max) q.status = NH_ERR_NOT_CONVERGED;
                else fin = false;
                if (fin) {
                    q.done = 1;
                    s.done = 1; s.status = q.status; s.rel_res = q.rel; s.iters = q.iters;
                } else {
                    // set up the next inner FP32 solve: right-hand side rhs32
                    s.bnorm2 = rr32; s.bnorm = sqrt(rr32); s.done = 0; s.iters = 0;
                    s.status = NH_OK; s.s_conv = 0; s.rel_res = 0.0;
                    atomicAdd(&a.ctl->ir_pending, 1);
                }
            }
        }
    }
}

// x64 += e32 on the active cells of members that ran an inner solve in this
// pass (those not yet done after the previous residual).
static __global__ void k_ir_update(IRArgs a)
{
    const size_t total = (size_t)a.nb * a.pitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
         q += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(q / a.pitch), k = (int)(q - (size_t)b * a.pitch);
        if (!a.ir[b].done && k < a.ms[b].n_active) a.x64[q] += (double)a.e32[q];
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

// Captured runs: accept the step (advance the device time) or abort the run.
static __global__ void k_commit(const Summary* __restrict__ S, TimeCtl* tc)
{
    if (threadIdx.x != 0 || blockIdx.x != 0 || tc->abort) return;
    if (S->status == NH_OK) {
        tc->n += 1;
        tc->done += 1;
        tc->prev_ok = 1;
        tc->iters_total += S->iters;
        tc->active_total += S->n_active;
    } else {
        tc->abort = 1;
        tc->fail_status = S->status;
    }
}

static __global__ void k_summary(const MState* ms, int nb, const double* mass_part, int nparts, double dx,
                          Summary* out, const TimeCtl* tc)
{
    if (tc && tc->abort) return;
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
