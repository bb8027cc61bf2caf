// nh_mg2d.cuh -- conjugate gradients preconditioned by an aggregation
// multigrid V-cycle, for the 2D elliptic problem -div(K grad psi) + gamma psi
// = R on each member's active cells (the symmetric 9-point rows k2_assemble
// writes; a5 on 2D grids).
//
// Levels.  Level 0 is the member's compact list of active cells.  Coarse level
// l >= 1 holds the aggregates (I, J) = (i >> l, j >> l) of the fine cells
// (i, j) inside the bounding box of the active cells, stored densely row by
// row; an aggregate with no active fine cell is an empty row (all values zero
// and never updated).  The operator of level l is the Galerkin product
// P^T A P with piecewise-constant prolongation P: coarse row (I, J) sums the
// rows of its (at most four) children, each coupling entered in the slot of
// the aggregate its column falls into.  Every coarse row is gathered by one
// thread in a fixed order (no atomics), so the set-up is deterministic.  A
// symmetric A gives a symmetric 9-point coarse operator; periodic sides whose
// whole extent is active wrap modulo the level's width.
//
// V-cycle (FP32, symmetric, so the preconditioner is a fixed SPD operator up
// to rounding): on every level above the coarsest one damped-Jacobi sweep
// from zero, the residual restricted to the next level by summing the
// children; on the coarsest level kMgSweeps damped-Jacobi sweeps; on the way
// up the coarse correction is added to every child and one damped-Jacobi
// sweep follows.
//
// Outer iteration (FP64 vectors and reductions): PCG with the flexible
// (Polak-Ribiere) beta = (<z, r_new> - <z, r_old>) / <z_old, r_old>, which
// tolerates the FP32 rounding of the preconditioner; the same convergence
// test as the line-preconditioned solve (||r|| <= rtol ||R||).
//
// Work split.  Members are independent: each runs on a group of CTAs of one
// cooperative launch (k2_mg_assign gives a member more CTAs the more active
// cells it has, one CTA for small members).  A one-CTA group synchronises
// with __syncthreads; larger groups with a bounded barrier on a per-member
// counter in global memory (NH_ERR_TIMEOUT when it gives up).  Group sums are
// formed per CTA and then added in CTA order, identically in every CTA of the
// group, so all of them take the same decisions.
#pragma once

#include "nh_kernels2d.cuh"

namespace nh {

constexpr int kMgThreads = 1024;     // threads per CTA of the multigrid solve
constexpr int kMgLevels = 12;        // coarse levels at most
constexpr int kMgCoarsest = 16;      // a level of at most this many cells is the coarsest
constexpr int kMgSweeps = 7;         // damped-Jacobi sweeps on the coarsest level (odd)
constexpr int kMgRowsPerCta = 4096;  // active cells per CTA before a member gets another one
constexpr float kMgOmega = 0.7f;     // Jacobi damping

// Coarse level of one member: box origin (level coordinates) and size; wx / wy
// set when the box spans a periodic extent (neighbours wrap modulo w / h);
// off = first cell of the level in the member's coarse region.
struct MgLev {
    int i0, j0, w, h;
    int wx, wy, off, pad;
};

struct MgPlan {
    int nlev;                 // coarse levels (0: the fine smoother alone)
    int bi0, bi1, bj0, bj1;   // bounding box of the active cells (fine)
    int pad[3];
    MgLev lev[kMgLevels + 1];
};

struct MgJob {
    int b, rank, gsize, pad;
};

struct MgArgs {
    SolveArgs<double> s;      // outer PCG: vectors, fine rows, member state, controls
    const Geo2* geos;
    const int* inv;           // dense cell -> compact index (or -1), [nb * pitch]
    MgPlan* plan;             // [nb]
    const MgJob* jobs;        // [njobs]
    const int* njobs;
    unsigned* gbar;           // [2 * nb]: group barrier arrivals, generation
    double* gpart;            // [8 * coop grid]: group partial sums (two buffers of 4 per CTA)
    float* cf;                // [10][T]: fine FP32 rows (slots 0-8) and omega / diagonal (slot 9)
    float* z0;                // [T] fine pre-smoothed iterate
    float* t0;                // [T] fine residual
    float* cc;                // [10][CT]: coarse rows and omega / diagonal
    float* cb;                // [CT] coarse right-hand sides
    float* cza;               // [CT] coarse pre-smoothed iterates
    float* czb;               // [CT] coarse post-smoothed iterates
    float* ct;                // [CT] coarse residuals
    size_t T, CT;             // nb * pitch, nb * cpitch
    int cpitch;
    long long budget;         // group-barrier spin limit (clock cycles)
};

// Stencil slots: s = (dy + 1) * 3 + (dx + 1).
__device__ __forceinline__ int slot_dx(int s) { return s % 3 - 1; }
__device__ __forceinline__ int slot_dy(int s) { return s / 3 - 1; }

// Offset of a coarse neighbour reduced into {-1, 0, 1}: modulo the width w
// when the level wraps (any representative for w <= 2; the matvec wraps the
// same way), else as is.
__device__ __forceinline__ int wrap_off(int o, int w, int wrap)
{
    if (!wrap) return o;
    o %= w;
    if (o < 0) o += w;
    if (o == 0) return 0;
    if (o == 1) return 1;
    return -1;   // o == w - 1
}

// Compact indices of the 8 neighbours of fine row o (slot 4 = itself, unused).
__device__ __forceinline__ void fine_nbrs(const SolveArgs<double>& a, size_t o, int (&nk)[9])
{
    const size_t es = a.ext_stride;
    nk[3] = a.nbl[o];
    nk[5] = a.nbr[o];
    nk[1] = a.ext_k[o];
    nk[7] = a.ext_k[es + o];
    nk[0] = a.ext_k[2 * es + o];
    nk[2] = a.ext_k[3 * es + o];
    nk[6] = a.ext_k[4 * es + o];
    nk[8] = a.ext_k[5 * es + o];
    nk[4] = -1;
}

// ---------------------------------------------------------------- planning

// Bounding box of each member's active cells and its coarse levels (one CTA
// per member, after the compaction).
static __global__ void __launch_bounds__(1024) k2_mg_box(const Geo2* __restrict__ geos, const MState* __restrict__ ms,
                                                         const int* __restrict__ list, int pitch, MgPlan* plan)
{
    __shared__ int s_min[32], s_max[32];
    const int b = blockIdx.x;
    const int n = ms[b].n_active;
    const Geo2 G = geos[b];
    const int* L = list + (size_t)b * pitch;
    int lo = 1 << 30, hi = -1;
    for (int k = threadIdx.x; k < n; k += blockDim.x) {
        const int i = L[k] % G.nx;
        lo = min(lo, i);
        hi = max(hi, i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) { s_min[threadIdx.x >> 5] = lo; s_max[threadIdx.x >> 5] = hi; }
    __syncthreads();
    if (threadIdx.x != 0) return;
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) { lo = min(lo, s_min[w]); hi = max(hi, s_max[w]); }
    MgPlan P;
    P.nlev = 0;
    P.bi0 = P.bi1 = P.bj0 = P.bj1 = 0;
    P.pad[0] = P.pad[1] = P.pad[2] = 0;
    if (n > 0) {
        P.bi0 = lo; P.bi1 = hi;
        P.bj0 = L[0] / G.nx; P.bj1 = L[n - 1] / G.nx;
        const int wx = (G.bcx == NH_BC_PERIODIC && lo == 0 && hi == G.nx - 1);
        const int wy = (G.bcy == NH_BC_PERIODIC && P.bj0 == 0 && P.bj1 == G.ny - 1);
        long long prev = (long long)(hi - lo + 1) * (P.bj1 - P.bj0 + 1);
        int off = 0;
        for (int l = 1; l <= kMgLevels && prev > kMgCoarsest; ++l) {
            MgLev v;
            v.i0 = lo >> l; v.j0 = P.bj0 >> l;
            v.w = (hi >> l) - v.i0 + 1; v.h = (P.bj1 >> l) - v.j0 + 1;
            v.wx = wx; v.wy = wy; v.off = off; v.pad = 0;
            const long long area = (long long)v.w * v.h;
            if (area >= prev) break;
            P.lev[l] = v;
            P.nlev = l;
            off += (int)area;
            prev = area;
        }
    }
    plan[b] = P;
}

// Work split of the multigrid solve over the cooperative grid: members still
// solving with CG each get one CTA; when they are fewer than the grid, the
// spare CTAs go to members in proportion to their active cells, at most one
// per kMgRowsPerCta cells.  Job j runs on CTA j (or, with more members than
// CTAs, CTA j mod grid).  One CTA.
static __global__ void __launch_bounds__(1024) k2_mg_assign(const MState* __restrict__ ms, int nb, int grid,
                                                            MgJob* jobs, int* njobs)
{
    __shared__ long long s_tot[32];
    __shared__ int s_cnt[32];
    __shared__ int s_w[32];
    __shared__ int s_base;
    __shared__ long long s_total;
    __shared__ int s_nne;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5, nw = blockDim.x >> 5;
    long long tot = 0;
    int cnt = 0;
    for (int b = tid; b < nb; b += blockDim.x) {
        const MState& s = ms[b];
        if (!s.done && s.kind == NH_SOLVER_CG) { tot += s.n_active; cnt += 1; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        tot += __shfl_xor_sync(0xffffffffu, tot, o);
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    }
    if (lane == 0) { s_tot[wid] = tot; s_cnt[wid] = cnt; }
    __syncthreads();
    if (tid == 0) {
        long long t = 0;
        int c = 0;
        for (int w = 0; w < nw; ++w) { t += s_tot[w]; c += s_cnt[w]; }
        s_total = t; s_nne = c; s_base = 0;
    }
    __syncthreads();
    const long long total = s_total;
    const int nne = s_nne;
    const int spare = nne < grid ? grid - nne : 0;
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int b = b0 + tid;
        int gs = 0;
        if (b < nb && !ms[b].done && ms[b].kind == NH_SOLVER_CG) {
            const int n = ms[b].n_active;
            gs = 1;
            if (spare > 0 && total > 0) {
                const long long extra = (long long)spare * n / total;
                const int cap = max(1, (n + kMgRowsPerCta - 1) / kMgRowsPerCta);
                gs = (int)min((long long)cap, 1 + extra);
            }
        }
        int incl = gs;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        if (lane == 31) s_w[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            int x = lane < nw ? s_w[lane] : 0;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            s_w[lane] = x;
        }
        __syncthreads();
        const int first = s_base + incl - gs + (wid > 0 ? s_w[wid - 1] : 0);
        for (int r = 0; r < gs; ++r) jobs[first + r] = MgJob{b, r, gs, 0};
        __syncthreads();
        if (tid == 0) s_base += s_w[nw - 1];
        __syncthreads();
    }
    if (tid == 0) *njobs = s_base;
}

// ------------------------------------------------------------ group helpers

struct MgGroup {
    int b, rank, G;
    int base;                 // first CTA of the group (partials slot)
    int phase;                // alternates the partials buffer of successive sums
    unsigned* cnt;
    unsigned* gen;
};

// Barrier of the member's CTAs; false when the bounded wait gave up.
__device__ __forceinline__ bool mg_sync(const MgGroup& g, long long budget, Ctl* ctl)
{
    if (g.G == 1) {
        __syncthreads();
        return true;
    }
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned* gen = g.gen;
        const unsigned g0 = *gen;
        __threadfence();
        const unsigned arrived = atomicAdd(g.cnt, 1u) + 1u;
        int ok = 1;
        if (arrived == (unsigned)g.G) {
            *g.cnt = 0u;
            __threadfence();
            atomicAdd(g.gen, 1u);
        } else {
            const long long t0 = clock64();
            while (*gen == g0) {
                if (clock64() - t0 > budget) { ok = 0; atomicExch(&ctl->timeout, 1); break; }
                __nanosleep(32);
            }
        }
        __threadfence();
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

// Group sum of NV <= 4 values (every thread receives the sums); false on a
// barrier timeout.  `red` holds 32 * NV doubles, `bc` NV doubles.  Two
// buffers of partials alternate, so a CTA writing the next sum's partials
// cannot overwrite ones another CTA still reads (it passed the barrier in
// between).
template <int NV>
__device__ __forceinline__ bool mg_sum(MgGroup& g, double (&v)[NV], double* red, double* bc, double* gpart,
                                       long long budget, Ctl* ctl)
{
    block_sum<NV>(v, red);
    if (g.G == 1) {
        if (threadIdx.x == 0)
            for (int q = 0; q < NV; ++q) bc[q] = v[q];
        __syncthreads();
    } else {
        double* buf = gpart + 4 * g.phase;
        g.phase ^= 1;
        if (threadIdx.x == 0)
            for (int q = 0; q < NV; ++q) buf[8 * (g.base + g.rank) + q] = v[q];
        if (!mg_sync(g, budget, ctl)) return false;
        if (threadIdx.x == 0) {
            for (int q = 0; q < NV; ++q) {
                double t = 0.0;
                for (int r = 0; r < g.G; ++r) t += __ldcg(buf + 8 * (g.base + r) + q);
                bc[q] = t;
            }
        }
        __syncthreads();
    }
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = bc[q];
    return true;
}

// How the cells of one phase are split: over the whole group, or over the
// CTA of rank 0 alone for small coarse levels (then barriers are block-wide).
struct MgExec {
    int stride, t0;
    bool local;
};

__device__ __forceinline__ bool mg_bar(const MgGroup& g, const MgExec& ex, long long budget, Ctl* ctl)
{
    if (ex.local) {
        __syncthreads();
        return true;
    }
    return mg_sync(g, budget, ctl);
}

// -------------------------------------------------------- level operations

// rhs - (A v)_k on fine row k (FP32), v a fine FP32 vector.
__device__ __forceinline__ float fine_resid(const MgArgs& m, size_t mo, int k, float rhs, const float* v)
{
    const SolveArgs<double>& a = m.s;
    const size_t o = mo + k;
    int nk[9];
    fine_nbrs(a, o, nk);
    float y = m.cf[4 * m.T + o] * v[o];
#pragma unroll
    for (int s = 0; s < 9; ++s)
        if (s != 4 && nk[s] >= 0) y += m.cf[s * m.T + o] * v[mo + nk[s]];
    return rhs - y;
}

// rhs - (A v) at cell q of a coarse level (local coordinates il, jl).
__device__ __forceinline__ float coarse_resid(const MgArgs& m, const MgLev& L, size_t cbase, int q, float rhs,
                                              const float* v)
{
    const int il = q % L.w, jl = q / L.w;
    const size_t c0 = cbase + L.off;
    float y = 0.f;
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        int ii = il + slot_dx(s), jj = jl + slot_dy(s);
        if (L.wx) ii = (ii + L.w) % L.w;
        else if (ii < 0 || ii >= L.w) continue;
        if (L.wy) jj = (jj + L.h) % L.h;
        else if (jj < 0 || jj >= L.h) continue;
        y += m.cc[s * m.CT + c0 + q] * v[c0 + (size_t)jj * L.w + ii];
    }
    return rhs - y;
}

// Level 1 row of aggregate q: the Galerkin sum of its fine children's rows.
__device__ __forceinline__ void gather_level1(const MgArgs& m, const Geo2& G, const MgLev& L, size_t mo,
                                              size_t cbase, int q)
{
    const SolveArgs<double>& a = m.s;
    const int I = L.i0 + q % L.w, J = L.j0 + q / L.w;
    float acc[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) acc[s] = 0.f;
    bool any = false;
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
            const int i = 2 * I + di, j = 2 * J + dj;
            if (i >= G.nx || j >= G.ny) continue;
            const int k = m.inv[mo + (size_t)j * G.nx + i];
            if (k < 0) continue;
            any = true;
            const size_t o = mo + k;
            int nk[9];
            fine_nbrs(a, o, nk);
            acc[4] += m.cf[4 * m.T + o];
#pragma unroll
            for (int s = 0; s < 9; ++s) {
                if (s == 4 || nk[s] < 0) continue;
                int ii = i + slot_dx(s), jj = j + slot_dy(s);
                if (G.bcx == NH_BC_PERIODIC) ii = (ii + G.nx) % G.nx;
                if (G.bcy == NH_BC_PERIODIC) jj = (jj + G.ny) % G.ny;
                const int ox = wrap_off((ii >> 1) - I, L.w, L.wx);
                const int oy = wrap_off((jj >> 1) - J, L.h, L.wy);
                acc[(oy + 1) * 3 + ox + 1] += m.cf[s * m.T + o];
            }
        }
    const size_t c = cbase + L.off + q;
#pragma unroll
    for (int s = 0; s < 9; ++s) m.cc[s * m.CT + c] = any ? acc[s] : 0.f;
    m.cc[9 * m.CT + c] = (any && acc[4] != 0.f) ? kMgOmega / acc[4] : 0.f;
}

// Level l + 1 row of aggregate q from the dense level l (P: level l, L: level l + 1).
__device__ __forceinline__ void gather_coarse(const MgArgs& m, const MgLev& P, const MgLev& L, size_t cbase, int q)
{
    const int I = L.i0 + q % L.w, J = L.j0 + q / L.w;
    float acc[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) acc[s] = 0.f;
    bool any = false;
    const size_t p0 = cbase + P.off;
    for (int dj = 0; dj < 2; ++dj)
        for (int di = 0; di < 2; ++di) {
            const int ci = 2 * I + di - P.i0, cj = 2 * J + dj - P.j0;   // child, level-l local
            if (ci < 0 || ci >= P.w || cj < 0 || cj >= P.h) continue;
            const size_t pc = p0 + (size_t)cj * P.w + ci;
            if (m.cc[9 * m.CT + pc] == 0.f) continue;   // empty child
            any = true;
#pragma unroll
            for (int s = 0; s < 9; ++s) {
                const float cv = m.cc[s * m.CT + pc];
                if (cv == 0.f) continue;
                int ii = ci + slot_dx(s), jj = cj + slot_dy(s);
                if (P.wx) ii = (ii + P.w) % P.w;
                if (P.wy) jj = (jj + P.h) % P.h;
                const int ox = wrap_off(((ii + P.i0) >> 1) - I, L.w, L.wx);
                const int oy = wrap_off(((jj + P.j0) >> 1) - J, L.h, L.wy);
                acc[(oy + 1) * 3 + ox + 1] += cv;
            }
        }
    const size_t c = cbase + L.off + q;
#pragma unroll
    for (int s = 0; s < 9; ++s) m.cc[s * m.CT + c] = any ? acc[s] : 0.f;
    m.cc[9 * m.CT + c] = (any && acc[4] != 0.f) ? kMgOmega / acc[4] : 0.f;
}

// ------------------------------------------------------------------ V-cycle

// Down the V at coarse level l: right-hand side by summing the children's
// residuals, pre-smoothing from zero, and either the residual for the next
// level or, on the coarsest level, the Jacobi sweeps (result in czb).
__device__ __forceinline__ bool mg_down(const MgArgs& m, const MgGroup& g, const MgExec& ex, const MgPlan& P,
                                        const Geo2& G, int l, size_t mo, size_t cbase)
{
    Ctl* ctl = m.s.ctl;
    const MgLev& L = P.lev[l];
    const int area = L.w * L.h;
    const size_t c0 = cbase + L.off;
    for (int q = ex.t0; q < area; q += ex.stride) {
        const int I = L.i0 + q % L.w, J = L.j0 + q / L.w;
        float bsum = 0.f;
        if (l == 1) {
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    const int i = 2 * I + di, j = 2 * J + dj;
                    if (i >= G.nx || j >= G.ny) continue;
                    const int k = m.inv[mo + (size_t)j * G.nx + i];
                    if (k >= 0) bsum += m.t0[mo + k];
                }
        } else {
            const MgLev& Q = P.lev[l - 1];
            for (int dj = 0; dj < 2; ++dj)
                for (int di = 0; di < 2; ++di) {
                    const int ci = 2 * I + di - Q.i0, cj = 2 * J + dj - Q.j0;
                    if (ci < 0 || ci >= Q.w || cj < 0 || cj >= Q.h) continue;
                    bsum += m.ct[cbase + Q.off + (size_t)cj * Q.w + ci];
                }
        }
        m.cb[c0 + q] = bsum;
        m.cza[c0 + q] = m.cc[9 * m.CT + c0 + q] * bsum;
    }
    if (!mg_bar(g, ex, m.budget, ctl)) return false;
    if (l < P.nlev) {
        for (int q = ex.t0; q < area; q += ex.stride)
            m.ct[c0 + q] = m.cc[9 * m.CT + c0 + q] == 0.f ? 0.f : coarse_resid(m, L, cbase, q, m.cb[c0 + q], m.cza);
        return mg_bar(g, ex, m.budget, ctl);
    }
    // coarsest: kMgSweeps (odd) damped-Jacobi sweeps ping-ponging cza -> czb
    static_assert(kMgSweeps % 2 == 1, "the coarsest result must end in czb");
    float* src = m.cza;
    float* dst = m.czb;
    for (int sw = 0; sw < kMgSweeps; ++sw) {
        for (int q = ex.t0; q < area; q += ex.stride) {
            const float wd = m.cc[9 * m.CT + c0 + q];
            dst[c0 + q] = wd == 0.f ? 0.f : src[c0 + q] + wd * coarse_resid(m, L, cbase, q, m.cb[c0 + q], src);
        }
        if (!mg_bar(g, ex, m.budget, ctl)) return false;
        float* t = src; src = dst; dst = t;
    }
    return true;
}

// Up the V at coarse level l < nlev: the parent's correction, then one sweep into czb.
__device__ __forceinline__ bool mg_up(const MgArgs& m, const MgGroup& g, const MgExec& ex, const MgPlan& P, int l,
                                      size_t cbase)
{
    Ctl* ctl = m.s.ctl;
    const MgLev& L = P.lev[l];
    const MgLev& U = P.lev[l + 1];
    const int area = L.w * L.h;
    const size_t c0 = cbase + L.off;
    for (int q = ex.t0; q < area; q += ex.stride) {
        if (m.cc[9 * m.CT + c0 + q] == 0.f) continue;
        const int I = (L.i0 + q % L.w) >> 1, J = (L.j0 + q / L.w) >> 1;
        m.cza[c0 + q] += m.czb[cbase + U.off + (size_t)(J - U.j0) * U.w + (I - U.i0)];
    }
    if (!mg_bar(g, ex, m.budget, ctl)) return false;
    for (int q = ex.t0; q < area; q += ex.stride) {
        const float wd = m.cc[9 * m.CT + c0 + q];
        m.czb[c0 + q] = wd == 0.f ? 0.f : m.cza[c0 + q] + wd * coarse_resid(m, L, cbase, q, m.cb[c0 + q], m.cza);
    }
    return mg_bar(g, ex, m.budget, ctl);
}

// z = M r on member b's group (r: FP64 fine residual, z: FP64 out).  Levels
// of at most kMgLocal cells run on the group's first CTA alone (block
// barriers) while the others wait at one group barrier.  Returns false on a
// barrier timeout.
constexpr int kMgLocal = 8192;

__device__ bool mg_vcycle(const MgArgs& m, const MgGroup& g, const MgPlan& P, const Geo2& G, int n, size_t mo,
                          size_t cbase, const double* r, double* z)
{
    const SolveArgs<double>& a = m.s;
    Ctl* ctl = a.ctl;
    const MgExec ex{g.G * (int)blockDim.x, g.rank * (int)blockDim.x + (int)threadIdx.x, g.G == 1};
    const MgExec lx{(int)blockDim.x, (int)threadIdx.x, true};
    // fine pre-smoothing from zero and residual
    for (int k = ex.t0; k < n; k += ex.stride) m.z0[mo + k] = m.cf[9 * m.T + mo + k] * (float)r[mo + k];
    if (!mg_sync(g, m.budget, ctl)) return false;
    if (P.nlev > 0) {
        for (int k = ex.t0; k < n; k += ex.stride) m.t0[mo + k] = fine_resid(m, mo, k, (float)r[mo + k], m.z0);
        if (!mg_sync(g, m.budget, ctl)) return false;
        // first level small enough for one CTA
        int lloc = 1;
        if (g.G > 1) {
            lloc = P.nlev + 1;
            for (int l = 1; l <= P.nlev; ++l)
                if (P.lev[l].w * P.lev[l].h <= kMgLocal) { lloc = l; break; }
        }
        for (int l = 1; l < lloc; ++l)
            if (!mg_down(m, g, ex, P, G, l, mo, cbase)) return false;
        if (lloc <= P.nlev) {
            if (g.rank == 0) {
                for (int l = lloc; l <= P.nlev; ++l) mg_down(m, g, lx, P, G, l, mo, cbase);
                for (int l = P.nlev - 1; l >= lloc; --l) mg_up(m, g, lx, P, l, cbase);
            }
            if (!mg_sync(g, m.budget, ctl)) return false;
        }
        for (int l = lloc - 1; l >= 1; --l) {
            if (l == P.nlev) continue;   // the coarsest level has no parent
            if (!mg_up(m, g, ex, P, l, cbase)) return false;
        }
        // fine: coarse correction
        const MgLev& U = P.lev[1];
        for (int k = ex.t0; k < n; k += ex.stride) {
            const int c = a.list[mo + k];
            const int I = (c % G.nx) >> 1, J = (c / G.nx) >> 1;
            m.z0[mo + k] += m.czb[cbase + U.off + (size_t)(J - U.j0) * U.w + (I - U.i0)];
        }
        if (!mg_sync(g, m.budget, ctl)) return false;
    }
    // fine post-smoothing
    for (int k = ex.t0; k < n; k += ex.stride) {
        const float zk = m.z0[mo + k] + m.cf[9 * m.T + mo + k] * fine_resid(m, mo, k, (float)r[mo + k], m.z0);
        z[mo + k] = (double)zk;
    }
    return true;
}

// -------------------------------------------------------------- the solve

// Multigrid set-up and PCG for every member that solves with CG this step
// (after k_solve_init: x = warm start, r = R - A x, p = 0).  Cooperative
// launch of kMgThreads-thread CTAs.
static __global__ void __launch_bounds__(kMgThreads) k2_mg_pcg(MgArgs m)
{
    __shared__ double red[96];
    __shared__ double bc[4];
    __shared__ MgPlan P;
    const SolveArgs<double>& a = m.s;
    Ctl* ctl = a.ctl;
    const int nj = *m.njobs;
    for (int jb = blockIdx.x; jb < nj; jb += gridDim.x) {
        const MgJob job = m.jobs[jb];
        if (threadIdx.x == 0) P = m.plan[job.b];
        __syncthreads();
        MgGroup g;
        g.b = job.b; g.rank = job.rank; g.G = job.gsize; g.base = jb - job.rank; g.phase = 0;
        g.cnt = m.gbar + 2 * job.b; g.gen = m.gbar + 2 * job.b + 1;
        const int b = g.b;
        MState& st = a.ms[b];
        const int n = st.n_active;
        const size_t mo = (size_t)b * a.pitch;
        const size_t cbase = (size_t)b * m.cpitch;
        const Geo2 G = m.geos[b];
        const int stride = g.G * blockDim.x, t0i = g.rank * blockDim.x + threadIdx.x;
        // ---- set-up: FP32 fine rows, then the coarse rows level by level
        for (int k = t0i; k < n; k += stride) {
            const size_t o = mo + k, es = a.ext_stride;
            const double d = a.diag[o];
            m.cf[4 * m.T + o] = (float)d;
            m.cf[3 * m.T + o] = (float)a.offl[o];
            m.cf[5 * m.T + o] = (float)a.offr[o];
            m.cf[1 * m.T + o] = (float)a.ext_c[o];
            m.cf[7 * m.T + o] = (float)a.ext_c[es + o];
            m.cf[0 * m.T + o] = (float)a.ext_c[2 * es + o];
            m.cf[2 * m.T + o] = (float)a.ext_c[3 * es + o];
            m.cf[6 * m.T + o] = (float)a.ext_c[4 * es + o];
            m.cf[8 * m.T + o] = (float)a.ext_c[5 * es + o];
            m.cf[9 * m.T + o] = (float)((double)kMgOmega / d);
        }
        if (!mg_sync(g, m.budget, ctl)) return;
        for (int l = 1; l <= P.nlev; ++l) {
            const MgLev& L = P.lev[l];
            const int area = L.w * L.h;
            for (int q = t0i; q < area; q += stride) {
                if (l == 1) gather_level1(m, G, L, mo, cbase, q);
                else gather_coarse(m, P.lev[l - 1], L, cbase, q);
            }
            if (!mg_sync(g, m.budget, ctl)) return;
        }
        // ---- z = M r, rz = <r, z>
        if (!mg_vcycle(m, g, P, G, n, mo, cbase, a.r, a.z)) return;
        double v1[1] = {0.0};
        for (int k = t0i; k < n; k += stride) v1[0] += a.r[mo + k] * a.z[mo + k];
        if (!mg_sum<1>(g, v1, red, bc, m.gpart, m.budget, ctl)) return;
        double rz = v1[0], beta = 0.0, rel = 0.0;
        const double bnorm = st.bnorm;
        int status = NH_ERR_NOT_CONVERGED, iters = 0;
        bool breakdown = !isfinite(rz) || !(rz > 0.0);
        for (int it = 1; it <= a.max_iter && !breakdown; ++it) {
            const double* pold = (it & 1) ? a.p0 : a.p1;
            double* pnew = (it & 1) ? a.p1 : a.p0;
            const double* rold = (it & 1) ? a.r : a.r1;
            double* rnew = (it & 1) ? a.r1 : a.r;
            iters = it;
            for (int k = t0i; k < n; k += stride) pnew[mo + k] = a.z[mo + k] + beta * pold[mo + k];
            if (!mg_sync(g, m.budget, ctl)) return;
            double vq[1] = {0.0};
            for (int k = t0i; k < n; k += stride) {
                const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
                const double pk = pnew[mo + k];
                const double pl = kl >= 0 ? pnew[mo + kl] : 0.0;
                const double pr = kr >= 0 ? pnew[mo + kr] : 0.0;
                double qk = apply_row(a, mo, k, pk, pl, pr);
                qk += ext_terms(a, mo, k, [&](int j) { return pnew[mo + j]; });
                a.q[mo + k] = qk;
                vq[0] += pk * qk;
            }
            if (!mg_sum<1>(g, vq, red, bc, m.gpart, m.budget, ctl)) return;
            const double pq = vq[0];
            if (!isfinite(pq) || !(pq > 0.0)) { breakdown = true; break; }
            const double alpha = rz / pq;
            for (int k = t0i; k < n; k += stride) {
                a.x[mo + k] += alpha * pnew[mo + k];
                rnew[mo + k] = rold[mo + k] - alpha * a.q[mo + k];
            }
            if (!mg_vcycle(m, g, P, G, n, mo, cbase, rnew, a.z)) return;
            double v3[3] = {0.0, 0.0, 0.0};
            for (int k = t0i; k < n; k += stride) {
                const double zk = a.z[mo + k], rk = rnew[mo + k];
                v3[0] += zk * rk;
                v3[1] += zk * rold[mo + k];
                v3[2] += rk * rk;
            }
            if (!mg_sum<3>(g, v3, red, bc, m.gpart, m.budget, ctl)) return;
            const double zr = v3[0], zro = v3[1], rr = v3[2];
            if (!isfinite(rr)) { status = NH_ERR_NONFINITE; rel = NAN; break; }
            rel = sqrt(rr) / bnorm;
            if (sqrt(rr) <= a.rtol * bnorm) { status = NH_OK; break; }
            if (it >= a.max_iter) { status = NH_ERR_NOT_CONVERGED; break; }
            if (!isfinite(zr) || !(zr > 0.0)) { breakdown = true; break; }
            beta = (zr - zro) / rz;
            rz = zr;
        }
        if (g.rank == 0 && threadIdx.x == 0) {
            if (breakdown) {
                cg_breakdown<double>(st, ctl, iters);
            } else {
                st.beta = beta; st.rz = rz; st.alpha = 0.0;
                finish_member<double>(st, ctl, status, iters, rel);
            }
        }
        __syncthreads();
    }
}

}  // namespace nh
