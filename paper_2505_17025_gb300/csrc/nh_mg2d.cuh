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
constexpr int kMgSweeps = 3;         // damped-Jacobi sweeps on the coarsest level (odd)
constexpr int kMgRowsPerCta = 4096;  // active cells per CTA before a member gets another one
constexpr float kMgOmega = 0.85f;    // Jacobi damping (ensemble: 0.7 -> 30, 0.85 -> 26 PCG iterations per step; 0.95 -> 34, 1.0 fails)
constexpr float kMgCoarseScale = 1.5f;   // weight of the coarse-level correction (over-correction of the piecewise-constant prolongation)
constexpr int kMgSmemCells = 3840;   // coarse cells the group's first CTA keeps in shared memory
constexpr int kMgSmemFloats = 13;    // per such cell: 9 couplings, omega / diagonal, b, two iterates
constexpr size_t kMgSmemBytes = sizeof(float) * kMgSmemFloats * kMgSmemCells;

// Coarse level of one member: box origin (level coordinates) and size; wx / wy
// set when the box spans a periodic extent (neighbours wrap modulo w / h);
// off = first cell of the level in the member's coarse region; soff = its
// first cell in shared memory (levels lloc..nlev), else -1.
struct MgLev {
    int i0, j0, w, h;
    int wx, wy, off, soff;
};

struct MgPlan {
    int nlev;                 // coarse levels (0: the fine smoother alone)
    int lloc;                 // first level kept in shared memory (nlev + 1: none)
    int nloc;                 // cells in shared memory
    int bi0, bi1, bj0, bj1;   // bounding box of the active cells (fine)
    int pad;
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
    int* par;                 // [T] level-1 cell (local index) of each fine row
    float* cc;                // [10][CT]: coarse rows and omega / diagonal
    float* cb;                // [CT] coarse right-hand sides
    float* cza;               // [CT] coarse pre-smoothed iterates
    float* czb;               // [CT] coarse post-smoothed iterates
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
    P.nlev = 0; P.lloc = 1; P.nloc = 0;
    P.bi0 = P.bi1 = P.bj0 = P.bj1 = 0;
    P.pad = 0;
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
            v.wx = wx; v.wy = wy; v.off = off; v.soff = -1;
            const long long area = (long long)v.w * v.h;
            if (area >= prev) break;
            P.lev[l] = v;
            P.nlev = l;
            off += (int)area;
            prev = area;
        }
        // the coarsest levels that fit in shared memory together
        P.lloc = P.nlev + 1;
        long long tot = 0;
        for (int l = P.nlev; l >= 1; --l) {
            tot += (long long)P.lev[l].w * P.lev[l].h;
            if (tot > kMgSmemCells) break;
            P.lloc = l;
        }
        int so = 0;
        for (int l = P.lloc; l <= P.nlev; ++l) {
            P.lev[l].soff = so;
            so += P.lev[l].w * P.lev[l].h;
        }
        P.nloc = so;
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

// -------------------------------------------------------- level operations

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

// A coarse level's arrays, in global memory or in the first CTA's shared
// memory: couplings and omega / diagonal (planes c + s cs), right-hand side,
// pre-smoothed and post-smoothed iterates; box geometry.
struct LView {
    const float* c;
    size_t cs;
    float *b, *za, *zb;
    int i0, j0, w, h, wx, wy;
};

__device__ __forceinline__ LView lview_global(const MgArgs& m, const MgLev& L, size_t cbase)
{
    const size_t o = cbase + L.off;
    return LView{m.cc + o, m.CT, m.cb + o, m.cza + o, m.czb + o, L.i0, L.j0, L.w, L.h, L.wx, L.wy};
}

__device__ __forceinline__ LView lview_smem(float* sm, const MgLev& L)
{
    const size_t S = kMgSmemCells;
    return LView{sm + L.soff, S, sm + 10 * S + L.soff, sm + 11 * S + L.soff, sm + 12 * S + L.soff,
                 L.i0, L.j0, L.w, L.h, L.wx, L.wy};
}

// (A v)_q on a coarse level, v(j, i, jr) the vector at local index j = jr w + i
// (a callable).
template <typename F>
__device__ __forceinline__ float lv_apply(const LView& V, int q, F v)
{
    const int il = q % V.w, jl = q / V.w;
    // every load first (an outside neighbour reads the row's own cell), then
    // the sum over the neighbours inside: the loads overlap instead of
    // waiting on each bounds test
    float c[9], x[9];
    bool in[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        int ii = il + slot_dx(s), jj = jl + slot_dy(s);
        bool ok = true;
        if (V.wx) ii = (ii + V.w) % V.w;
        else ok = ii >= 0 && ii < V.w;
        if (V.wy) jj = (jj + V.h) % V.h;
        else ok = ok && jj >= 0 && jj < V.h;
        if (!ok) { ii = il; jj = jl; }
        in[s] = ok;
        c[s] = V.c[s * V.cs + q];
        x[s] = v(jj * V.w + ii, ii, jj);
    }
    float y = 0.f;
#pragma unroll
    for (int s = 0; s < 9; ++s)
        if (in[s]) y += c[s] * x[s];
    return y;
}

// Local index in U (one level coarser) of V's cell at local (i, jr).
__device__ __forceinline__ int lv_parent(const LView& V, const LView& U, int i, int jr)
{
    return (((V.j0 + jr) >> 1) - U.j0) * U.w + (((V.i0 + i) >> 1) - U.i0);
}

// (A v)_k on fine row k in FP32, v(j) the vector at compact index j.
template <typename F>
__device__ __forceinline__ float fine_apply(const MgArgs& m, size_t mo, int k, F v)
{
    const size_t o = mo + k;
    int nk[9];
    fine_nbrs(m.s, o, nk);
    // all loads first (a missing neighbour reads the row itself), then the sum
    float c[9], x[9];
#pragma unroll
    for (int s = 0; s < 9; ++s) {
        c[s] = m.cf[s * m.T + o];
        x[s] = v(s == 4 || nk[s] < 0 ? k : nk[s]);
    }
    float y = c[4] * x[4];
#pragma unroll
    for (int s = 0; s < 9; ++s)
        if (s != 4 && nk[s] >= 0) y += c[s] * x[s];
    return y;
}

// Level 1 (view V) from the fine level: b = the children's residuals
// r - A z0 summed, za = omega b / diag.
__device__ __forceinline__ void down_fine(const MgArgs& m, const Geo2& G, size_t mo, const double* r,
                                          const LView& V, int t0, int stride)
{
    const float* z0 = m.z0 + mo;
    const int area = V.w * V.h;
    for (int q = t0; q < area; q += stride) {
        const int I = V.i0 + q % V.w, J = V.j0 + q / V.w;
        // the four children's rows (an absent child evaluates row 0, unused):
        // their loads overlap
        int kk[4];
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            const int i = 2 * I + (ch & 1), j = 2 * J + (ch >> 1);
            const bool inb = i < G.nx && j < G.ny;
            const int kv = m.inv[mo + (inb ? (size_t)j * G.nx + i : 0)];
            kk[ch] = inb ? kv : -1;
        }
        float res[4];
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            const int k = kk[ch] >= 0 ? kk[ch] : 0;
            res[ch] = (float)r[mo + k] - fine_apply(m, mo, k, [&](int jj) { return z0[jj]; });
        }
        float bsum = 0.f;
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            if (kk[ch] >= 0) bsum += res[ch];
        V.b[q] = bsum;
        V.za[q] = V.c[9 * V.cs + q] * bsum;
    }
}

// Level V from the finer coarse level U: b = U's residuals summed over the children.
__device__ __forceinline__ void down_coarse(const LView& U, const LView& V, int t0, int stride)
{
    const int area = V.w * V.h;
    for (int q = t0; q < area; q += stride) {
        const int I = V.i0 + q % V.w, J = V.j0 + q / V.w;
        // the four children (an absent or empty one evaluates cell 0, unused)
        float res[4];
        bool use[4];
#pragma unroll
        for (int ch = 0; ch < 4; ++ch) {
            const int ci = 2 * I + (ch & 1) - U.i0, cj = 2 * J + (ch >> 1) - U.j0;
            const bool inb = ci >= 0 && ci < U.w && cj >= 0 && cj < U.h;
            const int c = inb ? cj * U.w + ci : 0;
            use[ch] = inb && U.c[9 * U.cs + c] != 0.f;
            res[ch] = U.b[c] - lv_apply(U, c, [&](int jj, int, int) { return U.za[jj]; });
        }
        float bsum = 0.f;
#pragma unroll
        for (int ch = 0; ch < 4; ++ch)
            if (use[ch]) bsum += res[ch];
        V.b[q] = bsum;
        V.za[q] = V.c[9 * V.cs + q] * bsum;
    }
}

// One damped-Jacobi sweep dst = src + omega (b - A src) / diag.
__device__ __forceinline__ void sweep(const LView& V, const float* src, float* dst, int t0, int stride)
{
    const int area = V.w * V.h;
    for (int q = t0; q < area; q += stride) {
        const float wd = V.c[9 * V.cs + q];
        dst[q] = wd == 0.f ? 0.f : src[q] + wd * (V.b[q] - lv_apply(V, q, [&](int jj, int, int) { return src[jj]; }));
    }
}

// Up at level V (parent level U): y = za + the parent's correction, then one
// sweep into zb, with y formed on the fly at the neighbours.
__device__ __forceinline__ void up_coarse(const LView& V, const LView& U, int t0, int stride)
{
    const int area = V.w * V.h;
    auto y = [&](int j, int i, int jr) { return V.za[j] + kMgCoarseScale * U.zb[lv_parent(V, U, i, jr)]; };
    for (int q = t0; q < area; q += stride) {
        const float wd = V.c[9 * V.cs + q];
        V.zb[q] = wd == 0.f ? 0.f : y(q, q % V.w, q / V.w) + wd * (V.b[q] - lv_apply(V, q, y));
    }
}

// The levels held in the first CTA's shared memory (lloc..nlev), block
// barriers only: level lloc's right-hand side and first iterate (computed
// here from level lloc - 1 or the fine level, or, with `pre`, already formed
// in global memory by the whole group and copied in), the way down, the
// coarsest sweeps, up to lloc; level lloc's result is copied to global memory.
__device__ void mg_local(const MgArgs& m, const MgPlan& P, const Geo2& G, size_t mo, size_t cbase, const double* r,
                         float* sm, bool pre)
{
    const int t0 = threadIdx.x, stride = blockDim.x;
    const int L0 = P.lloc, L1 = P.nlev;
    {
        const LView V = lview_smem(sm, P.lev[L0]);
        if (pre) {
            const LView Vg = lview_global(m, P.lev[L0], cbase);
            for (int q = t0; q < V.w * V.h; q += stride) { V.b[q] = Vg.b[q]; V.za[q] = Vg.za[q]; }
        } else if (L0 == 1) {
            down_fine(m, G, mo, r, V, t0, stride);
        } else {
            down_coarse(lview_global(m, P.lev[L0 - 1], cbase), V, t0, stride);
        }
    }
    __syncthreads();
    for (int l = L0 + 1; l <= L1; ++l) {
        down_coarse(lview_smem(sm, P.lev[l - 1]), lview_smem(sm, P.lev[l]), t0, stride);
        __syncthreads();
    }
    {
        const LView V = lview_smem(sm, P.lev[L1]);
        static_assert(kMgSweeps % 2 == 1, "the coarsest result must end in zb");
        for (int sw = 0; sw < kMgSweeps; ++sw) {
            if (sw % 2 == 0) sweep(V, V.za, V.zb, t0, stride);
            else sweep(V, V.zb, V.za, t0, stride);
            __syncthreads();
        }
    }
    for (int l = L1 - 1; l >= L0; --l) {
        up_coarse(lview_smem(sm, P.lev[l]), lview_smem(sm, P.lev[l + 1]), t0, stride);
        __syncthreads();
    }
    const LView V = lview_smem(sm, P.lev[L0]);
    const LView Vg = lview_global(m, P.lev[L0], cbase);
    for (int q = t0; q < V.w * V.h; q += stride) Vg.zb[q] = V.zb[q];
}

// z = M r on the member's group, given z0 = omega r / diag on the fine rows
// and a group barrier since (r: FP64 fine residual, z: FP64 out).  Returns
// false on a barrier timeout.
__device__ bool mg_vcycle(const MgArgs& m, MgGroup& g, const MgPlan& P, const Geo2& G, int n, size_t mo,
                          size_t cbase, const double* r, double* z, float* sm)
{
    Ctl* ctl = m.s.ctl;
    const int stride = g.G * blockDim.x, t0 = g.rank * blockDim.x + threadIdx.x;
    const float* z0 = m.z0 + mo;
    if (P.nlev > 0) {
        const int lg = min(P.lloc - 1, P.nlev);   // levels 1..lg in global memory, group-wide
        for (int l = 1; l <= lg; ++l) {
            const LView V = lview_global(m, P.lev[l], cbase);
            if (l == 1) down_fine(m, G, mo, r, V, t0, stride);
            else down_coarse(lview_global(m, P.lev[l - 1], cbase), V, t0, stride);
            if (!mg_sync(g, m.budget, ctl)) return false;
            if (l == P.nlev) {   // coarsest in global memory
                for (int sw = 0; sw < kMgSweeps; ++sw) {
                    if (sw % 2 == 0) sweep(V, V.za, V.zb, t0, stride);
                    else sweep(V, V.zb, V.za, t0, stride);
                    if (!mg_sync(g, m.budget, ctl)) return false;
                }
            }
        }
        if (P.lloc <= P.nlev) {
            // with several CTAs, the whole group forms level lloc's right-hand
            // side (the largest step of the shared-memory part) before the
            // first CTA takes over; the values are the same either way
            const bool pre = g.G > 1;
            if (pre) {
                const LView V = lview_global(m, P.lev[P.lloc], cbase);
                if (P.lloc == 1) down_fine(m, G, mo, r, V, t0, stride);
                else down_coarse(lview_global(m, P.lev[P.lloc - 1], cbase), V, t0, stride);
                if (!mg_sync(g, m.budget, ctl)) return false;
            }
            if (g.rank == 0) mg_local(m, P, G, mo, cbase, r, sm, pre);
            if (!mg_sync(g, m.budget, ctl)) return false;
        }
        for (int l = min(lg, P.nlev - 1); l >= 1; --l) {
            up_coarse(lview_global(m, P.lev[l], cbase), lview_global(m, P.lev[l + 1], cbase), t0, stride);
            if (!mg_sync(g, m.budget, ctl)) return false;
        }
        // fine: y = z0 + the level-1 correction, then one sweep
        const float* zb1 = m.czb + cbase + P.lev[1].off;
        const int* par = m.par + mo;
        auto y = [&](int j) { return z0[j] + kMgCoarseScale * zb1[par[j]]; };
        for (int k = t0; k < n; k += stride) {
            const float yk = y(k);
            z[mo + k] = (double)(yk + m.cf[9 * m.T + mo + k] * ((float)r[mo + k] - fine_apply(m, mo, k, y)));
        }
    } else {
        for (int k = t0; k < n; k += stride)
            z[mo + k] = (double)(z0[k] + m.cf[9 * m.T + mo + k] *
                                             ((float)r[mo + k] - fine_apply(m, mo, k, [&](int j) { return z0[j]; })));
    }
    return true;
}

// -------------------------------------------------------------- the solve

// Multigrid set-up and PCG for every member that solves with CG this step
// (after k_solve_init: x = warm start, r = R - A x, p = 0).  Cooperative
// launch of kMgThreads-thread CTAs with kMgSmemBytes of dynamic shared memory.
static __global__ void __launch_bounds__(kMgThreads) k2_mg_pcg(MgArgs m)
{
    extern __shared__ __align__(16) float mg_sm[];
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
        // ---- set-up: FP32 fine rows and level-1 parents, then the coarse rows level by level
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
            if (P.nlev > 0) {
                const int c = a.list[o];
                const MgLev& L = P.lev[1];
                m.par[o] = (((c / G.nx) >> 1) - L.j0) * L.w + (((c % G.nx) >> 1) - L.i0);
            }
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
        // the shared-memory levels' rows, once per solve
        if (g.rank == 0 && P.lloc <= P.nlev) {
            for (int l = P.lloc; l <= P.nlev; ++l) {
                const MgLev& L = P.lev[l];
                for (int q = threadIdx.x; q < L.w * L.h; q += blockDim.x)
#pragma unroll
                    for (int s2 = 0; s2 < 10; ++s2)
                        mg_sm[(size_t)s2 * kMgSmemCells + L.soff + q] = m.cc[s2 * m.CT + cbase + L.off + q];
            }
            __syncthreads();
        }
        float* z0 = m.z0 + mo;
        // ---- z = M r, rz = <r, z>
        for (int k = t0i; k < n; k += stride) z0[k] = m.cf[9 * m.T + mo + k] * (float)a.r[mo + k];
        if (!mg_sync(g, m.budget, ctl)) return;
        if (!mg_vcycle(m, g, P, G, n, mo, cbase, a.r, a.z, mg_sm)) return;
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
            // q = A p with p = z + beta p_old formed at the neighbours on the fly
            double vq[1] = {0.0};
            for (int k = t0i; k < n; k += stride) {
                auto pv = [&](int j) { return a.z[mo + j] + beta * pold[mo + j]; };
                const int kl = a.nbl[mo + k], kr = a.nbr[mo + k];
                const double pk = pv(k);
                const double pl = kl >= 0 ? pv(kl) : 0.0;
                const double pr = kr >= 0 ? pv(kr) : 0.0;
                double qk = apply_row(a, mo, k, pk, pl, pr);
                qk += ext_terms(a, mo, k, pv);
                pnew[mo + k] = pk;
                a.q[mo + k] = qk;
                vq[0] += pk * qk;
            }
            if (!mg_sum<1>(g, vq, red, bc, m.gpart, m.budget, ctl)) return;
            const double pq = vq[0];
            if (!isfinite(pq) || !(pq > 0.0)) { breakdown = true; break; }
            const double alpha = rz / pq;
            for (int k = t0i; k < n; k += stride) {
                a.x[mo + k] += alpha * pnew[mo + k];
                const double rk = rold[mo + k] - alpha * a.q[mo + k];
                rnew[mo + k] = rk;
                z0[k] = m.cf[9 * m.T + mo + k] * (float)rk;
            }
            if (!mg_sync(g, m.budget, ctl)) return;
            if (!mg_vcycle(m, g, P, G, n, mo, cbase, rnew, a.z, mg_sm)) return;
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
