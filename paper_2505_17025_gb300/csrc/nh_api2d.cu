// nh_api2d.cu -- host runtime behind include/nhswe2d.h (2D grids, FP64).
//
// A handle holds an ensemble of nb grids (one for nh2d_create), each with its
// own size, spacing, sides, static depth and slide; member b's cells sit at
// b * pitch in every per-cell buffer, all carved out of the caller's
// workspace.  One step runs, over all members at once: slide kinematics,
// depth at t^n and t^{n+1}, two Heun stages, criterion and Moore
// enlargement, row-major compaction, 9-point assembly, the line-
// preconditioned CG of the 1D members (each grid one member; S, N and the
// diagonal couplings as extra couplings) in one cooperative launch, and the
// correction.  nh2d_run replays that step from a captured CUDA graph.  With
// NH_MIXED_FP64_SOLVE the state lives in FP32 (zeta = h - d0, hu, hv, hw) in
// the same buffers and the predictor and criterion run in FP32; assembly,
// solve and the correction's arithmetic stay FP64.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "nh_mg2d.cuh"
#include "nh_pred2d.cuh"
#include "nhswe2d.h"

using namespace nh;

struct nh_grid2d {
    int nb, pitch;
    std::vector<nh_grid2d_desc> d;
    std::vector<Slide2> slide_h;
    std::vector<char> member_set;
    cudaStream_t stream, cap_stream;
    int maxch, maxpb, nblk, nmass, sms, items_grid, pcr_grid, egx, coop_grid;
    int ptile;                                      // kPredTiles candidate of the FP32 predictor (-1: untuned)
    long long barrier_budget, barrier_budget_default;
    int crit, enlarge, first_global;
    double knh;
    double rtol;
    int max_iter, guess;
    int prec;                                       // NH_FP64 or NH_MIXED_FP64_SOLVE
    bool has_state;
    double t_base, last_dt;
    long long n_since, steps;
    int cur, lcur;
    // device buffers ([nb * pitch] per field unless noted)
    double* q[2][4];
    double* qs[4];
    double* k1[4];
    double *d0, *dn, *dn1;                          // dn, dn1: depth (FP64) or mound (FP32 storage)
    float* d0f;                                     // FP32 copy of d0
    unsigned char *marks, *act;
    int *inv, *list[2], *nact[2], *bcnt, *boff;   // nact [nb]; bcnt, boff [nb * nblk]
    int2 *items, *pitems;
    double *diag, *offl, *offr, *R, *ext_c;
    int *ext_k, *nbl, *nbr;
    double *c6, *cx, *cy, *phi, *ddx, *ddy, *psi;
    double* cq;                                     // [kCq][T] per-cell fields of the assembly
    double *x, *r, *p0, *p1, *qv, *rh, *v0, *v1, *s, *t, *r1, *z;
    float2* pf;
    float* prb;
    MState* ms;
    Ctl* ctl;
    double* part;
    int* cnt;
    double* mass_part;
    Summary* summary;
    Geo2* geos;
    Slide2* slides;
    Kin2* kin;
    TimeCtl* tc;
    // multigrid preconditioner (nh_mg2d.cuh)
    int precond;                                    // NH_PRECOND_LINE or NH_PRECOND_MG
    int cpitch, mg_grid;
    MgPlan* mg_plan;
    MgJob* mg_jobs;
    int* mg_njobs;
    unsigned* mg_gbar;
    double* mg_gpart;
    float *mg_cf, *mg_z0, *mg_cc, *mg_cb, *mg_cza, *mg_czb;
    int* mg_par;
    // profiling (nh2d_set_profiling): event pairs around each launch on the
    // handle's stream, folded into per-class totals at synchronisations
    bool prof_on;
    double prof_ms[NH2_K_COUNT];
    long long prof_launches[NH2_K_COUNT];
    std::vector<cudaEvent_t> prof_pool;
    std::vector<int> prof_kind;
    size_t prof_used;
    // captured step: graph[p] starts from state buffer p
    cudaGraphExec_t graph[2];
    bool graph_valid, use_graphs;
    double graph_key[11];
    long long graph_runs;
};

namespace {

// Events around one launch of class `kind` when profiling and enqueuing on the
// handle's own stream (never inside a capture).
void prof2_pre(nh_grid2d* g, cudaStream_t st, int kind)
{
    if (!g->prof_on || st != g->stream) return;
    g->prof_launches[kind] += 1;
    const size_t need = 2 * (g->prof_used + 1);
    while (g->prof_pool.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { g->prof_on = false; return; }
        g->prof_pool.push_back(e);
    }
    if (g->prof_kind.size() < g->prof_used + 1) g->prof_kind.resize(g->prof_used + 1);
    g->prof_kind[g->prof_used] = kind;
    cudaEventRecord(g->prof_pool[2 * g->prof_used], st);
}

void prof2_post(nh_grid2d* g, cudaStream_t st)
{
    if (!g->prof_on || st != g->stream || g->prof_pool.size() < 2 * (g->prof_used + 1)) return;
    cudaEventRecord(g->prof_pool[2 * g->prof_used + 1], st);
    g->prof_used += 1;
}

// After a synchronisation of the handle's stream.
void prof2_fold(nh_grid2d* g)
{
    for (size_t q = 0; q < g->prof_used; ++q) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->prof_pool[2 * q], g->prof_pool[2 * q + 1]) == cudaSuccess)
            g->prof_ms[g->prof_kind[q]] += ms;
    }
    g->prof_used = 0;
}

#define P2(kind, launch)          \
    do {                          \
        prof2_pre(g, st, kind);   \
        launch;                   \
        prof2_post(g, st);        \
    } while (0)

constexpr size_t kAlign2 = 256;
constexpr int kPitchQuantum = 256;   // cells; keeps every member's slice 256-byte aligned

struct Carver2 {
    char* base;
    size_t off = 0;
    template <typename P>
    P* take(size_t count)
    {
        off = (off + kAlign2 - 1) / kAlign2 * kAlign2;
        P* p = base ? reinterpret_cast<P*>(base + off) : nullptr;
        off += sizeof(P) * count;
        return p;
    }
};

bool desc2_ok(const nh_grid2d_desc* d)
{
    if (!d) return false;
    if (d->nx < 3 || d->ny < 3) return false;
    if ((long long)d->nx * d->ny > (1LL << 26)) return false;
    if (d->bc_x != NH_BC_WALL && d->bc_x != NH_BC_PERIODIC) return false;
    if (d->bc_y != NH_BC_WALL && d->bc_y != NH_BC_PERIODIC) return false;
    if (d->limiter < NH_LIM_NONE || d->limiter > NH_LIM_MC) return false;
    if (!(d->dx > 0.0) || !(d->dy > 0.0) || !(d->g > 0.0) || !(d->rho > 0.0)) return false;
    if (!std::isfinite(d->x0) || !std::isfinite(d->y0)) return false;
    return true;
}

// Cells per member slot, or 0 when the ensemble is invalid or too large.
long long ens_pitch(int nb, const nh_grid2d_desc* descs)
{
    if (nb < 1 || nb > 4096 || !descs) return 0;
    long long mx = 0;
    for (int b = 0; b < nb; ++b) {
        if (!desc2_ok(&descs[b])) return 0;
        mx = std::max(mx, (long long)descs[b].nx * descs[b].ny);
    }
    const long long pitch = (mx + kPitchQuantum - 1) / kPitchQuantum * kPitchQuantum;
    if (pitch * nb > (1LL << 28)) return 0;
    return pitch;
}

// Mass partial sums per member: about 4096 cells per 256-thread block.
int mass_blocks(int pitch) { return std::max(1, std::min((pitch + 4095) / 4096, 512)); }

// Coarse cells per member slot of the multigrid levels: the sum over levels
// l = 1..kMgLevels of the member's grid coarsened l times, the largest member.
int mg_cpitch(int nb, const nh_grid2d_desc* descs)
{
    long long mx = 0;
    for (int b = 0; b < nb; ++b) {
        long long t = 0;
        for (int l = 1; l <= kMgLevels; ++l)
            t += (long long)(((descs[b].nx - 1) >> l) + 1) * (((descs[b].ny - 1) >> l) + 1);
        mx = std::max(mx, t);
    }
    return (int)((mx + kPitchQuantum - 1) / kPitchQuantum * kPitchQuantum);
}

constexpr int kMgMaxGrid = 4096;   // CTAs of the multigrid solve at most

size_t carve2(int nb, int pitch, int cpitch, nh_grid2d* g, char* base)
{
    const size_t T = (size_t)nb * pitch;
    const int maxch = (pitch + kChunk - 1) / kChunk;
    const int maxpb = (pitch + kPcrRows - 1) / kPcrRows;
    const int nblk = (pitch + kCompact2 - 1) / kCompact2;
    const int nmass = mass_blocks(pitch);
    Carver2 c{base};
    nh_grid2d tmp;
    nh_grid2d* G = g ? g : &tmp;
    for (int b = 0; b < 2; ++b)
        for (int f = 0; f < 4; ++f) G->q[b][f] = c.take<double>(T);
    for (int f = 0; f < 4; ++f) { G->qs[f] = c.take<double>(T); G->k1[f] = c.take<double>(T); }
    G->d0 = c.take<double>(T); G->dn = c.take<double>(T); G->dn1 = c.take<double>(T);
    G->d0f = c.take<float>(T);
    G->marks = c.take<unsigned char>(T); G->act = c.take<unsigned char>(T);
    G->inv = c.take<int>(T);
    for (int b = 0; b < 2; ++b) { G->list[b] = c.take<int>(T); G->nact[b] = c.take<int>(nb); }
    G->bcnt = c.take<int>((size_t)nb * nblk); G->boff = c.take<int>((size_t)nb * nblk);
    G->items = c.take<int2>((size_t)nb * maxch); G->pitems = c.take<int2>((size_t)nb * maxpb);
    G->diag = c.take<double>(T); G->offl = c.take<double>(T); G->offr = c.take<double>(T);
    G->R = c.take<double>(T);
    G->ext_c = c.take<double>(6 * T); G->ext_k = c.take<int>(6 * T);
    G->nbl = c.take<int>(T); G->nbr = c.take<int>(T);
    G->c6 = c.take<double>(T); G->cx = c.take<double>(T); G->cy = c.take<double>(T);
    G->phi = c.take<double>(T); G->ddx = c.take<double>(T); G->ddy = c.take<double>(T);
    G->cq = c.take<double>((size_t)kCq * T);
    G->psi = c.take<double>(T);
    G->x = c.take<double>(T); G->r = c.take<double>(T); G->p0 = c.take<double>(T); G->p1 = c.take<double>(T);
    G->qv = c.take<double>(T); G->rh = c.take<double>(T); G->v0 = c.take<double>(T); G->v1 = c.take<double>(T);
    G->s = c.take<double>(T); G->t = c.take<double>(T); G->r1 = c.take<double>(T); G->z = c.take<double>(T);
    G->pf = c.take<float2>((size_t)kPcrLevels * T); G->prb = c.take<float>(T);
    G->ms = c.take<MState>(nb); G->ctl = c.take<Ctl>(1);
    G->part = c.take<double>(4 * (size_t)nb * maxch); G->cnt = c.take<int>(nb);
    G->mass_part = c.take<double>((size_t)nb * nmass); G->summary = c.take<Summary>(1);
    G->geos = c.take<Geo2>(nb); G->slides = c.take<Slide2>(nb); G->kin = c.take<Kin2>(2 * (size_t)nb);
    G->tc = c.take<TimeCtl>(1);
    const size_t CT = (size_t)nb * cpitch;
    G->mg_plan = c.take<MgPlan>(nb);
    G->mg_jobs = c.take<MgJob>((size_t)std::max(nb, kMgMaxGrid));
    G->mg_njobs = c.take<int>(1);
    G->mg_gbar = c.take<unsigned>(2 * (size_t)nb);
    G->mg_gpart = c.take<double>(8 * (size_t)kMgMaxGrid);
    G->mg_cf = c.take<float>(10 * T);
    G->mg_z0 = c.take<float>(T); G->mg_par = c.take<int>(T);
    G->mg_cc = c.take<float>(10 * CT);
    G->mg_cb = c.take<float>(CT); G->mg_cza = c.take<float>(CT); G->mg_czb = c.take<float>(CT);
    if (g) { g->maxch = maxch; g->maxpb = maxpb; g->nblk = nblk; g->nmass = nmass; g->cpitch = cpitch; }
    return (c.off + kAlign2 - 1) / kAlign2 * kAlign2;
}

#define CK2(call)                                       \
    do {                                                \
        if ((call) != cudaSuccess) return NH_ERR_CUDA;  \
    } while (0)

Geo2 geo2(const nh_grid2d_desc& d)
{
    Geo2 G;
    G.nx = d.nx; G.ny = d.ny; G.bcx = d.bc_x; G.bcy = d.bc_y; G.lim = d.limiter;
    G.dx = d.dx; G.dy = d.dy; G.x0 = d.x0; G.y0 = d.y0; G.g = d.g;
    G.idx = 1.0 / d.dx; G.idy = 1.0 / d.dy;
    return G;
}

SolveArgs<double> solve_args2(nh_grid2d* g, int lnew, double gscale, const TimeCtl* tc)
{
    SolveArgs<double> a;
    a.nb = g->nb; a.pitch = g->pitch; a.maxch = g->maxch;
    const size_t T = (size_t)g->nb * g->pitch;
    a.list = g->list[lnew];
    a.diag = g->diag; a.offl = g->offl; a.offr = g->offr; a.R = g->R;
    a.nbl = g->nbl; a.nbr = g->nbr;
    a.psi_prev = g->psi; a.guess_scale = gscale;
    a.x = g->x; a.r = g->r; a.p0 = g->p0; a.p1 = g->p1; a.q = g->qv; a.rh = g->rh;
    a.v0 = g->v0; a.v1 = g->v1; a.s = g->s; a.t = g->t; a.r1 = g->r1; a.z = g->z;
    a.pf = g->pf; a.prb = g->prb; a.pf_stride = T;
    a.n_ext = 6; a.ext_c = g->ext_c; a.ext_k = g->ext_k; a.ext_stride = T;
    a.maxpb = g->maxpb; a.items = g->items; a.pitems = g->pitems;
    a.tc = tc; a.ms = g->ms; a.ctl = g->ctl; a.part = g->part; a.cnt = g->cnt;
    a.rtol = g->rtol; a.max_iter = g->max_iter; a.it = 0;
    return a;
}

// Everything of one step up to the assembled systems: kinematics, depth,
// predictor, criterion, mask, compaction, work items, assembly, mass.
template <typename TS>
TS* as(double* p) { return reinterpret_cast<TS*>(p); }

template <typename TS>
const TS* d0_storage(const nh_grid2d* g)
{
    if constexpr (sizeof(TS) == 8) return nullptr;
    else return g->d0f;
}

template <typename TS>
nh_status enqueue_mask_assembly(nh_grid2d* g, cudaStream_t st, int nxt, int lnew, double dt, bool all,
                                const TimeCtl* tc);

// float4 loads of Q^n and d0s need 16-byte aligned arrays and a member pitch
// of a multiple of 4 floats (each member's rows then also need nx % 4 == 0,
// checked in the kernel).
int fused_vec4(const FusedArgs& fa)
{
    auto al = [](const void* p) { return ((uintptr_t)p & 15) == 0; };
    return (fa.pitch % 4 == 0 && al(fa.z) && al(fa.hu) && al(fa.hv) && al(fa.hw) && al(fa.d0s)) ? 1 : 0;
}

// The one-launch FP32 predictor with tile candidate c (kPredTiles[c]): CTAs
// per member cover its largest tile count, at most 8 per SM over the members.
template <int TX, int TY>
cudaError_t launch_fused_t(nh_grid2d* g, cudaStream_t st, const FusedArgs& fa)
{
    int tiles = 1;
    for (const nh_grid2d_desc& d : g->d) tiles = std::max(tiles, ((d.nx + TX - 1) / TX) * ((d.ny + TY - 1) / TY));
    const int gx = std::max(1, std::min(tiles, (g->sms * 8 + g->nb - 1) / g->nb));
    prof2_pre(g, st, NH2_K_STAGE);
    k2_heun_fused<TX, TY><<<dim3(gx, g->nb), TX * TY, PTile<TX, TY>::smem, st>>>(fa);
    prof2_post(g, st);
    return cudaGetLastError();
}

cudaError_t launch_fused(nh_grid2d* g, cudaStream_t st, int c, const FusedArgs& fa)
{
    switch (c) {
        case 1: return launch_fused_t<64, 8>(g, st, fa);
        case 2: return launch_fused_t<32, 8>(g, st, fa);
        case 3: return launch_fused_t<64, 16>(g, st, fa);
        default: return launch_fused_t<32, 16>(g, st, fa);
    }
}

cudaError_t fused_attributes()
{
    cudaError_t e = cudaFuncSetAttribute(k2_heun_fused<32, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)PTile<32, 16>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k2_heun_fused<64, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PTile<64, 8>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k2_heun_fused<32, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PTile<32, 8>::smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k2_heun_fused<64, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)PTile<64, 16>::smem);
    return e;
}

template <typename TS>
nh_status enqueue_front(nh_grid2d* g, cudaStream_t st, int cur, int lnew, double dt, double t_n, double t_n1,
                        bool all, const TimeCtl* tc)
{
    const int nxt = cur ^ 1;
    const size_t T = (size_t)g->nb * g->pitch;
    const size_t P = (size_t)g->pitch;
    const dim3 eg(g->egx, g->nb);
    P2(NH2_K_KIN, (k2_kin<<<(g->nb + 127) / 128, 128, 0, st>>>(g->slides, g->nb, t_n, t_n1, tc, g->kin)));
    const TS* d0s = d0_storage<TS>(g);
    if constexpr (sizeof(TS) == 4) {
        // FP32 state: both Heun stages, the mound and the |eta/d| marks in one launch
        const bool fused_marks = !all && g->crit == NH_CRIT_ETA_D;
        FusedArgs fa;
        fa.geos = g->geos; fa.slides = g->slides; fa.kin = g->kin; fa.pitch = P;
        fa.z = as<float>(g->q[cur][0]); fa.hu = as<float>(g->q[cur][1]); fa.hv = as<float>(g->q[cur][2]);
        fa.hw = as<float>(g->q[cur][3]); fa.d0s = g->d0f;
        fa.oz = as<float>(g->q[nxt][0]); fa.ohu = as<float>(g->q[nxt][1]); fa.ohv = as<float>(g->q[nxt][2]);
        fa.ohw = as<float>(g->q[nxt][3]); fa.m1 = as<float>(g->dn1);
        fa.marks = fused_marks ? g->marks : nullptr; fa.knh = (float)g->knh; fa.dt = dt; fa.tc = tc;
        fa.vec4 = fused_vec4(fa);
        CK2(launch_fused(g, st, g->ptile, fa));
        if (all) CK2(cudaMemsetAsync(g->marks, 1, T, st));
        else if (g->crit == NH_CRIT_HYDROSTATIC) CK2(cudaMemsetAsync(g->marks, 0, T, st));
        else if (!fused_marks)
            P2(NH2_K_MARKS, (k2_marks<TS><<<eg, 256, 0, st>>>(g->geos, P, as<TS>(g->q[nxt][0]), as<TS>(g->q[nxt][1]),
                                                               as<TS>(g->q[nxt][2]), as<TS>(g->q[nxt][3]),
                                                               as<TS>(g->dn1), d0s, g->crit, g->knh, g->marks)));
        return enqueue_mask_assembly<TS>(g, st, nxt, lnew, dt, all, tc);
    }
    P2(NH2_K_DEPTH, (k2_depth<TS><<<eg, 256, 0, st>>>(g->geos, g->slides, g->kin, 0, P, g->d0, as<TS>(g->dn), tc)));
    P2(NH2_K_DEPTH, (k2_depth<TS><<<eg, 256, 0, st>>>(g->geos, g->slides, g->kin, 1, P, g->d0, as<TS>(g->dn1), tc)));
    StageArgs<TS> sa1;
    sa1.geos = g->geos; sa1.pitch = P; sa1.d0s = d0s;
    sa1.h = as<TS>(g->q[cur][0]); sa1.hu = as<TS>(g->q[cur][1]); sa1.hv = as<TS>(g->q[cur][2]);
    sa1.hw = as<TS>(g->q[cur][3]); sa1.d = as<TS>(g->dn);
    sa1.h0 = sa1.h; sa1.hu0 = sa1.hu; sa1.hv0 = sa1.hv; sa1.hw0 = sa1.hw;
    sa1.k1h = as<TS>(g->k1[0]); sa1.k1u = as<TS>(g->k1[1]); sa1.k1v = as<TS>(g->k1[2]); sa1.k1w = as<TS>(g->k1[3]);
    sa1.oh = as<TS>(g->qs[0]); sa1.ohu = as<TS>(g->qs[1]); sa1.ohv = as<TS>(g->qs[2]); sa1.ohw = as<TS>(g->qs[3]);
    sa1.dt = dt; sa1.stage = 1; sa1.tc = tc;
    P2(NH2_K_STAGE, (k2_stage<TS><<<eg, kTX * kTY, 0, st>>>(sa1)));
    StageArgs<TS> sa2 = sa1;
    sa2.h = sa1.oh; sa2.hu = sa1.ohu; sa2.hv = sa1.ohv; sa2.hw = sa1.ohw; sa2.d = as<TS>(g->dn1);
    sa2.oh = as<TS>(g->q[nxt][0]); sa2.ohu = as<TS>(g->q[nxt][1]); sa2.ohv = as<TS>(g->q[nxt][2]);
    sa2.ohw = as<TS>(g->q[nxt][3]);
    sa2.stage = 2;
    P2(NH2_K_STAGE, (k2_stage<TS><<<eg, kTX * kTY, 0, st>>>(sa2)));

    if (all) CK2(cudaMemsetAsync(g->marks, 1, T, st));
    else if (g->crit == NH_CRIT_HYDROSTATIC) CK2(cudaMemsetAsync(g->marks, 0, T, st));
    else P2(NH2_K_MARKS, (k2_marks<TS><<<eg, 256, 0, st>>>(g->geos, P, sa2.oh, sa2.ohu, sa2.ohv, sa2.ohw,
                                                           as<TS>(g->dn1), d0s, g->crit, g->knh, g->marks)));
    return enqueue_mask_assembly<TS>(g, st, nxt, lnew, dt, all, tc);
}

// After the predictor and the marks: enlargement, compaction, work items,
// assembly of the elliptic rows, mass partial sums.
template <typename TS>
nh_status enqueue_mask_assembly(nh_grid2d* g, cudaStream_t st, int nxt, int lnew, double dt, bool all,
                                const TimeCtl* tc)
{
    const size_t T = (size_t)g->nb * g->pitch;
    const size_t P = (size_t)g->pitch;
    const dim3 eg(g->egx, g->nb);
    P2(NH2_K_DILATE, (k2_dilate<<<eg, 256, 0, st>>>(g->geos, P, g->marks, all ? 0 : g->enlarge, g->act, tc)));
    P2(NH2_K_COMPACT, (k2_count<<<dim3(g->nblk, g->nb), kCompact2, 0, st>>>(g->geos, P, g->act, g->nblk, g->bcnt)));
    P2(NH2_K_COMPACT, (k2_scan<<<g->nb, 1024, 0, st>>>(g->bcnt, g->nblk, g->boff, g->nact[lnew], g->ms, tc)));
    P2(NH2_K_COMPACT, (k2_emit<<<dim3(g->nblk, g->nb), kCompact2, 0, st>>>(g->geos, P, g->act, g->nblk, g->boff,
                                                                             g->list[lnew], g->inv, tc)));
    P2(NH2_K_COMPACT, (k_items<<<1, 1024, 0, st>>>(g->ms, g->nb, g->items, g->pitems, g->ctl)));
    CK2(cudaMemsetAsync(g->cnt, 0, sizeof(int) * g->nb, st));

    Asm2Args<TS> aa;
    aa.geos = g->geos; aa.slides = g->slides; aa.kin = g->kin;
    aa.nb = g->nb; aa.pitch = g->pitch; aa.maxch = g->maxch;
    aa.ht = as<TS>(g->q[nxt][0]); aa.hut = as<TS>(g->q[nxt][1]); aa.hvt = as<TS>(g->q[nxt][2]);
    aa.hwt = as<TS>(g->q[nxt][3]);
    aa.d0 = g->d0; aa.d1 = as<TS>(g->dn1); aa.dt = dt;
    aa.list = g->list[lnew]; aa.inv = g->inv; aa.ms = g->ms;
    aa.diag = g->diag; aa.offl = g->offl; aa.offr = g->offr; aa.R = g->R;
    aa.nbl = g->nbl; aa.nbr = g->nbr;
    aa.ext_c = g->ext_c; aa.ext_k = g->ext_k; aa.ext_stride = T;
    aa.c6 = g->c6; aa.cx = g->cx; aa.cy = g->cy; aa.phi = g->phi; aa.ddx = g->ddx; aa.ddy = g->ddy;
    aa.cq = g->cq;
    aa.part = g->part; aa.cnt = g->cnt; aa.solver = NH_SOLVER_AUTO;
    aa.items = g->items; aa.ctl = g->ctl;
    P2(NH2_K_ASSEMBLE, (k2_cellq<TS><<<g->items_grid, kChunk, 0, st>>>(aa)));
    P2(NH2_K_ASSEMBLE, (k2_assemble<TS><<<g->items_grid, kChunk, 0, st>>>(aa)));
    P2(NH2_K_MASS, (k2_mass<TS><<<dim3(g->nmass, g->nb), 256, 0, st>>>(g->geos, P, as<TS>(g->q[nxt][0]), g->d0,
                                                                        g->mass_part)));
    return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

// The accepted step's tail: zero psi on the previous mask, correct on the new one.
template <typename TS>
nh_status enqueue_back(nh_grid2d* g, cudaStream_t st, int nxt, int lprev, int lnew, const TimeCtl* tc)
{
    const size_t T = (size_t)g->nb * g->pitch;
    ClearArgs cl;
    cl.nb = g->nb; cl.pitch = g->pitch; cl.maxlist = g->pitch;
    cl.list_prev = g->list[lprev]; cl.nact_prev = g->nact[lprev]; cl.psi = g->psi; cl.tc = tc;
    P2(NH2_K_CLEAR, (k_clear_prev<<<(int)std::min<size_t>((T + 255) / 256, (size_t)g->sms * 8), 256, 0, st>>>(cl)));
    Corr2Args<TS> co;
    co.geos = g->geos; co.pitch = g->pitch; co.list = g->list[lnew];
    co.nbl = g->nbl; co.nbr = g->nbr; co.ext_k = g->ext_k; co.ext_stride = T;
    co.x = g->x; co.c6 = g->c6; co.cx = g->cx; co.cy = g->cy; co.phi = g->phi;
    co.ddx = g->ddx; co.ddy = g->ddy; co.ms = g->ms;
    co.hu = as<TS>(g->q[nxt][1]); co.hv = as<TS>(g->q[nxt][2]); co.hw = as<TS>(g->q[nxt][3]); co.psi = g->psi;
    co.items = g->items; co.ctl = g->ctl; co.tc = tc;
    P2(NH2_K_CORRECT, (k2_correct<TS><<<g->items_grid, kChunk, 0, st>>>(co)));
    return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

nh_status launch_persistent(nh_grid2d* g, SolveArgs<double>& sa, cudaStream_t st)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g->coop_grid);
    cfg.blockDim = dim3(kPcrThreads);
    cfg.dynamicSmemBytes = 2 * sizeof(float) * (size_t)kPcrRows;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    long long budget = g->barrier_budget;
    prof2_pre(g, st, NH2_K_SOLVE);
    CK2(cudaLaunchKernelEx(&cfg, k_pcg_persistent<double, float>, sa, budget));
    prof2_post(g, st);
    return NH_OK;
}

std::mutex g_tune2_mutex;
std::map<std::vector<int>, int> g_tune2_cache;

// Tile of the FP32 one-launch predictor: each candidate of kPredTiles is
// timed (2 warm-up and 5 timed launches, CUDA events on the handle's stream)
// on the handle's live state, and the fastest is kept; the choice is cached
// per set of member sizes and limiters.  The launches only write the next
// step's buffers.
nh_status tune_fused(nh_grid2d* g, double dt)
{
    if (g->ptile >= 0) return NH_OK;
    std::vector<int> key;
    for (const nh_grid2d_desc& d : g->d) { key.push_back(d.nx); key.push_back(d.ny); key.push_back(d.limiter); }
    {
        std::lock_guard<std::mutex> lock(g_tune2_mutex);
        auto it = g_tune2_cache.find(key);
        if (it != g_tune2_cache.end()) { g->ptile = it->second; return NH_OK; }
    }
    cudaStream_t st = g->stream;
    const int cur = g->cur, nxt = cur ^ 1;
    const double t_n = g->t_base + (double)g->n_since * dt;
    k2_kin<<<(g->nb + 127) / 128, 128, 0, st>>>(g->slides, g->nb, t_n, t_n + dt, nullptr, g->kin);
    FusedArgs fa;
    fa.geos = g->geos; fa.slides = g->slides; fa.kin = g->kin; fa.pitch = (size_t)g->pitch;
    fa.z = as<float>(g->q[cur][0]); fa.hu = as<float>(g->q[cur][1]); fa.hv = as<float>(g->q[cur][2]);
    fa.hw = as<float>(g->q[cur][3]); fa.d0s = g->d0f;
    fa.oz = as<float>(g->q[nxt][0]); fa.ohu = as<float>(g->q[nxt][1]); fa.ohv = as<float>(g->q[nxt][2]);
    fa.ohw = as<float>(g->q[nxt][3]); fa.m1 = as<float>(g->dn1);
    fa.marks = g->marks; fa.knh = (float)g->knh; fa.dt = dt; fa.tc = nullptr;
    fa.vec4 = fused_vec4(fa);
    cudaEvent_t e0, e1;
    CK2(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return NH_ERR_CUDA; }
    const bool prof = g->prof_on;
    g->prof_on = false;
    float best = 1e30f;
    int best_c = 0;
    nh_status rc = NH_OK;
    for (int c = 0; c < 4 && rc == NH_OK; ++c) {
        for (int w = 0; w < 2; ++w)
            if (launch_fused(g, st, c, fa) != cudaSuccess) rc = NH_ERR_CUDA;
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5; ++r)
            if (launch_fused(g, st, c, fa) != cudaSuccess) rc = NH_ERR_CUDA;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) rc = NH_ERR_CUDA;
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rc == NH_OK && ms < best) { best = ms; best_c = c; }
    }
    g->prof_on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (rc != NH_OK) return rc;
    g->ptile = best_c;
    std::lock_guard<std::mutex> lock(g_tune2_mutex);
    g_tune2_cache[key] = best_c;
    return NH_OK;
}

// Multigrid-preconditioned CG of every member solving with CG (after
// k_solve_init): plan the levels, split the members over the cooperative
// grid, then the persistent solve.
nh_status launch_mg(nh_grid2d* g, const SolveArgs<double>& sa, cudaStream_t st)
{
    prof2_pre(g, st, NH2_K_SOLVE);
    k2_mg_box<<<g->nb, 1024, 0, st>>>(g->geos, g->ms, sa.list, g->pitch, g->mg_plan);
    k2_mg_assign<<<1, 1024, 0, st>>>(g->ms, g->nb, g->mg_grid, g->mg_jobs, g->mg_njobs);
    CK2(cudaMemsetAsync(g->mg_gbar, 0, 2 * sizeof(unsigned) * g->nb, st));
    MgArgs m;
    m.s = sa;
    m.geos = g->geos; m.inv = g->inv; m.plan = g->mg_plan; m.jobs = g->mg_jobs; m.njobs = g->mg_njobs;
    m.gbar = g->mg_gbar; m.gpart = g->mg_gpart;
    m.cf = g->mg_cf; m.z0 = g->mg_z0; m.par = g->mg_par;
    m.cc = g->mg_cc; m.cb = g->mg_cb; m.cza = g->mg_cza; m.czb = g->mg_czb;
    m.T = (size_t)g->nb * g->pitch; m.CT = (size_t)g->nb * g->cpitch; m.cpitch = g->cpitch;
    m.budget = g->barrier_budget;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g->mg_grid);
    cfg.blockDim = dim3(kMgThreads);
    cfg.dynamicSmemBytes = kMgSmemBytes;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    CK2(cudaLaunchKernelEx(&cfg, k2_mg_pcg, m));
    prof2_post(g, st);
    return NH_OK;
}

bool use_mg(const nh_grid2d* g) { return g->precond == NH_PRECOND_MG && g->mg_grid > 0; }

// One Krylov pass: set-up, then preconditioned CG in one cooperative launch,
// and preconditioned BiCGStab driven from the host for members that need it.
nh_status krylov2_pass(nh_grid2d* g, SolveArgs<double>& sa)
{
    cudaStream_t st = g->stream;
    CK2(cudaMemsetAsync(g->ctl, 0, 3 * sizeof(int), st));
    CK2(cudaMemsetAsync(g->cnt, 0, sizeof(int) * g->nb, st));
    P2(NH2_K_SOLVE_INIT, (k_solve_init<double><<<g->items_grid, kChunk, 0, st>>>(sa)));
    Ctl h;
    CK2(cudaMemcpyAsync(&h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK2(cudaStreamSynchronize(st));
    prof2_fold(g);
    const size_t pcr_smem = 2 * sizeof(float) * (size_t)kPcrRows;
    const bool mg = use_mg(g);
    if ((h.n_cg > 0 && !mg) || h.n_bicg > 0)
        P2(NH2_K_SOLVE, (k_pcr_factor<double, float><<<g->pcr_grid, kPcrThreads, 3 * sizeof(float) * kPcrRows, st>>>(sa)));
    if (h.n_cg > 0 && !mg) {
        sa.it = 0;
        P2(NH2_K_SOLVE, (k_pcr<double, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_PCG)));
    }
    if (h.not_done <= 0) return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
    if (h.n_cg > 0 && mg) {
        CK2(cudaMemsetAsync(&g->ctl->timeout, 0, 3 * sizeof(int), st));
        nh_status rc = launch_mg(g, sa, st);
        if (rc != NH_OK) return rc;
        int to = 0;
        CK2(cudaMemcpyAsync(&to, &g->ctl->timeout, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK2(cudaStreamSynchronize(st));
        if (to) return NH_ERR_TIMEOUT;
        if (h.n_bicg == 0) return NH_OK;
    }
    const bool coop_cg = h.n_cg > 0 && g->coop_grid > 0 && !mg;
    if (coop_cg) {
        CK2(cudaMemsetAsync(&g->ctl->timeout, 0, 3 * sizeof(int), st));
        nh_status rc = launch_persistent(g, sa, st);
        if (rc != NH_OK) return rc;
        int to = 0;
        CK2(cudaMemcpyAsync(&to, &g->ctl->timeout, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK2(cudaStreamSynchronize(st));
        if (to) return NH_ERR_TIMEOUT;
        if (h.n_bicg == 0) return NH_OK;
    }
    for (int it = 1; it <= g->max_iter; ++it) {
        sa.it = it;
        if (h.n_cg > 0 && !coop_cg && !mg) {
            k_pcg_a<double><<<g->items_grid, kChunk, 0, st>>>(sa);
            k_pcr<double, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_PCG_STEP);
        }
        if (h.n_bicg > 0) {
            k_pcr<double, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_BI_P);
            k_pbi_mv<double><<<g->items_grid, kChunk, 0, st>>>(sa, 0);
            k_pcr<double, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_BI_S);
            k_pbi_mv<double><<<g->items_grid, kChunk, 0, st>>>(sa, 1);
            k_pbi_upd<double><<<g->items_grid, kChunk, 0, st>>>(sa);
        }
        if (it % 8 == 0 || it == g->max_iter) {
            int nd = 0;
            CK2(cudaMemcpyAsync(&nd, &g->ctl->not_done, sizeof(int), cudaMemcpyDeviceToHost, st));
            CK2(cudaStreamSynchronize(st));
            if (nd <= 0) break;
        }
    }
    return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

nh_status krylov2(nh_grid2d* g, SolveArgs<double>& sa)
{
    cudaStream_t st = g->stream;
    CK2(cudaMemsetAsync(&g->ctl->n_fallback, 0, sizeof(int), st));
    nh_status rc = krylov2_pass(g, sa);
    if (rc != NH_OK) return rc;
    int nfb = 0;
    CK2(cudaMemcpyAsync(&nfb, &g->ctl->n_fallback, sizeof(int), cudaMemcpyDeviceToHost, st));
    CK2(cudaStreamSynchronize(st));
    if (nfb == 0) return NH_OK;
    k_fallback_reset<<<(g->nb + 127) / 128, 128, 0, st>>>(g->ms, g->nb);
    return krylov2_pass(g, sa);
}

void fill_info(const nh_grid2d* g, const Summary& S, nh_status status, double t, nh_step_info* info)
{
    info->step = g->steps;
    info->t = t;
    info->n_active = S.n_active;
    info->n_active_max = S.n_active_max;
    info->iters = S.iters;
    info->ir_passes = 0;
    info->solver = S.n_active == 0 ? -1 : (S.any_bicg ? NH_SOLVER_BICGSTAB : NH_SOLVER_CG);
    info->status = status;
    info->rel_res = S.rel_res;
    info->min_gamma = S.min_gamma;
    info->mass = S.mass;
}

nh_status step2(nh_grid2d* g, double dt, nh_step_info* info)
{
    cudaStream_t st = g->stream;
    if (g->last_dt != 0.0 && dt != g->last_dt) {
        g->t_base += (double)g->n_since * g->last_dt;
        g->n_since = 0;
    }
    const double t_n = g->t_base + (double)g->n_since * dt;
    const double t_n1 = g->t_base + (double)(g->n_since + 1) * dt;
    const int cur = g->cur, nxt = cur ^ 1, lprev = g->lcur, lnew = lprev ^ 1;
    const bool all = g->crit == NH_CRIT_GLOBAL || (g->first_global && g->steps == 0);
    if (g->prec != NH_FP64) {
        nh_status rt = tune_fused(g, dt);
        if (rt != NH_OK) return rt;
    }
    nh_status rc = g->prec == NH_FP64 ? enqueue_front<double>(g, st, cur, lnew, dt, t_n, t_n1, all, nullptr)
                                      : enqueue_front<float>(g, st, cur, lnew, dt, t_n, t_n1, all, nullptr);
    if (rc != NH_OK) return rc;
    const double gscale = (g->guess == NH_GUESS_PREV && g->last_dt > 0.0) ? dt / g->last_dt : 0.0;
    SolveArgs<double> sa = solve_args2(g, lnew, gscale, nullptr);
    rc = krylov2(g, sa);
    if (rc != NH_OK) return rc;
    P2(NH2_K_SUMMARY, (k_summary<<<1, 256, 0, st>>>(g->ms, g->nb, g->mass_part, g->nb * g->nmass, 1.0, g->summary,
                                                  nullptr)));
    Summary S;
    CK2(cudaMemcpyAsync(&S, g->summary, sizeof(Summary), cudaMemcpyDeviceToHost, st));
    CK2(cudaStreamSynchronize(st));
    prof2_fold(g);
    CK2(cudaGetLastError());
    const nh_status status = (nh_status)S.status;
    if (status == NH_OK) {
        rc = g->prec == NH_FP64 ? enqueue_back<double>(g, st, nxt, lprev, lnew, nullptr)
                                : enqueue_back<float>(g, st, nxt, lprev, lnew, nullptr);
        if (rc != NH_OK) return rc;
        g->cur = nxt;
        g->lcur = lnew;
        g->n_since += 1;
        g->steps += 1;
        g->last_dt = dt;
        if (g->prof_on) {
            CK2(cudaStreamSynchronize(st));
            prof2_fold(g);
        }
    }
    if (info) fill_info(g, S, status, status == NH_OK ? t_n1 : t_n, info);
    return status;
}

// ------------------------------------------------------------ captured runs

// One step with fixed buffer roles and no host round trip: the time control
// block supplies t, the commit kernel accepts the step or aborts the run, and
// every kernel that writes state skips after an abort.
nh_status enqueue_graph_step(nh_grid2d* g, cudaStream_t st, int cur, int lprev, double dt)
{
    const int nxt = cur ^ 1, lnew = lprev ^ 1;
    const bool all = g->crit == NH_CRIT_GLOBAL;
    nh_status rc = g->prec == NH_FP64 ? enqueue_front<double>(g, st, cur, lnew, dt, 0.0, 0.0, all, g->tc)
                                      : enqueue_front<float>(g, st, cur, lnew, dt, 0.0, 0.0, all, g->tc);
    if (rc != NH_OK) return rc;
    SolveArgs<double> sa = solve_args2(g, lnew, g->guess == NH_GUESS_PREV ? 1.0 : 0.0, g->tc);
    CK2(cudaMemsetAsync(g->ctl, 0, 3 * sizeof(int), st));
    CK2(cudaMemsetAsync(g->cnt, 0, sizeof(int) * g->nb, st));
    k_solve_init<double><<<g->items_grid, kChunk, 0, st>>>(sa);
    if (use_mg(g)) {
        CK2(cudaMemsetAsync(&g->ctl->timeout, 0, 3 * sizeof(int), st));
        rc = launch_mg(g, sa, st);
    } else {
        k_pcr_factor<double, float><<<g->pcr_grid, kPcrThreads, 3 * sizeof(float) * kPcrRows, st>>>(sa);
        k_pcr<double, float><<<g->pcr_grid, kPcrThreads, 2 * sizeof(float) * kPcrRows, st>>>(sa, PCR_PCG);
        CK2(cudaMemsetAsync(&g->ctl->timeout, 0, 3 * sizeof(int), st));
        rc = launch_persistent(g, sa, st);
    }
    if (rc != NH_OK) return rc;
    k_summary<<<1, 256, 0, st>>>(g->ms, g->nb, g->mass_part, g->nb * g->nmass, 1.0, g->summary, g->tc);
    k_commit<<<1, 32, 0, st>>>(g->summary, g->tc);
    return g->prec == NH_FP64 ? enqueue_back<double>(g, st, nxt, lprev, lnew, g->tc)
                              : enqueue_back<float>(g, st, nxt, lprev, lnew, g->tc);
}

bool graph_eligible(const nh_grid2d* g, double dt)
{
    return g->use_graphs && !g->prof_on && g->coop_grid > 0 && g->cap_stream != nullptr &&
           !(g->first_global && g->steps == 0) && (g->last_dt == 0.0 || g->last_dt == dt);
}

void graph_destroy(nh_grid2d* g)
{
    for (int p = 0; p < 2; ++p)
        if (g->graph[p]) { cudaGraphExecDestroy(g->graph[p]); g->graph[p] = nullptr; }
    g->graph_valid = false;
}

nh_status graph_prepare(nh_grid2d* g, double dt)
{
    const double key[11] = {dt, (double)g->crit, g->knh, (double)g->enlarge, g->rtol, (double)g->max_iter,
                            (double)g->guess, (double)(g->cur ^ g->lcur), (double)g->prec, (double)g->precond,
                            (double)g->ptile};
    if (g->graph_valid && std::memcmp(key, g->graph_key, sizeof(key)) == 0) return NH_OK;
    graph_destroy(g);
    for (int p = 0; p < 2; ++p) {
        const int cur = p, lprev = p ^ g->cur ^ g->lcur;
        cudaGraph_t graph = nullptr;
        CK2(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
        nh_status rc = enqueue_graph_step(g, g->cap_stream, cur, lprev, dt);
        cudaError_t e = cudaStreamEndCapture(g->cap_stream, &graph);
        if (rc != NH_OK || e != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            graph_destroy(g);
            return rc != NH_OK ? rc : NH_ERR_CUDA;
        }
        e = cudaGraphInstantiate(&g->graph[p], graph, 0);
        cudaGraphDestroy(graph);
        if (e != cudaSuccess) { g->graph[p] = nullptr; graph_destroy(g); return NH_ERR_CUDA; }
    }
    std::memcpy(g->graph_key, key, sizeof(key));
    g->graph_valid = true;
    return NH_OK;
}

// n_steps steps by replaying the captured graphs on the handle's stream; one
// synchronisation at the end.
nh_status graph_run(nh_grid2d* g, double dt, long long n_steps, nh_run_info* R)
{
    if (g->last_dt != 0.0 && dt != g->last_dt) {
        g->t_base += (double)g->n_since * g->last_dt;
        g->n_since = 0;
    }
    if (g->prec != NH_FP64) {
        nh_status rt = tune_fused(g, dt);
        if (rt != NH_OK) return rt;
    }
    nh_status rc = graph_prepare(g, dt);
    if (rc != NH_OK) return rc;
    cudaStream_t st = g->stream;
    TimeCtl tc;
    std::memset(&tc, 0, sizeof(tc));
    tc.t_base = g->t_base; tc.dt = dt; tc.n = g->n_since; tc.done = 0; tc.abort = 0;
    tc.prev_ok = (g->last_dt == dt) ? 1 : 0;
    CK2(cudaMemcpyAsync(g->tc, &tc, sizeof(tc), cudaMemcpyHostToDevice, st));
    for (long long k = 0; k < n_steps; ++k) CK2(cudaGraphLaunch(g->graph[(g->cur + k) & 1], st));
    Summary S;
    CK2(cudaMemcpyAsync(&tc, g->tc, sizeof(tc), cudaMemcpyDeviceToHost, st));
    CK2(cudaMemcpyAsync(&S, g->summary, sizeof(Summary), cudaMemcpyDeviceToHost, st));
    CK2(cudaStreamSynchronize(st));
    const long long done = tc.done;
    if (done & 1) { g->cur ^= 1; g->lcur ^= 1; }
    g->steps += done;
    g->n_since += done;
    if (done > 0) g->last_dt = dt;
    g->graph_runs += 1;
    R->steps = done;
    R->iters_total = tc.iters_total;
    R->active_total = tc.active_total;
    const nh_status st_last = tc.abort ? (nh_status)tc.fail_status : NH_OK;
    fill_info(g, S, st_last, g->t_base + (double)g->n_since * dt, &R->last);
    if (tc.abort)
        return (nh_status)(tc.fail_status == kStatusFallback ? NH_ERR_NONFINITE : tc.fail_status);
    return NH_OK;
}

bool member_ok(const nh_grid2d* g, int m) { return g && m >= 0 && m < g->nb; }

}  // namespace

extern "C" {

size_t nh2d_ensemble_workspace_bytes(int n_members, const nh_grid2d_desc* descs)
{
    const long long pitch = ens_pitch(n_members, descs);
    if (pitch == 0) return 0;
    return carve2(n_members, (int)pitch, mg_cpitch(n_members, descs), nullptr, nullptr);
}

size_t nh2d_workspace_bytes(const nh_grid2d_desc* desc) { return nh2d_ensemble_workspace_bytes(1, desc); }

nh_status nh2d_create_ensemble(int n_members, const nh_grid2d_desc* descs, const double* const* d0_host, void* ws,
                               size_t ws_bytes, void* stream, nh_grid2d** out)
{
    if (!out) return NH_ERR_ARG;
    *out = nullptr;
    const long long pitch = ens_pitch(n_members, descs);
    if (pitch == 0 || !d0_host || !ws) return NH_ERR_ARG;
    const int cpitch = mg_cpitch(n_members, descs);
    const size_t need = carve2(n_members, (int)pitch, cpitch, nullptr, nullptr);
    if (ws_bytes < need || ((uintptr_t)ws % kAlign2) != 0) return NH_ERR_ARG;
    for (int b = 0; b < n_members; ++b) {
        if (!d0_host[b]) return NH_ERR_ARG;
        const long long N = (long long)descs[b].nx * descs[b].ny;
        for (long long q = 0; q < N; ++q)
            if (!(d0_host[b][q] > 0.0) || !std::isfinite(d0_host[b][q])) return NH_ERR_ARG;
    }
    nh_grid2d* g = new (std::nothrow) nh_grid2d;
    if (!g) return NH_ERR_CUDA;
    g->nb = n_members;
    g->pitch = (int)pitch;
    g->d.assign(descs, descs + n_members);
    g->slide_h.assign(n_members, Slide2{0.0, 1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, NH_SLIDE_NONE, 0});
    g->member_set.assign(n_members, 0);
    g->stream = static_cast<cudaStream_t>(stream);
    g->cap_stream = nullptr;
    carve2(n_members, (int)pitch, cpitch, g, static_cast<char*>(ws));
    g->precond = NH_PRECOND_MG;
    g->mg_grid = 0;
    int dev = 0;
    cudaGetDevice(&dev);
    g->sms = 1;
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
    if (g->sms < 1) g->sms = 1;
    g->items_grid = (int)std::max(1LL, std::min((long long)g->maxch * g->nb, (long long)g->sms * 8));
    g->pcr_grid = (int)std::max(1LL, std::min((long long)g->maxpb * g->nb, (long long)g->sms * 2));
    g->egx = std::max(1, std::min((g->pitch + 255) / 256, (g->sms * 8 + g->nb - 1) / g->nb));
    g->ptile = -1;
    g->crit = NH_CRIT_GLOBAL; g->knh = 1e-3; g->enlarge = 1; g->first_global = 0;
    g->rtol = 1e-12; g->max_iter = 20000; g->guess = NH_GUESS_PREV;
    g->prec = NH_FP64;
    g->has_state = false;
    g->t_base = 0.0; g->last_dt = 0.0; g->n_since = 0; g->steps = 0; g->cur = 0; g->lcur = 0;
    g->graph[0] = g->graph[1] = nullptr;
    g->graph_valid = false; g->use_graphs = true; g->graph_runs = 0;
    g->prof_on = false; g->prof_used = 0;
    for (int k = 0; k < NH2_K_COUNT; ++k) { g->prof_ms[k] = 0.0; g->prof_launches[k] = 0; }
    std::memset(g->graph_key, 0, sizeof(g->graph_key));
    nh_status rc = NH_OK;
    cudaStream_t st = g->stream;
    do {
        const size_t pcr_smem = 2 * sizeof(float) * (size_t)kPcrRows;
        if (cudaFuncSetAttribute(k_pcr<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pcr_smem) != cudaSuccess ||
            cudaFuncSetAttribute(k_pcr_factor<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(3 * sizeof(float) * kPcrRows)) != cudaSuccess ||
            cudaFuncSetAttribute(k_pcg_persistent<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)pcr_smem) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        int coop = 0, per_sm = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
        g->coop_grid = 0;
        if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<double, float>,
                                                                  kPcrThreads, pcr_smem) == cudaSuccess &&
            per_sm > 0)
            g->coop_grid = per_sm * g->sms;
        per_sm = 0;
        if (cudaFuncSetAttribute(k2_mg_pcg, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMgSmemBytes) !=
                cudaSuccess ||
            fused_attributes() != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k2_mg_pcg, kMgThreads, kMgSmemBytes) ==
                        cudaSuccess &&
            per_sm > 0)
            g->mg_grid = std::min(per_sm * g->sms, kMgMaxGrid);
        int clk_khz = 0;
        cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
        g->barrier_budget = (long long)(clk_khz > 0 ? clk_khz : 2000000) * 1000LL;   // about one second
        g->barrier_budget_default = g->barrier_budget;
        if (cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
            g->cap_stream = nullptr; rc = NH_ERR_CUDA; break;
        }
        std::vector<Geo2> geo_h(n_members);
        for (int b = 0; b < n_members; ++b) geo_h[b] = geo2(descs[b]);
        if (cudaMemsetAsync(ws, 0, need, st) != cudaSuccess ||
            cudaMemcpyAsync(g->geos, geo_h.data(), sizeof(Geo2) * n_members, cudaMemcpyHostToDevice, st) !=
                cudaSuccess ||
            cudaMemcpyAsync(g->slides, g->slide_h.data(), sizeof(Slide2) * n_members, cudaMemcpyHostToDevice,
                            st) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        for (int b = 0; b < n_members && rc == NH_OK; ++b)
            if (cudaMemcpyAsync(g->d0 + (size_t)b * g->pitch, d0_host[b],
                                sizeof(double) * descs[b].nx * descs[b].ny, cudaMemcpyHostToDevice,
                                st) != cudaSuccess)
                rc = NH_ERR_CUDA;
        if (rc == NH_OK) {
            const size_t T = (size_t)n_members * g->pitch;
            k2_to_f32<<<(int)std::min<size_t>((T + 255) / 256, (size_t)g->sms * 8), 256, 0, st>>>(T, g->d0, g->d0f);
            if (cudaGetLastError() != cudaSuccess) rc = NH_ERR_CUDA;
        }
        // the host copies above are pageable: finish them before geo_h goes
        if (cudaStreamSynchronize(st) != cudaSuccess) rc = NH_ERR_CUDA;
    } while (0);
    if (rc != NH_OK) {
        if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
        delete g;
        return rc;
    }
    *out = g;
    return NH_OK;
}

nh_status nh2d_create(const nh_grid2d_desc* desc, const double* d0_host, void* ws, size_t ws_bytes,
                      void* stream, nh_grid2d** out)
{
    const double* d0s[1] = {d0_host};
    return nh2d_create_ensemble(1, desc, d0s, ws, ws_bytes, stream, out);
}

int nh2d_members(const nh_grid2d* g) { return g ? g->nb : 0; }

nh_status nh2d_set_member_bottom_motion(nh_grid2d* g, int m, const nh_slide2d_desc* s)
{
    if (!member_ok(g, m)) return NH_ERR_ARG;
    Slide2 S{0.0, 1.0, 1.0, 0.0, 0.0, 0.0, 1.0, 1.0, 1.0, NH_SLIDE_NONE, 0};
    if (s && s->shape != NH_SLIDE_NONE) {
        if (s->shape != NH_SLIDE_GAUSS_LNCOSH || !(s->Lx > 0.0) || !(s->Ly > 0.0) || !(s->t0 > 0.0) ||
            !std::isfinite(s->A) || !std::isfinite(s->xc0) || !std::isfinite(s->yc0) || !std::isfinite(s->s0))
            return NH_ERR_ARG;
        S.shape = NH_SLIDE_GAUSS_LNCOSH;
        S.A = s->A; S.Lx = s->Lx; S.Ly = s->Ly; S.xc0 = s->xc0; S.yc0 = s->yc0; S.s0 = s->s0; S.t0 = s->t0;
        S.iLx = 1.0 / s->Lx; S.iLy = 1.0 / s->Ly;
    }
    g->slide_h[m] = S;
    CK2(cudaMemcpyAsync(g->slides + m, &g->slide_h[m], sizeof(Slide2), cudaMemcpyHostToDevice, g->stream));
    CK2(cudaStreamSynchronize(g->stream));
    return NH_OK;
}

nh_status nh2d_set_bottom_motion(nh_grid2d* g, const nh_slide2d_desc* s)
{
    if (!g) return NH_ERR_ARG;
    for (int m = 0; m < g->nb; ++m) {
        const nh_status rc = nh2d_set_member_bottom_motion(g, m, s);
        if (rc != NH_OK) return rc;
    }
    return NH_OK;
}

nh_status nh2d_set_criterion(nh_grid2d* g, int kind, double k_nh, int enlarge, int first_step_global)
{
    if (!g || kind < NH_CRIT_GLOBAL || kind > NH_CRIT_W_X || !(k_nh > 0.0) || enlarge < 0 || enlarge > 16)
        return NH_ERR_ARG;
    g->crit = kind; g->knh = k_nh; g->enlarge = enlarge; g->first_global = first_step_global != 0;
    return NH_OK;
}

nh_status nh2d_set_solver(nh_grid2d* g, double rtol, int max_iter, int guess)
{
    if (!g || !(rtol > 0.0) || max_iter < 1 || (guess != NH_GUESS_ZERO && guess != NH_GUESS_PREV))
        return NH_ERR_ARG;
    g->rtol = rtol; g->max_iter = max_iter; g->guess = guess;
    return NH_OK;
}

nh_status nh2d_set_graphs(nh_grid2d* g, int on)
{
    if (!g) return NH_ERR_ARG;
    g->use_graphs = on != 0;
    if (!g->use_graphs) graph_destroy(g);
    return NH_OK;
}

nh_status nh2d_set_tile(nh_grid2d* g, int tile, int* chosen)
{
    if (!g || tile < -2 || tile > 3) return NH_ERR_ARG;
    if (tile >= 0 || tile == -2) {
        g->ptile = tile >= 0 ? tile : -1;
        graph_destroy(g);
    }
    if (chosen) *chosen = g->ptile;
    return NH_OK;
}

nh_status nh2d_set_profiling(nh_grid2d* g, int enable)
{
    if (!g) return NH_ERR_ARG;
    CK2(cudaStreamSynchronize(g->stream));
    g->prof_used = 0;
    g->prof_on = enable != 0;
    for (int k = 0; k < NH2_K_COUNT; ++k) { g->prof_ms[k] = 0.0; g->prof_launches[k] = 0; }
    return NH_OK;
}

nh_status nh2d_get_profile(nh_grid2d* g, double* ms, long long* launches)
{
    if (!g || !ms || !launches) return NH_ERR_ARG;
    CK2(cudaStreamSynchronize(g->stream));
    prof2_fold(g);
    for (int k = 0; k < NH2_K_COUNT; ++k) { ms[k] = g->prof_ms[k]; launches[k] = g->prof_launches[k]; }
    return NH_OK;
}

nh_status nh2d_set_preconditioner(nh_grid2d* g, int kind)
{
    if (!g || (kind != NH_PRECOND_LINE && kind != NH_PRECOND_MG)) return NH_ERR_ARG;
    g->precond = kind;
    graph_destroy(g);
    return NH_OK;
}

nh_status nh2d_set_wait_budget(nh_grid2d* g, long long cycles)
{
    if (!g || cycles < 0) return NH_ERR_ARG;
    g->barrier_budget = cycles > 0 ? cycles : g->barrier_budget_default;
    graph_destroy(g);
    return NH_OK;
}

nh_status nh2d_set_precision(nh_grid2d* g, int precision)
{
    if (!g || (precision != NH_FP64 && precision != NH_MIXED_FP64_SOLVE)) return NH_ERR_ARG;
    if (precision != g->prec) {
        g->prec = precision;
        graph_destroy(g);
        std::fill(g->member_set.begin(), g->member_set.end(), 0);
        g->has_state = false;
    }
    return NH_OK;
}

nh_status nh2d_set_member_state(nh_grid2d* g, int m, const double* h, const double* hu, const double* hv,
                                const double* hw, double t)
{
    if (!member_ok(g, m) || !h || !hu || !hv || !hw || !std::isfinite(t)) return NH_ERR_ARG;
    const size_t N = (size_t)g->d[m].nx * g->d[m].ny;
    for (size_t q = 0; q < N; ++q)
        if (!(h[q] > 0.0) || !std::isfinite(h[q]) || !std::isfinite(hu[q]) || !std::isfinite(hv[q]) ||
            !std::isfinite(hw[q]))
            return NH_ERR_ARG;
    cudaStream_t st = g->stream;
    const size_t mo = (size_t)m * g->pitch;
    const double* src[4] = {h, hu, hv, hw};
    if (g->prec == NH_FP64) {
        for (int f = 0; f < 4; ++f)
            CK2(cudaMemcpyAsync(g->q[g->cur][f] + mo, src[f], sizeof(double) * N, cudaMemcpyHostToDevice, st));
    } else {   // through the FP64 scratch of the stage buffers, then zeta = h - d0 etc. in FP32
        for (int f = 0; f < 4; ++f)
            CK2(cudaMemcpyAsync(g->qs[f] + mo, src[f], sizeof(double) * N, cudaMemcpyHostToDevice, st));
        const int grid = (int)std::min<size_t>((N + 255) / 256, (size_t)g->sms * 8);
        k2_store_f32<<<grid, 256, 0, st>>>((int)N, g->d0 + mo, g->qs[0] + mo, g->qs[1] + mo, g->qs[2] + mo,
                                           g->qs[3] + mo, as<float>(g->q[g->cur][0]) + mo,
                                           as<float>(g->q[g->cur][1]) + mo, as<float>(g->q[g->cur][2]) + mo,
                                           as<float>(g->q[g->cur][3]) + mo);
        CK2(cudaGetLastError());
    }
    CK2(cudaMemsetAsync(g->psi + mo, 0, sizeof(double) * g->pitch, st));
    CK2(cudaMemsetAsync(g->nact[0] + m, 0, sizeof(int), st));
    CK2(cudaMemsetAsync(g->nact[1] + m, 0, sizeof(int), st));
    CK2(cudaMemsetAsync(g->act + mo, 0, g->pitch, st));
    CK2(cudaStreamSynchronize(st));
    g->member_set[m] = 1;
    g->has_state = std::all_of(g->member_set.begin(), g->member_set.end(), [](char c) { return c != 0; });
    g->t_base = t; g->n_since = 0; g->steps = 0; g->last_dt = 0.0;
    return NH_OK;
}

nh_status nh2d_put_member_state(nh_grid2d* g, int m, const double* h, const double* hu, const double* hv,
                                const double* hw)
{
    if (!member_ok(g, m) || !h || !hu || !hv || !hw) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    cudaStream_t st = g->stream;
    const size_t N = (size_t)g->d[m].nx * g->d[m].ny;
    const size_t mo = (size_t)m * g->pitch;
    const double* src[4] = {h, hu, hv, hw};
    if (g->prec == NH_FP64) {
        for (int f = 0; f < 4; ++f)
            CK2(cudaMemcpyAsync(g->q[g->cur][f] + mo, src[f], sizeof(double) * N, cudaMemcpyHostToDevice, st));
    } else {
        for (int f = 0; f < 4; ++f)
            CK2(cudaMemcpyAsync(g->qs[f] + mo, src[f], sizeof(double) * N, cudaMemcpyHostToDevice, st));
        const int grid = (int)std::min<size_t>((N + 255) / 256, (size_t)g->sms * 8);
        k2_store_f32<<<grid, 256, 0, st>>>((int)N, g->d0 + mo, g->qs[0] + mo, g->qs[1] + mo, g->qs[2] + mo,
                                           g->qs[3] + mo, as<float>(g->q[g->cur][0]) + mo,
                                           as<float>(g->q[g->cur][1]) + mo, as<float>(g->q[g->cur][2]) + mo,
                                           as<float>(g->q[g->cur][3]) + mo);
        CK2(cudaGetLastError());
    }
    return NH_OK;
}

nh_status nh2d_set_state(nh_grid2d* g, const double* h, const double* hu, const double* hv, const double* hw,
                         double t)
{
    return nh2d_set_member_state(g, 0, h, hu, hv, hw, t);
}

nh_status nh2d_get_member_state(nh_grid2d* g, int m, double* h, double* hu, double* hv, double* hw, double* p_nh)
{
    if (!member_ok(g, m)) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    cudaStream_t st = g->stream;
    const size_t N = (size_t)g->d[m].nx * g->d[m].ny;
    const size_t mo = (size_t)m * g->pitch;
    double* dst[4] = {h, hu, hv, hw};
    double* srcs[4] = {g->q[g->cur][0] + mo, g->q[g->cur][1] + mo, g->q[g->cur][2] + mo, g->q[g->cur][3] + mo};
    if (g->prec != NH_FP64) {   // FP32 storage -> FP64 (h = zeta + d0) in the stage scratch
        for (int f = 0; f < 4; ++f) srcs[f] = g->qs[f] + mo;
        const int grid = (int)std::min<size_t>((N + 255) / 256, (size_t)g->sms * 8);
        k2_load_f32<<<grid, 256, 0, st>>>((int)N, g->d0 + mo, as<float>(g->q[g->cur][0]) + mo,
                                          as<float>(g->q[g->cur][1]) + mo, as<float>(g->q[g->cur][2]) + mo,
                                          as<float>(g->q[g->cur][3]) + mo, srcs[0], srcs[1], srcs[2], srcs[3]);
        CK2(cudaGetLastError());
    }
    for (int f = 0; f < 4; ++f)
        if (dst[f]) CK2(cudaMemcpyAsync(dst[f], srcs[f], sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    std::vector<double> hh, ps;
    if (p_nh) {
        hh.resize(N); ps.resize(N);
        CK2(cudaMemcpyAsync(hh.data(), srcs[0], sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        CK2(cudaMemcpyAsync(ps.data(), g->psi + mo, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    }
    CK2(cudaStreamSynchronize(st));
    if (p_nh) {
        const double sc = g->last_dt > 0.0 ? g->d[m].rho / g->last_dt : 0.0;   // p = rho psi / (dt h)
        for (size_t q = 0; q < N; ++q) p_nh[q] = sc * ps[q] / hh[q];
    }
    return NH_OK;
}

nh_status nh2d_get_state(nh_grid2d* g, double* h, double* hu, double* hv, double* hw, double* p_nh)
{
    return nh2d_get_member_state(g, 0, h, hu, hv, hw, p_nh);
}

nh_status nh2d_get_member_mask(nh_grid2d* g, int m, unsigned char* mask)
{
    if (!member_ok(g, m) || !mask) return NH_ERR_ARG;
    const size_t N = (size_t)g->d[m].nx * g->d[m].ny;
    CK2(cudaMemcpyAsync(mask, g->act + (size_t)m * g->pitch, N, cudaMemcpyDeviceToHost, g->stream));
    CK2(cudaStreamSynchronize(g->stream));
    return NH_OK;
}

nh_status nh2d_get_mask(nh_grid2d* g, unsigned char* mask) { return nh2d_get_member_mask(g, 0, mask); }

nh_status nh2d_get_member_info(nh_grid2d* g, int m, nh_step_info* info)
{
    if (!member_ok(g, m) || !info) return NH_ERR_ARG;
    MState s;
    std::vector<double> mp(g->nmass);
    CK2(cudaMemcpyAsync(&s, g->ms + m, sizeof(MState), cudaMemcpyDeviceToHost, g->stream));
    CK2(cudaMemcpyAsync(mp.data(), g->mass_part + (size_t)m * g->nmass, sizeof(double) * g->nmass,
                        cudaMemcpyDeviceToHost, g->stream));
    CK2(cudaStreamSynchronize(g->stream));
    double mass = 0.0;
    for (double v : mp) mass += v;
    info->step = g->steps;
    info->t = g->t_base + (double)g->n_since * g->last_dt;
    info->n_active = s.n_active;
    info->n_active_max = s.n_active;
    info->iters = s.iters;
    info->ir_passes = 0;
    info->solver = s.n_active == 0 ? -1 : s.kind;
    info->status = s.status;
    info->rel_res = s.rel_res;
    info->min_gamma = s.n_active > 0 ? s.min_gamma : 0.0;
    info->mass = mass;
    return NH_OK;
}

nh_status nh2d_step(nh_grid2d* g, double dt, nh_step_info* info)
{
    if (!g) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    if (!(dt > 0.0) || !std::isfinite(dt)) return NH_ERR_ARG;
    return step2(g, dt, info);
}

nh_status nh2d_run(nh_grid2d* g, double dt, long long n_steps, nh_run_info* info)
{
    if (!g || n_steps < 0) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    if (!(dt > 0.0) || !std::isfinite(dt)) return NH_ERR_ARG;
    nh_run_info R;
    std::memset(&R, 0, sizeof(R));
    nh_status rc = NH_OK;
    // a first step that is global by request runs on its own
    if (n_steps > 0 && g->first_global && g->steps == 0) {
        nh_step_info si;
        std::memset(&si, 0, sizeof(si));
        rc = step2(g, dt, &si);
        R.last = si;
        if (rc != NH_OK) {
            if (info) *info = R;
            return rc;
        }
        R.steps = 1; R.iters_total = si.iters; R.active_total = si.n_active;
        n_steps -= 1;
    }
    if (n_steps > 0 && graph_eligible(g, dt)) {
        nh_run_info Rg;
        std::memset(&Rg, 0, sizeof(Rg));
        rc = graph_run(g, dt, n_steps, &Rg);
        R.steps += Rg.steps; R.iters_total += Rg.iters_total; R.active_total += Rg.active_total;
        R.last = Rg.last;
        if (rc == NH_OK || Rg.steps == n_steps) {
            if (info) *info = R;
            return rc;
        }
        // a step failed inside the captured run: redo it step by step (this
        // also gives members whose CG broke down their BiCGStab fallback)
        n_steps -= Rg.steps;
        rc = NH_OK;
    }
    for (long long k = 0; k < n_steps; ++k) {
        nh_step_info si;
        std::memset(&si, 0, sizeof(si));
        rc = step2(g, dt, &si);
        R.last = si;
        if (rc != NH_OK) break;
        R.steps += 1;
        R.iters_total += si.iters;
        R.active_total += si.n_active;
    }
    if (info) *info = R;
    return rc;
}

long long nh2d_graph_runs(const nh_grid2d* g) { return g ? g->graph_runs : -1; }

void nh2d_destroy(nh_grid2d* g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    graph_destroy(g);
    for (cudaEvent_t e : g->prof_pool) cudaEventDestroy(e);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
}

}  // extern "C"
