// nh_api.cu -- host runtime behind include/nhswe.h (1D batched path).
//
// The handle carves every device buffer out of the caller's workspace, keeps
// two state buffers (Q^n and Q~/Q^{n+1}) and two active lists (this step and
// the previous one), and runs one step as a fixed sequence of kernels on the
// caller's stream.  The Krylov loop is driven from the host; the number of
// members still iterating is read back every `poll_every` iterations.
#include <cmath>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <array>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "nh_cnn.cuh"
#include "nh_kernels1d.cuh"

using namespace nh;

struct nh_grid {
    nh_grid_desc d;
    cudaStream_t stream;
    int nx, nb, pitch, wpitch, ntiles, maxch, sm_count, items_grid, pcr_grid;
    int coop_grid[2];            // persistent PCG CTAs (FP64 / FP32 vectors), 0 = unavailable
    int tile;                    // predictor tile (cells per CTA), chosen by the autotuner
    bool tuned;
    long long barrier_budget;    // clock cycles a grid barrier may spin
    long long barrier_budget_default;
    size_t es;                   // element size of the Krylov vectors
    bool mixed;                  // FP32 state and predictor (NH_MIXED, NH_MIXED_FP64_SOLVE)
    bool ir_mode;                // FP32 Krylov inside FP64 refinement (NH_MIXED)
    bool uneven;                 // members have different cell counts
    std::vector<int> nxh;        // cells per member
    std::vector<long long> offh; // host layout: member b at [offh[b], offh[b+1])
    long long ncells;            // sum of nxh
    int* nxd;                    // device copy of nxh
    long long* offd;             // device copy of offh
    void* ws_base;               // the caller's workspace
    TimeCtl* tc;                 // device time control of captured runs
    cudaStream_t cap_stream;     // private stream used only to capture graphs
    cudaGraphExec_t graph[2];    // one captured step per state-buffer parity
    bool graph_valid;
    double graph_key[12];        // settings the graphs were captured with
    int graph_runs;              // nh_run calls served by graphs (diagnostics)
    bool use_graphs;             // nh_run may replay captured graphs
    double mass0;                // sum of d0 dx over all members (FP64)
    // configuration
    int crit, enlarge, first_global;
    double knh;
    int solver, max_iter, guess, ir_max, precond, maxpb;
    double rtol, inner_rtol;
    int poll_every;
    // run state
    bool has_state;
    double t_base;               // time at the last (re)basing
    long long n_since;           // steps since t_base
    long long steps;             // steps since nh_set_state
    double last_dt;              // dt of the last completed step (0: none)
    int cur;                     // state buffer holding Q^n
    int lcur;                    // list buffer of the previous step
    // device buffers (inside the workspace)
    void* sz[2]; void* shu[2]; void* shw[2];   // zeta = h - d0, hu, hw (type T)
    void* d0;                                  // static depth (type T)
    double* d0d;                               // static depth (FP64)
    double* stage;                             // 3 * nb * nx FP64 host-layout staging
    Slide* slide; Kin* kin;
    uint32_t* marks; uint32_t* act;
    int* list[2]; int* nact[2];
    int2* items; int2* pitems;                 // work lists of the step
    double *diag, *offl, *offr, *R;            // FP64 operator and right-hand side
    float *diag32, *offl32, *offr32, *rhs32;   // mixed: FP32 operator and inner rhs
    void *c6, *cx, *phi, *ddx;                 // correction coefficients (type T)
    int *nbl, *nbr;
    void *x, *r, *p0, *p1, *q, *rh, *v0, *v1, *s, *t, *r1, *z;   // Krylov vectors (type T)
    double* x64;                               // mixed: FP64 outer iterate
    float2* pf; float* prb;                    // line preconditioner factors of the current solve
    IRState* ir;
    double* psi;
    MState* ms; Ctl* ctl; double* part; int* cnt;
    double* mass_part; Summary* summary;
    // learned guess (nh_cnn_attach): solution history, features, network
    bool cnn_attached, cnn_record;
    cnn::GuessBufs cnn;
    // profiling: event pairs recorded around launches, folded in at syncs
    bool prof_on;
    double prof_ms[NH_K_COUNT];
    long long prof_launches[NH_K_COUNT];
    std::vector<cudaEvent_t> prof_pool;
    std::vector<int> prof_kind;        // kind of each recorded pair
    size_t prof_used;                  // pairs recorded since the last fold
};

namespace {

constexpr size_t kAlign = 256;

struct Carver {
    char* base;
    size_t off = 0;
    void* take(size_t bytes)
    {
        off = (off + kAlign - 1) / kAlign * kAlign;
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    }
};

bool desc_ok(const nh_grid_desc* d)
{
    if (!d) return false;
    if (d->dim != 1) return false;
    if (d->nx < 8 || d->nx > (1 << 20)) return false;
    if (d->nbatch < 1 || d->nbatch > 65535) return false;
    if ((long long)d->nx * d->nbatch > (1LL << 30)) return false;
    if (d->bc != NH_BC_WALL && d->bc != NH_BC_PERIODIC) return false;
    if (d->precision != NH_FP64 && d->precision != NH_MIXED && d->precision != NH_MIXED_FP64_SOLVE) return false;
    if (d->limiter < NH_LIM_NONE || d->limiter > NH_LIM_MC) return false;
    if (!(d->dx > 0.0) || !(d->g > 0.0) || !(d->rho > 0.0) || !std::isfinite(d->x0)) return false;
    return true;
}

// Lay out every buffer; with base == nullptr only the size is computed.  d.nx
// is the largest member's cell count; ncells the sum over members.
size_t carve(const nh_grid_desc& d, long long ncells, nh_grid* g, char* base)
{
    const int nx = d.nx, nb = d.nbatch;
    const bool mixed = d.precision != NH_FP64;
    const bool ir_mode = d.precision == NH_MIXED;
    const int pitch = (nx + kPredTileMax - 1) / kPredTileMax * kPredTileMax;
    const int wpitch = pitch / 32;
    const int ntiles = pitch / kPredTile;
    const int ntiles_max = pitch / kPredTileMin;
    const int maxch = (nx + kChunk - 1) / kChunk;
    const int maxpb = (nx + kPcrRows - 1) / kPcrRows;
    const size_t N = (size_t)nb * pitch;
    const size_t es = mixed ? 4 : 8;        // state and correction coefficients
    const size_t ev = ir_mode ? 4 : 8;      // Krylov vectors
    Carver c{base};
    nh_grid tmp;
    nh_grid* G = g ? g : &tmp;
    for (int k = 0; k < 2; ++k) {
        G->sz[k] = c.take(N * es); G->shu[k] = c.take(N * es); G->shw[k] = c.take(N * es);
    }
    G->d0 = c.take(N * es);
    G->d0d = (double*)c.take(N * 8);
    G->stage = (double*)c.take(3 * (size_t)ncells * 8);
    G->nxd = (int*)c.take(sizeof(int) * nb);
    G->offd = (long long*)c.take(sizeof(long long) * (nb + 1));
    G->slide = (Slide*)c.take(sizeof(Slide) * nb);
    G->kin = (Kin*)c.take(sizeof(Kin) * nb);
    G->marks = (uint32_t*)c.take(sizeof(uint32_t) * (size_t)nb * wpitch);
    G->act = (uint32_t*)c.take(sizeof(uint32_t) * (size_t)nb * wpitch);
    for (int k = 0; k < 2; ++k) {
        G->list[k] = (int*)c.take(sizeof(int) * N);
        G->nact[k] = (int*)c.take(sizeof(int) * nb);
    }
    G->items = (int2*)c.take(sizeof(int2) * (size_t)nb * maxch);
    G->pitems = (int2*)c.take(sizeof(int2) * (size_t)nb * maxpb);
    G->diag = (double*)c.take(N * 8); G->offl = (double*)c.take(N * 8);
    G->offr = (double*)c.take(N * 8); G->R = (double*)c.take(N * 8);
    if (ir_mode) {
        G->diag32 = (float*)c.take(N * 4); G->offl32 = (float*)c.take(N * 4);
        G->offr32 = (float*)c.take(N * 4); G->rhs32 = (float*)c.take(N * 4);
        G->x64 = (double*)c.take(N * 8);
        G->ir = (IRState*)c.take(sizeof(IRState) * nb);
    } else {
        G->diag32 = G->offl32 = G->offr32 = G->rhs32 = nullptr;
        G->x64 = nullptr;
        G->ir = nullptr;
    }
    G->c6 = c.take(N * es); G->cx = c.take(N * es); G->phi = c.take(N * es); G->ddx = c.take(N * es);
    G->nbl = (int*)c.take(sizeof(int) * N); G->nbr = (int*)c.take(sizeof(int) * N);
    G->x = c.take(N * ev); G->r = c.take(N * ev); G->p0 = c.take(N * ev); G->p1 = c.take(N * ev);
    G->q = c.take(N * ev); G->rh = c.take(N * ev); G->v0 = c.take(N * ev); G->v1 = c.take(N * ev);
    G->s = c.take(N * ev); G->t = c.take(N * ev);
    G->r1 = c.take(N * ev); G->z = c.take(N * ev);
    G->psi = (double*)c.take(sizeof(double) * N);
    G->pf = (float2*)c.take(sizeof(float2) * kPcrLevels * N);
    G->prb = (float*)c.take(sizeof(float) * N);
    G->ms = (MState*)c.take(sizeof(MState) * nb);
    G->ctl = (Ctl*)c.take(sizeof(Ctl));
    G->part = (double*)c.take(sizeof(double) * 4 * (size_t)nb * maxch);
    G->cnt = (int*)c.take(sizeof(int) * nb);
    G->mass_part = (double*)c.take(sizeof(double) * (size_t)nb * ntiles_max);
    G->summary = (Summary*)c.take(sizeof(Summary));
    G->tc = (TimeCtl*)c.take(sizeof(TimeCtl));
    if (g) {
        g->nx = nx; g->nb = nb; g->pitch = pitch; g->wpitch = wpitch; g->ntiles = ntiles;
        g->maxch = maxch; g->es = ev; g->maxpb = maxpb; g->mixed = mixed; g->ir_mode = ir_mode;
    }
    return (c.off + kAlign - 1) / kAlign * kAlign;
}

#define CK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return NH_ERR_CUDA;      \
    } while (0)

void prof_pre(nh_grid* g, int kind)
{
    g->prof_launches[kind] += 1;
    if (!g->prof_on) return;
    const size_t need = 2 * (g->prof_used + 1);
    while (g->prof_pool.size() < need) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) { g->prof_on = false; return; }
        g->prof_pool.push_back(e);
    }
    if (g->prof_kind.size() < g->prof_used + 1) g->prof_kind.resize(g->prof_used + 1);
    g->prof_kind[g->prof_used] = kind;
    cudaEventRecord(g->prof_pool[2 * g->prof_used], g->stream);
}

void prof_post(nh_grid* g)
{
    if (!g->prof_on || g->prof_pool.size() < 2 * (g->prof_used + 1)) return;
    cudaEventRecord(g->prof_pool[2 * g->prof_used + 1], g->stream);
    g->prof_used += 1;
}

// Called after a stream synchronisation: every recorded pair is complete.
void prof_fold(nh_grid* g)
{
    for (size_t q = 0; q < g->prof_used; ++q) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, g->prof_pool[2 * q], g->prof_pool[2 * q + 1]) == cudaSuccess)
            g->prof_ms[g->prof_kind[q]] += ms;
    }
    g->prof_used = 0;
}

#define LAUNCH(kind, ...)          \
    do {                           \
        prof_pre(g, kind);         \
        __VA_ARGS__;               \
        prof_post(g);              \
    } while (0)

// synchronise the handle's stream and fold profiler events
#define SYNC()                                                     \
    do {                                                           \
        if (cudaStreamSynchronize(g->stream) != cudaSuccess)       \
            return NH_ERR_CUDA;                                    \
        prof_fold(g);                                              \
    } while (0)

template <typename T, int TILE>
cudaError_t predict_launch_t(int nb, int ntiles, cudaStream_t st, const PredArgs<T>& pa)
{
    k_predict<T, TILE><<<dim3(ntiles, nb), TILE, predict_smem_bytes<T, TILE>(), st>>>(pa);
    return cudaGetLastError();
}

// k_predict with the handle's tile; pa.G.ntiles must match the tile.
template <typename T>
cudaError_t predict_launch(int tile, int nb, int ntiles, cudaStream_t st, const PredArgs<T>& pa)
{
    switch (tile) {
    case 128: return predict_launch_t<T, 128>(nb, ntiles, st, pa);
    case 512: return predict_launch_t<T, 512>(nb, ntiles, st, pa);
    default: return predict_launch_t<T, 256>(nb, ntiles, st, pa);
    }
}

template <typename T>
cudaError_t predict_set_smem()
{
    cudaError_t e = cudaFuncSetAttribute(k_predict<T, 128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)predict_smem_bytes<T, 128>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_predict<T, 256>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)predict_smem_bytes<T, 256>());
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_predict<T, 512>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)predict_smem_bytes<T, 512>());
    return e;
}

Geo geo(const nh_grid* g)
{
    Geo G;
    G.nx = g->nx; G.nb = g->nb; G.pitch = g->pitch; G.wpitch = g->wpitch; G.bc = g->d.bc;
    G.lim = g->d.limiter; G.ntiles = g->pitch / g->tile; G.maxch = g->maxch;
    G.dx = g->d.dx; G.x0 = g->d.x0; G.g = g->d.g; G.idx = 1.0 / g->d.dx;
    G.i2dx = 1.0 / (2.0 * g->d.dx); G.idx2 = 1.0 / (g->d.dx * g->d.dx);
    G.nxv = g->uneven ? g->nxd : nullptr;
    return G;
}

// Krylov arguments over the vectors of type T; `diag`, `offl`, `offr`, `R`
// select the operator (FP64 for the FP64 path, FP32 copies for the inner
// solve of the mixed path).
template <typename T>
SolveArgs<T> solve_args(nh_grid* g, int lcur, const T* diag, const T* offl, const T* offr, const T* R,
                        double rtol)
{
    SolveArgs<T> a;
    a.nb = g->nb; a.pitch = g->pitch; a.maxch = g->maxch;
    a.list = g->list[lcur];
    a.diag = diag; a.offl = offl; a.offr = offr; a.R = R;
    a.nbl = g->nbl; a.nbr = g->nbr;
    a.psi_prev = g->psi; a.guess_scale = 0.0;
    a.x = (T*)g->x; a.r = (T*)g->r; a.p0 = (T*)g->p0; a.p1 = (T*)g->p1;
    a.q = (T*)g->q; a.rh = (T*)g->rh; a.v0 = (T*)g->v0; a.v1 = (T*)g->v1;
    a.s = (T*)g->s; a.t = (T*)g->t;
    a.r1 = (T*)g->r1; a.z = (T*)g->z; a.maxpb = g->maxpb;
    a.pf = g->pf; a.prb = g->prb; a.pf_stride = (size_t)g->nb * g->pitch;
    a.n_ext = 0; a.ext_c = nullptr; a.ext_k = nullptr; a.ext_stride = 0;
    a.items = g->items; a.pitems = g->pitems;
    a.tc = nullptr;
    a.ms = g->ms; a.ctl = g->ctl; a.part = g->part; a.cnt = g->cnt;
    a.rtol = rtol; a.max_iter = g->max_iter; a.it = 0;
    return a;
}

// Learned-guess geometry of the step whose mask bits are in g->act.
cnn::GuessGeo guess_geo(const nh_grid* g, const TimeCtl* tc)
{
    cnn::GuessGeo G;
    G.nb = g->nb; G.pitch = g->pitch; G.wpitch = g->wpitch; G.nxv = g->nxd; G.act = g->act;
    G.psi = g->psi; G.tc = tc; G.sms = g->sm_count;
    return G;
}

bool cnn_features_on(const nh_grid* g)
{
    return g->cnn_attached && (g->guess == NH_GUESS_CNN || g->cnn_record);
}

// Judge the three starting points of the solve (previous pressure,
// extrapolation, extrapolation + network) by their initial residual with the
// FP64 operator just assembled, and copy each member's winner into the guess.
cudaError_t judge_launch(nh_grid* g, int lnew, double gscale, const TimeCtl* tc, cudaStream_t st)
{
    JudgeArgs ja;
    ja.pitch = g->pitch; ja.stride = (size_t)g->nb * g->maxch;
    ja.list = g->list[lnew]; ja.nbl = g->nbl; ja.nbr = g->nbr;
    ja.diag = g->diag; ja.offl = g->offl; ja.offr = g->offr; ja.R = g->R;
    ja.cand0 = g->psi; ja.cand1 = g->cnn.base; ja.cand2 = g->cnn.guess;
    ja.guess_scale = gscale; ja.tc = tc;
    ja.items = g->items; ja.ms = g->ms; ja.ctl = g->ctl; ja.part = g->part; ja.cnt = g->cnt;
    ja.choice = g->cnn.choice; ja.counts = g->cnn.ctl->counts;
    k_guess_judge<<<g->items_grid, kChunk, 0, st>>>(ja);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cnn::launch_select(g->cnn, guess_geo(g, tc), st);
}

// Krylov solve on the active cells with the vectors of type T: set-up, then
// iterations until every member finished (read back every poll_every).
template <typename T>
nh_status krylov_pass(nh_grid* g, SolveArgs<T>& sa);

// Krylov solve; AUTO members whose CG broke down are solved again by BiCGStab.
template <typename T>
nh_status krylov(nh_grid* g, SolveArgs<T>& sa)
{
    cudaStream_t st = g->stream;
    CK(cudaMemsetAsync(&g->ctl->n_fallback, 0, sizeof(int), st));
    nh_status rc = krylov_pass<T>(g, sa);
    if (rc != NH_OK) return rc;
    int nfb = 0;
    CK(cudaMemcpyAsync(&nfb, &g->ctl->n_fallback, sizeof(int), cudaMemcpyDeviceToHost, st));
    SYNC();
    if (nfb == 0) return NH_OK;
    k_fallback_reset<<<(g->nb + 127) / 128, 128, 0, st>>>(g->ms, g->nb);
    CK(cudaGetLastError());
    return krylov_pass<T>(g, sa);
}

template <typename T>
nh_status krylov_pass(nh_grid* g, SolveArgs<T>& sa)
{
    cudaStream_t st = g->stream;
    CK(cudaMemsetAsync(g->ctl, 0, 3 * sizeof(int), st));
    CK(cudaMemsetAsync(g->cnt, 0, sizeof(int) * g->nb, st));
    LAUNCH(NH_K_SOLVE_INIT, k_solve_init<T><<<g->items_grid, kChunk, 0, st>>>(sa));
    Ctl hctl;
    CK(cudaMemcpyAsync(&hctl, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    SYNC();
    const bool pcg = g->precond == NH_PRECOND_LINE;
    const size_t pcr_smem = 2 * sizeof(float) * (size_t)kPcrRows;
    if (pcg && (hctl.n_cg > 0 || hctl.n_bicg > 0))
        LAUNCH(NH_K_PRECOND, k_pcr_factor<T, float><<<g->pcr_grid, kPcrThreads, 3 * sizeof(float) * kPcrRows, st>>>(sa));
    if (hctl.n_cg > 0 && pcg) {
        sa.it = 0;
        LAUNCH(NH_K_PRECOND, k_pcr<T, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_PCG));
    }
    if (hctl.not_done <= 0) return NH_OK;
    const int cg = g->coop_grid[sizeof(T) == 8 ? 0 : 1];
    if (pcg && hctl.n_cg > 0 && hctl.n_bicg == 0 && cg > 0) {
        // every PCG iteration in one cooperative launch, no host round trip
        CK(cudaMemsetAsync(&g->ctl->timeout, 0, 3 * sizeof(int), st));   // timeout, bar_count, bar_gen
        long long budget = g->barrier_budget;
        void* args[] = {(void*)&sa, (void*)&budget};
        prof_pre(g, NH_K_PCG_LOOP);
        cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_pcg_persistent<T, float>, dim3(cg),
                                                    dim3(kPcrThreads), args, pcr_smem, st);
        prof_post(g);
        if (e != cudaSuccess) return NH_ERR_CUDA;
        int to = 0;
        CK(cudaMemcpyAsync(&to, &g->ctl->timeout, sizeof(int), cudaMemcpyDeviceToHost, st));
        SYNC();
        return to ? NH_ERR_TIMEOUT : NH_OK;
    }
    for (int it = 1; it <= g->max_iter; ++it) {
        sa.it = it;
        if (hctl.n_cg > 0 && pcg) {
            LAUNCH(NH_K_PCG_A, k_pcg_a<T><<<g->items_grid, kChunk, 0, st>>>(sa));
            LAUNCH(NH_K_PRECOND, k_pcr<T, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_PCG_STEP));
        } else if (hctl.n_cg > 0) {
            LAUNCH(NH_K_CG_A, k_cg_a<T><<<g->items_grid, kChunk, 0, st>>>(sa));
            LAUNCH(NH_K_CG_B, k_cg_b<T><<<g->items_grid, kChunk, 0, st>>>(sa));
        }
        if (hctl.n_bicg > 0 && pcg) {
            LAUNCH(NH_K_PRECOND, k_pcr<T, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_BI_P));
            LAUNCH(NH_K_BI_1, k_pbi_mv<T><<<g->items_grid, kChunk, 0, st>>>(sa, 0));
            LAUNCH(NH_K_PRECOND, k_pcr<T, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_BI_S));
            LAUNCH(NH_K_BI_2, k_pbi_mv<T><<<g->items_grid, kChunk, 0, st>>>(sa, 1));
            LAUNCH(NH_K_BI_3, k_pbi_upd<T><<<g->items_grid, kChunk, 0, st>>>(sa));
        } else if (hctl.n_bicg > 0) {
            LAUNCH(NH_K_BI_1, k_bi_1<T><<<g->items_grid, kChunk, 0, st>>>(sa));
            LAUNCH(NH_K_BI_2, k_bi_2<T><<<g->items_grid, kChunk, 0, st>>>(sa));
            LAUNCH(NH_K_BI_3, k_bi_3<T><<<g->items_grid, kChunk, 0, st>>>(sa));
        }
        if (it % g->poll_every == 0 || it == g->max_iter) {
            int nd = 0;
            CK(cudaMemcpyAsync(&nd, &g->ctl->not_done, sizeof(int), cudaMemcpyDeviceToHost, st));
            SYNC();
            if (nd <= 0) break;
        }
    }
    return NH_OK;
}

// Mixed path: FP64 iterative refinement around FP32 Krylov solves.
nh_status refine(nh_grid* g, int lnew, double guess_scale, const double* guess_src)
{
    cudaStream_t st = g->stream;
    IRArgs ia;
    ia.nb = g->nb; ia.pitch = g->pitch; ia.maxch = g->maxch;
    ia.list = g->list[lnew]; ia.nbl = g->nbl; ia.nbr = g->nbr;
    ia.diag = g->diag; ia.offl = g->offl; ia.offr = g->offr; ia.R = g->R;
    ia.psi_prev = guess_src; ia.guess_scale = guess_scale;
    ia.x64 = g->x64; ia.e32 = (const float*)g->x; ia.rhs32 = g->rhs32;
    ia.ms = g->ms; ia.ir = g->ir; ia.ctl = g->ctl; ia.part = g->part; ia.cnt = g->cnt;
    ia.rtol = g->rtol; ia.ir_max = g->ir_max; ia.items = g->items;
    SolveArgs<float> sa = solve_args<float>(g, lnew, g->diag32, g->offl32, g->offr32, g->rhs32,
                                            g->inner_rtol);
    const size_t total = (size_t)g->nb * g->pitch;
    const int egrid = (int)std::min<size_t>((total + 255) / 256, (size_t)g->sm_count * 8);
    for (int pass = 0; pass <= g->ir_max; ++pass) {
        ia.pass = pass;
        if (pass > 0) LAUNCH(NH_K_CORRECT, k_ir_update<<<egrid, 256, 0, st>>>(ia));
        CK(cudaMemsetAsync(&g->ctl->ir_pending, 0, sizeof(int), st));
        LAUNCH(NH_K_SOLVE_INIT, k_ir_resid<<<g->items_grid, kChunk, 0, st>>>(ia));
        int pending = 0;
        CK(cudaMemcpyAsync(&pending, &g->ctl->ir_pending, sizeof(int), cudaMemcpyDeviceToHost, st));
        SYNC();
        if (pending == 0) break;
        nh_status rc = krylov<float>(g, sa);
        if (rc != NH_OK) return rc;
    }
    return NH_OK;
}

template <typename T>
nh_status step_t(nh_grid* g, double dt, nh_step_info* info)
{
    cudaStream_t st = g->stream;
    if (g->last_dt != 0.0 && dt != g->last_dt) {
        // keep t^n = t_base + n dt exact for a fixed dt; re-base when dt changes
        g->t_base = g->t_base + (double)g->n_since * g->last_dt;
        g->n_since = 0;
    }
    const double t_n = g->t_base + (double)g->n_since * dt;
    const double t_n1 = g->t_base + (double)(g->n_since + 1) * dt;
    const int cur = g->cur, nxt = cur ^ 1;
    const int lprev = g->lcur, lnew = lprev ^ 1;
    const Geo G = geo(g);
    const double gscale = (g->guess != NH_GUESS_ZERO && g->last_dt > 0.0) ? dt / g->last_dt : 0.0;

    LAUNCH(NH_K_KINEMATICS, k_kinematics<<<(g->nb + 127) / 128, 128, 0, st>>>(g->slide, g->kin, g->nb, t_n, t_n1));

    PredArgs<T> pa;
    pa.G = G;
    pa.z = (const T*)g->sz[cur]; pa.hu = (const T*)g->shu[cur]; pa.hw = (const T*)g->shw[cur];
    pa.zt = (T*)g->sz[nxt]; pa.hut = (T*)g->shu[nxt]; pa.hwt = (T*)g->shw[nxt];
    pa.d0 = (const T*)g->d0; pa.slide = g->slide; pa.kin = g->kin;
    pa.marks = g->marks; pa.mass_part = g->mass_part; pa.dt = dt; pa.knh = g->knh; pa.crit = g->crit;
    pa.all_global = (g->crit == NH_CRIT_GLOBAL) || (g->first_global && g->steps == 0);
    pa.tc = nullptr;
    LAUNCH(NH_K_PREDICT, predict_launch<T>(g->tile, g->nb, g->pitch / g->tile, st, pa));

    CompactArgs ca;
    ca.nx = g->nx; ca.pitch = g->pitch; ca.wpitch = g->wpitch; ca.bc = g->d.bc; ca.enlarge = g->enlarge;
    ca.marks = g->marks; ca.act = g->act; ca.list = g->list[lnew]; ca.nact = g->nact[lnew];
    ca.ms = g->ms; ca.ctl = g->ctl; ca.nxv = g->uneven ? g->nxd : nullptr; ca.tc = nullptr;
    const size_t csm = sizeof(uint32_t) * (size_t)((g->nx + 31) / 32);
    LAUNCH(NH_K_COMPACT, k_compact<<<g->nb, kCompactThreads, csm, st>>>(ca));
    LAUNCH(NH_K_COMPACT, k_items<<<1, 1024, 0, st>>>(g->ms, g->nb, g->items, g->pitems, g->ctl));

    AsmArgs<T> aa;
    aa.G = G;
    aa.zt = (const T*)g->sz[nxt]; aa.hut = (const T*)g->shu[nxt]; aa.hwt = (const T*)g->shw[nxt];
    aa.d0 = g->d0d; aa.slide = g->slide; aa.kin = g->kin;
    aa.list = g->list[lnew]; aa.act = g->act; aa.ms = g->ms;
    aa.diag = g->diag; aa.offl = g->offl; aa.offr = g->offr; aa.R = g->R;
    aa.diag32 = g->diag32; aa.offl32 = g->offl32; aa.offr32 = g->offr32;
    aa.nbl = g->nbl; aa.nbr = g->nbr;
    aa.c6 = (T*)g->c6; aa.cx = (T*)g->cx; aa.phi = (T*)g->phi; aa.ddx = (T*)g->ddx;
    aa.part = g->part; aa.cnt = g->cnt; aa.dt = dt; aa.solver = g->solver;
    aa.items = g->items; aa.ctl = g->ctl;

    const cnn::GuessGeo GG = guess_geo(g, nullptr);
    if (cnn_features_on(g)) LAUNCH(NH_K_CNN, CK(cnn::launch_features(g->cnn, GG, st)));
    bool learned = g->guess == NH_GUESS_CNN && gscale != 0.0;
    if (learned) LAUNCH(NH_K_CNN, CK(cnn::launch_guess(g->cnn, GG, st)));

    // assembly and solve from the learned guess; a failed solve from it is
    // redone (assembly included) from the plain warm start
    const double* xfinal = nullptr;
    Summary S;
    for (int attempt = 0; attempt < 2; ++attempt) {
        const double* src = learned ? g->cnn.guess : g->psi;
        LAUNCH(NH_K_ASSEMBLE, k_assemble<T><<<g->items_grid, kChunk, 0, st>>>(aa));
        if (learned) LAUNCH(NH_K_CNN, CK(judge_launch(g, lnew, gscale, nullptr, st)));
        if (g->ir_mode) {
            nh_status rc = refine(g, lnew, gscale, src);
            if (rc != NH_OK) return rc;
            xfinal = g->x64;
        } else {
            SolveArgs<double> sa = solve_args<double>(g, lnew, g->diag, g->offl, g->offr, g->R, g->rtol);
            sa.psi_prev = src;
            sa.guess_scale = gscale;
            nh_status rc = krylov<double>(g, sa);
            if (rc != NH_OK) return rc;
            xfinal = (const double*)g->x;
        }
        LAUNCH(NH_K_SUMMARY, k_summary<<<1, 256, 0, st>>>(g->ms, g->nb, g->mass_part, g->nb * (g->pitch / g->tile), g->d.dx, g->summary, nullptr));
        CK(cudaMemcpyAsync(&S, g->summary, sizeof(Summary), cudaMemcpyDeviceToHost, st));
        SYNC();
        CK(cudaGetLastError());
        if (!learned || S.status == NH_OK) break;
        learned = false;
    }
    int ir_passes = 0;
    if (g->ir_mode) {
        std::vector<IRState> irs(g->nb);
        CK(cudaMemcpyAsync(irs.data(), g->ir, sizeof(IRState) * g->nb, cudaMemcpyDeviceToHost, st));
        SYNC();
        for (const auto& q : irs) ir_passes = std::max(ir_passes, q.passes);
    }
    nh_status status = (nh_status)S.status;
    if (status == NH_OK) {
        if (g->cnn_attached) LAUNCH(NH_K_CNN, CK(cnn::launch_shift(g->cnn, GG, st)));
        ClearArgs cl;
        cl.nb = g->nb; cl.pitch = g->pitch; cl.maxlist = g->pitch;
        cl.list_prev = g->list[lprev]; cl.nact_prev = g->nact[lprev]; cl.psi = g->psi; cl.tc = nullptr;
        const size_t total = (size_t)g->nb * g->pitch;
        int cgrid = (int)std::min<size_t>((total + 255) / 256, (size_t)g->sm_count * 8);
        LAUNCH(NH_K_CLEAR, k_clear_prev<<<cgrid, 256, 0, st>>>(cl));
        CorrArgs<T> co;
        co.nb = g->nb; co.pitch = g->pitch; co.maxch = g->maxch; co.dx = g->d.dx;
        co.list = g->list[lnew]; co.nbl = g->nbl; co.nbr = g->nbr; co.x = xfinal;
        co.c6 = (const T*)g->c6; co.cx = (const T*)g->cx; co.phi = (const T*)g->phi;
        co.ddx = (const T*)g->ddx; co.ms = g->ms;
        co.hu = (T*)g->shu[nxt]; co.hw = (T*)g->shw[nxt]; co.psi = g->psi;
        co.items = g->items; co.ctl = g->ctl; co.tc = nullptr;
        LAUNCH(NH_K_CORRECT, k_correct<T><<<g->items_grid, kChunk, 0, st>>>(co));
        CK(cudaGetLastError());
        g->cur = nxt;
        g->lcur = lnew;
        g->n_since += 1;
        g->steps += 1;
        g->last_dt = dt;
    }
    if (info) {
        info->step = g->steps;
        info->t = (status == NH_OK) ? t_n1 : t_n;
        info->n_active = S.n_active;
        info->n_active_max = S.n_active_max;
        info->iters = S.iters;
        info->ir_passes = ir_passes;
        info->solver = S.n_active == 0 ? -1 : (S.any_bicg ? NH_SOLVER_BICGSTAB : NH_SOLVER_CG);
        info->status = status;
        info->rel_res = S.rel_res;
        info->min_gamma = S.min_gamma;
        info->mass = S.mass + g->mass0;
    }
    return status;
}

// ---------------------------------------------------------- captured runs

// Enqueue one step (FP64 solve; FP64 or FP32 state) on `st` with fixed buffer
// roles (no host round trip):
// the device time control block supplies t, the commit kernel accepts the step
// or aborts the run.  Used only while capturing a graph.
template <typename T>
nh_status enqueue_graph_step(nh_grid* g, cudaStream_t st, int cur, int lprev, double dt)
{
    const int nxt = cur ^ 1, lnew = lprev ^ 1;
    const Geo G = geo(g);
    k_kinematics_dev<<<(g->nb + 127) / 128, 128, 0, st>>>(g->slide, g->kin, g->nb, g->tc);
    PredArgs<T> pa;
    pa.G = G;
    pa.z = (const T*)g->sz[cur]; pa.hu = (const T*)g->shu[cur]; pa.hw = (const T*)g->shw[cur];
    pa.zt = (T*)g->sz[nxt]; pa.hut = (T*)g->shu[nxt]; pa.hwt = (T*)g->shw[nxt];
    pa.d0 = (const T*)g->d0; pa.slide = g->slide; pa.kin = g->kin;
    pa.marks = g->marks; pa.mass_part = g->mass_part; pa.dt = dt; pa.knh = g->knh; pa.crit = g->crit;
    pa.all_global = (g->crit == NH_CRIT_GLOBAL);
    pa.tc = g->tc;
    CK(predict_launch<T>(g->tile, g->nb, g->pitch / g->tile, st, pa));
    CompactArgs ca;
    ca.nx = g->nx; ca.pitch = g->pitch; ca.wpitch = g->wpitch; ca.bc = g->d.bc; ca.enlarge = g->enlarge;
    ca.marks = g->marks; ca.act = g->act; ca.list = g->list[lnew]; ca.nact = g->nact[lnew];
    ca.ms = g->ms; ca.ctl = g->ctl; ca.nxv = g->uneven ? g->nxd : nullptr; ca.tc = g->tc;
    k_compact<<<g->nb, kCompactThreads, sizeof(uint32_t) * (size_t)((g->nx + 31) / 32), st>>>(ca);
    k_items<<<1, 1024, 0, st>>>(g->ms, g->nb, g->items, g->pitems, g->ctl);
    AsmArgs<T> aa;
    aa.G = G;
    aa.zt = (const T*)g->sz[nxt]; aa.hut = (const T*)g->shu[nxt]; aa.hwt = (const T*)g->shw[nxt];
    aa.d0 = g->d0d; aa.slide = g->slide; aa.kin = g->kin;
    aa.list = g->list[lnew]; aa.act = g->act; aa.ms = g->ms;
    aa.diag = g->diag; aa.offl = g->offl; aa.offr = g->offr; aa.R = g->R;
    aa.diag32 = nullptr; aa.offl32 = nullptr; aa.offr32 = nullptr;
    aa.nbl = g->nbl; aa.nbr = g->nbr;
    aa.c6 = (T*)g->c6; aa.cx = (T*)g->cx; aa.phi = (T*)g->phi; aa.ddx = (T*)g->ddx;
    aa.part = g->part; aa.cnt = g->cnt; aa.dt = dt; aa.solver = g->solver;
    aa.items = g->items; aa.ctl = g->ctl;
    k_assemble<T><<<g->items_grid, kChunk, 0, st>>>(aa);
    const cnn::GuessGeo GG = guess_geo(g, g->tc);
    if (cnn_features_on(g)) CK(cnn::launch_features(g->cnn, GG, st));
    if (g->guess == NH_GUESS_CNN) {
        CK(cnn::launch_guess(g->cnn, GG, st));
        CK(judge_launch(g, lnew, 1.0, g->tc, st));
    }
    SolveArgs<double> sa = solve_args<double>(g, lnew, g->diag, g->offl, g->offr, g->R, g->rtol);
    sa.psi_prev = (g->guess == NH_GUESS_CNN) ? g->cnn.guess : g->psi;
    sa.guess_scale = (g->guess != NH_GUESS_ZERO) ? 1.0 : 0.0;
    sa.tc = g->tc;
    CK(cudaMemsetAsync(g->ctl, 0, 3 * sizeof(int), st));
    CK(cudaMemsetAsync(g->cnt, 0, sizeof(int) * g->nb, st));
    k_solve_init<double><<<g->items_grid, kChunk, 0, st>>>(sa);
    const size_t pcr_smem = 2 * sizeof(float) * (size_t)kPcrRows;
    sa.it = 0;
    k_pcr_factor<double, float><<<g->pcr_grid, kPcrThreads, 3 * sizeof(float) * kPcrRows, st>>>(sa);
    k_pcr<double, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_PCG);
    CK(cudaMemsetAsync(&g->ctl->timeout, 0, 3 * sizeof(int), st));
    {
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(g->coop_grid[0]);
        cfg.blockDim = dim3(kPcrThreads);
        cfg.dynamicSmemBytes = pcr_smem;
        cfg.stream = st;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeCooperative;
        attr[0].val.cooperative = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        long long budget = g->barrier_budget;
        CK(cudaLaunchKernelEx(&cfg, k_pcg_persistent<double, float>, sa, budget));
    }
    k_summary<<<1, 256, 0, st>>>(g->ms, g->nb, g->mass_part, g->nb * (g->pitch / g->tile), g->d.dx, g->summary, g->tc);
    k_commit<<<1, 32, 0, st>>>(g->summary, g->tc);
    if (g->cnn_attached) CK(cnn::launch_shift(g->cnn, GG, st));
    ClearArgs cl;
    cl.nb = g->nb; cl.pitch = g->pitch; cl.maxlist = g->pitch;
    cl.list_prev = g->list[lprev]; cl.nact_prev = g->nact[lprev]; cl.psi = g->psi; cl.tc = g->tc;
    const size_t total = (size_t)g->nb * g->pitch;
    k_clear_prev<<<(int)std::min<size_t>((total + 255) / 256, (size_t)g->sm_count * 8), 256, 0, st>>>(cl);
    CorrArgs<T> co;
    co.nb = g->nb; co.pitch = g->pitch; co.maxch = g->maxch; co.dx = g->d.dx;
    co.list = g->list[lnew]; co.nbl = g->nbl; co.nbr = g->nbr; co.x = (const double*)g->x;
    co.c6 = (const T*)g->c6; co.cx = (const T*)g->cx; co.phi = (const T*)g->phi;
    co.ddx = (const T*)g->ddx; co.ms = g->ms;
    co.hu = (T*)g->shu[nxt]; co.hw = (T*)g->shw[nxt]; co.psi = g->psi;
    co.items = g->items; co.ctl = g->ctl; co.tc = g->tc;
    k_correct<T><<<g->items_grid, kChunk, 0, st>>>(co);
    CK(cudaGetLastError());
    return NH_OK;
}

bool graph_eligible(const nh_grid* g, double dt)
{
    return !g->ir_mode && g->precond == NH_PRECOND_LINE && g->solver != NH_SOLVER_BICGSTAB &&
           g->coop_grid[0] > 0 && !g->prof_on && !(g->first_global && g->steps == 0) &&
           (g->last_dt == 0.0 || g->last_dt == dt) && g->cap_stream != nullptr;
}

void graph_destroy(nh_grid* g)
{
    for (int p = 0; p < 2; ++p)
        if (g->graph[p]) { cudaGraphExecDestroy(g->graph[p]); g->graph[p] = nullptr; }
    g->graph_valid = false;
}

nh_status graph_prepare(nh_grid* g, double dt)
{
    const double key[12] = {dt, (double)g->crit, g->knh, (double)g->enlarge, (double)g->solver, g->rtol,
                            (double)g->max_iter, (double)g->guess, (double)(g->cur ^ g->lcur), (double)g->tile,
                            (double)g->cnn_attached, (double)g->cnn_record};
    if (g->graph_valid && std::memcmp(key, g->graph_key, sizeof(key)) == 0) return NH_OK;
    graph_destroy(g);
    for (int p = 0; p < 2; ++p) {
        const int cur = p, lprev = p ^ g->cur ^ g->lcur;
        cudaGraph_t graph = nullptr;
        CK(cudaStreamBeginCapture(g->cap_stream, cudaStreamCaptureModeThreadLocal));
        nh_status rc = g->mixed ? enqueue_graph_step<float>(g, g->cap_stream, cur, lprev, dt)
                                : enqueue_graph_step<double>(g, g->cap_stream, cur, lprev, dt);
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

// n_steps steps by replaying the captured one-step graphs on the caller's
// stream; one synchronisation at the end.
nh_status graph_run(nh_grid* g, double dt, long long n_steps, nh_run_info* R)
{
    nh_status rc = graph_prepare(g, dt);
    if (rc != NH_OK) return rc;
    cudaStream_t st = g->stream;
    TimeCtl tc;
    std::memset(&tc, 0, sizeof(tc));
    tc.t_base = g->t_base; tc.dt = dt; tc.n = g->n_since; tc.done = 0; tc.abort = 0;
    tc.prev_ok = (g->last_dt == dt) ? 1 : 0;
    CK(cudaMemcpyAsync(g->tc, &tc, sizeof(tc), cudaMemcpyHostToDevice, st));
    for (long long k = 0; k < n_steps; ++k) CK(cudaGraphLaunch(g->graph[(g->cur + k) & 1], st));
    Summary S;
    CK(cudaMemcpyAsync(&tc, g->tc, sizeof(tc), cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(&S, g->summary, sizeof(Summary), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    const long long done = tc.done;
    if (done & 1) { g->cur ^= 1; g->lcur ^= 1; }
    g->steps += done;
    g->n_since += done;
    if (done > 0) g->last_dt = dt;
    g->graph_runs += 1;
    R->steps = done;
    R->iters_total = tc.iters_total;
    R->active_total = tc.active_total;
    nh_step_info& I = R->last;
    I.step = g->steps;
    I.t = g->t_base + (double)g->n_since * dt;
    I.n_active = S.n_active; I.n_active_max = S.n_active_max; I.iters = S.iters; I.ir_passes = 0;
    I.solver = S.n_active == 0 ? -1 : (S.any_bicg ? NH_SOLVER_BICGSTAB : NH_SOLVER_CG);
    I.status = tc.abort ? tc.fail_status : NH_OK;
    I.rel_res = S.rel_res; I.min_gamma = S.min_gamma; I.mass = S.mass + g->mass0;
    if (tc.abort) {
        // the failing step: AUTO members whose CG broke down are retried by the
        // step-by-step path (BiCGStab fallback) before the run is reported failed
        return (nh_status)(tc.fail_status == kStatusFallback ? NH_ERR_NONFINITE : tc.fail_status);
    }
    return NH_OK;
}

// Predictor tile autotuner: time each candidate on the handle's current state
// (outputs go to the step's scratch buffers) and keep the fastest; results are
// cached per (cells per member, members, precision, limiter) for the process.
std::mutex g_tune_mutex;
std::map<std::array<long long, 4>, int> g_tune_cache;

template <typename T>
nh_status autotune_t(nh_grid* g, double dt)
{
    const std::array<long long, 4> key = {g->pitch, g->nb, g->mixed ? 1 : 0, g->d.limiter};
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) { g->tile = it->second; g->tuned = true; return NH_OK; }
    }
    cudaStream_t st = g->stream;
    const int cur = g->cur, nxt = cur ^ 1;
    k_kinematics<<<(g->nb + 127) / 128, 128, 0, st>>>(g->slide, g->kin, g->nb, g->t_base, g->t_base + dt);
    PredArgs<T> pa;
    pa.G = geo(g);
    pa.z = (const T*)g->sz[cur]; pa.hu = (const T*)g->shu[cur]; pa.hw = (const T*)g->shw[cur];
    pa.zt = (T*)g->sz[nxt]; pa.hut = (T*)g->shu[nxt]; pa.hwt = (T*)g->shw[nxt];
    pa.d0 = (const T*)g->d0; pa.slide = g->slide; pa.kin = g->kin;
    pa.marks = g->marks; pa.mass_part = g->mass_part; pa.dt = dt; pa.knh = g->knh; pa.crit = g->crit;
    pa.all_global = 0; pa.tc = nullptr;
    cudaEvent_t e0, e1;
    CK(cudaEventCreate(&e0));
    if (cudaEventCreate(&e1) != cudaSuccess) { cudaEventDestroy(e0); return NH_ERR_CUDA; }
    const int cand[3] = {128, 256, 512};
    float best = 1e30f;
    int best_tile = kPredTile;
    nh_status rc = NH_OK;
    for (int c = 0; c < 3 && rc == NH_OK; ++c) {
        pa.G.ntiles = g->pitch / cand[c];
        for (int w = 0; w < 2; ++w) predict_launch<T>(cand[c], g->nb, pa.G.ntiles, st, pa);
        cudaEventRecord(e0, st);
        for (int r = 0; r < 5; ++r) predict_launch<T>(cand[c], g->nb, pa.G.ntiles, st, pa);
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) { rc = NH_ERR_CUDA; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (ms < best) { best = ms; best_tile = cand[c]; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (cudaGetLastError() != cudaSuccess) rc = NH_ERR_CUDA;
    if (rc != NH_OK) return rc;
    g->tile = best_tile;
    g->tuned = true;
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    g_tune_cache[key] = best_tile;
    return NH_OK;
}

nh_status do_step(nh_grid* g, double dt, nh_step_info* info)
{
    if (!g->has_state) return NH_ERR_STATE;
    if (!(dt > 0.0) || !std::isfinite(dt)) return NH_ERR_ARG;
    if (!g->tuned) {
        nh_status rc = g->mixed ? autotune_t<float>(g, dt) : autotune_t<double>(g, dt);
        if (rc != NH_OK) return rc;
    }
    return g->mixed ? step_t<float>(g, dt, info) : step_t<double>(g, dt, info);
}

template <typename T>
nh_status upload_state(nh_grid* g, const double* h, const double* hu, const double* hw)
{
    cudaStream_t st = g->stream;
    const size_t n = (size_t)g->ncells;
    CK(cudaMemcpyAsync(g->stage, h, n * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(g->stage + n, hu, n * 8, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(g->stage + 2 * n, hw, n * 8, cudaMemcpyHostToDevice, st));
    const int c = g->cur;
    const dim3 grid((unsigned)std::min<size_t>((g->nx + 255) / 256, 64), (unsigned)g->nb);
    k_state_in<T><<<grid, 256, 0, st>>>(g->stage, g->stage + n, g->stage + 2 * n, g->d0d, (T*)g->sz[c],
                                       (T*)g->shu[c], (T*)g->shw[c], g->nb, g->pitch, g->offd);
    CK(cudaGetLastError());
    return NH_OK;
}

template <typename T>
nh_status download_state(nh_grid* g, double* h, double* hu, double* hw, double* p)
{
    cudaStream_t st = g->stream;
    const size_t n = (size_t)g->ncells;
    const int c = g->cur;
    const double sc = g->last_dt > 0.0 ? g->d.rho / g->last_dt : 0.0;
    // p is formed in an FP64-sized solver vector: those are scratch between steps
    double* p_dev = g->es == 8 ? (double*)g->r1 : g->x64;
    const dim3 grid((unsigned)std::min<size_t>((g->nx + 255) / 256, 64), (unsigned)g->nb);
    k_state_out<T><<<grid, 256, 0, st>>>((const T*)g->sz[c], (const T*)g->shu[c], (const T*)g->shw[c],
                                        g->d0d, g->psi, g->stage, g->stage + n, g->stage + 2 * n, p_dev,
                                        sc, g->nb, g->pitch, g->offd);
    CK(cudaGetLastError());
    if (h) CK(cudaMemcpyAsync(h, g->stage, n * 8, cudaMemcpyDeviceToHost, st));
    if (hu) CK(cudaMemcpyAsync(hu, g->stage + n, n * 8, cudaMemcpyDeviceToHost, st));
    if (hw) CK(cudaMemcpyAsync(hw, g->stage + 2 * n, n * 8, cudaMemcpyDeviceToHost, st));
    if (p) CK(cudaMemcpyAsync(p, p_dev, n * 8, cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    return NH_OK;
}

// Shared body of nh_create_grid / nh_create_ensemble.  nxv: cells per member.
nh_status create_impl(const nh_grid_desc* desc_in, const int* nxv, const double* d0_host, void* ws,
                      size_t ws_bytes, void* stream, nh_grid** out)
{
    if (!out) return NH_ERR_ARG;
    *out = nullptr;
    if (!desc_in || !nxv || !d0_host || !ws) return NH_ERR_ARG;
    nh_grid_desc desc = *desc_in;
    long long ncells = 0;
    int nxmax = 0;
    bool uneven = false;
    for (int b = 0; b < desc.nbatch; ++b) {
        if (nxv[b] < 8 || nxv[b] > (1 << 20)) return NH_ERR_ARG;
        ncells += nxv[b];
        nxmax = std::max(nxmax, nxv[b]);
        if (nxv[b] != nxv[0]) uneven = true;
    }
    desc.nx = nxmax;
    if (!desc_ok(&desc)) return NH_ERR_ARG;
    if (((uintptr_t)ws % kAlign) != 0) return NH_ERR_ARG;
    const size_t need = carve(desc, ncells, nullptr, nullptr);
    if (ws_bytes < need) return NH_ERR_ARG;
    for (long long q = 0; q < ncells; ++q)
        if (!(d0_host[q] > 0.0) || !std::isfinite(d0_host[q])) return NH_ERR_ARG;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    nh_grid* g = new (std::nothrow) nh_grid();
    if (!g) return NH_ERR_ARG;
    g->d = desc;
    g->stream = (cudaStream_t)stream;
    carve(desc, ncells, g, (char*)ws);
    g->ws_base = ws;
    g->uneven = uneven;
    g->ncells = ncells;
    g->nxh.assign(nxv, nxv + desc.nbatch);
    g->offh.assign(desc.nbatch + 1, 0);
    for (int b = 0; b < desc.nbatch; ++b) g->offh[b + 1] = g->offh[b] + nxv[b];
    *out = g;
    return NH_OK;
}

// Learned-guess buffers inside the caller's second workspace.
size_t cnn_layout(const nh_grid* g, char* base, cnn::GuessBufs* B)
{
    const size_t N = (size_t)g->nb * g->pitch;
    Carver c{base};
    cnn::GuessBufs t;
    cnn::GuessBufs& b = B ? *B : t;
    b.h1 = (double*)c.take(sizeof(double) * N);
    b.h2 = (double*)c.take(sizeof(double) * N);
    b.feat = c.take((size_t)NH_CNN_IN * 2 * N);
    b.y = (float*)c.take(sizeof(float) * N);
    b.guess = (double*)c.take(sizeof(double) * N);
    b.d2 = (double*)c.take(sizeof(double) * N);
    b.base = (double*)c.take(sizeof(double) * N);
    b.choice = (int*)c.take(sizeof(int) * g->nb);
    b.params = (float*)c.take(sizeof(float) * NH_CNN_PARAMS);
    b.ctl = (cnn::GuessCtl*)c.take(sizeof(cnn::GuessCtl));
    return (c.off + kAlign - 1) / kAlign * kAlign;
}

}  // namespace

extern "C" {

size_t nh_workspace_bytes(const nh_grid_desc* desc)
{
    if (!desc_ok(desc)) return 0;
    return carve(*desc, (long long)desc->nx * desc->nbatch, nullptr, nullptr);
}

size_t nh_workspace_bytes_ensemble(const nh_grid_desc* desc, const int* nx_per_member)
{
    if (!desc || !nx_per_member || desc->nbatch < 1) return 0;
    nh_grid_desc d = *desc;
    long long ncells = 0;
    int nxmax = 0;
    for (int b = 0; b < d.nbatch; ++b) {
        if (nx_per_member[b] < 8 || nx_per_member[b] > (1 << 20)) return 0;
        ncells += nx_per_member[b];
        nxmax = std::max(nxmax, nx_per_member[b]);
    }
    d.nx = nxmax;
    if (!desc_ok(&d)) return 0;
    return carve(d, ncells, nullptr, nullptr);
}

static nh_status finish_create(nh_grid* g, const double* d0_host, int dev, int sms);

nh_status nh_create_grid(const nh_grid_desc* desc, const double* d0_host, void* ws, size_t ws_bytes,
                         void* stream, nh_grid** out)
{
    if (!out) return NH_ERR_ARG;
    *out = nullptr;
    if (!desc_ok(desc)) return NH_ERR_ARG;
    std::vector<int> nxv(desc->nbatch, desc->nx);
    return nh_create_ensemble(desc, nxv.data(), d0_host, ws, ws_bytes, stream, out);
}

nh_status nh_create_ensemble(const nh_grid_desc* desc, const int* nx_per_member, const double* d0_host,
                             void* ws, size_t ws_bytes, void* stream, nh_grid** out)
{
    nh_status rc0 = create_impl(desc, nx_per_member, d0_host, ws, ws_bytes, stream, out);
    if (rc0 != NH_OK) return rc0;
    nh_grid* g = *out;
    *out = nullptr;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { delete g; return NH_ERR_CUDA; }
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) { delete g; return NH_ERR_CUDA; }
    nh_status rc = finish_create(g, d0_host, dev, sms);
    if (rc != NH_OK) { delete g; return rc; }
    *out = g;
    return NH_OK;
}

static nh_status finish_create(nh_grid* g, const double* d0_host, int dev, int sms)
{
    void* ws = g->ws_base;
    const size_t need = carve(g->d, g->ncells, nullptr, nullptr);
    g->sm_count = sms;
    g->items_grid = (int)std::min<long long>((long long)g->nb * g->maxch, (long long)sms * 8);
    if (g->items_grid < 1) g->items_grid = 1;
    g->pcr_grid = (int)std::min<long long>((long long)g->nb * g->maxpb, (long long)sms * 2);
    if (g->pcr_grid < 1) g->pcr_grid = 1;
    g->crit = NH_CRIT_GLOBAL; g->knh = 1e-3; g->enlarge = 1; g->first_global = 0;
    g->solver = NH_SOLVER_AUTO; g->rtol = 1e-12; g->max_iter = 20000; g->guess = NH_GUESS_PREV;
    g->ir_max = 30; g->inner_rtol = 1e-5; g->poll_every = 4; g->precond = NH_PRECOND_LINE;
    g->has_state = false; g->t_base = 0.0; g->n_since = 0; g->steps = 0; g->last_dt = 0.0;
    g->cur = 0; g->lcur = 0;
    g->prof_on = false; g->prof_used = 0;
    for (int k = 0; k < NH_K_COUNT; ++k) { g->prof_ms[k] = 0.0; g->prof_launches[k] = 0; }
    g->graph[0] = g->graph[1] = nullptr; g->graph_valid = false; g->graph_runs = 0; g->use_graphs = true;
    g->cnn_attached = false; g->cnn_record = false;
    std::memset(&g->cnn, 0, sizeof(g->cnn));
    g->tile = kPredTile; g->tuned = false;
    if (cudaStreamCreateWithFlags(&g->cap_stream, cudaStreamNonBlocking) != cudaSuccess) g->cap_stream = nullptr;
    cudaStream_t st = g->stream;
    nh_status rc = NH_OK;
    do {
        if (cudaMemsetAsync(ws, 0, need, st) != cudaSuccess) { rc = NH_ERR_CUDA; break; }
        const size_t N = (size_t)g->nb * g->pitch;
        // member counts and offsets, then d0 scattered from the concatenated host layout
        if (cudaMemcpyAsync(g->nxd, g->nxh.data(), sizeof(int) * g->nb, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(g->offd, g->offh.data(), sizeof(long long) * (g->nb + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaMemcpyAsync(g->stage, d0_host, sizeof(double) * g->ncells, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        k_fill<<<(int)std::min<size_t>((N + 255) / 256, (size_t)sms * 8), 256, 0, st>>>(g->d0d, 1.0, N);
        k_scatter<<<dim3((unsigned)std::min((g->nx + 255) / 256, 64), (unsigned)g->nb), 256, 0, st>>>(
            g->stage, g->d0d, g->pitch, g->offd);
        if (cudaGetLastError() != cudaSuccess) { rc = NH_ERR_CUDA; break; }
        if (g->mixed) {
            k_to_float<<<(int)std::min<size_t>((N + 255) / 256, (size_t)sms * 8), 256, 0, st>>>(g->d0d, (float*)g->d0, N);
            if (cudaGetLastError() != cudaSuccess) { rc = NH_ERR_CUDA; break; }
        } else if (cudaMemcpyAsync(g->d0, g->d0d, N * 8, cudaMemcpyDeviceToDevice, st) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        double m0 = 0.0;
        for (long long q = 0; q < g->ncells; ++q) m0 += d0_host[q];
        g->mass0 = m0 * g->d.dx;
        std::vector<Slide> sl(g->nb);
        for (auto& s : sl) {
            s.A = 0; s.L = 1; s.iL = 1; s.xc0 = 0; s.s0 = 0; s.t0 = 1; s.t2 = 0; s.shape = NH_SLIDE_NONE; s.pad = 0;
        }
        if (cudaMemcpyAsync(g->slide, sl.data(), sizeof(Slide) * g->nb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) { rc = NH_ERR_CUDA; break; }
        if (predict_set_smem<double>() != cudaSuccess || predict_set_smem<float>() != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        if (cudaFuncSetAttribute(k_pcr<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * sizeof(float) * kPcrRows)) != cudaSuccess ||
            cudaFuncSetAttribute(k_pcr<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * sizeof(float) * kPcrRows)) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        if (cudaFuncSetAttribute(k_pcr_factor<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(3 * sizeof(float) * kPcrRows)) != cudaSuccess ||
            cudaFuncSetAttribute(k_pcr_factor<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(3 * sizeof(float) * kPcrRows)) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        if (cudaFuncSetAttribute(k_pcg_persistent<double, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * sizeof(float) * kPcrRows)) != cudaSuccess ||
            cudaFuncSetAttribute(k_pcg_persistent<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(2 * sizeof(float) * kPcrRows)) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        {
            int coop = 0, per_sm = 0;
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
            const size_t sm_bytes = 2 * sizeof(float) * kPcrRows;
            g->coop_grid[0] = g->coop_grid[1] = 0;
            if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<double, float>,
                                                                      kPcrThreads, sm_bytes) == cudaSuccess)
                g->coop_grid[0] = per_sm * sms;
            if (coop && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg_persistent<float, float>,
                                                                      kPcrThreads, sm_bytes) == cudaSuccess)
                g->coop_grid[1] = per_sm * sms;
            int clk_khz = 0;
            cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
            g->barrier_budget = (long long)(clk_khz > 0 ? clk_khz : 2000000) * 1000LL;   // about one second
            g->barrier_budget_default = g->barrier_budget;
        }
        if (cudaFuncSetAttribute(k_compact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(uint32_t) * ((g->nx + 31) / 32))) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
    } while (0);
    return rc;
}

nh_status nh_set_bottom_motion(nh_grid* g, const nh_slide_desc* slides)
{
    if (!g) return NH_ERR_ARG;
    std::vector<Slide> sl(g->nb);
    for (int b = 0; b < g->nb; ++b) {
        Slide s{0.0, 1.0, 0.0, 0.0, 1.0, 1.0, 0.0, NH_SLIDE_NONE, 0};
        if (slides) {
            const nh_slide_desc& q = slides[b];
            if (q.shape < NH_SLIDE_NONE || q.shape > NH_SLIDE_QUARTIC) return NH_ERR_ARG;
            if (q.shape != NH_SLIDE_NONE) {
                if (!(q.L > 0.0) || !(q.t0 > 0.0) || !std::isfinite(q.A) || !std::isfinite(q.xc0) ||
                    !std::isfinite(q.s0))
                    return NH_ERR_ARG;
                if (q.shape == NH_SLIDE_QUARTIC && !(q.t2 >= q.t0 && std::isfinite(q.t2))) return NH_ERR_ARG;
                s.A = q.A; s.L = q.L; s.iL = 1.0 / q.L; s.xc0 = q.xc0; s.s0 = q.s0; s.t0 = q.t0;
                s.t2 = q.shape == NH_SLIDE_QUARTIC ? q.t2 : 0.0;
                s.shape = q.shape;
            }
        }
        sl[b] = s;
    }
    CK(cudaMemcpyAsync(g->slide, sl.data(), sizeof(Slide) * g->nb, cudaMemcpyHostToDevice, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    return NH_OK;
}

nh_status nh_set_criterion(nh_grid* g, int kind, double k_nh, int enlarge, int first_step_global)
{
    if (!g) return NH_ERR_ARG;
    if (kind < NH_CRIT_GLOBAL || kind > NH_CRIT_W_X) return NH_ERR_ARG;
    if (!std::isfinite(k_nh) || enlarge < 0 || enlarge > 16) return NH_ERR_ARG;
    g->crit = kind; g->knh = k_nh; g->enlarge = enlarge; g->first_global = first_step_global != 0;
    return NH_OK;
}

nh_status nh_set_solver(nh_grid* g, int kind, double rtol, int max_iter, int guess, int ir_max,
                        double inner_rtol)
{
    if (!g) return NH_ERR_ARG;
    if (kind < NH_SOLVER_AUTO || kind > NH_SOLVER_BICGSTAB) return NH_ERR_ARG;
    if (!(rtol > 0.0) || max_iter < 1 || guess < NH_GUESS_ZERO || guess > NH_GUESS_CNN) return NH_ERR_ARG;
    if (ir_max < 1 || !(inner_rtol > 0.0)) return NH_ERR_ARG;
    if (guess == NH_GUESS_CNN && !g->cnn_attached) return NH_ERR_STATE;
    g->solver = kind; g->rtol = rtol; g->max_iter = max_iter; g->guess = guess;
    g->ir_max = ir_max; g->inner_rtol = inner_rtol;
    return NH_OK;
}

nh_status nh_set_preconditioner(nh_grid* g, int kind)
{
    if (!g) return NH_ERR_ARG;
    if (kind != NH_PRECOND_NONE && kind != NH_PRECOND_LINE) return NH_ERR_ARG;
    g->precond = kind;
    return NH_OK;
}

nh_status nh_set_state(nh_grid* g, const double* h, const double* hu, const double* hw, double t)
{
    if (!g || !h || !hu || !hw || !std::isfinite(t)) return NH_ERR_ARG;
    for (long long q = 0; q < g->ncells; ++q)
        if (!(h[q] > 0.0) || !std::isfinite(h[q]) || !std::isfinite(hu[q]) || !std::isfinite(hw[q]))
            return NH_ERR_ARG;
    cudaStream_t st = g->stream;
    g->cur = 0;
    g->lcur = 0;
    nh_status rc = g->mixed ? upload_state<float>(g, h, hu, hw) : upload_state<double>(g, h, hu, hw);
    if (rc != NH_OK) return rc;
    CK(cudaMemsetAsync(g->psi, 0, sizeof(double) * (size_t)g->nb * g->pitch, st));
    CK(cudaMemsetAsync(g->nact[0], 0, sizeof(int) * g->nb, st));
    CK(cudaMemsetAsync(g->nact[1], 0, sizeof(int) * g->nb, st));
    if (g->cnn_attached) CK(cudaMemsetAsync(g->cnn.ctl, 0, sizeof(cnn::GuessCtl), st));
    CK(cudaStreamSynchronize(st));
    g->has_state = true;
    g->t_base = t; g->n_since = 0; g->steps = 0; g->last_dt = 0.0;
    return NH_OK;
}

nh_status nh_put_state(nh_grid* g, const double* h, const double* hu, const double* hw)
{
    if (!g || !h || !hu || !hw) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    return g->mixed ? upload_state<float>(g, h, hu, hw) : upload_state<double>(g, h, hu, hw);
}

nh_status nh_set_tile(nh_grid* g, int tile, int* chosen)
{
    if (!g) return NH_ERR_ARG;
    if (tile != 0 && tile != 128 && tile != 256 && tile != 512) return NH_ERR_ARG;
    if (tile != 0) { g->tile = tile; g->tuned = true; }
    if (chosen) *chosen = g->tuned ? g->tile : 0;
    return NH_OK;
}

nh_status nh_set_run_mode(nh_grid* g, int use_graphs)
{
    if (!g) return NH_ERR_ARG;
    g->use_graphs = use_graphs != 0;
    return NH_OK;
}

nh_status nh_set_wait_budget(nh_grid* g, long long cycles)
{
    if (!g || cycles < 0) return NH_ERR_ARG;
    g->barrier_budget = cycles > 0 ? cycles : g->barrier_budget_default;
    graph_destroy(g);
    return NH_OK;
}

nh_status nh_set_profiling(nh_grid* g, int enable)
{
    if (!g) return NH_ERR_ARG;
    CK(cudaStreamSynchronize(g->stream));
    g->prof_used = 0;
    g->prof_on = enable != 0;
    for (int k = 0; k < NH_K_COUNT; ++k) { g->prof_ms[k] = 0.0; g->prof_launches[k] = 0; }
    return NH_OK;
}

nh_status nh_get_profile(nh_grid* g, double* ms, long long* launches)
{
    if (!g) return NH_ERR_ARG;
    CK(cudaStreamSynchronize(g->stream));
    prof_fold(g);
    for (int k = 0; k < NH_K_COUNT; ++k) {
        if (ms) ms[k] = g->prof_ms[k];
        if (launches) launches[k] = g->prof_launches[k];
    }
    return NH_OK;
}

nh_status nh_get_state(nh_grid* g, double* h, double* hu, double* hw, double* p_nh)
{
    if (!g) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    return g->mixed ? download_state<float>(g, h, hu, hw, p_nh) : download_state<double>(g, h, hu, hw, p_nh);
}

nh_status nh_get_mask(nh_grid* g, unsigned char* mask, int* iters, double* rel_res)
{
    if (!g) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    cudaStream_t st = g->stream;
    if (mask) {
        std::vector<uint32_t> w((size_t)g->nb * g->wpitch);
        CK(cudaMemcpyAsync(w.data(), g->act, sizeof(uint32_t) * w.size(), cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int b = 0; b < g->nb; ++b)
            for (int i = 0; i < g->nxh[b]; ++i)
                mask[g->offh[b] + i] = (w[(size_t)b * g->wpitch + (i >> 5)] >> (i & 31)) & 1u;
    }
    if (iters || rel_res) {
        std::vector<MState> ms(g->nb);
        CK(cudaMemcpyAsync(ms.data(), g->ms, sizeof(MState) * g->nb, cudaMemcpyDeviceToHost, st));
        CK(cudaStreamSynchronize(st));
        for (int b = 0; b < g->nb; ++b) {
            if (iters) iters[b] = ms[b].iters;
            if (rel_res) rel_res[b] = ms[b].rel_res;
        }
    }
    return NH_OK;
}

nh_status nh_step(nh_grid* g, double dt, nh_step_info* info)
{
    if (!g) return NH_ERR_ARG;
    return do_step(g, dt, info);
}

nh_status nh_run(nh_grid* g, double dt, long long n_steps, nh_run_info* info)
{
    if (!g || n_steps < 0) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    if (!(dt > 0.0) || !std::isfinite(dt)) return NH_ERR_ARG;
    nh_run_info R;
    std::memset(&R, 0, sizeof(R));
    nh_status rc = NH_OK;
    if (!g->tuned) {
        rc = g->mixed ? autotune_t<float>(g, dt) : autotune_t<double>(g, dt);
        if (rc != NH_OK) return rc;
    }
    if (g->use_graphs && n_steps > 0 && graph_eligible(g, dt)) {
        rc = graph_run(g, dt, n_steps, &R);
        if (rc == NH_OK || R.steps == n_steps) {
            if (info) *info = R;
            return rc;
        }
        // a step failed inside the captured run: redo it step by step (this
        // also gives AUTO members their BiCGStab fallback) and continue there;
        // R keeps the steps the replay accepted
        n_steps -= R.steps;
        rc = NH_OK;
    }
    for (long long k = 0; k < n_steps; ++k) {
        nh_step_info si;
        std::memset(&si, 0, sizeof(si));
        rc = do_step(g, dt, &si);
        R.last = si;
        if (rc != NH_OK) break;
        R.steps += 1;
        R.iters_total += si.iters;
        R.active_total += si.n_active;
    }
    if (info) *info = R;
    return rc;
}

// ------------------------------------------------------------ learned guess

size_t nh_cnn_attach_bytes(const nh_grid* g)
{
    if (!g) return 0;
    return cnn_layout(g, nullptr, nullptr);
}

nh_status nh_cnn_attach(nh_grid* g, void* ws, size_t ws_bytes)
{
    if (!g || !ws) return NH_ERR_ARG;
    const size_t need = cnn_layout(g, nullptr, nullptr);
    if (ws_bytes < need || ((uintptr_t)ws % kAlign) != 0) return NH_ERR_ARG;
    cnn::GuessBufs B;
    cnn_layout(g, (char*)ws, &B);
    CK(cudaMemsetAsync(ws, 0, need, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    if (cnn::prepare_device() != cudaSuccess) return NH_ERR_CUDA;
    g->cnn = B;
    g->cnn_attached = true;
    graph_destroy(g);
    return NH_OK;
}

nh_status nh_cnn_set_params(nh_grid* g, const float* params_dev)
{
    if (!g || !params_dev) return NH_ERR_ARG;
    if (!g->cnn_attached) return NH_ERR_STATE;
    CK(cudaMemcpyAsync(g->cnn.params, params_dev, sizeof(float) * NH_CNN_PARAMS, cudaMemcpyDeviceToDevice,
                       g->stream));
    return NH_OK;
}

nh_status nh_cnn_record(nh_grid* g, int record)
{
    if (!g) return NH_ERR_ARG;
    if (!g->cnn_attached) return NH_ERR_STATE;
    g->cnn_record = record != 0;
    return NH_OK;
}

nh_status nh_cnn_choices(nh_grid* g, long long* counts)
{
    if (!g || !counts) return NH_ERR_ARG;
    if (!g->cnn_attached) return NH_ERR_STATE;
    cnn::GuessCtl c;
    CK(cudaMemcpyAsync(&c, g->cnn.ctl, sizeof(c), cudaMemcpyDeviceToHost, g->stream));
    CK(cudaStreamSynchronize(g->stream));
    for (int k = 0; k < 3; ++k) counts[k] = (long long)c.counts[k];
    return NH_OK;
}

nh_status nh_cnn_harvest(nh_grid* g, void* feat_out, float* target_out, unsigned char* mask_out, double* scale,
                         int* pitch)
{
    if (!g || !feat_out || !target_out || !mask_out) return NH_ERR_ARG;
    if (!g->cnn_attached) return NH_ERR_STATE;
    cudaStream_t st = g->stream;
    cnn::GuessCtl c;
    CK(cudaMemcpyAsync(&c, g->cnn.ctl, sizeof(c), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (!c.built) return NH_ERR_STATE;
    const size_t N = (size_t)g->nb * g->pitch;
    CK(cudaMemcpyAsync(feat_out, g->cnn.feat, (size_t)NH_CNN_IN * 2 * N, cudaMemcpyDeviceToDevice, st));
    CK(cnn::launch_harvest(g->cnn, guess_geo(g, nullptr), target_out, mask_out, st));
    CK(cudaStreamSynchronize(st));
    if (scale) *scale = c.S2_used;
    if (pitch) *pitch = g->pitch;
    return NH_OK;
}

void nh_destroy(nh_grid* g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    for (cudaEvent_t e : g->prof_pool) cudaEventDestroy(e);
    graph_destroy(g);
    if (g->cap_stream) cudaStreamDestroy(g->cap_stream);
    delete g;
}

const char* nh_status_string(nh_status s)
{
    switch (s) {
    case NH_OK: return "NH_OK";
    case NH_ERR_ARG: return "NH_ERR_ARG: invalid argument";
    case NH_ERR_CUDA: return "NH_ERR_CUDA: CUDA runtime error";
    case NH_ERR_NOT_CONVERGED: return "NH_ERR_NOT_CONVERGED: Krylov solve reached max_iter";
    case NH_ERR_NONFINITE: return "NH_ERR_NONFINITE: non-finite residual";
    case NH_ERR_TIMEOUT: return "NH_ERR_TIMEOUT: bounded device wait expired";
    case NH_ERR_STATE: return "NH_ERR_STATE: call out of order";
    default: return "unknown nh_status";
    }
}

}  // extern "C"
