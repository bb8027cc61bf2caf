// nh_api2d.cu -- host runtime behind include/nhswe2d.h (one 2D grid, FP64).
//
// The handle carves every device buffer out of the caller's workspace and
// runs one step as: depth at t^n and t^{n+1}, two Heun stages, criterion and
// Moore enlargement, row-major compaction, 9-point assembly, the line-
// preconditioned CG of the 1D members (one member holding the whole active
// set; S, N and the diagonal couplings as extra couplings), correction.
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "nh_kernels2d.cuh"
#include "nhswe2d.h"

using namespace nh;

struct nh_grid2d {
    nh_grid2d_desc d;
    cudaStream_t stream;
    int nx, ny, N, maxch, maxpb, nblk, nmass, sms, items_grid, pcr_grid, elem_grid, coop_grid;
    long long barrier_budget;
    Slide2 slide;
    double s0, t0;
    int crit, enlarge, first_global;
    double knh;
    double rtol;
    int max_iter, guess;
    bool has_state;
    double t_base, last_dt;
    long long n_since, steps;
    int cur, lcur;
    double* q[2][4];
    double* qs[4];
    double* k1[4];
    double *d0, *dn, *dn1;
    unsigned char *marks, *act;
    int *inv, *list[2], *nact[2], *bcnt, *boff;
    int2 *items, *pitems;
    double *diag, *offl, *offr, *R, *ext_c;
    int *ext_k, *nbl, *nbr;
    double *c6, *cx, *cy, *phi, *ddx, *ddy, *psi;
    double *x, *r, *p0, *p1, *qv, *rh, *v0, *v1, *s, *t, *r1, *z;
    float2* pf;
    float* prb;
    MState* ms;
    Ctl* ctl;
    double* part;
    int* cnt;
    double* mass_part;
    Summary* summary;
};

namespace {

constexpr size_t kAlign2 = 256;

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

int mass_blocks(int N) { return std::max(1, std::min((N + 255) / 256, 1024)); }

size_t carve2(const nh_grid2d_desc& d, nh_grid2d* g, char* base)
{
    const int N = d.nx * d.ny;
    const int maxch = (N + kChunk - 1) / kChunk;
    const int maxpb = (N + kPcrRows - 1) / kPcrRows;
    const int nblk = (N + kCompact2 - 1) / kCompact2;
    Carver2 c{base};
    nh_grid2d tmp;
    nh_grid2d* G = g ? g : &tmp;
    for (int b = 0; b < 2; ++b)
        for (int f = 0; f < 4; ++f) G->q[b][f] = c.take<double>(N);
    for (int f = 0; f < 4; ++f) { G->qs[f] = c.take<double>(N); G->k1[f] = c.take<double>(N); }
    G->d0 = c.take<double>(N); G->dn = c.take<double>(N); G->dn1 = c.take<double>(N);
    G->marks = c.take<unsigned char>(N); G->act = c.take<unsigned char>(N);
    G->inv = c.take<int>(N);
    for (int b = 0; b < 2; ++b) { G->list[b] = c.take<int>(N); G->nact[b] = c.take<int>(1); }
    G->bcnt = c.take<int>(nblk); G->boff = c.take<int>(nblk);
    G->items = c.take<int2>(maxch); G->pitems = c.take<int2>(maxpb);
    G->diag = c.take<double>(N); G->offl = c.take<double>(N); G->offr = c.take<double>(N);
    G->R = c.take<double>(N);
    G->ext_c = c.take<double>(6 * (size_t)N); G->ext_k = c.take<int>(6 * (size_t)N);
    G->nbl = c.take<int>(N); G->nbr = c.take<int>(N);
    G->c6 = c.take<double>(N); G->cx = c.take<double>(N); G->cy = c.take<double>(N);
    G->phi = c.take<double>(N); G->ddx = c.take<double>(N); G->ddy = c.take<double>(N);
    G->psi = c.take<double>(N);
    G->x = c.take<double>(N); G->r = c.take<double>(N); G->p0 = c.take<double>(N); G->p1 = c.take<double>(N);
    G->qv = c.take<double>(N); G->rh = c.take<double>(N); G->v0 = c.take<double>(N); G->v1 = c.take<double>(N);
    G->s = c.take<double>(N); G->t = c.take<double>(N); G->r1 = c.take<double>(N); G->z = c.take<double>(N);
    G->pf = c.take<float2>((size_t)kPcrLevels * N); G->prb = c.take<float>(N);
    G->ms = c.take<MState>(1); G->ctl = c.take<Ctl>(1);
    G->part = c.take<double>(3 * (size_t)maxch); G->cnt = c.take<int>(1);
    G->mass_part = c.take<double>(mass_blocks(N)); G->summary = c.take<Summary>(1);
    if (g) { g->N = N; g->maxch = maxch; g->maxpb = maxpb; g->nblk = nblk; g->nmass = mass_blocks(N); }
    return (c.off + kAlign2 - 1) / kAlign2 * kAlign2;
}

#define CK2(call)                                       \
    do {                                                \
        if ((call) != cudaSuccess) return NH_ERR_CUDA;  \
    } while (0)

Kin2 kin_at(const nh_grid2d* g, double t)
{
    Kin2 k{0.0, 0.0, 0.0};
    if (g->slide.shape == NH_SLIDE_GAUSS_LNCOSH) {
        const double z = t / g->t0;
        k.s = g->s0 * std::log(std::cosh(z));
        k.sd = (g->s0 / g->t0) * std::tanh(z);
        k.sdd = (g->s0 / (g->t0 * g->t0)) / (std::cosh(z) * std::cosh(z));
    }
    return k;
}

Geo2 geo2(const nh_grid2d* g)
{
    Geo2 G;
    G.nx = g->nx; G.ny = g->ny; G.bcx = g->d.bc_x; G.bcy = g->d.bc_y; G.lim = g->d.limiter;
    G.dx = g->d.dx; G.dy = g->d.dy; G.x0 = g->d.x0; G.y0 = g->d.y0; G.g = g->d.g;
    return G;
}

SolveArgs<double> solve_args2(nh_grid2d* g, int lnew, double gscale)
{
    SolveArgs<double> a;
    a.nb = 1; a.pitch = g->N; a.maxch = g->maxch;
    a.list = g->list[lnew];
    a.diag = g->diag; a.offl = g->offl; a.offr = g->offr; a.R = g->R;
    a.nbl = g->nbl; a.nbr = g->nbr;
    a.psi_prev = g->psi; a.guess_scale = gscale;
    a.x = g->x; a.r = g->r; a.p0 = g->p0; a.p1 = g->p1; a.q = g->qv; a.rh = g->rh;
    a.v0 = g->v0; a.v1 = g->v1; a.s = g->s; a.t = g->t; a.r1 = g->r1; a.z = g->z;
    a.pf = g->pf; a.prb = g->prb; a.pf_stride = (size_t)g->N;
    a.n_ext = 6; a.ext_c = g->ext_c; a.ext_k = g->ext_k; a.ext_stride = (size_t)g->N;
    a.maxpb = g->maxpb; a.items = g->items; a.pitems = g->pitems;
    a.tc = nullptr; a.ms = g->ms; a.ctl = g->ctl; a.part = g->part; a.cnt = g->cnt;
    a.rtol = g->rtol; a.max_iter = g->max_iter; a.it = 0;
    return a;
}

// One Krylov pass: set-up, then preconditioned CG in one cooperative launch,
// or preconditioned BiCGStab driven from the host.
nh_status krylov2_pass(nh_grid2d* g, SolveArgs<double>& sa)
{
    cudaStream_t st = g->stream;
    CK2(cudaMemsetAsync(g->ctl, 0, 3 * sizeof(int), st));
    CK2(cudaMemsetAsync(g->cnt, 0, sizeof(int), st));
    k_solve_init<double><<<g->items_grid, kChunk, 0, st>>>(sa);
    Ctl h;
    CK2(cudaMemcpyAsync(&h, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK2(cudaStreamSynchronize(st));
    const size_t pcr_smem = 2 * sizeof(float) * (size_t)kPcrRows;
    if (h.n_cg > 0 || h.n_bicg > 0)
        k_pcr_factor<double, float><<<g->pcr_grid, kPcrThreads, 3 * sizeof(float) * kPcrRows, st>>>(sa);
    if (h.n_cg > 0) {
        sa.it = 0;
        k_pcr<double, float><<<g->pcr_grid, kPcrThreads, pcr_smem, st>>>(sa, PCR_PCG);
    }
    if (h.not_done <= 0) return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
    if (h.n_cg > 0 && g->coop_grid > 0) {
        CK2(cudaMemsetAsync(&g->ctl->timeout, 0, 3 * sizeof(int), st));
        long long budget = g->barrier_budget;
        void* args[] = {(void*)&sa, (void*)&budget};
        CK2(cudaLaunchCooperativeKernel((const void*)k_pcg_persistent<double, float>, dim3(g->coop_grid),
                                        dim3(kPcrThreads), args, pcr_smem, st));
        int to = 0;
        CK2(cudaMemcpyAsync(&to, &g->ctl->timeout, sizeof(int), cudaMemcpyDeviceToHost, st));
        CK2(cudaStreamSynchronize(st));
        return to ? NH_ERR_TIMEOUT : NH_OK;
    }
    for (int it = 1; it <= g->max_iter; ++it) {
        sa.it = it;
        if (h.n_cg > 0) {
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
    k_fallback_reset<<<1, 32, 0, st>>>(g->ms, 1);
    return krylov2_pass(g, sa);
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
    const Geo2 G = geo2(g);
    const Kin2 Kn = kin_at(g, t_n), Kn1 = kin_at(g, t_n1);
    const int eg = g->elem_grid;

    k2_depth<<<eg, 256, 0, st>>>(G, g->d0, g->slide, Kn.s, g->dn);
    k2_depth<<<eg, 256, 0, st>>>(G, g->d0, g->slide, Kn1.s, g->dn1);
    StageArgs sa1;
    sa1.G = G;
    sa1.h = g->q[cur][0]; sa1.hu = g->q[cur][1]; sa1.hv = g->q[cur][2]; sa1.hw = g->q[cur][3]; sa1.d = g->dn;
    sa1.h0 = g->q[cur][0]; sa1.hu0 = g->q[cur][1]; sa1.hv0 = g->q[cur][2]; sa1.hw0 = g->q[cur][3];
    sa1.k1h = g->k1[0]; sa1.k1u = g->k1[1]; sa1.k1v = g->k1[2]; sa1.k1w = g->k1[3];
    sa1.oh = g->qs[0]; sa1.ohu = g->qs[1]; sa1.ohv = g->qs[2]; sa1.ohw = g->qs[3];
    sa1.dt = dt; sa1.stage = 1;
    k2_stage<<<eg, 256, 0, st>>>(sa1);
    StageArgs sa2 = sa1;
    sa2.h = g->qs[0]; sa2.hu = g->qs[1]; sa2.hv = g->qs[2]; sa2.hw = g->qs[3]; sa2.d = g->dn1;
    sa2.oh = g->q[nxt][0]; sa2.ohu = g->q[nxt][1]; sa2.ohv = g->q[nxt][2]; sa2.ohw = g->q[nxt][3];
    sa2.stage = 2;
    k2_stage<<<eg, 256, 0, st>>>(sa2);

    const bool all = g->crit == NH_CRIT_GLOBAL || (g->first_global && g->steps == 0);
    if (all) CK2(cudaMemsetAsync(g->marks, 1, g->N, st));
    else if (g->crit == NH_CRIT_HYDROSTATIC) CK2(cudaMemsetAsync(g->marks, 0, g->N, st));
    else k2_marks<<<eg, 256, 0, st>>>(G, g->q[nxt][0], g->q[nxt][1], g->q[nxt][2], g->q[nxt][3], g->dn1,
                                     g->crit, g->knh, g->marks);
    k2_dilate<<<eg, 256, 0, st>>>(G, g->marks, all ? 0 : g->enlarge, g->act);
    k2_count<<<g->nblk, kCompact2, 0, st>>>(g->act, g->N, g->bcnt);
    k2_scan<<<1, 1024, 0, st>>>(g->bcnt, g->nblk, g->boff, g->nact[lnew], g->ms);
    k2_emit<<<g->nblk, kCompact2, 0, st>>>(g->act, g->N, g->boff, g->list[lnew], g->inv);
    k_items<<<1, 1024, 0, st>>>(g->ms, 1, g->items, g->pitems, g->ctl);
    CK2(cudaMemsetAsync(g->cnt, 0, sizeof(int), st));

    Asm2Args aa;
    aa.G = G;
    aa.ht = g->q[nxt][0]; aa.hut = g->q[nxt][1]; aa.hvt = g->q[nxt][2]; aa.hwt = g->q[nxt][3];
    aa.d0 = g->d0; aa.d1 = g->dn1; aa.S = g->slide; aa.K = Kn1; aa.dt = dt;
    aa.list = g->list[lnew]; aa.inv = g->inv; aa.ms = g->ms;
    aa.diag = g->diag; aa.offl = g->offl; aa.offr = g->offr; aa.R = g->R;
    aa.nbl = g->nbl; aa.nbr = g->nbr;
    aa.ext_c = g->ext_c; aa.ext_k = g->ext_k; aa.ext_stride = (size_t)g->N;
    aa.c6 = g->c6; aa.cx = g->cx; aa.cy = g->cy; aa.phi = g->phi; aa.ddx = g->ddx; aa.ddy = g->ddy;
    aa.part = g->part; aa.cnt = g->cnt; aa.solver = NH_SOLVER_AUTO;
    aa.items = g->items; aa.ctl = g->ctl;
    k2_assemble<<<g->items_grid, kChunk, 0, st>>>(aa);
    CK2(cudaGetLastError());

    const double gscale = (g->guess == NH_GUESS_PREV && g->last_dt > 0.0) ? dt / g->last_dt : 0.0;
    SolveArgs<double> sa = solve_args2(g, lnew, gscale);
    nh_status rc = krylov2(g, sa);
    if (rc != NH_OK) return rc;

    k2_mass<<<g->nmass, 256, 0, st>>>(g->q[nxt][0], g->N, g->mass_part);
    k_summary<<<1, 256, 0, st>>>(g->ms, 1, g->mass_part, g->nmass, g->d.dx * g->d.dy, g->summary, nullptr);
    Summary S;
    CK2(cudaMemcpyAsync(&S, g->summary, sizeof(Summary), cudaMemcpyDeviceToHost, st));
    CK2(cudaStreamSynchronize(st));
    CK2(cudaGetLastError());
    const nh_status status = (nh_status)S.status;
    if (status == NH_OK) {
        ClearArgs cl;
        cl.nb = 1; cl.pitch = g->N; cl.maxlist = g->N;
        cl.list_prev = g->list[lprev]; cl.nact_prev = g->nact[lprev]; cl.psi = g->psi; cl.tc = nullptr;
        k_clear_prev<<<eg, 256, 0, st>>>(cl);
        if (S.n_active > 0) {
            Corr2Args co;
            co.G = G; co.n = (int)S.n_active; co.list = g->list[lnew];
            co.nbl = g->nbl; co.nbr = g->nbr; co.ext_k = g->ext_k; co.ext_stride = (size_t)g->N;
            co.x = g->x; co.c6 = g->c6; co.cx = g->cx; co.cy = g->cy; co.phi = g->phi;
            co.ddx = g->ddx; co.ddy = g->ddy; co.ms = g->ms;
            co.hu = g->q[nxt][1]; co.hv = g->q[nxt][2]; co.hw = g->q[nxt][3]; co.psi = g->psi;
            k2_correct<<<eg, 256, 0, st>>>(co);
        }
        CK2(cudaGetLastError());
        g->cur = nxt;
        g->lcur = lnew;
        g->n_since += 1;
        g->steps += 1;
        g->last_dt = dt;
    }
    if (info) {
        info->step = g->steps;
        info->t = status == NH_OK ? t_n1 : t_n;
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
    return status;
}

}  // namespace

extern "C" {

size_t nh2d_workspace_bytes(const nh_grid2d_desc* desc)
{
    if (!desc2_ok(desc)) return 0;
    return carve2(*desc, nullptr, nullptr);
}

nh_status nh2d_create(const nh_grid2d_desc* desc, const double* d0_host, void* ws, size_t ws_bytes,
                      void* stream, nh_grid2d** out)
{
    if (!out || !desc2_ok(desc) || !d0_host || !ws) return NH_ERR_ARG;
    *out = nullptr;
    const size_t need = carve2(*desc, nullptr, nullptr);
    if (ws_bytes < need || ((uintptr_t)ws % kAlign2) != 0) return NH_ERR_ARG;
    const long long N = (long long)desc->nx * desc->ny;
    for (long long q = 0; q < N; ++q)
        if (!(d0_host[q] > 0.0) || !std::isfinite(d0_host[q])) return NH_ERR_ARG;
    nh_grid2d* g = new (std::nothrow) nh_grid2d;
    if (!g) return NH_ERR_CUDA;
    std::memset(static_cast<void*>(g), 0, sizeof(*g));
    g->d = *desc;
    g->stream = static_cast<cudaStream_t>(stream);
    g->nx = desc->nx; g->ny = desc->ny;
    carve2(*desc, g, static_cast<char*>(ws));
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, dev);
    if (g->sms < 1) g->sms = 1;
    g->items_grid = std::max(1, std::min(g->maxch, g->sms * 8));
    g->pcr_grid = std::max(1, std::min(g->maxpb, g->sms * 2));
    g->elem_grid = std::max(1, std::min((g->N + 255) / 256, g->sms * 8));
    g->slide.shape = NH_SLIDE_NONE; g->slide.A = 0.0; g->slide.Lx = g->slide.Ly = 1.0;
    g->s0 = 0.0; g->t0 = 1.0;
    g->crit = NH_CRIT_GLOBAL; g->knh = 1e-3; g->enlarge = 1; g->first_global = 0;
    g->rtol = 1e-12; g->max_iter = 20000; g->guess = NH_GUESS_PREV;
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
        int clk_khz = 0;
        cudaDeviceGetAttribute(&clk_khz, cudaDevAttrClockRate, dev);
        g->barrier_budget = (long long)(clk_khz > 0 ? clk_khz : 2000000) * 1000LL;   // about one second
        if (cudaMemsetAsync(ws, 0, need, st) != cudaSuccess ||
            cudaMemcpyAsync(g->d0, d0_host, sizeof(double) * N, cudaMemcpyHostToDevice, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
    } while (0);
    if (rc != NH_OK) { delete g; return rc; }
    *out = g;
    return NH_OK;
}

nh_status nh2d_set_bottom_motion(nh_grid2d* g, const nh_slide2d_desc* s)
{
    if (!g) return NH_ERR_ARG;
    if (!s || s->shape == NH_SLIDE_NONE) {
        g->slide.shape = NH_SLIDE_NONE;
        return NH_OK;
    }
    if (s->shape != NH_SLIDE_GAUSS_LNCOSH || !(s->Lx > 0.0) || !(s->Ly > 0.0) || !(s->t0 > 0.0) ||
        !std::isfinite(s->A) || !std::isfinite(s->xc0) || !std::isfinite(s->yc0) || !std::isfinite(s->s0))
        return NH_ERR_ARG;
    g->slide.shape = NH_SLIDE_GAUSS_LNCOSH;
    g->slide.A = s->A; g->slide.Lx = s->Lx; g->slide.Ly = s->Ly; g->slide.xc0 = s->xc0; g->slide.yc0 = s->yc0;
    g->s0 = s->s0; g->t0 = s->t0;
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

nh_status nh2d_set_state(nh_grid2d* g, const double* h, const double* hu, const double* hv, const double* hw,
                         double t)
{
    if (!g || !h || !hu || !hv || !hw || !std::isfinite(t)) return NH_ERR_ARG;
    const size_t N = (size_t)g->N;
    for (size_t q = 0; q < N; ++q)
        if (!(h[q] > 0.0) || !std::isfinite(h[q]) || !std::isfinite(hu[q]) || !std::isfinite(hv[q]) ||
            !std::isfinite(hw[q]))
            return NH_ERR_ARG;
    cudaStream_t st = g->stream;
    const double* src[4] = {h, hu, hv, hw};
    for (int f = 0; f < 4; ++f)
        CK2(cudaMemcpyAsync(g->q[0][f], src[f], sizeof(double) * N, cudaMemcpyHostToDevice, st));
    CK2(cudaMemsetAsync(g->psi, 0, sizeof(double) * N, st));
    CK2(cudaMemsetAsync(g->nact[0], 0, sizeof(int), st));
    CK2(cudaMemsetAsync(g->nact[1], 0, sizeof(int), st));
    CK2(cudaMemsetAsync(g->act, 0, N, st));
    CK2(cudaStreamSynchronize(st));
    g->cur = 0; g->lcur = 0;
    g->has_state = true;
    g->t_base = t; g->n_since = 0; g->steps = 0; g->last_dt = 0.0;
    return NH_OK;
}

nh_status nh2d_get_state(nh_grid2d* g, double* h, double* hu, double* hv, double* hw, double* p_nh)
{
    if (!g) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    cudaStream_t st = g->stream;
    const size_t N = (size_t)g->N;
    double* dst[4] = {h, hu, hv, hw};
    for (int f = 0; f < 4; ++f)
        if (dst[f]) CK2(cudaMemcpyAsync(dst[f], g->q[g->cur][f], sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    std::vector<double> hh, ps;
    if (p_nh) {
        hh.resize(N); ps.resize(N);
        CK2(cudaMemcpyAsync(hh.data(), g->q[g->cur][0], sizeof(double) * N, cudaMemcpyDeviceToHost, st));
        CK2(cudaMemcpyAsync(ps.data(), g->psi, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    }
    CK2(cudaStreamSynchronize(st));
    if (p_nh) {
        const double sc = g->last_dt > 0.0 ? g->d.rho / g->last_dt : 0.0;   // p = rho psi / (dt h)
        for (size_t q = 0; q < N; ++q) p_nh[q] = sc * ps[q] / hh[q];
    }
    return NH_OK;
}

nh_status nh2d_get_mask(nh_grid2d* g, unsigned char* mask)
{
    if (!g || !mask) return NH_ERR_ARG;
    CK2(cudaMemcpyAsync(mask, g->act, (size_t)g->N, cudaMemcpyDeviceToHost, g->stream));
    CK2(cudaStreamSynchronize(g->stream));
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
    for (long long k = 0; k < n_steps; ++k) {
        nh_step_info si;
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

void nh2d_destroy(nh_grid2d* g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    delete g;
}

}  // extern "C"
