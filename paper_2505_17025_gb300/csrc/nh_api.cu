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
#include <new>
#include <vector>

#include "nh_kernels1d.cuh"

using namespace nh;

struct nh_grid {
    nh_grid_desc d;
    cudaStream_t stream;
    int nx, nb, pitch, wpitch, ntiles, maxch, sm_count, items_grid;
    size_t es;                   // element size of state / vectors
    // configuration
    int crit, enlarge, first_global;
    double knh;
    int solver, max_iter, guess, ir_max;
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
    void* sh[2]; void* shu[2]; void* shw[2];
    void* d0;
    Slide* slide; Kin* kin;
    uint32_t* marks; uint32_t* act;
    int* list[2]; int* nact[2];
    void *diag, *offl, *offr, *R, *c6, *cx, *phi, *ddx;
    int *nbl, *nbr;
    void *x, *r, *p0, *p1, *q, *rh, *v0, *v1, *s, *t;
    double* psi;
    MState* ms; Ctl* ctl; double* part; int* cnt;
    double* mass_part; Summary* summary;
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
    if (d->precision != NH_FP64) return false;
    if (d->limiter < NH_LIM_NONE || d->limiter > NH_LIM_MC) return false;
    if (!(d->dx > 0.0) || !(d->g > 0.0) || !(d->rho > 0.0) || !std::isfinite(d->x0)) return false;
    return true;
}

// Lay out every buffer; with base == nullptr only the size is computed.
size_t carve(const nh_grid_desc& d, nh_grid* g, char* base)
{
    const int nx = d.nx, nb = d.nbatch;
    const int pitch = (nx + kPredTile - 1) / kPredTile * kPredTile;
    const int wpitch = pitch / 32;
    const int ntiles = pitch / kPredTile;
    const int maxch = (nx + kChunk - 1) / kChunk;
    const size_t N = (size_t)nb * pitch;
    const size_t es = 8;
    Carver c{base};
    nh_grid tmp;
    nh_grid* G = g ? g : &tmp;
    for (int k = 0; k < 2; ++k) {
        G->sh[k] = c.take(N * es); G->shu[k] = c.take(N * es); G->shw[k] = c.take(N * es);
    }
    G->d0 = c.take(N * es);
    G->slide = (Slide*)c.take(sizeof(Slide) * nb);
    G->kin = (Kin*)c.take(sizeof(Kin) * nb);
    G->marks = (uint32_t*)c.take(sizeof(uint32_t) * (size_t)nb * wpitch);
    G->act = (uint32_t*)c.take(sizeof(uint32_t) * (size_t)nb * wpitch);
    for (int k = 0; k < 2; ++k) {
        G->list[k] = (int*)c.take(sizeof(int) * N);
        G->nact[k] = (int*)c.take(sizeof(int) * nb);
    }
    G->diag = c.take(N * es); G->offl = c.take(N * es); G->offr = c.take(N * es);
    G->R = c.take(N * es);
    G->c6 = c.take(N * es); G->cx = c.take(N * es); G->phi = c.take(N * es); G->ddx = c.take(N * es);
    G->nbl = (int*)c.take(sizeof(int) * N); G->nbr = (int*)c.take(sizeof(int) * N);
    G->x = c.take(N * es); G->r = c.take(N * es); G->p0 = c.take(N * es); G->p1 = c.take(N * es);
    G->q = c.take(N * es); G->rh = c.take(N * es); G->v0 = c.take(N * es); G->v1 = c.take(N * es);
    G->s = c.take(N * es); G->t = c.take(N * es);
    G->psi = (double*)c.take(sizeof(double) * N);
    G->ms = (MState*)c.take(sizeof(MState) * nb);
    G->ctl = (Ctl*)c.take(sizeof(Ctl));
    G->part = (double*)c.take(sizeof(double) * 3 * (size_t)nb * maxch);
    G->cnt = (int*)c.take(sizeof(int) * nb);
    G->mass_part = (double*)c.take(sizeof(double) * (size_t)nb * ntiles);
    G->summary = (Summary*)c.take(sizeof(Summary));
    if (g) {
        g->nx = nx; g->nb = nb; g->pitch = pitch; g->wpitch = wpitch; g->ntiles = ntiles;
        g->maxch = maxch; g->es = es;
    }
    return (c.off + kAlign - 1) / kAlign * kAlign;
}

#define CK(call)                                        \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return NH_ERR_CUDA;      \
    } while (0)

Geo geo(const nh_grid* g)
{
    Geo G;
    G.nx = g->nx; G.nb = g->nb; G.pitch = g->pitch; G.wpitch = g->wpitch; G.bc = g->d.bc;
    G.lim = g->d.limiter; G.ntiles = g->ntiles; G.maxch = g->maxch;
    G.dx = g->d.dx; G.x0 = g->d.x0; G.g = g->d.g;
    return G;
}

SolveArgs<double> solve_args(nh_grid* g, int lcur)
{
    SolveArgs<double> a;
    a.nb = g->nb; a.pitch = g->pitch; a.maxch = g->maxch;
    a.list = g->list[lcur];
    a.diag = (const double*)g->diag; a.offl = (const double*)g->offl; a.offr = (const double*)g->offr;
    a.nbl = g->nbl; a.nbr = g->nbr; a.R = (const double*)g->R;
    a.psi_prev = g->psi; a.guess_scale = 0.0;
    a.x = (double*)g->x; a.r = (double*)g->r; a.p0 = (double*)g->p0; a.p1 = (double*)g->p1;
    a.q = (double*)g->q; a.rh = (double*)g->rh; a.v0 = (double*)g->v0; a.v1 = (double*)g->v1;
    a.s = (double*)g->s; a.t = (double*)g->t;
    a.ms = g->ms; a.ctl = g->ctl; a.part = g->part; a.cnt = g->cnt;
    a.rtol = g->rtol; a.max_iter = g->max_iter; a.it = 0;
    return a;
}

// One step; on success swaps the state and list buffers.
nh_status do_step(nh_grid* g, double dt, nh_step_info* info)
{
    if (!g->has_state) return NH_ERR_STATE;
    if (!(dt > 0.0) || !std::isfinite(dt)) return NH_ERR_ARG;
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

    k_kinematics<<<(g->nb + 127) / 128, 128, 0, st>>>(g->slide, g->kin, g->nb, t_n, t_n1);

    PredArgs<double> pa;
    pa.G = G;
    pa.h = (const double*)g->sh[cur]; pa.hu = (const double*)g->shu[cur]; pa.hw = (const double*)g->shw[cur];
    pa.ht = (double*)g->sh[nxt]; pa.hut = (double*)g->shu[nxt]; pa.hwt = (double*)g->shw[nxt];
    pa.d0 = (const double*)g->d0; pa.slide = g->slide; pa.kin = g->kin;
    pa.marks = g->marks; pa.mass_part = g->mass_part; pa.dt = dt; pa.knh = g->knh; pa.crit = g->crit;
    pa.all_global = (g->crit == NH_CRIT_GLOBAL) || (g->first_global && g->steps == 0);
    k_predict<double><<<dim3(g->ntiles, g->nb), kPredTile, 0, st>>>(pa);

    CompactArgs ca;
    ca.nx = g->nx; ca.pitch = g->pitch; ca.wpitch = g->wpitch; ca.bc = g->d.bc; ca.enlarge = g->enlarge;
    ca.marks = g->marks; ca.act = g->act; ca.list = g->list[lnew]; ca.nact = g->nact[lnew];
    ca.ms = g->ms; ca.ctl = g->ctl;
    const size_t csm = sizeof(uint32_t) * (size_t)((g->nx + 31) / 32);
    k_compact<<<g->nb, kCompactThreads, csm, st>>>(ca);

    AsmArgs<double> aa;
    aa.G = G;
    aa.ht = (const double*)g->sh[nxt]; aa.hut = (const double*)g->shu[nxt]; aa.hwt = (const double*)g->shw[nxt];
    aa.d0 = (const double*)g->d0; aa.slide = g->slide; aa.kin = g->kin;
    aa.list = g->list[lnew]; aa.act = g->act; aa.ms = g->ms;
    aa.diag = (double*)g->diag; aa.offl = (double*)g->offl; aa.offr = (double*)g->offr; aa.R = (double*)g->R;
    aa.nbl = g->nbl; aa.nbr = g->nbr;
    aa.c6 = (double*)g->c6; aa.cx = (double*)g->cx; aa.phi = (double*)g->phi; aa.ddx = (double*)g->ddx;
    aa.part = g->part; aa.cnt = g->cnt; aa.dt = dt; aa.solver = g->solver;
    k_assemble<double><<<g->items_grid, kChunk, 0, st>>>(aa);

    SolveArgs<double> sa = solve_args(g, lnew);
    sa.guess_scale = (g->guess == NH_GUESS_PREV && g->last_dt > 0.0) ? dt / g->last_dt : 0.0;
    k_solve_init<double><<<g->items_grid, kChunk, 0, st>>>(sa);
    Ctl hctl;
    CK(cudaMemcpyAsync(&hctl, g->ctl, sizeof(Ctl), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    if (hctl.not_done > 0) {
        for (int it = 1; it <= g->max_iter; ++it) {
            sa.it = it;
            if (hctl.n_cg > 0) {
                k_cg_a<double><<<g->items_grid, kChunk, 0, st>>>(sa);
                k_cg_b<double><<<g->items_grid, kChunk, 0, st>>>(sa);
            }
            if (hctl.n_bicg > 0) {
                k_bi_1<double><<<g->items_grid, kChunk, 0, st>>>(sa);
                k_bi_2<double><<<g->items_grid, kChunk, 0, st>>>(sa);
                k_bi_3<double><<<g->items_grid, kChunk, 0, st>>>(sa);
            }
            if (it % g->poll_every == 0 || it == g->max_iter) {
                int nd = 0;
                CK(cudaMemcpyAsync(&nd, &g->ctl->not_done, sizeof(int), cudaMemcpyDeviceToHost, st));
                CK(cudaStreamSynchronize(st));
                if (nd <= 0) break;
            }
        }
    }
    k_summary<<<1, 256, 0, st>>>(g->ms, g->nb, g->mass_part, g->nb * g->ntiles, g->d.dx, g->summary);
    Summary S;
    CK(cudaMemcpyAsync(&S, g->summary, sizeof(Summary), cudaMemcpyDeviceToHost, st));
    CK(cudaStreamSynchronize(st));
    CK(cudaGetLastError());
    nh_status status = (nh_status)S.status;
    if (status == NH_OK) {
        ClearArgs cl;
        cl.nb = g->nb; cl.pitch = g->pitch; cl.maxlist = g->pitch;
        cl.list_prev = g->list[lprev]; cl.nact_prev = g->nact[lprev]; cl.psi = g->psi;
        const size_t total = (size_t)g->nb * g->pitch;
        int cgrid = (int)std::min<size_t>((total + 255) / 256, (size_t)g->sm_count * 8);
        k_clear_prev<<<cgrid, 256, 0, st>>>(cl);
        CorrArgs<double> co;
        co.nb = g->nb; co.pitch = g->pitch; co.maxch = g->maxch; co.dx = g->d.dx;
        co.list = g->list[lnew]; co.nbl = g->nbl; co.nbr = g->nbr; co.x = (const double*)g->x;
        co.c6 = (const double*)g->c6; co.cx = (const double*)g->cx; co.phi = (const double*)g->phi;
        co.ddx = (const double*)g->ddx; co.ms = g->ms;
        co.hu = (double*)g->shu[nxt]; co.hw = (double*)g->shw[nxt]; co.psi = g->psi;
        k_correct<double><<<g->items_grid, kChunk, 0, st>>>(co);
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

size_t nh_workspace_bytes(const nh_grid_desc* desc)
{
    if (!desc_ok(desc)) return 0;
    return carve(*desc, nullptr, nullptr);
}

nh_status nh_create_grid(const nh_grid_desc* desc, const double* d0_host, void* ws, size_t ws_bytes,
                         void* stream, nh_grid** out)
{
    if (!out) return NH_ERR_ARG;
    *out = nullptr;
    if (!desc_ok(desc) || !d0_host || !ws) return NH_ERR_ARG;
    if (((uintptr_t)ws % kAlign) != 0) return NH_ERR_ARG;
    const size_t need = carve(*desc, nullptr, nullptr);
    if (ws_bytes < need) return NH_ERR_ARG;
    for (size_t q = 0; q < (size_t)desc->nx * desc->nbatch; ++q)
        if (!(d0_host[q] > 0.0) || !std::isfinite(d0_host[q])) return NH_ERR_ARG;
    int dev = 0;
    CK(cudaGetDevice(&dev));
    int sms = 0;
    CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    nh_grid* g = new (std::nothrow) nh_grid();
    if (!g) return NH_ERR_ARG;
    g->d = *desc;
    g->stream = (cudaStream_t)stream;
    carve(*desc, g, (char*)ws);
    g->sm_count = sms;
    g->items_grid = (int)std::min<long long>((long long)g->nb * g->maxch, (long long)sms * 8);
    if (g->items_grid < 1) g->items_grid = 1;
    g->crit = NH_CRIT_GLOBAL; g->knh = 1e-3; g->enlarge = 1; g->first_global = 0;
    g->solver = NH_SOLVER_AUTO; g->rtol = 1e-12; g->max_iter = 20000; g->guess = NH_GUESS_PREV;
    g->ir_max = 8; g->inner_rtol = 1e-5; g->poll_every = 16;
    g->has_state = false; g->t_base = 0.0; g->n_since = 0; g->steps = 0; g->last_dt = 0.0;
    g->cur = 0; g->lcur = 0;
    cudaStream_t st = g->stream;
    const size_t hp = (size_t)g->nx * sizeof(double), dp = (size_t)g->pitch * sizeof(double);
    nh_status rc = NH_OK;
    do {
        if (cudaMemsetAsync(ws, 0, need, st) != cudaSuccess) { rc = NH_ERR_CUDA; break; }
        if (cudaMemcpy2DAsync(g->d0, dp, d0_host, hp, hp, g->nb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        std::vector<Slide> sl(g->nb);
        for (auto& s : sl) { s.A = 0; s.L = 1; s.xc0 = 0; s.s0 = 0; s.t0 = 1; s.shape = NH_SLIDE_NONE; s.pad = 0; }
        if (cudaMemcpyAsync(g->slide, sl.data(), sizeof(Slide) * g->nb, cudaMemcpyHostToDevice, st) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
        if (cudaStreamSynchronize(st) != cudaSuccess) { rc = NH_ERR_CUDA; break; }
        if (cudaFuncSetAttribute(k_compact, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(sizeof(uint32_t) * ((g->nx + 31) / 32))) != cudaSuccess) {
            rc = NH_ERR_CUDA; break;
        }
    } while (0);
    if (rc != NH_OK) { delete g; return rc; }
    *out = g;
    return NH_OK;
}

nh_status nh_set_bottom_motion(nh_grid* g, const nh_slide_desc* slides)
{
    if (!g) return NH_ERR_ARG;
    std::vector<Slide> sl(g->nb);
    for (int b = 0; b < g->nb; ++b) {
        Slide s{0.0, 1.0, 0.0, 0.0, 1.0, NH_SLIDE_NONE, 0};
        if (slides) {
            const nh_slide_desc& q = slides[b];
            if (q.shape != NH_SLIDE_NONE && q.shape != NH_SLIDE_GAUSS_LNCOSH) return NH_ERR_ARG;
            if (q.shape == NH_SLIDE_GAUSS_LNCOSH) {
                if (!(q.L > 0.0) || !(q.t0 > 0.0) || !std::isfinite(q.A) || !std::isfinite(q.xc0) ||
                    !std::isfinite(q.s0))
                    return NH_ERR_ARG;
                s.A = q.A; s.L = q.L; s.xc0 = q.xc0; s.s0 = q.s0; s.t0 = q.t0; s.shape = q.shape;
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
    if (!(rtol > 0.0) || max_iter < 1 || (guess != NH_GUESS_ZERO && guess != NH_GUESS_PREV)) return NH_ERR_ARG;
    if (ir_max < 1 || !(inner_rtol > 0.0)) return NH_ERR_ARG;
    g->solver = kind; g->rtol = rtol; g->max_iter = max_iter; g->guess = guess;
    g->ir_max = ir_max; g->inner_rtol = inner_rtol;
    return NH_OK;
}

nh_status nh_set_state(nh_grid* g, const double* h, const double* hu, const double* hw, double t)
{
    if (!g || !h || !hu || !hw || !std::isfinite(t)) return NH_ERR_ARG;
    cudaStream_t st = g->stream;
    const size_t hp = (size_t)g->nx * sizeof(double), dp = (size_t)g->pitch * sizeof(double);
    g->cur = 0;
    g->lcur = 0;
    CK(cudaMemcpy2DAsync(g->sh[0], dp, h, hp, hp, g->nb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpy2DAsync(g->shu[0], dp, hu, hp, hp, g->nb, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpy2DAsync(g->shw[0], dp, hw, hp, hp, g->nb, cudaMemcpyHostToDevice, st));
    CK(cudaMemsetAsync(g->psi, 0, sizeof(double) * (size_t)g->nb * g->pitch, st));
    CK(cudaMemsetAsync(g->nact[0], 0, sizeof(int) * g->nb, st));
    CK(cudaMemsetAsync(g->nact[1], 0, sizeof(int) * g->nb, st));
    CK(cudaStreamSynchronize(st));
    g->has_state = true;
    g->t_base = t; g->n_since = 0; g->steps = 0; g->last_dt = 0.0;
    return NH_OK;
}

nh_status nh_get_state(nh_grid* g, double* h, double* hu, double* hw, double* p_nh)
{
    if (!g) return NH_ERR_ARG;
    if (!g->has_state) return NH_ERR_STATE;
    cudaStream_t st = g->stream;
    const size_t hp = (size_t)g->nx * sizeof(double), dp = (size_t)g->pitch * sizeof(double);
    const int c = g->cur;
    if (h) CK(cudaMemcpy2DAsync(h, hp, g->sh[c], dp, hp, g->nb, cudaMemcpyDeviceToHost, st));
    if (hu) CK(cudaMemcpy2DAsync(hu, hp, g->shu[c], dp, hp, g->nb, cudaMemcpyDeviceToHost, st));
    if (hw) CK(cudaMemcpy2DAsync(hw, hp, g->shw[c], dp, hp, g->nb, cudaMemcpyDeviceToHost, st));
    std::vector<double> hh;
    if (p_nh) {
        CK(cudaMemcpy2DAsync(p_nh, hp, g->psi, dp, hp, g->nb, cudaMemcpyDeviceToHost, st));
        if (!h) {
            hh.resize((size_t)g->nx * g->nb);
            CK(cudaMemcpy2DAsync(hh.data(), hp, g->sh[c], dp, hp, g->nb, cudaMemcpyDeviceToHost, st));
        }
    }
    CK(cudaStreamSynchronize(st));
    if (p_nh) {
        const double* H = h ? h : hh.data();
        const double sc = g->last_dt > 0.0 ? g->d.rho / g->last_dt : 0.0;
        for (size_t q = 0; q < (size_t)g->nx * g->nb; ++q) p_nh[q] = sc * p_nh[q] / H[q];
    }
    return NH_OK;
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
            for (int i = 0; i < g->nx; ++i)
                mask[(size_t)b * g->nx + i] = (w[(size_t)b * g->wpitch + (i >> 5)] >> (i & 31)) & 1u;
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
    nh_run_info R;
    std::memset(&R, 0, sizeof(R));
    nh_status rc = NH_OK;
    for (long long k = 0; k < n_steps; ++k) {
        nh_step_info si;
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

void nh_destroy(nh_grid* g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
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
