// nh_cnn.cu -- the learned initial guess: four width-3 convolutions over the
// cells of each member, run as implicit GEMMs on the 5th-generation tensor
// cores (tcgen05.mma, BF16 operands in shared memory, FP32 accumulators in
// tensor memory), with the training kernels (loss, dgrad, wgrad, Adam).
//
// Network (identical to the FP64 oracle in oracle/cnn.py): channels
// 16 -> 32 -> 32 -> 32 -> 16, ReLU after the first three layers, output =
// channel 0 of the last layer, zero padding outside each member's cells.
// Parameters: one FP32 vector, per layer W[c_out][3 c_in] then b[c_out]; W's
// column k c_in + c weights input channel c of the cell at offset k - 1.
//
// GEMM mapping (M = 128 rows = cells of a tile, K-major BF16 operands with no
// swizzle: 8-row x 16-byte core matrices, leading-dimension step 128 B between
// K-neighbours, stride step between 8-row groups):
//   forward / dgrad : D[cell][n] = sum_K A[cell][K] B[n][K]
//   wgrad           : D[(k, c)][c_out] = sum_cells A'[(k, c)][cell] B'[c_out][cell]
// Every wait on the MMA completion barrier is bounded by a clock budget; on
// expiry the kernel records the failure, waits once more (bounded) for its
// MMAs in flight, releases its tensor memory and returns.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>
#include <utility>

#include "nh_cnn.cuh"

namespace nh {
namespace cnn {

typedef __nv_bfloat16 bf16;

constexpr int kRows = 128;                    // cells per GEMM tile (M)
constexpr int kHalo = 4;                      // four width-3 layers
constexpr int kTileOut = kRows - 2 * kHalo;   // output cells per forward tile
constexpr int kCh = 32;                       // channel stride of activation rows

__host__ __device__ constexpr int cin(int l) { return l == 0 ? 16 : 32; }
__host__ __device__ constexpr int cout(int l) { return l == 3 ? 16 : 32; }
__host__ __device__ constexpr int wsize(int l) { return cout(l) * 3 * cin(l); }
__host__ __device__ constexpr int woff(int l) { return l == 0 ? 0 : woff(l - 1) + wsize(l - 1) + cout(l - 1); }
__host__ __device__ constexpr int boff(int l) { return woff(l) + wsize(l); }
__host__ __device__ constexpr int sw_off(int l) { return l == 0 ? 0 : sw_off(l - 1) + wsize(l - 1); }
__host__ __device__ constexpr int sb_off(int l) { return l == 0 ? 0 : sb_off(l - 1) + cout(l - 1); }
constexpr int kNParams = boff(3) + cout(3);
constexpr int kWElems = sw_off(3) + wsize(3);
constexpr int kBias = sb_off(3) + cout(3);
static_assert(kNParams == NH_CNN_PARAMS, "parameter count");

// ----------------------------------------------------- tcgen05 building blocks

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Element offset of (row r, column k) in a K-major no-swizzle operand whose K
// extent is 8 nkc: core matrix (r/8, k/8) is 8 rows x 8 elements (16 bytes per
// row), core matrices ordered row-group major.
__device__ __forceinline__ int core_off(int r, int k, int nkc)
{
    return ((r >> 3) * nkc + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7);
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset 128 (K-neighbour core matrices), stride byte offset `sbo` (8-row
// groups), descriptor version 1, no swizzle.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)(128u >> 4) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N = n, M = 128.
__device__ __forceinline__ uint32_t idesc(int n)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(kRows >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id, uint32_t acc)
{
    asm volatile("{\n.reg .pred p;\nsetp.ne.u32 p, %4, 0;\n"
                 "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                 :: "r"(tmem), "l"(a), "l"(b), "r"(id), "r"(acc));
}

__device__ __forceinline__ void commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 :: "r"(smem_u32(mbar)));
}

__device__ __forceinline__ bool mbar_wait(uint64_t* mbar, uint32_t parity, long long budget)
{
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}"
                     : "=r"(done) : "r"(smem_u32(mbar)), "r"(parity));
        if (done) return true;
        if (clock64() - t0 > budget) return false;
    }
}

// Wait for the MMAs committed to `mbar` (phase `parity`); the outcome is
// agreed by the whole CTA, so every thread leaves its tile loop together.  On
// expiry the flag is raised once and each thread that gave up waits one more
// budget for the MMAs still in flight before the tensor memory is released.
__device__ __forceinline__ bool block_wait(uint64_t* mbar, uint32_t parity, long long budget, int* status)
{
    const bool mine = mbar_wait(mbar, parity, budget);
    if (__syncthreads_and(mine)) return true;
    if (threadIdx.x == 0 && status) atomicExch(status, NH_ERR_TIMEOUT);
    if (!mine) mbar_wait(mbar, parity, budget);
    return false;
}

__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v)
{
    uint32_t r[32];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                 "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
                   "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
                   "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v)
{
    uint32_t r[16];
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
                 "%14,%15}, [%16];"
                 : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
                   "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
                   "=r"(r[14]), "=r"(r[15])
                 : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;");
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// Tensor memory: 32 columns (128 lanes x 32 FP32) per CTA, allocated by warp 0.
__device__ __forceinline__ void tmem_alloc(uint32_t* slot)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 32;" :: "r"(smem_u32(slot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 32;" :: "r"(tmem));
}

__device__ __forceinline__ void mbar_init(uint64_t* mbar)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
}

__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;"); }
__device__ __forceinline__ void tc_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;"); }
__device__ __forceinline__ void tc_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;"); }

__device__ __forceinline__ int member_cells(const int* nxv, int b) { return nxv[b]; }

// ----------------------------------------------------------------- forward

struct FwdArgs {
    const bf16* feat;        // [nb * pitch][16]
    const int* nxv;          // cells per member (device)
    int nb, pitch, ntiles;   // ntiles = forward tiles per member
    const float* params;     // FP32 master parameters
    float* y;                // [nb * pitch] output (channel 0) times out_scale
    float out_scale;
    bf16* acts;              // nullable: [3][nb * pitch][32] hidden activations (training)
    const uint32_t* act;     // nullable: mask bits [nb][wpitch]; tiles with no marked output cell are skipped
    int wpitch;
    int* status;             // nullable: NH_ERR_TIMEOUT when a bounded wait expired
    long long budget;
};

constexpr size_t kFwdSmem = sizeof(bf16) * (kRows * 96 + kWElems + kRows * kCh) + sizeof(float) * kBias + 16;

// One CTA (128 threads, thread = row) per 120-cell tile at a time: the tile's
// 128 rows (4-cell halo each side) pass through all four layers with the
// activations kept in shared memory; rows 4..123 are exact after layer 4.
__global__ void __launch_bounds__(kRows) k_forward(FwdArgs a)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    bf16* sA = reinterpret_cast<bf16*>(smraw);            // 128 x K (core layout)
    bf16* sW = sA + kRows * 96;                            // all weights (core layout)
    bf16* sAct = sW + kWElems;                             // 128 rows x 32 channels
    float* sBias = reinterpret_cast<float*>(sAct + kRows * kCh);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sBias + kBias);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5;

    for (int l = 0; l < 4; ++l) {
        const int K = 3 * cin(l), nkc = K / 8;
        for (int e = tid; e < wsize(l); e += kRows)
            sW[sw_off(l) + core_off(e / K, e % K, nkc)] = __float2bfloat16(a.params[woff(l) + e]);
        for (int e = tid; e < cout(l); e += kRows) sBias[sb_off(l) + e] = a.params[boff(l) + e];
    }
    if (warp == 0) tmem_alloc(tslot);
    if (tid == 0) mbar_init(mbar);
    fence_async_smem();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t parity = 0;
    bool ok = true;

    const int total = a.nb * a.ntiles;
    for (int w = blockIdx.x; w < total && ok; w += gridDim.x) {
        const int b = w / a.ntiles, t = w - b * a.ntiles;
        const int nxb = member_cells(a.nxv, b);
        if (t * kTileOut >= nxb) continue;                 // block-uniform
        if (a.act) {
            // skip the tile unless one of its output cells is marked
            const int c0 = t * kTileOut, c1 = min(c0 + kTileOut, nxb);
            bool hit = false;
            const int w0 = c0 >> 5, w1 = (c1 - 1) >> 5;
            if (tid <= w1 - w0) {
                const int w = w0 + tid;
                uint32_t bits = a.act[(size_t)b * a.wpitch + w];
                const int lo = max(c0 - 32 * w, 0), hi = min(c1 - 32 * w, 32);
                const uint32_t keep = (hi >= 32 ? 0xFFFFFFFFu : ((1u << hi) - 1u)) & ~((1u << lo) - 1u);
                hit = (bits & keep) != 0;
            }
            if (!__syncthreads_or(hit)) continue;
        }
        const int cell = t * kTileOut - kHalo + tid;
        const bool valid = cell >= 0 && cell < nxb;
        const size_t gi = (size_t)b * a.pitch + cell;
        uint4 f0 = make_uint4(0, 0, 0, 0), f1 = f0;
        if (valid) {
            const uint4* src = reinterpret_cast<const uint4*>(a.feat + gi * 16);
            f0 = src[0];
            f1 = src[1];
        }
        reinterpret_cast<uint4*>(sAct + tid * kCh)[0] = f0;
        reinterpret_cast<uint4*>(sAct + tid * kCh)[1] = f1;
        for (int l = 0; l < 4 && ok; ++l) {
            const int Ci = cin(l), Co = cout(l), K = 3 * Ci, nkc = K / 8;
            __syncthreads();
            // operand A: row tid = [act(row-1), act(row), act(row+1)] (zero off the tile)
            for (int k = 0; k < 3; ++k) {
                const int rr = tid + k - 1;
                for (int q = 0; q < Ci / 8; ++q) {
                    uint4 v = make_uint4(0, 0, 0, 0);
                    if (rr >= 0 && rr < kRows) v = reinterpret_cast<const uint4*>(sAct + rr * kCh)[q];
                    *reinterpret_cast<uint4*>(sA + core_off(tid, k * Ci + q * 8, nkc)) = v;
                }
            }
            fence_async_smem();
            __syncthreads();
            if (tid == 0) {
                tc_after_sync();
                const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sW + sw_off(l));
                for (int kk = 0; kk < K / 16; ++kk)
                    mma(tmem, sdesc(aaddr + kk * 256, nkc * 128), sdesc(baddr + kk * 256, nkc * 128), idesc(Co),
                        kk > 0 ? 1u : 0u);
                commit(mbar);
            }
            if (!block_wait(mbar, parity, a.budget, a.status)) {
                ok = false;
                break;
            }
            parity ^= 1u;
            tc_after_sync();
            float v[32];
            if (Co == 32) tmem_ld32(trow, v); else tmem_ld16(trow, v);
            tc_before_sync();
            const bool out_row = tid >= kHalo && tid < kRows - kHalo;
            if (l < 3) {
                __align__(16) bf16 o[32];
#pragma unroll
                for (int j = 0; j < 32; ++j) {
                    float z = fmaxf(v[j] + sBias[sb_off(l) + j], 0.0f);
                    o[j] = __float2bfloat16(valid ? z : 0.0f);
                }
                uint4* dst = reinterpret_cast<uint4*>(sAct + tid * kCh);
                const uint4* srcv = reinterpret_cast<const uint4*>(o);
#pragma unroll
                for (int q = 0; q < 4; ++q) dst[q] = srcv[q];
                if (a.acts && out_row && valid) {
                    uint4* g = reinterpret_cast<uint4*>(a.acts + ((size_t)l * a.nb * a.pitch + gi) * kCh);
#pragma unroll
                    for (int q = 0; q < 4; ++q) g[q] = srcv[q];
                }
            } else if (out_row && valid) {
                a.y[gi] = (v[0] + sBias[sb_off(3)]) * a.out_scale;
            }
        }
    }
    __syncthreads();
    if (warp == 0) tmem_free(tmem);
}

// ------------------------------------------------------------------- loss

// dz3[cell][0] = 2 mask (y - t) / count, other channels 0; loss += mask (y - t)^2 / count.
__global__ void k_loss(const float* __restrict__ y, const float* __restrict__ t, const unsigned char* __restrict__ m,
                       const int* __restrict__ nxv, int nb, int pitch, float inv_count, bf16* dz, double* loss)
{
    __shared__ double red[32];
    double acc[1] = {0.0};
    const size_t total = (size_t)nb * pitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(q / pitch), i = (int)(q - (size_t)b * pitch);
        float g = 0.0f;
        if (i < nxv[b] && m[q]) {
            const float r = y[q] - t[q];
            g = 2.0f * r * inv_count;
            acc[0] += (double)r * (double)r * (double)inv_count;
        }
        bf16* row = dz + q * kCh;
        row[0] = __float2bfloat16(g);
#pragma unroll
        for (int j = 1; j < 16; ++j) row[j] = __float2bfloat16(0.0f);
    }
    block_sum<1>(acc, red);
    if (threadIdx.x == 0) atomicAdd(loss, acc[0]);
}

// ------------------------------------------------------------------- dgrad

struct DgradArgs {
    const int* nxv;
    int nb, pitch, ntiles;    // 128-cell tiles per member
    const float* params;
    int layer;                // l >= 1: produces dz of layer l - 1
    const bf16* dz_in;        // [cells][32] gradient w.r.t. layer l's pre-activation
    const bf16* act;          // [cells][32] post-activation of layer l - 1
    bf16* dz_out;             // [cells][32]
    int* status;
    long long budget;
};

constexpr size_t kDgradSmem = sizeof(bf16) * (kRows * 96 + 32 * 96 + (kRows + 2) * kCh) + 16;

// dA[cell][c] = sum_k sum_o dz[cell - k + 1][o] W[o][k c_in + c]; dz_out = dA * (act > 0).
__global__ void __launch_bounds__(kRows) k_dgrad(DgradArgs a)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    bf16* sA = reinterpret_cast<bf16*>(smraw);           // 128 x 3 Co
    bf16* sB = sA + kRows * 96;                           // Ci x 3 Co
    bf16* sD = sB + 32 * 96;                              // 130 rows of dz_in
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sD + (kRows + 2) * kCh);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, l = a.layer;
    const int Ci = cin(l), Co = cout(l), K = 3 * Co, nkc = K / 8;
    // B[c][k Co + o] = W[o][k Ci + c]
    for (int e = tid; e < Ci * K; e += kRows) {
        const int c = e / K, kk = e - c * K, k = kk / Co, o = kk - k * Co;
        sB[core_off(c, kk, nkc)] = __float2bfloat16(a.params[woff(l) + o * 3 * Ci + k * Ci + c]);
    }
    if (warp == 0) tmem_alloc(tslot);
    if (tid == 0) mbar_init(mbar);
    fence_async_smem();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t parity = 0;
    const int total = a.nb * a.ntiles;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int b = w / a.ntiles, t = w - b * a.ntiles;
        const int nxb = member_cells(a.nxv, b);
        if (t * kRows >= nxb) continue;
        const int c0 = t * kRows;
        // rows c0-1 .. c0+128 of dz_in (zero outside the member)
        for (int r = tid; r < kRows + 2; r += kRows) {
            const int cell = c0 - 1 + r;
            uint4 v[4] = {make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0), make_uint4(0, 0, 0, 0)};
            if (cell >= 0 && cell < nxb) {
                const uint4* src = reinterpret_cast<const uint4*>(a.dz_in + ((size_t)b * a.pitch + cell) * kCh);
#pragma unroll
                for (int q = 0; q < 4; ++q) v[q] = src[q];
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) reinterpret_cast<uint4*>(sD + r * kCh)[q] = v[q];
        }
        __syncthreads();
        // A[row][k Co + o] = dz[cell + 1 - k][o]; local row of cell c0 + tid is tid + 1
        for (int k = 0; k < 3; ++k) {
            const int rr = tid + 2 - k;
            for (int q = 0; q < Co / 8; ++q)
                *reinterpret_cast<uint4*>(sA + core_off(tid, k * Co + q * 8, nkc)) =
                    reinterpret_cast<const uint4*>(sD + rr * kCh)[q];
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_after_sync();
            const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sB);
            for (int kk = 0; kk < K / 16; ++kk)
                mma(tmem, sdesc(aaddr + kk * 256, nkc * 128), sdesc(baddr + kk * 256, nkc * 128), idesc(Ci),
                    kk > 0 ? 1u : 0u);
            commit(mbar);
        }
        if (!block_wait(mbar, parity, a.budget, a.status)) break;
        parity ^= 1u;
        tc_after_sync();
        float v[32];
        tmem_ld32(trow, v);       // Ci = 32 for every layer with a dgrad
        tc_before_sync();
        const int cell = c0 + tid;
        if (cell < nxb) {
            const size_t gi = (size_t)b * a.pitch + cell;
            const bf16* act = a.act + gi * kCh;
            __align__(16) bf16 o[32];
#pragma unroll
            for (int j = 0; j < 32; ++j)
                o[j] = __float2bfloat16(__bfloat162float(act[j]) > 0.0f ? v[j] : 0.0f);
            uint4* dst = reinterpret_cast<uint4*>(a.dz_out + gi * kCh);
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[q] = reinterpret_cast<const uint4*>(o)[q];
        }
        __syncthreads();
    }
    __syncthreads();
    if (warp == 0) tmem_free(tmem);
}

// ------------------------------------------------------------------- wgrad

struct WgradArgs {
    const int* nxv;
    int nb, pitch, ntiles;      // 128-cell tiles per member
    int layer;
    const bf16* act_in;         // layer input: features ([cells][16]) or activations ([cells][32])
    int in_stride;              // 16 or 32
    const bf16* dz;             // [cells][32] gradient w.r.t. the layer's pre-activation
    float* grad;                // FP32 gradient vector (atomically accumulated)
    int* status;
    long long budget;
};

constexpr size_t kWgradSmem = sizeof(bf16) * (kRows * kRows + 32 * kRows) + 16;

// D[(k, c)][o] = sum_cells act_in[cell + k - 1][c] dz[cell][o], accumulated in
// tensor memory over this CTA's tiles, then added to dW[o][k c_in + c]; the
// bias gradient is the column sum of dz.
__global__ void __launch_bounds__(kRows) k_wgrad(WgradArgs a)
{
    extern __shared__ __align__(128) unsigned char smraw[];
    bf16* sA = reinterpret_cast<bf16*>(smraw);     // 128 rows (k, c) x 128 cells
    bf16* sB = sA + kRows * kRows;                  // Co rows x 128 cells
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sB + 32 * kRows);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    __shared__ float sbias[32];
    const int tid = threadIdx.x, warp = tid >> 5, l = a.layer;
    const int Ci = cin(l), Co = cout(l), Mv = 3 * Ci, nkc = kRows / 8;
    for (int e = tid; e < kRows * kRows; e += kRows) sA[e] = __float2bfloat16(0.0f);
    if (tid < 32) sbias[tid] = 0.0f;
    if (warp == 0) tmem_alloc(tslot);
    if (tid == 0) mbar_init(mbar);
    fence_async_smem();
    __syncthreads();
    tc_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
    uint32_t parity = 0;
    bool any = false, ok = true;
    float bacc[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) bacc[j] = 0.0f;
    const int total = a.nb * a.ntiles;
    for (int w = blockIdx.x; w < total; w += gridDim.x) {
        const int b = w / a.ntiles, t = w - b * a.ntiles;
        const int nxb = member_cells(a.nxv, b);
        if (t * kRows >= nxb) continue;
        const int cell = t * kRows + tid;
        const bool valid = cell < nxb;
        const size_t gi = (size_t)b * a.pitch + cell;
        // A[(k, c)][tid] = act_in[cell + k - 1][c] (zero outside the member)
        for (int k = 0; k < 3; ++k) {
            const int cc = cell + k - 1;
            const bool in = valid && cc >= 0 && cc < nxb;
            const bf16* src = a.act_in + ((size_t)b * a.pitch + cc) * a.in_stride;
            for (int c = 0; c < Ci; ++c)
                sA[core_off(k * Ci + c, tid, nkc)] = in ? src[c] : __float2bfloat16(0.0f);
        }
        for (int o = 0; o < Co; ++o) {
            const bf16 g = valid ? a.dz[gi * kCh + o] : __float2bfloat16(0.0f);
            sB[core_off(o, tid, nkc)] = g;
            bacc[o] += __bfloat162float(g);
        }
        fence_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_after_sync();
            const uint32_t aaddr = smem_u32(sA), baddr = smem_u32(sB);
            for (int kk = 0; kk < kRows / 16; ++kk)
                mma(tmem, sdesc(aaddr + kk * 256, nkc * 128), sdesc(baddr + kk * 256, nkc * 128), idesc(Co),
                    (any || kk > 0) ? 1u : 0u);
            commit(mbar);
        }
        any = true;
        if (!block_wait(mbar, parity, a.budget, a.status)) {
            ok = false;
            break;
        }
        parity ^= 1u;
        tc_after_sync();
        __syncthreads();     // operands may be overwritten for the next tile
    }
    for (int o = 0; o < Co; ++o) atomicAdd(&sbias[o], bacc[o]);
    __syncthreads();
    if (any && ok) {
        float v[32];
        tc_after_sync();
        if (Co == 32) tmem_ld32(trow, v); else tmem_ld16(trow, v);
        tc_before_sync();
        if (tid < Mv)
            for (int o = 0; o < Co; ++o) atomicAdd(&a.grad[woff(l) + o * 3 * Ci + tid], v[o]);
        if (tid < Co) atomicAdd(&a.grad[boff(l) + tid], sbias[tid]);
    }
    __syncthreads();
    if (warp == 0) tmem_free(tmem);
}

// -------------------------------------------------------------------- Adam

__global__ void k_adam(float* p, const float* __restrict__ g, float* m, float* v, int n, float lr, float b1,
                       float b2, float eps, float c1, float c2)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}


// ------------------------------------------------------- the learned guess
//
// With psi^n the pressure unknown (zero off the active cells) and h1, h2 the
// two solutions before it, a cell has a first difference d1 = psi^n - h1 when
// psi^n and h1 are both nonzero there (and h1 exists), and a second
// difference D2 = d1 - (h1 - h2) when h2 is nonzero too (and exists).  The
// guess is psi^n + d1 + D2 + S2 y: quadratic extrapolation in time plus the
// network's correction y in units of S2 = max |D2|.

__device__ __forceinline__ bool marked(const uint32_t* act, int wpitch, int b, int i)
{
    return (act[(size_t)b * wpitch + (i >> 5)] >> (i & 31)) & 1u;
}

struct Hist {
    double p, d1, d0, D2;
    bool v1, v2;
};

__device__ __forceinline__ Hist history(const GuessBufs& B, const GuessGeo& G, size_t q, int v1, int v2)
{
    Hist H;
    H.p = G.psi[q];
    const double a1 = v1 ? B.h1[q] : 0.0;
    const double a2 = v2 ? B.h2[q] : 0.0;
    H.v1 = H.p != 0.0 && a1 != 0.0;
    H.v2 = H.v1 && a2 != 0.0;
    H.d1 = H.v1 ? H.p - a1 : 0.0;
    H.d0 = H.v2 ? a1 - a2 : 0.0;
    H.D2 = H.v2 ? H.d1 - H.d0 : 0.0;
    return H;
}

// smax1_bits = max |d1|, smax2_bits = max |D2| over the member cells.
__global__ void k_guess_scale(GuessBufs B, GuessGeo G)
{
    __shared__ double red[32];
    if (G.tc && G.tc->abort) return;
    const int v1 = B.ctl->v1, v2 = B.ctl->v2;
    double m1 = 0.0, m2 = 0.0;
    const size_t total = (size_t)G.nb * G.pitch;
    if (v1) {
        for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
             q += (size_t)gridDim.x * blockDim.x) {
            const int b = (int)(q / G.pitch), i = (int)(q - (size_t)b * G.pitch);
            if (i >= G.nxv[b]) continue;
            const Hist H = history(B, G, q, v1, v2);
            m1 = fmax(m1, fabs(H.d1));
            m2 = fmax(m2, fabs(H.D2));
        }
    }
    m1 = -block_min(-m1, red);
    m2 = -block_min(-m2, red);
    if (threadIdx.x == 0) {
        if (m1 > 0.0) atomicMax(&B.ctl->smax1_bits, (unsigned long long)__double_as_longlong(m1));
        if (m2 > 0.0) atomicMax(&B.ctl->smax2_bits, (unsigned long long)__double_as_longlong(m2));
    }
}

// Features of the step being solved (channel list in nhswe_cnn.h).
__global__ void k_guess_features(GuessBufs B, GuessGeo G)
{
    if (G.tc && G.tc->abort) return;
    const int v1 = B.ctl->v1, v2 = B.ctl->v2;
    const double S1 = v1 ? __longlong_as_double((long long)B.ctl->smax1_bits) : 0.0;
    const double S2 = v2 ? __longlong_as_double((long long)B.ctl->smax2_bits) : 0.0;
    const double i1 = S1 > 0.0 ? 1.0 / S1 : 0.0, i2 = S2 > 0.0 ? 1.0 / S2 : 0.0;
    if (blockIdx.x == 0 && threadIdx.x == 0) { B.ctl->S1_used = S1; B.ctl->S2_used = S2; B.ctl->built = 1; }
    const size_t total = (size_t)G.nb * G.pitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(q / G.pitch), i = (int)(q - (size_t)b * G.pitch);
        __align__(16) bf16 f[16];
#pragma unroll
        for (int j = 0; j < 16; ++j) f[j] = __float2bfloat16(0.0f);
        if (i < G.nxv[b]) {
            const Hist H = history(B, G, q, v1, v2);
            f[0] = __float2bfloat16((float)(H.d1 * i1));
            f[1] = __float2bfloat16((float)(H.d0 * i1));
            f[2] = __float2bfloat16(marked(G.act, G.wpitch, b, i) ? 1.0f : 0.0f);
            f[3] = __float2bfloat16(H.p != 0.0 ? 1.0f : 0.0f);
            f[4] = __float2bfloat16((float)(H.D2 * i2));
            f[5] = __float2bfloat16(H.v2 ? 1.0f : 0.0f);
            B.d2[q] = H.D2;
        }
        uint4* dst = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(B.feat) + q * 16);
        dst[0] = reinterpret_cast<const uint4*>(f)[0];
        dst[1] = reinterpret_cast<const uint4*>(f)[1];
    }
}

// base = psi + d1 (+ D2 where D2 exists) on marked cells, psi elsewhere;
// guess = base + S2 y, or psi where S2 y is not finite.
__global__ void k_guess_apply(GuessBufs B, GuessGeo G)
{
    if (G.tc && G.tc->abort) return;
    const int v1 = B.ctl->v1, v2 = B.ctl->v2;
    const double S2 = B.ctl->S2_used;
    const size_t total = (size_t)G.nb * G.pitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(q / G.pitch), i = (int)(q - (size_t)b * G.pitch);
        const double p = G.psi[q];
        double xb = p, xg = p;
        if (v1 && i < G.nxv[b] && marked(G.act, G.wpitch, b, i)) {
            const Hist H = history(B, G, q, v1, v2);
            xb = p + H.d1 + H.D2;
            const double d = (H.v2 && S2 > 0.0) ? S2 * (double)B.y[q] : 0.0;
            xg = isfinite(d) ? xb + d : p;
        }
        B.base[q] = xb;
        B.guess[q] = xg;
    }
}

__global__ void k_guess_select(GuessBufs B, GuessGeo G)
{
    if (G.tc && G.tc->abort) return;
    const size_t total = (size_t)G.nb * G.pitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(q / G.pitch);
        const int c = B.choice[b];
        if (c == 0) B.guess[q] = G.psi[q];
        else if (c == 1) B.guess[q] = B.base[q];
    }
}

__global__ void k_guess_shift(GuessBufs B, GuessGeo G)
{
    if (G.tc && G.tc->abort) return;
    const size_t total = (size_t)G.nb * G.pitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        B.h2[q] = B.h1[q];
        B.h1[q] = G.psi[q];
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        B.ctl->v2 = B.ctl->v1;
        B.ctl->v1 = 1;
    }
}

// After the step (h1 = psi^n, h2 = psi^{n-1}, psi = psi^{n+1}, d2 = D2 of
// that step): the target (psi^{n+1} - psi^n - d1 - D2) / S2 on marked cells
// with a second difference.
__global__ void k_guess_harvest(GuessBufs B, GuessGeo G, float* target, unsigned char* mask)
{
    const double S2 = B.ctl->S2_used;
    const double inv = S2 > 0.0 ? 1.0 / S2 : 0.0;
    const size_t total = (size_t)G.nb * G.pitch;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int b = (int)(q / G.pitch), i = (int)(q - (size_t)b * G.pitch);
        const bool in = S2 > 0.0 && i < G.nxv[b] && marked(G.act, G.wpitch, b, i);
        const bool feat_v2 = in && __bfloat162float(reinterpret_cast<const bf16*>(B.feat)[q * 16 + 5]) != 0.0f;
        const double pn = B.h1[q], pm = B.h2[q], pnew = G.psi[q];
        const bool m = feat_v2 && pnew != 0.0;
        target[q] = m ? (float)((pnew - pn - (pn - pm) - B.d2[q]) * inv) : 0.0f;
        mask[q] = m ? 1 : 0;
    }
}

}  // namespace cnn
}  // namespace nh

using namespace nh;
using namespace nh::cnn;

namespace {

struct CnnWs {
    bf16* acts;      // [3][cells][32]
    bf16* dz0;       // [cells][32]
    bf16* dz1;       // [cells][32]
    float* y;        // [cells]
    double* loss;
    int* status;
};

size_t ws_layout(int nb, int pitch, char* base, CnnWs* w)
{
    const size_t cells = (size_t)nb * pitch;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        off = (off + 255) / 256 * 256;
        void* p = base ? base + off : nullptr;
        off += bytes;
        return p;
    };
    CnnWs t;
    CnnWs& W = w ? *w : t;
    W.acts = (bf16*)take(sizeof(bf16) * 3 * cells * kCh);
    W.dz0 = (bf16*)take(sizeof(bf16) * cells * kCh);
    W.dz1 = (bf16*)take(sizeof(bf16) * cells * kCh);
    W.y = (float*)take(sizeof(float) * cells);
    W.loss = (double*)take(sizeof(double));
    W.status = (int*)take(sizeof(int));
    return (off + 255) / 256 * 256;
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

long long clock_budget()
{
    int dev = 0, khz = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev);
    return (long long)(khz > 0 ? khz : 2000000) * 1000LL;   // about one second
}

// Opt the tensor-core kernels into their dynamic shared memory, once per device.
constexpr int kMaxDevices = 64;
std::mutex g_smem_mutex;
bool g_smem_done[kMaxDevices] = {};

cudaError_t set_smem()
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_smem_mutex);
    if (g_smem_done[dev]) return cudaSuccess;
    if ((e = cudaFuncSetAttribute(k_forward, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kFwdSmem)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_dgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kDgradSmem)) != cudaSuccess ||
        (e = cudaFuncSetAttribute(k_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kWgradSmem)) != cudaSuccess)
        return e;
    g_smem_done[dev] = true;
    return cudaSuccess;
}

cudaError_t forward_impl(const bf16* feat, const int* nxv, int nb, int pitch, const float* params, float* y,
                         float out_scale, bf16* acts, const uint32_t* act, int wpitch, int* status, cudaStream_t st)
{
    cudaError_t e = set_smem();
    if (e != cudaSuccess) return e;
    FwdArgs a;
    a.feat = feat; a.nxv = nxv; a.nb = nb; a.pitch = pitch; a.ntiles = (pitch + kTileOut - 1) / kTileOut;
    a.params = params; a.y = y; a.out_scale = out_scale; a.acts = acts; a.act = act; a.wpitch = wpitch;
    a.status = status; a.budget = clock_budget();
    const int total = nb * a.ntiles;
    const int grid = std::min(total, sm_count() * 4);
    k_forward<<<grid, kRows, kFwdSmem, st>>>(a);
    return cudaGetLastError();
}

int elem_grid(const GuessGeo& G)
{
    const size_t total = (size_t)G.nb * G.pitch;
    return (int)std::min<size_t>((total + 255) / 256, (size_t)std::max(G.sms, 1) * 8);
}

}  // namespace

namespace nh {
namespace cnn {

cudaError_t prepare_device() { return set_smem(); }

cudaError_t launch_features(const GuessBufs& B, const GuessGeo& G, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(&B.ctl->smax1_bits, 0, 2 * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    k_guess_scale<<<elem_grid(G), 256, 0, st>>>(B, G);
    k_guess_features<<<elem_grid(G), 256, 0, st>>>(B, G);
    return cudaGetLastError();
}

cudaError_t launch_guess(const GuessBufs& B, const GuessGeo& G, cudaStream_t st)
{
    cudaError_t e = forward_impl((const bf16*)B.feat, G.nxv, G.nb, G.pitch, B.params, B.y, 1.0f, nullptr, G.act,
                                 G.wpitch, &B.ctl->status, st);
    if (e != cudaSuccess) return e;
    k_guess_apply<<<elem_grid(G), 256, 0, st>>>(B, G);
    return cudaGetLastError();
}

cudaError_t launch_select(const GuessBufs& B, const GuessGeo& G, cudaStream_t st)
{
    k_guess_select<<<elem_grid(G), 256, 0, st>>>(B, G);
    return cudaGetLastError();
}

cudaError_t launch_shift(const GuessBufs& B, const GuessGeo& G, cudaStream_t st)
{
    k_guess_shift<<<elem_grid(G), 256, 0, st>>>(B, G);
    return cudaGetLastError();
}

cudaError_t launch_harvest(const GuessBufs& B, const GuessGeo& G, float* target, unsigned char* mask,
                           cudaStream_t st)
{
    k_guess_harvest<<<elem_grid(G), 256, 0, st>>>(B, G, target, mask);
    return cudaGetLastError();
}

}  // namespace cnn
}  // namespace nh

extern "C" {

size_t nh_cnn_workspace_bytes(int nbatch, int pitch)
{
    if (nbatch < 1 || pitch < 1) return 0;
    return ws_layout(nbatch, pitch, nullptr, nullptr);
}

nh_status nh_cnn_forward(const void* feat, const int* nx_dev, int nbatch, int pitch, const float* params,
                         float* y, float out_scale, int* status_dev, void* stream)
{
    if (!feat || !nx_dev || !params || !y || nbatch < 1 || pitch < 8 || (pitch % 8) != 0) return NH_ERR_ARG;
    if (((uintptr_t)feat % 16) != 0) return NH_ERR_ARG;
    return forward_impl((const bf16*)feat, nx_dev, nbatch, pitch, params, y, out_scale, nullptr, nullptr, 0,
                        status_dev, (cudaStream_t)stream) == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

nh_status nh_cnn_loss_grad(const void* feat, const int* nx_dev, int nbatch, int pitch, const float* params,
                           const float* target, const unsigned char* mask, long long mask_count, float* grad,
                           double* loss, void* ws, size_t ws_bytes, void* stream)
{
    if (!feat || !nx_dev || !params || !target || !mask || !grad || !ws || nbatch < 1 || pitch < 8 ||
        (pitch % 8) != 0 || ((uintptr_t)feat % 16) != 0 || mask_count < 0)
        return NH_ERR_ARG;
    if (ws_bytes < ws_layout(nbatch, pitch, nullptr, nullptr) || ((uintptr_t)ws % 256) != 0) return NH_ERR_ARG;
    cudaStream_t st = (cudaStream_t)stream;
    CnnWs W;
    ws_layout(nbatch, pitch, (char*)ws, &W);
    if (cudaMemsetAsync(W.loss, 0, sizeof(double), st) != cudaSuccess ||
        cudaMemsetAsync(W.status, 0, sizeof(int), st) != cudaSuccess ||
        cudaMemsetAsync(grad, 0, sizeof(float) * kNParams, st) != cudaSuccess)
        return NH_ERR_CUDA;
    if (forward_impl((const bf16*)feat, nx_dev, nbatch, pitch, params, W.y, 1.0f, W.acts, nullptr, 0, W.status,
                     st) != cudaSuccess)
        return NH_ERR_CUDA;
    const size_t cells = (size_t)nbatch * pitch;
    const int sms = sm_count();
    const float inv = 1.0f / (float)std::max<long long>(1, mask_count);
    cnn::k_loss<<<(int)std::min<size_t>((cells + 255) / 256, (size_t)sms * 8), 256, 0, st>>>(
        W.y, target, mask, nx_dev, nbatch, pitch, inv, W.dz0, W.loss);
    const int nt = (pitch + kRows - 1) / kRows;
    const int grid = std::min(nbatch * nt, sms * 4);
    bf16* dz_cur = W.dz0;
    bf16* dz_nxt = W.dz1;
    for (int l = 3; l >= 0; --l) {
        WgradArgs wa;
        wa.nxv = nx_dev; wa.nb = nbatch; wa.pitch = pitch; wa.ntiles = nt; wa.layer = l;
        wa.act_in = l == 0 ? (const bf16*)feat : W.acts + (size_t)(l - 1) * cells * kCh;
        wa.in_stride = l == 0 ? 16 : kCh;
        wa.dz = dz_cur; wa.grad = grad; wa.status = W.status; wa.budget = clock_budget();
        cnn::k_wgrad<<<grid, kRows, kWgradSmem, st>>>(wa);
        if (l > 0) {
            DgradArgs da;
            da.nxv = nx_dev; da.nb = nbatch; da.pitch = pitch; da.ntiles = nt; da.params = params; da.layer = l;
            da.dz_in = dz_cur; da.act = W.acts + (size_t)(l - 1) * cells * kCh; da.dz_out = dz_nxt;
            da.status = W.status; da.budget = clock_budget();
            cnn::k_dgrad<<<grid, kRows, kDgradSmem, st>>>(da);
            std::swap(dz_cur, dz_nxt);
        }
    }
    if (cudaGetLastError() != cudaSuccess) return NH_ERR_CUDA;
    int status = 0;
    double L = 0.0;
    if (cudaMemcpyAsync(&status, W.status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&L, W.loss, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return NH_ERR_CUDA;
    if (loss) *loss = L;
    return status ? NH_ERR_TIMEOUT : NH_OK;
}

nh_status nh_cnn_adam(float* params, const float* grad, float* m, float* v, int step, float lr, void* stream)
{
    if (!params || !grad || !m || !v || step < 1 || !(lr > 0.0f)) return NH_ERR_ARG;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - powf(b1, (float)step), c2 = 1.0f - powf(b2, (float)step);
    cnn::k_adam<<<(kNParams + 255) / 256, 256, 0, (cudaStream_t)stream>>>(params, grad, m, v, kNParams, lr, b1, b2,
                                                                         1e-8f, c1, c2);
    return cudaGetLastError() == cudaSuccess ? NH_OK : NH_ERR_CUDA;
}

}  // extern "C"
