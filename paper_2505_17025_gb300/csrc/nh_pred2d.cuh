// nh_pred2d.cuh -- both Heun stages of the 2D hydrostatic predictor in one
// launch, for the FP32 state (a2 on 2D grids; Sec. 3.1, Eqs. 8-9).
//
// The two-launch form (k2_stage) writes the stage-1 state and rates to
// global memory and reads them back; here a CTA keeps them on chip.  For an
// output tile of kPX x kPY cells it loads Q^n on the tile plus a four-cell
// halo (two MUSCL stencils deep), computes stage 1 on the tile plus a
// two-cell halo, and stage 2 on the tile, so each step reads Q^n (and the
// static depth) once and writes Q~ once.  The mound of the moving bottom is
// evaluated in registers at t^n and t^{n+1} (the t^{n+1} values of the tile
// are stored, for the criterion and the assembly), and the |eta/d| criterion
// is evaluated on the tile's new state in the epilogue.
//
// The arithmetic per face and per cell is k2_stage's (face_flux, the
// well-balanced momentum update); the stage-1 state of halo cells outside a
// walled side is the mirror image of the interior stage-1 state, as the
// two-launch form reads it, and periodic sides compute the wrapped cells'
// stage 1 from wrapped inputs.
#pragma once

#include "nh_kernels2d.cuh"

namespace nh {

// Tile geometry of the one-launch predictor: TX x TY output cells (one
// thread each), the Q^n region (halo 4), the stage-1 region (halo 2), and the
// face counts of both stages.  The tile is chosen per handle by timing the
// candidates (kPredTiles) on the live state.
template <int TX, int TY>
struct PTile {
    static constexpr int X = TX, Y = TY, threads = TX * TY;
    static constexpr int AX = TX + 8, AY = TY + 8, BX = TX + 4, BY = TY + 4;
    static constexpr int A = AX * AY, B = BX * BY;
    static constexpr int F1X = (BX + 1) * BY, F1Y = BX * (BY + 1);
    static constexpr int F2X = (TX + 1) * TY, F2Y = TX * (TY + 1);
    static constexpr int F = F1X + F1Y;
    static constexpr size_t smem = sizeof(float) * (9 * A + 5 * B + 5 * F + 4 * threads);
};

struct FusedArgs {
    const Geo2* geos;
    const Slide2* slides;
    const Kin2* kin;          // kin[2b], kin[2b + 1]: slide at t^n and t^{n+1}
    size_t pitch;
    const float *z, *hu, *hv, *hw;   // Q^n (zeta = h - d0, hu, hv, hw)
    const float* d0s;                // FP32 static depth
    float *oz, *ohu, *ohv, *ohw;     // Q~
    float* m1;                       // mound at t^{n+1} (tile cells)
    unsigned char* marks;            // |eta/d| > knh at t^{n+1}, or null (criterion evaluated elsewhere)
    float knh;
    double dt;
    const TimeCtl* tc;
    int vec4;                        // Q^n and d0s 16-byte aligned with a pitch of 4k floats: float4 loads
};

// Per-CTA FP32 mound evaluator at one time: the slide centre as an integer
// cell offset plus an FP32 fraction (computed in FP64), as k2_depth does.
struct MoundF {
    int ic, jc;
    float fx, fy, sx, sy, A;
    bool on;
    __device__ __forceinline__ float at(int i, int j) const
    {
        if (!on) return 0.0f;
        const float xi = ((float)(i - ic) - fx) * sx;
        if (xi * xi > (float)kMoundCut) return 0.0f;   // r2 >= xi^2: beyond the cut-off
        const float ze = ((float)(j - jc) - fy) * sy;
        const float r2 = xi * xi + ze * ze;
        return r2 <= (float)kMoundCut ? A * expf(-r2) : 0.0f;
    }
};

__device__ __forceinline__ MoundF mound_f(const Geo2& G, const Slide2& S, double s)
{
    MoundF M;
    M.on = S.shape == NH_SLIDE_GAUSS_LNCOSH;
    const double cx = (S.xc0 + s - G.x0) * G.idx - 0.5, cy = (S.yc0 - G.y0) * G.idy - 0.5;
    const double fx = floor(cx), fy = floor(cy);
    M.ic = (int)fmax(fmin(fx, 1e9), -1e9); M.jc = (int)fmax(fmin(fy, 1e9), -1e9);
    M.fx = (float)(cx - fx); M.fy = (float)(cy - fy);
    M.sx = (float)(G.dx * S.iLx); M.sy = (float)(G.dy * S.iLy); M.A = (float)S.A;
    return M;
}

// Rates of the cell at (lx, ly) of a primitive region (row width W) from its
// four faces (fx: x-faces, row width FXW; fy: y-faces, row width FYW; cell
// (cx, cy) of the face arrays).  The well-balanced normal-momentum update of
// k2_stage.
__device__ __forceinline__ void cell_rates(const float* e, const float* d, int W, int lx, int ly, const float* fxb,
                                           int nfx, int FXW, const float* fyb, int nfy, int FYW, int cx, int cy,
                                           float g, float idx, float idy, int lim, float r[4])
{
    const float h2 = 0.5f;
    const int c = ly * W + lx;
    const float ec = e[c], dc = d[c];
    const float sex = slope2(lim, e[c - 1], ec, e[c + 1]);
    const float hbx = ec + h2 * (h2 * (d[c - 1] + dc) + h2 * (dc + d[c + 1]));
    const float sey = slope2(lim, e[c - W], ec, e[c + W]);
    const float hby = ec + h2 * (h2 * (d[c - W] + dc) + h2 * (dc + d[c + W]));
    auto FX = [&](int k, int x) { return fxb[k * nfx + cy * FXW + x]; };
    auto FY = [&](int k, int y) { return fyb[k * nfy + y * FYW + cx]; };
    r[0] = -(FX(0, cx + 1) - FX(0, cx)) * idx - (FY(0, cy + 1) - FY(0, cy)) * idy;
    r[1] = -((FX(1, cx + 1) - FX(1, cx)) + (FX(2, cx + 1) + FX(2, cx)) + g * hbx * sex) * idx
           - (FY(3, cy + 1) - FY(3, cy)) * idy;
    r[2] = -(FX(3, cx + 1) - FX(3, cx)) * idx
           - ((FY(1, cy + 1) - FY(1, cy)) + (FY(2, cy + 1) + FY(2, cy)) + g * hby * sey) * idy;
    r[3] = -(FX(4, cx + 1) - FX(4, cx)) * idx - (FY(4, cy + 1) - FY(4, cy)) * idy;
}

// x-faces (nfx = (RW + 1) * RH) and y-faces (RW * (RH + 1)) of an RW x RH
// region whose cell (0, 0) sits at (ox, oy) of a primitive region of row width W.
__device__ __forceinline__ void region_faces(const float* e, const float* u, const float* v, const float* w,
                                             const float* d, int W, int ox, int oy, int RW, int RH, float* fxb,
                                             float* fyb, float g, int lim)
{
    const int nfx = (RW + 1) * RH, nfy = RW * (RH + 1);
    for (int q = threadIdx.x; q < nfx + nfy; q += blockDim.x) {
        float F[5];
        if (q < nfx) {
            const int fx = q % (RW + 1), r = q / (RW + 1);
            const int c = (oy + r) * W + ox + fx;
            face_flux<float>(g, lim, e + c, u + c, v + c, w + c, d + c, 1, F);
#pragma unroll
            for (int k = 0; k < 5; ++k) fxb[k * nfx + q] = F[k];
        } else {
            const int q2 = q - nfx, col = q2 % RW, fy = q2 / RW;
            const int c = (oy + fy) * W + ox + col;
            face_flux<float>(g, lim, e + c, v + c, u + c, w + c, d + c, W, F);
#pragma unroll
            for (int k = 0; k < 5; ++k) fyb[k * nfy + q2] = F[k];
        }
    }
}

template <int TX, int TY>
static __global__ void __launch_bounds__(TX * TY, TX * TY <= 256 ? 4 : (TX * TY <= 512 ? 2 : 1))
    k2_heun_fused(FusedArgs a)
{
    using PT = PTile<TX, TY>;
    constexpr int kPX = PT::X, kPY = PT::Y, kPThreads = PT::threads;
    constexpr int kPAX = PT::AX, kPBX = PT::BX, kPBY = PT::BY;
    constexpr int kPA = PT::A, kPB = PT::B;
    constexpr int kPF1X = PT::F1X, kPF1Y = PT::F1Y, kPF2X = PT::F2X, kPF2Y = PT::F2Y, kPF = PT::F;
    if (a.tc && a.tc->abort) return;
    extern __shared__ __align__(16) float pred2_sm[];
    // Q^n region: conserved (z, hu, hv, hw) and primitives (e, u, v, w, d)
    float* Az = pred2_sm;
    float* Ahu = Az + kPA;
    float* Ahv = Ahu + kPA;
    float* Ahw = Ahv + kPA;
    float* Ae = Ahw + kPA;
    float* Au = Ae + kPA;
    float* Av = Au + kPA;
    float* Aw = Av + kPA;
    float* Ad = Aw + kPA;
    // stage-1 region: primitives of Q* and the depth at t^{n+1}
    float* Be = Ad + kPA;
    float* Bu = Be + kPB;
    float* Bv = Bu + kPB;
    float* Bw = Bv + kPB;
    float* Bd = Bw + kPB;
    // faces (stage 1, then stage 2) and the tile's stage-1 rates
    float* Fb = Bd + kPB;
    float* K1 = Fb + 5 * kPF;
    const int b = blockIdx.y;
    const size_t mo = (size_t)b * a.pitch;
    const Geo2 G = a.geos[b];
    const Slide2 S = a.slides[b];
    __shared__ MoundF s_m[2];
    __shared__ float s_k[5];
    if (threadIdx.x == 0) {
        s_m[0] = mound_f(G, S, a.kin[2 * b].s);
        s_m[1] = mound_f(G, S, a.kin[2 * b + 1].s);
        s_k[0] = (float)G.g; s_k[1] = (float)G.idx; s_k[2] = (float)G.idy; s_k[3] = (float)a.dt;
        s_k[4] = (float)(0.5 * a.dt);
    }
    __syncthreads();
    const MoundF M0 = s_m[0], M1 = s_m[1];
    const float g = s_k[0], idx = s_k[1], idy = s_k[2], dt = s_k[3], hdt = s_k[4];
    const int tiles_x = (G.nx + kPX - 1) / kPX, tiles = tiles_x * ((G.ny + kPY - 1) / kPY);
    const float* z = a.z + mo; const float* hu = a.hu + mo; const float* hv = a.hv + mo; const float* hw = a.hw + mo;
    const float* d0s = a.d0s + mo;
    const bool vec4 = a.vec4 && (G.nx & 3) == 0;
    for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
        const int i0 = (tile % tiles_x) * kPX, j0 = (tile / tiles_x) * kPY;
        // 1. Q^n and its primitives on the region (mirrored / wrapped)
        auto put = [&](int q, float zc, float huc, float hvc, float hwc, float dz, float m) {
            const float hc = zc + dz;
            const float rh = 1.0f / hc;
            Az[q] = zc; Ahu[q] = huc; Ahv[q] = hvc; Ahw[q] = hwc;
            Ae[q] = zc + m;
            Ad[q] = dz - m;
            Au[q] = huc * rh;
            Av[q] = hvc * rh;
            Aw[q] = hwc * rh;
        };
        auto put_cell = [&](int q, int ax, int ay) {
            int ox, oy;
            const int ci = g2_index1(G.bcx, G.nx, i0 - 4 + ax, &ox);
            const int cj = g2_index1(G.bcy, G.ny, j0 - 4 + ay, &oy);
            const int c = cj * G.nx + ci;
            put(q, z[c], flip(ox, hu[c]), flip(oy, hv[c]), hw[c], d0s[c], M0.at(ci, cj));
        };
        if (vec4) {
            // four cells of a row per thread: one float4 per field where the four
            // lie inside the domain (i0 - 4 + ax is a multiple of 4, so the address
            // is 16-byte aligned), the per-cell mirrored path elsewhere
            static_assert(kPAX % 4 == 0, "region rows split into groups of four cells");
            constexpr int kQ4 = kPAX / 4;
            for (int q4 = threadIdx.x; q4 < kPA / 4; q4 += kPThreads) {
                const int ax = (q4 % kQ4) * 4, ay = q4 / kQ4, q = ay * kPAX + ax;
                const int gi = i0 - 4 + ax, gj = j0 - 4 + ay;
                if (gi >= 0 && gi + 3 < G.nx && gj >= 0 && gj < G.ny) {
                    const int c = gj * G.nx + gi;
                    const float4 z4 = *reinterpret_cast<const float4*>(z + c);
                    const float4 u4 = *reinterpret_cast<const float4*>(hu + c);
                    const float4 v4 = *reinterpret_cast<const float4*>(hv + c);
                    const float4 w4 = *reinterpret_cast<const float4*>(hw + c);
                    const float4 d4 = *reinterpret_cast<const float4*>(d0s + c);
                    put(q, z4.x, u4.x, v4.x, w4.x, d4.x, M0.at(gi, gj));
                    put(q + 1, z4.y, u4.y, v4.y, w4.y, d4.y, M0.at(gi + 1, gj));
                    put(q + 2, z4.z, u4.z, v4.z, w4.z, d4.z, M0.at(gi + 2, gj));
                    put(q + 3, z4.w, u4.w, v4.w, w4.w, d4.w, M0.at(gi + 3, gj));
                } else {
#pragma unroll
                    for (int e = 0; e < 4; ++e) put_cell(q + e, ax + e, ay);
                }
            }
        } else {
            for (int q = threadIdx.x; q < kPA; q += kPThreads) put_cell(q, q % kPAX, q / kPAX);
        }
        __syncthreads();
        // 2. stage-1 faces of the stage-1 region (its cell (0, 0) at A (2, 2))
        region_faces(Ae, Au, Av, Aw, Ad, kPAX, 2, 2, kPBX, kPBY, Fb, Fb + 5 * kPF1X, g, G.lim);
        __syncthreads();
        // 3. stage 1: Q* = Q^n + dt k1 on the stage-1 region, its primitives at t^{n+1}
        for (int q = threadIdx.x; q < kPB; q += kPThreads) {
            const int bx = q % kPBX, by = q / kPBX;
            float r[4];
            cell_rates(Ae, Ad, kPAX, bx + 2, by + 2, Fb, kPF1X, kPBX + 1, Fb + 5 * kPF1X, kPF1Y, kPBX, bx, by, g,
                       idx, idy, G.lim, r);
            const int ca = (by + 2) * kPAX + bx + 2;
            const float zs = Az[ca] + dt * r[0];
            const float hus = Ahu[ca] + dt * r[1];
            const float hvs = Ahv[ca] + dt * r[2];
            const float hws = Ahw[ca] + dt * r[3];
            int ox, oy;
            const int ci = g2_index1(G.bcx, G.nx, i0 - 2 + bx, &ox);
            const int cj = g2_index1(G.bcy, G.ny, j0 - 2 + by, &oy);
            const int c = cj * G.nx + ci;
            const float m = M1.at(ci, cj), dz = d0s[c];
            const float rh = 1.0f / (zs + dz);
            Be[q] = zs + m;
            Bd[q] = dz - m;
            Bu[q] = hus * rh;
            Bv[q] = hvs * rh;
            Bw[q] = hws * rh;
            if (bx >= 2 && bx < kPX + 2 && by >= 2 && by < kPY + 2) {
                const int t = (by - 2) * kPX + (bx - 2);
                K1[t] = r[0]; K1[kPThreads + t] = r[1]; K1[2 * kPThreads + t] = r[2]; K1[3 * kPThreads + t] = r[3];
            }
        }
        __syncthreads();
        // 3b. halo cells beyond a walled side take the mirror of the interior
        //     stage-1 state (the two cells next to the side: no in-domain
        //     stencil reaches further)
        if (G.bcx != NH_BC_PERIODIC || G.bcy != NH_BC_PERIODIC) {
            for (int q = threadIdx.x; q < kPB; q += kPThreads) {
                const int bx = q % kPBX, by = q / kPBX;
                const int i = i0 - 2 + bx, j = j0 - 2 + by;
                const bool outx = (i < 0 || i >= G.nx) && G.bcx != NH_BC_PERIODIC;
                const bool outy = (j < 0 || j >= G.ny) && G.bcy != NH_BC_PERIODIC;
                if (!outx && !outy) continue;
                if (outx && (i < -2 || i > G.nx + 1)) continue;
                if (outy && (j < -2 || j > G.ny + 1)) continue;
                const int mi = outx ? (i < 0 ? -1 - i : 2 * G.nx - 1 - i) : i;
                const int mj = outy ? (j < 0 ? -1 - j : 2 * G.ny - 1 - j) : j;
                const int mq = (mj - (j0 - 2)) * kPBX + (mi - (i0 - 2));
                // the mirror cell lies in the region: the side is within two cells of the tile
                Be[q] = Be[mq]; Bd[q] = Bd[mq]; Bw[q] = Bw[mq];
                Bu[q] = outx ? -Bu[mq] : Bu[mq];
                Bv[q] = outy ? -Bv[mq] : Bv[mq];
            }
            __syncthreads();
        }
        // 4. stage-2 faces of the tile (its cell (0, 0) at B (2, 2))
        region_faces(Be, Bu, Bv, Bw, Bd, kPBX, 2, 2, kPX, kPY, Fb, Fb + 5 * kPF2X, g, G.lim);
        __syncthreads();
        // 5. stage 2: Q~ = Q^n + dt/2 (k1 + k2); mound at t^{n+1}; |eta/d| criterion
        {
            const int tx = threadIdx.x % kPX, ty = threadIdx.x / kPX;
            const int i = i0 + tx, j = j0 + ty;
            if (i < G.nx && j < G.ny) {
                float r[4];
                cell_rates(Be, Bd, kPBX, tx + 2, ty + 2, Fb, kPF2X, kPX + 1, Fb + 5 * kPF2X, kPF2Y, kPX, tx, ty, g,
                           idx, idy, G.lim, r);
                const int ca = (ty + 4) * kPAX + tx + 4;
                const int t = threadIdx.x;
                const size_t c = mo + (size_t)j * G.nx + i;
                const float zt = Az[ca] + hdt * (K1[t] + r[0]);
                a.oz[c] = zt;
                a.ohu[c] = Ahu[ca] + hdt * (K1[kPThreads + t] + r[1]);
                a.ohv[c] = Ahv[ca] + hdt * (K1[2 * kPThreads + t] + r[2]);
                a.ohw[c] = Ahw[ca] + hdt * (K1[3 * kPThreads + t] + r[3]);
                const float m = M1.at(i, j);
                a.m1[c] = m;
                if (a.marks) {
                    const float eta = zt + m, d = d0s[(size_t)j * G.nx + i] - m;
                    a.marks[c] = fabsf(eta / d) > a.knh ? 1 : 0;
                }
            }
        }
        __syncthreads();
    }
}

// Tile candidates (x, y) of the autotuner.
constexpr int kPredTiles[4][2] = {{32, 16}, {64, 8}, {32, 8}, {64, 16}};

}  // namespace nh
