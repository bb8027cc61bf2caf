// nh_static.cu -- one hydrostatic predictor step on caller-provided device
// buffers, with every scratch buffer in a fixed device array owned by this
// file, so the call allocates nothing.
//
// Who needs it: code that must not allocate device memory once it is running
// -- a host framework that plans all device memory up front, a real-time loop
// that may not block in the allocator, or a caller that cannot size and keep a
// workspace -- can still run the predictor on buffers it already has.
//
// The scratch (the input thickness deviation, per-tile partial sums, the
// criterion bit words and the slide kinematics) lives in `nh_static_scratch`
// below: a file-scope device array of kStaticBytes (about 2.2 MB) that every
// GPU which loads this library keeps until the process exits.  Host code
// cannot pass the array's name to a kernel (in host code it is only a
// stand-in, not a device address), so the first call on each device looks up
// its device address with cudaGetSymbolAddress, with that device current, and
// caches it.  Make that first call outside any stream capture.
//
// All calls share the one array: calls that overlap on the GPU (on different
// streams, or from different threads) race on it.  The array keeps the last
// call's contents; nothing in it has to start at zero (every word a call
// reads, it first writes).
#include <cmath>
#include <cstdint>
#include <mutex>

#include "nh_kernels1d.cuh"

using namespace nh;

namespace {

constexpr int kStaticMaxCells = NH_STATIC_MAX_CELLS;
constexpr int kStaticTiles = kStaticMaxCells / kPredTile;
constexpr int kStaticWords = kStaticMaxCells / 32;

// byte offsets of the scratch regions (each 256-byte aligned)
constexpr size_t kOffZ = 0;
constexpr size_t kOffMass = kOffZ + sizeof(double) * kStaticMaxCells;
constexpr size_t kOffMarks = kOffMass + sizeof(double) * kStaticTiles;
constexpr size_t kOffSlide = kOffMarks + sizeof(uint32_t) * kStaticWords;
constexpr size_t kOffKin = kOffSlide + 256;
constexpr size_t kOffSum = kOffKin + 256;
constexpr size_t kStaticBytes = kOffSum + 256;

static __device__ __align__(256) unsigned char nh_static_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch[kMaxDevices] = {};

// Device address of the scratch array on the current device (looked up once).
nh_status scratch_base(unsigned char** out)
{
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return NH_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_scratch[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, nh_static_scratch) != cudaSuccess || !p) return NH_ERR_CUDA;
        g_scratch[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch[dev]);
    return NH_OK;
}

__global__ void k_static_prepare(Slide s, Slide* dst, const double* __restrict__ h,
                                 const double* __restrict__ d0, double* __restrict__ z, int nx)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) *dst = s;
    if (i < nx) z[i] = h[i] - d0[i];
}

// h_out = zeta~ + d0 in place, and the FP64 sum of h_out (one CTA).
__global__ void __launch_bounds__(1024) k_static_finish(double* h_out, const double* __restrict__ d0,
                                                        int nx, double* sum)
{
    __shared__ double red[32];
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < nx; i += blockDim.x) {
        const double hh = h_out[i] + d0[i];
        h_out[i] = hh;
        v[0] += hh;
    }
    block_sum<1>(v, red);
    if (threadIdx.x == 0) *sum = v[0];
}

}  // namespace

extern "C" nh_status nh_predict_static(const double* h, const double* hu, const double* hw,
                                       const double* d0, double* h_out, double* hu_out, double* hw_out,
                                       int nx, double dx, double x0, int bc, int limiter, double g,
                                       const nh_slide_desc* slide, double t, double dt, double* mass,
                                       void* stream)
{
    if (!h || !hu || !hw || !d0 || !h_out || !hu_out || !hw_out) return NH_ERR_ARG;
    if (nx < 8 || nx > kStaticMaxCells) return NH_ERR_ARG;
    if (h_out == h || hu_out == hu || hw_out == hw) return NH_ERR_ARG;
    if (!(dx > 0.0) || !(g > 0.0) || !(dt > 0.0) || !std::isfinite(t) || !std::isfinite(x0)) return NH_ERR_ARG;
    if (bc != NH_BC_WALL && bc != NH_BC_PERIODIC) return NH_ERR_ARG;
    if (limiter < NH_LIM_NONE || limiter > NH_LIM_MC) return NH_ERR_ARG;
    Slide s{0.0, 1.0, 0.0, 0.0, 1.0, 1.0, 0.0, NH_SLIDE_NONE, 0};
    if (slide && slide->shape >= NH_SLIDE_GAUSS_LNCOSH && slide->shape <= NH_SLIDE_QUARTIC) {
        if (!(slide->L > 0.0) || !(slide->t0 > 0.0) || !std::isfinite(slide->L) || !std::isfinite(slide->t0))
            return NH_ERR_ARG;
        if (!std::isfinite(slide->A) || !std::isfinite(slide->xc0) || !std::isfinite(slide->s0)) return NH_ERR_ARG;
        if (slide->shape == NH_SLIDE_QUARTIC && !(slide->t2 >= slide->t0 && std::isfinite(slide->t2)))
            return NH_ERR_ARG;
        s.A = slide->A; s.L = slide->L; s.iL = 1.0 / slide->L; s.xc0 = slide->xc0; s.s0 = slide->s0; s.t0 = slide->t0;
        s.t2 = slide->shape == NH_SLIDE_QUARTIC ? slide->t2 : 0.0;
        s.shape = slide->shape;
    } else if (slide && slide->shape != NH_SLIDE_NONE) {
        return NH_ERR_ARG;
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    // reading the mass synchronises the stream, which a stream capture forbids
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) != cudaSuccess) return NH_ERR_CUDA;
    if (mass && cap != cudaStreamCaptureStatusNone) return NH_ERR_ARG;
    // an error left pending by earlier CUDA work is not this call's: refuse
    // to launch rather than report (and clear) it as ours
    if (cudaPeekAtLastError() != cudaSuccess) return NH_ERR_CUDA;
    unsigned char* base = nullptr;
    nh_status rc = scratch_base(&base);
    if (rc != NH_OK) return rc;
    double* z = reinterpret_cast<double*>(base + kOffZ);
    double* mass_part = reinterpret_cast<double*>(base + kOffMass);
    uint32_t* marks = reinterpret_cast<uint32_t*>(base + kOffMarks);
    Slide* slide_dev = reinterpret_cast<Slide*>(base + kOffSlide);
    Kin* kin_dev = reinterpret_cast<Kin*>(base + kOffKin);
    double* sum_dev = reinterpret_cast<double*>(base + kOffSum);

    k_static_prepare<<<(nx + 255) / 256, 256, 0, st>>>(s, slide_dev, h, d0, z, nx);
    k_kinematics<<<1, 32, 0, st>>>(slide_dev, kin_dev, 1, t, t + dt);
    PredArgs<double> pa;
    const int ntiles = (nx + kPredTile - 1) / kPredTile;
    pa.G.nx = nx; pa.G.nb = 1; pa.G.pitch = ntiles * kPredTile; pa.G.wpitch = ntiles * kPredTile / 32;
    pa.G.bc = bc; pa.G.lim = limiter; pa.G.ntiles = ntiles; pa.G.maxch = 1;
    pa.G.dx = dx; pa.G.x0 = x0; pa.G.g = g; pa.G.idx = 1.0 / dx;
    pa.G.i2dx = 1.0 / (2.0 * dx); pa.G.idx2 = 1.0 / (dx * dx);
    pa.z = z; pa.hu = hu; pa.hw = hw;
    pa.zt = h_out; pa.hut = hu_out; pa.hwt = hw_out;
    pa.d0 = d0; pa.slide = slide_dev; pa.kin = kin_dev;
    pa.marks = marks; pa.mass_part = mass_part;
    pa.dt = dt; pa.knh = 0.0; pa.crit = NH_CRIT_HYDROSTATIC; pa.all_global = 0;
    pa.tc = nullptr;
    pa.G.nxv = nullptr;
    k_predict<double, kPredTile><<<dim3(ntiles, 1), kPredTile, predict_smem_bytes<double, kPredTile>(), st>>>(pa);
    k_static_finish<<<1, 1024, 0, st>>>(h_out, d0, nx, sum_dev);
    if (cudaGetLastError() != cudaSuccess) return NH_ERR_CUDA;
    if (mass) {
        double sum = 0.0;
        if (cudaMemcpyAsync(&sum, sum_dev, sizeof(double), cudaMemcpyDeviceToHost, st) != cudaSuccess)
            return NH_ERR_CUDA;
        if (cudaStreamSynchronize(st) != cudaSuccess) return NH_ERR_CUDA;
        *mass = sum * dx;
    }
    return NH_OK;
}
