// FP64 residual of a caller's value field that allocates no memory.
//
// Some callers cannot allocate device memory at the point where they need the
// residual: a control loop with a latency budget (cudaMalloc/cudaFree can
// synchronise the whole device), or a process whose device memory is entirely
// owned by another allocator (a framework's caching pool, a fixed memory budget),
// where one more allocation may fail or stall.  hjb_residual_noalloc serves them:
// the caller passes every input and the output as device pointers, and the only
// scratch -- one partial maximum per 32x16-node tile -- lives in a file-scope
// device array of fixed size, resident on every GPU that loads the library until
// the process exits.
#include <cmath>
#include <mutex>

#include "hjb.h"
#include "hjb_kernels.h"

namespace hjb {

namespace {

constexpr int kTileX = 32;
constexpr int kTileY = 16;
constexpr int kMaxTiles = 65536;   // 512 KiB of partial maxima
constexpr int kMaxDevices = 64;

// Shared by every call on a device; each call overwrites the partials it reads.
static __device__ __align__(256) double g_partials[kMaxTiles];

// Host copies of g_partials' device address, one per device ordinal.
double* g_addr[kMaxDevices] = {};
std::mutex g_addr_mutex;

// One thread per node, 32x8 threads covering a 32x16-node tile; neighbours are
// read straight from global memory, so any interpolation reach is served.
// Each block writes the max over its free nodes of |T2 u - u| (eq. SLscheme2).
template <bool SIG>
__global__ void __launch_bounds__(kTileX * 8)
k_residual_partials(GridView g, const double* __restrict__ u, double* partials) {
    __shared__ double red[32];
    const int n = g.n;
    double lmax = 0.0;
    for (int r = 0; r < kTileY / 8; ++r) {
        const int i = blockIdx.x * kTileX + threadIdx.x;
        const int j = blockIdx.y * kTileY + threadIdx.y + r * 8;
        if (i >= n || j >= n) continue;
        const size_t k = (size_t)j * n + i;
        if (g.mask[k] != kFree) continue;
        const double uk = u[k];
        const double c = (double)g.speed[k];
        double bx = 0.0, by = 0.0;
        if (g.drift) {
            const float2 b = g.drift[k];
            bx = (double)b.x;
            by = (double)b.y;
        }
        // non-free vertices take the scheme's fixed values (0 on the target, the
        // obstacle value on obstacles) whatever the caller's array holds there
        const double* base = u + k;
        const uint8_t* mbase = g.mask + k;
        auto U = [&](int dx, int dy) {
            const ptrdiff_t o = (ptrdiff_t)dy * n + dx;
            const uint8_t m = __ldg(mbase + o);
            return m == kFree ? __ldg(base + o) : (m == kTarget ? 0.0 : g.uob64);
        };
        auto C = [&](int m) { return g.ctrl64[m]; };
        double N, D;
        int M;
        best_over_controls<double, SIG>(g, 2, i, j, uk, c, bx, by, 0, 1, C, U, N, D, M);
        // a NaN increment (non-finite values in u or in the inputs) makes the
        // residual +infinity: fmax alone would drop it
        const double inc = fabs(N / D);
        lmax = inc == inc ? fmax(lmax, inc) : INFINITY;
    }
    const double bm = block_max<double>(lmax, red);
    if (threadIdx.x == 0 && threadIdx.y == 0) partials[blockIdx.y * gridDim.x + blockIdx.x] = bm;
}

__global__ void __launch_bounds__(1024) k_max_partials(const double* partials, int count,
                                                       double* out) {
    __shared__ double red[32];
    double m = 0.0;
    for (int t = threadIdx.x; t < count; t += blockDim.x) {
        const double p = partials[t];
        m = p == p ? fmax(m, p) : INFINITY;
    }
    const double bm = block_max<double>(m, red);
    if (threadIdx.x == 0) *out = bm;
}

}  // namespace

}  // namespace hjb

extern "C" int hjb_residual_noalloc(const hjb_desc* desc, const float* speed, const uint8_t* mask,
                                   const float* drift, const double* controls, const double* u,
                                   double* residual_out, void* cuda_stream) {
    using namespace hjb;
    if (!desc || !speed || !mask || !controls || !u || !residual_out) return HJB_ERR_INVALID_ARG;
    const int n = desc->n;
    if (n < 3 || desc->n_controls < 1 || desc->n_controls > HJB_MAX_CONTROLS) return HJB_ERR_INVALID_ARG;
    if (!(desc->lambda >= 0.0) || !(desc->sigma >= 0.0) || !(desc->cost > 0.0) ||
        !std::isfinite(desc->lambda) || !std::isfinite(desc->sigma) || !std::isfinite(desc->cost) ||
        !std::isfinite(desc->h))
        return HJB_ERR_INVALID_ARG;
    const long long tx = (n + kTileX - 1) / kTileX;
    const long long ty = (n + kTileY - 1) / kTileY;
    if (tx * ty > kMaxTiles) return HJB_ERR_INVALID_ARG;   // grid larger than the static scratch
    if (((uintptr_t)controls & 15u) != 0 || ((uintptr_t)u & 7u) != 0 ||
        ((uintptr_t)residual_out & 7u) != 0 || (drift && ((uintptr_t)drift & 7u) != 0))
        return HJB_ERR_INVALID_ARG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return HJB_ERR_CUDA;
    double* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_addr_mutex);
        if (!g_addr[dev]) {
            // first call on this device: resolve the array's device address
            double* ptr = nullptr;
            if (cudaGetSymbolAddress((void**)&ptr, g_partials) != cudaSuccess || !ptr)
                return HJB_ERR_CUDA;
            g_addr[dev] = ptr;
        }
        scratch = g_addr[dev];
    }

    const double dx = 2.0 / (n - 1);
    const double h = desc->h > 0.0 ? desc->h : dx;
    const double beta = 1.0 / (1.0 + desc->lambda * h);
    GridView g{};
    g.n = n;
    g.na = desc->n_controls;
    g.speed = speed;
    g.drift = reinterpret_cast<const float2*>(drift);
    g.mask = mask;
    g.ctrl32 = nullptr;
    g.ctrl64 = reinterpret_cast<const double2*>(controls);
    g.s64 = h / dx;
    g.d64 = std::sqrt(2.0 * h) * desc->sigma / dx;
    g.beta64 = beta;
    g.hl64 = h * desc->cost;
    g.uob64 = desc->lambda > 0.0 ? g.hl64 / (1.0 - beta) : 1e6;
    g.s32 = (float)g.s64;
    g.d32 = (float)g.d64;
    g.beta32 = (float)beta;
    g.hl32 = (float)g.hl64;
    g.uob32 = (float)g.uob64;

    cudaStream_t st = (cudaStream_t)cuda_stream;
    const dim3 grid((unsigned)tx, (unsigned)ty);
    const dim3 block(kTileX, 8);
    count_launches(2);
    if (g.d64 > 0.0)
        k_residual_partials<true><<<grid, block, 0, st>>>(g, u, scratch);
    else
        k_residual_partials<false><<<grid, block, 0, st>>>(g, u, scratch);
    k_max_partials<<<1, 1024, 0, st>>>(scratch, (int)(tx * ty), residual_out);
    return cudaGetLastError() == cudaSuccess ? HJB_OK : HJB_ERR_CUDA;
}
