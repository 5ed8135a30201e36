// Full-grid application of the semi-Lagrangian scheme operator (Cacace &
// Falcone, Section 3, eqs. SLscheme2 / SLscheme3; Section 4.1 for the 2-D
// isotropic diffusion): one thread per node, a 32x16-node tile of u plus a halo
// of R cells staged in shared memory, controls broadcast from shared memory.
// Used as the plain full-grid Jacobi value iteration (the static comparator),
// as a one-shot operator application and as the FP64 residual.
#include <cmath>

#include "hjb_kernels.h"

namespace hjb {

namespace {

constexpr int kTileX = 32;
constexpr int kTileY = 16;
constexpr int kBlockY = 8;

template <typename T> struct IncBits;
template <> struct IncBits<float> { using type = unsigned int; };
template <> struct IncBits<double> { using type = unsigned long long; };

template <typename T, bool SIG>
__global__ void __launch_bounds__(kTileX * kBlockY)
k_sweep_tile(GridView g, int scheme, int R, const T* __restrict__ uin, T* __restrict__ uout,
             int32_t* __restrict__ argmin, typename IncBits<T>::type* incmax) {
    using V2 = typename RealOf<T>::V2;
    extern __shared__ __align__(16) unsigned char smem[];
    V2* sctrl = reinterpret_cast<V2*>(smem);
    const size_t ctrl_bytes = ((size_t)g.na * sizeof(V2) + 15) & ~(size_t)15;
    T* tile = reinterpret_cast<T*>(smem + ctrl_bytes);
    __shared__ T red[32];

    const int n = g.n;
    const int W = kTileX + 2 * R;
    const int H = kTileY + 2 * R;
    const int gx0 = blockIdx.x * kTileX - R;
    const int gy0 = blockIdx.y * kTileY - R;
    const int tid = threadIdx.y * kTileX + threadIdx.x;
    const int nthreads = kTileX * kBlockY;

    for (int m = tid; m < g.na; m += nthreads) sctrl[m] = RealOf<T>::ctrl(g, m);
    // Stage the tile + halo; positions outside the grid are never read (points
    // are projected onto the square), they load a clamped node to stay in bounds.
    for (int t = tid; t < W * H; t += nthreads) {
        const int ty = t / W;
        const int tx = t - ty * W;
        const int gx = min(max(gx0 + tx, 0), n - 1);
        const int gy = min(max(gy0 + ty, 0), n - 1);
        tile[t] = uin[(size_t)gy * n + gx];
    }
    __syncthreads();

    T lmax = T(0);
#pragma unroll 1
    for (int r = 0; r < kTileY / kBlockY; ++r) {
        const int i = blockIdx.x * kTileX + threadIdx.x;
        const int j = blockIdx.y * kTileY + threadIdx.y + r * kBlockY;
        if (i >= n || j >= n) continue;
        const size_t k = (size_t)j * n + i;
        const int lx = i - gx0;
        const int ly = j - gy0;
        const T uk = tile[ly * W + lx];
        T out = uk;
        int am = -1;
        if (g.mask[k] == kFree) {
            const T c = (T)g.speed[k];
            T bx = T(0), by = T(0);
            if (g.drift) {
                const float2 b = g.drift[k];
                bx = (T)b.x;
                by = (T)b.y;
            }
            const T* base = tile + ly * W + lx;
            auto U = [&](int dx, int dy) { return base[dy * W + dx]; };
            auto C = [&](int m) { return sctrl[m]; };
            T N, D;
            int M;
            best_over_controls<T, SIG>(g, scheme, i, j, uk, c, bx, by, 0, 1, C, U, N, D, M);
            const T du = N / D;
            out = uk + du;
            am = M;
            lmax = fmax(lmax, fabs(du));
        }
        if (uout) uout[k] = out;
        if (argmin) argmin[k] = am;
    }
    const T bm = block_max<T>(lmax, red);
    if (tid == 0) atomic_max_nonneg(incmax, bm);
}

template <typename T, bool SIG>
cudaError_t launch_sweep_impl(const GridView& g, int scheme, int R, const T* uin, T* uout,
                              int32_t* argmin, typename IncBits<T>::type* incmax, cudaStream_t st) {
    using V2 = typename RealOf<T>::V2;
    const size_t ctrl_bytes = ((size_t)g.na * sizeof(V2) + 15) & ~(size_t)15;
    const size_t smem = ctrl_bytes + (size_t)(kTileX + 2 * R) * (kTileY + 2 * R) * sizeof(T);
    auto kern = k_sweep_tile<T, SIG>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 block(kTileX, kBlockY);
    dim3 grid((g.n + kTileX - 1) / kTileX, (g.n + kTileY - 1) / kTileY);
    count_launches(1);
    kern<<<grid, block, smem, st>>>(g, scheme, R, uin, uout, argmin, incmax);
    return cudaGetLastError();
}

}  // namespace

// Every Q1 vertex of a point at offset d (|d| <= reach) from its node lies
// within floor(|d|) + 1 cells of it.  The reach is computed in FP64 on the host
// while the kernels form offsets in FP32, so a relative margin covers the FP32
// rounding of the offset.
int sweep_halo(double reach_cells) { return (int)std::floor(reach_cells * (1.0 + 1e-5) + 1e-5) + 1; }

cudaError_t launch_sweep_f32(const GridView& g, bool sig, int scheme, int halo, const float* uin,
                             float* uout, int32_t* argmin, unsigned int* incmax, cudaStream_t st) {
    return sig ? launch_sweep_impl<float, true>(g, scheme, halo, uin, uout, argmin, incmax, st)
               : launch_sweep_impl<float, false>(g, scheme, halo, uin, uout, argmin, incmax, st);
}

cudaError_t launch_sweep_f64(const GridView& g, bool sig, int scheme, int halo, const double* uin,
                             double* uout, int32_t* argmin, unsigned long long* incmax,
                             cudaStream_t st) {
    return sig ? launch_sweep_impl<double, true>(g, scheme, halo, uin, uout, argmin, incmax, st)
               : launch_sweep_impl<double, false>(g, scheme, halo, uin, uout, argmin, incmax, st);
}

}  // namespace hjb
