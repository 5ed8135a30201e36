// Full-grid application of the semi-Lagrangian scheme operator (Cacace &
// Falcone, Section 3, eqs. SLscheme2 / SLscheme3; Section 4.1 for the 2-D
// isotropic diffusion): one thread per node, a 32x16-node tile of u plus a halo
// of R cells staged in shared memory, controls broadcast from shared memory.
// Used as the plain full-grid Jacobi value iteration (the static comparator),
// as a one-shot operator application and as the FP64 residual.
#include <cmath>

#include "hjb_kernels.h"
#include "sweep_device.cuh"

namespace hjb {

namespace {

constexpr int kTileX = 32;
constexpr int kTileY = 16;
constexpr int kBlockY = 8;

template <typename T> struct IncBits;
template <> struct IncBits<float> { using type = unsigned int; };
template <> struct IncBits<double> { using type = unsigned long long; };

template <typename T, bool SIG, bool GEN>
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

    // staged window inside the grid: every point of every node stays inside the
    // square, so the projection is skipped
    const bool interior = gx0 >= 0 && gy0 >= 0 && gx0 + W <= n && gy0 + H <= n;
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
            const T* base = tile + ly * W + lx;
            auto C = [&](int m) { return sctrl[m]; };
            int M;
            const T du = interior ? node_increment<T, SIG, false, GEN>(g, scheme, i, j, k, base, W, C, M)
                                  : node_increment<T, SIG, true, GEN>(g, scheme, i, j, k, base, W, C, M);
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
    // problems with general terms (Section 5.3) take their own instantiation
    auto kern = g.gen ? k_sweep_tile<T, SIG, true> : k_sweep_tile<T, SIG, false>;
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

// FP64 sup-residual ||T2 u - u|| (eq. SLscheme2) with exact FP32 screening.
// Per node an FP32 pass finds the smallest candidate v32_min over the controls;
// a control whose FP32 candidate exceeds v32_min by more than `margin` cannot be
// the FP64 minimiser as long as |v32 - v64| <= margin / 2 for every control
// (the host sizes the margin from the FP32 rounding of the values), so only
// the remaining controls are evaluated in FP64.  The result is the FP64 min,
// hence the same residual as the unscreened FP64 evaluation.
template <bool SIG>
__global__ void __launch_bounds__(kTileX * kBlockY)
k_residual_screened(GridView g, int R, const double* __restrict__ u, float margin,
                    unsigned long long* incmax, float* rfield, uint8_t* afield) {
    extern __shared__ __align__(16) unsigned char smem[];
    double2* c64 = reinterpret_cast<double2*>(smem);
    const size_t cb64 = ((size_t)g.na * sizeof(double2) + 15) & ~(size_t)15;
    float2* c32 = reinterpret_cast<float2*>(smem + cb64);
    const size_t cb32 = ((size_t)g.na * sizeof(float2) + 15) & ~(size_t)15;
    const int n = g.n;
    const int W = kTileX + 2 * R;
    const int H = kTileY + 2 * R;
    double* t64 = reinterpret_cast<double*>(smem + cb64 + cb32);
    float* t32 = reinterpret_cast<float*>(t64 + (size_t)W * H);
    __shared__ double red[32];
    const int gx0 = blockIdx.x * kTileX - R;
    const int gy0 = blockIdx.y * kTileY - R;
    const int tid = threadIdx.y * kTileX + threadIdx.x;
    const int nthreads = kTileX * kBlockY;
    for (int m = tid; m < g.na; m += nthreads) {
        c64[m] = g.ctrl64[m];
        c32[m] = g.ctrl32[m];
    }
    for (int t = tid; t < W * H; t += nthreads) {
        const int ty = t / W;
        const int tx = t - ty * W;
        const int gx = min(max(gx0 + tx, 0), n - 1);
        const int gy = min(max(gy0 + ty, 0), n - 1);
        const double v = u[(size_t)gy * n + gx];
        t64[t] = v;
        t32[t] = (float)v;
    }
    __syncthreads();
    double lmax = 0.0;
#pragma unroll 1
    for (int r = 0; r < kTileY / kBlockY; ++r) {
        const int i = blockIdx.x * kTileX + threadIdx.x;
        const int j = blockIdx.y * kTileY + threadIdx.y + r * kBlockY;
        if (i >= n || j >= n) continue;
        const size_t k = (size_t)j * n + i;
        if (g.mask[k] != kFree) {
            if (rfield) {
                rfield[k] = 0.0f;
                afield[k] = 0;
            }
            continue;
        }
        const int off = (j - gy0) * W + (i - gx0);
        if (rfield) {
            double v;
            int m;
            lmax = fmax(lmax, residual_node<SIG>(g, i, j, k, t32, t64, off, W, c32, c64, margin, &v, &m));
            rfield[k] = (float)v;
            afield[k] = (uint8_t)m;
        } else {
            lmax = fmax(lmax, residual_node<SIG>(g, i, j, k, t32, t64, off, W, c32, c64, margin));
        }
    }
    const double bm = block_max<double>(lmax, red);
    if (tid == 0) atomic_max_nonneg(incmax, bm);
}

// One Jacobi sweep of the correction equation of the FP64 stage: with the
// residual r = T2 u - u (eq. SLscheme2) and its minimising control a fixed per
// node, the correction e solves e = beta P_a e + r (P_a: the Markov-chain
// transition of eq. SLscheme2 under control a), i.e. one policy evaluation of
// the linearised scheme; it is swept in the self-weight-free form of eq.
// SLscheme3, e_i <- e_i + (beta S'_a + r_i - (1 - beta) e_i) / (1 - beta Lambda0_a),
// in FP32 (e is small: its rounding is relative to e, not to u).  Non-free
// nodes hold e = 0.
template <bool SIG>
__global__ void __launch_bounds__(kTileX * kBlockY)
k_correction_sweep(GridView g, int R, const uint8_t* __restrict__ act, const float* __restrict__ r,
                   const float* __restrict__ ein, float* __restrict__ eout, unsigned int* incmax) {
    extern __shared__ __align__(16) unsigned char smem[];
    float* tile = reinterpret_cast<float*>(smem);
    __shared__ float red[32];
    const int n = g.n;
    const int W = kTileX + 2 * R;
    const int H = kTileY + 2 * R;
    const int gx0 = blockIdx.x * kTileX - R;
    const int gy0 = blockIdx.y * kTileY - R;
    const int tid = threadIdx.y * kTileX + threadIdx.x;
    for (int t = tid; t < W * H; t += kTileX * kBlockY) {
        const int ty = t / W;
        const int tx = t - ty * W;
        const int gx = min(max(gx0 + tx, 0), n - 1);
        const int gy = min(max(gy0 + ty, 0), n - 1);
        tile[t] = ein[(size_t)gy * n + gx];
    }
    __syncthreads();
    const float beta = g.beta32, s = g.s32;
    const float bq = SIG ? beta * 0.25f : beta;
    float lmax = 0.0f;
#pragma unroll 1
    for (int rr = 0; rr < kTileY / kBlockY; ++rr) {
        const int i = blockIdx.x * kTileX + threadIdx.x;
        const int j = blockIdx.y * kTileY + threadIdx.y + rr * kBlockY;
        if (i >= n || j >= n) continue;
        const size_t k = (size_t)j * n + i;
        if (g.mask[k] != kFree) {
            eout[k] = 0.0f;
            continue;
        }
        const float* base = tile + (j - gy0) * W + (i - gx0);
        const float ek = base[0];
        auto U = [&](int dx, int dy) { return base[dy * W + dx]; };
        float bx = 0.0f, by = 0.0f;
        if (g.drift) {
            const float2 b = g.drift[k];
            bx = b.x;
            by = b.y;
        }
        const NodeBox<float> box = node_box<float>(i, j, n);
        const float c0 = fmaf(-(1.0f - beta), ek, r[k]);
        float N, D;
        candidate<float, SIG, true>(g, 3, box, s, bq, c0, ek, g.speed[k], bx, by, g.ctrl32[act[k]], U, N, D);
        const float de = N / D;
        eout[k] = ek + de;
        lmax = fmaxf(lmax, fabsf(de));
    }
    const float bm = block_max<float>(lmax, red);
    if (tid == 0) atomicMax(incmax, __float_as_uint(bm));
}

// u <- u + e on free nodes (FP64 values, FP32 correction)
__global__ void k_add_correction(long long N, const uint8_t* __restrict__ mask, const float* __restrict__ e,
                                 double* u) {
    const long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N && mask[k] == kFree) u[k] += (double)e[k];
}

}  // namespace

// Every Q1 vertex of a point at offset d (|d| <= reach) from its node lies
// within floor(|d|) + 1 cells of it.  The reach is computed in FP64 on the host
// while the kernels form offsets in FP32, so a relative margin covers the FP32
// rounding of the offset.
int sweep_halo(double reach_cells) { return (int)std::floor(reach_cells * (1.0 + 1e-5) + 1e-5) + 1; }

size_t residual_screened_smem(int na, int R) {
    const size_t cb64 = ((size_t)na * sizeof(double2) + 15) & ~(size_t)15;
    const size_t cb32 = ((size_t)na * sizeof(float2) + 15) & ~(size_t)15;
    const size_t wh = (size_t)(kTileX + 2 * R) * (kTileY + 2 * R);
    return cb64 + cb32 + wh * (sizeof(double) + sizeof(float));
}

cudaError_t launch_residual_screened(const GridView& g, bool sig, int halo, const double* u,
                                     float margin, unsigned long long* incmax, cudaStream_t st,
                                     float* rfield, uint8_t* afield) {
    const size_t smem = residual_screened_smem(g.na, halo);
    auto kern = sig ? k_residual_screened<true> : k_residual_screened<false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 block(kTileX, kBlockY);
    dim3 grid((g.n + kTileX - 1) / kTileX, (g.n + kTileY - 1) / kTileY);
    count_launches(1);
    kern<<<grid, block, smem, st>>>(g, halo, u, margin, incmax, rfield, afield);
    return cudaGetLastError();
}

cudaError_t launch_correction_sweep(const GridView& g, bool sig, int halo, const uint8_t* act,
                                    const float* r, const float* ein, float* eout, unsigned int* incmax,
                                    cudaStream_t st) {
    const size_t smem = (size_t)(kTileX + 2 * halo) * (kTileY + 2 * halo) * sizeof(float);
    auto kern = sig ? k_correction_sweep<true> : k_correction_sweep<false>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    dim3 block(kTileX, kBlockY);
    dim3 grid((g.n + kTileX - 1) / kTileX, (g.n + kTileY - 1) / kTileY);
    count_launches(1);
    kern<<<grid, block, smem, st>>>(g, halo, act, r, ein, eout, incmax);
    return cudaGetLastError();
}

cudaError_t launch_add_correction(long long N, const uint8_t* mask, const float* e, double* u, cudaStream_t st) {
    count_launches(1);
    k_add_correction<<<(unsigned)((N + 255) / 256), 256, 0, st>>>(N, mask, e, u);
    return cudaGetLastError();
}

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
