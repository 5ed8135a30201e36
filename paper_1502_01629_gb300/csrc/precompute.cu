// Pre-computation of the patchy decomposition (Cacace & Falcone, Section 4.3):
// coarse grid data, Q1 interpolation u_hat,
// feedback synthesis (eq. discrete-synthesis) with the causal band keys
// (Section 4.2), winner-take-all transport successors (eq. discrete-advection),
// labels by pointer jumping and the (band, patch) ordering of the free nodes.
#include <cfloat>
#include <cmath>

#include "hjb_kernels.h"
#include "precompute_device.cuh"

namespace hjb {

namespace {

constexpr int kThreads = 256;

inline int blocks_for(long long n, int t = kThreads) { return (int)((n + t - 1) / t); }

// ---------------------------------------------------------------- coarse grid
__global__ void k_coarse_data(int n, int nc, const float* __restrict__ speed,
                              const float2* __restrict__ drift, const uint8_t* __restrict__ mask,
                              float* speed_c, float2* drift_c, uint8_t* mask_c) {
    const int kc = blockIdx.x * blockDim.x + threadIdx.x;
    if (kc >= nc * nc) return;
    coarse_data_node(kc, n, nc, speed, drift, mask, speed_c, drift_c, mask_c);
}

// u_hat: Q1 interpolation of u_c at the fine nodes (nested grids, ratio r).
__global__ void k_interp(int nc, const float* __restrict__ uc, int n,
                         const uint8_t* __restrict__ mask, float u_obst, float* uhat) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * n) return;
    uhat[k] = interp_node(k, nc, uc, n, mask, u_obst);
}

// Synthesis a* and the causal band key of every free node; the largest key is
// folded into *max_key.
__global__ void k_synthesis(GridView g, const float* __restrict__ uhat, BandMap bm, uint8_t* a_out,
                            int32_t* key, int* max_key) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* sctrl = reinterpret_cast<float2*>(smem);
    const int n = g.n;
    for (int m = threadIdx.x; m < g.na; m += blockDim.x) sctrl[m] = g.ctrl32[m];
    __syncthreads();
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    int kk = -1;
    if (k < (size_t)n * n) {
        if (g.mask[k] != kFree) {
            a_out[k] = 255;
            key[k] = -1;
        } else {
            auto C = [&](int m) { return sctrl[m]; };
            a_out[k] = (uint8_t)synthesis_node(g, k, uhat, C);
            kk = band_key(uhat[k], bm);
            key[k] = kk;
        }
    }
    // block max of the keys -> one atomic per warp
    int wm = kk;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wm = max(wm, __shfl_xor_sync(0xffffffffu, wm, off));
    if ((threadIdx.x & 31) == 0 && wm >= 0) atomicMax(max_key, wm);
}

// Band key of the current value (same mapping as in k_synthesis).
__global__ void k_keys_from_values(int N, const uint8_t* __restrict__ mask,
                                   const float* __restrict__ u, BandMap bm, int32_t* key,
                                   int* max_key) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    int kk = -1;
    if (k < N) {
        if (mask[k] != kFree) {
            key[k] = -1;
        } else {
            kk = band_key(u[k], bm);
            key[k] = kk;
        }
    }
    int wm = kk;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wm = max(wm, __shfl_xor_sync(0xffffffffu, wm, off));
    if ((threadIdx.x & 31) == 0 && wm >= 0) atomicMax(max_key, wm);
}

// Successor of each free node (non-free nodes point to themselves).
__global__ void k_successors(GridView g, const uint8_t* __restrict__ a, int32_t* succ) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int n = g.n;
    if (k >= (size_t)n * n) return;
    succ[k] = g.mask[k] != kFree ? (int32_t)k : successor_node(g, k, a[k]);
}

// Pointer jumping: out[k] = in[in[k]].
__global__ void k_jump(int N, const int32_t* __restrict__ in, int32_t* __restrict__ out) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) out[k] = in[in[k]];
}

// After enough jumps every pointer sits on its chain's terminal (a non-free
// node) or inside a cycle of free nodes.
__global__ void k_label_from_end(int N, const int32_t* __restrict__ end,
                                 const uint8_t* __restrict__ mask, const int8_t* __restrict__ sector,
                                 int n_patches, int8_t* label) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int t = end[k];
    int8_t lab = (int8_t)n_patches;
    if (mask[t] == kTarget && sector && sector[t] >= 0) lab = sector[t];
    label[k] = lab;
}

// ------------------------------------------------------------------ ordering
// Bin of a free node = band * (N_P + 1) + label; counting sort by bin.
__global__ void k_hist(int N, const int32_t* __restrict__ key, const int8_t* __restrict__ label,
                       const uint8_t* __restrict__ mask, int stride, int32_t* count) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N || mask[k] != kFree) return;
    atomicAdd(&count[key[k] * stride + label[k]], 1);
}

// Exclusive scan of count[0..nb) into off[0..nb], one block.
__global__ void __launch_bounds__(1024) k_scan(int nb, const int32_t* __restrict__ count,
                                               int32_t* off) {
    __shared__ int32_t part[1024];
    const int t = threadIdx.x;
    const int per = (nb + blockDim.x - 1) / blockDim.x;
    const int b0 = min(t * per, nb), b1 = min(b0 + per, nb);
    int32_t s = 0;
    for (int b = b0; b < b1; ++b) s += count[b];
    part[t] = s;
    __syncthreads();
    for (int o = 1; o < blockDim.x; o <<= 1) {
        int32_t v = (t >= o) ? part[t - o] : 0;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    int32_t run = (t == 0) ? 0 : part[t - 1];
    for (int b = b0; b < b1; ++b) {
        off[b] = run;
        run += count[b];
    }
    if (t == blockDim.x - 1) off[nb] = part[t];
}

__global__ void k_scatter(int N, const int32_t* __restrict__ key, const int8_t* __restrict__ label,
                          const uint8_t* __restrict__ mask, int stride, int32_t* cursor,
                          int32_t* order) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N || mask[k] != kFree) return;
    const int pos = atomicAdd(&cursor[key[k] * stride + label[k]], 1);
    order[pos] = k;
}

__global__ void k_hist_key(int N, const int32_t* __restrict__ key, int32_t* count) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int b = key[k];
    if (b >= 0) atomicAdd(&count[b], 1);
}

__global__ void k_scatter_key(int N, const int32_t* __restrict__ key, int32_t* cursor,
                              int32_t* order) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int b = key[k];
    if (b < 0) return;
    order[atomicAdd(&cursor[b], 1)] = k;
}

__global__ void k_band_off(int n_bands, int stride, const int32_t* __restrict__ bin_off,
                           int32_t* band_off) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b <= n_bands) band_off[b] = bin_off[b * stride];
}

// u64 = u32 on free nodes; the exact FP64 held values elsewhere (0 on targets,
// the obstacle value on obstacles -- promoting its FP32 rounding would move the
// FP64 fixed point)
__global__ void k_promote(int N, const float* __restrict__ a, const uint8_t* __restrict__ mask, double uob64,
                          double* b) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int mk = mask[k];
    b[k] = mk == kFree ? (double)a[k] : (mk == kTarget ? 0.0 : uob64);
}

__global__ void k_demote(int N, const double* __restrict__ a, float* b) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k < N) b[k] = (float)a[k];
}

__global__ void k_init_values(int N, const uint8_t* __restrict__ mask, float free_val, float uob,
                              float* u32, double* u64, double uob64) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int mk = mask[k];
    if (u32) u32[k] = (mk == kFree) ? free_val : (mk == kTarget ? 0.0f : uob);
    if (u64) u64[k] = (mk == kFree) ? (double)free_val : (mk == kTarget ? 0.0 : uob64);
}

__global__ void k_fix_nonfree(int N, const uint8_t* __restrict__ mask, float uob, double uob64,
                              float* u32, double* u64) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= N) return;
    const int mk = mask[k];
    if (mk == kFree) return;
    if (u32) u32[k] = (mk == kTarget) ? 0.0f : uob;
    if (u64) u64[k] = (mk == kTarget) ? 0.0 : uob64;
}

}  // namespace

cudaError_t launch_coarse_data(int n, int nc, const float* speed, const float2* drift,
                               const uint8_t* mask, float* speed_c, float2* drift_c,
                               uint8_t* mask_c, cudaStream_t st) {
    count_launches(1);
    k_coarse_data<<<blocks_for((long long)nc * nc), kThreads, 0, st>>>(n, nc, speed, drift, mask,
                                                                         speed_c, drift_c, mask_c);
    return cudaGetLastError();
}

cudaError_t launch_interp(int nc, const float* uc, int n, const uint8_t* mask, float u_obst,
                          float* uhat, cudaStream_t st) {
    count_launches(1);
    k_interp<<<blocks_for((long long)n * n), kThreads, 0, st>>>(nc, uc, n, mask, u_obst, uhat);
    return cudaGetLastError();
}

void band_edges(double lambda, double w, int cap, std::vector<double>& e) {
    e.clear();
    if (!(lambda > 0.0)) return;
    const double span = std::floor(std::log(1e6) / (lambda * w));
    const int L = span + 2.0 < (double)cap ? (int)span + 2 : cap;
    e.resize(L);
    e[0] = 0.0;
    for (int k = 1; k < L; ++k) e[k] = (1.0 - std::exp(-(lambda * ((double)k * w)))) / lambda;
}

cudaError_t launch_synthesis(const GridView& g, const float* uhat, const BandMap& bm, uint8_t* a,
                             int32_t* key, int* max_key, cudaStream_t st) {
    const size_t smem = (size_t)g.na * sizeof(float2);
    count_launches(1);
    k_synthesis<<<blocks_for((long long)g.n * g.n), kThreads, smem, st>>>(g, uhat, bm, a, key, max_key);
    return cudaGetLastError();
}

cudaError_t launch_keys_from_values(int N, const uint8_t* mask, const float* u, const BandMap& bm,
                                    int32_t* key, int* max_key, cudaStream_t st) {
    count_launches(1);
    k_keys_from_values<<<blocks_for(N), kThreads, 0, st>>>(N, mask, u, bm, key, max_key);
    return cudaGetLastError();
}

cudaError_t launch_successors(const GridView& g, const uint8_t* a, int32_t* succ, cudaStream_t st) {
    count_launches(1);
    k_successors<<<blocks_for((long long)g.n * g.n), kThreads, 0, st>>>(g, a, succ);
    return cudaGetLastError();
}

cudaError_t launch_labels(int N, const int32_t* succ, const uint8_t* mask, const int8_t* sector,
                          int n_patches, int32_t* jump_a, int32_t* jump_b, int8_t* label,
                          cudaStream_t st) {
    // 2^rounds >= N: every chain has reached its end or a cycle.
    int rounds = 1;
    while ((1LL << rounds) < (long long)N) ++rounds;
    const int32_t* in = succ;
    int32_t* bufs[2] = {jump_a, jump_b};
    for (int r = 0; r < rounds; ++r) {
        int32_t* out = bufs[r & 1];
        count_launches(1);
        k_jump<<<blocks_for(N), kThreads, 0, st>>>(N, in, out);
        in = out;
    }
    count_launches(1);
    k_label_from_end<<<blocks_for(N), kThreads, 0, st>>>(N, in, mask, sector, n_patches, label);
    return cudaGetLastError();
}

cudaError_t launch_pointer_jumps(long long N, const int32_t* succ, int rounds, int32_t* jump_a,
                                 int32_t* jump_b, const int32_t** result, cudaStream_t st) {
    const int32_t* in = succ;
    int32_t* bufs[2] = {jump_a, jump_b};
    for (int r = 0; r < rounds; ++r) {
        int32_t* out = bufs[r & 1];
        count_launches(1);
        k_jump<<<blocks_for(N), kThreads, 0, st>>>((int)N, in, out);
        in = out;
    }
    *result = in;
    return cudaGetLastError();
}

cudaError_t launch_exclusive_scan(int n, const int32_t* in, int32_t* out, cudaStream_t st) {
    count_launches(1);
    k_scan<<<1, 1024, 0, st>>>(n, in, out);
    return cudaGetLastError();
}

cudaError_t launch_order(int N, const int32_t* key, const int8_t* label, const uint8_t* mask,
                         int n_patches, int n_bands, int32_t* bin_count, int32_t* bin_off,
                         int32_t* order, int32_t* band_off, cudaStream_t st) {
    const int stride = n_patches + 1;
    const int nb = n_bands * stride;
    cudaError_t e = cudaMemsetAsync(bin_count, 0, sizeof(int32_t) * (size_t)nb, st);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_hist<<<blocks_for(N), kThreads, 0, st>>>(N, key, label, mask, stride, bin_count);
    count_launches(1);
    k_scan<<<1, 1024, 0, st>>>(nb, bin_count, bin_off);
    // bin_count becomes the scatter cursor
    e = cudaMemcpyAsync(bin_count, bin_off, sizeof(int32_t) * (size_t)nb, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_scatter<<<blocks_for(N), kThreads, 0, st>>>(N, key, label, mask, stride, bin_count, order);
    count_launches(1);
    k_band_off<<<blocks_for(n_bands + 1), kThreads, 0, st>>>(n_bands, stride, bin_off, band_off);
    return cudaGetLastError();
}

cudaError_t launch_counting_sort(int N, const int32_t* key, int nbins, int32_t* count,
                                 int32_t* off, int32_t* order, cudaStream_t st) {
    cudaError_t e = cudaMemsetAsync(count, 0, sizeof(int32_t) * (size_t)nbins, st);
    if (e != cudaSuccess) return e;
    count_launches(3);
    k_hist_key<<<blocks_for(N), kThreads, 0, st>>>(N, key, count);
    k_scan<<<1, 1024, 0, st>>>(nbins, count, off);
    e = cudaMemcpyAsync(count, off, sizeof(int32_t) * (size_t)nbins, cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    k_scatter_key<<<blocks_for(N), kThreads, 0, st>>>(N, key, count, order);
    return cudaGetLastError();
}

cudaError_t launch_strided_gather(int nb, int stride, const int32_t* off, int32_t* out,
                                  cudaStream_t st) {
    count_launches(1);
    k_band_off<<<blocks_for(nb + 1), kThreads, 0, st>>>(nb, stride, off, out);
    return cudaGetLastError();
}

cudaError_t launch_promote(int N, const float* u32, const uint8_t* mask, double uob64, double* u64,
                           cudaStream_t st) {
    count_launches(1);
    k_promote<<<blocks_for(N), kThreads, 0, st>>>(N, u32, mask, uob64, u64);
    return cudaGetLastError();
}

cudaError_t launch_demote(int N, const double* u64, float* u32, cudaStream_t st) {
    count_launches(1);
    k_demote<<<blocks_for(N), kThreads, 0, st>>>(N, u64, u32);
    return cudaGetLastError();
}

cudaError_t launch_init_values(int N, const uint8_t* mask, float free_val, float uob, float* u32,
                               double* u64, double uob64, cudaStream_t st) {
    count_launches(1);
    k_init_values<<<blocks_for(N), kThreads, 0, st>>>(N, mask, free_val, uob, u32, u64, uob64);
    return cudaGetLastError();
}

cudaError_t launch_fix_nonfree(int N, const uint8_t* mask, float uob, double uob64, float* u32,
                               double* u64, cudaStream_t st) {
    count_launches(1);
    k_fix_nonfree<<<blocks_for(N), kThreads, 0, st>>>(N, mask, uob, uob64, u32, u64);
    return cudaGetLastError();
}


namespace {

// The checks and reductions of the per-node inputs at problem creation, on the
// device (the inputs were just uploaded): one partial result per block, summed
// by the host in block order so that the mean speed is reproducible, and the
// smallest bad index per check folded with atomicMin.
__global__ void __launch_bounds__(kThreads)
k_scan_inputs(long long N, const float* __restrict__ speed, const uint8_t* __restrict__ mask,
              const int8_t* __restrict__ sector, int n_patches, const float2* __restrict__ drift,
              float amax, InputScan* __restrict__ out, unsigned long long* __restrict__ first_bad) {
    float cmax = 0.0f, bmax = 0.0f, fs = 0.0f;
    unsigned long long nfree = 0;
    unsigned flags = 0;
    for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < N;
         k += (long long)gridDim.x * blockDim.x) {
        const float sv = speed[k];
        const unsigned mk = mask[k];
        if (!(sv >= 0.0f && sv <= FLT_MAX)) {
            flags |= 1u;
            atomicMin(first_bad + 0, (unsigned long long)k);
        }
        if (mk > (unsigned)kObstacle) {
            flags |= 2u;
            atomicMin(first_bad + 1, (unsigned long long)k);
        }
        if (sector && mk == (unsigned)kTarget && (sector[k] < -1 || sector[k] >= n_patches)) {
            flags |= 4u;
            atomicMin(first_bad + 2, (unsigned long long)k);
        }
        float bn = 0.0f;
        if (drift) {
            const float2 b = drift[k];
            if (!(fabsf(b.x) <= FLT_MAX && fabsf(b.y) <= FLT_MAX)) {
                flags |= 8u;
                atomicMin(first_bad + 3, (unsigned long long)k);
            }
            bn = hypotf(b.x, b.y);
        }
        if (mk == (unsigned)kObstacle) flags |= 16u;
        if (mk == (unsigned)kFree) {
            ++nfree;
            cmax = fmaxf(cmax, sv);
            if (drift) bmax = fmaxf(bmax, bn);
            fs += sv * amax + bn;
        }
    }
    __shared__ double s_fs[kThreads / 32];
    __shared__ unsigned long long s_nf[kThreads / 32];
    __shared__ float s_cm[kThreads / 32], s_bm[kThreads / 32];
    __shared__ unsigned s_fl[kThreads / 32];
    double fsd = fs;
    for (int off = 16; off > 0; off >>= 1) {
        fsd += __shfl_xor_sync(0xffffffffu, fsd, off);
        nfree += __shfl_xor_sync(0xffffffffu, nfree, off);
        cmax = fmaxf(cmax, __shfl_xor_sync(0xffffffffu, cmax, off));
        bmax = fmaxf(bmax, __shfl_xor_sync(0xffffffffu, bmax, off));
        flags |= __shfl_xor_sync(0xffffffffu, flags, off);
    }
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0) {
        s_fs[w] = fsd;
        s_nf[w] = nfree;
        s_cm[w] = cmax;
        s_bm[w] = bmax;
        s_fl[w] = flags;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        InputScan r{0.0, 0ull, 0.0f, 0.0f, 0u, 0u};
        for (int i = 0; i < kThreads / 32; ++i) {
            r.fsum += s_fs[i];
            r.nfree += s_nf[i];
            r.cmax = fmaxf(r.cmax, s_cm[i]);
            r.bmax = fmaxf(r.bmax, s_bm[i]);
            r.flags |= s_fl[i];
        }
        out[blockIdx.x] = r;
    }
}

}  // namespace

int scan_inputs_blocks(long long N) {
    const long long b = (N + kThreads - 1) / kThreads;
    return (int)(b < 1024 ? (b < 1 ? 1 : b) : 1024);
}

cudaError_t launch_scan_inputs(long long N, const float* speed, const uint8_t* mask, const int8_t* sector,
                               int n_patches, const float2* drift, float amax, InputScan* out,
                               unsigned long long* first_bad, int blocks, cudaStream_t st) {
    count_launches(1);
    k_scan_inputs<<<blocks, kThreads, 0, st>>>(N, speed, mask, sector, n_patches, drift, amax, out, first_bad);
    return cudaGetLastError();
}

}  // namespace hjb
