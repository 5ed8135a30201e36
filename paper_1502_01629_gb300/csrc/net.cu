// Learned warm start for the coarse solve: a 6-layer 3x3 convolutional network
// (32 channels, BF16 weights and activations, FP32 accumulation) that maps a
// coarse instance (speed, target mask, obstacle mask, sigma, lambda) to the
// coarse value and the feedback control index.  The coarse solve of Section 4.3
// has the last word: the prediction only replaces its initial value, and a plain
// start is restored when the value after K sweeps still moves by more than a
// threshold, so the fixed point is unchanged and only the sweep count moves.
//
// Convolutions run on the 5th-generation tensor cores as implicit GEMMs: a CTA
// takes 128 consecutive pixels (NHWC, channels contiguous); its threads gather
// each pixel's 3x3 neighbourhood (16-byte chunks of 8 channels, zero outside the
// image) straight into the canonical K-major shared-memory layout of the A
// operand [128 x 9 Cin]; the weights arrive pre-packed in the same layout as the
// B operand [Cout x 9 Cin]; one thread issues the K/16 tcgen05.mma (BF16 x BF16 ->
// FP32 in tensor memory) and commits to an mbarrier; the epilogue reads the
// accumulator with tcgen05.ld and applies bias, ReLU or the ReLU mask of the
// backward pass.  The input gradient (dgrad) is the same kernel with the
// weights flipped and transposed; the weight gradient (wgrad) is a third
// implicit GEMM on the tensor cores whose reduction runs over the pixels.
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "hjb_kernels.h"
#include "tc.cuh"

namespace hjb {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kConvThreads = 128;   // 4 warps: one TMEM lane quarter each
constexpr int kMmaWaitIters = 1 << 24;

// ------------------------------------------------------------ forward / dgrad
// out[p, n] = epilogue( sum_{t, ci} x[p + off_t, ci] * w[n, t, ci] ), n < NPAD,
// for p < total pixels (images of H x W, NHWC with CIN channels).
// epilogue: + bias[n] (if bias and n < nbias), max(0, .) (if relu),
// * (mask[p, n] > 0) (if mask).
template <int CIN, int NPAD, bool OUT_F32>
__global__ void __launch_bounds__(kConvThreads)
k_conv3x3_tc(const bf16* __restrict__ x, const uint8_t* __restrict__ wpack,
             const float* __restrict__ bias, int nbias, int relu, const bf16* __restrict__ mask, int total,
             int H, int W, int dil, void* __restrict__ out, int* err) {
    constexpr int K = 9 * CIN;
    constexpr int KC = K / 8;                      // 16-byte chunks per operand row
    constexpr int TMC = NPAD <= 32 ? 32 : 64;      // tensor-memory columns
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                      // 128 x K bf16, canonical
    unsigned char* sB = smem + 128 * K * 2;        // NPAD x K bf16, canonical
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_taddr;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const long long p0 = (long long)blockIdx.x * 128;
    const int HW = H * W;

    if (tid == 0) tc::mbar_init(&mbar, 1);
    if (warp == 0) tc::tmem_alloc<TMC>(&s_taddr);
    {
        const uint4* src = reinterpret_cast<const uint4*>(wpack);
        uint4* dst = reinterpret_cast<uint4*>(sB);
        for (int i = tid; i < NPAD * KC; i += kConvThreads) dst[i] = src[i];
    }
    // thread m gathers pixel p0 + m (its image coordinates formed once), chunk by
    // chunk: at a given chunk a warp writes four whole 128-byte core-matrix
    // blocks (no bank conflicts) and reads the same tap of 32 consecutive pixels
    {
        const int m = tid;
        const long long p = p0 + m;
        const bool pv = p < total;
        int py = 0, px = 0;
        if (pv) {
            const int r = (int)(p % HW);
            py = r / W;
            px = r - py * W;
        }
        for (int kc = 0; kc < KC; ++kc) {
            const int t = kc / (CIN / 8), cc = kc - t * (CIN / 8);
            const int dyt = (t / 3 - 1) * dil, dxt = (t % 3 - 1) * dil;
            const int yy = py + dyt, xq = px + dxt;
            uint4 v = make_uint4(0u, 0u, 0u, 0u);
            if (pv && yy >= 0 && yy < H && xq >= 0 && xq < W)
                v = *reinterpret_cast<const uint4*>(x + (size_t)(p + (long long)dyt * W + dxt) * CIN + cc * 8);
            *reinterpret_cast<uint4*>(sA + ((m >> 3) * KC + kc) * 128 + (m & 7) * 16) = v;
        }
    }
    tc::fence_async_smem();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s_taddr;
    if (tid == 0) {
        constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NPAD);
        const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
        for (int s = 0; s < K / 16; ++s) {
            const uint64_t ad = tc::desc_noswizzle(a0 + s * 256, 128, KC * 128);
            const uint64_t bd = tc::desc_noswizzle(b0 + s * 256, 128, KC * 128);
            tc::mma_bf16(taddr, ad, bd, idesc, s > 0 ? 1u : 0u);
        }
        tc::mma_commit(&mbar);
    }
    const bool ok = tc::mbar_wait(&mbar, 0, kMmaWaitIters);
    if (!ok && lane == 0) atomicExch(err, 1);
    tc::fence_after_sync();
    if (ok) {
        const int m = warp * 32 + lane;
        const long long p = p0 + m;
        for (int c = 0; c < NPAD / 16; ++c) {
            uint32_t r[16];
            tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + c * 16, r);
            tc::tmem_ld_wait();
            if (p < total) {
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = c * 16 + q;
                    float a = __uint_as_float(r[q]);
                    if (bias && n < nbias) a += bias[n];
                    if (relu) a = fmaxf(a, 0.0f);
                    if (mask && !(__bfloat162float(mask[(size_t)p * NPAD + n]) > 0.0f)) a = 0.0f;
                    v[q] = a;
                }
                if constexpr (OUT_F32) {
                    float4* o = reinterpret_cast<float4*>(reinterpret_cast<float*>(out) + (size_t)p * NPAD + c * 16);
#pragma unroll
                    for (int q = 0; q < 4; ++q) o[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                } else {
                    __align__(16) bf16 h[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) h[q] = __float2bfloat16(v[q]);
                    uint4* o = reinterpret_cast<uint4*>(reinterpret_cast<bf16*>(out) + (size_t)p * NPAD + c * 16);
                    o[0] = reinterpret_cast<const uint4*>(h)[0];
                    o[1] = reinterpret_cast<const uint4*>(h)[1];
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc<TMC>(taddr);
}

// ------------------------------------------------------------------ wgrad
// dw[n, t * CIN + ci] += sum_p dy[p, n] x[p + off_t, ci]; db[n] += sum_p dy[p, n]
// for n < cout (dw rows of K = 9 CIN floats), over the pixels [blockIdx.x * chunk,
// ... + chunk); FP32 accumulation.
template <int CIN, int NPAD>
__global__ void __launch_bounds__(256)
k_conv3x3_wgrad(const bf16* __restrict__ x, const bf16* __restrict__ dy, int total, int H, int W,
                int dil, int chunk, int cout, float* dw, float* db) {
    constexpr int K = 9 * CIN;
    constexpr int NOUT = NPAD * K;
    constexpr int PER = (NOUT + 255) / 256;
    constexpr int SUB = 32;
    extern __shared__ __align__(1024) unsigned char smem[];
    float* sdy = reinterpret_cast<float*>(smem);           // SUB x NPAD
    float* sx = sdy + SUB * NPAD;                           // SUB x K
    const int tid = threadIdx.x;
    const int HW = H * W;
    float acc[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) acc[j] = 0.0f;
    float bacc = 0.0f;
    const long long pbeg = (long long)blockIdx.x * chunk;
    const long long pend = pbeg + chunk < total ? pbeg + chunk : (long long)total;
    for (long long s = pbeg; s < pend; s += SUB) {
        for (int e = tid; e < SUB * NPAD; e += 256) {
            const int q = e / NPAD, c = e - q * NPAD;
            const long long p = s + q;
            sdy[e] = p < pend ? __bfloat162float(dy[(size_t)p * NPAD + c]) : 0.0f;
        }
        for (int e = tid; e < SUB * K; e += 256) {
            const int q = e / K, k = e - q * K;
            const int t = k / CIN, ci = k - t * CIN;
            const long long p = s + q;
            float v = 0.0f;
            if (p < pend) {
                const int b = (int)(p / HW), r = (int)(p - (long long)b * HW);
                const int yy = r / W + (t / 3 - 1) * dil, xq = r % W + (t % 3 - 1) * dil;
                if (yy >= 0 && yy < H && xq >= 0 && xq < W)
                    v = __bfloat162float(x[((size_t)b * HW + (size_t)yy * W + xq) * CIN + ci]);
            }
            sx[e] = v;
        }
        __syncthreads();
#pragma unroll
        for (int j = 0; j < PER; ++j) {
            const int o = tid + 256 * j;
            if (o < NOUT) {
                const int n = o / K, k = o - (o / K) * K;
                float a = acc[j];
                // two shared loads per FMA: a short unroll keeps the code (and
                // the build) small at no cost
#pragma unroll 4
                for (int q = 0; q < SUB; ++q) a = fmaf(sdy[q * NPAD + n], sx[q * K + k], a);
                acc[j] = a;
            }
        }
        if (tid < NPAD)
            for (int q = 0; q < SUB; ++q) bacc += sdy[q * NPAD + tid];
        __syncthreads();
    }
#pragma unroll
    for (int j = 0; j < PER; ++j) {
        const int o = tid + 256 * j;
        if (o < cout * K && acc[j] != 0.0f) atomicAdd(dw + o, acc[j]);
    }
    if (tid < cout && db && bacc != 0.0f) atomicAdd(db + tid, bacc);
}

// --------------------------------------------------- wgrad on tensor cores
// dW[n, m] = sum_p X[p, m] dy[p, n] with X the 3x3 (dilated) im2col of x
// (m = t * CIN + ci) is a GEMM whose reduction runs over the pixels:
// D[m, n] = sum_p A[m, p] B[n, p] with A = X^T and B = dy^T.  A CTA takes a chunk
// of pixels in tiles of 128; per tile its threads transpose x and dy into the
// canonical K-major layout of A (MT tiles of 128 rows m, the pixels along K) and
// B (NPAD rows n), one thread issues MT x 8 tcgen05.mma (K = 16 pixels each)
// accumulating D in tensor memory across the chunk, and the epilogue adds the
// chunk's partial dW (and, from a row of ones in A, the bias gradient
// sum_p dy[p, n]) to dw / db with FP32 atomics.
template <int CIN, int NPAD>
struct WgradShape {
    static constexpr int K = 9 * CIN;                 // dW row length (taps x channels)
    static constexpr int MT = (K + 1 + 127) / 128;    // 128-row tiles of A (row K: ones)
    static constexpr int TMC = MT * NPAD <= 64 ? 64 : (MT * NPAD <= 128 ? 128 : 256);
    static constexpr size_t smem = (size_t)MT * 128 * 128 * 2 + (size_t)NPAD * 128 * 2;
};

template <int CIN, int NPAD>
__global__ void __launch_bounds__(kConvThreads)
k_conv3x3_wgrad_tc(const bf16* __restrict__ x, const bf16* __restrict__ dy, int total, int H, int W,
                   int dil, int chunk, int cout, float* dw, float* db, int* err) {
    using S = WgradShape<CIN, NPAD>;
    constexpr int K = S::K, MT = S::MT;
    extern __shared__ __align__(1024) unsigned char smem[];
    unsigned char* sA = smem;                               // MT x [128 x 128] bf16
    unsigned char* sB = smem + (size_t)MT * 128 * 128 * 2;  // NPAD x 128 bf16
    __shared__ __align__(8) uint64_t mbar;
    __shared__ uint32_t s_taddr;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int HW = H * W;
    const long long pbeg = (long long)blockIdx.x * chunk;
    const long long pend = pbeg + chunk < total ? pbeg + chunk : (long long)total;
    if (tid == 0) tc::mbar_init(&mbar, 1);
    if (warp == 0) tc::tmem_alloc<S::TMC>(&s_taddr);
    // rows past K + 1 stay zero for the whole chunk
    for (int i = tid; i < (int)(S::smem / 16); i += kConvThreads)
        reinterpret_cast<uint4*>(smem)[i] = make_uint4(0u, 0u, 0u, 0u);
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t taddr = s_taddr;
    const uint32_t a0 = tc::smem_addr(sA), b0 = tc::smem_addr(sB);
    constexpr uint32_t idesc = tc::idesc_bf16_f32(128, NPAD);
    bool ok = true;
    uint32_t phase = 0;
    int tiles = 0;
    // the transposes into the K-major layout (pixels along K) go through
    // stmatrix.trans: a warp takes 32 pixels q0 .. q0 + 31 and one 8-channel
    // chunk as four 8x8 matrices (rows = pixels, lane L holding channels
    // 2(L%4), +1 of pixel q0 + 8i + L/4 in matrix i) and stores each transposed:
    // row j = channel j of the chunk over 8 consecutive pixels, one 16-byte
    // canonical row (whole 128-byte core-matrix blocks, no bank conflicts)
    const int fr = lane >> 2, fc = lane & 3;       // fragment row (pixel), column pair
    const int sm = lane >> 3, sj = lane & 7;       // stored matrix, row (channel)
    const int q0 = warp * 32;                      // the warp's 32 pixels of a tile
    for (long long s = pbeg; s < pend; s += 128, ++tiles) {
        // the lane's four fragment pixels s + q0 + 8i + fr, coordinates formed once
        long long pp[4];
        int py[4], px[4];
        bool pv[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            pp[i] = s + q0 + 8 * i + fr;
            pv[i] = pp[i] < pend;
            py[i] = px[i] = 0;
            if (pv[i]) {
                const int r = (int)(pp[i] % HW);
                py[i] = r / W;
                px[i] = r - py[i] * W;
            }
        }
        // A: element (m, q) = x at pixel s + q shifted by tap t = m / CIN, channel
        // m % CIN (0 outside the image or past the chunk); row K = 1 for a pixel
#pragma unroll 2
        for (int it = 0; it < 9 * (CIN / 8); ++it) {
            const int t = it / (CIN / 8), cc = it - t * (CIN / 8);
            const int dyt = (t / 3 - 1) * dil, dxt = (t % 3 - 1) * dil;
            uint32_t rv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const int yy = py[i] + dyt, xq = px[i] + dxt;
                rv[i] = (pv[i] && yy >= 0 && yy < H && xq >= 0 && xq < W)
                            ? *reinterpret_cast<const uint32_t*>(
                                  x + (size_t)(pp[i] + (long long)dyt * W + dxt) * CIN + cc * 8 + 2 * fc)
                            : 0u;
            }
            const int m = t * CIN + cc * 8 + sj;
            const uint32_t dst = a0 + (uint32_t)((m >> 7) * 128 * 128 * 2) +
                                 tc::canon_offset(m & 127, q0 + 8 * sm, 128);
            tc::stmatrix_x4_trans(dst, rv[0], rv[1], rv[2], rv[3]);
        }
        if (tid < 128) {
            const int m = K;
            *reinterpret_cast<bf16*>(sA + (size_t)(m >> 7) * 128 * 128 * 2 + tc::canon_offset(m & 127, tid, 128)) =
                __float2bfloat16(s + tid < pend ? 1.0f : 0.0f);
        }
        // B: element (n, q) = dy[s + q, n]
        for (int c8 = 0; c8 < NPAD / 8; ++c8) {
            uint32_t rv[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                rv[i] = pv[i] ? *reinterpret_cast<const uint32_t*>(dy + (size_t)pp[i] * NPAD + c8 * 8 + 2 * fc)
                              : 0u;
            const uint32_t dst = b0 + tc::canon_offset(c8 * 8 + sj, q0 + 8 * sm, 128);
            tc::stmatrix_x4_trans(dst, rv[0], rv[1], rv[2], rv[3]);
        }
        tc::fence_async_smem();
        tc::fence_before_sync();
        __syncthreads();
        tc::fence_after_sync();
        if (tid == 0) {
            for (int mt = 0; mt < MT; ++mt)
                for (int ks = 0; ks < 8; ++ks) {
                    const uint64_t ad =
                        tc::desc_noswizzle(a0 + mt * 128 * 128 * 2 + ks * 256, 128, 16 * 128);
                    const uint64_t bd = tc::desc_noswizzle(b0 + ks * 256, 128, 16 * 128);
                    tc::mma_bf16(taddr + mt * NPAD, ad, bd, idesc, (tiles > 0 || ks > 0) ? 1u : 0u);
                }
            tc::mma_commit(&mbar);
        }
        // the operands are overwritten by the next tile: wait for the MMAs
        ok = ok && tc::mbar_wait(&mbar, phase, kMmaWaitIters);
        phase ^= 1u;
        tc::fence_after_sync();
        if (!ok) break;
    }
    if (!ok && lane == 0) atomicExch(err, 1);
    if (ok && tiles > 0) {
        // D rows m = mt * 128 + warp * 32 + lane, columns n
        for (int mt = 0; mt < MT; ++mt) {
            const int m = mt * 128 + warp * 32 + lane;
            for (int c = 0; c < NPAD / 16; ++c) {
                uint32_t r[16];
                tc::tmem_ld16(taddr + ((uint32_t)(warp * 32) << 16) + mt * NPAD + c * 16, r);
                tc::tmem_ld_wait();
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    const int n = c * 16 + q;
                    const float v = __uint_as_float(r[q]);
                    if (n >= cout || v == 0.0f) continue;
                    if (m < K)
                        atomicAdd(dw + (size_t)n * K + m, v);
                    else if (m == K && db)
                        atomicAdd(db + n, v);
                }
            }
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc<S::TMC>(taddr);
}

// -------------------------------------------------------- weight packing
// forward B operand: (n, k = t * CINP + ci) = w[n, t, ci] (w: [cout][9][cin]), zero padded
__global__ void k_pack_fwd(const float* __restrict__ w, int cout, int cin, int CINP, int NPAD,
                           uint8_t* out) {
    const int K = 9 * CINP;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NPAD * K) return;
    const int n = e / K, k = e - n * K;
    const int t = k / CINP, ci = k - t * CINP;
    const float v = (n < cout && ci < cin) ? w[((size_t)n * 9 + t) * cin + ci] : 0.0f;
    *reinterpret_cast<bf16*>(out + tc::canon_offset(n, k, K)) = __float2bfloat16(v);
}

// dgrad B operand: the input gradient is the 3x3 correlation of the output
// gradient (channels COP = padded cout) with w'[ci, t', co] = w[co, 8 - t', ci]
// (taps mirrored, channels swapped): (n' = ci, k' = t' * COP + co)
__global__ void k_pack_dgrad(const float* __restrict__ w, int cout, int cin, int COP, int NPAD,
                             uint8_t* out) {
    const int K = 9 * COP;
    const int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= NPAD * K) return;
    const int n = e / K, k = e - n * K;
    const int t = k / COP, co = k - t * COP;
    const float v = (n < cin && co < cout) ? w[((size_t)co * 9 + (8 - t)) * cin + n] : 0.0f;
    *reinterpret_cast<bf16*>(out + tc::canon_offset(n, k, K)) = __float2bfloat16(v);
}

// ------------------------------------------------------------------- loss
// Per free pixel: value loss (o0 - t)^2 and cross-entropy of the control logits
// o1..o32 against the target index; gradients (scaled by the weights over the
// number of free pixels) as BF16 into dz [p][48]; sums into loss[0..1].
__global__ void k_loss(const float* __restrict__ out, const float* __restrict__ tval,
                       const uint8_t* __restrict__ tctrl, const uint8_t* __restrict__ freem, int total,
                       int n_ctrl, float wv, float wc, float inv_nfree, bf16* dz, double* loss) {
    const long long p = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double lv = 0.0, lc = 0.0;
    if (p < total) {
        float g[48];
#pragma unroll
        for (int c = 0; c < 48; ++c) g[c] = 0.0f;
        if (freem[p]) {
            const float* o = out + (size_t)p * 48;
            const float d = o[0] - tval[p];
            lv = (double)d * d;
            g[0] = 2.0f * d * wv * inv_nfree;
            float mx = -INFINITY;
            for (int j = 0; j < n_ctrl; ++j) mx = fmaxf(mx, o[1 + j]);
            float sum = 0.0f;
            for (int j = 0; j < n_ctrl; ++j) sum += __expf(o[1 + j] - mx);
            const int tc_ = tctrl[p];
            lc = (double)(logf(sum) + mx - o[1 + tc_]);
            for (int j = 0; j < n_ctrl; ++j) {
                const float pj = __expf(o[1 + j] - mx) / sum;
                g[1 + j] = (pj - (j == tc_ ? 1.0f : 0.0f)) * wc * inv_nfree;
            }
        }
        uint4* dst = reinterpret_cast<uint4*>(dz + (size_t)p * 48);
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            __align__(16) bf16 h[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) h[r] = __float2bfloat16(g[8 * q + r]);
            dst[q] = *reinterpret_cast<const uint4*>(h);
        }
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        lv += __shfl_xor_sync(0xffffffffu, lv, off);
        lc += __shfl_xor_sync(0xffffffffu, lc, off);
    }
    if ((threadIdx.x & 31) == 0 && (lv != 0.0 || lc != 0.0)) {
        atomicAdd(loss, lv);
        atomicAdd(loss + 1, lc);
    }
}

// Adam step on every parameter (bias-corrected moments)
__global__ void k_adam(int n, float* __restrict__ w, const float* __restrict__ g, float* m, float* v,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.0f - b1) * gi;
    const float vi = b2 * v[i] + (1.0f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// value channel of the last layer (x scale) as the coarse initial value of free
// nodes; targets 0, obstacles their held value
__global__ void k_warm_values(const float* __restrict__ out, const uint8_t* __restrict__ mask, int P,
                              float scale, float umax, float uob, float* u0) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= P) return;
    const int mk = mask[k];
    u0[k] = mk == kFree ? fminf(fmaxf(out[(size_t)k * 48] * scale, 0.0f), umax)
                        : (mk == kTarget ? 0.0f : uob);
}

// ----------------------------------------------------------- launch helpers
template <int CIN, int NPAD, bool F32>
cudaError_t conv_impl(const bf16* x, const uint8_t* wpack, const float* bias, int nbias, int relu,
                      const bf16* mask, int total, int H, int W, int dil, void* out, int* err, cudaStream_t st) {
    const size_t smem = (size_t)(128 + NPAD) * 9 * CIN * 2;
    auto kern = k_conv3x3_tc<CIN, NPAD, F32>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    count_launches(1);
    kern<<<(total + 127) / 128, kConvThreads, smem, st>>>(x, wpack, bias, nbias, relu, mask, total, H, W, dil,
                                                          out, err);
    return cudaGetLastError();
}

cudaError_t conv_launch(int cinp, int npad, bool f32, const bf16* x, const uint8_t* wpack, const float* bias,
                        int nbias, int relu, const bf16* mask, int total, int H, int W, int dil, void* out, int* err,
                        cudaStream_t st) {
#define HJB_CONV(C, N)                                                                                              \
    if (cinp == C && npad == N)                                                                                     \
        return f32 ? conv_impl<C, N, true>(x, wpack, bias, nbias, relu, mask, total, H, W, dil, out, err, st)      \
                   : conv_impl<C, N, false>(x, wpack, bias, nbias, relu, mask, total, H, W, dil, out, err, st);
    HJB_CONV(16, 32) HJB_CONV(16, 48) HJB_CONV(32, 32) HJB_CONV(32, 48) HJB_CONV(48, 32) HJB_CONV(48, 48)
#undef HJB_CONV
    return cudaErrorInvalidValue;
}

template <int CIN, int NPAD>
cudaError_t wgrad_impl(const bf16* x, const bf16* dy, int total, int H, int W, int dil, int cout, float* dw,
                       float* db, int* err, cudaStream_t st) {
    if (err) {
        // tensor cores: D = X^T dy accumulated in tensor memory over a chunk of pixels
        using S = WgradShape<CIN, NPAD>;
        auto kern = k_conv3x3_wgrad_tc<CIN, NPAD>;
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)S::smem);
        if (e != cudaSuccess) return e;
        const int chunk = 4096;
        count_launches(1);
        kern<<<(total + chunk - 1) / chunk, kConvThreads, S::smem, st>>>(x, dy, total, H, W, dil, chunk, cout,
                                                                         dw, db, err);
        return cudaGetLastError();
    }
    const size_t smem = (size_t)32 * (NPAD + 9 * CIN) * sizeof(float);
    auto kern = k_conv3x3_wgrad<CIN, NPAD>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    const int chunk = 2048;
    count_launches(1);
    kern<<<(total + chunk - 1) / chunk, 256, smem, st>>>(x, dy, total, H, W, dil, chunk, cout, dw, db);
    return cudaGetLastError();
}

// err != nullptr: the tensor-core kernel (its bounded MMA wait sets *err on
// expiry); nullptr: the FP32 CUDA-core reduction
cudaError_t wgrad_launch(int cinp, int npad, const bf16* x, const bf16* dy, int total, int H, int W, int dil,
                         int cout, float* dw, float* db, int* err, cudaStream_t st) {
#define HJB_WG(C, N) \
    if (cinp == C && npad == N) return wgrad_impl<C, N>(x, dy, total, H, W, dil, cout, dw, db, err, st);
    HJB_WG(16, 32) HJB_WG(16, 48) HJB_WG(32, 32) HJB_WG(32, 48) HJB_WG(48, 32) HJB_WG(48, 48)
#undef HJB_WG
    return cudaErrorInvalidValue;
}

int pad_channels(int c) { return c <= 16 ? 16 : (c <= 32 ? 32 : 48); }
int pad_outputs(int c) { return c <= 32 ? 32 : 48; }

}  // namespace
}  // namespace hjb

// ====================================================================== host
#include "hjb.h"

using namespace hjb;

namespace {

constexpr int kLayers = 6;
constexpr int kCh = 32;          // hidden channels
constexpr int kInCh = 5;         // speed, target, obstacle, sigma, lambda
constexpr int kInPad = 16;
constexpr int kOutCh = 33;       // value + 32 control logits
constexpr int kOutPad = 48;

struct LayerShape {
    int cin, cinp, cout, npad, dil;
};
// dilations 1, 2, ..., 32: the receptive field (127 cells) spans the 129^2 coarse
// grid, so every pixel sees the targets its travel time depends on
constexpr LayerShape kShape[kLayers] = {{kInCh, kInPad, kCh, 32, 1}, {kCh, kCh, kCh, 32, 2},
                                        {kCh, kCh, kCh, 32, 4},      {kCh, kCh, kCh, 32, 8},
                                        {kCh, kCh, kCh, 32, 16},     {kCh, kCh, kOutCh, kOutPad, 32}};

int nfail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_last_error(code, buf);
}

#define NCU(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return nfail(e_ == cudaErrorMemoryAllocation ? HJB_ERR_OOM : HJB_ERR_CUDA,         \
                         "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

// parameter layout: per layer w [cout][9][cinp] then b [cout]
long long layer_wcount(int l) { return (long long)kShape[l].cout * 9 * kShape[l].cinp; }
long long param_offset_w(int l) {
    long long o = 0;
    for (int q = 0; q < l; ++q) o += layer_wcount(q) + kShape[q].cout;
    return o;
}
long long param_offset_b(int l) { return param_offset_w(l) + layer_wcount(l); }
long long param_total() { return param_offset_w(kLayers); }

template <typename T>
void nfree_ptr(T*& p) {
    if (p) cudaFree((void*)p);
    p = nullptr;
}

}  // namespace

struct hjb_net {
    int max_batch = 0, H = 0, W = 0;
    cudaStream_t st = nullptr;
    float* params = nullptr;     // FP32 master parameters
    float* grads = nullptr;
    float* adam_m = nullptr;
    float* adam_v = nullptr;
    uint8_t* wfwd[kLayers] = {};
    uint8_t* wdgr[kLayers] = {};
    bf16* act[kLayers] = {};     // act[l] = input of layer l (act[0] is supplied)
    float* out = nullptr;        // last layer, [B][P][48]
    bf16* dz_last = nullptr;     // [B][P][48]
    bf16* dz[2] = {};            // [B][P][32]
    double* loss = nullptr;
    int* err = nullptr;
    long long step = 0;
};

namespace {

int pack_all(hjb_net* nt) {
    for (int l = 0; l < kLayers; ++l) {
        const LayerShape& L = kShape[l];
        const float* w = nt->params + param_offset_w(l);
        const int nf = L.npad * 9 * L.cinp;
        count_launches(1);
        k_pack_fwd<<<(nf + 255) / 256, 256, 0, nt->st>>>(w, L.cout, L.cinp, L.cinp, L.npad, nt->wfwd[l]);
        if (l > 0) {
            const int nd = 32 * 9 * L.npad;
            count_launches(1);
            k_pack_dgrad<<<(nd + 255) / 256, 256, 0, nt->st>>>(w, L.cout, L.cinp, L.npad, 32, nt->wdgr[l]);
        }
    }
    NCU(cudaGetLastError());
    return HJB_OK;
}

int check_err(hjb_net* nt) {
    int e = 0;
    NCU(cudaMemcpyAsync(&e, nt->err, sizeof(int), cudaMemcpyDeviceToHost, nt->st));
    NCU(cudaStreamSynchronize(nt->st));
    if (e) return nfail(HJB_ERR_TIMEOUT, "tensor-core wait exceeded its limit");
    return HJB_OK;
}

// forward pass of `batch` images whose input (bf16 [B][H][W][16]) is at x
int forward(hjb_net* nt, int batch, const bf16* x) {
    const int total = batch * nt->H * nt->W;
    const bf16* in = x;
    for (int l = 0; l < kLayers; ++l) {
        const LayerShape& L = kShape[l];
        const float* b = nt->params + param_offset_b(l);
        if (l + 1 < kLayers) {
            NCU(conv_launch(L.cinp, L.npad, false, in, nt->wfwd[l], b, L.cout, 1, nullptr, total, nt->H, nt->W,
                            L.dil, nt->act[l + 1], nt->err, nt->st));
            in = nt->act[l + 1];
        } else {
            NCU(conv_launch(L.cinp, L.npad, true, in, nt->wfwd[l], b, L.cout, 0, nullptr, total, nt->H, nt->W,
                            L.dil, nt->out, nt->err, nt->st));
        }
    }
    return HJB_OK;
}

}  // namespace

extern "C" {

long long hjb_net_param_count(void) { return param_total(); }

int hjb_net_create(int32_t max_batch, int32_t height, int32_t width, void* cuda_stream, hjb_net** out) {
    clear_last_error();
    if (!out) return nfail(HJB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (max_batch < 1 || height < 3 || width < 3 || (long long)max_batch * height * width > (1LL << 30))
        return nfail(HJB_ERR_INVALID_ARG, "bad batch / image size");
    hjb_net* nt = new hjb_net();
    nt->max_batch = max_batch;
    nt->H = height;
    nt->W = width;
    nt->st = (cudaStream_t)cuda_stream;
    auto bail = [&](int code) {
        hjb_net_destroy(nt);
        return code;
    };
#define NCUP(call)                                                                             \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return bail(nfail(e_ == cudaErrorMemoryAllocation ? HJB_ERR_OOM : HJB_ERR_CUDA,    \
                              "%s failed: %s", #call, cudaGetErrorString(e_)));                \
    } while (0)
    const size_t np = (size_t)param_total();
    NCUP(cudaMalloc(&nt->params, np * sizeof(float)));
    NCUP(cudaMalloc(&nt->grads, np * sizeof(float)));
    NCUP(cudaMalloc(&nt->adam_m, np * sizeof(float)));
    NCUP(cudaMalloc(&nt->adam_v, np * sizeof(float)));
    NCUP(cudaMemsetAsync(nt->params, 0, np * sizeof(float), nt->st));
    NCUP(cudaMemsetAsync(nt->adam_m, 0, np * sizeof(float), nt->st));
    NCUP(cudaMemsetAsync(nt->adam_v, 0, np * sizeof(float), nt->st));
    const size_t P = (size_t)max_batch * height * width;
    for (int l = 0; l < kLayers; ++l) {
        NCUP(cudaMalloc(&nt->wfwd[l], (size_t)kShape[l].npad * 9 * kShape[l].cinp * 2));
        NCUP(cudaMalloc(&nt->wdgr[l], (size_t)32 * 9 * kShape[l].npad * 2));
        if (l > 0) NCUP(cudaMalloc(&nt->act[l], P * kCh * sizeof(bf16)));
    }
    NCUP(cudaMalloc(&nt->out, P * kOutPad * sizeof(float)));
    NCUP(cudaMalloc(&nt->dz_last, P * kOutPad * sizeof(bf16)));
    NCUP(cudaMalloc(&nt->dz[0], P * kCh * sizeof(bf16)));
    NCUP(cudaMalloc(&nt->dz[1], P * kCh * sizeof(bf16)));
    NCUP(cudaMalloc(&nt->loss, 2 * sizeof(double)));
    NCUP(cudaMalloc(&nt->err, sizeof(int)));
    NCUP(cudaMemsetAsync(nt->err, 0, sizeof(int), nt->st));
    NCUP(cudaStreamSynchronize(nt->st));
#undef NCUP
    *out = nt;
    return HJB_OK;
}

int hjb_net_set_params(hjb_net* nt, const float* params) {
    clear_last_error();
    if (!nt || !params) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    for (long long i = 0; i < param_total(); ++i)
        if (!std::isfinite(params[i])) return nfail(HJB_ERR_INVALID_ARG, "params[%lld] not finite", i);
    NCU(cudaMemcpyAsync(nt->params, params, sizeof(float) * param_total(), cudaMemcpyHostToDevice, nt->st));
    NCU(cudaMemsetAsync(nt->adam_m, 0, sizeof(float) * param_total(), nt->st));
    NCU(cudaMemsetAsync(nt->adam_v, 0, sizeof(float) * param_total(), nt->st));
    nt->step = 0;
    int rc = pack_all(nt);
    if (rc) return rc;
    NCU(cudaStreamSynchronize(nt->st));
    return HJB_OK;
}

int hjb_net_get_params(const hjb_net* nt, float* params) {
    clear_last_error();
    if (!nt || !params) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    NCU(cudaMemcpyAsync(params, nt->params, sizeof(float) * param_total(), cudaMemcpyDeviceToHost, nt->st));
    NCU(cudaStreamSynchronize(nt->st));
    return HJB_OK;
}

int hjb_net_output_device(const hjb_net* nt, const float** out) {
    clear_last_error();
    if (!nt || !out) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    *out = nt->out;
    return HJB_OK;
}

int hjb_net_get_grads(const hjb_net* nt, float* grads) {
    clear_last_error();
    if (!nt || !grads) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    NCU(cudaMemcpyAsync(grads, nt->grads, sizeof(float) * param_total(), cudaMemcpyDeviceToHost, nt->st));
    NCU(cudaStreamSynchronize(nt->st));
    return HJB_OK;
}

int hjb_net_forward(hjb_net* nt, int32_t batch, const void* x, float* out_host) {
    clear_last_error();
    if (!nt || !x) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (batch < 1 || batch > nt->max_batch) return nfail(HJB_ERR_INVALID_ARG, "batch %d out of range", batch);
    int rc = forward(nt, batch, reinterpret_cast<const bf16*>(x));
    if (rc) return rc;
    if (out_host)
        NCU(cudaMemcpyAsync(out_host, nt->out, sizeof(float) * (size_t)batch * nt->H * nt->W * kOutPad,
                            cudaMemcpyDeviceToHost, nt->st));
    return check_err(nt);
}

int hjb_net_train_step(hjb_net* nt, int32_t batch, const void* x, const float* tval, const uint8_t* tctrl,
                       const uint8_t* freem, int64_t n_free, float lr, float w_value, float w_ctrl,
                       double* loss_out) {
    clear_last_error();
    if (!nt || !x || !tval || !tctrl || !freem) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (batch < 1 || batch > nt->max_batch) return nfail(HJB_ERR_INVALID_ARG, "batch %d out of range", batch);
    if (!(lr > 0.0f) || n_free < 1) return nfail(HJB_ERR_INVALID_ARG, "bad lr / n_free");
    const int total = batch * nt->H * nt->W;
    const bf16* x0 = reinterpret_cast<const bf16*>(x);
    int rc = forward(nt, batch, x0);
    if (rc) return rc;
    NCU(cudaMemsetAsync(nt->loss, 0, 2 * sizeof(double), nt->st));
    count_launches(1);
    k_loss<<<(total + 255) / 256, 256, 0, nt->st>>>(nt->out, tval, tctrl, freem, total, 32, w_value, w_ctrl,
                                                     1.0f / (float)n_free, nt->dz_last, nt->loss);
    NCU(cudaGetLastError());
    NCU(cudaMemsetAsync(nt->grads, 0, sizeof(float) * param_total(), nt->st));
    // backward: layer 5 .. 0
    const bf16* dzl = nt->dz_last;
    for (int l = kLayers - 1; l >= 0; --l) {
        const LayerShape& L = kShape[l];
        const bf16* xin = l == 0 ? x0 : nt->act[l];
        NCU(wgrad_launch(L.cinp, L.npad, xin, dzl, total, nt->H, nt->W, L.dil, L.cout,
                         nt->grads + param_offset_w(l), nt->grads + param_offset_b(l), nt->err, nt->st));
        if (l > 0) {
            bf16* dnext = nt->dz[l & 1];
            NCU(conv_launch(L.npad, 32, false, dzl, nt->wdgr[l], nullptr, 0, 0, nt->act[l], total, nt->H,
                            nt->W, L.dil, dnext, nt->err, nt->st));
            dzl = dnext;
        }
    }
    ++nt->step;
    const float b1 = 0.9f, b2 = 0.999f;
    const float c1 = 1.0f - std::pow(b1, (float)nt->step), c2 = 1.0f - std::pow(b2, (float)nt->step);
    const int np = (int)param_total();
    count_launches(1);
    k_adam<<<(np + 255) / 256, 256, 0, nt->st>>>(np, nt->params, nt->grads, nt->adam_m, nt->adam_v, lr, b1, b2,
                                                  1e-8f, c1, c2);
    NCU(cudaGetLastError());
    rc = pack_all(nt);
    if (rc) return rc;
    if (loss_out) {
        double h[2];
        NCU(cudaMemcpyAsync(h, nt->loss, sizeof(h), cudaMemcpyDeviceToHost, nt->st));
        NCU(cudaStreamSynchronize(nt->st));
        loss_out[0] = h[0] / (double)n_free;
        loss_out[1] = h[1] / (double)n_free;
    }
    return check_err(nt);
}

int hjb_net_warm_values(hjb_net* nt, int32_t index, const uint8_t* mask, float scale, float umax, float uob,
                        float* u0) {
    clear_last_error();
    if (!nt || !mask || !u0) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (index < 0 || index >= nt->max_batch) return nfail(HJB_ERR_INVALID_ARG, "index out of range");
    const int P = nt->H * nt->W;
    count_launches(1);
    k_warm_values<<<(P + 255) / 256, 256, 0, nt->st>>>(nt->out + (size_t)index * P * kOutPad, mask, P, scale,
                                                        umax, uob, u0);
    NCU(cudaGetLastError());
    return HJB_OK;
}

void hjb_net_destroy(hjb_net* nt) {
    if (!nt) return;
    if (nt->st) cudaStreamSynchronize(nt->st);
    else cudaDeviceSynchronize();
    nfree_ptr(nt->params); nfree_ptr(nt->grads); nfree_ptr(nt->adam_m); nfree_ptr(nt->adam_v);
    for (int l = 0; l < kLayers; ++l) {
        nfree_ptr(nt->wfwd[l]);
        nfree_ptr(nt->wdgr[l]);
        nfree_ptr(nt->act[l]);
    }
    nfree_ptr(nt->out); nfree_ptr(nt->dz_last); nfree_ptr(nt->dz[0]); nfree_ptr(nt->dz[1]);
    nfree_ptr(nt->loss); nfree_ptr(nt->err);
    delete nt;
}

// ----------------------------------------------------- single layers (tests)
namespace {
struct LayerBufs {
    bf16* x = nullptr;
    bf16* y = nullptr;
    bf16* mask = nullptr;
    float* w = nullptr;
    float* b = nullptr;
    uint8_t* wp = nullptr;
    float* out = nullptr;
    int* err = nullptr;
    ~LayerBufs() {
        nfree_ptr(x); nfree_ptr(y); nfree_ptr(mask); nfree_ptr(w); nfree_ptr(b); nfree_ptr(wp);
        nfree_ptr(out); nfree_ptr(err);
    }
};

// host [P][c] bf16 bits -> device [P][cp] (zero channels c..cp-1)
int upload_padded(const uint16_t* h, long long P, int c, int cp, bf16** d) {
    std::vector<uint16_t> buf((size_t)P * cp, 0);
    for (long long p = 0; p < P; ++p)
        for (int q = 0; q < c; ++q) buf[(size_t)p * cp + q] = h[(size_t)p * c + q];
    NCU(cudaMalloc(d, buf.size() * 2));
    NCU(cudaMemcpy(*d, buf.data(), buf.size() * 2, cudaMemcpyHostToDevice));
    return HJB_OK;
}

int check_layer_args(int batch, int H, int W, int cin, int cout) {
    if (batch < 1 || H < 1 || W < 1 || (long long)batch * H * W > (1LL << 28))
        return nfail(HJB_ERR_INVALID_ARG, "bad batch / image size");
    if (cin < 1 || cin > 48 || cout < 1 || cout > 48) return nfail(HJB_ERR_INVALID_ARG, "cin, cout must be 1..48");
    return HJB_OK;
}
int check_dil(int dil) {
    if (dil < 1 || dil > 1024) return nfail(HJB_ERR_INVALID_ARG, "dilation must be 1..1024");
    return HJB_OK;
}
}  // namespace

int hjb_conv3x3_forward(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dil,
                        const uint16_t* x, const float* w, const float* b, int32_t relu, float* y) {
    clear_last_error();
    if (!x || !w || !y) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    int rc = check_layer_args(batch, H, W, cin, cout);
    if (!rc) rc = check_dil(dil);
    if (rc) return rc;
    const long long P = (long long)batch * H * W;
    const int cinp = pad_channels(cin), npad = pad_outputs(cout);
    LayerBufs B;
    rc = upload_padded(x, P, cin, cinp, &B.x);
    if (rc) return rc;
    NCU(cudaMalloc(&B.w, sizeof(float) * cout * 9 * cin));
    NCU(cudaMemcpy(B.w, w, sizeof(float) * cout * 9 * cin, cudaMemcpyHostToDevice));
    std::vector<float> hb(npad, 0.0f);
    if (b) std::copy(b, b + cout, hb.begin());
    NCU(cudaMalloc(&B.b, sizeof(float) * npad));
    NCU(cudaMemcpy(B.b, hb.data(), sizeof(float) * npad, cudaMemcpyHostToDevice));
    NCU(cudaMalloc(&B.wp, (size_t)npad * 9 * cinp * 2));
    NCU(cudaMalloc(&B.out, sizeof(float) * P * npad));
    NCU(cudaMalloc(&B.err, sizeof(int)));
    NCU(cudaMemset(B.err, 0, sizeof(int)));
    count_launches(1);
    k_pack_fwd<<<(npad * 9 * cinp + 255) / 256, 256>>>(B.w, cout, cin, cinp, npad, B.wp);
    NCU(cudaGetLastError());
    NCU(conv_launch(cinp, npad, true, B.x, B.wp, B.b, cout, relu, nullptr, (int)P, H, W, dil, B.out, B.err,
                    nullptr));
    std::vector<float> h((size_t)P * npad);
    NCU(cudaMemcpy(h.data(), B.out, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
    int e = 0;
    NCU(cudaMemcpy(&e, B.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) return nfail(HJB_ERR_TIMEOUT, "tensor-core wait exceeded its limit");
    for (long long p = 0; p < P; ++p)
        for (int q = 0; q < cout; ++q) y[(size_t)p * cout + q] = h[(size_t)p * npad + q];
    return HJB_OK;
}

int hjb_conv3x3_dgrad(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dil,
                      const uint16_t* dy, const float* w, const uint16_t* mask, float* dx) {
    clear_last_error();
    if (!dy || !w || !dx) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    int rc = check_layer_args(batch, H, W, cin, cout);
    if (!rc) rc = check_dil(dil);
    if (rc) return rc;
    const long long P = (long long)batch * H * W;
    const int coutp = pad_channels(cout), npad = pad_outputs(cin);
    LayerBufs B;
    rc = upload_padded(dy, P, cout, coutp, &B.x);
    if (rc) return rc;
    if (mask) {
        rc = upload_padded(mask, P, cin, npad, &B.mask);
        if (rc) return rc;
    }
    NCU(cudaMalloc(&B.w, sizeof(float) * cout * 9 * cin));
    NCU(cudaMemcpy(B.w, w, sizeof(float) * cout * 9 * cin, cudaMemcpyHostToDevice));
    NCU(cudaMalloc(&B.wp, (size_t)npad * 9 * coutp * 2));
    NCU(cudaMalloc(&B.out, sizeof(float) * P * npad));
    NCU(cudaMalloc(&B.err, sizeof(int)));
    NCU(cudaMemset(B.err, 0, sizeof(int)));
    count_launches(1);
    k_pack_dgrad<<<(npad * 9 * coutp + 255) / 256, 256>>>(B.w, cout, cin, coutp, npad, B.wp);
    NCU(cudaGetLastError());
    NCU(conv_launch(coutp, npad, true, B.x, B.wp, nullptr, 0, 0, B.mask, (int)P, H, W, dil, B.out, B.err,
                    nullptr));
    std::vector<float> h((size_t)P * npad);
    NCU(cudaMemcpy(h.data(), B.out, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
    int e = 0;
    NCU(cudaMemcpy(&e, B.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) return nfail(HJB_ERR_TIMEOUT, "tensor-core wait exceeded its limit");
    for (long long p = 0; p < P; ++p)
        for (int q = 0; q < cin; ++q) dx[(size_t)p * cin + q] = h[(size_t)p * npad + q];
    return HJB_OK;
}

int hjb_conv3x3_wgrad(int32_t batch, int32_t H, int32_t W, int32_t cin, int32_t cout, int32_t dil,
                      const uint16_t* x, const uint16_t* dy, float* dw, float* db) {
    clear_last_error();
    if (!x || !dy || !dw) return nfail(HJB_ERR_INVALID_ARG, "NULL argument");
    int rc = check_layer_args(batch, H, W, cin, cout);
    if (!rc) rc = check_dil(dil);
    if (rc) return rc;
    const long long P = (long long)batch * H * W;
    const int cinp = pad_channels(cin), npad = pad_outputs(cout);
    LayerBufs B;
    rc = upload_padded(x, P, cin, cinp, &B.x);
    if (rc) return rc;
    rc = upload_padded(dy, P, cout, npad, &B.y);
    if (rc) return rc;
    NCU(cudaMalloc(&B.w, sizeof(float) * cout * 9 * cinp));
    NCU(cudaMalloc(&B.b, sizeof(float) * cout));
    NCU(cudaMemset(B.w, 0, sizeof(float) * cout * 9 * cinp));
    NCU(cudaMemset(B.b, 0, sizeof(float) * cout));
    NCU(cudaMalloc(&B.err, sizeof(int)));
    NCU(cudaMemset(B.err, 0, sizeof(int)));
    NCU(wgrad_launch(cinp, npad, B.x, B.y, (int)P, H, W, dil, cout, B.w, B.b, B.err, nullptr));
    std::vector<float> h((size_t)cout * 9 * cinp);
    NCU(cudaMemcpy(h.data(), B.w, h.size() * sizeof(float), cudaMemcpyDeviceToHost));
    int e = 0;
    NCU(cudaMemcpy(&e, B.err, sizeof(int), cudaMemcpyDeviceToHost));
    if (e) return nfail(HJB_ERR_TIMEOUT, "tensor-core wait exceeded its limit");
    for (int n = 0; n < cout; ++n)
        for (int t = 0; t < 9; ++t)
            for (int q = 0; q < cin; ++q) dw[((size_t)n * 9 + t) * cin + q] = h[((size_t)n * 9 + t) * cinp + q];
    if (db) NCU(cudaMemcpy(db, B.b, sizeof(float) * cout, cudaMemcpyDeviceToHost));
    return HJB_OK;
}

}  // extern "C"
