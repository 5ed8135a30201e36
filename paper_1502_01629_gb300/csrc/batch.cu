// Batched patchy solve: many independent problems (their own grid size, speed,
// targets, obstacles, sigma, lambda, coarse grid and patch count; one control
// set) carried through the pre-computation and the patch solve of Section 4.3
// (Cacace & Falcone) together.  Every stage is one launch over all instances:
//   * element-wise stages (coarse data, interpolation, synthesis, successors,
//     labels) run over the concatenated node arrays with a block -> (instance,
//     first node) table, each block inside one instance;
//   * the coarse solves (sigma = 0) run one thread block per instance with the
//     whole coarse field in shared memory (no grid-wide waits);
//   * the patch solve is the warp-tile kernel over the tiles of every
//     instance (a tile -> instance table; waves, queues and the grid barrier
//     are shared, so a step carries the fronts of all instances at once);
//   * the FP64 residual is one launch over the 32x16 tiles of all instances,
//     with a per-instance maximum.
// The plain full-grid Jacobi comparator is batched the same way.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "hjb_kernels.h"
#include "precompute_device.cuh"
#include "sweep_device.cuh"

namespace hjb {

// Per-instance data of the batched stages (device copy).
struct BatchInst {
    GridView g;          // fine grid (pointers into the concatenated arrays)
    GridView gc;         // coarse grid: sigma = 0, h_c = h r
    float* uhat;
    float* uc;
    float* speed_c;
    uint8_t* mask_c;
    uint8_t* a;
    int32_t* key;
    const int8_t* sector;
    int8_t* label;
    long long node_off;  // first node of the instance in the concatenated arrays
    int nc;
    int n_patches;
    int R;               // halo of the fine operator
    float lambda;        // band map
    float band_w;
    BandMap bm;          // exact band keys (edges into the batch's edge array)
    float uc0;           // coarse initial value on free nodes: l/lambda + h_c l
    float uob32;         // value held on obstacle nodes
    float sigma;
    double uob64;
};

namespace {

constexpr int kBT = 256;        // element-wise block size
constexpr int kCoarseThreads = 1024;
constexpr int kRX = 32, kRY = 16, kRBY = 8;   // residual / Jacobi tiles

// ------------------------------------------------------ element-wise stages
__global__ void k_b_coarse_data(const BatchInst* __restrict__ I, const int2* __restrict__ blk) {
    const int2 bl = blk[blockIdx.x];
    const BatchInst& B = I[bl.x];
    const int kc = bl.y + threadIdx.x;
    if (kc >= B.nc * B.nc) return;
    coarse_data_node(kc, B.g.n, B.nc, B.g.speed, nullptr, B.g.mask, B.speed_c, nullptr, B.mask_c);
}

__global__ void k_b_interp(const BatchInst* __restrict__ I, const int2* __restrict__ blk) {
    const int2 bl = blk[blockIdx.x];
    const BatchInst& B = I[bl.x];
    const int k = bl.y + threadIdx.x;
    if (k >= B.g.n * B.g.n) return;
    B.uhat[k] = interp_node(k, B.nc, B.uc, B.g.n, B.g.mask, B.uob32);
}

// synthesis a*, band key, per-instance largest key
__global__ void k_b_synthesis(const BatchInst* __restrict__ I, const int2* __restrict__ blk,
                              int band_cap, int* max_key) {
    extern __shared__ __align__(16) unsigned char smem[];
    float2* sctrl = reinterpret_cast<float2*>(smem);
    const int2 bl = blk[blockIdx.x];
    const BatchInst& B = I[bl.x];
    const GridView& g = B.g;
    for (int m = threadIdx.x; m < g.na; m += blockDim.x) sctrl[m] = g.ctrl32[m];
    __syncthreads();
    const int k = bl.y + threadIdx.x;
    int kk = -1;
    if (k < g.n * g.n) {
        if (g.mask[k] != kFree) {
            B.a[k] = 255;
            B.key[k] = -1;
        } else {
            auto C = [&](int m) { return sctrl[m]; };
            B.a[k] = (uint8_t)synthesis_node(g, k, B.uhat, C);
            kk = band_key(B.uhat[k], B.bm);
            B.key[k] = kk;
        }
    }
    int wm = kk;
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) wm = max(wm, __shfl_xor_sync(0xffffffffu, wm, off));
    if ((threadIdx.x & 31) == 0 && wm >= 0) atomicMax(max_key + bl.x, wm);
}

// network input of each instance's coarse grid (bf16 [count][nc][nc][16]):
// speed / 2, target indicator, obstacle indicator, 10 sigma, lambda / 2, zeros
__global__ void k_b_net_inputs(const BatchInst* __restrict__ I, const int2* __restrict__ blk, int nc,
                               __nv_bfloat16* x) {
    const int2 bl = blk[blockIdx.x];
    const BatchInst& B = I[bl.x];
    const int k = bl.y + threadIdx.x;
    if (k >= B.nc * B.nc) return;
    const int mk = B.mask_c[k];
    float v[16] = {};
    v[0] = 0.5f * B.speed_c[k];
    v[1] = mk == kTarget ? 1.0f : 0.0f;
    v[2] = mk == kObstacle ? 1.0f : 0.0f;
    v[3] = 10.0f * B.sigma;
    v[4] = 0.5f * B.lambda;
    __nv_bfloat16* o = x + ((size_t)bl.x * nc * nc + k) * 16;
    for (int c = 0; c < 16; ++c) o[c] = __float2bfloat16(v[c]);
}

// training targets at each instance's coarse nodes: u_c / u_max, the feedback
// control a* of the fine node (rI, rJ), and 1 on free coarse nodes
__global__ void k_b_net_targets(const BatchInst* __restrict__ I, const int2* __restrict__ blk, int nc,
                                float* tval, uint8_t* tctrl, uint8_t* freem) {
    const int2 bl = blk[blockIdx.x];
    const BatchInst& B = I[bl.x];
    const int k = bl.y + threadIdx.x;
    if (k >= B.nc * B.nc) return;
    const int n = B.g.n;
    const int r = (n - 1) / (B.nc - 1);
    const int ci = k % B.nc, cj = k / B.nc;
    const size_t o = (size_t)bl.x * nc * nc + k;
    const bool fr = B.mask_c[k] == kFree;
    const int a = B.a[(size_t)(r * cj) * n + r * ci];
    tval[o] = B.uc[k] / B.uc0;
    tctrl[o] = (fr && a < 255) ? (uint8_t)a : 0;
    freem[o] = (fr && a < 255) ? 1 : 0;
}

// coarse initial values from the network output (FP32 [count][nc][nc][48], value
// channel 0 = u / u_max): clamp(o0 * u_max, 0, u_max) on free nodes
__global__ void k_b_warm_values(const BatchInst* __restrict__ I, const int2* __restrict__ blk, int nc,
                                const float* __restrict__ out, int first, int count,
                                const long long* __restrict__ coarse_off, float* init) {
    const int2 bl = blk[blockIdx.x];
    if (bl.x < first || bl.x >= first + count) return;
    const BatchInst& B = I[bl.x];
    const int k = bl.y + threadIdx.x;
    if (k >= B.nc * B.nc) return;
    const float um = B.uc0;
    const float v = out[((size_t)(bl.x - first) * nc * nc + k) * 48] * um;
    init[coarse_off[bl.x] + k] = fminf(fmaxf(v, 0.0f), um);
}

// successors as indices of the concatenated arrays
__global__ void k_b_successors(const BatchInst* __restrict__ I, const int2* __restrict__ blk,
                               int32_t* succ) {
    const int2 bl = blk[blockIdx.x];
    const BatchInst& B = I[bl.x];
    const int k = bl.y + threadIdx.x;
    if (k >= B.g.n * B.g.n) return;
    const int32_t loc = B.g.mask[k] != kFree ? k : successor_node(B.g, k, B.a[k]);
    succ[B.node_off + k] = (int32_t)(B.node_off + loc);
}

// label of the chain's end (global index): its sector on a target, else N_P
__global__ void k_b_labels(const BatchInst* __restrict__ I, const int2* __restrict__ blk,
                           const int32_t* __restrict__ end, const uint8_t* __restrict__ mask_all,
                           const int8_t* __restrict__ sector_all) {
    const int2 bl = blk[blockIdx.x];
    const BatchInst& B = I[bl.x];
    const int k = bl.y + threadIdx.x;
    if (k >= B.g.n * B.g.n) return;
    const int t = end[B.node_off + k];
    int8_t lab = (int8_t)B.n_patches;
    if (mask_all[t] == kTarget && sector_all[t] >= 0) lab = sector_all[t];
    B.label[k] = lab;
}

// ------------------------------------------------------------ coarse solves
// One block per instance (largest first): the coarse field lives in shared
// memory; each sweep updates every free coarse node in place (one warp per
// node, lanes over the controls, SLscheme3 with sigma = 0) and ends with a
// block barrier; stops when a sweep's sup-increment is <= tol.
// With a warm start (init != nullptr) free nodes start from init (the
// instance's slice of the concatenated coarse arrays) and the solve stops after
// k_warm sweeps when the last sweep changed no node by more than tol_fb (the
// refined prediction is accepted as the coarse value); otherwise the free nodes
// restart from the plain initial value, the solve runs to tol and fallback[b]
// is set.
__global__ void __launch_bounds__(kCoarseThreads)
k_b_coarse_solve(const BatchInst* __restrict__ I, const int* __restrict__ order, float tol,
                 int max_sweeps, int* sweeps_out, float* inc_out, const float* __restrict__ init,
                 const long long* __restrict__ coarse_off, int k_warm, float tol_fb, uint8_t* fallback) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int b = order[blockIdx.x];
    const BatchInst& B = I[b];
    const GridView& g = B.gc;
    const int nc = g.n;
    const int Nc = nc * nc;
    float2* sctrl = reinterpret_cast<float2*>(smem);
    const size_t cb = ((size_t)g.na * sizeof(float2) + 15) & ~(size_t)15;
    float* su = reinterpret_cast<float*>(smem + cb);
    __shared__ float red[32];
    __shared__ int s_done;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    for (int m = threadIdx.x; m < g.na; m += blockDim.x) sctrl[m] = g.ctrl32[m];
    const float* ini = init ? init + coarse_off[b] : nullptr;
    for (int k = threadIdx.x; k < Nc; k += blockDim.x) {
        const int mk = g.mask[k];
        su[k] = mk == kFree ? (ini ? ini[k] : B.uc0) : (mk == kTarget ? 0.0f : g.uob32);
    }
    __syncthreads();
    bool fell_back = false;
    auto C = [&](int m) { return sctrl[m]; };
    // a tolerance below half an FP32 ulp of the largest value could stall
    tol = fmaxf(tol, 1.01f * ldexpf(fmaxf(1.0f, B.uc0), -23));
    int sweep = 0;
    float last = 0.0f;
    for (sweep = 0; sweep < max_sweeps;) {
        float wmax = 0.0f;
        for (int k = warp; k < Nc; k += nwarps) {
            if (g.mask[k] != kFree) continue;
            const int i = k % nc, j = k / nc;
            float* base = su + k;
            const float uk = base[0];
            auto U = [&](int dx, int dy) { return base[dy * nc + dx]; };
            float N, D;
            int M;
            best_over_controls<float, false, true>(g, 3, i, j, uk, g.speed[k], 0.0f, 0.0f, lane, 32,
                                                   C, U, N, D, M);
            const float du = warp_min_increment(N, D, M);
            if (lane == 0) base[0] = uk + du;
            wmax = fmaxf(wmax, fabsf(du));
        }
        const float bm = block_max<float>(wmax, red);
        ++sweep;
        if (threadIdx.x == 0) {
            last = bm;
            s_done = bm <= tol ? 1 : 0;
            if (ini && !fell_back && sweep == k_warm && !s_done) s_done = bm <= tol_fb ? 1 : 2;
        }
        __syncthreads();
        if (s_done == 1) break;
        if (s_done == 2) {
            // the prediction is too far off: the plain initial value instead
            fell_back = true;
            for (int k = threadIdx.x; k < Nc; k += blockDim.x)
                if (g.mask[k] == kFree) su[k] = B.uc0;
            __syncthreads();
        }
    }
    for (int k = threadIdx.x; k < Nc; k += blockDim.x) B.uc[k] = su[k];
    if (threadIdx.x == 0) {
        sweeps_out[b] = sweep;
        inc_out[b] = last;
        if (fallback) fallback[b] = fell_back ? 1 : 0;
    }
}

// --------------------------------------------------- residual and Jacobi
// Block = one 32x16 tile of one instance: rblk = (instance, tile x, tile y).
template <bool SIG>
__global__ void __launch_bounds__(kRX * kRBY)
k_b_residual(const BatchInst* __restrict__ I, const int4* __restrict__ rblk,
             const double* __restrict__ u_all, const float* __restrict__ margin,
             const uint8_t* __restrict__ active, unsigned long long* res_bits,
             float* __restrict__ rfield, uint8_t* __restrict__ afield) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 bl = rblk[blockIdx.x];
    if (active && !active[bl.x]) return;
    const BatchInst& B = I[bl.x];
    const GridView& g = B.g;
    double2* c64 = reinterpret_cast<double2*>(smem);
    const size_t cb64 = ((size_t)g.na * sizeof(double2) + 15) & ~(size_t)15;
    float2* c32 = reinterpret_cast<float2*>(smem + cb64);
    const size_t cb32 = ((size_t)g.na * sizeof(float2) + 15) & ~(size_t)15;
    const int n = g.n;
    const int R = B.R;
    const int W = kRX + 2 * R;
    const int H = kRY + 2 * R;
    double* t64 = reinterpret_cast<double*>(smem + cb64 + cb32);
    float* t32 = reinterpret_cast<float*>(t64 + (size_t)W * H);
    __shared__ double red[32];
    const double* u = u_all + B.node_off;
    const int gx0 = bl.y * kRX - R;
    const int gy0 = bl.z * kRY - R;
    const int tid = threadIdx.y * kRX + threadIdx.x;
    const int nthreads = kRX * kRBY;
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
    for (int r = 0; r < kRY / kRBY; ++r) {
        const int i = bl.y * kRX + threadIdx.x;
        const int j = bl.z * kRY + threadIdx.y + r * kRBY;
        if (i >= n || j >= n) continue;
        const size_t k = (size_t)j * n + i;
        if (g.mask[k] != kFree) {
            if (rfield) {
                rfield[B.node_off + k] = 0.0f;
                afield[B.node_off + k] = 0;
            }
            continue;
        }
        const int off = (j - gy0) * W + (i - gx0);
        if (rfield) {
            // the residual r = T2 u - u and its minimising control, for the
            // correction rounds of the FP64 stage
            double v;
            int m;
            lmax = fmax(lmax, residual_node<SIG>(g, i, j, k, t32, t64, off, W, c32, c64, margin[bl.x], &v, &m));
            rfield[B.node_off + k] = (float)v;
            afield[B.node_off + k] = (uint8_t)m;
        } else {
            lmax = fmax(lmax, residual_node<SIG>(g, i, j, k, t32, t64, off, W, c32, c64, margin[bl.x]));
        }
    }
    const double bm = block_max<double>(lmax, red);
    if (tid == 0) atomic_max_nonneg(res_bits + bl.x, bm);
}

// One plain Jacobi sweep uout = T uin over the tiles of the active instances;
// per-instance sup-increment (float bits) in inc_bits.
template <bool SIG>
__global__ void __launch_bounds__(kRX * kRBY)
k_b_jacobi(const BatchInst* __restrict__ I, const int4* __restrict__ rblk, int scheme,
           const float* __restrict__ uin_all, float* __restrict__ uout_all,
           const uint8_t* __restrict__ active, unsigned int* inc_bits) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 bl = rblk[blockIdx.x];
    if (!active[bl.x]) return;
    const BatchInst& B = I[bl.x];
    const GridView& g = B.g;
    float2* sctrl = reinterpret_cast<float2*>(smem);
    const size_t cb = ((size_t)g.na * sizeof(float2) + 15) & ~(size_t)15;
    float* tile = reinterpret_cast<float*>(smem + cb);
    __shared__ float red[32];
    const int n = g.n;
    const int R = B.R;
    const int W = kRX + 2 * R;
    const int H = kRY + 2 * R;
    const float* uin = uin_all + B.node_off;
    float* uout = uout_all + B.node_off;
    const int gx0 = bl.y * kRX - R;
    const int gy0 = bl.z * kRY - R;
    const int tid = threadIdx.y * kRX + threadIdx.x;
    const int nthreads = kRX * kRBY;
    for (int m = tid; m < g.na; m += nthreads) sctrl[m] = g.ctrl32[m];
    for (int t = tid; t < W * H; t += nthreads) {
        const int ty = t / W;
        const int tx = t - ty * W;
        const int gx = min(max(gx0 + tx, 0), n - 1);
        const int gy = min(max(gy0 + ty, 0), n - 1);
        tile[t] = uin[(size_t)gy * n + gx];
    }
    __syncthreads();
    const bool interior = gx0 >= 0 && gy0 >= 0 && gx0 + W <= n && gy0 + H <= n;
    auto C = [&](int m) { return sctrl[m]; };
    float lmax = 0.0f;
    for (int r = 0; r < kRY / kRBY; ++r) {
        const int i = bl.y * kRX + threadIdx.x;
        const int j = bl.z * kRY + threadIdx.y + r * kRBY;
        if (i >= n || j >= n) continue;
        const size_t k = (size_t)j * n + i;
        const float* base = tile + (j - gy0) * W + (i - gx0);
        float out = base[0];
        if (g.mask[k] == kFree) {
            int M;
            const float du = interior
                                 ? node_increment<float, SIG, false>(g, scheme, i, j, k, base, W, C, M)
                                 : node_increment<float, SIG, true>(g, scheme, i, j, k, base, W, C, M);
            out = base[0] + du;
            lmax = fmaxf(lmax, fabsf(du));
        }
        uout[k] = out;
    }
    const float bm = block_max<float>(lmax, red);
    if (tid == 0 && bm > 0.0f) atomicMax(inc_bits + bl.x, __float_as_uint(bm));
}

// After a Jacobi sweep: instances whose sup-increment is <= tol stop; their
// sweep count is recorded (its parity tells which buffer holds the result).
__global__ void k_b_jacobi_mark(int count, float tol, int sweep, uint8_t* active,
                                unsigned int* inc_bits, int* sweeps, int* n_active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count || !active[b]) return;
    const float inc = __uint_as_float(inc_bits[b]);
    inc_bits[b] = 0u;
    if (inc <= tol) {
        active[b] = 0;
        sweeps[b] = sweep;
    } else {
        atomicAdd(n_active, 1);
    }
}

// One Jacobi sweep of the correction equation e = beta P_a e + r of the FP64
// stage (the residual r = T2 u - u and its minimising control a per node, from
// k_b_residual with fields) over the tiles of the active instances, in the
// self-weight-free form of eq. SLscheme3 (one control per node); per-instance
// sup-increment in inc_bits.  Non-free nodes hold e = 0.
template <bool SIG>
__global__ void __launch_bounds__(kRX * kRBY)
k_b_corr_sweep(const BatchInst* __restrict__ I, const int4* __restrict__ rblk,
               const float* __restrict__ r_all, const uint8_t* __restrict__ a_all,
               const float* __restrict__ ein_all, float* __restrict__ eout_all,
               const uint8_t* __restrict__ active, unsigned int* inc_bits) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int4 bl = rblk[blockIdx.x];
    if (!active[bl.x]) return;
    const BatchInst& B = I[bl.x];
    const GridView& g = B.g;
    float* tile = reinterpret_cast<float*>(smem);
    __shared__ float red[32];
    const int n = g.n;
    const int R = B.R;
    const int W = kRX + 2 * R;
    const int H = kRY + 2 * R;
    const float* ein = ein_all + B.node_off;
    float* eout = eout_all + B.node_off;
    const float* r = r_all + B.node_off;
    const uint8_t* act = a_all + B.node_off;
    const int gx0 = bl.y * kRX - R;
    const int gy0 = bl.z * kRY - R;
    const int tid = threadIdx.y * kRX + threadIdx.x;
    for (int t = tid; t < W * H; t += kRX * kRBY) {
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
    for (int rr = 0; rr < kRY / kRBY; ++rr) {
        const int i = bl.y * kRX + threadIdx.x;
        const int j = bl.z * kRY + threadIdx.y + rr * kRBY;
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
            const float2 b2 = g.drift[k];
            bx = b2.x;
            by = b2.y;
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
    if (tid == 0 && bm > 0.0f) atomicMax(inc_bits + bl.x, __float_as_uint(bm));
}

// After a correction sweep: instances whose sup-increment is <= their own
// tolerance stop (sweep count recorded: its parity tells the buffer).
__global__ void k_b_corr_mark(int count, const float* __restrict__ tol, int sweep, uint8_t* active,
                              unsigned int* inc_bits, int* sweeps, int* n_active) {
    const int b = blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= count || !active[b]) return;
    const float inc = __uint_as_float(inc_bits[b]);
    inc_bits[b] = 0u;
    if (inc <= tol[b]) {
        active[b] = 0;
        sweeps[b] = sweep;
    } else {
        atomicAdd(n_active, 1);
    }
}

// u64 += e on the free nodes of the instances flagged in `sel` (e from buffer a
// or b by the parity of the instance's sweep count)
__global__ void k_b_add_corr(const BatchInst* __restrict__ I, const int2* __restrict__ blk,
                             const float* __restrict__ ea, const float* __restrict__ eb,
                             const int* __restrict__ sweeps, const uint8_t* __restrict__ sel, double* u64) {
    const int2 bl = blk[blockIdx.x];
    if (!sel[bl.x]) return;
    const BatchInst& B = I[bl.x];
    const int k = bl.y + threadIdx.x;
    if (k >= B.g.n * B.g.n || B.g.mask[k] != kFree) return;
    const float* src = (sweeps[bl.x] & 1) ? eb : ea;
    u64[B.node_off + k] += (double)src[B.node_off + k];
}

// u64 = u (FP32 result of each instance, from buffer a or b by the parity of
// its sweep count when `sweeps` is given)
__global__ void k_b_promote(const BatchInst* __restrict__ I, const int2* __restrict__ blk,
                            const float* __restrict__ ua, const float* __restrict__ ub,
                            const int* __restrict__ sweeps, double* u64) {
    const int2 bl = blk[blockIdx.x];
    const BatchInst& B = I[bl.x];
    const int k = bl.y + threadIdx.x;
    if (k >= B.g.n * B.g.n) return;
    const float* src = (sweeps && (sweeps[bl.x] & 1)) ? ub : ua;
    const int mk = B.g.mask[k];
    // exact FP64 held values on non-free nodes (their FP32 rounding would move
    // the FP64 fixed point)
    u64[B.node_off + k] = mk == kFree ? (double)src[B.node_off + k] : (mk == kTarget ? 0.0 : B.uob64);
}

// Jacobi start: u = 0 on free and target nodes, the obstacle value elsewhere.
__global__ void k_b_init_zero(const BatchInst* __restrict__ I, const int2* __restrict__ blk, float* ua,
                              float* ub) {
    const int2 bl = blk[blockIdx.x];
    const BatchInst& B = I[bl.x];
    const int k = bl.y + threadIdx.x;
    if (k >= B.g.n * B.g.n) return;
    const float v = B.g.mask[k] == kObstacle ? B.uob32 : 0.0f;
    ua[B.node_off + k] = v;
    ub[B.node_off + k] = v;
}

}  // namespace
}  // namespace hjb

// ====================================================================== host
#include "hjb.h"

using namespace hjb;

struct hjb_batch {
    GraphCache pre_graph;        // the pre-computation sequence (fixed buffers)
    InputScan* scan_tmp = nullptr;   // creation-time input scan records
    int count = 0;
    int na = 0;
    int scheme = 3;
    bool ctrl_sym32 = false;     // 32 controls in opposite pairs (two-node visits)
    bool ctrl_rot32 = false;     // and closed under quarter turns (four-node visits)
    int D = 2;
    int shape = 2;               // warp-tile shape code: 1 8x8, 2 8x4, 3 4x4
    int B = 2;                   // bands per tile wave
    double cost = 1.0;
    double band_width = 1.0;
    bool any_sigma = false;
    int num_sms = 0;
    cudaStream_t st = nullptr;
    bool own_stream = false;
    std::vector<hjb_batch_inst> desc;
    std::vector<long long> node_off;     // count + 1
    std::vector<long long> coarse_off;   // count + 1
    std::vector<double> uob;             // per instance
    long long N = 0, Nc = 0;
    std::vector<BatchInst> hinst;
    BatchInst* dinst = nullptr;
    std::vector<TileInst> htile;
    TileInst* dtile = nullptr;
    // concatenated node arrays
    float* speed = nullptr;
    uint8_t* mask = nullptr;
    int8_t* sector = nullptr;
    float* u32 = nullptr;
    float* u32b = nullptr;
    double* u64 = nullptr;
    double* band_e = nullptr;            // every instance's band edges, concatenated
    int sched_mode = 0;                  // hjb_batch_desc.schedule (0, 3, 4)
    bool async = false;                  // FP32 passes from the asynchronous worklist
    int32_t* a_state = nullptr;          // worklist: per-tile state and first-visit counters
    int32_t* a_deps = nullptr;
    unsigned long long* a_queue = nullptr;
    int a_cap = 0;
    AsyncCtl* a_ctl = nullptr;
    float* uhat = nullptr;
    uint8_t* a = nullptr;
    int32_t* key = nullptr;
    int32_t* succ = nullptr;
    int32_t* jump_a = nullptr;
    int32_t* jump_b = nullptr;
    int8_t* label = nullptr;
    float* speed_c = nullptr;
    uint8_t* mask_c = nullptr;
    float* uc = nullptr;
    float2* ctrl32 = nullptr;
    double2* ctrl64 = nullptr;
    // block tables
    int2* fblk = nullptr;
    int nfblk = 0;
    int2* cblk = nullptr;
    int ncblk = 0;
    int4* rblk = nullptr;
    int nrblk = 0;
    int* corder = nullptr;
    // tiles (sized for the finest shape)
    long long nt_cap = 0;
    int NT = 0;
    int32_t* tile_inst = nullptr;
    int32_t* wt_nodes = nullptr;
    float* wt_speed = nullptr;
    int32_t* wt_count = nullptr;
    int32_t* tile_min = nullptr;
    int32_t* tile_wave = nullptr;
    int32_t* tile_key = nullptr;
    int32_t* tile_list = nullptr;
    unsigned int* tile_inc = nullptr;
    int32_t* stamp = nullptr;
    int32_t* queue = nullptr;
    int32_t* qcount = nullptr;
    unsigned int* step_inc = nullptr;
    int32_t* sched_count = nullptr;
    int32_t* sched_off = nullptr;
    int sched_cap = 0;
    int n_waves = 1;
    int32_t* cb_wave = nullptr;          // warm restart: checkerboard waves
    int32_t* cb_key = nullptr;
    int32_t* cb_list = nullptr;
    int32_t* cb_off = nullptr;
    int32_t* cb_count = nullptr;
    int32_t* rank_flags = nullptr;       // dense-wave scratch
    int32_t* rank_scan = nullptr;
    int32_t* rank_boff = nullptr;        // count + 1
    int* n_waves_dev = nullptr;
    int rank_cap = 0;
    int max_wh = 0;
    int max_R = 0;
    int tiles_shape = 0;         // shape the tile arrays were built for (0: none)
    // per-instance scalars
    int* max_key = nullptr;
    int* c_sweeps = nullptr;
    float* c_inc = nullptr;
    unsigned long long* res_bits = nullptr;
    float* margin = nullptr;
    uint8_t* active = nullptr;
    // correction rounds of the FP64 stage (allocated on first use)
    float* corr_r = nullptr;             // N: residual field
    uint8_t* corr_a = nullptr;           // N: its minimising control
    float* corr_tol = nullptr;           // count: inner tolerances
    uint8_t* corr_sel = nullptr;         // count: instances of the round
    unsigned int* inc_bits = nullptr;
    int* j_sweeps = nullptr;
    int* n_active = nullptr;
    GridSync* sync = nullptr;
    WaveResult* wres = nullptr;
    WaveResult* h_wres = nullptr;        // pinned
    // warm start of the coarse solves
    float* coarse_init = nullptr;        // Nc
    long long* d_coarse_off = nullptr;   // count + 1
    uint8_t* c_fallback = nullptr;       // count
    bool warm_on = false;
    int warm_k = 0;
    double warm_tol = 0.0;
    std::vector<long long> n_free;       // free fine nodes per instance
    std::vector<long long> n_free_c;     // free coarse nodes per instance
    bool built = false;
    bool tuned = false;
    bool value_f64 = false;              // u64 holds the latest values
};

namespace {

int bfail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    return set_last_error(code, buf);
}

#define BCU(call)                                                                              \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return bfail(e_ == cudaErrorMemoryAllocation ? HJB_ERR_OOM : HJB_ERR_CUDA,         \
                         "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)

template <typename T>
cudaError_t dalloc(T*& p, size_t count, cudaStream_t st) {
    return pool_alloc((void**)&p, std::max<size_t>(count, 1) * sizeof(T), st);
}
template <typename T>
void dfree(T*& p, cudaStream_t st) {
    pool_free((void*)p, st);
    p = nullptr;
}

struct BTimer {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaStream_t st;
    explicit BTimer(cudaStream_t s) : st(s) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, st);
    }
    double stop() {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float ms = 0.0f;
        cudaEventElapsedTime(&ms, e0, e1);
        return ms;
    }
    ~BTimer() {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
    }
};

int halo_of(double reach) { return sweep_halo(reach); }

// block -> (instance, first element) over per-instance element counts
std::vector<int2> block_table(const std::vector<long long>& counts, int per_block) {
    std::vector<int2> t;
    for (size_t b = 0; b < counts.size(); ++b)
        for (long long s = 0; s < counts[b]; s += per_block) t.push_back(make_int2((int)b, (int)s));
    return t;
}

}  // namespace

namespace {

// Per-instance tile layout for a warp-tile shape; uploads the TileInst records
// and the tile -> instance table.
int setup_tiles(hjb_batch* b, int shape) {
    if (b->tiles_shape == shape) return HJB_OK;
    int tw, th;
    wtile_dims(shape, &tw, &th);
    std::vector<int32_t> tinst;
    tinst.reserve((size_t)b->nt_cap);
    int off = 0;
    b->max_wh = 0;
    for (int i = 0; i < b->count; ++i) {
        TileInst& t = b->htile[i];
        const int n = b->desc[i].n;
        t.ntx = (n + tw - 1) / tw;
        t.nty = (n + th - 1) / th;
        t.tile_off = off;
        t.act_radius = std::max(1, (t.R + std::min(tw, th) - 1) / std::min(tw, th));
        const int nti = t.ntx * t.nty;
        for (int q = 0; q < nti; ++q) tinst.push_back(i);
        off += nti;
        b->max_wh = std::max(b->max_wh, (tw + 2 * t.R) * (th + 2 * t.R));
    }
    b->NT = off;
    BCU(cudaMemcpyAsync(b->dtile, b->htile.data(), sizeof(TileInst) * b->count, cudaMemcpyHostToDevice,
                        b->st));
    BCU(cudaMemcpyAsync(b->tile_inst, tinst.data(), sizeof(int32_t) * tinst.size(),
                        cudaMemcpyHostToDevice, b->st));
    BCU(cudaStreamSynchronize(b->st));
    b->tiles_shape = shape;
    return HJB_OK;
}

int validate_batch(const hjb_batch_desc* d, int32_t count, const hjb_batch_inst* in) {
    if (!d || !in) return bfail(HJB_ERR_INVALID_ARG, "desc / insts is NULL");
    if (count < 1) return bfail(HJB_ERR_INVALID_ARG, "count=%d must be >= 1", count);
    if (d->n_controls < 1 || d->n_controls > HJB_MAX_CONTROLS)
        return bfail(HJB_ERR_INVALID_ARG, "n_controls=%d out of range", d->n_controls);
    if (d->scheme != 0 && d->scheme != 2 && d->scheme != 3)
        return bfail(HJB_ERR_INVALID_ARG, "scheme must be 2 or 3");
    if (d->tile_shape < -1 || d->tile_shape > 2)
        return bfail(HJB_ERR_INVALID_ARG, "tile_shape must be -1, 0, 1 or 2");
    if (d->schedule != 0 && d->schedule != 3 && d->schedule != 4)
        return bfail(HJB_ERR_INVALID_ARG, "schedule must be 0, 3 or 4");
    if (!(d->cost > 0.0) || !std::isfinite(d->cost)) return bfail(HJB_ERR_INVALID_ARG, "cost must be > 0");
    if (!std::isfinite(d->band_width)) return bfail(HJB_ERR_INVALID_ARG, "bad band_width");
    long long N = 0;
    for (int i = 0; i < count; ++i) {
        const hjb_batch_inst& x = in[i];
        if (x.n < 9 || x.n > 16385) return bfail(HJB_ERR_INVALID_ARG, "instance %d: n=%d out of range", i, x.n);
        if (x.coarse_n < 5 || x.coarse_n > x.n || (x.n - 1) % (x.coarse_n - 1) != 0)
            return bfail(HJB_ERR_INVALID_ARG, "instance %d: coarse_n=%d does not nest in n=%d", i,
                         x.coarse_n, x.n);
        if (x.coarse_n > 181)
            return bfail(HJB_ERR_INVALID_ARG, "instance %d: coarse_n=%d above 181 (shared memory)", i,
                         x.coarse_n);
        if (x.n_patches < 1 || x.n_patches > HJB_MAX_PATCHES)
            return bfail(HJB_ERR_INVALID_ARG, "instance %d: n_patches=%d out of range", i, x.n_patches);
        if (x.reserved != 0) return bfail(HJB_ERR_INVALID_ARG, "instance %d: reserved must be 0", i);
        if (!(x.lambda > 0.0) || !std::isfinite(x.lambda))
            return bfail(HJB_ERR_INVALID_ARG, "instance %d: lambda must be > 0", i);
        if (!(x.sigma >= 0.0) || !std::isfinite(x.sigma))
            return bfail(HJB_ERR_INVALID_ARG, "instance %d: bad sigma", i);
        if (!std::isfinite(x.h)) return bfail(HJB_ERR_INVALID_ARG, "instance %d: bad h", i);
        N += (long long)x.n * x.n;
    }
    if (N >= (1LL << 31)) return bfail(HJB_ERR_INVALID_ARG, "batch holds %lld nodes (max 2^31 - 1)", N);
    return HJB_OK;
}

}  // namespace

// The host inputs of a batch: either concatenated arrays (instance i's nodes
// after those of instances 0 .. i-1) or one array per instance.
struct BatchHostInputs {
    const float* speed = nullptr;
    const uint8_t* mask = nullptr;
    const int8_t* sector = nullptr;
    const float* const* speed_list = nullptr;
    const uint8_t* const* mask_list = nullptr;
    const int8_t* const* sector_list = nullptr;
    bool lists() const { return speed_list != nullptr; }
};

int batch_create(const hjb_batch_desc* desc, int32_t count, const hjb_batch_inst* insts,
                 const BatchHostInputs& in, const double* controls, void* cuda_stream,
                 hjb_batch** out) {
    clear_last_error();
    if (!out) return bfail(HJB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate_batch(desc, count, insts);
    if (rc) return rc;
    if (!controls) return bfail(HJB_ERR_INVALID_ARG, "controls are required");
    if (in.lists()) {
        if (!in.mask_list) return bfail(HJB_ERR_INVALID_ARG, "speed and mask lists are required");
        for (int i = 0; i < count; ++i)
            if (!in.speed_list[i] || !in.mask_list[i])
                return bfail(HJB_ERR_INVALID_ARG, "instance %d: speed / mask is NULL", i);
    } else if (!in.speed || !in.mask) {
        return bfail(HJB_ERR_INVALID_ARG, "speed, mask and controls are required");
    }
    const int na = desc->n_controls;
    double amax = 0.0;
    for (int m = 0; m < na; ++m) {
        if (!std::isfinite(controls[2 * m]) || !std::isfinite(controls[2 * m + 1]))
            return bfail(HJB_ERR_INVALID_ARG, "control %d is not finite", m);
        amax = std::max(amax, std::max(std::fabs(controls[2 * m]), std::fabs(controls[2 * m + 1])));
    }
    hjb_batch* b = new hjb_batch();
    auto bail = [&](int code) {
        hjb_batch_destroy(b);
        return code;
    };
    b->count = count;
    b->na = na;
    b->scheme = desc->scheme == 0 ? 3 : desc->scheme;
    b->D = desc->tile_period <= 0 ? 2 : desc->tile_period;
    b->shape = desc->tile_shape < 0 ? 2 : desc->tile_shape + 1;
    b->B = desc->tile_waves <= 0 ? 2 : desc->tile_waves;
    b->tuned = desc->tile_shape >= 0 && desc->tile_waves > 0;
    b->cost = desc->cost;
    b->band_width = desc->band_width > 0.0 ? desc->band_width : 1.0;
    b->sched_mode = desc->schedule;
    b->async = desc->schedule == 3;
    b->desc.assign(insts, insts + count);
    b->node_off.assign(count + 1, 0);
    b->coarse_off.assign(count + 1, 0);
    for (int i = 0; i < count; ++i) {
        b->node_off[i + 1] = b->node_off[i] + (long long)insts[i].n * insts[i].n;
        b->coarse_off[i + 1] = b->coarse_off[i] + (long long)insts[i].coarse_n * insts[i].coarse_n;
    }
    b->N = b->node_off[count];
    b->Nc = b->coarse_off[count];
    std::vector<float> cmax(count, 0.0f);
    if (cuda_stream) {
        b->st = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->st, cudaStreamNonBlocking) != cudaSuccess)
            return bail(bfail(HJB_ERR_CUDA, "cudaStreamCreate failed"));
        b->own_stream = true;
    }
#define BCUP(call)                                                                             \
    do {                                                                                       \
        cudaError_t e_ = (call);                                                               \
        if (e_ != cudaSuccess)                                                                 \
            return bail(bfail(e_ == cudaErrorMemoryAllocation ? HJB_ERR_OOM : HJB_ERR_CUDA,    \
                              "%s failed: %s", #call, cudaGetErrorString(e_)));                \
    } while (0)
    int dev = 0;
    BCUP(cudaGetDevice(&dev));
    BCUP(cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev));
    const size_t N = (size_t)b->N, Nc = (size_t)b->Nc;
    BCUP(dalloc(b->speed, N, b->st));
    BCUP(dalloc(b->mask, N, b->st));
    BCUP(dalloc(b->sector, N, b->st));
    BCUP(dalloc(b->u32, N, b->st));
    BCUP(dalloc(b->u32b, N, b->st));
    BCUP(dalloc(b->u64, N, b->st));
    BCUP(dalloc(b->uhat, N, b->st));
    BCUP(dalloc(b->a, N, b->st));
    BCUP(dalloc(b->key, N, b->st));
    BCUP(dalloc(b->succ, N, b->st));
    BCUP(dalloc(b->jump_a, N, b->st));
    BCUP(dalloc(b->jump_b, N, b->st));
    BCUP(dalloc(b->label, N, b->st));
    BCUP(dalloc(b->speed_c, Nc, b->st));
    BCUP(dalloc(b->mask_c, Nc, b->st));
    BCUP(dalloc(b->uc, Nc, b->st));
    BCUP(dalloc(b->ctrl32, na, b->st));
    BCUP(dalloc(b->ctrl64, na, b->st));
    // uploads: one copy per array, or per instance and array (no host-side
    // concatenation); absent sectors: sector 0 on target nodes, -1 elsewhere
    for (int i = 0; i < (in.lists() ? count : 1); ++i) {
        const long long o = in.lists() ? b->node_off[i] : 0;
        const size_t Ni = in.lists() ? (size_t)(b->node_off[i + 1] - o) : N;
        const float* sp = in.lists() ? in.speed_list[i] : in.speed;
        const uint8_t* mk = in.lists() ? in.mask_list[i] : in.mask;
        const int8_t* sc = in.lists() ? (in.sector_list ? in.sector_list[i] : nullptr) : in.sector;
        BCUP(cudaMemcpyAsync(b->speed + o, sp, Ni * sizeof(float), cudaMemcpyHostToDevice, b->st));
        BCUP(cudaMemcpyAsync(b->mask + o, mk, Ni, cudaMemcpyHostToDevice, b->st));
        if (sc) {
            BCUP(cudaMemcpyAsync(b->sector + o, sc, Ni, cudaMemcpyHostToDevice, b->st));
        } else {
            std::vector<int8_t> sec(Ni);
            for (size_t k = 0; k < Ni; ++k) sec[k] = mk[k] == HJB_MASK_TARGET ? 0 : -1;
            BCUP(cudaMemcpyAsync(b->sector + o, sec.data(), Ni, cudaMemcpyHostToDevice, b->st));
            BCUP(cudaStreamSynchronize(b->st));
        }
    }
    const bool has_sector = in.lists() ? in.sector_list != nullptr : in.sector != nullptr;
    {
        // per-instance checks and speed maxima on the device, after the upload
        // (the host never walks the concatenated arrays)
        constexpr int kScanBlocks = 64;
        BCUP(dalloc(b->scan_tmp, (size_t)count * kScanBlocks + (size_t)count, b->st));
        InputScan* rec = b->scan_tmp;
        unsigned long long* bad = reinterpret_cast<unsigned long long*>(rec + (size_t)count * kScanBlocks);
        BCUP(cudaMemsetAsync(bad, 0xff, sizeof(unsigned long long) * 4 * (size_t)count, b->st));
        std::vector<int> nbk(count);
        for (int i = 0; i < count; ++i) {
            const long long o = b->node_off[i], Ni = b->node_off[i + 1] - o;
            nbk[i] = std::min(kScanBlocks, scan_inputs_blocks(Ni));
            BCUP(launch_scan_inputs(Ni, b->speed + o, b->mask + o, has_sector ? b->sector + o : nullptr,
                                    insts[i].n_patches, nullptr, 1.0f, rec + (size_t)i * kScanBlocks,
                                    bad + 4 * (size_t)i, nbk[i], b->st));
        }
        std::vector<InputScan> hr((size_t)count * kScanBlocks);
        std::vector<unsigned long long> hb(4 * (size_t)count);
        BCUP(cudaMemcpyAsync(hr.data(), rec, sizeof(InputScan) * hr.size(), cudaMemcpyDeviceToHost, b->st));
        BCUP(cudaMemcpyAsync(hb.data(), bad, sizeof(unsigned long long) * hb.size(), cudaMemcpyDeviceToHost,
                             b->st));
        BCUP(cudaStreamSynchronize(b->st));
        dfree(b->scan_tmp, b->st);
        b->n_free.assign(count, 0);
        for (int i = 0; i < count; ++i) {
            unsigned flags = 0;
            for (int q = 0; q < nbk[i]; ++q) {
                const InputScan& r = hr[(size_t)i * kScanBlocks + q];
                flags |= r.flags;
                cmax[i] = std::max(cmax[i], r.cmax);
                b->n_free[i] += (long long)r.nfree;
            }
            if (flags & 1u)
                return bail(bfail(HJB_ERR_INVALID_ARG, "instance %d: speed[%llu] is negative or not finite", i,
                                  hb[4 * (size_t)i]));
            if (flags & 2u)
                return bail(bfail(HJB_ERR_INVALID_ARG, "instance %d: mask[%llu] invalid", i, hb[4 * (size_t)i + 1]));
            if (flags & 4u)
                return bail(bfail(HJB_ERR_INVALID_ARG, "instance %d: sector[%llu] out of range", i,
                                  hb[4 * (size_t)i + 2]));
        }
    }
    {
        std::vector<float2> c32(na);
        std::vector<double2> c64(na);
        for (int m = 0; m < na; ++m) {
            c32[m] = make_float2((float)controls[2 * m], (float)controls[2 * m + 1]);
            c64[m] = make_double2(controls[2 * m], controls[2 * m + 1]);
        }
        // 32 controls in opposite pairs a_{m+16} = -a_m (to 1e-12): the FP32 warp
        // tiles update two nodes at a time, two controls a lane (mirrored geometry)
        b->ctrl_sym32 = na == 32;
        for (int m = 0; m < 16 && b->ctrl_sym32; ++m)
            b->ctrl_sym32 = std::fabs(controls[2 * (m + 16)] + controls[2 * m]) <= 1e-12 &&
                            std::fabs(controls[2 * (m + 16) + 1] + controls[2 * m + 1]) <= 1e-12;
        // closed under quarter turns as well: four nodes at a time, four controls a lane
        b->ctrl_rot32 = b->ctrl_sym32;
        for (int m = 0; m < 8 && b->ctrl_rot32; ++m)
            b->ctrl_rot32 = std::fabs(controls[2 * (m + 8)] + controls[2 * m + 1]) <= 1e-12 &&
                            std::fabs(controls[2 * (m + 8) + 1] - controls[2 * m]) <= 1e-12 &&
                            std::fabs(controls[2 * (m + 24)] - controls[2 * m + 1]) <= 1e-12 &&
                            std::fabs(controls[2 * (m + 24) + 1] + controls[2 * m]) <= 1e-12;
        BCUP(cudaMemcpyAsync(b->ctrl32, c32.data(), sizeof(float2) * na, cudaMemcpyHostToDevice, b->st));
        BCUP(cudaMemcpyAsync(b->ctrl64, c64.data(), sizeof(double2) * na, cudaMemcpyHostToDevice, b->st));
        BCUP(cudaStreamSynchronize(b->st));
    }
    // per-instance records
    b->hinst.resize(count);
    b->htile.resize(count);
    b->uob.resize(count);
    std::vector<float> hmargin(count);
    std::vector<long long> fcount(count), ccount(count);
    long long nt_cap = 0;
    int nc_max = 0;
    std::vector<double> edges;
    for (int i = 0; i < count; ++i) {
        const hjb_batch_inst& x = insts[i];
        const int n = x.n, nc = x.coarse_n;
        const double dx = 2.0 / (n - 1);
        const double h = x.h > 0.0 ? x.h : dx;
        const double beta = 1.0 / (1.0 + x.lambda * h);
        const double hl = h * b->cost;
        const double uob = hl / (1.0 - beta);
        const int r = (n - 1) / (nc - 1);
        const double hc = h * r;
        const double beta_c = 1.0 / (1.0 + x.lambda * hc);
        const double hl_c = hc * b->cost;
        const double uob_c = hl_c / (1.0 - beta_c);
        const double reach = (h * cmax[i] * amax + std::sqrt(2.0 * h) * x.sigma) / dx;
        const int R = halo_of(reach);
        if (R > 64)
            return bail(bfail(HJB_ERR_INVALID_ARG, "instance %d: interpolation reach %.1f cells too large",
                              i, reach));
        b->any_sigma = b->any_sigma || x.sigma > 0.0;
        const long long o = b->node_off[i], oc = b->coarse_off[i];
        GridView g{};
        g.n = n;
        g.na = na;
        g.speed = b->speed + o;
        g.drift = nullptr;
        g.mask = b->mask + o;
        g.ctrl32 = b->ctrl32;
        g.ctrl64 = b->ctrl64;
        g.s32 = (float)(h / dx);
        g.s64 = h / dx;
        g.d32 = (float)(std::sqrt(2.0 * h) * x.sigma / dx);
        g.d64 = std::sqrt(2.0 * h) * x.sigma / dx;
        g.beta32 = (float)beta;
        g.beta64 = beta;
        g.hl32 = (float)hl;
        g.hl64 = hl;
        g.uob32 = (float)uob;
        g.uob64 = uob;
        GridView gc = g;
        gc.n = nc;
        gc.speed = b->speed_c + oc;
        gc.mask = b->mask_c + oc;
        gc.d32 = 0.0f;
        gc.d64 = 0.0;
        gc.s32 = (float)(hc / (2.0 / (nc - 1)));
        gc.s64 = hc / (2.0 / (nc - 1));
        gc.beta32 = (float)beta_c;
        gc.beta64 = beta_c;
        gc.hl32 = (float)hl_c;
        gc.hl64 = hl_c;
        gc.uob32 = (float)uob;    // obstacles hold the fine scheme's value on both grids
        gc.uob64 = uob;
        BatchInst& B = b->hinst[i];
        B = BatchInst{};
        B.g = g;
        B.gc = gc;
        B.uhat = b->uhat + o;
        B.uc = b->uc + oc;
        B.speed_c = b->speed_c + oc;
        B.mask_c = b->mask_c + oc;
        B.a = b->a + o;
        B.key = b->key + o;
        B.sector = b->sector + o;
        B.label = b->label + o;
        B.node_off = o;
        B.nc = nc;
        B.n_patches = x.n_patches;
        B.R = R;
        B.lambda = (float)x.lambda;
        B.band_w = (float)(b->band_width * h);
        {
            std::vector<double> e;
            band_edges(x.lambda, b->band_width * h, kBandCap, e);
            B.bm.lambda = B.lambda;
            B.bm.w64 = b->band_width * h;
            B.bm.w32 = B.band_w;
            B.bm.n_edges = (int)e.size();
            B.bm.cap = kBandCap;
            B.bm.edges = reinterpret_cast<const double*>((uintptr_t)edges.size());   // offset until upload
            edges.insert(edges.end(), e.begin(), e.end());
        }
        B.uc0 = (float)uob_c;
        B.uob32 = (float)uob;
        B.sigma = (float)x.sigma;
        B.uob64 = uob;
        TileInst& T = b->htile[i];
        T = TileInst{};
        T.g = g;
        T.u32 = b->u32 + o;
        T.u64 = b->u64 + o;
        T.uhat = b->uhat + o;
        T.lambda = B.lambda;
        T.band_w = B.band_w;
        T.R = R;
        b->max_R = std::max(b->max_R, R);
        b->uob[i] = uob;
        // FP32 screening margin of the FP64 residual: 2.2 x the FP32 candidate error
        // bound (20 + 10 reach) 2^-24 max(1, U) (the single-problem residual's)
        hmargin[i] = (float)(2.2 * (20.0 + 10.0 * reach) * std::ldexp(1.0, -24) * std::max(1.0, uob));
        fcount[i] = (long long)n * n;
        ccount[i] = (long long)nc * nc;
        nt_cap += (long long)((n + 3) / 4) * ((n + 3) / 4);
        nc_max = std::max(nc_max, nc);
    }
    b->nt_cap = nt_cap;
    if (!edges.empty()) {
        BCUP(dalloc(b->band_e, edges.size(), b->st));
        BCUP(cudaMemcpyAsync(b->band_e, edges.data(), sizeof(double) * edges.size(), cudaMemcpyHostToDevice,
                             b->st));
    }
    for (int i = 0; i < count; ++i)
        b->hinst[i].bm.edges = b->band_e ? b->band_e + (uintptr_t)b->hinst[i].bm.edges : nullptr;
    BCUP(dalloc(b->dinst, count, b->st));
    BCUP(dalloc(b->dtile, count, b->st));
    BCUP(cudaMemcpyAsync(b->dinst, b->hinst.data(), sizeof(BatchInst) * count, cudaMemcpyHostToDevice,
                         b->st));
    // block tables
    {
        auto fb = block_table(fcount, kBT);
        auto cbk = block_table(ccount, kBT);
        std::vector<int4> rb;
        for (int i = 0; i < count; ++i) {
            const int n = insts[i].n;
            for (int ty = 0; ty < (n + kRY - 1) / kRY; ++ty)
                for (int tx = 0; tx < (n + kRX - 1) / kRX; ++tx) rb.push_back(make_int4(i, tx, ty, 0));
        }
        std::vector<int> ord(count);
        for (int i = 0; i < count; ++i) ord[i] = i;
        std::stable_sort(ord.begin(), ord.end(),
                         [&](int p, int q) { return insts[p].coarse_n > insts[q].coarse_n; });
        b->nfblk = (int)fb.size();
        b->ncblk = (int)cbk.size();
        b->nrblk = (int)rb.size();
        BCUP(dalloc(b->fblk, fb.size(), b->st));
        BCUP(dalloc(b->cblk, cbk.size(), b->st));
        BCUP(dalloc(b->rblk, rb.size(), b->st));
        BCUP(dalloc(b->corder, count, b->st));
        BCUP(cudaMemcpyAsync(b->fblk, fb.data(), sizeof(int2) * fb.size(), cudaMemcpyHostToDevice, b->st));
        BCUP(cudaMemcpyAsync(b->cblk, cbk.data(), sizeof(int2) * cbk.size(), cudaMemcpyHostToDevice, b->st));
        BCUP(cudaMemcpyAsync(b->rblk, rb.data(), sizeof(int4) * rb.size(), cudaMemcpyHostToDevice, b->st));
        BCUP(cudaMemcpyAsync(b->corder, ord.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->st));
        BCUP(cudaStreamSynchronize(b->st));
    }
    // tiles, sized for the finest shape (4x4)
    const size_t ntc = (size_t)nt_cap;
    BCUP(dalloc(b->tile_inst, ntc, b->st));
    BCUP(dalloc(b->wt_nodes, ntc * kWarpTileNodes, b->st));
    BCUP(dalloc(b->wt_speed, ntc * kWarpTileNodes, b->st));
    BCUP(dalloc(b->wt_count, ntc, b->st));
    BCUP(dalloc(b->tile_min, ntc, b->st));
    BCUP(dalloc(b->tile_wave, ntc, b->st));
    BCUP(dalloc(b->tile_key, ntc, b->st));
    BCUP(dalloc(b->tile_list, ntc, b->st));
    BCUP(dalloc(b->tile_inc, ntc, b->st));
    BCUP(dalloc(b->stamp, ntc, b->st));
    BCUP(dalloc(b->queue, ntc * (size_t)(b->D + 2), b->st));
    BCUP(dalloc(b->cb_wave, ntc, b->st));
    BCUP(dalloc(b->cb_key, ntc, b->st));
    BCUP(dalloc(b->cb_list, ntc, b->st));
    BCUP(dalloc(b->cb_off, 3, b->st));
    BCUP(dalloc(b->cb_count, 2, b->st));
    BCUP(dalloc(b->qcount, b->D + 2, b->st));
    BCUP(dalloc(b->step_inc, 2 * b->D, b->st));
    // per-instance scalars
    BCUP(dalloc(b->max_key, count, b->st));
    BCUP(dalloc(b->c_sweeps, count, b->st));
    BCUP(dalloc(b->c_inc, count, b->st));
    BCUP(dalloc(b->res_bits, count, b->st));
    BCUP(dalloc(b->margin, count, b->st));
    BCUP(dalloc(b->active, count, b->st));
    BCUP(dalloc(b->inc_bits, count, b->st));
    BCUP(dalloc(b->j_sweeps, count, b->st));
    BCUP(dalloc(b->n_active, 1, b->st));
    BCUP(dalloc(b->rank_boff, count + 1, b->st));
    BCUP(dalloc(b->d_coarse_off, count + 1, b->st));
    BCUP(dalloc(b->c_fallback, count, b->st));
    BCUP(cudaMemsetAsync(b->c_fallback, 0, count, b->st));
    BCUP(cudaMemcpyAsync(b->d_coarse_off, b->coarse_off.data(), sizeof(long long) * (count + 1),
                         cudaMemcpyHostToDevice, b->st));
    BCUP(dalloc(b->n_waves_dev, 1, b->st));
    BCUP(dalloc(b->sync, 1, b->st));
    BCUP(dalloc(b->wres, 1, b->st));
    BCUP(cudaMallocHost((void**)&b->h_wres, sizeof(WaveResult)));
    BCUP(cudaMemcpyAsync(b->margin, hmargin.data(), sizeof(float) * count, cudaMemcpyHostToDevice, b->st));
    // coarse data (inputs are fixed)
    count_launches(1);
    k_b_coarse_data<<<b->ncblk, kBT, 0, b->st>>>(b->dinst, b->cblk);
    BCUP(cudaGetLastError());
    {
        const size_t smem = (((size_t)na * sizeof(float2) + 15) & ~(size_t)15) + (size_t)nc_max * nc_max * 4;
        BCUP(cudaFuncSetAttribute(k_b_coarse_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    }
    rc = setup_tiles(b, b->shape);
    if (rc) return bail(rc);
    BCUP(cudaStreamSynchronize(b->st));
    {
        // free coarse nodes (the fine ones came with the input scan)
        b->n_free_c.assign(count, 0);
        std::vector<uint8_t> mc((size_t)b->Nc);
        BCUP(cudaMemcpyAsync(mc.data(), b->mask_c, (size_t)b->Nc, cudaMemcpyDeviceToHost, b->st));
        BCUP(cudaStreamSynchronize(b->st));
        for (int i = 0; i < count; ++i)
            for (long long k = b->coarse_off[i]; k < b->coarse_off[i + 1]; ++k) b->n_free_c[i] += mc[k] == 0;
    }
#undef BCUP
    *out = b;
    return HJB_OK;
}

extern "C" {

int hjb_batch_create(const hjb_batch_desc* desc, int32_t count, const hjb_batch_inst* insts,
                     const float* speed, const uint8_t* mask, const int8_t* sector,
                     const double* controls, void* cuda_stream, hjb_batch** out) {
    BatchHostInputs in;
    in.speed = speed;
    in.mask = mask;
    in.sector = sector;
    return batch_create(desc, count, insts, in, controls, cuda_stream, out);
}

int hjb_batch_create_lists(const hjb_batch_desc* desc, int32_t count, const hjb_batch_inst* insts,
                           const float* const* speed, const uint8_t* const* mask,
                           const int8_t* const* sector, const double* controls, void* cuda_stream,
                           hjb_batch** out) {
    if (!speed || !mask) {
        clear_last_error();
        if (out) *out = nullptr;
        return bfail(HJB_ERR_INVALID_ARG, "speed and mask lists are required");
    }
    BatchHostInputs in;
    in.speed_list = speed;
    in.mask_list = mask;
    in.sector_list = sector;
    return batch_create(desc, count, insts, in, controls, cuda_stream, out);
}

void hjb_batch_destroy(hjb_batch* b) {
    if (!b) return;
    b->pre_graph.reset();
    dfree(b->scan_tmp, b->st);
    if (b->st) cudaStreamSynchronize(b->st);
    dfree(b->dinst, b->st); dfree(b->dtile, b->st);
    dfree(b->speed, b->st); dfree(b->mask, b->st); dfree(b->sector, b->st); dfree(b->u32, b->st); dfree(b->u32b, b->st); dfree(b->u64, b->st); dfree(b->band_e, b->st);
    dfree(b->a_state, b->st); dfree(b->a_deps, b->st); dfree(b->a_queue, b->st); dfree(b->a_ctl, b->st);
    dfree(b->uhat, b->st); dfree(b->a, b->st); dfree(b->key, b->st); dfree(b->succ, b->st); dfree(b->jump_a, b->st); dfree(b->jump_b, b->st);
    dfree(b->label, b->st); dfree(b->speed_c, b->st); dfree(b->mask_c, b->st); dfree(b->uc, b->st); dfree(b->ctrl32, b->st); dfree(b->ctrl64, b->st);
    dfree(b->fblk, b->st); dfree(b->cblk, b->st); dfree(b->rblk, b->st); dfree(b->corder, b->st);
    dfree(b->tile_inst, b->st); dfree(b->wt_nodes, b->st); dfree(b->wt_speed, b->st); dfree(b->wt_count, b->st); dfree(b->tile_min, b->st);
    dfree(b->tile_wave, b->st); dfree(b->tile_key, b->st); dfree(b->tile_list, b->st); dfree(b->tile_inc, b->st); dfree(b->stamp, b->st);
    dfree(b->queue, b->st); dfree(b->qcount, b->st); dfree(b->step_inc, b->st); dfree(b->sched_count, b->st); dfree(b->sched_off, b->st);
    dfree(b->max_key, b->st); dfree(b->c_sweeps, b->st); dfree(b->c_inc, b->st); dfree(b->res_bits, b->st); dfree(b->margin, b->st);
    dfree(b->corr_r, b->st); dfree(b->corr_a, b->st); dfree(b->corr_tol, b->st); dfree(b->corr_sel, b->st);
    dfree(b->active, b->st); dfree(b->inc_bits, b->st); dfree(b->j_sweeps, b->st); dfree(b->n_active, b->st); dfree(b->sync, b->st);
    dfree(b->coarse_init, b->st); dfree(b->d_coarse_off, b->st); dfree(b->c_fallback, b->st);
    dfree(b->cb_wave, b->st); dfree(b->cb_key, b->st); dfree(b->cb_list, b->st); dfree(b->cb_off, b->st); dfree(b->cb_count, b->st);
    dfree(b->wres, b->st); dfree(b->rank_flags, b->st); dfree(b->rank_scan, b->st); dfree(b->rank_boff, b->st); dfree(b->n_waves_dev, b->st);
    if (b->h_wres) cudaFreeHost(b->h_wres);
    if (b->own_stream && b->st) cudaStreamDestroy(b->st);
    delete b;
}

}  // extern "C"

// ------------------------------------------------------------------ stages
namespace {

size_t coarse_smem(const hjb_batch* b) {
    int nc_max = 0;
    for (const auto& x : b->desc) nc_max = std::max(nc_max, x.coarse_n);
    return (((size_t)b->na * sizeof(float2) + 15) & ~(size_t)15) + (size_t)nc_max * nc_max * 4;
}

// coarse solves; returns node updates
int stage_coarse(hjb_batch* b, double tol_c, int max_sweeps, long long* nodes, bool* conv) {
    count_launches(1);
    k_b_coarse_solve<<<b->count, kCoarseThreads, coarse_smem(b), b->st>>>(
        b->dinst, b->corder, (float)tol_c, max_sweeps, b->c_sweeps, b->c_inc,
        b->warm_on ? b->coarse_init : nullptr, b->d_coarse_off, b->warm_k, (float)b->warm_tol, b->c_fallback);
    BCU(cudaGetLastError());
    std::vector<int> sw(b->count);
    BCU(cudaMemcpyAsync(sw.data(), b->c_sweeps, sizeof(int) * b->count, cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    long long nd = 0;
    bool ok = true;
    for (int i = 0; i < b->count; ++i) {
        nd += (long long)sw[i] * b->n_free_c[i];
        ok = ok && sw[i] < max_sweeps;
    }
    *nodes = nd;
    *conv = ok;
    return HJB_OK;
}

// interpolation, synthesis, bands, successors, labels; u32 = u_hat.  A fixed
// sequence of about 25 short kernels over the batch's buffers, replayed from a
// CUDA graph after the first call.
int stage_precompute(hjb_batch* b) {
    long long nmax = 0;
    for (const auto& x : b->desc) nmax = std::max(nmax, (long long)x.n * x.n);
    int rounds = 1;
    while ((1LL << rounds) < nmax) ++rounds;
    BCU(b->pre_graph.run(b->st, [&](cudaStream_t st) {
        count_launches(1);
        k_b_interp<<<b->nfblk, kBT, 0, st>>>(b->dinst, b->fblk);
        cudaError_t e = cudaMemsetAsync(b->max_key, 0, sizeof(int) * b->count, st);
        if (e != cudaSuccess) return e;
        count_launches(1);
        k_b_synthesis<<<b->nfblk, kBT, (size_t)b->na * sizeof(float2), st>>>(b->dinst, b->fblk, kBandCap,
                                                                          b->max_key);
        count_launches(1);
        k_b_successors<<<b->nfblk, kBT, 0, st>>>(b->dinst, b->fblk, b->succ);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        const int32_t* end = nullptr;
        e = launch_pointer_jumps(b->N, b->succ, rounds, b->jump_a, b->jump_b, &end, st);
        if (e != cudaSuccess) return e;
        count_launches(1);
        k_b_labels<<<b->nfblk, kBT, 0, st>>>(b->dinst, b->fblk, end, b->mask, b->sector);
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
        return cudaMemcpyAsync(b->u32, b->uhat, sizeof(float) * (size_t)b->N, cudaMemcpyDeviceToDevice, st);
    }));
    b->value_f64 = false;
    return HJB_OK;
}

// warp tiles for the current shape and bands per wave
int stage_tiles(hjb_batch* b) {
    int rc = setup_tiles(b, b->shape);
    if (rc) return rc;
    std::vector<int> mk(b->count);
    BCU(cudaMemcpyAsync(mk.data(), b->max_key, sizeof(int) * b->count, cudaMemcpyDeviceToHost, b->st));
    BCU(launch_wtile_build(b->shape, b->dtile, b->tile_inst, b->NT, false, kBandCap, b->wt_nodes,
                           b->wt_speed, b->wt_count, b->tile_min, b->st));
    BCU(cudaStreamSynchronize(b->st));
    // dense waves: per instance, rank of each tile's lowest band among the
    // distinct ones (no step waits on a band no tile starts at)
    std::vector<int32_t> boff(b->count + 1, 0);
    for (int i = 0; i < b->count; ++i) boff[i + 1] = boff[i] + std::max(mk[i], 0) + 1;
    const int S = boff[b->count];
    if (S + 1 > b->rank_cap) {
        dfree(b->rank_flags, b->st);
        dfree(b->rank_scan, b->st);
        BCU(dalloc(b->rank_flags, (size_t)S + 1, b->st));
        BCU(dalloc(b->rank_scan, (size_t)S + 1, b->st));
        b->rank_cap = S + 1;
    }
    BCU(cudaMemcpyAsync(b->rank_boff, boff.data(), sizeof(int32_t) * (b->count + 1), cudaMemcpyHostToDevice,
                        b->st));
    BCU(launch_dense_waves(b->NT, b->tile_min, b->tile_inst, b->count, b->rank_boff, S, b->B,
                           b->rank_flags, b->rank_scan, b->tile_wave, b->tile_key, b->n_waves_dev, b->st));
    int nw = 1;
    BCU(cudaMemcpyAsync(&nw, b->n_waves_dev, sizeof(int), cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    b->n_waves = std::max(1, nw);
    if (b->n_waves > b->sched_cap) {
        dfree(b->sched_count, b->st);
        dfree(b->sched_off, b->st);
        BCU(dalloc(b->sched_count, b->n_waves, b->st));
        BCU(dalloc(b->sched_off, b->n_waves + 1, b->st));
        b->sched_cap = b->n_waves;
    }
    BCU(launch_counting_sort(b->NT, b->tile_key, b->n_waves, b->sched_count, b->sched_off, b->tile_list,
                             b->st));
    // warm-restart schedule: every tile with free nodes in two checkerboard waves
    BCU(launch_checker_waves(b->dtile, b->tile_inst, b->NT, b->wt_count, b->cb_wave, b->cb_key, b->st));
    BCU(launch_counting_sort(b->NT, b->cb_key, 2, b->cb_count, b->cb_off, b->cb_list, b->st));
    b->built = true;
    return HJB_OK;
}

// persistent warp-tile passes over every instance (f64: u64, only the instances
// flagged in b->active when use_active); warm: every tile visited in the first
// two steps in checkerboard order instead of along the causal waves
int stage_passes(hjb_batch* b, bool f64, double tol, int max_passes, bool use_active, WaveResult* out,
                 bool warm = false) {
    const int32_t* waves = warm ? b->cb_wave : b->tile_wave;
    const int n_waves = warm ? 2 : b->n_waves;
    BCU(cudaMemsetAsync(b->wres, 0, sizeof(WaveResult), b->st));
    BCU(cudaMemsetAsync(b->sync, 0, sizeof(GridSync), b->st));
    BCU(cudaMemsetAsync(b->step_inc, 0, sizeof(unsigned int) * 2 * b->D, b->st));
    BCU(cudaMemsetAsync(b->qcount, 0, sizeof(int32_t) * (b->D + 2), b->st));
    BCU(launch_tile_stamps(b->NT, waves, b->stamp, b->st));
    TileArgs a{};
    a.g = b->hinst[0].g;
    a.scheme = b->scheme;
    a.warp_tiles = b->shape;
    a.nodes = b->wt_nodes;
    a.wt_count = b->wt_count;
    a.tile_list = warm ? b->cb_list : b->tile_list;
    a.wave_off = warm ? b->cb_off : b->sched_off;
    a.tile_wave = waves;
    a.slot_speed = b->wt_speed;
    a.stamp = b->stamp;
    a.queue = b->queue;
    a.qcount = b->qcount;
    a.nt = b->NT;
    a.step_inc = b->step_inc;
    a.n_waves = n_waves;
    a.period = b->D;
    a.local_sweeps = 1;
    a.max_steps = n_waves + max_passes * b->D;
    a.tol = (float)tol;
    a.sync = b->sync;
    a.res = b->wres;
    a.timeout_ns = kTimeoutNs;
    a.insts = b->dtile;
    a.tile_inst = b->tile_inst;
    a.inst_active = use_active ? b->active : nullptr;
    a.max_wh = b->max_wh;
    a.node_pairs = f64 ? 0 : (b->ctrl_rot32 ? 3 : (b->ctrl_sym32 ? 2 : 0));
    const int per_sm = wtile_blocks_per_sm(f64, b->any_sigma, b->na, b->max_wh, b->shape);
    if (per_sm < 1) return bfail(HJB_ERR_INVALID_ARG, "warp-tile kernel does not fit on an SM");
    if (b->async && !f64 && !warm) {
        // the asynchronous worklist (see hjb_desc.schedule 3)
        const int warps = per_sm * b->num_sms * (tile_threads(false, b->shape) / 32);
        int cap = 1024;
        while (cap < b->NT + warps + 64) cap <<= 1;
        if (cap > b->a_cap) {
            dfree(b->a_state, b->st); dfree(b->a_deps, b->st); dfree(b->a_queue, b->st);
            BCU(dalloc(b->a_state, (size_t)b->NT, b->st));
            BCU(dalloc(b->a_deps, (size_t)b->NT, b->st));
            BCU(dalloc(b->a_queue, (size_t)cap, b->st));
            b->a_cap = cap;
        }
        if (!b->a_ctl) BCU(dalloc(b->a_ctl, 1, b->st));
        BCU(cudaMemsetAsync(b->a_queue, 0, sizeof(unsigned long long) * (size_t)b->a_cap, b->st));
        BCU(cudaMemsetAsync(b->a_ctl, 0, sizeof(AsyncCtl), b->st));
        a.astate = b->a_state;
        a.adeps = b->a_deps;
        a.aqueue = b->a_queue;
        a.aq_cap = b->a_cap;
        a.actl = b->a_ctl;
        a.max_visits = (long long)max_passes * b->NT;
        a.tile_cap = std::min(max_passes, kTileVisitCap);
        BCU(launch_wtiles_async(a, b->any_sigma, per_sm * b->num_sms, b->st));
        AsyncCtl hc{};
        GridSync hs{};
        BCU(cudaMemcpyAsync(b->h_wres, b->wres, sizeof(WaveResult), cudaMemcpyDeviceToHost, b->st));
        BCU(cudaMemcpyAsync(&hc, b->a_ctl, sizeof(AsyncCtl), cudaMemcpyDeviceToHost, b->st));
        BCU(cudaMemcpyAsync(&hs, b->sync, sizeof(GridSync), cudaMemcpyDeviceToHost, b->st));
        BCU(cudaStreamSynchronize(b->st));
        if (hs.err == HJB_ERR_TIMEOUT) return bfail(HJB_ERR_TIMEOUT, "batch tile worklist: a wait exceeded its limit");
        if (hs.err != 0) return bfail(hs.err, "batch tile worklist: internal error");
        *out = *b->h_wres;
        out->passes = (int)((hc.visits + b->NT - 1) / std::max(1, b->NT));
        out->converged = (hc.stop || hc.capped) ? 0 : 1;
        out->last_increment = (float)tol;
        return HJB_OK;
    }
    BCU(launch_wtiles(a, f64, b->any_sigma, per_sm * b->num_sms, b->st));
    GridSync hs{};
    BCU(cudaMemcpyAsync(b->h_wres, b->wres, sizeof(WaveResult), cudaMemcpyDeviceToHost, b->st));
    BCU(cudaMemcpyAsync(&hs, b->sync, sizeof(GridSync), cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    *out = *b->h_wres;
    if (hs.err == HJB_ERR_TIMEOUT) return bfail(HJB_ERR_TIMEOUT, "batch tile kernel: a grid-wide wait exceeded its limit");
    if (hs.err != 0) return bfail(hs.err, "batch tile kernel: tile queue overflow (internal error)");
    return HJB_OK;
}

// FP64 residuals of the instances (all, or those flagged in b->active); u64
// must hold the values.  res[i] is updated for the evaluated instances.
int stage_residual(hjb_batch* b, bool use_active, std::vector<double>& res, bool fields = false) {
    BCU(cudaMemsetAsync(b->res_bits, 0, sizeof(unsigned long long) * b->count, b->st));
    const size_t smem = residual_screened_smem(b->na, b->max_R);
    auto kern = b->any_sigma ? k_b_residual<true> : k_b_residual<false>;
    if (smem > 48 * 1024)
        BCU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    count_launches(1);
    kern<<<b->nrblk, dim3(kRX, kRBY), smem, b->st>>>(b->dinst, b->rblk, b->u64, b->margin,
                                                      use_active ? b->active : nullptr, b->res_bits,
                                                      fields ? b->corr_r : nullptr,
                                                      fields ? b->corr_a : nullptr);
    BCU(cudaGetLastError());
    std::vector<unsigned long long> bits(b->count);
    std::vector<uint8_t> act;
    if (use_active) {
        act.resize(b->count);
        BCU(cudaMemcpyAsync(act.data(), b->active, b->count, cudaMemcpyDeviceToHost, b->st));
    }
    BCU(cudaMemcpyAsync(bits.data(), b->res_bits, sizeof(unsigned long long) * b->count,
                        cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    res.resize(b->count);
    for (int i = 0; i < b->count; ++i) {
        if (use_active && !act[i]) continue;
        double v;
        std::memcpy(&v, &bits[i], sizeof(v));
        res[i] = v;
    }
    return HJB_OK;
}

// The FP64 stage by mixed-precision correction for the instances above tol64
// (scheme 3; every batch instance has a discount): per round, with the FP64
// residual r = T2 u - u and its minimising controls a (residual fields), FP32
// Jacobi sweeps of e = beta P_a e + r until each instance's sup-increment is below
// max(0.2 tol64, 2^-21 r_i / (1 - beta_i)), u += e in FP64, the residual again.
// Howard's policy iteration per instance: a round can raise an instance's
// residual where its minimising controls switch; an instance leaves after two
// rounds in a row that do not halve its residual, or if it grows past 1e3 times
// its first value (the FP64 passes then take it over).  The e buffers are the
// FP32 value arrays (u32, u32b), free once the values are in u64.
int stage_correction(hjb_batch* b, double tol64, int rounds, std::vector<double>& res, int* sweeps_out,
                     long long* nodes_out, int* n_res) {
    const int count = b->count;
    const size_t N = (size_t)b->N;
    if (!b->corr_r) {
        BCU(dalloc(b->corr_r, N, b->st));
        BCU(dalloc(b->corr_a, N, b->st));
        BCU(dalloc(b->corr_tol, (size_t)count, b->st));
        BCU(dalloc(b->corr_sel, (size_t)count, b->st));
    }
    constexpr int kMaxSweeps = 20000;
    const int big = 0x7fffffff;
    const std::vector<double> res0 = res;
    std::vector<int> stalled(count, 0);
    std::vector<uint8_t> sel(count);
    std::vector<float> tin(count);
    const size_t smem = (size_t)(kRX + 2 * b->max_R) * (kRY + 2 * b->max_R) * sizeof(float);
    auto kern = b->any_sigma ? k_b_corr_sweep<true> : k_b_corr_sweep<false>;
    if (smem > 48 * 1024)
        BCU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    bool fields = false;
    for (int round = 0; round < rounds; ++round) {
        int n_sel = 0;
        for (int i = 0; i < count; ++i) {
            sel[i] = res[i] > tol64 && stalled[i] < 2 && res[i] <= 1e3 * res0[i];
            n_sel += sel[i];
            const double omb = 1.0 - b->hinst[i].g.beta64;
            tin[i] = (float)std::max(0.2 * tol64, std::ldexp(res[i] / omb, -21));
        }
        if (n_sel == 0) break;
        BCU(cudaMemcpyAsync(b->corr_sel, sel.data(), count, cudaMemcpyHostToDevice, b->st));
        BCU(cudaMemcpyAsync(b->active, sel.data(), count, cudaMemcpyHostToDevice, b->st));
        if (!fields) {
            // residual fields of the selected instances (their residuals unchanged)
            std::vector<double> r2 = res;
            int rc = stage_residual(b, true, r2, true);
            if (rc) return rc;
            ++*n_res;
            fields = true;
        }
        BCU(cudaMemcpyAsync(b->corr_tol, tin.data(), sizeof(float) * count, cudaMemcpyHostToDevice, b->st));
        BCU(cudaMemsetAsync(b->u32, 0, sizeof(float) * N, b->st));
        BCU(cudaMemsetAsync(b->u32b, 0, sizeof(float) * N, b->st));
        BCU(cudaMemsetAsync(b->inc_bits, 0, sizeof(unsigned int) * count, b->st));
        std::vector<int> init(count, big);
        BCU(cudaMemcpyAsync(b->j_sweeps, init.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->st));
        int sweep = 0, h_active = n_sel;
        while (sweep < kMaxSweeps && h_active > 0) {
            const float* ein = (sweep & 1) ? b->u32b : b->u32;
            float* eout = (sweep & 1) ? b->u32 : b->u32b;
            count_launches(1);
            kern<<<b->nrblk, dim3(kRX, kRBY), smem, b->st>>>(b->dinst, b->rblk, b->corr_r, b->corr_a, ein, eout,
                                                              b->active, b->inc_bits);
            ++sweep;
            BCU(cudaMemsetAsync(b->n_active, 0, sizeof(int), b->st));
            count_launches(1);
            k_b_corr_mark<<<(count + 255) / 256, 256, 0, b->st>>>(count, b->corr_tol, sweep, b->active,
                                                                b->inc_bits, b->j_sweeps, b->n_active);
            BCU(cudaGetLastError());
            if ((sweep & 15) == 0 || sweep == kMaxSweeps) {
                BCU(cudaMemcpyAsync(&h_active, b->n_active, sizeof(int), cudaMemcpyDeviceToHost, b->st));
                BCU(cudaStreamSynchronize(b->st));
            }
        }
        std::vector<int> sw(count);
        BCU(cudaMemcpyAsync(sw.data(), b->j_sweeps, sizeof(int) * count, cudaMemcpyDeviceToHost, b->st));
        BCU(cudaStreamSynchronize(b->st));
        int smax = 0;
        for (int i = 0; i < count; ++i) {
            if (!sel[i]) continue;
            if (sw[i] == big) sw[i] = sweep;     // still moving: the last sweep's values
            smax = std::max(smax, sw[i]);
            *nodes_out += (long long)sw[i] * b->n_free[i];
        }
        *sweeps_out += smax;
        BCU(cudaMemcpyAsync(b->j_sweeps, sw.data(), sizeof(int) * count, cudaMemcpyHostToDevice, b->st));
        count_launches(1);
        k_b_add_corr<<<b->nfblk, kBT, 0, b->st>>>(b->dinst, b->fblk, b->u32, b->u32b, b->j_sweeps, b->corr_sel,
                                                  b->u64);
        BCU(cudaGetLastError());
        // the new residuals (and fields) of the round's instances
        BCU(cudaMemcpyAsync(b->active, sel.data(), count, cudaMemcpyHostToDevice, b->st));
        const std::vector<double> before = res;
        int rc = stage_residual(b, true, res, true);
        if (rc) return rc;
        ++*n_res;
        for (int i = 0; i < count; ++i)
            if (sel[i]) stalled[i] = res[i] < 0.5 * before[i] ? 0 : stalled[i] + 1;
    }
    return HJB_OK;
}

long long free_total(const hjb_batch* b) {
    long long s = 0;
    for (long long v : b->n_free) s += v;
    return s;
}

void fill_stats(hjb_stats* st) {
    if (st) std::memset(st, 0, sizeof(*st));
}

}  // namespace

extern "C" {

int hjb_batch_solve(hjb_batch* b, double tol_c, double tol32, double tol64, int32_t max_passes,
                    hjb_stats* stats, double* residuals) {
    clear_last_error();
    fill_stats(stats);
    if (!b) return bfail(HJB_ERR_INVALID_ARG, "batch is NULL");
    if (!(tol_c > 0.0) || !(tol32 > 0.0) || !(tol64 >= 0.0) || max_passes < 1)
        return bfail(HJB_ERR_INVALID_ARG, "bad tolerances / max_passes");
    double ms_coarse = 0, ms_pre = 0, ms32 = 0, ms_res = 0, ms64 = 0;
    long long nodes_c = 0;
    bool conv_c = true;
    int rc;
    {
        BTimer t(b->st);
        rc = stage_coarse(b, tol_c, 100000, &nodes_c, &conv_c);
        if (rc) return rc;
        ms_coarse = t.stop();
    }
    {
        BTimer t(b->st);
        rc = stage_precompute(b);
        if (rc) return rc;
        rc = stage_tiles(b);
        if (rc) return rc;
        ms_pre = t.stop();
    }
    WaveResult w32{};
    double umax = 1.0;
    for (double v : b->uob) umax = std::max(umax, v);
    tol32 = std::max(tol32, fp32_tol_floor(umax));
    {
        BTimer t(b->st);
        rc = stage_passes(b, false, tol32, max_passes, false, &w32);
        if (rc) return rc;
        ms32 = t.stop();
    }
    std::vector<double> res(b->count, 0.0);
    int n_res = 0;
    unsigned long long nodes64 = 0;
    int passes64 = 0;
    int corr_sweeps = 0;
    long long corr_nodes = 0;
    if (tol64 > 0.0) {
        BTimer t(b->st);
        count_launches(1);
        k_b_promote<<<b->nfblk, kBT, 0, b->st>>>(b->dinst, b->fblk, b->u32, b->u32, nullptr, b->u64);
        BCU(cudaGetLastError());
        b->value_f64 = true;
        rc = stage_residual(b, false, res);
        if (rc) return rc;
        ++n_res;
        ms_res += t.stop();
        // instances above tol64 first continue in FP32 from their current value
        // with tighter tolerances (warm: every tile of theirs visited once, then
        // the queues), as far as FP32 can resolve tol64
        double tol_w = tol32;
        for (int tries = 0; tries < 2 && 0.25 * tol_w >= fp32_tol_floor(umax); ++tries) {
            std::vector<uint8_t> act(b->count);
            int n_act = 0;
            for (int i = 0; i < b->count; ++i) {
                act[i] = res[i] > tol64 && tol64 >= 4.0 * fp32_tol_floor(b->uob[i]);
                n_act += act[i];
            }
            if (n_act == 0) break;
            tol_w *= 0.25;
            BCU(cudaMemcpyAsync(b->active, act.data(), b->count, cudaMemcpyHostToDevice, b->st));
            BTimer tw(b->st);
            WaveResult ww{};
            rc = stage_passes(b, false, tol_w, max_passes, true, &ww, true);
            if (rc) return rc;
            w32.passes += ww.passes;
            w32.nodes += ww.nodes;
            ms32 += tw.stop();
            BTimer tr(b->st);
            count_launches(1);
            k_b_promote<<<b->nfblk, kBT, 0, b->st>>>(b->dinst, b->fblk, b->u32, b->u32, nullptr, b->u64);
            BCU(cudaGetLastError());
            rc = stage_residual(b, true, res);
            if (rc) return rc;
            ++n_res;
            ms_res += tr.stop();
        }
        // mixed-precision correction rounds (scheme 3)
        if (b->scheme == 3) {
            BTimer tc(b->st);
            rc = stage_correction(b, tol64, 12, res, &corr_sweeps, &corr_nodes, &n_res);
            if (rc) return rc;
            ms64 += tc.stop();
        }
        // FP64 passes for the instances still above tol64
        double tol_pass = tol64;
        for (int round = 0; round < 4; ++round) {
            std::vector<uint8_t> act(b->count);
            int n_act = 0;
            for (int i = 0; i < b->count; ++i) {
                act[i] = res[i] > tol64;
                n_act += act[i];
            }
            if (n_act == 0 || passes64 >= max_passes) break;
            BCU(cudaMemcpyAsync(b->active, act.data(), b->count, cudaMemcpyHostToDevice, b->st));
            BTimer t2(b->st);
            WaveResult w64{};
            // warm: the instances' values are close to the fixed point already
            rc = stage_passes(b, true, tol_pass, max_passes - passes64, true, &w64, true);
            if (rc) return rc;
            passes64 += w64.passes;
            nodes64 += w64.nodes;
            ms64 += t2.stop();
            BTimer t3(b->st);
            rc = stage_residual(b, true, res);
            if (rc) return rc;
            ++n_res;
            ms_res += t3.stop();
            tol_pass *= 0.25;
        }
    }
    double rmax = 0.0;
    // with tol64 > 0 the FP64 residual decides (the FP32 phase may stop at its
    // visit caps and leave the rest to the FP64 stage)
    bool ok = conv_c && (tol64 > 0.0 || w32.converged);
    for (int i = 0; i < b->count; ++i) {
        rmax = std::max(rmax, res[i]);
        if (tol64 > 0.0 && res[i] > tol64) ok = false;
    }
    if (residuals)
        for (int i = 0; i < b->count; ++i) residuals[i] = tol64 > 0.0 ? res[i] : -1.0;
    rc = ok ? HJB_OK : HJB_ERR_NOT_CONVERGED;
    if (stats) {
        const long long nf = free_total(b);
        stats->sweeps = w32.passes + passes64;
        stats->fp32_passes = w32.passes;
        stats->fp64_passes = passes64;
        stats->node_updates = (long long)w32.nodes + (long long)nodes64 + corr_nodes;
        stats->fp64_node_updates = (long long)nodes64;
        // a correction sweep evaluates one control per node
        stats->node_control_updates =
            (nodes_c + (long long)w32.nodes + (long long)nodes64 + (long long)n_res * nf) * b->na + corr_nodes;
        stats->corr_sweeps = corr_sweeps;
        stats->residual_evals = n_res;
        stats->residual = tol64 > 0.0 ? rmax : -1.0;
        stats->increment = w32.last_increment;
        stats->ms_stage[0] = ms32;
        stats->ms_stage[1] = ms_res;
        stats->ms_stage[2] = ms64;
        stats->ms_stage[3] = ms_coarse;
        stats->ms_stage[4] = ms_pre;
        stats->ms_total = ms_coarse + ms_pre + ms32 + ms_res + ms64;
        stats->status = rc;
    }
    if (rc) bfail(rc, "batch solve did not converge (largest residual %.3e)", rmax);
    return rc;
}

int hjb_batch_autotune(hjb_batch* b, double tol_c, double tol32, int32_t* shape_out,
                       int32_t* waves_out, double* ms_out) {
    clear_last_error();
    if (!b) return bfail(HJB_ERR_INVALID_ARG, "batch is NULL");
    if (!(tol_c > 0.0) || !(tol32 > 0.0)) return bfail(HJB_ERR_INVALID_ARG, "bad tolerances");
    long long nc = 0;
    bool conv = true;
    int rc = stage_coarse(b, tol_c, 100000, &nc, &conv);
    if (rc) return rc;
    rc = stage_precompute(b);
    if (rc) return rc;
    double umax = 1.0;
    for (double v : b->uob) umax = std::max(umax, v);
    tol32 = std::max(tol32, fp32_tol_floor(umax));
    const int shapes[3] = {1, 2, 3};
    const int waves[2] = {1, 2};
    double best = 1e300;
    int bs = b->shape, bw = b->B;
    int c = 0;
    for (int si = 0; si < 3; ++si) {
        for (int wi = 0; wi < 2; ++wi, ++c) {
            b->shape = shapes[si];
            b->B = waves[wi];
            rc = stage_tiles(b);
            if (rc) return rc;
            BCU(cudaMemcpyAsync(b->u32, b->uhat, sizeof(float) * (size_t)b->N, cudaMemcpyDeviceToDevice,
                                b->st));
            BTimer t(b->st);
            WaveResult w{};
            rc = stage_passes(b, false, tol32, 100000, false, &w);
            if (rc) return rc;
            const double ms = t.stop();
            if (ms_out) ms_out[c] = ms;
            if (w.converged && ms < best) {
                best = ms;
                bs = b->shape;
                bw = b->B;
            }
        }
    }
    // the asynchronous worklist with each shape (one band per wave)
    bool ba = b->sched_mode == 3;
    const bool was_async = b->async;
    if (b->sched_mode == 0) {
        for (int si = 0; si < 3; ++si, ++c) {
            b->shape = shapes[si];
            b->B = 1;
            b->async = true;
            rc = stage_tiles(b);
            if (rc) return rc;
            BCU(cudaMemcpyAsync(b->u32, b->uhat, sizeof(float) * (size_t)b->N, cudaMemcpyDeviceToDevice,
                                b->st));
            BTimer t(b->st);
            WaveResult w{};
            rc = stage_passes(b, false, tol32, 100000, false, &w);
            b->async = was_async;
            if (rc) return rc;
            const double ms = t.stop();
            if (ms_out) ms_out[c] = ms;
            if (w.converged && ms < best) {
                best = ms;
                bs = b->shape;
                bw = 1;
                ba = true;
            }
        }
    }
    b->shape = bs;
    b->B = bw;
    b->async = ba;
    b->tuned = true;
    b->built = false;
    if (shape_out) *shape_out = bs - 1;
    if (waves_out) *waves_out = bw;
    return HJB_OK;
}

int hjb_batch_solve_full(hjb_batch* b, double tol32, double tol64, int32_t max_sweeps,
                         hjb_stats* stats, double* residuals) {
    clear_last_error();
    fill_stats(stats);
    if (!b) return bfail(HJB_ERR_INVALID_ARG, "batch is NULL");
    if (!(tol32 > 0.0) || !(tol64 >= 0.0) || max_sweeps < 1)
        return bfail(HJB_ERR_INVALID_ARG, "bad tolerances / max_sweeps");
    double umax = 1.0;
    for (double v : b->uob) umax = std::max(umax, v);
    tol32 = std::max(tol32, fp32_tol_floor(umax));
    BTimer t(b->st);
    count_launches(1);
    k_b_init_zero<<<b->nfblk, kBT, 0, b->st>>>(b->dinst, b->fblk, b->u32, b->u32b);
    BCU(cudaMemsetAsync(b->active, 1, b->count, b->st));
    BCU(cudaMemsetAsync(b->inc_bits, 0, sizeof(unsigned int) * b->count, b->st));
    const int big = 0x7fffffff;
    std::vector<int> init_sweeps(b->count, big);
    BCU(cudaMemcpyAsync(b->j_sweeps, init_sweeps.data(), sizeof(int) * b->count, cudaMemcpyHostToDevice,
                        b->st));
    const size_t smem = (((size_t)b->na * sizeof(float2) + 15) & ~(size_t)15) +
                        (size_t)(kRX + 2 * b->max_R) * (kRY + 2 * b->max_R) * sizeof(float);
    auto kern = b->any_sigma ? k_b_jacobi<true> : k_b_jacobi<false>;
    if (smem > 48 * 1024)
        BCU(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    int sweep = 0;
    int h_active = b->count;
    while (sweep < max_sweeps && h_active > 0) {
        const float* uin = (sweep & 1) ? b->u32b : b->u32;
        float* uout = (sweep & 1) ? b->u32 : b->u32b;
        count_launches(1);
        kern<<<b->nrblk, dim3(kRX, kRBY), smem, b->st>>>(b->dinst, b->rblk, b->scheme, uin, uout,
                                                          b->active, b->inc_bits);
        ++sweep;
        BCU(cudaMemsetAsync(b->n_active, 0, sizeof(int), b->st));
        count_launches(1);
        k_b_jacobi_mark<<<(b->count + 255) / 256, 256, 0, b->st>>>(b->count, (float)tol32, sweep, b->active,
                                                                   b->inc_bits, b->j_sweeps, b->n_active);
        BCU(cudaGetLastError());
        if ((sweep & 15) == 0 || sweep == max_sweeps) {
            BCU(cudaMemcpyAsync(&h_active, b->n_active, sizeof(int), cudaMemcpyDeviceToHost, b->st));
            BCU(cudaStreamSynchronize(b->st));
        }
    }
    std::vector<int> sw(b->count);
    BCU(cudaMemcpyAsync(sw.data(), b->j_sweeps, sizeof(int) * b->count, cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    // unconverged instances: their latest values are those of the last sweep
    long long nodes = 0;
    int smax = 0;
    bool conv = true;
    for (int i = 0; i < b->count; ++i) {
        if (sw[i] == big) {
            sw[i] = sweep;
            conv = false;
        }
        nodes += (long long)sw[i] * b->n_free[i];
        smax = std::max(smax, sw[i]);
    }
    BCU(cudaMemcpyAsync(b->j_sweeps, sw.data(), sizeof(int) * b->count, cudaMemcpyHostToDevice, b->st));
    count_launches(1);
    k_b_promote<<<b->nfblk, kBT, 0, b->st>>>(b->dinst, b->fblk, b->u32, b->u32b, b->j_sweeps, b->u64);
    BCU(cudaGetLastError());
    b->value_f64 = true;
    const double ms32 = t.stop();
    std::vector<double> res(b->count, 0.0);
    double ms_res = 0.0;
    int n_res = 0;
    if (tol64 > 0.0) {
        BTimer t2(b->st);
        int rc = stage_residual(b, false, res);
        if (rc) return rc;
        ++n_res;
        ms_res = t2.stop();
    }
    double rmax = 0.0;
    for (int i = 0; i < b->count; ++i) {
        rmax = std::max(rmax, res[i]);
        if (tol64 > 0.0 && res[i] > tol64) conv = false;
    }
    if (residuals)
        for (int i = 0; i < b->count; ++i) residuals[i] = tol64 > 0.0 ? res[i] : -1.0;
    const int rc = conv ? HJB_OK : HJB_ERR_NOT_CONVERGED;
    if (stats) {
        stats->sweeps = smax;
        stats->fp32_passes = smax;
        stats->node_updates = nodes;
        stats->node_control_updates = (nodes + (long long)n_res * free_total(b)) * b->na;
        stats->residual_evals = n_res;
        stats->residual = tol64 > 0.0 ? rmax : -1.0;
        stats->ms_stage[0] = ms32;
        stats->ms_stage[1] = ms_res;
        stats->ms_total = ms32 + ms_res;
        stats->status = rc;
    }
    if (rc) bfail(rc, "batch Jacobi did not converge (largest residual %.3e)", rmax);
    return rc;
}

int hjb_batch_get_value(const hjb_batch* b, int32_t index, double* u_out) {
    clear_last_error();
    if (!b || !u_out) return bfail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (index < 0 || index >= b->count) return bfail(HJB_ERR_INVALID_ARG, "index %d out of range", index);
    const long long o = b->node_off[index], n = b->node_off[index + 1] - o;
    if (b->value_f64) {
        BCU(cudaMemcpyAsync(u_out, b->u64 + o, sizeof(double) * n, cudaMemcpyDeviceToHost, b->st));
        BCU(cudaStreamSynchronize(b->st));
    } else {
        std::vector<float> h(n);
        BCU(cudaMemcpyAsync(h.data(), b->u32 + o, sizeof(float) * n, cudaMemcpyDeviceToHost, b->st));
        BCU(cudaStreamSynchronize(b->st));
        for (long long k = 0; k < n; ++k) u_out[k] = h[k];
    }
    return HJB_OK;
}

int hjb_batch_get_values(const hjb_batch* b, double* u_out) {
    clear_last_error();
    if (!b || !u_out) return bfail(HJB_ERR_INVALID_ARG, "NULL argument");
    const long long n = b->node_off[b->count];
    if (b->value_f64) {
        BCU(cudaMemcpyAsync(u_out, b->u64, sizeof(double) * n, cudaMemcpyDeviceToHost, b->st));
        BCU(cudaStreamSynchronize(b->st));
    } else {
        std::vector<float> h(n);
        BCU(cudaMemcpyAsync(h.data(), b->u32, sizeof(float) * n, cudaMemcpyDeviceToHost, b->st));
        BCU(cudaStreamSynchronize(b->st));
        for (long long k = 0; k < n; ++k) u_out[k] = h[k];
    }
    return HJB_OK;
}

int hjb_batch_get_feedback(const hjb_batch* b, int32_t index, uint8_t* a_out) {
    clear_last_error();
    if (!b || !a_out) return bfail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (index < 0 || index >= b->count) return bfail(HJB_ERR_INVALID_ARG, "index %d out of range", index);
    const long long o = b->node_off[index], n = b->node_off[index + 1] - o;
    BCU(cudaMemcpyAsync(a_out, b->a + o, n, cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    return HJB_OK;
}

int hjb_batch_get_labels(const hjb_batch* b, int32_t index, int8_t* label_out) {
    clear_last_error();
    if (!b || !label_out) return bfail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (index < 0 || index >= b->count) return bfail(HJB_ERR_INVALID_ARG, "index %d out of range", index);
    const long long o = b->node_off[index], n = b->node_off[index + 1] - o;
    BCU(cudaMemcpyAsync(label_out, b->label + o, n, cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    return HJB_OK;
}

int hjb_batch_get_uhat(const hjb_batch* b, int32_t index, float* uhat_out) {
    clear_last_error();
    if (!b || !uhat_out) return bfail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (index < 0 || index >= b->count) return bfail(HJB_ERR_INVALID_ARG, "index %d out of range", index);
    const long long o = b->node_off[index], n = b->node_off[index + 1] - o;
    BCU(cudaMemcpyAsync(uhat_out, b->uhat + o, sizeof(float) * n, cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    return HJB_OK;
}

}  // extern "C"

// ------------------------------------------------------ warm-start support
namespace {
int same_coarse_size(const hjb_batch* b) {
    const int nc = b->desc[0].coarse_n;
    for (const auto& x : b->desc)
        if (x.coarse_n != nc) return 0;
    return nc;
}
}  // namespace

extern "C" {

int hjb_batch_net_inputs(const hjb_batch* b, void* x) {
    clear_last_error();
    if (!b || !x) return bfail(HJB_ERR_INVALID_ARG, "NULL argument");
    const int nc = same_coarse_size(b);
    if (!nc) return bfail(HJB_ERR_INVALID_ARG, "instances have different coarse sizes");
    count_launches(1);
    k_b_net_inputs<<<b->ncblk, kBT, 0, b->st>>>(b->dinst, b->cblk, nc, reinterpret_cast<__nv_bfloat16*>(x));
    BCU(cudaGetLastError());
    BCU(cudaStreamSynchronize(b->st));
    return HJB_OK;
}

int hjb_batch_coarse_warm(hjb_batch* b, const float* net_out, int32_t first, int32_t count,
                          int32_t k_sweeps, double fallback_tol) {
    clear_last_error();
    if (!b) return bfail(HJB_ERR_INVALID_ARG, "batch is NULL");
    if (!net_out) {
        b->warm_on = false;
        return HJB_OK;
    }
    if (k_sweeps < 1 || !(fallback_tol > 0.0)) return bfail(HJB_ERR_INVALID_ARG, "bad k_sweeps / fallback_tol");
    if (first < 0 || count < 1 || first + count > b->count)
        return bfail(HJB_ERR_INVALID_ARG, "instances [%d, %d) out of range", first, first + count);
    const int nc = same_coarse_size(b);
    if (!nc) return bfail(HJB_ERR_INVALID_ARG, "instances have different coarse sizes");
    if (!b->coarse_init) {
        BCU(dalloc(b->coarse_init, (size_t)b->Nc, b->st));
        // instances without a prediction keep the plain start
        std::vector<float> plain((size_t)b->Nc);
        for (int i = 0; i < b->count; ++i)
            for (long long k = b->coarse_off[i]; k < b->coarse_off[i + 1]; ++k) plain[k] = b->hinst[i].uc0;
        BCU(cudaMemcpyAsync(b->coarse_init, plain.data(), sizeof(float) * plain.size(), cudaMemcpyHostToDevice,
                            b->st));
    }
    count_launches(1);
    k_b_warm_values<<<b->ncblk, kBT, 0, b->st>>>(b->dinst, b->cblk, nc, net_out, first, count, b->d_coarse_off,
                                                 b->coarse_init);
    BCU(cudaGetLastError());
    BCU(cudaStreamSynchronize(b->st));
    b->warm_on = true;
    b->warm_k = k_sweeps;
    b->warm_tol = fallback_tol;
    return HJB_OK;
}

int hjb_batch_coarse_solve(hjb_batch* b, double tol_c, int32_t max_sweeps, hjb_stats* stats,
                           int32_t* sweeps_out, uint8_t* fallback_out) {
    clear_last_error();
    fill_stats(stats);
    if (!b) return bfail(HJB_ERR_INVALID_ARG, "batch is NULL");
    if (!(tol_c > 0.0) || max_sweeps < 1) return bfail(HJB_ERR_INVALID_ARG, "bad tol_c / max_sweeps");
    BTimer t(b->st);
    long long nodes = 0;
    bool conv = true;
    int rc = stage_coarse(b, tol_c, max_sweeps, &nodes, &conv);
    if (rc) return rc;
    const double ms = t.stop();
    if (sweeps_out)
        BCU(cudaMemcpyAsync(sweeps_out, b->c_sweeps, sizeof(int) * b->count, cudaMemcpyDeviceToHost, b->st));
    if (fallback_out) BCU(cudaMemcpyAsync(fallback_out, b->c_fallback, b->count, cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    rc = conv ? HJB_OK : HJB_ERR_NOT_CONVERGED;
    if (stats) {
        stats->node_updates = nodes;
        stats->node_control_updates = nodes * b->na;
        stats->ms_stage[3] = ms;
        stats->ms_total = ms;
        stats->status = rc;
    }
    return rc;
}

int hjb_batch_precompute(hjb_batch* b, double tol_c, hjb_stats* stats) {
    clear_last_error();
    fill_stats(stats);
    if (!b) return bfail(HJB_ERR_INVALID_ARG, "batch is NULL");
    if (!(tol_c > 0.0)) return bfail(HJB_ERR_INVALID_ARG, "bad tol_c");
    BTimer t(b->st);
    long long nodes = 0;
    bool conv = true;
    int rc = stage_coarse(b, tol_c, 100000, &nodes, &conv);
    if (rc) return rc;
    rc = stage_precompute(b);
    if (rc) return rc;
    BCU(cudaStreamSynchronize(b->st));
    const double ms = t.stop();
    if (stats) {
        stats->node_updates = nodes;
        stats->node_control_updates = nodes * b->na;
        stats->ms_total = ms;
        stats->status = conv ? HJB_OK : HJB_ERR_NOT_CONVERGED;
    }
    return conv ? HJB_OK : HJB_ERR_NOT_CONVERGED;
}

int hjb_batch_net_targets(const hjb_batch* b, float* tval, uint8_t* tctrl, uint8_t* freem) {
    clear_last_error();
    if (!b || !tval || !tctrl || !freem) return bfail(HJB_ERR_INVALID_ARG, "NULL argument");
    const int nc = same_coarse_size(b);
    if (!nc) return bfail(HJB_ERR_INVALID_ARG, "instances have different coarse sizes");
    count_launches(1);
    k_b_net_targets<<<b->ncblk, kBT, 0, b->st>>>(b->dinst, b->cblk, nc, tval, tctrl, freem);
    BCU(cudaGetLastError());
    BCU(cudaStreamSynchronize(b->st));
    return HJB_OK;
}

int hjb_batch_get_coarse_value(const hjb_batch* b, int32_t index, float* uc_out) {
    clear_last_error();
    if (!b || !uc_out) return bfail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (index < 0 || index >= b->count) return bfail(HJB_ERR_INVALID_ARG, "index %d out of range", index);
    const long long o = b->coarse_off[index], n = b->coarse_off[index + 1] - o;
    BCU(cudaMemcpyAsync(uc_out, b->uc + o, sizeof(float) * n, cudaMemcpyDeviceToHost, b->st));
    BCU(cudaStreamSynchronize(b->st));
    return HJB_OK;
}

}  // extern "C"
