// Computation step of the patchy algorithm (Cacace & Falcone, Section 4.3):
// the free nodes, sorted by (causal band, patch) from u_hat (Section 4.2),
// are updated in place with eq. SLscheme3 on one shared array -- the
// patches share sharp interfaces, so the transmission condition
// u_p = min(u_p, u_q) is the identity -- in increasing band order.  A group of
// `group` consecutive bands is one grid-wide wave whose nodes are taken in
// sorted order, round-robin over the warps in flight (so a node is updated
// about one launch-width of nodes after its predecessors in the order): a warp
// per node, its lanes spread over the controls, the min taken by warp
// shuffles.  A persistent cooperative kernel separates the waves with a bounded
// grid barrier; passes are repeated until a pass's sup-increment is below the
// tolerance, and after the first pass a group is revisited only if a group
// within `window` of it changed by more than the tolerance (in the previous
// pass, or earlier in this pass for upwind groups).
//
// Values written by other SMs during the kernel are read through L2
// (ld.global.cg), never from a possibly stale L1 line.
#include <algorithm>
#include "hjb_kernels.h"

namespace hjb {

namespace {

constexpr int kWaveThreads = 256;
constexpr int kWarps = kWaveThreads / 32;

__device__ __forceinline__ float ld_l2(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_l2(const double* p) { return __ldcg(p); }
__device__ __forceinline__ void st_l2(float* p, float v) { __stcg(p, v); }
__device__ __forceinline__ void st_l2(double* p, double v) { __stcg(p, v); }

__device__ __forceinline__ float inc_to_float(float v) { return v; }
__device__ __forceinline__ float inc_to_float(double v) { return __double2float_ru(v); }

template <typename T, bool SIG>
__global__ void __launch_bounds__(kWaveThreads)
k_waves(WaveArgs a, T* u) {
    using V2 = typename RealOf<T>::V2;
    extern __shared__ __align__(16) unsigned char smem[];
    V2* sctrl = reinterpret_cast<V2*>(smem);
    __shared__ float red[32];
    __shared__ int s_flag;
    __shared__ unsigned long long s_nodes;

    const GridView& g = a.g;
    const int n = g.n;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    // consecutive nodes of a wave go to different blocks (SMs) first
    const int gw = warp * gridDim.x + blockIdx.x;
    const int nw = gridDim.x * kWarps;
    const unsigned int nblocks = gridDim.x;
    const unsigned int tol_bits = __float_as_uint(a.tol);

    for (int m = threadIdx.x; m < g.na; m += blockDim.x) sctrl[m] = RealOf<T>::ctrl(g, m);
    if (threadIdx.x == 0) s_nodes = 0ull;
    __syncthreads();
    auto C = [&](int m) { return sctrl[m]; };

    int pass = 0;
    int converged = 0;
    float pass_max = 0.0f;
    bool ok = true;
    for (pass = 0; pass < a.max_passes && ok; ++pass) {
        unsigned int* cur = a.inc_bits + (size_t)(pass & 1) * a.n_groups;
        const unsigned int* prev = a.inc_bits + (size_t)((pass + 1) & 1) * a.n_groups;
        // clear this pass's per-group maxima (nobody reads them before the barrier)
        for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < a.n_groups; q += gridDim.x * blockDim.x)
            cur[q] = 0u;
        ok = grid_sync(a.sync, nblocks, a.timeout_ns);
        if (!ok) break;

        for (int q = 0; q < a.n_groups; ++q) {
            const int beg = a.band_off[q * a.group];
            const int end = a.band_off[min((q + 1) * a.group, a.n_bands)];
            if (beg == end) continue;
            if (pass > 0) {
                // activity test, identical in every block (it reads values fixed
                // before the last barrier)
                if (threadIdx.x == 0) s_flag = 0;
                __syncthreads();
                const int lo = max(q - a.window, 0);
                const int hi = min(q + a.window, a.n_groups - 1);
                for (int t = lo + (int)threadIdx.x; t <= hi; t += blockDim.x) {
                    if (__ldcg(prev + t) > tol_bits || (t < q && __ldcg(cur + t) > tol_bits))
                        s_flag = 1;
                }
                __syncthreads();
                if (!s_flag) continue;
            }
            // nodes of the group in sorted order, round-robin over the warps in flight
            float lmax = 0.0f;
            unsigned long long cnt = 0;
            for (int t = beg + gw; t < end; t += nw) {
                const int k = a.order[t];
                const int i = k % n, j = k / n;
                const T uk = ld_l2(u + k);
                const T c = (T)g.speed[k];
                T bx = T(0), by = T(0);
                if (g.drift) {
                    const float2 bb = g.drift[k];
                    bx = (T)bb.x;
                    by = (T)bb.y;
                }
                const T* base = u + k;
                auto U = [&](int dx, int dy) { return ld_l2(base + (ptrdiff_t)dy * n + dx); };
                T N, D;
                int M;
                best_over_controls<T, SIG>(g, a.scheme, i, j, uk, c, bx, by, lane, 32, C, U, N, D, M);
                warp_argmin<T>(N, D, M);
                const T du = N / D;
                if (lane == 0) {
                    st_l2(u + k, uk + du);
                    ++cnt;
                }
                lmax = fmaxf(lmax, inc_to_float(fabs(du)));
            }
            if (lane == 0 && cnt) atomicAdd(&s_nodes, cnt);
            const float bm = block_max<float>(lmax, red);
            if (threadIdx.x == 0 && bm > 0.0f) atomicMax(cur + q, __float_as_uint(bm));
            ok = grid_sync(a.sync, nblocks, a.timeout_ns);
            if (!ok) break;
        }
        if (!ok) break;
        // all waves of the pass are done in every block: the maxima are final
        ok = grid_sync(a.sync, nblocks, a.timeout_ns);
        if (!ok) break;
        float lm = 0.0f;
        for (int t = threadIdx.x; t < a.n_groups; t += blockDim.x)
            lm = fmaxf(lm, __uint_as_float(__ldcg(cur + t)));
        pass_max = block_max<float>(lm, red);
        if (threadIdx.x == 0) s_flag = (pass_max <= a.tol) ? 1 : 0;
        __syncthreads();
        if (s_flag) {
            converged = 1;
            ++pass;
            break;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&a.res->nodes, s_nodes);
        if (blockIdx.x == 0) {
            a.res->passes = pass;
            a.res->converged = converged;
            a.res->last_increment = pass_max;
        }
    }
}

// Coarse-grid relaxation in one cooperative launch (the coarse solve of
// Section 4.3, eq. SLscheme3 with sigma = 0): block b owns a fixed TW x TH tile
// of G_c and keeps the tile's speed, drift and mask in shared memory for the
// whole solve.  A global sweep stages the tile and a halo of R cells from u,
// runs `local_sweeps` in-place relaxations of the tile (alternating direction;
// a warp per node, lanes over the controls), writes the tile back and meets the
// other blocks at the grid barrier.  Information thus crosses a whole tile per
// global sweep.  The solve stops once the first local sweep after a staging --
// the increment of the operator on the staged field -- is <= tol everywhere.
// Without diffusion (the coarse problem) the geometry of every (node, control)
// pair -- the foot's cell in the window, its fractions and 1/(1 - beta L) --
// does not change across sweeps; when it fits (a.pre) it is formed once into
// shared memory and a candidate costs four loads and three FMAs.
constexpr int kRelaxThreads = 512;
constexpr int kRelaxWarps = kRelaxThreads / 32;
constexpr int kRelaxTW = 16;    // tile width (a power of two: node coordinates by shifts)

struct RelaxGeo {
    float fx, fy;   // fractions of the foot in its cell
    float rd;       // 1 / (1 - beta L), 0 when the candidate is excluded (D <= 0)
    int off;        // window offset of the cell's lower-left vertex from the node
};

__host__ __device__ inline size_t relax_tile_bytes(int tw, int th, int R, int na, bool pre) {
    const size_t ctrl = ((size_t)na * sizeof(float2) + 15) & ~(size_t)15;
    const size_t win = (((size_t)(tw + 2 * R) * (th + 2 * R) * sizeof(float)) + 15) & ~(size_t)15;
    const size_t per = (size_t)tw * th;
    const size_t geo = pre ? per * na * sizeof(RelaxGeo) + per * sizeof(float) : 0;
    return ctrl + geo + win + per * (sizeof(float2) + sizeof(float)) + ((per + 15) & ~(size_t)15);
}

template <bool SIG>
__global__ void __launch_bounds__(kRelaxThreads)
k_grid_relax(RelaxArgs a, float* u) {
    extern __shared__ __align__(16) unsigned char smem[];
    const GridView& g = a.g;
    const int n = g.n;
    constexpr int TW = kRelaxTW;
    const int TH = a.th, R = a.halo;
    const int W = TW + 2 * R, H = TH + 2 * R;
    const int P = TW * TH;
    float2* sctrl = reinterpret_cast<float2*>(smem);
    const bool pre = !SIG && a.pre;
    RelaxGeo* sgeo = reinterpret_cast<RelaxGeo*>(smem + (((size_t)g.na * sizeof(float2) + 15) & ~(size_t)15));
    float* shl = reinterpret_cast<float*>(sgeo + (pre ? (size_t)P * g.na : 0));   // h l(x) per node
    unsigned char* p0 = reinterpret_cast<unsigned char*>(shl + (pre ? P : 0));
    float* su = reinterpret_cast<float*>(p0);
    unsigned char* p1 = p0 + ((((size_t)W * H * sizeof(float)) + 15) & ~(size_t)15);
    float2* sdrift = reinterpret_cast<float2*>(p1);
    float* sspeed = reinterpret_cast<float*>(p1 + (size_t)P * sizeof(float2));
    uint8_t* smask = reinterpret_cast<uint8_t*>(p1 + (size_t)P * (sizeof(float2) + sizeof(float)));
    __shared__ float red[32];
    __shared__ int s_flag;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int bi = (blockIdx.x % a.ntx) * TW, bj = (blockIdx.x / a.ntx) * TH;
    const int gx0 = bi - R, gy0 = bj - R;
    for (int m = threadIdx.x; m < g.na; m += blockDim.x) sctrl[m] = g.ctrl32[m];
    for (int e = threadIdx.x; e < P; e += blockDim.x) {
        const int i = bi + e % TW, j = bj + e / TW;
        const bool in = i < n && j < n;
        const size_t k = in ? (size_t)j * n + i : 0;
        smask[e] = in ? g.mask[k] : (uint8_t)kTarget;    // outside the grid: never updated
        sspeed[e] = in ? g.speed[k] : 0.0f;
        sdrift[e] = (in && g.drift) ? g.drift[k] : make_float2(0.0f, 0.0f);
    }
    auto C = [&](int m) { return sctrl[m]; };
    const float beta = g.beta32;
    __syncthreads();
    if (pre) {
        // the geometry of eq. SLscheme3 with sigma = 0 per (node, control), as
        // control_terms4 / candidate form it
        for (int q = threadIdx.x; q < P * g.na; q += blockDim.x) {
            const int e = q / g.na, m = q - e * g.na;
            RelaxGeo r{0.0f, 0.0f, 0.0f, 0};
            if (smask[e] == kFree) {
                const int i = bi + e % TW, j = bj + e / TW;
                const NodeBox<float> box = node_box<float>(i, j, n);
                const float2 ac = sctrl[m];
                const float2 b = sdrift[e];
                const float fx = g.s32 * fmaf(sspeed[e], ac.x, b.x);
                const float fy = g.s32 * fmaf(sspeed[e], ac.y, b.y);
                const Axis<float> x0 = axis_cell<float, true>(fx, box.lox, box.hix, box.capx);
                const Axis<float> y0 = axis_cell<float, true>(fy, box.loy, box.hiy, box.capy);
                const float D = fmaf(-beta, x0.sw * y0.sw, 1.0f);
                r.fx = x0.fr;
                r.fy = y0.fr;
                r.rd = D > 0.0f ? 1.0f / D : 0.0f;
                r.off = y0.off * W + x0.off;
            }
            sgeo[q] = r;
        }
        for (int e = threadIdx.x; e < P; e += blockDim.x) {
            const int i = bi + e % TW, j = bj + e / TW;
            shl[e] = (g.costf && smask[e] == kFree) ? g.h32 * g.costf[(size_t)j * n + i] : g.hl32;
        }
    }
    int s = 0;
    int converged = 0;
    float last = 0.0f;
    for (s = 0; s < a.max_sweeps; ++s) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.sweep_inc[(s + 1) % 3] = 0u;
            a.sweep_umax[(s + 1) % 3] = 0u;
        }
        for (int e = threadIdx.x; e < W * H; e += blockDim.x) {
            const int gx = min(max(gx0 + e % W, 0), n - 1);
            const int gy = min(max(gy0 + e / W, 0), n - 1);
            su[e] = __ldcg(u + (size_t)gy * n + gx);
        }
        __syncthreads();
        float lmax = 0.0f, umax = 0.0f;
        for (int ls = 0; ls < a.local_sweeps; ++ls) {
            for (int t = warp; t < P; t += kRelaxWarps) {
                const int e = ((s + ls) & 1) ? (P - 1 - t) : t;
                if (smask[e] != kFree) continue;
                const int ex = e % TW, ey = e / TW;
                float* base = su + (R + ey) * W + (R + ex);
                const float uk = base[0];
                float du;
                if (pre) {
                    // (beta Sd + h l - (1 - beta) uk + h m) / D, lanes over the controls
                    const float c0 = fmaf(-(1.0f - beta), uk, shl[e]);
                    float v = INFINITY;
                    for (int m = lane; m < g.na; m += 32) {
                        const RelaxGeo r = sgeo[e * g.na + m];
                        const float* q = base + r.off;
                        const float a0 = fmaf(r.fx, q[1] - q[0], q[0] - uk);
                        const float a1 = fmaf(r.fx, q[W + 1] - q[W], q[W] - uk);
                        const float Sd = fmaf(r.fy, a1 - a0, a0);
                        const float cm = g.hm32 ? c0 + g.hm32[m] : c0;
                        const float N = fmaf(beta, Sd, cm);
                        if (r.rd > 0.0f) v = fminf(v, N * r.rd);
                    }
                    du = order_val(__reduce_min_sync(0xffffffffu, order_key(v)));
                } else {
                    const float2 b = sdrift[e];
                    auto U = [&](int dx, int dy) { return base[dy * W + dx]; };
                    float Nn, D;
                    int M;
                    best_over_controls<float, SIG>(g, 3, bi + ex, bj + ey, uk, sspeed[e], b.x, b.y, lane, 32,
                                                   C, U, Nn, D, M);
                    du = warp_min_increment(Nn, D, M);
                }
                __syncwarp();
                if (lane == 0) base[0] = uk + du;
                if (ls == 0) lmax = fmaxf(lmax, fabsf(du));
                if (ls == a.local_sweeps - 1) umax = fmaxf(umax, fabsf(uk + du));
            }
            __syncthreads();
        }
        for (int e = threadIdx.x; e < P; e += blockDim.x) {
            if (smask[e] != kFree) continue;
            const int ex = e % TW, ey = e / TW;
            __stcg(u + (size_t)(bj + ey) * n + bi + ex, su[(R + ey) * W + (R + ex)]);
        }
        const float bm = block_max<float>(lmax, red);
        if (threadIdx.x == 0 && bm > 0.0f) atomicMax(a.sweep_inc + s % 3, __float_as_uint(bm));
        const float bu = block_max<float>(umax, red);
        if (threadIdx.x == 0 && bu > 0.0f) atomicMax(a.sweep_umax + s % 3, __float_as_uint(bu));
        if (!grid_sync(a.sync, gridDim.x, a.timeout_ns)) break;
        if (threadIdx.x == 0) {
            last = __uint_as_float(__ldcg(a.sweep_inc + s % 3));
            // FP32 floor of the largest free value: 1.01 ulp(max(1, U)) / 2 times
            // the amplification of the scheme's division
            const float Uv = __uint_as_float(__ldcg(a.sweep_umax + s % 3));
            const float tol = fmaxf(a.tol, 1.01f * 1.1920929e-7f * fmaxf(1.0f, Uv) * a.floor_amp);
            s_flag = last <= tol ? 1 : 0;
        }
        __syncthreads();
        if (s_flag) {
            converged = 1;
            ++s;
            break;
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.res->passes = s;
        a.res->converged = converged;
        a.res->last_increment = last;
    }
}

template <typename T, bool SIG>
cudaError_t launch_impl(const WaveArgs& a, T* u, int blocks, cudaStream_t st) {
    using V2 = typename RealOf<T>::V2;
    const size_t smem = (size_t)a.g.na * sizeof(V2);
    void* args[] = {(void*)&a, (void*)&u};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void*)k_waves<T, SIG>, dim3(blocks),
                                       dim3(kWaveThreads), args, smem, st);
}

template <typename T, bool SIG>
int blocks_per_sm_impl(int na) {
    using V2 = typename RealOf<T>::V2;
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_waves<T, SIG>, kWaveThreads,
                                                  (size_t)na * sizeof(V2));
    return nb;
}

}  // namespace

int wave_threads() { return kWaveThreads; }

int grid_relax_plan(int n, int na, int halo, int num_sms, bool sig, RelaxArgs* a) {
    // 16-wide tiles, as many rows per tile as it takes to give every block of
    // one co-resident wave a tile; the per-(node, control) geometry is kept in
    // shared memory when a plan with it exists
    const void* kern = sig ? (const void*)k_grid_relax<true> : (const void*)k_grid_relax<false>;
    // one block per SM where the tiles allow it: a second block on one SM would
    // make every other block wait for it at each barrier
    const int tw = kRelaxTW;
    const int ntx = (n + tw - 1) / tw;
    for (int pass = 0; pass < 2; ++pass)
    for (int pre = sig ? 0 : 1; pre >= 0; --pre) {
        for (int th = 8; th <= 4 * n; th = th < 16 ? th + 1 : 2 * th) {
            const size_t smem = relax_tile_bytes(tw, th, halo, na, pre != 0);
            if (smem > 200 * 1024) break;
            int per_sm = 0;
            if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kRelaxThreads, smem) != cudaSuccess)
                return 0;
            const int nty = (n + th - 1) / th;
            const int cap = pass == 0 ? std::min(per_sm, 1) * num_sms : per_sm * num_sms;
            if (per_sm > 0 && ntx * nty <= cap && (pass == 1 || th <= 32)) {
                a->tw = tw;
                a->th = th;
                a->ntx = ntx;
                a->halo = halo;
                a->pre = pre;
                return ntx * nty;
            }
        }
    }
    return 0;
}

cudaError_t launch_grid_relax(const RelaxArgs& a, float* u, bool sig, int blocks, cudaStream_t st) {
    const size_t smem = relax_tile_bytes(a.tw, a.th, a.halo, a.g.na, a.pre != 0);
    const void* kern = sig ? (const void*)k_grid_relax<true> : (const void*)k_grid_relax<false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {(void*)&a, (void*)&u};
    count_launches(1);
    return cudaLaunchCooperativeKernel(kern, dim3(blocks), dim3(kRelaxThreads), args, smem, st);
}

int grid_relax_threads() { return kRelaxThreads; }

size_t wave_smem(bool f64, int na) { return (size_t)na * (f64 ? sizeof(double2) : sizeof(float2)); }

int wave_blocks_per_sm(bool f64, bool sig, int na) {
    if (f64) return sig ? blocks_per_sm_impl<double, true>(na) : blocks_per_sm_impl<double, false>(na);
    return sig ? blocks_per_sm_impl<float, true>(na) : blocks_per_sm_impl<float, false>(na);
}

cudaError_t launch_waves_f32(const WaveArgs& a, float* u, bool sig, int blocks, cudaStream_t st) {
    return sig ? launch_impl<float, true>(a, u, blocks, st) : launch_impl<float, false>(a, u, blocks, st);
}

cudaError_t launch_waves_f64(const WaveArgs& a, double* u, bool sig, int blocks, cudaStream_t st) {
    return sig ? launch_impl<double, true>(a, u, blocks, st) : launch_impl<double, false>(a, u, blocks, st);
}

}  // namespace hjb
