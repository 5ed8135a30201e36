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

// Whole-grid relaxation in one cooperative launch (used for the coarse solve,
// Section 4.3): at the start of every sweep each block copies the whole value
// field into its shared memory (the coarse grid is small), then updates its
// share of the free nodes from that copy -- a warp per node, lanes over the
// controls -- and writes them back; the node order alternates between
// row-major and reverse; a grid barrier closes each sweep and the loop stops
// once a sweep's sup-increment is <= tol.  One block of kRelaxThreads per SM.
constexpr int kRelaxThreads = 1024;
constexpr int kRelaxWarps = kRelaxThreads / 32;

template <bool SIG>
__global__ void __launch_bounds__(kRelaxThreads)
k_grid_relax(RelaxArgs a, float* u) {
    extern __shared__ __align__(16) unsigned char smem[];
    const GridView& g = a.g;
    const int n = g.n;
    const int N = n * n;
    float2* sctrl = reinterpret_cast<float2*>(smem);
    float* su = reinterpret_cast<float*>(smem + (((size_t)g.na * sizeof(float2) + 15) & ~(size_t)15));
    __shared__ float red[32];
    __shared__ int s_flag;
    const int lane = threadIdx.x & 31;
    const int gw = (threadIdx.x >> 5) * gridDim.x + blockIdx.x;
    const int nw = gridDim.x * kRelaxWarps;
    for (int m = threadIdx.x; m < g.na; m += blockDim.x) sctrl[m] = g.ctrl32[m];
    auto C = [&](int m) { return sctrl[m]; };
    int s = 0;
    int converged = 0;
    float last = 0.0f;
    for (s = 0; s < a.max_sweeps; ++s) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.sweep_inc[(s + 1) % 3] = 0u;
            a.sweep_umax[(s + 1) % 3] = 0u;
        }
        for (int k = threadIdx.x; k < N; k += blockDim.x) su[k] = __ldcg(u + k);
        __syncthreads();
        float lmax = 0.0f, umax = 0.0f;
        for (int t = gw; t < N; t += nw) {
            const int k = (s & 1) ? (N - 1 - t) : t;
            if (g.mask[k] != kFree) continue;
            const int i = k % n, j = k / n;
            const float uk = su[k];
            const float c = g.speed[k];
            float bx = 0.0f, by = 0.0f;
            if (g.drift) {
                const float2 bb = g.drift[k];
                bx = bb.x;
                by = bb.y;
            }
            const float* base = su + k;
            auto U = [&](int dx, int dy) { return base[dy * n + dx]; };
            float Nn, D;
            int M;
            best_over_controls<float, SIG>(g, 3, i, j, uk, c, bx, by, lane, 32, C, U, Nn, D, M);
            const float du = warp_min_increment(Nn, D, M);
            if (lane == 0) __stcg(u + k, uk + du);
            lmax = fmaxf(lmax, fabsf(du));
            umax = fmaxf(umax, fabsf(uk + du));
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
            const float U = __uint_as_float(__ldcg(a.sweep_umax + s % 3));
            const float tol = fmaxf(a.tol, 1.01f * 1.1920929e-7f * fmaxf(1.0f, U) * a.floor_amp);
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

size_t grid_relax_smem(int n, int na) {
    return (((size_t)na * sizeof(float2) + 15) & ~(size_t)15) + (size_t)n * n * sizeof(float);
}

cudaError_t launch_grid_relax(const RelaxArgs& a, float* u, bool sig, int blocks, cudaStream_t st) {
    const size_t smem = grid_relax_smem(a.g.n, a.g.na);
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
