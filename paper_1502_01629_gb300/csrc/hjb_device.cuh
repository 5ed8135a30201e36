// Device-side building blocks of the solver: the per-control evaluation of the
// Markov-chain semi-Lagrangian scheme (Cacace & Falcone, Section 3, eqs.
// SLscheme2 / SLscheme3 and the 2-D isotropic form of Section 4.1), the
// warp-level argmin over controls, block reductions and the bounded grid-wide
// barrier used by the persistent band-wave kernel.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hjb.h"

namespace hjb {

constexpr int kFree = HJB_MASK_FREE;
constexpr int kTarget = HJB_MASK_TARGET;
constexpr int kObstacle = HJB_MASK_OBSTACLE;

// Everything a kernel needs to evaluate the scheme on one grid, by value.
struct GridView {
    int n;                  // nodes per side
    int na;                 // number of controls
    const float* speed;     // c(x), n*n
    const float2* drift;    // b(x), n*n, or nullptr
    const uint8_t* mask;    // n*n
    const float2* ctrl32;   // a_m in FP32
    const double2* ctrl64;  // a_m in FP64
    float s32;   double s64;     // h / dx
    float d32;   double d64;     // sqrt(2h) sigma / dx: diffusion offset in cells
    float beta32; double beta64; // 1 / (1 + lambda h)
    float hl32;  double hl64;    // h * l
    float uob32; double uob64;   // value held on obstacle nodes
    // General terms (Section 5.3); zero / null for a constant sigma and cost.
    int gen;                     // 1 when any of the fields below is in use
    int along;                   // diffusion sigma(x) a: two points along the control
    const float* sigf;           // sigma(x) per node, or nullptr (d32 / d64 everywhere)
    const float* costf;          // l(x) per node, or nullptr (hl32 / hl64 everywhere)
    const float* hm32;           // h m(a_m) per control, or nullptr (m = 0)
    const double* hm64;
    float du32;  double du64;    // sqrt(2h) / dx: offset in cells per unit of sigma
    float h32;   double h64;     // h
};

// The causal band map of the ordering (Section 4.2): band edges in FP64 (see
// band_key in precompute_device.cuh).
struct BandMap {
    float lambda;
    float w32;             // band width w = band_width h, FP32 (the estimate)
    double w64;            // the same in FP64
    const double* edges;   // L entries, edges[0] = 0 (unused)
    int n_edges;           // L (0 when lambda = 0)
    int cap;               // keys are capped at cap - 1
};

template <typename T> struct RealOf;
template <typename T> struct V2Of_;
template <> struct V2Of_<float> { using type = float2; };
template <> struct V2Of_<double> { using type = double2; };
template <typename T> using V2Of = typename V2Of_<T>::type;
template <> struct RealOf<float> {
    using V2 = float2;
    __device__ static float s(const GridView& g) { return g.s32; }
    __device__ static float d(const GridView& g) { return g.d32; }
    __device__ static float beta(const GridView& g) { return g.beta32; }
    __device__ static float hl(const GridView& g) { return g.hl32; }
    __device__ static float uob(const GridView& g) { return g.uob32; }
    __device__ static float2 ctrl(const GridView& g, int m) { return g.ctrl32[m]; }
    __device__ static float du(const GridView& g) { return g.du32; }
    __device__ static float h(const GridView& g) { return g.h32; }
    __device__ static float hm(const GridView& g, int m) { return g.hm32[m]; }
};
template <> struct RealOf<double> {
    using V2 = double2;
    __device__ static double s(const GridView& g) { return g.s64; }
    __device__ static double d(const GridView& g) { return g.d64; }
    __device__ static double beta(const GridView& g) { return g.beta64; }
    __device__ static double hl(const GridView& g) { return g.hl64; }
    __device__ static double uob(const GridView& g) { return g.uob64; }
    __device__ static double2 ctrl(const GridView& g, int m) { return g.ctrl64[m]; }
    __device__ static double du(const GridView& g) { return g.du64; }
    __device__ static double h(const GridView& g) { return g.h64; }
    __device__ static double hm(const GridView& g, int m) { return g.hm64[m]; }
};

// One axis of a point's Q1 cell, relative to the node: the point sits at offset
// `d` (grid units) from node index i.  The projection onto the square clamps the
// absolute coordinate to [0, n-1], i.e. the offset to [lo, hi] = [-i, n-1-i];
// the cell is floor(), capped at hi - 1 so that a point on the last grid line
// uses the last cell with fraction 1.  Working with the small offset keeps the
// fraction exact in FP32 at any grid size.  `sw` is the Q1 weight of node i
// along this axis: the hat function max(0, 1 - |d|) of the clamped offset (it
// equals 1 - fr when the cell starts at the node, fr when it ends there, 0
// otherwise).
template <typename T>
struct Axis {
    int off;
    T fr;
    T sw;
};

// Clamp bounds of the offsets around one node, computed once per node.
template <typename T>
struct NodeBox {
    T lox, hix, capx;   // capx = hix - 1
    T loy, hiy, capy;
};

template <typename T>
__device__ __forceinline__ NodeBox<T> node_box(int i, int j, int n) {
    NodeBox<T> b;
    b.lox = (T)(-i);
    b.hix = (T)(n - 1 - i);
    b.capx = b.hix - T(1);
    b.loy = (T)(-j);
    b.hiy = (T)(n - 1 - j);
    b.capy = b.hiy - T(1);
    return b;
}

// CLAMP = false: the caller guarantees lo < d < hi and floor(d) <= cap (the node
// lies at least the interpolation reach inside the grid), so the projection is
// the identity and is skipped.
template <typename T, bool CLAMP = true>
__device__ __forceinline__ Axis<T> axis_cell(T d, T lo, T hi, T cap) {
    if (CLAMP) d = fmin(fmax(d, lo), hi);
    T fl = floor(d);
    if (CLAMP) fl = fmin(fl, cap);
    Axis<T> a;
    a.off = (int)fl;
    a.fr = d - fl;
    a.sw = fmax(T(1) - fabs(d), T(0));
    return a;
}

// FP32: floor by rounding.  Adding 1.5 * 2^23 with rounding toward -infinity
// leaves floor(d) in the low mantissa bits of the sum (its ulp is 1) for
// |d| < 2^22; the integer is read from the bits and floor(d) as a float is the
// sum minus 1.5 * 2^23 (exact).  Same results as floor() and a conversion,
// computed on the FMA and integer pipes instead of the conversion unit.
template <>
__device__ __forceinline__ Axis<float> axis_cell<float, true>(float d, float lo, float hi, float cap) {
    constexpr float kRound = 12582912.0f;            // 1.5 * 2^23
    d = fminf(fmaxf(d, lo), hi);
    const float t = fminf(__fadd_rd(d, kRound), cap + kRound);
    Axis<float> a;
    a.off = __float_as_int(t) - 0x4B400000;          // bits of 1.5 * 2^23
    a.fr = d - (t - kRound);
    a.sw = fmaxf(1.0f - fabsf(d), 0.0f);
    return a;
}
template <>
__device__ __forceinline__ Axis<float> axis_cell<float, false>(float d, float, float, float) {
    constexpr float kRound = 12582912.0f;
    const float t = __fadd_rd(d, kRound);
    Axis<float> a;
    a.off = __float_as_int(t) - 0x4B400000;
    a.fr = d - (t - kRound);
    a.sw = fmaxf(1.0f - fabsf(d), 0.0f);
    return a;
}

// Q1 value at the point whose axis cells are ax, ay, relative to the node's
// value uk: sum_v lambda_v (u_v - uk).  The weights sum to one, so this is the
// interpolated value minus uk; forming it from differences keeps the rounding
// proportional to the (small) differences, and the node itself, if it is a
// vertex, contributes exactly zero.  U(dx, dy) returns u at node (i+dx, j+dy).
template <typename T, typename Acc>
__device__ __forceinline__ T bilinear_rel(const Axis<T>& ax, const Axis<T>& ay, T uk, const Acc& U) {
    const T v00 = U(ax.off, ay.off);
    const T v10 = U(ax.off + 1, ay.off);
    const T v01 = U(ax.off, ay.off + 1);
    const T v11 = U(ax.off + 1, ay.off + 1);
    const T a = fma(ax.fr, v10 - v00, v00 - uk);
    const T b = fma(ax.fr, v11 - v01, v01 - uk);
    return fma(ay.fr, b - a, a);
}

// For one control: Sd4 = sum_{k,s} (I[u](x_{i,k}^{a,s}) - u_i) and
// L4 = sum_{k,s} lambda_{i0,k}^{a,s} (four times the self weight Lambda0 of eq.
// SLimplicit; the 1/2d = 1/4 is applied by the caller).  SIG = false: sigma = 0,
// the four points coincide with the foot (Sd4, L4 are then the single point's
// terms, already "averaged").
template <typename T, bool SIG, bool CLAMP, typename Acc>
__device__ __forceinline__ void control_terms4d(const NodeBox<T>& bx, T fx, T fy, T d, T uk,
                                                const Acc& U, T& Sd, T& L) {
    if (SIG) {
        const Axis<T> xm = axis_cell<T, CLAMP>(fx - d, bx.lox, bx.hix, bx.capx);
        const Axis<T> x0 = axis_cell<T, CLAMP>(fx, bx.lox, bx.hix, bx.capx);
        const Axis<T> xp = axis_cell<T, CLAMP>(fx + d, bx.lox, bx.hix, bx.capx);
        const Axis<T> ym = axis_cell<T, CLAMP>(fy - d, bx.loy, bx.hiy, bx.capy);
        const Axis<T> y0 = axis_cell<T, CLAMP>(fy, bx.loy, bx.hiy, bx.capy);
        const Axis<T> yp = axis_cell<T, CLAMP>(fy + d, bx.loy, bx.hiy, bx.capy);
        Sd = (bilinear_rel<T>(xp, y0, uk, U) + bilinear_rel<T>(xm, y0, uk, U)) +
             (bilinear_rel<T>(x0, yp, uk, U) + bilinear_rel<T>(x0, ym, uk, U));
        L = y0.sw * (xp.sw + xm.sw) + x0.sw * (yp.sw + ym.sw);
    } else {
        const Axis<T> x0 = axis_cell<T, CLAMP>(fx, bx.lox, bx.hix, bx.capx);
        const Axis<T> y0 = axis_cell<T, CLAMP>(fy, bx.loy, bx.hiy, bx.capy);
        Sd = bilinear_rel<T>(x0, y0, uk, U);
        L = x0.sw * y0.sw;
    }
}

template <typename T, bool SIG, bool CLAMP, typename Acc>
__device__ __forceinline__ void control_terms4(const GridView& g, const NodeBox<T>& bx, T fx, T fy,
                                               T uk, const Acc& U, T& Sd, T& L) {
    control_terms4d<T, SIG, CLAMP>(bx, fx, fy, SIG ? RealOf<T>::d(g) : T(0), uk, U, Sd, L);
}

// Sd and L with the 1/2d = 1/4 applied (for callers that need the terms).
template <typename T, bool SIG, bool CLAMP = true, typename Acc>
__device__ __forceinline__ void control_terms(const GridView& g, const NodeBox<T>& bx, T fx, T fy,
                                              T uk, const Acc& U, T& Sd, T& L) {
    control_terms4<T, SIG, CLAMP>(g, bx, fx, fy, uk, U, Sd, L);
    if (SIG) {
        Sd *= T(0.25);
        L *= T(0.25);
    }
}

// Candidates of the min, written as increments over the node's value uk.
// With Sd and L as above and c0 = h l - (1 - beta) uk,
//   scheme 3 (eq. SLscheme3 with the discount):
//       (beta (S - L uk) + h l) / (1 - beta L) - uk = (beta Sd + c0) / (1 - beta L),
//   scheme 2 (eq. SLscheme2):
//       beta S + h l - uk = beta Sd + c0,
// so each candidate is a fraction N/D (D > 0) and candidates are compared by
// cross-multiplication; the new value is uk + N*/D*.  With sigma > 0 the 1/4 is
// folded into beta (beta/4 times the four-point sums; a power-of-two scaling,
// so the products are the same numbers).
template <typename T>
__device__ __forceinline__ bool better(T na, T da, int ma, T nb, T db, int mb) {
    const T l = na * db, r = nb * da;
    return (l < r) || (l == r && ma < mb);
}

template <typename T, bool SIG, bool CLAMP, typename Acc>
__device__ __forceinline__ void candidate(const GridView& g, int scheme, const NodeBox<T>& box, T s,
                                          T bq, T c0, T uk, T c, T bx, T by, const V2Of<T>& a,
                                          const Acc& U, T& N, T& D) {
    const T fx = s * fma(c, (T)a.x, bx);
    const T fy = s * fma(c, (T)a.y, by);
    T Sd, L;
    control_terms4<T, SIG, CLAMP>(g, box, fx, fy, uk, U, Sd, L);
    N = fma(bq, Sd, c0);
    D = T(1);
    if (scheme == 3) {
        D = fma(-bq, L, T(1));
        if (!(D > T(0))) {
            N = T(INFINITY);
            D = T(1);
        }
    }
}

// best_over_controls with the general terms of Section 5.3: the offset
// d = sqrt(2h) sigma(x) / dx of the node (or the constant one), the two points
// foot +- d a of the diffusion sigma(x) a along the control (weight 1/2: their
// pair sums are doubled so that the common beta/4 of the four-point form
// applies), and the running cost h l(x) + h m(a).  Same candidates, fractions
// and tie rule as the constant-coefficient form.
template <typename T, bool SIG, bool CLAMP, typename CtrlFn, typename Acc>
__device__ __forceinline__ void best_over_controls_gen(const GridView& g, int scheme, int i, int j,
                                                       T uk, T c, T bx, T by, int m0, int stride,
                                                       const CtrlFn& ctrl, const Acc& U,
                                                       T& bestN, T& bestD, int& bestM) {
    const size_t k = (size_t)j * g.n + i;
    const T s = RealOf<T>::s(g);
    const T beta = RealOf<T>::beta(g);
    const T bq = SIG ? beta * T(0.25) : beta;
    const T hl = g.costf ? RealOf<T>::h(g) * (T)g.costf[k] : RealOf<T>::hl(g);
    const T c0 = fma(-(T(1) - beta), uk, hl);
    T d = T(0);
    if (SIG) d = g.sigf ? RealOf<T>::du(g) * (T)g.sigf[k] : RealOf<T>::d(g);
    const NodeBox<T> box = node_box<T>(i, j, g.n);
    bestN = T(INFINITY);
    bestD = T(1);
    bestM = 0x7fffffff;
    for (int m = m0; m < g.na; m += stride) {
        const V2Of<T> a = ctrl(m);
        const T fx = s * fma(c, (T)a.x, bx);
        const T fy = s * fma(c, (T)a.y, by);
        T Sd, L;
        if (SIG && g.along) {
            const T ex = d * (T)a.x, ey = d * (T)a.y;
            const Axis<T> xp = axis_cell<T, CLAMP>(fx + ex, box.lox, box.hix, box.capx);
            const Axis<T> yp = axis_cell<T, CLAMP>(fy + ey, box.loy, box.hiy, box.capy);
            const Axis<T> xm = axis_cell<T, CLAMP>(fx - ex, box.lox, box.hix, box.capx);
            const Axis<T> ym = axis_cell<T, CLAMP>(fy - ey, box.loy, box.hiy, box.capy);
            Sd = T(2) * (bilinear_rel<T>(xp, yp, uk, U) + bilinear_rel<T>(xm, ym, uk, U));
            L = T(2) * (xp.sw * yp.sw + xm.sw * ym.sw);
        } else {
            control_terms4d<T, SIG, CLAMP>(box, fx, fy, d, uk, U, Sd, L);
        }
        const T cm = g.hm32 ? c0 + RealOf<T>::hm(g, m) : c0;
        T N = fma(bq, Sd, cm);
        T D = T(1);
        if (scheme == 3) {
            D = fma(-bq, L, T(1));
            if (!(D > T(0))) {
                N = T(INFINITY);
                D = T(1);
            }
        }
        if (N * bestD < bestN * D) {
            bestN = N;
            bestD = D;
            bestM = m;
        }
    }
}

// Evaluate every control handled by this thread (m = m0, m0+stride, ...) for
// node (i, j) with value uk, speed c, drift (bx, by); returns the best
// increment as a fraction N/D and its control index (ties: lowest index).
// GEN = false compiles the constant-coefficient form only (for kernels whose
// launcher sends general problems to their GEN = true instantiation).
template <typename T, bool SIG, bool CLAMP = true, bool GEN = true, typename CtrlFn, typename Acc>
__device__ __forceinline__ void best_over_controls(const GridView& g, int scheme, int i, int j,
                                                   T uk, T c, T bx, T by, int m0, int stride,
                                                   const CtrlFn& ctrl, const Acc& U,
                                                   T& bestN, T& bestD, int& bestM) {
    if (GEN && g.gen) {
        best_over_controls_gen<T, SIG, CLAMP>(g, scheme, i, j, uk, c, bx, by, m0, stride, ctrl, U,
                                              bestN, bestD, bestM);
        return;
    }
    const T s = RealOf<T>::s(g);
    const T beta = RealOf<T>::beta(g);
    const T bq = SIG ? beta * T(0.25) : beta;
    const T c0 = fma(-(T(1) - beta), uk, RealOf<T>::hl(g));
    const NodeBox<T> box = node_box<T>(i, j, g.n);
    bestN = T(INFINITY);
    bestD = T(1);
    bestM = 0x7fffffff;
    int m = m0;
    if (m < g.na) {
        // first control: taken without comparison
        candidate<T, SIG, CLAMP>(g, scheme, box, s, bq, c0, uk, c, bx, by, ctrl(m), U, bestN, bestD);
        bestM = bestN < T(INFINITY) ? m : 0x7fffffff;   // an excluded candidate is not taken
        m += stride;
    }
    for (; m < g.na; m += stride) {
        T N, D;
        candidate<T, SIG, CLAMP>(g, scheme, box, s, bq, c0, uk, c, bx, by, ctrl(m), U, N, D);
        if (N * bestD < bestN * D) {
            bestN = N;
            bestD = D;
            bestM = m;
        }
    }
}

// Argmin over the aligned group of LPN lanes (LPN = 32: the whole warp).
template <typename T, int LPN>
__device__ __forceinline__ void group_argmin(T& N, T& D, int& M) {
#pragma unroll
    for (int off = LPN / 2; off > 0; off >>= 1) {
        const T oN = __shfl_xor_sync(0xffffffffu, N, off);
        const T oD = __shfl_xor_sync(0xffffffffu, D, off);
        const int oM = __shfl_xor_sync(0xffffffffu, M, off);
        if (better<T>(oN, oD, oM, N, D, M)) {
            N = oN;
            D = oD;
            M = oM;
        }
    }
}

template <typename T>
__device__ __forceinline__ void warp_argmin(T& N, T& D, int& M) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
        const T oN = __shfl_xor_sync(0xffffffffu, N, off);
        const T oD = __shfl_xor_sync(0xffffffffu, D, off);
        const int oM = __shfl_xor_sync(0xffffffffu, M, off);
        if (better<T>(oN, oD, oM, N, D, M)) {
            N = oN;
            D = oD;
            M = oM;
        }
    }
}

// Warp min of the candidates (FP32): each lane turns its best fraction into a
// value N/D, the warp takes the min of the values with redux.sync on
// order-preserving bit patterns, then the lowest control index among the lanes
// holding that value.  Returns the min value (the increment); M gets its control.
__device__ __forceinline__ unsigned int order_key(float v) {
    const unsigned int b = __float_as_uint(v);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_val(unsigned int k) {
    return __uint_as_float((k & 0x80000000u) ? (k ^ 0x80000000u) : ~k);
}
__device__ __forceinline__ float group_min_increment(float N, float D, int& M, unsigned int mask) {
    const float v = (M == 0x7fffffff) ? INFINITY : __fdividef(N, D);
    const unsigned int key = order_key(v);
    const unsigned int kmin = __reduce_min_sync(mask, key);
    const unsigned int mc = (key == kmin) ? (unsigned int)M : 0xffffffffu;
    M = (int)__reduce_min_sync(mask, mc);
    return order_val(kmin);
}
__device__ __forceinline__ float warp_min_increment(float N, float D, int& M) {
    return group_min_increment(N, D, M, 0xffffffffu);
}

// ------------------------------------------------------------- reductions

// Non-negative floats compare like their bit patterns as unsigned integers.
__device__ __forceinline__ void atomic_max_nonneg(unsigned int* addr, float v) {
    if (v > 0.0f) atomicMax(addr, __float_as_uint(v));
}
__device__ __forceinline__ void atomic_max_nonneg(unsigned long long* addr, double v) {
    if (v > 0.0) atomicMax(addr, (unsigned long long)__double_as_longlong(v));
}

template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
    return v;
}

// Block-wide max of a non-negative value; valid in thread 0.  blockDim.x*y <= 1024.
template <typename T>
__device__ __forceinline__ T block_max(T v, T* scratch32) {
    const int tid = threadIdx.x + threadIdx.y * blockDim.x;
    const int nt = blockDim.x * blockDim.y;
    v = warp_max(v);
    __syncthreads();
    if ((tid & 31) == 0) scratch32[tid >> 5] = v;
    __syncthreads();
    T r = T(0);
    if (tid < 32) {
        r = (tid < (nt + 31) / 32) ? scratch32[tid] : T(0);
        r = warp_max(r);
    }
    return r;
}

// ------------------------------------------------------------ grid barrier

// State of the grid-wide barrier of a cooperative (co-resident) launch.  Blocks
// arrive on one of kSyncGroups group counters (each on its own 128-byte line);
// the last arriver of a group arrives on the top counter `count`.  `gen` is
// unused (kept for the layout).
constexpr int kSyncGroups = 16;
struct GridSync {
    unsigned int count;
    unsigned int gen;
    int err;          // 0, or a negative HJB_ERR_* code set by any block
    int pad[29];
    unsigned int group[kSyncGroups * 32];
};

__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned int ld_acquire_u32(const unsigned int* p) {
    unsigned int v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ int ld_relaxed_s32(const int* p) {
    int v;
    asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Two-level counting barrier.  The counters only grow: a block arriving at the
// e-th barrier of the launch (e = 0, 1, ...) finds its group counter at
// e * members + k (k earlier arrivals of its group), so the epoch e is known from
// the arrival itself; the last arriver of a group adds one to the top counter,
// and the barrier is complete once the top counter reaches (e + 1) * G.  No
// counter is reset and no generation word is written, so the last block's path
// through the barrier is two atomics and the waiters' next poll.  Every wait is
// bounded by `timeout_ns` of global time; on expiry the block records
// HJB_ERR_TIMEOUT and every block leaves at its next barrier.  Returns false
// when the grid must stop.  Requires all blocks to be co-resident
// (cudaLaunchCooperativeKernel) and the GridSync zeroed before the launch; the
// counters allow 2^32 / (blocks per group) barriers per launch.
__device__ __forceinline__ bool grid_sync(GridSync* gs, unsigned int nblocks,
                                          unsigned long long timeout_ns) {
    __syncthreads();
    if (threadIdx.x == 0 && threadIdx.y == 0) {
        const unsigned int G = nblocks < (unsigned int)kSyncGroups ? nblocks : (unsigned int)kSyncGroups;
        const unsigned int my = blockIdx.x % G;
        const unsigned int members = nblocks / G + (my < nblocks % G ? 1u : 0u);
        __threadfence();
        const unsigned int old = atomicAdd(&gs->group[my * 32], 1u);
        const unsigned int epoch = old / members;
        const unsigned int target = (epoch + 1u) * G;
        if (old == (epoch + 1u) * members - 1u) {
            __threadfence();
            atomicAdd(&gs->count, 1u);
        }
        const unsigned long long t0 = global_ns();
        while (ld_acquire_u32(&gs->count) < target) {
            if (ld_relaxed_s32(&gs->err) != 0) break;
            if (global_ns() - t0 > timeout_ns) {
                atomicCAS(&gs->err, 0, HJB_ERR_TIMEOUT);
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
    }
    __syncthreads();
    return ld_relaxed_s32(&gs->err) == 0;
}

}  // namespace hjb
