// Per-node arithmetic of the full-grid operator kernels (Cacace & Falcone,
// Section 3, eqs. SLscheme2 / SLscheme3), shared by the single-problem kernels
// (sweep.cu) and the batched ones (batch.cu).  Both read u from a tile staged
// in shared memory with a halo of R cells (row stride W).
#pragma once

#include "hjb_device.cuh"

namespace hjb {

// One application of the scheme at free node k = (i, j) whose value sits at
// base[0] in the staged tile: returns the increment N/D of the best control and
// its index.  CLAMP = false when the staged window lies inside the grid.
template <typename T, bool SIG, bool CLAMP, bool GEN = true, typename CtrlFn>
__device__ __forceinline__ T node_increment(const GridView& g, int scheme, int i, int j, size_t k,
                                            const T* base, int W, const CtrlFn& C, int& M) {
    const T uk = base[0];
    const T c = (T)g.speed[k];
    T bx = T(0), by = T(0);
    if (g.drift) {
        const float2 b = g.drift[k];
        bx = (T)b.x;
        by = (T)b.y;
    }
    auto U = [&](int dx, int dy) { return base[dy * W + dx]; };
    T N, D;
    best_over_controls<T, SIG, CLAMP, GEN>(g, scheme, i, j, uk, c, bx, by, 0, 1, C, U, N, D, M);
    return N / D;
}

// |T2 u - u| (eq. SLscheme2) at free node k = (i, j) in FP64 with exact FP32
// screening: an FP32 pass finds the smallest candidate over the controls; a
// control whose FP32 candidate exceeds it by more than `margin` cannot be the
// FP64 minimiser as long as |v32 - v64| <= margin / 2 for every control, so
// only the remaining controls are evaluated in FP64.  off = index of the node
// in the staged FP32 / FP64 tiles (row stride W).
template <bool SIG>
__device__ __forceinline__ double residual_node(const GridView& g, int i, int j, size_t k,
                                                const float* t32, const double* t64, int off,
                                                int W, const float2* c32, const double2* c64,
                                                float margin, double* vbest = nullptr,
                                                int* mbest = nullptr) {
    const int n = g.n;
    const float* b32 = t32 + off;
    const double* b64 = t64 + off;
    auto U32 = [&](int dx, int dy) { return b32[dy * W + dx]; };
    auto U64 = [&](int dx, int dy) { return b64[dy * W + dx]; };
    const float ck32 = g.speed[k];
    float bx32 = 0.0f, by32 = 0.0f;
    if (g.drift) {
        const float2 b = g.drift[k];
        bx32 = b.x;
        by32 = b.y;
    }
    const float uk32 = b32[0];
    const double uk64 = b64[0];
    if (g.gen) {
        // general terms (Section 5.3): every control in FP64, no screening
        auto C64 = [&](int m) { return c64[m]; };
        double N, D;
        int M;
        best_over_controls<double, SIG>(g, 2, i, j, uk64, (double)ck32, (double)bx32, (double)by32,
                                        0, 1, C64, U64, N, D, M);
        if (vbest) *vbest = N / D;
        if (mbest) *mbest = M;
        return fabs(N / D);
    }
    // FP32 screening pass
    const float s32 = g.s32, beta32 = g.beta32;
    const float c0_32 = fmaf(-(1.0f - beta32), uk32, g.hl32);
    const NodeBox<float> box32 = node_box<float>(i, j, n);
    float vmin = INFINITY;
    for (int m = 0; m < g.na; ++m) {
        const float2 a = c32[m];
        const float fx = s32 * fmaf(ck32, a.x, bx32);
        const float fy = s32 * fmaf(ck32, a.y, by32);
        float Sd, L;
        control_terms<float, SIG>(g, box32, fx, fy, uk32, U32, Sd, L);
        vmin = fminf(vmin, fmaf(beta32, Sd, c0_32));
    }
    const float keep = vmin + margin;
    // FP64 evaluation of the controls the screening cannot exclude
    const double s64 = g.s64, beta64 = g.beta64;
    const double c0_64 = fma(-(1.0 - beta64), uk64, g.hl64);
    const NodeBox<double> box64 = node_box<double>(i, j, n);
    const double ck64 = (double)ck32, bx64 = (double)bx32, by64 = (double)by32;
    double best = INFINITY;
    int bm = 0;
    for (int m = 0; m < g.na; ++m) {
        const float2 a = c32[m];
        const float fx = s32 * fmaf(ck32, a.x, bx32);
        const float fy = s32 * fmaf(ck32, a.y, by32);
        float Sd, L;
        control_terms<float, SIG>(g, box32, fx, fy, uk32, U32, Sd, L);
        if (fmaf(beta32, Sd, c0_32) > keep) continue;
        const double2 a64 = c64[m];
        const double fx64 = s64 * fma(ck64, a64.x, bx64);
        const double fy64 = s64 * fma(ck64, a64.y, by64);
        double Sd64, L64;
        control_terms<double, SIG>(g, box64, fx64, fy64, uk64, U64, Sd64, L64);
        const double v = fma(beta64, Sd64, c0_64);
        if (v < best) {
            best = v;
            bm = m;
        }
    }
    if (vbest) *vbest = best;
    if (mbest) *mbest = bm;
    return fabs(best);
}

}  // namespace hjb
