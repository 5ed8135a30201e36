// Per-node arithmetic of the pre-computation (Cacace & Falcone, Section 4.3),
// shared by the single-problem kernels (precompute.cu) and the batched ones
// (batch.cu): coarse grid data, Q1 interpolation u_hat, the causal band key,
// the feedback synthesis (eq. discrete-synthesis) and the winner-take-all
// transport successor (eq. discrete-advection).
#pragma once

#include "hjb_device.cuh"

namespace hjb {

// Coarse node (I,J) is fine node (rI, rJ).  It is a target when some fine target
// node lies within r/2 fine cells in both axes, else an obstacle if its fine
// node is one.  Speed and drift are the fine ones there.
__device__ __forceinline__ void coarse_data_node(int kc, int n, int nc, const float* speed,
                                                 const float2* drift, const uint8_t* mask,
                                                 float* speed_c, float2* drift_c, uint8_t* mask_c) {
    const int r = (n - 1) / (nc - 1);
    const int hw = r / 2;
    const int I = kc % nc, J = kc / nc;
    const size_t kf = (size_t)(r * J) * n + (size_t)(r * I);
    speed_c[kc] = speed[kf];
    if (drift_c) drift_c[kc] = drift[kf];
    bool tgt = false;
    for (int dj = -hw; dj <= hw && !tgt; ++dj) {
        const int fj = r * J + dj;
        if (fj < 0 || fj >= n) continue;
        for (int di = -hw; di <= hw; ++di) {
            const int fi = r * I + di;
            if (fi < 0 || fi >= n) continue;
            if (mask[(size_t)fj * n + fi] == kTarget) {
                tgt = true;
                break;
            }
        }
    }
    mask_c[kc] = tgt ? kTarget : (mask[kf] == kObstacle ? kObstacle : kFree);
}

// u_hat at fine node k: Q1 interpolation of u_c (nested grids, ratio r); the
// value the fine scheme holds on non-free nodes.
__device__ __forceinline__ float interp_node(size_t k, int nc, const float* uc, int n,
                                             const uint8_t* mask, float u_obst) {
    const int mk = mask[k];
    if (mk != kFree) return (mk == kTarget) ? 0.0f : u_obst;
    const int i = (int)(k % n), j = (int)(k / n);
    const int r = (n - 1) / (nc - 1);
    const int cx = min(i / r, nc - 2), cy = min(j / r, nc - 2);
    const float fx = (float)(i - cx * r) / (float)r;
    const float fy = (float)(j - cy * r) / (float)r;
    const float* b = uc + (size_t)cy * nc + cx;
    const float a0 = fmaf(fx, b[1] - b[0], b[0]);
    const float a1 = fmaf(fx, b[nc + 1] - b[nc], b[nc]);
    return fmaf(fy, a1 - a0, a0);
}

// Causal band of a value: floor(T(u)/w), T(u) = -log(1 - lambda u)/lambda
// (lambda u clipped at 1 - 1e-6; T = u when lambda = 0), capped at band_cap - 1.
__device__ __forceinline__ int band_of(float u, float lambda, float band_w, int band_cap) {
    u = fmaxf(u, 0.0f);
    float T;
    if (lambda > 0.0f) {
        const float lu = fminf(lambda * u, 1.0f - 1e-6f);
        T = -log1pf(-lu) / lambda;
    } else {
        T = u;
    }
    return min((int)floorf(T / band_w), band_cap - 1);
}

// The causal band key of a value, exactly: with lambda > 0 the band edges are
// e_k = (1 - exp(-(lambda (k w)))) / lambda, k = 1 .. L-1 (the values whose travel
// time T(u) = -log(1 - lambda u)/lambda is k w), computed in FP64 on the host;
// the key of u is the number of edges <= u (the value widened to FP64, compared
// exactly).  With lambda = 0 the key is floor(u / w) in FP64.  Capped at cap - 1.
// The float estimate band_of starts the search, which then moves to the exact
// count (edges are increasing, so it ends).
__device__ __forceinline__ int band_key(float u, const BandMap& bm) {
    u = fmaxf(u, 0.0f);
    const double ud = (double)u;
    if (bm.n_edges == 0) {
        const double b = floor(ud / bm.w64);
        return b >= (double)(bm.cap - 1) ? bm.cap - 1 : (int)b;
    }
    int k = min(band_of(u, bm.lambda, bm.w32, bm.cap), bm.n_edges - 1);
    while (k + 1 < bm.n_edges && __ldg(bm.edges + k + 1) <= ud) ++k;
    while (k > 0 && __ldg(bm.edges + k) > ud) --k;
    return min(k, bm.cap - 1);
}

// Synthesis a*(x_i) = argmin_a beta u_hat(x_i + h f(x_i, a)) + h l (sigma = 0,
// self vertex included, ties to the lowest index) at free node k = (i, j).
template <typename CtrlFn>
__device__ __forceinline__ int synthesis_node(const GridView& g, size_t k, const float* uhat,
                                              const CtrlFn& C) {
    const int n = g.n;
    const int i = (int)(k % n), j = (int)(k / n);
    const float c = g.speed[k];
    float bx = 0.0f, by = 0.0f;
    if (g.drift) {
        const float2 b = g.drift[k];
        bx = b.x;
        by = b.y;
    }
    const float* base = uhat + k;
    auto U = [&](int dx, int dy) { return __ldg(base + (ptrdiff_t)dy * n + dx); };
    float Nn, D;
    int M;
    best_over_controls<float, false>(g, 2, i, j, 0.0f, c, bx, by, 0, 1, C, U, Nn, D, M);
    return M;
}

// Successor of free node k (winner-take-all transport step of eq.
// discrete-advection), as a node index of the same grid.  The foot uses the
// prescribed IEEE FP32 sequence
//   t = c*ax; t = t + bx; t = s*t; xi = (float)i + t    (round-to-nearest, no FMA)
// so that the result is bit-reproducible on any IEEE machine; the heaviest Q1
// vertex rounds each coordinate (0.5 rounds down); if it is the node itself the
// neighbour along the axis whose fraction is closer to 1/2 is taken (equal:
// lower linear index); a foot exactly on the node is a self-loop.
__device__ __forceinline__ int32_t successor_node(const GridView& g, size_t k, int m) {
    const int n = g.n;
    const int i = (int)(k % n), j = (int)(k / n);
    const float2 ctrl = g.ctrl32[min(m, g.na - 1)];
    const float c = g.speed[k];
    float bx = 0.0f, by = 0.0f;
    if (g.drift) {
        const float2 b = g.drift[k];
        bx = b.x;
        by = b.y;
    }
    const float s = g.s32;
    float tx = __fmul_rn(c, ctrl.x);
    tx = __fadd_rn(tx, bx);
    tx = __fmul_rn(s, tx);
    float ty = __fmul_rn(c, ctrl.y);
    ty = __fadd_rn(ty, by);
    ty = __fmul_rn(s, ty);
    const float top = (float)(n - 1);
    float xi = __fadd_rn((float)i, tx);
    float eta = __fadd_rn((float)j, ty);
    xi = fminf(fmaxf(xi, 0.0f), top);
    eta = fminf(fmaxf(eta, 0.0f), top);
    int cx = (int)floorf(xi), cy = (int)floorf(eta);
    cx = min(cx, n - 2);
    cy = min(cy, n - 2);
    const float fx = __fsub_rn(xi, (float)cx);
    const float fy = __fsub_rn(eta, (float)cy);
    const int vx = cx + (fx > 0.5f ? 1 : 0);
    const int vy = cy + (fy > 0.5f ? 1 : 0);
    if (vx == i && vy == j) {
        if (xi == (float)i && eta == (float)j) return (int32_t)k;
        const float ex = fabsf(__fsub_rn(fx, 0.5f));
        const float ey = fabsf(__fsub_rn(fy, 0.5f));
        const int ox = (vx == cx) ? cx + 1 : cx;
        const int oy = (vy == cy) ? cy + 1 : cy;
        const int32_t kx = vy * n + ox;
        const int32_t ky = oy * n + vx;
        return (ex < ey) ? kx : ((ey < ex) ? ky : min(kx, ky));
    }
    return vy * n + vx;
}

}  // namespace hjb
