// Tile-pipelined causal patch solve (Cacace & Falcone, Section 4.3
// "Computation", with the ordering of Section 4.2).
//
// The grid is cut into 16x16-node tiles.  Inside a tile the free nodes are
// visited in causal-band order (bands of T(u_hat), as in the band ordering of
// the patches), one thread block per tile with the tile and a halo of u staged
// in shared memory, so consecutive bands are separated only by __syncthreads.
// Tiles are grouped into waves by their lowest band (wave q = floor(b_min / B))
// and scheduled cyclically: at step s every wave q <= s with q = s (mod D) is
// processed, then a grid-wide barrier.  Each tile is therefore visited once per
// D steps, always right after the wave upwind of it, and a new ordered pass
// enters the pipeline every D steps; about n_tiles / D tiles run per step.
// A tile is skipped when neither it nor any of its 8 neighbours changed by more
// than the tolerance at their last visit (a fast-marching-like active set).
// The solve stops when no tile visited during the last D steps changed by more
// than the tolerance.  All patches share one array (sharp interfaces), so the
// transmission condition is the identity; values written by other blocks are
// read through L2 (ld.global.cg).
#include <type_traits>

#include "hjb_kernels.h"

namespace hjb {

namespace {

constexpr int kTS = kTileSize;
constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// Block size of the warp-tile kernel: one 768-thread block per SM in FP32 (a
// cheap grid barrier; 85 registers a thread hold the pipelined node loop
// without spilling), 256 threads in FP64 (more registers per thread).
template <typename T>
struct WTBlock {
    static constexpr int threads = sizeof(T) == 4 ? 768 : 256;
    static constexpr int warps = threads / 32;
};

__device__ __forceinline__ float ld_l2(const float* p) { return __ldcg(p); }
__device__ __forceinline__ double ld_l2(const double* p) { return __ldcg(p); }
__device__ __forceinline__ void st_l2(float* p, float v) { __stcg(p, v); }
__device__ __forceinline__ void st_l2(double* p, double v) { __stcg(p, v); }
__device__ __forceinline__ float inc_to_float(float v) { return v; }
__device__ __forceinline__ float inc_to_float(double v) { return __double2float_ru(v); }

template <typename T, bool SIG>
__global__ void __launch_bounds__(kThreads)
k_tiles(TileArgs a, T* u) {
    using V2 = typename RealOf<T>::V2;
    extern __shared__ __align__(16) unsigned char smem[];
    const GridView& g = a.g;
    const int n = g.n;
    const int R = a.halo;
    const int W = kTS + 2 * R;
    V2* sctrl = reinterpret_cast<V2*>(smem);
    const size_t ctrl_bytes = ((size_t)g.na * sizeof(V2) + 15) & ~(size_t)15;
    int* soff = reinterpret_cast<int*>(smem + ctrl_bytes);                  // kLocalBands + 1
    T* su = reinterpret_cast<T*>(smem + ctrl_bytes + (((kLocalBands + 1) * sizeof(int) + 15) & ~(size_t)15));
    __shared__ float red[32];
    __shared__ int s_flag;
    __shared__ unsigned long long s_nodes;

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const unsigned int nblocks = gridDim.x;
    const unsigned int tol_bits = __float_as_uint(a.tol);
    for (int m = threadIdx.x; m < g.na; m += blockDim.x) sctrl[m] = RealOf<T>::ctrl(g, m);
    if (threadIdx.x == 0) s_nodes = 0ull;
    __syncthreads();
    auto C = [&](int m) { return sctrl[m]; };

    const int D = a.period;
    const int ring = 2 * D;
    int step = 0;
    int converged = 0;
    float last_max = 0.0f;
    bool ok = true;
    for (step = 0; step < a.max_steps; ++step) {
        if (blockIdx.x == 0 && threadIdx.x == 0) a.step_inc[(step + 1) % ring] = 0u;
        const int r = step % D;
        const int lbeg = a.res_off[r];
        const int lend = a.res_off[r + 1];
        float bmax = 0.0f;
        for (int idx = lbeg + (int)blockIdx.x; idx < lend; idx += gridDim.x) {
            const int t = a.tile_list[idx];
            if (a.tile_wave[t] > step) break;       // entries are sorted by wave
            const int tcx = t % a.ntx, tcy = t / a.ntx;
            // activity: this tile or a neighbour changed by more than tol at its last visit
            if (threadIdx.x == 0) s_flag = 0;
            __syncthreads();
            if (threadIdx.x < 9) {
                const int nx = tcx + (int)(threadIdx.x % 3) - 1;
                const int ny = tcy + (int)(threadIdx.x / 3) - 1;
                if (nx >= 0 && ny >= 0 && nx < a.ntx && ny < a.nty &&
                    __ldcg(a.tile_inc + ny * a.ntx + nx) > tol_bits)
                    s_flag = 1;
            }
            __syncthreads();
            if (!s_flag) continue;
            // stage the tile + halo
            const int gx0 = tcx * kTS - R, gy0 = tcy * kTS - R;
            for (int e = threadIdx.x; e < W * W; e += blockDim.x) {
                const int ey = e / W, ex = e - ey * W;
                const int gx = min(max(gx0 + ex, 0), n - 1);
                const int gy = min(max(gy0 + ey, 0), n - 1);
                su[e] = ld_l2(u + (size_t)gy * n + gx);
            }
            for (int e = threadIdx.x; e <= kLocalBands; e += blockDim.x)
                soff[e] = a.bin_off[(size_t)t * kLocalBands + e];
            __syncthreads();
            float tmax = 0.0f;
            unsigned long long cnt = 0;
            for (int sw = 0; sw < a.local_sweeps; ++sw) {
                for (int lb = 0; lb < kLocalBands; ++lb) {
                    const int b0 = soff[lb], b1 = soff[lb + 1];
                    if (b0 == b1) continue;
                    for (int q = b0 + warp; q < b1; q += kWarps) {
                        const int k = a.nodes[q];
                        const int i = k % n, j = k / n;
                        const int lx = i - gx0, ly = j - gy0;
                        T* base = su + ly * W + lx;
                        const T uk = base[0];
                        const T c = (T)g.speed[k];
                        T bx = T(0), by = T(0);
                        if (g.drift) {
                            const float2 bb = g.drift[k];
                            bx = (T)bb.x;
                            by = (T)bb.y;
                        }
                        auto U = [&](int dx, int dy) { return base[dy * W + dx]; };
                        T N, Dn;
                        int M;
                        best_over_controls<T, SIG>(g, a.scheme, i, j, uk, c, bx, by, lane, 32, C, U,
                                                   N, Dn, M);
                        warp_argmin<T>(N, Dn, M);
                        const T du = N / Dn;
                        __syncwarp();
                        if (lane == 0) {
                            base[0] = uk + du;
                            ++cnt;
                        }
                        tmax = fmaxf(tmax, inc_to_float(fabs(du)));
                    }
                    __syncthreads();
                }
            }
            // write back the tile's free nodes
            for (int e = threadIdx.x; e < kTS * kTS; e += blockDim.x) {
                const int i = tcx * kTS + (e % kTS), j = tcy * kTS + (e / kTS);
                if (i >= n || j >= n) continue;
                const size_t k = (size_t)j * n + i;
                if (g.mask[k] != kFree) continue;
                st_l2(u + k, su[(j - gy0) * W + (i - gx0)]);
            }
            if (lane == 0 && cnt) atomicAdd(&s_nodes, cnt);
            const float tm = block_max<float>(tmax, red);
            if (threadIdx.x == 0) {
                __stcg(a.tile_inc + t, __float_as_uint(tm));
                bmax = fmaxf(bmax, tm);
            }
            __syncthreads();
        }
        if (threadIdx.x == 0 && bmax > 0.0f) atomicMax(a.step_inc + step % ring, __float_as_uint(bmax));
        ok = grid_sync(a.sync, nblocks, a.timeout_ns);
        if (!ok) break;
        // convergence: no tile visited in the last D steps (after every wave
        // has been reached) changed by more than tol
        if (step >= a.n_waves - 1 + D) {
            if (threadIdx.x == 0) {
                float m = 0.0f;
                for (int d = 0; d < D; ++d)
                    m = fmaxf(m, __uint_as_float(__ldcg(a.step_inc + (step - d) % ring)));
                last_max = m;
                s_flag = (m <= a.tol) ? 1 : 0;
            }
            __syncthreads();
            if (s_flag) {
                converged = 1;
                ++step;
                break;
            }
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&a.res->nodes, s_nodes);
        if (blockIdx.x == 0) {
            a.res->passes = step;
            a.res->converged = converged;
            a.res->last_increment = last_max;
        }
    }
}

// ------------------------------------------- FP32 node-control geometry
// Everything of one node-control candidate that does not depend on u: the
// shared-memory index of the first vertex of each point's Q1 cell, the cell
// fractions and the reciprocal of the denominator D = 1 - beta L (scheme 3;
// -1 marks an excluded candidate, D <= 0).  Split out so the geometry of the
// next node can be formed while the current node's gathers, warp reduction and
// store are in flight.  Same arithmetic as control_terms4 and candidate(), with
// the foot's displacement sc a in cells (sc = s c, or s for a drift already in a)
// and 1/D from the approximate reciprocal: a candidate's relative error stays a
// few ulp, the minimum picks among candidates within that, and the increment
// it gives is a few ulp of itself off (it vanishes at the fixed point).
// NOL: no point's cell has the node as a vertex (the diffusion offset reaches
// past the foot by more than a cell, or scheme 2, which keeps the self weight
// in the sum): L = 0, D = 1, no reciprocal.
template <bool SIG>
struct Geo32 {
    int o[SIG ? 4 : 1];       // SIG: (xp, y0), (xm, y0), (x0, yp), (x0, ym)
    float fx[SIG ? 3 : 1];    // SIG: xp, xm, x0
    float fy[SIG ? 3 : 1];    // SIG: y0, yp, ym
    float rD;
};

__device__ __forceinline__ float rcp_approx(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}

template <bool SIG, bool CLAMP, bool NOL>
__device__ __forceinline__ Geo32<SIG> geo32(const GridView& g, int scheme, float sc, float bq, int i,
                                            int j, int kb, int W, float2 a) {
    Geo32<SIG> r;
    const NodeBox<float> box = node_box<float>(i, j, g.n);
    const float fx = sc * a.x;
    const float fy = sc * a.y;
    float L = 0.0f;
    if constexpr (SIG) {
        const float d = g.d32;
        const Axis<float> xm = axis_cell<float, CLAMP>(fx - d, box.lox, box.hix, box.capx);
        const Axis<float> x0 = axis_cell<float, CLAMP>(fx, box.lox, box.hix, box.capx);
        const Axis<float> xp = axis_cell<float, CLAMP>(fx + d, box.lox, box.hix, box.capx);
        const Axis<float> ym = axis_cell<float, CLAMP>(fy - d, box.loy, box.hiy, box.capy);
        const Axis<float> y0 = axis_cell<float, CLAMP>(fy, box.loy, box.hiy, box.capy);
        const Axis<float> yp = axis_cell<float, CLAMP>(fy + d, box.loy, box.hiy, box.capy);
        r.o[0] = kb + y0.off * W + xp.off;
        r.o[1] = kb + y0.off * W + xm.off;
        r.o[2] = kb + yp.off * W + x0.off;
        r.o[3] = kb + ym.off * W + x0.off;
        r.fx[0] = xp.fr; r.fx[1] = xm.fr; r.fx[2] = x0.fr;
        r.fy[0] = y0.fr; r.fy[1] = yp.fr; r.fy[2] = ym.fr;
        if constexpr (!NOL) L = y0.sw * (xp.sw + xm.sw) + x0.sw * (yp.sw + ym.sw);
    } else {
        const Axis<float> x0 = axis_cell<float, CLAMP>(fx, box.lox, box.hix, box.capx);
        const Axis<float> y0 = axis_cell<float, CLAMP>(fy, box.loy, box.hiy, box.capy);
        r.o[0] = kb + y0.off * W + x0.off;
        r.fx[0] = x0.fr;
        r.fy[0] = y0.fr;
        if constexpr (!NOL) L = x0.sw * y0.sw;
    }
    if constexpr (NOL) {
        r.rD = 1.0f;
    } else {
        const float D = scheme == 3 ? fmaf(-bq, L, 1.0f) : 1.0f;
        r.rD = D > 0.0f ? rcp_approx(D) : -1.0f;
    }
    return r;
}

// The geometry of a control a and of its opposite -a together (interior tiles:
// no projection).  The points of -a are the mirror images of those of a, so
// each axis cell of -a follows from one of a: floor(-y) = -floor(y) - 1 and
// frac(-y) = 1 - frac(y) when y is not an integer (-floor(y) and 0 when it is);
// the self weights, and with them D, are the same.  Same cells as geo32 on -a
// (the floors are exact); the fractions agree to an ulp.
__device__ __forceinline__ void mirror_cell(const Axis<float>& c, int& off, float& fr) {
    const bool f = c.fr > 0.0f;
    off = f ? -c.off - 1 : -c.off;
    fr = f ? 1.0f - c.fr : 0.0f;
}

template <bool SIG, bool NOL>
__device__ __forceinline__ void geo32_pair(const GridView& g, int scheme, float sc, float bq, int kb,
                                           int W, float2 a, Geo32<SIG>& ra, Geo32<SIG>& rb) {
    const float fx = sc * a.x;
    const float fy = sc * a.y;
    float L = 0.0f;
    if constexpr (SIG) {
        const float d = g.d32;
        const Axis<float> xm = axis_cell<float, false>(fx - d, 0.0f, 0.0f, 0.0f);
        const Axis<float> x0 = axis_cell<float, false>(fx, 0.0f, 0.0f, 0.0f);
        const Axis<float> xp = axis_cell<float, false>(fx + d, 0.0f, 0.0f, 0.0f);
        const Axis<float> ym = axis_cell<float, false>(fy - d, 0.0f, 0.0f, 0.0f);
        const Axis<float> y0 = axis_cell<float, false>(fy, 0.0f, 0.0f, 0.0f);
        const Axis<float> yp = axis_cell<float, false>(fy + d, 0.0f, 0.0f, 0.0f);
        ra.o[0] = kb + y0.off * W + xp.off;
        ra.o[1] = kb + y0.off * W + xm.off;
        ra.o[2] = kb + yp.off * W + x0.off;
        ra.o[3] = kb + ym.off * W + x0.off;
        ra.fx[0] = xp.fr; ra.fx[1] = xm.fr; ra.fx[2] = x0.fr;
        ra.fy[0] = y0.fr; ra.fy[1] = yp.fr; ra.fy[2] = ym.fr;
        // -a: its +d point mirrors a's -d point and so on
        int oxp, oxm, ox0, oyp, oym, oy0;
        float fxp, fxm, fx0, fyp, fym, fy0;
        mirror_cell(xm, oxp, fxp);
        mirror_cell(xp, oxm, fxm);
        mirror_cell(x0, ox0, fx0);
        mirror_cell(ym, oyp, fyp);
        mirror_cell(yp, oym, fym);
        mirror_cell(y0, oy0, fy0);
        rb.o[0] = kb + oy0 * W + oxp;
        rb.o[1] = kb + oy0 * W + oxm;
        rb.o[2] = kb + oyp * W + ox0;
        rb.o[3] = kb + oym * W + ox0;
        rb.fx[0] = fxp; rb.fx[1] = fxm; rb.fx[2] = fx0;
        rb.fy[0] = fy0; rb.fy[1] = fyp; rb.fy[2] = fym;
        if constexpr (!NOL) L = y0.sw * (xp.sw + xm.sw) + x0.sw * (yp.sw + ym.sw);
    } else {
        const Axis<float> x0 = axis_cell<float, false>(fx, 0.0f, 0.0f, 0.0f);
        const Axis<float> y0 = axis_cell<float, false>(fy, 0.0f, 0.0f, 0.0f);
        ra.o[0] = kb + y0.off * W + x0.off;
        ra.fx[0] = x0.fr;
        ra.fy[0] = y0.fr;
        int ox, oy;
        float frx, fry;
        mirror_cell(x0, ox, frx);
        mirror_cell(y0, oy, fry);
        rb.o[0] = kb + oy * W + ox;
        rb.fx[0] = frx;
        rb.fy[0] = fry;
        if constexpr (!NOL) L = x0.sw * y0.sw;
    }
    if constexpr (NOL) {
        ra.rD = 1.0f;
    } else {
        const float D = scheme == 3 ? fmaf(-bq, L, 1.0f) : 1.0f;
        ra.rD = D > 0.0f ? rcp_approx(D) : -1.0f;
    }
    rb.rD = ra.rD;
}

// Q1 value at a point minus uk from the vertex block at su[o] (row stride W).
__device__ __forceinline__ float bil32(const float* su, int o, int W, float frx, float fry, float uk) {
    const float v00 = su[o], v10 = su[o + 1], v01 = su[o + W], v11 = su[o + W + 1];
    const float a = fmaf(frx, v10 - v00, v00 - uk);
    const float b = fmaf(frx, v11 - v01, v01 - uk);
    return fmaf(fry, b - a, a);
}

// One visit of warp tile t (global index, instance from a.tile_inst): the warp
// stages the tile and a halo of R cells from u into its slice su, updates the
// tile's free nodes in increasing u_hat (the forms below), and writes them back.
// `hook` runs once, as soon as some node has changed by more than a.tol, so a
// schedule can queue the neighbours while the rest of the tile is visited.
// Returns the largest |increment|; *nn_out = the tile's free nodes.
template <typename T, bool SIG, int TW, int TH, typename Hook>
__device__ __forceinline__ float wt_visit(const TileArgs& a, int t, T* su,
                                          const typename RealOf<T>::V2* sctrl, int na, int lane,
                                          Hook& hook, int* nn_out, int4* changed = nullptr) {
    const int b = a.tile_inst ? a.tile_inst[t] : 0;
    const TileInst& I = a.insts[b];
    auto C = [&](int m) { return sctrl[m]; };
    const GridView& g = I.g;
    const int n = g.n;
    const int R = I.R;
    const int Wv = TW + 2 * R;       // staged window width
    // row pitch of the staged window: with node-per-lane visits, 8 or 24
    // (mod 32), so that 4 rows x 8 nodes fall in 32 distinct banks
    const int W = a.node_lanes ? tile_pitch(Wv) : Wv;
    const int H = TH + 2 * R;
    T* u;
    if constexpr (sizeof(T) == 4) u = I.u32; else u = I.u64;
    const int tl = t - I.tile_off;
    const int tcx = tl % I.ntx, tcy = tl / I.ntx;
    const int bi = tcx * TW, bj = tcy * TH;
    const int gx0 = bi - R, gy0 = bj - R;
    for (int e = lane; e < Wv * H; e += 32) {
        const int ey = e / Wv, ex = e - ey * Wv;
        const int gx = min(max(gx0 + ex, 0), n - 1);
        const int gy = min(max(gy0 + ey, 0), n - 1);
        su[ey * W + ex] = ld_l2(u + (size_t)gy * n + gx);
    }
    const int nn = a.wt_count[t];
    const int* tn = a.nodes + (size_t)t * kWarpTileNodes;
    const float* tsp = a.slot_speed + (size_t)t * kWarpTileNodes;
    // tile-local indices e (row-major TW x TH) of the nodes, in visiting order
    const int e0 = lane < nn ? tn[lane] : 0;
    const int e1 = lane + 32 < nn ? tn[lane + 32] : 0;
    const float c0 = lane < nn ? tsp[lane] : 0.0f;
    const float c1 = lane + 32 < nn ? tsp[lane + 32] : 0.0f;
    __syncwarp();
    float tmax = 0.0f;
    bool claimed = false;
    auto claim = [&]() {
        claimed = true;
        hook();
    };
    // tile-local box of the nodes that changed by more than tol (warp-uniform:
    // the increment and the node of the one-node forms are the same in every lane)
    int cx0 = TW, cx1 = -1, cy0 = TH, cy1 = -1;
    auto mark = [&](int e, float adu) {
        if (adu > a.tol) {
            const int ex = e % TW, ey = e / TW;
            cx0 = min(cx0, ex);
            cx1 = max(cx1, ex);
            cy0 = min(cy0, ey);
            cy1 = max(cy1, ey);
        }
    };
    // staged window inside the grid: the projection is the identity
    const bool interior = gx0 >= 0 && gy0 >= 0 && gx0 + Wv <= n && gy0 + H <= n;
    auto visit = [&](auto clamp_tag) {
      constexpr bool CL = decltype(clamp_tag)::value;
      for (int sw = 0; sw < a.local_sweeps; ++sw) {
        for (int q = 0; q < nn; ++q) {
            const int e = __shfl_sync(0xffffffffu, q < 32 ? e0 : e1, q & 31);
            const T c = (T)__shfl_sync(0xffffffffu, q < 32 ? c0 : c1, q & 31);
            const int ex = e % TW, ey = e / TW;
            const int i = bi + ex, j = bj + ey;
            T* base = su + (R + ey) * W + (R + ex);
            const T uk = base[0];
            T bx = T(0), by = T(0);
            if (g.drift) {
                const float2 bb = g.drift[j * n + i];
                bx = (T)bb.x;
                by = (T)bb.y;
            }
            auto U = [&](int dx, int dy) { return base[dy * W + dx]; };
            T N, Dn;
            int M;
            best_over_controls<T, SIG, CL>(g, a.scheme, i, j, uk, c, bx, by, lane, 32, C,
                                           U, N, Dn, M);
            T du;
            if constexpr (sizeof(T) == 4) {
                du = warp_min_increment(N, Dn, M);
            } else {
                warp_argmin<T>(N, Dn, M);
                du = N / Dn;
            }
            if (lane == 0) base[0] = uk + du;
            __syncwarp();
            tmax = fmaxf(tmax, inc_to_float(fabs(du)));
            mark(e, inc_to_float(fabs(du)));
            if (!claimed && tmax > a.tol) claim();
        }
      }
    };
    // FP32, no drift, at most one control per lane: the geometry of node
    // q + 1 is formed during node q (software pipelining)
    auto visit32 = [&](auto clamp_tag, auto nol_tag) {
      constexpr bool CL = decltype(clamp_tag)::value;
      constexpr bool NOL = decltype(nol_tag)::value;
      const float s = g.s32, beta = g.beta32, hl = g.hl32;
      const float bq = SIG ? beta * 0.25f : beta;
      const float omb = 1.0f - beta;
      const bool has = lane < na;
      const float2 ac = has ? g.ctrl32[lane] : make_float2(0.0f, 0.0f);
      auto node_geo = [&](int q, int& kb, int& e) {
          e = __shfl_sync(0xffffffffu, q < 32 ? e0 : e1, q & 31);
          const float c = __shfl_sync(0xffffffffu, q < 32 ? c0 : c1, q & 31);
          const int ex = e % TW, ey = e / TW;
          kb = (R + ey) * W + (R + ex);
          return geo32<SIG, CL, NOL>(g, a.scheme, s * c, bq, bi + ex, bj + ey, kb, W, ac);
      };
      float* sf = reinterpret_cast<float*>(su);
      for (int sw = 0; sw < a.local_sweeps; ++sw) {
        int kbn, en;
        Geo32<SIG> gn = node_geo(0, kbn, en);
        for (int q = 0; q < nn; ++q) {
            const Geo32<SIG> gc = gn;
            const int kb = kbn;
            const int ecur = en;
            gn = node_geo(min(q + 1, nn - 1), kbn, en);
            const float uk = sf[kb];
            const float cc0 = fmaf(-omb, uk, hl);
            float Sd;
            if constexpr (SIG) {
                Sd = (bil32(sf, gc.o[0], W, gc.fx[0], gc.fy[0], uk) +
                      bil32(sf, gc.o[1], W, gc.fx[1], gc.fy[0], uk)) +
                     (bil32(sf, gc.o[2], W, gc.fx[2], gc.fy[1], uk) +
                      bil32(sf, gc.o[3], W, gc.fx[2], gc.fy[2], uk));
            } else {
                Sd = bil32(sf, gc.o[0], W, gc.fx[0], gc.fy[0], uk);
            }
            const float N = fmaf(bq, Sd, cc0);
            float v;
            if constexpr (NOL)
                v = has ? N : INFINITY;
            else
                v = (has && gc.rD > 0.0f) ? N * gc.rD : INFINITY;
            const float du = order_val(__reduce_min_sync(0xffffffffu, order_key(v)));
            if (lane == 0) sf[kb] = uk + du;
            __syncwarp();
            tmax = fmaxf(tmax, fabsf(du));
            mark(ecur, fabsf(du));
            if (!claimed && tmax > a.tol) claim();
        }
      }
    };
    // FP32, constant coefficients: the tile's nodes 32 at a time, one per
    // lane, each lane evaluating every control itself (no cross-lane
    // reduction on the chain).  A group is 32 consecutive tile positions
    // (4 rows of 8), so a gather of the warp hits 32 distinct banks; the
    // nodes of a group read each other's previous values, and the group
    // holding the tile's lowest u_hat goes first.
    auto visit_ln = [&](auto clamp_tag, auto nol_tag) {
      constexpr bool CL = decltype(clamp_tag)::value;
      constexpr bool NOL = decltype(nol_tag)::value;
      constexpr int NG = (TW * TH + 31) / 32;
      const float s = g.s32, beta = g.beta32, hl = g.hl32;
      const float bq = SIG ? beta * 0.25f : beta;
      const float omb = 1.0f - beta;
      float* sf = reinterpret_cast<float*>(su);
      const float2* sc = reinterpret_cast<const float2*>(sctrl);
      // free positions of the tile, from its node slots
      unsigned long long fm = 0ull;
      if (lane < nn) fm |= 1ull << e0;
      if (lane + 32 < nn) fm |= 1ull << e1;
      const unsigned flo = __reduce_or_sync(0xffffffffu, (unsigned)fm);
      const unsigned fhi = __reduce_or_sync(0xffffffffu, (unsigned)(fm >> 32));
      const int g0 = __shfl_sync(0xffffffffu, e0, 0) >> 5;   // group of the lowest u_hat
      static_assert(NG <= 2, "tiles of at most 64 nodes");
      // this lane's node in each group: free?, speed (registers, no indexing)
      const bool fr0 = lane < TW * TH && ((flo >> lane) & 1u);
      const bool fr1 = NG > 1 && ((fhi >> lane) & 1u);
      const float cg0 = fr0 ? g.speed[(size_t)(bj + lane / TW) * n + bi + lane % TW] : 0.0f;
      const float cg1 = fr1 ? g.speed[(size_t)(bj + (32 + lane) / TW) * n + bi + (32 + lane) % TW]
                            : 0.0f;
      for (int sw = 0; sw < a.local_sweeps; ++sw) {
#pragma unroll
        for (int t2 = 0; t2 < NG; ++t2) {
            const int gi = NG == 1 ? 0 : (g0 + t2) & 1;
            const bool act = gi ? fr1 : fr0;
            const int e = gi * 32 + lane;
            const float c = gi ? cg1 : cg0;
            const int ex = e % TW, ey = e / TW;
            const int kb = (R + ey) * W + (R + ex);
            float uk = 0.0f, du = 0.0f;
            if (act) {
                uk = sf[kb];
                const float cc0 = fmaf(-omb, uk, hl);
                float bx = 0.0f, by = 0.0f;
                if (g.drift) {
                    const float2 bb = g.drift[(size_t)(bj + ey) * n + bi + ex];
                    bx = bb.x;
                    by = bb.y;
                }
                float best = INFINITY;
#pragma unroll 2
                for (int m = 0; m < na; ++m) {
                    const float2 am = sc[m];
                    // the foot's drift c a + b, formed as in the other visits
                    const float2 f = make_float2(fmaf(c, am.x, bx), fmaf(c, am.y, by));
                    const Geo32<SIG> gc = geo32<SIG, CL, NOL>(g, a.scheme, s, bq, bi + ex,
                                                              bj + ey, kb, W, f);
                    float Sd;
                    if constexpr (SIG) {
                        Sd = (bil32(sf, gc.o[0], W, gc.fx[0], gc.fy[0], uk) +
                              bil32(sf, gc.o[1], W, gc.fx[1], gc.fy[0], uk)) +
                             (bil32(sf, gc.o[2], W, gc.fx[2], gc.fy[1], uk) +
                              bil32(sf, gc.o[3], W, gc.fx[2], gc.fy[2], uk));
                    } else {
                        Sd = bil32(sf, gc.o[0], W, gc.fx[0], gc.fy[0], uk);
                    }
                    const float N = fmaf(bq, Sd, cc0);
                    if constexpr (NOL)
                        best = fminf(best, N);
                    else
                        best = fminf(best, gc.rD > 0.0f ? N * gc.rD : INFINITY);
                }
                du = best;
            }
            __syncwarp();
            if (act) sf[kb] = uk + du;
            __syncwarp();
            // |du| >= 0: its bits order like the values
            const float gm = __uint_as_float(__reduce_max_sync(0xffffffffu,
                                                               __float_as_uint(fabsf(du))));
            tmax = fmaxf(tmax, gm);
            if (gm > a.tol) {
                const bool ch = fabsf(du) > a.tol;
                cx0 = min(cx0, (int)__reduce_min_sync(0xffffffffu, ch ? (unsigned)ex : 0xffffu));
                cx1 = max(cx1, (int)__reduce_max_sync(0xffffffffu, ch ? (unsigned)ex : 0u));
                cy0 = min(cy0, (int)__reduce_min_sync(0xffffffffu, ch ? (unsigned)ey : 0xffffu));
                cy1 = max(cy1, (int)__reduce_max_sync(0xffffffffu, ch ? (unsigned)ey : 0u));
            }
            if (!claimed && tmax > a.tol) claim();
        }
      }
    };
    // FP32, no drift, 33..64 controls: two controls per lane (m = lane and
    // lane + 32), both geometries formed at the node, the lane's smaller
    // candidate into the warp minimum
    auto visit32k2 = [&](auto clamp_tag, auto nol_tag, auto sym_tag) {
      constexpr bool CL = decltype(clamp_tag)::value;
      constexpr bool NOL = decltype(nol_tag)::value;
      constexpr bool SYM = decltype(sym_tag)::value && !CL;
      const float s = g.s32, beta = g.beta32, hl = g.hl32;
      const float bq = SIG ? beta * 0.25f : beta;
      const float omb = 1.0f - beta;
      const bool has1 = lane + 32 < na;
      const float2 ac0 = g.ctrl32[lane];
      const float2 ac1 = has1 ? g.ctrl32[lane + 32] : make_float2(0.0f, 0.0f);
      float* sf = reinterpret_cast<float*>(su);
      auto cand = [&](const Geo32<SIG>& gc, float uk, float cc0) {
          float Sd;
          if constexpr (SIG) {
              Sd = (bil32(sf, gc.o[0], W, gc.fx[0], gc.fy[0], uk) +
                    bil32(sf, gc.o[1], W, gc.fx[1], gc.fy[0], uk)) +
                   (bil32(sf, gc.o[2], W, gc.fx[2], gc.fy[1], uk) +
                    bil32(sf, gc.o[3], W, gc.fx[2], gc.fy[2], uk));
          } else {
              Sd = bil32(sf, gc.o[0], W, gc.fx[0], gc.fy[0], uk);
          }
          const float N = fmaf(bq, Sd, cc0);
          if constexpr (NOL) return N;
          return gc.rD > 0.0f ? N * gc.rD : INFINITY;
      };
      for (int sw = 0; sw < a.local_sweeps; ++sw) {
        for (int q = 0; q < nn; ++q) {
            const int e = __shfl_sync(0xffffffffu, q < 32 ? e0 : e1, q & 31);
            const float c = __shfl_sync(0xffffffffu, q < 32 ? c0 : c1, q & 31);
            const int ex = e % TW, ey = e / TW;
            const int kb = (R + ey) * W + (R + ex);
            const float sc2 = s * c;
            Geo32<SIG> ga, gb;
            if constexpr (SYM) {
                geo32_pair<SIG, NOL>(g, a.scheme, sc2, bq, kb, W, ac0, ga, gb);
            } else {
                ga = geo32<SIG, CL, NOL>(g, a.scheme, sc2, bq, bi + ex, bj + ey, kb, W, ac0);
                gb = geo32<SIG, CL, NOL>(g, a.scheme, sc2, bq, bi + ex, bj + ey, kb, W, ac1);
            }
            const float uk = sf[kb];
            const float cc0 = fmaf(-omb, uk, hl);
            const float va = cand(ga, uk, cc0);
            const float vb = has1 ? cand(gb, uk, cc0) : INFINITY;
            const float du = order_val(__reduce_min_sync(0xffffffffu, order_key(fminf(va, vb))));
            if (lane == 0) sf[kb] = uk + du;
            __syncwarp();
            tmax = fmaxf(tmax, fabsf(du));
            mark(e, fabsf(du));
            if (!claimed && tmax > a.tol) claim();
        }
      }
    };
    // FP32, no drift, interior tiles: NG nodes at a time (q .. q + NG - 1 of the
    // visiting order on 32 / NG lanes each; a node reads the group's other nodes'
    // values of before the group).  With the NA controls closed under quarter
    // turns a lane takes four (m, m + NA/4, m + NA/2, m + 3NA/4 for m = lane %
    // (32 / NG): 64 controls two nodes at a time, 32 four at a time); with
    // opposite pairs only, two (m, m + NA/2).  The six axis cells of a_m give every
    // point of the four controls: -a_m takes their mirror images, the quarter
    // turns (-a.y, a.x) and (a.y, -a.x) swap the axes with one of them mirrored;
    // the self weight, and with it 1/D, is the same for all four.  Each
    // control's four points are summed in the order geo32 uses for it.
    auto visit_pairs = [&](auto nol_tag, auto quad_tag, auto group_tag) {
      constexpr bool NOL = decltype(nol_tag)::value;
      // QUAD: four controls a lane (a_m and its mirror and quarter turns), else two
      // (a_m and its mirror); NG nodes at a time on 32 / NG lanes each
      constexpr bool QUAD = decltype(quad_tag)::value;
      constexpr int NG = decltype(group_tag)::value;
      constexpr int LPN = 32 / NG;                  // lanes per node
      const float s = g.s32, beta = g.beta32, hl = g.hl32;
      const float bq = SIG ? beta * 0.25f : beta;
      const float omb = 1.0f - beta;
      const int half = lane / LPN;
      const float2 ac = g.ctrl32[lane % LPN];
      float* sf = reinterpret_cast<float*>(su);
      auto N4 = [&](int o0, float fx0, float fy0, int o1, float fx1, float fy1, int o2, float fx2, float fy2,
                    int o3, float fx3, float fy3, float uk, float cc0) {
          float Sd;
          if constexpr (SIG) {
              Sd = (bil32(sf, o0, W, fx0, fy0, uk) + bil32(sf, o1, W, fx1, fy1, uk)) +
                   (bil32(sf, o2, W, fx2, fy2, uk) + bil32(sf, o3, W, fx3, fy3, uk));
          } else {
              Sd = bil32(sf, o0, W, fx0, fy0, uk);
          }
          return fmaf(bq, Sd, cc0);
      };
      for (int sw = 0; sw < a.local_sweeps; ++sw) {
        for (int q = 0; q < nn; q += NG) {
            const int qq = q + half;
            const bool valid = qq < nn;
            const int src = qq & 31;
            const int ev0 = __shfl_sync(0xffffffffu, e0, src), ev1 = __shfl_sync(0xffffffffu, e1, src);
            const float cv0 = __shfl_sync(0xffffffffu, c0, src), cv1 = __shfl_sync(0xffffffffu, c1, src);
            const int e = valid ? (qq < 32 ? ev0 : ev1) : 0;
            const float c = valid ? (qq < 32 ? cv0 : cv1) : 0.0f;
            const int ex = e % TW, ey = e / TW;
            const int kb = (R + ey) * W + (R + ex);
            const float sc = s * c;
            const float fx = sc * ac.x, fy = sc * ac.y;
            const float uk = sf[kb];
            const float cc0 = fmaf(-omb, uk, hl);
            float v;
            if constexpr (SIG) {
                const float d = g.d32;
                const Axis<float> xm = axis_cell<float, false>(fx - d, 0.0f, 0.0f, 0.0f);
                const Axis<float> x0 = axis_cell<float, false>(fx, 0.0f, 0.0f, 0.0f);
                const Axis<float> xp = axis_cell<float, false>(fx + d, 0.0f, 0.0f, 0.0f);
                const Axis<float> ym = axis_cell<float, false>(fy - d, 0.0f, 0.0f, 0.0f);
                const Axis<float> y0 = axis_cell<float, false>(fy, 0.0f, 0.0f, 0.0f);
                const Axis<float> yp = axis_cell<float, false>(fy + d, 0.0f, 0.0f, 0.0f);
                // mirror images: M(c) is the cell of -y for the cell c of y
                int mxm, mx0, mxp, mym, my0, myp;
                float fmxm, fmx0, fmxp, fmym, fmy0, fmyp;
                mirror_cell(xm, mxm, fmxm);
                mirror_cell(x0, mx0, fmx0);
                mirror_cell(xp, mxp, fmxp);
                mirror_cell(ym, mym, fmym);
                mirror_cell(y0, my0, fmy0);
                mirror_cell(yp, myp, fmyp);
                // a: (x+d, y), (x-d, y), (x, y+d), (x, y-d)
                const float va = N4(kb + y0.off * W + xp.off, xp.fr, y0.fr, kb + y0.off * W + xm.off, xm.fr, y0.fr,
                                    kb + yp.off * W + x0.off, x0.fr, yp.fr, kb + ym.off * W + x0.off, x0.fr, ym.fr,
                                    uk, cc0);
                // -a: foot (-x, -y)
                const float vb = N4(kb + my0 * W + mxm, fmxm, fmy0, kb + my0 * W + mxp, fmxp, fmy0,
                                    kb + mym * W + mx0, fmx0, fmym, kb + myp * W + mx0, fmx0, fmyp, uk, cc0);
                v = fminf(va, vb);
                if constexpr (QUAD) {
                    // quarter turn (-a.y, a.x): foot (-y, x)
                    const float vc = N4(kb + x0.off * W + mym, fmym, x0.fr, kb + x0.off * W + myp, fmyp, x0.fr,
                                        kb + xp.off * W + my0, fmy0, xp.fr, kb + xm.off * W + my0, fmy0, xm.fr, uk,
                                        cc0);
                    // quarter turn (a.y, -a.x): foot (y, -x)
                    const float vd = N4(kb + mx0 * W + yp.off, yp.fr, fmx0, kb + mx0 * W + ym.off, ym.fr, fmx0,
                                        kb + mxm * W + y0.off, y0.fr, fmxm, kb + mxp * W + y0.off, y0.fr, fmxp, uk,
                                        cc0);
                    v = fminf(v, fminf(vc, vd));
                }
                if constexpr (!NOL) {
                    const float L = y0.sw * (xp.sw + xm.sw) + x0.sw * (yp.sw + ym.sw);
                    const float D = a.scheme == 3 ? fmaf(-bq, L, 1.0f) : 1.0f;
                    // the same positive D for the four: the minimum of N / D is
                    // the minimum of N divided by D
                    v = D > 0.0f ? v * rcp_approx(D) : INFINITY;
                }
            } else {
                const Axis<float> x0 = axis_cell<float, false>(fx, 0.0f, 0.0f, 0.0f);
                const Axis<float> y0 = axis_cell<float, false>(fy, 0.0f, 0.0f, 0.0f);
                int mx0, my0;
                float fmx0, fmy0;
                mirror_cell(x0, mx0, fmx0);
                mirror_cell(y0, my0, fmy0);
                const float va = N4(kb + y0.off * W + x0.off, x0.fr, y0.fr, 0, 0.f, 0.f, 0, 0.f, 0.f, 0, 0.f, 0.f, uk, cc0);
                const float vb = N4(kb + my0 * W + mx0, fmx0, fmy0, 0, 0.f, 0.f, 0, 0.f, 0.f, 0, 0.f, 0.f, uk, cc0);
                v = fminf(va, vb);
                if constexpr (QUAD) {
                    const float vc =
                        N4(kb + x0.off * W + my0, fmy0, x0.fr, 0, 0.f, 0.f, 0, 0.f, 0.f, 0, 0.f, 0.f, uk, cc0);
                    const float vd =
                        N4(kb + mx0 * W + y0.off, y0.fr, fmx0, 0, 0.f, 0.f, 0, 0.f, 0.f, 0, 0.f, 0.f, uk, cc0);
                    v = fminf(v, fminf(vc, vd));
                }
                if constexpr (!NOL) {
                    const float L = x0.sw * y0.sw;
                    const float D = a.scheme == 3 ? fmaf(-bq, L, 1.0f) : 1.0f;
                    v = D > 0.0f ? v * rcp_approx(D) : INFINITY;
                }
            }
            // minimum over the node's lanes (order-preserving bits)
            unsigned int key = order_key(valid ? v : INFINITY);
#pragma unroll
            for (int o = LPN / 2; o >= 1; o >>= 1) key = min(key, __shfl_xor_sync(0xffffffffu, key, o));
            const float du = order_val(key);
            __syncwarp();
            if (lane % LPN == 0 && valid) sf[kb] = uk + du;
            __syncwarp();
#pragma unroll
            for (int k = 0; k < NG; ++k) {
                const float duk = __shfl_sync(0xffffffffu, du, k * LPN);
                const int ek = __shfl_sync(0xffffffffu, e, k * LPN);
                if (q + k < nn) {
                    tmax = fmaxf(tmax, fabsf(duk));
                    mark(ek, fabsf(duk));
                }
            }
            if (!claimed && tmax > a.tol) claim();
        }
      }
    };
    bool piped = false;
    if constexpr (sizeof(T) == 4) {
        // no self weight: scheme 2 everywhere, a wide diffusion in interior tiles
        const bool nol = a.no_self == 2 || (a.no_self == 1 && interior);
        if (a.node_lanes && !g.gen) {
            piped = true;
            if (interior) {
                if (nol) visit_ln(std::false_type{}, std::true_type{});
                else visit_ln(std::false_type{}, std::false_type{});
            } else {
                if (nol) visit_ln(std::true_type{}, std::true_type{});
                else visit_ln(std::true_type{}, std::false_type{});
            }
        } else if (g.drift == nullptr && na == 32 && !g.gen && a.node_pairs == 2 && interior) {
            piped = true;
            if (nol) visit_pairs(std::true_type{}, std::false_type{}, std::integral_constant<int, 2>{});
            else visit_pairs(std::false_type{}, std::false_type{}, std::integral_constant<int, 2>{});
        } else if (g.drift == nullptr && na == 32 && !g.gen && a.node_pairs == 3 && interior) {
            piped = true;
            if (nol) visit_pairs(std::true_type{}, std::true_type{}, std::integral_constant<int, 4>{});
            else visit_pairs(std::false_type{}, std::true_type{}, std::integral_constant<int, 4>{});
        } else if (g.drift == nullptr && na <= 32 && !g.gen) {
            piped = true;
            if (interior) {
                if (nol) visit32(std::false_type{}, std::true_type{});
                else visit32(std::false_type{}, std::false_type{});
            } else {
                if (nol) visit32(std::true_type{}, std::true_type{});
                else visit32(std::true_type{}, std::false_type{});
            }
        } else if (g.drift == nullptr && na == 64 && !g.gen && a.node_pairs == 1 && interior) {
            piped = true;
            if (nol) visit_pairs(std::true_type{}, std::true_type{}, std::integral_constant<int, 2>{});
            else visit_pairs(std::false_type{}, std::true_type{}, std::integral_constant<int, 2>{});
        } else if (g.drift == nullptr && na <= 64 && !g.gen) {
            piped = true;
            if (interior) {
                if (a.ctrl_sym) {
                    if (nol) visit32k2(std::false_type{}, std::true_type{}, std::true_type{});
                    else visit32k2(std::false_type{}, std::false_type{}, std::true_type{});
                } else {
                    if (nol) visit32k2(std::false_type{}, std::true_type{}, std::false_type{});
                    else visit32k2(std::false_type{}, std::false_type{}, std::false_type{});
                }
            } else {
                if (nol) visit32k2(std::true_type{}, std::true_type{}, std::false_type{});
                else visit32k2(std::true_type{}, std::false_type{}, std::false_type{});
            }
        }
    }
    if (!piped) {
        if (interior)
            visit(std::false_type{});
        else
            visit(std::true_type{});
    }
    // write back this tile's free nodes
    if (lane < nn) st_l2(u + (size_t)(bj + e0 / TW) * n + bi + e0 % TW,
                         su[(R + e0 / TW) * W + (R + e0 % TW)]);
    if (lane + 32 < nn) st_l2(u + (size_t)(bj + e1 / TW) * n + bi + e1 % TW,
                              su[(R + e1 / TW) * W + (R + e1 % TW)]);
    *nn_out = nn;
    if (changed) *changed = make_int4(cx0, cx1, cy0, cy1);
    return tmax;
}

// ------------------------------------------------- one warp per TW x TH tile
// Each warp owns one tile per visit: it stages the tile and its halo in its own
// slice of shared memory and updates the tile's free nodes one after another in
// increasing u_hat (the Gauss-Seidel order of Section 4.2 restricted to the
// tile), its lanes spread over the controls.  Warps never wait for each other
// inside a step.
//
// Work of step s: the tiles of wave s (first visit, a contiguous range of the
// wave-sorted tile list) and the tiles queued for step s.  A tile whose visit
// changed some node by more than tol queues every tile within `act_radius`
// tiles (enough to cover the interpolation reach) for that tile's next step
// s' > s with s' = wave (mod D); a per-tile stamp (the last step it was queued
// for, initially its own wave) keeps each tile at most once in a step's queue.
// The queues form a ring of D + 2 slots: slot s is read in step s, filled during
// steps s - D .. s - 1 and cleared in step s + 1.  The solve stops once every
// wave has had its first visit and the queues of the next D steps are empty.
template <typename T, bool SIG, int TW, int TH>
__global__ void __launch_bounds__(WTBlock<T>::threads)
k_wtiles(TileArgs a) {
    constexpr int kWarpsW = WTBlock<T>::warps;
    using V2 = typename RealOf<T>::V2;
    extern __shared__ __align__(16) unsigned char smem[];
    const int na = a.insts[0].g.na;           // one control set for every instance
    V2* sctrl = reinterpret_cast<V2*>(smem);
    const size_t ctrl_bytes = ((size_t)na * sizeof(V2) + 15) & ~(size_t)15;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    T* su = reinterpret_cast<T*>(smem + ctrl_bytes) + (size_t)warp * a.max_wh;
    __shared__ float red[32];
    __shared__ int s_flag;
    __shared__ unsigned long long s_nodes;

    const unsigned int nblocks = gridDim.x;
    // consecutive tiles of a step go to different blocks (SMs) first
    const int gw = warp * gridDim.x + blockIdx.x;
    const int nw = gridDim.x * kWarpsW;
    for (int m = threadIdx.x; m < na; m += blockDim.x) sctrl[m] = RealOf<T>::ctrl(a.insts[0].g, m);
    if (threadIdx.x == 0) s_nodes = 0ull;
    __syncthreads();
    auto C = [&](int m) { return sctrl[m]; };

    const int D = a.period;
    const int QS = D + 2;
    const int ring = 2 * D;
    int step = 0;
    int converged = 0;
    float last_max = 0.0f;
    bool ok = true;
    unsigned long long cnt = 0;
    for (step = 0; step < a.max_steps; ++step) {
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            a.step_inc[(step + 1) % ring] = 0u;
            if (step >= 1) a.qcount[(step - 1) % QS] = 0;   // slot of step s - 1 = s + D + 1
        }
        const int slot = step % QS;
        int fbeg = 0, fn = 0;
        if (step < a.n_waves) {
            fbeg = a.wave_off[step];
            fn = a.wave_off[step + 1] - fbeg;
        }
        const int total = fn + min(__ldcg(a.qcount + slot), a.nt);
        const int32_t* queue = a.queue + (size_t)slot * a.nt;
        float wmax = 0.0f;
        for (int idx = gw; idx < total; idx += nw) {
            const int t = idx < fn ? a.tile_list[fbeg + idx] : __ldcg(queue + (idx - fn));
            const int b = a.tile_inst ? a.tile_inst[t] : 0;
            if (a.inst_active && !a.inst_active[b]) continue;
            const TileInst& I = a.insts[b];
            const int ar = I.act_radius;
            const int aw = 2 * ar + 1;
            const int nnb = aw * aw;
            const int tl = t - I.tile_off;
            const int tcx = tl % I.ntx, tcy = tl / I.ntx;
            // this lane's neighbour tile (lane < nnb): its wave decides the step it
            // would be queued for; -1 = none
            int nbw = -1;
            if (lane < nnb) {
                const int nx = tcx + lane % aw - ar, ny = tcy + lane / aw - ar;
                if (nx >= 0 && ny >= 0 && nx < I.ntx && ny < I.nty) {
                    const int w = a.tile_wave[I.tile_off + ny * I.ntx + nx];
                    if (w <= step) nbw = w;
                }
            }
            int old = 0x7fffffff;    // stamp before this visit claimed the neighbour
            bool claimed = false;
            auto claim = [&]() {
                // claim the neighbours as soon as the tile has changed; the queue
                // slots are taken after the visit, so the atomics overlap the
                // remaining nodes
                claimed = true;
                if (nbw >= 0) {
                    const int tgt = step + 1 + ((nbw - step - 1) % D + D) % D;
                    const int nx = tcx + lane % aw - ar, ny = tcy + lane / aw - ar;
                    old = atomicMax(a.stamp + I.tile_off + ny * I.ntx + nx, tgt);
                }
            };
            int nn = 0;
            const float tmax = wt_visit<T, SIG, TW, TH>(a, t, su, sctrl, na, lane, claim, &nn);
            if (claimed) {
                // lanes 0..31 claimed above; tiles past the 32nd neighbour (radius > 2)
                // are claimed here
                for (int q = lane; q < nnb; q += 32) {
                    const int nx = tcx + q % aw - ar, ny = tcy + q / aw - ar;
                    int w = -1;
                    if (q == lane) {
                        w = nbw;
                    } else if (nx >= 0 && ny >= 0 && nx < I.ntx && ny < I.nty) {
                        const int ww = a.tile_wave[I.tile_off + ny * I.ntx + nx];
                        if (ww <= step) w = ww;
                    }
                    if (w < 0) continue;
                    const int tt = I.tile_off + ny * I.ntx + nx;
                    const int tgt = step + 1 + ((w - step - 1) % D + D) % D;
                    const int prev = q == lane ? old : atomicMax(a.stamp + tt, tgt);
                    if (prev < tgt) {
                        const int qs = tgt % QS;
                        const int pos = atomicAdd(a.qcount + qs, 1);
                        if (pos < a.nt) {
                            __stcg(a.queue + (size_t)qs * a.nt + pos, tt);
                        } else {
                            atomicCAS(&a.sync->err, 0, HJB_ERR_CUDA);   // cannot happen
                        }
                    }
                }
            }
            if (lane == 0) cnt += (unsigned long long)nn * a.local_sweeps;
            wmax = fmaxf(wmax, tmax);
            __syncwarp();
        }
        const float bm = block_max<float>(wmax, red);
        if (threadIdx.x == 0 && bm > 0.0f) atomicMax(a.step_inc + step % ring, __float_as_uint(bm));
        ok = grid_sync(a.sync, nblocks, a.timeout_ns);
        if (!ok) break;
        if (step >= a.n_waves - 1) {
            if (threadIdx.x == 0) {
                int pending = 0;
                for (int d = 1; d <= D; ++d) pending += __ldcg(a.qcount + (step + d) % QS);
                float m = 0.0f;
                for (int d = 0; d < D && d <= step; ++d)
                    m = fmaxf(m, __uint_as_float(__ldcg(a.step_inc + (step - d) % ring)));
                last_max = m;
                s_flag = pending == 0 ? 1 : 0;
            }
            __syncthreads();
            if (s_flag) {
                converged = 1;
                ++step;
                break;
            }
        }
    }
    if (lane == 0 && cnt) atomicAdd(&s_nodes, cnt);
    __syncthreads();
    if (threadIdx.x == 0) {
        atomicAdd(&a.res->nodes, s_nodes);
        if (blockIdx.x == 0) {
            a.res->passes = step;
            a.res->converged = converged;
            a.res->last_increment = last_max;
        }
    }
}

// ---------------------------------------- asynchronous worklist (schedule 3)
// The same tile visits without a grid-wide barrier: warps take tiles from one
// FIFO ring and put tiles back as their inputs change, so no warp idles while
// there is work.  The causal order of Section 4.2 is kept for the first visits:
// a tile is released for its first visit once every neighbour within the
// interpolation reach (act_radius tiles) with a lower wave has made its first
// visit (a counter per tile, which then counts the tile's visits down from -1).
// After that, a visit that changed some node by more than tol puts back every
// released neighbour and itself; a tile is in the ring at most once (per-tile
// state: idle, queued, being visited, being visited and put back again).  A
// tile visited tile_cap times is not put back again (FP32 rounding can keep a
// few tiles changing by more than a tol below what FP32 resolves there; the
// solve then reports no convergence and leaves those nodes to the FP64 stage).
// The solve ends when no tile is queued or being visited.  Every wait is
// bounded by a.timeout_ns of global time.

__device__ __forceinline__ unsigned long long ld_acq_u64(const unsigned long long* p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_rel_u64(unsigned long long* p, unsigned long long v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ int ld_acq_s32(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
// tag of ring position pos (never 0, so 0 marks an empty entry)
__device__ __forceinline__ unsigned int aq_tag(unsigned long long pos) {
    return (unsigned int)(pos & 0x7fffffffull) | 0x80000000u;
}

__device__ __forceinline__ void aq_fail(const TileArgs& a, int code) {
    atomicCAS(&a.sync->err, 0, code);
    atomicExch(&a.actl->stop, 1);
}

// append tile t (its state already says queued)
__device__ __forceinline__ void aq_enqueue(const TileArgs& a, int t) {
    const unsigned long long pos = atomicAdd(&a.actl->tail, 1ull);
    unsigned long long* slot = a.aqueue + (pos & (unsigned long long)(a.aq_cap - 1));
    // the entry cap positions back has been taken by now (at most nt entries are
    // queued and at most one ticket per warp waits ahead of the tail)
    const unsigned long long t0 = global_ns();
    while (ld_acq_u64(slot) != 0ull) {
        if (global_ns() - t0 > a.timeout_ns) {
            aq_fail(a, HJB_ERR_TIMEOUT);
            return;
        }
        __nanosleep(32);
    }
    st_rel_u64(slot, ((unsigned long long)aq_tag(pos) << 32) | (unsigned int)t);
}

// tile t needs a visit: idle -> queued (appended), being visited -> put back
// after the visit; already queued: nothing
__device__ __forceinline__ void aq_push(const TileArgs& a, int t) {
    int s = ld_acq_s32(a.astate + t);
    for (int it = 0; it < 64; ++it) {
        if (s == 0) {
            const int o = atomicCAS(a.astate + t, 0, 1);
            if (o == 0) {
                atomicAdd(&a.actl->pending, 1);
                aq_enqueue(a, t);
                return;
            }
            s = o;
        } else if (s == 2) {
            const int o = atomicCAS(a.astate + t, 2, 3);
            if (o == 2) return;
            s = o;
        } else {
            return;
        }
    }
}

// next ticket's tile, or -1 when nothing is queued or being visited (or on stop)
__device__ __forceinline__ int aq_pop(const TileArgs& a) {
    if (ld_acq_s32(&a.actl->stop)) return -1;
    const unsigned long long pos = atomicAdd(&a.actl->head, 1ull);
    unsigned long long* slot = a.aqueue + (pos & (unsigned long long)(a.aq_cap - 1));
    const unsigned int tag = aq_tag(pos);
    const unsigned long long t0 = global_ns();
    // poll the own entry; the shared words only every 8th time, with a growing
    // pause (the waiting warps must not crowd L2 while others compute)
    for (unsigned int spin = 0;; ++spin) {
        const unsigned long long v = ld_acq_u64(slot);
        if ((unsigned int)(v >> 32) == tag) {
            st_rel_u64(slot, 0ull);
            return (int)(unsigned int)v;
        }
        if ((spin & 7u) == 7u) {
            if (ld_acq_s32(&a.actl->pending) == 0 || ld_acq_s32(&a.actl->stop)) return -1;
            if (global_ns() - t0 > a.timeout_ns) {
                aq_fail(a, HJB_ERR_TIMEOUT);
                return -1;
            }
        }
        __nanosleep(spin < 8 ? 64u : (spin < 32 ? 256u : 1024u));
    }
}

// per tile: state idle; first-visit counter = neighbours (act box) of lower wave
__global__ void k_async_deps(TileArgs a) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.nt) return;
    a.astate[t] = 0;
    const int wt = a.tile_wave[t];
    if (wt == 0x7fffffff) {        // no free node: never visited
        a.adeps[t] = -2;
        return;
    }
    const TileInst& I = a.insts[a.tile_inst ? a.tile_inst[t] : 0];
    const int ar = I.act_radius;
    const int tl = t - I.tile_off;
    const int tcx = tl % I.ntx, tcy = tl / I.ntx;
    int cnt = 0;
    for (int dy = -ar; dy <= ar; ++dy)
        for (int dx = -ar; dx <= ar; ++dx) {
            const int nx = tcx + dx, ny = tcy + dy;
            if (nx < 0 || ny < 0 || nx >= I.ntx || ny >= I.nty) continue;
            const int wn = a.tile_wave[I.tile_off + ny * I.ntx + nx];
            if (wn != 0x7fffffff && wn < wt) ++cnt;
        }
    a.adeps[t] = cnt;
}

// queue the tiles released from the start, in tile_list (wave) order per warp
__global__ void k_async_seed(TileArgs a) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const int listed = a.wave_off[a.n_waves];
    int t = -1;
    if (i < listed) {
        t = a.tile_list[i];
        if (a.adeps[t] != 0 || (a.inst_active && !a.inst_active[a.tile_inst ? a.tile_inst[t] : 0])) t = -1;
    }
    const unsigned m = __ballot_sync(0xffffffffu, t >= 0);
    if (m == 0u) return;
    unsigned long long base = 0;
    if (lane == 0) {
        base = atomicAdd(&a.actl->tail, (unsigned long long)__popc(m));
        atomicAdd(&a.actl->pending, __popc(m));
    }
    base = __shfl_sync(0xffffffffu, base, 0);
    if (t >= 0) {
        const unsigned long long pos = base + __popc(m & ((1u << lane) - 1u));
        a.astate[t] = 1;
        st_rel_u64(a.aqueue + (pos & (unsigned long long)(a.aq_cap - 1)),
                   ((unsigned long long)aq_tag(pos) << 32) | (unsigned int)t);
    }
}

template <bool SIG, int TW, int TH>
__global__ void __launch_bounds__(WTBlock<float>::threads)
k_wtiles_async(TileArgs a) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int na = a.insts[0].g.na;
    float2* sctrl = reinterpret_cast<float2*>(smem);
    const size_t ctrl_bytes = ((size_t)na * sizeof(float2) + 15) & ~(size_t)15;
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    float* su = reinterpret_cast<float*>(smem + ctrl_bytes) + (size_t)warp * a.max_wh;
    __shared__ unsigned long long s_nodes;
    for (int m = threadIdx.x; m < na; m += blockDim.x) sctrl[m] = a.insts[0].g.ctrl32[m];
    if (threadIdx.x == 0) s_nodes = 0ull;
    __syncthreads();
    unsigned long long cnt = 0;
    auto nohook = [] {};
    while (true) {
        int t = -1;
        if (lane == 0) {
            t = aq_pop(a);
            if (t >= 0) {
                if (atomicAdd(&a.actl->visits, 1ull) >= (unsigned long long)a.max_visits) {
                    atomicExch(&a.actl->stop, 1);   // the visit cap: not converged
                    t = -1;
                } else {
                    atomicExch(a.astate + t, 2);
                }
            }
        }
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t < 0) break;
        int first = 0;
        if (lane == 0) first = atomicSub(a.adeps + t, 1) == 0;
        first = __shfl_sync(0xffffffffu, first, 0);
        int nn = 0;
        int4 chg;
        const float tmax = wt_visit<float, SIG, TW, TH>(a, t, su, sctrl, na, lane, nohook, &nn, &chg);
        // the tile's new values are in L2 before any neighbour is put back
        __threadfence();
        const bool changed = tmax > a.tol;
        const TileInst& I = a.insts[a.tile_inst ? a.tile_inst[t] : 0];
        const int ar = I.act_radius;
        const int aw = 2 * ar + 1;
        const int tl = t - I.tile_off;
        const int tcx = tl % I.ntx, tcy = tl / I.ntx;
        const int wt = a.tile_wave[t];
        if (first || changed) {
            for (int q = lane; q < aw * aw; q += 32) {
                const int nx = tcx + q % aw - ar, ny = tcy + q / aw - ar;
                if (nx < 0 || ny < 0 || nx >= I.ntx || ny >= I.nty) continue;
                const int nb = I.tile_off + ny * I.ntx + nx;
                const int wn = a.tile_wave[nb];
                if (wn == 0x7fffffff) continue;
                // release: this was the last lower-wave neighbour's first visit
                if (first && nb != t && wn > wt && atomicSub(a.adeps + nb, 1) == 1) aq_push(a, nb);
                // put back the released neighbours (and this tile) after a change,
                // those whose nodes read a changed node: within the staged halo R
                // of the box of changed nodes along both axes
                if (changed) {
                    const int ox = (q % aw - ar) * TW, oy = (q / aw - ar) * TH;
                    const int gx = max(0, max(ox - chg.y, chg.x - (ox + TW - 1)));
                    const int gy = max(0, max(oy - chg.w, chg.z - (oy + TH - 1)));
                    if (gx <= I.R && gy <= I.R) {
                        const int d = ld_acq_s32(a.adeps + nb);
                        if (d <= 0) {
                            if (a.tile_cap <= 0 || d > -a.tile_cap)
                                aq_push(a, nb);
                            else
                                atomicExch(&a.actl->capped, 1);
                        }
                    }
                }
            }
        }
        __syncwarp();
        if (lane == 0) {
            const int o = atomicCAS(a.astate + t, 2, 0);
            if (o == 3) {
                atomicExch(a.astate + t, 1);
                aq_enqueue(a, t);
            } else {
                atomicSub(&a.actl->pending, 1);
            }
            cnt += (unsigned long long)nn * a.local_sweeps;
        }
        __syncwarp();
    }
    if (lane == 0 && cnt) atomicAdd(&s_nodes, cnt);
    __syncthreads();
    if (threadIdx.x == 0) atomicAdd(&a.res->nodes, s_nodes);
}

// Build of the warp tiles: one warp per tile gathers the tile's free nodes,
// sorts them by the key (u_hat, or the current value when re-sorting) with a
// 64-element bitonic sort held two per lane, writes them to slots
// t*64 .. t*64+count-1, and records the band of the smallest key (the tile's wave
// is derived from it).
template <int TW, int TH>
__global__ void k_wtile_build(const TileInst* __restrict__ insts, const int32_t* __restrict__ tile_inst,
                              int nt, bool key_u32, int band_cap, int32_t* nodes,
                              float* slot_speed, int32_t* count, int* tile_min) {
    const int lane = threadIdx.x & 31;
    const int t = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (t >= nt) return;
    const TileInst& I = insts[tile_inst ? tile_inst[t] : 0];
    const int n = I.g.n;
    const float* key_val = key_u32 ? I.u32 : I.uhat;
    const uint8_t* mask = I.g.mask;
    const float* speed = I.g.speed;
    const float lambda = I.lambda, band_w = I.band_w;
    const int tl = t - I.tile_off;
    const int tcx = tl % I.ntx, tcy = tl / I.ntx;
    // lane holds tile cells lane and lane + 32 (row-major TW x TH; slots past
    // TW*TH stay empty)
    float kv[2];
    int kn[2];
    for (int h = 0; h < 2; ++h) {
        const int e = lane + 32 * h;
        const int i = tcx * TW + e % TW, j = tcy * TH + e / TW;
        kv[h] = INFINITY;
        kn[h] = -1;
        if (e < TW * TH && i < n && j < n) {
            const int k = j * n + i;
            if (mask[k] == kFree) {
                kv[h] = key_val[k];
                kn[h] = k;
            }
        }
    }
    // bitonic sort of 64 (key, node) pairs; element e = lane + 32*h
    for (int size = 2; size <= 64; size <<= 1) {
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            for (int h = 0; h < 2; ++h) {
                const int e = lane + 32 * h;
                const int partner = e ^ stride;
                float pv;
                int pn;
                if (stride == 32) {
                    pv = kv[1 - h];
                    pn = kn[1 - h];
                } else {
                    pv = __shfl_xor_sync(0xffffffffu, kv[h], stride);
                    pn = __shfl_xor_sync(0xffffffffu, kn[h], stride);
                }
                const bool up = ((e & size) == 0);
                const bool lower = e < partner;
                // keep the smaller in the lower slot for an ascending block
                const bool mine_first = (kv[h] < pv) || (kv[h] == pv && kn[h] <= pn);
                const bool keep_mine = (lower == up) ? mine_first : !mine_first;
                if (stride == 32) {
                    // both halves of the lane exchange at once below
                } else if (!keep_mine) {
                    kv[h] = pv;
                    kn[h] = pn;
                }
            }
            if (stride == 32) {
                // element e (h=0) pairs with e+32 (h=1) in the same lane
                const bool up = ((lane & size) == 0);
                const bool first_le = (kv[0] < kv[1]) || (kv[0] == kv[1] && kn[0] <= kn[1]);
                if (up != first_le) {
                    const float tv = kv[0];
                    kv[0] = kv[1];
                    kv[1] = tv;
                    const int tn = kn[0];
                    kn[0] = kn[1];
                    kn[1] = tn;
                }
            }
        }
    }
    const unsigned m0 = __ballot_sync(0xffffffffu, kn[0] >= 0);
    const unsigned m1 = __ballot_sync(0xffffffffu, kn[1] >= 0);
    const int cnt = __popc(m0) + __popc(m1);
    // empty slots (INFINITY) sort last, so the first cnt elements are the nodes
    // store tile-local indices e = (j - 8 tcy) * 8 + (i - 8 tcx)
    auto local = [&](int k) { return ((k / n) - tcy * TH) * TW + (k % n) - tcx * TW; };
    const size_t sb = (size_t)t * kWarpTileNodes;
    if (lane < cnt) {
        nodes[sb + lane] = local(kn[0]);
        slot_speed[sb + lane] = speed[kn[0]];
    }
    if (lane + 32 < cnt) {
        nodes[sb + lane + 32] = local(kn[1]);
        slot_speed[sb + lane + 32] = speed[kn[1]];
    }
    if (lane == 0) {
        count[t] = cnt;
        int bm = 0x7f7f7f7f;
        if (cnt > 0) {
            const float v = fmaxf(kv[0], 0.0f);
            float T;
            if (lambda > 0.0f) {
                const float lu = fminf(lambda * v, 1.0f - 1e-6f);
                T = -log1pf(-lu) / lambda;
            } else {
                T = v;
            }
            bm = min((int)floorf(T / band_w), band_cap - 1);
        }
        tile_min[t] = bm;
    }
}

// shape code: 1 = warp 8x8, 2 = warp 8x4, 3 = warp 4x4
template <typename T, bool SIG>
auto wtile_kernel(int shape) -> void (*)(TileArgs) {
    switch (shape) {
        case 2: return k_wtiles<T, SIG, 8, 4>;
        case 3: return k_wtiles<T, SIG, 4, 4>;
        default: return k_wtiles<T, SIG, 8, 8>;
    }
}

template <typename T, bool SIG>
cudaError_t launch_wtiles_impl(const TileArgs& a, int blocks, cudaStream_t st) {
    const size_t smem = wtile_smem(sizeof(T) == 8, a.g.na, a.max_wh);
    auto kern = wtile_kernel<T, SIG>(a.warp_tiles);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void* args[] = {(void*)&a};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(WTBlock<T>::threads),
                                       args, smem, st);
}

template <typename T, bool SIG>
int wtile_blocks_per_sm_impl(int na, int max_wh, int shape) {
    const size_t smem = wtile_smem(sizeof(T) == 8, na, max_wh);
    auto kern = wtile_kernel<T, SIG>(shape);
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, WTBlock<T>::threads, smem);
    return nb;
}

// block tiles (16x16, one block per tile)
template <typename T, bool SIG>
cudaError_t launch_impl(const TileArgs& a, T* u, int blocks, cudaStream_t st) {
    const size_t smem = tile_smem(sizeof(T) == 8, a.g.na, a.halo, 0);
    auto kern = k_tiles<T, SIG>;
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void* args[] = {(void*)&a, (void*)&u};
    count_launches(1);
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(kThreads), args, smem, st);
}

template <typename T, bool SIG>
int blocks_per_sm_impl(int na, int halo) {
    const size_t smem = tile_smem(sizeof(T) == 8, na, halo, 0);
    auto kern = k_tiles<T, SIG>;
    if (smem > 48 * 1024)
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kern, kThreads, smem);
    return nb;
}

// ------------------------------------------------------------ schedule prep
// lowest band of each tile's free nodes
__global__ void k_tile_min(int n, int ntx, const int32_t* __restrict__ key,
                           const uint8_t* __restrict__ mask, int* tile_min) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * n || mask[k] != kFree) return;
    const int i = (int)(k % n), j = (int)(k / n);
    atomicMin(tile_min + (j / kTS) * ntx + (i / kTS), key[k]);
}

// bin of a free node: tile * kLocalBands + (band - tile's lowest band), capped
__global__ void k_tile_node_keys(int n, int ntx, const int32_t* __restrict__ key,
                                 const uint8_t* __restrict__ mask, const int* __restrict__ tile_min,
                                 int32_t* key2) {
    const size_t k = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= (size_t)n * n) return;
    if (mask[k] != kFree) {
        key2[k] = -1;
        return;
    }
    const int i = (int)(k % n), j = (int)(k / n);
    const int t = (j / kTS) * ntx + (i / kTS);
    key2[k] = t * kLocalBands + min(key[k] - tile_min[t], kLocalBands - 1);
}

// wave of each tile and its bin in the cyclic schedule: (wave mod D) * n_waves + wave
// (tile_inc starts "changed" for tiles with free nodes, "quiet" for the others)
__global__ void k_tile_waves(int nt, const int* __restrict__ tile_min, int band_group, int D,
                             int n_waves, int32_t* tile_wave, int32_t* tile_key,
                             unsigned int* tile_inc) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int bm = tile_min[t];
    if (bm >= 0x7f7f7f7f) {          // no free node (tile_min keeps its fill value)
        tile_wave[t] = 0x7fffffff;
        tile_key[t] = -1;
        tile_inc[t] = 0u;
        return;
    }
    const int q = min(bm / band_group, n_waves - 1);
    tile_wave[t] = q;
    tile_key[t] = (q % D) * n_waves + q;
    tile_inc[t] = 0x7f7fffffu;       // FLT_MAX: visit at least once
}

// checkerboard wave (tx + ty) mod 2 of each tile with free nodes; sort key
__global__ void k_checker_waves(const TileInst* __restrict__ insts,
                                const int32_t* __restrict__ tile_inst, int nt,
                                const int32_t* __restrict__ count, int32_t* wave, int32_t* key) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    if (count[t] > 0) {
        const TileInst& I = insts[tile_inst ? tile_inst[t] : 0];
        const int tl = t - I.tile_off;
        const int w = ((tl % I.ntx) + (tl / I.ntx)) & 1;
        wave[t] = w;
        key[t] = w;
    } else {
        wave[t] = 0x7fffffff;
        key[t] = -1;
    }
}

// flags[band_off[b] + lowest band of tile] = 1 for every tile with free nodes
__global__ void k_mark_bands(int nt, const int* __restrict__ tile_min,
                             const int32_t* __restrict__ tile_inst, const int32_t* __restrict__ band_off,
                             int32_t* flags) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int bm = tile_min[t];
    if (bm >= 0x7f7f7f7f) return;
    const int b = tile_inst ? tile_inst[t] : 0;
    flags[band_off[b] + bm] = 1;
}

// wave = rank of the tile's lowest band among its instance's distinct ones / B
__global__ void k_rank_waves(int nt, const int* __restrict__ tile_min,
                             const int32_t* __restrict__ tile_inst, const int32_t* __restrict__ band_off,
                             const int32_t* __restrict__ scan, int band_group, int32_t* tile_wave,
                             int32_t* tile_key, int* n_waves) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nt) return;
    const int bm = tile_min[t];
    if (bm >= 0x7f7f7f7f) {
        tile_wave[t] = 0x7fffffff;
        tile_key[t] = -1;
        return;
    }
    const int b = tile_inst ? tile_inst[t] : 0;
    const int rank = scan[band_off[b] + bm] - scan[band_off[b]];
    const int q = rank / band_group;
    tile_wave[t] = q;
    tile_key[t] = q;
    atomicMax(n_waves, q + 1);
}

__global__ void k_tile_stamps(int nt, const int32_t* __restrict__ tile_wave, int32_t* stamp) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t < nt) stamp[t] = tile_wave[t];
}

}  // namespace

void wtile_dims(int shape, int* tw, int* th) {
    *tw = shape == 3 ? 4 : 8;
    *th = shape == 1 ? 8 : 4;
}

size_t wtile_smem(bool f64, int na, int max_wh) {
    const size_t v2 = f64 ? sizeof(double2) : sizeof(float2);
    const size_t ctrl = ((size_t)na * v2 + 15) & ~(size_t)15;
    const size_t rs = f64 ? sizeof(double) : sizeof(float);
    const size_t warps = f64 ? WTBlock<double>::warps : WTBlock<float>::warps;
    return ctrl + warps * (size_t)max_wh * rs;
}

size_t tile_smem(bool f64, int na, int halo, int shape) {
    if (shape > 0) {
        int tw, th;
        wtile_dims(shape, &tw, &th);
        return wtile_smem(f64, na, (tw + 2 * halo) * (th + 2 * halo));
    }
    const size_t v2 = f64 ? sizeof(double2) : sizeof(float2);
    const size_t ctrl = ((size_t)na * v2 + 15) & ~(size_t)15;
    const size_t rs = f64 ? sizeof(double) : sizeof(float);
    const size_t off = (((size_t)kLocalBands + 1) * sizeof(int) + 15) & ~(size_t)15;
    const size_t w = (size_t)(kTileSize + 2 * halo);
    return ctrl + off + w * w * rs;
}

int tile_blocks_per_sm(bool f64, bool sig, int na, int halo, int shape) {
    if (shape > 0) {
        int tw, th;
        wtile_dims(shape, &tw, &th);
        return wtile_blocks_per_sm(f64, sig, na, (tw + 2 * halo) * (th + 2 * halo), shape);
    }
    if (f64) return sig ? blocks_per_sm_impl<double, true>(na, halo)
                        : blocks_per_sm_impl<double, false>(na, halo);
    return sig ? blocks_per_sm_impl<float, true>(na, halo) : blocks_per_sm_impl<float, false>(na, halo);
}

int wtile_blocks_per_sm(bool f64, bool sig, int na, int max_wh, int shape) {
    if (f64) return sig ? wtile_blocks_per_sm_impl<double, true>(na, max_wh, shape)
                        : wtile_blocks_per_sm_impl<double, false>(na, max_wh, shape);
    return sig ? wtile_blocks_per_sm_impl<float, true>(na, max_wh, shape)
               : wtile_blocks_per_sm_impl<float, false>(na, max_wh, shape);
}

cudaError_t launch_wtiles(const TileArgs& a, bool f64, bool sig, int blocks, cudaStream_t st) {
    if (f64) return sig ? launch_wtiles_impl<double, true>(a, blocks, st)
                        : launch_wtiles_impl<double, false>(a, blocks, st);
    return sig ? launch_wtiles_impl<float, true>(a, blocks, st)
               : launch_wtiles_impl<float, false>(a, blocks, st);
}

template <bool SIG>
auto wtile_async_kernel(int shape) -> void (*)(TileArgs) {
    switch (shape) {
        case 2: return k_wtiles_async<SIG, 8, 4>;
        case 3: return k_wtiles_async<SIG, 4, 4>;
        default: return k_wtiles_async<SIG, 8, 8>;
    }
}

cudaError_t launch_wtiles_async(const TileArgs& a, bool sig, int blocks, cudaStream_t st) {
    count_launches(3);
    k_async_deps<<<(a.nt + 255) / 256, 256, 0, st>>>(a);
    k_async_seed<<<(a.nt + 255) / 256, 256, 0, st>>>(a);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = wtile_smem(false, a.g.na, a.max_wh);
    auto kern = sig ? wtile_async_kernel<true>(a.warp_tiles) : wtile_async_kernel<false>(a.warp_tiles);
    if (smem > 48 * 1024) {
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    void* args[] = {(void*)&a};
    return cudaLaunchCooperativeKernel((const void*)kern, dim3(blocks), dim3(WTBlock<float>::threads), args,
                                       smem, st);
}

cudaError_t launch_wtile_build(int shape, const TileInst* insts, const int32_t* tile_inst, int nt,
                               bool key_u32, int band_cap, int32_t* nodes, float* slot_speed,
                               int32_t* count, int* tile_min, cudaStream_t st) {
    count_launches(1);
    const long long threads = (long long)nt * 32;
    auto kern = shape == 3 ? k_wtile_build<4, 4> : (shape == 2 ? k_wtile_build<8, 4> : k_wtile_build<8, 8>);
    kern<<<(int)((threads + 255) / 256), 256, 0, st>>>(insts, tile_inst, nt, key_u32, band_cap,
                                                        nodes, slot_speed, count, tile_min);
    return cudaGetLastError();
}

cudaError_t launch_checker_waves(const TileInst* insts, const int32_t* tile_inst, int nt,
                                 const int32_t* count, int32_t* wave, int32_t* key, cudaStream_t st) {
    count_launches(1);
    k_checker_waves<<<(nt + 255) / 256, 256, 0, st>>>(insts, tile_inst, nt, count, wave, key);
    return cudaGetLastError();
}

cudaError_t launch_dense_waves(int nt, const int* tile_min, const int32_t* tile_inst, int nb,
                               const int32_t* band_off, int S, int band_group, int32_t* flags,
                               int32_t* scan, int32_t* tile_wave, int32_t* tile_key, int* n_waves,
                               cudaStream_t st) {
    (void)nb;
    cudaError_t e = cudaMemsetAsync(flags, 0, sizeof(int32_t) * (size_t)(S + 1), st);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(n_waves, 0, sizeof(int), st);
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_mark_bands<<<(nt + 255) / 256, 256, 0, st>>>(nt, tile_min, tile_inst, band_off, flags);
    e = launch_exclusive_scan(S, flags, scan, st);   // scan[0..S]
    if (e != cudaSuccess) return e;
    count_launches(1);
    k_rank_waves<<<(nt + 255) / 256, 256, 0, st>>>(nt, tile_min, tile_inst, band_off, scan, band_group,
                                                    tile_wave, tile_key, n_waves);
    return cudaGetLastError();
}

cudaError_t launch_tile_stamps(int nt, const int32_t* tile_wave, int32_t* stamp, cudaStream_t st) {
    count_launches(1);
    k_tile_stamps<<<(nt + 255) / 256, 256, 0, st>>>(nt, tile_wave, stamp);
    return cudaGetLastError();
}

int tile_threads(bool f64, int shape) {
    if (!shape) return kThreads;
    return f64 ? WTBlock<double>::threads : WTBlock<float>::threads;
}

cudaError_t launch_tiles_f32(const TileArgs& a, float* u, bool sig, int blocks, cudaStream_t st) {
    return sig ? launch_impl<float, true>(a, u, blocks, st) : launch_impl<float, false>(a, u, blocks, st);
}

cudaError_t launch_tiles_f64(const TileArgs& a, double* u, bool sig, int blocks, cudaStream_t st) {
    return sig ? launch_impl<double, true>(a, u, blocks, st) : launch_impl<double, false>(a, u, blocks, st);
}

cudaError_t launch_tile_min(int n, int ntx, const int32_t* key, const uint8_t* mask, int* tile_min,
                            cudaStream_t st) {
    const long long N = (long long)n * n;
    count_launches(1);
    k_tile_min<<<(int)((N + 255) / 256), 256, 0, st>>>(n, ntx, key, mask, tile_min);
    return cudaGetLastError();
}

cudaError_t launch_tile_node_keys(int n, int ntx, const int32_t* key, const uint8_t* mask,
                                  const int* tile_min, int32_t* key2, cudaStream_t st) {
    const long long N = (long long)n * n;
    count_launches(1);
    k_tile_node_keys<<<(int)((N + 255) / 256), 256, 0, st>>>(n, ntx, key, mask, tile_min, key2);
    return cudaGetLastError();
}

cudaError_t launch_tile_waves(int nt, const int* tile_min, int band_group, int D, int n_waves,
                              int32_t* tile_wave, int32_t* tile_key, unsigned int* tile_inc,
                              cudaStream_t st) {
    count_launches(1);
    k_tile_waves<<<(nt + 255) / 256, 256, 0, st>>>(nt, tile_min, band_group, D, n_waves, tile_wave,
                                                    tile_key, tile_inc);
    return cudaGetLastError();
}

}  // namespace hjb
