// Host-side launch wrappers of the solver's kernels (one translation unit per
// group), called by the C ABI in api.cu.  All launches go to the given stream
// and return the cudaError_t of the launch.
#pragma once

#include <cuda_runtime.h>
#include <cmath>
#include <stdint.h>
#include <vector>

#include "hjb_device.cuh"

namespace hjb {

// Stream-ordered device memory from the library's pool (one per device; freed
// blocks stay cached for later allocations, hjb_trim_memory releases them).
cudaError_t pool_alloc(void** ptr, size_t bytes, cudaStream_t st);
void pool_free(void* ptr, cudaStream_t st);

// Number of kernels this library has launched (all threads), for reporting.
void count_launches(long long k);
long long launches();

// Error text returned by hjb_last_error (calling thread).
int set_last_error(int code, const char* msg);
void clear_last_error();

// Smallest FP32 sup-increment tolerance an FP32 iteration can meet: half an
// ulp of the largest value (with 1% to spare).  At the FP32 fixed point every
// node's increment is at most half an ulp of its value (a larger one would
// change it), so a tolerance below this could stall short of it.
inline double fp32_tol_floor(double umax) { return 1.01 * std::ldexp(umax > 1.0 ? umax : 1.0, -23); }

// A launch sequence recorded once as a CUDA graph and replayed: for stages made
// of many short kernels (the pointer-jumping rounds of the labels) the launch
// latency is paid once per replay instead of once per kernel.  body(st) issues
// the sequence on st and may depend only on values fixed for the graph's
// owner (buffers, sizes); if recording or instantiation fails, the body runs
// directly from then on.  The launch counter counts each replay's kernels.
struct GraphCache {
    cudaGraphExec_t exec = nullptr;
    long long kernels = 0;
    bool failed = false;

    template <typename F>
    cudaError_t run(cudaStream_t st, F&& body) {
        if (exec) {
            count_launches(kernels);
            return cudaGraphLaunch(exec, st);
        }
        if (!failed && st != nullptr) {
            const long long k0 = launches();
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                const cudaError_t eb = body(st);
                const cudaError_t ee = cudaStreamEndCapture(st, &g);
                const long long k = launches() - k0;
                count_launches(-k);                    // recorded, not run
                if (eb == cudaSuccess && ee == cudaSuccess && g != nullptr &&
                    cudaGraphInstantiate(&exec, g, 0) == cudaSuccess) {
                    cudaGraphDestroy(g);
                    kernels = k;
                    count_launches(kernels);
                    return cudaGraphLaunch(exec, st);
                }
                if (g) cudaGraphDestroy(g);
                exec = nullptr;
            }
            cudaGetLastError();
            failed = true;
        }
        return body(st);
    }
    void reset() {
        if (exec) cudaGraphExecDestroy(exec);
        exec = nullptr;
        kernels = 0;
        failed = false;
    }
};

constexpr int kBandCap = 1 << 20;                          // causal bands per problem
constexpr unsigned long long kTimeoutNs = 4000000000ull;   // grid-wide wait limit: 4 s
// visits of one tile in one worklist solve after which it is not put back: the
// 4097^2 workload with sigma = 0.01 needs 44 visits per tile on average and
// between 1024 and 2048 at its busiest tile; with sigma = 0 a few tiles keep
// changing by FP32 rounding (6.6e-7 > tol) and run into the cap (~10 us a visit)
constexpr int kTileVisitCap = 4096;

// ---------------------------------------------------------------- sweep.cu
// Halo (cells) a tile needs so that every Q1 vertex of every point lies inside.
int sweep_halo(double reach_cells);

// One full-grid application of the scheme: uout = T uin on free nodes (uin
// copied elsewhere); argmin (nullable) gets the minimising control; the block
// maxima of |T uin - uin| over free nodes are folded into *incmax (bit pattern
// of a non-negative float / double).  uout may be nullptr (residual only).
cudaError_t launch_sweep_f32(const GridView& g, bool sig, int scheme, int halo, const float* uin,
                             float* uout, int32_t* argmin, unsigned int* incmax, cudaStream_t st);
cudaError_t launch_sweep_f64(const GridView& g, bool sig, int scheme, int halo, const double* uin,
                             double* uout, int32_t* argmin, unsigned long long* incmax,
                             cudaStream_t st);

// FP64 residual with exact FP32 screening of the controls (see sweep.cu);
// margin must exceed twice the largest |FP32 - FP64| candidate difference.
cudaError_t launch_residual_screened(const GridView& g, bool sig, int halo, const double* u,
                                     float margin, unsigned long long* incmax, cudaStream_t st,
                                     float* rfield = nullptr, uint8_t* afield = nullptr);
// The FP64 stage by correction: one FP32 Jacobi sweep of e = beta P_a e + r (a, r
// from the residual field), and u += e on free nodes.
cudaError_t launch_correction_sweep(const GridView& g, bool sig, int halo, const uint8_t* act,
                                    const float* r, const float* ein, float* eout, unsigned int* incmax,
                                    cudaStream_t st);
cudaError_t launch_add_correction(long long N, const uint8_t* mask, const float* e, double* u, cudaStream_t st);
size_t residual_screened_smem(int na, int R);

// ------------------------------------------------------------ precompute.cu
struct CoarseResult {
    int sweeps;
    float increment;
};

cudaError_t launch_coarse_data(int n, int nc, const float* speed, const float2* drift,
                               const uint8_t* mask, float* speed_c, float2* drift_c,
                               uint8_t* mask_c, cudaStream_t st);
cudaError_t launch_interp(int nc, const float* uc, int n, const uint8_t* mask, float u_obst,
                          float* uhat, cudaStream_t st);
// Band edges of the causal ordering, host FP64: with lambda > 0,
// e[k] = (1 - exp(-(lambda (k w)))) / lambda for k = 1 .. L-1 (e[0] = 0), where
// L = min(cap, floor(log(1e6) / (lambda w)) + 2) (travel times up to log(1e6) /
// lambda, lambda u <= 1 - 1e-6); empty when lambda = 0.
void band_edges(double lambda, double w, int cap, std::vector<double>& e);
cudaError_t launch_synthesis(const GridView& g, const float* uhat, const BandMap& bm, uint8_t* a,
                             int32_t* key, int* max_key, cudaStream_t st);
// Band key from the current value (re-sorting), same mapping as the synthesis.
cudaError_t launch_keys_from_values(int N, const uint8_t* mask, const float* u, const BandMap& bm,
                                    int32_t* key, int* max_key, cudaStream_t st);
cudaError_t launch_successors(const GridView& g, const uint8_t* a, int32_t* succ, cudaStream_t st);
cudaError_t launch_labels(int N, const int32_t* succ, const uint8_t* mask, const int8_t* sector,
                          int n_patches, int32_t* jump_a, int32_t* jump_b, int8_t* label,
                          cudaStream_t st);
// `rounds` pointer-jumping passes out[k] = in[in[k]] starting from succ over N
// nodes, alternating between jump_a and jump_b; *result = the last output.
cudaError_t launch_pointer_jumps(long long N, const int32_t* succ, int rounds, int32_t* jump_a,
                                 int32_t* jump_b, const int32_t** result, cudaStream_t st);
// Counting sort of the indices k with key[k] >= 0 by key (nbins bins):
// off[0..nbins] = bin offsets, order = indices grouped by bin (order inside a bin
// is unspecified).  count is scratch of nbins entries.
cudaError_t launch_counting_sort(int N, const int32_t* key, int nbins, int32_t* count,
                                 int32_t* off, int32_t* order, cudaStream_t st);
// out[0..n] = exclusive prefix sums of in[0..n) (one block).
cudaError_t launch_exclusive_scan(int n, const int32_t* in, int32_t* out, cudaStream_t st);
// out[b] = off[b * stride] for b = 0..nb (inclusive).
cudaError_t launch_strided_gather(int nb, int stride, const int32_t* off, int32_t* out,
                                  cudaStream_t st);
cudaError_t launch_order(int N, const int32_t* key, const int8_t* label, const uint8_t* mask,
                         int n_patches, int n_bands, int32_t* bin_count, int32_t* bin_off,
                         int32_t* order, int32_t* band_off, cudaStream_t st);
// u64 = u32 on free nodes, the exact FP64 held values on the others
cudaError_t launch_promote(int N, const float* u32, const uint8_t* mask, double uob64, double* u64,
                           cudaStream_t st);
cudaError_t launch_demote(int N, const double* u64, float* u32, cudaStream_t st);
// Per-node input checks and reductions at problem creation (one record per
// block, `blocks` <= scan_inputs_blocks(N) of them).  flags: 1 speed not finite
// or < 0, 2 mask > obstacle, 4 sector outside -1..n_patches-1 on a target node, 8 drift not
// finite, 16 some obstacle.  first_bad[0..3]: smallest bad index per check
// (set to all ones by the caller).  fsum: sum of c |a|_max + |b| over free nodes.
struct InputScan {
    double fsum;
    unsigned long long nfree;
    float cmax, bmax;
    unsigned flags, pad;
};
int scan_inputs_blocks(long long N);
cudaError_t launch_scan_inputs(long long N, const float* speed, const uint8_t* mask, const int8_t* sector,
                               int n_patches, const float2* drift, float amax, InputScan* out,
                               unsigned long long* first_bad, int blocks, cudaStream_t st);
cudaError_t launch_init_values(int N, const uint8_t* mask, float free_val, float uob,
                               float* u32, double* u64, double uob64, cudaStream_t st);
cudaError_t launch_fix_nonfree(int N, const uint8_t* mask, float uob, double uob64, float* u32,
                               double* u64, cudaStream_t st);

// ---------------------------------------------------------------- waves.cu
struct WaveResult {
    int passes;          // passes completed
    int converged;       // 1 if a pass met the tolerance
    unsigned long long nodes;   // free-node updates performed
    float last_increment;       // sup-increment of the last pass
    int pad;
};

struct WaveArgs {
    GridView g;
    int scheme;
    const int32_t* order;     // free nodes grouped by band
    const int32_t* band_off;  // n_bands + 1
    int n_bands;
    int group;                // bands per wave
    int n_groups;             // ceil(n_bands / group)
    int window;               // activity window, in groups
    float tol;                // sup-increment tolerance of a pass
    int max_passes;
    unsigned int* inc_bits;   // 2 * n_groups, per-group max increment (float bits)
    GridSync* sync;
    WaveResult* res;
    unsigned long long timeout_ns;
};

// Whole-grid in-place relaxation in one cooperative launch (coarse solve).
struct RelaxArgs {
    GridView g;
    float tol;
    int max_sweeps;
    unsigned int* sweep_inc;  // ring of 3 per-sweep maxima (float bits), zeroed by the host
    unsigned int* sweep_umax; // ring of 3 per-sweep largest free values (float bits), zeroed
    float floor_amp;          // FP32 floor factor (1 / distance of the foot in cells, >= 1)
    int tw, th, ntx;          // block tiles of the grid (set by grid_relax_plan)
    int halo;                 // R: cells staged around a tile (>= the interpolation reach)
    int local_sweeps;         // in-place relaxations of a tile per global sweep
    int pre;                  // 1: the per-(node, control) geometry is kept in shared memory
    GridSync* sync;
    WaveResult* res;
    unsigned long long timeout_ns;
};
// Plans the block tiles of an n x n grid (sets tw, th, ntx, halo) so that every
// tile has a co-resident block; returns the number of blocks, 0 if impossible.
constexpr int kCoarseLocalSweeps = 4;   // local relaxations of a coarse tile per global sweep
int grid_relax_plan(int n, int na, int halo, int num_sms, bool sig, RelaxArgs* a);
cudaError_t launch_grid_relax(const RelaxArgs& a, float* u, bool sig, int blocks, cudaStream_t st);
int grid_relax_threads();

// Persistent cooperative kernel: max_passes passes of band-ordered waves over
// u (FP32 or FP64) in place.  blocks = co-resident block count.
cudaError_t launch_waves_f32(const WaveArgs& a, float* u, bool sig, int blocks, cudaStream_t st);
cudaError_t launch_waves_f64(const WaveArgs& a, double* u, bool sig, int blocks, cudaStream_t st);
int wave_blocks_per_sm(bool f64, bool sig, int na);
int wave_threads();
size_t wave_smem(bool f64, int na);

// ---------------------------------------------------------------- tiles.cu
constexpr int kTileSize = 16;     // tile edge in nodes (block tiles)
constexpr int kLocalBands = 64;   // band slots per block tile (the last one takes the rest)
constexpr int kWarpTile = 8;      // tile edge in nodes (warp tiles)
constexpr int kWarpTileNodes = kWarpTile * kWarpTile;

// Per-instance data of the warp-tile kernel; a single problem is a batch of one.
struct TileInst {
    GridView g;          // grid, speed, mask, controls (shared by a batch) and scheme constants
    float* u32;          // the instance's values (n*n)
    double* u64;
    const float* uhat;   // the coarse-grid interpolant (tile build key)
    float lambda;        // band map: band = floor(T(u) / band_w), T(u) = -log(1 - lambda u)/lambda
    float band_w;
    int R;               // halo cells staged around a tile
    int ntx, nty;        // tiles per row / column
    int tile_off;        // global index of the instance's tile 0
    int act_radius;      // tiles around a tile whose change re-queues it
    int pad;
};

// Control words of the asynchronous tile worklist (each on its own 128-byte line).
struct AsyncCtl {
    unsigned long long head;        // next ticket to take
    unsigned long long pad0[15];
    unsigned long long tail;        // next position to fill
    unsigned long long pad1[15];
    int pending;                    // tiles queued or being visited
    int stop;                       // set on the visit cap or an error
    int capped;                     // a tile reached tile_cap visits (not put back)
    int pad3;
    unsigned long long visits;      // tile visits so far
    unsigned long long pad2[14];
};

struct TileArgs {
    GridView g;
    int scheme;
    int halo;                  // cells staged around the tile
    int warp_tiles;            // tile shape: 0 block 16x16; warp tiles 1: 8x8, 2: 8x4, 3: 4x4
    int act_radius;            // tiles around a tile whose change re-activates it
    const int32_t* nodes;      // block tiles: free nodes sorted by (tile, local band);
                               // warp tiles: 64 slots per tile, sorted by u_hat
    const int32_t* bin_off;    // block tiles: n_tiles * kLocalBands + 1
    const int32_t* wt_count;   // warp tiles: free nodes per tile
    const int32_t* tile_list;  // block tiles: sorted by (wave mod period, wave); warp tiles: by wave
    const int32_t* res_off;    // block tiles: period + 1
    const int32_t* wave_off;   // warp tiles: n_waves + 1 offsets into tile_list
    const int32_t* tile_wave;  // wave of each tile
    unsigned int* tile_inc;    // block tiles: max increment of each tile's last visit (float bits)
    const float* slot_speed;   // warp tiles: speed of each node slot (64 per tile)
    int32_t* stamp;            // warp tiles: last step each tile was queued for
    int32_t* queue;            // warp tiles: (period + 2) x nt queued tiles
    int32_t* qcount;           // warp tiles: period + 2 queue lengths
    int nt;                    // number of tiles (all instances)
    const TileInst* insts;     // warp tiles: per-instance data
    const int32_t* tile_inst;  // warp tiles: instance of each tile (nullptr: all instance 0)
    const uint8_t* inst_active;// warp tiles: first visits only for instances flagged 1 (nullable)
    int max_wh;                // warp tiles: largest (TW + 2R)(TH + 2R) over the instances
    unsigned int* step_inc;    // ring of 2 * period per-step maxima (float bits)
    int ntx, nty;              // tiles per row / column
    int n_waves;
    int period;                // D
    int local_sweeps;
    int node_lanes;            // warp tiles, FP32: 1 = 32 nodes at a time (a node per lane,
                               // every control in the lane), 0 = one node at a time
                               // (a control per lane, warp minimum)
    int no_self;               // warp tiles, FP32: 2 = no candidate has a self weight (scheme 2),
                               // 1 = none in interior tiles (diffusion offset > 1 + the drift's
                               // reach in cells), 0 = compute it
    int ctrl_sym;              // 1: 64 controls with a_{m+32} = -a_m (to 1e-12): the second
                               // control of a lane takes the mirror of the first's geometry
    int node_pairs;            // two nodes at a time (16 lanes each), interior tiles: 1 with
                               // 64 controls, four per lane (m, m+16, m+32, m+48: one
                               // geometry, its mirror and quarter turns); 2 with 32 controls,
                               // two per lane (m and its mirror m+16); 3: four nodes at a
                               // time (8 lanes each), 32 controls, four per lane
    int max_steps;
    float tol;
    // asynchronous worklist (schedule 3): per-tile state 0 idle, 1 queued,
    // 2 being visited, 3 being visited and queued again; per-tile count of
    // lower-wave neighbours whose first visit is still to come (-1 once the tile's
    // own first visit has started); a ring of aq_cap tagged entries
    int32_t* astate;
    int32_t* adeps;
    unsigned long long* aqueue;
    int aq_cap;                // power of two > nt + warps in flight
    AsyncCtl* actl;
    long long max_visits;
    int tile_cap;              // visits of one tile after which it is not put back
                               // (<= 0: no cap)
    GridSync* sync;
    WaveResult* res;
    unsigned long long timeout_ns;
};

void wtile_dims(int shape, int* tw, int* th);
// Row pitch of a staged warp-tile window of width w for node-per-lane visits:
// the smallest 16 k + 8 >= w (8 or 24 mod 32: rows 0..3 of an 8-wide block of
// nodes map to distinct shared-memory banks).
__host__ __device__ inline int tile_pitch(int w) { return w <= 8 ? 8 : ((w - 8 + 15) / 16) * 16 + 8; }
size_t tile_smem(bool f64, int na, int halo, int shape);
// launch of the warp-tile kernel with the slices sized by a.max_wh
size_t wtile_smem(bool f64, int na, int max_wh);
int tile_blocks_per_sm(bool f64, bool sig, int na, int halo, int shape);
// Warp-tile build over nt tiles of the instances (tile_inst: instance of each
// tile, nullptr = all instance 0); key = u32 (re-sorting) or u_hat.
cudaError_t launch_wtile_build(int shape, const TileInst* insts, const int32_t* tile_inst, int nt,
                               bool key_u32, int band_cap, int32_t* nodes, float* slot_speed,
                               int32_t* count, int* tile_min, cudaStream_t st);
// wave[t] = (tx + ty) mod 2 (tile coordinates within its instance) for tiles with
// free nodes (INT_MAX otherwise), key the same (-1 for empty tiles): the
// warm-restart schedule
cudaError_t launch_checker_waves(const TileInst* insts, const int32_t* tile_inst, int nt,
                                 const int32_t* count, int32_t* wave, int32_t* key, cudaStream_t st);
// The warp-tile kernel (shape 1..3) over a.insts / a.tile_inst.
cudaError_t launch_wtiles(const TileArgs& a, bool f64, bool sig, int blocks, cudaStream_t st);
// The asynchronous worklist form (FP32): initialises the per-tile state and the
// queue (the released tiles in tile_list order) and runs the persistent kernel.
// a.aqueue (aq_cap entries) and a.actl must be zeroed by the caller.
cudaError_t launch_wtiles_async(const TileArgs& a, bool sig, int blocks, cudaStream_t st);
int wtile_blocks_per_sm(bool f64, bool sig, int na, int max_wh, int shape);
// Dense tile waves (warp tiles): within each instance the distinct lowest bands
// of its tiles are ranked in increasing order and wave = rank / band_group, so
// no step waits on a band no tile starts at.  band_off[b] = first slot of
// instance b in the flag array (nb instances, band_off[nb] = S slots); flags and
// scan are scratch of S + 1 ints; *n_waves (device) receives the largest wave + 1.
cudaError_t launch_dense_waves(int nt, const int* tile_min, const int32_t* tile_inst, int nb,
                               const int32_t* band_off, int S, int band_group, int32_t* flags,
                               int32_t* scan, int32_t* tile_wave, int32_t* tile_key, int* n_waves,
                               cudaStream_t st);
// stamp[t] = tile_wave[t] (a tile is never queued for a step up to its first visit)
cudaError_t launch_tile_stamps(int nt, const int32_t* tile_wave, int32_t* stamp, cudaStream_t st);
int tile_threads(bool f64, int shape);
cudaError_t launch_tiles_f32(const TileArgs& a, float* u, bool sig, int blocks, cudaStream_t st);
cudaError_t launch_tiles_f64(const TileArgs& a, double* u, bool sig, int blocks, cudaStream_t st);
cudaError_t launch_tile_min(int n, int ntx, const int32_t* key, const uint8_t* mask, int* tile_min,
                            cudaStream_t st);
cudaError_t launch_tile_node_keys(int n, int ntx, const int32_t* key, const uint8_t* mask,
                                  const int* tile_min, int32_t* key2, cudaStream_t st);
cudaError_t launch_tile_waves(int nt, const int* tile_min, int band_group, int D, int n_waves,
                              int32_t* tile_wave, int32_t* tile_key, unsigned int* tile_inc,
                              cudaStream_t st);

}  // namespace hjb
