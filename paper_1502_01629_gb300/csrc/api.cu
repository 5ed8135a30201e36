// C ABI of the solver (declared in include/hjb.h): problem construction and
// device memory, the patchy call sequence of Section 4.3 (coarse solve ->
// pre-computation -> band-ordered patch solve with FP64 polish), the plain
// full-grid comparator, the regime helper of Section 4.1 and the getters.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <mutex>
#include <vector>

#include "hjb.h"
#include "hjb_kernels.h"

using namespace hjb;

namespace hjb {
namespace {
std::atomic<long long> g_launches{0};
}
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }
long long launches() { return g_launches.load(std::memory_order_relaxed); }
}  // namespace hjb

namespace {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return code;
}

}  // namespace

namespace hjb {
int set_last_error(int code, const char* msg) {
    g_last_error = msg ? msg : "";
    return code;
}
void clear_last_error() { g_last_error.clear(); }
}  // namespace hjb

namespace {

#define CU(call)                                                                              \
    do {                                                                                      \
        cudaError_t e_ = (call);                                                              \
        if (e_ != cudaSuccess)                                                                \
            return fail(e_ == cudaErrorMemoryAllocation ? HJB_ERR_OOM : HJB_ERR_CUDA,         \
                        "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
    } while (0)


// Device memory of the problems comes from one stream-ordered pool per device
// that keeps freed blocks (release threshold: unlimited): creating and
// destroying a problem then costs no device-wide synchronisation and almost no
// driver time.  hjb_trim_memory hands the cached blocks back.
std::mutex g_pool_mu;
cudaMemPool_t g_pools[64] = {};

cudaError_t problem_pool(cudaMemPool_t* out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lk(g_pool_mu);
    if (!g_pools[dev]) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        e = cudaMemPoolCreate(&g_pools[dev], &props);
        if (e != cudaSuccess) {
            g_pools[dev] = nullptr;
            return e;
        }
        uint64_t keep = UINT64_MAX;
        cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep);
    }
    *out = g_pools[dev];
    return cudaSuccess;
}

}  // namespace

namespace hjb {
cudaError_t pool_alloc(void** ptr, size_t bytes, cudaStream_t st) {
    cudaMemPool_t pool;
    cudaError_t e = problem_pool(&pool);
    if (e != cudaSuccess) return e;
    return cudaMallocFromPoolAsync(ptr, bytes, pool, st);
}
void pool_free(void* ptr, cudaStream_t st) {
    if (ptr) cudaFreeAsync(ptr, st);
}
}  // namespace hjb

namespace {

template <typename T>
cudaError_t palloc(T** ptr, size_t bytes, cudaStream_t st) {
    return hjb::pool_alloc(reinterpret_cast<void**>(ptr), bytes, st);
}

template <typename T>
void pfree(T*& ptr, cudaStream_t st) {
    hjb::pool_free((void*)ptr, st);
    ptr = nullptr;
}

// Pinned host words for the small results the host reads back: one slab of
// slots shared by the problems (cudaMallocHost / cudaFreeHost per problem cost
// a page pinning each); past the slab, a plain pinned allocation.
constexpr int kPinnedSlots = 128;
constexpr size_t kPinnedSlot = 4096;
std::mutex g_pin_mu;
unsigned char* g_pin_slab = nullptr;
bool g_pin_used[kPinnedSlots] = {};

cudaError_t pinned_alloc(void** out, size_t bytes) {
    if (bytes <= kPinnedSlot) {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        if (!g_pin_slab) {
            void* slab = nullptr;
            if (cudaMallocHost(&slab, kPinnedSlots * kPinnedSlot) == cudaSuccess)
                g_pin_slab = static_cast<unsigned char*>(slab);
        }
        if (g_pin_slab) {
            for (int i = 0; i < kPinnedSlots; ++i) {
                if (!g_pin_used[i]) {
                    g_pin_used[i] = true;
                    *out = g_pin_slab + (size_t)i * kPinnedSlot;
                    return cudaSuccess;
                }
            }
        }
    }
    return cudaMallocHost(out, bytes);
}

void pinned_free(void* ptr) {
    if (!ptr) return;
    {
        std::lock_guard<std::mutex> lk(g_pin_mu);
        unsigned char* q = static_cast<unsigned char*>(ptr);
        if (g_pin_slab && q >= g_pin_slab && q < g_pin_slab + kPinnedSlots * kPinnedSlot) {
            g_pin_used[(q - g_pin_slab) / kPinnedSlot] = false;
            return;
        }
    }
    cudaFreeHost(ptr);
}

// Device allocation released at scope exit (test-path temporaries only).
struct DevBuf {
    void* ptr = nullptr;
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&ptr, bytes); }
    ~DevBuf() {
        if (ptr) cudaFree(ptr);
    }
};

// Stage timer on the problem's stream.
struct Timer {
    cudaEvent_t ev[10];
    int n = 0;
    cudaStream_t st;
    explicit Timer(cudaStream_t s) : st(s) {
        for (auto& e : ev) cudaEventCreate(&e);
    }
    ~Timer() {
        for (auto& e : ev) cudaEventDestroy(e);
    }
    void mark() {
        if (n < 10) cudaEventRecord(ev[n++], st);
    }
    // elapsed ms between marks a and b (after a stream sync)
    double ms(int a, int b) {
        float t = 0.0f;
        if (a < n && b < n && cudaEventSynchronize(ev[b]) == cudaSuccess)
            cudaEventElapsedTime(&t, ev[a], ev[b]);
        return (double)t;
    }
};

void clear_stats(hjb_stats* s) {
    if (!s) return;
    std::memset(s, 0, sizeof(*s));
    s->residual = -1.0;
}

}  // namespace

struct hjb_problem {
    hjb_desc desc{};
    int n = 0, N = 0, na = 0, nc = 0, r = 0, np = 1;
    double dx = 0, h = 0, beta = 0, hl = 0, uob = 0, sigma = 0, lambda = 0;
    double reach = 0;     // max |h f| / dx + d, cells
    int halo = 1;
    int halo_c = 1;       // coarse grid: reach without the diffusion (Section 4: the coarse solve is first order), same h/dx
    RelaxArgs relax_plan{};   // coarse relaxation tiles (tw, th, ntx, halo)
    int relax_blocks = 0;
    GraphCache labels_graph;  // successors + label rounds (fixed buffers)
    InputScan* scan_tmp = nullptr;   // creation-time input scan records
    cudaStream_t st = nullptr;
    bool own_stream = false;
    int device = 0, num_sms = 0;
    bool has_drift = false;
    // general terms (Section 5.3)
    bool gen = false, along = false;
    bool ctrl_sym = false;         // 64 controls, a_{m+32} = -a_m
    bool ctrl_rot = false;         // and a_{m+16}, a_{m+48} the quarter turns of a_m
    bool ctrl_sym32 = false;       // 32 controls, a_{m+16} = -a_m
    bool ctrl_rot32 = false;       // and a_{m+8}, a_{m+24} the quarter turns of a_m
    bool visit_auto = false;       // desc.visit was 0 (automatic)
    float* sigf = nullptr;         // sigma(x), n*n
    float* costf = nullptr;        // l(x), n*n
    float* costf_c = nullptr;      // l(x) at the coarse nodes
    float* hm32 = nullptr;         // h m(a_m)
    double* hm64 = nullptr;
    float* hmc32 = nullptr;        // h_c m(a_m) for the coarse grid
    double* hmc64 = nullptr;
    double lmax = 0;               // max l(x) + max m(a)
    double amp32 = 1.0;            // FP32 noise amplification 1/D of SLscheme3 (>= 1)
    double uc_max = 0;             // largest coarse value (set by hjb_coarse_solve)

    // FP32 tolerance floor: half an ulp of the largest value (an FP32 iteration cannot settle finer), times the
    // amplification 1/(1 - beta Lambda0) of eq. SLscheme3, which divides the
    // rounding of the numerator by the foot's distance from the node in cells
    double floor32(double U) const { return fp32_tol_floor(U) * amp32; }

    // fine data
    float* speed = nullptr;
    float2* drift = nullptr;
    uint8_t* mask = nullptr;
    int8_t* sector = nullptr;
    float2* ctrl32 = nullptr;
    double2* ctrl64 = nullptr;
    // values
    float* u32 = nullptr;
    float* u32b = nullptr;
    double* u64 = nullptr;
    double* u64b = nullptr;
    bool value_f64 = false;
    // coarse grid
    float* speed_c = nullptr;
    float2* drift_c = nullptr;
    uint8_t* mask_c = nullptr;
    float* uc = nullptr;
    double hc = 0, beta_c = 0, hl_c = 0, uob_c = 0;
    // pre-computation
    float* uhat = nullptr;
    uint8_t* a = nullptr;
    int32_t* succ = nullptr;
    int32_t* jump_a = nullptr;
    int32_t* jump_b = nullptr;
    int8_t* label = nullptr;
    int32_t* key = nullptr;
    int32_t* order = nullptr;
    int32_t* bin_count = nullptr;
    int32_t* bin_off = nullptr;
    int32_t* band_off = nullptr;
    double* band_e = nullptr;     // band edges (FP64), band_L entries
    int band_L = 0;
    unsigned int* inc_bits = nullptr;
    int n_bands = 0, n_free = 0, bins_cap = 0, bands_cap = 0;
    // tile schedule
    int ntx = 0, nty = 0, nt = 0, n_waves = 0, sched_cap = 0;
    int shape = 0;        // 0 block tiles 16x16; warp tiles 1: 8x8, 2: 8x4, 3: 4x4
    int act_radius = 1;
    int32_t* tile_min = nullptr;
    int32_t* tile_wave = nullptr;
    int32_t* tile_key = nullptr;
    int32_t* tile_list = nullptr;
    unsigned int* tile_inc = nullptr;
    int32_t* tile_key2 = nullptr;
    int32_t* tile_nodes = nullptr;
    int32_t* tile_bin_count = nullptr;
    int32_t* tile_bin_off = nullptr;
    int32_t* wt_nodes = nullptr;
    int32_t* wt_count = nullptr;
    float* wt_speed = nullptr;     // speed per node slot (warp tiles)
    int32_t* wt_stamp = nullptr;   // per-tile queue stamps (warp tiles)
    bool async = false;            // schedule 3: the asynchronous worklist for the FP32 phase
    float* corr_r = nullptr;       // FP64 stage by correction: residual field (FP32) ...
    uint8_t* corr_a = nullptr;     // ... and its minimising control per node
    int32_t* a_state = nullptr;    // worklist: per-tile state and first-visit counters
    int32_t* a_deps = nullptr;
    unsigned long long* a_queue = nullptr;
    int a_cap = 0;
    int32_t* wt_queue = nullptr;   // (tile_period + 2) x nt queued tiles
    int32_t* wt_qcount = nullptr;  // tile_period + 2 queue lengths
    int32_t* cb_wave = nullptr;    // warm restart: checkerboard wave (0/1) of each tile
    int32_t* cb_key = nullptr;
    int32_t* cb_list = nullptr;    // tiles sorted by checkerboard wave
    int32_t* cb_off = nullptr;     // 3 offsets
    int32_t* cb_count = nullptr;   // 2 counters (sort scratch)
    TileInst* tinst = nullptr;     // warp tiles: the problem as a one-instance batch (device)
    int32_t* rank_flags = nullptr; // dense-wave scratch (n_bands + 1)
    int32_t* rank_scan = nullptr;
    int32_t* rank_boff = nullptr;  // {0, n_bands}
    int rank_cap = 0;
    int max_wh = 0;                // (TW + 2R)(TH + 2R)
    int32_t* sched_count = nullptr;
    int32_t* sched_off = nullptr;
    int32_t* res_off = nullptr;
    unsigned int* step_inc = nullptr;
    int tile_blocks32 = 0, tile_blocks64 = 0;
    long long n_free_total = 0;   // free nodes of G
    bool coarse_done = false, built = false;
    // scratch
    void* scratch = nullptr;      // small device scalars
    void* host_pinned = nullptr;  // small pinned host scalars
    unsigned int* inc_hist32 = nullptr;
    unsigned long long* inc_hist64 = nullptr;
    int hist_cap = 0;
    int wave_blocks32 = 0, wave_blocks64 = 0;

    // A bound on the values the solve meets: the obstacle value l/lambda + h l
    // with a discount; without one, four times the largest coarse value once the
    // coarse solve has run (the value is a minimum time of the same order),
    // else the placeholder obstacle value.
    double value_bound() const {
        if (lambda > 0.0 || !coarse_done) return uob;
        return std::max(1.0, 4.0 * uc_max);
    }

    void set_general(GridView& g, double hh, double dxx, bool coarse) const {
        g.gen = (sigf && !coarse) || costf || hm32 ? 1 : 0;
        g.along = along && !coarse ? 1 : 0;
        g.sigf = coarse ? nullptr : sigf;
        g.costf = coarse ? costf_c : costf;
        g.hm32 = coarse ? hmc32 : hm32;
        g.hm64 = coarse ? hmc64 : hm64;
        const double du = coarse ? 0.0 : std::sqrt(2.0 * hh) / dxx;
        g.du32 = (float)du;
        g.du64 = du;
        g.h32 = (float)hh;
        g.h64 = hh;
    }

    BandMap band_map() const {
        BandMap b{};
        b.lambda = (float)lambda;
        b.w64 = desc.band_width * h;
        b.w32 = (float)b.w64;
        b.edges = band_e;
        b.n_edges = band_L;
        b.cap = kBandCap;
        return b;
    }

    GridView fine_view() const {
        GridView g{};
        g.n = n;
        g.na = na;
        g.speed = speed;
        g.drift = has_drift ? drift : nullptr;
        g.mask = mask;
        g.ctrl32 = ctrl32;
        g.ctrl64 = ctrl64;
        const double s = h / dx;
        const double d = std::sqrt(2.0 * h) * sigma / dx;
        g.s32 = (float)s;
        g.s64 = s;
        g.d32 = (float)d;
        g.d64 = d;
        g.beta32 = (float)beta;
        g.beta64 = beta;
        g.hl32 = (float)hl;
        g.hl64 = hl;
        g.uob32 = (float)uob;
        g.uob64 = uob;
        set_general(g, h, dx, false);
        return g;
    }
    GridView coarse_view() const {
        GridView g{};
        g.n = nc;
        g.na = na;
        g.speed = speed_c;
        g.drift = has_drift ? drift_c : nullptr;
        g.mask = mask_c;
        g.ctrl32 = ctrl32;
        g.ctrl64 = ctrl64;
        const double dxc = 2.0 / (nc - 1);
        const double s = hc / dxc;
        g.s32 = (float)s;
        g.s64 = s;
        g.d32 = 0.0f;
        g.d64 = 0.0;
        g.beta32 = (float)beta_c;
        g.beta64 = beta_c;
        g.hl32 = (float)hl_c;
        g.hl64 = hl_c;
        g.uob32 = (float)uob;     // obstacles hold the fine scheme's value on both grids
        g.uob64 = uob;
        set_general(g, hc, dxc, true);
        return g;
    }
};

namespace {

struct Scalars {
    unsigned int relax_inc[3];
    unsigned int relax_umax[3];
    unsigned int inc32;
    int max_key;
    int n_waves;
    unsigned long long inc64;
    CoarseResult coarse;
    WaveResult wave;
    GridSync sync;
    AsyncCtl actl;
};

static_assert(sizeof(Scalars) <= kPinnedSlot, "a problem's pinned scalars must fit one pinned slot");

Scalars* dscal(hjb_problem* p) { return reinterpret_cast<Scalars*>(p->scratch); }
Scalars* hscal(hjb_problem* p) { return reinterpret_cast<Scalars*>(p->host_pinned); }

int validate_desc(const hjb_desc* d) {
    if (!d) return fail(HJB_ERR_INVALID_ARG, "desc is NULL");
    if (d->n < 3 || d->n > 16385) return fail(HJB_ERR_INVALID_ARG, "n=%d out of range [3,16385]", d->n);
    if (d->n_controls < 1 || d->n_controls > HJB_MAX_CONTROLS)
        return fail(HJB_ERR_INVALID_ARG, "n_controls=%d out of range", d->n_controls);
    if (!(d->lambda >= 0.0) || !std::isfinite(d->lambda)) return fail(HJB_ERR_INVALID_ARG, "bad lambda");
    if (!(d->sigma >= 0.0) || !std::isfinite(d->sigma)) return fail(HJB_ERR_INVALID_ARG, "bad sigma");
    if (!(d->cost > 0.0) || !std::isfinite(d->cost)) return fail(HJB_ERR_INVALID_ARG, "cost must be > 0");
    if (!std::isfinite(d->h)) return fail(HJB_ERR_INVALID_ARG, "bad h");
    if (d->scheme != 2 && d->scheme != 3 && d->scheme != 0)
        return fail(HJB_ERR_INVALID_ARG, "scheme must be 2 or 3");
    if (d->n_patches < 1 || d->n_patches > HJB_MAX_PATCHES)
        return fail(HJB_ERR_INVALID_ARG, "n_patches=%d out of range", d->n_patches);
    if (d->coarse_n != 0) {
        if (d->coarse_n < 3 || d->coarse_n > d->n || (d->n - 1) % (d->coarse_n - 1) != 0)
            return fail(HJB_ERR_INVALID_ARG, "coarse_n=%d does not nest in n=%d", d->coarse_n, d->n);
    }
    if (!std::isfinite(d->band_width)) return fail(HJB_ERR_INVALID_ARG, "bad band_width");
    if (d->resort_passes < 0) return fail(HJB_ERR_INVALID_ARG, "resort_passes must be >= 0");
    if (d->schedule < 0 || d->schedule > 4) return fail(HJB_ERR_INVALID_ARG, "schedule must be 0 .. 4");
    if (d->tile_shape < -1 || d->tile_shape > 2)
        return fail(HJB_ERR_INVALID_ARG, "tile_shape must be -1 (auto), 0 (8x8), 1 (8x4) or 2 (4x4)");
    if (d->visit < 0 || d->visit > 4)
        return fail(HJB_ERR_INVALID_ARG,
                    "visit must be 0 (auto), 1 (a node at a time), 2 (32 nodes at a time), 3 (two nodes at a "
                    "time) or 4 (four nodes at a time)");
    return HJB_OK;
}

int create_common(const hjb_desc* desc, const float* speed, const uint8_t* mask,
                  const int8_t* sector, const double* controls, const float* drift,
                  void* cuda_stream, hjb_problem** out, bool device_inputs,
                  const hjb_terms* terms = nullptr) {
    g_last_error.clear();
    if (!out) return fail(HJB_ERR_INVALID_ARG, "out is NULL");
    *out = nullptr;
    int rc = validate_desc(desc);
    if (rc) return rc;
    if (!speed || !mask || !controls) return fail(HJB_ERR_INVALID_ARG, "speed, mask and controls are required");
    const int n = desc->n;
    const size_t N = (size_t)n * n;
    const int na = desc->n_controls;

    double amax = 0.0;
    for (int m = 0; m < na; ++m) {
        if (!std::isfinite(controls[2 * m]) || !std::isfinite(controls[2 * m + 1]))
            return fail(HJB_ERR_INVALID_ARG, "control %d is not finite", m);
        amax = std::fmax(amax, std::hypot(controls[2 * m], controls[2 * m + 1]));
    }

    // general terms (host arrays; the mask is read on the host only for them)
    double sig_max = desc->sigma, lx_max = desc->cost, ma_max = 0.0;
    if (terms) {
        if (device_inputs) return fail(HJB_ERR_INVALID_ARG, "general terms take host inputs");
        if (terms->reserved != 0) return fail(HJB_ERR_INVALID_ARG, "terms->reserved must be 0");
        if (terms->diffusion != HJB_DIFFUSION_ISOTROPIC && terms->diffusion != HJB_DIFFUSION_CONTROL)
            return fail(HJB_ERR_INVALID_ARG, "terms->diffusion=%d unknown", terms->diffusion);
        if (terms->sigma_field) {
            sig_max = 0.0;
            for (size_t k = 0; k < N; ++k) {
                const float v = terms->sigma_field[k];
                if (!std::isfinite(v) || v < 0.0f) return fail(HJB_ERR_INVALID_ARG, "sigma_field[%zu] invalid", k);
                if (mask[k] == HJB_MASK_FREE) sig_max = std::fmax(sig_max, (double)v);
            }
        }
        if (terms->cost_field) {
            lx_max = 0.0;
            for (size_t k = 0; k < N; ++k) {
                const float v = terms->cost_field[k];
                if (!std::isfinite(v) || !(v > 0.0f)) return fail(HJB_ERR_INVALID_ARG, "cost_field[%zu] invalid", k);
                lx_max = std::fmax(lx_max, (double)v);
            }
        }
        if (terms->control_cost) {
            for (int m = 0; m < na; ++m) {
                const double v = terms->control_cost[m];
                if (!std::isfinite(v) || v < 0.0) return fail(HJB_ERR_INVALID_ARG, "control_cost[%d] invalid", m);
                ma_max = std::fmax(ma_max, v);
            }
        }
    }
    const bool along = terms && terms->diffusion == HJB_DIFFUSION_CONTROL;

    hjb_problem* p = new hjb_problem();
    auto bail = [&](int code) {
        hjb_destroy(p);
        return code;
    };
#define CUP(call)                                                                         \
    do {                                                                                  \
        cudaError_t e_ = (call);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return bail(fail(e_ == cudaErrorMemoryAllocation ? HJB_ERR_OOM : HJB_ERR_CUDA, \
                             "%s failed: %s", #call, cudaGetErrorString(e_)));           \
    } while (0)

    CUP(cudaGetDevice(&p->device));
    CUP(cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device));
    if (cuda_stream) {
        p->st = (cudaStream_t)cuda_stream;
    } else {
        CUP(cudaStreamCreateWithFlags(&p->st, cudaStreamNonBlocking));
        p->own_stream = true;
    }
    // upload the per-node inputs, then check and reduce them on the device: the
    // host never walks the arrays (on a coherent host, pages the GPU has read
    // can sit in device memory, where a host pass over them is slow)
    const cudaMemcpyKind kind = device_inputs ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    CUP(palloc(&p->speed, N * sizeof(float), p->st));
    CUP(palloc(&p->mask, N, p->st));
    CUP(palloc(&p->sector, N, p->st));
    CUP(cudaMemcpyAsync(p->speed, speed, N * sizeof(float), kind, p->st));
    CUP(cudaMemcpyAsync(p->mask, mask, N, kind, p->st));
    if (sector) {
        CUP(cudaMemcpyAsync(p->sector, sector, N, kind, p->st));
    } else {
        CUP(cudaMemsetAsync(p->sector, 0xff, N, p->st));
    }
    if (drift) {
        CUP(palloc(&p->drift, N * sizeof(float2), p->st));
        CUP(cudaMemcpyAsync(p->drift, drift, N * sizeof(float2), kind, p->st));
    }
    double cmax = 0.0, bmax = 0.0;
    double fsum = 0.0;             // sum of c |a|_max + |b| over free nodes (for the FP32 floor)
    long long n_free_total = 0;
    bool any_obstacle = false;
    {
        const int nb = scan_inputs_blocks((long long)N);
        CUP(palloc(&p->scan_tmp, nb * sizeof(InputScan) + 4 * sizeof(unsigned long long), p->st));
        InputScan* d_scan = p->scan_tmp;
        unsigned long long* d_bad = reinterpret_cast<unsigned long long*>(d_scan + nb);
        CUP(cudaMemsetAsync(d_bad, 0xff, 4 * sizeof(unsigned long long), p->st));
        CUP(launch_scan_inputs((long long)N, p->speed, p->mask, sector ? p->sector : nullptr, desc->n_patches,
                               p->drift, (float)amax, d_scan, d_bad, nb, p->st));
        std::vector<InputScan> hs(nb);
        unsigned long long hb[4];
        CUP(cudaMemcpyAsync(hs.data(), d_scan, nb * sizeof(InputScan), cudaMemcpyDeviceToHost, p->st));
        CUP(cudaMemcpyAsync(hb, d_bad, sizeof(hb), cudaMemcpyDeviceToHost, p->st));
        CUP(cudaStreamSynchronize(p->st));
        pfree(p->scan_tmp, p->st);
        unsigned flags = 0;
        for (const InputScan& r : hs) {
            fsum += r.fsum;
            n_free_total += (long long)r.nfree;
            cmax = std::fmax(cmax, (double)r.cmax);
            bmax = std::fmax(bmax, (double)r.bmax);
            flags |= r.flags;
        }
        if (flags & 1u) return bail(fail(HJB_ERR_INVALID_ARG, "speed[%llu] invalid", hb[0]));
        if (flags & 2u) return bail(fail(HJB_ERR_INVALID_ARG, "mask[%llu] invalid", hb[1]));
        if (flags & 4u) return bail(fail(HJB_ERR_INVALID_ARG, "sector[%llu] out of range", hb[2]));
        if (flags & 8u) return bail(fail(HJB_ERR_INVALID_ARG, "drift[%llu] not finite", hb[3]));
        any_obstacle = (flags & 16u) != 0;
    }
    if (any_obstacle && desc->lambda <= 0.0)
        return bail(fail(HJB_ERR_INVALID_ARG, "obstacles need lambda > 0 (their value is l/lambda + h l)"));

    p->desc = *desc;
    // warp tiles: the FP32 phase steps through waves between grid-wide barriers
    // (schedule 4) or runs from the asynchronous worklist (schedule 3); schedule 0
    // takes the worklist above 3073 nodes per side, where the steps hold enough
    // tiles that barrier waits and idle warps outweigh its extra visits (measured
    // on the 64-control obstacle workload: 4097^2 241 vs 302 ms, 2049^2 66 vs 55 ms)
    if (p->desc.schedule == 3 || p->desc.schedule == 4 || p->desc.schedule == 0) {
        p->async = p->desc.schedule == 3 || (p->desc.schedule == 0 && desc->n > 3073);
        p->desc.schedule = 0;
    }
    if (p->desc.scheme == 0) p->desc.scheme = 3;
    if (p->desc.band_width <= 0.0) p->desc.band_width = 1.0;
    if (p->desc.band_window <= 0) p->desc.band_window = 8;
    if (p->desc.band_group <= 0) p->desc.band_group = 1;
    // warp tiles revisit queued tiles every step (period 1; 1025^2: sigma 0.1
    // 50.5 -> 31.4 ms, sigma 0.02 9.9 -> 8.8 ms, sigma 0 6.7 -> 6.5 ms against period 2)
    if (p->desc.tile_period <= 0) p->desc.tile_period = p->desc.schedule == 0 ? 1 : 2;
    p->n = n;
    p->N = (int)N;
    p->na = na;
    p->np = desc->n_patches;
    p->dx = 2.0 / (n - 1);
    p->h = desc->h > 0.0 ? desc->h : p->dx;
    p->lambda = desc->lambda;
    p->sigma = sig_max;           // the largest sigma(x): selects the diffusion kernels and the reach
    p->beta = 1.0 / (1.0 + p->lambda * p->h);
    p->hl = p->h * desc->cost;
    p->lmax = lx_max + ma_max;
    p->uob = p->lambda > 0.0 ? p->h * p->lmax / (1.0 - p->beta) : 1e6;
    p->has_drift = drift != nullptr;
    p->n_free_total = n_free_total;
    p->along = along;
    {
        // the foot moves about h |f| / dx cells, so 1 - beta Lambda0 ~ that distance and
        // FP32 rounding of the numerator of eq. SLscheme3 grows by its inverse; the
        // mean |f| over free nodes stands for the minimising controls' speed
        const double fmean = n_free_total > 0 ? fsum / (double)n_free_total : 1.0;
        const double cells = p->h * fmean / p->dx;
        p->amp32 = cells > 0.0 ? std::min(64.0, std::max(1.0, 1.0 / cells)) : 64.0;
    }
    // offsets: |h f| <= h (c |a| + |b|); the diffusion adds sqrt(2h) sigma (axes)
    // or sqrt(2h) sigma |a| (along the control)
    p->reach = (p->h * (cmax * amax + bmax) + std::sqrt(2.0 * p->h) * p->sigma * (along ? amax : 1.0)) /
               p->dx;
    p->halo = sweep_halo(p->reach);
    p->halo_c = sweep_halo(p->h * (cmax * amax + bmax) / p->dx);
    if (p->halo > 64)
        return bail(fail(HJB_ERR_INVALID_ARG, "interpolation reach %.1f cells is too large (max 63)", p->reach));
    {
        // automatic tile schedule: when the diffusion offset sqrt(2h) sigma reaches
        // past one cell the scheme couples nodes of equal value (no upwind
        // diffusion ball, Section 4.1) and 8x8 tiles in single-band waves are
        // faster; otherwise 8x4 tiles in two-band waves (measured on the
        // 1025^2 workload and on the 4097^2 / 64-control workload); grids above 2049^2 or more
        // than 32 controls keep enough tiles in flight per step that the larger
        // 8x8 tiles (half the halo staging per node) win there too
        const double dcell = std::sqrt(2.0 * p->h) * p->sigma / p->dx;
        const bool wide = dcell > 1.0;
        const bool big = desc->n > 2049 || desc->n_controls > 32;
        if (p->desc.tile_shape < 0) p->desc.tile_shape = (wide || big) ? 0 : 1;
        if (p->desc.tile_waves <= 0) p->desc.tile_waves = wide ? 1 : 2;
        // one node at a time (lanes over controls) by default: with a period of
        // one step it is the fastest form at every diffusion measured (1025^2,
        // sigma 0.1: 31.4 ms against 46.9 ms for 32 nodes at a time); node-per-lane
        // visits (visit 2) sweep a tile three times per visit (the group of 32 is a
        // Jacobi step)
        // with 64 controls closed under quarter turns, two nodes at a time
        // (visit 3: 4097^2 FP32 passes 235 -> 210 ms, 2049^2 55 -> 51 ms), decided
        // once the control table is known
        p->visit_auto = p->desc.visit == 0;
        if (p->desc.visit == 0) p->desc.visit = 1;
        if (p->desc.local_sweeps <= 0)
            p->desc.local_sweeps = (p->desc.schedule == 0 && p->desc.visit == 2) ? 3 : 1;
    }
    p->shape = p->desc.schedule == 0 ? 1 + p->desc.tile_shape : 0;
    if (p->desc.schedule != 1 && p->desc.coarse_n > 0 &&
        tile_smem(true, desc->n_controls, p->halo, p->shape) > 200 * 1024)
        return bail(fail(HJB_ERR_INVALID_ARG,
                         "interpolation reach %.1f cells is too large for the tile schedules "
                         "(shared memory); use schedule 1", p->reach));
    if (terms && terms->sigma_field) {
        CUP(palloc(&p->sigf, N * sizeof(float), p->st));
        CUP(cudaMemcpyAsync(p->sigf, terms->sigma_field, N * sizeof(float), cudaMemcpyHostToDevice, p->st));
    }
    if (terms && terms->cost_field) {
        CUP(palloc(&p->costf, N * sizeof(float), p->st));
        CUP(cudaMemcpyAsync(p->costf, terms->cost_field, N * sizeof(float), cudaMemcpyHostToDevice, p->st));
    }
    if (terms && terms->control_cost) {
        std::vector<float> h32(na);
        std::vector<double> h64(na);
        for (int m = 0; m < na; ++m) {
            h64[m] = p->h * terms->control_cost[m];
            h32[m] = (float)h64[m];
        }
        CUP(palloc(&p->hm32, na * sizeof(float), p->st));
        CUP(palloc(&p->hm64, na * sizeof(double), p->st));
        CUP(cudaMemcpyAsync(p->hm32, h32.data(), na * sizeof(float), cudaMemcpyHostToDevice, p->st));
        CUP(cudaMemcpyAsync(p->hm64, h64.data(), na * sizeof(double), cudaMemcpyHostToDevice, p->st));
    }
    p->gen = p->sigf || p->costf || p->hm32;
    {
        std::vector<float2> c32(na);
        std::vector<double2> c64(na);
        for (int m = 0; m < na; ++m) {
            c32[m] = make_float2((float)controls[2 * m], (float)controls[2 * m + 1]);
            c64[m] = make_double2(controls[2 * m], controls[2 * m + 1]);
        }
        // opposite pairs a_{m+32} = -a_m up to 1e-12 (evenly spaced directions
        // from cos/sin: components near zero differ by ~1e-16); the foot points
        // of such a pair then mirror each other to far below the FP32 rounding
        // of the cell fractions (6e-8 of a cell)
        p->ctrl_sym = na == 64;
        for (int m = 0; m < 32 && p->ctrl_sym; ++m)
            p->ctrl_sym = std::fabs(controls[2 * (m + 32)] + controls[2 * m]) <= 1e-12 &&
                          std::fabs(controls[2 * (m + 32) + 1] + controls[2 * m + 1]) <= 1e-12;
        // 32 controls in opposite pairs a_{m+16} = -a_m
        p->ctrl_sym32 = na == 32;
        for (int m = 0; m < 16 && p->ctrl_sym32; ++m)
            p->ctrl_sym32 = std::fabs(controls[2 * (m + 16)] + controls[2 * m]) <= 1e-12 &&
                            std::fabs(controls[2 * (m + 16) + 1] + controls[2 * m + 1]) <= 1e-12;
        // and quarter turns: a_{m+8} = (-a_m.y, a_m.x), a_{m+24} = (a_m.y, -a_m.x)
        p->ctrl_rot32 = p->ctrl_sym32;
        for (int m = 0; m < 8 && p->ctrl_rot32; ++m)
            p->ctrl_rot32 = std::fabs(controls[2 * (m + 8)] + controls[2 * m + 1]) <= 1e-12 &&
                            std::fabs(controls[2 * (m + 8) + 1] - controls[2 * m]) <= 1e-12 &&
                            std::fabs(controls[2 * (m + 24)] - controls[2 * m + 1]) <= 1e-12 &&
                            std::fabs(controls[2 * (m + 24) + 1] + controls[2 * m]) <= 1e-12;
        // quarter turns as well: a_{m+16} = (-a_m.y, a_m.x), a_{m+48} = (a_m.y, -a_m.x)
        p->ctrl_rot = p->ctrl_sym;
        for (int m = 0; m < 16 && p->ctrl_rot; ++m)
            p->ctrl_rot = std::fabs(controls[2 * (m + 16)] + controls[2 * m + 1]) <= 1e-12 &&
                          std::fabs(controls[2 * (m + 16) + 1] - controls[2 * m]) <= 1e-12 &&
                          std::fabs(controls[2 * (m + 48)] - controls[2 * m + 1]) <= 1e-12 &&
                          std::fabs(controls[2 * (m + 48) + 1] + controls[2 * m]) <= 1e-12;
        CUP(palloc(&p->ctrl32, na * sizeof(float2), p->st));
        CUP(palloc(&p->ctrl64, na * sizeof(double2), p->st));
        CUP(cudaMemcpyAsync(p->ctrl32, c32.data(), na * sizeof(float2), cudaMemcpyHostToDevice, p->st));
        CUP(cudaMemcpyAsync(p->ctrl64, c64.data(), na * sizeof(double2), cudaMemcpyHostToDevice, p->st));
    }
    CUP(palloc(&p->u32, N * sizeof(float), p->st));
    CUP(palloc(&p->u32b, N * sizeof(float), p->st));
    CUP(palloc(&p->u64, N * sizeof(double), p->st));
    CUP(palloc(&p->u64b, N * sizeof(double), p->st));
    CUP(palloc(&p->scratch, sizeof(Scalars), p->st));
    CUP(cudaMemsetAsync(p->scratch, 0, sizeof(Scalars), p->st));
    CUP(pinned_alloc(&p->host_pinned, sizeof(Scalars)));
    CUP(launch_init_values(p->N, p->mask, 0.0f, (float)p->uob, p->u32, p->u64, p->uob, p->st));
    {
        // band edges of the causal ordering (exact keys, see band_key)
        std::vector<double> e;
        band_edges(p->lambda, p->desc.band_width * p->h, kBandCap, e);
        p->band_L = (int)e.size();
        if (p->band_L > 0) {
            CUP(palloc(&p->band_e, e.size() * sizeof(double), p->st));
            CUP(cudaMemcpyAsync(p->band_e, e.data(), e.size() * sizeof(double), cudaMemcpyHostToDevice,
                                p->st));
        }
    }

    if (desc->coarse_n > 0) {
        const int nc = desc->coarse_n;
        p->nc = nc;
        p->r = (n - 1) / (nc - 1);
        p->hc = p->h * p->r;
        p->beta_c = 1.0 / (1.0 + p->lambda * p->hc);
        p->hl_c = p->hc * desc->cost;
        p->uob_c = p->lambda > 0.0 ? p->hc * p->lmax / (1.0 - p->beta_c) : 1e6;
        const size_t Nc = (size_t)nc * nc;
        if (terms && terms->cost_field) {
            // l(x) of the coarse grid: the fine value at the nested node (rI, rJ)
            std::vector<float> lc(Nc);
            for (int J = 0; J < nc; ++J)
                for (int I = 0; I < nc; ++I)
                    lc[(size_t)J * nc + I] = terms->cost_field[(size_t)(p->r * J) * n + (size_t)(p->r * I)];
            CUP(palloc(&p->costf_c, Nc * sizeof(float), p->st));
            CUP(cudaMemcpyAsync(p->costf_c, lc.data(), Nc * sizeof(float), cudaMemcpyHostToDevice, p->st));
        }
        if (terms && terms->control_cost) {
            std::vector<float> h32(na);
            std::vector<double> h64(na);
            for (int m = 0; m < na; ++m) {
                h64[m] = p->hc * terms->control_cost[m];
                h32[m] = (float)h64[m];
            }
            CUP(palloc(&p->hmc32, na * sizeof(float), p->st));
            CUP(palloc(&p->hmc64, na * sizeof(double), p->st));
            CUP(cudaMemcpyAsync(p->hmc32, h32.data(), na * sizeof(float), cudaMemcpyHostToDevice, p->st));
            CUP(cudaMemcpyAsync(p->hmc64, h64.data(), na * sizeof(double), cudaMemcpyHostToDevice, p->st));
        }
        p->relax_blocks = grid_relax_plan(nc, na, p->halo_c, p->num_sms, false, &p->relax_plan);
        if (p->relax_blocks <= 0)
            return bail(fail(HJB_ERR_INVALID_ARG, "coarse_n=%d: no co-resident tiling for the coarse "
                                                  "solve", nc));
        CUP(palloc(&p->speed_c, Nc * sizeof(float), p->st));
        CUP(palloc(&p->mask_c, Nc, p->st));
        CUP(palloc(&p->uc, Nc * sizeof(float), p->st));
        if (drift) CUP(palloc(&p->drift_c, Nc * sizeof(float2), p->st));
        CUP(launch_coarse_data(n, nc, p->speed, p->drift, p->mask, p->speed_c, p->drift_c,
                               p->mask_c, p->st));
        CUP(palloc(&p->uhat, N * sizeof(float), p->st));
        CUP(palloc(&p->a, N, p->st));
        CUP(palloc(&p->succ, N * sizeof(int32_t), p->st));
        CUP(palloc(&p->jump_a, N * sizeof(int32_t), p->st));
        CUP(palloc(&p->jump_b, N * sizeof(int32_t), p->st));
        CUP(palloc(&p->label, N, p->st));
        CUP(palloc(&p->key, N * sizeof(int32_t), p->st));
        CUP(palloc(&p->order, N * sizeof(int32_t), p->st));
        const bool warp_tiles = p->desc.schedule == 0;
        int tw = kTileSize, th = kTileSize;
        if (warp_tiles) wtile_dims(p->shape, &tw, &th);
        p->ntx = (n + tw - 1) / tw;
        p->nty = (n + th - 1) / th;
        p->nt = p->ntx * p->nty;
        p->act_radius = std::max(1, (p->halo + std::min(tw, th) - 1) / std::min(tw, th));
        const size_t nt = p->nt;
        CUP(palloc(&p->tile_min, nt * sizeof(int32_t), p->st));
        CUP(palloc(&p->tile_wave, nt * sizeof(int32_t), p->st));
        CUP(palloc(&p->tile_key, nt * sizeof(int32_t), p->st));
        CUP(palloc(&p->tile_list, nt * sizeof(int32_t), p->st));
        CUP(palloc(&p->tile_inc, nt * sizeof(unsigned int), p->st));
        if (warp_tiles) {
            CUP(palloc(&p->wt_nodes, nt * kWarpTileNodes * sizeof(int32_t), p->st));
            CUP(palloc(&p->wt_speed, nt * kWarpTileNodes * sizeof(float), p->st));
            CUP(palloc(&p->wt_count, nt * sizeof(int32_t), p->st));
            CUP(palloc(&p->wt_stamp, nt * sizeof(int32_t), p->st));
            CUP(palloc(&p->wt_queue, (p->desc.tile_period + 2) * nt * sizeof(int32_t), p->st));
            CUP(palloc(&p->wt_qcount, (p->desc.tile_period + 2) * sizeof(int32_t), p->st));
            CUP(palloc(&p->cb_wave, nt * sizeof(int32_t), p->st));
            CUP(palloc(&p->cb_key, nt * sizeof(int32_t), p->st));
            CUP(palloc(&p->cb_list, nt * sizeof(int32_t), p->st));
            CUP(palloc(&p->cb_off, 3 * sizeof(int32_t), p->st));
            CUP(palloc(&p->cb_count, 2 * sizeof(int32_t), p->st));
            CUP(palloc(&p->tinst, sizeof(TileInst), p->st));
            CUP(palloc(&p->rank_boff, 2 * sizeof(int32_t), p->st));
        } else {
            CUP(palloc(&p->tile_key2, N * sizeof(int32_t), p->st));
            CUP(palloc(&p->tile_nodes, N * sizeof(int32_t), p->st));
            CUP(palloc(&p->tile_bin_count, nt * kLocalBands * sizeof(int32_t), p->st));
            CUP(palloc(&p->tile_bin_off, (nt * kLocalBands + 1) * sizeof(int32_t), p->st));
        }
        CUP(palloc(&p->res_off, (p->desc.tile_period + 1) * sizeof(int32_t), p->st));
        CUP(palloc(&p->step_inc, 2 * p->desc.tile_period * sizeof(unsigned int), p->st));
    }
    const bool sig = p->sigma > 0.0;
    {
        p->tile_blocks32 = std::max(1, tile_blocks_per_sm(false, sig, na, p->halo, p->shape)) * p->num_sms;
        p->tile_blocks64 = std::max(1, tile_blocks_per_sm(true, sig, na, p->halo, p->shape)) * p->num_sms;
    }
    if (p->tinst) {
        // the problem as a one-instance batch of the warp-tile kernel
        int tw, th;
        wtile_dims(p->shape, &tw, &th);
        TileInst ti{};
        ti.g = p->fine_view();
        ti.u32 = p->u32;
        ti.u64 = p->u64;
        ti.uhat = p->uhat;
        ti.lambda = (float)p->lambda;
        ti.band_w = (float)(p->desc.band_width * p->h);
        ti.R = p->halo;
        ti.ntx = p->ntx;
        ti.nty = p->nty;
        ti.tile_off = 0;
        ti.act_radius = p->act_radius;
        const int wv = tw + 2 * p->halo;
        p->max_wh = (p->desc.visit == 2 ? tile_pitch(wv) : wv) * (th + 2 * p->halo);
        CUP(cudaMemcpyAsync(p->tinst, &ti, sizeof(ti), cudaMemcpyHostToDevice, p->st));
        // blocks per SM with the (padded) staging slices the launches use
        p->tile_blocks32 = std::max(1, wtile_blocks_per_sm(false, sig, na, p->max_wh, p->shape)) * p->num_sms;
        p->tile_blocks64 = std::max(1, wtile_blocks_per_sm(true, sig, na, p->max_wh, p->shape)) * p->num_sms;
    }
    p->wave_blocks32 = std::max(1, wave_blocks_per_sm(false, sig, na)) * p->num_sms;
    p->wave_blocks64 = std::max(1, wave_blocks_per_sm(true, sig, na)) * p->num_sms;
    CUP(cudaStreamSynchronize(p->st));
#undef CUP
    *out = p;
    return HJB_OK;
}

int ensure_hist(hjb_problem* p, int cap) {
    if (p->hist_cap >= cap) return HJB_OK;
    pfree(p->inc_hist32, p->st);
    pfree(p->inc_hist64, p->st);
    CU(palloc(&p->inc_hist32, sizeof(unsigned int) * (size_t)cap, p->st));
    CU(palloc(&p->inc_hist64, sizeof(unsigned long long) * (size_t)cap, p->st));
    p->hist_cap = cap;
    return HJB_OK;
}

// Plain Jacobi sweeps u <- T u (double buffered) until the sup-increment of a
// sweep is <= tol; the increment of every sweep lands in inc_hist, checked on
// the host every kCheck sweeps.  Returns the sweeps done in *sweeps and the
// last increment in *last; the result is in buf[0].
// Plain Jacobi sweeps u <- T u (double buffered) on the grid `g` until the
// sup-increment of a sweep is <= tol; the increment of every sweep lands in
// inc_hist, checked on the host every kCheck sweeps.  Returns the sweeps done
// in *sweeps and the last increment in *last; the result is in buf0.
template <typename T, typename Bits, typename Launch>
int jacobi_loop_impl(hjb_problem* p, Bits* hist, T* buf0, T* buf1, int N, double tol,
                     int max_sweeps, int* sweeps, double* last, bool* converged,
                     const Launch& launch) {
    constexpr int kCheck = 8;
    CU(cudaMemsetAsync(hist, 0, sizeof(Bits) * (size_t)(max_sweeps + kCheck), p->st));
    std::vector<Bits> h(kCheck);
    T* cur = buf0;
    T* nxt = buf1;
    int s = 0;
    *converged = false;
    *last = -1.0;
    while (s < max_sweeps) {
        const int chunk = std::min(kCheck, max_sweeps - s);
        for (int c = 0; c < chunk; ++c) {
            CU(launch(cur, nxt, hist + s + c));
            std::swap(cur, nxt);
        }
        CU(cudaMemcpyAsync(h.data(), hist + s, sizeof(Bits) * chunk, cudaMemcpyDeviceToHost, p->st));
        CU(cudaStreamSynchronize(p->st));
        s += chunk;
        // first sweep of the chunk that met the tolerance
        for (int c = 0; c < chunk; ++c) {
            T v;
            std::memcpy(&v, &h[c], sizeof(T));
            *last = (double)v;
            if ((double)v <= tol) {
                *converged = true;
                break;
            }
        }
        if (*converged) break;
    }
    if (cur != buf0) CU(cudaMemcpyAsync(buf0, cur, sizeof(T) * (size_t)N, cudaMemcpyDeviceToDevice, p->st));
    *sweeps = s;
    return HJB_OK;
}

int jacobi32(hjb_problem* p, const GridView& g, int halo, float* buf0, float* buf1, double tol,
             int max_sweeps, int* sweeps, double* last, bool* converged) {
    int rc = ensure_hist(p, max_sweeps + 8);
    if (rc) return rc;
    const bool sig = g.d64 > 0.0;
    const int scheme = p->desc.scheme;
    return jacobi_loop_impl<float>(p, p->inc_hist32, buf0, buf1, g.n * g.n, tol, max_sweeps, sweeps,
                                   last, converged,
                                   [&](const float* a, float* b, unsigned int* inc) {
                                       return launch_sweep_f32(g, sig, scheme, halo, a, b, nullptr,
                                                               inc, p->st);
                                   });
}

int jacobi64(hjb_problem* p, double* buf0, double* buf1, double tol, int max_sweeps, int* sweeps,
             double* last, bool* converged) {
    int rc = ensure_hist(p, max_sweeps + 8);
    if (rc) return rc;
    const GridView g = p->fine_view();
    const bool sig = p->sigma > 0.0;
    const int scheme = p->desc.scheme;
    return jacobi_loop_impl<double>(p, p->inc_hist64, buf0, buf1, p->N, tol, max_sweeps, sweeps,
                                    last, converged,
                                    [&](const double* a, double* b, unsigned long long* inc) {
                                        return launch_sweep_f64(g, sig, scheme, p->halo, a, b,
                                                                nullptr, inc, p->st);
                                    });
}

// Screening margin of the FP64 residual.  With every value in [0, U]
// (U = l/lambda + h l; eps = 2^-24), an FP32 candidate beta Sd + c0 differs from
// the FP64 one by at most E = (20 + 10 reach) eps U:
//  - the FP32 copies of the values: 2 eps U in Sd (a node's and a vertex's);
//  - the arithmetic on the differences v - uk (each of magnitude <= U): 9 eps U
//    per bilinear point, 12 eps U for the four points' sums and the quarter, about
//    6 eps U for beta, c0 = h l - (1 - beta) uk and the last FMA: 18 eps U;
//  - the point positions: the foot s c a and the offset d carry at most 5 eps
//    reach cells of rounding per axis, and the interpolant moves by at most U per
//    cell along each axis: 10 eps reach U.
// The margin is 2.2 E (the FP64 candidates' own rounding is far below the 0.2 E
// left over): every control within it of the FP32 minimum is evaluated in FP64,
// so the FP64 minimiser always survives and the result is the full FP64
// residual; at the 4097^2 workload's reach (2.4 cells) 5.8e-6 U.
float screening_margin(const hjb_problem* p) {
    const double U = std::max(1.0, p->value_bound());
    const double E = (20.0 + 10.0 * p->reach) * std::ldexp(1.0, -24) * U;
    return (float)(2.2 * E);
}

// FP64 sup-residual ||T2 u - u|| of u64 (FP32-screened, exact FP64 value).
int residual64(hjb_problem* p, double* out, bool fields = false) {
    Scalars* ds = dscal(p);
    if (fields && !p->corr_r) {
        CU(palloc(&p->corr_r, sizeof(float) * (size_t)p->N, p->st));
        CU(palloc(&p->corr_a, (size_t)p->N, p->st));
    }
    CU(cudaMemsetAsync(&ds->inc64, 0, sizeof(unsigned long long), p->st));
    CU(launch_residual_screened(p->fine_view(), p->sigma > 0.0, p->halo, p->u64,
                                screening_margin(p), &ds->inc64, p->st,
                                fields ? p->corr_r : nullptr, fields ? p->corr_a : nullptr));
    unsigned long long bits = 0;
    CU(cudaMemcpyAsync(&hscal(p)->inc64, &ds->inc64, sizeof(bits), cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    bits = hscal(p)->inc64;
    std::memcpy(out, &bits, sizeof(double));
    return HJB_OK;
}

// Band-ordered passes on u32 (f64 = false) or u64 (f64 = true).
int run_waves(hjb_problem* p, bool f64, double tol, int max_passes, WaveResult* out) {
    Scalars* ds = dscal(p);
    CU(cudaMemsetAsync(&ds->wave, 0, sizeof(WaveResult), p->st));
    CU(cudaMemsetAsync(&ds->sync, 0, sizeof(GridSync), p->st));
    WaveArgs a{};
    a.g = p->fine_view();
    a.scheme = p->desc.scheme;
    a.order = p->order;
    a.band_off = p->band_off;
    a.n_bands = p->n_bands;
    a.group = p->desc.band_group;
    a.n_groups = (p->n_bands + a.group - 1) / a.group;
    a.window = std::max(1, (p->desc.band_window + a.group - 1) / a.group);
    a.tol = (float)tol;
    a.max_passes = max_passes;
    a.inc_bits = p->inc_bits;
    a.sync = &ds->sync;
    a.res = &ds->wave;
    a.timeout_ns = kTimeoutNs;
    const bool sig = p->sigma > 0.0;
    int blocks = f64 ? p->wave_blocks64 : p->wave_blocks32;
    if (p->desc.wave_warps > 0) {
        const int want = (p->desc.wave_warps + wave_threads() / 32 - 1) / (wave_threads() / 32);
        blocks = std::max(1, std::min(blocks, want));
    }
    if (f64) {
        CU(launch_waves_f64(a, p->u64, sig, blocks, p->st));
    } else {
        CU(launch_waves_f32(a, p->u32, sig, blocks, p->st));
    }
    CU(cudaMemcpyAsync(&hscal(p)->wave, &ds->wave, sizeof(WaveResult), cudaMemcpyDeviceToHost, p->st));
    CU(cudaMemcpyAsync(&hscal(p)->sync, &ds->sync, sizeof(GridSync), cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    *out = hscal(p)->wave;
    if (hscal(p)->sync.err != 0)
        return fail(hscal(p)->sync.err, "band-wave kernel: a grid-wide wait exceeded its limit");
    return HJB_OK;
}

int rebuild_order(hjb_problem* p) {
    // successors -> labels -> (band, patch) ordering, from p->a and p->key
    const GridView g = p->fine_view();
    // successors and the pointer-jumping rounds of the labels: a short-kernel
    // sequence over fixed buffers, replayed from a CUDA graph
    CU(p->labels_graph.run(p->st, [&](cudaStream_t st) {
        cudaError_t e = launch_successors(g, p->a, p->succ, st);
        if (e != cudaSuccess) return e;
        return launch_labels(p->N, p->succ, p->mask, p->sector, p->np, p->jump_a, p->jump_b, p->label, st);
    }));
    const int bins = p->n_bands * (p->np + 1);
    if (bins > p->bins_cap) {
        pfree(p->bin_count, p->st);
        pfree(p->bin_off, p->st);
        CU(palloc(&p->bin_count, sizeof(int32_t) * (size_t)bins, p->st));
        CU(palloc(&p->bin_off, sizeof(int32_t) * (size_t)(bins + 1), p->st));
        p->bins_cap = bins;
    }
    if (p->n_bands > p->bands_cap) {
        pfree(p->band_off, p->st);
        pfree(p->inc_bits, p->st);
        CU(palloc(&p->band_off, sizeof(int32_t) * (size_t)(p->n_bands + 1), p->st));
        CU(palloc(&p->inc_bits, sizeof(unsigned int) * 2 * (size_t)p->n_bands, p->st));
        p->bands_cap = p->n_bands;
    }
    CU(cudaMemsetAsync(p->inc_bits, 0, sizeof(unsigned int) * 2 * (size_t)p->n_bands, p->st));
    CU(launch_order(p->N, p->key, p->label, p->mask, p->np, p->n_bands, p->bin_count, p->bin_off,
                    p->order, p->band_off, p->st));
    return HJB_OK;
}

// Tile schedule from the band keys.  Warp tiles: nodes of each tile sorted by
// the key value, tiles grouped into waves by their lowest band and sorted by
// wave.  Block tiles: nodes sorted by (tile, local band), tiles sorted by
// (wave mod D, wave).
int build_tiles(hjb_problem* p, const float* key_val) {
    if (p->desc.schedule == 1) return HJB_OK;     // band waves need no tiles
    const int B = p->desc.tile_waves, D = p->desc.tile_period;
    if (p->desc.schedule == 0) {
        // warp tiles: per-tile exact order by the key value (u_hat or current value)
        CU(launch_wtile_build(p->shape, p->tinst, nullptr, p->nt, key_val == p->u32, kBandCap,
                              p->wt_nodes, p->wt_speed, p->wt_count, p->tile_min, p->st));
    } else {
        CU(cudaMemsetAsync(p->tile_min, 0x7f, sizeof(int32_t) * (size_t)p->nt, p->st));
        CU(launch_tile_min(p->n, p->ntx, p->key, p->mask, p->tile_min, p->st));
        CU(launch_tile_node_keys(p->n, p->ntx, p->key, p->mask, p->tile_min, p->tile_key2, p->st));
        CU(launch_counting_sort(p->N, p->tile_key2, p->nt * kLocalBands, p->tile_bin_count,
                                p->tile_bin_off, p->tile_nodes, p->st));
    }
    p->n_waves = (std::max(p->n_bands, 1) - 1) / B + 1;
    if (p->desc.schedule == 0) {
        // dense waves: rank of each tile's lowest band among the distinct ones
        const int S = std::max(p->n_bands, 1);
        if (S + 1 > p->rank_cap) {
            pfree(p->rank_flags, p->st);
            pfree(p->rank_scan, p->st);
            CU(palloc(&p->rank_flags, sizeof(int32_t) * (size_t)(S + 1), p->st));
            CU(palloc(&p->rank_scan, sizeof(int32_t) * (size_t)(S + 1), p->st));
            p->rank_cap = S + 1;
        }
        const int32_t boff[2] = {0, S};
        CU(cudaMemcpyAsync(p->rank_boff, boff, sizeof(boff), cudaMemcpyHostToDevice, p->st));
        Scalars* ds = dscal(p);
        CU(launch_dense_waves(p->nt, p->tile_min, nullptr, 1, p->rank_boff, S, B, p->rank_flags,
                              p->rank_scan, p->tile_wave, p->tile_key, &ds->n_waves, p->st));
        CU(cudaMemcpyAsync(&hscal(p)->n_waves, &ds->n_waves, sizeof(int), cudaMemcpyDeviceToHost, p->st));
        CU(cudaStreamSynchronize(p->st));
        p->n_waves = std::max(1, hscal(p)->n_waves);
    }
    // warp tiles: sorted by wave alone (sched_off = wave offsets); block tiles:
    // by (wave mod D, wave)
    const int Dk = p->desc.schedule == 0 ? 1 : D;
    const int bins = Dk * p->n_waves;
    if (bins > p->sched_cap) {
        pfree(p->sched_count, p->st);
        pfree(p->sched_off, p->st);
        CU(palloc(&p->sched_count, sizeof(int32_t) * (size_t)bins, p->st));
        CU(palloc(&p->sched_off, sizeof(int32_t) * (size_t)(bins + 1), p->st));
        p->sched_cap = bins;
    }
    if (p->desc.schedule != 0)
        CU(launch_tile_waves(p->nt, p->tile_min, B, Dk, p->n_waves, p->tile_wave, p->tile_key,
                             p->tile_inc, p->st));
    CU(launch_counting_sort(p->nt, p->tile_key, bins, p->sched_count, p->sched_off, p->tile_list,
                            p->st));
    if (p->desc.schedule != 0) {
        CU(launch_strided_gather(D, p->n_waves, p->sched_off, p->res_off, p->st));
    } else {
        // warm-restart schedule: tiles with free nodes in two checkerboard waves
        CU(launch_checker_waves(p->tinst, nullptr, p->nt, p->wt_count, p->cb_wave, p->cb_key, p->st));
        CU(launch_counting_sort(p->nt, p->cb_key, 2, p->cb_count, p->cb_off, p->cb_list, p->st));
    }
    return HJB_OK;
}

// Tile-pipelined passes on u32 (f64 = false) or u64 (f64 = true).  warm (warp
// tiles only): every tile is visited in the first two steps, in checkerboard
// order, instead of along the causal waves -- for a value already close to
// the fixed point.
int run_tiles(hjb_problem* p, bool f64, double tol, int max_passes, WaveResult* out,
              bool warm = false) {
    warm = warm && p->desc.schedule == 0;
    const int32_t* waves = warm ? p->cb_wave : p->tile_wave;
    const int n_waves = warm ? 2 : p->n_waves;
    Scalars* ds = dscal(p);
    const int B = p->desc.tile_waves, D = p->desc.tile_period;
    CU(cudaMemsetAsync(&ds->wave, 0, sizeof(WaveResult), p->st));
    CU(cudaMemsetAsync(&ds->sync, 0, sizeof(GridSync), p->st));
    CU(cudaMemsetAsync(p->step_inc, 0, sizeof(unsigned int) * 2 * D, p->st));
    if (p->desc.schedule == 0) {
        // empty queues; no tile is queued for a step up to its own wave
        CU(cudaMemsetAsync(p->wt_qcount, 0, sizeof(int32_t) * (D + 2), p->st));
        CU(launch_tile_stamps(p->nt, waves, p->wt_stamp, p->st));
    } else {
        // every tile with free nodes starts as changed
        CU(launch_tile_waves(p->nt, p->tile_min, B, D, p->n_waves, p->tile_wave, p->tile_key,
                             p->tile_inc, p->st));
    }
    TileArgs a{};
    a.g = p->fine_view();
    a.scheme = p->desc.scheme;
    a.halo = p->halo;
    a.warp_tiles = p->shape;
    a.act_radius = p->act_radius;
    a.nodes = a.warp_tiles ? p->wt_nodes : p->tile_nodes;
    a.bin_off = p->tile_bin_off;
    a.wt_count = p->wt_count;
    a.tile_list = warm ? p->cb_list : p->tile_list;
    a.res_off = p->res_off;
    a.tile_wave = waves;
    a.tile_inc = p->tile_inc;
    a.wave_off = warm ? p->cb_off : p->sched_off;
    a.slot_speed = p->wt_speed;
    a.stamp = p->wt_stamp;
    a.queue = p->wt_queue;
    a.qcount = p->wt_qcount;
    a.nt = p->nt;
    a.step_inc = p->step_inc;
    a.ntx = p->ntx;
    a.nty = p->nty;
    a.n_waves = n_waves;
    a.period = D;
    a.local_sweeps = p->desc.local_sweeps;
    a.node_lanes = p->desc.visit == 2 ? 1 : 0;
    a.ctrl_sym = p->ctrl_sym && !p->gen && p->drift == nullptr ? 1 : 0;
    {
        // the self weight of eq. self-dependency is zero for every candidate when
        // each diffusion point lies more than a cell from the node: offset d
        // beyond 1 + the drift's reach (interior tiles; the projection can pull
        // points back next to nodes at the edge).  Scheme 2 keeps it in the sum.
        const double dcell = std::sqrt(2.0 * p->h) * p->sigma / p->dx;
        const double drift_cells = p->reach - dcell;
        a.no_self = p->desc.scheme == 2 ? 2 : (p->sigma > 0.0 && dcell >= 1.0 + drift_cells + 1e-3 ? 1 : 0);
    }
    {
        // node groups, automatic where the control set allows them: 64 controls
        // closed under quarter turns two nodes at a time (visit 3; 4097^2: FP32
        // passes 235 -> 210 ms), 32 closed under quarter turns four at a time
        // (visit 4; 1025^2: sigma 0 6.62 -> 5.83 ms, 0.02 8.90 -> 8.14 ms, 0.1
        // 31.7 -> 29.1 ms), 32 opposite pairs only two at a time (visit 3)
        const bool plain = !p->gen && p->drift == nullptr;
        const bool aut = p->visit_auto;
        if (plain && (p->desc.visit == 3 || aut) && p->ctrl_sym && p->ctrl_rot)
            a.node_pairs = 1;
        else if (plain && (p->desc.visit == 4 || aut) && p->ctrl_rot32)
            a.node_pairs = 3;
        else if (plain && (p->desc.visit == 3 || (aut && a.no_self == 0)) && p->ctrl_sym32)
            a.node_pairs = 2;
        else
            a.node_pairs = 0;
    }
    a.max_steps = n_waves + max_passes * D;
    a.tol = (float)tol;
    a.sync = &ds->sync;
    a.res = &ds->wave;
    a.timeout_ns = kTimeoutNs;
    a.insts = p->tinst;
    a.tile_inst = nullptr;
    a.inst_active = nullptr;
    a.max_wh = p->max_wh;
    const bool sig = p->sigma > 0.0;
    int blocks = f64 ? p->tile_blocks64 : p->tile_blocks32;
    if (p->desc.wave_warps > 0) {
        const int wpb = tile_threads(f64, p->shape) / 32;
        const int want = (p->desc.wave_warps + wpb - 1) / wpb;
        blocks = std::max(1, std::min(blocks, want));
    }
    if (p->desc.schedule == 0 && p->async && !f64 && !warm) {
        // the asynchronous worklist: ring sized above the tiles plus one waiting
        // ticket per warp
        const int warps = blocks * (tile_threads(false, p->shape) / 32);
        int cap = 1024;
        while (cap < p->nt + warps + 64) cap <<= 1;
        if (cap > p->a_cap) {
            pfree(p->a_state, p->st); pfree(p->a_deps, p->st); pfree(p->a_queue, p->st);
    pfree(p->corr_r, p->st); pfree(p->corr_a, p->st);
            CU(palloc(&p->a_state, sizeof(int32_t) * (size_t)p->nt, p->st));
            CU(palloc(&p->a_deps, sizeof(int32_t) * (size_t)p->nt, p->st));
            CU(palloc(&p->a_queue, sizeof(unsigned long long) * (size_t)cap, p->st));
            p->a_cap = cap;
        }
        CU(cudaMemsetAsync(p->a_queue, 0, sizeof(unsigned long long) * (size_t)p->a_cap, p->st));
        CU(cudaMemsetAsync(&ds->actl, 0, sizeof(AsyncCtl), p->st));
        a.astate = p->a_state;
        a.adeps = p->a_deps;
        a.aqueue = p->a_queue;
        a.aq_cap = p->a_cap;
        a.actl = &ds->actl;
        a.max_visits = (long long)max_passes * p->nt;
        a.tile_cap = std::min(max_passes, kTileVisitCap);
        CU(launch_wtiles_async(a, sig, blocks, p->st));
        CU(cudaMemcpyAsync(&hscal(p)->actl, &ds->actl, sizeof(AsyncCtl), cudaMemcpyDeviceToHost, p->st));
        CU(cudaMemcpyAsync(&hscal(p)->wave, &ds->wave, sizeof(WaveResult), cudaMemcpyDeviceToHost, p->st));
        CU(cudaMemcpyAsync(&hscal(p)->sync, &ds->sync, sizeof(GridSync), cudaMemcpyDeviceToHost, p->st));
        CU(cudaStreamSynchronize(p->st));
        if (hscal(p)->sync.err == HJB_ERR_TIMEOUT)
            return fail(HJB_ERR_TIMEOUT, "tile worklist: a wait exceeded its limit");
        if (hscal(p)->sync.err != 0) return fail(hscal(p)->sync.err, "tile worklist: internal error");
        *out = hscal(p)->wave;
        // passes = visits per tile with free nodes (the worklist has no steps)
        const long long tiles = std::max(1, p->nt);
        out->passes = (int)((hscal(p)->actl.visits + tiles - 1) / tiles);
        out->converged = (hscal(p)->actl.stop || hscal(p)->actl.capped) ? 0 : 1;
        out->last_increment = (float)tol;
        return HJB_OK;
    }
    if (p->desc.schedule == 0) {
        CU(launch_wtiles(a, f64, sig, blocks, p->st));
    } else if (f64) {
        CU(launch_tiles_f64(a, p->u64, sig, blocks, p->st));
    } else {
        CU(launch_tiles_f32(a, p->u32, sig, blocks, p->st));
    }
    CU(cudaMemcpyAsync(&hscal(p)->wave, &ds->wave, sizeof(WaveResult), cudaMemcpyDeviceToHost, p->st));
    CU(cudaMemcpyAsync(&hscal(p)->sync, &ds->sync, sizeof(GridSync), cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    *out = hscal(p)->wave;
    if (hscal(p)->sync.err == HJB_ERR_TIMEOUT)
        return fail(HJB_ERR_TIMEOUT, "tile kernel: a grid-wide wait exceeded its limit");
    if (hscal(p)->sync.err != 0)
        return fail(hscal(p)->sync.err, "tile kernel: tile queue overflow (internal error)");
    return HJB_OK;
}

// One solve phase with the selected schedule.
int run_phase(hjb_problem* p, bool f64, double tol, int max_passes, WaveResult* out,
              bool warm = false) {
    return p->desc.schedule == 1 ? run_waves(p, f64, tol, max_passes, out)
                                 : run_tiles(p, f64, tol, max_passes, out, warm);
}

// Re-sort the free nodes by the current FP32 value (keys from u32, labels kept).
int resort_by_value(hjb_problem* p) {
    Scalars* ds = dscal(p);
    CU(cudaMemsetAsync(&ds->max_key, 0, sizeof(int), p->st));
    CU(launch_keys_from_values(p->N, p->mask, p->u32, p->band_map(), p->key, &ds->max_key, p->st));
    CU(cudaMemcpyAsync(&hscal(p)->max_key, &ds->max_key, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    p->n_bands = hscal(p)->max_key + 1;
    const int bins = p->n_bands * (p->np + 1);
    if (bins > p->bins_cap) {
        pfree(p->bin_count, p->st);
        pfree(p->bin_off, p->st);
        CU(palloc(&p->bin_count, sizeof(int32_t) * (size_t)bins, p->st));
        CU(palloc(&p->bin_off, sizeof(int32_t) * (size_t)(bins + 1), p->st));
        p->bins_cap = bins;
    }
    if (p->n_bands > p->bands_cap) {
        pfree(p->band_off, p->st);
        pfree(p->inc_bits, p->st);
        CU(palloc(&p->band_off, sizeof(int32_t) * (size_t)(p->n_bands + 1), p->st));
        CU(palloc(&p->inc_bits, sizeof(unsigned int) * 2 * (size_t)p->n_bands, p->st));
        p->bands_cap = p->n_bands;
    }
    CU(cudaMemsetAsync(p->inc_bits, 0, sizeof(unsigned int) * 2 * (size_t)p->n_bands, p->st));
    CU(launch_order(p->N, p->key, p->label, p->mask, p->np, p->n_bands, p->bin_count, p->bin_off,
                    p->order, p->band_off, p->st));
    return build_tiles(p, p->u32);
}

}  // namespace

extern "C" {

const char* hjb_status_string(int code) {
    switch (code) {
        case HJB_OK: return "ok";
        case HJB_ERR_INVALID_ARG: return "invalid argument";
        case HJB_ERR_CUDA: return "CUDA error";
        case HJB_ERR_OOM: return "out of device memory";
        case HJB_ERR_STATE: return "call out of order";
        case HJB_ERR_NOT_CONVERGED: return "not converged (iteration cap reached)";
        case HJB_ERR_TIMEOUT: return "device-side wait timed out";
        default: return "unknown status";
    }
}

const char* hjb_last_error(void) { return g_last_error.c_str(); }

long long hjb_kernel_launches(void) { return hjb::launches(); }

int hjb_regime(double dx, double f_min, double f_max, double eps, hjb_regime_info* out) {
    if (!out || !(dx > 0.0) || !(f_min > 0.0) || !(f_max >= f_min) || !(eps >= 0.0))
        return fail(HJB_ERR_INVALID_ARG, "hjb_regime: need dx>0, 0<f_min<=f_max, eps>=0");
    hjb_regime_info r{};
    r.upsilon = f_max / f_min;
    r.tau_dx = dx / (1.0 + r.upsilon);
    r.alpha = 1.0 / (1.0 + r.upsilon);
    r.eps_threshold = f_min * dx / (2.0 * (1.0 + r.upsilon));
    if (eps > 0.0) {
        r.omega = f_min / (2.0 * eps);
        const double q = r.omega * dx;
        r.alpha_lower = 1.0 / q;
        r.alpha_upper = 1.0 / r.upsilon - (std::sqrt(1.0 + 4.0 * q * r.upsilon) - 1.0) /
                                              (2.0 * q * r.upsilon * r.upsilon);
        r.holds = (1.0 / r.omega < r.tau_dx) ? 1 : 0;
    } else {
        r.omega = INFINITY;
        r.alpha_lower = 0.0;
        r.alpha_upper = 1.0 / r.upsilon;
        r.holds = 1;
    }
    r.h = r.alpha * dx / f_min;
    const double diff = std::sqrt(2.0 * eps * r.h);
    r.upper_ok = (r.h * f_max + diff < dx) ? 1 : 0;
    r.lower_ok = (r.h * f_min - diff > 0.0) ? 1 : 0;
    r.reach_cells = (int)std::ceil((r.h * f_max + diff) / dx);
    *out = r;
    return HJB_OK;
}

int hjb_create_problem(const hjb_desc* desc, const float* speed, const uint8_t* mask,
                       const int8_t* sector, const double* controls, const float* drift,
                       void* cuda_stream, hjb_problem** out) {
    return create_common(desc, speed, mask, sector, controls, drift, cuda_stream, out, false);
}

int hjb_trim_memory(void) {
    g_last_error.clear();
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (auto& pool : g_pools) {
        if (!pool) continue;
        CU(cudaMemPoolTrimTo(pool, 0));
    }
    return HJB_OK;
}

int hjb_create_problem_general(const hjb_desc* desc, const float* speed, const uint8_t* mask,
                               const int8_t* sector, const double* controls, const float* drift,
                               const hjb_terms* terms, void* cuda_stream, hjb_problem** out) {
    return create_common(desc, speed, mask, sector, controls, drift, cuda_stream, out, false, terms);
}

int hjb_create_problem_device(const hjb_desc* desc, const float* speed, const uint8_t* mask,
                              const int8_t* sector, const double* controls, const float* drift,
                              void* cuda_stream, hjb_problem** out) {
    return create_common(desc, speed, mask, sector, controls, drift, cuda_stream, out, true);
}

void hjb_destroy(hjb_problem* p) {
    if (!p) return;
    if (p->st) cudaStreamSynchronize(p->st);
    pfree(p->speed, p->st); pfree(p->drift, p->st); pfree(p->mask, p->st); pfree(p->sector, p->st);
    pfree(p->scan_tmp, p->st);
    pfree(p->ctrl32, p->st); pfree(p->ctrl64, p->st);
    pfree(p->u32, p->st); pfree(p->u32b, p->st); pfree(p->u64, p->st); pfree(p->u64b, p->st);
    pfree(p->speed_c, p->st); pfree(p->drift_c, p->st); pfree(p->mask_c, p->st); pfree(p->uc, p->st);
    pfree(p->sigf, p->st); pfree(p->costf, p->st); pfree(p->costf_c, p->st); pfree(p->hm32, p->st); pfree(p->hm64, p->st);
    pfree(p->hmc32, p->st); pfree(p->hmc64, p->st);
    pfree(p->uhat, p->st); pfree(p->a, p->st); pfree(p->succ, p->st); pfree(p->jump_a, p->st); pfree(p->jump_b, p->st);
    pfree(p->label, p->st); pfree(p->key, p->st); pfree(p->order, p->st); pfree(p->bin_count, p->st); pfree(p->bin_off, p->st);
    pfree(p->band_off, p->st); pfree(p->band_e, p->st); pfree(p->inc_bits, p->st); pfree(p->inc_hist32, p->st); pfree(p->inc_hist64, p->st);
    pfree(p->tile_min, p->st); pfree(p->tile_wave, p->st); pfree(p->tile_key, p->st); pfree(p->tile_list, p->st);
    pfree(p->tile_inc, p->st); pfree(p->tile_key2, p->st); pfree(p->tile_nodes, p->st); pfree(p->tile_bin_count, p->st);
    pfree(p->tile_bin_off, p->st); pfree(p->wt_nodes, p->st); pfree(p->wt_count, p->st); pfree(p->wt_speed, p->st);
    pfree(p->wt_stamp, p->st); pfree(p->wt_queue, p->st); pfree(p->wt_qcount, p->st);
    pfree(p->a_state, p->st); pfree(p->a_deps, p->st); pfree(p->a_queue, p->st);
    pfree(p->cb_wave, p->st); pfree(p->cb_key, p->st); pfree(p->cb_list, p->st); pfree(p->cb_off, p->st); pfree(p->cb_count, p->st);
    pfree(p->tinst, p->st); pfree(p->rank_flags, p->st); pfree(p->rank_scan, p->st); pfree(p->rank_boff, p->st); pfree(p->sched_count, p->st); pfree(p->sched_off, p->st); pfree(p->res_off, p->st);
    pfree(p->step_inc, p->st);
    p->labels_graph.reset();
    pfree(p->scratch, p->st);
    pinned_free(p->host_pinned);
    p->host_pinned = nullptr;
    if (p->own_stream && p->st) cudaStreamDestroy(p->st);
    delete p;
}

int hjb_coarse_solve(hjb_problem* p, double tol_c, int32_t max_sweeps, hjb_stats* stats) {
    g_last_error.clear();
    clear_stats(stats);
    if (!p) return fail(HJB_ERR_INVALID_ARG, "problem is NULL");
    if (p->nc == 0) return fail(HJB_ERR_STATE, "problem has no coarse grid");
    if (!(tol_c > 0.0) || max_sweeps < 1) return fail(HJB_ERR_INVALID_ARG, "bad tol_c / max_sweeps");
    Timer tm(p->st);
    tm.mark();
    const GridView gc = p->coarse_view();
    const int Nc = p->nc * p->nc;
    CU(launch_init_values(Nc, p->mask_c, (float)p->uob_c, (float)p->uob, p->uc, nullptr, p->uob, p->st));
    // one cooperative launch: in-place sweeps until the sup-increment is <= tol_c
    Scalars* ds = dscal(p);
    CU(cudaMemsetAsync(&ds->wave, 0, sizeof(WaveResult), p->st));
    CU(cudaMemsetAsync(&ds->sync, 0, sizeof(GridSync), p->st));
    CU(cudaMemsetAsync(ds->relax_inc, 0, sizeof(ds->relax_inc), p->st));
    CU(cudaMemsetAsync(ds->relax_umax, 0, sizeof(ds->relax_umax), p->st));
    RelaxArgs ra{};
    ra.g = gc;
    // FP32 floor: from the obstacle value with a discount; without one the
    // kernel takes it from the largest value of each sweep
    ra.tol = (float)(p->lambda > 0.0 ? std::max(tol_c, p->floor32(p->uob_c)) : tol_c);
    ra.floor_amp = (float)p->amp32;
    ra.max_sweeps = max_sweeps;
    ra.sweep_inc = ds->relax_inc;
    ra.sweep_umax = ds->relax_umax;
    ra.sync = &ds->sync;
    ra.res = &ds->wave;
    ra.timeout_ns = kTimeoutNs;
    ra.tw = p->relax_plan.tw;
    ra.th = p->relax_plan.th;
    ra.ntx = p->relax_plan.ntx;
    ra.halo = p->relax_plan.halo;
    ra.local_sweeps = kCoarseLocalSweeps;
    ra.pre = p->relax_plan.pre;
    CU(launch_grid_relax(ra, p->uc, false, p->relax_blocks, p->st));
    tm.mark();
    CU(cudaMemcpyAsync(&hscal(p)->wave, &ds->wave, sizeof(WaveResult), cudaMemcpyDeviceToHost, p->st));
    CU(cudaMemcpyAsync(&hscal(p)->sync, &ds->sync, sizeof(GridSync), cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    if (hscal(p)->sync.err != 0)
        return fail(hscal(p)->sync.err, "coarse solve: a grid-wide wait exceeded its limit");
    const int sweeps = hscal(p)->wave.passes;
    const double last = hscal(p)->wave.last_increment;
    const bool conv = hscal(p)->wave.converged != 0;
    CoarseResult cr;
    cr.sweeps = conv ? sweeps : -sweeps;
    cr.increment = (float)last;
    if (p->lambda <= 0.0) {
        // largest coarse value over free nodes (the value bound without a discount)
        std::vector<float> hu((size_t)Nc);
        std::vector<uint8_t> hmk((size_t)Nc);
        CU(cudaMemcpyAsync(hu.data(), p->uc, (size_t)Nc * sizeof(float), cudaMemcpyDeviceToHost, p->st));
        CU(cudaMemcpyAsync(hmk.data(), p->mask_c, (size_t)Nc, cudaMemcpyDeviceToHost, p->st));
        CU(cudaStreamSynchronize(p->st));
        double mx = 0.0;
        for (int k = 0; k < Nc; ++k)
            if (hmk[k] == HJB_MASK_FREE && std::isfinite(hu[k])) mx = std::max(mx, (double)hu[k]);
        p->uc_max = mx;
    }
    p->coarse_done = true;
    p->built = false;
    int rc = cr.sweeps > 0 ? HJB_OK : HJB_ERR_NOT_CONVERGED;
    if (stats) {
        stats->sweeps = cr.sweeps > 0 ? cr.sweeps : -cr.sweeps;
        stats->increment = cr.increment;
        stats->ms_total = tm.ms(0, 1);
        stats->ms_stage[0] = stats->ms_total;
        stats->node_updates = (long long)stats->sweeps * kCoarseLocalSweeps * (long long)p->nc * p->nc;
        stats->node_control_updates = stats->node_updates * p->na;
        stats->status = rc;
    }
    if (rc) fail(rc, "coarse solve did not reach tol_c in %d sweeps", max_sweeps);
    return rc;
}

namespace {

// The pre-computation that follows u_hat (Section 4.3): synthesis a* with the
// band keys, successors, labels, ordering, tiles, and the start value u = u_hat.
int precompute_from_uhat(hjb_problem* p, Timer& tm) {
    Scalars* ds = dscal(p);
    const GridView g = p->fine_view();
    CU(cudaMemsetAsync(&ds->max_key, 0, sizeof(int), p->st));
    CU(launch_synthesis(g, p->uhat, p->band_map(), p->a, p->key, &ds->max_key, p->st));
    CU(cudaMemcpyAsync(&hscal(p)->max_key, &ds->max_key, sizeof(int), cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    tm.mark();
    p->n_bands = hscal(p)->max_key + 1;
    int rc = rebuild_order(p);
    if (rc) return rc;
    rc = build_tiles(p, p->uhat);
    if (rc) return rc;
    tm.mark();
    // the fine iteration starts from u_hat
    CU(cudaMemcpyAsync(p->u32, p->uhat, sizeof(float) * p->N, cudaMemcpyDeviceToDevice, p->st));
    CU(launch_fix_nonfree(p->N, p->mask, (float)p->uob, p->uob, p->u32, nullptr, p->st));
    p->value_f64 = false;
    int32_t nfree = 0;
    CU(cudaMemcpyAsync(&nfree, p->band_off + p->n_bands, sizeof(int32_t), cudaMemcpyDeviceToHost, p->st));
    tm.mark();
    CU(cudaStreamSynchronize(p->st));
    p->n_free = nfree;
    p->built = true;
    return HJB_OK;
}

}  // namespace

int hjb_build_patches(hjb_problem* p, hjb_stats* stats) {
    g_last_error.clear();
    clear_stats(stats);
    if (!p) return fail(HJB_ERR_INVALID_ARG, "problem is NULL");
    if (!p->coarse_done) return fail(HJB_ERR_STATE, "hjb_coarse_solve has not run");
    Timer tm(p->st);
    tm.mark();
    CU(launch_interp(p->nc, p->uc, p->n, p->mask, (float)p->uob, p->uhat, p->st));
    tm.mark();
    const int rc = precompute_from_uhat(p, tm);
    if (rc) return rc;
    if (stats) {
        stats->ms_stage[0] = tm.ms(0, 1);
        stats->ms_stage[1] = tm.ms(1, 2);
        stats->ms_stage[3] = tm.ms(2, 3);
        stats->ms_total = tm.ms(0, 4);
        stats->sweeps = p->n_bands;
        stats->status = HJB_OK;
    }
    return HJB_OK;
}

int hjb_set_uhat(hjb_problem* p, const float* uhat) {
    g_last_error.clear();
    if (!p || !uhat) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!p->built) return fail(HJB_ERR_STATE, "hjb_build_patches has not run");
    std::vector<uint8_t> m(p->N);
    CU(cudaMemcpyAsync(m.data(), p->mask, p->N, cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    std::vector<float> v(uhat, uhat + p->N);
    for (int k = 0; k < p->N; ++k) {
        if (m[k] == HJB_MASK_FREE) {
            if (!std::isfinite(v[k])) return fail(HJB_ERR_INVALID_ARG, "uhat[%d] is not finite", k);
        } else {
            v[k] = m[k] == HJB_MASK_TARGET ? 0.0f : (float)p->uob;
        }
    }
    CU(cudaMemcpyAsync(p->uhat, v.data(), sizeof(float) * p->N, cudaMemcpyHostToDevice, p->st));
    Timer tm(p->st);
    tm.mark();
    return precompute_from_uhat(p, tm);
}

int hjb_set_feedback(hjb_problem* p, const uint8_t* a) {
    g_last_error.clear();
    if (!p || !a) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!p->built) return fail(HJB_ERR_STATE, "hjb_build_patches has not run");
    std::vector<uint8_t> m(p->N);
    CU(cudaMemcpyAsync(m.data(), p->mask, p->N, cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    std::vector<uint8_t> clean(a, a + p->N);
    for (int k = 0; k < p->N; ++k) {
        if (m[k] == HJB_MASK_FREE) {
            if (clean[k] >= p->na) return fail(HJB_ERR_INVALID_ARG, "a[%d]=%d >= n_controls", k, clean[k]);
        } else {
            clean[k] = 255;
        }
    }
    CU(cudaMemcpyAsync(p->a, clean.data(), p->N, cudaMemcpyHostToDevice, p->st));
    int rc = rebuild_order(p);
    if (rc) return rc;
    CU(cudaStreamSynchronize(p->st));
    return HJB_OK;
}

namespace {

// The FP64 stage by mixed-precision correction (iterative refinement): with the
// FP64 residual r = T2 u - u and its minimising control a per node (written by
// the last residual64(p, &res, true)), solve the linear correction equation
// e = beta P_a e + r in FP32 by Jacobi sweeps to a sup-increment of tol_in, add
// e to u in FP64 and take the FP64 residual again; each round is one policy
// evaluation of the linearised scheme, so the residual falls by orders of
// magnitude per round while every sweep is FP32 with one control per node.
// The rounds are Howard's policy iteration on the FP64 values: where the
// minimising control switches (sigma = 0, ties along shocks) a round can raise
// the residual, and the next round, with the new controls, brings it down.
// Stops at res <= tol64, after `rounds`, after two rounds in a row that fail
// to halve the residual, or when it grows past 1e3 times the stage's first
// one (the FP64 passes then take over).  *sweeps / *nodes count the correction
// sweeps and their node updates (one control each).
int correction_stage(hjb_problem* p, double tol64, int rounds, double* res, int* sweeps,
                     unsigned long long* nodes, int* n_res) {
    const GridView g = p->fine_view();
    const bool sig = p->sigma > 0.0;
    constexpr int kMaxSweeps = 20000;
    int rc = ensure_hist(p, kMaxSweeps + 8);
    if (rc) return rc;
    const double res0 = *res;
    int stalled = 0;
    for (int it = 0; it < rounds && *res > tol64; ++it) {
        const double before = *res;
        CU(cudaMemsetAsync(p->u32, 0, sizeof(float) * (size_t)p->N, p->st));
        int sw = 0;
        double last = 0.0;
        bool conv = false;
        // the correction is at most res / (1 - beta); its FP32 increments cannot
        // resolve much below 2^-21 of that, so the round stops there at the latest
        // (the next round starts from a residual that much smaller)
        const double tol_in = std::max(0.2 * tol64, std::ldexp(*res / (1.0 - p->beta), -21));
        rc = jacobi_loop_impl<float>(p, p->inc_hist32, p->u32, p->u32b, p->N, tol_in, kMaxSweeps, &sw,
                                     &last, &conv, [&](const float* a, float* b, unsigned int* inc) {
                                         return launch_correction_sweep(g, sig, p->halo, p->corr_a, p->corr_r,
                                                                        a, b, inc, p->st);
                                     });
        if (rc) return rc;
        *sweeps += sw;
        *nodes += (unsigned long long)sw * (unsigned long long)p->n_free;
        CU(launch_add_correction(p->N, p->mask, p->u32, p->u64, p->st));
        rc = residual64(p, res, true);
        if (rc) return rc;
        ++*n_res;
        stalled = *res < 0.5 * before ? 0 : stalled + 1;
        if (stalled >= 2 || !(*res <= 1e3 * res0)) break;
    }
    return HJB_OK;
}

}  // namespace

int hjb_solve_patches(hjb_problem* p, double tol32, double tol64, int32_t max_passes,
                      hjb_stats* stats) {
    g_last_error.clear();
    clear_stats(stats);
    if (!p) return fail(HJB_ERR_INVALID_ARG, "problem is NULL");
    if (!p->built) return fail(HJB_ERR_STATE, "hjb_build_patches has not run");
    if (!(tol32 > 0.0) || max_passes < 1 || !(tol64 >= 0.0))
        return fail(HJB_ERR_INVALID_ARG, "bad tolerances / max_passes");
    tol32 = std::max(tol32, p->floor32(p->value_bound()));
    Timer tm(p->st);
    tm.mark();
    WaveResult w32{}, w64{};
    int rc = HJB_OK;
    if (p->value_f64) {
        CU(launch_demote(p->N, p->u64, p->u32, p->st));
        p->value_f64 = false;
    }
    {
        // optional single passes followed by a re-sort by the current value
        int done = 0;
        unsigned long long nodes = 0;
        WaveResult w{};
        w.converged = 0;
        for (int r = 0; r < p->desc.resort_passes && done < max_passes && !w.converged; ++r) {
            rc = run_phase(p, false, tol32, 1, &w);
            if (rc) return rc;
            done += w.passes;
            nodes += w.nodes;
            if (!w.converged) {
                rc = resort_by_value(p);
                if (rc) return rc;
            }
        }
        if (!w.converged && done < max_passes) {
            rc = run_phase(p, false, tol32, max_passes - done, &w);
            if (rc) return rc;
            done += w.passes;
            nodes += w.nodes;
        }
        w32 = w;
        w32.passes = done;
        w32.nodes = nodes;
    }
    tm.mark();
    // Without an FP64 stage the FP32 phase must converge; with one, the FP64
    // residual decides (the FP32 phase may stop at its visit caps where FP32
    // rounding keeps a few tiles changing, and the FP64 stage resolves them).
    if (!w32.converged && !(tol64 > 0.0)) rc = HJB_ERR_NOT_CONVERGED;
    double res = -1.0;
    double ms_promote = 0.0, ms64 = 0.0, ms_warm32 = 0.0;
    unsigned long long nodes64 = 0;
    int passes64 = 0;
    int n_res = 0;
    double last = w32.last_increment;
    int corr_sweeps = 0;
    unsigned long long corr_nodes = 0;
    // the FP64 stage by correction: constant coefficients, a discount, scheme 3
    const bool corr = !p->gen && p->lambda > 0.0 && p->desc.scheme == 3;
    if (tol64 > 0.0 && rc == HJB_OK) {
        Timer t2(p->st);
        t2.mark();
        CU(launch_promote(p->N, p->u32, p->mask, p->uob, p->u64, p->st));
        p->value_f64 = true;
        int r2 = residual64(p, &res, corr);
        if (r2) return r2;
        ++n_res;
        t2.mark();
        ms_promote += t2.ms(0, 1);
        // The FP32 stop (sup-increment of the last visits) does not bound the
        // residual tightly.  If the FP64 residual misses tol64 but tol64 lies
        // well above what FP32 values can resolve (4 ulp of the largest value),
        // tighten the FP32 tolerance and continue in FP32 from the current
        // value (warm: every tile in the first two steps) before any FP64 pass.
        // The tightened tolerance stays at 8 ulp or more: nearer the rounding
        // noise of a converged FP32 field every tile would keep re-queueing.
        const double floor32 = std::ldexp(std::max(1.0, p->value_bound()), -22) * p->amp32;
        double tol_w = tol32;
        for (int tries = 0; tries < 2 && w32.converged && res > tol64 && tol64 >= floor32 &&
                            0.25 * tol_w >= 2.0 * floor32 && p->desc.schedule == 0 &&
                            w32.passes < max_passes; ++tries) {
            Timer tw(p->st);
            tw.mark();
            tol_w = 0.25 * tol_w;
            WaveResult ww{};
            r2 = run_phase(p, false, tol_w, max_passes - w32.passes, &ww, true);
            if (r2) return r2;
            w32.passes += ww.passes;
            w32.nodes += ww.nodes;
            last = ww.last_increment;
            tw.mark();
            CU(launch_promote(p->N, p->u32, p->mask, p->uob, p->u64, p->st));
            r2 = residual64(p, &res, corr);
            if (r2) return r2;
            ++n_res;
            tw.mark();
            ms_warm32 += tw.ms(0, 1);
            ms_promote += tw.ms(1, 2);
        }
        if (corr && res > tol64) {
            Timer tc(p->st);
            tc.mark();
            r2 = correction_stage(p, tol64, 12, &res, &corr_sweeps, &corr_nodes, &n_res);
            if (r2) return r2;
            tc.mark();
            ms64 += tc.ms(0, 1);
        }
        double tol_pass = tol64;
        while (res > tol64 && passes64 < max_passes) {
            Timer t3(p->st);
            t3.mark();
            r2 = run_phase(p, true, tol_pass, max_passes - passes64, &w64);
            if (r2) return r2;
            t3.mark();
            passes64 += w64.passes;
            nodes64 += w64.nodes;
            last = w64.last_increment;
            r2 = residual64(p, &res);
            if (r2) return r2;
            ++n_res;
            t3.mark();
            ms64 += t3.ms(0, 1);
            ms_promote += t3.ms(1, 2);
            tol_pass *= 0.25;
        }
        if (res > tol64) rc = HJB_ERR_NOT_CONVERGED;
    }
    if (stats) {
        stats->fp32_passes = w32.passes;
        stats->fp64_passes = passes64;
        stats->sweeps = w32.passes + passes64;
        stats->node_updates = (long long)(w32.nodes + nodes64 + corr_nodes);
        // a correction sweep evaluates one control per node
        stats->node_control_updates = (long long)(w32.nodes + nodes64) * p->na + (long long)corr_nodes;
        stats->corr_sweeps = corr_sweeps;
        stats->fp64_node_updates = (long long)nodes64;
        stats->residual_evals = n_res;
        stats->residual = res;
        stats->increment = last;
        stats->ms_stage[0] = tm.ms(0, 1) + ms_warm32;
        stats->ms_stage[1] = ms_promote;
        stats->ms_stage[2] = ms64;
        stats->ms_total = stats->ms_stage[0] + ms_promote + ms64;
        stats->status = rc;
    }
    if (rc) fail(rc, "patch solve did not converge (FP32 passes %d, FP64 passes %d, residual %.3e)",
                 w32.passes, passes64, res);
    return rc;
}

int hjb_solve_full(hjb_problem* p, int32_t precision, double tol, double tol64, int32_t max_sweeps,
                   hjb_stats* stats) {
    g_last_error.clear();
    clear_stats(stats);
    if (!p) return fail(HJB_ERR_INVALID_ARG, "problem is NULL");
    if ((precision != 32 && precision != 64) || !(tol > 0.0) || max_sweeps < 1 || !(tol64 >= 0.0))
        return fail(HJB_ERR_INVALID_ARG, "bad precision / tolerance / max_sweeps");
    Timer tm(p->st);
    int rc = HJB_OK;
    int s32 = 0, s64 = 0;
    double last = -1.0, res = -1.0;
    bool conv = false;
    tm.mark();
    if (precision == 32) {
        CU(launch_init_values(p->N, p->mask, 0.0f, (float)p->uob, p->u32, nullptr, p->uob, p->st));
        CU(launch_init_values(p->N, p->mask, 0.0f, (float)p->uob, p->u32b, nullptr, p->uob, p->st));
        rc = jacobi32(p, p->fine_view(), p->halo, p->u32, p->u32b, std::max(tol, p->floor32(p->value_bound())),
                      max_sweeps, &s32, &last, &conv);
        if (rc) return rc;
        p->value_f64 = false;
        if (!conv) rc = HJB_ERR_NOT_CONVERGED;
    }
    tm.mark();
    if (precision == 64 || (tol64 > 0.0 && rc == HJB_OK)) {
        bool need = true;
        if (precision == 64) {
            CU(launch_init_values(p->N, p->mask, 0.0f, (float)p->uob, nullptr, p->u64, p->uob, p->st));
        } else {
            // FP64 sweeps only if the FP32 result misses the FP64 residual tolerance
            CU(launch_promote(p->N, p->u32, p->mask, p->uob, p->u64, p->st));
            int r2 = residual64(p, &res);
            if (r2) return r2;
            p->value_f64 = true;
            need = res > tol64;
        }
        if (need) {
            CU(cudaMemcpyAsync(p->u64b, p->u64, sizeof(double) * p->N, cudaMemcpyDeviceToDevice, p->st));
            const double t = precision == 64 ? tol : tol64;
            int r2 = jacobi64(p, p->u64, p->u64b, t, max_sweeps, &s64, &last, &conv);
            if (r2) return r2;
            p->value_f64 = true;
            rc = conv ? HJB_OK : HJB_ERR_NOT_CONVERGED;
            r2 = residual64(p, &res);
            if (r2) return r2;
        }
    }
    tm.mark();
    CU(cudaStreamSynchronize(p->st));
    if (stats) {
        stats->fp32_passes = s32;
        stats->fp64_passes = s64;
        stats->sweeps = s32 + s64;
        stats->node_updates = (long long)(s32 + s64) * p->n_free_total;
        stats->node_control_updates = stats->node_updates * p->na;
        stats->fp64_node_updates = (long long)s64 * p->n_free_total;
        stats->residual_evals = (precision == 32 && tol64 > 0.0 ? 1 : 0) + (s64 > 0 ? 1 : 0);
        stats->residual = res;
        stats->increment = last;
        stats->ms_stage[0] = tm.ms(0, 1);
        stats->ms_stage[1] = tm.ms(1, 2);
        stats->ms_total = tm.ms(0, 2);
        stats->status = rc;
    }
    if (rc) fail(rc, "full-grid iteration did not converge in %d sweeps", max_sweeps);
    return rc;
}

int hjb_apply_operator(hjb_problem* p, int32_t precision, int32_t scheme, const double* u,
                       double* out, int32_t* argmin) {
    g_last_error.clear();
    if (!p || !u || !out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if ((precision != 32 && precision != 64) || (scheme != 2 && scheme != 3))
        return fail(HJB_ERR_INVALID_ARG, "precision must be 32/64 and scheme 2/3");
    const size_t N = p->N;
    DevBuf d_arg, din, dout;
    if (argmin) CU(d_arg.alloc(N * sizeof(int32_t)));
    Scalars* ds = dscal(p);
    const GridView g = p->fine_view();
    const bool sig = p->sigma > 0.0;
    if (precision == 64) {
        CU(din.alloc(N * sizeof(double)));
        CU(dout.alloc(N * sizeof(double)));
        CU(cudaMemcpyAsync(din.ptr, u, N * sizeof(double), cudaMemcpyHostToDevice, p->st));
        CU(launch_sweep_f64(g, sig, scheme, p->halo, (const double*)din.ptr, (double*)dout.ptr,
                            (int32_t*)d_arg.ptr, &ds->inc64, p->st));
        CU(cudaMemcpyAsync(out, dout.ptr, N * sizeof(double), cudaMemcpyDeviceToHost, p->st));
        CU(cudaStreamSynchronize(p->st));
    } else {
        std::vector<float> h32(N);
        for (size_t k = 0; k < N; ++k) h32[k] = (float)u[k];
        CU(din.alloc(N * sizeof(float)));
        CU(dout.alloc(N * sizeof(float)));
        CU(cudaMemcpyAsync(din.ptr, h32.data(), N * sizeof(float), cudaMemcpyHostToDevice, p->st));
        CU(launch_sweep_f32(g, sig, scheme, p->halo, (const float*)din.ptr, (float*)dout.ptr,
                            (int32_t*)d_arg.ptr, &ds->inc32, p->st));
        CU(cudaMemcpyAsync(h32.data(), dout.ptr, N * sizeof(float), cudaMemcpyDeviceToHost, p->st));
        CU(cudaStreamSynchronize(p->st));
        for (size_t k = 0; k < N; ++k) out[k] = (double)h32[k];
    }
    if (argmin) {
        CU(cudaMemcpyAsync(argmin, d_arg.ptr, N * sizeof(int32_t), cudaMemcpyDeviceToHost, p->st));
        CU(cudaStreamSynchronize(p->st));
    }
    return HJB_OK;
}

int hjb_residual(hjb_problem* p, double* residual) {
    g_last_error.clear();
    if (!p || !residual) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!p->value_f64) {
        CU(launch_promote(p->N, p->u32, p->mask, p->uob, p->u64, p->st));
    }
    return residual64(p, residual);
}

int hjb_set_value(hjb_problem* p, const double* u) {
    g_last_error.clear();
    if (!p || !u) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    for (int k = 0; k < p->N; ++k)
        if (!std::isfinite(u[k])) return fail(HJB_ERR_INVALID_ARG, "u[%d] not finite", k);
    std::vector<float> h32(p->N);
    for (int k = 0; k < p->N; ++k) h32[k] = (float)u[k];
    CU(cudaMemcpyAsync(p->u64, u, sizeof(double) * p->N, cudaMemcpyHostToDevice, p->st));
    CU(cudaMemcpyAsync(p->u32, h32.data(), sizeof(float) * p->N, cudaMemcpyHostToDevice, p->st));
    CU(launch_fix_nonfree(p->N, p->mask, (float)p->uob, p->uob, p->u32, p->u64, p->st));
    CU(cudaStreamSynchronize(p->st));
    p->value_f64 = false;
    return HJB_OK;
}

int hjb_get_value(hjb_problem* p, double* u_out) {
    g_last_error.clear();
    if (!p || !u_out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (p->value_f64) {
        CU(cudaMemcpyAsync(u_out, p->u64, sizeof(double) * p->N, cudaMemcpyDeviceToHost, p->st));
        CU(cudaStreamSynchronize(p->st));
    } else {
        std::vector<float> h(p->N);
        CU(cudaMemcpyAsync(h.data(), p->u32, sizeof(float) * p->N, cudaMemcpyDeviceToHost, p->st));
        CU(cudaStreamSynchronize(p->st));
        for (int k = 0; k < p->N; ++k) u_out[k] = (double)h[k];
    }
    return HJB_OK;
}

int hjb_get_coarse_value(hjb_problem* p, double* uc_out) {
    g_last_error.clear();
    if (!p || !uc_out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!p->coarse_done) return fail(HJB_ERR_STATE, "hjb_coarse_solve has not run");
    std::vector<float> h((size_t)p->nc * p->nc);
    CU(cudaMemcpyAsync(h.data(), p->uc, sizeof(float) * h.size(), cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    for (size_t k = 0; k < h.size(); ++k) uc_out[k] = (double)h[k];
    return HJB_OK;
}

int hjb_get_uhat(hjb_problem* p, double* uhat_out) {
    g_last_error.clear();
    if (!p || !uhat_out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!p->built) return fail(HJB_ERR_STATE, "hjb_build_patches has not run");
    std::vector<float> h(p->N);
    CU(cudaMemcpyAsync(h.data(), p->uhat, sizeof(float) * p->N, cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    for (int k = 0; k < p->N; ++k) uhat_out[k] = (double)h[k];
    return HJB_OK;
}

int hjb_get_feedback(hjb_problem* p, uint8_t* a_out) {
    g_last_error.clear();
    if (!p || !a_out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!p->built) return fail(HJB_ERR_STATE, "hjb_build_patches has not run");
    CU(cudaMemcpyAsync(a_out, p->a, p->N, cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    return HJB_OK;
}

int hjb_get_successors(hjb_problem* p, int32_t* succ_out) {
    g_last_error.clear();
    if (!p || !succ_out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!p->built) return fail(HJB_ERR_STATE, "hjb_build_patches has not run");
    CU(cudaMemcpyAsync(succ_out, p->succ, sizeof(int32_t) * p->N, cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    return HJB_OK;
}

int hjb_get_labels(hjb_problem* p, int8_t* label_out) {
    g_last_error.clear();
    if (!p || !label_out) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!p->built) return fail(HJB_ERR_STATE, "hjb_build_patches has not run");
    CU(cudaMemcpyAsync(label_out, p->label, p->N, cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    return HJB_OK;
}

int hjb_get_order(hjb_problem* p, int32_t* keys_out, int32_t* order_out, int32_t* band_off_out,
                  int32_t* n_free, int32_t* n_bands) {
    g_last_error.clear();
    if (!p) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (!p->built) return fail(HJB_ERR_STATE, "hjb_build_patches has not run");
    if (keys_out) CU(cudaMemcpyAsync(keys_out, p->key, sizeof(int32_t) * p->N, cudaMemcpyDeviceToHost, p->st));
    if (order_out) CU(cudaMemcpyAsync(order_out, p->order, sizeof(int32_t) * p->n_free, cudaMemcpyDeviceToHost, p->st));
    if (band_off_out)
        CU(cudaMemcpyAsync(band_off_out, p->band_off, sizeof(int32_t) * (p->n_bands + 1), cudaMemcpyDeviceToHost, p->st));
    CU(cudaStreamSynchronize(p->st));
    if (n_free) *n_free = p->n_free;
    if (n_bands) *n_bands = p->n_bands;
    return HJB_OK;
}

int hjb_device_info(hjb_problem* p, int32_t* num_sms, int32_t* wave_blocks32, int32_t* wave_blocks64) {
    if (!p) return fail(HJB_ERR_INVALID_ARG, "NULL argument");
    if (num_sms) *num_sms = p->num_sms;
    if (wave_blocks32) *wave_blocks32 = p->wave_blocks32;
    if (wave_blocks64) *wave_blocks64 = p->wave_blocks64;
    return HJB_OK;
}

}  // extern "C"
