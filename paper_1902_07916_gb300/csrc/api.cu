// The C ABI of include/zmc.h: handles, argument checks, device buffers, the
// per-level launch sequence (captured once into a CUDA graph and replayed),
// tracing, and the single host <-> device crossing of a run.
#include <ctype.h>
#include <cuda_runtime.h>
#include <math.h>
#include <nvtx3/nvToolsExt.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <tuple>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "jit.h"
#include "zmc_internal.h"

using namespace zmc;

namespace {
// The sampling kernel of a registry integrand fn (0 .. kNumIntegrands - 1)
// in mode MODE at dimension d, from the part that holds it.
template <int MODE>
const void* registry_kernel(int fn, int d, bool batched) {
    switch (fn >> 1) {
    case 0: return batched ? batch_kernel_part<MODE, 0>(fn, d) : eval_kernel_part<MODE, 0>(fn, d);
    case 1: return batched ? batch_kernel_part<MODE, 1>(fn, d) : eval_kernel_part<MODE, 1>(fn, d);
    case 2: return batched ? batch_kernel_part<MODE, 2>(fn, d) : eval_kernel_part<MODE, 2>(fn, d);
    case 3: return batched ? batch_kernel_part<MODE, 3>(fn, d) : eval_kernel_part<MODE, 3>(fn, d);
    default: return nullptr;
    }
}
static_assert(kNumIntegrands == 2 * kKernelParts, "one part per pair of registry integrands");

const void* registry_kernel(int mode, int fn, int d, bool batched) {
    if (fn < 0 || fn >= kNumIntegrands) return nullptr;
    switch (mode) {
    case ZMC_FP64: return registry_kernel<ZMC_FP64>(fn, d, batched);
    case ZMC_FP32_FP64ACC: return registry_kernel<ZMC_FP32_FP64ACC>(fn, d, batched);
    default: return registry_kernel<ZMC_FP32_KAHAN>(fn, d, batched);
    }
}
}  // namespace

struct TraceLevel {
    int64_t cells = 0, flagged = 0;
    double stats4[4] = {0, 0, 0, 0};
    std::vector<double> sums, cell_stats;
    std::vector<uint32_t> parents_out;
};

struct zmc_ctx {
    // configuration (host)
    int dim = 0, k = 0, T = 0, depth = 0;
    int64_t n = 0;
    double m = 0.0;
    uint64_t seed = 0;
    std::vector<double> lo, hi;
    int integrand = -1;
    std::vector<double> params;
    std::string expr;
    int mode = ZMC_FP64;
    int64_t max_cells = int64_t(1) << 24;
    int64_t max_samples = int64_t(1) << 40;
    bool trace = false;
    std::vector<TraceLevel> trace_levels;
    std::string last_error;

    // device side
    int device = -1;
    int num_sms = 0;
    Buffers buf{};
    int64_t cap_cells = 0, cap_parents = 0;
    Desc* h_desc = nullptr;          // pinned staging of the descriptor
    zmc_result* h_result = nullptr;  // pinned landing zone of the result
    bool desc_dirty = true;
    JitKernel jit{};                 // expression integrand, if any
    int launch_threads = 0, launch_per_sm = 0;  // 0: autotuned
    int tuning = ZMC_TUNE_SHAPE;                // what the autotuner may choose
    bool plan_set = false;                      // zmc_set_work_plan fixed the plan
    WorkPlan plan = kDefaultPlan;               // the plan of the next / last run
    EvalShape shapes[ZMC_MAX_DEPTH + 1] = {};  // per level, set before capture
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph = nullptr;
    bool graph_stale = true;
    int64_t graph_kernels = 0;
    bool profiling = false;
    cudaEvent_t ev[ZMC_MAX_DEPTH + 1][2] = {};  // around each level's sampling kernel
};

namespace {

thread_local std::string g_error;

int fail(zmc_handle h, int code, const std::string& msg) {
    if (h) h->last_error = msg; else g_error = msg;
    return code;
}

int cuda_fail(zmc_handle h, cudaError_t e, const char* what) {
    std::string msg = std::string(what) + ": " + cudaGetErrorString(e);
    return fail(h, e == cudaErrorMemoryAllocation ? ZMC_ERR_OOM : ZMC_ERR_CUDA, msg);
}

// NVTX ranges (header-only NVTX3: without a profiler attached a push/pop is
// a check of one pointer) around the API calls, the graph capture, the
// launch-shape tuner and each level where the host sees levels (traced runs,
// the batched form's per-level graphs); in a graph replay the levels run on
// the device, timed by zmc_set_profiling's events instead.
class Range {
  public:
    explicit Range(const char* name) { nvtxRangePushA(name); }
    Range(const char* what, int level) {
        char buf[48];
        snprintf(buf, sizeof buf, "%s %d", what, level);
        nvtxRangePushA(buf);
    }
    ~Range() { nvtxRangePop(); }
    Range(const Range&) = delete;
    Range& operator=(const Range&) = delete;
};

bool fault_injected(const char* what) {
    const char* f = getenv("ZMC_FAULT");
    return f && strcmp(f, what) == 0;
}

// Saturating k^e in int64.
int64_t ipow_sat(int64_t k, int e, int64_t cap) {
    int64_t r = 1;
    for (int i = 0; i < e; ++i) {
        if (r > cap / k) return cap;
        r *= k;
    }
    return r;
}

struct RegistryEntry {
    const char* name;
    int id;
};
const RegistryEntry kRegistry[] = {
    {"constant", kConstant},       {"linear", kLinear},
    {"sin_sum", kSinSum},          {"gauss_norm", kGaussNorm},
    {"genz_osc", kGenzOsc},        {"genz_prodpeak", kGenzProdPeak},
    {"genz_gauss", kGenzGauss},    {"genz_corner", kGenzCorner},
};

int expected_params(int id, int d) {
    switch (id) {
    case kConstant: return 1;
    case kLinear: return 1 + d;
    case kSinSum: return 0;
    case kGaussNorm: return 1;
    case kGenzOsc: return 1 + d;
    case kGenzProdPeak: return 2 * d;
    case kGenzGauss: return 2 * d;
    case kGenzCorner: return d;
    default: return -1;
    }
}

// Lay the user's parameters out as the kernels read them (pa_i, pb_i, c[]).
void fill_integrand(Desc& D, int id, const std::vector<double>& p) {
    const int d = D.d;
    for (int i = 0; i < ZMC_MAX_DIM; ++i) D.pa[i] = D.pb[i] = 0.0;
    for (int i = 0; i < 4; ++i) D.c[i] = 0.0;
    switch (id) {
    case kConstant: D.c[0] = p[0]; break;
    case kLinear:
        D.c[0] = p[0];
        for (int i = 0; i < d; ++i) D.pa[i] = p[1 + i];
        break;
    case kSinSum: break;
    case kGaussNorm: {
        const double s = p[0];
        D.c[0] = -1.0 / (2.0 * s * s);
        D.c[1] = pow(sqrt(2.0 * M_PI) * s, -(double)d);
        D.c[2] = D.c[0] * M_LOG2E;        // the FP32 modes' log2-domain exponent
        break;
    }
    case kGenzOsc:
        D.c[0] = 2.0 * M_PI * p[0];
        D.c[1] = p[0];                    // the phase in turns (FP32 modes)
        for (int i = 0; i < d; ++i) D.pa[i] = p[1 + i];
        break;
    case kGenzProdPeak:
        for (int i = 0; i < d; ++i) {
            D.pa[i] = p[d + i];                 // u_i
            D.pb[i] = 1.0 / (p[i] * p[i]);      // a_i^-2
        }
        break;
    case kGenzGauss:
        for (int i = 0; i < d; ++i) {
            D.pa[i] = p[i];                     // a_i
            D.pb[i] = p[d + i];                 // u_i
        }
        break;
    case kGenzCorner:
        for (int i = 0; i < d; ++i) D.pa[i] = p[i];
        break;
    default: break;
    }
}

// Capacity of the per-level buffers: the most cells any level can hold under
// the limits (level L has at most K^L cells).
int64_t capacity(const zmc_ctx* h) {
    const int64_t per_cell = h->n * (int64_t)h->T;
    int64_t cap = std::min(h->max_cells, h->max_samples / per_cell);
    const int64_t K = ipow_sat(h->k, h->dim, INT64_MAX);
    cap = std::min(cap, ipow_sat(K, h->depth, INT64_MAX));
    cap = std::min<int64_t>(cap, 0xFFFFFFFFll);
    return std::max(cap, K);
}

void free_device(zmc_ctx* h) {
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    if (h->cap_stream) cudaStreamDestroy(h->cap_stream);
    h->cap_stream = nullptr;
    for (auto& pair : h->ev)
        for (cudaEvent_t& e : pair) {
            if (e) cudaEventDestroy(e);
            e = nullptr;
        }
    Buffers& b = h->buf;
    void* ptrs[] = {b.desc, b.state, b.sums, b.cell_stats, b.parents[0], b.parents[1],
                    b.part_stats, b.part_count, b.part_offset, b.part_margin, b.part_acc,
                    b.result};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    b = Buffers{};
    if (h->h_desc) cudaFreeHost(h->h_desc);
    if (h->h_result) cudaFreeHost(h->h_result);
    h->h_desc = nullptr;
    h->h_result = nullptr;
    h->cap_cells = h->cap_parents = 0;
}

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (dev >= 0 && dev != prev_) cudaSetDevice(dev);
    }
    ~DeviceGuard() { cudaSetDevice(prev_); }
  private:
    int prev_ = 0;
};

// Allocate (or re-size) the device buffers for the current limits.
int ensure_device(zmc_ctx* h) {
    if (h->device < 0) {
        cudaError_t e = cudaGetDevice(&h->device);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGetDevice");
        e = cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaDeviceGetAttribute");
    }
    const int64_t cap = capacity(h);
    const int64_t K = ipow_sat(h->k, h->dim, INT64_MAX);
    const int64_t cap_par = cap / K + 1;
    if (h->buf.desc && cap == h->cap_cells && cap_par == h->cap_parents) return ZMC_OK;
    free_device(h);
    if (fault_injected("alloc")) return fail(h, ZMC_ERR_OOM, "injected allocation failure");
    Buffers& b = h->buf;
    struct Req { void** p; size_t bytes; };
    const Req reqs[] = {
        {(void**)&b.desc, sizeof(Desc)},
        {(void**)&b.state, sizeof(State)},
        // partial sums of the sampling kernel's units: a level with `tiles`
        // tiles has at most tiles + kTargetUnits unit slots (see unit_chunks;
        // a lane-tile unit writes one slot per tile)
        {(void**)&b.sums, sizeof(double2) * ((size_t)cap * h->T + (size_t)kTargetUnits)},
        {(void**)&b.cell_stats, sizeof(double2) * (size_t)cap},
        {(void**)&b.parents[0], sizeof(uint32_t) * (size_t)cap_par * h->dim},
        {(void**)&b.parents[1], sizeof(uint32_t) * (size_t)cap_par * h->dim},
        {(void**)&b.part_stats, sizeof(double) * 3 * kSelGrid},
        {(void**)&b.part_count, sizeof(int64_t) * kSelGrid},
        {(void**)&b.part_offset, sizeof(int64_t) * kSelGrid},
        {(void**)&b.part_margin, sizeof(double) * kSelGrid},
        {(void**)&b.part_acc, sizeof(double) * kPartAccDoubles},
        {(void**)&b.result, sizeof(zmc_result)},
    };
    for (const Req& r : reqs) {
        cudaError_t e = cudaMalloc(r.p, r.bytes);
        if (e != cudaSuccess) {
            free_device(h);
            return cuda_fail(h, e, "cudaMalloc of the level buffers");
        }
    }
    cudaError_t e = cudaMemset(b.part_acc, 0, sizeof(double) * kPartAccDoubles);
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_desc, sizeof(Desc));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&h->h_result, sizeof(zmc_result));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        free_device(h);
        return cuda_fail(h, e, "device set-up");
    }
    h->cap_cells = cap;
    h->cap_parents = cap_par;
    h->desc_dirty = true;
    h->graph_stale = true;
    return ZMC_OK;
}

void build_desc(const zmc_ctx* h, Desc& D) {
    memset(&D, 0, sizeof D);
    D.d = h->dim; D.k = h->k; D.T = h->T; D.depth = h->depth;
    D.integrand = h->integrand; D.mode = h->mode;
    D.n = h->n;
    D.K = ipow_sat(h->k, h->dim, INT64_MAX);
    for (int i = 0; i < h->dim; ++i) D.kpow[i] = ipow_sat(h->k, i, INT64_MAX);
    D.key[0] = (uint32_t)(h->seed & 0xFFFFFFFFu);
    D.key[1] = (uint32_t)(h->seed >> 32);
    D.m = h->m;
    D.max_cells = h->max_cells;
    D.max_samples = h->max_samples;
    D.cap_cells = h->cap_cells;
    // ZMC_FAULT=capacity (a test of the bounds-guarded build): the kernels
    // are told half of level 1's size as the capacity while the buffers keep
    // their real size, so the guards fire on in-bounds memory
    if (fault_injected("capacity")) D.cap_cells = std::max<int64_t>(1, D.K / 2);
    D.plan = h->plan;
    for (int i = 0; i < h->dim; ++i) D.lo[i] = h->lo[i];
    for (int L = 1; L <= h->depth; ++L) {
        const double kL = (double)ipow_sat(h->k, L, INT64_MAX);   // exact below 2^53
        double vol = 1.0;
        for (int i = 0; i < h->dim; ++i) {
            D.width[L][i] = (h->hi[i] - h->lo[i]) / kL;
            vol *= D.width[L][i];
        }
        D.volume[L] = vol;
    }
    if (h->integrand >= 0 && h->integrand < kNumIntegrands)
        fill_integrand(D, h->integrand, h->params);
    if (h->integrand == kExpression) {
        // expression parameters are read straight from pa/pb/c in order
        for (size_t j = 0; j < h->params.size(); ++j) {
            if (j < ZMC_MAX_DIM) D.pa[j] = h->params[j];
            else if (j < 2 * ZMC_MAX_DIM) D.pb[j - ZMC_MAX_DIM] = h->params[j];
            else D.c[j - 2 * ZMC_MAX_DIM] = h->params[j];
        }
    }
}

const void* batch_kernel(int mode, int fn, int d) { return registry_kernel(mode, fn, d, true); }

const void* eval_kernel(const zmc_ctx* h) {
    if (h->integrand == kExpression) return h->jit.kernel;
    return registry_kernel(h->mode, h->integrand, h->dim, false);
}

// ------------------------------------------------------------ autotuner
// The sampling kernel's results do not depend on its launch shape (the work
// units and their order of summation depend only on the level's size, n and
// the precision), so the shape is free to tune.  Candidates: 128 or 256
// threads per CTA, and from the occupancy limit down to half of it CTAs per
// SM.  Each is timed once on a truncated level 1 of the caller's own
// problem (about 2^29 points), the fastest is kept per (kernel, dimension)
// for the life of the process (and, with ZMC_TUNE_CACHE, in a file; see
// below).  ZMC_TUNE=0 in the environment, or an explicit zmc_set_launch(),
// skips it.
struct Tuned {
    int threads, per_sm;
};
std::mutex g_tune_mu;
std::map<std::pair<const void*, int>, Tuned> g_tuned;

#ifndef ZMC_BUILD_ID
#define ZMC_BUILD_ID 0ULL   // the build passes a hash of the library's sources
#endif

// ------------------------------------------------- persisted tuner cache
// With ZMC_TUNE_CACHE=<path> in the environment the tuner's choices are also
// kept in that file, one JSON object per line, appended as they are made, so
// that a later process running the same build of the library on the same
// kind of GPU skips the timing runs.  A line's key names the device (name,
// SM count, compute capability), the build (a hash of the library's
// sources), the kernel (precision mode and registry integrand, or a hash of
// the expression) and the problem's shape.  Lines that do not parse, or whose
// values a setter would reject, are ignored; a file that cannot be read or
// written is not an error.  Without the variable nothing is read or written.
bool plan_ok(const WorkPlan& w) {
    return w.target_units >= 1 && w.target_units <= kTargetUnits && w.min_unit_groups >= 1 &&
           w.lane_tile_groups >= 0 && w.lane_tile_max_groups >= 0 &&
           w.lane_tile_min_tiles >= 1;
}

struct DiskCache {
    std::string path;                          // the file loaded ("" before any)
    std::map<std::string, Tuned> shapes;       // by shape_key
    std::map<std::string, WorkPlan> plans;     // by plan_key
    std::map<int, std::string> device_tags;    // by device ordinal
};
DiskCache g_disk;   // guarded by g_tune_mu

const char* tune_cache_path() {
    const char* p = getenv("ZMC_TUNE_CACHE");
    return (p && *p) ? p : nullptr;
}

uint64_t fnv1a64(const std::string& text) {
    uint64_t x = 0xcbf29ce484222325ULL;
    for (unsigned char c : text) x = (x ^ c) * 0x100000001b3ULL;
    return x;
}

// Caller holds g_tune_mu.
const std::string& device_tag_locked(int device) {
    auto it = g_disk.device_tags.find(device);
    if (it != g_disk.device_tags.end()) return it->second;
    std::string tag = "unknown";
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, device) == cudaSuccess) {
        std::string name = prop.name;
        for (char& c : name)
            if (!isalnum((unsigned char)c)) c = '_';
        char buf[384];
        snprintf(buf, sizeof buf, "%s/sm%d/cc%d.%d/build%016llx", name.c_str(),
                 prop.multiProcessorCount, prop.major, prop.minor,
                 (unsigned long long)ZMC_BUILD_ID);
        tag = buf;
    } else {
        cudaGetLastError();
    }
    return g_disk.device_tags[device] = tag;
}

std::string kernel_tag(const zmc_ctx* h) {
    char buf[96];
    if (h->integrand == kExpression)
        snprintf(buf, sizeof buf, "expr/m%d/p%zu/%016llx", h->mode, h->params.size(),
                 (unsigned long long)fnv1a64(h->expr));
    else
        snprintf(buf, sizeof buf, "reg/m%d/f%d", h->mode, h->integrand);
    return buf;
}

std::string shape_key(const std::string& dev, const std::string& ker, int d) {
    return dev + " " + ker + " d" + std::to_string(d);
}
std::string plan_key(const std::string& dev, const std::string& ker, int d, long long n,
                     long long tiles) {
    return shape_key(dev, ker, d) + " n" + std::to_string(n) + " t" + std::to_string(tiles);
}

static_assert(ZMC_PLAN_FIELDS == 5, "the cache's plan lines hold five fields");
constexpr const char* kShapeLine =
    "{\"kind\": \"shape\", \"device\": \"%s\", \"kernel\": \"%s\", \"d\": %d, "
    "\"threads\": %d, \"per_sm\": %d}\n";
constexpr const char* kPlanLine =
    "{\"kind\": \"plan\", \"device\": \"%s\", \"kernel\": \"%s\", \"d\": %d, "
    "\"n\": %lld, \"tiles\": %lld, \"plan\": [%lld, %lld, %lld, %lld, %lld]}\n";

// Caller holds g_tune_mu.  Reads the file once per path.
void disk_load_locked(const char* path) {
    if (g_disk.path == path) return;
    g_disk.path = path;
    g_disk.shapes.clear();
    g_disk.plans.clear();
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[1024];
    while (fgets(line, sizeof line, f)) {
        char dev[320], ker[96];
        int d = 0, threads = 0, per_sm = 0;
        long long n = 0, tiles = 0, p[ZMC_PLAN_FIELDS];
        if (sscanf(line,
                   " {\"kind\": \"shape\", \"device\": \"%319[^\"]\", \"kernel\": "
                   "\"%95[^\"]\", \"d\": %d, \"threads\": %d, \"per_sm\": %d}",
                   dev, ker, &d, &threads, &per_sm) == 5) {
            if ((threads == 64 || threads == 128 || threads == 256) && per_sm >= 1)
                g_disk.shapes[shape_key(dev, ker, d)] = Tuned{threads, per_sm};
        } else if (sscanf(line,
                          " {\"kind\": \"plan\", \"device\": \"%319[^\"]\", \"kernel\": "
                          "\"%95[^\"]\", \"d\": %d, \"n\": %lld, \"tiles\": %lld, "
                          "\"plan\": [%lld, %lld, %lld, %lld, %lld]}",
                          dev, ker, &d, &n, &tiles, &p[0], &p[1], &p[2], &p[3], &p[4]) == 10) {
            const WorkPlan w{p[0], p[1], p[2], p[3], p[4]};
            if (plan_ok(w)) g_disk.plans[plan_key(dev, ker, d, n, tiles)] = w;
        }
    }
    fclose(f);
}

void disk_append(const char* path, const char* line) {
    FILE* f = fopen(path, "a");
    if (!f) return;
    fputs(line, f);
    fclose(f);
}

int occupancy(const void* kernel, int threads) {
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
    return std::max(per_sm, 1);
}

Tuned default_shape(const zmc_ctx* h) {
    return Tuned{256, occupancy(eval_kernel(h), 256)};
}

float time_level1(zmc_ctx* h, Tuned c, int64_t cells, cudaEvent_t e0, cudaEvent_t e1) {
    cudaStream_t s = h->cap_stream;
    const Buffers& b = h->buf;
    const PhiloxKeys keys = philox_keys(h->seed);
    const uint32_t* parents = b.parents[1];
    int level = 1;
    void* args[] = {(void*)&b.desc, (void*)&b.state, (void*)&parents, (void*)&b.sums,
                    (void*)&level, (void*)&keys};
    if (launch_init(b, cells, s) != cudaSuccess) return -1.f;
    cudaEventRecord(e0, s);
    if (cudaLaunchKernel(eval_kernel(h), dim3(c.per_sm * h->num_sms), dim3(c.threads), args, 0,
                         s) != cudaSuccess)
        return -1.f;
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return -1.f;
    float ms = -1.f;
    cudaEventElapsedTime(&ms, e0, e1);
    return ms;
}

Tuned tuned_shape(zmc_ctx* h, cudaStream_t s) {
    Range range("zmc launch-shape tuner");
    if (h->launch_threads > 0) {
        const int occ = occupancy(eval_kernel(h), h->launch_threads);
        const int per_sm = h->launch_per_sm > 0 ? std::min(h->launch_per_sm, occ) : occ;
        return Tuned{h->launch_threads, per_sm};
    }
    const char* env = getenv("ZMC_TUNE");
    if ((env && strcmp(env, "0") == 0) || !(h->tuning & ZMC_TUNE_SHAPE)) return default_shape(h);
    const std::pair<const void*, int> key(eval_kernel(h), h->dim);
    const char* cache = tune_cache_path();
    std::string dev, ker = kernel_tag(h);
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned.find(key);
        if (it != g_tuned.end()) return it->second;
        if (cache) {
            dev = device_tag_locked(h->device);
            disk_load_locked(cache);
            auto jt = g_disk.shapes.find(shape_key(dev, ker, h->dim));
            if (jt != g_disk.shapes.end()) {
                Tuned t = jt->second;
                t.per_sm = std::min(t.per_sm, occupancy(eval_kernel(h), t.threads));
                g_tuned[key] = t;
                return t;
            }
        }
    }
    // Nothing may be timed while the caller's stream is being captured: the
    // default shape then (not cached, so a later uncaptured run tunes).
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return default_shape(h);
    }
    // The timing runs go on the handle's own stream after the caller's stream
    // has passed the descriptor upload (an event, not a device-wide sync, so
    // other streams of the process keep running); each candidate waits only
    // for its own end event.
    cudaEvent_t ready = nullptr;
    if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(ready, s) != cudaSuccess ||
        cudaStreamWaitEvent(h->cap_stream, ready, 0) != cudaSuccess) {
        if (ready) cudaEventDestroy(ready);
        cudaGetLastError();
        return default_shape(h);
    }
    cudaEventDestroy(ready);
    const int64_t K = ipow_sat(h->k, h->dim, INT64_MAX);
    const int64_t per_cell = h->n * (int64_t)h->T;
    const int64_t cells = std::max<int64_t>(1, std::min<int64_t>(K, (int64_t(1) << 29) / per_cell));
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return default_shape(h);
    }
    std::vector<Tuned> cands;
    for (int threads : {256, 128}) {
        const int occ = occupancy(eval_kernel(h), threads);
        for (int per_sm = occ; per_sm >= std::max(1, occ / 2); --per_sm)
            cands.push_back(Tuned{threads, per_sm});
    }
    Tuned best = cands.front();
    float best_ms = -1.f;
    time_level1(h, best, cells, e0, e1);   // warm-up
    for (const Tuned& c : cands) {
        const float ms = time_level1(h, c, cells, e0, e1);
        if (ms > 0.f && (best_ms < 0.f || ms < best_ms)) {
            best_ms = ms;
            best = c;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    std::lock_guard<std::mutex> lock(g_tune_mu);
    g_tuned[key] = best;
    if (cache) {
        g_disk.shapes[shape_key(dev, ker, h->dim)] = best;
        char line[640];
        snprintf(line, sizeof line, kShapeLine, dev.c_str(), ker.c_str(), h->dim, best.threads,
                 best.per_sm);
        disk_append(cache, line);
    }
    return best;
}

// ---------------------------------------------------- work-plan tuner
// With ZMC_TUNE_PLAN the tuner also chooses the work plan, which changes the
// order of summation (so the choice is recorded in every result): level 1 of
// the handle's own problem, whole, is timed under the tuned shape for
// lane_tile_min_tiles in {2^15, 2^16, 2^17, 2^18, never}, then, with the best
// of those, min_unit_groups in {256, 512, 1024, 2048, 4096}; a candidate
// replaces the current one only when at least 2% faster.  Levels of more
// than 2^31 points keep the default (there the plan's rules leave one unit
// per tile and no lane tiles anyway).  Cached per (kernel, dimension, n,
// level-1 tiles) for the process.
struct PlanKey {
    const void* kernel;
    int d;
    int64_t n, tiles;
    bool operator<(const PlanKey& o) const {
        return std::tie(kernel, d, n, tiles) < std::tie(o.kernel, o.d, o.n, o.tiles);
    }
};
std::map<PlanKey, WorkPlan> g_tuned_plan;
constexpr int64_t kPlanTuneMaxPoints = int64_t(1) << 31;

float time_plan(zmc_ctx* h, Tuned shape, const WorkPlan& plan, cudaEvent_t e0, cudaEvent_t e1) {
    const WorkPlan keep = h->plan;
    h->plan = plan;
    build_desc(h, *h->h_desc);
    h->plan = keep;
    cudaStream_t s = h->cap_stream;
    if (cudaMemcpyAsync(h->buf.desc, h->h_desc, sizeof(Desc), cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return -1.f;
    return time_level1(h, shape, ipow_sat(h->k, h->dim, INT64_MAX), e0, e1);
}

WorkPlan tuned_plan(zmc_ctx* h, Tuned shape, cudaStream_t s) {
    if (h->plan_set || !(h->tuning & ZMC_TUNE_PLAN) || h->integrand == kExpression)
        return h->plan_set ? h->plan : kDefaultPlan;
    const int64_t K = ipow_sat(h->k, h->dim, INT64_MAX);
    if (K > kPlanTuneMaxPoints / (h->n * (int64_t)h->T)) return kDefaultPlan;
    const PlanKey key{eval_kernel(h), h->dim, h->n, K * h->T};
    const char* cache = tune_cache_path();
    std::string dkey;
    {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        auto it = g_tuned_plan.find(key);
        if (it != g_tuned_plan.end()) return it->second;
        if (cache) {
            dkey = plan_key(device_tag_locked(h->device), kernel_tag(h), h->dim, h->n,
                            K * h->T);
            disk_load_locked(cache);
            auto jt = g_disk.plans.find(dkey);
            if (jt != g_disk.plans.end()) return g_tuned_plan[key] = jt->second;
        }
    }
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
        cudaGetLastError();
        return kDefaultPlan;
    }
    Range range("zmc work-plan tuner");
    // The candidates' descriptors are staged in the handle's pinned buffer,
    // which the caller's stream may still be copying from: wait (on the host)
    // until that stream has passed this call's own upload.
    cudaEvent_t ready = nullptr, e0 = nullptr, e1 = nullptr;
    const bool ok = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) == cudaSuccess &&
                    cudaEventRecord(ready, s) == cudaSuccess &&
                    cudaEventSynchronize(ready) == cudaSuccess &&
                    cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    WorkPlan best = kDefaultPlan;
    if (ok) {
        time_plan(h, shape, best, e0, e1);   // warm-up
        float best_ms = time_plan(h, shape, best, e0, e1);
        auto consider = [&](WorkPlan c) {
            const float ms = time_plan(h, shape, c, e0, e1);
            if (ms > 0.f && best_ms > 0.f && ms < 0.98f * best_ms) {
                best_ms = ms;
                best = c;
            }
        };
        for (int64_t t : {int64_t(1) << 15, int64_t(1) << 16, int64_t(1) << 17, INT64_MAX}) {
            WorkPlan c = best;
            c.lane_tile_min_tiles = t;
            consider(c);
        }
        const WorkPlan base = best;
        for (int64_t g : {256, 512, 2048, 4096}) {
            WorkPlan c = base;
            c.min_unit_groups = g;
            consider(c);
        }
    }
    for (cudaEvent_t e : {ready, e0, e1})
        if (e) cudaEventDestroy(e);
    cudaGetLastError();
    if (ok) {
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tuned_plan[key] = best;
        if (cache) {
            g_disk.plans[dkey] = best;
            char line[768];
            snprintf(line, sizeof line, kPlanLine, device_tag_locked(h->device).c_str(),
                     kernel_tag(h).c_str(), h->dim, (long long)h->n, (long long)(K * h->T),
                     (long long)best.target_units, (long long)best.min_unit_groups,
                     (long long)best.lane_tile_groups, (long long)best.lane_tile_max_groups,
                     (long long)best.lane_tile_min_tiles);
            disk_append(cache, line);
        }
    }
    return best;
}

EvalShape eval_shape(zmc_ctx* h, int level, Tuned t) {
    EvalShape sh;
    sh.threads = t.threads;
    int64_t grid = (int64_t)h->num_sms * t.per_sm;
    if (level == 1) {
        // no more CTAs than level 1 has units for their warps
        Desc D;
        build_desc(h, D);
        const int64_t units = level_plan(D, ipow_sat(h->k, h->dim, INT64_MAX)).units;
        grid = std::min(grid, (units + t.threads / 32 - 1) / (t.threads / 32));
    }
    sh.grid = (int)std::max<int64_t>(grid, 1);
    return sh;
}

int upload_desc(zmc_ctx* h, cudaStream_t s);

// Occupancy queries and tuning happen here, outside any stream capture.  If
// the tuner chose another work plan, the run's descriptor is uploaded again
// on the caller's stream (the tuner's own runs have finished by then).
int plan_shapes(zmc_ctx* h, cudaStream_t s) {
    const Tuned t = tuned_shape(h, s);
    const WorkPlan plan = tuned_plan(h, t, s);
    const bool changed = memcmp(&plan, &h->plan, sizeof plan) != 0;
    h->plan = plan;
    for (int L = 1; L <= h->depth; ++L) h->shapes[L] = eval_shape(h, L, t);
    if (changed || (h->tuning & ZMC_TUNE_PLAN)) return upload_desc(h, s);
    return ZMC_OK;
}

cudaError_t enqueue_eval(zmc_ctx* h, int level, const uint32_t* parents_prev, cudaStream_t s) {
    const EvalShape sh = h->shapes[level];
    const Buffers& b = h->buf;
    const PhiloxKeys keys = philox_keys(h->seed);
    void* args[] = {(void*)&b.desc, (void*)&b.state, (void*)&parents_prev, (void*)&b.sums,
                    (void*)&level, (void*)&keys};
    return cudaLaunchKernel(eval_kernel(h), dim3(sh.grid), dim3(sh.threads), args, 0, s);
}

// Every level, unconditionally: kernels of a level that has no cells return
// at once, so the host never needs to know how deep the tree went.
cudaError_t enqueue_levels(zmc_ctx* h, cudaStream_t s, int only_level = 0) {
    const Buffers& b = h->buf;
    cudaError_t e = cudaSuccess;
    const int first = only_level ? only_level : 1;
    const int last = only_level ? only_level : h->depth;
    if (first == 1) {
        e = launch_init(b, ipow_sat(h->k, h->dim, INT64_MAX), s);
        if (e != cudaSuccess) return e;
    }
    for (int L = first; L <= last; ++L) {
        const uint32_t* prev = b.parents[L & 1];       // written by level L-1
        uint32_t* next = b.parents[(L + 1) & 1];
        if (h->profiling && (e = cudaEventRecordWithFlags(h->ev[L][0], s, cudaEventRecordExternal)) != cudaSuccess) return e;
        e = enqueue_eval(h, L, prev, s);
        if (e != cudaSuccess) return e;
        if (h->profiling && (e = cudaEventRecordWithFlags(h->ev[L][1], s, cudaEventRecordExternal)) != cudaSuccess) return e;
        e = launch_select(b, L, prev, next, s);
        if (e != cudaSuccess) return e;
    }
    if (last == h->depth) e = launch_final(b, s);
    return e;
}

int upload_desc(zmc_ctx* h, cudaStream_t s) {
    build_desc(h, *h->h_desc);
    cudaError_t e = cudaMemcpyAsync(h->buf.desc, h->h_desc, sizeof(Desc),
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "descriptor upload");
    h->desc_dirty = false;
    return ZMC_OK;
}

int ensure_events(zmc_ctx* h) {
    if (!h->profiling) return ZMC_OK;
    for (int L = 1; L <= h->depth; ++L)
        for (cudaEvent_t& ev : h->ev[L])
            if (!ev) {
                cudaError_t e = cudaEventCreate(&ev);
                if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventCreate");
            }
    return ZMC_OK;
}

int ensure_graph(zmc_ctx* h, cudaStream_t s) {
    if (!h->graph_stale && h->graph) return ZMC_OK;
    Range range("zmc graph capture");
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->graph = nullptr;
    if (int rc = plan_shapes(h, s)) return rc;
    if (int rc = ensure_events(h)) return rc;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->cap_stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamBeginCapture");
    cudaError_t le = enqueue_levels(h, h->cap_stream);
    e = cudaStreamEndCapture(h->cap_stream, &g);
    if (le != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return cuda_fail(h, le, "kernel launch during capture");
    }
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaStreamEndCapture");
    size_t nn = 0;
    cudaGraphGetNodes(g, nullptr, &nn);
    std::vector<cudaGraphNode_t> nodes(nn);
    if (nn) cudaGraphGetNodes(g, nodes.data(), &nn);
    h->graph_kernels = 0;
    for (cudaGraphNode_t node : nodes) {
        cudaGraphNodeType t;
        if (cudaGraphNodeGetType(node, &t) == cudaSuccess && t == cudaGraphNodeTypeKernel)
            ++h->graph_kernels;
    }
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphInstantiate");
    h->graph_stale = false;
    return ZMC_OK;
}

int check_ready(zmc_ctx* h) {
    if (h->integrand < 0) return fail(h, ZMC_ERR_NOINTEGRAND, "zmc_set_integrand was not called");
    if (!eval_kernel(h))
        return fail(h, ZMC_ERR_ARG, "this build of the library has no sampling kernel for the "
                                    "integrand (the bounds-guarded build carries sin_sum and "
                                    "genz_corner only)");
    return ZMC_OK;
}

int finish_result(zmc_ctx* h, zmc_result* out) {
    *out = *h->h_result;
    memcpy(out->work_plan, &h->plan, sizeof out->work_plan);
    if (out->status == ZMC_ERR_CHECK) {
        State st;
        uint32_t site = 0;
        if (cudaMemcpy(&st, h->buf.state, sizeof st, cudaMemcpyDeviceToHost) == cudaSuccess)
            site = st.check_site;
        h->last_error = "bounds check failed (site " + std::to_string(site) +
                        "): an index was outside its buffer; the access was skipped";
        return out->status;
    }
    if (out->status != ZMC_OK) {
        h->last_error = out->status == ZMC_ERR_BUDGET
                            ? "refinement stopped by the cell / sample budget"
                            : "the integrand produced a non-finite value";
    }
    return out->status;
}

// Device tables and per-level graphs of the last batch, reused while the
// same handles (same buffers, precision and depth) come back.
// Integrals of a batch that share a sampling kernel (same integrand, dimension
// in 1..8 or 9..16): a contiguous range of the device table.
struct BatchGroup {
    const void* kernel;
    int start, count, grid;
};
constexpr int kMaxBatchGroups = 2 * kNumIntegrands;

struct BatchCache {
    int device = -1, capacity = 0;
    int count = 0, mode = -1, depth = 0;
    std::vector<Buffers> sel;
    std::vector<BatchEval> eval;
    std::vector<BatchGroup> groups;
    Desc* d_desc = nullptr;
    Desc* h_desc = nullptr;            // pinned
    Buffers* d_sel = nullptr;
    BatchEval* d_eval = nullptr;
    int64_t* d_l1 = nullptr;
    int64_t* d_offsets = nullptr;
    unsigned long long* d_head = nullptr;
    zmc_result* d_out = nullptr;
    zmc_result* h_out = nullptr;       // pinned
    cudaStream_t cap = nullptr;
    cudaStream_t side[kMaxBatchGroups] = {};     // branches of a level's graph
    cudaEvent_t fork = nullptr, join[kMaxBatchGroups] = {};
    std::vector<cudaGraphExec_t> graphs;

    void drop_graphs() {
        for (cudaGraphExec_t g : graphs) cudaGraphExecDestroy(g);
        graphs.clear();
        count = 0;
    }
    void release() {
        drop_graphs();
        void* dev_ptrs[] = {d_desc, d_sel, d_eval, d_l1, d_offsets, d_head, d_out};
        for (void* p : dev_ptrs)
            if (p) cudaFree(p);
        if (h_desc) cudaFreeHost(h_desc);
        if (h_out) cudaFreeHost(h_out);
        if (cap) cudaStreamDestroy(cap);
        for (int g = 0; g < kMaxBatchGroups; ++g) {
            if (side[g]) cudaStreamDestroy(side[g]);
            if (join[g]) cudaEventDestroy(join[g]);
        }
        if (fork) cudaEventDestroy(fork);
        *this = BatchCache{};
    }
    int reserve(int n, int dev) {
        if (dev == device && n <= capacity) return ZMC_OK;
        release();
        if (fault_injected("alloc")) return fail(nullptr, ZMC_ERR_OOM, "injected allocation failure");
        cudaError_t e = cudaMalloc(&d_desc, sizeof(Desc) * n);
        if (e == cudaSuccess) e = cudaMallocHost(&h_desc, sizeof(Desc) * n);
        if (e == cudaSuccess) e = cudaMalloc(&d_sel, sizeof(Buffers) * n);
        if (e == cudaSuccess) e = cudaMalloc(&d_eval, sizeof(BatchEval) * n);
        if (e == cudaSuccess) e = cudaMalloc(&d_l1, sizeof(int64_t) * n);
        if (e == cudaSuccess) e = cudaMalloc(&d_offsets, sizeof(int64_t) * (n + kMaxBatchGroups));
        if (e == cudaSuccess) e = cudaMalloc(&d_head, sizeof(unsigned long long) * kMaxBatchGroups);
        if (e == cudaSuccess) e = cudaMalloc(&d_out, sizeof(zmc_result) * n);
        if (e == cudaSuccess) e = cudaMallocHost(&h_out, sizeof(zmc_result) * n);
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking);
        for (int g = 0; e == cudaSuccess && g < kMaxBatchGroups; ++g) {
            e = cudaStreamCreateWithFlags(&side[g], cudaStreamNonBlocking);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&join[g], cudaEventDisableTiming);
        }
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            release();
            return cuda_fail(nullptr, e, "batch tables");
        }
        device = dev;
        capacity = n;
        return ZMC_OK;
    }
};

std::mutex g_batch_mu;
BatchCache g_batch;

int run_traced(zmc_ctx* h, cudaStream_t s) {
    h->trace_levels.clear();
    if (int rc = plan_shapes(h, s)) return rc;
    if (int rc = ensure_events(h)) return rc;
    cudaError_t e = cudaSuccess;
    for (int L = 1; L <= h->depth; ++L) {
        Range range("zmc level", L);
        e = enqueue_levels(h, s, L);
        if (e != cudaSuccess) return cuda_fail(h, e, "traced level launch");
        State st;
        e = cudaMemcpyAsync(&st, h->buf.state, sizeof st, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_fail(h, e, "traced level read-back");
        TraceLevel tl;
        tl.cells = st.cells[L];
        if (tl.cells > 0) {
            tl.flagged = st.flagged[L];
            tl.stats4[0] = st.mu[L]; tl.stats4[1] = st.sigma[L];
            tl.stats4[2] = st.theta[L]; tl.stats4[3] = st.min_margin[L];
            tl.sums.resize((size_t)tl.cells * h->T * 2);
            tl.cell_stats.resize((size_t)tl.cells * 2);
            tl.parents_out.resize((size_t)tl.flagged * h->dim);
            const uint32_t* next = h->buf.parents[(L + 1) & 1];
            // the statistics kernel left each tile's total in its first unit slot
            Desc D;
            build_desc(h, D);
            const int64_t chunks = level_plan(D, tl.cells).chunks;
            e = cudaMemcpy2D(tl.sums.data(), sizeof(double2), h->buf.sums,
                             sizeof(double2) * (size_t)chunks, sizeof(double2),
                             (size_t)tl.cells * h->T, cudaMemcpyDeviceToHost);
            if (e == cudaSuccess)
                e = cudaMemcpy(tl.cell_stats.data(), h->buf.cell_stats, tl.cell_stats.size() * 8,
                               cudaMemcpyDeviceToHost);
            if (e == cudaSuccess && tl.flagged > 0)
                e = cudaMemcpy(tl.parents_out.data(), next, tl.parents_out.size() * 4,
                               cudaMemcpyDeviceToHost);
            if (e != cudaSuccess) return cuda_fail(h, e, "traced level copy");
        }
        h->trace_levels.push_back(std::move(tl));
    }
    return ZMC_OK;
}

}  // namespace

// ==================================================================== ABI

extern "C" {

ZMC_API int zmc_create(zmc_handle* out, int dim, const double* lo, const double* hi, int k,
                       int64_t n, int num_trials, int depth, double sigma_multiplier,
                       uint64_t seed) {
    if (!out) return fail(nullptr, ZMC_ERR_ARG, "out is NULL");
    if (dim < 1 || dim > ZMC_MAX_DIM) return fail(nullptr, ZMC_ERR_ARG, "dim must be in 1..16");
    if (!lo || !hi) return fail(nullptr, ZMC_ERR_ARG, "lo/hi is NULL");
    for (int i = 0; i < dim; ++i)
        if (!(isfinite(lo[i]) && isfinite(hi[i]) && lo[i] < hi[i]))
            return fail(nullptr, ZMC_ERR_ARG, "need finite lo[i] < hi[i]");
    if (k < 2) return fail(nullptr, ZMC_ERR_ARG, "k must be >= 2");
    if (n < 2) return fail(nullptr, ZMC_ERR_ARG, "n must be >= 2");
    if (num_trials < 2 || num_trials > 1024)
        return fail(nullptr, ZMC_ERR_ARG, "num_trials must be in 2..1024");
    if (depth < 1 || depth > ZMC_MAX_DEPTH) return fail(nullptr, ZMC_ERR_ARG, "depth must be in 1..16");
    if (!(isfinite(sigma_multiplier) && sigma_multiplier >= 0.0))
        return fail(nullptr, ZMC_ERR_ARG, "sigma_multiplier must be finite and >= 0");
    const int64_t lim = int64_t(1) << 32;
    if (ipow_sat(k, dim, lim) >= lim) return fail(nullptr, ZMC_ERR_ARG, "k^dim must be < 2^32");
    if (ipow_sat(k, depth, lim) >= lim) return fail(nullptr, ZMC_ERR_ARG, "k^depth must be < 2^32");
    if (((n + 3) / 4) * dim > 0xFFFFFFFFll)
        return fail(nullptr, ZMC_ERR_ARG, "n * dim must be < 2^34");
    zmc_ctx* h = new zmc_ctx;
    h->dim = dim; h->k = k; h->n = n; h->T = num_trials; h->depth = depth;
    h->m = sigma_multiplier; h->seed = seed;
    h->lo.assign(lo, lo + dim);
    h->hi.assign(hi, hi + dim);
    const int64_t K = ipow_sat(k, dim, INT64_MAX);
    // default limits never refuse level 1
    h->max_cells = std::max<int64_t>(h->max_cells, K);
    const int64_t l1 = (K > INT64_MAX / (n * num_trials)) ? INT64_MAX : K * n * num_trials;
    h->max_samples = std::max<int64_t>(h->max_samples, l1);
    *out = h;
    return ZMC_OK;
}

ZMC_API int zmc_set_integrand(zmc_handle h, const char* name, const double* params,
                              int n_params) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if (!name) return fail(h, ZMC_ERR_ARG, "NULL integrand name");
    if (n_params < 0 || (n_params > 0 && !params)) return fail(h, ZMC_ERR_ARG, "bad params");
    std::vector<double> p(params, params + n_params);
    for (double v : p)
        if (!isfinite(v)) return fail(h, ZMC_ERR_ARG, "parameters must be finite");
    if (strncmp(name, "expr:", 5) == 0) {
        if (n_params > 2 * ZMC_MAX_DIM + 4)
            return fail(h, ZMC_ERR_ARG, "at most 36 expression parameters");
        DeviceGuard g(h->device);
        std::string log;
        JitKernel jk{};
        int rc = jit_compile(name + 5, h->dim, n_params, h->mode, &jk, &log);
        if (rc != ZMC_OK) return fail(h, rc, log);
        h->jit = jk;
        h->expr = name + 5;
        h->integrand = kExpression;
        h->params = p;
        h->desc_dirty = true;
        h->graph_stale = true;
        return ZMC_OK;
    }
    for (const RegistryEntry& r : kRegistry) {
        if (strcmp(name, r.name) == 0) {
            const int want = expected_params(r.id, h->dim);
            if (n_params != want) {
                char msg[160];
                snprintf(msg, sizeof msg, "%s takes %d parameters for dim %d, got %d", name, want,
                         h->dim, n_params);
                return fail(h, ZMC_ERR_ARG, msg);
            }
            if (r.id == kGaussNorm && !(p[0] > 0.0)) return fail(h, ZMC_ERR_ARG, "sigma must be > 0");
            if (r.id == kGenzProdPeak || r.id == kGenzGauss)
                for (int i = 0; i < h->dim; ++i)
                    if (p[i] == 0.0) return fail(h, ZMC_ERR_ARG, "a_i must be nonzero");
            h->integrand = r.id;
            h->params = p;
            h->expr.clear();
            h->desc_dirty = true;
            h->graph_stale = true;
            return ZMC_OK;
        }
    }
    return fail(h, ZMC_ERR_ARG, std::string("unknown integrand: ") + name);
}

ZMC_API int zmc_set_precision(zmc_handle h, int mode) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if (mode != ZMC_FP64 && mode != ZMC_FP32_FP64ACC && mode != ZMC_FP32_KAHAN)
        return fail(h, ZMC_ERR_ARG, "unknown precision mode");
    if (mode == h->mode) return ZMC_OK;
    h->mode = mode;
    if (h->integrand == kExpression) {
        DeviceGuard g(h->device);
        std::string log;
        JitKernel jk{};
        int rc = jit_compile(h->expr.c_str(), h->dim, (int)h->params.size(), mode, &jk, &log);
        if (rc != ZMC_OK) return fail(h, rc, log);
        h->jit = jk;
    }
    h->desc_dirty = true;
    h->graph_stale = true;
    return ZMC_OK;
}

ZMC_API int zmc_set_limits(zmc_handle h, int64_t max_cells, int64_t max_samples) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    const int64_t K = ipow_sat(h->k, h->dim, INT64_MAX);
    if (max_cells < K) return fail(h, ZMC_ERR_ARG, "max_cells_per_level below level 1");
    if (max_samples / (h->n * (int64_t)h->T) < K)
        return fail(h, ZMC_ERR_ARG, "max_samples below level 1");
    h->max_cells = max_cells;
    h->max_samples = max_samples;
    h->desc_dirty = true;
    h->graph_stale = true;
    return ZMC_OK;
}

ZMC_API int zmc_set_launch(zmc_handle h, int threads, int ctas_per_sm) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if (threads != 0 && threads != 64 && threads != 128 && threads != 256)
        return fail(h, ZMC_ERR_ARG, "threads must be 0 (tuned), 64, 128 or 256");
    if (ctas_per_sm < 0) return fail(h, ZMC_ERR_ARG, "ctas_per_sm must be >= 0");
    h->launch_threads = threads;
    h->launch_per_sm = ctas_per_sm;
    h->graph_stale = true;
    return ZMC_OK;
}

ZMC_API int zmc_set_work_plan(zmc_handle h, const int64_t* plan) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if (!plan) {
        h->plan_set = false;
        h->plan = kDefaultPlan;
    } else {
        WorkPlan w;
        memcpy(&w, plan, sizeof w);
        if (!plan_ok(w))
            return fail(h, ZMC_ERR_ARG,
                        "work plan: need 1 <= target_units <= 2^18, min_unit_groups >= 1, "
                        "lane_tile_groups >= 0, lane_tile_max_groups >= 0, "
                        "lane_tile_min_tiles >= 1");
        h->plan_set = true;
        h->plan = w;
    }
    h->desc_dirty = true;
    h->graph_stale = true;
    return ZMC_OK;
}

ZMC_API int zmc_set_tuning(zmc_handle h, int flags) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if (flags & ~(ZMC_TUNE_SHAPE | ZMC_TUNE_PLAN))
        return fail(h, ZMC_ERR_ARG, "tuning flags: ZMC_TUNE_SHAPE | ZMC_TUNE_PLAN");
    h->tuning = flags;
    if (!h->plan_set) h->plan = kDefaultPlan;
    h->desc_dirty = true;
    h->graph_stale = true;
    return ZMC_OK;
}

ZMC_API int zmc_launch_shape(zmc_handle h, int* threads, int* grid) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if (!h->graph && h->trace_levels.empty()) return fail(h, ZMC_ERR_ARG, "nothing has run yet");
    if (threads) *threads = h->shapes[1].threads;
    if (grid) *grid = h->shapes[std::min(2, h->depth)].grid;
    return ZMC_OK;
}

ZMC_API int zmc_set_trace(zmc_handle h, int on) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    h->trace = on != 0;
    h->trace_levels.clear();
    return ZMC_OK;
}

ZMC_API int zmc_trace_level(zmc_handle h, int level, int64_t* cells, int64_t* flagged,
                            double* stats4, double* sums, double* cell_stats,
                            uint32_t* parents_out) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if (level < 1 || level > (int)h->trace_levels.size())
        return fail(h, ZMC_ERR_ARG, "level not traced");
    const TraceLevel& t = h->trace_levels[level - 1];
    if (cells) *cells = t.cells;
    if (flagged) *flagged = t.flagged;
    if (stats4) memcpy(stats4, t.stats4, sizeof t.stats4);
    if (sums && !t.sums.empty()) memcpy(sums, t.sums.data(), t.sums.size() * 8);
    if (cell_stats && !t.cell_stats.empty())
        memcpy(cell_stats, t.cell_stats.data(), t.cell_stats.size() * 8);
    if (parents_out && !t.parents_out.empty())
        memcpy(parents_out, t.parents_out.data(), t.parents_out.size() * 4);
    return ZMC_OK;
}

ZMC_API int zmc_enqueue(zmc_handle h, void* stream) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    Range range("zmc_enqueue");
    int rc = check_ready(h);
    if (rc) return rc;
    DeviceGuard g(h->device);
    rc = ensure_device(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if (h->desc_dirty && (rc = upload_desc(h, s))) return rc;
    if ((rc = ensure_graph(h, s))) return rc;
    cudaError_t e = cudaGraphLaunch(h->graph, s);
    if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
    return ZMC_OK;
}

ZMC_API int zmc_read_result(zmc_handle h, void* stream, zmc_result* out) {
    if (!h || !out) return fail(h, ZMC_ERR_ARG, "NULL argument");
    if (!h->buf.result) return fail(h, ZMC_ERR_ARG, "nothing was enqueued");
    DeviceGuard g(h->device);
    cudaStream_t s = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(h->h_result, h->buf.result, sizeof(zmc_result),
                                    cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(h, e, "result read-back");
    return finish_result(h, out);
}

ZMC_API int zmc_integrate(zmc_handle h, void* stream, zmc_result* out) {
    if (!h || !out) return fail(h, ZMC_ERR_ARG, "NULL argument");
    Range range("zmc_integrate");
    int rc = check_ready(h);
    if (rc) return rc;
    DeviceGuard g(h->device);
    rc = ensure_device(h);
    if (rc) return rc;
    cudaStream_t s = (cudaStream_t)stream;
    if ((rc = upload_desc(h, s))) return rc;   // the run's inputs, every call
    if (h->trace) {
        if ((rc = run_traced(h, s))) return rc;
    } else {
        if ((rc = ensure_graph(h, s))) return rc;
        cudaError_t e = cudaGraphLaunch(h->graph, s);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaGraphLaunch");
    }
    return zmc_read_result(h, stream, out);
}

ZMC_API int zmc_integrate_batch(int count, const zmc_handle* hs, void* stream,
                                zmc_result* outs) {
    if (count < 0 || (count > 0 && (!hs || !outs)))
        return fail(nullptr, ZMC_ERR_ARG, "bad batch arguments");
    if (count == 0) return ZMC_OK;
    if (count > 65535) return fail(nullptr, ZMC_ERR_ARG, "at most 65535 integrals per batch");
    Range range("zmc_integrate_batch");
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    const int mode = hs[0] ? hs[0]->mode : -1;
    int depth = 0;
    for (int i = 0; i < count; ++i) {
        zmc_ctx* h = hs[i];
        if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle in batch");
        if (h->integrand < 0) return fail(nullptr, ZMC_ERR_NOINTEGRAND, "an integral has no integrand");
        if (h->integrand >= kNumIntegrands)
            return fail(nullptr, ZMC_ERR_ARG, "batched integrals need registry integrands");
        if (h->mode != mode) return fail(nullptr, ZMC_ERR_ARG, "all integrals need the same precision");
        if (h->device >= 0 && h->device != dev)
            return fail(nullptr, ZMC_ERR_ARG, "all integrals must live on the current device");
        depth = std::max(depth, h->depth);
    }
    std::lock_guard<std::mutex> lock(g_batch_mu);
    BatchCache& B = g_batch;
    for (int i = 0; i < count; ++i) {
        int rc = ensure_device(hs[i]);
        if (rc != ZMC_OK) {
            g_error = hs[i]->last_error;
            return rc;
        }
    }
    int rc = B.reserve(count, dev);
    if (rc != ZMC_OK) return rc;
    // what the kernels are told about each integral; the sampling table is
    // ordered by kernel so that each group is a contiguous range
    std::vector<Buffers> sel(count);
    std::vector<BatchEval> ev(count);
    std::vector<int64_t> l1(count);
    std::vector<const void*> kern(count);
    for (int i = 0; i < count; ++i) {
        zmc_ctx* h = hs[i];
        sel[i] = h->buf;
        sel[i].desc = B.d_desc + i;
        ev[i].desc = B.d_desc + i;
        ev[i].st = h->buf.state;
        ev[i].sums = h->buf.sums;
        ev[i].parents[0] = h->buf.parents[0];
        ev[i].parents[1] = h->buf.parents[1];
        ev[i].keys = philox_keys(h->seed);
        ev[i].fn = h->integrand;
        kern[i] = batch_kernel(mode, ev[i].fn, h->dim);
        if (!kern[i])
            return fail(nullptr, ZMC_ERR_ARG, "this build of the library has no batched kernel "
                                              "for an integrand of the batch");
        l1[i] = ipow_sat(h->k, h->dim, INT64_MAX);
        build_desc(h, B.h_desc[i]);
    }
    std::vector<int> order(count);
    for (int i = 0; i < count; ++i) order[i] = i;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
        return std::make_pair(ev[a].fn, hs[a]->dim > 8) < std::make_pair(ev[b].fn, hs[b]->dim > 8);
    });
    std::vector<BatchEval> ev_sorted(count);
    std::vector<BatchGroup> groups;
    for (int r = 0; r < count; ++r) {
        ev_sorted[r] = ev[order[r]];
        if (groups.empty() || groups.back().kernel != kern[order[r]])
            groups.push_back(BatchGroup{kern[order[r]], r, 0, 0});
        ++groups.back().count;
    }
    ev.swap(ev_sorted);
    cudaStream_t s = (cudaStream_t)stream;
    const bool same = B.count == count && B.mode == mode && B.depth == depth &&
                      !B.graphs.empty() &&
                      memcmp(B.sel.data(), sel.data(), sizeof(Buffers) * count) == 0 &&
                      memcmp(B.eval.data(), ev.data(), sizeof(BatchEval) * count) == 0;
    if (!same) {
        B.drop_graphs();
        e = cudaMemcpy(B.d_sel, sel.data(), sizeof(Buffers) * count, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(B.d_eval, ev.data(), sizeof(BatchEval) * count, cudaMemcpyHostToDevice);
        if (e == cudaSuccess)
            e = cudaMemcpy(B.d_l1, l1.data(), sizeof(int64_t) * count, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch tables upload");
        B.sel = sel;
        B.eval = ev;
        B.count = count;
        B.mode = mode;
        B.depth = depth;
        int sms = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        for (BatchGroup& g : groups) {
            int per_sm = 0;
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, g.kernel, kBatchThreads, 0);
            g.grid = std::max(1, per_sm) * std::max(1, sms);
        }
        B.groups = groups;
        for (int L = 1; L <= depth; ++L) {
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(B.cap, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch capture");
            cudaError_t le = cudaSuccess;
            if (L == 1) le = launch_init_batch(B.d_sel, B.d_l1, count, B.cap);
            // one branch per group: its plan and sampling kernels
            if (le == cudaSuccess && groups.size() > 1) le = cudaEventRecord(B.fork, B.cap);
            for (size_t j = 0; le == cudaSuccess && j < groups.size(); ++j) {
                const BatchGroup& G = groups[j];
                cudaStream_t bs = j == 0 ? B.cap : B.side[j];
                if (j > 0) le = cudaStreamWaitEvent(bs, B.fork, 0);
                if (le == cudaSuccess)
                    le = launch_batch_level(B.d_eval + G.start, G.count, L,
                                            B.d_offsets + G.start + j, B.d_head + j, G.kernel,
                                            G.grid, bs);
                if (le == cudaSuccess && j > 0) le = cudaEventRecord(B.join[j], bs);
                if (le == cudaSuccess && j > 0) le = cudaStreamWaitEvent(B.cap, B.join[j], 0);
            }
            if (le == cudaSuccess) le = launch_select_batch(B.d_sel, count, L, B.cap);
            if (le == cudaSuccess && L == depth) le = launch_final_batch(B.d_sel, B.d_out, count, B.cap);
            e = cudaStreamEndCapture(B.cap, &g);
            if (le != cudaSuccess || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                B.drop_graphs();
                return cuda_fail(nullptr, le != cudaSuccess ? le : e, "batch level capture");
            }
            cudaGraphExec_t x = nullptr;
            e = cudaGraphInstantiate(&x, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                B.drop_graphs();
                return cuda_fail(nullptr, e, "batch graph instantiate");
            }
            B.graphs.push_back(x);
        }
    }
    // the integrals' parameters, every call; then every level; then results
    e = cudaMemcpyAsync(B.d_desc, B.h_desc, sizeof(Desc) * count, cudaMemcpyHostToDevice, s);
    for (size_t L = 0; e == cudaSuccess && L < B.graphs.size(); ++L) {
        Range level("zmc batch level", (int)L + 1);
        e = cudaGraphLaunch(B.graphs[L], s);
    }
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(B.h_out, B.d_out, sizeof(zmc_result) * count, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch run");
    int first = ZMC_OK;
    for (int i = 0; i < count; ++i) {
        outs[i] = B.h_out[i];
        memcpy(outs[i].work_plan, &hs[i]->plan, sizeof outs[i].work_plan);
        // keep the handles' own descriptors in step for later single runs
        hs[i]->desc_dirty = true;
        if (outs[i].status != ZMC_OK && first == ZMC_OK) first = outs[i].status;
    }
    return first;
}

ZMC_API int zmc_philox_words(uint64_t seed, uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                             int64_t count, uint32_t* out, void* stream) {
    if (count < 0 || (count > 0 && !out)) return fail(nullptr, ZMC_ERR_ARG, "bad arguments");
    cudaError_t e = launch_philox(seed, c0, c1, c2, c3, count, out, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "philox launch");
    return ZMC_OK;
}

ZMC_API int zmc_set_profiling(zmc_handle h, int on) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if ((on != 0) != h->profiling) {
        h->profiling = on != 0;
        h->graph_stale = true;
    }
    return ZMC_OK;
}

ZMC_API int zmc_profile(zmc_handle h, double* eval_ms, int* levels) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if (!h->profiling || !h->graph) return fail(h, ZMC_ERR_ARG, "profiling was not on for a run");
    DeviceGuard g(h->device);
    State st;
    cudaError_t e = cudaMemcpy(&st, h->buf.state, sizeof st, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(h, e, "state read-back");
    int ran = 0;
    for (int L = 1; L <= h->depth; ++L) {
        float ms = 0.f;
        e = cudaEventElapsedTime(&ms, h->ev[L][0], h->ev[L][1]);
        if (e != cudaSuccess) return cuda_fail(h, e, "cudaEventElapsedTime");
        if (eval_ms) eval_ms[L - 1] = ms;
        if (st.cells[L] > 0) ++ran;
    }
    if (levels) *levels = ran;
    return ZMC_OK;
}

ZMC_API int zmc_run_info(zmc_handle h, int64_t* kernels, int64_t* h2d_bytes, int64_t* d2h_bytes) {
    if (!h) return fail(nullptr, ZMC_ERR_ARG, "NULL handle");
    if (kernels) *kernels = h->graph_kernels;
    if (h2d_bytes) *h2d_bytes = (int64_t)sizeof(Desc);
    if (d2h_bytes) *d2h_bytes = (int64_t)sizeof(zmc_result);
    return ZMC_OK;
}

ZMC_API int zmc_pipe_probe(int kind, int64_t iters, int blocks, int threads, uint32_t* sink,
                           int64_t* clocks, void* stream) {
    if (!pipe_probe_kind_valid(kind) || iters < 1 || blocks < 1 || threads < 32 ||
        threads > 256 || threads % 32 != 0 || !sink || !clocks)
        return fail(nullptr, ZMC_ERR_ARG, "bad probe arguments");
    cudaError_t e = launch_pipe_probe(kind, iters, blocks, threads, sink, (long long*)clocks,
                                      (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "probe launch");
    return ZMC_OK;
}

ZMC_API int zmc_uniforms(uint64_t seed, int level, uint32_t slot, uint32_t trial, int dim,
                         int mode, int64_t first, int64_t count, double* out, void* stream) {
    if (level < 1 || dim < 1 || dim > ZMC_MAX_DIM || first < 0 || count < 0 ||
        (count > 0 && !out) ||
        (mode != ZMC_FP64 && mode != ZMC_FP32_FP64ACC && mode != ZMC_FP32_KAHAN))
        return fail(nullptr, ZMC_ERR_ARG, "bad arguments");
    const int G = points_per_group(mode), B = blocks_per_group(mode);
    if (((first + count + G - 1) / G) * dim * B > 0xFFFFFFFFll)
        return fail(nullptr, ZMC_ERR_ARG, "points beyond the 2^32-block counter range");
    cudaError_t e = launch_uniforms(seed, level, slot, trial, dim, mode, first, count, out,
                                    (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "uniforms launch");
    return ZMC_OK;
}

ZMC_API int zmc_level_stats_noalloc(const double* sums, int64_t cells, int trials, int64_t n,
                                    double volume, double sigma_multiplier, double* cell_stats,
                                    double* level_stats, void* stream) {
    const int rc = level_stats_noalloc(sums, cells, trials, n, volume, sigma_multiplier,
                                       cell_stats, level_stats, (cudaStream_t)stream);
    if (rc != ZMC_OK) return fail(nullptr, rc, noalloc_last_error());
    return ZMC_OK;
}

ZMC_API int zmc_check_expression(const char* expr, int dim, int mode, int cc_major, int cc_minor,
                                 char* log, size_t log_size) {
    if (log && log_size) log[0] = '\0';
    if (dim < 1 || dim > ZMC_MAX_DIM || cc_major < 1 || cc_minor < 0 || (log_size && !log) ||
        (mode != ZMC_FP64 && mode != ZMC_FP32_FP64ACC && mode != ZMC_FP32_KAHAN))
        return fail(nullptr, ZMC_ERR_ARG, "bad arguments");
    std::string msg;
    const int rc = jit_check(expr, dim, mode, cc_major, cc_minor, &msg);
    if (log && log_size) {
        const size_t m = std::min(msg.size(), log_size - 1);
        memcpy(log, msg.data(), m);
        log[m] = '\0';
    }
    if (rc != ZMC_OK) return fail(nullptr, rc, msg.c_str());
    return ZMC_OK;
}

ZMC_API const char* zmc_last_error(zmc_handle h) {
    return h ? h->last_error.c_str() : g_error.c_str();
}

ZMC_API int zmc_destroy(zmc_handle h) {
    if (!h) return ZMC_OK;
    if (h->device >= 0) {
        DeviceGuard g(h->device);
        free_device(h);
    }
    jit_release(&h->jit);
    delete h;
    return ZMC_OK;
}

}  // extern "C"
