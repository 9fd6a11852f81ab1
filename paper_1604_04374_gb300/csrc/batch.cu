// batch.cu -- many applies at once: a lane scheduler (longest processing time
// first over a pool of streams), replay of a whole batch as one CUDA graph
// launch, and the autotuner that picks, per plan, the column FFT variant
// (one-warp 32 x 32 four-step or radix-8 Stockham for columns of 1024) and
// the right-hand sides per launch, with an optional JSON-lines cache.
//
// The batch runs the same kernels as pce_apply; only the issue order, the
// streams and the scratch buffers differ, so every task's result is bitwise
// the result of pce_apply / pce_apply_adjoint with the same chunking.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "pce.h"
#include "plan.h"

using pce_rt::fail;

#define PCE_BCK(call)                                                                      \
    do {                                                                                   \
        cudaError_t e_ = (call);                                                           \
        if (e_ != cudaSuccess)                                                             \
            return fail(e_ == cudaErrorMemoryAllocation ? PCE_ERR_OOM : PCE_ERR_CUDA,      \
                        "%s failed: %s", #call, cudaGetErrorString(e_));                   \
    } while (0)

namespace {

constexpr int kMaxLanes = 64;
constexpr int kPoolLanes = 16;
// FP32 flops per millisecond used to turn the work model into a cost when a
// plan has not been autotuned (an order of magnitude is all LPT needs).
constexpr double kModelFlopsPerMs = 1.5e10;

long long round_up(long long v, long long a) { return (v + a - 1) / a * a; }

// Estimated milliseconds of one task.
double task_cost(const pce_task& t) {
    const pce_plan* p = t.plan;
    if (p->tuned_ms > 0.0) return p->tuned_ms * (double)t.batch;
    return pce_rt::model_flops(p, t.batch) / kModelFlopsPerMs;
}

// Right-hand sides per launch a task runs with.
int task_chunk(const pce_task& t) {
    const int c = pce_rt::plan_scratch(t.plan).chunk;
    return (int)std::max<long long>(1, std::min<long long>(c, t.batch));
}

// float2 of lane scratch a task needs (Z region rounded to 256 bytes, then A).
long long task_scratch(const pce_task& t, long long& zs, long long& as, int& chunk) {
    pce_rt::scratch_per_rhs(t.plan, zs, as);
    chunk = task_chunk(t);
    if (zs == 0 && as == 0) return 0;
    return round_up(zs * chunk, 32) + round_up(as * chunk, 32);
}

pce_status check_task(const pce_task& t, int device, int i) {
    if (!t.plan) return fail(PCE_ERR_INVALID, "task %d: plan is NULL", i);
    if (t.adjoint != 0 && t.adjoint != 1) return fail(PCE_ERR_INVALID, "task %d: adjoint must be 0 or 1", i);
    if (t.plan->device != device)
        return fail(PCE_ERR_INVALID, "task %d: plan belongs to device %d, current is %d", i, t.plan->device,
                    device);
    if (t.plan->flags & PCE_FLAG_UNFUSED)
        return fail(PCE_ERR_UNSUPPORTED, "task %d: plans with PCE_FLAG_UNFUSED do not run in batches", i);
    pce_status st = pce_rt::check_io(t.plan, t.in, t.out, t.batch);
    if (st) return fail(st, "task %d: %s", i, pce_last_error_string());
    return PCE_OK;
}

// No task may write memory another task reads or writes.
pce_status check_independent(const pce_task* tasks, int n) {
    struct Range {
        const char* lo;
        const char* hi;
        int task;
        bool write;
    };
    std::vector<Range> r;
    r.reserve(2 * (size_t)n);
    for (int i = 0; i < n; ++i) {
        const pce_plan* p = tasks[i].plan;
        const long long bytes = (long long)p->ny * p->nx * tasks[i].batch * (long long)sizeof(float);
        if (bytes == 0) continue;
        const char* a = reinterpret_cast<const char*>(tasks[i].in);
        const char* b = reinterpret_cast<const char*>(tasks[i].out);
        r.push_back({a, a + bytes, i, false});
        r.push_back({b, b + bytes, i, true});
    }
    std::sort(r.begin(), r.end(), [](const Range& x, const Range& y) { return x.lo < y.lo; });
    // sweep: ranges sorted by start; compare each with every earlier range still open
    for (size_t j = 0; j < r.size(); ++j) {
        for (size_t i = j; i-- > 0;) {
            if (r[i].hi <= r[j].lo) continue;
            if (r[i].task != r[j].task && (r[i].write || r[j].write))
                return fail(PCE_ERR_INVALID, "tasks %d and %d overlap in memory one of them writes",
                            std::min(r[i].task, r[j].task), std::max(r[i].task, r[j].task));
        }
    }
    return PCE_OK;
}

// Longest processing time first: tasks by decreasing cost, each to the lane
// with the least load so far (ties: lowest lane, then lowest task index).
double lpt(const std::vector<double>& cost, int lanes, std::vector<int>& lane_of) {
    const int n = (int)cost.size();
    std::vector<int> idx(n);
    std::iota(idx.begin(), idx.end(), 0);
    std::stable_sort(idx.begin(), idx.end(), [&](int a, int b) { return cost[a] > cost[b]; });
    std::vector<double> load(lanes, 0.0);
    lane_of.assign(n, 0);
    for (int i : idx) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        lane_of[i] = l;
        load[l] += cost[i];
    }
    return lanes > 0 ? *std::max_element(load.begin(), load.end()) : 0.0;
}

}  // namespace

extern "C" pce_status pce_schedule_lpt(const double* cost, int n, int lanes, int* lane_of,
                                       double* makespan) {
    if (n < 0 || (n > 0 && (!cost || !lane_of))) return fail(PCE_ERR_INVALID, "cost and lane_of must hold n entries");
    if (lanes < 1) return fail(PCE_ERR_INVALID, "lanes must be >= 1 (got %d)", lanes);
    std::vector<double> c(cost, cost + n);
    for (int i = 0; i < n; ++i)
        if (!(c[i] >= 0.0)) return fail(PCE_ERR_INVALID, "cost[%d] must be >= 0", i);
    std::vector<int> lo;
    const double ms = lpt(c, lanes, lo);
    for (int i = 0; i < n; ++i) lane_of[i] = lo[i];
    if (makespan) *makespan = ms;
    return PCE_OK;
}

// ----------------------------------------------------------------- batches

struct pce_batch {
    int device = 0;
    int lanes = 0;
    std::vector<pce_task> tasks;
    std::vector<std::vector<int>> order;        // per lane: task indices in issue order
    std::vector<pce_rt::Scratch> scr;           // per task: its view of its lane's scratch
    std::vector<cudaStream_t> streams;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
    float2* lane_mem = nullptr;
    long long scratch_bytes = 0;
    double makespan_ms = 0.0;
    long long launches = 0;
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int col_policy = -1, row_policy = -1;   // -1: every plan's own variants
    std::vector<double> tune_log;           // (col policy, row policy, ms per run)

    void drop_graph() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        exec = nullptr;
        graph = nullptr;
    }

    ~pce_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (cudaStream_t s : streams)
            if (s) cudaStreamDestroy(s);
        if (cap) cudaStreamDestroy(cap);
        if (fork) cudaEventDestroy(fork);
        for (cudaEvent_t e : join)
            if (e) cudaEventDestroy(e);
        if (lane_mem) cudaFree(lane_mem);
    }
};

namespace {

// Fork from `s` onto the lanes, issue every lane's tasks, join back into `s`.
pce_status issue(const std::vector<pce_task>& tasks, const std::vector<std::vector<int>>& order,
                 const std::vector<pce_rt::Scratch>& scr, const std::vector<cudaStream_t>& streams,
                 cudaEvent_t fork, const std::vector<cudaEvent_t>& join, cudaStream_t s) {
    PCE_BCK(cudaEventRecord(fork, s));
    for (size_t l = 0; l < order.size(); ++l) {
        if (order[l].empty()) continue;
        PCE_BCK(cudaStreamWaitEvent(streams[l], fork, 0));
        for (int i : order[l]) {
            const pce_task& t = tasks[i];
            if (t.batch == 0) continue;
            pce_status st = pce_rt::apply_with(t.plan, t.in, t.out, t.batch, t.adjoint != 0, streams[l], scr[i],
                                               false);
            if (st) return fail(st, "task %d: %s", i, pce_last_error_string());
        }
        PCE_BCK(cudaEventRecord(join[l], streams[l]));
        PCE_BCK(cudaStreamWaitEvent(s, join[l], 0));
    }
    return PCE_OK;
}

pce_status make_lanes(int lanes, std::vector<cudaStream_t>& streams, cudaEvent_t& fork,
                      std::vector<cudaEvent_t>& join) {
    streams.assign(lanes, nullptr);
    join.assign(lanes, nullptr);
    PCE_BCK(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming));
    for (int l = 0; l < lanes; ++l) {
        PCE_BCK(cudaStreamCreateWithFlags(&streams[l], cudaStreamNonBlocking));
        PCE_BCK(cudaEventCreateWithFlags(&join[l], cudaEventDisableTiming));
    }
    return PCE_OK;
}

pce_status validate_tasks(const pce_task* tasks, int n, int& device) {
    if (n < 0) return fail(PCE_ERR_INVALID, "n must be >= 0 (got %d)", n);
    if (n > 0 && !tasks) return fail(PCE_ERR_INVALID, "tasks is NULL");
    PCE_BCK(cudaGetDevice(&device));
    for (int i = 0; i < n; ++i) {
        pce_status st = check_task(tasks[i], device, i);
        if (st) return st;
    }
    return check_independent(tasks, n);
}

}  // namespace

extern "C" pce_status pce_batch_create(pce_batch_t* out, const pce_task* tasks, int n, int lanes) {
    if (!out) return fail(PCE_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (lanes < 1 || lanes > kMaxLanes) return fail(PCE_ERR_INVALID, "lanes must be in [1, %d] (got %d)", kMaxLanes, lanes);
    int device = 0;
    pce_status st = validate_tasks(tasks, n, device);
    if (st) return st;
    pce_batch* b = new pce_batch();
    b->device = device;
    b->lanes = lanes;
    b->tasks.assign(tasks, tasks + n);
    std::vector<double> cost(n);
    for (int i = 0; i < n; ++i) cost[i] = task_cost(tasks[i]);
    std::vector<int> lane_of;
    b->makespan_ms = lpt(cost, lanes, lane_of);
    b->order.assign(lanes, {});
    for (int i = 0; i < n; ++i) b->order[lane_of[i]].push_back(i);
    // lane scratch: each lane holds the largest need of its tasks
    std::vector<long long> need(lanes, 0);
    std::vector<long long> zs(n), as(n);
    std::vector<int> ch(n);
    for (int i = 0; i < n; ++i) {
        need[lane_of[i]] = std::max(need[lane_of[i]], task_scratch(tasks[i], zs[i], as[i], ch[i]));
        b->launches += pce_launch_count(tasks[i].plan, tasks[i].adjoint, tasks[i].batch);
    }
    std::vector<long long> off(lanes + 1, 0);
    for (int l = 0; l < lanes; ++l) off[l + 1] = off[l] + round_up(need[l], 32);
    b->scratch_bytes = off[lanes] * (long long)sizeof(float2);
    if (off[lanes] > 0) {
        cudaError_t e = cudaMalloc(&b->lane_mem, (size_t)b->scratch_bytes);
        if (e != cudaSuccess) {
            delete b;
            return fail(e == cudaErrorMemoryAllocation ? PCE_ERR_OOM : PCE_ERR_CUDA,
                        "lane scratch of %lld bytes: %s", b->scratch_bytes, cudaGetErrorString(e));
        }
    }
    b->scr.resize(n);
    for (int i = 0; i < n; ++i) {
        pce_rt::Scratch& s = b->scr[i];
        float2* base = b->lane_mem ? b->lane_mem + off[lane_of[i]] : nullptr;
        s.zstride = zs[i];
        s.astride = as[i];
        s.chunk = ch[i];
        s.Z = base;
        s.A = base ? base + round_up(zs[i] * ch[i], 32) : nullptr;
    }
    if ((st = make_lanes(lanes, b->streams, b->fork, b->join))) {
        delete b;
        return st;
    }
    *out = b;
    return PCE_OK;
}

extern "C" pce_status pce_batch_run(pce_batch_t b, void* stream) {
    if (!b) return fail(PCE_ERR_INVALID, "batch is NULL");
    int dev = 0;
    PCE_BCK(cudaGetDevice(&dev));
    if (dev != b->device) return fail(PCE_ERR_INVALID, "batch belongs to device %d, current is %d", b->device, dev);
    return issue(b->tasks, b->order, b->scr, b->streams, b->fork, b->join, static_cast<cudaStream_t>(stream));
}

extern "C" pce_status pce_batch_launch(pce_batch_t b, void* stream) {
    if (!b) return fail(PCE_ERR_INVALID, "batch is NULL");
    int dev = 0;
    PCE_BCK(cudaGetDevice(&dev));
    if (dev != b->device) return fail(PCE_ERR_INVALID, "batch belongs to device %d, current is %d", b->device, dev);
    if (!b->exec) {
        if (!b->cap) PCE_BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
        PCE_BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
        pce_status st = issue(b->tasks, b->order, b->scr, b->streams, b->fork, b->join, b->cap);
        cudaGraph_t g = nullptr;
        cudaError_t e = cudaStreamEndCapture(b->cap, &g);
        if (st) {
            if (g) cudaGraphDestroy(g);
            return st;
        }
        if (e != cudaSuccess) {
            if (g) cudaGraphDestroy(g);
            return fail(PCE_ERR_CUDA, "graph capture of the batch: %s", cudaGetErrorString(e));
        }
        e = cudaGraphInstantiate(&b->exec, g, 0);
        if (e != cudaSuccess) {
            cudaGraphDestroy(g);
            b->exec = nullptr;
            return fail(PCE_ERR_CUDA, "graph instantiation: %s", cudaGetErrorString(e));
        }
        b->graph = g;
    }
    PCE_BCK(cudaGraphLaunch(b->exec, static_cast<cudaStream_t>(stream)));
    return PCE_OK;
}

extern "C" pce_status pce_batch_info(pce_batch_t b, int* lanes, int64_t* scratch_bytes, int64_t* launches,
                                     double* model_makespan_ms, int* lane_of) {
    if (!b) return fail(PCE_ERR_INVALID, "batch is NULL");
    if (lanes) *lanes = b->lanes;
    if (scratch_bytes) *scratch_bytes = b->scratch_bytes;
    if (launches) *launches = b->launches;
    if (model_makespan_ms) *model_makespan_ms = b->makespan_ms;
    if (lane_of)
        for (int l = 0; l < b->lanes; ++l)
            for (int i : b->order[l]) lane_of[i] = l;
    return PCE_OK;
}

extern "C" pce_status pce_batch_destroy(pce_batch_t b) {
    if (!b) return PCE_OK;
    cudaError_t e = cudaDeviceSynchronize();
    delete b;
    if (e != cudaSuccess) return fail(PCE_ERR_CUDA, "synchronise before free: %s", cudaGetErrorString(e));
    return PCE_OK;
}

// -------------------------------------------- one-shot batches (plan scratch)

namespace {

struct Pool {
    bool ready = false;
    std::vector<cudaStream_t> streams;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> join;
};
Pool g_pools[kMaxLanes];   // per device
std::mutex g_pool_mutex;

}  // namespace

extern "C" pce_status pce_apply_batch(const pce_task* tasks, int n, void* stream) {
    int device = 0;
    pce_status st = validate_tasks(tasks, n, device);
    if (st) return st;
    if (n == 0) return PCE_OK;
    if (device >= kMaxLanes) return fail(PCE_ERR_UNSUPPORTED, "device %d is beyond the stream pools", device);
    // tasks of one plan share its scratch: one group per plan, issued in order on one lane
    std::vector<const pce_plan*> plans;
    std::vector<int> group(n);
    for (int i = 0; i < n; ++i) {
        auto it = std::find(plans.begin(), plans.end(), tasks[i].plan);
        group[i] = (int)(it - plans.begin());
        if (it == plans.end()) plans.push_back(tasks[i].plan);
    }
    const int ng = (int)plans.size();
    std::vector<double> gcost(ng, 0.0);
    for (int i = 0; i < n; ++i) gcost[group[i]] += task_cost(tasks[i]);
    const int lanes = std::min(ng, kPoolLanes);
    std::vector<int> lane_of_group;
    lpt(gcost, lanes, lane_of_group);
    std::vector<std::vector<int>> order(lanes);
    std::vector<pce_task> tv(tasks, tasks + n);
    std::vector<pce_rt::Scratch> scr(n);
    for (int i = 0; i < n; ++i) {
        order[lane_of_group[group[i]]].push_back(i);
        scr[i] = pce_rt::plan_scratch(tasks[i].plan);
    }
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    Pool& pool = g_pools[device];
    if (!pool.ready) {
        if ((st = make_lanes(kPoolLanes, pool.streams, pool.fork, pool.join))) return st;
        pool.ready = true;
    }
    std::vector<cudaStream_t> ls(pool.streams.begin(), pool.streams.begin() + lanes);
    std::vector<cudaEvent_t> lj(pool.join.begin(), pool.join.begin() + lanes);
    return issue(tv, order, scr, ls, pool.fork, lj, static_cast<cudaStream_t>(stream));
}

// ------------------------------------------------------------------ autotuner

namespace {

__global__ void k_fill_pattern(float* x, long long n) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned h = (unsigned)(i * 2654435761ull) >> 8;
        x[i] = (float)(h & 0xffff) * (1.0f / 65536.0f) - 0.5f;
    }
}

std::string tune_key(const pce_plan* p, int64_t batch) {
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, p->device) != cudaSuccess) {
        cudaGetLastError();
        std::memset(&prop, 0, sizeof prop);
    }
    unsigned long long h = 1469598103934665603ull;   // FNV-1a over the support boxes
    for (const Box& b : p->box) {
        const int v[4] = {b.r0, b.nr, b.c0, b.nc};
        for (int x : v)
            for (int k = 0; k < 4; ++k) {
                h ^= (unsigned)(x >> (8 * k)) & 0xffu;
                h *= 1099511628211ull;
            }
    }
    std::string name(prop.name);
    std::replace(name.begin(), name.end(), '"', '\'');
    char buf[512];
    snprintf(buf, sizeof buf, "%s|sm%d%d|nd%d|%dx%d|m%d|f%u|box%016llx|b%lld", name.c_str(), prop.major,
             prop.minor, p->ndims, p->ny, p->nx, p->m, p->flags, h, (long long)batch);
    return buf;
}

bool cache_lookup(const char* path, const std::string& key, int& chunk, int& variant, int& rvariant,
                  double& ms) {
    FILE* f = std::fopen(path, "r");
    if (!f) return false;
    const std::string pat = "\"key\": \"" + key + "\"";
    bool found = false;
    char line[2048];
    while (std::fgets(line, sizeof line, f)) {
        if (!std::strstr(line, pat.c_str())) continue;
        const char* c = std::strstr(line, "\"chunk\": ");
        const char* v = std::strstr(line, "\"variant\": ");
        const char* t = std::strstr(line, "\"ms_per_apply\": ");
        const char* rv = std::strstr(line, "\"row_variant\": ");
        int rr = 0;
        if (rv && (std::sscanf(rv + 15, "%d", &rr) != 1 || rr < 0 || rr > 2)) continue;
        int cc = 0, vv = 0;
        double tt = 0.0;
        if (c && v && t && std::sscanf(c + 9, "%d", &cc) == 1 && std::sscanf(v + 11, "%d", &vv) == 1 &&
            std::sscanf(t + 16, "%lf", &tt) == 1 && cc >= 1 && vv >= 0 && vv <= 4) {
            chunk = cc;
            variant = vv;
            rvariant = rr;
            ms = tt;
            found = true;   // the last matching line wins
        }
    }
    std::fclose(f);
    return found;
}

pce_status cache_store(const char* path, const std::string& key, int chunk, int variant, int rvariant,
                       double ms) {
    FILE* f = std::fopen(path, "a");
    if (!f) return fail(PCE_ERR_INVALID, "cannot open the tuning cache %s for appending", path);
    std::fprintf(f, "{\"key\": \"%s\", \"chunk\": %d, \"variant\": %d, \"row_variant\": %d, \"ms_per_apply\": %.6g}\n",
                 key.c_str(), chunk, variant, rvariant, ms);
    std::fclose(f);
    return PCE_OK;
}

}  // namespace

extern "C" pce_status pce_plan_autotune(pce_plan_t p, int64_t batch, const char* cache_path, void* stream) {
    if (!p) return fail(PCE_ERR_INVALID, "plan is NULL");
    if (batch < 1 || batch > (1 << 20)) return fail(PCE_ERR_INVALID, "batch must be in [1, 2^20] (got %lld)", (long long)batch);
    int dev = 0;
    PCE_BCK(cudaGetDevice(&dev));
    if (dev != p->device) return fail(PCE_ERR_INVALID, "plan belongs to device %d, current is %d", p->device, dev);
    if (p->flags & PCE_FLAG_UNFUSED) return fail(PCE_ERR_UNSUPPORTED, "plans with PCE_FLAG_UNFUSED have nothing to tune");
    const std::string key = tune_key(p, batch);
    const int cmax = (int)std::max<long long>(1, std::min<long long>(p->bchunk, batch));
    if (cache_path) {
        int c = 0, v = 0, rv = 0;
        double ms = 0.0;
        if (cache_lookup(cache_path, key, c, v, rv, ms)) {
            p->tune_log.clear();
            p->run_chunk = std::min(c, cmax);
            const bool ok = p->ndims == 2 && (p->ny == 512 || p->ny == 1024 || p->ny == 2048) && v >= 0 &&
                            (v < 2 || (p->sep && p->ny == 1024) || (v == 2 && p->sep && p->ny == 512)) &&
                            (v != 3 || p->sep_prune) &&
                            (v != 4 || p->nslots > 1);
            p->col_variant = ok ? v : 0;
            p->row_variant = (p->ndims == 2 && rv >= 0 && rv <= 2) ? rv : 0;
            p->tuned_ms = ms;
            return PCE_OK;
        }
    }
    // candidates
    // a sectioned plan runs its own kernels and chunks: one candidate, timed
    std::vector<int> variants = {0};
    if (p->ndims == 2 && !p->sect && (p->ny == 512 || p->ny == 1024 || p->ny == 2048)) variants.push_back(1);
    if (p->sep && !p->sect && (p->ny == 1024 || p->ny == 512)) variants.push_back(2);
    if (p->sep && p->sep_prune && !p->sect && p->ny == 1024) variants.push_back(3);
    if (p->sep && p->nslots > 1 && !p->sect && p->ny == 1024) variants.push_back(4);
    std::vector<int> rvariants = {0};
    if (p->ndims == 2 && !p->sect) rvariants.push_back(1);
    if (p->ndims == 2 && !p->sect && !(p->flags & PCE_FLAG_UNFUSED)) rvariants.push_back(2);
    std::vector<int> chunks;
    if ((p->ndims == 2 && !p->sect) || p->l1) {
        for (int c = 1; c < cmax; c *= 2) chunks.push_back(c);
    }
    chunks.push_back(cmax);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long P = (long long)p->ny * p->nx;
    float* in = nullptr;
    float* out = nullptr;
    void* flush = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t flush_bytes = 192ull << 20;   // larger than the L2
    auto cleanup = [&]() {
        if (in) cudaFree(in);
        if (out) cudaFree(out);
        if (flush) cudaFree(flush);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&in, sizeof(float) * P * batch);
    if (e == cudaSuccess) e = cudaMalloc(&out, sizeof(float) * P * batch);
    if (e == cudaSuccess) e = cudaMalloc(&flush, flush_bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        k_fill_pattern<<<1024, 256, 0, s>>>(in, P * batch);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) {
        cleanup();
        return fail(e == cudaErrorMemoryAllocation ? PCE_ERR_OOM : PCE_ERR_CUDA, "autotune set-up: %s",
                    cudaGetErrorString(e));
    }
    const int saved_chunk = p->run_chunk, saved_variant = p->col_variant, saved_rv = p->row_variant;
    p->tune_log.clear();
    double best = 1e300;
    int best_c = cmax, best_v = 0, best_r = 0;
    pce_status st = PCE_OK;
    for (int v : variants) {
      for (int rv : rvariants) {
        for (int c : chunks) {
            p->col_variant = v;
            p->row_variant = rv;
            p->run_chunk = c;
            const pce_rt::Scratch scr = pce_rt::plan_scratch(p);
            float tmin = 1e30f;
            for (int rep = 0; rep < 4 && st == PCE_OK; ++rep) {   // rep 0 warms up
                e = cudaMemsetAsync(flush, rep, flush_bytes, s);
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                if (e != cudaSuccess) break;
                st = pce_rt::apply_with(p, in, out, batch, false, s, scr, false);
                if (st == PCE_OK) st = pce_rt::apply_with(p, in, out, batch, true, s, scr, false);
                if (st) break;
                e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) break;
                if (rep > 0) tmin = std::min(tmin, ms);
            }
            if (st == PCE_OK && e != cudaSuccess)
                st = fail(PCE_ERR_CUDA, "autotune timing: %s", cudaGetErrorString(e));
            if (st) break;
            const double per_apply = (double)tmin / (2.0 * (double)batch);
            p->tune_log.insert(p->tune_log.end(), {(double)c, (double)v, (double)rv, per_apply});
            if (per_apply < best) {
                best = per_apply;
                best_c = c;
                best_v = v;
                best_r = rv;
            }
        }
        if (st) break;
      }
      if (st) break;
    }
    cleanup();
    if (st) {
        p->run_chunk = saved_chunk;
        p->col_variant = saved_variant;
        p->row_variant = saved_rv;
        return st;
    }
    p->run_chunk = best_c;
    p->col_variant = best_v;
    p->row_variant = best_r;
    p->tuned_ms = best;
    if (cache_path) return cache_store(cache_path, key, best_c, best_v, best_r, best);
    return PCE_OK;
}

extern "C" pce_status pce_plan_set_tuning(pce_plan_t p, int chunk, int col_variant, int row_variant) {
    if (!p) return fail(PCE_ERR_INVALID, "plan is NULL");
    if (chunk < 0) return fail(PCE_ERR_INVALID, "chunk must be >= 0 (got %d)", chunk);
    if (col_variant < 0 || col_variant > 4 || row_variant < 0 || row_variant > 2)
        return fail(PCE_ERR_INVALID, "column variant must be 0..4 and row variant 0..2 (got %d, %d)", col_variant,
                    row_variant);
    if (col_variant == 1 && !(p->ndims == 2 && (p->ny == 512 || p->ny == 1024 || p->ny == 2048)))
        return fail(PCE_ERR_UNSUPPORTED, "column variant 1 needs a 2D plan with 512, 1024 or 2048 rows");
    if (col_variant == 2 && !(p->sep && (p->ny == 1024 || p->ny == 512)))
        return fail(PCE_ERR_UNSUPPORTED, "column variant 2 needs a separable plan with 1024 or 512 rows");
    if (col_variant == 3 && !(p->sep && p->sep_prune))
        return fail(PCE_ERR_UNSUPPORTED,
                    "column variant 3 needs a separable plan with 1024 rows whose row factors each lie in "
                    "512 rows starting on a multiple of 32");
    if (col_variant == 4 && !(p->sep && p->ny == 1024 && p->nslots > 1))
        return fail(PCE_ERR_UNSUPPORTED, "column variant 4 needs a separable plan with 1024 rows and two or more slots");
    if (row_variant != 0 && p->ndims != 2) return fail(PCE_ERR_UNSUPPORTED, "row variants 1, 2 need a 2D plan");
    p->run_chunk = chunk == 0 ? 0 : std::min(chunk, p->bchunk);
    p->col_variant = col_variant;
    p->row_variant = row_variant;
    return PCE_OK;
}

extern "C" pce_status pce_plan_tuning(pce_plan_t p, int* chunk, int* col_variant, int* row_variant,
                                      double* ms_per_apply) {
    if (!p) return fail(PCE_ERR_INVALID, "plan is NULL");
    if (chunk) *chunk = p->run_chunk > 0 ? std::min(p->run_chunk, p->bchunk) : p->bchunk;
    if (col_variant) *col_variant = p->col_variant;
    if (row_variant) *row_variant = p->row_variant;
    if (ms_per_apply) *ms_per_apply = p->tuned_ms;
    return PCE_OK;
}

extern "C" int pce_plan_tuning_log(pce_plan_t p, int max_entries, int* chunk, int* col_variant,
                                   int* row_variant, double* ms_per_apply) {
    if (!p) return 0;
    const int n = (int)(p->tune_log.size() / 4);
    for (int i = 0; i < std::min(n, max_entries); ++i) {
        if (chunk) chunk[i] = (int)p->tune_log[4 * i];
        if (col_variant) col_variant[i] = (int)p->tune_log[4 * i + 1];
        if (row_variant) row_variant[i] = (int)p->tune_log[4 * i + 2];
        if (ms_per_apply) ms_per_apply[i] = p->tune_log[4 * i + 3];
    }
    return n;
}

// ------------------------------------------------------ batch-level tuning

extern "C" pce_status pce_batch_autotune(pce_batch_t b, void* stream) {
    if (!b) return fail(PCE_ERR_INVALID, "batch is NULL");
    int dev = 0;
    PCE_BCK(cudaGetDevice(&dev));
    if (dev != b->device) return fail(PCE_ERR_INVALID, "batch belongs to device %d, current is %d", b->device, dev);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    void* flush = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const size_t flush_bytes = 192ull << 20;
    auto cleanup = [&]() {
        if (flush) cudaFree(flush);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
    };
    cudaError_t e = cudaMalloc(&flush, flush_bytes);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) {
        cleanup();
        return fail(PCE_ERR_CUDA, "batch autotune set-up: %s", cudaGetErrorString(e));
    }
    const int pol[] = {-1, 0, 1, 2};
    double best = 1e300;
    int best_c = -1, best_r = -1;
    b->tune_log.clear();
    pce_status st = PCE_OK;
    for (int cp : pol) {
        for (int rp : pol) {
            for (size_t i = 0; i < b->scr.size(); ++i) {
                b->scr[i].col_variant = cp;
                b->scr[i].row_variant = rp;
            }
            b->drop_graph();
            float tmin = 1e30f;
            for (int rep = 0; rep < 4 && st == PCE_OK; ++rep) {   // rep 0 captures and warms up
                e = cudaMemsetAsync(flush, rep, flush_bytes, s);
                if (e == cudaSuccess) e = cudaEventRecord(e0, s);
                if (e != cudaSuccess) break;
                if ((st = pce_batch_launch(b, stream))) break;
                e = cudaEventRecord(e1, s);
                if (e == cudaSuccess) e = cudaEventSynchronize(e1);
                float ms = 0.f;
                if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
                if (e != cudaSuccess) break;
                if (rep > 0) tmin = std::min(tmin, ms);
            }
            if (st == PCE_OK && e != cudaSuccess) st = fail(PCE_ERR_CUDA, "batch autotune timing: %s", cudaGetErrorString(e));
            if (st) break;
            b->tune_log.insert(b->tune_log.end(), {(double)cp, (double)rp, (double)tmin});
            if (tmin < best) {
                best = tmin;
                best_c = cp;
                best_r = rp;
            }
        }
        if (st) break;
    }
    cleanup();
    if (st) {
        best_c = best_r = -1;
    }
    for (size_t i = 0; i < b->scr.size(); ++i) {
        b->scr[i].col_variant = best_c;
        b->scr[i].row_variant = best_r;
    }
    b->col_policy = best_c;
    b->row_policy = best_r;
    b->drop_graph();
    return st;
}

extern "C" int pce_batch_tuning_log(pce_batch_t b, int max_entries, int* col_policy, int* row_policy,
                                    double* ms_per_run) {
    if (!b) return 0;
    const int n = (int)(b->tune_log.size() / 3);
    for (int i = 0; i < std::min(n, max_entries); ++i) {
        if (col_policy) col_policy[i] = (int)b->tune_log[3 * i];
        if (row_policy) row_policy[i] = (int)b->tune_log[3 * i + 1];
        if (ms_per_run) ms_per_run[i] = b->tune_log[3 * i + 2];
    }
    return n;
}

extern "C" pce_status pce_batch_set_tuning(pce_batch_t b, int col_policy, int row_policy) {
    if (!b) return fail(PCE_ERR_INVALID, "batch is NULL");
    if (col_policy < -1 || col_policy > 4 || row_policy < -1 || row_policy > 2)
        return fail(PCE_ERR_INVALID, "column policy must be -1..4 and row policy -1..2 (got %d, %d)", col_policy,
                    row_policy);
    for (size_t i = 0; i < b->scr.size(); ++i) {
        b->scr[i].col_variant = col_policy;
        b->scr[i].row_variant = row_policy;
    }
    b->col_policy = col_policy;
    b->row_policy = row_policy;
    b->drop_graph();
    return PCE_OK;
}

extern "C" pce_status pce_batch_tuning(pce_batch_t b, int* col_policy, int* row_policy) {
    if (!b) return fail(PCE_ERR_INVALID, "batch is NULL");
    if (col_policy) *col_policy = b->col_policy;
    if (row_policy) *row_policy = b->row_policy;
    return PCE_OK;
}
