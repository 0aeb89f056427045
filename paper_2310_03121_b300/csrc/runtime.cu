// Process-wide runtime pieces: thread-local error messages, the device
// allocator hook, launch counting and per-kernel CUDA-event timing.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <set>
#include <utility>
#include <string>
#include <vector>

#include "engine.cuh"
#include "kernels.cuh"

namespace mlp {

// ------------------------------------------------------------------ errors
static thread_local std::string g_err;

int set_error(int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}
const char* last_error() { return g_err.c_str(); }
void clear_error() { g_err.clear(); }

int cuda_error(cudaError_t e, const char* where) {
    return set_error(-5, "%s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
}

// ------------------------------------------------------------------ allocator
static AllocFn g_alloc = nullptr;
static FreeFn g_free = nullptr;
static void* g_alloc_ctx = nullptr;
static std::atomic<long long> g_fail_after{-1};   // fault injection: fail the Nth allocation from now

void set_allocator(AllocFn a, FreeFn f, void* ctx) {
    g_alloc = a;
    g_free = f;
    g_alloc_ctx = ctx;
}

void set_alloc_failure(long long after) { g_fail_after = after; }

void* dev_alloc(size_t bytes) {
    long long fa = g_fail_after.load();
    if (fa >= 0) {
        if (fa == 0) {
            g_fail_after = -1;
            return nullptr;
        }
        g_fail_after = fa - 1;
    }
    if (bytes == 0) bytes = 256;
    if (g_alloc) return g_alloc(bytes, g_alloc_ctx);
    void* p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void* p) {
    if (!p) return;
    if (g_free) {
        g_free(p, g_alloc_ctx);
        return;
    }
    cudaFree(p);
}

// ------------------------------------------------------------------ launches / profiling
static std::atomic<long long> g_launches{0};
static std::atomic<int> g_profile{0};

struct PendingTiming {
    const char* name;
    cudaEvent_t a, b;
};
struct ProfState {
    std::mutex mu;
    std::vector<cudaEvent_t> pool;
    std::vector<PendingTiming> pending;
    std::map<std::string, std::pair<double, long long>> totals;
    std::vector<std::string> names;   // stable storage for returned names
    // open begin events per stream (launches on one stream are issued in order
    // by one host thread)
    std::map<std::pair<cudaStream_t, const char*>, cudaEvent_t> open;
};
static ProfState& prof() {
    static ProfState* p = new ProfState();
    return *p;
}

static cudaEvent_t take_event(ProfState& P) {
    if (!P.pool.empty()) {
        cudaEvent_t e = P.pool.back();
        P.pool.pop_back();
        return e;
    }
    cudaEvent_t e;
    cudaEventCreate(&e);
    return e;
}

static void resolve_locked(ProfState& P) {
    for (auto& t : P.pending) {
        cudaEventSynchronize(t.b);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        auto& slot = P.totals[t.name];
        slot.first += ms;
        slot.second += 1;
        P.pool.push_back(t.a);
        P.pool.push_back(t.b);
    }
    P.pending.clear();
}

void launch_begin(const char* name, cudaStream_t st) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    if (!g_profile.load(std::memory_order_relaxed)) return;
    ProfState& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    cudaEvent_t a = take_event(P);
    cudaEventRecord(a, st);
    P.open[{st, name}] = a;
}

void launch_end(const char* name, cudaStream_t st) {
    if (!g_profile.load(std::memory_order_relaxed)) return;
    ProfState& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    auto it = P.open.find({st, name});
    if (it == P.open.end()) return;
    cudaEvent_t b = take_event(P);
    cudaEventRecord(b, st);
    P.pending.push_back({name, it->second, b});
    P.open.erase(it);
    if (P.pending.size() > 4096) resolve_locked(P);
}

long long launch_count() { return g_launches.load(); }

int profile_enable(int on) {
    int prev = g_profile.exchange(on ? 1 : 0);
    return prev;
}

int profile_read(const char** names, double* ms, long long* launches, int cap) {
    ProfState& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    resolve_locked(P);
    P.names.clear();
    for (auto& kv : P.totals) P.names.push_back(kv.first);
    int k = 0;
    for (auto& kv : P.totals) {
        if (k < cap) {
            if (names) names[k] = P.names[k].c_str();
            if (ms) ms[k] = kv.second.first;
            if (launches) launches[k] = kv.second.second;
        }
        ++k;
    }
    return k;
}

void profile_reset() {
    ProfState& P = prof();
    std::lock_guard<std::mutex> lk(P.mu);
    resolve_locked(P);
    P.totals.clear();
}

std::mutex& once_mutex() {
    static std::mutex mu;
    return mu;
}

bool once_first(int device, const void* key) {
    static std::set<std::pair<int, const void*>> seen;
    return seen.insert({device, key}).second;
}

int sm_count() {
    static int cache[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(once_mutex());
    int& c = cache[dev & 63];
    if (c <= 0) {
        int v = 0;
        if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0) {
            cudaGetLastError();
            v = 148;
        }
        c = v;
    }
    return c;
}

}  // namespace mlp
