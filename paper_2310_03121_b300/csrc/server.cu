// Serving loop: continuous batching of energy+force requests for independent
// open-boundary molecules.
//
// Clients queue molecules with mlp_submit (never blocks, takes no lock):
// the request (one pooled heap block holding its inputs and its result
// area) gets a ticket from an atomic counter, is published in a ticket ring
// (the lookup table of mlp_poll / mlp_wait) and pushed on an intrusive
// multi-producer queue. One server thread drains that queue and owns
// `streams` slots; each slot is a reserved device workspace with its own
// CUDA stream and pinned staging. Whenever a slot is free and requests are
// waiting, the thread packs the oldest ones (up to the slot's atom and
// molecule limits, and while the bytes held by in-flight batches stay within
// the HBM budget) into one batch, copies it to the device and enqueues the
// evaluation; batches on different slots overlap on the GPU while the next
// one is being packed. Completion is detected with CUDA events; results are
// written into their requests, which are then marked done and waiters woken.
// Energies are reduced per molecule in a fixed order, so a molecule's energy
// does not depend on the batch it was packed into (forces agree to FP64
// atomic rounding).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "../../include/mlp.h"
#include "engine.cuh"

using namespace mlp;

namespace {

using Clock = std::chrono::steady_clock;

inline int64_t now_ns() {
    return std::chrono::duration_cast<std::chrono::nanoseconds>(Clock::now().time_since_epoch()).count();
}
inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// One heap block per request: header, inputs (xyz, species) and the result
// area (forces). Blocks come in power-of-two atom capacities (2^cls).
struct Request {
    std::atomic<Request*> next;   // link of the submission queue
    mlp_ticket id;
    int n;
    int cls;
    int status;
    std::atomic<bool> done;       // results written (release) / readable (acquire)
    int64_t t_submit;
    double E;
    double* xyz() { return reinterpret_cast<double*>(this + 1); }
    float* F() { return reinterpret_cast<float*>(xyz() + 3 * ((size_t)1 << cls)); }
    int8_t* species() { return reinterpret_cast<int8_t*>(F() + 3 * ((size_t)1 << cls)); }
    static size_t bytes(int cls) { return sizeof(Request) + 37 * ((size_t)1 << cls); }
};
// Blocks are carved on 256 bytes and hold at least 8 atoms, so with a header
// of a multiple of 16 bytes every array of a block starts on 16 bytes (the
// serving kernels move them in 16-byte words).
static_assert(sizeof(Request) % 16 == 0, "request header keeps the block's arrays 16-byte aligned");

// Request blocks live in page-locked host slabs (the serving kernels read a
// request's inputs and write its results through their unified addresses,
// so no host thread copies request data). Free blocks are kept per capacity
// class in 8 shards picked by the calling thread, so that concurrent clients
// rarely share a lock; slabs are returned only when the server is destroyed
// (a serving process in steady state allocates and page-faults no memory).
struct RequestPool {
    static constexpr int kShards = 8;
    static constexpr size_t kSlab = 8u << 20;
    struct alignas(64) Shard {
        std::mutex mu;
        std::vector<Request*> free_[32];
    };
    Shard shards[kShards];
    std::mutex slab_mu;
    std::vector<void*> slabs;
    int device = 0;   // the server's device, current while a slab is allocated
    char* cur = nullptr;
    size_t left = 0;
    void* carve(size_t bytes) {
        bytes = (bytes + 255) / 256 * 256;
        std::lock_guard<std::mutex> lk(slab_mu);
        if (bytes > left) {
            const size_t sz = bytes > kSlab ? bytes : kSlab;
            void* p = nullptr;
            int prev = 0;
            cudaGetDevice(&prev);
            if (prev != device) cudaSetDevice(device);
            const cudaError_t e = cudaHostAlloc(&p, sz, cudaHostAllocPortable);
            if (prev != device) cudaSetDevice(prev);
            if (e != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            slabs.push_back(p);
            cur = static_cast<char*>(p);
            left = sz;
        }
        void* p = cur;
        cur += bytes;
        left -= bytes;
        return p;
    }
    static int shard_of_thread() {
        static thread_local int s = (int)(std::hash<std::thread::id>()(std::this_thread::get_id()) % kShards);
        return s;
    }
    Request* get(int n) {
        int cls = 3;
        while (((int64_t)1 << cls) < n) ++cls;
        Request* r = nullptr;
        Shard& sh = shards[shard_of_thread()];
        {
            std::lock_guard<std::mutex> lk(sh.mu);
            if (!sh.free_[cls].empty()) {
                r = sh.free_[cls].back();
                sh.free_[cls].pop_back();
            }
        }
        if (!r) {
            void* p = carve(Request::bytes(cls));
            if (!p) return nullptr;
            r = new (p) Request();
        }
        r->n = n;
        r->cls = cls;
        r->status = MLP_OK;
        r->done.store(false, std::memory_order_relaxed);
        r->E = 0.0;
        return r;
    }
    void put(Request* r) {
        Shard& sh = shards[shard_of_thread()];
        std::lock_guard<std::mutex> lk(sh.mu);
        sh.free_[r->cls].push_back(r);
    }
    ~RequestPool() {
        for (void* p : slabs) cudaFreeHost(p);
    }
};

// Intrusive multi-producer / single-consumer FIFO (a stub node and an
// exchanged tail): push is wait-free for any number of clients, pop is run
// by the server thread only.
struct SubmitQueue {
    Request stub_;
    std::atomic<Request*> tail{&stub_};
    Request* head = &stub_;
    SubmitQueue() { stub_.next.store(nullptr, std::memory_order_relaxed); }
    void push(Request* r) {
        r->next.store(nullptr, std::memory_order_relaxed);
        Request* prev = tail.exchange(r, std::memory_order_acq_rel);
        prev->next.store(r, std::memory_order_release);
    }
    Request* pop() {
        Request* h = head;
        Request* nx = h->next.load(std::memory_order_acquire);
        if (h == &stub_) {
            if (!nx) return nullptr;
            head = nx;
            h = nx;
            nx = nx->next.load(std::memory_order_acquire);
        }
        if (nx) {
            head = nx;
            return h;
        }
        if (h != tail.load(std::memory_order_acquire)) return nullptr;   // a push is half done: later
        push(&stub_);
        nx = h->next.load(std::memory_order_acquire);
        if (nx) {
            head = nx;
            return h;
        }
        return nullptr;
    }
};

struct Slot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaStream_t io = nullptr;                  // gather / scatter, highest priority
    cudaEvent_t done = nullptr;
    cudaEvent_t in_ready = nullptr, out_ready = nullptr;
    void* dev_block = nullptr;
    void* host_block = nullptr;
    int *d_mol_start = nullptr, *h_mol_start = nullptr;
    MolRef *d_refs = nullptr, *h_refs = nullptr;   // per molecule: its request's input and result areas
    int8_t* d_species = nullptr;
    double* d_xyz = nullptr;
    double* d_E = nullptr;
    float* d_F = nullptr;
    bool busy = false;
    size_t footprint = 0;
    int n_atoms = 0, n_mols = 0;
    std::vector<Request*> reqs;
};

}  // namespace

struct mlp_server {
    mlp_server_opts o{};
    const mlp_weights* w = nullptr;
    int device = 0;
    std::vector<Slot> slots;
    size_t bytes_per_atom = 0;
    // ticket ring: ticket t lives in entry t & ring_mask until taken; a
    // submit whose entry is still held by an uncollected request is refused
    std::vector<std::atomic<Request*>> ring;
    uint64_t ring_mask = 0;
    RequestPool pool;
    SubmitQueue sq;
    std::deque<Request*> pending;   // drained from sq, not yet batched (server thread only)
    int64_t pending_atoms = 0;      // atoms in pending
    int64_t min_batch = 0;          // batching under load (from the options)
    int64_t max_wait_ns = 0;
    alignas(64) std::atomic<uint64_t> next_id{1};
    alignas(64) std::atomic<int64_t> queued{0};   // pushed on sq and not yet drained
    alignas(64) std::atomic<bool> sleeping{false};
    std::atomic<bool> stop{false};
    std::atomic<int64_t> submitted{0};
    // guarded by mu: statistics, latencies, in-flight bytes; cv_done waiters
    alignas(64) std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::vector<int64_t> latencies;
    int64_t inflight_bytes = 0;
    mlp_server_stats st{};
    std::thread th;

    bool init_tables() {
        size_t r = 8;
        while (r < (size_t)o.queue_capacity) r <<= 1;
        try {
            ring = std::vector<std::atomic<Request*>>(r);
        } catch (...) {
            return false;
        }
        for (auto& e : ring) e.store(nullptr, std::memory_order_relaxed);
        ring_mask = r - 1;
        return true;
    }
    Request* lookup(mlp_ticket t) {
        if (t == 0) return nullptr;
        Request* r = ring[t & ring_mask].load(std::memory_order_acquire);
        return (r && r->id == t) ? r : nullptr;
    }
};

struct mlp_weights;   // defined in api.cu; the server only passes it through
namespace mlp {
const DevWeights& weights_of(const mlp_weights* w);
}

namespace {

void slot_destroy(Slot& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    if (s.io) cudaStreamSynchronize(s.io);
    workspace_destroy(s.ws);
    dev_free(s.dev_block);
    if (s.host_block) cudaFreeHost(s.host_block);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.io) cudaStreamDestroy(s.io);
    if (s.done) cudaEventDestroy(s.done);
    if (s.in_ready) cudaEventDestroy(s.in_ready);
    if (s.out_ready) cudaEventDestroy(s.out_ready);
    s = Slot();
}

int slot_create(Slot& s, const mlp_server_opts& o, int nets) {
    int rc = workspace_create(s.ws, o.max_batch_atoms, o.max_batch_mols, o.precision, false, kDefaultNbrCap, 0, nets);
    if (rc) return rc;
    const size_t A = o.max_batch_atoms, M = o.max_batch_mols;
    const size_t dev = al256(4 * (M + 1)) + al256(sizeof(MolRef) * M) + al256(A) + al256(24 * A) + al256(8 * M) +
                       al256(12 * A);
    s.dev_block = dev_alloc(dev);
    if (!s.dev_block) return set_error(MLP_ENOMEM, "device allocation of a serving slot failed");
    cudaError_t e;
    const size_t host = al256(4 * (M + 1)) + al256(sizeof(MolRef) * M);
    if ((e = cudaMallocHost(&s.host_block, host)) != cudaSuccess) return cuda_error(e, "cudaMallocHost(slot)");
    if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_error(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s.in_ready, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s.out_ready, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_error(e, "cudaEventCreate");
    // The gather and scatter kernels read and write the requests' page-locked
    // host blocks over PCIe: on a stream of the highest priority their blocks
    // are scheduled ahead of the other slot's compute blocks, so the transfers
    // overlap that batch's kernels instead of queueing behind them.
    int lo_prio = 0, hi_prio = 0;
    cudaDeviceGetStreamPriorityRange(&lo_prio, &hi_prio);
    if ((e = cudaStreamCreateWithPriority(&s.io, cudaStreamNonBlocking, hi_prio)) != cudaSuccess)
        return cuda_error(e, "cudaStreamCreateWithPriority");
    char* d = static_cast<char*>(s.dev_block);
    char* h = static_cast<char*>(s.host_block);
    s.d_mol_start = reinterpret_cast<int*>(d);
    s.h_mol_start = reinterpret_cast<int*>(h);
    d += al256(4 * (M + 1));
    h += al256(4 * (M + 1));
    s.d_refs = reinterpret_cast<MolRef*>(d);
    s.h_refs = reinterpret_cast<MolRef*>(h);
    d += al256(sizeof(MolRef) * M);
    s.d_species = reinterpret_cast<int8_t*>(d);
    d += al256(A);
    s.d_xyz = reinterpret_cast<double*>(d);
    d += al256(24 * A);
    s.d_E = reinterpret_cast<double*>(d);
    d += al256(8 * M);
    s.d_F = reinterpret_cast<float*>(d);
    return MLP_OK;
}

size_t slot_bytes(const mlp_server_opts& o, int nets) {
    const size_t A = o.max_batch_atoms, M = o.max_batch_mols;
    return workspace_bytes(o.max_batch_atoms, o.max_batch_mols, o.precision, false, kDefaultNbrCap, 0, nets) +
           al256(4 * (M + 1)) + al256(sizeof(MolRef) * M) + al256(A) + al256(24 * A) + al256(8 * M) + al256(12 * A);
}

// Enqueues one batch: a table of the molecules' host blocks and offsets goes
// to the device; a gather kernel reads the inputs from the blocks, the
// evaluation runs, a scatter kernel writes energies and forces back.
int launch_slot(mlp_server* S, Slot& s) {
    int off = 0;
    s.h_mol_start[0] = 0;
    for (size_t m = 0; m < s.reqs.size(); ++m) {
        Request* r = s.reqs[m];
        s.h_refs[m] = MolRef{r->xyz(), r->species(), r->F(), &r->E};
        off += r->n;
        s.h_mol_start[m + 1] = off;
    }
    s.n_atoms = off;
    s.n_mols = (int)s.reqs.size();
    cudaStream_t st = s.stream, io = s.io;
    cudaMemcpyAsync(s.d_mol_start, s.h_mol_start, 4 * (size_t)(s.n_mols + 1), cudaMemcpyHostToDevice, io);
    cudaMemcpyAsync(s.d_refs, s.h_refs, sizeof(MolRef) * (size_t)s.n_mols, cudaMemcpyHostToDevice, io);
    launch_gather_batch(io, s.n_mols, s.d_refs, s.d_mol_start, s.d_xyz, s.d_species);
    cudaEventRecord(s.in_ready, io);
    cudaStreamWaitEvent(st, s.in_ready, 0);
    EvalSpec sp;
    sp.n_atoms = s.n_atoms;
    sp.n_mols = s.n_mols;
    sp.d_mol_start = s.d_mol_start;
    sp.d_species = s.d_species;
    sp.d_xyz = s.d_xyz;
    sp.r_list = kRcRad;
    sp.d_E = s.d_E;
    sp.d_F = s.d_F;
    int rc = enqueue_eval(s.ws, weights_of(S->w), sp, st);
    if (rc) return rc;
    cudaEventRecord(s.out_ready, st);
    cudaStreamWaitEvent(io, s.out_ready, 0);
    launch_scatter_results(io, s.n_mols, s.d_refs, s.d_mol_start, s.d_E, s.d_F);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "serving kernels");
    e = cudaEventRecord(s.done, io);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    return MLP_OK;
}

void finish_slot(mlp_server* S, Slot& s, int status) {
    if (status == MLP_OK) status = check_counters(s.ws);
    const int64_t t = now_ns();
    // energies and forces are already in the requests (scatter kernel)
    std::vector<int64_t> lat;
    lat.reserve(s.reqs.size());
    for (Request* r : s.reqs) {
        r->status = status;
        lat.push_back(t - r->t_submit);
        r->done.store(true, std::memory_order_release);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->latencies.insert(S->latencies.end(), lat.begin(), lat.end());
        if (S->latencies.size() > (1u << 22))
            S->latencies.erase(S->latencies.begin(), S->latencies.begin() + (1 << 20));
        S->st.completed += (int64_t)s.reqs.size();
        S->st.batches += 1;
        S->st.atoms += s.n_atoms;
        S->inflight_bytes -= (int64_t)s.footprint;
    }
    s.reqs.clear();
    s.busy = false;
    S->cv_done.notify_all();
}

// The serving thread: drains the submission queue, polls completions and
// forms batches; it takes the lock only for statistics and for sleeping.
void server_loop(mlp_server* S) {
    cudaSetDevice(S->device);
    std::vector<Request*> batch;
    int idle = 0;
    for (;;) {
        bool progressed = false, any_busy = false;
        int64_t drained = 0;
        while (Request* r = S->sq.pop()) {
            S->pending.push_back(r);
            S->pending_atoms += r->n;
            ++drained;
        }
        if (drained) S->queued.fetch_sub(drained);
        Slot* free_slot = nullptr;
        for (Slot& s : S->slots) {
            if (s.busy) {
                cudaError_t q = cudaEventQuery(s.done);
                if (q != cudaErrorNotReady) {
                    finish_slot(S, s, q == cudaSuccess ? MLP_OK : cuda_error(q, "batch"));
                    progressed = true;
                }
            }
            if (s.busy)
                any_busy = true;
            else if (!free_slot)
                free_slot = &s;
        }
        // under load (another batch on the device) wait for a batch worth its
        // fixed cost, or until the oldest request has waited max_wait_us
        bool launch = free_slot && !S->pending.empty();
        if (launch && any_busy && S->pending_atoms < S->min_batch &&
            (int64_t)S->pending.size() < S->o.max_batch_mols)
            launch = now_ns() - S->pending.front()->t_submit >= S->max_wait_ns;
        if (launch) {
            // admission: oldest first, within the slot's limits and the HBM budget
            int atoms = 0;
            batch.clear();
            int64_t inflight;
            {
                std::lock_guard<std::mutex> lk(S->mu);
                inflight = S->inflight_bytes;
            }
            while (!S->pending.empty()) {
                Request* r = S->pending.front();
                if (atoms + r->n > S->o.max_batch_atoms || (int)batch.size() >= S->o.max_batch_mols) break;
                int64_t fp = (int64_t)S->bytes_per_atom * (atoms + r->n);
                if (inflight + fp > S->o.budget_bytes && !batch.empty()) break;
                if (inflight + fp > S->o.budget_bytes && any_busy) break;   // wait for memory
                batch.push_back(r);
                atoms += r->n;
                S->pending_atoms -= r->n;
                S->pending.pop_front();
            }
            if (!batch.empty()) {
                free_slot->footprint = S->bytes_per_atom * (size_t)atoms;
                {
                    std::lock_guard<std::mutex> lk(S->mu);
                    S->inflight_bytes += (int64_t)free_slot->footprint;
                    S->st.peak_inflight_bytes = std::max(S->st.peak_inflight_bytes, S->inflight_bytes);
                }
                free_slot->reqs = batch;
                free_slot->busy = true;
                int rc = launch_slot(S, *free_slot);
                if (rc) {
                    cudaStreamSynchronize(free_slot->stream);
                    cudaStreamSynchronize(free_slot->io);
                    finish_slot(S, *free_slot, rc);
                }
                idle = 0;
                continue;
            }
        }
        if (progressed || drained) {
            idle = 0;
            continue;
        }
        if (any_busy || !S->pending.empty()) {
            // batches in flight: poll again soon (yield first, then short sleeps)
            if (++idle < 64)
                std::this_thread::yield();
            else
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            continue;
        }
        if (S->stop.load() && S->queued.load() == 0) return;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            S->sleeping.store(true);
            if (S->queued.load() == 0 && !S->stop.load()) S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            S->sleeping.store(false);
        }
        idle = 0;
    }
}

}  // namespace

extern "C" {

void mlp_server_opts_default(mlp_server_opts* o) {
    if (!o) return;
    o->precision = MLP_BF16;
    o->max_batch_atoms = 131072;
    o->max_batch_mols = 4096;
    o->max_atoms_per_mol = 256;
    o->streams = 3;
    o->queue_capacity = 65536;
    o->budget_bytes = 40LL * 1000 * 1000 * 1000;
    o->min_batch_atoms = 16384;
    o->max_wait_us = 500;
}

int mlp_server_create(const mlp_weights* w, const mlp_server_opts* opts, mlp_server** out) {
    clear_error();
    if (!out) return set_error(MLP_EINVAL, "NULL out");
    *out = nullptr;
    if (!w) return set_error(MLP_EINVAL, "NULL weights");
    mlp_server_opts o;
    mlp_server_opts_default(&o);
    if (opts) o = *opts;
    if (o.precision < MLP_FP32 || o.precision > MLP_BF16_1PASS) return set_error(MLP_EINVAL, "unknown precision");
    if (o.precision != MLP_FP32 && !mlp_tc_available()) return set_error(MLP_EINVAL, "BF16 network not available");
    if (o.max_batch_atoms <= 0 || o.max_batch_mols <= 0 || o.max_atoms_per_mol <= 0 ||
        o.max_atoms_per_mol > o.max_batch_atoms || o.streams <= 0 || o.streams > 16 || o.queue_capacity <= 0 ||
        o.budget_bytes <= 0 || o.max_wait_us < 0)
        return set_error(MLP_EINVAL, "bad server options");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return set_error(MLP_ECUDA, "no usable CUDA device");
    }
    init_constants_for_current_device();
    const size_t sb = slot_bytes(o, weights_of(w).n_nets);
    long long fit = o.budget_bytes / (long long)sb;
    if (fit < 1)
        return set_error(MLP_ENOMEM, "budget of %lld bytes holds no slot of %zu bytes", (long long)o.budget_bytes, sb);
    if (fit < o.streams) o.streams = (int)fit;
    mlp_server* S = new (std::nothrow) mlp_server();
    if (!S) return set_error(MLP_ENOMEM, "host allocation failed");
    S->o = o;
    S->min_batch = std::min<int64_t>(std::max(0, o.min_batch_atoms), o.max_batch_atoms);
    S->max_wait_ns = (int64_t)std::max(0, o.max_wait_us) * 1000;
    S->w = w;
    cudaGetDevice(&S->device);
    S->pool.device = S->device;
    S->bytes_per_atom = (sb + o.max_batch_atoms - 1) / o.max_batch_atoms;
    if (!S->init_tables()) {
        delete S;
        return set_error(MLP_ENOMEM, "host allocation failed");
    }
    S->slots.resize(o.streams);
    for (Slot& s : S->slots) {
        int rc = slot_create(s, o, weights_of(w).n_nets);
        if (rc) {
            for (Slot& t : S->slots) slot_destroy(t);
            delete S;
            return rc;
        }
    }
    try {
        S->th = std::thread(server_loop, S);
    } catch (...) {
        for (Slot& t : S->slots) slot_destroy(t);
        delete S;
        return set_error(MLP_ENOMEM, "could not start the server thread");
    }
    *out = S;
    return MLP_OK;
}

void mlp_server_destroy(mlp_server* S) {
    if (!S) return;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop.store(true);
    }
    S->cv_work.notify_all();
    if (S->th.joinable()) S->th.join();
    for (Slot& s : S->slots) slot_destroy(s);
    for (auto& e : S->ring) {   // queued, in flight or not collected
        Request* r = e.load();
        if (r) S->pool.put(r);
    }
    delete S;
}

int mlp_submit(mlp_server* S, int32_t n, const int8_t* species, const double* coords, mlp_ticket* out) {
    clear_error();
    if (!S || !species || !coords || !out) return set_error(MLP_EINVAL, "NULL argument");
    if (n <= 0 || n > S->o.max_atoms_per_mol)
        return set_error(MLP_EINVAL, "molecule of %d atoms outside [1, %d]", n, S->o.max_atoms_per_mol);
    // branch-free scans (vectorizable); the failing index is looked up only on error
    int bad = 0;
    for (int i = 0; i < n; ++i) bad |= (species[i] < 0) | (species[i] >= kNSpecies);
    if (bad)
        for (int i = 0; i < n; ++i)
            if (species[i] < 0 || species[i] >= kNSpecies)
                return set_error(MLP_EINVAL, "species[%d] = %d", i, species[i]);
    uint64_t nonfinite = 0;
    for (int q = 0; q < 3 * n; ++q) {
        uint64_t b;
        std::memcpy(&b, coords + q, 8);
        nonfinite |= (uint64_t)((b & 0x7ff0000000000000ull) == 0x7ff0000000000000ull);
    }
    if (nonfinite) return set_error(MLP_EINVAL, "non-finite coordinate");
    Request* r = S->pool.get(n);
    if (!r) return set_error(MLP_ENOMEM, "host allocation failed");
    std::memcpy(r->species(), species, n);
    std::memcpy(r->xyz(), coords, 24 * (size_t)n);
    r->t_submit = now_ns();
    const mlp_ticket t = S->next_id.fetch_add(1);
    r->id = t;
    Request* expected = nullptr;
    if (!S->ring[t & S->ring_mask].compare_exchange_strong(expected, r, std::memory_order_acq_rel)) {
        S->pool.put(r);
        return set_error(MLP_EAGAIN, "server full: %d requests outstanding", S->o.queue_capacity);
    }
    S->submitted.fetch_add(1, std::memory_order_relaxed);
    S->sq.push(r);
    S->queued.fetch_add(1);
    if (S->sleeping.load()) {
        std::lock_guard<std::mutex> lk(S->mu);
        S->cv_work.notify_one();
    }
    *out = t;
    return MLP_OK;
}

// Takes a done request out of the ring (only one caller can); MLP_ENOTFOUND
// if another caller took the ticket first.
static int take_result(mlp_server* S, mlp_ticket t, Request* r, double* energy, float* forces) {
    Request* expected = r;
    if (!S->ring[t & S->ring_mask].compare_exchange_strong(expected, nullptr, std::memory_order_acq_rel))
        return set_error(MLP_ENOTFOUND, "unknown ticket %llu", (unsigned long long)t);
    if (r->id != t) {   // the block was recycled under another ticket: not ours
        S->ring[t & S->ring_mask].store(r, std::memory_order_release);
        return set_error(MLP_ENOTFOUND, "unknown ticket %llu", (unsigned long long)t);
    }
    const int status = r->status;
    if (status == MLP_OK) {
        if (energy) *energy = r->E;
        if (forces) std::memcpy(forces, r->F(), 12 * (size_t)r->n);
    }
    S->pool.put(r);
    if (status) set_error(status, "request failed");
    return status;
}

int mlp_poll(mlp_server* S, mlp_ticket t, double* energy, float* forces) {
    clear_error();
    if (!S) return set_error(MLP_EINVAL, "NULL server");
    Request* r = S->lookup(t);
    if (!r) return set_error(MLP_ENOTFOUND, "unknown ticket %llu", (unsigned long long)t);
    if (!r->done.load(std::memory_order_acquire)) return MLP_PENDING;
    return take_result(S, t, r, energy, forces);
}

int mlp_wait(mlp_server* S, mlp_ticket t, int64_t timeout_ns, double* energy, float* forces) {
    clear_error();
    if (!S) return set_error(MLP_EINVAL, "NULL server");
    const auto deadline = Clock::now() + std::chrono::nanoseconds(timeout_ns < 0 ? 0 : timeout_ns);
    bool timed_out = false;
    for (;;) {
        Request* r = S->lookup(t);
        if (!r) return set_error(MLP_ENOTFOUND, "unknown ticket %llu", (unsigned long long)t);
        if (r->done.load(std::memory_order_acquire)) return take_result(S, t, r, energy, forces);
        if (timed_out)
            return set_error(MLP_ETIMEDOUT, "ticket %llu not done within %lld ns", (unsigned long long)t,
                             (long long)timeout_ns);
        std::unique_lock<std::mutex> lk(S->mu);
        // done is set before finish_slot takes the lock to notify: checked again under it
        if (r->done.load(std::memory_order_acquire) || S->lookup(t) != r) continue;
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) timed_out = true;
    }
}

int mlp_server_get_stats(mlp_server* S, mlp_server_stats* out) {
    clear_error();
    if (!S || !out) return set_error(MLP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->submitted = S->submitted.load();
    out->inflight_bytes = S->inflight_bytes;
    out->mean_batch_atoms = S->st.batches ? (double)S->st.atoms / (double)S->st.batches : 0.0;
    out->slot_bytes = (int64_t)slot_bytes(S->o, weights_of(S->w).n_nets);
    out->slots = (int32_t)S->slots.size();
    return MLP_OK;
}

int mlp_server_latencies(mlp_server* S, int64_t* out, int cap) {
    clear_error();
    if (!S) return set_error(MLP_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    int k = (int)std::min<size_t>(S->latencies.size(), cap > 0 ? (size_t)cap : 0);
    if (out && k > 0) std::memcpy(out, S->latencies.data(), 8 * (size_t)k);
    S->latencies.clear();
    return k;
}

int mlp_server_replay_clients(mlp_server* S, int32_t n_req, const int64_t* arrival_ns, const int32_t* mol_start,
                              const int8_t* species, const double* coords, double* energies, float* forces,
                              int32_t clients, int64_t* wall_ns) {
    clear_error();
    if (!S || !arrival_ns || !mol_start || !species || !coords || !energies || n_req <= 0 || clients < 1 ||
        clients > 64)
        return set_error(MLP_EINVAL, "bad replay arguments");
    std::vector<mlp_ticket> tickets(n_req);
    std::atomic<int> status{MLP_OK};
    const int64_t t0 = now_ns();
    // client c submits requests c, c + clients, ... at their arrival times,
    // then collects the results of its own requests
    auto client = [&](int c) {
        for (int r = c; r < n_req && status.load() == MLP_OK; r += clients) {
            const int64_t due = t0 + arrival_ns[r];
            for (;;) {
                int64_t now = now_ns();
                if (now >= due) break;
                if (due - now > 200000)
                    std::this_thread::sleep_for(std::chrono::nanoseconds(due - now - 100000));
                else
                    std::this_thread::yield();
            }
            const int a = mol_start[r], b = mol_start[r + 1];
            for (;;) {
                int rc = mlp_submit(S, b - a, species + a, coords + 3 * (size_t)a, &tickets[r]);
                if (rc == MLP_OK) break;
                if (rc != MLP_EAGAIN) {
                    status.store(rc);
                    return;
                }
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
        for (int r = c; r < n_req && status.load() == MLP_OK; r += clients) {
            const int a = mol_start[r];
            int rc = mlp_wait(S, tickets[r], 600LL * 1000000000LL, &energies[r], forces ? forces + 3 * (size_t)a : nullptr);
            if (rc) status.store(rc);
        }
    };
    std::vector<std::thread> th;
    try {
        for (int c = 1; c < clients; ++c) th.emplace_back(client, c);
    } catch (...) {
        status.store(MLP_ENOMEM);
    }
    client(0);
    for (auto& t : th) t.join();
    if (status.load() != MLP_OK) return set_error(status.load(), "replay: a request failed or could not be submitted");
    if (wall_ns) *wall_ns = now_ns() - t0;
    return MLP_OK;
}

int mlp_server_replay(mlp_server* S, int32_t n_req, const int64_t* arrival_ns, const int32_t* mol_start,
                      const int8_t* species, const double* coords, double* energies, float* forces,
                      int64_t* wall_ns) {
    return mlp_server_replay_clients(S, n_req, arrival_ns, mol_start, species, coords, energies, forces, 1, wall_ns);
}

}  // extern "C"
