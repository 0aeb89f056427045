// Serving loop: continuous batching of energy+force requests for independent
// open-boundary molecules.
//
// Clients queue molecules with mlp_submit (never blocks). One server thread
// owns `streams` slots; each slot is a reserved device workspace with its own
// CUDA stream and pinned staging. Whenever a slot is free and requests are
// queued, the thread packs the oldest requests (up to the slot's atom and
// molecule limits, and while the bytes held by in-flight batches stay within
// the HBM budget) into one batch, copies it to the device and enqueues the
// evaluation; batches on different slots overlap on the GPU while the next
// one is being packed. Completion is detected with CUDA events; results are
// scattered to their tickets and waiters are woken. Energies are reduced per
// molecule in a fixed order, so a molecule's energy does not depend on the
// batch it was packed into (forces agree to FP64 atomic rounding).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
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
// area (forces), written by the server thread before the request is marked
// done under the lock.
struct Request {
    mlp_ticket id;
    int n;
    int status;
    bool done;
    int64_t t_submit;
    double E;
    double* xyz() { return reinterpret_cast<double*>(this + 1); }
    float* F() { return reinterpret_cast<float*>(xyz() + 3 * (size_t)n); }
    int8_t* species() { return reinterpret_cast<int8_t*>(F() + 3 * (size_t)n); }
    static Request* make(int n) {
        void* p = std::malloc(sizeof(Request) + 24 * (size_t)n + 12 * (size_t)n + (size_t)n);
        if (!p) return nullptr;
        Request* r = static_cast<Request*>(p);
        r->n = n;
        r->status = MLP_OK;
        r->done = false;
        r->E = 0.0;
        return r;
    }
    static void release(Request* r) { std::free(r); }
};
static_assert(sizeof(Request) % 8 == 0, "request header keeps the coordinates 8-byte aligned");

struct Slot {
    Workspace ws;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    void* dev_block = nullptr;
    void* host_block = nullptr;
    int *d_mol_start = nullptr, *h_mol_start = nullptr;
    int8_t *d_species = nullptr, *h_species = nullptr;
    double *d_xyz = nullptr, *h_xyz = nullptr;
    double *d_E = nullptr, *h_E = nullptr;
    float *d_F = nullptr, *h_F = nullptr;
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
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Request*> queue;
    std::unordered_map<mlp_ticket, Request*> results;   // submitted and not yet taken
    std::vector<int64_t> latencies;
    std::atomic<bool> stop{false};
    bool sleeping = false;              // the server thread waits for new requests (submit must wake it)
    std::atomic<int64_t> queued{0};     // requests in `queue` (read without the lock by the server loop)
    std::thread th;
    mlp_ticket next_id = 1;
    int64_t inflight_bytes = 0;
    mlp_server_stats st{};
};

struct mlp_weights;   // defined in api.cu; the server only passes it through
namespace mlp {
const DevWeights& weights_of(const mlp_weights* w);
}

namespace {

void slot_destroy(Slot& s) {
    if (s.stream) cudaStreamSynchronize(s.stream);
    workspace_destroy(s.ws);
    dev_free(s.dev_block);
    if (s.host_block) cudaFreeHost(s.host_block);
    if (s.stream) cudaStreamDestroy(s.stream);
    if (s.done) cudaEventDestroy(s.done);
    s = Slot();
}

int slot_create(Slot& s, const mlp_server_opts& o) {
    int rc = workspace_create(s.ws, o.max_batch_atoms, o.max_batch_mols, o.precision, false, kDefaultNbrCap, 0);
    if (rc) return rc;
    const size_t A = o.max_batch_atoms, M = o.max_batch_mols;
    const size_t io = al256(4 * (M + 1)) + al256(A) + al256(24 * A) + al256(8 * M) + al256(12 * A);
    s.dev_block = dev_alloc(io);
    if (!s.dev_block) return set_error(MLP_ENOMEM, "device allocation of a serving slot failed");
    cudaError_t e;
    if ((e = cudaMallocHost(&s.host_block, io)) != cudaSuccess) return cuda_error(e, "cudaMallocHost(slot)");
    if ((e = cudaStreamCreateWithFlags(&s.stream, cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_error(e, "cudaStreamCreate");
    if ((e = cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming)) != cudaSuccess)
        return cuda_error(e, "cudaEventCreate");
    char* d = static_cast<char*>(s.dev_block);
    char* h = static_cast<char*>(s.host_block);
    auto carve = [&](size_t bytes, void** dp, void** hp) {
        *dp = d;
        *hp = h;
        d += al256(bytes);
        h += al256(bytes);
    };
    carve(4 * (M + 1), (void**)&s.d_mol_start, (void**)&s.h_mol_start);
    carve(A, (void**)&s.d_species, (void**)&s.h_species);
    carve(24 * A, (void**)&s.d_xyz, (void**)&s.h_xyz);
    carve(8 * M, (void**)&s.d_E, (void**)&s.h_E);
    carve(12 * A, (void**)&s.d_F, (void**)&s.h_F);
    return MLP_OK;
}

size_t slot_bytes(const mlp_server_opts& o) {
    const size_t A = o.max_batch_atoms, M = o.max_batch_mols;
    return workspace_bytes(o.max_batch_atoms, o.max_batch_mols, o.precision, false, kDefaultNbrCap, 0) +
           al256(4 * (M + 1)) + al256(A) + al256(24 * A) + al256(8 * M) + al256(12 * A);
}

// Packs slot.reqs into the slot's staging and enqueues copies + evaluation.
int launch_slot(mlp_server* S, Slot& s) {
    int off = 0;
    s.h_mol_start[0] = 0;
    for (size_t m = 0; m < s.reqs.size(); ++m) {
        Request* r = s.reqs[m];
        std::memcpy(s.h_species + off, r->species(), r->n);
        std::memcpy(s.h_xyz + 3 * (size_t)off, r->xyz(), 24 * (size_t)r->n);
        off += r->n;
        s.h_mol_start[m + 1] = off;
    }
    s.n_atoms = off;
    s.n_mols = (int)s.reqs.size();
    cudaStream_t st = s.stream;
    cudaMemcpyAsync(s.d_mol_start, s.h_mol_start, 4 * (size_t)(s.n_mols + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s.d_species, s.h_species, s.n_atoms, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(s.d_xyz, s.h_xyz, 24 * (size_t)s.n_atoms, cudaMemcpyHostToDevice, st);
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
    cudaMemcpyAsync(s.h_E, s.d_E, 8 * (size_t)s.n_mols, cudaMemcpyDeviceToHost, st);
    cudaMemcpyAsync(s.h_F, s.d_F, 12 * (size_t)s.n_atoms, cudaMemcpyDeviceToHost, st);
    cudaError_t e = cudaEventRecord(s.done, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    return MLP_OK;
}

void finish_slot(mlp_server* S, Slot& s, int status) {
    if (status == MLP_OK) status = check_counters(s.ws);
    const int64_t t = now_ns();
    // results go into the requests without the lock (nobody reads a request
    // before it is marked done); only the done flags are published under it
    std::vector<int64_t> lat;
    lat.reserve(s.reqs.size());
    int off = 0;
    for (size_t m = 0; m < s.reqs.size(); ++m) {
        Request* r = s.reqs[m];
        r->status = status;
        r->E = s.h_E[m];
        std::memcpy(r->F(), s.h_F + 3 * (size_t)off, 12 * (size_t)r->n);
        off += r->n;
        lat.push_back(t - r->t_submit);
    }
    {
        std::lock_guard<std::mutex> lk(S->mu);
        for (Request* r : s.reqs) r->done = true;
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

// The loop takes the lock only to move requests from the queue into a batch
// (and to publish completions): completions are polled and the queue length
// is read (an atomic) without it, so submitters rarely meet a held lock.
void server_loop(mlp_server* S) {
    cudaSetDevice(S->device);
    std::vector<Request*> batch;
    int idle = 0;
    for (;;) {
        bool progressed = false, any_busy = false;
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
        if (free_slot && S->queued.load(std::memory_order_acquire) > 0) {
            int atoms = 0;
            batch.clear();
            {
                std::lock_guard<std::mutex> lk(S->mu);
                // admission: oldest first, within the slot's limits and the HBM budget
                while (!S->queue.empty()) {
                    Request* r = S->queue.front();
                    if (atoms + r->n > S->o.max_batch_atoms || (int)batch.size() >= S->o.max_batch_mols) break;
                    int64_t fp = (int64_t)S->bytes_per_atom * (atoms + r->n);
                    if (S->inflight_bytes + fp > S->o.budget_bytes && !batch.empty()) break;
                    if (S->inflight_bytes + fp > S->o.budget_bytes && any_busy) break;   // wait for memory
                    batch.push_back(r);
                    atoms += r->n;
                    S->queue.pop_front();
                }
                S->queued.store((int64_t)S->queue.size(), std::memory_order_release);
                if (!batch.empty()) {
                    free_slot->footprint = S->bytes_per_atom * (size_t)atoms;
                    S->inflight_bytes += (int64_t)free_slot->footprint;
                    S->st.peak_inflight_bytes = std::max(S->st.peak_inflight_bytes, S->inflight_bytes);
                }
            }
            if (!batch.empty()) {
                free_slot->reqs = batch;
                free_slot->busy = true;
                progressed = true;
                int rc = launch_slot(S, *free_slot);
                if (rc) {
                    cudaStreamSynchronize(free_slot->stream);
                    finish_slot(S, *free_slot, rc);
                }
                continue;
            }
        }
        if (progressed) {
            idle = 0;
            continue;
        }
        if (any_busy) {
            // batches in flight: poll again soon (yield first, then short sleeps)
            if (++idle < 64)
                std::this_thread::yield();
            else
                std::this_thread::sleep_for(std::chrono::microseconds(5));
            continue;
        }
        std::unique_lock<std::mutex> lk(S->mu);
        if (S->stop.load() && S->queue.empty()) return;
        if (S->queue.empty()) {
            S->sleeping = true;
            S->cv_work.wait_for(lk, std::chrono::milliseconds(50));
            S->sleeping = false;
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
    o->streams = 2;
    o->queue_capacity = 65536;
    o->budget_bytes = 40LL * 1000 * 1000 * 1000;
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
        o.budget_bytes <= 0)
        return set_error(MLP_EINVAL, "bad server options");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return set_error(MLP_ECUDA, "no usable CUDA device");
    }
    init_constants_for_current_device();
    const size_t sb = slot_bytes(o);
    long long fit = o.budget_bytes / (long long)sb;
    if (fit < 1)
        return set_error(MLP_ENOMEM, "budget of %lld bytes holds no slot of %zu bytes", (long long)o.budget_bytes, sb);
    if (fit < o.streams) o.streams = (int)fit;
    mlp_server* S = new (std::nothrow) mlp_server();
    if (!S) return set_error(MLP_ENOMEM, "host allocation failed");
    S->o = o;
    S->w = w;
    cudaGetDevice(&S->device);
    S->bytes_per_atom = (sb + o.max_batch_atoms - 1) / o.max_batch_atoms;
    S->results.reserve(2 * (size_t)o.queue_capacity);
    S->slots.resize(o.streams);
    for (Slot& s : S->slots) {
        int rc = slot_create(s, o);
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
    for (auto& kv : S->results) Request::release(kv.second);   // queued, in flight or not taken
    delete S;
}

int mlp_submit(mlp_server* S, int32_t n, const int8_t* species, const double* coords, mlp_ticket* out) {
    clear_error();
    if (!S || !species || !coords || !out) return set_error(MLP_EINVAL, "NULL argument");
    if (n <= 0 || n > S->o.max_atoms_per_mol)
        return set_error(MLP_EINVAL, "molecule of %d atoms outside [1, %d]", n, S->o.max_atoms_per_mol);
    for (int i = 0; i < n; ++i)
        if (species[i] < 0 || species[i] >= kNSpecies) return set_error(MLP_EINVAL, "species[%d] = %d", i, species[i]);
    for (int q = 0; q < 3 * n; ++q)
        if (!std::isfinite(coords[q])) return set_error(MLP_EINVAL, "non-finite coordinate");
    Request* r = Request::make(n);
    if (!r) return set_error(MLP_ENOMEM, "host allocation failed");
    std::memcpy(r->species(), species, n);
    std::memcpy(r->xyz(), coords, 24 * (size_t)n);
    r->t_submit = now_ns();
    bool wake;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if ((int)S->queue.size() >= S->o.queue_capacity) {
            Request::release(r);
            return set_error(MLP_EAGAIN, "server queue full (%d requests)", S->o.queue_capacity);
        }
        r->id = S->next_id++;
        S->results.emplace(r->id, r);
        S->queue.push_back(r);
        S->queued.store((int64_t)S->queue.size(), std::memory_order_release);
        S->st.submitted += 1;
        *out = r->id;
        wake = S->sleeping;
    }
    if (wake) S->cv_work.notify_one();
    return MLP_OK;
}

static int take_result(mlp_server* S, std::unordered_map<mlp_ticket, Request*>::iterator it, double* energy,
                       float* forces) {
    Request* r = it->second;
    const int status = r->status;
    if (status == MLP_OK) {
        if (energy) *energy = r->E;
        if (forces) std::memcpy(forces, r->F(), 12 * (size_t)r->n);
    }
    S->results.erase(it);
    Request::release(r);
    return status;
}

int mlp_poll(mlp_server* S, mlp_ticket t, double* energy, float* forces) {
    clear_error();
    if (!S) return set_error(MLP_EINVAL, "NULL server");
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->results.find(t);
    if (it == S->results.end()) return set_error(MLP_ENOTFOUND, "unknown ticket %llu", (unsigned long long)t);
    if (!it->second->done) return MLP_PENDING;
    int rc = take_result(S, it, energy, forces);
    if (rc) set_error(rc, "request failed");
    return rc;
}

int mlp_wait(mlp_server* S, mlp_ticket t, int64_t timeout_ns, double* energy, float* forces) {
    clear_error();
    if (!S) return set_error(MLP_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto deadline = Clock::now() + std::chrono::nanoseconds(timeout_ns < 0 ? 0 : timeout_ns);
    for (;;) {
        auto it = S->results.find(t);
        if (it == S->results.end()) return set_error(MLP_ENOTFOUND, "unknown ticket %llu", (unsigned long long)t);
        if (it->second->done) {
            int rc = take_result(S, it, energy, forces);
            if (rc) set_error(rc, "request failed");
            return rc;
        }
        if (S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout) {
            auto it2 = S->results.find(t);
            if (it2 != S->results.end() && it2->second->done) continue;
            return set_error(MLP_ETIMEDOUT, "ticket %llu not done within %lld ns", (unsigned long long)t,
                             (long long)timeout_ns);
        }
    }
}

int mlp_server_get_stats(mlp_server* S, mlp_server_stats* out) {
    clear_error();
    if (!S || !out) return set_error(MLP_EINVAL, "NULL argument");
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->inflight_bytes = S->inflight_bytes;
    out->mean_batch_atoms = S->st.batches ? (double)S->st.atoms / (double)S->st.batches : 0.0;
    out->slot_bytes = (int64_t)slot_bytes(S->o);
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

int mlp_server_replay(mlp_server* S, int32_t n_req, const int64_t* arrival_ns, const int32_t* mol_start,
                      const int8_t* species, const double* coords, double* energies, float* forces,
                      int64_t* wall_ns) {
    clear_error();
    if (!S || !arrival_ns || !mol_start || !species || !coords || !energies || n_req <= 0)
        return set_error(MLP_EINVAL, "bad replay arguments");
    std::vector<mlp_ticket> tickets(n_req);
    int status = MLP_OK;
    const int64_t t0 = now_ns();
    std::thread gen([&]() {
        for (int r = 0; r < n_req; ++r) {
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
                    status = rc;
                    tickets[r] = 0;
                    break;
                }
                std::this_thread::sleep_for(std::chrono::microseconds(20));
            }
        }
    });
    gen.join();
    if (status != MLP_OK) return set_error(status, "replay submit failed");
    for (int r = 0; r < n_req; ++r) {
        const int a = mol_start[r];
        int rc = mlp_wait(S, tickets[r], 600LL * 1000000000LL, &energies[r], forces ? forces + 3 * (size_t)a : nullptr);
        if (rc) return rc;
    }
    if (wall_ns) *wall_ns = now_ns() - t0;
    return MLP_OK;
}

}  // extern "C"
