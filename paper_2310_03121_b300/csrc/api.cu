// C-ABI of libmlp (declared in include/mlp.h): weights, systems, batches,
// introspection and kernel-level test access. The serving loop is in
// server.cu. Every entry point validates its arguments on the host before
// anything reaches a kernel, and converts failures into MLP_* codes.
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/mlp.h"
#include "engine.cuh"
#include "system.cuh"

using namespace mlp;

struct mlp_batch {
    int precision = 0;
    int max_atoms_per_mol = 256;
    const mlp_weights* w = nullptr;
    Workspace ws;
    cudaStream_t stream = nullptr;
    void* dev_block = nullptr;
    int* d_mol_start = nullptr;
    int8_t* d_species = nullptr;
    double* d_xyz = nullptr;
    double* d_E = nullptr;
    float* d_F = nullptr;
    void* h_block = nullptr;   // pinned staging
    int* h_mol_start = nullptr;
    int8_t* h_species = nullptr;
    double* h_xyz = nullptr;
    double* h_E = nullptr;
    float* h_F = nullptr;
    cudaEvent_t done = nullptr;
    bool pending = false;
};

namespace mlp {
const DevWeights& weights_of(const mlp_weights* w) { return w->dw; }
}  // namespace mlp

namespace mlp {

int check_cuda_device() {
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return set_error(MLP_ECUDA, "no usable CUDA device (%s)", e == cudaSuccess ? "none" : cudaGetErrorString(e));
    }
    init_constants_for_current_device();
    return MLP_OK;
}

int sys_finish_pending(mlp_system* s) {
    if (!s->pending) return MLP_OK;
    cudaError_t e = cudaEventSynchronize(s->done);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventSynchronize");
    s->pending = false;
    int rc = check_counters(s->ws);
    if (rc) {   // reported now: not again as an earlier evaluation's error
        cudaMemset(s->ws.err_sticky, 0, sizeof(int));
        cudaStreamSynchronize(nullptr);
        return rc;
    }
    // errors of earlier evaluations that were not checked one by one
    int sticky = 0;
    e = cudaMemcpy(&sticky, s->ws.err_sticky, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(error flags)");
    if (sticky) {
        cudaMemset(s->ws.err_sticky, 0, sizeof(int));
        cudaStreamSynchronize(nullptr);   // cleared before the system's (non-blocking) stream runs again
        if (sticky & 4)
            return set_error(MLP_EINVAL, "bad input (element code or ML-region index) in an earlier evaluation");
        if (sticky & 8) return set_error(MLP_ECUDA, "tensor-core network kernel error in an earlier evaluation");
        return set_error(MLP_EOVERFLOW, "neighbor capacity exceeded in an earlier evaluation");
    }
    return MLP_OK;
}

// Device-path calls do not wait for the previous evaluation: its flags are
// checked here when it has already finished, otherwise they stay in the
// device's sticky error word until mlp_sync (or a host-path call) reads them.
int sys_check_if_done(mlp_system* s) {
    if (!s->pending) return MLP_OK;
    cudaError_t q = cudaEventQuery(s->done);
    if (q == cudaErrorNotReady) return MLP_OK;
    if (q != cudaSuccess) return cuda_error(q, "cudaEventQuery");
    s->pending = false;
    const int rc = check_counters(s->ws);
    if (rc) {   // reported now, not again later (error path only: clear before any new launch)
        cudaMemset(s->ws.err_sticky, 0, sizeof(int));
        cudaStreamSynchronize(nullptr);
    }
    return rc;
}

}  // namespace mlp

namespace {

inline size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// float -> bf16 (round to nearest even) on the host
inline __nv_bfloat16 to_bf16(float f) { return __float2bfloat16_rn(f); }

int sys_make_workspace(mlp_system* s, int nbr_cap) {
    // open systems: at most ~2 cells per atom plus slack
    // at most ~2 cells per atom plus slack (periodic boxes: never more cells
    // than that either, however large the box)
    const long long cell_cap = 2LL * s->n + 64;
    int max_cells = s->periodic ? make_periodic_grid(s->L, (float)(s->cut.rc_rad + s->cut.skin), cell_cap).ncell
                                : (int)cell_cap;
    int rc = workspace_create(s->ws, s->n, 1, s->precision, true, nbr_cap, max_cells, s->w->dw.n_nets);
    if (rc) return rc;
    if (s->periodic) {
        Grid g = make_periodic_grid(s->L, (float)(s->cut.rc_rad + s->cut.skin), cell_cap);
        cudaError_t e = cudaMemcpy(s->ws.grid, &g, sizeof(Grid), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(grid)");
    }
    s->nbr_valid = false;
    return MLP_OK;
}

}  // namespace

namespace mlp {
EvalSpec sys_spec(mlp_system* s, const double* d_xyz) {
    EvalSpec sp;
    sp.n_atoms = s->n;
    sp.n_mols = 1;
    sp.d_species = s->d_species;
    sp.d_xyz = d_xyz;
    sp.periodic = s->periodic;
    for (int a = 0; a < 3; ++a) sp.L[a] = s->L[a];
    sp.r_list = (float)(s->cut.rc_rad + s->cut.skin);
    double hs = 0.5 * s->cut.skin;
    sp.half_skin2 = (float)(hs * hs);
    sp.force_rebuild = !s->nbr_valid || s->cut.skin <= 0.0 || (s->calls % s->rebuild_interval) == 0;
    return sp;
}

}  // namespace mlp

namespace {
int sys_enqueue(mlp_system* s, EvalSpec& sp, cudaStream_t st) {
    int rc = enqueue_eval(s->ws, s->w->dw, sp, st);
    if (rc) return rc;
    cudaError_t e = cudaEventRecord(s->done, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    s->pending = true;
    s->nbr_valid = true;
    s->calls++;
    return MLP_OK;
}

}  // namespace

extern "C" {

const char* mlp_last_error(void) { return last_error(); }

int64_t mlp_launch_count(void) { return (int64_t)launch_count(); }

int mlp_profile_enable(int on) { return profile_enable(on); }

int mlp_profile_read(const char** names, double* total_ms, int64_t* launches, int cap) {
    std::vector<long long> tmp(cap > 0 ? cap : 1);
    int k = profile_read(names, total_ms, tmp.data(), cap);
    if (launches)
        for (int q = 0; q < cap && q < k; ++q) launches[q] = tmp[q];
    return k;
}

void mlp_profile_reset(void) { profile_reset(); }

void mlp_set_allocator(void* (*alloc_fn)(size_t, void*), void (*free_fn)(void*, void*), void* ctx) {
    set_allocator(alloc_fn, free_fn, ctx);
}

void mlp_debug_fail_alloc(long long after) { set_alloc_failure(after); }

// ------------------------------------------------------------------ weights
int mlp_weights_create(const mlp_weights_host* w, int n_nets, mlp_weights** out) {
    clear_error();
    if (!w || !out) return set_error(MLP_EINVAL, "NULL argument");
    *out = nullptr;
    if (n_nets < 1 || n_nets > kMaxNets) return set_error(MLP_EINVAL, "n_nets %d outside [1, %d]", n_nets, kMaxNets);
    if (!w->W1 || !w->b1 || !w->W2 || !w->b2 || !w->W3 || !w->b3 || !w->W4 || !w->b4)
        return set_error(MLP_EINVAL, "NULL weight array");
    int rc = check_cuda_device();
    if (rc) return rc;
    const int S = kNSpecies;
    const size_t K = (size_t)n_nets;
    // per-net sizes (elements)
    const size_t nW1 = (size_t)S * kH1 * kAevLen, nb1 = S * kH1, nW2 = (size_t)S * kH2 * kH1, nb2 = S * kH2,
                 nW3 = (size_t)S * kH3 * kH2, nb3 = S * kH3, nW4 = S * kH3, nb4 = S;
    const size_t nW1p = (size_t)S * kH1 * kAevLd;   // padded K for the BF16 operands
    for (size_t q = 0; q < nW1 * K; ++q)
        if (!std::isfinite(w->W1[q])) return set_error(MLP_EINVAL, "non-finite weight in W1");
    // Every array holds the K nets back to back ("net-major"), so that net k
    // of element s is block k * 7 + s of one matrix: one TMA map per weight
    // matrix covers the whole ensemble.
    // FP32 block: W1 b1 W2 b2 W3 b3 W4 b4 W1t W2t W3t
    const size_t f32_cnt[11] = {nW1, nb1, nW2, nb2, nW3, nb3, nW4, nb4, nW1, nW2, nW3};
    size_t f32_off[11], f32_bytes = 0;
    for (int q = 0; q < 11; ++q) {
        f32_off[q] = f32_bytes;
        f32_bytes += al256(f32_cnt[q] * K * 4);
    }
    // BF16 block: W1 W2 W3 W1t W2t W3t W1lo W2lo W3lo (W1 K padded to 1024, W1t rows >= 1008 zero)
    const size_t bf_cnt[9] = {nW1p, nW2, nW3, nW1p, nW2, nW3, nW1p, nW2, nW3};
    size_t bf_off[9], bf_bytes = 0;
    for (int q = 0; q < 9; ++q) {
        bf_off[q] = bf_bytes;
        bf_bytes += al256(bf_cnt[q] * K * 2);
    }
    mlp_weights* mw = new (std::nothrow) mlp_weights();
    if (!mw) return set_error(MLP_ENOMEM, "host allocation failed");
    mw->dw.n_nets = n_nets;
    cudaGetDevice(&mw->dw.device);
    mw->dw.blk_f32 = dev_alloc(f32_bytes);
    mw->dw.blk_bf16 = dev_alloc(bf_bytes);
    if (!mw->dw.blk_f32 || !mw->dw.blk_bf16) {
        mlp_weights_destroy(mw);
        return set_error(MLP_ENOMEM, "device allocation of the weights failed");
    }
    std::vector<char> hf(f32_bytes, 0), hb(bf_bytes, 0);
    auto F = [&](int q, size_t net) { return reinterpret_cast<float*>(hf.data() + f32_off[q]) + net * f32_cnt[q]; };
    auto B = [&](int q, size_t net) {
        return reinterpret_cast<__nv_bfloat16*>(hb.data() + bf_off[q]) + net * bf_cnt[q];
    };
    // remainder after BF16 rounding, itself rounded to BF16
    auto lo_of = [](float x) { return to_bf16(x - __bfloat162float(to_bf16(x))); };
    for (size_t net = 0; net < K; ++net) {
        const float* W1 = w->W1 + net * nW1;
        const float* W2 = w->W2 + net * nW2;
        const float* W3 = w->W3 + net * nW3;
        std::memcpy(F(0, net), W1, nW1 * 4);
        std::memcpy(F(1, net), w->b1 + net * nb1, nb1 * 4);
        std::memcpy(F(2, net), W2, nW2 * 4);
        std::memcpy(F(3, net), w->b2 + net * nb2, nb2 * 4);
        std::memcpy(F(4, net), W3, nW3 * 4);
        std::memcpy(F(5, net), w->b3 + net * nb3, nb3 * 4);
        std::memcpy(F(6, net), w->W4 + net * nW4, nW4 * 4);
        std::memcpy(F(7, net), w->b4 + net * nb4, nb4 * 4);
        float *W1t = F(8, net), *W2t = F(9, net), *W3t = F(10, net);
        __nv_bfloat16 *bW1 = B(0, net), *bW2 = B(1, net), *bW3 = B(2, net), *bW1t = B(3, net), *bW2t = B(4, net),
                      *bW3t = B(5, net), *bW1lo = B(6, net), *bW2lo = B(7, net), *bW3lo = B(8, net);
        for (int s = 0; s < S; ++s) {
            for (int o = 0; o < kH1; ++o)
                for (int c = 0; c < kAevLen; ++c) {
                    const float x = W1[(size_t)s * kH1 * kAevLen + (size_t)o * kAevLen + c];
                    const __nv_bfloat16 v = to_bf16(x);
                    W1t[(size_t)s * kAevLen * kH1 + (size_t)c * kH1 + o] = x;
                    bW1[(size_t)s * kH1 * kAevLd + (size_t)o * kAevLd + c] = v;
                    bW1lo[(size_t)s * kH1 * kAevLd + (size_t)o * kAevLd + c] = lo_of(x);
                    bW1t[(size_t)s * kAevLd * kH1 + (size_t)c * kH1 + o] = v;
                }
            for (int o = 0; o < kH2; ++o)
                for (int c = 0; c < kH1; ++c) {
                    const float x = W2[(size_t)s * kH2 * kH1 + o * kH1 + c];
                    const __nv_bfloat16 v = to_bf16(x);
                    W2t[(size_t)s * kH1 * kH2 + c * kH2 + o] = x;
                    bW2[(size_t)s * kH2 * kH1 + o * kH1 + c] = v;
                    bW2lo[(size_t)s * kH2 * kH1 + o * kH1 + c] = lo_of(x);
                    bW2t[(size_t)s * kH1 * kH2 + c * kH2 + o] = v;
                }
            for (int o = 0; o < kH3; ++o)
                for (int c = 0; c < kH2; ++c) {
                    const float x = W3[(size_t)s * kH3 * kH2 + o * kH2 + c];
                    const __nv_bfloat16 v = to_bf16(x);
                    W3t[(size_t)s * kH2 * kH3 + c * kH3 + o] = x;
                    bW3[(size_t)s * kH3 * kH2 + o * kH2 + c] = v;
                    bW3lo[(size_t)s * kH3 * kH2 + o * kH2 + c] = lo_of(x);
                    bW3t[(size_t)s * kH2 * kH3 + c * kH3 + o] = v;
                }
        }
    }
    cudaError_t e = cudaMemcpy(mw->dw.blk_f32, hf.data(), f32_bytes, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(mw->dw.blk_bf16, hb.data(), bf_bytes, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        mlp_weights_destroy(mw);
        return cuda_error(e, "cudaMemcpy(weights)");
    }
    const char* df = static_cast<const char*>(mw->dw.blk_f32);
    const char* db = static_cast<const char*>(mw->dw.blk_bf16);
    auto DF = [&](int q, size_t net) { return reinterpret_cast<const float*>(df + f32_off[q]) + net * f32_cnt[q]; };
    auto DB = [&](int q) { return reinterpret_cast<const __nv_bfloat16*>(db + bf_off[q]); };
    for (size_t net = 0; net < K; ++net) {
        NetF32& nf = mw->dw.f32[net];
        nf.W1 = DF(0, net);
        nf.b1 = DF(1, net);
        nf.W2 = DF(2, net);
        nf.b2 = DF(3, net);
        nf.W3 = DF(4, net);
        nf.b3 = DF(5, net);
        nf.W4 = DF(6, net);
        nf.b4 = DF(7, net);
        nf.W1t = DF(8, net);
        nf.W2t = DF(9, net);
        nf.W3t = DF(10, net);
    }
    NetBF16& nb = mw->dw.bf16;
    nb.n_nets = n_nets;
    nb.W1 = DB(0);
    nb.W2 = DB(1);
    nb.W3 = DB(2);
    nb.W1t = DB(3);
    nb.W2t = DB(4);
    nb.W3t = DB(5);
    nb.W1lo = DB(6);
    nb.W2lo = DB(7);
    nb.W3lo = DB(8);
    nb.b1 = DF(1, 0);
    nb.b2 = DF(3, 0);
    nb.b3 = DF(5, 0);
    nb.W4 = DF(6, 0);
    nb.b4 = DF(7, 0);
    if (!make_weight_maps(nb)) {
        mlp_weights_destroy(mw);
        return set_error(MLP_ECUDA, "TMA tensor map creation for the weights failed");
    }
    *out = mw;
    return MLP_OK;
}

void mlp_weights_destroy(mlp_weights* w) {
    if (!w) return;
    dev_free(w->dw.blk_f32);
    dev_free(w->dw.blk_bf16);
    delete w;
}

// ------------------------------------------------------------------ systems
int mlp_create(const int8_t* species, const double* coords, int32_t n, const double* cell, const mlp_cutoffs* cut,
               const mlp_weights* w, int precision, mlp_system** out) {
    clear_error();
    if (!out) return set_error(MLP_EINVAL, "NULL out");
    *out = nullptr;
    if (!species || !cut || !w) return set_error(MLP_EINVAL, "NULL argument");
    if (n <= 0) return set_error(MLP_EINVAL, "n = %d must be positive", n);
    if (precision < MLP_FP32 || precision > MLP_BF16_1PASS) return set_error(MLP_EINVAL, "unknown precision %d", precision);
    if (precision != MLP_FP32 && !mlp_tc_available())
        return set_error(MLP_EINVAL, "BF16 tensor-core network is not available in this build");
    if (std::fabs(cut->rc_rad - 5.1) > 1e-12 || std::fabs(cut->rc_ang - 3.5) > 1e-12)
        return set_error(MLP_EINVAL, "cutoffs must be rc_rad = 5.1 and rc_ang = 3.5 (the AEV's own)");
    if (!(cut->skin >= 0.0) || cut->skin > 2.0) return set_error(MLP_EINVAL, "skin must be in [0, 2]");
    for (int i = 0; i < n; ++i)
        if (species[i] < 0 || species[i] >= kNSpecies) return set_error(MLP_EINVAL, "species[%d] = %d", i, species[i]);
    if (cell) {
        for (int a = 0; a < 3; ++a)
            if (!(cell[a] >= 2.0 * (cut->rc_rad + cut->skin)) || !std::isfinite(cell[a]))
                return set_error(MLP_EINVAL, "box length %g below 2 (rc_rad + skin)", cell[a]);
    }
    if (coords)
        for (long q = 0; q < 3L * n; ++q)
            if (!std::isfinite(coords[q])) return set_error(MLP_EINVAL, "non-finite coordinate");
    int rc = check_cuda_device();
    if (rc) return rc;
    mlp_system* s = new (std::nothrow) mlp_system();
    if (!s) return set_error(MLP_ENOMEM, "host allocation failed");
    s->n = n;
    s->periodic = cell ? 1 : 0;
    if (cell)
        for (int a = 0; a < 3; ++a) s->L[a] = cell[a];
    s->cut = *cut;
    s->w = w;
    s->precision = precision;
    // a list with a skin reaches (rc + skin)^3 / rc^3 times as many neighbors
    // and is kept for several steps while atoms move: rows of the largest
    // capacity from the start (no regrowth in the middle of a trajectory)
    rc = sys_make_workspace(s, cut->skin > 0.0 ? kMaxNbrCap : kDefaultNbrCap);
    if (rc) {
        mlp_destroy(s);
        return rc;
    }
    size_t db = al256((size_t)n) + al256(24 * (size_t)n) + al256(8) + al256(12 * (size_t)n);
    s->dev_block = dev_alloc(db);
    if (!s->dev_block) {
        mlp_destroy(s);
        return set_error(MLP_ENOMEM, "device allocation failed");
    }
    char* p = static_cast<char*>(s->dev_block);
    s->d_species = reinterpret_cast<int8_t*>(p);
    p += al256(n);
    s->d_xyz = reinterpret_cast<double*>(p);
    p += al256(24 * (size_t)n);
    s->d_E = reinterpret_cast<double*>(p);
    p += al256(8);
    s->d_F = reinterpret_cast<float*>(p);
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&s->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void**>(&s->h_xyz), 24 * (size_t)n)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void**>(&s->h_E), 8)) != cudaSuccess ||
        (e = cudaMallocHost(reinterpret_cast<void**>(&s->h_F), 12 * (size_t)n)) != cudaSuccess) {
        mlp_destroy(s);
        return cuda_error(e, "mlp_create");
    }
    e = cudaMemcpy(s->d_species, species, n, cudaMemcpyHostToDevice);
    if (e == cudaSuccess && coords) e = cudaMemcpy(s->d_xyz, coords, 24 * (size_t)n, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        mlp_destroy(s);
        return cuda_error(e, "mlp_create copy");
    }
    *out = s;
    return MLP_OK;
}

void mlp_destroy(mlp_system* s) {
    if (!s) return;
    if (s->stream) cudaStreamSynchronize(s->stream);
    workspace_destroy(s->ws);
    dev_free(s->dev_block);
    if (s->stream) cudaStreamDestroy(s->stream);
    if (s->done) cudaEventDestroy(s->done);
    if (s->h_xyz) cudaFreeHost(s->h_xyz);
    if (s->h_E) cudaFreeHost(s->h_E);
    if (s->h_F) cudaFreeHost(s->h_F);
    delete s;
}

int mlp_sync(mlp_system* s) {
    clear_error();
    if (!s) return set_error(MLP_EINVAL, "NULL system");
    return sys_finish_pending(s);
}

int mlp_energy_forces(mlp_system* s, const double* coords, double* energy, float* forces) {
    clear_error();
    if (!s || !energy) return set_error(MLP_EINVAL, "NULL argument");
    int rc = sys_finish_pending(s);
    if (rc) return rc;
    const size_t nb = 24 * (size_t)s->n;
    if (coords) {
        for (long q = 0; q < 3L * s->n; ++q)
            if (!std::isfinite(coords[q])) return set_error(MLP_EINVAL, "non-finite coordinate");
        std::memcpy(s->h_xyz, coords, nb);
        cudaError_t e = cudaMemcpyAsync(s->d_xyz, s->h_xyz, nb, cudaMemcpyHostToDevice, s->stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(coords)");
    }
    for (int attempt = 0; attempt < 2; ++attempt) {
        s->kept = false;
        EvalSpec sp = sys_spec(s, s->d_xyz);
        sp.d_E = s->d_E;
        sp.d_F = forces ? s->d_F : nullptr;
        rc = sys_enqueue(s, sp, s->stream);
        if (rc) return rc;
        cudaMemcpyAsync(s->h_E, s->d_E, 8, cudaMemcpyDeviceToHost, s->stream);
        if (forces) cudaMemcpyAsync(s->h_F, s->d_F, 12 * (size_t)s->n, cudaMemcpyDeviceToHost, s->stream);
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
        s->pending = false;
        rc = check_counters(s->ws);
        if (rc == MLP_EOVERFLOW && s->ws.h_ctr->nbr_overflow && s->ws.nbr_cap < kMaxNbrCap && attempt == 0) {
            // grow the neighbor rows once and redo the evaluation
            workspace_destroy(s->ws);
            rc = sys_make_workspace(s, kMaxNbrCap);
            if (rc) return rc;
            continue;
        }
        if (rc) return rc;
        break;
    }
    *energy = *s->h_E;
    if (forces) std::memcpy(forces, s->h_F, 12 * (size_t)s->n);
    return MLP_OK;
}

int mlp_energy_forces_device(mlp_system* s, const double* d_coords, double* d_energy, float* d_forces, void* stream) {
    clear_error();
    if (!s || !d_coords || !d_energy) return set_error(MLP_EINVAL, "NULL argument");
    int rc = sys_check_if_done(s);
    if (rc) return rc;
    s->kept = false;
    EvalSpec sp = sys_spec(s, d_coords);
    sp.d_E = d_energy;
    sp.d_F = d_forces;
    return sys_enqueue(s, sp, static_cast<cudaStream_t>(stream));
}

int mlp_energy_forces_subset_device(mlp_system* s, const double* d_coords_full, int64_t n_full,
                                    const int32_t* d_index, double* d_energy, float* d_forces_full, int accumulate,
                                    void* stream) {
    clear_error();
    if (!s || !d_coords_full || !d_index || !d_energy) return set_error(MLP_EINVAL, "NULL argument");
    if (n_full < s->n || n_full > (int64_t)INT32_MAX)
        return set_error(MLP_EINVAL, "n_full %lld outside [%d, 2^31)", (long long)n_full, s->n);
    int rc = sys_check_if_done(s);
    if (rc) return rc;
    s->kept = false;
    EvalSpec sp = sys_spec(s, s->d_xyz);   // the region's positions: gathered into the system's own buffer
    sp.d_index = d_index;
    sp.d_coords_full = d_coords_full;
    sp.n_full = n_full;
    sp.accumulate = accumulate != 0;
    sp.d_E = d_energy;
    sp.d_F = d_forces_full;
    return sys_enqueue(s, sp, static_cast<cudaStream_t>(stream));
}

int mlp_forward_device(mlp_system* s, const double* d_coords, double* d_energy, int keep_aev, void* stream) {
    clear_error();
    if (!s || !d_coords || !d_energy) return set_error(MLP_EINVAL, "NULL argument");
    int rc = sys_check_if_done(s);
    if (rc) return rc;
    EvalSpec sp = sys_spec(s, d_coords);
    sp.network_backward = false;
    sp.d_E = d_energy;
    rc = sys_enqueue(s, sp, static_cast<cudaStream_t>(stream));
    s->kept = rc == MLP_OK && keep_aev;
    s->kept_coords = d_coords;
    return rc;
}

int mlp_backward_device(mlp_system* s, const double* d_coords, const double* d_grad_energy, float* d_grad_coords,
                        void* stream) {
    clear_error();
    if (!s || !d_coords || !d_grad_coords) return set_error(MLP_EINVAL, "NULL argument");
    int rc = sys_check_if_done(s);
    if (rc) return rc;
    EvalSpec sp = sys_spec(s, d_coords);
    sp.reuse_aev = s->kept && s->kept_coords == d_coords;
    sp.network_backward = true;
    sp.energy = false;
    sp.d_F = d_grad_coords;
    sp.d_grad_scale = d_grad_energy;
    sp.sign = 1.f;
    if (sp.reuse_aev) sp.force_rebuild = false;
    rc = sys_enqueue(s, sp, static_cast<cudaStream_t>(stream));
    return rc;
}

// ------------------------------------------------------------------ batches
int mlp_batch_create(const mlp_weights* w, int precision, int32_t max_atoms, int32_t max_mols,
                     int32_t max_atoms_per_mol, mlp_batch** out) {
    clear_error();
    if (!out) return set_error(MLP_EINVAL, "NULL out");
    *out = nullptr;
    if (!w) return set_error(MLP_EINVAL, "NULL weights");
    if (precision < MLP_FP32 || precision > MLP_BF16_1PASS) return set_error(MLP_EINVAL, "unknown precision %d", precision);
    if (precision != MLP_FP32 && !mlp_tc_available())
        return set_error(MLP_EINVAL, "BF16 tensor-core network is not available in this build");
    if (max_atoms <= 0 || max_mols <= 0 || max_atoms_per_mol <= 0 || max_atoms_per_mol > max_atoms)
        return set_error(MLP_EINVAL, "bad batch dimensions");
    int rc = check_cuda_device();
    if (rc) return rc;
    mlp_batch* b = new (std::nothrow) mlp_batch();
    if (!b) return set_error(MLP_ENOMEM, "host allocation failed");
    b->precision = precision;
    b->max_atoms_per_mol = max_atoms_per_mol;
    b->w = w;
    rc = workspace_create(b->ws, max_atoms, max_mols, precision, false, kDefaultNbrCap, 0, w->dw.n_nets);
    if (rc) {
        mlp_batch_destroy(b);
        return rc;
    }
    const size_t A = max_atoms, Mo = max_mols;
    size_t db = al256(4 * (Mo + 1)) + al256(A) + al256(24 * A) + al256(8 * Mo) + al256(12 * A);
    b->dev_block = dev_alloc(db);
    if (!b->dev_block) {
        mlp_batch_destroy(b);
        return set_error(MLP_ENOMEM, "device allocation failed");
    }
    char* p = static_cast<char*>(b->dev_block);
    b->d_mol_start = reinterpret_cast<int*>(p);
    p += al256(4 * (Mo + 1));
    b->d_species = reinterpret_cast<int8_t*>(p);
    p += al256(A);
    b->d_xyz = reinterpret_cast<double*>(p);
    p += al256(24 * A);
    b->d_E = reinterpret_cast<double*>(p);
    p += al256(8 * Mo);
    b->d_F = reinterpret_cast<float*>(p);
    cudaError_t e;
    if ((e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking)) != cudaSuccess ||
        (e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming)) != cudaSuccess ||
        (e = cudaMallocHost(&b->h_block, db)) != cudaSuccess) {
        mlp_batch_destroy(b);
        return cuda_error(e, "mlp_batch_create");
    }
    char* h = static_cast<char*>(b->h_block);
    b->h_mol_start = reinterpret_cast<int*>(h);
    h += al256(4 * (Mo + 1));
    b->h_species = reinterpret_cast<int8_t*>(h);
    h += al256(A);
    b->h_xyz = reinterpret_cast<double*>(h);
    h += al256(24 * A);
    b->h_E = reinterpret_cast<double*>(h);
    h += al256(8 * Mo);
    b->h_F = reinterpret_cast<float*>(h);
    *out = b;
    return MLP_OK;
}

void mlp_batch_destroy(mlp_batch* b) {
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    workspace_destroy(b->ws);
    dev_free(b->dev_block);
    if (b->stream) cudaStreamDestroy(b->stream);
    if (b->done) cudaEventDestroy(b->done);
    if (b->h_block) cudaFreeHost(b->h_block);
    delete b;
}

int mlp_batch_sync(mlp_batch* b) {
    clear_error();
    if (!b) return set_error(MLP_EINVAL, "NULL batch");
    if (!b->pending) return MLP_OK;
    cudaError_t e = cudaEventSynchronize(b->done);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventSynchronize");
    b->pending = false;
    return check_counters(b->ws);
}

int mlp_batch_run_device(mlp_batch* b, int32_t n_mols, int32_t n_atoms, const int32_t* d_mol_start,
                         const int8_t* d_species, const double* d_coords, double* d_energy, float* d_forces,
                         void* stream) {
    clear_error();
    if (!b || !d_mol_start || !d_species || !d_coords || !d_energy) return set_error(MLP_EINVAL, "NULL argument");
    if (n_mols <= 0 || n_mols > b->ws.cap_mols) return set_error(MLP_EINVAL, "n_mols %d outside [1, %d]", n_mols, b->ws.cap_mols);
    if (n_atoms <= 0 || n_atoms > b->ws.cap_atoms)
        return set_error(MLP_EINVAL, "n_atoms %d outside [1, %d]", n_atoms, b->ws.cap_atoms);
    int rc = mlp_batch_sync(b);
    if (rc) return rc;
    EvalSpec sp;
    sp.n_atoms = n_atoms;
    sp.n_mols = n_mols;
    sp.d_mol_start = d_mol_start;
    sp.d_species = d_species;
    sp.d_xyz = d_coords;
    sp.r_list = kRcRad;
    sp.d_E = d_energy;
    sp.d_F = d_forces;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    rc = enqueue_eval(b->ws, b->w->dw, sp, st);
    if (rc) return rc;
    cudaError_t e = cudaEventRecord(b->done, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    b->pending = true;
    return MLP_OK;
}

int mlp_batch_run(mlp_batch* b, int32_t n_mols, const int32_t* mol_start, const int8_t* species, const double* coords,
                  double* energy, float* forces) {
    clear_error();
    if (!b || !mol_start || !species || !coords || !energy) return set_error(MLP_EINVAL, "NULL argument");
    if (n_mols <= 0 || n_mols > b->ws.cap_mols) return set_error(MLP_EINVAL, "n_mols %d outside [1, %d]", n_mols, b->ws.cap_mols);
    if (mol_start[0] != 0) return set_error(MLP_EINVAL, "mol_start[0] must be 0");
    for (int m = 0; m < n_mols; ++m) {
        int sz = mol_start[m + 1] - mol_start[m];
        if (sz <= 0 || sz > b->max_atoms_per_mol)
            return set_error(MLP_EINVAL, "molecule %d has %d atoms (allowed 1..%d)", m, sz, b->max_atoms_per_mol);
    }
    const int n = mol_start[n_mols];
    if (n > b->ws.cap_atoms) return set_error(MLP_EINVAL, "%d atoms above capacity %d", n, b->ws.cap_atoms);
    for (int i = 0; i < n; ++i)
        if (species[i] < 0 || species[i] >= kNSpecies) return set_error(MLP_EINVAL, "species[%d] = %d", i, species[i]);
    for (long q = 0; q < 3L * n; ++q)
        if (!std::isfinite(coords[q])) return set_error(MLP_EINVAL, "non-finite coordinate");
    int rc = mlp_batch_sync(b);
    if (rc) return rc;
    std::memcpy(b->h_mol_start, mol_start, 4 * (size_t)(n_mols + 1));
    std::memcpy(b->h_species, species, n);
    std::memcpy(b->h_xyz, coords, 24 * (size_t)n);
    cudaStream_t st = b->stream;
    cudaMemcpyAsync(b->d_mol_start, b->h_mol_start, 4 * (size_t)(n_mols + 1), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(b->d_species, b->h_species, n, cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(b->d_xyz, b->h_xyz, 24 * (size_t)n, cudaMemcpyHostToDevice, st);
    rc = mlp_batch_run_device(b, n_mols, n, b->d_mol_start, b->d_species, b->d_xyz, b->d_E, forces ? b->d_F : nullptr,
                              st);
    if (rc) return rc;
    cudaMemcpyAsync(b->h_E, b->d_E, 8 * (size_t)n_mols, cudaMemcpyDeviceToHost, st);
    if (forces) cudaMemcpyAsync(b->h_F, b->d_F, 12 * (size_t)n, cudaMemcpyDeviceToHost, st);
    // the completion event must follow the result copies
    cudaError_t e = cudaEventRecord(b->done, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    rc = mlp_batch_sync(b);
    if (rc) return rc;
    std::memcpy(energy, b->h_E, 8 * (size_t)n_mols);
    if (forces) std::memcpy(forces, b->h_F, 12 * (size_t)n);
    return MLP_OK;
}

// ------------------------------------------------------------------ kernel-level access
int mlp_debug_neighbors(mlp_system* s, int32_t* counts, int32_t* list, int32_t cap) {
    clear_error();
    if (!s) return set_error(MLP_EINVAL, "NULL system");
    int rc = sys_finish_pending(s);
    if (rc) return rc;
    cudaStreamSynchronize(s->stream);
    const int n = s->n, C = s->ws.nbr_cap;
    if (counts) cudaMemcpy(counts, s->ws.nbr_cnt, 4 * (size_t)n, cudaMemcpyDeviceToHost);
    if (list) {
        std::vector<int> tmp((size_t)n * C);
        cudaMemcpy(tmp.data(), s->ws.nbr, 4 * tmp.size(), cudaMemcpyDeviceToHost);
        for (int i = 0; i < n; ++i)
            for (int q = 0; q < cap; ++q) list[(size_t)i * cap + q] = q < C ? tmp[(size_t)i * C + q] : -1;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "mlp_debug_neighbors");
    return C;
}

// dE/dG of a workspace as FP32 on the host (the BF16 networks store it as BF16).
// Per-atom energies of the last evaluation (the mean over the nets of an ensemble).
static cudaError_t copy_e_to_host(const Workspace& ws, int n, float* out) {
    const int K = ws.e_nets();
    if (K == 1) return cudaMemcpy(out, ws.e, 4 * (size_t)n, cudaMemcpyDeviceToHost);
    std::vector<float> all((size_t)K * ws.cap_atoms);
    cudaError_t e = cudaMemcpy(all.data(), ws.e, 4 * all.size(), cudaMemcpyDeviceToHost);
    for (int i = 0; i < n; ++i) {
        double acc = 0.0;
        for (int k = 0; k < K; ++k) acc += all[(size_t)k * ws.cap_atoms + i];
        out[i] = (float)(acc / K);
    }
    return e;
}

static cudaError_t copy_dG_to_host(const Workspace& ws, std::vector<float>& out) {
    const size_t cnt = (size_t)ws.rows_cap * kAevLd;
    out.resize(cnt);
    if (ws.dG) return cudaMemcpy(out.data(), ws.dG, 4 * cnt, cudaMemcpyDeviceToHost);
    std::vector<__nv_bfloat16> tmp(cnt);
    cudaError_t e = cudaMemcpy(tmp.data(), ws.dG16, 2 * cnt, cudaMemcpyDeviceToHost);
    for (size_t q = 0; q < cnt; ++q) out[q] = __bfloat162float(tmp[q]);
    return e;
}

// Row of every atom in the element-grouped matrices (host copy of the counters).
static int atom_rows(mlp_system* s, std::vector<int>& rows) {
    const int n = s->n;
    std::vector<int> rank(n);
    cudaMemcpy(rank.data(), s->ws.rank, 4 * (size_t)n, cudaMemcpyDeviceToHost);
    Counters c;
    cudaMemcpy(&c, s->ws.ctr, sizeof(c), cudaMemcpyDeviceToHost);
    std::vector<int8_t> sp(n);
    cudaMemcpy(sp.data(), s->d_species, n, cudaMemcpyDeviceToHost);
    int base[kNSpecies];
    int b = 0;
    for (int q = 0; q < kNSpecies; ++q) {
        base[q] = b;
        b += (c.species[q] + kTileRows - 1) / kTileRows * kTileRows;
    }
    rows.resize(n);
    for (int i = 0; i < n; ++i) rows[i] = base[sp[i]] + rank[i];
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? 0 : cuda_error(e, "atom_rows");
}

int mlp_debug_aev(mlp_system* s, float* G) {
    clear_error();
    if (!s || !G) return set_error(MLP_EINVAL, "NULL argument");
    int rc = sys_finish_pending(s);
    if (rc) return rc;
    cudaStreamSynchronize(s->stream);
    std::vector<int> rows;
    rc = atom_rows(s, rows);
    if (rc) return rc;
    const size_t R = s->ws.rows_cap;
    if (s->precision == MLP_FP32) {
        std::vector<float> all(R * kAevLd);
        cudaMemcpy(all.data(), s->ws.G32, 4 * all.size(), cudaMemcpyDeviceToHost);
        for (int i = 0; i < s->n; ++i) std::memcpy(G + (size_t)i * kAevLen, &all[(size_t)rows[i] * kAevLd], 4 * kAevLen);
    } else {
        // the value the network consumes: G_hi + G_lo (split path) or G_hi
        std::vector<__nv_bfloat16> all(R * kAevLd), lo;
        cudaMemcpy(all.data(), s->ws.G16, 2 * all.size(), cudaMemcpyDeviceToHost);
        if (s->ws.G16lo) {
            lo.resize(R * kAevLd);
            cudaMemcpy(lo.data(), s->ws.G16lo, 2 * lo.size(), cudaMemcpyDeviceToHost);
        }
        for (int i = 0; i < s->n; ++i)
            for (int c = 0; c < kAevLen; ++c) {
                const size_t q = (size_t)rows[i] * kAevLd + c;
                G[(size_t)i * kAevLen + c] = __bfloat162float(all[q]) + (lo.empty() ? 0.f : __bfloat162float(lo[q]));
            }
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLP_OK : cuda_error(e, "mlp_debug_aev");
}

int mlp_debug_aev_split(mlp_system* s, float* G_hi, float* G_lo) {
    clear_error();
    if (!s || !G_hi) return set_error(MLP_EINVAL, "NULL argument");
    if (s->precision == MLP_FP32) return set_error(MLP_EINVAL, "the FP32 path stores no BF16 AEV rows");
    int rc = sys_finish_pending(s);
    if (rc) return rc;
    cudaStreamSynchronize(s->stream);
    std::vector<int> rows;
    rc = atom_rows(s, rows);
    if (rc) return rc;
    const size_t R = s->ws.rows_cap;
    std::vector<__nv_bfloat16> hi(R * kAevLd), lo;
    cudaMemcpy(hi.data(), s->ws.G16, 2 * hi.size(), cudaMemcpyDeviceToHost);
    if (s->ws.G16lo) {
        lo.resize(R * kAevLd);
        cudaMemcpy(lo.data(), s->ws.G16lo, 2 * lo.size(), cudaMemcpyDeviceToHost);
    }
    for (int i = 0; i < s->n; ++i)
        for (int c = 0; c < kAevLen; ++c) {
            const size_t q = (size_t)rows[i] * kAevLd + c;
            G_hi[(size_t)i * kAevLen + c] = __bfloat162float(hi[q]);
            if (G_lo) G_lo[(size_t)i * kAevLen + c] = lo.empty() ? 0.f : __bfloat162float(lo[q]);
        }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLP_OK : cuda_error(e, "mlp_debug_aev_split");
}

int mlp_debug_forces(mlp_system* s, const float* dEdG, double* forces) {
    clear_error();
    if (!s || !dEdG || !forces) return set_error(MLP_EINVAL, "NULL argument");
    int rc = sys_finish_pending(s);
    if (rc) return rc;
    cudaStreamSynchronize(s->stream);
    std::vector<int> rows;
    rc = atom_rows(s, rows);
    if (rc) return rc;
    Workspace& ws = s->ws;
    const size_t R = ws.rows_cap;
    const int n = s->n;
    cudaError_t e;
    // inputs and the zeroed force sums go in on the system's own stream (a
    // non-blocking stream: the legacy stream's work would not order with it)
    std::vector<float> all32;
    std::vector<__nv_bfloat16> all16;
    if (ws.dG) {
        all32.assign(R * kAevLd, 0.f);
        for (int i = 0; i < n; ++i) std::memcpy(&all32[(size_t)rows[i] * kAevLd], dEdG + (size_t)i * kAevLen, 4 * kAevLen);
        e = cudaMemcpyAsync(ws.dG, all32.data(), 4 * all32.size(), cudaMemcpyHostToDevice, s->stream);
    } else {
        all16.assign(R * kAevLd, to_bf16(0.f));
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < kAevLen; ++c) all16[(size_t)rows[i] * kAevLd + c] = to_bf16(dEdG[(size_t)i * kAevLen + c]);
        e = cudaMemcpyAsync(ws.dG16, all16.data(), 2 * all16.size(), cudaMemcpyHostToDevice, s->stream);
    }
    if (e == cudaSuccess) e = cudaMemsetAsync(ws.grad, 0, sizeof(double) * 3 * (size_t)n, s->stream);
    if (e != cudaSuccess) return cuda_error(e, "mlp_debug_forces (inputs)");
    AevArgs aa;
    aa.n = n;
    aa.hi = ws.hi;
    aa.lo = ws.lo;
    aa.nbr = ws.nbr;
    aa.nbr_cnt = ws.nbr_cnt;
    aa.cap = ws.nbr_cap;
    aa.box = make_box(s->periodic, s->L);
    aa.ctr = ws.ctr;
    aa.rank = ws.rank;
    aa.big_list = ws.ang_big_list;
    aa.big_flag = ws.ang_big_flag;
    launch_forces(s->stream, aa, ws.dG, ws.dG16, ws.grad, ws.precision != MLP_FP32);
    e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_error(e, "mlp_debug_forces");
    std::vector<double> grad(3 * (size_t)n);
    e = cudaMemcpyAsync(grad.data(), ws.grad, sizeof(double) * grad.size(), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    if (e != cudaSuccess) return cuda_error(e, "mlp_debug_forces (copy)");
    for (size_t q = 0; q < grad.size(); ++q) forces[q] = -grad[q];
    s->nbr_valid = false;   // the next evaluation rebuilds everything it reads
    s->kept = false;        // and a following backward recomputes its AEVs (the force sums were used here)
    return MLP_OK;
}

int mlp_debug_atom_energies(mlp_system* s, float* e_out, float* dEdG) {
    clear_error();
    if (!s || !e_out) return set_error(MLP_EINVAL, "NULL argument");
    int rc = sys_finish_pending(s);
    if (rc) return rc;
    cudaStreamSynchronize(s->stream);
    copy_e_to_host(s->ws, s->n, e_out);
    if (dEdG) {
        std::vector<int> rows;
        rc = atom_rows(s, rows);
        if (rc) return rc;
        std::vector<float> all((size_t)s->ws.rows_cap * kAevLd);
        copy_dG_to_host(s->ws, all);
        for (int i = 0; i < s->n; ++i)
            std::memcpy(dEdG + (size_t)i * kAevLen, &all[(size_t)rows[i] * kAevLd], 4 * kAevLen);
    }
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLP_OK : cuda_error(e, "mlp_debug_atom_energies");
}

int mlp_debug_network(const mlp_weights* w, int precision, int32_t n, const int8_t* species, const float* G,
                      float* e_out, float* dEdG) {
    clear_error();
    if (!w || !species || !G || !e_out) return set_error(MLP_EINVAL, "NULL argument");
    if (n <= 0) return set_error(MLP_EINVAL, "n must be positive");
    if (precision < MLP_FP32 || precision > MLP_BF16_1PASS) return set_error(MLP_EINVAL, "unknown precision");
    if (precision != MLP_FP32 && !mlp_tc_available()) return set_error(MLP_EINVAL, "BF16 network not available");
    int rc = check_cuda_device();
    if (rc) return rc;
    Workspace ws;
    rc = workspace_create(ws, n, 1, precision, false, 1, 0, w->dw.n_nets);
    if (rc) return rc;
    // element-grouped rows: stable order inside each element
    Counters c;
    std::memset(&c, 0, sizeof(c));
    std::vector<int> rank(n);
    for (int i = 0; i < n; ++i) {
        if (species[i] < 0 || species[i] >= kNSpecies) {
            workspace_destroy(ws);
            return set_error(MLP_EINVAL, "species[%d] = %d", i, species[i]);
        }
        rank[i] = c.species[species[i]]++;
    }
    int base[kNSpecies], b = 0;
    for (int q = 0; q < kNSpecies; ++q) {
        base[q] = b;
        b += (c.species[q] + kTileRows - 1) / kTileRows * kTileRows;
    }
    const size_t R = ws.rows_cap;
    std::vector<int> row_atom(R, 0);
    std::vector<int> rows(n);
    for (int i = 0; i < n; ++i) {
        rows[i] = base[species[i]] + rank[i];
        row_atom[rows[i]] = i;
    }
    cudaMemcpy(ws.ctr, &c, sizeof(c), cudaMemcpyHostToDevice);
    cudaMemcpy(ws.row_atom, row_atom.data(), 4 * R, cudaMemcpyHostToDevice);
    if (precision == MLP_FP32) {
        std::vector<float> all(R * kAevLd, 0.f);
        for (int i = 0; i < n; ++i) std::memcpy(&all[(size_t)rows[i] * kAevLd], G + (size_t)i * kAevLen, 4 * kAevLen);
        cudaMemcpy(ws.G32, all.data(), 4 * all.size(), cudaMemcpyHostToDevice);
        for (int k = 0; k < w->dw.n_nets; ++k)
            launch_mlp_f32(nullptr, ws.rows_cap, ws.ctr, w->dw.f32[k], ws.G32, ws.row_atom, ws.fb, ws.e, ws.dG, true,
                           k, w->dw.n_nets);
    } else {
        std::vector<__nv_bfloat16> all(R * kAevLd, to_bf16(0.f)), all_lo(R * kAevLd, to_bf16(0.f));
        for (int i = 0; i < n; ++i)
            for (int q = 0; q < kAevLen; ++q) {
                const float x = G[(size_t)i * kAevLen + q];
                all[(size_t)rows[i] * kAevLd + q] = to_bf16(x);
                all_lo[(size_t)rows[i] * kAevLd + q] = to_bf16(x - __bfloat162float(to_bf16(x)));
            }
        cudaMemcpy(ws.G16, all.data(), 2 * all.size(), cudaMemcpyHostToDevice);
        if (ws.G16lo) cudaMemcpy(ws.G16lo, all_lo.data(), 2 * all_lo.size(), cudaMemcpyHostToDevice);
        if (!launch_mlp_bf16(nullptr, ws.rows_cap, ws.ctr, w->dw.bf16, ws.G16, ws.G16lo, precision == MLP_BF16,
                             ws.row_atom, ws.e, ws.cap_atoms, ws.dG16, ws.g1ens, true, ws.tc_err)) {
            workspace_destroy(ws);
            return MLP_ECUDA;
        }
    }
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = copy_e_to_host(ws, n, e_out);
    if (e == cudaSuccess && dEdG) {
        std::vector<float> all(R * kAevLd);
        e = copy_dG_to_host(ws, all);
        for (int i = 0; i < n; ++i) std::memcpy(dEdG + (size_t)i * kAevLen, &all[(size_t)rows[i] * kAevLd], 4 * kAevLen);
    }
    int tc = 0;
    if (e == cudaSuccess && precision != MLP_FP32) e = cudaMemcpy(&tc, ws.tc_err, 4, cudaMemcpyDeviceToHost);
    workspace_destroy(ws);
    if (e != cudaSuccess) return cuda_error(e, "mlp_debug_network");
    if (tc) return set_error(MLP_ECUDA, "tensor-core kernel reported error %d", tc);
    return MLP_OK;
}

int mlp_debug_wait_timeout(int32_t* timed_out, int32_t* code) {
    clear_error();
    if (!timed_out || !code) return set_error(MLP_EINVAL, "NULL argument");
    int rc = check_cuda_device();
    if (rc) return rc;
    int t = 0, c = 0;
    const int e = debug_wait_timeout(&t, &c);
    if (e) return cuda_error((cudaError_t)e, "mlp_debug_wait_timeout");
    *timed_out = t;
    *code = c;
    return MLP_OK;
}

}  // extern "C"
