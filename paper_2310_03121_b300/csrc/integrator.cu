// Langevin dynamics around the energy+force evaluation: the LF-Middle
// discretization (paper, section "New Integrators"; the ML simulations of
// section "Performance of MLPs", Table 3, use a Langevin integrator with a
// 2 fs step). One step, velocities at half steps, forces F(x_t) from the
// system's evaluation:
//   v <- v + dt F / m;  x <- x + dt/2 v;  v <- a v + sqrt((1 - a^2) kT / m) R;  x <- x + dt/2 v
// with a = exp(-gamma dt). The normal deviates R come from Philox4x64-10
// (Salmon et al., SC 2011; counter (step, atom, 0, 0), key (seed, 0)) by
// Box-Muller, so a trajectory is a pure function of (x0, v0, seed, step0).
//
// A step is the evaluation's launches plus two small kernels (the update, and
// a tick that records the step's potential energy and advances the device
// step counter). Everything a step reads that changes from step to step
// lives in device memory, so the step can be captured once as a CUDA graph
// and replayed: the per-step host cost drops to one graph launch.
#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <new>

#include "kernels.cuh"
#include "system.cuh"

using namespace mlp;

namespace {

constexpr double kAcc = 9.648533212e-3;   // (eV / A) / amu -> A / fs^2
constexpr double kKE = 103.6426965;       // amu A^2 / fs^2 -> eV
constexpr double kBoltz = 8.617333262e-5; // eV / K
// element masses (amu): H, C, N, O, S, F, Cl
constexpr double kMass[kNSpecies] = {1.008, 12.011, 14.007, 15.999, 32.06, 18.998, 35.45};

struct LgvConsts {
    double dt;                    // fs
    double a;                     // exp(-gamma dt)
    double acc_m[8];              // kAcc / m per element
    double sigma[8];              // sqrt((1 - a^2) kT / m), A / fs, per element
    unsigned long long seed;
};

// Philox4x64-10: ten rounds of two 64 x 64 -> 128-bit products, key bumped by
// the Weyl constants between rounds.
__device__ __forceinline__ void philox4x64_10(unsigned long long c[4], unsigned long long k0, unsigned long long k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const unsigned long long p0 = 0xD2E7470EE14C6C93ull * c[0], h0 = __umul64hi(0xD2E7470EE14C6C93ull, c[0]);
        const unsigned long long p1 = 0xCA5A826395121157ull * c[2], h1 = __umul64hi(0xCA5A826395121157ull, c[2]);
        const unsigned long long n0 = h1 ^ c[1] ^ k0, n2 = h0 ^ c[3] ^ k1;
        c[0] = n0;
        c[1] = p1;
        c[2] = n2;
        c[3] = p0;
        k0 += 0x9E3779B97F4A7C15ull;
        k1 += 0xBB67AE8584CAA73Bull;
    }
}

// The three normal deviates of atom i at step t (Box-Muller on words (0, 1)
// and (2, 3) of the Philox block; uniforms (w >> 11) 2^-53).
__device__ __forceinline__ void normals3(unsigned long long seed, unsigned long long step, int i, double R[3]) {
    unsigned long long w[4] = {step, (unsigned long long)i, 0ull, 0ull};
    philox4x64_10(w, seed, 0ull);
    double u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = (double)(w[q] >> 11) * 0x1.0p-53;
    const double r0 = sqrt(-2.0 * log(1.0 - u[0])), r1 = sqrt(-2.0 * log(1.0 - u[2]));
    double s0, c0, s1, c1;
    sincospi(2.0 * u[1], &s0, &c0);
    sincospi(2.0 * u[3], &s1, &c1);
    R[0] = r0 * c0;
    R[1] = r0 * s0;
    R[2] = r1 * c1;
}

// step[0]: index of the current step; step[1]: first step of the run.
__global__ void k_lfmiddle(int n, const int8_t* __restrict__ species, double* __restrict__ x, double* __restrict__ v,
                           const float* __restrict__ F, LgvConsts c, const long long* __restrict__ step) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int s = species[i] & 7;
    double R[3];
    normals3(c.seed, (unsigned long long)step[0], i, R);
    const double am = c.acc_m[s], sg = c.sigma[s];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
        double vv = v[3 * i + q] + c.dt * (double)F[3 * i + q] * am;
        double xx = x[3 * i + q] + 0.5 * c.dt * vv;
        vv = c.a * vv + sg * R[q];
        xx += 0.5 * c.dt * vv;
        v[3 * i + q] = vv;
        x[3 * i + q] = xx;
    }
}

// Records the step's potential energy (E_series[step - first], when given)
// and advances the step counter.
__global__ void k_step_tick(long long* step, const double* __restrict__ E_now, double* __restrict__ E_series) {
    if (E_series) E_series[step[0] - step[1]] = *E_now;
    step[0] += 1;
}

__global__ void k_normals(unsigned long long seed, long long step, int n, double* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double R[3];
    normals3(seed, (unsigned long long)step, i, R);
    out[3 * i] = R[0];
    out[3 * i + 1] = R[1];
    out[3 * i + 2] = R[2];
}

}  // namespace

struct mlp_langevin {
    mlp_system* s = nullptr;
    mlp_langevin_params p{};
    LgvConsts c{};
    void* dev_block = nullptr;
    long long* d_step = nullptr;   // [2]
    double* d_Enow = nullptr;
    float* d_F = nullptr;          // [n][3]
    long long* h_step = nullptr;   // pinned [2]
    cudaStream_t own = nullptr;    // graph mode runs here (the legacy default stream cannot be captured)
    cudaEvent_t after_caller = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    // what the captured step was built for
    double* g_x = nullptr;
    double* g_v = nullptr;
    double* g_E = nullptr;
    bool started = false;          // the system's list was built by a step of this integrator
};

namespace {

void drop_graph(mlp_langevin* L) {
    if (L->exec) cudaGraphExecDestroy(L->exec);
    if (L->graph) cudaGraphDestroy(L->graph);
    L->exec = nullptr;
    L->graph = nullptr;
}

// One step: evaluation at x, then the update and the tick.
int enqueue_step(mlp_langevin* L, double* d_x, double* d_v, double* d_energy, cudaStream_t st, bool rebuild) {
    mlp_system* s = L->s;
    EvalSpec sp = sys_spec(s, d_x);
    sp.force_rebuild = rebuild;
    sp.d_E = L->d_Enow;
    sp.d_F = L->d_F;
    int rc = enqueue_eval(s->ws, s->w->dw, sp, st);
    if (rc) return rc;
    const int n = s->n;
    MLP_LAUNCH("lfmiddle", st,
               k_lfmiddle<<<(n + 127) / 128, 128, 0, st>>>(n, s->d_species, d_x, d_v, L->d_F, L->c, L->d_step));
    MLP_LAUNCH("step_tick", st, k_step_tick<<<1, 1, 0, st>>>(L->d_step, L->d_Enow, d_energy));
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? MLP_OK : cuda_error(e, "integrator launch");
}

}  // namespace

extern "C" {

int mlp_langevin_create(mlp_system* s, const mlp_langevin_params* p, mlp_langevin** out) {
    clear_error();
    if (!s || !p || !out) return set_error(MLP_EINVAL, "NULL argument");
    *out = nullptr;
    if (!(p->dt_fs > 0.0 && p->dt_fs < 1e3) || !(p->friction_per_ps >= 0.0 && p->friction_per_ps < 1e9) ||
        !(p->temperature_K >= 0.0 && p->temperature_K < 1e9))
        return set_error(MLP_EINVAL, "need dt > 0, friction >= 0, temperature >= 0 (finite)");
    int rc = sys_finish_pending(s);
    if (rc) return rc;
    mlp_langevin* L = new (std::nothrow) mlp_langevin();
    if (!L) return set_error(MLP_ENOMEM, "host allocation failed");
    L->s = s;
    L->p = *p;
    const double a = exp(-p->friction_per_ps * 1e-3 * p->dt_fs);
    const double kT = kBoltz * p->temperature_K;
    L->c.dt = p->dt_fs;
    L->c.a = a;
    for (int e = 0; e < 8; ++e) {
        const double m = kMass[e < kNSpecies ? e : 0];
        L->c.acc_m[e] = kAcc / m;
        L->c.sigma[e] = sqrt((1.0 - a * a) * kT / (m * kKE));
    }
    L->c.seed = p->seed;
    const size_t n = (size_t)s->n;
    const size_t bytes = 256 + 256 + ((12 * n + 255) / 256) * 256;
    L->dev_block = dev_alloc(bytes);
    if (!L->dev_block) {
        delete L;
        return set_error(MLP_ENOMEM, "device allocation of the integrator state failed");
    }
    char* d = static_cast<char*>(L->dev_block);
    L->d_step = reinterpret_cast<long long*>(d);
    L->d_Enow = reinterpret_cast<double*>(d + 256);
    L->d_F = reinterpret_cast<float*>(d + 512);
    cudaError_t e = cudaMallocHost(reinterpret_cast<void**>(&L->h_step), 2 * sizeof(long long));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&L->own, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&L->after_caller, cudaEventDisableTiming);
    if (e != cudaSuccess) {
        mlp_langevin_destroy(L);
        return cuda_error(e, "integrator setup");
    }
    *out = L;
    return MLP_OK;
}

void mlp_langevin_destroy(mlp_langevin* L) {
    if (!L) return;
    if (L->own) cudaStreamSynchronize(L->own);
    drop_graph(L);
    if (L->after_caller) cudaEventDestroy(L->after_caller);
    if (L->own) cudaStreamDestroy(L->own);
    if (L->h_step) cudaFreeHost(L->h_step);
    dev_free(L->dev_block);
    delete L;
}

int mlp_langevin_run(mlp_langevin* L, double* d_x, double* d_v, int64_t step0, int32_t n_steps, double* d_energy,
                     void* stream) {
    clear_error();
    if (!L || !d_x || !d_v) return set_error(MLP_EINVAL, "NULL argument");
    if (n_steps < 0 || step0 < 0) return set_error(MLP_EINVAL, "n_steps and step0 must be >= 0");
    if (n_steps == 0) return MLP_OK;
    mlp_system* s = L->s;
    int rc = sys_finish_pending(s);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (L->p.use_graph) {
        // graph mode: the integrator's own stream, after the caller's work
        cudaError_t e0 = cudaEventRecord(L->after_caller, st);
        if (e0 == cudaSuccess) e0 = cudaStreamWaitEvent(L->own, L->after_caller, 0);
        if (e0 != cudaSuccess) return cuda_error(e0, "stream ordering");
        st = L->own;
    }
    const bool skin = s->cut.skin > 0.0;
    // the step counter and the run's first step, in device memory
    L->h_step[0] = step0;
    L->h_step[1] = step0;
    cudaError_t e = cudaMemcpyAsync(L->d_step, L->h_step, 2 * sizeof(long long), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync(step)");
    int done = 0;
    // first step: (re)builds the list when there is no valid one; with a skin
    // the later steps rely on the device's displacement guard
    if (!skin || !L->started || !s->nbr_valid) {
        rc = enqueue_step(L, d_x, d_v, d_energy, st, true);
        if (rc) return rc;
        ++done;
        L->started = true;
        s->nbr_valid = true;
    }
    const bool rebuild = !skin;
    if (L->p.use_graph && done < n_steps) {
        if (L->exec && (L->g_x != d_x || L->g_v != d_v || L->g_E != d_energy)) drop_graph(L);
        if (!L->exec) {
            e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
            if (e != cudaSuccess) return cuda_error(e, "cudaStreamBeginCapture");
            rc = enqueue_step(L, d_x, d_v, d_energy, st, rebuild);
            cudaGraph_t g = nullptr;
            e = cudaStreamEndCapture(st, &g);
            if (rc) {
                if (g) cudaGraphDestroy(g);
                return rc;
            }
            if (e != cudaSuccess) return cuda_error(e, "cudaStreamEndCapture");
            e = cudaGraphInstantiate(&L->exec, g, 0);
            if (e != cudaSuccess) {
                cudaGraphDestroy(g);
                L->exec = nullptr;
                return cuda_error(e, "cudaGraphInstantiate");
            }
            L->graph = g;
            L->g_x = d_x;
            L->g_v = d_v;
            L->g_E = d_energy;
        }
        for (; done < n_steps; ++done) {
            e = cudaGraphLaunch(L->exec, st);
            if (e != cudaSuccess) return cuda_error(e, "cudaGraphLaunch");
        }
    } else {
        for (; done < n_steps; ++done) {
            rc = enqueue_step(L, d_x, d_v, d_energy, st, rebuild);
            if (rc) return rc;
        }
    }
    s->calls += n_steps;
    s->kept = false;
    // every step's error flags went to the sticky word: read them once
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    rc = check_counters(s->ws);
    int sticky = 0;
    e = cudaMemcpy(&sticky, s->ws.err_sticky, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpy(error flags)");
    if (sticky) {
        cudaMemset(s->ws.err_sticky, 0, sizeof(int));
        cudaStreamSynchronize(nullptr);
        if (!rc) {
            if (sticky & 4) return set_error(MLP_EINVAL, "bad input during the run");
            if (sticky & 8) return set_error(MLP_ECUDA, "tensor-core network kernel error during the run");
            return set_error(MLP_EOVERFLOW, "neighbor capacity exceeded during the run");
        }
    }
    return rc;
}

int mlp_debug_langevin_normals(uint64_t seed, int64_t step, int32_t n, double* normals) {
    clear_error();
    if (!normals || n <= 0) return set_error(MLP_EINVAL, "bad arguments");
    int rc = check_cuda_device();
    if (rc) return rc;
    double* d = static_cast<double*>(dev_alloc(24 * (size_t)n));
    if (!d) return set_error(MLP_ENOMEM, "device allocation failed");
    k_normals<<<(n + 127) / 128, 128>>>(seed, step, n, d);
    cudaError_t e = cudaMemcpy(normals, d, 24 * (size_t)n, cudaMemcpyDeviceToHost);
    dev_free(d);
    return e == cudaSuccess ? MLP_OK : cuda_error(e, "mlp_debug_langevin_normals");
}

}  // extern "C"
