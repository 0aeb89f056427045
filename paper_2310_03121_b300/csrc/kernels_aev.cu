// Atomic environment vectors (forward) and their backward to forces.
//
// AEV of atom i (ANI atom-centered symmetry functions; the paper names them
// as the NNPOps bottleneck, section "Optimization Through NNPOps"):
//   radial  G[16 s_j + k]            += 0.25 exp(-eta_R (r_ij - R_k)^2) fc(r_ij; 5.1)
//   angular G[112 + 32 p + 8 a + z]  += 2 ((1 + cos(theta' - Z_z)) / 2)^zeta
//                                       exp(-eta_A ((r_ij + r_ik)/2 - A_a)^2)
//                                       fc(r_ij; 3.5) fc(r_ik; 3.5)
// for unordered neighbor pairs (j, k), theta' = acos(0.95 cos theta_ijk),
// p = unordered element pair index. cos(theta' - Z) is formed as
// cos theta' cos Z + sin theta' sin Z, so no acos is evaluated.
//
// Work decomposition (one warp per atom, 8 warps per block):
//   * the atom's neighbors within 5.1 A are staged in shared memory as
//     (dx, dy, dz, r) with their cutoff values; the ones within 3.5 A form
//     the angular sub-list;
//   * radial: lane = (half, k): 16 shift lanes x 2 neighbor streams, each
//     lane owns its own accumulator column per element -> no atomics;
//   * angular: triples are taken four at a time, lane = (t, z): the lane
//     evaluates the angle factor of section z and the distance factor of
//     shift z & 3 for triple t; then, for each of the four triples in turn,
//     lane (a, z) multiplies the shuffled factors and adds them to its own
//     column 32 p + 8 a + z (conflict-free, fixed order -> deterministic).
// The backward recomputes the same terms with their derivatives, contracts
// them with dE/dG, and accumulates per-neighbor gradients in shared memory
// before one FP64 atomic per (atom, neighbor, axis) into the global sums.
#include <cuda_bf16.h>

#include "common.cuh"
#include "kernels.cuh"

namespace mlp {

__constant__ AevConsts c_aev;

void init_constants_for_current_device() {
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 64 && done[dev]) return;
    AevConsts h;
    const double pi = 3.14159265358979323846;
    for (int k = 0; k < kRadShifts; ++k) h.shf_r[k] = (float)(0.8 + k * (4.9 - 0.8) / 15.0);
    for (int a = 0; a < kAngA; ++a) h.shf_a[a] = (float)(0.8 + a * (kRcAng - 0.8) / 4.0);
    for (int z = 0; z < kAngZ; ++z) {
        double Z = (2.0 * z + 1.0) * pi / 16.0;
        h.cos_z[z] = (float)cos(Z);
        h.sin_z[z] = (float)sin(Z);
    }
    cudaMemcpyToSymbol(c_aev, &h, sizeof(h));
    if (dev < 64) done[dev] = true;
}

namespace {

constexpr int kWarps = 8;
constexpr int kMaxRad = 160;
constexpr unsigned kFull = 0xffffffffu;

template <bool FAST>
struct M;
template <>
struct M<false> {   // accurate FP32 library functions (FP32 path)
    static __device__ __forceinline__ float ex(float x) { return expf(x); }
    static __device__ __forceinline__ float pw(float b, float e) { return powf(b, e); }
    static __device__ __forceinline__ float cpi(float x) { return cospif(x); }
    static __device__ __forceinline__ float spi(float x) { return sinpif(x); }
    static __device__ __forceinline__ float sq(float x) { return sqrtf(x); }
    static __device__ __forceinline__ float dv(float a, float b) { return a / b; }
};
template <>
struct M<true> {    // hardware approximations (BF16-network path)
    static __device__ __forceinline__ float ex(float x) { return __expf(x); }
    static __device__ __forceinline__ float pw(float b, float e) { return __powf(b, e); }
    static __device__ __forceinline__ float cpi(float x) { return __cosf(3.14159265358979f * x); }
    static __device__ __forceinline__ float spi(float x) { return __sinf(3.14159265358979f * x); }
    static __device__ __forceinline__ float sq(float x) { return x * rsqrtf(fmaxf(x, 1e-30f)); }
    static __device__ __forceinline__ float dv(float a, float b) { return __fdividef(a, b); }
};

struct NbrStage {
    float4 d[kMaxRad];    // dx, dy, dz, r of neighbors within 5.1 A
    float fc[kMaxRad];    // fc(r; 5.1)
    float dfc[kMaxRad];   // d fc / dr
    int sp[kMaxRad];      // element
    int idx[kMaxRad];     // atom index
    int ang[kMaxAng];     // slot (into the arrays above) of neighbors within 3.5 A
    float fca[kMaxAng];   // fc(r; 3.5)
    float dfca[kMaxAng];
};

constexpr int kAccFloats = 2 * kRadLen + kAngLen;   // two radial halves + angular
constexpr size_t kAevSmemPerWarp = sizeof(NbrStage) + kAccFloats * sizeof(float);
constexpr size_t kForceSmemPerWarp = sizeof(NbrStage) + (kAevLen + 3 * kMaxRad) * sizeof(float);

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Stages atom i's neighbors; returns the radial count, sets the angular one.
template <bool FAST, bool DERIV>
__device__ __forceinline__ int stage(const AevArgs& a, int i, int lane, const float4& hi_i, const float4& lo_i,
                                     NbrStage& s, int& mA) {
    const int cnt = min(a.nbr_cnt[i], a.cap);
    const int* row = a.nbr + (size_t)i * a.cap;
    int mR = 0;
    mA = 0;
    for (int base = 0; base < cnt; base += 32) {
        int q = base + lane;
        bool inR = false, inA = false;
        float3 d = make_float3(0.f, 0.f, 0.f);
        float r = 0.f;
        int sj = 0, j = 0;
        if (q < cnt) {
            j = row[q];
            float4 hj = a.hi[j], lj = a.lo[j];
            d = displacement(hi_i, lo_i, hj, lj, a.box);
            r = sqrtf(d.x * d.x + d.y * d.y + d.z * d.z);
            inR = r < kRcRad;
            inA = r < kRcAng;
            sj = species_of(hj);
        }
        unsigned bR = __ballot_sync(kFull, inR);
        unsigned bA = __ballot_sync(kFull, inA);
        int pR = mR + __popc(bR & lanemask_lt());
        int pA = mA + __popc(bA & lanemask_lt());
        if (inR && pR < kMaxRad) {
            s.d[pR] = make_float4(d.x, d.y, d.z, r);
            s.sp[pR] = sj;
            s.idx[pR] = j;
            s.fc[pR] = 0.5f * M<FAST>::cpi(r * (1.f / kRcRad)) + 0.5f;
            if (DERIV) s.dfc[pR] = -0.5f * (3.14159265358979f / kRcRad) * M<FAST>::spi(r * (1.f / kRcRad));
            if (inA && pA < kMaxAng) {
                s.ang[pA] = pR;
                s.fca[pA] = 0.5f * M<FAST>::cpi(r * (1.f / kRcAng)) + 0.5f;
                if (DERIV) s.dfca[pA] = -0.5f * (3.14159265358979f / kRcAng) * M<FAST>::spi(r * (1.f / kRcAng));
            }
        }
        mR += __popc(bR);
        mA += __popc(bA);
    }
    if (mR > kMaxRad || mA > kMaxAng) {
        // the evaluation is reported invalid by the host; keep every index in range
        if (lane == 0) atomicMax(&a.ctr->ang_overflow, max(mR, mA));
        mR = min(mR, kMaxRad);
        mA = 0;
    }
    __syncwarp();
    return mR;
}

// Next unordered pair (j < k) `step` positions further in row-major order.
__device__ __forceinline__ void advance_pair(int& j, int& k, int step, int m) {
    k += step;
    while (k >= m && j < m) {
        k = k - m + j + 2;
        ++j;
    }
}

template <bool FAST, typename OutT>
__device__ __forceinline__ void store_row(OutT* out, const float* acc, int lane);

template <>
__device__ __forceinline__ void store_row<false, float>(float* out, const float* acc, int lane) {
    for (int c = lane; c < kAevLd; c += 32) {
        float v = c < kRadLen ? acc[c] + acc[kRadLen + c] : (c < kAevLen ? acc[kRadLen + c] : 0.f);
        out[c] = v;
    }
}
template <>
__device__ __forceinline__ void store_row<true, float>(float* out, const float* acc, int lane) {
    store_row<false, float>(out, acc, lane);
}
// BF16 row; with out_lo != nullptr also the BF16 rounding of the remainder
// (G = G_hi + G_lo to ~16 bits), for the split-precision network.
template <bool FAST>
__device__ __forceinline__ void store_row_bf16(__nv_bfloat16* out, __nv_bfloat16* out_lo, const float* acc,
                                               int lane) {
    for (int c = 2 * lane; c < kAevLd; c += 64) {
        float v0, v1;
        v0 = c < kRadLen ? acc[c] + acc[kRadLen + c] : (c < kAevLen ? acc[kRadLen + c] : 0.f);
        int c1 = c + 1;
        v1 = c1 < kRadLen ? acc[c1] + acc[kRadLen + c1] : (c1 < kAevLen ? acc[kRadLen + c1] : 0.f);
        const __nv_bfloat162 h = __floats2bfloat162_rn(v0, v1);
        *reinterpret_cast<__nv_bfloat162*>(out + c) = h;
        if (out_lo) {
            const float2 f = __bfloat1622float2(h);
            *reinterpret_cast<__nv_bfloat162*>(out_lo + c) = __floats2bfloat162_rn(v0 - f.x, v1 - f.y);
        }
    }
}

template <bool FAST, typename OutT>
__global__ void __launch_bounds__(kWarps * 32) k_aev(AevArgs a, OutT* __restrict__ G, OutT* __restrict__ G_lo,
                                                      int* __restrict__ row_atom) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kWarps + w;
    if (i >= a.n) return;
    NbrStage& s = *reinterpret_cast<NbrStage*>(smem + w * kAevSmemPerWarp);
    float* acc = reinterpret_cast<float*>(smem + w * kAevSmemPerWarp + sizeof(NbrStage));
    const float4 hi_i = a.hi[i], lo_i = a.lo[i];

    for (int c = lane; c < kAccFloats; c += 32) acc[c] = 0.f;
    int mA;
    const int mR = stage<FAST, false>(a, i, lane, hi_i, lo_i, s, mA);

    // radial: lane (h, k) handles neighbors h, h + 2, ... for shift k
    {
        const int k = lane & 15, h = lane >> 4;
        const float Rk = c_aev.shf_r[k];
        float* accR = acc + h * kRadLen;
        for (int q = h; q < mR; q += 2) {
            float dr = s.d[q].w - Rk;
            accR[s.sp[q] * kRadShifts + k] += 0.25f * M<FAST>::ex(-kEtaRad * dr * dr) * s.fc[q];
        }
    }
    // angular: four triples per step
    {
        float* accA = acc + 2 * kRadLen;
        const int t = lane >> 3, z = lane & 7;
        const float cz = c_aev.cos_z[z], sz = c_aev.sin_z[z];
        const float Aown = c_aev.shf_a[z & 3];
        const int P = mA * (mA - 1) / 2;
        int j = 0, k = 1 + t;
        advance_pair(j, k, 0, mA);
        for (int base = 0; base < P; base += 4) {
            float Pz = 0.f, Ra = 0.f, f = 0.f;
            int p = 0;
            if (base + t < P) {
                const int js = s.ang[j], ks = s.ang[k];
                const float4 dj = s.d[js], dk = s.d[ks];
                float cos0 = M<FAST>::dv(dj.x * dk.x + dj.y * dk.y + dj.z * dk.z, dj.w * dk.w);
                float c = 0.95f * cos0;
                float sn = M<FAST>::sq(1.f - c * c);
                float b = 0.5f + 0.5f * (c * cz + sn * sz);
                Pz = 2.f * M<FAST>::pw(b, kZeta);
                float dr = 0.5f * (dj.w + dk.w) - Aown;
                Ra = M<FAST>::ex(-kEtaAng * dr * dr);
                f = s.fca[j] * s.fca[k];
                p = pair_index(s.sp[js], s.sp[ks]);
            }
#pragma unroll
            for (int tt = 0; tt < 4; ++tt) {
                float Pv = __shfl_sync(kFull, Pz, tt * 8 + (lane & 7));
                float Rv = __shfl_sync(kFull, Ra, tt * 8 + (lane >> 3));
                float fv = __shfl_sync(kFull, f, tt * 8);
                int pv = __shfl_sync(kFull, p, tt * 8);
                if (base + tt < P) accA[pv * 32 + lane] += Pv * Rv * fv;
            }
            advance_pair(j, k, 4, mA);
        }
    }
    __syncwarp();
    const int si = species_of(hi_i);
    const int row = row_base(a.ctr->species, si) + a.rank[i];
    if constexpr (sizeof(OutT) == 4) {
        store_row<FAST, float>(reinterpret_cast<float*>(G) + (size_t)row * kAevLd, acc, lane);
    } else {
        store_row_bf16<FAST>(reinterpret_cast<__nv_bfloat16*>(G) + (size_t)row * kAevLd,
                             G_lo ? reinterpret_cast<__nv_bfloat16*>(G_lo) + (size_t)row * kAevLd : nullptr, acc,
                             lane);
    }
    if (lane == 0) row_atom[row] = i;
}

template <bool FAST>
__global__ void __launch_bounds__(kWarps * 32) k_forces(AevArgs a, const float* __restrict__ dG,
                                                         double* __restrict__ grad) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kWarps + w;
    if (i >= a.n) return;
    NbrStage& s = *reinterpret_cast<NbrStage*>(smem + w * kForceSmemPerWarp);
    float* gs = reinterpret_cast<float*>(smem + w * kForceSmemPerWarp + sizeof(NbrStage));
    float* fslot = gs + kAevLen;
    const float4 hi_i = a.hi[i], lo_i = a.lo[i];
    const int si = species_of(hi_i);
    const int row = row_base(a.ctr->species, si) + a.rank[i];
    const float* grow = dG + (size_t)row * kAevLd;
    for (int c = lane; c < kAevLen; c += 32) gs[c] = grow[c];
    for (int c = lane; c < 3 * kMaxRad; c += 32) fslot[c] = 0.f;
    int mA;
    const int mR = stage<FAST, true>(a, i, lane, hi_i, lo_i, s, mA);

    float fix = 0.f, fiy = 0.f, fiz = 0.f;   // dE/dr_i partial sums of this lane
    // radial: dT/dr = 0.25 exp(-eta (r-R)^2) (-2 eta (r-R) fc + fc')
    {
        const int k = lane & 15, h = lane >> 4;
        const float Rk = c_aev.shf_r[k];
        const int nq = (mR + 1) >> 1;
        for (int q2 = 0; q2 < nq; ++q2) {
            const int q = 2 * q2 + h;
            float term = 0.f;
            if (q < mR) {
                float dr = s.d[q].w - Rk;
                term = gs[s.sp[q] * kRadShifts + k] * 0.25f * M<FAST>::ex(-kEtaRad * dr * dr) *
                       (-2.f * kEtaRad * dr * s.fc[q] + s.dfc[q]);
            }
            term += __shfl_xor_sync(kFull, term, 8);
            term += __shfl_xor_sync(kFull, term, 4);
            term += __shfl_xor_sync(kFull, term, 2);
            term += __shfl_xor_sync(kFull, term, 1);
            if (q < mR && k == 0) {
                const float4 d = s.d[q];
                const float sc = M<FAST>::dv(term, d.w);
                fslot[3 * q] += sc * d.x;
                fslot[3 * q + 1] += sc * d.y;
                fslot[3 * q + 2] += sc * d.z;
                fix -= sc * d.x;
                fiy -= sc * d.y;
                fiz -= sc * d.z;
            }
        }
    }
    __syncwarp();
    // angular
    {
        const int t = lane >> 3, z = lane & 7;
        const float cz = c_aev.cos_z[z], sz = c_aev.sin_z[z];
        const int P = mA * (mA - 1) / 2;
        int j = 0, k = 1 + t;
        advance_pair(j, k, 0, mA);
        for (int base = 0; base < P; base += 4) {
            const bool valid = base + t < P;
            float Sc = 0.f, Srj = 0.f, Srk = 0.f;
            float4 dj = make_float4(0.f, 0.f, 0.f, 1.f), dk = dj;
            int js = 0, ks = 0;
            float cos0 = 0.f;
            if (valid) {
                js = s.ang[j];
                ks = s.ang[k];
                dj = s.d[js];
                dk = s.d[ks];
                cos0 = M<FAST>::dv(dj.x * dk.x + dj.y * dk.y + dj.z * dk.z, dj.w * dk.w);
                const float c = 0.95f * cos0;
                const float sn = M<FAST>::sq(1.f - c * c);
                const float cm = c * cz + sn * sz;
                const float sm = sn * cz - c * sz;
                const float b = 0.5f + 0.5f * cm;
                const float Pz = 2.f * M<FAST>::pw(b, kZeta);
                const float dPdc = M<FAST>::dv(kZeta * Pz * sm, 2.f * b * sn);
                const float fj = s.fca[j], fk = s.fca[k], dfj = s.dfca[j], dfk = s.dfca[k];
                const float f = fj * fk;
                const float rbar = 0.5f * (dj.w + dk.w);
                const int p = pair_index(s.sp[js], s.sp[ks]);
                const float* gp = gs + kRadLen + 32 * p + z;
#pragma unroll
                for (int aa = 0; aa < kAngA; ++aa) {
                    const float dr = rbar - c_aev.shf_a[aa];
                    const float R = M<FAST>::ex(-kEtaAng * dr * dr);
                    const float dR = -2.f * kEtaAng * dr * R;
                    const float gg = gp[8 * aa];
                    Sc += gg * dPdc * R * f;
                    Srj += gg * Pz * (0.5f * dR * f + R * dfj * fk);
                    Srk += gg * Pz * (0.5f * dR * f + R * fj * dfk);
                }
            }
#pragma unroll
            for (int o = 4; o > 0; o >>= 1) {
                Sc += __shfl_xor_sync(kFull, Sc, o);
                Srj += __shfl_xor_sync(kFull, Srj, o);
                Srk += __shfl_xor_sync(kFull, Srk, o);
            }
            if (valid && z == 0) {
                const float rj = dj.w, rk = dk.w;
                const float A = 0.95f * Sc * M<FAST>::dv(1.f, rj * rk);
                const float Bj = 0.95f * Sc * cos0 * M<FAST>::dv(1.f, rj * rj) - M<FAST>::dv(Srj, rj);
                const float Bk = 0.95f * Sc * cos0 * M<FAST>::dv(1.f, rk * rk) - M<FAST>::dv(Srk, rk);
                // dE/d(d_ij) = A d_ik - Bj d_ij ; dE/d(d_ik) = A d_ij - Bk d_ik
                const float gjx = A * dk.x - Bj * dj.x, gjy = A * dk.y - Bj * dj.y, gjz = A * dk.z - Bj * dj.z;
                const float gkx = A * dj.x - Bk * dk.x, gky = A * dj.y - Bk * dk.y, gkz = A * dj.z - Bk * dk.z;
                atomicAdd(&fslot[3 * js], gjx);
                atomicAdd(&fslot[3 * js + 1], gjy);
                atomicAdd(&fslot[3 * js + 2], gjz);
                atomicAdd(&fslot[3 * ks], gkx);
                atomicAdd(&fslot[3 * ks + 1], gky);
                atomicAdd(&fslot[3 * ks + 2], gkz);
                fix -= gjx + gkx;
                fiy -= gjy + gky;
                fiz -= gjz + gkz;
            }
            advance_pair(j, k, 4, mA);
        }
    }
    __syncwarp();
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        fix += __shfl_xor_sync(kFull, fix, o);
        fiy += __shfl_xor_sync(kFull, fiy, o);
        fiz += __shfl_xor_sync(kFull, fiz, o);
    }
    if (lane == 0) {
        atomicAdd(&grad[3 * (size_t)i], (double)fix);
        atomicAdd(&grad[3 * (size_t)i + 1], (double)fiy);
        atomicAdd(&grad[3 * (size_t)i + 2], (double)fiz);
    }
    for (int q = lane; q < mR; q += 32) {
        const int j = s.idx[q];
        atomicAdd(&grad[3 * (size_t)j], (double)fslot[3 * q]);
        atomicAdd(&grad[3 * (size_t)j + 1], (double)fslot[3 * q + 1]);
        atomicAdd(&grad[3 * (size_t)j + 2], (double)fslot[3 * q + 2]);
    }
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

}  // namespace

void launch_aev_f32(cudaStream_t st, const AevArgs& a, float* G, int* row_atom, bool fast) {
    const size_t sm = kWarps * kAevSmemPerWarp;
    const int gs = (a.n + kWarps - 1) / kWarps;
    if (fast) {
        static bool once = (set_smem(k_aev<true, float>, sm), true);
        (void)once;
        MLP_LAUNCH("aev", st, k_aev<true, float><<<gs, kWarps * 32, sm, st>>>(a, G, nullptr, row_atom));
    } else {
        static bool once = (set_smem(k_aev<false, float>, sm), true);
        (void)once;
        MLP_LAUNCH("aev", st, k_aev<false, float><<<gs, kWarps * 32, sm, st>>>(a, G, nullptr, row_atom));
    }
}

void launch_aev_bf16(cudaStream_t st, const AevArgs& a, __nv_bfloat16* G, __nv_bfloat16* G_lo, int* row_atom,
                     bool fast) {
    const size_t sm = kWarps * kAevSmemPerWarp;
    const int gs = (a.n + kWarps - 1) / kWarps;
    if (fast) {
        static bool once = (set_smem(k_aev<true, __nv_bfloat16>, sm), true);
        (void)once;
        MLP_LAUNCH("aev", st, k_aev<true, __nv_bfloat16><<<gs, kWarps * 32, sm, st>>>(a, G, G_lo, row_atom));
    } else {
        static bool once = (set_smem(k_aev<false, __nv_bfloat16>, sm), true);
        (void)once;
        MLP_LAUNCH("aev", st, k_aev<false, __nv_bfloat16><<<gs, kWarps * 32, sm, st>>>(a, G, G_lo, row_atom));
    }
}

void launch_forces(cudaStream_t st, const AevArgs& a, const float* dG, double* grad, bool fast) {
    const size_t sm = kWarps * kForceSmemPerWarp;
    const int gs = (a.n + kWarps - 1) / kWarps;
    if (fast) {
        static bool once = (set_smem(k_forces<true>, sm), true);
        (void)once;
        MLP_LAUNCH("forces", st, k_forces<true><<<gs, kWarps * 32, sm, st>>>(a, dG, grad));
    } else {
        static bool once = (set_smem(k_forces<false>, sm), true);
        (void)once;
        MLP_LAUNCH("forces", st, k_forces<false><<<gs, kWarps * 32, sm, st>>>(a, dG, grad));
    }
}

}  // namespace mlp
