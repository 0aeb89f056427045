// Per-element networks on the 5th-generation tensor cores (BF16 x BF16 ->
// FP32): the one dense contraction of the path (paper, section "Performance
// of MLPs": one ANI net per element, evaluated for every atom).
//
// One CTA (4 warps; thread r owns row r of the tile = TMEM lane r) processes
// 128-row tiles of one element, persistent over the tiles. The six GEMMs of
// the forward and backward run back to back without leaving the SM:
//   F1  D[128x256] = G[128x1024] W1^T   G and W1 streamed by TMA in 64-wide K chunks (4 stages)
//   E1  h1 = celu(D + b1)               -> shared memory, BF16, A-operand layout
//   F2  D[128x192] = h1 W2^T            W2 streamed (2 stages)
//   E2  h2 = celu(D + b2)               -> shared memory
//   F3  D[128x160] = h2 W3^T            W3 streamed
//   E3  e = w4 . celu(D + b3) + b4      -> global; g3 = w4 * celu'(z3) -> shared memory
//   B3  D[128x192] = g3 W3              W3^T streamed;  g2 = D * celu'(z2) (over h2)
//   B2  D[128x256] = g2 W2              W2^T streamed;  g1 = D * celu'(z1) (over h1)
//   B1  dE/dG[128x1024] = g1 W1         W1^T streamed in four 256-column blocks -> global FP32
// celu'(z) comes from the stored BF16 activation: 1 if h > 0 else h / alpha + 1.
// Accumulators live in tensor memory (512 columns: two 256-column halves).
// Thread 0 issues the TMA loads (cp.async.bulk.tensor) and the tcgen05.mma
// instructions; all 128 threads run the epilogues (tcgen05.ld -> registers ->
// shared or global memory). Operands in shared memory use the 128-byte
// swizzled K-major layout that TMA writes. Every wait is bounded in time: on
// expiry the CTA records an error, drains its own copies and MMAs, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "common.cuh"
#include "engine.cuh"
#include "kernels.cuh"

namespace mlp {
namespace {

constexpr int kThreads = 128;
constexpr uint32_t kAtom = 128 * 128;          // 128 rows x 64 BF16 (one K atom of a 128-row operand)
constexpr uint32_t kOffH1 = 0;                 // h1 / g1: 4 atoms
constexpr uint32_t kOffH2 = 4 * kAtom;         // h2 / g2: 3 atoms
constexpr uint32_t kOffG3 = 7 * kAtom;         // g3: 3 atoms (160 of 192 columns used)
constexpr uint32_t kOffRB = 10 * kAtom;        // streamed weights: 2 stages x 32 KB
constexpr uint32_t kRBStage = 32768;
constexpr uint32_t kF1Stage = 49152;           // F1: A (16 KB) + B (32 KB) per stage, overlaying [0, 192 KB)
constexpr int kNF1 = 4;
constexpr uint32_t kSmemUsed = kOffRB + 2 * kRBStage;   // 229,376 bytes
constexpr uint32_t kSmemAlloc = kSmemUsed + 1024;       // + alignment slack
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

enum { kBarF1Full = 0, kBarF1Empty = 4, kBarRBFull = 8, kBarRBEmpty = 10, kBarDone = 12, kNBars = 13 };

struct TcArgs {
    const Counters* ctr;
    const int* row_atom;
    const float *b1, *b2, *b3, *W4, *b4;
    float* e;
    float* dG;
    int backward;
    int* err;
};

// ------------------------------------------------------------------ PTX helpers
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on a phase: false after kWaitNs.
__device__ __noinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
    if (mbar_try(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitNs) return false;
    }
}
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar)
        : "memory");
}
__device__ __forceinline__ void fence_proxy_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups
// 1024 bytes apart (stride byte offset), descriptor version 1 (sm_100 family).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;             // leading byte offset: unused for swizzled K-major
    d |= (uint64_t)(1024 >> 4) << 32;   // stride byte offset
    d |= (uint64_t)1 << 46;             // descriptor version
    d |= (uint64_t)2 << 61;             // SWIZZLE_128B
    return d;
}
// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major, M x N.
__device__ __forceinline__ uint32_t idesc_bf16(int M, int N) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q) v[q] = __uint_as_float(r[q]);
}
__device__ __forceinline__ void st_shared_v4(uint32_t addr, uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
    asm volatile("st.shared.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(a), "r"(b), "r"(c), "r"(d) : "memory");
}
__device__ __forceinline__ uint4 ld_shared_v4(uint32_t addr) {
    uint4 v;
    asm volatile("ld.shared.v4.b32 {%0, %1, %2, %3}, [%4];" : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w) : "r"(addr)
                 : "memory");
    return v;
}

// Byte offset of (row, col) -- col a multiple of 8 -- in an operand region of
// 64-column swizzled atoms (the TMA SWIZZLE_128B image of a [rows x 64] box).
__device__ __forceinline__ uint32_t op_off(int row, int col) {
    const int atom = col >> 6, chunk = ((col & 63) >> 3) ^ (row & 7);
    return (uint32_t)atom * kAtom + (uint32_t)row * 128u + (uint32_t)chunk * 16u;
}
__device__ __forceinline__ uint32_t pack_bf16(float a, float b) {
    __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
    return *reinterpret_cast<uint32_t*>(&v);
}
__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }
__device__ __forceinline__ float celu_f(float x) { return x > 0.f ? x : kCeluAlpha * (__expf(x * (1.f / kCeluAlpha)) - 1.f); }
__device__ __forceinline__ float dcelu_f(float x) { return x > 0.f ? 1.f : __expf(x * (1.f / kCeluAlpha)); }
__device__ __forceinline__ float dcelu_h(float h) { return h > 0.f ? 1.f : h * (1.f / kCeluAlpha) + 1.f; }

// ------------------------------------------------------------------ issuing thread state
// Stage slots 0..3: F1 (A + B), 4..5: streamed weights of the other GEMMs.
struct Issuer {
    uint32_t bar0;          // shared address of barrier 0 (barriers are 8 bytes apart)
    uint32_t nfull[6];      // phases consumed per full barrier
    uint32_t nempty[6];     // phases consumed per empty barrier
    uint32_t pend;          // slots with an MMA commit not yet waited for
    uint32_t loaded;        // slots with a TMA load not yet consumed
    uint32_t f1_next, rb_next;
    bool ok;

    __device__ uint32_t bar(int i) const { return bar0 + 8u * (uint32_t)i; }
    __device__ uint32_t full(int si) const { return si < 4 ? bar(kBarF1Full + si) : bar(kBarRBFull + si - 4); }
    __device__ uint32_t empty(int si) const { return si < 4 ? bar(kBarF1Empty + si) : bar(kBarRBEmpty + si - 4); }

    __device__ bool acquire(int si) {
        if (pend & (1u << si)) {
            if (!mbar_wait(empty(si), nempty[si] & 1u)) return ok = false;
            nempty[si]++;
            pend &= ~(1u << si);
        }
        return true;
    }
    __device__ bool consume(int si) {
        if (!mbar_wait(full(si), nfull[si] & 1u)) return ok = false;
        nfull[si]++;
        loaded &= ~(1u << si);
        tc_fence_after();
        return true;
    }
    __device__ void release(int si) {
        mma_commit(empty(si));
        pend |= 1u << si;
    }
};

struct Job {
    const CUtensorMap* map;
    int brow;          // first weight row (element block + column block)
    int nc;            // K chunks of 64
    int lastk;         // 16-wide K steps in the last chunk
    uint32_t a_off;    // A operand region
    uint32_t d_col;    // TMEM column of the accumulator
    int N;
    uint32_t bytes;    // TMA bytes per chunk (N rows x 128 B)
    int st[4];
};

__device__ __forceinline__ bool load_rb(Issuer& I, uint32_t sbase, Job& J, int c) {
    const int si = J.st[c];
    if (!I.acquire(si)) return false;
    const uint32_t dst = sbase + kOffRB + (uint32_t)(si - 4) * kRBStage;
    mbar_expect_tx(I.full(si), J.bytes);
    tma_load_2d(dst, J.map, c * 64, J.brow, I.full(si));
    I.loaded |= 1u << si;
    return true;
}

__device__ bool job_prefetch(Issuer& I, uint32_t sbase, Job& J) {
    for (int c = 0; c < 2 && c < J.nc; ++c) {
        J.st[c] = 4 + (int)(I.rb_next & 1u);
        I.rb_next++;
        if (!load_rb(I, sbase, J, c)) return false;
    }
    return true;
}

__device__ bool job_run(Issuer& I, uint32_t sbase, uint32_t tmem, Job& J) {
    const uint32_t idesc = idesc_bf16(128, J.N);
    for (int c = 0; c < J.nc; ++c) {
        const int si = J.st[c];
        if (!I.consume(si)) return false;
        const uint32_t b_base = sbase + kOffRB + (uint32_t)(si - 4) * kRBStage;
        const uint32_t a_base = sbase + J.a_off + (uint32_t)c * kAtom;
        const int ks = (c == J.nc - 1) ? J.lastk : 4;
        for (int k = 0; k < ks; ++k)
            mma_bf16(tmem + J.d_col, sdesc(a_base + 32u * k), sdesc(b_base + 32u * k), idesc,
                     (c > 0 || k > 0) ? 1u : 0u);
        I.release(si);
        if (c >= 1 && c + 1 < J.nc) {
            J.st[c + 1] = J.st[c - 1];
            if (!load_rb(I, sbase, J, c + 1)) return false;
        }
    }
    mma_commit(I.bar(kBarDone));
    return true;
}

__device__ bool f1_run(Issuer& I, uint32_t sbase, uint32_t tmem, const CUtensorMap* mG, const CUtensorMap* mW1,
                       int row0, int s) {
    constexpr int nc = kAevLd / 64;   // 16
    const uint32_t idesc = idesc_bf16(128, kH1);
    int st[nc];
    auto load = [&](int c) -> bool {
        const int si = st[c];
        if (!I.acquire(si)) return false;
        const uint32_t dst = sbase + (uint32_t)si * kF1Stage;
        mbar_expect_tx(I.full(si), kF1Stage);
        tma_load_2d(dst, mG, c * 64, row0, I.full(si));
        tma_load_2d(dst + 16384u, mW1, c * 64, s * kH1, I.full(si));
        I.loaded |= 1u << si;
        return true;
    };
    for (int c = 0; c < kNF1; ++c) {
        st[c] = (int)(I.f1_next & 3u);
        I.f1_next++;
        if (!load(c)) return false;
    }
    for (int c = 0; c < nc; ++c) {
        const int si = st[c];
        if (!I.consume(si)) return false;
        const uint32_t a_base = sbase + (uint32_t)si * kF1Stage;
        for (int k = 0; k < 4; ++k)
            mma_bf16(tmem, sdesc(a_base + 32u * k), sdesc(a_base + 16384u + 32u * k), idesc,
                     (c > 0 || k > 0) ? 1u : 0u);
        I.release(si);
        if (c >= 1 && c + 3 < nc) {
            st[c + 3] = st[c - 1];
            if (!load(c + 3)) return false;
        }
    }
    mma_commit(I.bar(kBarDone));
    return true;
}

__global__ void __launch_bounds__(kThreads, 1)
    k_mlp_tc(const __grid_constant__ CUtensorMap mG, const __grid_constant__ CUtensorMap mW1,
             const __grid_constant__ CUtensorMap mW2, const __grid_constant__ CUtensorMap mW3,
             const __grid_constant__ CUtensorMap mW3t, const __grid_constant__ CUtensorMap mW2t,
             const __grid_constant__ CUtensorMap mW1t, TcArgs p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) unsigned long long bars[kNBars];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;

    Issuer I;
    I.bar0 = smem_u32(&bars[0]);
    for (int q = 0; q < 6; ++q) I.nfull[q] = I.nempty[q] = 0;
    I.pend = I.loaded = 0;
    I.f1_next = I.rb_next = 0;
    I.ok = true;
    uint32_t n_done = 0;

    if (tid == 0) {
        for (int q = 0; q < kNBars; ++q) mbar_init(smem_u32(&bars[q]), 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const uint32_t tl = tmem + ((uint32_t)(warp * 32) << 16);   // this warp's TMEM lanes
    const int r = tid;

    auto wait_done = [&]() {
        if (!mbar_wait(I.bar(kBarDone), n_done & 1u)) atomicExch(&abort_flag, 1);
        n_done++;
        __syncwarp();   // the epilogue's tcgen05.ld are warp-collective
        tc_fence_after();
    };
    auto sync_all = [&]() -> bool {
        fence_proxy_async();
        tc_fence_before();
        __syncthreads();
        tc_fence_after();
        return abort_flag == 0;
    };
    auto issue_fail = [&]() { atomicExch(&abort_flag, 1); };

    for (int t = blockIdx.x;; t += gridDim.x) {
        int s, row0, nvalid;
        if (!tile_info(p.ctr->species, t, s, row0, nvalid)) break;
        const float* b1 = p.b1 + s * kH1;
        const float* b2 = p.b2 + s * kH2;
        const float* b3 = p.b3 + s * kH3;
        const float* w4 = p.W4 + s * kH3;
        Job jF2{&mW2, s * kH2, 4, 4, kOffH1, 256, kH2, (uint32_t)kH2 * 128u, {0, 0, 0, 0}};
        Job jF3{&mW3, s * kH3, 3, 4, kOffH2, 0, kH3, (uint32_t)kH3 * 128u, {0, 0, 0, 0}};
        Job jB3{&mW3t, s * kH2, 3, 2, kOffG3, 256, kH2, (uint32_t)kH2 * 128u, {0, 0, 0, 0}};
        Job jB2{&mW2t, s * kH1, 3, 4, kOffH2, 0, kH1, (uint32_t)kH1 * 128u, {0, 0, 0, 0}};

        // ---- F1 -> E1
        if (tid == 0 && !f1_run(I, sbase, tmem, &mG, &mW1, row0, s)) issue_fail();
        wait_done();
        if (tid == 0 && I.ok && !job_prefetch(I, sbase, jF2)) issue_fail();
        for (int c0 = 0; c0 < kH1; c0 += 16) {
            float v[16];
            tmem_ld16(tl + (uint32_t)c0, v);
            uint32_t pk[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                pk[q] = pack_bf16(celu_f(v[2 * q] + __ldg(b1 + c0 + 2 * q)), celu_f(v[2 * q + 1] + __ldg(b1 + c0 + 2 * q + 1)));
            st_shared_v4(sbase + kOffH1 + op_off(r, c0), pk[0], pk[1], pk[2], pk[3]);
            st_shared_v4(sbase + kOffH1 + op_off(r, c0 + 8), pk[4], pk[5], pk[6], pk[7]);
        }
        if (!sync_all()) break;

        // ---- F2 -> E2
        if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jF2)) issue_fail();
        wait_done();
        if (tid == 0 && I.ok && !job_prefetch(I, sbase, jF3)) issue_fail();
        for (int c0 = 0; c0 < kH2; c0 += 16) {
            float v[16];
            tmem_ld16(tl + 256u + (uint32_t)c0, v);
            uint32_t pk[8];
#pragma unroll
            for (int q = 0; q < 8; ++q)
                pk[q] = pack_bf16(celu_f(v[2 * q] + __ldg(b2 + c0 + 2 * q)), celu_f(v[2 * q + 1] + __ldg(b2 + c0 + 2 * q + 1)));
            st_shared_v4(sbase + kOffH2 + op_off(r, c0), pk[0], pk[1], pk[2], pk[3]);
            st_shared_v4(sbase + kOffH2 + op_off(r, c0 + 8), pk[4], pk[5], pk[6], pk[7]);
        }
        if (!sync_all()) break;

        // ---- F3 -> E3 (energy, g3)
        if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jF3)) issue_fail();
        wait_done();
        if (tid == 0 && I.ok && p.backward && !job_prefetch(I, sbase, jB3)) issue_fail();
        {
            float es = 0.f;
            for (int c0 = 0; c0 < kH3; c0 += 16) {
                float v[16];
                tmem_ld16(tl + (uint32_t)c0, v);
                uint32_t pk[8];
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const float z0 = v[2 * q] + __ldg(b3 + c0 + 2 * q), z1 = v[2 * q + 1] + __ldg(b3 + c0 + 2 * q + 1);
                    const float w0 = __ldg(w4 + c0 + 2 * q), w1 = __ldg(w4 + c0 + 2 * q + 1);
                    es = fmaf(w0, celu_f(z0), es);
                    es = fmaf(w1, celu_f(z1), es);
                    pk[q] = pack_bf16(w0 * dcelu_f(z0), w1 * dcelu_f(z1));
                }
                if (p.backward) {
                    st_shared_v4(sbase + kOffG3 + op_off(r, c0), pk[0], pk[1], pk[2], pk[3]);
                    st_shared_v4(sbase + kOffG3 + op_off(r, c0 + 8), pk[4], pk[5], pk[6], pk[7]);
                }
            }
            if (r < nvalid) p.e[p.row_atom[row0 + r]] = es + __ldg(p.b4 + s);
        }
        if (!sync_all()) break;
        if (!p.backward) continue;

        // ---- B3 -> g2 (over h2)
        if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jB3)) issue_fail();
        wait_done();
        if (tid == 0 && I.ok && !job_prefetch(I, sbase, jB2)) issue_fail();
        for (int c0 = 0; c0 < kH2; c0 += 16) {
            float v[16];
            tmem_ld16(tl + 256u + (uint32_t)c0, v);
#pragma unroll
            for (int hlf = 0; hlf < 2; ++hlf) {
                const uint32_t a = sbase + kOffH2 + op_off(r, c0 + 8 * hlf);
                const uint4 h = ld_shared_v4(a);
                const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
                uint32_t o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float* vv = v + 8 * hlf + 2 * q;
                    o[q] = pack_bf16(vv[0] * dcelu_h(bf_lo(hw[q])), vv[1] * dcelu_h(bf_hi(hw[q])));
                }
                st_shared_v4(a, o[0], o[1], o[2], o[3]);
            }
        }
        if (!sync_all()) break;

        // ---- B2 -> g1 (over h1)
        if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jB2)) issue_fail();
        wait_done();
        Job jB1{&mW1t, s * kAevLd, 4, 4, kOffH1, 0, 256, 256u * 128u, {0, 0, 0, 0}};
        if (tid == 0 && I.ok && !job_prefetch(I, sbase, jB1)) issue_fail();
        for (int c0 = 0; c0 < kH1; c0 += 16) {
            float v[16];
            tmem_ld16(tl + (uint32_t)c0, v);
#pragma unroll
            for (int hlf = 0; hlf < 2; ++hlf) {
                const uint32_t a = sbase + kOffH1 + op_off(r, c0 + 8 * hlf);
                const uint4 h = ld_shared_v4(a);
                const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
                uint32_t o[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const float* vv = v + 8 * hlf + 2 * q;
                    o[q] = pack_bf16(vv[0] * dcelu_h(bf_lo(hw[q])), vv[1] * dcelu_h(bf_hi(hw[q])));
                }
                st_shared_v4(a, o[0], o[1], o[2], o[3]);
            }
        }
        if (!sync_all()) break;

        // ---- B1: four 256-column blocks of dE/dG, alternating TMEM halves
        bool aborted = false;
        for (int j = 0; j < 4; ++j) {
            if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jB1)) issue_fail();
            wait_done();
            const uint32_t dcol = jB1.d_col;
            if (j < 3) {
                jB1.brow = s * kAevLd + 256 * (j + 1);
                jB1.d_col = 256u * (uint32_t)((j + 1) & 1);
                if (tid == 0 && I.ok && !job_prefetch(I, sbase, jB1)) issue_fail();
            }
            float* out = p.dG + (size_t)(row0 + r) * kAevLd + 256 * j;
            for (int c0 = 0; c0 < 256; c0 += 16) {
                float v[16];
                tmem_ld16(tl + dcol + (uint32_t)c0, v);
                if (r < nvalid) {
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *reinterpret_cast<float4*>(out + c0 + 4 * q) = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
            }
            if (!sync_all()) {
                aborted = true;
                break;
            }
        }
        if (aborted) break;
    }

    // ---- teardown: drain own copies and MMAs (bounded), free tensor memory
    __syncthreads();
    if (abort_flag) {
        if (tid == 0) {
            atomicOr(p.err, 1);
            for (int si = 0; si < 6; ++si)
                if (I.loaded & (1u << si)) (void)mbar_wait(I.full(si), I.nfull[si] & 1u);
            mma_commit(I.bar(kBarDone));
            (void)mbar_wait(I.bar(kBarDone), n_done & 1u);
        }
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        else
            cudaGetLastError();
    }
    return fn;
}

// 2-D BF16 map over a row-major [rows x cols] matrix, box [box_rows x 64],
// 128-byte swizzle, zero fill outside the matrix.
bool make_map(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {64, box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace

bool mlp_tc_available() { return true; }

bool make_weight_maps(NetBF16& w) {
    bool ok = true;
    ok &= make_map(&w.tmW1, w.W1, kAevLd, (uint64_t)kNSpecies * kH1, kH1);
    ok &= make_map(&w.tmW2, w.W2, kH1, (uint64_t)kNSpecies * kH2, kH2);
    ok &= make_map(&w.tmW3, w.W3, kH2, (uint64_t)kNSpecies * kH3, kH3);
    ok &= make_map(&w.tmW3t, w.W3t, kH3, (uint64_t)kNSpecies * kH2, kH2);
    ok &= make_map(&w.tmW2t, w.W2t, kH2, (uint64_t)kNSpecies * kH1, kH1);
    ok &= make_map(&w.tmW1t, w.W1t, kH1, (uint64_t)kNSpecies * kAevLd, 256);
    w.maps_ok = ok;
    return ok;
}

bool launch_mlp_bf16(cudaStream_t st, int rows_cap, const Counters* ctr, const NetBF16& w, const __nv_bfloat16* G,
                     const int* row_atom, float* e, float* dG, bool backward, int* err_flag) {
    CUtensorMap mG;
    if (!w.maps_ok || !make_map(&mG, G, kAevLd, (uint64_t)rows_cap, 128)) {
        set_error(-5, "TMA tensor map creation failed");
        return false;
    }
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAlloc);
        attr = true;
    }
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 148;
    }
    const int tiles = rows_cap / kTileRows;
    const int grid = tiles < sms ? tiles : sms;
    TcArgs a{ctr, row_atom, w.b1, w.b2, w.b3, w.W4, w.b4, e, dG, backward ? 1 : 0, err_flag};
    MLP_LAUNCH("mlp_tc", st,
               k_mlp_tc<<<grid, kThreads, kSmemAlloc, st>>>(mG, w.tmW1, w.tmW2, w.tmW3, w.tmW3t, w.tmW2t, w.tmW1t, a));
    return true;
}

}  // namespace mlp
