// Per-element networks on the 5th-generation tensor cores (BF16 x BF16 ->
// FP32): the one dense contraction of the path (paper, section "Performance
// of MLPs": one ANI net per element, evaluated for every atom).
//
// One CTA (16 warps; TMEM lane r = row r of the tile) processes
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
// Split mode (the default BF16 precision): every forward GEMM is computed from
// BF16 hi/lo pairs of both operands, X = X_hi + X_lo with X_lo the BF16
// rounding of the remainder, as A_hi B_hi + A_lo B_hi + A_hi B_lo (three MMAs
// per K step, FP32 accumulation), so the energy carries ~16 bits of operand
// precision; the backward (forces) uses the single BF16 terms.
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

constexpr int kThreads = 512;   // 16 warps: warp w serves TMEM lanes 32 (w % 4) .. +32 and column part w / 4
constexpr int kParts = kThreads / 128;
constexpr uint32_t kAtom = 128 * 128;          // 128 rows x 64 BF16 (one K atom of a 128-row operand)
// Shared memory map (224 KB, offsets from the 1024-aligned base):
//   [0, 64K)      h1 / g1                         (4 atoms)
//   [64K, 112K)   h2 / g2                         (3 atoms)
//   [112K, 160K)  g3                              (3 atoms, 160 of 192 columns used)
//   [160K, 224K)  weight ring of the backward GEMMs (2 x 32 KB)
// Split mode also keeps h1_lo at [64K, 128K) during F2 (ring [128K, 224K),
// 4 x 24 KB) and h2_lo at [112K, 160K) during F3 (ring [160K, 224K), 3 x 20 KB).
// F1 streams G and W1 chunks through stages overlaying [0, 192K): 4 x 48 KB,
// or 2 x 96 KB in split mode (G_hi, G_lo, W1_hi, W1_lo per chunk).
constexpr uint32_t kOffH1 = 0;
constexpr uint32_t kOffH2 = 4 * kAtom;
constexpr uint32_t kOffG3 = 7 * kAtom;
constexpr uint32_t kOffH1lo = 4 * kAtom;
constexpr uint32_t kOffH2lo = 7 * kAtom;
constexpr uint32_t kOffRB = 10 * kAtom;
constexpr uint32_t kOffEPart = 216 * 1024;       // energy partial sums during E3 (2 KB)
constexpr uint32_t kSmemUsed = 14 * kAtom;               // 229,376 bytes
constexpr uint32_t kSmemAlloc = kSmemUsed + 1024;       // + alignment slack
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

enum { kBarF1Full = 0, kBarF1Empty = 4, kBarRBFull = 8, kBarRBEmpty = 12, kBarDone = 16, kNBars = 17 };

struct TcArgs {
    const Counters* ctr;
    const int* row_atom;
    const float *b1, *b2, *b3, *W4, *b4;
    float* e;
    __nv_bfloat16* dG;   // [rows][1024] BF16
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
// Slots 0..3: F1 stages; slots 4..7: weight-ring slots of the other GEMMs.
struct Issuer {
    uint32_t bar0;          // shared address of barrier 0 (barriers are 8 bytes apart)
    uint32_t nfull[8];      // phases consumed per full barrier
    uint32_t nempty[8];     // phases consumed per empty barrier
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

// One GEMM D[128 x N] = A[128 x K] B^T with B streamed by TMA through a ring
// of slots, one sub-chunk (N rows x 64 K columns) per slot. In split mode
// every K chunk c brings two sub-chunks, B_hi(c) then B_lo(c), and the MMAs
// are A_hi(c) B_hi(c) + A_lo(c) B_hi(c) and A_hi(c) B_lo(c).
struct Job {
    const CUtensorMap* map;      // B (hi)
    const CUtensorMap* map_lo;   // B lo (split only)
    int brow;                    // first B row (element block + column block)
    int nc;                      // K chunks of 64
    int lastk;                   // 16-wide K steps in the last chunk
    uint32_t a_off, a_lo_off;    // A operand regions (lo: split only)
    uint32_t d_col;              // TMEM column of the accumulator
    int N;
    uint32_t ring_off, slot_bytes;
    int slots;
    int split;
    int st[8];                   // slot of each sub-chunk
    __device__ int nq() const { return split ? 2 * nc : nc; }
};

__device__ __forceinline__ bool load_sub(Issuer& I, uint32_t sbase, Job& J, int q) {
    const int si = J.st[q];
    if (!I.acquire(si)) return false;
    const uint32_t dst = sbase + J.ring_off + (uint32_t)(si - 4) * J.slot_bytes;
    const int c = J.split ? (q >> 1) : q;
    const CUtensorMap* m = (J.split && (q & 1)) ? J.map_lo : J.map;
    mbar_expect_tx(I.full(si), (uint32_t)J.N * 128u);
    tma_load_2d(dst, m, c * 64, J.brow, I.full(si));
    I.loaded |= 1u << si;
    return true;
}

__device__ bool job_prefetch(Issuer& I, uint32_t sbase, Job& J) {
    const int nq = J.nq();
    for (int q = 0; q < J.slots && q < nq; ++q) {
        J.st[q] = 4 + (int)(I.rb_next % (uint32_t)J.slots);
        I.rb_next++;
        if (!load_sub(I, sbase, J, q)) return false;
    }
    return true;
}

__device__ bool job_run(Issuer& I, uint32_t sbase, uint32_t tmem, Job& J) {
    const uint32_t idesc = idesc_bf16(128, J.N);
    const int nq = J.nq();
    bool first = true;
    for (int q = 0; q < nq; ++q) {
        const int si = J.st[q];
        if (!I.consume(si)) return false;
        const int c = J.split ? (q >> 1) : q;
        const bool lo_b = J.split && (q & 1);
        const uint32_t b_base = sbase + J.ring_off + (uint32_t)(si - 4) * J.slot_bytes;
        const uint32_t a_hi = sbase + J.a_off + (uint32_t)c * kAtom;
        const uint32_t a_lo = sbase + J.a_lo_off + (uint32_t)c * kAtom;
        const int ks = (c == J.nc - 1) ? J.lastk : 4;
        for (int k = 0; k < ks; ++k) {
            const uint64_t b = sdesc(b_base + 32u * k);
            mma_bf16(tmem + J.d_col, sdesc(a_hi + 32u * k), b, idesc, first ? 0u : 1u);
            first = false;
            if (J.split && !lo_b) mma_bf16(tmem + J.d_col, sdesc(a_lo + 32u * k), b, idesc, 1u);
        }
        I.release(si);
        const int nxt = q - 1 + J.slots;
        if (q >= 1 && nxt < nq) {
            J.st[nxt] = J.st[q - 1];
            if (!load_sub(I, sbase, J, nxt)) return false;
        }
    }
    mma_commit(I.bar(kBarDone));
    return true;
}

// Layer 1: A (G) and B (W1) both streamed, K = 1024 in 16 chunks.
template <bool SPLIT>
__device__ bool f1_run(Issuer& I, uint32_t sbase, uint32_t tmem, const CUtensorMap* mG, const CUtensorMap* mGlo,
                       const CUtensorMap* mW1, const CUtensorMap* mW1lo, int row0, int s) {
    constexpr int nc = kAevLd / 64;                       // 16
    constexpr int nst = SPLIT ? 2 : 4;
    constexpr uint32_t stage = SPLIT ? 98304u : 49152u;   // A (+A_lo) 16 KB each, B (+B_lo) 32 KB each
    const uint32_t idesc = idesc_bf16(128, kH1);
    int st[nc];
    auto load = [&](int c) -> bool {
        const int si = st[c];
        if (!I.acquire(si)) return false;
        const uint32_t dst = sbase + (uint32_t)si * stage;
        mbar_expect_tx(I.full(si), stage);
        tma_load_2d(dst, mG, c * 64, row0, I.full(si));
        if (SPLIT) {
            tma_load_2d(dst + 16384u, mGlo, c * 64, row0, I.full(si));
            tma_load_2d(dst + 32768u, mW1, c * 64, s * kH1, I.full(si));
            tma_load_2d(dst + 65536u, mW1lo, c * 64, s * kH1, I.full(si));
        } else {
            tma_load_2d(dst + 16384u, mW1, c * 64, s * kH1, I.full(si));
        }
        I.loaded |= 1u << si;
        return true;
    };
    for (int c = 0; c < nst; ++c) {
        st[c] = (int)(I.f1_next % (uint32_t)nst);
        I.f1_next++;
        if (!load(c)) return false;
    }
    for (int c = 0; c < nc; ++c) {
        const int si = st[c];
        if (!I.consume(si)) return false;
        const uint32_t base = sbase + (uint32_t)si * stage;
        for (int k = 0; k < 4; ++k) {
            const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
            if (SPLIT) {
                const uint64_t ah = sdesc(base + 32u * k), al = sdesc(base + 16384u + 32u * k);
                const uint64_t bh = sdesc(base + 32768u + 32u * k), bl = sdesc(base + 65536u + 32u * k);
                mma_bf16(tmem, ah, bh, idesc, acc);
                mma_bf16(tmem, al, bh, idesc, 1u);
                mma_bf16(tmem, ah, bl, idesc, 1u);
            } else {
                mma_bf16(tmem, sdesc(base + 32u * k), sdesc(base + 16384u + 32u * k), idesc, acc);
            }
        }
        I.release(si);
        if (c >= 1 && c - 1 + nst < nc) {
            st[c - 1 + nst] = st[c - 1];
            if (!load(c - 1 + nst)) return false;
        }
    }
    mma_commit(I.bar(kBarDone));
    return true;
}

// Epilogue helper: 16 values of this thread's row -> BF16 hi (and lo) in the
// operand layout at column c0.
template <bool SPLIT>
__device__ __forceinline__ void store_act(uint32_t sbase, uint32_t off_hi, uint32_t off_lo, int r, int c0,
                                          const float (&h)[16]) {
    uint32_t hi[8], lo[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        __nv_bfloat162 v = __floats2bfloat162_rn(h[2 * q], h[2 * q + 1]);
        hi[q] = *reinterpret_cast<uint32_t*>(&v);
        if (SPLIT) {
            const float2 f = __bfloat1622float2(v);
            lo[q] = pack_bf16(h[2 * q] - f.x, h[2 * q + 1] - f.y);
        }
    }
    st_shared_v4(sbase + off_hi + op_off(r, c0), hi[0], hi[1], hi[2], hi[3]);
    st_shared_v4(sbase + off_hi + op_off(r, c0 + 8), hi[4], hi[5], hi[6], hi[7]);
    if (SPLIT) {
        st_shared_v4(sbase + off_lo + op_off(r, c0), lo[0], lo[1], lo[2], lo[3]);
        st_shared_v4(sbase + off_lo + op_off(r, c0 + 8), lo[4], lo[5], lo[6], lo[7]);
    }
}

#ifdef MLP_TC_TRACE
// Phase timestamps (%globaltimer, ns) of the first tiles of the first CTAs,
// for performance investigation builds only (-DMLP_TC_TRACE).
constexpr int kTraceCtas = 8, kTraceTiles = 4, kTracePoints = 32;
__device__ unsigned long long g_tc_trace[kTraceCtas][kTraceTiles][kTracePoints];
#define MLP_TC_MARK(k)                                                                                  \
    do {                                                                                                \
        if (tid == 0 && blockIdx.x < kTraceCtas && tile_no < kTraceTiles) g_tc_trace[blockIdx.x][tile_no][k] = globaltimer(); \
    } while (0)
#else
#define MLP_TC_MARK(k) \
    do {               \
    } while (0)
#endif

struct TcMaps {
    CUtensorMap G, Glo, W1, W1lo, W2, W2lo, W3, W3lo, W3t, W2t, W1t;
};

template <bool SPLIT>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_tc(const __grid_constant__ TcMaps M, TcArgs p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) unsigned long long bars[kNBars];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int part = warp >> 2;   // which 16-column chunks this warp takes: part, part + kParts, ...
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;

    Issuer I;
    I.bar0 = smem_u32(&bars[0]);
    for (int q = 0; q < 8; ++q) I.nfull[q] = I.nempty[q] = 0;
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
    const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);   // this warp's TMEM lanes
    const int r = (warp & 3) * 32 + lane;                              // tile row = TMEM lane

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

    int tile_no = -1;
    (void)tile_no;
    for (int t = blockIdx.x;; t += gridDim.x) {
        ++tile_no;
        MLP_TC_MARK(0);
        int s, row0, nvalid;
        if (!tile_info(p.ctr->species, t, s, row0, nvalid)) break;
        const float* b1 = p.b1 + s * kH1;
        const float* b2 = p.b2 + s * kH2;
        const float* b3 = p.b3 + s * kH3;
        const float* w4 = p.W4 + s * kH3;
        // forward jobs (ring geometry depends on the mode), backward jobs
        Job jF2 = SPLIT ? Job{&M.W2, &M.W2lo, s * kH2, 4, 4, kOffH1, kOffH1lo, 256, kH2, 8 * kAtom,
                              (uint32_t)kH2 * 128u, 4, 1, {0}}
                        : Job{&M.W2, nullptr, s * kH2, 4, 4, kOffH1, 0, 256, kH2, kOffRB, 32768u, 2, 0, {0}};
        Job jF3 = SPLIT ? Job{&M.W3, &M.W3lo, s * kH3, 3, 4, kOffH2, kOffH2lo, 0, kH3, kOffRB, (uint32_t)kH3 * 128u,
                              3, 1, {0}}
                        : Job{&M.W3, nullptr, s * kH3, 3, 4, kOffH2, 0, 0, kH3, kOffRB, 32768u, 2, 0, {0}};
        Job jB3{&M.W3t, nullptr, s * kH2, 3, 2, kOffG3, 0, 256, kH2, kOffRB, 32768u, 2, 0, {0}};
        Job jB2{&M.W2t, nullptr, s * kH1, 3, 4, kOffH2, 0, 0, kH1, kOffRB, 32768u, 2, 0, {0}};

        // ---- F1 -> E1
        if (tid == 0 && !f1_run<SPLIT>(I, sbase, tmem, &M.G, &M.Glo, &M.W1, &M.W1lo, row0, s)) issue_fail();
        MLP_TC_MARK(1);
        wait_done();
        MLP_TC_MARK(2);
        if (tid == 0 && I.ok && !job_prefetch(I, sbase, jF2)) issue_fail();
        for (int c0 = 16 * part; c0 < kH1; c0 += 16 * kParts) {
            float v[16];
            tmem_ld16(tl + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = celu_f(v[q] + __ldg(b1 + c0 + q));
            store_act<SPLIT>(sbase, kOffH1, kOffH1lo, r, c0, v);
        }
        if (!sync_all()) break;
        MLP_TC_MARK(3);

        // ---- F2 -> E2
        if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jF2)) issue_fail();
        MLP_TC_MARK(4);
        wait_done();
        MLP_TC_MARK(5);
        if (tid == 0 && I.ok && !job_prefetch(I, sbase, jF3)) issue_fail();
        for (int c0 = 16 * part; c0 < kH2; c0 += 16 * kParts) {
            float v[16];
            tmem_ld16(tl + 256u + (uint32_t)c0, v);
#pragma unroll
            for (int q = 0; q < 16; ++q) v[q] = celu_f(v[q] + __ldg(b2 + c0 + q));
            store_act<SPLIT>(sbase, kOffH2, kOffH2lo, r, c0, v);
        }
        if (!sync_all()) break;
        MLP_TC_MARK(6);

        // ---- F3 -> E3 (energy, g3). Each part sums its own column chunks of
        // w4 . celu(z3); the four partial sums of a row meet in [216K, 218K),
        // a corner no load touches during E3 (the B3 prefetch fills
        // [160K, 184K) and [192K, 216K)), and are added in fixed order.
        if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jF3)) issue_fail();
        MLP_TC_MARK(7);
        wait_done();
        MLP_TC_MARK(8);
        if (tid == 0 && I.ok && p.backward && !job_prefetch(I, sbase, jB3)) issue_fail();
        {
            float es = 0.f;
            for (int c0 = 16 * part; c0 < kH3; c0 += 16 * kParts) {
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
            float* e_part = reinterpret_cast<float*>(smem_raw + (sbase - smem_u32(smem_raw)) + kOffEPart);
            e_part[part * 128 + r] = es;
            __syncthreads();
            if (part == 0 && r < nvalid) {
                float t = __ldg(p.b4 + s);
#pragma unroll
                for (int q = 0; q < kParts; ++q) t += e_part[q * 128 + r];
                p.e[p.row_atom[row0 + r]] = t;
            }
        }
        if (!sync_all()) break;
        MLP_TC_MARK(9);
        if (!p.backward) continue;

        // ---- B3 -> g2 (over h2)
        if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jB3)) issue_fail();
        MLP_TC_MARK(10);
        wait_done();
        MLP_TC_MARK(11);
        if (tid == 0 && I.ok && !job_prefetch(I, sbase, jB2)) issue_fail();
        for (int c0 = 16 * part; c0 < kH2; c0 += 16 * kParts) {
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
        MLP_TC_MARK(12);

        // ---- B2 -> g1 (over h1)
        if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jB2)) issue_fail();
        MLP_TC_MARK(13);
        wait_done();
        MLP_TC_MARK(14);
        Job jB1{&M.W1t, nullptr, s * kAevLd, 4, 4, kOffH1, 0, 0, 256, kOffRB, 32768u, 2, 0, {0}};
        if (tid == 0 && I.ok && !job_prefetch(I, sbase, jB1)) issue_fail();
        for (int c0 = 16 * part; c0 < kH1; c0 += 16 * kParts) {
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
        MLP_TC_MARK(15);

        // ---- B1: four 256-column blocks of dE/dG, alternating TMEM halves
        bool aborted = false;
        for (int j = 0; j < 4; ++j) {
            if (tid == 0 && I.ok && !job_run(I, sbase, tmem, jB1)) issue_fail();
            MLP_TC_MARK(16 + 2 * j);
            wait_done();
            MLP_TC_MARK(17 + 2 * j);
            const uint32_t dcol = jB1.d_col;
            if (j < 3) {
                jB1.brow = s * kAevLd + 256 * (j + 1);
                jB1.d_col = 256u * (uint32_t)((j + 1) & 1);
                if (tid == 0 && I.ok && !job_prefetch(I, sbase, jB1)) issue_fail();
            }
            __nv_bfloat16* out = p.dG + (size_t)(row0 + r) * kAevLd + 256 * j;
            for (int c0 = 16 * part; c0 < 256; c0 += 16 * kParts) {
                float v[16];
                tmem_ld16(tl + dcol + (uint32_t)c0, v);
                if (r < nvalid) {
                    uint4 o0, o1;
                    o0.x = pack_bf16(v[0], v[1]);
                    o0.y = pack_bf16(v[2], v[3]);
                    o0.z = pack_bf16(v[4], v[5]);
                    o0.w = pack_bf16(v[6], v[7]);
                    o1.x = pack_bf16(v[8], v[9]);
                    o1.y = pack_bf16(v[10], v[11]);
                    o1.z = pack_bf16(v[12], v[13]);
                    o1.w = pack_bf16(v[14], v[15]);
                    *reinterpret_cast<uint4*>(out + c0) = o0;
                    *reinterpret_cast<uint4*>(out + c0 + 8) = o1;
                }
            }
            if (!sync_all()) {
                aborted = true;
                break;
            }
        }
        if (aborted) break;
        MLP_TC_MARK(24);
    }

    // ---- teardown: drain own copies and MMAs (bounded), free tensor memory
    __syncthreads();
    if (abort_flag) {
        if (tid == 0) {
            atomicOr(p.err, 1);
            for (int si = 0; si < 8; ++si)
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

#ifdef MLP_TC_TRACE
extern "C" __attribute__((visibility("default"))) int mlp_tc_trace_read(unsigned long long* out, int cap) {
    const int n = kTraceCtas * kTraceTiles * kTracePoints;
    if (cap < n) return -n;
    cudaMemcpyFromSymbol(out, g_tc_trace, sizeof(unsigned long long) * n);
    return n;
}
#endif

bool make_weight_maps(NetBF16& w) {
    bool ok = true;
    ok &= make_map(&w.tmW1, w.W1, kAevLd, (uint64_t)kNSpecies * kH1, kH1);
    ok &= make_map(&w.tmW2, w.W2, kH1, (uint64_t)kNSpecies * kH2, kH2);
    ok &= make_map(&w.tmW3, w.W3, kH2, (uint64_t)kNSpecies * kH3, kH3);
    ok &= make_map(&w.tmW1lo, w.W1lo, kAevLd, (uint64_t)kNSpecies * kH1, kH1);
    ok &= make_map(&w.tmW2lo, w.W2lo, kH1, (uint64_t)kNSpecies * kH2, kH2);
    ok &= make_map(&w.tmW3lo, w.W3lo, kH2, (uint64_t)kNSpecies * kH3, kH3);
    ok &= make_map(&w.tmW3t, w.W3t, kH3, (uint64_t)kNSpecies * kH2, kH2);
    ok &= make_map(&w.tmW2t, w.W2t, kH2, (uint64_t)kNSpecies * kH1, kH1);
    ok &= make_map(&w.tmW1t, w.W1t, kH1, (uint64_t)kNSpecies * kAevLd, 256);
    w.maps_ok = ok;
    return ok;
}

bool launch_mlp_bf16(cudaStream_t st, int rows_cap, const Counters* ctr, const NetBF16& w, const __nv_bfloat16* G,
                     const __nv_bfloat16* G_lo, bool split, const int* row_atom, float* e, __nv_bfloat16* dG,
                     bool backward, int* err_flag) {
    TcMaps M;
    if (!w.maps_ok || !make_map(&M.G, G, kAevLd, (uint64_t)rows_cap, 128) ||
        (split && (!G_lo || !make_map(&M.Glo, G_lo, kAevLd, (uint64_t)rows_cap, 128)))) {
        set_error(-5, "TMA tensor map creation failed");
        return false;
    }
    if (!split) M.Glo = M.G;
    M.W1 = w.tmW1;
    M.W1lo = w.tmW1lo;
    M.W2 = w.tmW2;
    M.W2lo = w.tmW2lo;
    M.W3 = w.tmW3;
    M.W3lo = w.tmW3lo;
    M.W3t = w.tmW3t;
    M.W2t = w.tmW2t;
    M.W1t = w.tmW1t;
    static bool attr = false;
    if (!attr) {
        cudaFuncSetAttribute(k_mlp_tc<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAlloc);
        cudaFuncSetAttribute(k_mlp_tc<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAlloc);
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
    if (split)
        MLP_LAUNCH("mlp_tc", st, k_mlp_tc<true><<<grid, kThreads, kSmemAlloc, st>>>(M, a));
    else
        MLP_LAUNCH("mlp_tc", st, k_mlp_tc<false><<<grid, kThreads, kSmemAlloc, st>>>(M, a));
    return true;
}

}  // namespace mlp
