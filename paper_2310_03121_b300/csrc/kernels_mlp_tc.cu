// Per-element networks on the 5th-generation tensor cores (BF16 x BF16 ->
// FP32): the one dense contraction of the path (paper, section "Performance
// of MLPs": one ANI net per element, evaluated for every atom).
//
// One persistent CTA per SM processes 128-row tiles of one element (TMEM lane
// r = row r of the tile). The six GEMMs of the forward and backward run back
// to back without leaving the SM:
//   F1  D[128x256] = G[128x1024] W1^T   G and W1 streamed by TMA in 32- or 64-wide K chunks
//   E1  h1 = celu(D + b1)               -> shared memory, BF16, A-operand layout
//   F2  D[128x192] = h1 W2^T            W2 streamed
//   E2  h2 = celu(D + b2)               -> shared memory
//   F3  D[128x160] = h2 W3^T            W3 streamed
//   E3  e = w4 . celu(D + b3) + b4      -> global; g3 = w4 * celu'(z3) -> shared memory
//   B3  D[128x192] = g3 W3              W3^T streamed;  g2 = D * celu'(z2) (over h2)
//   B2  D[128x256] = g2 W2              W2^T streamed;  g1 = D * celu'(z1) (over h1)
//   B1  dE/dG[128x1024] = g1 W1         W1^T streamed, four 256-column blocks -> global BF16 by TMA store
// celu'(z) comes from the stored BF16 activation: 1 if h > 0 else h / alpha + 1.
// Split mode (the default BF16 precision): every forward GEMM is computed from
// BF16 hi/lo pairs of both operands, X = X_hi + X_lo with X_lo the BF16
// rounding of the remainder, as A_hi B_hi + A_lo B_hi + A_hi B_lo (three MMAs
// per K step, FP32 accumulation), so the energy carries ~16 bits of operand
// precision; the backward (forces) uses the single BF16 terms.
// Ensemble (section "Performance of MLPs": ANI-2x averages eight nets): each
// tile runs F1..B2 once per net k (weights block k * 7 + s of the net-major
// matrices), G coming back from L2 for every net. The energy of a row is
// summed over the nets in registers and written once, times 1 / K. Instead of
// B1, every net's g1 (BF16, the B1 A operand) is written out by TMA, and a
// second kernel (k_mlp_b1_ens) forms the mean dE/dG as one GEMM with the nets
// stacked along the contraction, dE/dG = (1/K) [g1_0 .. g1_K-1] [W1_0; ..;
// W1_K-1], accumulated in tensor memory: one dE/dG epilogue per tile instead
// of K, and no partial sums through L2.
//
// Warp roles (14 warps, at most 4 per SM sub-partition so that the epilogue
// warps get up to 128 registers):
//   warp 0       TMA producer (one lane): streams G and weight sub-chunks into
//                shared-memory rings as soon as slots free up, running ahead
//                across GEMMs (no L2 prefetch of the next tile's G: its
//                requests held up the current tile's loads and stores);
//   warp 1       MMA issuer (one lane): tcgen05.mma into tensor memory (512
//                columns: two 256-column accumulator halves), tcgen05.commit
//                to the ring-slot and accumulator barriers;
//   warps 2..13  epilogues (tcgen05.ld -> registers -> shared operand or
//                global); warp w reads TMEM lanes 32 (w % 4) .. +32 and takes
//                column part (w - 2) / 4 of 3: the 16-column chunks
//                part, part + 3, part + 6, ...
// Every hand-off is an mbarrier: ring slot full / empty (producer <-> MMA),
// accumulator half full (MMA -> epilogue), operand atom ready (each GEMM
// after F1 starts on the 64-column atoms of its A operand as the previous
// epilogue writes them), accumulator half read and B1 half read (epilogue ->
// MMA), tile done with shared memory (epilogue -> producer). Every
// wait is bounded in time and also gives up when another role has aborted; on
// abort the CTA records an error, drains its own copies, MMAs and stores,
// frees its tensor memory and returns. Operands in shared memory use the
// 128-byte swizzled K-major layout that TMA writes.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstring>

#include "common.cuh"
#include "engine.cuh"
#include "kernels.cuh"

namespace mlp {
namespace {

constexpr int kEpiWarps = 12;
constexpr int kParts = kEpiWarps / 4;            // column parts per TMEM lane quarter
constexpr int kThreads = 32 * (2 + kEpiWarps);   // 448
constexpr uint32_t kAtom = 128 * 128;            // 128 rows x 64 BF16 (one K atom of a 128-row operand)
// Shared memory map (224 KB, offsets from the 1024-aligned base):
//   [0, 64K)      h1 / g1                          (4 atoms)
//   [64K, 112K)   h2 / g2                          (3 atoms)
//   [112K, 160K)  g3 (3 atoms, 160 of 192 columns; column chunk 160..167 of
//                 each row holds the three E3 energy partial sums of the row)
//   split only:   h1_lo [64K, 128K) from E1 to F2, h2_lo [112K, 160K) from E2 to F3
//   B1 only:      dE/dG staging [64K, 112K), one 32-row x 64-column box (4 KB) per epilogue warp
//   weight rings: F2 [128K, 224K) 4 x 24 KB, F3 [160K, 220K) 3 x 20 KB,
//                 B3 [160K, 208K) 2 x 24 KB, B2 and B1 [112K, 208K) 3 x 32 KB
//                 (g3 is free once B3's MMAs are done); the F2 and F3 rings
//                 hold one more weight sub-chunk than at 208 KB: 1.5% faster
//   F1 stages over [0, 192K): 4 x 48 KB; split: 32 K columns per stage (G_hi, G_lo
//   8 KB each, W1_hi, W1_lo 16 KB each; 64-byte swizzle), so that three stages
//   are in flight while one is consumed; one pass: 64 K columns (G 16 KB, W1 32 KB)
// The producer switches between region layouts only after the MMAs reading
// the previous layout have completed, and starts a tile's F1 only after the
// previous tile's epilogues are done with shared memory.
constexpr uint32_t kOffH1 = 0;
constexpr uint32_t kOffH2 = 4 * kAtom;
constexpr uint32_t kOffG3 = 7 * kAtom;
constexpr uint32_t kOffH1lo = 4 * kAtom;
constexpr uint32_t kOffH2lo = 7 * kAtom;
constexpr uint32_t kOffStage = 4 * kAtom;
constexpr uint32_t kOffEPart = kOffG3 + 2 * kAtom;   // + row * 128 + (4 ^ (row & 7)) * 16
constexpr uint32_t kSmemUsed = 14 * kAtom;           // 229,376 bytes
constexpr uint32_t kSmemAlloc = kSmemUsed + 1024;    // + alignment slack
constexpr unsigned long long kWaitNs = 2000000000ull;   // 2 s per wait

enum {
    kBarF1Full = 0,     // 4: F1 stage loaded (expect_tx + TMA bytes)
    kBarF1Empty = 4,    // 4: F1 stage consumed (MMA commit)
    kBarRFull = 8,      // 4: weight ring slot loaded
    kBarREmpty = 12,    // 4: weight ring slot consumed
    kBarAcc = 16,       // 2: accumulator half complete (MMA commit)
    kBarOp = 18,        // 1: an epilogue finished (operand written, accumulator read); one arrival per epilogue warp
    kBarB1Free = 19,    // 2: a B1 accumulator half read; one arrival per epilogue warp
    kBarStage = 21,     // 1: a tile's epilogues are done with shared memory; one arrival per epilogue warp
    kBarEPart = 22,     // 1: E3 partial sums written; one arrival per epilogue warp
    kBarDrain = 23,     // 1: teardown MMA drain
    kBarG1 = 24,        // 1: ensemble, g1 written to shared memory; one arrival per epilogue warp
    kBarOpA = 25,       // 4: 64-column atom a of the next GEMM's A operand written; one arrival per epilogue warp
    kNBars = 29
};

struct TcArgs {
    const Counters* ctr;
    const int* row_atom;
    const float *b1, *b2, *b3, *W4, *b4;   // net-major: block k * 7 + s
    float* e;         // per-atom energies; an ensemble: [K][e_stride], one row per net
    int e_stride;
    int backward;
    int nets;         // ensemble size K (1: single net)
    float inv_nets;   // 1 / K
    int* err;
};

struct TcMaps {
    CUtensorMap G, Glo, W1, W1lo, W2, W2lo, W3, W3lo, W3t, W2t, W1t, dG;
    CUtensorMap G1;   // ensemble: g1 of every net, BF16 [rows][K * 256]
    // split F1: 32-column boxes, 64-byte swizzle (4 stages of 48 KB)
    CUtensorMap Gn, Glon, W1n, W1lon;
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
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
// try_wait with a suspend-time hint: a waiting thread is parked by the
// hardware until the phase completes (or the hint expires) instead of
// spinning, so waiting roles take no issue slots from the working ones.
constexpr uint32_t kSuspendNs = 1000000u;
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Bounded wait on a phase: false after kWaitNs (and the abort flag is set), or
// as soon as another role has set the abort flag. The completed-phase case is
// a single inline test; only a real wait takes the out-of-line loop.
__device__ __noinline__ bool mbar_wait_slow(uint32_t bar, uint32_t parity, volatile int* abrt) {
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        {
            if (*abrt) return false;
            if (globaltimer() - t0 > kWaitNs) {   // record the waiting warp and barrier
                *abrt = (int)(0x40000000u | ((threadIdx.x >> 5) << 20) | bar);
                return false;
            }
        }
    }
}
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abrt) {
    return mbar_test(bar, parity) || mbar_wait_slow(bar, parity, abrt);
}
// Bounded wait used by the teardown drains (no abort check).
__device__ __noinline__ bool mbar_wait_plain(uint32_t bar, uint32_t parity) {
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitNs) return false;
    }
}
// TMA tile load with an L2 eviction-priority policy (createpolicy): the
// weights stay in L2 while G and dE/dG stream through it.
__device__ __forceinline__ void tma_load_2d_hint(uint32_t dst, const CUtensorMap* map, int x, int y, uint32_t bar,
                                                 uint64_t policy) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%2, "
        "%3}], [%4], %5;" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(bar), "l"(policy)
        : "memory");
}
__device__ __forceinline__ uint64_t policy_evict_last() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_normal() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ uint64_t policy_evict_first() {
    uint64_t p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}
__device__ __forceinline__ void tma_store_2d(const CUtensorMap* map, int x, int y, uint32_t src, uint64_t policy) {
    asm volatile("cp.async.bulk.tensor.2d.global.shared::cta.bulk_group.L2::cache_hint [%0, {%1, %2}], [%3], %4;" ::"l"(
                     reinterpret_cast<uint64_t>(map)),
                 "r"(x), "r"(y), "r"(src), "l"(policy)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
}
__device__ __forceinline__ void bulk_wait_read0() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
__device__ __forceinline__ void bulk_wait0() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void prefetch_map(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
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
// The same for 64-byte swizzled rows (32 BF16 columns): 8-row groups 512
// bytes apart, layout type SWIZZLE_64B.
__device__ __forceinline__ uint64_t sdesc64(uint32_t addr) {
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;             // SWIZZLE_64B
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
// 16 consecutive FP32 columns of this thread's TMEM lane (no wait).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
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
__device__ __forceinline__ float dcelu_h(float h) { return h > 0.f ? 1.f : h * (1.f / kCeluAlpha) + 1.f; }

#ifdef MLP_TC_TRACE
// Phase timestamps (%globaltimer, ns) of the first tiles of the first CTAs,
// for performance investigation builds only (-DMLP_TC_TRACE). Points 0..19:
// epilogue warp 2; 20..26: MMA issuer; 27..31: producer.
constexpr int kTraceCtas = 8, kTraceTiles = 4, kTracePoints = 32;
__device__ unsigned long long g_tc_trace[kTraceCtas][kTraceTiles][kTracePoints];
#define MLP_TC_MARK(k)                                                                   \
    do {                                                                                 \
        if (blockIdx.x < kTraceCtas && tile_no < kTraceTiles && (threadIdx.x & 31) == 0) \
            g_tc_trace[blockIdx.x][tile_no][k] = globaltimer();                          \
    } while (0)
#else
#define MLP_TC_MARK(k) \
    do {               \
    } while (0)
#endif

// ------------------------------------------------------------------ GEMM jobs
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
    __device__ int nq() const { return split ? 2 * nc : nc; }
    __device__ uint32_t geom() const { return (ring_off >> 10) | ((slot_bytes >> 10) << 8) | ((uint32_t)slots << 16); }
};

enum { kJobF2 = 0, kJobF3 = 1, kJobB3 = 2, kJobB2 = 3, kJobB1 = 4 };   // B1 block j: kJobB1 + j

template <bool SPLIT>
__device__ __forceinline__ Job make_job(const TcMaps& M, int k, int s) {
    switch (k) {
        case kJobF2:
            return Job{&M.W2, &M.W2lo, s * kH2, 4, 4, kOffH1, kOffH1lo, 256, kH2, 8 * kAtom, (uint32_t)kH2 * 128u,
                       4, SPLIT ? 1 : 0};
        case kJobF3:
            return Job{&M.W3, &M.W3lo, s * kH3, 3, 4, kOffH2, kOffH2lo, 0, kH3, 10 * kAtom, (uint32_t)kH3 * 128u,
                       3, SPLIT ? 1 : 0};
        case kJobB3:
            return Job{&M.W3t, nullptr, s * kH2, 3, 2, kOffG3, 0, 256, kH2, 10 * kAtom, 24576u, 2, 0};
        case kJobB2:
            return Job{&M.W2t, nullptr, s * kH1, 3, 4, kOffH2, 0, 0, kH1, 7 * kAtom, 32768u, 3, 0};
        default: {
            const int j = k - kJobB1;
            return Job{&M.W1t, nullptr, s * kAevLd + 256 * j, 4, 4, kOffH1, 0, 256u * (uint32_t)(j & 1), 256,
                       7 * kAtom, 32768u, 3, 0};
        }
    }
}

// ------------------------------------------------------------------ producer
// Slot state lives in registers as bit masks over 8 slots: bits 0..3 the F1
// stages, bits 4..7 the weight ring slots. Barrier of slot b: full
// b < 4 ? b : b + 4, consumed b < 4 ? b + 4 : b + 8.
__device__ __forceinline__ uint32_t full_bar(uint32_t bar0, int b) { return bar0 + 8u * (uint32_t)(b < 4 ? b : b + 4); }
__device__ __forceinline__ uint32_t empty_bar(uint32_t bar0, int b) { return bar0 + 8u * (uint32_t)(b < 4 ? b + 4 : b + 8); }

struct ProdState {
    uint32_t pend;   // slots whose last load has not been seen consumed
    uint32_t epar;   // parity of the next consumed phase to wait for, per slot
    uint32_t lpar;   // parity of the number of loads issued, per slot
    uint32_t f1pos, rpos, geom;
};

// Wait until slot b may be overwritten (its last load consumed by the MMAs).
__device__ __forceinline__ bool prod_free(ProdState& P, uint32_t bar0, int b, volatile int* abrt) {
    const uint32_t m = 1u << b;
    if (P.pend & m) {
        if (!mbar_wait(empty_bar(bar0, b), (P.epar >> b) & 1u, abrt)) return false;
        P.epar ^= m;
        P.pend &= ~m;
    }
    return true;
}
__device__ __forceinline__ bool prod_drain(ProdState& P, uint32_t bar0, uint32_t mask, volatile int* abrt) {
    for (int b = 0; b < 8; ++b)
        if ((mask >> b) & 1u)
            if (!prod_free(P, bar0, b, abrt)) return false;
    return true;
}

__device__ __forceinline__ bool prod_job(ProdState& P, const Job& J, uint32_t sbase, uint32_t bar0, volatile int* abrt,
                                         uint64_t keep) {
    if (J.geom() != P.geom) {   // new slot layout: every slot of the old one must be consumed
        if (!prod_drain(P, bar0, 0xf0u, abrt)) return false;
        P.geom = J.geom();
        P.rpos = 0;
    }
    const int nq = J.nq();
    for (int q = 0; q < nq; ++q) {
        const int si = (int)P.rpos;
        P.rpos = (P.rpos + 1u == (uint32_t)J.slots) ? 0u : P.rpos + 1u;
        if (!prod_free(P, bar0, 4 + si, abrt)) return false;
        const int c = J.split ? (q >> 1) : q;
        const CUtensorMap* m = (J.split && (q & 1)) ? J.map_lo : J.map;
        const uint32_t full = full_bar(bar0, 4 + si);
        mbar_expect_tx(full, (uint32_t)J.N * 128u);
        tma_load_2d_hint(sbase + J.ring_off + (uint32_t)si * J.slot_bytes, m, c * 64, J.brow, full, keep);
        P.pend |= 1u << (4 + si);
        P.lpar ^= 1u << (4 + si);
    }
    return true;
}

template <bool SPLIT>
__device__ void producer(const TcMaps& M, const int* counts, uint32_t sbase, uint32_t bar0, volatile int* abrt,
                         bool backward, bool b1, int nets, ProdState& P) {
    // split: 4 stages of 32 K columns (G_hi, G_lo 8 KB each, W1_hi, W1_lo 16 KB each);
    // one pass: 4 stages of 64 K columns (G 16 KB, W1 32 KB)
    constexpr int nst = 4;
    constexpr uint32_t stage = 49152u;
    constexpr int kw = SPLIT ? 32 : 64;   // K columns per stage
    const CUtensorMap* maps[16] = {&M.G,  &M.Glo, &M.W1,  &M.W1lo, &M.W2, &M.W2lo, &M.W3,  &M.W3lo,
                                   &M.W3t, &M.W2t, &M.W1t, &M.dG,  &M.Gn, &M.Glon, &M.W1n, &M.W1lon};
    for (int q = 0; q < 16; ++q) prefetch_map(maps[q]);
    const uint64_t keep = policy_evict_last(), evict = policy_evict_first();
    auto job = [&](int k, int s) -> bool { return prod_job(P, make_job<SPLIT>(M, k, s), sbase, bar0, abrt, keep); };
    const uint64_t gpol = nets > 1 ? policy_evict_normal() : evict;   // see the G loads below
    // units u = blockIdx.x + i * gridDim.x: (tile u / nets, net u % nets)
    for (int u = blockIdx.x, tile_no = 0;; u += gridDim.x, ++tile_no) {
        const int t = u / nets, net = u - t * nets;
        int s, row0, nvalid;
        if (!tile_info(counts, t, s, row0, nvalid)) break;
        {
            const int es = net * kNSpecies + s;   // weight block of (net, element)
            // F1 stages cover every region: the previous unit's epilogues and MMAs must be done with them
            if (tile_no > 0 && !mbar_wait(bar0 + 8u * kBarStage, (uint32_t)(tile_no - 1) & 1u, abrt)) break;
            if (!prod_drain(P, bar0, 0xf0u, abrt)) break;
            bool f1 = true;
            for (int c = 0; c < kAevLd / kw; ++c) {
                const int st = (int)P.f1pos;
                P.f1pos = (P.f1pos + 1u) & (uint32_t)(nst - 1);
                if (!prod_free(P, bar0, st, abrt)) {
                    f1 = false;
                    break;
                }
                const uint32_t full = bar0 + 8u * (kBarF1Full + st), dst = sbase + (uint32_t)st * stage;
                // one net: G streams through L2 (evict-first, the weights stay); an
                // ensemble: the nets of a tile run on neighbouring CTAs at the same
                // time and share each G chunk through L2 (normal priority)
                mbar_expect_tx(full, stage);
                if (SPLIT) {
                    tma_load_2d_hint(dst, &M.Gn, c * kw, row0, full, gpol);
                    tma_load_2d_hint(dst + 8192u, &M.Glon, c * kw, row0, full, gpol);
                    tma_load_2d_hint(dst + 16384u, &M.W1n, c * kw, es * kH1, full, keep);
                    tma_load_2d_hint(dst + 32768u, &M.W1lon, c * kw, es * kH1, full, keep);
                } else {
                    tma_load_2d_hint(dst, &M.G, c * kw, row0, full, gpol);
                    tma_load_2d_hint(dst + 16384u, &M.W1, c * kw, es * kH1, full, keep);
                }
                P.pend |= 1u << st;
                P.lpar ^= 1u << st;
                if (c == 0) MLP_TC_MARK(27);
            }
            if (!f1) break;
            MLP_TC_MARK(28);
            // the F2 ring overlays the F1 stages
            if (!prod_drain(P, bar0, 0x0fu, abrt)) break;
            if (!job(kJobF2, es)) break;
            MLP_TC_MARK(29);
            if (!job(kJobF3, es)) break;
            if (backward && (!job(kJobB3, es) || !job(kJobB2, es))) break;
            if (b1 && (!job(kJobB1 + 0, es) || !job(kJobB1 + 1, es) || !job(kJobB1 + 2, es) || !job(kJobB1 + 3, es)))
                break;
            // No L2 prefetch of the next unit's G: prefetch requests occupy the
            // SM's TMA unit like loads, and 64 of them (1 MB) queued ahead of
            // this unit's last dE/dG stores and the next unit's F1 loads
            // (measured: 10% slower with the prefetch)
            MLP_TC_MARK(30);
        }
    }
}

// ------------------------------------------------------------------ MMA issuer
struct MmaState {
    uint32_t fpar;   // parity of the number of loads consumed, per slot (bits as in ProdState)
    uint32_t f1pos, rpos, geom;
};

// Operand atoms: the epilogue writes the next GEMM's A operand atom by atom
// (64 columns) and arrives on barrier kBarOpA + a for each; the GEMM's MMAs
// for K chunk a start as soon as atom a is in (the rest of the epilogue
// overlaps them). n: phases waited for, per atom barrier.
struct AtomWait {
    uint32_t n[4];
};
__device__ __forceinline__ bool wait_atom(AtomWait& W, uint32_t bar0, int a, volatile int* abrt) {
    if (!mbar_wait(bar0 + 8u * (kBarOpA + a), W.n[a] & 1u, abrt)) return false;
    ++W.n[a];
    tc_fence_after();
    return true;
}

__device__ __forceinline__ bool mma_job(MmaState& S, const Job& J, uint32_t sbase, uint32_t tmem, uint32_t bar0,
                                        volatile int* abrt, AtomWait* aw = nullptr) {
    const uint32_t geom = J.geom();
    if (S.geom != geom) {
        S.geom = geom;
        S.rpos = 0;
    }
    const uint32_t idesc = idesc_bf16(128, J.N);
    const uint32_t d = tmem + J.d_col;
    const int nq = J.nq();
    for (int q = 0; q < nq; ++q) {
        const int si = (int)S.rpos;
        S.rpos = (S.rpos + 1u == (uint32_t)J.slots) ? 0u : S.rpos + 1u;
        const int c = J.split ? (q >> 1) : q;
        if (aw && (!J.split || (q & 1) == 0) && !wait_atom(*aw, bar0, c, abrt)) return false;   // A atom c written
        if (!mbar_wait(full_bar(bar0, 4 + si), (S.fpar >> (4 + si)) & 1u, abrt)) return false;
        S.fpar ^= 1u << (4 + si);
        tc_fence_after();
        const bool lo_b = J.split && (q & 1);
        const int ks = (c == J.nc - 1) ? J.lastk : 4;
        // one 16-wide K step advances a K-major SW128 descriptor by 32 bytes (2 in the address field)
        const uint64_t bd = sdesc(sbase + J.ring_off + (uint32_t)si * J.slot_bytes);
        const uint64_t ad = sdesc(sbase + J.a_off + (uint32_t)c * kAtom);
        const uint64_t ald = sdesc(sbase + J.a_lo_off + (uint32_t)c * kAtom);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            if (k < ks) {
                if (lo_b) {
                    mma_bf16(d, ad + 2u * k, bd + 2u * k, idesc, 1u);
                } else {
                    mma_bf16(d, ad + 2u * k, bd + 2u * k, idesc, (q == 0 && k == 0) ? 0u : 1u);
                    if (J.split) mma_bf16(d, ald + 2u * k, bd + 2u * k, idesc, 1u);
                }
            }
        }
        mma_commit(empty_bar(bar0, 4 + si));
    }
    return true;
}

template <bool SPLIT>
__device__ void mma_issuer(const TcMaps& M, const int* counts, uint32_t sbase, uint32_t tmem, uint32_t bar0,
                           volatile int* abrt, bool backward, bool b1, int nets, MmaState& S) {
    constexpr int nst = 4;
    constexpr uint32_t stage = 49152u;
    constexpr int kw = SPLIT ? 32 : 64;
    const uint32_t idesc1 = idesc_bf16(128, kH1);
    uint32_t n_op = 0, n_b1[2] = {0, 0};
    auto wait_op = [&]() -> bool {
        if (!mbar_wait(bar0 + 8u * kBarOp, n_op & 1u, abrt)) return false;
        ++n_op;
        tc_fence_after();
        return true;
    };
    auto wait_b1 = [&](int h) -> bool {
        if (!mbar_wait(bar0 + 8u * (kBarB1Free + h), n_b1[h] & 1u, abrt)) return false;
        ++n_b1[h];
        tc_fence_after();
        return true;
    };
    AtomWait aw{{0u, 0u, 0u, 0u}};
    // a GEMM whose A operand an epilogue is still writing waits per K chunk (atoms)
    auto job = [&](int k, int s, int half, bool atoms) -> bool {
        Job J = make_job<SPLIT>(M, k, s);
        J.d_col = 256u * (uint32_t)half;
        if (!mma_job(S, J, sbase, tmem, bar0, abrt, atoms ? &aw : nullptr)) return false;
        mma_commit(bar0 + 8u * (kBarAcc + half));
        return true;
    };
    for (int u = blockIdx.x, tile_no = 0;; u += gridDim.x, ++tile_no) {
        const int t = u / nets, net = u - t * nets;
        int s, row0, nvalid;
        if (!tile_info(counts, t, s, row0, nvalid)) break;
        {
            const int es = net * kNSpecies + s;
            // F1 writes accumulator half 0: the previous unit's last reader of it
            // (EB1 block 2, else E3 or EB2, which arrive on the operand barrier) must be done
            if (tile_no > 0 && !(b1 ? wait_b1(0) : wait_op())) break;
            MLP_TC_MARK(20);
            bool f1 = true;
            for (int c = 0; c < kAevLd / kw; ++c) {
                const int st = (int)S.f1pos;
                S.f1pos = (S.f1pos + 1u) & (uint32_t)(nst - 1);
                if (!mbar_wait(full_bar(bar0, st), (S.fpar >> st) & 1u, abrt)) {
                    f1 = false;
                    break;
                }
                S.fpar ^= 1u << st;
                tc_fence_after();
                const uint32_t base = sbase + (uint32_t)st * stage;
                if (SPLIT) {
                    const uint64_t ah = sdesc64(base), al = sdesc64(base + 8192u);
                    const uint64_t bh = sdesc64(base + 16384u), bl = sdesc64(base + 32768u);
#pragma unroll
                    for (int k = 0; k < 2; ++k) {
                        const uint32_t acc = (c > 0 || k > 0) ? 1u : 0u;
                        mma_bf16(tmem, ah + 2u * k, bh + 2u * k, idesc1, acc);
                        mma_bf16(tmem, al + 2u * k, bh + 2u * k, idesc1, 1u);
                        mma_bf16(tmem, ah + 2u * k, bl + 2u * k, idesc1, 1u);
                    }
                } else {
                    const uint64_t ah = sdesc(base), bh = sdesc(base + 16384u);
#pragma unroll
                    for (int k = 0; k < 4; ++k) mma_bf16(tmem, ah + 2u * k, bh + 2u * k, idesc1, (c > 0 || k > 0) ? 1u : 0u);
                }
                mma_commit(empty_bar(bar0, st));
            }
            if (!f1) break;
            mma_commit(bar0 + 8u * kBarAcc);
            MLP_TC_MARK(21);
            // F2 writes half 1: the previous unit's last B1 block must have been read
            if (b1 && tile_no > 0 && !wait_b1(1)) break;
            // Each GEMM of the chain starts on the atoms of its A operand as
            // the previous epilogue writes them (F2 on E1's h1, F3 on E2's h2,
            // B3 on E3's g3, B2 on EB3's g2, B1's first block on EB2's g1); its
            // accumulator half was last read by an epilogue that finished
            // before the previous GEMM completed.
            if (!job(kJobF2, es, 1, true)) break;
            MLP_TC_MARK(22);
            if (!job(kJobF3, es, 0, true)) break;
            MLP_TC_MARK(23);
            if (backward) {
                if (!job(kJobB3, es, 1, true)) break;
                MLP_TC_MARK(24);
                if (!job(kJobB2, es, 0, true)) break;
                MLP_TC_MARK(25);
            }
            if (b1) {
                // block 0 in half 1 (last read by EB3), block 1 in half 0 once
                // EB2 has read all of it, then each half after EB1's previous
                // block in it
                if (!job(kJobB1 + 0, es, 1, true)) break;
                if (!wait_op() || !job(kJobB1 + 1, es, 0, false)) break;   // after EB2
                if (!wait_b1(1) || !job(kJobB1 + 2, es, 1, false)) break;
                if (!wait_b1(0) || !job(kJobB1 + 3, es, 0, false)) break;
                MLP_TC_MARK(26);
            }
        }
    }
}

// ------------------------------------------------------------------ epilogues
// 16 values of this thread's row -> BF16 hi (and lo) in the operand layout at column c0.
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

// g = D * celu'(h) over the stored activation h (in place), 16 columns at c0.
__device__ __forceinline__ void store_grad(uint32_t sbase, uint32_t off, int r, int c0, const uint32_t (&d)[16]) {
#pragma unroll
    for (int hlf = 0; hlf < 2; ++hlf) {
        const uint32_t a = sbase + off + op_off(r, c0 + 8 * hlf);
        const uint4 h = ld_shared_v4(a);
        const uint32_t hw[4] = {h.x, h.y, h.z, h.w};
        uint32_t o[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const float d0 = __uint_as_float(d[8 * hlf + 2 * q]), d1 = __uint_as_float(d[8 * hlf + 2 * q + 1]);
            o[q] = pack_bf16(d0 * dcelu_h(bf_lo(hw[q])), d1 * dcelu_h(bf_hi(hw[q])));
        }
        st_shared_v4(a, o[0], o[1], o[2], o[3]);
    }
}

struct EpiCtx {
    uint32_t sbase, bar0, tl;   // tl: TMEM address of this warp's lane quarter
    volatile int* abrt;
    int lane, part, r;
    uint32_t n_acc[2];
};

// Lane 0 waits, the warp follows (one decision per warp).
__device__ __forceinline__ bool epi_wait(EpiCtx& X, uint32_t bar, uint32_t parity) {
    int ok = 1;
    if (X.lane == 0) ok = mbar_wait(bar, parity, X.abrt) ? 1 : 0;
    ok = __shfl_sync(0xffffffffu, ok, 0);
    tc_fence_after();
    return ok != 0;
}
__device__ __forceinline__ bool epi_acc(EpiCtx& X, int half) {
    const bool ok = epi_wait(X, X.bar0 + 8u * (kBarAcc + half), X.n_acc[half] & 1u);
    X.n_acc[half]++;
    return ok;
}
// This warp's shared-memory writes and TMEM reads are done: one arrival.
__device__ __forceinline__ void epi_arrive(EpiCtx& X, uint32_t bar) {
    fence_proxy_async();
    tc_fence_before();
    __syncwarp();
    if (X.lane == 0) mbar_arrive(bar);
}

// Epilogue loops take one 16-column chunk per iteration, chunks c0 = 16
// (part + kParts k) < N, and are kept rolled: the code of every phase stays
// small, so the epilogue warps keep hitting in the instruction cache.
template <bool SPLIT, bool ENS>
__device__ void epilogue(const TcMaps& M, const TcArgs& p, const int* counts, EpiCtx& X, int warp) {
    const uint32_t sbase = X.sbase, bar0 = X.bar0;
    const uint32_t op_bar = bar0 + 8u * kBarOp;
    const int r = X.r, part = X.part;
    const uint32_t stage_box = sbase + kOffStage + (uint32_t)(warp - 2) * 4096u;
    const uint64_t stream_out = policy_evict_first();
    const int nets = ENS ? p.nets : 1;
    uint32_t n_epart = 0;
    (void)warp;
    const bool b1_here = p.backward && !ENS;   // B1 runs in this kernel (one net)
    // This warp's part of operand atoms [a0, a1) of the next GEMM is written:
    // one arrival on each atom's barrier (the shared stores made visible to
    // the tensor core first).
    auto arrive_atoms = [&](int a0, int a1) {
        if (a0 >= a1) return;
        fence_proxy_async();
        tc_fence_before();
        __syncwarp();
        if (X.lane == 0)
            for (int a = a0; a < a1; ++a) mbar_arrive(bar0 + 8u * (kBarOpA + a));
    };
    // after chunk c0 of a phase of N columns: the atoms this warp has no
    // further chunk in are done (from its previous chunk's atom, or from 0
    // after its first chunk, up to its next chunk's atom)
    auto chunk_done = [&](int c0, int N) {
        const int nxt = c0 + 16 * kParts < N ? (c0 + 16 * kParts) >> 6 : (N + 63) >> 6;
        arrive_atoms(c0 < 16 * kParts ? 0 : c0 >> 6, nxt);
    };
    for (int u = blockIdx.x, tile_no = 0;; u += gridDim.x, ++tile_no) {
        const int t = u / nets, net = u - t * nets;
        int s, row0, nvalid;
        if (!tile_info(counts, t, s, row0, nvalid)) break;
        {
            const int es = net * kNSpecies + s;
            if (warp == 2) MLP_TC_MARK(0);
            const float* b1 = p.b1 + es * kH1;
            const float* b2 = p.b2 + es * kH2;
            const float* b3 = p.b3 + es * kH3;
            const float* w4 = p.W4 + es * kH3;

            // ---- E1: h1 = celu(D + b1)
            if (!epi_acc(X, 0)) break;
            if (warp == 2) MLP_TC_MARK(1);
#pragma unroll 1
            for (int c0 = 16 * part; c0 < kH1; c0 += 16 * kParts) {
                uint32_t d[16];
                tmem_ld16(X.tl + (uint32_t)c0, d);
                tmem_wait_ld();
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = celu_f(__uint_as_float(d[q]) + __ldg(b1 + c0 + q));
                store_act<SPLIT>(sbase, kOffH1, kOffH1lo, r, c0, v);
                chunk_done(c0, kH1);   // F2 starts on the finished atoms of h1
            }
            if (warp == 2) MLP_TC_MARK(2);

            // ---- E2: h2 = celu(D + b2)
            if (!epi_acc(X, 1)) break;
            if (warp == 2) MLP_TC_MARK(3);
#pragma unroll 1
            for (int c0 = 16 * part; c0 < kH2; c0 += 16 * kParts) {
                uint32_t d[16];
                tmem_ld16(X.tl + 256u + (uint32_t)c0, d);
                tmem_wait_ld();
                float v[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) v[q] = celu_f(__uint_as_float(d[q]) + __ldg(b2 + c0 + q));
                store_act<SPLIT>(sbase, kOffH2, kOffH2lo, r, c0, v);
                chunk_done(c0, kH2);   // F3 starts on the finished atoms of h2
            }
            if (warp == 2) MLP_TC_MARK(4);

            // ---- E3: energy (column-part partial sums per row, added in
            // fixed order by the last part, which has 3 of the 10 16-column
            // chunks, part 0 has 4) and g3 = w4 * celu'(z3). The finishing
            // part's global reads are issued before the accumulator is ready.
            int e_atom = 0;
            float e_b4 = 0.f;
            if (part == kParts - 1 && r < nvalid) {
                e_atom = p.row_atom[row0 + r];
                e_b4 = __ldg(p.b4 + es);
            }
            if (!epi_acc(X, 0)) break;
            if (warp == 2) MLP_TC_MARK(5);
            {
                float es_part = 0.f;
    #pragma unroll 1
                for (int c0 = 16 * part; c0 < kH3; c0 += 16 * kParts) {
                    uint32_t d[16];
                    tmem_ld16(X.tl + (uint32_t)c0, d);
                    tmem_wait_ld();
                    uint32_t pk[8];
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        // one exponential per element: exp(min(z, 0) / alpha) gives celu and celu'
                        const float z0 = __uint_as_float(d[2 * q]) + __ldg(b3 + c0 + 2 * q);
                        const float z1 = __uint_as_float(d[2 * q + 1]) + __ldg(b3 + c0 + 2 * q + 1);
                        const float w0 = __ldg(w4 + c0 + 2 * q), w1 = __ldg(w4 + c0 + 2 * q + 1);
                        const float x0 = __expf(fminf(z0, 0.f) * (1.f / kCeluAlpha));
                        const float x1 = __expf(fminf(z1, 0.f) * (1.f / kCeluAlpha));
                        es_part = fmaf(w0, z0 > 0.f ? z0 : kCeluAlpha * (x0 - 1.f), es_part);
                        es_part = fmaf(w1, z1 > 0.f ? z1 : kCeluAlpha * (x1 - 1.f), es_part);
                        pk[q] = pack_bf16(z0 > 0.f ? w0 : w0 * x0, z1 > 0.f ? w1 : w1 * x1);
                    }
                    if (p.backward) {
                        st_shared_v4(sbase + kOffG3 + op_off(r, c0), pk[0], pk[1], pk[2], pk[3]);
                        st_shared_v4(sbase + kOffG3 + op_off(r, c0 + 8), pk[4], pk[5], pk[6], pk[7]);
                        chunk_done(c0, kH3);   // B3 starts on the finished atoms of g3
                    }
                }
                const uint32_t ep = sbase + kOffEPart + (uint32_t)r * 128u + (uint32_t)((4 ^ (r & 7)) << 4);
                asm volatile("st.shared.f32 [%0], %1;" ::"r"(ep + 4u * (uint32_t)part), "f"(es_part) : "memory");
                __syncwarp();
                if (X.lane == 0) mbar_arrive(bar0 + 8u * kBarEPart);
                if (part == kParts - 1) {
                    if (!epi_wait(X, bar0 + 8u * kBarEPart, n_epart & 1u)) break;
                    if (r < nvalid) {
                        const uint4 v = ld_shared_v4(ep);
                        float e = e_b4;
                        e += __uint_as_float(v.x);
                        e += __uint_as_float(v.y);
                        e += __uint_as_float(v.z);
                        // ensemble: net k's energies go to row k of e[K][e_stride]
                        p.e[(ENS ? (size_t)net * (size_t)p.e_stride : 0) + e_atom] = e;
                    }
                }
                ++n_epart;
            }
            if (warp == 2) MLP_TC_MARK(6);
            if (!p.backward) {
                epi_arrive(X, op_bar);   // the next tile's F1 overwrites the half E3 read
                __syncwarp();
                if (X.lane == 0) mbar_arrive(bar0 + 8u * kBarStage);
                continue;
            }
            tc_fence_before();   // E3's accumulator reads are done (B3 writes the other half; B2 this one)

            // ---- EB3: g2 = D * celu'(z2) over h2
            if (!epi_acc(X, 1)) break;
            if (warp == 2) MLP_TC_MARK(7);
#pragma unroll 1
            for (int c0 = 16 * part; c0 < kH2; c0 += 16 * kParts) {
                uint32_t d[16];
                tmem_ld16(X.tl + 256u + (uint32_t)c0, d);
                tmem_wait_ld();
                store_grad(sbase, kOffH2, r, c0, d);
                chunk_done(c0, kH2);   // B2 starts on the finished atoms of g2
            }
            if (warp == 2) MLP_TC_MARK(8);

            // ---- EB2: g1 = D * celu'(z1) over h1
            if (!epi_acc(X, 0)) break;
            if (warp == 2) MLP_TC_MARK(9);
#pragma unroll 1
            for (int c0 = 16 * part; c0 < kH1; c0 += 16 * kParts) {
                uint32_t d[16];
                tmem_ld16(X.tl + (uint32_t)c0, d);
                tmem_wait_ld();
                store_grad(sbase, kOffH1, r, c0, d);
                if (b1_here) chunk_done(c0, kH1);   // B1's first block starts on the finished atoms of g1
            }
            epi_arrive(X, op_bar);   // accumulator half 0 read (B1's second block; an ensemble: the next F1)
            if (warp == 2) MLP_TC_MARK(10);

            if (ENS) {
                // ---- ensemble: g1 of this net -> global (four 128 x 64 boxes,
                // straight from the operand region) once every warp has written its part
                if (X.lane == 0) mbar_arrive(bar0 + 8u * kBarG1);
                if (warp == 2) {
                    int gok = 1;
                    if (X.lane == 0) {
                        gok = mbar_wait(bar0 + 8u * kBarG1, (uint32_t)tile_no & 1u, X.abrt) ? 1 : 0;
                        if (gok) {
                            for (int c = 0; c < kH1 / 64; ++c)
                                tma_store_2d(&M.G1, kH1 * net + 64 * c, row0, sbase + kOffH1 + (uint32_t)c * kAtom,
                                             stream_out);
                            bulk_wait_read0();   // read out of shared memory before the next unit's F1
                        }
                    }
                    if (!__shfl_sync(0xffffffffu, gok, 0)) break;
                }
                __syncwarp();
                if (X.lane == 0) mbar_arrive(bar0 + 8u * kBarStage);
                continue;
            }

            // ---- EB1: four 256-column blocks of dE/dG, 16 boxes of 64 columns
            // per tile; box g = 4 j + b goes to part g % 3. A warp converts its
            // boxes (its 32 rows) to BF16 in its 4 KB swizzled staging box and
            // writes each with one TMA store.
            bool jok = true;
            for (int j = 0; j < 4; ++j) {
                const int h = (j & 1) ^ 1;   // block 0 in half 1, block 1 in half 0, ...
                if (!epi_acc(X, h)) {
                    jok = false;
                    break;
                }
                if (warp == 2) MLP_TC_MARK(11 + 2 * j);
#pragma unroll 1
                for (int b = 0; b < 4; ++b) {
                    if ((4 * j + b) % kParts != part) continue;
                    uint32_t d[4][16];
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        tmem_ld16(X.tl + 256u * (uint32_t)h + (uint32_t)(64 * b + 16 * k), d[k]);
                    tmem_wait_ld();
                    const uint32_t rowb = stage_box + (uint32_t)X.lane * 128u;
                    const int y = row0 + 32 * (warp & 3);
                    if (X.lane == 0) bulk_wait_read0();   // the previous store has read the staging box
                    __syncwarp();
#pragma unroll
                    for (int k = 0; k < 4; ++k) {
#pragma unroll
                        for (int hh = 0; hh < 2; ++hh) {
                            const uint32_t* v = d[k] + 8 * hh;
                            const uint32_t chunk = (uint32_t)((2 * k + hh) ^ (X.lane & 7));
                            st_shared_v4(rowb + chunk * 16u,
                                         pack_bf16(__uint_as_float(v[0]), __uint_as_float(v[1])),
                                         pack_bf16(__uint_as_float(v[2]), __uint_as_float(v[3])),
                                         pack_bf16(__uint_as_float(v[4]), __uint_as_float(v[5])),
                                         pack_bf16(__uint_as_float(v[6]), __uint_as_float(v[7])));
                        }
                    }
                    fence_proxy_async();
                    __syncwarp();
                    if (X.lane == 0) tma_store_2d(&M.dG, 256 * j + 64 * b, y, stage_box, stream_out);
                }
                // this warp is done reading accumulator half h
                tc_fence_before();
                __syncwarp();
                if (X.lane == 0) mbar_arrive(bar0 + 8u * (kBarB1Free + h));
                if (warp == 2) MLP_TC_MARK(12 + 2 * j);
            }
            if (!jok) break;
            if (X.lane == 0) {
                bulk_wait_read0();
                mbar_arrive(bar0 + 8u * kBarStage);
            }
            __syncwarp();
            if (warp == 2) MLP_TC_MARK(19);
        }
    }
}

// ------------------------------------------------------------------ kernel
template <bool SPLIT, bool ENS>
__global__ void __launch_bounds__(kThreads, 1) k_mlp_tc(const __grid_constant__ TcMaps M, TcArgs p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) unsigned long long bars[kNBars];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int counts[8];
    __shared__ uint32_t consumed_par;   // teardown: the MMA issuer's consumed-load parities

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t bar0 = smem_u32(&bars[0]);
    volatile int* abrt = &abort_flag;

    if (tid == 0) {
        for (int q = 0; q < kNBars; ++q) {
            const bool epi = q == kBarOp || q == kBarB1Free || q == kBarB1Free + 1 || q == kBarStage ||
                             q == kBarEPart || q == kBarG1 || (q >= kBarOpA && q < kBarOpA + 4);
            mbar_init(bar0 + 8u * q, epi ? (uint32_t)kEpiWarps : 1u);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (tid < 8) counts[tid] = tid < kNSpecies ? p.ctr->species[tid] : 0;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    const bool backward = p.backward != 0;
    const int nets = ENS ? p.nets : 1;
    const bool b1 = backward && !ENS;   // the ensemble's B1 is k_mlp_b1_ens

    ProdState P;
    MmaState S;
    P.pend = P.epar = P.lpar = 0;
    S.fpar = 0;
    P.f1pos = P.rpos = S.f1pos = S.rpos = 0;
    P.geom = S.geom = 0xffffffffu;

    if (warp == 0) {
        if (lane == 0) producer<SPLIT>(M, counts, sbase, bar0, abrt, backward, b1, nets, P);
    } else if (warp == 1) {
        if (lane == 0) mma_issuer<SPLIT>(M, counts, sbase, tmem, bar0, abrt, backward, b1, nets, S);
    } else {
        EpiCtx X;
        X.sbase = sbase;
        X.bar0 = bar0;
        X.tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        X.abrt = abrt;
        X.lane = lane;
        X.part = (warp - 2) >> 2;
        X.r = (warp & 3) * 32 + lane;
        X.n_acc[0] = X.n_acc[1] = 0;
        epilogue<SPLIT, ENS>(M, p, counts, X, warp);
    }
    __syncwarp();

    // ---- teardown: drain own copies, MMAs and stores (bounded), free tensor memory
    if (warp == 1 && lane == 0) consumed_par = S.fpar;
    __syncthreads();
    if (warp == 0 && lane == 0 && abort_flag) {
        // at most one load per slot is ahead of the MMAs: the one whose count parity differs
        const uint32_t out = P.lpar ^ consumed_par;
        for (int b = 0; b < 8; ++b)
            if ((out >> b) & 1u) (void)mbar_wait_plain(full_bar(bar0, b), (consumed_par >> b) & 1u);
    }
    if (warp == 1 && lane == 0) {
        mma_commit(bar0 + 8u * kBarDrain);
        (void)mbar_wait_plain(bar0 + 8u * kBarDrain, 0u);
    }
    if (warp >= 2 && lane == 0) bulk_wait0();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && abort_flag) {
        // 1 | warp << 4 | barrier index << 12 for a timed-out wait
        const uint32_t a = (uint32_t)abort_flag;
        const uint32_t code = (a & 0x40000000u) ? 1u | (((a >> 20) & 0x3fu) << 4) | ((((a & 0xfffffu) - bar0) / 8u) << 12) : 1u;
        atomicOr(p.err, (int)code);
    }
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ ensemble dE/dG
// The ensemble's last backward layer as one GEMM per work item (tile t of
// 128 rows of element s, 256-column block j of dE/dG):
//   D[128 x 256] = sum over nets k, K chunks c of g1_k[:, 64c..] W1_k^T[256j.., 64c..]^T
//   dE/dG[rows, 256j ..] = BF16(D / K)
// A (g1, written by k_mlp_tc for every net) and B (W1^T of net k, element s)
// stream through a 4-stage ring; two TMEM accumulators of 256 columns let the
// epilogue of item i overlap the MMAs of item i + 1.
// Warps: 0 TMA producer, 1 MMA issuer, 2..5 epilogue (TMEM lane quarter
// warp % 4: 32 rows each, four 64-column boxes stored by TMA).
constexpr int kEnsStages = 4;
constexpr uint32_t kEnsStage = 3u * 16384u;                         // A 16 KB + B 32 KB
constexpr uint32_t kEnsOffStaging = (uint32_t)kEnsStages * kEnsStage;   // 4 x 4 KB, one per epilogue warp
constexpr uint32_t kEnsSmemAlloc = kEnsOffStaging + 4u * 4096u + 1024u;
constexpr int kEnsThreads = 32 * 6;
enum {
    kEnsFull = 0,       // 4: stage loaded
    kEnsEmpty = 4,      // 4: stage consumed (MMA commit)
    kEnsAccFull = 8,    // 2: accumulator complete (MMA commit)
    kEnsAccEmpty = 10,  // 2: accumulator read; one arrival per epilogue warp
    kEnsDrain = 12,     // 1: teardown MMA drain
    kEnsNBars = 13
};

struct EnsArgs {
    const Counters* ctr;
    int nets;
    float inv_nets;
    int* err;
};
struct EnsMaps {
    CUtensorMap G1, W1t, dG;
};

__global__ void __launch_bounds__(kEnsThreads, 1) k_mlp_b1_ens(const __grid_constant__ EnsMaps M, EnsArgs p) {
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    __shared__ __align__(8) unsigned long long bars[kEnsNBars];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_flag;
    __shared__ int counts[8];
    __shared__ uint32_t consumed_par;

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const uint32_t sbase = (smem_u32(smem_raw) + 1023u) & ~1023u;
    const uint32_t bar0 = smem_u32(&bars[0]);
    volatile int* abrt = &abort_flag;
    const int nq = 4 * p.nets;   // K chunks of 64 per item

    if (tid == 0) {
        for (int q = 0; q < kEnsNBars; ++q)
            mbar_init(bar0 + 8u * q, (q == kEnsAccEmpty || q == kEnsAccEmpty + 1) ? 4u : 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        abort_flag = 0;
    }
    if (tid < 8) counts[tid] = tid < kNSpecies ? p.ctr->species[tid] : 0;
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 512;" ::"r"(smem_u32(&tmem_slot))
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;
    uint32_t lpar = 0, fpar = 0;   // per stage: loads issued / loads consumed, parity

    if (warp == 0 && lane == 0) {
        prefetch_map(&M.G1);
        prefetch_map(&M.W1t);
        const uint64_t keep = policy_evict_last(), evict = policy_evict_first();
        uint32_t pend = 0, epar = 0;
        int pos = 0;
        bool ok = true;
        for (int i = blockIdx.x; ok; i += gridDim.x) {
            int s, row0, nvalid;
            if (!tile_info(counts, i >> 2, s, row0, nvalid)) break;
            const int j = i & 3;
            for (int q = 0; q < nq; ++q) {
                const int st = pos;
                pos = (pos + 1) & (kEnsStages - 1);
                const uint32_t m = 1u << st;
                if (pend & m) {
                    if (!mbar_wait(bar0 + 8u * (kEnsEmpty + st), (epar >> st) & 1u, abrt)) {
                        ok = false;
                        break;
                    }
                    epar ^= m;
                }
                const int k = q >> 2, c = q & 3;
                const uint32_t full = bar0 + 8u * (kEnsFull + st), dst = sbase + (uint32_t)st * kEnsStage;
                mbar_expect_tx(full, kEnsStage);
                // g1 tile: read by the four column-block items of the tile, then done
                tma_load_2d_hint(dst, &M.G1, kH1 * k + 64 * c, row0, full, j == 3 ? evict : keep);
                tma_load_2d_hint(dst + 16384u, &M.W1t, 64 * c, (k * kNSpecies + s) * kAevLd + 256 * j, full, keep);
                pend |= m;
                lpar ^= m;
            }
        }
    } else if (warp == 1 && lane == 0) {
        const uint32_t idesc = idesc_bf16(128, 256);
        int pos = 0, n_item = 0;
        bool ok = true;
        for (int i = blockIdx.x; ok; i += gridDim.x, ++n_item) {
            int s, row0, nvalid;
            if (!tile_info(counts, i >> 2, s, row0, nvalid)) break;
            const int h = n_item & 1;
            // accumulator h was last used by item n_item - 2: its epilogue must be done
            if (n_item >= 2 && !mbar_wait(bar0 + 8u * (kEnsAccEmpty + h), (uint32_t)((n_item >> 1) + 1) & 1u, abrt))
                break;
            tc_fence_after();
            const uint32_t d = tmem + 256u * (uint32_t)h;
            for (int q = 0; q < nq; ++q) {
                const int st = pos;
                pos = (pos + 1) & (kEnsStages - 1);
                if (!mbar_wait(bar0 + 8u * (kEnsFull + st), (fpar >> st) & 1u, abrt)) {
                    ok = false;
                    break;
                }
                fpar ^= 1u << st;
                tc_fence_after();
                const uint32_t base = sbase + (uint32_t)st * kEnsStage;
                const uint64_t ad = sdesc(base), bd = sdesc(base + 16384u);
#pragma unroll
                for (int k = 0; k < 4; ++k) mma_bf16(d, ad + 2u * k, bd + 2u * k, idesc, (q > 0 || k > 0) ? 1u : 0u);
                mma_commit(bar0 + 8u * (kEnsEmpty + st));
            }
            if (!ok) break;
            mma_commit(bar0 + 8u * (kEnsAccFull + h));
        }
    } else if (warp >= 2) {
        const uint32_t tl = tmem + ((uint32_t)((warp & 3) * 32) << 16);
        const uint32_t stage_box = sbase + kEnsOffStaging + (uint32_t)(warp - 2) * 4096u;
        const uint64_t stream_out = policy_evict_first();
        const float sc = p.inv_nets;
        int n_item = 0;
        for (int i = blockIdx.x;; i += gridDim.x, ++n_item) {
            int s, row0, nvalid;
            if (!tile_info(counts, i >> 2, s, row0, nvalid)) break;
            const int j = i & 3, h = n_item & 1;
            int ok = 1;
            if (lane == 0) ok = mbar_wait(bar0 + 8u * (kEnsAccFull + h), (uint32_t)(n_item >> 1) & 1u, abrt) ? 1 : 0;
            if (!__shfl_sync(0xffffffffu, ok, 0)) break;
            tc_fence_after();
            const uint32_t rowb = stage_box + (uint32_t)lane * 128u;
#pragma unroll 1
            for (int b = 0; b < 4; ++b) {
                uint32_t d[4][16];
#pragma unroll
                for (int k = 0; k < 4; ++k) tmem_ld16(tl + 256u * (uint32_t)h + (uint32_t)(64 * b + 16 * k), d[k]);
                tmem_wait_ld();
                if (lane == 0) bulk_wait_read0();   // the previous store has read the staging box
                __syncwarp();
#pragma unroll
                for (int k = 0; k < 4; ++k) {
#pragma unroll
                    for (int hh = 0; hh < 2; ++hh) {
                        const uint32_t* v = d[k] + 8 * hh;
                        const uint32_t chunk = (uint32_t)((2 * k + hh) ^ (lane & 7));
                        st_shared_v4(rowb + chunk * 16u,
                                     pack_bf16(__uint_as_float(v[0]) * sc, __uint_as_float(v[1]) * sc),
                                     pack_bf16(__uint_as_float(v[2]) * sc, __uint_as_float(v[3]) * sc),
                                     pack_bf16(__uint_as_float(v[4]) * sc, __uint_as_float(v[5]) * sc),
                                     pack_bf16(__uint_as_float(v[6]) * sc, __uint_as_float(v[7]) * sc));
                    }
                }
                fence_proxy_async();
                __syncwarp();
                if (lane == 0) tma_store_2d(&M.dG, 256 * j + 64 * b, row0 + 32 * (warp & 3), stage_box, stream_out);
            }
            // accumulator h read: the MMAs of item n_item + 2 may overwrite it
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(bar0 + 8u * (kEnsAccEmpty + h));
        }
    }
    __syncwarp();

    // ---- teardown: drain own copies, MMAs and stores (bounded), free tensor memory
    if (warp == 1 && lane == 0) consumed_par = fpar;
    __syncthreads();
    if (warp == 0 && lane == 0 && abort_flag) {
        const uint32_t out = lpar ^ consumed_par;   // at most one load per stage is ahead of the MMAs
        for (int b = 0; b < kEnsStages; ++b)
            if ((out >> b) & 1u) (void)mbar_wait_plain(bar0 + 8u * (kEnsFull + b), (consumed_par >> b) & 1u);
    }
    if (warp == 1 && lane == 0) {
        mma_commit(bar0 + 8u * kEnsDrain);
        (void)mbar_wait_plain(bar0 + 8u * kEnsDrain, 0u);
    }
    if (warp >= 2 && lane == 0) bulk_wait0();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0 && abort_flag) {
        const uint32_t a = (uint32_t)abort_flag;
        const uint32_t code = (a & 0x40000000u) ? 1u | (((a >> 20) & 0x3fu) << 4) | ((((a & 0xfffffu) - bar0) / 8u) << 12) : 1u;
        atomicOr(p.err, (int)(code | 0x100000u));   // bit 20: the ensemble dE/dG kernel
    }
    if (warp == 1) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 512;" ::"r"(tmem) : "memory");
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static const PFN_cuTensorMapEncodeTiled_v12000 fn = []() -> PFN_cuTensorMapEncodeTiled_v12000 {
        cudaDriverEntryPointQueryResult q;
        void* p = nullptr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
        cudaGetLastError();
        return nullptr;
    }();
    return fn;
}

// 2-D BF16 map over a row-major [rows x cols] matrix, box [box_rows x 64],
// 128-byte swizzle, zero fill outside the matrix.
bool make_map(CUtensorMap* m, const void* base, uint64_t cols, uint64_t rows, uint32_t box_rows,
              uint32_t box_cols = 64) {
    auto fn = encode_fn();
    if (!fn) return false;
    cuuint64_t dims[2] = {cols, rows};
    cuuint64_t strides[1] = {cols * 2};
    cuuint32_t box[2] = {box_cols, box_rows};
    cuuint32_t es[2] = {1, 1};
    CUresult r = fn(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, es,
                    CU_TENSOR_MAP_INTERLEAVE_NONE,
                    box_cols == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
                    CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
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

namespace {
// The network kernels' bounded wait on a barrier phase that never completes
// (nothing arrives): returns false after the 2 s limit with the waiting warp
// and barrier recorded, and the kernel exits normally (no copies or tensor
// memory outstanding). out[0] = 1 if the wait timed out, out[1] = the code.
__global__ void k_debug_wait_timeout(int* out) {
    __shared__ __align__(8) unsigned long long bar;
    __shared__ int abrt;
    const uint32_t b = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(b) : "memory");
        abrt = 0;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = mbar_wait(b, 0u, &abrt);
        out[0] = ok ? 0 : 1;
        out[1] = abrt;
    }
}
}  // namespace

int debug_wait_timeout(int* timed_out, int* code) {
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, 2 * sizeof(int));
    if (e != cudaSuccess) return (int)e;
    cudaMemset(d, 0, 2 * sizeof(int));
    k_debug_wait_timeout<<<1, 32>>>(d);
    int h[2] = {0, 0};
    e = cudaMemcpy(h, d, sizeof(h), cudaMemcpyDeviceToHost);
    cudaFree(d);
    if (e != cudaSuccess) return (int)e;
    *timed_out = h[0];
    *code = h[1];
    return 0;
}

// One map per weight matrix over all nets: rows of (net, element) block
// k * 7 + s start at (k * 7 + s) * rows-per-block.
bool make_weight_maps(NetBF16& w) {
    const uint64_t blocks = (uint64_t)w.n_nets * kNSpecies;
    bool ok = w.n_nets >= 1;
    ok &= make_map(&w.tmW1, w.W1, kAevLd, blocks * kH1, kH1);
    ok &= make_map(&w.tmW2, w.W2, kH1, blocks * kH2, kH2);
    ok &= make_map(&w.tmW3, w.W3, kH2, blocks * kH3, kH3);
    ok &= make_map(&w.tmW1lo, w.W1lo, kAevLd, blocks * kH1, kH1);
    ok &= make_map(&w.tmW2lo, w.W2lo, kH1, blocks * kH2, kH2);
    ok &= make_map(&w.tmW3lo, w.W3lo, kH2, blocks * kH3, kH3);
    ok &= make_map(&w.tmW3t, w.W3t, kH3, blocks * kH2, kH2);
    ok &= make_map(&w.tmW2t, w.W2t, kH2, blocks * kH1, kH1);
    ok &= make_map(&w.tmW1t, w.W1t, kH1, blocks * kAevLd, 256);
    w.maps_ok = ok;
    return ok;
}

bool launch_mlp_bf16(cudaStream_t st, int rows_cap, const Counters* ctr, const NetBF16& w, const __nv_bfloat16* G,
                     const __nv_bfloat16* G_lo, bool split, const int* row_atom, float* e, int e_stride,
                     __nv_bfloat16* dG, __nv_bfloat16* g1, bool backward, int* err_flag) {
    TcMaps M;
    const bool ens = w.n_nets > 1;
    if (!w.maps_ok || !make_map(&M.G, G, kAevLd, (uint64_t)rows_cap, 128) ||
        (split && (!G_lo || !make_map(&M.Glo, G_lo, kAevLd, (uint64_t)rows_cap, 128))) ||
        (backward && (!dG || !make_map(&M.dG, dG, kAevLd, (uint64_t)rows_cap, 32))) ||
        (backward && ens && (!g1 || !make_map(&M.G1, g1, (uint64_t)kH1 * w.n_nets, (uint64_t)rows_cap, 128)))) {
        set_error(-5, "TMA tensor map creation failed");
        return false;
    }
    if (!(backward && ens)) M.G1 = M.G;   // not used
    {   // split F1 boxes (32 columns); the W1 maps cover every net like the 64-column ones
        const uint64_t blocks = (uint64_t)w.n_nets * kNSpecies;
        if (!make_map(&M.Gn, G, kAevLd, (uint64_t)rows_cap, 128, 32) ||
            !make_map(&M.Glon, split ? G_lo : G, kAevLd, (uint64_t)rows_cap, 128, 32) ||
            !make_map(&M.W1n, w.W1, kAevLd, blocks * kH1, kH1, 32) ||
            !make_map(&M.W1lon, w.W1lo, kAevLd, blocks * kH1, kH1, 32)) {
            set_error(-5, "TMA tensor map creation failed");
            return false;
        }
    }
    if (!split) M.Glo = M.G;
    if (!backward) M.dG = M.G;   // not used
    M.W1 = w.tmW1;
    M.W1lo = w.tmW1lo;
    M.W2 = w.tmW2;
    M.W2lo = w.tmW2lo;
    M.W3 = w.tmW3;
    M.W3lo = w.tmW3lo;
    M.W3t = w.tmW3t;
    M.W2t = w.tmW2t;
    M.W1t = w.tmW1t;
    once_per_device((const void*)k_mlp_b1_ens, [] {
        cudaFuncSetAttribute(k_mlp_tc<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAlloc);
        cudaFuncSetAttribute(k_mlp_tc<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAlloc);
        cudaFuncSetAttribute(k_mlp_tc<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAlloc);
        cudaFuncSetAttribute(k_mlp_tc<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemAlloc);
        cudaFuncSetAttribute(k_mlp_b1_ens, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kEnsSmemAlloc);
    });
    const int sms = sm_count();
    const int tiles = rows_cap / kTileRows;
    const int units = tiles * w.n_nets;   // (tile, net) pairs, spread over the CTAs
    const int grid = units < sms ? units : sms;
    TcArgs a{ctr,          row_atom,   w.b1, w.b2, w.b3, w.W4, w.b4, e, e_stride, backward ? 1 : 0, w.n_nets,
             1.f / (float)w.n_nets, err_flag};
    if (ens) {
        if (split)
            MLP_LAUNCH("mlp_tc", st, k_mlp_tc<true, true><<<grid, kThreads, kSmemAlloc, st>>>(M, a));
        else
            MLP_LAUNCH("mlp_tc", st, k_mlp_tc<false, true><<<grid, kThreads, kSmemAlloc, st>>>(M, a));
        if (backward) {
            // mean dE/dG over the nets: one work item per (tile, 256-column block)
            EnsMaps EM;
            EM.G1 = M.G1;
            EM.W1t = w.tmW1t;
            EM.dG = M.dG;
            EnsArgs ea{ctr, w.n_nets, a.inv_nets, err_flag};
            const int items = 4 * tiles;
            const int egrid = items < sms ? items : sms;
            MLP_LAUNCH("mlp_tc_b1_ens", st, k_mlp_b1_ens<<<egrid, kEnsThreads, kEnsSmemAlloc, st>>>(EM, ea));
        }
    } else {
        if (split)
            MLP_LAUNCH("mlp_tc", st, k_mlp_tc<true, false><<<grid, kThreads, kSmemAlloc, st>>>(M, a));
        else
            MLP_LAUNCH("mlp_tc", st, k_mlp_tc<false, false><<<grid, kThreads, kSmemAlloc, st>>>(M, a));
    }
    return true;
}

}  // namespace mlp
