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
// Work decomposition (one warp per atom; 1 warp per block forward, 2 backward):
//   * the neighbor list is read 32 entries at a time, one neighbor per lane
//     (displacement, distance, element, cutoff value in registers); only the
//     neighbors within 3.5 A are staged in shared memory, as unit vector,
//     distance, 1/r and cutoff values (the angular sub-list);
//   * radial (forward): four neighbors per step, taken from the lanes that
//     loaded them by shuffles, a quarter-warp each with two shifts per lane;
//     each lane owns its accumulator columns per element and quarter -> no
//     atomics, fixed order;
//   * angular: pairs are taken 32 at a time, ordered by element pair: one
//     pair per lane computes its 8 angle factors and 4 distance factors into
//     shared memory, then lane (a, z) adds the products, pair by pair, into
//     its own column 32 p + 8 a + z, written when the block's last pair is
//     in (conflict-free, fixed order -> deterministic).
// The backward recomputes the terms with their derivatives and contracts
// them with dE/dG (staged in shared memory as FP32: radial rows XOR-swizzled,
// angular rows padded): radial one neighbor per lane (16 unrolled
// exponentials), angular one pair per lane with its 4 distance and 8 angle
// factors in registers. Gradients on neighbors go to FP64 global sums:
// radial ones per neighbor; angular ones summed per angular neighbor first
// (in the registers of the lane that owns the neighbor for up to 16 or 21 to
// 32 of them, else in shared memory) and added once.
#include <cuda_bf16.h>

#include <type_traits>

#include "common.cuh"
#include "kernels.cuh"

namespace mlp {

__constant__ AevConsts c_aev;

void init_constants_for_current_device() {
    once_per_device(&c_aev, [] {
        AevConsts h;
        const double pi = 3.14159265358979323846;
        for (int k = 0; k < kRadShifts; ++k) h.shf_r[k] = (float)(0.8 + k * (4.9 - 0.8) / 15.0);
        for (int a = 0; a < kAngA; ++a) h.shf_a[a] = (float)(0.8 + a * (kRcAng - 0.8) / 4.0);
        for (int z = 0; z < kAngZ; ++z) {
            double Z = (2.0 * z + 1.0) * pi / 16.0;
            h.cos_z[z] = (float)cos(Z);
            h.sin_z[z] = (float)sin(Z);
            h.hcos_z[z] = (float)(0.5 * cos(Z));
            h.hsin_z[z] = (float)(0.5 * sin(Z));
            h.kzcos_z[z] = (float)(0.5 * 14.1 * cos(Z));   // zeta = 14.1
        }
        cudaMemcpyToSymbol(c_aev, &h, sizeof(h));
    });
}

namespace {

// Warps (one atom each) per block. Small blocks: a block's shared memory is
// released only when its slowest atom is done, so with atoms of uneven
// neighbor counts fewer warps per block keep more warps busy (measured:
// AEV 1 warp 12% faster than 8 per block; forces 2 warps 10% faster than 8,
// 1 warp 2.3% faster than 2).
constexpr int kAevWarps = 1;
constexpr int kForceWarps = 1;
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
    static __device__ __forceinline__ float rcp(float x) { return 1.f / x; }
    static __device__ __forceinline__ float gauss(float eta, float d) { return expf(-eta * d * d); }
};
template <>
struct M<true> {    // hardware approximations with subnormals flushed (BF16-network path)
    static __device__ __forceinline__ float ex2(float x) {
        float y;
        asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float lg2(float x) {
        float y;
        asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float rcp(float x) {
        float y;
        asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    static __device__ __forceinline__ float rsq(float x) {
        float y;
        asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
        return y;
    }
    // exp(x) = 2^(x log2 e); b^e = 2^(e log2 b)
    static __device__ __forceinline__ float ex(float x) { return ex2(x * 1.4426950408889634f); }
    static __device__ __forceinline__ float pw(float b, float e) { return ex2(e * lg2(b)); }
    // exp(-eta d^2) with -eta log2 e folded into one constant (eta is a compile-time constant)
    static __device__ __forceinline__ float gauss(float eta, float d) { return ex2((-eta * 1.4426950408889634f) * d * d); }
    static __device__ __forceinline__ float cpi(float x) {
        float y;
        asm("cos.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(3.14159265358979f * x));
        return y;
    }
    static __device__ __forceinline__ float spi(float x) {
        float y;
        asm("sin.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(3.14159265358979f * x));
        return y;
    }
    static __device__ __forceinline__ float sq(float x) { return x * rsq(fmaxf(x, 1e-30f)); }
    static __device__ __forceinline__ float dv(float a, float b) { return a * rcp(b); }
};

// Angular sub-list of one atom (neighbors within 3.5 A), CAP slots.
template <int CAP>
struct AngStage {
    float4 u[CAP];     // unit vector d / r, and r
    float4 w[CAP];     // 1 / r, fc(r; 3.5), d fc / dr, element (int bits): one 16-byte load
    int idx[CAP];      // atom index
};

// Angular pairs are processed in super-chunks of kSC pairs: one pair per
// lane computes its 8 section factors and 4 distance factors into rows of
// kFacRow floats (rows start 16-byte aligned, on banks 4 apart: the eight
// lanes of a quarter-warp reading four consecutive pairs of eight section
// rows cover all 32 banks), then lane (a, z) sums column 8 a + z of every
// element-pair block of the super-chunk. 32 pairs per super-chunk (measured
// 4% faster than 64: the smaller stage lets 32 instead of 26 one-warp blocks
// share an SM).
constexpr int kSC = 32;
constexpr int kFacRow = kSC + 4;

// Forward scratch of one warp (after its angular stage).
template <int CAP>
struct AevScratch {
    float accR[4 * kRadLen];    // radial accumulators [element][quarter][shift]: a warp's
                                // quarters (8 lanes, 2 shifts each) take one neighbor each;
                                // the two quarters of a half-warp use disjoint banks
    float pfT[kAngZ * kFacRow]; // 2 fc_j fc_k P_z of the super-chunk's pairs, section-major
    float rfT[kAngA * kFacRow]; // the 4 distance Gaussians, shift-major
    int ord[CAP];               // sorted (by element) position -> stage slot
    int blk[3 * kNPairs];       // present element-pair blocks, compacted: first pair, descriptor, pair index
};
// per-warp regions start on 16-byte boundaries (the stage holds float4)
__host__ __device__ constexpr size_t round16(size_t b) { return (b + 15) / 16 * 16; }
template <int CAP>
__host__ __device__ constexpr size_t aev_smem_per_warp() { return round16(sizeof(AngStage<CAP>) + sizeof(AevScratch<CAP>)); }
static_assert(sizeof(AngStage<kAngCap>) % 16 == 0 && sizeof(AngStage<kAngCapBig>) % 16 == 0,
              "AngStage must keep the per-warp regions 16-byte aligned");
// dE/dG staged for the backward as FP32, read as 16-byte groups of four
// columns: the radial block in rows of 16 floats per element, group g of row
// q stored at group g ^ (q & 3); the angular block in rows of 36 floats per
// element pair (32 columns and 4 of padding: rows start 4 banks apart), so
// that lanes reading the same group of rows of different element pairs hit
// different banks and every group sits at a fixed offset from its row.
constexpr int kGsRadStride = 16;
constexpr int kGsAngStride = 36;
constexpr int kGsRad = kNSpecies * kGsRadStride;
constexpr int kGsFloats = kGsRad + kNPairs * kGsAngStride;
__device__ __forceinline__ int gs_rad(int s, int g) { return kGsRadStride * s + 4 * (g ^ (s & 3)); }
__device__ __forceinline__ int gs_ang(int p, int g) { return kGsRad + kGsAngStride * p + 4 * g; }
template <int CAP>
__host__ __device__ constexpr size_t force_smem_per_warp() { return round16(sizeof(AngStage<CAP>) + (kGsFloats + 3 * CAP) * sizeof(float)); }
static_assert(aev_smem_per_warp<kAngCap>() % 16 == 0 && force_smem_per_warp<kAngCap>() % 16 == 0 &&
              force_smem_per_warp<kAngCapBig>() % 16 == 0, "per-warp shared regions must be 16-byte aligned");
static_assert(kRadLen % 8 == 0 && kAevLd % 8 == 0, "element-pair blocks of an AEV row start on 16 bytes");
static_assert(offsetof(AevScratch<kAngCap>, pfT) % 16 == 0 && offsetof(AevScratch<kAngCap>, rfT) % 16 == 0 &&
              offsetof(AevScratch<kAngCapBig>, pfT) % 16 == 0 && offsetof(AevScratch<kAngCapBig>, rfT) % 16 == 0 &&
              kFacRow % 4 == 0 && kSC == 32, "factor rows load four floats at a time; one pair per lane");
static_assert(offsetof(AevScratch<kAngCap>, accR) % 16 == 0 && sizeof(AngStage<kAngCap>) % 16 == 0 && kRadLen % 4 == 0,
              "radial accumulators are zeroed and read four at a time");
static_assert((sizeof(AngStage<kAngCap>) % 16) == 0 && (kGsRad % 4) == 0 && kGsRadStride == 16 &&
              kGsAngStride % 4 == 0 && (kGsAngStride / 4) % 2 == 1,
              "staged dE/dG rows are read as float4 groups (4 per radial row, 8 per angular row); angular rows "
              "start an odd number of 4-bank groups apart");
static_assert(kForceWarps * force_smem_per_warp<kAngCap>() + 1024 <= 233472 / (28 / kForceWarps),
              "28 force warps fit an SM's shared memory (each block also reserves 1 KB)");

__device__ __forceinline__ unsigned lanemask_lt() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}
__device__ __forceinline__ unsigned lanemask_le() {
    unsigned m;
    asm("mov.u32 %0, %%lanemask_le;" : "=r"(m));
    return m;
}

// One neighbor per lane: displacement, distance, element, atom index.
struct NbrLane {
    float3 d;
    float r;
    int sp, j;
    bool inR, inA;
};

template <bool FAST>
__device__ __forceinline__ NbrLane make_neighbor(int j, const float4& hj, const float4& lj, const float4& hi_i,
                                                 const float4& lo_i, const Box& box) {
    NbrLane nl;
    nl.d = make_float3(0.f, 0.f, 0.f);
    nl.r = 1.f;
    nl.sp = 0;
    nl.j = 0;
    nl.inR = nl.inA = false;
    if (j >= 0) {
        nl.j = j;
        nl.d = displacement(hi_i, lo_i, hj, lj, box);
        const float r2 = nl.d.x * nl.d.x + nl.d.y * nl.d.y + nl.d.z * nl.d.z;
        nl.r = FAST ? M<true>::sq(r2) : sqrtf(r2);
        nl.inR = nl.r < kRcRad;
        nl.inA = nl.r < kRcAng;
        nl.sp = species_of(hj);
    }
    return nl;
}

template <bool FAST>
__device__ __forceinline__ NbrLane load_neighbor(const AevArgs& a, const int* row, int q, int cnt,
                                                 const float4& hi_i, const float4& lo_i) {
    const int j = q < cnt ? row[q] : -1;
    float4 hj = make_float4(0.f, 0.f, 0.f, 0.f), lj = hj;
    if (j >= 0) {
        hj = a.hi[j];
        lj = a.lo[j];
    }
    return make_neighbor<FAST>(j, hj, lj, hi_i, lo_i, a.box);
}

// The first two chunks (list positions q and q + 32) with both chunks' loads
// in flight together: two dependent memory round trips instead of five for
// an atom with 33 to 64 neighbors. Returns the atom's neighbor count.
template <bool FAST>
__device__ __forceinline__ int load_neighbors2(const AevArgs& a, const int* row, const int* cnt_p, int q,
                                               const float4& hi_i, const float4& lo_i, NbrLane& n0, NbrLane& n1) {
    // the list entries are read up to the row's capacity before the count is
    // known (slots past the count hold stale indices and are discarded), so
    // count and entries take one round trip together
    int j0 = q < a.cap ? row[q] : -1, j1 = q + 32 < a.cap ? row[q + 32] : -1;
    const int cnt = min(*cnt_p, a.cap);
    if (q >= cnt) j0 = -1;
    if (q + 32 >= cnt) j1 = -1;
    float4 h0 = make_float4(0.f, 0.f, 0.f, 0.f), l0 = h0, h1 = h0, l1 = h0;
    if (j0 >= 0) {
        h0 = a.hi[j0];
        l0 = a.lo[j0];
    }
    if (j1 >= 0) {
        h1 = a.hi[j1];
        l1 = a.lo[j1];
    }
    n0 = make_neighbor<FAST>(j0, h0, l0, hi_i, lo_i, a.box);
    n1 = make_neighbor<FAST>(j1, h1, l1, hi_i, lo_i, a.box);
    return cnt;
}

// Appends this chunk's angular neighbors to the stage; returns the new count
// (which may exceed CAP: only the first CAP are staged). pA_out: this lane's
// slot in the stage (or -1: not an angular neighbor or past the stage).
template <bool FAST, int CAP>
__device__ __forceinline__ int stage_angular(const NbrLane& nl, int mA, AngStage<CAP>& s, int* pA_out = nullptr) {
    const unsigned bA = __ballot_sync(kFull, nl.inA);
    const int pA = mA + __popc(bA & lanemask_lt());
    if (pA_out) *pA_out = (nl.inA && pA < CAP) ? pA : -1;
    if (nl.inA && pA < CAP) {
        const float ir = M<FAST>::rcp(nl.r);
        s.u[pA] = make_float4(nl.d.x * ir, nl.d.y * ir, nl.d.z * ir, nl.r);
        s.w[pA] = make_float4(ir, 0.5f * M<FAST>::cpi(nl.r * (1.f / kRcAng)) + 0.5f,
                              -0.5f * (3.14159265358979f / kRcAng) * M<FAST>::spi(nl.r * (1.f / kRcAng)),
                              __int_as_float(nl.sp));
        s.idx[pA] = nl.j;
    }
    return mA + __popc(bA);
}

// Unordered pairs of the m angular neighbors, enumerated by rotation: for
// t = 1 .. (m - 1) / 2 the m pairs (j, (j + t) mod m), j = 0 .. m - 1, then
// for even m the m / 2 pairs (j, j + m / 2). Each pair appears once; pairs
// of consecutive positions have distinct j and distinct k as long as they
// span less than one rotation, so one pair per lane gives (nearly)
// conflict-free shared-memory traffic on both atoms of the pair.
struct PairIt {
    int j, t, m, tfull;
    __device__ __forceinline__ void init(int m_, int start) {
        m = m_;
        tfull = (m - 1) / 2;
        j = start;
        t = 1;
        norm();
    }
    __device__ __forceinline__ void norm() {
        while (t <= tfull && j >= m) {
            j -= m;
            ++t;
        }
    }
    __device__ __forceinline__ void advance(int step) {
        j += step;
        norm();
    }
    __device__ __forceinline__ int k() const {
        if (t > tfull) return j + (m >> 1);
        const int x = j + t;
        return x >= m ? x - m : x;
    }
};

// floor(l / c) for 0 <= l and 1 <= c. (l + 1/2) / c lies at least 1 / (2 c)
// from an integer; the approximate reciprocal and the product (relative
// error <= 2^-22 together) move it by at most l 2^-22 / c, which is below
// 1 / (2 c) for l < 2^21 — exact without a check for the main kernels
// (l < 60 * 59 / 2). The second launch stages up to 256 neighbors
// (l < 2^15); one correction step there makes it exact as well.
template <bool CHECK>
__device__ __forceinline__ int small_div(int l, int c) {
    int q = (int)(((float)l + 0.5f) * M<true>::rcp((float)c));
    if (CHECK) {
        if (q * c > l) --q;
        else if ((q + 1) * c <= l) ++q;
    }
    return q;
}

// One AEV value into the output row: FP32, or BF16 and (with out_lo) the
// BF16 rounding of the remainder (G = G_hi + G_lo to ~16 bits) for the
// split-precision network.
__device__ __forceinline__ void put_g(float* out, float*, int c, float v) { out[c] = v; }
__device__ __forceinline__ void put_g(__nv_bfloat16* out, __nv_bfloat16* out_lo, int c, float v) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    out[c] = h;
    if (out_lo) out_lo[c] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// Four consecutive AEV values (c a multiple of 4) in one 16-byte (FP32) or
// two 8-byte (BF16 hi, lo) stores; the same roundings as put_g.
__device__ __forceinline__ void put_g4(float* out, float*, int c, float4 v) { *reinterpret_cast<float4*>(out + c) = v; }
__device__ __forceinline__ void put_g4(__nv_bfloat16* out, __nv_bfloat16* out_lo, int c, float4 v) {
    const __nv_bfloat162 h01 = __floats2bfloat162_rn(v.x, v.y), h23 = __floats2bfloat162_rn(v.z, v.w);
    *reinterpret_cast<uint2*>(out + c) =
        make_uint2(*reinterpret_cast<const uint32_t*>(&h01), *reinterpret_cast<const uint32_t*>(&h23));
    if (out_lo) {
        const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
        const __nv_bfloat162 l01 = __floats2bfloat162_rn(v.x - f01.x, v.y - f01.y);
        const __nv_bfloat162 l23 = __floats2bfloat162_rn(v.z - f23.x, v.w - f23.y);
        *reinterpret_cast<uint2*>(out_lo + c) =
            make_uint2(*reinterpret_cast<const uint32_t*>(&l01), *reinterpret_cast<const uint32_t*>(&l23));
    }
}

// Zeros columns [c0, c1) of an AEV row (and of its lo row) with 16-byte
// stores; c0 and c1 are multiples of 16 bytes' worth of columns (every
// element-pair block starts on one: 112 + 32 p columns).
template <typename OutT>
__device__ __forceinline__ void zero_cols(OutT* out, OutT* out_lo, int c0, int c1, int lane) {
    constexpr int per = 16 / (int)sizeof(OutT);
    const int n = (c1 - c0) / per;
    uint4* d = reinterpret_cast<uint4*>(out + c0);
    uint4* dl = out_lo ? reinterpret_cast<uint4*>(out_lo + c0) : nullptr;
    for (int q = lane; q < n; q += 32) {
        d[q] = make_uint4(0u, 0u, 0u, 0u);
        if (dl) dl[q] = make_uint4(0u, 0u, 0u, 0u);
    }
}

// Element pair p (pair_index order: (0,0), (0,1), .., (0,6), (1,1), ..) as
// s1 | s2 << 4, eight pairs of 8 bits per 64-bit word (compile-time table).
__host__ __device__ constexpr unsigned long long pair_code_word(int w) {
    unsigned long long v = 0;
    int p = 0;
    for (int a = 0; a < kNSpecies; ++a)
        for (int b = a; b < kNSpecies; ++b, ++p)
            if (p / 8 == w) v |= (unsigned long long)(a | (b << 4)) << (8 * (p % 8));
    return v;
}
// Every entry p of the table decodes to the (s1, s2) whose pair_index
// (s1 7 - s1 (s1 - 1) / 2 + s2 - s1, the AEV column block) is p.
__host__ __device__ constexpr bool pair_table_ok() {
    for (int p = 0; p < kNPairs; ++p) {
        const int code = (int)((pair_code_word(p / 8) >> (8 * (p % 8))) & 0xffu), a = code & 15, b = code >> 4;
        if (!(a <= b && b < kNSpecies && a * kNSpecies - (a * (a - 1)) / 2 + (b - a) == p)) return false;
    }
    return true;
}
static_assert(kNPairs == 28 && pair_table_ok(), "element-pair table in pair_index order");

// Orders the m staged neighbors by element: ord[sorted position] = stage
// slot (stable within an element); lane e < 7 gets the size (cnt_e) and
// first sorted position (g_e) of element e's group.
template <int CAP>
__device__ __forceinline__ void sort_by_element(const AngStage<CAP>& s, int m, int* ord, int lane, int& cnt_e,
                                                int& g_e) {
    constexpr int NCH = (CAP + 31) / 32;
    int spv[NCH];
#pragma unroll
    for (int c = 0; c < NCH; ++c) spv[c] = c * 32 + lane < m ? __float_as_int(s.w[c * 32 + lane].w) : -1;
    const unsigned lt = lanemask_lt();
    int base = 0;
    cnt_e = 0;
    g_e = 0;
    for (int e = 0; e < kNSpecies; ++e) {
        int ce = 0;
#pragma unroll
        for (int c = 0; c < NCH; ++c) {
            if (c * 32 < m) {   // warp-uniform
                const unsigned b = __ballot_sync(kFull, spv[c] == e);
                if (spv[c] == e) ord[base + ce + __popc(b & lt)] = c * 32 + lane;
                ce += __popc(b);
            }
        }
        if (lane == e) {
            cnt_e = ce;
            g_e = base;
        }
        base += ce;
    }
}

// AEV row of atom i. Returns false (nothing written) when the atom has more
// than CAP angular neighbors.
template <bool FAST, typename OutT, int CAP>
__device__ __forceinline__ bool aev_atom(const AevArgs& a, OutT* __restrict__ G, OutT* __restrict__ G_lo,
                                         int* __restrict__ row_atom, int i, unsigned char* wsmem) {
    const int lane = threadIdx.x & 31;
    AngStage<CAP>& s = *reinterpret_cast<AngStage<CAP>*>(wsmem);
    AevScratch<CAP>& X = *reinterpret_cast<AevScratch<CAP>*>(wsmem + sizeof(AngStage<CAP>));
    const float4 hi_i = a.hi[i], lo_i = a.lo[i];
    int4 cs0, cs1;
    load_counts(a.ctr, cs0, cs1);
    const int rank_i = a.rank[i];
    const int* row = a.nbr + (size_t)i * a.cap;
    NbrLane nl0, nl1;
    const int cnt = load_neighbors2<FAST>(a, row, a.nbr_cnt + i, lane, hi_i, lo_i, nl0, nl1);
    for (int c = lane; c < kRadLen; c += 32) reinterpret_cast<float4*>(X.accR)[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    __syncwarp();

    // radial: four neighbors per step, a quarter-warp each, shifts 2 k2 and 2 k2 + 1 per lane
    const int k2 = 2 * (lane & 7), h = lane >> 3;
    const float R0 = c_aev.shf_r[k2], R1 = c_aev.shf_r[k2 + 1];
    float* accR = X.accR + h * kRadShifts + k2;
    int mA = 0;
    // radial terms straight from the lanes that loaded the neighbors
    auto chunk = [&](const NbrLane& nl, int base) {
        // fc(r) / 4: the radial prefactor folded into the shuffled cutoff value
        const float fcr = nl.inR ? fmaf(0.125f, M<FAST>::cpi(nl.r * (1.f / kRcRad)), 0.125f) : 0.f;
        const int nq = min(32, cnt - base);
        for (int q = 0; q < nq; q += 4) {
            const int src = q + h;
            const float rr = __shfl_sync(kFull, nl.r, src);
            const int ss = __shfl_sync(kFull, nl.sp, src);
            const float ff = __shfl_sync(kFull, fcr, src);
            if (src < nq && ff > 0.f) {
                float2* acc2 = reinterpret_cast<float2*>(accR + ss * 4 * kRadShifts);
                float2 v = *acc2;
                v.x += M<FAST>::gauss(kEtaRad, rr - R0) * ff;
                v.y += M<FAST>::gauss(kEtaRad, rr - R1) * ff;
                *acc2 = v;
            }
        }
        mA = stage_angular<FAST, CAP>(nl, mA, s);
    };
    if (cnt > 0) chunk(nl0, 0);
    if (cnt > 32) chunk(nl1, 32);
    for (int base = 64; base < cnt; base += 32) chunk(load_neighbor<FAST>(a, row, base + lane, cnt, hi_i, lo_i), base);
    if (mA > CAP) return false;   // warp-uniform
    __syncwarp();
    const int si = species_of(hi_i);
    const int rw = row_base(cs0, cs1, si) + rank_i;
    OutT* out = G + (size_t)rw * kAevLd;
    OutT* out_lo = G_lo ? G_lo + (size_t)rw * kAevLd : nullptr;

    // ---- angular. The sub-list is ordered by element (ord); the pairs are
    // enumerated element pair by element pair (the present blocks p, in
    // order), so that lane (a, z) sums its column of one 32-column block in a
    // register over the block's pairs and writes the block once: no
    // accumulator array, fixed order (deterministic).
    int cnt_e, g_e;   // lane e < 7: size and first sorted position of element e's group
    sort_by_element<CAP>(s, mA, X.ord, lane, cnt_e, g_e);
    int my_off, my_end, my_desc, my_p, np, P;
    {
        // lane p < 28: element pair (s1 <= s2) in pair_index order and its pair count
        const int pl = lane < kNPairs ? lane : 0;
        const unsigned long long pw = (pl >> 3) == 0   ? pair_code_word(0)
                                      : (pl >> 3) == 1 ? pair_code_word(1)
                                      : (pl >> 3) == 2 ? pair_code_word(2)
                                                       : pair_code_word(3);
        const int pcode = (int)((pw >> (8 * (pl & 7))) & 0xffu);
        const int s1 = pcode & 15, s2 = pcode >> 4;
        const int c1 = __shfl_sync(kFull, cnt_e, s1), c2 = __shfl_sync(kFull, cnt_e, s2);
        const int g1 = __shfl_sync(kFull, g_e, s1), g2 = __shfl_sync(kFull, g_e, s2);
        const int n = lane < kNPairs ? (s1 < s2 ? c1 * c2 : c1 * (c1 - 1) / 2) : 0;
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        P = __shfl_sync(kFull, incl, kNPairs - 1);
        // compact the present blocks: block q of np holds first pair, descriptor
        // (group starts g1, g2 and the divisor of its pair decoding: c2 for two
        // groups, c1 for one), element pair index
        const unsigned present = __ballot_sync(kFull, n > 0);
        np = __popc(present);
        if (n > 0) {
            const int q = __popc(present & lanemask_lt());
            X.blk[q] = incl - n;
            X.blk[kNPairs + q] = g1 | (g2 << 8) | ((s1 < s2 ? c2 : c1) << 16);
            X.blk[2 * kNPairs + q] = lane;
        }
        __syncwarp();
        my_off = lane < np ? X.blk[lane] : P;
        my_desc = lane < np ? X.blk[kNPairs + lane] : 0;
        my_p = lane < np ? X.blk[2 * kNPairs + lane] : kNPairs;
        my_end = __shfl_down_sync(kFull, my_off, 1);
        if (lane == 31) my_end = P;
    }
    {
        const int z = lane & 7, aa = lane >> 3;
        const float* pz = X.pfT + z * kFacRow;
        const float* ra = X.rfT + aa * kFacRow;
        // The angular columns start as zeros (absent blocks stay zero); each
        // present block's 32 columns are written once, when its last pair has
        // been added.
        zero_cols(out, out_lo, kRadLen, kAevLd, lane);
        __syncwarp();
        float acc = 0.f;
        for (int sb = 0; sb < P; sb += kSC) {
            const int n = min(kSC, P - sb);
            // block of pair e = sb + lane: blocks starting before sb, plus those
            // starting inside this super-chunk at or before the lane
            const unsigned before = __ballot_sync(kFull, my_off < sb);
            const unsigned starts = __reduce_or_sync(
                kFull, (lane < np && my_off >= sb && my_off < sb + 32) ? (1u << (my_off - sb)) : 0u);
            const int b = max(0, __popc(before) - 1 + __popc(starts & lanemask_le()));
            const int off_b = __shfl_sync(kFull, my_off, b);
            const int end_b = __shfl_sync(kFull, my_end, b);
            const int dsc = __shfl_sync(kFull, my_desc, b);
            const int p_b = __shfl_sync(kFull, my_p, b);
            const int e = sb + lane;
            bool last = false;   // pair e is the last of its block
            if (lane < n) {
                const int l = e - off_b;
                const int g1 = dsc & 255, g2 = (dsc >> 8) & 255, cdiv = dsc >> 16;
                const int q = small_div<(CAP > 64)>(l, cdiv);
                const int r = l - q * cdiv;
                int jj, kk;
                if (g1 != g2) {   // two groups: pair (q, r) of the rectangle
                    jj = g1 + q;
                    kk = g2 + r;
                } else {          // one group of cdiv: rotation q + 1, position r
                    const int x = r + q + 1;
                    jj = g1 + r;
                    kk = g1 + (x >= cdiv ? x - cdiv : x);
                }
                const int J = X.ord[jj], K = X.ord[kk];
                const float4 uj = s.u[J], uk = s.u[K], wj = s.w[J], wk = s.w[K];
                const float c = 0.95f * (uj.x * uk.x + uj.y * uk.y + uj.z * uk.z);
                const float sn = M<FAST>::sq(1.f - c * c);
                const float f2 = 2.f * wj.y * wk.y;
                // fast path: f2 b^zeta = 2^(zeta log2 b + log2 f2), one multiply fewer per section
                const float lf2 = FAST ? M<true>::lg2(f2) : 0.f;
                // sections z and 7 - z share sin: theta_(7-z) = pi - theta_z
#pragma unroll
                for (int zz = 0; zz < kAngZ / 2; ++zz) {
                    const float y = fmaf(sn, c_aev.hsin_z[zz], 0.5f);
                    const float b0 = fmaf(c, c_aev.hcos_z[zz], y);
                    const float b1 = fmaf(-c, c_aev.hcos_z[zz], y);
                    X.pfT[zz * kFacRow + lane] = FAST ? M<true>::ex2(fmaf(kZeta, M<true>::lg2(b0), lf2))
                                                      : f2 * M<false>::pw(b0, kZeta);
                    X.pfT[(kAngZ - 1 - zz) * kFacRow + lane] =
                        FAST ? M<true>::ex2(fmaf(kZeta, M<true>::lg2(b1), lf2)) : f2 * M<false>::pw(b1, kZeta);
                }
                const float rbar = 0.5f * (uj.w + uk.w);
#pragma unroll
                for (int q4 = 0; q4 < kAngA; ++q4)
                    X.rfT[q4 * kFacRow + lane] = M<FAST>::gauss(kEtaAng, rbar - c_aev.shf_a[q4]);
                last = e + 1 == end_b;
            }
            const unsigned ends = __ballot_sync(kFull, last);
            __syncwarp();
            // Lane (a, z) adds the super-chunk's products in pair order, four
            // pairs per pair of 16-byte loads (a quad with no block end as two
            // fused pair sums: one dependent add per quad); at a block's last
            // pair the sum goes to the block's column and restarts (the last
            // block may continue into the next super-chunk; its sum stays in
            // acc). Factors past n are stale, but no block ends there: what
            // they add is never written.
#pragma unroll
            for (int q = 0; q < kSC; q += 4) {
                if (q >= n) break;   // warp-uniform
                const float4 p4 = *reinterpret_cast<const float4*>(pz + q);
                const float4 r4 = *reinterpret_cast<const float4*>(ra + q);
                const unsigned e4 = (ends >> q) & 15u;
                if (e4 == 0u) {   // warp-uniform
                    acc += fmaf(p4.y, r4.y, p4.x * r4.x) + fmaf(p4.w, r4.w, p4.z * r4.z);
                } else {
                    const float pv[4] = {p4.x, p4.y, p4.z, p4.w}, rv[4] = {r4.x, r4.y, r4.z, r4.w};
#pragma unroll
                    for (int t = 0; t < 4; ++t) {
                        acc = fmaf(pv[t], rv[t], acc);
                        if (e4 & (1u << t)) {   // warp-uniform
                            const int pp = __shfl_sync(kFull, p_b, q + t);
                            put_g(out, out_lo, kRadLen + 32 * pp + lane, acc);
                            acc = 0.f;
                        }
                    }
                }
            }
            __syncwarp();   // the next super-chunk overwrites the factors
        }
    }
    // radial block (four quarters, added in a fixed order), four columns per lane
    if (lane < kRadLen / 4) {
        const float4* a4 = reinterpret_cast<const float4*>(X.accR + 4 * kRadShifts * (lane >> 2) + 4 * (lane & 3));
        const float4 q0 = a4[0], q1 = a4[kRadShifts / 4], q2 = a4[2 * kRadShifts / 4], q3 = a4[3 * kRadShifts / 4];
        put_g4(out, out_lo, 4 * lane,
               make_float4((q0.x + q1.x) + (q2.x + q3.x), (q0.y + q1.y) + (q2.y + q3.y), (q0.z + q1.z) + (q2.z + q3.z),
                           (q0.w + q1.w) + (q2.w + q3.w)));
    }
    if (lane == 0) row_atom[rw] = i;
    return true;
}

// Main AEV launch: one warp per atom, kAngCap staged angular neighbors; an
// atom with more is listed for k_aev_big (its flag is set, nothing written).
template <bool FAST, typename OutT>
__global__ void __launch_bounds__(kAevWarps * 32) k_aev(AevArgs a, OutT* __restrict__ G, OutT* __restrict__ G_lo,
                                                      int* __restrict__ row_atom) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int i = blockIdx.x * kAevWarps + w;
    if (i >= a.n) return;
    const bool done = aev_atom<FAST, OutT, kAngCap>(a, G, G_lo, row_atom, i, smem + w * aev_smem_per_warp<kAngCap>());
    if (lane == 0) {
        a.big_flag[i] = done ? 0 : 1;
        if (!done) a.big_list[atomicAdd(&a.ctr->ang_big, 1)] = i;
    }
}

// Second AEV launch: the listed atoms (usually none), kAngCapBig staged
// angular neighbors, one warp per atom, a fixed grid striding over the list.
template <bool FAST, typename OutT>
__global__ void __launch_bounds__(32) k_aev_big(AevArgs a, OutT* __restrict__ G, OutT* __restrict__ G_lo,
                                              int* __restrict__ row_atom) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nb = a.ctr->ang_big;
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        const int i = a.big_list[t];
        if (!aev_atom<FAST, OutT, kAngCapBig>(a, G, G_lo, row_atom, i, smem) && (threadIdx.x & 31) == 0)
            atomicMax(&a.ctr->ang_overflow, kAngCapBig + 1);
        __syncwarp();
    }
}

// d/dr of sum_k g_k 0.25 exp(-eta (r - R_k)^2) fc(r): the radial part of the
// backward for one neighbor (the 16 dE/dG entries of its element sp, staged
// in shared memory).
template <bool FAST>
__device__ __forceinline__ float radial_dEdr(const float* gs, int sp, float r, float fc, float dfc) {
    float gv[kRadShifts];
#pragma unroll
    for (int q = 0; q < kRadShifts / 4; ++q) {
        const float4 v = *reinterpret_cast<const float4*>(gs + gs_rad(sp, q));
        gv[4 * q] = v.x;
        gv[4 * q + 1] = v.y;
        gv[4 * q + 2] = v.z;
        gv[4 * q + 3] = v.w;
    }
    float s = 0.f;
    if constexpr (!FAST) {
#pragma unroll
        for (int k = 0; k < kRadShifts; ++k) {
            const float dk = r - c_aev.shf_r[k];
            s += gv[k] * M<false>::ex(-kEtaRad * dk * dk) * (-2.f * kEtaRad * dk * fc + dfc);
        }
    } else {
        // fast path: the 16 Gaussians as hardware exponentials, fully unrolled
        // (shifts from constant memory); measured 8% faster for the whole force
        // kernel than a two-sided recurrence from the nearest shift (3
        // exponentials, but rolled loops)
#pragma unroll
        for (int k = 0; k < kRadShifts; ++k) {
            const float dk = r - c_aev.shf_r[k];
            s = fmaf(gv[k] * M<true>::ex2(-kEtaRad * 1.4426950408889634f * dk * dk), -2.f * kEtaRad * dk * fc + dfc, s);
        }
    }
    return 0.25f * s;
}

// 8 consecutive dE/dG values (16-byte aligned) as floats
__device__ __forceinline__ void load8(const float* p, float (&v)[8]) {
    const float4 a = __ldg(reinterpret_cast<const float4*>(p)), b = __ldg(reinterpret_cast<const float4*>(p) + 1);
    v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
    v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}
__device__ __forceinline__ void load8(const __nv_bfloat16* p, float (&v)[8]) {
    const uint4 u = __ldg(reinterpret_cast<const uint4*>(p));
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        v[2 * q] = __uint_as_float(w[q] << 16);
        v[2 * q + 1] = __uint_as_float(w[q] & 0xffff0000u);
    }
}

// Forces of atom i's AEV terms (the AEV backward for one atom): gradients on
// i and on its neighbors into the FP64 sums grad. Returns false (nothing
// added) when the atom has more than CAP angular neighbors: the AEV's main
// launch has listed such an atom for the second launches.
template <bool FAST, typename TG, int CAP>
__device__ __forceinline__ bool force_atom(const AevArgs& a, const TG* __restrict__ dG, double* __restrict__ grad,
                                           int i, unsigned char* wsmem) {
    const int lane = threadIdx.x & 31;
    AngStage<CAP>& s = *reinterpret_cast<AngStage<CAP>*>(wsmem);
    float* gs = reinterpret_cast<float*>(wsmem + sizeof(AngStage<CAP>));
    float* fslot = gs + kGsFloats;
    const float4 hi_i = a.hi[i], lo_i = a.lo[i];
    int4 cs0, cs1;
    load_counts(a.ctr, cs0, cs1);
    const int si = species_of(hi_i);
    const int rw = row_base(cs0, cs1, si) + a.rank[i];
    const TG* grow = dG + (size_t)rw * kAevLd;
    // 8 columns per lane and load (16 B of BF16 or 32 B of FP32); the 8 stay
    // inside one radial block or one 32-column angular row. All of a lane's
    // loads are issued before the first store, so the row costs one memory
    // round trip, not four.
    const int* row = a.nbr + (size_t)i * a.cap;
    NbrLane nl0, nl1;
    int cnt;
    {
        float v[4][8];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = 8 * lane + 256 * q;
            if (c < kAevLen) load8(grow + c, v[q]);
        }
        // the first 64 neighbors' loads overlap the dE/dG row's
        cnt = load_neighbors2<FAST>(a, row, a.nbr_cnt + i, lane, hi_i, lo_i, nl0, nl1);
        // columns c .. c + 7 (groups g0 and g0 + 1 of one row): a radial row
        // for lanes 0..13 of q = 0, else angular column x = c - 112 of row
        // x / 32, staged at kGsRad + 36 (x / 32) + x % 32 = kGsRad + x + 4 (x / 32)
        static_assert(kGsAngStride == 36 && kRadLen == 112, "staging offsets below");
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int c = 8 * lane + 256 * q;
            if (c < kAevLen) {
                int o0, o1;
                if (q == 0 && c < kRadLen) {
                    const int rowq = c >> 4, g0 = (c & 15) >> 2;
                    o0 = gs_rad(rowq, g0);
                    o1 = gs_rad(rowq, g0 + 1);
                } else {
                    const int x = c - kRadLen;
                    o0 = kGsRad + x + 4 * (x >> 5);
                    o1 = o0 + 4;
                }
                *reinterpret_cast<float4*>(gs + o0) = make_float4(v[q][0], v[q][1], v[q][2], v[q][3]);
                *reinterpret_cast<float4*>(gs + o1) = make_float4(v[q][4], v[q][5], v[q][6], v[q][7]);
            }
        }
    }
    __syncwarp();

    // The angular neighbor count decides first whether the atom fits the
    // stage (nothing is added to grad before): from the first two chunks'
    // ballots, plus a counting pass over any further chunks (atoms with more
    // than 64 list entries).
    {
        int m = __popc(__ballot_sync(kFull, nl0.inA)) + __popc(__ballot_sync(kFull, nl1.inA));
        for (int base = 64; base < cnt; base += 32)
            m += __popc(__ballot_sync(kFull, load_neighbor<FAST>(a, row, base + lane, cnt, hi_i, lo_i).inA));
        if (m > CAP) return false;   // warp-uniform
    }

    float fix = 0.f, fiy = 0.f, fiz = 0.f;   // dE/dr_i partial sums of this lane
    int mA = 0;
    // radial: one neighbor per lane, staging the angular neighbors as it goes.
    // The gradient on an angular neighbor goes to its shared-memory slot
    // (every staged slot is written here: r < 3.5 A implies r < 5.1 A), added
    // to its angular gradient and flushed once; other neighbors go straight
    // to the FP64 sums.
    auto chunk = [&](const NbrLane& nl) {
        int pA;
        mA = stage_angular<FAST, CAP>(nl, mA, s, &pA);
        if (nl.inR) {
            const float x = nl.r * (1.f / kRcRad);
            const float fc = 0.5f * M<FAST>::cpi(x) + 0.5f;
            const float dfc = -0.5f * (3.14159265358979f / kRcRad) * M<FAST>::spi(x);
            const float sc = radial_dEdr<FAST>(gs, nl.sp, nl.r, fc, dfc) * M<FAST>::rcp(nl.r);
            const float gx = sc * nl.d.x, gy = sc * nl.d.y, gz = sc * nl.d.z;
            if (pA >= 0) {
                fslot[3 * pA] = gx;
                fslot[3 * pA + 1] = gy;
                fslot[3 * pA + 2] = gz;
            } else {
                atomicAdd(&grad[3 * (size_t)nl.j], (double)gx);
                atomicAdd(&grad[3 * (size_t)nl.j + 1], (double)gy);
                atomicAdd(&grad[3 * (size_t)nl.j + 2], (double)gz);
            }
            fix -= gx;
            fiy -= gy;
            fiz -= gz;
        }
    };
    if (cnt > 0) chunk(nl0);
    if (cnt > 32) chunk(nl1);
    for (int base = 64; base < cnt; base += 32) chunk(load_neighbor<FAST>(a, row, base + lane, cnt, hi_i, lo_i));
    __syncwarp();

    // angular: one pair (j, k) per lane, all 32 (shift, section) terms in registers.
    // pair_grad: the pair's gradients on j and k (and minus their sum on i).
    auto pair_grad = [&](int j, int kk, float3& gj, float3& gk) {
        const float4 uj = s.u[j], uk = s.u[kk], wj = s.w[j], wk = s.w[kk];
        const float cos0 = uj.x * uk.x + uj.y * uk.y + uj.z * uk.z;
        const float c = 0.95f * cos0;
        const float sn = M<FAST>::sq(1.f - c * c);
        // With Q_z = 2 b_z^(zeta - 1): P_z = 2 b_z^zeta = Q_z b_z and
        // dP_z/dc = (zeta / 2) Q_z sin(theta - theta_z) / sin theta
        //         = Q_z (K_z - B sin theta_z), K_z = (zeta / 2) cos theta_z,
        // B = (zeta / 2) c / sin theta (sin theta / sin theta cancels), no
        // reciprocal of b (b >= 0.066 for |c| <= 0.95 and the eight theta_z).
        const float B = 0.5f * kZeta * c * M<FAST>::rcp(sn);
        const float rbar = 0.5f * (uj.w + uk.w);
        const float fj = wj.y, fk = wk.y, dfj = wj.z, dfk = wk.z;
        const int p = pair_index(__float_as_int(wj.w), __float_as_int(wk.w));
        float P[kAngZ], D[kAngZ];
#pragma unroll
        for (int zz = 0; zz < kAngZ / 2; ++zz) {
            // sections zz and 7 - zz: theta_(7-zz) = pi - theta_zz (cos flips, sin stays)
            const float y = fmaf(sn, c_aev.hsin_z[zz], 0.5f);
            const float b0 = fmaf(c, c_aev.hcos_z[zz], y), b1 = fmaf(-c, c_aev.hcos_z[zz], y);
            float Q0, Q1;
            if (FAST) {
                Q0 = M<true>::ex2(fmaf(kZeta - 1.f, M<true>::lg2(b0), 1.f));
                Q1 = M<true>::ex2(fmaf(kZeta - 1.f, M<true>::lg2(b1), 1.f));
            } else {
                Q0 = 2.f * M<false>::pw(b0, kZeta - 1.f);
                Q1 = 2.f * M<false>::pw(b1, kZeta - 1.f);
            }
            const float t = B * c_aev.sin_z[zz];
            P[zz] = Q0 * b0;
            P[kAngZ - 1 - zz] = Q1 * b1;
            D[zz] = Q0 * (c_aev.kzcos_z[zz] - t);
            D[kAngZ - 1 - zz] = -Q1 * (c_aev.kzcos_z[zz] + t);
        }
        // Contracted over the sections first: W_a = sum_z g[a][z] P_z and
        // Wd_a = sum_z g[a][z] dP_z/dc (the pair's dE/dG row read as two
        // 4-column groups per shift); then T1 = sum_a W_a R_a, Sc = sum_a
        // Wd_a R_a, T2 = sum_a W_a dR_a/drbar with dR_a/drbar = -2 eta
        // (rbar - A_a) R_a.
        float Sc = 0.f, T1 = 0.f, T2 = 0.f;
#pragma unroll
        for (int aa = 0; aa < kAngA; ++aa) {
            const float4 g0 = *reinterpret_cast<const float4*>(gs + gs_ang(p, 2 * aa));
            const float4 g1 = *reinterpret_cast<const float4*>(gs + gs_ang(p, 2 * aa + 1));
            const float gg[8] = {g0.x, g0.y, g0.z, g0.w, g1.x, g1.y, g1.z, g1.w};
            float W = 0.f, Wd = 0.f;
#pragma unroll
            for (int z = 0; z < kAngZ; ++z) {
                W = fmaf(gg[z], P[z], W);
                Wd = fmaf(gg[z], D[z], Wd);
            }
            const float dr = rbar - c_aev.shf_a[aa];
            const float Ra = M<FAST>::gauss(kEtaAng, dr);
            const float WR = W * Ra;
            T1 += WR;
            T2 = fmaf(WR, dr, T2);
            Sc = fmaf(Wd, Ra, Sc);
        }
        T2 *= -2.f * kEtaAng;
        const float f = fj * fk;
        Sc *= f;
        const float Srj = 0.5f * f * T2 + dfj * fk * T1;
        const float Srk = 0.5f * f * T2 + fj * dfk * T1;
        // dE/d(d_ij) = (0.95 Sc / r_ij)(u_k - cos0 u_j) + Srj u_j
        //            = aj u_k + (Srj - aj cos0) u_j, and j <-> k
        const float aj = 0.95f * Sc * wj.x, ak = 0.95f * Sc * wk.x;
        const float cj = fmaf(-aj, cos0, Srj), ck = fmaf(-ak, cos0, Srk);
        const float gjx = fmaf(cj, uj.x, aj * uk.x), gjy = fmaf(cj, uj.y, aj * uk.y), gjz = fmaf(cj, uj.z, aj * uk.z);
        const float gkx = fmaf(ck, uk.x, ak * uj.x), gky = fmaf(ck, uk.y, ak * uj.y), gkz = fmaf(ck, uk.z, ak * uj.z);
        gj = make_float3(gjx, gjy, gjz);
        gk = make_float3(gkx, gky, gkz);
        fix -= gjx + gkx;
        fiy -= gjy + gky;
        fiz -= gjz + gkz;
    };
    if (CAP <= 64 && (mA <= 16 || (mA >= 21 && mA <= 32))) {   // warp-uniform
        // Slot owners, no shared-memory atomics: lane l = r m + j of group
        // r < g = 32 / m owns slot j. Group r takes rotations t = r + 1,
        // g + r + 1, ... (pairs (j, (j + t) mod m); for even m the last
        // rotation, t = m / 2, only for j < m / 2: every pair once). The
        // gradient on j stays in the lane's registers; the one on k goes to
        // k's owner in the same group (same t) by a shuffle. The groups' sums
        // of a slot are added into group 0 at the end (fixed order). For 17
        // to 20 slots one group leaves 12 to 15 lanes idle and takes m / 2
        // passes against ~m^2 / 64 packed ones: there the packed order with
        // shared atomics below measured faster (forces per served-stream
        // step: 3.03 ms with owners up to 32 slots, 2.98 with 17..20 packed,
        // 3.01 with 17..23, 3.04 with 17..27).
        float Fx = 0.f, Fy = 0.f, Fz = 0.f;
        if (mA >= 2) {
            const int g = 32 / mA, r = lane / mA, j = lane - r * mA;
            const int tf = (mA - 1) >> 1, T = (mA & 1) ? tf : tf + 1;
            for (int rho = 0; rho < T; rho += g) {
                const int t = rho + r + 1;
                const bool act = r < g && (t <= tf || (t == T && j < (mA >> 1)));
                float3 gj = make_float3(0.f, 0.f, 0.f), gk = gj;
                if (act) {
                    const int kk = j + t >= mA ? j + t - mA : j + t;
                    pair_grad(j, kk, gj, gk);
                }
                // the owner of slot j receives from the lane whose k is j (its j is j - t)
                const int src = r * mA + (j >= t ? j - t : j - t + mA);
                Fx += gj.x + __shfl_sync(kFull, gk.x, src);
                Fy += gj.y + __shfl_sync(kFull, gk.y, src);
                Fz += gj.z + __shfl_sync(kFull, gk.z, src);
            }
            const float ox = Fx, oy = Fy, oz = Fz;
            for (int q = 1; q < g; ++q) {
                Fx += __shfl_sync(kFull, ox, lane + q * mA);
                Fy += __shfl_sync(kFull, oy, lane + q * mA);
                Fz += __shfl_sync(kFull, oz, lane + q * mA);
            }
        }
        if (lane < mA) {   // slot lane: its angular sum plus its radial gradient
            const int jj = s.idx[lane];
            atomicAdd(&grad[3 * (size_t)jj], (double)(fslot[3 * lane] + Fx));
            atomicAdd(&grad[3 * (size_t)jj + 1], (double)(fslot[3 * lane + 1] + Fy));
            atomicAdd(&grad[3 * (size_t)jj + 2], (double)(fslot[3 * lane + 2] + Fz));
        }
    } else {
        // 17 to 20 or more than 32 slots (the latter rare in the main
        // launch; every atom of the second): pairs packed 32 per pass in
        // rotation order, the gradients added to the slots in shared memory
        // (atomics), flushed once
        const int P = mA * (mA - 1) / 2;
        PairIt it;
        it.init(mA, lane);
        for (int base = 0; base < P; base += 32) {
            if (base + lane < P) {
                const int j = it.j, kk = it.k();
                float3 gj, gk;
                pair_grad(j, kk, gj, gk);
                atomicAdd(&fslot[3 * j], gj.x);
                atomicAdd(&fslot[3 * j + 1], gj.y);
                atomicAdd(&fslot[3 * j + 2], gj.z);
                atomicAdd(&fslot[3 * kk], gk.x);
                atomicAdd(&fslot[3 * kk + 1], gk.y);
                atomicAdd(&fslot[3 * kk + 2], gk.z);
            }
            it.advance(32);
        }
        __syncwarp();
        for (int q = lane; q < mA; q += 32) {
            const int jj = s.idx[q];
            atomicAdd(&grad[3 * (size_t)jj], (double)fslot[3 * q]);
            atomicAdd(&grad[3 * (size_t)jj + 1], (double)fslot[3 * q + 1]);
            atomicAdd(&grad[3 * (size_t)jj + 2], (double)fslot[3 * q + 2]);
        }
    }
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
    return true;
}

// Main force launch: one warp per atom; an atom with more than kAngCap
// angular neighbors is left to the second launch (the AEV listed it).
// The BF16 instance (the served path) is held to 64 registers (shared
// memory then allows 29 one-warp blocks per SM); the FP32 instances would
// spill there (24 warps: <= 85 registers).
template <bool FAST, typename TG>
__global__ void __launch_bounds__(kForceWarps * 32, std::is_same<TG, __nv_bfloat16>::value ? 32 / kForceWarps : 24 / kForceWarps) k_forces(AevArgs a, const TG* __restrict__ dG,
                                                         double* __restrict__ grad) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int w = threadIdx.x >> 5;
    const int i = blockIdx.x * kForceWarps + w;
    if (i >= a.n) return;
    if (!force_atom<FAST, TG, kAngCap>(a, dG, grad, i, smem + w * force_smem_per_warp<kAngCap>()) &&
        (threadIdx.x & 31) == 0 && !a.big_flag[i])
        atomicMax(&a.ctr->ang_overflow, kAngCapBig + 1);   // not listed by the AEV: a mismatch, reported
}

// Second force launch: the atoms the AEV listed (usually none).
template <bool FAST, typename TG>
__global__ void __launch_bounds__(32) k_forces_big(AevArgs a, const TG* __restrict__ dG, double* __restrict__ grad) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int nb = a.ctr->ang_big;
    for (int t = blockIdx.x; t < nb; t += gridDim.x) {
        if (!force_atom<FAST, TG, kAngCapBig>(a, dG, grad, a.big_list[t], smem) && (threadIdx.x & 31) == 0)
            atomicMax(&a.ctr->ang_overflow, kAngCapBig + 1);
        __syncwarp();
    }
}

template <typename K>
void set_smem(K kernel, size_t bytes) {
    cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Grid of the second launches (listed atoms, usually none): they stride over
// the list; a small grid keeps an empty launch cheap (it only reads the count).
constexpr int kBigGrid = 32;

template <bool FAST, typename OutT>
void launch_aev_t(cudaStream_t st, const AevArgs& a, OutT* G, OutT* G_lo, int* row_atom) {
    const size_t sm = kAevWarps * aev_smem_per_warp<kAngCap>();
    const size_t smb = aev_smem_per_warp<kAngCapBig>();
    once_per_device((const void*)k_aev<FAST, OutT>, [&] {
        set_smem(k_aev<FAST, OutT>, sm);
        set_smem(k_aev_big<FAST, OutT>, smb);
    });
    const int gs = (a.n + kAevWarps - 1) / kAevWarps;
    MLP_LAUNCH("aev", st, k_aev<FAST, OutT><<<gs, kAevWarps * 32, sm, st>>>(a, G, G_lo, row_atom));
    MLP_LAUNCH("aev_big", st, k_aev_big<FAST, OutT><<<kBigGrid, 32, smb, st>>>(a, G, G_lo, row_atom));
}

template <bool FAST, typename TG>
void launch_forces_t(cudaStream_t st, const AevArgs& a, const TG* dG, double* grad) {
    const size_t sm = kForceWarps * force_smem_per_warp<kAngCap>();
    const size_t smb = force_smem_per_warp<kAngCapBig>();
    once_per_device((const void*)k_forces<FAST, TG>, [&] {
        set_smem(k_forces<FAST, TG>, sm);
        set_smem(k_forces_big<FAST, TG>, smb);
    });
    const int gs = (a.n + kForceWarps - 1) / kForceWarps;
    MLP_LAUNCH("forces", st, k_forces<FAST, TG><<<gs, kForceWarps * 32, sm, st>>>(a, dG, grad));
    MLP_LAUNCH("forces_big", st, k_forces_big<FAST, TG><<<kBigGrid, 32, smb, st>>>(a, dG, grad));
}

}  // namespace

void launch_aev_f32(cudaStream_t st, const AevArgs& a, float* G, int* row_atom, bool fast) {
    if (fast)
        launch_aev_t<true, float>(st, a, G, nullptr, row_atom);
    else
        launch_aev_t<false, float>(st, a, G, nullptr, row_atom);
}

void launch_aev_bf16(cudaStream_t st, const AevArgs& a, __nv_bfloat16* G, __nv_bfloat16* G_lo, int* row_atom,
                     bool fast) {
    if (fast)
        launch_aev_t<true, __nv_bfloat16>(st, a, G, G_lo, row_atom);
    else
        launch_aev_t<false, __nv_bfloat16>(st, a, G, G_lo, row_atom);
}

void launch_forces(cudaStream_t st, const AevArgs& a, const float* dG, const __nv_bfloat16* dG16, double* grad,
                   bool fast) {
    if (dG16)
        launch_forces_t<true, __nv_bfloat16>(st, a, dG16, grad);
    else if (fast)
        launch_forces_t<true, float>(st, a, dG, grad);
    else
        launch_forces_t<false, float>(st, a, dG, grad);
}

}  // namespace mlp
