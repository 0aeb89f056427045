// Shared definitions of the CUDA path: AEV and network dimensions, device
// constant tables, the split-FP32 position format and small helpers.
//
// AEV hyper-parameters (ANI-2x shape; paper, section "OpenMM-ML"): radial
// cutoff 5.1 A with 16 Gaussian shifts evenly spaced over [0.8, 4.9] A and
// eta 19.7; angular cutoff 3.5 A with 4 distance shifts 0.8 + a * 0.675 A,
// 8 angle sections (2z + 1) pi / 16, eta 12.5, zeta 14.1. AEV length
// 7 * 16 + 28 * 4 * 8 = 1008, stored in rows of 1024 (zero padded).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace mlp {

constexpr int kNSpecies = 7;
constexpr int kRadShifts = 16;
constexpr int kAngA = 4;
constexpr int kAngZ = 8;
constexpr int kNPairs = 28;
constexpr int kRadLen = kNSpecies * kRadShifts;            // 112
constexpr int kAngLen = kNPairs * kAngA * kAngZ;           // 896
constexpr int kAevLen = kRadLen + kAngLen;                 // 1008
constexpr int kAevLd = 1024;                               // row stride of G / dG
constexpr int kH1 = 256, kH2 = 192, kH3 = 160;
constexpr int kTileRows = 128;                             // element-grouped row tile

constexpr float kRcRad = 5.1f;
constexpr float kEtaRad = 19.7f;
constexpr float kRcAng = 3.5f;
constexpr float kEtaAng = 12.5f;
constexpr float kZeta = 14.1f;
constexpr float kCeluAlpha = 0.1f;

// Angular neighbors (within 3.5 A) staged per atom by the AEV and force
// kernels: up to kAngCap in the main launches (the force kernel's fast path,
// one slot owner per lane, takes atoms with up to 32); atoms with more are
// handed to a second launch that stages up to kAngCapBig (more than any
// neighbor list holds: rows have at most 256 entries).
constexpr int kAngCap = 48;
constexpr int kAngCapBig = 256;

// Device constant tables, filled once per device by init_constants().
struct AevConsts {
    float shf_r[kRadShifts];
    float shf_a[kAngA];
    float cos_z[kAngZ];
    float sin_z[kAngZ];
    float hcos_z[kAngZ];   // cos_z / 2, sin_z / 2: 1 + cos(theta - theta_z) over 2 in two FMAs
    float hsin_z[kAngZ];
    float kzcos_z[kAngZ];  // (zeta / 2) cos_z: the section factors' derivative (force kernel)
};

// Orthorhombic box: L (float), split L = Lhi + Llo, 1/L; periodic = 0 for open.
struct Box {
    int periodic;
    float L[3];
    float Lhi[3];
    float Llo[3];
    float invL[3];
};

// Cell grid (cell path of the neighbor search), written on the device for
// open systems (bounding box) and on the host for periodic boxes.
struct Grid {
    int nc[3];
    int ncell;
    float origin[3];
    float inv_cs[3];
};

// Counters reset at the start of every evaluation.
struct alignas(16) Counters {
    int species[8];        // atoms per element (read as two 16-byte words)
    int nbr_overflow;      // largest neighbor count seen above capacity (0 = fine)
    int ang_overflow;      // largest angular neighbor count above kAngCapBig (0 = fine)
    int bad_species;       // bad input: 1 element code outside [0, 7), 2 molecule offsets, 4 ML-region index
    int rebuild;           // 1 if this evaluation rebuilds the neighbor list
    int net_error;         // tensor-core network kernel gave up on a bounded wait (0 = fine; else a code)
    int ang_big;           // atoms with more than kAngCap angular neighbors (listed for the second launch)
    int pad[2];
    // bounding box of an open system as order-preserving unsigned keys of
    // max(x) and max(-x), so that an all-zero reset is the identity
    unsigned bbox_max_key[3];
    unsigned bbox_negmin_key[3];
    int pad2[2];
};

__host__ __device__ inline int pair_index(int a, int b) {
    if (a > b) { int t = a; a = b; b = t; }
    return a * kNSpecies - (a * (a - 1)) / 2 + (b - a);
}

// Rows reserved for element s: counts padded to whole 128-row tiles.
__device__ __forceinline__ int padded_rows(int c) { return ((c + kTileRows - 1) / kTileRows) * kTileRows; }

__device__ __forceinline__ int row_base(const int* counts, int s) {
    int b = 0;
    for (int q = 0; q < s; ++q) b += padded_rows(counts[q]);
    return b;
}
// The same for a kernel that loads the element counts as two 16-byte words
// together with the atom's own data (one memory round trip instead of two:
// the prefix over the elements below s is formed in registers).
__device__ __forceinline__ void load_counts(const Counters* ctr, int4& c0, int4& c1) {
    c0 = reinterpret_cast<const int4*>(ctr->species)[0];
    c1 = reinterpret_cast<const int4*>(ctr->species)[1];
}
__device__ __forceinline__ int row_base(const int4& c0, const int4& c1, int s) {
    const int c[kNSpecies] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z};
    int b = 0;
#pragma unroll
    for (int q = 0; q < kNSpecies; ++q) b += q < s ? padded_rows(c[q]) : 0;
    return b;
}

// Tile t of the element-grouped row space -> (element, first row, valid rows);
// returns false past the last tile.
__device__ __forceinline__ bool tile_info(const int* counts, int t, int& s, int& row0, int& nvalid) {
    int base = 0;
    for (int q = 0; q < kNSpecies; ++q) {
        int c = counts[q];
        int ts = (c + kTileRows - 1) / kTileRows;
        if (t < ts) {
            s = q;
            row0 = base + t * kTileRows;
            nvalid = min(kTileRows, c - t * kTileRows);
            return true;
        }
        t -= ts;
        base += ts * kTileRows;
    }
    return false;
}

__device__ __forceinline__ float celu(float x) {
    return x > 0.f ? x : kCeluAlpha * (expf(x * (1.f / kCeluAlpha)) - 1.f);
}
__device__ __forceinline__ float celu_deriv(float x) { return x > 0.f ? 1.f : expf(x * (1.f / kCeluAlpha)); }

// Displacement x_j - x_i from split positions (hi + lo per axis), with the
// minimum image in periodic boxes. The hi difference is taken exactly as
// s + err (two-sum), the image shift n * Lhi is exact (n in {-1, 0, 1} for
// wrapped positions, Sterbenz), so only the final rounding to FP32 and the
// small lo terms add error: |error| ~ 1e-7 |d|, independent of the box size.
__device__ __forceinline__ float disp_axis(float hi_i, float lo_i, float hi_j, float lo_j, int periodic,
                                           float L, float Lhi, float Llo, float invL) {
    float s = hi_j - hi_i;
    float bb = s - hi_j;
    float err = (hi_j - (s - bb)) + (-hi_i - bb);
    float n = periodic ? rintf(s * invL) : 0.f;
    float main = s - n * Lhi;
    float rest = err + (lo_j - lo_i) - n * Llo;
    (void)L;
    return main + rest;
}

__device__ __forceinline__ float3 displacement(const float4& hi_i, const float4& lo_i, const float4& hi_j,
                                               const float4& lo_j, const Box& b) {
    float3 d;
    d.x = disp_axis(hi_i.x, lo_i.x, hi_j.x, lo_j.x, b.periodic, b.L[0], b.Lhi[0], b.Llo[0], b.invL[0]);
    d.y = disp_axis(hi_i.y, lo_i.y, hi_j.y, lo_j.y, b.periodic, b.L[1], b.Lhi[1], b.Llo[1], b.invL[1]);
    d.z = disp_axis(hi_i.z, lo_i.z, hi_j.z, lo_j.z, b.periodic, b.L[2], b.Lhi[2], b.Llo[2], b.invL[2]);
    return d;
}

__device__ __forceinline__ int species_of(const float4& hi) { return __float_as_int(hi.w); }

}  // namespace mlp
