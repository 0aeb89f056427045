// Staging and neighbor search.
//
// Staging turns FP64 coordinates into split FP32 positions (hi = rounded
// value, lo = remainder), wraps periodic positions into [0, L), counts atoms
// per element (the rank of each atom inside its element fixes its row in the
// element-grouped AEV matrix) and clears the FP64 force accumulators.
//
// Neighbor search ("building neighbor lists", paper section "Optimization
// Through NNPOps") produces a full list: every ordered pair (i, j), j != i,
// with |d_ij| < r_list, stored per atom in a fixed-capacity row nbr[i][cap]
// with the true count in nbr_cnt[i] (overflow is reported, never written
// past the row). Two builders:
//   * cell list: cells of side >= r_list over the periodic box (minimum
//     image) or over the bounding box of an open system; one warp per atom
//     scans the 27 surrounding cells, candidates in cell order and, inside a
//     cell, in atom order, so the list order is deterministic;
//   * all pairs inside each molecule, for batches of small open molecules
//     (the one-cell case of the same search).
#include "common.cuh"
#include "kernels.cuh"

#include <algorithm>

namespace mlp {

namespace {

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

// Order-preserving float -> unsigned key (0 below every float), for atomicMax.
__device__ __forceinline__ unsigned float_key(float f) {
    int i = __float_as_int(f);
    i = i >= 0 ? i : i ^ 0x7fffffff;
    return (unsigned)i ^ 0x80000000u;
}
__device__ __forceinline__ float key_float(unsigned k) {
    int i = (int)(k ^ 0x80000000u);
    return __int_as_float(i >= 0 ? i : i ^ 0x7fffffff);
}

// Warp-aggregated per-element counter: returns the atom's rank in its element.
__device__ __forceinline__ int element_rank(bool valid, int s, Counters* ctr) {
    int key = valid ? s : -1;
    unsigned grp = __match_any_sync(0xffffffffu, key);
    int leader = __ffs(grp) - 1;
    int lane = threadIdx.x & 31;
    int base = 0;
    if (valid && lane == leader) base = atomicAdd(&ctr->species[s], __popc(grp));
    base = __shfl_sync(0xffffffffu, base, leader);
    return base + __popc(grp & lanemask_lt());
}

__device__ __forceinline__ void split(double x, float& h, float& l) {
    h = (float)x;
    l = (float)(x - (double)h);
}

// Persistent lists: ref holds the positions of the last rebuild; an atom that
// moved more than half the skin since then (or force_rebuild) sets
// ctr->rebuild, and the cell/neighbor kernels of this evaluation run in full.
__global__ void k_stage_system(int n, const double* __restrict__ xyz, const int8_t* __restrict__ species,
                               double L0, double L1, double L2, int periodic, int want_bbox,
                               float4* __restrict__ hi, float4* __restrict__ lo, int* __restrict__ rank,
                               Counters* ctr, double* __restrict__ grad, const float4* __restrict__ ref,
                               float half_skin2, int force_rebuild) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    bool valid = i < n;
    if (force_rebuild && i == 0) ctr->rebuild = 1;
    int s = 0;
    float hx = 0.f, hy = 0.f, hz = 0.f;
    if (valid) {
        double x = xyz[3 * (size_t)i], y = xyz[3 * (size_t)i + 1], z = xyz[3 * (size_t)i + 2];
        if (periodic) {
            x -= L0 * floor(x / L0);
            y -= L1 * floor(y / L1);
            z -= L2 * floor(z / L2);
        }
        float lx, ly, lz;
        split(x, hx, lx);
        split(y, hy, ly);
        split(z, hz, lz);
        s = species[i];
        if (s < 0 || s >= kNSpecies) {
            atomicOr(&ctr->bad_species, 1);   // invalid element code: reported by the host
            s = 0;
        }
        hi[i] = make_float4(hx, hy, hz, __int_as_float(s));
        lo[i] = make_float4(lx, ly, lz, __int_as_float(0));
        grad[3 * (size_t)i] = 0.0;
        grad[3 * (size_t)i + 1] = 0.0;
        grad[3 * (size_t)i + 2] = 0.0;
        if (!force_rebuild && half_skin2 > 0.f) {
            float4 p = ref[i];
            float dx = hx - p.x, dy = hy - p.y, dz = hz - p.z;
            if (periodic) {
                dx -= (float)L0 * rintf(dx / (float)L0);
                dy -= (float)L1 * rintf(dy / (float)L1);
                dz -= (float)L2 * rintf(dz / (float)L2);
            }
            if (dx * dx + dy * dy + dz * dz > half_skin2) atomicOr(&ctr->rebuild, 1);
        }
    }
    int r = element_rank(valid, s, ctr);
    if (valid) rank[i] = r;
    if (want_bbox) {
        float mn[3] = {valid ? hx : 3.0e38f, valid ? hy : 3.0e38f, valid ? hz : 3.0e38f};
        float mx[3] = {valid ? hx : -3.0e38f, valid ? hy : -3.0e38f, valid ? hz : -3.0e38f};
        for (int a = 0; a < 3; ++a) {
            for (int o = 16; o > 0; o >>= 1) {
                mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
                mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
            }
        }
        if ((threadIdx.x & 31) == 0) {
            for (int a = 0; a < 3; ++a) {
                atomicMax(&ctr->bbox_negmin_key[a], float_key(-mn[a]));
                atomicMax(&ctr->bbox_max_key[a], float_key(mx[a]));
            }
        }
    }
}

// One block per molecule: atoms mol_start[m] .. mol_start[m+1]; lo.w = m.
// Molecule bounds outside [0, n_atoms] (device input) are flagged as bad
// input and skipped; the host then reports the evaluation invalid.
__global__ void k_stage_batch(int n_mols, int n_atoms, const int* __restrict__ mol_start,
                              const double* __restrict__ xyz, const int8_t* __restrict__ species,
                              float4* __restrict__ hi, float4* __restrict__ lo, int* __restrict__ rank,
                              Counters* ctr, double* __restrict__ grad) {
    // mol_start == nullptr: one molecule of n_atoms atoms (a small open system)
    int m = blockIdx.x;
    int a = mol_start ? mol_start[m] : 0, b = mol_start ? mol_start[m + 1] : n_atoms;
    if (mol_start && m == 0 && threadIdx.x == 0 && (a != 0 || mol_start[n_mols] != n_atoms))
        atomicOr(&ctr->bad_species, 2);
    if (a < 0 || b < a || b > n_atoms) {
        if (threadIdx.x == 0) atomicOr(&ctr->bad_species, 2);
        return;
    }
    // element ranks aggregated per block: one global atomic per element
    // present in the block's chunk (a molecule's atoms) instead of one per
    // element and warp
    __shared__ int cnt[kNSpecies], off[kNSpecies];
    for (int base = a; base < b; base += blockDim.x) {
        int i = base + threadIdx.x;
        bool valid = i < b;
        int s = 0;
        if (threadIdx.x < kNSpecies) cnt[threadIdx.x] = 0;
        __syncthreads();
        int local = 0;
        if (valid) {
            float hx, hy, hz, lx, ly, lz;
            split(xyz[3 * (size_t)i], hx, lx);
            split(xyz[3 * (size_t)i + 1], hy, ly);
            split(xyz[3 * (size_t)i + 2], hz, lz);
            s = species[i];
            if (s < 0 || s >= kNSpecies) {
                atomicOr(&ctr->bad_species, 1);
                s = 0;
            }
            hi[i] = make_float4(hx, hy, hz, __int_as_float(s));
            lo[i] = make_float4(lx, ly, lz, __int_as_float(m));
            grad[3 * (size_t)i] = 0.0;
            grad[3 * (size_t)i + 1] = 0.0;
            grad[3 * (size_t)i + 2] = 0.0;
            local = atomicAdd(&cnt[s], 1);
        }
        __syncthreads();
        if (threadIdx.x < kNSpecies && cnt[threadIdx.x] > 0)
            off[threadIdx.x] = atomicAdd(&ctr->species[threadIdx.x], cnt[threadIdx.x]);
        __syncthreads();
        if (valid) rank[i] = off[s] + local;
    }
}

// Warp per atom: every j of the atom's molecule (mol_start == nullptr: the
// n atoms are one molecule).
__global__ void k_nbr_allpairs(int n, int n_mols, const int* __restrict__ mol_start, NbrArgs a, Counters* ctr) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n) return;
    int i = warp;
    float4 hi_i = a.hi[i], lo_i = a.lo[i];
    int m = __float_as_int(lo_i.w);
    int beg = 0, end = 0;
    if (m >= 0 && m < n_mols) {   // mol_start == nullptr: one molecule [0, n)
        beg = mol_start ? mol_start[m] : 0;
        end = mol_start ? mol_start[m + 1] : n;
    }
    if (beg < 0 || end > n || beg > end || i < beg || i >= end) {
        // atom not covered by a valid molecule (bad device input, already flagged)
        beg = end = 0;
    }
    Box box{};
    int count = 0;
    int* row = a.nbr + (size_t)i * a.cap;
    // r_ij < r_list from the hi parts alone unless r^2 falls within the
    // bound of that shortcut's error of r_list^2; there the split-precision
    // displacement decides, so the list is the one the exact test gives.
    // Error of the hi-only displacement per axis <= 2^-23 (|x_i| + |x_j|)
    // (the lo parts and one rounding), taken twice: tau = 2^-22 times the L1
    // norms; |r^2 - r^2_exact| <= 2 |d| tau + tau^2 + roundings of the sums.
    const float rl = sqrtf(a.rl2);
    const float l1_i = fabsf(hi_i.x) + fabsf(hi_i.y) + fabsf(hi_i.z);
    auto within = [&](const float4& hj, int j) -> bool {
        const float dx = hj.x - hi_i.x, dy = hj.y - hi_i.y, dz = hj.z - hi_i.z;
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float tau = 2.384185791015625e-7f * (l1_i + fabsf(hj.x) + fabsf(hj.y) + fabsf(hj.z));
        const float margin = fmaf(4.f * rl, tau, fmaf(2.f * tau, tau, 9.5367431640625e-7f * a.rl2));
        if (r2 < a.rl2 - margin) return true;
        if (r2 > a.rl2 + margin) return false;
        const float4 lj = a.lo[j];   // the lo parts only for the rare pairs near the list radius
        const float3 d = displacement(hi_i, lo_i, hj, lj, box);
        return d.x * d.x + d.y * d.y + d.z * d.z < a.rl2;
    };
    auto emit = [&](int j, bool ok) {
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        int pos = count + __popc(mask & lanemask_lt());
        if (ok && pos < a.cap) row[pos] = j;
        count += __popc(mask);
    };
    // two chunks of 32 candidates per pass, both chunks' positions loaded
    // before either is tested (one memory round trip per 64 candidates)
    for (int base = beg; base < end; base += 64) {
        const int j0 = base + lane, j1 = base + 32 + lane;
        const float4 z4 = make_float4(0.f, 0.f, 0.f, 0.f);
        float4 h0 = z4, h1 = z4;
        if (j0 < end) h0 = a.hi[j0];
        if (j1 < end) h1 = a.hi[j1];
        emit(j0, j0 < end && j0 != i && within(h0, j0));
        if (base + 32 < end) emit(j1, j1 < end && j1 != i && within(h1, j1));
    }
    if (lane == 0) {
        a.nbr_cnt[i] = count;
        if (count > a.cap) atomicMax(&ctr->nbr_overflow, count);
    }
}

// Grid over the bounding box of an open system (single thread).
__global__ void k_grid_setup(Counters* ctr, Grid* g, float r_list, int max_cells) {
    if (!ctr->rebuild) return;
    float mn[3], ext[3];
    for (int a = 0; a < 3; ++a) {
        mn[a] = -key_float(ctr->bbox_negmin_key[a]);
        float mx = key_float(ctr->bbox_max_key[a]);
        ext[a] = fmaxf(mx - mn[a], 0.f) + 2e-3f;
        mn[a] -= 1e-3f;
    }
    float cs = r_list;
    int nc[3] = {1, 1, 1};
    bool fits = false;
    for (int it = 0; it < 96 && !fits; ++it) {
        long long tot = 1;
        for (int a = 0; a < 3; ++a) {
            float f = floorf(ext[a] / cs);
            nc[a] = (f >= 1.f && f < 1.0e6f) ? (int)f : (f >= 1.0e6f ? 1000000 : 1);
            tot *= nc[a];
        }
        fits = tot <= max_cells;
        if (!fits) cs *= 1.25f;
    }
    if (!fits) nc[0] = nc[1] = nc[2] = 1;   // degenerate input: one cell, still exact
    for (int a = 0; a < 3; ++a) {
        g->nc[a] = nc[a];
        g->origin[a] = mn[a];
        // cells are at least r_list wide: ext / nc >= cs >= r_list
        g->inv_cs[a] = (float)nc[a] / ext[a];
    }
    g->ncell = nc[0] * nc[1] * nc[2];
}

__device__ __forceinline__ int cell_coord(float x, float origin, float inv_cs, int nc) {
    int c = (int)floorf((x - origin) * inv_cs);
    return min(max(c, 0), nc - 1);
}

__global__ void k_cell_count(int n, const float4* __restrict__ hi, const Grid* __restrict__ g,
                             int* __restrict__ cell_of_atom, int* __restrict__ cell_rank,
                             int* __restrict__ cell_count, const Counters* __restrict__ ctr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !ctr->rebuild) return;
    float4 p = hi[i];
    int cx = cell_coord(p.x, g->origin[0], g->inv_cs[0], g->nc[0]);
    int cy = cell_coord(p.y, g->origin[1], g->inv_cs[1], g->nc[1]);
    int cz = cell_coord(p.z, g->origin[2], g->inv_cs[2], g->nc[2]);
    int c = (cz * g->nc[1] + cy) * g->nc[0] + cx;
    cell_of_atom[i] = c;
    cell_rank[i] = atomicAdd(&cell_count[c], 1);
}

// Exclusive scan of the cell counts: one block of 1024 threads, each thread
// summing kScanPer consecutive cells per round (16,384 cells a round).
constexpr int kScanPer = 16;
__global__ void __launch_bounds__(1024) k_cell_scan(const Grid* __restrict__ g, const int* __restrict__ cell_count,
                            int* __restrict__ cell_start, const Counters* __restrict__ ctr) {
    if (!ctr->rebuild) return;
    __shared__ int warp_sums[32];
    __shared__ int carry;
    const int ncell = g->ncell;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    for (int base = 0; base < ncell; base += kScanPer * 1024) {
        const int c0 = base + kScanPer * threadIdx.x;
        int v[kScanPer], t = 0;
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            v[k] = c0 + k < ncell ? cell_count[c0 + k] : 0;
            t += v[k];
        }
        int x = t;
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        if (w == 0) {
            int sm = warp_sums[lane];
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, sm, o);
                if (lane >= o) sm += y;
            }
            warp_sums[lane] = sm;
        }
        __syncthreads();
        int run = x - t + (w > 0 ? warp_sums[w - 1] : 0) + carry;   // exclusive start of this thread's cells
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) {
            if (c0 + k < ncell) cell_start[c0 + k] = run;
            run += v[k];
        }
        __syncthreads();
        if (threadIdx.x == 1023) carry = run;
        __syncthreads();
    }
    if (threadIdx.x == 0) cell_start[ncell] = carry;
}

__global__ void k_cell_scatter(int n, const int* __restrict__ cell_of_atom, const int* __restrict__ cell_rank,
                               const int* __restrict__ cell_start, int* __restrict__ cell_atoms,
                               const Counters* __restrict__ ctr) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || !ctr->rebuild) return;
    cell_atoms[cell_start[cell_of_atom[i]] + cell_rank[i]] = i;
}

// Each cell's atoms in index order, so that the neighbor order does not
// depend on the order of the counting atomics: one warp per cell; an atom's
// place is the number of atoms of the cell with a smaller index (cells of up
// to 256 atoms, read once into registers; larger ones, which only degenerate
// inputs make, are sorted by one lane).
constexpr int kSortChunks = 8;
__device__ __forceinline__ void sort_cell(int a, int m, int* __restrict__ cell_atoms, int lane) {
    if (m <= 1) return;
    if (m > 32 * kSortChunks) {
        if (lane == 0)
            for (int p = a + 1; p < a + m; ++p) {
                const int v = cell_atoms[p];
                int q = p - 1;
                while (q >= a && cell_atoms[q] > v) {
                    cell_atoms[q + 1] = cell_atoms[q];
                    --q;
                }
                cell_atoms[q + 1] = v;
            }
        return;
    }
    int v[kSortChunks], rank[kSortChunks];
#pragma unroll
    for (int k = 0; k < kSortChunks; ++k) {
        v[k] = 32 * k + lane < m ? cell_atoms[a + 32 * k + lane] : 0x7fffffff;
        rank[k] = 0;
    }
    const int nch = (m + 31) >> 5;
#pragma unroll
    for (int k2 = 0; k2 < kSortChunks; ++k2) {
        if (k2 >= nch) break;   // warp-uniform
        for (int u = 0; u < 32; ++u) {
            const int w = __shfl_sync(0xffffffffu, v[k2], u);
#pragma unroll
            for (int k = 0; k < kSortChunks; ++k)
                if (k < nch) rank[k] += w < v[k] ? 1 : 0;
        }
    }
    __syncwarp();
#pragma unroll
    for (int k = 0; k < kSortChunks; ++k)
        if (32 * k + lane < m) cell_atoms[a + rank[k]] = v[k];
}

__global__ void k_cell_sort(const Grid* __restrict__ g, const int* __restrict__ cell_start,
                            int* __restrict__ cell_atoms, const Counters* __restrict__ ctr) {
    const int lane = threadIdx.x & 31;
    if (!ctr->rebuild) return;
    const int ncell = g->ncell, nw = (gridDim.x * blockDim.x) >> 5;
    for (int c = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncell; c += nw)   // warp-uniform
        sort_cell(cell_start[c], cell_start[c + 1] - cell_start[c], cell_atoms, lane);
}

constexpr int kNbrCellWarps = 8;   // warps (atoms) per block of k_nbr_cell

__global__ void k_nbr_cell(int n, NbrArgs a, Box box, const Grid* __restrict__ g,
                           const int* __restrict__ cell_of_atom, const int* __restrict__ cell_start,
                           const int* __restrict__ cell_atoms, Counters* ctr, float4* __restrict__ ref) {
    int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int lane = threadIdx.x & 31;
    if (warp >= n || !ctr->rebuild) return;
    int i = warp;
    float4 hi_i = a.hi[i], lo_i = a.lo[i];
    if (lane == 0) ref[i] = hi_i;
    int nc0 = g->nc[0], nc1 = g->nc[1], nc2 = g->nc[2];
    int c = cell_of_atom[i];
    int cx = c % nc0, cy = (c / nc0) % nc1, cz = c / (nc0 * nc1);
    int count = 0;
    int* row = a.nbr + (size_t)i * a.cap;
    // per axis: three relative cells, or (periodic box with fewer than three
    // cells along the axis) every cell once
    int lo3[3], hi3[3], rel[3];
    const int ncs[3] = {nc0, nc1, nc2};
    for (int ax = 0; ax < 3; ++ax) {
        if (box.periodic && ncs[ax] < 3) {
            lo3[ax] = 0;
            hi3[ax] = ncs[ax] - 1;
            rel[ax] = 0;
        } else {
            lo3[ax] = -1;
            hi3[ax] = 1;
            rel[ax] = 1;
        }
    }
    const int cc[3] = {cx, cy, cz};
    // r_ij < r_list from the hi parts alone (minimum image with the FP32 box)
    // unless r^2 falls within that shortcut's error bound of r_list^2; there
    // the split-precision displacement decides (as in k_nbr_allpairs; the
    // image shift adds at most 2^-24 L per axis to the error)
    const float rl = sqrtf(a.rl2);
    const float l1_i = fabsf(hi_i.x) + fabsf(hi_i.y) + fabsf(hi_i.z) +
                       (box.periodic ? box.Lhi[0] + box.Lhi[1] + box.Lhi[2] : 0.f);
    auto within = [&](int j) -> bool {
        const float4 hj = a.hi[j];
        float dx = hj.x - hi_i.x, dy = hj.y - hi_i.y, dz = hj.z - hi_i.z;
        if (box.periodic) {
            dx -= rintf(dx * box.invL[0]) * box.Lhi[0];
            dy -= rintf(dy * box.invL[1]) * box.Lhi[1];
            dz -= rintf(dz * box.invL[2]) * box.Lhi[2];
        }
        const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float tau = 2.384185791015625e-7f * (l1_i + fabsf(hj.x) + fabsf(hj.y) + fabsf(hj.z));
        const float margin = fmaf(4.f * rl, tau, fmaf(2.f * tau, tau, 9.5367431640625e-7f * a.rl2));
        if (r2 < a.rl2 - margin) return true;
        if (r2 > a.rl2 + margin) return false;
        const float3 d = displacement(hi_i, lo_i, hj, a.lo[j], box);
        return d.x * d.x + d.y * d.y + d.z * d.z < a.rl2;
    };
    // The (at most 27) cells to visit, in (z, y, x) order: lane v takes visit
    // v and loads its cell's range, so all ranges take one memory round trip;
    // the non-empty ones are compacted (lane k < ne: the k-th, first candidate
    // position coff, first entry cbeg in cell_atoms). Candidates are then
    // taken 32 at a time in the same order as visiting the cells one by one
    // (cells in (z, y, x) order, atoms in index order within a cell).
    const int nv0 = hi3[0] - lo3[0] + 1, nv1 = hi3[1] - lo3[1] + 1, nv2 = hi3[2] - lo3[2] + 1;
    int beg = 0, len = 0;
    if (lane < nv0 * nv1 * nv2) {
        const int o[3] = {lo3[0] + lane % nv0, lo3[1] + (lane / nv0) % nv1, lo3[2] + lane / (nv0 * nv1)};
        int v[3];
        bool inside = true;
        for (int ax = 0; ax < 3; ++ax) {
            v[ax] = rel[ax] ? cc[ax] + o[ax] : o[ax];
            if (rel[ax]) {
                if (box.periodic) v[ax] = (v[ax] + ncs[ax]) % ncs[ax];
                else if (v[ax] < 0 || v[ax] >= ncs[ax]) inside = false;
            }
        }
        if (inside) {
            const int cell = (v[2] * nc1 + v[1]) * nc0 + v[0];
            beg = cell_start[cell];
            len = cell_start[cell + 1] - beg;
        }
    }
    const unsigned nonempty = __ballot_sync(0xffffffffu, len > 0);
    const int ne = __popc(nonempty);
    int total = len;   // inclusive prefix over the visits
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, total, o);
        if (lane >= o) total += t;
    }
    const int off = total - len;
    total = __shfl_sync(0xffffffffu, total, 31);
    // compact: lane k < ne gets the k-th non-empty visit's (off, beg)
    __shared__ int2 visit_sm[kNbrCellWarps][32];
    int2* vs = visit_sm[threadIdx.x >> 5];
    if (len > 0) vs[__popc(nonempty & lanemask_lt())] = make_int2(off, beg);
    __syncwarp();
    const int2 cv = lane < ne ? vs[lane] : make_int2(total, 0);
    const int coff = cv.x, cbeg = cv.y;
    for (int base = 0; base < total; base += 32) {
        // candidate q = base + lane: the non-empty visit holding it
        const unsigned before = __ballot_sync(0xffffffffu, lane < ne && coff < base);
        const unsigned starts = __reduce_or_sync(
            0xffffffffu, (lane < ne && coff >= base && coff < base + 32) ? (1u << (coff - base)) : 0u);
        const int b = max(0, __popc(before) - 1 + __popc(starts & lanemask_le()));
        const int off_b = __shfl_sync(0xffffffffu, coff, b), beg_b = __shfl_sync(0xffffffffu, cbeg, b);
        const int q = base + lane;
        bool ok = false;
        int j = -1;
        if (q < total) {
            j = cell_atoms[beg_b + (q - off_b)];
            ok = j != i && within(j);
        }
        unsigned mask = __ballot_sync(0xffffffffu, ok);
        int pos = count + __popc(mask & lanemask_lt());
        if (ok && pos < a.cap) row[pos] = j;
        count += __popc(mask);
    }
    if (lane == 0) {
        a.nbr_cnt[i] = count;
        if (count > a.cap) atomicMax(&ctr->nbr_overflow, count);
    }
}

}  // namespace

void launch_stage_system(cudaStream_t st, int n, const double* xyz, const int8_t* species, const double* Ld,
                         int periodic, int want_bbox, float4* hi, float4* lo, int* rank, Counters* ctr,
                         double* grad, const float4* ref, float half_skin2, int force_rebuild) {
    int bs = 256, gs = (n + bs - 1) / bs;
    MLP_LAUNCH("stage", st,
               k_stage_system<<<gs, bs, 0, st>>>(n, xyz, species, Ld[0], Ld[1], Ld[2], periodic, want_bbox, hi,
                                                 lo, rank, ctr, grad, ref, half_skin2, force_rebuild));
}

void launch_stage_batch(cudaStream_t st, int n_mols, int n_atoms, const int* mol_start, const double* xyz,
                        const int8_t* species, float4* hi, float4* lo, int* rank, Counters* ctr, double* grad) {
    MLP_LAUNCH("stage", st,
               k_stage_batch<<<n_mols, 128, 0, st>>>(n_mols, n_atoms, mol_start, xyz, species, hi, lo, rank, ctr,
                                                     grad));
}

void launch_nbr_allpairs(cudaStream_t st, int n, int n_mols, const int* mol_start, const NbrArgs& a, Counters* ctr) {
    int warps_per_block = 8;
    int gs = (n + warps_per_block - 1) / warps_per_block;
    MLP_LAUNCH("neighbors_allpairs", st,
               k_nbr_allpairs<<<gs, 32 * warps_per_block, 0, st>>>(n, n_mols, mol_start, a, ctr));
}

void launch_grid_setup(cudaStream_t st, Counters* ctr, Grid* g, float r_list, int max_cells) {
    MLP_LAUNCH("grid_setup", st, k_grid_setup<<<1, 1, 0, st>>>(ctr, g, r_list, max_cells));
}

void launch_cell_build(cudaStream_t st, int n, const float4* hi, const Grid* g, int max_cells, int* cell_of_atom,
                       int* cell_rank, int* cell_count, int* cell_start, int* cell_atoms, const Counters* ctr) {
    int bs = 256, gs = (n + bs - 1) / bs;
    MLP_LAUNCH("cell_count", st,
               k_cell_count<<<gs, bs, 0, st>>>(n, hi, g, cell_of_atom, cell_rank, cell_count, ctr));
    MLP_LAUNCH("cell_scan", st, k_cell_scan<<<1, 1024, 0, st>>>(g, cell_count, cell_start, ctr));
    MLP_LAUNCH("cell_scatter", st,
               k_cell_scatter<<<gs, bs, 0, st>>>(n, cell_of_atom, cell_rank, cell_start, cell_atoms, ctr));
    // a warp per cell, at most 16 blocks of 8 warps per SM (cells are taken grid-stride)
    const int sort_blocks = (int)std::min<long long>(((long long)max_cells * 32 + 255) / 256, 148LL * 16);
    MLP_LAUNCH("cell_sort", st, k_cell_sort<<<sort_blocks, 256, 0, st>>>(g, cell_start, cell_atoms, ctr));
}

void launch_nbr_cell(cudaStream_t st, int n, const NbrArgs& a, const Box& box, const Grid* g,
                     const int* cell_of_atom, const int* cell_start, const int* cell_atoms, Counters* ctr,
                     float4* ref) {
    int gs = (n + kNbrCellWarps - 1) / kNbrCellWarps;
    MLP_LAUNCH("neighbors_cell", st,
               k_nbr_cell<<<gs, 32 * kNbrCellWarps, 0, st>>>(n, a, box, g, cell_of_atom, cell_start, cell_atoms,
                                                             ctr, ref));
}

}  // namespace mlp
