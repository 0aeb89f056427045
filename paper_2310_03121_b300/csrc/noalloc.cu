// Neighbor list of one system built without allocating any memory.
//
// Who needs this: callers that cannot call cudaMalloc once they are running —
// for example an MD engine or plugin that receives a fixed memory plan from
// its host and must not grow its footprint afterwards, a host framework that
// owns every device allocation through its own pool and forbids others, or a
// time-critical loop that cannot afford the latency or the possible failure
// of an allocation in the middle of a trajectory. mlp_neighbors_static gives
// them the cell-list neighbor search of this library with all of its working
// memory (split positions, cell counts, cell lists, counters) in one
// file-scope __device__ array of fixed size, reserved when the library is
// loaded and held by every GPU that loads it until the process exits.
//
// Limits: at most kStaticMaxAtoms atoms (more are rejected with MLP_EINVAL
// before any work is enqueued) and kStaticMaxCells cells (a box or an open
// system that would need more gets fewer, wider cells).
//
// The array is shared by every call in the process: each call clears the
// parts that must start at zero (counters and cell counts) on its stream
// before using it. Calls whose work overlaps on the GPU (different streams,
// or different host threads) race on the array and must be ordered by the
// caller.
//
// The kernels are the library's own cell-list kernels (binning, scan,
// scatter, in-cell sort, warp-per-atom search), fed from the static array.
#include <cmath>
#include <mutex>

#include "../../include/mlp.h"
#include "engine.cuh"
#include "kernels.cuh"

namespace mlp {
namespace {

constexpr int kStaticMaxAtoms = 32768;
constexpr int kStaticMaxCells = 32768;

constexpr size_t al256(size_t b) { return (b + 255) / 256 * 256; }

// byte offsets inside the array
constexpr size_t kOffCtr = 0;
constexpr size_t kOffCellCount = kOffCtr + al256(sizeof(Counters));
constexpr size_t kZeroBytes = kOffCellCount + al256(sizeof(int) * (size_t)kStaticMaxCells);   // cleared per call
constexpr size_t kOffGrid = kZeroBytes;
constexpr size_t kOffHi = kOffGrid + al256(sizeof(Grid));
constexpr size_t kOffLo = kOffHi + al256(sizeof(float4) * (size_t)kStaticMaxAtoms);
constexpr size_t kOffRef = kOffLo + al256(sizeof(float4) * (size_t)kStaticMaxAtoms);
constexpr size_t kOffCellOf = kOffRef + al256(sizeof(float4) * (size_t)kStaticMaxAtoms);
constexpr size_t kOffCellRank = kOffCellOf + al256(sizeof(int) * (size_t)kStaticMaxAtoms);
constexpr size_t kOffCellStart = kOffCellRank + al256(sizeof(int) * (size_t)kStaticMaxAtoms);
constexpr size_t kOffCellAtoms = kOffCellStart + al256(sizeof(int) * ((size_t)kStaticMaxCells + 1));
constexpr size_t kStaticBytes = kOffCellAtoms + al256(sizeof(int) * (size_t)kStaticMaxAtoms);   // ~2.2 MB

static __device__ __align__(256) unsigned char g_nbr_scratch[kStaticBytes];

// Device address of g_nbr_scratch per device, resolved once per device with
// that device current (in host code the symbol names a host-side stand-in,
// not device memory, so it is never passed to a kernel directly).
std::mutex g_scratch_mu;
void* g_scratch_addr[64] = {nullptr};

int scratch_address(unsigned char** out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= 64) return set_error(MLP_EINVAL, "device index %d out of range", dev);
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_nbr_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(static neighbor scratch)");
        g_scratch_addr[dev] = p;
    }
    *out = static_cast<unsigned char*>(g_scratch_addr[dev]);
    return MLP_OK;
}

__device__ __forceinline__ unsigned bbox_key(float f) {
    int i = __float_as_int(f);
    i = i >= 0 ? i : i ^ 0x7fffffff;
    return (unsigned)i ^ 0x80000000u;
}

// Split FP64 positions into FP32 hi/lo (wrapped into [0, L) in periodic
// boxes), bounding box of open systems, grid and rebuild flag.
__global__ void k_static_stage(int n, const double* __restrict__ xyz, int periodic, double L0, double L1, double L2,
                               Grid grid, unsigned char* __restrict__ scratch) {
    Counters* ctr = reinterpret_cast<Counters*>(scratch + kOffCtr);
    float4* hi = reinterpret_cast<float4*>(scratch + kOffHi);
    float4* lo = reinterpret_cast<float4*>(scratch + kOffLo);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) {
        ctr->rebuild = 1;
        if (periodic) *reinterpret_cast<Grid*>(scratch + kOffGrid) = grid;
    }
    const bool valid = i < n;
    float h[3] = {0.f, 0.f, 0.f};
    if (valid) {
        const double L[3] = {L0, L1, L2};
        float l[3];
        for (int a = 0; a < 3; ++a) {
            double x = xyz[3 * (size_t)i + a];
            if (periodic) x -= L[a] * floor(x / L[a]);
            h[a] = (float)x;
            l[a] = (float)(x - (double)h[a]);
        }
        hi[i] = make_float4(h[0], h[1], h[2], __int_as_float(0));
        lo[i] = make_float4(l[0], l[1], l[2], __int_as_float(0));
    }
    if (!periodic) {
        float mn[3], mx[3];
        for (int a = 0; a < 3; ++a) {
            mn[a] = valid ? h[a] : 3.0e38f;
            mx[a] = valid ? h[a] : -3.0e38f;
            for (int o = 16; o > 0; o >>= 1) {
                mn[a] = fminf(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
                mx[a] = fmaxf(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
            }
        }
        if ((threadIdx.x & 31) == 0)
            for (int a = 0; a < 3; ++a) {
                atomicMax(&ctr->bbox_negmin_key[a], bbox_key(-mn[a]));
                atomicMax(&ctr->bbox_max_key[a], bbox_key(mx[a]));
            }
    }
}

}  // namespace
}  // namespace mlp

using namespace mlp;

extern "C" int mlp_neighbors_static(const double* d_coords, int32_t n, const double* cell, double cutoff,
                                    int32_t* d_counts, int32_t* d_list, int32_t cap, void* stream) {
    clear_error();
    if (!d_coords || !d_counts || !d_list) return set_error(MLP_EINVAL, "NULL argument");
    if (n <= 0 || n > kStaticMaxAtoms)
        return set_error(MLP_EINVAL, "n = %d outside [1, %d], the size of the static neighbor array", n,
                         kStaticMaxAtoms);
    if (cap <= 0 || cap > 4096) return set_error(MLP_EINVAL, "cap = %d outside [1, 4096]", cap);
    if (!(cutoff > 0.0) || cutoff > 20.0) return set_error(MLP_EINVAL, "cutoff %g outside (0, 20] A", cutoff);
    double L[3] = {1.0, 1.0, 1.0};
    Grid g{};
    const int periodic = cell ? 1 : 0;
    if (periodic) {
        for (int a = 0; a < 3; ++a) {
            if (!std::isfinite(cell[a]) || !(cell[a] >= 2.0 * cutoff))
                return set_error(MLP_EINVAL, "box length %g below 2 x cutoff", cell[a]);
            L[a] = cell[a];
        }
        // a box that would need more cells than the array holds gets fewer,
        // wider cells (still exact)
        g = make_periodic_grid(L, (float)cutoff, kStaticMaxCells);
        if (g.ncell < 1 || g.ncell > kStaticMaxCells)
            return set_error(MLP_EINVAL, "box needs %d cells; the static array holds %d", g.ncell, kStaticMaxCells);
    }
    unsigned char* scratch = nullptr;
    int rc = scratch_address(&scratch);
    if (rc) return rc;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    Counters* ctr = reinterpret_cast<Counters*>(scratch + kOffCtr);
    Grid* grid = reinterpret_cast<Grid*>(scratch + kOffGrid);
    float4* hi = reinterpret_cast<float4*>(scratch + kOffHi);
    float4* lo = reinterpret_cast<float4*>(scratch + kOffLo);
    float4* ref = reinterpret_cast<float4*>(scratch + kOffRef);
    int* cell_of = reinterpret_cast<int*>(scratch + kOffCellOf);
    int* cell_rank = reinterpret_cast<int*>(scratch + kOffCellRank);
    int* cell_count = reinterpret_cast<int*>(scratch + kOffCellCount);
    int* cell_start = reinterpret_cast<int*>(scratch + kOffCellStart);
    int* cell_atoms = reinterpret_cast<int*>(scratch + kOffCellAtoms);

    // counters and cell counts start at zero on every call
    cudaError_t e = cudaMemsetAsync(scratch, 0, kZeroBytes, st);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(static neighbor scratch)");
    const int bs = 256;
    MLP_LAUNCH("static_stage", st,
               k_static_stage<<<(n + bs - 1) / bs, bs, 0, st>>>(n, d_coords, periodic, L[0], L[1], L[2], g,
                                                                scratch));
    if (!periodic) launch_grid_setup(st, ctr, grid, (float)cutoff, kStaticMaxCells);
    launch_cell_build(st, n, hi, grid, kStaticMaxCells, cell_of, cell_rank, cell_count, cell_start, cell_atoms, ctr);
    NbrArgs na{hi, lo, d_list, d_counts, cap, (float)(cutoff * cutoff)};
    launch_nbr_cell(st, n, na, make_box(periodic, L), grid, cell_of, cell_start, cell_atoms, ctr, ref);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "mlp_neighbors_static launch");
    return MLP_OK;
}
