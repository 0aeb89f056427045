// Final reductions: per-molecule energy E_m = sum_i e_i in FP64 (one block
// per molecule, fixed reduction tree -> identical result for a molecule
// evaluated alone or inside any batch), and the FP32 force output
// F = sign * scale * dE/dr from the FP64 per-atom accumulators.
#include "common.cuh"
#include "kernels.cuh"

namespace mlp {
namespace {

constexpr int kEBlock = 128;

// Blocks [0, n_mols) reduce energies; the remaining blocks convert forces.
// mol_start == nullptr means one molecule made of all n_atoms atoms.
__global__ void k_finalize(int n_mols, const int* __restrict__ mol_start, int n_atoms, const float* __restrict__ e,
                           const double* __restrict__ grad, double* __restrict__ E, float* __restrict__ F,
                           const double* __restrict__ grad_scale, float sign, const Counters* __restrict__ ctr,
                           int* __restrict__ sticky, const int* __restrict__ F_index, long long n_full,
                           int accumulate, int e_nets, int e_stride) {
    if (blockIdx.x == 0 && threadIdx.x == 0 && sticky) {
        // error flags of this evaluation, kept until the host reads and clears them
        const int f = (ctr->nbr_overflow ? 1 : 0) | (ctr->ang_overflow ? 2 : 0) | (ctr->bad_species ? 4 : 0) |
                      (ctr->net_error ? 8 : 0);
        if (f) atomicOr(sticky, f);
    }
    if ((int)blockIdx.x < n_mols) {
        const int m = blockIdx.x;
        const int a = mol_start ? mol_start[m] : 0;
        const int b = mol_start ? mol_start[m + 1] : n_atoms;
        double acc = 0.0;
        if (e_nets == 1) {
            for (int i = a + threadIdx.x; i < b; i += kEBlock) acc += (double)e[i];
        } else {   // ensemble: atom energy = mean over the nets (fixed order)
            const double inv = 1.0 / (double)e_nets;
            for (int i = a + threadIdx.x; i < b; i += kEBlock) {
                double ei = 0.0;
                for (int k = 0; k < e_nets; ++k) ei += (double)e[(size_t)k * e_stride + i];
                acc += ei * inv;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        __shared__ double ws[kEBlock / 32];
        if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
        __syncthreads();
        if (threadIdx.x == 0) {
            double t = 0.0;
            for (int q = 0; q < kEBlock / 32; ++q) t += ws[q];
            if (E) E[m] = t;
        }
        return;
    }
    const double scale = (grad_scale ? *grad_scale : 1.0) * (double)sign;
    if (!F) return;
    const int fb = blockIdx.x - n_mols;
    const int nfb = gridDim.x - n_mols;
    if (!F_index) {
        for (int q = fb * kEBlock + threadIdx.x; q < 3 * n_atoms; q += nfb * kEBlock) F[q] = (float)(scale * grad[q]);
        return;
    }
    // ML/MM region: into the full system's force rows
    for (int q = fb * kEBlock + threadIdx.x; q < 3 * n_atoms; q += nfb * kEBlock) {
        const int i = q / 3, c = q - 3 * i;
        const int row = F_index[i];
        if (row < 0 || (long long)row >= n_full) continue;
        float* dst = F + 3 * (size_t)row + c;
        const float v = (float)(scale * grad[q]);
        *dst = accumulate ? *dst + v : v;
    }
}

__global__ void k_gather_subset(int n, const int* __restrict__ index, const double* __restrict__ full,
                                long long n_full, double* __restrict__ xyz, Counters* __restrict__ ctr) {
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= 3 * n) return;
    const int i = q / 3, c = q - 3 * i;
    const int row = index[i];
    if (row < 0 || (long long)row >= n_full) {
        if (c == 0) atomicOr(&ctr->bad_species, 4);
        xyz[q] = 0.0;
        return;
    }
    xyz[q] = full[3 * (size_t)row + c];
}

// One block per molecule: contiguous copies between the molecule's host
// block (read / written through its unified address) and the batch arrays.
__global__ void k_gather_batch(const MolRef* __restrict__ refs, const int* __restrict__ mol_start,
                               double* __restrict__ xyz, int8_t* __restrict__ species) {
    // The request's arrays start on 16 bytes (host blocks): read over PCIe in
    // 16-byte (coordinates) and 4-byte (elements) words, fewer transactions.
    const int m = blockIdx.x;
    const MolRef r = refs[m];
    const int a = mol_start[m], n = mol_start[m + 1] - a;
    double* dst = xyz + 3 * (size_t)a;
    const double2* src2 = reinterpret_cast<const double2*>(r.xyz);
    const int n3 = 3 * n;
    for (int q = threadIdx.x; q < n3 / 2; q += blockDim.x) {
        const double2 v = src2[q];
        dst[2 * q] = v.x;
        dst[2 * q + 1] = v.y;
    }
    if ((n3 & 1) && threadIdx.x == 0) dst[n3 - 1] = r.xyz[n3 - 1];
    const uint32_t* s4 = reinterpret_cast<const uint32_t*>(r.species);
    for (int q = threadIdx.x; q < n / 4; q += blockDim.x) {
        const uint32_t w = s4[q];
#pragma unroll
        for (int b = 0; b < 4; ++b) species[a + 4 * q + b] = (int8_t)(w >> (8 * b));
    }
    for (int q = 4 * (n / 4) + threadIdx.x; q < n; q += blockDim.x) species[a + q] = r.species[q];
}

__global__ void k_scatter_results(const MolRef* __restrict__ refs, const int* __restrict__ mol_start,
                                  const double* __restrict__ E, const float* __restrict__ F) {
    // written to the request's host block (16-byte aligned) in 16-byte words
    const int m = blockIdx.x;
    const MolRef r = refs[m];
    const int a = mol_start[m], n = mol_start[m + 1] - a;
    const float* src = F + 3 * (size_t)a;
    float4* dst4 = reinterpret_cast<float4*>(r.F);
    const int n3 = 3 * n;
    for (int q = threadIdx.x; q < n3 / 4; q += blockDim.x)
        dst4[q] = make_float4(src[4 * q], src[4 * q + 1], src[4 * q + 2], src[4 * q + 3]);
    for (int q = 4 * (n3 / 4) + threadIdx.x; q < n3; q += blockDim.x) r.F[q] = src[q];
    if (threadIdx.x == 0) *r.E = E[m];
}

}  // namespace

void launch_gather_batch(cudaStream_t st, int n_mols, const MolRef* refs, const int* mol_start, double* d_xyz,
                         int8_t* d_species) {
    if (n_mols <= 0) return;
    MLP_LAUNCH("gather", st, k_gather_batch<<<n_mols, 128, 0, st>>>(refs, mol_start, d_xyz, d_species));
}

void launch_scatter_results(cudaStream_t st, int n_mols, const MolRef* refs, const int* mol_start, const double* d_E,
                            const float* d_F) {
    if (n_mols <= 0) return;
    MLP_LAUNCH("scatter", st, k_scatter_results<<<n_mols, 128, 0, st>>>(refs, mol_start, d_E, d_F));
}

void launch_gather_subset(cudaStream_t st, int n, const int* index, const double* coords_full, long long n_full,
                          double* xyz, Counters* ctr) {
    if (n <= 0) return;
    MLP_LAUNCH("gather_subset", st,
               k_gather_subset<<<(3 * n + 255) / 256, 256, 0, st>>>(n, index, coords_full, n_full, xyz, ctr));
}

void launch_finalize(cudaStream_t st, int n_mols, const int* mol_start, int n_atoms, const float* e,
                     const double* grad, double* E, float* F, const double* grad_scale, float sign,
                     const Counters* ctr, int* sticky, const int* F_index, long long n_full, bool accumulate,
                     int e_nets, int e_stride) {
    const int fblocks = F ? (3 * n_atoms + kEBlock * 4 - 1) / (kEBlock * 4) : 0;
    const int eblocks = E ? n_mols : 0;
    const int blocks = eblocks + fblocks > 0 ? eblocks + fblocks : 1;
    MLP_LAUNCH("finalize", st,
               k_finalize<<<blocks, kEBlock, 0, st>>>(eblocks, mol_start, n_atoms, e, grad, E, F, grad_scale, sign,
                                                      ctr, sticky, F_index, n_full, accumulate ? 1 : 0, e_nets,
                                                      e_stride));
}

}  // namespace mlp
