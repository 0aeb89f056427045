// Per-element networks in FP32 on the CUDA cores (the FP32 path).
//
// Each layer is one element-grouped GEMM C[rows, N] = A[rows, K] W^T with
// the weights of the element that owns the 128-row tile (rows are grouped by
// element and padded to whole tiles), plus a fused epilogue:
//   forward   z1 = G W1^T + b1, h1 = celu(z1); z2, h2 likewise;
//             z3 = h2 W3^T + b3 -> h3 = celu(z3), g3 = w4 * celu'(z3);
//             e = w4 . h3 + b4 (separate row reduction, fixed order)
//   backward  g2 = (g3 W3) * celu'(z2); g1 = (g2 W2) * celu'(z1); dE/dG = g1 W1
// (paper, section "PyTorch Model Support": forces by backpropagation).
// An ensemble of K nets (section "Performance of MLPs") runs these launches
// once per net; e and dE/dG take each net's output scaled by 1 / K, written
// by net 0 and added by the others in net order, which leaves the means.
// SIMT tiling: 128 x 64 output tile per block of 256 threads, 8 x 4 outputs
// per thread, K in steps of 16 through double-buffered shared memory.
#include "common.cuh"
#include "kernels.cuh"

namespace mlp {
namespace {

enum { EPI_BIAS_CELU = 0, EPI_G3 = 1, EPI_DSIG = 2, EPI_PLAIN = 3 };

constexpr int BM = 128, BN = 64, BK = 16;

template <int EPI>
__global__ void __launch_bounds__(256) k_gemm(const Counters* __restrict__ ctr, const float* __restrict__ A, int lda,
                                              const float* __restrict__ B, int ldb, size_t b_elem_stride, int N,
                                              int K, const float* __restrict__ bias, const float* __restrict__ aux,
                                              int ldaux, float* __restrict__ C0, float* __restrict__ C1, int ldc,
                                              float oscale, int oacc) {
    int s, row0, nvalid;
    if (!tile_info(ctr->species, blockIdx.y, s, row0, nvalid)) return;
    const int n0 = blockIdx.x * BN;
    const float* Bs_g = B + (size_t)s * b_elem_stride;

    __shared__ __align__(16) float As[2][BK][BM + 4];
    __shared__ __align__(16) float Bsh[2][BK][BN + 4];

    const int tid = threadIdx.x;
    const int tx = tid & 15, ty = tid >> 4;
    // loaders
    const int a_row = tid >> 2, a_kq = (tid & 3) * 4;   // rows a_row and a_row + 64
    const int b_row = tid >> 2, b_kq = (tid & 3) * 4;   // n = n0 + b_row
    const float* Arow0 = A + (size_t)(row0 + a_row) * lda;
    const float* Arow1 = A + (size_t)(row0 + a_row + 64) * lda;
    const bool b_ok = n0 + b_row < N;
    const float* Brow = Bs_g + (size_t)(n0 + b_row) * ldb;

    float acc[8][4];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;

    float4 ra0 = *reinterpret_cast<const float4*>(Arow0 + a_kq);
    float4 ra1 = *reinterpret_cast<const float4*>(Arow1 + a_kq);
    float4 rb = b_ok ? *reinterpret_cast<const float4*>(Brow + b_kq) : make_float4(0.f, 0.f, 0.f, 0.f);
    const int nk = K / BK;
    for (int kt = 0; kt < nk; ++kt) {
        const int buf = kt & 1;
        As[buf][a_kq + 0][a_row] = ra0.x;
        As[buf][a_kq + 1][a_row] = ra0.y;
        As[buf][a_kq + 2][a_row] = ra0.z;
        As[buf][a_kq + 3][a_row] = ra0.w;
        As[buf][a_kq + 0][a_row + 64] = ra1.x;
        As[buf][a_kq + 1][a_row + 64] = ra1.y;
        As[buf][a_kq + 2][a_row + 64] = ra1.z;
        As[buf][a_kq + 3][a_row + 64] = ra1.w;
        Bsh[buf][b_kq + 0][b_row] = rb.x;
        Bsh[buf][b_kq + 1][b_row] = rb.y;
        Bsh[buf][b_kq + 2][b_row] = rb.z;
        Bsh[buf][b_kq + 3][b_row] = rb.w;
        __syncthreads();
        if (kt + 1 < nk) {
            const int ko = (kt + 1) * BK;
            ra0 = *reinterpret_cast<const float4*>(Arow0 + ko + a_kq);
            ra1 = *reinterpret_cast<const float4*>(Arow1 + ko + a_kq);
            rb = b_ok ? *reinterpret_cast<const float4*>(Brow + ko + b_kq) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
#pragma unroll
        for (int kk = 0; kk < BK; ++kk) {
            const float4 a0 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8]);
            const float4 a1 = *reinterpret_cast<const float4*>(&As[buf][kk][ty * 8 + 4]);
            const float4 b = *reinterpret_cast<const float4*>(&Bsh[buf][kk][tx * 4]);
            const float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
            const float bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
            for (int i = 0; i < 8; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
        }
        // the next iteration writes the other buffer; the one read here is
        // rewritten two iterations later, after the barrier above
    }

#pragma unroll
    for (int i = 0; i < 8; ++i) {
        const int r = ty * 8 + i;
        if (r >= nvalid) continue;
        const size_t row = (size_t)(row0 + r);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tx * 4 + j;
            if (n >= N) continue;
            const float v = acc[i][j];
            if (EPI == EPI_BIAS_CELU) {
                const float z = v + bias[s * N + n];
                C0[row * ldc + n] = z;
                C1[row * ldc + n] = celu(z);
            } else if (EPI == EPI_G3) {
                const float z = v + bias[s * N + n];
                C0[row * ldc + n] = celu(z);
                C1[row * ldc + n] = aux[s * N + n] * celu_deriv(z);
            } else if (EPI == EPI_DSIG) {
                C0[row * ldc + n] = v * celu_deriv(aux[row * ldaux + n]);
            } else {   // plain output: net 0 of K writes v / K, the others add theirs
                const float o = v * oscale;
                C0[row * ldc + n] = oacc ? C0[row * ldc + n] + o : o;
            }
        }
    }
}

// e[atom] = w4 . h3 + b4 for every valid row (one warp per row, fixed order).
__global__ void k_energy_rows(const Counters* __restrict__ ctr, const float* __restrict__ H3,
                              const float* __restrict__ W4, const float* __restrict__ b4,
                              const int* __restrict__ row_atom, float* __restrict__ e, float oscale, int oacc) {
    int s, row0, nvalid;
    if (!tile_info(ctr->species, blockIdx.x, s, row0, nvalid)) return;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    for (int r = w; r < nvalid; r += 8) {
        const float* h = H3 + (size_t)(row0 + r) * kH3;
        float acc = 0.f;
        for (int c = lane; c < kH3; c += 32) acc = fmaf(W4[s * kH3 + c], h[c], acc);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) {
            const int a = row_atom[row0 + r];
            const float o = (acc + b4[s]) * oscale;
            e[a] = oacc ? e[a] + o : o;
        }
    }
}

}  // namespace

void launch_mlp_f32(cudaStream_t st, int rows_cap, const Counters* ctr, const NetF32& w, const float* G,
                    const int* row_atom, MlpF32Bufs& b, float* e, float* dG, bool backward, int net, int nets) {
    const int tiles = rows_cap / kTileRows;
    const float osc = nets > 1 ? 1.f / (float)nets : 1.f;
    const int oacc = net > 0 ? 1 : 0;
    auto grid = [&](int N) { return dim3((N + BN - 1) / BN, tiles); };
    MLP_LAUNCH("mlp_f32_l1", st,
               k_gemm<EPI_BIAS_CELU><<<grid(kH1), 256, 0, st>>>(ctr, G, kAevLd, w.W1, kAevLen, (size_t)kH1 * kAevLen,
                                                                kH1, kAevLen, w.b1, nullptr, 0, b.Z1, b.H1, kH1, 1.f, 0));
    MLP_LAUNCH("mlp_f32_l2", st,
               k_gemm<EPI_BIAS_CELU><<<grid(kH2), 256, 0, st>>>(ctr, b.H1, kH1, w.W2, kH1, (size_t)kH2 * kH1, kH2,
                                                                kH1, w.b2, nullptr, 0, b.Z2, b.H2, kH2, 1.f, 0));
    MLP_LAUNCH("mlp_f32_l3", st,
               k_gemm<EPI_G3><<<grid(kH3), 256, 0, st>>>(ctr, b.H2, kH2, w.W3, kH2, (size_t)kH3 * kH2, kH3, kH2,
                                                         w.b3, w.W4, 0, b.H3, b.G3, kH3, 1.f, 0));
    MLP_LAUNCH("mlp_f32_energy", st, k_energy_rows<<<tiles, 256, 0, st>>>(ctr, b.H3, w.W4, w.b4, row_atom, e, osc, oacc));
    if (!backward) return;
    MLP_LAUNCH("mlp_f32_b3", st,
               k_gemm<EPI_DSIG><<<grid(kH2), 256, 0, st>>>(ctr, b.G3, kH3, w.W3t, kH3, (size_t)kH2 * kH3, kH2, kH3,
                                                           nullptr, b.Z2, kH2, b.G2, nullptr, kH2, 1.f, 0));
    MLP_LAUNCH("mlp_f32_b2", st,
               k_gemm<EPI_DSIG><<<grid(kH1), 256, 0, st>>>(ctr, b.G2, kH2, w.W2t, kH2, (size_t)kH1 * kH2, kH1, kH2,
                                                           nullptr, b.Z1, kH1, b.G1, nullptr, kH1, 1.f, 0));
    MLP_LAUNCH("mlp_f32_b1", st,
               k_gemm<EPI_PLAIN><<<grid(kAevLen), 256, 0, st>>>(ctr, b.G1, kH1, w.W1t, kH1, (size_t)kAevLen * kH1,
                                                                kAevLen, kH1, nullptr, nullptr, 0, dG, nullptr,
                                                                kAevLd, osc, oacc));
}

}  // namespace mlp
