// Kernel launchers of the CUDA path (one evaluation = the launches below on
// one stream). Every launcher goes through MLP_LAUNCH, which counts launches
// and, when profiling is on, brackets them with CUDA events on that stream.
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"

namespace mlp {

// ---- launch accounting / per-kernel event timing (runtime.cu)
void launch_begin(const char* name, cudaStream_t st);
void launch_end(const char* name, cudaStream_t st);
void init_constants_for_current_device();

// One-time setup per (device, key) -- kernel attributes, constant tables --
// safe to call from several host threads: the setup runs under a lock, once
// for each device it is called on.
std::mutex& once_mutex();
bool once_first(int device, const void* key);   // caller holds once_mutex(); records the pair
template <typename F>
void once_per_device(const void* key, F&& setup) {
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> lk(once_mutex());
    if (once_first(dev, key)) setup();
}
// Streaming multiprocessors of the current device (queried once per device).
int sm_count();

#define MLP_LAUNCH(name, st, ...)            \
    do {                                     \
        ::mlp::launch_begin(name, st);       \
        __VA_ARGS__;                         \
        ::mlp::launch_end(name, st);         \
    } while (0)

// ---- staging and neighbor search (kernels_nbr.cu)
struct NbrArgs {
    const float4* hi;
    const float4* lo;
    int* nbr;        // [n][cap]
    int* nbr_cnt;    // [n]
    int cap;
    float rl2;       // list radius squared
};

void launch_stage_system(cudaStream_t st, int n, const double* xyz, const int8_t* species, const double* Ld,
                         int periodic, int want_bbox, float4* hi, float4* lo, int* rank, Counters* ctr,
                         double* grad, const float4* ref, float half_skin2, int force_rebuild);
void launch_stage_batch(cudaStream_t st, int n_mols, int n_atoms, const int* mol_start, const double* xyz,
                        const int8_t* species, float4* hi, float4* lo, int* rank, Counters* ctr, double* grad);
void launch_nbr_allpairs(cudaStream_t st, int n, int n_mols, const int* mol_start, const NbrArgs& a, Counters* ctr);
void launch_grid_setup(cudaStream_t st, Counters* ctr, Grid* g, float r_list, int max_cells);
void launch_cell_build(cudaStream_t st, int n, const float4* hi, const Grid* g, int max_cells, int* cell_of_atom,
                       int* cell_rank, int* cell_count, int* cell_start, int* cell_atoms, const Counters* ctr);
void launch_nbr_cell(cudaStream_t st, int n, const NbrArgs& a, const Box& box, const Grid* g,
                     const int* cell_of_atom, const int* cell_start, const int* cell_atoms, Counters* ctr,
                     float4* ref);

// ---- AEV forward and AEV backward -> forces (kernels_aev.cu)
struct AevArgs {
    int n;
    const float4* hi;
    const float4* lo;
    const int* nbr;
    const int* nbr_cnt;
    int cap;
    Box box;
    Counters* ctr;
    const int* rank;
    // atoms with more than kAngCap angular neighbors: listed by the AEV's main
    // launch (big_list[0 .. ctr->ang_big), big_flag[i] = 1) and done by its
    // second launch; the force kernels read the same list and flags
    int* big_list;
    unsigned char* big_flag;
};
void launch_aev_f32(cudaStream_t st, const AevArgs& a, float* G, int* row_atom, bool fast);
void launch_aev_bf16(cudaStream_t st, const AevArgs& a, __nv_bfloat16* G, __nv_bfloat16* G_lo, int* row_atom,
                     bool fast);
// dE/dG rows as FP32 (dG) or BF16 (dG16): exactly one of them non-null.
void launch_forces(cudaStream_t st, const AevArgs& a, const float* dG, const __nv_bfloat16* dG16, double* grad,
                   bool fast);

// ---- network, FP32 SIMT path (kernels_mlp_f32.cu)
struct NetF32 {   // device pointers, element-major, one net
    const float *W1, *b1, *W2, *b2, *W3, *b3, *W4, *b4;
    const float *W1t, *W2t, *W3t;   // transposes: [7][1008][256], [7][256][192], [7][192][160]
};
struct MlpF32Bufs {
    float *Z1, *H1, *Z2, *H2, *H3, *G3, *G2, *G1;   // [rows][256|192|160]
};
// Net `net` of an ensemble of `nets`: writes e and dE/dG scaled by 1 / nets
// when net == 0 and adds them (scaled) otherwise, so that after nets
// launches e and dE/dG hold the ensemble means.
void launch_mlp_f32(cudaStream_t st, int rows_cap, const Counters* ctr, const NetF32& w, const float* G,
                    const int* row_atom, MlpF32Bufs& b, float* e, float* dG, bool backward, int net = 0,
                    int nets = 1);

// ---- network, BF16 tcgen05 path (kernels_mlp_tc.cu)
// All nets of the ensemble: every array holds the nets back to back, so
// that block k * 7 + s of a matrix (or bias vector) is net k, element s.
struct NetBF16 {
    int n_nets;
    const __nv_bfloat16 *W1, *W2, *W3;       // [K][7][256][1024], [K][7][192][256], [K][7][160][192]
    const __nv_bfloat16 *W1lo, *W2lo, *W3lo; // BF16 remainders W - W_hi of the forward weights
    const __nv_bfloat16 *W1t, *W2t, *W3t;    // [K][7][1024][256], [K][7][256][192], [K][7][192][160]
    const float *b1, *b2, *b3, *W4, *b4;     // FP32 [K][7][...]
    // TMA descriptors of the weight matrices (built once per weight set)
    CUtensorMap tmW1, tmW2, tmW3, tmW1lo, tmW2lo, tmW3lo, tmW1t, tmW2t, tmW3t;
    bool maps_ok;
};
bool mlp_tc_available();
// Runs the network kernels' bounded barrier wait on a phase that never
// completes; returns a CUDA error code (0 on success).
int debug_wait_timeout(int* timed_out, int* code);
bool make_weight_maps(NetBF16& w);
// split = true: forward GEMMs from hi/lo BF16 pairs of both operands (G_lo
// required); false: single BF16 pass everywhere. Per-atom energies go to e
// and dE/dG to dG (BF16). An ensemble (w.n_nets = K > 1) writes net k's
// energies to e + k * e_stride (the finalize kernel averages them) and the
// mean dE/dG to dG; with backward it also needs g1, BF16 [rows_cap][K * 256]
// scratch for every net's last hidden-layer gradient (two launches: the
// network kernel over all (tile, net) pairs, then the mean dE/dG GEMM).
bool launch_mlp_bf16(cudaStream_t st, int rows_cap, const Counters* ctr, const NetBF16& w,
                     const __nv_bfloat16* G, const __nv_bfloat16* G_lo, bool split, const int* row_atom, float* e,
                     int e_stride, __nv_bfloat16* dG, __nv_bfloat16* g1, bool backward, int* err_flag);

// ---- serving batches (kernels_misc.cu): one molecule per request, its inputs
// and result area in page-locked host memory that kernels address directly
// (unified addressing), so that no host thread copies request data. Every
// array starts on a 16-byte boundary.
struct MolRef {
    const double* xyz;     // [n][3]
    const int8_t* species; // [n]
    float* F;              // [n][3] result
    double* E;             // result
};
// Gathers the molecules' inputs into d_xyz / d_species at mol_start offsets.
void launch_gather_batch(cudaStream_t st, int n_mols, const MolRef* refs, const int* mol_start, double* d_xyz,
                         int8_t* d_species);
// Scatters energies and forces back into the molecules' result areas.
void launch_scatter_results(cudaStream_t st, int n_mols, const MolRef* refs, const int* mol_start, const double* d_E,
                            const float* d_F);

// ---- ML/MM region (kernels_misc.cu): xyz[q] = coords_full[index[q]]; an
// index outside [0, n_full) sets bad-input flag 4 and its row is zero.
void launch_gather_subset(cudaStream_t st, int n, const int* index, const double* coords_full, long long n_full,
                          double* xyz, Counters* ctr);

// ---- finalize (kernels_misc.cu)
// Also ORs this evaluation's error flags (1 neighbor overflow, 2 AEV staging
// overflow, 4 bad input, 8 network kernel error) into *sticky when
// sticky != nullptr. With F_index, force row i goes to row F_index[i] of F
// (n_full rows; rows outside [0, n_full) skipped), added to it when
// accumulate is set. e_nets > 1: e holds e_nets rows of e_stride per-atom
// energies (one per net of an ensemble), averaged per atom in FP64.
void launch_finalize(cudaStream_t st, int n_mols, const int* mol_start, int n_atoms, const float* e,
                     const double* grad, double* E, float* F, const double* grad_scale, float sign,
                     const Counters* ctr, int* sticky, const int* F_index = nullptr, long long n_full = 0,
                     bool accumulate = false, int e_nets = 1, int e_stride = 0);

}  // namespace mlp
