// Host runtime: device weights, per-evaluation workspaces and the ordered
// list of launches that makes one energy+force evaluation.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

namespace mlp {

// ---- errors (runtime.cu); codes are the MLP_* values of the public header
int set_error(int code, const char* fmt, ...);
int cuda_error(cudaError_t e, const char* where);
const char* last_error();
void clear_error();

// ---- device memory (runtime.cu): every device buffer goes through here
typedef void* (*AllocFn)(size_t bytes, void* ctx);
typedef void (*FreeFn)(void* p, void* ctx);
void set_allocator(AllocFn a, FreeFn f, void* ctx);
void set_alloc_failure(long long after);
void* dev_alloc(size_t bytes);
void dev_free(void* p);

long long launch_count();
int profile_enable(int on);
int profile_read(const char** names, double* ms, long long* launches, int cap);
void profile_reset();

constexpr int kMaxNets = 8;
constexpr int kDefaultNbrCap = 160;
constexpr int kMaxNbrCap = 256;   // rows grow to this once; lists with a skin start here

struct DevWeights {
    int n_nets = 1;
    int device = 0;
    void* blk_f32 = nullptr;
    void* blk_bf16 = nullptr;
    NetF32 f32[kMaxNets];   // net k
    NetBF16 bf16;           // all nets
};

// precision: 0 = FP32 network, 1 = BF16 tensor cores with split-precision
// forward, 2 = BF16 tensor cores, single pass
struct Workspace {
    int cap_atoms = 0, cap_mols = 0, rows_cap = 0, nbr_cap = 0, max_cells = 0;
    int precision = 0;
    int nets = 1;   // ensemble size of the weights it serves
    // rows of per-atom energies: one per net for the BF16 ensemble (averaged
    // by the finalize kernel); the FP32 path accumulates the mean in place
    int e_nets() const { return (precision != 0 && nets > 1) ? nets : 1; }
    bool cell_path = false;
    size_t bytes = 0;
    std::vector<void*> owned;

    float4 *hi = nullptr, *lo = nullptr, *ref = nullptr;
    int *rank = nullptr, *nbr = nullptr, *nbr_cnt = nullptr, *row_atom = nullptr;
    Counters* ctr = nullptr;
    double* grad = nullptr;
    float* G32 = nullptr;
    __nv_bfloat16* G16 = nullptr;
    __nv_bfloat16* G16lo = nullptr;   // split-precision network only
    float* dG = nullptr;              // FP32 network
    __nv_bfloat16* dG16 = nullptr;    // BF16 networks
    __nv_bfloat16* g1ens = nullptr;   // BF16 ensemble: every net's g1, [rows][nets * 256]
    MlpF32Bufs fb{};
    float* e = nullptr;               // [e_nets()][cap_atoms]
    Grid* grid = nullptr;
    int *cell_of_atom = nullptr, *cell_rank = nullptr, *cell_count = nullptr, *cell_start = nullptr,
        *cell_atoms = nullptr;
    int* ang_big_list = nullptr;           // atoms with more than kAngCap angular neighbors
    unsigned char* ang_big_flag = nullptr;  // per atom: 1 if listed there
    int* tc_err = nullptr;
    int* err_sticky = nullptr;   // error flags of all evaluations since the host last cleared them
    Counters* h_ctr = nullptr;   // pinned host copy of the counters of the last evaluation
};

// Bytes a workspace of these dimensions occupies on the device.
size_t workspace_bytes(int cap_atoms, int cap_mols, int precision, bool cell_path, int nbr_cap, int max_cells,
                       int nets);
int workspace_create(Workspace& ws, int cap_atoms, int cap_mols, int precision, bool cell_path, int nbr_cap,
                     int max_cells, int nets);
void workspace_destroy(Workspace& ws);

// Open systems of at most this many atoms without a persistent neighbor list
// take the all-pairs neighbor search of the batch path.
constexpr int kAllPairsMaxAtoms = 1024;

struct EvalSpec {
    int n_atoms = 0;
    int n_mols = 1;
    const int* d_mol_start = nullptr;   // batch layout (all-pairs per molecule); nullptr = one system
    const int8_t* d_species = nullptr;
    const double* d_xyz = nullptr;
    // system geometry
    int periodic = 0;
    double L[3] = {0, 0, 0};
    float r_list = kRcRad;
    float half_skin2 = 0.f;             // > 0: displacement guard of a persistent list
    bool force_rebuild = true;
    bool reuse_aev = false;             // skip staging, neighbors and AEV (kept from the forward)
    bool network_backward = true;       // run the network backward and the force kernel
    bool energy = true;
    double* d_E = nullptr;              // [n_mols]
    float* d_F = nullptr;               // [n_atoms][3]
    const double* d_grad_scale = nullptr;
    float sign = -1.f;                  // -1: forces; +1: energy gradient
    // ML/MM region: d_xyz (n_atoms rows, owned by the caller of enqueue_eval)
    // is first gathered from rows d_index of d_coords_full [n_full][3], and
    // the forces go to rows d_index of d_F (n_full rows), added when
    // accumulate is set
    const int* d_index = nullptr;
    const double* d_coords_full = nullptr;
    long long n_full = 0;
    bool accumulate = false;
};

// Enqueues one evaluation on `st`; returns MLP_OK or an error code (argument
// or launch error). The counters are copied to ws.h_ctr at the end.
int enqueue_eval(Workspace& ws, const DevWeights& w, const EvalSpec& spec, cudaStream_t st);

// Reads the counters copied by the last evaluation (after the stream has been
// synchronized) and turns overflow / bad input into an error code.
int check_counters(const Workspace& ws);

Box make_box(int periodic, const double* L);
// Cell grid of an orthorhombic periodic box for a search radius r_list: cells
// at least r_list wide, at most max_cells of them (fewer, wider cells when
// floor(L / r_list) per axis would give more).
Grid make_periodic_grid(const double* L, float r_list, long long max_cells);

}  // namespace mlp
