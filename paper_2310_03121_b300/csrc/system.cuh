// Definitions shared by the C-ABI translation units (api.cu, integrator.cu):
// the opaque handles of include/mlp.h and the per-system helpers.
#pragma once

#include "../../include/mlp.h"
#include "engine.cuh"

struct mlp_weights {
    mlp::DevWeights dw;
};

struct mlp_system {
    int n = 0;
    int periodic = 0;
    double L[3] = {0, 0, 0};
    mlp_cutoffs cut{};
    const mlp_weights* w = nullptr;
    int precision = 0;
    mlp::Workspace ws;
    cudaStream_t stream = nullptr;
    int8_t* d_species = nullptr;
    double* d_xyz = nullptr;
    double* d_E = nullptr;
    float* d_F = nullptr;
    double* h_xyz = nullptr;   // pinned staging
    double* h_E = nullptr;
    float* h_F = nullptr;
    void* dev_block = nullptr;
    long long calls = 0;
    int rebuild_interval = 10;
    bool kept = false;
    const double* kept_coords = nullptr;
    bool nbr_valid = false;
    cudaEvent_t done = nullptr;
    bool pending = false;   // counters of an asynchronous call not yet checked
};

namespace mlp {
int check_cuda_device();
int sys_finish_pending(mlp_system* s);   // waits for the last evaluation and reports its errors
int sys_check_if_done(mlp_system* s);    // reports the last evaluation's errors if it has finished
EvalSpec sys_spec(mlp_system* s, const double* d_xyz);
}  // namespace mlp
