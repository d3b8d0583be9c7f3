// mlp_internal.cuh -- internal interfaces of the learned-operator path
// (network training and inference, migration with generated operators).
#pragma once

#include "fxmig_internal.cuh"

namespace fxmig_impl {

constexpr int kMlpMaxOut = 32;  // 2(L+1) network outputs, padded to the MMA tile: L <= 15
constexpr int kMlpMaxL = kMlpMaxOut / 2 - 1;
constexpr int kMlpMaxNx = 16384;  // one velocity row sorted in shared memory

int mlp_param_count(int L);
size_t mlp_train_ws_bytes(int L, int n);
// nsteps training steps (grad_out == nullptr) or one gradient evaluation
// (grad_out != nullptr: the summed gradient is written, parameters untouched).
cudaError_t launch_mlp_train(int L, float* params, float* m, float* v, int step0, int nsteps, float lr_max,
                             float lr_min, int schedule_steps, const double* kv, double k_max, const float* target,
                             int n, float* loss, float* grad_out, void* ws, cudaStream_t s);
cudaError_t launch_mlp_taps(int L, const float* params, const double* kv, double k_max, long long n, void* taps,
                            cudaStream_t s);
cudaError_t launch_mlp_block_taps(const fxmig_desc* d, int LT, const float* params, const float* uval,
                                  const int* cnt, const long long* base, int z0, int z1, float4* taps,
                                  cudaStream_t s);

struct MlpMigratePlan {
    int LT, groups, zc;  // compiled half-length, frequency tiles, rows per operator block
    int nparts;
    int persistent;      // depth steps by the persistent form (else one launch per row)
    MigratePlan pplan;   // its plan
};
int plan_mlp_migrate(const fxmig_desc* d, MlpMigratePlan* p);
size_t mlp_migrate_ws_bytes(const fxmig_desc* d);
cudaError_t launch_mlp_migrate(const fxmig_desc* d, const MlpMigratePlan& plan, void* slab, const float* vel,
                               const float* params, float* partials, int z_begin, int z_end, void* ws,
                               cudaStream_t s);

}  // namespace fxmig_impl
