// dpm_kernels.h -- host-side launchers of the library's kernels.
#pragma once

#include <cuda_runtime.h>

#include "dpm_internal.h"

namespace dpm {

void launch_history(const RunParams &R, uint64_t batch_size, int sm_count, int block, cudaStream_t st);
// The same kernel in FP64 arithmetic with FP64 tables (precision ablation).
void launch_history_f64(const RunParamsT<double> &R, uint64_t batch_size, int sm_count, cudaStream_t st);
// The paper's float tally (ablation): transport into float slabs (n_slab
// floats, zeroed by the caller), then their rounding into R.slabs.
void launch_history_paper(const RunParams &R, uint64_t batch_size, bool cas, float *fslabs, size_t n_slab,
                          int sm_count, cudaStream_t st);
void launch_fold(const unsigned long long *slabs, int nb, size_t V, const double *inv_nb, long long *S1, double *Q,
                 int sm_count, cudaStream_t st);
void launch_normalize(const long long *S1, const double *Q, const float *rho, size_t V, double n, double B,
                      double vox_cm3, double *dose, double *sigma, int sm_count, cudaStream_t st);

// D_max of the accumulated tally and its sigma: out = {dose Gy/history, sigma, voxel}.
void launch_dmax(const long long *S1, const double *Q, const float *rho, size_t V, double n, double B, double vox_cm3,
                 unsigned long long *key, double *out, int sm_count, cudaStream_t st);

void launch_diag_table(const DevTables &T, const DevPhantom &P, int which, int mat, int n, const double *E,
                       const double *aux, double *out, cudaStream_t st);
void launch_diag_sample(const DevTables &T, int which, double e, double aux, int n, const double *u, double *out,
                        cudaStream_t st);
void launch_diag_philox(int n, const uint32_t *ctr, const uint32_t *key, uint32_t *out, cudaStream_t st);
void launch_l2_atomic(unsigned long long *a, uint32_t mask, int iters, int blocks, cudaStream_t st);
void launch_atomic_replay(unsigned long long *slab, const uint32_t *ids, size_t n, int blocks, cudaStream_t st);
void launch_l2_read(const float4 *b, size_t n, int passes, float *sink, int blocks, cudaStream_t st);

}  // namespace dpm
