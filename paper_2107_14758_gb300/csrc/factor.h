// Host-side declarations of the set-up kernels.
#pragma once
#include <cuda_runtime.h>

#include "device.cuh"

namespace fdm {

struct FactorArgs {
  Grid g;
  const ClassDev *cls;
  const PatchDev *patches;
  const int *plist;     // patch ids of this batch (one CTA each)
  const double *mu;     // surrogate coefficients [ncell][3]
  const double *tab;    // FP64 1D tables
  double *S;            // workspace: one nG_max^2 dense matrix per batch slot
  int64_t ldS;
  double *L64;          // factor values (FP64)
  float *L32;           // factor values (FP32 copy) or nullptr
  int *status;          // set to 1 on a nonpositive pivot
};

size_t assemble_smem_bytes(int n);
void launch_factor_batch(const FactorArgs &a, int count, cudaStream_t st);
void launch_assemble_factor_only(const FactorArgs &a, int count, cudaStream_t st);
void launch_banded_inverse(int m, int bw, const double *Lb, double *out, cudaStream_t st);

}  // namespace fdm
