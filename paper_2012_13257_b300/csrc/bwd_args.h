// Arguments of the backward kernels, shared with the batched host code.
#pragma once

#include "common.cuh"

namespace gmi {

// Per-image backward arguments (device table in batched calls).
struct BwdImage {
  const float* image;   // [H,W,C] forward output
  const float* den;     // [H,W]
  const float* shift;   // [H,W] or null (all zero: truncated mode)
  const float* grad;    // [H,W,C] upstream gradient
  float* gpts;          // [N,2] or null
  float* gvals;         // [N,C] or null
  float* gsig;          // [1] or null
  float* gsigs;         // per-point sigma gradients, pp_kind floats per point, or null
  float inv_s2, inv_s3; // 1/sigma^2, 1/sigma^3
};

struct BwdArgs {
  BwdImage one;              // the image of a single-image call
  const BwdImage* table;     // batched: per-image table (else null)
  int trunc;
  int pp;                    // per-point sigmas (single image, truncated mode): 1 separable, 2 full
};

cudaError_t launch_backward(const KArgs& a, const BwdArgs& b, cudaStream_t s);

}  // namespace gmi
