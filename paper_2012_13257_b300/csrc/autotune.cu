// Autotuner core: times the single-image forward for every (micro-tile
// variant, bin edge) candidate on the caller's problem and reports the fastest.
// The caller (the Python Autotuner) keeps the winners per problem bucket.
// A tuning call, not the hot path: it allocates its own workspace and output.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "gmi.h"

extern "C" gmi_status gmi_autotune(const float* points, const float* values, int64_t N, int C, int H, int W,
                                   const gmi_params* p, const int* bins, int n_bins, int reps, gmi_params* best,
                                   float* times_ms, gmi_stream_t stream) {
  if (!p || !bins || n_bins < 1 || reps < 1 || !best) return GMI_ERR_INVALID_ARG;
  for (int k = 0; k < n_bins; ++k)
    if (bins[k] < 0 || bins[k] > 1024) return GMI_ERR_INVALID_ARG;
  const int variants[3] = {GMI_VARIANT_MT4x4, GMI_VARIANT_MT4x8, GMI_VARIANT_MT2x4};
  // the largest workspace any candidate needs (also validates the arguments)
  size_t ws_bytes = 0;
  for (int v : variants) {
    for (int k = 0; k < n_bins; ++k) {
      gmi_params q = *p;
      q.variant = v;
      q.bin_px = bins[k];
      q.flags &= ~GMI_FLAG_GRAPH;
      size_t b = 0;
      const gmi_status st = gmi_workspace_size(N, C, H, W, &q, &b);
      if (st != GMI_OK) return st;
      ws_bytes = std::max(ws_bytes, b);
    }
  }
  cudaStream_t s = (cudaStream_t)stream;
  void* ws = nullptr;
  float* img = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  gmi_status st = GMI_OK;
  if (cudaMalloc(&ws, ws_bytes) != cudaSuccess ||
      cudaMalloc((void**)&img, sizeof(float) * (size_t)H * (size_t)W * (size_t)C) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    st = GMI_ERR_CUDA;
  }
  float best_ms = -1.0f;
  std::vector<float> ms(reps);
  for (int vi = 0; vi < 3 && st == GMI_OK; ++vi) {
    for (int k = 0; k < n_bins && st == GMI_OK; ++k) {
      gmi_params q = *p;
      q.variant = variants[vi];
      q.bin_px = bins[k];
      q.flags &= ~GMI_FLAG_GRAPH;
      st = gmi_forward(points, values, N, C, H, W, &q, img, nullptr, nullptr, ws, ws_bytes, stream);   // warm-up
      for (int r = 0; r < reps && st == GMI_OK; ++r) {
        if (cudaEventRecord(e0, s) != cudaSuccess) st = GMI_ERR_CUDA;
        if (st == GMI_OK) st = gmi_forward(points, values, N, C, H, W, &q, img, nullptr, nullptr, ws, ws_bytes, stream);
        if (st == GMI_OK && (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
                             cudaEventElapsedTime(&ms[r], e0, e1) != cudaSuccess))
          st = GMI_ERR_CUDA;
      }
      if (st != GMI_OK) break;
      std::sort(ms.begin(), ms.end());
      const float med = ms[reps / 2];
      if (times_ms) times_ms[vi * n_bins + k] = med;
      if (best_ms < 0.0f || med < best_ms) {
        best_ms = med;
        *best = q;
        best->flags = p->flags;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (img) cudaFree(img);
  if (ws) cudaFree(ws);
  return st;
}
