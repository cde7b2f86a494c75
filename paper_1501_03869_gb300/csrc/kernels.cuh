// kernels.cuh -- launch interface of the back-projection kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace patbp {

// Storage of the Eq. (BP) integrand rows written by the preprocessing kernel.
enum BFormat : int {
  kBF32 = 0,    // float b_k; gather reads b_k and b_{k+1}
  kBBF16P = 1,  // bf16 pair (b_k, b_{k+1} - b_k) / sigma
  kBF16P = 2,   // fp16 pair (b_k, b_{k+1} - b_k) / sigma
};

inline int bformat_bytes(int f) { return f == kBF32 ? 4 : 4; }

// Device status bits (written with atomicOr, read by the host after a sync).
enum : int { kStatusTimeout = 1, kStatusBadConfig = 2 };

struct PreParams {
  const void* sig;       // [F][N_s][N_t] of dtype (0 f32, 1 bf16, 2 f16)
  const float* scales;   // [F][N_s] or null
  const float* weights;  // [N_s]
  void* b;               // [F][N_s][N_t_pad] entries of the format
  float* m;              // [F][N_s_pad] multipliers w_s * sigma
  int dtype, fmt;
  int n_sensors, n_sensors_pad, n_t, n_t_pad, n_frames;
};

struct GatherParams {
  const float* u;          // [n_tiles][N_s][P]
  const int32_t* base;     // [n_tiles][N_s] window base | (window length << 16)
  const int32_t* slot;     // [n_tiles * P] output index, -1 = padding
  const int32_t* zero_runs;// (start, length) pairs of outputs to clear
  int n_zero_runs;
  const void* b;           // integrand rows
  const float* m;          // [F][N_s_pad]
  float* out;              // [F][out_stride]
  int64_t out_stride;
  int n_sensors, n_sensors_pad, n_t_pad, n_tiles, n_frames;
  int Wst;                 // window entries one stage can need per frame (multiple of 8)
  int S;                   // sensors per pipeline stage (multiple of 4 and of SW, <= 32)
  int stages;              // pipeline depth
  int split;               // sensor splits per tile = cluster size (1..8)
  int split_len;           // sensors per split (multiple of 4)
  int* status;
  uint64_t timeout_ns;
};

struct GatherConfig {
  int P = 128;      // pixels per tile (128 or 256)
  int FB = 1;       // frames per CTA (1, 2, 4, 8)
  int SW = 4;       // sensor-phase warps per pixel group
  int S = 16;       // sensors per stage
  int stages = 4;
};

// Shared-memory bytes of one gather CTA.
size_t gather_smem_bytes(const GatherConfig& c, int fmt, int Wst);
int gather_threads(const GatherConfig& c);

cudaError_t launch_preprocess(const PreParams& p, cudaStream_t st);
cudaError_t launch_gather(const GatherConfig& c, int fmt, const GatherParams& p, cudaStream_t st);
cudaError_t launch_wait_probe(int* status, uint64_t timeout_ns, cudaStream_t st);

}  // namespace patbp
