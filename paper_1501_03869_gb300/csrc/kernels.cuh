// kernels.cuh -- launch interface of the back-projection kernels (internal).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace patbp {

// Storage of the Eq. (BP) integrand written by the preprocessing kernel.  Rows
// are frame-interleaved: entry (k, fb) of frame group g and sensor s sits at
// ((g * N_s + s) * N_t_pad + k) * FB + fb, so one window of FB frames is one
// contiguous block.
enum BFormat : int {
  kBF32 = 0,    // float b_k; the gather reads rows k and k + 1
  kBBF16P = 1,  // bf16 pair (b_k, b_{k+1} - b_k) / sigma in one 32-bit word
  kBF16P = 2,   // fp16 pair (b_k, b_{k+1} - b_k) / sigma in one 32-bit word
};

// Device status bits (written with atomicOr, read by the host after a sync).
enum : int { kStatusTimeout = 1, kStatusBadConfig = 2 };

constexpr int kMaxInst = 64;    // instances one gather launch can stream
constexpr int kMaxStages = 8;   // pipeline depth limit
constexpr int kMaxS = 32;       // sensors per stage limit
constexpr int kMaxG = 256;      // sensors per segment limit
constexpr int kTailRows = 16;   // rows of slack after the last integrand row

struct PreParams {
  const void* sig;       // [F][N_s][N_t] of dtype (0 f32, 1 bf16, 2 f16)
  const float* scales;   // [F][N_s] or null
  const float* weights;  // [N_s]
  void* b;               // [n_fg][N_s][N_t_pad][FB] entries of the format
  float* m;              // [n_fg][N_s_pad][FB] multipliers w_s * sigma (0 for absent frames)
  int dtype, fmt, FB;
  int n_sensors, n_sensors_pad, n_t, n_t_pad, n_frames;
};

// Preprocessing of several instances in one launch (same dtype, format, FB).
struct PreMultiParams {
  PreParams inst[kMaxInst];
  int64_t cta_begin[kMaxInst + 1];  // prefix sums of N_s * n_fg per instance
  int n_inst, dtype, fmt, FB;
};

// One speed map's on-line data for a gather launch.  Work is cut into units
// (frame group, tile, segment of G sensors); units of all instances form one
// sequence that the launch splits into contiguous ranges, one per CTA.
struct InstDesc {
  const float* u;           // [n_tiles][N_s][P] table offsets (stored-table delays)
  const float* anchor;      // [n_tiles][N_s_pad][8] per-sensor anchors (constant-speed delays)
  const float4* pix;        // [n_tiles][P] pixel terms (2D, |D|^2) (constant-speed delays or
                            // solid-angle weights)
  const float* wanchor;     // [n_tiles][N_s_pad][8] solid-angle weight anchors, or NULL
  const int32_t* base;      // [n_tiles][N_s_pad] window base | (window length << 16)
  const int32_t* slot;      // [n_tiles * P] output index, -1 = padding
  const int32_t* zero_runs; // (start, length) pairs of outputs to clear
  const void* b;            // integrand rows
  const float* m;           // multipliers
  float* out;               // [F][out_stride]
  float* part;              // [n_fg][n_tiles][n_seg][FB][P] segment partial sums
  int* counter;             // [n_fg][n_tiles] segments finished (returns to 0)
  int64_t out_stride;
  int64_t unit_begin;       // index of this instance's first unit
  int n_zero_runs;
  int n_sensors, n_sensors_pad, n_t_pad, n_tiles, n_frames, n_fg, n_seg, G, Wst;
  int W;                    // longest window of one (tile, sensor) (rows)
};

struct StreamParams {
  InstDesc inst[kMaxInst];
  int n_inst;
  int64_t n_units;
  int S;                    // sensors per pipeline stage (multiple of 4 and of SW, <= 32)
  int stages;               // pipeline depth
  int Wst;                  // window rows one stage can need (max over instances)
  int* status;
  int* host_status;         // host-mapped word the unstaged path's last kernel copies the
                            // status into, or NULL
  unsigned* sched;          // [4] zero-initialised: unit ticket (64-bit) and CTAs finished
  uint64_t timeout_ns;
};

struct GatherConfig {
  int P = 128;      // pixels per tile
  int FB = 1;       // frames per unit (1, 2, 4, 8)
  int SW = 4;       // sensor-phase warps
  int S = 16;       // sensors per stage
  int stages = 4;
  int delays = 0;   // 0 stored table, 1 constant speed computed in the kernel
  int wgt = 0;      // 1: solid-angle weights per (pixel, sensor)
  int direct = 0;   // 1: single frame through the unstaged kernels (gather_direct.cu)
  int no_window = 0;  // 1: the unstaged kernel gathers from L2, never from shared-memory windows
  int n_sm = 0;     // multiprocessors of the device (sizes the unstaged grid)
};

size_t gather_smem_bytes(const GatherConfig& c, int Wst);
int gather_threads(const GatherConfig& c);
// CTAs of one gather launch that fit on the device at once.
int gather_resident_ctas(const GatherConfig& c, int fmt, int Wst, int n_sm);

cudaError_t launch_preprocess(const PreParams& p, cudaStream_t st);
// Copy the device status word into a host-mapped word (after the stream's
// earlier work), so the host reads it after a stream synchronisation without
// a blocking copy.
cudaError_t launch_status_export(const int* status, int* host_status, cudaStream_t st);
cudaError_t launch_preprocess_multi(const PreMultiParams& p, cudaStream_t st);
const void* gather_kernel_func(const GatherConfig& c, int fmt);
const void* preprocess_multi_func(int dtype, int fmt, int FB);
cudaError_t launch_gather(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                          cudaStream_t st);
cudaError_t launch_wait_probe(int* status, uint64_t timeout_ns, cudaStream_t st);
// One frame of one instance through the unstaged gather and its reduction
// kernel (c.FB == 1; d.part holds direct_part_floats floats); same arithmetic
// and summation order as the staged kernel with one frame per unit.
// reduce = false launches the gather kernel only (its phase or segment sums;
// the image is not written): a measurement hook.
cudaError_t launch_gather_direct(const GatherConfig& c, int fmt, const InstDesc& d, int n_sm,
                                 int* status, int* host_status, uint64_t timeout_ns,
                                 cudaStream_t st, bool reduce = true);
// Phase sums the unstaged gather stores (floats).
size_t direct_part_floats(const GatherConfig& c, int n_tiles, int n_seg);

}  // namespace patbp
