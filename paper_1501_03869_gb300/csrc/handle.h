// handle.h -- internal state of a back-projection handle, shared by the C
// ABI translation units (single handle, multi-instance plans, serving).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/pat_bp.h"
#include "kernels.cuh"
#include "table.h"

namespace patbp {

pat_status fail(pat_status s, const std::string& msg);
pat_status cuda_fail(cudaError_t e, const char* what);
inline int round_up(int x, int m) { return (x + m - 1) / m * m; }

#define PAT_CUDA(call)                                  \
  do {                                                  \
    cudaError_t e_ = (call);                            \
    if (e_ != cudaSuccess) return patbp::cuda_fail(e_, #call); \
  } while (0)

}  // namespace patbp

struct pat_bp_s {
  int device = 0;
  int n_sm = 0;
  int max_smem = 232448;              // opt-in shared memory per block (bytes)
  int max_smem_sm = 233472;           // shared memory per multiprocessor (bytes)
  patbp::GridDesc g;
  int ns = 0, ns_pad = 0, nt = 0, nt_pad = 0;
  double dt = 0.0;
  unsigned flags = 0;
  bool compact = false;
  int P = 128, SW = 4, n_tiles = 0, W = 0;
  int delays = 0;                     // 0 fast-marching table, 1 constant speed c0
  double c0 = 0.0;
  int G = 64, n_seg = 1;              // sensors per segment, segments per tile
  int64_t n_pix = 0, grid_total = 0, out_stride = 0;
  int n_zero_runs = 0;
  double build_seconds = 0.0;
  std::vector<uint16_t> win_len;      // host copy of the window lengths [tile][sensor]
  int pre_frames = 0;                 // frames held by the integrand buffer
  int pre_fmt = 0;                    // their storage format
  int pre_fb = 1;                     // their frames per group
  int wst_cache[33] = {0};            // stage window bound per sensors-per-stage
  // launch shapes chosen by the autotuner: [frames-per-group index][format]
  int tuned_S[4][3] = {};
  int tuned_budget_kb[4][3] = {};
  float* d_u = nullptr;               // table offsets (delays == 0)
  float* d_anchor = nullptr;          // per (tile, sensor) anchors (delays == 1)
  float4* d_pix = nullptr;            // per-pixel terms (delays == 1 or wgt)
  float* d_wanchor = nullptr;         // solid-angle weight anchors (wgt)
  int wgt = 0;                        // 1: exact back projection (solid-angle weights)
  // host copies kept for pat_bp_set_solid_angle: sensor positions and the
  // dense slot map of the pixel layout
  std::vector<double> sensors_xyz;
  std::vector<int32_t> slot_dense;
  int32_t* d_base = nullptr;
  int32_t* d_slot = nullptr;
  int32_t* d_zero_runs = nullptr;
  float* d_w = nullptr;
  int* d_status = nullptr;
  unsigned* d_sched = nullptr;        // gather unit tickets (self-resetting)
  void* d_b = nullptr;
  size_t b_cap = 0;
  float* d_m = nullptr;
  size_t m_cap = 0;
  float* d_part = nullptr;            // segment partial sums (scratch)
  size_t part_cap = 0;
  int* d_counter = nullptr;           // per (frame group, tile) segment counters
  size_t counter_cap = 0;
  // staging of pat_bp_reconstruct_host
  cudaStream_t own_stream = nullptr;
  void* d_sig = nullptr;
  size_t sig_cap = 0;
  float* d_scales = nullptr;
  size_t scales_cap = 0;
  float* d_out = nullptr;
  size_t out_cap = 0;
  int* host_status = nullptr;         // host-mapped copy of the status word
  int* host_status_dev = nullptr;     // its device address
  // pinned host copy of the device table (PAT_FLAG_HOST_MIRROR): u (or the
  // anchors), base, slot, zero runs, weights, the per-pixel terms (constant
  // speed or solid-angle weights) and the solid-angle weight anchors; lets the
  // device copy be dropped and reloaded
  static constexpr int kMirrors = 7;
  void* mirror[kMirrors] = {};
  size_t mirror_bytes[kMirrors] = {};
  bool evicted = false;
  std::mutex mu;
};

namespace patbp {

// Fewer frames than this go through the unstaged single-frame kernels, one
// frame after the other.
constexpr int kStagedMinFrames = 4;
int frames_per_group(int n_frames);
// frames per unit a handle's reconstruction of n_frames uses (1 below kStagedMinFrames)
int frames_per_unit(pat_bp_t h, int n_frames);
int fb_index(int FB);
int fmt_for(pat_dtype dt);
// device buffers for n_frames frames grouped by FB (grown, zero-filled)
pat_status ensure_buffers_fb(pat_bp_t h, int n_frames, int FB);
// window rows one pipeline stage of S sensors can need
int stage_window(pat_bp_t h, int S);
// stages and window-row budget of a shape under a smem budget (false: nothing fits)
bool fit_stages(GatherConfig& c, int wmin, int wfull, size_t budget, int* wst);
// launch shape: frames per unit, sensors per stage, stages under a smem budget
GatherConfig config_for(pat_bp_t h, int FB, int S, size_t budget, int* wst);
GatherConfig pick_config(pat_bp_t h, int n_frames, int fmt, int* wst);
// one instance's preprocessing and gather descriptors for n_frames frames
PreParams make_pre(pat_bp_t h, const void* sig, pat_dtype dtype, const float* scales, int n_frames,
                   int FB);
InstDesc make_desc(pat_bp_t h, float* out, int n_frames, int FB, int wst);
// device bytes the handle holds now (table plus working buffers)
size_t resident_bytes(pat_bp_t h);
// device bytes of the table alone
size_t table_device_bytes(pat_bp_t h);
pat_status evict_locked(pat_bp_t h);
// preprocess + gather on stream (caller holds h->mu or owns h exclusively)
// With host_status set, the status word ends up there too: *exported tells
// whether the launches already copied it (the unstaged path), else the caller
// must.
pat_status reconstruct_locked(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                              const float* scales_dev, int n_frames, float* out_dev,
                              cudaStream_t stream, int* host_status = nullptr,
                              bool* exported = nullptr);
pat_status restore_locked(pat_bp_t h, cudaStream_t st);
// evict an idle handle by giving its device buffers to an evicted handle of the
// same sizes (no synchronisation or allocation); false if the sizes differ
bool donate_buffers_locked(pat_bp_t from, pat_bp_t to);
// resident gather CTAs for a config (cached per config)
int resident_ctas(const GatherConfig& c, int fmt, int wst, int n_sm);

}  // namespace patbp
