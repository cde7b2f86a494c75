// pat_bp.cu -- C ABI of the back-projection library (include/pat_bp.h).
//
// Off-line step (Sec. III): pat_bp_create runs the host fast marching of
// Sec. II-B for every sensor, lays the travel times out for the gather kernel
// and uploads them once.  On-line step: pat_bp_reconstruct enqueues the
// preprocessing kernel (Eq. (BP) integrand) and the gather kernel on the
// caller's stream.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "handle.h"

using namespace patbp;

namespace patbp {

thread_local std::string g_last_error;

pat_status fail(pat_status s, const std::string& msg) {
  g_last_error = msg;
  return s;
}

pat_status cuda_fail(cudaError_t e, const char* what) {
  g_last_error = std::string(what) + ": " + cudaGetErrorString(e);
  return PAT_ERR_CUDA;
}

}  // namespace patbp

extern "C" const char* pat_status_str(pat_status s) {
  switch (s) {
    case PAT_OK: return "ok";
    case PAT_ERR_INVALID: return "invalid argument";
    case PAT_ERR_OOM: return "out of memory";
    case PAT_ERR_CUDA: return "CUDA error";
    case PAT_ERR_TIMEOUT: return "timeout";
    case PAT_ERR_BUSY: return "busy";
    case PAT_ERR_NOT_FOUND: return "not found";
    case PAT_PENDING: return "pending";
  }
  return "unknown status";
}

extern "C" const char* pat_last_error(void) { return g_last_error.c_str(); }

static bool grid_from_abi(const pat_grid* pg, GridDesc& g, std::string& err) {
  if (!pg || (pg->ndim != 2 && pg->ndim != 3)) {
    err = "grid.ndim must be 2 or 3";
    return false;
  }
  g.ndim = pg->ndim;
  for (int d = 0; d < 3; ++d) {
    g.n[d] = d < pg->ndim ? pg->n[d] : 1;
    g.origin[d] = pg->origin[d];
    if (g.n[d] < 1 || (d < pg->ndim && g.n[d] < 2)) {
      err = "grid needs at least 2 nodes along every active axis";
      return false;
    }
  }
  g.dx = pg->dx;
  if (!(g.dx > 0.0) || !std::isfinite(g.dx)) {
    err = "grid.dx must be > 0";
    return false;
  }
  if (g.total() > (int64_t(1) << 31) - 1) {
    err = "grid too large (2^31 nodes at most)";
    return false;
  }
  return true;
}

static void free_handle(pat_bp_t h) {
  if (!h) return;
  cudaFree(h->d_u);
  cudaFree(h->d_anchor);
  cudaFree(h->d_pix);
  cudaFree(h->d_wanchor);
  cudaFree(h->d_base);
  cudaFree(h->d_slot);
  cudaFree(h->d_zero_runs);
  cudaFree(h->d_w);
  cudaFree(h->d_status);
  cudaFree(h->d_sched);
  cudaFree(h->d_b);
  cudaFree(h->d_m);
  cudaFree(h->d_part);
  cudaFree(h->d_counter);
  cudaFree(h->d_sig);
  cudaFree(h->d_scales);
  cudaFree(h->d_out);
  for (int i = 0; i < pat_bp_s::kMirrors; ++i) cudaFreeHost(h->mirror[i]);
  cudaFreeHost(h->host_status);
  if (h->own_stream) cudaStreamDestroy(h->own_stream);
  delete h;
}

template <typename T>
static pat_status upload(T** dst, const std::vector<T>& src, const char* what) {
  size_t bytes = std::max<size_t>(src.size(), 1) * sizeof(T);
  cudaError_t e = cudaMalloc(reinterpret_cast<void**>(dst), bytes);
  if (e != cudaSuccess) return fail(PAT_ERR_OOM, std::string("cudaMalloc ") + what);
  if (!src.empty()) PAT_CUDA(cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice));
  return PAT_OK;
}

// Checks shared by both create calls.
static pat_status check_create_args(const pat_grid* grid, const double* sensors_host, int n_sensors,
                                    double dt, int n_samples, GridDesc& g) {
  if (!sensors_host) return fail(PAT_ERR_INVALID, "sensors NULL");
  if (n_sensors < 1 || n_sensors > (1 << 20)) return fail(PAT_ERR_INVALID, "n_sensors out of range");
  if (!(dt > 0.0) || !std::isfinite(dt)) return fail(PAT_ERR_INVALID, "dt must be > 0");
  if (n_samples < 2 || n_samples > 32768) return fail(PAT_ERR_INVALID, "n_samples must be 2..32768");
  std::string err;
  if (!grid_from_abi(grid, g, err)) return fail(PAT_ERR_INVALID, err);
  return PAT_OK;
}

static pat_status new_handle(const GridDesc& g, int n_sensors, int n_samples, double dt,
                             unsigned flags, pat_bp_t* out) {
  pat_bp_t h = new (std::nothrow) pat_bp_s();
  if (!h) return fail(PAT_ERR_OOM, "handle");
  cudaDeviceProp prop;
  cudaError_t e = cudaGetDevice(&h->device);
  if (e == cudaSuccess) e = cudaGetDeviceProperties(&prop, h->device);
  if (e != cudaSuccess) {
    delete h;
    return cuda_fail(e, "device properties");
  }
  h->n_sm = prop.multiProcessorCount;
  h->max_smem = int(prop.sharedMemPerBlockOptin);
  h->max_smem_sm = int(prop.sharedMemPerMultiprocessor);
  h->g = g;
  h->ns = n_sensors;
  h->ns_pad = round_up(n_sensors, 4);
  h->nt = n_samples;
  h->nt_pad = round_up(n_samples + 1, 8);
  h->dt = dt;
  h->flags = flags;
  h->compact = (flags & PAT_FLAG_COMPACT_OUT) != 0;
  h->P = (flags & PAT_FLAG_TILE_256) ? 256 : 128;
  h->SW = h->P == 128 ? 4 : 2;
  h->grid_total = g.total();
  *out = h;
  return PAT_OK;
}

// Upload the built layout and finish the handle (frees it on failure).
static pat_status finish_create(pat_bp_t h, const HostTable& tab, const double* sensors_host,
                                const float* weights_host, pat_bp_t* out) {
  const int n_sensors = h->ns;
  h->sensors_xyz.assign(sensors_host, sensors_host + 3 * size_t(n_sensors));
  h->slot_dense = tab.slot_dense;
  h->n_tiles = tab.n_tiles;
  h->n_pix = tab.n_pix;
  h->W = tab.W;
  h->build_seconds = tab.build_seconds;
  h->out_stride = h->compact ? h->n_pix : h->grid_total;
  h->n_zero_runs = int(tab.zero_runs.size() / 2);
  h->win_len = tab.len;

  // Segments of G sensors per tile: the unit of work balancing and of the
  // fixed-order partial sums.  Fixed per handle so the summation order never
  // changes with the launch shape or the batch.
  h->G = 64;
  h->n_seg = (n_sensors + h->G - 1) / h->G;

  std::vector<float> w(n_sensors);
  for (int s = 0; s < n_sensors; ++s) w[s] = weights_host ? weights_host[s] : 1.0f / float(n_sensors);

  // device form of base and window length: base in the low 16 bits, length
  // in the high 16 bits (n_samples <= 32768 keeps both in range)
  // rows padded to N_s_pad entries so every segment's run is 16-byte aligned
  std::vector<int32_t> packed(size_t(h->n_tiles) * h->ns_pad, 0);
  for (int t = 0; t < h->n_tiles; ++t)
    for (int s = 0; s < n_sensors; ++s) {
      const size_t i = size_t(t) * n_sensors + s;
      packed[size_t(t) * h->ns_pad + s] = int32_t(uint32_t(tab.base[i]) | (uint32_t(tab.len[i]) << 16));
    }
  // constant speed: anchors padded to N_s_pad rows per tile like the bases
  std::vector<float> anchor;
  if (h->delays) {
    anchor.assign(size_t(h->n_tiles) * h->ns_pad * 8, 0.0f);
    for (int t = 0; t < h->n_tiles; ++t)
      std::memcpy(anchor.data() + size_t(t) * h->ns_pad * 8,
                  tab.anchor.data() + size_t(t) * n_sensors * 8, size_t(n_sensors) * 8 * 4);
  }
  const std::vector<float>& delay_data = h->delays ? anchor : tab.u;
  const std::vector<int32_t>& slots = h->compact ? tab.slot_compact : tab.slot_dense;
  pat_status st;
  if ((st = upload(h->delays ? &h->d_anchor : &h->d_u, delay_data, "delay data")) != PAT_OK ||
      (h->delays && (st = upload(reinterpret_cast<float**>(&h->d_pix), tab.pixq, "pixel terms")) != PAT_OK) ||
      (st = upload(&h->d_base, packed, "bases")) != PAT_OK ||
      (st = upload(&h->d_slot, slots, "slots")) != PAT_OK ||
      (st = upload(&h->d_zero_runs, tab.zero_runs, "zero runs")) != PAT_OK ||
      (st = upload(&h->d_w, w, "weights")) != PAT_OK) {
    free_handle(h);
    return st;
  }
  if (h->flags & PAT_FLAG_HOST_MIRROR) {
    const void* src[pat_bp_s::kMirrors] = {delay_data.data(), packed.data(), slots.data(),
                                           tab.zero_runs.data(), w.data(), tab.pixq.data()};
    const size_t bytes[pat_bp_s::kMirrors] = {
        std::max<size_t>(delay_data.size(), 1) * 4, packed.size() * 4, slots.size() * 4,
        std::max<size_t>(tab.zero_runs.size(), 1) * 4, w.size() * 4, tab.pixq.size() * 4};
    for (int i = 0; i < pat_bp_s::kMirrors; ++i) {
      if (bytes[i] == 0) continue;  // no per-pixel terms for a stored table
      if (cudaMallocHost(&h->mirror[i], bytes[i]) != cudaSuccess) {
        free_handle(h);
        return fail(PAT_ERR_OOM, "pinned host mirror");
      }
      h->mirror_bytes[i] = bytes[i];
      if (i != 3 || !tab.zero_runs.empty()) std::memcpy(h->mirror[i], src[i], bytes[i]);
    }
  }
  if (cudaMalloc(&h->d_status, sizeof(int)) != cudaSuccess) {
    free_handle(h);
    return fail(PAT_ERR_OOM, "status word");
  }
  cudaMemset(h->d_status, 0, sizeof(int));
  if (cudaMalloc(&h->d_sched, 4 * sizeof(unsigned)) != cudaSuccess) {
    free_handle(h);
    return fail(PAT_ERR_OOM, "scheduler words");
  }
  cudaMemset(h->d_sched, 0, 4 * sizeof(unsigned));
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    free_handle(h);
    return cuda_fail(e, "create");
  }
  *out = h;
  return PAT_OK;
}

extern "C" pat_status pat_bp_create(const float* speed_host, const pat_grid* grid,
                                    const double* sensors_host, int n_sensors,
                                    const uint8_t* mask_host, const float* weights_host,
                                    double dt, int n_samples, unsigned flags, pat_bp_t* out) {
  if (!out) return fail(PAT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!speed_host) return fail(PAT_ERR_INVALID, "speed NULL");
  GridDesc g;
  pat_status st = check_create_args(grid, sensors_host, n_sensors, dt, n_samples, g);
  if (st != PAT_OK) return st;
  for (int s = 0; s < n_sensors; ++s)
    for (int d = 0; d < g.ndim; ++d) {
      double x = (sensors_host[3 * s + d] - g.origin[d]) / g.dx;
      if (!(x >= 0.0 && x <= double(g.n[d] - 1)))
        return fail(PAT_ERR_INVALID, "sensor " + std::to_string(s) + " lies outside the grid");
    }
  pat_bp_t h = nullptr;
  if ((st = new_handle(g, n_sensors, n_samples, dt, flags, &h)) != PAT_OK) return st;
  HostTable tab;
  std::string err;
  if (!build_table(speed_host, g, sensors_host, n_sensors, mask_host, dt, n_samples, h->P,
                   h->compact, tab, err, (flags & PAT_FLAG_FMM_SECOND_ORDER) ? 2 : 1,
                   (flags & PAT_FLAG_GPU_TABLE) != 0)) {
    free_handle(h);
    return fail(PAT_ERR_INVALID, err);
  }
  return finish_create(h, tab, sensors_host, weights_host, out);
}

extern "C" pat_status pat_bp_create_constant(double c0, const pat_grid* grid,
                                             const double* sensors_host, int n_sensors,
                                             const uint8_t* mask_host, const float* weights_host,
                                             double dt, int n_samples, unsigned flags,
                                             pat_bp_t* out) {
  if (!out) return fail(PAT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!(c0 > 0.0) || !std::isfinite(c0)) return fail(PAT_ERR_INVALID, "c0 must be finite and > 0");
  GridDesc g;
  pat_status st = check_create_args(grid, sensors_host, n_sensors, dt, n_samples, g);
  if (st != PAT_OK) return st;
  pat_bp_t h = nullptr;
  if ((st = new_handle(g, n_sensors, n_samples, dt, flags, &h)) != PAT_OK) return st;
  h->delays = 1;
  h->c0 = c0;
  HostTable tab;
  std::string err;
  if (!build_constant_layout(c0, g, sensors_host, n_sensors, mask_host, dt, n_samples, h->P,
                             h->compact, tab, err)) {
    free_handle(h);
    return fail(PAT_ERR_INVALID, err);
  }
  return finish_create(h, tab, sensors_host, weights_host, out);
}

extern "C" pat_status pat_bp_set_solid_angle(pat_bp_t h, const double* normals_host,
                                             const double* elem_host, double omega0) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  if (!normals_host || !elem_host) return fail(PAT_ERR_INVALID, "normals or elements NULL");
  std::lock_guard<std::mutex> lk(h->mu);
  if (h->evicted) return fail(PAT_ERR_INVALID, "the handle's table is evicted (pat_bp_restore)");
  PAT_CUDA(cudaSetDevice(h->device));
  // the constant-speed handle's pixel terms are in units of kappa = dx / (c0 dt)
  const double unit = h->delays ? h->g.dx / (h->c0 * h->dt) : 1.0;
  std::vector<float> wanchor, pix;
  std::string err;
  if (!build_solid_angle_layout(h->g, h->slot_dense, h->P, h->n_tiles, h->sensors_xyz.data(),
                                normals_host, elem_host, h->ns, h->ns_pad, omega0, unit, !h->delays,
                                wanchor, pix, err))
    return fail(PAT_ERR_INVALID, err);
  PAT_CUDA(cudaDeviceSynchronize());  // no launch of this handle may still read the old buffers
  const std::vector<float> ones(size_t(h->ns), 1.0f);
  // Allocate everything first (device buffers and, with a host mirror, new
  // pinned mirrors), so a failure leaves the handle exactly as it was.
  float* d_wa = nullptr;
  float4* d_px = nullptr;
  void* new_mirror[2] = {nullptr, nullptr};  // pixel terms, weight anchors
  const std::vector<float>* src[2] = {&pix, &wanchor};
  auto release = [&]() {
    cudaFree(d_wa);
    cudaFree(d_px);
    for (void* m : new_mirror) cudaFreeHost(m);
  };
  bool ok = cudaMalloc(&d_wa, wanchor.size() * 4) == cudaSuccess &&
            (h->delays || cudaMalloc(&d_px, pix.size() * 4) == cudaSuccess);
  if (ok && h->mirror[0])
    for (int k = 0; k < 2 && ok; ++k) {
      if (k == 0 && h->delays) continue;  // the constant-speed pixel terms are unchanged
      ok = cudaMallocHost(&new_mirror[k], src[k]->size() * 4) == cudaSuccess;
    }
  if (!ok) {
    release();
    return fail(PAT_ERR_OOM, "solid-angle weights");
  }
  cudaError_t e = cudaMemcpy(d_wa, wanchor.data(), wanchor.size() * 4, cudaMemcpyHostToDevice);
  if (e == cudaSuccess && d_px) e = cudaMemcpy(d_px, pix.data(), pix.size() * 4, cudaMemcpyHostToDevice);
  // the solid angle replaces the per-sensor weights
  if (e == cudaSuccess) e = cudaMemcpy(h->d_w, ones.data(), ones.size() * 4, cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    release();
    return cuda_fail(e, "solid-angle weights upload");
  }
  cudaFree(h->d_wanchor);
  h->d_wanchor = d_wa;
  if (d_px) {
    cudaFree(h->d_pix);
    h->d_pix = d_px;
  }
  h->wgt = 1;
  if (h->mirror[0]) {  // keep the host mirror complete: weights, pixel terms, anchors
    std::memcpy(h->mirror[4], ones.data(), ones.size() * 4);
    for (int k = 0; k < 2; ++k) {
      if (!new_mirror[k]) continue;
      const int i = 5 + k;
      std::memcpy(new_mirror[k], src[k]->data(), src[k]->size() * 4);
      cudaFreeHost(h->mirror[i]);
      h->mirror[i] = new_mirror[k];
      h->mirror_bytes[i] = src[k]->size() * 4;
    }
  }
  return PAT_OK;
}

namespace patbp {

int fmt_for(pat_dtype dt) { return dt == PAT_F32 ? kBF32 : (dt == PAT_BF16 ? kBBF16P : kBF16P); }

int frames_per_group(int n_frames) {
  return n_frames >= 8 ? 8 : (n_frames >= 4 ? 4 : (n_frames >= 2 ? 2 : 1));
}

int frames_per_unit(pat_bp_t h, int n_frames) {
  if (n_frames < kStagedMinFrames && !(h->flags & PAT_FLAG_STAGED_SINGLE)) return 1;
  return frames_per_group(n_frames);
}

int fb_index(int FB) { return FB == 1 ? 0 : (FB == 2 ? 1 : (FB == 4 ? 2 : 3)); }

static pat_status grow_zeroed(void** p, size_t* cap, size_t need, const char* what) {
  if (need <= *cap) return PAT_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, need) != cudaSuccess) return fail(PAT_ERR_OOM, what);
  PAT_CUDA(cudaMemset(*p, 0, need));
  *cap = need;
  return PAT_OK;
}

pat_status ensure_buffers_fb(pat_bp_t h, int n_frames, int FB) {
  const size_t n_fg = size_t((n_frames + FB - 1) / FB);
  pat_status st;
  const size_t b_need = (n_fg * h->ns * h->nt_pad + kTailRows) * FB * 4;
  if ((st = grow_zeroed(&h->d_b, &h->b_cap, b_need, "integrand buffer")) != PAT_OK) return st;
  const size_t m_need = n_fg * h->ns_pad * FB * sizeof(float);
  if ((st = grow_zeroed(reinterpret_cast<void**>(&h->d_m), &h->m_cap, m_need, "multipliers")) != PAT_OK)
    return st;
  {
    // segment partials of the staged kernel, or one frame's phase sums
    const size_t part_need =
        n_fg * h->n_tiles * h->n_seg * std::max(FB, h->SW) * h->P * sizeof(float);
    if ((st = grow_zeroed(reinterpret_cast<void**>(&h->d_part), &h->part_cap, part_need,
                          "segment partials")) != PAT_OK)
      return st;
    const size_t cnt_need = n_fg * h->n_tiles * sizeof(int);
    if ((st = grow_zeroed(reinterpret_cast<void**>(&h->d_counter), &h->counter_cap, cnt_need,
                          "segment counters")) != PAT_OK)
      return st;
  }
  return PAT_OK;
}

// Largest sum of window lengths over the S-sensor stages of any tile: the
// window rows one pipeline stage must hold.
int stage_window(pat_bp_t h, int S) {
  if (S >= 1 && S <= 32 && h->wst_cache[S]) return h->wst_cache[S];
  int best = 8;
  for (int t = 0; t < h->n_tiles; ++t) {
    const uint16_t* len = h->win_len.data() + size_t(t) * h->ns;
    for (int s0 = 0; s0 < h->ns; s0 += S) {
      int sum = 0;
      for (int s = s0; s < std::min(h->ns, s0 + S); ++s) sum += len[s];
      best = std::max(best, sum);
    }
  }
  best = round_up(best, 8);
  if (S >= 1 && S <= 32) h->wst_cache[S] = best;
  return best;
}

// Stages and window-row budget of a launch shape under a shared-memory
// budget.  A stage takes as many of its (at most S) sensors as fit the row
// budget, so the budget must hold the longest single window (wmin) and never
// needs more than the longest S-sensor sum (wfull).  The deepest pipeline (6
// stages down to 3) whose row budget keeps at least half of wfull wins, else
// two stages with whatever fits above wmin.  False if even that does not fit.
bool fit_stages(GatherConfig& c, int wmin, int wfull, size_t budget, int* wst) {
  for (c.stages = 6; c.stages >= 2; --c.stages) {
    const size_t fixed = gather_smem_bytes(c, 0);       // everything but the window rows
    const size_t per_row = size_t(c.stages) * c.FB * 4;  // one more row in every stage
    if (fixed > budget) continue;
    int w = int(std::min<size_t>((budget - fixed) / per_row, size_t(wfull)));
    w &= ~7;
    const int need = c.stages > 2 ? std::max(wmin, wfull / 2) : wmin;
    if (w >= need) {
      *wst = std::max(w, 8);
      return true;
    }
  }
  c.stages = 2;
  *wst = wfull;
  return false;
}

// Launch shape under a shared-memory budget: stages and row budget as
// fit_stages decides; fewer sensors per stage if nothing fits.
GatherConfig config_for(pat_bp_t h, int FB, int S, size_t budget, int* wst) {
  GatherConfig c;
  c.P = h->P;
  c.SW = h->SW;
  c.delays = h->delays;
  c.wgt = h->wgt;
  c.n_sm = h->n_sm;
  c.FB = FB;
  c.S = S;
  const int wmin = stage_window(h, 1);
  for (;;) {
    if (fit_stages(c, wmin, stage_window(h, c.S), budget, wst) || c.S <= 4) break;
    c.S = c.S > 8 ? c.S - 8 : 4;
  }
  return c;
}

// Launch shape for a frame count: the autotuned one when the handle has it,
// else frames per unit by count, 16 (1 frame) or 8 sensors per stage and a
// shared-memory budget of three (1 frame) or two CTAs per SM.  When the stage windows are too
// long for that budget, the budget grows to the device limit and then fewer
// frames share a unit.  No choice here changes the summation order.
GatherConfig pick_config(pat_bp_t h, int n_frames, int fmt, int* wst) {
  const size_t limit = size_t(h->max_smem);
  if (n_frames < kStagedMinFrames && !(h->flags & PAT_FLAG_STAGED_SINGLE)) {
    // up to 3 frames: the unstaged kernels, one frame after the other (same
    // arithmetic and order as the staged kernel); units of 1 or 2 frames make
    // the staged kernel's window copies too small to pay (measured slower per
    // frame on the 3-D subject)
    GatherConfig c = config_for(h, 1, 16, 72 * 1024, wst);
    c.direct = 1;
    c.no_window = (h->flags & PAT_FLAG_NO_WINDOW) != 0;
    return c;
  }
  for (int FB = frames_per_group(n_frames); FB >= 1; FB /= 2) {
    const int fi = fb_index(FB);
    GatherConfig c;
    if (h->tuned_S[fi][fmt] > 0)
      c = config_for(h, FB, h->tuned_S[fi][fmt], size_t(h->tuned_budget_kb[fi][fmt]) * 1024, wst);
    else
      c = config_for(h, FB, FB == 1 ? 16 : 8, FB == 1 ? 72 * 1024 : 100 * 1024, wst);
    if (gather_smem_bytes(c, *wst) <= limit) return c;
    c = config_for(h, FB, 8, limit, wst);
    if (gather_smem_bytes(c, *wst) <= limit) return c;
  }
  return config_for(h, 1, 4, limit, wst);  // may not fit: the launch reports it
}

PreParams make_pre(pat_bp_t h, const void* sig, pat_dtype dtype, const float* scales, int n_frames,
                   int FB) {
  PreParams pp;
  pp.sig = sig;
  pp.scales = scales;
  pp.weights = h->d_w;
  pp.b = h->d_b;
  pp.m = h->d_m;
  pp.dtype = int(dtype);
  pp.fmt = fmt_for(dtype);
  pp.FB = FB;
  pp.n_sensors = h->ns;
  pp.n_sensors_pad = h->ns_pad;
  pp.n_t = h->nt;
  pp.n_t_pad = h->nt_pad;
  pp.n_frames = n_frames;
  return pp;
}

InstDesc make_desc(pat_bp_t h, float* out, int n_frames, int FB, int wst) {
  InstDesc d;
  std::memset(&d, 0, sizeof(d));
  d.u = h->d_u;
  d.anchor = h->d_anchor;
  d.pix = h->d_pix;
  d.wanchor = h->wgt ? h->d_wanchor : nullptr;
  d.base = h->d_base;
  d.slot = h->d_slot;
  d.zero_runs = h->d_zero_runs;
  d.n_zero_runs = h->n_zero_runs;
  d.b = h->d_b;
  d.m = h->d_m;
  d.out = out;
  d.part = h->d_part;
  d.counter = h->d_counter;
  d.out_stride = h->out_stride;
  d.unit_begin = 0;
  d.n_sensors = h->ns;
  d.n_sensors_pad = h->ns_pad;
  d.n_t_pad = h->nt_pad;
  d.n_tiles = h->n_tiles;
  d.n_frames = n_frames;
  d.n_fg = (n_frames + FB - 1) / FB;
  d.n_seg = h->n_seg;
  d.G = h->G;
  d.Wst = wst;
  d.W = h->W;
  return d;
}

int resident_ctas(const GatherConfig& c, int fmt, int wst, int n_sm) {
  // keyed by the current device too: devices of one process may differ in
  // multiprocessor count and shared memory
  struct Key {
    int dev, n_sm, P, FB, SW, S, stages, fmt, wst, delays, wgt, direct;
  };
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return 0;
  static std::mutex mu;
  static std::vector<std::pair<Key, int>> cache;
  std::lock_guard<std::mutex> lk(mu);
  for (auto& e : cache) {
    const Key& k = e.first;
    if (k.dev == dev && k.n_sm == n_sm && k.P == c.P && k.FB == c.FB && k.SW == c.SW &&
        k.S == c.S && k.stages == c.stages && k.fmt == fmt && k.wst == wst &&
        k.delays == c.delays && k.wgt == c.wgt && k.direct == c.direct)
      return e.second;
  }
  const int r = gather_resident_ctas(c, fmt, wst, n_sm);
  cache.push_back({Key{dev, n_sm, c.P, c.FB, c.SW, c.S, c.stages, fmt, wst, c.delays, c.wgt, c.direct}, r});
  return r;
}

}  // namespace patbp

namespace patbp {

// device bytes of the delay data: table offsets, or anchors and pixel terms
static size_t delay_bytes(pat_bp_t h) {
  const size_t wgt = h->wgt ? size_t(h->n_tiles) * h->ns_pad * 32 : 0;
  if (h->delays) return size_t(h->n_tiles) * h->ns_pad * 32 + size_t(h->n_tiles) * h->P * 16 + wgt;
  return size_t(h->n_tiles) * h->ns * h->P * 4 + (h->wgt ? size_t(h->n_tiles) * h->P * 16 : 0) + wgt;
}

size_t table_device_bytes(pat_bp_t h) {
  return delay_bytes(h) + size_t(h->n_tiles) * h->ns_pad * 4 +
         size_t(h->n_tiles) * h->P * 4 + std::max<size_t>(size_t(h->n_zero_runs) * 2, 1) * 4 +
         size_t(h->ns) * 4;
}

size_t resident_bytes(pat_bp_t h) {
  if (h->evicted) return 0;
  return table_device_bytes(h) + h->b_cap + h->m_cap + h->part_cap + h->counter_cap;
}

pat_status evict_locked(pat_bp_t h) {
  if (!h->mirror[0]) return fail(PAT_ERR_INVALID, "eviction needs PAT_FLAG_HOST_MIRROR");
  if (h->evicted) return PAT_OK;
  PAT_CUDA(cudaDeviceSynchronize());
  void** dev[12] = {reinterpret_cast<void**>(&h->d_u), reinterpret_cast<void**>(&h->d_anchor),
                    reinterpret_cast<void**>(&h->d_pix), reinterpret_cast<void**>(&h->d_wanchor),
                    reinterpret_cast<void**>(&h->d_base),
                    reinterpret_cast<void**>(&h->d_slot), reinterpret_cast<void**>(&h->d_zero_runs),
                    reinterpret_cast<void**>(&h->d_w), &h->d_b, reinterpret_cast<void**>(&h->d_m),
                    reinterpret_cast<void**>(&h->d_part), reinterpret_cast<void**>(&h->d_counter)};
  for (void** p : dev) {
    cudaFree(*p);
    *p = nullptr;
  }
  h->b_cap = h->m_cap = h->part_cap = h->counter_cap = 0;
  h->pre_frames = 0;
  h->evicted = true;
  return PAT_OK;
}

pat_status restore_locked(pat_bp_t h, cudaStream_t st) {
  if (!h->evicted) return PAT_OK;
  // buffers already present (handed over by donate_buffers_locked) are reused
  void** dev[pat_bp_s::kMirrors] = {
      h->delays ? reinterpret_cast<void**>(&h->d_anchor) : reinterpret_cast<void**>(&h->d_u),
      reinterpret_cast<void**>(&h->d_base), reinterpret_cast<void**>(&h->d_slot),
      reinterpret_cast<void**>(&h->d_zero_runs), reinterpret_cast<void**>(&h->d_w),
      reinterpret_cast<void**>(&h->d_pix), reinterpret_cast<void**>(&h->d_wanchor)};
  for (int i = 0; i < pat_bp_s::kMirrors; ++i) {
    if (!h->mirror[i]) continue;
    if (!*dev[i] && cudaMalloc(dev[i], h->mirror_bytes[i]) != cudaSuccess) {
      for (int j = 0; j <= i; ++j) {
        cudaFree(*dev[j]);
        *dev[j] = nullptr;
      }
      return fail(PAT_ERR_OOM, "table restore");
    }
    PAT_CUDA(cudaMemcpyAsync(*dev[i], h->mirror[i], h->mirror_bytes[i], cudaMemcpyHostToDevice, st));
  }
  h->evicted = false;
  return PAT_OK;
}

// Evict `from` (idle: none of its work in flight) by handing its device
// buffers to the evicted handle `to`, whose reload then fills them instead of
// allocating: no device synchronisation, no cudaFree, no cudaMalloc.  Only for
// handles whose table buffers have the same sizes (same layout kind); false
// (nothing changed) otherwise.
bool donate_buffers_locked(pat_bp_t from, pat_bp_t to) {
  if (from == to || from->evicted || !to->evicted || !from->mirror[0] || !to->mirror[0]) return false;
  if (from->delays != to->delays || from->wgt != to->wgt || from->device != to->device) return false;
  for (int i = 0; i < pat_bp_s::kMirrors; ++i)
    if (from->mirror_bytes[i] != to->mirror_bytes[i] || !from->mirror[i] != !to->mirror[i]) return false;
  void** src[pat_bp_s::kMirrors] = {
      from->delays ? reinterpret_cast<void**>(&from->d_anchor) : reinterpret_cast<void**>(&from->d_u),
      reinterpret_cast<void**>(&from->d_base), reinterpret_cast<void**>(&from->d_slot),
      reinterpret_cast<void**>(&from->d_zero_runs), reinterpret_cast<void**>(&from->d_w),
      reinterpret_cast<void**>(&from->d_pix), reinterpret_cast<void**>(&from->d_wanchor)};
  void** dst[pat_bp_s::kMirrors] = {
      to->delays ? reinterpret_cast<void**>(&to->d_anchor) : reinterpret_cast<void**>(&to->d_u),
      reinterpret_cast<void**>(&to->d_base), reinterpret_cast<void**>(&to->d_slot),
      reinterpret_cast<void**>(&to->d_zero_runs), reinterpret_cast<void**>(&to->d_w),
      reinterpret_cast<void**>(&to->d_pix), reinterpret_cast<void**>(&to->d_wanchor)};
  for (int i = 0; i < pat_bp_s::kMirrors; ++i) {
    if (!from->mirror[i]) continue;
    *dst[i] = *src[i];
    *src[i] = nullptr;
  }
  // working buffers: the counters must read zero, which they do between
  // launches (every launch returns them to zero)
  std::swap(to->d_b, from->d_b);
  std::swap(to->b_cap, from->b_cap);
  std::swap(to->d_m, from->d_m);
  std::swap(to->m_cap, from->m_cap);
  std::swap(to->d_part, from->d_part);
  std::swap(to->part_cap, from->part_cap);
  std::swap(to->d_counter, from->d_counter);
  std::swap(to->counter_cap, from->counter_cap);
  from->pre_frames = 0;
  from->evicted = true;
  return true;
}

}  // namespace patbp

extern "C" pat_status pat_bp_evict(pat_bp_t h) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  std::lock_guard<std::mutex> lk(h->mu);
  PAT_CUDA(cudaSetDevice(h->device));
  return evict_locked(h);
}

extern "C" pat_status pat_bp_restore(pat_bp_t h, pat_stream_t stream) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  std::lock_guard<std::mutex> lk(h->mu);
  PAT_CUDA(cudaSetDevice(h->device));
  return restore_locked(h, static_cast<cudaStream_t>(stream));
}

static pat_status ensure_buffers(pat_bp_t h, int n_frames) {
  return ensure_buffers_fb(h, n_frames, frames_per_group(n_frames));
}

extern "C" pat_status pat_bp_reserve(pat_bp_t h, int max_frames, pat_dtype dtype) {
  if (!h || max_frames < 1) return fail(PAT_ERR_INVALID, "bad handle or frame count");
  (void)dtype;
  std::lock_guard<std::mutex> lk(h->mu);
  PAT_CUDA(cudaSetDevice(h->device));
  return ensure_buffers(h, max_frames);
}

static pat_status preprocess_locked(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                                    const float* scales_dev, int n_frames, cudaStream_t stream) {
  if (h->evicted) return fail(PAT_ERR_INVALID, "the handle's table is evicted (pat_bp_restore)");
  if (!signals_dev) return fail(PAT_ERR_INVALID, "signals NULL");
  if (n_frames < 1 || n_frames > 65535) return fail(PAT_ERR_INVALID, "n_frames must be 1..65535");
  if (dtype != PAT_F32 && dtype != PAT_BF16 && dtype != PAT_F16)
    return fail(PAT_ERR_INVALID, "unknown dtype");
  if (dtype != PAT_F32 && !scales_dev) return fail(PAT_ERR_INVALID, "16-bit signals need scales");
  int wst = 0;
  const int FB = pick_config(h, n_frames, fmt_for(dtype), &wst).FB;
  pat_status st = ensure_buffers_fb(h, n_frames, FB);
  if (st != PAT_OK) return st;
  const PreParams pp = make_pre(h, signals_dev, dtype, scales_dev, n_frames, FB);
  cudaError_t e = launch_preprocess(pp, stream);
  if (e != cudaSuccess) return cuda_fail(e, "preprocess launch");
  h->pre_frames = n_frames;
  h->pre_fmt = pp.fmt;
  h->pre_fb = pp.FB;
  return PAT_OK;
}

static pat_status gather_locked(pat_bp_t h, int n_frames, float* out_dev, cudaStream_t stream,
                                int* host_status = nullptr, bool* exported = nullptr) {
  if (!out_dev) return fail(PAT_ERR_INVALID, "out NULL");
  if (n_frames < 1 || n_frames != h->pre_frames)
    return fail(PAT_ERR_INVALID, "gather needs the preprocess of the same n_frames first");
  int wst = 0;
  const GatherConfig c = pick_config(h, n_frames, h->pre_fmt, &wst);
  if (c.FB != h->pre_fb) return fail(PAT_ERR_INVALID, "frame grouping changed since preprocess");
  StreamParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.inst[0] = make_desc(h, out_dev, n_frames, c.FB, wst);
  const InstDesc& d = sp.inst[0];
  sp.n_inst = 1;
  sp.n_units = int64_t(d.n_fg) * d.n_tiles * d.n_seg;
  sp.S = c.S;
  sp.stages = c.stages;
  sp.Wst = wst;
  sp.status = h->d_status;
  sp.host_status = c.direct ? host_status : nullptr;
  if (exported) *exported = c.direct && host_status;
  sp.sched = h->d_sched;
  sp.timeout_ns = 2000000000ull;
  const int res = resident_ctas(c, h->pre_fmt, wst, h->n_sm);
  if (res <= 0) return fail(PAT_ERR_CUDA, "gather kernel does not fit on the device");
  const int grid = int(std::min<int64_t>(sp.n_units, res));
  cudaError_t e = launch_gather(c, h->pre_fmt, sp, grid, stream);
  if (e != cudaSuccess) return cuda_fail(e, "gather launch");
  return PAT_OK;
}

pat_status patbp::reconstruct_locked(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                                      const float* scales_dev, int n_frames, float* out_dev,
                                      cudaStream_t stream, int* host_status, bool* exported) {
  if (!out_dev) return fail(PAT_ERR_INVALID, "out NULL");
  if (exported) *exported = false;
  pat_status st = preprocess_locked(h, signals_dev, dtype, scales_dev, n_frames, stream);
  if (st != PAT_OK) return st;
  return gather_locked(h, n_frames, out_dev, stream, host_status, exported);
}

extern "C" pat_status pat_bp_preprocess(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                                        const float* scales_dev, int n_frames,
                                        pat_stream_t stream) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  std::lock_guard<std::mutex> lk(h->mu);
  PAT_CUDA(cudaSetDevice(h->device));
  return preprocess_locked(h, signals_dev, dtype, scales_dev, n_frames,
                           static_cast<cudaStream_t>(stream));
}

extern "C" pat_status pat_bp_gather(pat_bp_t h, int n_frames, float* out_dev, pat_stream_t stream) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  std::lock_guard<std::mutex> lk(h->mu);
  PAT_CUDA(cudaSetDevice(h->device));
  return gather_locked(h, n_frames, out_dev, static_cast<cudaStream_t>(stream));
}

extern "C" pat_status pat_bp_reconstruct(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                                         const float* scales_dev, int n_frames, float* out_dev,
                                         pat_stream_t stream) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  std::lock_guard<std::mutex> lk(h->mu);
  PAT_CUDA(cudaSetDevice(h->device));
  return reconstruct_locked(h, signals_dev, dtype, scales_dev, n_frames, out_dev,
                            static_cast<cudaStream_t>(stream));
}

static pat_status grow(void** p, size_t* cap, size_t need, const char* what) {
  if (need <= *cap) return PAT_OK;
  cudaFree(*p);
  *p = nullptr;
  *cap = 0;
  if (cudaMalloc(p, need) != cudaSuccess) return fail(PAT_ERR_OOM, what);
  *cap = need;
  return PAT_OK;
}

// Device address of a host pointer that the device can access in place
// (page-locked memory), or nullptr.
static void* device_address(const void* host_ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, host_ptr) != cudaSuccess) {
    cudaGetLastError();  // not a CUDA-known pointer: clear the error, stage the buffer
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

extern "C" pat_status pat_bp_reconstruct_host(pat_bp_t h, const void* signals_host, pat_dtype dtype,
                                              const float* scales_host, int n_frames,
                                              float* out_host) {
  if (!h || !signals_host || !out_host) return fail(PAT_ERR_INVALID, "NULL argument");
  if (n_frames < 1) return fail(PAT_ERR_INVALID, "n_frames < 1");
  std::lock_guard<std::mutex> lk(h->mu);
  PAT_CUDA(cudaSetDevice(h->device));
  if (!h->own_stream) PAT_CUDA(cudaStreamCreateWithFlags(&h->own_stream, cudaStreamNonBlocking));
  const size_t esz = dtype == PAT_F32 ? 4 : 2;
  const size_t sig_bytes = size_t(n_frames) * h->ns * h->nt * esz;
  const size_t sc_bytes = size_t(n_frames) * h->ns * sizeof(float);
  const size_t out_bytes = size_t(n_frames) * h->out_stride * sizeof(float);
  pat_status st;
  cudaStream_t s = h->own_stream;
  // Page-locked host buffers are addressable by the device (over NVLink-C2C on
  // a Grace host): the preprocessing kernel then reads the signals and scales
  // in place and the last kernel writes the image in place -- no staging
  // copies.  Pageable buffers go through device staging buffers.
  const void* sig_dev = device_address(signals_host);
  const float* sc_dev = scales_host ? static_cast<const float*>(device_address(scales_host)) : nullptr;
  float* out_dev = static_cast<float*>(device_address(out_host));
  if (!sig_dev) {
    if ((st = grow(&h->d_sig, &h->sig_cap, sig_bytes, "signal staging")) != PAT_OK) return st;
    PAT_CUDA(cudaMemcpyAsync(h->d_sig, signals_host, sig_bytes, cudaMemcpyHostToDevice, s));
    sig_dev = h->d_sig;
  }
  if (scales_host && !sc_dev) {
    if ((st = grow(reinterpret_cast<void**>(&h->d_scales), &h->scales_cap, sc_bytes, "scales")) != PAT_OK)
      return st;
    PAT_CUDA(cudaMemcpyAsync(h->d_scales, scales_host, sc_bytes, cudaMemcpyHostToDevice, s));
    sc_dev = h->d_scales;
  }
  const bool out_staged = out_dev == nullptr;
  if (out_staged) {
    if ((st = grow(reinterpret_cast<void**>(&h->d_out), &h->out_cap, out_bytes, "output staging")) != PAT_OK)
      return st;
    out_dev = h->d_out;
  }
  if (!h->host_status) {
    if (cudaHostAlloc(&h->host_status, sizeof(int), cudaHostAllocMapped) != cudaSuccess) {
      h->host_status = nullptr;
      return fail(PAT_ERR_OOM, "host status word");
    }
    PAT_CUDA(cudaHostGetDevicePointer(reinterpret_cast<void**>(&h->host_status_dev), h->host_status, 0));
  }
  *reinterpret_cast<volatile int*>(h->host_status) = 0;
  bool exported = false;
  st = reconstruct_locked(h, sig_dev, dtype, sc_dev, n_frames, out_dev, s, h->host_status_dev, &exported);
  if (st != PAT_OK) return st;
  if (out_staged) PAT_CUDA(cudaMemcpyAsync(out_host, out_dev, out_bytes, cudaMemcpyDeviceToHost, s));
  if (!exported) PAT_CUDA(launch_status_export(h->d_status, h->host_status_dev, s));
  PAT_CUDA(cudaStreamSynchronize(s));
  const int flag = *reinterpret_cast<volatile int*>(h->host_status);
  if (flag) {
    cudaMemset(h->d_status, 0, sizeof(int));
    if (h->d_counter) cudaMemset(h->d_counter, 0, h->counter_cap);
    cudaMemset(h->d_sched, 0, 4 * sizeof(unsigned));
    return fail(flag & kStatusTimeout ? PAT_ERR_TIMEOUT : PAT_ERR_CUDA,
                flag & kStatusTimeout ? "a device wait ran out of time" : "bad launch configuration");
  }
  return PAT_OK;
}

extern "C" pat_status pat_bp_sync(pat_bp_t h, pat_stream_t stream) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  PAT_CUDA(cudaSetDevice(h->device));
  PAT_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int flag = 0;
  PAT_CUDA(cudaMemcpy(&flag, h->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (flag) {
    PAT_CUDA(cudaMemset(h->d_status, 0, sizeof(int)));
    // an aborted launch can leave counters part-way: start clean
    if (h->d_counter) PAT_CUDA(cudaMemset(h->d_counter, 0, h->counter_cap));
    PAT_CUDA(cudaMemset(h->d_sched, 0, 4 * sizeof(unsigned)));
    return fail(flag & kStatusTimeout ? PAT_ERR_TIMEOUT : PAT_ERR_CUDA,
                flag & kStatusTimeout ? "a device wait ran out of time" : "bad launch configuration");
  }
  return PAT_OK;
}

extern "C" pat_status pat_bp_info(pat_bp_t h, pat_bp_info_t* info) {
  if (!h || !info) return fail(PAT_ERR_INVALID, "NULL argument");
  info->n_pix = h->n_pix;
  info->grid_total = h->grid_total;
  info->n_sensors = h->ns;
  info->n_samples = h->nt;
  info->n_samples_pad = h->nt_pad;
  info->tile_pix = h->P;
  info->n_tiles = h->n_tiles;
  info->window = h->W;
  info->split = h->n_seg;
  info->sensor_warps = h->SW;
  info->table_bytes = int64_t(delay_bytes(h));
  info->build_seconds = h->build_seconds;
  info->delays = h->delays;
  info->c0 = h->c0;
  info->solid_angle = h->wgt;
  info->gpu_table = (h->flags & PAT_FLAG_GPU_TABLE) != 0 && !h->delays;
  return PAT_OK;
}

extern "C" pat_status pat_bp_table(pat_bp_t h, float* u_host, int32_t* base_host, int32_t* pix_host) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  PAT_CUDA(cudaSetDevice(h->device));
  const size_t n = size_t(h->n_tiles) * h->ns;
  if (u_host && h->delays)
    return fail(PAT_ERR_INVALID, "a constant-speed handle stores no travel-time table");
  if (u_host) PAT_CUDA(cudaMemcpy(u_host, h->d_u, n * h->P * 4, cudaMemcpyDeviceToHost));
  if (base_host) {
    std::vector<int32_t> packed(size_t(h->n_tiles) * h->ns_pad);
    PAT_CUDA(cudaMemcpy(packed.data(), h->d_base, packed.size() * 4, cudaMemcpyDeviceToHost));
    for (int t = 0; t < h->n_tiles; ++t)
      for (int s = 0; s < h->ns; ++s)
        base_host[size_t(t) * h->ns + s] = packed[size_t(t) * h->ns_pad + s] & 0xffff;
  }
  if (pix_host) PAT_CUDA(cudaMemcpy(pix_host, h->d_slot, size_t(h->n_tiles) * h->P * 4, cudaMemcpyDeviceToHost));
  return PAT_OK;
}

extern "C" pat_status pat_bp_destroy(pat_bp_t h) {
  if (!h) return PAT_OK;
  cudaSetDevice(h->device);
  cudaDeviceSynchronize();
  free_handle(h);
  return PAT_OK;
}

extern "C" pat_status pat_fmm_host(const float* speed_host, const pat_grid* grid, const double* src_xyz,
                                   int order, double* T_out) {
  if (!speed_host || !src_xyz || !T_out) return fail(PAT_ERR_INVALID, "NULL argument");
  if (order != 1 && order != 2) return fail(PAT_ERR_INVALID, "order must be 1 or 2");
  GridDesc g;
  std::string err;
  if (!grid_from_abi(grid, g, err)) return fail(PAT_ERR_INVALID, err);
  for (int64_t v = 0; v < g.total(); ++v)
    if (!(speed_host[v] > 0.0f)) return fail(PAT_ERR_INVALID, "speed must be > 0");
  FastMarcher fm(g, speed_host, nullptr, order);
  std::vector<double> T;
  if (!fm.solve(src_xyz, T, std::numeric_limits<double>::infinity(), 0))
    return fail(PAT_ERR_INVALID, "source outside the grid");
  std::memcpy(T_out, T.data(), T.size() * sizeof(double));
  return PAT_OK;
}

extern "C" pat_status pat_fmm_gpu(const float* speed_host, const pat_grid* grid, const double* src_xyz,
                                  int n_src, double* T_out) {
  if (!speed_host || !src_xyz || !T_out) return fail(PAT_ERR_INVALID, "NULL argument");
  if (n_src < 1) return fail(PAT_ERR_INVALID, "n_src must be >= 1");
  GridDesc g;
  std::string err;
  if (!grid_from_abi(grid, g, err)) return fail(PAT_ERR_INVALID, err);
  if (g.total() > INT32_MAX) return fail(PAT_ERR_INVALID, "grid too large");
  for (int64_t v = 0; v < g.total(); ++v)
    if (!(speed_host[v] > 0.0f) || !std::isfinite(speed_host[v]))
      return fail(PAT_ERR_INVALID, "speed must be finite and > 0");
  for (int s = 0; s < n_src; ++s) {
    int64_t node[8];
    double dist[8];
    if (source_corners(g, src_xyz + 3 * size_t(s), node, dist) == 0)
      return fail(PAT_ERR_INVALID, "source " + std::to_string(s) + " outside the grid");
  }
  std::vector<int32_t> all(size_t(g.total()));
  for (int64_t v = 0; v < g.total(); ++v) all[v] = int32_t(v);
  const int batch = std::min(n_src, gpu_eikonal_batch(g, g.total(), size_t(8) << 30));
  GpuEikonal* e = gpu_eikonal_create(g, speed_host, all, batch, err);
  if (!e) return fail(PAT_ERR_CUDA, err);
  for (int s0 = 0; s0 < n_src; s0 += batch) {
    const int nb = std::min(batch, n_src - s0);
    if (!gpu_eikonal_slot_times(e, src_xyz + 3 * size_t(s0), nb, std::numeric_limits<double>::infinity(),
                                T_out + size_t(s0) * g.total(), err)) {
      gpu_eikonal_destroy(e);
      return fail(PAT_ERR_CUDA, err);
    }
  }
  gpu_eikonal_destroy(e);
  return PAT_OK;
}

extern "C" pat_status pat_table_host(const float* speed_host, const pat_grid* grid,
                                     const double* sensors_host, int n_sensors,
                                     const uint8_t* mask_host, double dt, int n_samples,
                                     unsigned flags, pat_bp_info_t* info, float* u_host,
                                     int32_t* base_host, int32_t* slot_host) {
  if (!speed_host || !sensors_host || !info) return fail(PAT_ERR_INVALID, "NULL argument");
  if (n_sensors < 1 || !(dt > 0.0) || n_samples < 2 || n_samples > 32768)
    return fail(PAT_ERR_INVALID, "bad sizes");
  GridDesc g;
  std::string err;
  if (!grid_from_abi(grid, g, err)) return fail(PAT_ERR_INVALID, err);
  const bool compact = (flags & PAT_FLAG_COMPACT_OUT) != 0;
  const int P = (flags & PAT_FLAG_TILE_256) ? 256 : 128;
  HostTable tab;
  if (!build_table(speed_host, g, sensors_host, n_sensors, mask_host, dt, n_samples, P, compact, tab,
                   err, (flags & PAT_FLAG_FMM_SECOND_ORDER) ? 2 : 1, (flags & PAT_FLAG_GPU_TABLE) != 0))
    return fail(PAT_ERR_INVALID, err);
  std::memset(info, 0, sizeof(*info));
  info->n_pix = tab.n_pix;
  info->grid_total = g.total();
  info->n_sensors = n_sensors;
  info->n_samples = n_samples;
  info->n_samples_pad = round_up(n_samples + 1, 8);
  info->tile_pix = P;
  info->n_tiles = tab.n_tiles;
  info->window = tab.W;
  info->table_bytes = int64_t(tab.u.size()) * 4;
  info->build_seconds = tab.build_seconds;
  info->gpu_table = (flags & PAT_FLAG_GPU_TABLE) != 0;
  if (u_host) std::memcpy(u_host, tab.u.data(), tab.u.size() * 4);
  if (base_host) std::memcpy(base_host, tab.base.data(), tab.base.size() * 4);
  if (slot_host) {
    const std::vector<int32_t>& sl = compact ? tab.slot_compact : tab.slot_dense;
    std::memcpy(slot_host, sl.data(), sl.size() * 4);
  }
  return PAT_OK;
}

extern "C" pat_status pat_test_gather_only(pat_bp_t h, pat_stream_t stream) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  std::lock_guard<std::mutex> lk(h->mu);
  PAT_CUDA(cudaSetDevice(h->device));
  if (h->pre_frames != 1) return fail(PAT_ERR_INVALID, "needs the preprocess of one frame first");
  int wst = 0;
  const GatherConfig c = pick_config(h, 1, h->pre_fmt, &wst);
  if (!c.direct || c.FB != h->pre_fb) return fail(PAT_ERR_INVALID, "the frame does not take the unstaged gather");
  const InstDesc d = make_desc(h, nullptr, 1, 1, wst);
  cudaError_t e = launch_gather_direct(c, h->pre_fmt, d, h->n_sm, h->d_status, nullptr, 2000000000ull,
                                       static_cast<cudaStream_t>(stream), false);
  if (e != cudaSuccess) return cuda_fail(e, "gather launch");
  return PAT_OK;
}

extern "C" pat_status pat_test_wait_timeout(uint64_t timeout_ns) {
  int* d = nullptr;
  PAT_CUDA(cudaMalloc(&d, sizeof(int)));
  cudaMemset(d, 0, sizeof(int));
  cudaError_t e = launch_wait_probe(d, timeout_ns, nullptr);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int flag = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&flag, d, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "wait probe");
  return flag ? PAT_ERR_TIMEOUT : PAT_OK;
}
