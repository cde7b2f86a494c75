// plan.cu -- many instances in persistent launches (include/pat_bp.h, plans).
//
// Every instance (one speed map's table, Sec. III) contributes its units of
// work to a persistent gather launch.  Instances are grouped by the frames
// that share one pass over a table tile (FB: the largest power of two up to
// 8 not above the instance's frame count), and every group ("class") has its
// own preprocessing launch (the Eq. (BP) integrand of all its instances) and
// its own gather launch; all preprocessing launches go first, then the
// gathers.  A 16-frame instance therefore streams its table twice, while a
// single-frame instance next to it does not pay for frames it does not have.
// A plan can replay the launches as a CUDA graph whose kernel-node parameters
// are refreshed per execution, and can time candidate launch shapes once
// (autotuning).  None of the shape choices changes the order in which a
// pixel's sensor terms are summed, so results never depend on the shape, the
// classes, the graph or the other instances.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "handle.h"

using namespace patbp;

namespace {

// Instances of a plan that share frames per unit: one preprocessing and one
// gather launch.
struct PlanClass {
  int FB = 1;
  std::vector<int> idx;  // the plan's instance indices, in plan order
  GatherConfig cfg;
  int wst = 8;
  int grid = 0;
  int64_t n_units = 0;
  std::unique_ptr<PreMultiParams> pre;
  std::unique_ptr<StreamParams> gat;
  cudaGraphNode_t pre_node = nullptr, gat_node = nullptr;
};

}  // namespace

struct pat_plan_s {
  std::vector<pat_bp_t> hs;
  std::vector<int> frames;
  pat_dtype dtype = PAT_F32;
  int fmt = 0;
  unsigned flags = 0;
  int device = 0, n_sm = 0, P = 128, SW = 4;
  int fb_uniform = 0;  // 0: each instance's own frames per unit; else this for all
  // launch shape shared by the classes
  int S = 16, budget_kb = 55;
  std::vector<PlanClass> cls;
  int64_t n_units = 0;
  bool tuned = false;
  double tune_ms = 0.0;
  // device words owned by the plan (the gathers run one after the other and
  // share them: the unit tickets return to zero at the end of every launch)
  int* d_status = nullptr;
  unsigned* d_sched = nullptr;
  // graph
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  std::mutex mu;
};

namespace {

int instance_fb(pat_plan_t pl, int i) {
  return pl->fb_uniform ? pl->fb_uniform : frames_per_group(pl->frames[i]);
}

// Classes and launch shapes for S sensors per stage under a shared-memory
// budget of budget_kb per CTA.
pat_status plan_shape(pat_plan_t pl, int S, int budget_kb) {
  pl->S = S;
  pl->budget_kb = budget_kb;
  std::vector<int> fbs;
  for (size_t i = 0; i < pl->hs.size(); ++i) fbs.push_back(instance_fb(pl, int(i)));
  std::vector<int> order(fbs);
  std::sort(order.begin(), order.end(), std::greater<int>());
  order.erase(std::unique(order.begin(), order.end()), order.end());
  std::vector<PlanClass> cls(order.size());
  for (size_t c = 0; c < order.size(); ++c) {
    cls[c].FB = order[c];
    for (size_t i = 0; i < pl->hs.size(); ++i)
      if (fbs[i] == order[c]) cls[c].idx.push_back(int(i));
  }
  const size_t budget = std::min(size_t(budget_kb) * 1024, size_t(pl->hs[0]->max_smem));
  int64_t total_units = 0;
  for (PlanClass& k : cls) {
    // one shape per class: the longest single window and the longest
    // S-sensor window sum of its instances bound the stages' row budget
    int wmin = 8, wfull = 8;
    for (int i : k.idx) {
      wmin = std::max(wmin, stage_window(pl->hs[i], 1));
      wfull = std::max(wfull, stage_window(pl->hs[i], S));
    }
    GatherConfig c;
    c.P = pl->P;
    c.SW = pl->SW;
    c.delays = pl->hs[0]->delays;
    c.wgt = pl->hs[0]->wgt;
    c.FB = k.FB;
    c.S = S;
    int wst = wfull;
    if (!fit_stages(c, wmin, wfull, budget, &wst))
      return fail(PAT_ERR_CUDA, "stage windows do not fit in shared memory for this shape");
    k.cfg = c;
    k.wst = wst;
    for (int i : k.idx) {
      pat_status st = ensure_buffers_fb(pl->hs[i], pl->frames[i], k.FB);
      if (st != PAT_OK) return st;
    }
    k.pre.reset(new (std::nothrow) PreMultiParams());
    k.gat.reset(new (std::nothrow) StreamParams());
    if (!k.pre || !k.gat) return fail(PAT_ERR_OOM, "plan parameters");
    StreamParams& sp = *k.gat;
    PreMultiParams& pm = *k.pre;
    std::memset(&sp, 0, sizeof(sp));
    std::memset(&pm, 0, sizeof(pm));
    int64_t units = 0, ctas = 0;
    for (size_t j = 0; j < k.idx.size(); ++j) {
      pat_bp_t h = pl->hs[k.idx[j]];
      const int F = pl->frames[k.idx[j]];
      sp.inst[j] = make_desc(h, nullptr, F, k.FB, wst);
      sp.inst[j].unit_begin = units;
      units += int64_t(sp.inst[j].n_fg) * sp.inst[j].n_tiles * sp.inst[j].n_seg;
      pm.inst[j] = make_pre(h, nullptr, pl->dtype, nullptr, F, k.FB);
      pm.cta_begin[j] = ctas;
      ctas += int64_t(h->ns) * sp.inst[j].n_fg;
    }
    if (ctas > 0x7fffffff) return fail(PAT_ERR_INVALID, "too many preprocessing rows in one plan");
    pm.cta_begin[k.idx.size()] = ctas;
    pm.n_inst = int(k.idx.size());
    pm.dtype = int(pl->dtype);
    pm.fmt = pl->fmt;
    pm.FB = k.FB;
    sp.n_inst = int(k.idx.size());
    sp.n_units = units;
    sp.S = c.S;
    sp.stages = c.stages;
    sp.Wst = wst;
    sp.status = pl->d_status;
    sp.sched = pl->d_sched;
    sp.timeout_ns = 2000000000ull;
    k.n_units = units;
    total_units += units;
    const int res = resident_ctas(c, pl->fmt, wst, pl->n_sm);
    if (res <= 0) return fail(PAT_ERR_CUDA, "gather kernel does not fit on the device");
    k.grid = int(std::min<int64_t>(std::max<int64_t>(units, 1), res));
  }
  pl->cls = std::move(cls);
  pl->n_units = total_units;
  return PAT_OK;
}

void fill_pointers(pat_plan_t pl, const void* const* sig, const float* const* scales,
                   float* const* outs) {
  for (PlanClass& k : pl->cls)
    for (size_t j = 0; j < k.idx.size(); ++j) {
      const int i = k.idx[j];
      k.pre->inst[j].sig = sig[i];
      k.pre->inst[j].scales = scales ? scales[i] : nullptr;
      k.gat->inst[j].out = outs[i];
    }
}

// All preprocessing launches, then all gathers.  A gather is a programmatic
// dependent of the launch before it; the first waits for the last
// preprocessing grid, whose stream predecessors (the other preprocessing
// grids) are complete by then, and every later gather starts after the
// gather before it has finished.
pat_status launch_all(pat_plan_t pl, cudaStream_t st) {
  for (PlanClass& k : pl->cls) {
    if (k.n_units == 0) continue;
    cudaError_t e = launch_preprocess_multi(*k.pre, st);
    if (e != cudaSuccess) return cuda_fail(e, "preprocess launch");
  }
  for (PlanClass& k : pl->cls) {
    if (k.n_units == 0) continue;
    cudaError_t e = launch_gather(k.cfg, pl->fmt, *k.gat, k.grid, st);
    if (e != cudaSuccess) return cuda_fail(e, "gather launch");
  }
  return PAT_OK;
}

void drop_graph(pat_plan_t pl) {
  if (pl->exec) cudaGraphExecDestroy(pl->exec);
  if (pl->graph) cudaGraphDestroy(pl->graph);
  pl->exec = nullptr;
  pl->graph = nullptr;
  for (PlanClass& k : pl->cls) k.pre_node = k.gat_node = nullptr;
}

// Point every descriptor at the handles' current buffers: a handle's own
// calls may have grown its working buffers since the plan was shaped, and an
// eviction and restore reallocates its table, so every handle-owned pointer
// is taken again.  A handle whose kernel mode changed since (solid-angle
// weights set) no longer fits the plan's launch shape.
pat_status refresh_buffers(pat_plan_t pl) {
  for (PlanClass& k : pl->cls)
    for (size_t j = 0; j < k.idx.size(); ++j) {
      const int i = k.idx[j];
      pat_bp_t h = pl->hs[i];
      if (h->evicted) return fail(PAT_ERR_INVALID, "a plan handle's table is evicted");
      if (h->wgt != k.cfg.wgt || h->delays != k.cfg.delays)
        return fail(PAT_ERR_INVALID, "a plan handle changed its weights since the plan was made");
      pat_status st = ensure_buffers_fb(h, pl->frames[i], k.FB);
      if (st != PAT_OK) return st;
      k.pre->inst[j].weights = h->d_w;
      k.pre->inst[j].b = h->d_b;
      k.pre->inst[j].m = h->d_m;
      InstDesc& d = k.gat->inst[j];
      d.u = h->d_u;
      d.anchor = h->d_anchor;
      d.pix = h->d_pix;
      d.wanchor = h->wgt ? h->d_wanchor : nullptr;
      d.base = h->d_base;
      d.slot = h->d_slot;
      d.zero_runs = h->d_zero_runs;
      d.b = h->d_b;
      d.m = h->d_m;
      d.part = h->d_part;
      d.counter = h->d_counter;
    }
  return PAT_OK;
}

// Capture the launches once; the graph's kernel nodes are told apart by their
// parameter blocks (two classes can share a kernel), which equal the classes'
// blocks at capture time.
pat_status capture(pat_plan_t pl) {
  if (!pl->cap_stream) PAT_CUDA(cudaStreamCreateWithFlags(&pl->cap_stream, cudaStreamNonBlocking));
  PAT_CUDA(cudaStreamBeginCapture(pl->cap_stream, cudaStreamCaptureModeThreadLocal));
  pat_status st = launch_all(pl, pl->cap_stream);
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamEndCapture(pl->cap_stream, &g);
  if (st != PAT_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "graph capture");
  size_t n = 0;
  PAT_CUDA(cudaGraphGetNodes(g, nullptr, &n));
  std::vector<cudaGraphNode_t> nodes(n);
  PAT_CUDA(cudaGraphGetNodes(g, nodes.data(), &n));
  for (cudaGraphNode_t nd : nodes) {
    cudaGraphNodeType t;
    PAT_CUDA(cudaGraphNodeGetType(nd, &t));
    if (t != cudaGraphNodeTypeKernel) continue;
    cudaKernelNodeParams kp;
    PAT_CUDA(cudaGraphKernelNodeGetParams(nd, &kp));
    if (!kp.kernelParams || !kp.kernelParams[0]) continue;
    for (PlanClass& k : pl->cls) {
      if (kp.func == preprocess_multi_func(int(pl->dtype), pl->fmt, k.FB) &&
          std::memcmp(kp.kernelParams[0], k.pre.get(), sizeof(PreMultiParams)) == 0)
        k.pre_node = nd;
      if (kp.func == gather_kernel_func(k.cfg, pl->fmt) &&
          std::memcmp(kp.kernelParams[0], k.gat.get(), sizeof(StreamParams)) == 0)
        k.gat_node = nd;
    }
  }
  for (PlanClass& k : pl->cls)
    if (k.n_units > 0 && (!k.pre_node || !k.gat_node)) {
      cudaGraphDestroy(g);
      for (PlanClass& c : pl->cls) c.pre_node = c.gat_node = nullptr;
      return fail(PAT_ERR_CUDA, "captured graph lacks the expected kernels");
    }
  pl->graph = g;
  PAT_CUDA(cudaGraphInstantiate(&pl->exec, g, 0));
  return PAT_OK;
}

pat_status refresh_graph(pat_plan_t pl) {
  for (PlanClass& k : pl->cls) {
    if (k.n_units == 0) continue;
    void* pre_args[1] = {k.pre.get()};
    void* gat_args[1] = {k.gat.get()};
    cudaKernelNodeParams kp;
    PAT_CUDA(cudaGraphKernelNodeGetParams(k.pre_node, &kp));
    kp.kernelParams = pre_args;
    kp.extra = nullptr;
    PAT_CUDA(cudaGraphExecKernelNodeSetParams(pl->exec, k.pre_node, &kp));
    PAT_CUDA(cudaGraphKernelNodeGetParams(k.gat_node, &kp));
    kp.kernelParams = gat_args;
    kp.extra = nullptr;
    PAT_CUDA(cudaGraphExecKernelNodeSetParams(pl->exec, k.gat_node, &kp));
  }
  return PAT_OK;
}

// Shapes chosen earlier in this process (and, with PAT_TUNE_CACHE set, in a
// text file of "signature S budget_kb" lines), keyed by the plan's shape.
std::mutex g_tune_mu;
std::map<std::string, std::vector<int>> g_tune;

std::string signature(pat_plan_t pl) {
  std::string s = "sm" + std::to_string(pl->n_sm) + ".dt" + std::to_string(int(pl->dtype)) +
                  ".fb" + std::to_string(pl->fb_uniform) + ".w" + std::to_string(pl->hs[0]->wgt) +
                  ".d" + std::to_string(pl->hs[0]->delays);
  for (size_t i = 0; i < pl->hs.size(); ++i) {
    pat_bp_t h = pl->hs[i];
    s += "|" + std::to_string(h->ns) + "x" + std::to_string(h->nt) + "x" + std::to_string(h->n_tiles) +
         "x" + std::to_string(h->W) + "f" + std::to_string(pl->frames[i]);
  }
  return s;
}

void tune_file_load() {
  static bool loaded = false;
  if (loaded) return;
  loaded = true;
  const char* path = std::getenv("PAT_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "r");
  if (!f) return;
  char key[4096];
  int s, b;
  while (std::fscanf(f, "%4095s %d %d", key, &s, &b) == 3) g_tune[key] = {s, b};
  std::fclose(f);
}

void tune_file_store(const std::string& key, int s, int b) {
  const char* path = std::getenv("PAT_TUNE_CACHE");
  if (!path) return;
  FILE* f = std::fopen(path, "a");
  if (!f) return;
  std::fprintf(f, "%s %d %d\n", key.c_str(), s, b);
  std::fclose(f);
}

// Times every candidate shape (sensors per stage x shared-memory budget) on
// the given inputs and keeps the fastest; the frames per unit of every
// instance follow from its frame count.
pat_status autotune(pat_plan_t pl, const void* const* sig, const float* const* scales,
                    float* const* outs, cudaStream_t st) {
  const std::string key = signature(pl);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    tune_file_load();
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      pat_status s = plan_shape(pl, it->second[0], it->second[1]);
      if (s == PAT_OK) pl->tuned = true;
      return s;
    }
  }
  const int Ss[4] = {4, 8, 16, 32};
  const int budgets[4] = {55, 72, 110, pl->hs[0]->max_smem / 1024};
  cudaEvent_t e0, e1;
  PAT_CUDA(cudaEventCreate(&e0));
  PAT_CUDA(cudaEventCreate(&e1));
  double best = 1e30;
  int bs = pl->S, bb = pl->budget_kb;
  pat_status st_all = PAT_OK;
  for (int S : Ss)
    for (int b : budgets) {
      if (S == 4 && b != budgets[3]) continue;  // 4 sensors per stage only as a last resort
      pat_status s = plan_shape(pl, S, b);
      if (s != PAT_OK) continue;
      if ((s = refresh_buffers(pl)) != PAT_OK) {
        st_all = s;
        continue;
      }
      fill_pointers(pl, sig, scales, outs);
      if (launch_all(pl, st) != PAT_OK) continue;  // warm-up
      float ms = 1e30f;
      for (int rep = 0; rep < 3; ++rep) {  // best of three
        cudaEventRecord(e0, st);
        if (launch_all(pl, st) != PAT_OK) break;
        cudaEventRecord(e1, st);
        if (cudaEventSynchronize(e1) != cudaSuccess) {
          cudaEventDestroy(e0);
          cudaEventDestroy(e1);
          return cuda_fail(cudaGetLastError(), "autotune run");
        }
        float t = 0.0f;
        cudaEventElapsedTime(&t, e0, e1);
        ms = std::min(ms, t);
      }
      if (ms < best) {
        best = ms;
        bs = S;
        bb = b;
      }
    }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best >= 1e30) return st_all != PAT_OK ? st_all : fail(PAT_ERR_CUDA, "no launch shape ran");
  pat_status s = plan_shape(pl, bs, bb);
  if (s != PAT_OK) return s;
  pl->tuned = true;
  pl->tune_ms = best;
  std::lock_guard<std::mutex> lk(g_tune_mu);
  g_tune[key] = {bs, bb};
  tune_file_store(key, bs, bb);
  return PAT_OK;
}

}  // namespace

static pat_status plan_new(const pat_bp_t* handles, const int* n_frames, int n, pat_dtype dtype,
                           unsigned flags, bool own_words, int fb_uniform, pat_plan_t* out) {
  if (!out) return fail(PAT_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (!handles || !n_frames || n < 1 || n > kMaxInst)
    return fail(PAT_ERR_INVALID, "a plan holds 1..64 handles");
  if (dtype != PAT_F32 && dtype != PAT_BF16 && dtype != PAT_F16) return fail(PAT_ERR_INVALID, "dtype");
  for (int i = 0; i < n; ++i) {
    if (!handles[i]) return fail(PAT_ERR_INVALID, "NULL handle");
    if (n_frames[i] < 1 || n_frames[i] > 65535) return fail(PAT_ERR_INVALID, "n_frames must be 1..65535");
    for (int j = 0; j < i; ++j)
      if (handles[j] == handles[i]) return fail(PAT_ERR_INVALID, "a handle appears twice in one plan");
    if (handles[i]->device != handles[0]->device || handles[i]->P != handles[0]->P)
      return fail(PAT_ERR_INVALID, "plan handles must share the device and the tile size");
    if (handles[i]->delays != handles[0]->delays)
      return fail(PAT_ERR_INVALID,
                  "plan handles must share the delay source (stored table or constant speed)");
    if (handles[i]->wgt != handles[0]->wgt)
      return fail(PAT_ERR_INVALID,
                  "plan handles must all have solid-angle weights or all not (one kernel mode)");
  }
  std::unique_ptr<pat_plan_s> pl(new (std::nothrow) pat_plan_s());
  if (!pl) return fail(PAT_ERR_OOM, "plan");
  pl->hs.assign(handles, handles + n);
  pl->frames.assign(n_frames, n_frames + n);
  pl->dtype = dtype;
  pl->fmt = fmt_for(dtype);
  pl->flags = flags;
  pl->device = handles[0]->device;
  pl->n_sm = handles[0]->n_sm;
  pl->P = handles[0]->P;
  pl->SW = handles[0]->SW;
  pl->fb_uniform = fb_uniform;
  PAT_CUDA(cudaSetDevice(pl->device));
  if (own_words) {
    if (cudaMalloc(&pl->d_status, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&pl->d_sched, 4 * sizeof(unsigned)) != cudaSuccess) {
      cudaFree(pl->d_status);
      return fail(PAT_ERR_OOM, "plan words");
    }
    PAT_CUDA(cudaMemset(pl->d_status, 0, sizeof(int)));
    PAT_CUDA(cudaMemset(pl->d_sched, 0, 4 * sizeof(unsigned)));
  } else {
    pl->d_status = handles[0]->d_status;
    pl->d_sched = handles[0]->d_sched;
  }
  // default shape: 8 sensors per stage in 100 KB; if the stage windows do not
  // fit, the device's limit, then 4 sensors per stage
  pat_status st = PAT_ERR_CUDA;
  const int limit_kb = handles[0]->max_smem / 1024;
  const int tries[3][2] = {{8, 100}, {8, limit_kb}, {4, limit_kb}};
  for (const auto& t : tries) {
    st = plan_shape(pl.get(), t[0], t[1]);
    if (st == PAT_OK) break;
  }
  if (st != PAT_OK) {
    if (own_words) {
      cudaFree(pl->d_status);
      cudaFree(pl->d_sched);
    }
    return st;
  }
  if (!own_words) pl->flags |= 0x80000000u;  // marks borrowed device words
  *out = pl.release();
  return PAT_OK;
}

// Locks every handle of a plan for one execution, in address order (so two
// plans that share handles cannot deadlock): an execution may grow a handle's
// working buffers and reads its table pointers, which the handle's own calls
// (reconstruct, evict, restore, set_solid_angle) change under the same lock.
struct HandleLocks {
  std::vector<std::unique_lock<std::mutex>> locks;
  explicit HandleLocks(const std::vector<pat_bp_t>& hs) {
    std::vector<pat_bp_t> order(hs);
    std::sort(order.begin(), order.end(), std::less<pat_bp_t>());
    locks.reserve(order.size());
    for (pat_bp_t h : order) locks.emplace_back(h->mu);
  }
};

static pat_status plan_run(pat_plan_t pl, const void* const* sig, const float* const* scales,
                           float* const* outs, cudaStream_t stream) {
  if (!sig || !outs) return fail(PAT_ERR_INVALID, "signals/outs NULL");
  for (size_t i = 0; i < pl->hs.size(); ++i) {
    if (!sig[i] || !outs[i]) return fail(PAT_ERR_INVALID, "NULL signal or output pointer");
    if (pl->dtype != PAT_F32 && (!scales || !scales[i]))
      return fail(PAT_ERR_INVALID, "16-bit signals need scales");
  }
  PAT_CUDA(cudaSetDevice(pl->device));
  const HandleLocks locks(pl->hs);
  pat_status st;
  if ((pl->flags & PAT_PLAN_AUTOTUNE) && !pl->tuned) {
    drop_graph(pl);
    if ((st = autotune(pl, sig, scales, outs, stream)) != PAT_OK) return st;
  }
  if ((st = refresh_buffers(pl)) != PAT_OK) return st;
  fill_pointers(pl, sig, scales, outs);
  if (!(pl->flags & PAT_PLAN_GRAPH)) return launch_all(pl, stream);
  if (!pl->exec) {
    if ((st = capture(pl)) != PAT_OK) return st;
  } else if ((st = refresh_graph(pl)) != PAT_OK) {
    return st;
  }
  PAT_CUDA(cudaGraphLaunch(pl->exec, stream));
  return PAT_OK;
}

static void plan_free(pat_plan_t pl) {
  if (!pl) return;
  cudaSetDevice(pl->device);
  cudaDeviceSynchronize();
  drop_graph(pl);
  if (pl->cap_stream) cudaStreamDestroy(pl->cap_stream);
  if (!(pl->flags & 0x80000000u)) {
    cudaFree(pl->d_status);
    cudaFree(pl->d_sched);
  }
  delete pl;
}

extern "C" pat_status pat_plan_create(const pat_bp_t* handles, const int* n_frames, int n,
                                      pat_dtype dtype, unsigned flags, pat_plan_t* out) {
  return plan_new(handles, n_frames, n, dtype, flags & (PAT_PLAN_AUTOTUNE | PAT_PLAN_GRAPH), true, 0,
                  out);
}

extern "C" pat_status pat_plan_execute(pat_plan_t plan, const void* const* signals_dev,
                                       const float* const* scales_dev, float* const* outs_dev,
                                       pat_stream_t stream) {
  if (!plan) return fail(PAT_ERR_INVALID, "NULL plan");
  std::lock_guard<std::mutex> lk(plan->mu);
  return plan_run(plan, signals_dev, scales_dev, outs_dev, static_cast<cudaStream_t>(stream));
}

extern "C" pat_status pat_plan_sync(pat_plan_t plan, pat_stream_t stream) {
  if (!plan) return fail(PAT_ERR_INVALID, "NULL plan");
  PAT_CUDA(cudaSetDevice(plan->device));
  PAT_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  int flag = 0;
  PAT_CUDA(cudaMemcpy(&flag, plan->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  if (!flag) return PAT_OK;
  PAT_CUDA(cudaMemset(plan->d_status, 0, sizeof(int)));
  PAT_CUDA(cudaMemset(plan->d_sched, 0, 4 * sizeof(unsigned)));
  for (pat_bp_t h : plan->hs)
    if (h->d_counter) PAT_CUDA(cudaMemset(h->d_counter, 0, h->counter_cap));
  return fail(flag & kStatusTimeout ? PAT_ERR_TIMEOUT : PAT_ERR_CUDA,
              flag & kStatusTimeout ? "a device wait ran out of time" : "bad launch configuration");
}

extern "C" pat_status pat_plan_info(pat_plan_t plan, pat_plan_info_t* info) {
  if (!plan || !info) return fail(PAT_ERR_INVALID, "NULL argument");
  std::lock_guard<std::mutex> lk(plan->mu);
  std::memset(info, 0, sizeof(*info));
  info->n_inst = int(plan->hs.size());
  info->sensors_per_stage = plan->S;
  info->smem_budget_kb = plan->budget_kb;
  info->n_units = plan->n_units;
  info->tuned = plan->tuned ? 1 : 0;
  info->graph = plan->exec ? 1 : 0;
  info->tune_ms = plan->tune_ms;
  info->n_classes = int(plan->cls.size());
  for (const PlanClass& k : plan->cls) {
    info->frames_per_unit = std::max(info->frames_per_unit, k.FB);
    info->stages = std::max(info->stages, k.cfg.stages);
    info->grid = std::max(info->grid, k.grid);
    info->fb_mask |= k.FB;
  }
  return PAT_OK;
}

extern "C" pat_status pat_plan_destroy(pat_plan_t plan) {
  plan_free(plan);
  return PAT_OK;
}

extern "C" pat_status pat_bp_reconstruct_multi(const pat_bp_t* handles, const void* const* signals_dev,
                                               pat_dtype dtype, const float* const* scales_dev,
                                               const int* n_frames, float* const* outs_dev, int n,
                                               pat_stream_t stream) {
  pat_plan_t pl = nullptr;
  pat_status st = plan_new(handles, n_frames, n, dtype, 0, false, 0, &pl);
  if (st != PAT_OK) return st;
  st = plan_run(pl, signals_dev, scales_dev, outs_dev, static_cast<cudaStream_t>(stream));
  // the plan's parameter blocks were copied at launch; its device words are
  // the first handle's, so nothing in flight depends on the plan object
  drop_graph(pl);
  delete pl;
  return st;
}

extern "C" pat_status pat_bp_autotune(pat_bp_t h, const void* signals_dev, pat_dtype dtype,
                                      const float* scales_dev, int n_frames, float* out_dev,
                                      pat_stream_t stream) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  std::lock_guard<std::mutex> lk(h->mu);
  pat_plan_t pl = nullptr;
  pat_status st = plan_new(&h, &n_frames, 1, dtype, 0, false, frames_per_group(n_frames), &pl);
  if (st != PAT_OK) return st;
  const void* sig[1] = {signals_dev};
  const float* sc[1] = {scales_dev};
  float* outs[1] = {out_dev};
  st = autotune(pl, sig, dtype == PAT_F32 ? (scales_dev ? sc : nullptr) : sc, outs,
                static_cast<cudaStream_t>(stream));
  if (st == PAT_OK) {
    const int fi = fb_index(pl->fb_uniform);
    h->tuned_S[fi][pl->fmt] = pl->S;
    h->tuned_budget_kb[fi][pl->fmt] = pl->budget_kb;
  }
  cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  drop_graph(pl);
  delete pl;
  return st;
}
