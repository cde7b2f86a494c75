// noalloc.cu -- a reconstruction entry point that allocates no device memory.
//
// Who needs it: hosts that own all device memory themselves and forbid a
// library to allocate (a framework with its own fixed pool or budget), and
// per-frame acquisition loops that must not call the CUDA allocator, whose
// cudaMalloc/cudaFree calls can synchronise the device and add latency
// jitter to every frame.  pat_bp_reconstruct grows the handle's own integrand
// and scratch buffers on demand; this variant instead takes all of its scratch
// (integrand rows, multipliers, segment partial sums, segment counters, unit
// tickets) from one file-scope device array of fixed size, kNoAllocBytes.
//
// Facts a caller must know:
//   * the array exists once per device that loads this library and stays
//     allocated until the process exits;
//   * the first call on a device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture;
//   * every call shares the array and finds the previous call's contents; the
//     parts that must start at zero are cleared on the stream by each call;
//   * calls whose work overlaps on the GPU (same or different streams, any
//     handles) race on the array: serialise them;
//   * device-side wait timeouts are reported by pat_bp_sync on the handle.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <mutex>
#include <string>

#include "handle.h"

using namespace patbp;

namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;  // 16 MiB per device
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

std::mutex g_addr_mu;
void* g_addr[kMaxDevices] = {};

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// Device address of the scratch array on the current device (looked up once).
pat_status scratch_address(int device, unsigned char** out) {
  if (device < 0 || device >= kMaxDevices) return fail(PAT_ERR_INVALID, "device index out of range");
  std::lock_guard<std::mutex> lk(g_addr_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress(no-allocation scratch)");
    g_addr[device] = p;
  }
  *out = static_cast<unsigned char*>(g_addr[device]);
  return PAT_OK;
}

}  // namespace

extern "C" pat_status pat_bp_reconstruct_noalloc(pat_bp_t h, const void* signals_dev,
                                                 pat_dtype dtype, const float* scales_dev,
                                                 int n_frames, float* out_dev,
                                                 pat_stream_t stream_) {
  if (!h) return fail(PAT_ERR_INVALID, "NULL handle");
  if (!signals_dev || !out_dev) return fail(PAT_ERR_INVALID, "signals/out NULL");
  if (n_frames < 1 || n_frames > 65535) return fail(PAT_ERR_INVALID, "n_frames must be 1..65535");
  if (dtype != PAT_F32 && dtype != PAT_BF16 && dtype != PAT_F16)
    return fail(PAT_ERR_INVALID, "unknown dtype");
  if (dtype != PAT_F32 && !scales_dev) return fail(PAT_ERR_INVALID, "16-bit signals need scales");
  std::lock_guard<std::mutex> lk(h->mu);
  if (h->evicted) return fail(PAT_ERR_INVALID, "the handle's table is evicted (pat_bp_restore)");
  cudaStream_t stream = static_cast<cudaStream_t>(stream_);
  PAT_CUDA(cudaSetDevice(h->device));
  const int fmt = fmt_for(dtype);
  int wst = 0;
  const GatherConfig c = pick_config(h, n_frames, fmt, &wst);
  const int FB = c.FB;
  const size_t n_fg = size_t((n_frames + FB - 1) / FB);

  // scratch layout: unit tickets | segment counters | partials | multipliers | integrand
  const size_t sched_bytes = 256;
  const size_t cnt_bytes = align256(n_fg * h->n_tiles * sizeof(int));
  const size_t part_bytes =
      align256(n_fg * h->n_tiles * h->n_seg * std::max(FB, h->SW) * h->P * sizeof(float));
  const size_t m_bytes = align256(n_fg * h->ns_pad * FB * sizeof(float));
  const size_t b_bytes = align256((n_fg * h->ns * h->nt_pad + kTailRows) * FB * 4);
  const size_t need = sched_bytes + cnt_bytes + part_bytes + m_bytes + b_bytes;
  if (need > kNoAllocBytes)
    return fail(PAT_ERR_INVALID, "this reconstruction needs " + std::to_string(need) +
                                     " bytes of scratch; the no-allocation path has " +
                                     std::to_string(kNoAllocBytes) + " (use fewer frames)");
  unsigned char* base = nullptr;
  pat_status st = scratch_address(h->device, &base);
  if (st != PAT_OK) return st;
  unsigned* sched = reinterpret_cast<unsigned*>(base);
  int* counter = reinterpret_cast<int*>(base + sched_bytes);
  float* part = reinterpret_cast<float*>(base + sched_bytes + cnt_bytes);
  float* m = reinterpret_cast<float*>(base + sched_bytes + cnt_bytes + part_bytes);
  void* b = base + sched_bytes + cnt_bytes + part_bytes + m_bytes;
  // what must start at zero: the unit tickets and the segment counters
  PAT_CUDA(cudaMemsetAsync(base, 0, sched_bytes + cnt_bytes, stream));

  PreParams pp = make_pre(h, signals_dev, dtype, scales_dev, n_frames, FB);
  pp.b = b;
  pp.m = m;
  cudaError_t e = launch_preprocess(pp, stream);
  if (e != cudaSuccess) return cuda_fail(e, "preprocess launch");

  StreamParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.inst[0] = make_desc(h, out_dev, n_frames, FB, wst);
  sp.inst[0].b = b;
  sp.inst[0].m = m;
  sp.inst[0].part = part;
  sp.inst[0].counter = counter;
  sp.n_inst = 1;
  sp.n_units = int64_t(sp.inst[0].n_fg) * sp.inst[0].n_tiles * sp.inst[0].n_seg;
  sp.S = c.S;
  sp.stages = c.stages;
  sp.Wst = wst;
  sp.status = h->d_status;
  sp.sched = sched;
  sp.timeout_ns = 2000000000ull;
  const int res = resident_ctas(c, fmt, wst, h->n_sm);
  if (res <= 0) return fail(PAT_ERR_CUDA, "gather kernel does not fit on the device");
  const int grid = int(std::min<int64_t>(sp.n_units, res));
  e = launch_gather(c, fmt, sp, grid, stream);
  if (e != cudaSuccess) return cuda_fail(e, "gather launch");
  return PAT_OK;
}
