// kernels.cu -- sm_103a kernels of the on-line back projection (Eq. (BP)).
//
//   preprocess_kernel  b_k = 2 p_k - 2 t_k dp/dt|_k per (frame, sensor) row,
//                      t_k = k dt, central difference inside and one-sided
//                      differences at the ends; optional 16-bit (value, slope)
//                      pairs with a per-row scale.  Since t_k / dt = k the
//                      interior value is 2 p_k - k (p_{k+1} - p_{k-1}).
//   gather_kernel      out[f][r] = sum_s w_s * b_{f,s}(T_s(r)/dt) with linear
//                      interpolation (Sec. II-C), defined in gather.cuh; this
//                      unit instantiates it for delays from the stored
//                      fast-marching table and holds the launchers.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdio>

#include "gather.cuh"

namespace patbp {
// ---------------------------------------------------------- preprocessing --
template <int DT>
__device__ __forceinline__ float load_sample(const void* sig, int64_t i) {
  if constexpr (DT == 0) {
    return __ldg(static_cast<const float*>(sig) + i);
  } else if constexpr (DT == 1) {
    return __bfloat162float(static_cast<const __nv_bfloat16*>(sig)[i]);
  } else {
    return __half2float(static_cast<const __half*>(sig)[i]);
  }
}

// p_k0 .. p_{k0+7} of a row, times sc, zero outside [0, n): one or two 16-byte
// loads when the run lies in the row and is aligned (so signals read in place
// from host memory cost few requests), else one load per sample.
template <int DT>
__device__ __forceinline__ void load_run8(const void* sig, int64_t row0, int k0, int n, float sc,
                                          float* v) {
  const size_t esz = DT == 0 ? 4 : 2;
  const unsigned char* ptr = static_cast<const unsigned char*>(sig) + (row0 + k0) * int64_t(esz);
  if (k0 >= 0 && k0 + 8 <= n && (reinterpret_cast<uintptr_t>(ptr) & 15) == 0) {
    if constexpr (DT == 0) {
      const float4 a = __ldg(reinterpret_cast<const float4*>(ptr));
      const float4 b = __ldg(reinterpret_cast<const float4*>(ptr) + 1);
      const float x[8] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) v[j] = __fmul_rn(x[j], sc);
    } else {
      const uint4 q = __ldg(reinterpret_cast<const uint4*>(ptr));
      const uint32_t w[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const unsigned short h = (unsigned short)(w[j >> 1] >> ((j & 1) * 16));
        const float x = DT == 1 ? __bfloat162float(__ushort_as_bfloat16(h)) : __half2float(__ushort_as_half(h));
        v[j] = __fmul_rn(x, sc);
      }
    }
  } else {
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int k = k0 + j;
      v[j] = (k >= 0 && k < n) ? __fmul_rn(load_sample<DT>(sig, row0 + k), sc) : 0.0f;
    }
  }
}

// The 16-bit (value, slope) pair of b_k and b_{k+1} scaled by inv: every
// product and difference is explicitly rounded, so the codes do not depend on
// how the compiler contracts the expression in the kernel that calls this.
template <int FMT>
__device__ __forceinline__ uint32_t encode_pair(float b0, float b1, float inv) {
  const float v0 = __fmul_rn(b0, inv), v1 = __fmul_rn(b1, inv);
  if constexpr (FMT == kBBF16P) {
    const __nv_bfloat16 q0 = __float2bfloat16_rn(v0);
    const __nv_bfloat16 q1 = __float2bfloat16_rn(__fsub_rn(v1, __bfloat162float(q0)));
    return uint32_t(__bfloat16_as_ushort(q0)) | (uint32_t(__bfloat16_as_ushort(q1)) << 16);
  } else {
    const __half q0 = __float2half_rn(v0);
    const __half q1 = __float2half_rn(__fsub_rn(v1, __half2float(q0)));
    return uint32_t(__half_as_ushort(q0)) | (uint32_t(__half_as_ushort(q1)) << 16);
  }
}

template <int N>
__device__ __forceinline__ void store_words(uint32_t* dst, const uint32_t (&w)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 4)
      *reinterpret_cast<uint4*>(dst + i) = make_uint4(w[i], w[i + 1], w[i + 2], w[i + 3]);
  } else if constexpr (N == 2) {
    *reinterpret_cast<uint2*>(dst) = make_uint2(w[0], w[1]);
  } else {
    dst[0] = w[0];
  }
}

// One CTA per (sensor, frame group) row; every thread owns K consecutive
// samples of the row for all FB frames and issues all its loads before any
// use; the samples just outside its run (p_{k0-1}, p_{k0+K}, p_{k0+K+1}) come
// from the neighbouring lanes by shuffles, so the loops run warp-uniformly.
// Rows are written frame-interleaved, K * FB words per thread.
template <int DT, int FMT, int FB>
__device__ __forceinline__ void preprocess_row(const PreParams& p, int s, int g) {
  constexpr int K = 8;
  __shared__ float red[8][FB];
  const int f0 = g * FB;
  const int fb_eff = min(FB, p.n_frames - f0);
  const int n = p.n_t;
  int64_t row0[FB];
  float sc[FB];
#pragma unroll
  for (int fb = 0; fb < FB; ++fb) {
    const int f = min(f0 + fb, p.n_frames - 1);
    const int64_t r = int64_t(f) * p.n_sensors + s;
    row0[fb] = r * n;
    sc[fb] = p.scales ? p.scales[r] : 1.0f;
  }
  // b_{k0..k0+K} of frame fb (K + 1 values; the last feeds the pair slope).
  // Products and differences are explicitly rounded (no contraction into
  // FMAs): the values do not depend on how the compiler schedules them.  All
  // lanes of a warp call it together (consecutive runs, k0 = lane K + ...).
  const int lane = threadIdx.x & 31;
  auto sample = [&](int fb, int k) {
    return (k >= 0 && k < n) ? __fmul_rn(load_sample<DT>(p.sig, row0[fb] + k), sc[fb]) : 0.0f;
  };
  auto b_run = [&](int fb, int k0, float (&b)[K + 1]) {
    static_assert(K == 8, "runs of 8 samples");
    float v[K + 3];  // p_{k0-1} .. p_{k0+K+1}
    load_run8<DT>(p.sig, row0[fb], k0, n, sc[fb], v + 1);
    const float prev = __shfl_up_sync(0xffffffffu, v[K], 1);
    const float nx1 = __shfl_down_sync(0xffffffffu, v[1], 1);
    const float nx2 = __shfl_down_sync(0xffffffffu, v[2], 1);
    v[0] = lane == 0 ? sample(fb, k0 - 1) : prev;
    v[K + 1] = lane == 31 ? sample(fb, k0 + K) : nx1;
    v[K + 2] = lane == 31 ? sample(fb, k0 + K + 1) : nx2;
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      const int k = k0 + j;
      float r;
      if (k >= n) r = 0.0f;
      else if (k == 0) r = 2.0f * v[j + 1];
      else if (k == n - 1) r = fmaf(-2.0f * float(k), __fsub_rn(v[j + 1], v[j]), 2.0f * v[j + 1]);
      else r = fmaf(-float(k), __fsub_rn(v[j + 2], v[j]), 2.0f * v[j + 1]);
      b[j] = r;
    }
  };
  float inv[FB], sigma[FB];
#pragma unroll
  for (int fb = 0; fb < FB; ++fb) sigma[fb] = inv[fb] = 1.0f;
  if constexpr (FMT != kBF32) {
    float mx[FB];
#pragma unroll
    for (int fb = 0; fb < FB; ++fb) mx[fb] = 0.0f;
    for (int kw = (threadIdx.x & ~31) * K; kw < n; kw += blockDim.x * K) {
      const int k0 = kw + lane * K;  // runs past the row give b = 0
#pragma unroll
      for (int fb = 0; fb < FB; ++fb) {
        float b[K + 1];
        b_run(fb, k0, b);
#pragma unroll
        for (int j = 0; j < K; ++j) mx[fb] = fmaxf(mx[fb], fabsf(b[j]));
      }
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
#pragma unroll
    for (int fb = 0; fb < FB; ++fb) {
      float v = mx[fb];
      for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
      if (l == 0) red[w][fb] = v;
    }
    __syncthreads();
#pragma unroll
    for (int fb = 0; fb < FB; ++fb) {
      float v = 0.0f;
      for (int q = 0; q < int(blockDim.x >> 5); ++q) v = fmaxf(v, red[q][fb]);
      sigma[fb] = v > 0.0f ? v : 1.0f;
      inv[fb] = 1.0f / sigma[fb];
    }
  }
  uint32_t* dst = static_cast<uint32_t*>(p.b) + (int64_t(g) * p.n_sensors + s) * p.n_t_pad * FB;
  for (int kw = (threadIdx.x & ~31) * K; kw < p.n_t_pad; kw += blockDim.x * K) {
    const int k0 = kw + lane * K;
    uint32_t w[K * FB];
#pragma unroll
    for (int fb = 0; fb < FB; ++fb) {
      if (fb < fb_eff) {
        float b[K + 1];
        b_run(fb, k0, b);
#pragma unroll
        for (int j = 0; j < K; ++j) {
          if constexpr (FMT == kBF32) w[j * FB + fb] = __float_as_uint(b[j]);
          else w[j * FB + fb] = encode_pair<FMT>(b[j], b[j + 1], inv[fb]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) w[j * FB + fb] = 0u;
      }
    }
    if (k0 < p.n_t_pad) store_words<K * FB>(dst + int64_t(k0) * FB, w);
  }
  if (threadIdx.x < FB) {
    const int fb = threadIdx.x;
    float mval = 0.0f;
#pragma unroll
    for (int q = 0; q < FB; ++q)
      if (q == fb && fb < fb_eff) mval = p.weights[s] * sigma[q];
    p.m[(int64_t(g) * p.n_sensors_pad + s) * FB + fb] = mval;
  }
}

// The same rows for FB >= 2 frames per group, laid out for occupancy: thread
// t works on frame t mod FB and runs of 8 samples, frames fastest across the
// lanes, so a run's neighbouring runs of the same frame sit FB lanes away
// (shuffles by FB), every store instruction writes whole 32-byte pieces of
// FB * 8 consecutive words, and a thread keeps 11 samples instead of FB x 11.
// Each sample is the same expression as in preprocess_row, so the integrand
// has the same bits whatever the frames per group.
template <int DT, int FMT, int FB>
__device__ __forceinline__ void preprocess_row_frames(const PreParams& p, int s, int g) {
  static_assert(FB >= 2 && FB <= 16 && (FB & (FB - 1)) == 0, "frames per group");
  constexpr int K = 8;
  constexpr int RUNS = 256 / FB;  // runs of one frame per block pass
  __shared__ float red[8][FB];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int fb = threadIdx.x & (FB - 1);
  const int run = threadIdx.x / FB;
  const int f0 = g * FB;
  const int fb_eff = min(FB, p.n_frames - f0);
  const int n = p.n_t;
  const int f = min(f0 + fb, p.n_frames - 1);
  const int64_t r = int64_t(f) * p.n_sensors + s;
  const int64_t row0 = r * n;
  const float sc = p.scales ? p.scales[r] : 1.0f;
  auto sample = [&](int k) {
    return (k >= 0 && k < n) ? __fmul_rn(load_sample<DT>(p.sig, row0 + k), sc) : 0.0f;
  };
  // b_{k0..k0+K} of this thread's frame; all lanes of a warp call it together
  auto b_run = [&](int k0, float (&b)[K + 1]) {
    float v[K + 3];  // p_{k0-1} .. p_{k0+K+1}
    load_run8<DT>(p.sig, row0, k0, n, sc, v + 1);
    const float prev = __shfl_up_sync(0xffffffffu, v[K], FB);
    const float nx1 = __shfl_down_sync(0xffffffffu, v[1], FB);
    const float nx2 = __shfl_down_sync(0xffffffffu, v[2], FB);
    v[0] = lane < FB ? sample(k0 - 1) : prev;
    v[K + 1] = lane >= 32 - FB ? sample(k0 + K) : nx1;
    v[K + 2] = lane >= 32 - FB ? sample(k0 + K + 1) : nx2;
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      const int k = k0 + j;
      float x;
      if (k >= n) x = 0.0f;
      else if (k == 0) x = 2.0f * v[j + 1];
      else if (k == n - 1) x = fmaf(-2.0f * float(k), __fsub_rn(v[j + 1], v[j]), 2.0f * v[j + 1]);
      else x = fmaf(-float(k), __fsub_rn(v[j + 2], v[j]), 2.0f * v[j + 1]);
      b[j] = x;
    }
  };
  float sigma = 1.0f, inv = 1.0f;
  if constexpr (FMT != kBF32) {
    float mx = 0.0f;
    for (int kw = 0; kw < n; kw += RUNS * K) {
      const int k0 = kw + run * K;  // runs past the row give b = 0
      float b[K + 1];
      b_run(k0, b);
#pragma unroll
      for (int j = 0; j < K; ++j) mx = fmaxf(mx, fabsf(b[j]));
    }
    for (int o = FB; o < 32; o <<= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane < FB) red[warp][lane] = mx;
    __syncthreads();
    float v = 0.0f;
    for (int q = 0; q < int(blockDim.x >> 5); ++q) v = fmaxf(v, red[q][fb]);
    sigma = v > 0.0f ? v : 1.0f;
    inv = 1.0f / sigma;
  }
  uint32_t* dst = static_cast<uint32_t*>(p.b) + (int64_t(g) * p.n_sensors + s) * p.n_t_pad * FB;
  const bool live = fb < fb_eff;
  for (int kw = 0; kw < p.n_t_pad; kw += RUNS * K) {
    const int k0 = kw + run * K;
    float b[K + 1];
    b_run(k0, b);
    if (k0 >= p.n_t_pad) continue;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      uint32_t wv = 0u;
      if (live) {
        if constexpr (FMT == kBF32) wv = __float_as_uint(b[j]);
        else wv = encode_pair<FMT>(b[j], b[j + 1], inv);
      }
      // 8-frame rows: the two 16-byte halves of rows with bit 2 of the row
      // index set are stored swapped (k0 is a multiple of 8, so that bit is
      // j's), which the gather's shared-memory reads undo (row_half_swap)
      const int pos = FB == 8 ? (fb ^ (((j >> 2) & 1) << 2)) : fb;
      dst[int64_t(k0 + j) * FB + pos] = wv;
    }
  }
  if (threadIdx.x < FB) p.m[(int64_t(g) * p.n_sensors_pad + s) * FB + fb] = live ? p.weights[s] * sigma : 0.0f;
}

// One (sensor, frame group) row per CTA: the frame-fast layout for groups of
// several frames, the sample-run layout (preprocess_row) for single frames.
template <int DT, int FMT, int FB>
__device__ __forceinline__ void preprocess_group(const PreParams& p, int s, int g) {
  if constexpr (FB == 1) preprocess_row<DT, FMT, FB>(p, s, g);
  else preprocess_row_frames<DT, FMT, FB>(p, s, g);
}

template <int DT, int FMT, int FB>
__global__ void __launch_bounds__(256) preprocess_kernel(const PreParams p) {
  // let the gather that depends on this kernel start its prologue now
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  preprocess_group<DT, FMT, FB>(p, blockIdx.x, blockIdx.y);
}

// Several instances in one launch: CTA x belongs to the instance whose range
// [cta_begin[i], cta_begin[i+1]) holds it; inside it, (sensor, frame group).
template <int DT, int FMT, int FB>
__global__ void __launch_bounds__(256) preprocess_multi_kernel(const __grid_constant__ PreMultiParams p) {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  int lo = 0, hi = p.n_inst - 1;
  const int64_t x = blockIdx.x;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (p.cta_begin[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  const PreParams& q = p.inst[lo];
  const int64_t loc = x - p.cta_begin[lo];
  preprocess_group<DT, FMT, FB>(q, int(loc % q.n_sensors), int(loc / q.n_sensors));
}


// ------------------------------------------------------------- wait probe --
__global__ void status_export_kernel(const int* status, int* host_status) { *host_status = *status; }

cudaError_t launch_status_export(const int* status, int* host_status, cudaStream_t st) {
  status_export_kernel<<<1, 1, 0, st>>>(status, host_status);
  return cudaGetLastError();
}

__global__ void wait_probe_kernel(int* status, uint64_t timeout_ns) {
  __shared__ uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    mbar_init_fence();
  }
  __syncthreads();
  // nothing ever arrives on `bar`: the bounded wait must give up
  if (threadIdx.x == 0) {
    if (!mbar_wait_bounded(&bar, 0, timeout_ns, nullptr)) atomicOr(status, kStatusTimeout);
    // complete the phase ourselves so the barrier is left in a clean state
    mbar_arrive(&bar);
  }
}

// --------------------------------------------------------------- launchers --
int gather_threads(const GatherConfig& c) { return 32 * ((c.P / 128) * c.SW + 3); }

size_t gather_smem_bytes(const GatherConfig& c, int Wst) {
  const StageLayout L(c.S, c.P, c.FB, Wst, c.delays | (c.wgt << 1));
  return size_t(kHeaderBytes) + kMetaBytes + L.bytes * c.stages + 2 * size_t(c.SW) * c.FB * c.P * 4;
}

template <int DT, int FMT>
static cudaError_t launch_pre_fb(const PreParams& p, cudaStream_t st) {
  dim3 grid(p.n_sensors, (p.n_frames + p.FB - 1) / p.FB);
  switch (p.FB) {
    case 1: preprocess_kernel<DT, FMT, 1><<<grid, 256, 0, st>>>(p); break;
    case 2: preprocess_kernel<DT, FMT, 2><<<grid, 256, 0, st>>>(p); break;
    case 4: preprocess_kernel<DT, FMT, 4><<<grid, 256, 0, st>>>(p); break;
    case 8: preprocess_kernel<DT, FMT, 8><<<grid, 256, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template <int DT, int FMT>
static cudaError_t launch_pre_multi_fb(const PreMultiParams& p, cudaStream_t st) {
  const int64_t ctas = p.cta_begin[p.n_inst];
  if (ctas <= 0) return cudaSuccess;
  const dim3 grid(static_cast<unsigned>(ctas), 1u, 1u);
  switch (p.FB) {
    case 1: preprocess_multi_kernel<DT, FMT, 1><<<grid, 256, 0, st>>>(p); break;
    case 2: preprocess_multi_kernel<DT, FMT, 2><<<grid, 256, 0, st>>>(p); break;
    case 4: preprocess_multi_kernel<DT, FMT, 4><<<grid, 256, 0, st>>>(p); break;
    case 8: preprocess_multi_kernel<DT, FMT, 8><<<grid, 256, 0, st>>>(p); break;
    default: return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

cudaError_t launch_preprocess_multi(const PreMultiParams& p, cudaStream_t st) {
  if (p.n_inst < 1 || p.n_inst > kMaxInst) return cudaErrorInvalidValue;
  for (int i = 0; i < p.n_inst; ++i)
    if (p.inst[i].dtype != p.dtype || p.inst[i].fmt != p.fmt || p.inst[i].FB != p.FB)
      return cudaErrorInvalidValue;
  if (p.dtype == 0 && p.fmt == kBF32) return launch_pre_multi_fb<0, kBF32>(p, st);
  if (p.dtype == 1 && p.fmt == kBBF16P) return launch_pre_multi_fb<1, kBBF16P>(p, st);
  if (p.dtype == 2 && p.fmt == kBF16P) return launch_pre_multi_fb<2, kBF16P>(p, st);
  return cudaErrorInvalidValue;
}

const void* gather_kernel_func(const GatherConfig& c, int fmt);
const void* preprocess_multi_func(int dtype, int fmt, int FB);

cudaError_t launch_preprocess(const PreParams& p, cudaStream_t st) {
  if (p.dtype == 0 && p.fmt == kBF32) return launch_pre_fb<0, kBF32>(p, st);
  if (p.dtype == 1 && p.fmt == kBBF16P) return launch_pre_fb<1, kBBF16P>(p, st);
  if (p.dtype == 2 && p.fmt == kBF16P) return launch_pre_fb<2, kBF16P>(p, st);
  return cudaErrorInvalidValue;
}

static cudaError_t gather_dispatch(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                                   cudaStream_t st, int* resident, int n_sm) {
  if (c.wgt)
    return c.delays ? gather_dispatch_wgt_const(c, fmt, p, grid, st, resident, n_sm)
                    : gather_dispatch_wgt(c, fmt, p, grid, st, resident, n_sm);
  if (c.delays) return gather_dispatch_const(c, fmt, p, grid, st, resident, n_sm);
  return gather_dispatch_t<0>(c, fmt, p, grid, st, resident, n_sm);
}

int gather_resident_ctas(const GatherConfig& c, int fmt, int Wst, int n_sm) {
  StreamParams dummy;
  dummy.Wst = Wst;
  int resident = 0;
  if (gather_dispatch(c, fmt, dummy, 0, nullptr, &resident, n_sm) != cudaSuccess) return 0;
  return resident;
}

cudaError_t launch_gather(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                          cudaStream_t st) {
  if (p.stages < 1 || p.stages > kMaxStages || p.S % 4 || p.S % c.SW || p.S > kMaxS ||
      p.Wst % 8 || p.n_inst < 1 || p.n_inst > kMaxInst || grid < 1)
    return cudaErrorInvalidValue;
  for (int i = 0; i < p.n_inst; ++i)
    if (p.inst[i].G % p.S || p.inst[i].G > kMaxG || p.inst[i].Wst > p.Wst) return cudaErrorInvalidValue;
  if (p.n_units == 0) return cudaSuccess;
  if (c.direct) {
    // one frame after the other: frame f's integrand rows and multipliers are
    // frame group f of the one-frame-per-group layout; the phase sums are reused
    if (p.n_inst != 1 || c.FB != 1) return cudaErrorInvalidValue;
    const InstDesc& d = p.inst[0];
    const size_t word = 4;  // integrand words are 32-bit in every format
    for (int f = 0; f < d.n_frames; ++f) {
      InstDesc df = d;
      df.n_frames = 1;
      df.n_fg = 1;
      df.b = static_cast<const unsigned char*>(d.b) + size_t(f) * d.n_sensors * d.n_t_pad * word;
      df.m = d.m + size_t(f) * d.n_sensors_pad;
      df.out = d.out + int64_t(f) * d.out_stride;
      cudaError_t e = launch_gather_direct(c, fmt, df, c.n_sm, p.status,
                                           f + 1 == d.n_frames ? p.host_status : nullptr, p.timeout_ns, st);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  return gather_dispatch(c, fmt, p, grid, st, nullptr, 0);
}

const void* gather_kernel_func(const GatherConfig& c, int fmt) {
  if (c.wgt) return c.delays ? gather_func_wgt_const(c, fmt) : gather_func_wgt(c, fmt);
  return c.delays ? gather_func_const(c, fmt) : gather_func_t<0>(c, fmt);
}

template <int DT, int FMT>
static const void* pre_multi_func_fb(int FB) {
  switch (FB) {
    case 1: return reinterpret_cast<const void*>(preprocess_multi_kernel<DT, FMT, 1>);
    case 2: return reinterpret_cast<const void*>(preprocess_multi_kernel<DT, FMT, 2>);
    case 4: return reinterpret_cast<const void*>(preprocess_multi_kernel<DT, FMT, 4>);
    case 8: return reinterpret_cast<const void*>(preprocess_multi_kernel<DT, FMT, 8>);
  }
  return nullptr;
}

const void* preprocess_multi_func(int dtype, int fmt, int FB) {
  if (dtype == 0 && fmt == kBF32) return pre_multi_func_fb<0, kBF32>(FB);
  if (dtype == 1 && fmt == kBBF16P) return pre_multi_func_fb<1, kBBF16P>(FB);
  if (dtype == 2 && fmt == kBF16P) return pre_multi_func_fb<2, kBF16P>(FB);
  return nullptr;
}

cudaError_t launch_wait_probe(int* status, uint64_t timeout_ns, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(status, timeout_ns);
  return cudaGetLastError();
}

}  // namespace patbp
