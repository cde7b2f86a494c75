// kernels.cu -- sm_103a kernels of the on-line back projection (Eq. (BP)).
//
//   preprocess_kernel  b_k = 2 p_k - 2 t_k dp/dt|_k per (frame, sensor) row,
//                      t_k = k dt, central difference inside and one-sided
//                      differences at the ends; optional 16-bit (value, slope)
//                      pairs with a per-row scale.  Since t_k / dt = k the
//                      interior value is 2 p_k - k (p_{k+1} - p_{k-1}).
//   gather_kernel      out[f][r] = sum_s w_s * b_{f,s}(T_s(r)/dt) with linear
//                      interpolation (Sec. II-C).  One CTA owns a tile of P
//                      pixels, a contiguous range of sensors (one rank of a
//                      thread-block cluster) and FB frames.  A producer warp
//                      streams, per stage of S sensors, the tile's table block
//                      u[S][P], the multipliers and each sensor's window of
//                      integrand samples (packed back to back) into shared
//                      memory with 1-D bulk copies (cp.async.bulk) completing
//                      on mbarriers; consumer
//                      warps interpolate from shared memory and accumulate in
//                      FP32 registers.  Sensor phases inside the CTA are summed
//                      in fixed order through shared memory, cluster ranks in
//                      fixed order through distributed shared memory, so the
//                      result does not depend on timing or on batch size.
//
// Every wait on an mbarrier is bounded by a wall-clock limit; on expiry the CTA
// records kStatusTimeout, drains its own copies in flight (bounded again) and
// exits without touching the output's remaining values.
#include <cooperative_groups.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdio>

#include "kernels.cuh"

namespace cg = cooperative_groups;

namespace patbp {

// ------------------------------------------------------------ PTX helpers --
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
               : "memory");
}

__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_addr(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Wait for the phase of `bar` with the given parity; false if it did not
// complete within timeout_ns or another warp of the CTA already gave up.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity,
                                                  uint64_t timeout_ns, volatile int* abort_flag) {
  if (mbar_try_wait(bar, parity)) return true;
  const uint64_t t0 = global_ns();
  for (;;) {
    if (mbar_try_wait(bar, parity)) return true;
    if (abort_flag && *abort_flag) return false;
    if (global_ns() - t0 > timeout_ns) return false;
  }
}

// 1-D bulk copy global -> shared of this CTA; completion counted in bytes on bar.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes,
                                         uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

__device__ __forceinline__ void named_barrier(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

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

// b_k from the pressure row in shared memory (zero past the record).
__device__ __forceinline__ float integrand(const float* prow, int k, int n) {
  if (k >= n) return 0.0f;
  const float pk = prow[k];
  if (k == 0) return 2.0f * pk;
  if (k == n - 1) return fmaf(-2.0f * float(k), pk - prow[k - 1], 2.0f * pk);
  return fmaf(-float(k), prow[k + 1] - prow[k - 1], 2.0f * pk);
}

__device__ __forceinline__ float block_max(float v, float* scratch) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) scratch[w] = v;
  __syncthreads();
  if (w == 0) {
    v = l < int(blockDim.x >> 5) ? scratch[l] : 0.0f;
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (l == 0) scratch[0] = v;
  }
  __syncthreads();
  v = scratch[0];
  __syncthreads();
  return v;
}

template <int DT, int FMT>
__global__ void __launch_bounds__(256) preprocess_kernel(const PreParams p) {
  extern __shared__ float prow[];  // n_t pressures, then 32 floats of scratch
  float* scratch = prow + ((p.n_t + 31) & ~31);
  const int s = blockIdx.x, f = blockIdx.y;
  const int64_t r = int64_t(f) * p.n_sensors + s;
  const float sc = p.scales ? p.scales[r] : 1.0f;
  const int64_t src0 = r * p.n_t;
  for (int k = threadIdx.x; k < p.n_t; k += blockDim.x) prow[k] = load_sample<DT>(p.sig, src0 + k) * sc;
  __syncthreads();
  const float w = p.weights[s];
  const int64_t dst0 = r * p.n_t_pad;
  if constexpr (FMT == kBF32) {
    float* b = static_cast<float*>(p.b) + dst0;
    for (int k = threadIdx.x; k < p.n_t_pad; k += blockDim.x) b[k] = integrand(prow, k, p.n_t);
    if (threadIdx.x == 0) p.m[int64_t(f) * p.n_sensors_pad + s] = w;
  } else {
    float mx = 0.0f;
    for (int k = threadIdx.x; k < p.n_t; k += blockDim.x) mx = fmaxf(mx, fabsf(integrand(prow, k, p.n_t)));
    mx = block_max(mx, scratch);
    const float sigma = mx > 0.0f ? mx : 1.0f;
    const float inv = 1.0f / sigma;
    uint32_t* b = static_cast<uint32_t*>(p.b) + dst0;
    for (int k = threadIdx.x; k < p.n_t_pad; k += blockDim.x) {
      const float v0 = integrand(prow, k, p.n_t) * inv;
      const float v1 = integrand(prow, k + 1, p.n_t) * inv;
      uint32_t word;
      if constexpr (FMT == kBBF16P) {
        const __nv_bfloat16 q0 = __float2bfloat16_rn(v0);
        const __nv_bfloat16 q1 = __float2bfloat16_rn(v1 - __bfloat162float(q0));
        word = uint32_t(__bfloat16_as_ushort(q0)) | (uint32_t(__bfloat16_as_ushort(q1)) << 16);
      } else {
        const __half q0 = __float2half_rn(v0);
        const __half q1 = __float2half_rn(v1 - __half2float(q0));
        word = uint32_t(__half_as_ushort(q0)) | (uint32_t(__half_as_ushort(q1)) << 16);
      }
      b[k] = word;
    }
    if (threadIdx.x == 0) p.m[int64_t(f) * p.n_sensors_pad + s] = w * sigma;
  }
}

// ------------------------------------------------------------------ gather --
template <int FMT>
__device__ __forceinline__ float lerp_window(const unsigned char* wrow, unsigned i, float ph) {
  if constexpr (FMT == kBF32) {
    const float* b = reinterpret_cast<const float*>(wrow);
    const float b0 = b[i], b1 = b[i + 1];
    return fmaf(ph, b1 - b0, b0);
  } else if constexpr (FMT == kBBF16P) {
    const uint32_t wd = reinterpret_cast<const uint32_t*>(wrow)[i];
    return fmaf(ph, __uint_as_float(wd & 0xffff0000u), __uint_as_float(wd << 16));
  } else {
    const uint32_t wd = reinterpret_cast<const uint32_t*>(wrow)[i];
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(&wd));
    return fmaf(ph, v.y, v.x);
  }
}

constexpr int kMaxStages = 8;
constexpr int kMaxS = 32;

// Shared-memory layout of one pipeline stage (byte offsets):
//   u      [S][P] float           the tile's table rows of the stage's sensors
//   m      [FB][S4] float         multipliers w_s * sigma per frame
//   off    [S] int                window offset of each sensor inside a frame region
//   win    [FB][Wst + 4] entries  the stage's windows packed at `off`, then 4
//                                 zero entries that out-of-record pixels read
struct StageLayout {
  size_t u, m, off, win, bytes;
  __host__ __device__ StageLayout(int S, int P, int FB, int Wst) {
    const int S4 = (S + 3) & ~3;
    u = 0;
    m = u + size_t(S) * P * 4;
    off = m + size_t(FB) * S4 * 4;
    win = off + size_t(((S + 3) & ~3)) * 4;
    bytes = win + size_t(FB) * (Wst + 4) * 4;
  }
};

template <int P, int FB, int FMT, int SW>
__global__ void __launch_bounds__(32 * ((P / 128) * SW + 1)) gather_kernel(const GatherParams p) {
  constexpr int PW = P / 128;       // warps across the tile's pixels
  constexpr int NWC = PW * SW;      // consumer warps
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kMaxStages;
  volatile int* abort_flag = reinterpret_cast<volatile int*>(empty + kMaxStages);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int tile = blockIdx.x, rank = blockIdx.y;
  const int f0 = blockIdx.z * FB;
  const int fb_eff = min(FB, p.n_frames - f0);
  const int s_begin = rank * p.split_len;
  const int s_end = min(p.n_sensors, s_begin + p.split_len);
  const int n_chunks = s_end > s_begin ? (s_end - s_begin + p.S - 1) / p.S : 0;
  const int S4 = (p.S + 3) & ~3;
  const int pitch = p.Wst + 4;  // entries per frame region of a stage
  const StageLayout L(p.S, P, FB, p.Wst);
  unsigned char* stage0 = smem + 256;
  float* red = reinterpret_cast<float*>(stage0 + L.bytes * p.stages);  // [SW][FB][P]
  float* fin = red + SW * FB * P;                                      // [FB][P]

  if (threadIdx.x == 0) {
    for (int st = 0; st < p.stages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], NWC);
    }
    *abort_flag = 0;
    mbar_init_fence();
  }
  // the 4 zero entries after every frame region of every stage
  for (int q = threadIdx.x; q < p.stages * FB * 4; q += blockDim.x) {
    const int st = q / (FB * 4), rem = q - st * FB * 4;
    const int fb = rem >> 2, k = rem & 3;
    reinterpret_cast<uint32_t*>(stage0 + st * L.bytes + L.win)[size_t(fb) * pitch + p.Wst + k] = 0u;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  if (warp == NWC) {
    // ------------------------------------------------------------ producer --
    int issued = 0;
    for (int c = 0; c < n_chunks; ++c) {
      const int st = c % p.stages, use = c / p.stages;
      if (use > 0 && !mbar_wait_bounded(&empty[st], (use - 1) & 1, p.timeout_ns, abort_flag)) {
        if (lane == 0) {
          atomicOr(p.status, kStatusTimeout);
          *abort_flag = 1;
        }
        break;
      }
      const int s0 = s_begin + c * p.S;
      const int se = min(p.S, s_end - s0);
      const int se4 = (se + 3) & ~3;
      unsigned char* sb = stage0 + st * L.bytes;
      // this lane's sensor (S <= 32): packed window base and length
      int bs = 0, wl = 0;
      if (lane < se) {
        const uint32_t word = uint32_t(__ldg(p.base + size_t(tile) * p.n_sensors + s0 + lane));
        bs = int(word & 0xffffu);
        wl = int(word >> 16);
      }
      // exclusive prefix sum of the window lengths = packed offsets
      int incl = wl;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int total_w = __shfl_sync(0xffffffffu, incl, 31);
      int off = incl - wl;
      if (total_w > p.Wst) {  // cannot happen with a host-computed Wst; stay in bounds
        if (lane == 0) atomicOr(p.status, kStatusBadConfig);
        wl = 0;
        off = 0;
      }
      const uint32_t wbytes = total_w > p.Wst ? 0u : uint32_t(total_w) * 4u;
      if (lane < se) reinterpret_cast<int*>(sb + L.off)[lane] = off;
      __syncwarp();
      const uint32_t bytes = uint32_t(se) * P * 4 + uint32_t(fb_eff) * (se4 * 4 + wbytes);
      if (lane == 0) mbar_arrive_expect_tx(&full[st], bytes);
      __syncwarp();
      if (lane == 0)
        bulk_g2s(sb + L.u, p.u + (size_t(tile) * p.n_sensors + s0) * P, uint32_t(se) * P * 4,
                 &full[st]);
      if (lane < fb_eff)
        bulk_g2s(sb + L.m + size_t(lane) * S4 * 4,
                 p.m + size_t(f0 + lane) * p.n_sensors_pad + s0, uint32_t(se4) * 4, &full[st]);
      if (wl > 0) {
        for (int fb = 0; fb < fb_eff; ++fb) {
          const unsigned char* src =
              static_cast<const unsigned char*>(p.b) +
              ((size_t(f0 + fb) * p.n_sensors + s0 + lane) * p.n_t_pad + bs) * 4;
          bulk_g2s(sb + L.win + (size_t(fb) * pitch + off) * 4, src, uint32_t(wl) * 4, &full[st]);
        }
      }
      issued = c + 1;
    }
    // drain the copies still in flight before the CTA may exit
    for (int c = max(0, issued - p.stages); c < issued; ++c)
      mbar_wait_bounded(&full[c % p.stages], (c / p.stages) & 1, p.timeout_ns, nullptr);
  } else {
    // ------------------------------------------------------------ consumers --
    const int pg = warp % PW, sp = warp / PW;
    if (rank == 0 && p.n_zero_runs > 0) {
      for (int fb = 0; fb < fb_eff; ++fb) {
        float* o = p.out + int64_t(f0 + fb) * p.out_stride;
        for (int r = tile + p.n_tiles * warp; r < p.n_zero_runs; r += p.n_tiles * NWC) {
          const int st0 = p.zero_runs[2 * r], len = p.zero_runs[2 * r + 1];
          for (int i = lane; i < len; i += 32) o[st0 + i] = 0.0f;
        }
      }
    }
    float acc[FB][4];
#pragma unroll
    for (int fb = 0; fb < FB; ++fb)
#pragma unroll
      for (int x = 0; x < 4; ++x) acc[fb][x] = 0.0f;
    for (int c = 0; c < n_chunks; ++c) {
      const int st = c % p.stages;
      if (!mbar_wait_bounded(&full[st], (c / p.stages) & 1, p.timeout_ns, abort_flag)) {
        if (lane == 0) {
          atomicOr(p.status, kStatusTimeout);
          *abort_flag = 1;
        }
        break;
      }
      const int se = min(p.S, s_end - (s_begin + c * p.S));
      const unsigned char* sb = stage0 + st * L.bytes;
      const float* su = reinterpret_cast<const float*>(sb + L.u) + pg * 128 + lane;
      const float* sm = reinterpret_cast<const float*>(sb + L.m);
      const int* soff = reinterpret_cast<const int*>(sb + L.off);
      const unsigned char* sw = sb + L.win;
      for (int sl = sp; sl < se; sl += SW) {
        const int off = soff[sl];
        const unsigned lim = unsigned(p.Wst - off);
        unsigned ii[4];
        float ph[4];
#pragma unroll
        for (int x = 0; x < 4; ++x) {
          const float uu = su[sl * P + x * 32];
          const unsigned i = min(unsigned(__float2int_rz(uu)), lim);
          ph[x] = uu - float(i);
          ii[x] = i + unsigned(off);
        }
#pragma unroll
        for (int fb = 0; fb < FB; ++fb) {
          if (fb < fb_eff) {
            const float mm = sm[fb * S4 + sl];
            const unsigned char* wrow = sw + size_t(fb) * pitch * 4;
#pragma unroll
            for (int x = 0; x < 4; ++x)
              acc[fb][x] = fmaf(mm, lerp_window<FMT>(wrow, ii[x], ph[x]), acc[fb][x]);
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[st]);
    }
    // fixed-order sum of the sensor phases
#pragma unroll
    for (int fb = 0; fb < FB; ++fb)
#pragma unroll
      for (int x = 0; x < 4; ++x) red[(sp * FB + fb) * P + pg * 128 + x * 32 + lane] = acc[fb][x];
    named_barrier(1, NWC * 32);
    for (int o = threadIdx.x; o < FB * P; o += NWC * 32) {
      float v = 0.0f;
#pragma unroll
      for (int q = 0; q < SW; ++q) v += red[q * FB * P + o];
      if (p.split == 1) {
        const int fb = o / P, pp = o - fb * P;
        if (fb < fb_eff) {
          const int idx = p.slot[size_t(tile) * P + pp];
          if (idx >= 0) p.out[int64_t(f0 + fb) * p.out_stride + idx] = v;
        }
      } else {
        fin[o] = v;
      }
    }
  }

  if (p.split > 1) {
    // fixed-order sum of the cluster ranks (sensor splits) through DSMEM
    cg::cluster_group cl = cg::this_cluster();
    cl.sync();
    if (warp < NWC) {
      const int total = FB * P;
      const int chunk = (total + p.split - 1) / p.split;
      const int o_end = min(total, (rank + 1) * chunk);
      for (int o = rank * chunk + threadIdx.x; o < o_end; o += NWC * 32) {
        float v = 0.0f;
        for (int q = 0; q < p.split; ++q) v += cl.map_shared_rank(fin, q)[o];
        const int fb = o / P, pp = o - fb * P;
        if (fb < fb_eff) {
          const int idx = p.slot[size_t(tile) * P + pp];
          if (idx >= 0) p.out[int64_t(f0 + fb) * p.out_stride + idx] = v;
        }
      }
    }
    cl.sync();
  }
}

// ------------------------------------------------------------- wait probe --
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
int gather_threads(const GatherConfig& c) { return 32 * ((c.P / 128) * c.SW + 1); }

size_t gather_smem_bytes(const GatherConfig& c, int fmt, int Wst) {
  (void)fmt;
  const StageLayout L(c.S, c.P, c.FB, Wst);
  return 256 + L.bytes * c.stages + size_t(c.SW) * c.FB * c.P * 4 + size_t(c.FB) * c.P * 4;
}

cudaError_t launch_preprocess(const PreParams& p, cudaStream_t st) {
  const size_t smem = (size_t((p.n_t + 31) & ~31) + 32) * sizeof(float);
  dim3 grid(p.n_sensors, p.n_frames);
  void (*kern)(const PreParams) = nullptr;
#define PAT_PRE_CASE(DT, FMT) \
  if (p.dtype == DT && p.fmt == FMT) kern = preprocess_kernel<DT, FMT>;
  PAT_PRE_CASE(0, kBF32)
  PAT_PRE_CASE(0, kBBF16P)
  PAT_PRE_CASE(0, kBF16P)
  PAT_PRE_CASE(1, kBF32)
  PAT_PRE_CASE(1, kBBF16P)
  PAT_PRE_CASE(1, kBF16P)
  PAT_PRE_CASE(2, kBF32)
  PAT_PRE_CASE(2, kBBF16P)
  PAT_PRE_CASE(2, kBF16P)
#undef PAT_PRE_CASE
  if (!kern) return cudaErrorInvalidValue;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  kern<<<grid, 256, smem, st>>>(p);
  return cudaGetLastError();
}

template <int P, int FB, int FMT, int SW>
static cudaError_t launch_gather_t(const GatherParams& p, size_t smem, cudaStream_t st) {
  auto kern = gather_kernel<P, FB, FMT, SW>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p.n_tiles, p.split, (p.n_frames + FB - 1) / FB);
  cfg.blockDim = dim3(32 * ((P / 128) * SW + 1));
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  int na = 0;
  if (p.split > 1) {
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = 1;
    attr[0].val.clusterDim.y = p.split;
    attr[0].val.clusterDim.z = 1;
    na = 1;
  }
  cfg.attrs = attr;
  cfg.numAttrs = na;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int P, int FMT, int SW>
static cudaError_t launch_gather_fb(int FB, const GatherParams& p, size_t smem, cudaStream_t st) {
  switch (FB) {
    case 1: return launch_gather_t<P, 1, FMT, SW>(p, smem, st);
    case 2: return launch_gather_t<P, 2, FMT, SW>(p, smem, st);
    case 4: return launch_gather_t<P, 4, FMT, SW>(p, smem, st);
    case 8: return launch_gather_t<P, 8, FMT, SW>(p, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_gather(const GatherConfig& c, int fmt, const GatherParams& p, cudaStream_t st) {
  if (p.stages < 1 || p.stages > kMaxStages || p.S % 4 || p.S % c.SW || p.S > kMaxS ||
      p.split < 1 || p.split > 8 || p.split_len % 4 || p.Wst % 8)
    return cudaErrorInvalidValue;
  const size_t smem = gather_smem_bytes(c, fmt, p.Wst);
  if (c.P == 128 && c.SW == 4) {
    if (fmt == kBF32) return launch_gather_fb<128, kBF32, 4>(c.FB, p, smem, st);
    if (fmt == kBBF16P) return launch_gather_fb<128, kBBF16P, 4>(c.FB, p, smem, st);
    if (fmt == kBF16P) return launch_gather_fb<128, kBF16P, 4>(c.FB, p, smem, st);
  } else if (c.P == 256 && c.SW == 2) {
    if (fmt == kBF32) return launch_gather_fb<256, kBF32, 2>(c.FB, p, smem, st);
    if (fmt == kBBF16P) return launch_gather_fb<256, kBBF16P, 2>(c.FB, p, smem, st);
    if (fmt == kBF16P) return launch_gather_fb<256, kBF16P, 2>(c.FB, p, smem, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t launch_wait_probe(int* status, uint64_t timeout_ns, cudaStream_t st) {
  wait_probe_kernel<<<1, 32, 0, st>>>(status, timeout_ns);
  return cudaGetLastError();
}

}  // namespace patbp
