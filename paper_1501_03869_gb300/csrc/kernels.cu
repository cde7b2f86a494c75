// kernels.cu -- sm_103a kernels of the on-line back projection (Eq. (BP)).
//
//   preprocess_kernel  b_k = 2 p_k - 2 t_k dp/dt|_k per (frame, sensor) row,
//                      t_k = k dt, central difference inside and one-sided
//                      differences at the ends; optional 16-bit (value, slope)
//                      pairs with a per-row scale.  Since t_k / dt = k the
//                      interior value is 2 p_k - k (p_{k+1} - p_{k-1}).
//   gather_kernel      out[f][r] = sum_s w_s * b_{f,s}(T_s(r)/dt) with linear
//                      interpolation (Sec. II-C).  Persistent: the work of one
//                      launch is a sequence of units (instance, frame group,
//                      tile of P pixels, segment of G sensors), cut into one
//                      contiguous range per CTA.  A producer warp streams, per
//                      stage of S sensors, the tile's table rows u[S][P], the
//                      multipliers and every sensor's window of integrand rows
//                      (packed back to back, FB frames per row) into shared
//                      memory with 1-D bulk copies (cp.async.bulk) completing on
//                      mbarriers; the windows' bases are fetched one unit ahead.
//                      Consumer warps interpolate from shared memory and
//                      accumulate in FP32 registers.  Sensor phases are summed
//                      in fixed order through shared memory and segments in
//                      fixed order by the last CTA to finish a tile, so the
//                      result depends neither on timing nor on how frames or
//                      instances are batched.
//
// Every wait on an mbarrier is bounded by a wall-clock limit; on expiry the CTA
// records kStatusTimeout, drains its own copies in flight (bounded again) and
// exits without touching the output's remaining values.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include <cstdio>

#include "kernels.cuh"

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

__device__ __forceinline__ int atomic_add_acq_rel(int* p, int v) {
  int old;
  asm volatile("atom.acq_rel.gpu.global.add.s32 %0, [%1], %2;" : "=r"(old) : "l"(p), "r"(v) : "memory");
  return old;
}

__device__ __forceinline__ void named_barrier(int id, int threads) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

__device__ __forceinline__ void named_barrier_arrive(int id, int threads) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(threads) : "memory");
}

// Hand-off barriers of the double-buffered unit sums, with literal ids so the
// compiler reserves only the ids it sees: "full" 1/2 and "free" 3/4 per buffer.
__device__ __forceinline__ void red_full_sync(int buf, int n) {
  if (buf) asm volatile("bar.sync 2, %0;" ::"r"(n) : "memory");
  else asm volatile("bar.sync 1, %0;" ::"r"(n) : "memory");
}
__device__ __forceinline__ void red_full_arrive(int buf, int n) {
  if (buf) asm volatile("bar.arrive 2, %0;" ::"r"(n) : "memory");
  else asm volatile("bar.arrive 1, %0;" ::"r"(n) : "memory");
}
__device__ __forceinline__ void red_free_sync(int buf, int n) {
  if (buf) asm volatile("bar.sync 4, %0;" ::"r"(n) : "memory");
  else asm volatile("bar.sync 3, %0;" ::"r"(n) : "memory");
}
__device__ __forceinline__ void red_free_arrive(int buf, int n) {
  if (buf) asm volatile("bar.arrive 4, %0;" ::"r"(n) : "memory");
  else asm volatile("bar.arrive 3, %0;" ::"r"(n) : "memory");
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

// b_k of one pressure row (zero past the record): 2 p_k - 2 t_k dp/dt with
// t_k / dt = k, central difference inside, one-sided at both ends.
template <int DT>
__device__ __forceinline__ float integrand(const void* sig, int64_t row0, float sc, int k, int n) {
  if (k >= n) return 0.0f;
  const float pk = load_sample<DT>(sig, row0 + k) * sc;
  if (k == 0) return 2.0f * pk;
  const float pm = load_sample<DT>(sig, row0 + k - 1) * sc;
  if (k == n - 1) return fmaf(-2.0f * float(k), pk - pm, 2.0f * pk);
  const float pp = load_sample<DT>(sig, row0 + k + 1) * sc;
  return fmaf(-float(k), pp - pm, 2.0f * pk);
}

template <int FMT>
__device__ __forceinline__ uint32_t encode_pair(float v0, float v1) {
  if constexpr (FMT == kBBF16P) {
    const __nv_bfloat16 q0 = __float2bfloat16_rn(v0);
    const __nv_bfloat16 q1 = __float2bfloat16_rn(v1 - __bfloat162float(q0));
    return uint32_t(__bfloat16_as_ushort(q0)) | (uint32_t(__bfloat16_as_ushort(q1)) << 16);
  } else {
    const __half q0 = __float2half_rn(v0);
    const __half q1 = __float2half_rn(v1 - __half2float(q0));
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
// use.  Rows are written frame-interleaved, K * FB words per thread.
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
  // b_{k0..k0+K} of frame fb (K + 1 values; the last feeds the pair slope)
  auto b_run = [&](int fb, int k0, float (&b)[K + 1]) {
    float v[K + 3];  // p_{k0-1} .. p_{k0+K+1}
#pragma unroll
    for (int j = 0; j < K + 3; ++j) {
      const int k = k0 - 1 + j;
      v[j] = (k >= 0 && k < n) ? load_sample<DT>(p.sig, row0[fb] + k) * sc[fb] : 0.0f;
    }
#pragma unroll
    for (int j = 0; j <= K; ++j) {
      const int k = k0 + j;
      float r;
      if (k >= n) r = 0.0f;
      else if (k == 0) r = 2.0f * v[j + 1];
      else if (k == n - 1) r = fmaf(-2.0f * float(k), v[j + 1] - v[j], 2.0f * v[j + 1]);
      else r = fmaf(-float(k), v[j + 2] - v[j], 2.0f * v[j + 1]);
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
    for (int k0 = threadIdx.x * K; k0 < n; k0 += blockDim.x * K) {
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
  for (int k0 = threadIdx.x * K; k0 < p.n_t_pad; k0 += blockDim.x * K) {
    uint32_t w[K * FB];
#pragma unroll
    for (int fb = 0; fb < FB; ++fb) {
      if (fb < fb_eff) {
        float b[K + 1];
        b_run(fb, k0, b);
#pragma unroll
        for (int j = 0; j < K; ++j) {
          if constexpr (FMT == kBF32) w[j * FB + fb] = __float_as_uint(b[j]);
          else w[j * FB + fb] = encode_pair<FMT>(b[j] * inv[fb], b[j + 1] * inv[fb]);
        }
      } else {
#pragma unroll
        for (int j = 0; j < K; ++j) w[j * FB + fb] = 0u;
      }
    }
    store_words<K * FB>(dst + int64_t(k0) * FB, w);
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

template <int DT, int FMT, int FB>
__global__ void __launch_bounds__(256) preprocess_kernel(const PreParams p) {
  // let the gather that depends on this kernel start its prologue now
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  preprocess_row<DT, FMT, FB>(p, blockIdx.x, blockIdx.y);
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
  preprocess_row<DT, FMT, FB>(q, int(loc % q.n_sensors), int(loc / q.n_sensors));
}

// ------------------------------------------------------------------ gather --
template <int N>
__device__ __forceinline__ void load_words(const uint32_t* src, uint32_t (&w)[N]) {
  if constexpr (N % 4 == 0) {
#pragma unroll
    for (int i = 0; i < N; i += 4) {
      const uint4 v = *reinterpret_cast<const uint4*>(src + i);
      w[i] = v.x; w[i + 1] = v.y; w[i + 2] = v.z; w[i + 3] = v.w;
    }
  } else if constexpr (N == 2) {
    const uint2 v = *reinterpret_cast<const uint2*>(src);
    w[0] = v.x; w[1] = v.y;
  } else {
    w[0] = src[0];
  }
}

// One sensor of a stage for this lane's 4 pixels and FB frames.
template <int P, int FB, int FMT>
__device__ __forceinline__ void gather_sensor(float (&acc)[FB][4], const float* su, const uint32_t* sm,
                                              const int* soff, const uint32_t* sw, int sl, int Wst) {
  const int off = soff[sl];
  const unsigned lim = unsigned(Wst - off);
  float mm[FB];
  {
    uint32_t mw[FB];
    load_words<FB>(sm + sl * FB, mw);
#pragma unroll
    for (int fb = 0; fb < FB; ++fb) mm[fb] = __uint_as_float(mw[fb]);
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const float uu = su[sl * P + x * 32];
    const unsigned i = min(unsigned(__float2int_rz(uu)), lim);
    const float ph = uu - float(i);
    const uint32_t* row = sw + size_t(i + unsigned(off)) * FB;
    uint32_t w0[FB];
    load_words<FB>(row, w0);
    if constexpr (FMT == kBF32) {
      uint32_t w1[FB];
      load_words<FB>(row + FB, w1);
#pragma unroll
      for (int fb = 0; fb < FB; ++fb) {
        const float b0 = __uint_as_float(w0[fb]), b1 = __uint_as_float(w1[fb]);
        acc[fb][x] = fmaf(mm[fb], fmaf(ph, b1 - b0, b0), acc[fb][x]);
      }
    } else if constexpr (FMT == kBBF16P) {
#pragma unroll
      for (int fb = 0; fb < FB; ++fb) {
        const float v = fmaf(ph, __uint_as_float(w0[fb] & 0xffff0000u), __uint_as_float(w0[fb] << 16));
        acc[fb][x] = fmaf(mm[fb], v, acc[fb][x]);
      }
    } else {
#pragma unroll
      for (int fb = 0; fb < FB; ++fb) {
        const float2 h = __half22float2(*reinterpret_cast<const __half2*>(&w0[fb]));
        acc[fb][x] = fmaf(mm[fb], fmaf(ph, h.y, h.x), acc[fb][x]);
      }
    }
  }
}

// Shared-memory layout of one pipeline stage (byte offsets):
//   u    [S][P] float            the tile's table rows of the stage's sensors
//   m    [S4][FB] float          multipliers w_s * sigma
//   off  [S4] int                window offset (rows) of each sensor
//   win  [Wst + 4][FB] words     the stage's windows packed at `off`, then 4
//                                zero rows that out-of-record pixels read
struct StageLayout {
  size_t u, m, off, win, bytes;
  __host__ __device__ StageLayout(int S, int P, int FB, int Wst) {
    const int S4 = (S + 3) & ~3;
    u = 0;
    m = u + size_t(S) * P * 4;
    off = m + size_t(S4) * FB * 4;
    win = off + size_t(S4) * 4;
    bytes = win + size_t(Wst + 4) * FB * 4;
  }
};

constexpr int kHeaderBytes = 512;   // mbarriers, unit ring and flags
constexpr int kMetaBytes = 2 * kMaxG * 4;

struct UnitPos {
  int inst, fg, tile, seg, s_lo, s_hi;
};

__device__ __forceinline__ UnitPos decode_unit(const StreamParams& p, int64_t u, int& inst) {
  while (inst + 1 < p.n_inst && u >= p.inst[inst + 1].unit_begin) ++inst;
  const InstDesc& d = p.inst[inst];
  const int64_t loc = u - d.unit_begin;
  const int64_t per_fg = int64_t(d.n_tiles) * d.n_seg;
  UnitPos q;
  q.inst = inst;
  q.fg = int(loc / per_fg);
  const int64_t r = loc - int64_t(q.fg) * per_fg;
  q.tile = int(r / d.n_seg);
  q.seg = int(r - int64_t(q.tile) * d.n_seg);
  q.s_lo = q.seg * d.G;
  q.s_hi = min(d.n_sensors, q.s_lo + d.G);
  return q;
}

constexpr int kRing = 16;  // unit indices in flight between the producer and the consumers

// Warp roles: consumers 0..NWC-1 (gather), producer NWC (copies), epilogues
// NWC+1 and NWC+2 (alternate units: phase sum, segment partials, tile sums).
// Units are handed out by an atomic ticket (sched[0]); the last CTA to finish
// resets the tickets (sched[1] counts finished CTAs), so a launch -- or a
// replay of a captured graph -- always starts from zero.
template <int P, int FB, int FMT, int SW>
__global__ void __launch_bounds__(32 * ((P / 128) * SW + 3))
    gather_kernel(const __grid_constant__ StreamParams p) {
  constexpr int PW = P / 128;   // warps across the tile's pixels
  constexpr int NWC = PW * SW;  // consumer warps
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kMaxStages;
  uint64_t* meta_bar = empty + kMaxStages;
  int64_t* unit_ring = reinterpret_cast<int64_t*>(meta_bar + 2);  // [kRing]
  int64_t* red_unit = unit_ring + kRing;                           // [2]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(red_unit + 2);
  int* meta = reinterpret_cast<int*>(smem + kHeaderBytes);  // [2][kMaxG] packed bases
  const StageLayout L(p.S, P, FB, p.Wst);
  unsigned char* stage0 = smem + kHeaderBytes + kMetaBytes;
  float* red = reinterpret_cast<float*>(stage0 + L.bytes * p.stages);  // [2][SW][FB][P]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int S4 = (p.S + 3) & ~3;
  const int64_t N = p.n_units;

  if (threadIdx.x == 0) {
    for (int st = 0; st < p.stages; ++st) {
      mbar_init(&full[st], 1);
      mbar_init(&empty[st], NWC);
    }
    mbar_init(&meta_bar[0], 1);
    mbar_init(&meta_bar[1], 1);
    *abort_flag = 0;
    mbar_init_fence();
  }
  // zero rows after the windows of every stage
  for (int q = threadIdx.x; q < p.stages * 4 * FB; q += blockDim.x) {
    const int st = q / (4 * FB), k = q - st * 4 * FB;
    reinterpret_cast<uint32_t*>(stage0 + st * L.bytes + L.win)[size_t(p.Wst) * FB + k] = 0u;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  if (warp == NWC) {
    // ------------------------------------------------------------ producer --
    int inst = 0;
    int64_t seq = 0;  // chunks (stage uses) issued by this CTA
    auto abort_now = [&]() {
      if (lane == 0) {
        atomicOr(p.status, kStatusTimeout);
        *abort_flag = 1;
      }
    };
    auto issue_meta = [&](int64_t u, int slot) {
      int ii = 0;
      const UnitPos q = decode_unit(p, u, ii);
      const InstDesc& d = p.inst[q.inst];
      const uint32_t n4 = uint32_t((q.s_hi - q.s_lo + 3) & ~3);
      if (lane == 0) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive_expect_tx(&meta_bar[slot], n4 * 4);
        bulk_g2s(meta + slot * kMaxG, d.base + int64_t(q.tile) * d.n_sensors_pad + q.s_lo, n4 * 4,
                 &meta_bar[slot]);
      }
    };
    // wait until stage st may be refilled (its previous use consumed)
    auto acquire_stage = [&](int st) -> bool {
      const int64_t use = seq / p.stages;
      if (use == 0) return true;
      if (mbar_wait_bounded(&empty[st], uint32_t((use - 1) & 1), p.timeout_ns, abort_flag)) return true;
      abort_now();
      return false;
    };
    // Issue stage st for sensors [s0, s0 + S) of unit q: the table block (part
    // & 1) and/or the multipliers and windows (part & 2), which come from the
    // preprocessing grid.  The stage's expected bytes are posted with the
    // table block (or with everything when part == 3).
    auto issue_chunk = [&](const UnitPos& q, const InstDesc& d, const int* mrow, int s0, int st,
                           int part) {
      const int se = min(p.S, q.s_hi - s0);
      const int se4 = (se + 3) & ~3;
      unsigned char* sb = stage0 + st * L.bytes;
      int bs = 0, wl = 0;
      if (lane < se) {
        const uint32_t word = uint32_t(mrow[s0 - q.s_lo + lane]);
        bs = int(word & 0xffffu);
        wl = int(word >> 16);
      }
      int incl = wl;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
      }
      const int total_w = __shfl_sync(0xffffffffu, incl, 31);
      int off = incl - wl;
      uint32_t wrows = uint32_t(total_w);
      if (total_w > p.Wst) {  // cannot happen with a host-computed Wst; stay in bounds
        if (lane == 0 && (part & 1)) atomicOr(p.status, kStatusBadConfig);
        wl = 0;
        off = 0;
        wrows = 0;
      }
      if (part & 1) {
        if (lane < S4) reinterpret_cast<int*>(sb + L.off)[lane] = lane < se ? off : 0;
        __syncwarp();
        const uint32_t bytes = uint32_t(se) * P * 4 + uint32_t(se4) * FB * 4 + wrows * FB * 4;
        if (lane == 0) {
          mbar_arrive_expect_tx(&full[st], bytes);
          bulk_g2s(sb + L.u, d.u + (int64_t(q.tile) * d.n_sensors + s0) * P, uint32_t(se) * P * 4,
                   &full[st]);
        }
      }
      if (part & 2) {
        if (lane == 0)
          bulk_g2s(sb + L.m, d.m + (int64_t(q.fg) * d.n_sensors_pad + s0) * FB,
                   uint32_t(se4) * FB * 4, &full[st]);
        if (wl > 0) {
          const unsigned char* src =
              static_cast<const unsigned char*>(d.b) +
              ((int64_t(q.fg) * d.n_sensors + s0 + lane) * d.n_t_pad + bs) * (FB * 4);
          bulk_g2s(sb + L.win + size_t(off) * FB * 4, src, uint32_t(wl) * FB * 4, &full[st]);
        }
      }
    };
    // the first unit of every CTA is blockIdx.x (no ticket round trip at the
    // start); later units come from the ticket, offset by the grid size
    auto next_ticket = [&]() -> int64_t {
      int64_t t = N;
      if (lane == 0)
        t = int64_t(gridDim.x) + int64_t(atomicAdd(reinterpret_cast<unsigned long long*>(p.sched), 1ull));
      return t;
    };
    int64_t t_cur = int64_t(blockIdx.x) < N ? int64_t(blockIdx.x) : N;
    int64_t t_next = t_cur < N ? next_ticket() : N;
    t_next = __shfl_sync(0xffffffffu, t_next, 0);
    if (t_next > N) t_next = N;
    if (t_cur < N) issue_meta(t_cur, 0);
    int64_t meta_last = t_cur < N ? 0 : -1;  // unit counter j of the last base copy requested
    bool ok = true;
    bool waited_inputs = false;
    int64_t j = 0;
    for (; t_cur < N && ok; ++j) {
      const int slot = int(j & 1);
      const UnitPos q = decode_unit(p, t_cur, inst);
      const InstDesc& d = p.inst[q.inst];
      if (!mbar_wait_bounded(&meta_bar[slot], uint32_t((j >> 1) & 1), p.timeout_ns, abort_flag)) {
        abort_now();
        break;
      }
      __syncwarp();
      int64_t t_next2 = N;
      if (t_next < N) {
        issue_meta(t_next, slot ^ 1);
        meta_last = j + 1;
        t_next2 = next_ticket();
      }
      if (lane == 0) unit_ring[j % kRing] = t_cur;
      const int* mrow = meta + slot * kMaxG;
      int s0 = q.s_lo;
      if (!waited_inputs) {
        // table blocks of the first stages stream while the preprocessing grid
        // still runs; its outputs (multipliers, windows) only after the wait
        const int64_t seq0 = seq;
        int k = 0;
        for (int s = q.s_lo; s < q.s_hi && k < p.stages; s += p.S, ++k)
          issue_chunk(q, d, mrow, s, int((seq0 + k) % p.stages), 1);
        asm volatile("griddepcontrol.wait;" ::: "memory");
        waited_inputs = true;
        for (int i = 0; i < k; ++i, s0 += p.S, ++seq)
          issue_chunk(q, d, mrow, s0, int(seq % p.stages), 2);
      }
      for (; s0 < q.s_hi; s0 += p.S, ++seq) {
        const int st = int(seq % p.stages);
        if (!acquire_stage(st)) {
          ok = false;
          break;
        }
        issue_chunk(q, d, mrow, s0, st, 3);
      }
      t_cur = t_next;
      t_next = __shfl_sync(0xffffffffu, t_next2, 0);
      if (t_next > N) t_next = N;
    }
    // end of work: an empty stage whose unit index is -1
    if (ok) {
      const int st = int(seq % p.stages);
      if (acquire_stage(st)) {
        if (lane == 0) {
          unit_ring[j % kRing] = -1;
          mbar_arrive(&full[st]);
        }
        ++seq;
      }
    }
    // drain the copies still in flight before the CTA may exit
    for (int64_t c = seq > p.stages ? seq - p.stages : 0; c < seq; ++c)
      mbar_wait_bounded(&full[c % p.stages], uint32_t((c / p.stages) & 1), p.timeout_ns, nullptr);
    if (meta_last >= 0)
      mbar_wait_bounded(&meta_bar[meta_last & 1], uint32_t((meta_last >> 1) & 1), p.timeout_ns, nullptr);
  } else if (warp < NWC) {
    // ------------------------------------------------------------ consumers --
    const int pg = warp % PW, sp = warp / PW;
    int inst = 0;
    int64_t seq = 0, j = 0;
    bool ok = true;
    auto wait_full = [&](int st) -> bool {
      if (mbar_wait_bounded(&full[st], uint32_t((seq / p.stages) & 1), p.timeout_ns, abort_flag)) return true;
      if (lane == 0) {
        atomicOr(p.status, kStatusTimeout);
        *abort_flag = 1;
      }
      return false;
    };
    for (;; ++j) {
      if (!wait_full(int(seq % p.stages))) break;
      const int64_t u = unit_ring[j % kRing];
      if (u < 0) break;
      const UnitPos q = decode_unit(p, u, inst);
      float acc[FB][4];
#pragma unroll
      for (int fb = 0; fb < FB; ++fb)
#pragma unroll
        for (int x = 0; x < 4; ++x) acc[fb][x] = 0.0f;
      for (int s0 = q.s_lo; s0 < q.s_hi; s0 += p.S, ++seq) {
        const int st = int(seq % p.stages);
        if (s0 != q.s_lo && !wait_full(st)) {
          ok = false;
          break;
        }
        const int se = min(p.S, q.s_hi - s0);
        const unsigned char* sb = stage0 + st * L.bytes;
        const float* su = reinterpret_cast<const float*>(sb + L.u) + pg * 128 + lane;
        const uint32_t* sm = reinterpret_cast<const uint32_t*>(sb + L.m);
        const int* soff = reinterpret_cast<const int*>(sb + L.off);
        const uint32_t* sw = reinterpret_cast<const uint32_t*>(sb + L.win);
        int sl = sp;
        for (; sl + SW < se; sl += 2 * SW) {
          gather_sensor<P, FB, FMT>(acc, su, sm, soff, sw, sl, p.Wst);
          gather_sensor<P, FB, FMT>(acc, su, sm, soff, sw, sl + SW, p.Wst);
        }
        if (sl < se) gather_sensor<P, FB, FMT>(acc, su, sm, soff, sw, sl, p.Wst);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[st]);
      }
      if (!ok) break;
      // hand the unit's sums to the epilogue warp j & 1 through red[j & 1]
      const int buf = int(j & 1);
      if (j >= 2) red_free_sync(buf, (NWC + 1) * 32);
      float* rb = red + size_t(buf) * SW * FB * P;
#pragma unroll
      for (int fb = 0; fb < FB; ++fb)
#pragma unroll
        for (int x = 0; x < 4; ++x) rb[(sp * FB + fb) * P + pg * 128 + x * 32 + lane] = acc[fb][x];
      if (threadIdx.x == 0) red_unit[buf] = u;
      red_full_arrive(buf, (NWC + 1) * 32);
    }
    // no more units: one end marker for each epilogue warp
    for (int e = 0; e < 2; ++e) {
      const int64_t idx = j + e;
      const int buf = int(idx & 1);
      if (idx >= 2) red_free_sync(buf, (NWC + 1) * 32);
      if (threadIdx.x == 0) red_unit[buf] = -1;
      red_full_arrive(buf, (NWC + 1) * 32);
    }
  } else {
    // ------------------------------------------------------------ epilogues --
    const int ew = warp - NWC - 1;
    for (int i = 0; i < p.n_inst; ++i) {
      const InstDesc& d = p.inst[i];
      for (int f = 0; f < d.n_frames && d.n_zero_runs > 0; ++f)
        for (int64_t r = int64_t(blockIdx.x) * 2 + ew; r < d.n_zero_runs; r += int64_t(gridDim.x) * 2) {
          const int st0 = d.zero_runs[2 * r], len = d.zero_runs[2 * r + 1];
          float* o = d.out + int64_t(f) * d.out_stride + st0;
          for (int i2 = lane; i2 < len; i2 += 32) o[i2] = 0.0f;
        }
    }
    constexpr int KO = P / 32;  // outputs of one frame per lane
    int inst = 0;
    for (;;) {
      red_full_sync(ew, (NWC + 1) * 32);
      const int64_t u = red_unit[ew];
      if (u < 0) break;
      const UnitPos q = decode_unit(p, u, inst);
      const InstDesc& d = p.inst[q.inst];
      const int f0 = q.fg * FB;
      const int fb_eff = min(FB, d.n_frames - f0);
      const float* rb = red + size_t(ew) * SW * FB * P;
      float v[FB][KO];
#pragma unroll
      for (int fb = 0; fb < FB; ++fb)
#pragma unroll
        for (int k = 0; k < KO; ++k) {
          const int o = fb * P + k * 32 + lane;
          float a = 0.0f;
#pragma unroll
          for (int ph = 0; ph < SW; ++ph) a += rb[ph * FB * P + o];  // fixed phase order
          v[fb][k] = a;
        }
      red_free_arrive(ew, (NWC + 1) * 32);  // red[ew] free again
      int slot_idx[KO];
#pragma unroll
      for (int k = 0; k < KO; ++k) slot_idx[k] = __ldg(d.slot + int64_t(q.tile) * P + k * 32 + lane);
      const int64_t pbase = ((int64_t(q.fg) * d.n_tiles + q.tile) * d.n_seg) * FB * P;
      if (d.n_seg == 1) {
#pragma unroll
        for (int fb = 0; fb < FB; ++fb)
#pragma unroll
          for (int k = 0; k < KO; ++k)
            if (fb < fb_eff && slot_idx[k] >= 0) d.out[int64_t(f0 + fb) * d.out_stride + slot_idx[k]] = v[fb][k];
        continue;
      }
      float* mine = d.part + pbase + int64_t(q.seg) * FB * P;
#pragma unroll
      for (int fb = 0; fb < FB; ++fb)
#pragma unroll
        for (int k = 0; k < KO; ++k) __stcg(mine + fb * P + k * 32 + lane, v[fb][k]);
      // the last segment of a tile to finish sums all segments in fixed order;
      // the counter's release/acquire orders the partials of every lane (the
      // warp barrier before it makes the other lanes' stores part of the release)
      __syncwarp();
      int last = 0;
      if (lane == 0) last = atomic_add_acq_rel(d.counter + int64_t(q.fg) * d.n_tiles + q.tile, 1) == d.n_seg - 1;
      last = __shfl_sync(0xffffffffu, last, 0);
      if (!last) continue;
#pragma unroll
      for (int fb = 0; fb < FB; ++fb) {
        if (fb >= fb_eff) break;
        float t[KO];
#pragma unroll
        for (int k = 0; k < KO; ++k) t[k] = 0.0f;
        for (int sg = 0; sg < d.n_seg; ++sg) {
          const float* src = d.part + pbase + int64_t(sg) * FB * P + fb * P + lane;
          float x[KO];
#pragma unroll
          for (int k = 0; k < KO; ++k) x[k] = __ldcg(src + k * 32);
#pragma unroll
          for (int k = 0; k < KO; ++k) t[k] += x[k];
        }
#pragma unroll
        for (int k = 0; k < KO; ++k)
          if (slot_idx[k] >= 0) d.out[int64_t(f0 + fb) * d.out_stride + slot_idx[k]] = t[k];
      }
      __syncwarp();
      if (lane == 0) atomicExch(d.counter + int64_t(q.fg) * d.n_tiles + q.tile, 0);
    }
  }
  // the last CTA out resets the unit tickets for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(p.sched + 2, 1u) == gridDim.x - 1) {
      atomicExch(reinterpret_cast<unsigned long long*>(p.sched), 0ull);
      atomicExch(p.sched + 2, 0u);
    }
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
int gather_threads(const GatherConfig& c) { return 32 * ((c.P / 128) * c.SW + 3); }

size_t gather_smem_bytes(const GatherConfig& c, int Wst) {
  const StageLayout L(c.S, c.P, c.FB, Wst);
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

template <int P, int FB, int FMT, int SW>
static cudaError_t gather_t(const StreamParams& p, size_t smem, int grid, cudaStream_t st,
                            int* resident, int n_sm) {
  auto kern = gather_kernel<P, FB, FMT, SW>;
  static size_t smem_set = 0;  // largest dynamic smem granted so far (per instantiation)
  if (smem > smem_set) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
    if (e != cudaSuccess) return e;
    smem_set = smem;
  }
  const int threads = 32 * ((P / 128) * SW + 3);
  if (resident) {
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem);
    if (e != cudaSuccess) return e;
    *resident = per_sm * n_sm;
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, p);
}

template <int P, int FMT, int SW>
static cudaError_t gather_fb(int FB, const StreamParams& p, size_t smem, int grid, cudaStream_t st,
                             int* resident, int n_sm) {
  switch (FB) {
    case 1: return gather_t<P, 1, FMT, SW>(p, smem, grid, st, resident, n_sm);
    case 2: return gather_t<P, 2, FMT, SW>(p, smem, grid, st, resident, n_sm);
    case 4: return gather_t<P, 4, FMT, SW>(p, smem, grid, st, resident, n_sm);
    case 8: return gather_t<P, 8, FMT, SW>(p, smem, grid, st, resident, n_sm);
    default: return cudaErrorInvalidValue;
  }
}

static cudaError_t gather_dispatch(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                                   cudaStream_t st, int* resident, int n_sm) {
  const size_t smem = gather_smem_bytes(c, p.Wst);
  if (c.P == 128 && c.SW == 4) {
    if (fmt == kBF32) return gather_fb<128, kBF32, 4>(c.FB, p, smem, grid, st, resident, n_sm);
    if (fmt == kBBF16P) return gather_fb<128, kBBF16P, 4>(c.FB, p, smem, grid, st, resident, n_sm);
    if (fmt == kBF16P) return gather_fb<128, kBF16P, 4>(c.FB, p, smem, grid, st, resident, n_sm);
  } else if (c.P == 256 && c.SW == 2) {
    if (fmt == kBF32) return gather_fb<256, kBF32, 2>(c.FB, p, smem, grid, st, resident, n_sm);
    if (fmt == kBBF16P) return gather_fb<256, kBBF16P, 2>(c.FB, p, smem, grid, st, resident, n_sm);
    if (fmt == kBF16P) return gather_fb<256, kBF16P, 2>(c.FB, p, smem, grid, st, resident, n_sm);
  }
  return cudaErrorInvalidValue;
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
  return gather_dispatch(c, fmt, p, grid, st, nullptr, 0);
}

// Kernel entry addresses (identify graph nodes when refreshing their parameters).
template <int P, int FMT, int SW>
static const void* gather_func_fb(int FB) {
  switch (FB) {
    case 1: return reinterpret_cast<const void*>(gather_kernel<P, 1, FMT, SW>);
    case 2: return reinterpret_cast<const void*>(gather_kernel<P, 2, FMT, SW>);
    case 4: return reinterpret_cast<const void*>(gather_kernel<P, 4, FMT, SW>);
    case 8: return reinterpret_cast<const void*>(gather_kernel<P, 8, FMT, SW>);
  }
  return nullptr;
}

const void* gather_kernel_func(const GatherConfig& c, int fmt) {
  if (c.P == 128 && c.SW == 4) {
    if (fmt == kBF32) return gather_func_fb<128, kBF32, 4>(c.FB);
    if (fmt == kBBF16P) return gather_func_fb<128, kBBF16P, 4>(c.FB);
    if (fmt == kBF16P) return gather_func_fb<128, kBF16P, 4>(c.FB);
  } else if (c.P == 256 && c.SW == 2) {
    if (fmt == kBF32) return gather_func_fb<256, kBF32, 2>(c.FB);
    if (fmt == kBBF16P) return gather_func_fb<256, kBBF16P, 2>(c.FB);
    if (fmt == kBF16P) return gather_func_fb<256, kBF16P, 2>(c.FB);
  }
  return nullptr;
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
