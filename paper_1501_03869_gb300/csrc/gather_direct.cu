// gather_direct.cu -- the single-frame gather of Eq. (BP) without the staged
// pipeline.
//
// Two gathers share the reduction kernel below.  gather_window_kernel (stored
// tables without weights, every window at most 288 samples) copies each
// sensor's integrand window into shared memory per warp and interpolates
// there; gather_direct_kernel, described next, gathers from L2 and takes every
// other case.  Both give the same bits.
//
// Two launches.  The gather kernel is persistent: CTA c takes units (tile,
// segment of G sensors) c, c + grid, c + 2 grid, ... in tile-major order, and
// (constant speed) asks L2 for each unit's delay data two units ahead with one
// bulk prefetch.
// Its warps are the (pixel group, sensor phase) pairs of the staged kernel's
// consumers; a warp reads the delay data (table offsets, or the constant-
// speed anchors) and the window bases for a chunk of its sensors, then
// gathers the integrand rows from L2 with loads that never branch (an arrival
// after the record reads a zero padding row), and finally stores its phase
// sums -- no barrier, fence or atomic anywhere, so no warp ever waits for
// another.  The reduction kernel then forms every pixel's sum over phases and
// segments and scatters it to the image.
//
// Both kernels are launched as programmatic dependents, which can start before
// the kernels ahead of them in the stream have finished; lines that an earlier
// kernel left in an SM's L1 are then not reliably dropped, so every global load
// here goes through L2 only (ld.global.cg), never the non-coherent L1 path.
//
// Arithmetic and summation order are those of the staged kernel with one
// frame per unit (gather.cuh): phase sp of a segment accumulates sensors
// s_lo + sp, s_lo + sp + SW, ... with acc = fma(m_s, fma(ph, b1 - b0, b0), acc),
// phases are summed in order 0..SW-1 and segments in order 0..n_seg-1.  A frame
// therefore gives the same bits here as inside any batch that the staged kernel
// reconstructs.
//
// With solid-angle weights (WGT = 1, the exact back projection of Sec. II-C)
// each term carries its own weight w(pixel, sensor), evaluated from the
// sensor's 32-byte weight anchor and the pixel's position terms by the same
// function as the staged kernel: acc = fma(m_s, w * lerp, acc).
#include <algorithm>

#include "gather.cuh"

namespace patbp {

namespace {

constexpr int kDirectChunk = 1;    // sensors of a phase whose loads are issued together
constexpr int kDirectMinCtas = 8;  // resident CTAs per SM the registers must allow

struct DirectParams {
  const float* u;
  const float* anchor;
  const float4* pix;
  const float* wanchor;
  const int32_t* base;
  const int32_t* slot;
  const int32_t* zero_runs;
  const void* b;
  const float* m;
  float* out;
  float* part;  // [n_tiles][n_seg][SW][P] phase sums
  int* status;
  int* host_status;  // the reduction copies *status here when set
  uint64_t timeout_ns;  // bound of every device-side wait
  int n_zero_runs, n_sensors, n_sensors_pad, n_t_pad, n_tiles, n_seg, G;
  int W;  // longest window of one (tile, sensor) (rows)
};

// One sensor's contribution to this lane's 4 pixels; `row` points at the
// sensor's window base in the integrand.  Offsets above `cap` are after the
// record: they read the zero row `zrow` (a padding row after the record) with
// phase 0, which adds m * 0 exactly as the staged kernel's zero rows do.
template <int FMT, int WGT>
__device__ __forceinline__ void direct_accumulate(float (&acc)[4], const float (&uu)[4], float cap,
                                                  const uint32_t* row, unsigned zrow, float mm,
                                                  const float (&ww)[4]) {
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const bool in = uu[x] <= cap;
    const unsigned t = unsigned(__float2int_rz(uu[x]));
    const unsigned i = in ? t : zrow;
    const float ph = in ? uu[x] - float(t) : 0.0f;
    const uint32_t w0 = __ldcg(row + i);
    float v;
    if constexpr (FMT == kBF32) {
      const float b0 = __uint_as_float(w0), b1 = __uint_as_float(__ldcg(row + i + 1));
      v = fmaf(ph, b1 - b0, b0);
    } else if constexpr (FMT == kBBF16P) {
      v = fmaf(ph, __uint_as_float(w0 & 0xffff0000u), __uint_as_float(w0 << 16));
    } else {
      const float2 h = __half22float2(*reinterpret_cast<const __half2*>(&w0));
      v = fmaf(ph, h.y, h.x);
    }
    if constexpr (WGT != 0) v = __fmul_rn(ww[x], v);
    acc[x] = fmaf(mm, v, acc[x]);
  }
}

__device__ __forceinline__ void bulk_prefetch_l2(const void* src, uint32_t bytes) {
  asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

// Pull the delay data of `unit` (one contiguous block) into L2.
template <int P, int DELAYS>
__device__ __forceinline__ void prefetch_unit(const DirectParams& p, int64_t unit, int64_t n_units) {
  if (unit >= n_units) return;
  const int tile = int(unit / p.n_seg), seg = int(unit - int64_t(tile) * p.n_seg);
  const int s_lo = seg * p.G, n = min(p.n_sensors, s_lo + p.G) - s_lo;
  if constexpr (DELAYS == 0)
    bulk_prefetch_l2(p.u + (int64_t(tile) * p.n_sensors + s_lo) * P, uint32_t(n) * P * 4);
  else
    bulk_prefetch_l2(p.anchor + (int64_t(tile) * p.n_sensors_pad + s_lo) * 8, uint32_t(n) * 32);
}

template <int P, int SW, int FMT, int DELAYS, int WGT>
__global__ void __launch_bounds__(32 * (P / 128) * SW, kDirectMinCtas)
    gather_direct_kernel(const __grid_constant__ DirectParams p) {
  constexpr int PW = P / 128;
  constexpr int CH = kDirectChunk;
  // the reduction kernel may start now; it waits for this grid's results
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pg = warp % PW, sp = warp / PW;
  const int px0 = pg * 128 + lane;
  const int64_t n_units = int64_t(p.n_tiles) * p.n_seg;
  if (DELAYS != 0 && threadIdx.x == 0) {
    prefetch_unit<P, DELAYS>(p, blockIdx.x, n_units);
    prefetch_unit<P, DELAYS>(p, int64_t(blockIdx.x) + gridDim.x, n_units);
  }
  const uint32_t* bsrc = static_cast<const uint32_t*>(p.b);
  bool waited = false;
  for (int64_t unit = blockIdx.x; unit < n_units; unit += gridDim.x) {
    if (DELAYS != 0 && threadIdx.x == 0)
      prefetch_unit<P, DELAYS>(p, unit + 2 * int64_t(gridDim.x), n_units);
    const int tile = int(unit / p.n_seg);
    const int seg = int(unit - int64_t(tile) * p.n_seg);
    const int s_lo = seg * p.G, s_hi = min(p.n_sensors, s_lo + p.G);
    float4 pq[4];
    if constexpr (DELAYS != 0 || WGT != 0) {
#pragma unroll
      for (int x = 0; x < 4; ++x) pq[x] = __ldcg(p.pix + int64_t(tile) * P + px0 + x * 32);
    }
    const float4* wrow = WGT != 0 ? reinterpret_cast<const float4*>(p.wanchor) +
                                        int64_t(tile) * p.n_sensors_pad * 2
                                  : nullptr;
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    float ww[4] = {1.0f, 1.0f, 1.0f, 1.0f};
    if constexpr (DELAYS == 0) {
      // Table offsets: one sensor at a time, software-pipelined -- the next
      // sensor's offsets and window base are in flight while this one
      // gathers (the first ones before waiting for the preprocessing grid).
      float un[4];
      uint32_t bn = 0u;
      float4 wn0 = make_float4(0.f, 0.f, 0.f, 0.f), wn1 = wn0;
      auto load_next = [&](int s) {
        bn = uint32_t(__ldcg(p.base + int64_t(tile) * p.n_sensors_pad + s));
        const float* urow = p.u + (int64_t(tile) * p.n_sensors + s) * P + px0;
#pragma unroll
        for (int x = 0; x < 4; ++x) un[x] = __ldcg(urow + x * 32);
        if constexpr (WGT != 0) {
          wn0 = __ldcg(wrow + 2 * s);
          wn1 = __ldcg(wrow + 2 * s + 1);
        }
      };
      if (s_lo + sp < s_hi) load_next(s_lo + sp);
      for (int s = s_lo + sp; s < s_hi; s += SW) {
        const float uu[4] = {un[0], un[1], un[2], un[3]};
        const unsigned bs = bn & 0xffffu;
        if constexpr (WGT != 0) solid_angle_weights(ww, pq, wn0, wn1);
        if (s + SW < s_hi) load_next(s + SW);
        if (!waited) {
          // integrand and multipliers come from the preprocessing grid
          asm volatile("griddepcontrol.wait;" ::: "memory");
          waited = true;
        }
        const float mm = __ldcg(p.m + s);
        const uint32_t* row = bsrc + int64_t(s) * p.n_t_pad + bs;
        direct_accumulate<FMT, WGT>(acc, uu, 1.0e29f, row, unsigned(p.n_t_pad - 1) - bs, mm, ww);
      }
    } else {
      // Sensors of this phase in chunks of CH: the loads that do not depend on
      // the preprocessing (delay data, window bases) are issued for the chunk
      // first -- for the first chunk before waiting for the preprocessing grid.
      for (int c0 = s_lo + sp; c0 < s_hi; c0 += CH * SW) {
        uint32_t bw[CH];
        float uu[CH][4];
        float4 an[DELAYS ? CH : 1][2];
        float4 wa[WGT ? CH : 1][2];
  #pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int s = c0 + j * SW;
          const bool ok = s < s_hi;
          bw[j] = ok ? uint32_t(__ldcg(p.base + int64_t(tile) * p.n_sensors_pad + s)) : 0u;
          if constexpr (DELAYS == 0) {
            const float* urow = p.u + (int64_t(tile) * p.n_sensors + s) * P + px0;
  #pragma unroll
            for (int x = 0; x < 4; ++x) uu[j][x] = ok ? __ldcg(urow + x * 32) : kFarOffset;
          } else {
            const float4* ap = reinterpret_cast<const float4*>(p.anchor) +
                               (int64_t(tile) * p.n_sensors_pad + (ok ? s : s_lo)) * 2;
            an[j][0] = __ldcg(ap);
            an[j][1] = __ldcg(ap + 1);
            if (!ok) an[j][1].y = -1.0f;  // cap below every offset: nothing to add
          }
          if constexpr (WGT != 0) {
            wa[j][0] = __ldcg(wrow + 2 * (ok ? s : s_lo));
            wa[j][1] = __ldcg(wrow + 2 * (ok ? s : s_lo) + 1);
          }
        }
        if (!waited) {
          // integrand and multipliers come from the preprocessing grid
          asm volatile("griddepcontrol.wait;" ::: "memory");
          waited = true;
        }
        float mm[CH];
  #pragma unroll
        for (int j = 0; j < CH; ++j) mm[j] = c0 + j * SW < s_hi ? __ldcg(p.m + c0 + j * SW) : 0.0f;
  #pragma unroll
        for (int j = 0; j < CH; ++j) {
          const int s = min(c0 + j * SW, s_hi - 1);
          if constexpr (DELAYS != 0) {
            const float4 A = an[j][0], B = an[j][1];
            if (B.w == 0.0f) {
              const float m2u0 = -2.0f * A.w;
  #pragma unroll
              for (int x = 0; x < 4; ++x) {
                const float num =
                    fmaf(pq[x].x, A.x, fmaf(pq[x].y, A.y, fmaf(pq[x].z, A.z, pq[x].w)));
                const float sq = num + B.z;
                const float y = rsqrtf(sq);
                const float da = sq * y - A.w;
                const float r = fmaf(-da, da, fmaf(m2u0, da, num));
                const float v = fmaf(r, 0.5f * y, da) + B.x;
                uu[j][x] = v > B.y ? kFarOffset : fmaxf(v, 0.0f);
              }
            } else {
  #pragma unroll
              for (int x = 0; x < 4; ++x) {
                const float d0 = fmaf(0.5f, pq[x].x, A.x), d1 = fmaf(0.5f, pq[x].y, A.y),
                            d2 = fmaf(0.5f, pq[x].z, A.z);
                const float sq = fmaxf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)), 1.0e-30f);
                const float v = (sq * rsqrtf(sq) - A.w) + B.x;
                uu[j][x] = v > B.y ? kFarOffset : fmaxf(v, 0.0f);
              }
            }
          }
          const unsigned bs = bw[j] & 0xffffu;
          const uint32_t* row = bsrc + int64_t(s) * p.n_t_pad + bs;
          if constexpr (WGT != 0) solid_angle_weights(ww, pq, wa[j][0], wa[j][1]);
          direct_accumulate<FMT, WGT>(acc, uu[j], 1.0e29f, row, unsigned(p.n_t_pad - 1) - bs, mm[j],
                                      ww);
        }
      }
    }
    float* dst = p.part + ((int64_t(tile) * p.n_seg + seg) * SW + sp) * P + px0;
#pragma unroll
    for (int x = 0; x < 4; ++x) dst[x * 32] = acc[x];
  }
  if (!waited) asm volatile("griddepcontrol.wait;" ::: "memory");
}

// Sum of every pixel over phases (in order) and segments (in order), written
// to its place in the image (SW = 1: the part buffer holds segment sums); also clears the image outside the mask.  The
// loads of 8 segments are issued before their sums, so a pixel costs about
// one L2 round trip per 8 segments.
template <int P, int SW>
__global__ void __launch_bounds__(256) direct_reduce_kernel(const __grid_constant__ DirectParams p) {
  constexpr int K = 8;
  for (int64_t r = blockIdx.x; r < p.n_zero_runs; r += gridDim.x) {
    const int st0 = p.zero_runs[2 * r], len = p.zero_runs[2 * r + 1];
    for (int i2 = threadIdx.x; i2 < len; i2 += blockDim.x) p.out[st0 + i2] = 0.0f;
  }
  asm volatile("griddepcontrol.wait;" ::: "memory");
  // the kernels before this one are complete: their status is final
  if (p.host_status && blockIdx.x == 0 && threadIdx.x == 0) *p.host_status = __ldcg(p.status);
  const int64_t n = int64_t(p.n_tiles) * P;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < n;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int o = __ldcg(p.slot + idx);
    const int64_t tile = idx / P;
    const int q = int(idx - tile * P);
    const float* src = p.part + tile * p.n_seg * SW * P + q;
    float t = 0.0f;
    for (int s0 = 0; s0 < p.n_seg; s0 += K) {
      // (the first batch is loaded together with the slot, before its test)
      float x[K][SW];
#pragma unroll
      for (int k = 0; k < K; ++k)
#pragma unroll
        for (int ph = 0; ph < SW; ++ph)
          x[k][ph] = s0 + k < p.n_seg ? __ldcg(src + (int64_t(s0 + k) * SW + ph) * P) : 0.0f;
      if (o < 0) break;
#pragma unroll
      for (int k = 0; k < K; ++k) {
        if (s0 + k >= p.n_seg) break;
        if constexpr (SW == 1) {
          t += x[k][0];  // phases already summed, in the same order, by the gather
        } else {
          float v = 0.0f;
#pragma unroll
          for (int ph = 0; ph < SW; ++ph) v += x[k][ph];
          t += v;
        }
      }
    }
    if (o >= 0) p.out[o] = t;
  }
}

// ------------------------------------------------------ windowed variant --
// Stored tables without solid-angle weights, when every window of the table
// fits a shared-memory slot of WB rows.  The four warps of a CTA are the four
// (pixel group, sensor phase) pairs of one unit, as above; a warp takes its
// sensors two at a time.  For each sensor it copies the tile's integrand
// window (rows base .. base + len) into a slot of its own with 16-byte
// cp.async copies, two steps ahead, while its lanes' table offsets come from
// global memory one step ahead; the interpolation then reads shared memory.
// Each slot ends in 8 zero rows at row WB: an offset after the record (the
// table's out-of-record value) is clamped to WB, which gives phase 0 and the
// zero rows, so it adds m * 0 as in the kernel above.  The CTA sums its four
// phase sums per pixel in order before storing, so the reduction kernel sums
// segments only.  Arithmetic and summation order are those of
// gather_direct_kernel: the image has the same bits.
//
// Offsets in the window are found from the FP32 bits: for 0 <= u < 2^23,
// u + 2^23 rounded toward zero is 2^23 + floor(u) exactly, its bit pattern is
// 0x4B000000 + floor(u), and (u + 2^23) - 2^23 = floor(u) exactly.
constexpr int kWindowMaxRows = 288;  // largest slot (rows); longer windows take the kernel above

template <int P, int SW, int FMT, int WB>
__global__ void __launch_bounds__(128, kDirectMinCtas + 1)
    gather_window_kernel(const __grid_constant__ DirectParams p) {
  constexpr int PW = P / 128;
  static_assert(PW * SW == 4, "a unit is four warps");
  constexpr int SLOT = WB + 8;  // rows of one slot: window, then 8 zero rows
  constexpr int D = 2;          // steps of two sensors whose windows are in flight
  constexpr int NC = (WB + 127) / 128;  // 16-byte copies per lane for one window
  __shared__ __align__(16) uint32_t swin[4][2 * D][SLOT];
  __shared__ __align__(16) uint2 sbm[4][32];  // (window base word, multiplier) per sensor of the warp
  __shared__ float ssum[SW][P];
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int pg = warp % PW, sp = warp / PW;
  const int px0 = pg * 128 + lane;
  uint32_t* ring = &swin[warp][0][0];
  for (int k = lane; k < 2 * D * 8; k += 32) ring[(k >> 3) * SLOT + WB + (k & 7)] = 0u;
  const uint32_t ring_s = smem_addr(ring);
  const int64_t n_units = int64_t(p.n_tiles) * p.n_seg;
  const uint32_t* bsrc = static_cast<const uint32_t*>(p.b);
  const uint2* bm = sbm[warp];
  // integrand and multipliers come from the preprocessing grid
  asm volatile("griddepcontrol.wait;" ::: "memory");
  for (int64_t unit = blockIdx.x; unit < n_units; unit += gridDim.x) {
    const int tile = int(unit / p.n_seg);
    const int seg = int(unit - int64_t(tile) * p.n_seg);
    const int s_lo = seg * p.G, s_hi = min(p.n_sensors, s_lo + p.G);
    const int s0 = s_lo + sp;  // this warp's sensors: s0, s0 + SW, ...
    const int nj = s0 < s_hi ? (s_hi - s0 + SW - 1) / SW : 0;  // <= 32 (G <= 32 SW)
    const float* ubase = p.u + (int64_t(tile) * p.n_sensors + s0) * P + px0;
    if (unit != int64_t(blockIdx.x) && threadIdx.x == 0) {
      // a CTA's later units (launches with more units than resident CTAs)
      // start at staggered times: their table block is asked into L2 at once.
      // (Not the first unit: every CTA asking for its block at the launch's
      // start delayed the first offsets behind the whole table.)
      const int n_sen = s_hi - s_lo;
      bulk_prefetch_l2(p.u + (int64_t(tile) * p.n_sensors + s_lo) * P, uint32_t(n_sen) * P * 4);
    }
    const uint32_t* wsrc = bsrc + int64_t(s0) * p.n_t_pad + lane * 4;
    const int64_t ustep = int64_t(SW) * P, wstep = int64_t(SW) * p.n_t_pad;
    // the lanes' offsets of the sensors 2k, 2k + 1
    auto load_u = [&](int k, float (&d)[2][4]) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float* ur = ubase + min(2 * k + h, nj - 1) * ustep;
#pragma unroll
        for (int x = 0; x < 4; ++x) d[h][x] = __ldcg(ur + 32 * x);
      }
    };
    const int nk = (nj + 1) >> 1;
    float un[2][4];
    if (nk > 0) load_u(0, un);  // in flight with the window bases below
    if (lane < nj) {
      const int s = s0 + lane * SW;
      sbm[warp][lane] = make_uint2(uint32_t(__ldcg(p.base + int64_t(tile) * p.n_sensors_pad + s)),
                                   __float_as_uint(__ldcg(p.m + s)));
    }
    __syncwarp();
    // windows of the sensors 2k, 2k + 1 into slots 2 slot, 2 slot + 1; one group per step
    auto issue = [&](int k, int slot) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = 2 * k + h;
        if (j < nj) {
          const uint32_t b = bm[j].x;
          const int len = int(b >> 16);
          const uint32_t sa = ring_s + uint32_t(((2 * slot + h) * SLOT + lane * 4) * 4);
          const uint32_t* src = wsrc + j * wstep + (b & 0xffffu);
#pragma unroll
          for (int c = 0; c < NC; ++c)
            if (lane * 4 + c * 128 < len) cp_async16(sa + c * 512, src + c * 128);
        }
      }
      cp_async_commit();
    };
    // interpolation of one sensor at the lane's 4 offsets; wadj = the slot's
    // row 0 minus 4 * 0x4B000000 (shared addresses wrap modulo 2^32)
    auto lerp4 = [&](uint32_t wadj, const float (&uu)[4], float (&v)[4]) {
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        const float uc = fminf(uu[x], float(WB));
        const float t = __fadd_rz(uc, 8388608.0f);
        const float ph = __fsub_rn(uc, __fsub_rn(t, 8388608.0f));
        const uint32_t a = wadj + 4u * __float_as_uint(t);
        const uint32_t w0 = lds_u32(a);
        if constexpr (FMT == kBF32) {
          const float b0 = __uint_as_float(w0), b1 = __uint_as_float(lds_u32(a + 4));
          v[x] = fmaf(ph, b1 - b0, b0);
        } else if constexpr (FMT == kBBF16P) {
          v[x] = fmaf(ph, __uint_as_float(w0 & 0xffff0000u), __uint_as_float(w0 << 16));
        } else {
          const float2 hf = __half22float2(*reinterpret_cast<const __half2*>(&w0));
          v[x] = fmaf(ph, hf.y, hf.x);
        }
      }
    };
#pragma unroll
    for (int k = 0; k < D; ++k) issue(k, k);
    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    int slot = 0;
    for (int k = 0; k < nk; ++k) {
      float uc[2][4];
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int x = 0; x < 4; ++x) uc[h][x] = un[h][x];
      if (k + 1 < nk) load_u(k + 1, un);
      cp_async_wait<D - 1>();
      __syncwarp();
      const int j = 2 * k;
      const uint4 q = *reinterpret_cast<const uint4*>(bm + j);  // sensors j and j + 1
      const uint32_t wa = ring_s + uint32_t(2 * slot * SLOT * 4) - 4u * 0x4B000000u;
      float va[4];
      lerp4(wa, uc[0], va);
      if (j + 1 < nj) {
        float vb[4];
        lerp4(wa + SLOT * 4, uc[1], vb);
        const float ma = __uint_as_float(q.y), mb = __uint_as_float(q.w);
#pragma unroll
        for (int x = 0; x < 4; ++x) acc[x] = fmaf(mb, vb[x], fmaf(ma, va[x], acc[x]));
      } else {
        const float ma = __uint_as_float(q.y);
#pragma unroll
        for (int x = 0; x < 4; ++x) acc[x] = fmaf(ma, va[x], acc[x]);
      }
      __syncwarp();  // every lane has read the slots before they are refilled
      issue(k + D, slot);
      slot ^= 1;
    }
    cp_async_wait<0>();
#pragma unroll
    for (int x = 0; x < 4; ++x) ssum[sp][px0 + 32 * x] = acc[x];
    __syncthreads();
    for (int q = threadIdx.x; q < P; q += 128) {
      float v = 0.0f;
#pragma unroll
      for (int ph = 0; ph < SW; ++ph) v += ssum[ph][q];
      p.part[(int64_t(tile) * p.n_seg + seg) * P + q] = v;
    }
    __syncthreads();
  }
}

template <typename K>
cudaError_t launch_pdl(K kern, unsigned grid, unsigned threads, const DirectParams& dp, cudaStream_t st) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid, 1u, 1u);
  cfg.blockDim = dim3(threads, 1u, 1u);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, dp);
}

constexpr int kMaxDevices = 64;

// Resident CTAs per SM of one kernel, looked up once per device (devices of a
// process may differ).
struct PerDevice {
  int per_sm[kMaxDevices] = {};
};

template <int P, int SW, int FMT, int DELAYS, int WGT>
cudaError_t launch_direct_fmt(const DirectParams& dp, int n_sm, cudaStream_t st, bool reduce) {
  auto kern = gather_direct_kernel<P, SW, FMT, DELAYS, WGT>;
  const int threads = 32 * (P / 128) * SW;
  static PerDevice cache;  // resident CTAs per SM, per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (cache.per_sm[dev] == 0) {
    int v = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, threads, 0);
    if (e != cudaSuccess) return e;
    cache.per_sm[dev] = v > 0 ? v : 1;
  }
  const int64_t n_units = int64_t(dp.n_tiles) * dp.n_seg;
  const unsigned grid = unsigned(std::min<int64_t>(n_units, int64_t(cache.per_sm[dev]) * n_sm));
  e = launch_pdl(kern, grid, unsigned(threads), dp, st);
  if (e != cudaSuccess || !reduce) return e;
  const int64_t n = int64_t(dp.n_tiles) * P;
  const unsigned rgrid = unsigned(std::min<int64_t>((n + 255) / 256, int64_t(n_sm) * 8));
  return launch_pdl(direct_reduce_kernel<P, SW>, std::max(rgrid, 1u), 256u, dp, st);
}

template <int P, int SW, int FMT, int WB>
cudaError_t launch_window_fmt(const DirectParams& dp, int n_sm, cudaStream_t st, bool reduce) {
  auto kern = gather_window_kernel<P, SW, FMT, WB>;
  static PerDevice cache;  // resident CTAs per SM, per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  if (cache.per_sm[dev] == 0) {
    int v = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, kern, 128, 0);
    if (e != cudaSuccess) return e;
    cache.per_sm[dev] = v > 0 ? v : 1;
  }
  const int64_t n_units = int64_t(dp.n_tiles) * dp.n_seg;
  const unsigned grid = unsigned(std::min<int64_t>(n_units, int64_t(cache.per_sm[dev]) * n_sm));
  e = launch_pdl(kern, grid, 128u, dp, st);
  if (e != cudaSuccess || !reduce) return e;
  const int64_t n = int64_t(dp.n_tiles) * P;
  const unsigned rgrid = unsigned(std::min<int64_t>((n + 255) / 256, int64_t(n_sm) * 8));
  return launch_pdl(direct_reduce_kernel<P, 1>, std::max(rgrid, 1u), 256u, dp, st);
}

template <int P, int SW, int WB>
cudaError_t launch_window_w(int fmt, const DirectParams& dp, int n_sm, cudaStream_t st, bool reduce) {
  if (fmt == kBF32) return launch_window_fmt<P, SW, kBF32, WB>(dp, n_sm, st, reduce);
  if (fmt == kBBF16P) return launch_window_fmt<P, SW, kBBF16P, WB>(dp, n_sm, st, reduce);
  if (fmt == kBF16P) return launch_window_fmt<P, SW, kBF16P, WB>(dp, n_sm, st, reduce);
  return cudaErrorInvalidValue;
}

// The smallest slot (128, 192 or 288 rows) that holds every window.
template <int P, int SW>
cudaError_t launch_window(int fmt, const DirectParams& dp, int n_sm, cudaStream_t st, bool reduce) {
  if (dp.W <= 128) return launch_window_w<P, SW, 128>(fmt, dp, n_sm, st, reduce);
  if (dp.W <= 192) return launch_window_w<P, SW, 192>(fmt, dp, n_sm, st, reduce);
  return launch_window_w<P, SW, kWindowMaxRows>(fmt, dp, n_sm, st, reduce);
}

template <int P, int SW, int DELAYS, int WGT>
cudaError_t launch_direct_w(int fmt, const DirectParams& dp, int n_sm, cudaStream_t st, bool reduce) {
  if (fmt == kBF32) return launch_direct_fmt<P, SW, kBF32, DELAYS, WGT>(dp, n_sm, st, reduce);
  if (fmt == kBBF16P) return launch_direct_fmt<P, SW, kBBF16P, DELAYS, WGT>(dp, n_sm, st, reduce);
  if (fmt == kBF16P) return launch_direct_fmt<P, SW, kBF16P, DELAYS, WGT>(dp, n_sm, st, reduce);
  return cudaErrorInvalidValue;
}

template <int P, int SW, int DELAYS>
cudaError_t launch_direct_t(int fmt, const DirectParams& dp, int n_sm, cudaStream_t st, bool reduce) {
  return dp.wanchor ? launch_direct_w<P, SW, DELAYS, 1>(fmt, dp, n_sm, st, reduce)
                    : launch_direct_w<P, SW, DELAYS, 0>(fmt, dp, n_sm, st, reduce);
}

}  // namespace

size_t direct_part_floats(const GatherConfig& c, int n_tiles, int n_seg) {
  return size_t(n_tiles) * n_seg * c.SW * c.P;
}

cudaError_t launch_gather_direct(const GatherConfig& c, int fmt, const InstDesc& d, int n_sm,
                                 int* status, int* host_status, uint64_t timeout_ns,
                                 cudaStream_t st, bool reduce) {
  if (d.n_frames != 1 || c.FB != 1 || d.n_fg != 1 || n_sm < 1 || !d.part) return cudaErrorInvalidValue;
  DirectParams dp;
  dp.u = d.u;
  dp.anchor = d.anchor;
  dp.pix = d.pix;
  dp.wanchor = d.wanchor;
  dp.base = d.base;
  dp.slot = d.slot;
  dp.zero_runs = d.zero_runs;
  dp.b = d.b;
  dp.m = d.m;
  dp.out = d.out;
  dp.part = d.part;
  dp.status = status;
  dp.host_status = host_status;
  dp.timeout_ns = timeout_ns;
  dp.n_zero_runs = d.n_zero_runs;
  dp.n_sensors = d.n_sensors;
  dp.n_sensors_pad = d.n_sensors_pad;
  dp.n_t_pad = d.n_t_pad;
  dp.n_tiles = d.n_tiles;
  dp.n_seg = d.n_seg;
  dp.G = d.G;
  dp.W = d.W;
  // stored tables without weights: the windowed kernel when every window fits a slot
  const bool window = !c.delays && !dp.wanchor && !c.no_window && dp.W >= 0 &&
                      dp.W <= kWindowMaxRows && dp.G <= 32 * c.SW;
  if (window && c.P == 128 && c.SW == 4) return launch_window<128, 4>(fmt, dp, n_sm, st, reduce);
  if (window && c.P == 256 && c.SW == 2) return launch_window<256, 2>(fmt, dp, n_sm, st, reduce);
  if (c.P == 128 && c.SW == 4)
    return c.delays ? launch_direct_t<128, 4, 1>(fmt, dp, n_sm, st, reduce)
                    : launch_direct_t<128, 4, 0>(fmt, dp, n_sm, st, reduce);
  if (c.P == 256 && c.SW == 2)
    return c.delays ? launch_direct_t<256, 2, 1>(fmt, dp, n_sm, st, reduce)
                    : launch_direct_t<256, 2, 0>(fmt, dp, n_sm, st, reduce);
  return cudaErrorInvalidValue;
}

}  // namespace patbp
