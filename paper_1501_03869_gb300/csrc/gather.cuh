// gather.cuh -- the persistent gather kernel of Eq. (BP) and its launch
// templates (internal).  Two translation units instantiate it: kernels.cu for
// delays read from the stored fast-marching table, gather_const.cu for the
// conventional constant-speed delays computed in the kernel (Sec. II-C).
//
//   out[f][r] = sum_s w_s * b_{f,s}(T_s(r)/dt) with linear interpolation.
//   The work of one launch is a sequence of units (instance, frame group, tile
//   of P pixels, segment of G sensors), handed to CTAs by ticket.  A producer
//   warp streams, per stage of S sensors, the tile's delay data (table rows
//   u[S][P], or one 32-byte anchor per sensor for constant speed), the
//   multipliers and every sensor's window of integrand rows (packed back to
//   back, FB frames per row) into shared memory with 1-D bulk copies
//   (cp.async.bulk) completing on mbarriers; the windows' bases are fetched one
//   unit ahead.  Consumer warps interpolate from shared memory and accumulate
//   in FP32 registers.  Sensor phases are summed in fixed order through shared
//   memory and segments in fixed order by the last CTA to finish a tile, so the
//   result depends neither on timing nor on how frames or instances are
//   batched.
//
// The kernel is launched as a programmatic dependent of the preprocessing grid
// and may start before it finishes; lines an earlier kernel left in an SM's L1
// are then not reliably dropped, so its plain global loads use ld.global.cg
// (L2 only) and everything else arrives by bulk copies, which read L2.
//
// Every wait on an mbarrier is bounded by a wall-clock limit; on expiry the CTA
// records kStatusTimeout, drains its own copies in flight (bounded again) and
// exits without touching the output's remaining values.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "device.cuh"
#include "kernels.cuh"

namespace patbp {

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

// Offset that selects the zero rows after the windows (an arrival after the
// record): it truncates to an index above every window and its phase times
// the zero rows' values is zero.
constexpr float kFarOffset = 1.0e30f;

// Solid-angle weights of a lane's 4 pixels for one sensor (the exact back
// projection that Eq. (BP) approximates, Sec. II-C): v = D + e from the pixel
// terms pq = (2 D, |D|^2) and the sensor's weight anchor E = (e, scale),
// N = (n, d); w = scale (n . v) / |v|^d, d = 2 or 3 (the same for every sensor
// of a handle: a uniform branch).  Both gathers use this function, so a frame
// gets the same weights alone and in a batch.
__device__ __forceinline__ float solid_angle_weight(const float4 pq, float4 E, float4 N) {
  const float v0 = fmaf(0.5f, pq.x, E.x), v1 = fmaf(0.5f, pq.y, E.y), v2 = fmaf(0.5f, pq.z, E.z);
  const float r2 = fmaxf(fmaf(v0, v0, fmaf(v1, v1, v2 * v2)), 1.0e-30f);
  const float nv = fmaf(N.x, v0, fmaf(N.y, v1, N.z * v2));
  const float y = rsqrtf(r2);
  const float inv = N.w == 3.0f ? y * y * y : y * y;
  return E.w * (nv * inv);
}

__device__ __forceinline__ void solid_angle_weights(float (&ww)[4], const float4 (&pq)[4], float4 E,
                                                    float4 N) {
#pragma unroll
  for (int x = 0; x < 4; ++x) ww[x] = solid_angle_weight(pq[x], E, N);
}

// Rows of 8 frames (32 bytes, four to a 128-byte line of shared-memory banks)
// are stored with their two 16-byte halves swapped when bit 2 of the row index
// is set.  The 8 lanes of a 16-byte load phase read rows of 8 pixels; without
// the swap two of them conflict whenever their rows agree mod 4, with it only
// when they agree mod 8.  Windows start at rows that are multiples of 8 in
// global and shared memory, so a row's swap is the same in both.
__device__ __forceinline__ void load_row8(const uint32_t* sw, unsigned r, uint32_t (&w)[8]) {
  const unsigned x = (r >> 2) & 1u;
  const uint4 lo = *reinterpret_cast<const uint4*>(sw + r * 8u + 4u * x);
  const uint4 hi = *reinterpret_cast<const uint4*>(sw + r * 8u + 4u * (x ^ 1u));
  w[0] = lo.x; w[1] = lo.y; w[2] = lo.z; w[3] = lo.w;
  w[4] = hi.x; w[5] = hi.y; w[6] = hi.z; w[7] = hi.w;
}

// Frames fb of row r of a window in shared memory (FB words per row; 8-frame
// rows as load_row8 describes).
template <int FB>
__device__ __forceinline__ void load_row(const uint32_t* sw, unsigned r, uint32_t (&w)[FB]) {
  if constexpr (FB == 8) load_row8(sw, r, w);
  else load_words<FB>(sw + size_t(r) * FB, w);
}

// Interpolate one sensor's integrand at the lane's 4 window offsets uu (rows
// from the start of the sensor's window at `off`) and accumulate FB frames
// weighted by the multipliers sm (and, WGT = 1, by the per-pixel weights ww:
// acc = fma(m, w * lerp, acc)).  Offsets past the stage's windows read the
// zero rows.
template <int FB, int FMT, int WGT>
__device__ __forceinline__ void lerp_accumulate(float (&acc)[FB][4], const float (&uu)[4],
                                                const float (&ww)[4], const uint32_t* sm, int off,
                                                const uint32_t* sw, int Wst) {
  const unsigned lim = unsigned(Wst - off);
  float mm[FB];
  {
    uint32_t mw[FB];
    load_words<FB>(sm, mw);
#pragma unroll
    for (int fb = 0; fb < FB; ++fb) mm[fb] = __uint_as_float(mw[fb]);
  }
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    const unsigned i = min(unsigned(__float2int_rz(uu[x])), lim);
    const float ph = uu[x] - float(i);
    const unsigned r = i + unsigned(off);
    uint32_t w0[FB];
    load_row<FB>(sw, r, w0);
    if constexpr (FMT == kBF32) {
      uint32_t w1[FB];
      load_row<FB>(sw, r + 1u, w1);
#pragma unroll
      for (int fb = 0; fb < FB; ++fb) {
        const float b0 = __uint_as_float(w0[fb]), b1 = __uint_as_float(w1[fb]);
        float v = fmaf(ph, b1 - b0, b0);
        if constexpr (WGT != 0) v = __fmul_rn(ww[x], v);
        acc[fb][x] = fmaf(mm[fb], v, acc[fb][x]);
      }
    } else if constexpr (FMT == kBBF16P) {
#pragma unroll
      for (int fb = 0; fb < FB; ++fb) {
        float v = fmaf(ph, __uint_as_float(w0[fb] & 0xffff0000u), __uint_as_float(w0[fb] << 16));
        if constexpr (WGT != 0) v = __fmul_rn(ww[x], v);
        acc[fb][x] = fmaf(mm[fb], v, acc[fb][x]);
      }
    } else {
#pragma unroll
      for (int fb = 0; fb < FB; ++fb) {
        const float2 h = __half22float2(*reinterpret_cast<const __half2*>(&w0[fb]));
        float v = fmaf(ph, h.y, h.x);
        if constexpr (WGT != 0) v = __fmul_rn(ww[x], v);
        acc[fb][x] = fmaf(mm[fb], v, acc[fb][x]);
      }
    }
  }
}

// One sensor of a stage, delays from the stored table: u[sl][P] in shared
// memory; with WGT the sensor's weight anchor is swa[2 sl], swa[2 sl + 1].
template <int P, int FB, int FMT, int WGT>
__device__ __forceinline__ void gather_sensor(float (&acc)[FB][4], const float* su, const uint32_t* sm,
                                              const int* soff, const uint32_t* sw, int sl, int Wst,
                                              const float4 (&pq)[4], const float4* swa) {
  float uu[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) uu[x] = su[sl * P + x * 32];
  float ww[4] = {1.0f, 1.0f, 1.0f, 1.0f};
  if constexpr (WGT != 0) solid_angle_weights(ww, pq, swa[2 * sl], swa[2 * sl + 1]);
  lerp_accumulate<FB, FMT, WGT>(acc, uu, ww, sm + sl * FB, soff[sl], sw, Wst);
}

// One sensor of a stage, constant-speed delays computed here (Sec. II-C: the
// conventional back projection takes t = |r - r_s| / c).  In sample units
// (kappa = dx / (c dt) samples per node spacing), with r0 the tile's anchor
// node and D = kappa (r - r0):
//   u(r) = |kappa (r - r_s)| = |D + e| = sqrt(u0^2 + num),
//   e = kappa (r0 - r_s),  u0 = |e|,  num = |D|^2 + 2 D.e.
// The window offset is (u0 - base) + (u - u0).  Far from the sensor (the
// host's flag 0: u0 > 4 max|D| over the tile) u - u0 is the root delta of
// delta^2 + 2 u0 delta = num, started from the hardware reciprocal square root
// of u0^2 + num and refined by one Newton step whose residual is formed from
// num itself, so it keeps the accuracy of num (a few 1e-6 samples) where a
// plain FP32 evaluation of |D + e| would lose ulp(u) ~ 1e-4.  Near the sensor
// (flag 1, u and u0 small) |D + e| is evaluated directly, which is accurate
// there while the Newton step would divide by u ~ 0.
// Anchor of the sensor (two float4): (e.x, e.y, e.z, u0), (u0 - base, cap,
// u0^2, flag), cap = (N_t - 1) - base; offsets above cap are after the
// record.  Per pixel (registers): pq = (2 D.x, 2 D.y, 2 D.z, |D|^2).
template <int FB, int FMT, int WGT>
__device__ __forceinline__ void gather_sensor_const(float (&acc)[FB][4], const float4 (&pq)[4],
                                                    const float4* sa, const uint32_t* sm,
                                                    const int* soff, const uint32_t* sw, int sl,
                                                    int Wst, const float4* swa) {
  const float4 A = sa[2 * sl], B = sa[2 * sl + 1];
  float uu[4];
  if (B.w == 0.0f) {  // the same sensor for the whole warp: a uniform branch
    const float m2u0 = -2.0f * A.w;
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const float num = fmaf(pq[x].x, A.x, fmaf(pq[x].y, A.y, fmaf(pq[x].z, A.z, pq[x].w)));
      const float s = num + B.z;
      const float y = rsqrtf(s);
      const float da = s * y - A.w;
      const float r = fmaf(-da, da, fmaf(m2u0, da, num));  // num - delta_a (delta_a + 2 u0)
      const float v = fmaf(r, 0.5f * y, da) + B.x;
      uu[x] = v > B.y ? kFarOffset : fmaxf(v, 0.0f);
    }
  } else {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const float d0 = fmaf(0.5f, pq[x].x, A.x), d1 = fmaf(0.5f, pq[x].y, A.y),
                  d2 = fmaf(0.5f, pq[x].z, A.z);
      const float s = fmaxf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)), 1.0e-30f);
      const float v = (s * rsqrtf(s) - A.w) + B.x;
      uu[x] = v > B.y ? kFarOffset : fmaxf(v, 0.0f);
    }
  }
  float ww[4] = {1.0f, 1.0f, 1.0f, 1.0f};
  if constexpr (WGT != 0) solid_angle_weights(ww, pq, swa[2 * sl], swa[2 * sl + 1]);
  lerp_accumulate<FB, FMT, WGT>(acc, uu, ww, sm + sl * FB, soff[sl], sw, Wst);
}

// Shared-memory layout of one pipeline stage (byte offsets); `mode` is the
// kernel's: bit 0 constant-speed delays, bit 1 solid-angle weights.  A stage
// holds up to S consecutive sensors of a segment -- as many as the row budget
// Wst of the windows allows (the producer decides and writes (se, m_shift) to
// the stage's header).
//   u    [S][P] float            the tile's table rows of the stage's sensors,
//                                or [S][8] float anchors (constant speed)
//   wa   [S][8] float            solid-angle weight anchors (bit 1 only)
//   m    [S4 + 4][FB] float      multipliers w_s * sigma, copied from the
//                                16-byte-aligned sensor at or below the first
//                                (the first sensor's sit m_shift entries in)
//   off  [S4] int                window offset (rows) of each sensor
//   win  [Wst + 4][FB] words     the stage's windows packed at `off`, then 4
//                                zero rows that out-of-record pixels read
struct StageLayout {
  size_t u, wa, m, off, win, bytes;
  __host__ __device__ StageLayout(int S, int P, int FB, int Wst, int mode) {
    const int S4 = (S + 3) & ~3;
    u = 0;
    wa = u + ((mode & 1) ? size_t(S) * 32 : size_t(S) * P * 4);
    m = wa + ((mode & 2) ? size_t(S) * 32 : 0);
    off = m + size_t(S4 + 4) * FB * 4;
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
// MODE bit 0 (DELAYS): 0 = offsets from the stored table (u block per stage),
// 1 = constant-speed delays computed by the consumers (an anchor per sensor).
// MODE bit 1 (WGT): solid-angle weights per (pixel, sensor), from a weight
// anchor per sensor copied into each stage and the pixel terms.  The computed
// delays hold more live registers; the minimum of resident CTAs keeps the
// compiler from spilling them (0 leaves the table variants unconstrained).
template <int P, int FB, int FMT, int SW, int MODE>
__global__ void __launch_bounds__(32 * ((P / 128) * SW + 3), (MODE & 1) ? (FB == 1 ? 3 : 2) : 0)
    gather_kernel(const __grid_constant__ StreamParams p) {
  constexpr int DELAYS = MODE & 1, WGT = (MODE >> 1) & 1;
  constexpr int PW = P / 128;   // warps across the tile's pixels
  static_assert((SW & (SW - 1)) == 0, "sensor phases: a power of two");
  constexpr int NWC = PW * SW;  // consumer warps
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t* full = reinterpret_cast<uint64_t*>(smem);
  uint64_t* empty = full + kMaxStages;
  uint64_t* meta_bar = empty + kMaxStages;
  int64_t* unit_ring = reinterpret_cast<int64_t*>(meta_bar + 2);  // [kRing]
  int64_t* red_unit = unit_ring + kRing;                           // [2]
  volatile int* abort_flag = reinterpret_cast<volatile int*>(red_unit + 2);
  int2* stage_hdr = reinterpret_cast<int2*>(smem + 320);  // [kMaxStages] (sensors, m shift)
  int* meta = reinterpret_cast<int*>(smem + kHeaderBytes);  // [2][kMaxG] packed bases
  const StageLayout L(p.S, P, FB, p.Wst, MODE);
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
    // Issue stage st of unit q from sensor s0: the sensors it takes are the
    // longest run of at most S (and at most the segment's rest) whose windows
    // fit the row budget Wst (at least one: Wst is at least the longest single
    // window).  Part 1 posts the expected bytes and copies the table block
    // (delay data), part 2 the multipliers and windows, which come from the
    // preprocessing grid (part 3: both).  Returns the sensors taken; both
    // parts compute the same.
    auto issue_chunk = [&](const UnitPos& q, const InstDesc& d, const int* mrow, int s0, int st,
                           int part) -> int {
      const int avail = min(p.S, q.s_hi - s0);
      unsigned char* sb = stage0 + st * L.bytes;
      int bs = 0, wl = 0;
      if (lane < avail) {
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
      const unsigned fit = __ballot_sync(0xffffffffu, lane < avail && incl <= p.Wst);
      int se = __popc(fit);  // the windows' prefix sums grow: the fitting lanes are a prefix
      bool bad = false;
      if (se == 0) {  // cannot happen with a host-computed Wst; stay in bounds
        bad = true;
        se = 1;
      }
      if (lane >= se || bad) wl = 0;
      const int total_w = bad ? 0 : __shfl_sync(0xffffffffu, incl, se - 1);
      const int off = bad ? 0 : incl - wl;
      const int ma = s0 & ~3;                               // aligned first multiplier
      const int mcount = ((s0 + se + 3) & ~3) - ma;         // <= S4 + 4
      if (part & 1) {
        if (lane < S4) reinterpret_cast<int*>(sb + L.off)[lane] = lane < se ? off : 0;
        if (lane == 0) {
          stage_hdr[st] = make_int2(se, s0 - ma);
          if (bad) atomicOr(p.status, kStatusBadConfig);
        }
        __syncwarp();
        const uint32_t dbytes = DELAYS ? uint32_t(se) * 32 : uint32_t(se) * P * 4;
        const uint32_t wbytes = WGT ? uint32_t(se) * 32 : 0u;
        const uint32_t bytes = dbytes + wbytes + uint32_t(mcount) * FB * 4 + uint32_t(total_w) * FB * 4;
        if (lane == 0) {
          mbar_arrive_expect_tx(&full[st], bytes);
          const float* src = DELAYS ? d.anchor + (int64_t(q.tile) * d.n_sensors_pad + s0) * 8
                                    : d.u + (int64_t(q.tile) * d.n_sensors + s0) * P;
          bulk_g2s(sb + L.u, src, dbytes, &full[st]);
          if (WGT)
            bulk_g2s(sb + L.wa, d.wanchor + (int64_t(q.tile) * d.n_sensors_pad + s0) * 8, wbytes,
                     &full[st]);
        }
      }
      if (part & 2) {
        if (lane == 0)
          bulk_g2s(sb + L.m, d.m + (int64_t(q.fg) * d.n_sensors_pad + ma) * FB,
                   uint32_t(mcount) * FB * 4, &full[st]);
        if (wl > 0) {
          const unsigned char* src =
              static_cast<const unsigned char*>(d.b) +
              ((int64_t(q.fg) * d.n_sensors + s0 + lane) * d.n_t_pad + bs) * (FB * 4);
          bulk_g2s(sb + L.win + size_t(off) * FB * 4, src, uint32_t(wl) * FB * 4, &full[st]);
        }
      }
      return se;
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
        for (int s = q.s_lo; s < q.s_hi && k < p.stages; ++k)
          s += issue_chunk(q, d, mrow, s, int((seq0 + k) % p.stages), 1);
        asm volatile("griddepcontrol.wait;" ::: "memory");
        waited_inputs = true;
        for (int i = 0; i < k; ++i, ++seq) s0 += issue_chunk(q, d, mrow, s0, int(seq % p.stages), 2);
      }
      for (; s0 < q.s_hi; ++seq) {
        const int st = int(seq % p.stages);
        if (!acquire_stage(st)) {
          ok = false;
          break;
        }
        s0 += issue_chunk(q, d, mrow, s0, st, 3);
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
      float4 pq[4];  // constant speed or weights: the lane's pixels relative to the tile anchor
      if constexpr (DELAYS != 0 || WGT != 0) {
        const float4* src = p.inst[q.inst].pix + int64_t(q.tile) * P + pg * 128 + lane;
#pragma unroll
        for (int x = 0; x < 4; ++x) pq[x] = __ldcg(src + x * 32);
      }
      float acc[FB][4];
#pragma unroll
      for (int fb = 0; fb < FB; ++fb)
#pragma unroll
        for (int x = 0; x < 4; ++x) acc[fb][x] = 0.0f;
      for (int s0 = q.s_lo; s0 < q.s_hi; ++seq) {
        const int st = int(seq % p.stages);
        if (s0 != q.s_lo && !wait_full(st)) {
          ok = false;
          break;
        }
        const int2 hdr = stage_hdr[st];  // sensors of the stage, multiplier shift
        const int se = hdr.x;
        // phase sp takes the sensors s with (s - s_lo) mod SW == sp, whatever
        // sensor the stage starts at
        const int sl0 = (sp - (s0 - q.s_lo)) & (SW - 1);
        s0 += se;
        const unsigned char* sb = stage0 + st * L.bytes;
        const float* su = reinterpret_cast<const float*>(sb + L.u) + pg * 128 + lane;
        const uint32_t* sm = reinterpret_cast<const uint32_t*>(sb + L.m) + hdr.y * FB;
        const int* soff = reinterpret_cast<const int*>(sb + L.off);
        const uint32_t* sw = reinterpret_cast<const uint32_t*>(sb + L.win);
        const float4* swa = reinterpret_cast<const float4*>(sb + L.wa);
        int sl = sl0;
        if constexpr (DELAYS == 0) {
          for (; sl + SW < se; sl += 2 * SW) {
            gather_sensor<P, FB, FMT, WGT>(acc, su, sm, soff, sw, sl, p.Wst, pq, swa);
            gather_sensor<P, FB, FMT, WGT>(acc, su, sm, soff, sw, sl + SW, p.Wst, pq, swa);
          }
          if (sl < se) gather_sensor<P, FB, FMT, WGT>(acc, su, sm, soff, sw, sl, p.Wst, pq, swa);
        } else {
          const float4* sa = reinterpret_cast<const float4*>(sb + L.u);
          for (; sl + SW < se; sl += 2 * SW) {
            gather_sensor_const<FB, FMT, WGT>(acc, pq, sa, sm, soff, sw, sl, p.Wst, swa);
            gather_sensor_const<FB, FMT, WGT>(acc, pq, sa, sm, soff, sw, sl + SW, p.Wst, swa);
          }
          if (sl < se) gather_sensor_const<FB, FMT, WGT>(acc, pq, sa, sm, soff, sw, sl, p.Wst, swa);
        }
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
      for (int k = 0; k < KO; ++k) slot_idx[k] = __ldcg(d.slot + int64_t(q.tile) * P + k * 32 + lane);
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

// ------------------------------------------------------- launch templates --
template <int P, int FB, int FMT, int SW, int MODE>
static cudaError_t gather_t(const StreamParams& p, size_t smem, int grid, cudaStream_t st,
                            int* resident, int n_sm) {
  auto kern = gather_kernel<P, FB, FMT, SW, MODE>;
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

template <int P, int FMT, int SW, int MODE>
static cudaError_t gather_fb(int FB, const StreamParams& p, size_t smem, int grid, cudaStream_t st,
                             int* resident, int n_sm) {
  switch (FB) {
    case 1: return gather_t<P, 1, FMT, SW, MODE>(p, smem, grid, st, resident, n_sm);
    case 2: return gather_t<P, 2, FMT, SW, MODE>(p, smem, grid, st, resident, n_sm);
    case 4: return gather_t<P, 4, FMT, SW, MODE>(p, smem, grid, st, resident, n_sm);
    case 8: return gather_t<P, 8, FMT, SW, MODE>(p, smem, grid, st, resident, n_sm);
    default: return cudaErrorInvalidValue;
  }
}

// Launch (resident == nullptr) or count resident CTAs of the instantiation
// that matches the config and the integrand format.
template <int MODE>
static cudaError_t gather_dispatch_t(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                                     cudaStream_t st, int* resident, int n_sm) {
  const size_t smem = gather_smem_bytes(c, p.Wst);
  if (c.P == 128 && c.SW == 4) {
    if (fmt == kBF32) return gather_fb<128, kBF32, 4, MODE>(c.FB, p, smem, grid, st, resident, n_sm);
    if (fmt == kBBF16P) return gather_fb<128, kBBF16P, 4, MODE>(c.FB, p, smem, grid, st, resident, n_sm);
    if (fmt == kBF16P) return gather_fb<128, kBF16P, 4, MODE>(c.FB, p, smem, grid, st, resident, n_sm);
  } else if (c.P == 256 && c.SW == 2) {
    if (fmt == kBF32) return gather_fb<256, kBF32, 2, MODE>(c.FB, p, smem, grid, st, resident, n_sm);
    if (fmt == kBBF16P) return gather_fb<256, kBBF16P, 2, MODE>(c.FB, p, smem, grid, st, resident, n_sm);
    if (fmt == kBF16P) return gather_fb<256, kBF16P, 2, MODE>(c.FB, p, smem, grid, st, resident, n_sm);
  }
  return cudaErrorInvalidValue;
}

// Kernel entry addresses (identify graph nodes when refreshing their parameters).
template <int P, int FMT, int SW, int MODE>
static const void* gather_func_fb(int FB) {
  switch (FB) {
    case 1: return reinterpret_cast<const void*>(gather_kernel<P, 1, FMT, SW, MODE>);
    case 2: return reinterpret_cast<const void*>(gather_kernel<P, 2, FMT, SW, MODE>);
    case 4: return reinterpret_cast<const void*>(gather_kernel<P, 4, FMT, SW, MODE>);
    case 8: return reinterpret_cast<const void*>(gather_kernel<P, 8, FMT, SW, MODE>);
  }
  return nullptr;
}

template <int MODE>
static const void* gather_func_t(const GatherConfig& c, int fmt) {
  if (c.P == 128 && c.SW == 4) {
    if (fmt == kBF32) return gather_func_fb<128, kBF32, 4, MODE>(c.FB);
    if (fmt == kBBF16P) return gather_func_fb<128, kBBF16P, 4, MODE>(c.FB);
    if (fmt == kBF16P) return gather_func_fb<128, kBF16P, 4, MODE>(c.FB);
  } else if (c.P == 256 && c.SW == 2) {
    if (fmt == kBF32) return gather_func_fb<256, kBF32, 2, MODE>(c.FB);
    if (fmt == kBBF16P) return gather_func_fb<256, kBBF16P, 2, MODE>(c.FB);
    if (fmt == kBF16P) return gather_func_fb<256, kBF16P, 2, MODE>(c.FB);
  }
  return nullptr;
}

// The other modes' instantiations live in their own translation units so the
// families compile in parallel: constant-speed delays (gather_const.cu, mode
// 1), solid-angle weights with table or constant-speed delays (gather_wgt.cu,
// modes 2 and 3).
cudaError_t gather_dispatch_const(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                                  cudaStream_t st, int* resident, int n_sm);
const void* gather_func_const(const GatherConfig& c, int fmt);
cudaError_t gather_dispatch_wgt(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                                cudaStream_t st, int* resident, int n_sm);
const void* gather_func_wgt(const GatherConfig& c, int fmt);
cudaError_t gather_dispatch_wgt_const(const GatherConfig& c, int fmt, const StreamParams& p, int grid,
                                      cudaStream_t st, int* resident, int n_sm);
const void* gather_func_wgt_const(const GatherConfig& c, int fmt);

}  // namespace patbp
