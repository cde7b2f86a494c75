// eikonal.cu -- first-order arrival times of many point sources on the GPU
// (Sec. II-B), for the table build.
//
// The first-order Godunov upwind system sum_d max(T - a_d, 0)^2 = (h/c)^2 has
// one solution, the one fast marching finds, and every node's value is the
// local solve of its neighbours' values.  Instead of marching (a serial heap),
// the GPU iterates that local solve to its fixed point, block by block: each
// CTA holds one block of one source (16 x 16 nodes in 2-D, 8 x 8 x 4 in 3-D)
// with a one-node halo in shared memory and sweeps it (Jacobi) until nothing
// changes or a sweep budget is spent; the next round takes the blocks that
// changed and their face neighbours.  Values only decrease, from +inf, so the
// loop ends, and when a round changes nothing every node is at the fixed point
// (to rounding: FP64 gives the host march's values to about 1e-12).
//
// Work per node is kept small: a node is solved again only when a neighbour
// moved BELOW its own value in the previous sweep (a neighbour at or above it
// is not upwind and cannot lower it: in the Godunov equation its term is zero),
// and at a block's first sweep only next to halo nodes that changed since the
// block last settled.  Comparisons run on the bit patterns (non-negative
// doubles order like their integer images), and the local solve uses the
// difference form of the quadratic with a Newton-refined square root, so the
// scarce FP64 pipe does little beyond the arithmetic itself.
//
// Blocks are launched in two colours ((bx + by + bz) & 1); face neighbours have
// different colours, so no block reads a node another block of the launch
// writes: the result is a fixed function of the input, whatever the order the
// blocks run in and whatever else is in the batch.  The source cell's corners
// are fixed at distance / c (as the host march fixes them), and values above
// the record end (stop_after) are never written; they cannot lower earlier
// arrivals.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <limits>
#include <string>
#include <vector>

#include "table.h"

namespace patbp {

namespace {

constexpr int kMaxSeeds = 8;  // corners of the source cell
constexpr int kUnclean = -2;  // block state: its nodes may not solve to their own values
constexpr long long kInfBits = 0x7ff0000000000000LL;

struct EikParams {
  double* T;            // [nb][total] arrival times (s)
  const double* hf;     // [total] dx / c
  const int64_t* seed;  // [nb][kMaxSeeds] fixed nodes (-1 = none)
  const int2* list;     // active (source, block) pairs
  int n_list;
  int* changed;         // [nb][n_blocks] set when a block's values changed
  int* stamp;           // [nb][total] phase of a node's last change (-1 never, 0 seed)
  int* visited;         // [nb][n_blocks] phase of the last visit that settled the
                        // block (-1 never visited, kUnclean: left unsettled)
  int phase;            // 2 * round + colour + 1
  int* pending;         // [nb][n_blocks] set while a block holds a lowering above tau
  uint8_t* defer;       // [nb][total] set while a node's last solve was above tau
  double tau;           // this round's acceptance bound (s)
  int n[3];             // nodes per axis (x first)
  int bn[3];            // blocks per axis
  int64_t total;
  int n_blocks;
  double stop_after;
  int sweeps;           // sweep budget per block visit
};

// Non-negative doubles (and +inf) order like their bit patterns; comparing
// those keeps the comparisons off the FP64 pipe.
__device__ __forceinline__ long long bits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool lt(double a, double b) { return bits(a) < bits(b); }
__device__ __forceinline__ double min2(double a, double b) { return lt(b, a) ? b : a; }

// sqrt(x) for x > 0: the FP32 reciprocal square root refined by one Newton
// (Heron) step in FP64, s' = s + (x - s^2) / (2 s), which takes the relative
// error from about 2^-23 to about 2^-46 (a few 1e-14).
__device__ __forceinline__ double sqrt_newton(double x) {
  const double r = double(rsqrtf(float(x)));
  const double s = x * r;
  const double e = fma(-s, s, x);
  return fma(0.5 * r, e, s);
}

// First-order Godunov update from the per-axis upwind values a0 <= a1 <= a2
// (+inf where an axis has none): the one-axis root a0 + h/c while it stays at
// or below a1, else the two-axis root (a0 + a1 + sqrt(2 (h/c)^2 - (a1 - a0)^2)) / 2
// while it stays at or below a2, else the three-axis root with the
// discriminant 3 (h/c)^2 - sum of the squared pairwise differences.  The
// difference form is the quadratic's discriminant without cancellation.
// hf2 = 2 (h/c)^2 and hf3 = 3 (h/c)^2 are the node's constants.
__device__ __forceinline__ double godunov(double a0, double a1, double a2, double hf, double hf2,
                                          double hf3) {
  if (bits(a0) >= kInfBits) return CUDART_INF;
  double r = a0 + hf;
  if (!lt(a1, r)) return r;
  const double d01 = a1 - a0;
  const double disc2 = fma(-d01, d01, hf2);  // > (h/c)^2 since a1 - a0 < h/c
  r = 0.5 * (a0 + a1 + sqrt_newton(disc2));
  if (!lt(a2, r)) return r;
  const double d02 = a2 - a0, d12 = a2 - a1;
  const double disc3 = fma(-d01, d01, fma(-d02, d02, fma(-d12, d12, hf3)));
  const double s3 = disc3 > 0.0 ? sqrt_newton(disc3) : 0.0;
  return (a0 + a1 + a2 + s3) * (1.0 / 3.0);
}

__device__ __forceinline__ void sort3(double& a0, double& a1, double& a2) {
  if (lt(a1, a0)) { const double t = a0; a0 = a1; a1 = t; }
  if (lt(a2, a1)) { const double t = a1; a1 = a2; a2 = t; }
  if (lt(a1, a0)) { const double t = a0; a0 = a1; a1 = t; }
}

// Tile with a one-node halo: extents B + 2 per active axis.
template <int B0, int B1, int B2>
struct Tile {
  static constexpr int X = B0 + 2, Y = B1 + 2, Z = B2 > 1 ? B2 + 2 : 1;
  static constexpr int N = X * Y * Z;
};

template <int B0, int B1, int B2>
__global__ void __launch_bounds__(B0 * B1 * B2, 6) eik_sweep_kernel(const EikParams p) {
  using TL = Tile<B0, B1, B2>;
  constexpr int NT = B0 * B1 * B2, NW = NT / 32;
  constexpr int SY = TL::X, SZ = TL::X * TL::Y;
  __shared__ double tile[TL::N];
  // moved[j][i]: node i changed in the sweep before one that reads moved[j]
  __shared__ uint8_t moved[2][TL::N];
  // stamps of the halo (-1 inside the block and outside the grid)
  __shared__ int hstamp[TL::N];
  // per sweep, the nodes (thread ids) that need a solve, packed densely so the
  // FP64 work runs in full warps; their h/c and their candidates
  __shared__ int queue[NT];
  __shared__ double hf_s[NT], cand_s[NT];
  __shared__ int warp_count[NW];
  const int2 job = p.list[blockIdx.x];
  const int src = job.x, blk = job.y;
  const int bx = blk % p.bn[0], by = (blk / p.bn[0]) % p.bn[1], bz = blk / (p.bn[0] * p.bn[1]);
  const int x0 = bx * B0, y0 = by * B1, z0 = bz * B2;
  double* T = p.T + int64_t(src) * p.total;
  int* stamp = p.stamp + int64_t(src) * p.total;
  const int hz = B2 > 1 ? 1 : 0;
  // load the block and its halo; nodes outside the grid are +inf
  for (int i = threadIdx.x; i < TL::N; i += blockDim.x) {
    const int tx = i % TL::X, ty = (i / TL::X) % TL::Y, tz = i / (TL::X * TL::Y);
    const int x = x0 + tx - 1, y = y0 + ty - 1, z = z0 + tz - hz;
    const bool halo = tx == 0 || tx == TL::X - 1 || ty == 0 || ty == TL::Y - 1 ||
                      (B2 > 1 && (tz == 0 || tz == TL::Z - 1));
    double v = CUDART_INF;
    int st = -1;
    if (x >= 0 && x < p.n[0] && y >= 0 && y < p.n[1] && z >= 0 && z < p.n[2]) {
      const int64_t g = (int64_t(z) * p.n[1] + y) * p.n[0] + x;
      v = __ldcg(T + g);
      if (halo) st = __ldcg(stamp + g);
    }
    tile[i] = v;
    hstamp[i] = st;
    moved[0][i] = 0;
    moved[1][i] = 0;
  }
  // A settled block's nodes solve to their own values from the halo it saw then;
  // only a node next to a halo node that has since dropped below it needs solving.
  const int last = p.visited[int64_t(src) * p.n_blocks + blk];
  const bool full = last == kUnclean;
  const int lx = threadIdx.x % B0, ly = (threadIdx.x / B0) % B1, lz = threadIdx.x / (B0 * B1);
  const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
  const bool inside = x < p.n[0] && y < p.n[1] && z < p.n[2];
  const int64_t v = (int64_t(z) * p.n[1] + y) * p.n[0] + x;
  const int me = ((lz + hz) * TL::Y + (ly + 1)) * TL::X + (lx + 1);
  bool fixed = !inside;
  if (inside)
    for (int k = 0; k < kMaxSeeds; ++k) fixed |= p.seed[src * kMaxSeeds + k] == v;
  hf_s[threadIdx.x] = inside ? p.hf[v] : 0.0;
  uint8_t* defer = p.defer + int64_t(src) * p.total;
  const bool was_deferred = inside && __ldcg(defer + v) != 0;
  constexpr int n_nbr = B2 > 1 ? 6 : 4;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  bool changed = false, settled = false, deferred = was_deferred;
  __syncthreads();
  for (int it = 0; it < p.sweeps; ++it) {
    const double mine = tile[me];
    bool need = it == 0 && (full || was_deferred);
    const uint8_t* mv = moved[it & 1];
#pragma unroll
    for (int k = 0; k < n_nbr; ++k) {
      const int off = (k & 1 ? 1 : -1) * (k < 2 ? 1 : (k < 4 ? SY : SZ));
      const bool fresh = it == 0 ? hstamp[me + off] > last : mv[me + off] != 0;
      need |= fresh && lt(tile[me + off], mine);
    }
    need &= !fixed;
    // pack the nodes that need a solve: warp ballots, then a prefix over warps
    const unsigned ballot = __ballot_sync(0xffffffffu, need);
    if (lane == 0) warp_count[warp] = __popc(ballot);
    __syncthreads();
    int base = 0, n_work = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) {
      const int c = warp_count[w];
      base += w < warp ? c : 0;
      n_work += c;
    }
    if (need) queue[base + __popc(ballot & ((1u << lane) - 1u))] = threadIdx.x;
    __syncthreads();
    for (int j = threadIdx.x; j < n_work; j += NT) {
      const int q = queue[j];
      const int qx = q % B0, qy = (q / B0) % B1, qz = q / (B0 * B1);
      const int m = ((qz + hz) * TL::Y + (qy + 1)) * TL::X + (qx + 1);
      // per axis the smaller neighbour (the halo is +inf outside the grid)
      double a0 = min2(tile[m - 1], tile[m + 1]);
      double a1 = min2(tile[m - SY], tile[m + SY]);
      double a2 = B2 > 1 ? min2(tile[m - SZ], tile[m + SZ]) : CUDART_INF;
      sort3(a0, a1, a2);
      const double hf = hf_s[q];
      cand_s[q] = godunov(a0, a1, a2, hf, 2.0 * hf * hf, 3.0 * hf * hf);
    }
    __syncthreads();  // every read of this sweep precedes its writes (Jacobi)
    bool upd = false;
    if (need) {
      const double cand = cand_s[threadIdx.x];
      deferred = false;
      if (lt(cand, mine) && !lt(p.stop_after, cand)) {
        // a lowering above this round's bound waits for a later round
        upd = !lt(p.tau, cand);
        deferred = !upd;
      }
      if (upd) {
        tile[me] = cand;
        changed = true;
      }
    }
    moved[(it + 1) & 1][me] = upd;
    if (!__syncthreads_or(upd)) {  // also orders these writes before the next reads
      settled = true;
      break;
    }
  }
  if (changed) {
    T[v] = tile[me];
    stamp[v] = p.phase;
  }
  if (deferred != was_deferred) defer[v] = deferred;
  const bool any = __syncthreads_or(changed);
  const bool waits = __syncthreads_or(deferred);
  if (threadIdx.x == 0) {
    const int64_t b = int64_t(src) * p.n_blocks + blk;
    if (any) p.changed[b] = 1;
    p.pending[b] = waits;
    // deferred nodes are remembered one by one, so they do not unsettle the block
    p.visited[b] = settled ? p.phase : kUnclean;
  }
}

// Next round's blocks: those that changed and their face neighbours, split by
// colour (bx + by + bz) & 1 into list[0..) and list[cap..).  Face neighbours
// have different colours, so the blocks of one colour never read a node that
// another block of the launch writes: each launch, and so the whole solve, is
// a fixed function of its input whatever order the blocks run in.
__global__ void eik_next_kernel(const int* changed, const int* pending, int nb, int n_blocks, int bn0,
                                int bn1, int bn2, int2* list, int64_t cap, int* n_list) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(nb) * n_blocks) return;
  const int src = int(i / n_blocks), blk = int(i - int64_t(src) * n_blocks);
  const int bx = blk % bn0, by = (blk / bn0) % bn1, bz = blk / (bn0 * bn1);
  const int* c = changed + int64_t(src) * n_blocks;
  bool act = c[blk] != 0 || pending[int64_t(src) * n_blocks + blk] != 0;
  act |= bx > 0 && c[blk - 1];
  act |= bx + 1 < bn0 && c[blk + 1];
  act |= by > 0 && c[blk - bn0];
  act |= by + 1 < bn1 && c[blk + bn0];
  act |= bz > 0 && c[blk - bn0 * bn1];
  act |= bz + 1 < bn2 && c[blk + bn0 * bn1];
  if (!act) return;
  const int colour = (bx + by + bz) & 1;
  list[colour * cap + atomicAdd(n_list + colour, 1)] = make_int2(src, blk);
}

__global__ void eik_fill_kernel(double* T, int64_t n, double v) {
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x)
    T[i] = v;
}

// Seeds: fixed values at the source cells' corners (stamped 0); their blocks
// count as changed and unsettled.
__global__ void eik_seed_kernel(double* T, int* stamp, const int64_t* seed, const double* seed_t,
                                int nb, int64_t total, int* changed, int* visited, int n_blocks, int n0,
                                int n1, int B0, int B1, int B2, int bn0, int bn1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * kMaxSeeds) return;
  const int64_t v = seed[i];
  if (v < 0) return;
  const int src = i / kMaxSeeds;
  T[int64_t(src) * total + v] = seed_t[i];
  stamp[int64_t(src) * total + v] = 0;
  const int x = int(v % n0), y = int((v / n0) % n1), z = int(v / (int64_t(n0) * n1));
  const int blk = ((z / B2) * bn1 + (y / B1)) * bn0 + (x / B0);
  changed[int64_t(src) * n_blocks + blk] = 1;
  visited[int64_t(src) * n_blocks + blk] = kUnclean;
}

// Values at the table's slots (tile order): [nb][n_slots], +inf for padding.
__global__ void eik_gather_kernel(const double* T, int64_t total, const int32_t* slot,
                                  int64_t n_slots, int nb, double* out) {
  const int64_t n = int64_t(nb) * n_slots;
  for (int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += int64_t(gridDim.x) * blockDim.x) {
    const int src = int(i / n_slots);
    const int32_t s = slot[i - int64_t(src) * n_slots];
    out[i] = s >= 0 ? T[int64_t(src) * total + s] : CUDART_INF;
  }
}

template <int B0, int B1, int B2>
cudaError_t launch_sweep(const EikParams& p, cudaStream_t st) {
  eik_sweep_kernel<B0, B1, B2><<<p.n_list, B0 * B1 * B2, 0, st>>>(p);
  return cudaGetLastError();
}

}  // namespace

struct GpuEikonal {
  GridDesc g;
  int B[3] = {1, 1, 1}, bn[3] = {1, 1, 1};
  int n_blocks = 0, batch = 0;
  int64_t total = 0, n_slots = 0;
  std::vector<double> c;  // host copy of the speed (source corners)
  double* d_hf = nullptr;
  int32_t* d_slot = nullptr;
  double* d_T = nullptr;
  int* d_changed = nullptr;
  int* d_stamp = nullptr;
  int* d_visited = nullptr;
  int* d_pending = nullptr;
  uint8_t* d_defer = nullptr;
  double hf_mean = 0.0, hf_max = 0.0;
  int2* d_list = nullptr;
  int* d_count = nullptr;
  int64_t* d_seed = nullptr;
  double* d_seed_t = nullptr;
  double* d_out = nullptr;
  cudaStream_t st = nullptr;
};

void gpu_eikonal_destroy(GpuEikonal* e) {
  if (!e) return;
  cudaFree(e->d_hf);
  cudaFree(e->d_slot);
  cudaFree(e->d_T);
  cudaFree(e->d_changed);
  cudaFree(e->d_stamp);
  cudaFree(e->d_visited);
  cudaFree(e->d_pending);
  cudaFree(e->d_defer);
  cudaFree(e->d_list);
  cudaFree(e->d_count);
  cudaFree(e->d_seed);
  cudaFree(e->d_seed_t);
  cudaFree(e->d_out);
  if (e->st) cudaStreamDestroy(e->st);
  delete e;
}

static bool cuda_ok(cudaError_t r, const char* what, std::string& err) {
  if (r == cudaSuccess) return true;
  err = std::string(what) + ": " + cudaGetErrorString(r);
  return false;
}

GpuEikonal* gpu_eikonal_create(const GridDesc& g, const float* speed,
                               const std::vector<int32_t>& slot_dense, int batch, std::string& err) {
  GpuEikonal* e = new GpuEikonal();
  e->g = g;
  e->batch = std::max(1, batch);
  e->total = g.total();
  e->n_slots = int64_t(slot_dense.size());
  if (g.ndim == 2) {
    e->B[0] = 16; e->B[1] = 16; e->B[2] = 1;
  } else {
    e->B[0] = 8; e->B[1] = 8; e->B[2] = 4;
  }
  for (int d = 0; d < 3; ++d) e->bn[d] = (g.n[d] + e->B[d] - 1) / e->B[d];
  e->n_blocks = e->bn[0] * e->bn[1] * e->bn[2];
  e->c.resize(size_t(e->total));
  std::vector<double> hf(size_t(e->total));
  for (int64_t v = 0; v < e->total; ++v) {
    e->c[v] = double(speed[v]);
    hf[v] = g.dx / e->c[v];
    e->hf_mean += hf[v];
    e->hf_max = std::max(e->hf_max, hf[v]);
  }
  e->hf_mean /= double(e->total);
  const size_t nbb = size_t(e->batch) * e->n_blocks;
  bool ok = cuda_ok(cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking), "stream", err) &&
            cuda_ok(cudaMalloc(&e->d_hf, size_t(e->total) * 8), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_slot, std::max<size_t>(slot_dense.size(), 1) * 4), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_T, size_t(e->batch) * e->total * 8), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_changed, nbb * 4), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_stamp, size_t(e->batch) * e->total * 4), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_visited, nbb * 4), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_pending, nbb * 4), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_defer, size_t(e->batch) * e->total), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_list, 2 * nbb * sizeof(int2)), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_count, 8), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_seed, size_t(e->batch) * kMaxSeeds * 8), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_seed_t, size_t(e->batch) * kMaxSeeds * 8), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_out, size_t(e->batch) * std::max<int64_t>(e->n_slots, 1) * 8),
                    "cudaMalloc", err) &&
            cuda_ok(cudaMemcpy(e->d_hf, hf.data(), hf.size() * 8, cudaMemcpyHostToDevice), "upload", err) &&
            (slot_dense.empty() ||
             cuda_ok(cudaMemcpy(e->d_slot, slot_dense.data(), slot_dense.size() * 4, cudaMemcpyHostToDevice),
                     "upload", err));
  if (!ok) {
    gpu_eikonal_destroy(e);
    return nullptr;
  }
  return e;
}

bool gpu_eikonal_slot_times(GpuEikonal* e, const double* sensors, int nb, double stop_after,
                            double* out, std::string& err) {
  if (nb < 1 || nb > e->batch) {
    err = "bad eikonal batch";
    return false;
  }
  const GridDesc& g = e->g;
  // source cells: corners fixed at distance / c, as the host march seeds them
  std::vector<int64_t> seed(size_t(nb) * kMaxSeeds, -1);
  std::vector<double> seed_t(size_t(nb) * kMaxSeeds, 0.0);
  for (int b = 0; b < nb; ++b) {
    int64_t* node = seed.data() + size_t(b) * kMaxSeeds;
    double* t = seed_t.data() + size_t(b) * kMaxSeeds;
    const int n = source_corners(g, sensors + 3 * size_t(b), node, t);
    if (n == 0) {
      err = "a sensor lies outside the grid box";
      return false;
    }
    for (int k = 0; k < n; ++k) t[k] = t[k] / e->c[node[k]];
  }
  cudaStream_t st = e->st;
  const int64_t nT = int64_t(nb) * e->total;
  const size_t nbb = size_t(nb) * e->n_blocks;
  if (!cuda_ok(cudaMemcpyAsync(e->d_seed, seed.data(), seed.size() * 8, cudaMemcpyHostToDevice, st), "seeds", err) ||
      !cuda_ok(cudaMemcpyAsync(e->d_seed_t, seed_t.data(), seed_t.size() * 8, cudaMemcpyHostToDevice, st), "seeds", err) ||
      !cuda_ok(cudaMemsetAsync(e->d_changed, 0, nbb * 4, st), "memset", err) ||
      !cuda_ok(cudaMemsetAsync(e->d_stamp, 0xFF, size_t(nT) * 4, st), "memset", err) ||
      !cuda_ok(cudaMemsetAsync(e->d_visited, 0xFF, nbb * 4, st), "memset", err) ||
      !cuda_ok(cudaMemsetAsync(e->d_pending, 0, nbb * 4, st), "memset", err) ||
      !cuda_ok(cudaMemsetAsync(e->d_defer, 0, size_t(nT), st), "memset", err))
    return false;
  eik_fill_kernel<<<1024, 256, 0, st>>>(e->d_T, nT, std::numeric_limits<double>::infinity());
  eik_seed_kernel<<<(nb * kMaxSeeds + 127) / 128, 128, 0, st>>>(
      e->d_T, e->d_stamp, e->d_seed, e->d_seed_t, nb, e->total, e->d_changed, e->d_visited,
      e->n_blocks, g.n[0], g.n[1], e->B[0], e->B[1], e->B[2], e->bn[0], e->bn[1]);
  if (!cuda_ok(cudaGetLastError(), "seed launch", err)) return false;

  EikParams p;
  p.T = e->d_T;
  p.hf = e->d_hf;
  p.seed = e->d_seed;
  p.list = e->d_list;
  p.changed = e->d_changed;
  p.stamp = e->d_stamp;
  p.visited = e->d_visited;
  p.pending = e->d_pending;
  p.defer = e->d_defer;
  // Rounds accept lowerings up to tau = (round + 1) * dtau (a bucketed
  // Dijkstra order): a node takes a value only once the values upwind of it
  // are final or nearly so, instead of passing provisional values far ahead
  // of the front.  dtau is a quarter block edge of the mean medium (8 x 8 x 4
  // blocks: two node spacings; 16 x 16: four), or 1/1024 of the time span
  // when that is coarser.
  const double t_end = std::min(stop_after, double(g.n[0] + g.n[1] + g.n[2]) * e->hf_max);
  const double dtau = std::max(0.25 * e->B[0] * e->hf_mean, t_end / 1024.0);
  for (int d = 0; d < 3; ++d) {
    p.n[d] = g.n[d];
    p.bn[d] = e->bn[d];
  }
  p.total = e->total;
  p.n_blocks = e->n_blocks;
  p.stop_after = stop_after;
  p.sweeps = 2 * std::max(e->B[0], std::max(e->B[1], e->B[2]));
  // rounds until no block changes; the cap only guards against a logic error
  const int64_t max_rounds = 1024 * int64_t(e->bn[0] + e->bn[1] + e->bn[2]) + 4096;
  const int64_t cap = int64_t(e->batch) * e->n_blocks;
  int n_list[2] = {0, 0};
  for (int64_t round = 0;; ++round) {
    if (round >= max_rounds) {
      err = "eikonal iteration did not settle";
      return false;
    }
    if (!cuda_ok(cudaMemsetAsync(e->d_count, 0, 8, st), "memset", err)) return false;
    const int64_t nthr = int64_t(nb) * e->n_blocks;
    eik_next_kernel<<<unsigned((nthr + 255) / 256), 256, 0, st>>>(
        e->d_changed, e->d_pending, nb, e->n_blocks, e->bn[0], e->bn[1], e->bn[2], e->d_list, cap,
        e->d_count);
    if (!cuda_ok(cudaMemcpyAsync(n_list, e->d_count, 8, cudaMemcpyDeviceToHost, st), "count", err) ||
        !cuda_ok(cudaStreamSynchronize(st), "eikonal round", err))
      return false;
    if (n_list[0] == 0 && n_list[1] == 0) break;
    if (!cuda_ok(cudaMemsetAsync(e->d_changed, 0, nbb * 4, st), "memset", err)) return false;
    for (int colour = 0; colour < 2; ++colour) {
      if (n_list[colour] == 0) continue;
      p.list = e->d_list + colour * cap;
      p.n_list = n_list[colour];
      p.phase = int(2 * round + colour + 1);
      p.tau = double(round + 1) * dtau;
      const cudaError_t r = g.ndim == 2 ? launch_sweep<16, 16, 1>(p, st) : launch_sweep<8, 8, 4>(p, st);
      if (!cuda_ok(r, "eikonal sweep launch", err)) return false;
    }
  }
  eik_gather_kernel<<<1024, 256, 0, st>>>(e->d_T, e->total, e->d_slot, e->n_slots, nb, e->d_out);
  if (!cuda_ok(cudaGetLastError(), "gather launch", err) ||
      !cuda_ok(cudaMemcpyAsync(out, e->d_out, size_t(nb) * e->n_slots * 8, cudaMemcpyDeviceToHost, st),
               "download", err) ||
      !cuda_ok(cudaStreamSynchronize(st), "eikonal", err))
    return false;
  return true;
}

int gpu_eikonal_batch(const GridDesc& g, int64_t n_slots, size_t budget) {
  const int64_t nodes = g.total();
  const int64_t blocks = nodes / 64 + 64;  // generous bound on blocks per source
  const int64_t per = nodes * 13 + n_slots * 8 + blocks * 28 + kMaxSeeds * 16;
  return int(std::max<int64_t>(1, std::min<int64_t>(64, int64_t(budget) / per)));
}

}  // namespace patbp
