// eikonal.cu -- arrival times of many point sources on the GPU (Sec. II-B),
// equal bit for bit to the host fast marching (first order).
//
// The first-order Godunov upwind system has one solution (the fast marching
// solution), and every node's value is the local solve of its neighbours'
// final values.  So instead of marching, the GPU iterates that local solve to
// its exact fixed point, block by block: each CTA holds one block of nodes of
// one source (16 x 16 in 2-D, 8 x 8 x 4 in 3-D) with a one-node halo in shared
// memory and sweeps it (Jacobi) until nothing changes or a sweep budget is
// spent; the next round processes the blocks that changed and their face
// neighbours.  Values only decrease, from +inf, and the loop ends when a round
// changes nothing: every node then equals the local solve of its neighbours.
//
// Bitwise equality with the host march needs the same arithmetic: the source
// cell's corners are fixed at distance / c, the local solve sorts the axis
// minima with the host's compare-and-swap steps and grows the set of axes with
// the same sums, every operation explicitly rounded (no FMA contraction; the
// host file is compiled without contraction too).  Values above the record end
// (stop_after) are never written, as the host march stops there; they cannot
// influence earlier arrivals.
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

struct EikParams {
  double* T;            // [nb][total] arrival times (s)
  const double* hf;     // [total] dx / c
  const int64_t* seed;  // [nb][kMaxSeeds] fixed nodes (-1 = none)
  const int2* list;     // active (source, block) pairs
  int n_list;
  int* changed;         // [nb][n_blocks] set when a block's values changed
  int n[3];             // nodes per axis (x first)
  int bn[3];            // blocks per axis
  int ndim;
  int64_t total;
  int n_blocks;
  double stop_after;
  int sweeps;           // sweep budget per block visit
};

// The host fast marching's first-order local solve, operation for operation.
// a holds the per-axis upwind values, +inf for an axis without one; the host
// sorts only its m finite values, and sorting all three gives the same
// ascending finite values, so the sums below are the host's.
__device__ __forceinline__ double root_step(double S, double Q, double hf2, int k) {
  const double kk = double(k + 1);  // kk * x is exact for kk = 1, 2 and rounded once for 3
  double disc = __dsub_rn(__dmul_rn(S, S), __dmul_rn(kk, __dsub_rn(Q, hf2)));
  if (disc < 0.0) disc = 0.0;
  const double num = __dadd_rn(S, __dsqrt_rn(disc));
  // x / 1 and x / 2 are exact as x and x * 0.5: the same bits as the host's division
  return k == 0 ? num : (k == 1 ? __dmul_rn(num, 0.5) : __ddiv_rn(num, 3.0));
}

__device__ double local_solve(double a0, double a1, double a2, double hf) {
  if (a1 < a0) { const double t = a0; a0 = a1; a1 = t; }
  if (a2 < a1) { const double t = a1; a1 = a2; a2 = t; }
  if (a1 < a0) { const double t = a0; a0 = a1; a1 = t; }
  if (!(a0 < CUDART_INF)) return CUDART_INF;
  const double hf2 = __dmul_rn(hf, hf);
  double S = a0, Q = __dmul_rn(a0, a0);  // 0 + x is x
  double root = root_step(S, Q, hf2, 0);
  if (!(a1 < CUDART_INF) || !(root > a1)) return root;
  S = __dadd_rn(S, a1);
  Q = __dadd_rn(Q, __dmul_rn(a1, a1));
  root = root_step(S, Q, hf2, 1);
  if (!(a2 < CUDART_INF) || !(root > a2)) return root;
  S = __dadd_rn(S, a2);
  Q = __dadd_rn(Q, __dmul_rn(a2, a2));
  return root_step(S, Q, hf2, 2);
}

// Tile with a one-node halo: extents B + 2 per active axis.
template <int B0, int B1, int B2>
struct Tile {
  static constexpr int X = B0 + 2, Y = B1 + 2, Z = B2 > 1 ? B2 + 2 : 1;
  static constexpr int N = X * Y * Z;
};

template <int B0, int B1, int B2>
__global__ void __launch_bounds__(B0 * B1 * B2) eik_sweep_kernel(const EikParams p) {
  using TL = Tile<B0, B1, B2>;
  constexpr int SY = TL::X, SZ = TL::X * TL::Y;
  __shared__ double tile[TL::N];
  // moved[j][i]: node i changed in the sweep before one that reads moved[j]
  // (a node whose neighbours did not move would solve to the same value)
  __shared__ uint8_t moved[2][TL::N];
  const int2 job = p.list[blockIdx.x];
  const int src = job.x, blk = job.y;
  const int bx = blk % p.bn[0], by = (blk / p.bn[0]) % p.bn[1], bz = blk / (p.bn[0] * p.bn[1]);
  const int x0 = bx * B0, y0 = by * B1, z0 = bz * B2;
  double* T = p.T + int64_t(src) * p.total;
  const int hz = B2 > 1 ? 1 : 0;
  // load the block and its halo; nodes outside the grid are +inf
  for (int i = threadIdx.x; i < TL::N; i += blockDim.x) {
    const int tx = i % TL::X, ty = (i / TL::X) % TL::Y, tz = i / (TL::X * TL::Y);
    const int x = x0 + tx - 1, y = y0 + ty - 1, z = z0 + tz - hz;
    double v = CUDART_INF;
    if (x >= 0 && x < p.n[0] && y >= 0 && y < p.n[1] && z >= 0 && z < p.n[2])
      v = __ldcg(T + (int64_t(z) * p.n[1] + y) * p.n[0] + x);
    tile[i] = v;
    moved[0][i] = 0;
    moved[1][i] = 0;
  }
  const int lx = threadIdx.x % B0, ly = (threadIdx.x / B0) % B1, lz = threadIdx.x / (B0 * B1);
  const int x = x0 + lx, y = y0 + ly, z = z0 + lz;
  const bool inside = x < p.n[0] && y < p.n[1] && z < p.n[2];
  const int64_t v = (int64_t(z) * p.n[1] + y) * p.n[0] + x;
  const int me = ((lz + hz) * TL::Y + (ly + 1)) * TL::X + (lx + 1);
  bool fixed = !inside;
  if (inside)
    for (int k = 0; k < kMaxSeeds; ++k) fixed |= p.seed[src * kMaxSeeds + k] == v;
  const double hf = inside ? p.hf[v] : 0.0;
  bool changed = false;
  __syncthreads();
  for (int it = 0; it < p.sweeps; ++it) {
    double cand = CUDART_INF;
    const uint8_t* mv = moved[it & 1];
    bool need = it == 0 || mv[me - 1] || mv[me + 1] || mv[me - SY] || mv[me + SY];
    if (B2 > 1) need = need || mv[me - SZ] || mv[me + SZ];
    if (!fixed && need) {
      // per axis the smaller neighbour (the halo is +inf outside the grid)
      const double x_lo = tile[me - 1], x_hi = tile[me + 1];
      const double y_lo = tile[me - SY], y_hi = tile[me + SY];
      double wz = CUDART_INF;
      if (B2 > 1) {
        const double z_lo = tile[me - SZ], z_hi = tile[me + SZ];
        wz = z_lo < z_hi ? z_lo : z_hi;
      }
      cand = local_solve(x_lo < x_hi ? x_lo : x_hi, y_lo < y_hi ? y_lo : y_hi, wz, hf);
    }
    __syncthreads();  // every read of this sweep precedes its writes (Jacobi)
    bool upd = false;
    if (cand < tile[me] && cand <= p.stop_after) {
      tile[me] = cand;
      changed = true;
      upd = true;
    }
    moved[(it + 1) & 1][me] = upd;
    if (!__syncthreads_or(upd)) break;  // also orders these writes before the next reads
  }
  if (changed) T[v] = tile[me];
  if (__syncthreads_or(changed) && threadIdx.x == 0) p.changed[int64_t(src) * p.n_blocks + blk] = 1;
}

// Next round's blocks: those that changed and their face neighbours, split by
// colour (bx + by + bz) & 1 into list[0..) and list[cap..).  Face neighbours
// have different colours, so the blocks of one colour never read a node that
// another block of the launch writes: each launch, and so the whole solve, is
// a fixed function of its input whatever order the blocks run in.
__global__ void eik_next_kernel(const int* changed, int nb, int n_blocks, int bn0, int bn1, int bn2,
                                int2* list, int64_t cap, int* n_list) {
  const int64_t i = int64_t(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= int64_t(nb) * n_blocks) return;
  const int src = int(i / n_blocks), blk = int(i - int64_t(src) * n_blocks);
  const int bx = blk % bn0, by = (blk / bn0) % bn1, bz = blk / (bn0 * bn1);
  const int* c = changed + int64_t(src) * n_blocks;
  bool act = c[blk] != 0;
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

// Seeds: fixed values at the source cells' corners; their blocks count as changed.
__global__ void eik_seed_kernel(double* T, const int64_t* seed, const double* seed_t, int nb,
                                int64_t total, int* changed, int n_blocks, int n0, int n1, int B0,
                                int B1, int B2, int bn0, int bn1) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nb * kMaxSeeds) return;
  const int64_t v = seed[i];
  if (v < 0) return;
  const int src = i / kMaxSeeds;
  T[int64_t(src) * total + v] = seed_t[i];
  const int x = int(v % n0), y = int((v / n0) % n1), z = int(v / (int64_t(n0) * n1));
  const int blk = ((z / B2) * bn1 + (y / B1)) * bn0 + (x / B0);
  changed[int64_t(src) * n_blocks + blk] = 1;
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
  }
  const size_t nbb = size_t(e->batch) * e->n_blocks;
  bool ok = cuda_ok(cudaStreamCreateWithFlags(&e->st, cudaStreamNonBlocking), "stream", err) &&
            cuda_ok(cudaMalloc(&e->d_hf, size_t(e->total) * 8), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_slot, std::max<size_t>(slot_dense.size(), 1) * 4), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_T, size_t(e->batch) * e->total * 8), "cudaMalloc", err) &&
            cuda_ok(cudaMalloc(&e->d_changed, nbb * 4), "cudaMalloc", err) &&
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
      !cuda_ok(cudaMemsetAsync(e->d_changed, 0, nbb * 4, st), "memset", err))
    return false;
  eik_fill_kernel<<<1024, 256, 0, st>>>(e->d_T, nT, std::numeric_limits<double>::infinity());
  eik_seed_kernel<<<(nb * kMaxSeeds + 127) / 128, 128, 0, st>>>(
      e->d_T, e->d_seed, e->d_seed_t, nb, e->total, e->d_changed, e->n_blocks, g.n[0], g.n[1], e->B[0],
      e->B[1], e->B[2], e->bn[0], e->bn[1]);
  if (!cuda_ok(cudaGetLastError(), "seed launch", err)) return false;

  EikParams p;
  p.T = e->d_T;
  p.hf = e->d_hf;
  p.seed = e->d_seed;
  p.list = e->d_list;
  p.changed = e->d_changed;
  for (int d = 0; d < 3; ++d) {
    p.n[d] = g.n[d];
    p.bn[d] = e->bn[d];
  }
  p.ndim = g.ndim;
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
        e->d_changed, nb, e->n_blocks, e->bn[0], e->bn[1], e->bn[2], e->d_list, cap, e->d_count);
    if (!cuda_ok(cudaMemcpyAsync(n_list, e->d_count, 8, cudaMemcpyDeviceToHost, st), "count", err) ||
        !cuda_ok(cudaStreamSynchronize(st), "eikonal round", err))
      return false;
    if (n_list[0] == 0 && n_list[1] == 0) break;
    if (!cuda_ok(cudaMemsetAsync(e->d_changed, 0, nbb * 4, st), "memset", err)) return false;
    for (int colour = 0; colour < 2; ++colour) {
      if (n_list[colour] == 0) continue;
      p.list = e->d_list + colour * cap;
      p.n_list = n_list[colour];
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
  const int64_t per = nodes * 8 + n_slots * 8 + blocks * 12 + kMaxSeeds * 16;
  return int(std::max<int64_t>(1, std::min<int64_t>(64, int64_t(budget) / per)));
}

}  // namespace patbp
