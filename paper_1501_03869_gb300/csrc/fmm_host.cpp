// fmm_host.cpp -- host fast marching and travel-time table build.
//
// Sec. II-B: the eikonal equation |grad T|^2 = 1/c^2 is solved by fast
// marching, one run per sensor used as the point source (ray paths are
// reversible, so one run per sensor serves every pixel).  The update is the
// first-order Godunov upwind discretisation sum_d max(T - a_d, 0)^2 = (h/c)^2,
// a_d the smaller accepted neighbour along axis d.  Sec. III: this is the
// off-line step, done once per speed map and sensor layout.
//
// Implementation choices of this file: a one-node ghost layer around the grid
// (no bounds tests in the neighbour loop), an indexed 4-ary heap of (T, node)
// entries with the key held inline and decrease-key (ordered by (T, node), so
// the pop order is that of any exact priority queue), the root of the m-axis
// quadratic written as
// (S + sqrt(S^2 - m (Q - (h/c)^2))) / m, early exit once every wanted pixel is
// accepted or the front passes the end of the record, and one std::thread per
// core, each marching whole sensors.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <limits>
#include <thread>

#include "table.h"

namespace patbp {

namespace {
constexpr uint8_t kFar = 0, kTrial = 1, kAccepted = 2, kGhost = 3;
constexpr int kPad = 2;  // ghost layers per active side (the second-order stencil looks two nodes out)
constexpr double kInf = std::numeric_limits<double>::infinity();
}  // namespace

FastMarcher::FastMarcher(const GridDesc& g, const float* speed, const uint8_t* targets, int order)
    : g_(g), order_(order == 2 ? 2 : 1) {
  ptotal_ = 1;
  for (int d = 0; d < 3; ++d) {
    pn_[d] = d < g.ndim ? g.n[d] + 2 * kPad : 1;
    pstride_[d] = ptotal_;
    ptotal_ *= pn_[d];
  }
  t_.assign(ptotal_, kInf);
  st_.assign(ptotal_, kGhost);
  pos_.assign(ptotal_, -1);
  hf_.assign(ptotal_, 0.0);
  c_.assign(ptotal_, 0.0);
  wanted_.assign(ptotal_, 0);
  heap_.reserve(1 << 16);
  for (int64_t v = 0; v < g.total(); ++v) {
    int64_t pv = to_padded(v);
    c_[pv] = double(speed[v]);
    hf_[pv] = g.dx / c_[pv];
    wanted_[pv] = targets ? (targets[v] ? 1 : 0) : 0;
  }
}

int64_t FastMarcher::to_padded(int64_t v) const {
  int64_t p = 0;
  for (int d = 0; d < 3; ++d) {
    int64_t c = v % g_.n[d];
    v /= g_.n[d];
    p += (d < g_.ndim ? c + kPad : c) * pstride_[d];
  }
  return p;
}

// The pop order depends only on the total order of (T, node), not on the
// heap's shape, so the accepted sequence (and every value) is that of any
// exact priority queue with this order.
void FastMarcher::heap_up(int64_t i) {
  const HeapEntry e = heap_[i];
  while (i > 0) {
    const int64_t up = (i - 1) >> 2;
    if (!key_less(e, heap_[up])) break;
    heap_[i] = heap_[up];
    pos_[heap_[i].node] = int32_t(i);
    i = up;
  }
  heap_[i] = e;
  pos_[e.node] = int32_t(i);
}

void FastMarcher::heap_down(int64_t i) {
  const int64_t n = int64_t(heap_.size());
  const HeapEntry e = heap_[i];
  for (;;) {
    const int64_t c0 = 4 * i + 1;
    if (c0 >= n) break;
    int64_t c = c0;
    const int64_t c_end = std::min(c0 + 4, n);
    for (int64_t k = c0 + 1; k < c_end; ++k)
      if (key_less(heap_[k], heap_[c])) c = k;
    if (!key_less(heap_[c], e)) break;
    heap_[i] = heap_[c];
    pos_[heap_[i].node] = int32_t(i);
    i = c;
  }
  heap_[i] = e;
  pos_[e.node] = int32_t(i);
}

double FastMarcher::local_solve(int64_t pv, double hf) const {
  double a[3];
  int m = 0;
  for (int d = 0; d < g_.ndim; ++d) {
    const int64_t s = pstride_[d];
    double lo = st_[pv - s] == kAccepted ? t_[pv - s] : kInf;
    double hi = st_[pv + s] == kAccepted ? t_[pv + s] : kInf;
    double v = lo < hi ? lo : hi;
    if (v < kInf) a[m++] = v;
  }
  if (m == 0) return kInf;
  if (m > 1 && a[1] < a[0]) std::swap(a[0], a[1]);
  if (m > 2) {
    if (a[2] < a[1]) std::swap(a[1], a[2]);
    if (a[1] < a[0]) std::swap(a[0], a[1]);
  }
  // Grow the set of contributing axes while the root lies above the next a.
  double S = 0.0, Q = 0.0, root = kInf;
  const double hf2 = hf * hf;
  for (int k = 0; k < m; ++k) {
    S += a[k];
    Q += a[k] * a[k];
    const double kk = double(k + 1);
    double disc = S * S - kk * (Q - hf2);
    if (disc < 0.0) disc = 0.0;
    root = (S + std::sqrt(disc)) / kk;
    if (k + 1 == m || !(root > a[k + 1])) break;
  }
  return root;
}

// Second-order local solve (the printed stencil of Sec. II-B, the one-sided
// difference (3 T_i - 4 T_{i-1} + T_{i-2}) / 2h).  Per axis the upwind side is
// the accepted neighbour with the smaller time (the lower side on a tie); when
// the next node out on that side is accepted and not later, the axis enters as
// (9/4)(T - (4 t1 - t2)/3)^2, else as the first-order (T - t1)^2.  Axes join in
// increasing offset (a stable order) while the root lies above the next
// offset; an axis whose inclusion leaves no real root is not included.
// Unlike the first-order update the result can hinge on exact ties (the test
// t2 <= t1 at a source in a cell centre), so the arithmetic is kept in one
// fixed form -- one axis a + hf / sqrt(w), then sums W, M and C = sum w a^2 -
// hf^2 grown axis by axis -- and this file is compiled without contraction
// into FMAs, giving the same bits on every host.
double FastMarcher::local_solve2(int64_t pv, double hf) const {
  struct Axis {
    double off, w;
  } ax[3];
  int m = 0;
  for (int d = 0; d < g_.ndim; ++d) {
    const int64_t s = pstride_[d];
    const bool lo_ok = st_[pv - s] == kAccepted, hi_ok = st_[pv + s] == kAccepted;
    if (!lo_ok && !hi_ok) continue;
    const int64_t dir = (lo_ok && (!hi_ok || t_[pv - s] <= t_[pv + s])) ? -s : s;
    const double t1 = t_[pv + dir];
    const int64_t q2 = pv + 2 * dir;
    if (st_[q2] == kAccepted && t_[q2] <= t1)
      ax[m++] = Axis{(4.0 * t1 - t_[q2]) / 3.0, 2.25};
    else
      ax[m++] = Axis{t1, 1.0};
  }
  if (m == 0) return kInf;
  // stable ascending order of at most three axes (swap only when strictly out of order)
  for (int pass = 0; pass < 2; ++pass)
    for (int i = 0; i + 1 < m; ++i)
      if (ax[i].off > ax[i + 1].off) std::swap(ax[i], ax[i + 1]);
  double W = ax[0].w, M = ax[0].w * ax[0].off, C = ax[0].w * ax[0].off * ax[0].off - hf * hf;
  double root = ax[0].off + hf / std::sqrt(ax[0].w);
  for (int k = 1; k < m; ++k) {
    if (!(root > ax[k].off)) break;
    const double W2 = W + ax[k].w, M2 = M + ax[k].w * ax[k].off;
    const double C2 = C + ax[k].w * ax[k].off * ax[k].off;
    const double disc = M2 * M2 - W2 * C2;
    if (disc < 0.0) break;
    W = W2;
    M = M2;
    C = C2;
    root = (M + std::sqrt(disc)) / W;
  }
  return root;
}

int source_corners(const GridDesc& g, const double* src, int64_t* node, double* dist) {
  int cell[3] = {0, 0, 0};
  for (int d = 0; d < g.ndim; ++d) {
    if (g.n[d] < 2) return 0;
    double x = (src[d] - g.origin[d]) / g.dx;
    if (!(x >= 0.0) || !(x <= double(g.n[d] - 1))) return 0;
    int i = int(std::floor(x));
    cell[d] = std::min(i, g.n[d] - 2);
  }
  const int n = 1 << g.ndim;
  for (int corner = 0; corner < n; ++corner) {
    int64_t v = 0, mul = 1;
    double r2 = 0.0;
    for (int d = 0; d < g.ndim; ++d) {
      int i = cell[d] + ((corner >> d) & 1);
      double off = g.origin[d] + double(i) * g.dx - src[d];
      r2 += off * off;
      v += int64_t(i) * mul;
      mul *= g.n[d];
    }
    node[corner] = v;
    dist[corner] = std::sqrt(r2);
  }
  return n;
}

bool FastMarcher::solve(const double* src, std::vector<double>& T, double stop_after,
                        int64_t n_targets) {
  // reset interior nodes; ghosts keep kGhost
  std::fill(t_.begin(), t_.end(), kInf);
  std::fill(pos_.begin(), pos_.end(), -1);
  heap_.clear();
  const int nz = g_.ndim > 2 ? g_.n[2] : 1, ny = g_.ndim > 1 ? g_.n[1] : 1, nx = g_.n[0];
  const int oz = g_.ndim > 2 ? kPad : 0, oy = g_.ndim > 1 ? kPad : 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j) {
      int64_t row = (k + oz) * pstride_[2] + (j + oy) * pstride_[1] + kPad;
      std::fill(st_.begin() + row, st_.begin() + row + nx, kFar);
    }

  // Source cell: corners accepted with distance times local slowness.
  int64_t corner_node[8];
  double corner_dist[8];
  const int n_corners = source_corners(g_, src, corner_node, corner_dist);
  if (n_corners == 0) return false;
  int64_t wanted_left = n_targets;
  std::vector<int64_t> seeds;
  for (int corner = 0; corner < n_corners; ++corner) {
    int64_t pv = to_padded(corner_node[corner]);
    if (st_[pv] == kAccepted) continue;
    t_[pv] = corner_dist[corner] / c_[pv];
    st_[pv] = kAccepted;
    seeds.push_back(pv);
    if (wanted_[pv]) --wanted_left;
  }

  auto relax_neighbours = [&](int64_t pv) {
    for (int d = 0; d < g_.ndim; ++d) {
      for (int side = -1; side <= 1; side += 2) {
        int64_t q = pv + side * pstride_[d];
        uint8_t s = st_[q];
        if (s == kAccepted || s == kGhost) continue;
        double cand = order_ == 2 ? local_solve2(q, hf_[q]) : local_solve(q, hf_[q]);
        if (cand < t_[q]) {
          t_[q] = cand;
          if (s == kFar) {
            st_[q] = kTrial;
            heap_.push_back(HeapEntry{cand, q});
            heap_up(int64_t(heap_.size()) - 1);
          } else {
            heap_[pos_[q]].t = cand;  // a decrease: the entry moves up only
            heap_up(pos_[q]);
          }
        }
      }
    }
  };
  for (int64_t pv : seeds) relax_neighbours(pv);

  while (!heap_.empty()) {
    if (n_targets > 0 && wanted_left <= 0) break;
    const int64_t pv = heap_[0].node;
    if (heap_[0].t > stop_after) break;
    const HeapEntry last = heap_.back();
    heap_.pop_back();
    pos_[pv] = -1;
    if (!heap_.empty()) {
      heap_[0] = last;
      pos_[last.node] = 0;
      heap_down(0);
    }
    st_[pv] = kAccepted;
    if (wanted_[pv]) --wanted_left;
    relax_neighbours(pv);
  }

  // Export accepted values; anything not accepted is +inf (never reached or
  // beyond the early stop).
  T.resize(size_t(g_.total()));
  int64_t v = 0;
  for (int k = 0; k < nz; ++k)
    for (int j = 0; j < ny; ++j) {
      int64_t row = (k + oz) * pstride_[2] + (j + oy) * pstride_[1] + kPad;
      for (int i = 0; i < nx; ++i, ++v) T[v] = st_[row + i] == kAccepted ? t_[row + i] : kInf;
    }
  return true;
}

// ------------------------------------------------------------ pixel order --
namespace {
uint64_t hilbert_key(uint32_t side, uint32_t x, uint32_t y) {
  // Position of (x, y) along the Hilbert curve filling a side x side square
  // (side a power of two): quadrant digits, rotating the frame per level.
  uint64_t d = 0;
  for (uint32_t s = side >> 1; s > 0; s >>= 1) {
    uint32_t rx = (x & s) ? 1u : 0u;
    uint32_t ry = (y & s) ? 1u : 0u;
    d += uint64_t(s) * s * ((3u * rx) ^ ry);
    if (ry == 0) {
      if (rx == 1) {
        x = (s - 1) - (x & (s - 1));
        y = (s - 1) - (y & (s - 1));
      }
      std::swap(x, y);
    }
  }
  return d;
}

uint64_t morton_key(uint32_t x, uint32_t y, uint32_t z) {
  uint64_t k = 0;
  for (int b = 0; b < 21; ++b) {
    k |= uint64_t((x >> b) & 1u) << (3 * b);
    k |= uint64_t((y >> b) & 1u) << (3 * b + 1);
    k |= uint64_t((z >> b) & 1u) << (3 * b + 2);
  }
  return k;
}
}  // namespace

std::vector<int32_t> curve_order(const GridDesc& g, const uint8_t* mask) {
  std::vector<std::pair<uint64_t, int32_t>> keyed;
  const int64_t total = g.total();
  keyed.reserve(size_t(total));
  uint32_t side = 1;
  while (side < uint32_t(std::max(g.n[0], g.n[1]))) side <<= 1;
  for (int64_t v = 0; v < total; ++v) {
    if (mask && !mask[v]) continue;
    uint32_t x = uint32_t(v % g.n[0]);
    uint32_t y = uint32_t((v / g.n[0]) % g.n[1]);
    uint32_t z = uint32_t(v / (int64_t(g.n[0]) * g.n[1]));
    uint64_t key = g.ndim == 3 ? morton_key(x, y, z) : hilbert_key(side, x, y);
    keyed.emplace_back(key, int32_t(v));
  }
  std::sort(keyed.begin(), keyed.end());
  std::vector<int32_t> order(keyed.size());
  for (size_t i = 0; i < keyed.size(); ++i) order[i] = keyed[i].second;
  return order;
}

// ------------------------------------------------------------ pixel layout --
bool layout_pixels(const GridDesc& g, const uint8_t* mask, int P, bool compact_out, HostTable& out,
                   std::vector<int32_t>& order, std::string& err) {
  const int64_t total = g.total();
  order = curve_order(g, mask);
  const int64_t n_pix = int64_t(order.size());
  if (n_pix == 0) {
    err = "mask selects no pixel";
    return false;
  }
  const int n_tiles = int((n_pix + P - 1) / P);
  out.P = P;
  out.n_tiles = n_tiles;
  out.n_pix = n_pix;
  out.slot_dense.assign(size_t(n_tiles) * P, -1);
  out.slot_compact.assign(size_t(n_tiles) * P, -1);
  std::vector<int32_t> rank(size_t(total), -1);
  {
    int32_t r = 0;
    for (int64_t v = 0; v < total; ++v)
      if (!mask || mask[v]) rank[v] = r++;
  }
  for (int64_t i = 0; i < n_pix; ++i) {
    out.slot_dense[i] = order[i];
    out.slot_compact[i] = rank[order[i]];
  }
  out.zero_runs.clear();
  if (!compact_out && mask) {
    int64_t v = 0;
    while (v < total) {
      if (mask[v]) { ++v; continue; }
      int64_t s = v;
      while (v < total && !mask[v]) ++v;
      out.zero_runs.push_back(int32_t(s));
      out.zero_runs.push_back(int32_t(v - s));
    }
  }
  return true;
}

// ------------------------------------------------------------ table build --
namespace {

// Windows and offsets of one sensor over all tiles from the arrival times of
// the tile slots (time_at(t, p), s); returns the widest window.  Per tile the
// window [base, base + len) holds floor(u), floor(u) + 1 of every pixel heard
// within the record and one more sample for an offset that rounds up to the
// next integer in FP32; base is a multiple of 8 and len of 8.
template <class TimeAt>
int fill_sensor(HostTable& out, int s, double dt, double last_u, TimeAt time_at) {
  const int P = out.P, n_sensors = out.n_sensors;
  int span = 0;
  for (int t = 0; t < out.n_tiles; ++t) {
    const int32_t* slot = out.slot_dense.data() + size_t(t) * P;
    int64_t lo = std::numeric_limits<int64_t>::max(), hi = -1;
    for (int p = 0; p < P; ++p) {
      if (slot[p] < 0) continue;
      double u = time_at(t, p) / dt;
      if (!(u <= last_u)) continue;  // after the record (or unreached)
      int64_t i = int64_t(std::floor(u));
      lo = std::min(lo, i);
      hi = std::max(hi, i);
    }
    float* urow = out.u.data() + (size_t(t) * n_sensors + s) * P;
    if (hi < 0) {
      out.base[size_t(t) * n_sensors + s] = 0;
      continue;
    }
    int64_t base = lo & ~int64_t(7);
    int len = (int(hi - base + 3) + 7) & ~7;
    out.base[size_t(t) * n_sensors + s] = int32_t(base);
    out.len[size_t(t) * n_sensors + s] = uint16_t(len);
    span = std::max(span, len);
    for (int p = 0; p < P; ++p) {
      if (slot[p] < 0) continue;
      double u = time_at(t, p) / dt;
      if (!(u <= last_u)) continue;
      urow[p] = float(u - double(base));
    }
  }
  return span;
}

// Runs body(i) for i in [0, n) on all host threads; returns the largest result.
template <class Body>
int parallel_max(int n, Body body) {
  unsigned n_threads = std::max(1u, std::thread::hardware_concurrency());
  n_threads = std::min<unsigned>(n_threads, unsigned(std::max(n, 1)));
  std::atomic<int> next{0};
  std::vector<int> best(n_threads, 0);
  auto worker = [&](unsigned tid) {
    for (;;) {
      const int i = next.fetch_add(1);
      if (i >= n) break;
      best[tid] = std::max(best[tid], body(i));
    }
  };
  std::vector<std::thread> pool;
  for (unsigned i = 0; i < n_threads; ++i) pool.emplace_back(worker, i);
  for (auto& th : pool) th.join();
  return *std::max_element(best.begin(), best.end());
}

// The GPU solver's batches; the host fills batch k while the GPU solves k + 1.
bool table_times_gpu(const float* speed, const GridDesc& g, const double* sensors, int n_sensors,
                     double dt, double last_u, double stop_after, HostTable& out, int& span,
                     std::string& err) {
  const int64_t n_slots = int64_t(out.n_tiles) * out.P;
  const int batch = std::min(n_sensors, gpu_eikonal_batch(g, n_slots, size_t(8) << 30));
  GpuEikonal* e = gpu_eikonal_create(g, speed, out.slot_dense, batch, err);
  if (!e) return false;
  std::vector<double> buf[2];
  buf[0].resize(size_t(batch) * n_slots);
  buf[1].resize(size_t(batch) * n_slots);
  std::thread filler;
  int fill_span = 0;
  bool ok = true;
  for (int s0 = 0, k = 0; s0 < n_sensors; s0 += batch, ++k) {
    const int nb = std::min(batch, n_sensors - s0);
    double* Tk = buf[k & 1].data();  // the filler still reads the other buffer
    if (!gpu_eikonal_slot_times(e, sensors + 3 * size_t(s0), nb, stop_after, Tk, err)) {
      ok = false;
      break;
    }
    if (filler.joinable()) filler.join();
    filler = std::thread([&out, &fill_span, Tk, s0, nb, n_slots, dt, last_u]() {
      const int sp = parallel_max(nb, [&](int b) {
        const double* Tb = Tk + size_t(b) * n_slots;
        const int P = out.P;
        return fill_sensor(out, s0 + b, dt, last_u,
                           [Tb, P](int t, int p) { return Tb[size_t(t) * P + p]; });
      });
      fill_span = std::max(fill_span, sp);
    });
  }
  if (filler.joinable()) filler.join();
  gpu_eikonal_destroy(e);
  span = std::max(span, fill_span);
  return ok;
}

}  // namespace

bool build_table(const float* speed, const GridDesc& g, const double* sensors, int n_sensors,
                 const uint8_t* mask, double dt, int n_samples, int P, bool compact_out,
                 HostTable& out, std::string& err, int fmm_order, bool gpu_eikonal) {
  auto t_start = std::chrono::steady_clock::now();
  const int64_t total = g.total();
  for (int64_t v = 0; v < total; ++v) {
    if (!(speed[v] > 0.0f) || !std::isfinite(speed[v])) {
      err = "speed must be finite and > 0 at every node";
      return false;
    }
  }
  if (gpu_eikonal && fmm_order != 1) {
    err = "the GPU table build solves the first-order scheme only";
    return false;
  }
  std::vector<int32_t> order;
  if (!layout_pixels(g, mask, P, compact_out, out, order, err)) return false;
  const int64_t n_pix = out.n_pix;
  const int n_tiles = out.n_tiles;
  out.n_sensors = n_sensors;
  out.u.assign(size_t(n_tiles) * n_sensors * P, kOutOfRecord);
  out.base.assign(size_t(n_tiles) * n_sensors, 0);
  out.len.assign(size_t(n_tiles) * n_sensors, 0);
  for (int s = 0; s < n_sensors; ++s) {
    int64_t node[8];
    double dist[8];
    if (source_corners(g, sensors + 3 * s, node, dist) == 0) {
      err = "a sensor lies outside the grid box";
      return false;
    }
  }

  const double last_u = double(n_samples - 1);
  const double stop_after = last_u * dt * (1.0 + 1e-9);
  int span = 8;
  if (gpu_eikonal) {
    if (!table_times_gpu(speed, g, sensors, n_sensors, dt, last_u, stop_after, out, span, err))
      return false;
  } else {
    std::vector<uint8_t> wanted(size_t(total), 0);
    for (int32_t v : order) wanted[v] = 1;
    unsigned n_threads = std::max(1u, std::thread::hardware_concurrency());
    n_threads = std::min<unsigned>(n_threads, unsigned(n_sensors));
    std::atomic<int> next{0};
    std::vector<int> span_max(n_threads, 0);
    auto worker = [&](unsigned tid) {
      FastMarcher fm(g, speed, wanted.data(), fmm_order);
      std::vector<double> T;
      for (;;) {
        int s = next.fetch_add(1);
        if (s >= n_sensors) break;
        fm.solve(sensors + 3 * s, T, stop_after, n_pix);  // sources checked above
        const int32_t* slot = out.slot_dense.data();
        span_max[tid] = std::max(span_max[tid], fill_sensor(out, s, dt, last_u, [&](int t, int p) {
          return T[slot[size_t(t) * P + p]];
        }));
      }
    };
    std::vector<std::thread> pool;
    for (unsigned i = 0; i < n_threads; ++i) pool.emplace_back(worker, i);
    for (auto& th : pool) th.join();
    for (int sp : span_max) span = std::max(span, sp);
  }
  out.W = span;
  out.build_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return true;
}

}  // namespace patbp
