// const_host.cpp -- host layout of the conventional (constant-speed) back
// projection, the comparison method of Sec. III: Eq. (BP) with
// t_sj = |r_j - r_s| / c0 computed analytically instead of by fast marching
// (Sec. II-C).  Nothing is stored per (pixel, sensor): the gather kernel
// evaluates the delays from a 32-byte anchor per (tile, sensor) and 16 bytes
// per pixel, so its memory stream is the integrand windows alone.
//
// In sample units, kappa = dx / (c0 dt) samples per node spacing.  Each tile
// has an anchor node r0 (the centre of its pixels' bounding box, rounded down
// to a node); per sensor s the anchor holds e = kappa (r0 - r_s), u0 = |e|,
// u0 - base, the record cap (N_t - 1) - base, u0^2 and the evaluation mode;
// per pixel the terms 2 D and |D|^2 with D = kappa (r - r0).  The kernel's
// refinement from u0 errs by about eps |D| u0 / u and the direct evaluation
// of |D + e| by about eps (u0 + |D|) (eps the FP32 rounding), so the mode is
// direct (1) only where the sensor comes close to the tile:
// 2 min(u) (u0 + max|D|) < max|D| u0.  All of them are formed in FP64 and
// rounded once to FP32.  The windows (base, len) follow the stored-table rule
// with a margin of 1e-3 samples at both ends, which covers the kernel's FP32
// evaluation of the delays (a few 1e-6 samples).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <thread>

#include "table.h"

namespace patbp {

void tile_nodes(const GridDesc& g, const std::vector<int32_t>& slot_dense, int P, int n_tiles,
                std::vector<int32_t>& node, std::vector<int32_t>& anchor_node) {
  node.assign(size_t(n_tiles) * P * 3, 0);
  anchor_node.assign(size_t(n_tiles) * 3, 0);
  for (int t = 0; t < n_tiles; ++t) {
    int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
    for (int p = 0; p < P; ++p) {
      const int32_t v = slot_dense[size_t(t) * P + p];
      if (v < 0) continue;
      int32_t* x = node.data() + (size_t(t) * P + p) * 3;
      x[0] = int32_t(v % g.n[0]);
      x[1] = int32_t((v / g.n[0]) % g.n[1]);
      x[2] = int32_t(int64_t(v) / (int64_t(g.n[0]) * g.n[1]));
      for (int d = 0; d < 3; ++d) {
        lo[d] = std::min(lo[d], x[d]);
        hi[d] = std::max(hi[d], x[d]);
      }
    }
    int32_t* a = anchor_node.data() + size_t(t) * 3;
    for (int d = 0; d < 3; ++d) a[d] = hi[d] >= 0 ? (lo[d] + hi[d]) / 2 : 0;
  }
}

bool build_solid_angle_layout(const GridDesc& g, const std::vector<int32_t>& slot_dense, int P,
                              int n_tiles, const double* sensors, const double* normals,
                              const double* elem, int n_sensors, int n_sensors_pad, double omega0,
                              double unit, bool make_pix, std::vector<float>& wanchor,
                              std::vector<float>& pix, std::string& err) {
  if (!(omega0 > 0.0) || !std::isfinite(omega0)) {
    err = "omega0 must be finite and > 0";
    return false;
  }
  const int nd = g.ndim;
  std::vector<double> nrm(size_t(n_sensors) * 3, 0.0);
  for (int s = 0; s < n_sensors; ++s) {
    double len2 = 0.0;
    for (int d = 0; d < nd; ++d) {
      const double c = normals[3 * s + d];
      if (!std::isfinite(c) || !std::isfinite(sensors[3 * s + d])) {
        err = "sensor positions and normals must be finite";
        return false;
      }
      len2 += c * c;
    }
    if (!(len2 > 0.0)) {
      err = "sensor " + std::to_string(s) + " has a zero normal";
      return false;
    }
    if (!(elem[s] >= 0.0) || !std::isfinite(elem[s])) {
      err = "element sizes must be finite and >= 0";
      return false;
    }
    for (int d = 0; d < nd; ++d) nrm[3 * s + d] = normals[3 * s + d] / std::sqrt(len2);
  }
  std::vector<int32_t> node, anchor_node;
  tile_nodes(g, slot_dense, P, n_tiles, node, anchor_node);
  // w = elem (n . v_m) / |v_m|^d / omega0 with v_m = (dx / unit) v in the
  // kernel's units: scale = elem / omega0 * (unit / dx)^(d - 1)
  const double to_unit = unit / g.dx;
  wanchor.assign(size_t(n_tiles) * n_sensors_pad * 8, 0.0f);
  for (int t = 0; t < n_tiles; ++t) {
    const int32_t* a = anchor_node.data() + size_t(t) * 3;
    for (int s = 0; s < n_sensors; ++s) {
      float* w = wanchor.data() + (size_t(t) * n_sensors_pad + s) * 8;
      for (int d = 0; d < nd; ++d) {
        const double rs = (sensors[3 * s + d] - g.origin[d]) / g.dx;  // node units
        w[d] = float(unit * (double(a[d]) - rs));
        w[4 + d] = float(nrm[3 * s + d]);
      }
      w[3] = float(elem[s] / omega0 * std::pow(to_unit, double(nd - 1)));
      w[7] = float(nd);
    }
  }
  if (make_pix) {
    pix.assign(size_t(n_tiles) * P * 4, 0.0f);
    for (int t = 0; t < n_tiles; ++t) {
      const int32_t* a = anchor_node.data() + size_t(t) * 3;
      for (int p = 0; p < P; ++p) {
        if (slot_dense[size_t(t) * P + p] < 0) continue;
        const int32_t* x = node.data() + (size_t(t) * P + p) * 3;
        double D[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < nd; ++d) D[d] = unit * double(x[d] - a[d]);
        float* q = pix.data() + (size_t(t) * P + p) * 4;
        q[0] = float(2.0 * D[0]);
        q[1] = float(2.0 * D[1]);
        q[2] = float(2.0 * D[2]);
        q[3] = float(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
      }
    }
  }
  return true;
}

bool build_constant_layout(double c0, const GridDesc& g, const double* sensors, int n_sensors,
                           const uint8_t* mask, double dt, int n_samples, int P, bool compact_out,
                           HostTable& out, std::string& err) {
  const auto t_start = std::chrono::steady_clock::now();
  if (!(c0 > 0.0) || !std::isfinite(c0)) {
    err = "the constant sound speed must be finite and > 0";
    return false;
  }
  for (int s = 0; s < n_sensors; ++s)
    for (int d = 0; d < 3; ++d)
      if (!std::isfinite(sensors[3 * s + d])) {
        err = "sensor positions must be finite";
        return false;
      }
  std::vector<int32_t> order;
  if (!layout_pixels(g, mask, P, compact_out, out, order, err)) return false;
  out.n_sensors = n_sensors;
  const int n_tiles = out.n_tiles;
  const int nd = g.ndim;
  const double kappa = g.dx / (c0 * dt);
  const double last_u = double(n_samples - 1);
  constexpr double kMargin = 1e-3;

  // node coordinates of every slot and the anchor node of every tile
  std::vector<int32_t> node, anchor_node;
  tile_nodes(g, out.slot_dense, P, n_tiles, node, anchor_node);
  std::vector<double> reach(size_t(n_tiles), 0.0);  // max |D| over the tile
  out.pixq.assign(size_t(n_tiles) * P * 4, 0.0f);
  for (int t = 0; t < n_tiles; ++t) {
    const int32_t* a = anchor_node.data() + size_t(t) * 3;
    for (int p = 0; p < P; ++p) {
      if (out.slot_dense[size_t(t) * P + p] < 0) continue;  // padding: the anchor itself
      const int32_t* x = node.data() + (size_t(t) * P + p) * 3;
      double D[3] = {0.0, 0.0, 0.0};
      for (int d = 0; d < nd; ++d) D[d] = kappa * double(x[d] - a[d]);
      float* q = out.pixq.data() + (size_t(t) * P + p) * 4;
      q[0] = float(2.0 * D[0]);
      q[1] = float(2.0 * D[1]);
      q[2] = float(2.0 * D[2]);
      q[3] = float(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]);
      reach[t] = std::max(reach[t], std::sqrt(D[0] * D[0] + D[1] * D[1] + D[2] * D[2]));
    }
  }

  out.u.clear();
  out.anchor.assign(size_t(n_tiles) * n_sensors * 8, 0.0f);
  out.base.assign(size_t(n_tiles) * n_sensors, 0);
  out.len.assign(size_t(n_tiles) * n_sensors, 0);
  unsigned n_threads = std::max(1u, std::thread::hardware_concurrency());
  n_threads = std::min<unsigned>(n_threads, unsigned(n_sensors));
  std::atomic<int> next{0};
  std::vector<int> span_max(n_threads, 8);
  auto worker = [&](unsigned tid) {
    int span = 8;
    for (;;) {
      const int s = next.fetch_add(1);
      if (s >= n_sensors) break;
      double rs[3] = {0.0, 0.0, 0.0};  // sensor in node units
      for (int d = 0; d < nd; ++d) rs[d] = (sensors[3 * s + d] - g.origin[d]) / g.dx;
      for (int t = 0; t < n_tiles; ++t) {
        const int32_t* a = anchor_node.data() + size_t(t) * 3;
        double e[3] = {0.0, 0.0, 0.0};
        for (int d = 0; d < nd; ++d) e[d] = kappa * (double(a[d]) - rs[d]);
        const double u0 = std::sqrt(e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        double umin = INFINITY, umax = -INFINITY, uclose = INFINITY;
        for (int p = 0; p < P; ++p) {
          if (out.slot_dense[size_t(t) * P + p] < 0) continue;
          const int32_t* x = node.data() + (size_t(t) * P + p) * 3;
          double r2 = 0.0;
          for (int d = 0; d < nd; ++d) r2 += (double(x[d]) - rs[d]) * (double(x[d]) - rs[d]);
          const double u = kappa * std::sqrt(r2);
          uclose = std::min(uclose, u);
          if (u > last_u + kMargin) continue;  // after the record
          umin = std::min(umin, u);
          umax = std::max(umax, u);
        }
        const size_t i = size_t(t) * n_sensors + s;
        float* an = out.anchor.data() + i * 8;
        an[0] = float(e[0]);
        an[1] = float(e[1]);
        an[2] = float(e[2]);
        an[3] = float(u0);
        an[6] = float(u0 * u0);
        an[7] = 2.0 * uclose * (u0 + reach[t]) < reach[t] * u0 || u0 == 0.0 ? 1.0f : 0.0f;
        if (!(umax >= 0.0)) {  // no pixel of the tile hears the sensor within the record
          an[4] = float(u0);
          an[5] = -1.0f;
          continue;
        }
        const int64_t lo = std::max<int64_t>(0, int64_t(std::floor(umin - kMargin)));
        const int64_t hi = int64_t(std::floor(umax + kMargin));
        const int64_t base = lo & ~int64_t(7);
        const int len = (int(hi - base + 3) + 7) & ~7;
        out.base[i] = int32_t(base);
        out.len[i] = uint16_t(len);
        span = std::max(span, len);
        an[4] = float(u0 - double(base));
        an[5] = float(last_u - double(base));
      }
    }
    span_max[tid] = span;
  };
  std::vector<std::thread> pool;
  for (unsigned i = 0; i < n_threads; ++i) pool.emplace_back(worker, i);
  for (auto& th : pool) th.join();
  out.W = *std::max_element(span_max.begin(), span_max.end());
  out.build_seconds =
      std::chrono::duration<double>(std::chrono::steady_clock::now() - t_start).count();
  return true;
}

}  // namespace patbp
