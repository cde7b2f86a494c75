// host_sanitize.cpp -- test harness: the library's host-side table code (fast
// marching of both orders, table and window build, pixel layout, constant-speed
// and solid-angle layouts) run on small 2-D and 3-D cases, built with the
// address and undefined-behaviour sanitizers by tests/test_host_sanitizers.py.
// The GPU solver's entry points are stubbed: nothing here touches a GPU.
#include <cmath>
#include <cstdio>
#include <random>
#include <string>
#include <vector>

#include "table.h"

namespace patbp {
struct GpuEikonal {};
GpuEikonal* gpu_eikonal_create(const GridDesc&, const float*, const std::vector<int32_t>&, int,
                               std::string& err) {
  err = "no GPU in this harness";
  return nullptr;
}
bool gpu_eikonal_slot_times(GpuEikonal*, const double*, int, double, double*, std::string& err) {
  err = "no GPU in this harness";
  return false;
}
void gpu_eikonal_destroy(GpuEikonal*) {}
int gpu_eikonal_batch(const GridDesc&, int64_t, size_t) { return 1; }
}  // namespace patbp

using namespace patbp;

static int fails = 0;
#define CHECK(c)                                                  \
  do {                                                            \
    if (!(c)) {                                                   \
      std::printf("FAILED %s:%d %s\n", __FILE__, __LINE__, #c);   \
      ++fails;                                                    \
    }                                                             \
  } while (0)

static void run_case(int ndim, const int n[3], int n_sensors, int n_samples, bool with_mask,
                     unsigned seed) {
  GridDesc g;
  g.ndim = ndim;
  for (int d = 0; d < 3; ++d) g.n[d] = d < ndim ? n[d] : 1;
  g.dx = 1e-4;
  std::mt19937 rng(seed);
  std::uniform_real_distribution<double> U(0.0, 1.0);
  std::vector<float> speed(size_t(g.total()));
  for (auto& c : speed) c = float(1400.0 + 1600.0 * U(rng));
  std::vector<uint8_t> mask(size_t(g.total()), 1);
  if (with_mask)
    for (auto& m : mask) m = U(rng) < 0.6 ? 1 : 0;
  mask[0] = 1;
  std::vector<double> sensors(size_t(n_sensors) * 3, 0.0);
  for (int s = 0; s < n_sensors; ++s)
    for (int d = 0; d < ndim; ++d) sensors[3 * s + d] = U(rng) * (g.n[d] - 1) * g.dx;
  // sensors exactly on the grid's corners and on its far boundary
  for (int d = 0; d < ndim; ++d) sensors[d] = 0.0;
  if (n_sensors > 1)
    for (int d = 0; d < ndim; ++d) sensors[3 + d] = (g.n[d] - 1) * g.dx;
  const double dt = 2e-8;
  for (int order = 1; order <= 2; ++order) {
    FastMarcher fm(g, speed.data(), mask.data(), order);
    std::vector<double> T;
    for (int s = 0; s < n_sensors; ++s) {
      CHECK(fm.solve(sensors.data() + 3 * s, T, 1e30, 0));
      CHECK(T.size() == size_t(g.total()));
      for (double t : T) CHECK(t >= 0.0 && std::isfinite(t));
    }
    for (int P : {128, 256}) {
      HostTable tab;
      std::string err;
      CHECK(build_table(speed.data(), g, sensors.data(), n_sensors, with_mask ? mask.data() : nullptr,
                        dt, n_samples, P, with_mask, tab, err, order, false));
      CHECK(tab.u.size() == size_t(tab.n_tiles) * n_sensors * P);
      CHECK(tab.W % 8 == 0);
      // the GPU route reports its error instead of running
      HostTable tab2;
      if (order == 1)
        CHECK(!build_table(speed.data(), g, sensors.data(), n_sensors, nullptr, dt, n_samples, P, false,
                           tab2, err, 1, true));
      HostTable ct;
      CHECK(build_constant_layout(1540.0, g, sensors.data(), n_sensors, with_mask ? mask.data() : nullptr,
                                  dt, n_samples, P, false, ct, err));
      const int ns_pad = (n_sensors + 3) & ~3;
      std::vector<double> normals(size_t(n_sensors) * 3, 0.0), elem(size_t(n_sensors), 1e-4);
      for (int s = 0; s < n_sensors; ++s) normals[3 * s] = 1.0;
      std::vector<float> wa, pix;
      CHECK(build_solid_angle_layout(g, tab.slot_dense, P, tab.n_tiles, sensors.data(), normals.data(),
                                     elem.data(), n_sensors, ns_pad, 2.0 * M_PI, 1.0, true, wa, pix, err));
      CHECK(wa.size() == size_t(tab.n_tiles) * ns_pad * 8 && pix.size() == size_t(tab.n_tiles) * P * 4);
      normals[0] = 0.0;
      CHECK(!build_solid_angle_layout(g, tab.slot_dense, P, tab.n_tiles, sensors.data(), normals.data(),
                                      elem.data(), n_sensors, ns_pad, 2.0 * M_PI, 1.0, true, wa, pix, err));
    }
  }
  // a source outside the grid is refused
  int64_t node[8];
  double dist[8];
  double outside[3] = {-1e-3, 0.0, 0.0};
  CHECK(source_corners(g, outside, node, dist) == 0);
}

int main() {
  const int a[3] = {37, 29, 1}, b[3] = {13, 11, 9}, c[3] = {2, 2, 2};
  run_case(2, a, 5, 300, true, 1u);
  run_case(2, a, 3, 40, false, 2u);  // a record that ends inside the grid
  run_case(3, b, 4, 200, true, 3u);
  run_case(3, c, 2, 8, false, 4u);   // the smallest grid
  std::printf(fails ? "failures: %d\n" : "ok\n", fails);
  return fails ? 1 : 0;
}
