// table.h -- host-side travel-time table of the back projection (internal).
//
// The table is the product of the off-line step of Sec. III: fast-marching
// arrival times T_s(r) (Sec. II-B) for every sensor s and every reconstructed
// pixel r, stored for the on-line gather of Eq. (BP).
//
// Layout (all row-major, built for the gather kernel's TMA staging):
//   pixels are ordered along a space-filling curve (Hilbert in 2-D, Morton in
//   3-D) and cut into tiles of P consecutive pixels, so the pixels of a tile
//   are close in space and their arrival times from one sensor span few
//   samples;
//   u[tile][sensor][P]   FP32 offset u = T/dt - base, or kOutOfRecord when the
//                        arrival falls after the last sample (or the slot is
//                        padding);
//   base[tile][sensor]   int32 first sample of the window the tile needs from
//                        that sensor, a multiple of 8;
//   len[tile][sensor]    samples of that window, a multiple of 8 (0 when no
//                        pixel of the tile hears the sensor within the
//                        record); every in-record offset has floor(u) + 2 < len;
//   W                    the largest len (at least 8).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

namespace patbp {

constexpr float kOutOfRecord = 1.0e30f;

struct GridDesc {
  int ndim = 2;
  int n[3] = {1, 1, 1};
  double dx = 0.0;
  double origin[3] = {0.0, 0.0, 0.0};
  int64_t total() const { return int64_t(n[0]) * n[1] * n[2]; }
};

struct HostTable {
  int P = 0;
  int n_tiles = 0;
  int n_sensors = 0;
  int W = 0;
  int64_t n_pix = 0;
  std::vector<float> u;             // [n_tiles][n_sensors][P]
  std::vector<int32_t> base;        // [n_tiles][n_sensors]
  std::vector<uint16_t> len;        // [n_tiles][n_sensors]
  std::vector<int32_t> slot_dense;  // [n_tiles * P] dense grid index or -1
  std::vector<int32_t> slot_compact;// [n_tiles * P] raster rank among mask pixels or -1
  std::vector<int32_t> zero_runs;   // pairs (start, length) of non-mask runs of the grid
  // constant-speed delays (build_constant_layout): no u; instead
  std::vector<float> anchor;        // [n_tiles][n_sensors][8] per-sensor anchor of each tile
  std::vector<float> pixq;          // [n_tiles][P][4] per-pixel terms relative to the anchor
  double build_seconds = 0.0;
};

// Fast marching from one point source (Sec. II-B) on the host in FP64: the
// first-order Godunov update, or (order 2) the printed second-order stencil.
// speed[v] = c(v) > 0 at the nodes; `targets` (optional, total() bytes,
// nonzero = wanted) marks the nodes the caller needs.  solve() writes
// total() values to T; nodes never accepted hold +inf.  The march ends early
// once the smallest tentative time exceeds `stop_after` (s) or once all
// n_targets wanted nodes are accepted (n_targets = 0: never); values of
// accepted nodes never depend on either early stop.
class FastMarcher {
 public:
  FastMarcher(const GridDesc& g, const float* speed, const uint8_t* targets, int order = 1);
  bool solve(const double* src, std::vector<double>& T, double stop_after, int64_t n_targets);

 private:
  GridDesc g_;
  int order_ = 1;
  int pn_[3];            // padded extents (two ghost layers per active side)
  int64_t pstride_[3];
  int64_t ptotal_;
  std::vector<double> t_;     // padded arrival times
  std::vector<uint8_t> st_;   // padded states
  // Trial nodes in a 4-ary min-heap of (T, node) entries ordered by T, then
  // node id; the key lives in the entry, so sifting does not chase t_.
  struct HeapEntry {
    double t;
    int64_t node;
  };
  std::vector<int32_t> pos_;     // heap position of each padded node, -1 if absent
  std::vector<HeapEntry> heap_;
  std::vector<double> hf_;    // padded dx / c
  std::vector<double> c_;     // padded c
  std::vector<uint8_t> wanted_;
  int64_t to_padded(int64_t v) const;
  void heap_up(int64_t i);
  void heap_down(int64_t i);
  static bool key_less(const HeapEntry& a, const HeapEntry& b) {
    return a.t < b.t || (a.t == b.t && a.node < b.node);
  }
  double local_solve(int64_t pv, double hf) const;
  double local_solve2(int64_t pv, double hf) const;
};

// The grid cell holding a point source: its 2^ndim corners (dense indices)
// and their distances to the source (m); the march fixes each corner at
// distance / c.  Returns the number of corners, 0 if the source lies outside
// the grid box or an active axis has fewer than two nodes.
int source_corners(const GridDesc& g, const double* src, int64_t* node, double* dist);

// Builds the table for every sensor.  The arrival times come from the host
// march (all host threads) or, with gpu_eikonal (first order only), from the
// GPU fixed-point solver below; either way the windows are filled on the host
// by the same code, so both give the same table.
bool build_table(const float* speed, const GridDesc& g, const double* sensors, int n_sensors,
                 const uint8_t* mask, double dt, int n_samples, int P, bool compact_out,
                 HostTable& out, std::string& err, int fmm_order = 1, bool gpu_eikonal = false);

// First-order arrival times of batches of point sources on the current CUDA
// device (eikonal.cu): the Godunov system iterated block by block to its
// fixed point with the host march's arithmetic, so every value equals the
// host march's.  create() uploads dx / c and the table's slot map (dense
// index per tile slot, -1 padding) and sizes buffers for `batch` sources.
// slot_times() solves nb <= batch sources (xyz per source) and writes
// out[b][slot] = T (s), +inf for padding slots and for nodes later than
// stop_after.  Errors return nullptr / false with a message in err.
struct GpuEikonal;
GpuEikonal* gpu_eikonal_create(const GridDesc& g, const float* speed,
                               const std::vector<int32_t>& slot_dense, int batch, std::string& err);
bool gpu_eikonal_slot_times(GpuEikonal* e, const double* sensors, int nb, double stop_after,
                            double* out, std::string& err);
void gpu_eikonal_destroy(GpuEikonal* e);
// sources per batch that fit a device-memory budget (bytes)
int gpu_eikonal_batch(const GridDesc& g, int64_t n_slots, size_t budget);

// Pixel order used by the table: mask pixels (dense indices) sorted along the
// space-filling curve of the grid.
std::vector<int32_t> curve_order(const GridDesc& g, const uint8_t* mask);

// Tiles of the curve order: sets P, n_tiles, n_pix, both slot maps and the
// zero runs of `out`; `order` receives the curve order.  False if the mask is empty.
bool layout_pixels(const GridDesc& g, const uint8_t* mask, int P, bool compact_out, HostTable& out,
                   std::vector<int32_t>& order, std::string& err);

// Constant-speed delays (the conventional back projection, Sec. II-C):
// T_s(r) = |r - r_s| / c0, nothing stored per pixel and sensor.  Fills the
// pixel layout, the windows (base, len, W) exactly as build_table would for
// these delays (with a 1e-3-sample margin on both ends for the kernel's FP32
// evaluation), the anchors and the per-pixel terms.  Sensors may lie anywhere
// (inside the grid box or not); in 2-D only their x and y count.
bool build_constant_layout(double c0, const GridDesc& g, const double* sensors, int n_sensors,
                           const uint8_t* mask, double dt, int n_samples, int P, bool compact_out,
                           HostTable& out, std::string& err);

// Node coordinates of every tile slot ([n_tiles * P][3], padding slots 0) and
// every tile's anchor node (the centre of its pixels' bounding box, rounded
// down), the reference point of the per-pixel terms.
void tile_nodes(const GridDesc& g, const std::vector<int32_t>& slot_dense, int P, int n_tiles,
                std::vector<int32_t>& node, std::vector<int32_t>& anchor_node);

// Weights of the exact back projection (the solid angle of sensor s's element
// at pixel r over omega0, Sec. II-C): w = elem_s (n_s . (r - r_s)) /
// |r - r_s|^d / omega0, d = ndim (2-D: plane angle, x and y only).  The
// kernels evaluate it from a per-(tile, sensor) anchor [n_tiles][ns_pad][8] =
// (e.xyz, scale, n.xyz, d), e = unit (r0 - r_s) in node units times `unit`,
// and the per-pixel terms (2 D, |D|^2), D = unit (r - r0), as v = D + e:
// w = scale (n . v) / |v|^d with scale = elem / omega0 (unit / dx)^(d - 1).
// `unit` is the scale of the handle's existing per-pixel terms (the constant-
// speed kappa) or 1 when the layout makes them (make_pix).  Normals are
// normalised here; errors (zero normal, negative element, omega0 <= 0) return
// false with a message.
bool build_solid_angle_layout(const GridDesc& g, const std::vector<int32_t>& slot_dense, int P,
                              int n_tiles, const double* sensors, const double* normals,
                              const double* elem, int n_sensors, int n_sensors_pad, double omega0,
                              double unit, bool make_pix, std::vector<float>& wanchor,
                              std::vector<float>& pix, std::string& err);

}  // namespace patbp
