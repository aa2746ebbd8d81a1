// Uniform grid over a cylinder forest that lists, per cell, the only cylinders that can be
// the nearest one for a point of the cell (host side; the quadrotor rollout's cost role
// searches the list of its cell instead of every cylinder).
//
// For a cell box B (widened by kGridMargin) and a cylinder j with centre c_j and radius r_j,
// the distance to its surface over B lies in [dist(c_j, B) - r_j, maxdist(c_j, B) - r_j].
// Let U = min_j (maxdist(c_j, B) - r_j).  A cylinder with dist(c_j, B) - r_j > U + kGridMargin
// is farther than some other cylinder by more than kGridMargin at every point of B, so it can
// be neither the exact nearest nor, since the FP32 distances are within about 1e-5 m of the
// exact ones, the FP32 nearest.  The minimum over the list is therefore the same float as the
// minimum over all cylinders (a minimum is exact in any order).  Points outside the grid use
// every cylinder.  Cells are 1 m (a power of two, so the FP32 cell index of a point is off by
// far less than the margin), doubled until the grid and its lists fit the caps.  Every list
// holds at least one cylinder (the device reads each list's last entry unconditionally).
#pragma once
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

namespace mppi {

constexpr double kGridMargin = 1e-3;   // metres
constexpr double kGridPad = 3.0;       // metres of grid around the outermost cylinders
constexpr int kGridMaxCells = 2048;
constexpr int kGridMaxIndices = 16384;

struct ForestGrid {
  float ox = 0.0f, oy = 0.0f, inv_h = 0.0f;
  int nx = 0, ny = 0;
  std::vector<uint16_t> off;  // [nx * ny + 1] start of each cell's list in idx
  std::vector<uint8_t> idx;   // cylinder indices, cell by cell
  size_t bytes() const { return sizeof(uint16_t) * off.size() + idx.size(); }
};

// obs: [n][3] (x, y, radius).  Returns false (no grid: every query searches all cylinders)
// for an empty forest or when no cell size up to 64 m fits the caps.
inline bool build_forest_grid(const float *obs, int n, ForestGrid &g) {
  g = ForestGrid{};
  if (n <= 0 || n > 256) return false;
  double xmin = INFINITY, xmax = -INFINITY, ymin = INFINITY, ymax = -INFINITY, rmax = 0.0;
  for (int j = 0; j < n; ++j) {
    xmin = std::min(xmin, static_cast<double>(obs[3 * j]));
    xmax = std::max(xmax, static_cast<double>(obs[3 * j]));
    ymin = std::min(ymin, static_cast<double>(obs[3 * j + 1]));
    ymax = std::max(ymax, static_cast<double>(obs[3 * j + 1]));
    rmax = std::max(rmax, static_cast<double>(obs[3 * j + 2]));
  }
  if (!std::isfinite(xmin + xmax + ymin + ymax + rmax)) return false;
  const double x0 = std::floor(xmin - rmax - kGridPad), y0 = std::floor(ymin - rmax - kGridPad);
  for (double h = 1.0; h <= 64.0; h *= 2.0) {
    const int nx = static_cast<int>(std::ceil((xmax + rmax + kGridPad - x0) / h));
    const int ny = static_cast<int>(std::ceil((ymax + rmax + kGridPad - y0) / h));
    if (static_cast<long>(nx) * ny > kGridMaxCells) continue;
    std::vector<uint16_t> off(static_cast<size_t>(nx) * ny + 1, 0);
    std::vector<uint8_t> idx;
    bool fits = true;
    std::vector<double> lb(n);
    for (int iy = 0; iy < ny && fits; ++iy)
      for (int ix = 0; ix < nx && fits; ++ix) {
        const double bx0 = x0 + ix * h - kGridMargin, bx1 = x0 + (ix + 1) * h + kGridMargin;
        const double by0 = y0 + iy * h - kGridMargin, by1 = y0 + (iy + 1) * h + kGridMargin;
        double ub_min = INFINITY;
        for (int j = 0; j < n; ++j) {
          const double cx = obs[3 * j], cy = obs[3 * j + 1], r = obs[3 * j + 2];
          const double dxl = std::max(0.0, std::max(bx0 - cx, cx - bx1));
          const double dyl = std::max(0.0, std::max(by0 - cy, cy - by1));
          const double dxu = std::max(std::fabs(bx0 - cx), std::fabs(cx - bx1));
          const double dyu = std::max(std::fabs(by0 - cy), std::fabs(cy - by1));
          lb[j] = std::hypot(dxl, dyl) - r;
          ub_min = std::min(ub_min, std::hypot(dxu, dyu) - r);
        }
        const size_t before = idx.size();
        for (int j = 0; j < n; ++j)
          if (lb[j] <= ub_min + kGridMargin) idx.push_back(static_cast<uint8_t>(j));
        if (idx.size() == before) return false;  // never: the cylinder attaining ub_min is listed
        if (idx.size() > static_cast<size_t>(kGridMaxIndices)) fits = false;
        off[static_cast<size_t>(iy) * nx + ix + 1] = static_cast<uint16_t>(idx.size());
      }
    if (!fits) continue;
    g.ox = static_cast<float>(x0);
    g.oy = static_cast<float>(y0);
    g.inv_h = static_cast<float>(1.0 / h);
    g.nx = nx;
    g.ny = ny;
    g.off = std::move(off);
    g.idx = std::move(idx);
    return true;
  }
  return false;
}

}  // namespace mppi
