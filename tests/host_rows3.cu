// Host check of the 3D direct kernel's row partition (rows3 / edge_row in d3.cuh): the interior launch and
// the edge launch together cover every (y, z) row exactly once, interior rows lie VMAX or more away from
// the y and z faces, edge rows do not, and a split is chosen only where edge rows are at most an eighth.
#include <cstdio>
#include <set>
#include <utility>

#include "d3.cuh"

template <int V>
static int check(int nx, int ny, int nz) {
  lbm::Geom3 g{};
  g.nx = nx;
  g.ny = ny;
  g.nz = nz;
  const lbm::Rows3 r = lbm::rows3<V>(g);
  std::set<std::pair<int, int>> seen;
  long long n = 0;
  if (r.interior == 0) {  // one launch over every row
    for (int z = 0; z < nz; ++z)
      for (int y = 0; y < ny; ++y) {
        seen.insert({y, z});
        ++n;
      }
  } else {
    for (int rb = 0; rb < r.interior; ++rb) {
      const int z = V + rb / r.ny_in, y = V + rb % r.ny_in;
      if (!(y >= V && y < ny - V && z >= V && z < nz - V)) return 1;
      seen.insert({y, z});
      ++n;
    }
    for (long long e = 0; e < r.edge; ++e) {
      int y, z;
      lbm::edge_row<V>(g, e, y, z);
      if (y < 0 || y >= ny || z < 0 || z >= nz) return 2;
      if (y >= V && y < ny - V && z >= V && z < nz - V) return 3;
      seen.insert({y, z});
      ++n;
    }
    if (8 * r.edge > (long long)ny * nz) return 4;
  }
  if (n != (long long)ny * nz || (long long)seen.size() != n) return 5;
  return 0;
}

int main() {
  int bad = 0;
  const int sizes[] = {1, 2, 3, 5, 7, 8, 13, 16, 48, 64, 100, 257};
  for (int ny : sizes)
    for (int nz : sizes)
      for (int nx : {1, 3, 8}) {
        const int a = check<1>(nx, ny, nz), b = check<3>(nx, ny, nz);
        if (a || b) {
          std::printf("FAIL nx=%d ny=%d nz=%d: %d %d\n", nx, ny, nz, a, b);
          ++bad;
        }
      }
  std::printf(bad ? "partition FAILED\n" : "partition ok\n");
  return bad != 0;
}
