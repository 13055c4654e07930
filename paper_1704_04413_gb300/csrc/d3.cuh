// Kernels of the 3D lattices (Tab. II): fused pull-stream-and-collide and the field kernels (initial state,
// moments, population planes, FP64 conservation sums).  Populations are SoA f[i][z][y][x]: rows padded to
// 128 bytes (pitch), planes of ny rows, population blocks of nz planes.
#pragma once
#include <cuda_runtime.h>

#include "bulk.cuh"
#include "collide3.cuh"
#include "step.cuh"

namespace lbm {

struct Geom3 {
  long long pstride;  // elements per population block (nz * plane)
  long long plane;    // elements per z plane (ny * pitch)
  int pitch;          // elements per row
  int nx, ny, nz;
  int bc[3];          // BC_PERIODIC / BC_ZERO_GRADIENT per axis
  int* status;        // device word: nonzero after a staged step kernel gave up waiting on its copies
  unsigned long long wait_ns;  // limit of the staged kernels' bounded waits (kBulkWaitNs by default)
  int fault_block;     // test hook: this block's producer announces but never issues its last tile's copies
};

template <int Q>
struct PullOffsets3 {
  long long src[Q];  // byte offset of the pulled source of population i from the cell's address in block 0
  long long dst[Q];  // byte offset of population i's block
  int cy[Q], cz[Q];  // velocity components, indexed at run time by the copy-issuing lanes
};

// Blocks per SM the register allocation must allow.  D3Q103 in FP32 fits 128 registers without spills
// (four 128-thread blocks a SM, against two at the 255 it takes unbounded); in FP64 a cap spills kilobytes.
template <class L, class Real>
struct Step3Blocks {
  static constexpr int MIN = L::Q > 40 ? (sizeof(Real) == 4 ? 4 : 1) : (L::Q > 20 ? 3 : 4);
};

// The same for the staged kernel's 160-thread blocks.  Measured at 256^3: D3Q27 and D3V39 with 16-bit
// storage gain from a fourth block (96 registers, 1.07x); their FP32 kernels (three blocks fit the
// shared memory anyway) and D3Q19 (at 72 registers for five blocks) lose to the tighter schedule.
template <class L, class S>
struct Staged3Blocks {
  static constexpr int MIN = L::Q > 20 ? (sizeof(S) == 2 ? 4 : 3) : 4;
};

// Storage formats: all five on every lattice.  D3Q103's kernels are the largest, so its 16-bit step kernels
// are built in translation units of their own (d3_q103_<collision>16.cu), compiled in parallel with the
// FP64 / FP32 ones.
template <class L>
struct Storages3 {
  static constexpr bool SIXTEEN_BIT = true;
};

// Rows of the direct kernel: interior rows (at least VMAX away from the y and z faces, nx >= VMAX) and the
// others.  On large grids each class runs in a launch of its own, so that neither kernel carries the
// other's load sequence (the two together overflowed the instruction cache on D3Q103: 74 % of the stall
// samples were no_instruction); where edge rows are more than an eighth of the grid, the second launch
// would be a fraction of a wave and one launch of the kernel with both sequences is faster (D3Q103 FP32:
// 256^3, 4.7 % edge rows, split 5.14 -> 5.46 GLUPS; 128 x 64 x 64, 18 %, combined 2.43, split 1.99, the
// general sequence alone 0.97).
struct Rows3 {
  int interior;     // count of interior rows; 0 = one launch over every row (ROWS_ALL)
  int ny_in;        // interior rows per plane
  long long edge;   // count of edge rows
};
constexpr int ROWS_ALL = 0, ROWS_INTERIOR = 1, ROWS_EDGE = 2;

template <int V>
__host__ __device__ inline Rows3 rows3(const Geom3& g) {
  Rows3 r{};
  const long long all = (long long)g.ny * g.nz;
  if (g.ny > 2 * V && g.nz > 2 * V && g.nx >= V) {
    r.ny_in = g.ny - 2 * V;
    r.interior = r.ny_in * (g.nz - 2 * V);
    r.edge = (long long)2 * V * g.ny + (long long)(g.nz - 2 * V) * 2 * V;
    if (8 * r.edge > all) r = Rows3{0, 0, 0};
  }
  return r;
}

// Edge row e -> (y, z): the 2 V planes nearest the z faces whole, then 2 V rows of every other plane.
template <int V>
__host__ __device__ __forceinline__ void edge_row(const Geom3& g, long long e, int& y, int& z) {
  if (e < (long long)2 * V * g.ny) {
    const int k = (int)(e / g.ny);
    y = (int)(e - (long long)k * g.ny);
    z = k < V ? k : g.nz - 2 * V + k;
  } else {
    const long long e2 = e - (long long)2 * V * g.ny;
    const int k = (int)(e2 % (2 * V));
    z = V + (int)(e2 / (2 * V));
    y = k < V ? k : g.ny - 2 * V + k;
  }
}

// One thread per cell; a block is STEP_BX consecutive x of one (y, z) row.  Interior rows take one load
// sequence with the x wrap folded into a base pointer per x-velocity; edge rows (and grids thinner than the
// stencil) the general per-population source coordinates.  ROWS selects the rows of a launch.
template <class L, int COLL, class Real, class S, int ROWS>
__global__ void __launch_bounds__(STEP_BX, Step3Blocks<L, Real>::MIN)
    k_step3(const S* __restrict__ fin, S* __restrict__ fout, Geom3 g, int nbx, Rows3 rows, CollParams<Real> P,
            const __grid_constant__ PullOffsets3<L::Q> off) {
  const int rb = blockIdx.x / nbx;
  const int bx = blockIdx.x - rb * nbx;
  int y, z;
  if constexpr (ROWS == ROWS_EDGE) {
    edge_row<L::VMAX>(g, rb, y, z);
  } else if constexpr (ROWS == ROWS_INTERIOR) {
    z = L::VMAX + rb / rows.ny_in;
    y = L::VMAX + (rb - (rb / rows.ny_in) * rows.ny_in);
  } else {
    y = rb % g.ny;
    z = rb / g.ny;
  }
  const int x_raw = bx * STEP_BX + threadIdx.x;
  const bool act = x_raw < g.nx;  // no early return: D3Q103's blocks meet at a barrier below
  const int x = act ? x_raw : g.nx - 1;
  const long long cen = (long long)z * g.plane + (long long)y * g.pitch + x;
  Real q[L::Q];
  const bool interior = ROWS == ROWS_INTERIOR ||
                        (ROWS == ROWS_ALL && y >= L::VMAX && y + L::VMAX < g.ny && z >= L::VMAX &&
                         z + L::VMAX < g.nz && g.nx >= L::VMAX);
  if (ROWS != ROWS_EDGE && interior) {
    const char* c = reinterpret_cast<const char*>(fin + cen);
    const char* cb[2 * L::VMAX + 1];
    sfor<0, 2 * L::VMAX + 1>([&](auto J) {
      constexpr int j = LBM_CI(J);
      constexpr int cx = j - L::VMAX;
      if constexpr (cx == 0) {
        cb[j] = c;
      } else {
        const int xs = x - cx;
        int fix;
        if (g.bc[0] == BC_PERIODIC)
          fix = (xs < 0 ? g.nx : 0) - (xs >= g.nx ? g.nx : 0);
        else
          fix = (xs < 0 ? -xs : 0) - (xs >= g.nx ? xs - g.nx + 1 : 0);
        cb[j] = c + (long long)fix * (long long)sizeof(S);
      }
    });
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      q[i] = (Real)ld_raw<S>(cb[L::CX[i] + L::VMAX] + off.src[i]);
    });
  } else {
    const char* b = reinterpret_cast<const char*>(fin);
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      const int xs = src_coord(x, L::CX[i], g.nx, g.bc[0]);
      const int ys = src_coord(y, L::CY[i], g.ny, g.bc[1]);
      const int zs = src_coord(z, L::CZ[i], g.nz, g.bc[2]);
      q[i] = (Real)ld_raw<S>(b + off.dst[i] +
                             ((long long)zs * g.plane + (long long)ys * g.pitch + xs) * (long long)sizeof(S));
    });
  }
  // D3Q103's collision does not fit the instruction cache: the block's warps enter it together, so that they
  // fetch the same code at the same time (256^3 FP32: 5.46 -> 5.60 GLUPS; binary16 unchanged)
  if constexpr (L::Q > 100) __syncthreads();
  collide3<L, COLL, Store<S>::SHIFTED, Real>(q, P);
  if (!act) return;
  char* o = reinterpret_cast<char*>(fout + cen);
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    Store<S>::st(reinterpret_cast<S*>(o + off.dst[i]), q[i]);
  });
}

// Two cells a thread for the interior rows of D3Q103 with the RR collision, on x-periodic grids of even nx:
// thread t of a block takes columns x = 2 t, 2 t + 1 of its row and collides both in packed FP32x2
// (vec2.cuh), one instruction for both cells, which halves the instructions fetched per cell of this
// lattice's long, fully unrolled collision (the one-cell kernel is bound by instruction fetch).  The
// collision runs as a stream (collide3_rr): each pulled population pair enters the moments as it arrives and
// each rebuilt pair is stored at once, so neither the 103 pulled nor the 103 rebuilt pairs stay live.  An
// even x-velocity is pulled with one aligned load for both cells, an odd one with one load a cell; each
// store is one aligned pair.
// Four 128-thread blocks a SM (128 registers, no spills): measured at 256^3 (FP32 / binary16 GLUPS) against
// 5.29 / 6.49 at two blocks, 6.15 / 7.26 at three and 5.92 / 7.34 at five (88 B of spills); the one-cell
// kernel ran 5.70 / 6.64.
template <class L, class S>
struct Step3Pair {
  static constexpr bool ENABLED = L::Q > 100;
  static constexpr int MIN_BLOCKS = 4;
};

// ROWS as for k_step3: interior rows take one base pointer per x-velocity; edge rows (and every row of a grid
// without the split) the per-population source coordinates (periodic or zero-gradient y and z faces).
template <class L, class S, int ROWS>
__global__ void __launch_bounds__(STEP_BX, Step3Pair<L, S>::MIN_BLOCKS)
    k_step3_pair(const S* __restrict__ fin, S* __restrict__ fout, Geom3 g, int nbx, Rows3 rows, CollParams<F2> P,
                 const __grid_constant__ PullOffsets3<L::Q> off) {
  const int rb = blockIdx.x / nbx;
  const int bx = blockIdx.x - rb * nbx;
  int y, z;
  if constexpr (ROWS == ROWS_EDGE) {
    edge_row<L::VMAX>(g, rb, y, z);
  } else if constexpr (ROWS == ROWS_INTERIOR) {
    z = L::VMAX + rb / rows.ny_in;
    y = L::VMAX + (rb - (rb / rows.ny_in) * rows.ny_in);
  } else {
    y = rb % g.ny;
    z = rb / g.ny;
  }
  const int x = 2 * (bx * STEP_BX + (int)threadIdx.x);
  if (x >= g.nx) return;  // nx is even: a pair is whole or absent (no barrier below)
  const long long cen = (long long)z * g.plane + (long long)y * g.pitch + x;
  char* o = reinterpret_cast<char*>(fout + cen);
  auto store = [&](auto I, F2 v) {
    constexpr int i = LBM_CI(I);
    st_pair<S>(reinterpret_cast<S*>(o + off.dst[i]), v);
  };
  if constexpr (ROWS == ROWS_INTERIOR) {
    const char* c = reinterpret_cast<const char*>(fin + cen);
    // one base pointer per x-velocity and cell, moved by a whole row where x - c_x leaves [0, nx) (periodic x,
    // nx >= VMAX: one fold); an even c_x moves both cells of the pair together
    const char* cb0[2 * L::VMAX + 1];
    const char* cb1[2 * L::VMAX + 1];
    auto fold = [&](int xs) { return (xs < 0 ? g.nx : 0) - (xs >= g.nx ? g.nx : 0); };
    sfor<0, 2 * L::VMAX + 1>([&](auto J) {
      constexpr int j = LBM_CI(J);
      constexpr int cx = j - L::VMAX;
      if constexpr (cx == 0) {
        cb0[j] = c;
        cb1[j] = c;
      } else {
        cb0[j] = c + (long long)fold(x - cx) * (long long)sizeof(S);
        cb1[j] = (cx % 2 == 0) ? cb0[j] : c + (long long)fold(x + 1 - cx) * (long long)sizeof(S);
      }
    });
    collide3_rr<L, Store<S>::SHIFTED, F2>(
        [&](auto I) -> F2 {
          constexpr int i = LBM_CI(I);
          constexpr int j = L::CX[i] + L::VMAX;
          const long long so = off.src[i];
          if constexpr (L::CX[i] % 2 == 0) {
            return ld_pair<S>(cb0[j] + so);
          } else {
            const float a = ld_raw<S>(cb0[j] + so);
            const float b = ld_raw<S>(cb1[j] + so + (long long)sizeof(S));
            return F2(a, b);
          }
        },
        P, store);
  } else {
    // source columns per x-velocity (periodic x, even nx: an even c_x keeps the pair together and aligned),
    // source row and plane per population
    int xs0[2 * L::VMAX + 1], xs1[2 * L::VMAX + 1];
    sfor<0, 2 * L::VMAX + 1>([&](auto J) {
      constexpr int j = LBM_CI(J);
      constexpr int cx = j - L::VMAX;
      xs0[j] = src_coord(x, cx, g.nx, BC_PERIODIC);
      xs1[j] = (cx % 2 == 0) ? xs0[j] + 1 : src_coord(x + 1, cx, g.nx, BC_PERIODIC);
    });
    const char* base = reinterpret_cast<const char*>(fin);
    collide3_rr<L, Store<S>::SHIFTED, F2>(
        [&](auto I) -> F2 {
          constexpr int i = LBM_CI(I);
          constexpr int j = L::CX[i] + L::VMAX;
          const int ys = src_coord(y, L::CY[i], g.ny, g.bc[1]);
          const int zs = src_coord(z, L::CZ[i], g.nz, g.bc[2]);
          const char* row = base + off.dst[i] + ((long long)zs * g.plane + (long long)ys * g.pitch) * (long long)sizeof(S);
          if constexpr (L::CX[i] % 2 == 0) {
            return ld_pair<S>(row + (long long)xs0[j] * (long long)sizeof(S));
          } else {
            const float a = ld_raw<S>(row + (long long)xs0[j] * (long long)sizeof(S));
            const float b = ld_raw<S>(row + (long long)xs1[j] * (long long)sizeof(S));
            return F2(a, b);
          }
        },
        P, store);
  }
}

// Staged variant for x-periodic grids whose rows are whole 16-byte units: a persistent block walks row tiles
// of BXT cells (256, or 128 where a 256-cell stage would exceed 44 KB).  A producer warp copies every
// population's source row segment of a tile, pull-shifted in y and z, with cp.async.bulk into a ring of
// STAGES shared-memory stages; 4 compute warps (BXT / 128 cells a thread) read the pulled populations from
// the stage, collide, and store to global memory.  A row that fits one tile is copied whole, one copy per
// population, and the periodic x wrap is an index inside it; a longer row is tiled with PAD cells of margin
// on both sides and its two edge tiles add the wrapped columns as copies of their own.  Each stage has a
// full barrier (the copied bytes) and an empty barrier (one arrival per compute warp), so the copies run up
// to STAGES tiles ahead of the compute and no warp waits for another one's arithmetic.  The copy count, not
// the byte count, is what the copy engine's throughput is spent on, hence the wide tiles.
template <class L, class S>
struct Stage3 {
  static constexpr int UNIT = 16 / (int)sizeof(S);                           // cells per 16 bytes
  static constexpr int PAD = (L::VMAX + UNIT - 1) / UNIT * UNIT;              // stencil margin, whole units
  // 256-cell tiles where a stage stays within 44 KB (every 3D lattice below D3Q103 except FP64 storage)
  static constexpr int BXT = L::Q * (256 + 2 * PAD) * (int)sizeof(S) <= 44 * 1024 ? 256 : 128;
  static constexpr int CPT = BXT / 128;                                       // cells a compute thread
  static constexpr int W = BXT + 2 * PAD;                                     // cells per staged row
  static constexpr int ROW_BYTES = W * (int)sizeof(S);
  static constexpr int STAGE_BYTES = L::Q * ROW_BYTES;
  static constexpr int STAGES_FIT = 56 * 1024 / STAGE_BYTES;
  static constexpr int STAGES = STAGES_FIT < 2 ? 2 : (STAGES_FIT > 4 ? 4 : STAGES_FIT);
  static constexpr int SMEM = STAGES * STAGE_BYTES + 128;                    // + alignment slack
  static constexpr int CW = 4;                                                // compute warps
  static constexpr int THREADS = 32 * CW + 32;                                // + the producer warp
  // D3Q103's collision holds 255 registers a thread: one staged block of 160 threads a SM against the
  // direct kernel's two of 128 (measured 2.1 against 3.7 GLUPS at 256^3, FP32); it keeps the direct kernel
  static constexpr bool ENABLED = L::Q < 100;
};

// Row tiles (bx, y, z), x-tile fastest; a block of the staged kernel walks one contiguous run of them.
struct TileWalk {
  int bx, y, z;
  __device__ TileWalk(long long t, int nbx, int ny) {
    const long long row = t / nbx;
    bx = (int)(t - row * nbx);
    y = (int)(row % ny);
    z = (int)(row / ny);
  }
  __device__ __forceinline__ void next(int nbx, int ny) {
    if (++bx == nbx) {
      bx = 0;
      if (++y == ny) {
        y = 0;
        ++z;
      }
    }
  }
};

template <class L, int COLL, class Real, class S>
__global__ void __launch_bounds__(Stage3<L, S>::THREADS, Staged3Blocks<L, S>::MIN)
    k_step3_staged(const S* __restrict__ fin, S* __restrict__ fout, Geom3 g, int nbx, long long ntiles,
                   CollParams<Real> P, const __grid_constant__ PullOffsets3<L::Q> off) {
  using St = Stage3<L, S>;
  constexpr int NS = St::STAGES;
  extern __shared__ unsigned char smem_raw[];
  __shared__ uint64_t full[NS], empty[NS];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~uintptr_t(127));
  const int tid = threadIdx.x;
  const int warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], St::CW);
    }
    mbar_init_fence();
  }
  __syncthreads();
  const bool whole_rows = nbx == 1;  // the x wrap is an index inside the staged row
  // this block's tiles: [t_begin, t_begin + n_mine), an equal share of the grid's
  const long long t_begin = blockIdx.x * ntiles / gridDim.x;
  const int n_mine = (int)((blockIdx.x + 1LL) * ntiles / gridDim.x - t_begin);

  if (warp == St::CW) {
    // producer: tile k of this block goes to stage k % NS once the compute warps released its previous use
    TileWalk tw(t_begin, nbx, g.ny);
    int k = 0;
    bool ok = true;
    for (; k < n_mine; ++k, tw.next(nbx, g.ny)) {
      const int s = k % NS;
      if (k >= NS) ok = mbar_wait(&empty[s], (uint32_t)(((k / NS) + 1) & 1), g.wait_ns);
      if (!__all_sync(0xffffffffu, ok)) break;
      // test hook: the last tile's copies are announced but not issued (every earlier stage has been
      // consumed, so no copy is in flight when the block ends)
      const bool skip = (int)blockIdx.x == g.fault_block && k == n_mine - 1;
      const int y = tw.y, z = tw.z;
      const int x0 = tw.bx * St::BXT;
      const int xa = max(x0 - St::PAD, 0), xb = min(x0 + St::BXT + St::PAD, g.nx);
      const int left = (!whole_rows && x0 - St::PAD < 0) ? St::PAD : 0;
      const int right =
          (!whole_rows && x0 + St::BXT + St::PAD > g.nx) ? min(x0 + St::BXT + St::PAD - g.nx, St::PAD) : 0;
      const uint32_t per_row = (uint32_t)(xb - xa + left + right) * (uint32_t)sizeof(S);
      if (lane == 0) mbar_arrive_expect_tx(&full[s], per_row * (uint32_t)L::Q);
      __syncwarp();
      unsigned char* st = sm + (size_t)s * St::STAGE_BYTES;
      const char* base = reinterpret_cast<const char*>(fin);
      for (int i = lane; i < L::Q && !skip; i += 32) {  // one population per lane
        const int ys = src_coord(y, off.cy[i], g.ny, g.bc[1]);
        const int zs = src_coord(z, off.cz[i], g.nz, g.bc[2]);
        const char* src =
            base + off.dst[i] + ((long long)zs * g.plane + (long long)ys * g.pitch) * (long long)sizeof(S);
        unsigned char* dst = st + i * St::ROW_BYTES;
        bulk_g2s(dst + (xa - x0 + St::PAD) * (int)sizeof(S), src + (long long)xa * sizeof(S),
                 (uint32_t)(xb - xa) * (uint32_t)sizeof(S), &full[s]);
        if (left)
          bulk_g2s(dst, src + (long long)(g.nx - St::PAD) * sizeof(S), (uint32_t)St::PAD * (uint32_t)sizeof(S),
                   &full[s]);
        if (right)
          bulk_g2s(dst + (g.nx - x0 + St::PAD) * (int)sizeof(S), src, (uint32_t)right * (uint32_t)sizeof(S),
                   &full[s]);
      }
    }
    if (!ok) {
      // a compute warp stopped releasing stages: flag it, and wait (bounded) for this block's copies that may
      // still be in flight, the last use of every stage, before the block's shared memory is released
      if (lane == 0) {
        atomicExch(g.status, 1);
        for (int j = 1; j <= NS; ++j)
          if (k - j >= 0) mbar_wait(&full[(k - j) % NS], (uint32_t)(((k - j) / NS) & 1), g.wait_ns);
      }
    }
    return;
  }

  // compute warps
  TileWalk tw(t_begin, nbx, g.ny);
  for (int k = 0; k < n_mine; ++k, tw.next(nbx, g.ny)) {
    const int s = k % NS;
    if (!__all_sync(0xffffffffu, mbar_wait(&full[s], (uint32_t)((k / NS) & 1), g.wait_ns))) {
      // the copies of this tile did not arrive: flag it and stop (the producer then gives up on this stage)
      if (lane == 0) atomicExch(g.status, 1);
      return;
    }
    const int y = tw.y, z = tw.z;
    const int x0 = tw.bx * St::BXT;
    const S* sp = reinterpret_cast<const S*>(sm + (size_t)s * St::STAGE_BYTES);
    sfor<0, St::CPT>([&](auto Cc) {
      constexpr int c = LBM_CI(Cc);
      const int x = x0 + c * 128 + tid;
      const bool active = x < g.nx;
      Real q[L::Q];
      if (active) {
        // staged position of the pulled source x - cx, per x-velocity
        int pos[2 * L::VMAX + 1];
        sfor<0, 2 * L::VMAX + 1>([&](auto J) {
          constexpr int j = LBM_CI(J);
          int xs = x - (j - L::VMAX);
          if (whole_rows) xs += (xs < 0 ? g.nx : 0) - (xs >= g.nx ? g.nx : 0);
          pos[j] = xs - x0 + St::PAD;
        });
        sfor<0, L::Q>([&](auto I) {
          constexpr int i = LBM_CI(I);
          constexpr int j = L::CX[i] + L::VMAX;
          const S v = sp[i * St::W + pos[j]];
          if constexpr (sizeof(S) == 8)
            q[i] = (Real)sm_decode_d(v);
          else
            q[i] = (Real)sm_decode<S>(v);
        });
      }
      if constexpr (c == St::CPT - 1) {
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);  // this warp has read the stage: the producer may refill it
      }
      if (active) {
        collide3<L, COLL, Store<S>::SHIFTED, Real>(q, P);
        char* o = reinterpret_cast<char*>(fout + ((long long)z * g.plane + (long long)y * g.pitch + x));
        sfor<0, L::Q>([&](auto I) {
          constexpr int i = LBM_CI(I);
          Store<S>::st(reinterpret_cast<S*>(o + off.dst[i]), q[i]);
        });
      }
    });
  }
}

// Blocks of the staged kernel resident per SM, times the SM count (per device, taken once).
template <class L, int COLL, class Real, class S>
inline int staged_grid(int* out) {
  static int dev_cached = -1, grid_cached = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return (int)e;
  if (dev != dev_cached) {
    auto k = k_step3_staged<L, COLL, Real, S>;
    e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, Stage3<L, S>::SMEM);
    if (e != cudaSuccess) return (int)e;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, Stage3<L, S>::THREADS, Stage3<L, S>::SMEM);
    if (e != cudaSuccess) return (int)e;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return (int)e;
    if (per_sm < 1) return (int)cudaErrorInvalidConfiguration;
    grid_cached = per_sm * sms;
    dev_cached = dev;
  }
  *out = grid_cached;
  return 0;
}

template <class L, int COLL, class Real, class S>
inline cudaError_t launch_step3_t(const void* fin, void* fout, const Geom3& g, const CollParamsD& pd,
                                  cudaStream_t st) {
  PullOffsets3<L::Q> off;
  for (int i = 0; i < L::Q; ++i) {
    off.cy[i] = L::CY[i];
    off.cz[i] = L::CZ[i];
    off.dst[i] = (long long)i * g.pstride * (long long)sizeof(S);
    off.src[i] = off.dst[i] -
                 ((long long)L::CZ[i] * g.plane + (long long)L::CY[i] * g.pitch + L::CX[i]) * (long long)sizeof(S);
  }
  if constexpr (Stage3<L, S>::ENABLED) {  // (not instantiated at all where disabled: D3Q103)
    if (g.bc[0] == BC_PERIODIC && g.nx % Stage3<L, S>::UNIT == 0 && g.nx >= Stage3<L, S>::PAD &&
        g.status != nullptr) {
      const int nbt = (g.nx + Stage3<L, S>::BXT - 1) / Stage3<L, S>::BXT;
      const long long ntiles = (long long)nbt * g.ny * g.nz;
      int grid = 0;
      const int e = staged_grid<L, COLL, Real, S>(&grid);
      if (e) return (cudaError_t)e;
      const long long nb = ntiles < grid ? ntiles : grid;
      k_step3_staged<L, COLL, Real, S><<<(unsigned)nb, Stage3<L, S>::THREADS, Stage3<L, S>::SMEM, st>>>(
          (const S*)fin, (S*)fout, g, nbt, ntiles, cast_params<Real>(pd), off);
      return cudaGetLastError();
    }
  }
  const int nbx = (g.nx + STEP_BX - 1) / STEP_BX;
  const Rows3 rows = rows3<L::VMAX>(g);
  const CollParams<Real> P = cast_params<Real>(pd);
  // D3Q103 RR with FP32 arithmetic on x-periodic grids of even nx: the two-cell kernel for every row
  bool pairs = false;
  if constexpr (Step3Pair<L, S>::ENABLED && COLL == COLL_RR && sizeof(Real) == 4)
    pairs = g.bc[0] == BC_PERIODIC && g.nx % 2 == 0 && g.nx >= L::VMAX;
  const int nbx2 = (g.nx + 2 * STEP_BX - 1) / (2 * STEP_BX);
  if (rows.interior == 0) {
    const long long nb = (long long)(pairs ? nbx2 : nbx) * g.ny * g.nz;
    if (nb > 0x7fffffffLL) return cudaErrorInvalidValue;
    if (pairs) {
      if constexpr (Step3Pair<L, S>::ENABLED && COLL == COLL_RR && sizeof(Real) == 4)
        k_step3_pair<L, S, ROWS_ALL><<<(unsigned)nb, STEP_BX, 0, st>>>((const S*)fin, (S*)fout, g, nbx2, rows,
                                                                      cast_params<F2>(pd), off);
    } else {
      k_step3<L, COLL, Real, S, ROWS_ALL><<<(unsigned)nb, STEP_BX, 0, st>>>((const S*)fin, (S*)fout, g, nbx, rows,
                                                                          P, off);
    }
    return cudaGetLastError();
  }
  const int nbr = pairs ? nbx2 : nbx;
  const long long nb_in = (long long)nbr * rows.interior, nb_edge = (long long)nbr * rows.edge;
  if (nb_in > 0x7fffffffLL || nb_edge > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (pairs) {
    if constexpr (Step3Pair<L, S>::ENABLED && COLL == COLL_RR && sizeof(Real) == 4) {
      const CollParams<F2> P2 = cast_params<F2>(pd);
      k_step3_pair<L, S, ROWS_INTERIOR><<<(unsigned)nb_in, STEP_BX, 0, st>>>((const S*)fin, (S*)fout, g, nbx2,
                                                                            rows, P2, off);
      k_step3_pair<L, S, ROWS_EDGE><<<(unsigned)nb_edge, STEP_BX, 0, st>>>((const S*)fin, (S*)fout, g, nbx2, rows,
                                                                          P2, off);
    }
  } else {
    k_step3<L, COLL, Real, S, ROWS_INTERIOR><<<(unsigned)nb_in, STEP_BX, 0, st>>>((const S*)fin, (S*)fout, g, nbx,
                                                                                  rows, P, off);
    k_step3<L, COLL, Real, S, ROWS_EDGE><<<(unsigned)nb_edge, STEP_BX, 0, st>>>((const S*)fin, (S*)fout, g, nbx,
                                                                              rows, P, off);
  }
  return cudaGetLastError();
}

template <class L, int COLL>
inline cudaError_t launch_step3_prec_wide(int prec, const void* fin, void* fout, const Geom3& g,
                                          const CollParamsD& pd, cudaStream_t st) {
  switch (prec) {
    case PREC_F64: return launch_step3_t<L, COLL, double, double>(fin, fout, g, pd, st);
    case PREC_F32: return launch_step3_t<L, COLL, float, float>(fin, fout, g, pd, st);
  }
  return cudaErrorInvalidValue;
}

template <class L, int COLL>
inline cudaError_t launch_step3_prec_16(int prec, const void* fin, void* fout, const Geom3& g, const CollParamsD& pd,
                                        cudaStream_t st) {
  switch (prec) {
    case PREC_F16: return launch_step3_t<L, COLL, float, __half>(fin, fout, g, pd, st);
    case PREC_BF16: return launch_step3_t<L, COLL, float, __nv_bfloat16>(fin, fout, g, pd, st);
    case PREC_I16: return launch_step3_t<L, COLL, float, short>(fin, fout, g, pd, st);
  }
  return cudaErrorInvalidValue;
}

template <class L, int COLL>
inline cudaError_t launch_step3_prec(int prec, const void* fin, void* fout, const Geom3& g, const CollParamsD& pd,
                                     cudaStream_t st) {
  if (prec == PREC_F64 || prec == PREC_F32) return launch_step3_prec_wide<L, COLL>(prec, fin, fout, g, pd, st);
  return launch_step3_prec_16<L, COLL>(prec, fin, fout, g, pd, st);
}

// Step launchers of one (lattice, collision) pair: one translation unit each, so that the 3D kernels
// compile in parallel (d3_<lattice>_<collision>.cu).
#define LBM3_STEP_SIG(name) \
  cudaError_t name(int prec, const void* fin, void* fout, const lbm::Geom3& g, const lbm::CollParamsD& pd, \
                   cudaStream_t st)

// ---------------------------------------------------------------------------
// Field kernels (double precision; not on the time-stepping path).  Fields are dense [nz][ny][nx].
// ---------------------------------------------------------------------------
constexpr int FB3 = 128;

template <class L, class S, int i>
__device__ __forceinline__ double decode3(const S* f, long long off, double rho0, double inv_s) {
  const double q = (double)Store<S>::ld(f + off);
  [[maybe_unused]] constexpr double w = L::W[i];
  if constexpr (Store<S>::SHIFTED)
    return w * (rho0 + q * inv_s);
  else
    return q;
}

struct Init3Params {
  int neq;
  double tau, rho0, s;
};

// f = f^(0) + f^(1) (Sec. III.B): f^(1) from the Chapman-Enskog a1^(2) = -tau rho cs^2 (d_a u_b + d_b u_a)
// of the velocity gradients grad[a][b] = d u_a / d x_b ([9][cells], may be null) and its recursion to
// every order of the lattice.
template <class L, class S>
__global__ void __launch_bounds__(FB3) k_init3(const double* __restrict__ rho, const double* __restrict__ u,
                                               const double* __restrict__ grad, S* __restrict__ f, Geom3 g,
                                               Init3Params ip) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  const long long c = (long long)blockIdx.x * FB3 + threadIdx.x;
  if (c >= n) return;
  const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((long long)g.nx * g.ny));
  constexpr double c2 = L::CS2;
  const double r = rho[c];
  const double uu[3] = {u[c], u[n + c], u[2 * n + c]};
  double pw[3][5];
  for (int d = 0; d < 3; ++d) {
    pw[d][0] = 1.0;
    for (int k = 1; k < 5; ++k) pw[d][k] = pw[d][k - 1] * uu[d];
  }
  double b2[6] = {0, 0, 0, 0, 0, 0};
  if (grad) {
    const double pre = -ip.tau * r * c2;
    auto gr = [&](int a, int b) { return grad[(long long)(3 * a + b) * n + c]; };
    b2[0] = pre * 2.0 * gr(0, 0);
    b2[1] = pre * 2.0 * gr(1, 1);
    b2[2] = pre * 2.0 * gr(2, 2);
    b2[3] = pre * (gr(0, 1) + gr(1, 0));
    b2[4] = pre * (gr(0, 2) + gr(2, 0));
    b2[5] = pre * (gr(1, 2) + gr(2, 1));
  }
  double C[5][5][5];
  sfor<0, 5>([&](auto Aa) {
    constexpr int a = LBM_CI(Aa);
    sfor<0, 5>([&](auto Bb) {
      constexpr int b = LBM_CI(Bb);
      sfor<0, 5>([&](auto Cc) {
        constexpr int cc = LBM_CI(Cc);
        constexpr int nn = a + b + cc;
        if constexpr (nn <= L::NMAX && L::keep(a, b, cc)) {
          constexpr double sc = 1.0 / (factorial(a) * factorial(b) * factorial(cc) * ipow(c2, nn));
          double v = (nn <= ip.neq) ? r * pw[0][a] * pw[1][b] * pw[2][cc] : 0.0;
          if constexpr (nn >= 2) {
            double a1 = 0.0;
            if constexpr (a >= 2) a1 += choose2(a) * b2[0] * pw[0][a - 2] * pw[1][b] * pw[2][cc];
            if constexpr (b >= 2) a1 += choose2(b) * b2[1] * pw[0][a] * pw[1][b - 2] * pw[2][cc];
            if constexpr (cc >= 2) a1 += choose2(cc) * b2[2] * pw[0][a] * pw[1][b] * pw[2][cc - 2];
            if constexpr (a >= 1 && b >= 1) a1 += a * b * b2[3] * pw[0][a - 1] * pw[1][b - 1] * pw[2][cc];
            if constexpr (a >= 1 && cc >= 1) a1 += a * cc * b2[4] * pw[0][a - 1] * pw[1][b] * pw[2][cc - 1];
            if constexpr (b >= 1 && cc >= 1) a1 += b * cc * b2[5] * pw[0][a] * pw[1][b - 1] * pw[2][cc - 1];
            v += a1;
          }
          C[a][b][cc] = v * sc;
        }
      });
    });
  });
  const long long o = (long long)z * g.plane + (long long)y * g.pitch + x;
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    double acc = 0.0;
    sfor<0, 5>([&](auto Aa) {
      constexpr int a = LBM_CI(Aa);
      sfor<0, 5>([&](auto Bb) {
        constexpr int b = LBM_CI(Bb);
        sfor<0, 5>([&](auto Cc) {
          constexpr int cc = LBM_CI(Cc);
          if constexpr (a + b + cc <= L::NMAX && L::keep(a, b, cc)) {
            constexpr double h = he(a, L::CX[i], c2) * he(b, L::CY[i], c2) * he(cc, L::CZ[i], c2);
            if constexpr (h != 0.0) acc += h * C[a][b][cc];
          }
        });
      });
    });
    // acc = f_i / w_i
    [[maybe_unused]] constexpr double w = L::W[i];
    double v;
    if constexpr (Store<S>::SHIFTED)
      v = ip.s * (acc - ip.rho0);
    else
      v = w * acc;
    Store<S>::st(f + (long long)i * g.pstride + o, v);
  });
}

// rho and u of the stored state (Sec. II.A); u is [3][cells].
template <class L, class S>
__global__ void __launch_bounds__(FB3) k_moments3(const S* __restrict__ f, Geom3 g, double rho0, double inv_s,
                                                  double* __restrict__ rho, double* __restrict__ u) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  const long long c = (long long)blockIdx.x * FB3 + threadIdx.x;
  if (c >= n) return;
  const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((long long)g.nx * g.ny));
  const long long o = (long long)z * g.plane + (long long)y * g.pitch + x;
  double r = 0, j[3] = {0, 0, 0};
  sfor<0, L::Q>([&](auto I) {
    constexpr int i = LBM_CI(I);
    constexpr double cx = L::CX[i], cy = L::CY[i], cz = L::CZ[i];
    const double fi = decode3<L, S, i>(f, (long long)i * g.pstride + o, rho0, inv_s);
    r += fi;
    j[0] += cx * fi;
    j[1] += cy * fi;
    j[2] += cz * fi;
  });
  if (rho) rho[c] = r;
  if (u) {
    u[c] = j[0] / r;
    u[n + c] = j[1] / r;
    u[2 * n + c] = j[2] / r;
  }
}

// Decoded population i (weight wi) of every cell to dense doubles, and the inverse.
template <class S>
__global__ void __launch_bounds__(FB3) k_get_plane3(const S* __restrict__ f, Geom3 g, int i, double wi,
                                                    double rho0, double inv_s, double* __restrict__ out) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  const long long c = (long long)blockIdx.x * FB3 + threadIdx.x;
  if (c >= n) return;
  const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((long long)g.nx * g.ny));
  const double q = (double)Store<S>::ld(f + (long long)i * g.pstride + (long long)z * g.plane +
                                        (long long)y * g.pitch + x);
  out[c] = Store<S>::SHIFTED ? wi * (rho0 + q * inv_s) : q;
}
template <class S>
__global__ void __launch_bounds__(FB3) k_set_plane3(S* __restrict__ f, Geom3 g, int i, double wi, double rho0,
                                                    double s, const double* __restrict__ in) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  const long long c = (long long)blockIdx.x * FB3 + threadIdx.x;
  if (c >= n) return;
  const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((long long)g.nx * g.ny));
  const double v = Store<S>::SHIFTED ? s * (in[c] / wi - rho0) : in[c];
  Store<S>::st(f + (long long)i * g.pstride + (long long)z * g.plane + (long long)y * g.pitch + x, v);
}

// FP64 mass and momentum: each block sums a fixed range of cells in a fixed order into partials[4][block];
// k_sum_partials3 then adds the partials in an order fixed by their count (deterministic, two passes).
template <class L, class S>
__global__ void __launch_bounds__(FB3) k_conservation3(const S* __restrict__ f, Geom3 g, double rho0, double inv_s,
                                                       long long per_block, double* __restrict__ partials) {
  const long long n = (long long)g.nx * g.ny * g.nz;
  const long long c0 = (long long)blockIdx.x * per_block;
  double acc[4] = {0, 0, 0, 0};
  for (long long c = c0 + threadIdx.x; c < c0 + per_block && c < n; c += FB3) {
    const int x = (int)(c % g.nx), y = (int)((c / g.nx) % g.ny), z = (int)(c / ((long long)g.nx * g.ny));
    const long long o = (long long)z * g.plane + (long long)y * g.pitch + x;
    sfor<0, L::Q>([&](auto I) {
      constexpr int i = LBM_CI(I);
      constexpr double cx = L::CX[i], cy = L::CY[i], cz = L::CZ[i];
      const double fi = decode3<L, S, i>(f, (long long)i * g.pstride + o, rho0, inv_s);
      acc[0] += fi;
      acc[1] += cx * fi;
      acc[2] += cy * fi;
      acc[3] += cz * fi;
    });
  }
  __shared__ double sh[4][FB3];
  for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  for (int w = FB3 / 2; w > 0; w >>= 1) {
    if ((int)threadIdx.x < w)
      for (int k = 0; k < 4; ++k) sh[k][threadIdx.x] += sh[k][threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0)
    for (int k = 0; k < 4; ++k) partials[(long long)k * gridDim.x + blockIdx.x] = sh[k][0];
}
// Second pass: one block of SUM3_T threads, thread t adding the partials t, t + SUM3_T, ... of each component
// (coalesced), then a shuffle tree and the warps in order; the addition order depends on nblocks alone.
constexpr int SUM3_T = 256;
template <int K>
__global__ void __launch_bounds__(SUM3_T) k_sum_partials3(const double* __restrict__ partials, int nblocks,
                                                         double* __restrict__ out) {
  __shared__ double sh[SUM3_T / 32][K];
  const int t = threadIdx.x, lane = t & 31, wid = t >> 5;
  double a[K];
#pragma unroll
  for (int k = 0; k < K; ++k) a[k] = 0.0;
  for (int b = t; b < nblocks; b += SUM3_T)
#pragma unroll
    for (int k = 0; k < K; ++k) a[k] += partials[(long long)k * nblocks + b];
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a[k] += __shfl_down_sync(0xffffffffu, a[k], o);
    if (lane == 0) sh[wid][k] = a[k];
  }
  __syncthreads();
  if (t < K) {
    double r = 0.0;
    for (int w = 0; w < SUM3_T / 32; ++w) r += sh[w][t];
    out[t] = r;
  }
}

// ---------------------------------------------------------------------------
// Launchers of one lattice, dispatched on the storage format; the field translation unit of each lattice
// exports them as a Lat3Ops table (api3.cu selects by lattice id).
// ---------------------------------------------------------------------------
struct Lat3Ops {
  cudaError_t (*step)(int coll, int prec, const void* fin, void* fout, const Geom3& g, const CollParamsD& pd,
                      cudaStream_t st);
  cudaError_t (*init)(int prec, const double* rho, const double* u, const double* grad, void* f, const Geom3& g,
                      const Init3Params& ip, cudaStream_t st);
  cudaError_t (*moments)(int prec, const void* f, const Geom3& g, double rho0, double inv_s, double* rho,
                         double* u, cudaStream_t st);
  cudaError_t (*get_plane)(int prec, const void* f, const Geom3& g, int i, double rho0, double inv_s, double* out,
                           cudaStream_t st);
  cudaError_t (*set_plane)(int prec, void* f, const Geom3& g, int i, double rho0, double s, const double* in,
                           cudaStream_t st);
  cudaError_t (*conservation)(int prec, const void* f, const Geom3& g, double rho0, double inv_s, double* partials,
                              int nblocks, double* out4, cudaStream_t st);
  int V;
  const int *cx, *cy, *cz;
  const double* w;
  double cs2;
  int nmax, vmax;
  int sixteen_bit;  // 16-bit storage formats built
};

template <class L, class F>
inline cudaError_t with_storage(int prec, F&& f) {
  switch (prec) {
    case PREC_F64: return f(double{});
    case PREC_F32: return f(float{});
  }
  if constexpr (Storages3<L>::SIXTEEN_BIT) {
    switch (prec) {
      case PREC_F16: return f(__half{});
      case PREC_BF16: return f(__nv_bfloat16{});
      case PREC_I16: return f(short{});
    }
  }
  return cudaErrorInvalidValue;
}

inline unsigned blocks3(const Geom3& g) {
  return (unsigned)(((long long)g.nx * g.ny * g.nz + FB3 - 1) / FB3);
}

// Field launchers of a lattice; `step` comes from the three per-collision translation units.
template <class L>
struct Ops3 {
  static cudaError_t init(int prec, const double* rho, const double* u, const double* grad, void* f,
                          const Geom3& g, const Init3Params& ip, cudaStream_t st) {
    return with_storage<L>(prec, [&](auto tag) {
      using S = decltype(tag);
      k_init3<L, S><<<blocks3(g), FB3, 0, st>>>(rho, u, grad, (S*)f, g, ip);
      return cudaGetLastError();
    });
  }
  static cudaError_t moments(int prec, const void* f, const Geom3& g, double rho0, double inv_s, double* rho,
                             double* u, cudaStream_t st) {
    return with_storage<L>(prec, [&](auto tag) {
      using S = decltype(tag);
      k_moments3<L, S><<<blocks3(g), FB3, 0, st>>>((const S*)f, g, rho0, inv_s, rho, u);
      return cudaGetLastError();
    });
  }
  static cudaError_t get_plane(int prec, const void* f, const Geom3& g, int i, double rho0, double inv_s,
                               double* out, cudaStream_t st) {
    return with_storage<L>(prec, [&](auto tag) {
      using S = decltype(tag);
      k_get_plane3<S><<<blocks3(g), FB3, 0, st>>>((const S*)f, g, i, L::W[i], rho0, inv_s, out);
      return cudaGetLastError();
    });
  }
  static cudaError_t set_plane(int prec, void* f, const Geom3& g, int i, double rho0, double s, const double* in,
                               cudaStream_t st) {
    return with_storage<L>(prec, [&](auto tag) {
      using S = decltype(tag);
      k_set_plane3<S><<<blocks3(g), FB3, 0, st>>>((S*)f, g, i, L::W[i], rho0, s, in);
      return cudaGetLastError();
    });
  }
  static cudaError_t conservation(int prec, const void* f, const Geom3& g, double rho0, double inv_s,
                                  double* partials, int nblocks, double* out4, cudaStream_t st) {
    const long long n = (long long)g.nx * g.ny * g.nz;
    const long long per_block = (n + nblocks - 1) / nblocks;
    return with_storage<L>(prec, [&](auto tag) {
      using S = decltype(tag);
      k_conservation3<L, S><<<nblocks, FB3, 0, st>>>((const S*)f, g, rho0, inv_s, per_block, partials);
      k_sum_partials3<4><<<1, SUM3_T, 0, st>>>(partials, nblocks, out4);
      return cudaGetLastError();
    });
  }
  static Lat3Ops table(decltype(Lat3Ops::step) step) {
    return Lat3Ops{step, init, moments, get_plane, set_plane, conservation, L::Q, L::CX, L::CY, L::CZ, L::W,
                   L::CS2, L::NMAX, L::VMAX, Storages3<L>::SIXTEEN_BIT ? 1 : 0};
  }
};

}  // namespace lbm
