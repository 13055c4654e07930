// Batched stream-and-collide: many independent grids (D2Q9, D2V17 and
// isothermal D2V37, uneven sizes and relaxation times) advanced by one kernel
// launch per time step, the launches captured in a CUDA graph (one kernel node
// per step).
//
// Work item = `rows` consecutive rows x (cells per thread * threads) columns of
// one instance (two cells per thread on D2Q9 / D2V17, one on D2V37, as the
// single-grid kernels); the items of all instances are numbered consecutively,
// those of the lattices with the most work per cell first (D2V37, D2V17,
// D2Q9), and either one block per item or a persistent grid of (SMs x blocks
// per SM) blocks walks them.  The instance table travels as a kernel parameter
// (constant bank); each item finds its instance by a binary search over the
// first-item offsets and takes that instance's lattice (a block-uniform
// branch).  Per cell the arithmetic is the single-grid kernels' (step2_cells,
// step_cell), so a batched step is bitwise identical to per-instance lbm_step
// calls.  A batch holding D2V37 runs 128-thread blocks at the D2V37 kernel's
// register cap (72, seven blocks a SM).
//
// The launch shape (threads per block, rows per item, blocks per SM) is chosen
// by lbm_batch_autotune, which times every candidate on the batch itself.
#include <cuda_runtime.h>

#include <cstdio>
#include <new>
#include <vector>

#include "../../include/lbm.h"
#include "ctx.h"
#include "step.cuh"

namespace lbm {

constexpr int kBatchMax = LBM_BATCH_MAX;

struct BatchInst {
  const void* fin;
  void* fout;
  StepGeom g;
  union {
    CollParams<F2> P;      // D2Q9 / D2V17: two cells a thread
    CollParams<float> Pf;  // D2V37: one cell a thread, read in place from the constant bank
  };
  int ntx;         // items per row band
  int lattice;     // LBM_D2Q9, LBM_D2V17 or LBM_D2V37
  long long item0; // first work item of the instance
};

struct BatchDesc {
  int n;
  int rows;         // rows per work item
  long long total;  // work items of all instances
  BatchInst inst[kBatchMax];
};
static_assert(sizeof(BatchDesc) <= 32764, "the instance table travels as one kernel parameter");

// The rows of one work item of instance I on lattice L.
template <class L, int COLL, class S>
__device__ __forceinline__ void batch_item(const BatchInst& I, int rows, int band, int x, int xw) {
  const S* fin = static_cast<const S*>(I.fin);
  S* fout = static_cast<S*>(I.fout);
  const GeomOffsets<L, S> off{I.g.plane * (long long)sizeof(S), (long long)I.g.pitch * (long long)sizeof(S)};
  for (int r = 0; r < rows; ++r) {
    const int y = band * rows + r;
    if (y >= I.g.ny) break;
    step2_cells<L, COLL, S, GeomOffsets<L, S>, true>(fin, fout, I.g, I.P, off, x, y, xw);
  }
}

// The rows of one work item of a D2V37 instance, one cell per thread.
template <int COLL, class S>
__device__ __forceinline__ void batch_item_v37(const BatchInst& I, int rows, int band, int x) {
  const S* fin = static_cast<const S*>(I.fin);
  S* fout = static_cast<S*>(I.fout);
  const GeomOffsets<D2V37, S> off{I.g.plane * (long long)sizeof(S), (long long)I.g.pitch * (long long)sizeof(S)};
  for (int r = 0; r < rows; ++r) {
    const int y = band * rows + r;
    if (y >= I.g.ny) break;
    step_cell<D2V37, COLL, false, float, S, false>(fin, fout, I.g, I.Pf, off, nullptr, x, y);
  }
}

// V37: the batch holds D2V37 instances (128-thread blocks, the register cap of the D2V37 kernel).
template <int COLL, class S, bool V37>
__global__ void __launch_bounds__(V37 ? 128 : 256, V37 ? 7 : 1) k_batch(const __grid_constant__ BatchDesc d) {
  for (long long it = blockIdx.x; it < d.total; it += gridDim.x) {
    int lo = 0, hi = d.n - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (d.inst[mid].item0 <= it) lo = mid; else hi = mid - 1;
    }
    const BatchInst& I = d.inst[lo];
    const long long local = it - I.item0;
    const int band = (int)(local / I.ntx);
    const int tx = (int)(local - (long long)band * I.ntx);
    if constexpr (V37) {
      if (I.lattice == LBM_D2V37) {
        const int x = tx * (int)blockDim.x + (int)threadIdx.x;
        if (x < I.g.nx) batch_item_v37<COLL, S>(I, d.rows, band, x);
        continue;
      }
    }
    const int x = 2 * (tx * (int)blockDim.x + (int)threadIdx.x);
    const int xw = 2 * (tx * (int)blockDim.x + (int)(threadIdx.x & ~31u));
    if (x >= I.g.nx) continue;
    if (I.lattice == LBM_D2V17)
      batch_item<D2V17, COLL, S>(I, d.rows, band, x, xw);
    else
      batch_item<D2Q9, COLL, S>(I, d.rows, band, x, xw);
  }
}

// blocks_per_sm == 0: one block per work item; > 0: persistent grid of blocks_per_sm x SMs blocks.
template <int COLL, class S>
cudaError_t batch_launch_t(const BatchDesc& d, int threads, int blocks_per_sm, int nsm, cudaStream_t st) {
  if (d.n == 0 || d.total == 0) return cudaSuccess;
  long long grid = blocks_per_sm > 0 ? (long long)blocks_per_sm * nsm : d.total;
  if (grid > d.total) grid = d.total;
  if (grid > 0x7fffffffLL) grid = 0x7fffffffLL;
  bool v37 = false;
  for (int k = 0; k < d.n; ++k) v37 = v37 || d.inst[k].lattice == LBM_D2V37;
  if (v37) {
    if (threads != 128) return cudaErrorInvalidValue;
    k_batch<COLL, S, true><<<(unsigned)grid, threads, 0, st>>>(d);
  } else {
    k_batch<COLL, S, false><<<(unsigned)grid, threads, 0, st>>>(d);
  }
  return cudaGetLastError();
}

template <class S>
cudaError_t batch_launch_s(int coll, const BatchDesc& d, int threads, int bps, int nsm, cudaStream_t st) {
  switch (coll) {
    case COLL_BGK: return batch_launch_t<COLL_BGK, S>(d, threads, bps, nsm, st);
    case COLL_PR: return batch_launch_t<COLL_PR, S>(d, threads, bps, nsm, st);
    case COLL_RR: return batch_launch_t<COLL_RR, S>(d, threads, bps, nsm, st);
  }
  return cudaErrorInvalidValue;
}

cudaError_t batch_launch(int coll, int prec, const BatchDesc& d, int threads, int bps, int nsm, cudaStream_t st) {
  switch (prec) {
    case PREC_F32: return batch_launch_s<float>(coll, d, threads, bps, nsm, st);
    case PREC_F16: return batch_launch_s<__half>(coll, d, threads, bps, nsm, st);
    case PREC_BF16: return batch_launch_s<__nv_bfloat16>(coll, d, threads, bps, nsm, st);
    case PREC_I16: return batch_launch_s<short>(coll, d, threads, bps, nsm, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbm

using namespace lbm;

struct lbm_batch {
  int n = 0;
  lbm_ctx* ctx[kBatchMax] = {nullptr};
  int coll = 0, prec = 0;
  int threads = 128, rows = 1, blocks_per_sm = 0;  // launch shape (0 = as many as fit)
  bool v37 = false;                                 // holds D2V37 instances: 128-thread blocks only
  cudaStream_t st = nullptr;       // the instances' stream
  cudaStream_t capture = nullptr;  // private stream used to record the graph
  cudaGraphExec_t graph[2] = {nullptr, nullptr};  // two steps, from parity 0 / 1 of the first instance
  int nsm = 1;
  int device = 0;
};

namespace {

// Launch descriptor of every instance, each reading buffer cur ^ flip: the items of D2V37, then D2V17,
// then D2Q9 instances.
BatchDesc make_desc(const lbm_batch* b, int flip) {
  BatchDesc d{};
  d.n = 0;
  d.rows = b->rows;
  long long item = 0;
  for (int lattice : {LBM_D2V37, LBM_D2V17, LBM_D2Q9})
    for (int k = 0; k < b->n; ++k) {
      const lbm_ctx* c = b->ctx[k];
      if (c->p.lattice != lattice) continue;
      BatchInst& I = d.inst[d.n++];
      const int cur = c->cur ^ flip;
      I.fin = c->buf[cur];
      I.fout = c->buf[cur ^ 1];
      I.g = c->g;
      const CollParamsD pd = lbm_ctx_coll_params(c);
      const double s_store = c->prec >= PREC_F16 ? pd.s : 1.0;  // the shifted 16-bit formats
      if (lattice == LBM_D2V37) {
        I.Pf = cast_params<float>(pd);
        set_coef_factors<D2V37>(I.Pf, c->p.collision, pd.neq, pd.nreg, pd.omega, pd.om1, pd.om1_3, pd.om1_4, s_store);
      } else {
        I.P = cast_params<F2>(pd);
        if (lattice == LBM_D2V17)
          set_coef_factors<D2V17>(I.P, c->p.collision, pd.neq, pd.nreg, pd.omega, pd.om1, pd.om1_3, pd.om1_4, s_store);
        else
          set_coef_factors<D2Q9>(I.P, c->p.collision, pd.neq, pd.nreg, pd.omega, pd.om1, pd.om1_3, pd.om1_4, s_store);
      }
      const int cells = lattice == LBM_D2V37 ? b->threads : 2 * b->threads;  // columns of an item
      I.ntx = (c->p.nx + cells - 1) / cells;
      I.lattice = lattice;
      I.item0 = item;
      item += (long long)I.ntx * ((c->p.ny + b->rows - 1) / b->rows);
    }
  d.total = item;
  return d;
}

// One batched time step: one launch over the instances of both lattices.
cudaError_t batch_step_launch(const lbm_batch* b, int flip, cudaStream_t st) {
  return batch_launch(b->coll, b->prec, make_desc(b, flip), b->threads, b->blocks_per_sm, b->nsm, st);
}

void drop_graphs(lbm_batch* b) {
  for (int k = 0; k < 2; ++k)
    if (b->graph[k]) {
      cudaGraphExecDestroy(b->graph[k]);
      b->graph[k] = nullptr;
    }
}

// Two consecutive steps from the instances' current buffers, recorded on the private stream.
cudaError_t build_graph(lbm_batch* b, cudaGraphExec_t* exec) {
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(b->capture, cudaStreamCaptureModeThreadLocal);
  if (e != cudaSuccess) return e;
  for (int s = 0; s < 2 && e == cudaSuccess; ++s)
    e = batch_step_launch(b, s, b->capture);
  cudaError_t e2 = cudaStreamEndCapture(b->capture, &g);
  if (e == cudaSuccess) e = e2;
  if (e == cudaSuccess) e = cudaGraphInstantiate(exec, g, 0);
  if (g) cudaGraphDestroy(g);
  return e;
}

void advance(lbm_batch* b, int n) {
  for (int k = 0; k < b->n; ++k) {
    b->ctx[k]->cur ^= (n & 1);
    b->ctx[k]->steps += n;
  }
}

}  // namespace

extern "C" {

int lbm_batch_create(const lbm_params* ps, int n, lbm_batch** out) {
  if (!out) return LBM_EINVAL;
  *out = nullptr;
  if (!ps || n < 1 || n > kBatchMax) return LBM_EINVAL;
  for (int k = 0; k < n; ++k) {
    const lbm_params& p = ps[k];
    if (p.lattice != LBM_D2Q9 && p.lattice != LBM_D2V17 && p.lattice != LBM_D2V37) return LBM_EINVAL;
    if (p.thermal || p.compute != LBM_F32 || p.storage == LBM_F64) return LBM_EINVAL;
    if (p.a1_source != LBM_A1_PROJECTION) return LBM_EINVAL;  // the batched kernel projects a1
    if (p.collision != ps[0].collision || p.storage != ps[0].storage || p.stream != ps[0].stream) return LBM_EINVAL;
  }
  lbm_batch* b = new (std::nothrow) lbm_batch();
  if (!b) return LBM_ENOMEM;
  for (int k = 0; k < n; ++k) {
    const int rc = lbm_create(&ps[k], &b->ctx[k]);
    if (rc != LBM_OK) {
      b->n = k;
      lbm_batch_destroy(b);
      return rc;
    }
  }
  b->n = n;
  for (int k = 0; k < n; ++k) b->v37 = b->v37 || ps[k].lattice == LBM_D2V37;
  b->coll = ps[0].collision;
  b->prec = b->ctx[0]->prec;
  b->st = static_cast<cudaStream_t>(ps[0].stream);
  b->device = b->ctx[0]->device;
  b->nsm = b->ctx[0]->g.nsm;
  if (cudaStreamCreateWithFlags(&b->capture, cudaStreamNonBlocking) != cudaSuccess) {
    lbm_batch_destroy(b);
    return LBM_ECUDA;
  }
  *out = b;
  return LBM_OK;
}

void lbm_batch_destroy(lbm_batch* b) {
  if (!b) return;
  cudaSetDevice(b->device);
  drop_graphs(b);
  if (b->capture) cudaStreamDestroy(b->capture);
  for (int k = 0; k < b->n; ++k) lbm_destroy(b->ctx[k]);
  delete b;
}

lbm_ctx* lbm_batch_context(lbm_batch* b, int i) {
  if (!b || i < 0 || i >= b->n) return nullptr;
  return b->ctx[i];
}

int lbm_batch_step(lbm_batch* b, int n) {
  if (!b || n < 0) return LBM_EINVAL;
  if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ECUDA;
  // every instance must sit on the same buffer parity (it does unless one was stepped on its own)
  const int par = b->ctx[0]->cur;
  for (int k = 1; k < b->n; ++k)
    if (b->ctx[k]->cur != par) return LBM_EINVAL;
  int done = 0;
  if (n >= 2) {
    // one graph per buffer parity (all instances move together); each replay is two steps
    if (!b->graph[par] && build_graph(b, &b->graph[par]) != cudaSuccess) return LBM_ECUDA;
    for (; done + 2 <= n; done += 2)
      if (cudaGraphLaunch(b->graph[par], b->st) != cudaSuccess) return LBM_ECUDA;
  }
  if (done < n) {
    if (batch_step_launch(b, 0, b->st) != cudaSuccess) return LBM_ECUDA;
  }
  advance(b, n);
  return LBM_OK;
}

int lbm_batch_set_launch(lbm_batch* b, int threads, int rows, int blocks_per_sm) {
  if (!b || (threads != 64 && threads != 128 && threads != 256) || rows < 1 || rows > 64 || blocks_per_sm < 0)
    return LBM_EINVAL;
  if (b->v37 && threads != 128) return LBM_EINVAL;
  b->threads = threads;
  b->rows = rows;
  b->blocks_per_sm = blocks_per_sm;
  drop_graphs(b);
  return LBM_OK;
}

int lbm_batch_get_launch(const lbm_batch* b, int* threads, int* rows, int* blocks_per_sm) {
  if (!b) return LBM_EINVAL;
  if (threads) *threads = b->threads;
  if (rows) *rows = b->rows;
  if (blocks_per_sm) *blocks_per_sm = b->blocks_per_sm;
  return LBM_OK;
}

int lbm_batch_autotune(lbm_batch* b, int steps, double* best_ms) {
  if (!b || steps < 1) return LBM_EINVAL;
  if (cudaSetDevice(b->device) != cudaSuccess) return LBM_ECUDA;
  const int threads_c[] = {64, 128, 256};
  const int rows_c[] = {1, 2, 4, 8};
  const int bps_c[] = {0, 2, 4, 8};
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return LBM_ECUDA;
  float best = 1e30f;
  int bt = b->threads, br = b->rows, bb = b->blocks_per_sm;
  int rc = LBM_OK;
  for (int t : threads_c)
    for (int r : rows_c)
      if (!b->v37 || t == 128)
      for (int q : bps_c) {
        b->threads = t;
        b->rows = r;
        b->blocks_per_sm = q;
        // warm-up step, then `steps` timed steps (each one advances the instances)
        bool ok = true;
        for (int s = 0; s <= steps && ok; ++s) {
          if (s == 1) ok = cudaEventRecord(e0, b->st) == cudaSuccess;
          ok = ok && batch_step_launch(b, 0, b->st) == cudaSuccess;
          if (ok) advance(b, 1);
        }
        ok = ok && cudaEventRecord(e1, b->st) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0;
        ok = ok && cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
        if (!ok) {
          rc = LBM_ECUDA;
          break;
        }
        ms /= steps;
        if (ms < best) {
          best = ms;
          bt = t;
          br = r;
          bb = q;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->threads = bt;
  b->rows = br;
  b->blocks_per_sm = bb;
  drop_graphs(b);
  if (best_ms) *best_ms = best;
  return rc;
}

}  // extern "C"
