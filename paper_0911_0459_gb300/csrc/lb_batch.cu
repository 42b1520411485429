// Host side of the batched capillary sweep (lb_batch_* in include/lb.h).
//
// lb_batch_create validates every lattice, lays the lattices out one after the
// other in one arena per buffer (offsets padded to 64 elements, zeroed), builds
// the flat tile list (capillary, column block, row band; all-solid tiles left
// out) and the reduction chunks, and sets each lattice's default initial state.
// A launch runs n steps of the persistent kernel of the chosen body (sliding
// window, staged shallow or deep ring, or the moment strips): the tiles are
// assigned to CTAs on the host, longest estimated cost first, so that every CTA
// carries about the same work each step.  lb_batch_run_sampled captures the
// launches between samples and the FP64 reductions at each sample into one CUDA
// graph.  The autotuner times every body and tile on the batch itself.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "lb.h"
#include "lb_batch.cuh"
#include "lb_ops.h"

using namespace lbk;

namespace {

thread_local char g_batch_create_err[512] = "";
constexpr unsigned long long kDefaultLimitNs = 2000000000ull;

}  // namespace

struct lb_batch {
  int n;
  int storage;
  std::vector<lb_grid> grids;
  std::vector<lb_walls> walls;
  std::vector<lb_params> params;
  std::vector<size_t> off_f, off_g, off_g0;
  std::vector<long> fluid;
  cudaStream_t stream;
  cudaStream_t cap;
  lb_alloc alloc;
  int have_alloc;
  void* f[2];
  void* g[2];
  float* g0[2];
  size_t bytes_f, bytes_g, bytes_g0;  // arena sizes
  void* d_caps;
  TileDesc* d_tiles;   // tiles in schedule order: CTA k takes d_tiles[start[k] .. start[k+1])
  int* d_start;
  int ntiles;
  RedChunk* d_chunks;  // reduction chunks of every lattice, lattice by lattice
  int2* d_range;       // per lattice: first chunk, number of chunks
  double* d_part;      // three partial sums per chunk
  int nchunks;
  GridBarrier* d_bar;
  int* d_err;
  double* d_out;
  size_t out_cap;  // doubles
  int parity;
  long t;
  int tile_x, tile_y;
  int kernel;      // 0 automatic, 1 sliding-window body, 2 staged body
  int deep;        // staged body: the deeper of its two rings
  int staged_ok;   // every lattice fits the staged body (nx % 8 == 0, 9 nx ny < 2^32)
  int grid_blocks;
  unsigned int extra_arrivals;
  unsigned long long limit_ns;
  int poisoned;
  int graph_fallbacks;
  char err[512];
  std::vector<void*> owned;
};

static void berr(lb_batch* b, const char* fmt, ...) {
  char* dst = b ? b->err : g_batch_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
}

#define BCK(call)                                                                              \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      berr(b, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__);     \
      return LB_ERR_CUDA;                                                                      \
    }                                                                                          \
  } while (0)

static void* balloc(lb_batch* b, size_t bytes) {
  void* p = NULL;
  if (b->have_alloc) {
    p = b->alloc.malloc_fn(bytes, (void*)b->stream, b->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = NULL;
  }
  if (p) b->owned.push_back(p);
  return p;
}

static void bfree_all(lb_batch* b) {
  for (void* p : b->owned) {
    if (b->have_alloc)
      b->alloc.free_fn(p, (void*)b->stream, b->alloc.user);
    else
      cudaFree(p);
  }
  b->owned.clear();
}

static size_t elem_size(int storage) {
  return storage == LB_STORAGE_F64 ? 8
       : ((storage == LB_STORAGE_F32 || storage == LB_STORAGE_MOMENTS || storage == LB_STORAGE_F32_BLOCKED) ? 4 : 2);
}

// Columns of a tile of tile_x threads (the moment kernel's warps produce 30).
static int tile_cols(const lb_batch* b) {
  return b->storage == LB_STORAGE_MOMENTS ? (b->tile_x / 32) * kMomCols : b->tile_x;
}

static int solid_h(const lb_grid& g, const lb_walls& w, int x, int y) {
  if (w.tube_len <= 0) return 0;
  int dx = ((x - w.tube_x0) % g.nx + g.nx) % g.nx;
  int dy = ((y - w.tube_y0) % g.ny + g.ny) % g.ny;
  return dx < w.tube_len && dy >= w.tube_h;
}

// Op arguments addressing lattice i of buffer k (for the per-lattice kernels).
static OpArgs lattice_args(const lb_batch* b, int i, int k) {
  OpArgs a;
  memset(&a, 0, sizeof a);
  const lb_grid& g = b->grids[i];
  const lb_walls& w = b->walls[i];
  const lb_params& p = b->params[i];
  a.nx = g.nx; a.ny = g.ny;
  a.tube_x0 = w.tube_x0; a.tube_len = w.tube_len; a.tube_y0 = w.tube_y0; a.tube_h = w.tube_h;
  a.kappa = p.kappa; a.a = p.a; a.b = p.b; a.T = p.T; a.Acoef = p.A; a.M = p.M;
  a.nu_l = p.nu_l; a.nu_g = p.nu_g; a.nu = p.nu; a.lambda_scale = p.lambda_scale; a.h = w.wall_grad;
  a.lut = p.nu_table >= 2 ? p.nu_table - 1 : 0;
  a.rho_l = p.rho_l; a.rho_g = p.rho_g;
  const size_t el = elem_size(b->storage);
  OpBufs ob;
  ob.f = (char*)b->f[k] + b->off_f[i] * el;
  ob.g = b->storage == LB_STORAGE_F32_BLOCKED ? (char*)ob.f + el  // g_i after f_i in every block
                                              : (b->g[k] ? (char*)b->g[k] + b->off_g[i] * el : NULL);
  ob.g0 = b->g0[k] ? b->g0[k] + b->off_g0[i] : NULL;
  if (b->storage == LB_STORAGE_F16_BLOCKED) {  // g_i after f_i, g_0 at byte 1088 of every block
    ob.g = (char*)ob.f + 2;
    ob.g0 = (float*)((char*)ob.f + 1088);
  }
  a.src = ob;
  a.dst = ob;
  return a;
}

static OpsFn batch_ops(int storage) {
  if (storage == LB_STORAGE_MOMENTS) return ops_bin_m32;
  if (storage == LB_STORAGE_F32_BLOCKED) return ops_bin_f32b;
  if (storage == LB_STORAGE_F16_BLOCKED) return ops_bin_f16b;
  return storage == LB_STORAGE_F64 ? ops_bin_f64 : (storage == LB_STORAGE_F32 ? ops_bin_f32 : ops_bin_f16);
}

static lb_status init_lattice(lb_batch* b, int i) {
  const lb_grid& g = b->grids[i];
  const lb_walls& w = b->walls[i];
  const lb_params& p = b->params[i];
  // the initial state as for lb_create: at rest, tanh profiles along x, one value per
  // column (the init kernel takes no input at solid nodes)
  const size_t N = (size_t)g.nx;
  std::vector<double> host(4 * N, 0.0);
  const double wdt = sqrt(2.0);
  const double xa = w.gas_cols, xb = (double)w.tube_x0 + p.l0;
  for (int x = 0; x < g.nx; ++x) {
    const double chi = 0.5 * (tanh((x - xa) / wdt) - tanh((x - xb) / wdt));
    host[x] = 1.0;
    host[3 * N + x] = 2.0 * chi - 1.0;
  }
  double* d = NULL;
  if (b->have_alloc)
    d = (double*)b->alloc.malloc_fn(4 * N * sizeof(double), (void*)b->stream, b->alloc.user);
  else if (cudaMalloc((void**)&d, 4 * N * sizeof(double)) != cudaSuccess)
    d = NULL;
  if (!d) return berr(b, "device allocation failed"), LB_ERR_NOMEM;
  cudaError_t e = cudaMemcpyAsync(d, host.data(), 4 * N * sizeof(double), cudaMemcpyHostToDevice, b->stream);
  OpArgs a = lattice_args(b, i, 0);
  a.in0 = d; a.in1 = d + N; a.in2 = d + 2 * N; a.in3 = d + 3 * N;
  a.in_cols = 1;
  if (e == cudaSuccess) e = batch_ops(b->storage)(OP_INIT, a, b->stream);
  cudaError_t e2 = cudaStreamSynchronize(b->stream);
  if (b->have_alloc)
    b->alloc.free_fn(d, (void*)b->stream, b->alloc.user);
  else
    cudaFree(d);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return berr(b, "init of lattice %d failed: %s", i, cudaGetErrorString(e)), LB_ERR_CUDA;
  return LB_OK;
}

// 1 or 2: the body the next launch uses
static int batch_variant(const lb_batch* b) {
  if (b->storage == LB_STORAGE_MOMENTS) return 4;
  if (b->kernel == 0) return b->staged_ok ? 2 : 1;
  return b->kernel;
}

template <class S>
static void fill_args(const lb_batch* b, int nsteps, BatchArgs<S>& a) {
  a.caps = (const CapDesc<typename S::A>*)b->d_caps;
  a.tiles = b->d_tiles;
  a.start = b->d_start;
  a.fa = (typename S::T*)b->f[0]; a.ga = (typename S::T*)b->g[0]; a.g0a = b->g0[0];
  a.fb = (typename S::T*)b->f[1]; a.gb = (typename S::T*)b->g[1]; a.g0b = b->g0[1];
  a.nsteps = nsteps;
  a.parity = b->parity;
  a.bar = b->d_bar;
  a.expected = (unsigned)b->grid_blocks + b->extra_arrivals;
  a.limit_ns = b->limit_ns;
  a.err = b->d_err;
}

// Either launches the current body over nsteps steps (per == NULL) or returns
// in *per how many of its CTAs are resident on one SM.
template <class S, int BX>
static cudaError_t run_sliding(lb_batch* b, int nsteps, cudaStream_t s, int* per) {
  if (per) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, batch_step_kernel<S, BX>, BX, 0);
  BatchArgs<S> a;
  fill_args(b, nsteps, a);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid_blocks);
  cfg.blockDim = dim3(BX);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_step_kernel<S, BX>, a);
}

template <class S, int BX, int NS>
static cudaError_t run_staged(lb_batch* b, int nsteps, cudaStream_t s, int* per) {
  using L = TmaLayout<MODEL_BINARY, S, BX, NS>;
  static bool configured = false;  // dynamic shared memory opt-in, once per process
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(batch_tma_kernel<S, BX, NS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  if (per) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, batch_tma_kernel<S, BX, NS>, BX + 32, L::BYTES);
  BatchArgs<S> a;
  fill_args(b, nsteps, a);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid_blocks);
  cfg.blockDim = dim3(BX + 32);
  cfg.dynamicSmemBytes = L::BYTES;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_tma_kernel<S, BX, NS>, a);
}

template <int NW>
static cudaError_t run_moment(lb_batch* b, int nsteps, cudaStream_t s, int* per) {
  if (per) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per, batch_moment_kernel<NW>, NW * 32, 0);
  BatchArgs<SM32> a;
  fill_args(b, nsteps, a);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(b->grid_blocks);
  cfg.blockDim = dim3(NW * 32);
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, batch_moment_kernel<NW>, a);
}

template <class S>
static cudaError_t run_s(lb_batch* b, int nsteps, cudaStream_t s, int* per) {
  if (batch_variant(b) == 2) {
    // ring depths as for the single-lattice staged kernel
    if (b->tile_x == 64) return b->deep ? run_staged<S, 64, 8>(b, nsteps, s, per) : run_staged<S, 64, 4>(b, nsteps, s, per);
    if (b->tile_x == 128) return b->deep ? run_staged<S, 128, 6>(b, nsteps, s, per) : run_staged<S, 128, 4>(b, nsteps, s, per);
    return b->deep ? run_staged<S, 256, 4>(b, nsteps, s, per) : run_staged<S, 256, 3>(b, nsteps, s, per);
  }
  if (b->tile_x == 64) return run_sliding<S, 64>(b, nsteps, s, per);
  if (b->tile_x == 128) return run_sliding<S, 128>(b, nsteps, s, per);
  return run_sliding<S, 256>(b, nsteps, s, per);
}

static cudaError_t run_batch(lb_batch* b, int nsteps, cudaStream_t s, int* per) {
  if (b->storage == LB_STORAGE_MOMENTS) {
    if (b->tile_x == 64) return run_moment<2>(b, nsteps, s, per);
    if (b->tile_x == 128) return run_moment<4>(b, nsteps, s, per);
    return run_moment<8>(b, nsteps, s, per);
  }
  if (b->storage == LB_STORAGE_F64) return run_s<SF64>(b, nsteps, s, per);
  if (b->storage == LB_STORAGE_F32) return run_s<SF32>(b, nsteps, s, per);
  if (b->storage == LB_STORAGE_F32_BLOCKED) return run_s<SF32B>(b, nsteps, s, per);
  if (b->storage == LB_STORAGE_F16_BLOCKED) return run_s<SF16B>(b, nsteps, s, per);
  return run_s<SF16>(b, nsteps, s, per);
}

static cudaError_t launch_batch(lb_batch* b, int nsteps, cudaStream_t s) { return run_batch(b, nsteps, s, NULL); }

static void free_owned(lb_batch* b, void* p) {
  if (!p) return;
  if (b->have_alloc)
    b->alloc.free_fn(p, (void*)b->stream, b->alloc.user);
  else
    cudaFree(p);
  b->owned.erase(std::remove(b->owned.begin(), b->owned.end(), p), b->owned.end());
}

// Tiles of every lattice for the current body and tile shape, and their
// schedule.  A CTA of the persistent kernel takes a fixed list of tiles every
// step and all CTAs meet at a grid barrier after it, so a step lasts as long as
// the longest list.  The lists are balanced by longest-processing-time-first on
// an estimated cost (every staged row costs its row sums across the tile's
// width, every fluid node its collision), then each list is put back in tile
// order so that CTAs working at the same time touch neighbouring rows.
static lb_status build_tiles(lb_batch* b) {
  std::vector<TileDesc> tiles;
  std::vector<double> cost;
  for (int i = 0; i < b->n; ++i) {
    const lb_grid& g = b->grids[i];
    const lb_walls& w = b->walls[i];
    // solid nodes are the tube's columns outside its band of rows: count them
    // from prefix sums of tube columns and of rows outside the band
    std::vector<long> tc(g.nx + 1, 0), ob(g.ny + 1, 0);
    for (int x = 0; x < g.nx; ++x) tc[x + 1] = tc[x] + solid_h(g, w, x, (w.tube_y0 + w.tube_h) % g.ny);
    for (int y = 0; y < g.ny; ++y) ob[y + 1] = ob[y] + solid_h(g, w, w.tube_x0, y);
    const int tw = tile_cols(b);
    for (int y0 = 0; y0 < g.ny; y0 += b->tile_y)
      for (int xb = 0; xb < g.nx; xb += tw) {
        const int y1 = std::min(y0 + b->tile_y, g.ny);
        const int x1 = std::min(xb + tw, g.nx);
        const long fluid = (long)(y1 - y0) * (x1 - xb) - (tc[x1] - tc[xb]) * (ob[y1] - ob[y0]);
        if (fluid) {
          tiles.push_back(TileDesc{i, xb, y0, y1});
          cost.push_back(0.3 * (y1 - y0 + 2) * tw + (double)fluid);
        }
      }
  }
  b->ntiles = (int)tiles.size();
  int dev = 0, sms = 0, per = 0;
  BCK(cudaGetDevice(&dev));
  BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  BCK(run_batch(b, 0, b->stream, &per));
  if (per < 1) return berr(b, "the persistent kernel does not fit on an SM"), LB_ERR_CUDA;
  const int blocks = std::max(1, std::min(per * sms, b->ntiles));
  // longest processing time first onto the least loaded CTA
  std::vector<int> order(tiles.size());
  for (size_t k = 0; k < order.size(); ++k) order[k] = (int)k;
  std::stable_sort(order.begin(), order.end(), [&](int p, int q) { return cost[p] > cost[q]; });
  std::vector<std::pair<double, int>> heap;
  for (int k = 0; k < blocks; ++k) heap.push_back({0.0, k});
  auto cmp = [](const std::pair<double, int>& p, const std::pair<double, int>& q) {
    return p.first > q.first || (p.first == q.first && p.second > q.second);
  };
  std::make_heap(heap.begin(), heap.end(), cmp);
  std::vector<std::vector<int>> lists(blocks);
  for (int t : order) {
    std::pop_heap(heap.begin(), heap.end(), cmp);
    heap.back().first += cost[t];
    lists[heap.back().second].push_back(t);
    std::push_heap(heap.begin(), heap.end(), cmp);
  }
  std::vector<TileDesc> sched;
  std::vector<int> start(blocks + 1, 0);
  sched.reserve(tiles.size());
  for (int k = 0; k < blocks; ++k) {
    std::sort(lists[k].begin(), lists[k].end());
    for (int t : lists[k]) sched.push_back(tiles[t]);
    start[k + 1] = (int)sched.size();
  }
  free_owned(b, b->d_tiles);
  free_owned(b, b->d_start);
  b->d_tiles = (TileDesc*)balloc(b, std::max<size_t>(1, sched.size()) * sizeof(TileDesc));
  b->d_start = (int*)balloc(b, start.size() * sizeof(int));
  if (!b->d_tiles || !b->d_start) return berr(b, "device allocation failed"), LB_ERR_NOMEM;
  BCK(cudaMemcpyAsync(b->d_tiles, sched.data(), sched.size() * sizeof(TileDesc), cudaMemcpyHostToDevice,
                      b->stream));
  BCK(cudaMemcpyAsync(b->d_start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  b->grid_blocks = blocks;
  return LB_OK;
}

template <class S>
static cudaError_t launch_reduce_s(lb_batch* b, int buf, int nsamples, int col, double* out, cudaStream_t s) {
  const CapDesc<typename S::A>* caps = (const CapDesc<typename S::A>*)b->d_caps;
  typename S::T* f = (typename S::T*)b->f[buf];
  typename S::T* g = (typename S::T*)b->g[buf];
  batch_partials_kernel<S><<<b->nchunks, RED_THREADS, 0, s>>>(caps, b->d_chunks, f, g, b->g0[buf], b->d_part);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_final_kernel<S><<<b->n, 1024, 0, s>>>(caps, b->d_range, b->n, f, g, b->g0[buf], b->d_part, nsamples, col,
                                              out);
  return cudaGetLastError();
}

// Reduction chunks: consecutive node ranges of kRedChunk nodes (the last one of
// a lattice ragged), so that the first pass has enough blocks for any batch.
static constexpr int kRedChunk = 1 << 13;

static lb_status build_chunks(lb_batch* b) {
  std::vector<RedChunk> chunks;
  std::vector<int2> range(b->n);
  for (int i = 0; i < b->n; ++i) {
    const int N = b->grids[i].nx * b->grids[i].ny;
    range[i].x = (int)chunks.size();
    for (int n0 = 0; n0 < N; n0 += kRedChunk) chunks.push_back(RedChunk{i, n0, std::min(N, n0 + kRedChunk)});
    range[i].y = (int)chunks.size() - range[i].x;
  }
  b->nchunks = (int)chunks.size();
  b->d_chunks = (RedChunk*)balloc(b, chunks.size() * sizeof(RedChunk));
  b->d_range = (int2*)balloc(b, range.size() * sizeof(int2));
  b->d_part = (double*)balloc(b, chunks.size() * 3 * sizeof(double));
  if (!b->d_chunks || !b->d_range || !b->d_part) return berr(b, "device allocation failed"), LB_ERR_NOMEM;
  BCK(cudaMemcpyAsync(b->d_chunks, chunks.data(), chunks.size() * sizeof(RedChunk), cudaMemcpyHostToDevice,
                      b->stream));
  BCK(cudaMemcpyAsync(b->d_range, range.data(), range.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return LB_OK;
}

static cudaError_t launch_reduce(lb_batch* b, int buf, int nsamples, int col, double* out, cudaStream_t s) {
  if (b->storage == LB_STORAGE_MOMENTS) return launch_reduce_s<SM32>(b, buf, nsamples, col, out, s);
  if (b->storage == LB_STORAGE_F64) return launch_reduce_s<SF64>(b, buf, nsamples, col, out, s);
  if (b->storage == LB_STORAGE_F32) return launch_reduce_s<SF32>(b, buf, nsamples, col, out, s);
  if (b->storage == LB_STORAGE_F32_BLOCKED) return launch_reduce_s<SF32B>(b, buf, nsamples, col, out, s);
  if (b->storage == LB_STORAGE_F16_BLOCKED) return launch_reduce_s<SF16B>(b, buf, nsamples, col, out, s);
  return launch_reduce_s<SF16>(b, buf, nsamples, col, out, s);
}

template <typename A>
static void fill_caps(lb_batch* b, std::vector<CapDesc<A>>& caps) {
  caps.resize(b->n);
  for (int i = 0; i < b->n; ++i) {
    const lb_grid& g = b->grids[i];
    const lb_walls& w = b->walls[i];
    const lb_params& p = b->params[i];
    CapDesc<A>& c = caps[i];
    c.G = Geom{g.nx, g.ny, w.tube_x0, w.tube_len, w.tube_y0, w.tube_h};
    c.P.kappa = A(p.kappa); c.P.a = A(p.a); c.P.b = A(p.b); c.P.T = A(p.T);
    c.P.Acoef = A(p.A); c.P.M = A(p.M); c.P.nu_l = A(p.nu_l); c.P.nu_g = A(p.nu_g);
    c.P.nu = A(p.nu); c.P.lambda_scale = A(p.lambda_scale); c.P.h = A(w.wall_grad);
    c.P.lut = A(p.nu_table >= 2 ? p.nu_table - 1 : 0);
    c.P.lut_inv = p.nu_table >= 2 ? A(1.0 / (p.nu_table - 1)) : A(0);
    c.P.omega = A(2.0 / (6.0 * p.nu + 1.0));  // liquid-gas only; a batch holds the binary model
    c.off_f = b->off_f[i];
    c.off_g = b->off_g[i];
    c.off_g0 = b->off_g0[i];
    c.r = rest_offsets_binary(p.A);
    c.Q = mom_phys(p.kappa, p.A, p.M, p.nu_l, p.nu_g, p.lambda_scale, w.wall_grad,
                   p.nu_table >= 2 ? p.nu_table - 1 : 0);
    c.thr = 0.0;
    c.rho_l = p.rho_l;
    c.rho_g = p.rho_g;
  }
}

static lb_status check_err(lb_batch* b) {
  int h = 0;
  BCK(cudaMemcpy(&h, b->d_err, sizeof h, cudaMemcpyDeviceToHost));
  if (h) {
    b->poisoned = 1;
    berr(b, "a wait of the persistent kernel timed out (state is unreliable)");
    return LB_ERR_TIMEOUT;
  }
  return LB_OK;
}

static lb_status ensure_out(lb_batch* b, size_t ndoubles) {
  if (b->out_cap >= ndoubles) return LB_OK;
  double* p = (double*)balloc(b, ndoubles * sizeof(double));
  if (!p) return berr(b, "device allocation failed"), LB_ERR_NOMEM;
  b->d_out = p;
  b->out_cap = ndoubles;
  return LB_OK;
}

extern "C" {

lb_status lb_batch_create(int n, const lb_grid* grids, const lb_walls* walls, const lb_params* params,
                          const lb_alloc* alloc, void* stream, lb_batch** out) {
  if (!out || n < 1 || !grids || !walls || !params) return berr(NULL, "invalid arguments"), LB_ERR_ARG;
  *out = NULL;
  const int storage = params[0].storage;
  if (storage != LB_STORAGE_F64 && storage != LB_STORAGE_F32 && storage != LB_STORAGE_F16DEV &&
      storage != LB_STORAGE_MOMENTS && storage != LB_STORAGE_F32_BLOCKED && storage != LB_STORAGE_F16_BLOCKED)
    return berr(NULL, "unknown storage %d", storage), LB_ERR_ARG;
  for (int i = 0; i < n; ++i) {
    if (params[i].model != LB_MODEL_BINARY) return berr(NULL, "batches hold binary lattices"), LB_ERR_ARG;
    if (params[i].storage != storage) return berr(NULL, "all lattices of a batch share one storage"), LB_ERR_ARG;
    const lb_grid& g = grids[i];
    const lb_walls& w = walls[i];
    if (g.nx < 3 || g.ny < 3 || (long)g.nx * g.ny > (1L << 31) - 1) return berr(NULL, "lattice %d: bad grid", i), LB_ERR_ARG;
    if (storage == LB_STORAGE_MOMENTS && (unsigned long long)M_PLANES * g.nx * g.ny >= (1ull << 32))
      return berr(NULL, "lattice %d: the moment storage holds at most 715827882 nodes", i), LB_ERR_ARG;
    if (storage == LB_STORAGE_F32_BLOCKED && 18ull * (((unsigned long long)g.nx * g.ny + 31) / 32 * 32) >= (1ull << 32))
      return berr(NULL, "lattice %d: the block storage holds at most 238609280 nodes", i), LB_ERR_ARG;
    if (storage == LB_STORAGE_F16_BLOCKED && 19ull * (((unsigned long long)g.nx * g.ny + 31) / 32 * 32) >= (1ull << 32))
      return berr(NULL, "lattice %d: the FP16 block storage holds at most 226050880 nodes", i), LB_ERR_ARG;
    if (!isfinite(w.wall_grad)) return berr(NULL, "lattice %d: wall_grad not finite", i), LB_ERR_ARG;
    if (!(params[i].M >= 0)) return berr(NULL, "lattice %d: mobility must be >= 0", i), LB_ERR_ARG;
    if (w.tube_len < 0 || w.tube_len > g.nx) return berr(NULL, "lattice %d: tube_len outside [0, nx]", i), LB_ERR_ARG;
    if (w.tube_len > 0 && (w.tube_x0 < 0 || w.tube_x0 >= g.nx || w.tube_y0 < 0 || w.tube_y0 >= g.ny ||
                           w.tube_h < 2 || w.tube_h >= g.ny || (w.tube_len < g.nx && g.nx - w.tube_len < 2)))
      return berr(NULL, "lattice %d: invalid tube geometry", i), LB_ERR_ARG;
    if (params[i].nu_table < 0 || params[i].nu_table == 1)
      return berr(NULL, "lattice %d: nu_table must be 0 or >= 2", i), LB_ERR_ARG;
    if (!(params[i].nu_l > 0) || !(params[i].nu_g > 0) || !(params[i].A > 0) || !(params[i].kappa > 0))
      return berr(NULL, "lattice %d: invalid binary parameters", i), LB_ERR_ARG;
  }
  if (alloc && (!alloc->malloc_fn || !alloc->free_fn)) return berr(NULL, "incomplete allocator"), LB_ERR_ARG;
  lb_batch* b = new (std::nothrow) lb_batch();
  if (!b) return berr(NULL, "out of host memory"), LB_ERR_NOMEM;
  b->n = n;
  b->storage = storage;
  b->grids.assign(grids, grids + n);
  b->walls.assign(walls, walls + n);
  b->params.assign(params, params + n);
  b->stream = (cudaStream_t)stream;
  b->have_alloc = alloc != NULL;
  if (alloc) b->alloc = *alloc;
  b->tile_x = 128;
  b->tile_y = 8;
  b->staged_ok = 1;
  for (int i = 0; i < n; ++i)  // the block storages stage whole blocks at any nx
    b->staged_ok = b->staged_ok && (storage == LB_STORAGE_F32_BLOCKED || storage == LB_STORAGE_F16_BLOCKED ||
                                    staged_fits(grids[i].nx, grids[i].ny));
  b->limit_ns = kDefaultLimitNs;
  if (cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) != cudaSuccess) {
    berr(NULL, "cudaStreamCreate failed");
    delete b;
    return LB_ERR_CUDA;
  }
  const size_t el = elem_size(storage);
  const int moments = storage == LB_STORAGE_MOMENTS;
  // f and g in 32-node blocks, one arena: elements per 32 nodes (floats or halves)
  const int blocked = storage == LB_STORAGE_F32_BLOCKED ? 18 : (storage == LB_STORAGE_F16_BLOCKED ? 19 : 0);
  const int nf = moments ? M_PLANES : 9;
  const int ng = (moments || blocked) ? 0 : (storage == LB_STORAGE_F16DEV ? 8 : 9);
  size_t of = 0, og = 0, o0 = 0;
  for (int i = 0; i < n; ++i) {
    const size_t N = (size_t)grids[i].nx * grids[i].ny;
    b->off_f.push_back(of);
    b->off_g.push_back(og);
    b->off_g0.push_back(o0);
    of += blocked ? (blocked * ((N + 31) / 32 * 32) + 63) / 64 * 64 : (nf * N + 63) / 64 * 64;
    og += (ng * N + 63) / 64 * 64;
    o0 += (N + 63) / 64 * 64;
    // solid nodes: the tube's columns outside its band
    b->fluid.push_back((long)N - (walls[i].tube_len > 0 ? (long)walls[i].tube_len * (grids[i].ny - walls[i].tube_h) : 0));
  }
  for (int k = 0; k < 2; ++k) {
    b->f[k] = balloc(b, of * el);
    b->g[k] = og ? balloc(b, og * el) : NULL;
    b->g0[k] = storage == LB_STORAGE_F16DEV ? (float*)balloc(b, o0 * sizeof(float)) : NULL;
    b->bytes_f = of * el;
    b->bytes_g = og ? og * el : 0;
    b->bytes_g0 = storage == LB_STORAGE_F16DEV ? o0 * sizeof(float) : 0;
    if (!b->f[k] || (og && !b->g[k]) || (storage == LB_STORAGE_F16DEV && !b->g0[k])) {
      snprintf(g_batch_create_err, sizeof g_batch_create_err, "device allocation of the batch state failed");
      lb_batch_destroy(b);
      return LB_ERR_NOMEM;
    }
    // solid nodes are never written by a step: start them (and everything) at 0
    cudaError_t ez = cudaMemsetAsync(b->f[k], 0, of * el, b->stream);
    if (ez == cudaSuccess && og) ez = cudaMemsetAsync(b->g[k], 0, og * el, b->stream);
    if (ez == cudaSuccess && b->g0[k]) ez = cudaMemsetAsync(b->g0[k], 0, o0 * sizeof(float), b->stream);
    if (ez != cudaSuccess) {
      snprintf(g_batch_create_err, sizeof g_batch_create_err, "clearing the batch state failed");
      lb_batch_destroy(b);
      return LB_ERR_CUDA;
    }
  }
  const size_t capbytes = (size_t)n * std::max(sizeof(CapDesc<double>), sizeof(CapDesc<float>));
  b->d_caps = balloc(b, capbytes);
  b->d_bar = (GridBarrier*)balloc(b, 256);
  b->d_err = (int*)balloc(b, 256);
  if (!b->d_caps || !b->d_bar || !b->d_err) {
    snprintf(g_batch_create_err, sizeof g_batch_create_err, "device allocation failed");
    lb_batch_destroy(b);
    return LB_ERR_NOMEM;
  }
  cudaError_t e = cudaSuccess;
  if (storage == LB_STORAGE_F64) {
    std::vector<CapDesc<double>> caps;
    fill_caps(b, caps);
    e = cudaMemcpy(b->d_caps, caps.data(), n * sizeof(CapDesc<double>), cudaMemcpyHostToDevice);
  } else {
    std::vector<CapDesc<float>> caps;
    fill_caps(b, caps);
    e = cudaMemcpy(b->d_caps, caps.data(), n * sizeof(CapDesc<float>), cudaMemcpyHostToDevice);
  }
  if (e == cudaSuccess) e = cudaMemset(b->d_bar, 0, 256);
  if (e == cudaSuccess) e = cudaMemset(b->d_err, 0, 256);
  lb_status st = e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
  if (st == LB_OK) st = build_tiles(b);
  if (st == LB_OK) st = build_chunks(b);
  for (int i = 0; i < n && st == LB_OK; ++i) st = init_lattice(b, i);
  if (st != LB_OK) {
    snprintf(g_batch_create_err, sizeof g_batch_create_err, "%s", e != cudaSuccess ? cudaGetErrorString(e) : b->err);
    lb_batch_destroy(b);
    return st;
  }
  *out = b;
  return LB_OK;
}

void lb_batch_destroy(lb_batch* b) {
  if (!b) return;
  cudaStreamSynchronize(b->stream);
  bfree_all(b);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

lb_status lb_batch_step(lb_batch* b, long n) {
  NvtxRange range("lb_batch_step");
  if (!b) return LB_ERR_ARG;
  if (n < 0 || n > (1L << 30)) return berr(b, "step count out of range"), LB_ERR_ARG;
  if (b->poisoned) return berr(b, "batch holds a timed-out state"), LB_ERR_STATE;
  if (n == 0) return LB_OK;
  BCK(launch_batch(b, (int)n, b->stream));
  b->parity = (b->parity + (int)(n & 1)) & 1;
  b->t += n;
  return LB_OK;
}

size_t lb_batch_state_bytes(const lb_batch* b) { return b ? b->bytes_f + b->bytes_g + b->bytes_g0 : 0; }

// The arenas of the current state as they are held on the device: f, then g, then g_0.
lb_status lb_batch_save_state(lb_batch* b, void* host, size_t bytes) {
  if (!b || !host) return b ? (berr(b, "host is NULL"), LB_ERR_ARG) : LB_ERR_ARG;
  if (bytes != lb_batch_state_bytes(b)) return berr(b, "bytes must equal lb_batch_state_bytes"), LB_ERR_ARG;
  const int k = b->parity;
  unsigned char* h = static_cast<unsigned char*>(host);
  BCK(cudaMemcpyAsync(h, b->f[k], b->bytes_f, cudaMemcpyDeviceToHost, b->stream));
  if (b->bytes_g) BCK(cudaMemcpyAsync(h + b->bytes_f, b->g[k], b->bytes_g, cudaMemcpyDeviceToHost, b->stream));
  if (b->bytes_g0)
    BCK(cudaMemcpyAsync(h + b->bytes_f + b->bytes_g, b->g0[k], b->bytes_g0, cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return LB_OK;
}

lb_status lb_batch_load_state(lb_batch* b, const void* host, size_t bytes, long time) {
  if (!b || !host || time < 0) return b ? (berr(b, "host is NULL or time < 0"), LB_ERR_ARG) : LB_ERR_ARG;
  if (bytes != lb_batch_state_bytes(b)) return berr(b, "bytes must equal lb_batch_state_bytes"), LB_ERR_ARG;
  const unsigned char* h = static_cast<const unsigned char*>(host);
  BCK(cudaMemcpyAsync(b->f[0], h, b->bytes_f, cudaMemcpyHostToDevice, b->stream));
  if (b->bytes_g) BCK(cudaMemcpyAsync(b->g[0], h + b->bytes_f, b->bytes_g, cudaMemcpyHostToDevice, b->stream));
  if (b->bytes_g0)
    BCK(cudaMemcpyAsync(b->g0[0], h + b->bytes_f + b->bytes_g, b->bytes_g0, cudaMemcpyHostToDevice, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  b->parity = 0;
  b->t = time;
  return LB_OK;
}

lb_status lb_batch_lengths(lb_batch* b, double* out) {
  NvtxRange range("lb_batch_lengths");
  if (!b || !out) return LB_ERR_ARG;
  lb_status st = ensure_out(b, (size_t)b->n * 4);
  if (st) return st;
  BCK(launch_reduce(b, b->parity, 1, 0, b->d_out, b->stream));
  BCK(cudaMemcpyAsync(out, b->d_out, (size_t)b->n * 4 * sizeof(double), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return check_err(b);
}

lb_status lb_batch_run_sampled(lb_batch* b, int nsamples, const long* at, double* out) {
  NvtxRange range("lb_batch_run_sampled");
  if (!b || nsamples < 1 || !at || !out) return LB_ERR_ARG;
  if (b->poisoned) return berr(b, "batch holds a timed-out state"), LB_ERR_STATE;
  long prev = 0;
  for (int k = 0; k < nsamples; ++k) {
    if (at[k] < prev || at[k] - prev > (1L << 30)) return berr(b, "sample steps must be non-decreasing"), LB_ERR_ARG;
    prev = at[k];
  }
  lb_status st = ensure_out(b, (size_t)b->n * nsamples * 4);
  if (st) return st;
  // one graph: for each sample, a persistent launch for the steps since the last
  // sample and a reduction into that sample's column
  BCK(cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeThreadLocal));
  int parity = b->parity;
  long t = 0;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < nsamples && e == cudaSuccess; ++k) {
    const long d = at[k] - t;
    if (d > 0) {
      const int save = b->parity;
      b->parity = parity;
      e = launch_batch(b, (int)d, b->cap);
      b->parity = save;
      parity = (parity + (int)(d & 1)) & 1;
      t = at[k];
    }
    if (e == cudaSuccess) e = launch_reduce(b, parity, nsamples, k, b->d_out, b->cap);
  }
  cudaGraph_t graph = NULL;
  cudaError_t e2 = cudaStreamEndCapture(b->cap, &graph);
  if (e == cudaSuccess) e = e2;
  cudaGraphExec_t exec = NULL;
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (e == cudaSuccess) {
    e = cudaGraphLaunch(exec, b->stream);
  } else {
    // CUDA refused the graph: issue the same sequence directly
    cudaGetLastError();
    parity = b->parity;
    t = 0;
    e = cudaSuccess;
    for (int k = 0; k < nsamples && e == cudaSuccess; ++k) {
      const long d = at[k] - t;
      if (d > 0) {
        const int save = b->parity;
        b->parity = parity;
        e = launch_batch(b, (int)d, b->stream);
        b->parity = save;
        parity = (parity + (int)(d & 1)) & 1;
        t = at[k];
      }
      if (e == cudaSuccess) e = launch_reduce(b, parity, nsamples, k, b->d_out, b->stream);
    }
    b->graph_fallbacks++;
  }
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(out, b->d_out, (size_t)b->n * nsamples * 4 * sizeof(double), cudaMemcpyDeviceToHost,
                        b->stream);
  cudaError_t e3 = cudaStreamSynchronize(b->stream);
  if (exec) cudaGraphExecDestroy(exec);
  if (e == cudaSuccess) e = e3;
  if (e != cudaSuccess) return berr(b, "lb_batch_run_sampled: %s", cudaGetErrorString(e)), LB_ERR_CUDA;
  b->parity = parity;
  b->t += t;
  return check_err(b);
}

lb_status lb_batch_moments(lb_batch* b, int i, double* m) {
  if (!b || i < 0 || i >= b->n || !m) return LB_ERR_ARG;
  const size_t N = (size_t)b->grids[i].nx * b->grids[i].ny;
  double* d = NULL;
  if (b->have_alloc)
    d = (double*)b->alloc.malloc_fn(M_PLANES * N * sizeof(double), (void*)b->stream, b->alloc.user);
  else if (cudaMalloc((void**)&d, M_PLANES * N * sizeof(double)) != cudaSuccess)
    d = NULL;
  if (!d) return berr(b, "device allocation failed"), LB_ERR_NOMEM;
  OpArgs a = lattice_args(b, i, b->parity);
  a.out0 = d;
  cudaError_t e = batch_ops(b->storage)(OP_MOMENTS_OUT, a, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m, d, M_PLANES * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  cudaError_t e2 = cudaStreamSynchronize(b->stream);
  if (b->have_alloc)
    b->alloc.free_fn(d, (void*)b->stream, b->alloc.user);
  else
    cudaFree(d);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return berr(b, "lb_batch_moments: %s", cudaGetErrorString(e)), LB_ERR_CUDA;
  return LB_OK;
}

lb_status lb_batch_populations(lb_batch* b, int i, double* f, double* g, int rested) {
  if (!b || i < 0 || i >= b->n || !f) return LB_ERR_ARG;
  if (b->storage == LB_STORAGE_MOMENTS)
    return berr(b, "the moment storage keeps no populations (lb_batch_moments)"), LB_ERR_ARG;
  const size_t N = (size_t)b->grids[i].nx * b->grids[i].ny;
  double* d = NULL;
  if (b->have_alloc)
    d = (double*)b->alloc.malloc_fn(18 * N * sizeof(double), (void*)b->stream, b->alloc.user);
  else if (cudaMalloc((void**)&d, 18 * N * sizeof(double)) != cudaSuccess)
    d = NULL;
  if (!d) return berr(b, "device allocation failed"), LB_ERR_NOMEM;
  OpArgs a = lattice_args(b, i, b->parity);
  a.flag = rested;
  a.out0 = d;
  a.out1 = d + 9 * N;
  cudaError_t e = batch_ops(b->storage)(OP_POPS_OUT, a, b->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  if (e == cudaSuccess && g) e = cudaMemcpyAsync(g, d + 9 * N, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, b->stream);
  cudaError_t e2 = cudaStreamSynchronize(b->stream);
  if (b->have_alloc)
    b->alloc.free_fn(d, (void*)b->stream, b->alloc.user);
  else
    cudaFree(d);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) return berr(b, "lb_batch_populations: %s", cudaGetErrorString(e)), LB_ERR_CUDA;
  return LB_OK;
}

lb_status lb_batch_set_tile(lb_batch* b, int tile_x, int tile_y) {
  if (!b) return LB_ERR_ARG;
  if (tile_x != 64 && tile_x != 128 && tile_x != 256) return berr(b, "tile_x must be 64, 128 or 256"), LB_ERR_ARG;
  if (tile_y < 1 || tile_y > 4096) return berr(b, "tile_y out of range"), LB_ERR_ARG;
  BCK(cudaStreamSynchronize(b->stream));
  b->tile_x = tile_x;
  b->tile_y = tile_y;
  return build_tiles(b);
}

lb_status lb_batch_autotune(lb_batch* b, int steps, int* tile_x, int* tile_y, double* ms_per_step) {
  NvtxRange range("lb_batch_autotune");
  if (!b || steps < 1) return LB_ERR_ARG;
  if (b->poisoned) return LB_ERR_STATE;
  // tuning runs advance the state: run an even number of steps per candidate and
  // restore nothing else (callers tune before they start a measured run).
  // Candidates: the sliding-window body, and the staged body with its shallow
  // and deep rings (when every nx % 8 == 0), each over the tiles below; an
  // explicit lb_batch_set_kernel choice limits the bodies tried.
  // The moment storage has one body (band heights as in lb_autotune).
  const int moments = b->storage == LB_STORAGE_MOMENTS;
  const int cx[3] = {64, 128, 256};
  const std::vector<int> cy = moments ? std::vector<int>{8, 12, 16, 20, 24, 32, 48}
                                      : std::vector<int>{4, 8, 16, 32, 64};
  struct Body {
    int kernel, deep;
  };
  Body bodies[3];
  int nb = 0;
  if (moments) {
    bodies[nb++] = Body{0, 0};
  } else {
    if (b->kernel != 2) bodies[nb++] = Body{1, 0};
    if (b->kernel != 1 && b->staged_ok) {
      bodies[nb++] = Body{2, 0};
      bodies[nb++] = Body{2, 1};
    }
  }
  const int keep_kernel = b->kernel;
  int bx = b->tile_x, by = b->tile_y, bk = batch_variant(b), bd = b->deep;
  float best = 1e30f;
  cudaEvent_t e0, e1;
  BCK(cudaEventCreate(&e0));
  BCK(cudaEventCreate(&e1));
  lb_status st = LB_OK;
  for (int v = 0; v < nb && st == LB_OK; ++v)
    for (int i = 0; i < 3 && st == LB_OK; ++i)
      for (size_t j = 0; j < cy.size() && st == LB_OK; ++j) {
        b->kernel = bodies[v].kernel;
        b->deep = bodies[v].deep;
        st = lb_batch_set_tile(b, cx[i], cy[j]);
        if (st) break;
        st = lb_batch_step(b, 2);
        if (st) break;
        cudaEventRecord(e0, b->stream);
        st = lb_batch_step(b, 2 * steps);
        cudaEventRecord(e1, b->stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (st == LB_OK && ms < best) {
          best = ms;
          bx = cx[i];
          by = cy[j];
          bk = bodies[v].kernel;
          bd = bodies[v].deep;
        }
      }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  b->kernel = keep_kernel;
  if (st) return st;
  st = check_err(b);
  if (st) return st;
  // an automatic choice stays automatic unless tuning preferred the other body
  if (!moments && (keep_kernel != 0 || bk != batch_variant(b))) b->kernel = bk;
  b->deep = bd;
  st = lb_batch_set_tile(b, bx, by);  // rebuilds the schedule for this body
  if (st) return st;
  if (tile_x) *tile_x = bx;
  if (tile_y) *tile_y = by;
  if (ms_per_step) *ms_per_step = best / (2.0 * steps);
  return LB_OK;
}

lb_status lb_batch_set_barrier(lb_batch* b, unsigned int absent_blocks, double limit_seconds) {
  if (!b || !(limit_seconds > 0) || limit_seconds > 60) return LB_ERR_ARG;
  BCK(cudaStreamSynchronize(b->stream));
  b->extra_arrivals = absent_blocks;
  b->limit_ns = (unsigned long long)(limit_seconds * 1e9);
  BCK(cudaMemset(b->d_bar, 0, 256));
  return LB_OK;
}

lb_status lb_batch_set_kernel(lb_batch* b, int variant) {
  if (!b) return LB_ERR_ARG;
  if (b->storage == LB_STORAGE_MOMENTS)
    return variant == 0 || variant == 4 ? LB_OK : (berr(b, "the moment storage has one body (variant 4)"), LB_ERR_ARG);
  if (variant < 0 || variant > 3) return berr(b, "kernel variant must be 0, 1, 2 or 3"), LB_ERR_ARG;
  if (variant >= 2 && !b->staged_ok)
    return berr(b, "the staged body needs nx %% 8 == 0 and at most 477218588 nodes in every lattice"), LB_ERR_ARG;
  BCK(cudaStreamSynchronize(b->stream));
  b->kernel = variant == 3 ? 2 : variant;
  if (variant >= 2) b->deep = variant == 3;
  return build_tiles(b);  // resident CTAs, hence the schedule, depend on the body
}

lb_status lb_batch_get_kernel(const lb_batch* b, int* variant) {
  if (!b || !variant) return LB_ERR_ARG;
  const int k = batch_variant(b);
  *variant = k == 2 && b->deep ? 3 : k;
  return LB_OK;
}

lb_status lb_batch_check_report(lb_batch* b, int* enabled, unsigned long long* bad, unsigned long long* first_bad) {
  if (!b) return LB_ERR_ARG;
  BCK(cudaStreamSynchronize(b->stream));
  unsigned long long h[3] = {0, 0, 0};
  BCK(read_check_counters(h));
  if (enabled) *enabled = (int)h[0];
  if (bad) *bad = h[1];
  if (first_bad) *first_bad = h[2];
  return LB_OK;
}

long lb_batch_time(const lb_batch* b) { return b ? b->t : -1; }

long lb_batch_fluid_nodes(const lb_batch* b, int i) {
  if (!b) return -1;
  if (i >= 0) return i < b->n ? b->fluid[i] : -1;
  long s = 0;
  for (long v : b->fluid) s += v;
  return s;
}

const char* lb_batch_last_error(const lb_batch* b) { return b ? b->err : g_batch_create_err; }

}  // extern "C"
