// Host library behind include/lb.h: context, device memory, stream, CUDA-graph
// replay of the step kernel, reductions, kernel and tile autotuner, state import,
// export and byte-exact checkpoints.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <new>
#include <vector>

#include "lb.h"
#include "lb_aux.cuh"
#include "lb_ops.h"

using namespace lbk;

namespace {

constexpr int kGraphSteps = 64;  // steps per captured graph (even: parity preserved)
constexpr int kRedPartsPerSM = 4;  // blocks of the first reduction pass per SM

thread_local char g_create_err[512] = "";

}  // namespace

struct lb_ctx {
  lb_grid grid;
  lb_walls walls;
  lb_params prm;
  cudaStream_t stream;
  cudaStream_t cap;  // private stream used only to capture graphs
  lb_alloc alloc;
  int have_alloc;
  OpsFn ops;
  OpBufs buf[2];
  int cur;
  long t;
  long fluid;
  double* partials;
  int nparts;    // blocks of the first reduction pass (partials holds nparts x RED_PARTS)
  double* red_out;
  int tile_x, tile_y;
  int kernel;   // 0 auto, 1 sliding window, 2 staged
  int deep;     // staged kernel ring depth choice
  int* errflag; // device error word written by the staged kernel
  cudaGraphExec_t gexec;
  int poisoned;
  char err[512];
  std::vector<void*> owned;
};

static void set_err(lb_ctx* c, const char* fmt, ...) {
  char* dst = c ? c->err : g_create_err;
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(dst, 512, fmt, ap);
  va_end(ap);
}

#define CK(call)                                                                          \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      set_err(c, "%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return LB_ERR_CUDA;                                                                 \
    }                                                                                     \
  } while (0)

static void* dev_alloc(lb_ctx* c, size_t bytes) {
  void* p = NULL;
  if (c->have_alloc) {
    p = c->alloc.malloc_fn(bytes, (void*)c->stream, c->alloc.user);
  } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    p = NULL;
  }
  return p;
}

static void dev_free(lb_ctx* c, void* p) {
  if (!p) return;
  if (c->have_alloc)
    c->alloc.free_fn(p, (void*)c->stream, c->alloc.user);
  else
    cudaFree(p);
}

static void* dev_alloc_owned(lb_ctx* c, size_t bytes) {
  void* p = dev_alloc(c, bytes);
  if (p) c->owned.push_back(p);
  return p;
}

static OpsFn pick_ops(int model, int storage) {
  if (model == LB_MODEL_LIQUID_GAS) {
    if (storage == LB_STORAGE_F64) return ops_lg_f64;
    if (storage == LB_STORAGE_F32) return ops_lg_f32;
    return NULL;
  }
  if (model == LB_MODEL_BINARY) {
    if (storage == LB_STORAGE_F64) return ops_bin_f64;
    if (storage == LB_STORAGE_F32) return ops_bin_f32;
    if (storage == LB_STORAGE_F16DEV) return ops_bin_f16;
    if (storage == LB_STORAGE_MOMENTS) return ops_bin_m32;
    if (storage == LB_STORAGE_MOMENTS_F16) return ops_bin_m16;
    if (storage == LB_STORAGE_F32_GELIM) return ops_bin_g32;
    if (storage == LB_STORAGE_F32_BLOCKED) return ops_bin_f32b;
    if (storage == LB_STORAGE_F16_BLOCKED) return ops_bin_f16b;
  }
  return NULL;
}

// The staged population kernel applies: 16-byte aligned rows of the planar
// storages (nx % 8 == 0) and 32-bit offsets; the block storage stages whole
// blocks at any nx (its node limit is checked at creation).
static bool staged_ok(int storage, int nx, int ny) {
  return storage == LB_STORAGE_F32_BLOCKED || storage == LB_STORAGE_F16_BLOCKED || staged_fits(nx, ny);
}

static OpArgs base_args(const lb_ctx* c) {
  OpArgs a;
  memset(&a, 0, sizeof a);
  a.nx = c->grid.nx;
  a.ny = c->grid.ny;
  a.tube_x0 = c->walls.tube_x0;
  a.tube_len = c->walls.tube_len;
  a.tube_y0 = c->walls.tube_y0;
  a.tube_h = c->walls.tube_h;
  const lb_params& p = c->prm;
  a.kappa = p.kappa; a.a = p.a; a.b = p.b; a.T = p.T;
  a.Acoef = p.A; a.M = p.M; a.nu_l = p.nu_l; a.nu_g = p.nu_g;
  a.nu = p.nu; a.lambda_scale = p.lambda_scale; a.h = c->walls.wall_grad;
  a.lut = p.model == LB_MODEL_BINARY && p.nu_table >= 2 ? p.nu_table - 1 : 0;
  a.rho_l = p.rho_l; a.rho_g = p.rho_g;
  a.thr = p.model == LB_MODEL_LIQUID_GAS ? 0.5 * (p.rho_l + p.rho_g) : 0.0;
  a.bx = c->tile_x;
  a.yc = c->tile_y;
  a.staged = c->kernel == 2 || (c->kernel == 0 && staged_ok(c->prm.storage, c->grid.nx, c->grid.ny));
  a.deep = c->deep;
  a.err = c->errflag;
  return a;
}

// After a synchronisation: a device-side wait that gave up poisons the context.
static lb_status check_device_error(lb_ctx* c) {
  int h = 0;
  CK(cudaMemcpy(&h, c->errflag, sizeof h, cudaMemcpyDeviceToHost));
  if (h) {
    c->poisoned = 1;
    set_err(c, "a device-side wait of the step kernel timed out (state is unreliable)");
    return LB_ERR_TIMEOUT;
  }
  return LB_OK;
}

// A new state clears a timed-out condition: the device error word as well as the
// host flag, or the next waiting call would report the old timeout again.
static cudaError_t clear_device_error(lb_ctx* c) {
  return cudaMemsetAsync(c->errflag, 0, sizeof(int), c->stream);
}

static lb_status launch_one(lb_ctx* c, cudaStream_t s, int from) {
  OpArgs a = base_args(c);
  a.src = c->buf[from];
  a.dst = c->buf[1 - from];
  CK(c->ops(OP_STEP, a, s));
  return LB_OK;
}

static void drop_graph(lb_ctx* c) {
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  c->gexec = NULL;
}

static lb_status build_graph(lb_ctx* c) {
  drop_graph(c);
  CK(cudaStreamBeginCapture(c->cap, cudaStreamCaptureModeThreadLocal));
  lb_status st = LB_OK;
  for (int k = 0; k < kGraphSteps && st == LB_OK; ++k) st = launch_one(c, c->cap, k & 1);
  cudaGraph_t g = NULL;
  cudaError_t e = cudaStreamEndCapture(c->cap, &g);
  if (st != LB_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  CK(e);
  e = cudaGraphInstantiate(&c->gexec, g, 0);
  cudaGraphDestroy(g);
  CK(e);
  return LB_OK;
}

// Storages advanced by the pull kernel (the state is not the eighteen populations).
static bool pull_storage(int storage) {
  return storage == LB_STORAGE_MOMENTS || storage == LB_STORAGE_MOMENTS_F16 || storage == LB_STORAGE_F32_GELIM;
}

static size_t state_bytes(int model, int storage, size_t N, size_t* fb, size_t* gb, size_t* g0b) {
  if (pull_storage(storage)) {  // everything in the f buffer
    *fb = storage == LB_STORAGE_MOMENTS ? (size_t)M_PLANES * N * sizeof(float)
        : storage == LB_STORAGE_MOMENTS_F16 ? m16_layout(N).total
                                            : 10 * N * sizeof(float);
    *gb = 0;
    *g0b = 0;
    return *fb;
  }
  if (storage == LB_STORAGE_F32_BLOCKED || storage == LB_STORAGE_F16_BLOCKED) {
    // f and g of every 32-node block together, in the f buffer
    *fb = (N + 31) / 32 * (storage == LB_STORAGE_F32_BLOCKED ? 2304 : 1216);
    *gb = 0;
    *g0b = 0;
    return *fb;
  }
  size_t el = storage == LB_STORAGE_F64 ? 8 : (storage == LB_STORAGE_F32 ? 4 : 2);
  *fb = 9 * N * el;
  *gb = model == LB_MODEL_BINARY ? (storage == LB_STORAGE_F16DEV ? 8 : 9) * N * el : 0;
  *g0b = (model == LB_MODEL_BINARY && storage == LB_STORAGE_F16DEV) ? N * 4 : 0;
  return *fb + *gb + *g0b;
}

static lb_status validate(const lb_grid* g, const lb_walls* w, const lb_params* p, lb_ctx* c) {
  if (!g || !w || !p) return set_err(c, "NULL argument"), LB_ERR_ARG;
  if (g->nx < 3 || g->ny < 3) return set_err(c, "grid must be at least 3x3"), LB_ERR_ARG;
  if ((long)g->nx * g->ny > (1L << 31) - 1) return set_err(c, "grid too large"), LB_ERR_ARG;
  if (!pick_ops(p->model, p->storage)) return set_err(c, "unsupported model/storage pair"), LB_ERR_ARG;
  if (p->storage == LB_STORAGE_MOMENTS && (unsigned long long)M_PLANES * g->nx * g->ny >= (1ull << 32))
    return set_err(c, "the moment storage holds at most 715827882 nodes"), LB_ERR_ARG;
  if (p->storage == LB_STORAGE_F32_GELIM && 10ull * g->nx * g->ny >= (1ull << 32))
    return set_err(c, "the g-eliminated storage holds at most 429496729 nodes"), LB_ERR_ARG;
  if (p->storage == LB_STORAGE_F32_BLOCKED && 18ull * (((unsigned long long)g->nx * g->ny + 31) / 32 * 32) >= (1ull << 32))
    return set_err(c, "the block storage holds at most 238609280 nodes"), LB_ERR_ARG;
  if (p->storage == LB_STORAGE_F16_BLOCKED && 19ull * (((unsigned long long)g->nx * g->ny + 31) / 32 * 32) >= (1ull << 32))
    return set_err(c, "the FP16 block storage holds at most 226050880 nodes"), LB_ERR_ARG;
  if (w->tube_len < 0 || w->tube_len > g->nx) return set_err(c, "tube_len outside [0, nx]"), LB_ERR_ARG;
  if (w->tube_len > 0) {
    if (w->tube_x0 < 0 || w->tube_x0 >= g->nx || w->tube_y0 < 0 || w->tube_y0 >= g->ny)
      return set_err(c, "tube origin outside the grid"), LB_ERR_ARG;
    if (w->tube_h < 2 || w->tube_h >= g->ny) return set_err(c, "need 2 <= tube_h < ny"), LB_ERR_ARG;
    if (w->tube_len < g->nx && g->nx - w->tube_len < 2)
      return set_err(c, "need at least 2 reservoir columns"), LB_ERR_ARG;
  }
  if (!isfinite(w->wall_grad)) return set_err(c, "wall_grad not finite"), LB_ERR_ARG;
  if (p->model == LB_MODEL_LIQUID_GAS) {
    if (!(p->nu > 0)) return set_err(c, "nu must be > 0 (omega in (0, 2))"), LB_ERR_ARG;
    if (!(p->b > 0) || !(p->T > 0) || !(p->kappa >= 0)) return set_err(c, "invalid van der Waals parameters"), LB_ERR_ARG;
    if (!(p->rho_l > p->rho_g) || !(p->rho_l * p->b < 1.0))
      return set_err(c, "need rho_g < rho_l < 1/b"), LB_ERR_ARG;
  } else {
    if (!(p->nu_l > 0) || !(p->nu_g > 0)) return set_err(c, "nu_l, nu_g must be > 0"), LB_ERR_ARG;
    if (!(p->A > 0) || !(p->kappa > 0) || !(p->M >= 0)) return set_err(c, "invalid binary parameters"), LB_ERR_ARG;
    if (p->nu_table < 0 || p->nu_table == 1) return set_err(c, "nu_table must be 0 or >= 2"), LB_ERR_ARG;
  }
  return LB_OK;
}

// cols: the four fields are given as one value per column (every row alike)
static lb_status upload_and_init(lb_ctx* c, const double* rho, const double* ux, const double* uy,
                                 const double* phi, bool cols = false) {
  const size_t N = cols ? (size_t)c->grid.nx : (size_t)c->grid.nx * c->grid.ny;
  double* d = (double*)dev_alloc(c, 4 * N * sizeof(double));
  if (!d) return set_err(c, "device allocation of %zu bytes failed", 4 * N * sizeof(double)), LB_ERR_NOMEM;
  lb_status st = LB_OK;
  const double* src[4] = {rho, ux, uy, phi};
  for (int k = 0; k < 4 && st == LB_OK; ++k) {
    cudaError_t e = src[k] ? cudaMemcpyAsync(d + k * N, src[k], N * sizeof(double), cudaMemcpyHostToDevice, c->stream)
                           : cudaMemsetAsync(d + k * N, 0, N * sizeof(double), c->stream);
    if (e != cudaSuccess) {
      set_err(c, "upload failed: %s", cudaGetErrorString(e));
      st = LB_ERR_CUDA;
    }
  }
  if (st == LB_OK) {
    OpArgs a = base_args(c);
    a.dst = c->buf[0];
    a.in0 = d;
    a.in1 = d + N;
    a.in2 = d + 2 * N;
    a.in3 = d + 3 * N;
    a.in_cols = cols;
    cudaError_t e = c->ops(OP_INIT, a, c->stream);
    if (e == cudaSuccess) e = clear_device_error(c);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
      set_err(c, "init failed: %s", cudaGetErrorString(e));
      st = LB_ERR_CUDA;
    }
  }
  cudaStreamSynchronize(c->stream);
  dev_free(c, d);
  if (st == LB_OK) {
    c->cur = 0;
    c->t = 0;
    c->poisoned = 0;
  }
  return st;
}

// The initial state of Sec. 2.2 / 3.2: at rest, with tanh profiles along x (so one
// value per column; solid nodes take no input values, the init kernel zeroes them).
static lb_status default_state(lb_ctx* c) {
  const int nx = c->grid.nx;
  std::vector<double> rho(nx), z(nx, 0.0), phi(nx);
  const lb_params& p = c->prm;
  const double wdt = p.model == LB_MODEL_LIQUID_GAS ? 2.0 : sqrt(2.0);
  const double xa = c->walls.gas_cols, xb = (double)c->walls.tube_x0 + p.l0;
  for (int x = 0; x < nx; ++x) {
    const double chi = 0.5 * (tanh((x - xa) / wdt) - tanh((x - xb) / wdt));
    if (p.model == LB_MODEL_LIQUID_GAS) {
      rho[x] = p.rho_g + (p.rho_l - p.rho_g) * chi;
      phi[x] = 0.0;
    } else {
      rho[x] = 1.0;
      phi[x] = 2.0 * chi - 1.0;
    }
  }
  return upload_and_init(c, rho.data(), z.data(), z.data(), phi.data(), true);
}

extern "C" {

lb_status lb_create(const lb_grid* grid, const lb_walls* walls, const lb_params* params, const lb_alloc* alloc,
                    void* stream, lb_ctx** out) {
  lb_ctx* c = NULL;
  if (!out) return set_err(NULL, "out is NULL"), LB_ERR_ARG;
  *out = NULL;
  lb_status st = validate(grid, walls, params, NULL);
  if (st != LB_OK) return st;
  if (alloc && (!alloc->malloc_fn || !alloc->free_fn)) return set_err(NULL, "incomplete allocator"), LB_ERR_ARG;
  c = new (std::nothrow) lb_ctx();
  if (!c) return set_err(NULL, "out of host memory"), LB_ERR_NOMEM;
  c->grid = *grid;
  c->walls = *walls;
  c->prm = *params;
  c->stream = (cudaStream_t)stream;
  c->have_alloc = alloc != NULL;
  if (alloc) c->alloc = *alloc;
  c->ops = pick_ops(params->model, params->storage);
  c->tile_x = 128;
  c->tile_y = grid->ny < 16 ? grid->ny : 16;
  c->gexec = NULL;
  c->err[0] = 0;
  if (cudaStreamCreateWithFlags(&c->cap, cudaStreamNonBlocking) != cudaSuccess) {
    set_err(NULL, "cudaStreamCreate failed: %s", cudaGetErrorString(cudaGetLastError()));
    delete c;
    return LB_ERR_CUDA;
  }
  const size_t N = (size_t)grid->nx * grid->ny;
  size_t fb, gb, g0b;
  state_bytes(params->model, params->storage, N, &fb, &gb, &g0b);
  for (int k = 0; k < 2; ++k) {
    c->buf[k].f = dev_alloc_owned(c, fb);
    c->buf[k].g = gb ? dev_alloc_owned(c, gb) : NULL;
    c->buf[k].g0 = g0b ? (float*)dev_alloc_owned(c, g0b) : NULL;
    // the block storage keeps g beside f in every block
    // the block storages: g_i is the element after f_i; the FP16 blocks keep g_0 at
    // byte 1088 of every block
    if (params->storage == LB_STORAGE_F32_BLOCKED && c->buf[k].f) c->buf[k].g = (float*)c->buf[k].f + 1;
    if (params->storage == LB_STORAGE_F16_BLOCKED && c->buf[k].f) {
      c->buf[k].g = (char*)c->buf[k].f + 2;
      c->buf[k].g0 = (float*)((char*)c->buf[k].f + 1088);
    }
    if (!c->buf[k].f || (gb && !c->buf[k].g) || (g0b && !c->buf[k].g0)) {
      set_err(NULL, "device allocation of the state (%zu bytes) failed", 2 * (fb + gb + g0b));
      lb_destroy(c);
      return LB_ERR_NOMEM;
    }
    // solid nodes are never written by a step: start them (and everything) at 0
    cudaError_t ez = cudaMemsetAsync(c->buf[k].f, 0, fb, c->stream);
    if (ez == cudaSuccess && gb) ez = cudaMemsetAsync(c->buf[k].g, 0, gb, c->stream);
    if (ez == cudaSuccess && g0b) ez = cudaMemsetAsync(c->buf[k].g0, 0, g0b, c->stream);
    if (ez != cudaSuccess) {
      set_err(NULL, "clearing the state failed: %s", cudaGetErrorString(ez));
      lb_destroy(c);
      return LB_ERR_CUDA;
    }
  }
  c->nparts = kRedPartsPerSM * device_sm_count();
  c->partials = (double*)dev_alloc_owned(c, (size_t)c->nparts * RED_PARTS * sizeof(double));
  c->red_out = (double*)dev_alloc_owned(c, 4 * sizeof(double));
  c->errflag = (int*)dev_alloc_owned(c, 256);
  if (c->errflag && cudaMemsetAsync(c->errflag, 0, 256, c->stream) != cudaSuccess) c->errflag = NULL;
  if (!c->partials || !c->red_out || !c->errflag) {
    set_err(NULL, "device allocation failed");
    lb_destroy(c);
    return LB_ERR_NOMEM;
  }
  // solid nodes: the tube's columns outside its band
  c->fluid = (long)grid->nx * grid->ny - (walls->tube_len > 0 ? (long)walls->tube_len * (grid->ny - walls->tube_h) : 0);
  st = default_state(c);
  if (st != LB_OK) {
    snprintf(g_create_err, sizeof g_create_err, "%s", c->err);
    lb_destroy(c);
    return st;
  }
  *out = c;
  return LB_OK;
}

void lb_destroy(lb_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->cap) cudaStreamSynchronize(c->cap);
  drop_graph(c);
  for (void* p : c->owned) dev_free(c, p);
  if (c->cap) cudaStreamDestroy(c->cap);
  delete c;
}

lb_status lb_init_fields(lb_ctx* c, const double* rho, const double* ux, const double* uy, const double* phi) {
  if (!c || !rho || !ux || !uy) return c ? (set_err(c, "NULL field"), LB_ERR_ARG) : LB_ERR_ARG;
  if (c->prm.model == LB_MODEL_BINARY && !phi) return set_err(c, "phi is required for the binary model"), LB_ERR_ARG;
  return upload_and_init(c, rho, ux, uy, c->prm.model == LB_MODEL_BINARY ? phi : NULL);
}

lb_status lb_step(lb_ctx* c, long n) {
  NvtxRange range("lb_step");
  if (!c) return LB_ERR_ARG;
  if (n < 0) return set_err(c, "negative step count"), LB_ERR_ARG;
  if (c->poisoned) return set_err(c, "context holds a non-finite or timed-out state"), LB_ERR_STATE;
  long rem = n;
  if (rem > 0 && c->cur == 1) {
    lb_status st = launch_one(c, c->stream, 1);
    if (st) return st;
    c->cur = 0;
    c->t++;
    rem--;
  }
  if (rem >= kGraphSteps) {
    if (!c->gexec) {
      lb_status st = build_graph(c);
      if (st) return st;
    }
    while (rem >= kGraphSteps) {
      CK(cudaGraphLaunch(c->gexec, c->stream));
      rem -= kGraphSteps;
      c->t += kGraphSteps;
    }
  }
  while (rem > 0) {
    lb_status st = launch_one(c, c->stream, c->cur);
    if (st) return st;
    c->cur ^= 1;
    c->t++;
    rem--;
  }
  return LB_OK;
}

lb_status lb_fields(lb_ctx* c, double* rho, double* ux, double* uy, double* phi) {
  if (!c) return LB_ERR_ARG;
  const size_t N = (size_t)c->grid.nx * c->grid.ny;
  double* d = (double*)dev_alloc(c, 4 * N * sizeof(double));
  if (!d) return set_err(c, "device allocation failed"), LB_ERR_NOMEM;
  OpArgs a = base_args(c);
  a.src = c->buf[c->cur];
  a.out0 = d;
  a.out1 = d + N;
  a.out2 = d + 2 * N;
  a.out3 = d + 3 * N;
  lb_status st = LB_OK;
  cudaError_t e = c->ops(OP_FIELDS, a, c->stream);
  double* dst[4] = {rho, ux, uy, phi};
  for (int k = 0; k < 4 && e == cudaSuccess; ++k)
    if (dst[k]) e = cudaMemcpyAsync(dst[k], d + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e2 = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = e2;
  if (e != cudaSuccess) {
    set_err(c, "lb_fields: %s", cudaGetErrorString(e));
    st = LB_ERR_CUDA;
  }
  dev_free(c, d);
  return st;
}

lb_status lb_filled_length(lb_ctx* c, double* l_centre, double* l_vol, double* mass, double* phi_sum) {
  NvtxRange range("lb_filled_length");
  if (!c) return LB_ERR_ARG;
  OpArgs a = base_args(c);
  a.src = c->buf[c->cur];
  a.nparts = c->nparts;
  a.partials = c->partials;
  a.red_out = c->red_out;
  CK(c->ops(OP_RED_PARTIALS, a, c->stream));
  CK(c->ops(OP_RED_FINAL, a, c->stream));
  double h[4];
  CK(cudaMemcpyAsync(h, c->red_out, sizeof h, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  lb_status dst = check_device_error(c);
  if (dst != LB_OK) return dst;
  if (l_centre) *l_centre = h[0];
  if (l_vol) *l_vol = h[1];
  if (mass) *mass = h[2];
  if (phi_sum) *phi_sum = h[3];
  if (!isfinite(h[2]) || !isfinite(h[3])) {
    c->poisoned = 1;
    set_err(c, "non-finite mass or phi sum at step %ld", c->t);
    return LB_ERR_NONFINITE;
  }
  return LB_OK;
}

lb_status lb_get_populations(lb_ctx* c, double* f, double* g, int rested) {
  if (!c || !f) return c ? (set_err(c, "f is NULL"), LB_ERR_ARG) : LB_ERR_ARG;
  if (c->prm.storage == LB_STORAGE_MOMENTS || c->prm.storage == LB_STORAGE_MOMENTS_F16)
    return set_err(c, "the moment storages keep no populations (lb_get_moments)"), LB_ERR_ARG;
  const size_t N = (size_t)c->grid.nx * c->grid.ny;
  const int bin = c->prm.model == LB_MODEL_BINARY;
  double* d = (double*)dev_alloc(c, (bin ? 18 : 9) * N * sizeof(double));
  if (!d) return set_err(c, "device allocation failed"), LB_ERR_NOMEM;
  OpArgs a = base_args(c);
  a.src = c->buf[c->cur];
  a.flag = rested;
  a.out0 = d;
  a.out1 = bin ? d + 9 * N : NULL;
  cudaError_t e = c->ops(OP_POPS_OUT, a, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(f, d, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess && bin && g)
    e = cudaMemcpyAsync(g, d + 9 * N, 9 * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e2 = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = e2;
  dev_free(c, d);
  if (e != cudaSuccess) return set_err(c, "lb_get_populations: %s", cudaGetErrorString(e)), LB_ERR_CUDA;
  return LB_OK;
}

lb_status lb_set_populations(lb_ctx* c, const double* f, const double* g) {
  if (!c || !f) return c ? (set_err(c, "f is NULL"), LB_ERR_ARG) : LB_ERR_ARG;
  const int bin = c->prm.model == LB_MODEL_BINARY;
  if (bin && !g) return set_err(c, "g is required for the binary model"), LB_ERR_ARG;
  const size_t N = (size_t)c->grid.nx * c->grid.ny;
  double* d = (double*)dev_alloc(c, (bin ? 18 : 9) * N * sizeof(double));
  if (!d) return set_err(c, "device allocation failed"), LB_ERR_NOMEM;
  cudaError_t e = cudaMemcpyAsync(d, f, 9 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  if (e == cudaSuccess && bin) e = cudaMemcpyAsync(d + 9 * N, g, 9 * N * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  OpArgs a = base_args(c);
  a.dst = c->buf[0];
  a.in0 = d;
  a.in1 = bin ? d + 9 * N : NULL;
  if (e == cudaSuccess) e = c->ops(OP_POPS_IN, a, c->stream);
  if (e == cudaSuccess) e = clear_device_error(c);
  cudaError_t e2 = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = e2;
  dev_free(c, d);
  if (e != cudaSuccess) return set_err(c, "lb_set_populations: %s", cudaGetErrorString(e)), LB_ERR_CUDA;
  c->cur = 0;
  c->poisoned = 0;
  return LB_OK;
}

size_t lb_state_bytes(const lb_ctx* c) {
  if (!c) return 0;
  size_t fb, gb, g0b;
  return state_bytes(c->prm.model, c->prm.storage, (size_t)c->grid.nx * c->grid.ny, &fb, &gb, &g0b);
}

// The stored state as the storage holds it: the f planes, then the g planes, then the
// FP32 g_0 plane (FP16 storage), each as in device memory.
lb_status lb_save_state(lb_ctx* c, void* host, size_t bytes) {
  if (!c || !host) return c ? (set_err(c, "host is NULL"), LB_ERR_ARG) : LB_ERR_ARG;
  size_t fb, gb, g0b;
  const size_t total = state_bytes(c->prm.model, c->prm.storage, (size_t)c->grid.nx * c->grid.ny, &fb, &gb, &g0b);
  if (bytes != total) return set_err(c, "bytes must equal lb_state_bytes (%zu)", total), LB_ERR_ARG;
  const OpBufs& b = c->buf[c->cur];
  unsigned char* h = static_cast<unsigned char*>(host);
  CK(cudaMemcpyAsync(h, b.f, fb, cudaMemcpyDeviceToHost, c->stream));
  if (gb) CK(cudaMemcpyAsync(h + fb, b.g, gb, cudaMemcpyDeviceToHost, c->stream));
  if (g0b) CK(cudaMemcpyAsync(h + fb + gb, b.g0, g0b, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return LB_OK;
}

lb_status lb_load_state(lb_ctx* c, const void* host, size_t bytes, long time) {
  if (!c || !host || time < 0) return c ? (set_err(c, "host is NULL or time < 0"), LB_ERR_ARG) : LB_ERR_ARG;
  size_t fb, gb, g0b;
  const size_t total = state_bytes(c->prm.model, c->prm.storage, (size_t)c->grid.nx * c->grid.ny, &fb, &gb, &g0b);
  if (bytes != total) return set_err(c, "bytes must equal lb_state_bytes (%zu)", total), LB_ERR_ARG;
  const OpBufs& b = c->buf[0];
  const unsigned char* h = static_cast<const unsigned char*>(host);
  CK(cudaMemcpyAsync(b.f, h, fb, cudaMemcpyHostToDevice, c->stream));
  if (gb) CK(cudaMemcpyAsync(b.g, h + fb, gb, cudaMemcpyHostToDevice, c->stream));
  if (g0b) CK(cudaMemcpyAsync(b.g0, h + fb + gb, g0b, cudaMemcpyHostToDevice, c->stream));
  CK(clear_device_error(c));
  CK(cudaStreamSynchronize(c->stream));
  c->cur = 0;
  c->t = time;
  c->poisoned = 0;
  return LB_OK;
}

lb_status lb_get_moments(lb_ctx* c, double* m) {
  if (!c || !m) return c ? (set_err(c, "m is NULL"), LB_ERR_ARG) : LB_ERR_ARG;
  const size_t N = (size_t)c->grid.nx * c->grid.ny;
  double* d = (double*)dev_alloc(c, (size_t)M_PLANES * N * sizeof(double));
  if (!d) return set_err(c, "device allocation failed"), LB_ERR_NOMEM;
  OpArgs a = base_args(c);
  a.src = c->buf[c->cur];
  a.out0 = d;
  cudaError_t e = c->ops(OP_MOMENTS_OUT, a, c->stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(m, d, (size_t)M_PLANES * N * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
  cudaError_t e2 = cudaStreamSynchronize(c->stream);
  if (e == cudaSuccess) e = e2;
  dev_free(c, d);
  if (e != cudaSuccess) return set_err(c, "lb_get_moments: %s", cudaGetErrorString(e)), LB_ERR_CUDA;
  return LB_OK;
}

lb_status lb_inject_wait_timeout(lb_ctx* c) {
  if (!c) return LB_ERR_ARG;
  const int one = 1;
  CK(cudaMemcpyAsync(c->errflag, &one, sizeof one, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return LB_OK;
}

lb_status lb_check_report(lb_ctx* c, int* enabled, unsigned long long* bad, unsigned long long* first_bad) {
  if (!c) return LB_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  unsigned long long h[3] = {0, 0, 0};
  OpArgs a = base_args(c);
  a.check_out = h;
  CK(c->ops(OP_CHECK, a, c->stream));
  if (enabled) *enabled = (int)h[0];
  if (bad) *bad = h[1];
  if (first_bad) *first_bad = h[2];
  return LB_OK;
}

lb_status lb_sync(lb_ctx* c) {
  if (!c) return LB_ERR_ARG;
  CK(cudaStreamSynchronize(c->stream));
  return check_device_error(c);
}

lb_status lb_get_kernel(const lb_ctx* c, int* variant) {
  if (!c || !variant) return LB_ERR_ARG;
  if (pull_storage(c->prm.storage)) {
    *variant = 4;
    return LB_OK;
  }
  const int k = c->kernel == 0 ? (staged_ok(c->prm.storage, c->grid.nx, c->grid.ny) ? 2 : 1) : c->kernel;
  *variant = k == 2 && c->deep ? 3 : k;
  return LB_OK;
}

lb_status lb_set_kernel(lb_ctx* c, int variant) {
  if (!c) return LB_ERR_ARG;
  if (pull_storage(c->prm.storage) && variant != 0 && variant != 4)
    return set_err(c, "this storage has one step kernel (variant 4)"), LB_ERR_ARG;
  if (pull_storage(c->prm.storage)) return LB_OK;
  if (variant < 0 || variant > 3) return set_err(c, "kernel variant must be 0, 1, 2 or 3"), LB_ERR_ARG;
  if (variant >= 2 && !staged_ok(c->prm.storage, c->grid.nx, c->grid.ny)) {
    if (c->grid.nx % 8 != 0) return set_err(c, "the staged kernel needs nx %% 8 == 0"), LB_ERR_ARG;
    return set_err(c, "the staged kernel holds at most 477218588 nodes"), LB_ERR_ARG;
  }
  const int kernel = variant == 3 ? 2 : variant;
  const int deep = variant == 3 ? 1 : (variant == 2 ? 0 : c->deep);
  if (kernel != c->kernel || deep != c->deep) {
    CK(cudaStreamSynchronize(c->stream));
    drop_graph(c);
  }
  c->kernel = kernel;
  c->deep = deep;
  return LB_OK;
}

long lb_time(const lb_ctx* c) { return c ? c->t : -1; }

long lb_fluid_nodes(const lb_ctx* c) { return c ? c->fluid : -1; }

lb_status lb_set_tile(lb_ctx* c, int tile_x, int tile_y) {
  if (!c) return LB_ERR_ARG;
  if (tile_x != 64 && tile_x != 128 && tile_x != 256) return set_err(c, "tile_x must be 64, 128 or 256"), LB_ERR_ARG;
  if (tile_y < 1 || tile_y > c->grid.ny) return set_err(c, "tile_y must be in [1, ny]"), LB_ERR_ARG;
  if (tile_x != c->tile_x || tile_y != c->tile_y) {
    CK(cudaStreamSynchronize(c->stream));
    drop_graph(c);
  }
  c->tile_x = tile_x;
  c->tile_y = tile_y;
  return LB_OK;
}

lb_status lb_get_tile(const lb_ctx* c, int* tile_x, int* tile_y) {
  if (!c) return LB_ERR_ARG;
  if (tile_x) *tile_x = c->tile_x;
  if (tile_y) *tile_y = c->tile_y;
  return LB_OK;
}

lb_status lb_autotune(lb_ctx* c, int* tile_x, int* tile_y, double* us_per_step) {
  NvtxRange range("lb_autotune");
  if (!c) return LB_ERR_ARG;
  if (c->poisoned) return LB_ERR_STATE;
  const size_t N = (size_t)c->grid.nx * c->grid.ny;
  size_t fb, gb, g0b;
  const size_t total = state_bytes(c->prm.model, c->prm.storage, N, &fb, &gb, &g0b);
  CK(cudaStreamSynchronize(c->stream));
  // save the current state so that tuning leaves it untouched
  char* save = (char*)dev_alloc(c, total);
  if (!save) return set_err(c, "device allocation failed"), LB_ERR_NOMEM;
  const OpBufs cur = c->buf[c->cur];
  lb_status st = LB_OK;
  cudaError_t e = cudaMemcpyAsync(save, cur.f, fb, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && gb) e = cudaMemcpyAsync(save + fb, cur.g, gb, cudaMemcpyDeviceToDevice, c->stream);
  if (e == cudaSuccess && g0b) e = cudaMemcpyAsync(save + fb + gb, cur.g0, g0b, cudaMemcpyDeviceToDevice, c->stream);
  const int cand_x[3] = {64, 128, 256};
  // band heights: the moment kernel's time depends on how its warps fill the
  // GPU in waves, so it gets a finer set (12 rows suit the FP16 blocks: 57.3
  // against 58.0 us for their best power-of-two band on 16384 x 256)
  const int moments = pull_storage(c->prm.storage);
  const std::vector<int> cand_y = moments ? std::vector<int>{4, 8, 12, 14, 16, 18, 20, 22, 24, 32, 48, 64}
                                          : std::vector<int>{1, 2, 4, 8, 12, 16, 32, 64};
  const int saved_kernel = c->kernel, saved_deep = c->deep;
  int best_x = c->tile_x, best_y = c->tile_y, best_k = saved_kernel, best_d = saved_deep;
  float best = 1e30f;
  cudaEvent_t e0 = NULL, e1 = NULL;
  if (e == cudaSuccess) e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int reps = 10, trials = 3;  // each candidate: best of 3 timings of 10 steps
  // variants: sliding window, staged (shallow ring), staged (deep ring); the staged
  // kernel only where it fits (16-byte aligned rows, 32-bit offsets)
  const int nk = moments ? 1 : (staged_ok(c->prm.storage, c->grid.nx, c->grid.ny) ? 3 : 1);
  for (int ik = 0; ik < nk && e == cudaSuccess && st == LB_OK; ++ik)
  for (int ix = 0; ix < 3 && e == cudaSuccess && st == LB_OK; ++ix)
    for (size_t iy = 0; iy < cand_y.size() && e == cudaSuccess && st == LB_OK; ++iy) {
      if (cand_y[iy] > c->grid.ny) continue;
      if (!moments) {
        c->kernel = ik == 0 ? 1 : 2;
        c->deep = ik == 2;
      }
      c->tile_x = cand_x[ix];
      c->tile_y = cand_y[iy];
      int from = c->cur;
      for (int k = 0; k < 2 && st == LB_OK; ++k, from ^= 1) st = launch_one(c, c->stream, from);
      float ms = 1e30f;
      for (int tr = 0; tr < trials && e == cudaSuccess && st == LB_OK; ++tr) {
        e = cudaEventRecord(e0, c->stream);
        for (int k = 0; k < reps && st == LB_OK; ++k, from ^= 1) st = launch_one(c, c->stream, from);
        if (e == cudaSuccess) e = cudaEventRecord(e1, c->stream);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        float t = 0.f;
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, e0, e1);
        if (e == cudaSuccess && t < ms) ms = t;
      }
      if (e == cudaSuccess && ms < best) {
        best = ms;
        best_x = cand_x[ix];
        best_y = cand_y[iy];
        best_k = c->kernel;
        best_d = c->deep;
      }
    }
  c->kernel = saved_kernel;
  c->deep = saved_deep;
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  // restore
  cudaError_t er = cudaMemcpyAsync(cur.f, save, fb, cudaMemcpyDeviceToDevice, c->stream);
  if (er == cudaSuccess && gb) er = cudaMemcpyAsync(cur.g, save + fb, gb, cudaMemcpyDeviceToDevice, c->stream);
  if (er == cudaSuccess && g0b) er = cudaMemcpyAsync(cur.g0, save + fb + gb, g0b, cudaMemcpyDeviceToDevice, c->stream);
  cudaStreamSynchronize(c->stream);
  dev_free(c, save);
  c->tile_x = best_x;
  c->tile_y = best_y;
  c->kernel = best_k;
  c->deep = best_d;
  drop_graph(c);
  if (st != LB_OK) return st;
  if (e != cudaSuccess || er != cudaSuccess)
    return set_err(c, "lb_autotune: %s", cudaGetErrorString(e != cudaSuccess ? e : er)), LB_ERR_CUDA;
  if (tile_x) *tile_x = best_x;
  if (tile_y) *tile_y = best_y;
  if (us_per_step) *us_per_step = 1000.0 * best / reps;
  return LB_OK;
}

const char* lb_last_error(const lb_ctx* c) { return c ? c->err : g_create_err; }

}  // extern "C"
