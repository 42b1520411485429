// lb_filled_length_noalloc: the FP64 reductions of lb_filled_length for callers
// that cannot allocate device memory.
//
// The first reduction pass writes partials per block (mass, sum of phi, filled
// volume, first meniscus column).  lb_filled_length keeps those partials in
// memory that the context allocated; this entry point keeps them in the
// file-scope array below instead, so it needs no context and calls no
// allocator.  Every GPU that loads the library holds the array
// (LB_NOALLOC_MAX_BLOCKS x 4 doubles) until the process exits.
#include <cuda.h>
#include <cuda_runtime.h>

#include <math.h>

#include <mutex>

#include "lb.h"
#include "lb_aux.cuh"

namespace {

static __device__ __align__(256) double lb_noalloc_partials[LB_NOALLOC_MAX_BLOCKS * lbk::RED_PARTS];

constexpr int kMaxDevices = 256;
std::mutex g_mu;
// Device address of lb_noalloc_partials per device, with the unique ID of the
// context it was looked up in: a module's symbols get new addresses in a new
// context (after cudaDeviceReset, or in a context made current through the
// driver API), so an address is reused only in the context that produced it.
struct ScratchEntry {
  unsigned long long ctx_id;
  double* addr;
};
ScratchEntry g_scratch[kMaxDevices];

// The two driver functions that identify the current context, taken from the
// driver through the runtime (the library does not link the driver library
// itself, so that it still loads on a machine without a GPU driver).
using CtxGetCurrentFn = CUresult (*)(CUcontext*);
using CtxGetIdFn = CUresult (*)(CUcontext, unsigned long long*);
CtxGetCurrentFn g_ctx_get_current;
CtxGetIdFn g_ctx_get_id;

lb_status driver_functions() {  // called with g_mu held
  if (g_ctx_get_current && g_ctx_get_id) return LB_OK;
  void* a = nullptr;
  void* b = nullptr;
  cudaDriverEntryPointQueryResult qa, qb;
  if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
      cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
      qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
    return LB_ERR_CUDA;
  g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
  g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(b);
  return LB_OK;
}

lb_status current_context_id(unsigned long long* id, bool* have) {  // called with g_mu held
  CUcontext ctx = nullptr;
  if (g_ctx_get_current(&ctx) != CUDA_SUCCESS) return LB_ERR_CUDA;
  *have = ctx != nullptr;
  if (ctx && g_ctx_get_id(ctx, id) != CUDA_SUCCESS) return LB_ERR_CUDA;
  return LB_OK;
}

// Resolve the device address of the scratch array in the current context, once
// per (device, context).
lb_status scratch_address(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LB_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  lb_status st = driver_functions();
  if (st != LB_OK) return st;
  unsigned long long id = 0;
  bool have = false;
  st = current_context_id(&id, &have);
  if (st != LB_OK) return st;
  if (!have || !g_scratch[dev].addr || g_scratch[dev].ctx_id != id) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, lb_noalloc_partials) != cudaSuccess || !p) return LB_ERR_CUDA;
    if (!have) {  // the lookup made the device's primary context current
      st = current_context_id(&id, &have);
      if (st != LB_OK || !have) return LB_ERR_CUDA;
    }
    g_scratch[dev].ctx_id = id;
    g_scratch[dev].addr = static_cast<double*>(p);
  }
  *out = g_scratch[dev].addr;
  return LB_OK;
}

template <int MODEL, class S>
cudaError_t reduce(const lbk::Geom& G, const lbk::Buf<S>& B, double rho_l, double rho_g, double thr, int nblocks,
                   double* partials, double* out, cudaStream_t s) {
  lbk::reduce_partials_kernel<MODEL, S><<<nblocks, lbk::RED_THREADS, 0, s>>>(G, B, rho_l, rho_g, thr, partials);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  lbk::reduce_final_kernel<MODEL, S><<<1, 32, 0, s>>>(G, B, thr, nblocks, partials, out);
  return cudaGetLastError();
}

bool geometry_ok(const lb_grid* g, const lb_walls* w) {
  if (g->nx < 3 || g->ny < 3 || (long)g->nx * g->ny > (1L << 31) - 1) return false;
  if (w->tube_len < 0 || w->tube_len > g->nx) return false;
  if (w->tube_len > 0) {
    if (w->tube_x0 < 0 || w->tube_x0 >= g->nx || w->tube_y0 < 0 || w->tube_y0 >= g->ny) return false;
    if (w->tube_h < 2 || w->tube_h >= g->ny) return false;
  }
  return true;
}

}  // namespace

extern "C" lb_status lb_filled_length_noalloc(const lb_grid* grid, const lb_walls* walls, const lb_params* params,
                                              const void* f, const void* g, const void* g0, int nblocks,
                                              double* out, void* stream) {
  if (!grid || !walls || !params || !f || !out) return LB_ERR_ARG;
  if (nblocks < 1 || nblocks > LB_NOALLOC_MAX_BLOCKS) return LB_ERR_ARG;
  if (!geometry_ok(grid, walls)) return LB_ERR_ARG;
  const int bin = params->model == LB_MODEL_BINARY;
  if (!bin && params->model != LB_MODEL_LIQUID_GAS) return LB_ERR_ARG;
  // population storages only (the moment storage keeps no populations); FP16 and the
  // 32-node blocks are binary only
  const int blocked = params->storage == LB_STORAGE_F32_BLOCKED || params->storage == LB_STORAGE_F16_BLOCKED;
  const int st_ok = params->storage == LB_STORAGE_F64 || params->storage == LB_STORAGE_F32 ||
                    (bin && (params->storage == LB_STORAGE_F16DEV || blocked));
  if (!st_ok) return LB_ERR_ARG;
  if (bin && !blocked && !g) return LB_ERR_ARG;
  // the block storages' node limits (as lb_create)
  const unsigned long long n32 = ((unsigned long long)grid->nx * grid->ny + 31) / 32 * 32;
  if (params->storage == LB_STORAGE_F32_BLOCKED && 18ull * n32 >= (1ull << 32)) return LB_ERR_ARG;
  if (params->storage == LB_STORAGE_F16_BLOCKED && 19ull * n32 >= (1ull << 32)) return LB_ERR_ARG;
  if (bin && params->storage == LB_STORAGE_F16DEV && !g0) return LB_ERR_ARG;
  // the liquid fraction of the liquid-gas model divides by rho_l - rho_g
  if (!bin && !(isfinite(params->rho_l) && isfinite(params->rho_g) && params->rho_l > params->rho_g))
    return LB_ERR_ARG;
  double* partials = nullptr;
  lb_status st = scratch_address(&partials);
  if (st != LB_OK) return st;
  const lbk::Geom G{grid->nx, grid->ny, walls->tube_x0, walls->tube_len, walls->tube_y0, walls->tube_h};
  const double thr = bin ? 0.0 : 0.5 * (params->rho_l + params->rho_g);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  float* g0f = static_cast<float*>(const_cast<void*>(g0));
  cudaError_t e = cudaErrorInvalidValue;
  if (!bin && params->storage == LB_STORAGE_F64) {
    lbk::Buf<lbk::SF64> B{(double*)f, nullptr, nullptr};
    e = reduce<lbk::MODEL_LG>(G, B, params->rho_l, params->rho_g, thr, nblocks, partials, out, s);
  } else if (!bin && params->storage == LB_STORAGE_F32) {
    lbk::Buf<lbk::SF32> B{(float*)f, nullptr, nullptr};
    e = reduce<lbk::MODEL_LG>(G, B, params->rho_l, params->rho_g, thr, nblocks, partials, out, s);
  } else if (bin && params->storage == LB_STORAGE_F64) {
    lbk::Buf<lbk::SF64> B{(double*)f, (double*)g, nullptr};
    e = reduce<lbk::MODEL_BINARY>(G, B, params->rho_l, params->rho_g, thr, nblocks, partials, out, s);
  } else if (bin && params->storage == LB_STORAGE_F32) {
    lbk::Buf<lbk::SF32> B{(float*)f, (float*)g, nullptr};
    e = reduce<lbk::MODEL_BINARY>(G, B, params->rho_l, params->rho_g, thr, nblocks, partials, out, s);
  } else if (bin && params->storage == LB_STORAGE_F16DEV) {
    // the stored deviations are taken from the bulk rest weights of this lattice's A
    lbk::Buf<lbk::SF16> B{(__half*)f, (__half*)g, g0f, lbk::rest_offsets_binary(params->A)};
    e = reduce<lbk::MODEL_BINARY>(G, B, params->rho_l, params->rho_g, thr, nblocks, partials, out, s);
  } else if (bin && params->storage == LB_STORAGE_F32_BLOCKED) {
    // g_i is the element after f_i in every block
    float* ff = static_cast<float*>(const_cast<void*>(f));
    lbk::Buf<lbk::SF32B> B{ff, ff + lbk::SF32B::kGOff, nullptr};
    e = reduce<lbk::MODEL_BINARY>(G, B, params->rho_l, params->rho_g, thr, nblocks, partials, out, s);
  } else if (bin && params->storage == LB_STORAGE_F16_BLOCKED) {
    // g_i is the half after f_i and g_0 an FP32 run at byte 1088 of every block
    __half* fh = static_cast<__half*>(const_cast<void*>(f));
    lbk::Buf<lbk::SF16B> B{fh, fh + lbk::SF16B::kGOff, reinterpret_cast<float*>(fh) + lbk::SF16B::kG0,
                           lbk::rest_offsets_binary(params->A)};
    e = reduce<lbk::MODEL_BINARY>(G, B, params->rho_l, params->rho_g, thr, nblocks, partials, out, s);
  } else {
    return LB_ERR_ARG;
  }
  return e == cudaSuccess ? LB_OK : LB_ERR_CUDA;
}
