// Launch wrappers of every kernel for one (model, storage) pair.
#pragma once

#include "lb_aux.cuh"
#include "lb_device.cuh"
#include "lb_ops.h"
#include "lb_step_tma.cuh"

namespace lbk {

template <class S>
static Buf<S> to_buf(const OpBufs& b, const OpArgs& a) {
  return Buf<S>{(typename S::T*)b.f, (typename S::T*)b.g, b.g0, rest_offsets_binary(a.Acoef)};
}

static inline Geom to_geom(const OpArgs& a) {
  return Geom{a.nx, a.ny, a.tube_x0, a.tube_len, a.tube_y0, a.tube_h};
}

template <typename A>
static Phys<A> to_phys(const OpArgs& a) {
  Phys<A> p;
  p.kappa = A(a.kappa); p.a = A(a.a); p.b = A(a.b); p.T = A(a.T);
  p.Acoef = A(a.Acoef); p.M = A(a.M); p.nu_l = A(a.nu_l); p.nu_g = A(a.nu_g);
  p.nu = A(a.nu); p.lambda_scale = A(a.lambda_scale); p.h = A(a.h);
  p.lut = A(a.lut);
  p.lut_inv = a.lut > 0 ? A(1.0 / a.lut) : A(0);
  p.omega = A(2.0 / (6.0 * a.nu + 1.0));
  return p;
}

// Blocks of a 1-D step grid: column blocks x row bands (see tile_of_block).
static inline unsigned tiles_1d(int ncb, int ny, int yc) {
  return (unsigned)ncb * (unsigned)((ny + yc - 1) / yc);
}

// Grid of a grid-stride kernel over n items: at most 16 blocks per SM of the
// current device.
static inline int grid_for(size_t n, int threads) {
  const size_t cap = 16 * (size_t)device_sm_count();
  size_t b = (n + threads - 1) / threads;
  return (int)(b > cap ? cap : (b < 1 ? 1 : b));
}

template <int MODEL, class S, int BX>
static cudaError_t launch_step(const OpArgs& a, cudaStream_t s) {
  StepArgs<MODEL, S> k;
  k.G = to_geom(a);
  k.P = to_phys<typename S::A>(a);
  k.Q = mom_phys(a.kappa, a.Acoef, a.M, a.nu_l, a.nu_g, a.lambda_scale, a.h, a.lut);
  k.src = to_buf<S>(a.src, a);
  k.dst = to_buf<S>(a.dst, a);
  k.yc = a.yc;
  const unsigned grid = tiles_1d((a.nx + BX - 1) / BX, a.ny, a.yc);
  step_kernel<MODEL, S, BX><<<grid, BX, 0, s>>>(k);
  return cudaGetLastError();
}

template <int MODEL, class S, int BX, int NS>
static cudaError_t launch_staged(const OpArgs& a, cudaStream_t s) {
  using L = TmaLayout<MODEL, S, BX, NS>;
  static bool configured = false;  // dynamic shared memory opt-in, once per process
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(step_tma_kernel<MODEL, S, BX, NS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L::BYTES);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  TmaArgs<MODEL, S> k;
  k.G = to_geom(a);
  k.P = to_phys<typename S::A>(a);
  k.Q = mom_phys(a.kappa, a.Acoef, a.M, a.nu_l, a.nu_g, a.lambda_scale, a.h, a.lut);
  k.src = to_buf<S>(a.src, a);
  k.dst = to_buf<S>(a.dst, a);
  k.yc = a.yc;
  k.err = a.err;
  const unsigned grid = tiles_1d((a.nx + BX - 1) / BX, a.ny, a.yc);
  step_tma_kernel<MODEL, S, BX, NS><<<grid, BX + 32, L::BYTES, s>>>(k);
  return cudaGetLastError();
}

template <int NW, class S>
static cudaError_t launch_moment(const OpArgs& a, cudaStream_t s) {
  MomArgs k;
  k.G = to_geom(a);
  k.Q = mom_phys(a.kappa, a.Acoef, a.M, a.nu_l, a.nu_g, a.lambda_scale, a.h, a.lut);
  k.src = a.src.f;
  k.dst = a.dst.f;
  k.yc = a.yc;
  const unsigned grid = tiles_1d((a.nx + NW * kMomCols - 1) / (NW * kMomCols), a.ny, a.yc);
  moment_step_kernel<NW, S><<<grid, NW * 32, 0, s>>>(k);
  return cudaGetLastError();
}

template <int MODEL, class S>
cudaError_t ops_impl(OpKind op, const OpArgs& a, cudaStream_t s) {
  using A = typename S::A;
  const Geom G = to_geom(a);
  const size_t N = (size_t)a.nx * a.ny;
  if constexpr (is_moments<S>::value) {
    static_assert(MODEL == MODEL_BINARY, "the moment storage holds the binary model");
    if (op == OP_STEP) {
      if (a.bx == 64) return launch_moment<2, S>(a, s);
      if (a.bx == 128) return launch_moment<4, S>(a, s);
      if (a.bx == 256) return launch_moment<8, S>(a, s);
      return cudaErrorInvalidValue;
    }
    // the moment storages keep no populations (g eliminated keeps f and phi)
    if (op == OP_POPS_OUT && pull_kind<S>::value != 2) return cudaErrorNotSupported;
  }
  switch (op) {
    case OP_STEP:
      if constexpr (!is_moments<S>::value) {
        if (a.staged) {
          if ((!is_blocked<S>::value && !staged_fits(a.nx, a.ny)) || !a.err) return cudaErrorInvalidValue;
          if (a.bx == 64) return a.deep ? launch_staged<MODEL, S, 64, 8>(a, s) : launch_staged<MODEL, S, 64, 4>(a, s);
          if (a.bx == 128) return a.deep ? launch_staged<MODEL, S, 128, 6>(a, s) : launch_staged<MODEL, S, 128, 4>(a, s);
          if (a.bx == 256) return a.deep ? launch_staged<MODEL, S, 256, 4>(a, s) : launch_staged<MODEL, S, 256, 3>(a, s);
          return cudaErrorInvalidValue;
        }
        if (a.bx == 64) return launch_step<MODEL, S, 64>(a, s);
        if (a.bx == 128) return launch_step<MODEL, S, 128>(a, s);
        if (a.bx == 256) return launch_step<MODEL, S, 256>(a, s);
      }
      return cudaErrorInvalidValue;
    case OP_INIT:
      init_kernel<MODEL, S><<<grid_for(N, 256), 256, 0, s>>>(G, to_phys<A>(a), to_buf<S>(a.dst, a), a.in0, a.in1,
                                                              a.in2, a.in3, a.in_cols ? size_t(0) : size_t(a.nx));
      return cudaGetLastError();
    case OP_FIELDS:
      fields_kernel<MODEL, S><<<grid_for(N, 256), 256, 0, s>>>(G, to_buf<S>(a.src, a), a.out0, a.out1, a.out2, a.out3);
      return cudaGetLastError();
    case OP_POPS_OUT:
      if constexpr (!is_moments<S>::value || pull_kind<S>::value == 2)
        pops_out_kernel<MODEL, S><<<grid_for(N, 256), 256, 0, s>>>(G, to_buf<S>(a.src, a), a.flag, a.out0, a.out1);
      return cudaGetLastError();
    case OP_MOMENTS_OUT:
      moments_out_kernel<MODEL, S><<<grid_for(N, 256), 256, 0, s>>>(G, to_buf<S>(a.src, a), a.out0);
      return cudaGetLastError();
    case OP_POPS_IN:
      pops_in_kernel<MODEL, S><<<grid_for(N, 256), 256, 0, s>>>(G, to_buf<S>(a.dst, a), a.in0, a.in1);
      return cudaGetLastError();
    case OP_RED_PARTIALS:
      reduce_partials_kernel<MODEL, S><<<a.nparts, RED_THREADS, 0, s>>>(G, to_buf<S>(a.src, a), a.rho_l, a.rho_g, a.thr,
                                                                        a.partials);
      return cudaGetLastError();
    case OP_CHECK:
      return read_check_counters(a.check_out);
    case OP_RED_FINAL:
      reduce_final_kernel<MODEL, S><<<1, 32, 0, s>>>(G, to_buf<S>(a.src, a), a.thr, a.nparts, a.partials, a.red_out);
      return cudaGetLastError();
  }
  return cudaErrorInvalidValue;
}

}  // namespace lbk
