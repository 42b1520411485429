// Host-side, type-erased interface between the C ABI (lb_capi.cu) and the
// kernel instantiations (one translation unit per model x storage).
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stddef.h>

namespace lbk {

// The staged step kernel reads 16-byte-aligned rows (nx % 8 == 0) and stores at
// 32-bit element offsets (9 planes of nx * ny nodes below 2^32).
inline bool staged_fits(int nx, int ny) {
  return nx % 8 == 0 && 9ull * (unsigned long long)nx * (unsigned long long)ny < (1ull << 32);
}

// Streaming multiprocessors of the current device (queried once per device;
// 152 on GB300, but nothing assumes it).
inline int device_sm_count() {
  static int cache[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 1;
  if (cache[dev] <= 0) {
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) return 1;
    cache[dev] = n;
  }
  return cache[dev];
}

// An NVTX range around a host call (named in timelines of profilers; a no-op
// when no tool is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

enum OpKind { OP_STEP, OP_INIT, OP_FIELDS, OP_POPS_OUT, OP_POPS_IN, OP_RED_PARTIALS, OP_RED_FINAL, OP_MOMENTS_OUT,
              OP_CHECK };

struct OpBufs {
  void* f;
  void* g;
  float* g0;
};

struct OpArgs {
  // geometry
  int nx, ny, tube_x0, tube_len, tube_y0, tube_h;
  // physics (converted to the arithmetic type by the instantiation)
  double kappa, a, b, T, Acoef, M, nu_l, nu_g, nu, lambda_scale, h;
  double lut;  // viscosity table steps K - 1 (0: exact)
  double rho_l, rho_g, thr;
  // buffers
  OpBufs src, dst;
  // step tile and kernel variant (0: sliding window, 1: bulk-copy staged)
  int bx, yc;
  int staged;
  int deep;      // staged kernel: 0 = shallow ring (more CTAs per SM), 1 = deeper ring
  int* err;      // device error word (a device-side wait gave up)
  // field / population / reduction arguments (device pointers)
  const double *in0, *in1, *in2, *in3;
  int in_cols;   // OP_INIT: in0..in3 hold one value per column (every row alike)
  double *out0, *out1, *out2, *out3;  // OP_MOMENTS_OUT: out0 holds 6 planes
  int flag;      // rested flag for OP_POPS_OUT
  int nparts;    // reduction partial blocks
  double* partials;
  double* red_out;
  unsigned long long* check_out;  // OP_CHECK: host array {enabled, bad accesses, first bad index + 1}
};

typedef cudaError_t (*OpsFn)(OpKind, const OpArgs&, cudaStream_t);

cudaError_t ops_lg_f64(OpKind, const OpArgs&, cudaStream_t);
cudaError_t ops_lg_f32(OpKind, const OpArgs&, cudaStream_t);
cudaError_t ops_bin_f64(OpKind, const OpArgs&, cudaStream_t);
cudaError_t ops_bin_f32(OpKind, const OpArgs&, cudaStream_t);
cudaError_t ops_bin_f16(OpKind, const OpArgs&, cudaStream_t);
cudaError_t ops_bin_m32(OpKind, const OpArgs&, cudaStream_t);  // moment storage
cudaError_t ops_bin_m16(OpKind, const OpArgs&, cudaStream_t);  // FP16 moments, FP32 phi
cudaError_t ops_bin_g32(OpKind, const OpArgs&, cudaStream_t);  // f and phi (g eliminated)
cudaError_t ops_bin_f32b(OpKind, const OpArgs&, cudaStream_t);  // FP32 populations in 32-node blocks
cudaError_t ops_bin_f16b(OpKind, const OpArgs&, cudaStream_t);  // FP16 deviations in 32-node blocks

}  // namespace lbk
