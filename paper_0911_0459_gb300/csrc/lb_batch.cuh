// Batched capillaries: one persistent kernel advances every capillary of a
// sweep.  The lattices live in one arena (two buffers); a flat list of tiles
// (capillary, column block, row band) covers all of them.  Each CTA processes
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... of a time step with the
// sliding-window band update, then waits at a grid barrier before the next
// step.  The launch is cooperative, so all CTAs are resident; the barrier still
// gives up after a time limit, records LB_ERR_TIMEOUT in the error word and
// every CTA returns.
#pragma once

#include "lb_aux.cuh"
#include "lb_device.cuh"
#include "lb_step_tma.cuh"

namespace lbk {

template <typename A>
struct CapDesc {
  Geom G;
  Phys<A> P;
  size_t off_f;     // offset of this lattice's f planes in a buffer's f arena (elements)
  size_t off_g;     // offset of its g planes in the g arena
  size_t off_g0;    // offset of its g_0 plane (FP16 storage)
  double thr, rho_l, rho_g;
};

struct TileDesc {
  int cap, xb, y0, y1;
};

struct GridBarrier {
  unsigned int count;
  unsigned int gen;
};

// All CTAs arrive; returns false (in every thread of the CTA) when the barrier
// did not complete within limit_ns.  extra: arrivals that never come, so that a
// test can make the wait run out.
__device__ __forceinline__ bool grid_barrier(GridBarrier* b, unsigned int expected, unsigned long long limit_ns) {
  __shared__ int ok_sh;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = &b->gen;
    const unsigned int g = *vgen;
    __threadfence();
    const unsigned int arrived = atomicAdd(&b->count, 1u);
    int ok = 1;
    if (arrived == expected - 1) {
      atomicExch(&b->count, 0u);
      __threadfence();
      atomicAdd(&b->gen, 1u);
    } else {
      const unsigned long long t0 = globaltimer_ns();
      while (*vgen == g) {
        if (globaltimer_ns() - t0 > limit_ns) {
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

template <class S>
struct BatchArgs {
  const CapDesc<typename S::A>* caps;
  const TileDesc* tiles;
  int ntiles;
  typename S::T* fa;   // buffer A: f planes of every lattice
  typename S::T* ga;
  float* g0a;
  typename S::T* fb;   // buffer B
  typename S::T* gb;
  float* g0b;
  int nsteps;
  int parity;          // 0: A holds the current state
  GridBarrier* bar;
  unsigned int expected;
  unsigned long long limit_ns;
  int* err;
};

template <class S>
__device__ __forceinline__ Buf<S> cap_buf(typename S::T* f, typename S::T* g, float* g0,
                                          const CapDesc<typename S::A>& c) {
  return Buf<S>{f + c.off_f, g + c.off_g, g0 ? g0 + c.off_g0 : nullptr};
}

template <class S, int BX>
__global__ void __launch_bounds__(BX) batch_step_kernel(BatchArgs<S> a) {
  __shared__ StepSmem<MODEL_BINARY, S, BX> sm;
  for (int s = 0; s < a.nsteps; ++s) {
    const bool fromA = ((a.parity + s) & 1) == 0;
    for (int t = blockIdx.x; t < a.ntiles; t += gridDim.x) {
      const TileDesc td = a.tiles[t];
      const CapDesc<typename S::A> c = a.caps[td.cap];
      const Buf<S> src = fromA ? cap_buf<S>(a.fa, a.ga, a.g0a, c) : cap_buf<S>(a.fb, a.gb, a.g0b, c);
      const Buf<S> dst = fromA ? cap_buf<S>(a.fb, a.gb, a.g0b, c) : cap_buf<S>(a.fa, a.ga, a.g0a, c);
      step_band<MODEL_BINARY, S, BX, true>(c.G, c.P, src, dst, td.xb, td.y0, td.y1, sm);
      __syncthreads();
    }
    if (!grid_barrier(a.bar, a.expected, a.limit_ns)) {
      if (threadIdx.x == 0) atomicExch(a.err, 1);
      return;
    }
  }
}

// One block per lattice: mass, sum of phi, filled volume and l (as in
// reduce_partials/reduce_final, for every lattice of the batch).  out[c * 4 + k]
// or, with a sample column, out[(c * nsamples + col) * 4 + k].
template <class S>
__global__ void __launch_bounds__(1024) batch_reduce_kernel(const CapDesc<typename S::A>* caps, int ncaps,
                                                            typename S::T* f, typename S::T* g, float* g0,
                                                            int nsamples, int col, double* out) {
  using A = typename S::A;
  const int ci = blockIdx.x;
  if (ci >= ncaps) return;
  const CapDesc<A> c = caps[ci];
  const Geom& G = c.G;
  const Buf<S> B = cap_buf<S>(f, g, g0, c);
  const size_t N = (size_t)G.nx * G.ny;
  double acc[3] = {0.0, 0.0, 0.0};
  for (size_t n = threadIdx.x; n < N; n += blockDim.x) {
    const int x = (int)(n % G.nx), y = (int)(n / G.nx);
    if (is_solid(G, x, y)) continue;
    A fv[9], gv[9];
    load_node<MODEL_BINARY, S, true>(B, N, n, fv, gv);
    double r = 0.0, p = 0.0;
    for (int i = 0; i < 9; ++i) r += (double)fv[i];
    for (int i = 0; i < 9; ++i) p += (double)gv[i];
    acc[0] += r;
    acc[1] += p;
    if (G.tube_len > 0 && col_in_tube(G, x) && row_in_band(G, y)) acc[2] += 0.5 * (p + 1.0);
  }
  __shared__ double sh[3][32];
  __shared__ int first;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (threadIdx.x == 0) first = INT_MAX;
  for (int k = 0; k < 3; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) sh[k][wid] = v;
  }
  __syncthreads();
  const int L = G.tube_len;
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    const double c0 = centre_value<MODEL_BINARY, S>(G, B, N, k, c.thr);
    bool hit = false;
    if (k == 0 && !(c0 > 0.0)) hit = true;
    if (!hit && k + 1 < L && c0 > 0.0) hit = !(centre_value<MODEL_BINARY, S>(G, B, N, k + 1, c.thr) > 0.0);
    if (hit) atomicMin(&first, k);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot[3];
    for (int k = 0; k < 3; ++k) {
      double s = 0.0;
      for (int w = 0; w < (int)(blockDim.x + 31) / 32; ++w) s += sh[k][w];
      tot[k] = s;
    }
    double l;
    if (L <= 0) {
      l = 0.0;
    } else if (first == INT_MAX) {
      l = (double)L;
    } else {
      const int k = first;
      const double c0 = centre_value<MODEL_BINARY, S>(G, B, N, k, c.thr);
      l = (k == 0 && !(c0 > 0.0)) ? 0.0 : k + c0 / (c0 - centre_value<MODEL_BINARY, S>(G, B, N, k + 1, c.thr));
    }
    double* o = out + ((size_t)ci * nsamples + col) * 4;
    o[0] = l;
    o[1] = L > 0 ? tot[2] / G.tube_h : 0.0;
    o[2] = tot[0];
    o[3] = tot[1];
  }
}

}  // namespace lbk
