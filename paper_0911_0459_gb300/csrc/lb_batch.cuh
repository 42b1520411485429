// Batched capillaries: one persistent kernel advances every capillary of a
// sweep.  The lattices live in one arena (two buffers); a flat list of tiles
// (capillary, column block, row band) covers all of them.  Each CTA processes
// its own list of tiles (balanced on the host) every time step, then waits at
// a grid barrier before the next step.  The launch is cooperative, so all CTAs
// are resident; the barrier still gives up after a time limit, records
// LB_ERR_TIMEOUT in the error word and every CTA returns.
#pragma once

#include "lb_aux.cuh"
#include "lb_device.cuh"
#include "lb_moment.cuh"
#include "lb_step_tma.cuh"

namespace lbk {

template <typename A>
struct CapDesc {
  Geom G;
  Phys<A> P;
  size_t off_f;     // offset of this lattice's f planes in a buffer's f arena (elements)
  size_t off_g;     // offset of its g planes in the g arena
  size_t off_g0;    // offset of its g_0 plane (FP16 storage)
  Rest r;           // its FP16 deviation offsets
  MomPhys Q;        // its moment-collision constants (moment storage)
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
  const TileDesc* tiles;  // CTA k takes tiles[start[k] .. start[k + 1]) every step
  const int* start;
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
  if constexpr (std::is_same<S, SF32B>::value)  // g_i after f_i in every 32-node block
    return Buf<S>{f + c.off_f, f + c.off_f + SF32B::kGOff, nullptr, c.r};
  if constexpr (std::is_same<S, SF16B>::value)  // g_i after f_i, g_0 apart, in every 32-node block
    return Buf<S>{f + c.off_f, f + c.off_f + SF16B::kGOff, reinterpret_cast<float*>(f + c.off_f) + SF16B::kG0, c.r};
  return Buf<S>{f + c.off_f, g ? g + c.off_g : nullptr, g0 ? g0 + c.off_g0 : nullptr, c.r};
}

template <class S, int BX>
__global__ void __launch_bounds__(BX) batch_step_kernel(BatchArgs<S> a) {
  __shared__ StepSmem<MODEL_BINARY, S, BX> sm;
  for (int s = 0; s < a.nsteps; ++s) {
    const bool fromA = ((a.parity + s) & 1) == 0;
    for (int t = a.start[blockIdx.x]; t < a.start[blockIdx.x + 1]; ++t) {
      const TileDesc td = a.tiles[t];
      const CapDesc<typename S::A> c = a.caps[td.cap];
      const Buf<S> src = fromA ? cap_buf<S>(a.fa, a.ga, a.g0a, c) : cap_buf<S>(a.fb, a.gb, a.g0b, c);
      const Buf<S> dst = fromA ? cap_buf<S>(a.fb, a.gb, a.g0b, c) : cap_buf<S>(a.fa, a.ga, a.g0a, c);
      step_band<MODEL_BINARY, S, BX, true>(c.G, c.P, c.Q, src, dst, td.xb, td.y0, td.y1, sm);
      __syncthreads();
    }
    if (!grid_barrier(a.bar, a.expected, a.limit_ns)) {
      if (threadIdx.x == 0) atomicExch(a.err, 1);
      return;
    }
  }
}

// Grid barrier of the staged batch kernel: every thread passes in whether its
// own work failed; a failure anywhere sets the error word before the CTA
// arrives, and every CTA reads the word after the barrier, so that all of them
// leave at the same step.  Returns false when the CTA must stop.
__device__ __forceinline__ bool grid_barrier_checked(GridBarrier* b, unsigned int expected,
                                                     unsigned long long limit_ns, bool failed, int* err) {
  __shared__ int ok_sh;
  const int any = __syncthreads_or(failed ? 1 : 0);
  if (threadIdx.x == 0) {
    if (any) atomicExch(err, 1);
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
          atomicExch(err, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
    if (*(volatile int*)err != 0) ok = 0;
    ok_sh = ok;
  }
  __syncthreads();
  return ok_sh != 0;
}

// The staged update (bulk copies into a shared-memory ring by a producer warp,
// BX/32 consumer warps) over the batch's tiles.  The ring's row counter runs on
// across tiles and steps, so the producer keeps copying while the consumers
// finish the previous tile.  Every lattice's nx is a multiple of 8 (the copies'
// 16-byte alignment).  Per-node arithmetic is the single-lattice kernels', so
// results are bitwise those of lb_step with the staged kernel.
// Resident CTAs per SM of the staged batch body: those of the single-lattice
// kernel, except that the FP16 block storage keeps 80 registers per thread (its
// batch body, which also walks the tile list, spilled at 72: 46.4 instead of
// 43.6 GLUPS on the 256-capillary sweep with one CTA fewer per SM).
template <class S, int BX, int NS>
constexpr int batch_min_blocks() {
  if constexpr (std::is_same<S, SF16B>::value) {
    using L = TmaLayout<MODEL_BINARY, S, BX, NS>;
    constexpr int by_smem = int(233472 / (L::BYTES + 1024));
    constexpr int by_regs = 65536 / ((BX + 32) * 80);
    constexpr int b = by_smem < by_regs ? by_smem : by_regs;
    return b < 1 ? 1 : (b > 8 ? 8 : b);
  } else {
    return tma_min_blocks_of<MODEL_BINARY, S, BX, NS>();
  }
}

template <class S, int BX, int NS>
__global__ void __launch_bounds__(BX + 32, (batch_min_blocks<S, BX, NS>())) batch_tma_kernel(BatchArgs<S> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Ring<MODEL_BINARY, S, BX, NS> R = ring_init<MODEL_BINARY, S, BX, NS>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool producer = warp == BX / 32;
  unsigned k = 0, issued = 0;
  bool ok = true;
  for (int s = 0; s < a.nsteps; ++s) {
    const bool fromA = ((a.parity + s) & 1) == 0;
    if (producer && lane == 0) {
      // bulk copies read through the async proxy what other CTAs stored through
      // the generic proxy before the grid barrier
      asm volatile("fence.proxy.async.global;" ::: "memory");
    }
    for (int t = a.start[blockIdx.x]; t < a.start[blockIdx.x + 1]; ++t) {
      const TileDesc td = a.tiles[t];
      const CapDesc<typename S::A>& c = a.caps[td.cap];
      if (ok) {
        if (producer) {
          if (lane == 0) {
            const Buf<S> src = fromA ? cap_buf<S>(a.fa, a.ga, a.g0a, c) : cap_buf<S>(a.fb, a.gb, a.g0b, c);
            ok = produce_tile<MODEL_BINARY, S, BX, NS>(R, c.G, src, td.xb, td.y0, td.y1, k, issued);
          }
        } else {
          const Buf<S> dst = fromA ? cap_buf<S>(a.fb, a.gb, a.g0b, c) : cap_buf<S>(a.fa, a.ga, a.g0a, c);
          // a value copy: the per-node arithmetic then compiles as in the single-lattice
          // kernel (parameters that live behind a pointer the pushes might alias led the
          // compiler to fuse multiply-adds differently, a last-bit difference)
          const Phys<typename S::A> P = c.P;
          if constexpr (TmaLayout<MODEL_BINARY, S, BX, NS>::BLK) {
            ok = c.G.nx % 32 != 0
                     ? consume_tile<MODEL_BINARY, S, BX, NS, true>(R, c.G, P, c.Q, dst, td.xb, td.y0, td.y1, k, warp, lane)
                     : consume_tile<MODEL_BINARY, S, BX, NS, false>(R, c.G, P, c.Q, dst, td.xb, td.y0, td.y1, k, warp, lane);
          } else {
            ok = consume_tile<MODEL_BINARY, S, BX, NS>(R, c.G, P, c.Q, dst, td.xb, td.y0, td.y1, k, warp, lane);
          }
        }
      }
      k += (unsigned)(td.y1 - td.y0 + 2);
      // only k mod 2 NS (stage and phase) and whether k >= NS matter: keep the
      // counter small so that long runs cannot wrap it
      if (k >= 4 * NS) {
        const unsigned shift = (k - 2 * NS) / (2 * NS) * (2 * NS);
        k -= shift;
        issued = issued >= shift ? issued - shift : 0;
      }
    }
    if (!grid_barrier_checked(a.bar, a.expected, a.limit_ns, !ok, a.err)) break;
  }
  if (producer && lane == 0) drain_ring<MODEL_BINARY, S, BX, NS>(R, issued);
}

// The moment storage over the batch's tiles: each warp of a CTA advances its
// 30-column strip of the tile (the single-lattice moment kernel's strip), read
// through L2 since other CTAs wrote the state earlier in the same launch.
template <int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 2 : (NW == 4 ? 5 : 10)) batch_moment_kernel(BatchArgs<SM32> a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int s = 0; s < a.nsteps; ++s) {
    const bool fromA = ((a.parity + s) & 1) == 0;
    for (int t = a.start[blockIdx.x]; t < a.start[blockIdx.x + 1]; ++t) {
      const TileDesc td = a.tiles[t];
      const CapDesc<float>& c = a.caps[td.cap];
      const float* src = (fromA ? a.fa : a.fb) + c.off_f;
      float* dst = (fromA ? a.fb : a.fa) + c.off_f;
      moment_strip<true, SM32>(c.G, c.Q, src, dst, td.xb + warp * kMomCols, td.y0, td.y1, lane);
    }
    if (!grid_barrier(a.bar, a.expected, a.limit_ns)) {
      if (threadIdx.x == 0) atomicExch(a.err, 1);
      return;
    }
  }
}

// Reductions of every lattice (mass, sum of phi, filled volume, l), in two
// passes so that large lattices do not serialise on one block.  The nodes of
// each lattice are cut into chunks of consecutive node indices; pass 1 gives
// every chunk a block and writes its three partial sums, pass 2 gives every
// lattice a block that adds its chunks' partials in chunk order (the result does
// not depend on scheduling) and finds l from the centre line.
struct RedChunk {
  int cap;     // lattice
  int n0, n1;  // node range [n0, n1) of the lattice
};

template <class S>
__global__ void __launch_bounds__(RED_THREADS) batch_partials_kernel(const CapDesc<typename S::A>* caps,
                                                                     const RedChunk* chunks, typename S::T* f,
                                                                     typename S::T* g, float* g0, double* part) {
  using A = typename S::A;
  const RedChunk ch = chunks[blockIdx.x];
  const CapDesc<A> c = caps[ch.cap];
  const Geom& G = c.G;
  const Buf<S> B = cap_buf<S>(f, g, g0, c);
  const size_t N = (size_t)G.nx * G.ny;
  RedAcc ra;
  for (int n = ch.n0 + threadIdx.x; n < ch.n1; n += blockDim.x) {
    const int x = n % G.nx, y = n / G.nx;
    if (is_solid(G, x, y)) continue;
    red_add_node<MODEL_BINARY, S>(G, B, N, (size_t)n, x, y, ra);
  }
  const double acc[3] = {ra.mass, ra.phi, finish_volume<MODEL_BINARY>(ra, 0.0, 0.0)};
  __shared__ double sh[3][RED_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 3; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) sh[k][wid] = v;
  }
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < RED_THREADS / 32; ++w) s += sh[threadIdx.x][w];
    part[(size_t)blockIdx.x * 3 + threadIdx.x] = s;
  }
}

// Pass 2: one block per lattice.  range[c] = {first chunk, number of chunks}.
// out[c * 4 + k] or, with a sample column, out[(c * nsamples + col) * 4 + k].
template <class S>
__global__ void __launch_bounds__(1024) batch_final_kernel(const CapDesc<typename S::A>* caps, const int2* range,
                                                           int ncaps, typename S::T* f, typename S::T* g,
                                                           float* g0, const double* part, int nsamples, int col,
                                                           double* out) {
  using A = typename S::A;
  const int ci = blockIdx.x;
  if (ci >= ncaps) return;
  const CapDesc<A> c = caps[ci];
  const Geom& G = c.G;
  const Buf<S> B = cap_buf<S>(f, g, g0, c);
  const size_t N = (size_t)G.nx * G.ny;
  __shared__ int first;
  if (threadIdx.x == 0) first = INT_MAX;
  __syncthreads();
  const int L = G.tube_len;
  for (int k = threadIdx.x; k < L; k += blockDim.x) {
    const double c0 = centre_value<MODEL_BINARY, S>(G, B, N, k, c.thr);
    bool hit = false;
    if (k == 0 && !(c0 > 0.0)) hit = true;
    if (!hit && k + 1 < L && c0 > 0.0) hit = !(centre_value<MODEL_BINARY, S>(G, B, N, k + 1, c.thr) > 0.0);
    if (hit) atomicMin(&first, k);
  }
  // warp 0 adds the lattice's chunk partials: lane j takes chunks j, j + 32, ...
  // in order, then a fixed shuffle tree (independent of scheduling)
  __shared__ double tot[3];
  if (threadIdx.x < 32) {
    const int2 r = range[ci];
    double t[3] = {0.0, 0.0, 0.0};
    for (int j = threadIdx.x; j < r.y; j += 32)
      for (int k = 0; k < 3; ++k) t[k] += part[(size_t)(r.x + j) * 3 + k];
    for (int k = 0; k < 3; ++k) {
      const double v = warp_sum(t[k]);
      if (threadIdx.x == 0) tot[k] = v;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
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
