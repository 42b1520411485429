// Device code of the fused D2Q9 free-energy MRT step (stencils + equilibria +
// collision + streaming + walls) for sm_103a.
//
// Layout: structure of arrays, plane i of f at f + i*N (N = nx*ny), node (x, y)
// at y*nx + x.  A CTA owns BX consecutive columns and a band of rows; it walks
// up the band with a 4-slot ring of rho/phi rows in shared memory (the 3x3
// stencils of Eq. (best) need rows y-1, y, y+1) while the populations of the
// next two rows are already in flight in registers.  Post-collision populations
// are pushed to r + e_i in the other buffer; a push into a solid node returns
// to the source node in the opposite direction (bounce-back, Sec. 2.2).  The
// stored state is the post-streaming state before the boundary-node rest rule;
// that rule (Sec. 2.2) is applied when a boundary node is next read, which
// leaves rho unchanged and therefore leaves the stencils unchanged.
//
// Collision: with S = diag(0,1,1,0,1,0,1,w,w) (App. A) every mode except the
// two stress modes pxx, pxy relaxes fully, so f - M^-1 S M (f - f^eq) equals
// f^eq + (1 - w) M^-1 (0,...,0, dm_xx, dm_xy) with dm the stress-mode
// non-equilibrium; the columns of M^-1 for those modes are (row of M)/4.
#pragma once

#include <type_traits>

#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbk {

enum { MODEL_LG = 0, MODEL_BINARY = 1 };

struct Geom {
  int nx, ny;
  int tube_x0, tube_len;  // tube columns [x0, x0 + len) mod nx; len == 0: no solid
  int tube_y0, tube_h;    // fluid band [y0, y0 + h) mod ny inside the tube
};

template <typename A>
struct Phys {
  A kappa, a, b, T;    // van der Waals (Sec. 2)
  A Acoef, M;          // phi^4 coefficient and mobility (Sec. 3.1)
  A nu_l, nu_g;        // Eq. (nu)
  A nu;                // liquid-gas viscosity
  A lambda_scale;      // lambda = lambda_scale * nu_local
  A h;                 // wall gradient of the wetted field
  A lut, lut_inv;      // viscosity table of App. A: K - 1 steps (0: exact nu) and 1 / (K - 1)
  A omega;             // liquid-gas: 2 / (6 nu + 1) (Eq. (omega)), for the FP64 pair-form collision
};

// ---------------------------------------------------------- bounds checks
//
// Debug build (-DLB_CHECK): every global load and store of the step kernels
// checks its element index against its buffer.  An index outside records
// itself in two device words of the translation unit (a count and the first
// offending index + 1) and the access is skipped (a load gives 0); nothing
// traps.  In the normal build the checks compile to nothing.
#ifdef LB_CHECK
static __device__ unsigned long long lb_check_hits;
static __device__ unsigned long long lb_check_first;
__device__ __forceinline__ bool lb_in(unsigned long long idx, unsigned long long lim) {
  if (idx < lim) return true;
  atomicAdd(&lb_check_hits, 1ull);
  atomicCAS(&lb_check_first, 0ull, idx + 1);
  return false;
}
#define LB_GUARD(idx, lim, ret)                                                       \
  do {                                                                                \
    if (!::lbk::lb_in((unsigned long long)(idx), (unsigned long long)(lim))) return ret; \
  } while (0)
#else
#define LB_GUARD(idx, lim, ret) \
  do {                          \
  } while (0)
#endif

// Host side: read and clear this translation unit's counters into
// out = {enabled, bad accesses, first bad index + 1}.
inline cudaError_t read_check_counters(unsigned long long* out) {
#ifdef LB_CHECK
  unsigned long long h = 0, f = 0, z = 0;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&h, lb_check_hits, sizeof h);
  if (e == cudaSuccess) e = cudaMemcpyFromSymbol(&f, lb_check_first, sizeof f);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(lb_check_hits, &z, sizeof z);
  if (e == cudaSuccess) e = cudaMemcpyToSymbol(lb_check_first, &z, sizeof z);
  out[0] = 1;
  out[1] = h;
  out[2] = f;
  return e;
#else
  out[0] = out[1] = out[2] = 0;
  return cudaSuccess;
#endif
}

// ------------------------------------------------------------------ storage

// Offsets of the FP16 deviation storage: f_i is stored as f_i - w_i rho0 with
// rho0 = 1 and w_i the rest weights of Eq. (equilibrium) for the bulk phases,
// i.e. f^eq at rest and without gradients, where P0 = p0(rho0, phi = +-1):
// w_0 = 1 - 5 P0 / 3, w_1..4 = P0 / 3, w_5..8 = P0 / 12 (the standard 4/9,
// 1/9, 1/36 when P0 = rho0 / 3).  Unused by the other storages.
struct Rest {
  float w0, w1, w5;
};
__device__ __forceinline__ float rest_w(const Rest& r, int i) { return i == 0 ? r.w0 : (i < 5 ? r.w1 : r.w5); }
// Binary model: p0 = rho/3 + A (-phi^2/2 + 3 phi^4/4) = 1/3 + A/4 at rho0 = 1, phi = +-1.
inline Rest rest_offsets_binary(double A) {
  const double P0 = 1.0 / 3.0 + 0.25 * A;
  return Rest{float(1.0 - 5.0 * P0 / 3.0), float(P0 / 3.0), float(P0 / 12.0)};
}

struct SF64 {
  using T = double;
  using A = double;
  __device__ static A pf(const T* f, int W, int c, int i, const Rest&) { return f[i * W + c]; }
  __device__ static A pg(const T* g, const float*, int W, int c, int i) { return g[i * W + c]; }
  __device__ static A lf(const T* __restrict__ f, size_t N, size_t n, int i, const Rest&) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __ldg(f + i * N + n);
  }
  __device__ static void sf(T* __restrict__ f, size_t N, size_t n, int i, A v, const Rest&) {
    LB_GUARD(i * N + n, 9 * N, );
    f[i * N + n] = v;
  }
  __device__ static A lg(const T* __restrict__ g, const float* __restrict__, size_t N, size_t n, int i) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __ldg(g + i * N + n);
  }
  __device__ static void sg(T* __restrict__ g, float* __restrict__, size_t N, size_t n, int i, A v) {
    LB_GUARD(i * N + n, 9 * N, );
    g[i * N + n] = v;
  }
  // L2-coherent loads, for buffers written earlier in the same launch
  __device__ static A lfc(const T* f, size_t N, size_t n, int i, const Rest&) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __ldcg(f + i * N + n);
  }
  __device__ static A lgc(const T* g, const float*, size_t N, size_t n, int i) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __ldcg(g + i * N + n);
  }
  // stores at 32-bit element offsets (node n of plane i at i * N + n; needs 9N < 2^32)
  __device__ static void sfo(T* __restrict__ f, uint32_t N, uint32_t n, int i, A v, const Rest&) {
    LB_GUARD((unsigned long long)i * N + n, 9ull * N, );
    f[i * N + n] = v;
  }
  __device__ static void sgo(T* __restrict__ g, float* __restrict__, uint32_t N, uint32_t n, int i, A v) {
    LB_GUARD((unsigned long long)i * N + n, 9ull * N, );
    g[i * N + n] = v;
  }
  // zero bits at f_i of node n (a solid node, as in a fresh buffer)
  __device__ static void zf(T* __restrict__ f, size_t N, size_t n, int i) {
    LB_GUARD(i * N + n, 9 * N, );
    f[i * N + n] = T(0);
  }
};

struct SF32 {
  using T = float;
  using A = float;
  __device__ static A pf(const T* f, int W, int c, int i, const Rest&) { return f[i * W + c]; }
  __device__ static A pg(const T* g, const float*, int W, int c, int i) { return g[i * W + c]; }
  __device__ static A lf(const T* __restrict__ f, size_t N, size_t n, int i, const Rest&) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __ldg(f + i * N + n);
  }
  __device__ static void sf(T* __restrict__ f, size_t N, size_t n, int i, A v, const Rest&) {
    LB_GUARD(i * N + n, 9 * N, );
    f[i * N + n] = v;
  }
  __device__ static A lg(const T* __restrict__ g, const float* __restrict__, size_t N, size_t n, int i) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __ldg(g + i * N + n);
  }
  __device__ static void sg(T* __restrict__ g, float* __restrict__, size_t N, size_t n, int i, A v) {
    LB_GUARD(i * N + n, 9 * N, );
    g[i * N + n] = v;
  }
  __device__ static A lfc(const T* f, size_t N, size_t n, int i, const Rest&) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __ldcg(f + i * N + n);
  }
  __device__ static A lgc(const T* g, const float*, size_t N, size_t n, int i) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __ldcg(g + i * N + n);
  }
  __device__ static void sfo(T* __restrict__ f, uint32_t N, uint32_t n, int i, A v, const Rest&) {
    LB_GUARD((unsigned long long)i * N + n, 9ull * N, );
    f[i * N + n] = v;
  }
  __device__ static void sgo(T* __restrict__ g, float* __restrict__, uint32_t N, uint32_t n, int i, A v) {
    LB_GUARD((unsigned long long)i * N + n, 9ull * N, );
    g[i * N + n] = v;
  }
  // zero bits at f_i of node n (a solid node, as in a fresh buffer)
  __device__ static void zf(T* __restrict__ f, size_t N, size_t n, int i) {
    LB_GUARD(i * N + n, 9 * N, );
    f[i * N + n] = T(0);
  }
};

struct SF16 {
  using T = __half;
  using A = float;
  // plain loads (shared memory): planes of W elements
  __device__ static A pf(const T* f, int W, int c, int i, const Rest& r) {
    return __half2float(f[i * W + c]) + rest_w(r, i);
  }
  __device__ static A pg(const T* g, const float* g0, int W, int c, int i) {
    return i == 0 ? g0[c] : __half2float(g[(i - 1) * W + c]);
  }
  __device__ static A lf(const T* __restrict__ f, size_t N, size_t n, int i, const Rest& r) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __half2float(__ldg(f + i * N + n)) + rest_w(r, i);
  }
  __device__ static void sf(T* __restrict__ f, size_t N, size_t n, int i, A v, const Rest& r) {
    LB_GUARD(i * N + n, 9 * N, );
    f[i * N + n] = __float2half_rn(v - rest_w(r, i));
  }
  __device__ static A lfc(const T* f, size_t N, size_t n, int i, const Rest& r) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __half2float(__ldcg(f + i * N + n)) + rest_w(r, i);
  }
  __device__ static A lgc(const T* g, const float* g0, size_t N, size_t n, int i) {
    LB_GUARD(i == 0 ? n : (i - 1) * N + n, i == 0 ? N : 8 * N, A(0));
    return i == 0 ? __ldcg(g0 + n) : __half2float(__ldcg(g + (i - 1) * N + n));
  }
  // g_1..g_8 in FP16 planes 0..7; g_0 (which carries phi) in an FP32 plane.
  __device__ static A lg(const T* __restrict__ g, const float* __restrict__ g0, size_t N, size_t n, int i) {
    LB_GUARD(i == 0 ? n : (i - 1) * N + n, i == 0 ? N : 8 * N, A(0));
    return i == 0 ? __ldg(g0 + n) : __half2float(__ldg(g + (i - 1) * N + n));
  }
  __device__ static void sg(T* __restrict__ g, float* __restrict__ g0, size_t N, size_t n, int i, A v) {
    LB_GUARD(i == 0 ? n : (i - 1) * N + n, i == 0 ? N : 8 * N, );
    if (i == 0)
      g0[n] = v;
    else
      g[(i - 1) * N + n] = __float2half_rn(v);
  }
  __device__ static void sfo(T* __restrict__ f, uint32_t N, uint32_t n, int i, A v, const Rest& r) {
    LB_GUARD((unsigned long long)i * N + n, 9ull * N, );
    f[i * N + n] = __float2half_rn(v - rest_w(r, i));
  }
  __device__ static void sgo(T* __restrict__ g, float* __restrict__ g0, uint32_t N, uint32_t n, int i, A v) {
    LB_GUARD(i == 0 ? (unsigned long long)n : (unsigned long long)(i - 1) * N + n, i == 0 ? N : 8ull * N, );
    if (i == 0)
      g0[n] = v;
    else
      g[(i - 1) * N + n] = __float2half_rn(v);
  }
  // the stored deviations f_i - w_i themselves (the population kernels compute in
  // deviations for this storage)
  __device__ static A pfr(const T* f, int W, int c, int i) { return __half2float(f[i * W + c]); }
  __device__ static A lfr(const T* __restrict__ f, size_t N, size_t n, int i) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __half2float(__ldg(f + i * N + n));
  }
  __device__ static A lfcr(const T* f, size_t N, size_t n, int i) {
    LB_GUARD(i * N + n, 9 * N, A(0));
    return __half2float(__ldcg(f + i * N + n));
  }
  __device__ static void sfr(T* __restrict__ f, size_t N, size_t n, int i, A v) {
    LB_GUARD(i * N + n, 9 * N, );
    f[i * N + n] = __float2half_rn(v);
  }
  __device__ static void sfor(T* __restrict__ f, uint32_t N, uint32_t n, int i, A v) {
    LB_GUARD((unsigned long long)i * N + n, 9ull * N, );
    f[i * N + n] = __float2half_rn(v);
  }
  __device__ static void zf(T* __restrict__ f, size_t N, size_t n, int i) {
    LB_GUARD(i * N + n, 9 * N, );
    f[i * N + n] = __float2half_rn(0.0f);
  }
};

// FP32 populations of the binary model in blocks of 32 consecutive nodes: block
// b = n / 32 holds, for i = 0..8, the pairs (f_i, g_i) of its 32 nodes in node
// order, so f_i of node n is element 576 b + 64 i + 2 (n % 32) of the buffer and
// g_i the element after it (Buf::g = Buf::f + 1).  A node's f_i and g_i always
// stream to the same destination and direction, so the step kernels load and
// store them as one 8-byte pair.  With nx % 32 == 0 the nodes of a row segment
// of whole blocks, all eighteen populations, are one contiguous range, which the
// staged step kernel copies with a single bulk copy per row (other widths: the
// whole blocks over the segment, and one more block at an x-wrap).  The last
// block is padded to 32 nodes.  Same values and arithmetic as SF32.
struct SF32B {
  using T = float;
  using A = float;
  static constexpr int kBlock = 576;       // elements per block of 32 nodes
  static constexpr int kBlockBytes = 2304;
  static constexpr int kGOff = 1;          // g_i is the element after f_i
  static constexpr int kG0 = 0;            // (g_0 pairs with f_0)
  __device__ static size_t at(size_t n, int i) { return (n >> 5) * kBlock + 64 * i + 2 * (n & 31); }
  __device__ static uint32_t at32(uint32_t n, int i) { return (n >> 5) * kBlock + 64 * i + 2 * (n & 31); }
  // elements of a state of N nodes (the last block padded)
  __device__ static unsigned long long lim(unsigned long long N) { return 18ull * ((N + 31) & ~31ull); }
  // shared-memory stage of whole blocks: stage column c lies in block c / 32
  __device__ static int sat(int c, int i) { return (c >> 5) * kBlock + 64 * i + 2 * (c & 31); }
  __device__ static A pf(const T* f, int, int c, int i, const Rest&) { return f[sat(c, i)]; }
  __device__ static A pg(const T* g, const float*, int, int c, int i) { return g[sat(c, i)]; }
  // the pair (f_i, g_i) of stage column c in one load (f: the stage's f base)
  __device__ static void pfg(const T* f, const float*, int c, int i, A& fv, A& gv) {
    const float2 v = *reinterpret_cast<const float2*>(f + sat(c, i));
    fv = v.x;
    gv = v.y;
  }
  __device__ static A lf(const T* __restrict__ f, size_t N, size_t n, int i, const Rest&) {
    LB_GUARD(at(n, i), lim(N), A(0));
    return __ldg(f + at(n, i));
  }
  __device__ static void sf(T* __restrict__ f, size_t N, size_t n, int i, A v, const Rest&) {
    LB_GUARD(at(n, i), lim(N), );
    f[at(n, i)] = v;
  }
  __device__ static A lg(const T* __restrict__ g, const float* __restrict__, size_t N, size_t n, int i) {
    LB_GUARD(at(n, i), lim(N) - 1, A(0));
    return __ldg(g + at(n, i));
  }
  __device__ static void sg(T* __restrict__ g, float* __restrict__, size_t N, size_t n, int i, A v) {
    LB_GUARD(at(n, i), lim(N) - 1, );
    g[at(n, i)] = v;
  }
  __device__ static A lfc(const T* f, size_t N, size_t n, int i, const Rest&) {
    LB_GUARD(at(n, i), lim(N), A(0));
    return __ldcg(f + at(n, i));
  }
  __device__ static A lgc(const T* g, const float*, size_t N, size_t n, int i) {
    LB_GUARD(at(n, i), lim(N) - 1, A(0));
    return __ldcg(g + at(n, i));
  }
  // 32-bit element offsets (needs 18 * 32 * ceil(N / 32) < 2^32)
  __device__ static void sfo(T* __restrict__ f, uint32_t N, uint32_t n, int i, A v, const Rest&) {
    LB_GUARD(at32(n, i), lim(N), );
    f[at32(n, i)] = v;
  }
  __device__ static void sgo(T* __restrict__ g, float* __restrict__, uint32_t N, uint32_t n, int i, A v) {
    LB_GUARD(at32(n, i), lim(N) - 1, );
    g[at32(n, i)] = v;
  }
  __device__ static void zf(T* __restrict__ f, size_t N, size_t n, int i) {
    LB_GUARD(at(n, i), lim(N), );
    f[at(n, i)] = 0.0f;
  }
};

// The FP16 deviations of SF16 in blocks of 32 consecutive nodes: block b = n / 32
// is 1216 bytes (608 halves): f_0 - w_0 of its 32 nodes (FP16, halves 0..31), then
// for i = 1..8 the pairs (f_i - w_i, g_i) of its nodes in node order (FP16,
// halves 32..543), then g_0 (FP32, floats 272..303).  So f_i of node n is half
// 608 b + n % 32 (i = 0) or 608 b + 32 + 64 (i - 1) + 2 (n % 32) (i >= 1) of the
// buffer, g_i (i >= 1) the half after it (Buf::g = Buf::f + 1 half) and g_0 float
// 304 b + 272 + n % 32 (Buf::g0 = Buf::f + 1088 bytes).  A row segment of whole
// blocks is again one contiguous range, which the staged kernel copies with one
// bulk copy per row, and the pairs take one 4-byte load or store.  The last
// block is padded to 32 nodes.  Same values and arithmetic as SF16.
struct SF16B {
  using T = __half;
  using A = float;
  static constexpr int kBlock = 608;       // halves per block of 32 nodes
  static constexpr int kBlockBytes = 1216;
  static constexpr int kGOff = 1;          // g_i (i >= 1) is the half after f_i
  static constexpr int kG0 = 272;          // floats from a block's start to its g_0
  static constexpr int kG0Stride = 304;    // floats per block
  __device__ static int off(int r, int i) { return i == 0 ? r : 32 + 64 * (i - 1) + 2 * r; }
  __device__ static size_t at(size_t n, int i) { return (n >> 5) * kBlock + off((int)(n & 31), i); }
  __device__ static uint32_t at32(uint32_t n, int i) { return (n >> 5) * kBlock + off((int)(n & 31), i); }
  __device__ static size_t at0(size_t n) { return (n >> 5) * kG0Stride + (n & 31); }
  // halves of a state of N nodes (the last block padded)
  __device__ static unsigned long long lim(unsigned long long N) { return 19ull * ((N + 31) & ~31ull); }
  __device__ static unsigned long long lim0(unsigned long long N) { return lim(N) / 2 - kG0; }
  // shared-memory stage of whole blocks: stage column c lies in block c / 32
  __device__ static int sat(int c, int i) { return (c >> 5) * kBlock + off(c & 31, i); }
  __device__ static A pf(const T* f, int, int c, int i, const Rest& r) { return __half2float(f[sat(c, i)]) + rest_w(r, i); }
  __device__ static A pfr(const T* f, int, int c, int i) { return __half2float(f[sat(c, i)]); }
  __device__ static A pg(const T* g, const float* g0, int, int c, int i) {
    return i == 0 ? g0[(c >> 5) * kG0Stride + (c & 31)] : __half2float(g[sat(c, i)]);
  }
  // the pair (f_i - w_i, g_i), i >= 1, of stage column c in one load (f: the
  // stage's f base)
  __device__ static void pfg(const T* f, const float*, int c, int i, A& fv, A& gv) {
    const float2 v = __half22float2(*reinterpret_cast<const __half2*>(f + sat(c, i)));
    fv = v.x;
    gv = v.y;
  }
  __device__ static A lf(const T* __restrict__ f, size_t N, size_t n, int i, const Rest& r) {
    LB_GUARD(at(n, i), lim(N), A(0));
    return __half2float(__ldg(f + at(n, i))) + rest_w(r, i);
  }
  __device__ static A lfr(const T* __restrict__ f, size_t N, size_t n, int i) {
    LB_GUARD(at(n, i), lim(N), A(0));
    return __half2float(__ldg(f + at(n, i)));
  }
  __device__ static A lfc(const T* f, size_t N, size_t n, int i, const Rest& r) {
    LB_GUARD(at(n, i), lim(N), A(0));
    return __half2float(__ldcg(f + at(n, i))) + rest_w(r, i);
  }
  __device__ static A lfcr(const T* f, size_t N, size_t n, int i) {
    LB_GUARD(at(n, i), lim(N), A(0));
    return __half2float(__ldcg(f + at(n, i)));
  }
  __device__ static void sf(T* __restrict__ f, size_t N, size_t n, int i, A v, const Rest& r) {
    LB_GUARD(at(n, i), lim(N), );
    f[at(n, i)] = __float2half_rn(v - rest_w(r, i));
  }
  __device__ static void sfr(T* __restrict__ f, size_t N, size_t n, int i, A v) {
    LB_GUARD(at(n, i), lim(N), );
    f[at(n, i)] = __float2half_rn(v);
  }
  __device__ static A lg(const T* __restrict__ g, const float* __restrict__ g0, size_t N, size_t n, int i) {
    if (i == 0) {
      LB_GUARD(at0(n), lim0(N), A(0));
      return __ldg(g0 + at0(n));
    }
    LB_GUARD(at(n, i), lim(N) - kGOff, A(0));
    return __half2float(__ldg(g + at(n, i)));
  }
  __device__ static A lgc(const T* g, const float* g0, size_t N, size_t n, int i) {
    if (i == 0) {
      LB_GUARD(at0(n), lim0(N), A(0));
      return __ldcg(g0 + at0(n));
    }
    LB_GUARD(at(n, i), lim(N) - kGOff, A(0));
    return __half2float(__ldcg(g + at(n, i)));
  }
  __device__ static void sg(T* __restrict__ g, float* __restrict__ g0, size_t N, size_t n, int i, A v) {
    if (i == 0) {
      LB_GUARD(at0(n), lim0(N), );
      g0[at0(n)] = v;
      return;
    }
    LB_GUARD(at(n, i), lim(N) - kGOff, );
    g[at(n, i)] = __float2half_rn(v);
  }
  // 32-bit element offsets (needs 19 * 32 * ceil(N / 32) < 2^32)
  __device__ static void sfo(T* __restrict__ f, uint32_t N, uint32_t n, int i, A v, const Rest& r) {
    LB_GUARD(at32(n, i), lim(N), );
    f[at32(n, i)] = __float2half_rn(v - rest_w(r, i));
  }
  __device__ static void sfor(T* __restrict__ f, uint32_t N, uint32_t n, int i, A v) {
    LB_GUARD(at32(n, i), lim(N), );
    f[at32(n, i)] = __float2half_rn(v);
  }
  __device__ static void sgo(T* __restrict__ g, float* __restrict__ g0, uint32_t N, uint32_t n, int i, A v) {
    if (i == 0) {
      const uint32_t o = (n >> 5) * kG0Stride + (n & 31);
      LB_GUARD(o, lim0(N), );
      g0[o] = v;
      return;
    }
    LB_GUARD(at32(n, i), lim(N) - kGOff, );
    g[at32(n, i)] = __float2half_rn(v);
  }
  __device__ static void zf(T* __restrict__ f, size_t N, size_t n, int i) {
    LB_GUARD(at(n, i), lim(N), );
    f[at(n, i)] = __float2half_rn(0.0f);
  }
};

// Population storages in 32-node blocks (one bulk copy per staged row).
template <class S>
struct is_blocked {
  static constexpr bool value = std::is_same<S, SF32B>::value || std::is_same<S, SF16B>::value;
};

// Population storages whose step kernels compute in deviations from the stored
// rest offsets (the FP16 storages): raw loads and stores, collide_node_f16.
template <class S>
struct dev_arith {
  static constexpr bool value = std::is_same<S, SF16>::value || std::is_same<S, SF16B>::value;
};

template <class S>
struct Buf {
  typename S::T* f;
  typename S::T* g;
  float* g0;
  Rest r;  // FP16 deviation offsets of this lattice
};

// ----------------------------------------------------------------- geometry

__device__ __forceinline__ bool col_in_tube(const Geom& G, int x) {
  int d = x - G.tube_x0;
  if (d < 0) d += G.nx;
  return d < G.tube_len;
}
__device__ __forceinline__ bool row_in_band(const Geom& G, int y) {
  int d = y - G.tube_y0;
  if (d < 0) d += G.ny;
  return d < G.tube_h;
}
__device__ __forceinline__ bool is_solid(const Geom& G, int x, int y) {
  return G.tube_len > 0 && col_in_tube(G, x) && !row_in_band(G, y);
}
__device__ __forceinline__ int wrapi(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Step launches use a 1-D grid over (column block, row band) tiles, column blocks
// fastest: a 2-D grid would limit the bands to 65535 (gridDim.y), while the tile
// count stays below nx * ny < 2^31.  ncb = number of column blocks.
__device__ __forceinline__ void tile_of_block(int ncb, int& cb, int& band) {
  band = (int)(blockIdx.x / (unsigned)ncb);
  cb = (int)blockIdx.x - band * ncb;
}

// Solid flags of the 3x3 neighbourhood of (x, y), s[j][i] <-> offset (i-1, j-1).
__device__ __forceinline__ void neighbour_solids(const Geom& G, int x, int y, bool s[3][3], bool& any) {
  bool tc[3], rb[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    tc[k] = G.tube_len > 0 && col_in_tube(G, wrapi(x + k - 1, G.nx));
    rb[k] = row_in_band(G, wrapi(y + k - 1, G.ny));
  }
  any = false;
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      s[j][i] = tc[i] && !rb[j];
      any = any || s[j][i];
    }
}

// Ghost values for solid neighbours (wetting condition of Sec. 2.2): mirror
// through the fluid node; across a y-facing wall the mirror value is lowered by
// 2h so that the centred normal derivative equals h.  Mirror nodes are fluid
// for every geometry the host accepts.
template <typename A>
__device__ __forceinline__ void apply_ghosts(A v[3][3], const bool s[3][3], A h) {
  A out[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      out[j][i] = v[j][i];
      if (!s[j][i]) continue;
      if (j == 1)
        out[j][i] = v[1][2 - i];                       // end face: neutral
      else if (i == 1)
        out[j][i] = v[2 - j][1] - A(2) * h;            // wall row
      else if (!s[2 - j][i])
        out[j][i] = v[2 - j][i] - A(2) * h;            // corner, y-mirror
      else
        out[j][i] = v[j][2 - i];                       // corner, x-mirror
    }
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) v[j][i] = out[j][i];
}

// Eq. (best): isotropic gradient and Laplacian on the 3x3 neighbourhood.
template <typename A>
__device__ __forceinline__ void stencil3(const A v[3][3], A& dx, A& dy, A& lap) {
  dx = ((v[0][2] - v[0][0]) + A(4) * (v[1][2] - v[1][0]) + (v[2][2] - v[2][0])) * A(1.0 / 12.0);
  dy = ((v[2][0] + A(4) * v[2][1] + v[2][2]) - (v[0][0] + A(4) * v[0][1] + v[0][2])) * A(1.0 / 12.0);
  lap = ((v[0][0] + v[0][2] + v[2][0] + v[2][2]) + A(4) * (v[0][1] + v[1][0] + v[1][2] + v[2][1]) -
         A(20) * v[1][1]) * A(1.0 / 6.0);
}

// ------------------------------------------------------------- equilibria

// f^eq_1..8 of Eq. (equilibrium), grouped by direction; f^eq_0 = rho - sum.
template <typename A>
__device__ __forceinline__ void feq9(A rho, A jx, A jy, A ux, A uy, A P0, A kap, A gpx, A gpy, A grx,
                                     A gry, A lam, A fe[9]) {
  const A udr = ux * grx + uy * gry;
  const A Txx = jx * ux + lam * (A(2) * ux * grx + udr);
  const A Tyy = jy * uy + lam * (A(2) * uy * gry + udr);
  const A Txy = jx * uy + lam * (ux * gry + uy * grx);
  const A tr3 = (Txx + Tyy) * A(1.0 / 3.0);
  const A ax = A(1.5) * (Txx - tr3);
  const A ay = A(1.5) * (Tyy - tr3);
  const A dp = A(1.5) * (Txx + Tyy + A(2) * Txy - tr3);
  const A dm = A(1.5) * (Txx + Tyy - A(2) * Txy - tr3);
  const A Gxx = kap * gpx * gpx, Gyy = kap * gpy * gpy, Gxy = kap * gpx * gpy;
  const A k13 = Gxx * A(1.0 / 3.0) - Gyy * A(1.0 / 6.0);
  const A k24 = Gyy * A(1.0 / 3.0) - Gxx * A(1.0 / 6.0);
  const A kd = -(Gxx + Gyy) * A(1.0 / 24.0);
  const A kxy = Gxy * A(0.25);
  fe[1] = (P0 + jx + ax) * A(1.0 / 3.0) + k13;
  fe[2] = (P0 - jx + ax) * A(1.0 / 3.0) + k13;
  fe[3] = (P0 + jy + ay) * A(1.0 / 3.0) + k24;
  fe[4] = (P0 - jy + ay) * A(1.0 / 3.0) + k24;
  fe[5] = (P0 + jx + jy + dp) * A(1.0 / 12.0) + kd + kxy;
  fe[6] = (P0 - jx - jy + dp) * A(1.0 / 12.0) + kd + kxy;
  fe[7] = (P0 - jx + jy + dm) * A(1.0 / 12.0) + kd - kxy;
  fe[8] = (P0 + jx - jy + dm) * A(1.0 / 12.0) + kd - kxy;
  fe[0] = rho - (((fe[1] + fe[2]) + (fe[3] + fe[4])) + ((fe[5] + fe[6]) + (fe[7] + fe[8])));
}

// g^eq of Appendix A (dt = 1).
template <typename A>
__device__ __forceinline__ void geq9(A phi, A ux, A uy, A Q, A ge[9]) {
  const A u2 = (ux * ux + uy * uy) * A(1.0 / 3.0);
  const A px = phi * ux, py = phi * uy;
  const A sx = A(1.5) * phi * (ux * ux - u2);
  const A sy = A(1.5) * phi * (uy * uy - u2);
  const A upp = ux + uy, ump = ux - uy;
  const A sp = A(1.5) * phi * (upp * upp - u2);
  const A sm = A(1.5) * phi * (ump * ump - u2);
  ge[1] = (Q + px + sx) * A(1.0 / 3.0);
  ge[2] = (Q - px + sx) * A(1.0 / 3.0);
  ge[3] = (Q + py + sy) * A(1.0 / 3.0);
  ge[4] = (Q - py + sy) * A(1.0 / 3.0);
  ge[5] = (Q + px + py + sp) * A(1.0 / 12.0);
  ge[6] = (Q - px - py + sp) * A(1.0 / 12.0);
  ge[7] = (Q - px + py + sm) * A(1.0 / 12.0);
  ge[8] = (Q + px - py + sm) * A(1.0 / 12.0);
  ge[0] = phi - (((ge[1] + ge[2]) + (ge[3] + ge[4])) + ((ge[5] + ge[6]) + (ge[7] + ge[8])));
}

template <typename A>
__device__ __forceinline__ A sum9(const A v[9]) {
  return v[0] + (((v[1] + v[2]) + (v[3] + v[4])) + ((v[5] + v[6]) + (v[7] + v[8])));
}
template <typename A>
__device__ __forceinline__ A momx(const A f[9]) { return (f[1] - f[2]) + ((f[5] - f[6]) - (f[7] - f[8])); }
template <typename A>
__device__ __forceinline__ A momy(const A f[9]) { return (f[3] - f[4]) + ((f[5] - f[6]) + (f[7] - f[8])); }

// Rest rule of Sec. 2.2 at a boundary node: f_i -= w_i e_i . j (w = 1/3, 1/12)
// removes the momentum and keeps the density.
template <typename A>
__device__ __forceinline__ void rest(A f[9]) {
  const A jx = momx(f), jy = momy(f);
  const A a = jx * A(1.0 / 3.0), b = jy * A(1.0 / 3.0);
  const A c = (jx + jy) * A(1.0 / 12.0), d = (jy - jx) * A(1.0 / 12.0);
  f[1] -= a; f[2] += a; f[3] -= b; f[4] += b;
  f[5] -= c; f[6] += c; f[7] -= d; f[8] += d;
}

// Local viscosity, Eq. (nu), with (phi + 1)/2 clamped to [0, 1]; with the table of
// App. A, the nearest of its evenly spaced viscosities.
template <typename A>
__device__ __forceinline__ A local_nu_binary(const Phys<A>& P, A phi) {
  A c = (phi + A(1)) * A(0.5);
  c = c < A(0) ? A(0) : (c > A(1) ? A(1) : c);
  if (P.lut > A(0)) c = rint(c * P.lut) * P.lut_inv;
  // explicit fused multiply-add: the same rounding in every kernel that inlines this
  return fma(c, P.nu_l - P.nu_g, P.nu_g);
}

// Lattice velocities (Sec. 2.1, c = 1) as compile-time functions of i.
__host__ __device__ constexpr int EXd(int i) { return (i == 1 || i == 5 || i == 8) ? 1 : ((i == 2 || i == 6 || i == 7) ? -1 : 0); }
__host__ __device__ constexpr int EYd(int i) { return (i == 3 || i == 5 || i == 7) ? 1 : ((i == 4 || i == 6 || i == 8) ? -1 : 0); }
__host__ __device__ constexpr int OPPd(int i) { return i == 0 ? 0 : ((i & 1) ? i + 1 : i - 1); }

// Reciprocal, correctly rounded (equal to 1/v) in both precisions.
__device__ __forceinline__ float rcp_rn(float v) { return __frcp_rn(v); }
__device__ __forceinline__ double rcp_rn(double v) { return 1.0 / v; }

// Hardware reciprocal (relative error below 2^-22), for 1/rho and omega.
__device__ __forceinline__ float rcp_fast(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// ---------------------------------------------------------------- collision

// Constants of the collision, with the stencils' normalisations folded in: the
// gradient stencils enter as 12 x the gradient and the Laplacian as 6 x the
// Laplacian (see stencil_rows).
struct MomPhys {
  float A;          // phi^4 coefficient (Sec. 3.1)
  float nkap6;      // -kappa / 6: -kappa lap = nkap6 (6 lap)
  float kap144;     // kappa / 144: kappa (d phi)^2 = kap144 (12 d phi)^2
  float lam12;      // lambda_scale / 12: lambda u . d rho = (lam12 nu) u . (12 d rho)
  float nu_g, dnu;  // Eq. (nu): nu = nu_g + c (nu_l - nu_g)
  float M3, M12;    // 2M/3 and 2M/12, g^eq's mobility terms (App. A)
  float h;          // wall gradient d_n phi|_b
  float lut, lut_inv;
  float p0off;      // -A / 4: P0 of the FP16 deviation storage's rest offsets (P0 = 1/3 + A/4) less 1/3
};

inline MomPhys mom_phys(double kappa, double A, double M, double nu_l, double nu_g, double lambda_scale, double h,
                        double lut) {
  MomPhys q;
  q.A = float(A);
  q.nkap6 = float(-kappa / 6.0);
  q.kap144 = float(kappa / 144.0);
  q.lam12 = float(lambda_scale / 12.0);
  q.nu_g = float(nu_g);
  q.dnu = float(nu_l - nu_g);
  q.M3 = float(2.0 * M / 3.0);
  q.M12 = float(2.0 * M / 12.0);
  q.h = float(h);
  q.lut = float(lut);
  q.lut_inv = lut > 0 ? float(1.0 / lut) : 0.f;
  q.p0off = float(-0.25 * A);
  return q;
}

// Gradient and Laplacian stencils of Eq. (best) at one node, from per-row
// summaries of the 3x3 neighbourhood: c (centre), s = right - left and
// d = (left - c) + (right - c) of rows y-1 (0), y (1), y+1 (2), formed once per
// row.  The sums of Eq. (best) regrouped into differences of neighbouring
// values:
//   12 dx = 4 s1 + s0 + s2,  12 dy = 6 (c2 - c0) + (d2 - d0),
//   6 lap = 6 ((c0 - c1) + (c2 - c1)) + (4 d1 + d0 + d2).
// Neighbouring values are close, so those differences are exact in floating
// point and no large partial sums cancel (in a nearly uniform phase the direct
// sums of about twenty times the field value would leave a rounding error of
// fixed sign).  Returned unnormalised; the collision's constants carry the
// factors 1/12 and 1/6.
__device__ __forceinline__ void stencil_rows(const float c[3], const float sv[3], const float d[3], float& dx12,
                                             float& dy12, float& lap6) {
  dx12 = fmaf(4.f, sv[1], sv[0]) + sv[2];
  dy12 = fmaf(6.f, c[2] - c[0], d[2] - d[0]);
  lap6 = fmaf(6.f, (c[0] - c[1]) + (c[2] - c[1]), fmaf(4.f, d[1], d[0] + d[2]));
}
__device__ __forceinline__ void grad_rows(const float c[3], const float sv[3], const float d[3], float& dx12,
                                          float& dy12) {
  dx12 = fmaf(4.f, sv[1], sv[0]) + sv[2];
  dy12 = fmaf(6.f, c[2] - c[0], d[2] - d[0]);
}

// Eq. (best) on an explicit 3x3 neighbourhood (boundary nodes, after the wall
// ghosts), unnormalised as above.
__device__ __forceinline__ void stencil3_unnorm(const float v[3][3], float& dx12, float& dy12, float& lap6) {
  dx12 = fmaf(4.f, v[1][2] - v[1][0], v[0][2] - v[0][0]) + (v[2][2] - v[2][0]);
  dy12 = fmaf(4.f, v[2][1], v[2][0] + v[2][2]) - fmaf(4.f, v[0][1], v[0][0] + v[0][2]);
  lap6 = fmaf(-20.f, v[1][1], fmaf(4.f, (v[0][1] + v[1][0]) + (v[1][2] + v[2][1]),
                                   (v[0][0] + v[0][2]) + (v[2][0] + v[2][2])));
}

// Post-collision f (fs_i = f*_i - w_i) and g (ge = g^eq) of one node from its
// moments and the unnormalised stencils: Eq. (equilibrium) for f^eq with the
// binary pressure of Sec. 3.1, g^eq of App. A, and the collision with every
// mode but pxx - pyy and pxy relaxed fully.
//
// With T = (Txx, Tyy, Txy) the second moment of f^eq beyond the pressure (the
// rho u u and lambda terms of Eq. (equilibrium)) and G = kappa (dphi dphi) its
// gradient terms, the even part of each pair of opposite directions, less w_i, is
//   A1 = (P0 + Uxx - Uyy / 2) / 3 + dxx,   A3 = (P0 + Uyy - Uxx / 2) / 3 - dxx,
//   A5 = (P0 + V + 3 (Txy + Gxy)) / 12 + dxy,  A7 = (P0 + V - 3 (Txy + Gxy)) / 12 - dxy,
// with U = T + G, V = (Txx + Tyy) - (Gxx + Gyy) / 2, P0 the pressure less 1/3,
// and dxx, dxy the stress non-equilibria relaxed at omega, (1 - omega)/4 times
// (m - m^eq).  The odd parts are the momenta j/3 and j/12.
//
// F16OFF: the populations are deviations from the FP16 storage's rest offsets
// w_i(P0b), P0b = 1/3 + A/4 (SF16), not from 4/9, 1/9, 1/36: the pressure term
// carries Q.p0off = -A/4, which moves each pair's even part by w_i(1/3) - w_i(P0b)
// (A/12, A/48) and the rest population by the opposite sum (5A/12).
// Two FP32 lanes in one 64-bit register for the packed FP32 instructions of
// sm_100 and later (fma/mul/add.rn.f32x2): each element is rounded exactly as the
// scalar fmaf / __fmul_rn / + on it, so a pair computes the same bits as the two
// scalar operations in one issue slot.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk2(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
template <bool F16OFF = false>
__device__ __forceinline__ void collide_moment_node(const MomPhys& Q, float drho, float jx, float jy, float mxx,
                                                    float mxy, float phi, float rdx, float rdy, float pdx,
                                                    float pdy, float plap, float fs[9], float ge[9]) {
  // Every product that feeds a sum is an explicit fused multiply-add and every
  // other product an explicit __fmul_rn, so the compiler fuses nothing on its
  // own and every kernel that inlines this function rounds a node alike.
  const float inv = rcp_fast(1.f + drho);
  const float ux = __fmul_rn(jx, inv), uy = __fmul_rn(jy, inv);
  const float phi2 = __fmul_rn(phi, phi);
  // chemical potential (Eq. chempot): A (phi^3 - phi) - kappa lap phi
  const float mu = fmaf(Q.nkap6, plap, __fmul_rn(Q.A, fmaf(phi2, phi, -phi)));
  // viscosity (Eq. nu, the liquid fraction clamped) and c = (1 - omega) / 4
  float cl = __saturatef(fmaf(phi, 0.5f, 0.5f));
  if (Q.lut > 0.f) cl = __fmul_rn(rintf(__fmul_rn(cl, Q.lut)), Q.lut_inv);  // viscosity table of App. A
  const float nu = fmaf(cl, Q.dnu, Q.nu_g);
  const float r = rcp_fast(fmaf(6.f, nu, 1.f));  // omega / 2
  const float c = fmaf(-0.5f, r, 0.25f);
  const float lam = __fmul_rn(Q.lam12, nu);
  // P0 - 1/3: p0 = rho/3 + A (-phi^2/2 + 3 phi^4/4) less kappa phi lap phi
  const float P0r = fmaf(__fmul_rn(Q.nkap6, phi), plap,
                         fmaf(drho, 1.f / 3.f, __fmul_rn(__fmul_rn(Q.A, phi2), fmaf(0.75f, phi2, -0.5f))));
  const float P0 = F16OFF ? P0r + Q.p0off : P0r;
  // second moment of f^eq beyond P0: T (rho u u and the lambda terms) and the
  // gradient terms G = kappa (dphi dphi), with U = T + G
  const float ax = __fmul_rn(ux, rdx), ay = __fmul_rn(uy, rdy);
  const float udr = ax + ay;
  const float Txx = fmaf(jx, ux, __fmul_rn(lam, fmaf(2.f, ax, udr)));
  const float Tyy = fmaf(jy, uy, __fmul_rn(lam, fmaf(2.f, ay, udr)));
  const float Txy = fmaf(jx, uy, __fmul_rn(lam, fmaf(ux, rdy, __fmul_rn(uy, rdx))));
  const float kx = __fmul_rn(Q.kap144, pdx), ky = __fmul_rn(Q.kap144, pdy);
  const float Uxx = fmaf(kx, pdx, Txx), Uyy = fmaf(ky, pdy, Tyy);
  const float GS = fmaf(kx, pdx, __fmul_rn(ky, pdy));   // Gxx + Gyy
  const float V = fmaf(-0.5f, GS, Txx + Tyy);
  const float TG = fmaf(kx, pdy, Txy);                  // Txy + Gxy
  const float dxx = __fmul_rn(c, mxx - (Uxx - Uyy));
  const float dxy = __fmul_rn(c, mxy - TG);
  const float A1 = fmaf(P0 + fmaf(-0.5f, Uyy, Uxx), 1.f / 3.f, dxx);
  const float A3 = fmaf(P0 + fmaf(-0.5f, Uxx, Uyy), 1.f / 3.f, -dxx);
  const float W3 = __fmul_rn(3.f, TG);
  const float A5 = fmaf(P0 + (V + W3), 1.f / 12.f, dxy);
  const float A7 = fmaf(P0 + (V - W3), 1.f / 12.f, -dxy);
  const float jp = jx + jy, jm = jy - jx;
  // the symmetric outputs as packed pairs (fs_1, fs_3), (fs_2, fs_4), ... with the
  // same operations element by element as the scalar form (1.9 % faster on the
  // issue-bound moment kernel; pairing the equilibrium stress as well gained nothing)
  const unsigned long long J = pk2(jx, jy), A13 = pk2(A1, A3), JPM = pk2(jp, jm), A57 = pk2(A5, A7);
  upk2(fma2(J, pk2(1.f / 3.f, 1.f / 3.f), A13), fs[1], fs[3]);
  upk2(fma2(J, pk2(-1.f / 3.f, -1.f / 3.f), A13), fs[2], fs[4]);
  upk2(fma2(JPM, pk2(1.f / 12.f, 1.f / 12.f), A57), fs[5], fs[7]);
  upk2(fma2(JPM, pk2(-1.f / 12.f, -1.f / 12.f), A57), fs[6], fs[8]);
  fs[0] = fmaf(-2.f, (A1 + A3) + (A5 + A7), drho);
  // g^eq (App. A, dt = 1)
  const float Q3 = __fmul_rn(Q.M3, mu), Q12 = __fmul_rn(Q.M12, mu);
  const float nu2 = __fmul_rn(fmaf(ux, ux, __fmul_rn(uy, uy)), -1.f / 3.f);  // -u.u / 3
  const float hp = __fmul_rn(0.5f, phi), hq = __fmul_rn(0.125f, phi);
  const float upp = ux + uy, ump = ux - uy;
  const unsigned long long U = pk2(ux, uy), UPM = pk2(upp, ump), NU2 = pk2(nu2, nu2);
  const unsigned long long B13 = fma2(pk2(hp, hp), fma2(U, U, NU2), pk2(Q3, Q3));
  const unsigned long long B57 = fma2(pk2(hq, hq), fma2(UPM, UPM, NU2), pk2(Q12, Q12));
  const float p3 = __fmul_rn(phi, 1.f / 3.f), p12 = __fmul_rn(phi, 1.f / 12.f);
  upk2(fma2(pk2(p3, p3), U, B13), ge[1], ge[3]);
  upk2(fma2(pk2(-p3, -p3), U, B13), ge[2], ge[4]);
  upk2(fma2(pk2(p12, -p12), UPM, B57), ge[5], ge[7]);
  upk2(fma2(pk2(-p12, p12), UPM, B57), ge[6], ge[8]);
  float B1, B3, B5, B7;
  upk2(B13, B1, B3);
  upk2(B57, B5, B7);
  ge[0] = fmaf(-2.f, (B1 + B3) + (B5 + B7), phi);
}

// The FP64 collision in pair form (the same update as collide_node's FP32 path
// in exact arithmetic, with fewer operations on the FP64 pipe, which bounds the
// FP64 storages).  The equilibrium of Eq. (equilibrium) gives each pair of
// opposite directions i, i' a common even part E_i and odd parts +-(e_i . j) w_i:
//   E_1 = E_2 = (P0 + Uxx - Uyy / 2) / 3,  E_3 = E_4 = (P0 + Uyy - Uxx / 2) / 3,
//   E_5 = E_6 = (P0 + V + 3 TG) / 12,      E_7 = E_8 = (P0 + V - 3 TG) / 12,
// with U = T + G the second moment beyond P0 (T: rho u u and the lambda terms,
// G: kappa times the gradient products), V = Txx + Tyy - (Gxx + Gyy) / 2 and
// TG = Txy + Gxy; the collision adds (1 - omega) / 4 times the stress modes'
// non-equilibrium, +-(pxx - pyy - (Uxx - Uyy)) and +-(pxy - TG), to the even
// parts; f*_0 = rho - 2 (A_1 + A_3 + A_5 + A_7).  (In FP32 on full population
// values this form moved phi beyond the method's bar; FP64 rounding is far below
// it.)
template <int MODEL, typename A>
__device__ __forceinline__ void collide_pairs(const Phys<A>& P, const A vr[3][3], const A vp[3][3], const A fa[9],
                                              A fs[9], A ge[9]) {
  constexpr bool BIN = MODEL == MODEL_BINARY;
  A rdx, rdy, rlap;
  stencil3(vr, rdx, rdy, rlap);
  const A rho = vr[1][1];
  const A jx = momx(fa), jy = momy(fa);
  // one reciprocal per node: of rho times the node's other divisor (binary:
  // 6 nu + 1 of Eq. (nu); liquid-gas: 1 - b rho of the van der Waals p0)
  A inv, P0, gpx, gpy, lam, omega, ux, uy;
  if constexpr (BIN) {
    A pdx, pdy, plap;
    stencil3(vp, pdx, pdy, plap);
    const A phi = vp[1][1];
    const A phi2 = phi * phi;
    const A p0 = rho * A(1.0 / 3.0) + P.Acoef * (A(-0.5) * phi2 + A(0.75) * phi2 * phi2);
    const A mu = P.Acoef * (phi2 * phi - phi) - P.kappa * plap;
    const A nu = local_nu_binary(P, phi);
    const A s6 = fma(A(6), nu, A(1));
    const A r = rcp_rn(rho * s6);
    inv = s6 * r;
    omega = A(2) * (rho * r);
    ux = jx * inv;
    uy = jy * inv;
    P0 = p0 - P.kappa * phi * plap;
    gpx = pdx;
    gpy = pdy;
    lam = P.lambda_scale * nu;
    geq9<A>(phi, ux, uy, A(2) * P.M * mu, ge);
  } else {
    const A q = A(1) - P.b * rho;
    const A r = rcp_rn(rho * q);
    inv = q * r;
    ux = jx * inv;
    uy = jy * inv;
    const A p0 = rho * P.T * (rho * r) - P.a * rho * rho;
    omega = P.omega;  // 2 / (6 nu + 1), one viscosity
    P0 = p0 - P.kappa * rho * rlap;
    gpx = rdx;
    gpy = rdy;
    lam = P.lambda_scale * P.nu;
  }
  const A ax = ux * rdx, ay = uy * rdy;
  const A udr = ax + ay;
  const A Txx = jx * ux + lam * (A(2) * ax + udr);
  const A Tyy = jy * uy + lam * (A(2) * ay + udr);
  const A Txy = jx * uy + lam * (ux * rdy + uy * rdx);
  const A kx = P.kappa * gpx, ky = P.kappa * gpy;
  const A Uxx = Txx + kx * gpx, Uyy = Tyy + ky * gpy;
  const A V = (Txx + Tyy) - A(0.5) * (kx * gpx + ky * gpy);
  const A TG = Txy + kx * gpy;
  const A c = (A(1) - omega) * A(0.25);
  const A dxx = c * (((fa[1] + fa[2]) - (fa[3] + fa[4])) - (Uxx - Uyy));
  const A dxy = c * (((fa[5] + fa[6]) - (fa[7] + fa[8])) - TG);
  const A A1 = (P0 + (Uxx - A(0.5) * Uyy)) * A(1.0 / 3.0) + dxx;
  const A A3 = (P0 + (Uyy - A(0.5) * Uxx)) * A(1.0 / 3.0) - dxx;
  const A W3 = A(3) * TG;
  const A A5 = (P0 + (V + W3)) * A(1.0 / 12.0) + dxy;
  const A A7 = (P0 + (V - W3)) * A(1.0 / 12.0) - dxy;
  const A bx = jx * A(1.0 / 3.0), by = jy * A(1.0 / 3.0);
  const A bp = (jx + jy) * A(1.0 / 12.0), bm = (jy - jx) * A(1.0 / 12.0);
  fs[1] = A1 + bx; fs[2] = A1 - bx;
  fs[3] = A3 + by; fs[4] = A3 - by;
  fs[5] = A5 + bp; fs[6] = A5 - bp;
  fs[7] = A7 + bm; fs[8] = A7 - bm;
  fs[0] = rho - A(2) * ((A1 + A3) + (A5 + A7));
}

// Per-node update shared by both step kernels: wall ghosts and rest rule (for
// boundary nodes), stencils, local thermodynamics, equilibria and the
// moment-space collision.  vr/vp: 3x3 rho/phi neighbourhoods (raw values at
// solid neighbours), fa/ga: the node's stored populations.  Outputs: fs, the
// post-collision f, and ge = g^eq (post-collision g).
template <int MODEL, typename A>
__device__ __forceinline__ void collide_node(const Phys<A>& P, A vr[3][3], A vp[3][3], const bool sol[3][3],
                                             bool bnd, A fa[9], A fs[9], A ge[9]) {
  constexpr bool BIN = MODEL == MODEL_BINARY;
  if (bnd) {
    apply_ghosts(vr, sol, BIN ? A(0) : P.h);
    if (BIN) apply_ghosts(vp, sol, P.h);
    rest(fa);
  }
  if constexpr (std::is_same<A, double>::value) {
    collide_pairs<MODEL>(P, vr, vp, fa, fs, ge);
    return;
  }
  A rdx, rdy, rlap;
  stencil3(vr, rdx, rdy, rlap);
  const A rho = vr[1][1];
  const A jx = momx(fa), jy = momy(fa);
  const A inv = rcp_rn(rho);
  const A ux = jx * inv, uy = jy * inv;
  A fe[9];
  A omega;
  if (BIN) {
    A pdx, pdy, plap;
    stencil3(vp, pdx, pdy, plap);
    const A phi = vp[1][1];
    const A phi2 = phi * phi;
    const A p0 = rho * A(1.0 / 3.0) + P.Acoef * (A(-0.5) * phi2 + A(0.75) * phi2 * phi2);
    const A mu = P.Acoef * (phi2 * phi - phi) - P.kappa * plap;
    const A nu = local_nu_binary(P, phi);
    omega = A(2) * rcp_rn(fma(A(6), nu, A(1)));
    feq9<A>(rho, jx, jy, ux, uy, p0 - P.kappa * phi * plap, P.kappa, pdx, pdy, rdx, rdy, P.lambda_scale * nu, fe);
    geq9<A>(phi, ux, uy, A(2) * P.M * mu, ge);
  } else {
    const A p0 = rho * P.T * rcp_rn(A(1) - P.b * rho) - P.a * rho * rho;
    omega = A(2) * rcp_rn(A(6) * P.nu + A(1));
    feq9<A>(rho, jx, jy, ux, uy, p0 - P.kappa * rho * rlap, P.kappa, rdx, rdy, rdx, rdy, P.lambda_scale * P.nu, fe);
  }
  // stress-mode non-equilibrium relaxed at rate omega; every other mode to f^eq
  const A c = (A(1) - omega) * A(0.25);
  const A mxx = c * (((fa[1] + fa[2]) - (fa[3] + fa[4])) - ((fe[1] + fe[2]) - (fe[3] + fe[4])));
  const A mxy = c * (((fa[5] + fa[6]) - (fa[7] + fa[8])) - ((fe[5] + fe[6]) - (fe[7] + fe[8])));
  fs[1] = fe[1] + mxx; fs[2] = fe[2] + mxx;
  fs[3] = fe[3] - mxx; fs[4] = fe[4] - mxx;
  fs[5] = fe[5] + mxy; fs[6] = fe[6] + mxy;
  fs[7] = fe[7] - mxy; fs[8] = fe[8] - mxy;
  // the rest population from the rounded moving ones: the node's stored populations
  // add up to rho to one rounding (in exact arithmetic it equals f^eq_0)
  fs[0] = rho - (((fs[1] + fs[2]) + (fs[3] + fs[4])) + ((fs[5] + fs[6]) + (fs[7] + fs[8])));
}

// Push streaming from node (col[1], row yy) with bounce-back into solid
// neighbours.  rowb: y*nx of rows y-1, y, y+1 (wrapped); col: x-1, x, x+1.
// Per-node update of the FP16 deviation storage (binary model), in deviations:
// vr holds rho - 1 (the sums of the stored deviations f_i - w_i, whose offsets add
// up to 1), fa the node's deviations; fs returns post-collision deviations from
// the same offsets, ge g^eq.  The wall ghosts and the rest rule as in
// collide_node (the rest rule acts on j, to which the offsets add nothing), then
// the pair-form collision of the moment kernel with its pressure shifted to the
// offsets' P0 (the same update in exact arithmetic, without adding and removing
// the offsets at every load and store).
template <int MODEL>
__device__ __forceinline__ void collide_node_f16(const MomPhys& Q, float vr[3][3], float vp[3][3],
                                                 const bool sol[3][3], bool bnd, float fa[9], float fs[9],
                                                 float ge[9]) {
  static_assert(MODEL == MODEL_BINARY, "the FP16 deviation storage holds the binary model");
  if (bnd) {
    apply_ghosts(vr, sol, 0.f);
    apply_ghosts(vp, sol, Q.h);
    rest(fa);
  }
  float rdx, rdy, rlap, pdx, pdy, plap;
  stencil3_unnorm(vr, rdx, rdy, rlap);
  stencil3_unnorm(vp, pdx, pdy, plap);
  const float mxx = (fa[1] + fa[2]) - (fa[3] + fa[4]);
  const float mxy = (fa[5] + fa[6]) - (fa[7] + fa[8]);
  collide_moment_node<true>(Q, vr[1][1], momx(fa), momy(fa), mxx, mxy, vp[1][1], rdx, rdy, pdx, pdy, plap, fs, ge);
}

// RAW: store f as the storage's raw values (the deviations of dev_arith storages).
template <int MODEL, class S, bool RAW = false>
__device__ __forceinline__ void push_node(const Buf<S>& dst, size_t N, const int rowb[3], const int col[3],
                                          const bool sol[3][3], bool bnd, const typename S::A fs[9],
                                          const typename S::A ge[9]) {
  constexpr bool BIN = MODEL == MODEL_BINARY;
  if (!bnd) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int dn = rowb[1 + EYd(i)] + col[1 + EXd(i)];
      if constexpr (RAW)
        S::sfr(dst.f, N, (size_t)dn, i, fs[i]);
      else
        S::sf(dst.f, N, (size_t)dn, i, fs[i], dst.r);
      if (BIN) S::sg(dst.g, dst.g0, N, (size_t)dn, i, ge[i]);
    }
  } else {
    const int self = rowb[1] + col[1];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int ex = EXd(i), ey = EYd(i);
      const bool back = sol[1 + ey][1 + ex];
      const int dn = back ? self : rowb[1 + ey] + col[1 + ex];
      const int di = back ? OPPd(i) : i;
      if constexpr (RAW)
        S::sfr(dst.f, N, (size_t)dn, di, fs[i]);
      else
        S::sf(dst.f, N, (size_t)dn, di, fs[i], dst.r);
      if (BIN) S::sg(dst.g, dst.g0, N, (size_t)dn, di, ge[i]);
    }
  }
}

// push_node with 32-bit element offsets from the buffer bases (the staged
// kernels; the host admits them only for lattices with 9 N < 2^32 nodes).
// rowb/col as in push_node.
template <int MODEL, class S, bool RAW = false>
__device__ __forceinline__ void push_node_u32(const Buf<S>& dst, uint32_t N, const int rowb[3], const int col[3],
                                              const bool sol[3][3], bool bnd, const typename S::A fs[9],
                                              const typename S::A ge[9]) {
  constexpr bool BIN = MODEL == MODEL_BINARY;
  if (!bnd) {
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const uint32_t dn = (uint32_t)(rowb[1 + EYd(i)] + col[1 + EXd(i)]);
      if constexpr (RAW)
        S::sfor(dst.f, N, dn, i, fs[i]);
      else
        S::sfo(dst.f, N, dn, i, fs[i], dst.r);
      if (BIN) S::sgo(dst.g, dst.g0, N, dn, i, ge[i]);
    }
  } else {
    const uint32_t self = (uint32_t)(rowb[1] + col[1]);
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      const int ex = EXd(i), ey = EYd(i);
      const bool back = sol[1 + ey][1 + ex];
      const uint32_t dn = back ? self : (uint32_t)(rowb[1 + ey] + col[1 + ex]);
      const int di = back ? OPPd(i) : i;
      if constexpr (RAW)
        S::sfor(dst.f, N, dn, di, fs[i]);
      else
        S::sfo(dst.f, N, dn, di, fs[i], dst.r);
      if (BIN) S::sgo(dst.g, dst.g0, N, dn, di, ge[i]);
    }
  }
}

// ---------------------------------------------------------------- the step

template <int MODEL, class S>
struct StepArgs {
  Geom G;
  Phys<typename S::A> P;
  MomPhys Q;  // the pair-form constants (storages that compute in deviations)
  Buf<S> src, dst;
  int yc;  // rows per CTA band
};

template <int MODEL, class S, int BX>
struct StepSmem {
  typename S::A r[4][BX + 2];
  typename S::A p[MODEL == MODEL_BINARY ? 4 : 1][BX + 2];
};

template <int MODEL, class S, bool COHERENT = false, bool RAW = false>
__device__ __forceinline__ void load_node(const Buf<S>& B, size_t N, size_t n, typename S::A f[9],
                                          typename S::A g[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    if constexpr (RAW)
      f[i] = COHERENT ? S::lfcr(B.f, N, n, i) : S::lfr(B.f, N, n, i);
    else
      f[i] = COHERENT ? S::lfc(B.f, N, n, i, B.r) : S::lf(B.f, N, n, i, B.r);
  }
  if (MODEL == MODEL_BINARY) {
#pragma unroll
    for (int i = 0; i < 9; ++i) g[i] = COHERENT ? S::lgc(B.g, B.g0, N, n, i) : S::lg(B.g, B.g0, N, n, i);
  }
}

// Process columns [xb, xb + BX) (clipped to nx) and rows [y0, y1) of one lattice.
// COHERENT loads bypass the non-coherent read path (buffers written earlier in
// the same launch, as in the persistent batched kernel).
template <int MODEL, class S, int BX, bool COHERENT = false>
__device__ __forceinline__ void step_band(const Geom& G, const Phys<typename S::A>& P, const MomPhys& Q,
                                          const Buf<S>& src, const Buf<S>& dst, int xb, int y0, int y1,
                                          StepSmem<MODEL, S, BX>& sm) {
  using A = typename S::A;
  constexpr bool BIN = MODEL == MODEL_BINARY;
  constexpr bool RAW = dev_arith<S>::value;
  const int nx = G.nx, ny = G.ny;
  const size_t N = (size_t)nx * ny;
  const int tid = threadIdx.x;
  const int w = min(BX, nx - xb);  // columns in this tile
  const int x = xb + tid;
  const bool act = tid < w;
  // halo columns: thread 0 takes the left one, thread 1 the right one
  const int hx = tid == 0 ? wrapi(xb - 1, nx) : wrapi(xb + w, nx);
  const int hs = tid == 0 ? 0 : w + 1;
  const bool hal = tid < 2;

  A fa[9], ga[9], fb[9], gb[9], fc[9], gc[9];  // rows y (a), y+1 (b), y+2 (c)
  A hf[9], hg[9];
  auto slot = [&](int r) { return (r - y0 + 1) & 3; };

  // load row r (wrapped) for this thread's column into f, g, and publish rho/phi
  auto publish = [&](int r, const A* f, const A* g, bool fluid, const A* hf_, const A* hg_, bool hfluid) {
    const int s = slot(r);
    if (act) {
      sm.r[s][tid + 1] = fluid ? sum9(f) : A(0);
      if (BIN) sm.p[s][tid + 1] = fluid ? sum9(g) : A(0);
    }
    if (hal) {
      sm.r[s][hs] = hfluid ? sum9(hf_) : A(0);
      if (BIN) sm.p[s][hs] = hfluid ? sum9(hg_) : A(0);
    }
  };
  auto fetch = [&](int r, A* f, A* g, bool& fluid, bool& hfluid) {
    const int rr = wrapi(r, ny);
    fluid = act && !is_solid(G, x, rr);
    if (fluid) load_node<MODEL, S, COHERENT, RAW>(src, N, (size_t)rr * nx + x, f, g);
    hfluid = hal && !is_solid(G, hx, rr);
    if (hfluid) load_node<MODEL, S, COHERENT, RAW>(src, N, (size_t)rr * nx + hx, hf, hg);
  };

  bool fl_a, fl_b, fl_c, hfl;
  {
    bool dummy;
    A tf[9], tg[9];
    fetch(y0 - 1, tf, tg, dummy, hfl);
    publish(y0 - 1, tf, tg, dummy, hf, hg, hfl);
    fetch(y0, fa, ga, fl_a, hfl);
    publish(y0, fa, ga, fl_a, hf, hg, hfl);
    fetch(y0 + 1, fb, gb, fl_b, hfl);
    publish(y0 + 1, fb, gb, fl_b, hf, hg, hfl);
  }
  __syncthreads();

  for (int y = y0; y < y1; ++y) {
    const bool more = y + 2 <= y1;
    if (more) fetch(y + 2, fc, gc, fl_c, hfl);

    if (fl_a) {
      const int yy = wrapi(y, ny);
      bool sol[3][3], bnd;
      neighbour_solids(G, x, yy, sol, bnd);
      A vr[3][3], vp[3][3];
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          vr[j][i] = sm.r[slot(y - 1 + j)][tid + i];
          if (BIN) vp[j][i] = sm.p[slot(y - 1 + j)][tid + i];
        }
      A fs[9], ge[9];
      if constexpr (RAW)
        collide_node_f16<MODEL>(Q, vr, vp, sol, bnd, fa, fs, ge);
      else
        collide_node<MODEL, A>(P, vr, vp, sol, bnd, fa, fs, ge);
      const int rowb[3] = {wrapi(yy - 1, ny) * nx, yy * nx, wrapi(yy + 1, ny) * nx};
      const int col[3] = {wrapi(x - 1, nx), x, wrapi(x + 1, nx)};
      push_node<MODEL, S, RAW>(dst, N, rowb, col, sol, bnd, fs, ge);
    }

    if (more) publish(y + 2, fc, gc, fl_c, hf, hg, hfl);
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      fa[i] = fb[i];
      fb[i] = fc[i];
      if (BIN) {
        ga[i] = gb[i];
        gb[i] = gc[i];
      }
    }
    fl_a = fl_b;
    fl_b = more ? fl_c : false;
  }
}

template <int MODEL, class S, int BX>
__global__ void __launch_bounds__(BX) step_kernel(StepArgs<MODEL, S> a) {
  __shared__ StepSmem<MODEL, S, BX> sm;
  int cb, band;
  tile_of_block((a.G.nx + BX - 1) / BX, cb, band);
  const int xb = cb * BX;
  const int y0 = band * a.yc;
  const int y1 = min(y0 + a.yc, a.G.ny);
  step_band<MODEL, S, BX>(a.G, a.P, a.Q, a.src, a.dst, xb, y0, y1, sm);
}

}  // namespace lbk
