// Auxiliary kernels: equilibrium initialisation from macroscopic fields, field
// and population export/import, and the FP64 reductions behind
// lb_filled_length (mass, sum of phi, filled volume, meniscus position l).
#pragma once

#include "lb_device.cuh"
#include "lb_moment.cuh"

namespace lbk {

// Gather the 3x3 neighbourhood of a double field around fluid node (x, y).
template <typename A>
// 3x3 neighbourhood of a field with row stride sy (nx: a full field; 0: one value per
// column); solid nodes read as 0 (the wall ghosts replace them).
__device__ __forceinline__ void gather_field(const Geom& G, const double* __restrict__ v, size_t sy, int x, int y,
                                             A out[3][3]) {
#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const int xx = wrapi(x + i - 1, G.nx), yy = wrapi(y + j - 1, G.ny);
      out[j][i] = is_solid(G, xx, yy) ? A(0) : A(v[(size_t)yy * sy + xx]);
    }
}

// f = f^eq and g = g^eq of the given fields (stencils with the wall ghosts); the
// fields have row stride sy (nx, or 0 for fields given as one value per column).
template <int MODEL, class S>
__global__ void init_kernel(Geom G, Phys<typename S::A> P, Buf<S> B, const double* __restrict__ rho_in,
                            const double* __restrict__ ux_in, const double* __restrict__ uy_in,
                            const double* __restrict__ phi_in, size_t sy) {
  using A = typename S::A;
  constexpr bool BIN = MODEL == MODEL_BINARY;
  const size_t N = (size_t)G.nx * G.ny;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % G.nx), y = (int)(n / G.nx);
    if (is_solid(G, x, y)) {
      if constexpr (is_moments<S>::value) {
        const float z[M_PLANES] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if constexpr (pull_kind<S>::value == 2) {
          const float zf[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
          sg_store(B.f, N, n, zf, 0.f);
        } else {
          pull_store_moments<S>(B.f, N, n, z);
        }
      } else {
        // zero bits in every plane (with the FP16 offsets a stored 0 would not be),
        // the same as a fresh buffer: no step reads or writes a solid node
        for (int i = 0; i < 9; ++i) {
          S::zf(B.f, N, n, i);
          if (BIN) S::sg(B.g, B.g0, N, n, i, A(0));
        }
      }
      continue;
    }
    bool sol[3][3], bnd;
    neighbour_solids(G, x, y, sol, bnd);
    A vr[3][3], vp[3][3];
    gather_field(G, rho_in, sy, x, y, vr);
    if (BIN) gather_field(G, phi_in, sy, x, y, vp);
    if (bnd) {
      apply_ghosts(vr, sol, BIN ? A(0) : P.h);
      if (BIN) apply_ghosts(vp, sol, P.h);
    }
    A rdx, rdy, rlap;
    stencil3(vr, rdx, rdy, rlap);
    const size_t nin = (size_t)y * sy + x;
    const A rho = vr[1][1], ux = A(ux_in[nin]), uy = A(uy_in[nin]);
    const A jx = rho * ux, jy = rho * uy;
    A fe[9], ge[9];
    if (BIN) {
      A pdx, pdy, plap;
      stencil3(vp, pdx, pdy, plap);
      const A phi = vp[1][1], phi2 = phi * phi;
      const A p0 = rho * A(1.0 / 3.0) + P.Acoef * (A(-0.5) * phi2 + A(0.75) * phi2 * phi2);
      const A mu = P.Acoef * (phi2 * phi - phi) - P.kappa * plap;
      const A nu = local_nu_binary(P, phi);
      feq9<A>(rho, jx, jy, ux, uy, p0 - P.kappa * phi * plap, P.kappa, pdx, pdy, rdx, rdy, P.lambda_scale * nu, fe);
      geq9<A>(phi, ux, uy, A(2) * P.M * mu, ge);
    } else {
      const A p0 = rho * P.T / (A(1) - P.b * rho) - P.a * rho * rho;
      feq9<A>(rho, jx, jy, ux, uy, p0 - P.kappa * rho * rlap, P.kappa, rdx, rdy, rdx, rdy, P.lambda_scale * P.nu, fe);
    }
    if constexpr (is_moments<S>::value) {
      if constexpr (pull_kind<S>::value == 2) {
        // f as deviations from the rest weights (exact: f^eq_i and w_i are close), phi
        float fd[9];
        for (int i = 0; i < 9; ++i) fd[i] = fe[i] - (float)WREST(i);
        sg_store(B.f, N, n, fd, (float)phi_in[nin]);
      } else {
        A m[M_PLANES];
        pops_to_moments(fe, ge, m);
        m[M_RHO] = (A)(rho_in[nin] - 1.0);  // stored as rho - 1
        pull_store_moments<S>(B.f, N, n, m);
      }
    } else {
      for (int i = 0; i < 9; ++i) {
        S::sf(B.f, N, n, i, fe[i], B.r);
        if (BIN) S::sg(B.g, B.g0, N, n, i, ge[i]);
      }
    }
  }
}

// The six moments of node n of a pull-kernel storage in FP64 (rho as rho - 1):
// read (SM32, SM16) or summed in FP64 from the f deviations (SG32).
template <class S>
__device__ __forceinline__ void pull_moments_f64(const void* base, size_t N, size_t n, double m[M_PLANES]) {
  if constexpr (pull_kind<S>::value == 2) {
    float fd[9], ph;
    sg_load(base, N, n, fd, ph);
    double f[9], g[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < 9; ++i) f[i] = (double)fd[i];
    g[0] = (double)ph;
    pops_to_moments(f, g, m);
  } else {
    float mf[M_PLANES];
    pull_load<S>(base, N, n, mf);
    for (int k = 0; k < M_PLANES; ++k) m[k] = (double)mf[k];
  }
}

template <int MODEL, class S>
__device__ __forceinline__ bool node_state(const Geom& G, const Buf<S>& B, size_t N, int x, int y, bool rested,
                                           typename S::A f[9], typename S::A g[9]) {
  if (is_solid(G, x, y)) return false;
  load_node<MODEL, S>(B, N, (size_t)y * G.nx + x, f, g);
  if (rested) {
    bool sol[3][3], bnd;
    neighbour_solids(G, x, y, sol, bnd);
    if (bnd) rest(f);
  }
  return true;
}

// rho, u = j / rho, phi per node (boundary nodes after the rest rule).
template <int MODEL, class S>
__global__ void fields_kernel(Geom G, Buf<S> B, double* __restrict__ rho, double* __restrict__ ux,
                              double* __restrict__ uy, double* __restrict__ phi) {
  using A = typename S::A;
  const size_t N = (size_t)G.nx * G.ny;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % G.nx), y = (int)(n / G.nx);
    if constexpr (is_moments<S>::value) {
      if (is_solid(G, x, y)) {
        rho[n] = ux[n] = uy[n] = phi[n] = 0.0;
        continue;
      }
      bool sol[3][3], bnd;
      neighbour_solids(G, x, y, sol, bnd);
      double m[M_PLANES];
      pull_moments_f64<S>(B.f, N, n, m);
      const double r = 1.0 + m[M_RHO];
      rho[n] = r;
      ux[n] = bnd ? 0.0 : m[M_JX] / r;  // rest rule at boundary nodes
      uy[n] = bnd ? 0.0 : m[M_JY] / r;
      phi[n] = m[M_PHI];
    } else {
      A f[9], g[9];
      if (!node_state<MODEL, S>(G, B, N, x, y, true, f, g)) {
        rho[n] = ux[n] = uy[n] = phi[n] = 0.0;
        continue;
      }
      const A r = sum9(f);
      rho[n] = (double)r;
      ux[n] = (double)(momx(f) / r);
      uy[n] = (double)(momy(f) / r);
      phi[n] = MODEL == MODEL_BINARY ? (double)sum9(g) : 0.0;
    }
  }
}

template <int MODEL, class S>
__global__ void pops_out_kernel(Geom G, Buf<S> B, int rested, double* __restrict__ fo, double* __restrict__ go) {
  using A = typename S::A;
  const size_t N = (size_t)G.nx * G.ny;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % G.nx), y = (int)(n / G.nx);
    if constexpr (pull_kind<S>::value == 2) {
      // the f populations (deviations plus the rest weights, in FP64); for g the
      // populations (phi, 0, ..., 0), which carry the only moment of g a step uses
      double f[9], g[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
      const bool fl = !is_solid(G, x, y);
      if (fl) {
        float fd[9], ph;
        sg_load(B.f, N, n, fd, ph);
        for (int i = 0; i < 9; ++i) f[i] = (double)fd[i] + WREST(i);
        g[0] = (double)ph;
        bool sol[3][3], bnd;
        neighbour_solids(G, x, y, sol, bnd);
        if (rested && bnd) rest(f);
      }
      for (int i = 0; i < 9; ++i) {
        fo[i * N + n] = fl ? f[i] : 0.0;
        if (go) go[i * N + n] = fl ? g[i] : 0.0;
      }
    } else {
      A f[9], g[9];
      const bool fl = node_state<MODEL, S>(G, B, N, x, y, rested != 0, f, g);
      for (int i = 0; i < 9; ++i) {
        fo[i * N + n] = fl ? (double)f[i] : 0.0;
        if (MODEL == MODEL_BINARY && go) go[i * N + n] = fl ? (double)g[i] : 0.0;
      }
    }
  }
}

template <int MODEL, class S>
__global__ void pops_in_kernel(Geom G, Buf<S> B, const double* __restrict__ fi, const double* __restrict__ gi) {
  using A = typename S::A;
  const size_t N = (size_t)G.nx * G.ny;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % G.nx), y = (int)(n / G.nx);
    const bool sol = is_solid(G, x, y);
    if constexpr (is_moments<S>::value) {
      // moments (or f deviations and phi) of the given populations, formed in
      // FP64 and rounded once
      double f[9], g[9], m[M_PLANES];
      for (int i = 0; i < 9; ++i) {
        f[i] = fi[i * N + n];
        g[i] = MODEL == MODEL_BINARY ? gi[i * N + n] : 0.0;
      }
      if constexpr (pull_kind<S>::value == 2) {
        float fd[9];
        for (int i = 0; i < 9; ++i) fd[i] = sol ? 0.f : (float)(f[i] - WREST(i));
        sg_store(B.f, N, n, fd, sol ? 0.f : (float)sum9(g));
      } else {
        pops_to_moments(f, g, m);
        m[M_RHO] -= 1.0;  // stored as rho - 1
        float mf[M_PLANES];
        for (int k = 0; k < M_PLANES; ++k) mf[k] = sol ? 0.f : (float)m[k];
        pull_store_moments<S>(B.f, N, n, mf);
      }
    } else {
      for (int i = 0; i < 9; ++i) {
        if (sol)
          S::zf(B.f, N, n, i);  // zero bits, as in init_kernel
        else
          S::sf(B.f, N, n, i, A(fi[i * N + n]), B.r);
        if (MODEL == MODEL_BINARY) S::sg(B.g, B.g0, N, n, i, sol ? A(0) : A(gi[i * N + n]));
      }
    }
  }
}

// The six moments of the stored state (plane-major [M_PLANES][ny][nx]); for the
// population storages they are summed in FP64 from the stored populations.
// Solid nodes give zeros.
template <int MODEL, class S>
__global__ void moments_out_kernel(Geom G, Buf<S> B, double* __restrict__ out) {
  using A = typename S::A;
  const size_t N = (size_t)G.nx * G.ny;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % G.nx), y = (int)(n / G.nx);
    const bool sol = is_solid(G, x, y);
    double m[M_PLANES];
    if constexpr (is_moments<S>::value) {
      pull_moments_f64<S>(B.f, N, n, m);
      m[M_RHO] += 1.0;
    } else {
      A fa[9], ga[9];
      load_node<MODEL, S>(B, N, n, fa, ga);
      double f[9], g[9];
      for (int i = 0; i < 9; ++i) {
        f[i] = (double)fa[i];
        g[i] = MODEL == MODEL_BINARY ? (double)ga[i] : 0.0;
      }
      pops_to_moments(f, g, m);
    }
    for (int k = 0; k < M_PLANES; ++k) out[k * N + n] = sol ? 0.0 : m[k];
  }
}

// ------------------------------------------------------------- reductions

constexpr int RED_THREADS = 256;
constexpr int RED_PARTS = 4;  // mass, phi sum, tube liquid volume, first meniscus column

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Per-node sums for the reductions: rho and phi of one node as the step
// computes them (sum9 in the arithmetic type), then widened to FP64 for the
// sums over nodes.  (FP64 arithmetic is scarce on this GPU: one widening per
// node and field, not one per population.)  The tube's liquid volume is
// accumulated as a sum of the node values and a node count and finished per
// thread by finish_volume, which is exact up to rounding.
struct RedAcc {
  double mass = 0.0, phi = 0.0, tube = 0.0;
  int ntube = 0;
};

template <int MODEL, class S>
__device__ __forceinline__ void red_add_node(const Geom& G, const Buf<S>& B, size_t N, size_t n, int x, int y,
                                             RedAcc& acc) {
  using A = typename S::A;
  double r, p;
  if constexpr (is_moments<S>::value) {
    const float2 v = pull_rho_phi<S>(B.f, N, n);
    r = 1.0 + (double)v.x;
    p = (double)v.y;
  } else {
    A f[9], g[9];
    load_node<MODEL, S, true>(B, N, n, f, g);
    r = (double)sum9(f);
    p = MODEL == MODEL_BINARY ? (double)sum9(g) : 0.0;
  }
  acc.mass += r;
  acc.phi += p;
  if (G.tube_len > 0 && col_in_tube(G, x) && row_in_band(G, y)) {
    acc.tube += MODEL == MODEL_BINARY ? p : r;
    ++acc.ntube;
  }
}

// Liquid volume of the tube nodes a thread visited: sum of (phi + 1) / 2
// (binary) or of (rho - rho_g) / (rho_l - rho_g) (liquid-gas).
template <int MODEL>
__device__ __forceinline__ double finish_volume(const RedAcc& acc, double rho_l, double rho_g) {
  return MODEL == MODEL_BINARY ? 0.5 * (acc.tube + (double)acc.ntube)
                               : (acc.tube - (double)acc.ntube * rho_g) / (rho_l - rho_g);
}

// Centre-line value of the tube at tube column k: phi (binary) or rho - threshold.
template <int MODEL, class S>
__device__ __forceinline__ double centre_value(const Geom& G, const Buf<S>& B, size_t N, int k, double thr) {
  using A = typename S::A;
  int ya, yb;
  if (G.tube_h & 1) {
    ya = yb = wrapi(G.tube_y0 + (G.tube_h - 1) / 2, G.ny);
  } else {
    ya = wrapi(G.tube_y0 + G.tube_h / 2 - 1, G.ny);
    yb = wrapi(G.tube_y0 + G.tube_h / 2, G.ny);
  }
  const int x = wrapi(G.tube_x0 + k, G.nx);
  double va = 0.0, vb = 0.0;
  if constexpr (is_moments<S>::value) {
    const float2 a = pull_rho_phi<S>(B.f, N, (size_t)ya * G.nx + x), b = pull_rho_phi<S>(B.f, N, (size_t)yb * G.nx + x);
    // binary: phi; liquid-gas: rho (stored as rho - 1)
    va = MODEL == MODEL_BINARY ? (double)a.y : 1.0 + (double)a.x;
    vb = MODEL == MODEL_BINARY ? (double)b.y : 1.0 + (double)b.x;
  } else {
    A f[9], g[9];
    load_node<MODEL, S>(B, N, (size_t)ya * G.nx + x, f, g);
    for (int i = 0; i < 9; ++i) va += MODEL == MODEL_BINARY ? (double)g[i] : (double)f[i];
    load_node<MODEL, S>(B, N, (size_t)yb * G.nx + x, f, g);
    for (int i = 0; i < 9; ++i) vb += MODEL == MODEL_BINARY ? (double)g[i] : (double)f[i];
  }
  return 0.5 * (va + vb) - thr;
}

// Block partial sums in FP64 (see red_add_node), and the first tube column k of
// the block's share whose centre line changes sign between k and k + 1 (k = 0
// counts when the inlet is already gas); INT_MAX if none.
// partials[b * RED_PARTS + k].
template <int MODEL, class S>
__global__ void __launch_bounds__(RED_THREADS) reduce_partials_kernel(Geom G, Buf<S> B, double rho_l, double rho_g,
                                                                      double thr, double* __restrict__ partials) {
  const size_t N = (size_t)G.nx * G.ny;
  RedAcc ra;
  for (size_t n = blockIdx.x * (size_t)blockDim.x + threadIdx.x; n < N; n += (size_t)gridDim.x * blockDim.x) {
    const int x = (int)(n % G.nx), y = (int)(n / G.nx);
    if (is_solid(G, x, y)) continue;
    red_add_node<MODEL, S>(G, B, N, n, x, y, ra);
  }
  int first = INT_MAX;
  const int L = G.tube_len;
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
    const double c0 = centre_value<MODEL, S>(G, B, N, k, thr);
    const bool hit = (k == 0 && !(c0 > 0.0)) ||
                     (k + 1 < L && c0 > 0.0 && !(centre_value<MODEL, S>(G, B, N, k + 1, thr) > 0.0));
    if (hit) {
      first = k;  // k grows: the thread's first hit is its smallest
      break;
    }
  }
  const double acc[3] = {ra.mass, ra.phi, finish_volume<MODEL>(ra, rho_l, rho_g)};
  __shared__ double sh[3][RED_THREADS / 32];
  __shared__ int shf[RED_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int k = 0; k < 3; ++k) {
    const double v = warp_sum(acc[k]);
    if (lane == 0) sh[k][wid] = v;
  }
  for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
  if (lane == 0) shf[wid] = first;
  __syncthreads();
  if (threadIdx.x < 3) {
    double s = 0.0;
    for (int w = 0; w < RED_THREADS / 32; ++w) s += sh[threadIdx.x][w];
    partials[blockIdx.x * RED_PARTS + threadIdx.x] = s;
  } else if (threadIdx.x == 3) {
    int f = INT_MAX;
    for (int w = 0; w < RED_THREADS / 32; ++w) f = min(f, shf[w]);
    partials[blockIdx.x * RED_PARTS + 3] = (double)f;
  }
}

// One block: sums the partials in a fixed order (deterministic), takes the first
// centre-line sign change over all blocks and interpolates l there.
// out = {l_centre, l_vol, mass, phi_sum}.
template <int MODEL, class S>
__global__ void __launch_bounds__(32) reduce_final_kernel(Geom G, Buf<S> B, double thr, int nparts,
                                                         const double* __restrict__ partials,
                                                         double* __restrict__ out) {
  const size_t N = (size_t)G.nx * G.ny;
  // lane j takes blocks j, j + 32, ... in order, then a fixed shuffle tree
  double t[3] = {0.0, 0.0, 0.0};
  double fm = (double)INT_MAX;
  for (int b = threadIdx.x; b < nparts; b += 32) {
    for (int k = 0; k < 3; ++k) t[k] += partials[b * RED_PARTS + k];
    fm = fmin(fm, partials[b * RED_PARTS + 3]);
  }
  for (int k = 0; k < 3; ++k) t[k] = warp_sum(t[k]);
  for (int o = 16; o > 0; o >>= 1) fm = fmin(fm, __shfl_xor_sync(0xffffffffu, fm, o));
  if (threadIdx.x == 0) {
    const int L = G.tube_len;
    double l = 0.0;
    if (L <= 0) {
      l = 0.0;
    } else if (fm >= (double)INT_MAX) {
      l = (double)L;
    } else {
      const int k = (int)fm;
      const double c0 = centre_value<MODEL, S>(G, B, N, k, thr);
      if (k == 0 && !(c0 > 0.0)) {
        l = 0.0;
      } else {
        const double c1 = centre_value<MODEL, S>(G, B, N, k + 1, thr);
        l = k + c0 / (c0 - c1);
      }
    }
    out[0] = l;
    out[1] = L > 0 ? t[2] / G.tube_h : 0.0;
    out[2] = t[0];
    out[3] = t[1];
  }
}

}  // namespace lbk
