// Reduced representations of the binary-model state and their step kernel.
//
// With the relaxation matrix of App. A every mode of f except the two stress
// modes relaxes fully to equilibrium, and g relaxes fully to g^eq (Sec. 3.1).
// The post-collision populations of a node therefore depend on its f only
// through rho, jx, jy, pxx - pyy and pxy, and on its g only through phi (plus
// the rho and phi stencils of Eq. (best)).  So the state need not hold all
// eighteen populations.  Three storages use this, all advanced by the same pull
// kernel:
//   SM32  six FP32 moments per node (rho - 1, jx, jy, pxx - pyy, pxy, phi):
//         48 bytes per lattice update (six read, six written) instead of 144;
//   SM16  the same moments with rho - 1, j and the stresses in FP16 and phi in
//         FP32: 28 bytes per update;
//   SG32  the nine f populations in FP32 and phi in place of the nine g
//         populations ("g eliminated"): 80 bytes per update.
// The result is the population scheme's in exact arithmetic; only the rounding
// differs (and, for SM16, the FP16 storage of five of the six moments).
//
// The stored state is the post-streaming state before the boundary-node rest
// rule of Sec. 2.2, as in the population storages.  That rule sets j to zero and
// leaves rho, pxx - pyy and pxy unchanged, so it is applied when a boundary node
// is read.
//
// The binary model keeps rho close to 1 (Sec. 3.1), so the density is stored
// as rho - 1 and the populations are formed and streamed as deviations
// f_i - w_i from the rest weights w = 4/9, 1/9, 1/36 (whose contributions to
// every streamed moment cancel exactly: sum w_i = 1, sum w_i e_i = 0 and the
// stress combinations of w vanish); SG32 stores those deviations.  Rounding then
// acts on numbers of the size of the flow, not on the populations themselves:
// in a nearly uniform phase every node rounds almost the same population the
// same way, and at 1/9 that fixed-sign error would accumulate into a drift of
// the interface.
//
// Step (a pull): the new state of node r is made of the populations that
// arrive there, f_i(r) = f*_i(r - e_i), or f*_opp(i)(r) by bounce-back where
// r - e_i is solid; likewise g_i(r) = g^eq_i(r - e_i).  A warp owns 32
// consecutive columns and every lane collides its own node; lanes 1..30 collect
// the populations of their neighbours by warp shuffles, so a warp produces 30
// columns and its two edge lanes only supply the halo.  The warp walks up a
// band of rows: the populations of row k go to rows k - 1, k and k + 1, and row
// k - 1 is complete (and stored) once row k has been distributed.  The rho/phi
// rows of the stencil window are loaded two rows ahead of the collision, the
// remaining values one row ahead.  Values of solid nodes are never loaded, and a
// row whose whole window is wall under every column of the warp is skipped.
#pragma once

#include <cuda_fp16.h>

#include <type_traits>

#include "lb_device.cuh"

namespace lbk {

// Storage traits of the pull kernel's representations.
struct SM32 {  // six FP32 moments: three float2 planes (rho - 1, phi), (jx, jy), (pxx - pyy, pxy)
  using T = float;
  using A = float;
  static constexpr int kind = 0;
};
struct SM16 {  // FP16 moments, FP32 phi: planes phi (float), rho - 1 (half), j (half2), stresses (half2)
  using T = __half;
  using A = float;
  static constexpr int kind = 1;
};
struct SG32 {  // g eliminated: nine FP32 planes f_i - w_i, then a FP32 plane of phi
  using T = float;
  using A = float;
  static constexpr int kind = 2;
};
enum { M_RHO = 0, M_JX = 1, M_JY = 2, M_XX = 3, M_XY = 4, M_PHI = 5, M_PLANES = 6 };
enum { MP_RP = 0, MP_J = 1, MP_S = 2 };  // float2 planes of SM32

template <class S>
struct is_moments {  // advanced by the pull kernel (populations are not all kept)
  static constexpr bool value = false;
};
template <>
struct is_moments<SM32> {
  static constexpr bool value = true;
};
template <>
struct is_moments<SM16> {
  static constexpr bool value = true;
};
template <>
struct is_moments<SG32> {
  static constexpr bool value = true;
};

// Which pull storage a storage trait is (0 SM32, 1 SM16, 2 SG32), -1 for the
// population storages.
template <class S>
struct pull_kind {
  static constexpr int value = -1;
};
template <>
struct pull_kind<SM32> {
  static constexpr int value = 0;
};
template <>
struct pull_kind<SM16> {
  static constexpr int value = 1;
};
template <>
struct pull_kind<SG32> {
  static constexpr int value = 2;
};

// Byte offsets of the SM16 planes for N nodes (each plane 256-byte aligned).
struct M16Layout {
  size_t phi, r, j, m, total;
};
__host__ __device__ inline M16Layout m16_layout(size_t N) {
  auto up = [](size_t b) { return (b + 255) / 256 * 256; };
  M16Layout L;
  L.phi = 0;
  L.j = up(4 * N);
  L.m = L.j + up(4 * N);
  L.r = L.m + up(4 * N);
  L.total = L.r + up(2 * N);
  return L;
}

// Rest weights of the deviations f_i - w_i.
__host__ __device__ constexpr double WREST(int i) { return i == 0 ? 4.0 / 9.0 : (i < 5 ? 1.0 / 9.0 : 1.0 / 36.0); }

// The six stored moments of one node's populations (m[M_RHO] = sum f).
template <typename A>
__device__ __forceinline__ void pops_to_moments(const A f[9], const A g[9], A m[6]) {
  m[M_RHO] = sum9(f);
  m[M_JX] = momx(f);
  m[M_JY] = momy(f);
  m[M_XX] = (f[1] + f[2]) - (f[3] + f[4]);
  m[M_XY] = (f[5] + f[6]) - (f[7] + f[8]);
  m[M_PHI] = sum9(g);
}

// ------------------------------------------------------ per-node accessors
//
// Used by the initialisation, export, import and reduction kernels (one node
// at a time).  Moments are those of the stored state, rho as rho - 1.

template <bool COHERENT, class P>
__device__ __forceinline__ P ldx(const P* p) {
  if constexpr (COHERENT) return __ldcg(p);
  return *p;
}

// The six moments of node n: SM32 and SM16 read them, SG32 sums its f
// deviations (in FP32, in the order the step kernel sums them).
template <class S, bool COHERENT = false>
__device__ __forceinline__ void pull_load(const void* base, size_t N, size_t n, float m[M_PLANES]) {
  if constexpr (S::kind == 0) {
    const float2* P = static_cast<const float2*>(base);
    const float2 a = ldx<COHERENT>(P + MP_RP * N + n), b = ldx<COHERENT>(P + MP_J * N + n);
    const float2 c = ldx<COHERENT>(P + MP_S * N + n);
    m[M_RHO] = a.x; m[M_PHI] = a.y; m[M_JX] = b.x; m[M_JY] = b.y; m[M_XX] = c.x; m[M_XY] = c.y;
  } else if constexpr (S::kind == 1) {
    const char* b = static_cast<const char*>(base);
    const M16Layout L = m16_layout(N);
    m[M_PHI] = ldx<COHERENT>(reinterpret_cast<const float*>(b + L.phi) + n);
    m[M_RHO] = __half2float(ldx<COHERENT>(reinterpret_cast<const __half*>(b + L.r) + n));
    const float2 j = __half22float2(ldx<COHERENT>(reinterpret_cast<const __half2*>(b + L.j) + n));
    const float2 s = __half22float2(ldx<COHERENT>(reinterpret_cast<const __half2*>(b + L.m) + n));
    m[M_JX] = j.x; m[M_JY] = j.y; m[M_XX] = s.x; m[M_XY] = s.y;
  } else {
    const float* F = static_cast<const float*>(base);
    float f[9], g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = ldx<COHERENT>(F + i * N + n);
    g[0] = ldx<COHERENT>(F + 9 * N + n);
    pops_to_moments(f, g, m);
  }
}

// Store the six moments of node n (SM32, SM16).
template <class S>
__device__ __forceinline__ void pull_store_moments(void* base, size_t N, size_t n, const float m[M_PLANES]) {
  if constexpr (S::kind == 0) {
    float2* P = static_cast<float2*>(base);
    P[MP_RP * N + n] = make_float2(m[M_RHO], m[M_PHI]);
    P[MP_J * N + n] = make_float2(m[M_JX], m[M_JY]);
    P[MP_S * N + n] = make_float2(m[M_XX], m[M_XY]);
  } else if constexpr (S::kind == 1) {
    char* b = static_cast<char*>(base);
    const M16Layout L = m16_layout(N);
    reinterpret_cast<float*>(b + L.phi)[n] = m[M_PHI];
    reinterpret_cast<__half*>(b + L.r)[n] = __float2half_rn(m[M_RHO]);
    reinterpret_cast<__half2*>(b + L.j)[n] = __floats2half2_rn(m[M_JX], m[M_JY]);
    reinterpret_cast<__half2*>(b + L.m)[n] = __floats2half2_rn(m[M_XX], m[M_XY]);
  }
}

// SG32: the f deviations and phi of node n.
__device__ __forceinline__ void sg_load(const void* base, size_t N, size_t n, float fd[9], float& phi) {
  const float* F = static_cast<const float*>(base);
#pragma unroll
  for (int i = 0; i < 9; ++i) fd[i] = F[i * N + n];
  phi = F[9 * N + n];
}
__device__ __forceinline__ void sg_store(void* base, size_t N, size_t n, const float fd[9], float phi) {
  float* F = static_cast<float*>(base);
#pragma unroll
  for (int i = 0; i < 9; ++i) F[i * N + n] = fd[i];
  F[9 * N + n] = phi;
}

// (rho - 1, phi) of node n as the step kernel sees it, read through L2.
template <class S>
__device__ __forceinline__ float2 pull_rho_phi(const void* base, size_t N, size_t n) {
  if constexpr (S::kind == 0) {
    return __ldcg(static_cast<const float2*>(base) + MP_RP * N + n);
  } else if constexpr (S::kind == 1) {
    const char* b = static_cast<const char*>(base);
    const M16Layout L = m16_layout(N);
    return make_float2(__half2float(__ldcg(reinterpret_cast<const __half*>(b + L.r) + n)),
                       __ldcg(reinterpret_cast<const float*>(b + L.phi) + n));
  } else {
    const float* F = static_cast<const float*>(base);
    float f[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) f[i] = __ldcg(F + i * N + n);
    return make_float2(sum9(f), __ldcg(F + 9 * N + n));
  }
}

// Sign of population i in pxx - pyy and in pxy.
__host__ __device__ constexpr int SXXd(int i) { return (i == 1 || i == 2) ? 1 : ((i == 3 || i == 4) ? -1 : 0); }
__host__ __device__ constexpr int SXYd(int i) { return (i == 5 || i == 6) ? 1 : ((i == 7 || i == 8) ? -1 : 0); }

struct MomArgs {
  Geom G;
  MomPhys Q;
  const void* src;  // the state in the storage's layout (element offsets below 2^32)
  void* dst;
  int yc;           // rows per band
};

// What a destination node has received so far: its moments (SM32, SM16), or
// its f populations (as deviations) and phi (SG32).
template <class S>
struct PullAcc {
  float r, jx, jy, xx, xy, p;
};
template <>
struct PullAcc<SG32> {
  float f[9], p;
};

// Columns produced per warp.
constexpr int kMomCols = 30;

// One warp advances columns [xo, xo + 30) of rows [y0, y1) of one lattice by
// one step (every lane of the warp calls it, with the same arguments).
// COHERENT: read src through L2 (a persistent launch whose other CTAs wrote
// src earlier in the same launch).
template <bool COHERENT, class S>
__device__ __forceinline__ void moment_strip(const Geom& G, const MomPhys& Q, const void* src_v, void* dst_v, int xo,
                                             int y0, int y1, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  constexpr int K = S::kind;
  const int nx = G.nx, ny = G.ny;
  const unsigned N = (unsigned)nx * (unsigned)ny;
  if (xo >= nx) return;                                // whole warp
  const int xl = xo - 1 + lane;                        // this lane's column before wrapping
  const int x = ((xl % nx) + nx) % nx;
  const int xm = x == 0 ? nx - 1 : x - 1;
  const int xp = x + 1 == nx ? 0 : x + 1;
  const bool edge = lane == 0 || lane == 31;
  const int xe = lane == 0 ? xm : xp;                  // outer stencil column of an edge lane
  const int xo_own_or_edge = edge ? xe : x;
  const bool store_lane = lane >= 1 && lane <= kMomCols && xl < nx;
  const bool tubed = G.tube_len > 0;
  const bool tc0 = tubed && col_in_tube(G, xm);
  const bool tc1 = tubed && col_in_tube(G, x);
  const bool tc2 = tubed && col_in_tube(G, xp);
  const bool tce = lane == 0 ? tc0 : tc2;              // the edge column lies in the tube
  const bool warp_tube = __any_sync(FULL, tc0 || tc1 || tc2);
  const bool warp_all_tube = __all_sync(FULL, tc0 && tc1 && tc2);
  // the storage's planes
  const char* __restrict__ sb = static_cast<const char*>(src_v);
  char* __restrict__ db = static_cast<char*>(dst_v);
  [[maybe_unused]] const M16Layout L16 = m16_layout(N);
  auto ldf = [&](const float* p) { return COHERENT ? __ldcg(p) : __ldg(p); };
  auto ldf2 = [&](const float2* p) { return COHERENT ? __ldcg(p) : __ldg(p); };
  auto ldh = [&](const __half* p) { return COHERENT ? __ldcg(p) : __ldg(p); };
  auto ldh2 = [&](const __half2* p) { return COHERENT ? __ldcg(p) : __ldg(p); };

  // one row of the stencil window: centre c, s = right - left and
  // d = (left - c) + (right - c) of rho and phi at this lane's column.  The
  // stored values of solid nodes are never used and may be anything: a solid
  // centre enters as 0 and solid neighbours as the centre value, so that a
  // boundary node recovers its fluid neighbours from c, s and d, then replaces
  // the solid ones by the wall ghosts.
  struct Row {
    float rc, rs, rh, pc, ps, ph;  // rh, ph hold d
  };
  // WALL: the row may hold solid nodes under this warp's columns (else the
  // solid handling is compiled out)
  auto make_row = [&](float r, float p, float re, float pe, bool in_band, auto WALL) {
    Row w;
    float rl = __shfl_up_sync(FULL, r, 1), rr = __shfl_down_sync(FULL, r, 1);
    float pl = __shfl_up_sync(FULL, p, 1), pr = __shfl_down_sync(FULL, p, 1);
    // the edge lanes' outer neighbours (selects, not branches)
    rl = lane == 0 ? re : rl;
    pl = lane == 0 ? pe : pl;
    rr = lane == 31 ? re : rr;
    pr = lane == 31 ? pe : pr;
    if (decltype(WALL)::value && warp_tube && !in_band) {
      if (tc1) {
        r = 0.f;
        p = 0.f;
      }
      if (tc0) {
        rl = r;
        pl = p;
      }
      if (tc2) {
        rr = r;
        pr = p;
      }
    }
    w.rc = r;
    w.rs = rr - rl;
    w.rh = (rl - r) + (rr - r);
    w.pc = p;
    w.ps = pr - pl;
    w.ph = (pl - p) + (pr - p);
    return w;
  };
  // j and the stresses of a node
  struct JM {
    float jx, jy, mx, my;
  };
  // rho - 1 and phi of node o; SG32 also gives the node's j and stresses, from
  // the same f (the step keeps them until the row's collision)
  auto load_node_rp = [&](unsigned o, float& rv, float& pv, JM& m) {
#ifdef LB_CHECK
    if (!lb_in(o, N)) {  // every plane holds N nodes
      rv = pv = 0.f;
      m = JM{0.f, 0.f, 0.f, 0.f};
      return;
    }
#endif
    if constexpr (K == 0) {
      const float2 v = ldf2(reinterpret_cast<const float2*>(sb) + MP_RP * N + o);
      rv = v.x;
      pv = v.y;
    } else if constexpr (K == 1) {
      pv = ldf(reinterpret_cast<const float*>(sb + L16.phi) + o);
      rv = __half2float(ldh(reinterpret_cast<const __half*>(sb + L16.r) + o));
    } else {
      const float* F = reinterpret_cast<const float*>(sb);
      float f[9], mm[6], g[9] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int i = 0; i < 9; ++i) f[i] = ldf(F + i * N + o);
      pops_to_moments(f, g, mm);
      rv = mm[M_RHO];
      pv = ldf(F + 9 * N + o);
      m = JM{mm[M_JX], mm[M_JY], mm[M_XX], mm[M_XY]};
    }
  };
  // row rowb: this lane's rho - 1, phi (and SG32 moments) and the edge column's
  // rho - 1, phi.  Solid nodes hold zeros; SG32 does not read them (ten values
  // a node), the moment storages read them rather than test for them.
  auto load_rp = [&](unsigned rowb, bool in_band, float& rv, float& pv, float& re, float& pe, JM& m) {
    re = pe = 0.f;
    if constexpr (K == 2) {
      rv = pv = 0.f;
      m = JM{0.f, 0.f, 0.f, 0.f};
      if (!(tc1 && !in_band)) load_node_rp(rowb + x, rv, pv, m);
      if (edge && !(tce && !in_band)) {
        JM unused;
        load_node_rp(rowb + xe, re, pe, unused);
      }
    } else {
      // every lane reads an "edge" value (its own node again unless it is an edge
      // lane): one more load, no divergent branch
      load_node_rp(rowb + x, rv, pv, m);
      JM unused;
      load_node_rp(rowb + xo_own_or_edge, re, pe, unused);
    }
  };
  auto load_jm = [&](unsigned rowb, bool in_band, JM& m) {
    if constexpr (K == 0 || K == 1) {
      const unsigned o = rowb + x;
#ifdef LB_CHECK
      if (!lb_in(o, N)) {
        m = JM{0.f, 0.f, 0.f, 0.f};
        return;
      }
#endif
      if constexpr (K == 0) {
        const float2 j = ldf2(reinterpret_cast<const float2*>(sb) + MP_J * N + o);
        const float2 s = ldf2(reinterpret_cast<const float2*>(sb) + MP_S * N + o);
        m = JM{j.x, j.y, s.x, s.y};
      } else {
        const float2 j = __half22float2(ldh2(reinterpret_cast<const __half2*>(sb + L16.j) + o));
        const float2 s = __half22float2(ldh2(reinterpret_cast<const __half2*>(sb + L16.m) + o));
        m = JM{j.x, j.y, s.x, s.y};
      }
    }
  };
  auto next_row = [&](int yy) { return yy + 1 == ny ? 0 : yy + 1; };

  // A slot of the three-row window: a row's stencil summaries, its index and
  // whether it lies in the tube's band.  The rows of collision row k are in
  // slots (k - 1, k, k + 1); the loop body is called with the slots (and the
  // accumulators) rotated, so that a new row lands in the slot the oldest row
  // leaves and nothing is copied between iterations.
  struct Slot {
    Row w;
    int y;
    bool rb;
  };
  Slot S0, S1, S2;
  S0.y = wrapi(y0 - 2, ny);
  S1.y = next_row(S0.y);
  S2.y = next_row(S1.y);
  S0.rb = row_in_band(G, S0.y);
  S1.rb = row_in_band(G, S1.y);
  S2.rb = row_in_band(G, S2.y);
  JM cm;     // j and stresses of the collision row
  JM stash;  // SG32: those of the row after it, taken from its f two rows ahead
  {
    float r, p, re, pe;
    JM m;
    load_rp((unsigned)S0.y * nx, S0.rb, r, p, re, pe, m);
    S0.w = make_row(r, p, re, pe, S0.rb, std::true_type{});
    load_rp((unsigned)S1.y * nx, S1.rb, r, p, re, pe, m);
    S1.w = make_row(r, p, re, pe, S1.rb, std::true_type{});
    cm = m;
    load_rp((unsigned)S2.y * nx, S2.rb, r, p, re, pe, m);
    S2.w = make_row(r, p, re, pe, S2.rb, std::true_type{});
    stash = m;
    if constexpr (K != 2) load_jm((unsigned)S1.y * nx, S1.rb, cm);
  }
  PullAcc<S> A0, A1, A2;
  if constexpr (K == 2) {
#pragma unroll
    for (int i = 0; i < 9; ++i) A0.f[i] = 0.f;
    A0.p = 0.f;
  } else {
    A0 = PullAcc<S>{0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  }
  A1 = A0;
  A2 = A0;
  const PullAcc<S> zero = A0;

  // collision row k: slots lo/mid/hi hold rows k - 1, k, k + 1; accumulators
  // a0 (row k - 1, stored here), a1 (row k) and a2 (row k + 1, started here)
  // WALL (std::true_type / std::false_type): whether walls can touch this strip's
  // rows; without, the step is compiled with no wall code at all
  auto step = [&](Slot& lo, Slot& mid, Slot& hi, PullAcc<S>& a0, PullAcc<S>& a1, PullAcc<S>& a2, int k, auto WALL) {
    constexpr bool CW = decltype(WALL)::value;
    // next rows in flight while this one collides
    const int yq = next_row(hi.y);  // row k + 2
    const bool qb = row_in_band(G, yq);
    float nr = 0.f, np = 0.f, ner = 0.f, nep = 0.f;
    JM njm = JM{0.f, 0.f, 0.f, 0.f}, qjm = JM{0.f, 0.f, 0.f, 0.f};
    if (k < y1) {
      if constexpr (K == 2) {
        njm = stash;
      } else {
        load_jm((unsigned)hi.y * nx, hi.rb, njm);
      }
      load_rp((unsigned)yq * nx, qb, nr, np, ner, nep, qjm);
    }
    // a row whose whole window is wall under every column sends and stores nothing
    const bool all_wall = CW && warp_all_tube && !lo.rb && !mid.rb && !hi.rb;
    if (!all_wall) {
      // walls can touch this warp only if it has tube columns and a row leaves the
      // band (warp-uniform); otherwise every node is fluid with fluid neighbours
      const bool walls = CW && warp_tube && !(lo.rb && mid.rb && hi.rb);
      float fs[9], ge[9];
      // populations the own node sent into a wall, returned to it (bounce-back)
      bool bounce[9] = {false, false, false, false, false, false, false, false, false};
      if (!walls) {
        float rdx, rdy, pdx, pdy, plap;
        const float rc[3] = {lo.w.rc, mid.w.rc, hi.w.rc}, rs[3] = {lo.w.rs, mid.w.rs, hi.w.rs};
        const float rh[3] = {lo.w.rh, mid.w.rh, hi.w.rh};
        const float pc[3] = {lo.w.pc, mid.w.pc, hi.w.pc}, ps[3] = {lo.w.ps, mid.w.ps, hi.w.ps};
        const float ph[3] = {lo.w.ph, mid.w.ph, hi.w.ph};
        grad_rows(rc, rs, rh, rdx, rdy);
        stencil_rows(pc, ps, ph, pdx, pdy, plap);
        collide_moment_node(Q, mid.w.rc, cm.jx, cm.jy, cm.mx, cm.my, mid.w.pc, rdx, rdy, pdx, pdy, plap, fs, ge);
      } else {
        const bool fluid = !(tc1 && !mid.rb);
        bool sol[3][3];
        bool bnd = false;
        {
          const bool tc[3] = {tc0, tc1, tc2};
          const bool rb[3] = {lo.rb, mid.rb, hi.rb};
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              sol[j][i] = tc[i] && !rb[j];
              bnd = bnd || sol[j][i];
            }
        }
        if (fluid) {
          float rdx, rdy, rlap, pdx, pdy, plap;
          float cjx = cm.jx, cjy = cm.jy;
          if (!bnd) {
            const float rc[3] = {lo.w.rc, mid.w.rc, hi.w.rc}, rs[3] = {lo.w.rs, mid.w.rs, hi.w.rs};
            const float rh[3] = {lo.w.rh, mid.w.rh, hi.w.rh};
            const float pc[3] = {lo.w.pc, mid.w.pc, hi.w.pc}, ps[3] = {lo.w.ps, mid.w.ps, hi.w.ps};
            const float ph[3] = {lo.w.ph, mid.w.ph, hi.w.ph};
            grad_rows(rc, rs, rh, rdx, rdy);
            stencil_rows(pc, ps, ph, pdx, pdy, plap);
          } else {
            // boundary node: wall ghosts on the full neighbourhood, and the rest rule
            const Row* wr[3] = {&lo.w, &mid.w, &hi.w};
            float vr[3][3], vp[3][3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
              vr[j][0] = fmaf(0.5f, wr[j]->rh - wr[j]->rs, wr[j]->rc);
              vr[j][1] = wr[j]->rc;
              vr[j][2] = fmaf(0.5f, wr[j]->rh + wr[j]->rs, wr[j]->rc);
              vp[j][0] = fmaf(0.5f, wr[j]->ph - wr[j]->ps, wr[j]->pc);
              vp[j][1] = wr[j]->pc;
              vp[j][2] = fmaf(0.5f, wr[j]->ph + wr[j]->ps, wr[j]->pc);
            }
            apply_ghosts(vr, sol, 0.f);
            apply_ghosts(vp, sol, Q.h);
            stencil3_unnorm(vr, rdx, rdy, rlap);
            stencil3_unnorm(vp, pdx, pdy, plap);
            cjx = 0.f;
            cjy = 0.f;
#pragma unroll
            for (int i = 1; i < 9; ++i) bounce[i] = sol[1 + EYd(i)][1 + EXd(i)];
          }
          collide_moment_node(Q, mid.w.rc, cjx, cjy, cm.mx, cm.my, mid.w.pc, rdx, rdy, pdx, pdy, plap, fs, ge);
        } else {
#pragma unroll
          for (int i = 0; i < 9; ++i) {
            fs[i] = 0.f;  // a solid node sends nothing
            ge[i] = 0.f;
          }
        }
      }
      // own node: the rest population, and bounce-back of what was sent into a
      // wall (all populations as deviations from w_i, which add up to 1, 0, 0, 0, 0)
      if constexpr (K == 2) {
        a1.f[0] += fs[0];
      } else {
        a1.r += fs[0];
      }
      a1.p += ge[0];
      if (walls) {
#pragma unroll
        for (int i = 1; i < 9; ++i)
          if (bounce[i]) {
            const float v = fs[i];
            if constexpr (K == 2) {
              a1.f[OPPd(i)] += v;
            } else {
              a1.r += v;
              a1.jx -= float(EXd(i)) * v;
              a1.jy -= float(EYd(i)) * v;
              a1.xx += float(SXXd(i)) * v;
              a1.xy += float(SXYd(i)) * v;
            }
            a1.p += ge[i];
          }
      }
      // populations moving in +x come from lane - 1, in -x from lane + 1
      const float f1 = __shfl_up_sync(FULL, fs[1], 1), f5 = __shfl_up_sync(FULL, fs[5], 1);
      const float f8 = __shfl_up_sync(FULL, fs[8], 1);
      const float f2 = __shfl_down_sync(FULL, fs[2], 1), f6 = __shfl_down_sync(FULL, fs[6], 1);
      const float f7 = __shfl_down_sync(FULL, fs[7], 1);
      const float g1 = __shfl_up_sync(FULL, ge[1], 1), g5 = __shfl_up_sync(FULL, ge[5], 1);
      const float g8 = __shfl_up_sync(FULL, ge[8], 1);
      const float g2 = __shfl_down_sync(FULL, ge[2], 1), g6 = __shfl_down_sync(FULL, ge[6], 1);
      const float g7 = __shfl_down_sync(FULL, ge[7], 1);
      a1.p += g1 + g2;
      a2.p = ge[3] + (g5 + g7);
      a0.p += ge[4] + (g6 + g8);
      if constexpr (K == 2) {
        // row k: 1 from x - 1, 2 from x + 1; row k + 1: 3 from here, 5 from x - 1,
        // 7 from x + 1; row k - 1: 4 from here, 8 from x - 1, 6 from x + 1
        a1.f[1] += f1;
        a1.f[2] += f2;
#pragma unroll
        for (int i = 0; i < 9; ++i) a2.f[i] = 0.f;
        a2.f[3] = fs[3];
        a2.f[5] = f5;
        a2.f[7] = f7;
        a0.f[4] += fs[4];
        a0.f[8] += f8;
        a0.f[6] += f6;
      } else {
        // row k: e = (+-1, 0)
        a1.r += f1 + f2;
        a1.jx += f1 - f2;
        a1.xx += f1 + f2;
        // row k + 1: e_y = +1 (3 from here, 5 from x - 1, 7 from x + 1)
        a2.r = fs[3] + (f5 + f7);
        a2.jx = f5 - f7;
        a2.jy = a2.r;
        a2.xx = -fs[3];
        a2.xy = f5 - f7;
        // row k - 1: e_y = -1 (4 from here, 8 from x - 1, 6 from x + 1)
        const float s4 = fs[4] + (f6 + f8);
        a0.r += s4;
        a0.jx += f8 - f6;
        a0.jy -= s4;
        a0.xx -= fs[4];
        a0.xy += f6 - f8;
      }
      // row k - 1 has received everything
      if (k > y0 && store_lane && !(tc1 && !lo.rb)) {
        const unsigned o = (unsigned)lo.y * nx + x;
#ifdef LB_CHECK
        if (lb_in(o, N))
#endif
        if constexpr (K == 0) {
          float2* P = reinterpret_cast<float2*>(db);
          P[MP_RP * N + o] = make_float2(a0.r, a0.p);
          P[MP_J * N + o] = make_float2(a0.jx, a0.jy);
          P[MP_S * N + o] = make_float2(a0.xx, a0.xy);
        } else if constexpr (K == 1) {
          reinterpret_cast<float*>(db + L16.phi)[o] = a0.p;
          reinterpret_cast<__half*>(db + L16.r)[o] = __float2half_rn(a0.r);
          reinterpret_cast<__half2*>(db + L16.j)[o] = __floats2half2_rn(a0.jx, a0.jy);
          reinterpret_cast<__half2*>(db + L16.m)[o] = __floats2half2_rn(a0.xx, a0.xy);
        } else {
          float* F = reinterpret_cast<float*>(db);
#pragma unroll
          for (int i = 0; i < 9; ++i) F[i * N + o] = a0.f[i];
          F[9 * N + o] = a0.p;
        }
      }
    } else {
      a2 = zero;
    }
    if (k < y1) {
      // row k + 2 takes the slot of row k - 1
      lo.y = yq;
      lo.rb = qb;
      lo.w = make_row(nr, np, ner, nep, qb, WALL);
      cm = njm;
      if constexpr (K == 2) stash = qjm;
    }
  };

  // Walls can touch the strip only if the warp has tube columns and one of the
  // rows y0 - 2 .. y1 + 1 leaves the band (warp-uniform).  Most strips of a long
  // tube lie inside the band, and their loop holds no wall code: compiled in, the
  // rarely taken wall path still cost the fast path about a tenth of its
  // instructions (values the compiler computes ahead of the branch).
  const int nrow = y1 - y0 + 4;
  const int d0 = ((y0 - 2 - G.tube_y0) % ny + ny) % ny;
  const bool strip_walls = warp_tube && !(d0 + nrow <= G.tube_h);
  auto run = [&](auto WALL) {
    int k = y0 - 1;
#pragma unroll 1
    while (true) {
      step(S0, S1, S2, A0, A1, A2, k, WALL);
      if (++k > y1) break;
      step(S1, S2, S0, A1, A2, A0, k, WALL);
      if (++k > y1) break;
      step(S2, S0, S1, A2, A0, A1, k, WALL);
      if (++k > y1) break;
    }
  };
  if (strip_walls)
    run(std::true_type{});
  else
    run(std::false_type{});
}

template <int NW, class S>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 3 : (NW == 4 ? 7 : 14)) moment_step_kernel(MomArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int cb, band;
  tile_of_block((a.G.nx + NW * kMomCols - 1) / (NW * kMomCols), cb, band);
  const int y0 = band * a.yc;
  moment_strip<false, S>(a.G, a.Q, a.src, a.dst, (cb * NW + warp) * kMomCols, y0, min(y0 + a.yc, a.G.ny), lane);
}

}  // namespace lbk
