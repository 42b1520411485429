// Moment representation of the binary-model state and its step kernel.
//
// With the relaxation matrix of App. A every mode of f except the two stress
// modes relaxes fully to equilibrium, and g relaxes fully to g^eq (Sec. 3.1).
// The post-collision populations of a node therefore depend on its f only
// through rho, jx, jy, pxx - pyy and pxy, and on its g only through phi (plus
// the rho and phi stencils of Eq. (best)).  The state can thus be kept as six
// numbers per node instead of eighteen populations: 48 bytes per lattice update
// in FP32 (six read, six written) instead of 144.  The result is the population
// scheme's in exact arithmetic; only the rounding differs.
//
// The stored moments are those of the post-streaming populations before the
// boundary-node rest rule of Sec. 2.2, as in the population storages.  That rule
// sets j to zero and leaves rho, pxx - pyy and pxy unchanged, so it is applied
// when a boundary node is read.
//
// The binary model keeps rho close to 1 (Sec. 3.1), so the density is stored
// as rho - 1 and the populations are formed and streamed as deviations
// f_i - w_i from the rest weights w = 4/9, 1/9, 1/36 (whose contributions to
// every streamed moment cancel exactly: sum w_i = 1, sum w_i e_i = 0 and the
// stress combinations of w vanish).  Rounding then acts on numbers of the size
// of the flow, not on the populations themselves: in a nearly uniform phase
// every node rounds almost the same population the same way, and at 1/9 that
// fixed-sign error would accumulate into a drift of the interface.
//
// Step (a pull): the new moments of node r are the moments of the populations
// that arrive there, f_i(r) = f*_i(r - e_i), or f*_opp(i)(r) by bounce-back
// where r - e_i is solid; likewise g_i(r) = g^eq_i(r - e_i).  A warp owns 32
// consecutive columns and every lane collides its own node; lanes 1..30 collect
// the populations of their neighbours by warp shuffles, so a warp produces 30
// columns and its two edge lanes only supply the halo.  The warp walks up a
// band of rows: the populations of row k go to rows k - 1, k and k + 1, and row
// k - 1 is complete (and stored) once row k has been distributed.  The rho/phi
// rows of the stencil window are loaded two rows ahead of the collision, the
// remaining moments one row ahead.
#pragma once

#include "lb_device.cuh"

namespace lbk {

// Storage trait of the moment representation: six FP32 numbers per node, kept
// as three planes of N float2, (rho - 1, phi), (jx, jy) and (pxx - pyy, pxy),
// so that a node's moments take three 8-byte accesses.  M_RHO .. M_PHI name
// the six moments in the order of the C interface.
struct SM32 {
  using T = float;
  using A = float;
};
enum { M_RHO = 0, M_JX = 1, M_JY = 2, M_XX = 3, M_XY = 4, M_PHI = 5, M_PLANES = 6 };
enum { MP_RP = 0, MP_J = 1, MP_S = 2 };  // float2 planes

// The six moments of node n (rho - 1 in m[M_RHO]).
template <bool COHERENT = false>
__device__ __forceinline__ void mom_load(const float* base, size_t N, size_t n, float m[M_PLANES]) {
  const float2* P = reinterpret_cast<const float2*>(base);
  const float2 a = COHERENT ? __ldcg(P + MP_RP * N + n) : P[MP_RP * N + n];
  const float2 b = COHERENT ? __ldcg(P + MP_J * N + n) : P[MP_J * N + n];
  const float2 c = COHERENT ? __ldcg(P + MP_S * N + n) : P[MP_S * N + n];
  m[M_RHO] = a.x;
  m[M_PHI] = a.y;
  m[M_JX] = b.x;
  m[M_JY] = b.y;
  m[M_XX] = c.x;
  m[M_XY] = c.y;
}
__device__ __forceinline__ void mom_store(float* base, size_t N, size_t n, const float m[M_PLANES]) {
  float2* P = reinterpret_cast<float2*>(base);
  P[MP_RP * N + n] = make_float2(m[M_RHO], m[M_PHI]);
  P[MP_J * N + n] = make_float2(m[M_JX], m[M_JY]);
  P[MP_S * N + n] = make_float2(m[M_XX], m[M_XY]);
}

template <class S>
struct is_moments {
  static constexpr bool value = false;
};
template <>
struct is_moments<SM32> {
  static constexpr bool value = true;
};

// The six stored moments of one node's populations.
template <typename A>
__device__ __forceinline__ void pops_to_moments(const A f[9], const A g[9], A m[6]) {
  m[M_RHO] = sum9(f);
  m[M_JX] = momx(f);
  m[M_JY] = momy(f);
  m[M_XX] = (f[1] + f[2]) - (f[3] + f[4]);
  m[M_XY] = (f[5] + f[6]) - (f[7] + f[8]);
  m[M_PHI] = sum9(g);
}

// Sign of population i in pxx - pyy and in pxy.
__host__ __device__ constexpr int SXXd(int i) { return (i == 1 || i == 2) ? 1 : ((i == 3 || i == 4) ? -1 : 0); }
__host__ __device__ constexpr int SXYd(int i) { return (i == 5 || i == 6) ? 1 : ((i == 7 || i == 8) ? -1 : 0); }

// Hardware reciprocal (relative error below 2^-22), for 1/rho and omega.
__device__ __forceinline__ float rcp_fast(float v) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
  return r;
}

// Gradient and Laplacian stencils of Eq. (best) at one node, from per-row
// summaries of the 3x3 neighbourhood: c (centre), s = right - left and
// d = (left - c) + (right - c) of rows y-1 (0), y (1), y+1 (2), formed once per
// row.  The sums of Eq. (best) regrouped into differences of neighbouring
// values: dy = [(d2 - d0) + 6 (c2 - c0)] / 12 and
// lap = [(d0 + d2 + 4 d1) + 6 ((c0 - c1) + (c2 - c1))] / 6.  Neighbouring values
// are close, so those differences are exact in floating point and no large
// partial sums cancel (in a nearly uniform phase the direct sums of about
// twenty times the field value would leave a rounding error of fixed sign).
__device__ __forceinline__ void stencil_rows(const float c[3], const float sv[3], const float d[3], float& dx,
                                             float& dy, float& lap) {
  dx = (fmaf(4.f, sv[1], sv[0]) + sv[2]) * (1.f / 12.f);
  dy = fmaf(6.f, c[2] - c[0], d[2] - d[0]) * (1.f / 12.f);
  lap = fmaf(6.f, (c[0] - c[1]) + (c[2] - c[1]), fmaf(4.f, d[1], d[0] + d[2])) * (1.f / 6.f);
}

// Post-collision f and g (ge = g^eq) of one node from its moments and
// stencils: Eq. (equilibrium) for f^eq with the binary pressure of Sec. 3.1,
// g^eq of App. A, and the collision with every mode but pxx - pyy and pxy
// relaxed fully.  The equilibrium stress moments enter in closed form,
// (f^eq_1 + f^eq_2) - (f^eq_3 + f^eq_4) = (Txx - Tyy) + kappa (dx phi^2 - dy phi^2)
// and (f^eq_5 + f^eq_6) - (f^eq_7 + f^eq_8) = Txy + kappa dx phi dy phi, and each
// pair of opposite directions shares its even part.  drho = rho - 1; fs
// receives f*_i - w_i.
__device__ __forceinline__ void collide_moment_node(const Phys<float>& P, float drho, float jx, float jy, float mxx,
                                                    float mxy, float phi, float rdx, float rdy, float pdx,
                                                    float pdy, float plap, float fs[9], float ge[9]) {
  const float inv = rcp_fast(1.f + drho);
  const float ux = jx * inv, uy = jy * inv;
  const float phi2 = phi * phi;
  const float mu = fmaf(-P.kappa, plap, P.Acoef * fmaf(phi2, phi, -phi));
  float cl = __saturatef(fmaf(phi, 0.5f, 0.5f));  // liquid fraction (Eq. nu, clamped)
  if (P.lut > 0.f) cl = rintf(cl * P.lut) * P.lut_inv;  // viscosity table of App. A
  const float nu = fmaf(cl, P.nu_l - P.nu_g, P.nu_g);
  const float omega = 2.f * rcp_fast(fmaf(6.f, nu, 1.f));
  const float lam = P.lambda_scale * nu;
  // P0 - 1/3: the pressure p0 = rho/3 + A(-phi^2/2 + 3 phi^4/4) less kappa phi lap phi
  const float P0 = fmaf(-P.kappa * phi, plap, fmaf(drho, 1.f / 3.f, P.Acoef * phi2 * fmaf(0.75f, phi2, -0.5f)));
  // second moment of f^eq beyond P0 (Eq. (equilibrium) with the lambda terms)
  const float udr = fmaf(ux, rdx, uy * rdy);
  const float Txx = fmaf(jx, ux, lam * fmaf(2.f * ux, rdx, udr));
  const float Tyy = fmaf(jy, uy, lam * fmaf(2.f * uy, rdy, udr));
  const float Txy = fmaf(jx, uy, lam * fmaf(ux, rdy, uy * rdx));
  const float tr3 = (Txx + Tyy) * (1.f / 3.f);
  const float ax = 1.5f * (Txx - tr3), ay = 1.5f * (Tyy - tr3);
  const float dp = 1.5f * (fmaf(2.f, Txy, Txx + Tyy) - tr3), dm = 1.5f * (fmaf(-2.f, Txy, Txx + Tyy) - tr3);
  const float Gxx = P.kappa * pdx * pdx, Gyy = P.kappa * pdy * pdy, Gxy = P.kappa * pdx * pdy;
  const float k13 = fmaf(Gxx, 1.f / 3.f, Gyy * (-1.f / 6.f));
  const float k24 = fmaf(Gyy, 1.f / 3.f, Gxx * (-1.f / 6.f));
  const float kd = (Gxx + Gyy) * (-1.f / 24.f);
  const float kxy = Gxy * 0.25f;
  // non-equilibrium of the two stress modes, relaxed at omega
  const float c = (1.f - omega) * 0.25f;
  const float dxx = c * (mxx - (Txx - Tyy) - (Gxx - Gyy));
  const float dxy = c * (mxy - Txy - Gxy);
  // even parts of the four direction pairs, less w_i
  const float A1 = fmaf(P0 + ax, 1.f / 3.f, k13 + dxx);
  const float A3 = fmaf(P0 + ay, 1.f / 3.f, k24 - dxx);
  const float A5 = fmaf(P0 + dp, 1.f / 12.f, kd + kxy + dxy);
  const float A7 = fmaf(P0 + dm, 1.f / 12.f, kd - kxy - dxy);
  const float bx = jx * (1.f / 3.f), by = jy * (1.f / 3.f);
  const float bp = (jx + jy) * (1.f / 12.f), bm = (jy - jx) * (1.f / 12.f);
  fs[1] = A1 + bx; fs[2] = A1 - bx;
  fs[3] = A3 + by; fs[4] = A3 - by;
  fs[5] = A5 + bp; fs[6] = A5 - bp;
  fs[7] = A7 + bm; fs[8] = A7 - bm;
  fs[0] = fmaf(-2.f, (A1 + A3) + (A5 + A7), drho);
  // g^eq (App. A, dt = 1)
  const float Q = 2.f * P.M * mu;
  const float u2 = fmaf(ux, ux, uy * uy) * (1.f / 3.f);
  const float h15 = 1.5f * phi;
  const float upp = ux + uy, ump = ux - uy;
  const float B1 = fmaf(h15, fmaf(ux, ux, -u2), Q) * (1.f / 3.f);
  const float B3 = fmaf(h15, fmaf(uy, uy, -u2), Q) * (1.f / 3.f);
  const float B5 = fmaf(h15, fmaf(upp, upp, -u2), Q) * (1.f / 12.f);
  const float B7 = fmaf(h15, fmaf(ump, ump, -u2), Q) * (1.f / 12.f);
  const float px = phi * ux * (1.f / 3.f), py = phi * uy * (1.f / 3.f);
  const float pp = phi * upp * (1.f / 12.f), pm = phi * (uy - ux) * (1.f / 12.f);
  ge[1] = B1 + px; ge[2] = B1 - px;
  ge[3] = B3 + py; ge[4] = B3 - py;
  ge[5] = B5 + pp; ge[6] = B5 - pp;
  ge[7] = B7 + pm; ge[8] = B7 - pm;
  ge[0] = fmaf(-2.f, (B1 + B3) + (B5 + B7), phi);
}

struct MomArgs {
  Geom G;
  Phys<float> P;
  const float* src;  // three float2 planes of N nodes (6 N < 2^32)
  float* dst;
  int yc;            // rows per band
};

// Moments of a destination node as they accumulate.
struct MAcc {
  float r, jx, jy, xx, xy, p;
};

// Columns produced per warp.
constexpr int kMomCols = 30;

// One warp advances columns [xo, xo + 30) of rows [y0, y1) of one lattice by
// one step (every lane of the warp calls it, with the same arguments).
// COHERENT: read src through L2 (a persistent launch whose other CTAs wrote
// src earlier in the same launch).
template <bool COHERENT>
__device__ __forceinline__ void moment_strip(const Geom& G, const Phys<float>& P, const float* src_f, float* dst_f,
                                             int xo, int y0, int y1, int lane) {
  constexpr unsigned FULL = 0xffffffffu;
  const int nx = G.nx, ny = G.ny;
  const unsigned N = (unsigned)nx * (unsigned)ny;
  if (xo >= nx) return;                                // whole warp
  const int xl = xo - 1 + lane;                        // this lane's column before wrapping
  const int x = ((xl % nx) + nx) % nx;
  const int xm = x == 0 ? nx - 1 : x - 1;
  const int xp = x + 1 == nx ? 0 : x + 1;
  const bool edge = lane == 0 || lane == 31;
  const int xe = lane == 0 ? xm : xp;                  // outer stencil column of an edge lane
  const bool store_lane = lane >= 1 && lane <= kMomCols && xl < nx;
  const bool tubed = G.tube_len > 0;
  const bool tc0 = tubed && col_in_tube(G, xm);
  const bool tc1 = tubed && col_in_tube(G, x);
  const bool tc2 = tubed && col_in_tube(G, xp);
  const bool warp_tube = __any_sync(FULL, tc0 || tc1 || tc2);
  const float2* __restrict__ src = reinterpret_cast<const float2*>(src_f);
  float2* __restrict__ dst = reinterpret_cast<float2*>(dst_f);
  auto ld2 = [&](unsigned i) { return COHERENT ? __ldcg(src + i) : __ldg(src + i); };

  // one row of the stencil window: centre c, s = right - left and
  // d = (left - c) + (right - c) of rho and phi at this lane's column.  The
  // stored values of solid nodes are never used and may be anything: a solid
  // centre enters as 0 and solid neighbours as the centre value, so that a
  // boundary node recovers its fluid neighbours from c, s and d, then replaces
  // the solid ones by the wall ghosts.
  struct Row {
    float rc, rs, rh, pc, ps, ph;  // rh, ph hold d
  };
  auto make_row = [&](float r, float p, float re, float pe, bool in_band) {
    Row w;
    float rl = __shfl_up_sync(FULL, r, 1), rr = __shfl_down_sync(FULL, r, 1);
    float pl = __shfl_up_sync(FULL, p, 1), pr = __shfl_down_sync(FULL, p, 1);
    if (lane == 0) {
      rl = re;
      pl = pe;
    }
    if (lane == 31) {
      rr = re;
      pr = pe;
    }
    if (warp_tube && !in_band) {
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
  auto load_rp = [&](unsigned rowb, float& rv, float& pv, float& re, float& pe) {
    const float2 v = ld2(MP_RP * N + rowb + x);
    rv = v.x;
    pv = v.y;
    re = 0.f;
    pe = 0.f;
    if (edge) {
      const float2 e = ld2(MP_RP * N + rowb + xe);
      re = e.x;
      pe = e.y;
    }
  };
  auto load_jm = [&](unsigned rowb, float& jx, float& jy, float& mx, float& my) {
    const unsigned o = rowb + x;
    const float2 j = ld2(MP_J * N + o);
    const float2 m = ld2(MP_S * N + o);
    jx = j.x;
    jy = j.y;
    mx = m.x;
    my = m.y;
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
  float jx, jy, mx, my;  // moments of the collision row
  {
    float r, p, re, pe;
    load_rp((unsigned)S0.y * nx, r, p, re, pe);
    S0.w = make_row(r, p, re, pe, S0.rb);
    load_rp((unsigned)S1.y * nx, r, p, re, pe);
    S1.w = make_row(r, p, re, pe, S1.rb);
    load_rp((unsigned)S2.y * nx, r, p, re, pe);
    S2.w = make_row(r, p, re, pe, S2.rb);
    load_jm((unsigned)S1.y * nx, jx, jy, mx, my);
  }
  MAcc A0 = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, A1 = A0, A2 = A0;

  // collision row k: slots lo/mid/hi hold rows k - 1, k, k + 1; accumulators
  // a0 (row k - 1, stored here), a1 (row k) and a2 (row k + 1, started here)
  auto step = [&](Slot& lo, Slot& mid, Slot& hi, MAcc& a0, MAcc& a1, MAcc& a2, int k) {
    // next rows in flight while this one collides
    const int yq = next_row(hi.y);  // row k + 2
    float nr = 0.f, np = 0.f, ner = 0.f, nep = 0.f, njx = 0.f, njy = 0.f, nmx = 0.f, nmy = 0.f;
    if (k < y1) {
      load_rp((unsigned)yq * nx, nr, np, ner, nep);
      load_jm((unsigned)hi.y * nx, njx, njy, nmx, nmy);
    }
    // walls can touch this warp only if it has tube columns and a row leaves the
    // band (warp-uniform); otherwise every node is fluid with fluid neighbours
    const bool walls = warp_tube && !(lo.rb && mid.rb && hi.rb);
    float fs[9], ge[9];
    if (!walls) {
      float rdx, rdy, rlap, pdx, pdy, plap;
      const float rc[3] = {lo.w.rc, mid.w.rc, hi.w.rc}, rs[3] = {lo.w.rs, mid.w.rs, hi.w.rs};
      const float rh[3] = {lo.w.rh, mid.w.rh, hi.w.rh};
      const float pc[3] = {lo.w.pc, mid.w.pc, hi.w.pc}, ps[3] = {lo.w.ps, mid.w.ps, hi.w.ps};
      const float ph[3] = {lo.w.ph, mid.w.ph, hi.w.ph};
      stencil_rows(rc, rs, rh, rdx, rdy, rlap);
      stencil_rows(pc, ps, ph, pdx, pdy, plap);
      collide_moment_node(P, mid.w.rc, jx, jy, mx, my, mid.w.pc, rdx, rdy, pdx, pdy, plap, fs, ge);
      a1.r += fs[0];
      a1.p += ge[0];
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
        float cjx = jx, cjy = jy;
        if (!bnd) {
          const float rc[3] = {lo.w.rc, mid.w.rc, hi.w.rc}, rs[3] = {lo.w.rs, mid.w.rs, hi.w.rs};
          const float rh[3] = {lo.w.rh, mid.w.rh, hi.w.rh};
          const float pc[3] = {lo.w.pc, mid.w.pc, hi.w.pc}, ps[3] = {lo.w.ps, mid.w.ps, hi.w.ps};
          const float ph[3] = {lo.w.ph, mid.w.ph, hi.w.ph};
          stencil_rows(rc, rs, rh, rdx, rdy, rlap);
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
          apply_ghosts(vp, sol, P.h);
          stencil3(vr, rdx, rdy, rlap);
          stencil3(vp, pdx, pdy, plap);
          cjx = 0.f;
          cjy = 0.f;
        }
        collide_moment_node(P, mid.w.rc, cjx, cjy, mx, my, mid.w.pc, rdx, rdy, pdx, pdy, plap, fs, ge);
        // own node: the rest population, and bounce-back of what was sent into a
        // wall (all populations as deviations from w_i, which add up to 1, 0, 0, 0, 0)
        a1.r += fs[0];
        a1.p += ge[0];
        if (bnd) {
#pragma unroll
          for (int i = 1; i < 9; ++i)
            if (sol[1 + EYd(i)][1 + EXd(i)]) {
              const float v = fs[i];
              a1.r += v;
              a1.jx -= float(EXd(i)) * v;
              a1.jy -= float(EYd(i)) * v;
              a1.xx += float(SXXd(i)) * v;
              a1.xy += float(SXYd(i)) * v;
              a1.p += ge[i];
            }
        }
      } else {
#pragma unroll
        for (int i = 0; i < 9; ++i) {
          fs[i] = 0.f;  // a solid node sends nothing
          ge[i] = 0.f;
        }
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
    // row k: e = (+-1, 0)
    a1.r += f1 + f2;
    a1.jx += f1 - f2;
    a1.xx += f1 + f2;
    a1.p += g1 + g2;
    // row k + 1: e_y = +1 (3 from here, 5 from x - 1, 7 from x + 1)
    a2.r = fs[3] + (f5 + f7);
    a2.jx = f5 - f7;
    a2.jy = a2.r;
    a2.xx = -fs[3];
    a2.xy = f5 - f7;
    a2.p = ge[3] + (g5 + g7);
    // row k - 1: e_y = -1 (4 from here, 8 from x - 1, 6 from x + 1)
    const float s4 = fs[4] + (f6 + f8);
    a0.r += s4;
    a0.jx += f8 - f6;
    a0.jy -= s4;
    a0.xx -= fs[4];
    a0.xy += f6 - f8;
    a0.p += ge[4] + (g6 + g8);
    // row k - 1 has received everything
    if (k > y0 && store_lane && !(tc1 && !lo.rb)) {
      const unsigned o = (unsigned)lo.y * nx + x;
      dst[MP_RP * N + o] = make_float2(a0.r, a0.p);
      dst[MP_J * N + o] = make_float2(a0.jx, a0.jy);
      dst[MP_S * N + o] = make_float2(a0.xx, a0.xy);
    }
    if (k < y1) {
      // row k + 2 takes the slot of row k - 1
      lo.y = yq;
      lo.rb = row_in_band(G, yq);
      lo.w = make_row(nr, np, ner, nep, lo.rb);
      jx = njx;
      jy = njy;
      mx = nmx;
      my = nmy;
    }
  };

  int k = y0 - 1;
#pragma unroll 1
  while (true) {
    step(S0, S1, S2, A0, A1, A2, k);
    if (++k > y1) break;
    step(S1, S2, S0, A1, A2, A0, k);
    if (++k > y1) break;
    step(S2, S0, S1, A2, A0, A1, k);
    if (++k > y1) break;
  }
}

template <int NW>
__global__ void __launch_bounds__(NW * 32, NW == 8 ? 3 : (NW == 4 ? 7 : 14)) moment_step_kernel(MomArgs a) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int cb, band;
  tile_of_block((a.G.nx + NW * kMomCols - 1) / (NW * kMomCols), cb, band);
  const int y0 = band * a.yc;
  moment_strip<false>(a.G, a.P, a.src, a.dst, (cb * NW + warp) * kMomCols, y0, min(y0 + a.yc, a.G.ny), lane);
}

}  // namespace lbk
