// Fused step kernel with bulk-copy (TMA) staging of the populations and warp
// specialisation.
//
// Same update as step_band in lb_device.cuh (stencils, equilibria, collision,
// push streaming with bounce-back, rest-on-read), organised for sm_103a:
//   - a CTA owns BX columns and walks up a band of rows.  One producer warp
//     brings every row of all 18 population planes (plus 8 halo columns either
//     side) into a shared-memory ring of NS stages with cp.async.bulk copies,
//     signalled on a per-stage "full" mbarrier (complete_tx).  The planar
//     storages take one copy per plane and row; the 32-node block storages
//     (SF32B, SF16B) one copy per row, of the whole blocks over the tile's nodes and
//     their neighbour columns: a CTA's bulk copies, not their bytes, limited
//     the planar ring;
//   - BX/32 consumer warps work independently: each keeps rho/phi of rows
//     y-1, y, y+1 for its 32 columns in registers, takes the neighbouring
//     columns by warp shuffles (eight of its lanes share the sums of the two halo
//     columns), collides row y from the stage and pushes the result to
//     global memory, then arrives on the stage's "empty" mbarrier;
//   - a consumer warp keeps the populations of a row in registers from the
//     moment it sums that row, so it releases the stage right away; the
//     producer refills a stage once every consumer warp has released it, which
//     keeps NS - 1 rows in flight;
//     there is no CTA-wide barrier in the main loop;
//   - destinations are 32-bit element offsets from the buffer bases; the wall
//     tests use column flags computed once per thread and row flags once per row;
//   - a row that is solid under every column a warp reads (inside the tube,
//     outside the band) is not summed: the wall ghosts replace all its values;
//     a tile whose nodes are all solid exits at once.
// Requires, for the planar storages, nx % 8 == 0 (16-byte aligned rows) and
// 9 nx ny < 2^32 (32-bit offsets); the block storages take any nx with
// 18 * 32 * ceil(nx ny / 32) < 2^32 (FP32) or 19 * 32 * ceil(nx ny / 32) < 2^32 (FP16).  BX % 32 == 0.  Halo columns at the x-wrap
// come from a second 16-byte-aligned copy of the 8 elements (the block storage:
// the 32-node block) at the other end of the row.
//
// Every mbarrier wait gives up after a time limit and records the failure in
// the error word; the producer waits (also with a limit) for the copies it
// issued before it exits, so no copy lands in released shared memory.
#pragma once

#include <type_traits>

#include "lb_device.cuh"

namespace lbk {

constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// A staged value in the arithmetic type.
__device__ __forceinline__ float stage_val(float v) { return v; }
__device__ __forceinline__ double stage_val(double v) { return v; }
__device__ __forceinline__ float stage_val(__half v) { return __half2float(v); }

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait: true when the phase completed, false after the time limit.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = globaltimer_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (globaltimer_ns() - t0 > kWaitLimitNs) return false;
  }
  return true;
}

// 1-D bulk copy global -> shared, completion counted on bar (bytes % 16 == 0,
// both addresses 16-byte aligned).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

// Source of a bulk copy of cnt elements at element offset off of a buffer of
// lim elements.  In the bounds-checked build a range that leaves the buffer is
// recorded and the copy reads the buffer's start instead (same size, so the
// barrier's byte count still completes).
template <class T>
__device__ __forceinline__ const T* copy_src(const T* base, size_t off, size_t cnt, size_t lim) {
#ifdef LB_CHECK
  if (!lb_in(off + cnt - 1, lim)) return base;
#endif
  return base + off;
}

template <class S>
struct NGPlanes {
  static constexpr int value = 9;
};
template <>
struct NGPlanes<SF16> {
  static constexpr int value = 8;
};

// Bytes of one 32-node block of a block storage (0 for the planar storages).
template <class S, bool = is_blocked<S>::value>
struct BlkBytes {
  static constexpr size_t value = 0;
};
template <class S>
struct BlkBytes<S, true> {
  static constexpr size_t value = S::kBlockBytes;
};

template <int MODEL, class S, int BX, int NS>
struct TmaLayout {
  using T = typename S::T;
  using A = typename S::A;
  static constexpr bool BIN = MODEL == MODEL_BINARY;
  static constexpr bool F16 = sizeof(T) == 2;
  // 32-node blocks (SF32B, SF16B): a stage row is whole blocks, one bulk copy
  static constexpr bool BLK = is_blocked<S>::value;
  static constexpr int HALO = BLK ? 32 : 8;          // staged columns either side of the tile
  static constexpr int W = BX + 2 * HALO;            // staged columns: xb-HALO .. xb+BX+HALO-1
  static constexpr int NF = 9;
  static constexpr int NG = BIN ? NGPlanes<S>::value : 0;
  static constexpr int NG0 = (BIN && F16 && !BLK) ? 1 : 0;  // FP32 g_0 plane of the planar FP16 storage
  static constexpr size_t STAGE_T = BLK ? (size_t)(W / 32) * BlkBytes<S>::value : (size_t)(NF + NG) * W * sizeof(T);
  static constexpr size_t STAGE_G0 = (size_t)NG0 * W * sizeof(float);
  static constexpr size_t STAGE = ((STAGE_T + STAGE_G0) + 127) / 128 * 128;
  static constexpr size_t BYTES = NS * STAGE + 2 * NS * 8;
  static_assert(!BLK || BIN, "the block storage holds the binary model");
};

// Block storage, rows that need not start on a block boundary (nx % 32 != 0):
// row rowoff's staged range is the whole blocks over nodes lo .. hi, the tile's
// columns with the neighbour column on either side that is not an x-wrap, at
// stage blocks 0, 1, ...; a tile at one end of a row that does not hold the whole
// row also stages the block of the wrapped neighbour (the row's last node for the
// first tile, its first node for the last) at stage block BX / 32 + 1.  Such a
// tile's range holds at most w + 1 <= BX + 1 nodes, so at most BX / 32 + 1 blocks;
// an interior tile's at most BX / 32 + 2.
template <int BX>
struct BlkRow {
  static constexpr int kSpare = (BX / 32 + 1) * 32;  // stage column of the spare block
  int sbase;       // node at stage column 0
  unsigned span;   // nodes the range's blocks cover
  int spare_node;  // node whose block is the spare (-1: none)
  __device__ BlkRow(int rowoff, int xb, int w, int nx) {
    const int lo = rowoff + (xb > 0 ? xb - 1 : 0);
    const int hi = rowoff + (xb + w < nx ? xb + w : nx - 1);
    sbase = lo & ~31;
    span = (unsigned)(((hi >> 5) + 1) * 32 - sbase);
    spare_node = w >= nx ? -1 : (xb == 0 ? rowoff + nx - 1 : (xb + w == nx ? rowoff : -1));
  }
  // stage column of node n (in the range, else in the spare block)
  __device__ int col(int n) const {
    const unsigned d = (unsigned)(n - sbase);
    return d < span ? (int)d : kSpare + (n & 31);
  }
};

template <int MODEL, class S>
struct TmaArgs {
  Geom G;
  Phys<typename S::A> P;
  MomPhys Q;  // the pair-form constants (storages that compute in deviations)
  Buf<S> src, dst;
  int yc;
  int* err;  // set to 1 when a wait gave up
};

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The shared-memory ring of one CTA.  Staged rows are numbered by a running
// counter k across every tile (and every step) the CTA processes: row k uses
// stage k % NS and completes phase k / NS of that stage's barriers.
template <int MODEL, class S, int BX, int NS>
struct Ring {
  using L = TmaLayout<MODEL, S, BX, NS>;
  using T = typename S::T;
  unsigned char* smem;
  uint64_t* full;
  uint64_t* empty;
  __device__ T* f(int s) const { return reinterpret_cast<T*>(smem + s * L::STAGE); }
  __device__ T* g(int s) const {
    if constexpr (L::BLK)
      return reinterpret_cast<T*>(smem + s * L::STAGE) + S::kGOff;
    else
      return reinterpret_cast<T*>(smem + s * L::STAGE) + 9 * L::W;
  }
  __device__ float* g0(int s) const {
    if constexpr (L::BLK)
      return reinterpret_cast<float*>(smem + s * L::STAGE) + S::kG0;  // inside each block (SF16B)
    else
      return reinterpret_cast<float*>(smem + s * L::STAGE + L::STAGE_T);
  }
};

template <int MODEL, class S, int BX, int NS>
__device__ __forceinline__ Ring<MODEL, S, BX, NS> ring_init(unsigned char* smem) {
  using L = TmaLayout<MODEL, S, BX, NS>;
  Ring<MODEL, S, BX, NS> R;
  R.smem = smem;
  R.full = reinterpret_cast<uint64_t*>(smem + NS * L::STAGE);
  R.empty = R.full + NS;
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; ++s) {
      mbar_init(&R.full[s], 1);
      mbar_init(&R.empty[s], BX / 32);
    }
    mbar_fence_init();
  }
  __syncthreads();
  return R;
}

// Producer (one lane): stage rows y0 - 1 .. y1 of the tile starting at column xb
// as ring rows kbase, kbase + 1, ...  Returns false if a wait ran out of time;
// `issued` counts the ring rows handed to the copy engine.
template <int MODEL, class S, int BX, int NS>
__device__ bool produce_tile(const Ring<MODEL, S, BX, NS>& R, const Geom& G, const Buf<S>& src, int xb, int y0,
                             int y1, unsigned kbase, unsigned& issued) {
  using L = TmaLayout<MODEL, S, BX, NS>;
  using T = typename S::T;
  constexpr bool BIN = L::BIN;
  constexpr int W = L::W;
  const int nx = G.nx, ny = G.ny;
  const size_t N = (size_t)nx * ny;
  const int w = min(BX, nx - xb);
  const int nrows = y1 - y0 + 2;
  constexpr int H = L::HALO;
  const int lo = xb >= H ? xb - H : 0;
  const int hi = min(xb + BX + H, nx);
  const int ncols = hi - lo;
  const bool wl = xb == 0;           // left halo wraps to the row end
  const bool wr = xb + BX + H > nx;  // right halo wraps to the row start
  const int so = lo - (xb - H);      // stage column of global column lo
  const int sr = nx - (xb - H);      // stage column of the right wrap chunk
  const uint32_t ecols = (uint32_t)(ncols + (wl ? H : 0) + (wr ? H : 0));
  const uint32_t total = L::BLK ? ecols * (uint32_t)(BlkBytes<S>::value / 32)
                                : ecols * (uint32_t)sizeof(T) * (L::NF + L::NG) + (L::NG0 ? ecols * 4u : 0u);
  auto planes = [&](const T* base, int nplanes, T* dst0, size_t rowoff, uint64_t* bar) {
    const size_t lim = (size_t)nplanes * N;
    for (int i = 0; i < nplanes; ++i) {
      const size_t po = (size_t)i * N + rowoff;
      T* d = dst0 + i * W;
      bulk_g2s(d + so, copy_src(base, po + lo, (size_t)ncols, lim), (uint32_t)ncols * sizeof(T), bar);
      if (wl) bulk_g2s(d, copy_src(base, po + (nx - H), H, lim), H * sizeof(T), bar);
      if (wr) bulk_g2s(d + sr, copy_src(base, po, H, lim), H * sizeof(T), bar);
    }
  };
  // whole 32-node blocks: nodes [n0, n0 + cnt) of the row to stage column c
  [[maybe_unused]] auto blocks = [&](T* dst0, size_t n0, int cnt, int c, uint64_t* bar) {
    if constexpr (L::BLK) {
      constexpr int B = S::kBlock;
      const size_t lim = (N + 31) / 32 * B;
      bulk_g2s(dst0 + (c / 32) * B, copy_src(src.f, (n0 / 32) * B, (size_t)(cnt / 32) * B, lim),
               (uint32_t)(cnt / 32) * B * sizeof(T), bar);
    }
  };
  // every staged column inside the tube: rows outside the band are all solid and
  // their populations are never read (ghosts replace them), so they are not copied
  int d0 = xb - H - G.tube_x0;
  d0 = ((d0 % nx) + nx) % nx;
  const bool all_tube = G.tube_len > 0 && d0 + w + 2 * H <= G.tube_len;
  for (int j = 0; j < nrows; ++j) {
    const unsigned k = kbase + j;
    const int s = k % NS;
    if (k >= NS && !mbar_wait(&R.empty[s], ((k / NS) - 1) & 1)) return false;
    const int yy = wrapi(y0 - 1 + j, ny);
    if (all_tube && !row_in_band(G, yy)) {
      mbar_arrive(&R.full[s]);
      issued = k + 1;
      continue;
    }
    const size_t rowoff = (size_t)yy * nx;
    if constexpr (L::BLK) {
      if (nx % 32 != 0) {
        // rows that start inside a block: the range's whole blocks, and the block
        // of a wrapped neighbour outside it
        constexpr int B = S::kBlock;
        const BlkRow<BX> br((int)rowoff, xb, w, nx);
        const int nb = (int)(br.span / 32);
        const uint32_t bytes = (uint32_t)(nb + (br.spare_node >= 0 ? 1 : 0)) * B * (uint32_t)sizeof(T);
        const size_t lim = (N + 31) / 32 * B;
        mbar_arrive_expect_tx(&R.full[s], bytes);
        bulk_g2s(R.f(s), copy_src(src.f, (size_t)(br.sbase / 32) * B, (size_t)nb * B, lim),
                 (uint32_t)nb * B * sizeof(T), &R.full[s]);
        if (br.spare_node >= 0)
          bulk_g2s(R.f(s) + (BlkRow<BX>::kSpare / 32) * B, copy_src(src.f, (size_t)(br.spare_node / 32) * B, B, lim),
                   B * sizeof(T), &R.full[s]);
        issued = k + 1;
        continue;
      }
      mbar_arrive_expect_tx(&R.full[s], total);
      blocks(R.f(s), rowoff + lo, ncols, so, &R.full[s]);
      if (wl) blocks(R.f(s), rowoff + (nx - H), H, 0, &R.full[s]);
      if (wr) blocks(R.f(s), rowoff, H, sr, &R.full[s]);
      issued = k + 1;
      continue;
    }
    mbar_arrive_expect_tx(&R.full[s], total);
    planes(src.f, L::NF, R.f(s), rowoff, &R.full[s]);
    if (BIN) planes(src.g, L::NG, R.g(s), rowoff, &R.full[s]);
    if (L::NG0) {
      float* d = R.g0(s);
      bulk_g2s(d + so, copy_src(src.g0, rowoff + lo, (size_t)ncols, N), (uint32_t)ncols * 4u, &R.full[s]);
      if (wl) bulk_g2s(d, copy_src(src.g0, rowoff + (nx - 8), 8, N), 32u, &R.full[s]);
      if (wr) bulk_g2s(d + sr, copy_src(src.g0, rowoff, 8, N), 32u, &R.full[s]);
    }
    issued = k + 1;
  }
  return true;
}

// Producer: wait (bounded) until the last copies issued have landed, so that none
// lands in shared memory after the CTA has released it.
template <int MODEL, class S, int BX, int NS>
__device__ void drain_ring(const Ring<MODEL, S, BX, NS>& R, unsigned issued) {
  const unsigned long long t0 = globaltimer_ns();
  for (unsigned k = issued > NS ? issued - NS : 0; k < issued; ++k)
    while (!mbar_try_wait(&R.full[k % NS], (k / NS) & 1) && globaltimer_ns() - t0 < kWaitLimitNs) {
    }
}

// Consumer warp `warp` (0 .. BX/32 - 1): collide rows y0 .. y1 - 1 of the tile
// from ring rows kbase, kbase + 1, ... and push the results to dst.  Returns
// false (in every lane of the warp) if a wait ran out of time.
// Push streaming into the block storages when rows start on block boundaries
// (nx % 32 == 0): node (x, y)'s pair addresses start at rpart(y) + cpart(x), with
// rpart = (y nx / 32) * (elements per block) and cpart = (x / 32) * (elements per
// block) + 2 (x % 32), so that every destination costs one add.  FP32 blocks
// (SF32B): the pair (f_i, g_i) lies 64 i further and goes out as one 8-byte
// store.  Bounce-back as in push_node_u32: f_i and g_i always share their
// destination and direction.  lim: elements of the state.
template <int MODEL>
__device__ __forceinline__ void push_node_blk(float* __restrict__ f, unsigned long long lim, const uint32_t rpart[3],
                                              const uint32_t cpart[3], const bool sol[3][3], bool bnd,
                                              const float fs[9], const float ge[9]) {
  static_assert(MODEL == MODEL_BINARY, "the block storage holds the binary model");
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    const int ex = EXd(i), ey = EYd(i);
    const bool back = bnd && sol[1 + ey][1 + ex];
    const uint32_t base = back ? rpart[1] + cpart[1] : rpart[1 + ey] + cpart[1 + ex];
    const int di = back ? OPPd(i) : i;
    LB_GUARD((unsigned long long)base + 64 * di + 1, lim, );
    *reinterpret_cast<float2*>(f + base + 64 * di) = make_float2(fs[i], ge[i]);
  }
}

// The same for the FP16 block storage (SF16B; elements are halves, 608 per
// block): the pair (f_i - w_i, g_i), i >= 1, lies 32 + 64 (i - 1) from the node's
// pair start and goes out as one 4-byte store of two halves; f_0 (at self_f0)
// and g_0 (the FP32 float self_g0 of the g_0 base) stay at the node (direction 0
// never bounces back).  lim: halves of the state.
template <int MODEL>
__device__ __forceinline__ void push_node_blk16(__half* __restrict__ f, float* __restrict__ g0, unsigned long long lim,
                                                const uint32_t rpart[3], const uint32_t cpart[3], uint32_t self_f0,
                                                uint32_t self_g0, const bool sol[3][3], bool bnd, const float fs[9],
                                                const float ge[9]) {
  static_assert(MODEL == MODEL_BINARY, "the block storage holds the binary model");
  LB_GUARD(self_f0, lim, );
  f[self_f0] = __float2half_rn(fs[0]);
  LB_GUARD(self_g0, lim / 2 - SF16B::kG0, );
  g0[self_g0] = ge[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) {
    const int ex = EXd(i), ey = EYd(i);
    const bool back = bnd && sol[1 + ey][1 + ex];
    const uint32_t base = back ? rpart[1] + cpart[1] : rpart[1 + ey] + cpart[1 + ex];
    const int di = back ? OPPd(i) : i;
    LB_GUARD((unsigned long long)base + 32 + 64 * (di - 1) + 1, lim, );
    *reinterpret_cast<__half2*>(f + base + 32 + 64 * (di - 1)) = __floats2half2_rn(fs[i], ge[i]);
  }
}

// UROWS: block storage with rows that start inside a block (nx % 32 != 0): the
// stage columns of a lane change from row to row (a separate instantiation, so
// that aligned rows keep constant columns and no per-row work).
template <int MODEL, class S, int BX, int NS, bool UROWS = false>
__device__ bool consume_tile(const Ring<MODEL, S, BX, NS>& R, const Geom& G, const Phys<typename S::A>& P,
                             const MomPhys& Q, const Buf<S>& dst, int xb, int y0, int y1, unsigned kbase, int warp,
                             int lane) {
  using L = TmaLayout<MODEL, S, BX, NS>;
  using A = typename S::A;
  constexpr bool RAW = dev_arith<S>::value;
  constexpr bool BIN = L::BIN;
  constexpr int W = L::W;
  const int nx = G.nx, ny = G.ny;
  const size_t N = (size_t)nx * ny;
  const int w = min(BX, nx - xb);
  const int c0 = xb + warp * 32;      // first column of this warp
  const int x = c0 + lane;
  const bool act = x < xb + w;
  const int sc = x - xb + L::HALO;    // stage column of this lane's node

  auto load_pop = [&](int s, int c, A f[9], A g[9]) {
    if constexpr (L::BLK) {
      // the block storages keep (f_i, g_i) as adjacent pairs: one load each
      if constexpr (std::is_same<S, SF32B>::value) {
        S::pfg(R.f(s), nullptr, c, 0, f[0], g[0]);
      } else {
        f[0] = S::pfr(R.f(s), W, c, 0);
        g[0] = S::pg(R.g(s), R.g0(s), W, c, 0);
      }
#pragma unroll
      for (int i = 1; i < 9; ++i) S::pfg(R.f(s), nullptr, c, i, f[i], g[i]);
    } else {
#pragma unroll
      for (int i = 0; i < 9; ++i) {
        if constexpr (RAW)
          f[i] = S::pfr(R.f(s), W, c, i);
        else
          f[i] = S::pf(R.f(s), W, c, i, dst.r);  // the stage holds this lattice
      }
      if (BIN) {
#pragma unroll
        for (int i = 0; i < 9; ++i) g[i] = S::pg(R.g(s), R.g0(s), W, c, i);
      }
    }
  };
  // One row of the stencil window: this lane's rho/phi and its left/right
  // neighbours (taken once per row, when the row is summed).
  struct Row {
    A rc, rl, rr, pc, pl, pr;
  };
  // extra column of the edge lanes: left neighbour of lane 0, right of lane 31
  const int sx = lane == 0 ? sc - 1 : sc + 1;
  // One value of a staged row for the halo sums: population i >= 1 of f (isg false)
  // or g (isg true) at stage column c, addressed so that f and g take one load.
  auto halo_val = [&](int s, int c, bool isg, int i) -> A {
    if constexpr (L::BLK) {
      return stage_val(R.f(s)[S::sat(c, i) + (isg ? 1 : 0)]);  // g_i follows f_i
    } else {
      constexpr int GS = L::NG == 8 ? 1 : 0;  // planar FP16: g_1..g_8 in planes 0..7
      const typename S::T* b = isg ? R.g(s) - GS * W : R.f(s);
      return stage_val(b[i * W + c]);
    }
  };
  // population 0 of f or g (the FP16 storages keep g_0 in FP32 apart)
  auto halo_val0 = [&](int s, int c, bool isg) -> A {
    if constexpr (dev_arith<S>::value)
      return isg ? S::pg(R.g(s), R.g0(s), W, c, 0) : S::pfr(R.f(s), W, c, 0);
    else if constexpr (L::BLK)
      return stage_val(R.f(s)[S::sat(c, 0) + (isg ? 1 : 0)]);
    else
      return stage_val((isg ? R.g(s) : R.f(s))[c]);
  };
  // Sum this lane's column (f, g keep its populations for the collision), and the
  // warp's two halo columns: lanes 0..7 each take half of one of the four 9-value
  // sums (f or g of the left or the right column; lane 2k values 1..4 and value 0,
  // lane 2k + 1 values 5..8), in sum9's order, so that the halo sums equal the sums
  // the neighbouring warp or kernel forms for those nodes bit for bit; then take
  // the neighbours by shuffles.  A row solid under all the warp's columns (skip) is
  // left unread.
  // Block storage with rows that start inside a block: this lane's stage columns
  // (own node, edge column) in the row of lattice row yr.  Elsewhere they are sc, sx.
  constexpr bool BR = L::BLK && UROWS;
  [[maybe_unused]] auto row_cols = [&](int yr, int& co, int& ce) {
    const int rowoff = wrapi(yr, ny) * nx;
    const BlkRow<BX> br(rowoff, xb, w, nx);
    // a lane past the row's end stands for the wrapped column (the last active
    // lane's right neighbour); lanes further on feed no active lane
    const int xw = x < nx ? x : (x - nx < nx ? x - nx : 0);
    const int t = lane == 0 ? (x == 0 ? nx - 1 : x - 1) : x + 1;
    const int xe = t < nx ? t : (t - nx < nx ? t - nx : 0);
    co = br.col(rowoff + xw);
    ce = br.col(rowoff + xe);
  };
  auto sums = [&](int s, A f[9], A g[9], Row& Rw, bool skip, int yr) {
    if (skip) {
      Rw.rc = Rw.rl = Rw.rr = A(0);
      Rw.pc = Rw.pl = Rw.pr = A(0);
      return;
    }
    int co = sc, ce = sx;
    if constexpr (BR) row_cols(yr, co, ce);
    load_pop(s, co, f, g);
    const A r = sum9(f);
    const A p = BIN ? sum9(g) : A(0);
    int cl = warp * 32 + L::HALO - 1, cr = warp * 32 + L::HALO + 32;  // the halo columns
    if constexpr (BR) {
      cl = __shfl_sync(0xffffffffu, ce, 0);
      cr = __shfl_sync(0xffffffffu, ce, 31);
    }
    const bool isg = (lane >> 1) & 1;
    const bool part = lane < 8 && (BIN || !isg);
    const int hc = lane < 4 ? cl : cr;
    const int i0 = (lane & 1) ? 5 : 1;
    A h = A(0);
    if (part)
      h = (halo_val(s, hc, isg, i0) + halo_val(s, hc, isg, i0 + 1)) +
          (halo_val(s, hc, isg, i0 + 2) + halo_val(s, hc, isg, i0 + 3));
    const A h2 = __shfl_down_sync(0xffffffffu, h, 1);
    A t = A(0);
    if (part && !(lane & 1)) t = halo_val0(s, hc, isg) + (h + h2);
    const A re = __shfl_sync(0xffffffffu, t, lane == 31 ? 4 : 0);
    const A pe = BIN ? __shfl_sync(0xffffffffu, t, lane == 31 ? 6 : 2) : A(0);
    const A rl = __shfl_up_sync(0xffffffffu, r, 1), rr = __shfl_down_sync(0xffffffffu, r, 1);
    Rw.rc = r;
    Rw.rl = lane == 0 ? re : rl;
    Rw.rr = lane == 31 ? re : rr;
    if (BIN) {
      const A pl = __shfl_up_sync(0xffffffffu, p, 1), pr = __shfl_down_sync(0xffffffffu, p, 1);
      Rw.pc = p;
      Rw.pl = lane == 0 ? pe : pl;
      Rw.pr = lane == 31 ? pe : pr;
    }
  };

  // column data of this lane
  const int xm = x == 0 ? nx - 1 : x - 1;
  const int xp = x + 1 >= nx ? 0 : x + 1;
  const bool tubed = G.tube_len > 0;
  bool tc[3];
  tc[0] = tubed && act && col_in_tube(G, xm);
  tc[1] = tubed && act && col_in_tube(G, x);
  tc[2] = tubed && act && col_in_tube(G, xp);
  const int col[3] = {xm, x, xp};
  const bool warp_tube = __any_sync(0xffffffffu, tc[0] || tc[1] || tc[2]);
  // every column this warp reads or writes lies in the tube: its rows outside the
  // band are solid throughout
  const bool warp_all_tube = __all_sync(0xffffffffu, tc[0] && tc[1] && tc[2]);
  auto solid_row = [&](int y) { return warp_all_tube && !row_in_band(G, wrapi(y, ny)); };
  const uint32_t N32 = (uint32_t)N;
  // block storage, rows on block boundaries: the column parts of this lane's three
  // destination columns' block addresses
  constexpr bool BA = L::BLK && !UROWS;
  [[maybe_unused]] uint32_t cpart[3] = {0u, 0u, 0u};
  [[maybe_unused]] uint32_t cpart_f0 = 0u;  // SF16B: this lane's f_0 half, less its row's part
  [[maybe_unused]] uint32_t cpart_g0 = 0u;  // SF16B: this lane's g_0 float, less its row's part
  [[maybe_unused]] unsigned long long blk_lim = 0;
  if constexpr (BA) {
    constexpr int B = S::kBlock;
#pragma unroll
    for (int i = 0; i < 3; ++i) cpart[i] = (uint32_t)(col[i] >> 5) * B + 2u * (uint32_t)(col[i] & 31);
    blk_lim = (unsigned long long)(N + 31) / 32 * B;
    if constexpr (!std::is_same<S, SF32B>::value) {
      cpart_f0 = (uint32_t)(x >> 5) * B + (uint32_t)(x & 31);
      cpart_g0 = (uint32_t)(x >> 5) * SF16B::kG0Stride + (uint32_t)(x & 31);
    }
  }
  auto push = [&](const int rowb[3], const bool sol[3][3], bool bnd, const A fs[9], const A ge[9]) {
    if constexpr (BA) {
      constexpr int B = S::kBlock;
      const uint32_t rpart[3] = {(uint32_t)(rowb[0] >> 5) * B, (uint32_t)(rowb[1] >> 5) * B,
                                 (uint32_t)(rowb[2] >> 5) * B};
      if constexpr (std::is_same<S, SF32B>::value)
        push_node_blk<MODEL>(reinterpret_cast<float*>(dst.f), blk_lim, rpart, cpart, sol, bnd, fs, ge);
      else
        push_node_blk16<MODEL>(dst.f, dst.g0, blk_lim, rpart, cpart, rpart[1] + cpart_f0,
                               (uint32_t)(rowb[1] >> 5) * SF16B::kG0Stride + cpart_g0, sol, bnd, fs, ge);
    } else {
      push_node_u32<MODEL, S, RAW>(dst, N32, rowb, col, sol, bnd, fs, ge);
    }
  };

  // rows k-1, k, k+1 of the stencil window
  Row Rw[3];
  A fa[9], ga[9];  // populations of the row to collide next
  // prologue: rows y0 - 1 (stencil halo only) and y0
  for (int j = 0; j < 2; ++j) {
    const unsigned k = kbase + j;
    if (!__all_sync(0xffffffffu, mbar_wait(&R.full[k % NS], (k / NS) & 1))) return false;
    sums(k % NS, fa, ga, Rw[j + 1], solid_row(y0 - 1 + j), y0 - 1 + j);
    // the populations are in registers now: the stage can be refilled
    __syncwarp();
    if (lane == 0) mbar_arrive(&R.empty[k % NS]);
  }

  // One collision row y.  WALL (std::true_type / std::false_type): whether walls
  // can touch this tile's rows under this warp; without, the row is compiled with
  // no wall code (no solid tests, ghosts, rest rule or bounce-back), which the
  // node arithmetic does not depend on.
  auto row_step = [&](int y, auto WALL) -> bool {
    constexpr bool CW = decltype(WALL)::value;
    const unsigned kn = kbase + (y - y0) + 2;  // ring row of y + 1
    const int sn = kn % NS;
    // shift the row window and add row y + 1
    Rw[0] = Rw[1];
    Rw[1] = Rw[2];
    if (!__all_sync(0xffffffffu, mbar_wait(&R.full[sn], (kn / NS) & 1))) return false;
    A fn[9], gn[9];
    sums(sn, fn, gn, Rw[2], CW && solid_row(y + 1), y + 1);
    __syncwarp();
    if (lane == 0) mbar_arrive(&R.empty[sn]);
    A vr[3][3], vp[3][3];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      vr[j][0] = Rw[j].rl;
      vr[j][1] = Rw[j].rc;
      vr[j][2] = Rw[j].rr;
      if (BIN) {
        vp[j][0] = Rw[j].pl;
        vp[j][1] = Rw[j].pc;
        vp[j][2] = Rw[j].pr;
      }
    }
    const int yy = wrapi(y, ny);
    const int ym = yy == 0 ? ny - 1 : yy - 1;
    const int yp = yy + 1 >= ny ? 0 : yy + 1;
    const int rowb[3] = {ym * nx, yy * nx, yp * nx};
    A fs[9], ge[9];
    if constexpr (CW) {
      const bool rb[3] = {row_in_band(G, ym), row_in_band(G, yy), row_in_band(G, yp)};
      const bool fluid = act && !(tc[1] && !rb[1]);
      // walls can touch this warp's nodes only if it has tube columns and one of
      // the three rows leaves the band (warp-uniform)
      const bool walls = warp_tube && !(rb[0] && rb[1] && rb[2]);
      if (fluid) {
        bool sol[3][3];
        bool bnd = false;
        if (walls) {
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              sol[j][i] = tc[i] && !rb[j];
              bnd = bnd || sol[j][i];
            }
        } else {
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int i = 0; i < 3; ++i) sol[j][i] = false;
        }
        if constexpr (RAW)
          collide_node_f16<MODEL>(Q, vr, vp, sol, bnd, fa, fs, ge);
        else
          collide_node<MODEL, A>(P, vr, vp, sol, bnd, fa, fs, ge);
        push(rowb, sol, bnd, fs, ge);
      }
    } else {
      const bool sol[3][3] = {{false, false, false}, {false, false, false}, {false, false, false}};
      if (act) {
        if constexpr (RAW)
          collide_node_f16<MODEL>(Q, vr, vp, sol, false, fa, fs, ge);
        else
          collide_node<MODEL, A>(P, vr, vp, sol, false, fa, fs, ge);
        push(rowb, sol, false, fs, ge);
      }
    }
#pragma unroll
    for (int i = 0; i < 9; ++i) {
      fa[i] = fn[i];
      if (BIN) ga[i] = gn[i];
    }
    return true;
  };
  // walls can touch the tile under this warp only if the warp has tube columns and
  // one of the rows y0 - 1 .. y1 leaves the band (warp-uniform)
  const int nrw = y1 - y0 + 2;
  const int d0 = ((y0 - 1 - G.tube_y0) % ny + ny) % ny;
  const bool tile_walls = warp_tube && !(d0 + nrw <= G.tube_h);
  if (tile_walls) {
    for (int y = y0; y < y1; ++y)
      if (!row_step(y, std::true_type{})) return false;
  } else {
    for (int y = y0; y < y1; ++y)
      if (!row_step(y, std::false_type{})) return false;
  }
  return true;
}

// True when every node of columns [xb, xb + w) x rows [y0, y1) is solid.
__device__ __forceinline__ bool tile_all_solid(const Geom& G, int xb, int w, int y0, int y1) {
  if (G.tube_len <= 0) return false;
  int d = xb - G.tube_x0;
  if (d < 0) d += G.nx;
  if (d + w > G.tube_len) return false;
  for (int y = y0; y < y1; ++y)
    if (row_in_band(G, wrapi(y, G.ny))) return false;
  return true;
}

// Resident CTAs per SM the staged kernels are compiled for (caps their registers).
// For the block storages the count is what the SM's 228 KB of shared memory holds
// (each CTA with its 1 KB reservation), but no more than leaves 72 registers per
// thread: the FP32 blocks at 128 columns and 4 stages fit four CTAs, which gives
// 96 registers instead of the 72 of a five-CTA bound (1 % faster on 16384 x 256).
constexpr int tma_min_blocks(int bx, int ns) {
  return bx == 64 ? (ns > 4 ? 4 : 8) : (bx == 128 ? (ns > 4 ? 3 : 5) : (ns > 3 ? 2 : 3));
}
template <int MODEL, class S, int BX, int NS>
constexpr int tma_min_blocks_of() {
  using L = TmaLayout<MODEL, S, BX, NS>;
  if constexpr (L::BLK) {
    constexpr int by_smem = int(233472 / (L::BYTES + 1024));
    constexpr int by_regs = 65536 / ((BX + 32) * 72);
    constexpr int b = by_smem < by_regs ? by_smem : by_regs;
    return b < 1 ? 1 : (b > 8 ? 8 : b);
  } else {
    return tma_min_blocks(BX, NS);
  }
}

template <int MODEL, class S, int BX, int NS>
__global__ void __launch_bounds__(BX + 32, (tma_min_blocks_of<MODEL, S, BX, NS>())) step_tma_kernel(TmaArgs<MODEL, S> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Ring<MODEL, S, BX, NS> R = ring_init<MODEL, S, BX, NS>(smem);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int cb, band;
  tile_of_block((a.G.nx + BX - 1) / BX, cb, band);
  const int xb = cb * BX;
  const int y0 = band * a.yc;
  const int y1 = min(y0 + a.yc, a.G.ny);
  if (tile_all_solid(a.G, xb, min(BX, a.G.nx - xb), y0, y1)) return;  // CTA-uniform, before any barrier
  if (warp == BX / 32) {
    if (lane != 0) return;
    unsigned issued = 0;
    if (!produce_tile<MODEL, S, BX, NS>(R, a.G, a.src, xb, y0, y1, 0u, issued)) atomicExch(a.err, 1);
    drain_ring<MODEL, S, BX, NS>(R, issued);
    return;
  }
  bool ok;
  if constexpr (TmaLayout<MODEL, S, BX, NS>::BLK) {
    ok = a.G.nx % 32 != 0 ? consume_tile<MODEL, S, BX, NS, true>(R, a.G, a.P, a.Q, a.dst, xb, y0, y1, 0u, warp, lane)
                          : consume_tile<MODEL, S, BX, NS, false>(R, a.G, a.P, a.Q, a.dst, xb, y0, y1, 0u, warp, lane);
  } else {
    ok = consume_tile<MODEL, S, BX, NS>(R, a.G, a.P, a.Q, a.dst, xb, y0, y1, 0u, warp, lane);
  }
  if (!ok && lane == 0)
    atomicExch(a.err, 1);
}

}  // namespace lbk
