// One kernel per full time step (both half-steps of Eqs. ss1-ss4 / Eqs.
// scheme2Deq ff.), out of place: every value is read once from HBM and
// written once, neighbours come from registers, shuffles and shared memory.
//
// (3+1)D: a block of 480 threads covers a 34 x 28 tile of cells in (x, y)
// and marches along z; every thread updates two cells stacked in y (rows ly,
// ly + 1), so the y neighbour inside the pair comes from registers.  Columns
// 0, 33 and rows 0, 27 are a one-cell halo: they load and compute the upper
// half-step like every other cell, so the new upper values the 32 x 26
// interior needs from outside the tile exist in shared memory, but they store
// nothing.  Per z level k the block
//   1. holds the old A(k+1), C(k+1), D(k+1) and B(k) (B, C sit at z+1/2) in
//      registers, loaded while level k-1 was computed, publishes C(k+1) and
//      D(k+1) in shared memory and starts the loads of level k+1,
//   2. (the old C(k), D(k) and the new A(k), B(k-1) are in shared memory,
//      every tile double-buffered by level parity),
//   3. computes the new A(k+1) and B(k)      (upper half-step, t -> t+dt/2),
//   4. publishes them,
//   5. computes the new C(k) and D(k)        (lower half-step, t -> t+dt),
// A run of levels starts one level early to rebuild that state (the upper
// half-step of that level only).  (Build option DIRAC_YPAIR=0: one cell per
// thread, 34 x 15 tiles of 512 threads, two blocks per SM.)
//
// (2+1)D: each warp owns a strip of 32 cells in x (30 interior) and marches
// along y with the same pipeline (u0 ~ A, u1 ~ B, v1 ~ C, v0 ~ D with y as the
// marching axis); x neighbours come from warp shuffles, no block barrier.
//
// Scheduling: the grid holds the blocks that fit on the GPU at once (fewer
// for small grids); these persistent workers (blocks in (3+1)D, warps in
// (2+1)D) take work items round-robin.  An item is one tile over one chunk of
// levels, ordered chunk-major and tile-minor, so every round processes
// neighbouring tiles at the same levels at the same time and the overlapping
// halo loads hit L2.  The chunk length balances full rounds against the one
// restart level of each item.
//
// Cells outside the grid (ragged last tiles) are wrapped periodically, so
// they compute correct duplicates and only the owning interior thread stores.
#include "kernels.cuh"

namespace dirac {

namespace {

// (3+1)D tile geometry (build-time choice).  DIRAC_YPAIR=1 (default): every
// thread updates two cells stacked in y, a 34 x 28 tile in 480 threads, one
// block per SM.  DIRAC_YPAIR=0: one cell per thread, a 34 x DIRAC_TILE_ROWS
// tile (15 rows: 512 threads, two blocks per SM; 30 rows: 1024 threads, one).
#ifndef DIRAC_YPAIR
#define DIRAC_YPAIR 1
#endif
#ifndef DIRAC_TILE_ROWS
#define DIRAC_TILE_ROWS 15
#endif
#ifndef DIRAC_PAIRS
#define DIRAC_PAIRS 14
#endif

#if DIRAC_YPAIR
constexpr int kPairs = DIRAC_PAIRS;     // row pairs per tile
constexpr int TW = 34, TH = 2 * kPairs;  // (3+1)D tile in cells
constexpr int CX = TW - 2, CY = TH - 2;  // interior
constexpr int kThreads3d = 32 * kPairs + 32;  // interior warps + one warp of halo columns and spares
constexpr int kBlocks3d = kPairs <= 7 ? 2 : 1;  // resident blocks per SM the registers are planned for
constexpr int kSmemRows = TH + 2;       // TH rows + the spare threads' pair of rows
static_assert(2 * kPairs <= 32 && 2 * kPairs + 4 <= 32, "halo columns and spares fill one warp");
#else
constexpr int TW = 34, TH = DIRAC_TILE_ROWS;  // (3+1)D tile in threads
constexpr int CX = TW - 2, CY = TH - 2; // interior
constexpr int kThreads3d = TH == 15 ? 512 : 1024;
constexpr int kBlocks3d = TH == 15 ? 2 : 1;  // resident blocks per SM the registers are planned for
constexpr int kSmemRows = TH + 1;       // TH rows + the spare threads' row
static_assert(32 * CY + 2 * TW + 2 * CY <= kThreads3d && kThreads3d - 32 * CY - 2 * TW - 2 * CY < TW,
              "interior rows as warps, the halo ring and fewer than a row of spare threads");
#endif

template <class T>
__device__ __forceinline__ T ld(const T* p) { return __ldg(p); }

__device__ __forceinline__ float2 shfl_up1(float2 v) {
  return make_float2(__shfl_up_sync(0xffffffffu, v.x, 1), __shfl_up_sync(0xffffffffu, v.y, 1));
}
__device__ __forceinline__ float2 shfl_down1(float2 v) {
  return make_float2(__shfl_down_sync(0xffffffffu, v.x, 1), __shfl_down_sync(0xffffffffu, v.y, 1));
}

__device__ __forceinline__ int wrapi(int i, int n) {
  i %= n;
  return i < 0 ? i + n : i;
}

constexpr int kSlots = kSmemRows * TW;  // shared-memory slots per plane tile
// sC, sD, sB, sA: [level parity][sublattice][slot]
constexpr size_t kSmem3d = (size_t)4 * 2 * 2 * kSlots * sizeof(float2);

// The eight values of one level load: A, C, D at level k+1 and B at level k.
template <class C>
struct LevelLoad {
  C A0, A1, B0, B1, C0, C1, D0, D1;
};

#if DIRAC_YPAIR
// Thread geometry inside the (3+1)D tile (two cells per thread, rows ly and
// ly + 1).  Warps 0..13 hold the columns 1..32 (lane -> x) of the row pairs
// (0,1), (2,3), .., (26,27); rows 0 and 27 are halo rows, so warp 0's lower
// cell and warp 13's upper cell are halo cells.  Warp 14 holds the halo
// columns 0 and 33 of every row pair (28 threads) and four spare threads
// (rows 28, 29 of shared memory, never stored).  Halo cells take part in the
// upper half-step only, whose values the interior needs.
struct Thread3d {
  int slot;                // the lower cell's shared-memory slot, ly * TW + lx (upper: slot + TW)
  int lx, ly;              // position of the lower cell in the 34 x 28 tile
  int sym, syp;            // slots of the lower cell's y- and the upper cell's y+ neighbour
                           // (clamped at the tile edge: halo cells then read their own slot)
  int sxm, sxp;            // x- / x+ neighbour of the lower cell (clamped likewise; + TW: the upper cell's)
  bool halo;               // warp-uniform: halo columns and spares (upper half-step only)
  bool h0, h1;             // warp-uniform: the lower / upper cell is a halo cell
};

__device__ __forceinline__ Thread3d thread3d() {
  Thread3d th;
  const int t = threadIdx.x, w = t >> 5;
  if (w < kPairs) {
    th.lx = (t & 31) + 1;
    th.ly = 2 * w;
    th.halo = false;
  } else {
    const int h = t - 32 * kPairs;
    th.halo = true;
    if (h < kPairs) { th.lx = 0; th.ly = 2 * h; }
    else if (h < 2 * kPairs) { th.lx = TW - 1; th.ly = 2 * (h - kPairs); }
    else { th.lx = h - 2 * kPairs; th.ly = TH; }  // spare: rows of their own
  }
  th.h0 = th.halo || th.ly == 0;
  th.h1 = th.halo || th.ly + 1 == TH - 1;
  th.slot = th.ly * TW + th.lx;
  th.sxm = th.lx > 0 ? th.slot - 1 : th.slot;
  th.sxp = th.lx < TW - 1 ? th.slot + 1 : th.slot;
  th.sym = th.ly > 0 ? th.slot - TW : th.slot;
  th.syp = th.ly + 2 < kSmemRows ? th.slot + 2 * TW : th.slot + TW;
  return th;
}
#else
// Thread geometry inside the (3+1)D tile.  Warps 0..12 hold the 13 interior
// rows, one aligned row of 32 cells each (lane -> x).  Warps 13..15 hold the
// 94 halo cells (rows 0 and 14, columns 0 and 33) and two spare threads; they
// only take part in the upper half-step, whose values the interior needs.
struct Thread3d {
  int slot;                // this cell's shared-memory slot, ly * TW + lx
  int lx, ly;              // position in the 34 x 15 tile
  int sxm, sxp, sym, syp;  // slots of the x/y neighbours (clamped at the tile
                           // edge: halo cells then read their own slot, values never used)
  bool halo;               // warp-uniform
};

__device__ __forceinline__ Thread3d thread3d() {
  Thread3d th;
  const int t = threadIdx.x, w = t >> 5;
  if (w < CY) {
    th.lx = (t & 31) + 1;
    th.ly = w + 1;
    th.halo = false;
  } else {
    const int h = t - 32 * CY;
    th.halo = true;
    if (h < TW) { th.lx = h; th.ly = 0; }
    else if (h < 2 * TW) { th.lx = h - TW; th.ly = TH - 1; }
    else if (h < 2 * TW + CY) { th.lx = 0; th.ly = h - 2 * TW + 1; }
    else if (h < 2 * TW + 2 * CY) { th.lx = TW - 1; th.ly = h - 2 * TW - CY + 1; }
    else { th.lx = h - 2 * TW - 2 * CY; th.ly = kSmemRows - 1; }  // spare: a row of its own
  }
  th.slot = th.ly * TW + th.lx;
  th.sxm = th.lx > 0 ? th.slot - 1 : th.slot;
  th.sxp = th.lx < TW - 1 ? th.slot + 1 : th.slot;
  th.sym = th.ly > 0 ? th.slot - TW : th.slot;
  th.syp = th.ly < kSmemRows - 1 ? th.slot + TW : th.slot;
  return th;
}

#endif

// work items of a (3+1)D launch: tiles x chunks of the `levels` updated levels
__host__ __device__ __forceinline__ long long items3d(const int (&N)[3], int levels, int chunk) {
  return (long long)((N[0] + CX - 1) / CX) * ((N[1] + CY - 1) / CY) * ((levels + chunk - 1) / chunk);
}

#if DIRAC_YPAIR
// One work item (one tile over one chunk of z levels) of one simulation, two
// cells per thread stacked in y: cell 0 at row ly, cell 1 at row ly + 1.  The
// y neighbour of a cell inside the pair comes from the other cell's registers;
// the pair's outer y neighbours and all x neighbours come from shared memory.
// `a` may live in the constant bank (kernel parameter) or in shared memory.
template <class P, int COEF, int LINK>
__device__ __forceinline__ void fused3d_item(const FusedArgs<P>& a, long long item, const Thread3d& th,
                                             unsigned char* smem_raw, double* e_acc) {
  using C = typename P::cplx;
  // every tile is double-buffered by level parity: slot [k & 1] holds level k
  C (*sC)[2][kSlots] = reinterpret_cast<C (*)[2][kSlots]>(smem_raw);  // old C(k)
  C (*sD)[2][kSlots] = sC + 2;                                         // old D(k)
  C (*sB)[2][kSlots] = sC + 4;                                         // new B(k)
  C (*sA)[2][kSlots] = sC + 6;                                         // new A(k)
  const int s0 = th.slot, s1 = th.slot + TW;  // the pair's slots
  const int lx = th.lx, ly = th.ly;
  const int xm0 = th.sxm, xp0 = th.sxp, xm1 = th.sxm + TW, xp1 = th.sxp + TW;
  const int sym = th.sym, syp = th.syp;
  const int Nx = a.N[0], Ny = a.N[1], Nz = a.N[2];
  // global level of the stored level k (wrapped on the global grid), for the
  // fields; zorg + k lies in [-1, 2 Nzg) (zorg in [-1, Nzg), k <= N[2] <= Nzg + 1)
  auto gz = [&](int k) {
    const int g = a.zorg + k;
    return g < 0 ? g + a.Nzg : (g >= a.Nzg ? g - a.Nzg : g);
  };
  const int tiles_x = (Nx + CX - 1) / CX;
  const long long tiles = (long long)tiles_x * ((Ny + CY - 1) / CY);
  const bool iso = a.iso != 0;
  // value offsets inside a plane: 32-bit (the host runs the fused kernels
  // only on grids of fewer than 2^31 cells), so an address is one wide
  // multiply-add
  using Off = unsigned;
  const Off nxy = (Off)Nx * (Off)Ny;
  const bool want_e = a.e_partials != nullptr;
  {
    const long long chunk = item / tiles, tile = item - chunk * tiles;
    const int z0 = a.zlo + (int)chunk * a.chunk;
    const int z1 = min(a.zlo + a.nzu, z0 + a.chunk);
    const int gx = (int)(tile % tiles_x) * CX + lx - 1;
    const int gy0 = (int)(tile / tiles_x) * CY + ly - 1, gy1 = gy0 + 1;
    const int x = wrapi(gx, Nx), y0 = wrapi(gy0, Ny), y1 = wrapi(gy1, Ny);
    const bool xin = lx >= 1 && lx <= CX && gx < Nx;
    const bool core0 = xin && !th.h0 && gy0 < Ny;
    const bool core1 = xin && !th.h1 && gy1 < Ny;
    const Off cxy0 = (Off)y0 * (Off)Nx + (Off)x, cxy1 = (Off)y1 * (Off)Nx + (Off)x;
    const int hx = 2 * x, hy0 = 2 * y0, hy1 = 2 * y1;
    // COEF_SOFTCORE: the x-y part of R = |x - c|^2 + a^2 of each cell of the
    // pair, as (hi, lo) pairs of two values: lanes (A0/C0, A1/C1) at (hx, hy),
    // (hx+1, hy+1) and (B0/D0, B1/D1) at (hx+1, hy), (hx, hy+1), kept in
    // shared memory (one record per thread and cell) so that they take no
    // registers through the z-march
    constexpr bool kSoft = COEF == COEF_SOFTCORE || COEF == COEF_SOFTCORR;
    __shared__ __align__(16) float4 sRxy[kSoft ? kThreads3d : 1][2][2];
    if constexpr (kSoft) {
      const float2 x0 = __ldg(a.hu.sc_sq[0] + hx), x1 = __ldg(a.hu.sc_sq[0] + hx + 1);
#pragma unroll
      for (int c = 0; c < 2; ++c) {
        const int hy = c ? hy1 : hy0;
        const float2 ya = __ldg(a.hu.sc_sq[1] + hy), yb = __ldg(a.hu.sc_sq[1] + hy + 1);
        const float2 d00 = padd(x0, ya), d11 = padd(x1, yb), a10 = padd(x1, ya), a01 = padd(x0, yb);
        sRxy[threadIdx.x][c][0] = make_float4(d00.x, d11.x, d00.y, d11.y);
        sRxy[threadIdx.x][c][1] = make_float4(a10.x, a01.x, a10.y, a01.y);
      }
    }
    // Per-level field constants, the same for the whole block, staged in
    // shared memory by threads 0..6 with copies that bypass the registers,
    // double-buffered by level parity (level k's copies are issued after the
    // first barrier of level k-1, when no thread reads that parity any more,
    // and waited for before the first barrier of level k):
    //   sLk[p][0..3]: plane-wave link factors along z (LINK_PLANE, table axis z)
    //                 of A (upper half, Z = 2zn), B (upper, 2zk+1), C (lower,
    //                 2zk+1), D (lower, 2zk)
    //   sZq[p][0..2]: soft-core z terms sc_sq[2][Z] of Z = 2zn, 2zk+1, 2zk
    using PL = typename PlaneLinkOf<P>::type;
    __shared__ __align__(16) PL sLk[2][4];
    __shared__ __align__(16) float2 sZq[2][3];
    // (the (3+1)D launchers run a plane wave along z polarised along x as
    // LINK_PLANE_ZX and send other plane waves to the general path)
    constexpr bool lk_z = LINK == LINK_PLANE_ZX;
    auto stage_level = [&](int k) {
      const int tid = threadIdx.x;
      if (tid >= 7) return;
      const int p = k & 1;
      const int zk = gz(k), zn = gz(k + 1);  // global levels: the tables are indexed by global Z
      if constexpr (LINK == LINK_PLANE_ZX) {
        if (tid < 4) {
          const int Z = tid == 0 ? 2 * zn : (tid == 3 ? 2 * zk : 2 * zk + 1);
          const PL* tab = static_cast<const PL*>(tid < 2 ? a.hu.ltab : a.hl.ltab);
          static_assert(sizeof(PL) % 16 == 0, "16-byte copies");
          for (int q = 0; q < (int)(sizeof(PL) / 16); ++q)
            cp_async16(reinterpret_cast<char*>(&sLk[p][tid]) + 16 * q,
                       reinterpret_cast<const char*>(tab + Z) + 16 * q);
        }
      }
      if constexpr (kSoft) {
        if (tid >= 4) {
          const int Z = tid == 4 ? 2 * zn : (tid == 5 ? 2 * zk + 1 : 2 * zk);
          cp_async8(&sZq[p][tid - 4], a.hu.sc_sq[2] + Z);
        }
      }
      cp_async_commit();
    };
    // the coefficients of a pair of values of cell c with the x-y parts
    // (Rh, Rl), the z term z and positions H0, H1 (softcore_R's sums, same order)
    auto pair_b = [&](const HalfFields<P>& h, int c, int which, float2 z, const int (&H0)[3],
                      const int (&H1)[3], float4 (&b)[2]) {
      if constexpr (COEF == COEF_SOFTCORE) {
        const float4 r = sRxy[threadIdx.x][c][which];  // which: 0 = (A, C) pairs, 1 = (B, D) pairs
        const float2 Rh = make_float2(r.x, r.y), Rl = make_float2(r.z, r.w);
        const float2 t0 = softcore_t0(h, H0), t1 = softcore_t0(h, H1);
        const SoftB2 bb = softcore_b2(padd(Rh, f2(z.x)), padd(Rl, f2(z.y)), make_float2(t0.x, t1.x),
                                      make_float2(t0.y, t1.y), h.sc_K_hi, h.sc_K_lo);
        b[0] = lane_b(bb, 0);
        b[1] = lane_b(bb, 1);
      }
    };
    // COEF_SOFTCORR: the FP32 estimates of a pair plus the two values' words w0, w1
    // of the correction record (R summed in softcore_R's order)
    auto pair_bc = [&](const HalfFields<P>& h, int c, int which, float2 z, const int (&H0)[3],
                       const int (&H1)[3], long long rec, int slot, float4 (&b)[2]) {
      if constexpr (COEF == COEF_SOFTCORR) {
        // the pair's two words of the level's correction record (read where used)
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(a.hu.sc_corr + 8 * rec + slot));
        const float4 r = sRxy[threadIdx.x][c][which];
        const float2 Rh = padd(make_float2(r.x, r.y), f2(z.x)), Rl = padd(make_float2(r.z, r.w), f2(z.y));
        float2 re, im;
        softcore_fast2(Rh, Rl, make_float2(softcore_t0(h, H0).x, softcore_t0(h, H1).x), h.sc_K_hi, re, im);
        const float2 c0 = corr_decode(w.x), c1 = corr_decode(w.y);
        b[0] = make_float4(re.x, c0.x, im.x, c0.y);
        b[1] = make_float4(re.y, c1.x, im.y, c1.y);
      }
    };
    constexpr bool kPre = kSoft;  // coefficients computed in pairs

    auto load = [&](int k, LevelLoad<C>& l0, LevelLoad<C>& l1) {
      const int zk = k < 0 ? k + Nz : k;
      const int zn = k + 1 >= Nz ? k + 1 - Nz : k + 1;
      const Off ok0 = (Off)zk * nxy + cxy0, on0 = (Off)zn * nxy + cxy0;
      const Off ok1 = (Off)zk * nxy + cxy1, on1 = (Off)zn * nxy + cxy1;
      l0.A0 = ld(a.in[0] + on0);
      l1.A0 = ld(a.in[0] + on1);
      l0.A1 = ld(a.in[1] + on0);
      l1.A1 = ld(a.in[1] + on1);
      l0.B0 = ld(a.in[2] + ok0);
      l1.B0 = ld(a.in[2] + ok1);
      l0.B1 = ld(a.in[3] + ok0);
      l1.B1 = ld(a.in[3] + ok1);
      l0.C0 = ld(a.in[4] + on0);
      l1.C0 = ld(a.in[4] + on1);
      l0.C1 = ld(a.in[5] + on0);
      l1.C1 = ld(a.in[5] + on1);
      l0.D0 = ld(a.in[6] + on0);
      l1.D0 = ld(a.in[6] + on1);
      l0.D1 = ld(a.in[7] + on0);
      l1.D1 = ld(a.in[7] + on1);
    };

    {  // old C, D of level z0-1 (the z- neighbours of the first level)
      const int p = (z0 - 1) & 1;
      const Off zo = (Off)wrapi(z0 - 1, Nz) * nxy;
      const Off o0 = zo + cxy0, o1 = zo + cxy1;
      sC[p][0][s0] = ld(a.in[4] + o0);
      sC[p][1][s0] = ld(a.in[5] + o0);
      sD[p][0][s0] = ld(a.in[6] + o0);
      sD[p][1][s0] = ld(a.in[7] + o0);
      sC[p][0][s1] = ld(a.in[4] + o1);
      sC[p][1][s1] = ld(a.in[5] + o1);
      sD[p][0][s1] = ld(a.in[6] + o1);
      sD[p][1][s1] = ld(a.in[7] + o1);
    }
    LevelLoad<C> c0, c1;  // the level loads of the two cells
    load(z0 - 1, c0, c1);
    constexpr bool kStage = LINK == LINK_PLANE_ZX || kSoft;
    if (kStage) stage_level(z0 - 1);

    for (int k = z0 - 1; k < z1; ++k) {
      const int zk = k < 0 ? k + Nz : k;
      const int zn = k + 1 >= Nz ? k + 1 - Nz : k + 1;
      const Off ok0 = (Off)zk * nxy + cxy0, on0 = (Off)zn * nxy + cxy0;
      const Off ok1 = (Off)zk * nxy + cxy1, on1 = (Off)zn * nxy + cxy1;
      const int pk = k & 1, pn = (k + 1) & 1, pm = (k - 1) & 1;
      const int Zk = 2 * gz(k), Zn = 2 * gz(k + 1);  // half-lattice z of levels k, k+1 (global)
      sC[pn][0][s0] = c0.C0;  // old C(k+1), D(k+1): z+ / x,y neighbours now,
      sC[pn][1][s0] = c0.C1;  // own old values at the next level
      sD[pn][0][s0] = c0.D0;
      sD[pn][1][s0] = c0.D1;
      sC[pn][0][s1] = c1.C0;
      sC[pn][1][s1] = c1.C1;
      sD[pn][0][s1] = c1.D0;
      sD[pn][1][s1] = c1.D1;
      // prefetch the next level while this one computes
      LevelLoad<C> n0 = c0, n1 = c1;
      if (k + 1 < z1) load(k + 1, n0, n1);
      if (kStage && threadIdx.x < 7) cp_async_wait_all();  // this level's staged constants
      __syncthreads();
      if (kStage && k + 1 < z1) stage_level(k + 1);
      const PL* lkA = lk_z ? &sLk[pk][0] : nullptr;  // compile-time choice: a shared-memory address
      const PL* lkB = lk_z ? &sLk[pk][1] : nullptr;

      // upper half-step: A(k+1) from C(k+1), C(k), D(k+1); B(k) from D(k+1), D(k), C(k)
      const C oC00 = sC[pk][0][s0], oC10 = sC[pk][1][s0];  // old C(k) of cell 0
      const C oC01 = sC[pk][0][s1], oC11 = sC[pk][1][s1];  // and of cell 1
      C nA0n0, nA1n0, nB0k0, nB1k0, nA0n1, nA1n1, nB0k1, nB1k1;
      float4 bv[2];
      {  // cell 0
        const int H0[3] = {hx, hy0, Zn}, H1[3] = {hx + 1, hy0 + 1, Zn};
        if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hu, 0, 0, sZq[pk][0], H0, H1, bv);
        if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hu, 0, 0, sZq[pk][0], H0, H1, ok0, 0, bv);
        C nb0[6] = {c0.D0, sD[pn][0][xm0], c0.D1, sD[pn][1][sym], c0.C0, oC00};
        nA0n0 = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 0, c0.A0, nb0, H0, on0, a.pstride,
                                              nullptr, kPre ? &bv[0] : nullptr, lkA);
        C nb1[6] = {sD[pn][1][xp0], c0.D1, c1.D0, c0.D0, c0.C1, oC10};
        nA1n0 = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 1, c0.A1, nb1, H1, on0, a.pstride,
                                              nullptr, kPre ? &bv[1] : nullptr, lkA);
      }
      {  // cell 1
        const int H0[3] = {hx, hy1, Zn}, H1[3] = {hx + 1, hy1 + 1, Zn};
        if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hu, 1, 0, sZq[pk][0], H0, H1, bv);
        if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hu, 1, 0, sZq[pk][0], H0, H1, ok1, 0, bv);
        C nb0[6] = {c1.D0, sD[pn][0][xm1], c1.D1, c0.D1, c1.C0, oC01};
        nA0n1 = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 0, c1.A0, nb0, H0, on1, a.pstride,
                                              nullptr, kPre ? &bv[0] : nullptr, lkA);
        C nb1[6] = {sD[pn][1][xp1], c1.D1, sD[pn][0][syp], c1.D0, c1.C1, oC11};
        nA1n1 = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 1, c1.A1, nb1, H1, on1, a.pstride,
                                              nullptr, kPre ? &bv[1] : nullptr, lkA);
      }
      {  // cell 0
        const int H0[3] = {hx + 1, hy0, Zk + 1}, H1[3] = {hx, hy0 + 1, Zk + 1};
        if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hu, 0, 1, sZq[pk][1], H0, H1, bv);
        if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hu, 0, 1, sZq[pk][1], H0, H1, ok0, 2, bv);
        C nb0[6] = {sC[pk][0][xp0], oC00, oC10, sC[pk][1][sym], c0.D0, sD[pk][0][s0]};
        nB0k0 = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 2, c0.B0, nb0, H0, ok0, a.pstride,
                                              nullptr, kPre ? &bv[0] : nullptr, lkB);
        C nb1[6] = {oC10, sC[pk][1][xm0], oC01, oC00, c0.D1, sD[pk][1][s0]};
        nB1k0 = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 3, c0.B1, nb1, H1, ok0, a.pstride,
                                              nullptr, kPre ? &bv[1] : nullptr, lkB);
      }
      {  // cell 1
        const int H0[3] = {hx + 1, hy1, Zk + 1}, H1[3] = {hx, hy1 + 1, Zk + 1};
        if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hu, 1, 1, sZq[pk][1], H0, H1, bv);
        if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hu, 1, 1, sZq[pk][1], H0, H1, ok1, 2, bv);
        C nb0[6] = {sC[pk][0][xp1], oC01, oC11, oC10, c1.D0, sD[pk][0][s1]};
        nB0k1 = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 2, c1.B0, nb0, H0, ok1, a.pstride,
                                              nullptr, kPre ? &bv[0] : nullptr, lkB);
        C nb1[6] = {oC11, sC[pk][1][xm1], sC[pk][0][syp], oC01, c1.D1, sD[pk][1][s1]};
        nB1k1 = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 3, c1.B1, nb1, H1, ok1, a.pstride,
                                              nullptr, kPre ? &bv[1] : nullptr, lkB);
      }
      sB[pk][0][s0] = nB0k0;
      sB[pk][1][s0] = nB1k0;
      sA[pn][0][s0] = nA0n0;
      sA[pn][1][s0] = nA1n0;
      sB[pk][0][s1] = nB0k1;
      sB[pk][1][s1] = nB1k1;
      sA[pn][0][s1] = nA0n1;
      sA[pn][1][s1] = nA1n1;
      __syncthreads();

      // lower half-step: C(k) from A(k+1), A(k), B(k); D(k) from B(k), B(k-1), A(k)
      // (interior cells only: nothing needs the halo's lower values; the
      // first level of a run only rebuilds A(z0) and B(z0-1))
      if (!th.halo) {
        auto n2 = [](C v) { return fmaf(v.x, v.x, v.y * v.y); };
        if (k >= z0) {
          const C nA00 = sA[pk][0][s0], nA10 = sA[pk][1][s0];  // new A(k) of cell 0
          const C nA01 = sA[pk][0][s1], nA11 = sA[pk][1][s1];  // and of cell 1
          const PL* lkC = lk_z ? &sLk[pk][2] : nullptr;
          const PL* lkD = lk_z ? &sLk[pk][3] : nullptr;
          if (!th.h0) {  // cell 0 (warp-uniform; one block of code per cell: computing
                         // the halo cells too, to interleave the two cells, was slower)
            C nC0, nC1, nD0, nD1, S;
            const bool acc = want_e && core0;  // this cell's new values count towards E
            float lc = 0.0f;
            {
              const int H0[3] = {hx, hy0, Zk + 1}, H1[3] = {hx + 1, hy0 + 1, Zk + 1};
              if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hl, 0, 0, sZq[pk][1], H0, H1, bv);
              if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hl, 0, 0, sZq[pk][1], H0, H1, ok0, 4, bv);
              C nb0[6] = {nB0k0, sB[pk][0][xm0], nB1k0, sB[pk][1][sym], nA0n0, nA00};
              nC0 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 4, oC00, nb0, H0, ok0, a.pstride,
                                                  &S, kPre ? &bv[0] : nullptr, lkC);
              if (acc) lc = fmaf(nC0.x, S.x, fmaf(nC0.y, S.y, lc));
              C nb1[6] = {sB[pk][1][xp0], nB1k0, nB0k1, nB0k0, nA1n0, nA10};
              nC1 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 5, oC10, nb1, H1, ok0, a.pstride,
                                                  &S, kPre ? &bv[1] : nullptr, lkC);
              if (acc) lc = fmaf(nC1.x, S.x, fmaf(nC1.y, S.y, lc));
            }
            {
              const int H0[3] = {hx + 1, hy0, Zk}, H1[3] = {hx, hy0 + 1, Zk};
              if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hl, 0, 1, sZq[pk][2], H0, H1, bv);
              if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hl, 0, 1, sZq[pk][2], H0, H1, ok0, 6, bv);
              C nb0[6] = {sA[pk][0][xp0], nA00, nA10, sA[pk][1][sym], nB0k0, sB[pm][0][s0]};
              nD0 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 6, sD[pk][0][s0], nb0, H0, ok0,
                                                  a.pstride, &S, kPre ? &bv[0] : nullptr, lkD);
              if (acc) lc = fmaf(nD0.x, S.x, fmaf(nD0.y, S.y, lc));
              C nb1[6] = {nA10, sA[pk][1][xm0], nA01, nA00, nB1k0, sB[pm][1][s0]};
              nD1 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 7, sD[pk][1][s0], nb1, H1, ok0,
                                                  a.pstride, &S, kPre ? &bv[1] : nullptr, lkD);
              if (acc) lc = fmaf(nD1.x, S.x, fmaf(nD1.y, S.y, lc));
            }
            if (acc) {  // this level's few terms in FP32, the running sums in FP64 (shared memory)
              e_acc[1] += lc;
              e_acc[0] += ((n2(nB0k0) + n2(nB1k0)) + (n2(nC0) + n2(nC1))) + (n2(nD0) + n2(nD1));
            }
            if (core0) {
              a.out[2][ok0] = nB0k0;
              a.out[3][ok0] = nB1k0;
              a.out[4][ok0] = nC0;
              a.out[5][ok0] = nC1;
              a.out[6][ok0] = nD0;
              a.out[7][ok0] = nD1;
            }
          }
          if (!th.h1) {  // cell 1 (warp-uniform)
            C nC0, nC1, nD0, nD1, S;
            const bool acc = want_e && core1;
            float lc = 0.0f;
            {
              const int H0[3] = {hx, hy1, Zk + 1}, H1[3] = {hx + 1, hy1 + 1, Zk + 1};
              if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hl, 1, 0, sZq[pk][1], H0, H1, bv);
              if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hl, 1, 0, sZq[pk][1], H0, H1, ok1, 4, bv);
              C nb0[6] = {nB0k1, sB[pk][0][xm1], nB1k1, nB1k0, nA0n1, nA01};
              nC0 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 4, oC01, nb0, H0, ok1, a.pstride,
                                                  &S, kPre ? &bv[0] : nullptr, lkC);
              if (acc) lc = fmaf(nC0.x, S.x, fmaf(nC0.y, S.y, lc));
              C nb1[6] = {sB[pk][1][xp1], nB1k1, sB[pk][0][syp], nB0k1, nA1n1, nA11};
              nC1 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 5, oC11, nb1, H1, ok1, a.pstride,
                                                  &S, kPre ? &bv[1] : nullptr, lkC);
              if (acc) lc = fmaf(nC1.x, S.x, fmaf(nC1.y, S.y, lc));
            }
            {
              const int H0[3] = {hx + 1, hy1, Zk}, H1[3] = {hx, hy1 + 1, Zk};
              if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hl, 1, 1, sZq[pk][2], H0, H1, bv);
              if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hl, 1, 1, sZq[pk][2], H0, H1, ok1, 6, bv);
              C nb0[6] = {sA[pk][0][xp1], nA01, nA11, nA10, nB0k1, sB[pm][0][s1]};
              nD0 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 6, sD[pk][0][s1], nb0, H0, ok1,
                                                  a.pstride, &S, kPre ? &bv[0] : nullptr, lkD);
              if (acc) lc = fmaf(nD0.x, S.x, fmaf(nD0.y, S.y, lc));
              C nb1[6] = {nA11, sA[pk][1][xm1], sA[pk][0][syp], nA01, nB1k1, sB[pm][1][s1]};
              nD1 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 7, sD[pk][1][s1], nb1, H1, ok1,
                                                  a.pstride, &S, kPre ? &bv[1] : nullptr, lkD);
              if (acc) lc = fmaf(nD1.x, S.x, fmaf(nD1.y, S.y, lc));
            }
            if (acc) {
              e_acc[1] += lc;
              e_acc[0] += ((n2(nB0k1) + n2(nB1k1)) + (n2(nC0) + n2(nC1))) + (n2(nD0) + n2(nD1));
            }
            if (core1) {
              a.out[2][ok1] = nB0k1;
              a.out[3][ok1] = nB1k1;
              a.out[4][ok1] = nC0;
              a.out[5][ok1] = nC1;
              a.out[6][ok1] = nD0;
              a.out[7][ok1] = nD1;
            }
          }
        }
        if (k + 1 < z1) {
          if (core0) {
            if (want_e) e_acc[0] += n2(nA0n0) + n2(nA1n0);
            a.out[0][on0] = nA0n0;
            a.out[1][on0] = nA1n0;
          }
          if (core1) {
            if (want_e) e_acc[0] += n2(nA0n1) + n2(nA1n1);
            a.out[0][on1] = nA0n1;
            a.out[1][on1] = nA1n1;
          }
        }
      }
      c0 = n0;
      c1 = n1;
    }
    __syncthreads();  // the next item rewrites the shared tiles
  }
}
#else
// One work item (one tile over one chunk of z levels) of one simulation.
// `a` may live in the constant bank (kernel parameter) or in shared memory.
template <class P, int COEF, int LINK>
__device__ __forceinline__ void fused3d_item(const FusedArgs<P>& a, long long item, const Thread3d& th,
                                             unsigned char* smem_raw, double* e_acc) {
  using C = typename P::cplx;
  // every tile is double-buffered by level parity: slot [k & 1] holds level k
  C (*sC)[2][kSlots] = reinterpret_cast<C (*)[2][kSlots]>(smem_raw);  // old C(k)
  C (*sD)[2][kSlots] = sC + 2;                                         // old D(k)
  C (*sB)[2][kSlots] = sC + 4;                                         // new B(k)
  C (*sA)[2][kSlots] = sC + 6;                                         // new A(k)
  const int t = th.slot, lx = th.lx, ly = th.ly;
  const int sxm = th.sxm, sxp = th.sxp, sym = th.sym, syp = th.syp;
  const int Nx = a.N[0], Ny = a.N[1], Nz = a.N[2];
  // global level of the stored level k (wrapped on the global grid), for the
  // fields; zorg + k lies in [-1, 2 Nzg) (zorg in [-1, Nzg), k <= N[2] <= Nzg + 1)
  auto gz = [&](int k) {
    const int g = a.zorg + k;
    return g < 0 ? g + a.Nzg : (g >= a.Nzg ? g - a.Nzg : g);
  };
  const int tiles_x = (Nx + CX - 1) / CX;
  const long long tiles = (long long)tiles_x * ((Ny + CY - 1) / CY);
  const bool iso = a.iso != 0;
  const long long nxy = (long long)Nx * Ny;
  const bool want_e = a.e_partials != nullptr;
  {
    const long long chunk = item / tiles, tile = item - chunk * tiles;
    const int z0 = a.zlo + (int)chunk * a.chunk;
    const int z1 = min(a.zlo + a.nzu, z0 + a.chunk);
    const int gx = (int)(tile % tiles_x) * CX + lx - 1;
    const int gy = (int)(tile / tiles_x) * CY + ly - 1;
    const int x = wrapi(gx, Nx), y = wrapi(gy, Ny);
    const bool core = lx >= 1 && lx <= CX && ly >= 1 && ly <= CY && gx < Nx && gy < Ny;
    const long long cxy = (long long)y * Nx + x;
    const int hx = 2 * x, hy = 2 * y;
    // COEF_SOFTCORE: the x-y part of R = |x - c|^2 + a^2 of this column, as
    // (hi, lo) pairs of two values: lanes (A0/C0, A1/C1) at (hx, hy),
    // (hx+1, hy+1) and (B0/D0, B1/D1) at (hx+1, hy), (hx, hy+1)
    // (kept in shared memory, one slot per thread: sRxy[t] = {Rd_h, Rd_l},
    // {Ra_h, Ra_l}, so that they take no registers through the z-march)
    constexpr bool kSoft = COEF == COEF_SOFTCORE || COEF == COEF_SOFTCORR;
    __shared__ __align__(16) float4 sRxy[kSoft ? kThreads3d : 1][2];
    if constexpr (kSoft) {
      const float2 x0 = __ldg(a.hu.sc_sq[0] + hx), x1 = __ldg(a.hu.sc_sq[0] + hx + 1);
      const float2 y0 = __ldg(a.hu.sc_sq[1] + hy), y1 = __ldg(a.hu.sc_sq[1] + hy + 1);
      const float2 d00 = padd(x0, y0), d11 = padd(x1, y1), a10 = padd(x1, y0), a01 = padd(x0, y1);
      sRxy[threadIdx.x][0] = make_float4(d00.x, d11.x, d00.y, d11.y);
      sRxy[threadIdx.x][1] = make_float4(a10.x, a01.x, a10.y, a01.y);
    }
    // Per-level field constants, the same for the whole block, staged in
    // shared memory by threads 0..6 with copies that bypass the registers,
    // double-buffered by level parity (level k's copies are issued after the
    // first barrier of level k-1, when no thread reads that parity any more,
    // and waited for before the first barrier of level k):
    //   sLk[p][0..3]: plane-wave link factors along z (LINK_PLANE, table axis z)
    //                 of A (upper half, Z = 2zn), B (upper, 2zk+1), C (lower,
    //                 2zk+1), D (lower, 2zk)
    //   sZq[p][0..2]: soft-core z terms sc_sq[2][Z] of Z = 2zn, 2zk+1, 2zk
    using PL = typename PlaneLinkOf<P>::type;
    __shared__ __align__(16) PL sLk[2][4];
    __shared__ __align__(16) float2 sZq[2][3];
    // (the (3+1)D launchers run a plane wave along z polarised along x as
    // LINK_PLANE_ZX and send other plane waves to the general path)
    constexpr bool lk_z = LINK == LINK_PLANE_ZX;
    auto stage_level = [&](int k) {
      const int tid = threadIdx.x;
      if (tid >= 7) return;
      const int p = k & 1;
      const int zk = gz(k), zn = gz(k + 1);  // global levels: the tables are indexed by global Z
      if constexpr (LINK == LINK_PLANE_ZX) {
        if (tid < 4) {
          const int Z = tid == 0 ? 2 * zn : (tid == 3 ? 2 * zk : 2 * zk + 1);
          const PL* tab = static_cast<const PL*>(tid < 2 ? a.hu.ltab : a.hl.ltab);
          static_assert(sizeof(PL) % 16 == 0, "16-byte copies");
          for (int q = 0; q < (int)(sizeof(PL) / 16); ++q)
            cp_async16(reinterpret_cast<char*>(&sLk[p][tid]) + 16 * q,
                       reinterpret_cast<const char*>(tab + Z) + 16 * q);
        }
      }
      if constexpr (kSoft) {
        if (tid >= 4) {
          const int Z = tid == 4 ? 2 * zn : (tid == 5 ? 2 * zk + 1 : 2 * zk);
          cp_async8(&sZq[p][tid - 4], a.hu.sc_sq[2] + Z);
        }
      }
      cp_async_commit();
    };
    // the coefficients of a pair of values with the x-y parts (Rh, Rl), the z
    // term z and positions H0, H1 (softcore_R's sums, same order)
    auto pair_b = [&](const HalfFields<P>& h, int which, float2 z, const int (&H0)[3], const int (&H1)[3],
                      float4 (&b)[2]) {
      if constexpr (COEF == COEF_SOFTCORE) {
        const float4 r = sRxy[threadIdx.x][which];  // which: 0 = (A, C) pairs, 1 = (B, D) pairs
        const float2 Rh = make_float2(r.x, r.y), Rl = make_float2(r.z, r.w);
        const float2 t0 = softcore_t0(h, H0), t1 = softcore_t0(h, H1);
        const SoftB2 bb = softcore_b2(padd(Rh, f2(z.x)), padd(Rl, f2(z.y)), make_float2(t0.x, t1.x),
                                      make_float2(t0.y, t1.y), h.sc_K_hi, h.sc_K_lo);
        b[0] = lane_b(bb, 0);
        b[1] = lane_b(bb, 1);
      }
    };
    // COEF_SOFTCORR: the FP32 estimates of a pair plus the two values' words w0, w1
    // of the correction record (R summed in softcore_R's order)
    auto pair_bc = [&](const HalfFields<P>& h, int which, float2 z, const int (&H0)[3], const int (&H1)[3],
                       long long rec, int slot, float4 (&b)[2]) {
      if constexpr (COEF == COEF_SOFTCORR) {
        // the pair's two words of the level's correction record (read where used)
        const uint2 w = __ldg(reinterpret_cast<const uint2*>(a.hu.sc_corr + 8 * rec + slot));
        const unsigned w0 = w.x, w1 = w.y;
        const float4 r = sRxy[threadIdx.x][which];
        const float2 Rh = padd(make_float2(r.x, r.y), f2(z.x)), Rl = padd(make_float2(r.z, r.w), f2(z.y));
        float2 re, im;
        softcore_fast2(Rh, Rl, make_float2(softcore_t0(h, H0).x, softcore_t0(h, H1).x), h.sc_K_hi, re, im);
        const float2 c0 = corr_decode(w0), c1 = corr_decode(w1);
        b[0] = make_float4(re.x, c0.x, im.x, c0.y);
        b[1] = make_float4(re.y, c1.x, im.y, c1.y);
      }
    };
    constexpr bool kPre = kSoft;  // coefficients computed in pairs

    auto load = [&](int k) {
      const int zk = k < 0 ? k + Nz : k;
      const int zn = k + 1 >= Nz ? k + 1 - Nz : k + 1;
      const long long ok = zk * nxy + cxy, on = zn * nxy + cxy;
      LevelLoad<C> l;
      l.A0 = ld(a.in[0] + on);
      l.A1 = ld(a.in[1] + on);
      l.B0 = ld(a.in[2] + ok);
      l.B1 = ld(a.in[3] + ok);
      l.C0 = ld(a.in[4] + on);
      l.C1 = ld(a.in[5] + on);
      l.D0 = ld(a.in[6] + on);
      l.D1 = ld(a.in[7] + on);
      return l;
    };

    {  // old C, D of level z0-1 (the z- neighbours of the first level)
      const int p = (z0 - 1) & 1;
      const long long o = (long long)wrapi(z0 - 1, Nz) * nxy + cxy;
      sC[p][0][t] = ld(a.in[4] + o);
      sC[p][1][t] = ld(a.in[5] + o);
      sD[p][0][t] = ld(a.in[6] + o);
      sD[p][1][t] = ld(a.in[7] + o);
    }
    LevelLoad<C> cur = load(z0 - 1);
    constexpr bool kStage = LINK == LINK_PLANE_ZX || kSoft;
    if (kStage) stage_level(z0 - 1);

    for (int k = z0 - 1; k < z1; ++k) {
      const int zk = k < 0 ? k + Nz : k;
      const int zn = k + 1 >= Nz ? k + 1 - Nz : k + 1;
      const long long ok = zk * nxy + cxy, on = zn * nxy + cxy;
      const int pk = k & 1, pn = (k + 1) & 1, pm = (k - 1) & 1;
      const int Zk = 2 * gz(k), Zn = 2 * gz(k + 1);  // half-lattice z of levels k, k+1 (global)
      sC[pn][0][t] = cur.C0;  // old C(k+1), D(k+1): z+ / x,y neighbours now,
      sC[pn][1][t] = cur.C1;  // own old values at the next level
      sD[pn][0][t] = cur.D0;
      sD[pn][1][t] = cur.D1;
      // prefetch the next level while this one computes
      LevelLoad<C> nxt = cur;
      if (k + 1 < z1) nxt = load(k + 1);
      if (kStage && threadIdx.x < 7) cp_async_wait_all();  // this level's staged constants
      __syncthreads();
      if (kStage && k + 1 < z1) stage_level(k + 1);
      const PL* lkA = lk_z ? &sLk[pk][0] : nullptr;  // compile-time choice: a shared-memory address
      const PL* lkB = lk_z ? &sLk[pk][1] : nullptr;

      // upper half-step: A(k+1) from C(k+1), C(k), D(k+1); B(k) from D(k+1), D(k), C(k)
      const C oC0 = sC[pk][0][t], oC1 = sC[pk][1][t];
      C nA0n, nA1n, nB0k, nB1k;
      float4 bv[2];
      {
        const int H0[3] = {hx, hy, Zn}, H1[3] = {hx + 1, hy + 1, Zn};
        if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hu, 0, sZq[pk][0], H0, H1, bv);
        if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hu, 0, sZq[pk][0], H0, H1, ok, 0, bv);
        C nb0[6] = {cur.D0, sD[pn][0][sxm], cur.D1, sD[pn][1][sym], cur.C0, oC0};
        nA0n = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 0, cur.A0, nb0, H0, on, a.pstride,
                                             nullptr, kPre ? &bv[0] : nullptr, lkA);
        C nb1[6] = {sD[pn][1][sxp], cur.D1, sD[pn][0][syp], cur.D0, cur.C1, oC1};
        nA1n = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 1, cur.A1, nb1, H1, on, a.pstride,
                                             nullptr, kPre ? &bv[1] : nullptr, lkA);
      }
      {
        const int H0[3] = {hx + 1, hy, Zk + 1}, H1[3] = {hx, hy + 1, Zk + 1};
        if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hu, 1, sZq[pk][1], H0, H1, bv);
        if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hu, 1, sZq[pk][1], H0, H1, ok, 2, bv);
        C nb0[6] = {sC[pk][0][sxp], oC0, oC1, sC[pk][1][sym], cur.D0, sD[pk][0][t]};
        nB0k = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 2, cur.B0, nb0, H0, ok, a.pstride,
                                             nullptr, kPre ? &bv[0] : nullptr, lkB);
        C nb1[6] = {oC1, sC[pk][1][sxm], sC[pk][0][syp], oC0, cur.D1, sD[pk][1][t]};
        nB1k = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 3, cur.B1, nb1, H1, ok, a.pstride,
                                             nullptr, kPre ? &bv[1] : nullptr, lkB);
      }
      sB[pk][0][t] = nB0k;
      sB[pk][1][t] = nB1k;
      sA[pn][0][t] = nA0n;
      sA[pn][1][t] = nA1n;
      __syncthreads();

      // lower half-step: C(k) from A(k+1), A(k), B(k); D(k) from B(k), B(k-1), A(k)
      // (interior warps only: nothing needs the halo's lower values; the
      // first level of a run only rebuilds A(z0) and B(z0-1))
      if (!th.halo) {
        auto n2 = [](C v) { return fmaf(v.x, v.x, v.y * v.y); };
        if (k >= z0) {
          const C nA0 = sA[pk][0][t], nA1 = sA[pk][1][t];
          C nC0, nC1, nD0, nD1, S;
          const bool acc = want_e && core;  // this cell's new values count towards E
          float lc = 0.0f;
          {
            const int H0[3] = {hx, hy, Zk + 1}, H1[3] = {hx + 1, hy + 1, Zk + 1};
            if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hl, 0, sZq[pk][1], H0, H1, bv);
            if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hl, 0, sZq[pk][1], H0, H1, ok, 4, bv);
            const PL* lkC = lk_z ? &sLk[pk][2] : nullptr;
            C nb0[6] = {nB0k, sB[pk][0][sxm], nB1k, sB[pk][1][sym], nA0n, nA0};
            nC0 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 4, oC0, nb0, H0, ok, a.pstride, &S,
                                                kPre ? &bv[0] : nullptr, lkC);
            if (acc) lc = fmaf(nC0.x, S.x, fmaf(nC0.y, S.y, lc));
            C nb1[6] = {sB[pk][1][sxp], nB1k, sB[pk][0][syp], nB0k, nA1n, nA1};
            nC1 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 5, oC1, nb1, H1, ok, a.pstride, &S,
                                                kPre ? &bv[1] : nullptr, lkC);
            if (acc) lc = fmaf(nC1.x, S.x, fmaf(nC1.y, S.y, lc));
          }
          {
            const int H0[3] = {hx + 1, hy, Zk}, H1[3] = {hx, hy + 1, Zk};
            if constexpr (COEF == COEF_SOFTCORE) pair_b(a.hl, 1, sZq[pk][2], H0, H1, bv);
            if constexpr (COEF == COEF_SOFTCORR) pair_bc(a.hl, 1, sZq[pk][2], H0, H1, ok, 6, bv);
            const PL* lkD = lk_z ? &sLk[pk][3] : nullptr;
            C nb0[6] = {sA[pk][0][sxp], nA0, nA1, sA[pk][1][sym], nB0k, sB[pm][0][t]};
            nD0 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 6, sD[pk][0][t], nb0, H0, ok,
                                                a.pstride, &S, kPre ? &bv[0] : nullptr, lkD);
            if (acc) lc = fmaf(nD0.x, S.x, fmaf(nD0.y, S.y, lc));
            C nb1[6] = {nA1, sA[pk][1][sxm], sA[pk][0][syp], nA0, nB1k, sB[pm][1][t]};
            nD1 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 7, sD[pk][1][t], nb1, H1, ok,
                                                a.pstride, &S, kPre ? &bv[1] : nullptr, lkD);
            if (acc) lc = fmaf(nD1.x, S.x, fmaf(nD1.y, S.y, lc));
          }
          if (acc) {  // this level's few terms in FP32, the running sums in FP64 (shared memory)
            e_acc[1] += lc;
            e_acc[0] += ((n2(nB0k) + n2(nB1k)) + (n2(nC0) + n2(nC1))) + (n2(nD0) + n2(nD1));
          }
          if (core) {
            a.out[2][ok] = nB0k;
            a.out[3][ok] = nB1k;
            a.out[4][ok] = nC0;
            a.out[5][ok] = nC1;
            a.out[6][ok] = nD0;
            a.out[7][ok] = nD1;
          }
        }
        if (k + 1 < z1 && core) {
          if (want_e) e_acc[0] += n2(nA0n) + n2(nA1n);
          a.out[0][on] = nA0n;
          a.out[1][on] = nA1n;
        }
      }
      cur = nxt;
    }
    __syncthreads();  // the next item rewrites the shared tiles
  }
}

#endif

// FP64 block reduction of the two conserved-functional accumulators into
// out[blockIdx.x][2] (all threads of the block call it)
__device__ __forceinline__ void block_store_e(double e_n, double e_c, double* out) {
  __shared__ double red[32][2];
  double n = e_n, c = e_c;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    n += __shfl_down_sync(0xffffffffu, n, o);
    c += __shfl_down_sync(0xffffffffu, c, o);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  __syncthreads();
  if (lane == 0) {
    red[w][0] = n;
    red[w][1] = c;
  }
  __syncthreads();
  if (w == 0) {
    n = lane < nw ? red[lane][0] : 0.0;
    c = lane < nw ? red[lane][1] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      n += __shfl_down_sync(0xffffffffu, n, o);
      c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      out[2LL * blockIdx.x] = n;
      out[2LL * blockIdx.x + 1] = c;
    }
  }
}

template <class P, int COEF, int LINK>
__global__ void __launch_bounds__(kThreads3d, kBlocks3d) fused3d_kernel(const FusedArgs<P> a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const Thread3d th = thread3d();
  const long long items = items3d(a.N, a.nzu, a.chunk);
  // running sums of the functional, one FP64 pair per thread, kept in shared
  // memory so that they take no registers in the z-march
  __shared__ double e_acc[kThreads3d][2];
  e_acc[threadIdx.x][0] = e_acc[threadIdx.x][1] = 0.0;
  for (long long item = blockIdx.x; item < items; item += a.workers)
    fused3d_item<P, COEF, LINK>(a, item, th, smem_raw, e_acc[threadIdx.x]);
  if (a.e_partials) block_store_e(e_acc[threadIdx.x][0], e_acc[threadIdx.x][1], a.e_partials);
}

// simulation of global item g: the last s with first[s] <= g
__device__ __forceinline__ int find_sim(const long long* first, int nsims, long long g) {
  int lo = 0, hi = nsims - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(first + mid) <= g) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// copy one simulation's arguments into shared memory (nthreads cooperating)
template <class P>
__device__ __forceinline__ void copy_args(FusedArgs<P>* dst, const FusedArgs<P>* src, int tid,
                                          int nthreads) {
  static_assert(sizeof(FusedArgs<P>) % 4 == 0, "word copy");
  const int* s = reinterpret_cast<const int*>(src);
  int* d = reinterpret_cast<int*>(dst);
  for (int i = tid; i < (int)(sizeof(FusedArgs<P>) / 4); i += nthreads) d[i] = __ldg(s + i);
}

// Several simulations in one persistent launch: global items are the
// simulations' items back to back; each block copies the arguments of the
// simulation its current item belongs to into shared memory.
template <class P, int COEF, int LINK>
__global__ void __launch_bounds__(kThreads3d, kBlocks3d) fused3d_batch_kernel(const BatchArgs<P> b) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ FusedArgs<P> sa;
  const Thread3d th = thread3d();
  const long long total = b.first_item[b.nsims];
  int cur = -1;
  for (long long g = blockIdx.x; g < total; g += b.workers) {
    const int s = find_sim(b.first_item, b.nsims, g);
    if (s != cur) {
      __syncthreads();  // everyone is done with the previous arguments
      copy_args(&sa, b.sims + s, (int)threadIdx.x, kThreads3d);
      __syncthreads();
      cur = s;
    }
    // (batched launches never accumulate the functional: e_partials is null)
    fused3d_item<P, COEF, LINK>(sa, g - b.first_item[s], th, smem_raw, nullptr);
  }
}

// work items of a (2+1)D one-step launch: strips x chunks of the `rows` updated rows
__host__ __device__ __forceinline__ long long items2d(const int (&N)[3], int rows, int chunk) {
  return (long long)((N[0] + kCore - 1) / kCore) * ((rows + chunk - 1) / chunk);
}

// One row of the (2+1)D pipeline at march position k.  In: the old u0, v0, v1
// of row k+1 and u1 of row k (the loads of row k), the old v0, v1 of row k,
// the new u0 of row k and the new u1 of row k-1.  Out: the new u0 of row k+1,
// u1, v1, v0 of row k.  Planes: 0 u0 (0,0)  1 u1 (1,1)  2 v0 (1,0)  3 v1 (0,1).
template <class P, int COEF, int LINK>
__device__ __forceinline__ void row2d(const FusedArgs<P>& a, bool iso, int hx, int yk, int yn,
                                      long long ok, long long on, typename P::cplx U0,
                                      typename P::cplx V0n, typename P::cplx V1n, typename P::cplx U1,
                                      typename P::cplx oV0, typename P::cplx oV1, typename P::cplx nU0,
                                      typename P::cplx nU1, typename P::cplx& nU0n,
                                      typename P::cplx& nU1k, typename P::cplx& nV1,
                                      typename P::cplx& nV0, typename P::cplx* SV1 = nullptr,
                                      typename P::cplx* SV0 = nullptr) {
  using C = typename P::cplx;
  // upper: u0(k+1) from v0(k+1) (x), v1(k+1), v1(k) (y); u1(k) from v1(k) (x), v0(k+1), v0(k) (y)
  {
    C nb[6] = {V0n, shfl_up1(V0n), V1n, oV1, V0n, V0n};
    const int H[3] = {hx, 2 * yn, 0};
    nU0n = site_update<P, 2, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 0, U0, nb, H, on, a.pstride, nullptr,
                                         nullptr, nullptr, a.N);
  }
  {
    C nb[6] = {shfl_down1(oV1), oV1, V0n, oV0, oV1, oV1};
    const int H[3] = {hx + 1, 2 * yk + 1, 0};
    nU1k = site_update<P, 2, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 1, U1, nb, H, ok, a.pstride, nullptr,
                                         nullptr, nullptr, a.N);
  }
  // lower: v1(k) from u1(k) (x), u0(k+1), u0(k) (y); v0(k) from u0(k) (x), u1(k), u1(k-1) (y)
  {
    C nb[6] = {nU1k, shfl_up1(nU1k), nU0n, nU0, nU1k, nU1k};
    const int H[3] = {hx, 2 * yk + 1, 0};
    nV1 = site_update<P, 2, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 3, oV1, nb, H, ok, a.pstride, SV1, nullptr,
                                        nullptr, a.N);
  }
  {
    C nb[6] = {shfl_down1(nU0), nU0, nU1k, nU1, nU0, nU0};
    const int H[3] = {hx + 1, 2 * yk, 0};
    nV0 = site_update<P, 2, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 2, oV0, nb, H, ok, a.pstride, SV0, nullptr,
                                        nullptr, a.N);
  }
}

// One work item (one 32-cell strip over one chunk of rows) of one simulation,
// processed by one warp.
template <class P, int COEF, int LINK>
__device__ __forceinline__ void fused2d_item(const FusedArgs<P>& a, long long item, int lane, double& e_n,
                                             double& e_c) {
  using C = typename P::cplx;
  const int Nx = a.N[0], Ny = a.N[1];
  const int strips = (Nx + kCore - 1) / kCore;
  const bool iso = a.iso != 0;
  const long long chunk = item / strips;
  const int strip = (int)(item - chunk * strips);
  // the updated rows zlo .. zlo + nzu - 1 (all rows of a whole grid, a slab's
  // own rows); fields at the global row (zorg + k, wrapped: in [-1, 2 Nzg))
  const int y0 = a.zlo + (int)chunk * a.chunk;
  const int y1 = min(a.zlo + a.nzu, y0 + a.chunk);
  auto gy = [&](int k) {
    const int g = a.zorg + k;
    return g < 0 ? g + a.Nzg : (g >= a.Nzg ? g - a.Nzg : g);
  };
  const int gx = strip * kCore + lane - 1;
  const int x = wrapi(gx, Nx);
  const bool core = lane >= 1 && lane <= kCore && gx < Nx;
  const int hx = 2 * x;
  long long o = (long long)wrapi(y0 - 1, Ny) * Nx + x;
  C oV0 = ld(a.in[2] + o), oV1 = ld(a.in[3] + o);
  C nU0 = oV0, nU1 = oV1;  // placeholders: only feed values never stored
  // the loads of row k: u0, v0, v1 at row k+1 and u1 at row k
  auto load = [&](int k, C& u0, C& v0, C& v1, C& u1) {
    const int yk = k < 0 ? k + Ny : (k >= Ny ? k - Ny : k);
    const int yn = k + 1 >= Ny ? k + 1 - Ny : (k + 1 < 0 ? k + 1 + Ny : k + 1);
    const long long okk = (long long)yk * Nx + x, onn = (long long)yn * Nx + x;
    u0 = ld(a.in[0] + onn);
    v0 = ld(a.in[2] + onn);
    v1 = ld(a.in[3] + onn);
    u1 = ld(a.in[1] + okk);
  };
  C U0, V0n, V1n, U1;
  load(y0 - 1, U0, V0n, V1n, U1);
  for (int k = y0 - 1; k < y1; ++k) {
    const int yk = k < 0 ? k + Ny : k;
    const int yn = k + 1 >= Ny ? k + 1 - Ny : k + 1;
    const long long ok = (long long)yk * Nx + x, on = (long long)yn * Nx + x;
    C pU0 = U0, pV0 = V0n, pV1 = V1n, pU1 = U1;  // next row, loaded while this one computes
    if (k + 1 < y1) load(k + 1, pU0, pV0, pV1, pU1);
    C nU0n, nU1k, nV1, nV0, S1, S0;
    row2d<P, COEF, LINK>(a, iso, hx, gy(k), gy(k + 1), ok, on, U0, V0n, V1n, U1, oV0, oV1, nU0, nU1, nU0n,
                         nU1k, nV1, nV0, &S1, &S0);
    if (core) {
      if (k >= y0) {
        a.out[1][ok] = nU1k;
        a.out[2][ok] = nV0;
        a.out[3][ok] = nV1;
        if (a.e_partials) {
          e_n += (fmaf(nU1k.x, nU1k.x, nU1k.y * nU1k.y) + fmaf(nV0.x, nV0.x, nV0.y * nV0.y)) +
                 fmaf(nV1.x, nV1.x, nV1.y * nV1.y);
          e_c += fmaf(nV1.x, S1.x, fmaf(nV1.y, S1.y, fmaf(nV0.x, S0.x, nV0.y * S0.y)));
        }
      }
      if (k + 1 < y1) {
        a.out[0][on] = nU0n;
        if (a.e_partials) e_n += fmaf(nU0n.x, nU0n.x, nU0n.y * nU0n.y);
      }
    }
    oV0 = V0n;
    oV1 = V1n;
    nU0 = nU0n;
    nU1 = nU1k;
    U0 = pU0;
    V0n = pV0;
    V1n = pV1;
    U1 = pU1;
  }
}

// Two time steps per pass ((2+1)D, fields without time dependence).  Step 1
// runs the row pipeline on the old state; step 2 runs it one row behind on
// step 1's results, which never leave registers.  A strip keeps 28 interior
// lanes (lanes 2..29): step 1 is valid on lanes 1..30, step 2 on 2..29.
// Step 1 starts two rows and step 2 one row before the chunk.
constexpr int kCoreTb = 28;

template <class P, int COEF, int LINK>
__device__ __forceinline__ void fused2d_tb2_item(const FusedArgs<P>& a, long long item, int lane,
                                                 double& e_n, double& e_c) {
  using C = typename P::cplx;
  const int Nx = a.N[0], Ny = a.N[1];
  const int strips = (Nx + kCoreTb - 1) / kCoreTb;
  const bool iso = a.iso != 0;
  const long long chunk = item / strips;
  const int strip = (int)(item - chunk * strips);
  const int y0 = (int)chunk * a.chunk;
  const int y1 = min(Ny, y0 + a.chunk);
  const int gx = strip * kCoreTb + lane - 2;
  const int x = wrapi(gx, Nx);
  const bool core = lane >= 2 && lane <= kCoreTb + 1 && gx < Nx;
  const int hx = 2 * x;
  auto wrapy = [&](int k) { return k < 0 ? k + Ny : (k >= Ny ? k - Ny : k); };
  auto load = [&](int k, C& u0, C& v0, C& v1, C& u1) {
    const long long okk = (long long)wrapy(k) * Nx + x, onn = (long long)wrapy(k + 1) * Nx + x;
    u0 = ld(a.in[0] + onn);
    v0 = ld(a.in[2] + onn);
    v1 = ld(a.in[3] + onn);
    u1 = ld(a.in[1] + okk);
  };
  // step-1 pipeline state (old v0, v1 of row k; new u0 of row k; new u1 of row k-1)
  long long o = (long long)wrapy(y0 - 2) * Nx + x;
  C oV0 = ld(a.in[2] + o), oV1 = ld(a.in[3] + o);
  C nU0 = oV0, nU1 = oV1;  // placeholders: only feed values never stored
  // step-2 pipeline state: step-1 v0, v1 of row k-1; step-2 u0 of row k-1, u1 of row k-2
  C qV0 = oV0, qV1 = oV1, mU0 = oV0, mU1 = oV1;
  C U0, V0n, V1n, U1;
  load(y0 - 2, U0, V0n, V1n, U1);
  for (int k = y0 - 2; k <= y1; ++k) {
    const int yk = wrapy(k), yn = wrapy(k + 1);
    const long long ok = (long long)yk * Nx + x, on = (long long)yn * Nx + x;
    C pU0 = U0, pV0 = V0n, pV1 = V1n, pU1 = U1;
    if (k + 1 <= y1) load(k + 1, pU0, pV0, pV1, pU1);
    // step 1 at row k
    C sU0n, sU1k, sV1, sV0;
    row2d<P, COEF, LINK>(a, iso, hx, yk, yn, ok, on, U0, V0n, V1n, U1, oV0, oV1, nU0, nU1, sU0n, sU1k,
                         sV1, sV0);
    if (k >= y0) {
      // step 2 at row k-1: its loads are step 1's u0, v0, v1 of row k and u1 of row k-1
      const int ym = wrapy(k - 1);
      const long long om = (long long)ym * Nx + x;
      C tU0n, tU1k, tV1, tV0, S1, S0;
      row2d<P, COEF, LINK>(a, iso, hx, ym, yk, om, ok, nU0, sV0, sV1, nU1, qV0, qV1, mU0, mU1, tU0n, tU1k,
                           tV1, tV0, &S1, &S0);
      if (core) {
        if (k - 1 >= y0) {
          a.out[1][om] = tU1k;
          a.out[2][om] = tV0;
          a.out[3][om] = tV1;
          if (a.e_partials) {
            e_n += (fmaf(tU1k.x, tU1k.x, tU1k.y * tU1k.y) + fmaf(tV0.x, tV0.x, tV0.y * tV0.y)) +
                   fmaf(tV1.x, tV1.x, tV1.y * tV1.y);
            e_c += fmaf(tV1.x, S1.x, fmaf(tV1.y, S1.y, fmaf(tV0.x, S0.x, tV0.y * S0.y)));
          }
        }
        if (k < y1) {
          a.out[0][ok] = tU0n;
          if (a.e_partials) e_n += fmaf(tU0n.x, tU0n.x, tU0n.y * tU0n.y);
        }
      }
      mU0 = tU0n;
      mU1 = tU1k;
    }
    qV0 = sV0;  // step-1 v0, v1 of row k become step 2's old row
    qV1 = sV1;
    oV0 = V0n;
    oV1 = V1n;
    nU0 = sU0n;
    nU1 = sU1k;
    U0 = pU0;
    V0n = pV0;
    V1n = pV1;
    U1 = pU1;
  }
}

template <class P, int COEF, int LINK>
__global__ void __launch_bounds__(32 * kFused2dWarps) fused2d_kernel(const FusedArgs<P> a) {
  const int lane = threadIdx.x & 31;
  const long long worker = (long long)blockIdx.x * kFused2dWarps + (threadIdx.x >> 5);
  const long long items = items2d(a.N, a.nzu, a.chunk);
  double e_n = 0.0, e_c = 0.0;
  for (long long item = worker; item < items; item += a.workers)  // uniform per warp
    fused2d_item<P, COEF, LINK>(a, item, lane, e_n, e_c);
  if (a.e_partials) block_store_e(e_n, e_c, a.e_partials);
}

template <class P, int COEF, int LINK>
__global__ void __launch_bounds__(32 * kFused2dWarps) fused2d_tb2_kernel(const FusedArgs<P> a) {
  const int lane = threadIdx.x & 31;
  const long long worker = (long long)blockIdx.x * kFused2dWarps + (threadIdx.x >> 5);
  const long long items = (long long)((a.N[0] + kCoreTb - 1) / kCoreTb) * ((a.N[1] + a.chunk - 1) / a.chunk);
  double e_n = 0.0, e_c = 0.0;
  for (long long item = worker; item < items; item += a.workers)  // uniform per warp
    fused2d_tb2_item<P, COEF, LINK>(a, item, lane, e_n, e_c);
  if (a.e_partials) block_store_e(e_n, e_c, a.e_partials);
}

template <class P, int COEF, int LINK>
__global__ void __launch_bounds__(32 * kFused2dWarps) fused2d_batch_kernel(const BatchArgs<P> b) {
  __shared__ FusedArgs<P> sa[kFused2dWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long worker = (long long)blockIdx.x * kFused2dWarps + w;
  const long long total = b.first_item[b.nsims];
  int cur = -1;
  for (long long g = worker; g < total; g += b.workers) {
    const int s = find_sim(b.first_item, b.nsims, g);
    if (s != cur) {
      __syncwarp();
      copy_args(&sa[w], b.sims + s, lane, 32);
      __syncwarp();
      cur = s;
    }
    double e_n = 0.0, e_c = 0.0;  // (batched launches never accumulate the functional)
    fused2d_item<P, COEF, LINK>(sa[w], g - b.first_item[s], lane, e_n, e_c);
  }
}

// Two time steps per pass for several (2+1)D simulations (time-independent
// fields): as fused2d_batch_kernel with the two-step item of each simulation.
template <class P, int COEF, int LINK>
__global__ void __launch_bounds__(32 * kFused2dWarps) fused2d_tb2_batch_kernel(const BatchArgs<P> b) {
  __shared__ FusedArgs<P> sa[kFused2dWarps];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const long long worker = (long long)blockIdx.x * kFused2dWarps + w;
  const long long total = b.first_item[b.nsims];
  int cur = -1;
  for (long long g = worker; g < total; g += b.workers) {
    const int s = find_sim(b.first_item, b.nsims, g);
    if (s != cur) {
      __syncwarp();
      copy_args(&sa[w], b.sims + s, lane, 32);
      __syncwarp();
      cur = s;
    }
    double e_n = 0.0, e_c = 0.0;  // (batched launches never accumulate the functional)
    fused2d_tb2_item<P, COEF, LINK>(sa[w], g - b.first_item[s], lane, e_n, e_c);
  }
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Chunk length (levels per item) for `tiles` items per level chunk, `levels`
// levels and `workers` persistent workers: maximise the busy fraction of the
// rounds times the useful fraction chunk/(chunk+restart) of each item, where
// `restart` is the cost of an item's extra first level in levels.
// The `max` best chunk lengths by that model, best first, into out; returns
// how many (at least one).
int rank_chunks(long long tiles, int levels, long long workers, int min_chunk, double restart, int* out,
                int max) {
  int n = 0, prev = -1;
  double eff_of[64];
  if (max > 64) max = 64;
  for (int c = 1; c <= levels; ++c) {
    const int len = (levels + c - 1) / c;  // non-increasing in c
    if (len < min_chunk && c > 1) break;
    if (len == prev) continue;
    prev = len;
    const int chunks = (levels + len - 1) / len;
    const long long items = tiles * chunks;
    const long long rounds = (items + workers - 1) / workers;
    // work of a round ~ len + restart levels; total time ~ rounds * (len + restart)
    const double eff = (double)tiles * levels / ((double)rounds * workers * (len + restart));
    // insert by efficiency (stable: on ties, fewer chunks first)
    int pos = n;
    while (pos > 0 && eff > eff_of[pos - 1] * 1.0001) --pos;
    if (pos >= max) continue;
    const int last = n < max ? n : max - 1;
    for (int i = last; i > pos; --i) {
      out[i] = out[i - 1];
      eff_of[i] = eff_of[i - 1];
    }
    out[pos] = len;
    eff_of[pos] = eff;
    if (n < max) ++n;
  }
  if (n == 0) out[n++] = levels;
  return n;
}

int plan_chunk(long long tiles, int levels, long long workers, int min_chunk, double restart) {
  int best = levels;
  rank_chunks(tiles, levels, workers, min_chunk, restart, &best, 1);
  return best;
}

template <class K>
int resident_blocks(K kernel, int threads, size_t smem = 0) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, smem);
  return (per_sm < 1 ? 1 : per_sm) * sm_count();
}

// resident workers of the fused kernels: blocks ((3+1)D) or warps ((2+1)D);
// computed once per kernel (the template argument is the kernel itself), the
// (3+1)D kernels also get their dynamic shared-memory limit raised once
template <auto K>
int workers3d() {
  static int r = [] {
    cudaFuncSetAttribute(K, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem3d);
    return resident_blocks(K, kThreads3d, kSmem3d);
  }();
  return r;
}
template <auto K>
int workers2d() {
  static int r = resident_blocks(K, 32 * kFused2dWarps) * kFused2dWarps;
  return r;
}

template <int COEF, int LINK>
int launch3d(FusedArgs<F32> a, cudaStream_t s) {
  auto k = fused3d_kernel<F32, COEF, LINK>;
  const int resident = workers3d<fused3d_kernel<F32, COEF, LINK>>();
  if (a.chunk <= 0 || a.chunk > a.nzu) {
    const int Np[3] = {a.N[0], a.N[1], a.nzu};
    a.chunk = fused_chunk(3, Np);
  }
  const long long items = items3d(a.N, a.nzu, a.chunk);
  a.workers = (int)(items < resident ? items : resident);
  // one E partial per block: never more blocks than the partials hold
  if (a.e_partials && a.workers > kFusedEMaxBlocks) a.workers = kFusedEMaxBlocks;
  k<<<(unsigned)a.workers, kThreads3d, kSmem3d, s>>>(a);
  return a.workers;
}

template <int COEF, int LINK>
int launch2d(FusedArgs<F32> a, cudaStream_t s) {
  auto k = fused2d_kernel<F32, COEF, LINK>;
  const int warps = workers2d<fused2d_kernel<F32, COEF, LINK>>();
  if (a.chunk <= 0 || a.chunk > a.nzu) {
    const int Np[3] = {a.N[0], a.nzu, 1};
    a.chunk = fused_chunk(2, Np);
  }
  const long long items = items2d(a.N, a.nzu, a.chunk);
  long long w = items < warps ? items : warps;
  // one E partial per block: never more blocks than the partials hold
  if (a.e_partials && w > (long long)kFusedEMaxBlocks * kFused2dWarps) w = (long long)kFusedEMaxBlocks * kFused2dWarps;
  a.workers = (int)w;
  const int blocks = (int)((w + kFused2dWarps - 1) / kFused2dWarps);
  k<<<(unsigned)blocks, 32 * kFused2dWarps, 0, s>>>(a);
  return blocks;
}

template <int COEF, int LINK>
void launch3d_batch(BatchArgs<F32> b, long long total, cudaStream_t s) {
  auto k = fused3d_batch_kernel<F32, COEF, LINK>;
  const int resident = workers3d<fused3d_batch_kernel<F32, COEF, LINK>>();
  b.workers = (int)(total < resident ? total : resident);
  k<<<(unsigned)b.workers, kThreads3d, kSmem3d, s>>>(b);
}

template <int COEF, int LINK>
void launch2d_batch(BatchArgs<F32> b, long long total, cudaStream_t s) {
  auto k = fused2d_batch_kernel<F32, COEF, LINK>;
  const int warps = workers2d<fused2d_batch_kernel<F32, COEF, LINK>>();
  const long long w = total < warps ? total : warps;
  b.workers = (int)w;
  k<<<(unsigned)((w + kFused2dWarps - 1) / kFused2dWarps), 32 * kFused2dWarps, 0, s>>>(b);
}

template <int COEF, int LINK>
void launch2d_tb2_batch(BatchArgs<F32> b, long long total, cudaStream_t s) {
  auto k = fused2d_tb2_batch_kernel<F32, COEF, LINK>;
  const int warps = workers2d<fused2d_tb2_batch_kernel<F32, COEF, LINK>>();
  const long long w = total < warps ? total : warps;
  b.workers = (int)w;
  k<<<(unsigned)((w + kFused2dWarps - 1) / kFused2dWarps), 32 * kFused2dWarps, 0, s>>>(b);
}

template <int DIMS, int COEF, int LINK>
int launch_dims(const FusedArgs<F32>& a, cudaStream_t s) {
  if constexpr (DIMS == 3) {
    // (3+1)D plane waves are dispatched before reaching here (LINK_PLANE_ZX)
    if constexpr (LINK == LINK_PLANE) return launch3d<kAnyMode, kAnyMode>(a, s);
    else return launch3d<COEF, LINK>(a, s);
  } else {
    return launch2d<COEF, LINK>(a, s);
  }
}

template <int DIMS>
int dispatch(const FusedArgs<F32>& a, cudaStream_t s) {
  const int c = a.hu.coef_mode, l = a.hu.link_mode;
  if (c == COEF_GENERAL || l == LINK_GENERAL) return launch_dims<DIMS, kAnyMode, kAnyMode>(a, s);
  // the fused (3+1)D kernel stages plane-wave link factors per z level: a wave
  // along z polarised along x runs as LINK_PLANE_ZX, other plane waves take
  // the general path there
  if (DIMS == 3 && l == LINK_PLANE) {
    if (a.hu.ltab_axis != 2 || a.hu.lpol != 0) return launch3d<kAnyMode, kAnyMode>(a, s);
    if (c == COEF_UNIFORM) return launch3d<COEF_UNIFORM, LINK_PLANE_ZX>(a, s);
    if (c == COEF_STEP) return launch3d<COEF_STEP, LINK_PLANE_ZX>(a, s);
    if (c == COEF_TABLE) return launch3d<COEF_TABLE, LINK_PLANE_ZX>(a, s);
    if (c == COEF_SOFTCORE) return launch3d<COEF_SOFTCORE, LINK_PLANE_ZX>(a, s);
    if (c == COEF_SOFTCORR) return launch3d<COEF_SOFTCORR, LINK_PLANE_ZX>(a, s);
    return launch3d<kAnyMode, kAnyMode>(a, s);
  }
  if (c == COEF_SOFTCORE) {
    if (l == LINK_NONE) return launch_dims<DIMS, COEF_SOFTCORE, LINK_NONE>(a, s);
    if (l == LINK_PLANE) return launch_dims<DIMS, COEF_SOFTCORE, LINK_PLANE>(a, s);
    return launch_dims<DIMS, kAnyMode, kAnyMode>(a, s);
  }
  if (c == COEF_SOFTCORR) {
    if (l == LINK_NONE) return launch_dims<DIMS, COEF_SOFTCORR, LINK_NONE>(a, s);
    if (l == LINK_PLANE) return launch_dims<DIMS, COEF_SOFTCORR, LINK_PLANE>(a, s);
    return launch_dims<DIMS, kAnyMode, kAnyMode>(a, s);
  }
  if (l == LINK_TABLE) {
    if (c == COEF_UNIFORM) return launch_dims<DIMS, COEF_UNIFORM, LINK_TABLE>(a, s);
    if (c == COEF_STEP) return launch_dims<DIMS, COEF_STEP, LINK_TABLE>(a, s);
    return launch_dims<DIMS, COEF_TABLE, LINK_TABLE>(a, s);
  }
  if (c == COEF_TABLE && l == LINK_NONE) return launch_dims<DIMS, COEF_TABLE, LINK_NONE>(a, s);
  if (c == COEF_TABLE && l == LINK_PLANE) return launch_dims<DIMS, COEF_TABLE, LINK_PLANE>(a, s);
  if (c == COEF_TABLE) return launch_dims<DIMS, kAnyMode, kAnyMode>(a, s);
  if (c == COEF_UNIFORM && l == LINK_PLANE) return launch_dims<DIMS, COEF_UNIFORM, LINK_PLANE>(a, s);
  if (c == COEF_STEP && l == LINK_PLANE) return launch_dims<DIMS, COEF_STEP, LINK_PLANE>(a, s);
  if (c == COEF_UNIFORM && l == LINK_NONE) return launch_dims<DIMS, COEF_UNIFORM, LINK_NONE>(a, s);
  if (c == COEF_STEP && l == LINK_NONE) return launch_dims<DIMS, COEF_STEP, LINK_NONE>(a, s);
  if (c == COEF_UNIFORM && l == LINK_CONST) return launch_dims<DIMS, COEF_UNIFORM, LINK_CONST>(a, s);
  return launch_dims<DIMS, COEF_STEP, LINK_CONST>(a, s);
}

template <int COEF, int LINK>
int launch2d_tb2(FusedArgs<F32> a, cudaStream_t s) {
  auto k = fused2d_tb2_kernel<F32, COEF, LINK>;
  const int warps = workers2d<fused2d_tb2_kernel<F32, COEF, LINK>>();
  const long long strips = (a.N[0] + kCoreTb - 1) / kCoreTb;
  if (a.chunk <= 0 || a.chunk > a.N[1]) a.chunk = plan_chunk(strips, a.N[1], warps, 32, 1.0);
  const long long items = strips * ((a.N[1] + a.chunk - 1) / a.chunk);
  long long w = items < warps ? items : warps;
  if (a.e_partials && w > (long long)kFusedEMaxBlocks * kFused2dWarps) w = (long long)kFusedEMaxBlocks * kFused2dWarps;
  a.workers = (int)w;
  const int blocks = (int)((w + kFused2dWarps - 1) / kFused2dWarps);
  k<<<(unsigned)blocks, 32 * kFused2dWarps, 0, s>>>(a);
  return blocks;
}

template <int DIMS, int COEF, int LINK>
void batch_dims(const BatchArgs<F32>& b, long long total, cudaStream_t s) {
  if (DIMS == 3) launch3d_batch<COEF, LINK>(b, total, s);
  else launch2d_batch<COEF, LINK>(b, total, s);
}

}  // namespace

int launch_fused2d_tb2(const FusedArgs<F32>& a, cudaStream_t s) {
  const int c = a.hu.coef_mode, l = a.hu.link_mode;
  if (c == COEF_UNIFORM && l == LINK_NONE) return launch2d_tb2<COEF_UNIFORM, LINK_NONE>(a, s);
  if (c == COEF_STEP && l == LINK_NONE) return launch2d_tb2<COEF_STEP, LINK_NONE>(a, s);
  if (c == COEF_UNIFORM && l == LINK_CONST) return launch2d_tb2<COEF_UNIFORM, LINK_CONST>(a, s);
  if (c == COEF_STEP && l == LINK_CONST) return launch2d_tb2<COEF_STEP, LINK_CONST>(a, s);
  if (c == COEF_TABLE && l == LINK_NONE) return launch2d_tb2<COEF_TABLE, LINK_NONE>(a, s);
  if (c == COEF_SOFTCORE && l == LINK_NONE) return launch2d_tb2<COEF_SOFTCORE, LINK_NONE>(a, s);
  if (c == COEF_SOFTCORR && l == LINK_NONE) return launch2d_tb2<COEF_SOFTCORR, LINK_NONE>(a, s);
  return 0;
}

int fused_chunk_tb2(const int N[3]) {
  const int warps = workers2d<fused2d_tb2_kernel<F32, COEF_UNIFORM, LINK_NONE>>();
  const long long strips = (N[0] + kCoreTb - 1) / kCoreTb;
  return plan_chunk(strips, N[1], warps, 32, 1.0);
}

long long fused_items_tb2(const int N[3], int chunk) {
  return (long long)((N[0] + kCoreTb - 1) / kCoreTb) * ((N[1] + chunk - 1) / chunk);
}

void launch_fused2d_tb2_batch(const BatchArgs<F32>& b, long long total, int coef, int link, cudaStream_t s) {
  if (coef == COEF_UNIFORM && link == LINK_NONE) return launch2d_tb2_batch<COEF_UNIFORM, LINK_NONE>(b, total, s);
  if (coef == COEF_STEP && link == LINK_NONE) return launch2d_tb2_batch<COEF_STEP, LINK_NONE>(b, total, s);
  if (coef == COEF_UNIFORM && link == LINK_CONST) return launch2d_tb2_batch<COEF_UNIFORM, LINK_CONST>(b, total, s);
  return launch2d_tb2_batch<COEF_STEP, LINK_CONST>(b, total, s);
}

int fused_chunk(int dims, const int N[3]) {
  if (dims == 3) {
    const int resident = workers3d<fused3d_kernel<F32, COEF_UNIFORM, LINK_NONE>>();
    const long long tiles = (long long)((N[0] + CX - 1) / CX) * ((N[1] + CY - 1) / CY);
    return plan_chunk(tiles, N[2], resident, 4, 0.5);
  }
  const int warps = workers2d<fused2d_kernel<F32, COEF_UNIFORM, LINK_NONE>>();
  const long long strips = (N[0] + kCore - 1) / kCore;
  return plan_chunk(strips, N[1], warps, 16, 1.0);
}

int fused_candidates(int dims, const int N[3], int two_step, int* out, int max) {
  if (dims == 3) {
    const int resident = workers3d<fused3d_kernel<F32, COEF_UNIFORM, LINK_NONE>>();
    const long long tiles = (long long)((N[0] + CX - 1) / CX) * ((N[1] + CY - 1) / CY);
    return rank_chunks(tiles, N[2], resident, 4, 0.5, out, max);
  }
  if (two_step) {
    const int warps = workers2d<fused2d_tb2_kernel<F32, COEF_UNIFORM, LINK_NONE>>();
    const long long strips = (N[0] + kCoreTb - 1) / kCoreTb;
    return rank_chunks(strips, N[1], warps, 32, 1.0, out, max);
  }
  const int warps = workers2d<fused2d_kernel<F32, COEF_UNIFORM, LINK_NONE>>();
  const long long strips = (N[0] + kCore - 1) / kCore;
  return rank_chunks(strips, N[1], warps, 16, 1.0, out, max);
}

long long fused_items(int dims, const int N[3], int chunk) {
  const int n[3] = {N[0], N[1], N[2]};
  return dims == 3 ? items3d(n, n[2], chunk) : items2d(n, n[1], chunk);
}

template <>
void launch_fused_batch<F32, 3>(const BatchArgs<F32>& b, long long total, int coef, int link,
                                cudaStream_t s) {
  if (coef == COEF_UNIFORM && link == LINK_NONE) return batch_dims<3, COEF_UNIFORM, LINK_NONE>(b, total, s);
  if (coef == COEF_STEP && link == LINK_NONE) return batch_dims<3, COEF_STEP, LINK_NONE>(b, total, s);
  if (coef == COEF_UNIFORM && link == LINK_CONST) return batch_dims<3, COEF_UNIFORM, LINK_CONST>(b, total, s);
  return batch_dims<3, COEF_STEP, LINK_CONST>(b, total, s);
}
template <>
void launch_fused_batch<F32, 2>(const BatchArgs<F32>& b, long long total, int coef, int link,
                                cudaStream_t s) {
  if (coef == COEF_UNIFORM && link == LINK_NONE) return batch_dims<2, COEF_UNIFORM, LINK_NONE>(b, total, s);
  if (coef == COEF_STEP && link == LINK_NONE) return batch_dims<2, COEF_STEP, LINK_NONE>(b, total, s);
  if (coef == COEF_UNIFORM && link == LINK_CONST) return batch_dims<2, COEF_UNIFORM, LINK_CONST>(b, total, s);
  return batch_dims<2, COEF_STEP, LINK_CONST>(b, total, s);
}

template <>
int launch_fused<F32, 3>(const FusedArgs<F32>& a, cudaStream_t s) {
  return dispatch<3>(a, s);
}
template <>
int launch_fused<F32, 2>(const FusedArgs<F32>& a, cudaStream_t s) {
  return dispatch<2>(a, s);
}

}  // namespace dirac
