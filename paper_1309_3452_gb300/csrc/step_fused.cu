// One kernel per full time step (both half-steps of Eqs. ss1-ss4 / Eqs.
// scheme2Deq ff.), out of place: every value is read once from HBM and
// written once, neighbours come from registers, shuffles and shared memory.
//
// (3+1)D: a block of 512 threads covers a 34 x 15 tile of cells in (x, y)
// (thread t sits at lx = t % 34, ly = t / 34; the last two threads are spare)
// and marches along z.  Columns 0, 33 and rows 0, 14 are a one-cell halo:
// they load and compute like every other thread, so the new upper values the
// 32 x 13 interior needs from outside the tile exist in shared memory, but
// they store nothing.  Per z level k the block
//   1. loads the old A(k+1), C(k+1), D(k+1) and B(k) (B, C sit at z+1/2),
//   2. publishes the old D(k+1), C(k) in shared memory,
//   3. computes the new A(k+1) and B(k)      (upper half-step, t -> t+dt/2),
//   4. publishes them,
//   5. computes the new C(k) and D(k)        (lower half-step, t -> t+dt),
// keeping old C, D and new A, B of the previous level in registers for the z
// differences.  A run of levels starts one level early to rebuild that state.
//
// (2+1)D: each warp owns a strip of 32 cells in x (30 interior) and marches
// along y with the same pipeline (u0 ~ A, u1 ~ B, v1 ~ C, v0 ~ D with y as the
// marching axis); x neighbours come from warp shuffles, no block barrier.
//
// Scheduling: the grid holds exactly the blocks that fit on the GPU at once
// (or fewer for small grids) and every block (warp, in (2+1)D) takes an equal
// contiguous run of the (tile, level) items, so all finish together; a run
// that crosses a tile boundary restarts the march there.
//
// Cells outside the grid (ragged last tiles) are wrapped periodically, so
// they compute correct duplicates and only the owning interior thread stores.
#include "kernels.cuh"

namespace dirac {

namespace {

constexpr int TW = 34, TH = 15;        // (3+1)D tile in threads
constexpr int CX = TW - 2, CY = TH - 2; // interior
constexpr int kThreads3d = 512;
constexpr int kSmemRows = 16;           // TH rows + the spare threads' row

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

template <class P, int COEF, int LINK>
__global__ void __launch_bounds__(kThreads3d, 2) fused3d_kernel(const FusedArgs<P> a) {
  using C = typename P::cplx;
  __shared__ C sC[2][kSmemRows * TW];     // old C(k), both sublattices
  __shared__ C sD[2][kSmemRows * TW];     // old D(k+1)
  __shared__ C sB[2][kSmemRows * TW];     // new B(k)
  __shared__ C sA[2][2][kSmemRows * TW];  // new A, double-buffered by level parity

  const int t = threadIdx.x;
  const int lx = t % TW, ly = t / TW;
  const int Nx = a.N[0], Ny = a.N[1], Nz = a.N[2];
  const int tiles_x = (Nx + CX - 1) / CX;
  const long long total = (long long)tiles_x * ((Ny + CY - 1) / CY) * Nz;
  long long i = (long long)blockIdx.x * a.per_worker;
  const long long iend = min(total, i + a.per_worker);
  // shared-memory slots of this thread and of its x/y neighbours (clamped at
  // the tile edge: halo threads then read their own slot, values never used)
  const int sxm = lx > 0 ? t - 1 : t, sxp = lx < TW - 1 ? t + 1 : t;
  const int sym = ly > 0 ? t - TW : t, syp = ly < kSmemRows - 1 ? t + TW : t;
  const bool iso = a.iso != 0;
  const long long nxy = (long long)Nx * Ny;

  while (i < iend) {
    const long long tile = i / Nz;
    const int z0 = (int)(i - tile * Nz);
    const int z1 = (int)min((long long)Nz, z0 + (iend - i));
    i += z1 - z0;
    const int gx = (int)(tile % tiles_x) * CX + lx - 1;
    const int gy = (int)(tile / tiles_x) * CY + ly - 1;
    const int x = wrapi(gx, Nx), y = wrapi(gy, Ny);
    const bool core = lx >= 1 && lx <= CX && ly >= 1 && ly <= CY && gx < Nx && gy < Ny;
    const long long cxy = (long long)y * Nx + x;
    const int hx = 2 * x, hy = 2 * y;

    long long o = (long long)wrapi(z0 - 1, Nz) * nxy + cxy;
    C oC0 = ld(a.in[4] + o), oC1 = ld(a.in[5] + o), oD0 = ld(a.in[6] + o), oD1 = ld(a.in[7] + o);
    C nA0 = oC0, nA1 = oC1, nB0 = oD0, nB1 = oD1;  // placeholders: only feed values never stored

    for (int k = z0 - 1; k < z1; ++k) {
      const int zk = k < 0 ? k + Nz : k;
      const int zn = k + 1 >= Nz ? k + 1 - Nz : k + 1;
      const long long ok = zk * nxy + cxy, on = zn * nxy + cxy;
      const C A0 = ld(a.in[0] + on), A1 = ld(a.in[1] + on);
      const C C0n = ld(a.in[4] + on), C1n = ld(a.in[5] + on);
      const C D0n = ld(a.in[6] + on), D1n = ld(a.in[7] + on);
      const C B0 = ld(a.in[2] + ok), B1 = ld(a.in[3] + ok);
      sD[0][t] = D0n;
      sD[1][t] = D1n;
      sC[0][t] = oC0;
      sC[1][t] = oC1;
      __syncthreads();

      // upper half-step: A(k+1) from C(k+1), C(k), D(k+1); B(k) from D(k+1), D(k), C(k)
      C nA0n, nA1n, nB0k, nB1k;
      {
        C nb[6] = {D0n, sD[0][sxm], D1n, sD[1][sym], C0n, oC0};
        const int H[3] = {hx, hy, 2 * zn};
        nA0n = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 0, A0, nb, H, on, a.pstride);
      }
      {
        C nb[6] = {sD[1][sxp], D1n, sD[0][syp], D0n, C1n, oC1};
        const int H[3] = {hx + 1, hy + 1, 2 * zn};
        nA1n = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 1, A1, nb, H, on, a.pstride);
      }
      {
        C nb[6] = {sC[0][sxp], oC0, oC1, sC[1][sym], D0n, oD0};
        const int H[3] = {hx + 1, hy, 2 * zk + 1};
        nB0k = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 2, B0, nb, H, ok, a.pstride);
      }
      {
        C nb[6] = {oC1, sC[1][sxm], sC[0][syp], oC0, D1n, oD1};
        const int H[3] = {hx, hy + 1, 2 * zk + 1};
        nB1k = site_update<P, 3, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 3, B1, nb, H, ok, a.pstride);
      }
      const int pn = (k + 1) & 1, pk = k & 1;
      sB[0][t] = nB0k;
      sB[1][t] = nB1k;
      sA[pn][0][t] = nA0n;
      sA[pn][1][t] = nA1n;
      __syncthreads();

      // lower half-step: C(k) from A(k+1), A(k), B(k); D(k) from B(k), B(k-1), A(k)
      C nC0, nC1, nD0, nD1;
      {
        C nb[6] = {nB0k, sB[0][sxm], nB1k, sB[1][sym], nA0n, nA0};
        const int H[3] = {hx, hy, 2 * zk + 1};
        nC0 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 4, oC0, nb, H, ok, a.pstride);
      }
      {
        C nb[6] = {sB[1][sxp], nB1k, sB[0][syp], nB0k, nA1n, nA1};
        const int H[3] = {hx + 1, hy + 1, 2 * zk + 1};
        nC1 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 5, oC1, nb, H, ok, a.pstride);
      }
      {
        C nb[6] = {sA[pk][0][sxp], nA0, nA1, sA[pk][1][sym], nB0k, nB0};
        const int H[3] = {hx + 1, hy, 2 * zk};
        nD0 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 6, oD0, nb, H, ok, a.pstride);
      }
      {
        C nb[6] = {nA1, sA[pk][1][sxm], sA[pk][0][syp], nA0, nB1k, nB1};
        const int H[3] = {hx, hy + 1, 2 * zk};
        nD1 = site_update<P, 3, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 7, oD1, nb, H, ok, a.pstride);
      }
      if (core) {
        if (k >= z0) {
          a.out[2][ok] = nB0k;
          a.out[3][ok] = nB1k;
          a.out[4][ok] = nC0;
          a.out[5][ok] = nC1;
          a.out[6][ok] = nD0;
          a.out[7][ok] = nD1;
        }
        if (k + 1 < z1) {
          a.out[0][on] = nA0n;
          a.out[1][on] = nA1n;
        }
      }
      oC0 = C0n;
      oC1 = C1n;
      oD0 = D0n;
      oD1 = D1n;
      nA0 = nA0n;
      nA1 = nA1n;
      nB0 = nB0k;
      nB1 = nB1k;
    }
  }
}

template <class P, int COEF, int LINK>
__global__ void __launch_bounds__(32 * kFused2dWarps) fused2d_kernel(const FusedArgs<P> a) {
  using C = typename P::cplx;
  const int lane = threadIdx.x & 31;
  const long long worker = (long long)blockIdx.x * kFused2dWarps + (threadIdx.x >> 5);
  const int Nx = a.N[0], Ny = a.N[1];
  const int strips = (Nx + kCore - 1) / kCore;
  const long long total = (long long)strips * Ny;
  long long i = worker * a.per_worker;
  const long long iend = min(total, i + a.per_worker);
  const bool iso = a.iso != 0;
  while (i < iend) {  // uniform per warp
    const int strip = (int)(i / Ny);
    const int y0 = (int)(i - (long long)strip * Ny);
    const int y1 = (int)min((long long)Ny, y0 + (iend - i));
    i += y1 - y0;
    const int gx = strip * kCore + lane - 1;
    const int x = wrapi(gx, Nx);
    const bool core = lane >= 1 && lane <= kCore && gx < Nx;
    const int hx = 2 * x;
    // planes: 0 u0 (0,0)  1 u1 (1,1)  2 v0 (1,0)  3 v1 (0,1)
    long long o = (long long)wrapi(y0 - 1, Ny) * Nx + x;
    C oV0 = ld(a.in[2] + o), oV1 = ld(a.in[3] + o);
    C nU0 = oV0, nU1 = oV1;  // placeholders: only feed values never stored
    for (int k = y0 - 1; k < y1; ++k) {
      const int yk = k < 0 ? k + Ny : k;
      const int yn = k + 1 >= Ny ? k + 1 - Ny : k + 1;
      const long long ok = (long long)yk * Nx + x, on = (long long)yn * Nx + x;
      const C U0 = ld(a.in[0] + on), V0n = ld(a.in[2] + on), V1n = ld(a.in[3] + on);
      const C U1 = ld(a.in[1] + ok);
      // upper: u0(k+1) from v0(k+1) (x), v1(k+1), v1(k) (y); u1(k) from v1(k) (x), v0(k+1), v0(k) (y)
      C nU0n, nU1k;
      {
        C nb[6] = {V0n, shfl_up1(V0n), V1n, oV1, V0n, V0n};
        const int H[3] = {hx, 2 * yn, 0};
        nU0n = site_update<P, 2, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 0, U0, nb, H, on, a.pstride);
      }
      {
        C nb[6] = {shfl_down1(oV1), oV1, V0n, oV0, oV1, oV1};
        const int H[3] = {hx + 1, 2 * yk + 1, 0};
        nU1k = site_update<P, 2, COEF, LINK>(a.hu, a.f, iso, a.ry, a.rz, 1, U1, nb, H, ok, a.pstride);
      }
      // lower: v1(k) from u1(k) (x), u0(k+1), u0(k) (y); v0(k) from u0(k) (x), u1(k), u1(k-1) (y)
      C nV0, nV1;
      {
        C nb[6] = {nU1k, shfl_up1(nU1k), nU0n, nU0, nU1k, nU1k};
        const int H[3] = {hx, 2 * yk + 1, 0};
        nV1 = site_update<P, 2, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 3, oV1, nb, H, ok, a.pstride);
      }
      {
        C nb[6] = {shfl_down1(nU0), nU0, nU1k, nU1, nU0, nU0};
        const int H[3] = {hx + 1, 2 * yk, 0};
        nV0 = site_update<P, 2, COEF, LINK>(a.hl, a.f, iso, a.ry, a.rz, 2, oV0, nb, H, ok, a.pstride);
      }
      if (core) {
        if (k >= y0) {
          a.out[1][ok] = nU1k;
          a.out[2][ok] = nV0;
          a.out[3][ok] = nV1;
        }
        if (k + 1 < y1) a.out[0][on] = nU0n;
      }
      oV0 = V0n;
      oV1 = V1n;
      nU0 = nU0n;
      nU1 = nU1k;
    }
  }
}

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
  return n > 0 ? n : 1;
}

// Grid of at most (resident blocks) with an equal run of items per worker,
// and at least `min_run` items per worker.
template <class K>
long long schedule(K kernel, int threads, long long total, int workers_per_block, int min_run,
                   long long& per_worker) {
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, threads, 0);
  if (per_sm < 1) per_sm = 1;
  long long workers = (long long)sm_count() * per_sm * workers_per_block;
  per_worker = (total + workers - 1) / workers;
  if (per_worker < min_run) per_worker = min_run;
  long long used = (total + per_worker - 1) / per_worker;
  return (used + workers_per_block - 1) / workers_per_block;
}

template <int COEF, int LINK>
void launch3d(FusedArgs<F32> a, cudaStream_t s) {
  auto k = fused3d_kernel<F32, COEF, LINK>;
  long long total = (long long)((a.N[0] + CX - 1) / CX) * ((a.N[1] + CY - 1) / CY) * a.N[2];
  long long blocks = schedule(k, kThreads3d, total, 1, 4, a.per_worker);
  k<<<(unsigned)blocks, kThreads3d, 0, s>>>(a);
}

template <int COEF, int LINK>
void launch2d(FusedArgs<F32> a, cudaStream_t s) {
  auto k = fused2d_kernel<F32, COEF, LINK>;
  long long total = (long long)((a.N[0] + kCore - 1) / kCore) * a.N[1];
  long long blocks = schedule(k, 32 * kFused2dWarps, total, kFused2dWarps, 16, a.per_worker);
  k<<<(unsigned)blocks, 32 * kFused2dWarps, 0, s>>>(a);
}

template <int DIMS, int COEF, int LINK>
void launch_dims(const FusedArgs<F32>& a, cudaStream_t s) {
  if (DIMS == 3) launch3d<COEF, LINK>(a, s);
  else launch2d<COEF, LINK>(a, s);
}

template <int DIMS>
void dispatch(const FusedArgs<F32>& a, cudaStream_t s) {
  const int c = a.hu.coef_mode, l = a.hu.link_mode;
  if (c == COEF_GENERAL || l == LINK_GENERAL) return launch_dims<DIMS, kAnyMode, kAnyMode>(a, s);
  if (c == COEF_UNIFORM && l == LINK_NONE) return launch_dims<DIMS, COEF_UNIFORM, LINK_NONE>(a, s);
  if (c == COEF_STEP && l == LINK_NONE) return launch_dims<DIMS, COEF_STEP, LINK_NONE>(a, s);
  if (c == COEF_UNIFORM && l == LINK_CONST) return launch_dims<DIMS, COEF_UNIFORM, LINK_CONST>(a, s);
  return launch_dims<DIMS, COEF_STEP, LINK_CONST>(a, s);
}

}  // namespace

template <>
void launch_fused<F32, 3>(const FusedArgs<F32>& a, cudaStream_t s) {
  dispatch<3>(a, s);
}
template <>
void launch_fused<F32, 2>(const FusedArgs<F32>& a, cudaStream_t s) {
  dispatch<2>(a, s);
}

}  // namespace dirac
