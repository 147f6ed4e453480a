// One kernel per full time step (both half-steps of Eqs. ss1-ss4 / Eqs.
// scheme2Deq ff.), out of place: every value is read once from HBM and
// written once, neighbours come from registers, shuffles and shared memory.
//
// (3+1)D: a block is a 32 x 16 tile of cells in (x, y) that marches along z
// over a chunk of levels.  Thread (lx, ly) owns the column (x, y).  Lanes 0 and
// 31 and rows 0 and 15 are a one-cell halo: they load and compute like every
// other thread (so the upper values the interior needs from outside the tile
// are available) but store nothing.  The interior is 30 x 14 cells; tiles
// overlap by two cells per axis.  Per z level k the block
//   1. loads the old A(k+1), C(k+1), D(k+1) and B(k) (B, C sit at z+1/2),
//   2. publishes the old D(k+1), C(k) in shared memory,
//   3. computes the new A(k+1) and B(k)      (upper half-step, t -> t+dt/2),
//   4. publishes them,
//   5. computes the new C(k) and D(k)        (lower half-step, t -> t+dt),
// keeping old C, D and new A, B of the previous level in registers for the z
// differences.  A chunk starts one level early to rebuild that state.
//
// (2+1)D: each warp owns a strip of 32 cells in x (30 interior) and marches
// along y with the same pipeline (u0 ~ A, u1 ~ B, v1 ~ C, v0 ~ D with y as the
// marching axis); x neighbours come from warp shuffles, no block barrier.
//
// Cells outside the grid (ragged last tiles) are wrapped periodically, so
// they compute correct duplicates and only the owning interior thread stores.
#include "kernels.cuh"

namespace dirac {

namespace {

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

template <class P, bool GENERAL>
__global__ void __launch_bounds__(32 * kFused3dRows, 2) fused3d_kernel(const FusedArgs<P> a) {
  using C = typename P::cplx;
  constexpr int WY = kFused3dRows;
  __shared__ C sC[2][WY][32];     // old C(k), both sublattices
  __shared__ C sD[2][WY][32];     // old D(k+1)
  __shared__ C sB[2][WY][32];     // new B(k)
  __shared__ C sA[2][2][WY][32];  // new A, double-buffered by level parity

  const int lx = threadIdx.x, ly = threadIdx.y;
  const int Nx = a.N[0], Ny = a.N[1], Nz = a.N[2];
  const int gx = blockIdx.x * kCore + lx - 1;
  const int gy = blockIdx.y * (WY - 2) + ly - 1;
  const int x = wrapi(gx, Nx), y = wrapi(gy, Ny);
  const bool core = lx >= 1 && lx <= kCore && ly >= 1 && ly <= WY - 2 && gx < Nx && gy < Ny;
  const int z0 = blockIdx.z * a.chunk;
  const int z1 = min(z0 + a.chunk, Nz);
  const long long nxy = (long long)Nx * Ny;
  const long long cxy = (long long)y * Nx + x;
  const int xm = max(lx - 1, 0), xp = min(lx + 1, 31), ym = max(ly - 1, 0), yp = min(ly + 1, WY - 1);
  const bool iso = a.iso != 0;
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
    sD[0][ly][lx] = D0n;
    sD[1][ly][lx] = D1n;
    sC[0][ly][lx] = oC0;
    sC[1][ly][lx] = oC1;
    __syncthreads();

    // upper half-step: A(k+1) from C(k+1), C(k), D(k+1); B(k) from D(k+1), D(k), C(k)
    C nA0n, nA1n, nB0k, nB1k;
    {
      C nb[6] = {D0n, sD[0][ly][xm], D1n, sD[1][ym][lx], C0n, oC0};
      const int H[3] = {hx, hy, 2 * zn};
      nA0n = site_update<P, 3, GENERAL>(a.hu, a.f, iso, a.ry, a.rz, 0, A0, nb, H, on, a.pstride);
    }
    {
      C nb[6] = {sD[1][ly][xp], D1n, sD[0][yp][lx], D0n, C1n, oC1};
      const int H[3] = {hx + 1, hy + 1, 2 * zn};
      nA1n = site_update<P, 3, GENERAL>(a.hu, a.f, iso, a.ry, a.rz, 1, A1, nb, H, on, a.pstride);
    }
    {
      C nb[6] = {sC[0][ly][xp], oC0, oC1, sC[1][ym][lx], D0n, oD0};
      const int H[3] = {hx + 1, hy, 2 * zk + 1};
      nB0k = site_update<P, 3, GENERAL>(a.hu, a.f, iso, a.ry, a.rz, 2, B0, nb, H, ok, a.pstride);
    }
    {
      C nb[6] = {oC1, sC[1][ly][xm], sC[0][yp][lx], oC0, D1n, oD1};
      const int H[3] = {hx, hy + 1, 2 * zk + 1};
      nB1k = site_update<P, 3, GENERAL>(a.hu, a.f, iso, a.ry, a.rz, 3, B1, nb, H, ok, a.pstride);
    }
    const int pn = (k + 1) & 1, pk = k & 1;
    sB[0][ly][lx] = nB0k;
    sB[1][ly][lx] = nB1k;
    sA[pn][0][ly][lx] = nA0n;
    sA[pn][1][ly][lx] = nA1n;
    __syncthreads();

    // lower half-step: C(k) from A(k+1), A(k), B(k); D(k) from B(k), B(k-1), A(k)
    C nC0, nC1, nD0, nD1;
    {
      C nb[6] = {nB0k, sB[0][ly][xm], nB1k, sB[1][ym][lx], nA0n, nA0};
      const int H[3] = {hx, hy, 2 * zk + 1};
      nC0 = site_update<P, 3, GENERAL>(a.hl, a.f, iso, a.ry, a.rz, 4, oC0, nb, H, ok, a.pstride);
    }
    {
      C nb[6] = {sB[1][ly][xp], nB1k, sB[0][yp][lx], nB0k, nA1n, nA1};
      const int H[3] = {hx + 1, hy + 1, 2 * zk + 1};
      nC1 = site_update<P, 3, GENERAL>(a.hl, a.f, iso, a.ry, a.rz, 5, oC1, nb, H, ok, a.pstride);
    }
    {
      C nb[6] = {sA[pk][0][ly][xp], nA0, nA1, sA[pk][1][ym][lx], nB0k, nB0};
      const int H[3] = {hx + 1, hy, 2 * zk};
      nD0 = site_update<P, 3, GENERAL>(a.hl, a.f, iso, a.ry, a.rz, 6, oD0, nb, H, ok, a.pstride);
    }
    {
      C nb[6] = {nA1, sA[pk][1][ly][xm], sA[pk][0][yp][lx], nA0, nB1k, nB1};
      const int H[3] = {hx, hy + 1, 2 * zk};
      nD1 = site_update<P, 3, GENERAL>(a.hl, a.f, iso, a.ry, a.rz, 7, oD1, nb, H, ok, a.pstride);
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

template <class P, bool GENERAL>
__global__ void __launch_bounds__(32 * kFused2dWarps) fused2d_kernel(const FusedArgs<P> a) {
  using C = typename P::cplx;
  const int lane = threadIdx.x & 31;
  const int strip = blockIdx.x * kFused2dWarps + (threadIdx.x >> 5);
  const int Nx = a.N[0], Ny = a.N[1];
  if (strip * kCore >= Nx) return;  // whole warp
  const int gx = strip * kCore + lane - 1;
  const int x = wrapi(gx, Nx);
  const bool core = lane >= 1 && lane <= kCore && gx < Nx;
  const int y0 = blockIdx.y * a.chunk;
  const int y1 = min(y0 + a.chunk, Ny);
  const bool iso = a.iso != 0;
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
      nU0n = site_update<P, 2, GENERAL>(a.hu, a.f, iso, a.ry, a.rz, 0, U0, nb, H, on, a.pstride);
    }
    {
      C nb[6] = {shfl_down1(oV1), oV1, V0n, oV0, oV1, oV1};
      const int H[3] = {hx + 1, 2 * yk + 1, 0};
      nU1k = site_update<P, 2, GENERAL>(a.hu, a.f, iso, a.ry, a.rz, 1, U1, nb, H, ok, a.pstride);
    }
    // lower: v1(k) from u1(k) (x), u0(k+1), u0(k) (y); v0(k) from u0(k) (x), u1(k), u1(k-1) (y)
    C nV0, nV1;
    {
      C nb[6] = {nU1k, shfl_up1(nU1k), nU0n, nU0, nU1k, nU1k};
      const int H[3] = {hx, 2 * yk + 1, 0};
      nV1 = site_update<P, 2, GENERAL>(a.hl, a.f, iso, a.ry, a.rz, 3, oV1, nb, H, ok, a.pstride);
    }
    {
      C nb[6] = {shfl_down1(nU0), nU0, nU1k, nU1, nU0, nU0};
      const int H[3] = {hx + 1, 2 * yk, 0};
      nV0 = site_update<P, 2, GENERAL>(a.hl, a.f, iso, a.ry, a.rz, 2, oV0, nb, H, ok, a.pstride);
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

}  // namespace

template <>
void launch_fused<F32, 3>(const FusedArgs<F32>& a, cudaStream_t s) {
  dim3 block(32, kFused3dRows);
  dim3 grid((a.N[0] + kCore - 1) / kCore, (a.N[1] + kFused3dRows - 3) / (kFused3dRows - 2),
            (a.N[2] + a.chunk - 1) / a.chunk);
  if (a.general)
    fused3d_kernel<F32, true><<<grid, block, 0, s>>>(a);
  else
    fused3d_kernel<F32, false><<<grid, block, 0, s>>>(a);
}

template <>
void launch_fused<F32, 2>(const FusedArgs<F32>& a, cudaStream_t s) {
  int strips = (a.N[0] + kCore - 1) / kCore;
  dim3 block(32 * kFused2dWarps);
  dim3 grid((strips + kFused2dWarps - 1) / kFused2dWarps, (a.N[1] + a.chunk - 1) / a.chunk);
  if (a.general)
    fused2d_kernel<F32, true><<<grid, block, 0, s>>>(a);
  else
    fused2d_kernel<F32, false><<<grid, block, 0, s>>>(a);
}

}  // namespace dirac
