// One kernel per half-step: every thread owns one cell and updates the values
// of one parity class (upper: A0,A1,B0,B1 / u0,u1; lower: C0,C1,D0,D1 /
// v0,v1) in place.  In-place is race-free: a half-step reads only values of
// the other parity (Eqs. ss1-ss4: A,B from C,D at t; C,D from the new A,B).
// This is the plain reference path (and the FP64 validation path); the fused
// kernels compute the same values with the same per-value arithmetic.
#include "kernels.cuh"

namespace dirac {

namespace {

template <class P, int DIMS, bool UPPER, int COEF, int LINK>
__global__ void __launch_bounds__(128) half_step_kernel(const HalfStepArgs<P> a) {
  using C = typename P::cplx;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 4 + threadIdx.y;
  const int z = blockIdx.z;
  const int Nx = a.N[0], Ny = a.N[1], Nz = DIMS == 3 ? a.N[2] : 1;
  if (x >= Nx || y >= Ny) return;
  const long long nxy = (long long)Nx * Ny;
  const long long cell = z * nxy + (long long)y * Nx + x;
  const int j[3] = {x, y, z};
  const int Nn[3] = {Nx, Ny, Nz};
  const long long stride[3] = {1, Nx, nxy};
  constexpr int half = nplanes<DIMS>() / 2;
  constexpr int first = UPPER ? 0 : half;
#pragma unroll
  for (int k = 0; k < half; ++k) {
    const int plane = first + k;
    C* self = a.pl[plane];
    int H[3];
#pragma unroll
    for (int ax = 0; ax < 3; ++ax) H[ax] = 2 * j[ax] + plane_off<DIMS>(plane, ax);
    C nb[6];
#pragma unroll
    for (int ax = 0; ax < DIMS; ++ax) {
      const C* src = a.pl[partner<DIMS>(plane, ax)];
#pragma unroll
      for (int dir = 0; dir < 2; ++dir) {
        int jj = j[ax] + nb_shift<DIMS>(plane, ax, dir == 0 ? +1 : -1);
        jj = jj >= Nn[ax] ? jj - Nn[ax] : (jj < 0 ? jj + Nn[ax] : jj);
        nb[2 * ax + dir] = src[cell + (long long)(jj - j[ax]) * stride[ax]];
      }
    }
    self[cell] = site_update<P, DIMS, COEF, LINK>(a.h, a.f, a.iso != 0, a.ry, a.rz, plane, self[cell],
                                               nb, H, cell, a.pstride, nullptr, nullptr, nullptr, a.N);
  }
}

template <class P, int DIMS, bool UPPER>
void launch_one(const HalfStepArgs<P>& a, cudaStream_t s) {
  dim3 block(32, 4);
  dim3 grid((a.N[0] + 31) / 32, (a.N[1] + 3) / 4, DIMS == 3 ? a.N[2] : 1);
  const int c = a.h.coef_mode, l = a.h.link_mode;
  constexpr bool f32 = sizeof(typename P::real) == 4;
  if (c == COEF_UNIFORM && l == LINK_NONE)
    half_step_kernel<P, DIMS, UPPER, COEF_UNIFORM, LINK_NONE><<<grid, block, 0, s>>>(a);
  else if (c == COEF_STEP && l == LINK_NONE)
    half_step_kernel<P, DIMS, UPPER, COEF_STEP, LINK_NONE><<<grid, block, 0, s>>>(a);
  else if (f32 && c == COEF_TABLE && l == LINK_NONE)  // the FP32 tabulated-potential paths
    half_step_kernel<P, DIMS, UPPER, COEF_TABLE, LINK_NONE><<<grid, block, 0, s>>>(a);
  else if (f32 && c == COEF_SOFTCORE && l == LINK_NONE)  // the FP32 analytic soft core
    half_step_kernel<P, DIMS, UPPER, COEF_SOFTCORE, LINK_NONE><<<grid, block, 0, s>>>(a);
  else if (f32 && c == COEF_SOFTCORE && l == LINK_PLANE)
    half_step_kernel<P, DIMS, UPPER, COEF_SOFTCORE, LINK_PLANE><<<grid, block, 0, s>>>(a);
  else if (f32 && c == COEF_SOFTCORR && l == LINK_NONE)
    half_step_kernel<P, DIMS, UPPER, COEF_SOFTCORR, LINK_NONE><<<grid, block, 0, s>>>(a);
  else if (f32 && c == COEF_SOFTCORR && l == LINK_PLANE)
    half_step_kernel<P, DIMS, UPPER, COEF_SOFTCORR, LINK_PLANE><<<grid, block, 0, s>>>(a);
  else if (f32 && c == COEF_TABLE && l == LINK_PLANE)
    half_step_kernel<P, DIMS, UPPER, COEF_TABLE, LINK_PLANE><<<grid, block, 0, s>>>(a);
  else if (f32 && c == COEF_UNIFORM && l == LINK_PLANE)
    half_step_kernel<P, DIMS, UPPER, COEF_UNIFORM, LINK_PLANE><<<grid, block, 0, s>>>(a);
  else if (f32 && c == COEF_STEP && l == LINK_PLANE)
    half_step_kernel<P, DIMS, UPPER, COEF_STEP, LINK_PLANE><<<grid, block, 0, s>>>(a);
  else
    half_step_kernel<P, DIMS, UPPER, kAnyMode, kAnyMode><<<grid, block, 0, s>>>(a);
}

}  // namespace

template <class P, int DIMS>
void launch_half_step(const HalfStepArgs<P>& a, bool upper, cudaStream_t s) {
  if (upper)
    launch_one<P, DIMS, true>(a, s);
  else
    launch_one<P, DIMS, false>(a, s);
}

template void launch_half_step<F64, 2>(const HalfStepArgs<F64>&, bool, cudaStream_t);
template void launch_half_step<F64, 3>(const HalfStepArgs<F64>&, bool, cudaStream_t);
template void launch_half_step<F32, 2>(const HalfStepArgs<F32>&, bool, cudaStream_t);
template void launch_half_step<F32, 3>(const HalfStepArgs<F32>&, bool, cudaStream_t);

}  // namespace dirac
