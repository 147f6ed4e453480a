// One kernel per half-step: every thread owns one cell and updates the values
// of one parity class (upper: A0,A1,B0,B1 / u0,u1; lower: C0,C1,D0,D1 /
// v0,v1) in place.  In-place is race-free: a half-step reads only values of
// the other parity (Eqs. ss1-ss4: A,B from C,D at t; C,D from the new A,B).
#include "kernels.cuh"

namespace dirac {

namespace {

__device__ __forceinline__ F64::Coef coef_from(const double2& a, const double2& g, F64*) {
  return F64::Coef{a, g};
}
__device__ __forceinline__ float2 hi2(double2 v) {
  return make_float2(__double2float_rn(v.x), __double2float_rn(v.y));
}
__device__ __forceinline__ float2 lo2(double2 v, float2 h) {
  return make_float2(__double2float_rn(v.x - (double)h.x), __double2float_rn(v.y - (double)h.y));
}
__device__ __forceinline__ F32::Coef coef_from(const double2& a, const double2& g, F32*) {
  F32::Coef c;
  c.a_hi = hi2(a);
  c.a_lo = lo2(a, c.a_hi);
  c.g_hi = hi2(g);
  c.g_lo = lo2(g, c.g_hi);
  return c;
}
__device__ __forceinline__ F64::Link link_from(double phi, F64*) {
  double s, c;
  sincos(phi, &s, &c);
  return F64::Link{make_double2(c, -s)};  // exp(-i phi)
}
__device__ __forceinline__ F32::Link link_from(double phi, F32*) {
  double s, c;
  sincos(phi, &s, &c);
  double2 u = make_double2(c, -s);
  F32::Link L;
  L.hi = hi2(u);
  L.lo = lo2(u, L.hi);
  return L;
}

template <class P, int DIMS, bool UPPER>
__global__ void __launch_bounds__(256) half_step_kernel(const HalfStepArgs<P> a) {
  using C = typename P::cplx;
  const long long N0 = a.N[0], N1 = a.N[1], N2 = (DIMS == 3) ? a.N[2] : 1;
  const long long ncell = N0 * N1 * N2;
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    const long long j[3] = {cell % N0, (cell / N0) % N1, cell / (N0 * N1)};
    const long long Nn[3] = {N0, N1, N2};
    constexpr int half = nplanes<DIMS>() / 2;
    constexpr int first = UPPER ? 0 : half;
#pragma unroll
    for (int k = 0; k < half; ++k) {
      const int plane = first + k;
      C* self = a.pl[plane];
      const C F = self[cell];
      long long H[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) H[ax] = 2 * j[ax] + plane_off<DIMS>(plane, ax);
      C d[3];
#pragma unroll
      for (int ax = 0; ax < DIMS; ++ax) {
        const C* nb = a.pl[partner<DIMS>(plane, ax)];
        const int sp = nb_shift<DIMS>(plane, ax, +1), sm = nb_shift<DIMS>(plane, ax, -1);
        long long jp = j[ax] + sp, jm = j[ax] + sm;
        jp = jp >= Nn[ax] ? jp - Nn[ax] : jp;
        jm = jm < 0 ? jm + Nn[ax] : jm;
        long long stride = ax == 0 ? 1 : (ax == 1 ? N0 : N0 * N1);
        C up = nb[cell + (jp - j[ax]) * stride];
        C dn = nb[cell + (jm - j[ax]) * stride];
        if (a.link_mode == LINK_CONST) {
          up = link_mul(a.L[ax], up);
          dn = link_mulc(a.L[ax], dn);
        } else if (a.link_mode == LINK_GENERAL) {
          up = link_mul(link_from(link_phase(a.f, DIMS, H, ax, +1, a.t), (P*)nullptr), up);
          // exp(+i phi-) = conj(exp(-i phi-))
          dn = link_mulc(link_from(link_phase(a.f, DIMS, H, ax, -1, a.t), (P*)nullptr), dn);
        }
        d[ax] = csub(up, dn);
      }
      if (DIMS == 2) d[2] = d[0];
      const C S = combine<P, DIMS>(d[0], d[1], d[2], sign_class<DIMS>(plane), a.iso != 0, a.ry, a.rz);
      typename P::Coef c = a.c_in;
      if (a.coef_mode == COEF_STEP) {
        if (H[a.step_axis] >= a.step_X) c = a.c_out;
      } else if (a.coef_mode == COEF_GENERAL) {
        double V = potential_at(a.f, DIMS, H[0], H[1], H[2], cell, a.pstride, plane, a.t);
        double th = a.f.dt * (a.beta * a.f.m + V) * 0.5;
        double2 al, ga;
        coef_from_theta(th, a.f.rx, al, ga);
        c = coef_from(al, ga, (P*)nullptr);
      }
      self[cell] = apply(c, F, S);
    }
  }
}

}  // namespace

template <class P, int DIMS>
void launch_half_step(const HalfStepArgs<P>& a, bool upper, cudaStream_t s) {
  long long ncell = (long long)a.N[0] * a.N[1] * (DIMS == 3 ? a.N[2] : 1);
  long long blocks = (ncell + 255) / 256;
  if (blocks > 152LL * 64) blocks = 152LL * 64;
  if (upper)
    half_step_kernel<P, DIMS, true><<<(unsigned)blocks, 256, 0, s>>>(a);
  else
    half_step_kernel<P, DIMS, false><<<(unsigned)blocks, 256, 0, s>>>(a);
}

template void launch_half_step<F64, 2>(const HalfStepArgs<F64>&, bool, cudaStream_t);
template void launch_half_step<F64, 3>(const HalfStepArgs<F64>&, bool, cudaStream_t);
template void launch_half_step<F32, 2>(const HalfStepArgs<F32>&, bool, cudaStream_t);
template void launch_half_step<F32, 3>(const HalfStepArgs<F32>&, bool, cudaStream_t);

}  // namespace dirac
