// Reductions of the stored state: the naive norm, the cross terms of the
// conserved functional (Lemma of Sect. 2, Eq. EPM, in its "lower" form; see
// dirac.h) and the partial density used for the Klein-step transmission.
// Every per-site term is formed in FP64 from the stored values (exact
// widening for FP32 states), summed per thread, per warp (shuffles), per
// block (shared memory) and finally over blocks in a fixed order, so the
// result is deterministic for a given grid.
#include "kernels.cuh"

namespace dirac {

namespace {

__device__ __forceinline__ double2 widen(double2 v) { return v; }
__device__ __forceinline__ double2 widen(float2 v) { return make_double2(v.x, v.y); }

__device__ __forceinline__ double2 mul_expm(double2 v, double phi) {  // v * exp(-i phi)
  double s, c;
  sincos(phi, &s, &c);
  return make_double2(c * v.x + s * v.y, c * v.y - s * v.x);
}
__device__ __forceinline__ double2 widen_link(const F64::Link& L) { return L.u; }
__device__ __forceinline__ double2 widen_link(const F32::Link& L) {
  return make_double2((double)L.hi.x + (double)L.lo.x, (double)L.hi.y + (double)L.lo.y);
}

template <int NS>
__device__ __forceinline__ void block_reduce_store(double (&v)[NS], double* out) {
  __shared__ double sh[32][NS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NS; ++k) sh[warp][k] = v[k];
  __syncthreads();
  if (warp == 0) {
    const int nw = blockDim.x >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double x = lane < nw ? sh[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) out[k] = x;
    }
  }
}

template <class P, int DIMS>
__global__ void __launch_bounds__(256) observables_kernel(const ObsArgs<P> a) {
  const long long N0 = a.N[0], N1 = a.N[1], N2 = (DIMS == 3) ? a.N[2] : 1;
  const long long ncell = N0 * N1 * N2;
  const long long Nn[3] = {N0, N1, N2};
  double acc[kObsSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  for (long long cell = blockIdx.x * (long long)blockDim.x + threadIdx.x; cell < ncell;
       cell += (long long)gridDim.x * blockDim.x) {
    const long long j[3] = {cell % N0, (cell / N0) % N1, cell / (N0 * N1)};
#pragma unroll
    for (int plane = 0; plane < nplanes<DIMS>(); ++plane) {
      const double2 G = widen(a.pl[plane][cell]);
      const double n2 = G.x * G.x + G.y * G.y;
      acc[0] += n2;
      long long H[3];
#pragma unroll
      for (int ax = 0; ax < 3; ++ax) H[ax] = 2 * j[ax] + plane_off<DIMS>(plane, ax);
      if (a.dens_axis >= 0 && H[a.dens_axis] >= a.dens_X) acc[4] += n2;
      if (is_upper<DIMS>(plane)) continue;
      const int p = sign_class<DIMS>(plane);
#pragma unroll
      for (int ax = 0; ax < DIMS; ++ax) {
        const typename P::cplx* nb = a.pl[partner<DIMS>(plane, ax)];
        long long jp = j[ax] + nb_shift<DIMS>(plane, ax, +1);
        long long jm = j[ax] + nb_shift<DIMS>(plane, ax, -1);
        jp = jp >= Nn[ax] ? jp - Nn[ax] : jp;
        jm = jm < 0 ? jm + Nn[ax] : jm;
        long long stride = ax == 0 ? 1 : (ax == 1 ? N0 : N0 * N1);
        double2 up = widen(nb[cell + (jp - j[ax]) * stride]);
        double2 dn = widen(nb[cell + (jm - j[ax]) * stride]);
        if (a.link_mode == LINK_CONST) {
          double2 u = widen_link(a.L[ax]);
          up = make_double2(u.x * up.x - u.y * up.y, u.x * up.y + u.y * up.x);
          dn = make_double2(u.x * dn.x + u.y * dn.y, u.x * dn.y - u.y * dn.x);
        } else if (a.link_mode == LINK_GENERAL) {
          up = mul_expm(up, link_phase(a.f, DIMS, H, ax, +1, a.t_links));
          dn = mul_expm(dn, -link_phase(a.f, DIMS, H, ax, -1, a.t_links));
        }
        double2 d = make_double2(up.x - dn.x, up.y - dn.y);
        // s_a d: s_x = 1; s_y = -i (p=0) / +i (p=1); s_z = +1 (p=0) / -1 (p=1)
        double2 sd = d;
        if (ax == 1) sd = p ? make_double2(-d.y, d.x) : make_double2(d.y, -d.x);
        if (ax == 2 && p) sd = make_double2(-d.x, -d.y);
        acc[1 + ax] += G.x * sd.x + G.y * sd.y;  // Re(conj(G) sd)
      }
    }
  }
  block_reduce_store<kObsSums>(acc, a.partials + (long long)blockIdx.x * kObsSums);
}

__global__ void finish_sums_kernel(const double* partials, int nblocks, double* out) {
  // one block of 32*kObsSums threads? keep it simple: warp k sums column k
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
  if (k >= kObsSums) return;
  double x = 0.0;
  for (int b = lane; b < nblocks; b += 32) x += partials[(long long)b * kObsSums + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if (lane == 0) out[k] = x;
}

__global__ void convert_in_kernel(const double2* __restrict__ src, float2* __restrict__ dst,
                                  long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = make_float2(__double2float_rn(src[i].x), __double2float_rn(src[i].y));
}
__global__ void convert_out_kernel(const float2* __restrict__ src, double2* __restrict__ dst,
                                   long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = make_double2(src[i].x, src[i].y);
}

}  // namespace

template <class P, int DIMS>
void launch_observables(const ObsArgs<P>& a, int blocks, cudaStream_t s) {
  observables_kernel<P, DIMS><<<blocks, 256, 0, s>>>(a);
}
template void launch_observables<F64, 2>(const ObsArgs<F64>&, int, cudaStream_t);
template void launch_observables<F64, 3>(const ObsArgs<F64>&, int, cudaStream_t);
template void launch_observables<F32, 2>(const ObsArgs<F32>&, int, cudaStream_t);
template void launch_observables<F32, 3>(const ObsArgs<F32>&, int, cudaStream_t);

void launch_finish_sums(const double* partials, int nblocks, double* out, cudaStream_t s) {
  finish_sums_kernel<<<1, 32 * kObsSums, 0, s>>>(partials, nblocks, out);
}

static unsigned grid_for(long long n) {
  long long b = (n + 255) / 256;
  return (unsigned)(b > 152LL * 32 ? 152LL * 32 : (b < 1 ? 1 : b));
}
void launch_convert_in(const double2* src, float2* dst, long long n, cudaStream_t s) {
  convert_in_kernel<<<grid_for(n), 256, 0, s>>>(src, dst, n);
}
void launch_convert_out(const float2* src, double2* dst, long long n, cudaStream_t s) {
  convert_out_kernel<<<grid_for(n), 256, 0, s>>>(src, dst, n);
}

}  // namespace dirac
