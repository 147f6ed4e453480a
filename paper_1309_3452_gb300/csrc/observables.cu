// Reductions of the stored state: the naive norm, the cross terms of the
// conserved functional (Lemma of Sect. 2, Eq. EPM, in its "lower" form; see
// dirac.h) and the partial density used for the Klein-step transmission.
// One thread per cell (z strided over the grid's z blocks): the cell's terms
// are summed in the state's precision, then accumulated in FP64 per thread,
// per warp (shuffles), per block (shared memory) and finally over blocks in a
// fixed order, so the result is deterministic for a given grid.
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

template <int NS>
__device__ __forceinline__ void block_reduce_store(double (&v)[NS], double* out) {
  __shared__ double sh[32][NS];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
  for (int k = 0; k < NS; ++k)
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_down_sync(0xffffffffu, v[k], o);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NS; ++k) sh[warp][k] = v[k];
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x * blockDim.y) >> 5;
#pragma unroll
    for (int k = 0; k < NS; ++k) {
      double x = lane < nw ? sh[lane][k] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
      if (lane == 0) out[k] = x;
    }
  }
}

// Per-cell terms are formed in the working precision of the state (FP32
// states: every term is a product of two stored floats, rounded once; the
// FP64 accumulation over cells keeps the sum accurate), except with
// plane-wave link factors, which are evaluated in FP64.
template <class P, int DIMS>
__global__ void __launch_bounds__(256) observables_kernel(const ObsArgs<P> a) {
  using C = typename P::cplx;
  using R = typename P::real;
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * 8 + threadIdx.y;
  const int Nx = a.N[0], Ny = a.N[1], Nz = DIMS == 3 ? a.N[2] : 1;
  const long long nxy = (long long)Nx * Ny;
  double acc[kObsSums] = {0.0, 0.0, 0.0, 0.0, 0.0};
  // (2+1)D: the summed rows zlo .. zlo + nzu - 1, fields at the global row
  const bool row_in = DIMS == 3 || (y >= a.zlo && y < a.zlo + a.nzu);
  int yg = y;
  if (DIMS == 2) {
    yg = a.zorg + y;  // in [-1, 2 Nzg): one wrap at most
    if (yg < 0) yg += a.Nzg;
    else if (yg >= a.Nzg) yg -= a.Nzg;
  }
  if (x < Nx && y < Ny && row_in) {
    // the summed levels zlo .. zlo + nzu - 1; fields at their global level
    for (int zz = blockIdx.z; zz < (DIMS == 3 ? a.nzu : 1); zz += gridDim.z) {
      const int z = DIMS == 3 ? a.zlo + zz : 0;
      int zg = DIMS == 3 ? a.zorg + z : 0;  // in [-1, 2 Nzg): one wrap at most
      if (zg < 0) zg += a.Nzg;
      else if (zg >= a.Nzg) zg -= a.Nzg;
      const long long cell = z * nxy + (long long)y * Nx + x;
      const int j[3] = {x, y, z};
      const int Nn[3] = {Nx, Ny, Nz};
      const long long stride[3] = {1, Nx, nxy};
      R cn = 0, cd = 0, cb[3] = {0, 0, 0};
#pragma unroll
      for (int plane = 0; plane < nplanes<DIMS>(); ++plane) {
        const C G = a.pl[plane][cell];
        const R n2 = G.x * G.x + G.y * G.y;
        cn += n2;
        long long H[3];
#pragma unroll
        for (int ax = 0; ax < 3; ++ax)
          H[ax] = 2 * (ax == 2 ? zg : (ax == 1 ? yg : j[ax])) + plane_off<DIMS>(plane, ax);
        const long long hd = a.dens_axis == 0 ? H[0] : (a.dens_axis == 1 ? H[1] : H[2]);
        if (a.dens_axis >= 0 && hd >= a.dens_X) cd += n2;
        if (is_upper<DIMS>(plane)) continue;
        const int p = sign_class<DIMS>(plane);
#pragma unroll
        for (int ax = 0; ax < DIMS; ++ax) {
          const C* nb = a.pl[partner<DIMS>(plane, ax)];
          int jp = j[ax] + nb_shift<DIMS>(plane, ax, +1);
          int jm = j[ax] + nb_shift<DIMS>(plane, ax, -1);
          jp = jp >= Nn[ax] ? jp - Nn[ax] : jp;
          jm = jm < 0 ? jm + Nn[ax] : jm;
          C up = nb[cell + (long long)(jp - j[ax]) * stride[ax]];
          C dn = nb[cell + (long long)(jm - j[ax]) * stride[ax]];
          R re, im;
          if (a.link_mode == LINK_PLANE) {
            // a plane wave with its wave vector across the polarisation (and no
            // constant A on other axes): a phase on the polarisation axis only,
            // the same for both links of the value (k has no component along them)
            if (ax == a.f.Apw_pol) {
              double sn, cs;
              sincos(link_phase(a.f, DIMS, H, ax, +1, a.t_links), &sn, &cs);
              const double2 u = widen(up), v = widen(dn);
              // exp(-i phi) up - exp(+i phi) dn = cos phi (up - dn) - i sin phi (up + dn)
              re = (R)(cs * (u.x - v.x) + sn * (u.y + v.y));
              im = (R)(cs * (u.y - v.y) - sn * (u.x + v.x));
            } else {
              re = up.x - dn.x;
              im = up.y - dn.y;
            }
          } else if (a.link_mode == LINK_GENERAL || a.link_mode == LINK_TABLE) {
            double2 u = mul_expm(widen(up), link_phase_site(a.f, DIMS, H, ax, +1, a.t_links, plane, cell));
            double2 v = mul_expm(widen(dn), -link_phase_site(a.f, DIMS, H, ax, -1, a.t_links, plane, cell));
            re = (R)(u.x - v.x);
            im = (R)(u.y - v.y);
          } else {
            if (a.link_mode == LINK_CONST) {
              up = link_mul(a.L[ax], up);
              dn = link_mulc(a.L[ax], dn);
            }
            re = up.x - dn.x;
            im = up.y - dn.y;
          }
          // s_a d: s_x = 1; s_y = -i (p=0) / +i (p=1); s_z = +1 (p=0) / -1 (p=1)
          R sre = re, sim = im;
          if (ax == 1) {
            sre = p ? -im : im;
            sim = p ? re : -re;
          }
          if (ax == 2 && p) {
            sre = -re;
            sim = -im;
          }
          cb[ax] += G.x * sre + G.y * sim;  // Re(conj(G) s d)
        }
      }
      acc[0] += (double)cn;
      acc[1] += (double)cb[0];
      acc[2] += (double)cb[1];
      acc[3] += (double)cb[2];
      acc[4] += (double)cd;
    }
  }
  const long long b = ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  block_reduce_store<kObsSums>(acc, a.partials + b * kObsSums);
}

__global__ void finish_sums2_kernel(const double* partials, int nblocks, double* out) {
  const int lane = threadIdx.x & 31, k = threadIdx.x >> 5;
  if (k >= 2) return;
  double x = 0.0;
  for (int b = lane; b < nblocks; b += 32) x += partials[2LL * b + k];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_down_sync(0xffffffffu, x, o);
  if (lane == 0) out[k] = x;
}

// exp(-i phi) in the plane-wave table's element type: F64::Link, or for the
// FP32 kernels c - i s as hi + lo pairs of cos phi and sin phi
__device__ __forceinline__ void plane_link_from(double phi, F64::Link* out) {
  *out = link_from(phi, (F64*)nullptr);
}
__device__ __forceinline__ void plane_link_from(double phi, PlaneLink32* out) {
  double sn, cs;
  sincos(phi, &sn, &cs);
  const float ch = __double2float_rn(cs), sh = __double2float_rn(sn);
  const float cl = __double2float_rn(cs - (double)ch), sl = __double2float_rn(sn - (double)sh);
  out->ch = make_float2(ch, ch);
  out->cl = make_float2(cl, cl);
  out->sh = make_float2(sh, -sh);
  out->sl = make_float2(sl, -sl);
}

template <class P>
__global__ void link_table_kernel(typename PlaneLinkOf<P>::type* tab, int n, const FieldDesc f, int dims,
                                  int axis, int pol, double t_up, double t_lo) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= 2 * n) return;
  const int half = i / n;
  long long HH[3] = {0, 0, 0};
  HH[axis] = i - half * n;
  // the same phase function as the per-link FP64 path
  plane_link_from(link_phase(f, dims, HH, pol, +1, half ? t_lo : t_up), tab + i);
}

// b = 1/(1 + i theta), theta = dt (beta m + V)/2 with V complex, of every site
// of one plane (blockIdx.y), V from the same FP64 potential functions as the
// per-site general path, at time 0 (the table serves time-independent
// potentials only); stored as {re hi, im hi, re lo, im lo}
template <int DIMS>
__global__ void coef_table_kernel(float4* __restrict__ tab, const FieldDesc f, int N0, int N1, int N2,
                                  long long pstride) {
  const int plane = blockIdx.y;
  const long long ncell = (long long)N0 * N1 * N2;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const long long x = c % N0, y = (c / N0) % N1, z = c / ((long long)N0 * N1);
    const long long X = 2 * x + plane_off<DIMS>(plane, 0), Y = 2 * y + plane_off<DIMS>(plane, 1),
                    Z = DIMS == 3 ? 2 * z + plane_off<DIMS>(plane, 2) : 0;
    const double V = potential_at(f, DIMS, X, Y, Z, c, pstride, plane, 0.0);
    const double beta = is_upper<DIMS>(plane) ? 1.0 : -1.0;
    const double ta = f.dt * (beta * f.m + V) * 0.5;  // theta = ta + i tb
    const double tb = f.dt * potential_imag_at(f, DIMS, X, Y, Z) * 0.5;
    // b = 1/((1 - tb) + i ta)
    const double k = 1.0 / ((1.0 - tb) * (1.0 - tb) + ta * ta);
    const double re = (1.0 - tb) * k, im = -ta * k;
    const float rh = __double2float_rn(re), ih = __double2float_rn(im);
    tab[plane * pstride + c] =
        make_float4(rh, ih, __double2float_rn(re - (double)rh), __double2float_rn(im - (double)ih));
  }
}

// COEF_SOFTCORR: the correction records (softcore_corr_index's layout) of a
// real soft-core potential: per value, (exact b) - (the kernels' FP32
// estimate softcore_fast2), b = 1/(1 + i dt (beta m + V)/2) with V from the
// same FP64 potential function as the per-site path, rounded to an integer
// multiple of 2^-35 per component and stored as two 16-bit integers; a value
// out of the 16-bit range sets *overflow (the estimate was off by more than
// the table can hold; the library then evaluates the soft core otherwise)
template <int DIMS>
__global__ void softcore_corr_kernel(unsigned* __restrict__ out, const HalfFields<F32> hu,
                                     const HalfFields<F32> hl, const FieldDesc f, int N0, int N1, int N2,
                                     int* overflow) {
  constexpr int np = nplanes<DIMS>();
  const int N[3] = {N0, N1, N2};
  const long long ncell = (long long)N0 * N1 * N2;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ncell * np;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / np;
    const int plane = (int)(i - r * np);
    const int x = (int)(r % N0), y = (int)((r / N0) % N1), zr = (int)(r / ((long long)N0 * N1));
    int yy = y, zz = zr;
    const bool shifted = DIMS == 3 ? plane < 2 : plane == 0;
    if (shifted) {
      if (DIMS == 3) zz = zr + 1 == N2 ? 0 : zr + 1;
      else yy = y + 1 == N1 ? 0 : y + 1;
    }
    const int H[3] = {2 * x + plane_off<DIMS>(plane, 0), 2 * yy + plane_off<DIMS>(plane, 1),
                      DIMS == 3 ? 2 * zz + plane_off<DIMS>(plane, 2) : 0};
    const bool upper = is_upper<DIMS>(plane);
    const HalfFields<F32>& h = upper ? hu : hl;
    float Rh, Rl;
    softcore_R<DIMS>(h, H, Rh, Rl);
    float2 re, im;
    softcore_fast2(f2(Rh), f2(Rl), f2(softcore_t0(h, H).x), h.sc_K_hi, re, im);
    const double V = potential_at(f, DIMS, H[0], H[1], H[2], 0, 0, plane, 0.0);
    const double th = f.dt * ((upper ? 1.0 : -1.0) * f.m + V) * 0.5;
    const double k = 1.0 / (1.0 + th * th);
    long long q[2] = {llrint((k - (double)re.x) * 34359738368.0), llrint((-th * k - (double)im.x) * 34359738368.0)};
    for (int c = 0; c < 2; ++c) {
      if (q[c] > 32767 || q[c] < -32767) {
        atomicOr(overflow, 1);
        q[c] = q[c] > 0 ? 32767 : -32767;
      }
    }
    out[i] = (unsigned)(q[0] & 0xffff) | ((unsigned)(q[1] & 0xffff) << 16);
  }
}

// q times the link integrals of every value in the state layout: the value's
// own link towards +dx_a/2 (slot 2a) and the link from its neighbour at
// -dx_a/2 to it (slot 2a+1), which that neighbour (partner plane, cell shifted
// with the periodic wrap) carries as its own up link
template <int DIMS>
__global__ void link_integral_table_kernel(double* __restrict__ out, const double* __restrict__ raw, int N0,
                                           int N1, int N2, long long pstride, double q) {
  const int plane = blockIdx.y, axis = blockIdx.z;
  const long long ncell = (long long)N0 * N1 * N2;
  const long long n = (long long)nplanes<DIMS>() * pstride;
  const double* raw_a = raw + (long long)axis * nplanes<DIMS>() * ncell;
  const int pp = partner<DIMS>(plane, axis);
  const int shift = nb_shift<DIMS>(plane, axis, -1);
  const int Nn[3] = {N0, N1, N2};
  const long long stride[3] = {1, N0, (long long)N0 * N1};
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const long long j[3] = {c % N0, (c / N0) % N1, c / ((long long)N0 * N1)};
    long long jm = j[axis] + shift;
    if (jm < 0) jm += Nn[axis];
    const long long cm = c + (jm - j[axis]) * stride[axis];
    out[(2LL * axis) * n + plane * pstride + c] = q * raw_a[(long long)plane * ncell + c];
    out[(2LL * axis + 1) * n + plane * pstride + c] = q * raw_a[(long long)pp * ncell + cm];
  }
}

// LINK_TABLE: the link factors exp(-i phi) of every value of a time-independent
// vector potential, phi from the same FP64 function as the per-site path
// (dir 0: the value's up link; dir 1: the link from its lower neighbour)
template <int DIMS>
__global__ void link_factor_table_kernel(F32::Link* __restrict__ out, const FieldDesc f, int N0, int N1, int N2,
                                         long long pstride) {
  const int plane = blockIdx.y, slot = blockIdx.z, axis = slot >> 1, dir = (slot & 1) ? -1 : 1;
  const long long ncell = (long long)N0 * N1 * N2;
  const long long n = (long long)nplanes<DIMS>() * pstride;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < ncell;
       c += (long long)gridDim.x * blockDim.x) {
    const long long x = c % N0, y = (c / N0) % N1, z = c / ((long long)N0 * N1);
    const long long H[3] = {2 * x + plane_off<DIMS>(plane, 0), 2 * y + plane_off<DIMS>(plane, 1),
                            DIMS == 3 ? 2 * z + plane_off<DIMS>(plane, 2) : 0};
    const double phi = link_phase_site(f, DIMS, H, axis, dir, 0.0, plane, c);
    out[slot * n + plane * pstride + c] = link_from(phi, (F32*)nullptr);
  }
}

__global__ void finish_sums_kernel(const double* partials, int nblocks, double* out) {
  // warp k sums column k: lane-strided, then a fixed shuffle tree
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

// FP64 FMA throughput: eight independent dependency chains of fused
// multiply-adds per thread (the FP64 pipe stays busy, nothing is read from
// memory); the result is stored only if it matches an impossible value, so
// the compiler keeps every operation
__global__ void __launch_bounds__(256) fp64_fma_rate_kernel(double* out, int iters) {
  const double m = 0.9999999999, c = 1e-12;
  double a[8];
#pragma unroll
  for (int j = 0; j < 8; ++j) a[j] = 1e-3 * (threadIdx.x + 1) + j;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int j = 0; j < 8; ++j) a[j] = fma(a[j], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int j = 0; j < 8; ++j) s += a[j];
  if (s == -1.0) out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// measured FP64 FMA rate of the current device in FP64 TFLOP/s (2 flops per
// FMA), or a negative value if a CUDA call failed
double measure_fp64_fma_tflops() {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return -1.0;
  double* sink = nullptr;
  const int blocks = 8 * sms, threads = 256, iters = 4096;
  if (cudaMalloc(&sink, sizeof(double) * blocks * threads) != cudaSuccess) return -1.0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms up
    cudaEventRecord(e0);
    fp64_fma_rate_kernel<<<blocks, threads>>>(sink, iters);
    cudaEventRecord(e1);
    cudaEventSynchronize(e1);
    float ms = 0.0f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && ms < best) best = ms;
  }
  const bool ok = cudaGetLastError() == cudaSuccess;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  if (!ok || best <= 0.0f) return -1.0;
  return 2.0 * 8.0 * iters * (double)blocks * threads / (best * 1e-3) / 1e12;
}

int observables_blocks(const int N[3], int dims) {
  const int gx = (N[0] + 31) / 32, gy = (N[1] + 7) / 8;
  const int nz = dims == 3 ? N[2] : 1;
  long long per_z = (long long)gx * gy;
  long long gz = (152LL * 8 + per_z - 1) / per_z;
  if (gz > nz) gz = nz;
  if (gz < 1) gz = 1;
  return (int)(per_z * gz);
}

template <class P, int DIMS>
void launch_observables(const ObsArgs<P>& a, int blocks, cudaStream_t s) {
  const int gx = (a.N[0] + 31) / 32, gy = (a.N[1] + 7) / 8;
  observables_kernel<P, DIMS><<<dim3(gx, gy, blocks / (gx * gy)), dim3(32, 8), 0, s>>>(a);
}
template void launch_observables<F64, 2>(const ObsArgs<F64>&, int, cudaStream_t);
template void launch_observables<F64, 3>(const ObsArgs<F64>&, int, cudaStream_t);
template void launch_observables<F32, 2>(const ObsArgs<F32>&, int, cudaStream_t);
template void launch_observables<F32, 3>(const ObsArgs<F32>&, int, cudaStream_t);

template <class P>
void launch_link_table(void* tab, int n, const FieldDesc& f, int dims, int axis, int pol, double t_up,
                       double t_lo, cudaStream_t s) {
  link_table_kernel<P><<<(2 * n + 127) / 128, 128, 0, s>>>(static_cast<typename PlaneLinkOf<P>::type*>(tab),
                                                           n, f, dims, axis, pol, t_up, t_lo);
}
template void launch_link_table<F64>(void*, int, const FieldDesc&, int, int, int, double, double, cudaStream_t);
template void launch_link_table<F32>(void*, int, const FieldDesc&, int, int, int, double, double, cudaStream_t);

void launch_coef_table(float4* tab, const FieldDesc& f, int dims, const int N[3], long long pstride,
                       cudaStream_t s) {
  const long long ncell = (long long)N[0] * N[1] * (dims == 3 ? N[2] : 1);
  long long bx = (ncell + 255) / 256;
  if (bx > 152 * 16) bx = 152 * 16;
  const dim3 grid((unsigned)bx, dims == 3 ? 8 : 4);
  if (dims == 3)
    coef_table_kernel<3><<<grid, 256, 0, s>>>(tab, f, N[0], N[1], N[2], pstride);
  else
    coef_table_kernel<2><<<grid, 256, 0, s>>>(tab, f, N[0], N[1], 1, pstride);
}

void launch_softcore_corr(unsigned* out, const HalfFields<F32>& hu, const HalfFields<F32>& hl, const FieldDesc& f,
                          int dims, const int N[3], int* overflow, cudaStream_t s) {
  const long long n = (long long)N[0] * N[1] * (dims == 3 ? N[2] : 1) * (dims == 3 ? 8 : 4);
  long long bx = (n + 255) / 256;
  if (bx > 152 * 32) bx = 152 * 32;
  if (dims == 3)
    softcore_corr_kernel<3><<<(unsigned)bx, 256, 0, s>>>(out, hu, hl, f, N[0], N[1], N[2], overflow);
  else
    softcore_corr_kernel<2><<<(unsigned)bx, 256, 0, s>>>(out, hu, hl, f, N[0], N[1], 1, overflow);
}

void launch_link_integral_table(double* out, const double* raw, int dims, const int N[3], long long pstride,
                                double q, cudaStream_t s) {
  const long long ncell = (long long)N[0] * N[1] * (dims == 3 ? N[2] : 1);
  long long bx = (ncell + 255) / 256;
  if (bx > 152 * 16) bx = 152 * 16;
  const dim3 grid((unsigned)bx, dims == 3 ? 8 : 4, dims);
  if (dims == 3)
    link_integral_table_kernel<3><<<grid, 256, 0, s>>>(out, raw, N[0], N[1], N[2], pstride, q);
  else
    link_integral_table_kernel<2><<<grid, 256, 0, s>>>(out, raw, N[0], N[1], 1, pstride, q);
}

void launch_link_factor_table(F32::Link* out, const FieldDesc& f, int dims, const int N[3], long long pstride,
                              cudaStream_t s) {
  const long long ncell = (long long)N[0] * N[1] * (dims == 3 ? N[2] : 1);
  long long bx = (ncell + 255) / 256;
  if (bx > 152 * 16) bx = 152 * 16;
  const dim3 grid((unsigned)bx, dims == 3 ? 8 : 4, 2 * dims);
  if (dims == 3)
    link_factor_table_kernel<3><<<grid, 256, 0, s>>>(out, f, N[0], N[1], N[2], pstride);
  else
    link_factor_table_kernel<2><<<grid, 256, 0, s>>>(out, f, N[0], N[1], 1, pstride);
}

void launch_finish_sums2(const double* partials, int nblocks, double* out, cudaStream_t s) {
  finish_sums2_kernel<<<1, 64, 0, s>>>(partials, nblocks, out);
}

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
