// dirac_norm_noalloc: the conserved functional of a state that lives in the
// caller's device memory, computed without allocating anything.
//
// Who needs this: callers that cannot call cudaMalloc at the point where they
// want the norm, e.g. a host framework that owns all device memory through
// its own pool and forbids other allocations, or a time-critical loop where
// the implicit device-wide synchronisation of cudaMalloc/cudaFree is not
// acceptable.  dirac_create allocates, so those callers cannot hold a
// dirac_sim there; this entry point takes the planes directly.
//
// The per-block partial sums of the reduction go to a file-scope device array
// of fixed size instead of a buffer owned by a simulation.  Every GPU that
// loads the library holds that array until the process exits.
#include <cmath>
#include <cstring>

#include "../../include/dirac.h"
#include "kernels.cuh"

using namespace dirac;

namespace {

// capacity: partial sums of this many reduction blocks, plus the final sums
constexpr int kNoAllocMaxBlocks = 8192;
static __device__ __align__(256) double g_noalloc_scratch[(kNoAllocMaxBlocks + 1) * kObsSums];


// E = naive + sum_a r_a B_a, written to the caller's output
__global__ void combine_kernel(const double* sums, double r0, double r1, double r2, int dims,
                               double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double e = sums[0] + r0 * sums[1] + r1 * sums[2];
    if (dims == 3) e += r2 * sums[3];
    out[0] = e;
    out[1] = sums[0];
  }
}

FieldDesc noalloc_field_desc(int dims, const double dx[3], double dt, const dirac_fields& f) {
  FieldDesc d;
  std::memset(&d, 0, sizeof(d));
  d.dt = dt;
  d.rx = dt / dx[0];
  for (int a = 0; a < 3; ++a) d.dx[a] = a < dims ? dx[a] : 1.0;
  d.q = f.q;
  for (int a = 0; a < 3; ++a) {
    d.A_const[a] = f.A_const[a];
    d.Apw_k[a] = f.Apw_k[a];
  }
  d.Apw_amp = f.Apw_amp;
  d.Apw_omega = f.Apw_omega;
  d.Apw_phase = f.Apw_phase;
  d.Apw_pol = f.Apw_pol;
  return d;
}

template <class P> typename P::Link noalloc_link(double phi);
template <> F64::Link noalloc_link<F64>(double phi) {
  return F64::Link{make_double2(std::cos(phi), -std::sin(phi))};
}
template <> F32::Link noalloc_link<F32>(double phi) {
  F32::Link L;
  double c = std::cos(phi), s = -std::sin(phi);
  L.hi = make_float2((float)c, (float)s);
  L.lo = make_float2((float)(c - (double)L.hi.x), (float)(s - (double)L.hi.y));
  return L;
}

template <class P>
void launch(int dims, const int N[3], const double dx[3], double dt, double t,
            const dirac_fields& f, const void* const* planes, double* scratch, int blocks,
            cudaStream_t s) {
  ObsArgs<P> a;
  std::memset(&a, 0, sizeof(a));
  const int np = dims == 3 ? 8 : 4;
  for (int k = 0; k < np; ++k) a.pl[k] = static_cast<const typename P::cplx*>(planes[k]);
  for (int k = 0; k < 3; ++k) a.N[k] = k < dims ? N[k] : 1;
  a.pstride = 0;
  bool any_A = f.A_const[0] != 0.0 || f.A_const[1] != 0.0 || f.A_const[2] != 0.0;
  a.link_mode = f.Apw_amp != 0.0 ? LINK_GENERAL : (any_A ? LINK_CONST : LINK_NONE);
  for (int k = 0; k < 3; ++k)
    a.L[k] = noalloc_link<P>(f.q * f.A_const[k] * (k < dims ? dx[k] : 1.0) / 2.0);
  a.f = noalloc_field_desc(dims, dx, dt, f);
  a.t_links = t - dt / 2.0;
  a.dens_axis = -1;
  a.partials = scratch;
  a.zlo = 0;
  a.nzu = a.Nzg = dims == 3 ? a.N[2] : a.N[1];  // every level of the marching axis
  a.zorg = 0;
  if (dims == 3) launch_observables<P, 3>(a, blocks, s);
  else launch_observables<P, 2>(a, blocks, s);
}

}  // namespace

extern "C" dirac_status dirac_norm_noalloc(int dims, const int N[3], const double dx[3], double dt,
                                           double t, const dirac_fields* fields,
                                           dirac_precision precision, const void* const* planes,
                                           double* out_dev, void* cuda_stream) {
  if ((dims != 2 && dims != 3) || !N || !dx || !planes || !out_dev) return DIRAC_ERR_INVALID;
  if (precision != DIRAC_FP32 && precision != DIRAC_FP64) return DIRAC_ERR_INVALID;
  for (int a = 0; a < dims; ++a)
    if (N[a] < 2 || !(dx[a] > 0.0)) return DIRAC_ERR_INVALID;
  if (!(dt > 0.0) || !std::isfinite(t)) return DIRAC_ERR_INVALID;
  for (int k = 0; k < (dims == 3 ? 8 : 4); ++k)
    if (!planes[k]) return DIRAC_ERR_INVALID;
  if ((long long)N[0] * N[1] >= (1LL << 31)) return DIRAC_ERR_UNSUPPORTED;
  // link integrals would need a device copy of A_links (an allocation)
  if (fields && fields->A_links) return DIRAC_ERR_UNSUPPORTED;
  dirac_fields f;
  if (fields) f = *fields; else dirac_fields_default(&f);
  // the parameters the functional reads: the vector potential's (as dirac_create checks them)
  const double vals[] = {f.q, f.A_const[0], f.A_const[1], f.A_const[2], f.Apw_amp, f.Apw_k[0],
                         f.Apw_k[1], f.Apw_k[2], f.Apw_omega, f.Apw_phase};
  for (double v : vals)
    if (!std::isfinite(v)) return DIRAC_ERR_INVALID;
  if (f.Apw_amp != 0.0 && (f.Apw_pol < 0 || f.Apw_pol >= dims)) return DIRAC_ERR_INVALID;
  // the reduction grid of this size must fit the fixed scratch array
  const int blocks = observables_blocks(N, dims);
  if (blocks > kNoAllocMaxBlocks) return DIRAC_ERR_UNSUPPORTED;

  // The host-side name of the array is not a device address: ask the runtime
  // for the address of the current device's copy.  This allocates nothing
  // and is done on every call, so a reset device or another context on the
  // same ordinal never sees an address from before.
  double* scratch = nullptr;
  {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return DIRAC_ERR_CUDA;
    scratch = static_cast<double*>(p);
  }
  cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
  // every reduction block overwrites its own partial slot and the final sums
  // are overwritten too, so nothing in the scratch needs clearing
  if (precision == DIRAC_FP64)
    launch<F64>(dims, N, dx, dt, t, f, planes, scratch, blocks, s);
  else
    launch<F32>(dims, N, dx, dt, t, f, planes, scratch, blocks, s);
  double* sums = scratch + (long long)kNoAllocMaxBlocks * kObsSums;
  launch_finish_sums(scratch, blocks, sums, s);
  combine_kernel<<<1, 32, 0, s>>>(sums, dt / dx[0], dt / dx[1], dims == 3 ? dt / dx[2] : 0.0, dims,
                                  out_dev);
  return cudaGetLastError() == cudaSuccess ? DIRAC_OK : DIRAC_ERR_CUDA;
}
