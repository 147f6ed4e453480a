// Shared device definitions of libdirac: precision traits, the staggered grid
// geometry and the per-value update of the leap-frog scheme (arXiv:1309.3452).
//
// Device layout: one array per plane (A0,A1,B0,B1,C0,C1,D0,D1 in (3+1)D;
// u0,u1,v0,v1 in (2+1)D), each [z][y][x] with x fastest, complex values
// interleaved (float2 / double2).  Plane k starts at base + k*pstride
// elements; pstride is a multiple of 64 elements.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <climits>

namespace dirac {

// ------------------------------------------------------------------ geometry
// Half-lattice offsets (units of dx/2) of each plane inside its cell: the grid
// definitions of Sect. 2 (A,B,C,D) and Sect. 3 (u,v).
//   plane:    A0      A1      B0      B1      C0      C1      D0      D1
__host__ __device__ constexpr int off3(int plane, int axis) {
  // bit 0 = x, bit 1 = y, bit 2 = z
  return (((plane == 0) ? 0 : (plane == 1) ? 3 : (plane == 2) ? 5 : (plane == 3) ? 6
         : (plane == 4) ? 4 : (plane == 5) ? 7 : (plane == 6) ? 1 : 2) >> axis) & 1;
}
//   plane:    u0      u1      v0      v1
__host__ __device__ constexpr int off2(int plane, int axis) {
  return axis == 2 ? 0 : ((((plane == 0) ? 0 : (plane == 1) ? 3 : (plane == 2) ? 1 : 2) >> axis) & 1);
}
template <int DIMS>
__host__ __device__ constexpr int plane_off(int plane, int axis) {
  return DIMS == 3 ? off3(plane, axis) : off2(plane, axis);
}
template <int DIMS>
__host__ __device__ constexpr int nplanes() { return DIMS == 3 ? 8 : 4; }
// upper planes (A,B / u) come first
template <int DIMS>
__host__ __device__ constexpr bool is_upper(int plane) { return plane < (DIMS == 3 ? 4 : 2); }

// The plane whose offset differs from `plane` only along `axis`: the
// neighbours at +-dx_a/2 of a value on `plane` live there.
template <int DIMS>
__host__ __device__ constexpr int partner(int plane, int axis) {
  // search the plane table for the flipped offset (constexpr-evaluated)
  int want[3] = {plane_off<DIMS>(plane, 0), plane_off<DIMS>(plane, 1), plane_off<DIMS>(plane, 2)};
  want[axis] ^= 1;
  int found = -1;
  for (int q = 0; q < nplanes<DIMS>(); ++q)
    if (plane_off<DIMS>(q, 0) == want[0] && plane_off<DIMS>(q, 1) == want[1] &&
        plane_off<DIMS>(q, 2) == want[2])
      found = q;
  return found;
}
// Cell shift of the neighbour at dir = +1 (x + dx_a/2) or -1 (x - dx_a/2):
// a value at half-lattice 2j+o has its neighbours at 2j+o+-1, i.e. in cell
// j (o=0,+ / o=1,-), j-1 (o=0,-) or j+1 (o=1,+).
template <int DIMS>
__host__ __device__ constexpr int nb_shift(int plane, int axis, int dir) {
  return plane_off<DIMS>(plane, axis) == 0 ? (dir > 0 ? 0 : -1) : (dir > 0 ? 1 : 0);
}
// p = (o_x + o_y) mod 2 selects the sign pattern of the y and z differences:
// p = 0 (A, C, u):  S = r_x dx - i r_y dy + r_z dz
// p = 1 (B, D, v):  S = r_x dx + i r_y dy - r_z dz        (Eqs. ss1-ss4)
template <int DIMS>
__host__ __device__ constexpr int sign_class(int plane) {
  return (plane_off<DIMS>(plane, 0) + plane_off<DIMS>(plane, 1)) & 1;
}

// ------------------------------------------------------------------ precision
struct F64 {
  using real = double;
  using cplx = double2;
  // F+ = alpha F - gamma S'   (alpha = (1-i th)/(1+i th), gamma = r_x/(1+i th))
  struct Coef { double2 a, g; };
  struct Ratio { double v; };      // r_y / r_x, r_z / r_x
  struct Link { double2 u; };      // exp(-i q A_a dx_a/2)
};
struct F32 {
  using real = float;
  using cplx = float2;
  // every coefficient carried as an unevaluated sum hi + lo of two floats so
  // that its rounding does not accumulate coherently over many steps
  struct Coef { float2 a_hi, a_lo, g_hi, g_lo; };
  struct Ratio { float hi, lo; };
  struct Link { float2 hi, lo; };
};
// A plane-wave link factor exp(-i phi) = c - i s of the FP32 kernels' per-step
// table (c = c_hi + c_lo, s = s_hi + s_lo), kept as the packed operand pairs
// of plane_link_diff: ch = (c_hi, c_hi), cl = (c_lo, c_lo), sh = (s_hi, -s_hi),
// sl = (s_lo, -s_lo)
struct PlaneLink32 {
  float2 ch, cl, sh, sl;
};

__device__ __forceinline__ double2 cmk(double a, double b) { return make_double2(a, b); }
__device__ __forceinline__ float2 cmk(float a, float b) { return make_float2(a, b); }

// explicit-rounding primitives (no contraction: every kernel variant that
// uses these helpers produces bit-identical values)
__device__ __forceinline__ double radd(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float radd(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double rsub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float rsub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double rmul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float rmul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double rfma(double a, double b, double c) { return __fma_rn(a, b, c); }
__device__ __forceinline__ float rfma(float a, float b, float c) { return __fmaf_rn(a, b, c); }

// Packed pairs of FP32 (the .f32x2 forms of sm_100 and later): one
// instruction rounds both lanes exactly as two scalar instructions would.
__device__ __forceinline__ unsigned long long pbits(float2 v) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(v.x), "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 punbits(unsigned long long r) {
  float2 v;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(v.x), "=f"(v.y) : "l"(r));
  return v;
}
__device__ __forceinline__ float2 padd(float2 a, float2 b) {
  unsigned long long r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pbits(a)), "l"(pbits(b)));
  return punbits(r);
}
__device__ __forceinline__ float2 psub(float2 a, float2 b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pbits(a)), "l"(pbits(b)));
  return punbits(r);
}
__device__ __forceinline__ float2 pmul(float2 a, float2 b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(pbits(a)), "l"(pbits(b)));
  return punbits(r);
}
__device__ __forceinline__ float2 pfma(float2 a, float2 b, float2 c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(pbits(a)), "l"(pbits(b)), "l"(pbits(c)));
  return punbits(r);
}

template <class C>
__device__ __forceinline__ C csub(C a, C b) { return cmk(rsub(a.x, b.x), rsub(a.y, b.y)); }
template <class C>
__device__ __forceinline__ C cadd(C a, C b) { return cmk(radd(a.x, b.x), radd(a.y, b.y)); }
template <>
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return psub(a, b); }
template <>
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return padd(a, b); }

// ------------------------------------------------------------------ links
__device__ __forceinline__ double2 link_mul(const F64::Link& L, double2 v) {
  return cmk(rfma(L.u.x, v.x, -rmul(L.u.y, v.y)), rfma(L.u.x, v.y, rmul(L.u.y, v.x)));
}
// conj(L) * v
__device__ __forceinline__ double2 link_mulc(const F64::Link& L, double2 v) {
  return cmk(rfma(L.u.x, v.x, rmul(L.u.y, v.y)), rfma(L.u.x, v.y, -rmul(L.u.y, v.x)));
}
__device__ __forceinline__ float2 link_mul(const F32::Link& L, float2 v) {
  float re = rfma(L.lo.x, v.x, -rmul(L.lo.y, v.y));
  float im = rfma(L.lo.x, v.y, rmul(L.lo.y, v.x));
  re = rfma(L.hi.x, v.x, rfma(-L.hi.y, v.y, re));
  im = rfma(L.hi.x, v.y, rfma(L.hi.y, v.x, im));
  return cmk(re, im);
}
__device__ __forceinline__ float2 link_mulc(const F32::Link& L, float2 v) {
  float re = rfma(L.lo.x, v.x, rmul(L.lo.y, v.y));
  float im = rfma(L.lo.x, v.y, -rmul(L.lo.y, v.x));
  re = rfma(L.hi.x, v.x, rfma(L.hi.y, v.y, re));
  im = rfma(L.hi.x, v.y, rfma(-L.hi.y, v.x, im));
  return cmk(re, im);
}

// ------------------------------------------------------------------ update
// Difference part of one update without the factor r_x:
//   S' = d_x + s_y (r_y/r_x) d_y + s_z (r_z/r_x) d_z,
// d_a = (neighbour at +dx_a/2) - (neighbour at -dx_a/2), s_y = -i (p=0) or +i
// (p=1), s_z = +1 (p=0) or -1 (p=1)  (Eqs. ss1-ss4; Eqs. scheme2Deq ff.).
// iso: r_x = r_y = r_z, so the ratios are exactly one.
template <class P, int DIMS>
__device__ __forceinline__ typename P::cplx combine(typename P::cplx dx, typename P::cplx dy,
                                                    typename P::cplx dz, int p, bool iso,
                                                    const typename P::Ratio& ry,
                                                    const typename P::Ratio& rz);

template <>
__device__ __forceinline__ double2 combine<F64, 3>(double2 dx, double2 dy, double2 dz, int p,
                                                   bool iso, const F64::Ratio& ry,
                                                   const F64::Ratio& rz) {
  double2 ty = p ? cmk(-dy.y, dy.x) : cmk(dy.y, -dy.x);
  double2 tz = p ? cmk(-dz.x, -dz.y) : dz;
  if (!iso) {
    ty = cmk(rmul(ry.v, ty.x), rmul(ry.v, ty.y));
    tz = cmk(rmul(rz.v, tz.x), rmul(rz.v, tz.y));
  }
  return cadd(cadd(dx, ty), tz);
}
template <>
__device__ __forceinline__ double2 combine<F64, 2>(double2 dx, double2 dy, double2, int p, bool iso,
                                                   const F64::Ratio& ry, const F64::Ratio&) {
  double2 ty = p ? cmk(-dy.y, dy.x) : cmk(dy.y, -dy.x);
  if (!iso) ty = cmk(rmul(ry.v, ty.x), rmul(ry.v, ty.y));
  return cadd(dx, ty);
}
__device__ __forceinline__ float2 ratio_mul(const F32::Ratio& r, float2 t) {
  return pfma(make_float2(r.hi, r.hi), t, pmul(make_float2(r.lo, r.lo), t));
}
// (dx + s_y dy) + s_z dz; with iso the y term is two scalar adds (the factor
// +-i swaps the lanes) and the z term one packed add
template <>
__device__ __forceinline__ float2 combine<F32, 3>(float2 dx, float2 dy, float2 dz, int p, bool iso,
                                                  const F32::Ratio& ry, const F32::Ratio& rz) {
  if (!iso) {
    float2 ty = p ? cmk(-dy.y, dy.x) : cmk(dy.y, -dy.x);
    float2 tz = p ? cmk(-dz.x, -dz.y) : dz;
    return padd(padd(dx, ratio_mul(ry, ty)), ratio_mul(rz, tz));
  }
  const float2 u = p ? cmk(rsub(dx.x, dy.y), radd(dx.y, dy.x)) : cmk(radd(dx.x, dy.y), rsub(dx.y, dy.x));
  return p ? psub(u, dz) : padd(u, dz);
}
template <>
__device__ __forceinline__ float2 combine<F32, 2>(float2 dx, float2 dy, float2, int p, bool iso,
                                                  const F32::Ratio& ry, const F32::Ratio&) {
  if (!iso) {
    float2 ty = p ? cmk(-dy.y, dy.x) : cmk(dy.y, -dy.x);
    return padd(dx, ratio_mul(ry, ty));
  }
  return p ? cmk(rsub(dx.x, dy.y), radd(dx.y, dy.x)) : cmk(radd(dx.x, dy.y), rsub(dx.y, dy.x));
}

// F+ = alpha F - gamma S'  (the Cayley form of Eqs. ss1-ss4:
//   F+ = ((1 - i th) F - S) / (1 + i th),  th = dt (beta m + V)/2)
__device__ __forceinline__ double2 apply(const F64::Coef& c, double2 F, double2 S) {
  double re = rfma(c.a.x, F.x, rfma(-c.a.y, F.y, rfma(-c.g.x, S.x, rmul(c.g.y, S.y))));
  double im = rfma(c.a.x, F.y, rfma(c.a.y, F.x, rfma(-c.g.x, S.y, -rmul(c.g.y, S.x))));
  return cmk(re, im);
}
__device__ __forceinline__ float2 apply(const F32::Coef& c, float2 F, float2 S) {
  // small (lo) products first, then the hi products on top; lane 0 = re, 1 = im
  const float2 Fs = make_float2(F.y, F.x), Ss = make_float2(S.y, S.x);
  float2 t = pmul(make_float2(c.g_lo.y, -c.g_lo.y), Ss);
  t = pfma(make_float2(-c.g_lo.x, -c.g_lo.x), S, t);
  t = pfma(make_float2(-c.a_lo.y, c.a_lo.y), Fs, t);
  t = pfma(make_float2(c.a_lo.x, c.a_lo.x), F, t);
  t = pfma(make_float2(c.g_hi.y, -c.g_hi.y), Ss, t);
  t = pfma(make_float2(-c.g_hi.x, -c.g_hi.x), S, t);
  t = pfma(make_float2(-c.a_hi.y, c.a_hi.y), Fs, t);
  return pfma(make_float2(c.a_hi.x, c.a_hi.x), F, t);
}

// ------------------------------------------------------------------ fields
// copies of 8 or 16 bytes from global to shared memory that bypass the
// registers (cp.async; completion by cp_async_wait_all of the issuing thread)
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 16;" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// COEF_TABLE: a time-independent scalar potential (soft core, static array,
// with V0 and a Klein step) whose coefficient b = 1/(1 + i theta), theta =
// dt (beta m + V)/2, is tabulated per site at creation, in FP64 rounded to a
// hi + lo pair of complex floats (FP32 kernels).  LINK_PLANE: a plane-wave vector potential whose wave vector lies
// along one axis other than its polarisation; its link factors come from a
// per-half-step table indexed by the half-lattice coordinate along that axis.
// LINK_TABLE: any other time-independent vector potential (FP32 kernels): the
// factors exp(-i phi) of every value's up and down link per axis, formed once
// in FP64 from the same phases as the per-site path and kept as hi + lo
// pairs.  GENERAL: per-site FP64.  COEF_SOFTCORE (FP32 kernels): a soft-core
// potential (with V0 and a Klein step, real) whose b is computed per value
// in compensated FP32 from |x - c|^2 + a^2, itself summed from three small
// per-axis tables of (X dx_a/2 - c_a)^2 (no per-site data).
// COEF_SOFTCORR (FP32 kernels): the same soft core with b formed in plain FP32
// (softcore_fast2) and completed by a per-value correction from a table of
// scaled 16-bit integer pairs (4 bytes per value; see softcore_corr_index).
enum CoefMode { COEF_UNIFORM = 0, COEF_STEP = 1, COEF_GENERAL = 2, COEF_TABLE = 3, COEF_SOFTCORE = 4,
                COEF_SOFTCORR = 5 };
enum LinkMode { LINK_NONE = 0, LINK_CONST = 1, LINK_GENERAL = 2, LINK_PLANE = 3, LINK_TABLE = 4 };
// Kernel-side specialisation of LINK_PLANE in the fused (3+1)D kernel: the
// wave travels along z and is polarised along x; the kernel stages the link
// factors of each z level and passes them in (never a simulation's link_mode)
constexpr int LINK_PLANE_ZX = 5;

// Analytic field description, FP64, for the per-site (general) paths.
struct FieldDesc {
  double dt, m, rx;
  double dx[3];
  double V0;
  int step_axis;       // < 0: no step
  int step_X;          // sites with half-lattice index >= step_X along the axis are beyond it
  double step_V;
  double sc_Z, sc_a2, sc_c[3];
  const double* Vstatic;  // device, one real per site, plane-major like the state (pstride)
  double Vmod_amp, Vmod_omega;
  double q, A_const[3], Apw_amp, Apw_k[3], Apw_omega, Apw_phase;
  int Apw_pol;
  // imaginary part of V: V0_imag - abs_W sum_{a in abs_axes} (1 - d_a/abs_width)^2
  // within abs_width of a face of the box [0, L_a)
  double V0_imag, abs_W, abs_width;
  int abs_axes;
  double L[3];
  // an arbitrary vector potential by its link integrals (Sect. 4): q times
  // the integral of A_a along the up link (dir +1, slot 2a) and the down link
  // (dir -1, slot 2a+1) of every value, at [slot * Alink_n + plane * Alink_ps
  // + site]; scaled at time t by 1 + Alink_amp cos(Alink_omega t); NULL: none
  const double* Alink;
  long long Alink_n, Alink_ps;
  double Alink_amp, Alink_omega;
};

// Compute alpha = (1 - i th)/(1 + i th) and gamma = r_x/(1 + i th) in FP64
// from th = ta + i tb (1 + i th = (1 - tb) + i ta).
__device__ __forceinline__ void coef_from_theta(double ta, double tb, double rx, double2& a, double2& g) {
  const double inv = 1.0 / ((1.0 - tb) * (1.0 - tb) + ta * ta);
  a = make_double2((1.0 - tb * tb - ta * ta) * inv, -2.0 * ta * inv);
  g = make_double2(rx * (1.0 - tb) * inv, -rx * ta * inv);
}

// imaginary part of the scalar potential at half-lattice point H (absorbing
// layers; time-independent), FP64
__device__ __forceinline__ double potential_imag_at(const FieldDesc& f, int dims, long long X, long long Y,
                                                    long long Z) {
  double W = 0.0;
  if (f.abs_W != 0.0) {
    const long long H[3] = {X, Y, Z};
    for (int a = 0; a < dims; ++a) {
      if (!((f.abs_axes >> a) & 1)) continue;
      const double x = (double)H[a] * f.dx[a] * 0.5;
      const double d = fmin(x, f.L[a] - x);
      if (d < f.abs_width) {
        const double u = 1.0 - d / f.abs_width;
        W += u * u;
      }
    }
  }
  return f.V0_imag - f.abs_W * W;
}

// scalar potential at half-lattice point (X,Y,Z) at time t, FP64
__device__ __forceinline__ double potential_at(const FieldDesc& f, int dims, long long X, long long Y,
                                               long long Z, long long site, long long pstride,
                                               int plane, double t) {
  double V = f.V0;
  long long H[3] = {X, Y, Z};
  const long long hs = f.step_axis == 0 ? X : (f.step_axis == 1 ? Y : Z);
  if (f.step_axis >= 0 && hs >= f.step_X) V += f.step_V;
  if (f.sc_Z != 0.0) {
    double r2 = 0.0;
    for (int a = 0; a < dims; ++a) {
      double d = (double)H[a] * f.dx[a] * 0.5 - f.sc_c[a];
      r2 += d * d;
    }
    V -= f.sc_Z / sqrt(r2 + f.sc_a2);
  }
  if (f.Vstatic) V += f.Vstatic[(long long)plane * pstride + site] * (1.0 + f.Vmod_amp * cos(f.Vmod_omega * t));
  return V;
}

// link phase phi = q * (line integral of A_a along the link, Sect. 4) for the
// link of length h = dx_a/2 from half-lattice point H towards dir (+1/-1)
// along axis a, midpoint H + dir/2: A_const h, plus for the plane wave
// amp h cos(k.mid - w t + phase) sin(k_a h/2)/(k_a h/2)
__device__ __forceinline__ double link_phase(const FieldDesc& f, int dims, const long long H[3],
                                             int axis, int dir, double t) {
  const double h = f.dx[axis] * 0.5;
  double I = f.A_const[axis] * h;
  if (f.Apw_amp != 0.0 && f.Apw_pol == axis) {
    double ph = -f.Apw_omega * t + f.Apw_phase;
    for (int b = 0; b < dims; ++b) {
      double y = (double)H[b] * f.dx[b] * 0.5;
      if (b == axis) y += dir * f.dx[b] * 0.25;
      ph += f.Apw_k[b] * y;
    }
    const double u = 0.5 * f.Apw_k[axis] * h;
    I += f.Apw_amp * h * cos(ph) * (u == 0.0 ? 1.0 : sin(u) / u);
  }
  return f.q * I;
}

// the phase of a value's link: the analytic part above plus, if given, the
// tabulated link integral of that value (plane, site)
__device__ __forceinline__ double link_phase_site(const FieldDesc& f, int dims, const long long H[3], int axis,
                                                  int dir, double t, int plane, long long site) {
  double phi = link_phase(f, dims, H, axis, dir, t);
  if (f.Alink) {
    const double mod = 1.0 + f.Alink_amp * cos(f.Alink_omega * t);
    const long long slot = 2 * axis + (dir > 0 ? 0 : 1);
    phi += mod * f.Alink[slot * f.Alink_n + (long long)plane * f.Alink_ps + site];
  }
  return phi;
}

// ------------------------------------------------------------------ compensated pairs
// Unevaluated sums hi + lo of two floats, two independent values at a time
// (lane .x and lane .y of each float2, packed instructions).  The error-free
// transformations are TwoSum (Knuth, TAOCP vol. 2, Sect. 4.2.2) and
// TwoProduct by FMA (Ogita, Rump, Oishi, SIAM J. Sci. Comput. 26, 2005).
__device__ __forceinline__ float2 f2(float v) { return make_float2(v, v); }
__device__ __forceinline__ float2 pneg(float2 a) { return make_float2(-a.x, -a.y); }
// s + e = a + b exactly
__device__ __forceinline__ void two_sum2(float2 a, float2 b, float2& s, float2& e) {
  s = padd(a, b);
  const float2 bb = psub(s, a);
  e = padd(psub(a, psub(s, bb)), psub(b, bb));
}
__device__ __forceinline__ float2 rsqrt2(float2 v) {
  float2 r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(v.x));
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(v.y));
  return r;
}
__device__ __forceinline__ float2 rcp2(float2 v) {
  float2 r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.x) : "f"(v.x));
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r.y) : "f"(v.y));
  return r;
}

// Cayley coefficient b = 1/(1 + i theta) of a soft-core potential, for two
// values at once (lanes), in compensated FP32:
//   theta = th0 + K / sqrt(R),   R = Rh + Rl > 0,  th0 = t0h + t0l,  K = Kh + Kl
// (K = -dt Z/2 for V = -Z/sqrt(|x - c|^2 + a^2), R = |x - c|^2 + a^2, th0 =
// dt (beta m + V0 [+ V_step])/2).  1/sqrt(R) is the hardware estimate refined
// by one Newton step y0 + y0 (1 - R y0^2)/2 whose residual is formed with y0^2
// split exactly (TwoProduct) and 1 - Rh y0^2 in one FMA rounding; theta =
// th0 + K y by TwoSum; 1 + theta^2 split into hi + lo by an FMA; b =
// (1 - i theta)/(1 + theta^2) with the reciprocal refined like the square
// root.  Result: b = (re_hi + re_lo) + i (im_hi + im_lo), relative
// error ~1e-13 for |theta| < 1, so |2b - 1| = 1 to that accuracy.
struct SoftB2 {
  float2 re_hi, re_lo, im_hi, im_lo;
};
__device__ __forceinline__ SoftB2 softcore_b2(float2 Rh, float2 Rl, float2 t0h, float2 t0l, float Kh,
                                              float Kl) {
  // y = 1/sqrt(R) as y0 + yl
  const float2 y0 = rsqrt2(Rh);
  const float2 ph = pmul(y0, y0);
  const float2 pl = pfma(y0, y0, pneg(ph));
  // e = 1 - R y0^2: 1 - Rh ph with one rounding (|e| ~ 2^-22, so its error
  // is ~2^-46), then the small terms
  float2 e = pfma(pneg(Rh), ph, f2(1.0f));
  e = pfma(pneg(Rh), pl, e);
  e = pfma(pneg(Rl), ph, e);                     // e = 1 - R y0^2
  const float2 yl = pmul(pmul(f2(0.5f), y0), e);
  // t = K y
  const float2 th = pmul(f2(Kh), y0);
  float2 tl = pfma(f2(Kh), y0, pneg(th));
  tl = pfma(f2(Kh), yl, tl);
  tl = pfma(f2(Kl), y0, tl);
  // theta = th0 + t
  float2 ah, ae;
  two_sum2(t0h, th, ah, ae);
  const float2 al = padd(ae, padd(t0l, tl));
  // D = 1 + theta^2 as dh + dl: dh = fl(1 + ah^2) >= 1 is a multiple of its
  // own ulp, and so is 1, so 1 - dh is exact; ah^2 + (1 - dh), rounded once,
  // is the rounding error of dh
  const float2 dh = pfma(ah, ah, f2(1.0f));
  float2 dl = pfma(ah, ah, psub(f2(1.0f), dh));
  dl = pfma(padd(ah, ah), al, dl);
  // 1/D as r0 + rl
  const float2 r0 = rcp2(dh);
  float2 g = pfma(pneg(dh), r0, f2(1.0f));
  g = pfma(pneg(dl), r0, g);
  const float2 rl = pmul(r0, g);
  // b = (1 - i theta)/D
  const float2 mh = pmul(ah, r0);
  float2 ml = pfma(ah, r0, pneg(mh));
  ml = pfma(ah, rl, ml);
  ml = pfma(al, r0, ml);
  return SoftB2{r0, rl, pneg(mh), pneg(ml)};
}
// The plain FP32 estimate of the soft-core b = 1/(1 + i theta) of two values
// (lanes): R = Rh + Rl rounded once, theta = K y + th0 with y the hardware
// 1/sqrt(R) estimate, b = (1 - i theta) r with r the hardware estimate of
// 1/(1 + theta^2).  Relative error below ~5e-7; COEF_SOFTCORR adds the
// tabulated difference to the exact b (the table is built with this very
// function, so the two agree bit for bit).
__device__ __forceinline__ void softcore_fast2(float2 Rh, float2 Rl, float2 t0h, float Kh, float2& re,
                                               float2& im) {
  const float2 y = rsqrt2(padd(Rh, Rl));
  const float2 th = pfma(f2(Kh), y, t0h);
  re = rcp2(pfma(th, th, f2(1.0f)));
  im = pmul(pneg(th), re);
}
// scale of the tabulated corrections: exact b - FP32 estimate = q * 2^-35
// per component, q a 16-bit integer (|difference| < 2^-20 ~ 9.5e-7)
constexpr float kCorrScale = 2.9103830456733704e-11f;  // 2^-35
__device__ __forceinline__ float2 corr_decode(unsigned w) {
  return make_float2(rmul((float)(short)(w & 0xffffu), kCorrScale), rmul((float)(short)(w >> 16), kCorrScale));
}

// one value's coefficient {re hi, re lo, im hi, im lo} from a lane of a pair
__device__ __forceinline__ float4 lane_b(const SoftB2& b, int lane) {
  return lane ? make_float4(b.re_hi.y, b.re_lo.y, b.im_hi.y, b.im_lo.y)
              : make_float4(b.re_hi.x, b.re_lo.x, b.im_hi.x, b.im_lo.x);
}

// F+ = b (2F - S) - F with S = r_x S' (Eqs. ss1-ss4 in the Cayley form with
// b = 1/(1 + i theta)); b = {re hi, re lo, im hi, im lo}, r_x = rxh + rxl
__device__ __forceinline__ float2 apply_b(float4 b, float rxh, float rxl, float2 F, float2 S) {
  // w = 2F - r_x S'  (small product first)
  const float2 w = pfma(f2(-rxh), S, pfma(f2(-rxl), S, padd(F, F)));
  // b w = re(b) (wx, wy) + im(b) (-wy, wx), small (lo) products first
  // (the rotated w is formed once; each product has the value of im(b) times
  // the rotated lane, so the result does not depend on where the sign sits)
  const float2 wr = make_float2(-w.y, w.x);
  float2 t = pmul(f2(b.y), w);
  t = pfma(f2(b.w), wr, t);
  t = pfma(f2(b.z), wr, t);
  t = pfma(f2(b.x), w, t);
  return psub(t, F);
}

// ------------------------------------------------------------------ site update
// FP64 -> coefficient / link of the working precision
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

// Field parameters of one half-step, shared by every kernel variant.
template <class P>
struct HalfFields {
  int coef_mode;            // CoefMode
  typename P::Coef c_in;    // uniform coefficient (or: before the Klein step)
  typename P::Coef c_out;   // beyond the Klein step
  int step_axis, step_X;    // Klein step: half-lattice index threshold
  int link_mode;            // LinkMode
  typename P::Link L[3];    // constant link factors exp(-i q A_a dx_a/2)
  double t;                 // field time of this half-step
  double beta;              // +1 upper (A,B,u), -1 lower (C,D,v)
  // COEF_TABLE: b of every site as {re hi, im hi, re lo, im lo}, one array
  // per plane (cell index as in the state), and r_x as hi + lo
  const float4* b_tab[8];
  float rx_hi, rx_lo;
  // LINK_PLANE: table of the link factors exp(-i phi) for this half-step,
  // indexed by the half-lattice coordinate along ltab_axis; applies on axis
  // lpol only (FP64 kernels: F64::Link; FP32 kernels: PlaneLink32)
  const void* ltab;
  int ltab_axis, lpol;
  // COEF_SOFTCORE: theta_0 = dt (beta m + V0)/2 before the Klein step
  // (sc_t0[0]) and beyond it (sc_t0[1]) as (hi, lo); K = -dt Z/2 as hi + lo;
  // per-axis tables sc_sq[a][X] = (X dx_a/2 - c_a)^2 (+ a^2 on axis 0) as
  // (hi, lo) for X in [0, 2 N_a), every hi a multiple of one power of two so
  // that sums of hi parts are exact in FP32
  float2 sc_t0[2];
  int sc_step;              // a Klein step is present (else sc_t0[0] everywhere)
  float sc_K_hi, sc_K_lo;
  const float2* sc_sq[3];
  // COEF_SOFTCORR: the correction records (softcore_corr_index), 32-bit words
  const unsigned* sc_corr;
  // LINK_TABLE: link factors [(2 axis + dir) * larr_n + plane * larr_ps + site],
  // dir 0 = the value's own link upwards, 1 = the link from its lower
  // neighbour (applied conjugated, like the per-site path)
  const typename P::Link* larr;
  long long larr_n, larr_ps;
};

// The tabulated-potential update (F32 only), the paper's form of the Cayley
// step (Eqs. ss1-ss4):  F+ = b (2F - S) - F,  b = 1/(1 + i theta),  S = r_x S'
// which is ((1 - i theta) F - S)/(1 + i theta).  b and r_x are carried as
// hi + lo pairs, so |2b - 1| = 1 holds to ~1e-14 and the rounding of the
// coefficients does not accumulate over steps.
template <class P>
__device__ __forceinline__ typename P::cplx apply_table(const HalfFields<P>& h, typename P::cplx F,
                                                        typename P::cplx S, int plane, long long site);
template <>
__device__ __forceinline__ double2 apply_table<F64>(const HalfFields<F64>&, double2 F, double2, int,
                                                    long long) {
  return F;  // not used: FP64 kernels take the general path
}
template <>
__device__ __forceinline__ float2 apply_table<F32>(const HalfFields<F32>& h, float2 F, float2 S, int plane,
                                                   long long site) {
  const float4 b = __ldg(h.b_tab[plane] + site);
  // w = 2F - r_x S'  (small product first)
  const float2 w = pfma(make_float2(-h.rx_hi, -h.rx_hi), S,
                        pfma(make_float2(-h.rx_lo, -h.rx_lo), S, padd(F, F)));
  // b w, small (lo) products first
  float re = rfma(b.z, w.x, -rmul(b.w, w.y));
  float im = rfma(b.z, w.y, rmul(b.w, w.x));
  re = rfma(b.x, w.x, rfma(-b.y, w.y, re));
  im = rfma(b.x, w.y, rfma(b.y, w.x, im));
  return psub(make_float2(re, im), F);
}

// LINK_PLANE difference along the polarisation, both neighbours sharing the
// link factor L = exp(-i phi) (the wave vector is perpendicular to the link):
//   L up - conj(L) dn = c (up - dn) - i s (up + dn),  L = c - i s
__device__ __forceinline__ double2 plane_link_diff(const F64::Link& L, double2 up, double2 dn) {
  return csub(link_mul(L, up), link_mulc(L, dn));
}
__device__ __forceinline__ float2 plane_link_diff(const PlaneLink32& L, float2 up, float2 dn) {
  const float2 D = psub(up, dn), Q = padd(up, dn);
  const float2 Qs = make_float2(Q.y, Q.x);
  // -i s Q = s (Q.y, -Q.x); small (lo) products first
  float2 t = pmul(L.cl, D);
  t = pfma(L.sl, Qs, t);
  t = pfma(L.sh, Qs, t);
  return pfma(L.ch, D, t);
}
template <class P> struct PlaneLinkOf { using type = F64::Link; };
template <> struct PlaneLinkOf<F32> { using type = PlaneLink32; };

// R = |x - c|^2 + a^2 of the value at half-lattice point H as (hi, lo):
// the hi parts add exactly, the lo parts in FP32 (same order everywhere)
template <int DIMS, class P>
__device__ __forceinline__ void softcore_R(const HalfFields<P>& h, const int (&H)[3], float& Rh, float& Rl) {
  float2 r = padd(__ldg(h.sc_sq[0] + H[0]), __ldg(h.sc_sq[1] + H[1]));
  if (DIMS == 3) r = padd(r, __ldg(h.sc_sq[2] + H[2]));
  Rh = r.x;
  Rl = r.y;
}
// theta_0 of the value: beyond the Klein step (if any) or before it
template <class P>
__device__ __forceinline__ float2 softcore_t0(const HalfFields<P>& h, const int (&H)[3]) {
  if (!h.sc_step) return h.sc_t0[0];
  const int hs = h.step_axis == 0 ? H[0] : (h.step_axis == 1 ? H[1] : H[2]);
  return hs >= h.step_X ? h.sc_t0[1] : h.sc_t0[0];
}

// COEF_SOFTCORR correction records: one record of nplanes 32-bit words per
// cell, in the order a z-level (y-row in (2+1)D) iteration of the fused
// kernels uses them: record r holds the upper values of level r+1 planes
// A0, A1 (u0) and the values of level r of every other plane.  So the value
// of plane p in cell (x, y, z) has its word at
//   ((z' Ny + y') Nx + x) * nplanes + p,  with z' = z - 1 (wrapped) for A0, A1
// ((2+1)D: y' = y - 1 for u0) and z' = z (y' = y) otherwise.
template <int DIMS>
__device__ __forceinline__ long long softcore_corr_index(int plane, const int (&H)[3], const int (&N)[3]) {
  const int x = H[0] >> 1, y = H[1] >> 1, z = H[2] >> 1;
  const bool shifted = DIMS == 3 ? plane < 2 : plane == 0;
  if (DIMS == 3) {
    const int zr = shifted ? (z == 0 ? N[2] - 1 : z - 1) : z;
    return (((long long)zr * N[1] + y) * N[0] + x) * 8 + plane;
  }
  const int yr = shifted ? (y == 0 ? N[1] - 1 : y - 1) : y;
  return ((long long)yr * N[0] + x) * 4 + plane;
}

// COEF_SOFTCORE update (FP32 only): b of this value from the caller's pair
// computation (bpre) or computed here (both lanes the same value, so the
// result is bit-identical to the value's lane of a pair)
template <int DIMS, class P>
__device__ __forceinline__ typename P::cplx apply_softcore(const HalfFields<P>& h, typename P::cplx F,
                                                           typename P::cplx S, const int (&H)[3],
                                                           const float4* bpre);
template <>
__device__ __forceinline__ double2 apply_softcore<2, F64>(const HalfFields<F64>&, double2 F, double2,
                                                          const int (&)[3], const float4*) {
  return F;  // not used: FP64 kernels take the general path
}
template <>
__device__ __forceinline__ double2 apply_softcore<3, F64>(const HalfFields<F64>&, double2 F, double2,
                                                          const int (&)[3], const float4*) {
  return F;
}
template <int DIMS>
__device__ __forceinline__ float2 apply_softcore_f32(const HalfFields<F32>& h, float2 F, float2 S,
                                                     const int (&H)[3], const float4* bpre) {
  float4 b;
  if (bpre) {
    b = *bpre;
  } else {
    float Rh, Rl;
    softcore_R<DIMS>(h, H, Rh, Rl);
    const float2 t0 = softcore_t0(h, H);
    b = lane_b(softcore_b2(f2(Rh), f2(Rl), f2(t0.x), f2(t0.y), h.sc_K_hi, h.sc_K_lo), 0);
  }
  return apply_b(b, h.rx_hi, h.rx_lo, F, S);
}
// COEF_SOFTCORR: the FP32 estimate of this value plus its tabulated correction
// (or the caller's pair computation, bpre)
template <int DIMS>
__device__ __forceinline__ float2 apply_softcorr_f32(const HalfFields<F32>& h, float2 F, float2 S,
                                                     const int (&H)[3], const float4* bpre, int plane,
                                                     const int (&N)[3]) {
  float4 b;
  if (bpre) {
    b = *bpre;
  } else {
    float Rh, Rl;
    softcore_R<DIMS>(h, H, Rh, Rl);
    float2 re, im;
    softcore_fast2(f2(Rh), f2(Rl), f2(softcore_t0(h, H).x), h.sc_K_hi, re, im);
    const float2 c = corr_decode(__ldg(h.sc_corr + softcore_corr_index<DIMS>(plane, H, N)));
    b = make_float4(re.x, c.x, im.x, c.y);
  }
  return apply_b(b, h.rx_hi, h.rx_lo, F, S);
}
template <>
__device__ __forceinline__ float2 apply_softcore<2, F32>(const HalfFields<F32>& h, float2 F, float2 S,
                                                         const int (&H)[3], const float4* bpre) {
  return apply_softcore_f32<2>(h, F, S, H, bpre);
}
template <>
__device__ __forceinline__ float2 apply_softcore<3, F32>(const HalfFields<F32>& h, float2 F, float2 S,
                                                         const int (&H)[3], const float4* bpre) {
  return apply_softcore_f32<3>(h, F, S, H, bpre);
}

// Field-path selectors for site_update: a fixed CoefMode / LinkMode compiles
// only that path; kAnyMode reads h.coef_mode / h.link_mode at run time and
// includes the per-site FP64 (general) paths.
constexpr int kAnyMode = -1;

// One value of the scheme (Eqs. ss1-ss4 / scheme2Deq ff.):
//   F+ = ((1 - i th) F - S) / (1 + i th)  as  alpha F - gamma S'.
// nb = neighbours {x+, x-, y+, y-, z+, z-} (z ignored in (2+1)D) at
// +-dx_a/2; H = half-lattice coordinates of the value; site = cell index
// inside its plane (for a static potential).  Every kernel computes every
// value through this function, so all kernel variants agree bit for bit.
template <class P, int DIMS, int COEF, int LINK>
__device__ __forceinline__ typename P::cplx site_update(
    const HalfFields<P>& h, const FieldDesc& f, bool iso, const typename P::Ratio& ry,
    const typename P::Ratio& rz, int plane, typename P::cplx F, typename P::cplx (&nb)[6],
    const int (&H)[3], long long site, long long pstride, typename P::cplx* S_out = nullptr,
    const float4* bpre = nullptr, const typename PlaneLinkOf<P>::type* lk = nullptr,
    const int* Ngrid_p = nullptr) {
  // grid extent (cells per axis) for the soft-core correction index
  const int Ngrid[3] = {Ngrid_p ? Ngrid_p[0] : 1, Ngrid_p ? Ngrid_p[1] : 1, Ngrid_p ? Ngrid_p[2] : 1};
  using C = typename P::cplx;
  const int link = LINK == kAnyMode ? h.link_mode : LINK;
  const int coef = COEF == kAnyMode ? h.coef_mode : COEF;
  C d[3];
#pragma unroll
  for (int ax = 0; ax < DIMS; ++ax) {
    C up = nb[2 * ax], dn = nb[2 * ax + 1];
    if (link == LINK_CONST) {
      up = link_mul(h.L[ax], up);
      dn = link_mulc(h.L[ax], dn);
    } else if (link == LINK_TABLE) {
      const long long i = (long long)plane * h.larr_ps + site;
      up = link_mul(h.larr[(2 * ax) * h.larr_n + i], up);
      dn = link_mulc(h.larr[(2 * ax + 1) * h.larr_n + i], dn);
    } else if (LINK == kAnyMode && (link == LINK_GENERAL || link == LINK_PLANE)) {
      long long HH[3] = {H[0], H[1], H[2]};
      up = link_mul(link_from(link_phase_site(f, DIMS, HH, ax, +1, h.t, plane, site), (P*)nullptr), up);
      // exp(+i phi-) = conj(exp(-i phi-))
      dn = link_mulc(link_from(link_phase_site(f, DIMS, HH, ax, -1, h.t, plane, site), (P*)nullptr), dn);
    }
    d[ax] = csub(up, dn);
  }
  if constexpr (LINK == LINK_PLANE_ZX) {
    d[0] = plane_link_diff(*lk, nb[0], nb[1]);  // the factor of the value's z level, staged by the caller
  }
  if constexpr (LINK == LINK_PLANE) {
    // the difference along the polarisation with the shared link factor of the
    // value's neighbours: staged by the caller (lk), or from the step's table
    using PL = typename PlaneLinkOf<P>::type;
    PL L;
    if (lk) {
      L = *lk;
    } else {
      const int hk = h.ltab_axis == 0 ? H[0] : (h.ltab_axis == 1 ? H[1] : H[2]);
      L = static_cast<const PL*>(h.ltab)[hk];
    }
    if (h.lpol == 0) d[0] = plane_link_diff(L, nb[0], nb[1]);
    else if (h.lpol == 1) d[1] = plane_link_diff(L, nb[2], nb[3]);
    else if (DIMS == 3) d[2] = plane_link_diff(L, nb[4], nb[5]);
  }
  if (DIMS == 2) d[2] = d[0];
  const C S = combine<P, DIMS>(d[0], d[1], d[2], sign_class<DIMS>(plane), iso, ry, rz);
  if (S_out) *S_out = S;  // the difference part S' (S = r_x S'), for the conserved functional
  if (coef == COEF_UNIFORM) return apply(h.c_in, F, S);
  if (coef == COEF_STEP) {
    const int hs = h.step_axis == 0 ? H[0] : (h.step_axis == 1 ? H[1] : H[2]);
    return hs >= h.step_X ? apply(h.c_out, F, S) : apply(h.c_in, F, S);
  }
  if (coef == COEF_TABLE) return apply_table(h, F, S, plane, site);
  if (coef == COEF_SOFTCORE) return apply_softcore<DIMS>(h, F, S, H, bpre);
  if (coef == COEF_SOFTCORR) {
    if constexpr (sizeof(typename P::real) == 4) return apply_softcorr_f32<DIMS>(h, F, S, H, bpre, plane, Ngrid);
    else return F;  // not used: FP64 kernels take the general path
  }
  double V = potential_at(f, DIMS, H[0], H[1], H[2], site, pstride, plane, h.t);
  double th = f.dt * (h.beta * f.m + V) * 0.5;
  double th_im = f.dt * potential_imag_at(f, DIMS, H[0], H[1], H[2]) * 0.5;
  double2 al, ga;
  coef_from_theta(th, th_im, f.rx, al, ga);
  return apply(coef_from(al, ga, (P*)nullptr), F, S);
}

}  // namespace dirac
