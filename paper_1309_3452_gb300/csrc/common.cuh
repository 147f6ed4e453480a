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
// COEF_TABLE: a time-independent scalar potential (soft core, static array,
// with V0 and a Klein step) whose coefficient b = 1/(1 + i theta), theta =
// dt (beta m + V)/2, is tabulated per site at creation, in FP64 rounded to a
// hi + lo pair of complex floats (FP32 kernels).  LINK_PLANE: a plane-wave vector potential whose wave vector lies
// along one axis other than its polarisation; its link factors come from a
// per-half-step table indexed by the half-lattice coordinate along that axis.
// LINK_TABLE: any other time-independent vector potential (FP32 kernels): the
// factors exp(-i phi) of every value's up and down link per axis, formed once
// in FP64 from the same phases as the per-site path and kept as hi + lo
// pairs.  GENERAL: per-site FP64.
enum CoefMode { COEF_UNIFORM = 0, COEF_STEP = 1, COEF_GENERAL = 2, COEF_TABLE = 3 };
enum LinkMode { LINK_NONE = 0, LINK_CONST = 1, LINK_GENERAL = 2, LINK_PLANE = 3, LINK_TABLE = 4 };

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

// ------------------------------------------------------------------ double-float
// Unevaluated sums hi + lo of two floats, with error-free transformations:
// TwoSum (Knuth, TAOCP vol. 2), FastTwoSum and TwoProduct via FMA (Dekker
// 1971; Ogita, Rump, Oishi 2005).  About 44 significant bits.
struct DF {
  float hi, lo;
};
__device__ __forceinline__ DF df_fast_two_sum(float a, float b) {  // |a| >= |b|
  const float s = radd(a, b);
  return DF{s, rsub(b, rsub(s, a))};
}
__device__ __forceinline__ DF df_two_sum(float a, float b) {
  const float s = radd(a, b);
  const float bb = rsub(s, a);
  return DF{s, radd(rsub(a, rsub(s, bb)), rsub(b, bb))};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
  const DF s = df_two_sum(a.hi, b.hi);
  return df_fast_two_sum(s.hi, radd(s.lo, radd(a.lo, b.lo)));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
  const float p = rmul(a.hi, b.hi);
  const float e = rfma(a.hi, b.hi, -p);
  return df_fast_two_sum(p, rfma(a.hi, b.lo, rfma(a.lo, b.hi, e)));
}
__device__ __forceinline__ DF df_mulf(DF a, float b) {
  const float p = rmul(a.hi, b);
  const float e = rfma(a.hi, b, -p);
  return df_fast_two_sum(p, rfma(a.lo, b, e));
}
// 1/q for q >= 1: the hardware estimate (rcp.approx, within one ulp) plus one
// Newton step y + y (1 - q y) on the residual formed in double-float
__device__ __forceinline__ DF df_rcp(DF q) {
  float y;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(q.hi));
  const DF qy = df_mulf(q, y);
  const float r = radd(rsub(1.0f, qy.hi), -qy.lo);    // 1 - q y (small)
  return df_fast_two_sum(y, rmul(y, r));
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
  // LINK_PLANE: table of exp(-i phi) for this half-step, indexed by the
  // half-lattice coordinate along ltab_axis; applies on axis lpol only
  const typename P::Link* ltab;
  int ltab_axis, lpol;
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
    const int (&H)[3], long long site, long long pstride, typename P::cplx* S_out = nullptr) {
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
    } else if (LINK == LINK_PLANE) {
      if (ax == h.lpol) {
        const int hk = h.ltab_axis == 0 ? H[0] : (h.ltab_axis == 1 ? H[1] : H[2]);
        const typename P::Link U = h.ltab[hk];
        up = link_mul(U, up);
        dn = link_mulc(U, dn);
      }
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
  if (DIMS == 2) d[2] = d[0];
  const C S = combine<P, DIMS>(d[0], d[1], d[2], sign_class<DIMS>(plane), iso, ry, rz);
  if (S_out) *S_out = S;  // the difference part S' (S = r_x S'), for the conserved functional
  if (coef == COEF_UNIFORM) return apply(h.c_in, F, S);
  if (coef == COEF_STEP) {
    const int hs = h.step_axis == 0 ? H[0] : (h.step_axis == 1 ? H[1] : H[2]);
    return hs >= h.step_X ? apply(h.c_out, F, S) : apply(h.c_in, F, S);
  }
  if (coef == COEF_TABLE) return apply_table(h, F, S, plane, site);
  double V = potential_at(f, DIMS, H[0], H[1], H[2], site, pstride, plane, h.t);
  double th = f.dt * (h.beta * f.m + V) * 0.5;
  double th_im = f.dt * potential_imag_at(f, DIMS, H[0], H[1], H[2]) * 0.5;
  double2 al, ga;
  coef_from_theta(th, th_im, f.rx, al, ga);
  return apply(coef_from(al, ga, (P*)nullptr), F, S);
}

}  // namespace dirac
