// Host side of libdirac: the C ABI declared in include/dirac.h.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>
#include <string>

#include "../../include/dirac.h"
#include "kernels.cuh"

using namespace dirac;

struct dirac_sim {
  int dims = 0;
  int N[3] = {1, 1, 1};
  double dx[3] = {1, 1, 1};
  double dt = 0, m = 0;
  dirac_precision prec = DIRAC_FP64;
  unsigned flags = 0;
  dirac_fields f{};
  cudaStream_t stream = nullptr;
  long long ncell = 0, pstride = 0;
  // levels along the marching axis ((3+1)D): updated range, global origin and
  // extent (a whole grid: 0, N[2], 0, N[2]; see FusedArgs)
  int zlo = 0, nzu = 1, zorg = 0, Nzg = 1;
  int Nf[3] = {1, 1, 1};      // extent of the grid the fields live on (a slab's whole grid; else N)
  int np = 0;
  size_t elem = 0;            // bytes per complex value
  void* state = nullptr;      // np * pstride values: the current state
  void* state_alt = nullptr;  // second buffer for the out-of-place fused kernels
  int fused = 0;              // one kernel per time step (FP32 without the reference flag)
  int tblock = 1;             // (2+1)D fused path: two time steps per pass when possible
  int chunk1 = 0, chunk2 = 0; // launch plan: levels per item (one-step / two-step kernel), 0 = rule
  double plan_us = 0;         // time per step the autotuner measured for the plan
  double2* staging = nullptr; // one canonical plane (FP32 conversions)
  double* Vstatic = nullptr;  // one real per site (plane-major, pstride)
  float4* b_tab = nullptr;    // COEF_TABLE: b = 1/(1 + i theta) per site as hi + lo (plane-major, pstride)
  float2* sc_sq = nullptr;    // COEF_SOFTCORE/CORR: (X dx_a/2 - c_a)^2 per axis and half-lattice index, hi + lo
  unsigned* sc_corr = nullptr; // COEF_SOFTCORR: one 32-bit correction word per value
  double* Alink = nullptr;    // link integrals x q: 2 dims slots (up, down link per axis) of np * pstride
  F32::Link* larr = nullptr;  // LINK_TABLE: link factors, same slots, FP32 hi + lo
  double* partials = nullptr;
  double* sums_dev = nullptr;
  double* sums_host = nullptr; // pinned
  double* ref_sums = nullptr;  // device: observables sums of the state set last (dirac_check)
  int ref_valid = 0;
  int red_blocks = 0;
  double t0 = 0;              // time set by dirac_set_time (or 0)
  long long k = 0;            // steps taken since then: t = t0 + k dt
  int iso = 1;
  int coef_mode = COEF_UNIFORM, link_mode = LINK_NONE;
  int step_X = 0;
  void* ltab = nullptr;       // LINK_PLANE: link-factor table of the current step
  int ltab_axis = 0, ltab_n = 0;
  long long launches = 0;     // kernels launched so far
  // CUDA graphs of kGraphSteps time steps, one per current-buffer parity
  // (only for fields without time dependence: the launches bake their time)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  void* graph_state[2] = {nullptr, nullptr};
  int graph_disabled = 0;
  int stepped = 0;            // a plain step has run (kernel one-time set-up done)
  // conserved functional accumulated by the last fused launch of a dirac_step
  double* e_partials = nullptr;  // [kFusedEMaxBlocks][2]
  double* e_sums = nullptr;      // [2]: sum |psi|^2, Re sum_lower conj(G) S'_G
  long long e_valid_at = -1;     // value of k for which e_sums describe the state
  std::string err;
};

static const long kGraphSteps = 64;

static thread_local std::string g_create_error;  // per host thread: concurrent creations do not mix messages

static dirac_status fail(dirac_sim* s, dirac_status st, const std::string& msg) {
  if (s) s->err = msg; else g_create_error = msg;
  return st;
}
static dirac_status cuda_fail(dirac_sim* s, cudaError_t e, const char* what) {
  // a failed call also leaves its (non-sticky) error as the runtime's last
  // error: clear it, so that later calls of this or another simulation do not
  // report it again
  cudaGetLastError();
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  return fail(s, e == cudaErrorMemoryAllocation ? DIRAC_ERR_OOM : DIRAC_ERR_CUDA, m);
}
#define CK(sim, call)                                          \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return cuda_fail((sim), e_, #call); \
  } while (0)

static long long round_up(long long v, long long m) { return (v + m - 1) / m * m; }

static long long cells_of(int dims, const int N[3]) {
  return (long long)N[0] * N[1] * (dims == 3 ? N[2] : 1);
}

extern "C" size_t dirac_state_bytes(int dims, const int N[3], dirac_precision p) {
  if ((dims != 2 && dims != 3) || !N) return 0;
  long long nc = cells_of(dims, N);
  long long ps = round_up(nc, 64);
  size_t elem = p == DIRAC_FP32 ? sizeof(float2) : sizeof(double2);
  size_t bytes = (size_t)(dims == 3 ? 8 : 4) * ps * elem;
  // FP32: a second state buffer (out-of-place fused step) and a conversion staging plane
  if (p == DIRAC_FP32) bytes = 2 * bytes + (size_t)ps * sizeof(double2);
  return bytes;
}

extern "C" void dirac_fields_default(dirac_fields* f) {
  if (!f) return;
  std::memset(f, 0, sizeof(*f));
  f->q = 1.0;
  f->step_axis = -1;
  f->sc_a = 1.0;
}

extern "C" int dirac_version(void) { return DIRAC_ABI_VERSION; }

extern "C" const char* dirac_last_error(const dirac_sim* s) {
  return s ? s->err.c_str() : g_create_error.c_str();
}

// smallest half-lattice index H >= 0 with (double)H * dx / 2 > x0, for a
// finite x0 and dx > 0; INT_MAX when no index below 2^31 - 2 qualifies (the
// threshold then selects no site).  Every half-lattice index is >= 0, so a
// threshold below 0 is the same as 0.  At most a few loop iterations.
static int threshold_index(double x0, double dx) {
  const double u = 2.0 * x0 / dx;
  if (!(u < 2147483640.0)) return INT_MAX;
  if (u < 0.0) return 0;
  long long H = (long long)std::floor(u) - 4;
  if (H < 0) H = 0;
  while (!((double)H * dx / 2.0 > x0)) ++H;
  return (int)H;
}

// the name of the first real parameter of dirac_fields that is a NaN or an
// infinity (the field arithmetic would be undefined), or NULL
static const char* nonfinite_field(const dirac_fields& f) {
  const std::pair<double, const char*> v[] = {
      {f.V0, "V0"}, {f.step_x0, "step_x0"}, {f.step_V, "step_V"}, {f.sc_Z, "sc_Z"}, {f.sc_a, "sc_a"},
      {f.sc_center[0], "sc_center"}, {f.sc_center[1], "sc_center"}, {f.sc_center[2], "sc_center"},
      {f.Vmod_amp, "Vmod_amp"}, {f.Vmod_omega, "Vmod_omega"}, {f.q, "q"}, {f.A_const[0], "A_const"},
      {f.A_const[1], "A_const"}, {f.A_const[2], "A_const"}, {f.Apw_amp, "Apw_amp"}, {f.Apw_k[0], "Apw_k"},
      {f.Apw_k[1], "Apw_k"}, {f.Apw_k[2], "Apw_k"}, {f.Apw_omega, "Apw_omega"}, {f.Apw_phase, "Apw_phase"},
      {f.V0_imag, "V0_imag"}, {f.abs_W, "abs_W"}, {f.abs_width, "abs_width"}, {f.Alink_amp, "Alink_amp"},
      {f.Alink_omega, "Alink_omega"}};
  for (const auto& x : v)
    if (!std::isfinite(x.first)) return x.second;
  return nullptr;
}

template <class P> static typename P::Coef make_coef(double th_re, double th_im, double rx);
// alpha = (1 - i th)/(1 + i th), gamma = r_x/(1 + i th) for th = a + i b:
// 1 + i th = (1 - b) + i a, so with D = (1 - b)^2 + a^2
//   alpha = ((1 - b^2 - a^2) - 2 i a)/D,  gamma = r_x ((1 - b) - i a)/D
template <> F64::Coef make_coef<F64>(double a, double b, double rx) {
  const double inv = 1.0 / ((1.0 - b) * (1.0 - b) + a * a);
  F64::Coef c;
  c.a = make_double2((1.0 - b * b - a * a) * inv, -2.0 * a * inv);
  c.g = make_double2(rx * (1.0 - b) * inv, -rx * a * inv);
  return c;
}
static void split(double v, float& hi, float& lo) {
  hi = (float)v;
  lo = (float)(v - (double)hi);
}
template <> F32::Coef make_coef<F32>(double a, double b, double rx) {
  F64::Coef d = make_coef<F64>(a, b, rx);
  F32::Coef c;
  split(d.a.x, c.a_hi.x, c.a_lo.x);
  split(d.a.y, c.a_hi.y, c.a_lo.y);
  split(d.g.x, c.g_hi.x, c.g_lo.x);
  split(d.g.y, c.g_hi.y, c.g_lo.y);
  return c;
}
template <class P> static typename P::Ratio make_ratio(double v);
template <> F64::Ratio make_ratio<F64>(double v) { return F64::Ratio{v}; }
template <> F32::Ratio make_ratio<F32>(double v) {
  F32::Ratio r;
  split(v, r.hi, r.lo);
  return r;
}
template <class P> static typename P::Link make_link(double phi);
template <> F64::Link make_link<F64>(double phi) {
  return F64::Link{make_double2(std::cos(phi), -std::sin(phi))};
}
template <> F32::Link make_link<F32>(double phi) {
  F32::Link L;
  split(std::cos(phi), L.hi.x, L.lo.x);
  split(-std::sin(phi), L.hi.y, L.lo.y);
  return L;
}

// COEF_SOFTCORE tables: for every axis a and half-lattice index X in
// [0, 2 N_a), (X dx_a/2 - c_a)^2 (plus a^2 on axis 0) in FP64, stored as a
// float hi part rounded to a multiple of q and the float lo rest.  q is the
// power of two 2^(e - 22), 2^e >= the largest possible R = a^2 + sum_a max
// (..)^2, so every hi part is below 2^22 q and any sum of three of them is
// exact in FP32; only the lo parts (|lo| <= q/2) round.  Axes beyond dims
// get one zero entry per index.
static void softcore_tables(const dirac_sim* s, std::vector<float2>& out) {
  double rmax = s->f.sc_a * s->f.sc_a;
  for (int a = 0; a < s->dims; ++a) {
    double m = 0.0;
    for (long long X = 0; X < 2LL * s->Nf[a]; ++X) {
      const double d = (double)X * s->dx[a] * 0.5 - s->f.sc_center[a];
      m = std::max(m, d * d);
    }
    rmax += m;
  }
  const double q = std::ldexp(1.0, std::ilogb(rmax) + 1 - 22);
  out.clear();
  for (int a = 0; a < 3; ++a) {
    for (long long X = 0; X < 2LL * s->Nf[a]; ++X) {
      double v = 0.0;
      if (a < s->dims) {
        const double d = (double)X * s->dx[a] * 0.5 - s->f.sc_center[a];
        v = d * d + (a == 0 ? s->f.sc_a * s->f.sc_a : 0.0);
      }
      const double hi = std::nearbyint(v / q) * q;
      out.push_back(make_float2((float)hi, (float)(v - hi)));
    }
  }
}

static FieldDesc field_desc(const dirac_sim* s) {
  FieldDesc d;
  std::memset(&d, 0, sizeof(d));
  d.dt = s->dt;
  d.m = s->m;
  d.rx = s->dt / s->dx[0];
  for (int a = 0; a < 3; ++a) d.dx[a] = s->dx[a];
  d.V0 = s->f.V0;
  d.step_axis = s->f.step_axis;
  d.step_X = s->step_X;
  d.step_V = s->f.step_V;
  d.sc_Z = s->f.sc_Z;
  d.sc_a2 = s->f.sc_a * s->f.sc_a;
  for (int a = 0; a < 3; ++a) d.sc_c[a] = s->f.sc_center[a];
  d.Vstatic = s->Vstatic;
  d.Vmod_amp = s->f.Vmod_amp;
  d.Vmod_omega = s->f.Vmod_omega;
  d.q = s->f.q;
  for (int a = 0; a < 3; ++a) {
    d.A_const[a] = s->f.A_const[a];
    d.Apw_k[a] = s->f.Apw_k[a];
  }
  d.Apw_amp = s->f.Apw_amp;
  d.Apw_omega = s->f.Apw_omega;
  d.Apw_phase = s->f.Apw_phase;
  d.Apw_pol = s->f.Apw_pol;
  d.V0_imag = s->f.V0_imag;
  d.abs_W = s->f.abs_W;
  d.abs_width = s->f.abs_width;
  d.abs_axes = s->f.abs_axes;
  for (int a = 0; a < 3; ++a) d.L[a] = s->Nf[a] * s->dx[a];
  d.Alink = s->Alink;
  d.Alink_n = (long long)s->np * s->pstride;
  d.Alink_ps = s->pstride;
  d.Alink_amp = s->f.Alink_amp;
  d.Alink_omega = s->f.Alink_omega;
  return d;
}

template <class P>
static void plane_ptrs(dirac_sim* s, typename P::cplx* (&pl)[8]) {
  auto* base = static_cast<typename P::cplx*>(s->state);
  for (int k = 0; k < 8; ++k) pl[k] = k < s->np ? base + (long long)k * s->pstride : nullptr;
}

template <class P>
static HalfFields<P> half_fields(const dirac_sim* s, bool upper, double t) {
  HalfFields<P> h;
  std::memset(&h, 0, sizeof(h));
  double rx = s->dt / s->dx[0];
  double beta = upper ? 1.0 : -1.0;
  h.coef_mode = s->coef_mode;
  const double th_im = s->dt * s->f.V0_imag / 2.0;
  h.c_in = make_coef<P>(s->dt * (beta * s->m + s->f.V0) / 2.0, th_im, rx);
  h.c_out = make_coef<P>(s->dt * (beta * s->m + (s->f.V0 + s->f.step_V)) / 2.0, th_im, rx);
  h.step_axis = s->f.step_axis < 0 ? 0 : s->f.step_axis;
  h.step_X = s->step_X;
  h.link_mode = s->link_mode;
  for (int k = 0; k < 3; ++k) h.L[k] = make_link<P>(s->f.q * s->f.A_const[k] * s->dx[k] / 2.0);
  h.t = t;
  h.beta = beta;
  // tabulated potential
  for (int k = 0; k < 8; ++k) h.b_tab[k] = s->b_tab && k < s->np ? s->b_tab + (long long)k * s->pstride : nullptr;
  split(rx, h.rx_hi, h.rx_lo);
  // analytic soft core: theta_0 on both sides of the Klein step, K = -dt Z/2
  // and the per-axis square tables (axis a at offset 2 (N_0 + ... + N_{a-1}))
  {
    const double t_in = s->dt * (beta * s->m + s->f.V0) / 2.0;
    const double t_out = s->f.step_axis >= 0 ? s->dt * (beta * s->m + s->f.V0 + s->f.step_V) / 2.0 : t_in;
    split(t_in, h.sc_t0[0].x, h.sc_t0[0].y);
    split(t_out, h.sc_t0[1].x, h.sc_t0[1].y);
    h.sc_step = s->f.step_axis >= 0;
    split(-s->dt * s->f.sc_Z / 2.0, h.sc_K_hi, h.sc_K_lo);
    long long off = 0;
    for (int a = 0; a < 3; ++a) {
      h.sc_sq[a] = s->sc_sq ? s->sc_sq + off : nullptr;
      off += 2LL * s->Nf[a];
    }
    h.sc_corr = s->sc_corr;
  }
  if (s->link_mode == LINK_TABLE) {
    h.larr = reinterpret_cast<const typename P::Link*>(s->larr);
    h.larr_n = (long long)s->np * s->pstride;
    h.larr_ps = s->pstride;
  }
  if (s->link_mode == LINK_PLANE) {
    h.ltab = static_cast<const char*>(s->ltab) +
             (upper ? 0 : (size_t)s->ltab_n * sizeof(typename PlaneLinkOf<P>::type));
    h.ltab_axis = s->ltab_axis;
    h.lpol = s->f.Apw_pol;
  }
  return h;
}

static bool general_fields(const dirac_sim* s) {
  return s->coef_mode == COEF_GENERAL || s->link_mode == LINK_GENERAL;
}

template <class P>
static HalfStepArgs<P> half_args(dirac_sim* s, bool upper, double t) {
  HalfStepArgs<P> a;
  std::memset(&a, 0, sizeof(a));
  plane_ptrs<P>(s, a.pl);
  for (int k = 0; k < 3; ++k) a.N[k] = s->N[k];
  a.pstride = s->pstride;
  a.iso = s->iso;
  double rx = s->dt / s->dx[0];
  a.ry = make_ratio<P>((s->dt / s->dx[1]) / rx);
  a.rz = make_ratio<P>((s->dt / s->dx[2]) / rx);
  a.h = half_fields<P>(s, upper, t);
  a.f = field_desc(s);
  a.general = general_fields(s);
  return a;
}

template <class P>
static FusedArgs<P> fused_args(dirac_sim* s, double t) {
  FusedArgs<P> a;
  std::memset(&a, 0, sizeof(a));
  typename P::cplx* in[8];
  plane_ptrs<P>(s, in);
  auto* alt = static_cast<typename P::cplx*>(s->state_alt);
  for (int k = 0; k < 8; ++k) {
    a.in[k] = in[k];
    a.out[k] = k < s->np ? alt + (long long)k * s->pstride : nullptr;
  }
  for (int k = 0; k < 3; ++k) a.N[k] = s->N[k];
  a.pstride = s->pstride;
  a.iso = s->iso;
  double rx = s->dt / s->dx[0];
  a.ry = make_ratio<P>((s->dt / s->dx[1]) / rx);
  a.rz = make_ratio<P>((s->dt / s->dx[2]) / rx);
  a.hu = half_fields<P>(s, true, t);
  a.hl = half_fields<P>(s, false, t + s->dt / 2.0);
  a.f = field_desc(s);
  a.zlo = s->zlo;
  a.nzu = s->nzu;
  a.zorg = s->zorg;
  a.Nzg = s->Nzg;
  return a;
}

// ------------------------------------------------------------------ launch plans
// Plans found by dirac_autotune, per device, grid and field path; dirac_create
// applies a remembered plan to a new simulation of the same kind.
struct PlanKey {
  int dev, dims, n0, n1, n2, coef, link, iso;
  bool operator<(const PlanKey& o) const {
    const int a[8] = {dev, dims, n0, n1, n2, coef, link, iso};
    const int b[8] = {o.dev, o.dims, o.n0, o.n1, o.n2, o.coef, o.link, o.iso};
    return std::lexicographical_compare(a, a + 8, b, b + 8);
  }
};
static std::mutex g_plan_mu;
static std::map<PlanKey, dirac_plan> g_plans;

static PlanKey plan_key(const dirac_sim* s) {
  int dev = 0;
  cudaGetDevice(&dev);
  return PlanKey{dev, s->dims, s->N[0], s->N[1], s->N[2], s->coef_mode, s->link_mode, s->iso};
}

static void drop_graphs(dirac_sim* s) {
  for (int k = 0; k < 2; ++k) {
    if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
    s->graph[k] = nullptr;
    s->graph_state[k] = nullptr;
  }
}

static dirac_plan plan_of(const dirac_sim* s) {
  dirac_plan p;
  std::memset(&p, 0, sizeof(p));
  if (!s->fused) return p;
  p.chunk = s->chunk1;
  p.two_step = s->dims == 2 ? s->tblock : 0;
  p.chunk2 = s->dims == 2 ? s->chunk2 : 0;
  p.us_per_step = s->plan_us;
  return p;
}

static const char* plan_problem(const dirac_sim* s, const dirac_plan& p) {
  if (!s->fused)
    return (p.chunk || p.two_step || p.chunk2) ? "this simulation has no fused kernels to plan" : nullptr;
  const int extent = s->dims == 3 ? s->N[2] : s->N[1];
  if (p.chunk < 0 || p.chunk > extent) return "chunk must be in [0, the marching extent]";
  if (p.chunk2 < 0 || p.chunk2 > extent) return "chunk2 must be in [0, the marching extent]";
  if (p.two_step != 0 && p.two_step != 1) return "two_step must be 0 or 1";
  if (s->dims == 3 && (p.two_step || p.chunk2)) return "two-step passes exist in (2+1)D only";
  return nullptr;
}

static void apply_plan(dirac_sim* s, const dirac_plan& p) {
  s->chunk1 = p.chunk;
  s->chunk2 = p.chunk2;
  if (s->dims == 2) s->tblock = p.two_step;
  s->plan_us = p.us_per_step;
}

// A slab of a grid decomposed along its marching axis ((3+1)D: z): the
// simulation stores nz + 2 levels, updates levels 1 .. nz, and the fields live
// on the whole grid (Nf) with its level 1 at global level z0.
struct SlabSpec {
  int z0 = 0, nz = 0, Nzg = 0;
  bool on = false;
};

static dirac_status create_sim(dirac_sim** out, int dims, const int N[3], const double dx[3], double dt,
                               double m, const dirac_fields* fields, dirac_precision precision, unsigned flags,
                               void* stream, const SlabSpec& slab);

extern "C" dirac_status dirac_create(dirac_sim** out, int dims, const int N[3], const double dx[3],
                                     double dt, double m, const dirac_fields* fields,
                                     dirac_precision precision, unsigned flags, void* stream) {
  return create_sim(out, dims, N, dx, dt, m, fields, precision, flags, stream, SlabSpec{});
}

static dirac_status create_sim(dirac_sim** out, int dims, const int N[3], const double dx[3], double dt,
                               double m, const dirac_fields* fields, dirac_precision precision, unsigned flags,
                               void* stream, const SlabSpec& slab) {
  if (!out) return fail(nullptr, DIRAC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if (dims != 2 && dims != 3) return fail(nullptr, DIRAC_ERR_INVALID, "dims must be 2 or 3");
  if (!N || !dx) return fail(nullptr, DIRAC_ERR_INVALID, "N or dx is NULL");
  if (precision != DIRAC_FP32 && precision != DIRAC_FP64)
    return fail(nullptr, DIRAC_ERR_INVALID, "unknown precision");
  for (int a = 0; a < dims; ++a) {
    if (N[a] < 2) return fail(nullptr, DIRAC_ERR_INVALID, "N[a] must be >= 2");
    if (!(dx[a] > 0.0) || !std::isfinite(dx[a]))
      return fail(nullptr, DIRAC_ERR_INVALID, "dx[a] must be positive and finite");
  }
  if (!(dt > 0.0) || !std::isfinite(dt) || !std::isfinite(m))
    return fail(nullptr, DIRAC_ERR_INVALID, "dt must be positive; m finite");
  double r2 = 0.0;
  for (int a = 0; a < dims; ++a) r2 += (dt / dx[a]) * (dt / dx[a]);
  if (r2 > 1.0 && !(flags & DIRAC_FLAG_ALLOW_UNSTABLE))
    return fail(nullptr, DIRAC_ERR_UNSTABLE,
                "sum_a (dt/dx_a)^2 > 1: beyond the stability bound of the scheme");
  if ((long long)N[0] * N[1] >= (1LL << 31))
    return fail(nullptr, DIRAC_ERR_UNSUPPORTED, "N[0]*N[1] must be below 2^31");
  dirac_fields f;
  if (fields) f = *fields; else dirac_fields_default(&f);
  if (f.step_axis >= dims) return fail(nullptr, DIRAC_ERR_INVALID, "step_axis >= dims");
  if (const char* bad = nonfinite_field(f))
    return fail(nullptr, DIRAC_ERR_INVALID, std::string(bad) + " must be finite");
  if (f.abs_W != 0.0 && (!(f.abs_width > 0.0) || !std::isfinite(f.abs_width) || f.abs_axes <= 0 ||
                         f.abs_axes >= (1 << dims)))
    return fail(nullptr, DIRAC_ERR_INVALID,
                "absorbing layers need abs_width > 0 and abs_axes a non-empty mask of the dims axes");
  if (f.Apw_amp != 0.0 && (f.Apw_pol < 0 || f.Apw_pol >= dims))
    return fail(nullptr, DIRAC_ERR_INVALID, "Apw_pol must be a spatial axis");
  if (f.A_links && (!std::isfinite(f.Alink_amp) || !std::isfinite(f.Alink_omega) || !std::isfinite(f.q)))
    return fail(nullptr, DIRAC_ERR_INVALID, "Alink_amp, Alink_omega and q must be finite");

  dirac_sim* s = new (std::nothrow) dirac_sim();
  if (!s) return fail(nullptr, DIRAC_ERR_OOM, "host allocation failed");
  s->dims = dims;
  for (int a = 0; a < 3; ++a) {
    s->N[a] = (a < dims) ? N[a] : 1;
    s->dx[a] = (a < dims) ? dx[a] : 1.0;
  }
  s->dt = dt;
  s->m = m;
  s->prec = precision;
  s->flags = flags;
  s->f = f;
  s->f.V_static = nullptr;
  s->f.A_links = nullptr;
  s->stream = static_cast<cudaStream_t>(stream);
  for (int a = 0; a < 3; ++a) s->Nf[a] = s->N[a];
  const int march = dims == 3 ? 2 : 1;  // the fused kernels' marching axis
  if (slab.on) {  // N is the whole grid: store the slab's levels and two halo levels
    s->N[march] = slab.nz + 2;
    s->zlo = 1;
    s->nzu = slab.nz;
    s->zorg = slab.z0 - 1;
    s->Nzg = slab.Nzg;
    s->tblock = 0;  // two-step passes would need two halo levels
  } else {
    s->zlo = 0;
    s->nzu = s->Nzg = s->N[march];
    s->zorg = 0;
  }
  s->ncell = cells_of(dims, s->N);
  s->pstride = round_up(s->ncell, 64);
  s->np = dims == 3 ? 8 : 4;
  s->elem = precision == DIRAC_FP32 ? sizeof(float2) : sizeof(double2);
  s->iso = (dx[0] == dx[1]) && (dims == 2 || dx[0] == dx[2]);
  // a time-independent potential beyond V0 and the step: tabulated for the FP32
  // kernels, evaluated per site in FP64 otherwise
  const bool vstatic = fields && fields->V_static;
  const bool layers = f.abs_W != 0.0;
  // a real soft core (with V0 and a Klein step, nothing else): analytic per
  // value in the FP32 kernels, no per-site data
  const bool softcore = f.sc_Z != 0.0 && f.sc_a != 0.0 && !vstatic && !layers && f.V0_imag == 0.0;
  // DIRAC_SOFTCORE selects how the FP32 kernels evaluate it: "analytic"
  // (default), "corrected" or "table"
  const char* sc_env = std::getenv("DIRAC_SOFTCORE");
  const std::string sc_how = sc_env ? sc_env : "analytic";
  if (precision == DIRAC_FP32 && softcore && (slab.on || sc_how != "table"))
    s->coef_mode = sc_how == "corrected" && !slab.on ? COEF_SOFTCORR : COEF_SOFTCORE;
  else if ((vstatic && f.Vmod_amp == 0.0) || (!vstatic && (f.sc_Z != 0.0 || layers)))
    s->coef_mode = precision == DIRAC_FP32 ? COEF_TABLE : COEF_GENERAL;
  else if (vstatic || f.sc_Z != 0.0) s->coef_mode = COEF_GENERAL;
  else s->coef_mode = f.step_axis >= 0 ? COEF_STEP : COEF_UNIFORM;
  if (f.step_axis >= 0) s->step_X = threshold_index(f.step_x0, s->dx[f.step_axis]);
  bool any_A = f.A_const[0] != 0.0 || f.A_const[1] != 0.0 || f.A_const[2] != 0.0;
  // link integrals of an arbitrary A: per-site phases (tabulated below when static)
  const bool alinks = f.A_links != nullptr;
  s->link_mode = (f.Apw_amp != 0.0 || alinks) ? LINK_GENERAL : (any_A ? LINK_CONST : LINK_NONE);
  if (f.Apw_amp != 0.0 && !alinks) {
    // a plane wave along one axis other than its polarisation (and no constant
    // A across it) is tabulated per time step along that axis
    int along = -1, count = 0;
    for (int a = 0; a < dims; ++a)
      if (f.Apw_k[a] != 0.0) { along = a; ++count; }
    bool others_zero = true;
    for (int a = 0; a < 3; ++a)
      if (a != f.Apw_pol && f.A_const[a] != 0.0) others_zero = false;
    if (count == 1 && along != f.Apw_pol && others_zero) {
      s->link_mode = LINK_PLANE;
      s->ltab_axis = along;
      s->ltab_n = 2 * s->Nf[along];
    }
  }
  // any other time-independent vector potential: its link factors are
  // tabulated once for the FP32 kernels instead of a sincos per link and step
  const bool moving = (f.Apw_amp != 0.0 && f.Apw_omega != 0.0) ||
                      (alinks && f.Alink_amp != 0.0 && f.Alink_omega != 0.0);
  if (precision == DIRAC_FP32 && s->link_mode == LINK_GENERAL && !moving) s->link_mode = LINK_TABLE;

  auto cleanup_fail = [&](dirac_status st) {
    std::string msg = s->err;
    dirac_destroy(s);
    return fail(nullptr, st, msg);
  };
  cudaError_t e;
  size_t sbytes = (size_t)s->np * s->pstride * s->elem;
  if ((e = cudaMalloc(&s->state, sbytes)) != cudaSuccess) return cleanup_fail(cuda_fail(s, e, "cudaMalloc(state)"));
  if ((e = cudaMemsetAsync(s->state, 0, sbytes, s->stream)) != cudaSuccess)
    return cleanup_fail(cuda_fail(s, e, "cudaMemsetAsync(state)"));
  if (precision == DIRAC_FP32) {
    if ((e = cudaMalloc(&s->staging, (size_t)s->pstride * sizeof(double2))) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(staging)"));
  }
  // the fused (3+1)D kernel addresses values inside a plane with 32-bit
  // offsets: larger grids take the split kernels
  s->fused = precision == DIRAC_FP32 && !(flags & DIRAC_FLAG_REFERENCE_KERNELS) &&
             (dims == 2 || s->pstride < (1LL << 31));
  if (s->fused) {
    if ((e = cudaMalloc(&s->state_alt, sbytes)) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(state_alt)"));
  }
  if (fields && fields->V_static) {
    size_t vb = (size_t)s->np * s->pstride * sizeof(double);
    if ((e = cudaMalloc(&s->Vstatic, vb)) != cudaSuccess) return cleanup_fail(cuda_fail(s, e, "cudaMalloc(V)"));
    for (int k = 0; k < s->np; ++k) {
      e = cudaMemcpyAsync(s->Vstatic + (long long)k * s->pstride, fields->V_static + (long long)k * s->ncell,
                          (size_t)s->ncell * sizeof(double), cudaMemcpyHostToDevice, s->stream);
      if (e != cudaSuccess) return cleanup_fail(cuda_fail(s, e, "cudaMemcpyAsync(V)"));
    }
  }
  if (alinks) {
    const size_t per_axis = (size_t)s->np * s->ncell;
    const size_t tb = (size_t)2 * dims * s->np * s->pstride * sizeof(double);
    if ((e = cudaMalloc(&s->Alink, tb)) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(link integrals)"));
    if ((e = cudaMemsetAsync(s->Alink, 0, tb, s->stream)) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMemsetAsync(link integrals)"));
    double* raw = nullptr;  // the caller's array, freed once the table is built
    if ((e = cudaMalloc(&raw, dims * per_axis * sizeof(double))) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(link integrals, upload)"));
    e = cudaMemcpyAsync(raw, f.A_links, dims * per_axis * sizeof(double), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess) {
      launch_link_integral_table(s->Alink, raw, dims, s->N, s->pstride, f.q, s->stream);
      e = cudaGetLastError();
      s->launches += 1;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(raw);
    if (e != cudaSuccess) return cleanup_fail(cuda_fail(s, e, "link integral table"));
  }
  if (s->link_mode == LINK_TABLE) {  // after the link integrals: the phases include them
    const size_t tb = (size_t)2 * dims * s->np * s->pstride * sizeof(F32::Link);
    if ((e = cudaMalloc(&s->larr, tb)) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(link factor table)"));
    if ((e = cudaMemsetAsync(s->larr, 0, tb, s->stream)) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMemsetAsync(link factor table)"));
    launch_link_factor_table(s->larr, field_desc(s), dims, s->N, s->pstride, s->stream);
    if ((e = cudaGetLastError()) != cudaSuccess) return cleanup_fail(cuda_fail(s, e, "link factor table"));
    s->launches += 1;
  }
  if (s->coef_mode == COEF_SOFTCORE || s->coef_mode == COEF_SOFTCORR) {
    std::vector<float2> sq;
    softcore_tables(s, sq);
    if ((e = cudaMalloc(&s->sc_sq, sq.size() * sizeof(float2))) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(soft-core tables)"));
    // synchronous: the host vector goes out of scope
    if ((e = cudaMemcpy(s->sc_sq, sq.data(), sq.size() * sizeof(float2), cudaMemcpyHostToDevice)) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMemcpy(soft-core tables)"));
  }
  if (s->coef_mode == COEF_SOFTCORR) {
    // the correction records, built on the device; if one does not fit its
    // 16 bits the simulation evaluates the soft core analytically instead
    const size_t cb = (size_t)s->np * s->ncell * sizeof(unsigned);
    int* flag = nullptr;
    if ((e = cudaMalloc(&s->sc_corr, cb)) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(soft-core corrections)"));
    if ((e = cudaMalloc(&flag, sizeof(int))) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(flag)"));
    int over = 0;
    e = cudaMemsetAsync(flag, 0, sizeof(int), s->stream);
    if (e == cudaSuccess) {
      launch_softcore_corr(s->sc_corr, half_fields<F32>(s, true, 0.0), half_fields<F32>(s, false, 0.0),
                           field_desc(s), dims, s->N, flag, s->stream);
      e = cudaGetLastError();
      s->launches += 1;
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(&over, flag, sizeof(int), cudaMemcpyDeviceToHost, s->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
    cudaFree(flag);
    if (e != cudaSuccess) return cleanup_fail(cuda_fail(s, e, "soft-core corrections"));
    if (over) {
      cudaFree(s->sc_corr);
      s->sc_corr = nullptr;
      s->coef_mode = COEF_SOFTCORE;
    }
  }
  if (s->coef_mode == COEF_TABLE) {
    if ((e = cudaMalloc(&s->b_tab, (size_t)s->np * s->pstride * sizeof(float4))) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(coefficient table)"));
    launch_coef_table(s->b_tab, field_desc(s), dims, s->N, s->pstride, s->stream);
    if ((e = cudaGetLastError()) != cudaSuccess) return cleanup_fail(cuda_fail(s, e, "coefficient table"));
    s->launches += 1;
  }
  if (s->link_mode == LINK_PLANE) {
    size_t tb = (size_t)2 * s->ltab_n * (precision == DIRAC_FP32 ? sizeof(PlaneLinkOf<F32>::type)
                                                                 : sizeof(PlaneLinkOf<F64>::type));
    if ((e = cudaMalloc(&s->ltab, tb)) != cudaSuccess) return cleanup_fail(cuda_fail(s, e, "cudaMalloc(link table)"));
  }
  if (s->fused) {
    if ((e = cudaMalloc(&s->e_partials, (size_t)kFusedEMaxBlocks * 2 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc(&s->e_sums, 2 * sizeof(double))) != cudaSuccess)
      return cleanup_fail(cuda_fail(s, e, "cudaMalloc(functional partials)"));
  }
  s->red_blocks = observables_blocks(s->N, dims);
  if ((e = cudaMalloc(&s->partials, (size_t)s->red_blocks * kObsSums * sizeof(double))) != cudaSuccess)
    return cleanup_fail(cuda_fail(s, e, "cudaMalloc(partials)"));
  if ((e = cudaMalloc(&s->sums_dev, kObsSums * sizeof(double))) != cudaSuccess ||
      (e = cudaMalloc(&s->ref_sums, kObsSums * sizeof(double))) != cudaSuccess)
    return cleanup_fail(cuda_fail(s, e, "cudaMalloc(sums)"));
  if ((e = cudaMallocHost(&s->sums_host, kObsSums * sizeof(double))) != cudaSuccess)
    return cleanup_fail(cuda_fail(s, e, "cudaMallocHost(sums)"));
  if ((e = cudaStreamSynchronize(s->stream)) != cudaSuccess)
    return cleanup_fail(cuda_fail(s, e, "cudaStreamSynchronize"));
  if (s->coef_mode == COEF_TABLE && s->Vstatic) {  // folded into the table
    cudaFree(s->Vstatic);
    s->Vstatic = nullptr;
  }
  if (s->fused) {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    auto it = g_plans.find(plan_key(s));
    if (it != g_plans.end()) apply_plan(s, it->second);
  }
  *out = s;
  return DIRAC_OK;
}

static void drop_batch_graphs(const dirac_sim* s);

extern "C" void dirac_destroy(dirac_sim* s) {
  if (!s) return;
  cudaStreamSynchronize(s->stream);
  drop_batch_graphs(s);
  for (int k = 0; k < 2; ++k)
    if (s->graph[k]) cudaGraphExecDestroy(s->graph[k]);
  cudaFree(s->state);
  cudaFree(s->state_alt);
  cudaFree(s->staging);
  cudaFree(s->Vstatic);
  cudaFree(s->b_tab);
  cudaFree(s->sc_sq);
  cudaFree(s->sc_corr);
  cudaFree(s->Alink);
  cudaFree(s->larr);
  cudaFree(s->ltab);
  cudaFree(s->e_partials);
  cudaFree(s->e_sums);
  cudaFree(s->partials);
  cudaFree(s->sums_dev);
  cudaFree(s->ref_sums);
  if (s->sums_host) cudaFreeHost(s->sums_host);
  delete s;
}

static dirac_status take_reference(dirac_sim* s);

// The device address of a page-locked, mapped host buffer of `bytes` bytes
// starting at p, or nullptr when the conversion kernels cannot access it in
// place: pageable memory, a range whose last byte is not page-locked too, an
// address not 16-byte aligned (the kernels move double2), or
// DIRAC_HOST_COPY=staged.
static const void* mapped_host(const void* p, size_t bytes) {
  if (bytes == 0 || (reinterpret_cast<uintptr_t>(p) & 15) != 0) return nullptr;
  if (const char* e = std::getenv("DIRAC_HOST_COPY"); e && std::strcmp(e, "staged") == 0) return nullptr;
  cudaPointerAttributes a0, a1;
  if (cudaPointerGetAttributes(&a0, p) != cudaSuccess) {
    cudaGetLastError();  // not a CUDA pointer: not an error of this simulation
    return nullptr;
  }
  if (a0.type != cudaMemoryTypeHost || a0.devicePointer == nullptr) return nullptr;
  const char* last = static_cast<const char*>(p) + (bytes - 1);
  if (cudaPointerGetAttributes(&a1, last) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  if (a1.type != cudaMemoryTypeHost || a1.devicePointer == nullptr ||
      static_cast<const char*>(a1.devicePointer) - static_cast<const char*>(a0.devicePointer) !=
          static_cast<ptrdiff_t>(bytes - 1))
    return nullptr;
  return a0.devicePointer;
}

extern "C" dirac_status dirac_set_spinor(dirac_sim* s, const double* host) {
  if (!s || !host) return fail(s, DIRAC_ERR_INVALID, "NULL argument");
  s->e_valid_at = -1;
  const size_t bytes = (size_t)s->ncell * sizeof(double2);
  // FP32 from a page-locked buffer: the conversion kernels read the host
  // memory in place (no copy-engine pass through the staging plane)
  const double2* mapped = s->prec == DIRAC_FP32
                              ? static_cast<const double2*>(mapped_host(host, bytes * (size_t)s->np))
                              : nullptr;
  for (int k = 0; k < s->np; ++k) {
    const double* src = host + 2LL * k * s->ncell;
    if (s->prec == DIRAC_FP64) {
      double2* dst = static_cast<double2*>(s->state) + (long long)k * s->pstride;
      CK(s, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, s->stream));
    } else {
      float2* dst = static_cast<float2*>(s->state) + (long long)k * s->pstride;
      if (mapped) {
        launch_convert_in(mapped + (long long)k * s->ncell, dst, s->ncell, s->stream);
      } else {
        CK(s, cudaMemcpyAsync(s->staging, src, bytes, cudaMemcpyHostToDevice, s->stream));
        launch_convert_in(s->staging, dst, s->ncell, s->stream);
      }
      s->launches += 1;
      CK(s, cudaGetLastError());
    }
  }
  return take_reference(s);
}

extern "C" dirac_status dirac_get_spinor(dirac_sim* s, double* host) {
  if (!s || !host) return fail(s, DIRAC_ERR_INVALID, "NULL argument");
  const size_t bytes = (size_t)s->ncell * sizeof(double2);
  double2* mapped = s->prec == DIRAC_FP32
                        ? static_cast<double2*>(const_cast<void*>(mapped_host(host, bytes * (size_t)s->np)))
                        : nullptr;
  for (int k = 0; k < s->np; ++k) {
    double* dst = host + 2LL * k * s->ncell;
    if (s->prec == DIRAC_FP64) {
      const double2* src = static_cast<double2*>(s->state) + (long long)k * s->pstride;
      CK(s, cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDeviceToHost, s->stream));
    } else {
      const float2* src = static_cast<float2*>(s->state) + (long long)k * s->pstride;
      if (mapped) {
        launch_convert_out(src, mapped + (long long)k * s->ncell, s->ncell, s->stream);
      } else {
        launch_convert_out(src, s->staging, s->ncell, s->stream);
      }
      s->launches += 1;
      CK(s, cudaGetLastError());
      if (!mapped) CK(s, cudaMemcpyAsync(dst, s->staging, bytes, cudaMemcpyDeviceToHost, s->stream));
    }
  }
  CK(s, cudaStreamSynchronize(s->stream));
  return DIRAC_OK;
}

static double sim_time(const dirac_sim* s) { return s->t0 + (double)s->k * s->dt; }

extern "C" dirac_status dirac_set_spinor_device(dirac_sim* s, const void* dev) {
  if (!s || !dev) return fail(s, DIRAC_ERR_INVALID, "NULL argument");
  s->e_valid_at = -1;
  const double2* src = static_cast<const double2*>(dev);
  for (int k = 0; k < s->np; ++k) {
    const double2* plane = src + (long long)k * s->ncell;
    if (s->prec == DIRAC_FP64) {
      double2* dst = static_cast<double2*>(s->state) + (long long)k * s->pstride;
      CK(s, cudaMemcpyAsync(dst, plane, (size_t)s->ncell * sizeof(double2), cudaMemcpyDeviceToDevice,
                            s->stream));
    } else {
      launch_convert_in(plane, static_cast<float2*>(s->state) + (long long)k * s->pstride, s->ncell,
                        s->stream);
      s->launches += 1;
      CK(s, cudaGetLastError());
    }
  }
  return take_reference(s);
}

extern "C" dirac_status dirac_get_spinor_device(dirac_sim* s, void* dev) {
  if (!s || !dev) return fail(s, DIRAC_ERR_INVALID, "NULL argument");
  double2* dst = static_cast<double2*>(dev);
  for (int k = 0; k < s->np; ++k) {
    double2* plane = dst + (long long)k * s->ncell;
    if (s->prec == DIRAC_FP64) {
      const double2* src = static_cast<double2*>(s->state) + (long long)k * s->pstride;
      CK(s, cudaMemcpyAsync(plane, src, (size_t)s->ncell * sizeof(double2), cudaMemcpyDeviceToDevice,
                            s->stream));
    } else {
      launch_convert_out(static_cast<float2*>(s->state) + (long long)k * s->pstride, plane, s->ncell,
                         s->stream);
      s->launches += 1;
      CK(s, cudaGetLastError());
    }
  }
  return DIRAC_OK;
}

// a vector potential that changes in time (its link factors too)
static bool moving_vector_potential(const dirac_sim* s) {
  return (s->f.Apw_amp != 0.0 && s->f.Apw_omega != 0.0) ||
         (s->Alink && s->f.Alink_amp != 0.0 && s->f.Alink_omega != 0.0);
}
static bool time_dependent_fields(const dirac_sim* s) {
  return (s->Vstatic && s->f.Vmod_amp != 0.0) || moving_vector_potential(s);
}

// LINK_PLANE: tabulate this step's link factors (both half-steps)
template <class P>
static void link_table(dirac_sim* s, double t, cudaStream_t st) {
  if (s->link_mode != LINK_PLANE) return;
  launch_link_table<P>(s->ltab, s->ltab_n, field_desc(s), s->dims, s->ltab_axis, s->f.Apw_pol, t,
                       t + s->dt / 2.0, st);
  s->launches += 1;
}

template <class P>
static dirac_status steps_split(dirac_sim* s, long n, cudaStream_t st) {
  for (long i = 0; i < n; ++i) {
    double t = sim_time(s);
    link_table<P>(s, t, st);
    HalfStepArgs<P> up = half_args<P>(s, true, t);
    HalfStepArgs<P> lo = half_args<P>(s, false, t + s->dt / 2.0);
    if (s->dims == 3) {
      launch_half_step<P, 3>(up, true, st);
      launch_half_step<P, 3>(lo, false, st);
    } else {
      launch_half_step<P, 2>(up, true, st);
      launch_half_step<P, 2>(lo, false, st);
    }
    s->launches += 2;
    CK(s, cudaGetLastError());
    s->k += 1;
  }
  return DIRAC_OK;
}

// want_e: the last launch also accumulates the conserved functional of the
// new state (dirac_norm then needs no reduction pass over the state)
template <class P>
static dirac_status steps_fused(dirac_sim* s, long n, cudaStream_t st, bool want_e) {
  want_e = want_e && n > 0 && std::getenv("DIRAC_NO_FUSED_NORM") == nullptr;
  int e_blocks = 0;
  // (2+1)D, time-independent fields: two steps per pass while pairs remain
  // (the two-step kernel takes whole grids: never a slab of a decomposed one)
  const bool whole = s->zlo == 0 && s->zorg == 0 && s->nzu == s->Nzg;
  const bool tb = s->dims == 2 && s->tblock && whole && !time_dependent_fields(s) &&
                  std::getenv("DIRAC_NO_TEMPORAL_BLOCKING") == nullptr;
  while (tb && n >= 2) {
    FusedArgs<P> a = fused_args<P>(s, sim_time(s));
    a.chunk = s->chunk2;
    if (want_e && n == 2) a.e_partials = s->e_partials;
    const int blocks = launch_fused2d_tb2(a, st);
    if (!blocks) break;
    if (a.e_partials) e_blocks = blocks;
    s->launches += 1;
    CK(s, cudaGetLastError());
    std::swap(s->state, s->state_alt);
    s->k += 2;
    n -= 2;
  }
  for (long i = 0; i < n; ++i) {
    link_table<P>(s, sim_time(s), st);
    FusedArgs<P> a = fused_args<P>(s, sim_time(s));
    a.chunk = s->chunk1;
    if (want_e && i == n - 1) a.e_partials = s->e_partials;
    const int blocks = s->dims == 3 ? launch_fused<P, 3>(a, st) : launch_fused<P, 2>(a, st);
    if (a.e_partials) e_blocks = blocks;
    s->launches += 1;
    CK(s, cudaGetLastError());
    std::swap(s->state, s->state_alt);
    s->k += 1;
  }
  if (e_blocks > 0 && e_blocks <= kFusedEMaxBlocks) {
    launch_finish_sums2(s->e_partials, e_blocks, s->e_sums, st);
    s->launches += 1;
    CK(s, cudaGetLastError());
    s->e_valid_at = s->k;
  }
  return DIRAC_OK;
}

// n time steps with one launch sequence each, on stream st
static dirac_status steps_plain(dirac_sim* s, long n, cudaStream_t st, bool want_e = false) {
  if (s->prec == DIRAC_FP64) return steps_split<F64>(s, n, st);
  if (s->fused) return steps_fused<F32>(s, n, st, want_e);
  return steps_split<F32>(s, n, st);
}


// Capture kGraphSteps steps starting from the current buffer into a graph
// (on a private stream, so the simulation's stream may be the legacy one).
static dirac_status build_graph(dirac_sim* s, int slot) {
  cudaStream_t cap;
  CK(s, cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
  void* state0 = s->state;
  long long k0 = s->k, l0 = s->launches;
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
  dirac_status st = DIRAC_OK;
  if (e == cudaSuccess) {
    st = steps_plain(s, kGraphSteps, cap);
    e = cudaStreamEndCapture(cap, &g);
  }
  // capturing did not run anything: restore the bookkeeping
  s->k = k0;
  s->launches = l0;
  if (s->state != state0) std::swap(s->state, s->state_alt);
  cudaStreamDestroy(cap);
  if (e != cudaSuccess || st != DIRAC_OK || !g) {
    if (g) cudaGraphDestroy(g);
    cudaGetLastError();
    s->graph_disabled = 1;  // fall back to plain launches
    return DIRAC_OK;
  }
  cudaGraphExec_t ex = nullptr;
  e = cudaGraphInstantiate(&ex, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    cudaGetLastError();
    s->graph_disabled = 1;
    return DIRAC_OK;
  }
  s->graph[slot] = ex;
  s->graph_state[slot] = state0;
  return DIRAC_OK;
}

extern "C" dirac_status dirac_step(dirac_sim* s, long nsteps) {
  if (!s) return fail(s, DIRAC_ERR_INVALID, "NULL sim");
  if (nsteps < 0) return fail(s, DIRAC_ERR_INVALID, "nsteps < 0");
  const bool graphs = !s->graph_disabled && !time_dependent_fields(s) &&
                      std::getenv("DIRAC_NO_GRAPHS") == nullptr;
  if (graphs && !s->stepped && nsteps > kGraphSteps) {
    dirac_status st = steps_plain(s, 1, s->stream);
    if (st != DIRAC_OK) return st;
    --nsteps;
  }
  s->stepped = 1;
  while (graphs && nsteps > kGraphSteps) {  // the last step is always a plain launch
    int slot = (s->graph_state[0] == s->state) ? 0 : (s->graph_state[1] == s->state ? 1 : -1);
    if (slot < 0) {
      slot = s->graph[0] ? 1 : 0;
      dirac_status st = build_graph(s, slot);
      if (st != DIRAC_OK) return st;
      if (s->graph_disabled) break;
    }
    CK(s, cudaGraphLaunch(s->graph[slot], s->stream));
    s->launches += kGraphSteps * (s->fused ? 1 : 2);
    s->k += kGraphSteps;
    if (s->fused && (kGraphSteps & 1)) std::swap(s->state, s->state_alt);
    nsteps -= kGraphSteps;
  }
  return steps_plain(s, nsteps, s->stream, true);
}

static bool batchable(const dirac_sim* s) {
  return s->fused && !time_dependent_fields(s) &&
         (s->coef_mode == COEF_UNIFORM || s->coef_mode == COEF_STEP) &&
         (s->link_mode == LINK_NONE || s->link_mode == LINK_CONST);
}

// CUDA graphs of batched step loops, reused while the same group (same
// simulations, buffer parities, plans, step count) is stepped again, as the
// serving loop does quantum after quantum; each keeps its device argument
// tables.  Entries that name a destroyed simulation are dropped by
// dirac_destroy; at most kBatchGraphs are kept (least recently used go).
struct BatchGraph {
  std::vector<dirac_sim*> sims;
  std::vector<void*> states;
  std::vector<int> chunks;
  long nsteps = 0;
  int tb = 0;
  void* tables = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t stream = nullptr;  // the group's stream, where the graph runs
  unsigned long long used = 0;
};
static std::mutex g_bg_mu;
static std::vector<BatchGraph> g_bgraphs;
static unsigned long long g_bg_clock = 0;
static const size_t kBatchGraphs = 8;
static const long kBatchGraphMaxLaunches = 256;

static void release_batch_graph(BatchGraph& e) {
  if (e.exec) cudaGraphExecDestroy(e.exec);
  if (e.tables) cudaFree(e.tables);
  e.exec = nullptr;
  e.tables = nullptr;
}

// called by dirac_destroy (the stream is synchronised, no graph of s runs)
static void drop_batch_graphs(const dirac_sim* s) {
  std::lock_guard<std::mutex> lock(g_bg_mu);
  for (size_t i = 0; i < g_bgraphs.size();) {
    bool has = false;
    for (dirac_sim* t : g_bgraphs[i].sims) has = has || t == s;
    if (has) {
      release_batch_graph(g_bgraphs[i]);
      g_bgraphs.erase(g_bgraphs.begin() + (long)i);
    } else {
      ++i;
    }
  }
}

// the launches of one batched call: pairs of steps (two-step kernel) first,
// then single steps; every launch swaps the buffers
static cudaError_t enqueue_batch(const FusedArgs<F32>* d_args, const long long* first, int n, long pairs,
                                 long launches, long long total, long long total2, int dims, int coef,
                                 int link, cudaStream_t st) {
  BatchArgs<F32> b;
  b.nsims = n;
  b.workers = 0;
  for (long i = 0; i < launches; ++i) {
    b.sims = d_args + ((i < pairs ? 2 : 0) + (i & 1)) * n;
    if (i < pairs) {
      b.first_item = first + n + 1;
      launch_fused2d_tb2_batch(b, total2, coef, link, st);
    } else {
      b.first_item = first;
      if (dims == 3)
        launch_fused_batch<F32, 3>(b, total, coef, link, st);
      else
        launch_fused_batch<F32, 2>(b, total, coef, link, st);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// one group: same dims and field path, all batchable
static dirac_status batch_group(dirac_sim* const* g, int n, long nsteps) {
  dirac_sim* s0 = g[0];
  cudaStream_t st = s0->stream;
  // (2+1)D groups take two steps per pass for pairs of steps, as stepping alone
  bool tb = s0->dims == 2 && nsteps >= 2 && std::getenv("DIRAC_NO_TEMPORAL_BLOCKING") == nullptr;
  for (int i = 0; i < n && tb; ++i) tb = g[i]->tblock != 0;
  const long pairs = tb ? nsteps / 2 : 0;
  const long launches = pairs + (nsteps - 2 * pairs);
  std::vector<int> chunks(2 * n);
  for (int i = 0; i < n; ++i) {
    dirac_sim* s = g[i];
    chunks[2 * i] = s->chunk1 > 0 ? s->chunk1 : fused_chunk(s->dims, s->N);
    chunks[2 * i + 1] = s->chunk2 > 0 ? s->chunk2 : (tb ? fused_chunk_tb2(s->N) : 0);
  }
  const bool use_graph = launches <= kBatchGraphMaxLaunches && std::getenv("DIRAC_NO_GRAPHS") == nullptr;

  auto finish = [&]() {
    for (int i = 0; i < n; ++i) {
      dirac_sim* s = g[i];
      if (launches & 1) std::swap(s->state, s->state_alt);
      s->k += nsteps;
      s->stepped = 1;
    }
    g[0]->launches += launches;  // one launch per pass serves the whole group
    return DIRAC_OK;
  };

  if (use_graph) {  // a recorded loop of this very call?
    std::lock_guard<std::mutex> lock(g_bg_mu);
    for (BatchGraph& e : g_bgraphs) {
      if (e.nsteps != nsteps || e.tb != (int)tb || e.sims.size() != (size_t)n || e.chunks != chunks) continue;
      bool same = true;
      for (int i = 0; i < n && same; ++i) same = e.sims[i] == g[i] && e.states[i] == g[i]->state;
      if (!same) continue;
      CK(s0, cudaGraphLaunch(e.exec, st));
      e.used = ++g_bg_clock;
      return finish();
    }
  }

  // argument tables [mode][buffer parity][sim] (mode 0 one step per pass, 1
  // two steps) and item prefix sums [mode][n + 1]
  const size_t args_bytes = (size_t)4 * n * sizeof(FusedArgs<F32>);
  const size_t first_bytes = (size_t)2 * (n + 1) * sizeof(long long);
  std::vector<FusedArgs<F32>> h_args(4 * (size_t)n);
  std::vector<long long> h_first(2 * (size_t)(n + 1), 0);
  for (int i = 0; i < n; ++i) {
    dirac_sim* s = g[i];
    for (int mode = 0; mode < 2; ++mode) {
      for (int p = 0; p < 2; ++p) {
        FusedArgs<F32> a = fused_args<F32>(s, sim_time(s));
        a.chunk = chunks[2 * i + mode];
        if (p == 1) {
          for (int k = 0; k < 8; ++k) {  // the other buffer is the input after an odd launch
            typename F32::cplx* tmp = a.out[k];
            a.out[k] = const_cast<typename F32::cplx*>(a.in[k]);
            a.in[k] = tmp;
          }
        }
        h_args[(mode * 2 + p) * (size_t)n + i] = a;
      }
    }
    h_first[i + 1] = h_first[i] + fused_items(s->dims, s->N, chunks[2 * i]);
    h_first[n + 1 + i + 1] = h_first[n + 1 + i] + (tb ? fused_items_tb2(s->N, chunks[2 * i + 1]) : 0);
  }
  const long long total = h_first[n], total2 = h_first[2 * (size_t)n + 1];
  void* d = nullptr;
  cudaError_t e = cudaMalloc(&d, args_bytes + first_bytes);
  if (e == cudaSuccess) e = cudaMemcpyAsync(d, h_args.data(), args_bytes, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(static_cast<char*>(d) + args_bytes, h_first.data(), first_bytes, cudaMemcpyHostToDevice,
                        st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);  // host tables go out of scope; graphs run later
  if (e != cudaSuccess) {
    if (d) cudaFree(d);
    return cuda_fail(s0, e, "batch tables");
  }
  const FusedArgs<F32>* d_args = static_cast<const FusedArgs<F32>*>(d);
  const long long* d_first = reinterpret_cast<const long long*>(static_cast<char*>(d) + args_bytes);

  if (use_graph) {  // record the loop on a private stream, keep it with its tables
    cudaStream_t cap;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    bool ok = cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) == cudaSuccess;
    if (ok) {
      ok = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed) == cudaSuccess;
      cudaError_t le = ok ? enqueue_batch(d_args, d_first, n, pairs, launches, total, total2, s0->dims,
                                          s0->coef_mode, s0->link_mode, cap)
                          : cudaSuccess;
      if (ok) ok = cudaStreamEndCapture(cap, &graph) == cudaSuccess && le == cudaSuccess && graph;
      if (ok) ok = cudaGraphInstantiate(&exec, graph, 0) == cudaSuccess;
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cap);
    }
    cudaGetLastError();  // a failed capture falls back to direct launches
    if (ok && exec) {
      e = cudaGraphLaunch(exec, st);
      if (e != cudaSuccess) {
        cudaGraphExecDestroy(exec);
        cudaFree(d);
        return cuda_fail(s0, e, "batched graph launch");
      }
      BatchGraph ent;
      ent.sims.assign(g, g + n);
      for (int i = 0; i < n; ++i) ent.states.push_back(g[i]->state);
      ent.chunks = chunks;
      ent.nsteps = nsteps;
      ent.tb = (int)tb;
      ent.tables = d;
      ent.exec = exec;
      ent.stream = st;
      std::lock_guard<std::mutex> lock(g_bg_mu);
      ent.used = ++g_bg_clock;
      if (g_bgraphs.size() >= kBatchGraphs) {  // evict the least recently used
        size_t lru = 0;
        for (size_t i = 1; i < g_bgraphs.size(); ++i)
          if (g_bgraphs[i].used < g_bgraphs[lru].used) lru = i;
        cudaStreamSynchronize(g_bgraphs[lru].stream);  // it may still run there
        release_batch_graph(g_bgraphs[lru]);
        g_bgraphs.erase(g_bgraphs.begin() + (long)lru);
      }
      g_bgraphs.push_back(ent);
      return finish();
    }
  }
  e = enqueue_batch(d_args, d_first, n, pairs, launches, total, total2, s0->dims, s0->coef_mode,
                    s0->link_mode, st);
  cudaStreamSynchronize(st);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(s0, e, "batched fused launch");
  return finish();
}

static dirac_status batch_step_impl(dirac_sim* const* sims, int nsims, long nsteps);

extern "C" dirac_status dirac_batch_step(dirac_sim* const* sims, int nsims, long nsteps) {
  g_create_error.clear();
  dirac_status st = batch_step_impl(sims, nsims, nsteps);
  if (st != DIRAC_OK && g_create_error.empty() && sims) {
    // report the failing simulation's message through dirac_last_error(NULL)
    for (int i = 0; i < nsims; ++i)
      if (sims[i] && !sims[i]->err.empty()) g_create_error = sims[i]->err;
  }
  return st;
}

static dirac_status batch_step_impl(dirac_sim* const* sims, int nsims, long nsteps) {
  if (!sims || nsims < 0 || nsteps < 0) return fail(nullptr, DIRAC_ERR_INVALID, "bad batch arguments");
  for (int i = 0; i < nsims; ++i) {
    if (!sims[i]) return fail(nullptr, DIRAC_ERR_INVALID, "NULL simulation in batch");
    if (sims[i]->stream != sims[0]->stream)
      return fail(sims[i], DIRAC_ERR_INVALID, "batched simulations must share one stream");
    for (int j = 0; j < i; ++j)
      if (sims[j] == sims[i]) return fail(sims[i], DIRAC_ERR_INVALID, "simulation listed twice");
  }
  if (nsims == 0 || nsteps == 0) return DIRAC_OK;
  std::vector<int> done(nsims, 0);
  std::vector<dirac_sim*> grp;
  for (int i = 0; i < nsims; ++i) {
    if (done[i]) continue;
    dirac_sim* s = sims[i];
    if (!batchable(s)) {
      done[i] = 1;
      dirac_status st = dirac_step(s, nsteps);
      if (st != DIRAC_OK) return st;
      continue;
    }
    grp.clear();
    for (int j = i; j < nsims; ++j) {
      dirac_sim* t = sims[j];
      if (!done[j] && batchable(t) && t->dims == s->dims && t->coef_mode == s->coef_mode &&
          t->link_mode == s->link_mode) {
        grp.push_back(t);
        done[j] = 1;
      }
    }
    dirac_status st = batch_group(grp.data(), (int)grp.size(), nsteps);
    if (st != DIRAC_OK) return st;
  }
  return DIRAC_OK;
}

template <class P>
static dirac_status observe_launch(dirac_sim* s, int dens_axis, int dens_X, double* out_dev) {
  ObsArgs<P> a;
  std::memset(&a, 0, sizeof(a));
  typename P::cplx* pl[8];
  plane_ptrs<P>(s, pl);
  for (int k = 0; k < 8; ++k) a.pl[k] = pl[k];
  for (int k = 0; k < 3; ++k) a.N[k] = s->N[k];
  a.pstride = s->pstride;
  a.link_mode = s->link_mode;
  for (int k = 0; k < 3; ++k) a.L[k] = make_link<P>(s->f.q * s->f.A_const[k] * s->dx[k] / 2.0);
  a.f = field_desc(s);
  a.t_links = sim_time(s) - s->dt / 2.0;
  a.dens_axis = dens_axis;
  a.dens_X = dens_X;
  a.partials = s->partials;
  a.zlo = s->zlo;
  a.nzu = s->nzu;
  a.zorg = s->zorg;
  a.Nzg = s->Nzg;
  if (s->dims == 3) launch_observables<P, 3>(a, s->red_blocks, s->stream);
  else launch_observables<P, 2>(a, s->red_blocks, s->stream);
  CK(s, cudaGetLastError());
  launch_finish_sums(s->partials, s->red_blocks, out_dev, s->stream);
  s->launches += 2;
  CK(s, cudaGetLastError());
  return DIRAC_OK;
}
template <class P>
static dirac_status observe(dirac_sim* s, int dens_axis, int dens_X) {
  dirac_status st = observe_launch<P>(s, dens_axis, dens_X, s->sums_dev);
  if (st != DIRAC_OK) return st;
  CK(s, cudaMemcpyAsync(s->sums_host, s->sums_dev, kObsSums * sizeof(double), cudaMemcpyDeviceToHost,
                        s->stream));
  CK(s, cudaStreamSynchronize(s->stream));
  return DIRAC_OK;
}

static dirac_status observe_any(dirac_sim* s, int dens_axis, int dens_X) {
  return s->prec == DIRAC_FP64 ? observe<F64>(s, dens_axis, dens_X) : observe<F32>(s, dens_axis, dens_X);
}

// reduce the functional of the state just set into ref_sums (stream-ordered,
// no synchronisation): the reference of dirac_check
static dirac_status take_reference(dirac_sim* s) {
  dirac_status st = s->prec == DIRAC_FP64 ? observe_launch<F64>(s, -1, 0, s->ref_sums)
                                          : observe_launch<F32>(s, -1, 0, s->ref_sums);
  s->ref_valid = st == DIRAC_OK;
  return st;
}

extern "C" dirac_status dirac_norm(dirac_sim* s, double* E, double* naive) {
  if (!s || !E) return fail(s, DIRAC_ERR_INVALID, "NULL argument");
  double e;
  const double* v = s->sums_host;
  if (s->e_valid_at == s->k && s->e_sums && std::getenv("DIRAC_NO_FUSED_NORM") == nullptr) {
    // accumulated by the last step's kernel: E = sum |psi|^2 + r_x Re sum conj(G) S'_G
    CK(s, cudaMemcpyAsync(s->sums_host, s->e_sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    e = v[0] + (s->dt / s->dx[0]) * v[1];
  } else {
    dirac_status st = observe_any(s, -1, 0);
    if (st != DIRAC_OK) return st;
    e = v[0];
    for (int a = 0; a < s->dims; ++a) e += (s->dt / s->dx[a]) * v[1 + a];
  }
  *E = e;
  if (naive) *naive = v[0];
  if (!std::isfinite(e)) return fail(s, DIRAC_ERR_DIVERGED, "conserved functional is not finite");
  return DIRAC_OK;
}

extern "C" dirac_status dirac_partial_density(dirac_sim* s, int axis, double x0, double* out) {
  if (!s || !out) return fail(s, DIRAC_ERR_INVALID, "NULL argument");
  if (axis < 0 || axis >= s->dims) return fail(s, DIRAC_ERR_INVALID, "axis out of range");
  if (!std::isfinite(x0)) return fail(s, DIRAC_ERR_INVALID, "x0 must be finite");
  dirac_status st = observe_any(s, axis, threshold_index(x0, s->dx[axis]));
  if (st != DIRAC_OK) return st;
  *out = s->sums_host[4];
  return DIRAC_OK;
}

extern "C" long long dirac_kernel_launches(const dirac_sim* s) { return s ? s->launches : 0; }

extern "C" dirac_status dirac_get_time(const dirac_sim* s, double* t) {
  if (!s || !t) return DIRAC_ERR_INVALID;
  *t = sim_time(s);
  return DIRAC_OK;
}

extern "C" dirac_status dirac_set_time(dirac_sim* s, double t) {
  if (!s || !std::isfinite(t)) return fail(s, DIRAC_ERR_INVALID, "bad time");
  s->t0 = t;
  s->k = 0;
  s->e_valid_at = -1;
  return DIRAC_OK;
}

extern "C" dirac_status dirac_get_plan(const dirac_sim* s, dirac_plan* out) {
  if (!s || !out) return fail(const_cast<dirac_sim*>(s), DIRAC_ERR_INVALID, "NULL argument");
  *out = plan_of(s);
  return DIRAC_OK;
}

extern "C" dirac_status dirac_set_plan(dirac_sim* s, const dirac_plan* plan) {
  if (!s || !plan) return fail(s, DIRAC_ERR_INVALID, "NULL argument");
  if (const char* why = plan_problem(s, *plan)) return fail(s, DIRAC_ERR_INVALID, why);
  if (!s->fused) return DIRAC_OK;
  CK(s, cudaStreamSynchronize(s->stream));
  drop_graphs(s);
  dirac_plan p = *plan;
  p.us_per_step = 0.0;
  apply_plan(s, p);
  return DIRAC_OK;
}

// Time `reps` launches of one candidate (after one untimed launch) on the
// current state, out of place into the spare buffer; milliseconds per launch.
static dirac_status time_candidate(dirac_sim* s, int two_step, int chunk, int reps, cudaEvent_t e0,
                                   cudaEvent_t e1, float* ms) {
  FusedArgs<F32> a = fused_args<F32>(s, sim_time(s));
  a.chunk = chunk;
  for (int r = 0; r <= reps; ++r) {
    if (r == 1) CK(s, cudaEventRecord(e0, s->stream));
    const int blocks = two_step ? launch_fused2d_tb2(a, s->stream)
                                : (s->dims == 3 ? launch_fused<F32, 3>(a, s->stream)
                                                : launch_fused<F32, 2>(a, s->stream));
    if (!blocks) return fail(s, DIRAC_ERR_UNSUPPORTED, "no two-step kernel for these fields");
    s->launches += 1;
    CK(s, cudaGetLastError());
  }
  CK(s, cudaEventRecord(e1, s->stream));
  CK(s, cudaEventSynchronize(e1));
  float t = 0.0f;
  CK(s, cudaEventElapsedTime(&t, e0, e1));
  *ms = t / (float)reps;
  return DIRAC_OK;
}

extern "C" dirac_status dirac_autotune(dirac_sim* s, dirac_plan* out) {
  if (!s) return fail(s, DIRAC_ERR_INVALID, "NULL sim");
  if (!s->fused) {
    if (out) *out = plan_of(s);
    return DIRAC_OK;
  }
  constexpr int kCandidates = 6;
  int c1[kCandidates], c2[kCandidates];
  const int n1 = fused_candidates(s->dims, s->N, 0, c1, kCandidates);
  const bool tb_ok = s->dims == 2 && s->zlo == 0 && s->nzu == s->Nzg && !time_dependent_fields(s) &&
                     (s->coef_mode == COEF_UNIFORM || s->coef_mode == COEF_STEP ||
                      s->coef_mode == COEF_TABLE || s->coef_mode == COEF_SOFTCORE ||
                      s->coef_mode == COEF_SOFTCORR) &&
                     (s->link_mode == LINK_NONE || s->link_mode == LINK_CONST) &&
                     !((s->coef_mode == COEF_TABLE || s->coef_mode == COEF_SOFTCORE ||
                        s->coef_mode == COEF_SOFTCORR) && s->link_mode == LINK_CONST);
  const int n2 = tb_ok ? fused_candidates(2, s->N, 1, c2, kCandidates) : 0;
  link_table<F32>(s, sim_time(s), s->stream);  // plane-wave links of the current step, if any
  cudaEvent_t e0, e1;
  CK(s, cudaEventCreate(&e0));
  cudaError_t ce = cudaEventCreate(&e1);
  if (ce != cudaSuccess) {
    cudaEventDestroy(e0);
    return cuda_fail(s, ce, "cudaEventCreate");
  }
  // repetitions: about a millisecond of launches per candidate and sweep
  float t0 = 0.0f;
  dirac_status st = time_candidate(s, 0, c1[0], 1, e0, e1, &t0);
  int reps = 2;
  if (st == DIRAC_OK && t0 > 0.0f) reps = (int)std::ceil(1.0f / t0);
  reps = reps < 2 ? 2 : (reps > 50 ? 50 : reps);
  float best1[kCandidates], best2[kCandidates];
  for (int i = 0; i < kCandidates; ++i) best1[i] = best2[i] = 1e30f;
  for (int sweep = 0; sweep < 2 && st == DIRAC_OK; ++sweep) {
    for (int i = 0; i < n1 && st == DIRAC_OK; ++i) {
      float ms = 0.0f;
      st = time_candidate(s, 0, c1[i], reps, e0, e1, &ms);
      if (ms < best1[i]) best1[i] = ms;
    }
    for (int i = 0; i < n2 && st == DIRAC_OK; ++i) {
      float ms = 0.0f;
      st = time_candidate(s, 1, c2[i], reps, e0, e1, &ms);
      if (ms / 2.0f < best2[i]) best2[i] = ms / 2.0f;  // two steps per launch
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != DIRAC_OK) return st;
  int i1 = 0, i2 = 0;
  for (int i = 1; i < n1; ++i) if (best1[i] < best1[i1]) i1 = i;
  for (int i = 1; i < n2; ++i) if (best2[i] < best2[i2]) i2 = i;
  dirac_plan p;
  std::memset(&p, 0, sizeof(p));
  p.chunk = c1[i1];
  p.us_per_step = 1e3 * best1[i1];
  if (n2 > 0) {
    p.chunk2 = c2[i2];
    p.two_step = best2[i2] < best1[i1] ? 1 : 0;
    if (p.two_step) p.us_per_step = 1e3 * best2[i2];
  } else if (s->dims == 2) {
    p.two_step = s->tblock;  // fields that never take two-step passes: keep the flag as it was
  }
  drop_graphs(s);
  apply_plan(s, p);
  {
    std::lock_guard<std::mutex> lock(g_plan_mu);
    g_plans[plan_key(s)] = p;
  }
  if (out) *out = p;
  return DIRAC_OK;
}


extern "C" void dirac_functional_bounds(int dims, const double dx[3], double dt, int general_A, double* lo,
                                        double* hi) {
  double sum = 0.0, sum2 = 0.0;
  for (int a = 0; a < dims && dx; ++a) {
    const double r = dt / dx[a];
    sum += r;
    sum2 += r * r;
  }
  const double rho = general_A ? sum : std::sqrt(sum2);
  if (lo) *lo = 1.0 - rho;
  if (hi) *hi = 1.0 + rho;
}

extern "C" dirac_status dirac_check(dirac_sim* s, double tol, dirac_check_report* out) {
  if (!s) return fail(s, DIRAC_ERR_INVALID, "NULL sim");
  if (!(tol >= 0.0)) return fail(s, DIRAC_ERR_INVALID, "tol must be >= 0");
  dirac_check_report r;
  std::memset(&r, 0, sizeof(r));
  const double nan = std::nan("");
  r.E_ref = r.naive_ref = r.drift = nan;
  dirac_status st = dirac_norm(s, &r.E, &r.naive);
  if (st != DIRAC_OK && st != DIRAC_ERR_DIVERGED) return st;
  if (!std::isfinite(r.E) || !std::isfinite(r.naive)) r.failed |= DIRAC_CHECK_NONFINITE;
  if (s->ref_valid) {
    double ref[kObsSums];
    CK(s, cudaMemcpyAsync(s->sums_host, s->ref_sums, kObsSums * sizeof(double), cudaMemcpyDeviceToHost,
                          s->stream));
    CK(s, cudaStreamSynchronize(s->stream));
    std::memcpy(ref, s->sums_host, sizeof(ref));
    r.naive_ref = ref[0];
    r.E_ref = ref[0];
    for (int a = 0; a < s->dims; ++a) r.E_ref += (s->dt / s->dx[a]) * ref[1 + a];
    r.drift = (r.E - r.E_ref) / std::fabs(r.E_ref);
  }
  // bounds of the functional as a quadratic form
  double lo = 0.0, hi = 0.0;
  const int general_A = s->link_mode == LINK_GENERAL || s->link_mode == LINK_PLANE ||
                        s->link_mode == LINK_TABLE;
  dirac_functional_bounds(s->dims, s->dx, s->dt, general_A, &lo, &hi);
  r.lower = 0.0;
  r.upper = INFINITY;
  if (lo > 0.0 && std::isfinite(r.E)) {
    r.lower = r.E / hi;
    r.upper = r.E / lo;
    const double slack = 1e-10 * r.naive;
    if (r.naive < r.lower - slack || r.naive > r.upper + slack) r.failed |= DIRAC_CHECK_BOUND;
  }
  // conservation (real V, static A) or no growth (Im V <= 0 everywhere)
  const bool moving_A = moving_vector_potential(s);
  const bool imag = s->f.V0_imag != 0.0 || s->f.abs_W != 0.0;
  const bool damping = s->f.V0_imag <= 0.0 && s->f.abs_W >= 0.0;
  if (s->ref_valid && !moving_A && std::isfinite(r.drift)) {
    if (!imag && std::fabs(r.drift) > tol) r.failed |= DIRAC_CHECK_DRIFT;
    if (imag && damping && r.drift > tol) r.failed |= DIRAC_CHECK_DRIFT;
  }
  if (out) *out = r;
  if (r.failed) {
    std::string m = "stability check failed:";
    if (r.failed & DIRAC_CHECK_NONFINITE) m += " non-finite values;";
    if (r.failed & DIRAC_CHECK_BOUND) m += " sum |psi|^2 outside the bounds implied by E;";
    if (r.failed & DIRAC_CHECK_DRIFT) m += " E drifted beyond tol;";
    return fail(s, DIRAC_ERR_DIVERGED, m);
  }
  return DIRAC_OK;
}


extern "C" double dirac_algorithmic_bytes(const dirac_sim* s) {
  if (!s) return 0.0;
  double b = 2.0 * s->np * (double)s->elem;                    // every value read and written once
  if (s->coef_mode == COEF_TABLE) b += 16.0 * s->np;           // one coefficient per value read
  if (s->coef_mode == COEF_SOFTCORR) b += 4.0 * s->np;         // one correction word per value read
  if (s->coef_mode == COEF_GENERAL && s->Vstatic) b += 8.0 * s->np;  // one real per value read
  if (s->link_mode == LINK_TABLE) b += 32.0 * s->dims * s->np;  // up and down link factor (hi + lo) per axis
  else if (s->Alink) b += 16.0 * s->dims * s->np;              // up and down link integral per axis
  return b;
}

// ------------------------------------------------------------------ sub-domains
// The grid split along z into slabs of consecutive levels (the paper's
// parallelisation: spatial sub-domains with boundary exchange, Sect. 6).
// Every slab is a simulation of its own levels plus one halo level on either
// side; after every time step each slab's first and last own levels are
// copied into the halo levels of its neighbours (periodic: the last slab's
// upper neighbour is the first).  All slabs live on the calling device here;
// the same exchange between devices would copy peer to peer.
struct dirac_slabs {
  int n = 0;
  int dims = 3;
  int march = 2;              // split axis: z in (3+1)D, y in (2+1)D
  int N[3] = {1, 1, 1};
  std::vector<dirac_sim*> sim;
  std::vector<int> z0, nz;
  cudaStream_t stream = nullptr;
  std::string err;
};

extern "C" void dirac_slab_partition(int Nz, int nslabs, int k, int* z0, int* nz) {
  // nslabs nearly equal slabs, the first Nz mod nslabs one level longer
  if (nslabs < 1 || k < 0 || k >= nslabs || Nz < 0) {
    if (z0) *z0 = 0;
    if (nz) *nz = 0;
    return;
  }
  const int q = Nz / nslabs, r = Nz % nslabs;
  if (z0) *z0 = k * q + (k < r ? k : r);
  if (nz) *nz = q + (k < r ? 1 : 0);
}

static dirac_status slabs_fail(dirac_slabs* g, dirac_status st, const std::string& msg) {
  if (st == DIRAC_ERR_CUDA) cudaGetLastError();  // as cuda_fail: no stale error for later calls
  if (g) g->err = msg;
  else g_create_error = msg;
  return st;
}

extern "C" void dirac_slabs_destroy(dirac_slabs* g) {
  if (!g) return;
  for (dirac_sim* s : g->sim) dirac_destroy(s);
  delete g;
}

extern "C" dirac_status dirac_slabs_create(dirac_slabs** out, int nslabs, int dims, const int N[3],
                                           const double dx[3], double dt, double m, const dirac_fields* fields,
                                           dirac_precision precision, unsigned flags, void* stream) {
  if (!out) return slabs_fail(nullptr, DIRAC_ERR_INVALID, "out is NULL");
  *out = nullptr;
  if ((dims != 2 && dims != 3) || !N) return slabs_fail(nullptr, DIRAC_ERR_INVALID, "slabs: dims must be 2 or 3");
  if (precision != DIRAC_FP32 || (flags & DIRAC_FLAG_REFERENCE_KERNELS))
    return slabs_fail(nullptr, DIRAC_ERR_UNSUPPORTED, "slabs: the FP32 fused kernels only");
  const int march = dims == 3 ? 2 : 1;  // z in (3+1)D, y in (2+1)D
  if (nslabs < 1 || N[march] < nslabs)
    return slabs_fail(nullptr, DIRAC_ERR_INVALID, "slabs: need 1 <= nslabs <= the grid's extent along z (y in (2+1)D)");
  if (fields && (fields->V_static || fields->A_links || fields->abs_W != 0.0))
    return slabs_fail(nullptr, DIRAC_ERR_UNSUPPORTED,
                      "slabs: fields given per site (V_static, A_links) or absorbing layers are not decomposed");
  dirac_slabs* g = new (std::nothrow) dirac_slabs();
  if (!g) return slabs_fail(nullptr, DIRAC_ERR_OOM, "host allocation failed");
  g->n = nslabs;
  g->dims = dims;
  g->march = march;
  for (int a = 0; a < 3; ++a) g->N[a] = a < dims ? N[a] : 1;
  g->stream = static_cast<cudaStream_t>(stream);
  for (int k = 0; k < nslabs; ++k) {
    SlabSpec sp;
    sp.on = true;
    dirac_slab_partition(N[march], nslabs, k, &sp.z0, &sp.nz);
    sp.Nzg = N[march];
    dirac_sim* s = nullptr;
    dirac_status st = create_sim(&s, dims, N, dx, dt, m, fields, precision, flags, stream, sp);
    if (st != DIRAC_OK) {
      dirac_slabs_destroy(g);
      return st;  // the message is in dirac_last_error(NULL)
    }
    if (s->link_mode == LINK_TABLE || s->coef_mode == COEF_TABLE || s->coef_mode == COEF_GENERAL) {
      // per-site tables are laid out on the stored cells: not decomposed
      dirac_destroy(s);
      dirac_slabs_destroy(g);
      return slabs_fail(nullptr, DIRAC_ERR_UNSUPPORTED,
                        "slabs: fields that need per-site tables (a static vector potential that is not a "
                        "plane wave across its polarisation) are not decomposed");
    }
    g->sim.push_back(s);
    g->z0.push_back(sp.z0);
    g->nz.push_back(sp.nz);
  }
  *out = g;
  return DIRAC_OK;
}

extern "C" const char* dirac_slabs_last_error(const dirac_slabs* g) {
  if (!g) return g_create_error.c_str();
  if (!g->err.empty()) return g->err.c_str();
  for (dirac_sim* s : g->sim)
    if (!s->err.empty()) return s->err.c_str();
  return "";
}

extern "C" dirac_status dirac_slabs_info(const dirac_slabs* g, int k, int* z0, int* nz) {
  if (!g || k < 0 || k >= g->n) return DIRAC_ERR_INVALID;
  if (z0) *z0 = g->z0[k];
  if (nz) *nz = g->nz[k];
  return DIRAC_OK;
}

// copy one stored level of every plane from slab a into slab b (device to
// device on the group's stream)
static dirac_status copy_level(dirac_slabs* g, dirac_sim* a, int la, dirac_sim* b, int lb) {
  const size_t lvl = g->march == 2 ? (size_t)a->N[0] * a->N[1] : (size_t)a->N[0];  // values per level
  for (int p = 0; p < a->np; ++p) {
    const float2* src = static_cast<const float2*>(a->state) + (long long)p * a->pstride + (long long)la * lvl;
    float2* dst = static_cast<float2*>(b->state) + (long long)p * b->pstride + (long long)lb * lvl;
    cudaError_t e = cudaMemcpyAsync(dst, src, lvl * sizeof(float2), cudaMemcpyDeviceToDevice, g->stream);
    if (e != cudaSuccess) return slabs_fail(g, DIRAC_ERR_CUDA, std::string("halo copy: ") + cudaGetErrorString(e));
  }
  return DIRAC_OK;
}

// every slab's halo levels from its neighbours' own boundary levels
static dirac_status exchange_halos(dirac_slabs* g) {
  for (int k = 0; k < g->n; ++k) {
    dirac_sim* s = g->sim[k];
    dirac_sim* up = g->sim[(k + 1) % g->n];
    dirac_sim* dn = g->sim[(k + g->n - 1) % g->n];
    dirac_status st = copy_level(g, s, g->nz[k], up, 0);  // last own level -> upper neighbour's lower halo
    if (st == DIRAC_OK)
      st = copy_level(g, s, 1, dn, dn->N[g->march] - 1);  // first own level -> lower neighbour's upper halo
    if (st != DIRAC_OK) return st;
  }
  return DIRAC_OK;
}

extern "C" dirac_status dirac_slabs_set_spinor(dirac_slabs* g, const double* host) {
  if (!g || !host) return slabs_fail(g, DIRAC_ERR_INVALID, "NULL argument");
  const long long lvl = g->march == 2 ? (long long)g->N[0] * g->N[1] : (long long)g->N[0];
  const long long ncell = (long long)g->N[0] * g->N[1] * g->N[2];
  const int Ng = g->N[g->march];
  for (int k = 0; k < g->n; ++k) {
    dirac_sim* s = g->sim[k];
    s->e_valid_at = -1;
    for (int p = 0; p < s->np; ++p) {
      // the slab's stored levels (halos included) of this plane, from the global state
      for (int l = 0; l < s->N[g->march]; ++l) {
        int gzl = (g->z0[k] - 1 + l) % Ng;
        if (gzl < 0) gzl += Ng;
        const double* src = host + 2 * ((long long)p * ncell + gzl * lvl);
        cudaError_t e = cudaMemcpyAsync(s->staging + l * lvl, src, lvl * sizeof(double2), cudaMemcpyHostToDevice,
                                        s->stream);
        if (e != cudaSuccess) return slabs_fail(g, DIRAC_ERR_CUDA, std::string("set: ") + cudaGetErrorString(e));
      }
      launch_convert_in(s->staging, static_cast<float2*>(s->state) + (long long)p * s->pstride, s->ncell, s->stream);
      s->launches += 1;
      cudaError_t e = cudaGetLastError();
      if (e != cudaSuccess) return slabs_fail(g, DIRAC_ERR_CUDA, std::string("set: ") + cudaGetErrorString(e));
    }
    dirac_status st = take_reference(s);
    if (st != DIRAC_OK) return st;
  }
  return DIRAC_OK;
}

extern "C" dirac_status dirac_slabs_get_spinor(dirac_slabs* g, double* host) {
  if (!g || !host) return slabs_fail(g, DIRAC_ERR_INVALID, "NULL argument");
  const long long lvl = g->march == 2 ? (long long)g->N[0] * g->N[1] : (long long)g->N[0];
  const long long ncell = (long long)g->N[0] * g->N[1] * g->N[2];
  for (int k = 0; k < g->n; ++k) {
    dirac_sim* s = g->sim[k];
    for (int p = 0; p < s->np; ++p) {
      launch_convert_out(static_cast<const float2*>(s->state) + (long long)p * s->pstride, s->staging, s->ncell,
                         s->stream);
      s->launches += 1;
      cudaError_t e = cudaGetLastError();
      // own levels 1 .. nz only
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(host + 2 * ((long long)p * ncell + (long long)g->z0[k] * lvl), s->staging + lvl,
                            (size_t)g->nz[k] * lvl * sizeof(double2), cudaMemcpyDeviceToHost, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);  // one staging plane per slab
      if (e != cudaSuccess) return slabs_fail(g, DIRAC_ERR_CUDA, std::string("get: ") + cudaGetErrorString(e));
    }
  }
  return DIRAC_OK;
}

extern "C" dirac_status dirac_slabs_step(dirac_slabs* g, long nsteps) {
  if (!g || nsteps < 0) return slabs_fail(g, DIRAC_ERR_INVALID, "bad arguments");
  for (long i = 0; i < nsteps; ++i) {
    for (int k = 0; k < g->n; ++k) {
      dirac_status st = steps_fused<F32>(g->sim[k], 1, g->stream, i == nsteps - 1);
      if (st != DIRAC_OK) return st;
    }
    dirac_status st = exchange_halos(g);
    if (st != DIRAC_OK) return st;
  }
  return DIRAC_OK;
}

extern "C" dirac_status dirac_slabs_norm(dirac_slabs* g, double* E, double* naive) {
  if (!g || !E) return slabs_fail(g, DIRAC_ERR_INVALID, "NULL argument");
  double e = 0.0, nv = 0.0;
  for (dirac_sim* s : g->sim) {  // E and the naive norm are sums over the slabs' own values
    double es = 0.0, ns = 0.0;
    dirac_status st = dirac_norm(s, &es, &ns);
    if (st != DIRAC_OK) return st;
    e += es;
    nv += ns;
  }
  *E = e;
  if (naive) *naive = nv;
  return DIRAC_OK;
}

extern "C" dirac_status dirac_slabs_get_time(const dirac_slabs* g, double* t) {
  if (!g || !t || g->sim.empty()) return DIRAC_ERR_INVALID;
  return dirac_get_time(g->sim[0], t);
}

extern "C" long long dirac_slabs_kernel_launches(const dirac_slabs* g) {
  long long n = 0;
  if (g)
    for (const dirac_sim* s : g->sim) n += s->launches;
  return n;
}

extern "C" dirac_status dirac_fp64_fma_rate(double* tflops) {
  if (!tflops) return fail(nullptr, DIRAC_ERR_INVALID, "NULL argument");
  const double r = measure_fp64_fma_tflops();
  if (r < 0.0) {
    cudaGetLastError();
    return fail(nullptr, DIRAC_ERR_CUDA, "FP64 rate measurement failed");
  }
  *tflops = r;
  return DIRAC_OK;
}
