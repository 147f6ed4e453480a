/*
 * FP64 CPU oracle of the staggered space-time leap-frog Dirac scheme
 * (arXiv:1309.3452).  TEST INFRASTRUCTURE ONLY: see dirac_oracle.h for the
 * formulation, the layout and who may use it.
 *
 * Built with -ffp-contract=off and without -ffast-math, so every operation
 * below rounds exactly as written.
 *
 * Readings of the paper taken here (each is pinned by a test):
 *  - Eq. Dirac-A prints "m^2 c"; the mass term is m c^2 (as in Eq. 3+3D and
 *    Eqs. sbegin, ss1).  With hbar = c = 1 it is m.
 *  - The time-average operator T (Eq. 3+3Ddis) acts on the mass/potential
 *    term only, so each site update is the Cayley form
 *        psi+ = ((1 - i th) psi- - S) / (1 + i th),  th = dt (beta m + V) / 2,
 *    beta = +1 on A,B,u and -1 on C,D,v (Eqs. ss1-ss4, scheme2Deq-scheme4thline).
 *  - V is taken at the time sheet of the neighbours: t for the upper
 *    half-step and t + dt/2 for the lower one (the superscripts j_o and
 *    j_o+1/2 of Eqs. ss1-ss4).
 *  - The vector potential enters through exact Peierls link factors
 *    (Sect. 4): in a difference along axis a the neighbour at +dx_a/2 is
 *    multiplied by exp(-i phi) and the one at -dx_a/2 by exp(+i phi'), where
 *    phi = q times the line integral of A_a along that link (of length
 *    dx_a/2) at the neighbours' time t_nb: A_const dx_a/2, the plane wave's
 *    exact integral (its midpoint value times sin(k_a dx_a/4)/(k_a dx_a/4)),
 *    and the caller's tabulated link integrals.  To first order in A this is
 *    the printed rule for spatial differences in Sect. 4; the printed rule
 *    for the time derivative belongs to the gauge-transformed picture and is
 *    not applied on top of the links.
 *  - Boundaries are periodic in units of the cell.
 */
#include "dirac_oracle.h"

#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

typedef struct {
  int dims;
  long M[3];  /* half-lattice extent per axis: 2 N_a (1 for an absent z axis) */
  long n;     /* number of half-lattice points */
  double* link[3];  /* A_links on the half lattice: link[a][f] belongs to the link f -> f + e_a */
} grid;

static grid make_grid(const oracle_problem* p) {
  grid g;
  g.dims = p->dims;
  g.M[0] = 2L * p->N[0];
  g.M[1] = 2L * p->N[1];
  g.M[2] = (p->dims == 3) ? 2L * p->N[2] : 1;
  g.n = g.M[0] * g.M[1] * g.M[2];
  g.link[0] = g.link[1] = g.link[2] = NULL;
  return g;
}

static long fine_index(const grid* g, long X, long Y, long Z) {
  return (Z * g->M[1] + Y) * g->M[0] + X;
}

static long wrap(long i, long M) {
  long r = i % M;
  return r < 0 ? r + M : r;
}

/* half-lattice offsets of each canonical plane inside its cell
   (Sect. 2 grid definitions; Sect. 3 fcr-u / fcr-v) */
static const int plane_offset3[8][3] = {
    {0, 0, 0}, /* A0 */ {1, 1, 0}, /* A1 */
    {1, 0, 1}, /* B0 */ {0, 1, 1}, /* B1 */
    {0, 0, 1}, /* C0 */ {1, 1, 1}, /* C1 */
    {1, 0, 0}, /* D0 */ {0, 1, 0}, /* D1 */
};
static const int plane_offset2[4][3] = {
    {0, 0, 0}, /* u0 */ {1, 1, 0}, /* u1 */
    {1, 0, 0}, /* v0 */ {0, 1, 0}, /* v1 */
};

static int n_planes(const oracle_problem* p) { return p->dims == 3 ? 8 : 4; }

static const int* plane_offset(const oracle_problem* p, int plane) {
  return p->dims == 3 ? plane_offset3[plane] : plane_offset2[plane];
}

static long cells(const oracle_problem* p) {
  return (long)p->N[0] * p->N[1] * (p->dims == 3 ? p->N[2] : 1);
}

/* canonical planes -> half-lattice array (and back) */
static void planes_to_fine(const oracle_problem* p, const grid* g, const double* planes, cplx* fine) {
  long nc = cells(p);
  int nz = p->dims == 3 ? p->N[2] : 1;
  for (int pl = 0; pl < n_planes(p); ++pl) {
    const int* o = plane_offset(p, pl);
    for (long jz = 0; jz < nz; ++jz)
      for (long jy = 0; jy < p->N[1]; ++jy)
        for (long jx = 0; jx < p->N[0]; ++jx) {
          long c = (jz * p->N[1] + jy) * p->N[0] + jx;
          const double* v = planes + 2 * (pl * nc + c);
          long f = fine_index(g, 2 * jx + o[0], 2 * jy + o[1], p->dims == 3 ? 2 * jz + o[2] : 0);
          fine[f] = v[0] + I * v[1];
        }
  }
}

static void fine_to_planes(const oracle_problem* p, const grid* g, const cplx* fine, double* planes) {
  long nc = cells(p);
  int nz = p->dims == 3 ? p->N[2] : 1;
  for (int pl = 0; pl < n_planes(p); ++pl) {
    const int* o = plane_offset(p, pl);
    for (long jz = 0; jz < nz; ++jz)
      for (long jy = 0; jy < p->N[1]; ++jy)
        for (long jx = 0; jx < p->N[0]; ++jx) {
          long c = (jz * p->N[1] + jy) * p->N[0] + jx;
          double* v = planes + 2 * (pl * nc + c);
          long f = fine_index(g, 2 * jx + o[0], 2 * jy + o[1], p->dims == 3 ? 2 * jz + o[2] : 0);
          v[0] = creal(fine[f]);
          v[1] = cimag(fine[f]);
        }
  }
}

/* one real per site, canonical plane layout -> half-lattice */
static double* real_planes_to_fine(const oracle_problem* p, const grid* g, const double* planes) {
  if (!planes) return NULL;
  double* fine = (double*)calloc((size_t)g->n, sizeof(double));
  long nc = cells(p);
  int nz = p->dims == 3 ? p->N[2] : 1;
  for (int pl = 0; pl < n_planes(p); ++pl) {
    const int* o = plane_offset(p, pl);
    for (long jz = 0; jz < nz; ++jz)
      for (long jy = 0; jy < p->N[1]; ++jy)
        for (long jx = 0; jx < p->N[0]; ++jx) {
          long c = (jz * p->N[1] + jy) * p->N[0] + jx;
          long f = fine_index(g, 2 * jx + o[0], 2 * jy + o[1], p->dims == 3 ? 2 * jz + o[2] : 0);
          fine[f] = planes[pl * nc + c];
        }
  }
  return fine;
}

/* A_links (one real per value and axis, canonical layout) -> g->link */
static void links_to_fine(const oracle_problem* p, grid* g) {
  if (!p->A_links) return;
  long per_axis = (long)n_planes(p) * cells(p);
  for (int a = 0; a < p->dims; ++a) g->link[a] = real_planes_to_fine(p, g, p->A_links + a * per_axis);
}

static void free_links(grid* g) {
  for (int a = 0; a < 3; ++a) free(g->link[a]);
}

/* physical position of a half-lattice point */
static void position(const oracle_problem* p, long X, long Y, long Z, double x[3]) {
  long F[3] = {X, Y, Z};
  for (int a = 0; a < 3; ++a) x[a] = (double)(F[a] + 2L * p->origin[a]) * p->dx[a] / 2.0;
  if (p->dims == 2) x[2] = 0.0;
}

/* imaginary part of the scalar potential: a uniform part and absorbing
   layers along the faces of the box (see dirac_oracle.h) */
static double potential_imag(const oracle_problem* p, const double x[3]) {
  double W = 0.0;
  if (p->abs_W != 0.0) {
    for (int a = 0; a < p->dims; ++a) {
      if (!((p->abs_axes >> a) & 1)) continue;
      double L = p->N[a] * p->dx[a];
      double d = x[a] < L - x[a] ? x[a] : L - x[a];
      if (d < p->abs_width) {
        double u = 1.0 - d / p->abs_width;
        W += u * u;
      }
    }
  }
  return p->V0_imag - p->abs_W * W;
}

/* scalar potential V(x, t) at half-lattice point f (complex: Sect. 3,
   growth factors) */
static cplx potential(const oracle_problem* p, const double* V_fine, long f, const double x[3],
                      double t) {
  double V = p->V0;
  if (p->step_axis >= 0 && p->step_axis < p->dims && x[p->step_axis] > p->step_x0) V += p->step_V;
  if (p->sc_Z != 0.0) {
    double r2 = 0.0;
    for (int a = 0; a < p->dims; ++a) {
      double d = x[a] - p->sc_c[a];
      r2 += d * d;
    }
    V -= p->sc_Z / sqrt(r2 + p->sc_a * p->sc_a);
  }
  if (V_fine) V += V_fine[f] * (1.0 + p->Vmod_amp * cos(p->Vmod_omega * t));
  return V + I * potential_imag(p, x);
}

static int has_vector_potential(const oracle_problem* p) {
  return p->A_const[0] != 0.0 || p->A_const[1] != 0.0 || p->A_const[2] != 0.0 || p->Apw_amp != 0.0 ||
         p->A_links != NULL;
}

/* Line integral of component a of the vector potential along the link of
   length h in direction a whose midpoint is y, at time t (Sect. 4: the
   Peierls phase is q times the line integral of A).  The constant part
   gives A_a h; the plane wave amp cos(k.x - w t + phase) gives, along a,
   amp h cos(k.y - w t + phase) sin(k_a h/2) / (k_a h/2). */
static double vector_potential_integral(const oracle_problem* p, int a, const double y[3], double h,
                                        double t) {
  double integral = p->A_const[a] * h;
  if (p->Apw_amp != 0.0 && p->Apw_pol == a) {
    double ph = -p->Apw_omega * t + p->Apw_phase;
    for (int b = 0; b < p->dims; ++b) ph += p->Apw_k[b] * y[b];
    double u = 0.5 * p->Apw_k[a] * h;
    double sinc = u == 0.0 ? 1.0 : sin(u) / u;
    integral += p->Apw_amp * h * cos(ph) * sinc;
  }
  return integral;
}

/* The difference part of one update at half-lattice point (X,Y,Z):
     S = sum_a  c_a r_a [ U+ psi(x + dx_a/2 e_a) - U- psi(x - dx_a/2 e_a) ],
   r_a = dt/dx_a, c_x = 1, c_y = -i (p=0: A,C,u) or +i (p=1: B,D,v),
   c_z = +1 (p=0) or -1 (p=1)  (Eqs. ss1-ss4; scheme2Deq-scheme4thline),
   and U+- the Peierls link factors evaluated at time t (Sect. 4). */
static cplx stencil(const oracle_problem* p, const grid* g, const cplx* psi, long X, long Y, long Z,
                    double t) {
  long C[3] = {X, Y, Z};
  int pb = (int)((X + Y) & 1);
  cplx coeff[3];
  coeff[0] = 1.0;
  coeff[1] = pb ? I : -I;
  coeff[2] = pb ? -1.0 : 1.0;
  int links = has_vector_potential(p);
  double xs[3];
  if (links) position(p, X, Y, Z, xs);
  cplx S = 0.0;
  for (int a = 0; a < p->dims; ++a) {
    long Cp[3] = {C[0], C[1], C[2]}, Cm[3] = {C[0], C[1], C[2]};
    Cp[a] = wrap(C[a] + 1, g->M[a]);
    Cm[a] = wrap(C[a] - 1, g->M[a]);
    cplx up = psi[fine_index(g, Cp[0], Cp[1], Cp[2])];
    cplx dn = psi[fine_index(g, Cm[0], Cm[1], Cm[2])];
    if (links) {
      double h = p->dx[a] / 2.0;
      double yp[3] = {xs[0], xs[1], xs[2]}, ym[3] = {xs[0], xs[1], xs[2]};
      yp[a] += h / 2.0;
      ym[a] -= h / 2.0;
      double phi_p = p->q * vector_potential_integral(p, a, yp, h, t);
      double phi_m = p->q * vector_potential_integral(p, a, ym, h, t);
      if (g->link[a]) {  /* own link upwards, the lower neighbour's link to this point */
        double mod = 1.0 + p->Alink_amp * cos(p->Alink_omega * t);
        phi_p += p->q * mod * g->link[a][fine_index(g, C[0], C[1], C[2])];
        phi_m += p->q * mod * g->link[a][fine_index(g, Cm[0], Cm[1], Cm[2])];
      }
      up = up * cexp(-I * phi_p);
      dn = dn * cexp(I * phi_m);
    }
    double r = p->dt / p->dx[a];
    S += coeff[a] * (r * (up - dn));
  }
  return S;
}

static int is_upper(long X, long Y, long Z) { return ((X + Y + Z) & 1) == 0; }

/* update every point of one parity (upper: beta = +1, lower: beta = -1) */
static void half_step(const oracle_problem* p, const grid* g, cplx* psi, const double* V_fine,
                      int upper, double t) {
  double beta = upper ? 1.0 : -1.0;
#pragma omp parallel for schedule(static)
  for (long ZY = 0; ZY < g->M[2] * g->M[1]; ++ZY) {
    long Z = ZY / g->M[1], Y = ZY % g->M[1];
    for (long X = 0; X < g->M[0]; ++X) {
      if (is_upper(X, Y, Z) != upper) continue;
      long f = fine_index(g, X, Y, Z);
      double x[3];
      position(p, X, Y, Z, x);
      cplx th = p->dt * (beta * p->m + potential(p, V_fine, f, x, t)) / 2.0;
      cplx S = stencil(p, g, psi, X, Y, Z, t);
      psi[f] = ((1.0 - I * th) * psi[f] - S) / (1.0 + I * th);
    }
  }
}

void oracle_step(const oracle_problem* p, double* planes, double t0, long nsteps) {
  grid g = make_grid(p);
  cplx* psi = (cplx*)malloc((size_t)g.n * sizeof(cplx));
  double* V_fine = real_planes_to_fine(p, &g, p->V_site);
  links_to_fine(p, &g);
  planes_to_fine(p, &g, planes, psi);
  double t = t0;
  for (long s = 0; s < nsteps; ++s) {
    half_step(p, &g, psi, V_fine, 1, t);             /* A,B (u): t-dt/2 -> t+dt/2 */
    half_step(p, &g, psi, V_fine, 0, t + p->dt / 2); /* C,D (v): t -> t+dt */
    t = t0 + (double)(s + 1) * p->dt;
  }
  fine_to_planes(p, &g, psi, planes);
  free(V_fine);
  free_links(&g);
  free(psi);
}

/*
 * Conserved functional.  The Lemma of Sect. 2 (Eq. EPM) reads, with the
 * scalar product (F,G) = sum F G* and the differences delta_i,
 *     E = sum |psi|^2 - Re sum_{upper} conj(F) S_F(lower),
 * i.e. the cross terms pair every upper value with the difference part of its
 * own update.  Summation by parts turns this into the "lower" form
 *     E = sum |psi|^2 + Re sum_{lower} conj(G) S_G(upper),
 * equal for time-independent vector potentials.  In (2+1)D the lower form is
 * ||u||^2 + ||v||^2 + r Re (delta_+ u, v): the Lemma of Sect. 3 prints
 * delta_- u, but its own proof multiplies Eq. scheme2ndline, whose difference
 * is delta_x u + i delta_y u = delta_+ u; with delta_- the functional is not
 * conserved by the scheme as printed (pinned by a test).
 * The lower form is evaluated with link factors at the upper sheet's time
 * t - dt/2, the upper form at the lower sheet's time t, matching the
 * half-steps that produced the stored values.
 */
void oracle_observables(const oracle_problem* p, const double* planes, double t, double out[3]) {
  grid g = make_grid(p);
  cplx* psi = (cplx*)malloc((size_t)g.n * sizeof(cplx));
  links_to_fine(p, &g);
  planes_to_fine(p, &g, planes, psi);
  double naive = 0.0, cross_lower = 0.0, cross_upper = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : naive, cross_lower, cross_upper)
  for (long ZY = 0; ZY < g.M[2] * g.M[1]; ++ZY) {
    long Z = ZY / g.M[1], Y = ZY % g.M[1];
    for (long X = 0; X < g.M[0]; ++X) {
      long f = fine_index(&g, X, Y, Z);
      cplx v = psi[f];
      naive += creal(v) * creal(v) + cimag(v) * cimag(v);
      if (is_upper(X, Y, Z)) {
        cplx S = stencil(p, &g, psi, X, Y, Z, t);
        cross_upper += creal(conj(v) * S);
      } else {
        cplx S = stencil(p, &g, psi, X, Y, Z, t - p->dt / 2);
        cross_lower += creal(conj(v) * S);
      }
    }
  }
  out[0] = naive + cross_lower;
  out[1] = naive - cross_upper;
  out[2] = naive;
  free_links(&g);
  free(psi);
}

double oracle_partial_density(const oracle_problem* p, const double* planes, int axis, double x0) {
  grid g = make_grid(p);
  cplx* psi = (cplx*)malloc((size_t)g.n * sizeof(cplx));
  planes_to_fine(p, &g, planes, psi);
  double sum = 0.0;
#pragma omp parallel for schedule(static) reduction(+ : sum)
  for (long ZY = 0; ZY < g.M[2] * g.M[1]; ++ZY) {
    long Z = ZY / g.M[1], Y = ZY % g.M[1];
    for (long X = 0; X < g.M[0]; ++X) {
      double x[3];
      position(p, X, Y, Z, x);
      if (x[axis] > x0) {
        cplx v = psi[fine_index(&g, X, Y, Z)];
        sum += creal(v) * creal(v) + cimag(v) * cimag(v);
      }
    }
  }
  free(psi);
  return sum;
}

int oracle_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
