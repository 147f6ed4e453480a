/*
 * Oracle for the single-cone staggered space-time leap-frog scheme for the
 * Dirac equation (Hammer, Poetz, Arnold, "Single-cone real-space finite
 * difference scheme for the time-dependent Dirac equation", arXiv:1309.3452).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 CPU restatement of
 * the scheme used to check the CUDA library.  Only the tests, the smoke check
 * and the benchmark's CPU-baseline leg may load it; the library never does.
 * It shares no code, header, table or helper with the CUDA path.
 *
 * Formulation ("fine grid"): every spinor value of the paper's grid sits on a
 * point of the half-lattice (X,Y,Z) = 2*(x,y,z)/dx with integer X,Y,Z.
 *   (3+1)D, Sect. 2 grid (A,B,C,D sublattices):  p = (X+Y) mod 2, q = Z mod 2,
 *       A: p=0,q=0   D: p=1,q=0   C: p=0,q=1   B: p=1,q=1.
 *   (2+1)D, Sect. 3 grid (fcr-u / fcr-v):  u: X+Y even, v: X+Y odd.
 * Every half-lattice point carries exactly one value, the "upper" values
 * (A,B / u, on half-integer time sheets) are the points with X+Y+Z even and
 * the "lower" values (C,D / v, on integer time sheets) those with X+Y+Z odd.
 * One time step (Eqs. ss1-ss4, Eq. 3+3Ddis; Eqs. scheme2Deq-scheme4thline)
 * updates all upper points from their lower neighbours at fine distance 1,
 * then all lower points from the new upper values.
 *
 * The interface uses the canonical plane layout shared with the library's
 * API: planes [plane][z][y][x] of complex128 (interleaved re, im), planes
 * A0,A1,B0,B1,C0,C1,D0,D1 in (3+1)D and u0,u1,v0,v1 in (2+1)D, where for
 * cell j = (jx,jy,jz):
 *   A0 (j)          A1 (j+(1/2,1/2,0))   B0 (j+(1/2,0,1/2)) B1 (j+(0,1/2,1/2))
 *   C0 (j+(0,0,1/2)) C1 (j+(1/2,1/2,1/2)) D0 (j+(1/2,0,0))  D1 (j+(0,1/2,0))
 * (Sect. 2, grid definitions; Sect. 3 for u,v = A,D without z).  Upper planes
 * hold values at time t - dt/2, lower planes at time t.
 */
#ifndef DIRAC_ORACLE_H
#define DIRAC_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int dims;          /* 2 or 3 */
  int N[3];          /* unit cells per axis (N[2] ignored when dims == 2) */
  double dx[3];      /* lattice constants Delta_x, Delta_y, Delta_z (hbar = c = 1) */
  double dt;         /* time step Delta_t */
  double m;          /* mass (constant) */
  /* scalar potential V(x,t) = V0 + step + soft core + V_site*(1+Vmod_amp*cos(Vmod_omega*t)) */
  double V0;
  int step_axis;     /* Klein step V_step * H(x_axis - step_x0); axis < 0 disables */
  double step_x0, step_V;
  double sc_Z, sc_a; /* soft core -sc_Z / sqrt(|x-c|^2 + sc_a^2); sc_Z == 0 disables */
  double sc_c[3];
  const double* V_site; /* optional, one real per site in canonical plane layout */
  double Vmod_amp, Vmod_omega;
  /* vector potential A(x,t) = A_const + e_pol * Apw_amp*cos(k.x - Apw_omega*t + Apw_phase) */
  double q;
  double A_const[3];
  double Apw_amp, Apw_k[3], Apw_omega, Apw_phase;
  int Apw_pol;
  /* cell offset of this grid inside a larger one; positions are
     x_a = (X + 2*origin_a) * dx_a / 2.  Used for light-cone windows. */
  int origin[3];
  /* imaginary part of V (Sect. 3, growth factors: Im V < 0 damps):
     Im V(x) = V0_imag - abs_W * sum_{a in abs_axes} w(d_a),
     d_a = min(x_a, L_a - x_a) the distance to the box face along a
     (L_a = N_a dx_a of this grid; windows with origin != 0 must not use
     layers), w(d) = (1 - d/abs_width)^2 for d < abs_width, else 0;
     abs_axes is a bit mask of axes. */
  double V0_imag;
  double abs_W, abs_width;
  int abs_axes;
  /* an arbitrary vector potential given by its line integrals (Sect. 4):
     A_links[a * P * cells + plane * cells + cell] is the integral of A_a
     along the link from that value's point to its neighbour at +dx_a/2
     (P planes, canonical layout, a < dims), at time t scaled by
     1 + Alink_amp cos(Alink_omega t); added to the analytic A above; NULL:
     none */
  const double* A_links;
  double Alink_amp, Alink_omega;
} oracle_problem;

/* Advance the state in place by nsteps full time steps.  `planes` is the
   canonical layout; t0 is the time of the lower sheet on entry. */
void oracle_step(const oracle_problem* p, double* planes, double t0, long nsteps);

/* Observables of the stored state (lower sheet at time t):
   out[0] = E, the conserved functional in its "lower" form (see the .c file),
   out[1] = E in its "upper" form (the Lemma of Sect. 2 / Sect. 3 as printed,
            with the sign reading of the (2+1)D cross term noted there),
   out[2] = naive norm sum |psi|^2 over all values (Sect. 3). */
void oracle_observables(const oracle_problem* p, const double* planes, double t, double out[3]);

/* sum of |psi|^2 over values whose position along `axis` exceeds x0 */
double oracle_partial_density(const oracle_problem* p, const double* planes, int axis, double x0);

/* number of OpenMP threads the oracle runs with (1 without OpenMP) */
int oracle_threads(void);

#ifdef __cplusplus
}
#endif
#endif
