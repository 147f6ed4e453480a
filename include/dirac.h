/*
 * libdirac -- GB300 (sm_103a) CUDA implementation of the single-cone
 * staggered space-time leap-frog scheme for the time-dependent Dirac equation
 * (R. Hammer, W. Poetz, A. Arnold, arXiv:1309.3452).
 *
 * The scheme (Sect. 2, Eqs. sbegin-send, compact form Eq. 3+3Ddis and
 * Eqs. ss1-ss4; Sect. 3, Eqs. scheme2Deq-scheme4thline) places each spinor
 * component on its own sublattice of a grid staggered in space and time and
 * advances it explicitly:  the "upper" components (A, B in (3+1)D; u in
 * (2+1)D) go from t - dt/2 to t + dt/2 using centred differences of the
 * "lower" ones (C, D; v) at t, then the lower components go from t to t + dt
 * using the new upper values.  Mass and scalar potential enter through the
 * time average of Eq. 3+3Ddis (a per-site Cayley factor), the vector
 * potential through Peierls link factors (Sect. 4).
 *
 * Units: hbar = c = 1.  Lengths dx[a] = Delta_a, time step dt = Delta_t,
 * r_a = dt / dx[a].  Periodic boundaries in units of the cell.
 *
 * ---------------------------------------------------------------------------
 * Canonical host layout (dirac_set_spinor / dirac_get_spinor)
 *   double[P][Nz][Ny][Nx][2]   (complex128, re then im; x fastest)
 *   (3+1)D: P = 8 planes  A0 A1 B0 B1 C0 C1 D0 D1
 *   (2+1)D: P = 4 planes  u0 u1 v0 v1  (Nz = 1)
 * For cell j = (jx, jy, jz) the planes hold the values at positions
 * (grid definitions of Sect. 2; fcr-u / fcr-v of Sect. 3)
 *   A0  j dx                 A1  (j + (1/2,1/2,0)) dx
 *   B0  (j + (1/2,0,1/2)) dx B1  (j + (0,1/2,1/2)) dx
 *   C0  (j + (0,0,1/2)) dx   C1  (j + (1/2,1/2,1/2)) dx
 *   D0  (j + (1/2,0,0)) dx   D1  (j + (0,1/2,0)) dx
 *   u0 = A0, u1 = A1, v0 = D0, v1 = D1 without z.
 * Upper planes (A, B, u) hold their values at time t - dt/2, lower planes
 * (C, D, v) at time t, where t is the simulation time (dirac_get_time).
 * One real per site (the optional static potential) uses the same layout
 * without the trailing [2].
 *
 * Ownership: the library allocates and owns all device memory of a
 * simulation; host buffers belong to the caller and are never retained (a
 * page-locked buffer given to dirac_set_spinor is read when the stream gets
 * there, see that call).
 *
 * Errors: every call returns a dirac_status; no exception or abort crosses
 * the ABI.  On failure dirac_last_error() describes the cause.  A CUDA error
 * leaves the simulation in an unspecified state (destroy it).
 *
 * Streams: all device work of a simulation runs on the stream given at
 * creation (NULL = the legacy default stream).  dirac_step, dirac_batch_step
 * and dirac_set_spinor(_device) only enqueue work; dirac_norm,
 * dirac_partial_density, dirac_get_spinor, dirac_check, dirac_autotune and
 * dirac_set_plan synchronise the stream before returning.
 *
 * Environment switches (read when the call runs; for comparisons and tests,
 * results stay within the FP32 tolerances):
 *   DIRAC_NO_GRAPHS             step loops as plain launches, no CUDA graphs
 *   DIRAC_NO_FUSED_NORM         dirac_norm always reduces the stored state
 *   DIRAC_NO_TEMPORAL_BLOCKING  (2+1)D FP32: one time step per pass
 *   DIRAC_HOST_COPY=staged      dirac_set_spinor / dirac_get_spinor of FP32
 *                               simulations copy page-locked buffers through a
 *                               device staging plane instead of converting them
 *                               in place
 *   DIRAC_SOFTCORE              (read by dirac_create) how the FP32 kernels
 *                               evaluate a soft-core potential's Cayley
 *                               coefficients: "analytic" (default; compensated
 *                               FP32 per value, no table), "corrected" (an FP32
 *                               estimate plus a 4-byte tabulated correction per
 *                               value) or "table" (16 bytes per value)
 * ---------------------------------------------------------------------------
 */
#ifndef DIRAC_H
#define DIRAC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct dirac_sim dirac_sim;

typedef enum {
  DIRAC_OK = 0,
  DIRAC_ERR_INVALID = 1,     /* bad argument (NULL pointer, dims, N < 2, dx <= 0, ...) */
  DIRAC_ERR_UNSTABLE = 2,    /* r_x^2 + r_y^2 (+ r_z^2) > 1 (Sect. 2.2 / Sect. 3 bound) */
  DIRAC_ERR_OOM = 3,         /* device allocation failed */
  DIRAC_ERR_CUDA = 4,        /* a CUDA call or kernel launch failed */
  DIRAC_ERR_DIVERGED = 5,    /* the functional became non-finite (dirac_norm) or a
                                stability check failed (dirac_check) */
  DIRAC_ERR_TIMEOUT = 6,     /* reserved for bounded device waits (no kernel of this
                                library waits on another, so none is returned) */
  DIRAC_ERR_UNSUPPORTED = 7  /* valid request this library does not implement */
} dirac_status;

typedef enum {
  DIRAC_FP64 = 0, /* complex128 state, FP64 arithmetic (validation mode) */
  DIRAC_FP32 = 1  /* complex64 state, FP32 stencil with compensated (hi+lo)
                     coefficients; FP64 reductions */
} dirac_precision;

/* flags for dirac_create */
#define DIRAC_FLAG_ALLOW_UNSTABLE 0x1u   /* accept r beyond the stability bound */
#define DIRAC_FLAG_REFERENCE_KERNELS 0x2u /* FP32: use the plain one-kernel-per-half-step
                                             path instead of the fused time-step kernel
                                             (same per-value arithmetic, same results);
                                             (3+1)D grids of 2^31 cells or more always
                                             take this path */

/*
 * External fields (Sect. 2: V in Eq. 3+3D; Sect. 4: vector potential).
 * Scalar potential, evaluated at every site's own position x:
 *   V(x,t) = V0
 *          + step_V * H(x[step_axis] - step_x0)        (Klein step, Sect. 5;
 *                                                        step_axis < 0: none)
 *          - sc_Z / sqrt(|x - sc_center|^2 + sc_a^2)    (soft core; sc_Z = 0: none)
 *          + V_static(x) * (1 + Vmod_amp * cos(Vmod_omega * t))
 * Vector potential, coupled with charge q through link factors:
 *   A(x,t) = A_const + e_{Apw_pol} * Apw_amp * cos(Apw_k . x - Apw_omega t + Apw_phase)
 * plus, optionally, an arbitrary A given by its line integrals (Sect. 4: the
 * Peierls phase of a link is q times the integral of A along it):
 *   A_links[(a * P + plane) * cells + cell], a < dims, P planes, canonical
 *   layout = integral of A_a along the link from that value's point x to
 *   x + (dx_a/2) e_a (the value's neighbour on the partner plane; at the far
 *   face the link wraps to the periodic image), multiplied at time t by
 *   1 + Alink_amp * cos(Alink_omega * t).
 * A must be periodic on the box for the link factors at the wrap to be
 * consistent.  A_links: NULL or a host array of dims * P * cells reals, copied
 * during dirac_create.  Link factors: a constant A, and a plane wave whose
 * wave vector lies along one axis other than its polarisation, need no
 * per-value data.  Any other A that does not change in time (Apw_omega = 0
 * or Apw_amp = 0; Alink_omega = 0 or Alink_amp = 0) has its factors
 * exp(-i phi) tabulated once per simulation for DIRAC_FP32 (FP64 phases,
 * hi + lo float pairs); otherwise they are evaluated per site in FP64.
 * dirac_norm_noalloc does not take A_links.  The upper
 * half-step uses the fields at time t, the lower half-step at t + dt/2 (the
 * time sheets of Eqs. ss1-ss4).
 * V_static: NULL, or a host array of one real per site (canonical layout);
 * it is copied during dirac_create.
 * Imaginary part of V (Sect. 3, growth factors: Im V < 0 damps, so layers of
 * negative Im V near the faces absorb outgoing waves):
 *   Im V(x) = V0_imag - abs_W * sum_{a in abs_axes} w(d_a),
 *   d_a = min(x_a, N_a dx_a - x_a), w(d) = (1 - d/abs_width)^2 for
 *   d < abs_width, else 0; abs_axes is a bit mask of axes (bit a = axis a).
 * abs_W != 0 needs abs_width > 0 and a non-empty mask of the grid's axes
 * (else DIRAC_ERR_INVALID).  With any Im V the functional E is no longer
 * conserved; with Im V <= 0 it does not grow.
 */
typedef struct {
  double V0;
  int step_axis;
  double step_x0, step_V;
  double sc_Z, sc_a, sc_center[3];
  const double* V_static;
  double Vmod_amp, Vmod_omega;
  double q;
  double A_const[3];
  double Apw_amp, Apw_k[3], Apw_omega, Apw_phase;
  int Apw_pol;
  double V0_imag;
  double abs_W, abs_width;
  int abs_axes;
  const double* A_links;
  double Alink_amp, Alink_omega;
} dirac_fields;

/* Zero fields: everything 0 except q = 1, step_axis = -1, sc_a = 1 (no
   imaginary part, no layers, no link integrals). */
void dirac_fields_default(dirac_fields* f);

/*
 * Create a simulation of the (dims+1)D scheme on an N[0] x N[1] (x N[2])
 * periodic grid of unit cells (each cell carries two sites of every
 * component), lattice constants dx[], time step dt, mass m.  fields may be
 * NULL (free particle).  Rejects N[a] < 2, dx[a] <= 0, dt <= 0, a NaN or an
 * infinity in any real parameter of fields (DIRAC_ERR_INVALID) and (unless
 * DIRAC_FLAG_ALLOW_UNSTABLE) sum_a (dt/dx[a])^2 > 1.  cuda_stream is a
 * cudaStream_t (may be NULL).  The state starts at zero with t = 0.
 * On success *out owns the simulation; free it with dirac_destroy.
 */
dirac_status dirac_create(dirac_sim** out, int dims, const int N[3], const double dx[3], double dt,
                          double m, const dirac_fields* fields, dirac_precision precision,
                          unsigned flags, void* cuda_stream);

/* Copy a full state in the canonical host layout (complex128) into the
   simulation (converted to the simulation's precision on the device).  The
   copies are enqueued on the simulation's stream: a pageable host buffer may
   be reused as soon as the call returns, a page-locked one only once the
   stream has passed this point (any synchronising call).  FP32: a
   page-locked, device-mapped buffer (cudaHostAlloc / pinned memory; every
   byte of the state's range page-locked, 16-byte aligned) is read in place
   by the conversion kernels, without a copy-engine pass; anything else goes
   through a device staging plane, one plane at a time.  The functional of
   the new state is reduced on the device as the reference of dirac_check
   (two more launches, no synchronisation). */
dirac_status dirac_set_spinor(dirac_sim* sim, const double* host);

/* Copy the current state out in the canonical host layout (complex128);
   synchronises the stream.  FP32: a page-locked, device-mapped buffer (as for
   dirac_set_spinor) is written in place by the conversion kernels. */
dirac_status dirac_get_spinor(dirac_sim* sim, double* host);

/* As dirac_set_spinor / dirac_get_spinor, but the canonical complex128
   state lives in device memory owned by the caller (same layout; 16-byte
   aligned).  Both only enqueue work on the simulation's stream; the caller's
   buffer must stay valid until that work has run. */
dirac_status dirac_set_spinor_device(dirac_sim* sim, const void* dev);
dirac_status dirac_get_spinor_device(dirac_sim* sim, void* dev);

/* Enqueue nsteps full time steps (both half-steps each; Eq. 3+3Ddis);
   t advances by nsteps*dt.  nsteps >= 0. */
dirac_status dirac_step(dirac_sim* sim, long nsteps);

/*
 * Advance several simulations by nsteps time steps each, together.  FP32
 * simulations with time-independent fields (no modulated static potential,
 * no moving plane wave; a static soft core or static array is not batched
 * either) that share dims and field path run as ONE persistent launch of the
 * fused kernel per time step ((2+1)D: per two time steps, with a single-step
 * pass for an odd remainder): the work items of all of them (tile x level
 * chunk) are dealt to the resident blocks together, so small grids fill the
 * GPU jointly.  Other simulations are stepped one after another as by
 * dirac_step.  The result of every simulation is identical, bit for bit, to
 * stepping it alone.  All simulations must have been created with the same
 * stream (else DIRAC_ERR_INVALID).  The call enqueues the work; its small
 * argument tables are copied synchronously before it returns.  Loops of up
 * to 256 launches are recorded as a CUDA graph, kept with their argument
 * tables (at most eight, least recently used evicted) and replayed when the
 * same simulations, in the same buffer state, with the same plans and step
 * count come back; dirac_destroy forgets the loops that name a simulation.
 * On failure dirac_last_error(NULL) describes the cause.
 */
dirac_status dirac_batch_step(dirac_sim* const* sims, int nsims, long nsteps);

/*
 * Conserved functional of the stored state (Lemma of Sect. 2, Eq. EPM, and
 * Lemma of Sect. 3), written with every lower value G paired with the
 * difference part S_G of its own update:
 *   E = sum |psi|^2 + Re sum_{lower sites} conj(G) S_G(upper),
 *   S_G = r_x dx(G) + s_y r_y dy(G) + s_z r_z dz(G)   (Eqs. ss3, ss4),
 * with link factors at the upper sheet's time t - dt/2.  Equal to Eq. EPM by
 * summation by parts for time-independent A.  In (2+1)D this is
 * ||u||^2 + ||v||^2 + r Re (delta_+ u, v); Sect. 3 prints delta_- u, which
 * the scheme as printed does not conserve.
 * *naive (may be NULL) receives sum |psi|^2 over all values (Sect. 3: the
 * naive norm, conserved only on average).  Accumulated in FP64 in a fixed
 * order (deterministic).  Synchronises the stream.
 * Returns DIRAC_ERR_DIVERGED if E is not finite.
 */
dirac_status dirac_norm(dirac_sim* sim, double* E, double* naive);

/* sum of |psi|^2 over the values whose position along axis exceeds x0
   (transmitted probability for the Klein step, Sect. 5).  x0 must be finite
   (else DIRAC_ERR_INVALID); beyond the box the sum is 0 or everything.
   Synchronises. */
dirac_status dirac_partial_density(dirac_sim* sim, int axis, double x0, double* out);

/* simulation time t of the lower sheet (upper planes are at t - dt/2) */
dirac_status dirac_get_time(const dirac_sim* sim, double* t);
dirac_status dirac_set_time(dirac_sim* sim, double t);

/* number of CUDA kernels this simulation has launched since creation
   (every launch of every call counts once) */
long long dirac_kernel_launches(const dirac_sim* sim);

/*
 * Launch plan of a simulation's FP32 fused kernels (the paper has no
 * counterpart: it only fixes what one time step computes, not how the work
 * is cut).  Plans change the speed only, never a value of the state; the
 * conserved functional fused into a call's last step is summed in another
 * order and may differ in the last bits.
 *   chunk       z levels ((3+1)D) or y rows ((2+1)D) per work item of the
 *               one-step kernel; 0 = the built-in rule
 *   two_step    (2+1)D: 1 = two time steps per pass whenever the fields do
 *               not depend on time (the default), 0 = one step per pass
 *   chunk2      rows per work item of the two-step kernel; 0 = the rule
 *   us_per_step time per step that dirac_autotune measured for this plan
 *               (0 when it was not measured)
 */
typedef struct {
  int chunk;
  int two_step;
  int chunk2;
  double us_per_step;
} dirac_plan;

/* current plan of sim (a zero plan for DIRAC_FP64 and reference-kernel
   simulations, which have none) */
dirac_status dirac_get_plan(const dirac_sim* sim, dirac_plan* out);

/* Set the plan (us_per_step is ignored).  DIRAC_ERR_INVALID for a negative
   chunk or chunk2, a chunk beyond the marching extent (N[2] in (3+1)D, N[1]
   in (2+1)D), two_step other than 0/1 or two_step in (3+1)D, or any
   non-zero plan on a simulation without fused kernels.  Synchronises the
   simulation's stream (recorded step graphs are rebuilt). */
dirac_status dirac_set_plan(dirac_sim* sim, const dirac_plan* plan);

/*
 * Autotuner: time the candidate plans of this simulation's fused kernels on
 * its current state (the best chunk lengths by the built-in model, for one-
 * and, in (2+1)D with time-independent fields, two-step passes), keep the
 * fastest, remember it for later simulations with the same grid, field path
 * and device (dirac_create applies a remembered plan), and copy it to *out
 * (may be NULL).  The state and the time are unchanged; the spare state
 * buffer is overwritten.  Synchronises the simulation's stream.  A
 * simulation without fused kernels keeps its zero plan (DIRAC_OK).
 */
dirac_status dirac_autotune(dirac_sim* sim, dirac_plan* out);

/*
 * Stability diagnostics (Props. 2 and 4, Sect. 2.2 and Sect. 3).
 *
 * dirac_functional_bounds: constants lo, hi with
 *     lo * sum|psi|^2 <= E <= hi * sum|psi|^2   for every state,
 * E the conserved functional.  Without a vector potential, or with a
 * constant one, lo = 1 - rho and hi = 1 + rho, rho = sqrt(sum_a (dt/dx_a)^2)
 * (the cross term of E is, per lattice momentum k, a Hermitian 2x2 block
 * pattern whose largest singular value is rho; the bounds are attained at the
 * zone corner) - a sharpened form of the paper's estimate.  With any other
 * vector potential the paper's estimate itself: lo = 1 - sum_a dt/dx_a,
 * hi = 1 + sum_a dt/dx_a.  lo <= 0 means E bounds nothing (beyond the
 * stability limit, or too coarse an estimate).  Host only: no device work.
 * general_A: 0 = no or constant vector potential, 1 = any other.
 */
void dirac_functional_bounds(int dims, const double dx[3], double dt, int general_A, double* lo,
                             double* hi);

/* Result of dirac_check.  E_ref and naive_ref are taken from the state set
   by the last dirac_set_spinor / dirac_set_spinor_device (NaN before any). */
typedef struct {
  double E, naive;          /* now (as dirac_norm) */
  double E_ref, naive_ref;  /* at the last set_spinor */
  double drift;             /* (E - E_ref) / |E_ref| */
  double lower, upper;      /* bounds on naive implied by E: E/hi <= naive <= E/lo
                               (0 and +inf where no bound applies) */
  unsigned failed;          /* DIRAC_CHECK_* bits of the checks that failed */
} dirac_check_report;
#define DIRAC_CHECK_NONFINITE 0x1u /* E or the naive norm is not finite */
#define DIRAC_CHECK_BOUND 0x2u     /* the naive norm is outside [lower, upper] */
#define DIRAC_CHECK_DRIFT 0x4u     /* |drift| > tol for a conserving field set (real V, no
                                      time-dependent A), or drift > tol with Im V <= 0 */

/*
 * Check the invariants the paper proves for the current state: E finite, E
 * conserved (real V and static A) or not growing (Im V <= 0 everywhere), and
 * sum|psi|^2 within the bounds that E implies (dirac_functional_bounds;
 * relative slack 1e-10 for the rounding of the sums).  Synchronises.  Fills
 * *out (may be NULL) and returns DIRAC_ERR_DIVERGED when a check failed,
 * DIRAC_OK otherwise.  Costs one dirac_norm (no pass over the state right
 * after a dirac_step of the FP32 fused path, whose last step accumulates E).
 */
dirac_status dirac_check(dirac_sim* sim, double tol, dirac_check_report* out);

/* Algorithmic HBM bytes of one site update (one cell advanced one full time
   step) on this simulation's path: every value read and written once, plus
   a per-site coefficient (16 bytes) or static potential (8 bytes) read per
   value where the potential needs one, and the vector potential's per-value
   link data where it has some: two tabulated link factors (32 bytes) per axis
   and value, or two link integrals (16 bytes) per axis and value on the
   per-site path.  The roofline numerator of a time step.  0 for NULL. */
double dirac_algorithmic_bytes(const dirac_sim* sim);

/* device bytes a simulation of this shape and precision allocates for a
   potential made of V0 and a Klein step only: the state, plus for
   DIRAC_FP32 a second state buffer and one complex128 conversion plane.
   Other potentials add one double per value (DIRAC_FP64, or a time-
   dependent static array) or the coefficient table, 16 bytes per value
   (DIRAC_FP32, time-independent), A_links 16 bytes per axis and value, a
   tabulated static vector potential (DIRAC_FP32) 32 bytes per axis and
   value, and every simulation a few KiB of reduction scratch. */
size_t dirac_state_bytes(int dims, const int N[3], dirac_precision precision);

/* human-readable description of the last failure on sim (or, when sim is
   NULL, of the calling thread's last failed dirac_create / dirac_batch_step) */
const char* dirac_last_error(const dirac_sim* sim);

/* free all device memory of sim (NULL is ignored); synchronises its stream */
void dirac_destroy(dirac_sim* sim);

/*
 * dirac_norm_noalloc: the value of dirac_norm for a state held in the
 * caller's own device memory, computed without allocating any memory.
 * The paper has no counterpart; this entry point exists for callers that
 * cannot call cudaMalloc where they need the norm: a host framework that
 * owns all device memory through its own pool and forbids other
 * allocations, or a time-critical loop that cannot afford the implicit
 * device synchronisation of cudaMalloc/cudaFree.  Such callers cannot hold a
 * dirac_sim (dirac_create allocates), so this call takes the planes directly.
 *
 * planes: dims == 3 ? 8 : 4 device pointers, in the plane order of the
 *   canonical layout (A0..D1 or u0..v1), each an N[0] x N[1] (x N[2]) array
 *   [z][y][x] of double2 (DIRAC_FP64) or float2 (DIRAC_FP32), owned and kept
 *   alive by the caller.  t is the time of the lower sheet (link factors of a
 *   vector potential are taken at t - dt/2, as in dirac_norm); fields may be
 *   NULL (only the vector potential matters for the functional).
 * out_dev: caller-owned device memory for two doubles, written with
 *   {E, sum |psi|^2}.  The call only enqueues work on cuda_stream (may be
 *   NULL); synchronise that stream before reading out_dev.
 * Scratch: the per-block partial sums go to one fixed array in the library's
 *   device memory (8193 x 5 doubles, about 320 KiB, held by every GPU that
 *   loads the library until the process exits).  Grids whose reduction needs
 *   more than 8192 blocks, i.e. ceil(N[0]/32) * ceil(N[1]/8) > 8192, are
 *   rejected with DIRAC_ERR_UNSUPPORTED before any device work, and so are
 *   fields with A_links (their device copy would be an allocation).  Every call
 *   shares that array and overwrites all of it that it reads, so nothing
 *   needs clearing between calls; calls that overlap on the GPU (other
 *   streams, or another host thread) race on it and must be serialised by
 *   the caller.
 * Set-up: every call looks up the array's address on the current device
 *   (cudaGetSymbolAddress, which allocates nothing), so a device reset or a
 *   new context never leaves a stale address behind.  The first call on a
 *   device may load the library's device code there; make that first call
 *   before any stream capture.
 * Returns DIRAC_ERR_INVALID for bad arguments (including non-finite q,
 *   A_const or plane-wave parameters, and a plane wave whose Apw_pol is not
 *   an axis of the grid, as dirac_create rejects them), DIRAC_ERR_CUDA if the
 *   address lookup or a launch fails.
 */
dirac_status dirac_norm_noalloc(int dims, const int N[3], const double dx[3], double dt, double t,
                                const dirac_fields* fields, dirac_precision precision,
                                const void* const* planes, double* out_dev, void* cuda_stream);

/*
 * Sub-domain decomposition (Sect. 6: the scheme is parallelised by spatial
 * sub-domains that exchange their boundary values).  A grid is split along
 * its marching axis (z in (3+1)D, y in (2+1)D) into nslabs slabs of
 * consecutive levels (dirac_slab_partition); every slab is stepped by the
 * fused one-step kernel as its own sub-domain, which stores one halo level on
 * either side, and after every time step each slab's first and last own
 * levels are copied into its neighbours' halo levels (periodic).  Fields are evaluated at every value's position on the
 * whole grid, so the stepped state equals, bit for bit, that of the whole
 * grid stepped as one simulation.  All slabs live on the calling device and
 * run on cuda_stream; the halo copies are device-to-device copies of one
 * level (Nx*Ny values in (3+1)D, Nx in (2+1)D) per plane and direction, the
 * data a multi-device split would exchange.
 *
 * dirac_slabs_create: as dirac_create for the whole grid N (FP32 only,
 *   1 <= nslabs <= N[2] in (3+1)D, N[1] in (2+1)D); fields given per site
 *   (V_static, A_links), absorbing layers and vector potentials that would
 *   need a per-site table (static A other than a constant or a plane wave
 *   across its polarisation) are not decomposed (DIRAC_ERR_UNSUPPORTED); a
 *   soft core is evaluated analytically; (2+1)D slabs take one time step per
 *   pass.
 * set/get_spinor: the whole grid in the canonical host layout (as
 *   dirac_set_spinor / dirac_get_spinor; get synchronises).
 * step: nsteps time steps of every slab, each followed by the halo exchange.
 * norm: E and the naive norm summed over the slabs' own values (synchronises).
 * dirac_slab_partition (host only): slab k of nslabs over Nz levels starts at
 *   level *z0 and has *nz levels; the first Nz mod nslabs slabs are one level
 *   longer.  Out-of-range arguments give *z0 = *nz = 0.
 * Errors: dirac_slabs_last_error (NULL: the last failed creation).
 */
typedef struct dirac_slabs dirac_slabs;
void dirac_slab_partition(int Nz, int nslabs, int k, int* z0, int* nz);
dirac_status dirac_slabs_create(dirac_slabs** out, int nslabs, int dims, const int N[3], const double dx[3],
                                double dt, double m, const dirac_fields* fields, dirac_precision precision,
                                unsigned flags, void* cuda_stream);
dirac_status dirac_slabs_set_spinor(dirac_slabs* g, const double* host);
dirac_status dirac_slabs_get_spinor(dirac_slabs* g, double* host);
dirac_status dirac_slabs_step(dirac_slabs* g, long nsteps);
dirac_status dirac_slabs_norm(dirac_slabs* g, double* E, double* naive);
dirac_status dirac_slabs_info(const dirac_slabs* g, int k, int* z0, int* nz);
dirac_status dirac_slabs_get_time(const dirac_slabs* g, double* t);
long long dirac_slabs_kernel_launches(const dirac_slabs* g);
const char* dirac_slabs_last_error(const dirac_slabs* g);
void dirac_slabs_destroy(dirac_slabs* g);

/* The current device's FP64 fused multiply-add rate in TFLOP/s (2 flops per
   FMA), measured by a kernel of independent FP64 FMA chains (a few ms; no
   memory traffic): the arithmetic ceiling the FP64 validation path is held
   against.  The paper has no counterpart.  Synchronises the device. */
dirac_status dirac_fp64_fma_rate(double* tflops);

/* ABI version: DIRAC_ABI_VERSION of the header the library was built with.
   A client checks it against the header it was compiled with; the version
   changes whenever a structure or a signature does (2: dirac_fields gained
   A_links, Alink_amp, Alink_omega). */
#define DIRAC_ABI_VERSION 2
int dirac_version(void);

#ifdef __cplusplus
}
#endif
#endif /* DIRAC_H */
