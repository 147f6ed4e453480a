// Kernel argument blocks and launcher declarations of libdirac.
#pragma once

#include "common.cuh"

namespace dirac {

// One half-step (all upper or all lower values) of the scheme, one kernel.
template <class P>
struct HalfStepArgs {
  typename P::cplx* pl[8];  // plane base pointers (updated in place)
  int N[3];
  long long pstride;
  int iso;                  // r_x = r_y (= r_z)
  typename P::Ratio ry, rz; // r_y/r_x, r_z/r_x
  HalfFields<P> h;
  FieldDesc f;
  int general;              // per-site FP64 field paths needed
};

template <class P, int DIMS>
void launch_half_step(const HalfStepArgs<P>& a, bool upper, cudaStream_t s);

// One full time step (both half-steps) in one kernel, out of place.
template <class P>
struct FusedArgs {
  const typename P::cplx* in[8];
  typename P::cplx* out[8];
  int N[3];
  int chunk;                // levels (z in (3+1)D, y in (2+1)D) per work item
  int workers;              // persistent workers: blocks ((3+1)D) or warps ((2+1)D)
  long long pstride;
  int iso;
  typename P::Ratio ry, rz;
  HalfFields<P> hu, hl;     // upper / lower half-step fields
  FieldDesc f;
  // non-null: accumulate the conserved functional of the new state (per block
  // [sum |psi|^2, Re sum_lower conj(G) S'_G]; E = first + r_x second)
  double* e_partials;
  // levels along the marching axis ((3+1)D: z, (2+1)D: y): the kernel updates
  // the nzu levels zlo .. zlo + nzu - 1 of the N[axis] stored ones; a level k
  // lies at global level (zorg + k) mod Nzg, where every field is evaluated.
  // A whole grid: zlo = 0, nzu = Nzg = N[axis], zorg = 0 (periodic wrap of
  // the stored levels); a slab of a decomposed grid: its own levels between
  // one halo level on either side (zlo = 1, nzu = N[axis] - 2), zorg = its
  // first global level - 1.  (The two-step (2+1)D kernel and the batched
  // kernels take whole grids only.)
  int zlo, nzu, zorg, Nzg;
};
constexpr int kFusedEMaxBlocks = 4096;  // capacity of the per-block E partials
// (2+1)D fused kernel geometry
constexpr int kFused2dWarps = 8;   // independent x strips per block
constexpr int kCore = 30;          // interior lanes of a 32-lane strip

// returns the number of blocks launched
template <class P, int DIMS>
int launch_fused(const FusedArgs<P>& a, cudaStream_t s);

// Two time steps per pass of the (2+1)D fused kernel (fields without time
// dependence: uniform / Klein-step / soft-core coefficients, no or constant
// links).  Returns the number of blocks launched, or 0, launching nothing,
// for other field paths.
int launch_fused2d_tb2(const FusedArgs<F32>& a, cudaStream_t s);

// Several simulations (same dims and time-independent field modes) in one
// persistent launch of the fused kernels.
template <class P>
struct BatchArgs {
  const FusedArgs<P>* sims;      // device array, one entry per simulation (chunk set)
  const long long* first_item;   // device array [nsims + 1]: prefix sums of the items
  int nsims;
  int workers;                   // set by the launcher
};
// levels per work item and number of items the fused kernels use for a grid
// (a FusedArgs chunk of 0 makes the launchers take fused_chunk's rule)
int fused_chunk(int dims, const int N[3]);
// chunk lengths worth timing, best first by the planner's model, for the
// one-step kernels or (two_step, (2+1)D) the two-step kernel; returns the count
int fused_candidates(int dims, const int N[3], int two_step, int* out, int max);
long long fused_items(int dims, const int N[3], int chunk);
template <class P, int DIMS>
void launch_fused_batch(const BatchArgs<P>& b, long long total_items, int coef_mode, int link_mode,
                        cudaStream_t s);
// (2+1)D two steps per pass: rows per item by the rule, items of a grid, and
// the batched launch (uniform / Klein-step coefficients, no / constant links)
int fused_chunk_tb2(const int N[3]);
long long fused_items_tb2(const int N[3], int chunk);
void launch_fused2d_tb2_batch(const BatchArgs<F32>& b, long long total_items, int coef_mode, int link_mode,
                              cudaStream_t s);

// Observables of the stored state: per-block FP64 partial sums of
// [sum|psi|^2, Bx, By, Bz, sum_{beyond} |psi|^2] with
// B_a = Re sum_lower conj(G) s_a d_a(G)  (E = naive + r_x Bx + r_y By + r_z Bz).
template <class P>
struct ObsArgs {
  const typename P::cplx* pl[8];
  int N[3];
  long long pstride;
  int link_mode;
  typename P::Link L[3];
  FieldDesc f;
  double t_links;           // time of the upper sheet (t - dt/2)
  int dens_axis, dens_X;    // partial density: half-lattice index >= dens_X along axis
  double* partials;         // [gridDim.x][5]
  int zlo, nzu, zorg, Nzg;  // levels summed along the marching axis and their global position, as in FusedArgs
};
constexpr int kObsSums = 5;

// number of blocks (= partial sums) the observables kernel uses for a grid
int observables_blocks(const int N[3], int dims);
template <class P, int DIMS>
void launch_observables(const ObsArgs<P>& a, int blocks, cudaStream_t s);
// fixed-order sum of partials[nblocks][5] into out[5]
void launch_finish_sums(const double* partials, int nblocks, double* out, cudaStream_t s);
// fixed-order sum of partials[nblocks][2] into out[2]
void launch_finish_sums2(const double* partials, int nblocks, double* out, cudaStream_t s);

// table of plane-wave link factors exp(-i phi) for both half-steps of one time
// step: tab[half * n + H], H = half-lattice coordinate along `axis`, n = 2 N_axis;
// elements of PlaneLinkOf<P>::type
template <class P>
void launch_link_table(void* tab, int n, const FieldDesc& f, int dims, int axis, int pol, double t_up,
                       double t_lo, cudaStream_t s);

// coefficient table of a time-independent potential (COEF_TABLE): every
// plane of the state layout (pstride), b = 1/(1 + i dt (beta m + V)/2) as
// {re hi, im hi, re lo, im lo}
void launch_coef_table(float4* tab, const FieldDesc& f, int dims, const int N[3], long long pstride,
                       cudaStream_t s);

// COEF_SOFTCORR correction records of a soft-core potential (one 32-bit word
// per value, softcore_corr_index's layout); *overflow (device) is or-ed with 1
// if a correction does not fit
void launch_softcore_corr(unsigned* out, const HalfFields<F32>& hu, const HalfFields<F32>& hl, const FieldDesc& f,
                          int dims, const int N[3], int* overflow, cudaStream_t s);

// link integrals of an arbitrary vector potential (Sect. 4): raw = the
// caller's integrals [axis][plane][cell] (canonical layout, cells dense), out
// = q times them per value in the state layout, slot 2a = the value's up link
// and 2a+1 = its down link: out[slot * P * pstride + plane * pstride + cell]
void launch_link_integral_table(double* out, const double* raw, int dims, const int N[3], long long pstride,
                                double q, cudaStream_t s);

// LINK_TABLE: exp(-i phi) of every value's up link (slot 2a) and down link
// (slot 2a+1) of a time-independent vector potential, FP32 hi + lo pairs:
// out[slot * P * pstride + plane * pstride + cell]
void launch_link_factor_table(F32::Link* out, const FieldDesc& f, int dims, const int N[3], long long pstride,
                              cudaStream_t s);

// measured FP64 FMA rate of the current device (TFLOP/s), < 0 on a CUDA failure
double measure_fp64_fma_tflops();

// canonical complex128 plane <-> device plane of the simulation precision
void launch_convert_in(const double2* src, float2* dst, long long n, cudaStream_t s);
void launch_convert_out(const float2* src, double2* dst, long long n, cudaStream_t s);

}  // namespace dirac
