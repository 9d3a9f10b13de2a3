/*
 * rm.h - C ABI of the GB300 R-matrix outer-region energy sweep.
 *
 * For every energy E on a mesh and every partial wave the library computes
 *   R_ij(E) = (1/2a) sum_k w_ik w_jk / (E_k - E)          (Eq. 1, as the
 *             matrix product of Eq. 2; sign and 1/2a: Rydberg form with
 *             surface amplitudes w_ik, dR/dE positive semidefinite),
 * matches it at r = a (Bloch constant b = 0) to zero-potential asymptotic
 * functions (Riccati-Bessel for open channels, decaying khat_l for closed
 * ones; the paper states the problem but not these formulae), solves for the
 * open-open K-matrix by LU with partial pivoting, and reduces K to
 * S = (I + iK)(I - iK)^-1, the eigenphase sum and partial cross sections
 * sigma_{i->j} = (pi / k_i^2) |T_ji|^2, T = S - I (weights (2J+1)/g_i = 1).
 * Cross sections and eigenphase sums (rm_xsec, rm_run) come by default from
 * the equivalent outgoing-wave form without K (see rm_solve_precision_t).
 * Units: Rydberg energies, bohr lengths, k^2 = E - e_i, sigma in bohr^2.
 *
 * Threading and streams.  A plan belongs to one CUDA device and one stream
 * (given at creation; NULL = the legacy default stream).  Every call
 * enqueues work on that stream.  Calls whose output memory is RM_MEM_HOST
 * return after the results are in host memory; calls with RM_MEM_DEVICE
 * outputs return as soon as the work is enqueued.  A plan must not be used
 * from two host threads at once.
 *
 * Errors.  Every call returns an rm_status_t; nothing aborts and no C++
 * exception crosses this boundary.  rm_last_error() gives a one-line
 * description of the most recent failure in the calling thread.  Numerical
 * trouble at a single energy is not an error: it is reported in the per-energy
 * flags (RM_FLAG_*).
 *
 * Fault injection for tests (host side only; read at each rm_plan_create):
 *   RM_FAULT_ALLOC=k        the k-th device allocation of the call fails as if
 *                           the device were out of memory (RM_ERR_NOMEM; the
 *                           partial plan is freed, *out stays NULL).
 *   RM_FAULT_WAIT_CYCLES=c  every mbarrier wait of the plan's unclustered
 *                           tensor-core launches gives up after c clock cycles
 *                           instead of about 2 s; an aborted tile lets its own
 *                           copies and MMAs finish, frees its TMEM and reports
 *                           RM_ERR_TIMEOUT through rm_sync / the next host-
 *                           memory call.  Clustered launches ignore it.
 * Tracing: every ABI call, and every kernel launch while per-kernel timing is
 * on, is an NVTX range named after it (no cost without a profiler).
 *
 * Layouts (all row-major, 0-based):
 *   W          n_ch x n_poles, w_ik at W[i*n_poles + k]
 *   R_packed   per energy, the upper triangle row by row:
 *              p(i,j) = i*n - i(i-1)/2 + (j-i), i <= j, n_p = n(n+1)/2;
 *              energy e of the range at R_packed[(e-e0)*n_p + p]
 *   K          per energy a dense n x n block at K[(e-e0)*n*n + i*n + j];
 *              the open-open n_o x n_o block is valid, the rest is zero
 *   sig_sel    per energy n_sel x n: sig_sel[((e-e0)*n_sel + q)*n + j]
 *              = sigma_{sel[q] -> j}; zero where either channel is closed
 *   sig_tot    per energy n_sel: sum over j of sig_sel
 *   eigsum     per energy: -arg det(I - iK) wrapped to (-pi, pi]; equal to
 *              sum_m arctan(lambda_m(K)) modulo 2 pi
 */
#ifndef RM_H
#define RM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RM_OK = 0,
  RM_ERR_ARG = 1,      /* null pointer, bad size, bad option, l out of range, NaN input */
  RM_ERR_ORDER = 2,    /* poles or thresholds (or the energy mesh) not sorted ascending */
  RM_ERR_NOMEM = 3,    /* device or host allocation failed */
  RM_ERR_CUDA = 4,     /* CUDA runtime error, or no usable sm_103 device */
  RM_ERR_TIMEOUT = 5,  /* a bounded device-side wait ran out */
  RM_ERR_STATE = 6     /* call not valid in the plan's current state */
} rm_status_t;

typedef enum { RM_MEM_HOST = 0, RM_MEM_DEVICE = 1 } rm_mem_t;

typedef enum {
  RM_PREC_FP64 = 0,        /* pole sum over all poles in FP64 (baseline form) */
  RM_PREC_SPLIT_BF16 = 1,  /* far poles: sliced BF16 tcgen05 GEMM, FP32 TMEM
                              accumulation; |E_k - E| < delta in FP64 */
  RM_PREC_SPLIT_FP16 = 2,  /* as SPLIT_BF16 with the slices held in FP16 */
  RM_PREC_FP32_SIMT = 3    /* far poles: plain FP32 products and FP32 accumulation
                              on the CUDA cores; near window in FP64 (comparison form) */
} rm_precision_t;

/* per-energy flag bits */
#define RM_FLAG_NUDGED 1u    /* energy was within 1e-9 Ry of a pole or threshold; moved up 1e-6 Ry */
#define RM_FLAG_ILLCOND 2u   /* min|pivot| / max|pivot| of the matching LU below 1e-12 (set where an LU runs:
                                rm_kmatrix, solve_prec FP64_LU / MIXED, and RM_FLAG_LU energies; the
                                outgoing-wave form forms no LU) */
#define RM_FLAG_NO_OPEN 4u   /* no open channel (E below every threshold); outputs are zero */
#define RM_FLAG_SINGULAR 8u  /* exact zero pivot; outputs are NaN */
#define RM_FLAG_ASYM 16u     /* a Coulomb / Whittaker continued fraction did not converge within its
                                iteration cap for some channel (z > 0 only), or (rm_xsec_from_r_static
                                only) a channel's l lay outside [0, RM_LMAX]; outputs are unreliable */
#define RM_FLAG_FP64 32u     /* solve_prec = RM_SOLVE_MIXED: the FP32 refinement did not converge (or hit a
                                zero pivot) and the matching system was solved in FP64 instead;
                                RM_SOLVE_FP64 (rm_run / rm_xsec): the double-float LDL^T of S'' that gives
                                the sign of det S_oo failed its growth or pivot check and S'' was
                                factored in FP64 instead, or (split precisions) the refinement of the
                                double-float solution of Z made a correction above 1e-7 and Z was
                                factored in FP64 instead (same results) */
#define RM_FLAG_LU 64u       /* rm_run / rm_xsec with solve_prec = RM_SOLVE_FP64: the outgoing-wave
                                factorisation failed its growth or pivot check and the energy was solved
                                by LU with partial pivoting instead (same results, more flops) */
#define RM_FLAG_NEAR_THRESHOLD 128u /* the input energy lies within 1e-6 Ry of a channel threshold (tested
                                       before any nudge): a channel opens there (k -> 0), so its results
                                       are reported, and judged, apart from the rest of the mesh */

#define RM_LMAX 32           /* largest supported channel angular momentum */
#define RM_DEFAULT_SLICES 15 /* slice products of the tensor-core pole sum when rm_options.slices = 0:
                                the cheapest set that keeps R and K within 1e-6 and cross sections
                                within 1e-8 of the FP64 oracle on the sampled n_ch = 256 mesh
                                (SPLIT_FP16, which cannot hold five slices, defaults to 13) */
#define RM_MAX_SEL 64        /* largest number of selected initial channels */

/* Matching solve.  FP64: rm_kmatrix solves for K by LU
   with partial pivoting, then the S-step by an LDL^T of I - iK; rm_run and rm_xsec go straight
   to the cross sections and eigenphase sum through the outgoing-wave form: the closed channels
   eliminated by a real LDL^T, then one complex symmetric LDL^T of
   Z = G - diag(h / (a h')), h = c + i s, on the open channels (about half the flops; an energy
   whose real elimination shows large growth or a tiny pivot goes through LU, RM_FLAG_LU);
   the sign of det S_oo comes from the inertia of S'' = V S_oo V (V = diag(c' / |h'|)), factored
   in double-float on the FP32 pipe, or in FP64 where that fails its checks (RM_FLAG_FP64);
   with split precisions Z itself is factored in double-float (FP32 hi + lo pairs, about 48 bits)
   and its solutions refined once against an FP64 residual (FP64 again where the correction
   exceeds 1e-7 of the solution, RM_FLAG_FP64; FP64 plans and dipole waves factor Z in FP64);
   dipole waves' photoionisation amplitudes come from one more right-hand side of Z.
   FP64_LU: the LU path for every energy.  MIXED: LU in FP32, then iterative refinement
   with residuals r = -B - M Y in double-float (FP32 hi + lo, error-free products and sums, about
   48 bits) and FP32 correction solves until the last correction is below 1e-11 of Y; an energy
   whose refinement stops contracting is solved again in FP64 (RM_FLAG_FP64).  The S-step stays
   FP64 (its eigenphase sum needs FP64 pivots). */
typedef enum { RM_SOLVE_FP64 = 0, RM_SOLVE_MIXED = 1, RM_SOLVE_FP64_LU = 2 } rm_solve_precision_t;

typedef struct rm_plan_s* rm_plan_t;

/* One partial wave (J-pi symmetry).  Pointer memory space: rm_options.mem. */
typedef struct {
  int32_t n_ch;          /* channels n, 1 <= n <= 640 */
  int32_t n_poles;       /* poles N, 1 <= N */
  double a;              /* R-matrix radius (bohr), > 0 */
  const int32_t* l;      /* [n] channel angular momenta, 0 <= l <= RM_LMAX */
  const double* thresh;  /* [n] channel thresholds e_i (Ry), sorted ascending */
  const double* pole_E;  /* [N] poles E_k (Ry), sorted ascending */
  const double* W;       /* [n*N] surface amplitudes w_ik, row-major */
  double z;              /* residual charge of the target seen by the scattered electron
                            (potential -2z/r, Ry units), finite and >= 0.  0: neutral target,
                            Riccati-Bessel / k-hat outer functions; > 0: ion, Coulomb functions
                            F_l, G_l (eta = -z/k) for open and Whittaker W_{z/kappa, l+1/2} for
                            closed channels.  The paper's targets are ions (B II, Ca II,
                            Fe III ...); it gives no outer-region formulas, so these are the
                            standard ones.  Repulsive fields (z < 0) are rejected. */
  const double* dip;     /* [N] bound-free dipole vector d_k = <psi_k|D|Psi_0> between the inner-region
                            eigenstates of this (final) symmetry and the initial bound state, or NULL
                            (no photoionisation).  With a dipole vector the pole sum carries it as
                            one more row of W, giving y_i(E) = (1/2a) sum_k w_ik d_k / (E_k - E). */
  double e0;             /* initial bound-state energy (Ry, same origin as the thresholds); the photon
                            energy is omega = E - e0.  Ignored without dip. */
} rm_wave;

typedef struct {
  int32_t prec;            /* rm_precision_t */
  double delta;            /* near-pole window half width (Ry) for split modes; > 0 */
  int32_t slices;          /* SPLIT_BF16 / SPLIT_FP16: slice products per far term P_pk D_ke.  Both
                              operands are cut into up to five 8-bit slices q_0..q_4, r_0..r_4
                              (orders of 2^-8; the last slice of a set is rounded); the product
                              sums q_u r_v over
                                3:  u + v <= 1 (two slices each),
                                6:  u + v <= 2 (three slices each),
                                10: u + v <= 3 (four slices each),
                                13: u + v <= 3 and (1,3), (2,2), (3,1),
                                15: u + v <= 4 (five slices each; SPLIT_BF16 only, two pipeline
                                    stages instead of three).
                              Relative error of one term about 2^-16, 2^-23, 2^-31, 2^-32, 2^-40.
                              0 = RM_DEFAULT_SLICES.  Fewer products are faster and less
                              accurate; other precisions take 0 only (else RM_ERR_ARG). */
  const int32_t* sel_init; /* host array of selected initial channels; NULL = {0} */
  int32_t n_sel;           /* entries in sel_init (ignored when sel_init is NULL) */
  int32_t mem;             /* rm_mem_t of every input pointer (waves and energies) */
  int32_t chunk;           /* energies per rm_run chunk; 0 = automatic: the whole mesh when its
                              R-matrices fit min(24 GiB, a third of free device memory), else
                              the largest multiple of 256 energies that does */
  int32_t autotune;        /* 1: at plan creation, time the tensor-core cluster shapes (split
                              modes, unless cluster_x/y are given) and, when the mesh does not
                              fit one chunk, chunk sizes 256 .. 8192 on the mesh's first
                              energies; keep the fastest */
  const char* tune_cache;  /* optional file caching autotuned choices (NULL = none) */
  int32_t cluster_x;       /* split modes, rm_run: CTAs per cluster sharing one energy tile
                              (each forms 1/cluster_x of the D slices): 1, 2 or 4; 0 = automatic.
                              With 1, the D slices of each chunk are written once by a separate
                              kernel and loaded by TMA (no formation in the pole-sum kernel; the
                              plan holds 8 bytes per energy and pole of the chunk for them) */
  int32_t cluster_y;       /* CTAs per cluster sharing one pair tile (each forms 1/cluster_y of
                              the P slices): 1, 2 or 4; 0 = automatic.  At most 8 CTAs per
                              cluster; a shape the device cannot co-schedule is rejected with
                              RM_ERR_ARG. */
  int32_t solve_prec;      /* rm_solve_precision_t of the matching solve (default FP64) */
  int32_t mma_pair;        /* split modes, rm_run, 1 x 2 clusters with D by TMA and 15 products:
                              0 (default) or 1 = the pole sum's MMAs run on the CTA pair as one
                              (tcgen05 cta_group::2, M = 256 energies, each SM reading its own D
                              slices and the P slices of the 64 pairs it forms); -1 = one-SM MMAs
                              with the two P halves exchanged between the CTAs.  Both compute
                              the same sum of the same slice products (see rm_plan_mma_pair). */
} rm_options;

/* Fill *opt with defaults: FP64, delta 0.05, sel {0}, host inputs, auto chunk. */
void rm_options_default(rm_options* opt);

/*
 * Create a plan: validate and copy the inputs to the device (the caller may
 * free them when this returns), nudge the energy mesh per wave (energies
 * within 1e-9 Ry of a pole or threshold move up by 1e-6 Ry, once), count the
 * open channels per energy and size the workspace.  energies[n_e] must be
 * sorted ascending.  cuda_stream is a cudaStream_t (NULL = default stream).
 * On failure *out is NULL.
 */
rm_status_t rm_plan_create(rm_plan_t* out, const rm_wave* waves, int32_t n_waves,
                           const double* energies, int64_t n_e, const rm_options* opt,
                           void* cuda_stream);

/* Replace the inputs of an existing plan by new ones of the same shapes
   (n_ch, n_poles, n_waves, n_e); pointers are in memory space `mem`. */
rm_status_t rm_plan_load(rm_plan_t plan, const rm_wave* waves, const double* energies,
                         int32_t mem);

/* Packed R-matrices of one wave for energies [e0, e1) (the pole sum of
   Eq. 1, in the plan's precision), R_packed[(e1-e0) * n_p]. */
rm_status_t rm_rmatrix(rm_plan_t plan, int32_t wave, int64_t e0, int64_t e1, double* R_packed,
                       int32_t mem);

/* K-matrices, open-channel counts and flags of one wave for [e0, e1).
   K[(e1-e0)*n*n], n_open[(e1-e0)], flags[(e1-e0)]; any may be NULL. */
rm_status_t rm_kmatrix(rm_plan_t plan, int32_t wave, int64_t e0, int64_t e1, double* K,
                       int32_t* n_open, uint8_t* flags, int32_t mem);

/* Eigenphase sums and cross sections of one wave for [e0, e1).
   eigsum[(e1-e0)], sig_tot[(e1-e0)*n_sel], sig_sel[(e1-e0)*n_sel*n]; any may be NULL. */
rm_status_t rm_xsec(rm_plan_t plan, int32_t wave, int64_t e0, int64_t e1, double* eigsum,
                    double* sig_tot, double* sig_sel, int32_t mem);

/* The whole sweep: every wave, every energy, R -> K -> S, eigenphase sum and
   cross sections into plan-owned device buffers (read them with
   rm_results).  All waves run together: one launch per kernel and energy
   chunk covers every wave (tensor-core tiles ordered longest first, solve
   units claimed dynamically in decreasing cost), and the whole sequence is
   captured once in a CUDA graph and replayed.  While per-kernel timing is
   enabled the same launches are issued directly (no graph) so that each
   can be bracketed by events.  This is the call the benchmark times. */
rm_status_t rm_run(rm_plan_t plan);

/* Copy results of the last rm_run for one wave and energies [e0, e1).
   Any output pointer may be NULL. */
rm_status_t rm_results(rm_plan_t plan, int32_t wave, int64_t e0, int64_t e1, double* eigsum,
                       double* sig_tot, double* sig_sel, int32_t* n_open, uint8_t* flags,
                       int32_t mem);

/* Photoionisation cross sections of one wave (it must carry a dipole vector) for [e0, e1),
   length form, standard R-matrix reading (the paper names its photoionisation module but prints
   no formulas): from the K-normalised solutions' boundary derivatives
   F'_im = s'_m delta_im + Lambda_i Y_im, the amplitudes M^K_m = sqrt(2) a sum_i F'_im y_i(E),
   the incoming-wave amplitudes M^- = (I + iK)^-1 M^K (computed, with RM_SOLVE_FP64, as
   M^-_m = -sqrt(2) (conj(Zhat)^-1 y)_m / conj(h'_m) from the outgoing-wave matrix, the same
   quantity), and
   sigma_PI,m = (4 pi alpha / 3) (E - e0) |M^-_m|^2 (a0^2; initial statistical weight 1;
   s, c = k^-1/2 sin, cos i.e. sqrt(pi) times per-Rydberg energy normalisation).
   sig_pi[(e1-e0)] total, sig_pi_ch[(e1-e0)*n] per final channel; either may be NULL. */
rm_status_t rm_photo(rm_plan_t plan, int32_t wave, int64_t e0, int64_t e1, double* sig_pi,
                     double* sig_pi_ch, int32_t mem);

/* Photoionisation results of the last rm_run (waves with a dipole vector), as rm_photo. */
rm_status_t rm_results_photo(rm_plan_t plan, int32_t wave, int64_t e0, int64_t e1, double* sig_pi,
                             double* sig_pi_ch, int32_t mem);

/* Post-processing (no plan needed).  The paper compares its cross sections with experiment after
   convolving them with a Gaussian of the experiment's full width at half maximum and averaging
   them over initial levels with statistical weights (2/3 ground + 1/3 metastable, fine-structure
   levels ...).  For a sorted mesh energies[n_e] and n_series cross-section series
   sigma[n_series * n_e] (series-major) on it:
     out[e] = sum_e' G(E_e - E_e') tw_e' m_e' / sum_e' G(E_e - E_e') tw_e',
     m_e' = sum_s f_s sigma[s * n_e + e'],
   G a Gaussian of full width at half maximum fwhm (same unit as the energies), tw the trapezoid
   weights of the mesh, the kernel truncated at 8 standard deviations; dividing by the kernel's
   own sum keeps a constant a constant at the mesh ends.  fwhm = 0 gives the weighted sum alone.
   weights: host array f[n_series] (NULL = 1/n_series each); 1 <= n_series <= 16, fwhm finite
   and >= 0.  energies, sigma and out are in memory space mem; the mesh must be sorted ascending
   (checked for host pointers only).  Device pointers: enqueued on cuda_stream (NULL = default)
   without waiting; host pointers: the call allocates device buffers and returns when done. */
rm_status_t rm_convolve(const double* energies, int64_t n_e, const double* sigma, int32_t n_series,
                        const double* weights, double fwhm, double* out, int32_t mem, void* cuda_stream);

/* Wait for the plan's stream; reports device-side error words. */
rm_status_t rm_sync(rm_plan_t plan);

/* Sizes: n_ch, n_poles of a wave; the plan's n_e, n_sel, rm_run energy-chunk size and device
   workspace bytes.  Any output may be NULL. */
rm_status_t rm_plan_info(rm_plan_t plan, int32_t wave, int32_t* n_ch, int32_t* n_poles,
                         int64_t* n_e, int32_t* n_sel, int32_t* chunk, int64_t* workspace_bytes);

/* Cluster shape of rm_run's tensor-core pole-sum launch (1 x 1 outside split modes). */
rm_status_t rm_plan_cluster(rm_plan_t plan, int32_t* cluster_x, int32_t* cluster_y);

/* *on = 1 when rm_run's tensor-core pole sum runs as 2-SM MMAs (rm_options.mma_pair), else 0. */
rm_status_t rm_plan_mma_pair(rm_plan_t plan, int32_t* on);

/* Slice products per far term of the plan's tensor-core pole sum (3, 6, 10, 13 or 15; 0 when
   the plan's precision has no tensor-core pole sum). */
rm_status_t rm_plan_slices(rm_plan_t plan, int32_t* products);

/* Number of kernel launches this plan has issued since creation. */
int64_t rm_plan_launches(rm_plan_t plan);

/* Kernel identifiers for per-kernel device timing. */
#define RM_KERNEL_POLESUM_FP64 0   /* FP64 pole sum (all poles) */
#define RM_KERNEL_POLESUM_SPLIT 1  /* sliced BF16 tcgen05 pole sum (far poles) */
#define RM_KERNEL_NEAR 2           /* FP64 near-pole window */
#define RM_KERNEL_ASYM 3           /* asymptotic functions */
#define RM_KERNEL_SOLVE 4          /* matching solve + S-step */
#define RM_KERNEL_DSLICE 5         /* D = 1/(E_k - E) slices for the tensor-core pole sum (rm_run, cluster_x = 1) */
#define RM_KERNEL_COUNT 6

/* Per-kernel device timing.  While enabled, every kernel launch of the plan
   is bracketed by CUDA events on the plan's stream.  rm_profile_read waits
   for the stream and returns, for one kernel id, the summed event time (ms)
   and the number of launches since the last read, then resets them. */
rm_status_t rm_profile_enable(rm_plan_t plan, int32_t on);
rm_status_t rm_profile_read(rm_plan_t plan, int32_t kernel, double* total_ms, int64_t* launches);

rm_status_t rm_plan_destroy(rm_plan_t plan);

/* Bounds-checked build (librm_checked.so, compiled with -DRM_CHECKED): the kernels guard their
   index arithmetic (output and workspace stores, staged tiles, per-energy ranges); a failing
   guard skips the access and records the source line of the first failure per translation unit,
   without trapping.  rm_checked_report waits for the device, returns the first recorded failure
   (unit: 0 prep, 1 tensor-core pole sum / D slices / near window, 2 FP64 pole sum, 3 FP32 pole
   sum, 4 asymptotic functions, 5 solve, 6 convolution, 7 allocation-free entry point; line: its
   source line) or unit -1, line 0 when none, and clears the records.  In the normal library it
   returns RM_ERR_STATE. */
rm_status_t rm_checked_report(int32_t* unit, int32_t* line);

const char* rm_status_str(rm_status_t s);
const char* rm_last_error(void);

/*
 * K-matrix / S-step without any device allocation.  The paper has no
 * counterpart to this call: it exists for callers that are not allowed to
 * call cudaMalloc (plug-ins bound to a host application's fixed memory pool,
 * real-time loops where an allocation may block or fail, code running where
 * the device allocator is off limits to it).  It computes what rm_kmatrix and
 * rm_xsec compute, from packed R-matrices the caller already holds, with the
 * same kernels; its only scratch is a static device array of
 * RM_STATIC_SCRATCH_BYTES inside this library, which every GPU that loads the
 * library holds until the process exits.  It allocates nothing, host or
 * device, and calls no allocating library routine.
 *
 * All array pointers are DEVICE pointers except sel_init (host; NULL = {0}),
 * which is read before the call returns (it travels as a kernel argument).
 *   R_packed  [n_e * n_p] packed upper triangles, energy-major (as rm_rmatrix)
 *   l, thresh [n_ch]; pole_E [n_poles] (used only to nudge energies that sit
 *             on a pole, exactly as rm_plan_create does); energies [n_e]
 *   outputs   as rm_kmatrix / rm_xsec (K [n_e*n*n], eigsum [n_e],
 *             sig_tot [n_e*n_sel], sig_sel [n_e*n_sel*n], flags, n_open);
 *             any may be NULL
 * Inputs are not validated on the device: thresholds and poles must be sorted
 * ascending and finite.  An l outside [0, RM_LMAX] is clamped for the
 * asymptotic functions and sets RM_FLAG_ASYM on every energy of the call.
 * The work is enqueued on cuda_stream (NULL = default stream) and the call
 * returns without waiting.
 * Sizes: 1 <= n_ch <= 640, as for rm_wave (larger n_ch returns RM_ERR_ARG);
 * 1 <= n_sel <= RM_MAX_SEL.  Each resident solve CTA needs a workspace of about
 * 4 n_ch^2 + 2 n_ch (n_sel + 1) doubles in the scratch (13 MB at n_ch = 640),
 * besides 32 n_ch bytes per energy of the current chunk, so the scratch holds at
 * most one workspace per SM and about 2^21 / n_ch^2 in all: from n_ch ~ 120 up
 * fewer solve CTAs run than a plan would use (30 at n_ch = 256, 5 at 640), the
 * price of not allocating.  rm_static_layout reports the energy chunk and the
 * number of solve workspaces a call will use.
 * Set-up: the first call on each device (with that device current) looks up
 * the scratch array's device address (cudaGetSymbolAddress) and the device's
 * attributes; make that first call before any stream capture.  All calls
 * share the one scratch array and every call overwrites it, so calls that may
 * overlap on the GPU (different streams, or threads) race and must be
 * serialised by the caller.  Errors: rm_static_last_error(), the message of the last failure of
 * this entry point in any thread (a fixed process-wide buffer, so that failing allocates nothing
 * either; failures in two threads at once may overwrite each other's message).
 */
#define RM_STATIC_SCRATCH_BYTES (64ll << 20)
rm_status_t rm_xsec_from_r_static(const double* R_packed, int32_t n_ch, int32_t n_poles, double a,
                                  const int32_t* l, const double* thresh, const double* pole_E,
                                  const double* energies, int64_t n_e, const int32_t* sel_init,
                                  int32_t n_sel, double* K, double* eigsum, double* sig_tot,
                                  double* sig_sel, uint8_t* flags, int32_t* n_open,
                                  void* cuda_stream);
const char* rm_static_last_error(void);
/* Energy chunk and number of solve workspaces rm_xsec_from_r_static uses for n_ch channels and
   n_sel selected channels on the current device; RM_ERR_ARG for sizes the call rejects.  Does
   the call's per-device set-up, no other device work. */
rm_status_t rm_static_layout(int32_t n_ch, int32_t n_sel, int32_t* chunk, int32_t* slots);

#ifdef __cplusplus
}
#endif

#endif /* RM_H */
