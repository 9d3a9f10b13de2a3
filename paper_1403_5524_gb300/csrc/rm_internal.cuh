// Internal declarations shared by the translation units of the R-matrix library.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/rm.h"

namespace rm {

// ---------------------------------------------------------------------------
// bounds-checked build
// ---------------------------------------------------------------------------
// Built with -DRM_CHECKED (librm_checked.so), RM_CHECK(cond) guards a global or shared memory
// access in the kernels: a false condition skips the access and records the source line of the
// first failure in this translation unit's device word (no trap, the kernel carries on);
// RM_CHECK_READER(unit) defines the host function that reads and clears that word, and
// rm_checked_report() collects them.  In the normal build RM_CHECK(cond) is `true` and costs
// nothing.
#ifdef RM_CHECKED
static __device__ int g_rm_check_line;
__device__ __forceinline__ bool rm_check(bool ok, int line) {
  if (!ok) atomicCAS(&g_rm_check_line, 0, line);
  return ok;
}
#define RM_CHECK(cond) (::rm::rm_check((cond), __LINE__))
#define RM_CHECK_READER(unit)                                            \
  int check_line_##unit(bool reset) {                                    \
    int v = 0;                                                           \
    if (cudaMemcpyFromSymbol(&v, g_rm_check_line, sizeof(int)) != cudaSuccess) { \
      cudaGetLastError();                                                \
      return -1;                                                         \
    }                                                                    \
    if (reset) {                                                         \
      const int z = 0;                                                   \
      cudaMemcpyToSymbol(g_rm_check_line, &z, sizeof(int));              \
    }                                                                    \
    return v;                                                            \
  }
#else
#define RM_CHECK(cond) true
#define RM_CHECK_READER(unit)
#endif
// one reader per translation unit with kernels (checked build only)
int check_line_prep(bool reset);
int check_line_polesum_tc(bool reset);
int check_line_polesum_fp64(bool reset);
int check_line_polesum_fp32(bool reset);
int check_line_asym(bool reset);
int check_line_solve(bool reset);
int check_line_convolve(bool reset);
int check_line_static(bool reset);

// ---------------------------------------------------------------------------
// device-side helpers
// ---------------------------------------------------------------------------
struct cplx {
  double re, im;
};
__host__ __device__ inline cplx make_c(double r, double i) { return cplx{r, i}; }
__host__ __device__ inline cplx operator+(cplx a, cplx b) { return cplx{a.re + b.re, a.im + b.im}; }
__host__ __device__ inline cplx operator-(cplx a, cplx b) { return cplx{a.re - b.re, a.im - b.im}; }
__host__ __device__ inline cplx operator*(cplx a, cplx b) {
  return cplx{fma(a.re, b.re, -a.im * b.im), fma(a.re, b.im, a.im * b.re)};
}

// Packed upper-triangle index p(i,j), i <= j.
__host__ __device__ inline int64_t pair_index(int n, int i, int j) {
  return (int64_t)i * n - ((int64_t)i * (i - 1)) / 2 + (j - i);
}

// ---------------------------------------------------------------------------
// per-wave device data
// ---------------------------------------------------------------------------
// Split-precision pole-sum data (RM_PREC_SPLIT_BF16).
struct SplitDev {
  float* omega = nullptr;   // [2n * Npad] w_ik / sigma_i: FP32 hi row 2i, lo row 2i+1
  float* pol = nullptr;     // [2 * Npad] poles as FP32 hi (row 0) + lo (row 1)
  double* sigma = nullptr;  // [n] power-of-two channel scales
  float* mult_p = nullptr;  // [n_p] 2^(e_p + 8)
  double* f_p = nullptr;    // [n_p] sigma_i sigma_j 2^-e_p 2^-16 / (2a)
  int32_t* klo = nullptr;   // [n_e] near window [klo, khi) in pole indices
  int32_t* khi = nullptr;
  double* tau = nullptr;    // [n_e] power-of-two D scale
  float* mult_e = nullptr;  // [n_e] 256 / tau
  float* Eh = nullptr;      // [n_e] energy FP32 hi
  float* El = nullptr;      // [n_e] energy FP32 lo
  int2* tiles = nullptr;    // [n_tiles] (8-channel i-block, 16-channel j-block)
  int n_tiles = 0;
  CUtensorMap map_omega;  // TMA descriptors (64-byte aligned type)
  CUtensorMap map_pol;
};

struct WaveDev {
  int n = 0;         // channels
  int nR = 0;        // rows of the pole-sum operand: n, or n + 1 with the dipole vector as row 0
  bool dip = false;  // photoionisation: row 0 of W is the dipole vector d_k
  double e0 = 0.0;   // initial bound-state energy (Ry)
  int N = 0;         // poles
  int Npad = 0;      // poles rounded up for aligned tiles
  double a = 0.0;
  double z = 0.0;    // residual target charge (0: neutral)
  int lmax = 0;
  int32_t* l = nullptr;     // [n]
  double* thr = nullptr;    // [n]
  double* poles = nullptr;  // [Npad], padding = +huge
  double* W = nullptr;      // [n * Npad], padding = 0
  double* E = nullptr;      // [n_e] nudged energies for this wave
  uint8_t* flags0 = nullptr;  // [n_e] flags from the nudge
  int32_t* n_open = nullptr;  // [n_e]
  // results of rm_run
  double* eta = nullptr;      // [n_e]
  double* sig_tot = nullptr;  // [n_e * n_sel]
  double* sig_sel = nullptr;  // [n_e * n_sel * n]
  uint8_t* flags = nullptr;   // [n_e]
  double* pi_tot = nullptr;   // [n_e] photoionisation (waves with a dipole vector)
  double* pi_ch = nullptr;    // [n_e * n]
  SplitDev split;
  // packed entries of one energy's pole sum (nR x nR), and where the n x n
  // channel block starts in them (after the dipole row's nR entries)
  int64_t npR() const { return (int64_t)nR * (nR + 1) / 2; }
  int64_t roff() const { return dip ? (int64_t)nR : 0; }
};

// Grouped (all waves in one launch per kernel) run of the sweep, captured in
// a CUDA graph; per-wave chunk buffers and the device-side work lists.
struct GroupDev {
  int chunk = 0;
  std::vector<double*> R;     // per wave [chunk * n_p]
  std::vector<double*> asym;  // per wave [4 * chunk * n]
  void* tc_waves = nullptr;   // per-wave tensor-core arguments
  CUtensorMap* maps = nullptr;  // [3 * n_waves] TMA descriptors (omega, poles, D slices)
  int4* tiles = nullptr;      // (wave, i-block, j-block), longest K first
  int n_tiles = 0;
  int tc_cx = 1, tc_cy = 1;   // tensor-core cluster shape (pair tiles x energy tiles)
  bool tc_pair = true;        // 1 x 2 clusters with D by TMA and 15 products: 2-SM MMAs
  std::vector<uint32_t*> D;   // per wave [4 or 5 slices][d_rows energies][Npad / 2 pole pairs] packed D slices
  int d_rows = 0;             // energy rows of each D buffer (the largest chunk); 0: none allocated
  void* dslice_waves = nullptr;
  // D slices staged by TMA (written by the D-slice kernel) instead of formed by the producers:
  // the shapes that share only P (one pair tile per cluster row)
  bool dt() const { return tc_cx == 1 && d_rows > 0; }
  void* near_waves = nullptr;
  int2* near_jobs = nullptr;  // (wave, first energy of an 8-energy block)
  int n_near_jobs = 0;
  int near_splits = 1;
  void* asym_waves = nullptr;
  void* solve_waves = nullptr;
  int2* units = nullptr;      // (wave, chunk energy), decreasing cost
  int n_units = 0;
  int* counter = nullptr;
  cudaStream_t cap = nullptr;
  cudaGraphExec_t exec = nullptr;
  int graph_kernels = 0;
  bool ready = false;
};

struct Plan {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_waves = 0;
  int64_t n_e = 0;
  int prec = RM_PREC_FP64;
  double delta = 0.05;
  int slices = 13;  // slice products per far term of the tensor-core pole sum: 3, 6, 10, 13 or 15
  int n_sel = 1;
  int32_t sel[RM_MAX_SEL] = {0};
  int32_t* sel_dev = nullptr;
  int chunk = 0;
  int n_max = 0;
  int nR_max = 0;   // largest pole-sum row count (n_ch + 1 with a dipole vector)
  int solve_mixed = 0;  // matching solve in FP32 + double-float iterative refinement
  int solve_lu = 0;     // cross sections through LU + LDL^T of I - iK for every energy
  int sm_count = 0;
  double* energies = nullptr;  // [n_e] raw mesh (device)
  std::vector<WaveDev> waves;
  // workspace
  double* Rbuf = nullptr;  // [chunk * n_p_max]
  double* asym = nullptr;  // [4 * chunk * n_max]: lam, s, sp, c
  double* slot = nullptr;  // solve workspace, solve_slots * slot_doubles
  int solve_slots = 0;
  int solve_bps = 2;  // resident solve CTAs per SM the kernels are launched for
  int64_t slot_doubles = 0;
  int32_t* err_word = nullptr;  // device error word (0 = ok)
  int64_t workspace_bytes = 0;
  int64_t launches = 0;
  bool ran = false;
  // per-kernel event timing (rm_profile_enable)
  bool prof = false;
  std::vector<cudaEvent_t> ev_pool;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> ev_live[RM_KERNEL_COUNT];
  double prof_ms[RM_KERNEL_COUNT] = {0};
  int64_t prof_n[RM_KERNEL_COUNT] = {0};
  GroupDev grp;
  bool autotuned = false;
  // test hooks, read from the environment at plan creation (host-side fault injection):
  // RM_FAULT_WAIT_CYCLES shortens every mbarrier wait of unclustered tensor-core launches
  long long fault_wait = 0;
  // RM_TEST_Z_FP64 = 1 makes every double-float solve of Z (split modes) take its FP64 fallback,
  // as if its refinement correction had been too large, so that a test can run that path
  int z_force_fp64 = 0;
};

// ---------------------------------------------------------------------------
// kernels (host launchers); each returns cudaGetLastError() of its launch
// ---------------------------------------------------------------------------
// Validation of one wave's inputs on the device: sortedness, l range, NaN.
cudaError_t launch_validate(const WaveDev& w, int N_real, const double* energies, int64_t n_e,
                            int32_t* err_word, cudaStream_t s);
// Nudge the mesh for one wave and count open channels.
cudaError_t launch_prep(const WaveDev& w, const double* energies, int64_t n_e, cudaStream_t s);
// R[e][p] = (1/2a) sum_k w_ik w_jk / (E_k - E_e) for e in [e0, e0+ne), FP64.
cudaError_t launch_polesum_fp64(const WaveDev& w, int64_t e0, int ne, double* R, cudaStream_t s);
// Asymptotic data (lam, s, s', c) per (energy, channel) for e in [e0, e0+ne).
cudaError_t launch_asym(const WaveDev& w, int64_t e0, int ne, double* asym, int ld_chunk,
                        cudaStream_t s);
// Matching LU -> K; complex LU of I - iK -> eigenphase sum, sigma.
struct SolveOut {
  double* K = nullptr;        // optional [ne * n * n]
  double* eta = nullptr;      // optional [ne]
  double* sig_tot = nullptr;  // optional [ne * n_sel]
  double* sig_sel = nullptr;  // optional [ne * n_sel * n]
  uint8_t* flags = nullptr;   // optional [ne]
  int32_t* n_open = nullptr;  // optional [ne]
  double* pi_tot = nullptr;   // optional [ne] photoionisation (waves with a dipole vector)
  double* pi_ch = nullptr;    // optional [ne * n]
  bool do_xsec = true;
};
cudaError_t launch_solve(const Plan& p, const WaveDev& w, int64_t e0, int ne, const double* R,
                         const double* asym, int ld_chunk, const SolveOut& out, cudaStream_t s);
size_t solve_smem_bytes(int n_max);
int solve_blocks_per_sm(int n_max, bool mixed);
int64_t solve_slot_doubles(int n_max, int n_sel, bool mixed);
int64_t solve_mix_offset(int n_max, int n_sel);

// Gaussian convolution / statistical averaging of cross sections (post-processing)
cudaError_t launch_convolve(const double* E, int64_t n_e, const double* sigma, int n_series, const double* f,
                            double fwhm, double* out, cudaStream_t s);
int convolve_max_series();

// split-precision pole sum
std::vector<int2> split_tiles(int n);
cudaError_t split_prepare(const Plan& p, WaveDev& w, cudaStream_t s);
cudaError_t launch_polesum_split(const Plan& p, const WaveDev& w, int64_t e0, int ne, double* R, cudaStream_t s);
cudaError_t launch_near(const Plan& p, const WaveDev& w, int64_t e0, int ne, double* R, cudaStream_t s);
cudaError_t launch_polesum_fp32(const WaveDev& w, int64_t e0, int ne, double* R, cudaStream_t s);
inline bool is_split_like(int prec) {
  return prec == RM_PREC_SPLIT_BF16 || prec == RM_PREC_SPLIT_FP16 || prec == RM_PREC_FP32_SIMT;
}
size_t polesum_tc_smem_bytes();
size_t near_smem_bytes(int n);

// grouped run (all waves per launch)
cudaError_t group_setup_split(Plan& p);
cudaError_t group_setup_asym(Plan& p);
cudaError_t group_setup_solve(Plan& p);
cudaError_t launch_polesum_split_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s);
// D slices of the chunk [e0, e0 + ne) for every wave (shapes with cluster_x = 1)
cudaError_t launch_dslice_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s);
// clusters of this shape can be resident (grouped tensor-core kernel with ns slices per operand)
bool polesum_cluster_ok(int cx, int cy, int ns, bool pair);
// the plan's rm_run pole sum is the 2-SM (cta_group::2) kernel
bool polesum_pair_runs(const Plan& p);
// slices per operand the tensor-core kernel stages for a product set (4, or 5 for 15 products)
int polesum_slice_planes(int nprod);
cudaError_t launch_near_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s);
cudaError_t launch_asym_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s);
cudaError_t launch_solve_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s);

}  // namespace rm
