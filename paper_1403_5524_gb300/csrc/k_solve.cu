// Per-energy matching solve and S-matrix step, FP64, one CTA per energy.
//
// Two forms.  Cross sections, eigenphase sums and photoionisation (rm_run,
// rm_xsec) come from the outgoing-wave form (sym_xsec below): the closed
// channels eliminated by a real LDL^T, one complex symmetric LDL^T of
// Z = G - diag(h / (a h')) on the open ones, no K.  With split-precision plans
// the LDL^T of Z runs in double-float on the FP32 pipe, its solutions refined
// once against an FP64 residual (z_ldl_refined).  The K-matrix (rm_kmatrix),
// the mixed-precision option, and energies whose real eliminations fail their
// checks take the LU form described next.
//
// Matching (Bloch constant b = 0; the paper states the problem but not the
// matching, so this is the standard zero-potential form): with the column of
// channel j divided by c_j (open) or e_j (closed),
//   [ I - a R Lambda | -B ],  B[:, m] = s_m delta_m - a R[:, m] s'_m  (m open),
// is reduced by LU with partial pivoting (row interchanges chosen on the
// first n columns, applied to all columns) followed by back substitution,
// which leaves Y = (I - a R Lambda)^-1 (-B) in the right-hand columns;
// K_jm = Y_jm / c_j for open j, m.
//
// S-step: A = I - iK (n_o x n_o, complex symmetric) with right-hand sides
// K[:, sel_q]; its LDL^T factorisation (no interchanges needed, see ldl_solve)
// gives X = A^-1 K[:, sel], T[:, sel_q] = 2i X[:, q] (T = S - I =
// 2iK(I - iK)^-1), sigma_{sel_q -> j} = (pi / k^2) |T_{j,sel_q}|^2, and the
// eigenphase sum -arg det(I - iK) = -sum_j arg d_j.
//
// Photoionisation (a wave whose pole sum carries the dipole vector as row 0,
// so that R holds y_i = (1/2a) sum_k w_ik d_k / (E_k - E) ahead of the channel
// block): the boundary derivatives of the K-normalised solutions are
// F'_im = s'_m delta_im + Lambda_i Y_im, the amplitudes
// M^K_m = sqrt(2) a sum_i F'_im y_i, and M^K is one more right-hand side of
// the complex LU: |((I - iK)^-1 M^K)_m| = |M^-_m| with M^- = (I + iK)^-1 M^K
// (K real symmetric), sigma_PI,m = (4 pi alpha / 3) (E - E_0) |M^-_m|^2.
//
// The blocked LU keeps a 16-column panel in shared memory, factors it with
// partial pivoting, and updates the columns to its right in 64-column tiles
// (row interchanges, triangular solve with the unit-lower panel block, then
// the rank-16 update).  Each matrix lives in a per-CTA global workspace slot
// that stays in L2 while the CTA works on it.  GB300 retires about two FP64
// FMAs per clock per SM; three 256-thread CTAs share an SM where their shared
// memory fits (n_ch up to about 390; two up to 640), so that one CTA's pivot
// chains, barriers and load latencies are covered by the others' FMAs.
#include <algorithm>
#include <vector>

#include "rm_internal.cuh"

namespace rm {

namespace {

constexpr int TC = 64;   // column tile of the trailing update
constexpr int PANEL_ROW_BYTES = 128;  // one panel row: 16 doubles or 8 complex values
constexpr int NT = 256;  // threads per CTA
constexpr int NWARP = NT / 32;

template <typename T>
struct Ops;

template <>
struct Ops<double> {
  __device__ static double zero() { return 0.0; }
  __device__ static double one() { return 1.0; }
  __device__ static double mag(double x) { return fabs(x); }
  __device__ static double inv(double x) { return 1.0 / x; }
  __device__ static double mul(double a, double b) { return a * b; }
  __device__ static double fms(double acc, double a, double b) { return fma(-a, b, acc); }
  __device__ static double fma_acc(double acc, double a, double b) { return fma(a, b, acc); }
  __device__ static void put(double* d, double x) { d[0] = x; }
  __device__ static double get(const double* d) { return d[0]; }
};

template <>
struct Ops<float> {
  __device__ static float zero() { return 0.0f; }
  __device__ static float one() { return 1.0f; }
  __device__ static double mag(float x) { return fabsf(x); }
  __device__ static float inv(float x) { return 1.0f / x; }
  __device__ static float mul(float a, float b) { return a * b; }
  __device__ static float fms(float acc, float a, float b) { return fmaf(-a, b, acc); }
  __device__ static float fma_acc(float acc, float a, float b) { return fmaf(a, b, acc); }
  __device__ static void put(double* d, float x) { d[0] = x; }
  __device__ static float get(const double* d) { return (float)d[0]; }
};

template <>
struct Ops<cplx> {
  __device__ static cplx zero() { return cplx{0.0, 0.0}; }
  __device__ static cplx one() { return cplx{1.0, 0.0}; }
  __device__ static double mag(cplx x) { return fabs(x.re) + fabs(x.im); }  // LAPACK cabs1
  __device__ static cplx inv(cplx x) {
    // 1 / (re + i im) = (re - i im) / (re^2 + im^2): one real division on the pivot's dependent
    // chain (Smith's form needs two in sequence); pivots here lie far inside the range where
    // re^2 + im^2 neither overflows nor underflows
    const double q = 1.0 / fma(x.re, x.re, x.im * x.im);
    return cplx{x.re * q, -x.im * q};
  }
  __device__ static cplx mul(cplx a, cplx b) { return a * b; }
  __device__ static cplx fms(cplx acc, cplx a, cplx b) {
    return cplx{fma(-a.re, b.re, fma(a.im, b.im, acc.re)), fma(-a.re, b.im, fma(-a.im, b.re, acc.im))};
  }
  __device__ static cplx fma_acc(cplx acc, cplx a, cplx b) {
    return cplx{fma(a.re, b.re, fma(-a.im, b.im, acc.re)), fma(a.re, b.im, fma(a.im, b.re, acc.im))};
  }
  __device__ static void put(double* d, cplx x) { d[0] = x.re; d[1] = x.im; }
  __device__ static cplx get(const double* d) { return cplx{d[0], d[1]}; }
};

// Double-float: a value hi + lo of two FP32 numbers (about 48 bits), with error-free products
// (FMA) and sums (Knuth's TwoSum) on the FP32 pipe, which GB300 runs about 64 times faster than
// its FP64 pipe.  Used for the inertia LDL^T of S'' (whose results only decide a sign) and, in
// complex pairs (cdf), for the LDL^T of Z (sym_xsec).  Same size as a double, so it factors in
// place of the FP64 matrix.
struct dfl {
  float hi, lo;
};
__device__ __forceinline__ dfl df_quick(float a, float b) {  // |a| >= |b| (or a = 0): a + b exactly
  const float s = __fadd_rn(a, b);
  return dfl{s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_from(double v) {
  const float h = __double2float_rn(v);
  return dfl{h, __double2float_rn(v - (double)h)};
}
__device__ __forceinline__ double df_to(dfl x) { return (double)x.hi + (double)x.lo; }
// As df_from, with integer and FP32 operations only (GB300's FP64 pipe, which also runs the
// double <-> float conversions, is 1/64 of the FP32 rate): hi takes v's sign, exponent and top 24
// significand bits, lo the remaining 29 bits (rounded to FP32), then one FastTwoSum rounds hi to
// nearest.  Values whose parts would leave FP32's normal range (zero, |v| < 2^-74, |v| >= 2^128,
// non-finite) take df_from.
__device__ __forceinline__ dfl df_from_fast(double v) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(v);
  const int ex = (int)((b >> 52) & 0x7FF);  // biased exponent
  if (ex < 949 || ex > 1150) return df_from(v);
  const unsigned int sgn = (unsigned int)(b >> 32) & 0x80000000u;
  const float hi = __uint_as_float(sgn | ((unsigned int)(ex - 896) << 23) | (unsigned int)((b >> 29) & 0x7FFFFFu));
  // the low 29 significand bits r = r1 2^23 + r0 as FP32 (exact parts, one rounding in the sum),
  // scaled by 2^(ex - 1075)
  const unsigned int r0 = (unsigned int)(b & 0x7FFFFFu), r1 = (unsigned int)((b >> 23) & 0x3Fu);
  const float f0 = __fsub_rn(__uint_as_float(0x4B000000u | r0), 8388608.0f);
  const float f1 = __fsub_rn(__uint_as_float(0x4B000000u | r1), 8388608.0f);
  const float mag = __fmul_rn(__fmaf_rn(f1, 8388608.0f, f0), __uint_as_float((unsigned int)(ex - 948) << 23));
  return df_quick(hi, sgn ? -mag : mag);
}

template <>
struct Ops<dfl> {
  __device__ static dfl zero() { return dfl{0.0f, 0.0f}; }
  __device__ static dfl one() { return dfl{1.0f, 0.0f}; }
  __device__ static double mag(dfl x) { return fabs(df_to(x)); }
  __device__ static dfl inv(dfl x) {
    // approximate FP32 reciprocal (about 2^-23), then one correction with the residual, exact in
    // its FP32 part: about 2^-46 relative, as for a correctly rounded first guess
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x.hi));
    float e = __fmaf_rn(-x.hi, r, 1.0f);
    e = __fmaf_rn(-x.lo, r, e);
    return df_quick(r, __fmul_rn(r, e));
  }
  __device__ static dfl mul(dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);  // exact rounding error of the product
    e = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, e));
    return df_quick(p, e);
  }
  // acc - a b: the product's error-free part and the two high parts summed by TwoSum
  __device__ static dfl fms(dfl acc, dfl a, dfl b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float pe = __fmaf_rn(a.hi, b.hi, -p);
    pe = __fmaf_rn(a.hi, b.lo, __fmaf_rn(a.lo, b.hi, pe));
    const float s = __fsub_rn(acc.hi, p);
    const float bb = __fsub_rn(s, acc.hi);
    const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(-p, bb));
    return df_quick(s, __fadd_rn(err, __fsub_rn(acc.lo, pe)));
  }
  __device__ static dfl fma_acc(dfl acc, dfl a, dfl b) { return fms(acc, dfl{-a.hi, -a.lo}, b); }
  // kept bitwise in the first 8 bytes of the 16-byte slot (no FP64 conversions on the FP32 path)
  __device__ static void put(double* d, dfl x) { *reinterpret_cast<dfl*>(d) = x; }
  __device__ static dfl get(const double* d) { return *reinterpret_cast<const dfl*>(d); }
};

// Complex double-float: real and imaginary parts as double-floats (16 bytes, the size of a complex
// double, so Z factors in place of its FP64 copy).  Each complex multiply-subtract is four
// double-float ones, about 48 FP32 instructions against 4 DFMA: on GB300 (128 FP32 lanes, 2 DFMA
// a clock per SM) about five times the rate.  Used for the LDL^T of Z, whose solutions are then
// refined against an FP64 residual (sym_xsec).
struct cdf {
  dfl re, im;
};

template <>
struct Ops<cdf> {
  using D = Ops<dfl>;
  __device__ static cdf zero() { return cdf{D::zero(), D::zero()}; }
  __device__ static cdf one() { return cdf{D::one(), D::zero()}; }
  __device__ static double mag(cdf x) { return fabs(df_to(x.re)) + fabs(df_to(x.im)); }  // cabs1
  __device__ static cdf inv(cdf x) {
    // conj(x) / |x|^2, as for the FP64 pivots
    const dfl q = D::inv(D::fma_acc(D::mul(x.re, x.re), x.im, x.im));
    const dfl im = D::mul(x.im, q);
    return cdf{D::mul(x.re, q), dfl{-im.hi, -im.lo}};
  }
  __device__ static cdf mul(cdf a, cdf b) {
    return cdf{D::fms(D::mul(a.re, b.re), a.im, b.im), D::fma_acc(D::mul(a.re, b.im), a.im, b.re)};
  }
  // acc - a b
  __device__ static cdf fms(cdf acc, cdf a, cdf b) {
    return cdf{D::fma_acc(D::fms(acc.re, a.re, b.re), a.im, b.im), D::fms(D::fms(acc.im, a.re, b.im), a.im, b.re)};
  }
  // acc + a b
  __device__ static cdf fma_acc(cdf acc, cdf a, cdf b) {
    return cdf{D::fms(D::fma_acc(acc.re, a.re, b.re), a.im, b.im), D::fma_acc(D::fma_acc(acc.im, a.re, b.im), a.im, b.re)};
  }
  // kept bitwise in the 16-byte slot (no FP64 conversions on the FP32 path)
  __device__ static void put(double* d, cdf x) { *reinterpret_cast<cdf*>(d) = x; }
  __device__ static cdf get(const double* d) { return *reinterpret_cast<const cdf*>(d); }
};

// Panel width: 16 columns for the real LU, 8 for the complex one, so that a
// panel row is 128 bytes either way and both LUs do the same FMAs per byte of
// trailing-matrix traffic (16 real or 8 complex multiply-adds per element).
template <typename T>
struct Blk {
  static constexpr int NB = (int)(PANEL_ROW_BYTES / sizeof(T));
};

constexpr int TILE_BYTES = Blk<double>::NB * TC * 8;  // NB x TC elements, either type
constexpr int TRI_BYTES = Blk<float>::NB * Blk<float>::NB * 4;  // the largest of the three types
static_assert(Blk<cplx>::NB * TC * (int)sizeof(cplx) == TILE_BYTES, "tile bytes");
static_assert(Blk<float>::NB * TC * (int)sizeof(float) == TILE_BYTES, "tile bytes");
static_assert(sizeof(dfl) == sizeof(double) && Blk<dfl>::NB == Blk<double>::NB, "double-float in place of FP64");
static_assert(sizeof(cdf) == sizeof(cplx) && Blk<cdf>::NB == Blk<cplx>::NB, "complex double-float in place of FP64");

// smallest power of two >= min(TC, w), at least 1
__device__ __forceinline__ int tile_width_pow2(int w) {
  w = w < TC ? w : TC;
  int p = 1;
  while (p < w) p <<= 1;
  return p;
}

struct LUStat {
  double pmin, pmax;
  int swaps;
  bool singular;
};

struct Red {
  double v[NWARP];
  int i[NWARP];
  int piv;
  double pinv[2];  // reciprocal of the chosen pivot (re, im; real types use [0])
};

// Block-wide argmax of Ops::mag over panel column j, rows [j, rows); ties -> smallest row.
// A NaN counts as the largest magnitude, and the result always lies in [j, rows): every later
// index (the row interchanges, the permutation of the unit right-hand sides) comes from it, so
// a column of NaN or garbage (an R-matrix a failed pole sum left unwritten) cannot send them
// outside the matrix; such an energy ends with NaN outputs instead.
template <typename T>
__device__ int panel_argmax(const T* panel, int rows, int j, Red* red) {
  constexpr int NB = Blk<T>::NB;
  double best = -1.0;
  int bidx = rows;
  for (int r = j + threadIdx.x; r < rows; r += NT) {
    double v = Ops<T>::mag(panel[r * NB + j]);
    if (v != v) v = INFINITY;
    if (v > best) { best = v; bidx = r; }
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const double ov = __shfl_down_sync(0xffffffffu, best, off);
    const int oi = __shfl_down_sync(0xffffffffu, bidx, off);
    if (ov > best || (ov == best && oi < bidx)) { best = ov; bidx = oi; }
  }
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) { red->v[w] = best; red->i[w] = bidx; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = red->v[0];
    int bi = red->i[0];
    for (int q = 1; q < NWARP; ++q)
      if (red->v[q] > b || (red->v[q] == b && red->i[q] < bi)) { b = red->v[q]; bi = red->i[q]; }
    if (bi < j || bi >= rows) bi = j;  // nothing compared above -1 (rows <= j cannot occur)
    red->piv = bi;
    // one reciprocal per pivot, shared by the block
    const T pv = (bi < rows) ? panel[bi * NB + j] : Ops<T>::zero();
    Ops<T>::put(red->pinv, (Ops<T>::mag(pv) == 0.0) ? Ops<T>::zero() : Ops<T>::inv(pv));
  }
  __syncthreads();
  return red->piv;
}

// LU with partial pivoting of the leading n x n block of A (row-major, ld),
// row operations applied to all m columns, then back substitution on
// columns [n, m).  smem: panel[n_max*NB], tile[NB*TC], tmp[NB*TC], tri[NB*NB],
// ipiv[n_max], with NB = Blk<T>::NB.
// A[r][col] -= sum_j L[r][j] * U[j] for rows r = r0, r0 + 4, ... < r1, where L[r][j] is
// panel row r (NB wide) and U[j] = tile[j * TC]; four rows per iteration so that
// four independent loads are in flight, the tile column held in registers.
template <typename T>
__device__ __forceinline__ void rank_update(T* __restrict__ A, int ld, int col, int r0, int r1, const T* panel,
                                            const T* tile, int nb, int RS) {
  using O = Ops<T>;
  constexpr int NB = Blk<T>::NB;
  T u[NB];
#pragma unroll
  for (int j = 0; j < NB; ++j) u[j] = (j < nb) ? tile[j * TC] : O::zero();
  int r = r0;
  for (; r + 3 * RS < r1; r += 4 * RS) {
    T v0 = A[(int64_t)r * ld + col];
    T v1 = A[(int64_t)(r + RS) * ld + col];
    T v2 = A[(int64_t)(r + 2 * RS) * ld + col];
    T v3 = A[(int64_t)(r + 3 * RS) * ld + col];
    const T* l0 = panel + (int64_t)r * NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) {
      v0 = O::fms(v0, l0[j], u[j]);
      v1 = O::fms(v1, l0[RS * NB + j], u[j]);
      v2 = O::fms(v2, l0[2 * RS * NB + j], u[j]);
      v3 = O::fms(v3, l0[3 * RS * NB + j], u[j]);
    }
    A[(int64_t)r * ld + col] = v0;
    A[(int64_t)(r + RS) * ld + col] = v1;
    A[(int64_t)(r + 2 * RS) * ld + col] = v2;
    A[(int64_t)(r + 3 * RS) * ld + col] = v3;
  }
  for (; r < r1; r += RS) {
    T v = A[(int64_t)r * ld + col];
    const T* l0 = panel + (int64_t)r * NB;
#pragma unroll
    for (int j = 0; j < NB; ++j) v = O::fms(v, l0[j], u[j]);
    A[(int64_t)r * ld + col] = v;
  }
}

template <typename T>
__device__ void lu_solve(T* __restrict__ A, int n, int m, int ld, T* panel, T* tile, T* tmp, T* tri,
                         int* ipiv, Red* red, LUStat& st) {
  using O = Ops<T>;
  constexpr int NB = Blk<T>::NB;
  const int t = threadIdx.x;
  st.pmin = INFINITY;
  st.pmax = 0.0;
  st.swaps = 0;
  st.singular = false;
  // ------------------------------------------------------------ factorisation
  for (int kb = 0; kb < n; kb += NB) {
    const int nb = min(NB, n - kb);
    const int rows = n - kb;
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      panel[idx] = (c < nb) ? A[(int64_t)(kb + r) * ld + kb + c] : O::zero();
    }
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
      const int p = panel_argmax(panel, rows, j, red);
      if (t < NB && p != j) {
        const T tmpv = panel[j * NB + t];
        panel[j * NB + t] = panel[p * NB + t];
        panel[p * NB + t] = tmpv;
      }
      if (t == 0) {
        ipiv[kb + j] = kb + p;
        if (p != j) st.swaps++;
      }
      __syncthreads();
      if (t == 0) {
        const double pm = O::mag(panel[j * NB + j]);
        st.pmin = fmin(st.pmin, pm);
        st.pmax = fmax(st.pmax, pm);
        if (pm == 0.0) st.singular = true;
      }
      const T pinv = O::get(red->pinv);
      for (int r = j + 1 + t; r < rows; r += NT) {
        const T lr = O::mul(panel[r * NB + j], pinv);
        panel[r * NB + j] = lr;
        for (int c = j + 1; c < nb; ++c) panel[r * NB + c] = O::fms(panel[r * NB + c], lr, panel[j * NB + c]);
      }
      __syncthreads();
    }
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      if (c < nb) A[(int64_t)(kb + r) * ld + kb + c] = panel[idx];
    }
    // row interchanges on every column outside the panel (all threads, one column each): right of
    // it for the elimination, left of it so that the stored L ends in the final row order (as
    // LAPACK's getrf leaves it), which lu_unit_solve and lu_resolve rely on
    for (int col = t; col < m; col += NT) {
      if (col >= kb && col < kb + nb) continue;
      for (int j = 0; j < nb; ++j) {
        const int r1 = kb + j, r2 = ipiv[kb + j];
        if (r1 != r2) {
          const T a1 = A[(int64_t)r1 * ld + col];
          A[(int64_t)r1 * ld + col] = A[(int64_t)r2 * ld + col];
          A[(int64_t)r2 * ld + col] = a1;
        }
      }
    }
    // inverse of the unit-lower diagonal block, column t by thread t
    if (t < NB) {
      for (int i = 0; i < NB; ++i) tri[i * NB + t] = (i == t) ? O::one() : O::zero();
      if (t < nb) {
        for (int i = t + 1; i < nb; ++i) {
          T acc = O::zero();
          for (int k = t; k < i; ++k) acc = O::fms(acc, panel[i * NB + k], tri[k * NB + t]);
          tri[i * NB + t] = acc;
        }
      }
    }
    __syncthreads();
    // columns right of the panel, in tiles of TC: U12 = L11^-1 A12, then the rank-nb update
    for (int c0 = kb + nb; c0 < m; c0 += TC) {
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        tmp[idx] = (j < nb && col < m) ? A[(int64_t)(kb + j) * ld + col] : O::zero();
      }
      __syncthreads();
      for (int idx = t; idx < NB * TC; idx += NT) {
        // L11^-1 is unit lower triangular: terms i <= j only (j is uniform across a warp)
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        if (col >= m) continue;  // columns past the matrix are never read
        T u = tmp[j * TC + c];
        for (int i = 0; i < j; ++i) u = O::fma_acc(u, tri[j * NB + i], tmp[i * TC + c]);
        tile[idx] = u;
        if (j < nb && col < m) A[(int64_t)(kb + j) * ld + col] = u;
      }
      __syncthreads();
      // threads over (column, row group); narrow tiles get more row groups so
      // that every warp instruction carries full lanes
      const int cwp = tile_width_pow2(m - c0);
      const int tc = t % cwp, tr = t / cwp;
      if (c0 + tc < m) rank_update<T>(A, ld, c0 + tc, kb + nb + tr, n, panel - (int64_t)kb * NB, tile + tc, nb, NT / cwp);
      __syncthreads();
    }
  }
  // ------------------------------------------------------- back substitution
  const int kb_last = ((n - 1) / NB) * NB;
  for (int kb = kb_last; kb >= 0; kb -= NB) {
    const int nb = min(NB, n - kb);
    const int rows = kb + nb;  // U[0 .. kb+nb)[kb .. kb+nb)
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      panel[idx] = (c < nb) ? A[(int64_t)r * ld + kb + c] : O::zero();
    }
    __syncthreads();
    // inverse of the upper diagonal block U11 (rows/cols kb..kb+nb), column t by thread t
    if (t < NB) {
      for (int i = 0; i < NB; ++i) tri[i * NB + t] = O::zero();
      if (t < nb) {
        const T* U = panel + (int64_t)kb * NB;  // U[i][k] = U[i * NB + k]
        const double dm = O::mag(U[t * NB + t]);
        tri[t * NB + t] = (dm == 0.0) ? O::zero() : O::inv(U[t * NB + t]);
        for (int i = t - 1; i >= 0; --i) {
          T acc = O::zero();
          for (int k = i + 1; k <= t; ++k) acc = O::fms(acc, U[i * NB + k], tri[k * NB + t]);
          const double di = O::mag(U[i * NB + i]);
          tri[i * NB + t] = (di == 0.0) ? O::zero() : O::mul(acc, O::inv(U[i * NB + i]));
        }
      }
    }
    __syncthreads();
    for (int c0 = n; c0 < m; c0 += TC) {
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        tmp[idx] = (j < nb && col < m) ? A[(int64_t)(kb + j) * ld + col] : O::zero();
      }
      __syncthreads();
      for (int idx = t; idx < NB * TC; idx += NT) {
        // U11^-1 is upper triangular: terms i >= j only (j is uniform across a warp)
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        if (col >= m) continue;  // columns past the matrix are never read
        T y = O::zero();
        for (int i = j; i < nb; ++i) y = O::fma_acc(y, tri[j * NB + i], tmp[i * TC + c]);
        tile[idx] = y;
        if (j < nb && col < m) A[(int64_t)(kb + j) * ld + col] = y;
      }
      __syncthreads();
      const int cwp = tile_width_pow2(m - c0);
      const int tc = t % cwp, tr = t / cwp;
      if (c0 + tc < m) rank_update<T>(A, ld, c0 + tc, tr, kb, panel, tile + tc, nb, NT / cwp);
      __syncthreads();
    }
  }
}

// LDL^T factorisation without pivoting of a complex symmetric matrix A (n x n,
// row-major, ld; only its lower triangle is read and kept up to date), the
// same elimination applied to the right-hand-side columns [n, m), then
// x = L^-T D^-1 L^-1 b on those columns.  Used for A = I - iK: every Schur
// complement of I - iK keeps a real part >= I (the real part of
// K21 (I - iK11)^-1 K12 is K21 (I + K11^2)^-1 K12 >= 0), so every pivot has
// |d| >= Re d >= 1 and the elimination needs no interchanges; it costs half
// the flops of LU and skips the pivot searches.  d_j is left on the diagonal.
// Blocked like lu_solve: an NB-column panel factored in shared memory, then
// the columns to its right in TC-column tiles, where a matrix column col takes
// the tile column d_j L[col][kb+j] straight from the panel and updates rows
// >= col only, and a right-hand-side column takes L11^-1 A12 as in lu_solve.
// With nf < n only the first nf pivots are taken: the trailing block [nf, n)
// is left holding its Schur complement, and the rows [nf, n) of the
// right-hand-side columns the matching forward elimination (no solve).
template <typename T>
__device__ void ldl_solve(T* __restrict__ A, int n, int m, int ld, T* panel, T* tile, T* tmp, T* tri,
                          LUStat& st, int nf = -1) {
  using O = Ops<T>;
  constexpr int NB = Blk<T>::NB;
  const int t = threadIdx.x;
  if (nf < 0) nf = n;
  __shared__ double s_pinv[Blk<T>::NB][2];  // pivot reciprocals of the current panel
  st.pmin = INFINITY;
  st.pmax = 0.0;
  st.swaps = 0;
  st.singular = false;
  // ------------------------------------------------------------ factorisation
  for (int kb = 0; kb < nf; kb += NB) {
    const int nb = min(NB, nf - kb);
    const int rows = n - kb;
    // panel rows kb.., columns kb..kb+nb; in the diagonal block the upper half comes from the
    // (current) lower half by symmetry
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      T v = O::zero();
      if (c < nb) v = (r >= c) ? A[(int64_t)(kb + r) * ld + kb + c] : A[(int64_t)(kb + c) * ld + kb + r];
      panel[idx] = v;
    }
    __syncthreads();
    // The nb x nb diagonal block by warp 0 (one reciprocal per pivot, lane 0); its upper half then
    // holds each pivot row as it was when eliminated, so every row below the block finishes its
    // nb panel entries on its own, in registers, with the same operations in the same order.
    if (t < 32) {
      for (int j = 0; j < nb; ++j) {
        if (t == 0) {
          const T pv = panel[j * NB + j];
          const double pm = O::mag(pv);
          st.pmin = fmin(st.pmin, pm);
          st.pmax = fmax(st.pmax, pm);
          if (pm == 0.0) st.singular = true;
          O::put(s_pinv[j], (pm == 0.0) ? O::zero() : O::inv(pv));
        }
        __syncwarp();
        const T pinv = O::get(s_pinv[j]);
        const int r = j + 1 + t;
        if (r < nb) {
          const T lr = O::mul(panel[r * NB + j], pinv);
          panel[r * NB + j] = lr;
          for (int c = j + 1; c < nb; ++c) panel[r * NB + c] = O::fms(panel[r * NB + c], lr, panel[j * NB + c]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    for (int r = nb + t; r < rows; r += NT) {
      T a[NB];
#pragma unroll
      for (int c = 0; c < NB; ++c) a[c] = panel[r * NB + c];
#pragma unroll
      for (int j = 0; j < NB; ++j) {
        if (j < nb) {
          a[j] = O::mul(a[j], O::get(s_pinv[j]));
#pragma unroll
          for (int c = j + 1; c < NB; ++c)
            if (c < nb) a[c] = O::fms(a[c], a[j], panel[j * NB + c]);
        }
      }
#pragma unroll
      for (int c = 0; c < NB; ++c) panel[r * NB + c] = a[c];
    }
    __syncthreads();
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      if (c < nb && r >= c) A[(int64_t)(kb + r) * ld + kb + c] = panel[idx];
    }
    // inverse of the unit-lower diagonal block (for the right-hand sides), column t by thread t
    if (m > n && t < NB) {
      for (int i = 0; i < NB; ++i) tri[i * NB + t] = (i == t) ? O::one() : O::zero();
      if (t < nb) {
        for (int i = t + 1; i < nb; ++i) {
          T acc = O::zero();
          for (int k = t; k < i; ++k) acc = O::fms(acc, panel[i * NB + k], tri[k * NB + t]);
          tri[i * NB + t] = acc;
        }
      }
    }
    __syncthreads();
    // Matrix columns in TC-wide tiles up to n, then the right-hand-side columns in tiles of their
    // own: those run every row below the panel, the matrix columns only the rows below their
    // tile's diagonal block, so sharing a warp would leave lanes idle.
    for (int c0 = kb + nb; c0 < m;) {
      const int ce = (c0 < n) ? min(c0 + TC, n) : min(c0 + TC, m);
      // tile column: d_j L[col][kb+j] for matrix columns, L11^-1 A12 for right-hand sides
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        tmp[idx] = (j < nb && col >= n && col < ce) ? A[(int64_t)(kb + j) * ld + col] : O::zero();
      }
      __syncthreads();
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        if (col >= ce) continue;
        T u;
        if (col < n) {
          u = (j < nb) ? O::mul(panel[j * NB + j], panel[(col - kb) * NB + j]) : O::zero();
        } else {
          u = tmp[j * TC + c];
          for (int i = 0; i < j; ++i) u = O::fma_acc(u, tri[j * NB + i], tmp[i * TC + c]);
          if (j < nb) A[(int64_t)(kb + j) * ld + col] = u;
        }
        tile[idx] = u;
      }
      __syncthreads();
      // matrix columns [c0, ce): the rows below the tile's diagonal block as one rectangle (every
      // lane of a warp runs the same rows), the block's lower triangle element by element;
      // right-hand-side columns: all rows below the panel
      const int cwp = tile_width_pow2(ce - c0);
      const int tc = t % cwp, tr = t / cwp;
      const int col = c0 + tc;
      if (col < ce) {
        const int rs = (col < n) ? max(kb + nb, ce) : kb + nb;
        rank_update<T>(A, ld, col, rs + tr, n, panel - (int64_t)kb * NB, tile + tc, nb, NT / cwp);
      }
      const int w = (c0 < n) ? ce - c0 : 0;
      for (int q = t; q < w * (w + 1) / 2; q += NT) {
        int rr = (int)((sqrtf(8.0f * (float)q + 1.0f) - 1.0f) * 0.5f);
        while (rr * (rr + 1) / 2 > q) --rr;
        while ((rr + 1) * (rr + 2) / 2 <= q) ++rr;
        const int cc = q - rr * (rr + 1) / 2;  // cc <= rr
        const int r = c0 + rr;
        T v = A[(int64_t)r * ld + c0 + cc];
        const T* l = panel + (int64_t)(r - kb) * NB;
#pragma unroll
        for (int j = 0; j < NB; ++j) v = O::fms(v, l[j], tile[j * TC + cc]);
        A[(int64_t)r * ld + c0 + cc] = v;
      }
      __syncthreads();
      c0 = ce;
    }
  }
  if (m == n || nf < n) return;
  // -------------------------------------------- D^-1, then back substitution
  for (int64_t idx = t; idx < (int64_t)n * (m - n); idx += NT) {
    const int i = (int)(idx / (m - n)), col = n + (int)(idx % (m - n));
    const T d = A[(int64_t)i * ld + i];
    A[(int64_t)i * ld + col] = (O::mag(d) == 0.0) ? O::zero() : O::mul(A[(int64_t)i * ld + col], O::inv(d));
  }
  __syncthreads();
  const int kb_last = ((n - 1) / NB) * NB;
  for (int kb = kb_last; kb >= 0; kb -= NB) {
    const int nb = min(NB, n - kb);
    const int rows = kb + nb;  // (L^T)[0 .. kb+nb)[kb .. kb+nb) = L[kb+c][r]
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      T v = O::zero();
      if (c < nb) {
        if (r < kb + c) v = A[(int64_t)(kb + c) * ld + r];
        else if (r == kb + c) v = O::one();
      }
      panel[idx] = v;
    }
    __syncthreads();
    // inverse of the unit-upper diagonal block, column t by thread t
    if (t < NB) {
      for (int i = 0; i < NB; ++i) tri[i * NB + t] = (i == t) ? O::one() : O::zero();
      if (t < nb) {
        const T* U = panel + (int64_t)kb * NB;
        for (int i = t - 1; i >= 0; --i) {
          T acc = O::zero();
          for (int k = i + 1; k <= t; ++k) acc = O::fms(acc, U[i * NB + k], tri[k * NB + t]);
          tri[i * NB + t] = acc;
        }
      }
    }
    __syncthreads();
    for (int c0 = n; c0 < m; c0 += TC) {
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        tmp[idx] = (j < nb && col < m) ? A[(int64_t)(kb + j) * ld + col] : O::zero();
      }
      __syncthreads();
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        if (col >= m) continue;
        T y = O::zero();
        for (int i = j; i < nb; ++i) y = O::fma_acc(y, tri[j * NB + i], tmp[i * TC + c]);
        tile[idx] = y;
        if (j < nb) A[(int64_t)(kb + j) * ld + col] = y;
      }
      __syncthreads();
      const int cwp = tile_width_pow2(m - c0);
      const int tc = t % cwp, tr = t / cwp;
      if (c0 + tc < m) rank_update<T>(A, ld, c0 + tc, tr, kb, panel, tile + tc, nb, NT / cwp);
      __syncthreads();
    }
  }
}

// Solve M X = P^T E for unit right-hand sides with the stored LU factors of M:
// column q of the block [n, n + no) of A gets the unit vector whose 1 sits
// at pivoted row posq[q] (sorted ascending), i.e. the interchanges are
// already applied.  L^-1 leaves a column zero above its 1, so panel kb of the
// forward elimination touches only the columns q with posq[q] < kb + nb --
// a prefix, because posq is sorted -- and the forward pass costs about n^3/3
// instead of n^2 no.  Back substitution as in lu_solve.
template <typename T>
__device__ void lu_unit_solve(T* __restrict__ A, int n, int no, int ld, T* panel, T* tile, T* tmp, T* tri,
                              const int* posq) {
  using O = Ops<T>;
  constexpr int NB = Blk<T>::NB;
  const int t = threadIdx.x;
  const int m = n + no;
  for (int64_t idx = t; idx < (int64_t)n * no; idx += NT) {
    const int r = (int)(idx / no), q = (int)(idx % no);
    A[(int64_t)r * ld + n + q] = (r == posq[q]) ? O::one() : O::zero();
  }
  __syncthreads();
  int active = 0;  // columns with their 1 above the current panel's end (uniform across the block)
  for (int kb = 0; kb < n; kb += NB) {
    const int nb = min(NB, n - kb);
    while (active < no && posq[active] < kb + nb) ++active;
    if (active == 0) continue;
    const int rows = n - kb;
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      panel[idx] = (c < nb) ? A[(int64_t)(kb + r) * ld + kb + c] : O::zero();
    }
    __syncthreads();
    if (t < NB) {
      for (int i = 0; i < NB; ++i) tri[i * NB + t] = (i == t) ? O::one() : O::zero();
      if (t < nb) {
        for (int i = t + 1; i < nb; ++i) {
          T acc = O::zero();
          for (int k = t; k < i; ++k) acc = O::fms(acc, panel[i * NB + k], tri[k * NB + t]);
          tri[i * NB + t] = acc;
        }
      }
    }
    __syncthreads();
    const int me = n + active;
    for (int c0 = n; c0 < me; c0 += TC) {
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        tmp[idx] = (j < nb && col < me) ? A[(int64_t)(kb + j) * ld + col] : O::zero();
      }
      __syncthreads();
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        if (col >= me) continue;
        T u = tmp[j * TC + c];
        for (int i = 0; i < j; ++i) u = O::fma_acc(u, tri[j * NB + i], tmp[i * TC + c]);
        tile[idx] = u;
        if (j < nb) A[(int64_t)(kb + j) * ld + col] = u;
      }
      __syncthreads();
      const int cwp = tile_width_pow2(me - c0);
      const int tc = t % cwp, tr = t / cwp;
      if (c0 + tc < me) rank_update<T>(A, ld, c0 + tc, kb + nb + tr, n, panel - (int64_t)kb * NB, tile + tc, nb, NT / cwp);
      __syncthreads();
    }
  }
  const int kb_last = ((n - 1) / NB) * NB;
  for (int kb = kb_last; kb >= 0; kb -= NB) {
    const int nb = min(NB, n - kb);
    const int rows = kb + nb;
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      panel[idx] = (c < nb) ? A[(int64_t)r * ld + kb + c] : O::zero();
    }
    __syncthreads();
    if (t < NB) {
      for (int i = 0; i < NB; ++i) tri[i * NB + t] = O::zero();
      if (t < nb) {
        const T* U = panel + (int64_t)kb * NB;
        const double dm = O::mag(U[t * NB + t]);
        tri[t * NB + t] = (dm == 0.0) ? O::zero() : O::inv(U[t * NB + t]);
        for (int i = t - 1; i >= 0; --i) {
          T acc = O::zero();
          for (int k = i + 1; k <= t; ++k) acc = O::fms(acc, U[i * NB + k], tri[k * NB + t]);
          const double di = O::mag(U[i * NB + i]);
          tri[i * NB + t] = (di == 0.0) ? O::zero() : O::mul(acc, O::inv(U[i * NB + i]));
        }
      }
    }
    __syncthreads();
    for (int c0 = n; c0 < m; c0 += TC) {
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        tmp[idx] = (j < nb && col < m) ? A[(int64_t)(kb + j) * ld + col] : O::zero();
      }
      __syncthreads();
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        if (col >= m) continue;
        T y = O::zero();
        for (int i = j; i < nb; ++i) y = O::fma_acc(y, tri[j * NB + i], tmp[i * TC + c]);
        tile[idx] = y;
        if (j < nb) A[(int64_t)(kb + j) * ld + col] = y;
      }
      __syncthreads();
      const int cwp = tile_width_pow2(m - c0);
      const int tc = t % cwp, tr = t / cwp;
      if (c0 + tc < m) rank_update<T>(A, ld, c0 + tc, tr, kb, panel, tile + tc, nb, NT / cwp);
      __syncthreads();
    }
  }
}

// ------------------------------------------------------------------------
// Mixed-precision matching solve: FP32 LU of [M | -B], then iterative
// refinement with residuals r = -B - M Y computed in double-float (FP32 hi +
// lo, error-free products and sums: about 48 bits) and corrections solved
// with the FP32 factors.  GB300 retires 64 FP32 FMAs for every FP64 FMA, so a
// double-float multiply-add (about 11 FP32 operations) costs about a sixth of
// an FP64 one, and the FP64 pipe is left to the complex S-step.

// s + e = a + b exactly
__device__ __forceinline__ void df_two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bb = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// Apply the stored LU factors (row interchanges ipiv, unit-lower L, upper U, in A) to the
// right-hand-side columns [n, m): all interchanges, forward elimination by panels, back
// substitution.
template <typename T>
__device__ void lu_resolve(T* __restrict__ A, int n, int m, int ld, T* panel, T* tile, T* tmp, T* tri,
                           const int* ipiv) {
  using O = Ops<T>;
  constexpr int NB = Blk<T>::NB;
  const int t = threadIdx.x;
  // the stored L is in the final row order: apply all interchanges to the right-hand sides first
  for (int col = n + t; col < m; col += NT) {
    for (int k = 0; k < n; ++k) {
      const int r2 = ipiv[k];
      if (r2 != k) {
        const T a1 = A[(int64_t)k * ld + col];
        A[(int64_t)k * ld + col] = A[(int64_t)r2 * ld + col];
        A[(int64_t)r2 * ld + col] = a1;
      }
    }
  }
  __syncthreads();
  for (int kb = 0; kb < n; kb += NB) {
    const int nb = min(NB, n - kb);
    const int rows = n - kb;
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      panel[idx] = (c < nb) ? A[(int64_t)(kb + r) * ld + kb + c] : O::zero();
    }
    __syncthreads();
    if (t < NB) {
      for (int i = 0; i < NB; ++i) tri[i * NB + t] = (i == t) ? O::one() : O::zero();
      if (t < nb) {
        for (int i = t + 1; i < nb; ++i) {
          T acc = O::zero();
          for (int k = t; k < i; ++k) acc = O::fms(acc, panel[i * NB + k], tri[k * NB + t]);
          tri[i * NB + t] = acc;
        }
      }
    }
    __syncthreads();
    for (int c0 = n; c0 < m; c0 += TC) {
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        tmp[idx] = (j < nb && col < m) ? A[(int64_t)(kb + j) * ld + col] : O::zero();
      }
      __syncthreads();
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        if (col >= m) continue;
        T u = tmp[j * TC + c];
        for (int i = 0; i < j; ++i) u = O::fma_acc(u, tri[j * NB + i], tmp[i * TC + c]);
        tile[idx] = u;
        if (j < nb) A[(int64_t)(kb + j) * ld + col] = u;
      }
      __syncthreads();
      const int cwp = tile_width_pow2(m - c0);
      const int tc = t % cwp, tr = t / cwp;
      if (c0 + tc < m) rank_update<T>(A, ld, c0 + tc, kb + nb + tr, n, panel - (int64_t)kb * NB, tile + tc, nb, NT / cwp);
      __syncthreads();
    }
  }
  const int kb_last = ((n - 1) / NB) * NB;
  for (int kb = kb_last; kb >= 0; kb -= NB) {
    const int nb = min(NB, n - kb);
    const int rows = kb + nb;
    for (int idx = t; idx < rows * NB; idx += NT) {
      const int r = idx / NB, c = idx % NB;
      panel[idx] = (c < nb) ? A[(int64_t)r * ld + kb + c] : O::zero();
    }
    __syncthreads();
    if (t < NB) {
      for (int i = 0; i < NB; ++i) tri[i * NB + t] = O::zero();
      if (t < nb) {
        const T* U = panel + (int64_t)kb * NB;
        const double dm = O::mag(U[t * NB + t]);
        tri[t * NB + t] = (dm == 0.0) ? O::zero() : O::inv(U[t * NB + t]);
        for (int i = t - 1; i >= 0; --i) {
          T acc = O::zero();
          for (int k = i + 1; k <= t; ++k) acc = O::fms(acc, U[i * NB + k], tri[k * NB + t]);
          const double di = O::mag(U[i * NB + i]);
          tri[i * NB + t] = (di == 0.0) ? O::zero() : O::mul(acc, O::inv(U[i * NB + i]));
        }
      }
    }
    __syncthreads();
    for (int c0 = n; c0 < m; c0 += TC) {
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        tmp[idx] = (j < nb && col < m) ? A[(int64_t)(kb + j) * ld + col] : O::zero();
      }
      __syncthreads();
      for (int idx = t; idx < NB * TC; idx += NT) {
        const int j = idx / TC, c = idx % TC, col = c0 + c;
        if (col >= m) continue;
        T y = O::zero();
        for (int i = j; i < nb; ++i) y = O::fma_acc(y, tri[j * NB + i], tmp[i * TC + c]);
        tile[idx] = y;
        if (j < nb) A[(int64_t)(kb + j) * ld + col] = y;
      }
      __syncthreads();
      const int cwp = tile_width_pow2(m - c0);
      const int tc = t % cwp, tr = t / cwp;
      if (c0 + tc < m) rank_update<T>(A, ld, c0 + tc, tr, kb, panel, tile + tc, nb, NT / cwp);
      __syncthreads();
    }
  }
}

// r = b - M y in double-float for the n x no block, b = A64[:, n + c] (FP64), M = Mh + Ml
// (n x n, ld ldm), y = Yh + Yl (n x no, ld ldy); r rounded to FP32 into R[i * ldr + c].
// 64 x 64 output tiles, 4 x 4 per thread, k-steps of 16 staged through 16 KB of shared memory.
__device__ void residual_df(const double* __restrict__ A64, int ldR, int n, int no, const float* __restrict__ Mh,
                            const float* __restrict__ Ml, int ldm, const float* __restrict__ Yh,
                            const float* __restrict__ Yl, int ldy, float* __restrict__ R, int ldr,
                            float* sM, float* sY) {
  constexpr int TT = 64, KR = 16;
  const int t = threadIdx.x;
  const int tx = t % 16, ty = t / 16;  // outputs rows ty*4.., cols tx*4..
  float* sMh = sM;                     // [TT][KR]
  float* sMl = sM + TT * KR;
  float* sYh = sY;                     // [KR][TT]
  float* sYl = sY + KR * TT;
  for (int i0 = 0; i0 < n; i0 += TT) {
    for (int c0 = 0; c0 < no; c0 += TT) {
      float sh[4][4], sl[4][4];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = i0 + ty * 4 + a, c = c0 + tx * 4 + b;
          const double v = (i < n && c < no) ? A64[(int64_t)i * ldR + n + c] : 0.0;
          const float h = (float)v;
          sh[a][b] = h;
          sl[a][b] = (float)(v - (double)h);
        }
      // each thread stages 4 elements of each operand per k-step; the next k-step's values are
      // loaded into registers before the current one is computed (latency hidden)
      float pm[4][2], py[4][2];
      auto fetch = [&](int k0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int idx = t + q * NT;
          const int r = idx / KR, k = idx % KR, i = i0 + r, j = k0 + k;
          const bool okm = i < n && j < n;
          pm[q][0] = okm ? Mh[(int64_t)i * ldm + j] : 0.0f;
          pm[q][1] = okm ? Ml[(int64_t)i * ldm + j] : 0.0f;
          const int ky = idx / TT, c = idx % TT, jy = k0 + ky, cc = c0 + c;
          const bool oky = jy < n && cc < no;
          py[q][0] = oky ? Yh[(int64_t)jy * ldy + cc] : 0.0f;
          py[q][1] = oky ? Yl[(int64_t)jy * ldy + cc] : 0.0f;
        }
      };
      fetch(0);
      for (int k0 = 0; k0 < n; k0 += KR) {
        __syncthreads();
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int idx = t + q * NT;
          sMh[idx] = pm[q][0];
          sMl[idx] = pm[q][1];
          sYh[idx] = py[q][0];
          sYl[idx] = py[q][1];
        }
        __syncthreads();
        if (k0 + KR < n) fetch(k0 + KR);
#pragma unroll 4
        for (int k = 0; k < KR; ++k) {
          const float4 yh = *reinterpret_cast<const float4*>(sYh + k * TT + tx * 4);
          const float4 yl = *reinterpret_cast<const float4*>(sYl + k * TT + tx * 4);
          const float yhv[4] = {yh.x, yh.y, yh.z, yh.w}, ylv[4] = {yl.x, yl.y, yl.z, yl.w};
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const float mh = sMh[(ty * 4 + a) * KR + k], ml = sMl[(ty * 4 + a) * KR + k];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
              const float p = __fmul_rn(mh, yhv[b]);
              float e = __fmaf_rn(mh, yhv[b], -p);
              e = __fmaf_rn(mh, ylv[b], __fmaf_rn(ml, yhv[b], e));
              float s, err;
              df_two_sum(sh[a][b], -p, s, err);
              sh[a][b] = s;
              sl[a][b] = __fsub_rn(__fadd_rn(sl[a][b], err), e);
            }
          }
        }
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          const int i = i0 + ty * 4 + a, c = c0 + tx * 4 + b;
          if (i < n && c < no) R[(int64_t)i * ldr + n + c] = __fadd_rn(sh[a][b], sl[a][b]);
        }
    }
  }
  __syncthreads();
}

struct SolveArgs {
  int n, n_sel;
  double a;
  const double* R;  // [ne * npR]: per energy [dipole row (y at 1..n)], then the n x n channel block
  int64_t npR;      // packed entries per energy
  int64_t roff;     // offset of the channel block (0 without a dipole row)
  int dip;          // 1: photoionisation amplitudes from y
  double e0;        // initial bound-state energy (Ry)
  int mixed;        // 1: matching solve in FP32 + double-float iterative refinement
  int lu_only;      // 1: no outgoing-wave path; every energy through LU
  int z_df;         // 1 (split-precision plans): Z factored in double-float and refined in FP64;
                    // 2: as 1, but every energy takes the FP64 fallback (test hook)
  int64_t mix_off;  // doubles from a slot's start to its mixed-precision area
  const double* asym;
  int64_t ld_asym;  // stride between lam, s, sp, c blocks
  const double* E;  // [ne]
  const double* thr;
  const int32_t* n_open_in;
  const uint8_t* flags_in;
  const int32_t* sel;
  int ne;
  double* slot;
  int64_t slot_doubles;
  int ldR;  // leading dimension of the real augmented matrix
  int ldC;  // leading dimension (complex elements) of the S-step matrix
  int n_slots;  // solve workspaces: one per CTA of the launch
  SolveOut out;
};

// The matching system [M | -B] of solve_energy by FP32 LU and double-float
// iterative refinement; on success the FP64 right-hand-side columns of A hold
// Y.  Returns false (A untouched) when the FP32 factorisation hits a zero
// pivot or the corrections stop contracting, and the caller solves in FP64.
__device__ bool mixed_matching(const SolveArgs& g, double* A, int n, int m, int no, unsigned char* panel_b,
                               unsigned char* tile_b, unsigned char* tmp_b, unsigned char* tri_b, int* ipiv,
                               Red& red, LUStat& st) {
  const int t = threadIdx.x;
  const int nmax = g.ldR / 2;
  float* A32 = reinterpret_cast<float*>(A + g.mix_off);
  float* Mh = A32 + (int64_t)nmax * g.ldR;
  float* Ml = Mh + (int64_t)nmax * nmax;
  float* Yh = Ml + (int64_t)nmax * nmax;
  float* Yl = Yh + (int64_t)nmax * nmax;
  for (int64_t idx = t; idx < (int64_t)n * m; idx += NT) {
    const int i = (int)(idx / m), j = (int)(idx % m);
    const double v = A[(int64_t)i * g.ldR + j];
    const float f = (float)v;
    A32[(int64_t)i * g.ldR + j] = f;
    if (j < n) {
      Mh[(int64_t)i * nmax + j] = f;
      Ml[(int64_t)i * nmax + j] = (float)(v - (double)f);
    }
  }
  __syncthreads();
  lu_solve<float>(A32, n, m, g.ldR, reinterpret_cast<float*>(panel_b), reinterpret_cast<float*>(tile_b),
                  reinterpret_cast<float*>(tmp_b), reinterpret_cast<float*>(tri_b), ipiv, &red, st);
  __shared__ int s_fail;
  if (t == 0) s_fail = st.singular ? 1 : 0;
  __syncthreads();
  if (s_fail) return false;
  for (int64_t idx = t; idx < (int64_t)n * no; idx += NT) {
    const int i = (int)(idx / no), c = (int)(idx % no);
    Yh[(int64_t)i * nmax + c] = A32[(int64_t)i * g.ldR + n + c];
    Yl[(int64_t)i * nmax + c] = 0.0f;
  }
  __syncthreads();
  float prev = INFINITY;
  bool conv = false;
  for (int it = 0; it < 5 && !conv; ++it) {
    residual_df(A, g.ldR, n, no, Mh, Ml, nmax, Yh, Yl, nmax, A32, g.ldR, reinterpret_cast<float*>(tile_b),
                reinterpret_cast<float*>(tmp_b));
    lu_resolve<float>(A32, n, m, g.ldR, reinterpret_cast<float*>(panel_b), reinterpret_cast<float*>(tile_b),
                      reinterpret_cast<float*>(tmp_b), reinterpret_cast<float*>(tri_b), ipiv);
    float dmax = 0.0f, ymax = 0.0f;
    for (int64_t idx = t; idx < (int64_t)n * no; idx += NT) {
      const int i = (int)(idx / no), c = (int)(idx % no);
      const int64_t q = (int64_t)i * nmax + c;
      const float d = A32[(int64_t)i * g.ldR + n + c];
      float s, e;
      df_two_sum(Yh[q], d, s, e);
      Yh[q] = s;
      Yl[q] = __fadd_rn(Yl[q], e);
      dmax = fmaxf(dmax, fabsf(d));
      ymax = fmaxf(ymax, fabsf(s));
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      dmax = fmaxf(dmax, __shfl_down_sync(0xffffffffu, dmax, off));
      ymax = fmaxf(ymax, __shfl_down_sync(0xffffffffu, ymax, off));
    }
    if ((t & 31) == 0) {
      red.v[t >> 5] = dmax;
      red.i[t >> 5] = __float_as_int(ymax);
    }
    __syncthreads();
    if (t == 0) {
      float dm = 0.0f, ym = 0.0f;
      for (int w = 0; w < NWARP; ++w) {
        dm = fmaxf(dm, (float)red.v[w]);
        ym = fmaxf(ym, __int_as_float(red.i[w]));
      }
      // converged: the last correction is below 1e-11 of the solution (a looser stop, 1e-8, let
      // single cross sections drift by 5e-8: elements of Y are more sensitive than its norm);
      // failed: the corrections stopped contracting
      red.piv = (dm <= 1e-11f * ym) ? 1 : ((dm < 0.5f * prev && isfinite(dm)) ? 0 : -1);
      red.v[0] = dm;
    }
    __syncthreads();
    const int verdict = red.piv;
    prev = (float)red.v[0];
    __syncthreads();
    if (verdict < 0) return false;
    conv = verdict > 0;
  }
  if (!conv) return false;
  for (int64_t idx = t; idx < (int64_t)n * no; idx += NT) {
    const int i = (int)(idx / no), c = (int)(idx % no);
    const int64_t q = (int64_t)i * nmax + c;
    A[(int64_t)i * g.ldR + n + c] = (double)Yh[q] + (double)Yl[q];
  }
  __syncthreads();
  return true;
}

// ------------------------------------------------------------------------
// Outgoing-wave symmetric solve (cross sections and eigenphase sum only).
//
// With M = R - diag(c / (a c')) on open channels and R - diag(1 / (a Lambda))
// on closed ones, the matching gives K = -diag(s'/c') - (1/a) C'^-1 X C'^-1,
// C' = diag(c'), X the open-open block of M^-1 = the inverse of the Schur
// complement S_oo = M_oo - M_oc M_cc^-1 M_co (Wronskian s c' - s' c = -1).
// Writing h = c + i s and G = S_oo + diag(c / (a c')) (R's open block less the
// closed channels' correction), the same algebra gives
//   (I - iK)^-1 = diag(c'/h') - (i/a) diag(1/h') Z^-1 diag(1/h'),
//   Z = G - diag(h / (a h'))   (complex symmetric, Im Z = diag(1/(a|h'|^2)) > 0),
// so T = S - I has T_ji = -(2i/a) (Z^-1)_ji / (h'_j h'_i) - 2i delta_ji s'_i / h'_i,
// and det(I - iK) = prod_j (c'_j h'_j) det Z / (det C'^2 det S_oo), whose
// argument needs only the sign of det S_oo: that of det S'' for the congruent
// S'' = V S_oo V = V G V - diag(c c' / (a |h'|^2)), V = diag(c' / |h'|), whose
// entries stay bounded where c and c' grow like (ka)^-l at thresholds, i.e.
// (-1)^(negative pivots of an LDL^T of S'').  Everything is regular where some
// c'_j vanishes.  The cost is a real LDL^T over the closed channels
// ((n^3 - n_o^3)/3 flops), one of S'' (n_o^3/3) and the complex one of Z
// ((4/3) n_o^3) against (2/3) n^3 + n^2 n_o + n^3/3 + (4/3) n_o^3 for LU, unit
// solves and the LDL^T of I - iK.  The real eliminations run without
// interchanges.  With D_pp = (|L||D||L^T|)_pp (it bounds the backward error of
// row p, and scales like the matrix under a diagonal congruence), max_p D_pp
// must stay within 1e4 of the largest entry of M for the closed elimination,
// which feeds Z (a backward error of at most about n u 1e4, below the split
// pole sum's error in R).  S'' decides only a sign, so it is factored in
// double-float first (pairs of floats, unit roundoff u_df = 2^-46 or so, on
// the FP32 pipe): its growth must stay within 1e4 of max|S''|, which keeps the
// backward error at about n u_df 1e4, so an eigenvalue would need to lie
// within about 4e-8 of zero (relative to max|S''|) to flip a sign.  If that
// fails, S'' is formed again and factored in FP64, where growth within 1e6
// gives the same margin (n u 1e6, about 3e-8).  Every pivot must keep
// |d_p| >= 1e-8 D_pp, far above its rounding error of about n u D_pp, so that
// no pivot is lost to cancellation.  An energy that fails a test is solved by
// the LU path.
constexpr double SYM_GROWTH_MAX = 1e4;             // closed elimination: max_p D_pp / max|M|
constexpr double SYM_GROWTH_MAX_INERTIA_DF = 1e4;  // S'' in double-float: max_p D_pp / max|S''|
constexpr double SYM_GROWTH_MAX_INERTIA = 1e6;     // S'' in FP64 (the retry)
constexpr double SYM_PIVOT_MIN = 1e-8;             // any of them: |d_p| / D_pp

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ double block_max(double v, Red& red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  if ((threadIdx.x & 31) == 0) red.v[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = red.v[0];
  for (int w = 1; w < NWARP; ++w) r = fmax(r, red.v[w]);
  __syncthreads();
  return r;
}

// fixed summation order: the same bits on every run
__device__ double block_sum(double v, Red& red) {
  v = warp_sum(v);
  if ((threadIdx.x & 31) == 0) red.v[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < NWARP; ++w) r += red.v[w];
  __syncthreads();
  return r;
}

// For the first nf pivots of an LDL^T held in A (L below the diagonal, d on
// it), with D_pp = sum_{k < min(p, nf)} L_pk^2 |d_k| (+ |d_p| for p < nf), the
// diagonal of |L||D||L^T|: gmax = max_p D_pp over all n rows and
// rmin = min_{p < nf} |d_p| / D_pp.  NaN counts as failing (gmax inf, rmin 0).
// One warp per row.
__device__ void ldl_check(const double* A, int n, int nf, int ld, Red& red, double& gmax, double& rmin) {
  const int lane = threadIdx.x & 31;
  double gm = 0.0, rm = INFINITY;
  for (int p = threadIdx.x >> 5; p < n; p += NWARP) {
    const int kend = min(p, nf);
    double acc = 0.0;
    for (int k = lane; k < kend; k += 32) {
      const double l = A[(int64_t)p * ld + k];
      acc = fma(l * l, fabs(A[(int64_t)k * ld + k]), acc);
    }
    acc = warp_sum(acc);
    if (p < nf) {
      const double d = fabs(A[(int64_t)p * ld + p]);
      acc += d;
      const double q = d / acc;
      rm = (q == q) ? fmin(rm, q) : 0.0;
    }
    gm = (acc == acc) ? fmax(gm, acc) : INFINITY;
  }
  gmax = block_max(gm, red);
  rmin = -block_max(-rm, red);
}

// ldl_check on double-float factors, from their high parts in FP32: the tests' thresholds (1e4, 1e-8)
// sit orders of magnitude away from FP32 rounding, and a non-finite sum fails them (the caller then
// factors in FP64), so no FP64 work is needed on the double-float path
__device__ void ldl_check_df(const dfl* A, int n, int nf, int ld, Red& red, double& gmax, double& rmin) {
  const int lane = threadIdx.x & 31;
  float gm = 0.0f, rm = INFINITY;
  for (int p = threadIdx.x >> 5; p < n; p += NWARP) {
    const int kend = min(p, nf);
    float acc = 0.0f;
    for (int k = lane; k < kend; k += 32) {
      const float l = A[(int64_t)p * ld + k].hi;
      acc = __fmaf_rn(__fmul_rn(l, l), fabsf(A[(int64_t)k * ld + k].hi), acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc = __fadd_rn(acc, __shfl_xor_sync(0xffffffffu, acc, o));
    if (p < nf) {
      const float d = fabsf(A[(int64_t)p * ld + p].hi);
      acc = __fadd_rn(acc, d);
      const float q = __fdiv_rn(d, acc);
      rm = (q == q) ? fminf(rm, q) : 0.0f;
    }
    gm = (acc == acc) ? fmaxf(gm, acc) : INFINITY;
  }
  gmax = block_max((double)gm, red);
  rmin = -block_max(-(double)rm, red);
}

// Photoionisation (a wave with a dipole row y): the boundary derivatives of the
// incoming-wave solutions are V = -(1/a) conj(Zhat)^-1 [diag(1/h'^*); 0], Zhat
// the full-channel form of Z, so M^-_m = sqrt(2) a (V^T y)_m
// = -sqrt(2) (conj(Zhat)^-1 y)_m / h'^*_m.  Eliminating the closed channels
// carries y along as a right-hand side (y_o - M_oc M_cc^-1 y_c, real), and
// conj(Z)^-1 of a real vector is the conjugate of Z^-1 of it, so
// |M^-_m|^2 = 2 |(Z^-1 y')_m|^2 / |h'_m|^2: one more right-hand side of Z.
//
// Returns true when energy e is finished (outputs written), false when its
// real eliminations fail the growth / pivot check and the caller must solve it
// by the LU path (the workspace is then free).
constexpr double Z_DF_CORR_MAX = 1e-7;  // refined double-float Z solve: largest accepted |d| / |x|

// Z x = e_sel (r unit right-hand sides) through the LDL^T of Z in double-float, then one step of
// iterative refinement: res = e_sel - Z x in FP64, Z d = res with the double-float factors,
// x += d.  Z is complex symmetric with a real off-diagonal part, so its FP64 copy is G (n x ld,
// row i, lower triangle: Re Z) plus its imaginary diagonal, kept in column no of G.  The factors'
// error in x is about n 2^-46 |K| (at a K pole |K| reaches 1e5, and double-float alone would leave
// T about 1e-7 out); after the step it is about that squared, so a correction below
// Z_DF_CORR_MAX of x leaves x at FP64 quality.  On success C holds, as FP64 complex values, what
// the FP64 factorisation leaves where the caller reads it: the pivots on the diagonal and x in
// columns no .. no + r.  Otherwise (false, uniform) C holds double-float factors and the caller
// forms Z again from G.
__device__ bool z_ldl_refined(cplx* C, int no, int r, int ldC, double* G, int ld, const int32_t* sel,
                              unsigned char* panel_b, unsigned char* tile_b, unsigned char* tmp_b,
                              unsigned char* tri_b, Red& red, bool force_fp64) {
  using O = Ops<cdf>;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int mc = no + r;
  // FP64 copy of Z: the real lower triangle and the imaginary diagonal
  for (int64_t idx = t; idx < (int64_t)no * no; idx += NT) {
    const int i = (int)(idx / no), j = (int)(idx % no);
    if (j > i) continue;
    const cplx v = C[(int64_t)i * ldC + j];
    G[(int64_t)i * ld + j] = v.re;
    if (j == i) G[(int64_t)i * ld + no] = v.im;
  }
  __syncthreads();
  // Z and the right-hand sides into double-float, in place
  cdf* Cd = reinterpret_cast<cdf*>(C);
  for (int64_t idx = t; idx < (int64_t)no * mc; idx += NT) {
    const int i = (int)(idx / mc), j = (int)(idx % mc);
    if (j < no && j > i) continue;
    const cplx v = C[(int64_t)i * ldC + j];
    Cd[(int64_t)i * ldC + j] = cdf{df_from_fast(v.re), df_from_fast(v.im)};
  }
  __syncthreads();
  LUStat st;
  ldl_solve<cdf>(Cd, no, mc, ldC, reinterpret_cast<cdf*>(panel_b), reinterpret_cast<cdf*>(tile_b),
                 reinterpret_cast<cdf*>(tmp_b), reinterpret_cast<cdf*>(tri_b), st);
  __syncthreads();
  // the panel area (a 128-byte row per channel) holds, per group of four right-hand sides,
  // x in FP64 (slots 0-3) and the residual, then the correction, in double-float (slots 4-7)
  cplx* xs = reinterpret_cast<cplx*>(panel_b);
  cdf* ys = reinterpret_cast<cdf*>(panel_b);
  bool good = true;
  for (int q0 = 0; q0 < r; q0 += 4) {
    const int nq = min(4, r - q0);
    for (int idx = t; idx < no * nq; idx += NT) {
      const int i = idx / nq, q = idx % nq;
      const cdf v = Cd[(int64_t)i * ldC + no + q0 + q];
      xs[i * 8 + q] = cplx{df_to(v.re), df_to(v.im)};
    }
    __syncthreads();
    // res = e - Z x, a warp per row: (Z x)_i = sum_j Re Z_ij x_j + i Im Z_ii x_i
    for (int i = warp; i < no; i += NWARP) {
      for (int q = 0; q < nq; ++q) {
        double ar = 0.0, ai = 0.0;
        for (int j = lane; j < no; j += 32) {
          const double z = (j <= i) ? G[(int64_t)i * ld + j] : G[(int64_t)j * ld + i];
          const cplx xv = xs[j * 8 + q];
          ar = fma(z, xv.re, ar);
          ai = fma(z, xv.im, ai);
        }
        ar = warp_sum(ar);
        ai = warp_sum(ai);
        if (lane == 0) {
          const double zi = G[(int64_t)i * ld + no];
          const cplx xi = xs[i * 8 + q];
          const double ev = (sel[q0 + q] == i) ? 1.0 : 0.0;
          ys[i * 8 + 4 + q] = cdf{df_from(ev - fma(-zi, xi.im, ar)), df_from(-fma(zi, xi.re, ai))};
        }
      }
    }
    __syncthreads();
    // d = L^-T D^-1 L^-1 res with the double-float factors (L unit lower, by columns, then rows)
    for (int k = 0; k + 1 < no; ++k) {
      for (int idx = t; idx < (no - 1 - k) * nq; idx += NT) {
        const int i = k + 1 + idx / nq, q = idx % nq;
        ys[i * 8 + 4 + q] = O::fms(ys[i * 8 + 4 + q], Cd[(int64_t)i * ldC + k], ys[k * 8 + 4 + q]);
      }
      __syncthreads();
    }
    for (int idx = t; idx < no * nq; idx += NT) {
      const int i = idx / nq, q = idx % nq;
      ys[i * 8 + 4 + q] = O::mul(ys[i * 8 + 4 + q], O::inv(Cd[(int64_t)i * ldC + i]));
    }
    __syncthreads();
    for (int k = no - 1; k > 0; --k) {
      for (int idx = t; idx < k * nq; idx += NT) {
        const int i = idx / nq, q = idx % nq;
        ys[i * 8 + 4 + q] = O::fms(ys[i * 8 + 4 + q], Cd[(int64_t)k * ldC + i], ys[k * 8 + 4 + q]);
      }
      __syncthreads();
    }
    // x += d, into C's solution columns (their double-float values are no longer needed)
    double dmax = 0.0, xmax = 0.0;
    for (int idx = t; idx < no * nq; idx += NT) {
      const int i = idx / nq, q = idx % nq;
      const cdf d = ys[i * 8 + 4 + q];
      const double dr = df_to(d.re), di = df_to(d.im);
      const cplx x = xs[i * 8 + q];
      const cplx xn = cplx{x.re + dr, x.im + di};
      dmax = fmax(dmax, fabs(dr) + fabs(di));
      xmax = fmax(xmax, fabs(xn.re) + fabs(xn.im));
      C[(int64_t)i * ldC + no + q0 + q] = xn;
      if (!(fabs(dr) + fabs(di) <= 1e300)) dmax = INFINITY;  // NaN from a zero pivot
    }
    dmax = block_max(dmax, red);
    xmax = block_max(xmax, red);
    if (!(dmax <= Z_DF_CORR_MAX * xmax)) good = false;
  }
  if (!good || force_fp64) return false;
  // the pivots, in FP64, on the diagonal
  for (int i = t; i < no; i += NT) {
    const cdf d = Cd[(int64_t)i * ldC + i];
    C[(int64_t)i * ldC + i] = cplx{df_to(d.re), df_to(d.im)};
  }
  __syncthreads();
  return true;
}

__device__ bool sym_xsec(const SolveArgs& g, int e, int no, uint8_t fl, unsigned char* smem_raw, Red& red) {
  const int n = g.n, nc = n - no, t = threadIdx.x, lane = t & 31;
  unsigned char* panel_b = smem_raw;
  unsigned char* tile_b = panel_b + (size_t)n * PANEL_ROW_BYTES;
  unsigned char* tmp_b = tile_b + TILE_BYTES;
  unsigned char* tri_b = tmp_b + TILE_BYTES;
  double* A = g.slot + (int64_t)blockIdx.x * g.slot_doubles;
  cplx* C = reinterpret_cast<cplx*>(A + (int64_t)n * g.ldR);
  const int ld = g.ldR;
  const double* Re = g.R + (int64_t)e * g.npR + g.roff;
  const double* lam = g.asym + 0 * g.ld_asym + (int64_t)e * n;
  const double* s = g.asym + 1 * g.ld_asym + (int64_t)e * n;
  const double* sp = g.asym + 2 * g.ld_asym + (int64_t)e * n;
  const double* c = g.asym + 3 * g.ld_asym + (int64_t)e * n;
  const bool photo = g.dip && (g.out.pi_tot || g.out.pi_ch);
  const double* ye = g.R + (int64_t)e * g.npR + 1;  // dipole vector y_i (rows with a dipole)
  // ------------------------------------- M, lower triangle, channels reversed (closed first)
  double gm = 0.0;
  for (int p = t >> 5; p < n; p += NWARP) {
    const int i = n - 1 - p;
    const double* Rrow = Re + pair_index(n, i, i);  // R_ij, j >= i, at Rrow[j - i]
    for (int q = lane; q <= p; q += 32) {
      const int j = n - 1 - q;
      double v = Rrow[j - i];
      if (q == p && i >= no) v -= 1.0 / (g.a * lam[i]);
      if (RM_CHECK(q < ld && pair_index(n, i, j) < g.npR - g.roff)) A[(int64_t)p * ld + q] = v;
      gm = fmax(gm, fabs(v));
    }
  }
  if (photo)  // the dipole vector as column n, channels reversed
    for (int p = t; p < n; p += NT) A[(int64_t)p * ld + n] = ye[n - 1 - p];
  gm = block_max(gm, red);
  LUStat st;
  double growth_c = 0.0, piv_c = INFINITY;
  if (nc > 0) {
    ldl_solve<double>(A, n, photo ? n + 1 : n, ld, reinterpret_cast<double*>(panel_b),
                      reinterpret_cast<double*>(tile_b), reinterpret_cast<double*>(tmp_b),
                      reinterpret_cast<double*>(tri_b), st, nc);
    ldl_check(A, n, nc, ld, red, growth_c, piv_c);
    growth_c /= gm;
  }
  // ------------------------------------- Z = G - diag(h / (a h')), unit right-hand sides, y'
  const int r = g.n_sel, mc = no + r + (photo ? 1 : 0);
  for (int64_t idx = t; idx < (int64_t)no * mc; idx += NT) {
    const int i = (int)(idx / mc), j = (int)(idx % mc);
    cplx v;
    if (j < no) {
      if (j > i) continue;  // the LDL^T reads the lower triangle only
      v = cplx{A[(int64_t)(n - 1 - j) * ld + (n - 1 - i)], 0.0};
      if (i == j) {
        const double cp = lam[i] * c[i];
        const double den = g.a * (cp * cp + sp[i] * sp[i]);
        v.re -= (c[i] * cp + s[i] * sp[i]) / den;  // h / h' = (c c' + s s' + i (s c' - c s')) / |h'|^2
        v.im -= (s[i] * cp - c[i] * sp[i]) / den;
      }
    } else if (j < no + r) {
      v = cplx{(g.sel[j - no] == i) ? 1.0 : 0.0, 0.0};
    } else {
      v = cplx{A[(int64_t)(n - 1 - i) * ld + n], 0.0};
    }
    if (RM_CHECK(j < g.ldC)) C[(int64_t)i * g.ldC + j] = v;
  }
  __syncthreads();
  // ------------------------------------- S'' = V G V - diag(c c' / (a |h'|^2)), in place, and its inertia
  double* As = A + (int64_t)nc * ld + nc;
  double* vsc = reinterpret_cast<double*>(tile_b);  // V_jj = c'_j / |h'_j| (tile area free until the LDL^T)
  // from_z: S_oo taken from Z's real part (C, not yet factored) instead of the eliminated block
  auto form_s2 = [&](bool from_z) {
    for (int j = t; j < no; j += NT) {
      const double cp = lam[j] * c[j];
      vsc[j] = cp / sqrt(cp * cp + sp[j] * sp[j]);
    }
    __syncthreads();
    double m = 0.0;
    for (int p = t >> 5; p < no; p += NWARP) {
      const int i = no - 1 - p;
      for (int q = lane; q <= p; q += 32) {
        const int j = no - 1 - q;
        double x = from_z ? C[(int64_t)j * g.ldC + i].re : As[(int64_t)p * ld + q];
        double v;
        if (q == p) {
          const double cp = lam[i] * c[i];
          const double den = g.a * (cp * cp + sp[i] * sp[i]);
          if (from_z) x += (c[i] * cp + s[i] * sp[i]) / den;  // undo Z's diagonal term h / (a h')
          v = vsc[i] * x * vsc[j] - c[i] * cp / den;
        } else {
          v = vsc[i] * x * vsc[j];
        }
        As[(int64_t)p * ld + q] = v;
        m = fmax(m, fabs(v));
      }
    }
    return block_max(m, red);
  };
  double growth_s, piv_s;
  auto negatives = [&]() {
    int neg = 0;
    for (int p = t; p < no; p += NT) neg += (As[(int64_t)p * ld + p] < 0.0) ? 1 : 0;
    return block_sum((double)neg, red);
  };
  double sm = form_s2(false);
  // S'' decides only signs (its inertia), with pivot and growth tests that leave a margin far
  // above double-float rounding (|d_p| >= 1e-8 D_pp against a backward error of about
  // n 2^-46 D_pp), so it is factored in double-float on the FP32 pipe, in place (same size),
  // then turned back into FP64 for the tests and the sign count
  dfl* Ad = reinterpret_cast<dfl*>(As);
  for (int p = t >> 5; p < no; p += NWARP)
    for (int q = lane; q <= p; q += 32) Ad[(int64_t)p * ld + q] = df_from_fast(As[(int64_t)p * ld + q]);
  __syncthreads();
  ldl_solve<dfl>(Ad, no, no, ld, reinterpret_cast<dfl*>(panel_b), reinterpret_cast<dfl*>(tile_b),
                 reinterpret_cast<dfl*>(tmp_b), reinterpret_cast<dfl*>(tri_b), st);
  __syncthreads();
  // the growth and pivot tests and the sign count on the factors' high parts, in FP32
  ldl_check_df(Ad, no, no, ld, red, growth_s, piv_s);
  growth_s /= sm;
  double negs;
  {
    int neg = 0;
    for (int p = t; p < no; p += NT) neg += (Ad[(int64_t)p * ld + p].hi < 0.0f) ? 1 : 0;
    negs = block_sum((double)neg, red);
  }
  const bool ok_c = (growth_c <= SYM_GROWTH_MAX) && (piv_c >= SYM_PIVOT_MIN);
  if (ok_c && !(growth_s <= SYM_GROWTH_MAX_INERTIA_DF && piv_s >= SYM_PIVOT_MIN)) {
    // the double-float factorisation is not trusted for this S'': form it again and factor in FP64
    sm = form_s2(true);
    ldl_solve<double>(As, no, no, ld, reinterpret_cast<double*>(panel_b), reinterpret_cast<double*>(tile_b),
                      reinterpret_cast<double*>(tmp_b), reinterpret_cast<double*>(tri_b), st);
    ldl_check(As, no, no, ld, red, growth_s, piv_s);
    growth_s /= sm;
    negs = negatives();
    fl |= RM_FLAG_FP64;
  }
  const bool ok = ok_c && (growth_s <= SYM_GROWTH_MAX_INERTIA) && (piv_s >= SYM_PIVOT_MIN);
  if (!ok) return false;  // uniform: the values come from block reductions
  // ------------------------------------- complex LDL^T of Z, x = Z^-1 e_sel
  // Split-precision plans: in double-float with one FP64 refinement step (z_ldl_refined; G: the
  // S'' block, free once its inertia is counted); FP64 for FP64 plans, for dipole waves and where
  // the refinement's correction is large.
  bool z_done = false;
  if (!photo && g.z_df) {
    z_done = z_ldl_refined(C, no, r, g.ldC, As, ld, g.sel, panel_b, tile_b, tmp_b, tri_b, red, g.z_df == 2);
    if (!z_done) {
      // Z again from its FP64 copy in G, with the unit right-hand sides
      for (int64_t idx = t; idx < (int64_t)no * mc; idx += NT) {
        const int i = (int)(idx / mc), j = (int)(idx % mc);
        cplx v;
        if (j < no) {
          if (j > i) continue;
          v = cplx{As[(int64_t)i * ld + j], (j == i) ? As[(int64_t)i * ld + no] : 0.0};
        } else {
          v = cplx{(g.sel[j - no] == i) ? 1.0 : 0.0, 0.0};
        }
        C[(int64_t)i * g.ldC + j] = v;
      }
      __syncthreads();
      fl |= RM_FLAG_FP64;
    }
  }
  if (!z_done)
    ldl_solve<cplx>(C, no, mc, g.ldC, reinterpret_cast<cplx*>(panel_b), reinterpret_cast<cplx*>(tile_b),
                    reinterpret_cast<cplx*>(tmp_b), reinterpret_cast<cplx*>(tri_b), st);
  // eta = -arg det(I - iK) = -(sum_j [arg h'_j + arg d_j + pi (c'_j < 0)] - pi neg(S''))  (mod 2 pi)
  double ph = 0.0;
  for (int j = t; j < no; j += NT) {
    const double cp = lam[j] * c[j];
    const cplx d = C[(int64_t)j * g.ldC + j];
    ph += atan2(sp[j], cp) + atan2(d.im, d.re) + ((cp < 0.0) ? M_PI : 0.0);
  }
  ph = block_sum(ph, red) - M_PI * negs;
  if (t == 0) {
    if (g.out.flags) g.out.flags[e] = fl;
    if (g.out.n_open) g.out.n_open[e] = no;
    if (g.out.eta) {
      double eta = -ph;
      eta = eta - 2.0 * M_PI * floor((eta + M_PI) / (2.0 * M_PI));  // [-pi, pi)
      if (eta == -M_PI) eta = M_PI;
      g.out.eta[e] = eta;
    }
  }
  // sigma_{i -> j} = (pi / k_i^2) |T_ji|^2 = (4 pi / k_i^2) |x_j / (a h'_j h'_i) + delta_ji s'_i / h'_i|^2
  for (int q = 0; q < r; ++q) {
    const int i = g.sel[q];
    const bool open_i = i < no;
    const double k2 = g.E[e] - g.thr[min(i, n - 1)];
    double part = 0.0;
    for (int j = t; j < n; j += NT) {
      double sig = 0.0;
      if (open_i && j < no) {
        const double cpi = lam[i] * c[i], cpj = lam[j] * c[j];
        const double di = cpi * cpi + sp[i] * sp[i], dj = cpj * cpj + sp[j] * sp[j];
        const cplx hi_inv = cplx{cpi / di, -sp[i] / di}, hj_inv = cplx{cpj / dj, -sp[j] / dj};
        const cplx x = C[(int64_t)j * g.ldC + no + q];
        cplx u = x * hj_inv * hi_inv;
        u = cplx{u.re / g.a, u.im / g.a};
        if (j == i) u = u + cplx{sp[i] * hi_inv.re, sp[i] * hi_inv.im};
        sig = 4.0 * M_PI / k2 * (u.re * u.re + u.im * u.im);
      }
      if (g.out.sig_sel) g.out.sig_sel[((int64_t)e * r + q) * n + j] = sig;
      part += sig;
    }
    part = block_sum(part, red);
    if (t == 0 && g.out.sig_tot) g.out.sig_tot[(int64_t)e * r + q] = part;
  }
  if (photo) {
    // sigma_PI,j = (4 pi alpha / 3) omega |M^-_j|^2 = (4 pi alpha / 3) omega 2 |x_j|^2 / |h'_j|^2
    const double pref = (4.0 * M_PI * 7.2973525693e-3 / 3.0) * (g.E[e] - g.e0);
    double part = 0.0;
    for (int j = t; j < n; j += NT) {
      double v = 0.0;
      if (j < no) {
        const double cp = lam[j] * c[j];
        const cplx x = C[(int64_t)j * g.ldC + no + r];
        v = pref * 2.0 * (x.re * x.re + x.im * x.im) / (cp * cp + sp[j] * sp[j]);
      }
      if (g.out.pi_ch) g.out.pi_ch[(int64_t)e * n + j] = v;
      part += v;
    }
    part = block_sum(part, red);
    if (t == 0 && g.out.pi_tot) g.out.pi_tot[e] = part;
  }
  __syncthreads();
  return true;
}

// One energy e of the argument block: build the matching system from R and the
// asymptotic data, LU -> K, then (optionally) the complex S-step.
template <bool MIXED>
__device__ void solve_energy(const SolveArgs& g, int e, unsigned char* smem_raw, Red& red, double& s_acc) {
  const int n = g.n;
  // shared by both LUs: panel n x 128 B, tile and tmp 8 KB each, tri 2 KB, ipiv
  unsigned char* panel_b = smem_raw;
  unsigned char* tile_b = panel_b + (size_t)n * PANEL_ROW_BYTES;
  unsigned char* tmp_b = tile_b + TILE_BYTES;
  unsigned char* tri_b = tmp_b + TILE_BYTES;
  int* ipiv = reinterpret_cast<int*>(tri_b + TRI_BYTES);
  int* perm = ipiv + g.ldR / 2;  // [n_max] row permutation, then sorted unit positions / channels
  int* posq = perm + g.ldR / 2;
  int* chq = posq + g.ldR / 2;
  cplx* panel_c = reinterpret_cast<cplx*>(panel_b);
  cplx* tile_c = reinterpret_cast<cplx*>(tile_b);
  cplx* tmp_c = reinterpret_cast<cplx*>(tmp_b);
  cplx* tri_c = reinterpret_cast<cplx*>(tri_b);
  double* panel_d = reinterpret_cast<double*>(panel_b);
  double* tile_d = reinterpret_cast<double*>(tile_b);
  double* A = g.slot + (int64_t)blockIdx.x * g.slot_doubles;
  cplx* C = reinterpret_cast<cplx*>(A + (int64_t)n * g.ldR);
  const int t = threadIdx.x;
  // this CTA's workspace and energy (uniform over the block): the real n x ldR matrix and the
  // complex n x ldC one must fit the slot, the energy must lie in the launch's range
  if (!RM_CHECK((int)blockIdx.x < g.n_slots && e >= 0 && e < g.ne && n <= g.ldR / 2 &&
                (int64_t)n * g.ldR + 2 * (int64_t)n * g.ldC <= g.slot_doubles))
    return;

  const int no = g.n_open_in[e];
  uint8_t fl = g.flags_in[e];
  const double* Re = g.R + (int64_t)e * g.npR + g.roff;
  const double* ye = g.R + (int64_t)e * g.npR + 1;  // dipole vector y_i (rows with a dipole)
  const double* lam = g.asym + 0 * g.ld_asym + (int64_t)e * n;
  const double* s = g.asym + 1 * g.ld_asym + (int64_t)e * n;
  const double* sp = g.asym + 2 * g.ld_asym + (int64_t)e * n;
  const double* c = g.asym + 3 * g.ld_asym + (int64_t)e * n;
  if (g.out.K) {
    for (int64_t idx = t; idx < (int64_t)n * n; idx += NT) g.out.K[(int64_t)e * n * n + idx] = 0.0;
  }
  if (no == 0) {
    fl |= RM_FLAG_NO_OPEN;
    if (t == 0) {
      if (g.out.flags) g.out.flags[e] = fl;
      if (g.out.n_open) g.out.n_open[e] = 0;
      if (g.out.eta) g.out.eta[e] = 0.0;
    }
    if (g.out.sig_tot)
      for (int q = t; q < g.n_sel; q += NT) g.out.sig_tot[(int64_t)e * g.n_sel + q] = 0.0;
    if (g.out.sig_sel)
      for (int64_t idx = t; idx < (int64_t)g.n_sel * n; idx += NT)
        g.out.sig_sel[(int64_t)e * g.n_sel * n + idx] = 0.0;
    if (g.out.pi_tot && t == 0) g.out.pi_tot[e] = 0.0;
    if (g.out.pi_ch)
      for (int j = t; j < n; j += NT) g.out.pi_ch[(int64_t)e * n + j] = 0.0;
    __syncthreads();
    return;
  }
  if constexpr (!MIXED) {
    if (g.out.do_xsec && !g.out.K && !g.lu_only) {
      if (sym_xsec(g, e, no, fl, smem_raw, red)) return;
      fl |= RM_FLAG_LU;
    }
  }
  // Unit right-hand sides: with the Wronskian s c' - s' c = -1, B = M D + diag(1/c') on the open
  // columns, D = diag(c s' / c'), so Y = -D + M^-1 diag(1/c') and only M^-1 on unit columns is
  // needed (lu_unit_solve: forward pass n^3/3 instead of n^2 n_o).  It divides by c'_m; the error
  // of K grows only like 1e-17 k^1/2 / |c'_m| (measured down to |c'| = 2e-5 k^1/2: 3e-13), and an
  // energy with |c'_m| < 1e-6 k_m^1/2 in some open channel keeps the dense right-hand sides.
  bool unit = false;
  if constexpr (!MIXED) {
    int bad = 0;
    for (int j = t; j < no; j += NT) {
      const double cp = lam[j] * c[j];
      const double k = sqrt(g.E[e] - g.thr[j]);
      if (!(fabs(cp) >= 1e-6 * sqrt(k))) bad = 1;
    }
    unit = !__syncthreads_or(bad);
  }
  // ---------------------------------------------------------------- build
  const int m = n + no;
  for (int64_t idx = t; idx < (int64_t)n * (unit ? n : m); idx += NT) {
    const int i = (int)(idx / (unit ? n : m)), j = (int)(idx % (unit ? n : m));
    double v;
    if (j < n) {
      const double rij = Re[pair_index(n, min(i, j), max(i, j))];
      v = ((i == j) ? 1.0 : 0.0) - g.a * rij * lam[j];
    } else {
      const int mo = j - n;
      const double rim = Re[pair_index(n, min(i, mo), max(i, mo))];
      v = -(((i == mo) ? s[mo] : 0.0) - g.a * rim * sp[mo]);
    }
    if (RM_CHECK(j < g.ldR)) A[(int64_t)i * g.ldR + j] = v;
  }
  __syncthreads();
  LUStat st;
  bool solved = false;
  if constexpr (MIXED) {
    solved = mixed_matching(g, A, n, m, no, panel_b, tile_b, tmp_b, tri_b, ipiv, red, st);
    if (!solved) fl |= RM_FLAG_FP64;
  }
  if (!solved && unit) {
    lu_solve<double>(A, n, n, g.ldR, panel_d, tile_d, reinterpret_cast<double*>(tmp_c),
                     reinterpret_cast<double*>(tri_c), ipiv, &red, st);
    // pivoted row of each open channel's unit vector, channels sorted by it
    if (t == 0) {
      for (int r = 0; r < n; ++r) perm[r] = r;
      for (int k = 0; k < n; ++k) {
        const int p2 = ipiv[k];
        const int tmpv = perm[k];
        perm[k] = perm[p2];
        perm[p2] = tmpv;
      }
      int q = 0;
      for (int r = 0; r < n; ++r)
        if (perm[r] < no) {
          posq[q] = r;
          chq[q] = perm[r];
          ++q;
        }
    }
    __syncthreads();
    lu_unit_solve<double>(A, n, no, g.ldR, panel_d, tile_d, reinterpret_cast<double*>(tmp_c),
                          reinterpret_cast<double*>(tri_c), posq);
    // X (columns in sorted order) -> Y_im = X_i,m / c'_m - delta_im c_m s'_m / c'_m in channel order,
    // through the complex area (free until the S-step)
    double* X = reinterpret_cast<double*>(C);
    for (int64_t idx = t; idx < (int64_t)n * no; idx += NT) {
      const int i = (int)(idx / no), q = (int)(idx % no);
      X[idx] = A[(int64_t)i * g.ldR + n + q];
    }
    __syncthreads();
    for (int64_t idx = t; idx < (int64_t)n * no; idx += NT) {
      const int i = (int)(idx / no), q = (int)(idx % no);
      const int mch = chq[q];
      const double cp = lam[mch] * c[mch];
      double y = X[idx] / cp;
      if (i == mch) y -= c[mch] * sp[mch] / cp;
      A[(int64_t)i * g.ldR + n + mch] = y;
    }
    __syncthreads();
    solved = true;
  }
  if (!solved)
    lu_solve<double>(A, n, m, g.ldR, panel_d, tile_d, reinterpret_cast<double*>(tmp_c),
                     reinterpret_cast<double*>(tri_c), ipiv, &red, st);
  __shared__ int s_singular;
  __shared__ double s_ratio;
  if (t == 0) {
    s_singular = st.singular ? 1 : 0;
    s_ratio = (st.pmax > 0.0) ? st.pmin / st.pmax : 0.0;
  }
  __syncthreads();
  if (s_singular) fl |= RM_FLAG_SINGULAR;
  else if (s_ratio < 1e-12) fl |= RM_FLAG_ILLCOND;
  // K_jm = Y_jm / c_j, with one reciprocal per row (kept in the free tmp area)
  double* rc = reinterpret_cast<double*>(tmp_c);
  for (int i = t; i < no; i += NT) rc[i] = 1.0 / c[i];
  __syncthreads();
  if (g.out.K) {
    for (int64_t idx = t; idx < (int64_t)no * no; idx += NT) {
      const int j = (int)(idx / no), mo = (int)(idx % no);
      g.out.K[(int64_t)e * n * n + (int64_t)j * n + mo] = A[(int64_t)j * g.ldR + n + mo] * rc[j];
    }
  }
  if (t == 0) {
    if (g.out.flags) g.out.flags[e] = fl;
    if (g.out.n_open) g.out.n_open[e] = no;
  }
  if (!g.out.do_xsec) {
    __syncthreads();
    return;
  }
  // ---------------------------------------------------- dipole amplitudes
  const bool photo = g.dip && (g.out.pi_tot || g.out.pi_ch);
  double* MK = tile_d;  // the tile area is free between the two LUs
  if (photo) {
    for (int m = t; m < no; m += NT) {
      double acc = sp[m] * ye[m];
      for (int i = 0; i < n; ++i) acc = fma(lam[i] * A[(int64_t)i * g.ldR + n + m], ye[i], acc);
      MK[m] = M_SQRT2 * g.a * acc;
    }
    __syncthreads();  // the complex build below reads every M^K_i (photo is uniform in the block)
  }
  // --------------------------------------------------------------- S-step
  const int r = g.n_sel;
  const int mc = no + r + (photo ? 1 : 0);
  for (int64_t idx = t; idx < (int64_t)no * mc; idx += NT) {
    const int i = (int)(idx / mc), j = (int)(idx % mc);
    cplx v;
    if (j < no) {
      if (j > i) continue;  // the LDL^T reads the lower triangle only
      const double kij = A[(int64_t)i * g.ldR + n + j] * rc[i];
      v = cplx{(i == j) ? 1.0 : 0.0, -kij};
    } else if (j < no + r) {
      const int sq = g.sel[j - no];
      v = cplx{(sq < no) ? A[(int64_t)i * g.ldR + n + sq] * rc[i] : 0.0, 0.0};
    } else {
      v = cplx{MK[i], 0.0};
    }
    if (RM_CHECK(j < g.ldC)) C[(int64_t)i * g.ldC + j] = v;
  }
  __syncthreads();
  ldl_solve<cplx>(C, no, mc, g.ldC, panel_c, tile_c, tmp_c, tri_c, st);
  if (t == 0 && g.out.eta) {
    double ph = 0.0;  // det(I - iK) = prod d_j (no interchanges)
    for (int j = 0; j < no; ++j) {
      const cplx d = C[(int64_t)j * g.ldC + j];
      ph += atan2(d.im, d.re);
    }
    double eta = -ph;
    eta = eta - 2.0 * M_PI * floor((eta + M_PI) / (2.0 * M_PI));  // [-pi, pi)
    if (eta == -M_PI) eta = M_PI;
    g.out.eta[e] = s_singular ? NAN : eta;
  }
  for (int q = 0; q < r; ++q) {
    const int sq = g.sel[q];
    const bool open_i = sq < no;
    const double k2 = g.E[e] - g.thr[min(sq, n - 1)];
    double part = 0.0;
    for (int j = t; j < n; j += NT) {
      double sig = 0.0;
      if (open_i && j < no) {
        const cplx x = C[(int64_t)j * g.ldC + no + q];
        sig = 4.0 * M_PI / k2 * (x.re * x.re + x.im * x.im);
      }
      if (s_singular) sig = NAN;
      if (g.out.sig_sel) g.out.sig_sel[((int64_t)e * r + q) * n + j] = sig;
      part += sig;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((t & 31) == 0) red.v[t >> 5] = part;
    __syncthreads();
    if (t == 0) {
      double tot = 0.0;  // fixed order: the same bits on every run
      for (int w = 0; w < NWARP; ++w) tot += red.v[w];
      if (g.out.sig_tot) g.out.sig_tot[(int64_t)e * r + q] = tot;
    }
    __syncthreads();
  }
  if (photo) {
    // sigma_PI,j = (4 pi alpha / 3) omega |X_j|^2, X = (I - iK)^-1 M^K
    const double pref = (4.0 * M_PI * 7.2973525693e-3 / 3.0) * (g.E[e] - g.e0);
    double part = 0.0;
    for (int j = t; j < n; j += NT) {
      double v = 0.0;
      if (j < no) {
        const cplx x = C[(int64_t)j * g.ldC + no + r];
        v = pref * (x.re * x.re + x.im * x.im);
      }
      if (s_singular) v = NAN;
      if (g.out.pi_ch) g.out.pi_ch[(int64_t)e * n + j] = v;
      part += v;
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) part += __shfl_down_sync(0xffffffffu, part, off);
    if ((t & 31) == 0) red.v[t >> 5] = part;
    __syncthreads();
    if (t == 0 && g.out.pi_tot) {
      double tot = 0.0;
      for (int w = 0; w < NWARP; ++w) tot += red.v[w];
      g.out.pi_tot[e] = tot;
    }
    __syncthreads();
  }
}

// MINB: CTAs per SM the registers are sized for (3 when three CTAs' shared memory fits).
template <bool MIXED, int MINB>
__global__ void __launch_bounds__(NT, MINB) solve_kernel(SolveArgs g) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Red red;
  __shared__ double s_acc;
  for (int e = blockIdx.x; e < g.ne; e += gridDim.x) solve_energy<MIXED>(g, e, smem_raw, red, s_acc);
}

// All waves of a plan: persistent CTAs claim (wave, chunk energy) units from a
// list sorted by decreasing cost through an atomic counter.  Per-wave
// arguments hold base pointers; the chunk offset e_begin is applied here.
template <bool MIXED, int MINB>
__global__ void __launch_bounds__(NT, MINB) solve_grouped_kernel(const SolveArgs* __restrict__ waves,
                                                              const int2* __restrict__ units, int n_units,
                                                              int64_t e_begin, int ne, int* counter) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ Red red;
  __shared__ double s_acc;
  __shared__ int s_unit;
  while (true) {
    if (threadIdx.x == 0) s_unit = atomicAdd(counter, 1);
    __syncthreads();
    const int u = s_unit;
    __syncthreads();
    if (u >= n_units) break;
    const int2 un = units[u];
    if (un.y >= ne) continue;
    SolveArgs g = waves[un.x];
    g.E += e_begin;
    g.n_open_in += e_begin;
    g.flags_in += e_begin;
    if (g.out.K) g.out.K += e_begin * g.n * g.n;
    if (g.out.eta) g.out.eta += e_begin;
    if (g.out.sig_tot) g.out.sig_tot += e_begin * g.n_sel;
    if (g.out.sig_sel) g.out.sig_sel += e_begin * g.n_sel * g.n;
    if (g.out.flags) g.out.flags += e_begin;
    if (g.out.n_open) g.out.n_open += e_begin;
    if (g.out.pi_tot) g.out.pi_tot += e_begin;
    if (g.out.pi_ch) g.out.pi_ch += e_begin * g.n;
    g.ne = ne;
    solve_energy<MIXED>(g, un.y, smem_raw, red, s_acc);
  }
}

}  // namespace

size_t solve_smem_bytes(int n_max) {
  // panel, tile, tmp, tri, then ipiv, perm, posq, chq (n_max ints each)
  return (size_t)n_max * PANEL_ROW_BYTES + 2 * (size_t)TILE_BYTES + TRI_BYTES + 4 * (size_t)n_max * sizeof(int) + 16;
}

// Resident solve CTAs per SM at this n_max: three when their shared memory fits (registers capped
// at 80 per thread), else two (one CTA's barrier, division and load latencies are filled by the
// others' FMAs).  The mixed-precision kernels need their 128 registers and stay at two.
int solve_blocks_per_sm(int n_max, bool mixed) {
  const int smem = (int)solve_smem_bytes(n_max);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (cudaFuncSetAttribute(solve_grouped_kernel<false, 2>, a, smem) != cudaSuccess ||
      cudaFuncSetAttribute(solve_grouped_kernel<false, 3>, a, smem) != cudaSuccess ||
      cudaFuncSetAttribute(solve_grouped_kernel<true, 2>, a, smem) != cudaSuccess ||
      cudaFuncSetAttribute(solve_kernel<false, 2>, a, smem) != cudaSuccess ||
      cudaFuncSetAttribute(solve_kernel<false, 3>, a, smem) != cudaSuccess ||
      cudaFuncSetAttribute(solve_kernel<true, 2>, a, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int b3 = 0, b2 = 0;
  if (!mixed && cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b3, solve_grouped_kernel<false, 3>, NT, smem) ==
                    cudaSuccess && b3 >= 3)
    return 3;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b2, solve_grouped_kernel<false, 2>, NT, smem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  return b2 < 1 ? 1 : (b2 > 2 ? 2 : b2);
}

// slot layout: real augmented matrix n_max x 2 n_max, complex n_max x (n_max + n_sel), then
// (mixed precision only) FP32 copy of the augmented matrix, M hi / lo, Y hi / lo: 3 n_max^2 doubles
int64_t solve_mix_offset(int n_max, int n_sel) {
  const int64_t ldR = 2 * (int64_t)n_max;
  const int64_t ldC = (int64_t)n_max + n_sel;
  return ((int64_t)n_max * ldR + 2 * (int64_t)n_max * ldC + 31) / 32 * 32;
}

int64_t solve_slot_doubles(int n_max, int n_sel, bool mixed) {
  const int64_t d = solve_mix_offset(n_max, n_sel) + (mixed ? 3 * (int64_t)n_max * n_max : 0);
  return (d + 31) / 32 * 32;
}

cudaError_t launch_solve(const Plan& p, const WaveDev& w, int64_t e0, int ne, const double* R,
                         const double* asym, int ld_chunk, const SolveOut& out, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  SolveArgs g;
  g.n = w.n;
  g.n_sel = p.n_sel;
  g.a = w.a;
  g.R = R;
  g.npR = w.npR();
  g.roff = w.roff();
  g.dip = w.dip ? 1 : 0;
  g.e0 = w.e0;
  g.mixed = p.solve_mixed;
  g.lu_only = p.solve_lu;
  g.z_df = is_split_like(p.prec) ? (p.z_force_fp64 ? 2 : 1) : 0;
  g.mix_off = solve_mix_offset(p.n_max, p.n_sel + 1);
  g.asym = asym;
  g.ld_asym = ld_chunk;
  g.E = w.E + e0;
  g.thr = w.thr;
  g.n_open_in = w.n_open + e0;
  g.flags_in = w.flags0 + e0;
  g.sel = p.sel_dev;
  g.ne = ne;
  g.slot = p.slot;
  g.slot_doubles = p.slot_doubles;
  g.ldR = 2 * p.n_max;
  g.ldC = p.n_max + p.n_sel + 1;  // + the dipole right-hand side
  g.n_slots = p.solve_slots;
  g.out = out;
  const size_t smem = solve_smem_bytes(p.n_max);
  auto kern = p.solve_mixed ? solve_kernel<true, 2> : (p.solve_bps >= 3 ? solve_kernel<false, 3> : solve_kernel<false, 2>);
  cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (err != cudaSuccess) return err;
  const int grid = min(ne, p.solve_slots);
  kern<<<grid, NT, smem, s>>>(g);
  return cudaGetLastError();
}

cudaError_t group_setup_solve(Plan& p) {
  GroupDev& G = p.grp;
  std::vector<SolveArgs> h(p.n_waves);
  for (int g = 0; g < p.n_waves; ++g) {
    const WaveDev& w = p.waves[g];
    SolveArgs a;
    a.n = w.n;
    a.n_sel = p.n_sel;
    a.a = w.a;
    a.R = G.R[g];
    a.npR = w.npR();
    a.roff = w.roff();
    a.dip = w.dip ? 1 : 0;
    a.e0 = w.e0;
    a.mixed = p.solve_mixed;
    a.lu_only = p.solve_lu;
    a.z_df = is_split_like(p.prec) ? (p.z_force_fp64 ? 2 : 1) : 0;
    a.mix_off = solve_mix_offset(p.n_max, p.n_sel + 1);
    a.asym = G.asym[g];
    a.ld_asym = (int64_t)G.chunk * w.n;
    a.E = w.E;
    a.thr = w.thr;
    a.n_open_in = w.n_open;
    a.flags_in = w.flags0;
    a.sel = p.sel_dev;
    a.ne = 0;
    a.slot = p.slot;
    a.slot_doubles = p.slot_doubles;
    a.ldR = 2 * p.n_max;
    a.ldC = p.n_max + p.n_sel + 1;
    a.n_slots = p.solve_slots;
    a.out = SolveOut();
    a.out.eta = w.eta;
    a.out.sig_tot = w.sig_tot;
    a.out.sig_sel = w.sig_sel;
    a.out.flags = w.flags;
    a.out.pi_tot = w.pi_tot;
    a.out.pi_ch = w.pi_ch;
    a.out.do_xsec = true;
    h[g] = a;
  }
  // units of one chunk, waves in decreasing cost (n^3), energies from the top of the chunk down:
  // a wave's thresholds are sorted and the mesh ascends, so the open-channel count and with it
  // the cost of an energy never fall with its index, and the cheapest units come last
  std::vector<int> order(p.n_waves);
  for (int g = 0; g < p.n_waves; ++g) order[g] = g;
  std::sort(order.begin(), order.end(), [&](int x, int y) { return p.waves[x].n > p.waves[y].n; });
  std::vector<int2> units;
  units.reserve((size_t)p.n_waves * G.chunk);
  for (int g : order)
    for (int e = G.chunk - 1; e >= 0; --e) units.push_back(make_int2(g, e));
  cudaError_t err;
  if (!G.solve_waves) {
    if ((err = cudaMalloc(&G.solve_waves, sizeof(SolveArgs) * p.n_waves)) != cudaSuccess) return err;
  }
  if (G.units && G.n_units != (int)units.size()) {
    cudaFree(G.units);
    G.units = nullptr;
  }
  if (!G.units) {
    if ((err = cudaMalloc(&G.units, sizeof(int2) * units.size())) != cudaSuccess) return err;
  }
  if (!G.counter) {
    if ((err = cudaMalloc(&G.counter, sizeof(int))) != cudaSuccess) return err;
  }
  G.n_units = (int)units.size();
  if ((err = cudaMemcpy(G.solve_waves, h.data(), sizeof(SolveArgs) * p.n_waves, cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  if ((err = cudaMemcpy(G.units, units.data(), sizeof(int2) * units.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
    return err;
  const int smem = (int)solve_smem_bytes(p.n_max);
  const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
  cudaError_t e2 = cudaFuncSetAttribute(solve_grouped_kernel<true, 2>, a, smem);
  if (e2 == cudaSuccess) e2 = cudaFuncSetAttribute(solve_grouped_kernel<false, 3>, a, smem);
  if (e2 != cudaSuccess) return e2;
  return cudaFuncSetAttribute(solve_grouped_kernel<false, 2>, a, smem);
}

cudaError_t launch_solve_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s) {
  const GroupDev& G = p.grp;
  cudaError_t err = cudaMemsetAsync(G.counter, 0, sizeof(int), s);
  if (err != cudaSuccess) return err;
  const int grid = std::min(p.solve_slots, p.n_waves * ne);
  auto kern = p.solve_mixed ? solve_grouped_kernel<true, 2>
                            : (p.solve_bps >= 3 ? solve_grouped_kernel<false, 3> : solve_grouped_kernel<false, 2>);
  kern<<<grid, NT, solve_smem_bytes(p.n_max), s>>>(
      reinterpret_cast<const SolveArgs*>(G.solve_waves), G.units, G.n_units, e0, ne, G.counter);
  return cudaGetLastError();
}

RM_CHECK_READER(solve)

}  // namespace rm
