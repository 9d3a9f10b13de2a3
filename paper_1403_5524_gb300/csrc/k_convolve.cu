// Post-processing to compare with experiment: Gaussian convolution of cross
// sections at the experiment's full width at half maximum, averaged over
// several initial levels with statistical weights,
//   out(E_e) = sum_e' G(E_e - E_e') tw_e' m_e' / sum_e' G(E_e - E_e') tw_e',
//   m_e' = sum_s f_s sigma_s(E_e'),  tw = trapezoid weights of the mesh,
// G a Gaussian of standard deviation FWHM / (2 sqrt(2 ln 2)).  Dividing by the
// kernel's own sum keeps a constant a constant at the mesh ends.  The kernel
// is truncated at 8 standard deviations (relative weight e^-32 beyond), and
// each output energy finds its window by binary search in the sorted mesh.
// FP64 throughout; one thread per output energy, reading its window through
// L1 (neighbouring outputs share most of their windows).
#include <cmath>

#include "rm_internal.cuh"

namespace rm {

namespace {

constexpr int CONV_MAX_SERIES = 16;
constexpr double CONV_TRUNC = 8.0;  // standard deviations

struct ConvWeights {
  double f[CONV_MAX_SERIES];
};

__device__ int lower_index(const double* E, int64_t n, double x) {
  int64_t lo = 0, hi = n;
  while (lo < hi) {
    const int64_t mid = (lo + hi) >> 1;
    if (E[mid] < x) lo = mid + 1; else hi = mid;
  }
  return (int)lo;
}

__global__ void convolve_kernel(const double* __restrict__ E, int64_t n_e, const double* __restrict__ sigma,
                                int n_series, ConvWeights fw, double sd, double* __restrict__ out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_e) return;
  auto mixed = [&](int64_t q) {
    double m = 0.0;
    for (int s = 0; s < n_series; ++s) m = fma(fw.f[s], sigma[(int64_t)s * n_e + q], m);
    return m;
  };
  if (sd == 0.0) {
    out[e] = mixed(e);
    return;
  }
  const double x = E[e];
  const int64_t lo = lower_index(E, n_e, x - CONV_TRUNC * sd);
  const int64_t hi = lower_index(E, n_e, x + CONV_TRUNC * sd);  // window [lo, hi) holds e unless 8 sd
                                                                   // vanishes next to x (then: no kernel)
  const double inv = 1.0 / sd;
  double num = 0.0, den = 0.0;
  if (!RM_CHECK(lo >= 0 && hi <= n_e && lo <= hi)) return;
  for (int64_t q = lo; q < hi; ++q) {
    const double el = q > 0 ? E[q - 1] : E[q];
    const double er = q + 1 < n_e ? E[q + 1] : E[q];
    const double tw = n_e > 1 ? 0.5 * (er - el) : 1.0;
    const double u = (x - E[q]) * inv;
    const double g = exp(-0.5 * u * u) * tw;
    num = fma(g, mixed(q), num);
    den += g;
  }
  out[e] = den > 0.0 ? num / den : mixed(e);
}

}  // namespace

cudaError_t launch_convolve(const double* E, int64_t n_e, const double* sigma, int n_series, const double* f,
                            double fwhm, double* out, cudaStream_t s) {
  if (n_e <= 0) return cudaSuccess;
  ConvWeights fw;
  for (int q = 0; q < CONV_MAX_SERIES; ++q) fw.f[q] = q < n_series ? f[q] : 0.0;
  const double sd = fwhm / (2.0 * std::sqrt(2.0 * std::log(2.0)));
  const int bs = 256;
  convolve_kernel<<<(unsigned)((n_e + bs - 1) / bs), bs, 0, s>>>(E, n_e, sigma, n_series, fw, sd, out);
  return cudaGetLastError();
}

int convolve_max_series() { return CONV_MAX_SERIES; }

RM_CHECK_READER(convolve)

}  // namespace rm
