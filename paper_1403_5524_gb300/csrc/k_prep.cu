// Input validation and energy-mesh preparation (nudge, open-channel count).
#include "rm_internal.cuh"

namespace rm {

namespace {

__device__ inline void set_err(int32_t* err, int code) { atomicMax(err, code); }

__global__ void validate_kernel(const int32_t* __restrict__ l, const double* __restrict__ thr,
                                int n, const double* __restrict__ poles, int N,
                                const double* __restrict__ W, int nW, int Npad,
                                const double* __restrict__ E, int64_t n_e, int32_t* err) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < (int64_t)nW * N; t += stride) {
    const int i = (int)(t / N), k = (int)(t % N);
    if (RM_CHECK(k < Npad) && !isfinite(W[(int64_t)i * Npad + k])) set_err(err, RM_ERR_ARG);
  }
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N; t += stride) {
    const double p = poles[t];
    if (!isfinite(p)) set_err(err, RM_ERR_ARG);
    if (t + 1 < N && !(p <= poles[t + 1])) set_err(err, RM_ERR_ORDER);
  }
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n; t += stride) {
    const double e = thr[t];
    if (!isfinite(e)) set_err(err, RM_ERR_ARG);
    if (t + 1 < n && !(e <= thr[t + 1])) set_err(err, RM_ERR_ORDER);
    if (l[t] < 0 || l[t] > RM_LMAX) set_err(err, RM_ERR_ARG);
  }
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n_e; t += stride) {
    const double e = E[t];
    if (!isfinite(e)) set_err(err, RM_ERR_ARG);
    if (t + 1 < n_e && !(e <= E[t + 1])) set_err(err, RM_ERR_ORDER);
  }
}

// first index with v[idx] >= x (v sorted ascending), in [0, m]
__device__ inline int lower_bound(const double* v, int m, double x) {
  int lo = 0, hi = m;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (v[mid] < x) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void prep_kernel(const double* __restrict__ energies, int64_t n_e,
                            const double* __restrict__ poles, int N,
                            const double* __restrict__ thr, int n, double* __restrict__ Eout,
                            uint8_t* __restrict__ flags0, int32_t* __restrict__ n_open) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_e) return;
  if (!RM_CHECK(N >= 1 && n >= 1)) return;
  double E = energies[e];
  double dmin = INFINITY, dthr = INFINITY;
  int k = lower_bound(poles, N, E);
  if (k < N) dmin = fmin(dmin, fabs(poles[k] - E));
  if (k > 0) dmin = fmin(dmin, fabs(poles[k - 1] - E));
  int i = lower_bound(thr, n, E);
  if (i < n) dthr = fmin(dthr, fabs(thr[i] - E));
  if (i > 0) dthr = fmin(dthr, fabs(thr[i - 1] - E));
  dmin = fmin(dmin, dthr);
  uint8_t f = 0;
  if (dthr < 1e-6) f |= RM_FLAG_NEAR_THRESHOLD;  // a channel opens within 1e-6 Ry of the input energy
  if (dmin < 1e-9) {  // one move of 1e-6 Ry up, no re-check
    E += 1e-6;
    f |= RM_FLAG_NUDGED;
  }
  Eout[e] = E;
  flags0[e] = f;
  n_open[e] = lower_bound(thr, n, E);  // #{i : e_i < E}
}

}  // namespace

cudaError_t launch_validate(const WaveDev& w, int N_real, const double* energies, int64_t n_e,
                            int32_t* err_word, cudaStream_t s) {
  validate_kernel<<<152 * 2, 256, 0, s>>>(w.l, w.thr, w.n, w.poles, N_real, w.W, w.nR, w.Npad, energies,
                                         n_e, err_word);
  return cudaGetLastError();
}

cudaError_t launch_prep(const WaveDev& w, const double* energies, int64_t n_e, cudaStream_t s) {
  const int bs = 256;
  const int64_t grid = (n_e + bs - 1) / bs;
  prep_kernel<<<(unsigned)grid, bs, 0, s>>>(energies, n_e, w.poles, w.N, w.thr, w.n, w.E,
                                           w.flags0, w.n_open);
  return cudaGetLastError();
}

RM_CHECK_READER(prep)

}  // namespace rm
