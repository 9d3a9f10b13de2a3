// Far-pole sum in plain FP32 on the CUDA cores (a comparison form of the
// pole sum of Eq. 1-2):
//   R_far(p, e) = (1/2a) sigma_i sigma_j sum_{k far} omega_ik omega_jk D_ke,
// with omega = w / sigma_i (FP32), D_ke = 1 / (E_k - E_e) formed from FP32
// hi + lo parts and rounded to FP32, FP32 products and FP32 accumulation.
// Poles inside the near window [klo, khi) are left to the FP64 window kernel,
// exactly as in the split-precision path.
#include "rm_internal.cuh"

namespace rm {

namespace {

constexpr int CB = 16;   // channels per block
constexpr int ET = 64;   // energies per tile
constexpr int KS = 16;   // poles per step
constexpr int NT = 256;

__global__ void __launch_bounds__(NT) polesum_fp32_kernel(
    const float* __restrict__ omega, int n, int Npad, int N, const float* __restrict__ pol,
    const float* __restrict__ Eh, const float* __restrict__ El, const int32_t* __restrict__ klo,
    const int32_t* __restrict__ khi, const double* __restrict__ sigma, int ne, double inv2a,
    double* __restrict__ R) {
  __shared__ float Wi[CB][KS + 1];
  __shared__ float Wj[CB][KS + 1];
  __shared__ float D[KS][ET];
  __shared__ float P[KS][CB * CB];
  const int nb = (n + CB - 1) / CB;
  int q = blockIdx.x, bi = 0;
  while (q >= nb - bi) { q -= nb - bi; ++bi; }
  const int bj = bi + q;
  const int e0 = blockIdx.y * ET;
  const int t = threadIdx.x;
  const int pg = t >> 3, eg = t & 7;
  float acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[r][s] = 0.0f;
  // energies of this thread's D entries
  float eh[4], el[4];
  int lo[4], hi[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int e = (t + u * NT) % ET;
    const int ge = min(e0 + e, ne - 1);
    eh[u] = Eh[ge];
    el[u] = El[ge];
    lo[u] = klo[ge];
    hi[u] = khi[ge];
    if (e0 + e >= ne) { lo[u] = 0; hi[u] = N; }  // no far poles for padding energies
  }
  for (int k0 = 0; k0 < N; k0 += KS) {
    {
      const int r = t / KS, k = t % KS;
      const int gi = bi * CB + r, gj = bj * CB + r;
      const bool in_k = RM_CHECK(k0 + k < Npad);
      Wi[r][k] = (gi < n && in_k) ? omega[(int64_t)(2 * gi) * Npad + k0 + k] : 0.0f;
      Wj[r][k] = (gj < n && in_k) ? omega[(int64_t)(2 * gj) * Npad + k0 + k] : 0.0f;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = t + u * NT;
      const int k = idx / ET, e = idx % ET;
      const int gk = k0 + k;
      float v = 0.0f;
      if (gk < N && (gk < lo[u] || gk >= hi[u])) v = 1.0f / ((pol[gk] - eh[u]) + (pol[Npad + gk] - el[u]));
      D[k][e] = v;
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < (KS * CB * CB) / NT; ++u) {
      const int idx = t + u * NT;
      const int k = idx / (CB * CB), pr = idx % (CB * CB);
      P[k][pr] = Wi[pr / CB][k] * Wj[pr % CB][k];
    }
    __syncthreads();
#pragma unroll 4
    for (int k = 0; k < KS; ++k) {
      float pv[8], dv[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) pv[r] = P[k][pg + 32 * r];
#pragma unroll
      for (int s = 0; s < 8; ++s) dv[s] = D[k][eg + 8 * s];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int s = 0; s < 8; ++s) acc[r][s] = fmaf(pv[r], dv[s], acc[r][s]);
    }
    __syncthreads();
  }
  const int64_t np = (int64_t)n * (n + 1) / 2;
#pragma unroll
  for (int r = 0; r < 8; ++r) {
    const int pr = pg + 32 * r;
    const int i = bi * CB + pr / CB, j = bj * CB + pr % CB;
    if (i >= n || j >= n || i > j) continue;
    const int64_t p = pair_index(n, i, j);
    const double f = sigma[i] * sigma[j] * inv2a;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int e = e0 + eg + 8 * s;
      if (e < ne && RM_CHECK(p >= 0 && p < np)) R[(int64_t)e * np + p] = (double)acc[r][s] * f;
    }
  }
}

}  // namespace

cudaError_t launch_polesum_fp32(const WaveDev& w, int64_t e0, int ne, double* R, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  const SplitDev& sd = w.split;
  const int nb = (w.nR + CB - 1) / CB;  // all rows of the pole-sum operand (dipole row included)
  dim3 grid(nb * (nb + 1) / 2, (ne + ET - 1) / ET);
  polesum_fp32_kernel<<<grid, NT, 0, s>>>(sd.omega, w.nR, w.Npad, w.N, sd.pol, sd.Eh + e0, sd.El + e0, sd.klo + e0,
                                          sd.khi + e0, sd.sigma, ne, 1.0 / (2.0 * w.a), R);
  return cudaGetLastError();
}

RM_CHECK_READER(polesum_fp32)

}  // namespace rm
