// Plain FP64 pole sum (the baseline form of Eq. 1-2):
//   R[e][p(i,j)] = (1/2a) sum_k w_ik w_jk / (E_k - E_e),  i <= j.
// Written as the product P(pair, k) D(k, e) with P_pk = w_ik w_jk formed per
// tile in shared memory from W rows, and D_ke = 1/(E_k - E_e) generated per
// tile; neither operand is stored in global memory.  GB300 retires about two
// FP64 FMAs per clock per SM, so this kernel is FP64-pipe bound by design.
#include "rm_internal.cuh"

namespace rm {

namespace {

constexpr int CB = 16;   // channels per block (pair tile = CB x CB)
constexpr int ET = 64;   // energies per tile
constexpr int KS = 16;   // poles per step
constexpr int NT = 256;  // threads

__global__ void __launch_bounds__(NT) polesum_fp64_kernel(
    const double* __restrict__ W, int n, int Npad, int N, const double* __restrict__ poles,
    const double* __restrict__ E, int ne, double inv2a, double* __restrict__ R) {
  __shared__ double Wi[CB][KS + 1];
  __shared__ double Wj[CB][KS + 1];
  __shared__ double D[KS][ET];
  __shared__ double P[KS][CB * CB];

  // block pair (bi <= bj) from the linear upper-triangle index
  const int nb = (n + CB - 1) / CB;
  int q = blockIdx.x, bi = 0;
  while (q >= nb - bi) { q -= nb - bi; ++bi; }
  const int bj = bi + q;
  const int e0 = blockIdx.y * ET;
  const int t = threadIdx.x;
  const int pg = t >> 3, eg = t & 7;

  double acc[8][8];
#pragma unroll
  for (int r = 0; r < 8; ++r)
#pragma unroll
    for (int s = 0; s < 8; ++s) acc[r][s] = 0.0;

  // energies of this thread's D loads
  double Eld[4];
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int idx = t + u * NT;      // 0..1023 -> (k, e)
    const int e = idx % ET;
    Eld[u] = E[min(e0 + e, ne - 1)];
  }

  for (int k0 = 0; k0 < N; k0 += KS) {
    {
      const int r = t / KS, k = t % KS;  // 256 threads -> 16 x 16
      const int gi = bi * CB + r, gj = bj * CB + r;
      const bool in_k = RM_CHECK(k0 + k < Npad);
      Wi[r][k] = (gi < n && in_k) ? W[(int64_t)gi * Npad + k0 + k] : 0.0;
      Wj[r][k] = (gj < n && in_k) ? W[(int64_t)gj * Npad + k0 + k] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int idx = t + u * NT;
      const int k = idx / ET, e = idx % ET;
      const int gk = k0 + k;
      D[k][e] = (gk < N) ? 1.0 / (poles[gk] - Eld[u]) : 0.0;
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
      double pv[8], dv[8];
#pragma unroll
      for (int r = 0; r < 8; ++r) pv[r] = P[k][pg + 32 * r];
#pragma unroll
      for (int s = 0; s < 8; ++s) dv[s] = D[k][eg + 8 * s];
#pragma unroll
      for (int r = 0; r < 8; ++r)
#pragma unroll
        for (int s = 0; s < 8; ++s) acc[r][s] = fma(pv[r], dv[s], acc[r][s]);
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
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      const int e = e0 + eg + 8 * s;
      if (e < ne && RM_CHECK(p >= 0 && p < np)) R[(int64_t)e * np + p] = acc[r][s] * inv2a;
    }
  }
}

}  // namespace

cudaError_t launch_polesum_fp64(const WaveDev& w, int64_t e0, int ne, double* R, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  const int nb = (w.nR + CB - 1) / CB;  // all rows of the pole-sum operand (dipole row included)
  dim3 grid(nb * (nb + 1) / 2, (ne + ET - 1) / ET);
  polesum_fp64_kernel<<<grid, NT, 0, s>>>(w.W, w.nR, w.Npad, w.N, w.poles, w.E + e0, ne,
                                          1.0 / (2.0 * w.a), R);
  return cudaGetLastError();
}

RM_CHECK_READER(polesum_fp64)

}  // namespace rm
