// Zero-potential asymptotic functions at r = a, one thread per (energy, channel).
//
// Open channel (E > e_i): k = sqrt(E - e_i), x = k a,
//   s = k^-1/2 jhat_l(x), s' = k^1/2 jhat_l'(x), c = -k^-1/2 nhat_l(x),
//   c' = -k^1/2 nhat_l'(x), Lambda = c'/c,
// with Riccati-Bessel jhat_l = x j_l, nhat_l = x y_l (~ -cos(x - l pi/2)).
// Closed channel: kappa = sqrt(e_i - E), x = kappa a, Lambda = kappa khat_l'/khat_l
// for the decaying Riccati function khat_l.  (The paper gives no formula for
// this step; these are the standard zero-potential solutions.)
//
// Recurrences: f_{l+1} = ((2l+1)/x) f_l - f_{l-1} holds for jhat and nhat;
// nhat is run upward (stable); jhat upward when x > l, else by Miller's
// downward recurrence normalised to sin x (or to jhat_1 near zeros of sin x).
// khat is run upward on the scaled sequence exp(x) khat_l:
// g_{l+1} = g_{l-1} + ((2l+1)/x) g_l, g_{-1} = g_0 = 1; the exponential
// cancels in the log-derivative, khat_l'/khat_l = (-g_{l-1} - (l/x) g_l)/g_l.
#include <vector>

#include "rm_internal.cuh"

namespace rm {

namespace {

__device__ void riccati_open(int l, double x, double& j, double& jp, double& y, double& yp) {
  double sx, cx;
  sincos(x, &sx, &cx);
  // nhat: upward
  if (l == 0) {
    y = -cx;
    yp = sx;
  } else {
    double n0 = -cx, n1 = -cx / x - sx;
    for (int m = 1; m < l; ++m) {
      const double n2 = ((2 * m + 1) / x) * n1 - n0;
      n0 = n1;
      n1 = n2;
    }
    y = n1;
    yp = n0 - (l / x) * n1;
  }
  // jhat
  if (l == 0) {
    j = sx;
    jp = cx;
    return;
  }
  if (x > (double)l) {
    double j0 = sx, j1 = sx / x - cx;
    for (int m = 1; m < l; ++m) {
      const double j2 = ((2 * m + 1) / x) * j1 - j0;
      j0 = j1;
      j1 = j2;
    }
    j = j1;
    jp = j0 - (l / x) * j1;
    return;
  }
  // Miller: f_{L+1} = 0, f_L = tiny, recur down to f_0
  const int L = l + 24 + (int)x;
  double fp1 = 0.0, f = 1e-280;
  double fl = 0.0, flm1 = 0.0;
  for (int m = L; m >= 1; --m) {
    const double fm1 = ((2 * m + 1) / x) * f - fp1;
    fp1 = f;
    f = fm1;  // now f = f_{m-1}, fp1 = f_m
    if (m == l) fl = fp1;
    if (m - 1 == l - 1) flm1 = f;
    if (fabs(f) > 1e250) {
      f *= 1e-250;
      fp1 *= 1e-250;
      fl *= 1e-250;
      flm1 *= 1e-250;
    }
  }
  // f = f_0, fp1 = f_1
  double scale;
  if (fabs(sx) > 0.1) scale = sx / f;
  else scale = (sx / x - cx) / fp1;
  j = fl * scale;
  jp = flm1 * scale - (l / x) * j;
}

__device__ double khat_logderiv(int l, double x) {
  double gm1 = 1.0, g = 1.0;  // g_{-1}, g_0
  for (int m = 0; m < l; ++m) {
    const double gp1 = gm1 + ((2 * m + 1) / x) * g;
    gm1 = g;
    g = gp1;
  }
  return (-gm1 - (l / x) * g) / g;
}

__global__ void asym_kernel(const int32_t* __restrict__ lch, const double* __restrict__ thr, int n,
                            double a, const double* __restrict__ E, int ne,
                            double* __restrict__ out, int64_t ld) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ne * n) return;
  const int e = (int)(t / n), i = (int)(t % n);
  const double k2 = E[e] - thr[i];
  const int l = lch[i];
  double lam, s = 0.0, sp = 0.0, c = 0.0;
  if (k2 > 0.0) {
    const double k = sqrt(k2), sk = sqrt(k);
    double j, jp, y, yp;
    riccati_open(l, k * a, j, jp, y, yp);
    s = j / sk;
    sp = jp * sk;
    c = -y / sk;
    lam = k * yp / y;  // c'/c
  } else {
    const double kap = sqrt(-k2);
    lam = kap * khat_logderiv(l, kap * a);
  }
  out[0 * ld + t] = lam;
  out[1 * ld + t] = s;
  out[2 * ld + t] = sp;
  out[3 * ld + t] = c;
}

struct AsymWave {
  const int32_t* l;
  const double* thr;
  const double* E;  // nudged mesh (base)
  double* out;      // chunk buffer [4][chunk * n]
  double a;
  int n;
};

// grid.y = wave; energies e_begin .. e_begin + ne of every wave
__global__ void asym_grouped_kernel(const AsymWave* __restrict__ waves, int64_t e_begin, int ne, int64_t ld_chunk) {
  const AsymWave w = waves[blockIdx.y];
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ne * w.n) return;
  // ld between the four quantities is chunk * n of this wave
  const int64_t ld = ld_chunk * w.n;
  const int e = (int)(t / w.n), i = (int)(t % w.n);
  const double k2 = w.E[e_begin + e] - w.thr[i];
  const int l = w.l[i];
  double lam, s = 0.0, sp = 0.0, c = 0.0;
  if (k2 > 0.0) {
    const double k = sqrt(k2), sk = sqrt(k);
    double j, jp, y, yp;
    riccati_open(l, k * w.a, j, jp, y, yp);
    s = j / sk;
    sp = jp * sk;
    c = -y / sk;
    lam = k * yp / y;
  } else {
    const double kap = sqrt(-k2);
    lam = kap * khat_logderiv(l, kap * w.a);
  }
  w.out[0 * ld + t] = lam;
  w.out[1 * ld + t] = s;
  w.out[2 * ld + t] = sp;
  w.out[3 * ld + t] = c;
}

}  // namespace

cudaError_t group_setup_asym(Plan& p) {
  GroupDev& G = p.grp;
  std::vector<AsymWave> h(p.n_waves);
  for (int g = 0; g < p.n_waves; ++g) {
    const WaveDev& w = p.waves[g];
    h[g] = AsymWave{w.l, w.thr, w.E, G.asym[g], w.a, w.n};
  }
  cudaError_t err;
  if (!G.asym_waves && (err = cudaMalloc(&G.asym_waves, sizeof(AsymWave) * p.n_waves)) != cudaSuccess) return err;
  return cudaMemcpy(G.asym_waves, h.data(), sizeof(AsymWave) * p.n_waves, cudaMemcpyHostToDevice);
}

cudaError_t launch_asym_grouped(const Plan& p, int64_t e0, int ne, cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  const int bs = 256;
  dim3 grid((unsigned)(((int64_t)ne * p.n_max + bs - 1) / bs), p.n_waves);
  asym_grouped_kernel<<<grid, bs, 0, s>>>(reinterpret_cast<const AsymWave*>(p.grp.asym_waves), e0, ne,
                                          (int64_t)p.grp.chunk);
  return cudaGetLastError();
}

cudaError_t launch_asym(const WaveDev& w, int64_t e0, int ne, double* asym, int ld_chunk,
                        cudaStream_t s) {
  if (ne <= 0) return cudaSuccess;
  const int64_t total = (int64_t)ne * w.n;
  const int bs = 256;
  asym_kernel<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(w.l, w.thr, w.n, w.a, w.E + e0, ne,
                                                              asym, (int64_t)ld_chunk);
  return cudaGetLastError();
}

}  // namespace rm
