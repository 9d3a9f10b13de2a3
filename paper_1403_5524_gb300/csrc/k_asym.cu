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
//
// Ionic targets (residual charge z > 0, potential -2z/r): open channels use
// the Coulomb functions F_l(eta, rho), G_l(eta, rho), eta = -z/k, rho = k a,
// with s = k^-1/2 F, c = k^-1/2 G (z = 0 gives jhat_l and -nhat_l back);
// closed channels the decaying Whittaker function W_{z/kappa, l+1/2}(2 kappa r).
// Coulomb functions by Barnett's arrangement of Steed's method (Barnett,
// Feng, Steed & Goldfarb 1974): the continued fraction CF1 for F_l'/F_l at the
// channel's l, whose partial denominators also give the sign of F_l; the
// recurrence down to order 0 for the unnormalised F; at order 0 (outside the
// turning point for every attractive field) the complex continued fraction
// CF2 for p + iq = (G' + iF')/(G + iF) and the Wronskian F'G - FG' = 1 fix
// F_0 and G_0; G runs up again to order l.  CF2 is written here through the
// Kummer function: G + iF = const e^(i rho) rho^(l+1) U(l+1+i eta, 2l+2, -2i rho),
// so p + iq = -i + i eta/rho - r/rho with r = U(a-1,b,x)/U(a,b,x), and r is the
// continued fraction of the recurrence
//   U(a-1) + (b - 2a - x) U(a) + a(a - b + 1) U(a+1) = 0
// in a (U is its minimal solution as a -> infinity).  The same fraction at real
// x = 2 kappa a, a = l + 1 - z/kappa, b = 2l + 2 gives the Whittaker
// log-derivative W'/W = 1/2 - (z/kappa + r)/x, because
// W_{k,m}(x) = e^(-x/2) x^(m+1/2) U(m - k + 1/2, 2m + 1, x).
// Every fraction runs under an iteration cap; a channel whose fraction does
// not converge sets RM_FLAG_ASYM on its energy.
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

constexpr int CF_MAXIT = 200000;      // iteration cap of every continued fraction
constexpr double CF_EPS = 4.5e-16;     // |delta - 1| at convergence (two ulps)
constexpr double CF_TINY = 1e-300;

// CF1: f = F_l'/F_l = S_{l+1} - R^2_{l+1} / (S_{l+1} + S_{l+2} - R^2_{l+2} / (...)),
// S_m = m/rho + eta/m, R^2_m = 1 + eta^2/m^2 (modified Lentz).  The sign of F_l
// is the parity of negative partial denominators (F_L > 0 for L -> infinity).
__device__ bool coulomb_cf1(int l, double eta, double rho, double& f, double& sign) {
  auto S = [&](int m) { return m / rho + eta / m; };
  f = S(l + 1);
  if (f == 0.0) f = CF_TINY;
  double C = f, D = 0.0;
  sign = 1.0;
  for (int k = 1; k < CF_MAXIT; ++k) {
    const int m = l + k;
    const double am = -(1.0 + (eta / m) * (eta / m));
    const double bm = S(m) + S(m + 1);
    D = bm + am * D;
    if (D == 0.0) D = CF_TINY;
    C = bm + am / C;
    if (C == 0.0) C = CF_TINY;
    D = 1.0 / D;
    const double delta = C * D;
    f *= delta;
    if (D < 0.0) sign = -sign;
    if (fabs(delta - 1.0) < CF_EPS) return true;
  }
  return false;
}

// complex quotient a / b (Smith's method)
__device__ cplx cdiv(cplx a, cplx b) {
  if (fabs(b.re) >= fabs(b.im)) {
    const double t = b.im / b.re, d = b.re + b.im * t;
    return cplx{(a.re + a.im * t) / d, (a.im - a.re * t) / d};
  }
  const double t = b.re / b.im, d = b.im + b.re * t;
  return cplx{(a.re * t + a.im) / d, (a.im * t - a.re) / d};
}

// r = U(a-1,b,x)/U(a,b,x) for complex a, x (b real) by the continued fraction of
// the recurrence in a: r = (2a + x - b) - a(a-b+1) / ((2a + 2 + x - b) - ...).
__device__ bool kummer_ratio(cplx a, double b, cplx x, cplx& r) {
  r = cplx{2.0 * a.re + x.re - b, 2.0 * a.im + x.im};
  if (r.re == 0.0 && r.im == 0.0) r = cplx{CF_TINY, 0.0};
  cplx C = r, D = cplx{0.0, 0.0};
  for (int k = 1; k < CF_MAXIT; ++k) {
    const cplx p = cplx{a.re + (k - 1), a.im} * cplx{a.re + (k - b), a.im};
    const cplx ak = cplx{-p.re, -p.im};
    const cplx bk = cplx{2.0 * (a.re + k) + x.re - b, 2.0 * a.im + x.im};
    D = bk + ak * D;
    if (D.re == 0.0 && D.im == 0.0) D = cplx{CF_TINY, 0.0};
    C = bk + cdiv(ak, C);
    if (C.re == 0.0 && C.im == 0.0) C = cplx{CF_TINY, 0.0};
    D = cdiv(cplx{1.0, 0.0}, D);
    const cplx delta = C * D;
    r = r * delta;
    if (fabs(delta.re - 1.0) + fabs(delta.im) < CF_EPS) return true;
  }
  return false;
}

// F_l, F_l', G_l, G_l' (derivatives in rho) for eta <= 0; false if a fraction
// did not converge.
__device__ bool coulomb_open(int l, double eta, double rho, double& F, double& Fp, double& G, double& Gp) {
  double f, sign;
  bool ok = coulomb_cf1(l, eta, rho, f, sign);
  // unnormalised F down to order 0: u_{m-1} = (S_m u_m + u_m')/R_m, u_{m-1}' = S_m u_{m-1} - R_m u_m
  double Fu = sign, Fpu = sign * f, scale = 1.0;
  for (int m = l; m >= 1; --m) {
    const double S = m / rho + eta / m;
    const double R = sqrt(1.0 + (eta / m) * (eta / m));
    const double Fm = (S * Fu + Fpu) / R;
    Fpu = S * Fm - R * Fu;
    Fu = Fm;
    if (fabs(Fu) > 1e250) {
      Fu *= 1e-250;
      Fpu *= 1e-250;
      scale *= 1e-250;  // F_l = (F_0 / Fu) * sign * scale
    }
  }
  const double f0 = Fpu / Fu;
  // CF2 at order 0: p + iq = -i + i eta/rho - r/rho, r from U(1 + i eta, 2, -2i rho)
  cplx r;
  ok = kummer_ratio(cplx{1.0, eta}, 2.0, cplx{0.0, -2.0 * rho}, r) && ok;
  const double p = r.re * (-1.0 / rho);
  const double q = -1.0 + eta / rho - r.im / rho;
  const double F0 = copysign(sqrt(q / ((f0 - p) * (f0 - p) + q * q)), Fu);
  double Gm = (f0 - p) * F0 / q;
  double Gpm = p * Gm - q * F0;
  F = (F0 / Fu) * sign * scale;
  Fp = F * f;
  // G upward: u_{m+1} = (S_{m+1} u_m - u_m')/R_{m+1}, u_{m+1}' = R_{m+1} u_m - S_{m+1} u_{m+1}
  for (int m = 0; m < l; ++m) {
    const double S = (m + 1) / rho + eta / (m + 1);
    const double R = sqrt(1.0 + (eta / (m + 1)) * (eta / (m + 1)));
    const double G1 = (S * Gm - Gpm) / R;
    Gpm = R * Gm - S * G1;
    Gm = G1;
  }
  G = Gm;
  Gp = Gpm;
  return ok && isfinite(F) && isfinite(G) && q > 0.0;
}

// W'/W of W_{kp, l+1/2}(x), x > 0, by the real Kummer-ratio fraction
__device__ bool whittaker_logderiv(int l, double kp, double x, double& d) {
  cplx r;
  const bool ok = kummer_ratio(cplx{l + 1.0 - kp, 0.0}, 2.0 * l + 2.0, cplx{x, 0.0}, r);
  d = 0.5 - (kp + r.re) / x;
  return ok && isfinite(d);
}

// Matching data of one (energy, channel): Lambda, s, s', c (s = s' = c = 0 closed).
__device__ bool channel_data(int l, double k2, double a, double z, double& lam, double& s, double& sp,
                             double& c) {
  s = sp = c = 0.0;
  if (k2 > 0.0) {
    const double k = sqrt(k2), sk = sqrt(k);
    if (z == 0.0) {
      double j, jp, y, yp;
      riccati_open(l, k * a, j, jp, y, yp);
      s = j / sk;
      sp = jp * sk;
      c = -y / sk;
      lam = k * yp / y;  // c'/c
      return true;
    }
    double F, Fp, G, Gp;
    const bool ok = coulomb_open(l, -z / k, k * a, F, Fp, G, Gp);
    s = F / sk;
    sp = Fp * sk;
    c = G / sk;
    lam = k * Gp / G;
    return ok;
  }
  const double kap = sqrt(-k2);
  if (z == 0.0) {
    lam = kap * khat_logderiv(l, kap * a);
    return true;
  }
  double d;
  const bool ok = whittaker_logderiv(l, z / kap, 2.0 * kap * a, d);
  lam = 2.0 * kap * d;
  return ok;
}

// flag the energy's byte in a uint8 flag array (atomically: several channels may fail)
__device__ void flag_energy(uint8_t* flags, int64_t e, uint8_t bit) {
  const uintptr_t addr = reinterpret_cast<uintptr_t>(flags + e);
  unsigned int* word = reinterpret_cast<unsigned int*>(addr & ~uintptr_t(3));
  atomicOr(word, (unsigned int)bit << (8 * (addr & 3)));
}

__global__ void asym_kernel(const int32_t* __restrict__ lch, const double* __restrict__ thr, int n,
                            double a, double z, const double* __restrict__ E, int ne,
                            double* __restrict__ out, int64_t ld, uint8_t* flags) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)ne * n) return;
  const int e = (int)(t / n), i = (int)(t % n);
  double lam, s, sp, c;
  if (!channel_data(lch[i], E[e] - thr[i], a, z, lam, s, sp, c)) flag_energy(flags, e, RM_FLAG_ASYM);
  if (!RM_CHECK(t < ld)) return;  // the four blocks of the chunk buffer are ld apart
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
  uint8_t* flags;   // per-energy input flags of the solve (base)
  double a;
  double z;
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
  double lam, s, sp, c;
  if (!channel_data(w.l[i], w.E[e_begin + e] - w.thr[i], w.a, w.z, lam, s, sp, c))
    flag_energy(w.flags, e_begin + e, RM_FLAG_ASYM);
  if (!RM_CHECK(t < ld)) return;
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
    h[g] = AsymWave{w.l, w.thr, w.E, G.asym[g], w.flags0, w.a, w.z, w.n};
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
  asym_kernel<<<(unsigned)((total + bs - 1) / bs), bs, 0, s>>>(w.l, w.thr, w.n, w.a, w.z, w.E + e0, ne,
                                                              asym, (int64_t)ld_chunk, w.flags0 + e0);
  return cudaGetLastError();
}

RM_CHECK_READER(asym)

}  // namespace rm
