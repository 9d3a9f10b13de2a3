// rm_xsec_from_r_static: the K-matrix / cross-section step for callers that
// cannot allocate device memory.
//
// Some callers must not call cudaMalloc at all: code running inside a
// captured CUDA graph region of someone else's stream, plug-ins that live
// under a host application's own memory pool and are forbidden to grow it,
// and hard-real-time loops where an allocation may block or fail.  This entry
// point takes R-matrices that the caller already holds in device memory and
// computes K, the eigenphase sum and cross sections using only a fixed block
// of device memory that belongs to this library: a file-scope static device
// array (RM_STATIC_SCRATCH_BYTES) that every GPU loading the library keeps
// until the process exits.  The existing kernels run unchanged on pointers
// carved out of that array.
#include <mutex>
#include <string>

#include "rm_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)RM_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
void* g_scratch_ptr[kMaxDevices] = {nullptr};

thread_local std::string g_static_err;

rm_status_t static_fail(rm_status_t s, const std::string& m) {
  g_static_err = m;
  return s;
}

// Device address of the scratch array on the current device; looked up once
// per device (the host-side symbol is only a stand-in, never a device address).
rm_status_t scratch_address(int dev, void** out) {
  if (dev < 0 || dev >= kMaxDevices) return static_fail(RM_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return static_fail(RM_ERR_CUDA, std::string("cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    }
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return RM_OK;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

}  // namespace

extern "C" rm_status_t rm_xsec_from_r_static(const double* R_packed, int32_t n_ch, int32_t n_poles, double a,
                                             const int32_t* l, const double* thresh, const double* pole_E,
                                             const double* energies, int64_t n_e, const int32_t* sel_init,
                                             int32_t n_sel, double* K, double* eigsum, double* sig_tot,
                                             double* sig_sel, uint8_t* flags, int32_t* n_open, void* cuda_stream) {
  using namespace rm;
  if (n_e < 0 || n_ch < 1 || n_poles < 1 || !(a > 0.0)) return static_fail(RM_ERR_ARG, "bad sizes or radius");
  if (n_e == 0) return RM_OK;
  if (!R_packed || !l || !thresh || !pole_E || !energies) return static_fail(RM_ERR_ARG, "null input pointer");
  int32_t sel_default = 0;
  if (!sel_init) {
    sel_init = &sel_default;
    n_sel = 1;
  }
  if (n_sel < 1 || n_sel > RM_MAX_SEL) return static_fail(RM_ERR_ARG, "n_sel out of range");
  for (int q = 0; q < n_sel; ++q)
    if (sel_init[q] < 0) return static_fail(RM_ERR_ARG, "negative selected channel");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return static_fail(RM_ERR_CUDA, "no CUDA device");
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) {
    cudaGetLastError();
    return static_fail(RM_ERR_CUDA, "cannot query device");
  }
  if (prop.major != 10 || prop.minor != 3) return static_fail(RM_ERR_CUDA, "needs an sm_103 (GB300) device");
  if (solve_smem_bytes(n_ch) > (size_t)prop.sharedMemPerBlockOptin)
    return static_fail(RM_ERR_ARG, "n_ch too large for the solve kernel's shared memory");

  // carve the scratch: selected channels, per-chunk energy data, asymptotic
  // data, solve slots.  Chunk and slot counts shrink to fit; sizes that leave
  // no room for one slot are rejected.
  const int n = n_ch;
  const int64_t slot_d = solve_slot_doubles(n, n_sel + 1, false);  // the solve's layout reserves a dipole column
  const size_t slot_b = (size_t)slot_d * sizeof(double);
  const size_t fixed = align256(sizeof(int32_t) * RM_MAX_SEL);
  int chunk = 256;
  auto per_chunk = [&](int c) {
    return align256(sizeof(double) * (size_t)c) + align256((size_t)c) + align256(sizeof(int32_t) * (size_t)c) +
           align256(sizeof(double) * 4 * (size_t)c * (size_t)n);
  };
  while (chunk > 1 && fixed + per_chunk(chunk) + slot_b > kScratchBytes) chunk /= 2;
  if (fixed + per_chunk(chunk) + slot_b > kScratchBytes)
    return static_fail(RM_ERR_ARG, "n_ch too large for the library's static scratch (RM_STATIC_SCRATCH_BYTES)");
  int slots = (int)((kScratchBytes - fixed - per_chunk(chunk)) / slot_b);
  if (slots > prop.multiProcessorCount) slots = prop.multiProcessorCount;

  void* base = nullptr;
  rm_status_t st = scratch_address(dev, &base);
  if (st != RM_OK) return st;
  unsigned char* cur = static_cast<unsigned char*>(base);
  int32_t* sel_dev = reinterpret_cast<int32_t*>(cur);
  cur += fixed;
  double* Ech = reinterpret_cast<double*>(cur);
  cur += align256(sizeof(double) * chunk);
  uint8_t* fl0 = cur;
  cur += align256((size_t)chunk);
  int32_t* nop = reinterpret_cast<int32_t*>(cur);
  cur += align256(sizeof(int32_t) * chunk);
  double* asym = reinterpret_cast<double*>(cur);
  cur += align256(sizeof(double) * 4 * (size_t)chunk * n);
  double* slot = reinterpret_cast<double*>(cur);

  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (cudaMemcpyAsync(sel_dev, sel_init, sizeof(int32_t) * n_sel, cudaMemcpyHostToDevice, s) != cudaSuccess) {
    cudaGetLastError();
    return static_fail(RM_ERR_CUDA, "copy of selected channels failed");
  }

  Plan p;  // host-side description only; every pointer is inside the scratch array
  p.device = dev;
  p.stream = s;
  p.n_sel = n_sel;
  p.sel_dev = sel_dev;
  p.n_max = n;
  p.sm_count = prop.multiProcessorCount;
  p.slot = slot;
  p.solve_slots = slots;
  p.slot_doubles = slot_d;
  WaveDev w;
  w.n = n;
  w.nR = n;  // no dipole row: R is the caller's n x n packed block
  w.N = n_poles;
  w.a = a;
  w.l = const_cast<int32_t*>(l);
  w.thr = const_cast<double*>(thresh);
  w.poles = const_cast<double*>(pole_E);
  w.E = Ech;
  w.flags0 = fl0;
  w.n_open = nop;

  const int64_t np = (int64_t)n * (n + 1) / 2;
  for (int64_t c0 = 0; c0 < n_e; c0 += chunk) {
    const int ne = (int)((n_e - c0) < chunk ? (n_e - c0) : chunk);
    cudaError_t e = launch_prep(w, energies + c0, ne, s);
    if (e == cudaSuccess) e = launch_asym(w, 0, ne, asym, chunk * n, s);
    SolveOut so;
    so.do_xsec = (eigsum || sig_tot || sig_sel);
    so.K = K ? K + c0 * n * n : nullptr;
    so.eta = eigsum ? eigsum + c0 : nullptr;
    so.sig_tot = sig_tot ? sig_tot + c0 * n_sel : nullptr;
    so.sig_sel = sig_sel ? sig_sel + c0 * n_sel * n : nullptr;
    so.flags = flags ? flags + c0 : nullptr;
    so.n_open = n_open ? n_open + c0 : nullptr;
    if (e == cudaSuccess) e = launch_solve(p, w, 0, ne, R_packed + c0 * np, asym, chunk * n, so, s);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return static_fail(RM_ERR_CUDA, std::string("kernel launch failed: ") + cudaGetErrorString(e));
    }
  }
  return RM_OK;
}

extern "C" const char* rm_static_last_error(void) { return g_static_err.c_str(); }
