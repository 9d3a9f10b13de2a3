// rm_xsec_from_r_static: the K-matrix / cross-section step for callers that
// cannot allocate device memory.
//
// Some callers must not call cudaMalloc at all: plug-ins that live under a
// host application's own memory pool and are forbidden to grow it, hard
// real-time loops where an allocation may block or fail, and code that runs
// where the device allocator is off limits to it.  This entry point takes
// R-matrices that the caller already holds in device memory and computes K,
// the eigenphase sum and cross sections using only a fixed block of device
// memory that belongs to this library: a file-scope static device array
// (RM_STATIC_SCRATCH_BYTES) that every GPU loading the library keeps until the
// process exits.  The existing kernels run unchanged on pointers carved out of
// that array; two small kernels of this file fill in what a plan would have
// copied from the host (the selected channels, passed by value as a kernel
// argument, and the channels' l clamped to [0, RM_LMAX]).
#include <cstring>
#include <mutex>

#include "rm_internal.cuh"

namespace {

constexpr size_t kScratchBytes = (size_t)RM_STATIC_SCRATCH_BYTES;
static __device__ __align__(256) unsigned char g_static_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
constexpr int kMaxChannels = 640;  // as rm_wave.n_ch: the largest channel count the solve is built and tested for
struct DeviceSetup {
  void* scratch = nullptr;  // device address of g_static_scratch on this device
  int sm_count = 0;
  int smem_optin = 0;
  bool sm103 = false;
};
std::mutex g_setup_mutex;
DeviceSetup g_setup[kMaxDevices];

// The last failure's message: a fixed process-wide buffer (a std::string, or thread-local
// storage in a loaded library, could allocate); concurrent failures may overwrite each other.
std::mutex g_err_mutex;
char g_static_err[256] = "";

rm_status_t static_fail(rm_status_t s, const char* m, const char* detail = nullptr) {
  std::lock_guard<std::mutex> lock(g_err_mutex);
  size_t k = 0;
  for (const char* p : {m, detail}) {
    if (!p) continue;
    const size_t len = std::strlen(p);
    const size_t room = sizeof(g_static_err) - 1 - k;
    const size_t c = len < room ? len : room;
    std::memcpy(g_static_err + k, p, c);
    k += c;
  }
  g_static_err[k] = 0;
  return s;
}

// Per-device set-up, once, with that device current: the scratch array's device
// address (the host-side symbol is only a stand-in, never a device address) and
// the attributes the launch sizes depend on.
rm_status_t device_setup(int dev, DeviceSetup* out) {
  if (dev < 0 || dev >= kMaxDevices) return static_fail(RM_ERR_CUDA, "device index out of range");
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  DeviceSetup& d = g_setup[dev];
  if (!d.scratch) {
    int major = 0, minor = 0, sms = 0, smem = 0;
    if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return static_fail(RM_ERR_CUDA, "cannot query device");
    }
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return static_fail(RM_ERR_CUDA, "cudaGetSymbolAddress failed: ", cudaGetErrorString(e));
    }
    d.sm103 = (major == 10 && minor == 3);
    d.sm_count = sms;
    d.smem_optin = smem;
    d.scratch = p;
  }
  *out = d;
  return RM_OK;
}

size_t align256(size_t b) { return (b + 255) / 256 * 256; }

// Carving of the scratch for n channels and n_sel selected channels: the selected channels,
// the clamped l and its flag word, per-chunk energy data and asymptotic data, then the solve
// slots (one per resident solve CTA, at most one per SM).  The per-chunk asymptotic data
// (32 n bytes per energy) competes with the slots (about 32 n^2 bytes each): the chunk starts
// at 256 energies and halves until the slots reach 90 % of the most that any chunk allows
// (capped at one per SM), so small chunks, each a round of launches, are taken only where they
// buy solve CTAs; false when not even one slot fits.
struct Layout {
  size_t fixed = 0;
  size_t slot_b = 0;
  int64_t slot_d = 0;
  int chunk = 0;
  int slots = 0;
};
size_t per_chunk_bytes(int c, int n) {
  return align256(sizeof(double) * (size_t)c) + align256((size_t)c) + align256(sizeof(int32_t) * (size_t)c) +
         align256(sizeof(double) * 4 * (size_t)c * (size_t)n);
}
bool make_layout(int n, int n_sel, int sm_count, Layout& L) {
  L.slot_d = rm::solve_slot_doubles(n, n_sel + 1, false);  // the solve's layout reserves a dipole column
  L.slot_b = (size_t)L.slot_d * sizeof(double);
  L.fixed = align256(sizeof(int32_t) * RM_MAX_SEL) + align256(sizeof(int32_t) * (size_t)n) + 256;
  auto slots_for = [&](int c) -> int64_t {
    const size_t used = L.fixed + per_chunk_bytes(c, n);
    return used >= kScratchBytes ? 0 : (int64_t)((kScratchBytes - used) / L.slot_b);
  };
  const int64_t best = slots_for(1) < sm_count ? slots_for(1) : sm_count;
  if (best < 1) return false;
  int chunk = 256;
  auto capped = [&](int c) { return slots_for(c) < sm_count ? slots_for(c) : (int64_t)sm_count; };
  while (chunk > 1 && (capped(chunk) < 1 || 10 * capped(chunk) < 9 * best)) chunk /= 2;
  const int64_t fit = slots_for(chunk);
  if (fit < 1) return false;
  L.chunk = chunk;
  L.slots = (int)(fit < sm_count ? fit : sm_count);
  return true;
}

struct SelArg {
  int32_t v[RM_MAX_SEL];
};

// The selected channels (a kernel argument, so nothing reads host memory after
// the call returns) and the channels' l, clamped to [0, RM_LMAX] so that the
// asymptotic functions' recurrences stay bounded; *bad records a clamped l.
__global__ void static_setup_kernel(SelArg sel, int n_sel, int32_t* __restrict__ sel_dev,
                                    const int32_t* __restrict__ l_in, int n, int32_t* __restrict__ l_dev,
                                    int32_t* __restrict__ bad) {
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  __syncthreads();
  for (int q = threadIdx.x; q < n_sel; q += blockDim.x) sel_dev[q] = sel.v[q];
  int b = 0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const int l = l_in[i];
    const bool ok = l >= 0 && l <= RM_LMAX;
    l_dev[i] = ok ? l : (l < 0 ? 0 : RM_LMAX);
    if (!ok) b = 1;
  }
  if (b) atomicOr(&s_bad, 1);
  __syncthreads();
  if (threadIdx.x == 0) *bad = s_bad;
}

// after the nudge of a chunk: a clamped l makes every energy's outputs unreliable
__global__ void static_flag_kernel(uint8_t* __restrict__ fl0, int ne, const int32_t* __restrict__ bad) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < ne && *bad) fl0[e] |= RM_FLAG_ASYM;
}

// the scratch carving must end inside the array (checked build)
__global__ void static_extent_kernel(const unsigned char* end) {
  RM_CHECK(end <= g_static_scratch + kScratchBytes);
}

}  // namespace

namespace rm {
RM_CHECK_READER(static)
}  // namespace rm

extern "C" rm_status_t rm_xsec_from_r_static(const double* R_packed, int32_t n_ch, int32_t n_poles, double a,
                                             const int32_t* l, const double* thresh, const double* pole_E,
                                             const double* energies, int64_t n_e, const int32_t* sel_init,
                                             int32_t n_sel, double* K, double* eigsum, double* sig_tot,
                                             double* sig_sel, uint8_t* flags, int32_t* n_open, void* cuda_stream) {
  using namespace rm;
  if (n_e < 0 || n_ch < 1 || n_poles < 1 || !(a > 0.0)) return static_fail(RM_ERR_ARG, "bad sizes or radius");
  if (n_ch > kMaxChannels) return static_fail(RM_ERR_ARG, "n_ch above 640, the largest channel count of the solve");
  if (n_e == 0) return RM_OK;
  if (!R_packed || !l || !thresh || !pole_E || !energies) return static_fail(RM_ERR_ARG, "null input pointer");
  SelArg sel;
  if (!sel_init) {
    sel.v[0] = 0;
    n_sel = 1;
  } else {
    if (n_sel < 1 || n_sel > RM_MAX_SEL) return static_fail(RM_ERR_ARG, "n_sel out of range");
    for (int q = 0; q < n_sel; ++q) {
      if (sel_init[q] < 0) return static_fail(RM_ERR_ARG, "negative selected channel");
      sel.v[q] = sel_init[q];
    }
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return static_fail(RM_ERR_CUDA, "no CUDA device");
  }
  DeviceSetup ds;
  rm_status_t st = device_setup(dev, &ds);
  if (st != RM_OK) return st;
  if (!ds.sm103) return static_fail(RM_ERR_CUDA, "needs an sm_103 (GB300) device");
  if (solve_smem_bytes(n_ch) > (size_t)ds.smem_optin)
    return static_fail(RM_ERR_ARG, "n_ch too large for the solve kernel's shared memory");

  const int n = n_ch;
  Layout L;
  if (!make_layout(n, n_sel, ds.sm_count, L))
    return static_fail(RM_ERR_ARG, "n_ch too large for the library's static scratch (RM_STATIC_SCRATCH_BYTES)");
  const int chunk = L.chunk;

  unsigned char* cur = static_cast<unsigned char*>(ds.scratch);
  int32_t* sel_dev = reinterpret_cast<int32_t*>(cur);
  cur += align256(sizeof(int32_t) * RM_MAX_SEL);
  int32_t* l_dev = reinterpret_cast<int32_t*>(cur);
  cur += align256(sizeof(int32_t) * (size_t)n);
  int32_t* bad = reinterpret_cast<int32_t*>(cur);
  cur += 256;
  double* Ech = reinterpret_cast<double*>(cur);
  cur += align256(sizeof(double) * chunk);
  uint8_t* fl0 = cur;
  cur += align256((size_t)chunk);
  int32_t* nop = reinterpret_cast<int32_t*>(cur);
  cur += align256(sizeof(int32_t) * chunk);
  double* asym = reinterpret_cast<double*>(cur);
  cur += align256(sizeof(double) * 4 * (size_t)chunk * n);
  double* slot = reinterpret_cast<double*>(cur);
#ifdef RM_CHECKED
  static_extent_kernel<<<1, 1, 0, reinterpret_cast<cudaStream_t>(cuda_stream)>>>(
      reinterpret_cast<unsigned char*>(slot + (int64_t)L.slots * L.slot_d));
#endif

  cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
  static_setup_kernel<<<1, 256, 0, s>>>(sel, n_sel, sel_dev, l, n, l_dev, bad);
  cudaError_t e0 = cudaGetLastError();
  if (e0 != cudaSuccess) return static_fail(RM_ERR_CUDA, "kernel launch failed: ", cudaGetErrorString(e0));

  Plan p;  // host-side description only; every pointer is inside the scratch array
  p.device = dev;
  p.stream = s;
  p.n_sel = n_sel;
  p.sel_dev = sel_dev;
  p.n_max = n;
  p.sm_count = ds.sm_count;
  p.slot = slot;
  p.solve_slots = L.slots;
  p.slot_doubles = L.slot_d;
  WaveDev w;
  w.n = n;
  w.nR = n;  // no dipole row: R is the caller's n x n packed block
  w.N = n_poles;
  w.a = a;
  w.l = l_dev;
  w.thr = const_cast<double*>(thresh);
  w.poles = const_cast<double*>(pole_E);
  w.E = Ech;
  w.flags0 = fl0;
  w.n_open = nop;

  const int64_t np = (int64_t)n * (n + 1) / 2;
  for (int64_t c0 = 0; c0 < n_e; c0 += chunk) {
    const int ne = (int)((n_e - c0) < chunk ? (n_e - c0) : chunk);
    cudaError_t e = launch_prep(w, energies + c0, ne, s);
    if (e == cudaSuccess) {
      static_flag_kernel<<<(ne + 255) / 256, 256, 0, s>>>(fl0, ne, bad);
      e = cudaGetLastError();
    }
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
      return static_fail(RM_ERR_CUDA, "kernel launch failed: ", cudaGetErrorString(e));
    }
  }
  return RM_OK;
}

extern "C" const char* rm_static_last_error(void) { return g_static_err; }

// Chunk and solve-slot counts the call would use for n_ch channels and n_sel selected channels on
// the current device (for tests and capacity planning; no device work).  Returns RM_ERR_ARG where
// the call itself would reject the sizes.
extern "C" rm_status_t rm_static_layout(int32_t n_ch, int32_t n_sel, int32_t* chunk_out, int32_t* slots_out) {
  using namespace rm;
  if (n_ch < 1 || n_sel < 1 || n_sel > RM_MAX_SEL) return static_fail(RM_ERR_ARG, "bad sizes");
  if (n_ch > kMaxChannels) return static_fail(RM_ERR_ARG, "n_ch above 640, the largest channel count of the solve");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return static_fail(RM_ERR_CUDA, "no CUDA device");
  }
  DeviceSetup ds;
  rm_status_t st = device_setup(dev, &ds);
  if (st != RM_OK) return st;
  if (solve_smem_bytes(n_ch) > (size_t)ds.smem_optin)
    return static_fail(RM_ERR_ARG, "n_ch too large for the solve kernel's shared memory");
  Layout L;
  if (!make_layout(n_ch, n_sel, ds.sm_count, L))
    return static_fail(RM_ERR_ARG, "n_ch too large for the library's static scratch (RM_STATIC_SCRATCH_BYTES)");
  if (chunk_out) *chunk_out = L.chunk;
  if (slots_out) *slots_out = L.slots;
  return RM_OK;
}
