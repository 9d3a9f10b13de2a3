// C ABI of the R-matrix outer-region sweep: plan management and the chunked
// per-energy pipeline (pole sum -> asymptotic data -> matching LU -> S-step).
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include <nvtx3/nvToolsExt.h>

#include "rm_internal.cuh"

using namespace rm;

namespace {


thread_local std::string g_err;

// Host-side fault injection for tests (no GPU fault is ever made): with RM_FAULT_ALLOC=k in the
// environment, the k-th device allocation of each rm_plan_create call fails as if cudaMalloc had
// run out of memory.  Read at the start of every rm_plan_create.
thread_local int g_alloc_fail_at = 0;
thread_local int g_alloc_count = 0;

long long env_ll(const char* name) {
  const char* v = std::getenv(name);
  if (!v || !*v) return 0;
  char* end = nullptr;
  const long long x = std::strtoll(v, &end, 10);
  return (end && *end == 0 && x > 0) ? x : 0;
}

// NVTX range around each ABI call and (with per-kernel timing) each kernel launch; a no-op unless
// a profiler is attached.
struct Nvtx {
  explicit Nvtx(const char* name) { nvtxRangePushA(name); }
  ~Nvtx() { nvtxRangePop(); }
};

rm_status_t fail(rm_status_t s, const std::string& msg) {
  g_err = msg;
  return s;
}

rm_status_t cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return e == cudaErrorMemoryAllocation ? RM_ERR_NOMEM : RM_ERR_CUDA;
}

#define RM_CUDA(call, where)                     \
  do {                                           \
    cudaError_t e__ = (call);                    \
    if (e__ != cudaSuccess) return cuda_fail(e__, where); \
  } while (0)

template <typename T>
rm_status_t dalloc(Plan* p, T** ptr, int64_t count) {
  *ptr = nullptr;
  if (count <= 0) return RM_OK;
  const size_t bytes = (size_t)count * sizeof(T);
  if (g_alloc_fail_at > 0 && ++g_alloc_count == g_alloc_fail_at)
    return fail(RM_ERR_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed (RM_FAULT_ALLOC)");
  cudaError_t e = cudaMalloc((void**)ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(RM_ERR_NOMEM, "device allocation of " + std::to_string(bytes) + " bytes failed");
  }
  p->workspace_bytes += (int64_t)bytes;
  return RM_OK;
}

void dfree(void* ptr) {
  if (ptr) cudaFree(ptr);
}

void free_plan(Plan* p) {
  if (!p) return;
  for (auto& w : p->waves) {
    dfree(w.l); dfree(w.thr); dfree(w.poles); dfree(w.W); dfree(w.E); dfree(w.flags0);
    dfree(w.n_open); dfree(w.eta); dfree(w.sig_tot); dfree(w.sig_sel); dfree(w.flags);
    dfree(w.pi_tot); dfree(w.pi_ch);
    SplitDev& sd = w.split;
    dfree(sd.omega); dfree(sd.pol); dfree(sd.sigma); dfree(sd.mult_p); dfree(sd.f_p); dfree(sd.klo);
    dfree(sd.khi); dfree(sd.tau); dfree(sd.mult_e); dfree(sd.Eh); dfree(sd.El); dfree(sd.tiles);
  }
  dfree(p->energies); dfree(p->sel_dev); dfree(p->Rbuf); dfree(p->asym); dfree(p->slot);
  dfree(p->err_word);
  GroupDev& G = p->grp;
  for (double* r : G.R) dfree(r);
  for (double* a : G.asym) dfree(a);
  for (uint32_t* d : G.D) dfree(d);
  dfree(G.dslice_waves);
  dfree(G.tc_waves); dfree(G.maps); dfree(G.tiles); dfree(G.near_waves); dfree(G.near_jobs);
  dfree(G.asym_waves); dfree(G.solve_waves); dfree(G.units); dfree(G.counter);
  if (G.exec) cudaGraphExecDestroy(G.exec);
  if (G.cap) cudaStreamDestroy(G.cap);
  for (int k = 0; k < RM_KERNEL_COUNT; ++k)
    for (auto& pr : p->ev_live[k]) { cudaEventDestroy(pr.first); cudaEventDestroy(pr.second); }
  for (auto e : p->ev_pool) cudaEventDestroy(e);
  delete p;
}

bool valid_mem(int32_t m) { return m == RM_MEM_HOST || m == RM_MEM_DEVICE; }

cudaMemcpyKind kind_in(int32_t mem) {
  return mem == RM_MEM_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
}
cudaMemcpyKind kind_out(int32_t mem) {
  return mem == RM_MEM_HOST ? cudaMemcpyDeviceToHost : cudaMemcpyDeviceToDevice;
}

rm_status_t check_wave_args(const rm_wave& w, int idx) {
  const std::string tag = "wave " + std::to_string(idx) + ": ";
  if (w.n_ch < 1 || w.n_ch > 640) return fail(RM_ERR_ARG, tag + "n_ch must be in [1, 640]");
  if (w.n_poles < 1) return fail(RM_ERR_ARG, tag + "n_poles must be >= 1");
  if (!(w.a > 0.0) || !(w.a < 1e300)) return fail(RM_ERR_ARG, tag + "radius a must be finite and > 0");
  if (!(w.z >= 0.0) || !(w.z < 1e300)) return fail(RM_ERR_ARG, tag + "charge z must be finite and >= 0");
  if (!w.l || !w.thresh || !w.pole_E || !w.W) return fail(RM_ERR_ARG, tag + "null input pointer");
  if (w.dip && !(w.e0 > -1e300 && w.e0 < 1e300)) return fail(RM_ERR_ARG, tag + "e0 must be finite");
  return RM_OK;
}

// Copy one wave's inputs into the plan's padded device buffers and validate.
rm_status_t upload_wave(Plan* p, WaveDev& d, const rm_wave& w, int32_t mem) {
  const cudaMemcpyKind k = kind_in(mem);
  cudaStream_t s = p->stream;
  RM_CUDA(cudaMemcpyAsync(d.l, w.l, sizeof(int32_t) * d.n, k, s), "copy l");
  RM_CUDA(cudaMemcpyAsync(d.thr, w.thresh, sizeof(double) * d.n, k, s), "copy thresholds");
  RM_CUDA(cudaMemcpyAsync(d.poles, w.pole_E, sizeof(double) * d.N, k, s), "copy poles");
  // pole-sum operand: [dipole row,] then the n channel rows, each padded to Npad
  RM_CUDA(cudaMemsetAsync(d.W, 0, sizeof(double) * (size_t)d.nR * d.Npad, s), "clear W");
  if (d.dip) RM_CUDA(cudaMemcpyAsync(d.W, w.dip, sizeof(double) * d.N, k, s), "copy dipole vector");
  RM_CUDA(cudaMemcpy2DAsync(d.W + (d.dip ? d.Npad : 0), sizeof(double) * d.Npad, w.W, sizeof(double) * d.N,
                            sizeof(double) * d.N, d.n, k, s), "copy W");
  d.e0 = w.e0;
  if (mem == RM_MEM_HOST) {
    int32_t lmax = 0;
    for (int i = 0; i < d.n; ++i) lmax = w.l[i] > lmax ? w.l[i] : lmax;
    d.lmax = lmax;
  }
  return RM_OK;
}

// Device work lists of the grouped run for the current group chunk.
rm_status_t group_setup(Plan* p) {
  if (p->n_e == 0) return RM_OK;
  if (is_split_like(p->prec)) RM_CUDA(group_setup_split(*p), "grouped split setup");
  RM_CUDA(group_setup_asym(*p), "grouped asymptotics setup");
  RM_CUDA(group_setup_solve(*p), "grouped solve setup");
  p->grp.ready = true;
  return RM_OK;
}

rm_status_t prepare(Plan* p, const rm_wave* waves, const double* energies, int32_t mem) {
  cudaStream_t s = p->stream;
  if (p->n_e > 0)
    RM_CUDA(cudaMemcpyAsync(p->energies, energies, sizeof(double) * p->n_e, kind_in(mem), s),
            "copy energies");
  RM_CUDA(cudaMemsetAsync(p->err_word, 0, sizeof(int32_t), s), "clear error word");
  for (int g = 0; g < p->n_waves; ++g) {
    WaveDev& d = p->waves[g];
    rm_status_t st = upload_wave(p, d, waves[g], mem);
    if (st != RM_OK) return st;
    // pad poles past N with a far value (D -> 0 there; W is zero there too)
    if (d.Npad > d.N) {
      std::vector<double> far(d.Npad - d.N, 1e300);
      RM_CUDA(cudaMemcpyAsync(d.poles + d.N, far.data(), sizeof(double) * far.size(),
                              cudaMemcpyHostToDevice, s), "pad poles");
      RM_CUDA(cudaStreamSynchronize(s), "pad poles");
    }
    RM_CUDA(launch_validate(d, d.N, p->energies, p->n_e, p->err_word, s), "validate kernel");
    p->launches++;
  }
  int32_t err = 0;
  RM_CUDA(cudaMemcpyAsync(&err, p->err_word, sizeof(int32_t), cudaMemcpyDeviceToHost, s), "read error word");
  RM_CUDA(cudaStreamSynchronize(s), "validate");
  if (err == RM_ERR_ORDER) return fail(RM_ERR_ORDER, "poles, thresholds or energies are not sorted ascending");
  if (err != 0) return fail(RM_ERR_ARG, "input contains NaN/Inf or an angular momentum outside [0, RM_LMAX]");
  for (int g = 0; g < p->n_waves; ++g) {
    WaveDev& d = p->waves[g];
    if (p->n_e > 0) {
      RM_CUDA(launch_prep(d, p->energies, p->n_e, s), "prep kernel");
      p->launches++;
    }
    if (p->n_e > 0) RM_CUDA(cudaMemsetAsync(d.flags, 0, p->n_e, s), "clear flags");
    if (is_split_like(p->prec)) {
      RM_CUDA(split_prepare(*p, d, s), "split-precision preparation");
      p->launches += 4;
    }
  }
  RM_CUDA(cudaStreamSynchronize(s), "prepare");
  for (int g = 0; g < p->n_waves; ++g)
    for (int q = 0; q < p->n_sel; ++q)
      if (p->sel[q] >= p->waves[g].n && p->n_waves == 1)
        return fail(RM_ERR_ARG, "selected initial channel out of range");
  rm_status_t st = group_setup(p);
  if (st != RM_OK) return st;
  p->ran = false;
  return RM_OK;
}

Plan* as_plan(rm_plan_t h) { return reinterpret_cast<Plan*>(h); }

cudaEvent_t pool_event(Plan* p) {
  if (!p->ev_pool.empty()) {
    cudaEvent_t e = p->ev_pool.back();
    p->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) { cudaGetLastError(); return nullptr; }
  return e;
}

// Bracket one kernel launch with events when profiling is on.
struct Prof {
  Plan* p;
  int k;
  cudaStream_t s;
  cudaEvent_t a = nullptr, b = nullptr;
  Prof(Plan* p_, int k_) : Prof(p_, k_, p_->prof, p_->stream, true) {}
  // count = false while capturing into a graph (graph launches are counted per replay)
  bool range = false;
  Prof(Plan* p_, int k_, bool on, cudaStream_t s_, bool count) : p(p_), k(k_), s(s_) {
    if (count) p->launches++;
    if (!on) return;
    static const char* names[RM_KERNEL_COUNT] = {"rm:polesum_fp64", "rm:polesum_split", "rm:near",
                                                 "rm:asym", "rm:solve", "rm:dslice"};
    nvtxRangePushA(names[k]);
    range = true;
    a = pool_event(p);
    b = pool_event(p);
    if (a) cudaEventRecord(a, s);
  }
  ~Prof() {
    if (range) nvtxRangePop();
    if (!a || !b) return;
    cudaEventRecord(b, s);
    p->ev_live[k].push_back({a, b});
  }
};

void prof_collect(Plan* p) {
  for (int k = 0; k < RM_KERNEL_COUNT; ++k) {
    for (auto& pr : p->ev_live[k]) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) {
        p->prof_ms[k] += ms;
        p->prof_n[k] += 1;
      } else {
        cudaGetLastError();
      }
      p->ev_pool.push_back(pr.first);
      p->ev_pool.push_back(pr.second);
    }
    p->ev_live[k].clear();
  }
}

rm_status_t check_range(Plan* p, int32_t wave, int64_t e0, int64_t e1) {
  if (!p) return fail(RM_ERR_ARG, "null plan");
  if (wave < 0 || wave >= p->n_waves) return fail(RM_ERR_ARG, "wave index out of range");
  if (e0 < 0 || e1 < e0 || e1 > p->n_e) return fail(RM_ERR_ARG, "energy range out of bounds");
  if (cudaSetDevice(p->device) != cudaSuccess) return fail(RM_ERR_CUDA, "cudaSetDevice failed");
  return RM_OK;
}

// Pole sum for one chunk into R (device, [ne * np]).
rm_status_t polesum_chunk(Plan* p, const WaveDev& w, int64_t c0, int ne, double* R) {
  if (p->prec == RM_PREC_FP64) {
    Prof pr(p, RM_KERNEL_POLESUM_FP64);
    RM_CUDA(launch_polesum_fp64(w, c0, ne, R, p->stream), "FP64 pole-sum kernel");
    return RM_OK;
  }
  if (p->prec == RM_PREC_FP32_SIMT) {
    Prof pr(p, RM_KERNEL_POLESUM_SPLIT);
    RM_CUDA(launch_polesum_fp32(w, c0, ne, R, p->stream), "FP32 pole-sum kernel");
  } else {
    Prof pr(p, RM_KERNEL_POLESUM_SPLIT);
    RM_CUDA(launch_polesum_split(*p, w, c0, ne, R, p->stream), "split pole-sum kernel");
  }
  {
    Prof pr(p, RM_KERNEL_NEAR);
    RM_CUDA(launch_near(*p, w, c0, ne, R, p->stream), "near-window kernel");
  }
  return RM_OK;
}

// Pipeline over [e0, e1) for one wave.  Any output may be null; device outputs
// are written directly, index 0 = energy e0.
struct RangeOut {
  double* R = nullptr;  // [ne * np]
  SolveOut so;          // K, eta, sig_tot, sig_sel, flags, n_open (offset by e0)
  bool need_solve = false;
};

rm_status_t run_range(Plan* p, int32_t wave, int64_t e0, int64_t e1, const RangeOut& o) {
  const WaveDev& w = p->waves[wave];
  const int64_t np = (int64_t)w.n * (w.n + 1) / 2;
  for (int64_t c0 = e0; c0 < e1; c0 += p->chunk) {
    const int ne = (int)((e1 - c0) < p->chunk ? (e1 - c0) : p->chunk);
    const int64_t off = c0 - e0;
    // with a dipole row the pole sum's rows are (dipole, channels): compute into the
    // workspace and hand out the channel block
    double* R = (o.R && !w.dip) ? o.R + off * np : p->Rbuf;
    rm_status_t st = polesum_chunk(p, w, c0, ne, R);
    if (st != RM_OK) return st;
    if (o.R && w.dip)
      RM_CUDA(cudaMemcpy2DAsync(o.R + off * np, sizeof(double) * np, R + w.roff(), sizeof(double) * w.npR(),
                                sizeof(double) * np, ne, cudaMemcpyDeviceToDevice, p->stream), "channel block of R");
    if (!o.need_solve) continue;
    const int ld = p->chunk * p->n_max;
    {
      Prof pr(p, RM_KERNEL_ASYM);
      RM_CUDA(launch_asym(w, c0, ne, p->asym, ld, p->stream), "asymptotic-function kernel");
    }
    SolveOut so = o.so;
    if (so.K) so.K += off * w.n * w.n;
    if (so.eta) so.eta += off;
    if (so.sig_tot) so.sig_tot += off * p->n_sel;
    if (so.sig_sel) so.sig_sel += off * p->n_sel * w.n;
    if (so.flags) so.flags += off;
    if (so.n_open) so.n_open += off;
    if (so.pi_tot) so.pi_tot += off;
    if (so.pi_ch) so.pi_ch += off * w.n;
    {
      Prof pr(p, RM_KERNEL_SOLVE);
      RM_CUDA(launch_solve(*p, w, c0, ne, R, p->asym, ld, so, p->stream), "solve kernel");
    }
  }
  return RM_OK;
}

// Read the device error word (after the stream was synchronised).
rm_status_t check_err_word(Plan* p) {
  int32_t err = 0;
  RM_CUDA(cudaMemcpy(&err, p->err_word, sizeof(int32_t), cudaMemcpyDeviceToHost), "read error word");
  if (err == RM_ERR_TIMEOUT) return fail(RM_ERR_TIMEOUT, "a device-side wait ran out (tensor-core pipeline)");
  if (err != 0) return fail((rm_status_t)err, "device reported an error");
  return RM_OK;
}

// device scratch for host-memory outputs of the per-range calls
struct Scratch {
  void* ptr = nullptr;
  ~Scratch() { if (ptr) cudaFree(ptr); }
};

template <typename T>
rm_status_t out_buf(Plan* p, T* user, int64_t count, int32_t mem, Scratch& sc, T** dev) {
  *dev = nullptr;
  if (!user || count <= 0) return RM_OK;
  if (mem == RM_MEM_DEVICE) { *dev = user; return RM_OK; }
  cudaError_t e = cudaMalloc(&sc.ptr, sizeof(T) * (size_t)count);
  if (e != cudaSuccess) { cudaGetLastError(); return fail(RM_ERR_NOMEM, "scratch allocation failed"); }
  *dev = reinterpret_cast<T*>(sc.ptr);
  return RM_OK;
}

template <typename T>
rm_status_t copy_back(Plan* p, T* user, T* dev, int64_t count, int32_t mem) {
  if (!user || mem != RM_MEM_HOST || count <= 0) return RM_OK;
  RM_CUDA(cudaMemcpyAsync(user, dev, sizeof(T) * (size_t)count, cudaMemcpyDeviceToHost, p->stream), "copy out");
  return RM_OK;
}

// Enqueue the grouped sweep (every wave per launch) on stream s.
rm_status_t enqueue_grouped(Plan* p, cudaStream_t s, bool prof, int* kernels, bool count) {
  GroupDev& G = p->grp;
  int nk = 0;
  for (int64_t c0 = 0; c0 < p->n_e; c0 += G.chunk) {
    const int ne = (int)((p->n_e - c0) < G.chunk ? (p->n_e - c0) : G.chunk);
    if (is_split_like(p->prec)) {
      if (p->prec == RM_PREC_FP32_SIMT) {
        for (int g = 0; g < p->n_waves; ++g) {
          Prof pr(p, RM_KERNEL_POLESUM_SPLIT, prof, s, count);
          RM_CUDA(launch_polesum_fp32(p->waves[g], c0, ne, G.R[g], s), "FP32 pole-sum kernel");
          ++nk;
        }
        --nk;
      } else {
        if (G.dt()) {
          Prof pr(p, RM_KERNEL_DSLICE, prof, s, count);
          RM_CUDA(launch_dslice_grouped(*p, c0, ne, s), "grouped D-slice kernel");
          ++nk;
        }
        Prof pr(p, RM_KERNEL_POLESUM_SPLIT, prof, s, count);
        RM_CUDA(launch_polesum_split_grouped(*p, c0, ne, s), "grouped split pole-sum kernel");
      }
      {
        Prof pr(p, RM_KERNEL_NEAR, prof, s, count);
        RM_CUDA(launch_near_grouped(*p, c0, ne, s), "grouped near-window kernel");
      }
      nk += 2;
    } else {
      for (int g = 0; g < p->n_waves; ++g) {
        Prof pr(p, RM_KERNEL_POLESUM_FP64, prof, s, count);
        RM_CUDA(launch_polesum_fp64(p->waves[g], c0, ne, G.R[g], s), "FP64 pole-sum kernel");
        ++nk;
      }
    }
    {
      Prof pr(p, RM_KERNEL_ASYM, prof, s, count);
      RM_CUDA(launch_asym_grouped(*p, c0, ne, s), "grouped asymptotics kernel");
    }
    {
      Prof pr(p, RM_KERNEL_SOLVE, prof, s, count);
      RM_CUDA(launch_solve_grouped(*p, c0, ne, s), "grouped solve kernel");
    }
    nk += 2;
  }
  if (kernels) *kernels = nk;
  return RM_OK;
}

// Capture the grouped sweep once into a CUDA graph (on a private stream).
rm_status_t build_graph(Plan* p) {
  GroupDev& G = p->grp;
  if (G.exec) return RM_OK;
  if (!G.cap) RM_CUDA(cudaStreamCreateWithFlags(&G.cap, cudaStreamNonBlocking), "create capture stream");
  RM_CUDA(cudaStreamBeginCapture(G.cap, cudaStreamCaptureModeThreadLocal), "begin capture");
  int nk = 0;
  rm_status_t st = enqueue_grouped(p, G.cap, false, &nk, false);
  cudaGraph_t graph = nullptr;
  cudaError_t e = cudaStreamEndCapture(G.cap, &graph);
  if (st != RM_OK) {
    if (graph) cudaGraphDestroy(graph);
    return st;
  }
  if (e != cudaSuccess) return cuda_fail(e, "end capture");
  e = cudaGraphInstantiate(&G.exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e != cudaSuccess) {
    G.exec = nullptr;
    return cuda_fail(e, "instantiate graph");
  }
  G.graph_kernels = nk;
  return RM_OK;
}

// Autotuned choices (energy chunk and tensor-core cluster shape) are cached in
// an optional text file, one "key|chunk cluster_x cluster_y" line per plan
// shape, keyed by the plan's sizes.
std::string tune_key(const Plan* p) {
  std::string k = "rm3 prec=" + std::to_string(p->prec) + " prod=" + std::to_string(p->slices) +
                  " pair=" + std::to_string(p->grp.tc_pair ? 1 : 0) + " ne=" + std::to_string(p->n_e) +
                  " sel=" + std::to_string(p->n_sel);
  for (const auto& w : p->waves) k += " " + std::to_string(w.nR) + "x" + std::to_string(w.N);
  return k;
}

struct Tuned {
  int chunk = 0, cx = 1, cy = 1;
};

bool cache_lookup(const char* path, const std::string& key, Tuned& t) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char line[8192];
  bool found = false;
  while (fgets(line, sizeof(line), f)) {
    std::string l(line);
    const size_t bar = l.rfind('|');
    if (bar == std::string::npos || l.substr(0, bar) != key) continue;
    Tuned v;
    if (sscanf(l.c_str() + bar + 1, "%d %d %d", &v.chunk, &v.cx, &v.cy) == 3) {
      t = v;
      found = true;
    }
  }
  fclose(f);
  return found;
}

void cache_store(const char* path, const std::string& key, const Tuned& t) {
  if (!path) return;
  FILE* f = fopen(path, "a");
  if (!f) return;
  fprintf(f, "%s|%d %d %d\n", key.c_str(), t.chunk, t.cx, t.cy);
  fclose(f);
}

// Device time of one grouped pass over the first ne_t energies (after one
// untimed pass), at the plan's current chunk and cluster shape.
rm_status_t time_grouped(Plan* p, int64_t ne_t, cudaEvent_t a, cudaEvent_t b, float* ms) {
  rm_status_t st = group_setup(p);
  if (st != RM_OK) return st;
  const int64_t n_e_saved = p->n_e;
  p->n_e = ne_t;
  st = enqueue_grouped(p, p->stream, false, nullptr, true);
  if (st == RM_OK) {
    cudaEventRecord(a, p->stream);
    st = enqueue_grouped(p, p->stream, false, nullptr, true);
    cudaEventRecord(b, p->stream);
  }
  p->n_e = n_e_saved;
  if (st != RM_OK) return st;
  RM_CUDA(cudaEventSynchronize(b), "autotune timing");
  RM_CUDA(cudaEventElapsedTime(ms, a, b), "autotune timing");
  return RM_OK;
}

// Tensor-core cluster shapes in order of preference (the automatic shape is the
// first one the device co-schedules).  Shapes with cluster_x = 1 take the D
// slices by TMA from the D-slice kernel; the others form them in the pole sum.
constexpr int kShapes[][2] = {{1, 2}, {1, 4}, {2, 2}, {1, 1}, {4, 1}, {2, 1}};

rm_status_t autotune(Plan* p, const char* cache, int chunk_max, bool tune_chunk, bool tune_cluster) {
  // 1. cluster shape: every co-schedulable shape, timed on the first
  //    min(n_e, chunk, 4096) energies (chunk: 2048 when it is tuned next);
  // 2. chunk (only when the mesh does not fit one chunk): 256, 512, ... up to
  //    8192 (and chunk_max), timed on the first min(n_e, largest candidate)
  //    energies; a smaller chunk must win by 3%.
  GroupDev& G = p->grp;
  const std::string key = tune_key(p);
  Tuned t;
  if (cache_lookup(cache, key, t) && t.chunk > 0 && t.chunk <= chunk_max &&
      (!tune_cluster || polesum_cluster_ok(t.cx, t.cy, polesum_slice_planes(p->slices), p->grp.tc_pair))) {
    if (tune_chunk) G.chunk = t.chunk;
    if (tune_cluster) {
      G.tc_cx = t.cx;
      G.tc_cy = t.cy;
    }
    return group_setup(p);
  }
  cudaEvent_t a = nullptr, b = nullptr;
  RM_CUDA(cudaEventCreate(&a), "event");
  RM_CUDA(cudaEventCreate(&b), "event");
  rm_status_t st = RM_OK;
  if (tune_cluster) {
    const int c0 = tune_chunk ? (chunk_max < 2048 ? chunk_max : 2048) : G.chunk;
    int64_t ne_t = p->n_e < c0 ? p->n_e : c0;
    if (ne_t > 4096) ne_t = 4096;  // the first 4096 energies are enough to rank the shapes
    if (tune_chunk) G.chunk = c0;
    double best_t = 1e300;
    int bx = G.tc_cx, by = G.tc_cy;
    for (const auto& sh : kShapes) {
      if (!polesum_cluster_ok(sh[0], sh[1], polesum_slice_planes(p->slices), p->grp.tc_pair)) continue;
      G.tc_cx = sh[0];
      G.tc_cy = sh[1];
      float ms = 0.f;
      if ((st = time_grouped(p, ne_t, a, b, &ms)) != RM_OK) break;
      if (ms < best_t) {
        best_t = ms;
        bx = sh[0];
        by = sh[1];
      }
    }
    G.tc_cx = bx;
    G.tc_cy = by;
  }
  if (st == RM_OK && tune_chunk) {
    const int c_top = chunk_max < 8192 ? chunk_max : 8192;
    const int64_t ne_t = p->n_e < c_top ? p->n_e : c_top;
    double best_t = 1e300;
    int best = c_top;
    std::vector<int> cands;
    cands.push_back(c_top);
    for (int c = 1 << 30; c >= 256; c >>= 1)
      if (c < c_top) cands.push_back(c);  // descending
    for (int c : cands) {
      G.chunk = c;
      float ms = 0.f;
      if ((st = time_grouped(p, ne_t, a, b, &ms)) != RM_OK) break;
      if (ms < best_t * 0.97) {  // a smaller chunk must be clearly faster
        best_t = ms;
        best = c;
      }
    }
    G.chunk = best;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != RM_OK) return st;
  st = group_setup(p);
  if (st == RM_OK) cache_store(cache, key, Tuned{G.chunk, G.tc_cx, G.tc_cy});
  p->autotuned = true;
  return st;
}

}  // namespace

extern "C" {

void rm_options_default(rm_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->prec = RM_PREC_FP64;
  opt->delta = 0.05;
  opt->slices = 0;
  opt->sel_init = nullptr;
  opt->n_sel = 0;
  opt->mem = RM_MEM_HOST;
  opt->chunk = 0;
}

const char* rm_status_str(rm_status_t s) {
  switch (s) {
    case RM_OK: return "ok";
    case RM_ERR_ARG: return "invalid argument";
    case RM_ERR_ORDER: return "input not sorted ascending";
    case RM_ERR_NOMEM: return "out of memory";
    case RM_ERR_CUDA: return "CUDA error";
    case RM_ERR_TIMEOUT: return "device wait timed out";
    case RM_ERR_STATE: return "invalid plan state";
  }
  return "unknown status";
}

const char* rm_last_error(void) { return g_err.c_str(); }

rm_status_t rm_plan_create(rm_plan_t* out, const rm_wave* waves, int32_t n_waves,
                           const double* energies, int64_t n_e, const rm_options* opt,
                           void* cuda_stream) {
  Nvtx range("rm_plan_create");
  try {
    if (!out) return fail(RM_ERR_ARG, "out is null");
    *out = nullptr;
    g_alloc_fail_at = (int)env_ll("RM_FAULT_ALLOC");
    g_alloc_count = 0;
    if (!waves || n_waves < 1) return fail(RM_ERR_ARG, "need at least one wave");
    if (n_e < 0 || (n_e > 0 && !energies)) return fail(RM_ERR_ARG, "bad energy mesh");
    rm_options o;
    if (opt) o = *opt; else rm_options_default(&o);
    if (!valid_mem(o.mem)) return fail(RM_ERR_ARG, "bad memory space");
    if (o.prec < RM_PREC_FP64 || o.prec > RM_PREC_FP32_SIMT) return fail(RM_ERR_ARG, "bad precision mode");
    if (o.prec != RM_PREC_FP64 && !(o.delta > 0.0)) return fail(RM_ERR_ARG, "delta must be > 0");
    if (o.chunk < 0) return fail(RM_ERR_ARG, "chunk must be >= 0");
    if (!(o.slices == 0 || o.slices == 3 || o.slices == 6 || o.slices == 10 || o.slices == 13 || o.slices == 15))
      return fail(RM_ERR_ARG, "slices must be 0 (default), 3, 6, 10, 13 or 15 slice products");
    if (o.slices != 0 && o.prec != RM_PREC_SPLIT_BF16 && o.prec != RM_PREC_SPLIT_FP16)
      return fail(RM_ERR_ARG, "slices applies to the tensor-core modes (SPLIT_BF16, SPLIT_FP16) only");
    if (o.slices == 15 && o.prec != RM_PREC_SPLIT_BF16)
      return fail(RM_ERR_ARG, "slices = 15 needs BF16 slices (FP16 cannot hold the fifth, 2^-25 small)");
    if (o.solve_prec != RM_SOLVE_FP64 && o.solve_prec != RM_SOLVE_MIXED && o.solve_prec != RM_SOLVE_FP64_LU)
      return fail(RM_ERR_ARG, "bad solve precision");
    if (o.mma_pair < -1 || o.mma_pair > 1) return fail(RM_ERR_ARG, "mma_pair must be -1, 0 or 1");
    if (!(o.cluster_x == 0 || o.cluster_x == 1 || o.cluster_x == 2 || o.cluster_x == 4) ||
        !(o.cluster_y == 0 || o.cluster_y == 1 || o.cluster_y == 2 || o.cluster_y == 4) ||
        (o.cluster_x > 0 && o.cluster_y > 0 && o.cluster_x * o.cluster_y > 8))
      return fail(RM_ERR_ARG, "cluster_x, cluster_y must be 0, 1, 2 or 4 with at most 8 CTAs per cluster");
    int n_sel = 1;
    int32_t sel[RM_MAX_SEL] = {0};
    if (o.sel_init) {
      if (o.n_sel < 1 || o.n_sel > RM_MAX_SEL) return fail(RM_ERR_ARG, "n_sel out of range");
      n_sel = o.n_sel;
      for (int q = 0; q < n_sel; ++q) {
        if (o.sel_init[q] < 0) return fail(RM_ERR_ARG, "negative selected channel");
        sel[q] = o.sel_init[q];
      }
    }
    for (int g = 0; g < n_waves; ++g) {
      rm_status_t st = check_wave_args(waves[g], g);
      if (st != RM_OK) return st;
    }
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) { cudaGetLastError(); return fail(RM_ERR_CUDA, "no CUDA device"); }
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) { cudaGetLastError(); return fail(RM_ERR_CUDA, "cannot query device"); }
    if (prop.major != 10 || prop.minor != 3)
      return fail(RM_ERR_CUDA, std::string("needs an sm_103 (GB300) device, found ") + prop.name);

    Plan* p = new (std::nothrow) Plan();
    if (!p) return fail(RM_ERR_NOMEM, "host allocation failed");
    int grp_chunk_max = 0;
    p->device = dev;
    p->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
    p->n_waves = n_waves;
    p->n_e = n_e;
    p->prec = o.prec;
    p->delta = o.delta;
    p->slices = o.slices ? o.slices : (o.prec == RM_PREC_SPLIT_FP16 ? 13 : RM_DEFAULT_SLICES);
    p->grp.tc_pair = o.mma_pair >= 0;
    p->fault_wait = env_ll("RM_FAULT_WAIT_CYCLES");
    p->z_force_fp64 = env_ll("RM_TEST_Z_FP64") == 1 ? 1 : 0;
    p->n_sel = n_sel;
    std::memcpy(p->sel, sel, sizeof(sel));
    p->sm_count = prop.multiProcessorCount;
    p->waves.resize(n_waves);
    int n_max = 0, nR_max = 0;
    int64_t np_max = 0;
    rm_status_t st = RM_OK;
    for (int g = 0; g < n_waves && st == RM_OK; ++g) {
      WaveDev& d = p->waves[g];
      d.n = waves[g].n_ch;
      d.N = waves[g].n_poles;
      d.Npad = (d.N + 63) / 64 * 64;
      d.a = waves[g].a;
      d.z = waves[g].z;
      d.dip = waves[g].dip != nullptr;
      d.e0 = waves[g].e0;
      d.nR = d.n + (d.dip ? 1 : 0);
      n_max = d.n > n_max ? d.n : n_max;
      nR_max = d.nR > nR_max ? d.nR : nR_max;
      const int64_t np = d.npR();
      np_max = np > np_max ? np : np_max;
      if ((st = dalloc(p, &d.l, d.n)) != RM_OK) break;
      if ((st = dalloc(p, &d.thr, d.n)) != RM_OK) break;
      if ((st = dalloc(p, &d.poles, d.Npad)) != RM_OK) break;
      if ((st = dalloc(p, &d.W, (int64_t)d.nR * d.Npad)) != RM_OK) break;
      if ((st = dalloc(p, &d.E, n_e)) != RM_OK) break;
      if ((st = dalloc(p, &d.flags0, n_e)) != RM_OK) break;
      if ((st = dalloc(p, &d.n_open, n_e)) != RM_OK) break;
      if ((st = dalloc(p, &d.eta, n_e)) != RM_OK) break;
      if ((st = dalloc(p, &d.sig_tot, n_e * n_sel)) != RM_OK) break;
      if ((st = dalloc(p, &d.sig_sel, n_e * n_sel * d.n)) != RM_OK) break;
      if ((st = dalloc(p, &d.flags, n_e)) != RM_OK) break;
      if (d.dip && (st = dalloc(p, &d.pi_tot, n_e)) != RM_OK) break;
      if (d.dip && (st = dalloc(p, &d.pi_ch, n_e * d.n)) != RM_OK) break;
      if (is_split_like(o.prec)) {
        SplitDev& sd = d.split;
        if ((st = dalloc(p, &sd.omega, 2ll * d.nR * d.Npad)) != RM_OK) break;
        if ((st = dalloc(p, &sd.pol, 2ll * d.Npad)) != RM_OK) break;
        if ((st = dalloc(p, &sd.sigma, d.nR)) != RM_OK) break;
        if ((st = dalloc(p, &sd.mult_p, np)) != RM_OK) break;
        if ((st = dalloc(p, &sd.f_p, np)) != RM_OK) break;
        if ((st = dalloc(p, &sd.klo, n_e)) != RM_OK) break;
        if ((st = dalloc(p, &sd.khi, n_e)) != RM_OK) break;
        if ((st = dalloc(p, &sd.tau, n_e)) != RM_OK) break;
        if ((st = dalloc(p, &sd.mult_e, n_e)) != RM_OK) break;
        if ((st = dalloc(p, &sd.Eh, n_e)) != RM_OK) break;
        if ((st = dalloc(p, &sd.El, n_e)) != RM_OK) break;
        std::vector<int2> tl = split_tiles(d.nR);
        sd.n_tiles = (int)tl.size();
        if ((st = dalloc(p, &sd.tiles, sd.n_tiles)) != RM_OK) break;
        if (cudaMemcpy(sd.tiles, tl.data(), sizeof(int2) * tl.size(), cudaMemcpyHostToDevice) != cudaSuccess) {
          st = fail(RM_ERR_CUDA, "copy tile list");
          break;
        }
      }
    }
    p->n_max = n_max;
    p->nR_max = nR_max;
    if (st == RM_OK) {
      int chunk = o.chunk;
      if (chunk == 0) {
        const int64_t budget = (is_split_like(o.prec) ? 288ll : 96ll) << 20;
        int64_t c = budget / (np_max * 8) / 128 * 128;
        c = c < 128 ? 128 : (c > 8192 ? 8192 : c);
        chunk = (int)c;
      }
      if (n_e > 0 && chunk > n_e) chunk = (int)n_e;
      if (chunk < 1) chunk = 1;
      p->chunk = chunk;
      p->solve_mixed = o.solve_prec == RM_SOLVE_MIXED ? 1 : 0;
      p->solve_bps = solve_blocks_per_sm(n_max, p->solve_mixed != 0);
      p->solve_slots = p->sm_count * p->solve_bps;
      p->solve_lu = o.solve_prec == RM_SOLVE_FP64_LU ? 1 : 0;
      p->slot_doubles = solve_slot_doubles(n_max, n_sel + 1, p->solve_mixed != 0);  // + the dipole column
      if (st == RM_OK) st = dalloc(p, &p->energies, n_e);
      if (st == RM_OK) st = dalloc(p, &p->sel_dev, n_sel);
      if (st == RM_OK) st = dalloc(p, &p->Rbuf, (int64_t)chunk * np_max);
      if (st == RM_OK) st = dalloc(p, &p->asym, 4ll * chunk * n_max);
      if (st == RM_OK) st = dalloc(p, &p->slot, (int64_t)p->solve_slots * p->slot_doubles);
      if (st == RM_OK) st = dalloc(p, &p->err_word, 1);
      // grouped-run buffers (all waves at once).  R for the whole mesh when it
      // fits min(24 GiB, a third of free device memory): one launch per kernel
      // and sweep, no chunk tails; otherwise chunks (autotuned when asked).
      // per energy and wave: R, the asymptotic data and (tensor-core modes) the D slices,
      // 4 or 5 x 2 bytes per pole (in units of 8 bytes)
      const bool dslices = is_split_like(o.prec) && o.prec != RM_PREC_FP32_SIMT;
      const int planes = polesum_slice_planes(p->slices);
      int64_t per_e = 0;
      for (const auto& w : p->waves)
        per_e += w.npR() + 4ll * w.n + (dslices ? ((int64_t)w.Npad * planes + 3) / 4 : 0);
      size_t free_b = 0, total_b = 0;
      if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); free_b = 2ull << 30; }
      int64_t budget = (int64_t)(free_b / 3);
      if (budget > (24ll << 30)) budget = 24ll << 30;
      int64_t cmax = o.chunk > 0 ? o.chunk : budget / (8 * per_e);
      if (o.chunk == 0 && cmax < n_e && cmax >= 256) cmax = cmax / 256 * 256;
      if (cmax < 1) cmax = 1;
      if (n_e > 0 && cmax > n_e) cmax = n_e;
      grp_chunk_max = (int)(cmax > (1 << 30) ? (1 << 30) : cmax);
      p->grp.chunk = o.chunk > 0 ? o.chunk : grp_chunk_max;
      p->grp.R.assign(n_waves, nullptr);
      p->grp.asym.assign(n_waves, nullptr);
      p->grp.D.assign(n_waves, nullptr);
      for (int g = 0; g < n_waves && st == RM_OK; ++g) {
        const WaveDev& d = p->waves[g];
        st = dalloc(p, &p->grp.R[g], cmax * d.npR());
        if (st == RM_OK) st = dalloc(p, &p->grp.asym[g], 4ll * cmax * d.n);
        if (st == RM_OK && dslices)
          st = dalloc(p, &p->grp.D[g], (int64_t)planes * cmax * (d.Npad / 2));  // planes x Npad/2 words
      }
      p->grp.d_rows = (st == RM_OK && dslices) ? (int)cmax : 0;
    }
    if (st == RM_OK) {
      if (cudaMemcpy(p->sel_dev, p->sel, sizeof(int32_t) * n_sel, cudaMemcpyHostToDevice) != cudaSuccess)
        st = fail(RM_ERR_CUDA, "copy selected channels");
    }
    if (st == RM_OK && solve_smem_bytes(n_max) > (size_t)prop.sharedMemPerBlockOptin)
      st = fail(RM_ERR_ARG, "n_ch too large for the solve kernel's shared memory");
    if (st == RM_OK && is_split_like(o.prec) &&
        (polesum_tc_smem_bytes() > (size_t)prop.sharedMemPerBlockOptin ||
         near_smem_bytes(nR_max) > (size_t)prop.sharedMemPerBlockOptin))
      st = fail(RM_ERR_ARG, "split-precision kernels do not fit this device's shared memory");
    if (st == RM_OK && is_split_like(o.prec)) {
      // explicit cluster shape (a missing dimension is 1); automatic: the first
      // shape of the preference list that the device co-schedules
      if (o.cluster_x > 0 || o.cluster_y > 0) {
        p->grp.tc_cx = o.cluster_x > 0 ? o.cluster_x : 1;
        p->grp.tc_cy = o.cluster_y > 0 ? o.cluster_y : 1;
        if (!polesum_cluster_ok(p->grp.tc_cx, p->grp.tc_cy, polesum_slice_planes(p->slices), p->grp.tc_pair))
          st = fail(RM_ERR_ARG, "cluster shape cannot be co-scheduled on this device");
      } else {
        p->grp.tc_cx = 1;
        p->grp.tc_cy = 1;
        for (const auto& sh : kShapes) {
          if (polesum_cluster_ok(sh[0], sh[1], polesum_slice_planes(p->slices), p->grp.tc_pair)) {
            p->grp.tc_cx = sh[0];
            p->grp.tc_cy = sh[1];
            break;
          }
        }
        cudaGetLastError();
      }
    }
    if (st == RM_OK) st = prepare(p, waves, energies, o.mem);
    if (st == RM_OK && o.autotune && n_e > 0) {
      // a whole-mesh chunk (when it fits) has the fewest launches and the shortest
      // solve tail, so the chunk is tuned only when the mesh must be split
      const bool tune_chunk = o.chunk == 0 && grp_chunk_max >= 256 && grp_chunk_max < n_e;
      const bool tune_cluster = is_split_like(o.prec) && o.cluster_x == 0 && o.cluster_y == 0;
      if (tune_chunk || tune_cluster) st = autotune(p, o.tune_cache, grp_chunk_max, tune_chunk, tune_cluster);
    }
    if (st != RM_OK) {
      free_plan(p);
      return st;
    }
    *out = reinterpret_cast<rm_plan_t>(p);
    return RM_OK;
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_plan_load(rm_plan_t h, const rm_wave* waves, const double* energies, int32_t mem) {
  Nvtx range("rm_plan_load");
  try {
    Plan* p = as_plan(h);
    if (!p) return fail(RM_ERR_ARG, "null plan");
    if (!waves || (p->n_e > 0 && !energies) || !valid_mem(mem)) return fail(RM_ERR_ARG, "bad arguments");
    for (int g = 0; g < p->n_waves; ++g) {
      rm_status_t st = check_wave_args(waves[g], g);
      if (st != RM_OK) return st;
      if (waves[g].n_ch != p->waves[g].n || waves[g].n_poles != p->waves[g].N ||
          (waves[g].dip != nullptr) != p->waves[g].dip)
        return fail(RM_ERR_ARG, "wave shape (or dipole presence) differs from the plan's");
      p->waves[g].a = waves[g].a;
      p->waves[g].z = waves[g].z;
    }
    if (cudaSetDevice(p->device) != cudaSuccess) return fail(RM_ERR_CUDA, "cudaSetDevice failed");
    return prepare(p, waves, energies, mem);
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_rmatrix(rm_plan_t h, int32_t wave, int64_t e0, int64_t e1, double* R_packed, int32_t mem) {
  Nvtx range("rm_rmatrix");
  try {
    Plan* p = as_plan(h);
    rm_status_t st = check_range(p, wave, e0, e1);
    if (st != RM_OK) return st;
    if (!R_packed || !valid_mem(mem)) return fail(RM_ERR_ARG, "bad output");
    const WaveDev& w = p->waves[wave];
    const int64_t np = (int64_t)w.n * (w.n + 1) / 2;
    if (mem == RM_MEM_DEVICE) {
      RangeOut o;
      o.R = R_packed;
      return run_range(p, wave, e0, e1, o);
    }
    for (int64_t c0 = e0; c0 < e1; c0 += p->chunk) {
      const int64_t c1 = (e1 - c0) < p->chunk ? e1 : c0 + p->chunk;
      RangeOut o;  // into Rbuf
      st = run_range(p, wave, c0, c1, o);
      if (st != RM_OK) return st;
      RM_CUDA(cudaMemcpy2DAsync(R_packed + (c0 - e0) * np, sizeof(double) * np, p->Rbuf + w.roff(),
                                sizeof(double) * w.npR(), sizeof(double) * np, c1 - c0, cudaMemcpyDeviceToHost,
                                p->stream), "copy R");
      RM_CUDA(cudaStreamSynchronize(p->stream), "rm_rmatrix");
    }
    return check_err_word(p);
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_kmatrix(rm_plan_t h, int32_t wave, int64_t e0, int64_t e1, double* K, int32_t* n_open,
                       uint8_t* flags, int32_t mem) {
  Nvtx range("rm_kmatrix");
  try {
    Plan* p = as_plan(h);
    rm_status_t st = check_range(p, wave, e0, e1);
    if (st != RM_OK) return st;
    if (!valid_mem(mem)) return fail(RM_ERR_ARG, "bad memory space");
    const WaveDev& w = p->waves[wave];
    const int64_t ne = e1 - e0;
    Scratch sK, sN, sF;
    RangeOut o;
    o.need_solve = true;
    o.so.do_xsec = false;
    if ((st = out_buf(p, K, ne * w.n * w.n, mem, sK, &o.so.K)) != RM_OK) return st;
    if ((st = out_buf(p, n_open, ne, mem, sN, &o.so.n_open)) != RM_OK) return st;
    if ((st = out_buf(p, flags, ne, mem, sF, &o.so.flags)) != RM_OK) return st;
    if ((st = run_range(p, wave, e0, e1, o)) != RM_OK) return st;
    if ((st = copy_back(p, K, o.so.K, ne * w.n * w.n, mem)) != RM_OK) return st;
    if ((st = copy_back(p, n_open, o.so.n_open, ne, mem)) != RM_OK) return st;
    if ((st = copy_back(p, flags, o.so.flags, ne, mem)) != RM_OK) return st;
    if (mem == RM_MEM_HOST) {
      RM_CUDA(cudaStreamSynchronize(p->stream), "rm_kmatrix");
      return check_err_word(p);
    }
    return RM_OK;
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_xsec(rm_plan_t h, int32_t wave, int64_t e0, int64_t e1, double* eigsum, double* sig_tot,
                    double* sig_sel, int32_t mem) {
  Nvtx range("rm_xsec");
  try {
    Plan* p = as_plan(h);
    rm_status_t st = check_range(p, wave, e0, e1);
    if (st != RM_OK) return st;
    if (!valid_mem(mem)) return fail(RM_ERR_ARG, "bad memory space");
    const WaveDev& w = p->waves[wave];
    const int64_t ne = e1 - e0;
    Scratch s1, s2, s3;
    RangeOut o;
    o.need_solve = true;
    o.so.do_xsec = true;
    if ((st = out_buf(p, eigsum, ne, mem, s1, &o.so.eta)) != RM_OK) return st;
    if ((st = out_buf(p, sig_tot, ne * p->n_sel, mem, s2, &o.so.sig_tot)) != RM_OK) return st;
    if ((st = out_buf(p, sig_sel, ne * p->n_sel * w.n, mem, s3, &o.so.sig_sel)) != RM_OK) return st;
    if ((st = run_range(p, wave, e0, e1, o)) != RM_OK) return st;
    if ((st = copy_back(p, eigsum, o.so.eta, ne, mem)) != RM_OK) return st;
    if ((st = copy_back(p, sig_tot, o.so.sig_tot, ne * p->n_sel, mem)) != RM_OK) return st;
    if ((st = copy_back(p, sig_sel, o.so.sig_sel, ne * p->n_sel * w.n, mem)) != RM_OK) return st;
    if (mem == RM_MEM_HOST) {
      RM_CUDA(cudaStreamSynchronize(p->stream), "rm_xsec");
      return check_err_word(p);
    }
    return RM_OK;
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_run(rm_plan_t h) {
  Nvtx range("rm_run");
  try {
    Plan* p = as_plan(h);
    if (!p) return fail(RM_ERR_ARG, "null plan");
    if (cudaSetDevice(p->device) != cudaSuccess) return fail(RM_ERR_CUDA, "cudaSetDevice failed");
    if (p->n_e == 0) {
      p->ran = true;
      return RM_OK;
    }
    if (!p->grp.ready) return fail(RM_ERR_STATE, "grouped work lists not prepared");
    if (p->prof) {
      rm_status_t st = enqueue_grouped(p, p->stream, true, nullptr, true);
      if (st != RM_OK) return st;
    } else {
      rm_status_t st = build_graph(p);
      if (st != RM_OK) return st;
      RM_CUDA(cudaGraphLaunch(p->grp.exec, p->stream), "graph launch");
      p->launches += p->grp.graph_kernels;
    }
    p->ran = true;
    return RM_OK;
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_photo(rm_plan_t h, int32_t wave, int64_t e0, int64_t e1, double* sig_pi, double* sig_pi_ch,
                     int32_t mem) {
  Nvtx range("rm_photo");
  try {
    Plan* p = as_plan(h);
    rm_status_t st = check_range(p, wave, e0, e1);
    if (st != RM_OK) return st;
    if (!valid_mem(mem)) return fail(RM_ERR_ARG, "bad memory space");
    const WaveDev& w = p->waves[wave];
    if (!w.dip) return fail(RM_ERR_ARG, "wave has no dipole vector");
    const int64_t ne = e1 - e0;
    Scratch s1, s2;
    RangeOut o;
    o.need_solve = true;
    o.so.do_xsec = true;
    if ((st = out_buf(p, sig_pi, ne, mem, s1, &o.so.pi_tot)) != RM_OK) return st;
    if ((st = out_buf(p, sig_pi_ch, ne * w.n, mem, s2, &o.so.pi_ch)) != RM_OK) return st;
    if ((st = run_range(p, wave, e0, e1, o)) != RM_OK) return st;
    if ((st = copy_back(p, sig_pi, o.so.pi_tot, ne, mem)) != RM_OK) return st;
    if ((st = copy_back(p, sig_pi_ch, o.so.pi_ch, ne * w.n, mem)) != RM_OK) return st;
    if (mem == RM_MEM_HOST) {
      RM_CUDA(cudaStreamSynchronize(p->stream), "rm_photo");
      return check_err_word(p);
    }
    return RM_OK;
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_results_photo(rm_plan_t h, int32_t wave, int64_t e0, int64_t e1, double* sig_pi,
                             double* sig_pi_ch, int32_t mem) {
  Nvtx range("rm_results_photo");
  try {
    Plan* p = as_plan(h);
    rm_status_t st = check_range(p, wave, e0, e1);
    if (st != RM_OK) return st;
    if (!valid_mem(mem)) return fail(RM_ERR_ARG, "bad memory space");
    if (!p->ran) return fail(RM_ERR_STATE, "rm_results_photo before rm_run");
    const WaveDev& w = p->waves[wave];
    if (!w.dip) return fail(RM_ERR_ARG, "wave has no dipole vector");
    const int64_t ne = e1 - e0;
    const cudaMemcpyKind k = kind_out(mem);
    if (ne > 0) {
      if (sig_pi) RM_CUDA(cudaMemcpyAsync(sig_pi, w.pi_tot + e0, sizeof(double) * ne, k, p->stream), "copy sig_pi");
      if (sig_pi_ch)
        RM_CUDA(cudaMemcpyAsync(sig_pi_ch, w.pi_ch + e0 * w.n, sizeof(double) * ne * w.n, k, p->stream),
                "copy sig_pi_ch");
    }
    if (mem == RM_MEM_HOST) {
      RM_CUDA(cudaStreamSynchronize(p->stream), "rm_results_photo");
      return check_err_word(p);
    }
    return RM_OK;
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_convolve(const double* energies, int64_t n_e, const double* sigma, int32_t n_series,
                        const double* weights, double fwhm, double* out, int32_t mem, void* cuda_stream) {
  Nvtx range("rm_convolve");
  try {
    if (n_e < 0 || (n_e > 0 && (!energies || !sigma || !out)) || !valid_mem(mem))
      return fail(RM_ERR_ARG, "bad arguments");
    if (n_series < 1 || n_series > convolve_max_series()) return fail(RM_ERR_ARG, "n_series must be in [1, 16]");
    if (!(fwhm >= 0.0) || !(fwhm < 1e300)) return fail(RM_ERR_ARG, "fwhm must be finite and >= 0");
    std::vector<double> f(n_series, 1.0 / n_series);
    if (weights)
      for (int s = 0; s < n_series; ++s) {
        if (!(weights[s] > -1e300 && weights[s] < 1e300)) return fail(RM_ERR_ARG, "weights must be finite");
        f[s] = weights[s];
      }
    if (n_e == 0) return RM_OK;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(cuda_stream);
    if (mem == RM_MEM_DEVICE) {
      RM_CUDA(launch_convolve(energies, n_e, sigma, n_series, f.data(), fwhm, out, s), "convolution kernel");
      return RM_OK;
    }
    for (int64_t e = 0; e + 1 < n_e; ++e)
      if (!(energies[e] <= energies[e + 1])) return fail(RM_ERR_ORDER, "energies are not sorted ascending");
    double *dE = nullptr, *dS = nullptr, *dO = nullptr;
    auto release = [&]() { dfree(dE); dfree(dS); dfree(dO); };
    if (cudaMalloc(&dE, sizeof(double) * n_e) != cudaSuccess || cudaMalloc(&dS, sizeof(double) * n_e * n_series) != cudaSuccess ||
        cudaMalloc(&dO, sizeof(double) * n_e) != cudaSuccess) {
      cudaGetLastError();
      release();
      return fail(RM_ERR_NOMEM, "device buffers for the convolution");
    }
    cudaError_t err = cudaMemcpyAsync(dE, energies, sizeof(double) * n_e, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess)
      err = cudaMemcpyAsync(dS, sigma, sizeof(double) * n_e * n_series, cudaMemcpyHostToDevice, s);
    if (err == cudaSuccess) err = launch_convolve(dE, n_e, dS, n_series, f.data(), fwhm, dO, s);
    if (err == cudaSuccess) err = cudaMemcpyAsync(out, dO, sizeof(double) * n_e, cudaMemcpyDeviceToHost, s);
    if (err == cudaSuccess) err = cudaStreamSynchronize(s);
    release();
    if (err != cudaSuccess) {
      cudaGetLastError();
      return fail(RM_ERR_CUDA, std::string("convolution: ") + cudaGetErrorString(err));
    }
    return RM_OK;
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_results(rm_plan_t h, int32_t wave, int64_t e0, int64_t e1, double* eigsum, double* sig_tot,
                       double* sig_sel, int32_t* n_open, uint8_t* flags, int32_t mem) {
  Nvtx range("rm_results");
  try {
    Plan* p = as_plan(h);
    rm_status_t st = check_range(p, wave, e0, e1);
    if (st != RM_OK) return st;
    if (!valid_mem(mem)) return fail(RM_ERR_ARG, "bad memory space");
    if (!p->ran) return fail(RM_ERR_STATE, "rm_results before rm_run");
    const WaveDev& w = p->waves[wave];
    const int64_t ne = e1 - e0;
    const cudaMemcpyKind k = kind_out(mem);
    cudaStream_t s = p->stream;
    if (ne > 0) {
      if (eigsum) RM_CUDA(cudaMemcpyAsync(eigsum, w.eta + e0, sizeof(double) * ne, k, s), "copy eta");
      if (sig_tot)
        RM_CUDA(cudaMemcpyAsync(sig_tot, w.sig_tot + e0 * p->n_sel, sizeof(double) * ne * p->n_sel, k, s), "copy sig_tot");
      if (sig_sel)
        RM_CUDA(cudaMemcpyAsync(sig_sel, w.sig_sel + e0 * p->n_sel * w.n, sizeof(double) * ne * p->n_sel * w.n, k, s),
                "copy sig_sel");
      if (n_open) RM_CUDA(cudaMemcpyAsync(n_open, w.n_open + e0, sizeof(int32_t) * ne, k, s), "copy n_open");
      if (flags) RM_CUDA(cudaMemcpyAsync(flags, w.flags + e0, ne, k, s), "copy flags");
    }
    if (mem == RM_MEM_HOST) {
      RM_CUDA(cudaStreamSynchronize(s), "rm_results");
      return check_err_word(p);
    }
    return RM_OK;
  } catch (...) {
    return fail(RM_ERR_NOMEM, "unexpected host exception");
  }
}

rm_status_t rm_sync(rm_plan_t h) {
  Nvtx range("rm_sync");
  Plan* p = as_plan(h);
  if (!p) return fail(RM_ERR_ARG, "null plan");
  RM_CUDA(cudaStreamSynchronize(p->stream), "rm_sync");
  return check_err_word(p);
}

rm_status_t rm_plan_info(rm_plan_t h, int32_t wave, int32_t* n_ch, int32_t* n_poles, int64_t* n_e,
                         int32_t* n_sel, int32_t* chunk, int64_t* workspace_bytes) {
  // chunk reports the energy-chunk size of rm_run (the grouped, graph-captured sweep)
  Plan* p = as_plan(h);
  if (!p) return fail(RM_ERR_ARG, "null plan");
  if (wave < 0 || wave >= p->n_waves) return fail(RM_ERR_ARG, "wave index out of range");
  if (n_ch) *n_ch = p->waves[wave].n;
  if (n_poles) *n_poles = p->waves[wave].N;
  if (n_e) *n_e = p->n_e;
  if (n_sel) *n_sel = p->n_sel;
  if (chunk) *chunk = p->grp.chunk;
  if (workspace_bytes) *workspace_bytes = p->workspace_bytes;
  return RM_OK;
}

rm_status_t rm_plan_cluster(rm_plan_t h, int32_t* cx, int32_t* cy) {
  Plan* p = as_plan(h);
  if (!p) return fail(RM_ERR_ARG, "null plan");
  if (cx) *cx = p->grp.tc_cx;
  if (cy) *cy = p->grp.tc_cy;
  return RM_OK;
}

rm_status_t rm_plan_mma_pair(rm_plan_t h, int32_t* on) {
  Plan* p = as_plan(h);
  if (!p || !on) return fail(RM_ERR_ARG, "null argument");
  *on = polesum_pair_runs(*p) ? 1 : 0;
  return RM_OK;
}

rm_status_t rm_plan_slices(rm_plan_t h, int32_t* products) {
  Plan* p = as_plan(h);
  if (!p || !products) return fail(RM_ERR_ARG, "null argument");
  *products = (p->prec == RM_PREC_SPLIT_BF16 || p->prec == RM_PREC_SPLIT_FP16) ? p->slices : 0;
  return RM_OK;
}

int64_t rm_plan_launches(rm_plan_t h) {
  Plan* p = as_plan(h);
  return p ? p->launches : -1;
}

rm_status_t rm_profile_enable(rm_plan_t h, int32_t on) {
  Plan* p = as_plan(h);
  if (!p) return fail(RM_ERR_ARG, "null plan");
  p->prof = on != 0;
  return RM_OK;
}

rm_status_t rm_profile_read(rm_plan_t h, int32_t kernel, double* total_ms, int64_t* launches) {
  Plan* p = as_plan(h);
  if (!p) return fail(RM_ERR_ARG, "null plan");
  if (kernel < 0 || kernel >= RM_KERNEL_COUNT) return fail(RM_ERR_ARG, "bad kernel id");
  RM_CUDA(cudaStreamSynchronize(p->stream), "rm_profile_read");
  prof_collect(p);
  if (total_ms) *total_ms = p->prof_ms[kernel];
  if (launches) *launches = p->prof_n[kernel];
  p->prof_ms[kernel] = 0.0;
  p->prof_n[kernel] = 0;
  return RM_OK;
}

rm_status_t rm_checked_report(int32_t* unit, int32_t* line) {
  if (unit) *unit = -1;
  if (line) *line = 0;
#ifdef RM_CHECKED
  int (*readers[])(bool) = {check_line_prep, check_line_polesum_tc, check_line_polesum_fp64,
                            check_line_polesum_fp32, check_line_asym, check_line_solve,
                            check_line_convolve, check_line_static};
  if (cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    return fail(RM_ERR_CUDA, "rm_checked_report: device synchronisation failed");
  }
  bool found = false;
  for (int u = 0; u < (int)(sizeof(readers) / sizeof(readers[0])); ++u) {
    const int v = readers[u](true);
    if (v < 0) return fail(RM_ERR_CUDA, "rm_checked_report: cannot read a check word");
    if (v > 0 && !found) {
      found = true;
      if (unit) *unit = u;
      if (line) *line = v;
    }
  }
  return RM_OK;
#else
  return fail(RM_ERR_STATE, "library built without RM_CHECKED");
#endif
}

rm_status_t rm_plan_destroy(rm_plan_t h) {
  Nvtx range("rm_plan_destroy");
  Plan* p = as_plan(h);
  if (!p) return RM_OK;
  cudaSetDevice(p->device);
  cudaStreamSynchronize(p->stream);
  free_plan(p);
  return RM_OK;
}

}  // extern "C"
