// Launchers of the compensated-operator apply (kernels in fft_kernels.cuh,
// instantiated per precision in fft_f32.cu / fft_f64.cu): vector chunking
// sized to L2, the context-owned scratch, the file-scope scratch of
// pcx_apply_noalloc, and the preconditioner launch.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>
#include <vector>

#include "pcx_internal.h"

// Scratch of pcx_apply_noalloc: a file-scope device array, present on every
// GPU that loads the library until the process exits.  Host code must not
// use this name as an address: the device address comes from
// cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) unsigned char g_apply_noalloc_scratch[PCX_NOALLOC_SCRATCH_BYTES];

namespace pcx {

template <typename T>
cudaError_t run_apply_t(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int chunk, void* sbuf,
                        const KParams* kps, int vec_per_k, cudaStream_t st, bool t0);
template <typename T>
cudaError_t run_precond_t(const pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, cudaStream_t s);
template <typename T>
cudaError_t run_div_norms_t(const pcx_ctx* c, const KParams& kp, const void* X, int nvec, double* out, cudaStream_t s);
template <typename T>
cudaError_t run_fft_t(const pcx_ctx* c, const void* X, void* Y, int nvec, int dir, cudaStream_t st);
template <typename T>
cudaError_t run_curl_h_t(const pcx_ctx* c, const KParams& kp, const void* X, void* U, int nvec, int pow, cudaStream_t s);
template <typename T>
cudaError_t run_curl_add_t(const pcx_ctx* c, const KParams& kp, const void* Wm, const void* R, void* Y, int nvec,
                           double scale_, int accumulate, cudaStream_t s);
template <typename T>
cudaError_t run_eps_cells_t(const pcx_ctx* c, const void* E, const void* Add, void* Mo, int nvec, double scale_,
                            cudaStream_t s);
extern template cudaError_t run_apply_t<float>(const pcx_ctx*, const KParams&, const void*, void*, int, int, void*,
                                               const KParams*, int, cudaStream_t, bool);
extern template cudaError_t run_apply_t<double>(const pcx_ctx*, const KParams&, const void*, void*, int, int, void*,
                                                const KParams*, int, cudaStream_t, bool);

namespace {
template <typename T>
cudaError_t dispatch_apply(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int chunk,
                           void* sbuf, cudaStream_t st, const KParams* kps = nullptr, int vec_per_k = 1) {
  return run_apply_t<T>(c, kp, X, Y, nvec, chunk, sbuf, kps, vec_per_k, st, false);
}
}  // namespace

int apply_chunk(const pcx_ctx* c, int precision) {
  if (c->apply_chunk > 0) return c->apply_chunk;
  const size_t vbytes = (size_t)3 * c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8);
  const size_t l2 = c->l2_bytes ? c->l2_bytes : ((size_t)126 << 20);
  const size_t k = (l2 / 2) / vbytes;
  return (int)(k < 1 ? 1 : (k > 64 ? 64 : k));
}

cudaError_t raise_dyn_smem(const void* func, size_t bytes) {
  struct Entry {
    const void* f;
    int dev;
    size_t bytes;
  };
  static std::mutex mu;
  static std::vector<Entry> seen;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  for (Entry& en : seen)
    if (en.f == func && en.dev == dev) {
      if (bytes <= en.bytes) return cudaSuccess;
      e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
      if (e == cudaSuccess) en.bytes = bytes;
      return e;
    }
  e = cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) e = cudaFuncSetAttribute(func, cudaFuncAttributePreferredSharedMemoryCarveout,
                                                 cudaSharedmemCarveoutMaxShared);
  if (e == cudaSuccess) seen.push_back(Entry{func, dev, bytes});
  return e;
}

int effective_apply_path(const pcx_ctx* c, int precision) {
  if (c->m_kind == PCX_M_CROSSDOF) return 7;
  const bool three = precision == PCX_FP32 && (c->n == 32 || c->n == 64 || c->n == 128);
  return three && c->apply_path != PCX_APPLY_FIVE_PASS ? PCX_APPLY_THREE_PASS : PCX_APPLY_FIVE_PASS;
}

// gamma kappa.x per vector of a chunk, and for M_CrossDoF the real-space
// field of the stencil pass (3 N^3) after it
size_t apply_scratch_bytes(const pcx_ctx* c, int precision, int nvec) {
  const int chunk = apply_chunk(c, precision);
  const int nv = nvec < chunk ? nvec : chunk;
  const size_t per = (size_t)c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8);
  return (size_t)nv * per * (c->m_kind == PCX_M_CROSSDOF ? 4 : 1);
}

cudaError_t launch_apply_scratch(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int precision,
                                 void* scratch, cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const int chunk = apply_chunk(c, precision);
  return precision == PCX_FP64 ? dispatch_apply<double>(c, kp, X, Y, nvec, chunk, scratch, s)
                               : dispatch_apply<float>(c, kp, X, Y, nvec, chunk, scratch, s);
}

// Device address of g_apply_noalloc_scratch on the current device, looked up
// once per device (the first pcx_apply_noalloc call on that device).
static cudaError_t noalloc_scratch(void** out) {
  static std::mutex mu;
  static void* ptr[256] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_apply_noalloc_scratch);
    if (e != cudaSuccess) return e;
    ptr[dev] = p;
  }
  *out = ptr[dev];
  return cudaSuccess;
}

cudaError_t launch_apply_noalloc(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int precision,
                                 cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t per_vec =
      (size_t)c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8) * (c->m_kind == PCX_M_CROSSDOF ? 4 : 1);
  if (per_vec > (size_t)PCX_NOALLOC_SCRATCH_BYTES) return cudaErrorInvalidValue;
  void* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return e;
  int chunk = apply_chunk(c, precision);
  const int fit = (int)((size_t)PCX_NOALLOC_SCRATCH_BYTES / per_vec);
  if (chunk > fit) chunk = fit;
  return precision == PCX_FP64 ? dispatch_apply<double>(c, kp, X, Y, nvec, chunk, scratch, s)
                               : dispatch_apply<float>(c, kp, X, Y, nvec, chunk, scratch, s);
}

namespace {

cudaError_t ensure_scratch(pcx_ctx* c, int precision, int nvec) {
  const size_t need = apply_scratch_bytes(c, precision, nvec);
  if (need > c->scratch_bytes) {
    // the previous scratch may still be in use by work queued on another stream
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    free_apply_graphs(c);   // graphs hold the old scratch address
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    e = cudaMalloc(&c->scratch, need);
    if (e != cudaSuccess) return e;
    c->scratch_bytes = need;
  }
  return cudaSuccess;
}

// One captured apply chain.  A key runs eagerly the first time it is seen
// (kernel attributes and module loading happen outside any capture) and is
// captured on its second use; later uses replay the graph.
struct GraphEntry {
  const void* X;
  void* Y;
  int nvec, precision, chunk;
  void* scratch;
  cudaStream_t stream;
  KParams kp;
  int seen = 0;
  cudaGraphExec_t exec = nullptr;
  bool same(const GraphEntry& o) const {
    return X == o.X && Y == o.Y && nvec == o.nvec && precision == o.precision && chunk == o.chunk &&
           scratch == o.scratch && stream == o.stream && std::memcmp(&kp, &o.kp, sizeof(KParams)) == 0;
  }
};
struct GraphCache {
  std::vector<GraphEntry> entries;
};
constexpr size_t kMaxGraphs = 64;

bool capturable(cudaStream_t s) { return s != nullptr && s != cudaStreamLegacy && s != cudaStreamPerThread; }

}  // namespace

void free_apply_graphs(pcx_ctx* c) {
  if (!c->graphs) return;
  auto* gc = static_cast<GraphCache*>(c->graphs);
  for (auto& e : gc->entries)
    if (e.exec) cudaGraphExecDestroy(e.exec);
  delete gc;
  c->graphs = nullptr;
}

cudaError_t launch_t0(pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, int precision,
                      cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  cudaError_t e = ensure_scratch(c, precision, nvec);
  if (e != cudaSuccess) return e;
  const int chunk = apply_chunk(c, precision);
  return precision == PCX_FP64
             ? run_apply_t<double>(c, kp, R, W, nvec, chunk, c->scratch, nullptr, 1, s, true)
             : run_apply_t<float>(c, kp, R, W, nvec, chunk, c->scratch, nullptr, 1, s, true);
}

cudaError_t launch_t0_scratch(const pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, int precision,
                              void* scratch, cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const int chunk = apply_chunk(c, precision);
  return precision == PCX_FP64 ? run_apply_t<double>(c, kp, R, W, nvec, chunk, scratch, nullptr, 1, s, true)
                               : run_apply_t<float>(c, kp, R, W, nvec, chunk, scratch, nullptr, 1, s, true);
}

cudaError_t launch_apply(pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int precision,
                         cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  cudaError_t e = ensure_scratch(c, precision, nvec);
  if (e != cudaSuccess) return e;
  if (!c->use_graphs || !capturable(s)) return launch_apply_scratch(c, kp, X, Y, nvec, precision, c->scratch, s);
  if (!c->graphs) c->graphs = new GraphCache;
  auto* gc = static_cast<GraphCache*>(c->graphs);
  GraphEntry key;
  std::memset(&key, 0, sizeof(key));
  key.X = X;
  key.Y = Y;
  key.nvec = nvec;
  key.precision = precision;
  key.chunk = apply_chunk(c, precision);
  key.scratch = c->scratch;
  key.stream = s;
  key.kp = kp;
  GraphEntry* ent = nullptr;
  for (auto& g : gc->entries)
    if (g.same(key)) ent = &g;
  if (!ent) {
    if (gc->entries.size() >= kMaxGraphs) {
      if (gc->entries.front().exec) cudaGraphExecDestroy(gc->entries.front().exec);
      gc->entries.erase(gc->entries.begin());
    }
    gc->entries.push_back(key);
    ent = &gc->entries.back();
  }
  if (ent->exec) return cudaGraphLaunch(ent->exec, s);
  if (ent->seen++ == 0) return launch_apply_scratch(c, kp, X, Y, nvec, precision, c->scratch, s);
  // capture the launch chain; on any capture failure run eagerly instead
  cudaGraph_t graph = nullptr;
  e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t el = launch_apply_scratch(c, kp, X, Y, nvec, precision, c->scratch, s);
    cudaError_t ec = cudaStreamEndCapture(s, &graph);
    if (el == cudaSuccess && ec == cudaSuccess && graph)
      e = cudaGraphInstantiate(&ent->exec, graph, 0);
    else
      e = el != cudaSuccess ? el : (ec != cudaSuccess ? ec : cudaErrorUnknown);
    if (graph) cudaGraphDestroy(graph);
  }
  if (e != cudaSuccess || !ent->exec) {
    cudaGetLastError();   // clear the capture error; this key stays eager
    ent->exec = nullptr;
    ent->seen = -1000000;
    return launch_apply_scratch(c, kp, X, Y, nvec, precision, c->scratch, s);
  }
  return cudaGraphLaunch(ent->exec, s);
}

cudaError_t launch_apply_kbatch(pcx_ctx* c, const KParams* kps_host, int nk, int vec_per_k, const void* X, void* Y,
                                int precision, cudaStream_t s) {
  const int nvec = nk * vec_per_k;
  if (nvec == 0) return cudaSuccess;
  const size_t bytes = sizeof(KParams) * (size_t)nk;
  cudaError_t e;
  if (bytes > c->ktab_bytes) {
    if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
    if (c->ktab) cudaFree(c->ktab);
    c->ktab = nullptr;
    c->ktab_bytes = 0;
    if ((e = cudaMalloc(&c->ktab, bytes)) != cudaSuccess) return e;
    c->ktab_bytes = bytes;
  }
  // pageable source: the call returns once the table is staged
  if ((e = cudaMemcpyAsync(c->ktab, kps_host, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess) return e;
  if ((e = ensure_scratch(c, precision, nvec)) != cudaSuccess) return e;
  const int chunk = apply_chunk(c, precision);
  const KParams* kt = static_cast<const KParams*>(c->ktab);
  return precision == PCX_FP64 ? dispatch_apply<double>(c, kps_host[0], X, Y, nvec, chunk, c->scratch, s, kt, vec_per_k)
                               : dispatch_apply<float>(c, kps_host[0], X, Y, nvec, chunk, c->scratch, s, kt, vec_per_k);
}

cudaError_t launch_precond(const pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, int precision,
                           cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  return precision == PCX_FP64 ? run_precond_t<double>(c, kp, R, W, nvec, s) : run_precond_t<float>(c, kp, R, W, nvec, s);
}

cudaError_t launch_curl_h(const pcx_ctx* c, const KParams& kp, const void* X, void* U, int nvec, int pow, int precision,
                          cudaStream_t s) {
  return precision == PCX_FP64 ? run_curl_h_t<double>(c, kp, X, U, nvec, pow, s)
                               : run_curl_h_t<float>(c, kp, X, U, nvec, pow, s);
}

cudaError_t launch_curl_add(const pcx_ctx* c, const KParams& kp, const void* Wm, const void* R, void* Y, int nvec,
                            double scale, int accumulate, int precision, cudaStream_t s) {
  return precision == PCX_FP64 ? run_curl_add_t<double>(c, kp, Wm, R, Y, nvec, scale, accumulate, s)
                               : run_curl_add_t<float>(c, kp, Wm, R, Y, nvec, scale, accumulate, s);
}

cudaError_t launch_eps_cells(const pcx_ctx* c, const void* E, const void* Add, void* Mo, int nvec, double scale,
                             int precision, cudaStream_t s) {
  return precision == PCX_FP64 ? run_eps_cells_t<double>(c, E, Add, Mo, nvec, scale, s)
                               : run_eps_cells_t<float>(c, E, Add, Mo, nvec, scale, s);
}

cudaError_t launch_fft(const pcx_ctx* c, const void* X, void* Y, int nvec, int dir, int precision, cudaStream_t s) {
  return precision == PCX_FP64 ? run_fft_t<double>(c, X, Y, nvec, dir, s) : run_fft_t<float>(c, X, Y, nvec, dir, s);
}

cudaError_t launch_div_norms(const pcx_ctx* c, const KParams& kp, const void* X, int nvec, int precision, double* out,
                             cudaStream_t s) {
  return precision == PCX_FP64 ? run_div_norms_t<double>(c, kp, X, nvec, out, s)
                               : run_div_norms_t<float>(c, kp, X, nvec, out, s);
}

}  // namespace pcx
