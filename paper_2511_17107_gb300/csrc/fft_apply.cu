// Launchers of the compensated-operator apply (kernels in fft_kernels.cuh,
// instantiated per precision in fft_f32.cu / fft_f64.cu): vector chunking
// sized to L2, the context-owned scratch, the file-scope scratch of
// pcx_apply_noalloc, and the preconditioner launch.
#include <cuda_runtime.h>

#include <mutex>

#include "pcx_internal.h"

// Scratch of pcx_apply_noalloc: a file-scope device array, present on every
// GPU that loads the library until the process exits.  Host code must not
// use this name as an address: the device address comes from
// cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) unsigned char g_apply_noalloc_scratch[PCX_NOALLOC_SCRATCH_BYTES];

namespace pcx {

template <typename T>
cudaError_t run_apply_t(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int chunk, void* sbuf,
                        cudaStream_t st);
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
                                               cudaStream_t);
extern template cudaError_t run_apply_t<double>(const pcx_ctx*, const KParams&, const void*, void*, int, int, void*,
                                                cudaStream_t);

namespace {
template <typename T>
cudaError_t dispatch_apply(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int chunk,
                           void* sbuf, cudaStream_t st) {
  return run_apply_t<T>(c, kp, X, Y, nvec, chunk, sbuf, st);
}
}  // namespace

int apply_chunk(const pcx_ctx* c, int precision) {
  if (c->apply_chunk > 0) return c->apply_chunk;
  const size_t vbytes = (size_t)3 * c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8);
  const size_t l2 = c->l2_bytes ? c->l2_bytes : ((size_t)126 << 20);
  const size_t k = (l2 / 2) / vbytes;
  return (int)(k < 1 ? 1 : (k > 64 ? 64 : k));
}

size_t apply_scratch_bytes(const pcx_ctx* c, int precision, int nvec) {
  const int chunk = apply_chunk(c, precision);
  const int nv = nvec < chunk ? nvec : chunk;
  return (size_t)nv * c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8);
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
  const size_t per_vec = (size_t)c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8);
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

cudaError_t launch_apply(pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int precision,
                         cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t need = apply_scratch_bytes(c, precision, nvec);
  if (need > c->scratch_bytes) {
    // the previous scratch may still be in use by work queued on another stream
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    e = cudaMalloc(&c->scratch, need);
    if (e != cudaSuccess) return e;
    c->scratch_bytes = need;
  }
  return launch_apply_scratch(c, kp, X, Y, nvec, precision, c->scratch, s);
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
