// Host orchestration of the learned preconditioner correction (cnn.cu):
// gates, forward and backward passes of the gated convolution net, the
// curl-sandwich approximate inverse T0 and the corrected preconditioner
// T(r) = T0 r + K_A F3_3^H g(F3_3 K_A^H r / |k|^2) / |k|^2, the training
// pairs (r, e = Op^{-1} r) and a block preconditioned conjugate gradient
// solver for Op e = r (Op Hermitian positive definite for k != 0; at k = 0
// the p = 0 mode is excluded by K_P^{-1}, Prop. 2.5).
//
// The paper has no learned component.  Every device step is a kernel of
// this library; the host only sequences launches and small reductions.
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "cnn.h"
#include "pcx_internal.h"

namespace pcx {

namespace {

// context-owned workspace, grown on demand (the previous one may still be in
// use by queued work, so growth synchronises the device)
cudaError_t ws_get(pcx_ctx* c, size_t bytes, char** out) {
  if (bytes > c->cnn_ws_bytes) {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    if (c->cnn_ws) cudaFree(c->cnn_ws);
    c->cnn_ws = nullptr;
    c->cnn_ws_bytes = 0;
    if ((e = cudaMalloc(&c->cnn_ws, bytes)) != cudaSuccess) return e;
    c->cnn_ws_bytes = bytes;
  }
  *out = static_cast<char*>(c->cnn_ws);
  return cudaSuccess;
}

size_t align_up(size_t b) { return (b + 255) & ~(size_t)255; }

struct Carve {
  char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = reinterpret_cast<T*>(base + off);
    off += align_up(count * sizeof(T));
    return p;
  }
};

constexpr int C = cnn::HIDDEN;

}  // namespace

#define CKE(x)                                 \
  do {                                         \
    cudaError_t _e = (x);                      \
    if (_e != cudaSuccess) return _e;          \
  } while (0)

cudaError_t cnn_gates(pcx_ctx* c, const float* params, float* gates, cudaStream_t s) {
  const size_t n3 = (size_t)c->n * c->n * c->n;
  char* ws;
  CKE(ws_get(c, align_up(9 * n3 * sizeof(float)), &ws));
  float* f = reinterpret_cast<float*>(ws);
  CKE(cnn::features(c, f, s));
  const cnn::View fv = cnn::shared_view(f, n3), none{};
  CKE(cnn::conv_fwd(9, C, cnn::MODE_SIGMOID, fv, cnn::dense_view(gates, C, n3), params + cnn::OFF_V1,
                    params + cnn::OFF_C1, none, none, 1, c->n, 1.f, s));
  CKE(cnn::conv_fwd(9, C, cnn::MODE_SIGMOID, fv, cnn::dense_view(gates + C * n3, C, n3), params + cnn::OFF_V2,
                    params + cnn::OFF_C2, none, none, 1, c->n, 1.f, s));
  return cudaSuccess;
}

// Y = g(Re U) + i g(Im U) for nv complex64 fields; h1, h2: 2 nv C N^3 floats each
static cudaError_t forward_chunk(pcx_ctx* c, const float* params, const float* gates, const void* U, void* Y, int nv,
                                 float* h1, float* h2, float out_scale, cudaStream_t s) {
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const int nb = 2 * nv;
  const cnn::View none{};
  CKE(cnn::conv_fwd(3, C, cnn::MODE_GATE, cnn::complex_view(const_cast<void*>(U), n3), cnn::dense_view(h1, C, n3),
                    params + cnn::OFF_W1, nullptr, cnn::shared_view(const_cast<float*>(gates), n3), none, nb, c->n,
                    1.f, s));
  CKE(cnn::conv_fwd(C, C, cnn::MODE_GATE, cnn::dense_view(h1, C, n3), cnn::dense_view(h2, C, n3),
                    params + cnn::OFF_W2, nullptr, cnn::shared_view(const_cast<float*>(gates) + C * n3, n3), none, nb,
                    c->n, 1.f, s));
  CKE(cnn::conv_fwd(C, 3, cnn::MODE_PLAIN, cnn::dense_view(h2, C, n3), cnn::complex_view(Y, n3), params + cnn::OFF_W3,
                    nullptr, none, none, nb, c->n, out_scale, s));
  return cudaSuccess;
}

// vectors per chunk so that the two hidden activations stay within ~2 GB
static int forward_chunk_size(const pcx_ctx* c, int nvec) {
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const size_t per = 2 * 2 * (size_t)C * n3 * sizeof(float);
  size_t k = ((size_t)2 << 30) / per;
  if (k < 1) k = 1;
  return (int)(k < (size_t)nvec ? k : (size_t)nvec);
}

cudaError_t cnn_forward(pcx_ctx* c, const float* params, const float* gates, const void* U, void* Y, int nvec,
                        cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const int chunk = forward_chunk_size(c, nvec);
  const size_t hb = align_up(2 * (size_t)chunk * C * n3 * sizeof(float));
  char* ws;
  CKE(ws_get(c, 2 * hb, &ws));
  float* h1 = reinterpret_cast<float*>(ws);
  float* h2 = reinterpret_cast<float*>(ws + hb);
  const size_t vlen = 3 * n3;
  for (int v0 = 0; v0 < nvec; v0 += chunk) {
    const int nv = nvec - v0 < chunk ? nvec - v0 : chunk;
    CKE(forward_chunk(c, params, gates, static_cast<const float2*>(U) + (size_t)v0 * vlen,
                      static_cast<float2*>(Y) + (size_t)v0 * vlen, nv, h1, h2, 1.f, s));
  }
  return cudaSuccess;
}

cudaError_t cnn_grad(pcx_ctx* c, const float* params, const void* U, const void* T, const double* wv_host, int nvec,
                     float* grad, int accumulate, double* loss_host, cudaStream_t s) {
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const int nb = 2 * nvec, n = c->n;
  const size_t act = (size_t)nb * C * n3;
  size_t need = 0;
  need += align_up(9 * n3 * 4) + align_up(2 * C * n3 * 4);           // f, gates
  need += 6 * align_up(act * 4);                                     // a1 h1 a2 h2 dh2 dh1
  need += 2 * align_up((size_t)nvec * 6 * n3 * 4);                   // Y, dY
  need += 2 * align_up(C * n3 * 4);                                  // dz1, dz2
  need += align_up(cnn::wgrad_scratch_floats(9, C) * 4);             // the largest wgrad scratch
  need += 2 * align_up(C * C * 27 * 4) + align_up(nvec * 8 + 8);     // adjoint weights, w, loss
  char* ws;
  CKE(ws_get(c, need, &ws));
  Carve cv{ws};
  float* f = cv.take<float>(9 * n3);
  float* g = cv.take<float>(2 * C * n3);
  float* a1 = cv.take<float>(act);
  float* h1 = cv.take<float>(act);
  float* a2 = cv.take<float>(act);
  float* h2 = cv.take<float>(act);
  float* dh2 = cv.take<float>(act);
  float* dh1 = cv.take<float>(act);
  float* Y = cv.take<float>((size_t)nvec * 6 * n3);
  float* dY = cv.take<float>((size_t)nvec * 6 * n3);
  float* dz1 = cv.take<float>(C * n3);
  float* dz2 = cv.take<float>(C * n3);
  float* scr = cv.take<float>(cnn::wgrad_scratch_floats(9, C));
  float* wt3 = cv.take<float>(C * C * 27);
  float* wt2 = cv.take<float>(C * C * 27);
  double* wdev = cv.take<double>(nvec + 1);
  double* ldev = wdev + nvec;
  const cnn::View none{};
  // gates and forward pass with the pre-gate activations kept
  CKE(cnn::features(c, f, s));
  const cnn::View fv = cnn::shared_view(f, n3);
  CKE(cnn::conv_fwd(9, C, cnn::MODE_SIGMOID, fv, cnn::dense_view(g, C, n3), params + cnn::OFF_V1, params + cnn::OFF_C1,
                    none, none, 1, n, 1.f, s));
  CKE(cnn::conv_fwd(9, C, cnn::MODE_SIGMOID, fv, cnn::dense_view(g + C * n3, C, n3), params + cnn::OFF_V2,
                    params + cnn::OFF_C2, none, none, 1, n, 1.f, s));
  const cnn::View Uv = cnn::complex_view(const_cast<void*>(U), n3);
  const cnn::View A1 = cnn::dense_view(a1, C, n3), H1 = cnn::dense_view(h1, C, n3);
  const cnn::View A2 = cnn::dense_view(a2, C, n3), H2 = cnn::dense_view(h2, C, n3);
  const cnn::View DH1 = cnn::dense_view(dh1, C, n3), DH2 = cnn::dense_view(dh2, C, n3);
  CKE(cnn::conv_fwd(3, C, cnn::MODE_GATE, Uv, H1, params + cnn::OFF_W1, nullptr, cnn::shared_view(g, n3), A1, nb, n, 1.f,
                    s));
  CKE(cnn::conv_fwd(C, C, cnn::MODE_GATE, H1, H2, params + cnn::OFF_W2, nullptr, cnn::shared_view(g + C * n3, n3), A2,
                    nb, n, 1.f, s));
  CKE(cnn::conv_fwd(C, 3, cnn::MODE_PLAIN, H2, cnn::complex_view(Y, n3), params + cnn::OFF_W3, nullptr, none, none, nb,
                    n, 1.f, s));
  // loss and dY
  CKE(cudaMemcpyAsync(wdev, wv_host, sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
  CKE(cudaMemsetAsync(ldev, 0, sizeof(double), s));
  CKE(cnn::loss_grad(Y, T, wdev, nvec, n3, dY, ldev, s));
  const cnn::View DY = cnn::complex_view(dY, n3);
  // layer 3
  CKE(cnn::conv_wgrad(C, 3, DY, H2, nb, n, grad + cnn::OFF_W3, accumulate, scr, s));
  CKE(cnn::adjoint_weights(params + cnn::OFF_W3, 3, C, wt3, s));
  CKE(cnn::conv_fwd(3, C, cnn::MODE_PLAIN, DY, DH2, wt3, nullptr, none, none, nb, n, 1.f, s));
  // gate 2 and layer 2
  CKE(cnn::gate_backward(DH2, A2, g + C * n3, nb, C, n3, dz2, s));
  CKE(cnn::conv_wgrad(C, C, DH2, H1, nb, n, grad + cnn::OFF_W2, accumulate, scr, s));
  CKE(cnn::adjoint_weights(params + cnn::OFF_W2, C, C, wt2, s));
  CKE(cnn::conv_fwd(C, C, cnn::MODE_PLAIN, DH2, DH1, wt2, nullptr, none, none, nb, n, 1.f, s));
  // gate 1 and layer 1
  CKE(cnn::gate_backward(DH1, A1, g, nb, C, n3, dz1, s));
  CKE(cnn::conv_wgrad(3, C, DH1, Uv, nb, n, grad + cnn::OFF_W1, accumulate, scr, s));
  // gate parameters
  CKE(cnn::conv_wgrad(9, C, cnn::dense_view(dz1, C, n3), fv, 1, n, grad + cnn::OFF_V1, accumulate, scr, s));
  CKE(cnn::bias_grad(dz1, C, n3, grad + cnn::OFF_C1, accumulate, s));
  CKE(cnn::conv_wgrad(9, C, cnn::dense_view(dz2, C, n3), fv, 1, n, grad + cnn::OFF_V2, accumulate, scr, s));
  CKE(cnn::bias_grad(dz2, C, n3, grad + cnn::OFF_C2, accumulate, s));
  if (loss_host) {
    CKE(cudaMemcpyAsync(loss_host, ldev, sizeof(double), cudaMemcpyDeviceToHost, s));
    CKE(cudaStreamSynchronize(s));
  }
  return cudaSuccess;
}

// T0 R = K_A F3^H eps F3 (K_A^H R / |k|^2) / |k|^2 + K_B R / (gamma |k|^4)
// on the five fused passes of the apply (fft_kernels.cuh, OP_*_T0).  W may
// alias R.
cudaError_t sandwich_precond(pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, int precision,
                             cudaStream_t s) {
  return launch_t0(c, kp, R, W, nvec, precision, s);
}

// T R = T0 R + K_A F3^H g(e) / |k|^2 with e = F3 (K_A^H R / |k|^2): the net's
// output joins eps e in real space before the forward transform.
cudaError_t cnn_precond(pcx_ctx* c, const KParams& kp, const float* params, const float* gates, const void* R, void* W,
                        int nvec, cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const int chunk = forward_chunk_size(c, nvec);
  const size_t hb = align_up(2 * (size_t)chunk * C * n3 * sizeof(float));
  const size_t tb = align_up((size_t)chunk * 3 * n3 * sizeof(float2));
  char* ws;
  CKE(ws_get(c, 2 * hb + 2 * tb, &ws));
  float* h1 = reinterpret_cast<float*>(ws);
  float* h2 = reinterpret_cast<float*>(ws + hb);
  float2* e = reinterpret_cast<float2*>(ws + 2 * hb);
  float2* y = reinterpret_cast<float2*>(ws + 2 * hb + tb);
  const size_t vlen = 3 * n3;
  const double inv_n3 = 1.0 / (double)n3;
  for (int v0 = 0; v0 < nvec; v0 += chunk) {
    const int nv = nvec - v0 < chunk ? nvec - v0 : chunk;
    const float2* r = static_cast<const float2*>(R) + (size_t)v0 * vlen;
    float2* w = static_cast<float2*>(W) + (size_t)v0 * vlen;
    CKE(launch_curl_h(c, kp, r, e, nv, 1, PCX_FP32, s));
    CKE(launch_fft(c, e, e, nv, +1, PCX_FP32, s));
    CKE(forward_chunk(c, params, gates, e, y, nv, h1, h2, 1.f, s));
    CKE(launch_eps_cells(c, e, y, e, nv, inv_n3, PCX_FP32, s));
    CKE(launch_fft(c, e, e, nv, -1, PCX_FP32, s));
    CKE(launch_curl_add(c, kp, e, r, w, nv, 1.0, 0, PCX_FP32, s));
  }
  return cudaSuccess;
}

// U = F3 (K_A^H R / |k|^2), T = F3 K_A^H (E - T0 R) (unitary F3), and
// enorm2 = ||K_A^H E||^2 per vector.
cudaError_t cnn_pairs(pcx_ctx* c, const KParams& kp, const void* R, const void* E, void* U, void* T, double* enorm2_host,
                      int nvec, cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const size_t nf = (size_t)nvec * 6 * n3;
  const float sc = (float)(1.0 / std::pow((double)n3, 0.5));
  CKE(sandwich_precond(c, kp, R, T, nvec, PCX_FP32, s));
  CKE(cnn::lincomb(static_cast<const float*>(E), 1.f, static_cast<const float*>(T), -1.f, static_cast<float*>(T), nf,
                   s));
  CKE(launch_curl_h(c, kp, T, T, nvec, 0, PCX_FP32, s));
  CKE(launch_fft(c, T, T, nvec, +1, PCX_FP32, s));
  CKE(cnn::lincomb(static_cast<const float*>(T), sc, nullptr, 0.f, static_cast<float*>(T), nf, s));
  if (enorm2_host) {
    CKE(launch_curl_h(c, kp, E, U, nvec, 0, PCX_FP32, s));
    char* ws;
    CKE(ws_get(c, align_up(2 * nvec * sizeof(double)), &ws));
    double* d = reinterpret_cast<double*>(ws);
    CKE(cnn::col_dots(U, U, nvec, 3 * n3, d, s));
    std::vector<double> h(2 * (size_t)nvec);
    CKE(cudaMemcpyAsync(h.data(), d, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, s));
    CKE(cudaStreamSynchronize(s));
    for (int v = 0; v < nvec; ++v) enorm2_host[v] = h[2 * v];
  }
  CKE(launch_curl_h(c, kp, R, U, nvec, 1, PCX_FP32, s));
  CKE(launch_fft(c, U, U, nvec, +1, PCX_FP32, s));
  CKE(cnn::lincomb(static_cast<const float*>(U), sc, nullptr, 0.f, static_cast<float*>(U), nf, s));
  return cudaSuccess;
}

// Block PCG for Op E = R (complex64 storage, FP64 scalars), one independent
// recursion per column, preconditioned by K_P^{-1}; stops when every
// ||R - Op E|| / ||R|| <= tol or after maxit iterations.
cudaError_t cg_solve(pcx_ctx* c, const KParams& kp, const void* R, void* E, int nvec, double tol, int maxit,
                     int* iters, double* relres, cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t n3 = (size_t)c->n * c->n * c->n, len = 3 * n3;
  const size_t vb = align_up((size_t)nvec * len * sizeof(float2));
  char* ws;
  CKE(ws_get(c, 4 * vb + align_up(6 * (size_t)nvec * sizeof(double)), &ws));
  float2* res = reinterpret_cast<float2*>(ws);
  float2* z = reinterpret_cast<float2*>(ws + vb);
  float2* p = reinterpret_cast<float2*>(ws + 2 * vb);
  float2* q = reinterpret_cast<float2*>(ws + 3 * vb);
  double* dots = reinterpret_cast<double*>(ws + 4 * vb);   // 2 nvec
  double* coef = dots + 2 * nvec;                          // alpha[nvec], beta[nvec]
  std::vector<double> h(2 * (size_t)nvec), r0(nvec), rz(nvec), al(nvec), be(nvec);
  auto dots_host = [&](const void* a, const void* b) -> cudaError_t {
    CKE(cnn::col_dots(a, b, nvec, len, dots, s));
    CKE(cudaMemcpyAsync(h.data(), dots, sizeof(double) * 2 * nvec, cudaMemcpyDeviceToHost, s));
    return cudaStreamSynchronize(s);
  };
  auto axpby = [&](const std::vector<double>& a, const void* x, const std::vector<double>& b, void* y) -> cudaError_t {
    CKE(cudaMemcpyAsync(coef, a.data(), sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
    CKE(cudaMemcpyAsync(coef + nvec, b.data(), sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
    CKE(cnn::col_axpby(coef, x, coef + nvec, y, nvec, len, s));
    return cudaStreamSynchronize(s);   // the coefficients are reused next call
  };
  CKE(cudaMemsetAsync(E, 0, (size_t)nvec * len * sizeof(float2), s));
  CKE(cudaMemcpyAsync(res, R, (size_t)nvec * len * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  CKE(dots_host(R, R));
  for (int v = 0; v < nvec; ++v) r0[v] = std::sqrt(h[2 * v]);
  CKE(launch_precond(c, kp, res, z, nvec, PCX_FP32, s));
  CKE(cudaMemcpyAsync(p, z, (size_t)nvec * len * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  CKE(dots_host(res, z));
  for (int v = 0; v < nvec; ++v) rz[v] = h[2 * v];
  std::vector<double> ones(nvec, 1.0), rel(nvec, 1.0);
  int it = 0;
  for (; it < maxit; ++it) {
    CKE(launch_apply(c, kp, p, q, nvec, PCX_FP32, s));
    CKE(dots_host(p, q));
    for (int v = 0; v < nvec; ++v) {
      const double pq = h[2 * v];
      al[v] = (pq > 0 && rz[v] > 0 && rel[v] > tol) ? rz[v] / pq : 0.0;
    }
    CKE(axpby(al, p, ones, E));
    for (int v = 0; v < nvec; ++v) al[v] = -al[v];
    CKE(axpby(al, q, ones, res));
    CKE(dots_host(res, res));
    bool done = true;
    for (int v = 0; v < nvec; ++v) {
      rel[v] = r0[v] > 0 ? std::sqrt(h[2 * v]) / r0[v] : 0.0;
      done = done && rel[v] <= tol;
    }
    if (done) {
      ++it;
      break;
    }
    CKE(launch_precond(c, kp, res, z, nvec, PCX_FP32, s));
    CKE(dots_host(res, z));
    for (int v = 0; v < nvec; ++v) {
      be[v] = rz[v] > 0 ? h[2 * v] / rz[v] : 0.0;
      rz[v] = h[2 * v];
    }
    CKE(axpby(ones, z, be, p));
  }
  if (iters) *iters = it;
  if (relres)
    for (int v = 0; v < nvec; ++v) relres[v] = rel[v];
  return cudaSuccess;
}

#undef CKE

}  // namespace pcx
