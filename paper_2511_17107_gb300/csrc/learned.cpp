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
#include "stream_scratch.h"

namespace pcx {

namespace {

// Workspace of the learned-correction kernels, keyed by (device, stream)
// and shared by every context: a training loop over many structures (one
// context each) holds one buffer, not one per context.  Grown on demand;
// growth synchronises the device, since queued work may still read the old
// buffer.
StreamScratch g_cnn_ws;

cudaError_t ws_get(cudaStream_t s, size_t bytes, char** out) {
  void* p = nullptr;
  cudaError_t e = g_cnn_ws.get(s, bytes, &p);
  *out = static_cast<char*>(p);
  return e;
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

void cnn_release_stream(cudaStream_t s) { g_cnn_ws.release(s); }

#define CKE(x)                                 \
  do {                                         \
    cudaError_t _e = (x);                      \
    if (_e != cudaSuccess) return _e;          \
  } while (0)

cudaError_t cnn_gates(pcx_ctx* c, const float* params, float* gates, cudaStream_t s) {
  const size_t n3 = (size_t)c->n * c->n * c->n;
  char* ws;
  CKE(ws_get(s, align_up(9 * n3 * sizeof(float)), &ws));
  float* f = reinterpret_cast<float*>(ws);
  CKE(cnn::features(c, f, s));
  const cnn::View fv = cnn::shared_view(f, n3), none{};
  const int bf = (c->cnn_form & PCX_CNN_BF16) ? 1 : 0;
  CKE(cnn::conv_fwd(9, C, cnn::MODE_SIGMOID, fv, cnn::dense_view(gates, C, n3), params + cnn::OFF_V1,
                    params + cnn::OFF_C1, none, none, 1, c->n, 1.f, s, bf));
  CKE(cnn::conv_fwd(9, C, cnn::MODE_SIGMOID, fv, cnn::dense_view(gates + C * n3, C, n3), params + cnn::OFF_V2,
                    params + cnn::OFF_C2, none, none, 1, c->n, 1.f, s, bf));
  return cudaSuccess;
}

// The transposed weights of the three layers (conv^T(., W) = conv(., adj W)):
// adj W3 [C][3][27], adj W2 [C][C][27], adj W1 [3][C][27].
constexpr size_t ADJ_FLOATS = (size_t)(C * 3 + C * C + 3 * C) * 27;
static cudaError_t adjoint_layers(const float* params, float* adj, cudaStream_t s) {
  CKE(cnn::adjoint_weights(params + cnn::OFF_W3, 3, C, adj, s));
  CKE(cnn::adjoint_weights(params + cnn::OFF_W2, C, C, adj + C * 3 * 27, s));
  CKE(cnn::adjoint_weights(params + cnn::OFF_W1, C, 3, adj + (C * 3 + C * C) * 27, s));
  return cudaSuccess;
}

// Y = g(Re U) + i g(Im U) for nv complex64 fields (with PCX_CNN_HERMITIAN,
// g_s = (g + g^T) / 2 in place of g); h1, h2: 2 nv C N^3 floats each; adj:
// ADJ_FLOATS floats (PCX_CNN_HERMITIAN only)
static cudaError_t forward_chunk(pcx_ctx* c, const float* params, const float* gates, const void* U, void* Y, int nv,
                                 float* h1, float* h2, float* adj, float out_scale, cudaStream_t s) {
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const int nb = 2 * nv;
  const cnn::View none{};
  const int bf = (c->cnn_form & PCX_CNN_BF16) ? 1 : 0;
  const bool herm = (c->cnn_form & PCX_CNN_HERMITIAN) != 0;
  const cnn::View Uv = cnn::complex_view(const_cast<void*>(U), n3);
  const cnn::View G1 = cnn::shared_view(const_cast<float*>(gates), n3);
  const cnn::View G2 = cnn::shared_view(const_cast<float*>(gates) + C * n3, n3);
  CKE(cnn::conv_fwd(3, C, cnn::MODE_GATE, Uv, cnn::dense_view(h1, C, n3), params + cnn::OFF_W1, nullptr, G1, none, nb,
                    c->n, 1.f, s, bf));
  CKE(cnn::conv_fwd(C, C, cnn::MODE_GATE, cnn::dense_view(h1, C, n3), cnn::dense_view(h2, C, n3),
                    params + cnn::OFF_W2, nullptr, G2, none, nb, c->n, 1.f, s, bf));
  CKE(cnn::conv_fwd(C, 3, cnn::MODE_PLAIN, cnn::dense_view(h2, C, n3), cnn::complex_view(Y, n3), params + cnn::OFF_W3,
                    nullptr, none, none, nb, c->n, herm ? 0.5f * out_scale : out_scale, s, bf));
  if (herm) {
    // g^T(u) = conv^T(g1 * conv^T(g2 * conv^T(u, W3), W2), W1), added with weight 1/2
    CKE(adjoint_layers(params, adj, s));
    CKE(cnn::conv_fwd(3, C, cnn::MODE_GATE, Uv, cnn::dense_view(h2, C, n3), adj, nullptr, G2, none, nb, c->n, 1.f, s,
                      bf));
    CKE(cnn::conv_fwd(C, C, cnn::MODE_GATE, cnn::dense_view(h2, C, n3), cnn::dense_view(h1, C, n3), adj + C * 3 * 27,
                      nullptr, G1, none, nb, c->n, 1.f, s, bf));
    CKE(cnn::conv_fwd(C, 3, cnn::MODE_PLAIN, cnn::dense_view(h1, C, n3), cnn::complex_view(h2, n3),
                      adj + (C * 3 + C * C) * 27, nullptr, none, none, nb, c->n, 0.5f * out_scale, s, bf));
    CKE(cnn::lincomb(static_cast<const float*>(Y), 1.f, h2, 1.f, static_cast<float*>(Y), (size_t)nv * 6 * n3, s));
  }
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
  CKE(ws_get(s, 2 * hb + align_up(ADJ_FLOATS * sizeof(float)), &ws));
  float* h1 = reinterpret_cast<float*>(ws);
  float* h2 = reinterpret_cast<float*>(ws + hb);
  float* adj = reinterpret_cast<float*>(ws + 2 * hb);
  const size_t vlen = 3 * n3;
  for (int v0 = 0; v0 < nvec; v0 += chunk) {
    const int nv = nvec - v0 < chunk ? nvec - v0 : chunk;
    CKE(forward_chunk(c, params, gates, static_cast<const float2*>(U) + (size_t)v0 * vlen,
                      static_cast<float2*>(Y) + (size_t)v0 * vlen, nv, h1, h2, adj, 1.f, s));
  }
  return cudaSuccess;
}

// Loss and gradient.  Plain form: y = g(u) (three layers, gates g1, g2).
// Hermitian form: y = (g(u) + g^T(u)) / 2; the transpose path
//   b3 = conv^T(u, W3), k2 = g2 b3, b2 = conv^T(k2, W2), k1 = g1 b2,
//   y' = conv^T(k1, W1)
// contributes dW1 += wgrad(k1 <- dy), dk1 = conv(dy, W1), db2 = g1 dk1,
// dW2 += wgrad(k2 <- db2), dk2 = conv(db2, W2), db3 = g2 dk2,
// dW3 += wgrad(u <- db3), and gate terms from (dk1, b2) and (dk2, b3), where
// wgrad(a <- b) = d/dW <a, conv(b, W)>.
cudaError_t cnn_grad(pcx_ctx* c, const float* params, const void* U, const void* T, const double* wv_host, int nvec,
                     float* grad, int accumulate, double* loss_host, cudaStream_t s) {
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const int nb = 2 * nvec, n = c->n;
  const size_t act = (size_t)nb * C * n3;
  const bool herm = (c->cnn_form & PCX_CNN_HERMITIAN) != 0;
  const int bf = (c->cnn_form & PCX_CNN_BF16) ? 1 : 0;
  size_t need = 0;
  need += align_up(9 * n3 * 4) + align_up(2 * C * n3 * 4);           // f, gates
  need += (herm ? 12 : 6) * align_up(act * 4);                       // activations and their gradients
  need += 3 * align_up((size_t)nvec * 6 * n3 * 4);                   // Y, dY, y' of the transpose path
  need += 4 * align_up(C * n3 * 4);                                  // dz1, dz2 and their transpose-path parts
  need += align_up(cnn::wgrad_scratch_floats(9, C) * 4);             // the largest wgrad scratch
  need += 2 * align_up(C * C * 27 * 4) + align_up(ADJ_FLOATS * 4) + align_up(nvec * 8 + 8);   // weights, w, loss
  char* ws;
  CKE(ws_get(s, need, &ws));
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
  float* Yt = cv.take<float>((size_t)nvec * 6 * n3);
  float* dz1 = cv.take<float>(C * n3);
  float* dz2 = cv.take<float>(C * n3);
  float* dz1t = cv.take<float>(C * n3);
  float* dz2t = cv.take<float>(C * n3);
  float* scr = cv.take<float>(cnn::wgrad_scratch_floats(9, C));
  float* wt3 = cv.take<float>(C * C * 27);
  float* wt2 = cv.take<float>(C * C * 27);
  float* adj = cv.take<float>(ADJ_FLOATS);
  double* wdev = cv.take<double>(nvec + 1);
  double* ldev = wdev + nvec;
  float *b3 = nullptr, *k2 = nullptr, *b2 = nullptr, *k1 = nullptr, *dk1 = nullptr, *dk2 = nullptr;
  if (herm) {
    b3 = cv.take<float>(act);
    k2 = cv.take<float>(act);
    b2 = cv.take<float>(act);
    k1 = cv.take<float>(act);
    dk1 = cv.take<float>(act);
    dk2 = cv.take<float>(act);
  }
  const cnn::View none{};
  // gates and forward pass with the pre-gate activations kept
  CKE(cnn::features(c, f, s));
  const cnn::View fv = cnn::shared_view(f, n3);
  CKE(cnn::conv_fwd(9, C, cnn::MODE_SIGMOID, fv, cnn::dense_view(g, C, n3), params + cnn::OFF_V1, params + cnn::OFF_C1,
                    none, none, 1, n, 1.f, s, bf));
  CKE(cnn::conv_fwd(9, C, cnn::MODE_SIGMOID, fv, cnn::dense_view(g + C * n3, C, n3), params + cnn::OFF_V2,
                    params + cnn::OFF_C2, none, none, 1, n, 1.f, s, bf));
  const cnn::View G1 = cnn::shared_view(g, n3), G2 = cnn::shared_view(g + C * n3, n3);
  const cnn::View Uv = cnn::complex_view(const_cast<void*>(U), n3);
  const cnn::View A1 = cnn::dense_view(a1, C, n3), H1 = cnn::dense_view(h1, C, n3);
  const cnn::View A2 = cnn::dense_view(a2, C, n3), H2 = cnn::dense_view(h2, C, n3);
  const cnn::View DH1 = cnn::dense_view(dh1, C, n3), DH2 = cnn::dense_view(dh2, C, n3);
  const float half = herm ? 0.5f : 1.f;
  CKE(cnn::conv_fwd(3, C, cnn::MODE_GATE, Uv, H1, params + cnn::OFF_W1, nullptr, G1, A1, nb, n, 1.f, s, bf));
  CKE(cnn::conv_fwd(C, C, cnn::MODE_GATE, H1, H2, params + cnn::OFF_W2, nullptr, G2, A2, nb, n, 1.f, s, bf));
  CKE(cnn::conv_fwd(C, 3, cnn::MODE_PLAIN, H2, cnn::complex_view(Y, n3), params + cnn::OFF_W3, nullptr, none, none, nb,
                    n, half, s, bf));
  if (herm) {
    CKE(adjoint_layers(params, adj, s));
    const cnn::View B3 = cnn::dense_view(b3, C, n3), K2 = cnn::dense_view(k2, C, n3);
    const cnn::View B2 = cnn::dense_view(b2, C, n3), K1 = cnn::dense_view(k1, C, n3);
    CKE(cnn::conv_fwd(3, C, cnn::MODE_GATE, Uv, K2, adj, nullptr, G2, B3, nb, n, 1.f, s, bf));
    CKE(cnn::conv_fwd(C, C, cnn::MODE_GATE, K2, K1, adj + C * 3 * 27, nullptr, G1, B2, nb, n, 1.f, s, bf));
    CKE(cnn::conv_fwd(C, 3, cnn::MODE_PLAIN, K1, cnn::complex_view(Yt, n3), adj + (C * 3 + C * C) * 27, nullptr, none,
                      none, nb, n, half, s, bf));
    CKE(cnn::lincomb(Y, 1.f, Yt, 1.f, Y, (size_t)nvec * 6 * n3, s));
  }
  // loss and dY (dL/dy; each path's output carries the factor 1/2 of g_s)
  CKE(cudaMemcpyAsync(wdev, wv_host, sizeof(double) * nvec, cudaMemcpyHostToDevice, s));
  CKE(cudaMemsetAsync(ldev, 0, sizeof(double), s));
  CKE(cnn::loss_grad(Y, T, wdev, nvec, n3, dY, ldev, s));
  if (herm) CKE(cnn::lincomb(dY, 0.5f, nullptr, 0.f, dY, (size_t)nvec * 6 * n3, s));
  const cnn::View DY = cnn::complex_view(dY, n3);
  // layer 3
  CKE(cnn::conv_wgrad(C, 3, DY, H2, nb, n, grad + cnn::OFF_W3, accumulate, scr, s));
  CKE(cnn::adjoint_weights(params + cnn::OFF_W3, 3, C, wt3, s));
  CKE(cnn::conv_fwd(3, C, cnn::MODE_PLAIN, DY, DH2, wt3, nullptr, none, none, nb, n, 1.f, s, bf));
  // gate 2 and layer 2
  CKE(cnn::gate_backward(DH2, A2, g + C * n3, nb, C, n3, dz2, s));
  CKE(cnn::conv_wgrad(C, C, DH2, H1, nb, n, grad + cnn::OFF_W2, accumulate, scr, s));
  CKE(cnn::adjoint_weights(params + cnn::OFF_W2, C, C, wt2, s));
  CKE(cnn::conv_fwd(C, C, cnn::MODE_PLAIN, DH2, DH1, wt2, nullptr, none, none, nb, n, 1.f, s, bf));
  // gate 1 and layer 1
  CKE(cnn::gate_backward(DH1, A1, g, nb, C, n3, dz1, s));
  CKE(cnn::conv_wgrad(3, C, DH1, Uv, nb, n, grad + cnn::OFF_W1, accumulate, scr, s));
  if (herm) {
    // the transpose path (gradients always add to what layers 1-3 wrote)
    const cnn::View K2 = cnn::dense_view(k2, C, n3), K1 = cnn::dense_view(k1, C, n3);
    const cnn::View B3 = cnn::dense_view(b3, C, n3), B2 = cnn::dense_view(b2, C, n3);
    const cnn::View DK1 = cnn::dense_view(dk1, C, n3), DK2 = cnn::dense_view(dk2, C, n3);
    CKE(cnn::conv_wgrad(3, C, K1, DY, nb, n, grad + cnn::OFF_W1, 1, scr, s));
    CKE(cnn::conv_fwd(3, C, cnn::MODE_PLAIN, DY, DK1, params + cnn::OFF_W1, nullptr, none, none, nb, n, 1.f, s, bf));
    CKE(cnn::gate_backward(DK1, B2, g, nb, C, n3, dz1t, s));   // dk1 <- g1 dk1 = db2
    CKE(cnn::conv_wgrad(C, C, K2, DK1, nb, n, grad + cnn::OFF_W2, 1, scr, s));
    CKE(cnn::conv_fwd(C, C, cnn::MODE_PLAIN, DK1, DK2, params + cnn::OFF_W2, nullptr, none, none, nb, n, 1.f, s, bf));
    CKE(cnn::gate_backward(DK2, B3, g + C * n3, nb, C, n3, dz2t, s));   // dk2 <- g2 dk2 = db3
    CKE(cnn::conv_wgrad(C, 3, Uv, DK2, nb, n, grad + cnn::OFF_W3, 1, scr, s));
    CKE(cnn::lincomb(dz1, 1.f, dz1t, 1.f, dz1, C * n3, s));
    CKE(cnn::lincomb(dz2, 1.f, dz2t, 1.f, dz2, C * n3, s));
  }
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

// T R = T0 R + K_A F3^H g(e) / |k|^2 with e = F3 (K_A^H R / |k|^2) (g_s for
// the Hermitian form): the net's output joins eps e in real space before the
// forward transform.
cudaError_t cnn_precond(pcx_ctx* c, const KParams& kp, const float* params, const float* gates, const void* R, void* W,
                        int nvec, cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const int chunk = forward_chunk_size(c, nvec);
  const size_t hb = align_up(2 * (size_t)chunk * C * n3 * sizeof(float));
  const size_t tb = align_up((size_t)chunk * 3 * n3 * sizeof(float2));
  char* ws;
  CKE(ws_get(s, 2 * hb + 2 * tb + align_up(ADJ_FLOATS * sizeof(float)), &ws));
  float* h1 = reinterpret_cast<float*>(ws);
  float* h2 = reinterpret_cast<float*>(ws + hb);
  float2* e = reinterpret_cast<float2*>(ws + 2 * hb);
  float2* y = reinterpret_cast<float2*>(ws + 2 * hb + tb);
  float* adj = reinterpret_cast<float*>(ws + 2 * hb + 2 * tb);
  const size_t vlen = 3 * n3;
  const double inv_n3 = 1.0 / (double)n3;
  for (int v0 = 0; v0 < nvec; v0 += chunk) {
    const int nv = nvec - v0 < chunk ? nvec - v0 : chunk;
    const float2* r = static_cast<const float2*>(R) + (size_t)v0 * vlen;
    float2* w = static_cast<float2*>(W) + (size_t)v0 * vlen;
    CKE(launch_curl_h(c, kp, r, e, nv, 1, PCX_FP32, s));
    CKE(launch_fft(c, e, e, nv, +1, PCX_FP32, s));
    CKE(forward_chunk(c, params, gates, e, y, nv, h1, h2, adj, 1.f, s));
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
    CKE(ws_get(s, align_up(2 * nvec * sizeof(double)), &ws));
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
  CKE(ws_get(s, 4 * vb + align_up(6 * (size_t)nvec * sizeof(double)), &ws));
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
