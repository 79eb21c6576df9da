// Internal interface of the learned-correction kernels (cnn.cu) and their
// orchestration (learned.cpp).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

struct pcx_ctx;

namespace pcx {
namespace cnn {

constexpr int HIDDEN = 8;   // hidden channels C
// flat parameter layout: W1 [C][3][27], W2 [C][C][27], W3 [3][C][27],
// V1 [C][9][27], c1 [C], V2 [C][9][27], c2 [C]
constexpr int OFF_W1 = 0;
constexpr int OFF_W2 = OFF_W1 + HIDDEN * 3 * 27;
constexpr int OFF_W3 = OFF_W2 + HIDDEN * HIDDEN * 27;
constexpr int OFF_V1 = OFF_W3 + 3 * HIDDEN * 27;
constexpr int OFF_C1 = OFF_V1 + HIDDEN * 9 * 27;
constexpr int OFF_V2 = OFF_C1 + HIDDEN;
constexpr int OFF_C2 = OFF_V2 + HIDDEN * 9 * 27;
constexpr int NPARAMS = OFF_C2 + HIDDEN;

enum { MODE_PLAIN = 0, MODE_GATE = 1, MODE_SIGMOID = 2 };

// A batch of multi-channel real fields on the N^3 grid: element (sample b,
// channel ch, voxel v) at p + (b / split) * s_hi + (b % split) * s_lo +
// ch * sc + v * sv (floats).  A complex64 block [nvec][3][N^3] viewed as
// 2 nvec real samples (re, im) has split 2, s_hi = 6 N^3, s_lo = 1,
// sc = 2 N^3, sv = 2; a sample-independent field has s_hi = 0.
struct View {
  float* p;
  long long s_hi, s_lo, sc;
  int split, sv;
};

inline View dense_view(float* p, int channels, size_t n3) {
  return View{p, (long long)channels * (long long)n3, 0, (long long)n3, 1, 1};
}
inline View shared_view(float* p, size_t n3) { return View{p, 0, 0, (long long)n3, 1, 1}; }
inline View complex_view(void* p, size_t n3) {
  return View{static_cast<float*>(p), 6 * (long long)n3, 1, 2 * (long long)n3, 2, 2};
}

// out = conv(in, w) (+ gate / sigmoid), nb samples on the n^3 grid; wbf16:
// the weights rounded to BF16 (round to nearest even) before use
cudaError_t conv_fwd(int cin, int cout, int mode, const View& in, const View& out, const float* w, const float* bias,
                     const View& gate, const View& pre, int nb, int n, float out_scale, cudaStream_t s, int wbf16 = 0);
// dw (+)= sum over samples of the weight gradient; scratch >= wgrad_scratch_floats(...)
cudaError_t conv_wgrad(int cin, int cout, const View& dy, const View& x, int nb, int n, float* dw, int accumulate,
                       float* scratch, cudaStream_t s);
size_t wgrad_scratch_floats(int cin, int cout);
cudaError_t adjoint_weights(const float* w, int cout, int cin, float* wt, cudaStream_t s);
// dz = (sum_b dh[b] a[b]) g (1 - g);  dh[b] <- dh[b] g   (gate backward)
cudaError_t gate_backward(const View& dh, const View& a, const float* g, int nb, int c, size_t n3, float* dz,
                          cudaStream_t s);
// db[ch] (+)= sum_v dz[ch][v]
cudaError_t bias_grad(const float* dz, int c, size_t n3, float* db, int accumulate, cudaStream_t s);
// dY = 2 w_v (Y - T) over complex64 blocks; loss[0] += sum_v w_v ||Y_v - T_v||^2
cudaError_t loss_grad(const void* Y, const void* T, const double* wv, int nvec, size_t n3, void* dY, double* loss,
                      cudaStream_t s);
// the 9 feature channels [9][N^3] of the cell blocks of M
cudaError_t features(const pcx_ctx* c, float* f, cudaStream_t s);
cudaError_t adam(float* p, const float* g, float* m, float* v, int np, int step, float lr, float b1, float b2, float eps,
                 cudaStream_t s);
cudaError_t init_params(float* p, unsigned long long seed, cudaStream_t s);
// z = alpha x + beta y over nfloat floats (y may be null)
cudaError_t lincomb(const float* x, float alpha, const float* y, float beta, float* z, size_t nfloat, cudaStream_t s);
// dots[2v], dots[2v+1] = sum conj(a_v) b_v (complex64 vectors of length len)
cudaError_t col_dots(const void* a, const void* b, int nvec, size_t len, double* dots, cudaStream_t s);
// y_v = alpha_v x_v + beta_v y_v (complex64; alpha, beta real, device doubles)
cudaError_t col_axpby(const double* alpha, const void* x, const double* beta, void* y, int nvec, size_t len,
                      cudaStream_t s);

}  // namespace cnn
}  // namespace pcx
