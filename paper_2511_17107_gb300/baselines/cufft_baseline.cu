// Library-call baselines of the apply and of the Gram products, timed beside
// the hand-written kernels and never used by them (libpcx_baselines.so is a
// separate library that nothing in libpcx loads).
//
// The apply follows the implementation the paper describes (Sec. 2.4 eq.
// matrixfree_kcform with the factorisation of Prop. 2.8; library FFT calls
// and elementwise kernels on stored per-mode symbols):
//   u = K_A^H x = -conj(kappa) x x and s = gamma kappa . x     (elementwise)
//   e = F3 u                    batched 3D cuFFT, positive exponent
//   m = M e / N^3               elementwise, one 3x3 Hermitian block per cell
//   w = F3^H m                  batched 3D cuFFT, negative exponent
//   y = kappa x w + conj(kappa) s                               (elementwise)
// with kappa stored as three complex arrays of N^3 entries (the symbol
// tables of Sec. 2.5) and M as nine real arrays of N^3 entries.  The Gram
// product G = A^H B is cublasCgemm / cublasZgemm.
#include <cublas_v2.h>
#include <cuda_runtime.h>
#include <cufft.h>

#include <cstdint>
#include <cstring>
#include <vector>

namespace {

template <typename T>
struct C2 {
  T x, y;
};

template <typename T>
__device__ __forceinline__ C2<T> cmul(C2<T> a, C2<T> b) {
  return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ C2<T> cmulc(C2<T> a, C2<T> b) {   // conj(a) b
  return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename T>
__device__ __forceinline__ C2<T> cadd(C2<T> a, C2<T> b) {
  return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ C2<T> csub(C2<T> a, C2<T> b) {
  return {a.x - b.x, a.y - b.y};
}

// u = -conj(kappa) x x (in U), s = gamma kappa . x
template <typename T>
__global__ void pre_kernel(const C2<T>* __restrict__ X, C2<T>* __restrict__ U, C2<T>* __restrict__ S,
                           const C2<T>* __restrict__ kap, size_t n3, int nvec, T gamma) {
  const size_t total = n3 * nvec;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e / n3, p = e % n3, b = v * 3 * n3 + p;
    const C2<T> k0 = kap[p], k1 = kap[n3 + p], k2 = kap[2 * n3 + p];
    const C2<T> x0 = X[b], x1 = X[b + n3], x2 = X[b + 2 * n3];
    const C2<T> s = cadd(cadd(cmul(k0, x0), cmul(k1, x1)), cmul(k2, x2));
    S[e] = {gamma * s.x, gamma * s.y};
    U[b] = csub(cmulc(k2, x1), cmulc(k1, x2));
    U[b + n3] = csub(cmulc(k0, x2), cmulc(k2, x0));
    U[b + 2 * n3] = csub(cmulc(k1, x0), cmulc(k0, x1));
  }
}

// m = M e / N^3 per cell, in place; M as [9][N^3]: d1 d2 d3 re12 im12 re13 im13 re23 im23
template <typename T>
__global__ void m_kernel(C2<T>* __restrict__ E, const T* __restrict__ M, size_t n3, int nvec, T inv_n3) {
  const size_t total = n3 * nvec;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e / n3, c = e % n3, b = v * 3 * n3 + c;
    const T d1 = M[c], d2 = M[n3 + c], d3 = M[2 * n3 + c];
    const C2<T> o12 = {M[3 * n3 + c], M[4 * n3 + c]}, o13 = {M[5 * n3 + c], M[6 * n3 + c]},
                o23 = {M[7 * n3 + c], M[8 * n3 + c]};
    const C2<T> e0 = E[b], e1 = E[b + n3], e2 = E[b + 2 * n3];
    const C2<T> m0 = cadd(cadd(C2<T>{d1 * e0.x, d1 * e0.y}, cmul(o12, e1)), cmul(o13, e2));
    const C2<T> m1 = cadd(cadd(cmulc(o12, e0), C2<T>{d2 * e1.x, d2 * e1.y}), cmul(o23, e2));
    const C2<T> m2 = cadd(cadd(cmulc(o13, e0), cmulc(o23, e1)), C2<T>{d3 * e2.x, d3 * e2.y});
    E[b] = {m0.x * inv_n3, m0.y * inv_n3};
    E[b + n3] = {m1.x * inv_n3, m1.y * inv_n3};
    E[b + 2 * n3] = {m2.x * inv_n3, m2.y * inv_n3};
  }
}

// y = kappa x w + conj(kappa) s, in place on W
template <typename T>
__global__ void post_kernel(C2<T>* __restrict__ W, const C2<T>* __restrict__ S, const C2<T>* __restrict__ kap,
                            size_t n3, int nvec) {
  const size_t total = n3 * nvec;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e / n3, p = e % n3, b = v * 3 * n3 + p;
    const C2<T> k0 = kap[p], k1 = kap[n3 + p], k2 = kap[2 * n3 + p];
    const C2<T> w0 = W[b], w1 = W[b + n3], w2 = W[b + 2 * n3];
    const C2<T> s = S[e];
    W[b] = cadd(csub(cmul(k1, w2), cmul(k2, w1)), cmulc(k0, s));
    W[b + n3] = cadd(csub(cmul(k2, w0), cmul(k0, w2)), cmulc(k1, s));
    W[b + 2 * n3] = cadd(csub(cmul(k0, w1), cmul(k1, w0)), cmulc(k2, s));
  }
}

struct Handle {
  int n = 0, precision = 0, chunk = 0;
  size_t n3 = 0;
  void* kap = nullptr;   // [3][N^3] complex
  void* M = nullptr;     // [9][N^3] real
  void* S = nullptr;     // [chunk][N^3] complex
  double gamma = 0;
  cufftHandle plan = 0;
};

template <typename T>
int upload(Handle* h, const double* kap_host, const double* blocks_host) {
  const size_t n3 = h->n3;
  std::vector<T> k(6 * n3), m(9 * n3);
  for (size_t i = 0; i < 6 * n3; ++i) k[i] = (T)kap_host[i];
  for (size_t c = 0; c < n3; ++c)
    for (int j = 0; j < 9; ++j) m[j * n3 + c] = (T)blocks_host[9 * c + j];
  if (cudaMalloc(&h->kap, k.size() * sizeof(T)) != cudaSuccess) return -2;
  if (cudaMalloc(&h->M, m.size() * sizeof(T)) != cudaSuccess) return -2;
  if (cudaMalloc(&h->S, (size_t)h->chunk * n3 * 2 * sizeof(T)) != cudaSuccess) return -2;
  if (cudaMemcpy(h->kap, k.data(), k.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return -6;
  if (cudaMemcpy(h->M, m.data(), m.size() * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) return -6;
  return 0;
}

template <typename T>
int apply_t(Handle* h, const void* X, void* Y, int nvec, cudaStream_t s) {
  const size_t n3 = h->n3;
  const int threads = 256;
  const bool dbl = sizeof(T) == 8;
  if (cufftSetStream(h->plan, s) != CUFFT_SUCCESS) return -6;
  for (int v0 = 0; v0 < nvec; v0 += h->chunk) {
    const int nv = nvec - v0 < h->chunk ? nvec - v0 : h->chunk;
    const C2<T>* x = static_cast<const C2<T>*>(X) + (size_t)v0 * 3 * n3;
    C2<T>* y = static_cast<C2<T>*>(Y) + (size_t)v0 * 3 * n3;
    const size_t total = n3 * nv;
    const unsigned blocks = (unsigned)((total + threads - 1) / threads < 152 * 16 ? (total + threads - 1) / threads : 152 * 16);
    pre_kernel<T><<<blocks, threads, 0, s>>>(x, y, static_cast<C2<T>*>(h->S), static_cast<const C2<T>*>(h->kap), n3, nv,
                                            (T)h->gamma);
    // the plan covers a full chunk (pcxb_apply takes whole chunks only)
    if (dbl ? cufftExecZ2Z(h->plan, (cufftDoubleComplex*)y, (cufftDoubleComplex*)y, CUFFT_INVERSE)
            : cufftExecC2C(h->plan, (cufftComplex*)y, (cufftComplex*)y, CUFFT_INVERSE))
      return -6;
    m_kernel<T><<<blocks, threads, 0, s>>>(y, static_cast<const T*>(h->M), n3, nv, (T)(1.0 / (double)n3));
    if (dbl ? cufftExecZ2Z(h->plan, (cufftDoubleComplex*)y, (cufftDoubleComplex*)y, CUFFT_FORWARD)
            : cufftExecC2C(h->plan, (cufftComplex*)y, (cufftComplex*)y, CUFFT_FORWARD))
      return -6;
    post_kernel<T><<<blocks, threads, 0, s>>>(y, static_cast<const C2<T>*>(h->S), static_cast<const C2<T>*>(h->kap),
                                             n3, nv);
  }
  return cudaGetLastError() == cudaSuccess ? 0 : -6;
}

}  // namespace

extern "C" {

// Baseline apply handle for one grid, one k and one precision (0: complex128,
// 1: complex64).  kappa_host: [3][N^3] complex128 (interleaved doubles), the
// per-mode symbol kappa_i(p); blocks_host: N^3 x 9 doubles, the packed cell
// blocks of M (d1 d2 d3 re12 im12 re13 im13 re23 im23); chunk: vectors per
// cuFFT batch (nvec of pcxb_apply must be a multiple).  Returns 0 or a
// negative status (-1 bad argument, -2 out of memory, -6 CUDA/cuFFT error).
int pcxb_create(int n, int precision, const double* kappa_host, const double* blocks_host, double gamma, int chunk,
                void** out) {
  if (n < 2 || chunk < 1 || !kappa_host || !blocks_host || !out) return -1;
  Handle* h = new Handle;
  h->n = n;
  h->precision = precision;
  h->chunk = chunk;
  h->n3 = (size_t)n * n * n;
  h->gamma = gamma;
  int st = precision == 0 ? upload<double>(h, kappa_host, blocks_host) : upload<float>(h, kappa_host, blocks_host);
  int dims[3] = {n, n, n};
  if (st == 0 && cufftPlanMany(&h->plan, 3, dims, nullptr, 1, (int)h->n3, nullptr, 1, (int)h->n3,
                               precision == 0 ? CUFFT_Z2Z : CUFFT_C2C, 3 * chunk) != CUFFT_SUCCESS)
    st = -6;
  if (st != 0) {
    if (h->plan) cufftDestroy(h->plan);
    cudaFree(h->kap);
    cudaFree(h->M);
    cudaFree(h->S);
    delete h;
    return st;
  }
  *out = h;
  return 0;
}

// Y = Op X for nvec vectors (a multiple of the handle's chunk), device
// buffers [nvec][3][N^3] in the handle's precision, on `stream`.
int pcxb_apply(void* handle, const void* X, void* Y, int nvec, void* stream) {
  Handle* h = static_cast<Handle*>(handle);
  if (!h || !X || !Y || nvec < 0 || nvec % h->chunk) return -1;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return h->precision == 0 ? apply_t<double>(h, X, Y, nvec, s) : apply_t<float>(h, X, Y, nvec, s);
}

void pcxb_destroy(void* handle) {
  Handle* h = static_cast<Handle*>(handle);
  if (!h) return;
  if (h->plan) cufftDestroy(h->plan);
  cudaFree(h->kap);
  cudaFree(h->M);
  cudaFree(h->S);
  delete h;
}

// G = A^H B (na x nb, column-major: G[i + na j] = sum_l conj(A[i][l]) B[j][l])
// for column blocks A [na][L], B [nb][L] (device), precision 0: complex128
// (cublasZgemm), 1: complex64 (cublasCgemm, G complex64).  A cuBLAS handle is
// created on first use and kept.
int pcxb_gram(const void* A, int na, const void* B, int nb, size_t L, int precision, void* G, void* stream) {
  static cublasHandle_t blas = nullptr;
  if (!blas && cublasCreate(&blas) != CUBLAS_STATUS_SUCCESS) return -6;
  if (cublasSetStream(blas, static_cast<cudaStream_t>(stream)) != CUBLAS_STATUS_SUCCESS) return -6;
  cublasStatus_t st;
  if (precision == 0) {
    const cuDoubleComplex one = {1.0, 0.0}, zero = {0.0, 0.0};
    st = cublasZgemm(blas, CUBLAS_OP_C, CUBLAS_OP_N, na, nb, (int)L, &one, (const cuDoubleComplex*)A, (int)L,
                     (const cuDoubleComplex*)B, (int)L, &zero, (cuDoubleComplex*)G, na);
  } else {
    const cuComplex one = {1.0f, 0.0f}, zero = {0.0f, 0.0f};
    st = cublasCgemm(blas, CUBLAS_OP_C, CUBLAS_OP_N, na, nb, (int)L, &one, (const cuComplex*)A, (int)L,
                     (const cuComplex*)B, (int)L, &zero, (cuComplex*)G, na);
  }
  return st == CUBLAS_STATUS_SUCCESS ? 0 : -6;
}

}  // extern "C"
