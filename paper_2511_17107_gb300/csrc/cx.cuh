// Small complex arithmetic and in-register DFTs shared by the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

namespace pcx {

template <typename T>
struct alignas(2 * sizeof(T)) cx {
  T x, y;
};

template <typename T>
__device__ __forceinline__ cx<T> mk(T a, T b) {
  cx<T> r;
  r.x = a;
  r.y = b;
  return r;
}
template <typename T>
__device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return mk(a.x + b.x, a.y + b.y); }
template <typename T>
__device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return mk(a.x - b.x, a.y - b.y); }
template <typename T>
__device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
  return mk(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
template <typename T>
__device__ __forceinline__ cx<T> scale(cx<T> a, T s) { return mk(a.x * s, a.y * s); }
template <typename T>
__device__ __forceinline__ cx<T> conjg(cx<T> a) { return mk(a.x, -a.y); }
// a + b * c
template <typename T>
__device__ __forceinline__ cx<T> cfma(cx<T> b, cx<T> c, cx<T> a) {
  return mk(fma(b.x, c.x, fma(-b.y, c.y, a.x)), fma(b.x, c.y, fma(b.y, c.x, a.y)));
}
// a + conj(b) * c
template <typename T>
__device__ __forceinline__ cx<T> cfma_conj(cx<T> b, cx<T> c, cx<T> a) {
  return mk(fma(b.x, c.x, fma(b.y, c.y, a.x)), fma(b.x, c.y, fma(-b.y, c.x, a.y)));
}
template <typename T>
__device__ __forceinline__ T norm2(cx<T> a) { return fma(a.x, a.x, a.y * a.y); }

// cos and sin of 2 pi m / 16, m = 0..15 (numeric values of the circle points).
__host__ __device__ constexpr double cos16(int m) {
  return m == 0 ? 1.0 : m == 1 ? 0.92387953251128675613 : m == 2 ? 0.70710678118654752440
       : m == 3 ? 0.38268343236508977173 : m == 4 ? 0.0 : m == 5 ? -0.38268343236508977173
       : m == 6 ? -0.70710678118654752440 : m == 7 ? -0.92387953251128675613 : m == 8 ? -1.0
       : m == 9 ? -0.92387953251128675613 : m == 10 ? -0.70710678118654752440
       : m == 11 ? -0.38268343236508977173 : m == 12 ? 0.0 : m == 13 ? 0.38268343236508977173
       : m == 14 ? 0.70710678118654752440 : 0.92387953251128675613;
}
__host__ __device__ constexpr double sin16(int m) { return cos16((m + 12) & 15); }

// b * exp(DIR * 2 pi i m / 16) with the trivial factors done exactly.
template <int DIR, typename T>
__device__ __forceinline__ cx<T> rot16(cx<T> b, int m) {
  if (m == 0) return b;
  if (m == 4) return DIR > 0 ? mk(-b.y, b.x) : mk(b.y, -b.x);
  if (m == 8) return mk(-b.x, -b.y);
  if (m == 12) return DIR > 0 ? mk(b.y, -b.x) : mk(-b.y, b.x);
  const T c = (T)cos16(m), s = (T)(DIR * sin16(m));
  return mk(fma(b.x, c, -b.y * s), fma(b.x, s, b.y * c));
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// In-register DFT of length R (power of two, <= 16):
//   V[s] = sum_r v[r] exp(DIR * 2 pi i r s / R)
// by radix-2 decimation in time (bit-reversed load, log2 R butterfly stages).
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft(cx<T>* v) {
  constexpr int B = ilog2(R);
  cx<T> t[R];
#pragma unroll
  for (int i = 0; i < R; ++i) t[i] = v[bitrev(i, B)];
#pragma unroll
  for (int len = 2; len <= R; len <<= 1) {
#pragma unroll
    for (int i = 0; i < R; i += len) {
#pragma unroll
      for (int k = 0; k < len / 2; ++k) {
        cx<T> a = t[i + k];
        cx<T> b = rot16<DIR>(t[i + k + len / 2], k * (16 / len));
        t[i + k] = a + b;
        t[i + k + len / 2] = a - b;
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) v[i] = t[i];
}

}  // namespace pcx
