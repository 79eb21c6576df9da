// Small complex arithmetic and in-register DFTs shared by the CUDA kernels.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>
#include <utility>

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

// Compile-time loop: f(std::integral_constant<int, I>) for I = 0..COUNT-1.
template <typename F, int... Is>
__device__ __forceinline__ void static_for_impl(F&& f, std::integer_sequence<int, Is...>) {
  (f(std::integral_constant<int, Is>{}), ...);
}
template <int COUNT, typename F>
__device__ __forceinline__ void static_for(F&& f) {
  static_for_impl(f, std::make_integer_sequence<int, COUNT>{});
}

// b * exp(DIR * 2 pi i M / 16), M a compile-time constant; the factors 1,
// +-i and -1 are applied exactly.
template <int DIR, int M, typename T>
__device__ __forceinline__ cx<T> rot16(cx<T> b) {
  if constexpr (M == 0) {
    return b;
  } else if constexpr (M == 4) {
    return DIR > 0 ? mk(-b.y, b.x) : mk(b.y, -b.x);
  } else if constexpr (M == 8) {
    return mk(-b.x, -b.y);
  } else if constexpr (M == 12) {
    return DIR > 0 ? mk(b.y, -b.x) : mk(-b.y, b.x);
  } else {
    constexpr double cd = cos16(M), sd = DIR * sin16(M);
    const T c = (T)cd, s = (T)sd;
    return mk(fma(b.x, c, -b.y * s), fma(b.x, s, b.y * c));
  }
}

__host__ __device__ constexpr int bitrev(int i, int bits) {
  int r = 0;
  for (int b = 0; b < bits; ++b) r |= ((i >> b) & 1) << (bits - 1 - b);
  return r;
}
__host__ __device__ constexpr int ilog2(int n) { return n <= 1 ? 0 : 1 + ilog2(n >> 1); }

// In-register DFT of length R (power of two, <= 16):
//   V[s] = sum_r v[r] exp(DIR * 2 pi i r s / R)
// by radix-2 decimation in time (bit-reversed load, log2 R butterfly
// stages); every index and twiddle is a compile-time constant.
template <int R, int DIR, typename T>
__device__ __forceinline__ void dft(cx<T>* v) {
  constexpr int B = ilog2(R);
  cx<T> t[R];
  static_for<R>([&](auto i) { t[decltype(i)::value] = v[bitrev(decltype(i)::value, B)]; });
  static_for<B>([&](auto lg) {
    constexpr int LEN = 2 << decltype(lg)::value;
    static_for<R / LEN>([&](auto blk) {
      static_for<LEN / 2>([&](auto kk) {
        constexpr int K = decltype(kk)::value;
        constexpr int A = decltype(blk)::value * LEN + K;
        const cx<T> a = t[A];
        const cx<T> b = rot16<DIR, K * (16 / LEN)>(t[A + LEN / 2]);
        t[A] = a + b;
        t[A + LEN / 2] = a - b;
      });
    });
  });
  static_for<R>([&](auto i) { v[decltype(i)::value] = t[decltype(i)::value]; });
}

}  // namespace pcx
