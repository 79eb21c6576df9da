// Mixed-precision Gram product G = A^H B with A complex128 and B complex64,
// accurate to about 2^-44 relative to ||A_i|| ||B_j||, on the FP32 pipes.
//
// This is the product the mixed-precision Rayleigh-Ritz step needs (Sec. 4,
// LOBPCG): the rows of G_A and G_B that belong to the FP64 block X, i.e.
// X^H [P W] and (Op X)^H [P W] with the search directions P, W in FP32.
// Their entries are of the size of the residual, far below the FP32 rounding
// of the products, so they are accumulated as double-float sums.
//
// Each FP64 entry of A is split once, when staged, into FP32 hi + lo with
// integer operations (hi = the leading 24 significand bits, lo = the
// remainder rounded to 24 bits), so the inner loop runs no FP64 instruction.
// B is FP32 and enters the products unsplit: a real term x*y becomes
// TwoProd(hi, y) + lo*y and is added to a (sum, compensation) pair with
// Knuth's TwoSum (TAOCP vol. 2, Sec. 4.2.2; Dekker 1971).  Entries of A with
// magnitude below 2^-126 are treated as 0; entries at or above 2^128 give NaN.
//
// Rows of A may come from two column blocks A1 (na1 columns) and A2 (the
// rest), so [X | Op X] is one launch without a copy.  Each CTA writes its
// partial sums to scratch; a second kernel adds them in a fixed order (the
// result does not depend on scheduling).
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "pcx_internal.h"

namespace pcx {
namespace {

constexpr int XT = 32;        // tile: 32 rows of A x 32 columns of B
constexpr int XL = 32;        // vector entries staged per step
constexpr int XTHREADS = 256; // 16 x 16 threads, 2 x 2 outputs each

// v = hi + lo up to 2^-47 |v| for 2^-126 <= |v| < 2^128.
__device__ __forceinline__ void split_f64(double v, float& hi, float& lo) {
  const unsigned long long b = static_cast<unsigned long long>(__double_as_longlong(v));
  const unsigned sign = static_cast<unsigned>(b >> 63) << 31;
  const int ex = static_cast<int>((b >> 52) & 0x7FF);
  const unsigned long long mant = b & 0xFFFFFFFFFFFFFull;
  const int fe = ex - 1023 + 127;
  if (fe <= 0) {   // zero, FP64 subnormal or below the FP32 normal range
    hi = lo = 0.f;
    return;
  }
  if (fe >= 255) {   // outside the FP32 range, Inf or NaN
    hi = lo = __uint_as_float(0x7fc00000u);
    return;
  }
  hi = __uint_as_float(sign | (static_cast<unsigned>(fe) << 23) | static_cast<unsigned>(mant >> 29));
  // remainder: low 29 significand bits, weight 2^(ex - 1075)
  const unsigned rem = static_cast<unsigned>(mant & 0x1FFFFFFFull);
  const int le = ex - 1075 + 127;
  const float scale = le > 0 ? __uint_as_float(static_cast<unsigned>(le) << 23) : 0.f;
  const float l = __fmul_rn(__uint2float_rn(rem), scale);
  lo = sign ? -l : l;
}

struct DF {
  float s, c;
};

// acc += (xh + xl) * y  (NEG: acc -= ...), error-free up to the lo*y rounding.
template <bool NEG>
__device__ __forceinline__ void df_mac(DF& acc, float xh, float xl, float y) {
  float p = __fmul_rn(xh, y);
  float e = fmaf(xh, y, -p);   // p + e == xh * y exactly
  e = fmaf(xl, y, e);
  if (NEG) {
    p = -p;
    e = -e;
  }
  const float s = __fadd_rn(acc.s, p);
  const float bb = __fsub_rn(s, acc.s);
  const float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.s = s;
  acc.c = __fadd_rn(acc.c, __fadd_rn(err, e));
}

// acc += (xh + xl) * (yh + yl)  (NEG: acc -= ...)
template <bool NEG>
__device__ __forceinline__ void df_mac2(DF& acc, float xh, float xl, float yh, float yl) {
  float p = __fmul_rn(xh, yh);
  float e = fmaf(xh, yh, -p);   // p + e == xh * yh exactly
  e = fmaf(xh, yl, e);
  e = fmaf(xl, yh, e);
  e = fmaf(xl, yl, e);
  if (NEG) {
    p = -p;
    e = -e;
  }
  const float s = __fadd_rn(acc.s, p);
  const float bb = __fsub_rn(s, acc.s);
  const float err = __fadd_rn(__fsub_rn(acc.s, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  acc.s = s;
  acc.c = __fadd_rn(acc.c, __fadd_rn(err, e));
}

// (s, c) <- (s + c, the rounding error of that sum): keeps the compensation
// at half an ulp of s, so that its own rounding stays at 2^-48 of s per add
// (Fast2Sum, valid since |c| <= |s| here or s = 0).
__device__ __forceinline__ void df_renorm(DF& a) {
  const float s = __fadd_rn(a.s, a.c);
  a.c = __fsub_rn(a.c, __fsub_rn(s, a.s));
  a.s = s;
}

// G = A^H B with A and B complex128, both split into FP32 hi + lo when
// staged; tile T x T (T = 16 or 32), 256 threads with (T/16)^2 outputs each.
template <int T>
__global__ void __launch_bounds__(XTHREADS, 4)
    gram_dd_kernel(const double2* __restrict__ A, int na, const double2* __restrict__ B, int nb, size_t L,
                   size_t rows_per_cta, double2* __restrict__ partial) {
  constexpr int O = T / 16;
  __shared__ float4 sa[XL][T + 1];
  __shared__ float4 sb[XL][T + 1];
  const int ti = blockIdx.x * T, tj = blockIdx.y * T;
  const size_t l0 = (size_t)blockIdx.z * rows_per_cta;
  const size_t l1 = (l0 + rows_per_cta < L) ? l0 + rows_per_cta : L;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  DF re[O][O], im[O][O];
#pragma unroll
  for (int a = 0; a < O; ++a)
#pragma unroll
    for (int b = 0; b < O; ++b) re[a][b] = im[a][b] = DF{0.f, 0.f};
  for (size_t base = l0; base < l1; base += XL) {
#pragma unroll
    for (int k = 0; k < XL * T / XTHREADS; ++k) {
      const int e = threadIdx.x + k * XTHREADS;
      const int r = e % XL, col = e / XL;
      const size_t l = base + r;
      const bool ok = l < l1;
      float4 av = make_float4(0.f, 0.f, 0.f, 0.f), bv = av;
      if (ok && ti + col < na) {
        const double2 v = A[(size_t)(ti + col) * L + l];
        split_f64(v.x, av.x, av.y);
        split_f64(v.y, av.z, av.w);
      }
      if (ok && tj + col < nb) {
        const double2 v = B[(size_t)(tj + col) * L + l];
        split_f64(v.x, bv.x, bv.y);
        split_f64(v.y, bv.z, bv.w);
      }
      sa[r][col] = av;
      sb[r][col] = bv;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < XL; ++r) {
      float4 ar[O], br[O];
#pragma unroll
      for (int a = 0; a < O; ++a) ar[a] = sa[r][ty + 16 * a];
#pragma unroll
      for (int b = 0; b < O; ++b) br[b] = sb[r][tx + 16 * b];
#pragma unroll
      for (int a = 0; a < O; ++a)
#pragma unroll
        for (int b = 0; b < O; ++b) {
          // conj(a) b: re = ar br + ai bi, im = ar bi - ai br
          df_mac2<false>(re[a][b], ar[a].x, ar[a].y, br[b].x, br[b].y);
          df_mac2<false>(re[a][b], ar[a].z, ar[a].w, br[b].z, br[b].w);
          df_mac2<false>(im[a][b], ar[a].x, ar[a].y, br[b].z, br[b].w);
          df_mac2<true>(im[a][b], ar[a].z, ar[a].w, br[b].x, br[b].y);
        }
    }
#pragma unroll
    for (int a = 0; a < O; ++a)
#pragma unroll
      for (int b = 0; b < O; ++b) {
        df_renorm(re[a][b]);
        df_renorm(im[a][b]);
      }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < O; ++a)
#pragma unroll
    for (int b = 0; b < O; ++b) {
      const int i = ti + ty + 16 * a, j = tj + tx + 16 * b;
      if (i < na && j < nb)
        partial[((size_t)blockIdx.z * na + i) * nb + j] =
            make_double2((double)re[a][b].s + (double)re[a][b].c, (double)im[a][b].s + (double)im[a][b].c);
    }
}

// TA rows of A (16 or 32) x XT columns of B per tile; thread (ty, tx) owns
// rows ty + 16 a (a < TA / 16) and columns tx, tx + 16.
template <int TA>
__global__ void __launch_bounds__(XTHREADS, 4)
    gram_x_kernel(const double2* __restrict__ A1, int na1, const double2* __restrict__ A2, int na,
                  const float2* __restrict__ B, int nb, size_t L, size_t rows_per_cta, double2* __restrict__ partial) {
  constexpr int OA = TA / 16;
  __shared__ float4 sa[XL][TA + 1];   // (re hi, re lo, im hi, im lo)
  __shared__ float2 sb[XL][XT + 1];
  const int ti = blockIdx.x * TA, tj = blockIdx.y * XT;
  const size_t l0 = (size_t)blockIdx.z * rows_per_cta;
  const size_t l1 = (l0 + rows_per_cta < L) ? l0 + rows_per_cta : L;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;
  DF re[OA][2], im[OA][2];
#pragma unroll
  for (int a = 0; a < OA; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) re[a][b] = im[a][b] = DF{0.f, 0.f};
  for (size_t base = l0; base < l1; base += XL) {
#pragma unroll
    for (int k = 0; k < XL * TA / XTHREADS; ++k) {
      const int e = threadIdx.x + k * XTHREADS;
      const int r = e % XL, col = e / XL;
      const size_t l = base + r;
      const int row = ti + col;
      float4 av = make_float4(0.f, 0.f, 0.f, 0.f);
      if (l < l1 && row < na) {
        const double2 v = row < na1 ? A1[(size_t)row * L + l] : A2[(size_t)(row - na1) * L + l];
        split_f64(v.x, av.x, av.y);
        split_f64(v.y, av.z, av.w);
      }
      sa[r][col] = av;
    }
#pragma unroll
    for (int k = 0; k < XL * XT / XTHREADS; ++k) {
      const int e = threadIdx.x + k * XTHREADS;
      const int r = e % XL, col = e / XL;
      const size_t l = base + r;
      sb[r][col] = (l < l1 && tj + col < nb) ? B[(size_t)(tj + col) * L + l] : make_float2(0.f, 0.f);
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < XL; ++r) {
      float4 ar[OA];
#pragma unroll
      for (int a = 0; a < OA; ++a) ar[a] = sa[r][ty + 16 * a];
      const float2 b0 = sb[r][tx], b1 = sb[r][tx + 16];
#pragma unroll
      for (int a = 0; a < OA; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const float4 av = ar[a];
          const float2 bv = b ? b1 : b0;
          // conj(a) b: re = ar br + ai bi, im = ar bi - ai br
          df_mac<false>(re[a][b], av.x, av.y, bv.x);
          df_mac<false>(re[a][b], av.z, av.w, bv.y);
          df_mac<false>(im[a][b], av.x, av.y, bv.y);
          df_mac<true>(im[a][b], av.z, av.w, bv.x);
        }
    }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < OA; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = ti + ty + 16 * a, j = tj + tx + 16 * b;
      if (i < na && j < nb)
        partial[((size_t)blockIdx.z * na + i) * nb + j] =
            make_double2((double)re[a][b].s + (double)re[a][b].c, (double)im[a][b].s + (double)im[a][b].c);
    }
}

// G[idx] = sum over z of partial[z][idx] in FP64: one block per entry.
__global__ void __launch_bounds__(XTHREADS) gram_x_reduce_kernel(const double2* __restrict__ partial, int nz, int na,
                                                                int nb, double* __restrict__ G) {
  __shared__ double red[2][XTHREADS / 32];
  const int idx = blockIdx.x;
  double re = 0.0, im = 0.0;
  for (int z = threadIdx.x; z < nz; z += XTHREADS) {
    const double2 p = partial[(size_t)z * na * nb + idx];
    re += p.x;
    im += p.y;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = re;
    red[1][threadIdx.x >> 5] = im;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    re = im = 0.0;
    for (int w = 0; w < XTHREADS / 32; ++w) {
      re += red[0][w];
      im += red[1][w];
    }
    G[2 * idx] = re;
    G[2 * idx + 1] = im;
  }
}

struct XScratch {
  std::mutex mu;
  void* partial[64] = {nullptr};
  size_t bytes[64] = {0};
};
XScratch& xscratch() {
  static XScratch s;
  return s;
}

}  // namespace

namespace {
// per-device partial-sum scratch of at least `bytes`
cudaError_t x_partials(size_t bytes, double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  XScratch& sc = xscratch();
  std::lock_guard<std::mutex> lock(sc.mu);
  if (bytes > sc.bytes[dev]) {
    if (sc.partial[dev]) {
      if ((e = cudaDeviceSynchronize()) != cudaSuccess) return e;
      cudaFree(sc.partial[dev]);
    }
    sc.partial[dev] = nullptr;
    sc.bytes[dev] = 0;
    if ((e = cudaMalloc(&sc.partial[dev], bytes)) != cudaSuccess) return e;
    sc.bytes[dev] = bytes;
  }
  *out = static_cast<double2*>(sc.partial[dev]);
  return cudaSuccess;
}
}  // namespace

cudaError_t launch_gram_dd(const void* A, int na, const void* B, int nb, size_t L, double* G, cudaStream_t s) {
  if (na < 1 || nb < 1 || !A || !B) return cudaErrorInvalidValue;
  if (L == 0) return cudaMemsetAsync(G, 0, sizeof(double) * 2 * (size_t)na * nb, s);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int T = (na <= 16 && nb <= 16) ? 16 : 32;
  const unsigned gx = (na + T - 1) / T, gy = (nb + T - 1) / T;
  size_t want = (size_t)8 * sms / (gx * gy);   // short double-float chains
  if (want < 1) want = 1;
  size_t rows = (L + want - 1) / want;
  rows = ((rows + XL - 1) / XL) * XL;
  const unsigned gz = (unsigned)((L + rows - 1) / rows);
  double2* partial = nullptr;
  if ((e = x_partials((size_t)gz * na * nb * sizeof(double2), &partial)) != cudaSuccess) return e;
  const dim3 grid(gx, gy, gz);
  if (T == 16)
    gram_dd_kernel<16><<<grid, XTHREADS, 0, s>>>(static_cast<const double2*>(A), na, static_cast<const double2*>(B), nb,
                                                 L, rows, partial);
  else
    gram_dd_kernel<32><<<grid, XTHREADS, 0, s>>>(static_cast<const double2*>(A), na, static_cast<const double2*>(B), nb,
                                                 L, rows, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  gram_x_reduce_kernel<<<(unsigned)(na * nb), XTHREADS, 0, s>>>(partial, (int)gz, na, nb, G);
  return cudaGetLastError();
}

cudaError_t launch_gram_x(const void* A1, int na1, const void* A2, int na2, const void* B, int nb, size_t L,
                          double* G, cudaStream_t s) {
  const int na = na1 + na2;
  if (na1 < 0 || na2 < 0 || na < 1 || nb < 1 || (na2 > 0 && !A2) || (na1 > 0 && !A1)) return cudaErrorInvalidValue;
  if (L == 0) return cudaMemsetAsync(G, 0, sizeof(double) * 2 * (size_t)na * nb, s);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const int TA = na <= 16 ? 16 : 32;
  const unsigned gx = (na + TA - 1) / TA, gy = (nb + XT - 1) / XT;
  // one resident wave: 4 CTAs of 256 threads per SM
  size_t want = (size_t)4 * sms / (gx * gy);
  if (want < 1) want = 1;
  size_t rows = (L + want - 1) / want;
  rows = ((rows + XL - 1) / XL) * XL;
  const unsigned gz = (unsigned)((L + rows - 1) / rows);
  double2* partial = nullptr;
  if ((e = x_partials((size_t)gz * na * nb * sizeof(double2), &partial)) != cudaSuccess) return e;
  const dim3 grid(gx, gy, gz);
  if (TA == 16)
    gram_x_kernel<16><<<grid, XTHREADS, 0, s>>>(static_cast<const double2*>(A1), na1, static_cast<const double2*>(A2),
                                                na, static_cast<const float2*>(B), nb, L, rows, partial);
  else
    gram_x_kernel<32><<<grid, XTHREADS, 0, s>>>(static_cast<const double2*>(A1), na1, static_cast<const double2*>(A2),
                                                na, static_cast<const float2*>(B), nb, L, rows, partial);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  gram_x_reduce_kernel<<<(unsigned)(na * nb), XTHREADS, 0, s>>>(partial, (int)gz, na, nb, G);
  return cudaGetLastError();
}

}  // namespace pcx
