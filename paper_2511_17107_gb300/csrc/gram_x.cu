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

#include "dfloat.cuh"
#include "pcx_internal.h"
#include "stream_scratch.h"

namespace pcx {
namespace {

constexpr int XT = 32;        // tile: 32 rows of A x 32 columns of B
constexpr int XL = 32;        // vector entries staged per step
constexpr int XTHREADS = 256; // 16 x 16 threads, 2 x 2 outputs each

using dfloat::DF;
using dfloat::split;

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
        split(v.x, av.x, av.y);
        split(v.y, av.z, av.w);
      }
      if (ok && tj + col < nb) {
        const double2 v = B[(size_t)(tj + col) * L + l];
        split(v.x, bv.x, bv.y);
        split(v.y, bv.z, bv.w);
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
          dfloat::mac2<false>(re[a][b], ar[a].x, ar[a].y, br[b].x, br[b].y);
          dfloat::mac2<false>(re[a][b], ar[a].z, ar[a].w, br[b].z, br[b].w);
          dfloat::mac2<false>(im[a][b], ar[a].x, ar[a].y, br[b].z, br[b].w);
          dfloat::mac2<true>(im[a][b], ar[a].z, ar[a].w, br[b].x, br[b].y);
        }
    }
#pragma unroll
    for (int a = 0; a < O; ++a)
#pragma unroll
      for (int b = 0; b < O; ++b) {
        dfloat::renorm(re[a][b]);
        dfloat::renorm(im[a][b]);
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
        split(v.x, av.x, av.y);
        split(v.y, av.z, av.w);
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
          dfloat::mac1<false>(re[a][b], av.x, av.y, bv.x);
          dfloat::mac1<false>(re[a][b], av.z, av.w, bv.y);
          dfloat::mac1<false>(im[a][b], av.x, av.y, bv.y);
          dfloat::mac1<true>(im[a][b], av.z, av.w, bv.x);
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

// partial sums, one buffer per (device, stream)
StreamScratch& xscratch() {
  static StreamScratch s;
  return s;
}

}  // namespace

namespace {
// partial-sum scratch of at least `bytes` for work on stream s
cudaError_t x_partials(size_t bytes, double2** out, cudaStream_t s) {
  void* p = nullptr;
  cudaError_t e = xscratch().get(s, bytes, &p);
  *out = static_cast<double2*>(p);
  return e;
}
}  // namespace

cudaError_t launch_gram_dd(const void* A, int na, const void* B, int nb, size_t L, double* G, cudaStream_t s) {
  if (na < 1 || nb < 1 || !A || !B) return cudaErrorInvalidValue;
  if (L == 0) return cudaMemsetAsync(G, 0, sizeof(double) * 2 * (size_t)na * nb, s);
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  // tiles of 32 x 32 where both sizes are multiples of 32, else 16 x 16
  // (48 x 48: 9 tiles of 16 against 4 of 32 that pad 48 to 64)
  const int T = (na % 32 == 0 && nb % 32 == 0) ? 32 : 16;
  const unsigned gx = (na + T - 1) / T, gy = (nb + T - 1) / T;
  size_t want = (size_t)8 * sms / (gx * gy);   // short double-float chains
  if (want < 1) want = 1;
  size_t rows = (L + want - 1) / want;
  rows = ((rows + XL - 1) / XL) * XL;
  const unsigned gz = (unsigned)((L + rows - 1) / rows);
  double2* partial = nullptr;
  if ((e = x_partials((size_t)gz * na * nb * sizeof(double2), &partial, s)) != cudaSuccess) return e;
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
  if ((e = x_partials((size_t)gz * na * nb * sizeof(double2), &partial, s)) != cudaSuccess) return e;
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

void gram_x_release_stream(cudaStream_t s) { xscratch().release(s); }

}  // namespace pcx
