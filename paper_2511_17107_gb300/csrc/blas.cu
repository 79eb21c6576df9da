// Block kernels of the Rayleigh-Ritz eigensolver (Sec. 4: LOBPCG): Gram
// products of tall-skinny blocks, the tall x small update, residuals and
// their norms (eq. exp_relativeresidual), random initial blocks and the
// k = 0 deflation of the constant fields (Prop. 2.5).
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cstdint>

#include "cx.cuh"
#include "dfloat.cuh"
#include "pcx_internal.h"

namespace pcx {
namespace {

// ---------------------------------------------------------------------------
// Gram: G[i][j] = sum_l conj(A_i[l]) B_j[l], FP64 output.
// CTA tile: 32 x 32 outputs, 256 threads each owning a 2 x 2 output block.
// The row range [l0, l1) of one CTA is walked in chunks of GL rows staged in
// shared memory; products accumulate in T within a chunk and in FP64 across
// chunks; CTA partials are added to G with FP64 atomics.
// ---------------------------------------------------------------------------
constexpr int GT = 32;
constexpr int GL = 32;
// Default complex64 Gram path by shape, from CUDA-event timings of both
// kernels at L = 3 * 128^3 on GB300 (ms, tensor cores / FP32 pipes):
// 16x16 0.73 / 0.52, 16x32 1.46 / 0.84, 16x48 1.88 / 1.25, 32x48 2.12 / 2.06,
// 48x48 2.37 / 3.65; A^H A: 16 0.76 / 0.34, 32 0.91 / 0.86, 48 1.11 / 2.21.
// The FMA count grows with na nb while the tensor-core kernel's cost is
// dominated by its per-element hi/lo conversion, so small products go to the
// FP32 pipes.
bool gram_fp32_pipes_faster(bool herm, int na, int nb) { return herm ? na <= 32 : na * nb <= 32 * 48; }

template <typename T>
__global__ void __launch_bounds__(256) gram_kernel(const cx<T>* __restrict__ A, int na, const cx<T>* __restrict__ B,
                                                   int nb, size_t L, size_t rows_per_cta, double* __restrict__ G) {
  __shared__ cx<T> sa[GL][GT + 1];
  __shared__ cx<T> sb[GL][GT + 1];
  const int ti = blockIdx.x * GT, tj = blockIdx.y * GT;
  const size_t l0 = (size_t)blockIdx.z * rows_per_cta;
  const size_t l1 = (l0 + rows_per_cta < L) ? l0 + rows_per_cta : L;
  const int tx = threadIdx.x % 16, ty = threadIdx.x / 16;   // output block (2ty.., 2tx..)
  double acc[2][2][2] = {};
  for (size_t base = l0; base < l1; base += GL) {
    // stage GL rows of 32 columns of A and B (row index fastest across threads)
    for (int e = threadIdx.x; e < GL * GT; e += 256) {
      const int r = e % GL, col = e / GL;
      const size_t l = base + r;
      const bool ok = l < l1;
      sa[r][col] = (ok && ti + col < na) ? A[(size_t)(ti + col) * L + l] : mk((T)0, (T)0);
      sb[r][col] = (ok && tj + col < nb) ? B[(size_t)(tj + col) * L + l] : mk((T)0, (T)0);
    }
    __syncthreads();
    cx<T> part[2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) part[a][b] = mk((T)0, (T)0);
#pragma unroll 8
    for (int r = 0; r < GL; ++r) {
      cx<T> av[2] = {sa[r][2 * ty], sa[r][2 * ty + 1]};
      cx<T> bv[2] = {sb[r][2 * tx], sb[r][2 * tx + 1]};
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b) part[a][b] = cfma_conj(av[a], bv[b], part[a][b]);
    }
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b) {
        acc[a][b][0] += (double)part[a][b].x;
        acc[a][b][1] += (double)part[a][b].y;
      }
    __syncthreads();
  }
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      const int i = ti + 2 * ty + a, j = tj + 2 * tx + b;
      if (i < na && j < nb) {
        atomicAdd(&G[2 * ((size_t)i * nb + j)], acc[a][b][0]);
        atomicAdd(&G[2 * ((size_t)i * nb + j) + 1], acc[a][b][1]);
      }
    }
}

// ---------------------------------------------------------------------------
// Double-float arithmetic on the FP32 pipes (GB300's FP64 rate is a small
// fraction of its FP32 rate) for the complex128 combinations: every FP64
// entry is split into FP32 hi + lo (about 48 significant bits); each real
// product x*y is formed as hi*hi exactly (TwoProd with an FMA) plus the cross
// terms, and accumulated in a double-float pair (Knuth's TwoSum), both
// error-free transformations of Dekker (1971) and Knuth (TAOCP vol. 2).
// __fadd_rn / __fmul_rn keep the compiler from fusing the steps.  Entries
// must stay inside the FP32 exponent range.  (The complex128 Gram products
// use the same scheme in gram_x.cu.)
// ---------------------------------------------------------------------------
using dfloat::DF;

// ---------------------------------------------------------------------------
// Combine: Y_j = sum_i S_i C[i][j] (+ beta Y_j), one row per thread, up to
// CY output columns per sweep; C staged in shared memory in T.
// ---------------------------------------------------------------------------
constexpr int CY = 16;

template <typename T>
__global__ void __launch_bounds__(256) combine_kernel(const cx<T>* __restrict__ S, int ns, const double* __restrict__ Cm,
                                                      int ny, int j0, double beta, cx<T>* __restrict__ Y, size_t L) {
  extern __shared__ __align__(16) unsigned char csm[];
  cx<T>* c = reinterpret_cast<cx<T>*>(csm);   // [ns][CY]
  const int nyl = (ny - j0 < CY) ? ny - j0 : CY;
  for (int e = threadIdx.x; e < ns * CY; e += blockDim.x) {
    const int i = e / CY, j = e % CY;
    c[e] = (j < nyl) ? mk((T)Cm[2 * ((size_t)i * ny + j0 + j)], (T)Cm[2 * ((size_t)i * ny + j0 + j) + 1])
                     : mk((T)0, (T)0);
  }
  __syncthreads();
  for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (size_t)gridDim.x * blockDim.x) {
    cx<T> acc[CY];
#pragma unroll
    for (int j = 0; j < CY; ++j) acc[j] = mk((T)0, (T)0);
    for (int i = 0; i < ns; ++i) {
      const cx<T> sv = S[(size_t)i * L + l];
#pragma unroll
      for (int j = 0; j < CY; ++j) acc[j] = cfma(sv, c[i * CY + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < CY; ++j) {
      if (j < nyl) {
        cx<T>* yp = Y + (size_t)(j0 + j) * L + l;
        cx<T> r = acc[j];
        if (beta != 0.0) r = r + scale(*yp, (T)beta);
        *yp = r;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Combine of complex64 columns with even L and 16-byte aligned columns: two
// rows l per thread (one 16-byte load of S_i per thread and i) and the
// coefficient pair (c_j, c_j+1) as one 16-byte shared load, so that each
// shared load feeds 16 FMAs (a shared load per 4 FMAs would saturate the
// shared-memory pipe before the FMA pipes).  ADD64: Y is complex128 and the
// FP32 sums are added to it (combine_add32); otherwise Y = sum (+ beta Y).
// ---------------------------------------------------------------------------
template <bool ADD64>
__global__ void __launch_bounds__(256) combine2_kernel(const float4* __restrict__ S, int ns,
                                                       const double* __restrict__ Cm, int ny, int j0, double beta,
                                                       void* __restrict__ Yv, size_t L2) {
  constexpr int CP = CY / 2;
  extern __shared__ __align__(16) unsigned char csm[];
  float4* c = reinterpret_cast<float4*>(csm);   // [ns][CP]: (c_j, c_j+1) of column pair jp
  const int nyl = (ny - j0 < CY) ? ny - j0 : CY;
  for (int e = threadIdx.x; e < ns * CP; e += blockDim.x) {
    const int i = e / CP, j = 2 * (e % CP);
    const double* ci = Cm + 2 * ((size_t)i * ny + j0 + j);
    float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
    if (j < nyl) {
      v.x = (float)ci[0];
      v.y = (float)ci[1];
    }
    if (j + 1 < nyl) {
      v.z = (float)ci[2];
      v.w = (float)ci[3];
    }
    c[e] = v;
  }
  __syncthreads();
  const float fb = (float)beta;
  for (size_t f = (size_t)blockIdx.x * blockDim.x + threadIdx.x; f < L2; f += (size_t)gridDim.x * blockDim.x) {
    float2 a0[CY], a1[CY];   // rows 2f and 2f + 1
#pragma unroll
    for (int j = 0; j < CY; ++j) a0[j] = a1[j] = make_float2(0.f, 0.f);
    // the loads of PF columns are issued before their products, so that
    // every thread keeps several 16-byte loads in flight
    constexpr int PF = 4;
    for (int i0 = 0; i0 < ns; i0 += PF) {
      float4 sv[PF];
#pragma unroll
      for (int u = 0; u < PF; ++u)
        sv[u] = i0 + u < ns ? S[(size_t)(i0 + u) * L2 + f] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < PF; ++u) {
        if (i0 + u >= ns) break;
        const float4* ci = c + (i0 + u) * CP;
#pragma unroll
        for (int jp = 0; jp < CP; ++jp) {
          const float4 cc = ci[jp];
          const float4 v = sv[u];
          // (s.re + i s.im)(c.re + i c.im) for the two rows and c_j, c_j+1
          a0[2 * jp].x = fmaf(-v.y, cc.y, fmaf(v.x, cc.x, a0[2 * jp].x));
          a0[2 * jp].y = fmaf(v.y, cc.x, fmaf(v.x, cc.y, a0[2 * jp].y));
          a1[2 * jp].x = fmaf(-v.w, cc.y, fmaf(v.z, cc.x, a1[2 * jp].x));
          a1[2 * jp].y = fmaf(v.w, cc.x, fmaf(v.z, cc.y, a1[2 * jp].y));
          a0[2 * jp + 1].x = fmaf(-v.y, cc.w, fmaf(v.x, cc.z, a0[2 * jp + 1].x));
          a0[2 * jp + 1].y = fmaf(v.y, cc.z, fmaf(v.x, cc.w, a0[2 * jp + 1].y));
          a1[2 * jp + 1].x = fmaf(-v.w, cc.w, fmaf(v.z, cc.z, a1[2 * jp + 1].x));
          a1[2 * jp + 1].y = fmaf(v.w, cc.z, fmaf(v.z, cc.w, a1[2 * jp + 1].y));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < CY; ++j) {
      if (j < nyl) {
        if constexpr (ADD64) {
          double2* yp = static_cast<double2*>(Yv) + (size_t)(j0 + j) * 2 * L2 + 2 * f;
          double2 y0 = yp[0], y1 = yp[1];
          y0.x += (double)a0[j].x;
          y0.y += (double)a0[j].y;
          y1.x += (double)a1[j].x;
          y1.y += (double)a1[j].y;
          yp[0] = y0;
          yp[1] = y1;
        } else {
          float4* yp = static_cast<float4*>(Yv) + (size_t)(j0 + j) * L2 + f;
          float4 r = make_float4(a0[j].x, a0[j].y, a1[j].x, a1[j].y);
          if (beta != 0.0) {
            const float4 o = *yp;
            r.x = fmaf(fb, o.x, r.x);
            r.y = fmaf(fb, o.y, r.y);
            r.z = fmaf(fb, o.z, r.z);
            r.w = fmaf(fb, o.w, r.w);
          }
          *yp = r;
        }
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Combine for complex128 on the FP32 pipes with FP64-level accuracy: the
// same split / TwoProd / TwoSum scheme as gram_ff_kernel.  Each row's inputs
// are split once and reused for the CY outputs of the sweep; C is split once
// per CTA into shared memory.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(128) combine_ff_kernel(const double2* __restrict__ S, int ns,
                                                         const double* __restrict__ Cm, int ny, int j0, double beta,
                                                         double2* __restrict__ Y, size_t L) {
  extern __shared__ __align__(16) unsigned char csm[];
  float4* c = reinterpret_cast<float4*>(csm);   // [ns][CY]: (re hi, re lo, im hi, im lo)
  const int nyl = (ny - j0 < CY) ? ny - j0 : CY;
  for (int e = threadIdx.x; e < ns * CY; e += blockDim.x) {
    const int i = e / CY, j = e % CY;
    float4 v = make_float4(0, 0, 0, 0);
    if (j < nyl) {
      const double re = Cm[2 * ((size_t)i * ny + j0 + j)], im = Cm[2 * ((size_t)i * ny + j0 + j) + 1];
      dfloat::split(re, v.x, v.y);
      dfloat::split(im, v.z, v.w);
    }
    c[e] = v;
  }
  __syncthreads();
  for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (size_t)gridDim.x * blockDim.x) {
    DF re[CY], im[CY];
#pragma unroll
    for (int j = 0; j < CY; ++j) re[j] = im[j] = DF{0.f, 0.f};
    for (int i = 0; i < ns; ++i) {
      const double2 sv = S[(size_t)i * L + l];
      float sr, srl, si, sil;   // integer splits: no FP64 instruction in the loop
      dfloat::split(sv.x, sr, srl);
      dfloat::split(sv.y, si, sil);
#pragma unroll
      for (int j = 0; j < CY; ++j) {
        const float4 cv = c[i * CY + j];
        // s c: re = sr cr - si ci, im = sr ci + si cr
        dfloat::mac2<false>(re[j], sr, srl, cv.x, cv.y);
        dfloat::mac2<true>(re[j], si, sil, cv.z, cv.w);
        dfloat::mac2<false>(im[j], sr, srl, cv.z, cv.w);
        dfloat::mac2<false>(im[j], si, sil, cv.x, cv.y);
      }
    }
#pragma unroll
    for (int j = 0; j < CY; ++j) {
      if (j < nyl) {
        double2* yp = Y + (size_t)(j0 + j) * L + l;
        double2 r = make_double2((double)re[j].s + (double)re[j].c, (double)im[j].s + (double)im[j].c);
        if (beta != 0.0) {
          const double2 y0 = *yp;
          r.x += beta * y0.x;
          r.y += beta * y0.y;
        }
        *yp = r;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Y64_j += sum_i S32_i C[i][j]: a combination of complex64 columns evaluated
// in FP32 and added into complex128 columns (the small correction part of a
// mixed-precision update).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) combine_add32_kernel(const cx<float>* __restrict__ S, int ns,
                                                            const double* __restrict__ Cm, int ny, int j0,
                                                            double2* __restrict__ Y, size_t L) {
  extern __shared__ __align__(16) unsigned char csm[];
  cx<float>* c = reinterpret_cast<cx<float>*>(csm);
  const int nyl = (ny - j0 < CY) ? ny - j0 : CY;
  for (int e = threadIdx.x; e < ns * CY; e += blockDim.x) {
    const int i = e / CY, j = e % CY;
    c[e] = (j < nyl) ? mk((float)Cm[2 * ((size_t)i * ny + j0 + j)], (float)Cm[2 * ((size_t)i * ny + j0 + j) + 1])
                     : mk(0.f, 0.f);
  }
  __syncthreads();
  for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (size_t)gridDim.x * blockDim.x) {
    cx<float> acc[CY];
#pragma unroll
    for (int j = 0; j < CY; ++j) acc[j] = mk(0.f, 0.f);
    for (int i = 0; i < ns; ++i) {
      const cx<float> sv = S[(size_t)i * L + l];
#pragma unroll
      for (int j = 0; j < CY; ++j) acc[j] = cfma(sv, c[i * CY + j], acc[j]);
    }
#pragma unroll
    for (int j = 0; j < CY; ++j) {
      if (j < nyl) {
        double2* yp = Y + (size_t)(j0 + j) * L + l;
        double2 y = *yp;
        y.x += (double)acc[j].x;
        y.y += (double)acc[j].y;
        *yp = y;
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Residual R_j = AX_j - theta_j X_j with ||R_j||^2 and ||X_j||^2 (FP64).
// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(256) residual_kernel(const cx<T>* __restrict__ X, const cx<T>* AX, const double* theta,
                                                       cx<T>* R, double* norms, int nvec, size_t L) {
  const int j = blockIdx.y;
  const T th = (T)theta[j];
  double rr = 0.0, xx = 0.0;
  const cx<T>* x = X + (size_t)j * L;
  const cx<T>* ax = AX + (size_t)j * L;
  cx<T>* r = R + (size_t)j * L;
  for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (size_t)gridDim.x * blockDim.x) {
    const cx<T> xv = x[l], av = ax[l];
    const cx<T> rv = mk(fma(-th, xv.x, av.x), fma(-th, xv.y, av.y));
    r[l] = rv;
    rr += (double)norm2(rv);
    xx += (double)norm2(xv);
  }
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    xx += __shfl_down_sync(0xffffffffu, xx, o);
  }
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  if (lane == 0) {
    red[0][wid] = rr;
    red[1][wid] = xx;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x / 32;
    rr = lane < nw ? red[0][lane] : 0.0;
    xx = lane < nw ? red[1][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      rr += __shfl_down_sync(0xffffffffu, rr, o);
      xx += __shfl_down_sync(0xffffffffu, xx, o);
    }
    if (lane == 0) {
      atomicAdd(&norms[j], rr);
      atomicAdd(&norms[nvec + j], xx);
    }
  }
}

// ---------------------------------------------------------------------------
// The residual of the mixed-precision refinement, R_j = AX_j - theta_j X_j,
// from the FP64 X and AX, stored rounded to complex64, with X_j rounded to
// complex64 alongside and ||R_j||^2, ||X_j||^2 summed from the rounded
// values (FP32 within a thread, FP64 across threads).  The difference is
// formed in double-float on the FP32 pipes: every FP64 operand split into
// FP32 hi + lo, theta x as TwoProd of the hi parts plus the cross terms,
// ax - theta x by TwoSum (Knuth), about 2^-48 of |ax| before the final
// rounding to FP32, the same as FP64 for a result stored in FP32 (GB300's
// FP64 pipes made the FP64 form three times slower than the memory traffic).
// ---------------------------------------------------------------------------
__device__ __forceinline__ float dd_residual(float ah, float al, float th, float tl, float xh, float xl) {
  const float p = __fmul_rn(th, xh);
  float e = fmaf(th, xh, -p);   // p + e == th * xh exactly
  e = fmaf(th, xl, e);
  e = fmaf(tl, xh, e);
  const float sm = __fsub_rn(ah, p);   // TwoSum(ah, -p)
  const float bb = __fsub_rn(sm, ah);
  const float err = __fadd_rn(__fsub_rn(ah, __fsub_rn(sm, bb)), __fsub_rn(-p, bb));
  const float lo = __fadd_rn(__fsub_rn(al, e), err);
  return __fadd_rn(sm, lo);
}

__global__ void __launch_bounds__(256) residual_mixed_kernel(const double2* __restrict__ X, const double2* AX,
                                                             const double* theta, float2* R32, float2* X32,
                                                             double* norms, int nvec, size_t L) {
  const int j = blockIdx.y;
  float th, tl;
  dfloat::split(theta[j], th, tl);
  float rrf = 0.f, xxf = 0.f;
  const double2* x = X + (size_t)j * L;
  const double2* ax = AX + (size_t)j * L;
  float2* r = R32 + (size_t)j * L;
  float2* x32 = X32 + (size_t)j * L;
  for (size_t l = (size_t)blockIdx.x * blockDim.x + threadIdx.x; l < L; l += (size_t)gridDim.x * blockDim.x) {
    const double2 xv = x[l], av = ax[l];
    float xh, xl, yh, yl, ah, al, bh, bl;
    dfloat::split(xv.x, xh, xl);
    dfloat::split(xv.y, yh, yl);
    dfloat::split(av.x, ah, al);
    dfloat::split(av.y, bh, bl);
    const float rx = dd_residual(ah, al, th, tl, xh, xl), ry = dd_residual(bh, bl, th, tl, yh, yl);
    const float x0 = __fadd_rn(xh, xl), x1 = __fadd_rn(yh, yl);
    r[l] = make_float2(rx, ry);
    x32[l] = make_float2(x0, x1);
    rrf = fmaf(rx, rx, fmaf(ry, ry, rrf));
    xxf = fmaf(x0, x0, fmaf(x1, x1, xxf));
  }
  double rr = rrf, xx = xxf;
  __shared__ double red[2][32];
  for (int o = 16; o > 0; o >>= 1) {
    rr += __shfl_down_sync(0xffffffffu, rr, o);
    xx += __shfl_down_sync(0xffffffffu, xx, o);
  }
  const int lane = threadIdx.x % 32, wid = threadIdx.x / 32;
  if (lane == 0) {
    red[0][wid] = rr;
    red[1][wid] = xx;
  }
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x / 32;
    rr = lane < nw ? red[0][lane] : 0.0;
    xx = lane < nw ? red[1][lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      rr += __shfl_down_sync(0xffffffffu, rr, o);
      xx += __shfl_down_sync(0xffffffffu, xx, o);
    }
    if (lane == 0) {
      atomicAdd(&norms[j], rr);
      atomicAdd(&norms[nvec + j], xx);
    }
  }
}

// ---------------------------------------------------------------------------
// Seeded complex Gaussian fill: SplitMix64 hash of (seed, index) -> two
// uniforms -> Box-Muller (uses the CUDA math library's log, sqrt, sincos).
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix(uint64_t z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void fill_random_kernel(cx<T>* X, size_t total, uint64_t seed) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const uint64_t h1 = splitmix(seed ^ splitmix(2 * e)), h2 = splitmix(seed ^ splitmix(2 * e + 1));
    const double u1 = ((h1 >> 11) + 1) * (1.0 / 9007199254740993.0);   // (0, 1]
    const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    X[e] = mk((T)(rad * cs), (T)(rad * sn));
  }
}

template <typename T>
__global__ void deflate_kernel(cx<T>* X, int nvec, size_t n3) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < 3 * nvec) X[(size_t)i * n3] = mk((T)0, (T)0);   // mode p = 0 of component i % 3 of vector i / 3
}

template <typename S, typename D>
__global__ void convert_kernel(const S* __restrict__ src, D* __restrict__ dst, size_t count) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < count; e += (size_t)gridDim.x * blockDim.x)
    dst[e] = (D)src[e];
}

// columns of even length starting on 16-byte boundaries (pairs of complex64
// entries load as one float4)
bool pair_ok(const void* S, const void* Y, size_t L) {
  return L % 2 == 0 && (reinterpret_cast<uintptr_t>(S) & 15) == 0 && (reinterpret_cast<uintptr_t>(Y) & 15) == 0;
}

unsigned grid_for(size_t work, int threads, unsigned cap = 152u * 32u) {
  return (unsigned)std::max<size_t>(1, std::min<size_t>((work + threads - 1) / threads, cap));
}

}  // namespace

namespace {
std::atomic<int> g_gram_path{0};
}  // namespace

void set_gram_path(int path) { g_gram_path.store(path); }
int get_gram_path() { return g_gram_path.load(); }

cudaError_t launch_gram(const void* A, int na, const void* B, int nb, size_t L, int precision, double* G,
                        cudaStream_t s) {
  if (precision == PCX_FP64) return launch_gram_dd(A, na, B, nb, L, G, s);   // gram_x.cu
  const int path = g_gram_path.load();
  const bool cc = L > 0 && gram_cc_supported(A, B, na, nb, L);
  const bool tc = L > 0 && gram_tc_supported(na, nb, L);
  if (cc && (path == 2 || (path == 0 && gram_fp32_pipes_faster(A == B && na == nb, na, nb))))
    return launch_gram_cc(A, na, B, nb, L, G, s);
  if (tc && path != 2) return launch_gram_tc(A, na, B, nb, L, G, s);
  if (cc) return launch_gram_cc(A, na, B, nb, L, G, s);
  return launch_gram_cuda_cores(A, na, B, nb, L, precision, G, s);
}

cudaError_t launch_gram_cuda_cores(const void* A, int na, const void* B, int nb, size_t L, int precision, double* G,
                                   cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(G, 0, sizeof(double) * 2 * (size_t)na * nb, s);
  if (e != cudaSuccess) return e;
  if (L == 0) return cudaSuccess;
  if (precision == PCX_FP64) return launch_gram_dd(A, na, B, nb, L, G, s);
  const int tile = GT;
  const int rows_step = GL;
  const unsigned gx = (na + tile - 1) / tile, gy = (nb + tile - 1) / tile;
  // enough CTAs to fill the GPU several times over
  const size_t want = std::max<size_t>(1, (size_t)152 * 8 / (gx * gy));
  size_t rows = (L + want - 1) / want;
  rows = ((rows + rows_step - 1) / rows_step) * rows_step;
  const unsigned gz = (unsigned)((L + rows - 1) / rows);
  dim3 grid(gx, gy, gz);
  gram_kernel<float><<<grid, 256, 0, s>>>(static_cast<const cx<float>*>(A), na, static_cast<const cx<float>*>(B), nb,
                                          L, rows, G);
  return cudaGetLastError();
}

cudaError_t launch_combine(const void* S, int ns, const double* C, int ny, double beta, void* Y, size_t L,
                           int precision, cudaStream_t s) {
  if (L == 0) return cudaSuccess;
  const int threads = 256;
  const unsigned blocks = grid_for(L, threads, 152u * 8u);
  for (int j0 = 0; j0 < ny; j0 += CY) {
    if (precision == PCX_FP64) {
      const size_t smem = (size_t)ns * CY * sizeof(float4);
      if (smem > 48 * 1024) {
        cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(combine_ff_kernel), smem);
        if (e != cudaSuccess) return e;
      }
      combine_ff_kernel<<<grid_for(L, 128, 152u * 16u), 128, smem, s>>>(static_cast<const double2*>(S), ns, C, ny,
                                                                         j0, beta, static_cast<double2*>(Y), L);
    } else if (pair_ok(S, Y, L)) {
      const size_t smem = (size_t)ns * CY * sizeof(cx<float>);
      combine2_kernel<false><<<grid_for(L / 2, threads, 152u * 8u), threads, smem, s>>>(
          static_cast<const float4*>(S), ns, C, ny, j0, beta, Y, L / 2);
    } else {
      const size_t smem = (size_t)ns * CY * sizeof(cx<float>);
      combine_kernel<float><<<blocks, threads, smem, s>>>(static_cast<const cx<float>*>(S), ns, C, ny, j0, beta,
                                                          static_cast<cx<float>*>(Y), L);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_combine_add32(const void* S32, int ns, const double* C, int ny, void* Y64, size_t L,
                                cudaStream_t s) {
  if (L == 0) return cudaSuccess;
  const unsigned blocks = grid_for(L, 256, 152u * 8u);
  const bool pairs = pair_ok(S32, Y64, L);
  for (int j0 = 0; j0 < ny; j0 += CY) {
    const size_t smem = (size_t)ns * CY * sizeof(cx<float>);
    if (pairs)
      combine2_kernel<true><<<grid_for(L / 2, 256, 152u * 8u), 256, smem, s>>>(static_cast<const float4*>(S32), ns,
                                                                              C, ny, j0, 0.0, Y64, L / 2);
    else
      combine_add32_kernel<<<blocks, 256, smem, s>>>(static_cast<const cx<float>*>(S32), ns, C, ny, j0,
                                                     static_cast<double2*>(Y64), L);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_residual(const void* X, const void* AX, const double* theta, void* R, double* norms, int nvec,
                            size_t L, int precision, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 2 * nvec, s);
  if (e != cudaSuccess || nvec == 0) return e;
  dim3 grid(grid_for(L, 256, 152u * 4u), nvec);
  if (precision == PCX_FP64)
    residual_kernel<double><<<grid, 256, 0, s>>>(static_cast<const cx<double>*>(X), static_cast<const cx<double>*>(AX),
                                                 theta, static_cast<cx<double>*>(R), norms, nvec, L);
  else
    residual_kernel<float><<<grid, 256, 0, s>>>(static_cast<const cx<float>*>(X), static_cast<const cx<float>*>(AX),
                                                theta, static_cast<cx<float>*>(R), norms, nvec, L);
  return cudaGetLastError();
}

cudaError_t launch_residual_mixed(const void* X, const void* AX, const double* theta, void* R32, void* X32,
                                  double* norms, int nvec, size_t L, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(norms, 0, sizeof(double) * 2 * nvec, s);
  if (e != cudaSuccess || nvec == 0) return e;
  dim3 grid(grid_for(L, 256, 152u * 4u), nvec);
  residual_mixed_kernel<<<grid, 256, 0, s>>>(static_cast<const double2*>(X), static_cast<const double2*>(AX), theta,
                                             static_cast<float2*>(R32), static_cast<float2*>(X32), norms, nvec, L);
  return cudaGetLastError();
}

cudaError_t launch_fill_random(void* X, int nvec, size_t L, uint64_t seed, int precision, cudaStream_t s) {
  const size_t total = (size_t)nvec * L;
  if (total == 0) return cudaSuccess;
  if (precision == PCX_FP64)
    fill_random_kernel<double><<<grid_for(total, 256), 256, 0, s>>>(static_cast<cx<double>*>(X), total, seed);
  else
    fill_random_kernel<float><<<grid_for(total, 256), 256, 0, s>>>(static_cast<cx<float>*>(X), total, seed);
  return cudaGetLastError();
}

cudaError_t launch_deflate_p0(void* X, int nvec, int n, int precision, cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t n3 = (size_t)n * n * n;
  const unsigned blocks = (3 * nvec + 127) / 128;
  if (precision == PCX_FP64)
    deflate_kernel<double><<<blocks, 128, 0, s>>>(static_cast<cx<double>*>(X), nvec, n3);
  else
    deflate_kernel<float><<<blocks, 128, 0, s>>>(static_cast<cx<float>*>(X), nvec, n3);
  return cudaGetLastError();
}

cudaError_t launch_convert(const void* src, int src_prec, void* dst, int dst_prec, size_t count, cudaStream_t s) {
  // count = number of complex entries
  const size_t reals = 2 * count;
  if (reals == 0) return cudaSuccess;
  const unsigned blocks = grid_for(reals, 256);
  if (src_prec == PCX_FP32 && dst_prec == PCX_FP64)
    convert_kernel<float, double><<<blocks, 256, 0, s>>>(static_cast<const float*>(src), static_cast<double*>(dst), reals);
  else if (src_prec == PCX_FP64 && dst_prec == PCX_FP32)
    convert_kernel<double, float><<<blocks, 256, 0, s>>>(static_cast<const double*>(src), static_cast<float*>(dst), reals);
  else
    return cudaMemcpyAsync(dst, src, reals * (src_prec == PCX_FP64 ? 8 : 4), cudaMemcpyDeviceToDevice, s);
  return cudaGetLastError();
}

}  // namespace pcx
