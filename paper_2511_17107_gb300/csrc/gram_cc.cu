// Gram products G = A^H B of complex64 column blocks on the FP32 pipes
// (Sec. 4, the Rayleigh-Ritz step of LOBPCG), for the skinny shapes of the
// eigensolver (na, nb <= 64 columns of L = 3 N^3 entries).
//
// At these shapes a contraction costs 4 na nb FP32 FMAs per row l against
// 8 (na + nb) bytes of operands: 16x16 and 16x32 products are bound by HBM,
// 48x48 ones by the FMA pipes at about half the HBM rate.  The tensor-core
// path (gram_tc.cu) must first split every FP32 operand into TF32 hi + lo
// and deinterleave re/im through shared memory, which costs more shared
// memory traffic than these FMAs; the dispatcher in blas.cu picks per shape.
//
// Layout: each CTA owns a contiguous range of rows l and streams it through
// shared memory in double-buffered stages of 32 or 64 rows (cp.async,
// 16-byte copies of two complex entries).  Thread (ti, tj) owns the TA x TB output
// entries (ti + a qa, tj + b qb), a < TA, b < TB, with qa = ceil(na / TA) and
// qb = ceil(nb / TB): rows at stride qa / qb, so that the lanes of a warp
// read distinct shared-memory banks.  Products are summed in FP32 over one
// stage and folded into a double-float (sum, compensation) pair per entry;
// each CTA writes its FP64 partial G, and a second kernel adds the partials
// of all CTAs in FP64 (deterministic).  For A^H A only the entries with
// a <= b are formed (the upper triangle; the sum kernel mirrors it).
#include <cuda_runtime.h>

#include <mutex>

#include "dfloat.cuh"
#include "pcx_internal.h"
#include "stream_scratch.h"

namespace pcx {
namespace {

constexpr int RED = 256;        // threads of the partial-sum kernel

// complex rows l per stage: 32 for 4 x 4 tiles (two CTAs of up to 96
// staged columns per SM), 64 for 2 x 2 tiles
template <int TA>
struct Stage {
  static constexpr int SL = TA >= 4 ? 32 : 64;
  static constexpr int SF = SL / 2;   // float4 (two complex entries) per row per stage
  static constexpr int RS = SF + 1;   // padded row stride in float4 (odd: conflict-free)
};

__device__ __forceinline__ void cp16(void* dst, const void* src, int bytes) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(d), "l"(src), "r"(bytes) : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// MAXT threads at most; MINB resident CTAs per SM asked of the register
// allocator (4 x 4 tiles of up to 48 x 48 entries: 160 threads, two CTAs,
// at most 168 registers so that three warps fit each scheduler's registers)
template <int TA, int TB, bool SYM, int MAXT, int MINB>
__global__ void __launch_bounds__(MAXT, MINB) gram_cc_kernel(const float4* __restrict__ A, int na,
                                                      const float4* __restrict__ B, int nb, long long L2,
                                                      long long per_cta, double2* __restrict__ part) {
  constexpr int SF = Stage<TA>::SF, RS = Stage<TA>::RS;
  extern __shared__ float4 sm[];
  const int qa = (na + TA - 1) / TA, qb = (nb + TB - 1) / TB;
  const int rows_a = qa * TA, rows_b = SYM ? 0 : qb * TB;
  const int nrow = rows_a + rows_b;
  float4* buf0 = sm;
  float4* buf1 = sm + (size_t)nrow * RS;
  const long long f0 = (long long)blockIdx.x * per_cta;
  const long long f1 = f0 + per_cta < L2 ? f0 + per_cta : L2;
  const int nst = f1 > f0 ? (int)((f1 - f0 + SF - 1) / SF) : 0;
  const int tid = threadIdx.x;
  const bool active = tid < qa * qb;
  const int ti = active ? tid / qb : 0, tj = active ? tid % qb : 0;

  auto load = [&](float4* s, long long fs) {
    for (int e = tid; e < nrow * SF; e += blockDim.x) {
      const int r = e / SF, f = e % SF;
      const long long g = fs + f;
      const float4* src = A;
      int bytes = 0;
      if (g < f1) {
        if (r < rows_a) {
          if (r < na) {
            src = A + (size_t)r * L2 + g;
            bytes = 16;
          }
        } else if (r - rows_a < nb) {
          src = B + (size_t)(r - rows_a) * L2 + g;
          bytes = 16;
        }
      }
      cp16(&s[r * RS + f], src, bytes);   // bytes = 0: zero fill
    }
    cp_commit();
  };

  dfloat::DF acc[TA][TB][2];
#pragma unroll
  for (int a = 0; a < TA; ++a)
#pragma unroll
    for (int b = 0; b < TB; ++b) acc[a][b][0] = acc[a][b][1] = dfloat::DF{0.f, 0.f};

  if (nst > 0) load(buf0, f0);
  for (int st = 0; st < nst; ++st) {
    float4* cur = (st & 1) ? buf1 : buf0;
    if (st + 1 < nst) {
      load((st & 1) ? buf0 : buf1, f0 + (long long)(st + 1) * SF);
      cp_wait<1>();
    } else {
      cp_wait<0>();
    }
    __syncthreads();
    if (active) {
      float pr[TA][TB], pi[TA][TB];
#pragma unroll
      for (int a = 0; a < TA; ++a)
#pragma unroll
        for (int b = 0; b < TB; ++b) pr[a][b] = pi[a][b] = 0.f;
      const float4* sa = cur + ti * RS;
      const float4* sb = cur + (SYM ? tj : rows_a + tj) * RS;
#pragma unroll 2
      for (int f = 0; f < SF; ++f) {
        float4 av[TA], bv[TB];
#pragma unroll
        for (int a = 0; a < TA; ++a) av[a] = sa[a * qa * RS + f];
#pragma unroll
        for (int b = 0; b < TB; ++b) bv[b] = sb[b * qb * RS + f];
#pragma unroll
        for (int a = 0; a < TA; ++a)
#pragma unroll
          for (int b = 0; b < TB; ++b) {
            if (SYM && a > b) continue;
            // conj(a) b over the two complex entries of the float4
            float r = pr[a][b], i = pi[a][b];
            r = fmaf(av[a].x, bv[b].x, r);
            r = fmaf(av[a].y, bv[b].y, r);
            r = fmaf(av[a].z, bv[b].z, r);
            r = fmaf(av[a].w, bv[b].w, r);
            i = fmaf(av[a].x, bv[b].y, i);
            i = fmaf(-av[a].y, bv[b].x, i);
            i = fmaf(av[a].z, bv[b].w, i);
            i = fmaf(-av[a].w, bv[b].z, i);
            pr[a][b] = r;
            pi[a][b] = i;
          }
      }
#pragma unroll
      for (int a = 0; a < TA; ++a)
#pragma unroll
        for (int b = 0; b < TB; ++b) {
          if (SYM && a > b) continue;
          dfloat::add(acc[a][b][0], pr[a][b], 0.f);
          dfloat::add(acc[a][b][1], pi[a][b], 0.f);
        }
    }
    __syncthreads();   // the buffer is refilled by the next iteration's load
  }
  if (!active) return;
  double2* p = part + (size_t)blockIdx.x * na * nb;
#pragma unroll
  for (int a = 0; a < TA; ++a)
#pragma unroll
    for (int b = 0; b < TB; ++b) {
      if (SYM && a > b) continue;
      const int i = ti + a * qa, j = tj + b * qb;
      if (i < na && j < nb && (!SYM || i <= j))
        p[i * nb + j] = make_double2((double)acc[a][b][0].s + (double)acc[a][b][0].c,
                                     (double)acc[a][b][1].s + (double)acc[a][b][1].c);
    }
}

// G[i][j] = sum over CTAs of the partials (FP64), one block per entry; for a
// Hermitian product the lower triangle is the conjugate of the upper one and
// the diagonal is real.
__global__ void __launch_bounds__(RED) gram_cc_sum_kernel(const double2* __restrict__ part, int nctas, int na, int nb,
                                                          int sym, double* __restrict__ G) {
  __shared__ double red[2][RED / 32];
  const int idx = blockIdx.x;
  int i = idx / nb, j = idx % nb;
  const bool mirror = sym && i > j;
  if (mirror) {
    const int t = i;
    i = j;
    j = t;
  }
  double re = 0.0, im = 0.0;
  for (int c = threadIdx.x; c < nctas; c += RED) {
    const double2 v = part[((size_t)c * na + i) * nb + j];
    re += v.x;
    im += v.y;
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
    for (int w = 0; w < RED / 32; ++w) {
      re += red[0][w];
      im += red[1][w];
    }
    G[2 * idx] = re;
    // the diagonal of A^H A is real (the FMA order leaves rounding residue)
    G[2 * idx + 1] = mirror ? -im : ((sym && i == j) ? 0.0 : im);
  }
}

// per-CTA partial sums, one buffer per (device, stream)
StreamScratch& scratch() {
  static StreamScratch s;
  return s;
}

template <int TA, int TB, bool SYM, int MAXT, int MINB>
cudaError_t run(const float4* A, int na, const float4* B, int nb, long long L2, int sms, double2* part_buf,
                size_t part_cap, double* G, cudaStream_t s, int* nctas_out) {
  const int qa = (na + TA - 1) / TA, qb = (nb + TB - 1) / TB;
  const int threads = ((qa * qb + 31) / 32) * 32;
  const int nrow = qa * TA + (SYM ? 0 : qb * TB);
  constexpr int SF = Stage<TA>::SF, RS = Stage<TA>::RS;
  const size_t smem = (size_t)2 * nrow * RS * sizeof(float4);
  auto kern = gram_cc_kernel<TA, TB, SYM, MAXT, MINB>;
  if (threads > MAXT) return cudaErrorInvalidConfiguration;
  cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, smem)) != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // one wave of resident CTAs (at most 8 per SM), whole stages per CTA
  const long long stages = (L2 + SF - 1) / SF;
  long long nctas = (long long)(per_sm < 8 ? per_sm : 8) * sms;
  if (nctas > stages) nctas = stages > 0 ? stages : 1;
  const long long st_per = (stages + nctas - 1) / nctas;
  nctas = stages > 0 ? (stages + st_per - 1) / st_per : 1;
  if ((size_t)nctas * na * nb * sizeof(double2) > part_cap) return cudaErrorInvalidValue;
  *nctas_out = (int)nctas;
  kern<<<(unsigned)nctas, threads, smem, s>>>(A, na, B, nb, L2, st_per * SF, part_buf);
  return cudaGetLastError();
}

}  // namespace

bool gram_cc_supported(const void* A, const void* B, int na, int nb, size_t L) {
  return na >= 1 && nb >= 1 && na <= 64 && nb <= 64 && L % 2 == 0 &&
         (reinterpret_cast<uintptr_t>(A) & 15) == 0 && (reinterpret_cast<uintptr_t>(B) & 15) == 0;
}

cudaError_t launch_gram_cc(const void* A, int na, const void* B, int nb, size_t L, double* G, cudaStream_t s) {
  if (!gram_cc_supported(A, B, na, nb, L)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  const bool sym = A == B && na == nb;
  const long long L2 = (long long)(L / 2);
  // partials for up to 8 CTAs per SM
  const size_t need = (size_t)8 * sms * na * nb * sizeof(double2);
  void* pv = nullptr;
  if ((e = scratch().get(s, need, &pv)) != cudaSuccess) return e;
  double2* part = static_cast<double2*>(pv);
  const size_t cap = scratch().capacity(s);
  const float4* a4 = static_cast<const float4*>(A);
  const float4* b4 = static_cast<const float4*>(B);
  int nctas = 0;
  // 4 x 4 entries per thread when that still gives at least two warps,
  // otherwise 2 x 2
  const int t4 = ((na + 3) / 4) * ((nb + 3) / 4);
  if (t4 < 64) {
    e = sym ? run<2, 2, true, 256, 1>(a4, na, a4, nb, L2, sms, part, cap, G, s, &nctas)
            : run<2, 2, false, 256, 1>(a4, na, b4, nb, L2, sms, part, cap, G, s, &nctas);
  } else if (t4 <= 192) {
    e = sym ? run<4, 4, true, 192, 2>(a4, na, a4, nb, L2, sms, part, cap, G, s, &nctas)
            : run<4, 4, false, 192, 2>(a4, na, b4, nb, L2, sms, part, cap, G, s, &nctas);
  } else {
    e = sym ? run<4, 4, true, 256, 1>(a4, na, a4, nb, L2, sms, part, cap, G, s, &nctas)
            : run<4, 4, false, 256, 1>(a4, na, b4, nb, L2, sms, part, cap, G, s, &nctas);
  }
  if (e != cudaSuccess) return e;
  gram_cc_sum_kernel<<<(unsigned)(na * nb), RED, 0, s>>>(part, nctas, na, nb, sym ? 1 : 0, G);
  return cudaGetLastError();
}

void gram_cc_release_stream(cudaStream_t s) { scratch().release(s); }

}  // namespace pcx
