// Gram products of complex64 column blocks on the tensor cores:
//   G = A^H B,  G_ij = sum_l conj(A_i[l]) B_j[l]
// (the Rayleigh-Ritz Gram matrices of the block eigensolver, Sec. 4).
//
// The complex product is a real one over stacked rows:
//   D = [Ar; Ai] [Br; Bi]^T  (contracted over l),
//   Re G = D[i][j] + D[na+i][nb+j],  Im G = D[i][nb+j] - D[na+i][j].
// D (M = 128 rows >= 2 na, N = NP columns >= 2 nb) accumulates in TMEM with
// tcgen05.mma kind::tf32.  FP32 inputs are split into TF32 hi + lo parts
// (round to nearest) and D += hi*hi + hi*lo + lo*hi, which keeps about the
// precision of FP32 products.  Every CTA contracts a contiguous range of l in
// chunks of KC rows staged in shared memory (double-buffered, tracked by two
// mbarriers); raw FP32 chunks arrive through cp.async two chunks ahead of
// their conversion.  Each CTA's FP32 partial D goes to global memory and a
// second kernel sums the partials of all CTAs in FP64.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>

#include "cx.cuh"
#include "pcx_internal.h"
#include "stream_scratch.h"
#include "tc.cuh"

namespace pcx {
namespace {

constexpr int KC = 32;        // rows of l per stage (4 MMAs of K = 8)
constexpr int MT = 128;       // M of the MMA: rows [Ar; Ai] padded
constexpr int TMEM_COLS = 128;
constexpr int NRAW = 3;       // raw FP32 chunk buffers (prefetch distance 2)
constexpr int THREADS = 256;
constexpr long WAIT_LIMIT = 1L << 22;   // mbarrier polls before giving up

// Operand tile of R rows x KC tf32: core matrix (row group g, K group kk) at
// kk * LBO + g * 128 bytes, rows 16 bytes apart inside it.  LBO = 16 R + 16
// makes stores that walk K (one row, 32 consecutive k) hit 32 banks.
__host__ __device__ constexpr int tile_lbo(int rows) { return 16 * rows + 16; }
__host__ __device__ constexpr int tile_bytes(int rows) { return (KC / 4) * tile_lbo(rows); }
__device__ __forceinline__ int tile_off(int rows, int row, int k) {
  return (k >> 2) * tile_lbo(rows) + (row >> 3) * 128 + (row & 7) * 16 + (k & 3) * 4;
}

struct GramArgs {
  const float2* A;
  const float2* B;
  int na, nb, np;       // np = N of the MMA (multiple of 16, >= 2 nb)
  int same;             // A == B and na == nb: one set of tiles serves both operands
  size_t L;
  long chunks_per_cta;
  long nchunks;
  float* partial;       // [gridDim.x][MT][np]
  int* err;
};

// write hi/lo TF32 parts of one complex entry of column `col` at k
__device__ __forceinline__ void put(unsigned char* hi, unsigned char* lo, int rows, int col, int ncol, int k,
                                    float2 v) {
  const float hr = tc::to_tf32(v.x), hm = tc::to_tf32(v.y);
  const float lr = tc::to_tf32(v.x - hr), lm = tc::to_tf32(v.y - hm);
  const int o0 = tile_off(rows, col, k), o1 = tile_off(rows, ncol + col, k);
  *reinterpret_cast<float*>(hi + o0) = hr;
  *reinterpret_cast<float*>(hi + o1) = hm;
  *reinterpret_cast<float*>(lo + o0) = lr;
  *reinterpret_cast<float*>(lo + o1) = lm;
}

constexpr int PRODUCERS = THREADS - 32;   // warps 0-6 stage and convert; warp 7 issues the MMAs

// Warp-specialised pipeline.  Producer warps keep raw chunks two ahead in
// flight (cp.async), convert chunk f into tile stage f % 2 once the MMAs of
// chunk f - 2 have released it (mbarrier empty[s], committed by the MMA
// warp) and signal full[s]; they synchronise among themselves with a named
// barrier only.  Lane 0 of warp 7 waits on full[s] and issues the MMAs.
// Every wait is bounded; a timeout sets a shared flag that every role reads
// at a uniform point, and the kernel reports it through g.err.
__global__ void __launch_bounds__(THREADS, 1) gram_tc_kernel(GramArgs g) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int abytes = tile_bytes(MT);
  const int bbytes = g.same ? 0 : tile_bytes(g.np);
  const int stage_bytes = 2 * abytes + 2 * bbytes;
  const int ncol = g.same ? g.na : g.na + g.nb;       // raw columns per chunk
  const int raw_bytes = ncol * KC * 8;
  unsigned char* raw0 = sm + 2 * stage_bytes;
  uint64_t* full = reinterpret_cast<uint64_t*>(raw0 + NRAW * raw_bytes);
  uint64_t* empty = full + 2;
  // last: the last chunk whose MMAs were committed (-1: none; 8-byte slot
  // right after the mbarriers); perr: written by thread 0 only, before the
  // producers' barrier (so every producer reads the same value after it);
  // merr: written by the MMA warp.  52 bytes in all.
  volatile long long* last = reinterpret_cast<volatile long long*>(empty + 2);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(const_cast<long long*>(last + 1));
  volatile int* perr = reinterpret_cast<volatile int*>(tslot + 1);
  volatile int* merr = perr + 1;
  const int tid = threadIdx.x, warp = tid / 32, lane = tid & 31;

  // zero the tiles once (padding rows stay zero), allocate TMEM, init barriers
  for (int i = tid; i < stage_bytes * 2 / 16; i += THREADS) reinterpret_cast<uint4*>(sm)[i] = make_uint4(0, 0, 0, 0);
  if (warp == 0) tc::tmem_alloc<TMEM_COLS>(tslot);
  if (tid == 0) {
    tc::mbar_init(&full[0], PRODUCERS);
    tc::mbar_init(&full[1], PRODUCERS);
    tc::mbar_init(&empty[0], 1);
    tc::mbar_init(&empty[1], 1);
    tc::mbar_fence_init();
    *perr = 0;
    *merr = 0;
    *last = -1;
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;

  const long c0 = (long)blockIdx.x * g.chunks_per_cta;
  const long c1 = c0 + g.chunks_per_cta < g.nchunks ? c0 + g.chunks_per_cta : g.nchunks;
  const long nfill = c1 > c0 ? c1 - c0 : 0;

  if (warp < PRODUCERS / 32) {
    // raw chunk f -> buffer f % NRAW: column c (A columns, then B columns),
    // KC complex numbers contiguous per column, 16-byte pieces
    auto prefetch = [&](long f) {
      if (f >= nfill) return;
      unsigned char* rb = raw0 + (f % NRAW) * raw_bytes;
      const size_t l0 = (size_t)(c0 + f) * KC;
      for (int e = tid; e < ncol * (KC / 2); e += PRODUCERS) {
        const int col = e / (KC / 2), piece = e % (KC / 2);
        const size_t l = l0 + 2 * piece;
        const float2* base = col < g.na ? g.A + (size_t)col * g.L : g.B + (size_t)(col - g.na) * g.L;
        const uint32_t bytes = l + 2 <= g.L ? 16u : (l < g.L ? 8u : 0u);
        tc::cp_async16(rb + (size_t)(col * KC + 2 * piece) * 8, base + (l < g.L ? l : 0), bytes);
      }
    };
    prefetch(0);
    tc::cp_async_commit();
    prefetch(1);
    tc::cp_async_commit();
    for (long f = 0; f < nfill; ++f) {
      tc::cp_async_wait<1>();                    // this thread's copies of chunk f are done
      const int s = (int)(f & 1);
      const long use = f >> 1;
      if (tid == 0 && use > 0 && !tc::mbar_wait(&empty[s], (uint32_t)((use - 1) & 1), WAIT_LIMIT)) *perr = 1;
      // chunk f has landed for every producer, chunk f - 1 is converted, stage s is free
      tc::named_barrier(1, PRODUCERS);
      if (*perr) break;                          // uniform: written before the barrier, read after it
      prefetch(f + 2);
      tc::cp_async_commit();
      unsigned char* ahi = sm + s * stage_bytes;
      unsigned char* alo = ahi + abytes;
      unsigned char* bhi = alo + abytes;
      unsigned char* blo = bhi + bbytes;
      const float2* rb = reinterpret_cast<const float2*>(raw0 + (f % NRAW) * raw_bytes);
      for (int e = tid; e < ncol * KC; e += PRODUCERS) {
        const int col = e / KC, k = e % KC;
        const float2 v = rb[e];
        if (col < g.na) put(ahi, alo, MT, col, g.na, k, v);
        else put(bhi, blo, g.np, col - g.na, g.nb, k, v);
      }
      tc::fence_proxy_async();                   // generic writes -> visible to the tensor core
      tc::mbar_arrive(&full[s]);
    }
    tc::cp_async_wait<0>();
  } else {
    const uint32_t idesc = tc::idesc_tf32(MT, g.np);
    long issued = 0;
    for (long f = 0; f < nfill; ++f) {
      const int s = (int)(f & 1);
      const long use = f >> 1;
      int ok = 1;
      if (lane == 0) ok = tc::mbar_wait(&full[s], (uint32_t)(use & 1), WAIT_LIMIT) ? 1 : 0;
      ok = __shfl_sync(0xffffffffu, ok, 0);
      if (!ok) {
        if (lane == 0) *merr = 1;
        break;
      }
      if (lane == 0) {
        tc::fence_after_sync();
        unsigned char* ahi = sm + s * stage_bytes;
        unsigned char* alo = ahi + abytes;
        unsigned char* bhi = alo + abytes;
        unsigned char* blo = bhi + bbytes;
        const uint32_t a_hi = tc::smem_addr(ahi), a_lo = tc::smem_addr(alo);
        const uint32_t b_hi = g.same ? a_hi : tc::smem_addr(bhi), b_lo = g.same ? a_lo : tc::smem_addr(blo);
        const uint32_t alb = tile_lbo(MT), blb = g.same ? tile_lbo(MT) : tile_lbo(g.np);
#pragma unroll
        for (int ks = 0; ks < KC / 8; ++ks) {
          const uint32_t ao = 2 * ks * alb, bo = 2 * ks * blb;
          const uint64_t dah = tc::smem_desc(a_hi + ao, alb, 128), dal = tc::smem_desc(a_lo + ao, alb, 128);
          const uint64_t dbh = tc::smem_desc(b_hi + bo, blb, 128), dbl = tc::smem_desc(b_lo + bo, blb, 128);
          tc::mma_tf32(tmem, dah, dbh, idesc, issued > 0 ? 1u : 0u);
          tc::mma_tf32(tmem, dah, dbl, idesc, 1u);
          tc::mma_tf32(tmem, dal, dbh, idesc, 1u);
          ++issued;
        }
        tc::mma_commit(&empty[s]);               // releases stage s when these MMAs complete
        *last = f;
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // the last commit covers every MMA issued; wait for it also on the error
  // path (with a shorter limit) so that no MMA is in flight when TMEM is freed
  bool ok = *perr == 0 && *merr == 0 && *last == nfill - 1;
  if (tid == 0 && *last >= 0) {
    const long fl = (long)*last;
    if (!tc::mbar_wait(&empty[fl & 1], (uint32_t)((fl >> 1) & 1), ok ? WAIT_LIMIT : WAIT_LIMIT / 16)) *merr = 1;
  }
  __syncthreads();
  ok = ok && *merr == 0;
  tc::fence_after_sync();
  if (!ok) {
    if (tid == 0) atomicExch(g.err, 1);
  } else if (warp < 4) {
    // epilogue: warp w reads TMEM lanes 32w..32w+31 (rows of D)
    const int row = warp * 32 + lane;
    float* out = g.partial + ((size_t)blockIdx.x * MT + row) * g.np;
    for (int cb = 0; cb < g.np; cb += 16) {
      float v[16];
      tc::tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)cb, v);
      if (nfill == 0) {
#pragma unroll
        for (int i = 0; i < 16; ++i) v[i] = 0.f;
      }
#pragma unroll
      for (int i = 0; i < 16; ++i) out[cb + i] = v[i];
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc<TMEM_COLS>(tmem);
}

// G[i][j] = sum over CTAs of the stacked-real products (FP64): one block per
// entry, its threads striding over the CTAs' partials, then a tree sum.
constexpr int RED_THREADS = 256;
__global__ void __launch_bounds__(RED_THREADS) gram_reduce_kernel(const float* __restrict__ partial, int nctas, int na,
                                                                 int nb, int np, const int* __restrict__ err,
                                                                 double* __restrict__ G) {
  __shared__ double red[2][RED_THREADS / 32];
  const int idx = blockIdx.x;
  const int i = idx / nb, j = idx % nb;
  double re = 0.0, im = 0.0;
  for (int c = threadIdx.x; c < nctas; c += RED_THREADS) {
    const float* p = partial + (size_t)c * MT * np;
    re += (double)p[i * np + j] + (double)p[(na + i) * np + nb + j];
    im += (double)p[i * np + nb + j] - (double)p[(na + i) * np + j];
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
    for (int w = 0; w < RED_THREADS / 32; ++w) {
      re += red[0][w];
      im += red[1][w];
    }
    if (*err) re = im = __longlong_as_double(0x7ff8000000000000LL);   // NaN: the kernel gave up
    G[2 * idx] = re;
    G[2 * idx + 1] = im;
  }
}

// per-CTA partial sums and the give-up flag, one buffer per (device, stream)
StreamScratch& scratch() {
  static StreamScratch s;
  return s;
}

}  // namespace

// 16-byte cp.async pieces need even column lengths (16-byte aligned columns)
bool gram_tc_supported(int na, int nb, size_t L) {
  return na >= 1 && nb >= 1 && 2 * na <= MT && 2 * nb <= TMEM_COLS && L % 2 == 0;
}

cudaError_t launch_gram_tc(const void* A, int na, const void* B, int nb, size_t L, double* G, cudaStream_t s) {
  if (!gram_tc_supported(na, nb, L)) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  GramArgs g;
  g.A = static_cast<const float2*>(A);
  g.B = static_cast<const float2*>(B);
  g.na = na;
  g.nb = nb;
  g.same = (A == B && na == nb) ? 1 : 0;
  g.np = g.same ? MT : ((2 * nb + 15) / 16) * 16;
  g.L = L;
  g.nchunks = (long)((L + KC - 1) / KC);
  long nctas = 8L * sms;   // short FP32 accumulation chains; partials are summed in FP64
  if (nctas > g.nchunks) nctas = g.nchunks > 0 ? g.nchunks : 1;
  g.chunks_per_cta = (g.nchunks + nctas - 1) / nctas;
  nctas = g.nchunks > 0 ? (g.nchunks + g.chunks_per_cta - 1) / g.chunks_per_cta : 1;
  const size_t pbytes = (size_t)nctas * MT * g.np * sizeof(float);
  void* buf = nullptr;   // [flag (256 bytes)][partials]
  if ((e = scratch().get(s, 256 + pbytes, &buf)) != cudaSuccess) return e;
  g.err = static_cast<int*>(buf);
  g.partial = reinterpret_cast<float*>(static_cast<char*>(buf) + 256);
  const int stage_bytes = 2 * tile_bytes(MT) + (g.same ? 0 : 2 * tile_bytes(g.np));
  const int ncol = g.same ? na : na + nb;
  const size_t smem = 2 * (size_t)stage_bytes + (size_t)NRAW * ncol * KC * 8 + 64;
  if ((e = cudaMemsetAsync(g.err, 0, sizeof(int), s)) != cudaSuccess) return e;
  if ((e = raise_dyn_smem(reinterpret_cast<const void*>(gram_tc_kernel), smem)) != cudaSuccess) return e;
  gram_tc_kernel<<<(unsigned)nctas, THREADS, smem, s>>>(g);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  gram_reduce_kernel<<<(unsigned)(na * nb), RED_THREADS, 0, s>>>(g.partial, (int)nctas, na, nb, g.np, g.err, G);
  return cudaGetLastError();
}

void gram_tc_release_stream(cudaStream_t s) { scratch().release(s); }

}  // namespace pcx
