// Kernels of the matrix-free apply of the compensated operator in the
// Fourier basis (Sec. 2.4 eq. matrixfree_kcform with the factorisation of
// Prop. 2.8) and of the FFT-diagonal preconditioner (eqs. matrixfree_diagP,
// matrixfree_finalform):
//
//   u = K_A^H x = -conj(kappa) x x          (per Fourier mode)
//   e = F3 u                                 (inverse DFT, positive exponent)
//   m = M e / N^3                            (per cell, Sec. 3.2.1 M_Trivial)
//   w = DFT(m)                               (negative exponent)
//   y = K_A w + gamma K_B x = kappa x w + gamma conj(kappa) (kappa . x)
//
// Five pencil passes, each a batch of 1D FFTs along one axis in shared
// memory, with the pointwise stages fused where all three components of a
// mode or a cell are at hand:
//   pass 1  x: C^H on load (and gamma kappa.x to scratch), inverse FFT
//   pass 2  y: inverse FFT
//   pass 3  z: inverse FFT, M sandwich, forward FFT
//   pass 4  y: forward FFT
//   pass 5  x: forward FFT, C w + gamma conj(kappa) (kappa.x) on store
// A CTA holds T pencils x 3 components x N points.  The 1D FFTs are Stockham
// radix-R stages (Govindaraju et al., SC 2008 formulation) with the small
// DFTs in registers.  Along y and z, where consecutive pencils are
// consecutive in memory, the first stage reads straight from global memory
// and the last stage writes straight to it; along x the tile is staged
// through shared memory with 16-byte accesses.
#pragma once

#include <cuda_runtime.h>

#include "cx.cuh"
#include "pcx_internal.h"

namespace pcx {
namespace fftk {

// OP_PLAIN_INV / OP_PLAIN_FWD: a bare unnormalised 1D DFT along the pass axis
// (positive / negative exponent), used for F3_3 and F3_3^H of whole vectors.
// OP_PRE_T0 / OP_SANDWICH_EPS / OP_POST_T0: the same five-pass chain for the
// curl-sandwich approximate inverse
//   T0 r = K_A F3^H eps F3 (K_A^H r / |k|^2) / |k|^2 + K_B r / (gamma |k|^4)
// (u and the scratch scaled by 1/|k|^2 and 1/(gamma |k|^4), eps = M^{-1}
// per cell by its adjugate, K_A w scaled by 1/|k|^2; a mode with |k| = 0
// maps to 0).
enum {
  OP_PRE = 0, OP_INV = 1, OP_SANDWICH = 2, OP_FWD = 3, OP_POST = 4, OP_PLAIN_INV = 5, OP_PLAIN_FWD = 6,
  OP_PRE_T0 = 7, OP_SANDWICH_EPS = 8, OP_POST_T0 = 9
};

// Radix plans: elements held per thread per stage E (16 complex floats or 8
// complex doubles), radices R0..R2 with N = R0 R1 R2 and every R <= E.
template <int N, int E>
struct Plan;
template <> struct Plan<8, 16> { static constexpr int R0 = 8, R1 = 0, R2 = 0, NST = 1; };
template <> struct Plan<16, 16> { static constexpr int R0 = 16, R1 = 0, R2 = 0, NST = 1; };
template <> struct Plan<32, 16> { static constexpr int R0 = 8, R1 = 4, R2 = 0, NST = 2; };
template <> struct Plan<64, 16> { static constexpr int R0 = 8, R1 = 8, R2 = 0, NST = 2; };
template <> struct Plan<128, 16> { static constexpr int R0 = 16, R1 = 8, R2 = 0, NST = 2; };
template <> struct Plan<256, 16> { static constexpr int R0 = 16, R1 = 16, R2 = 0, NST = 2; };
template <> struct Plan<8, 8> { static constexpr int R0 = 8, R1 = 0, R2 = 0, NST = 1; };
template <> struct Plan<16, 8> { static constexpr int R0 = 4, R1 = 4, R2 = 0, NST = 2; };
template <> struct Plan<32, 8> { static constexpr int R0 = 8, R1 = 4, R2 = 0, NST = 2; };
template <> struct Plan<64, 8> { static constexpr int R0 = 8, R1 = 8, R2 = 0, NST = 2; };
template <> struct Plan<128, 8> { static constexpr int R0 = 8, R1 = 4, R2 = 4, NST = 3; };
template <> struct Plan<128, 32> { static constexpr int R0 = 16, R1 = 8, R2 = 0, NST = 2; };
template <> struct Plan<128, 48> { static constexpr int R0 = 16, R1 = 8, R2 = 0, NST = 2; };
template <> struct Plan<256, 8> { static constexpr int R0 = 8, R1 = 8, R2 = 4, NST = 3; };

// Tile shape of the complex64 passes (elements per thread, pencils x points
// per component); build-time choices, overridable with -D for tuning builds.
#ifndef PCX_E32
#define PCX_E32 16
#endif
#ifndef PCX_TN32
#define PCX_TN32 2048
#endif

// Tile geometry: E elements per thread and stage, TN pencils x points per
// component (TP pencils per CTA).
// PAD: the row stride of y/z tiles is TP + PAD (see Tile).
template <typename T, int N, int TN_, int E_, int PAD_ = 1>
struct CfgG {
  static constexpr int E = E_;
  static constexpr int TN = TN_;
  static constexpr int TP = (TN / N < N * N) ? TN / N : N * N;   // pencils per CTA
  static constexpr int THREADS = 3 * TP * N / E;
  static constexpr int PAD = PAD_;
  static_assert(PAD >= 1 && N * PAD <= (N > 8 * TP ? N : 8 * TP), "row padding fits the component stride");
  // padded component stride: y/z tiles use N rows of TP + 1, x tiles TP
  // pencils of N + 8 (see Tile)
  static constexpr int CS = N * TP + (N > 8 * TP ? N : 8 * TP);
  // tile + twiddles + Lambda tables + kappa parts (3N per point, 3TP per pencil)
  static constexpr size_t SMEM = (size_t)(3 * CS + 3 * N + 3 * N + 3 * TP) * sizeof(cx<T>);
  using P = Plan<N, E>;
  static constexpr int RL = P::NST == 1 ? P::R0 : (P::NST == 2 ? P::R1 : P::R2);   // last radix
};
// the pass kernels' default geometry per precision
template <typename T, int N>
struct Cfg : CfgG<T, N, sizeof(T) == 4 ? PCX_TN32 : 1024, sizeof(T) == 4 ? PCX_E32 : 8> {};

struct PassArgs {
  const void* in;
  void* out;
  void* sbuf;          // [chunk][N^3]: gamma (kappa . x), written by pass 1, read by pass 5
  const void* lam;     // [2][N] Lambda_1, Lambda_0
  const void* tw;      // [N] exp(-2 pi i m / N)
  const void* M;       // [9][N^3] dense cell blocks (when mid == nullptr)
  const void* mid;     // [N^3] uchar4 material ids (E1, E2, E3, V)
  const void* mid3;    // the same ids in the order of the three-pass z tiles (or null)
  const void* mtab;    // [n_mat][9] block entries per material
  const void* mtab12;  // [n_mat][12] the same in 16-byte records (FP32; three-pass z tiles)
  int n_mat;
  KParams kp;
  // k-batched sweeps: vector v of the launch (v_base + v overall) uses
  // kps[(v_base + v) / vec_per_k] instead of kp (x passes only)
  const KParams* kps;
  int vec_per_k;
  int v_base;
};

template <typename T, int N, int AXIS, class CF = Cfg<T, N>>
struct Tile {
  static constexpr int TP = CF::TP;
  static constexpr int CS = CF::CS;
  // y/z tiles: pencils fastest, row stride TP + PAD (PAD = 1, an odd stride,
  // is conflict-free for pencil-fastest and point-fastest walks; the z tiles
  // of the three-pass chain choose theirs for their y-DFT staging).
  static constexpr int SN = TP + CF::PAD;
  // x tiles: points fastest within a pencil, pencil stride N + 8 (= 8 mod 16)
  // and the point index XOR-swizzled inside each group of 16, n ^ (n>>4 & 15),
  // so that radix-R writes at stride R, reads at stride N/R and point-fastest
  // walks all hit distinct banks.
  static constexpr int SP = N + 8;
  static __device__ __forceinline__ int swz(int n) { return N >= 32 ? (n ^ ((n >> 4) & 15)) : n; }
  static __device__ __forceinline__ int sidx(int c, int t, int n) {
    if constexpr (AXIS == 0) return c * CS + t * SP + swz(n);
    else return c * CS + n * SN + t;
  }
  // element offset (within one component block) of pencil q, point n
  static __device__ __forceinline__ int gidx(int q, int n) {
    if constexpr (AXIS == 0) return q * N + n;                           // q = z*N + y
    else if constexpr (AXIS == 1) return (q / N) * N * N + n * N + (q % N);   // q = z*N + x
    else return n * N * N + q;                                           // q = y*N + x
  }
  static constexpr int GSTRIDE = AXIS == 0 ? 1 : (AXIS == 1 ? N : N * N);   // offset step of n
  // butterfly walk: x tiles points fastest (coalesced global access along
  // x), y/z tiles pencils fastest
  static __device__ __forceinline__ void item(int w, int nb, int& t, int& j, int& c) {
    if constexpr (AXIS == 0) {
      j = w % nb;
      t = (w / nb) % TP;
      c = w / (nb * TP);
    } else {
      t = w % TP;
      j = (w / TP) % nb;
      c = w / (TP * nb);
    }
  }
};

// Penalty weight of one Fourier mode relative to kp.gamma (k2 = |kappa_p|^2):
// 1 in the scalar form; max(1, 1/k2) in the per-mode form; 1/k2 in the
// projector form.  The mode with kappa_p = 0 gets 0: its penalty term
// vanishes either way.
template <typename T>
__device__ __forceinline__ T penalty_weight(const KParams& kp, T k2) {
  if (!kp.per_mode || (kp.per_mode == 1 && k2 >= (T)1)) return (T)1;
  return k2 > (T)0 ? (T)1 / k2 : (T)0;
}

// Reciprocal of that weight (min(1, k2), k2 or 1): it scales 1/gamma into
// 1/gamma_p without a division.
template <typename T>
__device__ __forceinline__ T penalty_inv_weight(const KParams& kp, T k2) {
  if (kp.per_mode == 2) return k2;
  return kp.per_mode && k2 < (T)1 ? k2 : (T)1;
}

// kp.b[3 row + i] for a run-time column i in {0, 1, 2} (row a compile-time
// constant after unrolling), by selection: a run-time index into the
// parameter struct would make each thread keep a copy of it in local memory.
__device__ __forceinline__ double kp_b(const KParams& kp, int row, int i) {
  return i == 0 ? kp.b[3 * row] : (i == 1 ? kp.b[3 * row + 1] : kp.b[3 * row + 2]);
}

// kappa_i(p) = sum_j b_ji (L1(p_j) + i kt_j L0(p_j)) + i kq_i L0(p_i)
template <typename T>
__device__ __forceinline__ void kappa_at(const cx<T>* lam, int n, const KParams& kp, int p1, int p2, int p3,
                                         cx<T> kap[3]) {
  const int p[3] = {p1, p2, p3};
  cx<T> s[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    const cx<T> l1 = lam[p[j]], l0 = lam[n + p[j]];
    const T kt = (T)kp.kt[j];
    s[j] = mk(fma(-kt, l0.y, l1.x), fma(kt, l0.x, l1.y));
  }
  if (kp.diag_b) {
#pragma unroll
    for (int i = 0; i < 3; ++i) kap[i] = scale(s[i], (T)kp.b[4 * i]);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      kap[i] = mk((T)0, (T)0);
#pragma unroll
      for (int j = 0; j < 3; ++j)
        kap[i] = mk(fma((T)kp.b[3 * j + i], s[j].x, kap[i].x), fma((T)kp.b[3 * j + i], s[j].y, kap[i].y));
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (kp.kq[i] != 0.0) {
      const cx<T> l0 = lam[n + p[i]];
      const T kq = (T)kp.kq[i];
      kap[i] = mk(fma(-kq, l0.y, kap[i].x), fma(kq, l0.x, kap[i].y));
    }
  }
}

// two consecutive complex numbers, one 16-byte access for complex64
template <typename T>
__device__ __forceinline__ void ld2(const cx<T>* p, cx<T>& a, cx<T>& b) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    a = mk(v.x, v.y);
    b = mk(v.z, v.w);
  } else {
    a = p[0];
    b = p[1];
  }
}
template <typename T>
__device__ __forceinline__ void st2(cx<T>* p, cx<T> a, cx<T> b) {
  if constexpr (sizeof(T) == 4) {
    *reinterpret_cast<float4*>(p) = make_float4(a.x, a.y, b.x, b.y);
  } else {
    p[0] = a;
    p[1] = b;
  }
}

// Asynchronous copy of one complex element global -> shared (8 or 16 bytes).
template <typename T>
__device__ __forceinline__ void cp_async_cx(cx<T>* dst, const cx<T>* src) {
  const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(dst));
  if constexpr (sizeof(T) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

// Stockham stage of radix R (Ns = product of the radices already done).
// SRC: 0 = shared memory, 1 = global (first stage only, Ns = 1).
// DST: 0 = shared memory, 1 = global (last stage only, Ns = N / R).
// Threads walk butterflies with the pencil index fastest.
// Barrier of the threads that run a stage: the whole CTA by default; a
// named barrier over the first COUNT threads where one warp group of a
// warp-specialised kernel runs the stages (bar.sync: every warp of the group
// arrives and waits; the hardware barrier needs no spin loop).
struct CtaSync {
  static __device__ __forceinline__ void sync() { __syncthreads(); }
};
template <int ID, int COUNT>
struct GroupSync {
  static_assert(ID >= 1 && ID < 16 && COUNT % 32 == 0, "named barrier id and warp-multiple count");
  static __device__ __forceinline__ void sync() { asm volatile("bar.sync %0, %1;\n" ::"n"(ID), "n"(COUNT) : "memory"); }
};

template <typename T, int N, int AXIS, int R, int DIR, int SRC, int DST, class CF = Cfg<T, N>, class SYNC = CtaSync>
__device__ __forceinline__ void stage(cx<T>* s, const cx<T>* tw, int Ns, const cx<T>* gin, cx<T>* gout, int qb) {
  using C = CF;
  using TL = Tile<T, N, AXIS, CF>;
  constexpr int NB = N / R;
  constexpr int PER = C::E / R;
  constexpr int N3 = N * N * N;
  cx<T> v[PER][R];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    int t, j, c;
    TL::item(threadIdx.x + i * C::THREADS, NB, t, j, c);
    if constexpr (SRC == 1) {
      const cx<T>* g = gin + (c * N3 + TL::gidx(qb + t, j));
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = g[r * NB * TL::GSTRIDE];
    } else if constexpr (AXIS == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = s[TL::sidx(c, t, j + r * NB)];
    } else {
      const cx<T>* sp = s + TL::sidx(c, t, j);
#pragma unroll
      for (int r = 0; r < R; ++r) v[i][r] = sp[r * NB * TL::SN];
    }
  }
  if constexpr (SRC == 0 && DST == 0) SYNC::sync();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    int t, j, c;
    TL::item(threadIdx.x + i * C::THREADS, NB, t, j, c);
    const int k = j % Ns;
    if (SRC == 0 && Ns > 1) {
      const int step = N / (Ns * R);
#pragma unroll
      for (int r = 1; r < R; ++r) {
        cx<T> wt = tw[r * k * step];
        if (DIR > 0) wt.y = -wt.y;
        v[i][r] = v[i][r] * wt;
      }
    }
    dft<R, DIR>(v[i]);
    const int base = (j / Ns) * Ns * R + k;
    if constexpr (DST == 1) {
      cx<T>* g = gout + (c * N3 + TL::gidx(qb + t, base));
#pragma unroll
      for (int r = 0; r < R; ++r) g[r * Ns * TL::GSTRIDE] = v[i][r];
    } else if constexpr (AXIS == 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) s[TL::sidx(c, t, base + r * Ns)] = v[i][r];
    } else {
      cx<T>* sp = s + TL::sidx(c, t, base);
#pragma unroll
      for (int r = 0; r < R; ++r) sp[r * Ns * TL::SN] = v[i][r];
    }
  }
  if constexpr (DST == 0) SYNC::sync();
}

// Full 1D transform of the tile.  FROM_G: the first stage reads global
// memory; TO_G: the last stage writes global memory.
template <typename T, int N, int AXIS, int DIR, int FROM_G, int TO_G, class CF = Cfg<T, N>>
__device__ __forceinline__ void fft_tile(cx<T>* s, const cx<T>* tw, const cx<T>* gin, cx<T>* gout, int qb) {
  using P = typename CF::P;
  if constexpr (P::NST == 1) {
    stage<T, N, AXIS, P::R0, DIR, FROM_G, TO_G, CF>(s, tw, 1, gin, gout, qb);
  } else if constexpr (P::NST == 2) {
    stage<T, N, AXIS, P::R0, DIR, FROM_G, 0, CF>(s, tw, 1, gin, gout, qb);
    stage<T, N, AXIS, P::R1, DIR, 0, TO_G, CF>(s, tw, P::R0, gin, gout, qb);
  } else {
    stage<T, N, AXIS, P::R0, DIR, FROM_G, 0, CF>(s, tw, 1, gin, gout, qb);
    stage<T, N, AXIS, P::R1, DIR, 0, 0, CF>(s, tw, P::R0, gin, gout, qb);
    stage<T, N, AXIS, P::R2, DIR, 0, TO_G, CF>(s, tw, P::R0 * P::R1, gin, gout, qb);
  }
}

template <typename T, int N, int AXIS, int OP>
__global__ void __launch_bounds__(Cfg<T, N>::THREADS, sizeof(T) == 4 ? 3 : 1) pass_kernel(PassArgs a) {
  using C = Cfg<T, N>;
  using TL = Tile<T, N, AXIS>;
  constexpr int TP = C::TP;
  constexpr int N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = s + 3 * C::CS;
  cx<T>* ka = tw + N;          // [3][N]  kappa_i part that depends on p1
  cx<T>* kb = ka + 3 * N;      // [TP][3] kappa_i part that depends on the pencil (p2, p3)
  T* mtab = reinterpret_cast<T*>(kb + 3 * TP);

  const size_t q0 = (size_t)blockIdx.x * TP;       // first pencil (counted across the chunk's vectors)
  const size_t v = q0 / N2;
  const int qb = (int)(q0 % N2);
  const cx<T>* in = static_cast<const cx<T>*>(a.in) + v * 3 * N3;
  cx<T>* out = static_cast<cx<T>*>(a.out) + v * 3 * N3;

  const cx<T>* gtw = static_cast<const cx<T>*>(a.tw);
  for (int i = threadIdx.x; i < N; i += C::THREADS) tw[i] = gtw[i];
  KParams kp = a.kp;
  if (AXIS == 0 && a.kps) kp = a.kps[(a.v_base + (int)v) / a.vec_per_k];
  if constexpr (AXIS == 0 && OP != OP_PLAIN_INV && OP != OP_PLAIN_FWD) {
    // kappa_i(p) = sum_j b_ji S_j(p_j) + i kq_i L0(p_i),  S_j = L1 + i kt_j L0,
    // split as ka_i(p1) + kb_i(p2, p3)
    const cx<T>* glam = static_cast<const cx<T>*>(a.lam);
    for (int e = threadIdx.x; e < 3 * N + 3 * TP; e += C::THREADS) {
      if (e < 3 * N) {
        const int i = e / N, p = e % N;
        const cx<T> l1 = glam[p], l0 = glam[N + p];
        const T b0 = (T)kp_b(kp, 0, i);   // b_1i (row j = 0)
        const T kt = (T)kp.kt[0];
        cx<T> r = mk(b0 * fma(-kt, l0.y, l1.x), b0 * fma(kt, l0.x, l1.y));
        if (i == 0) r = mk(fma(-(T)kp.kq[0], l0.y, r.x), fma((T)kp.kq[0], l0.x, r.y));
        ka[e] = r;
      } else {
        const int f = e - 3 * N, t = f / 3, i = f % 3;
        const int q = qb + t, p[3] = {0, q % N, q / N};
        cx<T> r = mk((T)0, (T)0);
#pragma unroll
        for (int j = 1; j < 3; ++j) {
          const cx<T> l1 = glam[p[j]], l0 = glam[N + p[j]];
          const T bj = (T)kp_b(kp, j, i), kt = (T)kp.kt[j];
          r = mk(fma(bj, fma(-kt, l0.y, l1.x), r.x), fma(bj, fma(kt, l0.x, l1.y), r.y));
          if (i == j) r = mk(fma(-(T)kp.kq[j], l0.y, r.x), fma((T)kp.kq[j], l0.x, r.y));
        }
        kb[3 * t + i] = r;
      }
    }
  }
  if constexpr (OP == OP_SANDWICH || OP == OP_SANDWICH_EPS) {
    if (a.mid) {
      const T* gt = static_cast<const T*>(a.mtab);
      for (int i = threadIdx.x; i < 9 * a.n_mat; i += C::THREADS) mtab[i] = gt[i];
    }
  }

  if constexpr (OP == OP_PLAIN_INV || OP == OP_PLAIN_FWD) {
    __syncthreads();
    fft_tile<T, N, AXIS, OP == OP_PLAIN_INV ? +1 : -1, 1, 1>(s, tw, in, out, qb);
  } else if constexpr (AXIS == 0) {
    // ---- x-axis passes: staged through shared memory, points fastest ----
    __syncthreads();   // tables visible
    if constexpr (OP == OP_PRE || OP == OP_PRE_T0) {
      // u = -conj(kappa) x x per mode, and gamma_p kappa.x to the scratch
      // (T0: u / |k|^2 and kappa.x / (gamma_p |k|^4))
      cx<T>* sb = static_cast<cx<T>*>(a.sbuf) + v * N3;
      const T gam = (T)kp.gamma;
      const T igam = (T)(1.0 / kp.gamma);
      // the x tile lands in shared memory by asynchronous copies (all in
      // flight at once), then C^H is applied in place
      for (int e = threadIdx.x; e < TP * N; e += C::THREADS) {
        const int t = e / N, n = e % N;
        const int g = TL::gidx(qb + t, n);
#pragma unroll
        for (int c = 0; c < 3; ++c) cp_async_cx<T>(&s[TL::sidx(c, t, n)], &in[c * N3 + g]);
      }
      cp_async_commit_wait_all();
      __syncthreads();
      for (int e = threadIdx.x; e < TP * N; e += C::THREADS) {
        const int t = e / N, n = e % N;
        const int g = TL::gidx(qb + t, n);
        const cx<T> x0 = s[TL::sidx(0, t, n)], x1 = s[TL::sidx(1, t, n)], x2 = s[TL::sidx(2, t, n)];
        cx<T> kap[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) kap[i] = ka[i * N + n] + kb[3 * t + i];
        T su = (T)1, ss = gam;
        if constexpr (OP == OP_PRE_T0) {
          const T k2 = norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]);
          su = k2 > (T)0 ? (T)1 / k2 : (T)0;
          ss = su * su * igam * penalty_inv_weight(kp, k2);
        } else if (kp.per_mode) {
          ss = gam * penalty_weight(kp, norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]));
        }
        sb[g] = scale(cfma(kap[2], x2, cfma(kap[1], x1, kap[0] * x0)), ss);
        const cx<T> z = mk((T)0, (T)0);
        cx<T> u0 = cfma_conj(kap[2], x1, scale(cfma_conj(kap[1], x2, z), (T)-1));
        cx<T> u1 = cfma_conj(kap[0], x2, scale(cfma_conj(kap[2], x0, z), (T)-1));
        cx<T> u2 = cfma_conj(kap[1], x0, scale(cfma_conj(kap[0], x1, z), (T)-1));
        if constexpr (OP == OP_PRE_T0) {
          u0 = scale(u0, su);
          u1 = scale(u1, su);
          u2 = scale(u2, su);
        }
        s[TL::sidx(0, t, n)] = u0;
        s[TL::sidx(1, t, n)] = u1;
        s[TL::sidx(2, t, n)] = u2;
      }
      __syncthreads();
      fft_tile<T, N, 0, +1, 0, 1>(s, tw, nullptr, out, qb);
    } else {   // OP_POST
      // gamma kappa.x of the tile is fetched into shared memory while the
      // FFT runs
      const cx<T>* sb = static_cast<const cx<T>*>(a.sbuf) + v * N3;
      cx<T>* ssb = kb + 3 * TP;   // [TP * N], POST launches only
      for (int e = threadIdx.x; e < TP * N; e += C::THREADS) {
        const int t = e / N, n = e % N;
        cp_async_cx<T>(&ssb[e], &sb[TL::gidx(qb + t, n)]);
      }
      fft_tile<T, N, 0, -1, 1, 0>(s, tw, in, nullptr, qb);
      cp_async_commit_wait_all();
      __syncthreads();
      for (int e = threadIdx.x; e < TP * N; e += C::THREADS) {
        const int t = e / N, n = e % N;
        const int g = TL::gidx(qb + t, n);
        const cx<T> sk = ssb[e];
        cx<T> kap[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) kap[i] = ka[i * N + n] + kb[3 * t + i];
        const cx<T> w0 = s[TL::sidx(0, t, n)], w1 = s[TL::sidx(1, t, n)], w2 = s[TL::sidx(2, t, n)];
        cx<T> c0 = cfma(kap[1], w2, scale(kap[2] * w1, (T)-1));
        cx<T> c1 = cfma(kap[2], w0, scale(kap[0] * w2, (T)-1));
        cx<T> c2 = cfma(kap[0], w1, scale(kap[1] * w0, (T)-1));
        if constexpr (OP == OP_POST_T0) {
          const T k2 = norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]);
          const T su = k2 > (T)0 ? (T)1 / k2 : (T)0;
          c0 = scale(c0, su);
          c1 = scale(c1, su);
          c2 = scale(c2, su);
        }
        out[g] = cfma_conj(kap[0], sk, c0);
        out[N3 + g] = cfma_conj(kap[1], sk, c1);
        out[2 * N3 + g] = cfma_conj(kap[2], sk, c2);
      }
    }
  } else if constexpr (OP == OP_SANDWICH || OP == OP_SANDWICH_EPS) {
    // ---- z-axis: inverse FFT, per-cell M (Sec. 3.2.1; or eps = M^{-1}),
    // forward FFT ----
    __syncthreads();
    const T* M = static_cast<const T*>(a.M);
    const uchar4* mid = static_cast<const uchar4*>(a.mid);
    // material ids of the tile's cells, fetched into shared memory while
    // the z FFT runs
    uchar4* sid = reinterpret_cast<uchar4*>(mtab + 9 * a.n_mat);   // [TP * N], sandwich launches only
    if (mid) {
      for (int w = threadIdx.x; w < TP * N; w += C::THREADS) {
        const unsigned d = static_cast<unsigned>(__cvta_generic_to_shared(&sid[w]));
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(&mid[(w / TP) * N2 + (qb + w % TP)])
                     : "memory");
      }
    }
    fft_tile<T, N, 2, +1, 1, 0>(s, tw, in, nullptr, qb);
    cp_async_commit_wait_all();
    __syncthreads();
    const T inv_n3 = (T)(1.0 / (double)N3);
    for (int w = threadIdx.x; w < TP * N; w += C::THREADS) {   // pencils fastest
      const int t = w % TP, n = w / TP;
      const int cell = n * N2 + (qb + t);   // (x, y, z) = (q % N, q / N, n)
      T d1, d2, d3;
      cx<T> o12, o13, o23;
      if (mid) {
        const uchar4 id = sid[w];
        d1 = mtab[9 * id.x];
        d2 = mtab[9 * id.y + 1];
        d3 = mtab[9 * id.z + 2];
        const T* o = mtab + 9 * id.w;
        o12 = mk(o[3], o[4]);
        o13 = mk(o[5], o[6]);
        o23 = mk(o[7], o[8]);
      } else {
        d1 = M[cell];
        d2 = M[N3 + cell];
        d3 = M[2 * N3 + cell];
        o12 = mk(M[3 * N3 + cell], M[4 * N3 + cell]);
        o13 = mk(M[5 * N3 + cell], M[6 * N3 + cell]);
        o23 = mk(M[7 * N3 + cell], M[8 * N3 + cell]);
      }
      const int i0 = TL::sidx(0, t, n), i1 = TL::sidx(1, t, n), i2 = TL::sidx(2, t, n);
      const cx<T> e0 = s[i0], e1 = s[i1], e2 = s[i2];
      T sc = inv_n3;
      if constexpr (OP == OP_SANDWICH_EPS) {
        // eps = M^{-1} = adj(M) / det(M): the adjugate of the Hermitian block
        // (upper triangle) replaces M, the determinant joins the scale
        const T a11 = d2 * d3 - norm2(o23), a22 = d1 * d3 - norm2(o13), a33 = d1 * d2 - norm2(o12);
        const cx<T> a12 = o13 * conjg(o23) - scale(o12, d3);
        const cx<T> a13 = o12 * o23 - scale(o13, d2);
        const cx<T> a23 = o13 * conjg(o12) - scale(o23, d1);
        const T det = d1 * a11 + (o12 * conjg(a12)).x + (o13 * conjg(a13)).x;
        sc = inv_n3 / det;
        d1 = a11;
        d2 = a22;
        d3 = a33;
        o12 = a12;
        o13 = a13;
        o23 = a23;
      }
      const cx<T> m0 = cfma(o13, e2, cfma(o12, e1, scale(e0, d1)));
      const cx<T> m1 = cfma(o23, e2, cfma_conj(o12, e0, scale(e1, d2)));
      const cx<T> m2 = cfma_conj(o23, e1, cfma_conj(o13, e0, scale(e2, d3)));
      s[i0] = scale(m0, sc);
      s[i1] = scale(m1, sc);
      s[i2] = scale(m2, sc);
    }
    __syncthreads();
    fft_tile<T, N, 2, -1, 0, 1>(s, tw, nullptr, out, qb);
  } else {
    // ---- y-axis passes: straight from global and back ----
    __syncthreads();
    constexpr int DIR = OP == OP_INV ? +1 : -1;
    fft_tile<T, N, 1, DIR, 1, 1>(s, tw, in, out, qb);
  }
}

// W = K_P^{-1} R per mode: r/|k|^2 + (1/gamma_p - 1) conj(k) (k . r) / |k|^4.
template <typename T>
__global__ void precond_kernel(const cx<T>* __restrict__ R, cx<T>* __restrict__ W, const cx<T>* __restrict__ lam,
                               int n, int nvec, KParams kp) {
  const size_t n3 = (size_t)n * n * n;
  const int lg = __ffs(n) - 1;   // n is a power of two
  const size_t total = n3 * nvec;
  const T ig = (T)(1.0 / kp.gamma);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e >> (3 * lg), mode = e & (n3 - 1);
    const int p1 = (int)(mode & (n - 1)), p2 = (int)((mode >> lg) & (n - 1)), p3 = (int)(mode >> (2 * lg));
    cx<T> kap[3];
    kappa_at<T>(lam, n, kp, p1, p2, p3, kap);
    const size_t base = v * 3 * n3 + mode;
    const cx<T> r0 = R[base], r1 = R[base + n3], r2 = R[base + 2 * n3];
    const T k2 = norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]);
    cx<T> w0, w1, w2;
    if (k2 > (T)0) {
      const T ik2 = (T)1 / k2;
      const T cg = ig * penalty_inv_weight(kp, k2) - (T)1;
      cx<T> sk = cfma(kap[2], r2, cfma(kap[1], r1, kap[0] * r0));
      sk = scale(sk, cg * ik2 * ik2);
      w0 = cfma_conj(kap[0], sk, scale(r0, ik2));
      w1 = cfma_conj(kap[1], sk, scale(r1, ik2));
      w2 = cfma_conj(kap[2], sk, scale(r2, ik2));
    } else {
      w0 = w1 = w2 = mk((T)0, (T)0);
    }
    W[base] = w0;
    W[base + n3] = w1;
    W[base + 2 * n3] = w2;
  }
}

// Quadratic form of the penalty term per column: out[v] += sum over modes
// |kappa(p) . x_v(p)|^2 = x_v^H K_B x_v (= ||B x||^2 for the real-space
// field, Prop. 2.8), each mode weighted by gamma_p / gamma in the per-mode
// form, and out[nvec + v] += ||x_v||^2.  One block row per
// column (blockIdx.y); block sums are added with FP64 atomics.
template <typename T>
__global__ void __launch_bounds__(256) div_norm_kernel(const cx<T>* __restrict__ X, const cx<T>* __restrict__ lam,
                                                      int n, int nvec, KParams kp, double* __restrict__ out) {
  const size_t n3 = (size_t)n * n * n;
  const int lg = __ffs(n) - 1;   // n is a power of two
  const int v = blockIdx.y;
  const cx<T>* x = X + (size_t)v * 3 * n3;
  double sb = 0.0, sx = 0.0;
  for (size_t mode = (size_t)blockIdx.x * blockDim.x + threadIdx.x; mode < n3; mode += (size_t)gridDim.x * blockDim.x) {
    const int p1 = (int)(mode & (n - 1)), p2 = (int)((mode >> lg) & (n - 1)), p3 = (int)(mode >> (2 * lg));
    cx<T> kap[3];
    kappa_at<T>(lam, n, kp, p1, p2, p3, kap);
    const cx<T> x0 = x[mode], x1 = x[mode + n3], x2 = x[mode + 2 * n3];
    const cx<T> d = cfma(kap[2], x2, cfma(kap[1], x1, kap[0] * x0));
    T wb = (T)1;
    if (kp.per_mode) wb = penalty_weight(kp, norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]));
    sb += (double)(wb * norm2(d));
    sx += (double)norm2(x0) + (double)norm2(x1) + (double)norm2(x2);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    sb += __shfl_xor_sync(0xffffffffu, sb, o);
    sx += __shfl_xor_sync(0xffffffffu, sx, o);
  }
  __shared__ double red[2][8];
  const int warp = threadIdx.x / 32, lane = threadIdx.x % 32;
  if (lane == 0) {
    red[0][warp] = sb;
    red[1][warp] = sx;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tb = 0.0, tx = 0.0;
    for (int w = 0; w < (int)(blockDim.x / 32); ++w) {
      tb += red[0][w];
      tx += red[1][w];
    }
    atomicAdd(out + v, tb);
    atomicAdd(out + nvec + v, tx);
  }
}

// ---- pieces of the curl-sandwich approximate inverse --------------------
//   T0 r = K_A F3_3^H eps F3_3 (K_A^H r / |k|^2) / |k|^2 + K_B r / (gamma |k|^4)
// (Johnson and Joannopoulos 2001, with the symbols of Prop. 2.8; eps = M^{-1}
// cell by cell; |k|^2 = sum_i |kappa_i|^2; a mode with |k| = 0 maps to 0).

// U = K_A^H X / |k|^(2 POW) per mode, K_A^H x = -conj(kappa) x x
template <typename T>
__global__ void curl_h_kernel(const cx<T>* __restrict__ X, cx<T>* __restrict__ U, const cx<T>* __restrict__ lam,
                              int n, int nvec, KParams kp, int pow) {
  const size_t n3 = (size_t)n * n * n;
  const int lg = __ffs(n) - 1;   // n is a power of two
  const size_t total = n3 * nvec;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e >> (3 * lg), mode = e & (n3 - 1);
    const int p1 = (int)(mode & (n - 1)), p2 = (int)((mode >> lg) & (n - 1)), p3 = (int)(mode >> (2 * lg));
    cx<T> kap[3];
    kappa_at<T>(lam, n, kp, p1, p2, p3, kap);
    const size_t base = v * 3 * n3 + mode;
    const cx<T> x0 = X[base], x1 = X[base + n3], x2 = X[base + 2 * n3];
    const T k2 = norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]);
    const T sc = k2 > (T)0 ? (pow ? (T)1 / k2 : (T)1) : (T)0;
    const cx<T> z = mk((T)0, (T)0);
    U[base] = scale(cfma_conj(kap[2], x1, scale(cfma_conj(kap[1], x2, z), (T)-1)), sc);
    U[base + n3] = scale(cfma_conj(kap[0], x2, scale(cfma_conj(kap[2], x0, z), (T)-1)), sc);
    U[base + 2 * n3] = scale(cfma_conj(kap[1], x0, scale(cfma_conj(kap[0], x1, z), (T)-1)), sc);
  }
}

// Y (+)= s K_A Wm / |k|^2 + [R given] conj(kappa) (kappa . r) / (gamma_p |k|^4)
template <typename T>
__global__ void curl_add_kernel(const cx<T>* __restrict__ Wm, const cx<T>* __restrict__ R, cx<T>* __restrict__ Y,
                                const cx<T>* __restrict__ lam, int n, int nvec, KParams kp, T s, int accumulate) {
  const size_t n3 = (size_t)n * n * n;
  const int lg = __ffs(n) - 1;   // n is a power of two
  const size_t total = n3 * nvec;
  const T ig = (T)(1.0 / kp.gamma);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e >> (3 * lg), mode = e & (n3 - 1);
    const int p1 = (int)(mode & (n - 1)), p2 = (int)((mode >> lg) & (n - 1)), p3 = (int)(mode >> (2 * lg));
    cx<T> kap[3];
    kappa_at<T>(lam, n, kp, p1, p2, p3, kap);
    const size_t base = v * 3 * n3 + mode;
    const T k2 = norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]);
    cx<T> y0 = mk((T)0, (T)0), y1 = y0, y2 = y0;
    if (k2 > (T)0) {
      const T ik2 = (T)1 / k2;
      const cx<T> w0 = Wm[base], w1 = Wm[base + n3], w2 = Wm[base + 2 * n3];
      const T sw = s * ik2;
      y0 = scale(cfma(kap[1], w2, scale(kap[2] * w1, (T)-1)), sw);
      y1 = scale(cfma(kap[2], w0, scale(kap[0] * w2, (T)-1)), sw);
      y2 = scale(cfma(kap[0], w1, scale(kap[1] * w0, (T)-1)), sw);
      if (R) {
        const cx<T> r0 = R[base], r1 = R[base + n3], r2 = R[base + 2 * n3];
        const cx<T> sk =
            scale(cfma(kap[2], r2, cfma(kap[1], r1, kap[0] * r0)), ig * penalty_inv_weight(kp, k2) * ik2 * ik2);
        y0 = cfma_conj(kap[0], sk, y0);
        y1 = cfma_conj(kap[1], sk, y1);
        y2 = cfma_conj(kap[2], sk, y2);
      }
    }
    if (accumulate) {
      y0 = y0 + Y[base];
      y1 = y1 + Y[base + n3];
      y2 = y2 + Y[base + 2 * n3];
    }
    Y[base] = y0;
    Y[base + n3] = y1;
    Y[base + 2 * n3] = y2;
  }
}

// Mo = s (M_cell^{-1} E + Add) cell by cell (real-space fields; Add optional;
// Mo may alias E).  The inverse of the Hermitian 3x3 block (real diagonal
// d1, d2, d3, off-diagonal o12, o13, o23) by its adjugate.
template <typename T>
__global__ void eps_cells_kernel(const cx<T>* E, const cx<T>* __restrict__ Add, cx<T>* Mo, const uchar4* __restrict__ mid,
                                 const T* __restrict__ mtab, const T* __restrict__ M, int n, int nvec, T s) {
  const size_t n3 = (size_t)n * n * n;
  const int lg = __ffs(n) - 1;   // n is a power of two
  const size_t total = n3 * nvec;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e >> (3 * lg), cell = e & (n3 - 1);
    T d1, d2, d3;
    cx<T> o12, o13, o23;
    if (mid) {
      const uchar4 id = mid[cell];
      d1 = mtab[9 * id.x];
      d2 = mtab[9 * id.y + 1];
      d3 = mtab[9 * id.z + 2];
      const T* o = mtab + 9 * id.w;
      o12 = mk(o[3], o[4]);
      o13 = mk(o[5], o[6]);
      o23 = mk(o[7], o[8]);
    } else {
      d1 = M[cell];
      d2 = M[n3 + cell];
      d3 = M[2 * n3 + cell];
      o12 = mk(M[3 * n3 + cell], M[4 * n3 + cell]);
      o13 = mk(M[5 * n3 + cell], M[6 * n3 + cell]);
      o23 = mk(M[7 * n3 + cell], M[8 * n3 + cell]);
    }
    // adjugate entries (the inverse times det), upper triangle
    const T a11 = d2 * d3 - norm2(o23), a22 = d1 * d3 - norm2(o13), a33 = d1 * d2 - norm2(o12);
    const cx<T> a12 = o13 * conjg(o23) - scale(o12, d3);
    const cx<T> a13 = o12 * o23 - scale(o13, d2);
    const cx<T> a23 = o13 * conjg(o12) - scale(o23, d1);
    const T det = d1 * a11 + (o12 * conjg(a12)).x + (o13 * conjg(a13)).x;
    const T sc = s / det;
    const size_t base = v * 3 * n3 + cell;
    const cx<T> e0 = E[base], e1 = E[base + n3], e2 = E[base + 2 * n3];
    cx<T> m0 = cfma(a13, e2, cfma(a12, e1, scale(e0, a11)));
    cx<T> m1 = cfma(a23, e2, cfma_conj(a12, e0, scale(e1, a22)));
    cx<T> m2 = cfma_conj(a23, e1, cfma_conj(a13, e0, scale(e2, a33)));
    m0 = scale(m0, sc);
    m1 = scale(m1, sc);
    m2 = scale(m2, sc);
    if (Add) {
      m0 = m0 + scale(Add[base], s);
      m1 = m1 + scale(Add[base + n3], s);
      m2 = m2 + scale(Add[base + 2 * n3], s);
    }
    Mo[base] = m0;
    Mo[base + n3] = m1;
    Mo[base + 2 * n3] = m2;
  }
}

// Mo = s M_CrossDoF E on real-space fields (Sec. 3.2.2, eq. crossdof_herm;
// Mo must not alias E).  Diagonal entries as in M_Trivial; off the diagonal
// the symmetrised transfers
//   block (i, j) = ( diag(e_ij at E_i) T_ij + T_ij diag(e_ij at E_j) ) / 2,
//   block (j, i) = its conjugate transpose,
// with e_ij = (eps_1)_ij of the material at each point (from the material
// ids of the E1, E2, E3 point sets) and the four-point means of the
// componentwise template eq. crossdof_xytemplate, in array slots [z][y][x]:
//   T_01 f = (f + f[x-1] + f[y+1] + f[y+1, x-1]) / 4     (D0 on x, D0^T on y)
//   T_02 f = (f + f[x-1] + f[z+1] + f[z+1, x-1]) / 4     (D0 on x, D0^T on z)
//   T_12 f = (f + f[y-1] + f[z+1] + f[z+1, y-1]) / 4     (D0 on y, D0^T on z)
// and their transposes with every offset negated.  One thread per cell and
// vector; neighbours wrap periodically (N is a power of two).
template <typename T>
__global__ void crossdof_kernel(const cx<T>* __restrict__ E, cx<T>* __restrict__ Mo, const uchar4* __restrict__ mid,
                                const T* __restrict__ mtab, int n, int nvec, T s) {
  const size_t n3 = (size_t)n * n * n;
  const int lg = __ffs(n) - 1;   // n is a power of two
  const int msk = n - 1;
  const size_t total = n3 * nvec;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e >> (3 * lg);
    const int cell = (int)(e & (n3 - 1));
    const int x = cell & msk, y = (cell >> lg) & msk, z = cell >> (2 * lg);
    const cx<T>* ev = E + v * 3 * n3;
    auto at = [&](int dz, int dy, int dx) -> int {
      return (((z + dz) & msk) << (2 * lg)) | (((y + dy) & msk) << lg) | ((x + dx) & msk);
    };
    // (eps_1)_ij of the material at point set c of cell q; pair 0: 12, 1: 13, 2: 23
    auto off = [&](int q, int c, int pair) -> cx<T> {
      const uchar4 id = mid[q];
      const int m = c == 0 ? id.x : (c == 1 ? id.y : id.z);
      return mk(mtab[9 * m + 3 + 2 * pair], mtab[9 * m + 4 + 2 * pair]);
    };
    // T_ij (a f) at this cell, with f = component jc and a = e_pair at point set jc
    // (or 1); the four offsets (d0 along one axis, d0^T along another)
    auto tmean = [&](int jc, int pair, bool weighted, const int (*o)[3]) -> cx<T> {
      cx<T> r = mk((T)0, (T)0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int q = at(o[k][0], o[k][1], o[k][2]);
        cx<T> f = ev[(size_t)jc * n3 + q];
        if (weighted) f = off(q, jc, pair) * f;
        r = r + f;
      }
      return scale(r, (T)0.25);
    };
    auto tmean_c = [&](int jc, int pair, int wc, const int (*o)[3]) -> cx<T> {   // T^T (conj(a) f), a at set wc
      cx<T> r = mk((T)0, (T)0);
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int q = at(o[k][0], o[k][1], o[k][2]);
        r = r + conjg(off(q, wc, pair)) * ev[(size_t)jc * n3 + q];
      }
      return scale(r, (T)0.25);
    };
    // offsets (dz, dy, dx)
    const int t01[4][3] = {{0, 0, 0}, {0, 0, -1}, {0, 1, 0}, {0, 1, -1}};
    const int t01t[4][3] = {{0, 0, 0}, {0, 0, 1}, {0, -1, 0}, {0, -1, 1}};
    const int t02[4][3] = {{0, 0, 0}, {0, 0, -1}, {1, 0, 0}, {1, 0, -1}};
    const int t02t[4][3] = {{0, 0, 0}, {0, 0, 1}, {-1, 0, 0}, {-1, 0, 1}};
    const int t12[4][3] = {{0, 0, 0}, {0, -1, 0}, {1, 0, 0}, {1, -1, 0}};
    const int t12t[4][3] = {{0, 0, 0}, {0, 1, 0}, {-1, 0, 0}, {-1, 1, 0}};
    const uchar4 id = mid[cell];
    const T d1 = mtab[9 * id.x], d2 = mtab[9 * id.y + 1], d3 = mtab[9 * id.z + 2];
    const cx<T> e0 = ev[cell], e1 = ev[n3 + cell], e2 = ev[2 * n3 + cell];
    const T h = (T)0.5;
    // component 0 (E1 points): blocks (0, 1) and (0, 2)
    cx<T> m0 = scale(e0, d1);
    m0 = m0 + scale(off(cell, 0, 0) * tmean(1, 0, false, t01) + tmean(1, 0, true, t01), h);
    m0 = m0 + scale(off(cell, 0, 1) * tmean(2, 1, false, t02) + tmean(2, 1, true, t02), h);
    // component 1 (E2 points): block (1, 0) = (0, 1)^H and block (1, 2)
    cx<T> m1 = scale(e1, d2);
    m1 = m1 + scale(tmean_c(0, 0, 0, t01t) + conjg(off(cell, 1, 0)) * tmean(0, 0, false, t01t), h);
    m1 = m1 + scale(off(cell, 1, 2) * tmean(2, 2, false, t12) + tmean(2, 2, true, t12), h);
    // component 2 (E3 points): blocks (2, 0) = (0, 2)^H and (2, 1) = (1, 2)^H
    cx<T> m2 = scale(e2, d3);
    m2 = m2 + scale(tmean_c(0, 1, 0, t02t) + conjg(off(cell, 2, 1)) * tmean(0, 1, false, t02t), h);
    m2 = m2 + scale(tmean_c(1, 2, 1, t12t) + conjg(off(cell, 2, 2)) * tmean(1, 2, false, t12t), h);
    cx<T>* mo = Mo + v * 3 * n3;
    mo[cell] = scale(m0, s);
    mo[n3 + cell] = scale(m1, s);
    mo[2 * n3 + cell] = scale(m2, s);
  }
}

template <typename T, int N, int AXIS, int OP>
cudaError_t launch_pass(const PassArgs& a, size_t tiles, size_t smem, cudaStream_t st) {
  auto kern = pass_kernel<T, N, AXIS, OP>;
  cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)tiles, Cfg<T, N>::THREADS, smem, st>>>(a);
  return cudaGetLastError();
}

// Three-pass form of the apply (fft3_kernels.cuh): complex64 at N = 32, 64, 128.
template <typename T, int N>
__host__ __device__ constexpr bool has_pass3() {
  return sizeof(T) == 4 && (N == 32 || N == 64 || N == 128);
}
template <typename T, int N, int OP>
cudaError_t launch_pass3(const PassArgs& a, int nv, cudaStream_t st, int xv, int zv);

template <typename T, int N>
cudaError_t run_apply_n(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int chunk, void* sbuf,
                        cudaStream_t st, const KParams* kps, int vec_per_k, bool t0) {
  using C = Cfg<T, N>;
  const bool dbl = sizeof(T) == 8;
  const int n_mat = c->dev.mid ? c->dev.n_mat : 0;
  const size_t smem = C::SMEM;
  // + the gamma kappa.x tile (x POST); + the material table and the tile's ids (z sandwich)
  const size_t post_smem = C::SMEM + (size_t)C::TP * N * sizeof(cx<T>);
  const size_t sandwich_smem = C::SMEM + (((size_t)9 * n_mat * sizeof(T) + 15) & ~(size_t)15) + (size_t)C::TP * N * 4;
  PassArgs a;
  a.lam = dbl ? c->dev.lam64 : c->dev.lam32;
  a.tw = dbl ? c->dev.tw64 : c->dev.tw32;
  a.M = dbl ? c->dev.m64 : c->dev.m32;
  a.mid = c->dev.mid;
  a.mid3 = nullptr;
  a.mtab = dbl ? c->dev.mtab64 : c->dev.mtab32;
  a.mtab12 = dbl ? nullptr : c->dev.mtab12;
  a.n_mat = n_mat;
  a.kp = kp;
  a.kps = kps;
  a.vec_per_k = vec_per_k > 0 ? vec_per_k : 1;
  a.sbuf = sbuf;
  const size_t vlen = (size_t)3 * N * N * N;
  // M_CrossDoF: the z sandwich becomes an inverse z transform, the
  // real-space stencil pass into the scratch after the kappa.x part, and a
  // forward z transform
  const bool crossdof = c->m_kind == PCX_M_CROSSDOF && !t0;
  const int cap = nvec < chunk ? nvec : chunk;   // vectors the scratch holds
  cx<T>* tmp = static_cast<cx<T>*>(sbuf) + (size_t)cap * N * N * N;
  for (int v0 = 0; v0 < nvec; v0 += chunk) {
    const int nv = nvec - v0 < chunk ? nvec - v0 : chunk;
    a.v_base = v0;
    const size_t tiles = (size_t)nv * N * N / C::TP;
    const cx<T>* x = static_cast<const cx<T>*>(X) + (size_t)v0 * vlen;
    cx<T>* y = static_cast<cx<T>*>(Y) + (size_t)v0 * vlen;
    cudaError_t e;
    if (crossdof) {
      a.in = x;
      a.out = y;
      if ((e = launch_pass<T, N, 0, OP_PRE>(a, tiles, smem, st)) != cudaSuccess) return e;
      a.in = y;
      if ((e = launch_pass<T, N, 1, OP_INV>(a, tiles, smem, st)) != cudaSuccess) return e;
      if ((e = launch_pass<T, N, 2, OP_PLAIN_INV>(a, tiles, C::SMEM, st)) != cudaSuccess) return e;
      const size_t total = (size_t)nv * N * N * N;
      size_t blocks = (total + 255) / 256;
      if (blocks > 152u * 16u) blocks = 152u * 16u;
      crossdof_kernel<T><<<(unsigned)blocks, 256, 0, st>>>(y, tmp, static_cast<const uchar4*>(c->dev.mid),
                                                           static_cast<const T*>(a.mtab), N, nv,
                                                           (T)(1.0 / ((double)N * N * N)));
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      a.in = tmp;
      if ((e = launch_pass<T, N, 2, OP_PLAIN_FWD>(a, tiles, C::SMEM, st)) != cudaSuccess) return e;
      a.in = y;
      if ((e = launch_pass<T, N, 1, OP_FWD>(a, tiles, smem, st)) != cudaSuccess) return e;
      if ((e = launch_pass<T, N, 0, OP_POST>(a, tiles, post_smem, st)) != cudaSuccess) return e;
      continue;
    }
    a.in = x;
    a.out = y;
    if constexpr (has_pass3<T, N>()) {
      if (c->apply_path != PCX_APPLY_FIVE_PASS && (c->dev.mid3 || !c->dev.mid)) {
        // three passes, in place on y after the first
        a.mid3 = c->dev.mid3;
        const int xv = c->x3_variant, zv = c->z3_variant;
        if ((e = t0 ? launch_pass3<T, N, OP_PRE_T0>(a, nv, st, xv, zv) : launch_pass3<T, N, OP_PRE>(a, nv, st, xv, zv))
            != cudaSuccess)
          return e;
        a.in = y;
        if ((e = t0 ? launch_pass3<T, N, OP_SANDWICH_EPS>(a, nv, st, xv, zv)
                    : launch_pass3<T, N, OP_SANDWICH>(a, nv, st, xv, zv)) != cudaSuccess)
          return e;
        if ((e = t0 ? launch_pass3<T, N, OP_POST_T0>(a, nv, st, xv, zv) : launch_pass3<T, N, OP_POST>(a, nv, st, xv, zv))
            != cudaSuccess)
          return e;
        continue;
      }
    }
    if ((e = t0 ? launch_pass<T, N, 0, OP_PRE_T0>(a, tiles, smem, st) : launch_pass<T, N, 0, OP_PRE>(a, tiles, smem, st))
        != cudaSuccess)
      return e;
    a.in = y;
    if ((e = launch_pass<T, N, 1, OP_INV>(a, tiles, smem, st)) != cudaSuccess) return e;
    if ((e = t0 ? launch_pass<T, N, 2, OP_SANDWICH_EPS>(a, tiles, sandwich_smem, st)
                : launch_pass<T, N, 2, OP_SANDWICH>(a, tiles, sandwich_smem, st)) != cudaSuccess)
      return e;
    if ((e = launch_pass<T, N, 1, OP_FWD>(a, tiles, smem, st)) != cudaSuccess) return e;
    if ((e = t0 ? launch_pass<T, N, 0, OP_POST_T0>(a, tiles, post_smem, st)
                : launch_pass<T, N, 0, OP_POST>(a, tiles, post_smem, st)) != cudaSuccess)
      return e;
  }
  return cudaSuccess;
}

}  // namespace fftk

template <typename T>
cudaError_t run_apply_t(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int chunk, void* sbuf,
                        const KParams* kps, int vec_per_k, cudaStream_t st, bool t0) {
  switch (c->n) {
    case 8: return fftk::run_apply_n<T, 8>(c, kp, X, Y, nvec, chunk, sbuf, st, kps, vec_per_k, t0);
    case 16: return fftk::run_apply_n<T, 16>(c, kp, X, Y, nvec, chunk, sbuf, st, kps, vec_per_k, t0);
    case 32: return fftk::run_apply_n<T, 32>(c, kp, X, Y, nvec, chunk, sbuf, st, kps, vec_per_k, t0);
    case 64: return fftk::run_apply_n<T, 64>(c, kp, X, Y, nvec, chunk, sbuf, st, kps, vec_per_k, t0);
    case 128: return fftk::run_apply_n<T, 128>(c, kp, X, Y, nvec, chunk, sbuf, st, kps, vec_per_k, t0);
    case 256: return fftk::run_apply_n<T, 256>(c, kp, X, Y, nvec, chunk, sbuf, st, kps, vec_per_k, t0);
  }
  return cudaErrorInvalidValue;
}

// Unnormalised 3D DFT of every component of nvec vectors, X -> Y (Y may be
// X): dir > 0 positive exponent (N^{3/2} F3_3), dir < 0 negative exponent
// (N^{3/2} F3_3^H).  Three passes, x then y then z, the last two in place.
namespace fftk {
template <typename T, int N>
cudaError_t run_fft_n(const pcx_ctx* c, const void* X, void* Y, int nvec, int dir, cudaStream_t st) {
  using C = Cfg<T, N>;
  const bool dbl = sizeof(T) == 8;
  PassArgs a{};
  a.lam = dbl ? c->dev.lam64 : c->dev.lam32;
  a.tw = dbl ? c->dev.tw64 : c->dev.tw32;
  a.kp = KParams{};
  const size_t tiles = (size_t)nvec * N * N / C::TP;
  cudaError_t e;
  a.in = X;
  a.out = Y;
  if (dir > 0) {
    if ((e = launch_pass<T, N, 0, OP_PLAIN_INV>(a, tiles, C::SMEM, st)) != cudaSuccess) return e;
    a.in = Y;
    if ((e = launch_pass<T, N, 1, OP_PLAIN_INV>(a, tiles, C::SMEM, st)) != cudaSuccess) return e;
    return launch_pass<T, N, 2, OP_PLAIN_INV>(a, tiles, C::SMEM, st);
  }
  if ((e = launch_pass<T, N, 0, OP_PLAIN_FWD>(a, tiles, C::SMEM, st)) != cudaSuccess) return e;
  a.in = Y;
  if ((e = launch_pass<T, N, 1, OP_PLAIN_FWD>(a, tiles, C::SMEM, st)) != cudaSuccess) return e;
  return launch_pass<T, N, 2, OP_PLAIN_FWD>(a, tiles, C::SMEM, st);
}
}  // namespace fftk

template <typename T>
cudaError_t run_fft_t(const pcx_ctx* c, const void* X, void* Y, int nvec, int dir, cudaStream_t st) {
  if (nvec == 0) return cudaSuccess;
  switch (c->n) {
    case 8: return fftk::run_fft_n<T, 8>(c, X, Y, nvec, dir, st);
    case 16: return fftk::run_fft_n<T, 16>(c, X, Y, nvec, dir, st);
    case 32: return fftk::run_fft_n<T, 32>(c, X, Y, nvec, dir, st);
    case 64: return fftk::run_fft_n<T, 64>(c, X, Y, nvec, dir, st);
    case 128: return fftk::run_fft_n<T, 128>(c, X, Y, nvec, dir, st);
    case 256: return fftk::run_fft_n<T, 256>(c, X, Y, nvec, dir, st);
  }
  return cudaErrorInvalidValue;
}

template <typename T>
cudaError_t run_curl_h_t(const pcx_ctx* c, const KParams& kp, const void* X, void* U, int nvec, int pow,
                         cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t total = (size_t)c->n * c->n * c->n * nvec;
  size_t blocks = (total + 255) / 256;
  if (blocks > 152u * 16u) blocks = 152u * 16u;
  const void* lam = sizeof(T) == 8 ? c->dev.lam64 : c->dev.lam32;
  fftk::curl_h_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(static_cast<const cx<T>*>(X), static_cast<cx<T>*>(U),
                                                          static_cast<const cx<T>*>(lam), c->n, nvec, kp, pow);
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_curl_add_t(const pcx_ctx* c, const KParams& kp, const void* Wm, const void* R, void* Y, int nvec,
                           double scale_, int accumulate, cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t total = (size_t)c->n * c->n * c->n * nvec;
  size_t blocks = (total + 255) / 256;
  if (blocks > 152u * 16u) blocks = 152u * 16u;
  const void* lam = sizeof(T) == 8 ? c->dev.lam64 : c->dev.lam32;
  fftk::curl_add_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(
      static_cast<const cx<T>*>(Wm), static_cast<const cx<T>*>(R), static_cast<cx<T>*>(Y),
      static_cast<const cx<T>*>(lam), c->n, nvec, kp, (T)scale_, accumulate);
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_eps_cells_t(const pcx_ctx* c, const void* E, const void* Add, void* Mo, int nvec, double scale_,
                            cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t total = (size_t)c->n * c->n * c->n * nvec;
  size_t blocks = (total + 255) / 256;
  if (blocks > 152u * 16u) blocks = 152u * 16u;
  const bool dbl = sizeof(T) == 8;
  fftk::eps_cells_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(
      static_cast<const cx<T>*>(E), static_cast<const cx<T>*>(Add), static_cast<cx<T>*>(Mo),
      static_cast<const uchar4*>(c->dev.mid), static_cast<const T*>(dbl ? c->dev.mtab64 : c->dev.mtab32),
      static_cast<const T*>(dbl ? c->dev.m64 : c->dev.m32), c->n, nvec, (T)scale_);
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_div_norms_t(const pcx_ctx* c, const KParams& kp, const void* X, int nvec, double* out, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(out, 0, sizeof(double) * 2 * (size_t)nvec, s);
  if (e != cudaSuccess || nvec == 0) return e;
  const size_t n3 = (size_t)c->n * c->n * c->n;
  size_t bx = (n3 + 255) / 256;
  const size_t cap = (size_t)152 * 8 / (size_t)nvec;
  if (bx > cap) bx = cap > 0 ? cap : 1;
  const void* lam = sizeof(T) == 8 ? c->dev.lam64 : c->dev.lam32;
  fftk::div_norm_kernel<T><<<dim3((unsigned)bx, (unsigned)nvec), 256, 0, s>>>(
      static_cast<const cx<T>*>(X), static_cast<const cx<T>*>(lam), c->n, nvec, kp, out);
  return cudaGetLastError();
}

template <typename T>
cudaError_t run_precond_t(const pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, cudaStream_t s) {
  const size_t total = (size_t)c->n * c->n * c->n * nvec;
  const int threads = 256;
  size_t blocks = (total + threads - 1) / threads;
  if (blocks > 152u * 16u) blocks = 152u * 16u;
  const void* lam = sizeof(T) == 8 ? c->dev.lam64 : c->dev.lam32;
  fftk::precond_kernel<T><<<(unsigned)blocks, threads, 0, s>>>(static_cast<const cx<T>*>(R), static_cast<cx<T>*>(W),
                                                               static_cast<const cx<T>*>(lam), c->n, nvec, kp);
  return cudaGetLastError();
}

}  // namespace pcx
