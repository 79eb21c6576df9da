// The matrix-free apply of the compensated operator in the Fourier basis
// (Sec. 2.4 eq. matrixfree_kcform with the factorisation of Prop. 2.8):
//
//   u = K_A^H x = -conj(kappa) x x          (per Fourier mode)
//   e = F3 u                                 (inverse DFT, positive exponent)
//   m = M e / N^3                            (per cell, Sec. 3.2.1 M_Trivial)
//   w = DFT(m)                               (negative exponent)
//   y = K_A w + gamma K_B x = kappa x w + gamma conj(kappa) (kappa . x)
//
// and the preconditioner K_P^{-1} (eqs. matrixfree_diagP /
// matrixfree_finalform).
//
// The 3D transforms are split into five pencil passes over the block, each
// a batch of 1D FFTs along one axis done in shared memory; the pointwise
// stages ride in the passes that need all three components of a mode or a
// cell:
//   pass 1  x-axis: C^H  (Fourier) + inverse FFT along x
//   pass 2  y-axis: inverse FFT along y
//   pass 3  z-axis: inverse FFT along z, M sandwich, forward FFT along z
//   pass 4  y-axis: forward FFT along y
//   pass 5  x-axis: forward FFT along x + C w + gamma K_B x
// The output block Y is the work space of passes 2-4 (in place); pass 1 also
// stores gamma (kappa . x) per mode into a scratch array that pass 5 reads
// instead of X.  The block is processed in chunks of vectors small enough
// for the chunk's work space to stay resident in L2 across the five passes.
//
// A CTA holds T pencils x 3 components x N points in shared memory and runs
// Stockham radix-R stages (Govindaraju et al., SC 2008 formulation) with the
// small DFTs in registers.
#include <cuda_runtime.h>

#include <mutex>

#include "cx.cuh"
#include "pcx_internal.h"

// Scratch of pcx_apply_noalloc: a file-scope device array, present on every
// GPU that loads the library until the process exits.  Host code must not
// use this name as an address: the device address comes from
// cudaGetSymbolAddress (noalloc_scratch below).
static __device__ __align__(256) unsigned char g_apply_noalloc_scratch[PCX_NOALLOC_SCRATCH_BYTES];

namespace pcx {
namespace {

enum { OP_PRE = 0, OP_INV = 1, OP_SANDWICH = 2, OP_FWD = 3, OP_POST = 4 };

// Radix plans: elements held per thread per stage E (16 complex floats or 8
// complex doubles), radices R0..R2 with N = R0 R1 R2 and every R <= E.
template <int N, int E>
struct Plan;
template <> struct Plan<8, 16> { static constexpr int R0 = 8, R1 = 0, R2 = 0; };
template <> struct Plan<16, 16> { static constexpr int R0 = 16, R1 = 0, R2 = 0; };
template <> struct Plan<32, 16> { static constexpr int R0 = 8, R1 = 4, R2 = 0; };
template <> struct Plan<64, 16> { static constexpr int R0 = 8, R1 = 8, R2 = 0; };
template <> struct Plan<128, 16> { static constexpr int R0 = 16, R1 = 8, R2 = 0; };
template <> struct Plan<256, 16> { static constexpr int R0 = 16, R1 = 16, R2 = 0; };
template <> struct Plan<8, 8> { static constexpr int R0 = 8, R1 = 0, R2 = 0; };
template <> struct Plan<16, 8> { static constexpr int R0 = 4, R1 = 4, R2 = 0; };
template <> struct Plan<32, 8> { static constexpr int R0 = 8, R1 = 4, R2 = 0; };
template <> struct Plan<64, 8> { static constexpr int R0 = 8, R1 = 8, R2 = 0; };
template <> struct Plan<128, 8> { static constexpr int R0 = 8, R1 = 4, R2 = 4; };
template <> struct Plan<256, 8> { static constexpr int R0 = 8, R1 = 8, R2 = 4; };

template <typename T, int N>
struct Cfg {
  static constexpr int E = sizeof(T) == 4 ? 16 : 8;
  static constexpr int TN = sizeof(T) == 4 ? 2048 : 1024;        // pencils x points per component
  static constexpr int T_ = (TN / N < N * N) ? TN / N : N * N;   // pencils per CTA
  static constexpr int THREADS = 3 * T_ * N / E;
  static constexpr int CS = T_ * N + (T_ > N ? T_ : N);            // padded component stride
  static constexpr size_t SMEM = (size_t)(3 * CS + 3 * N) * sizeof(cx<T>);
};

struct PassArgs {
  const void* in;
  void* out;
  void* sbuf;          // [chunk][N^3]: gamma (kappa . x), written by pass 1, read by pass 5
  const void* lam;     // [2][N] Lambda_1, Lambda_0
  const void* tw;      // [N] exp(-2 pi i m / N)
  const void* M;       // [9][N^3] dense cell blocks (when mid == nullptr)
  const void* mid;     // [N^3] uchar4 material ids (E1, E2, E3, V)
  const void* mtab;    // [n_mat][9] block entries per material
  int n_mat;
  KParams kp;
  int axis;
  int op;
};

template <typename T, int N>
struct Tile {
  static constexpr int TP = Cfg<T, N>::T_;
  // shared-memory index of (component c, local pencil t, point n)
  static __device__ __forceinline__ int sidx(int axis, int c, int t, int n) {
    return axis == 0 ? c * Cfg<T, N>::CS + t * (N + 1) + n : c * Cfg<T, N>::CS + n * (TP + 1) + t;
  }
  // global element index (within one vector component block) of pencil q, point n
  static __device__ __forceinline__ size_t gidx(int axis, int q, int n) {
    if (axis == 0) return (size_t)q * N + n;                                    // q = z*N + y
    if (axis == 1) return (size_t)(q / N) * N * N + (size_t)n * N + (q % N);    // q = z*N + x
    return (size_t)n * N * N + q;                                               // q = y*N + x
  }
  // Fourier indices (p1, p2, p3) of pencil q, point n
  static __device__ __forceinline__ void modes(int axis, int q, int n, int& p1, int& p2, int& p3) {
    if (axis == 0) { p1 = n; p2 = q % N; p3 = q / N; }
    else if (axis == 1) { p1 = q % N; p2 = n; p3 = q / N; }
    else { p1 = q % N; p2 = q / N; p3 = n; }
  }
};

// kappa_i(p) = sum_j b_ji (L1(p_j) + i kt_j L0(p_j)) + i kq_i L0(p_i)
template <typename T>
__device__ __forceinline__ void kappa_at(const cx<T>* lam, int n, const KParams& kp, int p1, int p2, int p3,
                                         cx<T> kap[3]) {
  const int p[3] = {p1, p2, p3};
  cx<T> s[3];
#pragma unroll
  for (int j = 0; j < 3; ++j) {
    cx<T> l1 = lam[p[j]], l0 = lam[n + p[j]];
    T kt = (T)kp.kt[j];
    s[j] = mk(l1.x - kt * l0.y, l1.y + kt * l0.x);
  }
  if (kp.diag_b) {
#pragma unroll
    for (int i = 0; i < 3; ++i) kap[i] = scale(s[i], (T)kp.b[4 * i]);
  } else {
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      kap[i] = mk((T)0, (T)0);
#pragma unroll
      for (int j = 0; j < 3; ++j) kap[i] = mk(fma((T)kp.b[3 * j + i], s[j].x, kap[i].x), fma((T)kp.b[3 * j + i], s[j].y, kap[i].y));
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (kp.kq[i] != 0.0) {
      cx<T> l0 = lam[n + p[i]];
      T kq = (T)kp.kq[i];
      kap[i] = mk(kap[i].x - kq * l0.y, kap[i].y + kq * l0.x);
    }
  }
}

// One Stockham stage of radix R on every sequence of the tile (in place,
// through registers).  Ns = product of the radices already done.
template <typename T, int N, int R, int DIR>
__device__ __forceinline__ void stage(cx<T>* s, const cx<T>* tw, int axis, int Ns) {
  using C = Cfg<T, N>;
  constexpr int TP = C::T_;
  constexpr int NB = N / R;                       // butterflies per sequence
  constexpr int PER = C::E / R;                   // butterflies per thread
  cx<T> v[PER][R];
  int tt[PER], jj[PER], cc[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int w = threadIdx.x + i * C::THREADS;
    tt[i] = w % TP;
    jj[i] = (w / TP) % NB;
    cc[i] = w / (TP * NB);
#pragma unroll
    for (int r = 0; r < R; ++r) v[i][r] = s[Tile<T, N>::sidx(axis, cc[i], tt[i], jj[i] + r * NB)];
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int k = jj[i] % Ns;
    const int step = N / (Ns * R);
#pragma unroll
    for (int r = 1; r < R; ++r) {
      cx<T> w = tw[r * k * step];
      if (DIR > 0) w.y = -w.y;
      v[i][r] = v[i][r] * w;
    }
    dft<R, DIR>(v[i]);
    const int base = (jj[i] / Ns) * Ns * R + k;
#pragma unroll
    for (int r = 0; r < R; ++r) s[Tile<T, N>::sidx(axis, cc[i], tt[i], base + r * Ns)] = v[i][r];
  }
  __syncthreads();
}

template <typename T, int N, int DIR>
__device__ __forceinline__ void fft_tile(cx<T>* s, const cx<T>* tw, int axis) {
  using P = Plan<N, Cfg<T, N>::E>;
  stage<T, N, P::R0, DIR>(s, tw, axis, 1);
  if constexpr (P::R1 > 0) stage<T, N, P::R1, DIR>(s, tw, axis, P::R0);
  if constexpr (P::R2 > 0) stage<T, N, P::R2, DIR>(s, tw, axis, P::R0 * P::R1);
}

template <typename T, int N>
__global__ void __launch_bounds__(Cfg<T, N>::THREADS) pass_kernel(PassArgs a) {
  using C = Cfg<T, N>;
  using TL = Tile<T, N>;
  constexpr int TP = C::T_;
  constexpr size_t N2 = (size_t)N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = s + 3 * C::CS;
  cx<T>* lam = tw + N;
  T* mtab = reinterpret_cast<T*>(lam + 2 * N);

  const cx<T>* gtw = static_cast<const cx<T>*>(a.tw);
  const cx<T>* glam = static_cast<const cx<T>*>(a.lam);
  for (int i = threadIdx.x; i < N; i += C::THREADS) tw[i] = gtw[i];
  for (int i = threadIdx.x; i < 2 * N; i += C::THREADS) lam[i] = glam[i];
  if (a.op == OP_SANDWICH && a.mid) {
    const T* gt = static_cast<const T*>(a.mtab);
    for (int i = threadIdx.x; i < 9 * a.n_mat; i += C::THREADS) mtab[i] = gt[i];
  }

  const size_t q0 = (size_t)blockIdx.x * TP;       // first pencil (global across vectors)
  const size_t v = q0 / N2;
  const int qb = (int)(q0 % N2);
  const int axis = a.axis;
  const cx<T>* in = static_cast<const cx<T>*>(a.in) + v * 3 * N3;
  cx<T>* out = static_cast<cx<T>*>(a.out) + v * 3 * N3;

  // load the tile: consecutive threads walk the memory-contiguous index, two
  // complex numbers (16 bytes) per access for complex64
  if constexpr (sizeof(T) == 4) {
    for (int w2 = threadIdx.x; w2 < 3 * TP * N / 2; w2 += C::THREADS) {
      const int w = 2 * w2;
      const int c = w / (TP * N), rem = w % (TP * N);
      const int t = axis == 0 ? rem / N : rem % TP;
      const int n = axis == 0 ? rem % N : rem / TP;
      const float4 v4 = *reinterpret_cast<const float4*>(in + c * N3 + TL::gidx(axis, qb + t, n));
      s[TL::sidx(axis, c, t, n)] = mk((T)v4.x, (T)v4.y);
      s[axis == 0 ? TL::sidx(axis, c, t, n + 1) : TL::sidx(axis, c, t + 1, n)] = mk((T)v4.z, (T)v4.w);
    }
  } else {
    for (int w = threadIdx.x; w < 3 * TP * N; w += C::THREADS) {
      const int c = w / (TP * N), rem = w % (TP * N);
      const int t = axis == 0 ? rem / N : rem % TP;
      const int n = axis == 0 ? rem % N : rem / TP;
      s[TL::sidx(axis, c, t, n)] = in[c * N3 + TL::gidx(axis, qb + t, n)];
    }
  }
  __syncthreads();

  if (a.op == OP_PRE) {   // u = K_A^H x = -conj(kappa) x x
    for (int w = threadIdx.x; w < TP * N; w += C::THREADS) {
      const int t = axis == 0 ? w / N : w % TP;
      const int n = axis == 0 ? w % N : w / TP;
      int p1, p2, p3;
      TL::modes(axis, qb + t, n, p1, p2, p3);
      cx<T> kap[3];
      kappa_at<T>(lam, N, a.kp, p1, p2, p3, kap);
      cx<T> x0 = s[TL::sidx(axis, 0, t, n)], x1 = s[TL::sidx(axis, 1, t, n)], x2 = s[TL::sidx(axis, 2, t, n)];
      const cx<T> sk = cfma(kap[2], x2, cfma(kap[1], x1, kap[0] * x0));
      static_cast<cx<T>*>(a.sbuf)[v * N3 + TL::gidx(axis, qb + t, n)] = scale(sk, (T)a.kp.gamma);
      // conj(kappa_2) x1 - ... written with conj-multiplies
      cx<T> u0 = cfma_conj(kap[2], x1, scale(cfma_conj(kap[1], x2, mk((T)0, (T)0)), (T)-1));
      cx<T> u1 = cfma_conj(kap[0], x2, scale(cfma_conj(kap[2], x0, mk((T)0, (T)0)), (T)-1));
      cx<T> u2 = cfma_conj(kap[1], x0, scale(cfma_conj(kap[0], x1, mk((T)0, (T)0)), (T)-1));
      s[TL::sidx(axis, 0, t, n)] = u0;
      s[TL::sidx(axis, 1, t, n)] = u1;
      s[TL::sidx(axis, 2, t, n)] = u2;
    }
    __syncthreads();
  }

  if (a.op == OP_PRE || a.op == OP_INV || a.op == OP_SANDWICH) fft_tile<T, N, +1>(s, tw, axis);
  else fft_tile<T, N, -1>(s, tw, axis);

  if (a.op == OP_SANDWICH) {   // m = M e / N^3 per cell (axis == 2: q = y*N + x, n = z)
    const T* M = static_cast<const T*>(a.M);
    const uchar4* mid = static_cast<const uchar4*>(a.mid);
    const T inv_n3 = (T)(1.0 / (double)N3);
    for (int w = threadIdx.x; w < TP * N; w += C::THREADS) {
      const int t = w % TP, n = w / TP;
      const size_t cell = (size_t)n * N2 + (qb + t);
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
        d2 = M[N3 + cell];
        d3 = M[2 * N3 + cell];
        o12 = mk(M[3 * N3 + cell], M[4 * N3 + cell]);
        o13 = mk(M[5 * N3 + cell], M[6 * N3 + cell]);
        o23 = mk(M[7 * N3 + cell], M[8 * N3 + cell]);
      }
      const int i0 = TL::sidx(2, 0, t, n), i1 = TL::sidx(2, 1, t, n), i2 = TL::sidx(2, 2, t, n);
      const cx<T> e0 = s[i0], e1 = s[i1], e2 = s[i2];
      cx<T> m0 = cfma(o13, e2, cfma(o12, e1, scale(e0, d1)));
      cx<T> m1 = cfma(o23, e2, cfma_conj(o12, e0, scale(e1, d2)));
      cx<T> m2 = cfma_conj(o23, e1, cfma_conj(o13, e0, scale(e2, d3)));
      s[i0] = scale(m0, inv_n3);
      s[i1] = scale(m1, inv_n3);
      s[i2] = scale(m2, inv_n3);
    }
    __syncthreads();
    fft_tile<T, N, -1>(s, tw, axis);
  }

  if (a.op == OP_POST) {   // y = kappa x w + gamma conj(kappa) (kappa . x)
    const cx<T>* sb = static_cast<const cx<T>*>(a.sbuf) + v * N3;
    for (int w = threadIdx.x; w < TP * N; w += C::THREADS) {
      const int t = axis == 0 ? w / N : w % TP;
      const int n = axis == 0 ? w % N : w / TP;
      int p1, p2, p3;
      TL::modes(axis, qb + t, n, p1, p2, p3);
      cx<T> kap[3];
      kappa_at<T>(lam, N, a.kp, p1, p2, p3, kap);
      const size_t g = TL::gidx(axis, qb + t, n);
      const cx<T> w0 = s[TL::sidx(axis, 0, t, n)], w1 = s[TL::sidx(axis, 1, t, n)], w2 = s[TL::sidx(axis, 2, t, n)];
      const cx<T> sk = sb[g];
      cx<T> y0 = cfma_conj(kap[0], sk, cfma(kap[1], w2, scale(kap[2] * w1, (T)-1)));
      cx<T> y1 = cfma_conj(kap[1], sk, cfma(kap[2], w0, scale(kap[0] * w2, (T)-1)));
      cx<T> y2 = cfma_conj(kap[2], sk, cfma(kap[0], w1, scale(kap[1] * w0, (T)-1)));
      out[g] = y0;
      out[N3 + g] = y1;
      out[2 * N3 + g] = y2;
    }
    return;
  }

  for (int w = threadIdx.x; w < 3 * TP * N; w += C::THREADS) {
    const int c = w / (TP * N), rem = w % (TP * N);
    const int t = axis == 0 ? rem / N : rem % TP;
    const int n = axis == 0 ? rem % N : rem / TP;
    out[c * N3 + TL::gidx(axis, qb + t, n)] = s[TL::sidx(axis, c, t, n)];
  }
}

// W = K_P^{-1} R per mode: r/|k|^2 + (1/gamma - 1) conj(k) (k . r) / |k|^4.
template <typename T>
__global__ void precond_kernel(const cx<T>* __restrict__ R, cx<T>* __restrict__ W, const cx<T>* __restrict__ lam,
                               int n, int nvec, KParams kp) {
  const size_t n3 = (size_t)n * n * n;
  const size_t total = n3 * nvec;
  const T cg = (T)(1.0 / kp.gamma - 1.0);
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const size_t v = e / n3, mode = e % n3;
    const int p1 = (int)(mode % n), p2 = (int)((mode / n) % n), p3 = (int)(mode / ((size_t)n * n));
    cx<T> kap[3];
    kappa_at<T>(lam, n, kp, p1, p2, p3, kap);
    const size_t base = v * 3 * n3 + mode;
    const cx<T> r0 = R[base], r1 = R[base + n3], r2 = R[base + 2 * n3];
    const T k2 = norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]);
    cx<T> w0, w1, w2;
    if (k2 > (T)0) {
      const T ik2 = (T)1 / k2;
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

template <typename T, int N>
cudaError_t run_apply(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int chunk, void* sbuf,
                      cudaStream_t st) {
  using C = Cfg<T, N>;
  const bool dbl = sizeof(T) == 8;
  const int n_mat = c->dev.mid ? c->dev.n_mat : 0;
  const size_t smem = C::SMEM + (size_t)9 * n_mat * sizeof(T);
  cudaError_t e = cudaFuncSetAttribute(pass_kernel<T, N>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(pass_kernel<T, N>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             cudaSharedmemCarveoutMaxShared);
  if (e != cudaSuccess) return e;
  PassArgs a;
  a.lam = dbl ? c->dev.lam64 : c->dev.lam32;
  a.tw = dbl ? c->dev.tw64 : c->dev.tw32;
  a.M = dbl ? c->dev.m64 : c->dev.m32;
  a.mid = c->dev.mid;
  a.mtab = dbl ? c->dev.mtab64 : c->dev.mtab32;
  a.n_mat = n_mat;
  a.kp = kp;
  a.sbuf = sbuf;
  const size_t vlen = (size_t)3 * N * N * N;
  const int axes[5] = {0, 1, 2, 1, 0};
  const int ops[5] = {OP_PRE, OP_INV, OP_SANDWICH, OP_FWD, OP_POST};
  for (int v0 = 0; v0 < nvec; v0 += chunk) {
    const int nv = nvec - v0 < chunk ? nvec - v0 : chunk;
    const size_t tiles = (size_t)nv * N * N / C::T_;
    const cx<T>* x = static_cast<const cx<T>*>(X) + (size_t)v0 * vlen;
    cx<T>* y = static_cast<cx<T>*>(Y) + (size_t)v0 * vlen;
    for (int p = 0; p < 5; ++p) {
      a.axis = axes[p];
      a.op = ops[p];
      a.in = p == 0 ? static_cast<const void*>(x) : static_cast<const void*>(y);
      a.out = y;
      pass_kernel<T, N><<<(unsigned)tiles, C::THREADS, smem, st>>>(a);
      e = cudaGetLastError();
      if (e != cudaSuccess) return e;
    }
  }
  return cudaSuccess;
}

template <typename T>
cudaError_t dispatch_apply(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int chunk,
                           void* sbuf, cudaStream_t st) {
  switch (c->n) {
    case 8: return run_apply<T, 8>(c, kp, X, Y, nvec, chunk, sbuf, st);
    case 16: return run_apply<T, 16>(c, kp, X, Y, nvec, chunk, sbuf, st);
    case 32: return run_apply<T, 32>(c, kp, X, Y, nvec, chunk, sbuf, st);
    case 64: return run_apply<T, 64>(c, kp, X, Y, nvec, chunk, sbuf, st);
    case 128: return run_apply<T, 128>(c, kp, X, Y, nvec, chunk, sbuf, st);
    case 256: return run_apply<T, 256>(c, kp, X, Y, nvec, chunk, sbuf, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace

int apply_chunk(const pcx_ctx* c, int precision) {
  if (c->apply_chunk > 0) return c->apply_chunk;
  const size_t vbytes = (size_t)3 * c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8);
  const size_t l2 = c->l2_bytes ? c->l2_bytes : ((size_t)126 << 20);
  const size_t k = (l2 / 2) / vbytes;
  return (int)(k < 1 ? 1 : (k > 64 ? 64 : k));
}

size_t apply_scratch_bytes(const pcx_ctx* c, int precision, int nvec) {
  const int chunk = apply_chunk(c, precision);
  const int nv = nvec < chunk ? nvec : chunk;
  return (size_t)nv * c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8);
}

cudaError_t launch_apply_scratch(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int precision,
                                 void* scratch, cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const int chunk = apply_chunk(c, precision);
  return precision == PCX_FP64 ? dispatch_apply<double>(c, kp, X, Y, nvec, chunk, scratch, s)
                               : dispatch_apply<float>(c, kp, X, Y, nvec, chunk, scratch, s);
}

// Device address of g_apply_noalloc_scratch on the current device, looked up
// once per device (the first pcx_apply_noalloc call on that device).
static cudaError_t noalloc_scratch(void** out) {
  static std::mutex mu;
  static void* ptr[256] = {nullptr};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 256) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(mu);
  if (!ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_apply_noalloc_scratch);
    if (e != cudaSuccess) return e;
    ptr[dev] = p;
  }
  *out = ptr[dev];
  return cudaSuccess;
}

cudaError_t launch_apply_noalloc(const pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int precision,
                                 cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t per_vec = (size_t)c->n * c->n * c->n * (precision == PCX_FP64 ? 16 : 8);
  if (per_vec > (size_t)PCX_NOALLOC_SCRATCH_BYTES) return cudaErrorInvalidValue;
  void* scratch = nullptr;
  cudaError_t e = noalloc_scratch(&scratch);
  if (e != cudaSuccess) return e;
  int chunk = apply_chunk(c, precision);
  const int fit = (int)((size_t)PCX_NOALLOC_SCRATCH_BYTES / per_vec);
  if (chunk > fit) chunk = fit;
  return precision == PCX_FP64 ? dispatch_apply<double>(c, kp, X, Y, nvec, chunk, scratch, s)
                               : dispatch_apply<float>(c, kp, X, Y, nvec, chunk, scratch, s);
}

cudaError_t launch_apply(pcx_ctx* c, const KParams& kp, const void* X, void* Y, int nvec, int precision,
                         cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t need = apply_scratch_bytes(c, precision, nvec);
  if (need > c->scratch_bytes) {
    // the previous scratch may still be in use by work queued on another stream
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return e;
    if (c->scratch) cudaFree(c->scratch);
    c->scratch = nullptr;
    c->scratch_bytes = 0;
    e = cudaMalloc(&c->scratch, need);
    if (e != cudaSuccess) return e;
    c->scratch_bytes = need;
  }
  return launch_apply_scratch(c, kp, X, Y, nvec, precision, c->scratch, s);
}

cudaError_t launch_precond(const pcx_ctx* c, const KParams& kp, const void* R, void* W, int nvec, int precision,
                           cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const size_t total = (size_t)c->n * c->n * c->n * nvec;
  const int threads = 256;
  const unsigned blocks = (unsigned)std::min<size_t>((total + threads - 1) / threads, 152u * 16u);
  if (precision == PCX_FP64)
    precond_kernel<double><<<blocks, threads, 0, s>>>(static_cast<const cx<double>*>(R), static_cast<cx<double>*>(W),
                                                      static_cast<const cx<double>*>(c->dev.lam64), c->n, nvec, kp);
  else
    precond_kernel<float><<<blocks, threads, 0, s>>>(static_cast<const cx<float>*>(R), static_cast<cx<float>*>(W),
                                                     static_cast<const cx<float>*>(c->dev.lam32), c->n, nvec, kp);
  return cudaGetLastError();
}

}  // namespace pcx
