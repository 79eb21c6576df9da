// Three-pass form of the compensated-operator apply (Sec. 2.4 eq.
// matrixfree_kcform, factorised as in Prop. 2.8) for complex64 at
// N = 32, 64, 128.
//
// The five-pass chain (fft_kernels.cuh) moves every vector through HBM five
// times.  Here the two y transforms are split four-step (N = RA RB) and
// folded into the other passes, so each vector makes three round trips:
//
//   pass A (x tiles)  C^H and the gamma kappa.x scratch on load, inverse x
//                     DFT, then the RA-point half of the inverse y DFT
//   pass B (z tiles)  the RB-point half of the inverse y DFT on load,
//                     inverse z DFT, M per cell, forward z DFT, the RB-point
//                     half of the forward y DFT on store
//   pass C (x tiles)  the RA-point half of the forward y DFT on load,
//                     forward x DFT, C w + gamma conj(kappa) (kappa.x) on
//                     store
//
// Inverse y DFT (positive exponent), input row p = RB n1 + n2, output row
// k = k1 + RA k2:
//   T[k1][n2] = e^{+2 pi i n2 k1 / N} sum_n1 X[RB n1 + n2] e^{+2 pi i n1 k1 / RA}   (pass A)
//   Y[k1 + RA k2] = sum_n2 T[k1][n2] e^{+2 pi i n2 k2 / RB}                           (pass B)
// Forward y DFT (negative exponent), input row y = k1 + RA k2, output row
// m = m1 + RB m2:
//   U[k1][m1] = e^{-2 pi i k1 m1 / N} sum_k2 E[k1 + RA k2] e^{-2 pi i k2 m1 / RB}     (pass B)
//   W[m1 + RB m2] = sum_k1 U[k1][m1] e^{-2 pi i k1 m2 / RA}                           (pass C)
// The intermediates T and U are kept in the natural [c][z][y][x] layout of
// the output buffer with T[k1][n2] (and U[k1][m1]) in row RB k1 + n2.  Then
// pass A writes exactly the rows it reads (RB n1 + n2 for its n2), pass B
// reads and writes the RB consecutive rows RB k1 .. RB k1 + RB - 1 of its
// x columns, and pass C reads and writes the rows m1 + RB m2 of its m1: all
// three run in place on the output buffer.
#pragma once

#include <atomic>
#include <cstdint>
#include <type_traits>

#include "fft_kernels.cuh"

namespace pcx {
namespace fftk {

template <int N>
struct YSplit;
template <> struct YSplit<32> { static constexpr int RA = 8, RB = 4; };
template <> struct YSplit<64> { static constexpr int RA = 8, RB = 8; };
template <> struct YSplit<128> { static constexpr int RA = 16, RB = 8; };

// Geometry of the z tiles (pass B): RB rows x TPX columns of z pencils, at
// least 32 bytes of consecutive x per row so that every global access of
// the pass fills whole 32-byte sectors.  At N = 128 that is 32 pencils
// (96 KB of complex64 for the three components), two CTAs per SM of 256
// threads with 48 elements per thread and stage: the fused inverse-stage /
// M / forward-stage step holds three components of eight points, which
// needs more than the 80 registers a 384-thread CTA could have.
#ifndef PCX_Z128_TN
#define PCX_Z128_TN 4096
#endif
#ifndef PCX_Z128_E
#define PCX_Z128_E 48
#endif
#ifndef PCX_Z128_MINB
#define PCX_Z128_MINB 2
#endif
template <int N>
struct ZGeom {
  static constexpr int TN = 2048, E = 16, MINB = 2;
};
template <> struct ZGeom<128> { static constexpr int TN = PCX_Z128_TN, E = PCX_Z128_E, MINB = PCX_Z128_MINB; };

// Row padding of the z tiles.  Pass B's y DFTs stage two x columns per
// thread (one 16-byte global access); the lanes of a half-warp cover H =
// TPX / 2 column pairs at 16 / H points n.  Column xo of a tile row sits at
// pencil position perm(xo) = xo / 2 + H (xo % 2), so the two columns of a
// pair land H apart, and with a row stride SN = H (mod 16) the half-warp's
// 8-byte words n SN + xp (+ H) fall in 16 distinct bank pairs.
template <int N>
struct ZPad {
  static constexpr int TPZ = ZGeom<N>::TN / N;
  static constexpr int H = TPZ / YSplit<N>::RB / 2;
  static constexpr int R = ((H - TPZ) % 16 + 16) % 16;
  static constexpr int V = R == 0 ? 16 : R;
};
template <int TPX>
__host__ __device__ constexpr int zcol_pos(int xo) {   // pencil position of tile column xo
  return (xo >> 1) + (xo & 1) * (TPX / 2);
}
template <int TPX>
__host__ __device__ constexpr int zcol_of(int q) {     // tile column at pencil position q
  return q < TPX / 2 ? 2 * q : 2 * (q - TPX / 2) + 1;
}

template <typename T, int N>
struct Cfg3 {
  using C = Cfg<T, N>;                                           // x tiles (passes A and C)
  using CZ = CfgG<T, N, ZGeom<N>::TN, ZGeom<N>::E, ZPad<N>::V>;  // z tiles (pass B)
  static constexpr int TP = C::TP;                  // pencils (rows) per x tile
  static constexpr int THREADS = C::THREADS;
  static constexpr int TPZ = CZ::TP;                // pencils per z tile
  static constexpr int THREADSZ = CZ::THREADS;
  static constexpr int RA = YSplit<N>::RA, RB = YSplit<N>::RB;
  static constexpr int G = TP / RA;                 // row groups of RA rows per x tile
  static constexpr int TPX = TPZ / RB;              // x columns per z tile
  static constexpr int TILES = N * N / TP;          // x tiles per vector
  static constexpr int ZTILES = N * N / TPZ;        // z tiles per vector
  static constexpr int XI_PER_THREAD = 3 * G * N / THREADS;           // row-DFT items (RA points)
  static constexpr int ZI_PER_THREAD = 3 * N * (TPX / 2) / THREADSZ;  // row-DFT items (2 x RB points)
  static_assert(RA * RB == N && G >= 1 && G * RA == TP && TPX * RB == TPZ, "tile split");
  static_assert(TPX % 2 == 0 && XI_PER_THREAD >= 1 && ZI_PER_THREAD >= 1, "work split");
  static_assert(XI_PER_THREAD * THREADS == 3 * G * N && ZI_PER_THREAD * THREADSZ == 3 * N * (TPX / 2),
                "work split");
  // shared memory of the z tile: three components at stride CS (Tile)
  static constexpr size_t ZSMEM_TILE = (size_t)3 * CZ::CS * sizeof(cx<T>);
};

template <int OP>
__host__ __device__ constexpr bool is_z_op() {
  return OP == OP_SANDWICH || OP == OP_SANDWICH_EPS;
}
template <typename T, int N, int OP>
__host__ __device__ constexpr int pass3_threads() {
  return is_z_op<OP>() ? Cfg3<T, N>::THREADSZ : Cfg3<T, N>::THREADS;
}
// Kernel variants the autotuner chooses between at run time (the tile
// shapes themselves are fixed by the geometry above, which the pass-B id
// table depends on).  x tiles (passes A and C): PF rows whose global loads
// are issued together before their arithmetic, and the CTAs per SM the
// registers are sized for (MINB); variant 3 runs pass A as the persistent
// kernel that stages the next tile's rows with asynchronous copies
// (pass3x_async_kernel) and pass C as variant 1.  z tiles (pass B): one tile per CTA (0) or
// the warp-specialised persistent kernel (1).
template <int XV>
struct XVar;
template <> struct XVar<0> { static constexpr int PF = 1, MINB = 3; };
template <> struct XVar<1> { static constexpr int PF = 3, MINB = 3; };
template <> struct XVar<2> { static constexpr int PF = 6, MINB = 2; };
// (X3_VARIANTS, Z3_VARIANTS and the defaults PCX_X3_VARIANT, PCX_Z3_VARIANT
// are in pcx_internal.h, for the host side)
template <typename T, int N, int OP, int XV>
__host__ __device__ constexpr int pass3_minb() {
  return is_z_op<OP>() ? ZGeom<N>::MINB : XVar<XV>::MINB;
}

// Row of pencil t of x tile `tile` (within one vector): z, y, and the n2
// (or m1) index its row group carries.
template <typename T, int N>
__device__ __forceinline__ void x_row(int tile, int t, int& z, int& y, int& j) {
  using C3 = Cfg3<T, N>;
  const int gi = t / C3::RA, n1 = t % C3::RA;
  const int gg = tile * C3::G + gi;
  z = gg / C3::RB;
  j = gg % C3::RB;
  y = C3::RB * n1 + j;
}

// The kappa tables of the x tiles: ka[i][p1] and kb[t][i] with
// kappa_i(p) = ka[i][p1] + kb[t][i] (see pass_kernel).
template <typename T, int N>
__device__ __forceinline__ void x_kappa_tables(const cx<T>* glam, const KParams& kp, int tile, cx<T>* ka, cx<T>* kb) {
  using C3 = Cfg3<T, N>;
  for (int e = threadIdx.x; e < 3 * N + 3 * C3::TP; e += C3::THREADS) {
    if (e < 3 * N) {
      const int i = e / N, p = e % N;
      const cx<T> l1 = glam[p], l0 = glam[N + p];
      const T b0 = (T)kp_b(kp, 0, i);
      const T kt = (T)kp.kt[0];
      cx<T> r = mk(b0 * fma(-kt, l0.y, l1.x), b0 * fma(kt, l0.x, l1.y));
      if (i == 0) r = mk(fma(-(T)kp.kq[0], l0.y, r.x), fma((T)kp.kq[0], l0.x, r.y));
      ka[e] = r;
    } else {
      const int f = e - 3 * N, t = f / 3, i = f % 3;
      int z, y, j;
      x_row<T, N>(tile, t, z, y, j);
      const int p[3] = {0, y, z};
      cx<T> r = mk((T)0, (T)0);
#pragma unroll
      for (int jj = 1; jj < 3; ++jj) {
        const cx<T> l1 = glam[p[jj]], l0 = glam[N + p[jj]];
        const T bj = (T)kp_b(kp, jj, i), kt = (T)kp.kt[jj];
        r = mk(fma(bj, fma(-kt, l0.y, l1.x), r.x), fma(bj, fma(kt, l0.x, l1.y), r.y));
        if (i == jj) r = mk(fma(-(T)kp.kq[jj], l0.y, r.x), fma((T)kp.kq[jj], l0.x, r.y));
      }
      kb[3 * t + i] = r;
    }
  }
}

// The steps of passes A and C on one x tile (16 rows of N points at
// N = 128), shared by the one-tile-per-CTA kernel and pass A's persistent
// one, which stages the next tile's rows with asynchronous copies.  Pass
// A's rows come either straight from global memory or from such a staged
// copy raw[c][t][n] in shared memory; the arithmetic and its order are the
// same in both.
template <typename T, int N, int OP>
struct XTile {
  using C3 = Cfg3<T, N>;
  using C = typename C3::C;
  using TL = Tile<T, N, 0, C>;
  static constexpr int TP = C::TP, RA = C3::RA, RB = C3::RB, G = C3::G;
  static constexpr int N2 = N * N, N3 = N2 * N;
  static constexpr bool PRE = OP == OP_PRE || OP == OP_PRE_T0;
  static constexpr bool T0 = OP == OP_PRE_T0 || OP == OP_POST_T0;
  // THREADS is a multiple of N, so in the row sweeps every thread keeps one
  // point n and walks the rows t = t0, t0 + THREADS / N, ...
  static_assert(C::THREADS % N == 0, "x tiles: whole rows per thread sweep");
  static constexpr int TSTEP = C::THREADS / N;
  static constexpr int NI = (TP + TSTEP - 1) / TSTEP;
  static constexpr int CH = N * (int)sizeof(cx<T>) / 16;   // 16-byte pieces per row
  static constexpr int RAW = 3 * TP * N;                   // entries of a staged tile

  // global offset (within one vector, component 0) of pass A's row t of the tile
  static __device__ __forceinline__ int raw_row(int tile, int t) {
    int z, y, j;
    x_row<T, N>(tile, t, z, y, j);
    return z * N2 + y * N;
  }

  // asynchronous copies of pass A's 3 TP input rows into raw (16-byte
  // pieces; the vector's base must be 16-byte aligned, which the launcher
  // checks); completion: cp.async.wait_all by every thread, then a barrier
  static __device__ __forceinline__ void stage_rows(cx<T>* raw, const cx<T>* in, int tile) {
    static_assert(CH * 16 == N * (int)sizeof(cx<T>), "whole 16-byte pieces per row");
    for (int q = threadIdx.x; q < 3 * TP * CH; q += C::THREADS) {
      const int ch = q % CH, t = (q / CH) % TP, c = q / (CH * TP);
      const char* src = reinterpret_cast<const char*>(in + (size_t)c * N3 + raw_row(tile, t)) + 16 * ch;
      const unsigned dst =
          (unsigned)__cvta_generic_to_shared(reinterpret_cast<char*>(raw + (size_t)(c * TP + t) * N) + 16 * ch);
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(dst), "l"(src) : "memory");
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  }
  static __device__ __forceinline__ void wait_rows() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

  // Pass A, first step: u = -conj(kappa) x x per mode into the tile and
  // gamma_p kappa.x to the scratch sb (T0: u / |k|^2 and
  // kappa.x / (gamma_p |k|^4)); x from global memory (FROM_RAW false, PF
  // rows' loads in flight together) or from the staged rows.  The kappa
  // tables must be visible.
  template <int PF, bool FROM_RAW>
  static __device__ __forceinline__ void pre_rows(cx<T>* s, const cx<T>* in, const cx<T>* raw, cx<T>* sb,
                                                  const cx<T>* ka, const cx<T>* kb, const KParams& kp, int tile) {
    const T gam = (T)kp.gamma;
    const T igam = (T)(1.0 / kp.gamma);
    const int n = threadIdx.x % N, t0 = threadIdx.x / N;
    cx<T> kan[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) kan[i] = ka[i * N + n];
    constexpr int PFE = PF < NI ? PF : NI;
#pragma unroll
    for (int i0 = 0; i0 < NI; i0 += PFE) {
      // the rows of this batch: their loads in flight together
      cx<T> xv[PFE][3];
      int gv[PFE];
#pragma unroll
      for (int u = 0; u < PFE; ++u) {
        const int t = t0 + (i0 + u) * TSTEP;
        if (i0 + u < NI && t < TP) {
          int z, y, j;
          x_row<T, N>(tile, t, z, y, j);
          gv[u] = z * N2 + y * N + n;
#pragma unroll
          for (int c = 0; c < 3; ++c) {
            if constexpr (FROM_RAW) xv[u][c] = raw[(c * TP + t) * N + n];
            else xv[u][c] = in[c * N3 + gv[u]];
          }
        }
      }
#pragma unroll
      for (int u = 0; u < PFE; ++u) {
        const int t = t0 + (i0 + u) * TSTEP;
        if (i0 + u >= NI || t >= TP) break;
        const int g = gv[u];
        const cx<T> x0 = xv[u][0], x1 = xv[u][1], x2 = xv[u][2];
        cx<T> kap[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) kap[i] = kan[i] + kb[3 * t + i];
        T su = (T)1, ss = gam;
        if constexpr (T0) {
          const T k2 = norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]);
          su = k2 > (T)0 ? (T)1 / k2 : (T)0;
          ss = su * su * igam * fftk::penalty_inv_weight(kp, k2);
        } else if (kp.per_mode) {
          ss = gam * fftk::penalty_weight(kp, norm2(kap[0]) + norm2(kap[1]) + norm2(kap[2]));
        }
        sb[g] = scale(cfma(kap[2], x2, cfma(kap[1], x1, kap[0] * x0)), ss);
        const cx<T> zr = mk((T)0, (T)0);
        cx<T> u0 = cfma_conj(kap[2], x1, scale(cfma_conj(kap[1], x2, zr), (T)-1));
        cx<T> u1 = cfma_conj(kap[0], x2, scale(cfma_conj(kap[2], x0, zr), (T)-1));
        cx<T> u2 = cfma_conj(kap[1], x0, scale(cfma_conj(kap[0], x1, zr), (T)-1));
        if constexpr (T0) {
          u0 = scale(u0, su);
          u1 = scale(u1, su);
          u2 = scale(u2, su);
        }
        s[TL::sidx(0, t, n)] = u0;
        s[TL::sidx(1, t, n)] = u1;
        s[TL::sidx(2, t, n)] = u2;
      }
    }
  }

  // Pass A, last step: RA-point inverse y DFT over the rows of each group,
  // twiddle e^{+2 pi i n2 k1 / N}, stored to row RB k1 + n2
  static __device__ __forceinline__ void pre_ydft(const cx<T>* s, const cx<T>* tw, cx<T>* out, int tile) {
#pragma unroll
    for (int it = 0; it < C3::XI_PER_THREAD; ++it) {
      const int w = threadIdx.x + it * C::THREADS;
      const int n = w % N, gi = (w / N) % G, c = w / (N * G);
      int z, y, n2;
      x_row<T, N>(tile, gi * RA, z, y, n2);
      cx<T> r[RA];
#pragma unroll
      for (int i = 0; i < RA; ++i) r[i] = s[TL::sidx(c, gi * RA + i, n)];
      dft<RA, +1>(r);
      cx<T>* o = out + (size_t)c * N3 + z * N2 + n2 * N + n;
#pragma unroll
      for (int k1 = 0; k1 < RA; ++k1) {
        cx<T> wt = tw[n2 * k1];
        wt.y = -wt.y;
        o[(RB * k1) * N] = r[k1] * wt;
      }
    }
  }

  // Pass C, first step: RA-point forward y DFT, input rows RB k1 + m1 ->
  // Fourier rows m1 + RB m2 of the tile
  static __device__ __forceinline__ void post_ydft(cx<T>* s, const cx<T>* in, int tile) {
#pragma unroll
    for (int it = 0; it < C3::XI_PER_THREAD; ++it) {
      const int w = threadIdx.x + it * C::THREADS;
      const int n = w % N, gi = (w / N) % G, c = w / (N * G);
      int z, y, m1;
      x_row<T, N>(tile, gi * RA, z, y, m1);
      const cx<T>* ip = in + (size_t)c * N3 + z * N2 + m1 * N + n;
      cx<T> r[RA];
#pragma unroll
      for (int k1 = 0; k1 < RA; ++k1) r[k1] = ip[(RB * k1) * N];
      dft<RA, -1>(r);
#pragma unroll
      for (int m2 = 0; m2 < RA; ++m2) s[TL::sidx(c, gi * RA + m2, n)] = r[m2];
    }
  }

  // Pass C, last step: C w + gamma conj(kappa) (kappa . x) per mode (T0:
  // (C w) / |k|^2 + conj(kappa) s), the scratch read straight from global
  // memory with PF rows' loads in flight together; one point n per thread
  template <int PF>
  static __device__ __forceinline__ void post_rows(const cx<T>* s, const cx<T>* sb, cx<T>* out, const cx<T>* ka,
                                                   const cx<T>* kb, int tile) {
    const int n = threadIdx.x % N, t0 = threadIdx.x / N;
    cx<T> kan[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) kan[i] = ka[i * N + n];
    constexpr int PFE = PF < NI ? PF : NI;
#pragma unroll
    for (int i0 = 0; i0 < NI; i0 += PFE) {
      cx<T> skv[PFE];
      int gv[PFE];
#pragma unroll
      for (int u = 0; u < PFE; ++u) {
        const int t = t0 + (i0 + u) * TSTEP;
        if (i0 + u < NI && t < TP) {
          int z, y, j;
          x_row<T, N>(tile, t, z, y, j);
          gv[u] = z * N2 + y * N + n;
          skv[u] = sb[gv[u]];
        }
      }
#pragma unroll
      for (int u = 0; u < PFE; ++u) {
        const int t = t0 + (i0 + u) * TSTEP;
        if (i0 + u >= NI || t >= TP) break;
        const int g = gv[u];
        const cx<T> sk = skv[u];
        cx<T> kap[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) kap[i] = kan[i] + kb[3 * t + i];
        const cx<T> w0 = s[TL::sidx(0, t, n)], w1 = s[TL::sidx(1, t, n)], w2 = s[TL::sidx(2, t, n)];
        cx<T> c0 = cfma(kap[1], w2, scale(kap[2] * w1, (T)-1));
        cx<T> c1 = cfma(kap[2], w0, scale(kap[0] * w2, (T)-1));
        cx<T> c2 = cfma(kap[0], w1, scale(kap[1] * w0, (T)-1));
        if constexpr (T0) {
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
  }
};

// Where pass B reads its twiddles and its per-material table from.  Pass B
// waits on the queue of shared-memory instructions, and each cell costs five
// loads of material entries; global loads of the small, L1-resident material
// table go through the separate load/store queue instead (PCX_ZB_GTAB = 1,
// FP32, the 16-byte records of DeviceTables::mtab12: 9,554 -> 9,781
// vector-applies/s at 128^3).  Twiddles from the global table
// (PCX_ZB_GTW = 1) were slower (9,249): each twiddle feeds a product at
// once, and the L1 latency sits on that path.
#ifndef PCX_ZB_GTW
#define PCX_ZB_GTW 0
#endif
#ifndef PCX_ZB_GTAB
#define PCX_ZB_GTAB 1
#endif

template <bool G>
__device__ __forceinline__ cx<float> ld_tab(const cx<float>* p) {
  if constexpr (G) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return mk(v.x, v.y);
  } else {
    return *p;
  }
}
template <bool G>
__device__ __forceinline__ cx<double> ld_tab(const cx<double>* p) {
  if constexpr (G) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return mk(v.x, v.y);
  } else {
    return *p;
  }
}
template <bool G, typename V>
__device__ __forceinline__ V ld_tab(const V* p) {
  if constexpr (G) return __ldg(p);
  else return *p;
}

// The three steps of pass B on one z tile, shared by the one-tile-per-CTA
// kernel and the warp-specialised persistent one.  tile = k1 (N / TPX) + xr;
// pencil t = k2 TPX + q holds tile column xo = zcol_of(q) of real row
// y = k1 + RA k2, at x = xr TPX + xo.
template <typename T, int N, int OP>
struct ZTile {
  using C3 = Cfg3<T, N>;
  using C = typename C3::CZ;
  using TL = Tile<T, N, 2, C>;
  static constexpr int TP = C::TP, RA = C3::RA, RB = C3::RB, TPX = C3::TPX;
  static constexpr int N2 = N * N, N3 = N2 * N;
  static constexpr int ITEMS = 3 * N * (TPX / 2);   // y-DFT items (two x columns each)
  static constexpr bool GTW = PCX_ZB_GTW != 0;
  static constexpr bool GTAB = PCX_ZB_GTAB != 0 && sizeof(T) == 4;

  // RB-point inverse y DFT of rows RB k1 + n2 of the tile's columns into
  // the shared tile s, by NTHR threads (tid < NTHR): items tid + it NTHR
  template <int NTHR>
  static __device__ __forceinline__ void load(cx<T>* s, const cx<T>* in, int k1, int x0, int tid) {
    static_assert(ITEMS % NTHR == 0, "whole y-DFT items per thread");
#pragma unroll
    for (int it = 0; it < ITEMS / NTHR; ++it) {
      const int w = tid + it * NTHR;
      const int xp = w % (TPX / 2), z = (w / (TPX / 2)) % N, c = w / ((TPX / 2) * N);
      const cx<T>* ip = in + (size_t)c * N3 + z * N2 + (RB * k1) * N + x0 + 2 * xp;
      cx<T> r0[RB], r1[RB];
#pragma unroll
      for (int n2 = 0; n2 < RB; ++n2) ld2(ip + n2 * N, r0[n2], r1[n2]);
      dft<RB, +1>(r0);
      dft<RB, +1>(r1);
#pragma unroll
      for (int k2 = 0; k2 < RB; ++k2) {
        s[TL::sidx(c, k2 * TPX + zcol_pos<TPX>(2 * xp), z)] = r0[k2];
        s[TL::sidx(c, k2 * TPX + zcol_pos<TPX>(2 * xp + 1), z)] = r1[k2];
      }
    }
  }

  // RB-point forward y DFT over k2 with twiddle e^{-2 pi i k1 m1 / N}, from
  // the shared tile to rows RB k1 + m1
  template <int NTHR>
  static __device__ __forceinline__ void store(const cx<T>* s, const cx<T>* tw, cx<T>* out, int k1, int x0, int tid) {
    static_assert(ITEMS % NTHR == 0, "whole y-DFT items per thread");
#pragma unroll
    for (int it = 0; it < ITEMS / NTHR; ++it) {
      const int w = tid + it * NTHR;
      const int xp = w % (TPX / 2), z = (w / (TPX / 2)) % N, c = w / ((TPX / 2) * N);
      cx<T> r0[RB], r1[RB];
#pragma unroll
      for (int k2 = 0; k2 < RB; ++k2) {
        r0[k2] = s[TL::sidx(c, k2 * TPX + zcol_pos<TPX>(2 * xp), z)];
        r1[k2] = s[TL::sidx(c, k2 * TPX + zcol_pos<TPX>(2 * xp + 1), z)];
      }
      dft<RB, -1>(r0);
      dft<RB, -1>(r1);
      cx<T>* op = out + (size_t)c * N3 + z * N2 + (RB * k1) * N + x0 + 2 * xp;
#pragma unroll
      for (int m1 = 0; m1 < RB; ++m1) {
        const cx<T> wt = ld_tab<GTW>(tw + k1 * m1);
        st2(op + m1 * N, r0[m1] * wt, r1[m1] * wt);
      }
    }
  }

  // z transforms of the tile with plan (R0, R1): the inverse as two
  // Stockham stages (radix R0 at Ns = 1, radix R1 at Ns = R0), the forward
  // as radix R1 at Ns = 1 then radix R0 at Ns = R1.  The inverse's second
  // stage reads and writes the R1 points j + R0 r of a pencil, which are
  // also the inputs of the forward's first stage, so those two stages and
  // the cell-by-cell M between them run in registers on the same points
  // (all three components): two shared-memory round trips fewer.  The
  // forward's first stage leaves element r of butterfly j at position
  // j + R0 r (not at j R1 + r), which its second stage reads back.  Run by
  // the C::THREADS threads tid = threadIdx.x < C::THREADS; SYNC is their
  // barrier.  The tile must be complete in s on entry (the caller's
  // barrier); on return it holds the forward transform, visible to the
  // group.
  template <class SYNC>
  static __device__ __forceinline__ void transform(cx<T>* s, const cx<T>* tw, const T* mtab, const uchar4* tid3,
                                                   const T* M, int k1, int x0) {
    using P = typename C::P;
    constexpr int R0 = P::R0, R1 = P::R1;
    static_assert(P::NST == 2 && R0 * R1 == N, "two-stage z plan");
    stage<T, N, 2, R0, +1, 0, 0, C, SYNC>(s, tw, 1, nullptr, nullptr, 0);
    const T inv_n3 = (T)(1.0 / (double)N3);
    for (int w = threadIdx.x; w < TP * R0; w += C::THREADS) {
      const int t = w % TP, j = w / TP;
      cx<T> v[3][R1];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const cx<T>* sp = s + TL::sidx(c, t, j);
#pragma unroll
        for (int r = 0; r < R1; ++r) v[c][r] = sp[r * R0 * TL::SN];
      }
#pragma unroll
      for (int r = 1; r < R1; ++r) {
        cx<T> wt = ld_tab<GTW>(tw + r * j);   // inverse: e^{+2 pi i r j / N}
        wt.y = -wt.y;
#pragma unroll
        for (int c = 0; c < 3; ++c) v[c][r] = v[c][r] * wt;
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) dft<R1, +1>(v[c]);
#pragma unroll
      for (int r = 0; r < R1; ++r) {
        const int n = j + R0 * r;
        T d1, d2, d3;
        cx<T> o12, o13, o23;
        if (tid3) {
          const uchar4 id = tid3[n * TP + t];
          d1 = ld_tab<GTAB>(mtab + 12 * id.x);
          d2 = ld_tab<GTAB>(mtab + 12 * id.y + 1);
          d3 = ld_tab<GTAB>(mtab + 12 * id.z + 2);
          const T* o = mtab + 12 * id.w;
          if constexpr (sizeof(T) == 4) {
            const float4 q = ld_tab<GTAB>(reinterpret_cast<const float4*>(o + 4));
            const float2 q2 = ld_tab<GTAB>(reinterpret_cast<const float2*>(o + 8));
            o12 = mk(q.x, q.y);
            o13 = mk(q.z, q.w);
            o23 = mk(q2.x, q2.y);
          } else {
            o12 = mk(o[4], o[5]);
            o13 = mk(o[6], o[7]);
            o23 = mk(o[8], o[9]);
          }
        } else {
          const int cell = n * N2 + (k1 + RA * (t / TPX)) * N + x0 + zcol_of<TPX>(t % TPX);
          d1 = M[cell];
          d2 = M[N3 + cell];
          d3 = M[2 * N3 + cell];
          o12 = mk(M[3 * N3 + cell], M[4 * N3 + cell]);
          o13 = mk(M[5 * N3 + cell], M[6 * N3 + cell]);
          o23 = mk(M[7 * N3 + cell], M[8 * N3 + cell]);
        }
        T sc = inv_n3;
        if constexpr (OP == OP_SANDWICH_EPS) {
          // eps = M^{-1} = adj(M) / det(M) on the Hermitian block
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
        const cx<T> e0 = v[0][r], e1 = v[1][r], e2 = v[2][r];
        v[0][r] = scale(cfma(o13, e2, cfma(o12, e1, scale(e0, d1))), sc);
        v[1][r] = scale(cfma(o23, e2, cfma_conj(o12, e0, scale(e1, d2))), sc);
        v[2][r] = scale(cfma_conj(o23, e1, cfma_conj(o13, e0, scale(e2, d3))), sc);
      }
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        dft<R1, -1>(v[c]);
        cx<T>* sp = s + TL::sidx(c, t, j);
#pragma unroll
        for (int r = 0; r < R1; ++r) sp[r * R0 * TL::SN] = v[c][r];
      }
    }
    SYNC::sync();
    // forward second stage (radix R0 at Ns = R1): butterfly jj reads its R0
    // inputs from the consecutive positions R0 jj + q, twiddle
    // e^{-2 pi i q jj / N}, and writes the transform in natural order,
    // positions jj + R1 q
    constexpr int PER = 3 * TP * R1 / C::THREADS;
    static_assert(PER * C::THREADS == 3 * TP * R1, "forward second stage: whole items per thread");
    cx<T> v[PER][R0];
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int w = threadIdx.x + i * C::THREADS;
      const int t = w % TP, jj = (w / TP) % R1, c = w / (TP * R1);
      const cx<T>* sp = s + TL::sidx(c, t, R0 * jj);
#pragma unroll
      for (int q = 0; q < R0; ++q) v[i][q] = sp[q * TL::SN];
    }
    SYNC::sync();
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int w = threadIdx.x + i * C::THREADS;
      const int t = w % TP, jj = (w / TP) % R1, c = w / (TP * R1);
#pragma unroll
      for (int q = 1; q < R0; ++q) v[i][q] = v[i][q] * ld_tab<GTW>(tw + q * jj);
      dft<R0, -1>(v[i]);
      cx<T>* sp = s + TL::sidx(c, t, jj);
#pragma unroll
      for (int q = 0; q < R0; ++q) sp[q * R1 * TL::SN] = v[i][q];
    }
    SYNC::sync();
  }

  // the material table repacked to 12 entries per material: d1 d2 d3 -
  // re12 im12 re13 im13 re23 im23 - -, so that the off-diagonals of a cell
  // come in one 16-byte and one 8-byte load
  static __device__ __forceinline__ void stage_mtab(T* mtab, const void* gmtab, int n_mat, int tid, int nthr) {
    const T* gt = static_cast<const T*>(gmtab);
    for (int i = tid; i < 9 * n_mat; i += nthr) {
      const int m = i / 9, f = i % 9;
      mtab[12 * m + (f < 3 ? f : f + 1)] = gt[i];
    }
  }
};

template <typename T, int N, int OP, int XV>
__global__ void __launch_bounds__(pass3_threads<T, N, OP>(), pass3_minb<T, N, OP, XV>()) pass3_kernel(PassArgs a) {
  constexpr bool ZP = is_z_op<OP>();
  using C3 = Cfg3<T, N>;
  using C = std::conditional_t<ZP, typename C3::CZ, typename C3::C>;
  constexpr int AXIS = ZP ? 2 : 0;
  using TL = Tile<T, N, AXIS, C>;
  constexpr int TP = C::TP;
  constexpr int N2 = N * N, N3 = N2 * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = s + 3 * C::CS;    // the three components at stride CS (see Tile)
  cx<T>* ka = tw + N;          // [3][N]   (x tiles)
  cx<T>* kb = ka + 3 * N;      // [TP][3]  (x tiles)
  T* mtab = reinterpret_cast<T*>(tw + N);   // [n_mat][12] (z tiles, 16-byte aligned)

  constexpr int TILES = ZP ? C3::ZTILES : C3::TILES;
  const size_t v = blockIdx.x / TILES;
  const int tile = (int)(blockIdx.x % TILES);
  const cx<T>* in = static_cast<const cx<T>*>(a.in) + v * 3 * N3;
  cx<T>* out = static_cast<cx<T>*>(a.out) + v * 3 * N3;

  const cx<T>* gtw = static_cast<const cx<T>*>(a.tw);
  for (int i = threadIdx.x; i < N; i += C::THREADS) tw[i] = gtw[i];

  if constexpr (!ZP) {
    // ================= x tiles: pass A (PRE) and pass C (POST) =================
    using XT = XTile<T, N, OP>;
    KParams kp = a.kp;
    if (a.kps) kp = a.kps[(a.v_base + (int)v) / a.vec_per_k];
    x_kappa_tables<T, N>(static_cast<const cx<T>*>(a.lam), kp, tile, ka, kb);
    if constexpr (XT::PRE) {
      cx<T>* sb = static_cast<cx<T>*>(a.sbuf) + v * N3;
      __syncthreads();   // kappa tables
      XT::template pre_rows<XVar<XV>::PF, false>(s, in, nullptr, sb, ka, kb, kp, tile);
      __syncthreads();
      fft_tile<T, N, 0, +1, 0, 0>(s, tw, nullptr, nullptr, 0);
      XT::pre_ydft(s, tw, out, tile);
    } else {
      const cx<T>* sb = static_cast<const cx<T>*>(a.sbuf) + v * N3;
      XT::post_ydft(s, in, tile);
      __syncthreads();
      fft_tile<T, N, 0, -1, 0, 0>(s, tw, nullptr, nullptr, 0);
      XT::template post_rows<XVar<XV>::PF>(s, sb, out, ka, kb, tile);
    }
  } else {
    // ================= z tiles: pass B =================
    using ZT = ZTile<T, N, OP>;
    constexpr int TPX = C3::TPX;
    const int k1 = tile / (N / TPX), x0 = (tile % (N / TPX)) * TPX;
    if (a.mid && !ZT::GTAB) ZT::stage_mtab(mtab, a.mtab, a.n_mat, threadIdx.x, C::THREADS);
    const T* mt = ZT::GTAB ? static_cast<const T*>(a.mtab12) : mtab;
    const cx<T>* twz = ZT::GTW ? gtw : tw;
    ZT::template load<C::THREADS>(s, in, k1, x0, threadIdx.x);
    __syncthreads();   // the tile, the twiddles and the material table
    const uchar4* mid3 = static_cast<const uchar4*>(a.mid3);
    ZT::template transform<CtaSync>(s, twz, mt, mid3 ? mid3 + (size_t)tile * TP * N : nullptr,
                                    static_cast<const T*>(a.M), k1, x0);
    ZT::template store<C::THREADS>(s, twz, out, k1, x0, threadIdx.x);
  }
}

// Pass A as a persistent kernel (x variant 3): CTA b walks x tiles b, b +
// gridDim.x, ... and, once a tile's input rows have been consumed, copies
// the next tile's rows into shared memory with asynchronous copies
// (cp.async, 16-byte pieces), so that they are in flight during the x FFT
// and the y DFT of the current tile.  A tile-per-CTA kernel issues its
// global loads only in its first step.  The arithmetic is XTile's, as in
// pass3_kernel.  Shared memory: the tile, twiddles, kappa tables and one
// staged tile of rows (103 KB at N = 128: two CTAs per SM).  Pass C's
// strided y DFT measured slower from staged rows (431 against 386 us per
// launch of 16 vectors at 128^3), so pass C keeps the tile-per-CTA kernel.
template <typename T, int N>
__host__ __device__ constexpr size_t xasync_raw_offset() {
  using C = typename Cfg3<T, N>::C;
  return (((size_t)3 * C::CS + 4 * N + 3 * C::TP) + 1) & ~(size_t)1;   // entries, 16-byte aligned
}
template <typename T, int N>
__host__ __device__ constexpr size_t xasync_smem() {
  return (xasync_raw_offset<T, N>() + (size_t)XTile<T, N, OP_PRE>::RAW) * sizeof(cx<T>);
}

template <typename T, int N, int OP>
__global__ void __launch_bounds__(Cfg3<T, N>::THREADS, 2) pass3x_async_kernel(PassArgs a, int total_tiles) {
  using C3 = Cfg3<T, N>;
  using C = typename C3::C;
  using XT = XTile<T, N, OP>;
  static_assert(XT::PRE, "pass A only");
  constexpr int N3 = N * N * N, TILES = C3::TILES;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* s = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* tw = s + 3 * C::CS;
  cx<T>* ka = tw + N;       // [3][N]
  cx<T>* kb = ka + 3 * N;   // [TP][3]
  cx<T>* raw = s + xasync_raw_offset<T, N>();
  const cx<T>* gtw = static_cast<const cx<T>*>(a.tw);
  for (int i = threadIdx.x; i < N; i += C::THREADS) tw[i] = gtw[i];
  const cx<T>* gin = static_cast<const cx<T>*>(a.in);
  cx<T>* gout = static_cast<cx<T>*>(a.out);
  const int g0 = blockIdx.x;
  if (g0 < total_tiles) XT::stage_rows(raw, gin + (size_t)(g0 / TILES) * 3 * N3, g0 % TILES);
  for (int g = g0; g < total_tiles; g += gridDim.x) {
    const size_t v = (size_t)(g / TILES);
    const int tile = g % TILES;
    KParams kp = a.kp;
    if (a.kps) kp = a.kps[(a.v_base + (int)v) / a.vec_per_k];
    // the previous tile's last readers of ka, kb and s passed the barrier
    // at the end of its iteration
    x_kappa_tables<T, N>(static_cast<const cx<T>*>(a.lam), kp, tile, ka, kb);
    XT::wait_rows();
    __syncthreads();   // this tile's rows, the kappa tables (and the twiddles)
    XT::template pre_rows<1, true>(s, nullptr, raw, static_cast<cx<T>*>(a.sbuf) + v * N3, ka, kb, kp, tile);
    __syncthreads();   // the rows are consumed; the tile is complete
    const int gn = g + (int)gridDim.x;
    if (gn < total_tiles) XT::stage_rows(raw, gin + (size_t)(gn / TILES) * 3 * N3, gn % TILES);
    fft_tile<T, N, 0, +1, 0, 0>(s, tw, nullptr, nullptr, 0);
    XT::pre_ydft(s, tw, gout + v * 3 * N3, tile);
    __syncthreads();   // s, ka and kb are rewritten by the next tile
  }
  XT::wait_rows();
}

// Pass B as a persistent warp-specialised kernel: one CTA per SM walks z
// tiles blockIdx.x, blockIdx.x + gridDim.x, ... with two tile buffers in
// shared memory.  The first C::THREADS threads (the transform group) run
// the z transforms and M of tile i on buffer i % 2 while the other
// 512 - C::THREADS threads (the I/O group) store tile i - 1 from the other
// buffer and load tile i + 1 into it, so that global traffic and the
// transforms overlap inside the SM.  Hardware named barriers hand the
// buffers over (no spin loop): FULL[b] -- the I/O group arrives once it
// has loaded buffer b, the transform group waits on it; EMPTY[b] -- the
// transform group arrives once it has transformed buffer b, the I/O group
// waits on it before storing that tile and reusing the buffer.  ZB_T is the
// transform group's own barrier between stages, ZB_IO the I/O group's
// between reading a buffer out and refilling it.  Both groups walk the same
// tile sequence, so every phase of every barrier gets all 512 arrivals.
constexpr int ZB_T = 1, ZB_IO = 2, ZB_FULL = 3, ZB_EMPTY = 5;   // FULL 3, 4; EMPTY 5, 6
constexpr int ZWS_THREADS = 512;

__device__ __forceinline__ void zb_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void zb_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;\n" ::"r"(id), "r"(n) : "memory");
}

template <typename T, int N, int OP>
__global__ void __launch_bounds__(ZWS_THREADS, 1) pass3z_ws_kernel(PassArgs a, int total_tiles) {
  using C3 = Cfg3<T, N>;
  using C = typename C3::CZ;
  using ZT = ZTile<T, N, OP>;
  constexpr int CT = C::THREADS, IOT = ZWS_THREADS - CT;
  static_assert(CT % 32 == 0 && IOT >= 32 && IOT % 32 == 0, "whole warps in both groups");
  constexpr int TP = C::TP, TPX = C3::TPX, ZT_N = C3::ZTILES, N3 = N * N * N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  cx<T>* buf0 = reinterpret_cast<cx<T>*>(smem_raw);
  cx<T>* buf1 = buf0 + 3 * C::CS;
  cx<T>* tw = buf1 + 3 * C::CS;
  T* mtab = reinterpret_cast<T*>(tw + N);   // 16-byte aligned: 3 CS and N are even
  const cx<T>* gtw = static_cast<const cx<T>*>(a.tw);
  for (int i = threadIdx.x; i < N; i += ZWS_THREADS) tw[i] = gtw[i];
  if (a.mid && !ZT::GTAB) ZT::stage_mtab(mtab, a.mtab, a.n_mat, threadIdx.x, ZWS_THREADS);
  const T* mt = ZT::GTAB ? static_cast<const T*>(a.mtab12) : mtab;
  const cx<T>* twz = ZT::GTW ? gtw : tw;
  __syncthreads();
  const uchar4* mid3 = static_cast<const uchar4*>(a.mid3);
  if (threadIdx.x < CT) {
    // transform group
    const T* M = static_cast<const T*>(a.M);
    int i = 0;
    for (int g = blockIdx.x; g < total_tiles; g += gridDim.x, ++i) {
      const int b = i & 1;
      const int tile = g % ZT_N;
      const int k1 = tile / (N / TPX), x0 = (tile % (N / TPX)) * TPX;
      zb_sync(ZB_FULL + b, ZWS_THREADS);
      ZT::template transform<GroupSync<ZB_T, CT>>(b ? buf1 : buf0, twz, mt,
                                                  mid3 ? mid3 + (size_t)tile * TP * N : nullptr, M, k1, x0);
      zb_arrive(ZB_EMPTY + b, ZWS_THREADS);
    }
  } else {
    // I/O group: step i stores tile i - 2 (the previous user of buffer
    // i % 2) and loads tile i into it
    const int tid = threadIdx.x - CT;
    const cx<T>* in = static_cast<const cx<T>*>(a.in);
    cx<T>* out = static_cast<cx<T>*>(a.out);
    // this CTA's tile count; steps 0 .. nt + 1 (the last two only store)
    const int nt = (int)blockIdx.x < total_tiles ? (total_tiles - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x
                                                 : 0;
    for (int i = 0; i < nt + 2; ++i) {
      const long long gs = (long long)blockIdx.x + (long long)(i - 2) * gridDim.x;
      const long long gl = (long long)blockIdx.x + (long long)i * gridDim.x;
      const bool st = i >= 2;
      const bool ld = i < nt;
      const int b = i & 1;
      cx<T>* s = b ? buf1 : buf0;
      if (st) {
        const int tile = (int)(gs % ZT_N);
        const size_t v = (size_t)(gs / ZT_N);
        zb_sync(ZB_EMPTY + b, ZWS_THREADS);
        ZT::template store<IOT>(s, twz, out + v * 3 * N3, tile / (N / TPX), (tile % (N / TPX)) * TPX, tid);
      }
      if (ld) {
        if (st) zb_sync(ZB_IO, IOT);   // every read of the buffer done before it is refilled
        const int tile = (int)(gl % ZT_N);
        const size_t v = (size_t)(gl / ZT_N);
        ZT::template load<IOT>(s, in + v * 3 * N3, tile / (N / TPX), (tile % (N / TPX)) * TPX, tid);
        zb_arrive(ZB_FULL + b, ZWS_THREADS);
      }
    }
  }
}

// mid3[tile][w] = mid[cell] for the z tiles of pass B: tile = k1 (N / TPX) +
// xr, w = n TP + t, pencil t = k2 TPX + q holding tile column xo =
// zcol_of(q), cell (x, y, z) = (xr TPX + xo, k1 + RA k2, n).
template <int N>
__global__ void pass3_ids_kernel(const uchar4* __restrict__ mid, uchar4* __restrict__ mid3) {
  using C3 = Cfg3<float, N>;
  constexpr int TP = C3::TPZ, TPX = C3::TPX, RA = C3::RA;
  const size_t total = (size_t)N * N * N;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const int tile = (int)(e / ((size_t)TP * N)), w = (int)(e % ((size_t)TP * N));
    const int k1 = tile / (N / TPX), x0 = (tile % (N / TPX)) * TPX;
    const int t = w % TP, n = w / TP;
    mid3[e] = mid[(size_t)n * N * N + (size_t)(k1 + RA * (t / TPX)) * N + x0 + zcol_of<TPX>(t % TPX)];
  }
}

// One pass of the three-pass chain over nv vectors; the shared memory of
// each tile kind is fixed by its geometry (x tiles: the five-pass x layout
// plus the kappa tables; z tiles: the tile, the twiddles and the material
// table).
template <typename T, int N, int OP, int XV>
cudaError_t launch_pass3_tile(const PassArgs& a, int nv, cudaStream_t st) {
  using C3 = Cfg3<T, N>;
  constexpr bool ZP = is_z_op<OP>();
  size_t smem;
  if constexpr (ZP)
    smem = C3::ZSMEM_TILE + (size_t)N * sizeof(cx<T>) + (((size_t)12 * a.n_mat * sizeof(T) + 15) & ~(size_t)15);
  else
    smem = C3::C::SMEM;
  const size_t tiles = (size_t)nv * (ZP ? C3::ZTILES : C3::TILES);
  auto kern = pass3_kernel<T, N, OP, XV>;
  cudaError_t e = raise_dyn_smem(reinterpret_cast<const void*>(kern), smem);
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)tiles, pass3_threads<T, N, OP>(), smem, st>>>(a);
  return cudaGetLastError();
}

template <typename T, int N, int OP>
cudaError_t launch_pass3_ws(const PassArgs& a, int nv, cudaStream_t st) {
  using C3 = Cfg3<T, N>;
  const size_t smem = 2 * C3::ZSMEM_TILE + (size_t)N * sizeof(cx<T>) +
                      (((size_t)12 * a.n_mat * sizeof(T) + 15) & ~(size_t)15);
  const long long tiles = (long long)nv * C3::ZTILES;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  auto kern = pass3z_ws_kernel<T, N, OP>;
  if ((e = raise_dyn_smem(reinterpret_cast<const void*>(kern), smem)) != cudaSuccess) return e;
  const long long grid = tiles < sms ? tiles : sms;
  if (grid == 0) return cudaSuccess;
  kern<<<(unsigned)grid, ZWS_THREADS, smem, st>>>(a, (int)tiles);
  return cudaGetLastError();
}

template <typename T, int N, int OP>
cudaError_t launch_pass3_async(const PassArgs& a, int nv, cudaStream_t st) {
  using C3 = Cfg3<T, N>;
  const size_t smem = xasync_smem<T, N>();
  const long long tiles = (long long)nv * C3::TILES;
  if (tiles > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (tiles == 0) return cudaSuccess;
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  auto kern = pass3x_async_kernel<T, N, OP>;
  if ((e = raise_dyn_smem(reinterpret_cast<const void*>(kern), smem)) != cudaSuccess) return e;
  // resident CTAs per SM, queried once per device (not inside a capture)
  static std::atomic<int> resident[64];
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  per_sm = resident[dev].load();
  if (per_sm == 0) {
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, C3::THREADS, smem)) != cudaSuccess)
      return e;
    if (per_sm < 1) per_sm = 1;
    resident[dev].store(per_sm);
  }
  const long long fill = (long long)per_sm * sms;
  const long long grid = tiles < fill ? tiles : fill;
  kern<<<(unsigned)grid, C3::THREADS, smem, st>>>(a, (int)tiles);
  return cudaGetLastError();
}

// One pass of the three-pass chain over nv vectors; xv / zv pick the kernel
// variant of the x / z passes (out of range: the build-time default).  The
// asynchronous-copy x kernel (3) needs 16-byte aligned input vectors; other
// inputs take variant 1.
template <typename T, int N, int OP>
cudaError_t launch_pass3(const PassArgs& a, int nv, cudaStream_t st, int xv, int zv) {
  if constexpr (is_z_op<OP>()) {
    if (zv < 0 || zv >= Z3_VARIANTS) zv = PCX_Z3_VARIANT;
    return zv == 1 ? launch_pass3_ws<T, N, OP>(a, nv, st) : launch_pass3_tile<T, N, OP, 0>(a, nv, st);
  } else {
    if (xv < 0 || xv >= X3_VARIANTS) xv = PCX_X3_VARIANT;
    if (xv == 3 && (reinterpret_cast<uintptr_t>(a.in) & 15) != 0) xv = 1;
    switch (xv) {
      case 0:
        return launch_pass3_tile<T, N, OP, 0>(a, nv, st);
      case 2:
        return launch_pass3_tile<T, N, OP, 2>(a, nv, st);
      case 3:   // pass A persistent with staged rows, pass C as variant 1
        if constexpr (XTile<T, N, OP>::PRE) return launch_pass3_async<T, N, OP>(a, nv, st);
        else return launch_pass3_tile<T, N, OP, 1>(a, nv, st);
      default:
        return launch_pass3_tile<T, N, OP, 1>(a, nv, st);
    }
  }
}

// the pass-B order of the material ids (device, N^3 uchar4), built once per context
template <int N>
cudaError_t build_pass3_ids_n(const void* mid, void* mid3, cudaStream_t st) {
  const size_t total = (size_t)N * N * N;
  size_t blocks = (total + 255) / 256;
  if (blocks > 152u * 16u) blocks = 152u * 16u;
  pass3_ids_kernel<N><<<(unsigned)blocks, 256, 0, st>>>(static_cast<const uchar4*>(mid), static_cast<uchar4*>(mid3));
  return cudaGetLastError();
}

}  // namespace fftk
}  // namespace pcx
