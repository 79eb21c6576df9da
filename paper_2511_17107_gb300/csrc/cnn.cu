// Kernels of the learned preconditioner correction, which acts next to eps
// inside the curl-sandwich base preconditioner T0:
//
//   T(r) = T0 r + K_A F3_3^H g(F3_3 K_A^H r / |k|^2) / |k|^2
//
// with g a three-layer circular 3D convolution net (3 x 3 x 3 taps) on the
// real-space field, its hidden channels gated by sigmoid convolutions of the
// 9 reals of the per-cell blocks of M (Sec. 3.2.1).  The net acts on the real
// and imaginary parts of the complex field with shared weights, so T is
// complex-linear.  The paper has no learned component; the operator pieces
// it wraps are eqs. matrixfree_diagP / matrixfree_finalform (K_P^{-1}) and
// the Fourier basis x = F3_3^H H of Sec. 2.4.
//
// Arithmetic and accumulation are FP32; the convolutions optionally round
// their weights to BF16 as they load them (the learned form's BF16 flag).  A convolution CTA
// produces an 8 x 8 x 8 tile of output voxels for every output channel of
// one sample, from a 10 x 10 x 10 halo tile of all input channels staged in
// shared memory (periodic wrap on load).  The weight gradient is a
// per-CTA sum over tiles written to scratch and reduced in a fixed order.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstdint>

#include "cnn.h"
#include "pcx_internal.h"

namespace pcx {
namespace cnn {
namespace {

constexpr int TS = 8;                 // output tile edge
constexpr int HS = TS + 2;            // halo tile edge
constexpr int HV = HS * HS * HS;      // halo voxels
constexpr int TV = TS * TS * TS;      // tile voxels
constexpr int CT = 256;               // threads per CTA (2 voxels each)

__device__ __forceinline__ long long voff(const View& t, int b, int ch, long long v) {
  return (long long)(b / t.split) * t.s_hi + (long long)(b % t.split) * t.s_lo + (long long)ch * t.sc + v * t.sv;
}

__device__ __forceinline__ void tile_origin(int tile, int n, int& z0, int& y0, int& x0) {
  const int tpa = n / TS;
  z0 = (tile / (tpa * tpa)) * TS;
  y0 = ((tile / tpa) % tpa) * TS;
  x0 = (tile % tpa) * TS;
}

// Stage channels [0, CIN) of sample b around the tile at (z0, y0, x0).
template <int CIN>
__device__ __forceinline__ void load_halo(float (*sx)[HV], const View& in, int b, int n, int z0, int y0, int x0) {
  const int mask = n - 1;   // n is a power of two
  for (int e = threadIdx.x; e < CIN * HV; e += CT) {
    const int ci = e / HV, r = e % HV;
    const int hz = r / (HS * HS), hy = (r / HS) % HS, hx = r % HS;
    const int gz = (z0 - 1 + hz) & mask, gy = (y0 - 1 + hy) & mask, gx = (x0 - 1 + hx) & mask;
    sx[ci][r] = in.p[voff(in, b, ci, ((long long)gz * n + gy) * n + gx)];
  }
}

// out[b][co] = conv(in[b], w)[co]            (MODE_PLAIN), times out_scale
// out[b][co] = conv(in[b], w)[co] * gate[co] (MODE_GATE; pre-gate value to pre)
// out[b][co] = sigmoid(conv(in[b], w)[co] + bias[co])   (MODE_SIGMOID)
template <int CIN, int COUT, int MODE>
__global__ void __launch_bounds__(CT) conv_fwd_kernel(View in, View out, const float* __restrict__ w,
                                                      const float* __restrict__ bias, View gate, View pre, int n,
                                                      float out_scale, int wbf16) {
  // Each thread produces two neighbouring voxels along x for every output
  // channel.  The weights sit in shared memory as [ci][tap][co] (co padded
  // to a multiple of 4), so one 16-byte broadcast load feeds 8 FMAs, and
  // the four input values of a halo row serve the three x taps of both
  // voxels.
  constexpr int CP = (COUT + 3) / 4 * 4;
  static_assert(TV == 2 * CT, "two voxels per thread");
  __shared__ float sx[CIN][HV];
  __shared__ __align__(16) float sw[CIN * 27 * CP];
  const int b = blockIdx.y;
  int z0, y0, x0;
  tile_origin(blockIdx.x, n, z0, y0, x0);
  for (int i = threadIdx.x; i < CIN * 27 * CP; i += CT) {
    const int co = i % CP, t = (i / CP) % 27, ci = i / (CP * 27);
    float wv = co < COUT ? w[(co * CIN + ci) * 27 + t] : 0.f;
    if (wbf16) wv = __bfloat162float(__float2bfloat16_rn(wv));   // BF16 weights, FP32 accumulation
    sw[i] = wv;
  }
  load_halo<CIN>(sx, in, b, n, z0, y0, x0);
  __syncthreads();
  const int lz = threadIdx.x / (TS * TS / 2), ly = (threadIdx.x / (TS / 2)) % TS, lx = 2 * (threadIdx.x % (TS / 2));
  float a0[CP], a1[CP];
#pragma unroll
  for (int co = 0; co < CP; ++co) a0[co] = a1[co] = 0.f;
#pragma unroll 1
  for (int ci = 0; ci < CIN; ++ci) {
#pragma unroll
    for (int dz = 0; dz < 3; ++dz)
#pragma unroll
      for (int dy = 0; dy < 3; ++dy) {
        const float* row = &sx[ci][((lz + dz) * HS + (ly + dy)) * HS + lx];
        const float xr[4] = {row[0], row[1], row[2], row[3]};
#pragma unroll
        for (int dx = 0; dx < 3; ++dx) {
          const float4* wt = reinterpret_cast<const float4*>(&sw[(ci * 27 + dz * 9 + dy * 3 + dx) * CP]);
#pragma unroll
          for (int q = 0; q < CP / 4; ++q) {
            const float4 w4 = wt[q];
            a0[4 * q] = fmaf(w4.x, xr[dx], a0[4 * q]);
            a0[4 * q + 1] = fmaf(w4.y, xr[dx], a0[4 * q + 1]);
            a0[4 * q + 2] = fmaf(w4.z, xr[dx], a0[4 * q + 2]);
            a0[4 * q + 3] = fmaf(w4.w, xr[dx], a0[4 * q + 3]);
            a1[4 * q] = fmaf(w4.x, xr[dx + 1], a1[4 * q]);
            a1[4 * q + 1] = fmaf(w4.y, xr[dx + 1], a1[4 * q + 1]);
            a1[4 * q + 2] = fmaf(w4.z, xr[dx + 1], a1[4 * q + 2]);
            a1[4 * q + 3] = fmaf(w4.w, xr[dx + 1], a1[4 * q + 3]);
          }
        }
      }
  }
  const long long gv = ((long long)(z0 + lz) * n + (y0 + ly)) * n + (x0 + lx);
#pragma unroll
  for (int v = 0; v < 2; ++v) {
#pragma unroll
    for (int co = 0; co < COUT; ++co) {
      float r = v == 0 ? a0[co] : a1[co];
      if constexpr (MODE == MODE_SIGMOID) {
        r = 1.f / (1.f + expf(-(r + bias[co])));
      } else if constexpr (MODE == MODE_GATE) {
        if (pre.p) pre.p[voff(pre, b, co, gv + v)] = r;
        r *= gate.p[voff(gate, b, co, gv + v)];
      }
      out.p[voff(out, b, co, gv + v)] = r * out_scale;
    }
  }
}

// partial[blockIdx.x][co][ci][t] = sum over the CTA's (sample, tile) jobs of
// sum_v dy[b][co][v] x[b][ci][v + offset_t]
template <int CIN, int COUT>
__global__ void __launch_bounds__(CT) conv_wgrad_kernel(View dy, View x, int nb, int n, float* __restrict__ partial) {
  extern __shared__ __align__(16) float wg_smem[];
  float(*sx)[HV] = reinterpret_cast<float(*)[HV]>(wg_smem);              // [CIN][HV]
  float(*sd)[TV] = reinterpret_cast<float(*)[TV]>(wg_smem + CIN * HV);   // [COUT][TV]
  constexpr int NE = COUT * CIN * 27;
  constexpr int PER = (NE + CT - 1) / CT;
  const int tiles = (n / TS) * (n / TS) * (n / TS);
  float acc[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) acc[k] = 0.f;
  for (long long job = blockIdx.x; job < (long long)nb * tiles; job += gridDim.x) {
    const int b = (int)(job / tiles), tile = (int)(job % tiles);
    int z0, y0, x0;
    tile_origin(tile, n, z0, y0, x0);
    __syncthreads();   // the previous job's tiles are consumed
    load_halo<CIN>(sx, x, b, n, z0, y0, x0);
    for (int e = threadIdx.x; e < COUT * TV; e += CT) {
      const int co = e / TV, lv = e % TV;
      const int lz = lv / (TS * TS), ly = (lv / TS) % TS, lx = lv % TS;
      sd[co][lv] = dy.p[voff(dy, b, co, ((long long)(z0 + lz) * n + (y0 + ly)) * n + (x0 + lx))];
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      const int e = threadIdx.x + k * CT;
      if (e < NE) {
        const int co = e / (CIN * 27), ci = (e / 27) % CIN, t = e % 27;
        const int off = ((t / 9) * HS + (t / 3) % 3) * HS + t % 3;
        const float* xs = &sx[ci][off];
        const float* ds = sd[co];
        float s = 0.f;
#pragma unroll 4
        for (int lv = 0; lv < TV; ++lv) {
          const int lz = lv / (TS * TS), ly = (lv / TS) % TS, lx = lv % TS;
          s = fmaf(ds[lv], xs[(lz * HS + ly) * HS + lx], s);
        }
        acc[k] += s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const int e = threadIdx.x + k * CT;
    if (e < NE) partial[(size_t)blockIdx.x * NE + e] = acc[k];
  }
}

// out[e] (+)= sum_c partial[c][e], summed in FP64 in a fixed order
__global__ void reduce_partials_kernel(const float* __restrict__ partial, int nparts, int ne, float* __restrict__ out,
                                       int accumulate) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= ne) return;
  double s = 0.0;
  for (int c = 0; c < nparts; ++c) s += (double)partial[(size_t)c * ne + e];
  out[e] = accumulate ? (float)((double)out[e] + s) : (float)s;
}

// wt[ci][co][26 - t] = w[co][ci][t]: the weights of the adjoint convolution
__global__ void adjoint_weights_kernel(const float* __restrict__ w, int cout, int cin, float* __restrict__ wt) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= cout * cin * 27) return;
  const int co = e / (cin * 27), ci = (e / 27) % cin, t = e % 27;
  wt[(ci * cout + co) * 27 + (26 - t)] = w[e];
}

// dz[c][v] = (sum_b dh[b][c][v] a[b][c][v]) g (1 - g);  dh[b][c][v] *= g
__global__ void gate_backward_kernel(View dh, View a, const float* __restrict__ g, int nb, int c, size_t n3,
                                     float* __restrict__ dz) {
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < (size_t)c * n3;
       e += (size_t)gridDim.x * blockDim.x) {
    const int ch = (int)(e / n3);
    const long long v = (long long)(e % n3);
    const float gg = g[e];
    float s = 0.f;
    for (int b = 0; b < nb; ++b) {
      const long long o = voff(dh, b, ch, v);
      const float d = dh.p[o];
      s = fmaf(d, a.p[voff(a, b, ch, v)], s);
      dh.p[o] = d * gg;
    }
    dz[e] = s * gg * (1.f - gg);
  }
}

// db[ch] (+)= sum_v dz[ch][v]; one CTA per channel, FP64 partial sums
__global__ void bias_grad_kernel(const float* __restrict__ dz, size_t n3, float* __restrict__ db, int accumulate) {
  __shared__ double red[32];
  const int ch = blockIdx.x;
  double s = 0.0;
  for (size_t v = threadIdx.x; v < n3; v += blockDim.x) s += (double)dz[(size_t)ch * n3 + v];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    db[ch] = accumulate ? (float)((double)db[ch] + t) : (float)t;
  }
}

// dY = 2 w_v (Y - T); loss += sum w_v |Y - T|^2  (complex64 blocks, floats)
__global__ void loss_grad_kernel(const float* __restrict__ Y, const float* __restrict__ T,
                                 const double* __restrict__ wv, size_t per_vec, size_t total, float* __restrict__ dY,
                                 double* __restrict__ loss) {
  __shared__ double red[32];
  double s = 0.0;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (size_t)gridDim.x * blockDim.x) {
    const double w = wv[e / per_vec];
    const float d = Y[e] - T[e];
    dY[e] = (float)(2.0 * w) * d;
    s += w * (double)d * (double)d;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    atomicAdd(loss, t);
  }
}

// f[0..8][v]: d1, d2, d3, Re/Im M_12, Re/Im M_13, Re/Im M_23 of cell v
__global__ void features_kernel(const uchar4* __restrict__ mid, const float* __restrict__ mtab,
                                const float* __restrict__ dense, size_t n3, float* __restrict__ f) {
  for (size_t v = (size_t)blockIdx.x * blockDim.x + threadIdx.x; v < n3; v += (size_t)gridDim.x * blockDim.x) {
    if (mid) {
      const uchar4 id = mid[v];
      f[v] = mtab[9 * id.x];
      f[n3 + v] = mtab[9 * id.y + 1];
      f[2 * n3 + v] = mtab[9 * id.z + 2];
#pragma unroll
      for (int j = 3; j < 9; ++j) f[j * n3 + v] = mtab[9 * id.w + j];
    } else {
#pragma unroll
      for (int j = 0; j < 9; ++j) f[j * n3 + v] = dense[j * n3 + v];
    }
  }
}

__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, int np, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= np) return;
  const float gi = g[i];
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  p[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// SplitMix64 (Steele, Lea, Flood 2014) of the counter, two uniforms, Box-Muller
__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void init_kernel(float* __restrict__ p, unsigned long long seed) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= NPARAMS) return;
  const unsigned long long h1 = mix64(seed ^ mix64(2ull * (unsigned long long)i));
  const unsigned long long h2 = mix64(seed ^ mix64(2ull * (unsigned long long)i + 1ull));
  const double u1 = ((double)(h1 >> 11) + 0.5) * (1.0 / 9007199254740992.0);
  const double u2 = (double)(h2 >> 11) * (1.0 / 9007199254740992.0);
  const double z = sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
  double scale;
  if (i < OFF_W2) scale = 1.0 / sqrt(3.0 * 27.0);
  else if (i < OFF_W3) scale = 1.0 / sqrt((double)HIDDEN * 27.0);
  else if (i < OFF_V1) scale = 0.0;   // the correction starts at zero: T = K_P^{-1}
  else if (i < OFF_C1) scale = 1.0 / sqrt(9.0 * 27.0);
  else if (i < OFF_V2) scale = 0.0;
  else if (i < OFF_C2) scale = 1.0 / sqrt(9.0 * 27.0);
  else scale = 0.0;
  p[i] = (float)(scale * z);
}

__global__ void lincomb_kernel(const float* __restrict__ x, float alpha, const float* __restrict__ y, float beta,
                               float* __restrict__ z, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    z[i] = y ? fmaf(alpha, x[i], beta * y[i]) : alpha * x[i];
}

__global__ void col_dots_kernel(const float2* __restrict__ a, const float2* __restrict__ b, size_t len,
                                double* __restrict__ dots) {
  __shared__ double red[2][32];
  const int v = blockIdx.y;
  const float2* av = a + (size_t)v * len;
  const float2* bv = b + (size_t)v * len;
  double re = 0.0, im = 0.0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x) {
    const float2 x = av[i], y = bv[i];
    re += (double)x.x * y.x + (double)x.y * y.y;
    im += (double)x.x * y.y - (double)x.y * y.x;
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
    double tr = 0.0, ti = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
      tr += red[0][w];
      ti += red[1][w];
    }
    atomicAdd(dots + 2 * v, tr);
    atomicAdd(dots + 2 * v + 1, ti);
  }
}

__global__ void col_axpby_kernel(const double* __restrict__ alpha, const float2* __restrict__ x,
                                 const double* __restrict__ beta, float2* __restrict__ y, size_t len) {
  const int v = blockIdx.y;
  const float al = (float)alpha[v], be = (float)beta[v];
  const float2* xv = x + (size_t)v * len;
  float2* yv = y + (size_t)v * len;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += (size_t)gridDim.x * blockDim.x) {
    const float2 a = xv[i], b = yv[i];
    yv[i] = make_float2(fmaf(al, a.x, be * b.x), fmaf(al, a.y, be * b.y));
  }
}

unsigned grid_for(size_t n, int threads, unsigned cap) {
  size_t b = (n + threads - 1) / threads;
  if (b < 1) b = 1;
  return (unsigned)(b > cap ? cap : b);
}

}  // namespace

// ---- host launchers ---------------------------------------------------------

#define PCX_CONV_CASE(CI, CO, MD)                                                                       \
  if (cin == CI && cout == CO && mode == MD) {                                                          \
    conv_fwd_kernel<CI, CO, MD><<<grid, CT, 0, s>>>(in, out, w, bias, gate, pre, n, out_scale, wbf16); \
    return cudaGetLastError();                                                                          \
  }

cudaError_t conv_fwd(int cin, int cout, int mode, const View& in, const View& out, const float* w, const float* bias,
                     const View& gate, const View& pre, int nb, int n, float out_scale, cudaStream_t s, int wbf16) {
  if (n < TS || (n & (n - 1)) != 0 || nb < 1 || nb > 65535) return cudaErrorInvalidValue;
  const dim3 grid((unsigned)((n / TS) * (n / TS) * (n / TS)), (unsigned)nb);
  PCX_CONV_CASE(3, HIDDEN, MODE_GATE)
  PCX_CONV_CASE(HIDDEN, HIDDEN, MODE_GATE)
  PCX_CONV_CASE(HIDDEN, 3, MODE_PLAIN)
  PCX_CONV_CASE(9, HIDDEN, MODE_SIGMOID)
  PCX_CONV_CASE(3, HIDDEN, MODE_PLAIN)
  PCX_CONV_CASE(HIDDEN, HIDDEN, MODE_PLAIN)
  return cudaErrorInvalidValue;
}
#undef PCX_CONV_CASE

size_t wgrad_scratch_floats(int cin, int cout) { return (size_t)4 * 152 * cout * cin * 27; }

template <int CIN, int COUT>
static cudaError_t wgrad_t(const View& dy, const View& x, int nb, int n, float* dw, int accumulate, float* scratch,
                           cudaStream_t s) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long jobs = (long long)nb * (n / TS) * (n / TS) * (n / TS);
  long long grid = 4LL * (sms < 152 ? sms : 152);
  if (grid > jobs) grid = jobs;
  const size_t smem = (size_t)(CIN * HV + COUT * TV) * sizeof(float);
  if ((e = raise_dyn_smem(reinterpret_cast<const void*>(conv_wgrad_kernel<CIN, COUT>), smem)) != cudaSuccess) return e;
  conv_wgrad_kernel<CIN, COUT><<<(unsigned)grid, CT, smem, s>>>(dy, x, nb, n, scratch);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  constexpr int NE = COUT * CIN * 27;
  reduce_partials_kernel<<<(NE + 255) / 256, 256, 0, s>>>(scratch, (int)grid, NE, dw, accumulate);
  return cudaGetLastError();
}

cudaError_t conv_wgrad(int cin, int cout, const View& dy, const View& x, int nb, int n, float* dw, int accumulate,
                       float* scratch, cudaStream_t s) {
  if (n < TS || (n & (n - 1)) != 0 || nb < 1) return cudaErrorInvalidValue;
  if (cin == HIDDEN && cout == 3) return wgrad_t<HIDDEN, 3>(dy, x, nb, n, dw, accumulate, scratch, s);
  if (cin == HIDDEN && cout == HIDDEN) return wgrad_t<HIDDEN, HIDDEN>(dy, x, nb, n, dw, accumulate, scratch, s);
  if (cin == 3 && cout == HIDDEN) return wgrad_t<3, HIDDEN>(dy, x, nb, n, dw, accumulate, scratch, s);
  if (cin == 9 && cout == HIDDEN) return wgrad_t<9, HIDDEN>(dy, x, nb, n, dw, accumulate, scratch, s);
  return cudaErrorInvalidValue;
}

cudaError_t adjoint_weights(const float* w, int cout, int cin, float* wt, cudaStream_t s) {
  const int ne = cout * cin * 27;
  adjoint_weights_kernel<<<(ne + 255) / 256, 256, 0, s>>>(w, cout, cin, wt);
  return cudaGetLastError();
}

cudaError_t gate_backward(const View& dh, const View& a, const float* g, int nb, int c, size_t n3, float* dz,
                          cudaStream_t s) {
  gate_backward_kernel<<<grid_for((size_t)c * n3, 256, 152u * 16u), 256, 0, s>>>(dh, a, g, nb, c, n3, dz);
  return cudaGetLastError();
}

cudaError_t bias_grad(const float* dz, int c, size_t n3, float* db, int accumulate, cudaStream_t s) {
  bias_grad_kernel<<<(unsigned)c, 1024, 0, s>>>(dz, n3, db, accumulate);
  return cudaGetLastError();
}

cudaError_t loss_grad(const void* Y, const void* T, const double* wv, int nvec, size_t n3, void* dY, double* loss,
                      cudaStream_t s) {
  const size_t per = 6 * n3, total = per * (size_t)nvec;
  loss_grad_kernel<<<grid_for(total, 256, 152u * 8u), 256, 0, s>>>(static_cast<const float*>(Y),
                                                                   static_cast<const float*>(T), wv, per, total,
                                                                   static_cast<float*>(dY), loss);
  return cudaGetLastError();
}

cudaError_t features(const pcx_ctx* c, float* f, cudaStream_t s) {
  const size_t n3 = (size_t)c->n * c->n * c->n;
  const uchar4* mid = static_cast<const uchar4*>(c->dev.mid);
  features_kernel<<<grid_for(n3, 256, 152u * 16u), 256, 0, s>>>(mid, static_cast<const float*>(c->dev.mtab32),
                                                                static_cast<const float*>(c->dev.m32), n3, f);
  return cudaGetLastError();
}

cudaError_t adam(float* p, const float* g, float* m, float* v, int np, int step, float lr, float b1, float b2, float eps,
                 cudaStream_t s) {
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  adam_kernel<<<(np + 255) / 256, 256, 0, s>>>(p, g, m, v, np, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}

cudaError_t init_params(float* p, unsigned long long seed, cudaStream_t s) {
  init_kernel<<<(NPARAMS + 255) / 256, 256, 0, s>>>(p, seed);
  return cudaGetLastError();
}

cudaError_t lincomb(const float* x, float alpha, const float* y, float beta, float* z, size_t nfloat, cudaStream_t s) {
  lincomb_kernel<<<grid_for(nfloat, 256, 152u * 16u), 256, 0, s>>>(x, alpha, y, beta, z, nfloat);
  return cudaGetLastError();
}

cudaError_t col_dots(const void* a, const void* b, int nvec, size_t len, double* dots, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(dots, 0, sizeof(double) * 2 * (size_t)nvec, s);
  if (e != cudaSuccess || nvec == 0) return e;
  const dim3 grid(grid_for(len, 256, 152u * 4u), (unsigned)nvec);
  col_dots_kernel<<<grid, 256, 0, s>>>(static_cast<const float2*>(a), static_cast<const float2*>(b), len, dots);
  return cudaGetLastError();
}

cudaError_t col_axpby(const double* alpha, const void* x, const double* beta, void* y, int nvec, size_t len,
                      cudaStream_t s) {
  if (nvec == 0) return cudaSuccess;
  const dim3 grid(grid_for(len, 256, 152u * 4u), (unsigned)nvec);
  col_axpby_kernel<<<grid, 256, 0, s>>>(alpha, static_cast<const float2*>(x), beta, static_cast<float2*>(y), len);
  return cudaGetLastError();
}

}  // namespace cnn
}  // namespace pcx
