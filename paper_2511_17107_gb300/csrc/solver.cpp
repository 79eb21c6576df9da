// Block LOBPCG with soft locking for the compensated operator (Sec. 4:
// "LOBPCG with soft locking", Knyazev, SIAM J. Sci. Comput. 23 (2001) 517),
// preconditioned by K_P^{-1} (Sec. 2.4 eq. matrixfree_finalform), with the
// convergence test Res_j = ||Op x_j - theta_j x_j|| / ||x_j|| <= tol (Sec. 4
// eq. exp_relativeresidual).
//
// Device side: apply, preconditioner, Gram products, combinations and
// residuals run as CUDA kernels on the caller's stream.  Host side: the
// small Rayleigh-Ritz eigenproblems in FP64 (linalg.cpp); each iteration
// moves the two Gram matrices to the host and the coefficient matrix back.
//
// Column layout of the search space S (one contiguous allocation, columns
// of length L = 3 N^3):  S = [X (n) | P (np) | W (na)]  and AS = Op S.
// Mixed precision (PCX_FP32): the iteration runs with FP32 storage and FP32
// apply until every wanted Res_j <= switch_tol (or the residual stagnates),
// then continues with FP64 storage and apply from the converted block.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "linalg.h"
#include "pcx_internal.h"

namespace pcx {
namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t alloc(size_t b) {
    if (b <= bytes) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
    cudaError_t e = cudaMalloc(&p, b);
    if (e == cudaSuccess) bytes = b;
    return e;
  }
  ~DevBuf() {
    if (p) cudaFree(p);
  }
};

#define CK(x)                                    \
  do {                                           \
    cudaError_t _e = (x);                        \
    if (_e != cudaSuccess) return fail_cuda(_e); \
  } while (0)

struct Run {
  pcx_ctx* c;
  cudaStream_t s;
  int prec;          // PCX_FP32 or PCX_FP64
  size_t L;          // complex entries per vector
  size_t es;         // bytes per complex entry
  int n;             // block size
  KParams kp;
  bool k_zero;
  int verbose;
  // device buffers
  DevBuf S, AS, S2, AS2, R, G, C, theta, norms;
  std::string err;

  pcx_status fail_cuda(cudaError_t e) {
    err = std::string("pcx_solve: CUDA error ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PCX_ENOMEM : PCX_ECUDA;
  }
  char* col(DevBuf& b, int j) { return static_cast<char*>(b.p) + (size_t)j * L * es; }

  pcx_status alloc_all() {
    const size_t blk = (size_t)3 * n * L * es;
    CK(S.alloc(blk));
    CK(AS.alloc(blk));
    CK(S2.alloc(blk));
    CK(AS2.alloc(blk));
    CK(R.alloc((size_t)n * L * es));
    CK(G.alloc(sizeof(double) * 2 * (size_t)9 * n * n));
    CK(C.alloc(sizeof(double) * 2 * (size_t)9 * n * n));
    CK(theta.alloc(sizeof(double) * n));
    CK(norms.alloc(sizeof(double) * 2 * n));
    return PCX_OK;
  }

  // host copy of an m x m Gram matrix computed on the device
  pcx_status gram(const void* A, int na, const void* B, int nb, std::vector<cd>& out) {
    CK(launch_gram(A, na, B, nb, L, prec, static_cast<double*>(G.p), s));
    out.resize((size_t)na * nb);
    CK(cudaMemcpyAsync(out.data(), G.p, sizeof(cd) * na * nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    return PCX_OK;
  }

  pcx_status upload_c(const std::vector<cd>& cm) {
    CK(cudaMemcpyAsync(C.p, cm.data(), sizeof(cd) * cm.size(), cudaMemcpyHostToDevice, s));
    return PCX_OK;
  }

  // Orthonormalise the nw columns at `cols` (and their images if `acols`)
  // by Cholesky QR: V <- V R^{-1}.  Uses S2-side scratch `tmp`.
  pcx_status cholqr(void* cols, int nw, void* tmp, bool& ok) {
    std::vector<cd> g, r, ri;
    pcx_status st = gram(cols, nw, cols, nw, g);
    if (st != PCX_OK) return st;
    ok = cholesky_upper(nw, g, r);
    if (!ok) return PCX_OK;
    upper_inverse(nw, r, ri);
    if ((st = upload_c(ri)) != PCX_OK) return st;
    CK(launch_combine(cols, nw, static_cast<double*>(C.p), nw, 0.0, tmp, L, prec, s));
    CK(cudaMemcpyAsync(cols, tmp, (size_t)nw * L * es, cudaMemcpyDeviceToDevice, s));
    return PCX_OK;
  }
};

#undef CK
#define CK(x)                                      \
  do {                                             \
    cudaError_t _e = (x);                          \
    if (_e != cudaSuccess) return run.fail_cuda(_e); \
  } while (0)

// One LOBPCG run at fixed precision starting from the n columns already in
// run.S[0:n] (not necessarily orthonormal).  theta/res receive the Ritz
// values and residuals of all n columns.
pcx_status lobpcg(Run& run, int nev, double tol, int maxit, double stop_tol, int& iters, std::vector<double>& theta,
                  std::vector<double>& res, bool& stopped_early) {
  const int n = run.n;
  const size_t L = run.L, es = run.es;
  stopped_early = false;
  pcx_status st;
  bool ok = true;
  // orthonormalise X, AX = Op X, Rayleigh-Ritz on X
  if ((st = run.cholqr(run.S.p, n, run.S2.p, ok)) != PCX_OK) return st;
  if (!ok) {
    run.err = "pcx_solve: initial block is rank deficient";
    return PCX_ENUMERIC;
  }
  CK(launch_apply(run.c, run.kp, run.S.p, run.AS.p, n, run.prec, run.s));
  {
    std::vector<cd> ga, gb;
    if ((st = run.gram(run.S.p, n, run.AS.p, n, ga)) != PCX_OK) return st;
    if ((st = run.gram(run.S.p, n, run.S.p, n, gb)) != PCX_OK) return st;
    std::vector<double> th;
    std::vector<cd> cm;
    int r = gen_eig(n, ga, gb, 1e-14, th, cm);
    if (r < n) {
      run.err = "pcx_solve: initial Rayleigh-Ritz breakdown";
      return PCX_ENUMERIC;
    }
    theta.assign(th.begin(), th.begin() + n);
    if ((st = run.upload_c(cm)) != PCX_OK) return st;
    CK(launch_combine(run.S.p, n, static_cast<double*>(run.C.p), n, 0.0, run.S2.p, L, run.prec, run.s));
    CK(launch_combine(run.AS.p, n, static_cast<double*>(run.C.p), n, 0.0, run.AS2.p, L, run.prec, run.s));
    std::swap(run.S.p, run.S2.p);
    std::swap(run.AS.p, run.AS2.p);
  }
  int np = 0;   // P columns at S[n : n+np]
  std::vector<double> best_hist;
  double best = INFINITY;
  int since_best = 0;
  res.assign(n, INFINITY);
  for (iters = 0;; ++iters) {
    // residual R = AX - X theta and norms
    CK(cudaMemcpyAsync(run.theta.p, theta.data(), sizeof(double) * n, cudaMemcpyHostToDevice, run.s));
    CK(launch_residual(run.S.p, run.AS.p, static_cast<double*>(run.theta.p), run.R.p,
                       static_cast<double*>(run.norms.p), n, L, run.prec, run.s));
    std::vector<double> nrm(2 * n);
    CK(cudaMemcpyAsync(nrm.data(), run.norms.p, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, run.s));
    CK(cudaStreamSynchronize(run.s));
    double worst = 0;
    for (int j = 0; j < n; ++j) {
      res[j] = std::sqrt(nrm[j]) / std::sqrt(nrm[n + j]);
      if (!std::isfinite(res[j]) || !std::isfinite(theta[j])) {
        run.err = "pcx_solve: NaN or Inf in the residual";
        return PCX_ENUMERIC;
      }
      if (j < nev) worst = std::max(worst, res[j]);
    }
    if (run.verbose) {
      std::fprintf(stderr, "[pcx] %s it %d worst %.3e theta0 %.12g\n", run.prec == PCX_FP64 ? "fp64" : "fp32", iters,
                   worst, theta[0]);
    }
    if (worst <= tol) return PCX_OK;
    if (worst <= stop_tol) {
      stopped_early = true;
      return PCX_OK;
    }
    // stagnation guard (mixed phase): no progress for 8 iterations
    if (worst < best * 0.9) {
      best = worst;
      since_best = 0;
    } else if (++since_best >= 8 && stop_tol > tol) {
      stopped_early = true;
      return PCX_OK;
    }
    if (iters >= maxit) return PCX_ENOCONV;

    // soft locking: active columns get W (and P) columns
    std::vector<int> act;
    for (int j = 0; j < n; ++j)
      if (res[j] > tol) act.push_back(j);
    const int na = (int)act.size();
    const int w0 = n + np;   // W at S[w0 : w0+na]
    for (int a = 0; a < na; ++a)
      CK(launch_precond(run.c, run.kp, run.col(run.R, act[a]), run.col(run.S, w0 + a), 1, run.prec, run.s));
    // W <- W - X (X^H W), then orthonormalise W
    {
      std::vector<cd> xw;
      if ((st = run.gram(run.S.p, n, run.col(run.S, w0), na, xw)) != PCX_OK) return st;
      for (auto& v : xw) v = -v;
      if ((st = run.upload_c(xw)) != PCX_OK) return st;
      CK(launch_combine(run.S.p, n, static_cast<double*>(run.C.p), na, 1.0, run.col(run.S, w0), L, run.prec, run.s));
      if ((st = run.cholqr(run.col(run.S, w0), na, run.R.p, ok)) != PCX_OK) return st;
      if (!ok) {   // rank-deficient W: second orthogonalisation pass with SVQB fallback below
        ok = true;
      }
    }
    CK(launch_apply(run.c, run.kp, run.col(run.S, w0), run.col(run.AS, w0), na, run.prec, run.s));
    // Rayleigh-Ritz on S = [X P W]
    int m = n + np + na;
    std::vector<double> th;
    std::vector<cd> cm;
    int r = -1;
    for (int attempt = 0; attempt < 2; ++attempt) {
      std::vector<cd> ga, gb;
      if ((st = run.gram(run.S.p, m, run.AS.p, m, ga)) != PCX_OK) return st;
      if ((st = run.gram(run.S.p, m, run.S.p, m, gb)) != PCX_OK) return st;
      const double drop = run.prec == PCX_FP64 ? 1e-13 : 1e-7;
      r = gen_eig(m, ga, gb, drop, th, cm);
      if (r >= n) break;
      if (np == 0) break;
      // drop P and retry: move W down to S[n : n+na]
      CK(cudaMemcpyAsync(run.col(run.S, n), run.col(run.S, w0), (size_t)na * L * es, cudaMemcpyDeviceToDevice, run.s));
      CK(cudaMemcpyAsync(run.col(run.AS, n), run.col(run.AS, w0), (size_t)na * L * es, cudaMemcpyDeviceToDevice,
                         run.s));
      np = 0;
      m = n + na;
    }
    if (r < n) {
      run.err = "pcx_solve: Rayleigh-Ritz breakdown (search space rank " + std::to_string(r) + " < block)";
      return PCX_ENUMERIC;
    }
    // X' = S C[:, :n]  (C is m x r row-major; take the first n columns)
    std::vector<cd> cx((size_t)m * n);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < n; ++j) cx[(size_t)i * n + j] = cm[(size_t)i * r + j];
    if ((st = run.upload_c(cx)) != PCX_OK) return st;
    CK(launch_combine(run.S.p, m, static_cast<double*>(run.C.p), n, 0.0, run.S2.p, L, run.prec, run.s));
    CK(launch_combine(run.AS.p, m, static_cast<double*>(run.C.p), n, 0.0, run.AS2.p, L, run.prec, run.s));
    // P' = [P W] C[n:, act']: the part of the new Ritz vectors outside span(X)
    // kept for the columns that were active (converged ones are locked).
    std::vector<int> pact = act;
    const int npn = (int)pact.size();
    if (npn > 0 && m > n) {
      std::vector<cd> cp((size_t)(m - n) * npn);
      for (int i = n; i < m; ++i)
        for (int a = 0; a < npn; ++a) cp[(size_t)(i - n) * npn + a] = cm[(size_t)i * r + pact[a]];
      // C is reused: wait until the previous combines have consumed it
      CK(cudaStreamSynchronize(run.s));
      if ((st = run.upload_c(cp)) != PCX_OK) return st;
      CK(launch_combine(run.col(run.S, n), m - n, static_cast<double*>(run.C.p), npn, 0.0, run.col(run.S2, n), L,
                        run.prec, run.s));
      CK(launch_combine(run.col(run.AS, n), m - n, static_cast<double*>(run.C.p), npn, 0.0, run.col(run.AS2, n), L,
                        run.prec, run.s));
    }
    np = npn;
    theta.assign(th.begin(), th.begin() + n);
    std::swap(run.S.p, run.S2.p);
    std::swap(run.AS.p, run.AS2.p);
    std::swap(run.S.bytes, run.S2.bytes);
    std::swap(run.AS.bytes, run.AS2.bytes);
  }
}

}  // namespace

pcx_status solve(pcx_ctx* c, const double* kpts, int nk, int nev, double tol, const pcx_solve_opts* opts,
                 double* eig_out, double* res_out, int* iters_out, void* vec_out, cudaStream_t s) {
  pcx_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  const int n = o.block > 0 ? o.block : nev + 4;
  const int maxit = o.maxit > 0 ? o.maxit : 1000;
  const uint64_t seed = o.seed ? o.seed : 20251117ull;
  const double switch_tol = o.switch_tol > 0 ? o.switch_tol : 1e-4;
  if (nev < 1 || n < nev || n > 42 || nk < 0 || (nk > 0 && !kpts) || !(tol > 0)) {
    c->err = "pcx_solve: need 1 <= nev <= block <= 42, tol > 0, kpts";
    return PCX_EINVAL;
  }
  if (o.precision != PCX_FP64 && o.precision != PCX_FP32) {
    c->err = "pcx_solve: bad precision";
    return PCX_EINVAL;
  }
  const size_t L = (size_t)3 * c->n * c->n * c->n;
  pcx_status result = PCX_OK;
  for (int ik = 0; ik < nk; ++ik) {
    const double* k = kpts + 3 * ik;
    const bool kz = k[0] == 0 && k[1] == 0 && k[2] == 0;
    std::vector<double> theta, res;
    int iters_total = 0;
    pcx_status st;
    Run r64;
    r64.c = c;
    r64.s = s;
    r64.prec = PCX_FP64;
    r64.L = L;
    r64.es = 16;
    r64.n = n;
    r64.kp = make_kparams(c, k, 0.0);
    r64.k_zero = kz;
    r64.verbose = o.verbose;
    if ((st = r64.alloc_all()) != PCX_OK) {
      c->err = r64.err;
      return st;
    }
    if (o.precision == PCX_FP32) {
      Run r32;
      r32.c = c;
      r32.s = s;
      r32.prec = PCX_FP32;
      r32.L = L;
      r32.es = 8;
      r32.n = n;
      r32.kp = r64.kp;
      r32.k_zero = kz;
      r32.verbose = o.verbose;
      if ((st = r32.alloc_all()) != PCX_OK) {
        c->err = r32.err;
        return st;
      }
      cudaError_t e = launch_fill_random(r32.S.p, n, L, seed + ik, PCX_FP32, s);
      if (e == cudaSuccess && kz) e = launch_deflate_p0(r32.S.p, n, c->n, PCX_FP32, s);
      if (e != cudaSuccess) {
        c->err = std::string("pcx_solve: ") + cudaGetErrorString(e);
        return PCX_ECUDA;
      }
      int it32 = 0;
      bool early = false;
      st = lobpcg(r32, nev, tol, maxit, switch_tol, it32, theta, res, early);
      iters_total += it32;
      if (st != PCX_OK && st != PCX_ENOCONV) {
        c->err = r32.err;
        return st;
      }
      // refine in FP64 from the FP32 block
      e = launch_convert(r32.S.p, PCX_FP32, r64.S.p, PCX_FP64, (size_t)n * L, s);
      if (e != cudaSuccess) {
        c->err = std::string("pcx_solve: ") + cudaGetErrorString(e);
        return PCX_ECUDA;
      }
    } else {
      cudaError_t e = launch_fill_random(r64.S.p, n, L, seed + ik, PCX_FP64, s);
      if (e == cudaSuccess && kz) e = launch_deflate_p0(r64.S.p, n, c->n, PCX_FP64, s);
      if (e != cudaSuccess) {
        c->err = std::string("pcx_solve: ") + cudaGetErrorString(e);
        return PCX_ECUDA;
      }
    }
    int it64 = 0;
    bool early = false;
    st = lobpcg(r64, nev, tol, std::max(1, maxit - iters_total), 0.0, it64, theta, res, early);
    iters_total += it64;
    if (st != PCX_OK && st != PCX_ENOCONV) {
      c->err = r64.err;
      return st;
    }
    if (st == PCX_ENOCONV) {
      result = PCX_ENOCONV;
      c->err = "pcx_solve: iteration cap reached";
    }
    for (int j = 0; j < nev; ++j) {
      if (eig_out) eig_out[(size_t)ik * nev + j] = theta[j];
      if (res_out) res_out[(size_t)ik * nev + j] = res[j];
    }
    if (iters_out) iters_out[ik] = iters_total;
    if (vec_out) {
      cudaError_t e = cudaMemcpyAsync(static_cast<char*>(vec_out) + (size_t)ik * nev * L * 16, r64.S.p,
                                      (size_t)nev * L * 16, cudaMemcpyDeviceToDevice, s);
      if (e != cudaSuccess) {
        c->err = std::string("pcx_solve: ") + cudaGetErrorString(e);
        return PCX_ECUDA;
      }
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      c->err = std::string("pcx_solve: ") + cudaGetErrorString(e);
      return PCX_ECUDA;
    }
  }
  return result;
}

}  // namespace pcx
