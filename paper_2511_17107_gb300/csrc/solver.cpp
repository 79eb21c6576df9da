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
#include <atomic>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "cnn.h"
#include "linalg.h"
#include "pcx_internal.h"

// Projection-and-Cholesky-QR passes of the refinement's [P W] block against
// X.  One: the Rayleigh-Ritz step takes the X-[P W] couplings from exact
// double-float products of the FP64 X (launch_gram_x), so what FP32
// rounding leaves of X in [P W] is accounted for there and a second pass
// only costs time (measured at 128^3: the same iteration counts, 9% less
// time per solve).  A build-time choice for tuning builds.
#ifndef PCX_ORTH_PASSES
#define PCX_ORTH_PASSES 1
#endif

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

// Worst wanted residual after every iteration (opts.res_history), in the
// order the iterations run; k-points in flight append concurrently.
struct History {
  double* buf = nullptr;
  int cap = 0;
  std::atomic<int> len{0};
  void add(double v) {
    const int i = len.fetch_add(1);
    if (i < cap) buf[i] = v;
  }
};

#define CK(x)                                    \
  do {                                           \
    cudaError_t _e = (x);                        \
    if (_e != cudaSuccess) return fail_cuda(_e); \
  } while (0)

// Wall-clock attribution of solver phases (only when statistics are asked
// for: each tick synchronises the stream and charges the elapsed time).
struct Times {
  double apply = 0, gram = 0, rr = 0, other = 0, precond = 0;
  long long applies = 0;
};

// Learned-correction settings shared by the runs of one pcx_solve call.
struct Learned {
  const float* params = nullptr;   // device, cnn::NPARAMS floats (null: plain K_P^{-1})
  const float* gates = nullptr;    // device, from cnn_gates
  bool off = false;                // fallback to the base preconditioner for the rest of this k
  int fallbacks = 0;
  int kind = 0;                    // base preconditioner: 0 K_P^{-1}, 1 curl sandwich T0
  int patience = 3;                // iterations without a 10% drop before the fallback (< 0: never)
  // residual dump for training (FP32 phase)
  void* dump = nullptr;
  int dump_cap = 0, dump_every = 1, dumped = 0;
};

struct Run {
  Times* tm = nullptr;
  std::chrono::steady_clock::time_point own_clock = std::chrono::steady_clock::now();
  std::chrono::steady_clock::time_point* t0 = &own_clock;   // may be shared between runs
  void tick(double Times::*bucket) {
    if (!tm) return;
    cudaStreamSynchronize(s);
    const auto t1 = std::chrono::steady_clock::now();
    tm->*bucket += std::chrono::duration<double, std::milli>(t1 - *t0).count();
    *t0 = t1;
  }
  pcx_ctx* c;
  cudaStream_t s;
  int prec;          // PCX_FP32 or PCX_FP64
  size_t L;          // complex entries per vector
  size_t es;         // bytes per complex entry
  int n;             // block size
  KParams kp;
  bool k_zero;
  int verbose;
  History* hist = nullptr;   // per-iteration worst residuals (optional)
  double fp32_floor = 0;   // FP32 phase: stop once worst <= fp32_floor 2^-24 theta_top (0: off)
  double theta_top = 0;    // largest Ritz value of the last Rayleigh-Ritz step
  int np = 0;        // P columns at S[n : n+np] (valid when lobpcg returns)
  Learned* learned = nullptr;
  // device buffers
  DevBuf S, AS, S2, AS2, R, G, C, theta, norms;
  std::string err;

  pcx_status fail_cuda(cudaError_t e) {
    err = std::string("pcx_solve: CUDA error ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PCX_ENOMEM : PCX_ECUDA;
  }
  char* col(DevBuf& b, int j) { return static_cast<char*>(b.p) + (size_t)j * L * es; }

  // x_only: the FP64 run of the mixed scheme, which keeps only X and AX
  // (n columns each, with their combination targets) in FP64; its residual
  // goes straight to the FP32 run's R
  pcx_status alloc_all(bool x_only = false) {
    const size_t blk = (size_t)(x_only ? 1 : 3) * n * L * es;
    CK(S.alloc(blk));
    CK(AS.alloc(blk));
    CK(S2.alloc(blk));
    CK(AS2.alloc(blk));
    if (!x_only) CK(R.alloc((size_t)n * L * es));
    CK(G.alloc(sizeof(double) * 2 * (size_t)9 * n * n));
    CK(C.alloc(sizeof(double) * 2 * (size_t)9 * n * n));
    CK(theta.alloc(sizeof(double) * n));
    CK(norms.alloc(sizeof(double) * 2 * n));
    return PCX_OK;
  }

  // host copy of an m x m Gram matrix computed on the device
  pcx_status gram(const void* A, int na, const void* B, int nb, std::vector<cd>& out) {
    tick(&Times::other);
    CK(launch_gram(A, na, B, nb, L, prec, static_cast<double*>(G.p), s));
    out.resize((size_t)na * nb);
    CK(cudaMemcpyAsync(out.data(), G.p, sizeof(cd) * na * nb, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    tick(&Times::gram);
    return PCX_OK;
  }

  void* ascr = nullptr;   // apply / T0 scratch owned by the caller (k-points in flight), else the context's
  cudaError_t apply(const void* X, void* Y, int nvec) {
    tick(&Times::other);
    cudaError_t e = ascr ? launch_apply_scratch(c, kp, X, Y, nvec, prec, ascr, s) : launch_apply(c, kp, X, Y, nvec, prec, s);
    if (tm) tm->applies += nvec;
    tick(&Times::apply);
    return e;
  }

  // W = K_P^{-1} R for one column, or the learned T(R) when it is enabled
  // (FP32 storage only) and has not fallen back
  // W[:, w0 + a] = T R[:, act[a]] for the active columns, one batched call
  // per run of consecutive active columns
  cudaError_t precond_active(const std::vector<int>& act, int w0) {
    tick(&Times::other);
    cudaError_t e = cudaSuccess;
    const int na = (int)act.size();
    for (int a0 = 0; a0 < na && e == cudaSuccess;) {
      int a1 = a0 + 1;
      while (a1 < na && act[a1] == act[a1 - 1] + 1) ++a1;
      const void* r = col(R, act[a0]);
      void* w = col(S, w0 + a0);
      const int cnt = a1 - a0;
      if (learned && learned->params && !learned->off && prec == PCX_FP32)
        e = cnn_precond(c, kp, learned->params, learned->gates, r, w, cnt, s);
      else if (learned && learned->kind == 1)
        e = ascr ? launch_t0_scratch(c, kp, r, w, cnt, prec, ascr, s) : sandwich_precond(c, kp, r, w, cnt, prec, s);
      else
        e = launch_precond(c, kp, r, w, cnt, prec, s);
      a0 = a1;
    }
    tick(&Times::precond);
    return e;
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
    if (ok) upper_inverse(nw, r, ri);
    tick(&Times::rr);
    if (!ok) return PCX_OK;
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
  CK(run.apply(run.S.p, run.AS.p, n));
  {
    std::vector<cd> ga, gb;
    if ((st = run.gram(run.S.p, n, run.AS.p, n, ga)) != PCX_OK) return st;
    if ((st = run.gram(run.S.p, n, run.S.p, n, gb)) != PCX_OK) return st;
    std::vector<double> th;
    std::vector<cd> cm;
    int r = gen_eig(n, ga, gb, 1e-14, th, cm);
    run.tick(&Times::rr);
    if (r < n) {
      run.err = "pcx_solve: initial Rayleigh-Ritz breakdown";
      return PCX_ENUMERIC;
    }
    theta.assign(th.begin(), th.begin() + n);
    run.theta_top = th[r - 1];
    if ((st = run.upload_c(cm)) != PCX_OK) return st;
    CK(launch_combine(run.S.p, n, static_cast<double*>(run.C.p), n, 0.0, run.S2.p, L, run.prec, run.s));
    CK(launch_combine(run.AS.p, n, static_cast<double*>(run.C.p), n, 0.0, run.AS2.p, L, run.prec, run.s));
    std::swap(run.S.p, run.S2.p);
    std::swap(run.AS.p, run.AS2.p);
  }
  int& np = run.np;   // P columns at S[n : n+np]
  np = 0;
  std::vector<double> best_hist;
  double best = INFINITY;
  int since_best = 0;
  double lrn_best = INFINITY;
  int no_drop = 0;
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
    if (run.hist) run.hist->add(worst);
    if (run.verbose) {
      std::fprintf(stderr, "[pcx] %s it %d worst %.3e theta0 %.12g theta_top %.4e\n",
                   run.prec == PCX_FP64 ? "fp64" : "fp32", iters, worst, theta[0], run.theta_top);
    }
    if (worst <= tol) return PCX_OK;
    if (worst <= stop_tol) {
      stopped_early = true;
      return PCX_OK;
    }
    // FP32 phase: the residual has reached the size of the FP32 rounding of
    // Op x (2^-24 ||Op|| ||x||, ||Op|| estimated by the largest Ritz value)
    if (stop_tol > tol && run.prec == PCX_FP32 && run.fp32_floor > 0 &&
        worst <= run.fp32_floor * 0x1p-24 * run.theta_top) {
      stopped_early = true;
      return PCX_OK;
    }
    // stagnation guard (mixed phase): no 10% progress for 4 iterations
    if (worst < best * 0.9) {
      best = worst;
      since_best = 0;
    } else if (++since_best >= 4 && stop_tol > tol) {
      stopped_early = true;
      return PCX_OK;
    }
    if (iters >= maxit) return PCX_ENOCONV;
    Learned* lrn = run.learned;
    // learned correction: back to the base preconditioner once the worst
    // residual has not dropped 10% below its best for `patience` iterations
    if (lrn && lrn->params && !lrn->off && lrn->patience >= 0) {
      if (worst < 0.9 * lrn_best) {
        lrn_best = worst;
        no_drop = 0;
      } else if (++no_drop >= lrn->patience) {
        lrn->off = true;
        ++lrn->fallbacks;
      }
    }

    // soft locking: active columns get W (and P) columns
    std::vector<int> act;
    for (int j = 0; j < n; ++j)
      if (res[j] > tol) act.push_back(j);
    const int na = (int)act.size();
    // residual dump (training data of the learned correction)
    if (lrn && lrn->dump && run.prec == PCX_FP32 && iters % lrn->dump_every == 0)
      for (int a = 0; a < na && lrn->dumped < lrn->dump_cap; ++a, ++lrn->dumped)
        CK(cudaMemcpyAsync(static_cast<char*>(lrn->dump) + (size_t)lrn->dumped * L * 8, run.col(run.R, act[a]), L * 8,
                           cudaMemcpyDeviceToDevice, run.s));
    const int w0 = n + np;   // W at S[w0 : w0+na]
    CK(run.precond_active(act, w0));
    // W <- W - X (X^H W), then orthonormalise W
    {
      std::vector<cd> xw;
      if ((st = run.gram(run.S.p, n, run.col(run.S, w0), na, xw)) != PCX_OK) return st;
      for (auto& v : xw) v = -v;
      if ((st = run.upload_c(xw)) != PCX_OK) return st;
      CK(launch_combine(run.S.p, n, static_cast<double*>(run.C.p), na, 1.0, run.col(run.S, w0), L, run.prec, run.s));
      if ((st = run.cholqr(run.col(run.S, w0), na, run.R.p, ok)) != PCX_OK) return st;
      // A rank-deficient W (Cholesky of its Gram matrix fails) stays as it
      // is: the Rayleigh-Ritz step below works on the scaled Gram matrix of
      // [X P W] and drops every direction whose eigenvalue is below `drop`
      // of the largest, which removes W's dependent columns.
      ok = true;
    }
    CK(run.apply(run.col(run.S, w0), run.col(run.AS, w0), na));
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
      double lam_min_rel = 1.0;
      r = gen_eig(m, ga, gb, drop, th, cm, &lam_min_rel);
      run.tick(&Times::rr);
      if (r > 0) run.theta_top = th[r - 1];
      // FP64: P is not orthonormalised, and over hundreds of iterations it
      // can drift towards span[X W]; the rounding of S^H (AS) then reaches
      // the Ritz values amplified by 1 / lam_min_rel (10th-order stencils at
      // 32^3 turned them to noise).  Such a step drops P, a restart of the
      // search direction, and keeps the basis well conditioned.
      const bool ill = run.prec == PCX_FP64 && lam_min_rel < 1e-9;
      if (r >= n && !(ill && np > 0)) break;
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

// Mixed-precision refinement (PCX_FP32 mode, after the FP32 phase): X and
// AX = Op X are held and updated in FP64, so the residual R = AX - X Theta
// is FP64-accurate; the search directions W = K_P^{-1} R, P and their images
// are FP32 with FP32 applies.  The Rayleigh-Ritz matrices take their X rows
// from double-float products of the FP64 X, AX with the FP32 directions
// (launch_gram_x), their P/W blocks from tensor-core FP32 products, and their
// X-X blocks from the previous step (Theta, I).  [P W] is orthonormalised
// against X in FP32 each step.  An error in a direction block enters the new
// X scaled by that block's coefficient, which shrinks with the residual, so
// the FP64 residual keeps converging.  AX is recomputed with an FP64 apply,
// followed by a Rayleigh-Ritz step on X, every `refresh` iterations and
// before convergence is accepted.  r64.S/AS hold X64/AX64; r32.S/AS hold
// [X32 | P32 | W32] and their images, X32 rounded from X64.
pcx_status lobpcg_refine(Run& r64, Run& r32, int nev, double tol, int maxit, int& iters, std::vector<double>& theta,
                         std::vector<double>& res) {
  Run& run = r64;   // for CK
  const int n = r64.n;
  const size_t L = r64.L;
  pcx_status st;
  bool ok = true;
  // X64 from the FP32 block: orthonormalise in FP64, AX64 = Op X64, Rayleigh-Ritz
  CK(launch_convert(r32.S.p, PCX_FP32, r64.S.p, PCX_FP64, (size_t)n * L, r64.s));
  if ((st = r64.cholqr(r64.S.p, n, r64.S2.p, ok)) != PCX_OK) return st;
  if (!ok) {
    r64.err = "pcx_solve: refinement block is rank deficient";
    return PCX_ENUMERIC;
  }
  auto fresh_ax = [&]() -> pcx_status {
    CK(r64.apply(r64.S.p, r64.AS.p, n));
    return PCX_OK;
  };
  auto rr_x = [&]() -> pcx_status {   // Rayleigh-Ritz on span(X64), FP64
    std::vector<cd> ga, gb, cm;
    std::vector<double> th;
    pcx_status s2;
    if ((s2 = r64.gram(r64.S.p, n, r64.AS.p, n, ga)) != PCX_OK) return s2;
    if ((s2 = r64.gram(r64.S.p, n, r64.S.p, n, gb)) != PCX_OK) return s2;
    const int r = gen_eig(n, ga, gb, 1e-14, th, cm);
    r64.tick(&Times::rr);
    if (r < n) {
      r64.err = "pcx_solve: refinement Rayleigh-Ritz breakdown";
      return PCX_ENUMERIC;
    }
    theta.assign(th.begin(), th.begin() + n);
    if ((s2 = r64.upload_c(cm)) != PCX_OK) return s2;
    CK(launch_combine(r64.S.p, n, static_cast<double*>(r64.C.p), n, 0.0, r64.S2.p, L, PCX_FP64, r64.s));
    CK(launch_combine(r64.AS.p, n, static_cast<double*>(r64.C.p), n, 0.0, r64.AS2.p, L, PCX_FP64, r64.s));
    CK(cudaMemcpyAsync(r64.S.p, r64.S2.p, (size_t)n * L * 16, cudaMemcpyDeviceToDevice, r64.s));
    CK(cudaMemcpyAsync(r64.AS.p, r64.AS2.p, (size_t)n * L * 16, cudaMemcpyDeviceToDevice, r64.s));
    return PCX_OK;
  };
  if ((st = fresh_ax()) != PCX_OK) return st;
  if ((st = rr_x()) != PCX_OK) return st;
  int np = r32.np;          // P32 / AP32 from the FP32 phase stay valid directions
  const int refresh = 20;
  int since_fresh = 0;
  double lrn_best = INFINITY;
  int no_drop = 0;
  res.assign(n, INFINITY);
  for (iters = 0;; ++iters) {
    // FP64 residual
    CK(cudaMemcpyAsync(r64.theta.p, theta.data(), sizeof(double) * n, cudaMemcpyHostToDevice, r64.s));
    // FP64 residual of the FP64 X and AX, stored rounded to FP32 (the
    // directions and the AX rows below use it), with X rounded to FP32 in the
    // same pass
    CK(launch_residual_mixed(r64.S.p, r64.AS.p, static_cast<double*>(r64.theta.p), r32.R.p, r32.S.p,
                             static_cast<double*>(r64.norms.p), n, L, r64.s));
    std::vector<double> nrm(2 * n);
    CK(cudaMemcpyAsync(nrm.data(), r64.norms.p, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, r64.s));
    CK(cudaStreamSynchronize(r64.s));
    double worst = 0;
    for (int j = 0; j < n; ++j) {
      res[j] = std::sqrt(nrm[j]) / std::sqrt(nrm[n + j]);
      if (!std::isfinite(res[j]) || !std::isfinite(theta[j])) {
        r64.err = "pcx_solve: NaN or Inf in the refinement residual";
        return PCX_ENUMERIC;
      }
      if (j < nev) worst = std::max(worst, res[j]);
    }
    if (r64.hist) r64.hist->add(worst);
    if (r64.verbose)
      std::fprintf(stderr, "[pcx] refine it %d worst %.3e theta0 %.12g%s\n", iters, worst, theta[0],
                   since_fresh == 0 ? " (fresh AX)" : "");
    if (worst <= tol) {
      if (since_fresh == 0) return PCX_OK;   // accepted on an exactly recomputed AX
      if ((st = fresh_ax()) != PCX_OK) return st;
      if ((st = rr_x()) != PCX_OK) return st;
      since_fresh = 0;
      --iters;
      continue;
    }
    if (iters >= maxit) return PCX_ENOCONV;
    if (r32.learned && r32.learned->params && !r32.learned->off && r32.learned->patience >= 0) {
      if (worst < 0.9 * lrn_best) {
        lrn_best = worst;
        no_drop = 0;
      } else if (++no_drop >= r32.learned->patience) {
        r32.learned->off = true;
        ++r32.learned->fallbacks;
      }
    }
    if (++since_fresh >= refresh) {   // exact image of X and Rayleigh-Ritz on X; P is kept
      if ((st = fresh_ax()) != PCX_OK) return st;
      if ((st = rr_x()) != PCX_OK) return st;
      since_fresh = 0;
      --iters;
      continue;
    }
    std::vector<int> act;
    for (int j = 0; j < n; ++j)
      if (res[j] > tol) act.push_back(j);
    const int na = (int)act.size();
    const int w0 = n + np;
    // W32 = K_P^{-1} R (FP32; X32 and R32 come from the residual pass)
    CK(r32.precond_active(act, w0));
    // [P W] is orthogonalised against X and orthonormalised (Cholesky QR,
    // PCX_ORTH_PASSES passes) in FP32, so the FP32 part of the Gram matrices
    // is close to the identity; P is dropped when [P W] is numerically rank
    // deficient.
    auto orth_block = [&](int c0, int cnt, bool& okb) -> pcx_status {
      okb = true;
      for (int pass = 0; pass < PCX_ORTH_PASSES && okb; ++pass) {
        std::vector<cd> xw;
        pcx_status s2;
        if ((s2 = r32.gram(r32.S.p, n, r32.col(r32.S, c0), cnt, xw)) != PCX_OK) return s2;
        for (auto& v : xw) v = -v;
        if ((s2 = r32.upload_c(xw)) != PCX_OK) return s2;
        CK(launch_combine(r32.S.p, n, static_cast<double*>(r32.C.p), cnt, 1.0, r32.col(r32.S, c0), L, PCX_FP32,
                          r64.s));
        if ((s2 = r32.cholqr(r32.col(r32.S, c0), cnt, r32.col(r32.S2, c0), okb)) != PCX_OK) return s2;
      }
      return PCX_OK;
    };
    bool okb = true;
    if ((st = orth_block(n, np + na, okb)) != PCX_OK) return st;
    if (!okb && np > 0) {
      CK(cudaMemcpyAsync(r32.col(r32.S, n), r32.col(r32.S, w0), (size_t)na * L * 8, cudaMemcpyDeviceToDevice,
                         r64.s));
      np = 0;
      if ((st = orth_block(n, na, okb)) != PCX_OK) return st;
    }
    // (a W block that stays rank deficient is left to the drop tolerance of
    // the Rayleigh-Ritz step)
    CK(r32.apply(r32.col(r32.S, n), r32.col(r32.AS, n), np + na));
    const int m = n + np + na;
    const int mp = m - n;
    // Rows of X: X^H [P W] from the FP64 X against the FP32 directions with
    // double-float sums (these couplings are of the size of the residual, far
    // below the FP32 rounding of the products), and
    //   (AX)^H [P W] = Theta X^H [P W] + R^H [P W],  R = AX - X Theta,
    // the last term an FP32 product of the rounded FP64 residual (its entries
    // are of the residual's size, so FP32 relative accuracy is enough).  The
    // X-X blocks are Theta and I: X and AX are the Ritz vectors and images of
    // the previous Rayleigh-Ritz step (or of rr_x after an exact refresh).
    // The P/W-P/W blocks come from FP32 products on the tensor cores.
    std::vector<cd> gx, grw, gpa, gpb;
    {
      r64.tick(&Times::other);
      CK(launch_gram_x(r64.S.p, n, nullptr, 0, r32.col(r32.S, n), mp, L, static_cast<double*>(r64.G.p), r64.s));
      std::vector<cd> gxx((size_t)n * mp);
      CK(cudaMemcpyAsync(gxx.data(), r64.G.p, sizeof(cd) * gxx.size(), cudaMemcpyDeviceToHost, r64.s));
      CK(cudaStreamSynchronize(r64.s));
      r64.tick(&Times::gram);
      if ((st = r32.gram(r32.R.p, n, r32.col(r32.S, n), mp, grw)) != PCX_OK) return st;
      gx.resize((size_t)2 * n * mp);
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < mp; ++j) {
          gx[(size_t)i * mp + j] = gxx[(size_t)i * mp + j];
          gx[(size_t)(n + i) * mp + j] = theta[i] * gxx[(size_t)i * mp + j] + grw[(size_t)i * mp + j];
        }
    }
    if ((st = r32.gram(r32.col(r32.S, n), mp, r32.col(r32.AS, n), mp, gpa)) != PCX_OK) return st;
    if ((st = r32.gram(r32.col(r32.S, n), mp, r32.col(r32.S, n), mp, gpb)) != PCX_OK) return st;
    std::vector<cd> ga((size_t)m * m), gb((size_t)m * m);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j) {
        cd a, b;
        if (i < n && j < n) {
          a = i == j ? cd(theta[i], 0.0) : cd(0.0, 0.0);
          b = i == j ? cd(1.0, 0.0) : cd(0.0, 0.0);
        } else if (i < n) {
          a = gx[(size_t)(n + i) * mp + (j - n)];
          b = gx[(size_t)i * mp + (j - n)];
        } else if (j < n) {
          a = std::conj(gx[(size_t)(n + j) * mp + (i - n)]);
          b = std::conj(gx[(size_t)j * mp + (i - n)]);
        } else {
          a = gpa[(size_t)(i - n) * mp + (j - n)];
          b = gpb[(size_t)(i - n) * mp + (j - n)];
        }
        ga[(size_t)i * m + j] = a;
        gb[(size_t)i * m + j] = b;
      }
    std::vector<double> th;
    std::vector<cd> cm;
    const int r = gen_eig(m, ga, gb, 1e-7, th, cm);
    r64.tick(&Times::rr);
    if (r < n) {
      // drop P and restart the directions from a fresh FP64 image
      if ((st = fresh_ax()) != PCX_OK) return st;
      if ((st = rr_x()) != PCX_OK) return st;
      since_fresh = 0;
      np = 0;
      continue;
    }
    // X64' = X64 C_XX + [P32 W32] C_PX ;  AX64' likewise
    std::vector<cd> cxx((size_t)n * n), cpx((size_t)mp * n);
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < n; ++j) {
        if (i < n) cxx[(size_t)i * n + j] = cm[(size_t)i * r + j];
        else cpx[(size_t)(i - n) * n + j] = cm[(size_t)i * r + j];
      }
    if ((st = r64.upload_c(cxx)) != PCX_OK) return st;
    CK(launch_combine(r64.S.p, n, static_cast<double*>(r64.C.p), n, 0.0, r64.S2.p, L, PCX_FP64, r64.s));
    CK(launch_combine(r64.AS.p, n, static_cast<double*>(r64.C.p), n, 0.0, r64.AS2.p, L, PCX_FP64, r64.s));
    if ((st = r32.upload_c(cpx)) != PCX_OK) return st;
    CK(launch_combine_add32(r32.col(r32.S, n), m - n, static_cast<double*>(r32.C.p), n, r64.S2.p, L, r64.s));
    CK(launch_combine_add32(r32.col(r32.AS, n), m - n, static_cast<double*>(r32.C.p), n, r64.AS2.p, L, r64.s));
    // P32' = [P32 W32] C_P,act (FP32), the part of the new Ritz vectors outside span(X)
    const int npn = na;
    {
      std::vector<cd> cp((size_t)(m - n) * npn);
      for (int i = n; i < m; ++i)
        for (int a = 0; a < npn; ++a) cp[(size_t)(i - n) * npn + a] = cm[(size_t)i * r + act[a]];
      CK(cudaStreamSynchronize(r64.s));
      if ((st = r32.upload_c(cp)) != PCX_OK) return st;
      CK(launch_combine(r32.col(r32.S, n), m - n, static_cast<double*>(r32.C.p), npn, 0.0, r32.col(r32.S2, n), L,
                        PCX_FP32, r64.s));
    }
    np = npn;
    theta.assign(th.begin(), th.begin() + n);
    std::swap(r64.S.p, r64.S2.p);
    std::swap(r64.AS.p, r64.AS2.p);
    std::swap(r32.S.p, r32.S2.p);
    std::swap(r32.AS.p, r32.AS2.p);
  }
}

}  // namespace

// Everything one Bloch vector needs: the runs (device buffers) of both
// precisions and the counters of the call.
struct KSolve {
  pcx_ctx* c;
  cudaStream_t s;
  const pcx_solve_opts* o;
  int n, nev, maxit;
  double tol, switch_tol;
  uint64_t seed;
  Times *t32, *t64;
  int iters32 = 0, iters64 = 0;
  Learned* learned = nullptr;
  History* hist = nullptr;
  std::string* err = nullptr;   // where messages go (the context's, or a worker's own)
};

// LOBPCG for one k with penalty coefficient gamma (<= 0: the rule of Sec. 2).
// On return r64.S[0:nev] holds the FP64 eigenvectors.
pcx_status solve_one_k(KSolve& ks, const double k[3], double gamma, int ik, Run& r64, Run& r32,
                       std::vector<double>& theta, std::vector<double>& res, int& iters_total) {
  r64.learned = ks.learned;
  r32.learned = ks.learned;
  if (ks.learned) ks.learned->off = false;
  pcx_ctx* c = ks.c;
  const cudaStream_t s = ks.s;
  const int n = ks.n, nev = ks.nev, maxit = ks.maxit;
  const size_t L = (size_t)3 * c->n * c->n * c->n;
  const bool kz = k[0] == 0 && k[1] == 0 && k[2] == 0;
  iters_total = 0;
  pcx_status st;
  r64.c = c;
  r64.s = s;
  r64.prec = PCX_FP64;
  r64.L = L;
  r64.es = 16;
  r64.n = n;
  r64.kp = make_kparams(c, k, gamma);
  r64.k_zero = kz;
  r64.verbose = ks.o->verbose;
  r64.hist = ks.hist;
  if (ks.o->stats) r64.tm = ks.t64;
  if ((st = r64.alloc_all(ks.o->precision == PCX_FP32)) != PCX_OK) {
    *ks.err = r64.err;
    return st;
  }
  if (ks.o->precision == PCX_FP32) {
    r32.c = c;
    r32.s = s;
    r32.prec = PCX_FP32;
    r32.L = L;
    r32.es = 8;
    r32.n = n;
    r32.kp = r64.kp;
    r32.k_zero = kz;
    r32.verbose = ks.o->verbose;
    r32.hist = ks.hist;
    r32.fp32_floor = ks.o->fp32_floor == 0 ? 1024.0 : (ks.o->fp32_floor > 0 ? ks.o->fp32_floor : 0.0);
    r32.t0 = r64.t0;
    if (ks.o->stats) r32.tm = ks.t32;
    if ((st = r32.alloc_all()) != PCX_OK) {
      *ks.err = r32.err;
      return st;
    }
    cudaError_t e = ks.o->x0 ? launch_convert(ks.o->x0, PCX_FP64, r32.S.p, PCX_FP32, (size_t)n * L, s)
                             : launch_fill_random(r32.S.p, n, L, ks.seed + ik, PCX_FP32, s);
    if (e == cudaSuccess && kz) e = launch_deflate_p0(r32.S.p, n, c->n, PCX_FP32, s);
    if (e != cudaSuccess) {
      *ks.err = std::string("pcx_solve: ") + cudaGetErrorString(e);
      return PCX_ECUDA;
    }
    int it32 = 0;
    bool early = false;
    *r32.t0 = std::chrono::steady_clock::now();
    st = lobpcg(r32, nev, ks.tol, maxit, ks.switch_tol, it32, theta, res, early);
    r32.tick(&Times::other);
    iters_total += it32;
    ks.iters32 += it32;
    if (st != PCX_OK && st != PCX_ENOCONV) {
      *ks.err = r32.err;
      return st;
    }
    // refine: X, AX in FP64, directions in FP32
    int itr = 0;
    *r64.t0 = std::chrono::steady_clock::now();
    st = lobpcg_refine(r64, r32, nev, ks.tol, std::max(1, maxit - iters_total), itr, theta, res);
    r64.tick(&Times::other);
    iters_total += itr;
    ks.iters64 += itr;
    if (st != PCX_OK && st != PCX_ENOCONV) *ks.err = r64.err.empty() ? r32.err : r64.err;
    return st;
  }
  cudaError_t e = ks.o->x0 ? cudaMemcpyAsync(r64.S.p, ks.o->x0, (size_t)n * L * 16, cudaMemcpyDeviceToDevice, s)
                           : launch_fill_random(r64.S.p, n, L, ks.seed + ik, PCX_FP64, s);
  if (e == cudaSuccess && kz) e = launch_deflate_p0(r64.S.p, n, c->n, PCX_FP64, s);
  if (e != cudaSuccess) {
    *ks.err = std::string("pcx_solve: ") + cudaGetErrorString(e);
    return PCX_ECUDA;
  }
  int it64 = 0;
  bool early = false;
  *r64.t0 = std::chrono::steady_clock::now();
  st = lobpcg(r64, nev, ks.tol, std::max(1, maxit - iters_total), 0.0, it64, theta, res, early);
  r64.tick(&Times::other);
  iters_total += it64;
  ks.iters64 += it64;
  if (st != PCX_OK && st != PCX_ENOCONV) *ks.err = r64.err;
  return st;
}

// Spurious-mode guard: the largest share of the penalty term in a wanted
// Rayleigh quotient, max_j gamma x_j^H K_B x_j / (theta_j ||x_j||^2).  A
// physical eigenvector lies in ker B (Prop. 2.3: the spectrum splits into
// that of A M A^H and gamma times that of B^H B), so its share is at the
// rounding level; a penalty eigenvector has share ~1.
pcx_status penalty_share(Run& r64, int nev, const std::vector<double>& theta, double& worst) {
  Run& run = r64;
  CK(launch_div_norms(r64.c, r64.kp, r64.S.p, nev, PCX_FP64, static_cast<double*>(r64.norms.p), r64.s));
  std::vector<double> q(2 * (size_t)nev);
  CK(cudaMemcpyAsync(q.data(), r64.norms.p, sizeof(double) * q.size(), cudaMemcpyDeviceToHost, r64.s));
  CK(cudaStreamSynchronize(r64.s));
  worst = 0.0;
  for (int j = 0; j < nev; ++j) {
    const double den = std::fabs(theta[j]) * q[nev + j];
    const double share = den > 0 ? r64.kp.gamma * q[j] / den : INFINITY;
    worst = std::max(worst, share);
  }
  return PCX_OK;
}

// Host outputs of pcx_solve (any may be null) and the device eigenvector buffer.
struct KOut {
  double* eig;
  double* res;
  int* iters;
  void* vec;
};

// One k of pcx_solve: LOBPCG with the spurious-mode guard (gamma x4 while a
// wanted pair is a penalty mode), then the k's outputs.  r64 / r32 are the
// caller's runs, whose buffers carry over from one k to the next.
pcx_status solve_k(KSolve& ks, const double* k, int ik, double penalty_tol, const KOut& out, Run& r64, Run& r32,
                   int& raises, double& gamma_last, bool& noconv) {
  pcx_ctx* c = ks.c;
  const int nev = ks.nev;
  const int max_raises = 4;
  const size_t L = (size_t)3 * c->n * c->n * c->n;
  double gamma = ks.o->gamma > 0 ? ks.o->gamma : make_kparams(c, k, 0.0).gamma;
  std::vector<double> theta, res;
  int iters_total = 0;
  pcx_status st;
  for (int attempt = 0;; ++attempt) {
    iters_total = 0;
    st = solve_one_k(ks, k, gamma, ik, r64, r32, theta, res, iters_total);
    if (st != PCX_OK && st != PCX_ENOCONV) return st;
    if (st != PCX_OK || penalty_tol < 0) break;
    double share = 0.0;
    pcx_status sg = penalty_share(r64, nev, theta, share);
    if (sg != PCX_OK) {
      *ks.err = r64.err;
      return sg;
    }
    if (r64.verbose) std::fprintf(stderr, "[pcx] k %d gamma %.6g penalty share %.3e\n", ik, gamma, share);
    if (share <= penalty_tol) break;
    if (attempt >= max_raises) {
      *ks.err = "pcx_solve: penalty modes among the wanted eigenpairs after raising gamma " +
                std::to_string(max_raises) + " times";
      return PCX_ENUMERIC;
    }
    gamma *= 4.0;   // lift gamma * lambda_1^B above the wanted part of the spectrum
    ++raises;
  }
  gamma_last = gamma;
  noconv = st == PCX_ENOCONV;
  if (noconv) *ks.err = "pcx_solve: iteration cap reached";
  for (int j = 0; j < nev; ++j) {
    if (out.eig) out.eig[(size_t)ik * nev + j] = theta[j];
    if (out.res) out.res[(size_t)ik * nev + j] = res[j];
  }
  if (out.iters) out.iters[ik] = iters_total;
  if (out.vec) {
    cudaError_t e = cudaMemcpyAsync(static_cast<char*>(out.vec) + (size_t)ik * nev * L * 16, r64.S.p,
                                    (size_t)nev * L * 16, cudaMemcpyDeviceToDevice, ks.s);
    if (e != cudaSuccess) {
      *ks.err = std::string("pcx_solve: ") + cudaGetErrorString(e);
      return PCX_ECUDA;
    }
  }
  cudaError_t e = cudaStreamSynchronize(ks.s);
  if (e != cudaSuccess) {
    *ks.err = std::string("pcx_solve: ") + cudaGetErrorString(e);
    return PCX_ECUDA;
  }
  return PCX_OK;
}

// pcx_solve with `conc` k-points in flight: one host thread per slot, each
// with its own stream (kept in the context), search-space buffers, apply
// scratch and counters, taking the next k from a shared counter.  The GPU
// runs one k's kernels while another k's host does its Rayleigh-Ritz step.
// The slots' streams start after the work already queued on the caller's
// stream; every slot is synchronised before this returns.
pcx_status solve_concurrent(KSolve& base, const double* kpts, int nk, double penalty_tol, const KOut& out, int conc,
                            int& raises, double& gamma_last, pcx_status& result) {
  pcx_ctx* c = base.c;
  cudaError_t e;
  while ((int)c->solve_streams.size() < conc) {
    cudaStream_t st = nullptr;
    if ((e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)) != cudaSuccess) {
      c->err = std::string("pcx_solve: ") + cudaGetErrorString(e);
      return PCX_ECUDA;
    }
    c->solve_streams.push_back(st);
  }
  cudaEvent_t ready = nullptr;
  if ((e = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming)) != cudaSuccess ||
      (e = cudaEventRecord(ready, base.s)) != cudaSuccess) {
    if (ready) cudaEventDestroy(ready);
    c->err = std::string("pcx_solve: ") + cudaGetErrorString(e);
    return PCX_ECUDA;
  }
  // apply / T0 scratch of one slot: the larger of the two precisions' needs
  const int n3cols = 3 * base.n;
  const size_t scr = std::max(apply_scratch_bytes(c, PCX_FP64, n3cols), apply_scratch_bytes(c, PCX_FP32, n3cols));
  std::atomic<int> next{0};
  std::atomic<bool> failed{false};
  std::mutex mu;
  pcx_status first_err = PCX_OK;
  std::string first_msg;
  struct Slot {
    KSolve ks;
    Times t32, t64;
    Learned lrn;
    std::string err;
    int raises = 0;
    double gamma_last = 0.0;
    bool noconv = false;
  };
  std::vector<Slot> slots(conc);
  auto work = [&](int w) {
    Slot& sl = slots[w];
    sl.ks = base;
    sl.ks.s = c->solve_streams[w];
    sl.ks.t32 = &sl.t32;
    sl.ks.t64 = &sl.t64;
    sl.ks.iters32 = sl.ks.iters64 = 0;
    sl.ks.err = &sl.err;
    if (base.learned) {
      sl.lrn = *base.learned;
      sl.ks.learned = &sl.lrn;
    }
    auto fail = [&](pcx_status st, const std::string& msg) {
      std::lock_guard<std::mutex> lock(mu);
      if (first_err == PCX_OK) {
        first_err = st;
        first_msg = msg;
      }
      failed = true;
    };
    cudaError_t ee = cudaSetDevice(c->device);
    if (ee == cudaSuccess) ee = cudaStreamWaitEvent(sl.ks.s, ready, 0);
    DevBuf ascr;
    if (ee == cudaSuccess) ee = ascr.alloc(scr);
    if (ee != cudaSuccess) {
      fail(ee == cudaErrorMemoryAllocation ? PCX_ENOMEM : PCX_ECUDA,
           std::string("pcx_solve: ") + cudaGetErrorString(ee));
      return;
    }
    Run r64, r32;
    r64.ascr = ascr.p;
    r32.ascr = ascr.p;
    for (int ik = next++; ik < nk && !failed; ik = next++) {
      bool noconv = false;
      pcx_status st = solve_k(sl.ks, kpts + 3 * ik, ik, penalty_tol, out, r64, r32, sl.raises, sl.gamma_last, noconv);
      if (st != PCX_OK) {
        fail(st, sl.err);
        break;
      }
      sl.noconv = sl.noconv || noconv;
    }
    cudaStreamSynchronize(sl.ks.s);
  };
  std::vector<std::thread> threads;
  for (int w = 0; w < conc; ++w) threads.emplace_back(work, w);
  for (auto& t : threads) t.join();
  cudaEventDestroy(ready);
  // counters of the slots
  for (Slot& sl : slots) {
    for (double Times::*f : {&Times::apply, &Times::gram, &Times::rr, &Times::other, &Times::precond}) {
      base.t32->*f += sl.t32.*f;
      base.t64->*f += sl.t64.*f;
    }
    base.t32->applies += sl.t32.applies;
    base.t64->applies += sl.t64.applies;
    base.iters32 += sl.ks.iters32;
    base.iters64 += sl.ks.iters64;
    raises += sl.raises;
    gamma_last = std::max(gamma_last, sl.gamma_last);
    if (sl.noconv) {
      result = PCX_ENOCONV;
      c->err = "pcx_solve: iteration cap reached";
    }
    if (base.learned) base.learned->fallbacks += sl.lrn.fallbacks;
  }
  if (first_err != PCX_OK) {
    c->err = first_msg;
    return first_err;
  }
  return PCX_OK;
}

pcx_status solve(pcx_ctx* c, const double* kpts, int nk, int nev, double tol, const pcx_solve_opts* opts,
                 double* eig_out, double* res_out, int* iters_out, void* vec_out, cudaStream_t s) {
  pcx_solve_opts o;
  std::memset(&o, 0, sizeof(o));
  if (opts) o = *opts;
  const int n = o.block > 0 ? o.block : nev + 4;
  if (nev < 1 || n < nev || n > 42 || nk < 0 || (nk > 0 && !kpts) || !(tol > 0)) {
    c->err = "pcx_solve: need 1 <= nev <= block <= 42, tol > 0, kpts";
    return PCX_EINVAL;
  }
  if (o.precision != PCX_FP64 && o.precision != PCX_FP32) {
    c->err = "pcx_solve: bad precision";
    return PCX_EINVAL;
  }
  if (!(o.gamma >= 0) || !std::isfinite(o.gamma)) {
    c->err = "pcx_solve: gamma must be finite and >= 0";
    return PCX_EINVAL;
  }
  if (o.cnn_params && o.precision != PCX_FP32) {
    c->err = "pcx_solve: the learned correction needs precision PCX_FP32";
    return PCX_EINVAL;
  }
  if (o.dump_R && (o.dump_cap < 0 || o.dump_every < 0)) {
    c->err = "pcx_solve: dump_cap and dump_every must be >= 0";
    return PCX_EINVAL;
  }
  const double penalty_tol = o.penalty_tol == 0 ? 1e-6 : o.penalty_tol;
  pcx_status result = PCX_OK;
  Times t32, t64;
  KSolve ks;
  ks.c = c;
  ks.s = s;
  ks.o = &o;
  ks.n = n;
  ks.nev = nev;
  ks.maxit = o.maxit > 0 ? o.maxit : 1000;
  ks.tol = tol;
  ks.switch_tol = o.switch_tol > 0 ? o.switch_tol : 1e-4;
  ks.seed = o.seed ? o.seed : 20251117ull;
  ks.t32 = &t32;
  ks.t64 = &t64;
  int raises = 0;
  double gamma_last = 0.0;
  Learned lrn;
  DevBuf gates_buf;
  if (o.precond_kind != 0 && o.precond_kind != 1) {
    c->err = "pcx_solve: precond_kind must be 0 or 1";
    return PCX_EINVAL;
  }
  if (o.cnn_params || o.dump_R || o.precond_kind) {
    lrn.kind = o.precond_kind;
    lrn.patience = o.learned_patience == 0 ? 3 : o.learned_patience;
    lrn.params = o.cnn_params;
    lrn.dump = o.dump_R;
    lrn.dump_cap = o.dump_R ? o.dump_cap : 0;
    lrn.dump_every = o.dump_every > 0 ? o.dump_every : 1;
    if (o.cnn_params) {
      cudaError_t e = gates_buf.alloc(sizeof(float) * 2 * cnn::HIDDEN * (size_t)c->n * c->n * c->n);
      if (e == cudaSuccess) e = cnn_gates(c, o.cnn_params, static_cast<float*>(gates_buf.p), s);
      if (e != cudaSuccess) {
        c->err = std::string("pcx_solve: ") + cudaGetErrorString(e);
        return e == cudaErrorMemoryAllocation ? PCX_ENOMEM : PCX_ECUDA;
      }
      lrn.gates = static_cast<const float*>(gates_buf.p);
    }
    ks.learned = &lrn;
  }
  const auto t_start = std::chrono::steady_clock::now();
  if (o.stats) std::memset(o.stats, 0, sizeof(*o.stats));
  ks.err = &c->err;
  History hist;
  if (o.res_history && o.res_history_cap > 0) {
    hist.buf = o.res_history;
    hist.cap = o.res_history_cap;
    ks.hist = &hist;
  }
  const KOut kout{eig_out, res_out, iters_out, vec_out};
  const int conc = std::min(o.k_concurrency, nk);
  if (conc > 1 && !o.cnn_params && !o.dump_R) {
    pcx_status st = solve_concurrent(ks, kpts, nk, penalty_tol, kout, conc, raises, gamma_last, result);
    if (st != PCX_OK) return st;
  } else {
    Run r64, r32;   // buffers reused from one k to the next
    for (int ik = 0; ik < nk; ++ik) {
      bool noconv = false;
      pcx_status st = solve_k(ks, kpts + 3 * ik, ik, penalty_tol, kout, r64, r32, raises, gamma_last, noconv);
      if (st != PCX_OK) return st;
      if (noconv) result = PCX_ENOCONV;
    }
  }
  if (o.stats) {
    pcx_solve_stats& st = *o.stats;
    st.iters_fp32 = ks.iters32;
    st.iters_fp64 = ks.iters64;
    st.applies_fp32 = t32.applies;
    st.applies_fp64 = t64.applies;
    st.ms_apply = t32.apply + t64.apply;
    st.ms_gram = t32.gram + t64.gram;
    st.ms_rr = t32.rr + t64.rr;
    st.ms_other = t32.other + t64.other;
    st.ms_total = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
    st.gamma_raises = raises;
    st.gamma_last = gamma_last;
    st.ms_precond = t32.precond + t64.precond;
    st.learned_fallbacks = lrn.fallbacks;
    st.dumped = lrn.dumped;
    st.history_len = std::min(hist.len.load(), hist.cap);
  }
  return result;
}

}  // namespace pcx
