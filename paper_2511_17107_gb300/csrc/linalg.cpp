// Small dense FP64 complex linear algebra for the Rayleigh-Ritz step of the
// block eigensolver (host side): Householder tridiagonalisation and implicit
// QL for Hermitian matrices,
// Cholesky, triangular inverse, and the generalised Hermitian eigenproblem
// G_A c = theta G_B c solved through an eigen-decomposition of the scaled
// G_B that drops near-dependent directions (the SVQB construction of
// Stathopoulos and Wu, SIAM J. Sci. Comput. 23 (2002) 2165).
#include "linalg.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace pcx {

// Hermitian eigen-decomposition in three steps (Golub and Van Loan,
// "Matrix Computations", Secs. 8.3.1 and 8.3.4):
//  1. Householder reflections H_k = I - 2 v v^H reduce A to a Hermitian
//     tridiagonal T = Q^H A Q, Q = H_0 H_1 ... H_{n-3};
//  2. a diagonal unitary D makes the off-diagonal of T' = D^H T D real and
//     non-negative;
//  3. implicitly shifted QL iterations with Wilkinson-type shifts diagonalise
//     the real symmetric T' = Z diag(w) Z^T.
// The eigenvectors of A are the columns of Q D Z.  a: n x n row-major
// (overwritten); w: eigenvalues ascending; v: n x n row-major, column j is
// the eigenvector of w[j].
void herm_eig(int n, std::vector<cd>& a, std::vector<double>& w, std::vector<cd>& v) {
  auto A = [&](int r, int c) -> cd& { return a[(size_t)r * n + c]; };
  std::vector<cd> q((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i) q[(size_t)i * n + i] = 1.0;
  // 1. tridiagonalisation
  std::vector<cd> hv(n), p(n);
  for (int k = 0; k + 2 < n; ++k) {
    const int m = n - k - 1;   // length of the column below the diagonal
    double xn2 = 0;
    for (int i = 0; i < m; ++i) xn2 += std::norm(A(k + 1 + i, k));
    const double xn = std::sqrt(xn2);
    const double x0a = std::abs(A(k + 1, k));
    if (xn == 0.0 || xn - x0a <= 1e-300) continue;   // already tridiagonal in this column
    const cd ph = x0a > 0 ? A(k + 1, k) / x0a : cd(1, 0);
    const cd alpha = -ph * xn;   // H x = alpha e_1
    for (int i = 0; i < m; ++i) hv[i] = A(k + 1 + i, k);
    hv[0] -= alpha;
    double vn2 = 0;
    for (int i = 0; i < m; ++i) vn2 += std::norm(hv[i]);
    const double vinv = 1.0 / std::sqrt(vn2);
    for (int i = 0; i < m; ++i) hv[i] *= vinv;
    // p = A22 v, K = v^H p (real), w = p - K v;  A22 <- A22 - 2 v w^H - 2 w v^H
    for (int i = 0; i < m; ++i) {
      cd s = 0;
      for (int j = 0; j < m; ++j) s += A(k + 1 + i, k + 1 + j) * hv[j];
      p[i] = s;
    }
    double K = 0;
    for (int i = 0; i < m; ++i) K += (std::conj(hv[i]) * p[i]).real();
    for (int i = 0; i < m; ++i) p[i] -= K * hv[i];
    for (int i = 0; i < m; ++i)
      for (int j = 0; j < m; ++j)
        A(k + 1 + i, k + 1 + j) -= 2.0 * (hv[i] * std::conj(p[j]) + p[i] * std::conj(hv[j]));
    A(k + 1, k) = alpha;
    A(k, k + 1) = std::conj(alpha);
    for (int i = 1; i < m; ++i) A(k + 1 + i, k) = A(k, k + 1 + i) = 0.0;
    // Q <- Q H_k on columns k+1 .. n-1
    for (int r = 0; r < n; ++r) {
      cd s = 0;
      for (int j = 0; j < m; ++j) s += q[(size_t)r * n + k + 1 + j] * hv[j];
      s *= 2.0;
      for (int j = 0; j < m; ++j) q[(size_t)r * n + k + 1 + j] -= s * std::conj(hv[j]);
    }
  }
  // 2. real off-diagonal: delta_{i+1} = delta_i s_i / |s_i|
  std::vector<double> d(n), e(n, 0.0);
  std::vector<cd> delta(n, cd(1, 0));
  for (int i = 0; i < n; ++i) d[i] = A(i, i).real();
  for (int i = 0; i + 1 < n; ++i) {
    const cd si = A(i + 1, i);
    const double r = std::abs(si);
    e[i] = r;
    delta[i + 1] = r > 0 ? delta[i] * (si / r) : delta[i];
  }
  // 3. implicit symmetric QR steps with the Wilkinson shift (Golub and Van
  // Loan, Alg. 8.3.2) on the trailing unreduced block [lo, hi].  A rotation
  // R in the plane (k, k+1) maps T to R T R^T and Z to Z R^T, so that
  // T_initial = Z T Z^T throughout.
  // zt holds Z transposed (row k = column k of Z) so that a rotation runs
  // over two contiguous rows.
  std::vector<double> zt((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) zt[(size_t)i * n + i] = 1.0;
  auto rotate = [&](int k, double c, double sn) {
    const double ak = d[k], ak1 = d[k + 1], bk = e[k];
    d[k] = c * c * ak + 2 * c * sn * bk + sn * sn * ak1;
    d[k + 1] = sn * sn * ak - 2 * c * sn * bk + c * c * ak1;
    e[k] = c * sn * (ak1 - ak) + (c * c - sn * sn) * bk;
    double* zk = &zt[(size_t)k * n];
    double* zk1 = &zt[(size_t)(k + 1) * n];
    for (int r = 0; r < n; ++r) {
      const double u = zk[r], w1 = zk1[r];
      zk[r] = c * u + sn * w1;
      zk1[r] = -sn * u + c * w1;
    }
  };
  int hi = n - 1;
  for (int steps = 0; hi > 0 && steps < 40 * n; ) {
    for (int i = 0; i < hi; ++i)
      if (std::fabs(e[i]) <= 1e-16 * (std::fabs(d[i]) + std::fabs(d[i + 1]))) e[i] = 0.0;
    if (e[hi - 1] == 0.0) {
      --hi;
      continue;
    }
    int lo = hi - 1;
    while (lo > 0 && e[lo - 1] != 0.0) --lo;
    const double half = 0.5 * (d[hi - 1] - d[hi]), bb = e[hi - 1];
    const double mu = d[hi] - bb * bb / (half + (half >= 0 ? 1.0 : -1.0) * std::hypot(half, bb));
    double x = d[lo] - mu, y = e[lo];
    for (int k = lo; k < hi; ++k) {
      const double r = std::hypot(x, y);
      const double c = r > 0 ? x / r : 1.0, sn = r > 0 ? y / r : 0.0;
      if (k > lo) e[k - 1] = r;   // the bulge (k+1, k-1) is annihilated into (k, k-1)
      rotate(k, c, sn);
      if (k + 1 < hi) {
        x = e[k];
        y = sn * e[k + 1];        // new bulge at (k+2, k)
        e[k + 1] *= c;
      }
    }
    ++steps;
  }
  // eigenvectors: (Q D) Z, sorted ascending
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return d[x] < d[y]; });
  w.resize(n);
  std::vector<double> zs((size_t)n * n);   // zs[c][j] = Z[c][idx[j]]
  for (int j = 0; j < n; ++j)
    for (int c = 0; c < n; ++c) zs[(size_t)c * n + j] = zt[(size_t)idx[j] * n + c];
  v.assign((size_t)n * n, cd(0, 0));
  for (int r = 0; r < n; ++r) {
    cd* vr = &v[(size_t)r * n];
    for (int c = 0; c < n; ++c) {
      const cd qd = q[(size_t)r * n + c] * delta[c];
      if (qd == cd(0, 0)) continue;
      const double* zc = &zs[(size_t)c * n];
      for (int j = 0; j < n; ++j) vr[j] += qd * zc[j];
    }
  }
  for (int j = 0; j < n; ++j) w[j] = d[idx[j]];
}

bool cholesky_upper(int n, const std::vector<cd>& g, std::vector<cd>& r) {
  r.assign((size_t)n * n, cd(0, 0));
  for (int j = 0; j < n; ++j) {
    double d = g[(size_t)j * n + j].real();
    for (int k = 0; k < j; ++k) d -= std::norm(r[(size_t)k * n + j]);
    if (!(d > 0)) return false;
    const double rjj = std::sqrt(d);
    r[(size_t)j * n + j] = rjj;
    for (int i = j + 1; i < n; ++i) {
      cd s = g[(size_t)j * n + i];
      for (int k = 0; k < j; ++k) s -= std::conj(r[(size_t)k * n + j]) * r[(size_t)k * n + i];
      r[(size_t)j * n + i] = s / rjj;
    }
  }
  return true;
}

void upper_inverse(int n, const std::vector<cd>& r, std::vector<cd>& ri) {
  ri.assign((size_t)n * n, cd(0, 0));
  for (int j = 0; j < n; ++j) {
    ri[(size_t)j * n + j] = 1.0 / r[(size_t)j * n + j];
    for (int i = j - 1; i >= 0; --i) {
      cd s = 0;
      for (int k = i + 1; k <= j; ++k) s += r[(size_t)i * n + k] * ri[(size_t)k * n + j];
      ri[(size_t)i * n + j] = -s / r[(size_t)i * n + i];
    }
  }
}

int gen_eig(int m, const std::vector<cd>& ga, const std::vector<cd>& gb, double drop_tol, std::vector<double>& theta,
            std::vector<cd>& c, double* lam_min_rel) {
  // D = diag(gb)^{-1/2};  eig(D gb D) = V diag(lam) V^H;  keep lam > drop_tol * max
  std::vector<double> dsc(m);
  for (int i = 0; i < m; ++i) {
    const double g = gb[(size_t)i * m + i].real();
    if (!(g > 0)) return -1;
    dsc[i] = 1 / std::sqrt(g);
  }
  std::vector<cd> b((size_t)m * m);
  for (int i = 0; i < m; ++i)
    for (int j = 0; j < m; ++j) {
      const cd x = 0.5 * (gb[(size_t)i * m + j] + std::conj(gb[(size_t)j * m + i]));
      b[(size_t)i * m + j] = x * dsc[i] * dsc[j];
    }
  // T (m x r) with T^H gb T = I.  Fast path: Cholesky D gb D = R^H R and
  // T = D R^{-1}, taken only when it provably drops nothing:
  // lam_min >= 1 / ||R^{-1}||_F^2 and lam_max <= trace = m, so the test below
  // implies lam_min > drop_tol * lam_max.  Otherwise the eigen-decomposition
  // D gb D = V diag(lam) V^H, T = D V_keep lam_keep^{-1/2} with
  // lam > drop_tol * max (rank-revealing).
  std::vector<cd> t;
  int r = 0;
  {
    std::vector<cd> rr, ri;
    if (cholesky_upper(m, b, rr)) {
      upper_inverse(m, rr, ri);
      double fro2 = 0;
      for (const cd& x : ri) fro2 += std::norm(x);
      if (std::isfinite(fro2) && 1.0 / fro2 > 1e3 * drop_tol * m) {
        r = m;
        if (lam_min_rel) *lam_min_rel = 1.0 / (fro2 * m);
        t.assign((size_t)m * m, cd(0, 0));
        for (int i = 0; i < m; ++i)
          for (int j = i; j < m; ++j) t[(size_t)i * m + j] = dsc[i] * ri[(size_t)i * m + j];
      }
    }
  }
  if (r == 0) {
    std::vector<double> lam;
    std::vector<cd> v;
    herm_eig(m, b, lam, v);
    const double lmax = lam.back();
    if (!(lmax > 0) || !std::isfinite(lmax)) return -1;
    std::vector<int> keep;
    for (int j = 0; j < m; ++j)
      if (lam[j] > drop_tol * lmax) keep.push_back(j);
    r = (int)keep.size();
    if (lam_min_rel) *lam_min_rel = r > 0 ? lam[keep[0]] / lmax : 0.0;
    t.assign((size_t)m * r, cd(0, 0));
    for (int i = 0; i < m; ++i)
      for (int jj = 0; jj < r; ++jj)
        t[(size_t)i * r + jj] = dsc[i] * v[(size_t)i * m + keep[jj]] / std::sqrt(lam[keep[jj]]);
  }
  // H = T^H ga T  (r x r)
  std::vector<cd> gat((size_t)m * r, cd(0, 0));
  for (int i = 0; i < m; ++i) {
    cd* gi = &gat[(size_t)i * r];
    for (int k = 0; k < m; ++k) {
      const cd g = 0.5 * (ga[(size_t)i * m + k] + std::conj(ga[(size_t)k * m + i]));
      if (g == cd(0, 0)) continue;
      const cd* tk = &t[(size_t)k * r];
      for (int jj = 0; jj < r; ++jj) gi[jj] += g * tk[jj];
    }
  }
  std::vector<cd> h((size_t)r * r, cd(0, 0));
  for (int i = 0; i < m; ++i) {
    const cd* gi = &gat[(size_t)i * r];
    for (int a = 0; a < r; ++a) {
      const cd ta = std::conj(t[(size_t)i * r + a]);
      if (ta == cd(0, 0)) continue;
      cd* ha = &h[(size_t)a * r];
      for (int bb = 0; bb < r; ++bb) ha[bb] += ta * gi[bb];
    }
  }
  std::vector<cd> z;
  herm_eig(r, h, theta, z);
  // c = T z  (m x r)
  c.assign((size_t)m * r, cd(0, 0));
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < r; ++k) {
      const cd tik = t[(size_t)i * r + k];
      for (int j = 0; j < r; ++j) c[(size_t)i * r + j] += tik * z[(size_t)k * r + j];
    }
  return r;
}

}  // namespace pcx
