// Small dense FP64 complex linear algebra for the Rayleigh-Ritz step of the
// block eigensolver (host side): cyclic Jacobi for Hermitian matrices,
// Cholesky, triangular inverse, and the generalised Hermitian eigenproblem
// G_A c = theta G_B c solved through an eigen-decomposition of the scaled
// G_B that drops near-dependent directions (the SVQB construction of
// Stathopoulos and Wu, SIAM J. Sci. Comput. 23 (2002) 2165).
#include "linalg.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace pcx {

// Hermitian eigen-decomposition by cyclic Jacobi rotations.  a: n x n
// row-major (overwritten); w: eigenvalues ascending; v: n x n row-major,
// column j is the eigenvector of w[j].
void herm_eig(int n, std::vector<cd>& a, std::vector<double>& w, std::vector<cd>& v) {
  v.assign((size_t)n * n, cd(0, 0));
  for (int i = 0; i < n; ++i) v[(size_t)i * n + i] = 1.0;
  auto at = [&](int r, int c) -> cd& { return a[(size_t)r * n + c]; };
  double total = 0;
  for (auto& x : a) total += std::norm(x);
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0;
    for (int p = 0; p < n; ++p)
      for (int q = p + 1; q < n; ++q) off += std::norm(at(p, q));
    if (off <= 1e-32 * total || off == 0.0) break;
    for (int p = 0; p < n; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const cd apq = at(p, q);
        const double r = std::abs(apq);
        if (r == 0.0) continue;
        const double app = at(p, p).real(), aqq = at(q, q).real();
        if (r <= 1e-300) continue;
        const cd ph = apq / r;   // e^{i phi}
        const double tau = (aqq - app) / (2 * r);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1 + tau * tau));
        const double c = 1 / std::sqrt(1 + t * t), s = t * c;
        // U = [[c, s], [-s e^{-i phi}, c e^{-i phi}]] on columns p, q;  A <- U^H A U
        const cd up = std::conj(ph);
        for (int k = 0; k < n; ++k) {   // columns
          const cd akp = at(k, p), akq = at(k, q);
          at(k, p) = akp * c - akq * s * up;
          at(k, q) = akp * s + akq * c * up;
        }
        for (int k = 0; k < n; ++k) {   // rows (conjugate of U)
          const cd apk = at(p, k), aqk = at(q, k);
          at(p, k) = apk * c - aqk * s * ph;
          at(q, k) = apk * s + aqk * c * ph;
        }
        at(p, q) = 0;
        at(q, p) = 0;
        at(p, p) = at(p, p).real();
        at(q, q) = at(q, q).real();
        for (int k = 0; k < n; ++k) {
          const cd vkp = v[(size_t)k * n + p], vkq = v[(size_t)k * n + q];
          v[(size_t)k * n + p] = vkp * c - vkq * s * up;
          v[(size_t)k * n + q] = vkp * s + vkq * c * up;
        }
      }
    }
  }
  std::vector<int> idx(n);
  std::iota(idx.begin(), idx.end(), 0);
  std::vector<double> d(n);
  for (int i = 0; i < n; ++i) d[i] = at(i, i).real();
  std::stable_sort(idx.begin(), idx.end(), [&](int x, int y) { return d[x] < d[y]; });
  w.resize(n);
  std::vector<cd> vs((size_t)n * n);
  for (int j = 0; j < n; ++j) {
    w[j] = d[idx[j]];
    for (int k = 0; k < n; ++k) vs[(size_t)k * n + j] = v[(size_t)k * n + idx[j]];
  }
  v.swap(vs);
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
            std::vector<cd>& c) {
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
  std::vector<double> lam;
  std::vector<cd> v;
  herm_eig(m, b, lam, v);
  const double lmax = lam.back();
  if (!(lmax > 0) || !std::isfinite(lmax)) return -1;
  std::vector<int> keep;
  for (int j = 0; j < m; ++j)
    if (lam[j] > drop_tol * lmax) keep.push_back(j);
  const int r = (int)keep.size();
  // T = D V_keep diag(lam_keep)^{-1/2}  (m x r)
  std::vector<cd> t((size_t)m * r);
  for (int i = 0; i < m; ++i)
    for (int jj = 0; jj < r; ++jj) t[(size_t)i * r + jj] = dsc[i] * v[(size_t)i * m + keep[jj]] / std::sqrt(lam[keep[jj]]);
  // H = T^H ga T  (r x r)
  std::vector<cd> gat((size_t)m * r, cd(0, 0));
  for (int i = 0; i < m; ++i)
    for (int k = 0; k < m; ++k) {
      const cd g = 0.5 * (ga[(size_t)i * m + k] + std::conj(ga[(size_t)k * m + i]));
      if (g == cd(0, 0)) continue;
      for (int jj = 0; jj < r; ++jj) gat[(size_t)i * r + jj] += g * t[(size_t)k * r + jj];
    }
  std::vector<cd> h((size_t)r * r, cd(0, 0));
  for (int a = 0; a < r; ++a)
    for (int bb = 0; bb < r; ++bb) {
      cd s = 0;
      for (int i = 0; i < m; ++i) s += std::conj(t[(size_t)i * r + a]) * gat[(size_t)i * r + bb];
      h[(size_t)a * r + bb] = s;
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
