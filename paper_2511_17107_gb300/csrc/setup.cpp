// Host-side setup: staggered sampling of a structure, FP64 inversion of the
// material permittivities, packing of the per-cell blocks of M_Trivial, the
// HPD check, the circulant symbol tables and the FFT twiddles.
//
// Sec. 2.1 eqs. yee_edgefacedofs / yee_volumedofs (staggered points),
// Sec. 2.2 eq. ct_replacement (physical point A x'), Sec. 1
// eq. intro_permittivity (epsilon_1 = eps^{-1}), Sec. 3.1
// eq. permittivity_diagonal_case and Sec. 3.2.1 eq. trivial_trivial (cell
// blocks), Lemma 3.5 (block spectrum), Lemma 2.1 and Prop. 2.8 (symbols),
// Sec. 2.5 eqs. kc:highord:stencil / kc:high:coef (2m-th order rows),
// Remark 2.6 eq. kc_settingofgamma1 (gamma rule).
//
// Compiled with -ffp-contract=off: sample coordinates and distances are
// evaluated left to right without fused multiply-adds, so that a point on a
// shape boundary is classified reproducibly.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "linalg.h"
#include "pcx_internal.h"

namespace pcx {
namespace {

using ld = long double;

// Coefficients c_1..c_m of the 2m-th order staggered stencil (kind 1:
// derivative, kind 0: interpolation): sum_t ((2t-1)/2)^(2s+kind-2) c_t =
// delta_{s1} / 2, solved by Gaussian elimination in long double.
std::vector<ld> fd_coeffs(int m, int kind) {
  std::vector<std::vector<ld>> a(m, std::vector<ld>(m + 1, 0));
  for (int s = 1; s <= m; ++s) {
    for (int t = 1; t <= m; ++t) a[s - 1][t - 1] = std::pow((ld)(2 * t - 1) / 2, (ld)(2 * s + kind - 2));
    a[s - 1][m] = (s == 1) ? (ld)0.5 : (ld)0;
  }
  for (int col = 0; col < m; ++col) {
    int piv = col;
    for (int r = col + 1; r < m; ++r)
      if (std::fabs(a[r][col]) > std::fabs(a[piv][col])) piv = r;
    std::swap(a[col], a[piv]);
    for (int r = 0; r < m; ++r) {
      if (r == col) continue;
      ld f = a[r][col] / a[col][col];
      for (int cc = col; cc <= m; ++cc) a[r][cc] -= f * a[col][cc];
    }
  }
  std::vector<ld> c(m);
  for (int i = 0; i < m; ++i) c[i] = a[i][m] / a[i][i];
  return c;
}

// Eigenvalues of the circulant with (D phi)_i = sum_a w_a phi_{i+a}:
// lambda_p = sum_a w_a exp(2 pi i p a / N)  (Lemma 2.1).
void symbol_tables(int n, int m, std::vector<cd>& lam1, std::vector<cd>& lam0) {
  std::vector<ld> c1 = fd_coeffs(m, 1), c0 = fd_coeffs(m, 0);
  lam1.assign(n, cd(0, 0));
  lam0.assign(n, cd(0, 0));
  const ld two_pi = 6.283185307179586476925286766559005768L;
  for (int p = 0; p < n; ++p) {
    ld r1 = 0, i1 = 0, r0 = 0, i0 = 0;
    for (int s = 1; s <= m; ++s) {
      // offsets s-1 (weight +) and -s (weight - for D1, + for D0)
      ld ap = two_pi * (ld)(((long)p * (s - 1)) % n) / n;
      ld am = two_pi * (ld)(((long)p * (n - s % n)) % n) / n;
      ld w1 = c1[s - 1] * n;   // divided by h = 1/N
      r1 += w1 * (std::cos(ap) - std::cos(am));
      i1 += w1 * (std::sin(ap) - std::sin(am));
      r0 += c0[s - 1] * (std::cos(ap) + std::cos(am));
      i0 += c0[s - 1] * (std::sin(ap) + std::sin(am));
    }
    lam1[p] = cd((double)r1, (double)i1);
    lam0[p] = cd((double)r0, (double)i0);
  }
}

bool invert3(const double* a, double* inv) {   // row-major real 3x3
  double det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
               a[2] * (a[3] * a[7] - a[4] * a[6]);
  if (!(std::fabs(det) > 1e-300)) return false;
  inv[0] = (a[4] * a[8] - a[5] * a[7]) / det;
  inv[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  inv[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  inv[3] = (a[5] * a[6] - a[3] * a[8]) / det;
  inv[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  inv[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  inv[6] = (a[3] * a[7] - a[4] * a[6]) / det;
  inv[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  inv[8] = (a[0] * a[4] - a[1] * a[3]) / det;
  return true;
}

// Complex 3x3 inverse by Gauss-Jordan elimination with partial pivoting.
bool invert3c(const cd* a, cd* inv) {
  cd m[3][6];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 6; ++c) m[r][c] = (c < 3) ? a[3 * r + c] : cd(c - 3 == r ? 1 : 0, 0);
  for (int col = 0; col < 3; ++col) {
    int piv = col;
    for (int r = col + 1; r < 3; ++r)
      if (std::abs(m[r][col]) > std::abs(m[piv][col])) piv = r;
    if (!(std::abs(m[piv][col]) > 1e-300)) return false;
    for (int c = 0; c < 6; ++c) std::swap(m[col][c], m[piv][c]);
    cd f = 1.0 / m[col][col];
    for (int c = 0; c < 6; ++c) m[col][c] *= f;
    for (int r = 0; r < 3; ++r) {
      if (r == col) continue;
      cd g = m[r][col];
      for (int c = 0; c < 6; ++c) m[r][c] -= g * m[col][c];
    }
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) inv[3 * r + c] = m[r][c + 3];
  return true;
}

struct ShapeEval {
  int kind, material;
  double p[9];
  // derived
  double mid[3], u[3], half, r2;
  bool min_image;
};

ShapeEval prepare(const pcx_shape& s) {
  ShapeEval e;
  e.kind = s.kind;
  e.material = s.material;
  std::memcpy(e.p, s.p, sizeof(e.p));
  e.min_image = true;
  if (s.kind == PCX_SHAPE_SPHERE) {
    e.r2 = s.p[3] * s.p[3];
    e.min_image = s.p[3] < 0.5;
  } else if (s.kind == PCX_SHAPE_SEGMENT) {
    double ax[3];
    for (int i = 0; i < 3; ++i) {
      ax[i] = s.p[3 + i] - s.p[i];
      e.mid[i] = 0.5 * (s.p[i] + s.p[3 + i]);
    }
    double len = std::sqrt((ax[0] * ax[0] + ax[1] * ax[1]) + ax[2] * ax[2]);
    for (int i = 0; i < 3; ++i) e.u[i] = ax[i] / len;
    e.half = 0.5 * len;
    e.r2 = s.p[6] * s.p[6];
    e.min_image = std::sqrt(e.half * e.half + e.r2) < 0.5;
  }
  return e;
}

inline double wrap_half(double d) { return d - std::nearbyint(d); }

bool segment_hit(const ShapeEval& e, const double q[3]) {
  double t = (q[0] * e.u[0] + q[1] * e.u[1]) + q[2] * e.u[2];
  double a = q[0] - t * e.u[0], b = q[1] - t * e.u[1], c = q[2] - t * e.u[2];
  return std::fabs(t) <= e.half && ((a * a + b * b) + c * c) < e.r2;
}

bool inside(const ShapeEval& e, const double pt[3]) {
  switch (e.kind) {
    case PCX_SHAPE_SPHERE: {
      double d[3];
      for (int i = 0; i < 3; ++i) d[i] = wrap_half(pt[i] - e.p[i]);
      if (e.min_image) return ((d[0] * d[0] + d[1] * d[1]) + d[2] * d[2]) < e.r2;
      for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
          for (int c = -1; c <= 1; ++c) {
            double x = d[0] + a, y = d[1] + b, z = d[2] + c;
            if (((x * x + y * y) + z * z) < e.r2) return true;
          }
      return false;
    }
    case PCX_SHAPE_SEGMENT: {
      double d[3];
      for (int i = 0; i < 3; ++i) d[i] = wrap_half(pt[i] - e.mid[i]);
      if (e.min_image) return segment_hit(e, d);
      for (int a = -1; a <= 1; ++a)
        for (int b = -1; b <= 1; ++b)
          for (int c = -1; c <= 1; ++c) {
            double q[3] = {d[0] + a, d[1] + b, d[2] + c};
            if (segment_hit(e, q)) return true;
          }
      return false;
    }
    case PCX_SHAPE_BOX: {
      for (int i = 0; i < 3; ++i) {
        double x = pt[i] - std::floor(pt[i]);   // point wrapped to [0, 1)
        bool hit = false;
        for (int a = -1; a <= 1 && !hit; ++a) {
          double q = x + a;
          hit = (q >= e.p[i]) && (q < e.p[3 + i]);
        }
        if (!hit) return false;
      }
      return true;
    }
    case PCX_SHAPE_GYROID: {
      const double tp = 6.283185307179586;
      double x = tp * pt[0], y = tp * pt[1], z = tp * pt[2];
      double g = (std::sin(x) * std::cos(y) + std::sin(y) * std::cos(z)) + std::sin(z) * std::cos(x);
      return ((int)e.p[1] == 1) ? (std::fabs(g) > e.p[0]) : (g > e.p[0]);
    }
  }
  return false;
}

// Cholesky test of the Hermitian cell block [[d1,o12,o13],[.,d2,o23],[.,.,d3]].
bool block_hpd(const double* b) {
  double d1 = b[0], d2 = b[1], d3 = b[2];
  cd o12(b[3], b[4]), o13(b[5], b[6]), o23(b[7], b[8]);
  if (!(d1 > 0)) return false;
  double s22 = d2 - std::norm(o12) / d1;
  if (!(s22 > 0)) return false;
  cd s23 = o23 - std::conj(o12) * o13 / d1;
  double s33 = d3 - std::norm(o13) / d1;
  return (s33 - std::norm(s23) / s22) > 0;
}

template <typename T>
cudaError_t upload(void** dst, const std::vector<T>& src) {
  cudaError_t e = cudaMalloc(dst, src.size() * sizeof(T));
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice);
}

}  // namespace

double gamma_rule(const double k[3]) {
  double kn = std::sqrt(k[0] * k[0] + k[1] * k[1] + k[2] * k[2]);
  const double four_pi2 = 4.0 * M_PI * M_PI;
  if (kn == 0.0 || kn >= 1.0) return four_pi2;
  return four_pi2 / (kn * kn);
}

KParams make_kparams(const pcx_ctx* c, const double k[3], double gamma) {
  KParams kp{};   // value-initialised: graph keys compare KParams bytewise
  std::memcpy(kp.b, c->b, sizeof(kp.b));
  for (int j = 0; j < 3; ++j) {
    double kt = c->A[0 * 3 + j] * k[0] + c->A[1 * 3 + j] * k[1] + c->A[2 * 3 + j] * k[2];   // (A^T k)_j
    if (c->reading == PCX_CT_SUMMED) {
      kp.kt[j] = kt;
      kp.kq[j] = 0.0;
    } else {
      kp.kt[j] = 0.0;
      kp.kq[j] = k[j];
    }
  }
  // Per-mode form: the rule of Remark 2.6 applied to every Fourier mode with
  // that mode's own B eigenvalue |kappa_p|^2 (Lemma kc_ABblock) in place of
  // |k|^2, so gamma_p |kappa_p|^2 = 4 pi^2 max(1, |kappa_p|^2) >= 4 pi^2 for
  // every mode; the kernels take gamma_p = gamma max(1, 1/|kappa_p|^2).
  // Projector form: gamma_p = gamma / |kappa_p|^2, so that gamma_p K_B(p) is
  // gamma times the projector onto conj(kappa_p) and every penalty
  // eigenvalue equals gamma.  Its default is four times the rule's 4 pi^2:
  // all N^3 penalty eigenvalues sit at that one value, and a cluster that
  // close above the wanted ones would slow LOBPCG or enter the wanted set.
  kp.per_mode = c->penalty_form;
  const double four_pi2 = 4.0 * M_PI * M_PI;
  kp.gamma = gamma > 0 ? gamma : kp.per_mode == PCX_PENALTY_PROJECTOR ? 4.0 * four_pi2
                                                                      : kp.per_mode ? four_pi2 : gamma_rule(k);
  kp.diag_b = (c->b[1] == 0 && c->b[2] == 0 && c->b[3] == 0 && c->b[5] == 0 && c->b[6] == 0 && c->b[7] == 0);
  return kp;
}

pcx_status sample_blocks(const pcx_setup_desc* d, const double* A, std::vector<double>& blocks,
                         std::vector<int32_t>* ids, std::string& err) {
  const int n = d->n;
  const size_t n3 = (size_t)n * n * n;
  blocks.assign(n3 * 9, 0.0);
  if (ids) ids->assign(4 * n3, -1);
  if (d->cell_blocks) {
    std::memcpy(blocks.data(), d->cell_blocks, n3 * 9 * sizeof(double));
    return PCX_OK;
  }
  if (d->n_mat < 1 || !d->eps || d->background < 0 || d->background >= d->n_mat ||
      (d->n_shape > 0 && !d->shapes) || d->n_shape < 0) {
    err = "pcx_setup: bad material table or shape list";
    return PCX_EINVAL;
  }
  std::vector<cd> inv(9 * (size_t)d->n_mat);
  for (int mt = 0; mt < d->n_mat; ++mt) {
    cd a[9];
    for (int i = 0; i < 9; ++i) a[i] = cd(d->eps[18 * mt + 2 * i], d->eps[18 * mt + 2 * i + 1]);
    if (!invert3c(a, &inv[9 * mt])) {
      err = "pcx_setup: singular permittivity of material " + std::to_string(mt);
      return PCX_EINVAL;
    }
  }
  std::vector<ShapeEval> shapes;
  for (int s = 0; s < d->n_shape; ++s) {
    if (d->shapes[s].material < 0 || d->shapes[s].material >= d->n_mat || d->shapes[s].kind < 0 ||
        d->shapes[s].kind > 3) {
      err = "pcx_setup: bad shape " + std::to_string(s);
      return PCX_EINVAL;
    }
    shapes.push_back(prepare(d->shapes[s]));
  }
  const double h = 1.0 / n;
  const int bg = d->background;
  // half-index offsets of the point sets E1, E2, E3, V (Sec. 2.1)
  const double off[4][3] = {{0.5, 0, 0}, {0, 0.5, 0}, {0, 0, 0.5}, {0.5, 0.5, 0.5}};
#pragma omp parallel for schedule(dynamic, 1)
  for (int z = 0; z < n; ++z) {
    for (int y = 0; y < n; ++y) {
      for (int x = 0; x < n; ++x) {
        const size_t cell = ((size_t)z * n + y) * n + x;
        int mat[4];
        for (int set = 0; set < 4; ++set) {
          double f0 = ((x + 1) - off[set][0]) * h;
          double f1 = ((y + 1) - off[set][1]) * h;
          double f2 = ((z + 1) - off[set][2]) * h;
          double pt[3];
          for (int r = 0; r < 3; ++r) pt[r] = (A[3 * r] * f0 + A[3 * r + 1] * f1) + A[3 * r + 2] * f2;
          int id = bg;
          for (const ShapeEval& e : shapes)
            if (inside(e, pt)) {
              id = e.material;
              break;
            }
          mat[set] = id;
          if (ids) (*ids)[set * n3 + cell] = id;
        }
        double* blk = &blocks[9 * cell];
        blk[0] = inv[9 * mat[0] + 0].real();
        blk[1] = inv[9 * mat[1] + 4].real();
        blk[2] = inv[9 * mat[2] + 8].real();
        cd o12 = inv[9 * mat[3] + 1], o13 = inv[9 * mat[3] + 2], o23 = inv[9 * mat[3] + 5];
        blk[3] = o12.real();
        blk[4] = o12.imag();
        blk[5] = o13.real();
        blk[6] = o13.imag();
        blk[7] = o23.real();
        blk[8] = o23.imag();
      }
    }
  }
  return PCX_OK;
}

long long first_non_hpd(const std::vector<double>& blocks) {
  const size_t n3 = blocks.size() / 9;
  for (size_t i = 0; i < n3; ++i)
    if (!block_hpd(&blocks[9 * i])) return (long long)i;
  return -1;
}

// Sec. 3.3: sufficient conditions for M_CrossDoF (Sec. 3.2.2) to be HPD.
// Assumption 3.1 (the eigenvalues of every material's eps_1 lie in (0, 1])
// together with either Assumption 3.2 (strict diagonal dominance; with
// several materials it is checked row by row on the assembled matrix, whose
// off-diagonal rows hold the four-point means (e_ij(q) + e_ij(q')) / 8 of the
// symmetrised transfers) or Assumption 3.3 (a zero off-diagonal entry; with
// several materials, a position that is zero in every material, so that
// every eps_1 is tridiagonal in one common ordering).  Returns -1 when they
// hold, else the first cell where the guarantee fails (0 when a material
// breaks Assumption 3.1) and the reason in *why.
long long crossdof_unproven(int n, int n_mat, const double* eps, const std::vector<int32_t>& ids, std::string* why) {
  std::vector<cd> inv(9 * (size_t)n_mat);
  for (int mt = 0; mt < n_mat; ++mt) {
    cd a[9];
    for (int i = 0; i < 9; ++i) a[i] = cd(eps[18 * mt + 2 * i], eps[18 * mt + 2 * i + 1]);
    if (!invert3c(a, &inv[9 * mt])) {
      if (why) *why = "singular permittivity of material " + std::to_string(mt);
      return 0;
    }
    std::vector<cd> h(inv.begin() + 9 * mt, inv.begin() + 9 * mt + 9), v;
    std::vector<double> w;
    herm_eig(3, h, w, v);
    if (!(w[0] > 0) || w[2] > 1 + 1e-12) {
      if (why)
        *why = "eps_1 of material " + std::to_string(mt) + " has eigenvalues outside (0, 1] (Assumption 3.1)";
      return 0;
    }
  }
  // Assumption 3.3: an off-diagonal position that is zero in every material
  const int pos[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (const auto& pq : pos) {
    bool zero = true;
    for (int mt = 0; mt < n_mat && zero; ++mt) zero = inv[9 * mt + 3 * pq[0] + pq[1]] == cd(0, 0);
    if (zero) return -1;
  }
  // Assumption 3.2 on the assembled rows
  const size_t n3 = (size_t)n * n * n;
  int lg = 0;
  while ((1 << lg) < n) ++lg;   // n is a power of two
  const int msk = n - 1;
  auto at = [&](size_t q, const int* o) -> size_t {
    const int x = (int)(q & msk), y = (int)((q >> lg) & msk), z = (int)(q >> (2 * lg));
    return ((size_t)((z + o[0]) & msk) << (2 * lg)) | ((size_t)((y + o[1]) & msk) << lg) | (size_t)((x + o[2]) & msk);
  };
  auto e = [&](int mt, int i, int j) { return inv[9 * mt + 3 * i + j]; };
  // neighbour offsets (dz, dy, dx) of the transfers T_01, T_02, T_12 and of their transposes
  const int t01[4][3] = {{0, 0, 0}, {0, 0, -1}, {0, 1, 0}, {0, 1, -1}};
  const int t02[4][3] = {{0, 0, 0}, {0, 0, -1}, {1, 0, 0}, {1, 0, -1}};
  const int t12[4][3] = {{0, 0, 0}, {0, -1, 0}, {1, 0, 0}, {1, -1, 0}};
  const int* id0 = &ids[0];
  const int* id1 = &ids[n3];
  const int* id2 = &ids[2 * n3];
  for (size_t q = 0; q < n3; ++q) {
    double r0 = 0, r1 = 0, r2 = 0;
    for (int k = 0; k < 4; ++k) {
      const int m01[3] = {-t01[k][0], -t01[k][1], -t01[k][2]};
      const int m02[3] = {-t02[k][0], -t02[k][1], -t02[k][2]};
      const int m12[3] = {-t12[k][0], -t12[k][1], -t12[k][2]};
      r0 += std::abs(e(id0[q], 0, 1) + e(id1[at(q, t01[k])], 0, 1)) / 8;
      r0 += std::abs(e(id0[q], 0, 2) + e(id2[at(q, t02[k])], 0, 2)) / 8;
      r1 += std::abs(e(id0[at(q, m01)], 0, 1) + e(id1[q], 0, 1)) / 8;
      r1 += std::abs(e(id1[q], 1, 2) + e(id2[at(q, t12[k])], 1, 2)) / 8;
      r2 += std::abs(e(id0[at(q, m02)], 0, 2) + e(id2[q], 0, 2)) / 8;
      r2 += std::abs(e(id1[at(q, m12)], 1, 2) + e(id2[q], 1, 2)) / 8;
    }
    if (!(e(id0[q], 0, 0).real() > r0) || !(e(id1[q], 1, 1).real() > r1) || !(e(id2[q], 2, 2).real() > r2)) {
      if (why)
        *why = "no material position zero in every eps_1 (Assumption 3.3) and the assembled M_CrossDoF is "
               "not strictly diagonally dominant (Assumption 3.2)";
      return (long long)q;
    }
  }
  return -1;
}

pcx_status validate_desc(const pcx_setup_desc* d, std::string& err) {
  const int n = d->n;
  if (!is_pow2(n) || n < 8 || n > 256) {
    err = "pcx_setup: N must be a power of two in [8, 256]";
    return PCX_EINVAL;
  }
  if (d->stencil_m < 1 || d->stencil_m > 5 || n < 2 * d->stencil_m) {
    err = "pcx_setup: stencil_m must be in [1, 5] with N >= 2 m";
    return PCX_EINVAL;
  }
  if (d->ct_reading != PCX_CT_SUMMED && d->ct_reading != PCX_CT_LITERAL) {
    err = "pcx_setup: unknown ct_reading";
    return PCX_EINVAL;
  }
  if (d->m_kind != PCX_M_TRIVIAL && d->m_kind != PCX_M_CROSSDOF) {
    err = "pcx_setup: unknown m_kind";
    return PCX_EINVAL;
  }
  if (d->m_kind == PCX_M_CROSSDOF && (d->cell_blocks || d->n_mat > 255)) {
    err = "pcx_setup: M_CrossDoF needs a structure sampled from shapes with at most 255 materials";
    return PCX_EINVAL;
  }
  double inv[9];
  if (!invert3(d->lattice, inv)) {
    err = "pcx_setup: singular lattice matrix";
    return PCX_EINVAL;
  }
  return PCX_OK;
}

pcx_status setup_context(const pcx_setup_desc* d, pcx_ctx* c) {
  pcx_status st = validate_desc(d, c->err);
  if (st != PCX_OK) return st;
  const int n = d->n;
  c->n = n;
  c->m = d->stencil_m;
  c->reading = d->ct_reading;
  c->m_kind = d->m_kind;
  std::memcpy(c->A, d->lattice, sizeof(c->A));
  invert3(c->A, c->b);
  const size_t n3 = (size_t)n * n * n;
  std::vector<int32_t> ids;
  const bool use_ids = !d->cell_blocks && d->n_mat <= 255;
  st = sample_blocks(d, c->A, c->blocks, use_ids ? &ids : nullptr, c->err);
  if (st != PCX_OK) return st;
  if (c->m_kind == PCX_M_CROSSDOF && !d->crossdof_unchecked) {
    // M_CrossDoF: the sufficient conditions of Sec. 3.3
    std::string why;
    const long long bad = crossdof_unproven(n, d->n_mat, d->eps, ids, &why);
    if (bad >= 0) {
      long long x = bad % n, y = (bad / n) % n, z = bad / ((long long)n * n);
      c->err = "pcx_setup: M_CrossDoF not proven HPD (Sec. 3.3): " + why + "; first cell (x, y, z) = (" +
               std::to_string(x) + ", " + std::to_string(y) + ", " + std::to_string(z) + ")";
      return PCX_ENOTHPD;
    }
  }
  // HPD check of every cell block (Lemma 3.5: spectrum of M = union of blocks)
  const long long bad = c->m_kind == PCX_M_CROSSDOF ? -1 : first_non_hpd(c->blocks);
  if (bad >= 0) {
    long long x = bad % n, y = (bad / n) % n, z = bad / ((long long)n * n);
    c->err = "pcx_setup: cell block not HPD at (x, y, z) = (" + std::to_string(x) + ", " +
             std::to_string(y) + ", " + std::to_string(z) + ")";
    return PCX_ENOTHPD;
  }

  // device tables
  symbol_tables(n, c->m, c->lam1, c->lam0);
  std::vector<double> lam64(4 * (size_t)n);
  std::vector<float> lam32(4 * (size_t)n);
  for (int p = 0; p < n; ++p) {
    lam64[2 * p] = c->lam1[p].real();
    lam64[2 * p + 1] = c->lam1[p].imag();
    lam64[2 * n + 2 * p] = c->lam0[p].real();
    lam64[2 * n + 2 * p + 1] = c->lam0[p].imag();
  }
  for (size_t i = 0; i < lam64.size(); ++i) lam32[i] = (float)lam64[i];
  std::vector<double> tw64(2 * (size_t)n);
  std::vector<float> tw32(2 * (size_t)n);
  const ld two_pi = 6.283185307179586476925286766559005768L;
  for (int mm = 0; mm < n; ++mm) {
    ld a = two_pi * (ld)mm / (ld)n;
    tw64[2 * mm] = (double)std::cos(a);
    tw64[2 * mm + 1] = (double)(-std::sin(a));
    tw32[2 * mm] = (float)std::cos(a);
    tw32[2 * mm + 1] = (float)(-std::sin(a));
  }
  cudaError_t e;
  if ((e = cudaGetDevice(&c->device)) != cudaSuccess || (e = upload(&c->dev.lam64, lam64)) != cudaSuccess ||
      (e = upload(&c->dev.lam32, lam32)) != cudaSuccess || (e = upload(&c->dev.tw64, tw64)) != cudaSuccess ||
      (e = upload(&c->dev.tw32, tw32)) != cudaSuccess)
    goto cuda_error;
  if (use_ids) {
    // uchar4 per cell + per-material table of (epsilon_1)_11, _22, _33, _12, _13, _23
    std::vector<uint8_t> mid(4 * n3);
    for (int set = 0; set < 4; ++set)
      for (size_t i = 0; i < n3; ++i) mid[4 * i + set] = (uint8_t)ids[set * n3 + i];
    std::vector<cd> inv(9 * (size_t)d->n_mat);
    for (int mt = 0; mt < d->n_mat; ++mt) {
      cd a[9];
      for (int i = 0; i < 9; ++i) a[i] = cd(d->eps[18 * mt + 2 * i], d->eps[18 * mt + 2 * i + 1]);
      invert3c(a, &inv[9 * mt]);
    }
    std::vector<double> t64(9 * (size_t)d->n_mat);
    for (int mt = 0; mt < d->n_mat; ++mt) {
      const cd* v = &inv[9 * mt];
      const double row[9] = {v[0].real(), v[4].real(), v[8].real(), v[1].real(), v[1].imag(),
                             v[2].real(), v[2].imag(), v[5].real(), v[5].imag()};
      for (int f = 0; f < 9; ++f) t64[9 * mt + f] = row[f];
    }
    std::vector<float> t32(t64.begin(), t64.end());
    // the same entries in 16-byte aligned records of 12 (the three-pass z
    // tiles read a cell's off-diagonals with one 16-byte and one 8-byte load)
    std::vector<float> t12(12 * (size_t)d->n_mat, 0.f);
    for (int mt = 0; mt < d->n_mat; ++mt)
      for (int f = 0; f < 9; ++f) t12[12 * mt + (f < 3 ? f : f + 1)] = t32[9 * mt + f];
    c->dev.n_mat = d->n_mat;
    if ((e = upload(&c->dev.mid, mid)) != cudaSuccess || (e = upload(&c->dev.mtab64, t64)) != cudaSuccess ||
        (e = upload(&c->dev.mtab32, t32)) != cudaSuccess || (e = upload(&c->dev.mtab12, t12)) != cudaSuccess ||
        (e = build_pass3_ids(c)) != cudaSuccess)
      goto cuda_error;
  } else {
    std::vector<double> m64(9 * n3);
    for (size_t i = 0; i < n3; ++i)
      for (int f = 0; f < 9; ++f) m64[f * n3 + i] = c->blocks[9 * i + f];
    std::vector<float> m32(m64.begin(), m64.end());
    if ((e = upload(&c->dev.m64, m64)) != cudaSuccess || (e = upload(&c->dev.m32, m32)) != cudaSuccess)
      goto cuda_error;
  }
  {
    int l2 = 0;
    if (cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, c->device) == cudaSuccess) c->l2_bytes = (size_t)l2;
  }
  return PCX_OK;
cuda_error:
  {
    c->err = std::string("pcx_setup: CUDA error ") + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? PCX_ENOMEM : PCX_ECUDA;
  }
}

}  // namespace pcx
