// Small dense FP64 complex linear algebra (host) for Rayleigh-Ritz.
#pragma once

#include <complex>
#include <vector>

namespace pcx {

using cd = std::complex<double>;

// Hermitian eigen-decomposition (cyclic Jacobi). a: n x n row-major
// (destroyed); w ascending; column j of v (row-major n x n) pairs with w[j].
void herm_eig(int n, std::vector<cd>& a, std::vector<double>& w, std::vector<cd>& v);

// G = R^H R with R upper triangular (row-major). Returns false if G is not
// numerically positive definite.
bool cholesky_upper(int n, const std::vector<cd>& g, std::vector<cd>& r);

// Inverse of an upper-triangular matrix (row-major).
void upper_inverse(int n, const std::vector<cd>& r, std::vector<cd>& ri);

// Generalised Hermitian eigenproblem ga c = theta gb c on the span that gb
// resolves: directions whose scaled gb eigenvalue is <= drop_tol * max are
// dropped.  Returns the rank r kept (or -1 on breakdown); theta[r]
// ascending, c is m x r row-major with gb-orthonormal columns.  lam_min_rel
// (optional) receives the smallest kept eigenvalue of the unit-diagonal
// scaled gb over the largest (a lower bound of it on the Cholesky path): the
// rounding errors of ga reach theta amplified by about its inverse.
int gen_eig(int m, const std::vector<cd>& ga, const std::vector<cd>& gb, double drop_tol, std::vector<double>& theta,
            std::vector<cd>& c, double* lam_min_rel = nullptr);

}  // namespace pcx
