// Host-side parameter selection of phiks (Sec. 3.3) and quadrature rules.
#pragma once

#include <cstdint>
#include <vector>

namespace phiks {

struct Rect {  // [xlo, xhi] x i[ylo, yhi]
  double xlo = 0, xhi = 0, ylo = 0, yhi = 0;
};

// Nodes theta_1 < ... < theta_q on [0, 1] and weights: Gauss-Lobatto-Legendre
// (rule 0; theta_1 = 0, theta_q = 1) or Gauss-Legendre (rule 1).
void quad_rule(int rule, int q, std::vector<double>& theta, std::vector<double>& w);

// Rectangle enclosing the numerical range of a real n x n column-major A:
// real part in [lambda_min(H), lambda_max(H)], H = (A + A^T)/2; imaginary part
// in [-||S||_2, ||S||_2], S = (A - A^T)/2.
Rect numerical_range_rect(const double* A, int64_t n);

// Rectangle enclosing the numerical range of a complex n x n A (interleaved
// real and imaginary parts, column-major): real part in the eigenvalue range
// of H = (A + A^*)/2, imaginary part in that of S = (A - A^*)/(2i), both
// Hermitian, taken from their real representations [[Re, -Im], [Im, Re]]
// (real symmetric, the same eigenvalues each twice).
Rect numerical_range_rect_complex(const double* A, int64_t n);

// ||A||_1 (max column sum), column-major.
double norm1(const double* A, int64_t n);

struct Selection {
  int s = -1, q = -1, tcount = -1;
};

// Task kind: 0 = same vector (eq. Tpsv), 1 = linear combination (eq. Tlcp).
int tucker_count(int kind, int s, int nscales, int q, int p);

// Bounds b[l-1] >= ||R_q(f_l(., K/2^s))||_2 (eq. CPestimate), l = 1..p, for the
// rectangle `xi` enclosing W(tau K), for every q in qs (result row-major:
// out[iq * p + l - 1]).
void remainder_bounds(const Rect& xi, int s, const std::vector<int>& qs, int p, int rule,
                      std::vector<double>& out);

// The (s, q) of Sec. 3.3 for the task `kind`, given the vector norms (same
// vector: vnorms[0] = ||v||; linear combination: vnorms[l] = ||v_l||, l=0..p).
// Returns false when no (s, q) in range meets the tolerance.
bool select_params(const Rect& xi, int p, int kind, const double* vnorms, int nscales,
                   double tol, int qmin, int qmax, int rule, Selection* out);

}  // namespace phiks
