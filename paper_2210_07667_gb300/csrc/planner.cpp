// Parameter selection of phiks (Sec. 3.3), quadrature rules and numerical-
// range rectangles, on the host in FP64.
//
// Remainder of the quadrature (eq. remainder): R_q(f) = (1/2 pi i) oint k_q(z)
// f(z, K) dz, k_q(z) = int_0^1 pi_q(t) / (pi_q(z) (z - t)) dt.  Contour: the
// ellipse Gamma_r with foci {0, 1} and capacity r > 1/4,
// z(zeta) = r e^{i zeta} + 1/2 + e^{-i zeta}/(16 r).  Estimate (eq. CPestimate):
// ||R_q(f_l(., K))||_2 <= (1 + sqrt 2)/(2 pi) sup_{w on the boundary of Xi}
// | int_0^{2 pi} k_q(z) f_l(z, w) (r e^{i zeta} - e^{-i zeta}/(16 r)) dzeta |,
// f_l(z, w) = z^{l-1}/(l-1)! exp((1 - z) w).
//
// Readings of what the paper leaves open: the integral does not depend on r
// (Cauchy), so each trapezoidal value plus its estimated numerical error is
// minimised over 24 log-spaced values of r in [0.3, 8] separately for each
// (q, s, l); the boundary of Xi sampled
// with 64 points per side; the zeta integral by the 128-point trapezoidal
// rule; k_q by 128-point Gauss-Legendre in t; stopping rule: s = 0, 1, ...,
// q_s the smallest feasible q, stop at the first s whose T# exceeds the
// previous one (ties continue; an infeasible s counts as T# = infinity),
// s <= 64; s is raised to nscales - 1 if needed.
#include "planner.hpp"

#include <algorithm>
#include <cmath>
#include <complex>
#include <limits>
#include <map>
#include <mutex>
#include <thread>
#include <tuple>

namespace phiks {

using cd = std::complex<double>;

namespace {

constexpr int kNR = 24;
constexpr double kRLo = 0.3, kRHi = 8.0;
constexpr int kNSide = 64;
constexpr int kNZeta = 128;
constexpr int kNT = 128;
constexpr int kSMax = 64;
const double kPi = 3.14159265358979323846;

// Legendre P_n(x) and P'_n(x) by the three-term recurrence.
void legendre(int n, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (n == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 2; k <= n; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  // (1 - x^2) P'_n = n (P_{n-1} - x P_n)
  *dP = n * (p0 - x * p1) / (1.0 - x * x);
}

// Gauss-Legendre nodes/weights on [-1, 1] by Newton from Chebyshev guesses.
void gauss_legendre(int q, std::vector<double>& x, std::vector<double>& w) {
  x.assign(q, 0.0);
  w.assign(q, 0.0);
  for (int i = 0; i < q; ++i) {
    double z = std::cos(kPi * (i + 0.75) / (q + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(q, z, &P, &dP);
      double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP;
    legendre(q, z, &P, &dP);
    x[q - 1 - i] = z;
    w[q - 1 - i] = 2.0 / ((1.0 - z * z) * dP * dP);
  }
}

// Interior Gauss-Lobatto nodes: roots of P'_{m}, m = q - 1, by Newton with
// P''_m from the Legendre equation (1 - x^2) P'' = 2 x P' - m (m + 1) P.
void gll_interior(int q, std::vector<double>& x) {
  int m = q - 1;
  x.clear();
  for (int i = 1; i < m; ++i) {
    double z = -std::cos(kPi * i / m);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(m, z, &P, &dP);
      double d2P = (2.0 * z * dP - m * (m + 1.0) * P) / (1.0 - z * z);
      double dz = dP / d2P;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x.push_back(z);
  }
  std::sort(x.begin(), x.end());
}

// Largest and smallest eigenvalues of a symmetric tridiagonal matrix
// (diag a[0..n-1], off-diagonal b[0..n-2]) by Sturm-sequence bisection.
int sturm_count(const std::vector<double>& a, const std::vector<double>& b, double x) {
  // number of eigenvalues < x
  int cnt = 0;
  double dprev = 1.0;
  const size_t n = a.size();
  for (size_t i = 0; i < n; ++i) {
    double off = (i == 0) ? 0.0 : b[i - 1] * b[i - 1];
    double d = (a[i] - x) - (i == 0 ? 0.0 : off / dprev);
    if (d == 0.0) d = -1e-300;
    if (d < 0) ++cnt;
    dprev = d;
  }
  return cnt;
}

void tridiag_extremes(const std::vector<double>& a, const std::vector<double>& b, double* lmin,
                      double* lmax) {
  const size_t n = a.size();
  double lo = std::numeric_limits<double>::infinity(), hi = -lo;
  for (size_t i = 0; i < n; ++i) {
    double r = (i > 0 ? std::fabs(b[i - 1]) : 0.0) + (i + 1 < n ? std::fabs(b[i]) : 0.0);
    lo = std::min(lo, a[i] - r);
    hi = std::max(hi, a[i] + r);
  }
  double span = std::max(hi - lo, 1e-300);
  lo -= 1e-12 * span + 1e-300;
  hi += 1e-12 * span + 1e-300;
  auto bisect = [&](int k) {  // k-th smallest eigenvalue (0-based)
    double l = lo, h = hi;
    for (int it = 0; it < 200 && h - l > 1e-15 * std::max(std::fabs(l), std::fabs(h)) + 1e-300;
         ++it) {
      double mid = 0.5 * (l + h);
      if (sturm_count(a, b, mid) > k) h = mid; else l = mid;
    }
    return 0.5 * (l + h);
  };
  *lmin = bisect(0);
  *lmax = bisect((int)n - 1);
}

// Householder reduction of a symmetric column-major M (n x n, overwritten) to
// tridiagonal form: diagonal a, off-diagonal b.
void householder_tridiag(std::vector<double>& M, int64_t n, std::vector<double>& a,
                         std::vector<double>& b) {
  auto at = [&](int64_t i, int64_t j) -> double& { return M[i + n * j]; };
  std::vector<double> v(n), p(n), w(n);
  for (int64_t k = 0; k + 2 < n; ++k) {
    double alpha = 0;
    for (int64_t i = k + 1; i < n; ++i) alpha += at(i, k) * at(i, k);
    alpha = std::sqrt(alpha);
    if (alpha == 0) continue;
    if (at(k + 1, k) > 0) alpha = -alpha;
    double r = std::sqrt(0.5 * (alpha * alpha - at(k + 1, k) * alpha));
    if (r == 0) continue;
    for (int64_t i = 0; i < n; ++i) v[i] = 0;
    v[k + 1] = (at(k + 1, k) - alpha) / (2 * r);
    for (int64_t i = k + 2; i < n; ++i) v[i] = at(i, k) / (2 * r);
    // M <- H M H, H = I - 2 v v^T: p = M v, K = v^T p, w = p - K v, M -= 2(v w^T + w v^T)
    for (int64_t i = k; i < n; ++i) {
      double s = 0;
      for (int64_t j = k + 1; j < n; ++j) s += at(i, j) * v[j];
      p[i] = s;
    }
    double K = 0;
    for (int64_t i = k + 1; i < n; ++i) K += v[i] * p[i];
    for (int64_t i = k; i < n; ++i) w[i] = p[i] - K * v[i];
    for (int64_t j = k; j < n; ++j)
      for (int64_t i = k; i < n; ++i) at(i, j) -= 2.0 * (v[i] * w[j] + w[i] * v[j]);
  }
  a.resize(n);
  b.resize(n > 0 ? n - 1 : 0);
  for (int64_t i = 0; i < n; ++i) a[i] = at(i, i);
  for (int64_t i = 0; i + 1 < n; ++i) b[i] = at(i + 1, i);
}

bool is_tridiagonal(const std::vector<double>& M, int64_t n) {
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i)
      if ((i > j + 1 || j > i + 1) && M[i + n * j] != 0.0) return false;
  return true;
}

void sym_extremes(std::vector<double> M, int64_t n, double* lmin, double* lmax) {
  std::vector<double> a, b;
  if (is_tridiagonal(M, n)) {
    a.resize(n);
    b.resize(n > 0 ? n - 1 : 0);
    for (int64_t i = 0; i < n; ++i) a[i] = M[i + n * i];
    for (int64_t i = 0; i + 1 < n; ++i) b[i] = M[i + 1 + n * i];
  } else {
    householder_tridiag(M, n, a, b);
  }
  tridiag_extremes(a, b, lmin, lmax);
}

std::vector<double> r_grid() {
  std::vector<double> r(kNR);
  for (int i = 0; i < kNR; ++i)
    r[i] = std::exp(std::log(kRLo) + (std::log(kRHi) - std::log(kRLo)) * i / (kNR - 1));
  return r;
}

std::vector<cd> rect_boundary(const Rect& xi) {
  std::vector<cd> pts;
  if (xi.xhi > xi.xlo) {
    for (int k = 0; k < kNSide; ++k) {
      double t = (double)k / kNSide;
      pts.emplace_back(xi.xlo + (xi.xhi - xi.xlo) * t, xi.ylo);
    }
    for (int k = 0; k < kNSide; ++k) {
      double t = (double)k / kNSide;
      pts.emplace_back(xi.xhi - (xi.xhi - xi.xlo) * t, xi.yhi);
    }
  } else {
    pts.emplace_back(xi.xlo, xi.ylo);
    pts.emplace_back(xi.xlo, xi.yhi);
  }
  if (xi.yhi > xi.ylo) {
    for (int k = 0; k < kNSide; ++k) {
      double t = (double)k / kNSide;
      pts.emplace_back(xi.xhi, xi.ylo + (xi.yhi - xi.ylo) * t);
    }
    for (int k = 0; k < kNSide; ++k) {
      double t = (double)k / kNSide;
      pts.emplace_back(xi.xlo, xi.yhi - (xi.yhi - xi.ylo) * t);
    }
  } else {
    pts.emplace_back(xi.xlo, xi.ylo);
    pts.emplace_back(xi.xhi, xi.ylo);
  }
  return pts;
}

// k_q(z_m) on the ellipse of capacity r, for the q nodes.
void kernel_on_ellipse(const std::vector<double>& nodes, const std::vector<cd>& z,
                       const std::vector<double>& tgl, const std::vector<double>& wgl,
                       std::vector<cd>& k) {
  k.assign(z.size(), cd(0, 0));
  for (size_t m = 0; m < z.size(); ++m) {
    cd acc(0, 0);
    for (size_t j = 0; j < tgl.size(); ++j) {
      cd ratio(1, 0);
      for (double th : nodes) ratio *= (tgl[j] - th) / (z[m] - th);
      acc += wgl[j] * ratio / (z[m] - tgl[j]);
    }
    k[m] = acc;
  }
}

double factorial(int k) {
  double f = 1;
  for (int i = 2; i <= k; ++i) f *= i;
  return f;
}

bool feasible(int kind, const double* b, int s, int p, const double* vnorms, double tol) {
  if (kind == 0) {
    for (int l = 1; l <= p; ++l)
      if (!(b[l - 1] * vnorms[0] <= tol * std::ldexp(1.0, l * s))) return false;
    return true;
  }
  for (int l = 1; l <= p; ++l) {
    double tot = 0;
    for (int k = 1; k <= l; ++k)
      tot += b[l - k] * vnorms[p + 1 - k] / std::ldexp(1.0, (l - k + 1) * s);
    if (!(tot <= tol)) return false;
  }
  return true;
}

int smallest_q(const Rect& xi, int s, int p, int kind, const double* vnorms, double tol, int qmin,
               int qmax, int rule) {
  std::vector<int> qs;
  for (int q = qmin; q <= qmax; ++q) qs.push_back(q);
  std::vector<double> b;
  remainder_bounds(xi, s, qs, p, rule, b);
  for (size_t iq = 0; iq < qs.size(); ++iq)
    if (feasible(kind, &b[iq * p], s, p, vnorms, tol)) return qs[iq];
  return -1;
}

}  // namespace

void quad_rule(int rule, int q, std::vector<double>& theta, std::vector<double>& w) {
  theta.clear();
  w.clear();
  if (rule == 0) {
    std::vector<double> x;
    gll_interior(q, x);
    std::vector<double> all;
    all.push_back(-1.0);
    for (double v : x) all.push_back(v);
    all.push_back(1.0);
    for (double xv : all) {
      double P, dP;
      if (xv == 1.0 || xv == -1.0) {
        P = (xv == 1.0 || (q - 1) % 2 == 0) ? 1.0 : -1.0;
      } else {
        legendre(q - 1, xv, &P, &dP);
      }
      theta.push_back((xv + 1.0) / 2.0);
      w.push_back(1.0 / (q * (q - 1.0) * P * P));
    }
  } else {
    std::vector<double> x, ww;
    gauss_legendre(q, x, ww);
    for (int i = 0; i < q; ++i) {
      theta.push_back((x[i] + 1.0) / 2.0);
      w.push_back(ww[i] / 2.0);
    }
  }
}

double norm1(const double* A, int64_t n) {
  double m = 0;
  for (int64_t j = 0; j < n; ++j) {
    double s = 0;
    for (int64_t i = 0; i < n; ++i) s += std::fabs(A[i + n * j]);
    m = std::max(m, s);
  }
  return m;
}

Rect numerical_range_rect_complex(const double* A, int64_t n) {
  const int64_t m = 2 * n;
  std::vector<double> RH(m * m), RS(m * m);
  auto re = [&](int64_t i, int64_t j) { return A[2 * (i + n * j)]; };
  auto im = [&](int64_t i, int64_t j) { return A[2 * (i + n * j) + 1]; };
  auto put = [&](std::vector<double>& R, int64_t i, int64_t j, double xr, double xi) {
    R[i + m * j] = xr;
    R[n + i + m * j] = xi;
    R[i + m * (n + j)] = -xi;
    R[n + i + m * (n + j)] = xr;
  };
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      // H_ij = (A_ij + conj(A_ji)) / 2;  S_ij = (A_ij - conj(A_ji)) / (2i)
      put(RH, i, j, 0.5 * (re(i, j) + re(j, i)), 0.5 * (im(i, j) - im(j, i)));
      put(RS, i, j, 0.5 * (im(i, j) + im(j, i)), -0.5 * (re(i, j) - re(j, i)));
    }
  Rect r;
  sym_extremes(RH, m, &r.xlo, &r.xhi);
  sym_extremes(RS, m, &r.ylo, &r.yhi);
  return r;
}

Rect numerical_range_rect(const double* A, int64_t n) {
  std::vector<double> H(n * n), S2(n * n);
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) H[i + n * j] = 0.5 * (A[i + n * j] + A[j + n * i]);
  Rect r;
  sym_extremes(H, n, &r.xlo, &r.xhi);
  // ||S||_2 with S = (A - A^T)/2 skew: the tridiagonal form of a skew matrix
  // has zero diagonal and off-diagonal e; its singular values are the
  // eigenvalues of the symmetric tridiagonal with off-diagonal |e|.
  std::vector<double> S(n * n);
  bool zero = true;
  for (int64_t j = 0; j < n; ++j)
    for (int64_t i = 0; i < n; ++i) {
      S[i + n * j] = 0.5 * (A[i + n * j] - A[j + n * i]);
      if (S[i + n * j] != 0) zero = false;
    }
  double m = 0;
  if (!zero) {
    // -S^2 = S^T S is symmetric PSD; ||S||_2^2 = lambda_max(S^T S).  For a
    // tridiagonal S use the symmetric tridiagonal with off-diagonal |e|.
    if (is_tridiagonal(S, n)) {
      std::vector<double> a(n, 0.0), b(n > 0 ? n - 1 : 0);
      for (int64_t i = 0; i + 1 < n; ++i) b[i] = std::fabs(S[i + 1 + n * i]);
      double lmin, lmax;
      tridiag_extremes(a, b, &lmin, &lmax);
      m = std::max(std::fabs(lmin), std::fabs(lmax));
    } else {
      for (int64_t j = 0; j < n; ++j)
        for (int64_t i = 0; i < n; ++i) {
          double acc = 0;
          for (int64_t k = 0; k < n; ++k) acc += S[k + n * i] * S[k + n * j];
          S2[i + n * j] = acc;
        }
      double lmin, lmax;
      sym_extremes(S2, n, &lmin, &lmax);
      m = std::sqrt(std::max(lmax, 0.0));
    }
  }
  r.ylo = -m;
  r.yhi = m;
  return r;
}

int tucker_count(int kind, int s, int nscales, int q, int p) {
  return kind == 0 ? q + s * p + nscales : q * p + s * p + nscales;
}

namespace {

// k_q(z(zeta_m)) on the ellipse of capacity r_grid()[ir], for the rule's q
// nodes: independent of the operator, so computed once per process.
struct KernelKey {
  int rule, q, ir;
  bool operator<(const KernelKey& o) const {
    return std::tie(rule, q, ir) < std::tie(o.rule, o.q, o.ir);
  }
};
std::mutex g_kernel_mu;
std::map<KernelKey, std::vector<cd>> g_kernel_cache;

const std::vector<cd>& cached_kernel(int rule, int q, int ir, const std::vector<cd>& z) {
  {
    std::lock_guard<std::mutex> lk(g_kernel_mu);
    auto it = g_kernel_cache.find({rule, q, ir});
    if (it != g_kernel_cache.end()) return it->second;
  }
  std::vector<double> xg, wg, nodes, wts;
  gauss_legendre(kNT, xg, wg);
  for (int j = 0; j < kNT; ++j) {
    xg[j] = (xg[j] + 1.0) / 2.0;
    wg[j] /= 2.0;
  }
  quad_rule(rule, q, nodes, wts);
  std::vector<cd> k;
  kernel_on_ellipse(nodes, z, xg, wg, k);
  std::lock_guard<std::mutex> lk(g_kernel_mu);
  return g_kernel_cache.emplace(KernelKey{rule, q, ir}, std::move(k)).first->second;
}

}  // namespace

void remainder_bounds(const Rect& xi, int s, const std::vector<int>& qs, int p, int rule,
                      std::vector<double>& out) {
  const std::vector<double> rs = r_grid();
  std::vector<cd> w = rect_boundary(xi);
  const double scale = std::ldexp(1.0, -s);
  for (auto& x : w) x *= scale;
  const size_t nw = w.size();
  const double inf = std::numeric_limits<double>::infinity();
  const size_t nq = qs.size();
  std::vector<double> best_r(kNR * nq * p, inf);
  auto work = [&](int ir) {
    const double r = rs[ir];
    std::vector<cd> z(kNZeta), dz(kNZeta);
    for (int m = 0; m < kNZeta; ++m) {
      double zeta = 2.0 * kPi * m / kNZeta;
      cd e = std::exp(cd(0, zeta)), ei = std::exp(cd(0, -zeta));
      z[m] = r * e + 0.5 + ei / (16.0 * r);
      dz[m] = r * e - ei / (16.0 * r);
    }
    // exp((1 - z_m) w) as separate real and imaginary arrays and moduli, [w][m]
    std::vector<double> Er(nw * kNZeta), Ei(nw * kNZeta), Ea(nw * kNZeta);
    for (size_t iw = 0; iw < nw; ++iw)
      for (int m = 0; m < kNZeta; ++m) {
        cd e = std::exp((1.0 - z[m]) * w[iw]);
        Er[iw * kNZeta + m] = e.real();
        Ei[iw * kNZeta + m] = e.imag();
        Ea[iw * kNZeta + m] = std::abs(e);
      }
    std::vector<double> cr(kNZeta), ci(kNZeta), ca(kNZeta);
    for (size_t iq = 0; iq < nq; ++iq) {
      const std::vector<cd>& k = cached_kernel(rule, qs[iq], ir, z);
      for (int l = 1; l <= p; ++l) {
        const double fl = factorial(l - 1);
        for (int m = 0; m < kNZeta; ++m) {
          cd c = k[m] * std::pow(z[m], l - 1) / fl * dz[m];
          cr[m] = c.real();
          ci[m] = c.imag();
          ca[m] = std::abs(c);
        }
        // the integral is the same for every r (Cauchy): each value carries
        // its estimated numerical error, the rule on every other node
        // (|I_N - I_N/2|) and rounding (N 2^-53 sum |terms|), so that a value
        // small only because it is inaccurate is not the minimum over r
        double mx = 0;
        bool bad = false;
        for (size_t iw = 0; iw < nw; ++iw) {
          const double* er = &Er[iw * kNZeta];
          const double* ei = &Ei[iw * kNZeta];
          const double* ea = &Ea[iw * kNZeta];
          double sr = 0, si = 0, hr = 0, hi = 0, sa = 0;
          for (int m = 0; m < kNZeta; ++m) {
            const double tr = cr[m] * er[m] - ci[m] * ei[m];
            const double ti = cr[m] * ei[m] + ci[m] * er[m];
            sr += tr;
            si += ti;
            if ((m & 1) == 0) {
              hr += tr;
              hi += ti;
            }
            sa += ca[m] * ea[m];
          }
          const double a = std::hypot(sr, si) + std::hypot(sr - 2.0 * hr, si - 2.0 * hi) +
                           kNZeta * std::ldexp(1.0, -53) * sa;
          if (!std::isfinite(a)) {
            bad = true;
            break;
          }
          mx = std::max(mx, a);
        }
        double val = mx * (1.0 + std::sqrt(2.0)) / kNZeta;
        if (!bad && std::isfinite(val)) best_r[(ir * nq + iq) * p + (l - 1)] = val;
      }
    }
  };
  unsigned nth = std::max(1u, std::min<unsigned>(std::thread::hardware_concurrency(), kNR));
  std::vector<std::thread> th;
  for (unsigned t = 0; t < nth; ++t)
    th.emplace_back([&, t]() {
      for (int ir = (int)t; ir < kNR; ir += (int)nth) work(ir);
    });
  for (auto& x : th) x.join();
  out.assign(nq * p, inf);
  for (int ir = 0; ir < kNR; ++ir)
    for (size_t i = 0; i < nq * (size_t)p; ++i) out[i] = std::min(out[i], best_r[ir * nq * p + i]);
}

bool select_params(const Rect& xi, int p, int kind, const double* vnorms, int nscales, double tol,
                   int qmin, int qmax, int rule, Selection* out) {
  const double inf = std::numeric_limits<double>::infinity();
  bool have = false;
  int ps = -1, pq = -1;
  double pT = inf;
  for (int s = 0; s <= kSMax; ++s) {
    int q = smallest_q(xi, s, p, kind, vnorms, tol, qmin, qmax, rule);
    double T = q < 0 ? inf : (double)tucker_count(kind, s, nscales, q, p);
    if (have && T > pT) break;
    have = true;
    ps = s;
    pq = q;
    pT = T;
  }
  if (!have || pq < 0) return false;
  int s = ps, q = pq;
  if (s < nscales - 1) {
    s = nscales - 1;
    q = -1;
    while (q < 0 && s <= kSMax) {
      q = smallest_q(xi, s, p, kind, vnorms, tol, qmin, qmax, rule);
      if (q < 0) ++s;
    }
    if (q < 0) return false;
  }
  out->s = s;
  out->q = q;
  out->tcount = tucker_count(kind, s, nscales, q, p);
  return true;
}

}  // namespace phiks
