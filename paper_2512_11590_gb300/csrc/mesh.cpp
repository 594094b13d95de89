// Lagrange-Legendre mesh on (0, a) and the kinetic + Bloch matrix, on the host
// in IEEE double (Sec. 2 of the paper: Gauss-Legendre points r_i, weights
// lambda_i, Lagrange property f_i(r_j) = delta_ij / sqrt(lambda_j)).
//
// Compiled with -ffp-contract=off: every expression is a sequence of single
// rounded double operations, so the tables are reproducible bit for bit on any
// IEEE host.  The collision matrix is sensitive to the mesh nodes (a 1-ulp
// change of every node moves U by ~1e-10 at nlag = 50, because the closed-form
// kinetic matrix is exact only at the true zeros), so the nodes are polished to
// correctly rounded values with a double-double Newton step.
#include <cmath>
#include <vector>

#include "rmat_internal.h"

namespace {

struct dd {
  double hi, lo;
};

// Knuth two-sum and the fused-multiply-add two-product (both exact).
inline dd two_sum(double a, double b) {
  double s = a + b;
  double bb = s - a;
  double e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
inline dd quick_two_sum(double a, double b) {
  double s = a + b;
  return {s, b - (s - a)};
}
inline dd two_prod(double a, double b) {
  double p = a * b;
  return {p, std::fma(a, b, -p)};
}
inline dd dd_add(dd x, dd y) {
  dd s = two_sum(x.hi, y.hi);
  return two_sum(s.hi, s.lo + (x.lo + y.lo));
}
inline dd dd_mul(dd x, dd y) {
  dd p = two_prod(x.hi, y.hi);
  return quick_two_sum(p.hi, p.lo + (x.hi * y.lo + x.lo * y.hi));
}
inline dd dd_mul_d(dd x, double b) {
  dd p = two_prod(x.hi, b);
  return quick_two_sum(p.hi, p.lo + x.lo * b);
}
inline dd dd_div_d(dd x, double b) {
  double q1 = x.hi / b;
  dd p = two_prod(q1, b);
  double r = ((x.hi - p.hi) - p.lo + x.lo) / b;
  return quick_two_sum(q1, r);
}

// P_n(t) and P_{n-1}(t) by (j+1) P_{j+1} = (2j+1) t P_j - j P_{j-1}.
inline void legendre_pair(int n, double t, double* pn, double* pm) {
  double p0 = 1.0, p1 = t;
  for (int j = 1; j < n; ++j) {
    double p2 = ((2 * j + 1) * t * p1 - j * p0) / (j + 1);
    p0 = p1;
    p1 = p2;
  }
  *pn = (n > 1) ? p1 : t;
  *pm = (n > 1) ? p0 : 1.0;
}

}  // namespace

int rmat_mesh_host(int nlag, double a, double* x_out, double* omx_out, double* lam_out,
                   double* r_out, double* fa_out, double* T0_out) {
  if (nlag < 1 || nlag > 1024) return -1;
  if (!(a > 0.0) || !std::isfinite(a)) return -2;
  const int n = nlag;
  const double pi = 3.14159265358979323846;
  std::vector<double> x(n), omx(n), w(n);
  for (int k = 1; k <= n; ++k) {
    // Newton on theta with t = cos(theta) (node index k from the right end).
    double theta = pi * (k - 0.25) / (n + 0.5);
    for (int it = 0; it < 100; ++it) {
      double t = std::cos(theta), pn, pm;
      legendre_pair(n, t, &pn, &pm);
      double dp = n * (t * pn - pm) / (t * t - 1.0);
      double step = pn / (-std::sin(theta) * dp);
      theta -= step;
      if (std::fabs(step) < 1e-16) break;
    }
    // Newton polish of t in double-double.
    dd t = {std::cos(theta), 0.0};
    for (int it = 0; it < 3; ++it) {
      dd p0 = {1.0, 0.0}, p1 = t;
      for (int j = 1; j < n; ++j) {
        dd s = dd_mul_d(dd_mul(t, p1), (double)(2 * j + 1));
        dd q = dd_mul_d(p0, (double)j);
        dd c = dd_div_d(dd_add(s, {-q.hi, -q.lo}), (double)(j + 1));
        p0 = p1;
        p1 = c;
      }
      dd pn = (n > 1) ? p1 : t;
      double pmh = (n > 1) ? p0.hi : 1.0;
      double dp = n * (t.hi * pn.hi - pmh) / (t.hi * t.hi - 1.0);
      dd st = dd_div_d(pn, dp);
      t = dd_add(t, {-st.hi, -st.lo});
    }
    dd s = two_sum(1.0, t.hi);
    double xh = quick_two_sum(s.hi, s.lo + t.lo).hi;
    dd s2 = two_sum(1.0, -t.hi);
    double oh = quick_two_sum(s2.hi, s2.lo - t.lo).hi;
    const int idx = n - k;  // ascending x
    x[idx] = xh / 2.0;
    omx[idx] = oh / 2.0;
    double pn, pm;
    legendre_pair(n, t.hi, &pn, &pm);
    double dp = n * (pm - t.hi * pn) / (4.0 * x[idx] * omx[idx]);
    w[idx] = 2.0 / (4.0 * x[idx] * omx[idx] * dp * dp) / 2.0;
  }
  for (int i = 0; i < n; ++i) {
    if (x_out) x_out[i] = x[i];
    if (omx_out) omx_out[i] = omx[i];
    if (lam_out) lam_out[i] = w[i];
    if (r_out) r_out[i] = a * x[i];
    if (fa_out) {
      // (-1)^(n + i + 1) for 0-based i, i.e. (-1)^(n+i) with the paper's 1-based i
      double sgn = ((n + i + 1) % 2 == 0) ? 1.0 : -1.0;
      fa_out[i] = sgn / std::sqrt(a * x[i] * omx[i]);
    }
  }
  if (T0_out) {
    // T0 = int_0^a f_i' f_j' dr (kinetic energy + Bloch L(0), fm^-2), Baye's
    // closed forms for the regularised shifted-Legendre mesh; upper triangle
    // evaluated and mirrored.
    const double c_diag = (double)(4 * n * n + 4 * n + 3);
    const double c_off = (double)(n * n + n) + 1.0;
    for (int i = 0; i < n; ++i) {
      const double xi = x[i], oi = omx[i];
      double num = c_diag * xi * oi - 6.0 * xi + 1.0;
      double den = 3.0 * a * a * (xi * xi) * (oi * oi);
      T0_out[(size_t)i * n + i] = num / den;
      for (int j = i + 1; j < n; ++j) {
        const double xj = x[j], oj = omx[j];
        double sgn = ((i + j) % 2 == 0) ? 1.0 : -1.0;
        double d = xi - xj;
        double pre = sgn / (a * a * std::sqrt(xi * xj * oi * oj));
        double brk = c_off + (xi + xj - 2.0 * xi * xj) / (d * d) - 1.0 / oi - 1.0 / oj;
        double v = pre * brk;
        T0_out[(size_t)i * n + j] = v;
        T0_out[(size_t)j * n + i] = v;
      }
    }
  }
  return RMAT_OK;
}

// Mesh of a propagation sector (r1, r2): the Lagrange-Legendre basis without
// regularisation, f_i(r) = l_i(x) / sqrt(h w_i), x = (r - r1)/h, l_i the Lagrange
// polynomial through the Gauss-Legendre nodes of (0, 1), so f_i(r_j) =
// delta_ij / sqrt(h w_j) and f_i is non-zero at both ends.  Tables:
//   r_i = r1 + h x_i, lam_i = h w_i, fL_i = f_i(r1), fR_i = f_i(r2),
//   Kf_ij = int_{r1}^{r2} f_i' f_j' dr = sum_k w_k D_ki D_kj / (h^2 sqrt(w_i w_j)),
// D_ki = l_i'(x_k) (the integrand has degree 2n - 4 < 2n: the rule is exact).
// Barycentric weights of Gauss-Legendre nodes in closed form, beta_i ~
// (-1)^i sqrt(x_i (1 - x_i) w_i); D_ki = (beta_i / beta_k) / (x_k - x_i) for
// k != i and D_kk = -sum_{i != k} D_ki (the derivative of a constant vanishes).
int rmat_sector_mesh_host(int nlag, double r1, double r2, double* r, double* lam, double* fL,
                          double* fR, double* Kf) {
  if (nlag < 2 || nlag > 1024) return -1;
  if (!(r2 > r1) || !std::isfinite(r1) || !std::isfinite(r2) || r1 < 0.0) return -2;
  const int n = nlag;
  const double h = r2 - r1;
  std::vector<double> x(n), omx(n), w(n), rr(n), fa(n);
  RMAT_CHECK(rmat_mesh_host(n, 1.0, x.data(), omx.data(), w.data(), rr.data(), fa.data(), nullptr));
  std::vector<double> beta(n), D((size_t)n * n);
  for (int i = 0; i < n; ++i) beta[i] = ((i & 1) ? -1.0 : 1.0) * std::sqrt(x[i] * omx[i] * w[i]);
  for (int k = 0; k < n; ++k) {
    double diag = 0.0;
    for (int i = 0; i < n; ++i) {
      if (i == k) continue;
      const double d = (beta[i] / beta[k]) / (x[k] - x[i]);
      D[(size_t)k * n + i] = d;
      diag -= d;
    }
    D[(size_t)k * n + k] = diag;
  }
  // l_i(t) = (beta_i / (t - x_i)) / sum_m beta_m / (t - x_m) at t = 0 (t - x_m = -x_m)
  // and t = 1 (t - x_m = 1 - x_m, correctly rounded in omx)
  double s0 = 0.0, s1 = 0.0;
  for (int m = 0; m < n; ++m) {
    s0 += beta[m] / (-x[m]);
    s1 += beta[m] / omx[m];
  }
  for (int i = 0; i < n; ++i) {
    const double sc = 1.0 / std::sqrt(h * w[i]);
    if (r) r[i] = r1 + h * x[i];
    if (lam) lam[i] = h * w[i];
    if (fL) fL[i] = (beta[i] / (-x[i])) / s0 * sc;
    if (fR) fR[i] = (beta[i] / omx[i]) / s1 * sc;
  }
  if (Kf)
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        double acc = 0.0;
        for (int k = 0; k < n; ++k) acc += w[k] * D[(size_t)k * n + i] * D[(size_t)k * n + j];
        Kf[(size_t)i * n + j] = acc / (h * h * std::sqrt(w[i] * w[j]));
      }
  return RMAT_OK;
}

void rmat_kinetic_table(int nlag, double hm, double s1, const double* T0, const double* fa,
                        double* K) {
  for (int i = 0; i < nlag; ++i)
    for (int j = 0; j < nlag; ++j)
      K[(size_t)i * nlag + j] = hm * T0[(size_t)i * nlag + j] - s1 * (fa[i] * fa[j]);
}
