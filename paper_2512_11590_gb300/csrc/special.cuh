// Asymptotic channel functions (neutral and charged channels), FP64 device code
// shared by the collision kernels.
#pragma once
#include <cuda_runtime.h>

#include <cmath>

// F_l, G_l and derivatives (eta = 0).  G by upward recurrence from
// G_0 = cos, G_1 = cos/rho + sin; F by upward recurrence for rho >= l+1, else by
// the power series rho^(l+1) sum_k (-rho^2/2)^k / (k! (2l+2k+1)!!).
// X_l' = X_{l-1} - (l/rho) X_l.
__host__ __device__ inline void riccati_fg(int l, double rho, double* F, double* G, double* dF, double* dG) {
  const double s = sin(rho), c = cos(rho);
  if (l == 0) {
    *F = s; *G = c; *dF = c; *dG = -s;
    return;
  }
  double g0 = c, g1 = c / rho + s;
  for (int q = 1; q < l; ++q) {
    const double g2 = (2 * q + 1) / rho * g1 - g0;
    g0 = g1;
    g1 = g2;
  }
  double f0, f1;
  if (rho >= l + 1) {
    f0 = s;
    f1 = s / rho - c;
    for (int q = 1; q < l; ++q) {
      const double f2 = (2 * q + 1) / rho * f1 - f0;
      f0 = f1;
      f1 = f2;
    }
  } else {
    double fl[2];
    for (int L = l - 1; L <= l; ++L) {
      double df = 1.0;
      for (int q = 1; q <= 2 * L + 1; q += 2) df *= q;
      double term = pow(rho, L + 1) / df, acc = term;
      for (int k = 1; k < 200; ++k) {
        term *= -(rho * rho / 2.0) / (k * (2.0 * L + 2 * k + 1));
        acc += term;
        if (fabs(term) < 1e-18 * fabs(acc)) break;
      }
      fl[L - (l - 1)] = acc;
    }
    f0 = fl[0];
    f1 = fl[1];
  }
  *F = f1;
  *G = g1;
  *dF = f0 - l / rho * f1;
  *dG = g0 - l / rho * g1;
}

// e^-rho sum_{k=0}^{l} (l+k)!/(k!(l-k)!) (2 rho)^-k and its rho-derivative
__host__ __device__ inline void whittaker_w(int l, double rho, double* W, double* dW) {
  double w = 0.0, dw = 0.0, ck = 1.0;  // ck = (l+k)!/(k!(l-k)!) for k = 0
  for (int k = 0; k <= l; ++k) {
    if (k > 0) ck = ck * (double)(l + k) * (double)(l - k + 1) / (double)k;
    const double t = ck * pow(2.0 * rho, -k);
    w += t;
    dw += t * (-1.0 - k / rho);
  }
  const double e = exp(-rho);
  *W = e * w;
  *dW = e * dw;
}


// ---- charged channels (eta != 0) ------------------------------------------
//
// Coulomb functions F_l(eta, rho), G_l(eta, rho) (Sec. 4.1: Barnett's COULFG,
// i.e. Steed's method), per thread.  With S_L = L/rho + eta/L and
// R_L^2 = 1 + eta^2/L^2:
//   CF1  f = F'/F = S_{l+1} - R_{l+1}^2/(T_{l+1} - R_{l+2}^2/(T_{l+2} - ...)),
//        T_L = S_L + S_{L+1}, evaluated forward by the modified Lentz method;
//        the convergent denominators B_n solve the ladder recurrence of F in L
//        with B = 0 at L = l, so for large n B_n has the sign of F_l G_{l+n},
//        i.e. of F_l, and sign(F_l) = sign(B_n) = sign of the product of the
//        Lentz factors D_j = B_{j-1}/B_j;
//   CF2  p + iq = (G' + iF')/(G + iF) = i(1 - eta/rho) + (i/rho) K,
//        K = a_1/(b_1 + a_2/(b_2 + ...)), a_k = (l + k + i eta)(k - 1 - l + i eta),
//        b_k = 2(rho - eta) + 2k i, also by modified Lentz;
//   gamma = (f - p)/q, F = sign/sqrt(q (1 + gamma^2)), F' = f F, G = gamma F,
//   G' = (p gamma - q) F   (the Wronskian F'G - FG' = 1).
// CF2 loses accuracy inside the turning point rho_tp = eta + sqrt(eta^2 + l(l+1))
// (q becomes exponentially small next to p).  There G, G' come from Steed's
// method at rho_tp and are carried inward with Taylor-series steps of the
// Coulomb equation (G grows inward: stable), and F = 1/(f G - G') with CF1 at rho.
// Closed channels take the log-derivative of W_{-eta,l+1/2}(2 rho): the
// decaying solution is H+ continued to imaginary argument, where CF2 becomes
// the real fraction
//   W'/W = -(1 + eta/rho) + (1/rho) a_1/(beta_1 - a_2/(beta_2 - ...)),
//   a_k = (eta + l + k)(eta - l + k - 1),  beta_k = 2(rho + eta + k),
// valid for eta >= 0.  Only W'/W enters U (a closed channel's column of the
// matching matrix scales with W), so closed channels carry O = 1, O' = W'/W.
// Every loop is bounded; a function that does not converge returns false.

constexpr int kCoulIterMax = 200000;
constexpr double kCoulTiny = 1e-300;
constexpr double kCoulEps = 3e-16;  // accept a Lentz factor within one ulp of 1

__host__ __device__ inline bool coulomb_cf1(int l, double eta, double rho, double* f, int* sign) {
  double L = l + 1.0;
  double fv = L / rho + eta / L;
  if (fv == 0.0) fv = kCoulTiny;
  double C = fv, D = 0.0;
  int s = 1;
  double SL = fv;  // S_L at L = l + j
  for (int j = 1; j < kCoulIterMax; ++j) {
    L = l + j;
    const double SL1 = (L + 1.0) / rho + eta / (L + 1.0);
    const double a = -(1.0 + (eta / L) * (eta / L));
    const double b = SL + SL1;
    SL = SL1;
    D = b + a * D;
    if (D == 0.0) D = kCoulTiny;
    C = b + a / C;
    if (C == 0.0) C = kCoulTiny;
    D = 1.0 / D;
    if (D < 0.0) s = -s;
    const double delta = C * D;
    fv *= delta;
    if (fabs(delta - 1.0) < kCoulEps) {
      *f = fv;
      *sign = s;
      return true;
    }
  }
  return false;
}

__host__ __device__ inline bool coulomb_cf2(int l, double eta, double rho, double* p, double* q) {
  // complex Lentz: |C|^2 must stay representable, so the start value is 1e-150
  constexpr double tiny = 1e-150;
  double2 fv = make_double2(tiny, 0.0), C = fv, D = make_double2(0.0, 0.0);
  const double br = 2.0 * (rho - eta);
  for (int k = 1; k < kCoulIterMax; ++k) {
    const double ar = (double)(l + k) * (double)(k - 1 - l) - eta * eta;
    const double ai = eta * (2.0 * k - 1.0);
    const double bi = 2.0 * k;
    // D = 1 / (b + a D)
    double dr = br + ar * D.x - ai * D.y, di = bi + ar * D.y + ai * D.x;
    if (dr == 0.0 && di == 0.0) dr = tiny;
    double m = 1.0 / (dr * dr + di * di);
    D = make_double2(dr * m, -di * m);
    // C = b + a / C
    m = 1.0 / (C.x * C.x + C.y * C.y);
    const double icr = C.x * m, ici = -C.y * m;
    C = make_double2(br + ar * icr - ai * ici, bi + ar * ici + ai * icr);
    if (C.x == 0.0 && C.y == 0.0) C.x = tiny;
    const double2 delta = make_double2(C.x * D.x - C.y * D.y, C.x * D.y + C.y * D.x);
    fv = make_double2(fv.x * delta.x - fv.y * delta.y, fv.x * delta.y + fv.y * delta.x);
    if (fabs(delta.x - 1.0) + fabs(delta.y) < kCoulEps) {
      *p = -fv.y / rho;
      *q = (1.0 - eta / rho) + fv.x / rho;
      return true;
    }
  }
  return false;
}

// One Taylor step of u'' = (l(l+1)/x^2 + 2 eta/x - 1) u from x0 to x0 + h.
// With x = x0 + t and u = sum c_n t^n, multiplying the equation by x^2 gives
//   x0^2 (m+2)(m+1) c_{m+2} = (A - m(m-1)) c_m + B c_{m-1} - c_{m-2}
//                             - 2 x0 (m+1) m c_{m+1},
//   A = l(l+1) + 2 eta x0 - x0^2,  B = 2 eta - 2 x0.
__host__ __device__ inline bool coulomb_taylor_step(int l, double eta, double x0, double h, double* u,
                                           double* du) {
  const double A = (double)l * (l + 1.0) + 2.0 * eta * x0 - x0 * x0;
  const double B = 2.0 * eta - 2.0 * x0;
  const double x02 = x0 * x0;
  double cm2 = 0.0, cm1 = 0.0, cm = *u, cp1 = *du;  // c_{m-2}, c_{m-1}, c_m, c_{m+1}
  double s = cm + cp1 * h, ds = cp1, hp = h;         // hp = h^(m+1)
  int small = 0;
  for (int m = 0; m < 400; ++m) {
    const double cp2 = ((A - (double)m * (m - 1.0)) * cm + B * cm1 - cm2 -
                        2.0 * x0 * (m + 1.0) * m * cp1) /
                       (x02 * (m + 2.0) * (m + 1.0));
    ds += (m + 2.0) * cp2 * hp;
    hp *= h;
    const double t = cp2 * hp;
    s += t;
    cm2 = cm1;
    cm1 = cm;
    cm = cp1;
    cp1 = cp2;
    small = fabs(t) < 1e-17 * fabs(s) ? small + 1 : 0;
    if (m > 4 && small >= 2) {
      *u = s;
      *du = ds;
      return true;
    }
  }
  return false;
}

__host__ __device__ inline bool coulomb_steed(int l, double eta, double rho, double* F, double* G,
                                     double* dF, double* dG) {
  double f, p, q;
  int sgn;
  if (!coulomb_cf1(l, eta, rho, &f, &sgn) || !coulomb_cf2(l, eta, rho, &p, &q)) return false;
  if (!(q > 0.0)) return false;
  const double gam = (f - p) / q;
  const double Fv = sgn / sqrt(q * (1.0 + gam * gam));
  *F = Fv;
  *dF = f * Fv;
  *G = gam * Fv;
  *dG = (p * gam - q) * Fv;
  return true;
}

__host__ __device__ inline bool coulomb_fg(int l, double eta, double rho, double* F, double* G, double* dF,
                                  double* dG) {
  if (!(rho > 0.0)) return false;
  const double ll = (double)l * (l + 1.0);
  const double tp = eta + sqrt(eta * eta + ll);
  if (rho >= tp) return coulomb_steed(l, eta, rho, F, G, dF, dG);
  double Ft, Gt, dFt, dGt;
  if (!coulomb_steed(l, eta, tp, &Ft, &Gt, &dFt, &dGt)) return false;
  double x = tp, u = Gt, du = dGt;
  for (int it = 0; x > rho; ++it) {
    if (it >= 100000) return false;
    const double kl = sqrt(fabs(ll / (x * x) + 2.0 * eta / x - 1.0)) + 1e-300;
    double h = fmin(fmin(1.0, 0.4 * x), 4.0 / kl);
    const bool last = x - h <= rho;
    if (last) h = x - rho;
    if (!coulomb_taylor_step(l, eta, x, -h, &u, &du)) return false;
    x = last ? rho : x - h;
  }
  double f;
  int sgn;
  if (!coulomb_cf1(l, eta, rho, &f, &sgn)) return false;
  const double Fv = 1.0 / (f * u - du);
  *F = Fv;
  *dF = f * Fv;
  *G = u;
  *dG = du;
  return isfinite(Fv) && isfinite(u) && isfinite(du);
}

// W'/W (rho-derivative) of W_{-eta,l+1/2}(2 rho), eta >= 0.
__host__ __device__ inline bool whittaker_logd(int l, double eta, double rho, double* L) {
  double fv = kCoulTiny, C = fv, D = 0.0;
  for (int k = 1; k < kCoulIterMax; ++k) {
    const double ak = (eta + l + k) * (eta - l + k - 1.0);
    const double a = k == 1 ? ak : -ak;
    const double b = 2.0 * (rho + eta + k);
    D = b + a * D;
    if (D == 0.0) D = kCoulTiny;
    C = b + a / C;
    if (C == 0.0) C = kCoulTiny;
    D = 1.0 / D;
    const double delta = C * D;
    fv *= delta;
    if (fabs(delta - 1.0) < kCoulEps) {
      *L = -(1.0 + eta / rho) + fv / rho;
      return true;
    }
  }
  return false;
}

// Channel functions at rho = k a for one channel (Bloch-shifted derivatives):
// open (ecm > 0): I = G - iF, O = G + iF; closed: O = W (eta = 0: the reduced
// Whittaker function) or O = 1, O' = W'/W (eta > 0), I = 0.
// eta = zz / (2 hm k), zz = Z1 Z2 e^2 (0 for a neutral channel).
__host__ __device__ inline bool channel_functions(int l, double ecm, double hm, double a, double B,
                                         double zz, double2* I, double2* O, double2* dI,
                                         double2* dO, double* kout) {
  const double k = sqrt(fabs(ecm) / hm), rho = k * a;
  *kout = k;
  bool ok = true;
  if (ecm > 0) {
    double F = 0, G = 1, dF = 0, dG = 0;
    if (zz == 0.0) riccati_fg(l, rho, &F, &G, &dF, &dG);
    else ok = coulomb_fg(l, zz / (2.0 * hm * k), rho, &F, &G, &dF, &dG);
    *I = make_double2(G, -F);
    *O = make_double2(G, F);
    *dI = make_double2(dG, -dF);
    *dO = make_double2(dG, dF);
  } else {
    double W = 1, dW = 0;
    if (zz == 0.0) {
      whittaker_w(l, rho, &W, &dW);
    } else {
      W = 1.0;
      ok = whittaker_logd(l, zz / (2.0 * hm * k), rho, &dW);
    }
    *I = make_double2(0, 0);
    *dI = make_double2(0, 0);
    *O = make_double2(W, 0);
    *dO = make_double2(dW, 0);
  }
  dI->x -= B / rho * I->x;
  dI->y -= B / rho * I->y;
  dO->x -= B / rho * O->x;
  dO->y -= B / rho * O->y;
  ok = ok && isfinite(I->x) && isfinite(I->y) && isfinite(O->x) && isfinite(O->y) &&
       isfinite(dI->x) && isfinite(dI->y) && isfinite(dO->x) && isfinite(dO->y);
  if (!ok) {  // finite stand-ins keep the matching solve defined; the caller reports the failure
    *I = make_double2(0, 0);
    *O = make_double2(1, 0);
    *dI = make_double2(0, 0);
    *dO = make_double2(0, 0);
  }
  return ok;
}
