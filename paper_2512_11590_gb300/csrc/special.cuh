// Asymptotic channel functions for neutral channels (eta = 0), FP64 device code
// shared by the collision kernels.
#pragma once
#include <cuda_runtime.h>

// F_l, G_l and derivatives (eta = 0).  G by upward recurrence from
// G_0 = cos, G_1 = cos/rho + sin; F by upward recurrence for rho >= l+1, else by
// the power series rho^(l+1) sum_k (-rho^2/2)^k / (k! (2l+2k+1)!!).
// X_l' = X_{l-1} - (l/rho) X_l.
__device__ inline void riccati_fg(int l, double rho, double* F, double* G, double* dF, double* dG) {
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
__device__ inline void whittaker_w(int l, double rho, double* W, double* dW) {
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

