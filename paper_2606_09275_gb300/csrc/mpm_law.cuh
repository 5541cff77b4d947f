// Hencky / return-map law shared by the assembly and the adjoint kernels
// (Sec. 2.2; model 3, the CPT material's Willam-Warnke cone, Sec. 6.4):
// principal-space return in Kirchhoff stress, 3x3 symmetric
// eigen-decomposition, divided difference of the logarithm.
#pragma once
#include "mpm_internal.cuh"

namespace mpm {

struct Law {
  int model;
  double nu, eta, xi, etab;
  double ecc;  // model 3: tensile / compressive meridian radius, (3 - sin phi)/(3 + sin phi)
};

// Willam-Warnke deviatoric section (Sec. 6.4): r(theta) by the elliptic
// interpolation r = (4 a c^2 + b^2)/(2 a c + b sqrt(4 a c^2 + 5 e^2 - 4 e)),
// c = cos(theta), a = 1 - e^2, b = 2 e - 1 (theta the Lode angle, 0 on the
// tensile meridian where r = 1/e, pi/3 on the compressive one where r = 1),
// and dr/dzeta for zeta = cos(3 theta); at the compressive meridian the limit
// 4 a / (6 b^2 (2 c + 1)) of dr/dc over dzeta/dc is taken
__device__ inline double ww_section(double zeta, double e, double* drdz) {
  zeta = fmin(fmax(zeta, -1.0), 1.0);
  double c = cos(acos(zeta) / 3.0);
  double a = 1.0 - e * e, b = 2.0 * e - 1.0;
  double w = sqrt(4.0 * a * c * c + 5.0 * e * e - 4.0 * e);
  double N = 4.0 * a * c * c + b * b, D = 2.0 * a * c + b * w;
  double dN = 8.0 * a * c, dD = 2.0 * a + 4.0 * a * b * c / w;
  double rc = (dN * D - N * dD) / (D * D);
  double q = 4.0 * c * c - 1.0;
  *drdz = fabs(q) > 1e-5 ? rc / (3.0 * q) : 4.0 * a / (6.0 * b * b * (2.0 * c + 1.0));
  return N / D;
}

// symmetric 3x3 eigen-decomposition by cyclic Jacobi rotations; columns of Q
// are the eigenvectors (Q[3*i + a] = component i of vector a)
__device__ inline void jacobi3(double* A, double* lam, double* Q) {
#pragma unroll
  for (int i = 0; i < 9; ++i) Q[i] = (i == 0 || i == 4 || i == 8) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    double on = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off == 0.0 || off <= 1e-36 * on) break;
#pragma unroll
    for (int r = 0; r < 3; ++r) {
      const int p = (r == 2) ? 1 : 0, q = (r == 0) ? 1 : 2;
      double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      double h = A[3 * q + q] - A[3 * p + p];
      // tan of the rotation angle, smaller root of t^2 + (h/apq) t - 1 = 0
      double th = 0.5 * h / apq;
      double t = fabs(th) > 1e150 ? 0.5 / th : copysign(1.0, th) / (fabs(th) + sqrt(th * th + 1.0));
      double cs = rsqrt(t * t + 1.0);
      double sn = t * cs;
      // rows/columns p and q of A, and columns of Q
      double app = A[3 * p + p], aqq = A[3 * q + q];
      A[3 * p + p] = app - t * apq;
      A[3 * q + q] = aqq + t * apq;
      A[3 * p + q] = A[3 * q + p] = 0.0;
      const int o = 3 - p - q;
      double aop = A[3 * o + p], aoq = A[3 * o + q];
      A[3 * o + p] = A[3 * p + o] = cs * aop - sn * aoq;
      A[3 * o + q] = A[3 * q + o] = sn * aop + cs * aoq;
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        double qp = Q[3 * k + p], qq = Q[3 * k + q];
        Q[3 * k + p] = cs * qp - sn * qq;
        Q[3 * k + q] = sn * qp + cs * qq;
      }
    }
  }
  lam[0] = A[0];
  lam[1] = A[4];
  lam[2] = A[8];
}

// divided difference of the logarithm: (ln a - ln b)/(a - b), 1/b in the limit
__device__ inline double ln_divdiff(double a, double b) {
  double x = (a - b) / b;
  if (fabs(x) < 1e-6) return (1.0 + x * (-0.5 + x * (1.0 / 3.0 - 0.25 * x))) / b;
  return log1p(x) / (a - b);
}

// principal-space return: trial strains e -> tau_a, tangent d_ab = dtau_a/deps_b,
// shear ratio g = (tau_a - tau_b)/(eps_a - eps_b); Hencky moduli from E, nu
__device__ inline void principal_return(const Law& L, double E, double ys, const double* e, double* ta,
                                 double* dd, double* gr) {
  double mu = E / (2.0 * (1.0 + L.nu));
  double lm = E * L.nu / ((1.0 + L.nu) * (1.0 - 2.0 * L.nu));
  double kb = lm + 2.0 * mu / 3.0;
  double tr = e[0] + e[1] + e[2];
  double dev[3] = {e[0] - tr / 3.0, e[1] - tr / 3.0, e[2] - tr / 3.0};
  double dn = sqrt(dev[0] * dev[0] + dev[1] * dev[1] + dev[2] * dev[2]);
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    ta[a] = kb * tr + 2.0 * mu * dev[a];
#pragma unroll
    for (int b = 0; b < 3; ++b) dd[3 * a + b] = lm + (a == b ? 2.0 * mu : 0.0);
  }
  *gr = 2.0 * mu;
  if (L.model == 1) {
    // von Mises: q = sqrt(3/2)|s|, radial return onto q = ys
    double q = 1.224744871391589 * 2.0 * mu * dn;
    if (q <= ys) return;
    double fac = ys / q, g = 2.0 * mu * fac;
    double n0 = dev[0] / dn, n1 = dev[1] / dn, n2 = dev[2] / dn;
    double nn[3] = {n0, n1, n2};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      ta[a] = kb * tr + g * dev[a];
#pragma unroll
      for (int b = 0; b < 3; ++b) dd[3 * a + b] = kb + g * ((a == b ? 1.0 : 0.0) - 1.0 / 3.0 - nn[a] * nn[b]);
    }
    *gr = g;
  } else if (L.model == 2 || L.model == 3) {
    // Drucker-Prager cone: f = sqrt(J2) r + eta p - xi c with r = 1 (model 2)
    // or the Willam-Warnke section r(theta) (model 3); potential sqrt(J2) +
    // etab p, circular, so the return is radial in the deviatoric plane and
    // keeps theta: f(dg) = (sqrt(J2) - G dg) r + eta (p - K etab dg) - xi c
    double G = mu, pm = kb * tr;
    double sj = 1.4142135623730951 * G * dn;
    double r = 1.0, drz = 0.0, dz[3] = {0.0, 0.0, 0.0};
    if (L.model == 3 && dn > 0.0) {
      // zeta = cos(3 theta) = 3 sqrt6 e1 e2 e3 / |e|^3 of the trial deviator
      double pr = dev[0] * dev[1] * dev[2], dn3 = dn * dn * dn;
      double zeta = 7.348469228349534 * pr / dn3;
      r = ww_section(zeta, L.ecc, &drz);
      if (zeta > -1.0 && zeta < 1.0) {
        double mm[3] = {dev[1] * dev[2], dev[0] * dev[2], dev[0] * dev[1]};
        double M3 = (mm[0] + mm[1] + mm[2]) / 3.0;
#pragma unroll
        for (int b = 0; b < 3; ++b)
          dz[b] = 7.348469228349534 * ((mm[b] - M3) / dn3 - 3.0 * pr * dev[b] / (dn3 * dn * dn));
      }
    }
    double f = sj * r + L.eta * pm - L.xi * ys;
    if (f <= 0.0) return;
    double den = G * r + kb * L.eta * L.etab;
    double dg = f / den;
    if (sj - G * dg >= 0.0 && dn > 0.0) {
      double ratio = 1.0 - G * dg / sj;
      double pn = pm - kb * L.etab * dg;
      double nn[3] = {dev[0] / dn, dev[1] / dn, dev[2] / dn};
      double ddg[3];
#pragma unroll
      for (int b = 0; b < 3; ++b)
        ddg[b] = (1.4142135623730951 * G * nn[b] * r + (sj - G * dg) * drz * dz[b] + L.eta * kb) / den;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ta[a] = pn + 2.0 * G * ratio * dev[a];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
          double pd = (a == b ? 1.0 : 0.0) - 1.0 / 3.0;
          dd[3 * a + b] = 2.0 * G * pd -
                          1.4142135623730951 * G * (nn[a] * ddg[b] + dg * (pd - nn[a] * nn[b]) / dn) +
                          kb * (1.0 - L.etab * ddg[b]);
        }
      }
      *gr = 2.0 * G * ratio;
    } else {
      double pa = L.xi * ys / L.eta;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        ta[a] = pa;
#pragma unroll
        for (int b = 0; b < 3; ++b) dd[3 * a + b] = 0.0;
      }
      *gr = 0.0;
    }
  }
}

inline Law make_law(const mpm_material& mat) {
  Law L{};
  L.model = mat.model;
  L.nu = mat.nu;
  double sp = sin(mat.phi), ss = sin(mat.psi);
  L.eta = 6.0 * sp / (sqrt(3.0) * (3.0 - sp));
  L.xi = 6.0 * cos(mat.phi) / (sqrt(3.0) * (3.0 - sp));
  L.etab = 6.0 * ss / (sqrt(3.0) * (3.0 - ss));
  L.ecc = (3.0 - sp) / (3.0 + sp);
  return L;
}

}  // namespace mpm
