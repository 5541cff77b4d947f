/*
 * Oracle: Hencky hyperelasticity with perfect-plasticity return maps in
 * principal Kirchhoff space (Sec. 2.2) and the consistent spatial tangent.
 * TEST INFRASTRUCTURE ONLY.
 *
 * Readings (the paper defers the formulas to de Souza Neto and to AMPLE):
 *  - trial elastic strain eps = 1/2 ln(eig b_e^tr), b_e^tr = dF b_e,n dF^T;
 *  - tau_a = lambda tr(eps) + 2 mu eps_a (Hencky), sigma = tau / det F;
 *  - von Mises: f = sqrt(3 J2) - sigma_y, radial return;
 *  - Drucker-Prager: f = sqrt(J2) + eta p - xi c, p = tr(tau)/3 (tension +),
 *    outer-cone match eta = 6 sin(phi)/(sqrt3 (3 - sin phi)),
 *    xi = 6 cos(phi)/(sqrt3 (3 - sin phi)); potential uses psi; cone return,
 *    apex return when the cone return overshoots the apex;
 *  - model 3: the same cone with the Willam-Warnke deviatoric section
 *    (Sec. 6.4) and the circular Drucker-Prager potential;
 *  - tangent: A_ijkm = 2 (d tau_ij / d b_kl) b_lm, built in the eigenbasis of
 *    b^tr from the principal algorithmic tangent d_ab = d tau_a / d eps_b and
 *    the shear ratio g = (tau_a - tau_b)/(eps_a - eps_b); the divided difference
 *    of ln uses log1p with a series for nearly equal eigenvalues.
 */
#include "o_internal.h"
#include <math.h>
#include <string.h>

void o_mat33_mul(const double* a, const double* b, double* c) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += a[3 * i + k] * b[3 * k + j];
      c[3 * i + j] = s;
    }
}

double o_det33(const double* a) {
  return a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) +
         a[2] * (a[3] * a[7] - a[4] * a[6]);
}

void o_inv33(const double* a, double* ai) {
  double det = o_det33(a);
  ai[0] = (a[4] * a[8] - a[5] * a[7]) / det;
  ai[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  ai[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  ai[3] = (a[5] * a[6] - a[3] * a[8]) / det;
  ai[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  ai[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  ai[6] = (a[3] * a[7] - a[4] * a[6]) / det;
  ai[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  ai[8] = (a[0] * a[4] - a[1] * a[3]) / det;
}

/* cyclic Jacobi rotations on a symmetric 3x3 matrix; Q holds the eigenvectors
 * as columns (Q[3*i + a] = component i of eigenvector a) */
void o_eig_sym3(const double* a, double* lam, double* Q) {
  double A[9];
  memcpy(A, a, sizeof(A));
  A[1] = A[3] = 0.5 * (a[1] + a[3]);
  A[2] = A[6] = 0.5 * (a[2] + a[6]);
  A[5] = A[7] = 0.5 * (a[5] + a[7]);
  for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.0 : 0.0;
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = A[1] * A[1] + A[2] * A[2] + A[5] * A[5];
    double dia = A[0] * A[0] + A[4] * A[4] + A[8] * A[8];
    if (off <= 1e-36 * dia || off == 0.0) break;
    for (int pq = 0; pq < 3; ++pq) {
      int p = pq == 2 ? 1 : 0, q = pq == 0 ? 1 : 2;
      double apq = A[3 * p + q];
      if (apq == 0.0) continue;
      double theta = (A[3 * q + q] - A[3 * p + p]) / (2.0 * apq);
      double t;
      if (fabs(theta) > 1e150)
        t = 0.5 / theta;
      else
        t = (theta >= 0 ? 1.0 : -1.0) / (fabs(theta) + sqrt(theta * theta + 1.0));
      double c = 1.0 / sqrt(t * t + 1.0), s = t * c;
      /* A <- J^T A J with J the rotation in the (p,q) plane */
      for (int k = 0; k < 3; ++k) {
        double akp = A[3 * k + p], akq = A[3 * k + q];
        A[3 * k + p] = c * akp - s * akq;
        A[3 * k + q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {
        double apk = A[3 * p + k], aqk = A[3 * q + k];
        A[3 * p + k] = c * apk - s * aqk;
        A[3 * q + k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        double qkp = Q[3 * k + p], qkq = Q[3 * k + q];
        Q[3 * k + p] = c * qkp - s * qkq;
        Q[3 * k + q] = s * qkp + c * qkq;
      }
    }
  }
  lam[0] = A[0];
  lam[1] = A[4];
  lam[2] = A[8];
}

/* (ln a - ln b)/(a - b), and 1/b in the limit */
static double dlog(double a, double b) {
  double x = (a - b) / b;
  if (fabs(x) < 1e-6) return (1.0 - x / 2.0 + x * x / 3.0 - x * x * x / 4.0) / b;
  return log1p(x) / (a - b);
}

/* Willam-Warnke deviatoric section (Sec. 6.4, frictional cone of the CPT
 * material): with c = cos(theta), theta the Lode angle (0 on the tensile
 * meridian, pi/3 on the compressive one) and eccentricity e, the elliptic
 * interpolation
 *   r(c) = (4 a c^2 + b^2) / (2 a c + b sqrt(4 a c^2 + 5 e^2 - 4 e)),
 * a = 1 - e^2, b = 2 e - 1, gives r = 1 on the compressive meridian and 1/e on
 * the tensile one.  Returns r and dr/dzeta, zeta = cos(3 theta) (c solves
 * 4 c^3 - 3 c = zeta; near the compressive meridian, where dc/dzeta is
 * unbounded and dr/dc vanishes, the limit of their product is taken). */
static double ww_r(double zeta, double e, double* dr_dzeta) {
  if (zeta > 1.0) zeta = 1.0;
  if (zeta < -1.0) zeta = -1.0;
  double c = cos(acos(zeta) / 3.0);
  double a = 1.0 - e * e, b = 2.0 * e - 1.0;
  double w = sqrt(4.0 * a * c * c + 5.0 * e * e - 4.0 * e);
  double N = 4.0 * a * c * c + b * b, D = 2.0 * a * c + b * w;
  double r = N / D;
  double dN = 8.0 * a * c, dD = 2.0 * a + 4.0 * a * b * c / w;
  double rc = (dN * D - N * dD) / (D * D);
  double q = 4.0 * c * c - 1.0;
  if (fabs(q) > 1e-5)
    *dr_dzeta = rc / (3.0 * q);
  else
    *dr_dzeta = 4.0 * a / (6.0 * b * b * (2.0 * c + 1.0));
  return r;
}

/* principal return map: trial strains eps -> tau, d (3x3, d tau_a/d eps_b), g */
static int return_map(const o_params* p, double E, double ys, const double* eps, double* tau,
                      double* d, double* g, int* plastic) {
  double nu = p->nu;
  double mu = E / (2.0 * (1.0 + nu));
  double lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double Kb = lam + 2.0 * mu / 3.0;
  double tr = eps[0] + eps[1] + eps[2];
  for (int a = 0; a < 3; ++a) tau[a] = lam * tr + 2.0 * mu * eps[a];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) d[3 * a + b] = lam + (a == b ? 2.0 * mu : 0.0);
  *g = 2.0 * mu;
  *plastic = 0;
  if (p->model == 0) return 0;
  double e[3], en = 0.0;
  for (int a = 0; a < 3; ++a) {
    e[a] = eps[a] - tr / 3.0;
    en += e[a] * e[a];
  }
  en = sqrt(en);
  if (p->model == 1) {
    double pm = Kb * tr;
    double q = sqrt(1.5) * 2.0 * mu * en;
    if (q <= ys) return 0;
    *plastic = 1;
    double fac = ys / q;
    double gg = 2.0 * mu * fac;
    double eh[3] = {e[0] / en, e[1] / en, e[2] / en};
    for (int a = 0; a < 3; ++a) tau[a] = pm + 2.0 * mu * e[a] * fac;
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b)
        d[3 * a + b] = Kb + gg * ((a == b ? 1.0 : 0.0) - 1.0 / 3.0 - eh[a] * eh[b]);
    *g = gg;
    return 0;
  }
  if (p->model == 2) {
    double sphi = sin(p->phi), spsi = sin(p->psi);
    double eta = 6.0 * sphi / (sqrt(3.0) * (3.0 - sphi));
    double xi = 6.0 * cos(p->phi) / (sqrt(3.0) * (3.0 - sphi));
    double etab = 6.0 * spsi / (sqrt(3.0) * (3.0 - spsi));
    double G = mu, c = ys;
    double pm = Kb * tr;
    double sj2 = sqrt(2.0) * G * en;
    double f = sj2 + eta * pm - xi * c;
    if (f <= 0.0) return 0;
    *plastic = 1;
    double den = G + Kb * eta * etab;
    double dg = f / den;
    if (sj2 - G * dg >= 0.0 && en > 0.0) {
      double ratio = 1.0 - G * dg / sj2;
      double pn = pm - Kb * etab * dg;
      double eh[3] = {e[0] / en, e[1] / en, e[2] / en};
      for (int a = 0; a < 3; ++a) tau[a] = 2.0 * G * e[a] * ratio + pn;
      double ddg[3];
      for (int b = 0; b < 3; ++b) ddg[b] = (sqrt(2.0) * G * eh[b] + eta * Kb) / den;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double dev = (a == b ? 1.0 : 0.0) - 1.0 / 3.0;
          d[3 * a + b] = 2.0 * G * dev -
                         sqrt(2.0) * G * (eh[a] * ddg[b] + dg * (dev - eh[a] * eh[b]) / en) + Kb -
                         Kb * etab * ddg[b];
        }
      *g = 2.0 * G * ratio;
    } else {
      *plastic = 2;
      double pa = xi * c / eta;
      for (int a = 0; a < 3; ++a) tau[a] = pa;
      for (int i = 0; i < 9; ++i) d[i] = 0.0;
      *g = 0.0;
    }
    return 0;
  }
  if (p->model == 3) {
    /* frictional cone with the Willam-Warnke section and the non-associated
     * Drucker-Prager potential (Sec. 6.4): f = sqrt(J2) r(theta) + eta p - xi c
     * with the outer-cone eta, xi (r = 1 on the compressive meridian) and
     * e = (3 - sin phi)/(3 + sin phi), the Mohr-Coulomb ratio of the tensile
     * to the compressive meridian radius.  The potential sqrt(J2) + etab p has
     * a circular section, so the return shrinks the deviator radially and
     * keeps theta: f(dg) = (sqrt(J2) - G dg) r + eta (p - K etab dg) - xi c. */
    double sphi = sin(p->phi), spsi = sin(p->psi);
    double eta = 6.0 * sphi / (sqrt(3.0) * (3.0 - sphi));
    double xi = 6.0 * cos(p->phi) / (sqrt(3.0) * (3.0 - sphi));
    double etab = 6.0 * spsi / (sqrt(3.0) * (3.0 - spsi));
    double ecc = (3.0 - sphi) / (3.0 + sphi);
    double G = mu, c = ys;
    double pm = Kb * tr;
    double sj2 = sqrt(2.0) * G * en;
    double r = 1.0, drz = 0.0, dz[3] = {0.0, 0.0, 0.0};
    if (en > 0.0) {
      /* zeta = cos(3 theta) = (3 sqrt3 / 2) J3 / J2^(3/2) = 3 sqrt6 e1 e2 e3 / |e|^3 */
      double pr = e[0] * e[1] * e[2];
      double zeta = 3.0 * sqrt(6.0) * pr / (en * en * en);
      r = ww_r(zeta, ecc, &drz);
      double mm[3] = {e[1] * e[2], e[0] * e[2], e[0] * e[1]};
      double M = mm[0] + mm[1] + mm[2];
      for (int b = 0; b < 3; ++b)
        dz[b] = 3.0 * sqrt(6.0) * ((mm[b] - M / 3.0) / (en * en * en) - 3.0 * pr * e[b] / pow(en, 5.0));
      if (zeta >= 1.0 || zeta <= -1.0) dz[0] = dz[1] = dz[2] = 0.0;
    }
    double f = sj2 * r + eta * pm - xi * c;
    if (f <= 0.0) return 0;
    *plastic = 1;
    double den = G * r + Kb * eta * etab;
    double dg = f / den;
    if (sj2 - G * dg >= 0.0 && en > 0.0) {
      double ratio = 1.0 - G * dg / sj2;
      double pn = pm - Kb * etab * dg;
      double eh[3] = {e[0] / en, e[1] / en, e[2] / en};
      for (int a = 0; a < 3; ++a) tau[a] = 2.0 * G * e[a] * ratio + pn;
      double ddg[3];
      for (int b = 0; b < 3; ++b)
        ddg[b] = (sqrt(2.0) * G * eh[b] * r + (sj2 - G * dg) * drz * dz[b] + eta * Kb) / den;
      for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
          double dev = (a == b ? 1.0 : 0.0) - 1.0 / 3.0;
          d[3 * a + b] = 2.0 * G * dev -
                         sqrt(2.0) * G * (eh[a] * ddg[b] + dg * (dev - eh[a] * eh[b]) / en) + Kb -
                         Kb * etab * ddg[b];
        }
      *g = 2.0 * G * ratio;
    } else {
      *plastic = 2;
      double pa = xi * c / eta;
      for (int a = 0; a < 3; ++a) tau[a] = pa;
      for (int i = 0; i < 9; ++i) d[i] = 0.0;
      *g = 0.0;
    }
    return 0;
  }
  return O_ERR_ARG;
}

int o_constitutive(const o_params* p, double E, double ys, const double* be_n, const double* dF,
                   double* tau_out, double* be_new, double* A, int* plastic) {
  double bn[9] = {be_n[0], be_n[3], be_n[5], be_n[3], be_n[1], be_n[4], be_n[5], be_n[4], be_n[2]};
  double t1[9], btr[9], dFt[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) dFt[3 * i + j] = dF[3 * j + i];
  o_mat33_mul(dF, bn, t1);
  o_mat33_mul(t1, dFt, btr);
  double lam[3], Q[9];
  o_eig_sym3(btr, lam, Q);
  for (int a = 0; a < 3; ++a)
    if (!(lam[a] > 0.0) || !isfinite(lam[a])) return O_ERR_NAN;
  double eps[3] = {0.5 * log(lam[0]), 0.5 * log(lam[1]), 0.5 * log(lam[2])};
  double ta[3], d[9], g;
  int st = return_map(p, E, ys, eps, ta, d, &g, plastic);
  if (st) return st;
  /* tau and the elastic b_e after the return */
  double nu = p->nu;
  double mu = E / (2.0 * (1.0 + nu));
  double lamL = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  double trt = ta[0] + ta[1] + ta[2];
  double ee[3];
  for (int a = 0; a < 3; ++a) ee[a] = (ta[a] - lamL * trt / (3.0 * lamL + 2.0 * mu)) / (2.0 * mu);
  double bnew[9];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0, sb = 0.0;
      for (int a = 0; a < 3; ++a) {
        s += Q[3 * i + a] * ta[a] * Q[3 * j + a];
        sb += Q[3 * i + a] * exp(2.0 * ee[a]) * Q[3 * j + a];
      }
      tau_out[3 * i + j] = s;
      bnew[3 * i + j] = sb;
    }
  be_new[0] = bnew[0];
  be_new[1] = bnew[4];
  be_new[2] = bnew[8];
  be_new[3] = 0.5 * (bnew[1] + bnew[3]);
  be_new[4] = 0.5 * (bnew[5] + bnew[7]);
  be_new[5] = 0.5 * (bnew[2] + bnew[6]);
  if (!A) return O_OK;
  /* A_ijkm = sum_ab d_ab Q_ia Q_ja Q_kb Q_mb
   *        + sum_{a!=b} th_ab (lam_b Q_ia Q_jb Q_ka Q_mb + lam_a Q_ia Q_jb Q_kb Q_ma),
   * th_ab = (tau_a - tau_b)/(lam_a - lam_b) = g/2 * dlog(lam_a, lam_b) */
  double th[9];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b) th[3 * a + b] = a == b ? 0.0 : 0.5 * g * dlog(lam[a], lam[b]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int mm = 0; mm < 3; ++mm) {
          double s = 0.0;
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
              s += d[3 * a + b] * Q[3 * i + a] * Q[3 * j + a] * Q[3 * k + b] * Q[3 * mm + b];
              if (a != b)
                s += th[3 * a + b] * (lam[b] * Q[3 * i + a] * Q[3 * j + b] * Q[3 * k + a] * Q[3 * mm + b] +
                                      lam[a] * Q[3 * i + a] * Q[3 * j + b] * Q[3 * k + b] * Q[3 * mm + a]);
            }
          A[((i * 3 + j) * 3 + k) * 3 + mm] = s;
        }
  return O_OK;
}
