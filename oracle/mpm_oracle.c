/*
 * mpm_oracle.c -- plain FP64 CPU oracle of one MPM substep coupled to rigid
 * bodies through the convex frictional-contact problem (Yu et al., arXiv
 * 2503.05046, Sec. IV-V, Alg. 1).
 *
 * TEST INFRASTRUCTURE: see mpm_oracle.h. Serial, dense grid, no blocking, no
 * fusion; each function follows one passage of the paper or of the method it
 * cites, named in its comment. Where the paper is silent the reading taken is
 * stated beside the code.
 */
#include "mpm_oracle.h"

#include <float.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* ------------------------------------------------------------------------- */
/* small 3x3 helpers                                                          */
/* ------------------------------------------------------------------------- */

static void mat_mul(const double A[9], const double B[9], double C[9]) {
  double T[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * k + c];
      T[3 * r + c] = s;
    }
  memcpy(C, T, sizeof(T));
}

/* C = A B^T */
static void mat_mul_bt(const double A[9], const double B[9], double C[9]) {
  double T[9];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += A[3 * r + k] * B[3 * c + k];
      T[3 * r + c] = s;
    }
  memcpy(C, T, sizeof(T));
}

static double mat_det(const double A[9]) {
  return A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) +
         A[2] * (A[3] * A[7] - A[4] * A[6]);
}

/* cofactor matrix, equal to det(A) A^{-T} */
static void mat_cofactor(const double A[9], double K[9]) {
  K[0] = A[4] * A[8] - A[5] * A[7];
  K[1] = A[5] * A[6] - A[3] * A[8];
  K[2] = A[3] * A[7] - A[4] * A[6];
  K[3] = A[2] * A[7] - A[1] * A[8];
  K[4] = A[0] * A[8] - A[2] * A[6];
  K[5] = A[1] * A[6] - A[0] * A[7];
  K[6] = A[1] * A[5] - A[2] * A[4];
  K[7] = A[2] * A[3] - A[0] * A[5];
  K[8] = A[0] * A[4] - A[1] * A[3];
}

static void cross3(const double a[3], const double b[3], double c[3]) {
  double t0 = a[1] * b[2] - a[2] * b[1];
  double t1 = a[2] * b[0] - a[0] * b[2];
  double t2 = a[0] * b[1] - a[1] * b[0];
  c[0] = t0;
  c[1] = t1;
  c[2] = t2;
}

static double dot3(const double a[3], const double b[3]) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* ------------------------------------------------------------------------- */
/* MLS-MPM transfer kernel (Sec. IV-B, Eq. (6): the free motion is an explicit  */
/* MLS-MPM step with quadratic B-spline weights)                               */
/* ------------------------------------------------------------------------- */

void orc_bspline(double dx, const double origin[3], const double x[3], int base[3],
                 double fx[3], double w[9]) {
  for (int a = 0; a < 3; ++a) {
    double xi = (x[a] - origin[a]) / dx;
    base[a] = (int)floor(xi - 0.5);
    fx[a] = xi - (double)base[a];
    double f = fx[a];
    w[3 * a + 0] = 0.5 * (1.5 - f) * (1.5 - f);
    w[3 * a + 1] = 0.75 - (f - 1.0) * (f - 1.0);
    w[3 * a + 2] = 0.5 * (f - 0.5) * (f - 0.5);
  }
}

/* ------------------------------------------------------------------------- */
/* 3x3 SVD by one-sided (Hestenes) Jacobi rotations                           */
/* ------------------------------------------------------------------------- */

void orc_svd3(const double F[9], double U[9], double S[3], double V[9]) {
  double A[9];
  memcpy(A, F, sizeof(A));
  for (int i = 0; i < 9; ++i) V[i] = (i % 4 == 0) ? 1.0 : 0.0;
  static const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  for (int sweep = 0; sweep < 60; ++sweep) {
    int rotated = 0;
    for (int pi = 0; pi < 3; ++pi) {
      int p = pairs[pi][0], q = pairs[pi][1];
      double al = 0, be = 0, ga = 0;
      for (int r = 0; r < 3; ++r) {
        al += A[3 * r + p] * A[3 * r + p];
        be += A[3 * r + q] * A[3 * r + q];
        ga += A[3 * r + p] * A[3 * r + q];
      }
      if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
      rotated = 1;
      /* rotation that makes columns p and q orthogonal */
      double zeta = (be - al) / (2.0 * ga);
      double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
      double c = 1.0 / sqrt(1.0 + t * t), s = c * t;
      for (int r = 0; r < 3; ++r) {
        double ap = A[3 * r + p], aq = A[3 * r + q];
        A[3 * r + p] = c * ap - s * aq;
        A[3 * r + q] = s * ap + c * aq;
        double vp = V[3 * r + p], vq = V[3 * r + q];
        V[3 * r + p] = c * vp - s * vq;
        V[3 * r + q] = s * vp + c * vq;
      }
    }
    if (!rotated) break;
  }
  double sig[3];
  for (int c = 0; c < 3; ++c)
    sig[c] = sqrt(A[c] * A[c] + A[3 + c] * A[3 + c] + A[6 + c] * A[6 + c]);
  /* sort columns by decreasing singular value */
  int order[3] = {0, 1, 2};
  for (int i = 0; i < 3; ++i)
    for (int j = i + 1; j < 3; ++j)
      if (sig[order[j]] > sig[order[i]]) {
        int t = order[i];
        order[i] = order[j];
        order[j] = t;
      }
  double As[9], Vs[9];
  for (int c = 0; c < 3; ++c) {
    S[c] = sig[order[c]];
    for (int r = 0; r < 3; ++r) {
      As[3 * r + c] = A[3 * r + order[c]];
      Vs[3 * r + c] = V[3 * r + order[c]];
    }
  }
  memcpy(V, Vs, sizeof(Vs));
  /* left singular vectors; complete the basis where a singular value vanishes */
  double tiny = 1e-300 + 1e-14 * S[0];
  for (int c = 0; c < 3; ++c) {
    if (S[c] > tiny) {
      for (int r = 0; r < 3; ++r) U[3 * r + c] = As[3 * r + c] / S[c];
    } else if (c == 2) {
      double u0[3] = {U[0], U[3], U[6]}, u1[3] = {U[1], U[4], U[7]}, u2[3];
      cross3(u0, u1, u2);
      for (int r = 0; r < 3; ++r) U[3 * r + 2] = u2[r];
      S[2] = 0.0;
    } else if (c == 1) {
      double u0[3] = {U[0], U[3], U[6]};
      if (S[0] <= tiny) { /* F = 0 */
        u0[0] = 1; u0[1] = 0; u0[2] = 0;
        U[0] = 1; U[3] = 0; U[6] = 0;
      }
      double e[3] = {0, 0, 0};
      int a = (fabs(u0[0]) <= fabs(u0[1]) && fabs(u0[0]) <= fabs(u0[2])) ? 0
              : (fabs(u0[1]) <= fabs(u0[2])) ? 1 : 2;
      e[a] = 1.0;
      double u1[3];
      cross3(u0, e, u1);
      double nn = sqrt(dot3(u1, u1));
      for (int r = 0; r < 3; ++r) U[3 * r + 1] = u1[r] / nn;
      S[1] = 0.0;
    } else {
      U[0] = 1; U[3] = 0; U[6] = 0;
      S[0] = 0.0;
    }
  }
  /* proper rotations: push any reflection into the smallest singular value */
  if (mat_det(U) < 0) {
    for (int r = 0; r < 3; ++r) U[3 * r + 2] = -U[3 * r + 2];
    S[2] = -S[2];
  }
  if (mat_det(V) < 0) {
    for (int r = 0; r < 3; ++r) V[3 * r + 2] = -V[3 * r + 2];
    S[2] = -S[2];
  }
}

/* ------------------------------------------------------------------------- */
/* Constitutive models (Sec. IV-B: k_d holds the elastic-plastic forces).      */
/* ------------------------------------------------------------------------- */

void orc_lame(double E, double nu, double* mu, double* lam) {
  *mu = E / (2.0 * (1.0 + nu));
  *lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
}

/* fixed corotated: P = 2 mu (F - R) + lam (J - 1) J F^{-T}, R the rotation of
   the polar decomposition of F */
void orc_corotated_P(const double F[9], double mu, double lam, double P[9]) {
  double U[9], S[3], V[9], R[9], K[9];
  orc_svd3(F, U, S, V);
  mat_mul_bt(U, V, R);
  double J = mat_det(F);
  mat_cofactor(F, K);
  for (int i = 0; i < 9; ++i) P[i] = 2.0 * mu * (F[i] - R[i]) + lam * (J - 1.0) * K[i];
}

void orc_corotated_tau(const double F[9], double mu, double lam, double tau[9]) {
  double P[9];
  orc_corotated_P(F, mu, lam, P);
  mat_mul_bt(P, F, tau);
}

/* singular values below this are clamped before taking logarithms */
#define ORC_HENCKY_SIGMA_MIN 1e-4

void orc_hencky_P(const double F[9], double mu, double lam, double P[9]) {
  double U[9], S[3], V[9];
  orc_svd3(F, U, S, V);
  double e[3], tr = 0.0;
  for (int a = 0; a < 3; ++a) {
    S[a] = fmax(S[a], ORC_HENCKY_SIGMA_MIN);
    e[a] = log(S[a]);
    tr += e[a];
  }
  double D[9] = {0};
  for (int a = 0; a < 3; ++a) D[4 * a] = (2.0 * mu * e[a] + lam * tr) / S[a];
  double T[9];
  mat_mul(U, D, T);
  mat_mul_bt(T, V, P);
}

/* Kirchhoff stress of the Hencky model in principal form,
   tau = U diag(2 mu e + lam tr e) U^T with e = ln max(sigma, sigma_min): equal
   to P F^T while no singular value is clamped, and the stress of the clamped
   strain otherwise (also for an inverted F, whose negative singular value is
   clamped). */
void orc_hencky_tau(const double F[9], double mu, double lam, double tau[9]) {
  double U[9], S[3], V[9];
  orc_svd3(F, U, S, V);
  double e[3], tr = 0.0;
  for (int a = 0; a < 3; ++a) {
    e[a] = log(fmax(S[a], ORC_HENCKY_SIGMA_MIN));
    tr += e[a];
  }
  double D[9] = {0};
  for (int a = 0; a < 3; ++a) D[4 * a] = 2.0 * mu * e[a] + lam * tr;
  double T[9];
  mat_mul(U, D, T);
  mat_mul_bt(T, U, tau);
}

/* Drucker-Prager plasticity in Hencky strain space (the granular model the
   paper cites for sand, Sec. II-A): project the log singular values onto the
   cone; expansion projects to the tip (stress free). */
void orc_dp_project(const double F[9], double mu, double lam, double friction_angle_deg,
                    double Fout[9]) {
  double U[9], S[3], V[9];
  orc_svd3(F, U, S, V);
  int clamped = 0;
  double e[3], tr = 0.0;
  for (int a = 0; a < 3; ++a) {
    if (S[a] < ORC_HENCKY_SIGMA_MIN) {
      S[a] = ORC_HENCKY_SIGMA_MIN;
      clamped = 1;
    }
    e[a] = log(S[a]);
    tr += e[a];
  }
  double sphi = sin(friction_angle_deg * 3.14159265358979323846 / 180.0);
  double alpha = sqrt(2.0 / 3.0) * 2.0 * sphi / (3.0 - sphi);
  double ehat[3], nh = 0.0;
  for (int a = 0; a < 3; ++a) {
    ehat[a] = e[a] - tr / 3.0;
    nh += ehat[a] * ehat[a];
  }
  nh = sqrt(nh);
  double enew[3];
  int project = 0;
  if (tr >= 0.0) {
    enew[0] = enew[1] = enew[2] = 0.0;
    project = 1;
  } else {
    double dgamma = nh + (3.0 * lam + 2.0 * mu) / (2.0 * mu) * tr * alpha;
    if (dgamma > 0.0) {
      for (int a = 0; a < 3; ++a) enew[a] = e[a] - dgamma * ehat[a] / nh;
      project = 1;
    }
  }
  if (!project && !clamped) {
    if (Fout != F) memcpy(Fout, F, 9 * sizeof(double));
    return;
  }
  if (!project)
    for (int a = 0; a < 3; ++a) enew[a] = e[a];
  double D[9] = {0};
  for (int a = 0; a < 3; ++a) D[4 * a] = exp(enew[a]);
  double T[9];
  mat_mul(U, D, T);
  mat_mul_bt(T, V, Fout);
}

/* ------------------------------------------------------------------------- */
/* Rigid geometry (Sec. V-B: one contact per particle inside a geometry)       */
/* ------------------------------------------------------------------------- */

/* ---- cloth: corotated membrane energy of a triangle ----------------------- */

void orc_cloth_rest(const double X0[3], const double X1[3], const double X2[3],
                    double Dm_inv[4], double* area) {
  double e1[3], e2[3], nrm[3], t1[3], t2[3];
  for (int a = 0; a < 3; ++a) {
    e1[a] = X1[a] - X0[a];
    e2[a] = X2[a] - X0[a];
  }
  cross3(e1, e2, nrm);
  const double nn = sqrt(dot3(nrm, nrm)), l1 = sqrt(dot3(e1, e1));
  *area = 0.5 * nn;
  for (int a = 0; a < 3; ++a) {
    t1[a] = e1[a] / l1;
    nrm[a] /= nn;
  }
  cross3(nrm, t1, t2);
  /* the rest edges in the triangle's frame (t1, t2): Dm = [[|e1|, e2.t1], [0, e2.t2]] */
  const double a00 = l1, a01 = dot3(e2, t1), a11 = dot3(e2, t2);
  Dm_inv[0] = 1.0 / a00;
  Dm_inv[1] = -a01 / (a00 * a11);
  Dm_inv[2] = 0.0;
  Dm_inv[3] = 1.0 / a11;
}

double orc_cloth_triangle(const double x0[3], const double x1[3], const double x2[3],
                          const double Dm_inv[4], double vol, double mu, double lam,
                          double f[9]) {
  /* F = Ds Dm^-1, 3x2 row-major: F[2r + c] */
  double Ds[6], F[6];
  for (int r = 0; r < 3; ++r) {
    Ds[2 * r] = x1[r] - x0[r];
    Ds[2 * r + 1] = x2[r] - x0[r];
  }
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 2; ++c)
      F[2 * r + c] = Ds[2 * r] * Dm_inv[c] + Ds[2 * r + 1] * Dm_inv[2 + c];
  /* C = F^T F (2x2), S = sqrt(C) = (C + sqrt(det C) I) / sqrt(tr C + 2 sqrt(det C)) */
  double Cm[4] = {0, 0, 0, 0};
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b)
      for (int r = 0; r < 3; ++r) Cm[2 * a + b] += F[2 * r + a] * F[2 * r + b];
  const double detC = Cm[0] * Cm[3] - Cm[1] * Cm[2];
  const double J = sqrt(detC > 0.0 ? detC : 0.0);
  const double tnorm = sqrt(Cm[0] + Cm[3] + 2.0 * J);
  const double S[4] = {(Cm[0] + J) / tnorm, Cm[1] / tnorm, Cm[2] / tnorm, (Cm[3] + J) / tnorm};
  /* R = F S^-1 (det S = J) */
  const double Si[4] = {S[3] / J, -S[1] / J, -S[2] / J, S[0] / J};
  double R[6];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 2; ++c) R[2 * r + c] = F[2 * r] * Si[c] + F[2 * r + 1] * Si[2 + c];
  double fr2 = 0.0;
  for (int e = 0; e < 6; ++e) fr2 += (F[e] - R[e]) * (F[e] - R[e]);
  const double psi = mu * fr2 + 0.5 * lam * (J - 1.0) * (J - 1.0);
  if (f) {
    /* P = 2 mu (F - R) + lam (J - 1) J F C^-1 */
    const double Ci[4] = {Cm[3] / detC, -Cm[1] / detC, -Cm[2] / detC, Cm[0] / detC};
    double P[6];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 2; ++c)
        P[2 * r + c] = 2.0 * mu * (F[2 * r + c] - R[2 * r + c]) +
                       lam * (J - 1.0) * J * (F[2 * r] * Ci[c] + F[2 * r + 1] * Ci[2 + c]);
    /* dE/dDs = vol P Dm^-T; f1, f2 its columns negated, f0 = -(f1 + f2) */
    for (int r = 0; r < 3; ++r) {
      const double g1 = vol * (P[2 * r] * Dm_inv[0] + P[2 * r + 1] * Dm_inv[1]);
      const double g2 = vol * (P[2 * r] * Dm_inv[2] + P[2 * r + 1] * Dm_inv[3]);
      f[3 + r] = -g1;
      f[6 + r] = -g2;
      f[r] = g1 + g2;
    }
  }
  return vol * psi;
}

double orc_sdf(const orc_body* b, const double x[3], double n[3]) {
  /* body-frame point y = R^T (x - p) */
  double r[3] = {x[0] - b->p[0], x[1] - b->p[1], x[2] - b->p[2]};
  double y[3];
  for (int c = 0; c < 3; ++c) y[c] = b->R[c] * r[0] + b->R[3 + c] * r[1] + b->R[6 + c] * r[2];
  double nb[3] = {0, 0, 1};
  double phi;
  switch (b->shape) {
    case ORC_HALFSPACE:
      phi = y[2];
      break;
    case ORC_SPHERE: {
      double dist = sqrt(dot3(y, y));
      phi = dist - b->params[0];
      if (dist > 0) {
        nb[0] = y[0] / dist; nb[1] = y[1] / dist; nb[2] = y[2] / dist;
      }
      break;
    }
    case ORC_BOX: {
      double q[3];
      int amax = 0;
      for (int a = 0; a < 3; ++a) {
        q[a] = fabs(y[a]) - b->params[a];
        if (q[a] > q[amax]) amax = a;
      }
      if (q[amax] <= 0.0) { /* inside: nearest face, lowest axis on ties */
        phi = q[amax];
        nb[0] = nb[1] = nb[2] = 0.0;
        nb[amax] = (y[amax] >= 0.0) ? 1.0 : -1.0;
      } else {
        double o[3];
        for (int a = 0; a < 3; ++a) o[a] = (q[a] > 0.0 ? q[a] : 0.0) * (y[a] >= 0.0 ? 1.0 : -1.0);
        phi = sqrt(dot3(o, o));
        for (int a = 0; a < 3; ++a) nb[a] = o[a] / phi;
      }
      break;
    }
    case ORC_CAPSULE: {
      double L = b->params[0], rad = b->params[1];
      double cz = y[2] < -L ? -L : (y[2] > L ? L : y[2]);
      double o[3] = {y[0], y[1], y[2] - cz};
      double dist = sqrt(dot3(o, o));
      phi = dist - rad;
      if (dist > 0) {
        nb[0] = o[0] / dist; nb[1] = o[1] / dist; nb[2] = o[2] / dist;
      } else {
        nb[0] = 1; nb[1] = 0; nb[2] = 0;
      }
      break;
    }
    default:
      phi = 1e300;
  }
  for (int r2 = 0; r2 < 3; ++r2) n[r2] = b->R[3 * r2] * nb[0] + b->R[3 * r2 + 1] * nb[1] + b->R[3 * r2 + 2] * nb[2];
  return phi;
}

void orc_body_velocity(const orc_body* b, const double x[3], double vel[3]) {
  double r[3] = {x[0] - b->p[0], x[1] - b->p[1], x[2] - b->p[2]}, wr[3];
  cross3(b->omega, r, wr);
  for (int c = 0; c < 3; ++c) vel[c] = b->v[c] + wr[c];
}

/* Contact frame (Sec. IV-B: local frame whose z axis is the contact normal). */
void orc_contact_frame(const double n[3], double angle, double R[9]) {
  int a = (fabs(n[0]) <= fabs(n[1]) && fabs(n[0]) <= fabs(n[2])) ? 0
          : (fabs(n[1]) <= fabs(n[2])) ? 1 : 2;
  double e[3] = {0, 0, 0};
  e[a] = 1.0;
  double t1[3], t2[3];
  cross3(e, n, t1);
  double nt = sqrt(dot3(t1, t1));
  for (int c = 0; c < 3; ++c) t1[c] /= nt;
  cross3(n, t1, t2);
  double ca = cos(angle), sa = sin(angle);
  for (int r = 0; r < 3; ++r) {
    R[3 * r + 0] = ca * t1[r] + sa * t2[r];
    R[3 * r + 1] = -sa * t1[r] + ca * t2[r];
    R[3 * r + 2] = n[r];
  }
}

/* ------------------------------------------------------------------------- */
/* Lagged contact model (Sec. IV-B: gamma = -dl_c/dv_c, convex l_c).           */
/* Reading: compliant normal law with Hunt-Crossley dissipation, made convex   */
/* by integrating the impulse in v_n, plus regularised Coulomb friction whose  */
/* normal impulse n0 is lagged (held fixed during the solve).                  */
/* ------------------------------------------------------------------------- */

double orc_normal_impulse(double phi0, double k, double d, double h, double vn) {
  double a = phi0 - h * vn, c = 1.0 - d * vn;
  if (a <= 0.0 || c <= 0.0) return 0.0;
  return h * k * a * c;
}

/* antiderivative in v_n of (phi0 - h s)(1 - d s) */
static double normal_antiderivative(double phi0, double d, double h, double s) {
  return phi0 * s - 0.5 * (phi0 * d + h) * s * s + h * d * s * s * s / 3.0;
}

double orc_contact_potential(double phi0, double n0, double mu, double k, double d,
                             double h, double eps_s, const double vc[3], double grad[3],
                             double hess[9]) {
  double vn = vc[2];
  double vhat = phi0 / h;
  if (d > 0.0 && 1.0 / d < vhat) vhat = 1.0 / d;
  double N = 0.0, dN = 0.0, d2N = 0.0;
  if (vn < vhat) {
    N = h * k * (normal_antiderivative(phi0, d, h, vhat) - normal_antiderivative(phi0, d, h, vn));
    dN = -h * k * (phi0 - h * vn) * (1.0 - d * vn);
    d2N = h * k * (h * (1.0 - d * vn) + d * (phi0 - h * vn));
  }
  double s = sqrt(vc[0] * vc[0] + vc[1] * vc[1] + eps_s * eps_s);
  double c = mu * n0;
  double ell = N + c * (s - eps_s);
  if (grad) {
    grad[0] = c * vc[0] / s;
    grad[1] = c * vc[1] / s;
    grad[2] = dN;
  }
  if (hess) {
    double s3 = s * s * s;
    hess[0] = c * (1.0 / s - vc[0] * vc[0] / s3);
    hess[1] = -c * vc[0] * vc[1] / s3;
    hess[2] = 0.0;
    hess[3] = hess[1];
    hess[4] = c * (1.0 / s - vc[1] * vc[1] / s3);
    hess[5] = 0.0;
    hess[6] = 0.0;
    hess[7] = 0.0;
    hess[8] = d2N;
  }
  return ell;
}

/* ------------------------------------------------------------------------- */
/* The contact problem, Eq. (8)-(10)                                          */
/* ------------------------------------------------------------------------- */

static int is_fixed(const orc_problem* P, int i) { return P->fixed && P->fixed[i]; }

/* v_c = J v + b for every contact (J: world grid velocity -> contact frame) */
static void contact_velocities(const orc_problem* P, const double* v, int with_bias,
                               double* vc) {
  for (int p = 0; p < P->n_contacts; ++p) {
    double u[3] = {0, 0, 0};
    for (int s = 0; s < 27; ++s) {
      int i = P->nodes[27 * p + s];
      if (i < 0) continue;
      double w = P->w[27 * p + s];
      for (int c = 0; c < 3; ++c) u[c] += w * v[3 * i + c];
    }
    const double* R = P->R + 9 * p;
    for (int c = 0; c < 3; ++c) {
      vc[3 * p + c] = R[c] * u[0] + R[3 + c] * u[1] + R[6 + c] * u[2];
      if (with_bias) vc[3 * p + c] += P->b[3 * p + c];
    }
  }
}

static double contact_l(const orc_problem* P, int p, const double vc[3], double grad[3],
                        double hess[9]) {
  return orc_contact_potential(P->phi0[p], P->n0[p], P->mu[p], P->k[p], P->d[p], P->h,
                               P->eps_s, vc, grad, hess);
}

double orc_objective(const orc_problem* P, const double* v) {
  double f = 0.0;
  for (int i = 0; i < P->n_nodes; ++i)
    for (int c = 0; c < 3; ++c) {
      double dv = v[3 * i + c] - P->vstar[3 * i + c];
      f += 0.5 * P->m[i] * dv * dv;
    }
  double* vc = (double*)malloc(sizeof(double) * 3 * (P->n_contacts + 1));
  contact_velocities(P, v, 1, vc);
  for (int p = 0; p < P->n_contacts; ++p) f += contact_l(P, p, vc + 3 * p, NULL, NULL);
  free(vc);
  return f;
}

/* J^T (dl_c/dv_c): per node, sum over contacts of w R grad */
static void contact_force(const orc_problem* P, const double* vc, double* jc) {
  memset(jc, 0, sizeof(double) * 3 * P->n_nodes);
  for (int p = 0; p < P->n_contacts; ++p) {
    double gr[3];
    contact_l(P, p, vc + 3 * p, gr, NULL);
    const double* R = P->R + 9 * p;
    double gw[3];
    for (int r = 0; r < 3; ++r) gw[r] = R[3 * r] * gr[0] + R[3 * r + 1] * gr[1] + R[3 * r + 2] * gr[2];
    for (int s = 0; s < 27; ++s) {
      int i = P->nodes[27 * p + s];
      if (i < 0) continue;
      double w = P->w[27 * p + s];
      for (int c = 0; c < 3; ++c) jc[3 * i + c] += w * gw[c];
    }
  }
}

void orc_gradient(const orc_problem* P, const double* v, double* g) {
  double* vc = (double*)malloc(sizeof(double) * 3 * (P->n_contacts + 1));
  contact_velocities(P, v, 1, vc);
  contact_force(P, vc, g);
  for (int i = 0; i < P->n_nodes; ++i)
    for (int c = 0; c < 3; ++c) {
      if (is_fixed(P, i))
        g[3 * i + c] = 0.0;
      else
        g[3 * i + c] += P->m[i] * (v[3 * i + c] - P->vstar[3 * i + c]);
    }
  free(vc);
}

/* f'(alpha) and f''(alpha) of f(alpha) = l_p(v + alpha dv) with
   A = dv^T M dv, B = dv^T M (v - v*) (the grid part, Sec. V-B) */
static double ls_derivs(const orc_problem* P, const double* vc, const double* dvc, double A,
                        double B, double alpha, double* d2) {
  double d1 = B + alpha * A, dd = A;
  for (int p = 0; p < P->n_contacts; ++p) {
    double u[3], gr[3], H[9];
    for (int c = 0; c < 3; ++c) u[c] = vc[3 * p + c] + alpha * dvc[3 * p + c];
    contact_l(P, p, u, gr, H);
    const double* e = dvc + 3 * p;
    d1 += gr[0] * e[0] + gr[1] * e[1] + gr[2] * e[2];
    for (int r = 0; r < 3; ++r)
      for (int c = 0; c < 3; ++c) dd += e[r] * H[3 * r + c] * e[c];
  }
  *d2 = dd;
  return d1;
}

/* Exact line search of Alg. 1 (Sec. V-B: one-dimensional Newton falling back
   to bisection). Reading of the unstated details: bracket [0, a_hi] with
   a_hi = 1 doubled while f'(a_hi) < 0 (at most 2^10); inside the bracket a
   Newton step is taken unless it leaves the bracket or |f'| failed to halve
   since the previous iterate, in which case the bracket is bisected. */
static double line_search(const orc_problem* P, const orc_solver* S, const double* vc,
                          const double* dvc, double A, double B, int* evals, int* status) {
  double d2;
  double d0 = ls_derivs(P, vc, dvc, A, B, 0.0, &d2);
  ++*evals;
  if (!(d0 < 0.0)) return 0.0;
  double tol = S->ls_rel_tol * fabs(d0);
  double lo = 0.0, hi = 1.0;
  double dhi = ls_derivs(P, vc, dvc, A, B, hi, &d2);
  ++*evals;
  while (dhi < 0.0) {
    lo = hi;
    hi *= 2.0;
    if (hi > 1024.0) {
      *status = ORC_ERR_LINE_SEARCH;
      return lo;
    }
    dhi = ls_derivs(P, vc, dvc, A, B, hi, &d2);
    ++*evals;
  }
  if (fabs(dhi) <= tol) return hi;
  double a = hi, d1 = dhi, prev_abs = INFINITY;
  for (int it = 0; it < S->ls_max_iters; ++it) {
    /* d1, d2 hold f', f'' at a */
    if (d1 < 0.0)
      lo = a;
    else
      hi = a;
    double an = a - d1 / d2;
    int newton_ok = (d2 > 0.0) && (an > lo) && (an < hi) && (fabs(d1) <= 0.5 * prev_abs);
    prev_abs = fabs(d1);
    a = newton_ok ? an : 0.5 * (lo + hi);
    d1 = ls_derivs(P, vc, dvc, A, B, a, &d2);
    ++*evals;
    if (fabs(d1) <= tol) return a;
    if (hi - lo <= 1e-15 * hi) return a;
  }
  return a;
}

static void stopping_norms(const orc_problem* P, const double* v, const double* g,
                           const double* jc, double* G, double* Pn, double* Jn) {
  double sg = 0, sp = 0, sj = 0;
  for (int i = 0; i < P->n_nodes; ++i) {
    if (is_fixed(P, i)) continue;
    double m = P->m[i];
    for (int c = 0; c < 3; ++c) {
      sg += g[3 * i + c] * g[3 * i + c] / m;
      sp += m * v[3 * i + c] * v[3 * i + c];
      sj += jc[3 * i + c] * jc[3 * i + c] / m;
    }
  }
  *G = sqrt(sg);
  *Pn = sqrt(sp);
  *Jn = sqrt(sj);
}

/* 3x3 SPD solve by Cholesky; returns 0 if not SPD */
static int chol3_solve(const double H[9], const double g[3], double x[3]) {
  double l00 = H[0];
  if (!(l00 > 0)) return 0;
  l00 = sqrt(l00);
  double l10 = H[3] / l00, l20 = H[6] / l00;
  double t11 = H[4] - l10 * l10;
  if (!(t11 > 0)) return 0;
  double l11 = sqrt(t11);
  double l21 = (H[7] - l20 * l10) / l11;
  double t22 = H[8] - l20 * l20 - l21 * l21;
  if (!(t22 > 0)) return 0;
  double l22 = sqrt(t22);
  double y0 = g[0] / l00;
  double y1 = (g[1] - l10 * y0) / l11;
  double y2 = (g[2] - l20 * y0 - l21 * y1) / l22;
  x[2] = y2 / l22;
  x[1] = (y1 - l21 * x[2]) / l11;
  x[0] = (y0 - l10 * x[1] - l20 * x[2]) / l00;
  return 1;
}

static void final_impulses(const orc_problem* P, const double* v, double* gamma) {
  if (!gamma) return;
  double* vc = (double*)malloc(sizeof(double) * 3 * (P->n_contacts + 1));
  contact_velocities(P, v, 1, vc);
  for (int p = 0; p < P->n_contacts; ++p) {
    double gr[3];
    contact_l(P, p, vc + 3 * p, gr, NULL);
    /* gamma = -dl_c/dv_c (Sec. IV-B) */
    for (int c = 0; c < 3; ++c) gamma[3 * p + c] = -gr[c];
  }
  free(vc);
}

int orc_solve_qn(const orc_problem* P, const orc_solver* S, double* v, double* gamma,
                 orc_solve_info* info, double* hist) {
  int n = P->n_nodes, nc = P->n_contacts;
  double* vc = (double*)malloc(sizeof(double) * 3 * (nc + 1));
  double* dvc = (double*)malloc(sizeof(double) * 3 * (nc + 1));
  double* jc = (double*)malloc(sizeof(double) * 3 * (n + 1));
  double* g = (double*)malloc(sizeof(double) * 3 * (n + 1));
  double* H = (double*)malloc(sizeof(double) * 9 * (n + 1));
  double* dv = (double*)malloc(sizeof(double) * 3 * (n + 1));
  orc_solve_info inf = {0};
  inf.status = ORC_OK;
  for (int i = 0; i < n; ++i)
    if (is_fixed(P, i))
      for (int c = 0; c < 3; ++c) v[3 * i + c] = P->vstar[3 * i + c];
  int it = 0;
  for (;; ++it) {
    /* gradient, Eq. (9) */
    contact_velocities(P, v, 1, vc);
    contact_force(P, vc, jc);
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c)
        g[3 * i + c] = is_fixed(P, i) ? 0.0
                                      : P->m[i] * (v[3 * i + c] - P->vstar[3 * i + c]) + jc[3 * i + c];
    stopping_norms(P, v, g, jc, &inf.G, &inf.P, &inf.J);
    if (hist) hist[it] = orc_objective(P, v);
    double thr = S->eps_a + S->eps_r * fmax(inf.P, inf.J);
    if (inf.G < thr || inf.G == 0.0) {
      inf.converged = 1;
      break;
    }
    if (it >= S->max_iters) {
      inf.status = ORC_ERR_NOT_CONVERGED;
      break;
    }
    /* 3x3 diagonal blocks of the Hessian, Eq. (10) */
    for (int i = 0; i < n; ++i) {
      for (int e = 0; e < 9; ++e) H[9 * i + e] = 0.0;
      H[9 * i + 0] = H[9 * i + 4] = H[9 * i + 8] = P->m[i];
    }
    for (int p = 0; p < nc; ++p) {
      double gr[3], Gc[9], RG[9], Gw[9];
      contact_l(P, p, vc + 3 * p, gr, Gc);
      mat_mul(P->R + 9 * p, Gc, RG);
      mat_mul_bt(RG, P->R + 9 * p, Gw);
      for (int s = 0; s < 27; ++s) {
        int i = P->nodes[27 * p + s];
        if (i < 0) continue;
        double w2 = P->w[27 * p + s] * P->w[27 * p + s];
        for (int e = 0; e < 9; ++e) H[9 * i + e] += w2 * Gw[e];
      }
    }
    /* search direction: dv = -H^{-1} grad (Alg. 1) */
    double A = 0.0, B = 0.0;
    for (int i = 0; i < n; ++i) {
      double x[3] = {0, 0, 0};
      if (!is_fixed(P, i)) {
        double mg[3] = {-g[3 * i], -g[3 * i + 1], -g[3 * i + 2]};
        if (!chol3_solve(H + 9 * i, mg, x)) inf.status = ORC_ERR_NOT_SPD;
      }
      for (int c = 0; c < 3; ++c) {
        dv[3 * i + c] = x[c];
        A += P->m[i] * x[c] * x[c];
        B += P->m[i] * x[c] * (v[3 * i + c] - P->vstar[3 * i + c]);
      }
    }
    if (inf.status == ORC_ERR_NOT_SPD) break;
    contact_velocities(P, dv, 0, dvc);
    int ls_status = ORC_OK;
    double alpha = line_search(P, S, vc, dvc, A, B, &inf.ls_evals, &ls_status);
    if (ls_status != ORC_OK) inf.status = ls_status;
    for (int e = 0; e < 3 * n; ++e) v[e] += alpha * dv[e];
    if (ls_status != ORC_OK) {
      ++it;
      break;
    }
  }
  inf.iters = it;
  final_impulses(P, v, gamma);
  if (info) *info = inf;
  free(vc); free(dvc); free(jc); free(g); free(H); free(dv);
  return inf.status;
}

/* dense Cholesky factorisation in place (lower); 0 if not SPD */
static int dense_cholesky(double* A, int n) {
  for (int j = 0; j < n; ++j) {
    double s = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(s > 0)) return 0;
    double l = sqrt(s);
    A[(size_t)j * n + j] = l;
    for (int i = j + 1; i < n; ++i) {
      double t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = t / l;
    }
  }
  return 1;
}

static void dense_cholesky_solve(const double* L, int n, double* x) {
  for (int i = 0; i < n; ++i) {
    double t = x[i];
    for (int k = 0; k < i; ++k) t -= L[(size_t)i * n + k] * x[k];
    x[i] = t / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    double t = x[i];
    for (int k = i + 1; k < n; ++k) t -= L[(size_t)k * n + i] * x[k];
    x[i] = t / L[(size_t)i * n + i];
  }
}

int orc_solve_dense_newton(const orc_problem* P, const orc_solver* S, double* v,
                           double* gamma, orc_solve_info* info) {
  int n = P->n_nodes, nc = P->n_contacts, N3 = 3 * n;
  double* vc = (double*)malloc(sizeof(double) * 3 * (nc + 1));
  double* dvc = (double*)malloc(sizeof(double) * 3 * (nc + 1));
  double* jc = (double*)malloc(sizeof(double) * 3 * (n + 1));
  double* g = (double*)malloc(sizeof(double) * 3 * (n + 1));
  double* dv = (double*)malloc(sizeof(double) * 3 * (n + 1));
  double* Hd = (double*)malloc(sizeof(double) * (size_t)N3 * N3 + 8);
  orc_solve_info inf = {0};
  for (int i = 0; i < n; ++i)
    if (is_fixed(P, i))
      for (int c = 0; c < 3; ++c) v[3 * i + c] = P->vstar[3 * i + c];
  int it = 0;
  for (;; ++it) {
    contact_velocities(P, v, 1, vc);
    contact_force(P, vc, jc);
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c)
        g[3 * i + c] = is_fixed(P, i) ? 0.0
                                      : P->m[i] * (v[3 * i + c] - P->vstar[3 * i + c]) + jc[3 * i + c];
    stopping_norms(P, v, g, jc, &inf.G, &inf.P, &inf.J);
    double thr = S->eps_a + S->eps_r * fmax(inf.P, inf.J);
    if (inf.G < thr || inf.G == 0.0) {
      inf.converged = 1;
      break;
    }
    if (it >= S->max_iters) {
      inf.status = ORC_ERR_NOT_CONVERGED;
      break;
    }
    /* full Hessian of Eq. (10): M + J^T (d2 l_c) J; Dirichlet rows -> identity */
    memset(Hd, 0, sizeof(double) * (size_t)N3 * N3);
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) Hd[(size_t)(3 * i + c) * N3 + 3 * i + c] = P->m[i];
    for (int p = 0; p < nc; ++p) {
      double gr[3], Gc[9], RG[9], Gw[9];
      contact_l(P, p, vc + 3 * p, gr, Gc);
      mat_mul(P->R + 9 * p, Gc, RG);
      mat_mul_bt(RG, P->R + 9 * p, Gw);
      for (int s = 0; s < 27; ++s) {
        int i = P->nodes[27 * p + s];
        if (i < 0 || is_fixed(P, i)) continue;
        for (int t = 0; t < 27; ++t) {
          int j = P->nodes[27 * p + t];
          if (j < 0 || is_fixed(P, j)) continue;
          double ww = P->w[27 * p + s] * P->w[27 * p + t];
          for (int r = 0; r < 3; ++r)
            for (int c = 0; c < 3; ++c) Hd[(size_t)(3 * i + r) * N3 + 3 * j + c] += ww * Gw[3 * r + c];
        }
      }
    }
    if (!dense_cholesky(Hd, N3)) {
      inf.status = ORC_ERR_NOT_SPD;
      break;
    }
    for (int e = 0; e < N3; ++e) dv[e] = -g[e];
    dense_cholesky_solve(Hd, N3, dv);
    double A = 0.0, B = 0.0;
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) {
        if (is_fixed(P, i)) dv[3 * i + c] = 0.0;
        A += P->m[i] * dv[3 * i + c] * dv[3 * i + c];
        B += P->m[i] * dv[3 * i + c] * (v[3 * i + c] - P->vstar[3 * i + c]);
      }
    contact_velocities(P, dv, 0, dvc);
    int ls_status = ORC_OK;
    double alpha = line_search(P, S, vc, dvc, A, B, &inf.ls_evals, &ls_status);
    if (ls_status != ORC_OK) inf.status = ls_status;
    for (int e = 0; e < N3; ++e) v[e] += alpha * dv[e];
    if (ls_status != ORC_OK) {
      ++it;
      break;
    }
  }
  inf.iters = it;
  final_impulses(P, v, gamma);
  if (info) *info = inf;
  free(vc); free(dvc); free(jc); free(g); free(dv); free(Hd);
  return inf.status;
}

/* ------------------------------------------------------------------------- */
/* One substep over particles, Eq. (5): free motion (6), contact solve (7)-(8) */
/* ------------------------------------------------------------------------- */

struct orc_sim {
  orc_grid g;
  size_t nn;
  double* m;   /* [nn] */
  double* p;   /* [3nn] momentum, then v* */
  double* v;   /* [3nn] post-contact velocity */
  int* dof;    /* [nn] DoF index or -1 */
  int n_dof;
  int* dof_node; /* [nn] */
  /* last contacts */
  int n_con, con_cap;
  int* con_p;
  int* con_b;
  double* con_gamma;
  double* con_phi0;
  double* con_n0;
  /* cloth meshes (orc_set_cloth) and the forces of the current substep */
  int n_tris;
  int* tris;
  double* tri_Dm_inv;
  double* tri_area;
  int* tri_mat;
  double* fext;
  int fext_cap;
  /* pinned particles (orc_set_pins): ids, prescribed velocities, and their
     positions at the start of the current substep */
  int n_pins;
  int* pin_ids;
  double* pin_v;
  double* pin_x0;
};

orc_sim* orc_create(const orc_grid* grid) {
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->g = *grid;
  s->nn = (size_t)grid->res[0] * grid->res[1] * grid->res[2];
  s->m = (double*)calloc(s->nn, sizeof(double));
  s->p = (double*)calloc(3 * s->nn, sizeof(double));
  s->v = (double*)calloc(3 * s->nn, sizeof(double));
  s->dof = (int*)malloc(s->nn * sizeof(int));
  s->dof_node = (int*)malloc(s->nn * sizeof(int));
  for (size_t i = 0; i < s->nn; ++i) s->dof[i] = -1;
  return s;
}

int orc_set_cloth(orc_sim* s, int n_tris, const int* tris, const double* Dm_inv,
                  const double* vol, const int* mat_of_tri) {
  if (!s || n_tris < 0 || (n_tris > 0 && (!tris || !Dm_inv || !vol || !mat_of_tri)))
    return ORC_ERR_ARG;
  free(s->tris); free(s->tri_Dm_inv); free(s->tri_area); free(s->tri_mat);
  s->n_tris = n_tris;
  const size_t nt = (size_t)(n_tris > 0 ? n_tris : 1);
  s->tris = (int*)malloc(sizeof(int) * 3 * nt);
  s->tri_Dm_inv = (double*)malloc(sizeof(double) * 4 * nt);
  s->tri_area = (double*)malloc(sizeof(double) * nt);
  s->tri_mat = (int*)malloc(sizeof(int) * nt);
  if (n_tris > 0) {
    memcpy(s->tris, tris, sizeof(int) * 3 * (size_t)n_tris);
    memcpy(s->tri_Dm_inv, Dm_inv, sizeof(double) * 4 * (size_t)n_tris);
    memcpy(s->tri_area, vol, sizeof(double) * (size_t)n_tris);
    memcpy(s->tri_mat, mat_of_tri, sizeof(int) * (size_t)n_tris);
  }
  return ORC_OK;
}

int orc_set_pins(orc_sim* s, int n_pins, const int* ids, const double* v) {
  if (!s || n_pins < 0 || (n_pins > 0 && (!ids || !v))) return ORC_ERR_ARG;
  for (int j = 0; j < n_pins; ++j) {
    if (ids[j] < 0) return ORC_ERR_ARG;
    for (int k = 0; k < j; ++k)
      if (ids[k] == ids[j]) return ORC_ERR_ARG;
  }
  free(s->pin_ids); free(s->pin_v); free(s->pin_x0);
  const size_t np = (size_t)(n_pins > 0 ? n_pins : 1);
  s->n_pins = n_pins;
  s->pin_ids = (int*)malloc(sizeof(int) * np);
  s->pin_v = (double*)malloc(sizeof(double) * 3 * np);
  s->pin_x0 = (double*)malloc(sizeof(double) * 3 * np);
  if (n_pins > 0) {
    memcpy(s->pin_ids, ids, sizeof(int) * (size_t)n_pins);
    memcpy(s->pin_v, v, sizeof(double) * 3 * (size_t)n_pins);
  }
  return ORC_OK;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  free(s->pin_ids); free(s->pin_v); free(s->pin_x0);
  free(s->tris); free(s->tri_Dm_inv); free(s->tri_area); free(s->tri_mat); free(s->fext);
  free(s->m); free(s->p); free(s->v); free(s->dof); free(s->dof_node);
  free(s->con_p); free(s->con_b); free(s->con_gamma); free(s->con_phi0); free(s->con_n0);
  free(s);
}

static size_t node_id(const orc_grid* g, int ix, int iy, int iz) {
  return (size_t)ix + (size_t)g->res[0] * ((size_t)iy + (size_t)g->res[1] * (size_t)iz);
}

static int is_bc_node(const orc_grid* g, int ix, int iy, int iz) {
  int L = g->bc_layers;
  return ix < L || iy < L || iz < L || ix >= g->res[0] - L || iy >= g->res[1] - L ||
         iz >= g->res[2] - L;
}

static void kirchhoff_stress(const orc_material* mt, const double F[9], double tau[9]) {
  double mu, lam;
  orc_lame(mt->E, mt->nu, &mu, &lam);
  if (mt->model == ORC_CLOTH) {  /* the mesh carries the cloth's elasticity */
    for (int e = 0; e < 9; ++e) tau[e] = 0.0;
  } else if (mt->model == ORC_DRUCKER_PRAGER)
    orc_hencky_tau(F, mu, lam, tau);
  else
    orc_corotated_tau(F, mu, lam, tau);
}

/* P2G of particle q (MLS-MPM, Eq. (6)): its mass and its momentum with the
   affine and stress terms (and h times its mesh force, for cloth), scattered
   to the 27 nodes of its stencil. */
static void p2g_particle(orc_sim* s, int q, const double* x, const double* v, const double* C,
                         const double* F, const double* mass, const double* vol, const int* mat,
                         const orc_material* mats, double h, const double* fext) {
  const orc_grid* g = &s->g;
  const double dx = g->dx, Dinv = 4.0 / (dx * dx);
  int base[3];
  double fx[3], w[9], tau[9], aff[9];
  orc_bspline(dx, g->origin, x + 3 * q, base, fx, w);
  kirchhoff_stress(&mats[mat[q]], F + 9 * q, tau);
  for (int e = 0; e < 9; ++e) aff[e] = mass[q] * C[9 * q + e] - h * Dinv * vol[q] * tau[e];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) {
        double wt = w[a] * w[3 + b] * w[6 + c];
        double dpos[3] = {(a - fx[0]) * dx, (b - fx[1]) * dx, (c - fx[2]) * dx};
        size_t i = node_id(g, base[0] + a, base[1] + b, base[2] + c);
        s->m[i] += wt * mass[q];
        for (int r = 0; r < 3; ++r)
          s->p[3 * i + r] += wt * (mass[q] * v[3 * q + r] + aff[3 * r] * dpos[0] +
                                   aff[3 * r + 1] * dpos[1] + aff[3 * r + 2] * dpos[2] +
                                   (fext ? h * fext[3 * q + r] : 0.0));
      }
}

/* G2P of particle q with the constitutive update (Sec. V-A op (3)): velocity,
   affine matrix, position, deformation gradient, and for sand the
   Drucker-Prager return map. */
static void g2p_particle(const orc_sim* s, int q, double* x, double* v, double* C, double* F,
                         const int* mat, const orc_material* mats, double h) {
  const orc_grid* g = &s->g;
  const double dx = g->dx, Dinv = 4.0 / (dx * dx);
  int base[3];
  double fx[3], w[9];
  orc_bspline(dx, g->origin, x + 3 * q, base, fx, w);
  double vp[3] = {0, 0, 0}, Bm[9] = {0};
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c) {
        double wt = w[a] * w[3 + b] * w[6 + c];
        double dpos[3] = {(a - fx[0]) * dx, (b - fx[1]) * dx, (c - fx[2]) * dx};
        size_t i = node_id(g, base[0] + a, base[1] + b, base[2] + c);
        for (int r = 0; r < 3; ++r) {
          vp[r] += wt * s->v[3 * i + r];
          for (int cc = 0; cc < 3; ++cc) Bm[3 * r + cc] += wt * s->v[3 * i + r] * dpos[cc];
        }
      }
  for (int r = 0; r < 3; ++r) {
    v[3 * q + r] = vp[r];
    x[3 * q + r] += h * vp[r];
  }
  for (int e = 0; e < 9; ++e) C[9 * q + e] = Dinv * Bm[e];
  if (mats[mat[q]].model == ORC_CLOTH) return;  /* F stays I: no stress */
  double Fu[9];
  for (int e = 0; e < 9; ++e) Fu[e] = h * C[9 * q + e];
  Fu[0] += 1.0; Fu[4] += 1.0; Fu[8] += 1.0;
  mat_mul(Fu, F + 9 * q, F + 9 * q);
  const orc_material* mt = &mats[mat[q]];
  if (mt->model == ORC_DRUCKER_PRAGER) {
    double mu, lam;
    orc_lame(mt->E, mt->nu, &mu, &lam);
    orc_dp_project(F + 9 * q, mu, lam, mt->friction_angle_deg, F + 9 * q);
  }
}

#ifdef _OPENMP
/* Multi-threaded build (a CPU baseline over all host cores, not the checker):
   P2G over slabs of 4 nodes along the longest grid axis. A particle's stencil
   spans its base node and the next two, so particles of slabs two apart never
   touch the same node: the even slabs run in parallel, then the odd ones,
   each slab's particles in id order. Only the order in which a node sums its
   contributions differs from the serial build. */
static void p2g_slabs(orc_sim* s, int n, const double* x, const double* v, const double* C,
                      const double* F, const double* mass, const double* vol, const int* mat,
                      const orc_material* mats, double h, const double* fext) {
  const orc_grid* g = &s->g;
  int ax = 0;
  for (int a = 1; a < 3; ++a)
    if (g->res[a] > g->res[ax]) ax = a;
  const int n_slabs = (g->res[ax] + 3) / 4;
  int* slab = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
  int* start = (int*)calloc((size_t)n_slabs + 1, sizeof(int));
  int* order = (int*)malloc(sizeof(int) * (n > 0 ? n : 1));
#pragma omp parallel for schedule(static)
  for (int q = 0; q < n; ++q) {
    int base[3];
    double fx[3], w[9];
    orc_bspline(g->dx, g->origin, x + 3 * q, base, fx, w);
    slab[q] = base[ax] / 4;
  }
  for (int q = 0; q < n; ++q) start[slab[q] + 1] += 1;
  for (int k = 0; k < n_slabs; ++k) start[k + 1] += start[k];
  int* fill = (int*)malloc(sizeof(int) * ((size_t)n_slabs + 1));
  memcpy(fill, start, sizeof(int) * ((size_t)n_slabs + 1));
  for (int q = 0; q < n; ++q) order[fill[slab[q]]++] = q;
  for (int parity = 0; parity < 2; ++parity) {
#pragma omp parallel for schedule(dynamic, 1)
    for (int k = parity; k < n_slabs; k += 2)
      for (int t = start[k]; t < start[k + 1]; ++t)
        p2g_particle(s, order[t], x, v, C, F, mass, vol, mat, mats, h, fext);
  }
  free(slab); free(start); free(order); free(fill);
}
#endif

/* Contact records of one substep (Sec. V-B), grown by contacts_alloc. */
typedef struct {
  int cap;
  int *p, *b, *nodes;
  double *w, *R, *bias, *phi0, *n0, *mu, *k, *d;
} orc_contacts;

/* (Re)allocate the records for `cap` contacts, keeping the existing ones
   (K starts zeroed). */
static void contacts_alloc(orc_contacts* K, int cap) {
  K->cap = cap;
  K->p = (int*)realloc(K->p, sizeof(int) * cap);
  K->b = (int*)realloc(K->b, sizeof(int) * cap);
  K->nodes = (int*)realloc(K->nodes, sizeof(int) * 27 * cap);
  K->w = (double*)realloc(K->w, sizeof(double) * 27 * cap);
  K->R = (double*)realloc(K->R, sizeof(double) * 9 * cap);
  K->bias = (double*)realloc(K->bias, sizeof(double) * 3 * cap);
  K->phi0 = (double*)realloc(K->phi0, sizeof(double) * cap);
  K->n0 = (double*)realloc(K->n0, sizeof(double) * cap);
  K->mu = (double*)realloc(K->mu, sizeof(double) * cap);
  K->k = (double*)realloc(K->k, sizeof(double) * cap);
  K->d = (double*)realloc(K->d, sizeof(double) * cap);
}

/* Contact record slot of particle q inside body bd (phi < 0, outward normal
   nrm): stencil DoFs and weights, contact frame (z = n), bias
   b = -R^T v_rigid(x_p) so that v_c = R^T (v_particle - v_rigid), depth
   phi0 = -phi and the lagged normal impulse from the particle's
   start-of-substep relative normal velocity. */
static void register_contact(const orc_sim* s, orc_contacts* K, int slot, int q, int bi,
                             const orc_body* bd, double phi, const double nrm[3], const double* x,
                             const double* v, double h) {
  const orc_grid* g = &s->g;
  int base[3];
  double fx[3], w[9];
  orc_bspline(g->dx, g->origin, x + 3 * q, base, fx, w);
  int sidx = 0;
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      for (int c = 0; c < 3; ++c, ++sidx) {
        size_t i = node_id(g, base[0] + a, base[1] + b, base[2] + c);
        K->nodes[27 * slot + sidx] = s->dof[i];
        K->w[27 * slot + sidx] = w[a] * w[3 + b] * w[6 + c];
      }
  double* R = K->R + 9 * slot;
  orc_contact_frame(nrm, 0.0, R);
  double vr[3];
  orc_body_velocity(bd, x + 3 * q, vr);
  for (int c = 0; c < 3; ++c)
    K->bias[3 * slot + c] = -(R[c] * vr[0] + R[3 + c] * vr[1] + R[6 + c] * vr[2]);
  K->phi0[slot] = -phi;
  double vrel[3] = {v[3 * q] - vr[0], v[3 * q + 1] - vr[1], v[3 * q + 2] - vr[2]};
  double vn0 = dot3(nrm, vrel);
  K->n0[slot] = orc_normal_impulse(-phi, bd->k, bd->d, h, vn0);
  K->mu[slot] = bd->mu;
  K->k[slot] = bd->k;
  K->d[slot] = bd->d;
  K->p[slot] = q;
  K->b[slot] = bi;
}

int orc_substep(orc_sim* s, int n, double* x, double* v, double* C, double* F,
                const double* mass, const double* vol, const int* mat, int n_mat,
                const orc_material* mats, int nb, const orc_body* bodies, double h,
                const orc_solver* S, double* impulses, orc_substep_info* info) {
  const orc_grid* g = &s->g;
  const double dx = g->dx;
  orc_substep_info inf = {0};
  /* every stencil must lie inside the domain */
  for (int q = 0; q < n; ++q) {
    int base[3];
    double fx[3], w[9];
    orc_bspline(dx, g->origin, x + 3 * q, base, fx, w);
    for (int a = 0; a < 3; ++a)
      if (base[a] < 0 || base[a] + 2 > g->res[a] - 1) {
        inf.status = ORC_ERR_OUT_OF_DOMAIN;
        if (info) *info = inf;
        return inf.status;
      }
    if (mat[q] < 0 || mat[q] >= n_mat) {
      inf.status = ORC_ERR_ARG;
      if (info) *info = inf;
      return inf.status;
    }
  }
  /* pinned particles enter the substep on their prescribed motion */
  for (int j = 0; j < s->n_pins; ++j) {
    const int q = s->pin_ids[j];
    if (q >= n) {
      inf.status = ORC_ERR_ARG;
      if (info) *info = inf;
      return inf.status;
    }
    for (int r = 0; r < 3; ++r) {
      s->pin_x0[3 * j + r] = x[3 * q + r];
      v[3 * q + r] = s->pin_v[3 * j + r];
    }
    for (int r = 0; r < 9; ++r) C[9 * q + r] = 0.0;
  }
  memset(s->m, 0, s->nn * sizeof(double));
  memset(s->p, 0, 3 * s->nn * sizeof(double));

  /* cloth: the mesh forces at the substep's start positions */
  const double* fext = NULL;
  if (s->n_tris > 0) {
    if (s->fext_cap < n) {
      free(s->fext);
      s->fext = (double*)malloc(sizeof(double) * 3 * (size_t)n);
      s->fext_cap = n;
    }
    memset(s->fext, 0, sizeof(double) * 3 * (size_t)n);
    for (int t = 0; t < s->n_tris; ++t) {
      const int* v3 = s->tris + 3 * t;
      if (v3[0] < 0 || v3[0] >= n || v3[1] < 0 || v3[1] >= n || v3[2] < 0 || v3[2] >= n ||
          s->tri_mat[t] < 0 || s->tri_mat[t] >= n_mat) {
        inf.status = ORC_ERR_ARG;
        if (info) *info = inf;
        return inf.status;
      }
      double mu, lam, ft[9];
      orc_lame(mats[s->tri_mat[t]].E, mats[s->tri_mat[t]].nu, &mu, &lam);
      orc_cloth_triangle(x + 3 * v3[0], x + 3 * v3[1], x + 3 * v3[2], s->tri_Dm_inv + 4 * t,
                         s->tri_area[t], mu, lam, ft);
      for (int k = 0; k < 3; ++k)
        for (int r = 0; r < 3; ++r) s->fext[3 * v3[k] + r] += ft[3 * k + r];
    }
    /* a pinned vertex is held: the mesh does not push it */
    for (int j = 0; j < s->n_pins; ++j)
      for (int r = 0; r < 3; ++r) s->fext[3 * s->pin_ids[j] + r] = 0.0;
    fext = s->fext;
  }

  /* P2G (MLS-MPM): mass and momentum with the stress term, Eq. (6) */
#ifdef _OPENMP
  p2g_slabs(s, n, x, v, C, F, mass, vol, mat, mats, h, fext);
#else
  for (int q = 0; q < n; ++q) p2g_particle(s, q, x, v, C, F, mass, vol, mat, mats, h, fext);
#endif

  /* grid update: v* = p/m + h g; Dirichlet walls (reading: sticky, v = 0) */
  s->n_dof = 0;
  for (int iz = 0; iz < g->res[2]; ++iz)
    for (int iy = 0; iy < g->res[1]; ++iy)
      for (int ix = 0; ix < g->res[0]; ++ix) {
        size_t i = node_id(g, ix, iy, iz);
        if (s->m[i] > 0.0) {
          for (int r = 0; r < 3; ++r) s->p[3 * i + r] = s->p[3 * i + r] / s->m[i] + h * g->gravity[r];
          if (is_bc_node(g, ix, iy, iz))
            for (int r = 0; r < 3; ++r) s->p[3 * i + r] = 0.0;
          s->dof[i] = s->n_dof;
          s->dof_node[s->n_dof++] = (int)i;
        } else {
          s->dof[i] = -1;
        }
      }
  int nd = s->n_dof;
  inf.n_dofs = nd;
  double* dm = (double*)malloc(sizeof(double) * (nd + 1));
  double* dvs = (double*)malloc(sizeof(double) * 3 * (nd + 1));
  int* dfix = (int*)malloc(sizeof(int) * (nd + 1));
  for (int e = 0; e < nd; ++e) {
    size_t i = (size_t)s->dof_node[e];
    dm[e] = s->m[i];
    for (int r = 0; r < 3; ++r) dvs[3 * e + r] = s->p[3 * i + r];
    int ix = (int)(i % g->res[0]), iy = (int)((i / g->res[0]) % g->res[1]),
        iz = (int)(i / ((size_t)g->res[0] * g->res[1]));
    dfix[e] = is_bc_node(g, ix, iy, iz);
  }

  /* contact registration at the start of the substep (Sec. V-B): one contact
     per (particle, body) pair with the particle inside the body */
  orc_contacts K = {0};
  int nc = 0;
#ifdef _OPENMP
  /* count per particle, then fill in the serial order (particle-major, body
     order) at each particle's offset */
  int* first = (int*)calloc((size_t)n + 1, sizeof(int));
#pragma omp parallel for schedule(static)
  for (int q = 0; q < n; ++q) {
    int k = 0;
    for (int bi = 0; bi < nb; ++bi) {
      double nrm[3];
      if (orc_sdf(&bodies[bi], x + 3 * q, nrm) < 0.0) ++k;
    }
    first[q + 1] = k;
  }
  for (int q = 0; q < n; ++q) first[q + 1] += first[q];
  nc = first[n];
  contacts_alloc(&K, nc > 16 ? nc : 16);
#pragma omp parallel for schedule(static)
  for (int q = 0; q < n; ++q) {
    int k = first[q];
    for (int bi = 0; bi < nb; ++bi) {
      double nrm[3];
      double phi = orc_sdf(&bodies[bi], x + 3 * q, nrm);
      if (phi < 0.0) register_contact(s, &K, k++, q, bi, &bodies[bi], phi, nrm, x, v, h);
    }
  }
  free(first);
#else
  contacts_alloc(&K, 16);
  for (int q = 0; q < n; ++q) {
    for (int bi = 0; bi < nb; ++bi) {
      double nrm[3];
      double phi = orc_sdf(&bodies[bi], x + 3 * q, nrm);
      if (!(phi < 0.0)) continue;
      if (nc == K.cap) contacts_alloc(&K, 2 * K.cap);
      register_contact(s, &K, nc, q, bi, &bodies[bi], phi, nrm, x, v, h);
      ++nc;
    }
  }
#endif
  int *cp = K.p, *cb = K.b, *cn = K.nodes;
  double *cw = K.w, *cR = K.R, *cbias = K.bias, *cphi = K.phi0, *cn0 = K.n0, *cmu = K.mu,
         *ck = K.k, *cd = K.d;
  inf.n_contacts = nc;

  /* contact solve, Eq. (7)-(8) by Alg. 1, from v = v* */
  orc_problem P;
  P.n_nodes = nd; P.m = dm; P.vstar = dvs; P.fixed = dfix;
  P.n_contacts = nc; P.nodes = cn; P.w = cw; P.R = cR; P.b = cbias;
  P.phi0 = cphi; P.n0 = cn0; P.mu = cmu; P.k = ck; P.d = cd;
  P.h = h; P.eps_s = S->eps_s;
  double* vsol = (double*)malloc(sizeof(double) * 3 * (nd + 1));
  memcpy(vsol, dvs, sizeof(double) * 3 * nd);
  double* gam = (double*)malloc(sizeof(double) * 3 * (nc + 1));
  int st = ORC_OK;
  if (nc > 0) {
    orc_solve_info si;
    st = orc_solve_qn(&P, S, vsol, gam, &si, NULL);
    inf.iters = si.iters; inf.converged = si.converged;
    inf.G = si.G; inf.P = si.P; inf.J = si.J;
  } else {
    inf.converged = 1;
  }
  inf.status = st;

  /* impulses on the bodies, accumulated over the substeps (Eq. (3)) */
  if (s->con_cap < nc) {
    s->con_cap = nc;
    s->con_p = (int*)realloc(s->con_p, sizeof(int) * nc);
    s->con_b = (int*)realloc(s->con_b, sizeof(int) * nc);
    s->con_gamma = (double*)realloc(s->con_gamma, sizeof(double) * 3 * nc);
    s->con_phi0 = (double*)realloc(s->con_phi0, sizeof(double) * nc);
    s->con_n0 = (double*)realloc(s->con_n0, sizeof(double) * nc);
  }
  s->n_con = nc;
  for (int p = 0; p < nc; ++p) {
    const double* R = cR + 9 * p;
    double gw[3];
    for (int r = 0; r < 3; ++r)
      gw[r] = R[3 * r] * gam[3 * p] + R[3 * r + 1] * gam[3 * p + 1] + R[3 * r + 2] * gam[3 * p + 2];
    s->con_p[p] = cp[p];
    s->con_b[p] = cb[p];
    for (int r = 0; r < 3; ++r) s->con_gamma[3 * p + r] = gw[r];
    s->con_phi0[p] = cphi[p];
    s->con_n0[p] = cn0[p];
    if (impulses) {
      const orc_body* bd = &bodies[cb[p]];
      double arm[3] = {x[3 * cp[p]] - bd->p[0], x[3 * cp[p] + 1] - bd->p[1], x[3 * cp[p] + 2] - bd->p[2]};
      double on_body[3] = {-gw[0], -gw[1], -gw[2]}, mom[3];
      cross3(arm, on_body, mom);
      for (int r = 0; r < 3; ++r) {
        impulses[6 * cb[p] + r] += on_body[r];
        impulses[6 * cb[p] + 3 + r] += mom[r];
      }
    }
  }

  /* grid velocities after contact */
  memset(s->v, 0, 3 * s->nn * sizeof(double));
  for (int e = 0; e < nd; ++e)
    for (int r = 0; r < 3; ++r) s->v[3 * (size_t)s->dof_node[e] + r] = vsol[3 * e + r];

  /* G2P with the constitutive update (Sec. V-A op (3)) */
#ifdef _OPENMP
#pragma omp parallel for schedule(static)
#endif
  for (int q = 0; q < n; ++q) g2p_particle(s, q, x, v, C, F, mat, mats, h);

  /* pinned particles back on their prescribed path */
  for (int j = 0; j < s->n_pins; ++j) {
    const int q = s->pin_ids[j];
    for (int r = 0; r < 3; ++r) {
      x[3 * q + r] = s->pin_x0[3 * j + r] + h * s->pin_v[3 * j + r];
      v[3 * q + r] = s->pin_v[3 * j + r];
    }
    for (int r = 0; r < 9; ++r) C[9 * q + r] = 0.0;
  }

  free(dm); free(dvs); free(dfix); free(vsol); free(gam);
  free(cp); free(cb); free(cn); free(cw); free(cR); free(cbias); free(cphi); free(cn0);
  free(cmu); free(ck); free(cd);
  if (info) *info = inf;
  return inf.status == ORC_ERR_NOT_CONVERGED ? ORC_ERR_NOT_CONVERGED : inf.status;
}

int orc_last_grid(const orc_sim* s, int cap, int* ids, double* m, double* vstar, double* v) {
  int n = s->n_dof;
  for (int e = 0; e < n && e < cap; ++e) {
    size_t i = (size_t)s->dof_node[e];
    if (ids) ids[e] = (int)i;
    if (m) m[e] = s->m[i];
    for (int r = 0; r < 3; ++r) {
      if (vstar) vstar[3 * e + r] = s->p[3 * i + r];
      if (v) v[3 * e + r] = s->v[3 * i + r];
    }
  }
  return n;
}

int orc_last_contacts(const orc_sim* s, int cap, int* particle, int* body, double* gamma_world,
                      double* phi0, double* n0) {
  int n = s->n_con;
  for (int p = 0; p < n && p < cap; ++p) {
    if (particle) particle[p] = s->con_p[p];
    if (body) body[p] = s->con_b[p];
    for (int r = 0; r < 3; ++r)
      if (gamma_world) gamma_world[3 * p + r] = s->con_gamma[3 * p + r];
    if (phi0) phi0[p] = s->con_phi0[p];
    if (n0) n0[p] = s->con_n0[p];
  }
  return n;
}

/* rotation by angle |w| about w/|w| (Rodrigues) */
static void rotation_from_vector(const double w[3], double Q[9]) {
  double th = sqrt(dot3(w, w));
  for (int i = 0; i < 9; ++i) Q[i] = (i % 4 == 0) ? 1.0 : 0.0;
  if (th == 0.0) return;
  double a[3] = {w[0] / th, w[1] / th, w[2] / th};
  double c = cos(th), sn = sin(th), t = 1.0 - c;
  Q[0] = c + t * a[0] * a[0];
  Q[1] = t * a[0] * a[1] - sn * a[2];
  Q[2] = t * a[0] * a[2] + sn * a[1];
  Q[3] = t * a[1] * a[0] + sn * a[2];
  Q[4] = c + t * a[1] * a[1];
  Q[5] = t * a[1] * a[2] - sn * a[0];
  Q[6] = t * a[2] * a[0] - sn * a[1];
  Q[7] = t * a[2] * a[1] + sn * a[0];
  Q[8] = c + t * a[2] * a[2];
}

void orc_advance_kinematic(int nb, orc_body* bodies, double dt) {
  for (int b = 0; b < nb; ++b) {
    if (!bodies[b].kinematic) continue;
    for (int c = 0; c < 3; ++c) bodies[b].p[c] += dt * bodies[b].v[c];
    double wdt[3] = {dt * bodies[b].omega[0], dt * bodies[b].omega[1], dt * bodies[b].omega[2]};
    double Q[9];
    rotation_from_vector(wdt, Q);
    mat_mul(Q, bodies[b].R, bodies[b].R);
  }
}

void orc_rigid_dynamics_step(orc_body* b, const orc_dynamics* d, const double gravity[3],
                             const double impulse[6], double dt) {
  /* linear momentum */
  for (int c = 0; c < 3; ++c) {
    double f = d->force[c];
    if (d->gravity) f += d->mass * gravity[c];
    b->v[c] += (dt * f + impulse[c]) / d->mass;
  }
  /* angular momentum: I_w = R diag(I) R^T */
  double D[9] = {d->inertia[0], 0, 0, 0, d->inertia[1], 0, 0, 0, d->inertia[2]};
  double RD[9], Iw[9];
  mat_mul(b->R, D, RD);
  mat_mul_bt(RD, b->R, Iw);
  double Lw[3];
  for (int r = 0; r < 3; ++r)
    Lw[r] = Iw[3 * r] * b->omega[0] + Iw[3 * r + 1] * b->omega[1] + Iw[3 * r + 2] * b->omega[2];
  double gyro[3];
  cross3(b->omega, Lw, gyro);
  double rhs[3];
  for (int c = 0; c < 3; ++c) rhs[c] = dt * (d->torque[c] - gyro[c]) + impulse[3 + c];
  /* dw = I_w^-1 rhs with the adjugate: I_w^-1 = cof(I_w)^T / det (symmetric) */
  double K[9];
  mat_cofactor(Iw, K);
  const double det = mat_det(Iw);
  for (int r = 0; r < 3; ++r)
    b->omega[r] += (K[r] * rhs[0] + K[3 + r] * rhs[1] + K[6 + r] * rhs[2]) / det;
  for (int c = 0; c < 3; ++c) {
    if (!(d->dof_mask & (1 << c))) b->v[c] = 0.0;
    if (!(d->dof_mask & (1 << (3 + c)))) b->omega[c] = 0.0;
  }
  /* pose with the new velocity */
  for (int c = 0; c < 3; ++c) b->p[c] += dt * b->v[c];
  double wdt[3] = {dt * b->omega[0], dt * b->omega[1], dt * b->omega[2]};
  double Q[9];
  rotation_from_vector(wdt, Q);
  mat_mul(Q, b->R, b->R);
}

int orc_contact_adjoint(const orc_problem* P, const double* v, const double* vbar,
                        double* vstar_bar, double* b_bar, double* mu_bar) {
  const int n = P->n_nodes, nc = P->n_contacts, N3 = 3 * n;
  double* vc = (double*)malloc(sizeof(double) * 3 * (nc + 1));
  double* G = (double*)malloc(sizeof(double) * 9 * (nc + 1));    /* contact-frame Hessians */
  double* dg = (double*)malloc(sizeof(double) * 3 * (nc + 1));   /* d(grad l_c)/d mu */
  double* Hd = (double*)malloc(sizeof(double) * (size_t)N3 * N3 + 8);
  double* lam = (double*)malloc(sizeof(double) * (N3 + 1));
  double* jl = (double*)malloc(sizeof(double) * 3 * (nc + 1));
  contact_velocities(P, v, 1, vc);
  for (int p = 0; p < nc; ++p) {
    double gr[3], g1[3], g0[3], Hs[9];
    contact_l(P, p, vc + 3 * p, gr, G + 9 * p);
    /* the gradient is affine in mu: its mu-derivative is grad(mu=1) - grad(mu=0) */
    orc_contact_potential(P->phi0[p], P->n0[p], 1.0, P->k[p], P->d[p], P->h, P->eps_s, vc + 3 * p, g1, Hs);
    orc_contact_potential(P->phi0[p], P->n0[p], 0.0, P->k[p], P->d[p], P->h, P->eps_s, vc + 3 * p, g0, Hs);
    for (int c = 0; c < 3; ++c) dg[3 * p + c] = g1[c] - g0[c];
  }
  /* full Hessian on the free DoFs (Dirichlet rows and columns -> identity) */
  memset(Hd, 0, sizeof(double) * (size_t)N3 * N3);
  for (int i = 0; i < n; ++i)
    for (int c = 0; c < 3; ++c) Hd[(size_t)(3 * i + c) * N3 + 3 * i + c] = is_fixed(P, i) ? 1.0 : P->m[i];
  for (int p = 0; p < nc; ++p) {
    double RG[9], Gw[9];
    mat_mul(P->R + 9 * p, G + 9 * p, RG);
    mat_mul_bt(RG, P->R + 9 * p, Gw);
    for (int s = 0; s < 27; ++s) {
      int i = P->nodes[27 * p + s];
      if (i < 0 || is_fixed(P, i)) continue;
      for (int t = 0; t < 27; ++t) {
        int j = P->nodes[27 * p + t];
        if (j < 0 || is_fixed(P, j)) continue;
        double ww = P->w[27 * p + s] * P->w[27 * p + t];
        for (int r = 0; r < 3; ++r)
          for (int c = 0; c < 3; ++c) Hd[(size_t)(3 * i + r) * N3 + 3 * j + c] += ww * Gw[3 * r + c];
      }
    }
  }
  int status = ORC_OK;
  if (!dense_cholesky(Hd, N3)) {
    status = ORC_ERR_NOT_SPD;
  } else {
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c) lam[3 * i + c] = is_fixed(P, i) ? 0.0 : vbar[3 * i + c];
    dense_cholesky_solve(Hd, N3, lam);
    for (int i = 0; i < n; ++i)
      if (is_fixed(P, i)) for (int c = 0; c < 3; ++c) lam[3 * i + c] = 0.0;
    contact_velocities(P, lam, 0, jl); /* J lambda, contact frame */
    for (int i = 0; i < n; ++i)
      for (int c = 0; c < 3; ++c)
        vstar_bar[3 * i + c] = is_fixed(P, i) ? vbar[3 * i + c] : P->m[i] * lam[3 * i + c];
    for (int p = 0; p < nc; ++p) {
      const double* Gp = G + 9 * p;
      double gl[3];
      for (int r = 0; r < 3; ++r)
        gl[r] = Gp[3 * r] * jl[3 * p] + Gp[3 * r + 1] * jl[3 * p + 1] + Gp[3 * r + 2] * jl[3 * p + 2];
      for (int c = 0; c < 3; ++c) b_bar[3 * p + c] = -gl[c];
      mu_bar[p] = -(dg[3 * p] * jl[3 * p] + dg[3 * p + 1] * jl[3 * p + 1] + dg[3 * p + 2] * jl[3 * p + 2]);
      /* Dirichlet nodes in the stencil: - J_x^T (d2 l_c) J lambda */
      const double* R = P->R + 9 * p;
      double glw[3];
      for (int r = 0; r < 3; ++r) glw[r] = R[3 * r] * gl[0] + R[3 * r + 1] * gl[1] + R[3 * r + 2] * gl[2];
      for (int s2 = 0; s2 < 27; ++s2) {
        int i = P->nodes[27 * p + s2];
        if (i < 0 || !is_fixed(P, i)) continue;
        for (int c = 0; c < 3; ++c) vstar_bar[3 * i + c] -= P->w[27 * p + s2] * glw[c];
      }
    }
  }
  free(vc); free(G); free(dg); free(Hd); free(lam); free(jl);
  return status;
}

