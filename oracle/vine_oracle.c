/*
 * vine_oracle.c -- FP64 CPU oracle for the quasi-static growth step of planar
 * vine robots, "Parallel Simulation of Contact and Actuation for Soft Growing
 * Robots" (arXiv 2509.15180).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, plain reference that the
 * CUDA path is checked against.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library, and includes nothing
 * from it.
 *
 * Everything is IEEE double precision, loops are written out, and each
 * function names the passage of the paper it follows:
 *   - sPAM actuator model ........ Sec. 3.1, Eq. (sPAM_1), (sPAM_2), (phiRC),
 *                                  (sPAM_force); a = 1e-4; R_c, R_act (Sec. 4.2)
 *   - wrinkling restoring moment . Sec. 3.2, Eq. (wrinkling_model), (gamma)
 *   - combined moment ............ Sec. 3.3, Eq. (restoring_moment)
 *   - rigid-link chain, growth ... Sec. 3.3 and Sec. 4.1 (minimal coordinates,
 *                                  only the distal length changes)
 *   - cost and weights ........... Sec. 4.1, Eq. (pbd), w_a=160, w_b=15, w_c=1
 *   - simulation step ............ Sec. 4.1, Algorithm 1, read as "the
 *                                  equilibrium reached from the warm start"
 *
 * Where the paper is silent or garbled the readings are the ones listed in
 * the project's design notes (potential energy form of the moment term, ramp
 * below wrinkling onset, strain-coupled actuator force, penalty contact on
 * discs, quadratic growth spring, displacement-based convergence test).
 *
 * Elliptic integrals use Carlson's symmetric forms R_F and R_D with the
 * duplication algorithm (B. C. Carlson, "Numerical computation of real or
 * complex elliptic integrals", Numer. Algorithms 10, 1995; series terms as in
 * DLMF 19.36.1-19.36.2).  The wrinkling energy integral uses adaptive
 * Gauss-Kronrod (7,15) quadrature (Kronrod 1965 nodes and weights).
 */
#include <math.h>
#include <stdio.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_NKNOT 256
#define ORC_PI 3.14159265358979323846264338327950288

/* ------------------------------------------------------------------------ */
/* Parameters (defaults follow Sec. 4.1 weights and Sec. 3.1 / 4.2 constants) */
/* ------------------------------------------------------------------------ */
typedef struct {
  double w_a, w_b, w_c;   /* Eq. (pbd) weights, Sec. 4.1 */
  double eps_crit;        /* critical wrinkling strain (fitted, value not printed) */
  double R_c, R_act;      /* sPAM constriction and tube radius, Sec. 4.2 */
  double a_spam;          /* empirical correction a = 1e-4, Sec. 3.1 */
  double m_lo;            /* lower end of the tabulated m range */
  double pen_frac;        /* contact stiffness: penetration (fraction of R) per unit moment */
  double tol;             /* convergence: predicted displacement / robot length ... */
  double fval_eps;        /* cost changes below fval_eps x (sum of |terms|) read as rounding level */
  double armijo_c1;       /* sufficient-decrease constant */
  int32_t max_iter;       /* Newton iterations per growth step */
  int32_t discs_per_link; /* contact discs per link (K_s) */
  int32_t max_halvings;   /* line-search halvings */
  int32_t exact_hessian;  /* 1: exact Hessian of J when positive definite, else Gauss-Newton; 0: Gauss-Newton */
  int32_t mode;           /* 0: equilibrium; 1: Algorithm 1 read literally (frozen actuator force, descent) */
  int32_t gd_steps;       /* mode 1: descent steps per growth step (Algorithm 1: 50) */
  double gd_alpha;        /* mode 1: step as a fraction of the free-space Newton step (see gd_solve) */
  double tol_link;        /* ... and predicted displacement / link length (when > 0) */
} orc_params;

void orc_params_default(orc_params* p) {
  p->w_a = 160.0; p->w_b = 15.0; p->w_c = 1.0;
  p->eps_crit = 0.01;
  p->R_c = 0.005; p->R_act = 0.01718; p->a_spam = 1e-4;
  p->m_lo = 0.002;
  p->pen_frac = 0.01;
  p->tol = 1e-6;
  p->fval_eps = 1e-13; /* FP64 rounding level of a sum of a few hundred terms */
  p->armijo_c1 = 1e-4;
  p->max_iter = 100;
  p->discs_per_link = 2;
  p->max_halvings = 30;
  p->exact_hessian = 1;
  p->mode = 0;
  p->gd_steps = 50;
  p->gd_alpha = 0.005;
  p->tol_link = 2.5e-5;
}

/* ------------------------------------------------------------------------ */
/* Elliptic integrals (Carlson 1995)                                         */
/* ------------------------------------------------------------------------ */
static double carlson_rf(double x, double y, double z) {
  for (int it = 0; it < 200; ++it) {
    double A = (x + y + z) / 3.0;
    double X = (A - x) / A, Y = (A - y) / A, Z = -(X + Y);
    double e = fmax(fabs(X), fmax(fabs(Y), fabs(Z)));
    if (e < 1e-3) {
      double E2 = X * Y - Z * Z, E3 = X * Y * Z;
      return (1.0 - E2 / 10.0 + E3 / 14.0 + E2 * E2 / 24.0 - 3.0 * E2 * E3 / 44.0) / sqrt(A);
    }
    double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
    double lam = sx * sy + sy * sz + sz * sx;
    x = 0.25 * (x + lam); y = 0.25 * (y + lam); z = 0.25 * (z + lam);
  }
  return NAN;
}

static double carlson_rd(double x, double y, double z) {
  double sum = 0.0, fac = 1.0;
  for (int it = 0; it < 200; ++it) {
    double A = (x + y + 3.0 * z) / 5.0;
    double X = (A - x) / A, Y = (A - y) / A, Z = -(X + Y) / 3.0;
    double e = fmax(fabs(X), fmax(fabs(Y), fabs(Z)));
    if (e < 1e-3) {
      double E2 = X * Y - 6.0 * Z * Z;
      double E3 = (3.0 * X * Y - 8.0 * Z * Z) * Z;
      double E4 = 3.0 * (X * Y - Z * Z) * Z * Z;
      double E5 = X * Y * Z * Z * Z;
      double ser = 1.0 - 3.0 * E2 / 14.0 + E3 / 6.0 + 9.0 * E2 * E2 / 88.0 - 3.0 * E4 / 22.0
                   - 9.0 * E2 * E3 / 52.0 + 3.0 * E5 / 26.0;
      return 3.0 * sum + fac * ser / (A * sqrt(A));
    }
    double sx = sqrt(x), sy = sqrt(y), sz = sqrt(z);
    double lam = sx * sy + sy * sz + sz * sx;
    sum += fac / (sz * (z + lam));
    fac *= 0.25;
    x = 0.25 * (x + lam); y = 0.25 * (y + lam); z = 0.25 * (z + lam);
  }
  return NAN;
}

/* Incomplete elliptic integral of the first kind F(phi | m), parameter m = k^2,
 * 0 <= phi <= pi/2, 0 <= m < 1 (the convention read for Sec. 3.1). */
double orc_ellip_F(double phi, double m) {
  double s = sin(phi), c = cos(phi);
  return s * carlson_rf(c * c, 1.0 - m * s * s, 1.0);
}

/* Incomplete elliptic integral of the second kind E(phi | m). */
double orc_ellip_E(double phi, double m) {
  double s = sin(phi), c = cos(phi);
  double q = 1.0 - m * s * s;
  return s * carlson_rf(c * c, q, 1.0) - (m / 3.0) * s * s * s * carlson_rd(c * c, q, 1.0);
}

/* ------------------------------------------------------------------------ */
/* sPAM model, Sec. 3.1                                                      */
/* ------------------------------------------------------------------------ */
/* Residual of Eq. (sPAM_2) with l_a = l_0 (unsaturated branch, PPAM reading):
 *   F(phi,m) / (sqrt(m) cos phi) - (l_0 / R_c) (1 + a / (2 m cos^2 phi)). */
static double spam2_unsat(const orc_params* p, double phi, double m, double l0) {
  double c = cos(phi);
  if (phi <= 0.0) return -(l0 / p->R_c) * (1.0 + p->a_spam / (2.0 * m));
  return orc_ellip_F(phi, m) / (sqrt(m) * c) - (l0 / p->R_c) * (1.0 + p->a_spam / (2.0 * m * c * c));
}

/* Evaluate the sPAM model at contraction parameter m for cell length l0.
 * Returns 0 on success.  eps: actuator strain, f: F_t / P_act (m^2),
 * phi: phi_Rc used, sat: 1 if the saturated branch applies.
 * Branch rule: take the smallest root of Eq. (sPAM_2) in (0, phi_sat]
 * (unsaturated, l_a = l_0); if there is none, phi = phi_sat from Eq. (phiRC)
 * and l_a follows from Eq. (sPAM_2) (saturated).  Strain from Eq. (sPAM_1),
 * force from Eq. (sPAM_force). */
int orc_spam_eval(const orc_params* p, double m, double l0, double* eps, double* f, double* phi_out,
                  int* sat_out) {
  const double phi_sat = acos(p->R_c / p->R_act);
  const int nscan = 32;
  double lo = 0.0, hlo = spam2_unsat(p, 0.0, m, l0), hi = -1.0;
  for (int k = 1; k <= nscan; ++k) {
    double ph = phi_sat * (double)k / nscan;
    double hv = spam2_unsat(p, ph, m, l0);
    if (hv >= 0.0) { hi = ph; break; }
    lo = ph; hlo = hv;
  }
  (void)hlo;
  double phi, la;
  int sat;
  if (hi > 0.0) {
    for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (spam2_unsat(p, mid, m, l0) >= 0.0) hi = mid; else lo = mid;
    }
    phi = 0.5 * (lo + hi);
    la = l0;
    sat = 0;
  } else {
    phi = phi_sat;
    double c = cos(phi);
    la = p->R_c * orc_ellip_F(phi, m) / (sqrt(m) * c) / (1.0 + p->a_spam / (2.0 * m * c * c));
    sat = 1;
  }
  double c = cos(phi);
  double Fv = orc_ellip_F(phi, m), Ev = orc_ellip_E(phi, m);
  /* Eq. (sPAM_1): (E - F/2)/(sqrt(m) cos phi) = l_a/(2 R_c) (1 - (l_0/l_a) eps) */
  double lhs1 = (Ev - 0.5 * Fv) / (sqrt(m) * c);
  *eps = (la - 2.0 * p->R_c * lhs1) / l0;
  /* Eq. (sPAM_force) divided by P_act */
  *f = ORC_PI * p->R_c * p->R_c * (1.0 - 2.0 * m) / (2.0 * m * c * c);
  if (phi_out) *phi_out = phi;
  if (sat_out) *sat_out = sat;
  return (isfinite(*eps) && isfinite(*f)) ? 0 : 1;
}

/* Force-per-pressure table on ORC_NKNOT uniform strain knots between
 * eps(m_lo) and eps(0.5); each knot value is the exact model at that strain,
 * with m found by bisection (eps(m) is increasing). */
typedef struct {
  double l0, eps_lo, eps_hi, h;
  double f[ORC_NKNOT];
} orc_table;

static double spam_eps_of_m(const orc_params* p, double m, double l0, double* f) {
  double e, fv;
  orc_spam_eval(p, m, l0, &e, &fv, NULL, NULL);
  if (f) *f = fv;
  return e;
}

int orc_spam_table(const orc_params* p, double l0, double* eps_lo, double* eps_hi, double* f) {
  double flo;
  double elo = spam_eps_of_m(p, p->m_lo, l0, &flo);
  double ehi = spam_eps_of_m(p, 0.5, l0, NULL);
  if (!(ehi > elo)) return 1;
  double h = (ehi - elo) / (ORC_NKNOT - 1);
  f[0] = flo;
  f[ORC_NKNOT - 1] = 0.0;
  for (int k = 1; k < ORC_NKNOT - 1; ++k) {
    double target = elo + h * k;
    double a = p->m_lo, b = 0.5;
    for (int it = 0; it < 200 && b - a > 1e-16; ++it) {
      double mid = 0.5 * (a + b);
      if (mid <= a || mid >= b) break;
      if (spam_eps_of_m(p, mid, l0, NULL) < target) a = mid; else b = mid;
    }
    double fv;
    spam_eps_of_m(p, 0.5 * (a + b), l0, &fv);
    f[k] = fv;
  }
  *eps_lo = elo;
  *eps_hi = ehi;
  return 0;
}

/* Piecewise-linear force interpolant: held at f(eps_lo) below the table,
 * zero at and beyond eps(m = 0.5) where (1 - 2m) vanishes. */
static void table_f(const orc_table* t, double e, double* f, double* fp) {
  if (e <= t->eps_lo) { *f = t->f[0]; *fp = 0.0; return; }
  if (e >= t->eps_hi) { *f = 0.0; *fp = 0.0; return; }
  double u = (e - t->eps_lo) / t->h;
  int k = (int)floor(u);
  if (k > ORC_NKNOT - 2) k = ORC_NKNOT - 2;
  if (k < 0) k = 0;
  double s = u - k;
  *f = t->f[k] + s * (t->f[k + 1] - t->f[k]);
  *fp = (t->f[k + 1] - t->f[k]) / t->h;
}

/* G(e) = integral of the interpolant from eps_lo to e (extended linearly
 * below eps_lo, constant above eps_hi), summed cell by cell. */
static double table_G(const orc_table* t, double e) {
  if (e <= t->eps_lo) return t->f[0] * (e - t->eps_lo);
  double acc = 0.0;
  for (int k = 0; k < ORC_NKNOT - 1; ++k) {
    double a = t->eps_lo + t->h * k, b = t->eps_lo + t->h * (k + 1);
    if (e >= b) {
      acc += 0.5 * t->h * (t->f[k] + t->f[k + 1]);
    } else {
      double s = (e - a) / t->h;
      double fe = t->f[k] + s * (t->f[k + 1] - t->f[k]);
      acc += 0.5 * (e - a) * (t->f[k] + fe);
      return acc;
    }
  }
  return acc;
}

/* Exported for the tests: value, slope and integral from 0 of the interpolant. */
void orc_table_eval(double eps_lo, double eps_hi, const double* fk, double e, double* f, double* fp,
                    double* Phi) {
  orc_table t;
  t.l0 = 0; t.eps_lo = eps_lo; t.eps_hi = eps_hi; t.h = (eps_hi - eps_lo) / (ORC_NKNOT - 1);
  memcpy(t.f, fk, sizeof(t.f));
  table_f(&t, e, f, fp);
  *Phi = table_G(&t, e) - table_G(&t, 0.0);
}

/* ------------------------------------------------------------------------ */
/* Wrinkling-based restoring moment, Sec. 3.2                                */
/* ------------------------------------------------------------------------ */
/* M / (pi P R^3).  Above onset (sin(|theta|/2) > eps_c) this is the printed
 * formula with gamma_0 = acos(2 eps_c / sin(theta/2) - 1); at or below onset
 * the moment ramps linearly from 0 to its onset value 1/2 (reading for the
 * regime where the acos argument exceeds 1).  Odd in theta; |theta| beyond pi
 * uses sin(pi/2). */
static double wr_mhat(double th, double ec) {
  double a = fabs(th);
  double thc = 2.0 * asin(ec);
  if (a <= thc) return th / (2.0 * thc);
  double s = sin(0.5 * fmin(a, ORC_PI));
  double g = acos(2.0 * ec / s - 1.0);
  double v = (sin(2.0 * g) + 2.0 * ORC_PI - 2.0 * g) / (4.0 * (sin(g) + (ORC_PI - g) * cos(g)));
  return th >= 0 ? v : -v;
}

/* d(M / pi P R^3)/d theta, chain rule through gamma_0(s), s = sin(theta/2). */
static double wr_mhat_d(double th, double ec) {
  double a = fabs(th);
  double thc = 2.0 * asin(ec);
  if (a <= thc) return 1.0 / (2.0 * thc);
  if (a >= ORC_PI) return 0.0;
  double s = sin(0.5 * a);
  double g = acos(2.0 * ec / s - 1.0);
  double N = sin(2.0 * g) + 2.0 * ORC_PI - 2.0 * g;
  double D = 4.0 * (sin(g) + (ORC_PI - g) * cos(g));
  double dN = 2.0 * cos(2.0 * g) - 2.0;
  double dD = -4.0 * (ORC_PI - g) * sin(g);
  double dv_dg = (dN * D - N * dD) / (D * D);
  double dg_ds = 2.0 * ec / (s * s * sin(g));
  double ds_dth = 0.5 * cos(0.5 * a);
  return dv_dg * dg_ds * ds_dth;
}

/* Adaptive Gauss-Kronrod (7,15) integration of wr_mhat over [a, b]. */
static const double gk_x[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                               0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                               0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                               0.207784955007898467600689403773245, 0.0};
static const double gk_wk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
static const double gk_wg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                                0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

static double gk15(double a, double b, double ec, double* err) {
  double c = 0.5 * (a + b), h = 0.5 * (b - a);
  double fc = wr_mhat(c, ec);
  double rk = gk_wk[7] * fc, rg = gk_wg[3] * fc;
  for (int i = 0; i < 7; ++i) {
    double f1 = wr_mhat(c - h * gk_x[i], ec), f2 = wr_mhat(c + h * gk_x[i], ec);
    rk += gk_wk[i] * (f1 + f2);
    if (i % 2 == 1) rg += gk_wg[i / 2] * (f1 + f2);
  }
  *err = fabs((rk - rg) * h);
  return rk * h;
}

/* Globally adaptive integration (QUADPACK style): keep at most 400
 * subintervals, always bisect the one with the largest Kronrod-Gauss error
 * estimate, stop when the summed estimate is below tol or at the noise level
 * of the integrand (the printed formula cancels as gamma_0 approaches pi,
 * leaving ~1e-13 relative noise). */
#define GK_MAXSEG 400
static double gk_adapt(double a0, double b0, double ec, double tol) {
  double sa[GK_MAXSEG], sb[GK_MAXSEG], sr[GK_MAXSEG], se[GK_MAXSEG];
  int n = 1;
  sa[0] = a0; sb[0] = b0; sr[0] = gk15(a0, b0, ec, &se[0]);
  for (;;) {
    double tot = 0.0, err = 0.0;
    int worst = 0;
    for (int k = 0; k < n; ++k) {
      tot += sr[k]; err += se[k];
      if (se[k] > se[worst]) worst = k;
    }
    if (err <= tol || err <= 1e-13 * fabs(tot) || n >= GK_MAXSEG) return tot;
    double m = 0.5 * (sa[worst] + sb[worst]);
    sa[n] = m; sb[n] = sb[worst];
    sr[n] = gk15(m, sb[worst], ec, &se[n]);
    sb[worst] = m;
    sr[worst] = gk15(sa[worst], m, ec, &se[worst]);
    ++n;
  }
}

/* Uhat(theta) = integral_0^theta M / (pi P R^3): closed form on the ramp,
 * quadrature above onset, linear beyond pi. */
static double wr_uhat(double th, double ec) {
  double a = fabs(th);
  double thc = 2.0 * asin(ec);
  if (a <= thc) return a * a / (4.0 * thc);
  double b = fmin(a, ORC_PI);
  double u = thc / 4.0 + gk_adapt(thc, b, ec, 1e-15);
  if (a > ORC_PI) u += wr_mhat(ORC_PI, ec) * (a - ORC_PI);
  return u;
}

void orc_wrinkle(double th, double ec, double* mhat, double* mhat_d, double* uhat) {
  if (mhat) *mhat = wr_mhat(th, ec);
  if (mhat_d) *mhat_d = wr_mhat_d(th, ec);
  if (uhat) *uhat = wr_uhat(th, ec);
}

/* ------------------------------------------------------------------------ */
/* Batch description (CSR, double precision copies of the caller's inputs)   */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n_inst;
  const int32_t* n_links;
  const double *l_seg, *radius, *pressure, *base; /* base: [n_inst*3] x, y, heading */
  const int32_t* act_ptr;
  const double *act_begin, *act_end;
  const int32_t* act_side;
  const double *act_pressure, *act_l0;
  const int32_t* obs_ptr;
  const int32_t* obs_kind; /* 0 circle (a = radius), 1 axis-aligned box (a, b half-sizes) */
  const double *obs_cx, *obs_cy, *obs_a, *obs_b;
} orc_batch;

typedef struct {
  int n_tab;
  orc_table* tab;
  int32_t* act_tab; /* per actuator: index into tab */
} orc_tables;

/* One table per distinct cell length l0 among the batch's actuators. */
orc_tables* orc_tables_create(const orc_params* p, const orc_batch* b) {
  int n_act = b->act_ptr[b->n_inst];
  orc_tables* T = (orc_tables*)calloc(1, sizeof(orc_tables));
  T->tab = (orc_table*)calloc(n_act > 0 ? n_act : 1, sizeof(orc_table));
  T->act_tab = (int32_t*)calloc(n_act > 0 ? n_act : 1, sizeof(int32_t));
  for (int a = 0; a < n_act; ++a) {
    double l0 = b->act_l0[a];
    int found = -1;
    for (int t = 0; t < T->n_tab; ++t)
      if (T->tab[t].l0 == l0) { found = t; break; }
    if (found < 0) {
      orc_table* t = &T->tab[T->n_tab];
      t->l0 = l0;
      if (orc_spam_table(p, l0, &t->eps_lo, &t->eps_hi, t->f) != 0) {
        free(T->tab); free(T->act_tab); free(T);
        return NULL;
      }
      t->h = (t->eps_hi - t->eps_lo) / (ORC_NKNOT - 1);
      found = T->n_tab++;
    }
    T->act_tab[a] = found;
  }
  return T;
}

void orc_tables_free(orc_tables* T) {
  if (!T) return;
  free(T->tab); free(T->act_tab); free(T);
}

int orc_tables_count(const orc_tables* T) { return T->n_tab; }

void orc_tables_get(const orc_tables* T, int t, double* l0, double* eps_lo, double* eps_hi, double* f) {
  *l0 = T->tab[t].l0; *eps_lo = T->tab[t].eps_lo; *eps_hi = T->tab[t].eps_hi;
  memcpy(f, T->tab[t].f, sizeof(double) * ORC_NKNOT);
}

/* ------------------------------------------------------------------------ */
/* Chain geometry, Sec. 3.3 / 4.1                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
  const orc_params* p;
  const orc_batch* b;
  const orc_tables* T;
  int i;                 /* instance index */
  double l_seg, R, P, d; /* d = 2 R + R_act: moment arm of Eq. (restoring_moment) */
  double kc, kg;         /* contact and growth stiffness */
  int a0, a1, o0, o1;
  const double* th_frozen; /* mode 1: joint angles at which the actuator strains are frozen (else NULL) */
  int fix_l;             /* 1: the distal length is held fixed (relaxation for tip-steering) */
} inst_t;

static void inst_init(inst_t* I, const orc_params* p, const orc_batch* b, const orc_tables* T, int i) {
  I->p = p; I->b = b; I->T = T; I->i = i;
  I->l_seg = b->l_seg[i]; I->R = b->radius[i]; I->P = b->pressure[i];
  I->d = 2.0 * I->R + p->R_act;
  /* contact stiffness: at penetration pen_frac * R a contact one link from a
   * joint carries w_a times the full wrinkling moment pi P R^3 */
  I->kc = p->w_a * ORC_PI * I->P * I->R * I->R * I->R / (2.0 * p->pen_frac * I->R * I->l_seg);
  /* growth spring: tip force at l = 0 equals the eversion force pi P R^2 */
  I->kg = ORC_PI * I->P * I->R * I->R / (2.0 * I->l_seg);
  I->a0 = b->act_ptr[i]; I->a1 = b->act_ptr[i + 1];
  I->o0 = b->obs_ptr[i]; I->o1 = b->obs_ptr[i + 1];
  I->th_frozen = NULL;
  I->fix_l = 0;
}

/* Link start points p[0..N], unit directions u[0..N-1], lengths L[0..N-1]:
 * psi_i = psi_b + sum_{j<=i} theta_j, L_i = l_seg except the distal l. */
static void chain_fk(const inst_t* I, int N, const double* th, double l, double* px, double* py, double* ux,
                     double* uy, double* L) {
  double psi = I->b->base[3 * I->i + 2];
  double x = I->b->base[3 * I->i + 0], y = I->b->base[3 * I->i + 1];
  for (int k = 0; k < N; ++k) {
    psi += th[k];
    L[k] = (k == N - 1) ? l : I->l_seg;
    ux[k] = cos(psi); uy[k] = sin(psi);
    px[k] = x; py[k] = y;
    x += L[k] * ux[k]; y += L[k] * uy[k];
  }
  px[N] = x; py[N] = y;
}

/* Signed distance from point (x, y) to obstacle o and its outward normal.
 * Circle: |x - c| - r.  Box: distance to an axis-aligned rectangle with
 * half-sizes (a, b), negative inside (nearest face; ties go to the x face).
 * A point exactly at a circle's centre takes the normal (tx, ty). */
static double obs_sdf_k(const orc_batch* b, int o, double x, double y, double tx, double ty, double* nx,
                        double* ny, double* kappa) {
  double dx = x - b->obs_cx[o], dy = y - b->obs_cy[o];
  *kappa = 0.0;
  if (b->obs_kind[o] == 0) {
    double dist = sqrt(dx * dx + dy * dy);
    if (dist > 0.0) { *nx = dx / dist; *ny = dy / dist; *kappa = 1.0 / dist; }
    else { *nx = tx; *ny = ty; }
    return dist - b->obs_a[o];
  }
  double sx = dx >= 0.0 ? 1.0 : -1.0, sy = dy >= 0.0 ? 1.0 : -1.0;
  double qx = fabs(dx) - b->obs_a[o], qy = fabs(dy) - b->obs_b[o];
  if (qx > 0.0 && qy > 0.0) {
    double dist = sqrt(qx * qx + qy * qy);
    *nx = sx * qx / dist; *ny = sy * qy / dist;
    *kappa = 1.0 / dist;
    return dist;
  }
  if (qx > 0.0) { *nx = sx; *ny = 0.0; return qx; }
  if (qy > 0.0) { *nx = 0.0; *ny = sy; return qy; }
  if (qx >= qy) { *nx = sx; *ny = 0.0; return qx; }
  *nx = 0.0; *ny = sy; return qy;
}

/* Signed distance, outward normal n, and kappa: the Hessian of the signed
 * distance is kappa (I - n n^T) (1/distance to the centre or corner; 0 on a
 * box face and inside a box). */
static double obs_sdf(const orc_batch* b, int o, double x, double y, double tx, double ty, double* nx,
                      double* ny) {
  double k;
  return obs_sdf_k(b, o, x, y, tx, ty, nx, ny, &k);
}

/* Coverage of joint/link j by actuator span [b, e) (link units). */
static double coverage(double bgn, double end, int j) {
  double lo = fmax(bgn, (double)j), hi = fmin(end, (double)(j + 1));
  return hi > lo ? hi - lo : 0.0;
}

typedef struct {
  double *px, *py, *ux, *uy, *L;
} geo_t;

static int geo_alloc(geo_t* G, int N) {
  G->px = (double*)malloc(sizeof(double) * (N + 1));
  G->py = (double*)malloc(sizeof(double) * (N + 1));
  G->ux = (double*)malloc(sizeof(double) * (N + 1));
  G->uy = (double*)malloc(sizeof(double) * (N + 1));
  G->L = (double*)malloc(sizeof(double) * (N + 1));
  return G->px && G->py && G->ux && G->uy && G->L;
}
static void geo_free(geo_t* G) { free(G->px); free(G->py); free(G->ux); free(G->uy); free(G->L); }

/* ------------------------------------------------------------------------ */
/* Energy J of Eq. (pbd) (potential form), its gradient and the Gauss-Newton */
/* Hessian.  Unknowns x = (theta_0..theta_{N-1}, l); n = N + 1.             */
/*   J = w_a sum_j U_j(theta_j) + w_b k_g (l_seg - l)^2 + w_c k_c sum pen^2   */
/*   U_j = pi P R^3 Uhat(theta_j) - sum_a c_aj P_a l_seg Phi_a(eps_aj)        */
/* with dU_j/dtheta_j = M_tot,j of Eq. (restoring_moment).                    */
/* ------------------------------------------------------------------------ */
/* Also returns, in *mag (if non-null), the magnitude scale of J: the sum of
 * the absolute values of its terms, each contact counted at w_c k_c
 * (pen^2 + 2 R pen).  Cost changes below fval_eps times this scale are read
 * as rounding level by the line search. */
static double energy_h(const inst_t* I, int N, const double* th, double l, double* g, double* H, geo_t* G,
                       double* mag, int exact) {
  const orc_params* p = I->p;
  const orc_batch* b = I->b;
  const int n = N + 1;
  const double PR3 = ORC_PI * I->P * I->R * I->R * I->R;
  chain_fk(I, N, th, l, G->px, G->py, G->ux, G->uy, G->L);
  if (g) for (int k = 0; k < n; ++k) g[k] = 0.0;
  if (H) for (int k = 0; k < n * n; ++k) H[k] = 0.0;
  double J = 0.0, S = 0.0;
  /* bending and actuation, per joint */
  for (int j = 0; j < N; ++j) {
    double M = PR3 * wr_mhat(th[j], p->eps_crit);
    double dM = PR3 * wr_mhat_d(th[j], p->eps_crit);
    double U = PR3 * wr_uhat(th[j], p->eps_crit);
    double Um = fabs(U);
    for (int a = I->a0; a < I->a1; ++a) {
      double c = coverage(b->act_begin[a], b->act_end[a], j);
      if (c <= 0.0) continue;
      double s = (double)b->act_side[a];
      double Pa = b->act_pressure[a];
      const orc_table* t = &I->T->tab[I->T->act_tab[a]];
      double f, fp;
      if (I->th_frozen) {
        /* Algorithm 1: the force is computed once, at the step's initial
         * strain, and held while the joint angle moves (linear potential) */
        const double e0 = s * I->d * I->th_frozen[j] / I->l_seg;
        table_f(t, e0, &f, &fp);
        M -= c * s * Pa * f * I->d;
        const double Ua = c * s * Pa * f * I->d * th[j];
        U -= Ua;
        Um += fabs(Ua);
        continue;
      }
      double e = s * I->d * th[j] / I->l_seg; /* Eq. (restoring_moment), strain */
      table_f(t, e, &f, &fp);
      M -= c * s * Pa * f * I->d;
      dM -= c * Pa * fp * I->d * I->d / I->l_seg;
      const double Ua = c * Pa * I->l_seg * (table_G(t, e) - table_G(t, 0.0));
      U -= Ua;
      Um += fabs(Ua);
    }
    J += p->w_a * U;
    S += p->w_a * Um;
    if (g) g[j] += p->w_a * M;
    if (H) H[j * n + j] += fmax(p->w_a * dM, 1e-6 * p->w_a * PR3);
  }
  /* growth */
  J += p->w_b * I->kg * (I->l_seg - l) * (I->l_seg - l);
  S += p->w_b * I->kg * (I->l_seg - l) * (I->l_seg - l);
  if (g) g[N] += -2.0 * p->w_b * I->kg * (I->l_seg - l);
  if (H) H[N * n + N] += 2.0 * p->w_b * I->kg;
  /* contact: every disc of every link against every obstacle */
  const int KS = p->discs_per_link;
  double* v = (g || H) ? (double*)malloc(sizeof(double) * n) : NULL;
  for (int i = 0; i < N; ++i) {
    for (int k = 1; k <= KS; ++k) {
      double fr = (double)k / KS;
      double x = G->px[i] + fr * G->L[i] * G->ux[i];
      double y = G->py[i] + fr * G->L[i] * G->uy[i];
      for (int o = I->o0; o < I->o1; ++o) {
        double nx, ny, kap_sd;
        double sd = obs_sdf_k(b, o, x, y, -G->uy[i], G->ux[i], &nx, &ny, &kap_sd);
        double pen = I->R - sd;
        if (!(pen > 0.0)) continue;
        J += p->w_c * I->kc * pen * pen;
        S += p->w_c * I->kc * (pen * pen + 2.0 * I->R * pen);
        if (!v) continue;
        /* v = d pen / d x: rotation about p_j moves the disc by z x (x - p_j) */
        for (int q = 0; q < n; ++q) v[q] = 0.0;
        for (int j = 0; j <= i; ++j) {
          double rx = x - G->px[j], ry = y - G->py[j];
          v[j] = -(rx * ny - ry * nx);
        }
        if (i == N - 1) v[N] = -fr * (nx * G->ux[i] + ny * G->uy[i]);
        double kap = 2.0 * p->w_c * I->kc;
        if (g) for (int q = 0; q < n; ++q) g[q] += kap * pen * v[q];
        if (H) {
          for (int r = 0; r < n; ++r) {
            if (v[r] == 0.0) continue;
            for (int c2 = 0; c2 < n; ++c2) H[r * n + c2] += kap * v[r] * v[c2];
          }
          if (exact) {
            /* pen times the second derivatives of pen:
             *   d2/dth_j dth_m = -t_j^T Hsd t_m + n.(x - p_max(j,m)),
             *   d2/dl dth_j    = -fr t_j^T Hsd u - fr n.(z x u),
             *   d2/dl^2        = -fr^2 u^T Hsd u,
             * with t_j = z x (x - p_j) and Hsd = kappa (I - n n^T). */
            const double ux = G->ux[i], uy = G->uy[i];
            const int last = (i == N - 1);
            for (int j = 0; j <= i; ++j) {
              double tjx = -(y - G->py[j]), tjy = x - G->px[j];
              double tjn = tjx * nx + tjy * ny;
              for (int m = 0; m <= i; ++m) {
                double tmx = -(y - G->py[m]), tmy = x - G->px[m];
                double tmn = tmx * nx + tmy * ny;
                double curv = kap_sd * ((tjx * tmx + tjy * tmy) - tjn * tmn);
                int q = j > m ? j : m;
                double geo = nx * (x - G->px[q]) + ny * (y - G->py[q]);
                H[j * n + m] += kap * pen * (-curv + geo);
              }
              if (last) {
                double un = ux * nx + uy * ny;
                double curv = kap_sd * ((tjx * ux + tjy * uy) - tjn * un);
                double zu_n = -uy * nx + ux * ny;
                double val = kap * pen * (-fr * curv - fr * zu_n);
                H[j * n + N] += val;
                H[N * n + j] += val;
              }
            }
            if (last) {
              double un = ux * nx + uy * ny;
              H[N * n + N] += kap * pen * (-fr * fr * kap_sd * (1.0 - un * un));
            }
          }
        }
      }
    }
  }
  free(v);
  if (mag) *mag = S;
  return J;
}

/* Energy with the Gauss-Newton matrix (contact second derivatives dropped). */
static double energy(const inst_t* I, int N, const double* th, double l, double* g, double* H, geo_t* G,
                     double* mag) {
  return energy_h(I, N, th, l, g, H, G, mag, 0);
}

/* Cholesky solve of the leading m x m block of H (row stride n). */
static int chol_solve(double* H, int n, int m, const double* rhs, double* x) {
  double* Lm = (double*)malloc(sizeof(double) * m * m);
  for (int r = 0; r < m; ++r)
    for (int c = 0; c < m; ++c) Lm[r * m + c] = H[r * n + c];
  for (int c = 0; c < m; ++c) {
    double s = Lm[c * m + c];
    for (int k = 0; k < c; ++k) s -= Lm[c * m + k] * Lm[c * m + k];
    if (!(s > 0.0)) { free(Lm); return 1; }
    double dlt = sqrt(s);
    Lm[c * m + c] = dlt;
    for (int r = c + 1; r < m; ++r) {
      double t = Lm[r * m + c];
      for (int k = 0; k < c; ++k) t -= Lm[r * m + k] * Lm[c * m + k];
      Lm[r * m + c] = t / dlt;
    }
  }
  for (int r = 0; r < m; ++r) {
    double t = rhs[r];
    for (int k = 0; k < r; ++k) t -= Lm[r * m + k] * x[k];
    x[r] = t / Lm[r * m + r];
  }
  for (int r = m - 1; r >= 0; --r) {
    double t = x[r];
    for (int k = r + 1; k < m; ++k) t -= Lm[k * m + r] * x[k];
    x[r] = t / Lm[r * m + r];
  }
  free(Lm);
  return 0;
}

/* Predicted displacement of the step dx, relative to the robot length N l_seg:
 * max over link end points of |sum_{j<=i} dtheta_j z x (p_{i+1} - p_j)| (plus
 * dl u for the distal end) and l_seg |dtheta_j|. */
static double step_residual(const inst_t* I, int N, const double* dx, const geo_t* G) {
  double best = 0.0;
  for (int i = 0; i < N; ++i) {
    double ddx = 0.0, ddy = 0.0;
    for (int j = 0; j <= i; ++j) {
      double rx = G->px[i + 1] - G->px[j], ry = G->py[i + 1] - G->py[j];
      ddx += -dx[j] * ry;
      ddy += dx[j] * rx;
    }
    if (i == N - 1) { ddx += dx[N] * G->ux[i]; ddy += dx[N] * G->uy[i]; }
    best = fmax(best, sqrt(ddx * ddx + ddy * ddy));
    best = fmax(best, I->l_seg * fabs(dx[i]));
  }
  return best / (N * I->l_seg);
}

enum { ORC_OK = 0, ORC_MAXITER = 1, ORC_NONFINITE = 2, ORC_BADINPUT = 3 };

/* Diagnostic trace of the solver iterations to stderr (off by default). */
static int g_trace = 0;
void orc_set_trace(int on) { g_trace = on; }

/* Equilibrium of the current chain from the warm start (theta, l): Newton
 * steps (exact Hessian of J when positive definite, else the Gauss-Newton
 * matrix), the bound 0 <= l <= l_seg handled as an active set,
 * backtracking line search (Armijo, or approximate Wolfe when the cost change
 * is at rounding level; a search with no acceptable trial ends the step as
 * not converged), stop when the predicted displacement is at most tol
 * (the final step is applied).  Algorithm 1 of Sec. 4.1 read as "the stationary point
 * of Eq. (pbd) reached from the warm start". */
static int solve_step(const inst_t* I, int N, double* th, double* l, int* iters_out, double* resid_out,
                      long long* evals_out) {
  const orc_params* p = I->p;
  const int n = N + 1;
  geo_t G;
  if (!geo_alloc(&G, N)) return ORC_NONFINITE;
  double* g = (double*)malloc(sizeof(double) * n);
  double* H = (double*)malloc(sizeof(double) * n * n);
  double* dx = (double*)malloc(sizeof(double) * n);
  double* rhs = (double*)malloc(sizeof(double) * n);
  double* tt = (double*)malloc(sizeof(double) * n);
  double* gt = (double*)malloc(sizeof(double) * n);
  double* Ht = (double*)malloc(sizeof(double) * n * n);
  double* Hs = (double*)malloc(sizeof(double) * n * n);
  int status = ORC_MAXITER, it = 0;
  double r = INFINITY;
  long long evals = 0;
  double Smag = 0.0, Smt = 0.0;
  /* converged when no link end point moves by more than tol of the robot's
   * length, nor by more than tol_link link lengths */
  const double tol_eff = p->tol_link > 0.0 ? fmin(p->tol, p->tol_link / N) : p->tol;
  double J = energy(I, N, th, *l, g, H, &G, &Smag);
  ++evals;
  for (it = 1; it <= p->max_iter; ++it) {
    if (!isfinite(J)) { status = ORC_NONFINITE; break; }
    int lfix = I->fix_l || (*l <= 0.0 && g[N] > 0.0) || (*l >= I->l_seg && g[N] < 0.0);
    int m = lfix ? N : n;
    for (int k = 0; k < m; ++k) rhs[k] = -g[k];
    /* Newton step with the exact Hessian of J when it is positive definite,
     * else with the Gauss-Newton matrix (always positive definite). */
    int solved = 0;
    if (p->exact_hessian) {
      energy_h(I, N, th, *l, NULL, Hs, &G, NULL, 1);
      solved = chol_solve(Hs, n, m, rhs, dx) == 0;
      chain_fk(I, N, th, *l, G.px, G.py, G.ux, G.uy, G.L);
    }
    if (!solved && chol_solve(H, n, m, rhs, dx) != 0) { status = ORC_NONFINITE; break; }
    if (lfix) dx[N] = 0.0;
    r = step_residual(I, N, dx, &G);
    if (!isfinite(r)) { status = ORC_NONFINITE; break; }
    if (r <= tol_eff) {
      for (int k = 0; k < N; ++k) th[k] += dx[k];
      *l = fmin(fmax(*l + dx[N], 0.0), I->l_seg);
      status = ORC_OK;
      break;
    }
    /* Line search on the projected path x(a) = P(x + a dx): Armijo on J, or,
     * when the cost change is at the rounding level of J, the approximate
     * Wolfe condition of Hager and Zhang (2005) on the directional slope. */
    double gd = 0.0;
    for (int k = 0; k < N; ++k) gd += g[k] * dx[k];
    const int l_moves = !((*l <= 0.0 && dx[N] < 0.0) || (*l >= I->l_seg && dx[N] > 0.0));
    const double slope0 = gd + (l_moves ? g[N] * dx[N] : 0.0);
    double alpha = 1.0, Jt = J, lt = *l;
    int hcount = 0, accepted = 0;
    for (int h = 0; h <= p->max_halvings; ++h, ++hcount) {
      for (int k = 0; k < N; ++k) tt[k] = th[k] + alpha * dx[k];
      lt = fmin(fmax(*l + alpha * dx[N], 0.0), I->l_seg);
      Jt = energy(I, N, tt, lt, gt, Ht, &G, &Smt);
      ++evals;
      const double dec = alpha * gd + g[N] * (lt - *l);
      if (Jt <= J + p->armijo_c1 * dec) { accepted = 1; break; }
      if (fabs(Jt - J) <= p->fval_eps * fmax(Smag, Smt)) {
        double st = 0.0;
        for (int k = 0; k < N; ++k) st += gt[k] * dx[k];
        if (lt > 0.0 && lt < I->l_seg) st += gt[N] * dx[N];
        if (st <= (2.0 * p->armijo_c1 - 1.0) * slope0) { accepted = 1; break; }
      }
      alpha *= 0.5;
    }
    /* no acceptable trial: the step ends here, not converged */
    if (!accepted) { status = ORC_MAXITER; break; }
    if (g_trace)
      fprintf(stderr, "it %3d r %.3e J %.9e alpha %.3g halvings %d l %.5f lfix %d gd %.3e\n", it, r, J, alpha,
              hcount, *l, lfix, gd);
    for (int k = 0; k < N; ++k) th[k] = tt[k];
    *l = lt;
    J = Jt;
    Smag = Smt;
    memcpy(g, gt, sizeof(double) * n);
    memcpy(H, Ht, sizeof(double) * n * n);
  }
  if (it > p->max_iter) it = p->max_iter;
  *iters_out = it;
  *resid_out = r;
  if (evals_out) *evals_out = evals;
  free(g); free(H); free(dx); free(rhs); free(tt); free(gt); free(Ht); free(Hs);
  geo_free(&G);
  return status;
}

/* ------------------------------------------------------------------------ */
/* Exported entry points                                                     */
/* ------------------------------------------------------------------------ */
double orc_energy(const orc_params* p, const orc_batch* b, const orc_tables* T, int i, int N, const double* th,
                  double l, double* g, double* H) {
  inst_t I;
  inst_init(&I, p, b, T, i);
  geo_t G;
  geo_alloc(&G, N);
  double J = energy(&I, N, th, l, g, H, &G, NULL);
  geo_free(&G);
  return J;
}

/* Cost, gradient and the exact Hessian of J (contact second derivatives included). */
double orc_energy_exact(const orc_params* p, const orc_batch* b, const orc_tables* T, int i, int N,
                        const double* th, double l, double* g, double* H) {
  inst_t I;
  inst_init(&I, p, b, T, i);
  geo_t G;
  geo_alloc(&G, N);
  double J = energy_h(&I, N, th, l, g, H, &G, NULL, 1);
  geo_free(&G);
  return J;
}

int orc_solve(const orc_params* p, const orc_batch* b, const orc_tables* T, int i, int N, double* th, double* l,
              int* iters, double* resid, int fix_l) {
  inst_t I;
  inst_init(&I, p, b, T, i);
  I.fix_l = fix_l ? 1 : 0;
  return solve_step(&I, N, th, l, iters, resid, NULL);
}

/* The solver's Newton step at the state (theta, l) without moving it: the step
 * dx[0..N] (dx[N] for l; 0 when the bound on l is active), its predicted
 * displacement residual, and the cost.  Returns 0 on success. */
int orc_gn_step(const orc_params* p, const orc_batch* b, const orc_tables* T, int i, int N, const double* th,
                double l, double* dx, double* resid, double* J, int* lfix_out, int fix_l) {
  inst_t I;
  inst_init(&I, p, b, T, i);
  const int n = N + 1;
  geo_t G;
  geo_alloc(&G, N);
  double* g = (double*)malloc(sizeof(double) * n);
  double* H = (double*)malloc(sizeof(double) * n * n);
  double* rhs = (double*)malloc(sizeof(double) * n);
  *J = energy(&I, N, th, l, g, H, &G, NULL);
  int lfix = fix_l || (l <= 0.0 && g[N] > 0.0) || (l >= I.l_seg && g[N] < 0.0);
  int m = lfix ? N : n;
  for (int k = 0; k < m; ++k) rhs[k] = -g[k];
  int rc = 1;
  if (p->exact_hessian) {
    double* He = (double*)malloc(sizeof(double) * n * n);
    energy_h(&I, N, th, l, NULL, He, &G, NULL, 1);
    rc = chol_solve(He, n, m, rhs, dx);
    free(He);
    chain_fk(&I, N, th, l, G.px, G.py, G.ux, G.uy, G.L);
  }
  if (rc != 0) rc = chol_solve(H, n, m, rhs, dx);
  if (lfix) dx[N] = 0.0;
  *resid = rc == 0 ? step_residual(&I, N, dx, &G) : NAN;
  *lfix_out = lfix;
  free(g); free(H); free(rhs);
  geo_free(&G);
  return rc;
}

/* Adjoint of the tip-distance cost at an equilibrium of the last growth
 * step (implicit differentiation, for the design optimisation of Sec. 5).
 * At the state x* = (theta, l) with grad J(x*) = 0:
 *   cost c = |p_N - goal|, p_N the distal end point;
 *   lambda solves H lambda = dc/dx on the free unknowns, H the exact Hessian
 *     of J, with l dropped when its bound is active (the solver's rule);
 *   dc/dq = -lambda . d(grad J)/dq for the pressure q = P_a and the span ends
 *     q = b_a, e_a of each actuator of the instance.
 * grad J depends on P_a and the span only through the actuator moment
 * c_aj s_a P_a f_a(eps_aj) d of Eq. (restoring_moment): linearly in P_a,
 * and through the coverage c_aj = |[j, j+1) n [b_a, e_a)| in the ends, whose
 * (right) derivatives are -1 on link floor(b_a) and +1 on link floor(e_a)
 * (links that exist only).  The earlier growth steps do not enter: every
 * link but the distal one has its fixed length l_seg, so J at the last step
 * depends on the design only through the terms above.
 * Outputs dP, dB, dE have one entry per actuator of instance i.  Returns 0,
 * or 1 when the exact Hessian is not positive definite at x* (no gradient;
 * outputs NaN). */
/* The adjoint part shared by the costs: lambda = H^-1 rhs (rhs = dc/dx),
 * then dc/dq = -lambda . d(grad J)/dq for each actuator's pressure, begin and
 * end.  H is the exact Hessian at (th, l); the distal length is dropped when
 * its bound is active.  Returns 0, or 1 when H is not positive definite
 * (outputs NaN). */
static int adjoint_design(const inst_t* I, const orc_batch* b, const orc_tables* T, int N, const double* th,
                          double l, const double* H, const double* g, double* rhs, double* dP, double* dB,
                          double* dE) {
  const orc_params* p = I->p;
  const int n = N + 1, na = I->a1 - I->a0;
  double* Hc = (double*)malloc(sizeof(double) * n * n);
  double* lam = (double*)malloc(sizeof(double) * n);
  memcpy(Hc, H, sizeof(double) * n * n);
  const int lfix = (l <= 0.0 && g[N] > 0.0) || (l >= I->l_seg && g[N] < 0.0);
  const int m = lfix ? N : n;
  int rc = N > 0 ? chol_solve(Hc, n, m, rhs, lam) : 0;
  if (lfix) lam[N] = 0.0;
  for (int a = 0; a < na; ++a) {
    dP[a] = dB[a] = dE[a] = rc ? NAN : 0.0;
    if (rc) continue;
    const int ga = I->a0 + a;
    const double bg = b->act_begin[ga], en = b->act_end[ga];
    const double s = (double)b->act_side[ga], Pa = b->act_pressure[ga];
    const orc_table* t = &T->tab[T->act_tab[ga]];
    const double jb = floor(bg), je = floor(en);
    for (int j = 0; j < N; ++j) {
      double f, fp;
      table_f(t, s * I->d * th[j] / I->l_seg, &f, &fp);
      /* d g_j / d P_a = -w_a c_aj s f d */
      dP[a] += lam[j] * p->w_a * coverage(bg, en, j) * s * f * I->d;
      if (bg < en && (double)j == jb) dB[a] -= lam[j] * p->w_a * s * Pa * f * I->d;
      if (bg < en && (double)j == je) dE[a] += lam[j] * p->w_a * s * Pa * f * I->d;
    }
  }
  free(Hc); free(lam);
  return rc ? 1 : 0;
}

int orc_grad(const orc_params* p, const orc_batch* b, const orc_tables* T, int i, int N, const double* th,
             double l, double gx, double gy, double* cost, double* dP, double* dB, double* dE) {
  inst_t I;
  inst_init(&I, p, b, T, i);
  const int n = N + 1;
  geo_t G;
  geo_alloc(&G, N);
  double* g = (double*)malloc(sizeof(double) * n);
  double* H = (double*)malloc(sizeof(double) * n * n);
  double* rhs = (double*)malloc(sizeof(double) * n);
  energy_h(&I, N, th, l, g, H, &G, NULL, 1);
  const double ex = G.px[N] - gx, ey = G.py[N] - gy;
  const double c = sqrt(ex * ex + ey * ey);
  *cost = c;
  const double sx = c > 0.0 ? ex / c : 0.0, sy = c > 0.0 ? ey / c : 0.0;
  /* dc/dtheta_j = s . (z x (p_N - p_j)), dc/dl = s . u_{N-1} */
  for (int j = 0; j < N; ++j) rhs[j] = -sx * (G.py[N] - G.py[j]) + sy * (G.px[N] - G.px[j]);
  rhs[N] = N > 0 ? sx * G.ux[N - 1] + sy * G.uy[N - 1] : 0.0;
  const int rc = adjoint_design(&I, b, T, N, th, l, H, g, rhs, dP, dB, dE);
  free(g); free(H); free(rhs);
  geo_free(&G);
  return rc;
}

/* Path cost: the mean squared distance of the link end points p_1..p_N to
 * target points q_1..q_N (a path the robot should follow, sampled at its
 * link ends), c = (1/N) sum_k |p_k - q_k|^2, and its adjoint derivatives as
 * orc_grad.  qx, qy: N targets each.
 *   dc/dtheta_j = (2/N) sum_{k > j} e_k . (z x (p_k - p_j)),  e_k = p_k - q_k
 *   dc/dl       = (2/N) e_N . u_{N-1}                                       */
int orc_grad_path(const orc_params* p, const orc_batch* b, const orc_tables* T, int i, int N, const double* th,
                  double l, const double* qx, const double* qy, double* cost, double* dP, double* dB, double* dE) {
  inst_t I;
  inst_init(&I, p, b, T, i);
  const int n = N + 1;
  geo_t G;
  geo_alloc(&G, N);
  double* g = (double*)malloc(sizeof(double) * n);
  double* H = (double*)malloc(sizeof(double) * n * n);
  double* rhs = (double*)malloc(sizeof(double) * n);
  energy_h(&I, N, th, l, g, H, &G, NULL, 1);
  double c = 0.0;
  for (int k = 1; k <= N; ++k) {
    const double ex = G.px[k] - qx[k - 1], ey = G.py[k] - qy[k - 1];
    c += ex * ex + ey * ey;
  }
  *cost = N > 0 ? c / N : 0.0;
  for (int j = 0; j < N; ++j) {
    double s = 0.0;
    for (int k = j + 1; k <= N; ++k) {
      const double ex = G.px[k] - qx[k - 1], ey = G.py[k] - qy[k - 1];
      s += -ex * (G.py[k] - G.py[j]) + ey * (G.px[k] - G.px[j]);
    }
    rhs[j] = 2.0 * s / N;
  }
  rhs[N] = N > 0 ? 2.0 * ((G.px[N] - qx[N - 1]) * G.ux[N - 1] + (G.py[N] - qy[N - 1]) * G.uy[N - 1]) / N : 0.0;
  const int rc = adjoint_design(&I, b, T, N, th, l, H, g, rhs, dP, dB, dE);
  free(g); free(H); free(rhs);
  geo_free(&G);
  return rc;
}

/* Link start points p_0..p_N and headings psi_0..psi_{N-1}. */
void orc_poses(const orc_params* p, const orc_batch* b, const orc_tables* T, int i, int N, const double* th,
               double l, double* px, double* py, double* psi) {
  inst_t I;
  inst_init(&I, p, b, T, i);
  geo_t G;
  geo_alloc(&G, N);
  chain_fk(&I, N, th, l, px, py, G.ux, G.uy, G.L);
  double a = b->base[3 * i + 2];
  for (int k = 0; k < N; ++k) { a += th[k]; psi[k] = a; }
  geo_free(&G);
}

/* gap[k * n_obs + o] = min over the discs of link k of (sd_o - R); a pair is
 * in contact when its gap is negative. */
void orc_gaps(const orc_params* p, const orc_batch* b, const orc_tables* T, int i, int N, const double* th,
              double l, double* gap) {
  inst_t I;
  inst_init(&I, p, b, T, i);
  geo_t G;
  geo_alloc(&G, N);
  chain_fk(&I, N, th, l, G.px, G.py, G.ux, G.uy, G.L);
  int no = I.o1 - I.o0;
  for (int k = 0; k < N; ++k) {
    for (int o = I.o0; o < I.o1; ++o) {
      double best = INFINITY;
      for (int q = 1; q <= p->discs_per_link; ++q) {
        double fr = (double)q / p->discs_per_link;
        double x = G.px[k] + fr * G.L[k] * G.ux[k], y = G.py[k] + fr * G.L[k] * G.uy[k];
        double nx, ny;
        double sd = obs_sdf(b, o, x, y, -G.uy[k], G.ux[k], &nx, &ny);
        best = fmin(best, sd - I.R);
      }
      gap[k * no + (o - I.o0)] = best;
    }
  }
  geo_free(&G);
}

/* Signed distance and normal of one obstacle (for the tests). */
double orc_sdf(const orc_batch* b, int o, double x, double y, double* nx, double* ny) {
  return obs_sdf(b, o, x, y, 1.0, 0.0, nx, ny);
}

/* Algorithm 1 of Sec. 4.1 read literally (mode 1): the actuator forces are
 * evaluated once from the strains at the step's initial state and held; then
 * gd_steps steps of gradient descent on J.  The paper's single learning rate
 * alpha is not printed and would mix units (rad per N m for the joint
 * angles, m per N for the distal length), so each unknown gets the step
 * gd_alpha / (its free-space stiffness): w_a pi P R^3 / (2 theta_c), the
 * slope of the moment ramp below wrinkling onset, for the joint angles and
 * 2 w_b k_g for the distal length, which is kept in [0, l_seg].  With
 * gd_alpha = 1 a lone unactuated joint below onset would reach its
 * equilibrium in one step.  No convergence test: the step ends after
 * gd_steps updates (status OK unless the state becomes non-finite). */
static int gd_solve(const inst_t* I0, int N, double* th, double* l) {
  const orc_params* p = I0->p;
  inst_t I = *I0;
  const int n = N + 1;
  double* th0 = (double*)malloc(sizeof(double) * n);
  double* g = (double*)malloc(sizeof(double) * n);
  geo_t G;
  geo_alloc(&G, N);
  memcpy(th0, th, sizeof(double) * N);
  I.th_frozen = th0;
  const double thc = 2.0 * asin(p->eps_crit);
  const double PR3 = ORC_PI * I.P * I.R * I.R * I.R;
  const double a_th = p->gd_alpha * 2.0 * thc / (p->w_a * PR3);
  const double a_l = p->gd_alpha / (2.0 * p->w_b * I.kg);
  int status = ORC_OK;
  for (int k = 0; k < p->gd_steps; ++k) {
    const double J = energy_h(&I, N, th, *l, g, NULL, &G, NULL, 0);
    if (!isfinite(J)) { status = ORC_NONFINITE; break; }
    for (int j = 0; j < N; ++j) th[j] -= a_th * g[j];
    if (!I.fix_l) *l = fmin(fmax(*l - a_l * g[N], 0.0), I.l_seg);
  }
  for (int j = 0; j < N && status == ORC_OK; ++j)
    if (!isfinite(th[j])) status = ORC_NONFINITE;
  free(th0); free(g);
  geo_free(&G);
  return status;
}

/* Grow every instance by up to n_steps links (one link per step, capped at
 * n_links) and solve each step to equilibrium.  State is in/out:
 * N_state[i] links present, theta_state (CSR by n_links), l_state.
 * Per instance: iterations summed, largest final residual, status (sticky
 * worst), robot-link-steps of converged steps, converged steps, energy
 * evaluations.  OpenMP over instances when n_threads > 1. */
/* Relaxation at the present links (supplement, tip-steering): every
 * instance with at least one link is solved again from its state with the
 * present actuators, no link added; with fix_l the distal length is held
 * fixed (growth stunted), else it stays free in [0, l_seg].  Counters and
 * status are updated as by a growth step. */
int orc_relax(const orc_params* p, const orc_batch* b, const orc_tables* T, int fix_l, int32_t* N_state,
              double* theta_state, double* l_state, int32_t* iters_total, double* resid_max, int32_t* status,
              int64_t* rls, int32_t* conv_steps, int64_t* evals, int n_threads) {
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (b->n_inst + 1));
  off[0] = 0;
  for (int i = 0; i < b->n_inst; ++i) off[i + 1] = off[i] + b->n_links[i];
#ifdef _OPENMP
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int i = 0; i < b->n_inst; ++i) {
    if (status[i] != ORC_OK || N_state[i] < 1) continue;  /* stopped robots stay stopped */
    inst_t I;
    inst_init(&I, p, b, T, i);
    I.fix_l = fix_l ? 1 : 0;
    const int N = N_state[i];
    double* th = theta_state + off[i];
    int it = 0;
    double r = 0.0;
    long long ev = 0;
    int st;
    if (p->mode == 1) {
      st = gd_solve(&I, N, th, &l_state[i]);
      it = p->gd_steps;
      ev = p->gd_steps;
    } else {
      st = solve_step(&I, N, th, &l_state[i], &it, &r, &ev);
    }
    iters_total[i] += it;
    evals[i] += ev;
    if (st == ORC_OK) {
      rls[i] += N;
      conv_steps[i] += 1;
    } else if (st > status[i]) {
      status[i] = st;
    }
    if (r > resid_max[i] || !isfinite(r)) resid_max[i] = r;
  }
  free(off);
  return 0;
}

int orc_run(const orc_params* p, const orc_batch* b, const orc_tables* T, int n_steps, int32_t* N_state,
            double* theta_state, double* l_state, int32_t* iters_total, double* resid_max, int32_t* status,
            int64_t* rls, int32_t* conv_steps, int64_t* evals, int n_threads) {
  int64_t* off = (int64_t*)malloc(sizeof(int64_t) * (b->n_inst + 1));
  off[0] = 0;
  for (int i = 0; i < b->n_inst; ++i) off[i + 1] = off[i] + b->n_links[i];
#ifdef _OPENMP
  if (n_threads < 1) n_threads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(n_threads)
#endif
  for (int i = 0; i < b->n_inst; ++i) {
    inst_t I;
    inst_init(&I, p, b, T, i);
    double* th = theta_state + off[i];
    for (int s = 0; s < n_steps; ++s) {
      /* a step that did not reach equilibrium (or became non-finite) ends the
       * robot's growth: the next step would start from a state that is not
       * an equilibrium of the model */
      if (status[i] != ORC_OK) break;
      int N = N_state[i];
      if (N >= b->n_links[i]) break;
      th[N] = 0.0;
      N += 1;
      N_state[i] = N;
      l_state[i] = 0.0;
      int it = 0;
      double r = 0.0;
      long long ev = 0;
      int st;
      if (p->mode == 1) {
        st = gd_solve(&I, N, th, &l_state[i]);
        it = p->gd_steps;
        ev = p->gd_steps;
      } else {
        st = solve_step(&I, N, th, &l_state[i], &it, &r, &ev);
      }
      iters_total[i] += it;
      evals[i] += ev;
      if (st == ORC_OK) {
        rls[i] += N;
        conv_steps[i] += 1;
      } else if (st > status[i]) {
        status[i] = st;
      }
      if (r > resid_max[i] || !isfinite(r)) resid_max[i] = r;
    }
  }
  free(off);
  return 0;
}

int orc_num_knots(void) { return ORC_NKNOT; }
