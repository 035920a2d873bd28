// vine_tables.cu -- FP64 prologue kernels run once per batch:
//
//  * sPAM force-per-pressure tables, Sec. 3.1 Eq. (sPAM_1), (sPAM_2), (phiRC),
//    (sPAM_force): for each distinct cell length l0, 256 knots uniform in
//    actuator strain between eps(m_lo) and eps(m = 0.5); each knot is the
//    exact model at that strain.  Incomplete elliptic integrals by
//    Gauss-Legendre quadrature of their integrands (smooth for m <= 1/2);
//    the unsaturated root of Eq. (sPAM_2) by a coarse scan for the first sign
//    change followed by safeguarded Newton; m at each knot by the Illinois
//    variant of regula falsi.  One warp per knot: the scan points and the
//    quadrature nodes are spread over the lanes.  Branch rule: the smallest root in
//    (0, phi_sat], else the saturated branch phi = acos(R_c / R_act).
//  * the wrinkling energy table, Sec. 3.2 Eq. (wrinkling_model): the integral
//    of the restoring moment from onset to pi on 1024 cells, with the moment
//    itself at every knot, for cubic Hermite interpolation in the line search.
#include <cmath>

#include "vine_internal.cuh"

namespace vine {

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n.
void gauss_legendre(int n, GaussLegendre* gl) {
  gl->n = n;
  for (int i = 0; i < n; ++i) {
    double x = std::cos(kPiD * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = x;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (x * p1 - p0) / (x * x - 1.0);
      double dx = p1 / dp;
      x -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    gl->x[i] = x;
    gl->w[i] = 2.0 / ((1.0 - x * x) * dp * dp);
  }
}

namespace {

struct SpamConst {
  double Rc, Ract, a, m_lo, phi_sat;
};

// F(phi|m) and E(phi|m) by quadrature of (1 - m sin^2 t)^(-1/2) and its inverse.
__device__ void ellip_FE(const GaussLegendre& gl, double phi, double m, double* F, double* E) {
  double sf = 0.0, se = 0.0;
  const double hh = 0.5 * phi;
  for (int i = 0; i < gl.n; ++i) {
    double t = hh * (1.0 + gl.x[i]);
    double s = sin(t);
    double q = sqrt(1.0 - m * s * s);
    sf += gl.w[i] / q;
    se += gl.w[i] * q;
  }
  *F = hh * sf;
  *E = hh * se;
}

__device__ double ellip_F(const GaussLegendre& gl, double phi, double m) {
  double F, E;
  ellip_FE(gl, phi, m, &F, &E);
  return F;
}

// Residual of Eq. (sPAM_2) on the unsaturated branch (l_a = l_0), lam = l_0 / R_c,
// with the quadrature run by the calling thread alone.
__device__ double resid2(const GaussLegendre& gl, const SpamConst& c, double phi, double m, double lam) {
  if (phi <= 0.0) return -lam * (1.0 + c.a / (2.0 * m));
  double cp = cos(phi);
  return ellip_F(gl, phi, m) / (sqrt(m) * cp) - lam * (1.0 + c.a / (2.0 * m * cp * cp));
}

// The same quadrature of F(phi|m) and E(phi|m) spread over a warp: lane i
// takes node i, a butterfly sum, and lane 0's total broadcast so that every
// lane holds bit-identical values (the callers branch on them warp-uniformly).
__device__ void ellip_FE_warp(const GaussLegendre& gl, double phi, double m, int lane, double* F, double* E) {
  const double hh = 0.5 * phi;
  double sf = 0.0, se = 0.0;
  for (int i = lane; i < gl.n; i += 32) {
    const double t = hh * (1.0 + gl.x[i]);
    const double s = sin(t);
    const double q = sqrt(1.0 - m * s * s);
    sf += gl.w[i] / q;
    se += gl.w[i] * q;
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) {
    sf += __shfl_xor_sync(0xffffffffu, sf, d);
    se += __shfl_xor_sync(0xffffffffu, se, d);
  }
  *F = hh * __shfl_sync(0xffffffffu, sf, 0);
  *E = hh * __shfl_sync(0xffffffffu, se, 0);
}

// Model at contraction parameter m: strain eps and force per pressure f, by
// one warp (all lanes return the same values).  The first sign change of the
// residual on the 32-point scan of (0, phi_sat] is found with one scan point
// per lane.
__device__ void spam_model_warp(const GaussLegendre& gl, const SpamConst& c, double m, double l0, int lane,
                                double* eps, double* f, double* phi_out = nullptr, int* sat_out = nullptr) {
  const double lam = l0 / c.Rc;
  const int nscan = 32;
  const double ph_l = c.phi_sat * (double)(lane + 1) / nscan;
  const unsigned pos = __ballot_sync(0xffffffffu, resid2(gl, c, ph_l, m, lam) >= 0.0);
  double phi, la;
  const double sm = sqrt(m);
  if (pos != 0u) {
    const int kk = __ffs(pos) - 1;  // first scan point with a non-negative residual
    double hi = c.phi_sat * (double)(kk + 1) / nscan;
    double lo = kk == 0 ? 0.0 : c.phi_sat * (double)kk / nscan;
    // safeguarded Newton inside [lo, hi] (residual < 0 at lo, >= 0 at hi)
    double x = 0.5 * (lo + hi);
    for (int it = 0; it < 100; ++it) {
      double cp = cos(x), sp = sin(x);
      double F, E;
      ellip_FE_warp(gl, x, m, lane, &F, &E);
      double r = F / (sm * cp) - lam * (1.0 + c.a / (2.0 * m * cp * cp));
      if (r >= 0.0) hi = x; else lo = x;
      double dF = 1.0 / sqrt(1.0 - m * sp * sp);
      double dr = (dF * cp + F * sp) / (sm * cp * cp) - lam * c.a * sp / (m * cp * cp * cp);
      double xn = x - r / dr;
      if (!(xn > lo && xn < hi)) xn = 0.5 * (lo + hi);
      if (fabs(xn - x) <= 1e-16 * x || hi - lo <= 1e-16) {
        x = xn;
        break;
      }
      x = xn;
    }
    phi = x;
    la = l0;
  } else {
    phi = c.phi_sat;
    double cp = cos(phi);
    double F, E;
    ellip_FE_warp(gl, phi, m, lane, &F, &E);
    la = c.Rc * F / (sm * cp) / (1.0 + c.a / (2.0 * m * cp * cp));
  }
  double cp = cos(phi);
  double F, E;
  ellip_FE_warp(gl, phi, m, lane, &F, &E);
  // Eq. (sPAM_1) solved for the strain
  *eps = (la - 2.0 * c.Rc * (E - 0.5 * F) / (sm * cp)) / l0;
  // Eq. (sPAM_force) per unit actuation pressure
  *f = kPiD * c.Rc * c.Rc * (1.0 - 2.0 * m) / (2.0 * m * cp * cp);
  if (phi_out) *phi_out = phi;
  if (sat_out) *sat_out = pos != 0u ? 0 : 1;
}

// Samples of the exact model (training data of the surrogate): one warp per
// (m, l0): strain, phi_Rc, force per pressure and the branch.
__global__ void spam_samples_kernel(int n, const double* m, const double* l0, SpamConst c, GaussLegendre gl,
                                    double* eps, double* phi, double* f, int* sat) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (i >= n) return;  // whole warps leave together
  double e, ff, ph;
  int st;
  spam_model_warp(gl, c, m[i], l0[i], lane, &e, &ff, &ph, &st);
  if (lane == 0) {
    eps[i] = e;
    phi[i] = ph;
    f[i] = ff;
    sat[i] = st;
  }
}

// One warp per (table, knot): knots 1..254 by Illinois on eps(m) - target.
__global__ void spam_knots_kernel(const double* l0s, SpamConst c, GaussLegendre gl, const double* bounds,
                                  double* fknots) {
  const int t = blockIdx.y;
  const int lane = threadIdx.x & 31;
  const int k = 1 + blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (k > kKnots - 2) return;  // whole warps leave together
  const double l0 = l0s[t];
  const double elo = bounds[4 * t + 0], ehi = bounds[4 * t + 1];
  const double target = elo + (ehi - elo) * (double)k / (kKnots - 1);
  double a = c.m_lo, b = 0.5, fa = elo - target, fb = ehi - target;
  double m = a, e = 0.0, f = 0.0;
  int side = 0;
  for (int it = 0; it < 200; ++it) {
    m = (a * fb - b * fa) / (fb - fa);
    if (!(m > a && m < b)) m = 0.5 * (a + b);
    spam_model_warp(gl, c, m, l0, lane, &e, &f);
    double fm = e - target;
    if (fm == 0.0 || b - a <= 1e-15 * b) break;
    if ((fm < 0.0) == (fa < 0.0)) {
      a = m;
      fa = fm;
      if (side == -1) fb *= 0.5;
      side = -1;
    } else {
      b = m;
      fb = fm;
      if (side == 1) fa *= 0.5;
      side = 1;
    }
    if (fabs(fm) <= 1e-15 * (fabs(target) + 1e-3)) break;
  }
  if (lane == 0) fknots[t * kKnots + k] = f;
}

// One warp per table: eps at m_lo and m = 1/2 (the table's strain range).
__global__ void spam_bounds_kernel(const double* l0s, int n_tab, SpamConst c, GaussLegendre gl, double* bounds,
                                   double* fknots) {
  const int t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (t >= n_tab) return;
  double elo, flo, ehi, fhi;
  spam_model_warp(gl, c, c.m_lo, l0s[t], lane, &elo, &flo);
  spam_model_warp(gl, c, 0.5, l0s[t], lane, &ehi, &fhi);
  if (lane == 0) {
    bounds[4 * t + 0] = elo;
    bounds[4 * t + 1] = ehi;
    fknots[t * kKnots + 0] = flo;
    fknots[t * kKnots + kKnots - 1] = 0.0;
  }
}

// One thread per table: cumulative trapezoid integral from eps_lo (exact for
// the piecewise-linear interpolant), header and FP32 copies.
__global__ void spam_finish_kernel(int n_tab, const double* bounds, const double* fknots, float4* hdr, float2* tab) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n_tab) return;
  const double elo = bounds[4 * t + 0], ehi = bounds[4 * t + 1];
  const double h = (ehi - elo) / (kKnots - 1);
  const double* f = fknots + t * kKnots;
  double G = 0.0, G0 = 0.0;
  // G(0): integral from eps_lo to 0 (0 lies inside the range for l0 in use;
  // handled generally below)
  for (int k = 0; k < kKnots; ++k) {
    tab[t * kKnots + k] = make_float2((float)f[k], (float)G);
    if (k + 1 < kKnots) G += 0.5 * h * (f[k] + f[k + 1]);
  }
  if (0.0 <= elo) {
    G0 = f[0] * (0.0 - elo);
  } else if (0.0 >= ehi) {
    G0 = G;
  } else {
    double u = (0.0 - elo) / h;
    int k = (int)floor(u);
    if (k > kKnots - 2) k = kKnots - 2;
    double acc = 0.0;
    for (int q = 0; q < k; ++q) acc += 0.5 * h * (f[q] + f[q + 1]);
    double s = u - k;
    double fe = f[k] + s * (f[k + 1] - f[k]);
    acc += 0.5 * s * h * (f[k] + fe);
    G0 = acc;
  }
  hdr[t] = make_float4((float)elo, (float)h, (float)(1.0 / h), (float)G0);
}

// Wrinkling moment M / (pi P R^3) above onset, written through
// gamma_0 = 2 asin(sqrt(1 - eps_c / s)), s = sin(theta / 2).
__device__ double mhat_above(double th, double ec) {
  double s = sin(0.5 * fmin(th, kPiD));
  double g = 2.0 * asin(sqrt(1.0 - ec / s));
  return (sin(2.0 * g) + 2.0 * kPiD - 2.0 * g) / (4.0 * (sin(g) + (kPiD - g) * cos(g)));
}

// One thread per cell: integral of mhat over the cell (cells next to onset
// are split finer: the moment has a (theta - theta_c)^(3/2) term there) and
// mhat at the cell's left knot.
__global__ void wrinkle_cells_kernel(double ec, GaussLegendre gl, double* cells, double* knots) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k > kUCells) return;
  const double thc = 2.0 * asin(ec);
  const double h = (kPiD - thc) / kUCells;
  const double a = thc + h * k;
  knots[k] = (k == 0) ? 0.5 : mhat_above(fmin(a, kPiD), ec);
  if (k == kUCells) return;
  const int nsub = (k < 8) ? 64 : 1;
  double acc = 0.0;
  for (int q = 0; q < nsub; ++q) {
    double lo = a + h * q / nsub, hi = a + h * (q + 1) / nsub;
    if (k < 8) {  // geometric grading toward onset inside the first cells
      double r0 = (double)q / nsub, r1 = (double)(q + 1) / nsub;
      lo = a + h * r0 * r0;
      hi = a + h * r1 * r1;
    }
    double c = 0.5 * (lo + hi), w = 0.5 * (hi - lo), s = 0.0;
    for (int i = 0; i < gl.n; ++i) s += gl.w[i] * mhat_above(c + w * gl.x[i], ec);
    acc += w * s;
  }
  cells[k] = acc;
}

__global__ void wrinkle_finish_kernel(double ec, const double* cells, const double* knots, float2* utab,
                                      double* consts) {
  const double thc = 2.0 * asin(ec);
  double U = thc / 4.0;  // ramp part: integral of theta / (2 theta_c) up to theta_c
  for (int k = 0; k <= kUCells; ++k) {
    utab[k] = make_float2((float)U, (float)knots[k]);
    if (k < kUCells) U += cells[k];
  }
  consts[0] = U;  // integral up to pi
  consts[1] = knots[kUCells];
  consts[2] = thc;
  consts[3] = (kPiD - thc) / kUCells;
}

// ---- actuator design synthesis (Sec. 4.2) ----------------------------------
// Free-joint balance of a design (P, l0): h(theta) = pi P_v R^3 mhat(theta)
// - P f_l0(d theta / l_seg) d, with f_l0 the piecewise-linear force per
// pressure on the table's FP64 knots (its first knot below the strain range,
// zero beyond it).  h is increasing on (0, pi]: the equilibrium by bisection.
__device__ double synth_f(const double* bounds, const double* fk, int t, double eps) {
  const double elo = bounds[4 * t + 0], ehi = bounds[4 * t + 1];
  const double h = (ehi - elo) / (kKnots - 1);
  const double u = (eps - elo) / h;
  const double* f = fk + (size_t)t * kKnots;
  if (u <= 0.0) return f[0];
  if (u >= (double)(kKnots - 1)) return 0.0;
  const int k = (int)u;
  return f[k] + (u - k) * (f[k + 1] - f[k]);
}

__device__ double synth_mhat(double th, double ec) {
  const double thc = 2.0 * asin(ec);
  return th <= thc ? th / (2.0 * thc) : mhat_above(th, ec);
}

// One thread per (pressure, cell length): theta_eq, or pi when the actuator
// still wins at pi, or 0 when it cannot bend the joint at all.
__global__ void synth_pairs_kernel(int n_p, int n_l0, const double* pressures, const double* bounds,
                                   const double* fk, double R, double Pv, double ls, double R_act, double ec,
                                   double* theta_pair) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n_p * n_l0) return;
  const int ip = q / n_l0, il = q - ip * n_l0;
  const double P = pressures[ip], d = 2.0 * R + R_act, M0 = kPiD * Pv * R * R * R;
  auto h = [&](double th) { return M0 * synth_mhat(th, ec) - P * synth_f(bounds, fk, il, d * th / ls) * d; };
  double th;
  if (h(kPiD) <= 0.0) {
    th = kPiD;
  } else if (h(0.0) >= 0.0) {
    th = 0.0;
  } else {
    double lo = 0.0, hi = kPiD;
    for (int it = 0; it < 200 && hi - lo > 1e-15; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (h(mid) < 0.0) lo = mid; else hi = mid;
    }
    th = 0.5 * (lo + hi);
  }
  theta_pair[q] = th;
}

// One CTA per target: the feasible pair (|theta_eq - target| <= tol) of
// highest pressure, then closest angle, then shorter cell; a block-wide
// reduction over the pairs.
__global__ void synth_choose_kernel(int n_targets, const double* target, int n_p, int n_l0, const double* pressures,
                                    const double* theta_pair, double tol, int* p_index, int* l0_index,
                                    double* theta_eq) {
  __shared__ double kp[256], kd[256];
  __shared__ int kl[256], ki[256];
  const int t = blockIdx.x;
  if (t >= n_targets) return;
  const double tg = target[t];
  double bp = 0.0, bd = 0.0;
  int bl = 0, bi = -1;  // bi: pair index, -1 none
  for (int q = threadIdx.x; q < n_p * n_l0; q += blockDim.x) {
    const double dev = fabs(theta_pair[q] - tg);
    if (!(dev <= tol)) continue;
    const int ip = q / n_l0, il = q - ip * n_l0;
    const double P = pressures[ip];
    // key (-P, dev, il, ip), smaller is better
    const bool better = bi < 0 || P > bp || (P == bp && (dev < bd || (dev == bd && (il < bl ||
                        (il == bl && ip < bi / n_l0)))));
    if (better) {
      bp = P;
      bd = dev;
      bl = il;
      bi = q;
    }
  }
  kp[threadIdx.x] = bp;
  kd[threadIdx.x] = bd;
  kl[threadIdx.x] = bl;
  ki[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      const int o = threadIdx.x + w;
      const int ai = ki[threadIdx.x], oi = ki[o];
      bool take = false;
      if (oi >= 0) {
        if (ai < 0) take = true;
        else {
          const double ap = kp[threadIdx.x], op = kp[o], ad = kd[threadIdx.x], od = kd[o];
          const int al = kl[threadIdx.x], ol = kl[o];
          take = op > ap || (op == ap && (od < ad || (od == ad && (ol < al || (ol == al && oi / n_l0 < ai / n_l0)))));
        }
      }
      if (take) {
        kp[threadIdx.x] = kp[o];
        kd[threadIdx.x] = kd[o];
        kl[threadIdx.x] = kl[o];
        ki[threadIdx.x] = oi;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int q = ki[0];
    p_index[t] = q < 0 ? -1 : q / n_l0;
    l0_index[t] = q < 0 ? -1 : q % n_l0;
    theta_eq[t] = q < 0 ? __longlong_as_double(0x7ff8000000000000ll) : theta_pair[q];
  }
}

}  // namespace

cudaError_t launch_spam_tables(const double* l0, int n_tab, double R_c, double R_act, double a_spam, double m_lo,
                               const GaussLegendre& gl, float4* hdr, float2* tab, double* scratch,
                               cudaStream_t s) {
  if (n_tab <= 0) return cudaSuccess;
  SpamConst c{R_c, R_act, a_spam, m_lo, std::acos(R_c / R_act)};
  double* bounds = scratch;              // [4 n_tab]
  double* fk = scratch + 4 * n_tab;      // [n_tab * 256]
  spam_bounds_kernel<<<(n_tab + 3) / 4, 128, 0, s>>>(l0, n_tab, c, gl, bounds, fk);
  dim3 grid((kKnots - 2 + 3) / 4, n_tab);  // 4 warps per block, one knot each
  spam_knots_kernel<<<grid, 128, 0, s>>>(l0, c, gl, bounds, fk);
  spam_finish_kernel<<<(n_tab + 31) / 32, 32, 0, s>>>(n_tab, bounds, fk, hdr, tab);
  return cudaGetLastError();
}

cudaError_t launch_synth(int n_targets, const double* target, int n_p, int n_l0, const double* pressures,
                         const double* l0s, double R, double Pv, double ls, double tol, double R_c, double R_act,
                         double a_spam, double m_lo, double eps_c, const GaussLegendre& gl, double* scratch,
                         float4* hdr, float2* tab, double* theta_pair, int* p_index, int* l0_index,
                         double* theta_eq, int tables_ready, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (!tables_ready) e = launch_spam_tables(l0s, n_l0, R_c, R_act, a_spam, m_lo, gl, hdr, tab, scratch, s);
  if (e != cudaSuccess) return e;
  const double* bounds = scratch;
  const double* fk = scratch + 4 * n_l0;
  const int np = n_p * n_l0;
  synth_pairs_kernel<<<(np + 127) / 128, 128, 0, s>>>(n_p, n_l0, pressures, bounds, fk, R, Pv, ls, R_act, eps_c,
                                                      theta_pair);
  e = cudaGetLastError();
  if (e != cudaSuccess || n_targets == 0) return e;
  synth_choose_kernel<<<n_targets, 256, 0, s>>>(n_targets, target, n_p, n_l0, pressures, theta_pair, tol, p_index,
                                                l0_index, theta_eq);
  return cudaGetLastError();
}

cudaError_t launch_spam_samples(int n, const double* m, const double* l0, double R_c, double R_act, double a_spam,
                                const GaussLegendre& gl, double* eps, double* phi, double* f, int* sat,
                                cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  SpamConst c{R_c, R_act, a_spam, 0.0, std::acos(R_c / R_act)};
  spam_samples_kernel<<<(n + 3) / 4, 128, 0, s>>>(n, m, l0, c, gl, eps, phi, f, sat);
  return cudaGetLastError();
}

cudaError_t launch_wrinkle_table(double eps_c, const GaussLegendre& gl, float2* utab, double* scratch,
                                 double* consts, cudaStream_t s) {
  double* cells = scratch;               // [kUCells]
  double* knots = scratch + kUCells;     // [kUCells + 1]
  wrinkle_cells_kernel<<<(kUCells + 1 + 63) / 64, 64, 0, s>>>(eps_c, gl, cells, knots);
  wrinkle_finish_kernel<<<1, 1, 0, s>>>(eps_c, cells, knots, utab, consts);
  return cudaGetLastError();
}

}  // namespace vine

// ---------------------------------------------------------------------------
// Allocation-free variant of the sPAM table build.  The FP64 scratch lives in
// a file-scope device array; host code never uses the array's name as an
// address (it is a host-side stand-in), only the pointer that
// cudaGetSymbolAddress returns for the current device, fetched once per
// device on that device's first call.
// ---------------------------------------------------------------------------
#include <cstdint>
#include <mutex>

#include "vine.h"

namespace {

constexpr int kNoallocScratchDoubles = VINE_NOALLOC_MAX_TABLES * (4 + vine::kKnots);
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_table_scratch[kNoallocScratchDoubles];

std::mutex g_scratch_mu;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of the scratch array for the current device (set-up on the
// first call per device).  Returns cudaSuccess or the runtime's error.
cudaError_t scratch_for_current_device(double** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_ptr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_table_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" vine_status vine_spam_tables_noalloc(const double* l0, int32_t n_tab, const vine_params* params,
                                                float* hdr, float* knots, void* cuda_stream) {
  if (!l0 || !params || !hdr || !knots) {
    vine::set_last_error("vine_spam_tables_noalloc: null argument");
    return VINE_EINVAL;
  }
  if (n_tab < 1 || n_tab > VINE_NOALLOC_MAX_TABLES) {
    vine::set_last_error("vine_spam_tables_noalloc: n_tab must be 1..VINE_NOALLOC_MAX_TABLES (64)");
    return VINE_EINVAL;
  }
  if ((reinterpret_cast<uintptr_t>(hdr) & 15) != 0 || (reinterpret_cast<uintptr_t>(knots) & 7) != 0) {
    vine::set_last_error("vine_spam_tables_noalloc: hdr must be 16-byte and knots 8-byte aligned");
    return VINE_EINVAL;
  }
  const vine_params& p = *params;
  if (!(p.R_c > 0.0 && p.R_act > p.R_c) || !(p.m_lo > 0.0 && p.m_lo < 0.5) || !(p.a_spam >= 0.0)) {
    vine::set_last_error("vine_spam_tables_noalloc: parameter out of range");
    return VINE_EINVAL;
  }
  double* scratch = nullptr;
  cudaError_t e = scratch_for_current_device(&scratch);
  if (e == cudaSuccess) {
    vine::GaussLegendre gl;
    vine::gauss_legendre(24, &gl);
    // every scratch entry the kernels read is written earlier in the same
    // call, so nothing needs clearing between calls
    e = vine::launch_spam_tables(l0, n_tab, p.R_c, p.R_act, p.a_spam, p.m_lo, gl, reinterpret_cast<float4*>(hdr),
                                 reinterpret_cast<float2*>(knots), scratch, static_cast<cudaStream_t>(cuda_stream));
  }
  if (e != cudaSuccess) {
    vine::set_last_error("vine_spam_tables_noalloc: ", cudaGetErrorString(e));
    return VINE_ECUDA;
  }
  return VINE_OK;
}
