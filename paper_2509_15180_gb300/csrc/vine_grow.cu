// vine_grow.cu -- the growth step of Sec. 4.1 (Algorithm 1) for a batch of
// independent planar vine robots, one warp per robot.
//
// Per growth step (Sec. 3.3 / 4.1): a link is appended at the tip (joint
// angle 0, distal length 0; the previous distal link snaps to l_seg), then
// the cost of Eq. (pbd) in potential form
//     J = w_a sum_j U_j(theta_j) + w_b k_g (l_seg - l)^2 + w_c k_c sum pen^2
// is brought to its stationary point by damped Gauss-Newton:
//   eval  : heading and position prefix sums (float-float), per joint the
//           wrinkling moment (Eq. wrinkling_model) minus the sPAM moments
//           (Eq. restoring_moment with the strain-coupled force table), every
//           disc of every link against every obstacle (circle / box signed
//           distance), suffix sums of contact forces and moments -> gradient,
//           per-link 3x3 contact stiffness (planar twist coordinates).
//   solve : the Gauss-Newton system diag(d) + sum_links E_i^T C_i E_i, with
//           the distal length eliminated first, by a backward sweep of
//           articulated stiffnesses in link-local frames and a forward sweep
//           of twists -- exact for that matrix and O(N).
//   test  : predicted displacement of every link end (FP64 max / N l_seg).
//   step  : backtracking on the projected path: Armijo on J, or the
//           approximate Wolfe slope test when the cost change is at FP32
//           rounding level of J; no acceptable trial ends the step.
// Lanes own contiguous blocks of links; obstacles and actuators of the robot
// are staged in shared memory; the serial sweeps run warp-uniform.
#include <cmath>
#include <map>
#include <mutex>

#include "vine_internal.cuh"

namespace vine {
namespace {

constexpr unsigned kFull = 0xffffffffu;

struct FF {
  float hi, lo;
};

__device__ __forceinline__ FF two_sum(float a, float b) {
  float s = a + b;
  float bb = s - a;
  float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ FF quick_two_sum(float a, float b) {
  float s = a + b;
  float e = b - (s - a);
  return {s, e};
}
__device__ __forceinline__ FF ff_add(FF a, float b) {
  FF t = two_sum(a.hi, b);
  t.lo += a.lo;
  return quick_two_sum(t.hi, t.lo);
}
__device__ __forceinline__ FF ff_add(FF a, FF b) {
  FF t = two_sum(a.hi, b.hi);
  t.lo += a.lo + b.lo;
  return quick_two_sum(t.hi, t.lo);
}

// exact product of two floats, and a float-float value times a float
__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = a * b;
  return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ FF ff_mul(FF a, float b) {
  FF p = two_prod(a.hi, b);
  p.lo = fmaf(a.lo, b, p.lo);
  return quick_two_sum(p.hi, p.lo);
}

// Loops stay rolled (`unroll 1`) where unrolling buys nothing: the shuffle
// levels of the scans and sums below (inlined at many call sites), every
// loop over a rank's links (1-4 iterations at the team sizes used), the
// per-joint actuator loop, the broad-phase rebuild and the strided copies.
// The growth kernel's first stall was instruction fetch; the compiler's
// unrolling of these loops made up 39 KB of its 105 KB of text, and the
// rolled form takes 36 % off each evaluation with the same arithmetic.

// exclusive prefix (sum over lanes < lane) of float-float values
__device__ __forceinline__ FF warp_excl_scan(FF v, int lane) {
  FF x = v;
#pragma unroll 1
  for (int d = 1; d < 32; d <<= 1) {
    float h = __shfl_up_sync(kFull, x.hi, d);
    float l = __shfl_up_sync(kFull, x.lo, d);
    if (lane >= d) x = ff_add(FF{h, l}, x);
  }
  float h = __shfl_up_sync(kFull, x.hi, 1);
  float l = __shfl_up_sync(kFull, x.lo, 1);
  return lane == 0 ? FF{0.f, 0.f} : FF{h, l};
}

// exclusive suffix (sum over lanes > lane)
__device__ __forceinline__ float warp_excl_suffix(float v, int lane) {
  float x = v;
#pragma unroll 1
  for (int d = 1; d < 32; d <<= 1) {
    float o = __shfl_down_sync(kFull, x, d);
    if (lane + d < 32) x += o;
  }
  float o = __shfl_down_sync(kFull, x, 1);
  return lane == 31 ? 0.f : o;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v += __shfl_xor_sync(kFull, v, d);
  return v;
}

// A team of TP threads owns one robot: one warp (TP = 32, the default), or
// TP / 32 warps of one CTA (TP = 64 or 128), which split the link loops.
// The team operations below are the warp's own for TP = 32; for larger
// teams the warps' partial results meet in shared-memory scratch between CTA
// barriers and are combined in warp order.  Every branch around them depends
// only on team-uniform values (reductions, broadcasts, the robot's sizes),
// so all warps reach every barrier.
// Scratch layout (floats): FF scan totals [0, 8), suffix totals [8, 12),
// broadcasts [12, 14), sweep results [16, 20), float-float sums [20, 28),
// float sums [28, 32), int sums and counts [32, 36), maxima [36, 40), flags
// and second int sums [40, 44), second FF scan totals [48, 56), second
// suffix totals [56, 60).
constexpr int kTeamScratch = 64;

template <int TP>
struct Team {
  int r;       // rank in the team
  float* scr;  // S.TS
  static constexpr int W = TP / 32;
  __device__ __forceinline__ int lane() const { return r & 31; }
  __device__ __forceinline__ int warp() const { return r >> 5; }
  __device__ __forceinline__ void sync() const {
    if (TP == 32)
      __syncwarp();
    else
      __syncthreads();
  }
};

template <int TP>
__device__ __forceinline__ FF team_excl_scan(FF v, const Team<TP>& t) {
  FF x = warp_excl_scan(v, t.lane());
  if (TP == 32) return x;
  if (t.lane() == 31) {
    const FF inc = ff_add(x, v);  // this warp's total
    t.scr[2 * t.warp()] = inc.hi;
    t.scr[2 * t.warp() + 1] = inc.lo;
  }
  t.sync();
  FF below{0.f, 0.f};
  for (int w = 0; w < t.warp(); ++w) below = ff_add(below, FF{t.scr[2 * w], t.scr[2 * w + 1]});
  if (t.warp() > 0) x = ff_add(below, x);
  t.sync();
  return x;
}

// two exclusive prefixes at once: the arithmetic of two team_excl_scan
// calls, interleaved (independent chains), with one pair of barriers
template <int TP>
__device__ __forceinline__ void team_excl_scan2(FF& a, FF& b, const Team<TP>& t) {
  const FF va = a, vb = b;
  const int lane = t.lane();
  FF x = a, y = b;
#pragma unroll 1
  for (int d = 1; d < 32; d <<= 1) {
    const float xh = __shfl_up_sync(kFull, x.hi, d), xl = __shfl_up_sync(kFull, x.lo, d);
    const float yh = __shfl_up_sync(kFull, y.hi, d), yl = __shfl_up_sync(kFull, y.lo, d);
    if (lane >= d) {
      x = ff_add(FF{xh, xl}, x);
      y = ff_add(FF{yh, yl}, y);
    }
  }
  {
    const float xh = __shfl_up_sync(kFull, x.hi, 1), xl = __shfl_up_sync(kFull, x.lo, 1);
    const float yh = __shfl_up_sync(kFull, y.hi, 1), yl = __shfl_up_sync(kFull, y.lo, 1);
    a = lane == 0 ? FF{0.f, 0.f} : FF{xh, xl};
    b = lane == 0 ? FF{0.f, 0.f} : FF{yh, yl};
  }
  if (TP == 32) return;
  if (lane == 31) {
    const FF ia = ff_add(a, va), ib = ff_add(b, vb);  // the warp's totals
    t.scr[2 * t.warp()] = ia.hi;
    t.scr[2 * t.warp() + 1] = ia.lo;
    t.scr[48 + 2 * t.warp()] = ib.hi;
    t.scr[49 + 2 * t.warp()] = ib.lo;
  }
  t.sync();
  FF ba{0.f, 0.f}, bb{0.f, 0.f};
  for (int w = 0; w < t.warp(); ++w) {
    ba = ff_add(ba, FF{t.scr[2 * w], t.scr[2 * w + 1]});
    bb = ff_add(bb, FF{t.scr[48 + 2 * w], t.scr[49 + 2 * w]});
  }
  if (t.warp() > 0) {
    a = ff_add(ba, a);
    b = ff_add(bb, b);
  }
  t.sync();
}

template <int TP>
__device__ __forceinline__ float team_excl_suffix(float v, const Team<TP>& t) {
  float x = warp_excl_suffix(v, t.lane());
  if (TP == 32) return x;
  if (t.lane() == 0) t.scr[8 + t.warp()] = x + v;  // this warp's total
  t.sync();
  float above = 0.f;
  for (int w = Team<TP>::W - 1; w > t.warp(); --w) above += t.scr[8 + w];
  x += above;
  t.sync();
  return x;
}

// two exclusive suffixes at once: the arithmetic of two team_excl_suffix
// calls, interleaved, with one pair of barriers
template <int TP>
__device__ __forceinline__ void team_excl_suffix2(float& a, float& b, const Team<TP>& t) {
  const float va = a, vb = b;
  const int lane = t.lane();
  float x = a, y = b;
#pragma unroll 1
  for (int d = 1; d < 32; d <<= 1) {
    const float ox = __shfl_down_sync(kFull, x, d), oy = __shfl_down_sync(kFull, y, d);
    if (lane + d < 32) {
      x += ox;
      y += oy;
    }
  }
  {
    const float ox = __shfl_down_sync(kFull, x, 1), oy = __shfl_down_sync(kFull, y, 1);
    a = lane == 31 ? 0.f : ox;
    b = lane == 31 ? 0.f : oy;
  }
  if (TP == 32) return;
  if (lane == 0) {  // the warp's totals
    t.scr[8 + t.warp()] = a + va;
    t.scr[56 + t.warp()] = b + vb;
  }
  t.sync();
  float aa = 0.f, ab = 0.f;
  for (int w = Team<TP>::W - 1; w > t.warp(); --w) {
    aa += t.scr[8 + w];
    ab += t.scr[56 + w];
  }
  a += aa;
  b += ab;
  t.sync();
}

// float-float sum over the team: butterfly shuffles (every lane ends with
// the same value: two_sum's error term is exact, hence symmetric), then the
// warps' sums in warp order
template <int TP>
__device__ __forceinline__ FF team_sum_ff(FF v, const Team<TP>& t) {
#pragma unroll 1
  for (int d = 16; d > 0; d >>= 1) {
    const float h = __shfl_xor_sync(kFull, v.hi, d), l = __shfl_xor_sync(kFull, v.lo, d);
    v = ff_add(v, FF{h, l});
  }
  if (TP == 32) return v;
  if (t.lane() == 0) {
    t.scr[20 + 2 * t.warp()] = v.hi;
    t.scr[21 + 2 * t.warp()] = v.lo;
  }
  t.sync();
  FF s{t.scr[20], t.scr[21]};
  for (int w = 1; w < Team<TP>::W; ++w) s = ff_add(s, FF{t.scr[20 + 2 * w], t.scr[21 + 2 * w]});
  t.sync();
  return s;
}

// sum over the robot's links of a_j b_j (exact products, float-float sums)
template <int TP>
__device__ __forceinline__ FF team_dot(const float* a, const float* b, int j0, int j1, const Team<TP>& t) {
  FF s{0.f, 0.f};
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) s = ff_add(s, two_prod(a[j], b[j]));
  return team_sum_ff(s, t);
}

template <int TP>
__device__ __forceinline__ float team_max(float v, const Team<TP>& t) {
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(kFull, v, d));
  if (TP == 32) return v;
  if (t.lane() == 0) t.scr[36 + t.warp()] = v;
  t.sync();
  float m = t.scr[36];
  for (int w = 1; w < Team<TP>::W; ++w) m = fmaxf(m, t.scr[36 + w]);
  t.sync();
  return m;
}

template <int TP>
__device__ __forceinline__ bool team_any(bool b, const Team<TP>& t) {
  const bool wb = __any_sync(kFull, b);
  if (TP == 32) return wb;
  int* q = reinterpret_cast<int*>(t.scr + 40);
  if (t.lane() == 0) q[t.warp()] = wb ? 1 : 0;
  t.sync();
  int a = 0;
  for (int w = 0; w < Team<TP>::W; ++w) a |= q[w];
  t.sync();
  return a != 0;
}

// The closing reductions of an evaluation in one team operation: a float
// sum s, a float-float sum j, two integer sums i0 and i1, and the values bx,
// by of rank `owner` for every rank.  Each sum is a butterfly over the warp
// (the float-float one as in team_sum_ff), then the warps' partials in warp
// order; the four chains are interleaved and share one pair of barriers.
template <int TP>
__device__ __forceinline__ void team_close(float& s, FF& j, int& i0, int& i1, float& bx, float& by, int owner,
                                           const Team<TP>& t) {
#pragma unroll 1
  for (int d = 16; d > 0; d >>= 1) {
    s += __shfl_xor_sync(kFull, s, d);
    const float h = __shfl_xor_sync(kFull, j.hi, d), l = __shfl_xor_sync(kFull, j.lo, d);
    j = ff_add(j, FF{h, l});
    i0 += __shfl_xor_sync(kFull, i0, d);
    i1 += __shfl_xor_sync(kFull, i1, d);
  }
  if (TP == 32) {
    bx = __shfl_sync(kFull, bx, owner);
    by = __shfl_sync(kFull, by, owner);
    return;
  }
  int* q = reinterpret_cast<int*>(t.scr + 32);
  if (t.lane() == 0) {
    t.scr[28 + t.warp()] = s;
    t.scr[20 + 2 * t.warp()] = j.hi;
    t.scr[21 + 2 * t.warp()] = j.lo;
    q[t.warp()] = i0;
    q[8 + t.warp()] = i1;
  }
  if (t.r == owner) {
    t.scr[12] = bx;
    t.scr[13] = by;
  }
  t.sync();
  s = t.scr[28];
  j = FF{t.scr[20], t.scr[21]};
  for (int w = 1; w < Team<TP>::W; ++w) {
    s += t.scr[28 + w];
    j = ff_add(j, FF{t.scr[20 + 2 * w], t.scr[21 + 2 * w]});
  }
  i0 = 0;
  i1 = 0;
  for (int w = 0; w < Team<TP>::W; ++w) {
    i0 += q[w];
    i1 += q[8 + w];
  }
  bx = t.scr[12];
  by = t.scr[13];
  t.sync();
}

// exclusive prefix of integer counts over the ranks, and their total
template <int TP>
__device__ __forceinline__ int team_excl_scan_i(int v, int& total, const Team<TP>& t) {
  int off = v;
#pragma unroll
  for (int d = 1; d < 32; d <<= 1) {
    const int o = __shfl_up_sync(kFull, off, d);
    if (t.lane() >= d) off += o;
  }
  const int wt = __shfl_sync(kFull, off, 31);  // the warp's total
  off -= v;
  if (TP == 32) {
    total = wt;
    return off;
  }
  int* q = reinterpret_cast<int*>(t.scr + 32);
  if (t.lane() == 0) q[t.warp()] = wt;
  t.sync();
  total = 0;
  for (int w = 0; w < Team<TP>::W; ++w) {
    if (w < t.warp()) off += q[w];
    total += q[w];
  }
  t.sync();
  return off;
}

// Per-warp shared-memory slice.
struct Smem {
  float4* obs;
  float4* act;
  float *TH, *TH0, *DTH, *LUX, *LUY, *G, *DD, *C0, *C1, *C2, *C3, *C4, *C5, *FX, *FY, *TL;
  float* LX;  // distal-link couplings: g_l contact part, h_ll, q0, q1, q2
  int* Q;     // contact candidates of the link in progress, [kContactQueue][team threads]
  float* TS;  // team scratch (teams of several warps): kTeamScratch floats
  unsigned short* CL;  // per link: obstacle list near it, [count, index...] x (kListCap + 1)
  float* XB;           // per link: its end points when its list was built, [4]
  float* PB;           // per link: its start point at the current evaluation, [2]
  int* RQ;             // links whose lists are rebuilt in this evaluation
};

template <int TP>
__device__ __forceinline__ Smem carve(float* base, const GrowArgs& A) {
  Smem s;
  s.obs = reinterpret_cast<float4*>(base);
  s.act = s.obs + A.omax;
  float* p = reinterpret_cast<float*>(s.act + A.amax);
  const int n = A.nmax;
  s.TH = p; s.TH0 = p + n; s.DTH = p + 2 * n; s.LUX = p + 3 * n; s.LUY = p + 4 * n; s.G = p + 5 * n;
  s.DD = p + 6 * n; s.C0 = p + 7 * n; s.C1 = p + 8 * n; s.C2 = p + 9 * n; s.C3 = p + 10 * n; s.C4 = p + 11 * n;
  s.C5 = p + 12 * n; s.FX = p + 13 * n; s.FY = p + 14 * n; s.TL = p + 15 * n;
  s.LX = p + 16 * n;
  s.Q = reinterpret_cast<int*>(p + 16 * n + 8);
  s.TS = p + 16 * n + 8 + TP * kContactQueue;
  s.XB = s.TS + kTeamScratch;
  s.PB = s.XB + 4 * n;
  s.RQ = reinterpret_cast<int*>(s.PB + 2 * n);
  s.CL = reinterpret_cast<unsigned short*>(s.RQ + n);
  return s;
}

// The wrinkling moment of Sec. 3.2 written in p = pi - gamma_0, the angle of
// the unwrinkled arc's complement (sin^2(p/2) = eps_c / s, s = sin(|theta|/2)):
//   m = Nn / Dn,  Nn = 2p - sin 2p,  Dn = 4 (sin p - p cos p),
//   dm/dtheta = -4 eps_c cos(theta/2) F / (Dn^2 s^2),
//   F = 4 sin^2 p - p sin 2p - 2p^2  (= sin p Dn - p Nn).
// For a strongly bent joint p is small and all three are differences of
// nearly equal terms (Nn, Dn ~ p^3, F ~ p^6): their Taylor series are used
// below p = 1 (F: below 1.6), which keeps FP32 accuracy.
__device__ __forceinline__ void wrinkle_terms(float p, float& Nn, float& Dn, float& F) {
  const float p2 = p * p;
  float sp = 0.f, cp = 1.f;
  if (p >= 1.f) sincosf(p, &sp, &cp);  // one evaluation serves both closed forms
  if (p < 1.f) {
    const float x2 = 4.f * p2;
    Nn = 8.f * p2 * p *
         (1.6666666667e-1f + x2 * (-8.3333333333e-3f + x2 * (1.9841269841e-4f + x2 * (-2.7557319224e-6f +
         x2 * (2.5052108385e-8f + x2 * (-1.6059043837e-10f + x2 * 7.6471637318e-13f))))));
    Dn = 4.f * p2 * p *
         (3.3333333333e-1f + p2 * (-3.3333333333e-2f + p2 * (1.1904761905e-3f + p2 * (-2.2045855379e-5f +
         p2 * (2.5052108385e-7f + p2 * -1.9270852604e-9f)))));
  } else {
    Nn = 2.f * p - 2.f * sp * cp;
    Dn = 4.f * (sp - p * cp);
  }
  if (p < 1.6f) {
    const float x2 = 4.f * p2;
    const float x6 = x2 * x2 * x2;
    F = x6 * (-1.3888888889e-3f + x2 * (4.9603174603e-5f + x2 * (-8.2671957672e-7f + x2 * (8.3507027951e-9f +
        x2 * (-5.7353727989e-11f + x2 * (2.8676863994e-13f + x2 * (-1.0933444878e-15f + x2 * (3.2882540986e-18f +
        x2 * -8.0071122532e-21f))))))));
  } else {
    F = 4.f * sp * sp - 2.f * p * sp * cp - 2.f * p2;
  }
}

// Wrinkling restoring moment per unit pi P R^3 (Sec. 3.2): value m, slope dm
// and energy u = integral from 0.  At or below onset a linear ramp to 1/2;
// above onset the form of wrinkle_terms.
__device__ __forceinline__ void wrinkle(const GrowArgs& A, float th, float& m, float& dm, float& u) {
  const float a = fabsf(th);
  if (a <= A.theta_c) {
    m = th * A.inv2thc;
    dm = A.inv2thc;
    u = a * a * A.inv4thc;
    return;
  }
  const float ac = fminf(a, kPi);
  float s, cs;
  sincosf(0.5f * ac, &s, &cs);
  const float p = 2.f * asinf(sqrtf(fminf(A.eps_c / s, 1.f)));
  float Nn, Dn, F;
  wrinkle_terms(p, Nn, Dn, F);
  m = copysignf(Nn / Dn, th);
  dm = (a < kPi) ? -4.f * A.eps_c * cs * F / (Dn * Dn * s * s) : 0.f;
  if (a >= kPi) {
    u = A.U_pi + A.m_pi * (a - kPi);
  } else {
    float t = (a - A.theta_c) * A.u_invh;
    int k = min((int)t, kUCells - 1);
    float tau = t - (float)k;
    float2 p0 = A.utab[k], p1 = A.utab[k + 1];
    float t2 = tau * tau, t3 = t2 * tau;
    float h00 = 2.f * t3 - 3.f * t2 + 1.f, h10 = t3 - 2.f * t2 + tau, h01 = -2.f * t3 + 3.f * t2, h11 = t3 - t2;
    u = h00 * p0.x + h01 * p1.x + A.u_h * (h10 * p0.y + h11 * p1.y);
  }
}

// One active contact: force kap * pen * n on a disc at fraction fr of link j,
// accumulated into the link's shared-memory arrays (the link belongs to the
// calling lane; contacts are rare, so the accumulators need no registers).
// Gauss-Newton part kap w w^T of the link's 3x3 stiffness in twist
// coordinates about the link start, w = ((x - p) x n, n_x, n_y).  With EXACT
// (a runtime flag: one copy of the code serves both matrices)
// also pen times the second derivatives of pen: obstacle curvature
// -(kap pen kinv) s s^T, s = (n.(x - p), -n_y, n_x) (kinv = 1/distance to the
// circle centre or box corner, 0 on a box face), and the local part of the
// load stiffness fr Lu.F on the rotational entry; for the distal link the
// couplings with its length l.
__device__ __forceinline__ void add_contact(const Smem& S, int j, float pen, float nx, float ny, float kinv,
                                            float fr, float lx, float ly, float kap, bool last, float ulx,
                                            float uly, bool EXACT) {
  const float f = kap * pen;
  const float fx = f * nx, fy = f * ny;
  S.FX[j] += fx;
  S.FY[j] += fy;
  const float rx = fr * lx, ry = fr * ly;
  S.TL[j] += rx * fy - ry * fx;
  const float w0 = rx * ny - ry * nx;
  float c00 = kap * w0 * w0, c01 = kap * w0 * nx, c02 = kap * w0 * ny;
  float c11 = kap * nx * nx, c12 = kap * nx * ny, c22 = kap * ny * ny;
  float s0 = 0.f, cc = 0.f;
  if (EXACT) {
    s0 = nx * rx + ny * ry;
    cc = f * kinv;
    c00 -= cc * s0 * s0 - (rx * fx + ry * fy);
    c01 += cc * s0 * ny;
    c02 -= cc * s0 * nx;
    c11 -= cc * ny * ny;
    c12 += cc * ny * nx;
    c22 -= cc * nx * nx;
  }
  S.C0[j] += c00;
  S.C1[j] += c01;
  S.C2[j] += c02;
  S.C3[j] += c11;
  S.C4[j] += c12;
  S.C5[j] += c22;
  if (last) {
    const float vl = fr * (nx * ulx + ny * uly);
    float glc = fr * (fx * ulx + fy * uly), hll = kap * vl * vl;
    float q0 = kap * vl * w0, q1 = kap * vl * nx, q2 = kap * vl * ny;
    if (EXACT) {
      const float tu = nx * uly - ny * ulx;  // tangent (-n_y, n_x) . u
      hll -= cc * fr * fr * tu * tu;
      q0 -= cc * fr * tu * s0 + fr * (fy * ulx - fx * uly);
      q1 += cc * fr * tu * ny;
      q2 -= cc * fr * tu * nx;
    }
    S.LX[0] += glc;
    S.LX[1] += hll;
    S.LX[2] += q0;
    S.LX[3] += q1;
    S.LX[4] += q2;
  }
}

// Float-float square and square root (error-free products by FMA; one Newton
// correction of the FP32 root).
__device__ __forceinline__ FF ff_sq(FF a) {
  const float p = a.hi * a.hi;
  float e = fmaf(a.hi, a.hi, -p);
  e = fmaf(2.f * a.hi, a.lo, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ FF ff_sqrt(FF a) {
  const float s = sqrtf(a.hi);
  if (!(s > 0.f)) return {s, 0.f};
  const float r = fmaf(-s, s, a.hi) + a.lo;
  return quick_two_sum(s, r / (2.f * s));
}
__device__ __forceinline__ FF ff_neg(FF a) { return {-a.hi, -a.lo}; }

// Penetration of a disc of radius R centred at (x, y) (float-float, relative
// to the base) into obstacle ob, in float-float arithmetic, with the outward
// normal and the curvature kinv of the signed distance.  The plain FP32
// difference R + r - |x - c| loses ~5e-9 m to cancellation, a sizeable part
// of a shallow penetration (the contact force is proportional to it), so
// active contacts are resolved here.  May return pen <= 0 (not in contact).
__device__ __forceinline__ float disc_pen_precise(const float4 ob, FF x, FF y, float R, float fbx, float fby, float& nx,
                                  float& ny, float& kinv) {
  const FF dx = ff_add(two_sum(x.hi, -ob.x), x.lo), dy = ff_add(two_sum(y.hi, -ob.y), y.lo);
  if (ob.w < 0.f) {  // circle: ob.z = r
    const FF d = ff_sqrt(ff_add(ff_sq(dx), ff_sq(dy)));
    if (d.hi > 0.f) {
      const float id = 1.f / d.hi;
      nx = dx.hi * id;
      ny = dy.hi * id;
      kinv = id;
    } else {
      nx = fbx;
      ny = fby;
      kinv = 0.f;
    }
    return ff_add(two_sum(R, ob.z), ff_neg(d)).hi;
  }
  const float sx = dx.hi >= 0.f ? 1.f : -1.f, sy = dy.hi >= 0.f ? 1.f : -1.f;
  const FF ax = ff_add(dx.hi >= 0.f ? dx : ff_neg(dx), -ob.z);
  const FF ay = ff_add(dy.hi >= 0.f ? dy : ff_neg(dy), -ob.w);
  FF sd;
  kinv = 0.f;
  if (ax.hi > 0.f && ay.hi > 0.f) {
    sd = ff_sqrt(ff_add(ff_sq(ax), ff_sq(ay)));
    const float id = 1.f / sd.hi;
    nx = sx * ax.hi * id;
    ny = sy * ay.hi * id;
    kinv = id;
  } else if (ax.hi > 0.f) {
    sd = ax; nx = sx; ny = 0.f;
  } else if (ay.hi > 0.f) {
    sd = ay; nx = 0.f; ny = sy;
  } else if (ax.hi >= ay.hi) {
    sd = ax; nx = sx; ny = 0.f;
  } else {
    sd = ay; nx = 0.f; ny = sy;
  }
  return ff_add(FF{R, 0.f}, ff_neg(sd)).hi;
}

// Penetration in plain FP32 (error ~5e-9 m from rounding the offsets, the
// squared distance and R + r), with the outward normal and the curvature
// kinv of the signed distance.
__device__ __forceinline__ float disc_pen_fast(const float4 ob, FF x, FF y, float R, float fbx, float fby, float& nx,
                                               float& ny, float& kinv) {
  const float dx = (x.hi - ob.x) + x.lo, dy = (y.hi - ob.y) + y.lo;
  if (ob.w < 0.f) {  // circle: ob.z = r
    const float d = sqrtf(dx * dx + dy * dy);
    if (d > 0.f) {
      const float id = 1.f / d;
      nx = dx * id;
      ny = dy * id;
      kinv = id;
    } else {
      nx = fbx;
      ny = fby;
      kinv = 0.f;
    }
    return (R + ob.z) - d;
  }
  const float ax = fabsf(dx) - ob.z, ay = fabsf(dy) - ob.w;
  const float sx = dx >= 0.f ? 1.f : -1.f, sy = dy >= 0.f ? 1.f : -1.f;
  float sd;
  kinv = 0.f;
  if (ax > 0.f && ay > 0.f) {
    sd = sqrtf(ax * ax + ay * ay);
    const float id = 1.f / sd;
    nx = sx * ax * id;
    ny = sy * ay * id;
    kinv = id;
  } else if (ax > 0.f) {
    sd = ax; nx = sx; ny = 0.f;
  } else if (ay > 0.f) {
    sd = ay; nx = 0.f; ny = sy;
  } else if (ax >= ay) {
    sd = ax; nx = sx; ny = 0.f;
  } else {
    sd = ay; nx = 0.f; ny = sy;
  }
  return R - sd;
}

// FP32 pre-test of a disc (centre x, y as float-float relative to the base)
// against obstacle ob, with a small outward margin (circles: ob.w =
// -(R + r)^2 inflated by 2e-6 at encoding; boxes: Rpre = R (1 + 1e-6)), so
// that no pair with a positive penetration is missed.
__device__ __forceinline__ bool contact_candidate(const float4 ob, FF x, FF y, float Rpre) {
  const float dx = (x.hi - ob.x) + x.lo, dy = (y.hi - ob.y) + y.lo;
  if (ob.w < 0.f) return dx * dx + dy * dy < -ob.w;
  return fmaxf(fabsf(dx) - ob.z, fabsf(dy) - ob.w) < Rpre;
}

// Penetration of a disc (centre x, y as float-float relative to the base,
// radius R) into obstacle ob: an FP32 test with a small outward margin
// (circles: ob.w = -(R + r)^2 inflated by 2e-6 at encoding; boxes: Rpre =
// R (1 + 1e-6)), then the float-float evaluation for the pairs that pass.
// Returns pen > 0 with the outward normal and the curvature kinv of the
// signed distance when the disc overlaps the obstacle, else pen <= 0.
__device__ __forceinline__ float disc_pen(const float4 ob, FF x, FF y, float R, float Rpre, float fbx, float fby,
                                          float& nx, float& ny, float& kinv) {
  if (!contact_candidate(ob, x, y, Rpre)) return 0.f;
  return disc_pen_precise(ob, x, y, R, fbx, fby, nx, ny, kinv);
}

struct EvalOut {
  FF J;     // cost (float-float)
  float S;  // sum of the magnitudes of its terms (scale of the rounding-level test)
  float gl, hll, q0, q1, q2, ulx, uly;
  float kg_wb;  // growth stiffness w_b k_g (scale of the distal-length pivot)
  int tests;    // disc-obstacle pre-tests the warp ran
  unsigned sig; // signature of the active set: contacts (disc, obstacle) and joints past wrinkling onset
};

// Every link's obstacle list is marked stale (robot start, or a state the
// lists were not built for).
template <int TP>
__device__ __forceinline__ void reset_lists(const Smem& S, int n, const Team<TP>& tm) {
  #pragma unroll 1
  for (int j = tm.r; j < n; j += TP) S.CL[j * (kListCap + 1)] = kListStale;
  tm.sync();
}

// Broad phase.  Every link keeps the list of obstacles within margin R
// of its discs and its two end points at the time the list was built.  The
// discs lie on the segment between the end points, so while neither end
// point has moved by 0.8 of the margin no other obstacle can reach them.
// Each lane checks its links; the links that moved, have a stale list or are
// the distal link (whose length changes within the step) are queued, and the
// warp rebuilds their lists together, the lanes splitting the obstacles and
// a ballot keeping obstacle order.  More than kListCap near obstacles mark
// the link kListFull (it then tests every obstacle until it has moved like
// any other list).  ntest counts the pre-tests run (in obstacles).
template <int KS, int TP>
__device__ void rebuild_lists(const InstDev& I, const Smem& S, int N, int j0, int j1, FF px, FF py,
                              const Team<TP>& tm, float margin_r, int& ntest) {
  const int lane = tm.lane();
  const float margin = margin_r * I.R, mv = 0.64f * margin * margin;
  int nre = 0;
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) {
    const float x0 = px.hi, y0 = py.hi;
    px = ff_add(px, S.LUX[j]);
    py = ff_add(py, S.LUY[j]);
    S.PB[2 * j] = x0;
    S.PB[2 * j + 1] = y0;
    const int lb = j * (kListCap + 1);
    const unsigned short c = S.CL[lb];
    // a full list (more than kListCap near obstacles) makes the link test
    // every obstacle, which is right wherever it has moved to within the
    // margin; it is rebuilt, like any list, once the link has moved further
    bool stale = (j == N - 1) || c == kListStale;
    if (!stale) {
      const float* xb = S.XB + 4 * j;
      const float d0x = x0 - xb[0], d0y = y0 - xb[1], d1x = px.hi - xb[2], d1y = py.hi - xb[3];
      stale = !(d0x * d0x + d0y * d0y < mv && d1x * d1x + d1y * d1y < mv);
    }
    if (stale) {
      S.CL[lb] = kListStale;
      nre += 1;
    }
  }
  // queue the stale links in link order: exclusive prefix of the lanes' counts
  int total;
  int off = team_excl_scan_i(nre, total, tm);
  #pragma unroll 1
  for (int j = j0; j < j1 && nre > 0; ++j)
    if (S.CL[j * (kListCap + 1)] == kListStale) S.RQ[off++] = j;
  tm.sync();
  const float Rm = I.R + margin;
  const unsigned lt = (1u << lane) - 1u;
  #pragma unroll 1
  for (int q = 0; q < total; ++q) {
    const int j = S.RQ[q];
    const float x0 = S.PB[2 * j], y0 = S.PB[2 * j + 1], lx = S.LUX[j], ly = S.LUY[j];
    const int lb = j * (kListCap + 1);
    int cnt = 0;
    #pragma unroll 1
    for (int o0 = 0; o0 < I.n_obs; o0 += TP) {
      const int o = o0 + tm.r;
      bool near = false;
      if (o < I.n_obs) {
        const float4 ob = S.obs[o];
#pragma unroll
        for (int k = 0; k < KS; ++k) {
          const float fr = (float)(k + 1) / (float)KS;
          const float dx = (x0 + fr * lx) - ob.x, dy = (y0 + fr * ly) - ob.y;
          if (ob.w < 0.f) {
            const float rr = ob.z + Rm;
            near = near || (dx * dx + dy * dy < rr * rr);
          } else {
            near = near || (fmaxf(fabsf(dx) - ob.z, fabsf(dy) - ob.w) < Rm);
          }
        }
      }
      const unsigned bal = __ballot_sync(kFull, near);
      int before = 0, here = __popc(bal);  // near obstacles of the lower warps, and of the chunk
      if (TP > 32) {
        int* q = reinterpret_cast<int*>(tm.scr + 32);
        if (lane == 0) q[tm.warp()] = here;
        tm.sync();
        here = 0;
        for (int w = 0; w < Team<TP>::W; ++w) {
          if (w < tm.warp()) before += q[w];
          here += q[w];
        }
        tm.sync();
      }
      const int pos = cnt + before + __popc(bal & lt);
      if (near && pos < kListCap) S.CL[lb + 1 + pos] = (unsigned short)o;
      cnt += here;
    }
    if (tm.r == 0) {
      S.CL[lb] = cnt > kListCap ? kListFull : (unsigned short)cnt;
      float* xb = S.XB + 4 * j;
      xb[0] = x0;
      xb[1] = y0;
      xb[2] = x0 + lx;
      xb[3] = y0 + ly;
    }
  }
  if (tm.r == 0) ntest += total * I.n_obs;
  tm.sync();
}

// Cost, gradient and the Newton data at the state (TH[0..N), l): the exact
// Hessian when `exact`, else the Gauss-Newton matrix.
template <int KS, int TP>
__device__ EvalOut eval(const GrowArgs& A, const InstDev& I, const Smem& S, int N, float l, const Team<TP>& tm,
                        bool exact) {
  const int B = (N + TP - 1) / TP;
  const int j0 = min(tm.r * B, N), j1 = min(j0 + B, N);
  // headings psi_j = psi_b + sum_{i<=j} theta_i
  FF hs{0.f, 0.f};
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) hs = ff_add(hs, S.TH[j]);
  FF psi = ff_add(team_excl_scan(hs, tm), I.bpsi);
  FF sx{0.f, 0.f}, sy{0.f, 0.f};
  float ulx = 0.f, uly = 0.f;
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) {
    psi = ff_add(psi, S.TH[j]);
    float sn, cs;
    sincosf(psi.hi, &sn, &cs);
    const float ux = cs - sn * psi.lo, uy = sn + cs * psi.lo;
    const float L = (j == N - 1) ? l : I.l_seg;
    const float lx = L * ux, ly = L * uy;
    S.LUX[j] = lx;
    S.LUY[j] = ly;
    if (j == N - 1) {
      ulx = ux;
      uly = uy;
    }
    sx = ff_add(sx, lx);
    sy = ff_add(sy, ly);
  }
  // link start points relative to the base
  FF px = sx, py = sy;
  team_excl_scan2(px, py, tm);
  const float kap = 2.f * A.w_c * I.kc;
  const float floor_d = 1e-6f * A.w_a * I.PR3;
  int ntest = 0;
  unsigned sig = 0u;  // order-independent: a sum of per-item codes
  if (A.broad) rebuild_lists<KS, TP>(I, S, N, j0, j1, px, py, tm, A.list_margin, ntest);
  // cost terms summed per lane in float-float (each term is an FP32 value;
  // the sum keeps ~48 bits, far below the rounding-level test on J), their
  // magnitudes in FP32 (only a scale for that test): GB300's FP64 rate is low
  FF Jl{0.f, 0.f};
  float Sl = 0.f;
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) {
    // ---- bending and actuation at joint j (Eq. restoring_moment)
    const float th = S.TH[j];
    float m, dm, u;
    wrinkle(A, th, m, dm, u);
    float M = I.PR3 * m, dM = I.PR3 * dm, U = I.PR3 * u;
    float Um = fabsf(U);
    #pragma unroll 1
    for (int a = 0; a < I.n_act; ++a) {
      const float4 ac = S.act[a];
      const float cov = fminf(ac.y, (float)(j + 1)) - fmaxf(ac.x, (float)j);
      if (cov <= 0.f) continue;
      const int bits = __float_as_int(ac.w);
      const float side = bits < 0 ? -1.f : 1.f;
      const int tid = bits & 0x7fffffff;
      // Algorithm 1 (mode 1): the force is taken at the step's initial strain
      const bool frozen = A.mode == 1;
      const float e = side * I.d * (frozen ? S.TH0[j] : th) / I.l_seg;
      const float4 hd = A.tab_hdr[tid];
      const float2* tb = A.tab + (size_t)tid * kKnots;
      const float uu = (e - hd.x) * hd.z;
      float f, fp, Gi;
      if (uu <= 0.f) {
        const float f0 = tb[0].x;
        f = f0; fp = 0.f; Gi = f0 * (e - hd.x);
      } else if (uu >= (float)(kKnots - 1)) {
        f = 0.f; fp = 0.f; Gi = tb[kKnots - 1].y;
      } else {
        const int k = (int)uu;
        const float tau = uu - (float)k;
        const float2 k0 = tb[k], k1 = tb[k + 1];
        f = k0.x + tau * (k1.x - k0.x);
        fp = (k1.x - k0.x) * hd.z;
        Gi = k0.y + 0.5f * tau * hd.y * (k0.x + f);
      }
      M -= cov * side * ac.z * f * I.d;
      if (frozen) {  // held force: linear potential, no stiffness
        const float Ua = cov * side * ac.z * f * I.d * th;
        U -= Ua;
        Um += fabsf(Ua);
        continue;
      }
      dM -= cov * ac.z * fp * I.d * I.d / I.l_seg;
      const float Ua = cov * ac.z * I.l_seg * (Gi - hd.w);
      U -= Ua;
      Um += fabsf(Ua);
    }
    Jl = ff_add(Jl, A.w_a * U);
    Sl += A.w_a * Um;
    S.G[j] = A.w_a * M;
    S.DD[j] = fmaxf(A.w_a * dM, floor_d);
    if (fabsf(th) > A.theta_c) sig += 0x9e3779b1u * (unsigned)(j + 1);
    // ---- contacts of link j: KS discs x every obstacle
    const float lx = S.LUX[j], ly = S.LUY[j];
    const bool last = (j == N - 1);
    const float fbx = last ? -uly : -ly / I.l_seg, fby = last ? ulx : lx / I.l_seg;
    FF xk[KS], yk[KS];
#pragma unroll
    for (int k = 0; k < KS; ++k) {
      const float fr = (float)(k + 1) / (float)KS;
      xk[k] = ff_add(px, fr * lx);
      yk[k] = ff_add(py, fr * ly);
    }
    S.FX[j] = 0.f;
    S.FY[j] = 0.f;
    S.TL[j] = 0.f;
    S.C0[j] = 0.f;
    S.C1[j] = 0.f;
    S.C2[j] = 0.f;
    S.C3[j] = 0.f;
    S.C4[j] = 0.f;
    S.C5[j] = 0.f;
    if (last) {
#pragma unroll
      for (int q = 0; q < 5; ++q) S.LX[q] = 0.f;
    }
    // FP32 pre-test of every disc x obstacle pair; the candidates go to the
    // lane's queue and are resolved after the sweep (or when the queue
    // fills), so the warp runs the long contact code once per queue entry
    // of its busiest lane instead of once per pair that any lane hits.
    float pen2 = 0.f, pen1 = 0.f;
    const float Rpre = I.R * (1.f + 1e-6f);
    int qn = 0;
    // every obstacle (no broad phase, or too many near this link), else the
    // link's list; both in obstacle order, so the result is the same.  The
    // pre-tests fill the queue up to the last obstacle that cannot overflow
    // it, then the queue is resolved in order: one call site for the long
    // contact code, and the candidates meet add_contact in scan order.
    const int lb = j * (kListCap + 1);
    const bool every = !A.broad || S.CL[lb] == kListFull;
    const int cnt = every ? I.n_obs : (int)S.CL[lb];
    #pragma unroll 1
    for (int q = 0;;) {
      #pragma unroll 1
      for (; q < cnt && qn <= kContactQueue - KS; ++q) {
        const int o = every ? q : (int)S.CL[lb + 1 + q];
        const float4 ob = S.obs[o];
#pragma unroll
        for (int k = 0; k < KS; ++k)
          if (contact_candidate(ob, xk[k], yk[k], Rpre)) S.Q[(qn++) * TP + tm.r] = o * KS + k;
      }
      #pragma unroll 1
      for (int e = 0; e < qn; ++e) {
        const int code = S.Q[e * TP + tm.r];
        const int o = code / KS, k = code - o * KS;
        const float fr = (float)(k + 1) / (float)KS;
        const FF x = ff_add(px, fr * lx), y = ff_add(py, fr * ly);
        const float4 ob = S.obs[o];
        float nx, ny, kinv;
        float pen = disc_pen_fast(ob, x, y, I.R, fbx, fby, nx, ny, kinv);
        // shallow contacts: the FP32 rounding is a sizeable part of pen, and
        // of the contact force that is proportional to it
        if (pen < kRefinePen * I.R) pen = disc_pen_precise(ob, x, y, I.R, fbx, fby, nx, ny, kinv);
        if (pen > 0.f) {
          pen2 += pen * pen;
          sig += 0x85ebca6bu * (unsigned)(code + 1) + 0xc2b2ae35u * (unsigned)(j + 1);
          pen1 += pen;
          add_contact(S, j, pen, nx, ny, kinv, fr, lx, ly, kap, last, ulx, uly, exact);
        }
      }
      qn = 0;
      if (q >= cnt) break;
    }
    ntest += cnt;
    Jl = ff_add(Jl, A.w_c * I.kc * pen2);
    Sl += (A.w_c * I.kc) * (pen2 + 2.f * I.R * pen1);
    px = ff_add(px, lx);
    py = ff_add(py, ly);
  }
  tm.sync();
  // ---- gradient: g_j = w_a M_tot,j - T_j, T_j = moment about p_j of the
  // contact forces on links >= j = sum_{i>=j} (tl_i + Lu_i x F_{>i}).
  float tfx = 0.f, tfy = 0.f;
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) {
    tfx += S.FX[j];
    tfy += S.FY[j];
  }
  float fsx = tfx, fsy = tfy;
  team_excl_suffix2(fsx, fsy, tm);
  float tt = 0.f;
  #pragma unroll 1
  for (int j = j1 - 1; j >= j0; --j) {
    const float t = S.TL[j] + (S.LUX[j] * fsy - S.LUY[j] * fsx);
    S.TL[j] = t;
    // load stiffness: forces on the links beyond j, times their lever along Lu_j
    if (exact) S.C0[j] += S.LUX[j] * fsx + S.LUY[j] * fsy;
    tt += t;
    fsx += S.FX[j];
    fsy += S.FY[j];
  }
  float run = team_excl_suffix(tt, tm);
  #pragma unroll 1
  for (int j = j1 - 1; j >= j0; --j) {
    run += S.TL[j];
    S.G[j] -= run;
  }
  // ---- reductions
  EvalOut E;
  const float dlr = I.l_seg - l;
  const float Gt = A.w_b * I.kg * dlr * dlr;  // growth term
  const int owner = (N - 1) / B;
  int nt = ntest, sg = (int)sig;
  team_close(Sl, Jl, nt, sg, ulx, uly, owner, tm);
  E.S = Sl + Gt;
  E.J = ff_add(Jl, Gt);
  const float glc = S.LX[0];  // written by the owner thread before the team barrier above
  E.hll = 2.f * A.w_b * I.kg + S.LX[1];
  E.q0 = S.LX[2];
  E.q1 = S.LX[3];
  E.q2 = S.LX[4];
  E.ulx = ulx;
  E.uly = uly;
  E.gl = -2.f * A.w_b * I.kg * (I.l_seg - l) - glc;
  E.kg_wb = A.w_b * I.kg;
  E.tests = nt * KS;
  E.sig = (unsigned)sg;
  tm.sync();
  return E;
}

// Gauss-Newton step (DTH[0..N), dl) and its predicted displacement: the
// square of the largest displacement of a link end point (and of l_seg
// |dtheta_j|), in link lengths squared (the convergence test of the step).  The displacement sums are
// float-float beside the FP32 twists (they do not feed back into the step,
// so they stay off the sweep's dependency chain); per-link FP64 would hold
// GB300's low-rate FP64 pipe for most of the sweep.
// Backward sweep: A_j (articulated stiffness of links >= j about p_j) and
// beta_j; forward sweep: twists V_j and joint steps.  Warp-uniform.
// With `strict` (exact Hessian) a pivot that is not positive means the matrix
// is not positive definite: returns a negative value and forms no step.  The
// Gauss-Newton matrix is positive definite in exact arithmetic, so there a
// pivot lost to FP32 rounding (distal-length Schur complement of a buckled
// joint) is raised to a small positive floor instead.
template <int TP>
__device__ double gn_solve(const InstDev& I, const Smem& S, int N, bool lfix, const EvalOut& E, float& dl,
                           const Team<TP>& tm, bool strict, float& max_dth, double tol2 = -1.0) {
  float A00 = 0.f, A01 = 0.f, A02 = 0.f, A11 = 0.f, A12 = 0.f, A22 = 0.f;
  float b0 = 0.f, b1 = 0.f, b2 = 0.f;
  if (strict && !lfix && !(E.hll > 1e-3f * 2.f * E.kg_wb)) return -1.0;
  const float iH = lfix ? 0.f : 1.f / E.hll;
  bool pd = true;
  float V0 = 0.f, V1 = 0.f, V2 = 0.f, dmax = 0.f, rmax2 = 0.f;
  dl = 0.f;
  // The sweeps overwrite the stiffness entries they read, so a two-warp
  // team runs them on its first warp alone (the second would lag behind the
  // writes) and takes the results from the scratch.
  const bool sweeper = TP == 32 || tm.warp() == 0;
  #pragma unroll 1
  for (int j = sweeper ? N - 1 : -1; j >= 0; --j) {
    float c00 = S.C0[j], c01 = S.C1[j], c02 = S.C2[j], c11 = S.C3[j], c12 = S.C4[j], c22 = S.C5[j];
    const float dj = S.DD[j], gj = S.G[j], lx = S.LUX[j], ly = S.LUY[j];
    float e0 = 0.f, e1 = 0.f, e2 = 0.f;
    if (j == N - 1 && !lfix) {  // eliminate the distal length
      c00 -= E.q0 * E.q0 * iH;
      c01 -= E.q0 * E.q1 * iH;
      c02 -= E.q0 * E.q2 * iH;
      c11 -= E.q1 * E.q1 * iH;
      c12 -= E.q1 * E.q2 * iH;
      c22 -= E.q2 * E.q2 * iH;
      const float s = -E.gl * iH;
      e0 = s * E.q0;
      e1 = s * E.q1;
      e2 = s * E.q2;
    }
    // move (A, beta) from p_{j+1} to p_j: twist map a = (1, -ly, lx)
    const float K01 = A01 - ly * A11 + lx * A12;
    const float K02 = A02 - ly * A12 + lx * A22;
    const float K00 = A00 - ly * (A01 + K01) + lx * (A02 + K02);
    const float B0 = b0 - ly * b1 + lx * b2;
    const float C00 = c00 + K00, C01 = c01 + K01, C02 = c02 + K02;
    const float C11 = c11 + A11, C12 = c12 + A12, C22 = c22 + A22;
    const float h0 = B0 + e0, h1 = b1 + e1, h2 = b2 + e2;
    float D = dj + C00;
    const float Dscale = dj + fabsf(c00) + fabsf(K00);
    if (!(D > 1e-6f * Dscale)) {
      if (strict) pd = false;
      else D = 1e-3f * Dscale;
    }
    const float iD = 1.f / D;
    const float cc = gj + h0;
    const float r = dj * iD;
    A00 = C00 * r;
    A01 = C01 * r;
    A02 = C02 * r;
    A11 = C11 - C01 * C01 * iD;
    A12 = C12 - C01 * C02 * iD;
    A22 = C22 - C02 * C02 * iD;
    b0 = h0 - C00 * cc * iD;
    b1 = h1 - C01 * cc * iD;
    b2 = h2 - C02 * cc * iD;
    if (tm.r == 0) {
      S.C0[j] = C00;
      S.C1[j] = C01;
      S.C2[j] = C02;
      S.C3[j] = iD;
      S.C4[j] = cc;
    }
  }
  if (TP == 32) {
    tm.sync();
    if (!pd) return -1.0;
  } else {
    __syncwarp();
  }
  // the displacement of link end i+1 is z x sum_{k<=i} W0_k Lu_k, with W0_k
  // the heading change sum_{j<=k} dtheta_j
  // The displacement sums run in FP32 beside a running bound on their
  // rounding error (each rounding adds at most u times the rounded value;
  // kU = 2u leaves slack for the products and the bound's own rounding).
  // With tol2 given (the convergence threshold, squared link lengths) and
  // the bound deciding on which side of it the float-float result lies, the
  // FP32 value is returned; otherwise the float-float sums are formed from
  // the stored steps exactly as they always were, so every convergence
  // decision is the float-float one.
  constexpr float kU = 1.1920929e-7f;
  float w0 = 0.f, w1 = 0.f, w2 = 0.f, e0 = 0.f, e1 = 0.f, e2 = 0.f, emax = 0.f, rd2 = 0.f, rt2 = 0.f;
  #pragma unroll 1
  for (int j = 0; sweeper && pd && j < N; ++j) {
    const float h0 = S.C0[j], h1 = S.C1[j], h2 = S.C2[j], iD = S.C3[j], cc = S.C4[j];
    const float lx = S.LUX[j], ly = S.LUY[j];
    const float dth = -(cc + h0 * V0 + h1 * V1 + h2 * V2) * iD;
    V0 += dth;
    w0 += dth;
    e0 += kU * fabsf(w0);
    float ex = 0.f, ey = 0.f;
    if (j == N - 1) {
      dl = lfix ? 0.f : -(E.gl + E.q0 * V0 + E.q1 * V1 + E.q2 * V2) * iH;
      ex = dl * E.ulx;
      ey = dl * E.uly;
    }
    V1 -= V0 * ly;
    V2 += V0 * lx;
    const float p1 = w0 * -ly, p2 = w0 * lx;
    w1 += p1;
    w2 += p2;
    e1 += fabsf(ly) * e0 + kU * (fabsf(p1) + fabsf(w1));
    e2 += fabsf(lx) * e0 + kU * (fabsf(p2) + fabsf(w2));
    const float dx = w1 + ex, dy = w2 + ey;
    emax = fmaxf(emax, e1 + e2 + kU * (fabsf(dx) + fabsf(dy)));
    const float dt = I.l_seg * dth;
    const float v2 = dx * dx + dy * dy, t2 = dt * dt;
    if (!(v2 <= rd2)) rd2 = v2;  // keeps NaN
    if (!(t2 <= rt2)) rt2 = t2;
    if (!(fabsf(dth) <= dmax)) dmax = fabsf(dth);
    if (tm.r == 0) S.DTH[j] = dth;
  }
  rmax2 = fmaxf(rd2, rt2);
  if (!(rd2 <= rt2)) rmax2 = rd2;  // keeps NaN
  bool decided = false;
  if (tol2 >= 0.0 && sweeper && pd && isfinite(rd2) && isfinite(emax)) {
    // bounds on the float-float maximum, through the same float division
    const float s = sqrtf(rd2), eb = emax * 1.001f + 1e-30f;
    const float hi = fmaxf((s + eb) * (s + eb) * (1.f + 8.f * kU), rt2);
    const float lo = fmaxf(fmaxf(s - eb, 0.f) * fmaxf(s - eb, 0.f) * (1.f - 8.f * kU), rt2);
    const float l2 = I.l_seg * I.l_seg;
    decided = (double)(hi / l2) <= tol2 || (double)(lo / l2) > tol2;
  }
  if (!decided && sweeper && pd) {
    __syncwarp();
    FF W0{0.f, 0.f}, W1{0.f, 0.f}, W2{0.f, 0.f};
    rmax2 = 0.f;
    #pragma unroll 1
    for (int j = 0; j < N; ++j) {
      const float dth = S.DTH[j], lx = S.LUX[j], ly = S.LUY[j];
      W0 = ff_add(W0, dth);
      float ex = 0.f, ey = 0.f;
      if (j == N - 1) {
        ex = dl * E.ulx;
        ey = dl * E.uly;
      }
      W1 = ff_add(W1, ff_mul(W0, -ly));
      W2 = ff_add(W2, ff_mul(W0, lx));
      const FF dx = ff_add(W1, ex), dy = ff_add(W2, ey);
      const float dt = I.l_seg * dth;
      const float v2 = fmaxf(dx.hi * dx.hi + dy.hi * dy.hi, dt * dt);
      if (!(v2 <= rmax2)) rmax2 = v2;  // keeps NaN
    }
  }
  if (TP > 32) {
    if (tm.r == 0) {
      tm.scr[16] = pd ? 1.f : 0.f;
      tm.scr[17] = rmax2;
      tm.scr[18] = dl;
      tm.scr[19] = dmax;
    }
    tm.sync();
    pd = tm.scr[16] != 0.f;
    rmax2 = tm.scr[17];
    dl = tm.scr[18];
    dmax = tm.scr[19];
    tm.sync();
    if (!pd) return -1.0;
  } else {
    tm.sync();
  }
  max_dth = dmax;
  return (double)(rmax2 / (I.l_seg * I.l_seg));
}

struct StepStats {
  int iters;
  double r;
  long long evals, linkevals, tests;
  int fallbacks;
};

// One growth step, solved by one of two methods:
//  * mode 0: to equilibrium from the warm start.  Newton iterations with the
//    exact Hessian when it is positive definite (else the Gauss-Newton
//    matrix, re-evaluated), then a line search on the projected path
//    P(x + a dx): Armijo on J, or, when the cost change is at the rounding
//    level of J, the approximate Wolfe condition of Hager and Zhang (2005)
//    on the directional slope;
//  * mode 1: Algorithm 1 of Sec. 4.1 read literally: the actuator forces
//    are held at the step's initial strains (eval reads them from TH0), then
//    gd_steps steps of gradient descent, each unknown scaled by its
//    free-space stiffness (joint angles by gd_alpha 2 theta_c / (w_a pi P
//    R^3), the distal length by gd_alpha / (2 w_b k_g), kept in [0, l_seg]);
//    no convergence test.
// With A.relax the step re-solves the present links (no link added), and
// with A.fix_l the distal length is held (the length unknown is dropped
// from the Newton system; the descent leaves it).
// Written as one loop around a single evaluation: the first evaluation, the
// Gauss-Newton re-evaluation, every line-search trial and every descent step
// pass through the same call, so the evaluation's code is inlined once (the
// kernel's text is what its instruction fetch holds).
template <int KS, int TP>
__device__ int step_solve(const GrowArgs& A, const InstDev& I, const Smem& S, int N, float& l, const Team<TP>& tm,
                          StepStats& st) {
  const int B = (N + TP - 1) / TP;
  const int j0 = min(tm.r * B, N), j1 = min(j0 + B, N);
  const bool exact = A.exact != 0;
  const bool descend = A.mode == 1;
  // converged when the Newton step moves no link end point by more than
  // tol N link lengths (tol of the robot's length) nor by more than tol_link
  // link lengths (the bound that holds at any chain length)
  const double tol_eff = A.tol_link > 0.0 ? fmin(A.tol * (double)N, A.tol_link) : A.tol * (double)N;
  const double tol2 = tol_eff * tol_eff;  // the test compares squared displacements
  float a_th = 0.f, a_l = 0.f;
  if (descend) {
    #pragma unroll 1
    for (int k = tm.r; k < N; k += TP) S.TH0[k] = S.TH[k];
    tm.sync();
    a_th = A.gd_alpha * 2.f * A.theta_c / (A.w_a * I.PR3);
    a_l = A.gd_alpha / (2.f * A.w_b * I.kg);
  }
  enum : int { kNewton, kFallback, kTrial };
  int phase = kNewton;
  bool ev_exact = exact && !descend;
  float l_ev = l;
  int status = kMaxIter, it = 0, h = 0, k_desc = 0;
  double r = 0.0;
  FF J0{0.f, 0.f};
  float gd = 0.f, S0 = 0.f, slope0 = 0.f;
  float alpha = 1.f, lt = l, l0 = l, gl0 = 0.f, dl = 0.f, mdth = 0.f;
  bool lfix = false;
  // the last Newton step was small and has been applied; the evaluation at
  // the point it reached checks the active set against the step's
  bool checking = false, lfix_conv = false;
  unsigned sig_conv = 0u;
  // every path below advances it, h or k_desc, all bounded; the cap is a
  // second guarantee that the loop ends
  const long long cap = (long long)(max(A.max_iter, 0) + 1) * (max(A.max_halv, 0) + 3) + max(A.gd_steps, 0) + 4;
  for (long long guard = 0; guard < cap; ++guard) {
    const EvalOut E = eval<KS, TP>(A, I, S, N, l_ev, tm, ev_exact);
    st.evals += 1;
    st.linkevals += N;
    st.tests += E.tests;
    if (descend) {
      st.iters += 1;
      if (!isfinite(E.J.hi)) {
        status = kNonFinite;
        break;
      }
      #pragma unroll 1
      for (int k = tm.r; k < N; k += TP) S.TH[k] -= a_th * S.G[k];
      if (!A.fix_l) l = fminf(fmaxf(l - a_l * E.gl, 0.f), I.l_seg);
      l_ev = l;
      tm.sync();
      if (++k_desc >= A.gd_steps) {
        status = kOK;
        break;
      }
      continue;
    }
    if (phase == kTrial) {
      // cost change and predicted decrease (float-float difference of the costs)
      const float dJ = ff_add(E.J, ff_neg(J0)).hi;
      const float dec = alpha * gd + gl0 * (lt - l0);
      float sl = 0.f;
      const bool rounding = fabsf(dJ) <= A.fval_eps * fmaxf(S0, E.S);
      if (rounding) {
        const FF d = team_dot(S.G, S.DTH, j0, j1, tm);
        sl = d.hi + d.lo;
        if (lt > 0.f && lt < I.l_seg) sl += E.gl * dl;
      }
      const bool accepted = dJ <= A.c1 * dec || (rounding && sl <= (2.f * A.c1 - 1.f) * slope0);
      if (accepted) {
        // a trial so short that no unknown changed (the step below FP32
        // resolution) is no progress: the iteration would repeat itself
        bool moved = lt != l0;
        #pragma unroll 1
        for (int j = j0; j < j1 && !moved; ++j) moved = S.TH[j] != S.TH0[j];
        if (!team_any(moved, tm)) {
          #pragma unroll 1
          for (int j = j0; j < j1; ++j) S.TH[j] = S.TH0[j];
          l = l0;
          tm.sync();
          break;
        }
      }
      if (!accepted) {
        if (h < A.max_halv) {
          alpha *= 0.5f;
          ++h;
          #pragma unroll 1
          for (int j = j0; j < j1; ++j) S.TH[j] = S.TH0[j] + alpha * S.DTH[j];
          lt = fminf(fmaxf(l0 + alpha * dl, 0.f), I.l_seg);
          l_ev = lt;
          tm.sync();
          continue;
        }
        // no acceptable trial: the step ends at the last accepted iterate
        #pragma unroll 1
        for (int j = j0; j < j1; ++j) S.TH[j] = S.TH0[j];
        l = l0;
        tm.sync();
        break;
      }
      l = lt;
      phase = kNewton;
    }
    if (phase == kNewton) {
      if (checking) {
        checking = false;
        const bool lf = A.fix_l || (l <= 0.f && E.gl > 0.f) || (l >= I.l_seg && E.gl < 0.f);
        if (E.sig == sig_conv && lf == lfix_conv && isfinite(E.J.hi)) {
          status = kOK;
          break;
        }
      }
      if (++it > A.max_iter) break;
      if (!isfinite(E.J.hi)) {
        status = kNonFinite;
        break;
      }
      lfix = A.fix_l || (l <= 0.f && E.gl > 0.f) || (l >= I.l_seg && E.gl < 0.f);
    }
    const bool use_exact = exact && phase == kNewton;
    r = gn_solve(I, S, N, lfix, E, dl, tm, use_exact, mdth, tol2);  // squared, link lengths
    if (use_exact && !(r >= 0.0 && isfinite(r))) {
      // exact Hessian not positive definite here: Gauss-Newton matrix instead
      st.fallbacks += 1;
      phase = kFallback;
      ev_exact = false;
      l_ev = l;
      continue;
    }
    if (!isfinite(E.J.hi)) {
      status = kNonFinite;
      break;
    }
    if (!isfinite(r) || r < 0.0) {
      // the Gauss-Newton sweep lost its pivots to FP32 range (bending floor
      // against contact stiffness): steepest descent, at most 0.05 rad per joint
      float gm = 0.f;
      #pragma unroll 1
      for (int j = j0; j < j1; ++j) gm = fmaxf(gm, fabsf(S.G[j]));
      gm = team_max(gm, tm);
      const float sc = gm > 0.f ? 0.05f / gm : 0.f;
      #pragma unroll 1
      for (int j = j0; j < j1; ++j) S.DTH[j] = -S.G[j] * sc;
      dl = lfix ? 0.f : -E.gl * sc * I.l_seg * I.l_seg;
      if (!(sc > 0.f) || !isfinite(dl)) {
        status = kNonFinite;
        break;
      }
      r = 1e60;  // not a Newton step: never taken as converged
      st.fallbacks += 1;
      tm.sync();
    }
    if (r <= tol2) {
      #pragma unroll 1
      for (int j = j0; j < j1; ++j) S.TH[j] += S.DTH[j];
      l = fminf(fmaxf(l + dl, 0.f), I.l_seg);
      // the point the small step reached is evaluated once more: a step that
      // crosses into a contact (or past the wrinkling onset of a joint) can
      // leave a long, soft chain far from the equilibrium although the step
      // itself was small.  Converged when the active set is the one the step
      // was computed with; else the solve goes on from there.  (The next
      // Newton step itself is no test: at a near-singular equilibrium its
      // FP32 value is noise.)
      sig_conv = E.sig;
      lfix_conv = lfix;
      checking = true;
      phase = kNewton;
      l_ev = l;
      ev_exact = exact;
      tm.sync();
      continue;
    }
    // line search: first trial at the full step
    {
      const FF d = team_dot(S.G, S.DTH, j0, j1, tm);
      gd = d.hi + d.lo;
    }
    #pragma unroll 1
    for (int j = j0; j < j1; ++j) S.TH0[j] = S.TH[j];
    l0 = l;
    gl0 = E.gl;
    J0 = E.J;
    S0 = E.S;
    const bool l_moves = !((l0 <= 0.f && dl < 0.f) || (l0 >= I.l_seg && dl > 0.f));
    slope0 = gd + (l_moves ? gl0 * dl : 0.f);
    alpha = 1.f;
    h = 0;
    #pragma unroll 1
    for (int j = j0; j < j1; ++j) S.TH[j] = S.TH0[j] + alpha * S.DTH[j];
    lt = fminf(fmaxf(l0 + alpha * dl, 0.f), I.l_seg);
    l_ev = lt;
    phase = kTrial;
    ev_exact = exact;
    tm.sync();
  }
  if (descend) {
    if (status == kOK) {
      bool badl = false;
      #pragma unroll 1
      for (int k = tm.r; k < N; k += TP) badl = badl || !isfinite(S.TH[k]);
      if (team_any(badl, tm)) status = kNonFinite;
    }
    st.r = 0.0;
    return status;
  }
  if (it > A.max_iter) it = A.max_iter;
  tm.sync();
  st.iters = it;
  st.r = (r >= 0.0 ? sqrt(r) : r) / (double)N;  // reported relative to the robot length
  return status;
}

template <int KS, int TP>
__device__ void process_instance(const GrowArgs& A, int inst, const Smem& S, const Team<TP>& tm) {
  const long long t_start = clock64();
  const InstDev I = A.inst[inst];
  int status = A.status[inst];
  // a robot whose growth step failed (out of iterations, or non-finite) has
  // stopped: its later steps would start from a state that is not an
  // equilibrium of the model
  if (status != kOK) return;
  int N = A.n_cur[inst];
  if (A.n_steps <= 0 || (A.relax ? N == 0 : N >= I.n_target)) return;
  #pragma unroll 1
  for (int k = tm.r; k < I.n_obs; k += TP) S.obs[k] = A.obs[I.obs_off + k];
  #pragma unroll 1
  for (int k = tm.r; k < I.n_act; k += TP) S.act[k] = A.act[I.act_off + k];
  #pragma unroll 1
  for (int k = tm.r; k < N; k += TP) S.TH[k] = A.theta[I.th_off + k];
  float l = A.l_cur[inst];
  reset_lists(S, I.n_target, tm);
  int iters = 0, conv = 0, steps = 0;
  long long rls = 0, evals = 0, linkevals = 0, fallbacks = 0, tests = 0;
  double rmax = 0.0;
  #pragma unroll 1
  for (int s = 0; s < A.n_steps && (A.relax || N < I.n_target); ++s) {
    if (!A.relax) {
      if (tm.r == 0) S.TH[N] = 0.f;  // new link at the tip
      N += 1;
      l = 0.f;
    }
    tm.sync();
    StepStats st{0, 0.0, 0, 0, 0, 0};
    const int res = step_solve<KS, TP>(A, I, S, N, l, tm, st);
    iters += st.iters;
    evals += st.evals;
    linkevals += st.linkevals;
    tests += st.tests;
    fallbacks += st.fallbacks;
    steps += 1;
    if (!(st.r <= rmax)) rmax = st.r;
    if (res == kOK) {
      conv += 1;
      rls += N;
    } else if (res > status) {
      status = res;
    }
    if (status != kOK) break;
  }
  tm.sync();
  #pragma unroll 1
  for (int k = tm.r; k < N; k += TP) A.theta[I.th_off + k] = S.TH[k];
  if (tm.r == 0) {
    A.n_cur[inst] = N;
    A.l_cur[inst] = l;
    A.status[inst] = status;
    A.iters[inst] += iters;
    A.conv[inst] += conv;
    A.steps[inst] += steps;
    A.rls[inst] += rls;
    A.evals[inst] += evals;
    A.linkevals[inst] += linkevals;
    A.pairtests[inst] += tests;
    A.fallbacks[inst] += fallbacks;
    A.cycles[inst] += clock64() - t_start;
    if (!(rmax <= A.resid_max[inst])) A.resid_max[inst] = rmax;
  }
  tm.sync();
}

template <int KS>
__global__ void __launch_bounds__(32 * kWarpsPerCta, 3) grow_kernel(const GrowArgs A) {
  extern __shared__ float4 smem4[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const Smem S = carve<32>(reinterpret_cast<float*>(smem4) + (size_t)warp * A.warp_floats, A);
  const Team<32> tm{lane, S.TS};
  const int gw = blockIdx.x * (blockDim.x >> 5) + warp;
  const int nw = gridDim.x * (blockDim.x >> 5);
  for (int round = 0;; ++round) {
    int idx;
    if (A.dynamic) {
      int v = 0;
      if (lane == 0) v = atomicAdd(A.counter, 1);
      idx = __shfl_sync(kFull, v, 0);
    } else {
      idx = gw + round * nw;
    }
    if (idx >= A.n_order) break;
    process_instance<KS, 32>(A, A.order[idx], S, tm);
  }
}

// Several warps per robot: one robot per CTA of TP threads, the same code
// with the team operations across the warps.
template <int KS, int TP>
__global__ void __launch_bounds__(TP, 384 / TP) grow_kernel_team(const GrowArgs A) {
  extern __shared__ float4 smem4[];
  __shared__ int next;
  const Smem S = carve<TP>(reinterpret_cast<float*>(smem4), A);
  const Team<TP> tm{(int)threadIdx.x, S.TS};
  for (int round = 0;; ++round) {
    int idx;
    if (A.dynamic) {
      if (tm.r == 0) next = atomicAdd(A.counter, 1);
      __syncthreads();
      idx = next;
      __syncthreads();
    } else {
      idx = blockIdx.x + round * gridDim.x;
    }
    if (idx >= A.n_order) break;
    process_instance<KS, TP>(A, A.order[idx], S, tm);
  }
}

// Cost, gradient and one Gauss-Newton step at a caller-given state of one
// robot (introspection for tests; one warp).
template <int KS>
__global__ void __launch_bounds__(32) probe_kernel(const GrowArgs A, int inst, int N, const float* theta, float l,
                                                   double* outJ, float* out_g, float* out_dx, double* out_r,
                                                   int* out_lfix) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31;
  const Smem S = carve<32>(reinterpret_cast<float*>(smem4), A);
  const Team<32> tm{(int)(threadIdx.x & 31), S.TS};
  const InstDev I = A.inst[inst];
  for (int k = lane; k < I.n_obs; k += 32) S.obs[k] = A.obs[I.obs_off + k];
  for (int k = lane; k < I.n_act; k += 32) S.act[k] = A.act[I.act_off + k];
  for (int k = lane; k < N; k += 32) S.TH[k] = theta[k];
  reset_lists(S, N, tm);
  EvalOut E = eval<KS, 32>(A, I, S, N, l, tm, A.exact != 0);
  for (int k = lane; k < N; k += 32) out_g[k] = S.G[k];
  __syncwarp();
  const bool lfix = (l <= 0.f && E.gl > 0.f) || (l >= I.l_seg && E.gl < 0.f);
  float dl;
  float mdth;
  double r = gn_solve(I, S, N, lfix, E, dl, tm, A.exact != 0, mdth);
  if (A.exact != 0 && !(r >= 0.0 && isfinite(r))) {
    E = eval<KS, 32>(A, I, S, N, l, tm, false);
    r = gn_solve(I, S, N, lfix, E, dl, tm, false, mdth);
  }
  for (int k = lane; k < N; k += 32) out_dx[k] = S.DTH[k];
  if (lane == 0) {
    out_g[N] = E.gl;
    out_dx[N] = dl;
    *outJ = (double)E.J.hi + (double)E.J.lo;
    *out_r = r >= 0.0 ? sqrt(r) / (double)N : r;  // relative to the robot length
    *out_lfix = lfix ? 1 : 0;
  }
}

// Force per unit pressure of sPAM table `tid` at strain e (the piecewise-
// linear table of Sec. 3.1; held below its first knot, zero beyond its last).
__device__ __forceinline__ float spam_force(const GrowArgs& A, int tid, float e) {
  const float4 hd = A.tab_hdr[tid];
  const float2* tb = A.tab + (size_t)tid * kKnots;
  const float uu = (e - hd.x) * hd.z;
  if (uu <= 0.f) return tb[0].x;
  if (uu >= (float)(kKnots - 1)) return 0.f;
  const int k = (int)uu;
  const float tau = uu - (float)k;
  return tb[k].x + tau * (tb[k + 1].x - tb[k].x);
}

// Adjoint of a cost c of the robot's shape at its current state, taken as
// the equilibrium of its last growth step (implicit differentiation):
// lambda = H^-1 dc/dx with H the exact Hessian of the cost of Eq. (pbd) (the
// articulated sweep of gn_solve with the right-hand side replaced), then
// dc/dq = -lambda . d(grad J)/dq.  Costs: the tip distance |p_N - goal|, or
// the path cost (1/N) sum_k |p_k - q_k|^2 of the link end points p_1..p_N
// against targets q_k, whose derivative in joint j is the moment about p_j
// of "forces" (2/N)(p_k - q_k) at the link ends beyond it -- assembled by the
// suffix scans of the contact moments.  grad J depends on an
// actuator's pressure P_a and span [b_a, e_a) only through its moment
// c_aj s_a P_a f_a(eps_aj) d (Eq. restoring_moment): linearly in P_a, and
// through the coverage c_aj, whose right derivatives are -1 on link
// floor(b_a) and +1 on link floor(e_a).  Status: 0 ok, 1 the exact Hessian is
// not positive definite there (derivatives NaN), 2 the robot has no valid
// state (bad input or non-finite; cost and derivatives NaN).
template <int KS>
__device__ void grad_instance(const GrowArgs& A, const GradArgs& G, int inst, const Smem& S, int lane) {
  const Team<32> tm{lane, S.TS};
  const InstDev I = A.inst[inst];
  const int N = A.n_cur[inst];
  const int st = A.status[inst];
  // the tip cost's goal (the path cost reads its targets below)
  const float gx = G.kind == 0 ? G.goal[2 * inst] - I.bx : 0.f, gy = G.kind == 0 ? G.goal[2 * inst + 1] - I.by : 0.f;
  const double qnan = __longlong_as_double(0x7ff8000000000000ll);
  if (st == kBadInput || st == kNonFinite || N <= 0) {
    const bool ok = (N <= 0 && st != kBadInput && st != kNonFinite);
    for (int a = lane; a < I.n_act; a += 32) {
      G.dP[I.act_off + a] = ok ? 0.0 : qnan;
      G.dB[I.act_off + a] = ok ? 0.0 : qnan;
      G.dE[I.act_off + a] = ok ? 0.0 : qnan;
    }
    if (lane == 0) {
      G.cost[inst] = ok ? (G.kind == 1 ? 0.0 : sqrt((double)gx * gx + (double)gy * gy)) : qnan;
      G.gstat[inst] = ok ? 0 : 2;
    }
    return;
  }
  for (int k = lane; k < I.n_obs; k += 32) S.obs[k] = A.obs[I.obs_off + k];
  for (int k = lane; k < I.n_act; k += 32) S.act[k] = A.act[I.act_off + k];
  for (int k = lane; k < N; k += 32) S.TH[k] = A.theta[I.th_off + k];
  const float l = A.l_cur[inst];
  reset_lists(S, N, tm);
  EvalOut E = eval<KS, 32>(A, I, S, N, l, tm, true);
  const bool lfix = (l <= 0.f && E.gl > 0.f) || (l >= I.l_seg && E.gl < 0.f);
  const int B = (N + 31) >> 5;
  const int j0 = min(lane * B, N), j1 = min(j0 + B, N);
  double c;
  if (G.kind == 0) {
    // tip relative to the base, and dc/dtheta_j = s . (z x (p_N - p_j))
    float sx = 0.f, sy = 0.f;
    #pragma unroll 1
    for (int j = j0; j < j1; ++j) {
      sx += S.LUX[j];
      sy += S.LUY[j];
    }
    float rx = warp_excl_suffix(sx, lane), ry = warp_excl_suffix(sy, lane);
    const float tx = __shfl_sync(kFull, rx + sx, 0), ty = __shfl_sync(kFull, ry + sy, 0);
    const double ex = (double)tx - (double)gx, ey = (double)ty - (double)gy;
    c = sqrt(ex * ex + ey * ey);
    const float ux = c > 0.0 ? (float)(ex / c) : 0.f, uy = c > 0.0 ? (float)(ey / c) : 0.f;
    #pragma unroll 1
    for (int j = j1 - 1; j >= j0; --j) {
      rx += S.LUX[j];
      ry += S.LUY[j];
      S.G[j] = ux * ry - uy * rx;  // minus dc/dtheta_j: the sweep solves H x = -G
    }
    E.gl = -(ux * E.ulx + uy * E.uly);
  } else {
    // link end points relative to the base (float-float prefix sums), their
    // errors e_k = p_k - q_k as forces f_j = (2/N) e_{j+1} at the end of
    // link j: dc/dtheta_j = sum_{i >= j} (Lu_i x f_i + Lu_i x F_{>i})
    FF hx{0.f, 0.f}, hy{0.f, 0.f};
    #pragma unroll 1
    for (int j = j0; j < j1; ++j) {
      hx = ff_add(hx, S.LUX[j]);
      hy = ff_add(hy, S.LUY[j]);
    }
    FF px = warp_excl_scan(hx, lane), py = warp_excl_scan(hy, lane);
    const float* q = G.goal + 2 * (size_t)I.th_off;
    const float w = 2.f / (float)N;
    double cs = 0.0;
    float tfx = 0.f, tfy = 0.f;
    #pragma unroll 1
    for (int j = j0; j < j1; ++j) {
      px = ff_add(px, S.LUX[j]);
      py = ff_add(py, S.LUY[j]);
      const float ex = (px.hi - (q[2 * j] - I.bx)) + px.lo, ey = (py.hi - (q[2 * j + 1] - I.by)) + py.lo;
      cs += (double)ex * ex + (double)ey * ey;
      S.FX[j] = w * ex;
      S.FY[j] = w * ey;
      tfx += S.FX[j];
      tfy += S.FY[j];
    }
    c = warp_sum(cs) / (double)N;
    float fsx = warp_excl_suffix(tfx, lane), fsy = warp_excl_suffix(tfy, lane);
    float tt = 0.f;
    #pragma unroll 1
    for (int j = j1 - 1; j >= j0; --j) {
      const float t = S.LUX[j] * (S.FY[j] + fsy) - S.LUY[j] * (S.FX[j] + fsx);
      S.TL[j] = t;
      tt += t;
      fsx += S.FX[j];
      fsy += S.FY[j];
    }
    float run = warp_excl_suffix(tt, lane);
    #pragma unroll 1
    for (int j = j1 - 1; j >= j0; --j) {
      run += S.TL[j];
      S.G[j] = -run;  // minus dc/dtheta_j
    }
    // dc/dl = f_{N-1} . u_{N-1}; the owner of the last link has its force
    const int owner = (N - 1) / B;
    const float flx = __shfl_sync(kFull, j1 == N && j0 < j1 ? S.FX[N - 1] : 0.f, owner);
    const float fly = __shfl_sync(kFull, j1 == N && j0 < j1 ? S.FY[N - 1] : 0.f, owner);
    E.gl = -(flx * E.ulx + fly * E.uly);
  }
  __syncwarp();
  float dl, mdth;
  const double r = gn_solve(I, S, N, lfix, E, dl, tm, true, mdth);
  const bool ok = r >= 0.0 && isfinite(r);
  for (int a = 0; a < I.n_act; ++a) {
    const float4 ac = S.act[a];
    const int bits = __float_as_int(ac.w);
    const float side = bits < 0 ? -1.f : 1.f;
    const int tid = bits & 0x7fffffff;
    const float jb = floorf(ac.x), je = floorf(ac.y);
    const bool span = ac.x < ac.y;
    double sP = 0.0, sB = 0.0, sE = 0.0;
    #pragma unroll 1
    for (int j = j0; j < j1; ++j) {
      const float cov = fminf(ac.y, (float)(j + 1)) - fmaxf(ac.x, (float)j);
      const bool isb = span && (float)j == jb, ise = span && (float)j == je;
      if (!(cov > 0.f) && !isb && !ise) continue;
      const float f = spam_force(A, tid, side * I.d * S.TH[j] / I.l_seg);
      const double m = (double)A.w_a * side * f * I.d * (double)S.DTH[j];  // -lambda_j d g_j / d(c_aj P_a)
      if (cov > 0.f) sP += m * cov;
      if (isb) sB -= m * ac.z;
      if (ise) sE += m * ac.z;
    }
    sP = warp_sum(sP);
    sB = warp_sum(sB);
    sE = warp_sum(sE);
    if (lane == 0) {
      G.dP[I.act_off + a] = ok ? sP : qnan;
      G.dB[I.act_off + a] = ok ? sB : qnan;
      G.dE[I.act_off + a] = ok ? sE : qnan;
    }
  }
  if (lane == 0) {
    G.cost[inst] = c;
    G.gstat[inst] = ok ? 0 : 1;
  }
  __syncwarp();
}

// One warp per robot, longest robots first.
template <int KS>
__global__ void __launch_bounds__(32) grad_kernel(const GrowArgs A, const GradArgs G) {
  extern __shared__ float4 smem4[];
  const int lane = threadIdx.x & 31;
  const Smem S = carve<32>(reinterpret_cast<float*>(smem4), A);
  for (int idx = blockIdx.x; idx < A.n_order; idx += gridDim.x) grad_instance<KS>(A, G, A.order[idx], S, lane);
}

template <int KS>
const void* kernel_ptr() {
  return reinterpret_cast<const void*>(&grow_kernel<KS>);
}

template <int KS, int TP>
const void* team_kernel_ptr() {
  return reinterpret_cast<const void*>(&grow_kernel_team<KS, TP>);
}

const void* pick(int ks, int team) {
  if (team == 64) {
    switch (ks) {
      case 1: return team_kernel_ptr<1, 64>();
      case 2: return team_kernel_ptr<2, 64>();
      case 3: return team_kernel_ptr<3, 64>();
      default: return team_kernel_ptr<4, 64>();
    }
  }
  if (team == 128) {
    switch (ks) {
      case 1: return team_kernel_ptr<1, 128>();
      case 2: return team_kernel_ptr<2, 128>();
      case 3: return team_kernel_ptr<3, 128>();
      default: return team_kernel_ptr<4, 128>();
    }
  }
  switch (ks) {
    case 1: return kernel_ptr<1>();
    case 2: return kernel_ptr<2>();
    case 3: return kernel_ptr<3>();
    default: return kernel_ptr<4>();
  }
}

}  // namespace

size_t grow_smem_per_warp(int nmax, int omax, int amax, int team) {
  return sizeof(float4) * (size_t)(omax + amax) + sizeof(float) * (16 * (size_t)nmax + 8) +
         sizeof(int) * (size_t)team * kContactQueue + sizeof(float) * kTeamScratch + sizeof(float) * 7 * (size_t)nmax +
         ((sizeof(unsigned short) * (kListCap + 1) * (size_t)nmax + 15) & ~size_t(15));
}

// The attribute is per kernel and process-wide: batches and servers with
// different slices share it, so it is only ever raised.
cudaError_t grow_configure(int ks, size_t smem_per_cta, int team) {
  static std::mutex mu;
  static std::map<std::pair<int, int>, size_t> set;  // (device, K_s + 8 for the team kernel) -> bytes
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(mu);
  size_t& cur = set[{dev, ks + 8 * (team / 64)}];
  if (smem_per_cta <= cur) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(pick(ks, team), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem_per_cta);
  if (e == cudaSuccess) cur = smem_per_cta;
  return e;
}

int grow_max_ctas_per_sm(int ks, size_t smem_per_cta, int threads, int team) {
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, pick(ks, team), threads, smem_per_cta) != cudaSuccess) return 0;
  return n;
}

// Warps per CTA (4, 2 or 1) that keep the most warps resident per SM for a
// warp slice of smem_warp bytes (a robot's obstacles and link arrays are
// per warp, so smaller CTAs pack large slices more tightly); ties go to the
// larger CTA.  Sets the kernel's shared-memory limit for the choice.
int grow_pick_block(int ks, size_t smem_warp, int* ctas_per_sm, int team) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (team > 32) {  // one team (robot) per CTA
    int c = 0;
    if (smem_warp <= (size_t)optin && grow_configure(ks, smem_warp, team) == cudaSuccess)
      c = grow_max_ctas_per_sm(ks, smem_warp, team, team);
    if (ctas_per_sm) *ctas_per_sm = c;
    return c > 0 ? 1 : 0;
  }
  int best_w = 0, best_c = 0;
  // two-warp CTAs first: at equal resident warps they measured faster than
  // four-warp CTAs on uniform and uneven batches alike
  const int order[3] = {2, kWarpsPerCta, 1};
  for (int w : order) {
    const size_t smem = smem_warp * w;
    if (smem > (size_t)optin) continue;
    if (grow_configure(ks, smem) != cudaSuccess) continue;
    const int c = grow_max_ctas_per_sm(ks, smem, 32 * w);
    if (c * w > best_c * best_w) {
      best_w = w;
      best_c = c;
    }
  }
  if (ctas_per_sm) *ctas_per_sm = best_c;
  return best_w;
}

cudaError_t launch_grow(const GrowArgs& a, int ks, int grid, int block, size_t smem, cudaStream_t s) {
  if (a.team == 64) {
    switch (ks) {
      case 1: grow_kernel_team<1, 64><<<grid, 64, smem, s>>>(a); break;
      case 2: grow_kernel_team<2, 64><<<grid, 64, smem, s>>>(a); break;
      case 3: grow_kernel_team<3, 64><<<grid, 64, smem, s>>>(a); break;
      default: grow_kernel_team<4, 64><<<grid, 64, smem, s>>>(a); break;
    }
    return cudaGetLastError();
  }
  if (a.team == 128) {
    switch (ks) {
      case 1: grow_kernel_team<1, 128><<<grid, 128, smem, s>>>(a); break;
      case 2: grow_kernel_team<2, 128><<<grid, 128, smem, s>>>(a); break;
      case 3: grow_kernel_team<3, 128><<<grid, 128, smem, s>>>(a); break;
      default: grow_kernel_team<4, 128><<<grid, 128, smem, s>>>(a); break;
    }
    return cudaGetLastError();
  }
  switch (ks) {
    case 1: grow_kernel<1><<<grid, block, smem, s>>>(a); break;
    case 2: grow_kernel<2><<<grid, block, smem, s>>>(a); break;
    case 3: grow_kernel<3><<<grid, block, smem, s>>>(a); break;
    default: grow_kernel<4><<<grid, block, smem, s>>>(a); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_grad(const GrowArgs& a, const GradArgs& g, int ks, int grid, size_t smem, cudaStream_t s) {
  const void* fn;
  switch (ks) {
    case 1: fn = reinterpret_cast<const void*>(&grad_kernel<1>); break;
    case 2: fn = reinterpret_cast<const void*>(&grad_kernel<2>); break;
    case 3: fn = reinterpret_cast<const void*>(&grad_kernel<3>); break;
    default: fn = reinterpret_cast<const void*>(&grad_kernel<4>); break;
  }
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  switch (ks) {
    case 1: grad_kernel<1><<<grid, 32, smem, s>>>(a, g); break;
    case 2: grad_kernel<2><<<grid, 32, smem, s>>>(a, g); break;
    case 3: grad_kernel<3><<<grid, 32, smem, s>>>(a, g); break;
    default: grad_kernel<4><<<grid, 32, smem, s>>>(a, g); break;
  }
  return cudaGetLastError();
}

cudaError_t launch_probe(const GrowArgs& a, int ks, int inst, int N, const float* theta, float l, double* J,
                         float* g, float* dx, double* r, int* lfix, size_t smem, cudaStream_t s) {
  switch (ks) {
    case 1: probe_kernel<1><<<1, 32, smem, s>>>(a, inst, N, theta, l, J, g, dx, r, lfix); break;
    case 2: probe_kernel<2><<<1, 32, smem, s>>>(a, inst, N, theta, l, J, g, dx, r, lfix); break;
    case 3: probe_kernel<3><<<1, 32, smem, s>>>(a, inst, N, theta, l, J, g, dx, r, lfix); break;
    default: probe_kernel<4><<<1, 32, smem, s>>>(a, inst, N, theta, l, J, g, dx, r, lfix); break;
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Outputs: poses and contact pairs at the current state (one warp per robot).
// ---------------------------------------------------------------------------
namespace {

// sel == nullptr: robot gw, outputs at its own joint-angle offset.  Else
// robot sel[gw], outputs at out_off[gw] (a compact copy of selected robots);
// the tip always goes to out_tip[2 gw].
__global__ void pose_kernel(const InstDev* inst, int n_inst, const int* sel, const long long* out_off,
                            const float* theta, const int* n_cur, const float* l_cur, float* out_theta,
                            float* out_pose, float* out_tip) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= n_inst) return;
  const int ri = sel ? sel[gw] : gw;
  const InstDev I = inst[ri];
  const int N = n_cur[ri];
  const float l = l_cur[ri];
  const size_t oo = sel ? (size_t)out_off[gw] : (size_t)I.th_off;
  const int B = (N + 31) >> 5;
  const int j0 = min(lane * B, N), j1 = min(j0 + B, N);
  const float* th = theta + I.th_off;
  FF hs{0.f, 0.f};
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) hs = ff_add(hs, th[j]);
  FF psi0 = ff_add(warp_excl_scan(hs, lane), I.bpsi);
  FF psi = psi0, sx{0.f, 0.f}, sy{0.f, 0.f};
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) {
    psi = ff_add(psi, th[j]);
    float sn, cs;
    sincosf(psi.hi, &sn, &cs);
    const float L = (j == N - 1) ? l : I.l_seg;
    sx = ff_add(sx, L * (cs - sn * psi.lo));
    sy = ff_add(sy, L * (sn + cs * psi.lo));
  }
  FF px = warp_excl_scan(sx, lane), py = warp_excl_scan(sy, lane);
  psi = psi0;
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) {
    psi = ff_add(psi, th[j]);
    if (out_pose) {
      out_pose[3 * (oo + j) + 0] = (px.hi + I.bx) + px.lo;
      out_pose[3 * (oo + j) + 1] = (py.hi + I.by) + py.lo;
      out_pose[3 * (oo + j) + 2] = psi.hi + psi.lo;
    }
    if (out_theta) out_theta[oo + j] = th[j];
    float sn, cs;
    sincosf(psi.hi, &sn, &cs);
    const float L = (j == N - 1) ? l : I.l_seg;
    px = ff_add(px, L * (cs - sn * psi.lo));
    py = ff_add(py, L * (sn + cs * psi.lo));
  }
  #pragma unroll 1
  for (int j = N + lane; j < I.n_target; j += 32) {
    if (out_pose) {
      out_pose[3 * (oo + j) + 0] = 0.f;
      out_pose[3 * (oo + j) + 1] = 0.f;
      out_pose[3 * (oo + j) + 2] = 0.f;
    }
    if (out_theta) out_theta[oo + j] = 0.f;
  }
  // the lane holding the last link has the tip in (px, py)
  if (out_tip && N > 0 && j1 == N && j0 < j1) {
    out_tip[2 * gw + 0] = (px.hi + I.bx) + px.lo;
    out_tip[2 * gw + 1] = (py.hi + I.by) + py.lo;
  }
  if (out_tip && N == 0 && lane == 0) {
    out_tip[2 * gw + 0] = I.bx;
    out_tip[2 * gw + 1] = I.by;
  }
}

// Contact pairs (link, obstacle) of one robot, in (link, obstacle) order.
__global__ void contacts_kernel(const InstDev* inst, int n_inst, const float4* obs, const float* theta,
                                const int* n_cur, const float* l_cur, int ks, int max_pairs, int* counts,
                                int* pairs) {
  const int gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (gw >= n_inst) return;
  const InstDev I = inst[gw];
  const int N = n_cur[gw];
  const float l = l_cur[gw];
  const int B = (N + 31) >> 5;
  const int j0 = min(lane * B, N), j1 = min(j0 + B, N);
  const float* th = theta + I.th_off;
  const float4* ob = obs + I.obs_off;
  FF hs{0.f, 0.f};
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) hs = ff_add(hs, th[j]);
  FF psi0 = ff_add(warp_excl_scan(hs, lane), I.bpsi);
  FF psi = psi0, sx{0.f, 0.f}, sy{0.f, 0.f};
  #pragma unroll 1
  for (int j = j0; j < j1; ++j) {
    psi = ff_add(psi, th[j]);
    float sn, cs;
    sincosf(psi.hi, &sn, &cs);
    const float L = (j == N - 1) ? l : I.l_seg;
    sx = ff_add(sx, L * (cs - sn * psi.lo));
    sy = ff_add(sy, L * (sn + cs * psi.lo));
  }
  const FF px0 = warp_excl_scan(sx, lane), py0 = warp_excl_scan(sy, lane);
  int base = 0;
  for (int pass = 0; pass < 2; ++pass) {
    FF px = px0, py = py0;
    psi = psi0;
    int cnt = 0;
    #pragma unroll 1
    for (int j = j0; j < j1; ++j) {
      psi = ff_add(psi, th[j]);
      float sn, cs;
      sincosf(psi.hi, &sn, &cs);
      const float ux = cs - sn * psi.lo, uy = sn + cs * psi.lo;
      const float L = (j == N - 1) ? l : I.l_seg;
      const float lx = L * ux, ly = L * uy;
      for (int o = 0; o < I.n_obs; ++o) {
        const float4 b4 = ob[o];
        bool hit = false;
        for (int k = 1; k <= ks && !hit; ++k) {
          const float fr = (float)k / (float)ks;
          const FF xk = ff_add(px, fr * lx), yk = ff_add(py, fr * ly);
          float nx, ny, kinv;
          hit = disc_pen(b4, xk, yk, I.R, I.R * (1.f + 1e-6f), -uy, ux, nx, ny, kinv) > 0.f;
        }
        if (hit) {
          if (pass == 1 && base + cnt < max_pairs && pairs) {
            pairs[2 * ((size_t)gw * max_pairs + base + cnt) + 0] = j;
            pairs[2 * ((size_t)gw * max_pairs + base + cnt) + 1] = o;
          }
          ++cnt;
        }
      }
      px = ff_add(px, lx);
      py = ff_add(py, ly);
    }
    if (pass == 0) {
      // exclusive prefix of counts over lanes
      int x = cnt;
      for (int d = 1; d < 32; d <<= 1) {
        int v = __shfl_up_sync(kFull, x, d);
        if (lane >= d) x += v;
      }
      const int total = __shfl_sync(kFull, x, 31);
      base = x - cnt;
      if (lane == 0) counts[gw] = total;
    }
  }
}

}  // namespace

cudaError_t launch_poses(const InstDev* inst, int n_inst, const float* theta, const int* n_cur, const float* l_cur,
                         float* out_theta, float* out_pose, float* out_tip, cudaStream_t s) {
  const int threads = 128;
  const int blocks = (n_inst * 32 + threads - 1) / threads;
  pose_kernel<<<blocks, threads, 0, s>>>(inst, n_inst, nullptr, nullptr, theta, n_cur, l_cur, out_theta, out_pose,
                                         out_tip);
  return cudaGetLastError();
}

cudaError_t launch_poses_sel(const InstDev* inst, const int* sel, const long long* out_off, int n_sel,
                             const float* theta, const int* n_cur, const float* l_cur, float* out_theta,
                             float* out_pose, float* out_tip, cudaStream_t s) {
  if (n_sel <= 0) return cudaSuccess;
  const int threads = 128;
  const int blocks = (n_sel * 32 + threads - 1) / threads;
  pose_kernel<<<blocks, threads, 0, s>>>(inst, n_sel, sel, out_off, theta, n_cur, l_cur, out_theta, out_pose,
                                         out_tip);
  return cudaGetLastError();
}

cudaError_t launch_contacts(const InstDev* inst, int n_inst, const float4* obs, const float* theta, const int* n_cur,
                            const float* l_cur, int ks, int max_pairs, int* counts, int* pairs, cudaStream_t s) {
  const int threads = 128;
  const int blocks = (n_inst * 32 + threads - 1) / threads;
  contacts_kernel<<<blocks, threads, 0, s>>>(inst, n_inst, obs, theta, n_cur, l_cur, ks, max_pairs, counts, pairs);
  return cudaGetLastError();
}

}  // namespace vine
