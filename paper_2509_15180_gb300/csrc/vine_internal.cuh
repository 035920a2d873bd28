// vine_internal.cuh -- device layouts shared by the library's translation units.
//
// HBM layout of a batch (one cudaMalloc, carved in this order):
//   InstDev  inst[n]            80 B per instance: derived constants + CSR offsets
//   float4   obs[n_obs_total]   (cx - bx, cy - by, p, q): circle p = r, q = -(R + r)^2 (1 + 2e-6);
//                               box p = half-width, q = half-height (> 0)
//   float4   act[n_act_total]   (begin, end, P_act, table index as int bits, side in the sign bit)
//   float4   tab_hdr[n_tab]     (eps_lo, h, 1/h, G(0)) per sPAM force table
//   float2   tab[n_tab * 256]   (f_k, G_k): force per pressure at knot k and its
//                               integral from eps_lo
//   float2   utab[NU + 1]       wrinkling energy table (Uhat, mhat) on [theta_c, pi]
//   float    theta[sum n_links] joint angles (CSR by n_links)
//   per-instance state: N, l, status, counters
// Instances never share data; one warp owns one instance at a time.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace vine {

constexpr int kKnots = 256;        // sPAM force table knots (uniform in strain)
constexpr int kUCells = 1024;      // wrinkling energy table cells on [theta_c, pi]
constexpr int kWarpsPerCta = 4;    // warps per CTA of the growth kernel
constexpr int kContactQueue = 8;   // contact candidates a lane queues per link before resolving them
constexpr float kRefinePen = 2e-3f;  // penetrations below this fraction of R are re-evaluated in float-float
constexpr int kListCap = 7;            // obstacles a link's broad-phase list holds
constexpr float kListMargin = 1.0f;    // default broad-phase margin, in body radii
constexpr unsigned short kListStale = 0xffff;  // list not built for the current link geometry
constexpr unsigned short kListFull = 0xfffe;   // more than kListCap obstacles near the link
constexpr int kMaxLinks = 1024;
constexpr int kMaxObs = 1024;
constexpr int kMaxAct = 64;
constexpr float kPi = 3.14159265358979323846f;
constexpr double kPiD = 3.14159265358979323846;

enum InstStatus : int { kOK = 0, kMaxIter = 1, kNonFinite = 2, kBadInput = 3 };

struct __align__(16) InstDev {
  float l_seg, R, P, d;      // d = 2 R + R_act (moment arm, Eq. restoring_moment)
  float kc, kg, PR3, bpsi;   // contact / growth stiffness, pi P R^3, base heading
  float bx, by, pad0, pad1;  // base position (obstacles are stored relative to it)
  int n_target, act_off, n_act, obs_off;
  int n_obs, th_off, n_circ, pad2;
};

struct GrowArgs {
  const InstDev* inst;
  const float4* obs;
  const float4* act;
  const float4* tab_hdr;
  const float2* tab;
  const float2* utab;
  float* theta;
  int* n_cur;
  float* l_cur;
  int* status;
  int* iters;
  int* conv;
  int* steps;
  long long* rls;
  long long* evals;
  long long* linkevals;
  long long* pairtests;  // disc-obstacle pre-tests run (broad phase included)
  long long* fallbacks;  // Newton steps that fell back to the Gauss-Newton matrix
  long long* cycles;     // SM clock cycles the owning warp spent on the robot
  double* resid_max;
  const int* order;
  int n_order;
  int* counter;
  int dynamic;
  int n_steps;
  int nmax, omax, amax, warp_floats;
  // model constants
  float w_a, w_b, w_c;
  float theta_c, inv2thc, inv4thc, eps_c;
  float u_h, u_invh, U_pi, m_pi;
  float fval_eps, c1;
  double tol;       // convergence: predicted displacement <= tol N link lengths ...
  double tol_link;  // ... and <= tol_link link lengths (when > 0)
  int max_iter, max_halv;
  int exact;  // exact Hessian when positive definite (else Gauss-Newton)
  int broad;  // per-link obstacle lists (else every obstacle at every evaluation)
  float list_margin;  // broad-phase margin in body radii
  int mode;           // 0 equilibrium; 1 Algorithm 1 read literally (frozen actuator force, descent)
  int gd_steps;       // mode 1: descent steps per growth step
  float gd_alpha;     // mode 1: step as a fraction of the free-space Newton step
  int team;           // threads per robot: 32 (0 reads as 32) or 64
  int relax;          // 1: re-solve the present links without adding one (vine_relax)
  int fix_l;          // 1: hold the distal length fixed while solving
};

// Descriptor validation and encoding (vine_api.cu): raw device copies of a
// vine_batch_desc in, InstDev / obstacle / actuator records out.
struct InitArgs {
  int n_inst;
  const int32_t* n_links;
  const float *l_seg, *radius, *pressure, *base;
  const int32_t* act_ptr;
  const float *act_begin, *act_end;
  const int8_t* act_side;
  const float *act_pressure, *act_l0;
  const int32_t* obs_ptr;
  const uint8_t* obs_kind;
  const float *obs_cx, *obs_cy, *obs_a, *obs_b;
  const int* act_tab;   // per actuator: sPAM table index
  const int* th_off;    // per instance: offset into theta (batch layout)
  const int* status_h;  // per instance: structural check done on the host
  const int* slot;      // null: batch layout; else per instance its slot (slot layout)
  int nmax_s, omax_s, amax_s;  // slot capacities (slot layout)
  double R_act, w_a, pen_frac;
  InstDev* inst;
  float4* obs;
  float4* act;
  int* status;
};
cudaError_t launch_init(const InitArgs& a, cudaStream_t s);

// Adjoint outputs (vine_grad): device pointers.
struct GradArgs {
  int kind;           // 0: tip cost |p_N - goal|; 1: path cost (1/N) sum_k |p_k - q_k|^2
  const float* goal;  // kind 0: [2 n] goal points; kind 1: [2 sum n_links] link-end targets (absolute, CSR by robot)
  double* cost;       // [n]
  double* dP;         // [n_act_total] d cost / d actuator pressure (per Pa)
  double* dB;         // [n_act_total] d cost / d actuator begin (per link)
  double* dE;         // [n_act_total] d cost / d actuator end (per link)
  int* gstat;         // [n] 0 ok, 1 exact Hessian not positive definite, 2 no valid state
};

// Table build (FP64) -- vine_tables.cu
struct GaussLegendre {
  int n;
  double x[32];
  double w[32];
};

void gauss_legendre(int n, GaussLegendre* gl);
cudaError_t launch_spam_tables(const double* l0, int n_tab, double R_c, double R_act, double a_spam, double m_lo,
                               const GaussLegendre& gl, float4* hdr, float2* tab, double* scratch,
                               cudaStream_t s);
cudaError_t launch_wrinkle_table(double eps_c, const GaussLegendre& gl, float2* utab, double* scratch,
                                 double* consts /*device [4]: U(pi), m(pi), theta_c, h*/, cudaStream_t s);
// Exact sPAM model at (m[i], l0[i]): strain, phi_Rc, force per pressure,
// saturated flag (the surrogate's training data).
cudaError_t launch_spam_samples(int n, const double* m, const double* l0, double R_c, double R_act, double a_spam,
                                const GaussLegendre& gl, double* eps, double* phi, double* f, int* sat,
                                cudaStream_t s);

// Actuator design synthesis (vine_synthesize): sPAM tables for the cell
// lengths l0s[n_l0] (scratch >= (4 + kKnots) n_l0 doubles; hdr / tab as for
// launch_spam_tables), the free-joint equilibrium of every (pressure, cell
// length) pair into theta_pair[n_p n_l0], then the choice per target.  With
// tables_ready the scratch already holds the FP64 bounds and knots of these
// cell lengths (from an earlier call) and the table build is skipped.
cudaError_t launch_synth(int n_targets, const double* target, int n_p, int n_l0, const double* pressures,
                         const double* l0s, double R, double Pv, double ls, double tol, double R_c, double R_act,
                         double a_spam, double m_lo, double eps_c, const GaussLegendre& gl, double* scratch,
                         float4* hdr, float2* tab, double* theta_pair, int* p_index, int* l0_index,
                         double* theta_eq, int tables_ready, cudaStream_t s);

// Thread-local message returned by vine_last_error (fixed storage; vine_api.cu).
void set_last_error(const char* msg, const char* detail = nullptr);

// Growth kernel -- vine_grow.cu
// team: threads per robot, 32 (one warp; several robots per CTA) or 64 (two
// warps; one robot per CTA, a.team = 64 selects that kernel)
cudaError_t launch_grow(const GrowArgs& a, int ks, int grid, int block, size_t smem, cudaStream_t s);
size_t grow_smem_per_warp(int nmax, int omax, int amax, int team = 32);
cudaError_t grow_configure(int ks, size_t smem_per_cta, int team = 32);
int grow_max_ctas_per_sm(int ks, size_t smem_per_cta, int threads, int team = 32);
int grow_pick_block(int ks, size_t smem_warp, int* ctas_per_sm, int team = 32);  // robots per CTA, 0 if none fits
cudaError_t launch_probe(const GrowArgs& a, int ks, int inst, int N, const float* theta, float l, double* J,
                         float* g, float* dx, double* r, int* lfix, size_t smem, cudaStream_t s);
cudaError_t launch_grad(const GrowArgs& a, const GradArgs& g, int ks, int grid, size_t smem, cudaStream_t s);
cudaError_t launch_poses(const InstDev* inst, int n_inst, const float* theta, const int* n_cur, const float* l_cur,
                         float* out_theta, float* out_pose, float* out_tip, cudaStream_t s);
cudaError_t launch_poses_sel(const InstDev* inst, const int* sel, const long long* out_off, int n_sel,
                             const float* theta, const int* n_cur, const float* l_cur, float* out_theta,
                             float* out_pose, float* out_tip, cudaStream_t s);
cudaError_t launch_contacts(const InstDev* inst, int n_inst, const float4* obs, const float* theta, const int* n_cur,
                            const float* l_cur, int ks, int max_pairs, int* counts, int* pairs, cudaStream_t s);

}  // namespace vine
