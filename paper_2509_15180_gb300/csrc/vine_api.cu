// vine_api.cu -- host side of the C ABI declared in include/vine.h.
//
// Batch creation validates the descriptor, builds the FP64 prologue tables on
// the device, orders instances longest-first (cost ~ n_links^2 * n_obs: the
// contact work of a robot grown from one link), sizes the shared-memory slice
// of one warp for the largest robot and obstacle set, and records the
// persistent launch of vine_simulate in a CUDA graph.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <string>
#include <vector>

#include "vine.h"
#include "vine_internal.cuh"

using namespace vine;

namespace vine {
void set_last_error(const char* msg, const char* detail);
}

namespace {

// fixed storage: setting the message never allocates
thread_local char g_err[512];

vine_status fail(vine_status s, const char* msg) {
  std::snprintf(g_err, sizeof(g_err), "%s", msg);
  return s;
}

vine_status cuda_fail(cudaError_t e, const char* where) {
  std::snprintf(g_err, sizeof(g_err), "%s: %s", where, cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? VINE_ENOMEM : VINE_ECUDA;
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(e_, #call);  \
  } while (0)

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

__device__ bool fin(float v) { return isfinite(v); }

// Device-side validation and encoding, one warp per instance.  Batch layout
// (slot == nullptr): instance i at index i, its actuators and obstacles at
// their CSR positions.  Slot layout: instance i goes to slot[i], its
// actuators to slot[i] * amax_s + k, obstacles to slot[i] * omax_s + k and
// joint angles to slot[i] * nmax_s.
__global__ void init_kernel(const InitArgs A) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= A.n_inst) return;
  bool bad = A.status_h[i] != 0;
  const int dst = A.slot ? A.slot[i] : i;
  const float ls = A.l_seg[i], R = A.radius[i], P = A.pressure[i];
  const float bx = A.base[3 * i], by = A.base[3 * i + 1], bpsi = A.base[3 * i + 2];
  bad = bad || !(fin(ls) && ls > 0.f && fin(R) && R > 0.f && fin(P) && P > 0.f && fin(bx) && fin(by) && fin(bpsi));
  const int a0 = A.act_ptr[i], a1 = A.act_ptr[i + 1], o0 = A.obs_ptr[i], o1 = A.obs_ptr[i + 1];
  const int ad = A.slot ? dst * A.amax_s : a0, od = A.slot ? dst * A.omax_s : o0;
  bool badl = false;
  for (int a = a0 + lane; a < a1; a += 32) {
    const float b = A.act_begin[a], e = A.act_end[a], pa = A.act_pressure[a], l0 = A.act_l0[a];
    const int sd = A.act_side[a];
    badl = badl || !(fin(b) && fin(e) && b >= 0.f && e > b && (sd == 1 || sd == -1) && fin(pa) && pa >= 0.f &&
                     fin(l0) && l0 > 0.f);
    int bits = A.act_tab[a] | (sd < 0 ? (int)0x80000000 : 0);
    A.act[ad + (a - a0)] = make_float4(b, e, pa, __int_as_float(bits));
  }
  for (int o = o0 + lane; o < o1; o += 32) {
    const int k = A.obs_kind[o];
    const float cx = A.obs_cx[o], cy = A.obs_cy[o], a = A.obs_a[o], b = A.obs_b[o];
    const float rx = (float)((double)cx - (double)bx), ry = (float)((double)cy - (double)by);
    if (k == 0) {
      badl = badl || !(fin(cx) && fin(cy) && fin(a) && a > 0.f);
      // radius, and the squared contact distance (R + r)^2 with a 2e-6 margin
      // for the FP32 pre-test (the penetration itself is evaluated exactly)
      const double rr = (double)R + (double)a;
      A.obs[od + (o - o0)] = make_float4(rx, ry, a, -(float)(rr * rr * (1.0 + 2e-6)));
    } else {
      badl = badl || !(k == 1 && fin(cx) && fin(cy) && fin(a) && a > 0.f && fin(b) && b > 0.f);
      A.obs[od + (o - o0)] = make_float4(rx, ry, a, b);
    }
  }
  bad = __any_sync(0xffffffffu, badl) || bad;
  if (lane == 0) {
    InstDev d;
    const double Rd = R, Pd = P, ld = ls;
    d.l_seg = ls;
    d.R = R;
    d.P = P;
    d.d = (float)(2.0 * Rd + A.R_act);
    d.kc = (float)(A.w_a * kPiD * Pd * Rd * Rd * Rd / (2.0 * A.pen_frac * Rd * ld));
    d.kg = (float)(kPiD * Pd * Rd * Rd / (2.0 * ld));
    d.PR3 = (float)(kPiD * Pd * Rd * Rd * Rd);
    d.bpsi = bpsi;
    d.bx = bx;
    d.by = by;
    d.pad0 = d.pad1 = 0.f;
    d.n_target = A.n_links[i];
    d.act_off = ad;
    d.n_act = a1 - a0;
    d.obs_off = od;
    d.n_obs = o1 - o0;
    d.th_off = A.slot ? dst * A.nmax_s : A.th_off[i];
    d.n_circ = 0;
    d.pad2 = 0;
    A.inst[dst] = d;
    A.status[dst] = bad ? kBadInput : kOK;
  }
}

// New actuator pressures and spans for every instance (one warp per
// instance); the side and table index are kept.  Invalid values mark the
// instance BADINPUT, in the validated status too (so reset keeps it).
__global__ void actuator_update_kernel(const InstDev* inst, int n_inst, const float* pressure, const float* begin,
                                       const float* end, float4* act, int* status0, int* status) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n_inst) return;
  const InstDev I = inst[i];
  bool badl = false;
  for (int k = lane; k < I.n_act; k += 32) {
    const int a = I.act_off + k;
    const float b = begin[a], e = end[a], pa = pressure[a];
    badl = badl || !(fin(b) && fin(e) && b >= 0.f && e > b && fin(pa) && pa >= 0.f);
    act[a] = make_float4(b, e, pa, act[a].w);
  }
  if (__any_sync(0xffffffffu, badl) && lane == 0) {
    status0[i] = kBadInput;
    status[i] = kBadInput;
  }
}

// Loads caller states (vine_set_state), one warp per instance: the present
// link count, the joint angles in the batch's CSR layout and the distal
// length.  Entries past the present links are zeroed, as growth leaves them.
// A state outside its ranges marks the instance BADINPUT and leaves it empty.
__global__ void state_load_kernel(const InstDev* inst, int n_inst, const int* n_present, const float* theta,
                                  const float* l_last, float* th, int* n_cur, float* l_cur, const int* status0,
                                  int* status) {
  const int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (i >= n_inst) return;
  const InstDev I = inst[i];
  const int N = n_present[i];
  bool bad = !(N >= 0 && N <= I.n_target);
  const int n_ok = bad ? 0 : N;
  bool badl = false;
  for (int k = lane; k < I.n_target; k += 32) {
    const float t = k < n_ok ? theta[I.th_off + k] : 0.f;
    badl = badl || !fin(t);
    th[I.th_off + k] = t;
  }
  bad = __any_sync(0xffffffffu, badl) || bad;
  const float l = n_ok > 0 ? l_last[i] : 0.f;
  bad = bad || !(fin(l) && l >= 0.f && l <= I.l_seg);
  if (lane == 0) {
    n_cur[i] = bad ? 0 : N;
    l_cur[i] = bad ? 0.f : l;
    status[i] = (bad || status0[i] == kBadInput) ? kBadInput : status0[i];
  }
}

// Prologue tables already built in this process, per device: the
// wrinkling-energy table depends only on eps_crit, an sPAM force table only
// on its cell length and the sPAM constants.  Batch creation copies a cached
// table (device to device) instead of rebuilding it; the kernels that build
// them are deterministic, so the copy is bitwise the table a rebuild gives.
// Entries live until the process exits (2 KB per sPAM table, 8 KB per
// wrinkling table, at most kCacheSpam + kCacheWrinkle entries).
constexpr size_t kCacheSpam = 4096, kCacheWrinkle = 16;
struct SpamEntry {
  int dev;
  double l0, R_c, R_act, a, m_lo;
  float4* hdr;   // [1]
  float2* tab;   // [kKnots]
};
struct WrinkleEntry {
  int dev;
  double eps;
  float2* utab;  // [kUCells + 1]
  double cst[4];
};
// The FP64 sPAM bounds and knots of one synthesis grid of cell lengths
// (l0_min + k l0_step, k < n_l0), which vine_synthesize would otherwise
// rebuild on every call; at most kCacheSynth grids.
constexpr size_t kCacheSynth = 8;
struct SynthEntry {
  int dev;
  double l0_min, l0_step, R_c, R_act, a, m_lo;
  int n_l0;
  double* scr;  // [(4 + kKnots) n_l0]
};
struct TableCache {
  std::mutex mu;
  std::vector<SpamEntry> spam;
  std::vector<WrinkleEntry> wrinkle;
  std::vector<SynthEntry> synth;
};
TableCache& table_cache() {
  static TableCache* c = new TableCache();  // never destroyed: outlives CUDA teardown at exit
  return *c;
}
const SpamEntry* find_spam(const TableCache& c, int dev, double l0, const vine_params& p) {
  for (const SpamEntry& e : c.spam)
    if (e.dev == dev && e.l0 == l0 && e.R_c == p.R_c && e.R_act == p.R_act && e.a == p.a_spam && e.m_lo == p.m_lo)
      return &e;
  return nullptr;
}
const SynthEntry* find_synth(const TableCache& c, int dev, const vine_synth_spec& g, const vine_params& p) {
  for (const SynthEntry& e : c.synth)
    if (e.dev == dev && e.l0_min == g.l0_min && e.l0_step == g.l0_step && e.n_l0 == g.n_l0 && e.R_c == p.R_c &&
        e.R_act == p.R_act && e.a == p.a_spam && e.m_lo == p.m_lo)
      return &e;
  return nullptr;
}
const WrinkleEntry* find_wrinkle(const TableCache& c, int dev, double eps) {
  for (const WrinkleEntry& e : c.wrinkle)
    if (e.dev == dev && e.eps == eps) return &e;
  return nullptr;
}

}  // namespace

cudaError_t vine::launch_init(const InitArgs& a, cudaStream_t s) {
  if (a.n_inst <= 0) return cudaSuccess;
  init_kernel<<<(a.n_inst * 32 + 127) / 128, 128, 0, s>>>(a);
  return cudaGetLastError();
}

void vine::set_last_error(const char* msg, const char* detail) {
  std::snprintf(g_err, sizeof(g_err), "%s%s", msg, detail ? detail : "");
}

// One length class of a batch: its robots (a segment of the longest-first
// order) grow in one persistent launch of their own team size, shared-memory
// slice and work counter.
struct LaunchClass {
  int team = 32;             // threads per robot
  int wpc = kWarpsPerCta;    // robots (teams) per CTA
  int grid = 1;
  int nmax = 32, omax = 1, amax = 1, max_target = 0;
  size_t smem_warp = 0;      // shared memory per robot slice
  int off = 0, count = 0;    // segment of the order
};
constexpr int kMaxClass = 3;

struct vine_batch {
  int device = 0;
  int n_inst = 0;
  int64_t total_links = 0;
  int n_act = 0;
  int n_tab = 0;
  vine_params params{};
  int ks = 2;
  int n_class = 1;
  LaunchClass cls[kMaxClass];  // the longest robots' class first
  float margin = kListMargin;  // broad-phase margin of the growth launches
  size_t smem_warp = 0;  // one-warp slice for the batch's largest robot (adjoint, probe)
  int max_target = 0;
  cudaStream_t aux[kMaxClass - 1] = {};  // the other classes' launch streams
  cudaEvent_t ev_fork = nullptr, ev_join[kMaxClass - 1] = {};
  void* dmem = nullptr;
  void* stage = nullptr;  // lazily allocated host-output staging
  size_t stage_bytes = 0;
  GrowArgs args{};
  int* status0 = nullptr;  // status after validation (restored by reset)
  cudaStream_t cap_stream = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  std::vector<int> h_n_links, h_n_obs, h_n_circ;
  std::vector<int> h_order;
};

static void release_launch_streams(vine_batch* B) {
  for (int c = 0; c < kMaxClass - 1; ++c) {
    if (B->aux[c]) cudaStreamDestroy(B->aux[c]);
    if (B->ev_join[c]) cudaEventDestroy(B->ev_join[c]);
    B->aux[c] = nullptr;
    B->ev_join[c] = nullptr;
  }
  if (B->ev_fork) cudaEventDestroy(B->ev_fork);
  B->ev_fork = nullptr;
}

// Growth launch of the classes L[0..nc) over the robots d_order[L[c].off ..
// + L[c].count): class 0 on stream st, the others on the batch's streams,
// forked from st and joined back (parallel branches of a captured graph).
// The longest robots' class is launched first and so takes the SMs first;
// the other classes' CTAs fill them as its queue drains.
static cudaError_t launch_classes(vine_batch* B, const LaunchClass* L, int nc, const int* d_order, int n_steps,
                                  float margin, int relax, int fix_l, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(B->args.counter, 0, sizeof(int) * 4, st);
  if (e == cudaSuccess && nc > 1) {
    e = cudaEventRecord(B->ev_fork, st);
    for (int c = 1; c < nc && e == cudaSuccess; ++c) e = cudaStreamWaitEvent(B->aux[c - 1], B->ev_fork, 0);
  }
  for (int c = 0; c < nc && e == cudaSuccess; ++c) {
    GrowArgs a = B->args;
    a.order = d_order + L[c].off;
    a.n_order = L[c].count;
    a.counter = B->args.counter + c;
    a.nmax = L[c].nmax;
    a.omax = L[c].omax;
    a.amax = L[c].amax;
    a.warp_floats = (int)(L[c].smem_warp / sizeof(float));
    a.team = L[c].team;
    a.n_steps = n_steps;
    a.dynamic = 1;
    a.relax = relax;
    a.fix_l = fix_l;
    a.list_margin = margin;
    const cudaStream_t s = c == 0 ? st : B->aux[c - 1];
    e = grow_configure(B->ks, L[c].smem_warp * L[c].wpc, L[c].team);
    if (e == cudaSuccess) e = launch_grow(a, B->ks, L[c].grid, L[c].team * L[c].wpc, L[c].smem_warp * L[c].wpc, s);
    if (e == cudaSuccess && c > 0) {
      e = cudaEventRecord(B->ev_join[c - 1], s);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(st, B->ev_join[c - 1], 0);
    }
  }
  return e;
}

extern "C" {

const char* vine_last_error(void) { return g_err; }

vine_status vine_params_default(vine_params* p) {
  if (!p) return fail(VINE_EINVAL, "vine_params_default: null pointer");
  std::memset(p, 0, sizeof(*p));
  p->w_a = 160.0;
  p->w_b = 15.0;
  p->w_c = 1.0;
  p->eps_crit = 0.01;
  p->R_c = 0.005;
  p->R_act = 0.01718;
  p->a_spam = 1e-4;
  p->m_lo = 0.002;
  p->pen_frac = 0.01;
  p->tol = 1e-6;
  p->fval_eps = 1e-6;
  p->armijo_c1 = 1e-4;
  p->max_iter = 100;
  p->discs_per_link = 2;
  p->max_halvings = 30;
  p->mode = 0;
  p->gd_alpha = 0.005;
  p->gd_steps = 50;
  p->exact_hessian = 1;
  p->broad_phase = 1;
  p->threads_per_robot = 0;
  p->tol_link = 2.5e-5;
  return VINE_OK;
}

static vine_status copy_in(void* dst, const void* src, size_t bytes, int is_dev) {
  if (bytes == 0) return VINE_OK;
  if (!src) return fail(VINE_EINVAL, "vine_batch_create: null input array");
  if (is_dev) {
    CK(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost));
  } else {
    std::memcpy(dst, src, bytes);
  }
  return VINE_OK;
}

vine_status vine_batch_create(const vine_batch_desc* D, const vine_params* P, void* stream_v, vine_batch** out) {
  if (!D || !out) return fail(VINE_EINVAL, "vine_batch_create: null descriptor or output");
  *out = nullptr;
  vine_params prm;
  if (P) prm = *P; else vine_params_default(&prm);
  if (prm.discs_per_link < 1 || prm.discs_per_link > 4)
    return fail(VINE_EINVAL, "vine_batch_create: discs_per_link must be 1..4");
  if (!(prm.tol > 0.0) || prm.max_iter < 1 || prm.max_halvings < 0 || !(prm.eps_crit > 0.0 && prm.eps_crit < 1.0) ||
      !(prm.R_c > 0.0 && prm.R_act > prm.R_c) || !(prm.m_lo > 0.0 && prm.m_lo < 0.5) || !(prm.pen_frac > 0.0) || !(prm.fval_eps >= 0.0) || !(prm.armijo_c1 > 0.0 && prm.armijo_c1 < 0.5) ||
      (prm.mode != 0 && prm.mode != 1) || (prm.mode == 1 && (prm.gd_steps < 1 || !(prm.gd_alpha > 0.0))) ||
      (prm.threads_per_robot != 0 && prm.threads_per_robot != 32 && prm.threads_per_robot != 64 &&
       prm.threads_per_robot != 128))
    return fail(VINE_EINVAL, "vine_batch_create: parameter out of range");
  const int n = D->n_inst;
  if (n <= 0) return fail(VINE_EINVAL, "vine_batch_create: n_inst must be positive");
  const int dev = D->mem_is_device ? 1 : 0;
  cudaStream_t st = (cudaStream_t)stream_v;

  // ---- structure on the host
  std::vector<int32_t> nl(n), aptr(n + 1), optr(n + 1);
  vine_status s;
  if ((s = copy_in(nl.data(), D->n_links, sizeof(int32_t) * n, dev)) != VINE_OK) return s;
  if ((s = copy_in(aptr.data(), D->act_ptr, sizeof(int32_t) * (n + 1), dev)) != VINE_OK) return s;
  if ((s = copy_in(optr.data(), D->obs_ptr, sizeof(int32_t) * (n + 1), dev)) != VINE_OK) return s;
  if (aptr[0] != 0 || optr[0] != 0) return fail(VINE_EINVAL, "vine_batch_create: act_ptr/obs_ptr must start at 0");
  for (int i = 0; i < n; ++i)
    if (aptr[i + 1] < aptr[i] || optr[i + 1] < optr[i])
      return fail(VINE_EINVAL, "vine_batch_create: act_ptr/obs_ptr must be non-decreasing");
  const int n_act = aptr[n], n_obs = optr[n];
  std::vector<float> l0(n_act);
  std::vector<uint8_t> kind(n_obs);
  if ((s = copy_in(l0.data(), D->act_l0, sizeof(float) * n_act, dev)) != VINE_OK) return s;
  if ((s = copy_in(kind.data(), D->obs_kind, n_obs, dev)) != VINE_OK) return s;

  auto B = new vine_batch();
  B->params = prm;
  B->ks = prm.discs_per_link;
  B->n_inst = n;
  cudaGetDevice(&B->device);
  std::vector<int> status_h(n, 0), th_off(n, 0);
  B->h_n_links.resize(n);
  B->h_n_obs.resize(n);
  B->h_n_circ.resize(n);
  int64_t tot = 0;
  int nmax = 1, omax = 1, amax = 1;
  for (int i = 0; i < n; ++i) {
    const int nli = nl[i], na = aptr[i + 1] - aptr[i], no = optr[i + 1] - optr[i];
    const bool ok = nli >= 1 && nli <= kMaxLinks && na <= kMaxAct && no <= kMaxObs;
    status_h[i] = ok ? 0 : 1;
    th_off[i] = (int)tot;
    const int cap = std::max(nli, 0);
    tot += cap;
    B->h_n_links[i] = ok ? nli : 0;
    B->h_n_obs[i] = no;
    int nc = 0;
    for (int o = optr[i]; o < optr[i + 1]; ++o) nc += kind[o] == 0;
    B->h_n_circ[i] = nc;
    if (ok) {
      nmax = std::max(nmax, nli);
      omax = std::max(omax, no);
      amax = std::max(amax, na);
    }
  }
  if (tot > (int64_t)1 << 30) {
    delete B;
    return fail(VINE_EINVAL, "vine_batch_create: too many links in one batch");
  }
  B->total_links = tot;
  B->max_target = nmax;
  // ---- distinct sPAM cell lengths
  std::vector<double> tabs;
  std::vector<int> act_tab(n_act, 0);
  for (int a = 0; a < n_act; ++a) {
    const double v = l0[a];
    if (!(std::isfinite(v) && v > 0.0)) continue;  // flagged bad on the device
    auto it = std::find(tabs.begin(), tabs.end(), v);
    if (it == tabs.end()) {
      tabs.push_back(v);
      act_tab[a] = (int)tabs.size() - 1;
    } else {
      act_tab[a] = (int)(it - tabs.begin());
    }
  }
  B->n_tab = (int)tabs.size();
  B->n_act = n_act;
  const int nt = std::max(B->n_tab, 1);

  // ---- device memory
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(std::max<size_t>(bytes, 16));
    return o;
  };
  const size_t o_inst = take(sizeof(InstDev) * n), o_obs = take(sizeof(float4) * n_obs),
               o_act = take(sizeof(float4) * n_act), o_hdr = take(sizeof(float4) * nt),
               o_tab = take(sizeof(float2) * nt * kKnots), o_ut = take(sizeof(float2) * (kUCells + 1)),
               o_th = take(sizeof(float) * tot), o_n = take(sizeof(int) * n), o_l = take(sizeof(float) * n),
               o_st = take(sizeof(int) * n), o_st0 = take(sizeof(int) * n), o_it = take(sizeof(int) * n),
               o_cv = take(sizeof(int) * n), o_sp = take(sizeof(int) * n), o_rls = take(sizeof(long long) * n),
               o_ev = take(sizeof(long long) * n), o_le = take(sizeof(long long) * n),
               o_fb = take(sizeof(long long) * n), o_cy = take(sizeof(long long) * n),
               o_pt = take(sizeof(long long) * n), o_rm = take(sizeof(double) * n), o_ord = take(sizeof(int) * n),
               o_cnt = take(sizeof(int) * 4);
  const size_t persistent = off;
  // setup scratch (freed at the end of create)
  const size_t o_acttab = take(sizeof(int) * n_act), o_thoff = take(sizeof(int) * n),
               o_sth = take(sizeof(int) * n), o_l0 = take(sizeof(double) * nt),
               o_scr = take(sizeof(double) * (4 * nt + nt * kKnots + 2 * (kUCells + 1))),
               o_cst = take(sizeof(double) * 4);
  size_t o_raw = 0, raw_bytes = 0;
  if (!dev) {
    raw_bytes = sizeof(int32_t) * n + sizeof(float) * 6 * n + sizeof(int32_t) * 2 * (n + 1) +
                (sizeof(float) * 4 + 1) * n_act + (sizeof(float) * 4 + 1) * n_obs + 4096;
    o_raw = take(raw_bytes);
  }
  char* mem = nullptr;
  cudaError_t e = cudaMalloc(&mem, off);
  if (e != cudaSuccess) {
    delete B;
    return cuda_fail(e, "vine_batch_create: cudaMalloc");
  }
  B->dmem = mem;
  auto P_ = [&](size_t o) { return (void*)(mem + o); };

  // raw inputs on the device
  InitArgs ia{};
  ia.n_inst = n;
  if (dev) {
    ia.n_links = D->n_links; ia.l_seg = D->l_seg; ia.radius = D->radius; ia.pressure = D->pressure;
    ia.base = D->base; ia.act_ptr = D->act_ptr; ia.act_begin = D->act_begin; ia.act_end = D->act_end;
    ia.act_side = D->act_side; ia.act_pressure = D->act_pressure; ia.act_l0 = D->act_l0; ia.obs_ptr = D->obs_ptr;
    ia.obs_kind = D->obs_kind; ia.obs_cx = D->obs_cx; ia.obs_cy = D->obs_cy; ia.obs_a = D->obs_a;
    ia.obs_b = D->obs_b;
  } else {
    char* r = (char*)P_(o_raw);
    size_t ro = 0;
    auto put = [&](const void* src, size_t bytes) -> const void* {
      char* d = r + ro;
      if (bytes) {
        cudaMemcpyAsync(d, src, bytes, cudaMemcpyHostToDevice, st);
      }
      ro += (bytes + 15) & ~size_t(15);
      return d;
    };
    const bool ok_ptrs = D->n_links && D->l_seg && D->radius && D->pressure && D->base && D->act_ptr &&
                         D->obs_ptr && (n_act == 0 || (D->act_begin && D->act_end && D->act_side &&
                                                        D->act_pressure && D->act_l0)) &&
                         (n_obs == 0 || (D->obs_kind && D->obs_cx && D->obs_cy && D->obs_a && D->obs_b));
    if (!ok_ptrs) {
      cudaFree(mem);
      delete B;
      return fail(VINE_EINVAL, "vine_batch_create: null input array");
    }
    ia.n_links = (const int32_t*)put(D->n_links, 4 * n);
    ia.l_seg = (const float*)put(D->l_seg, 4 * n);
    ia.radius = (const float*)put(D->radius, 4 * n);
    ia.pressure = (const float*)put(D->pressure, 4 * n);
    ia.base = (const float*)put(D->base, 12 * n);
    ia.act_ptr = (const int32_t*)put(D->act_ptr, 4 * (n + 1));
    ia.act_begin = (const float*)put(D->act_begin, 4 * n_act);
    ia.act_end = (const float*)put(D->act_end, 4 * n_act);
    ia.act_side = (const int8_t*)put(D->act_side, n_act);
    ia.act_pressure = (const float*)put(D->act_pressure, 4 * n_act);
    ia.act_l0 = (const float*)put(D->act_l0, 4 * n_act);
    ia.obs_ptr = (const int32_t*)put(D->obs_ptr, 4 * (n + 1));
    ia.obs_kind = (const uint8_t*)put(D->obs_kind, n_obs);
    ia.obs_cx = (const float*)put(D->obs_cx, 4 * n_obs);
    ia.obs_cy = (const float*)put(D->obs_cy, 4 * n_obs);
    ia.obs_a = (const float*)put(D->obs_a, 4 * n_obs);
    ia.obs_b = (const float*)put(D->obs_b, 4 * n_obs);
  }
  auto cleanup = [&]() {
    cudaFree(mem);
    release_launch_streams(B);
    delete B;
  };
#define CKC(call)                                    \
  do {                                               \
    cudaError_t e_ = (call);                         \
    if (e_ != cudaSuccess) {                         \
      vine_status s_ = cuda_fail(e_, #call);         \
      cleanup();                                     \
      return s_;                                     \
    }                                                \
  } while (0)
  CKC(cudaMemcpyAsync(P_(o_acttab), act_tab.data(), sizeof(int) * n_act, cudaMemcpyHostToDevice, st));
  CKC(cudaMemcpyAsync(P_(o_thoff), th_off.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  CKC(cudaMemcpyAsync(P_(o_sth), status_h.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  if (B->n_tab) CKC(cudaMemcpyAsync(P_(o_l0), tabs.data(), sizeof(double) * B->n_tab, cudaMemcpyHostToDevice, st));
  ia.act_tab = (const int*)P_(o_acttab);
  ia.th_off = (const int*)P_(o_thoff);
  ia.status_h = (const int*)P_(o_sth);
  ia.R_act = prm.R_act;
  ia.w_a = prm.w_a;
  ia.pen_frac = prm.pen_frac;
  ia.inst = (InstDev*)P_(o_inst);
  ia.obs = (float4*)P_(o_obs);
  ia.act = (float4*)P_(o_act);
  ia.status = (int*)P_(o_st);
  // zero the per-instance state block (n .. resid) before validation writes status
  CKC(cudaMemsetAsync(P_(o_n), 0, (size_t)(o_ord - o_n), st));
  CKC(cudaMemsetAsync(P_(o_th), 0, sizeof(float) * std::max<int64_t>(tot, 1), st));
  CKC(launch_init(ia, st));
  CKC(cudaMemcpyAsync(P_(o_st0), P_(o_st), sizeof(int) * n, cudaMemcpyDeviceToDevice, st));
  // prologue tables: copied from the process's table cache where present,
  // else built (FP64) and added to it after the synchronisation below
  GaussLegendre gl;
  gauss_legendre(24, &gl);
  double* scr = (double*)P_(o_scr);
  int cur_dev = 0;
  cudaGetDevice(&cur_dev);
  bool spam_cached = true, wrinkle_cached = false;
  double cst[4];
  {
    TableCache& tc = table_cache();
    std::lock_guard<std::mutex> lk(tc.mu);
    for (int t = 0; t < B->n_tab && spam_cached; ++t) spam_cached = find_spam(tc, cur_dev, tabs[t], prm) != nullptr;
    if (spam_cached) {
      for (int t = 0; t < B->n_tab; ++t) {
        const SpamEntry* e = find_spam(tc, cur_dev, tabs[t], prm);
        CKC(cudaMemcpyAsync((float4*)P_(o_hdr) + t, e->hdr, sizeof(float4), cudaMemcpyDeviceToDevice, st));
        CKC(cudaMemcpyAsync((float2*)P_(o_tab) + (size_t)t * kKnots, e->tab, sizeof(float2) * kKnots,
                            cudaMemcpyDeviceToDevice, st));
      }
    }
    if (const WrinkleEntry* e = find_wrinkle(tc, cur_dev, prm.eps_crit)) {
      wrinkle_cached = true;
      CKC(cudaMemcpyAsync(P_(o_ut), e->utab, sizeof(float2) * (kUCells + 1), cudaMemcpyDeviceToDevice, st));
      std::memcpy(cst, e->cst, sizeof(cst));
    }
  }
  if (!spam_cached)
    CKC(launch_spam_tables((const double*)P_(o_l0), B->n_tab, prm.R_c, prm.R_act, prm.a_spam, prm.m_lo, gl,
                           (float4*)P_(o_hdr), (float2*)P_(o_tab), scr, st));
  if (!wrinkle_cached) {
    CKC(launch_wrinkle_table(prm.eps_crit, gl, (float2*)P_(o_ut), scr + 4 * nt + nt * kKnots, (double*)P_(o_cst),
                             st));
    CKC(cudaMemcpyAsync(cst, P_(o_cst), sizeof(cst), cudaMemcpyDeviceToHost, st));
  }
  // longest-first order
  B->h_order.resize(n);
  std::iota(B->h_order.begin(), B->h_order.end(), 0);
  std::vector<double> cost(n);
  for (int i = 0; i < n; ++i)
    cost[i] = (double)B->h_n_links[i] * B->h_n_links[i] * (B->ks * (double)B->h_n_obs[i] + 8.0);
  std::stable_sort(B->h_order.begin(), B->h_order.end(), [&](int a, int b) { return cost[a] > cost[b]; });
  CKC(cudaMemcpyAsync(P_(o_ord), B->h_order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
  CKC(cudaStreamSynchronize(st));
  if (!(std::isfinite(cst[0]) && std::isfinite(cst[1]))) {
    cleanup();
    return fail(VINE_ECUDA, "vine_batch_create: wrinkling table build failed");
  }
  if (!spam_cached || !wrinkle_cached) {  // keep the tables just built (best effort: a failed copy is not cached)
    TableCache& tc = table_cache();
    std::lock_guard<std::mutex> lk(tc.mu);
    if (!wrinkle_cached && tc.wrinkle.size() < kCacheWrinkle && !find_wrinkle(tc, cur_dev, prm.eps_crit)) {
      WrinkleEntry e{cur_dev, prm.eps_crit, nullptr, {cst[0], cst[1], cst[2], cst[3]}};
      if (cudaMalloc(&e.utab, sizeof(float2) * (kUCells + 1)) == cudaSuccess) {
        if (cudaMemcpyAsync(e.utab, P_(o_ut), sizeof(float2) * (kUCells + 1), cudaMemcpyDeviceToDevice, st) ==
                cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess)
          tc.wrinkle.push_back(e);
        else
          cudaFree(e.utab);
      }
    }
    for (int t = 0; !spam_cached && t < B->n_tab && tc.spam.size() < kCacheSpam; ++t) {
      if (find_spam(tc, cur_dev, tabs[t], prm)) continue;
      SpamEntry e{cur_dev, tabs[t], prm.R_c, prm.R_act, prm.a_spam, prm.m_lo, nullptr, nullptr};
      char* m = nullptr;
      if (cudaMalloc(&m, sizeof(float4) + sizeof(float2) * kKnots) != cudaSuccess) break;
      e.hdr = (float4*)m;
      e.tab = (float2*)(m + sizeof(float4));
      if (cudaMemcpyAsync(e.hdr, (float4*)P_(o_hdr) + t, sizeof(float4), cudaMemcpyDeviceToDevice, st) ==
              cudaSuccess &&
          cudaMemcpyAsync(e.tab, (float2*)P_(o_tab) + (size_t)t * kKnots, sizeof(float2) * kKnots,
                          cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
          cudaStreamSynchronize(st) == cudaSuccess)
        tc.spam.push_back(e);
      else
        cudaFree(m);
    }
    cudaGetLastError();  // a failed cache copy leaves no sticky error for the caller
  }
  // ---- launch configuration: length classes (threads per robot by the
  // robot's length: 32 up to 64 links, 64 up to 200, 128 beyond), or one
  // class of the caller's team size
  int dev_id = 0, nsm = 1;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev_id);
  {
    auto team_of = [&](int nl) {
      if (prm.threads_per_robot != 0) return prm.threads_per_robot;
      return nl <= 64 ? 32 : (nl <= 200 ? 64 : 128);
    };
    const int teams[kMaxClass] = {128, 64, 32};
    std::vector<int> by_class;
    by_class.reserve(n);
    B->n_class = 0;
    for (int t : teams) {
      LaunchClass L;
      L.team = t;
      L.off = (int)by_class.size();
      int cn = 1, co = 1, ca = 1;
      for (int i : B->h_order) {
        // robots with bad input stop at once: they ride in the last class
        const int ti = B->h_n_links[i] > 0 ? team_of(B->h_n_links[i]) : -1;
        if (ti != t && !(ti < 0 && t == 32)) continue;
        by_class.push_back(i);
        cn = std::max(cn, B->h_n_links[i]);
        co = std::max(co, B->h_n_obs[i]);
        ca = std::max(ca, aptr[i + 1] - aptr[i]);
      }
      L.count = (int)by_class.size() - L.off;
      if (L.count == 0) continue;
      L.max_target = cn;
      L.nmax = (cn + 31) & ~31;
      L.omax = co;
      L.amax = ca;
      L.smem_warp = grow_smem_per_warp(L.nmax, L.omax, L.amax, L.team);
      int per_sm = 0;
      L.wpc = grow_pick_block(B->ks, L.smem_warp, &per_sm, L.team);
      if (L.wpc == 0 || per_sm == 0) {
        cleanup();
        return fail(VINE_EINVAL, "vine_batch_create: robot or obstacle set too large for shared memory");
      }
      L.grid = std::max(1, std::min((L.count + L.wpc - 1) / L.wpc, nsm * per_sm));
      B->cls[B->n_class++] = L;
    }
    B->h_order = by_class;  // class by class, longest first within each
    CKC(cudaMemcpyAsync(P_(o_ord), B->h_order.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st));
    for (int c = 1; c < B->n_class; ++c) {
      CKC(cudaStreamCreateWithFlags(&B->aux[c - 1], cudaStreamNonBlocking));
      CKC(cudaEventCreateWithFlags(&B->ev_join[c - 1], cudaEventDisableTiming));
    }
    if (B->n_class > 1) CKC(cudaEventCreateWithFlags(&B->ev_fork, cudaEventDisableTiming));
    CKC(cudaStreamSynchronize(st));
  }
  B->smem_warp = grow_smem_per_warp((nmax + 31) & ~31, omax, amax, 32);

  GrowArgs& a = B->args;
  a.inst = (const InstDev*)P_(o_inst);
  a.obs = (const float4*)P_(o_obs);
  a.act = (const float4*)P_(o_act);
  a.tab_hdr = (const float4*)P_(o_hdr);
  a.tab = (const float2*)P_(o_tab);
  a.utab = (const float2*)P_(o_ut);
  a.theta = (float*)P_(o_th);
  a.n_cur = (int*)P_(o_n);
  a.l_cur = (float*)P_(o_l);
  a.status = (int*)P_(o_st);
  a.iters = (int*)P_(o_it);
  a.conv = (int*)P_(o_cv);
  a.steps = (int*)P_(o_sp);
  a.rls = (long long*)P_(o_rls);
  a.evals = (long long*)P_(o_ev);
  a.linkevals = (long long*)P_(o_le);
  a.pairtests = (long long*)P_(o_pt);
  a.fallbacks = (long long*)P_(o_fb);
  a.cycles = (long long*)P_(o_cy);
  a.resid_max = (double*)P_(o_rm);
  a.order = (const int*)P_(o_ord);
  a.n_order = n;
  a.counter = (int*)P_(o_cnt);
  a.dynamic = 1;
  a.n_steps = 0;
  a.nmax = (nmax + 31) & ~31;  // the batch's largest robot (adjoint and probe, one warp)
  a.omax = omax;
  a.amax = amax;
  a.warp_floats = (int)(B->smem_warp / sizeof(float));
  a.w_a = (float)prm.w_a;
  a.w_b = (float)prm.w_b;
  a.w_c = (float)prm.w_c;
  a.theta_c = (float)cst[2];
  a.inv2thc = (float)(1.0 / (2.0 * cst[2]));
  a.inv4thc = (float)(1.0 / (4.0 * cst[2]));
  a.eps_c = (float)prm.eps_crit;
  a.u_h = (float)cst[3];
  a.u_invh = (float)(1.0 / cst[3]);
  a.U_pi = (float)cst[0];
  a.m_pi = (float)cst[1];
  a.fval_eps = (float)prm.fval_eps;
  a.c1 = (float)prm.armijo_c1;
  a.tol = prm.tol;
  a.tol_link = prm.tol_link;
  a.max_iter = prm.max_iter;
  a.max_halv = prm.max_halvings;
  a.exact = prm.exact_hessian;
  a.broad = prm.broad_phase;
  a.team = 32;
  a.mode = prm.mode;
  a.gd_steps = prm.gd_steps;
  a.gd_alpha = (float)prm.gd_alpha;
  a.list_margin = kListMargin;
  B->status0 = (int*)P_(o_st0);
  (void)persistent;
  *out = B;
#undef CKC
  return VINE_OK;
}

static vine_status grow_launch(vine_batch* B, int n_steps, cudaStream_t st, int relax = 0, int fix_l = 0) {
  CK(launch_classes(B, B->cls, B->n_class, B->args.order, n_steps, B->margin, relax, fix_l, st));
  return VINE_OK;
}

vine_status vine_batch_reset(vine_batch* B, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_batch_reset: null batch");
  cudaStream_t st = (cudaStream_t)stream_v;
  const GrowArgs& a = B->args;
  CK(cudaMemsetAsync(a.theta, 0, sizeof(float) * std::max<int64_t>(B->total_links, 1), st));
  CK(cudaMemsetAsync(a.n_cur, 0, sizeof(int) * B->n_inst, st));
  CK(cudaMemsetAsync(a.l_cur, 0, sizeof(float) * B->n_inst, st));
  CK(cudaMemsetAsync(a.iters, 0, sizeof(int) * B->n_inst, st));
  CK(cudaMemsetAsync(a.conv, 0, sizeof(int) * B->n_inst, st));
  CK(cudaMemsetAsync(a.steps, 0, sizeof(int) * B->n_inst, st));
  CK(cudaMemsetAsync(a.rls, 0, sizeof(long long) * B->n_inst, st));
  CK(cudaMemsetAsync(a.evals, 0, sizeof(long long) * B->n_inst, st));
  CK(cudaMemsetAsync(a.linkevals, 0, sizeof(long long) * B->n_inst, st));
  CK(cudaMemsetAsync(a.pairtests, 0, sizeof(long long) * B->n_inst, st));
  CK(cudaMemsetAsync(a.fallbacks, 0, sizeof(long long) * B->n_inst, st));
  CK(cudaMemsetAsync(a.cycles, 0, sizeof(long long) * B->n_inst, st));
  CK(cudaMemsetAsync(a.resid_max, 0, sizeof(double) * B->n_inst, st));
  CK(cudaMemcpyAsync(a.status, B->status0, sizeof(int) * B->n_inst, cudaMemcpyDeviceToDevice, st));
  return VINE_OK;
}

vine_status vine_grow_step(vine_batch* B, int32_t n_steps, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_grow_step: null batch");
  if (n_steps < 0) return fail(VINE_EINVAL, "vine_grow_step: negative step count");
  if (n_steps == 0) return VINE_OK;
  return grow_launch(B, n_steps, (cudaStream_t)stream_v);
}

vine_status vine_relax(vine_batch* B, int32_t fix_length, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_relax: null batch");
  if (fix_length != 0 && fix_length != 1) return fail(VINE_EINVAL, "vine_relax: fix_length must be 0 or 1");
  return grow_launch(B, 1, (cudaStream_t)stream_v, 1, fix_length);
}

vine_status vine_simulate(vine_batch* B, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_simulate: null batch");
  cudaStream_t st = (cudaStream_t)stream_v;
  if (!B->graph_exec) {
    // record [reset work counter, persistent growth kernel] once
    CK(cudaStreamCreateWithFlags(&B->cap_stream, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(B->cap_stream, cudaStreamCaptureModeThreadLocal));
    vine_status s = grow_launch(B, B->max_target, B->cap_stream);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(B->cap_stream, &g);
    if (s != VINE_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    CK(e);
    B->graph = g;
    CK(cudaGraphInstantiate(&B->graph_exec, g, 0));
  }
  CK(cudaGraphLaunch(B->graph_exec, st));
  return VINE_OK;
}

static vine_status ensure_stage(const vine_batch* Bc, size_t bytes);

// A class's launch shape for a given team size (robots per CTA: for one-warp
// teams the caller's wpc, else one robot per CTA).  False if it does not fit.
static bool shape_class(const vine_batch* B, LaunchClass& L, int team, int wpc, int nsm) {
  L.team = team;
  L.smem_warp = grow_smem_per_warp(L.nmax, L.omax, L.amax, team);
  L.wpc = team > 32 ? 1 : wpc;
  const size_t smem = L.smem_warp * L.wpc;
  int optin = 0;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, B->device);
  if (smem > (size_t)optin || grow_configure(B->ks, smem, team) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  const int ctas = grow_max_ctas_per_sm(B->ks, smem, team * L.wpc, team);
  if (ctas <= 0) return false;
  L.grid = std::max(1, std::min((L.count + L.wpc - 1) / L.wpc, nsm * ctas));
  return true;
}

vine_status vine_autotune(vine_batch* B, int32_t sample, void* stream_v, vine_tune_result* out) {
  if (!B || !out) return fail(VINE_EINVAL, "vine_autotune: null argument");
  if (sample < 0) return fail(VINE_EINVAL, "vine_autotune: negative sample size");
  cudaStream_t st = (cudaStream_t)stream_v;
  const int n = B->n_inst;
  const int ns_all = std::min(n, sample > 0 ? sample : 4096);
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B->device);
  // per class a sample spread evenly over its longest-first segment (keeps
  // its cost mix), in proportion to the class's size, at least 64 robots
  LaunchClass SL[kMaxClass];
  std::vector<int> idx;
  for (int c = 0; c < B->n_class; ++c) {
    const LaunchClass& L = B->cls[c];
    const int k = std::min(L.count, std::max(std::min(64, L.count), (int)((int64_t)ns_all * L.count / n)));
    SL[c] = L;
    SL[c].off = (int)idx.size();
    SL[c].count = k;
    for (int q = 0; q < k; ++q) idx.push_back(B->h_order[L.off + (int64_t)q * L.count / k]);
  }
  const int ns = (int)idx.size();
  vine_status s = ensure_stage(B, 4 * (size_t)std::max(ns, 1));
  if (s != VINE_OK) return s;
  int* d_idx = (int*)B->stage;
  CK(cudaMemcpyAsync(d_idx, idx.data(), 4 * (size_t)ns, cudaMemcpyHostToDevice, st));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  std::memset(out, 0, sizeof(*out));
  out->sample = ns;
  out->n_class = B->n_class;
  vine_status rs = VINE_OK;
  // grows the sample's classes L[0..nc) from reset; time in ms (< 0: failed)
  auto timed = [&](const LaunchClass* L, int nc, float margin) -> double {
    if ((rs = vine_batch_reset(B, st)) != VINE_OK) return -1.0;
    int mt = 1;
    for (int c = 0; c < nc; ++c) mt = std::max(mt, L[c].max_target);
    cudaError_t e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) e = launch_classes(B, L, nc, d_idx, mt, margin, 0, 0, st);
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      rs = cuda_fail(e, "vine_autotune");
      return -1.0;
    }
    out->candidates += 1;
    return ms;
  };
  // the configuration chosen at creation, all classes together
  LaunchClass best[kMaxClass];
  for (int c = 0; c < B->n_class; ++c) {
    best[c] = SL[c];
    shape_class(B, best[c], SL[c].team, SL[c].wpc, nsm);
  }
  out->default_ms = timed(best, B->n_class, B->margin);
  // per class: threads per robot (32, 64, 128; one-warp teams also with 4,
  // 2 or 1 robots per CTA), each class timed alone on its sample
  for (int c = 0; c < B->n_class && rs == VINE_OK; ++c) {
    double cbest = 1e30;
    const int shapes[5][2] = {{32, 4}, {32, 2}, {32, 1}, {64, 1}, {128, 1}};
    for (const auto& sh : shapes) {
      LaunchClass L = SL[c];
      L.off = 0;  // this class alone: its sample segment at the start
      if (!shape_class(B, L, sh[0], sh[1], nsm)) continue;
      LaunchClass Lr = L;
      Lr.off = SL[c].off;
      const double ms = timed(&Lr, 1, B->margin);
      if (rs != VINE_OK) break;
      if (ms >= 0.0 && ms < cbest) {
        cbest = ms;
        best[c] = Lr;
      }
    }
    out->class_ms[c] = cbest;
  }
  // the broad-phase margin (0.5, 1, 2 body radii) for all classes together
  double bms = 1e30;
  float bm = B->margin;
  const float margins[3] = {0.5f, kListMargin, 2.0f};
  for (float m : margins) {
    if (rs != VINE_OK) break;
    const double ms = timed(best, B->n_class, m);
    if (ms >= 0.0 && ms < bms) {
      bms = ms;
      bm = m;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rs != VINE_OK) return rs;
  out->best_ms = bms;
  out->list_margin = bm;
  const bool adopt = bms < out->default_ms;
  for (int c = 0; c < B->n_class; ++c) {
    if (adopt) {
      LaunchClass L = B->cls[c];
      shape_class(B, L, best[c].team, best[c].wpc, nsm);  // the full class with the chosen shape
      B->cls[c] = L;
    }
    out->class_threads[c] = B->cls[c].team;
    out->class_robots_per_cta[c] = B->cls[c].wpc;
  }
  if (adopt) B->margin = bm;
  out->adopted = adopt ? 1 : 0;
  out->warps_per_cta = B->cls[0].wpc * B->cls[0].team / 32;
  if (!adopt) {
    out->best_ms = out->default_ms;
    out->list_margin = B->margin;
  }
  if (B->graph_exec) {  // the recorded launch carries the old configuration
    cudaGraphExecDestroy(B->graph_exec);
    cudaGraphDestroy(B->graph);
    B->graph_exec = nullptr;
    B->graph = nullptr;
  }
  return vine_batch_reset(B, st);
}

vine_status vine_simulate_plain(vine_batch* B, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_simulate_plain: null batch");
  cudaStream_t st = (cudaStream_t)stream_v;
  GrowArgs a = B->args;
  a.n_steps = B->max_target;
  a.dynamic = 0;
  a.n_order = 1;
  a.list_margin = B->margin;
  for (int c = 0; c < B->n_class; ++c) {
    const LaunchClass& L = B->cls[c];
    a.nmax = L.nmax;
    a.omax = L.omax;
    a.amax = L.amax;
    a.warp_floats = (int)(L.smem_warp / sizeof(float));
    a.team = L.team;
    CK(grow_configure(B->ks, L.smem_warp, L.team));
    for (int k = L.off; k < L.off + L.count; ++k) {
      a.order = B->args.order + k;
      CK(launch_grow(a, B->ks, 1, L.team, L.smem_warp, st));
    }
  }
  return VINE_OK;
}

static vine_status ensure_stage(const vine_batch* Bc, size_t bytes) {
  vine_batch* B = const_cast<vine_batch*>(Bc);
  if (B->stage_bytes >= bytes) return VINE_OK;
  if (B->stage) cudaFree(B->stage);
  B->stage = nullptr;
  B->stage_bytes = 0;
  CK(cudaMalloc(&B->stage, bytes));
  B->stage_bytes = bytes;
  return VINE_OK;
}

vine_status vine_get_state(const vine_batch* B, float* theta, float* l_last, float* link_pose, float* tip,
                           int32_t* n_present, int32_t* iterations, double* residual, int32_t* inst_status,
                           int32_t out_is_device, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_get_state: null batch");
  cudaStream_t st = (cudaStream_t)stream_v;
  const GrowArgs& a = B->args;
  const int n = B->n_inst;
  const int64_t T = B->total_links;
  if (out_is_device) {
    if (theta || link_pose || tip) CK(launch_poses(a.inst, n, a.theta, a.n_cur, a.l_cur, theta, link_pose, tip, st));
    if (l_last) CK(cudaMemcpyAsync(l_last, a.l_cur, 4 * n, cudaMemcpyDeviceToDevice, st));
    if (n_present) CK(cudaMemcpyAsync(n_present, a.n_cur, 4 * n, cudaMemcpyDeviceToDevice, st));
    if (iterations) CK(cudaMemcpyAsync(iterations, a.iters, 4 * n, cudaMemcpyDeviceToDevice, st));
    if (residual) CK(cudaMemcpyAsync(residual, a.resid_max, 8 * n, cudaMemcpyDeviceToDevice, st));
    if (inst_status) CK(cudaMemcpyAsync(inst_status, a.status, 4 * n, cudaMemcpyDeviceToDevice, st));
    return VINE_OK;
  }
  const size_t need = align256(4 * std::max<int64_t>(T, 1)) + align256(12 * std::max<int64_t>(T, 1)) +
                      align256(8 * (size_t)n);
  vine_status s = ensure_stage(B, need);
  if (s != VINE_OK) return s;
  char* sg = (char*)B->stage;
  float* d_th = (float*)sg;
  float* d_pose = (float*)(sg + align256(4 * std::max<int64_t>(T, 1)));
  float* d_tip = (float*)(sg + align256(4 * std::max<int64_t>(T, 1)) + align256(12 * std::max<int64_t>(T, 1)));
  if (theta || link_pose || tip)
    CK(launch_poses(a.inst, n, a.theta, a.n_cur, a.l_cur, theta ? d_th : nullptr, link_pose ? d_pose : nullptr,
                    tip ? d_tip : nullptr, st));
  if (theta) CK(cudaMemcpyAsync(theta, d_th, 4 * T, cudaMemcpyDeviceToHost, st));
  if (link_pose) CK(cudaMemcpyAsync(link_pose, d_pose, 12 * T, cudaMemcpyDeviceToHost, st));
  if (tip) CK(cudaMemcpyAsync(tip, d_tip, 8 * n, cudaMemcpyDeviceToHost, st));
  if (l_last) CK(cudaMemcpyAsync(l_last, a.l_cur, 4 * n, cudaMemcpyDeviceToHost, st));
  if (n_present) CK(cudaMemcpyAsync(n_present, a.n_cur, 4 * n, cudaMemcpyDeviceToHost, st));
  if (iterations) CK(cudaMemcpyAsync(iterations, a.iters, 4 * n, cudaMemcpyDeviceToHost, st));
  if (residual) CK(cudaMemcpyAsync(residual, a.resid_max, 8 * n, cudaMemcpyDeviceToHost, st));
  if (inst_status) CK(cudaMemcpyAsync(inst_status, a.status, 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return VINE_OK;
}

vine_status vine_get_contacts(const vine_batch* B, int32_t* counts, int32_t* pairs, int32_t max_pairs,
                              int32_t out_is_device, void* stream_v) {
  if (!B || !counts || max_pairs < 0 || (max_pairs > 0 && !pairs))
    return fail(VINE_EINVAL, "vine_get_contacts: bad arguments");
  cudaStream_t st = (cudaStream_t)stream_v;
  const GrowArgs& a = B->args;
  const int n = B->n_inst;
  if (out_is_device) {
    CK(launch_contacts(a.inst, n, a.obs, a.theta, a.n_cur, a.l_cur, B->ks, max_pairs, counts, pairs, st));
    return VINE_OK;
  }
  const size_t pb = 8 * (size_t)n * (size_t)max_pairs;
  vine_status s = ensure_stage(B, align256(4 * (size_t)n) + align256(std::max<size_t>(pb, 16)));
  if (s != VINE_OK) return s;
  int* d_c = (int*)B->stage;
  int* d_p = (int*)((char*)B->stage + align256(4 * (size_t)n));
  CK(launch_contacts(a.inst, n, a.obs, a.theta, a.n_cur, a.l_cur, B->ks, max_pairs, d_c, max_pairs ? d_p : nullptr,
                     st));
  CK(cudaMemcpyAsync(counts, d_c, 4 * (size_t)n, cudaMemcpyDeviceToHost, st));
  if (pb) CK(cudaMemcpyAsync(pairs, d_p, pb, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return VINE_OK;
}

vine_status vine_set_actuators(vine_batch* B, const float* pressure, const float* begin, const float* end,
                               int32_t ptrs_are_device, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_set_actuators: null batch");
  const size_t na = (size_t)B->n_act;
  if (na == 0) return VINE_OK;
  if (!pressure || !begin || !end) return fail(VINE_EINVAL, "vine_set_actuators: null argument");
  cudaStream_t st = (cudaStream_t)stream_v;
  const float *dp = pressure, *db = begin, *de = end;
  if (!ptrs_are_device) {
    vine_status s = ensure_stage(B, 3 * align256(4 * na));
    if (s != VINE_OK) return s;
    char* sg = (char*)B->stage;
    CK(cudaMemcpyAsync(sg, pressure, 4 * na, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sg + align256(4 * na), begin, 4 * na, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sg + 2 * align256(4 * na), end, 4 * na, cudaMemcpyHostToDevice, st));
    dp = (const float*)sg;
    db = (const float*)(sg + align256(4 * na));
    de = (const float*)(sg + 2 * align256(4 * na));
  }
  const GrowArgs& a = B->args;
  const int threads = 128, blocks = (B->n_inst * 32 + threads - 1) / threads;
  actuator_update_kernel<<<blocks, threads, 0, st>>>(a.inst, B->n_inst, dp, db, de, const_cast<float4*>(a.act),
                                                     B->status0, a.status);
  CK(cudaGetLastError());
  if (!ptrs_are_device) CK(cudaStreamSynchronize(st));
  return VINE_OK;
}

vine_status vine_set_state(vine_batch* B, const int32_t* n_present, const float* theta, const float* l_last,
                           int32_t ptrs_are_device, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_set_state: null batch");
  if (!n_present || !l_last || (B->total_links > 0 && !theta))
    return fail(VINE_EINVAL, "vine_set_state: null argument");
  cudaStream_t st = (cudaStream_t)stream_v;
  vine_status s = vine_batch_reset(B, stream_v);  // counters cleared, validation status restored
  if (s != VINE_OK) return s;
  const size_t n = (size_t)B->n_inst, nl = (size_t)B->total_links;
  if (n == 0) return VINE_OK;
  const int32_t* dn = n_present;
  const float *dt = theta, *dl = l_last;
  if (!ptrs_are_device) {
    s = ensure_stage(B, align256(4 * n) + align256(4 * n) + align256(4 * std::max<size_t>(nl, 1)));
    if (s != VINE_OK) return s;
    char* sg = (char*)B->stage;
    CK(cudaMemcpyAsync(sg, n_present, 4 * n, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(sg + align256(4 * n), l_last, 4 * n, cudaMemcpyHostToDevice, st));
    if (nl) CK(cudaMemcpyAsync(sg + 2 * align256(4 * n), theta, 4 * nl, cudaMemcpyHostToDevice, st));
    dn = (const int32_t*)sg;
    dl = (const float*)(sg + align256(4 * n));
    dt = (const float*)(sg + 2 * align256(4 * n));
  }
  const GrowArgs& a = B->args;
  const int threads = 128, blocks = (int)((n * 32 + threads - 1) / threads);
  state_load_kernel<<<blocks, threads, 0, st>>>(a.inst, B->n_inst, dn, dt, dl, a.theta, a.n_cur, a.l_cur,
                                                B->status0, a.status);
  CK(cudaGetLastError());
  if (!ptrs_are_device) CK(cudaStreamSynchronize(st));
  return VINE_OK;
}

vine_status vine_synthesize(const vine_synth_spec* spec, const vine_params* params, const double* theta_target,
                            int32_t n_targets, int32_t* p_index, int32_t* l0_index, double* theta_eq,
                            double* theta_pairs, void* stream_v) {
  if (!spec || n_targets < 0 || (n_targets > 0 && (!theta_target || !p_index || !l0_index || !theta_eq)))
    return fail(VINE_EINVAL, "vine_synthesize: null argument or negative count");
  const vine_synth_spec& c = *spec;
  auto pos = [](double v) { return std::isfinite(v) && v > 0.0; };
  if (!pos(c.R) || !pos(c.P_vine) || !pos(c.l_seg) || !pos(c.l0_min) || !(std::isfinite(c.l0_step) && c.l0_step >= 0.0) ||
      !(std::isfinite(c.tol) && c.tol >= 0.0) || c.n_p < 1 || c.n_l0 < 1 || c.n_p > 4096 || c.n_l0 > 4096 ||
      (int64_t)c.n_p * c.n_l0 > (1 << 20) || !c.pressures)
    return fail(VINE_EINVAL, "vine_synthesize: specification out of range");
  for (int i = 0; i < c.n_p; ++i)
    if (!pos(c.pressures[i])) return fail(VINE_EINVAL, "vine_synthesize: pressures must be finite and positive");
  vine_params prm;
  if (params) prm = *params; else vine_params_default(&prm);
  cudaStream_t st = (cudaStream_t)stream_v;
  const size_t nt = (size_t)n_targets, np = (size_t)c.n_p, nl = (size_t)c.n_l0, npl = np * nl;
  std::vector<double> l0s(nl);
  for (size_t k = 0; k < nl; ++k) l0s[k] = c.l0_min + (double)k * c.l0_step;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += align256(std::max<size_t>(bytes, 16));
    return o;
  };
  const size_t o_tg = take(8 * nt), o_pr = take(8 * np), o_l0 = take(8 * nl), o_scr = take(8 * (4 + kKnots) * nl),
               o_hdr = take(sizeof(float4) * nl), o_tab = take(sizeof(float2) * kKnots * nl), o_pair = take(8 * npl),
               o_pi = take(4 * nt), o_li = take(4 * nt), o_eq = take(8 * nt);
  char* mem = nullptr;
  CK(cudaMallocAsync((void**)&mem, off, st));
  struct Free {
    char* m;
    cudaStream_t s;
    ~Free() { cudaFreeAsync(m, s); }
  } fr{mem, st};
  if (nt) CK(cudaMemcpyAsync(mem + o_tg, theta_target, 8 * nt, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(mem + o_pr, c.pressures, 8 * np, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(mem + o_l0, l0s.data(), 8 * nl, cudaMemcpyHostToDevice, st));
  GaussLegendre gl;
  gauss_legendre(24, &gl);
  // the FP64 tables of this grid, if an earlier call built them (the build
  // is deterministic: the copy is bitwise what a rebuild gives)
  const size_t scr_bytes = 8 * (4 + (size_t)kKnots) * nl;
  int dev = 0;
  CK(cudaGetDevice(&dev));
  int ready = 0;
  {
    TableCache& tc = table_cache();
    std::lock_guard<std::mutex> lk(tc.mu);
    if (const SynthEntry* e = find_synth(tc, dev, c, prm)) {
      CK(cudaMemcpyAsync(mem + o_scr, e->scr, scr_bytes, cudaMemcpyDeviceToDevice, st));
      ready = 1;
    }
  }
  CK(launch_synth(n_targets, (const double*)(mem + o_tg), c.n_p, c.n_l0, (const double*)(mem + o_pr),
                  (const double*)(mem + o_l0), c.R, c.P_vine, c.l_seg, c.tol, prm.R_c, prm.R_act, prm.a_spam, prm.m_lo,
                  prm.eps_crit, gl, (double*)(mem + o_scr), (float4*)(mem + o_hdr), (float2*)(mem + o_tab),
                  (double*)(mem + o_pair), (int*)(mem + o_pi), (int*)(mem + o_li), (double*)(mem + o_eq), ready, st));
  if (nt) {
    CK(cudaMemcpyAsync(p_index, mem + o_pi, 4 * nt, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(l0_index, mem + o_li, 4 * nt, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(theta_eq, mem + o_eq, 8 * nt, cudaMemcpyDeviceToHost, st));
  }
  if (theta_pairs) CK(cudaMemcpyAsync(theta_pairs, mem + o_pair, 8 * npl, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  if (!ready) {  // keep this grid's tables for later calls
    TableCache& tc = table_cache();
    std::lock_guard<std::mutex> lk(tc.mu);
    if (tc.synth.size() < kCacheSynth && !find_synth(tc, dev, c, prm)) {
      double* keep = nullptr;
      if (cudaMalloc((void**)&keep, scr_bytes) == cudaSuccess) {
        if (cudaMemcpyAsync(keep, mem + o_scr, scr_bytes, cudaMemcpyDeviceToDevice, st) == cudaSuccess &&
            cudaStreamSynchronize(st) == cudaSuccess)
          tc.synth.push_back(SynthEntry{dev, c.l0_min, c.l0_step, prm.R_c, prm.R_act, prm.a_spam, prm.m_lo, c.n_l0, keep});
        else
          cudaFree(keep);
      } else {
        (void)cudaGetLastError();  // no room to keep the tables: not an error of this call
      }
    }
  }
  return VINE_OK;
}

// The adjoint launch shared by vine_grad (kind 0) and vine_grad_path (kind
// 1); `target` holds n_target floats (2 n goals or 2 sum n_links targets).
static vine_status grad_launch(const vine_batch* B, int kind, const float* target, size_t n_target, double* cost,
                               double* d_pressure, double* d_begin, double* d_end, int32_t* grad_status,
                               int32_t ptrs_are_device, cudaStream_t st, const char* who) {
  if (!B || !target || !cost || !grad_status || (B->n_act > 0 && (!d_pressure || !d_begin || !d_end)))
    return fail(VINE_EINVAL, who);
  const int n = B->n_inst;
  const size_t na = (size_t)B->n_act;
  int nsm = 1;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, B->device);
  // one warp per CTA, several CTAs per SM; the robots come longest first
  const int grid = std::max(1, std::min(n, 16 * nsm));
  GradArgs g{};
  g.kind = kind;
  if (ptrs_are_device) {
    g.goal = target;
    g.cost = cost;
    g.dP = d_pressure;
    g.dB = d_begin;
    g.dE = d_end;
    g.gstat = grad_status;
    CK(launch_grad(B->args, g, B->ks, grid, B->smem_warp, st));
    return VINE_OK;
  }
  const size_t o_goal = 0, o_cost = align256(4 * std::max<size_t>(n_target, 1)),
               o_stat = o_cost + align256(8 * (size_t)n), o_dp = o_stat + align256(4 * (size_t)n),
               o_db = o_dp + align256(8 * std::max<size_t>(na, 1)), o_de = o_db + align256(8 * std::max<size_t>(na, 1)),
               total = o_de + align256(8 * std::max<size_t>(na, 1));
  vine_status s = ensure_stage(B, total);
  if (s != VINE_OK) return s;
  char* sg = (char*)B->stage;
  g.goal = (const float*)(sg + o_goal);
  g.cost = (double*)(sg + o_cost);
  g.gstat = (int*)(sg + o_stat);
  g.dP = (double*)(sg + o_dp);
  g.dB = (double*)(sg + o_db);
  g.dE = (double*)(sg + o_de);
  CK(cudaMemcpyAsync(sg + o_goal, target, 4 * n_target, cudaMemcpyHostToDevice, st));
  CK(launch_grad(B->args, g, B->ks, grid, B->smem_warp, st));
  CK(cudaMemcpyAsync(cost, g.cost, 8 * (size_t)n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(grad_status, g.gstat, 4 * (size_t)n, cudaMemcpyDeviceToHost, st));
  if (na) {
    CK(cudaMemcpyAsync(d_pressure, g.dP, 8 * na, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(d_begin, g.dB, 8 * na, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(d_end, g.dE, 8 * na, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  return VINE_OK;
}

vine_status vine_grad(const vine_batch* B, const float* goal_xy, double* cost, double* d_pressure, double* d_begin,
                      double* d_end, int32_t* grad_status, int32_t ptrs_are_device, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_grad: null batch");
  return grad_launch(B, 0, goal_xy, 2 * (size_t)B->n_inst, cost, d_pressure, d_begin, d_end, grad_status,
                     ptrs_are_device, (cudaStream_t)stream_v, "vine_grad: null argument");
}

vine_status vine_grad_path(const vine_batch* B, const float* path_xy, double* cost, double* d_pressure,
                           double* d_begin, double* d_end, int32_t* grad_status, int32_t ptrs_are_device,
                           void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_grad_path: null batch");
  return grad_launch(B, 1, path_xy, 2 * (size_t)B->total_links, cost, d_pressure, d_begin, d_end, grad_status,
                     ptrs_are_device, (cudaStream_t)stream_v, "vine_grad_path: null argument");
}

vine_status vine_get_stats(const vine_batch* B, vine_stats* out, void* stream_v) {
  if (!B || !out) return fail(VINE_EINVAL, "vine_get_stats: null argument");
  cudaStream_t st = (cudaStream_t)stream_v;
  const GrowArgs& a = B->args;
  const int n = B->n_inst;
  std::vector<int> it(n), cv(n), sp(n), status(n);
  std::vector<long long> rls(n), ev(n), le(n), fb(n), pt(n);
  CK(cudaMemcpyAsync(it.data(), a.iters, 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(cv.data(), a.conv, 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(sp.data(), a.steps, 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(status.data(), a.status, 4 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(rls.data(), a.rls, 8 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(ev.data(), a.evals, 8 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(le.data(), a.linkevals, 8 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(fb.data(), a.fallbacks, 8 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(pt.data(), a.pairtests, 8 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::memset(out, 0, sizeof(*out));
  for (int i = 0; i < n; ++i) {
    out->robot_link_steps += rls[i];
    out->steps_converged += cv[i];
    out->steps_total += sp[i];
    out->iterations += it[i];
    out->evaluations += ev[i];
    out->link_evaluations += le[i];
    out->gn_fallbacks += fb[i];
    out->pair_tests += le[i] * B->ks * (int64_t)B->h_n_obs[i];
    out->circle_pair_tests += le[i] * B->ks * (int64_t)B->h_n_circ[i];
    out->pair_tests_executed += pt[i];
    out->n_maxiter += status[i] == kMaxIter;
    out->n_nonfinite += status[i] == kNonFinite;
    out->n_badinput += status[i] == kBadInput;
  }
  return VINE_OK;
}

vine_status vine_get_tables(const vine_batch* B, int32_t* n_tab, float* hdr, float* knots, float* utab,
                            double* consts) {
  if (!B || !n_tab) return fail(VINE_EINVAL, "vine_get_tables: null argument");
  *n_tab = B->n_tab;
  const GrowArgs& a = B->args;
  if (hdr && B->n_tab) CK(cudaMemcpy(hdr, a.tab_hdr, sizeof(float4) * B->n_tab, cudaMemcpyDeviceToHost));
  if (knots && B->n_tab)
    CK(cudaMemcpy(knots, a.tab, sizeof(float2) * B->n_tab * kKnots, cudaMemcpyDeviceToHost));
  if (utab) CK(cudaMemcpy(utab, a.utab, sizeof(float2) * (kUCells + 1), cudaMemcpyDeviceToHost));
  if (consts) {
    consts[0] = a.U_pi;
    consts[1] = a.m_pi;
    consts[2] = a.theta_c;
    consts[3] = a.u_h;
  }
  return VINE_OK;
}

vine_status vine_probe_state(const vine_batch* B, int32_t inst, int32_t n_links, const float* theta, float l_last,
                             double* cost, float* grad, float* step, double* residual, int32_t* l_fixed) {
  if (!B || !theta || !cost || !grad || !step || !residual) return fail(VINE_EINVAL, "vine_probe_state: null argument");
  if (inst < 0 || inst >= B->n_inst || n_links < 1 || n_links > B->h_n_links[inst])
    return fail(VINE_EINVAL, "vine_probe_state: instance or link count out of range");
  const size_t n = (size_t)n_links;
  char* d = nullptr;
  const size_t bytes = 256 + 4 * n + 4 * (n + 1) * 2 + 64;
  CK(cudaMalloc(&d, bytes));
  float* d_th = (float*)(d + 64);
  float* d_g = d_th + n;
  float* d_dx = d_g + n + 1;
  double* d_J = (double*)d;
  double* d_r = d_J + 1;
  int* d_lf = (int*)(d_J + 2);
  cudaError_t e = cudaMemcpy(d_th, theta, 4 * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = launch_probe(B->args, B->ks, inst, n_links, d_th, l_last, d_J, d_g, d_dx, d_r, d_lf,
                                         B->smem_warp, 0);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  int lf = 0;
  if (e == cudaSuccess) e = cudaMemcpy(cost, d_J, 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(residual, d_r, 8, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(&lf, d_lf, 4, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(grad, d_g, 4 * (n + 1), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess) e = cudaMemcpy(step, d_dx, 4 * (n + 1), cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(e, "vine_probe_state");
  if (l_fixed) *l_fixed = lf;
  return VINE_OK;
}

vine_status vine_get_robot_counters(const vine_batch* B, int32_t* steps_converged, int64_t* evaluations,
                                    int64_t* cycles, void* stream_v) {
  if (!B) return fail(VINE_EINVAL, "vine_get_robot_counters: null batch");
  cudaStream_t st = (cudaStream_t)stream_v;
  const GrowArgs& a = B->args;
  const int n = B->n_inst;
  if (steps_converged) CK(cudaMemcpyAsync(steps_converged, a.conv, 4 * n, cudaMemcpyDeviceToHost, st));
  if (evaluations) CK(cudaMemcpyAsync(evaluations, a.evals, 8 * n, cudaMemcpyDeviceToHost, st));
  if (cycles) CK(cudaMemcpyAsync(cycles, a.cycles, 8 * n, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return VINE_OK;
}

vine_status vine_batch_info(const vine_batch* B, int32_t* n_inst, int64_t* total_links) {
  if (!B) return fail(VINE_EINVAL, "vine_batch_info: null batch");
  if (n_inst) *n_inst = B->n_inst;
  if (total_links) *total_links = B->total_links;
  return VINE_OK;
}

vine_status vine_batch_launch(const vine_batch* B, int32_t* threads_per_robot, int32_t* robots_per_cta,
                              int32_t* grid) {
  if (!B) return fail(VINE_EINVAL, "vine_batch_launch: null batch");
  if (threads_per_robot) *threads_per_robot = B->cls[0].team;
  if (robots_per_cta) *robots_per_cta = B->cls[0].wpc;
  if (grid) *grid = B->cls[0].grid;
  return VINE_OK;
}

vine_status vine_batch_classes(const vine_batch* B, int32_t* n_class, int32_t* threads_per_robot, int32_t* robots,
                               int32_t* robots_per_cta, int32_t* grid, int32_t* max_links) {
  if (!B || !n_class) return fail(VINE_EINVAL, "vine_batch_classes: null argument");
  *n_class = B->n_class;
  for (int c = 0; c < B->n_class; ++c) {
    if (threads_per_robot) threads_per_robot[c] = B->cls[c].team;
    if (robots) robots[c] = B->cls[c].count;
    if (robots_per_cta) robots_per_cta[c] = B->cls[c].wpc;
    if (grid) grid[c] = B->cls[c].grid;
    if (max_links) max_links[c] = B->cls[c].max_target;
  }
  return VINE_OK;
}

vine_status vine_batch_destroy(vine_batch* B) {
  if (!B) return VINE_OK;
  cudaDeviceSynchronize();
  if (B->graph_exec) cudaGraphExecDestroy(B->graph_exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  if (B->cap_stream) cudaStreamDestroy(B->cap_stream);
  release_launch_streams(B);
  if (B->stage) cudaFree(B->stage);
  if (B->dmem) cudaFree(B->dmem);
  delete B;
  return VINE_OK;
}

}  // extern "C"
