// vine_serve.cu -- the serving loop behind vine_server_* (include/vine.h):
// continuous batching of growth requests on one GPU.
//
// Device memory (one cudaMalloc, carved in this order):
//   InstDev  inst[S]              per slot: derived constants + offsets
//   float4   obs[S * omax]        obstacles of slot s at s * omax
//   float4   act[S * amax]        actuators of slot s at s * amax
//   float    theta[S * nmax]      joint angles of slot s at s * nmax
//   per-slot state and counters   n_cur, l_cur, status, iters, ... [S]
//   int      order[S]             active slots of the current launch
//   float4 / float2               sPAM table headers and knots [max_tables]
//   float2   utab[kUCells + 1]    wrinkling-energy table
//   staging                       one request's raw descriptor (upload)
//   results                       compact outputs of retiring requests
// The worker thread owns the stream; callers only touch host structures
// under the server mutex.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "vine.h"
#include "vine_internal.cuh"

using namespace vine;

namespace {

double clock_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t up16(size_t x) { return (x + 15) & ~size_t(15); }
size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

vine_status sfail(vine_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

vine_status scuda(cudaError_t e, const char* where) {
  char b[384];
  std::snprintf(b, sizeof(b), "%s: %s", where, cudaGetErrorString(e));
  set_last_error(b);
  return e == cudaErrorMemoryAllocation ? VINE_ENOMEM : VINE_ECUDA;
}

// Array slots of a request's upload image (the raw descriptor, packed).
enum Field {
  F_NLINKS, F_LSEG, F_RADIUS, F_PRESSURE, F_BASE, F_ACTPTR, F_ABEGIN, F_AEND, F_ASIDE, F_APRESS, F_AL0,
  F_OBSPTR, F_OKIND, F_OCX, F_OCY, F_OA, F_OB, F_ACTTAB, F_STATUSH, F_SLOT, F_COUNT
};

struct Request {
  uint64_t id = 0;
  int n = 0, n_act = 0, n_obs = 0;
  int64_t links = 0;
  std::vector<char> image;  // packed descriptor + act_tab + status_h + slot
  size_t off[F_COUNT] = {};
  std::vector<int> n_links, n_obs_r;
  std::vector<double> l0;   // distinct cell lengths of the request
  std::vector<int> tabs;    // the table entries it holds (admitted requests)
  std::vector<int> slots;
  int64_t out_base = 0;     // offset in the tick's result buffers
  double t_submit = 0.0, t_admit = 0.0, t_done = 0.0;
  int state = 0;            // 0 waiting, 1 active, 2 done, 3 failed
  int lane = 0;             // launch lane its robots run in
  std::vector<float> theta, l_last, tip;
  std::vector<int32_t> n_present, status, iters;
  int64_t rls = 0;
};

// Per-robot results of retiring requests gathered into compact arrays.
__global__ void gather_meta_kernel(const int* sel, int n, const int* n_cur, const float* l_cur, const int* status,
                                   const int* iters, const long long* rls, int* o_n, float* o_l, int* o_status,
                                   int* o_iters, long long* o_rls) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int s = sel[k];
  o_n[k] = n_cur[s];
  o_l[k] = l_cur[s];
  o_status[k] = status[s];
  o_iters[k] = iters[s];
  o_rls[k] = rls[s];
}

// Fresh state for newly admitted slots.
__global__ void slot_reset_kernel(const int* slots, int n, int* n_cur, float* l_cur, int* iters, int* conv,
                                  int* steps, long long* rls, long long* evals, long long* linkevals,
                                  long long* fallbacks, long long* cycles, long long* pairtests,
                                  double* resid_max) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= n) return;
  const int s = slots[k];
  n_cur[s] = 0;
  l_cur[s] = 0.f;
  iters[s] = 0;
  conv[s] = 0;
  steps[s] = 0;
  rls[s] = 0;
  evals[s] = 0;
  linkevals[s] = 0;
  fallbacks[s] = 0;
  cycles[s] = 0;
  pairtests[s] = 0;
  resid_max[s] = 0.0;
}

}  // namespace

// A launch lane: its own stream, work queue and read-back buffers, so that
// while one lane's launch waits on its slowest robot another lane's launch
// fills the idle SMs.  Robots stay in the lane of their request.
struct Lane {
  cudaStream_t st = nullptr;
  cudaEvent_t ev = nullptr;
  int* d_order = nullptr;   // [S]
  int* d_counter = nullptr;
  int* h_order = nullptr;   // pinned [S]
  int* h_ncur = nullptr;    // pinned [S]
  int* h_status = nullptr;  // pinned [S]
  std::vector<int> robots;  // slots of the launch in flight
  bool busy = false;
  int load = 0;             // robots of its active requests
};

struct vine_server {
  vine_params prm{};
  vine_server_config cfg{};
  int device = 0;
  cudaStream_t stream = nullptr;
  int S = 0, nmax = 0, omax = 0, amax = 0, ks = 2, grid = 1, wpc = kWarpsPerCta;
  int team = 32;  // threads per robot
  size_t smem_warp = 0, stage_bytes = 0;
  char* dmem = nullptr;
  GrowArgs args{};
  // device pointers carved from dmem
  double* d_l0 = nullptr;
  double* d_scr = nullptr;
  char* d_stage = nullptr;
  int* d_sel = nullptr;           // [S] slots of retiring robots / admitted slots
  long long* d_outoff = nullptr;  // [S]
  float* d_res_theta = nullptr;   // [S * nmax]
  float* d_res_tip = nullptr;     // [2 S]
  int* d_res_n = nullptr;
  float* d_res_l = nullptr;
  int* d_res_status = nullptr;
  int* d_res_iters = nullptr;
  long long* d_res_rls = nullptr;
  // pinned host result staging
  char* h_res = nullptr;
  size_t h_res_bytes = 0;
  // host state (mu)
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Request*> waiting;
  std::vector<Request*> active;
  std::unordered_map<uint64_t, Request*> reqs;
  std::vector<int> free_slots;
  int promised = 0;  // slots of waiting requests
  // sPAM table entries: cell length and the number of live (admitted, not
  // retired) requests holding it; an entry held by none is reused for a new
  // cell length, so only the cell lengths live at one time count against
  // max_tables
  std::vector<double> tab_l0;
  std::vector<int> tab_ref;
  uint64_t next_id = 1;
  bool stop = false;
  std::string error;
  vine_server_stats stats{};
  // worker-only per-slot host info
  std::vector<int> slot_target, slot_nobs, slot_ncur, slot_status;
  std::vector<Lane> lanes;
  int window = 0;             // robots per launch and lane
  cudaEvent_t ev_admit = nullptr;
  std::thread worker;
};

namespace {

bool robot_done(int n_cur, int target, int status) {
  return n_cur >= target || status != kOK;  // a failed step ends the robot's growth
}

// Admission of one waiting request: slots, tables, upload, validation/encoding.
cudaError_t admit(vine_server* V, Request* R) {
  cudaStream_t st = V->stream;
  // table entries for the request's cell lengths: held ones are shared,
  // new cell lengths take a free entry (or a new one) and are built there
  std::vector<int> build;  // entries to (re)build
  {
    std::lock_guard<std::mutex> lk(V->mu);
    for (double v : R->l0) {
      int t = -1;
      for (int k = 0; k < (int)V->tab_l0.size() && t < 0; ++k)
        if (V->tab_ref[k] > 0 && V->tab_l0[k] == v) t = k;
      if (t < 0) {
        for (int k = 0; k < (int)V->tab_l0.size() && t < 0; ++k)
          if (V->tab_ref[k] == 0) t = k;
        if (t < 0) {
          t = (int)V->tab_l0.size();  // submit kept the live cell lengths within max_tables
          V->tab_l0.push_back(v);
          V->tab_ref.push_back(0);
        }
        V->tab_l0[t] = v;
        build.push_back(t);
      }
      V->tab_ref[t] += 1;
      R->tabs.push_back(t);
    }
  }
  for (int t : build) {
    const double v = V->tab_l0[t];
    cudaError_t e = cudaMemcpyAsync(V->d_l0 + t, &v, sizeof(double), cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return e;
    GaussLegendre gl;
    gauss_legendre(24, &gl);
    e = launch_spam_tables(V->d_l0 + t, 1, V->prm.R_c, V->prm.R_act, V->prm.a_spam, V->prm.m_lo, gl,
                           const_cast<float4*>(V->args.tab_hdr) + t, const_cast<float2*>(V->args.tab) + (size_t)t * kKnots,
                           V->d_scr, st);
    if (e != cudaSuccess) return e;
    e = cudaStreamSynchronize(st);  // the pageable source value and the shared scratch
    if (e != cudaSuccess) return e;
  }
  // actuator -> table index, and the slots, written into the image
  {
    const float* l0 = (const float*)(R->image.data() + R->off[F_AL0]);
    int* act_tab = (int*)(R->image.data() + R->off[F_ACTTAB]);
    for (int a = 0; a < R->n_act; ++a) {
      const double v = l0[a];
      int t = 0;  // invalid l0: flagged on the device
      for (size_t k = 0; k < R->l0.size(); ++k)
        if (R->l0[k] == v) t = R->tabs[k];
      act_tab[a] = t;
    }
    std::lock_guard<std::mutex> lk(V->mu);
    R->slots.resize(R->n);
    for (int k = 0; k < R->n; ++k) {
      R->slots[k] = V->free_slots.back();
      V->free_slots.pop_back();
    }
    V->promised -= R->n;
    std::memcpy(R->image.data() + R->off[F_SLOT], R->slots.data(), sizeof(int) * R->n);
  }
  // pageable source: the copy has consumed the image when the call returns
  cudaError_t e = cudaMemcpyAsync(V->d_stage, R->image.data(), R->image.size(), cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const char* d = V->d_stage;
  InitArgs ia{};
  ia.n_inst = R->n;
  ia.n_links = (const int32_t*)(d + R->off[F_NLINKS]);
  ia.l_seg = (const float*)(d + R->off[F_LSEG]);
  ia.radius = (const float*)(d + R->off[F_RADIUS]);
  ia.pressure = (const float*)(d + R->off[F_PRESSURE]);
  ia.base = (const float*)(d + R->off[F_BASE]);
  ia.act_ptr = (const int32_t*)(d + R->off[F_ACTPTR]);
  ia.act_begin = (const float*)(d + R->off[F_ABEGIN]);
  ia.act_end = (const float*)(d + R->off[F_AEND]);
  ia.act_side = (const int8_t*)(d + R->off[F_ASIDE]);
  ia.act_pressure = (const float*)(d + R->off[F_APRESS]);
  ia.act_l0 = (const float*)(d + R->off[F_AL0]);
  ia.obs_ptr = (const int32_t*)(d + R->off[F_OBSPTR]);
  ia.obs_kind = (const uint8_t*)(d + R->off[F_OKIND]);
  ia.obs_cx = (const float*)(d + R->off[F_OCX]);
  ia.obs_cy = (const float*)(d + R->off[F_OCY]);
  ia.obs_a = (const float*)(d + R->off[F_OA]);
  ia.obs_b = (const float*)(d + R->off[F_OB]);
  ia.act_tab = (const int*)(d + R->off[F_ACTTAB]);
  ia.th_off = nullptr;
  ia.status_h = (const int*)(d + R->off[F_STATUSH]);
  ia.slot = (const int*)(d + R->off[F_SLOT]);
  ia.nmax_s = V->nmax;
  ia.omax_s = V->omax;
  ia.amax_s = V->amax;
  ia.R_act = V->prm.R_act;
  ia.w_a = V->prm.w_a;
  ia.pen_frac = V->prm.pen_frac;
  ia.inst = const_cast<InstDev*>(V->args.inst);
  ia.obs = const_cast<float4*>(V->args.obs);
  ia.act = const_cast<float4*>(V->args.act);
  ia.status = V->args.status;
  e = launch_init(ia, st);
  if (e != cudaSuccess) return e;
  const GrowArgs& a = V->args;
  slot_reset_kernel<<<(R->n + 127) / 128, 128, 0, st>>>(ia.slot, R->n, a.n_cur, a.l_cur, a.iters, a.conv, a.steps,
                                                        a.rls, a.evals, a.linkevals, a.fallbacks, a.cycles,
                                                        a.pairtests, a.resid_max);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  for (int k = 0; k < R->n; ++k) {
    const int s = R->slots[k];
    V->slot_target[s] = R->n_links[k];
    V->slot_nobs[s] = R->n_obs_r[k];
    V->slot_ncur[s] = 0;
    V->slot_status[s] = kOK;
  }
  // the lane with the fewest robots
  int best = 0;
  for (int q = 1; q < (int)V->lanes.size(); ++q)
    if (V->lanes[q].load < V->lanes[best].load) best = q;
  R->lane = best;
  V->lanes[best].load += R->n;
  R->t_admit = clock_s();
  R->state = 1;
  V->active.push_back(R);
  return cudaSuccess;
}

// Launches one growth step batch in lane q: the robots of its requests that
// still grow, oldest requests first, at most `window` of them, ordered by
// their contact work for the coming steps (largest first) for the atomic
// queue.  Returns with *launched = false when the lane has nothing to grow.
cudaError_t launch_lane(vine_server* V, int q, bool* launched) {
  Lane& L = V->lanes[q];
  std::vector<std::pair<double, int>> work;
  for (Request* R : V->active) {
    if (R->lane != q) continue;
    for (int s : R->slots) {
      const int N = V->slot_ncur[s], T = V->slot_target[s];
      if (N >= T || V->slot_status[s] == kNonFinite || V->slot_status[s] == kBadInput) continue;
      const int M = std::min(T, N + V->cfg.steps_per_tick);
      // contact work of steps N+1..M: links x (discs x obstacles + joint terms)
      const double w = 0.5 * (double)(M - N) * (double)(N + 1 + M) * (V->ks * (double)V->slot_nobs[s] + 8.0);
      work.emplace_back(w, s);
    }
    if ((int)work.size() >= V->window) break;
  }
  *launched = !work.empty();
  if (work.empty()) return cudaSuccess;
  std::stable_sort(work.begin(), work.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
  L.robots.resize(work.size());
  for (size_t k = 0; k < work.size(); ++k) L.h_order[k] = L.robots[k] = work[k].second;
  cudaError_t e = cudaStreamWaitEvent(L.st, V->ev_admit, 0);  // admitted robots and new tables
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(L.d_order, L.h_order, sizeof(int) * work.size(), cudaMemcpyHostToDevice, L.st);
  GrowArgs a = V->args;
  a.order = L.d_order;
  a.counter = L.d_counter;
  a.n_order = (int)work.size();
  a.n_steps = V->cfg.steps_per_tick;
  a.dynamic = 1;
  if (e == cudaSuccess) e = cudaMemsetAsync(a.counter, 0, sizeof(int), L.st);
  if (e == cudaSuccess) e = grow_configure(V->ks, V->smem_warp * V->wpc, V->team);
  const int grid = std::max(1, std::min(V->grid, (a.n_order + V->wpc - 1) / V->wpc));
  if (e == cudaSuccess) e = launch_grow(a, V->ks, grid, V->team * V->wpc, V->smem_warp * V->wpc, L.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.h_ncur, a.n_cur, sizeof(int) * V->S, cudaMemcpyDeviceToHost, L.st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(L.h_status, a.status, sizeof(int) * V->S, cudaMemcpyDeviceToHost, L.st);
  if (e == cudaSuccess) e = cudaEventRecord(L.ev, L.st);
  if (e == cudaSuccess) L.busy = true;
  return e;
}

// Requests of lane q whose robots are all done: gather their results on the
// admission stream (the lane's launch has finished), free the slots.
cudaError_t retire(vine_server* V, int q) {
  cudaStream_t st = V->stream;
  std::vector<Request*> done;
  int64_t nsel = 0, links = 0;
  for (Request* R : V->active) {
    if (R->lane != q) continue;
    bool all = true;
    for (int k = 0; k < R->n && all; ++k) {
      const int s = R->slots[k];
      all = robot_done(V->slot_ncur[s], V->slot_target[s], V->slot_status[s]);
    }
    if (all) {
      done.push_back(R);
      nsel += R->n;
      links += R->links;
    }
  }
  if (done.empty()) return cudaSuccess;
  std::vector<int> sel;
  std::vector<long long> outoff;
  sel.reserve(nsel);
  outoff.reserve(nsel);
  long long o = 0;
  for (Request* R : done) {
    R->out_base = (int64_t)sel.size();
    for (int k = 0; k < R->n; ++k) {
      sel.push_back(R->slots[k]);
      outoff.push_back(o);
      o += R->n_links[k];
    }
  }
  const int n = (int)nsel;
  cudaError_t e = cudaMemcpyAsync(V->d_sel, sel.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(V->d_outoff, outoff.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, st);
  const GrowArgs& a = V->args;
  if (e == cudaSuccess)
    e = launch_poses_sel(a.inst, V->d_sel, V->d_outoff, n, a.theta, a.n_cur, a.l_cur, V->d_res_theta, nullptr,
                         V->d_res_tip, st);
  if (e != cudaSuccess) return e;
  gather_meta_kernel<<<(n + 127) / 128, 128, 0, st>>>(V->d_sel, n, a.n_cur, a.l_cur, a.status, a.iters, a.rls,
                                                      V->d_res_n, V->d_res_l, V->d_res_status, V->d_res_iters,
                                                      V->d_res_rls);
  e = cudaGetLastError();
  // results to pinned host memory: theta | tip | n | l | status | iters | rls
  char* h = V->h_res;
  const size_t b_th = sizeof(float) * (size_t)links, b_tip = sizeof(float) * 2 * n;
  float* h_th = (float*)h;
  float* h_tip = (float*)(h + up16(b_th));
  int* h_n = (int*)((char*)h_tip + up16(b_tip));
  float* h_l = (float*)((char*)h_n + up16(4 * (size_t)n));
  int* h_st = (int*)((char*)h_l + up16(4 * (size_t)n));
  int* h_it = (int*)((char*)h_st + up16(4 * (size_t)n));
  long long* h_rls = (long long*)((char*)h_it + up16(4 * (size_t)n));
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_th, V->d_res_theta, b_th, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_tip, V->d_res_tip, b_tip, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_n, V->d_res_n, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_l, V->d_res_l, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_st, V->d_res_status, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_it, V->d_res_iters, 4 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_rls, V->d_res_rls, 8 * (size_t)n, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  const double t = clock_s();
  std::lock_guard<std::mutex> lk(V->mu);
  long long th0 = 0;
  for (Request* R : done) {
    const int b = (int)R->out_base;
    R->theta.assign(h_th + th0, h_th + th0 + R->links);
    th0 += R->links;
    R->tip.assign(h_tip + 2 * b, h_tip + 2 * (b + R->n));
    R->n_present.assign(h_n + b, h_n + b + R->n);
    R->l_last.assign(h_l + b, h_l + b + R->n);
    R->status.assign(h_st + b, h_st + b + R->n);
    R->iters.assign(h_it + b, h_it + b + R->n);
    R->rls = 0;
    for (int k = 0; k < R->n; ++k) R->rls += h_rls[b + k];
    R->t_done = t;
    R->state = 2;
    V->lanes[R->lane].load -= R->n;
    for (int t : R->tabs) V->tab_ref[t] -= 1;  // entries no live request holds are reused
    R->tabs.clear();
    for (int s : R->slots) V->free_slots.push_back(s);
    R->slots.clear();
    R->image.clear();
    R->image.shrink_to_fit();
    V->stats.requests_done += 1;
    V->stats.robot_link_steps += R->rls;
  }
  V->active.erase(std::remove_if(V->active.begin(), V->active.end(), [](Request* R) { return R->state == 2; }),
                  V->active.end());
  V->cv_done.notify_all();
  return cudaSuccess;
}

void worker_main(vine_server* V) {
  cudaSetDevice(V->device);
  const int nl = (int)V->lanes.size();
  for (;;) {
    std::vector<Request*> adm;
    bool any_busy = false;
    for (const Lane& L : V->lanes) any_busy = any_busy || L.busy;
    {
      std::unique_lock<std::mutex> lk(V->mu);
      if (V->active.empty() && !any_busy)
        V->cv_work.wait(lk, [&] { return V->stop || !V->waiting.empty(); });
      if (V->stop) break;
      while (!V->waiting.empty()) {
        adm.push_back(V->waiting.front());
        V->waiting.pop_front();
      }
    }
    const double t0 = clock_s();
    cudaError_t e = cudaSuccess;
    for (Request* R : adm) {
      if (e == cudaSuccess) e = admit(V, R);
      if (e != cudaSuccess) {
        std::lock_guard<std::mutex> lk(V->mu);
        if (R->state == 0) {
          V->promised -= R->n;
          R->state = 3;
        }
      }
    }
    if (e == cudaSuccess && !adm.empty()) e = cudaEventRecord(V->ev_admit, V->stream);
    // idle lanes: retire what is done, launch what still grows
    bool progressed = !adm.empty();
    for (int q = 0; q < nl && e == cudaSuccess; ++q) {
      Lane& L = V->lanes[q];
      if (L.busy) {
        const cudaError_t qe = cudaEventQuery(L.ev);
        if (qe == cudaErrorNotReady) continue;
        if (qe != cudaSuccess) {
          e = qe;
          break;
        }
        for (int s : L.robots) {
          V->slot_ncur[s] = L.h_ncur[s];
          V->slot_status[s] = L.h_status[s];
        }
        L.busy = false;
        progressed = true;
        std::lock_guard<std::mutex> lk(V->mu);
        V->stats.ticks += 1;
      }
      e = retire(V, q);
      bool launched = false;
      if (e == cudaSuccess) e = launch_lane(V, q, &launched);
      progressed = progressed || launched;
    }
    if (e != cudaSuccess) {
      std::lock_guard<std::mutex> lk(V->mu);
      char b[384];
      std::snprintf(b, sizeof(b), "vine_server worker: %s", cudaGetErrorString(e));
      V->error = b;
      for (Request* R : V->active) R->state = 3;
      for (Request* R : V->waiting) R->state = 3;
      V->active.clear();
      V->waiting.clear();
      V->stop = true;
      V->cv_done.notify_all();
      break;
    }
    any_busy = false;
    for (const Lane& L : V->lanes) any_busy = any_busy || L.busy;
    if (any_busy) {
      std::unique_lock<std::mutex> lk(V->mu);
      V->stats.busy_s += clock_s() - t0;
      // a launch is in flight: look again shortly, or as soon as a request arrives
      if (!progressed) V->cv_work.wait_for(lk, std::chrono::microseconds(100));
    }
  }
  for (Lane& L : V->lanes)
    if (L.st) cudaStreamSynchronize(L.st);
}

}  // namespace

extern "C" {

vine_status vine_server_config_default(vine_server_config* c) {
  if (!c) return sfail(VINE_EINVAL, "vine_server_config_default: null pointer");
  std::memset(c, 0, sizeof(*c));
  c->device_mem_budget = (size_t)1 << 30;
  c->max_slots = 0;
  c->max_links = 320;
  c->max_obs = 256;
  c->max_act = 16;
  c->max_request = 256;
  c->steps_per_tick = 0;  // to completion: a robot grows to its full length within one launch
  c->max_tables = 256;
  c->lanes = 4;
  c->window = 0;
  return VINE_OK;
}

vine_status vine_serve_clock(double* seconds) {
  if (!seconds) return sfail(VINE_EINVAL, "vine_serve_clock: null pointer");
  *seconds = clock_s();
  return VINE_OK;
}

vine_status vine_server_create(const vine_params* params, const vine_server_config* config, vine_server** out) {
  if (!out) return sfail(VINE_EINVAL, "vine_server_create: null output");
  *out = nullptr;
  vine_params prm;
  if (params) {
    prm = *params;
  } else {
    vine_params_default(&prm);
  }
  if (!(prm.tol > 0.0) || prm.max_iter < 1 || prm.max_halvings < 0 || !(prm.eps_crit > 0.0 && prm.eps_crit < 1.0) ||
      !(prm.R_c > 0.0 && prm.R_act > prm.R_c) || !(prm.m_lo > 0.0 && prm.m_lo < 0.5) || !(prm.pen_frac > 0.0) ||
      !(prm.fval_eps >= 0.0) || !(prm.armijo_c1 > 0.0 && prm.armijo_c1 < 0.5) || prm.discs_per_link < 1 ||
      prm.discs_per_link > 4 || (prm.mode != 0 && prm.mode != 1) ||
      (prm.mode == 1 && (prm.gd_steps < 1 || !(prm.gd_alpha > 0.0))) ||
      (prm.threads_per_robot != 0 && prm.threads_per_robot != 32 && prm.threads_per_robot != 64 &&
       prm.threads_per_robot != 128))
    return sfail(VINE_EINVAL, "vine_server_create: parameter out of range");
  vine_server_config c;
  vine_server_config_default(&c);
  if (config) {
    if (config->device_mem_budget) c.device_mem_budget = config->device_mem_budget;
    if (config->max_slots) c.max_slots = config->max_slots;
    if (config->max_links) c.max_links = config->max_links;
    if (config->max_obs) c.max_obs = config->max_obs;
    if (config->max_act) c.max_act = config->max_act;
    if (config->max_request) c.max_request = config->max_request;
    c.steps_per_tick = config->steps_per_tick;
    if (config->max_tables) c.max_tables = config->max_tables;
    if (config->lanes) c.lanes = config->lanes;
    if (config->window) c.window = config->window;
  }
  if (c.max_slots < 0 || c.max_links < 1 || c.max_links > kMaxLinks || c.max_obs < 1 || c.max_obs > kMaxObs ||
      c.max_act < 1 || c.max_act > kMaxAct || c.max_request < 1 || c.steps_per_tick < 0 || c.max_tables < 1 ||
      c.lanes < 1 || c.lanes > 8 || c.window < 0)
    return sfail(VINE_EINVAL, "vine_server_create: configuration out of range");
  if (c.steps_per_tick == 0 || c.steps_per_tick > c.max_links) c.steps_per_tick = c.max_links;
  auto V = new vine_server();
  V->prm = prm;
  V->cfg = c;
  V->ks = prm.discs_per_link;
  V->nmax = (c.max_links + 31) & ~31;
  V->omax = c.max_obs;
  V->amax = c.max_act;
  cudaGetDevice(&V->device);
  const int T = c.max_tables;
  const size_t per_slot = sizeof(InstDev) + 16 * (size_t)(V->omax + V->amax) + 8 * (size_t)V->nmax + 72 +
                          4 * (size_t)c.lanes + 12 + 8 + 24 + 7 * 256 / 64;
  const size_t na_max = (size_t)c.max_request * c.max_act, no_max = (size_t)c.max_request * c.max_obs;
  const size_t n_req = (size_t)c.max_request;
  V->stage_bytes = up256(4 * n_req * 4 + 12 * n_req + 8 * (n_req + 1) + na_max * 21 + no_max * 17 + 4 * na_max +
                         8 * n_req + 32 * 16);
  const size_t fixed = 16 * (size_t)T + sizeof(float2) * (size_t)T * kKnots + 8 * (size_t)T +
                       8 * (4 * (size_t)T + (size_t)T * kKnots + 2 * (kUCells + 1)) + sizeof(float2) * (kUCells + 1) +
                       64 + V->stage_bytes + 40 * 256;
  if (c.device_mem_budget <= fixed) {
    delete V;
    return sfail(VINE_EINVAL, "vine_server_create: device memory budget too small");
  }
  int S = (int)std::min<size_t>((c.device_mem_budget - fixed) / per_slot, (size_t)1 << 20);
  if (c.max_slots > 0) {
    if (c.max_slots > S) {
      delete V;
      return sfail(VINE_EINVAL, "vine_server_create: max_slots does not fit the device memory budget");
    }
    S = c.max_slots;
  } else {
    S = std::min(S, 65536);
  }
  if (S < c.max_request) {
    delete V;
    return sfail(VINE_EINVAL, "vine_server_create: budget holds fewer slots than one maximal request");
  }
  V->S = S;
  V->cfg.max_slots = S;
  // ---- device memory
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off += up256(std::max<size_t>(bytes, 16));
    return o;
  };
  const size_t Ss = (size_t)S;
  const size_t o_inst = take(sizeof(InstDev) * Ss), o_obs = take(16 * Ss * V->omax), o_act = take(16 * Ss * V->amax),
               o_th = take(4 * Ss * V->nmax), o_n = take(4 * Ss), o_l = take(4 * Ss), o_st = take(4 * Ss),
               o_it = take(4 * Ss), o_cv = take(4 * Ss), o_sp = take(4 * Ss), o_rls = take(8 * Ss),
               o_ev = take(8 * Ss), o_le = take(8 * Ss), o_fb = take(8 * Ss), o_cy = take(8 * Ss),
               o_pt = take(8 * Ss), o_rm = take(8 * Ss), o_ord = take(4 * Ss * c.lanes), o_cnt = take(16 * (size_t)c.lanes),
               o_hdr = take(16 * (size_t)T),
               o_tab = take(sizeof(float2) * (size_t)T * kKnots), o_ut = take(sizeof(float2) * (kUCells + 1)),
               o_l0 = take(8 * (size_t)T), o_scr = take(8 * (4 * (size_t)T + (size_t)T * kKnots + 2 * (kUCells + 1))),
               o_cst = take(32), o_stage = take(V->stage_bytes), o_sel = take(4 * Ss), o_oo = take(8 * Ss),
               o_rth = take(4 * Ss * V->nmax), o_rtip = take(8 * Ss), o_rn = take(4 * Ss), o_rl = take(4 * Ss),
               o_rst = take(4 * Ss), o_rit = take(4 * Ss), o_rrls = take(8 * Ss);
  if (off > c.device_mem_budget) {
    delete V;
    return sfail(VINE_EINVAL, "vine_server_create: layout exceeds the device memory budget");
  }
  cudaError_t e = cudaMalloc(&V->dmem, off);
  if (e != cudaSuccess) {
    delete V;
    return scuda(e, "vine_server_create: cudaMalloc");
  }
  char* m = V->dmem;
  auto cleanup = [&]() {
    for (Lane& L : V->lanes) {
      if (L.h_order) cudaFreeHost(L.h_order);
      if (L.h_ncur) cudaFreeHost(L.h_ncur);
      if (L.h_status) cudaFreeHost(L.h_status);
      if (L.ev) cudaEventDestroy(L.ev);
      if (L.st) cudaStreamDestroy(L.st);
    }
    if (V->h_res) cudaFreeHost(V->h_res);
    if (V->ev_admit) cudaEventDestroy(V->ev_admit);
    if (V->stream) cudaStreamDestroy(V->stream);
    cudaFree(V->dmem);
    delete V;
  };
#define CKS(call)                                   \
  do {                                              \
    cudaError_t e_ = (call);                        \
    if (e_ != cudaSuccess) {                        \
      vine_status s_ = scuda(e_, #call);            \
      cleanup();                                    \
      return s_;                                    \
    }                                               \
  } while (0)
  CKS(cudaStreamCreateWithFlags(&V->stream, cudaStreamNonBlocking));
  CKS(cudaEventCreateWithFlags(&V->ev_admit, cudaEventDisableTiming));
  V->lanes.resize(c.lanes);
  for (int q = 0; q < c.lanes; ++q) {
    Lane& L = V->lanes[q];
    CKS(cudaStreamCreateWithFlags(&L.st, cudaStreamNonBlocking));
    CKS(cudaEventCreateWithFlags(&L.ev, cudaEventDisableTiming));
    CKS(cudaMallocHost(&L.h_order, 4 * Ss));
    CKS(cudaMallocHost(&L.h_ncur, 4 * Ss));
    CKS(cudaMallocHost(&L.h_status, 4 * Ss));
    L.d_order = (int*)(m + o_ord) + (size_t)q * Ss;
    L.d_counter = (int*)(m + o_cnt) + 4 * q;
  }
  V->h_res_bytes = up16(4 * Ss * V->nmax) + up16(8 * Ss) + 4 * up16(4 * Ss) + up16(8 * Ss) + 256;
  CKS(cudaMallocHost(&V->h_res, V->h_res_bytes));
  CKS(cudaMemsetAsync(m, 0, off, V->stream));
  // wrinkling table and the model constants derived from it
  GaussLegendre gl;
  gauss_legendre(24, &gl);
  double* scr = (double*)(m + o_scr);
  CKS(launch_wrinkle_table(prm.eps_crit, gl, (float2*)(m + o_ut), scr + 4 * (size_t)T + (size_t)T * kKnots,
                           (double*)(m + o_cst), V->stream));
  double cst[4];
  CKS(cudaMemcpyAsync(cst, m + o_cst, sizeof(cst), cudaMemcpyDeviceToHost, V->stream));
  CKS(cudaEventRecord(V->ev_admit, V->stream));
  CKS(cudaStreamSynchronize(V->stream));
  if (!(std::isfinite(cst[0]) && std::isfinite(cst[1]))) {
    cleanup();
    return sfail(VINE_ECUDA, "vine_server_create: wrinkling table build failed");
  }
  // launch configuration
  // threads per robot as for batches (by the slot capacity in links when 0)
  if (prm.threads_per_robot == 0)
    V->team = c.max_links <= 64 ? 32 : (c.max_links <= 200 ? 64 : 128);
  else
    V->team = prm.threads_per_robot;
  V->smem_warp = grow_smem_per_warp(V->nmax, V->omax, V->amax, V->team);
  int nsm = 1, per_sm = 0;
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, V->device);
  V->wpc = grow_pick_block(V->ks, V->smem_warp, &per_sm, V->team);
  if (V->wpc == 0 || per_sm == 0) {
    cleanup();
    return sfail(VINE_EINVAL, "vine_server_create: slot capacities too large for shared memory");
  }
  V->grid = nsm * per_sm;
  // twice the resident warps per lane: the lanes' launches queue their CTAs
  // behind each other, so the SMs a launch leaves idle while its slowest
  // robots finish are taken at once by the next launch
  V->window = c.window > 0 ? c.window : std::max(1, 2 * V->grid * V->wpc);
  V->cfg.window = V->window;
  GrowArgs& a = V->args;
  a.inst = (const InstDev*)(m + o_inst);
  a.obs = (const float4*)(m + o_obs);
  a.act = (const float4*)(m + o_act);
  a.tab_hdr = (const float4*)(m + o_hdr);
  a.tab = (const float2*)(m + o_tab);
  a.utab = (const float2*)(m + o_ut);
  a.theta = (float*)(m + o_th);
  a.n_cur = (int*)(m + o_n);
  a.l_cur = (float*)(m + o_l);
  a.status = (int*)(m + o_st);
  a.iters = (int*)(m + o_it);
  a.conv = (int*)(m + o_cv);
  a.steps = (int*)(m + o_sp);
  a.rls = (long long*)(m + o_rls);
  a.evals = (long long*)(m + o_ev);
  a.linkevals = (long long*)(m + o_le);
  a.pairtests = (long long*)(m + o_pt);
  a.fallbacks = (long long*)(m + o_fb);
  a.cycles = (long long*)(m + o_cy);
  a.resid_max = (double*)(m + o_rm);
  a.order = (const int*)(m + o_ord);
  a.n_order = 0;
  a.counter = (int*)(m + o_cnt);
  a.dynamic = 1;
  a.n_steps = c.steps_per_tick;
  a.nmax = V->nmax;
  a.omax = V->omax;
  a.amax = V->amax;
  a.warp_floats = (int)(V->smem_warp / sizeof(float));
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
  a.mode = prm.mode;
  a.gd_steps = prm.gd_steps;
  a.gd_alpha = (float)prm.gd_alpha;
  a.list_margin = kListMargin;
  a.team = V->team;
  V->d_l0 = (double*)(m + o_l0);
  V->d_scr = scr;
  V->d_stage = m + o_stage;
  V->d_sel = (int*)(m + o_sel);
  V->d_outoff = (long long*)(m + o_oo);
  V->d_res_theta = (float*)(m + o_rth);
  V->d_res_tip = (float*)(m + o_rtip);
  V->d_res_n = (int*)(m + o_rn);
  V->d_res_l = (float*)(m + o_rl);
  V->d_res_status = (int*)(m + o_rst);
  V->d_res_iters = (int*)(m + o_rit);
  V->d_res_rls = (long long*)(m + o_rrls);
#undef CKS
  V->free_slots.resize(S);
  for (int k = 0; k < S; ++k) V->free_slots[k] = S - 1 - k;  // slot 0 handed out first
  V->slot_target.assign(S, 0);
  V->slot_nobs.assign(S, 0);
  V->slot_ncur.assign(S, 0);
  V->slot_status.assign(S, 0);
  V->stats.max_slots = S;
  V->worker = std::thread(worker_main, V);
  *out = V;
  return VINE_OK;
}

vine_status vine_serve_submit(vine_server* V, const vine_batch_desc* D, uint64_t* request_id) {
  if (!V || !D || !request_id) return sfail(VINE_EINVAL, "vine_serve_submit: null argument");
  if (D->mem_is_device) return sfail(VINE_EINVAL, "vine_serve_submit: requests are read from host memory");
  const int n = D->n_inst;
  if (n < 1 || n > V->cfg.max_request) return sfail(VINE_EINVAL, "vine_serve_submit: robot count out of range");
  if (!D->n_links || !D->l_seg || !D->radius || !D->pressure || !D->base || !D->act_ptr || !D->obs_ptr)
    return sfail(VINE_EINVAL, "vine_serve_submit: null input array");
  if (D->act_ptr[0] != 0 || D->obs_ptr[0] != 0)
    return sfail(VINE_EINVAL, "vine_serve_submit: act_ptr/obs_ptr must start at 0");
  auto R = new Request();
  R->n = n;
  R->n_links.resize(n);
  R->n_obs_r.resize(n);
  for (int i = 0; i < n; ++i) {
    const int nl = D->n_links[i], na = D->act_ptr[i + 1] - D->act_ptr[i], no = D->obs_ptr[i + 1] - D->obs_ptr[i];
    if (nl < 1 || nl > V->cfg.max_links || na < 0 || na > V->amax || no < 0 || no > V->omax) {
      delete R;
      return sfail(VINE_EINVAL, "vine_serve_submit: a robot exceeds the slot capacities");
    }
    R->n_links[i] = nl;
    R->n_obs_r[i] = no;
    R->links += nl;
  }
  R->n_act = D->act_ptr[n];
  R->n_obs = D->obs_ptr[n];
  if ((R->n_act > 0 && (!D->act_begin || !D->act_end || !D->act_side || !D->act_pressure || !D->act_l0)) ||
      (R->n_obs > 0 && (!D->obs_kind || !D->obs_cx || !D->obs_cy || !D->obs_a || !D->obs_b))) {
    delete R;
    return sfail(VINE_EINVAL, "vine_serve_submit: null input array");
  }
  const size_t na = (size_t)R->n_act, no = (size_t)R->n_obs, nn = (size_t)n;
  const size_t sz[F_COUNT] = {4 * nn, 4 * nn, 4 * nn, 4 * nn, 12 * nn, 4 * (nn + 1), 4 * na, 4 * na, na, 4 * na,
                              4 * na, 4 * (nn + 1), no, 4 * no, 4 * no, 4 * no, 4 * no, 4 * na, 4 * nn, 4 * nn};
  const void* src[F_COUNT] = {D->n_links, D->l_seg, D->radius, D->pressure, D->base, D->act_ptr, D->act_begin,
                              D->act_end, D->act_side, D->act_pressure, D->act_l0, D->obs_ptr, D->obs_kind,
                              D->obs_cx, D->obs_cy, D->obs_a, D->obs_b, nullptr, nullptr, nullptr};
  size_t o = 0;
  for (int f = 0; f < F_COUNT; ++f) {
    R->off[f] = o;
    o += up16(std::max<size_t>(sz[f], 1));
  }
  if (o > V->stage_bytes) {
    delete R;
    return sfail(VINE_EINVAL, "vine_serve_submit: request larger than the upload staging");
  }
  R->image.assign(o, 0);
  for (int f = 0; f < F_COUNT; ++f)
    if (src[f] && sz[f]) std::memcpy(R->image.data() + R->off[f], src[f], sz[f]);
  for (int a = 0; a < R->n_act; ++a) {
    const double v = D->act_l0[a];
    if (std::isfinite(v) && v > 0.0 && std::find(R->l0.begin(), R->l0.end(), v) == R->l0.end()) R->l0.push_back(v);
  }
  std::lock_guard<std::mutex> lk(V->mu);
  if (V->stop) {
    delete R;
    return sfail(VINE_ECUDA, V->error.empty() ? "vine_serve_submit: server stopped" : V->error.c_str());
  }
  // the cell lengths live once this request is admitted: those held by
  // admitted requests, those of waiting requests, and its own
  if ((int)R->l0.size() > V->cfg.max_tables) {
    delete R;
    return sfail(VINE_EINVAL, "vine_serve_submit: more distinct sPAM cell lengths than the table capacity");
  }
  std::vector<double> known;
  for (size_t k = 0; k < V->tab_l0.size(); ++k)
    if (V->tab_ref[k] > 0) known.push_back(V->tab_l0[k]);
  for (Request* W : V->waiting)
    for (double v : W->l0)
      if (std::find(known.begin(), known.end(), v) == known.end()) known.push_back(v);
  for (double v : R->l0)
    if (std::find(known.begin(), known.end(), v) == known.end()) known.push_back(v);
  if ((int)known.size() > V->cfg.max_tables) {
    delete R;
    return sfail(VINE_EBUSY, "vine_serve_submit: more distinct live sPAM cell lengths than the table capacity; "
                             "retry when requests holding others have finished");
  }
  if ((int)V->free_slots.size() - V->promised < n) {
    delete R;
    return sfail(VINE_EBUSY, "vine_serve_submit: not enough free slots; retry later");
  }
  V->promised += n;
  R->id = V->next_id++;
  R->t_submit = clock_s();
  V->reqs[R->id] = R;
  V->waiting.push_back(R);
  *request_id = R->id;
  V->cv_work.notify_all();
  return VINE_OK;
}

vine_status vine_serve_poll(vine_server* V, uint64_t id, int32_t timeout_us, vine_request_info* info, float* theta,
                            float* l_last, float* tip, int32_t* n_present, int32_t* inst_status, int32_t* iterations) {
  if (!V) return sfail(VINE_EINVAL, "vine_serve_poll: null server");
  if (timeout_us < 0) return sfail(VINE_EINVAL, "vine_serve_poll: negative timeout");
  std::unique_lock<std::mutex> lk(V->mu);
  auto it = V->reqs.find(id);
  if (it == V->reqs.end()) return sfail(VINE_EINVAL, "vine_serve_poll: unknown request id");
  Request* R = it->second;
  const auto until = std::chrono::steady_clock::now() + std::chrono::microseconds(timeout_us);
  V->cv_done.wait_until(lk, until, [&] { return R->state >= 2; });
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->n_inst = R->n;
    info->total_links = R->links;
    info->t_submit = R->t_submit;
    info->t_admit = R->t_admit;
  }
  if (R->state == 3) {
    V->reqs.erase(it);
    delete R;
    return sfail(VINE_ECUDA, V->error.empty() ? "vine_serve_poll: request failed" : V->error.c_str());
  }
  if (R->state != 2) return sfail(VINE_ETIMEOUT, "vine_serve_poll: not finished");
  if (info) {
    info->robot_link_steps = R->rls;
    info->t_done = R->t_done;
  }
  const size_t n = (size_t)R->n;
  if (theta) std::memcpy(theta, R->theta.data(), sizeof(float) * R->theta.size());
  if (l_last) std::memcpy(l_last, R->l_last.data(), sizeof(float) * n);
  if (tip) std::memcpy(tip, R->tip.data(), sizeof(float) * 2 * n);
  if (n_present) std::memcpy(n_present, R->n_present.data(), sizeof(int32_t) * n);
  if (inst_status) std::memcpy(inst_status, R->status.data(), sizeof(int32_t) * n);
  if (iterations) std::memcpy(iterations, R->iters.data(), sizeof(int32_t) * n);
  V->reqs.erase(it);
  delete R;
  return VINE_OK;
}

vine_status vine_server_get_stats(vine_server* V, vine_server_stats* out) {
  if (!V || !out) return sfail(VINE_EINVAL, "vine_server_get_stats: null argument");
  std::lock_guard<std::mutex> lk(V->mu);
  *out = V->stats;
  int act = 0;
  for (Request* R : V->active) act += R->n;
  out->active_robots = act;
  out->waiting_requests = (int)V->waiting.size();
  out->free_slots = (int)V->free_slots.size() - V->promised;
  out->max_slots = V->S;
  return VINE_OK;
}

vine_status vine_server_destroy(vine_server* V) {
  if (!V) return VINE_OK;
  {
    std::lock_guard<std::mutex> lk(V->mu);
    V->stop = true;
    V->cv_work.notify_all();
  }
  if (V->worker.joinable()) V->worker.join();
  cudaStreamSynchronize(V->stream);
  for (auto& kv : V->reqs) delete kv.second;
  for (Lane& L : V->lanes) {
    cudaStreamSynchronize(L.st);
    cudaFreeHost(L.h_order);
    cudaFreeHost(L.h_ncur);
    cudaFreeHost(L.h_status);
    cudaEventDestroy(L.ev);
    cudaStreamDestroy(L.st);
  }
  cudaEventDestroy(V->ev_admit);
  cudaFreeHost(V->h_res);
  cudaStreamDestroy(V->stream);
  cudaFree(V->dmem);
  delete V;
  return VINE_OK;
}

}  // extern "C"
