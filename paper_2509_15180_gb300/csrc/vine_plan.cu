// vine_plan.cu -- tree operations of the batched SST* planner (Sec. 5.2,
// Algorithm 2) behind vine_sst_prune and vine_sst_select (include/vine.h).
//
// Both are all-pairs sweeps over tip poses: every new state (or sample)
// against every tree node.  One thread owns one query; the CTA's queries
// sweep a chunk of the candidate range, staged through shared memory in
// tiles, and the grid's second dimension splits the candidate range into
// chunks so that a few thousand queries still fill the 152 SMs.  Partial
// results per (chunk, query) are combined in chunk order by a second
// launch, so the result does not depend on scheduling.
//
// Distances: d^2 = dx^2 + dy^2 + (rho * dphi)^2 in float32 with every
// product and sum rounded on its own (__fmul_rn / __fadd_rn: no fused
// multiply-add), dphi wrapped by one add or subtract of 2 pi.  Two states
// overlap when d^2 < r^2 (r^2 rounded the same way).  Costs compare exactly
// (float64); ties go to the lower id, tree nodes numbered before new states.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "vine.h"
#include "vine_internal.cuh"

using namespace vine;

namespace {

constexpr int kQ = 128;     // queries (threads) per CTA
constexpr int kTile = 256;  // candidates per shared-memory tile
constexpr int kMaxChunks = 64;

vine_status pfail(vine_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

vine_status pcuda(cudaError_t e, const char* where) {
  char b[384];
  std::snprintf(b, sizeof(b), "%s: %s", where, cudaGetErrorString(e));
  set_last_error(b);
  return e == cudaErrorMemoryAllocation ? VINE_ENOMEM : VINE_ECUDA;
}

#define PK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return pcuda(e_, #call);   \
  } while (0)

__device__ __forceinline__ float se2_d2(float ax, float ay, float ap, float bx, float by, float bp, float rho) {
  const float kPiF = 3.14159265358979323846f, k2PiF = 6.28318530717958647692f;
  const float dx = __fsub_rn(ax, bx), dy = __fsub_rn(ay, by);
  float dp = __fsub_rn(ap, bp);
  if (dp > kPiF)
    dp = __fsub_rn(dp, k2PiF);
  else if (dp < -kPiF)
    dp = __fadd_rn(dp, k2PiF);
  const float rp = __fmul_rn(rho, dp);
  return __fadd_rn(__fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)), __fmul_rn(rp, rp));
}

// key (ca, ia) < key (cb, ib)
__device__ __forceinline__ bool key_less(double ca, long long ia, double cb, long long ib) {
  return ca < cb || (ca == cb && ia < ib);
}

struct Tile {
  float x[kTile], y[kTile], p[kTile];
  double c[kTile];
  unsigned char ok[kTile];
};

// Candidates are the concatenation [tree nodes (n_old) | new states (n_new)];
// candidate k has id k.  Stages tile [t0, t0 + kTile) of a chunk.
__device__ void stage(Tile& T, int t0, int t1, int n_old, const float* old_pose, const double* old_cost,
                      const unsigned char* old_ok, const float* new_pose, const double* new_cost) {
  for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
    const int g = t0 + k;
    if (g < t1) {
      const bool is_old = g < n_old;
      const int q = is_old ? g : g - n_old;
      const float* P = is_old ? old_pose : new_pose;
      T.x[k] = P[3 * q];
      T.y[k] = P[3 * q + 1];
      T.p[k] = P[3 * q + 2];
      const double c = is_old ? old_cost[q] : new_cost[q];
      T.c[k] = c;
      T.ok[k] = is_old ? (old_ok[q] != 0) : (isfinite(c) ? 1 : 0);
    } else {
      T.ok[k] = 0;
    }
  }
}

// Prune, pass 1: new state j is dominated when an overlapping candidate
// (active tree node or new state with finite cost) has a smaller key.
__global__ void __launch_bounds__(kQ) prune_dominated_kernel(int n_old, const float* old_pose, const double* old_cost,
                                                           const unsigned char* old_active, int n_new,
                                                           const float* new_pose, const double* new_cost, float r,
                                                           float rho, int chunk, int* dominated) {
  __shared__ Tile T;
  const int j = blockIdx.x * kQ + threadIdx.x;
  const bool live = j < n_new;
  const float qx = live ? new_pose[3 * j] : 0.f, qy = live ? new_pose[3 * j + 1] : 0.f,
              qp = live ? new_pose[3 * j + 2] : 0.f;
  const double qc = live ? new_cost[j] : 0.0;
  const long long qid = (long long)n_old + j;
  const float r2 = __fmul_rn(r, r);
  const int n_all = n_old + n_new;
  const int c0 = blockIdx.y * chunk, c1 = min(n_all, c0 + chunk);
  bool dom = false;
  for (int t0 = c0; t0 < c1; t0 += kTile) {
    const int t1 = min(c1, t0 + kTile);
    __syncthreads();
    stage(T, t0, t1, n_old, old_pose, old_cost, old_active, new_pose, new_cost);
    __syncthreads();
    if (live && !dom) {
      for (int k = 0; k < t1 - t0; ++k) {
        if (!T.ok[k] || !key_less(T.c[k], (long long)(t0 + k), qc, qid)) continue;
        if (se2_d2(qx, qy, qp, T.x[k], T.y[k], T.p[k], rho) < r2) {
          dom = true;
          break;
        }
      }
    }
  }
  if (live && dom) atomicOr(dominated + j, 1);
}

__global__ void prune_keep_kernel(int n_new, const double* new_cost, const int* dominated, unsigned char* keep) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < n_new) keep[j] = (!dominated[j] && isfinite(new_cost[j])) ? 1 : 0;
}

// Prune, pass 2: active tree node i is deactivated when a kept new state
// with a smaller key overlaps it.  Candidates are the new states only.
__global__ void __launch_bounds__(kQ) prune_deactivate_kernel(int n_old, const float* old_pose,
                                                            const double* old_cost, const unsigned char* old_active,
                                                            int n_new, const float* new_pose, const double* new_cost,
                                                            const unsigned char* keep, float r, float rho, int chunk,
                                                            int* deact) {
  __shared__ Tile T;
  const int i = blockIdx.x * kQ + threadIdx.x;
  const bool live = i < n_old && old_active[i] != 0;
  const float qx = live ? old_pose[3 * i] : 0.f, qy = live ? old_pose[3 * i + 1] : 0.f,
              qp = live ? old_pose[3 * i + 2] : 0.f;
  const double qc = live ? old_cost[i] : 0.0;
  const float r2 = __fmul_rn(r, r);
  const int c0 = blockIdx.y * chunk, c1 = min(n_new, c0 + chunk);
  bool hit = false;
  for (int t0 = c0; t0 < c1; t0 += kTile) {
    const int t1 = min(c1, t0 + kTile);
    __syncthreads();
    for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
      const int g = t0 + k;
      if (g < t1) {
        T.x[k] = new_pose[3 * g];
        T.y[k] = new_pose[3 * g + 1];
        T.p[k] = new_pose[3 * g + 2];
        T.c[k] = new_cost[g];
        T.ok[k] = keep[g];
      } else {
        T.ok[k] = 0;
      }
    }
    __syncthreads();
    if (live && !hit) {
      for (int k = 0; k < t1 - t0; ++k) {
        if (!T.ok[k] || !key_less(T.c[k], (long long)n_old + t0 + k, qc, (long long)i)) continue;
        if (se2_d2(qx, qy, qp, T.x[k], T.y[k], T.p[k], rho) < r2) {
          hit = true;
          break;
        }
      }
    }
  }
  if (live && hit) atomicOr(deact + i, 1);
}

__global__ void flags_to_bytes_kernel(int n, const int* f, unsigned char* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = f[i] ? 1 : 0;
}

struct SelPart {
  double best_c;  // smallest cost within delta (its node in best_i; -1 none)
  int best_i;
  float near_d2;  // smallest distance (its node in near_i; -1 none)
  int near_i;
};

__global__ void __launch_bounds__(kQ) select_partial_kernel(int n_nodes, const float* pose, const double* cost,
                                                          const unsigned char* active, int n_samples,
                                                          const float* spose, float delta, float rho, int chunk,
                                                          SelPart* part) {
  __shared__ Tile T;
  const int s = blockIdx.x * kQ + threadIdx.x;
  const bool live = s < n_samples;
  const float qx = live ? spose[3 * s] : 0.f, qy = live ? spose[3 * s + 1] : 0.f, qp = live ? spose[3 * s + 2] : 0.f;
  const float d2lim = __fmul_rn(delta, delta);
  const int c0 = blockIdx.y * chunk, c1 = min(n_nodes, c0 + chunk);
  SelPart P{0.0, -1, 0.f, -1};
  for (int t0 = c0; t0 < c1; t0 += kTile) {
    const int t1 = min(c1, t0 + kTile);
    __syncthreads();
    for (int k = threadIdx.x; k < kTile; k += blockDim.x) {
      const int g = t0 + k;
      if (g < t1) {
        T.x[k] = pose[3 * g];
        T.y[k] = pose[3 * g + 1];
        T.p[k] = pose[3 * g + 2];
        T.c[k] = cost[g];
        T.ok[k] = active[g] != 0;
      } else {
        T.ok[k] = 0;
      }
    }
    __syncthreads();
    if (live) {
      for (int k = 0; k < t1 - t0; ++k) {
        if (!T.ok[k]) continue;
        const int g = t0 + k;
        const float d2 = se2_d2(qx, qy, qp, T.x[k], T.y[k], T.p[k], rho);
        // candidates come in increasing index, so strict comparisons keep the lower index on ties
        if (d2 < d2lim && (P.best_i < 0 || key_less(T.c[k], g, P.best_c, P.best_i))) {
          P.best_c = T.c[k];
          P.best_i = g;
        }
        if (P.near_i < 0 || d2 < P.near_d2) {
          P.near_d2 = d2;
          P.near_i = g;
        }
      }
    }
  }
  if (live) part[(size_t)blockIdx.y * n_samples + s] = P;
}

__global__ void select_reduce_kernel(int n_samples, int n_chunks, const SelPart* part, int* chosen) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n_samples) return;
  SelPart B{0.0, -1, 0.f, -1};
  for (int c = 0; c < n_chunks; ++c) {  // chunks in increasing index order
    const SelPart P = part[(size_t)c * n_samples + s];
    if (P.best_i >= 0 && (B.best_i < 0 || key_less(P.best_c, P.best_i, B.best_c, B.best_i))) {
      B.best_c = P.best_c;
      B.best_i = P.best_i;
    }
    if (P.near_i >= 0 && (B.near_i < 0 || P.near_d2 < B.near_d2)) {
      B.near_d2 = P.near_d2;
      B.near_i = P.near_i;
    }
  }
  chosen[s] = B.best_i >= 0 ? B.best_i : B.near_i;
}

// Candidate range split: enough CTAs for about four waves of 152 SMs, at
// least one tile per chunk, at most kMaxChunks chunks.
int chunks_for(int n_queries, int n_cand) {
  const int qb = std::max(1, (n_queries + kQ - 1) / kQ);
  const int want = std::max(1, (4 * 152 + qb - 1) / qb);
  const int max_by_tiles = std::max(1, (n_cand + kTile - 1) / kTile);
  return std::max(1, std::min({want, max_by_tiles, kMaxChunks}));
}

bool bad_scalar(float v) { return !std::isfinite(v) || v < 0.f; }

// Device scratch for one call, stream-ordered.
struct Scratch {
  cudaStream_t st;
  void* p = nullptr;
  explicit Scratch(cudaStream_t s) : st(s) {}
  ~Scratch() {
    if (p) cudaFreeAsync(p, st);
  }
};

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

}  // namespace

extern "C" {

vine_status vine_sst_prune(int32_t n_old, const float* old_pose, const double* old_cost, const uint8_t* old_active,
                           int32_t n_new, const float* new_pose, const double* new_cost, float radius, float rho,
                           uint8_t* new_keep, uint8_t* old_deactivate, int32_t ptrs_are_device, void* stream_v) {
  if (n_old < 0 || n_new < 0 || (long long)n_old + n_new > 0x7fffffffLL)
    return pfail(VINE_EINVAL, "vine_sst_prune: count out of range");
  if (bad_scalar(radius) || bad_scalar(rho)) return pfail(VINE_EINVAL, "vine_sst_prune: radius or rho out of range");
  if ((n_old > 0 && (!old_pose || !old_cost || !old_active || !old_deactivate)) ||
      (n_new > 0 && (!new_pose || !new_cost || !new_keep)))
    return pfail(VINE_EINVAL, "vine_sst_prune: null argument");
  cudaStream_t st = (cudaStream_t)stream_v;
  if (n_old == 0 && n_new == 0) return VINE_OK;
  const size_t no = (size_t)n_old, nn = (size_t)n_new;
  // scratch: flags (dominated[n_new], deact[n_old]) + host-path copies
  const size_t o_dom = 0, o_dea = up256(4 * nn), o_end_flags = o_dea + up256(4 * no);
  size_t o_op = o_end_flags, o_oc = 0, o_oa = 0, o_np = 0, o_nc = 0, o_keep = 0, o_odea = 0, total = o_end_flags;
  if (!ptrs_are_device) {
    o_op = total;
    o_oc = o_op + up256(12 * no);
    o_oa = o_oc + up256(8 * no);
    o_np = o_oa + up256(no);
    o_nc = o_np + up256(12 * nn);
    o_keep = o_nc + up256(8 * nn);
    o_odea = o_keep + up256(nn);
    total = o_odea + up256(no);
  }
  Scratch S(st);
  PK(cudaMallocAsync(&S.p, std::max<size_t>(total, 256), st));
  char* sp = (char*)S.p;
  int* dom = (int*)(sp + o_dom);
  int* dea = (int*)(sp + o_dea);
  const float *op = old_pose, *np_ = new_pose;
  const double *oc = old_cost, *nc = new_cost;
  const unsigned char* oa = old_active;
  unsigned char *keep = new_keep, *odea = old_deactivate;
  if (!ptrs_are_device) {
    if (no) {
      PK(cudaMemcpyAsync(sp + o_op, old_pose, 12 * no, cudaMemcpyHostToDevice, st));
      PK(cudaMemcpyAsync(sp + o_oc, old_cost, 8 * no, cudaMemcpyHostToDevice, st));
      PK(cudaMemcpyAsync(sp + o_oa, old_active, no, cudaMemcpyHostToDevice, st));
    }
    if (nn) {
      PK(cudaMemcpyAsync(sp + o_np, new_pose, 12 * nn, cudaMemcpyHostToDevice, st));
      PK(cudaMemcpyAsync(sp + o_nc, new_cost, 8 * nn, cudaMemcpyHostToDevice, st));
    }
    op = (const float*)(sp + o_op);
    oc = (const double*)(sp + o_oc);
    oa = (const unsigned char*)(sp + o_oa);
    np_ = (const float*)(sp + o_np);
    nc = (const double*)(sp + o_nc);
    keep = (unsigned char*)(sp + o_keep);
    odea = (unsigned char*)(sp + o_odea);
  }
  PK(cudaMemsetAsync(sp, 0, o_end_flags, st));
  if (nn) {
    const int n_all = n_old + n_new;
    const int ch = chunks_for(n_new, n_all);
    const int chunk = (n_all + ch - 1) / ch;
    prune_dominated_kernel<<<dim3((n_new + kQ - 1) / kQ, ch), kQ, 0, st>>>(n_old, op, oc, oa, n_new, np_, nc, radius,
                                                                           rho, chunk, dom);
    PK(cudaGetLastError());
    prune_keep_kernel<<<(n_new + 255) / 256, 256, 0, st>>>(n_new, nc, dom, keep);
    PK(cudaGetLastError());
  }
  if (no) {
    if (nn) {
      const int ch = chunks_for(n_old, n_new);
      const int chunk = (n_new + ch - 1) / ch;
      prune_deactivate_kernel<<<dim3((n_old + kQ - 1) / kQ, ch), kQ, 0, st>>>(n_old, op, oc, oa, n_new, np_, nc, keep,
                                                                              radius, rho, chunk, dea);
      PK(cudaGetLastError());
    }
    flags_to_bytes_kernel<<<(n_old + 255) / 256, 256, 0, st>>>(n_old, dea, odea);
    PK(cudaGetLastError());
  }
  if (!ptrs_are_device) {
    if (nn) PK(cudaMemcpyAsync(new_keep, keep, nn, cudaMemcpyDeviceToHost, st));
    if (no) PK(cudaMemcpyAsync(old_deactivate, odea, no, cudaMemcpyDeviceToHost, st));
    PK(cudaStreamSynchronize(st));
  }
  return VINE_OK;
}

vine_status vine_sst_select(int32_t n_nodes, const float* pose, const double* cost, const uint8_t* active,
                            int32_t n_samples, const float* sample_pose, float delta, float rho, int32_t* chosen,
                            int32_t ptrs_are_device, void* stream_v) {
  if (n_nodes < 0 || n_samples < 0) return pfail(VINE_EINVAL, "vine_sst_select: count out of range");
  if (bad_scalar(delta) || bad_scalar(rho)) return pfail(VINE_EINVAL, "vine_sst_select: delta or rho out of range");
  if ((n_nodes > 0 && (!pose || !cost || !active)) || (n_samples > 0 && (!sample_pose || !chosen)))
    return pfail(VINE_EINVAL, "vine_sst_select: null argument");
  cudaStream_t st = (cudaStream_t)stream_v;
  if (n_samples == 0) return VINE_OK;
  const size_t nn = (size_t)n_nodes, ns = (size_t)n_samples;
  const int ch = chunks_for(n_samples, n_nodes);
  const int chunk = std::max(1, (n_nodes + ch - 1) / ch);
  const size_t o_part = 0, o_end = up256(sizeof(SelPart) * ns * ch);
  size_t o_p = o_end, o_c = 0, o_a = 0, o_s = 0, o_out = 0, total = o_end;
  if (!ptrs_are_device) {
    o_p = total;
    o_c = o_p + up256(12 * nn);
    o_a = o_c + up256(8 * nn);
    o_s = o_a + up256(nn);
    o_out = o_s + up256(12 * ns);
    total = o_out + up256(4 * ns);
  }
  Scratch S(st);
  PK(cudaMallocAsync(&S.p, std::max<size_t>(total, 256), st));
  char* sp = (char*)S.p;
  const float *P = pose, *SP = sample_pose;
  const double* Cc = cost;
  const unsigned char* A = active;
  int* out = chosen;
  if (!ptrs_are_device) {
    if (nn) {
      PK(cudaMemcpyAsync(sp + o_p, pose, 12 * nn, cudaMemcpyHostToDevice, st));
      PK(cudaMemcpyAsync(sp + o_c, cost, 8 * nn, cudaMemcpyHostToDevice, st));
      PK(cudaMemcpyAsync(sp + o_a, active, nn, cudaMemcpyHostToDevice, st));
    }
    PK(cudaMemcpyAsync(sp + o_s, sample_pose, 12 * ns, cudaMemcpyHostToDevice, st));
    P = (const float*)(sp + o_p);
    Cc = (const double*)(sp + o_c);
    A = (const unsigned char*)(sp + o_a);
    SP = (const float*)(sp + o_s);
    out = (int*)(sp + o_out);
  }
  SelPart* part = (SelPart*)(sp + o_part);
  select_partial_kernel<<<dim3((n_samples + kQ - 1) / kQ, ch), kQ, 0, st>>>(n_nodes, P, Cc, A, n_samples, SP, delta,
                                                                            rho, chunk, part);
  PK(cudaGetLastError());
  select_reduce_kernel<<<(n_samples + 255) / 256, 256, 0, st>>>(n_samples, ch, part, out);
  PK(cudaGetLastError());
  if (!ptrs_are_device) {
    PK(cudaMemcpyAsync(chosen, out, 4 * ns, cudaMemcpyDeviceToHost, st));
    PK(cudaStreamSynchronize(st));
  }
  return VINE_OK;
}

}  // extern "C"
