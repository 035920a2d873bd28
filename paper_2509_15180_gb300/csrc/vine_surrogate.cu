// vine_surrogate.cu -- the sPAM neural surrogate of Sec. 4.3 behind
// vine_spam_samples, vine_surrogate_train and vine_surrogate_eval
// (include/vine.h): a 2-32-2 network with ReLU hidden units from (actuator
// strain, cell length) to (m, phi_Rc), trained by mean squared error on
// normalised outputs with full-batch Adam.
//
// Training step, deterministic: one thread per sample computes the forward
// pass and the 162 gradient components of its sample; warps sum them with
// shuffles into a per-warp shared-memory row, the rows are summed in warp
// order into one partial per CTA, and a single CTA sums the partials in CTA
// order (FP64) and applies Adam (one thread per parameter).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>

#include "vine.h"
#include "vine_internal.cuh"

using namespace vine;

namespace {

constexpr int kH = 32;
constexpr int kP = kH * 2 + kH + 2 * kH + 2;  // 162
constexpr int kTrainThreads = 256;

vine_status sgfail(vine_status s, const char* msg) {
  set_last_error(msg);
  return s;
}

vine_status sgcuda(cudaError_t e, const char* where) {
  char b[384];
  std::snprintf(b, sizeof(b), "%s: %s", where, cudaGetErrorString(e));
  set_last_error(b);
  return e == cudaErrorMemoryAllocation ? VINE_ENOMEM : VINE_ECUDA;
}

#define SK(call)                                      \
  do {                                                \
    cudaError_t e_ = (call);                          \
    if (e_ != cudaSuccess) return sgcuda(e_, #call);  \
  } while (0)

struct Norm {
  float in_lo[2], in_scale[2], out_scale[2];
};

// inputs [n][2] raw (strain, cell length), targets [n][2] raw (m, phi) ->
// normalised float pairs
__global__ void normalise_kernel(int n, const double* in, const double* tg, Norm nm, float2* x, float2* t) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  x[i] = make_float2(((float)in[2 * i] - nm.in_lo[0]) * nm.in_scale[0],
                     ((float)in[2 * i + 1] - nm.in_lo[1]) * nm.in_scale[1]);
  if (tg) t[i] = make_float2((float)tg[2 * i] * nm.out_scale[0], (float)tg[2 * i + 1] * nm.out_scale[1]);
}

// Parameter layout: W1[32][2], b1[32], W2[2][32], b2[2].
__device__ __forceinline__ void net_forward(const float* th, float x0, float x1, float* a, float& y0, float& y1) {
  y0 = th[5 * kH];
  y1 = th[5 * kH + 1];
#pragma unroll
  for (int j = 0; j < kH; ++j) {
    const float aj = th[2 * kH + j] + th[2 * j] * x0 + th[2 * j + 1] * x1;
    a[j] = aj;
    const float hj = fmaxf(aj, 0.f);
    y0 += th[3 * kH + j] * hj;
    y1 += th[4 * kH + j] * hj;
  }
}

__global__ void __launch_bounds__(kTrainThreads) grad_partial_kernel(int n, const float2* x, const float2* t,
                                                                     const float* theta, float* partial) {
  __shared__ float th[kP];
  __shared__ float rows[kTrainThreads / 32][kP];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int k = threadIdx.x; k < kP; k += blockDim.x) th[k] = theta[k];
  for (int k = lane; k < kP; k += 32) rows[warp][k] = 0.f;
  __syncthreads();
  const float inv_n = 1.f / (float)n;
  for (int base = blockIdx.x * blockDim.x; base < n; base += gridDim.x * blockDim.x) {
    const int i = base + threadIdx.x;
    const bool live = i < n;
    float a[kH];
    float y0, y1, x0 = 0.f, x1 = 0.f, r0 = 0.f, r1 = 0.f;
    if (live) {
      x0 = x[i].x;
      x1 = x[i].y;
      net_forward(th, x0, x1, a, y0, y1);
      r0 = (y0 - t[i].x) * inv_n;  // dL/dy
      r1 = (y1 - t[i].y) * inv_n;
    } else {
#pragma unroll
      for (int j = 0; j < kH; ++j) a[j] = 0.f;
    }
    // gradient of this sample, summed over the warp component by component
#pragma unroll
    for (int j = 0; j < kH; ++j) {
      const float hj = fmaxf(a[j], 0.f);
      const float dj = (a[j] > 0.f) ? (r0 * th[3 * kH + j] + r1 * th[4 * kH + j]) : 0.f;
      float g[5] = {dj * x0, dj * x1, dj, r0 * hj, r1 * hj};
#pragma unroll
      for (int q = 0; q < 5; ++q)
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) g[q] += __shfl_xor_sync(0xffffffffu, g[q], d);
      if (lane == 0) {
        rows[warp][2 * j] += g[0];
        rows[warp][2 * j + 1] += g[1];
        rows[warp][2 * kH + j] += g[2];
        rows[warp][3 * kH + j] += g[3];
        rows[warp][4 * kH + j] += g[4];
      }
    }
    float gb[2] = {r0, r1};
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
      for (int d = 16; d > 0; d >>= 1) gb[q] += __shfl_xor_sync(0xffffffffu, gb[q], d);
    if (lane == 0) {
      rows[warp][5 * kH] += gb[0];
      rows[warp][5 * kH + 1] += gb[1];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < kP; k += blockDim.x) {
    float s = 0.f;
    for (int w = 0; w < kTrainThreads / 32; ++w) s += rows[w][k];
    partial[(size_t)blockIdx.x * kP + k] = s;
  }
}

// Sum of the CTA partials in CTA order (FP64) and one Adam step, one thread
// per parameter.
__global__ void adam_kernel(int n_part, const float* partial, float* theta, float* m, float* v, int step, float lr) {
  const int k = threadIdx.x;
  if (k >= kP) return;
  double g = 0.0;
  for (int b = 0; b < n_part; ++b) g += (double)partial[(size_t)b * kP + k];
  const float gf = (float)g;
  const float b1 = 0.9f, b2 = 0.999f;
  m[k] = b1 * m[k] + (1.f - b1) * gf;
  v[k] = b2 * v[k] + (1.f - b2) * gf * gf;
  const float mh = m[k] / (1.f - powf(b1, (float)step));
  const float vh = v[k] / (1.f - powf(b2, (float)step));
  theta[k] -= lr * mh / (sqrtf(vh) + 1e-8f);
}

// Loss of the current parameters (for the caller's history), FP64 sum in
// CTA order of per-CTA sums.
__global__ void __launch_bounds__(kTrainThreads) loss_partial_kernel(int n, const float2* x, const float2* t,
                                                                     const float* theta, double* partial) {
  __shared__ float th[kP];
  __shared__ double ws[kTrainThreads / 32];
  for (int k = threadIdx.x; k < kP; k += blockDim.x) th[k] = theta[k];
  __syncthreads();
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float a[kH], y0, y1;
    net_forward(th, x[i].x, x[i].y, a, y0, y1);
    const float r0 = y0 - t[i].x, r1 = y1 - t[i].y;
    acc += (double)(r0 * r0 + r1 * r1);
  }
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, d);
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kTrainThreads / 32; ++w) s += ws[w];
    partial[blockIdx.x] = s;
  }
}

__global__ void loss_final_kernel(int n_part, int n, const double* partial, float* out) {
  double s = 0.0;
  for (int b = 0; b < n_part; ++b) s += partial[b];
  *out = (float)(0.5 * s / (double)n);
}

__global__ void eval_kernel(int n, const double* in, const float* theta, Norm nm, double* out) {
  __shared__ float th[kP];
  for (int k = threadIdx.x; k < kP; k += blockDim.x) th[k] = theta[k];
  __syncthreads();
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x0 = ((float)in[2 * i] - nm.in_lo[0]) * nm.in_scale[0];
  const float x1 = ((float)in[2 * i + 1] - nm.in_lo[1]) * nm.in_scale[1];
  float a[kH], y0, y1;
  net_forward(th, x0, x1, a, y0, y1);
  out[2 * i] = (double)(y0 / nm.out_scale[0]);
  out[2 * i + 1] = (double)(y1 / nm.out_scale[1]);
}

size_t up256(size_t x) { return (x + 255) & ~size_t(255); }

bool norm_ok(const vine_surrogate* s) {
  for (int i = 0; i < 2; ++i)
    if (!(std::isfinite(s->in_lo[i]) && std::isfinite(s->in_scale[i]) && s->in_scale[i] != 0.f &&
          std::isfinite(s->out_scale[i]) && s->out_scale[i] != 0.f))
      return false;
  for (int k = 0; k < kP; ++k)
    if (!std::isfinite(s->theta[k])) return false;
  return true;
}

Norm norm_of(const vine_surrogate* s) {
  Norm nm;
  for (int i = 0; i < 2; ++i) {
    nm.in_lo[i] = s->in_lo[i];
    nm.in_scale[i] = s->in_scale[i];
    nm.out_scale[i] = s->out_scale[i];
  }
  return nm;
}

struct StreamFree {
  void* p;
  cudaStream_t s;
  ~StreamFree() {
    if (p) cudaFreeAsync(p, s);
  }
};

}  // namespace

extern "C" {

vine_status vine_spam_samples(const double* m, const double* l0, int32_t n, const vine_params* params, double* eps,
                              double* phi, double* f, int32_t* saturated, void* stream_v) {
  if (n < 0 || (n > 0 && (!m || !l0 || !eps || !phi || !f || !saturated)))
    return sgfail(VINE_EINVAL, "vine_spam_samples: null argument or negative count");
  if (n == 0) return VINE_OK;
  for (int i = 0; i < n; ++i)
    if (!(std::isfinite(m[i]) && m[i] > 0.0 && m[i] <= 0.5 && std::isfinite(l0[i]) && l0[i] > 0.0))
      return sgfail(VINE_EINVAL, "vine_spam_samples: m must lie in (0, 0.5] and l0 be positive");
  vine_params prm;
  if (params) prm = *params; else vine_params_default(&prm);
  cudaStream_t st = (cudaStream_t)stream_v;
  const size_t nn = (size_t)n;
  const size_t o_m = 0, o_l = up256(8 * nn), o_e = o_l + up256(8 * nn), o_p = o_e + up256(8 * nn),
               o_f = o_p + up256(8 * nn), o_s = o_f + up256(8 * nn), total = o_s + up256(4 * nn);
  char* mem = nullptr;
  SK(cudaMallocAsync((void**)&mem, total, st));
  StreamFree fr{mem, st};
  SK(cudaMemcpyAsync(mem + o_m, m, 8 * nn, cudaMemcpyHostToDevice, st));
  SK(cudaMemcpyAsync(mem + o_l, l0, 8 * nn, cudaMemcpyHostToDevice, st));
  GaussLegendre gl;
  gauss_legendre(24, &gl);
  SK(launch_spam_samples(n, (const double*)(mem + o_m), (const double*)(mem + o_l), prm.R_c, prm.R_act, prm.a_spam,
                         gl, (double*)(mem + o_e), (double*)(mem + o_p), (double*)(mem + o_f), (int*)(mem + o_s), st));
  SK(cudaMemcpyAsync(eps, mem + o_e, 8 * nn, cudaMemcpyDeviceToHost, st));
  SK(cudaMemcpyAsync(phi, mem + o_p, 8 * nn, cudaMemcpyDeviceToHost, st));
  SK(cudaMemcpyAsync(f, mem + o_f, 8 * nn, cudaMemcpyDeviceToHost, st));
  SK(cudaMemcpyAsync(saturated, mem + o_s, 4 * nn, cudaMemcpyDeviceToHost, st));
  SK(cudaStreamSynchronize(st));
  return VINE_OK;
}

vine_status vine_surrogate_train(vine_surrogate* net, const double* inputs, const double* targets, int32_t n,
                                 int32_t steps, float lr, float* loss_history, void* stream_v) {
  if (!net || n < 1 || steps < 0 || !inputs || !targets || !(std::isfinite(lr) && lr > 0.f))
    return sgfail(VINE_EINVAL, "vine_surrogate_train: invalid argument");
  if (!norm_ok(net)) return sgfail(VINE_EINVAL, "vine_surrogate_train: non-finite parameters or zero scales");
  cudaStream_t st = (cudaStream_t)stream_v;
  const size_t nn = (size_t)n;
  int nsm = 1, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = (int)std::max<size_t>(1, std::min<size_t>((nn + kTrainThreads - 1) / kTrainThreads,
                                                               (size_t)2 * nsm));
  const size_t o_in = 0, o_tg = up256(16 * nn), o_x = o_tg + up256(16 * nn), o_t = o_x + up256(8 * nn),
               o_th = o_t + up256(8 * nn), o_m = o_th + up256(4 * kP), o_v = o_m + up256(4 * kP),
               o_part = o_v + up256(4 * kP), o_lp = o_part + up256(4 * (size_t)kP * blocks),
               o_loss = o_lp + up256(8 * (size_t)blocks), total = o_loss + up256(4 * (size_t)std::max(steps, 1));
  char* mem = nullptr;
  SK(cudaMallocAsync((void**)&mem, total, st));
  StreamFree fr{mem, st};
  SK(cudaMemcpyAsync(mem + o_in, inputs, 16 * nn, cudaMemcpyHostToDevice, st));
  SK(cudaMemcpyAsync(mem + o_tg, targets, 16 * nn, cudaMemcpyHostToDevice, st));
  SK(cudaMemcpyAsync(mem + o_th, net->theta, 4 * kP, cudaMemcpyHostToDevice, st));
  SK(cudaMemsetAsync(mem + o_m, 0, up256(4 * kP) * 2, st));
  const Norm nm = norm_of(net);
  float2* x = (float2*)(mem + o_x);
  float2* t = (float2*)(mem + o_t);
  normalise_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, (const double*)(mem + o_in), (const double*)(mem + o_tg), nm,
                                                    x, t);
  SK(cudaGetLastError());
  float* th = (float*)(mem + o_th);
  float* part = (float*)(mem + o_part);
  for (int s = 1; s <= steps; ++s) {
    if (loss_history) {
      loss_partial_kernel<<<blocks, kTrainThreads, 0, st>>>(n, x, t, th, (double*)(mem + o_lp));
      loss_final_kernel<<<1, 1, 0, st>>>(blocks, n, (const double*)(mem + o_lp), (float*)(mem + o_loss) + (s - 1));
    }
    grad_partial_kernel<<<blocks, kTrainThreads, 0, st>>>(n, x, t, th, part);
    adam_kernel<<<1, 192, 0, st>>>(blocks, part, th, (float*)(mem + o_m), (float*)(mem + o_v), s, lr);
  }
  SK(cudaGetLastError());
  SK(cudaMemcpyAsync(net->theta, th, 4 * kP, cudaMemcpyDeviceToHost, st));
  if (loss_history && steps > 0)
    SK(cudaMemcpyAsync(loss_history, mem + o_loss, 4 * (size_t)steps, cudaMemcpyDeviceToHost, st));
  SK(cudaStreamSynchronize(st));
  return VINE_OK;
}

vine_status vine_surrogate_eval(const vine_surrogate* net, const double* inputs, int32_t n, double* outputs,
                                int32_t ptrs_are_device, void* stream_v) {
  if (!net || n < 0 || (n > 0 && (!inputs || !outputs))) return sgfail(VINE_EINVAL, "vine_surrogate_eval: null argument");
  if (!norm_ok(net)) return sgfail(VINE_EINVAL, "vine_surrogate_eval: non-finite parameters or zero scales");
  if (n == 0) return VINE_OK;
  cudaStream_t st = (cudaStream_t)stream_v;
  const size_t nn = (size_t)n;
  const size_t o_th = 0, o_in = up256(4 * kP), o_out = o_in + (ptrs_are_device ? 0 : up256(16 * nn)),
               total = o_out + (ptrs_are_device ? 0 : up256(16 * nn));
  char* mem = nullptr;
  SK(cudaMallocAsync((void**)&mem, total, st));
  StreamFree fr{mem, st};
  SK(cudaMemcpyAsync(mem + o_th, net->theta, 4 * kP, cudaMemcpyHostToDevice, st));
  const double* in = inputs;
  double* out = outputs;
  if (!ptrs_are_device) {
    SK(cudaMemcpyAsync(mem + o_in, inputs, 16 * nn, cudaMemcpyHostToDevice, st));
    in = (const double*)(mem + o_in);
    out = (double*)(mem + o_out);
  }
  eval_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, in, (const float*)(mem + o_th), norm_of(net), out);
  SK(cudaGetLastError());
  if (!ptrs_are_device) {
    SK(cudaMemcpyAsync(outputs, out, 16 * nn, cudaMemcpyDeviceToHost, st));
    SK(cudaStreamSynchronize(st));
  }
  return VINE_OK;
}

}  // extern "C"
