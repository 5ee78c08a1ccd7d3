// Learned block-norm predictor for step C (not in the paper): features of a
// (chi tile, K slab) task, the task's actual contribution norm (logging),
// a 2-hidden-layer ReLU network with bf16 weights and FP32 accumulation
// (forward, backward, Adam), and the compaction of task lists by prediction.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "k_mlp.h"

namespace gw {
namespace mlp {

constexpr int H = kMlpHidden;
constexpr int F = kMlpFeatures;

// parameter offsets in the flat vector: W1 [H][F], b1 [H], W2 [H][H], b2 [H], w3 [H], b3
constexpr int oW1 = 0, oB1 = H * F, oW2 = oB1 + H, oB2 = oW2 + H * H, oW3 = oB2 + H, oB3 = oW3 + H;

// ---------------------------------------------------------------------------
// features and targets
// ---------------------------------------------------------------------------
// norm of the X part of (slab, row tile) and of the Y part of (slab, col tile)
// from the kept blocks' squared norms
// (mu-atom chunk [mc0, mc0 + nmc) with AOs [mu0, mu0 + nmu); slab c covers
// chunk-local AOs [c naop_chunk, (c + 1) naop_chunk); block flags and norms
// are [sigma-atom][mu-atom of the chunk][RI atom from pa0])
__global__ void k_slab_tile_norms(const float* __restrict__ norm2, const unsigned char* __restrict__ flag,
                                  int nmc, int mc0, int npa, int pa0, int per, int naop_chunk,
                                  const int* __restrict__ atom_of_ao, const int* __restrict__ atom_of_ri,
                                  int mu0, int nmu, int row0, int rows, int ntile, int tile, int nslab,
                                  float* __restrict__ out) {
  const long long i = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (i >= static_cast<long long>(nslab) * ntile) return;
  const int t = static_cast<int>(i % ntile), slab = static_cast<int>(i / ntile);
  const int sl = slab / per, c = slab % per;
  const int a_lo = c * naop_chunk, a_hi = min(nmu, (c + 1) * naop_chunk) - 1;
  float s = 0.f;
  if (a_lo < nmu) {
    const int m0 = atom_of_ao[mu0 + a_lo], m1 = atom_of_ao[mu0 + a_hi];
    const int r_lo = row0 + t * tile, r_hi = min(row0 + rows, row0 + (t + 1) * tile) - 1;
    const int p0 = atom_of_ri[r_lo], p1 = atom_of_ri[r_hi];
    for (int m = m0; m <= m1; ++m)
      for (int p = p0; p <= p1; ++p) {
        const long long b = (static_cast<long long>(sl) * nmc + (m - mc0)) * npa + (p - pa0);
        if (flag[b]) s += norm2[b];
      }
  }
  out[i] = sqrtf(s);
}

__global__ void k_task_features(const int* __restrict__ tasks, const int* __restrict__ counts,
                                int nslab, int npt, int nqt, int per, int s0,
                                const float* __restrict__ xn, const float* __restrict__ yn,
                                const float* __restrict__ cent_p, const float* __restrict__ cent_q,
                                const float* __restrict__ cent_c, const float* __restrict__ xyz,
                                const int* __restrict__ n_ao, float log_tau,
                                float* __restrict__ feat) {
  const int t = blockIdx.x;
  const int cnt = counts[t];
  const int pt = t / nqt, qt = t % nqt;
  for (int i = threadIdx.x; i < cnt; i += blockDim.x) {
    const int slab = tasks[static_cast<long long>(t) * nslab + i];
    const int sl = slab / per, c = slab % per, s = s0 + sl;
    const float a = xn[static_cast<long long>(slab) * npt + pt];
    const float b = yn[static_cast<long long>(slab) * nqt + qt];
    const float la = log10f(fmaxf(a, 1e-30f)), lb = log10f(fmaxf(b, 1e-30f));
    auto dist = [](const float* u, const float* v) {
      const float dx = u[0] - v[0], dy = u[1] - v[1], dz = u[2] - v[2];
      return sqrtf(dx * dx + dy * dy + dz * dz);
    };
    float* f = feat + (static_cast<long long>(t) * nslab + i) * F;
    f[0] = la;
    f[1] = lb;
    f[2] = log_tau;
    f[3] = dist(xyz + 3 * s, cent_p + 3 * pt) * 0.1f;
    f[4] = dist(cent_c + 3 * c, cent_q + 3 * qt) * 0.1f;
    f[5] = dist(cent_p + 3 * pt, cent_q + 3 * qt) * 0.1f;
    f[6] = n_ao[s] / 13.0f;
    f[7] = la + lb;
  }
}

// log10 of the Frobenius norm of one task's contribution
//   sum_{k in slab} X[p][k] Y[q][k]  over the tile's rows p and columns q,
// operands rebuilt from their 16-bit slices (bf16, or binary16 holding the
// operand times a power of two: xinv / yinv undo it); one CTA (256 threads)
// per task.
__device__ __forceinline__ float slice_value(uint16_t b, int f16) {
  return f16 ? __half2float(__ushort_as_half(b)) : __bfloat162float(__ushort_as_bfloat16(b));
}
__global__ void k_task_norms(const uint16_t* __restrict__ xs, const uint16_t* __restrict__ ys,
                             int slices, int f16, float xinv, float yinv, long long xslice,
                             long long yslice, long long ldk,
                             int prow, int nri, const int* __restrict__ tasks,
                             const int* __restrict__ counts, int nslab, int nqt, int tile,
                             const long long* __restrict__ slab_k0, const int* __restrict__ slab_len,
                             float* __restrict__ target) {
  const int t = blockIdx.x;
  const int i = blockIdx.y;
  if (i >= counts[t]) return;
  const int pt = t / nqt, qt = t % nqt;
  const int slab = tasks[static_cast<long long>(t) * nslab + i];
  const long long k0 = slab_k0[slab];
  const int len = slab_len[slab];
  __shared__ float As[32][129];
  __shared__ float Bs[32][129];
  __shared__ float red[256];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;  // 16 x 16, 8 x 8 outputs each
  float acc[8][8] = {};
  for (int kk = 0; kk < len; kk += 32) {
    for (int e = tid; e < 32 * 128; e += 256) {
      const int r = e >> 5, k = e & 31;
      const int p = pt * tile + r, q = qt * tile + r;
      float va = 0.f, vb = 0.f;
      if (p < prow && kk + k < len)
        for (int s = 0; s < slices; ++s)
          va += xinv * slice_value(xs[s * xslice + static_cast<long long>(p) * ldk + k0 + kk + k], f16);
      if (q < nri && kk + k < len)
        for (int s = 0; s < slices; ++s)
          vb += yinv * slice_value(ys[s * yslice + static_cast<long long>(q) * ldk + k0 + kk + k], f16);
      As[k][r] = va;
      Bs[k][r] = vb;
    }
    __syncthreads();
    for (int k = 0; k < 32; ++k) {
      float a[8], b[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) a[u] = As[k][ty + 16 * u];
#pragma unroll
      for (int u = 0; u < 8; ++u) b[u] = Bs[k][tx + 16 * u];
#pragma unroll
      for (int u = 0; u < 8; ++u)
#pragma unroll
        for (int v = 0; v < 8; ++v) acc[u][v] = fmaf(a[u], b[v], acc[u][v]);
    }
    __syncthreads();
  }
  float s = 0.f;
#pragma unroll
  for (int u = 0; u < 8; ++u)
#pragma unroll
    for (int v = 0; v < 8; ++v) s += acc[u][v] * acc[u][v];
  red[tid] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) red[tid] += red[tid + o];
    __syncthreads();
  }
  if (tid == 0)
    target[static_cast<long long>(t) * nslab + i] = red[0] > 0.f ? 0.5f * log10f(red[0]) : -40.f;
}

// ---------------------------------------------------------------------------
// network
// ---------------------------------------------------------------------------
__device__ __forceinline__ float relu(float x) { return x > 0.f ? x : 0.f; }

// One thread per sample: z1, z2 (pre-activations) and y; weights (bf16) in smem.
// Samples may be strided with a validity test: sample s is valid iff
// valid == nullptr or (s % stride) < valid[s / stride].
__global__ void k_forward(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ x,
                          long long n, const int* __restrict__ valid, int stride,
                          float* __restrict__ z1, float* __restrict__ z2, float* __restrict__ y) {
  __shared__ float w[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  __syncthreads();
  const long long s = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  if (valid && (s % stride) >= valid[s / stride]) return;
  float in[F];
#pragma unroll
  for (int f = 0; f < F; ++f) in[f] = x[s * F + f];
  float h1[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    float a = w[oB1 + i];
#pragma unroll
    for (int f = 0; f < F; ++f) a = fmaf(w[oW1 + i * F + f], in[f], a);
    if (z1) z1[s * H + i] = a;
    h1[i] = relu(a);
  }
  float out = w[oB3] + in[kMlpBound];  // residual on the log norm-product bound
  for (int i = 0; i < H; ++i) {
    float a = w[oB2 + i];
#pragma unroll
    for (int j = 0; j < H; ++j) a = fmaf(w[oW2 + i * H + j], h1[j], a);
    if (z2) z2[s * H + i] = a;
    out = fmaf(w[oW3 + i], relu(a), out);
  }
  y[s] = out;
}

// per-sample output and hidden-layer gradients of L = mean (y - t)^2
__global__ void k_backward_samples(const __nv_bfloat16* __restrict__ wb, const float* __restrict__ z1,
                                   const float* __restrict__ z2, const float* __restrict__ y,
                                   const float* __restrict__ t, long long n, float* __restrict__ dy,
                                   float* __restrict__ dz1, float* __restrict__ dz2) {
  __shared__ float w[kMlpParams];
  for (int i = threadIdx.x; i < kMlpParams; i += blockDim.x) w[i] = __bfloat162float(wb[i]);
  __syncthreads();
  const long long s = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float g = 2.f * (y[s] - t[s]) / static_cast<float>(n);
  dy[s] = g;
  float d2[H];
#pragma unroll
  for (int i = 0; i < H; ++i) {
    d2[i] = z2[s * H + i] > 0.f ? g * w[oW3 + i] : 0.f;
    dz2[s * H + i] = d2[i];
  }
  for (int j = 0; j < H; ++j) {
    float a = 0.f;
#pragma unroll
    for (int i = 0; i < H; ++i) a = fmaf(d2[i], w[oW2 + i * H + j], a);
    dz1[s * H + j] = z1[s * H + j] > 0.f ? a : 0.f;
  }
}

// one thread per parameter: the sum over samples in sample order
__global__ void k_param_grads(const float* __restrict__ x, const float* __restrict__ z1,
                              const float* __restrict__ z2, const float* __restrict__ dy,
                              const float* __restrict__ dz1, const float* __restrict__ dz2, long long n,
                              float* __restrict__ grad) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  float a = 0.f;
  if (p < oB1) {
    const int i = p / F, f = p % F;
    for (long long s = 0; s < n; ++s) a = fmaf(dz1[s * H + i], x[s * F + f], a);
  } else if (p < oW2) {
    const int i = p - oB1;
    for (long long s = 0; s < n; ++s) a += dz1[s * H + i];
  } else if (p < oB2) {
    const int i = (p - oW2) / H, j = (p - oW2) % H;
    for (long long s = 0; s < n; ++s) a = fmaf(dz2[s * H + i], relu(z1[s * H + j]), a);
  } else if (p < oW3) {
    const int i = p - oB2;
    for (long long s = 0; s < n; ++s) a += dz2[s * H + i];
  } else if (p < oB3) {
    const int i = p - oW3;
    for (long long s = 0; s < n; ++s) a = fmaf(dy[s], relu(z2[s * H + i]), a);
  } else {
    for (long long s = 0; s < n; ++s) a += dy[s];
  }
  grad[p] = a;
}

__global__ void k_adam(float* __restrict__ theta, const float* __restrict__ grad, float* __restrict__ m,
                       float* __restrict__ v, int step, float lr, __nv_bfloat16* __restrict__ wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= kMlpParams) return;
  const float b1 = 0.9f, b2 = 0.999f;
  const float g = grad[p];
  const float mm = b1 * m[p] + (1.f - b1) * g;
  const float vv = b2 * v[p] + (1.f - b2) * g * g;
  m[p] = mm;
  v[p] = vv;
  const float mh = mm / (1.f - powf(b1, static_cast<float>(step)));
  const float vh = vv / (1.f - powf(b2, static_cast<float>(step)));
  const float th = theta[p] - lr * mh / (sqrtf(vh) + 1e-8f);
  theta[p] = th;
  wb[p] = __float2bfloat16_rn(th);
}

__global__ void k_round(const float* __restrict__ theta, __nv_bfloat16* __restrict__ wb) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < kMlpParams) wb[p] = __float2bfloat16_rn(theta[p]);
}

// per tile: keep task i iff pred + margin >= log_thr (order kept); rewrites
// the list, its count and its K total; skipped[t] = tasks dropped
__global__ void k_compact(int* __restrict__ tasks, int* __restrict__ counts, long long* __restrict__ kacc,
                          int nslab, const float* __restrict__ pred, const float* __restrict__ feat,
                          float margin, float log_thr, const int* __restrict__ slab_len,
                          int* __restrict__ skipped) {
  const int t = blockIdx.x;
  if (threadIdx.x >= 32) return;
  const int lane = threadIdx.x;
  const int cnt = counts[t];
  int* list = tasks + static_cast<long long>(t) * nslab;
  const float* pr = pred + static_cast<long long>(t) * nslab;
  // scale of the tile: the largest log10 norm-product bound of its tasks
  float lb = -1e30f;
  for (int i = lane; i < cnt; i += 32)
    lb = fmaxf(lb, feat[(static_cast<long long>(t) * nslab + i) * F + 7]);
  for (int o = 16; o > 0; o >>= 1) lb = fmaxf(lb, __shfl_xor_sync(0xffffffffu, lb, o));
  // skip below thr * min(1, bound scale of the tile)
  const float cut = log_thr + fminf(0.f, lb);
  int out = 0;
  long long ksum = 0;
  for (int base = 0; base < cnt; base += 32) {
    const int i = base + lane;
    const bool in = i < cnt;
    const int s = in ? list[i] : 0;
    const bool keep = in && (pr[i] + margin >= cut);
    const unsigned mk = __ballot_sync(0xffffffffu, keep);
    __syncwarp();
    if (keep) {
      list[out + __popc(mk & ((1u << lane) - 1))] = s;
      ksum += slab_len[s];
    }
    out += __popc(mk);
    __syncwarp();
  }
  for (int o = 16; o > 0; o >>= 1) ksum += __shfl_xor_sync(0xffffffffu, ksum, o);
  if (lane == 0) {
    skipped[t] = cnt - out;
    counts[t] = out;
    kacc[t] = ksum;
  }
}

}  // namespace mlp

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
void mlp_slab_tile_norms(const float* norm2, const unsigned char* flag, int nmc, int mc0, int npa, int pa0,
                         int per, int naop_chunk, const int* atom_of_ao, const int* atom_of_ri, int mu0,
                         int nmu, int row0, int rows, int ntile, int tile, int nslab, float* out,
                         cudaStream_t st) {
  const long long n = static_cast<long long>(nslab) * ntile;
  if (n == 0) return;
  mlp::k_slab_tile_norms<<<static_cast<unsigned>((n + 255) / 256), 256, 0, st>>>(
      norm2, flag, nmc, mc0, npa, pa0, per, naop_chunk, atom_of_ao, atom_of_ri, mu0, nmu, row0, rows,
      ntile, tile, nslab, out);
}

void mlp_task_features(const int* tasks, const int* counts, int nslab, int npt, int nqt, int per, int s0,
                       const float* xn, const float* yn, const float* cent_p, const float* cent_q,
                       const float* cent_c, const float* xyz, const int* n_ao, float log_tau,
                       float* feat, cudaStream_t st) {
  mlp::k_task_features<<<npt * nqt, 128, 0, st>>>(tasks, counts, nslab, npt, nqt, per, s0, xn, yn,
                                                  cent_p, cent_q, cent_c, xyz, n_ao, log_tau, feat);
}

void mlp_task_norms(const void* xs, const void* ys, int slices, int f16, float xinv, float yinv,
                    long long xslice, long long yslice, long long ldk, int prow, int nri, const int* tasks,
                    const int* counts, int nslab, int npt, int nqt, int max_count, int tile,
                    const long long* slab_k0, const int* slab_len, float* target, cudaStream_t st) {
  if (max_count == 0) return;
  dim3 g(npt * nqt, max_count);
  mlp::k_task_norms<<<g, 256, 0, st>>>(static_cast<const uint16_t*>(xs),
                                       static_cast<const uint16_t*>(ys), slices, f16, xinv, yinv,
                                       xslice, yslice,
                                       ldk, prow, nri, tasks, counts, nslab, nqt, tile, slab_k0, slab_len,
                                       target);
}

void mlp_forward(const void* wb, const float* x, long long n, const int* valid, int stride, float* z1,
                 float* z2, float* y, cudaStream_t st) {
  if (n == 0) return;
  mlp::k_forward<<<static_cast<unsigned>((n + 127) / 128), 128, 0, st>>>(
      static_cast<const __nv_bfloat16*>(wb), x, n, valid, stride, z1, z2, y);
}

void mlp_backward(const void* wb, const float* x, const float* z1, const float* z2, const float* y,
                  const float* t, long long n, float* dy, float* dz1, float* dz2, float* grad,
                  cudaStream_t st) {
  if (n == 0) return;
  mlp::k_backward_samples<<<static_cast<unsigned>((n + 127) / 128), 128, 0, st>>>(
      static_cast<const __nv_bfloat16*>(wb), z1, z2, y, t, n, dy, dz1, dz2);
  mlp::k_param_grads<<<(kMlpParams + 127) / 128, 128, 0, st>>>(x, z1, z2, dy, dz1, dz2, n, grad);
}

void mlp_adam(float* theta, const float* grad, float* m, float* v, int step, float lr, void* wb,
              cudaStream_t st) {
  mlp::k_adam<<<(kMlpParams + 127) / 128, 128, 0, st>>>(theta, grad, m, v, step, lr,
                                                        static_cast<__nv_bfloat16*>(wb));
}

void mlp_round(const float* theta, void* wb, cudaStream_t st) {
  mlp::k_round<<<(kMlpParams + 127) / 128, 128, 0, st>>>(theta, static_cast<__nv_bfloat16*>(wb));
}

void mlp_compact(int* tasks, int* counts, long long* kacc, int ntiles, int nslab, const float* pred,
                 const float* feat, float margin, float log_thr, const int* slab_len, int* skipped,
                 cudaStream_t st) {
  mlp::k_compact<<<ntiles, 32, 0, st>>>(tasks, counts, kacc, nslab, pred, feat, margin, log_thr,
                                        slab_len, skipped);
}

}  // namespace gw
