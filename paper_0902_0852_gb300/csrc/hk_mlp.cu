// Precision-predictor network: 2 -> 64 -> 64 -> 3 multilayer perceptron with
// exact GELU, float32, forward, back-propagation and Adam on the device.
//
// One CTA owns a tile of MT = 64 samples and keeps the whole network in shared
// memory (4547 floats) together with the tile's activations H = gelu(Z) and
// slopes G = gelu'(Z) of both hidden layers.  The backward pass overwrites the
// slopes with dZ = dH * G in place.  Each CTA writes the gradient summed over
// its own samples to a per-tile slot of the work area; k_mlp_reduce then adds
// the slots in tile order, so gradients and losses do not depend on
// scheduling.  The hidden-layer products are 64 x 64 per sample: the whole
// network costs a few microseconds per step at B = 4096, far below any
// roofline that would reward tensor cores, so plain FP32 FMAs are used.
#include "hk.h"
#include "hk_internal.h"

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace {

constexpr int HID = 64, NIN = 2, NOUT = 3;
constexpr int MT = 64;        // samples per CTA tile
constexpr int NTH = 256;      // threads per CTA
constexpr int W2S = HID + 1;  // padded row stride of W2 in shared memory
constexpr int OFF_W1 = 0, OFF_B1 = OFF_W1 + HID * NIN, OFF_W2 = OFF_B1 + HID, OFF_B2 = OFF_W2 + HID * HID,
              OFF_W3 = OFF_B2 + HID, OFF_B3 = OFF_W3 + NOUT * HID, NPARAM = OFF_B3 + NOUT;
static_assert(NPARAM == HK_MLP_NPARAMS, "parameter layout");
static_assert(NTH == HID + NOUT * HID, "one thread per dW3 entry beside the 64 bias threads");

// shared-memory carve (floats)
constexpr int S_W1 = 0, S_B1 = S_W1 + HID * NIN, S_W2 = S_B1 + HID, S_B2 = S_W2 + HID * W2S, S_W3 = S_B2 + HID,
              S_B3 = S_W3 + NOUT * HID, S_X = S_B3 + 4, S_T = S_X + MT * NIN, S_DY = S_T + MT * NOUT,
              S_H1 = S_DY + MT * NOUT, S_G1 = S_H1 + MT * HID, S_H2 = S_G1 + MT * HID, S_G2 = S_H2 + MT * HID,
              S_RED = S_G2 + MT * HID, S_TOTAL = S_RED + NTH / 32;
constexpr size_t SMEM_BYTES = sizeof(float) * S_TOTAL;

__device__ __forceinline__ float phi_cdf(float z) { return 0.5f * (1.0f + erff(z * 0.70710678118654752f)); }
__device__ __forceinline__ float gelu(float z) { return z * phi_cdf(z); }
__device__ __forceinline__ float gelu_slope(float z) {
  return phi_cdf(z) + z * 0.39894228040143268f * expf(-0.5f * z * z);
}

// TRAIN = false: write y.  TRAIN = true: per-tile gradient and loss sums.
template <bool TRAIN>
__global__ void __launch_bounds__(NTH) k_mlp_tile(const float *__restrict__ prm, const float *__restrict__ x,
                                                  const float *__restrict__ tgt, const float *__restrict__ wout, int B,
                                                  float *__restrict__ y, float *__restrict__ part) {
  extern __shared__ float sm[];
  const int tid = threadIdx.x;
  const int b0 = blockIdx.x * MT;
  const int nb = min(MT, B - b0);
  float *W1 = sm + S_W1, *B1 = sm + S_B1, *W2 = sm + S_W2, *B2 = sm + S_B2, *W3 = sm + S_W3, *B3 = sm + S_B3;
  float *X = sm + S_X, *T = sm + S_T, *DY = sm + S_DY;
  float *H1 = sm + S_H1, *G1 = sm + S_G1, *H2 = sm + S_H2, *G2 = sm + S_G2, *RED = sm + S_RED;

  for (int k = tid; k < HID * NIN; k += NTH) W1[k] = prm[OFF_W1 + k];
  for (int k = tid; k < HID; k += NTH) {
    B1[k] = prm[OFF_B1 + k];
    B2[k] = prm[OFF_B2 + k];
  }
  for (int k = tid; k < HID * HID; k += NTH) W2[(k / HID) * W2S + (k % HID)] = prm[OFF_W2 + k];
  for (int k = tid; k < NOUT * HID; k += NTH) W3[k] = prm[OFF_W3 + k];
  if (tid < NOUT) B3[tid] = prm[OFF_B3 + tid];
  for (int k = tid; k < MT * NIN; k += NTH) X[k] = (k / NIN < nb) ? x[(size_t)b0 * NIN + k] : 0.0f;
  if (TRAIN)
    for (int k = tid; k < MT * NOUT; k += NTH) T[k] = (k / NOUT < nb) ? tgt[(size_t)b0 * NOUT + k] : 0.0f;
  __syncthreads();

  // thread -> (unit o = tid % 64, samples b = tid / 64 + 4 r, r < 16)
  const int o = tid & (HID - 1);
  const int bq = tid >> 6;
  // layer 1
  for (int r = 0; r < MT / 4; r++) {
    const int b = bq + 4 * r;
    const float z = B1[o] + W1[o * NIN] * X[b * NIN] + W1[o * NIN + 1] * X[b * NIN + 1];
    H1[b * HID + o] = gelu(z);
    if (TRAIN) G1[b * HID + o] = gelu_slope(z);
  }
  __syncthreads();
  // layer 2: Z2[b][o] = b2[o] + sum_i W2[o][i] H1[b][i]
  {
    float acc[MT / 4];
#pragma unroll
    for (int r = 0; r < MT / 4; r++) acc[r] = B2[o];
    for (int i = 0; i < HID; i++) {
      const float w = W2[o * W2S + i];
#pragma unroll
      for (int r = 0; r < MT / 4; r++) acc[r] = fmaf(w, H1[(bq + 4 * r) * HID + i], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < MT / 4; r++) {
      const int b = bq + 4 * r;
      H2[b * HID + o] = gelu(acc[r]);
      if (TRAIN) G2[b * HID + o] = gelu_slope(acc[r]);
    }
  }
  __syncthreads();
  // layer 3 (threads 0..191: sample b = tid / 3, output k = tid % 3)
  float lsum = 0.0f;
  if (tid < MT * NOUT) {
    const int b = tid / NOUT, k = tid % NOUT;
    float acc = B3[k];
    for (int i = 0; i < HID; i++) acc = fmaf(W3[k * HID + i], H2[b * HID + i], acc);
    if (!TRAIN) {
      if (b < nb) y[(size_t)(b0 + b) * NOUT + k] = acc;
    } else {
      const float rr = (b < nb) ? acc - T[b * NOUT + k] : 0.0f;
      lsum = wout[k] * rr * rr;
      DY[b * NOUT + k] = 2.0f * wout[k] * rr / (float)B;
    }
  }
  if (!TRAIN) return;
  // tile loss: warp sums then the 8 warp partials in order
#pragma unroll
  for (int s = 16; s > 0; s >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, s);
  if ((tid & 31) == 0) RED[tid >> 5] = lsum;
  __syncthreads();
  float *out = part + (size_t)blockIdx.x * (NPARAM + 1);
  if (tid == 0) {
    float s = 0.0f;
    for (int w = 0; w < NTH / 32; w++) s += RED[w];
    out[NPARAM] = s;
  }
  // dZ2[b][o] = (sum_k dY[b][k] W3[k][o]) * G2[b][o]   (in place in G2)
  for (int r = 0; r < MT / 4; r++) {
    const int b = bq + 4 * r;
    float d = 0.0f;
#pragma unroll
    for (int k = 0; k < NOUT; k++) d = fmaf(DY[b * NOUT + k], W3[k * HID + o], d);
    G2[b * HID + o] *= d;
  }
  __syncthreads();
  // dZ1[b][i] = (sum_o dZ2[b][o] W2[o][i]) * G1[b][i]   (thread: i = tid % 64)
  {
    const int i = o;
    float acc[MT / 4];
#pragma unroll
    for (int r = 0; r < MT / 4; r++) acc[r] = 0.0f;
    for (int u = 0; u < HID; u++) {
      const float w = W2[u * W2S + i];
#pragma unroll
      for (int r = 0; r < MT / 4; r++) acc[r] = fmaf(G2[(bq + 4 * r) * HID + u], w, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < MT / 4; r++) G1[(bq + 4 * r) * HID + i] *= acc[r];
  }
  __syncthreads();
  // dW2[u][i] = sum_b dZ2[b][u] H1[b][i]   (thread: i = tid % 64, u = tid / 64 + 4 r)
  {
    float acc[MT / 4];
#pragma unroll
    for (int r = 0; r < MT / 4; r++) acc[r] = 0.0f;
    for (int b = 0; b < MT; b++) {
      const float h = H1[b * HID + o];
#pragma unroll
      for (int r = 0; r < MT / 4; r++) acc[r] = fmaf(G2[b * HID + bq + 4 * r], h, acc[r]);
    }
#pragma unroll
    for (int r = 0; r < MT / 4; r++) out[OFF_W2 + (bq + 4 * r) * HID + o] = acc[r];
  }
  // biases and the two small weight blocks
  if (tid < HID) {
    float s1 = 0.0f, s2 = 0.0f, w0 = 0.0f, w1 = 0.0f;
    for (int b = 0; b < MT; b++) {
      const float d1 = G1[b * HID + tid];
      s1 += d1;
      w0 = fmaf(d1, X[b * NIN], w0);
      w1 = fmaf(d1, X[b * NIN + 1], w1);
      s2 += G2[b * HID + tid];
    }
    out[OFF_B1 + tid] = s1;
    out[OFF_W1 + tid * NIN] = w0;
    out[OFF_W1 + tid * NIN + 1] = w1;
    out[OFF_B2 + tid] = s2;
    if (tid < NOUT) {
      float s3 = 0.0f;
      for (int b = 0; b < MT; b++) s3 += DY[b * NOUT + tid];
      out[OFF_B3 + tid] = s3;
    }
  } else {
    // threads 64..255: the 192 entries of dW3[k][u] = sum_b dY[b][k] H2[b][u]
    const int q = tid - HID, k = q / HID, u = q % HID;
    float s = 0.0f;
    for (int b = 0; b < MT; b++) s = fmaf(DY[b * NOUT + k], H2[b * HID + u], s);
    out[OFF_W3 + k * HID + u] = s;
  }
}

// grad[p] = sum over tiles (in tile order); loss = sum of tile losses / B.
__global__ void k_mlp_reduce(const float *__restrict__ part, int ntile, int B, float *__restrict__ grad,
                             float *__restrict__ loss) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < NPARAM) {
    float s = 0.0f;
    for (int c = 0; c < ntile; c++) s += part[(size_t)c * (NPARAM + 1) + p];
    grad[p] = s;
  } else if (p == NPARAM && loss) {
    float s = 0.0f;
    for (int c = 0; c < ntile; c++) s += part[(size_t)c * (NPARAM + 1) + NPARAM];
    *loss = s / (float)B;
  }
}

__global__ void k_adam(float *__restrict__ prm, const float *__restrict__ g, float *__restrict__ m,
                       float *__restrict__ v, int n, float lr, float b1, float b2, float eps, float bc1, float bc2) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= n) return;
  const float gp = g[p];
  const float mp = b1 * m[p] + (1.0f - b1) * gp;
  const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
  m[p] = mp;
  v[p] = vp;
  prm[p] -= lr * (mp / bc1) / (sqrtf(vp / bc2) + eps);
}

int ntiles(int B) { return (B + MT - 1) / MT; }

int smem_attr() {
  if (hk::allow_dynamic_smem((const void *)k_mlp_tile<true>) != cudaSuccess ||
      hk::allow_dynamic_smem((const void *)k_mlp_tile<false>) != cudaSuccess)
    return HK_ERR_CUDA;
  return HK_OK;
}

int enqueue_grad(const float *prm, const float *x, const float *t, const float *w, int B, float *grad, float *loss,
                 void *work, cudaStream_t s) {
  const int nt = ntiles(B);
  float *part = (float *)work;
  k_mlp_tile<true><<<nt, NTH, SMEM_BYTES, s>>>(prm, x, t, w, B, nullptr, part);
  k_mlp_reduce<<<(NPARAM + 1 + 255) / 256, 256, 0, s>>>(part, nt, B, grad, loss);
  return cudaGetLastError() == cudaSuccess ? HK_OK : HK_ERR_CUDA;
}

int enqueue_adam(float *prm, const float *g, float *m, float *v, int n, int step, float lr, float b1, float b2,
                 float eps, cudaStream_t s) {
  const float bc1 = (float)(1.0 - pow((double)b1, (double)step));
  const float bc2 = (float)(1.0 - pow((double)b2, (double)step));
  k_adam<<<(n + 255) / 256, 256, 0, s>>>(prm, g, m, v, n, lr, b1, b2, eps, bc1, bc2);
  return cudaGetLastError() == cudaSuccess ? HK_OK : HK_ERR_CUDA;
}

}  // namespace

extern "C" {

size_t hk_mlp_workspace_bytes(int B) {
  if (B < 1) return 0;
  return sizeof(float) * (size_t)ntiles(B) * (NPARAM + 1);
}

int hk_mlp_forward(const float *params, const float *x, int B, float *y, void *stream) {
  if (B < 1 || !params || !x || !y) return HK_ERR_ARG;
  if (smem_attr() != HK_OK) return HK_ERR_CUDA;
  k_mlp_tile<false><<<ntiles(B), NTH, SMEM_BYTES, (cudaStream_t)stream>>>(params, x, nullptr, nullptr, B, y,
                                                                           nullptr);
  return cudaGetLastError() == cudaSuccess ? HK_OK : HK_ERR_CUDA;
}

int hk_mlp_loss_grad(const float *params, const float *x, const float *t, const float *w, int B, float *grad,
                     float *loss, void *work, size_t work_bytes, void *stream) {
  if (B < 1 || !params || !x || !t || !w || !grad || !work) return HK_ERR_ARG;
  if (work_bytes < hk_mlp_workspace_bytes(B)) return HK_ERR_OOM;
  if (smem_attr() != HK_OK) return HK_ERR_CUDA;
  return enqueue_grad(params, x, t, w, B, grad, loss, work, (cudaStream_t)stream);
}

int hk_mlp_adam(float *params, const float *grad, float *m, float *v, int n, int step, float lr, float beta1,
                float beta2, float eps, void *stream) {
  if (n < 1 || step < 1 || !params || !grad || !m || !v) return HK_ERR_ARG;
  return enqueue_adam(params, grad, m, v, n, step, lr, beta1, beta2, eps, (cudaStream_t)stream);
}

int hk_mlp_train(float *params, float *m, float *v, float *grad, const float *x, const float *t, const float *w,
                 int B, int steps, int step0, float lr, float beta1, float beta2, float eps, float *loss_hist,
                 void *work, size_t work_bytes, void *stream) {
  if (B < 1 || steps < 0 || step0 < 0 || !params || !m || !v || !grad || !x || !t || !w || !work)
    return HK_ERR_ARG;
  if (work_bytes < hk_mlp_workspace_bytes(B)) return HK_ERR_OOM;
  if (smem_attr() != HK_OK) return HK_ERR_CUDA;
  cudaStream_t s = (cudaStream_t)stream;
  for (int k = 0; k < steps; k++) {
    int rc = enqueue_grad(params, x, t, w, B, grad, loss_hist ? loss_hist + k : nullptr, work, s);
    if (rc == HK_OK) rc = enqueue_adam(params, grad, m, v, NPARAM, step0 + k + 1, lr, beta1, beta2, eps, s);
    if (rc != HK_OK) return rc;
  }
  return HK_OK;
}

}  // extern "C"
