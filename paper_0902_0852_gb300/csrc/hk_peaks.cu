// Integer throughput probes that give the arithmetic roofline of the update
// kernel on the device at hand: the IMAD issue rate, the rate of the exact
// 3-word limb-product accumulation used by the update kernel, and the rate of
// the legacy warp-level INT8 tensor instruction (mma.sync m16n8k32 u8).
// Each probe runs a few milliseconds on every SM and reports operations per
// clock per SM, with the SM clock measured inside the kernels.
#include "hk.h"
#include "hk_internal.h"
#include "hk_mp.cuh"

namespace {

struct Stamp {
  unsigned long long c0, c1, t0, t1;
};

__device__ __forceinline__ unsigned long long gns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__global__ void p_imad(uint32_t *out, int iters, uint32_t seed, Stamp *st) {
  uint32_t x[8];
  for (int i = 0; i < 8; i++) x[i] = seed + threadIdx.x * 7 + i;
  const uint32_t m = seed | 1, c = seed ^ 0x9e37;
  const unsigned long long c0 = clock64(), t0 = gns();
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int r = 0; r < 16; r++) {
#pragma unroll
      for (int i = 0; i < 8; i++) asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(x[i]) : "r"(m), "r"(c));
    }
  }
  const unsigned long long c1 = clock64(), t1 = gns();
  uint32_t s = 0;
  for (int i = 0; i < 8; i++) s ^= x[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
  if (threadIdx.x == 0) st[blockIdx.x] = {c0, c1, t0, t1};
}

__global__ void p_mac3(uint32_t *out, int iters, uint32_t seed, Stamp *st) {
  uint32_t c0[8], c1[8], c2[8], w[8], a[8];
  for (int i = 0; i < 8; i++) {
    c0[i] = c1[i] = c2[i] = 0;
    w[i] = seed * (i + 5) + threadIdx.x;
    a[i] = seed ^ (i * 77u + threadIdx.x);
  }
  const unsigned long long k0 = clock64(), t0 = gns();
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int r = 0; r < 8; r++) {
#pragma unroll
      for (int i = 0; i < 8; i++) hk::mp::mac3(c0[i], c1[i], c2[i], a[r], w[i]);
    }
  }
  const unsigned long long k1 = clock64(), t1 = gns();
  uint32_t x = 0;
  for (int i = 0; i < 8; i++) x ^= c0[i] ^ c1[i] ^ c2[i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = x;
  if (threadIdx.x == 0) st[blockIdx.x] = {k0, k1, t0, t1};
}

__global__ void p_mma_u8(uint32_t *out, int iters, uint32_t seed, Stamp *st) {
  uint32_t A[4], B[2];
  int32_t C[4][4];
  for (int i = 0; i < 4; i++) A[i] = seed * (i + 1) + threadIdx.x;
  for (int i = 0; i < 2; i++) B[i] = seed ^ (i + threadIdx.x);
  for (int j = 0; j < 4; j++)
    for (int i = 0; i < 4; i++) C[j][i] = 0;
  const unsigned long long c0 = clock64(), t0 = gns();
  for (int it = 0; it < iters; it++) {
#pragma unroll
    for (int r = 0; r < 4; r++) {
#pragma unroll
      for (int j = 0; j < 4; j++)
        asm volatile(
            "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
            "{%0,%1,%2,%3};"
            : "+r"(C[j][0]), "+r"(C[j][1]), "+r"(C[j][2]), "+r"(C[j][3])
            : "r"(A[0]), "r"(A[1]), "r"(A[2]), "r"(A[3]), "r"(B[0]), "r"(B[1]));
    }
  }
  const unsigned long long c1 = clock64(), t1 = gns();
  int32_t s = 0;
  for (int j = 0; j < 4; j++)
    for (int i = 0; i < 4; i++) s ^= C[j][i];
  out[blockIdx.x * blockDim.x + threadIdx.x] = (uint32_t)s;
  if (threadIdx.x == 0) st[blockIdx.x] = {c0, c1, t0, t1};
}

typedef void (*Probe)(uint32_t *, int, uint32_t, Stamp *);

int run_probe(Probe fn, int iters, double ops_per_thread_iter, double *per_clk_sm, double *mhz) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nsm * 8, threads = 256;
  uint32_t *dout = nullptr;
  Stamp *dst = nullptr;
  // a private non-blocking stream: launches, events and the stamp copy are
  // ordered on it (no legacy-stream synchronous copies)
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return HK_ERR_CUDA;
  if (cudaMalloc(&dout, (size_t)blocks * threads * 4) != cudaSuccess) {
    cudaStreamDestroy(s);
    return HK_ERR_OOM;
  }
  if (cudaMalloc(&dst, (size_t)blocks * sizeof(Stamp)) != cudaSuccess) {
    cudaFree(dout);
    cudaStreamDestroy(s);
    return HK_ERR_OOM;
  }
  fn<<<blocks, threads, 0, s>>>(dout, 4, 1u, dst);
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, s);
  fn<<<blocks, threads, 0, s>>>(dout, iters, 12345u, dst);
  cudaEventRecord(e1, s);
  cudaError_t e = cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  Stamp *h = new Stamp[blocks];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, dst, blocks * sizeof(Stamp), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  double cyc = 0, ns = 0;
  for (int b = 0; b < blocks; b++) {
    cyc += (double)(h[b].c1 - h[b].c0);
    ns += (double)(h[b].t1 - h[b].t0);
  }
  delete[] h;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(dout);
  cudaFree(dst);
  cudaStreamDestroy(s);
  if (e != cudaSuccess || ms <= 0 || ns <= 0) return HK_ERR_CUDA;
  *mhz = cyc / ns * 1e3;
  const double rate = ops_per_thread_iter * iters * (double)blocks * threads / (ms * 1e-3);
  *per_clk_sm = rate / (*mhz * 1e6) / nsm;
  return HK_OK;
}

}  // namespace

extern "C" int hk_probe_int_peaks(int device, double *out, int n) {
  if (!out || n < 6) return HK_ERR_ARG;
  if (cudaSetDevice(device) != cudaSuccess) return HK_ERR_ARG;
  int rc = run_probe(p_imad, 2000, 16 * 8, &out[0], &out[1]);
  if (rc == HK_OK) rc = run_probe(p_mac3, 1000, 8 * 8, &out[2], &out[3]);
  if (rc == HK_OK) rc = run_probe(p_mma_u8, 2000, 4 * 4 * (16.0 * 8 * 32 / 32), &out[4], &out[5]);
  return rc;
}
