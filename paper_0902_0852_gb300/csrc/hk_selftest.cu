// Single-block driver of the device multiprecision library for unit tests:
// operands and work areas live in global memory, one operation per launch.
#include "hk.h"
#include "hk_internal.h"
#include "hk_mp.cuh"
#include <mutex>
#include <vector>

namespace hk {

namespace {

constexpr int NT_ST = 128;

__global__ void __launch_bounds__(NT_ST) k_selftest(int op, int L, const uint32_t *x, int nx, long long ex,
                                                    const uint32_t *y, int ny, long long ey, uint32_t *out,
                                                    long long *eo, uint32_t *scr, long long *cs, int cap) {
  __shared__ mp::Red red;
  mp::Work w;
  w.cs = cs;
  w.tmp = scr + 3 * cap;
  w.r = &red;
  mp::NBufs B;
  B.a = scr + 4 * cap;
  B.b = scr + 5 * cap;
  B.c = scr + 6 * cap;
  B.d = scr + 7 * cap;
  B.e = scr + 8 * cap;
  B.f = scr + 9 * cap;
  B.cap = cap;
  uint32_t *big = scr + 10 * cap, *q = scr + 11 * cap, *xs = scr + 12 * cap, *V = scr + 13 * cap;
  bool ok = true;
  if (op == 0) {
    mp::mul<NT_ST>(x, nx, y, ny, out, w);
  } else if (op == 1) {
    ok = mp::recip<NT_ST>(x, L, out, w, B);
  } else if (op == 2) {
    const mp::Rounded r = mp::sqrt_rne<NT_ST>(x, L, ex, out, w, B, big, xs, &ok);
    if (threadIdx.x == 0) *eo = r.exp;
  } else if (op == 3) {
    ok = mp::recip<NT_ST>(y, L, V, w, B, RECIP_EXTRA);
    bool ok2 = true;
    const mp::Rounded r = mp::div_rne<NT_ST>(x, ex, y, ey, V, L, out, w, big, q, &ok2, RECIP_EXTRA);
    ok = ok && ok2;
    if (threadIdx.x == 0) *eo = r.exp;
  } else if (op == 4) {
    const mp::Rounded r = mp::round_rne<NT_ST>(x, nx, ex, L, out, w);
    if (threadIdx.x == 0) *eo = r.nonzero ? r.exp : 0;
  }
  if (threadIdx.x == 0 && !ok) eo[1] = 1;
}

}  // namespace

int selftest_mp(int op, int L, const uint32_t *x, int nx, int64_t ex, const uint32_t *y, int ny, int64_t ey,
                uint32_t *out, int64_t *eo) {
  if (L < 1 || nx < 0 || ny < 0 || op < 0 || op > 4) return 1;
  const int cap = 5 * (nx + ny + L) + 128;
  int nout = 0;
  switch (op) {
    case 0: nout = nx + ny + 2; break;
    case 1: nout = L + 2; break;
    default: nout = L; break;
  }
  uint32_t *dx = nullptr, *dy = nullptr, *dout = nullptr, *scr = nullptr;
  long long *dcs = nullptr, *deo = nullptr;
  int rc = 0;
  auto ck = [&](cudaError_t e) {
    if (e != cudaSuccess && rc == 0) rc = 3;
  };
  // everything on a private non-blocking stream, ordered copies in and out
  // (no legacy-stream or pageable synchronous copies)
  cudaStream_t s = nullptr;
  ck(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  ck(cudaMalloc(&dx, 4 * (size_t)(nx + 1)));
  ck(cudaMalloc(&dy, 4 * (size_t)(ny + 1)));
  ck(cudaMalloc(&dout, 4 * (size_t)(cap)));
  ck(cudaMalloc(&scr, 4 * (size_t)cap * 14));
  ck(cudaMalloc(&dcs, 8 * (size_t)cap));
  ck(cudaMalloc(&deo, 16));
  long long h[2] = {0, 0};
  if (rc == 0) {
    ck(cudaMemcpyAsync(dx, x, 4 * (size_t)nx, cudaMemcpyHostToDevice, s));
    if (ny) ck(cudaMemcpyAsync(dy, y, 4 * (size_t)ny, cudaMemcpyHostToDevice, s));
    ck(cudaMemsetAsync(deo, 0, 16, s));
    ck(cudaMemsetAsync(dout, 0, 4 * (size_t)cap, s));
    ck(cudaMemsetAsync(scr, 0, 4 * (size_t)cap * 14, s));
    if (rc == 0) k_selftest<<<1, NT_ST, 0, s>>>(op, L, dx, nx, ex, dy, ny, ey, dout, deo, scr, dcs, cap);
    ck(cudaGetLastError());
    ck(cudaMemcpyAsync(out, dout, 4 * (size_t)nout, cudaMemcpyDeviceToHost, s));
    ck(cudaMemcpyAsync(h, deo, 16, cudaMemcpyDeviceToHost, s));
    ck(cudaStreamSynchronize(s));
    eo[0] = h[0];
    eo[1] = h[1];
  }
  cudaFree(dx);
  cudaFree(dy);
  cudaFree(dout);
  cudaFree(scr);
  cudaFree(dcs);
  cudaFree(deo);
  if (s) cudaStreamDestroy(s);
  return rc;
}

}  // namespace hk

// ---------------------------------------------------------------------------
// Allocation-free variant: the same single-block operation on caller device
// buffers, with its work area in a fixed device array instead of cudaMalloc.
// ---------------------------------------------------------------------------
namespace {

constexpr int NOALLOC_MAX_LIMBS = 4096;                    // nx + ny + L
constexpr int NOALLOC_CAP = 5 * NOALLOC_MAX_LIMBS + 128;   // limbs per work buffer
constexpr size_t NOALLOC_BYTES = (size_t)NOALLOC_CAP * (14 * 4 + 8);

// Work area shared by every call on a device; lives until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
std::mutex g_noalloc_mu;
unsigned char *g_noalloc_ptr[MAX_DEVICES] = {};

// device address of the work area for the current device (set up once per
// device, with that device current)
cudaError_t noalloc_area(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= MAX_DEVICES) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    g_noalloc_ptr[dev] = reinterpret_cast<unsigned char *>(p);
  }
  *out = g_noalloc_ptr[dev];
  return cudaSuccess;
}

}  // namespace

extern "C" int hk_mp_op_noalloc(int op, int L, const uint32_t *x, int nx, int64_t ex, const uint32_t *y, int ny,
                                int64_t ey, uint32_t *out, int64_t *eo, void *stream) {
  if (L < 1 || nx < 0 || ny < 0 || op < 0 || op > 4 || !x || !out || !eo || (ny > 0 && !y))
    return HK_ERR_ARG;
  if ((op == 1 || op == 2) && nx != L) return HK_ERR_ARG;
  if (op == 3 && (nx != L || ny != L)) return HK_ERR_ARG;
  // each size against the limit before any sum (no int overflow); the rounded
  // operations are argued for P = 32 L <= 32768 bits
  if (L > NOALLOC_MAX_LIMBS || nx > NOALLOC_MAX_LIMBS || ny > NOALLOC_MAX_LIMBS) return HK_ERR_ARG;
  if ((long long)nx + ny + L > NOALLOC_MAX_LIMBS) return HK_ERR_ARG;
  if (op >= 1 && 32LL * L > 32768) return HK_ERR_ARG;
  unsigned char *area = nullptr;
  if (noalloc_area(&area) != cudaSuccess) return HK_ERR_CUDA;
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  const int cap = 5 * (nx + ny + L) + 128;
  uint32_t *scr = reinterpret_cast<uint32_t *>(area);
  long long *cs = reinterpret_cast<long long *>(area + (size_t)NOALLOC_CAP * 14 * 4);
  // the allocating entry point starts from zeroed work buffers and exponent words
  if (cudaMemsetAsync(scr, 0, 4 * (size_t)cap * 14, s) != cudaSuccess) return HK_ERR_CUDA;
  if (cudaMemsetAsync(eo, 0, 2 * sizeof(int64_t), s) != cudaSuccess) return HK_ERR_CUDA;
  hk::k_selftest<<<1, hk::NT_ST, 0, s>>>(op, L, x, nx, ex, ny ? y : x, ny, ey, out,
                                          reinterpret_cast<long long *>(eo), scr, cs, cap);
  return cudaGetLastError() == cudaSuccess ? HK_OK : HK_ERR_CUDA;
}
