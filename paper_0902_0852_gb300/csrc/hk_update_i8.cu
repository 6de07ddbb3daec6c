// INT8 tensor-core form of the exact trailing update: the same contraction
// sum_t +-a_ti a_tj as the IMAD kernel, computed from bytes (radix 2^8 digits)
// with the warp-level instruction mma.sync.m16n8k32 u8 x u8 -> s32.  The
// integer result is identical, so R is bit-identical to the IMAD path.
//
// For one output row i and eight output columns j0..j0+7 (the N dimension of
// the instruction) the byte columns of the product are
//   col_{i,j}[d] = sum_q x[d - q] y_j[q],  x = bytes of a_ti, y_j = bytes of a_tj,
// i.e. C[m][n] = sum_k A[m][k] B[k][n] with m = 16 consecutive result columns d,
// k = 32 consecutive bytes q, A[m][k] = x[d0 + m - q0 - k] (a Toeplitz tile of x)
// and B[k][n] = y_n[q0 + k].  The Toeplitz operand is read from four byte-shifted,
// reversed, zero-padded copies of x in shared memory, so that every fragment
// register is one aligned 32-bit load.  Each t's s32 partial sums (at most
// (bytes of the entry) * 255^2 < 2^31) are added, with the sign of the product,
// into 64-bit byte-column sums held in registers; at the end they are split
// exactly into 32-bit limb columns and added atomically to the output's column
// sums.  The operand entries of each t are staged by 1-D TMA bulk copies.
#include "hk_internal.h"
#include "hk_mp.cuh"

namespace hk {

namespace {

constexpr int I8_NT = 256;      // 8 warps
constexpr int I8_DB = 2;        // 16-column blocks per warp
constexpr int I8_PADB = 64;     // zero bytes around the reversed copies of x
constexpr unsigned long long I8_WAIT_NS = 2000000000ull;

HK_DEV uint32_t su32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

HK_DEV bool i8_wait(uint64_t *bar, uint32_t parity, unsigned long long limit) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  for (long long i = 0; i < (1LL << 30); i++) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(su32(bar)), "r"(parity)
        : "memory");
    if (ok) return true;
    if ((i & 63) == 0) {
      unsigned long long t;
      asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
      if (t - t0 > limit) return false;
    }
  }
  return false;
}

HK_DEV void mma_u8(int32_t (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k32.row.col.s32.u8.u8.s32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};"
      : "+r"(c[0]), "+r"(c[1]), "+r"(c[2]), "+r"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// grid: x = blocks of I8_NT/32 * I8_DB 16-column groups, y = output octets, z = t chunks
__global__ void __launch_bounds__(I8_NT) k_update_i8(const __grid_constant__ UpdParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int W = p.astride;          // limbs per entry
  const int nb = 4 * W;             // bytes per entry
  const int NXR = (nb + 2 * I8_PADB) / 4 + 2;  // words per shifted reversed copy of x
  const int NY = (nb + I8_PADB) / 4;           // words per y slot
  uint32_t *xst = reinterpret_cast<uint32_t *>(smem_raw);    // W words, TMA target
  uint32_t *xr4 = xst + W;                                   // 4 x NXR words
  uint32_t *ys = xr4 + 4 * NXR;                              // 8 x NY words
  uint64_t *bar = reinterpret_cast<uint64_t *>(ys + 8 * NY + (((8 * NY + 4 * NXR + W) & 1) ? 1 : 0));
  int *sg = reinterpret_cast<int *>(bar + 1);                // 9 signs + valid mask + abort

  if (p.st->code != ST_OK) return;

  // output octet -> (i, j0)
  int i = p.ra;
  long long rem = blockIdx.y;
  while (rem >= (p.N - i + 7) / 8) {
    rem -= (p.N - i + 7) / 8;
    i++;
  }
  const int j0 = i + 8 * (int)rem;
  const int tb = p.t0 + blockIdx.z * p.tchunk;
  const int te = min(p.t1, tb + p.tchunk);
  const int nt = te - tb;
  if (nt <= 0) return;

  // zero the y slots (columns past N stay zero) and the padding of x copies
  for (int k = threadIdx.x; k < 8 * NY; k += I8_NT) ys[k] = 0;
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(bar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    sg[10] = 0;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int g = lane >> 2, tq = lane & 3;
  const int ngroups = (2 * nb - 1 + 15) / 16;  // 16-column groups of the product
  int gidx[I8_DB];
#pragma unroll
  for (int b = 0; b < I8_DB; b++) gidx[b] = (blockIdx.x * (I8_NT / 32) + warp) * I8_DB + b;
  long long acc[I8_DB][4];
#pragma unroll
  for (int b = 0; b < I8_DB; b++)
#pragma unroll
    for (int e = 0; e < 4; e++) acc[b][e] = 0;
  const int ncols = min(8, p.N - j0);
  const long long N = p.N;
  const unsigned char *xb = reinterpret_cast<const unsigned char *>(xst);

  for (int it = 0; it < nt; it++) {
    const int t = tb + it;
    if (threadIdx.x == 0) {
      // the previous t's shared-memory reads are complete (barrier below); order
      // them before the asynchronous copies that overwrite the buffers
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      const long long ia = tri_idx(t, i, N);
      const uint32_t bytes = (uint32_t)(nb * (1 + ncols));
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(bar)), "r"(bytes) : "memory");
      asm volatile(
          "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(su32(xst)),
          "l"(p.A + ia * W), "r"((uint32_t)nb), "r"(su32(bar))
          : "memory");
      sg[8] = p.Asign[ia];
      for (int n = 0; n < ncols; n++) {
        const long long ja = tri_idx(t, j0 + n, N);
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                su32(ys + n * NY)),
            "l"(p.A + ja * W), "r"((uint32_t)nb), "r"(su32(bar))
            : "memory");
        sg[n] = p.Asign[ja];
      }
      const unsigned long long lim = p.wait_ns > 0 ? (unsigned long long)p.wait_ns : I8_WAIT_NS;
      if (!i8_wait(bar, it & 1, lim)) {
        raise_timeout(p.st);
        sg[10] = 1;
        i8_wait(bar, it & 1, lim);  // bounded second wait for the copies in flight
      }
    }
    __syncthreads();
    if (sg[10]) return;
    // four byte-shifted reversed copies: xr_s[z] = xr[z + s], xr[z] = x[nb-1-(z-PADB)] (0 outside)
    for (int k = threadIdx.x; k < 4 * NXR; k += I8_NT) {
      const int s = k / NXR, wd = k - s * NXR;
      uint32_t v = 0;
#pragma unroll
      for (int by = 0; by < 4; by++) {
        const int z = 4 * wd + by + s - I8_PADB;
        const int xi = nb - 1 - z;
        const uint32_t bv = (z >= 0 && xi >= 0) ? xb[xi] : 0u;
        v |= bv << (8 * by);
      }
      xr4[k] = v;
    }
    __syncthreads();
    // signs of the eight products of this t (columns past N contribute zero)
    int negmask = 0;
    for (int n = 0; n < ncols; n++) negmask |= (sg[n] ^ sg[8]) << n;
    const int K0 = nb - 1 + I8_PADB;
#pragma unroll
    for (int b = 0; b < I8_DB; b++) {
      const int gi = gidx[b];
      if (gi >= ngroups) continue;
      const int d0 = 16 * gi;
      const int qlo = max(0, d0 - nb + 1), qhi = min(nb - 1, d0 + 15);
      int32_t c[4] = {0, 0, 0, 0};
      for (int q0 = qlo & ~31; q0 <= qhi; q0 += 32) {
        uint32_t a[4];
        // a0: (row g, k = 4tq..), a1: (row g+8, k = 4tq..), a2/a3: k + 16
#pragma unroll
        for (int r = 0; r < 4; r++) {
          const int m = g + ((r & 1) ? 8 : 0);
          const int k = 4 * tq + ((r & 2) ? 16 : 0);
          const int z0 = K0 - (d0 + m - q0) + k;
          const int s = z0 & 3;
          a[r] = xr4[s * NXR + ((z0 - s) >> 2)];
        }
        const uint32_t *yb = ys + g * NY;
        const uint32_t b0 = yb[(q0 >> 2) + tq];
        const uint32_t b1 = yb[(q0 >> 2) + 4 + tq];
        mma_u8(c, a, b0, b1);
      }
      // c0, c1: row g, columns 2tq, 2tq+1; c2, c3: row g+8, same columns
#pragma unroll
      for (int e = 0; e < 4; e++) {
        const int n = 2 * tq + (e & 1);
        acc[b][e] += ((negmask >> n) & 1) ? -(long long)c[e] : (long long)c[e];
      }
    }
    __syncthreads();
  }

  // flush: byte column d -> limb columns d/4 and d/4+1, split exactly
  const int k0 = i - p.r0;
  const long long rowoff = (long long)k0 * p.N - ((long long)k0 * (i + p.r0 - 1)) / 2;
#pragma unroll
  for (int b = 0; b < I8_DB; b++) {
    const int gi = gidx[b];
    if (gi >= ngroups) continue;
#pragma unroll
    for (int e = 0; e < 4; e++) {
      const int n = 2 * tq + (e & 1);
      if (n >= ncols) continue;
      const int d = 16 * gi + g + ((e & 2) ? 8 : 0);
      const long long v = acc[b][e];
      if (v == 0) continue;
      const int D = d >> 2, sh = 8 * (d & 3);
      const long long lowmask = (1LL << (32 - sh)) - 1;
      const long long lo = v & lowmask;          // 0 <= lo < 2^(32 - sh)
      const long long hi = (v - lo) >> (32 - sh);  // exact
      unsigned long long *dst =
          reinterpret_cast<unsigned long long *>(p.colsum + (rowoff + (j0 + n - i)) * p.C);
      if (D < p.C) atomicAdd(dst + D, (unsigned long long)(lo << sh));
      if (D + 1 < p.C && hi != 0) atomicAdd(dst + D + 1, (unsigned long long)hi);
    }
  }
}

}  // namespace

size_t update_i8_smem(int W) {
  const int nb = 4 * W;
  const int NXR = (nb + 2 * I8_PADB) / 4 + 2;
  const int NY = (nb + I8_PADB) / 4;
  return (size_t)4 * (W + 4 * NXR + 8 * NY + 2) + 16 + 64;
}

// FACTOR-mode update on plain aligned entries (astride = W limbs)
cudaError_t launch_update_i8(const UpdParams &p, cudaStream_t s) {
  if (p.nout <= 0 || p.t1 <= p.t0) return cudaSuccess;
  const int W = p.astride;
  const size_t smem = update_i8_smem(W);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_dynamic_smem((const void *)k_update_i8);
    if (e != cudaSuccess) return e;
  }
  long long noct = 0;
  for (int i = p.ra; i < p.rb; i++) noct += (p.N - i + 7) / 8;
  const int ngroups = (2 * 4 * W - 1 + 15) / 16;
  const int gpb = (I8_NT / 32) * I8_DB;
  dim3 grid((ngroups + gpb - 1) / gpb, (unsigned)noct, (p.t1 - p.t0 + p.tchunk - 1) / p.tchunk);
  k_update_i8<<<grid, I8_NT, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace hk
