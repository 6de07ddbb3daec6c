// The exact trailing-update contraction (the hot loop).
//
// For every output o it adds  sum_t sign_t * X_o(t) * Y_o(t)  exactly into 64-bit
// column sums colsum[o][*], where X_o(t), Y_o(t) are non-negative integers of
// Wx and Wy 32-bit limbs.  In the factorisation X_o(t) = a_ti and Y_o(t) = a_tj
// are entries of R written on the common binary grid of their column, so
// sum_{t<i} R_ti R_tj (the update of section "The LDL^T Determinant
// Algorithm", M[row][col] -= C[col] * CDivDiag[row], applied for all earlier
// columns at once) becomes this plain integer contraction; the same kernel
// computes the blocked triangular-solve products and the dot products of
// inverse iteration.
//
// Layout of the work: the Wx x Wy grid of limb products (p, q) of one output is
// cut into stripes of UC consecutive result columns d = p + q, and each stripe's
// p-range into chunks of UPC: one (stripe, chunk) "unit" per thread.  A thread
// keeps a 96-bit accumulator (three words, mad.lo.cc / madc.hi.cc / addc) per
// column of its stripe across all t of its chunk of the contraction, reading
// X[p] and a sliding window of Y held in registers (one new Y limb per p).
// Shared-memory operand rows are zero-padded so that products outside the
// valid triangle vanish.  Entries are streamed into a USTAGES-deep ring by a
// producer warp with 1-D TMA bulk copies (cp.async.bulk + mbarrier);
// the eight compute warps release each stage with an mbarrier arrival.  All
// waits are bounded: a wait that runs out records HK_ERR_TIMEOUT and the block
// returns after waiting (again bounded) for its own copies in flight.
#include "hk_internal.h"
#include "hk_mp.cuh"
#include <algorithm>
#include <vector>

namespace hk {

namespace {

constexpr int XPADR = ((UPC + 3) / 4) * 4;
constexpr int YPADL = ((UC + UPC + 3) / 4) * 4;
constexpr int YPADR = ((UC + 3) / 4) * 4;
constexpr long long SPIN_LIMIT = 1LL << 30;
constexpr unsigned long long WAIT_LIMIT_NS = 2000000000ull;  // 2 s

HK_DEV uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
HK_DEV void mbar_init(uint64_t *bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}
HK_DEV void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
HK_DEV void mbar_arrive(uint64_t *bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}
HK_DEV bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
HK_DEV unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// bounded wait (about WAIT_LIMIT_NS); false when the limit ran out
HK_DEV bool mbar_wait(uint64_t *bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long i = 0; i < SPIN_LIMIT; i++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 0 && global_ns() - t0 > WAIT_LIMIT_NS) return false;
  }
  return false;
}
HK_DEV void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

struct Operands {
  const uint32_t *x;
  const uint32_t *y;
  int neg;
};

// operand pointers of output (i, j) at contraction index t
HK_DEV Operands operands(const UpdParams &p, int oi, int oj, int t) {
  Operands r;
  const long long N = p.N;
  if (p.mode == M_FACTOR) {
    const long long ia = tri_idx(t, oi, N), ja = tri_idx(t, oj, N);
    r.x = p.A + ia * p.W;
    r.y = p.A + ja * p.W;
    r.neg = p.Asign[ia] ^ p.Asign[ja];
  } else if (p.mode == M_GEMV_FWD) {
    const long long ia = tri_idx(t, oi, N);
    r.x = p.A + ia * p.W;
    r.y = p.Vy + (long long)t * p.Wv;
    r.neg = p.Asign[ia] ^ p.Vysign[t];
  } else if (p.mode == M_GEMV_BACK) {
    const long long ia = tri_idx(oi, t, N);
    r.x = p.A + ia * p.W;
    r.y = p.Vy + (long long)t * p.Wv;
    r.neg = p.Asign[ia] ^ p.Vysign[t];
  } else {  // M_DOT: output 0 = <x,x>, output 1 = <x,y>
    r.x = p.Vx + (long long)t * p.Wv;
    r.y = (oj == 0 ? p.Vx : p.Vy) + (long long)t * p.Wv;
    r.neg = p.Vxsign[t] ^ (oj == 0 ? p.Vxsign[t] : p.Vysign[t]);
  }
  return r;
}

// output o -> (i, j) and its row of colsum
HK_DEV void decode_output(const UpdParams &p, int o, int *oi, int *oj, long long *crow) {
  if (p.mode == M_FACTOR) {
    int i = p.ra;
    long long rem = o;
    while (rem >= p.N - i) {
      rem -= p.N - i;
      i++;
    }
    *oi = i;
    *oj = i + (int)rem;
    const long long k = i - p.r0;
    *crow = k * p.N - (k * (i + p.r0 - 1)) / 2 + rem;
  } else if (p.mode == M_DOT) {
    *oi = 0;
    *oj = o;
    *crow = o;
  } else {
    *oi = p.ra + o;
    *oj = 0;
    *crow = p.ra + o - p.r0;
  }
}

__global__ void __launch_bounds__(UNT + 32) k_update(UpdParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int Xsz = ((p.Wx + XPADR + 3) / 4) * 4;
  const int Ysz = ((YPADL + p.Wy + YPADR + 3) / 4) * 4;
  uint32_t *bufs = reinterpret_cast<uint32_t *>(smem_raw);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)USTAGES * (Xsz + Ysz) * 4);
  uint64_t *empty = full + USTAGES;
  volatile int *abort_flag = reinterpret_cast<volatile int *>(empty + USTAGES);

  if (p.st->code != ST_OK) return;  // an earlier step failed: nothing to do

  const int o = blockIdx.y;
  int oi, oj;
  long long crow;
  decode_output(p, o, &oi, &oj, &crow);
  int tb = p.t0 + blockIdx.z * p.tchunk;
  int te = min(p.t1, tb + p.tchunk);
  if (p.mode == M_GEMV_FWD) te = min(te, oi);            // t < i
  if (p.mode == M_GEMV_BACK) tb = max(tb, oi + 1);       // t > i
  const int nt = te - tb;
  if (nt <= 0) return;

  // zero the whole ring once (pads stay zero; TMA writes only the middle)
  for (int k = threadIdx.x; k < USTAGES * (Xsz + Ysz); k += blockDim.x) bufs[k] = 0;
  if (threadIdx.x == 0) {
    for (int s = 0; s < USTAGES; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], UNT / 32);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const uint32_t bytesX = (uint32_t)p.Wx * 4u, bytesY = (uint32_t)p.Wy * 4u;

  if (warp == UNT / 32) {
    // ---------------- producer warp ----------------
    if (lane == 0) {
      int issued = 0;
      for (int it = 0; it < nt; it++) {
        const int s = it % USTAGES;
        if (it >= USTAGES) {
          if (!mbar_wait(&empty[s], ((it / USTAGES) - 1) & 1)) {
            atomicAdd(&p.st->timeout, 1);
            *abort_flag = 1;
            break;
          }
        }
        if (*abort_flag) break;
        const Operands op = operands(p, oi, oj, tb + it);
        uint32_t *xs = bufs + (size_t)s * (Xsz + Ysz);
        uint32_t *ys = xs + Xsz + YPADL;
        mbar_expect_tx(&full[s], bytesX + bytesY);
        bulk_g2s(xs, op.x, bytesX, &full[s]);
        bulk_g2s(ys, op.y, bytesY, &full[s]);
        issued = it + 1;
      }
      if (*abort_flag) {
        // wait (bounded) for our own copies in flight before leaving
        for (int it = max(0, issued - USTAGES); it < issued; it++)
          mbar_wait(&full[it % USTAGES], (it / USTAGES) & 1);
      }
    }
    return;
  }

  // ---------------- compute warps ----------------
  const int u = blockIdx.x * UNT + threadIdx.x;
  const bool active = u < p.nunits;
  Unit un = active ? p.units[u] : Unit{0, 0};
  uint32_t c0[UC], c1[UC], c2[UC];
#pragma unroll
  for (int m = 0; m < UC; m++) c0[m] = c1[m] = c2[m] = 0;

  for (int it = 0; it < nt; it++) {
    const int s = it % USTAGES;
    if (!mbar_wait(&full[s], (it / USTAGES) & 1)) {
      if (lane == 0) atomicAdd(&p.st->timeout, 1);
      *abort_flag = 1;
      break;
    }
    if (*abort_flag) break;
    const uint32_t *X = bufs + (size_t)s * (Xsz + Ysz);
    const uint32_t *Y = X + Xsz + YPADL;
    const Operands op = operands(p, oi, oj, tb + it);  // sign only
    if (active) {
      const int d0 = un.d0, p0 = un.p0;
      uint32_t wb[UC];
#pragma unroll
      for (int m = 1; m < UC; m++) wb[m] = Y[d0 + m - p0];
      if (!op.neg) {
#pragma unroll 1
        for (int b = 0; b < UPC / UC; b++) {
#pragma unroll
          for (int j = 0; j < UC; j++) {
            const int pp = p0 + b * UC + j;
            wb[(UC - j) % UC] = Y[d0 - pp];
            const uint32_t a = X[pp];
#pragma unroll
            for (int m = 0; m < UC; m++) mp::mac3(c0[m], c1[m], c2[m], a, wb[(m - j + UC) % UC]);
          }
        }
      } else {
#pragma unroll 1
        for (int b = 0; b < UPC / UC; b++) {
#pragma unroll
          for (int j = 0; j < UC; j++) {
            const int pp = p0 + b * UC + j;
            wb[(UC - j) % UC] = Y[d0 - pp];
            const uint32_t a = X[pp];
#pragma unroll
            for (int m = 0; m < UC; m++) mp::msub3(c0[m], c1[m], c2[m], a, wb[(m - j + UC) % UC]);
          }
        }
      }
    }
    __syncwarp();
    if (lane == 0) mbar_arrive(&empty[s]);
  }

  if (!active || *abort_flag) return;
  // flush: stripe words -> signed 64-bit column partial sums, added atomically
  unsigned long long *dst = reinterpret_cast<unsigned long long *>(p.colsum + crow * p.C + un.d0);
  const int lim = p.C - un.d0;
#pragma unroll
  for (int m = 0; m < UC + 2; m++) {
    long long v = 0;
    if (m < UC) v += (long long)c0[m];
    if (m >= 1 && m <= UC) v += (long long)c1[m - 1];
    if (m >= 2) v += (long long)(int32_t)c2[m - 2];
    if (v != 0 && m < lim) atomicAdd(dst + m, (unsigned long long)v);
  }
}

}  // namespace

int colsum_width(int Wx, int Wy) {
  const int S = (Wx + Wy - 1 + UC - 1) / UC;
  const int c = std::max(Wx + Wy + 2, S * UC + 2);
  return ((c + 3) / 4) * 4;
}

// Units in chunk-major order: for chunk k, consecutive stripes, so that the
// threads of a warp read X[p] at one address (or stride UC) and Y with stride UC
// (UC odd: no shared-memory bank conflicts).
int build_units(int Wx, int Wy, Unit *out, int cap) {
  const int S = (Wx + Wy - 1 + UC - 1) / UC;
  std::vector<int> plo(S), len(S);
  int kmax = 0;
  for (int s = 0; s < S; s++) {
    const int d0 = s * UC;
    const int lo = std::max(0, d0 - Wy + 1);
    const int hi = std::min(Wx - 1, d0 + UC - 1);
    plo[s] = lo;
    len[s] = hi >= lo ? hi - lo + 1 : 0;
    kmax = std::max(kmax, (len[s] + UPC - 1) / UPC);
  }
  int n = 0;
  for (int k = 0; k < kmax; k++)
    for (int s = 0; s < S; s++)
      if (k * UPC < len[s]) {
        if (out && n < cap) out[n] = Unit{s * UC, plo[s] + k * UPC};
        n++;
      }
  return n;
}

cudaError_t launch_update(const UpdParams &p, cudaStream_t s) {
  if (p.nout <= 0 || p.t1 <= p.t0 || p.nunits <= 0) return cudaSuccess;
  const int Xsz = ((p.Wx + XPADR + 3) / 4) * 4;
  const int Ysz = ((YPADL + p.Wy + YPADR + 3) / 4) * 4;
  const size_t smem = (size_t)USTAGES * (Xsz + Ysz) * 4 + 2 * USTAGES * 8 + 16;
  static size_t configured = 0;
  if (smem > 48 * 1024 && smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_update, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  const int nz = (p.t1 - p.t0 + p.tchunk - 1) / p.tchunk;
  dim3 grid((p.nunits + UNT - 1) / UNT, p.nout, nz);
  k_update<<<grid, UNT + 32, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace hk
