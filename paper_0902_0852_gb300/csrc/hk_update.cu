// The exact trailing-update contraction (the hot loop).
//
// For every output o it adds  sum_t sign_t * X_o(t) * Y_o(t)  exactly into 64-bit
// column sums colsum[o][*], where X_o(t), Y_o(t) are non-negative integers.  In the
// factorisation X_o(t) = a_ti and Y_o(t) = a_tj are entries of R written on the
// common binary grid of their column, so sum_{t<i} R_ti R_tj (the update of
// section "The LDL^T Determinant Algorithm", M[row][col] -= C[col] * CDivDiag[row],
// applied for all earlier columns at once) becomes this plain integer
// contraction; the same kernel computes the blocked triangular-solve products
// and the dot products of inverse iteration.
//
// Karatsuba on the whole dot product: with a = a0 + a1 B,
//   sum a_i a_j = C0 + B (Cs - C0 - C1) + B^2 C1,
//   C0 = sum a0_i a0_j, C1 = sum a1_i a1_j, Cs = sum (a0+a1)_i (a0+a1)_j,
// so one launch runs a list of smaller contractions ("sub-problems", 3^levels
// for up to four levels), each added to the column sums at its (offset, sign)
// terms (up to 2^levels of them).
// The identity is exact, so results do not depend on the expansion depth.
//
// Layout of the work: the wx x wy grid of limb products (p, q) of one
// sub-problem is cut into stripes of UC consecutive result columns d = p + q,
// and each stripe's p-range into chunks of `upc`: one (stripe, chunk) "unit"
// per thread.  A thread keeps a 96-bit accumulator (three words,
// mad.lo.cc / madc.hi.cc / addc) per column of its stripe across all t of its
// chunk of the contraction, reading X[p] and a sliding window of Y held in
// registers (one new Y limb per p).  Operand pieces are separated by zero gaps
// so that products outside the valid triangle vanish.  Entries are streamed
// into a USTAGES-deep ring by a producer warp with 1-D TMA bulk copies
// (cp.async.bulk + mbarrier); the eight compute warps release each stage with
// an mbarrier arrival.  All waits are bounded: a wait that runs out records
// HK_ERR_TIMEOUT and the block returns after waiting (again bounded) for its
// own copies in flight.
#include "hk_internal.h"
#include "hk_mp.cuh"
#include <algorithm>
#include <climits>
#include <cstdio>
#include <cstdlib>
#include <mutex>
#include <set>
#include <vector>

namespace hk {

namespace {

// right pad of a staged Y entry: a unit reads up to uc + 2 limbs past it (a
// stripe-8 unit's chunk may start up to three limbs early, see build_units)
__host__ __device__ inline int ypadr(int uc) { return ((uc + 6) / 4) * 4; }
__host__ __device__ inline int xpadr(int upc) { return ((upc + 3) / 4) * 4; }
__host__ __device__ inline int ypadl(int uc, int upc) { return ((uc + upc + 3) / 4) * 4; }
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
// bounded wait (about `limit` ns, at most SPIN_LIMIT polls); false when the
// limit ran out
HK_DEV bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit) {
  if (mbar_try_wait(bar, parity)) return true;
  const unsigned long long t0 = global_ns();
  for (long long i = 0; i < SPIN_LIMIT; i++) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63) == 0 && global_ns() - t0 > limit) return false;
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

// operand entries of output (i, j) at contraction index t
HK_DEV Operands operands(const UpdParams &p, int oi, int oj, int t) {
  Operands r;
  const long long N = p.N;
  if (p.mode == M_FACTOR) {
    const long long ia = tri_idx(t, oi, N), ja = tri_idx(t, oj, N);
    r.x = p.A + ia * p.astride;
    r.y = p.A + ja * p.astride;
    r.neg = p.Asign[ia] ^ p.Asign[ja];
  } else if (p.mode == M_LDLT) {
    // C_t[i] * CDivDiag_t[j]: column entry of row t against its quotient
    const long long ia = tri_idx(t, oi, N), ja = tri_idx(t, oj, N);
    r.x = p.A + ia * p.astride;
    r.y = p.B + ja * p.astride;
    r.neg = p.Asign[ia] ^ p.Bsign[ja];
  } else if (p.mode == M_GEMV_FWD) {
    const long long ia = tri_idx(t, oi, N);
    r.x = p.A + ia * p.astride;
    r.y = p.Vy + (long long)t * p.vstride;
    r.neg = p.Asign[ia] ^ p.Vysign[t];
  } else if (p.mode == M_GEMV_BACK) {
    const long long ia = tri_idx(oi, t, N);
    r.x = p.A + ia * p.astride;
    r.y = p.Vy + (long long)t * p.vstride;
    r.neg = p.Asign[ia] ^ p.Vysign[t];
  } else {  // M_DOT: output 0 = <x,x>, output 1 = <x,y>
    r.x = p.Vx + (long long)t * p.vstride;
    r.y = (oj == 0 ? p.Vx : p.Vy) + (long long)t * p.vstride;
    r.neg = p.Vxsign[t] ^ (oj == 0 ? p.Vxsign[t] : p.Vysign[t]);
  }
  return r;
}

// output o -> (i, j) and its row of colsum
HK_DEV void decode_output(const UpdParams &p, int o, int *oi, int *oj, long long *crow) {
  if (p.mode == M_FACTOR || p.mode == M_LDLT) {
    // column-major over the block's outputs: the rows i of one column j are
    // neighbours in launch order, so the operand entries (t, j) they share are
    // read from L2 by consecutive blocks (the entries (t, i) of the block's
    // few rows are shared by all and stay resident)
    const int n = p.rb - p.ra;
    const long long tri = (long long)n * (n + 1) / 2;
    int i, j;
    if (o < tri) {  // columns j < rb: rows ra .. j
      int c = 0;
      long long rem = o;
      while (rem > c) {
        rem -= c + 1;
        c++;
      }
      j = p.ra + c;
      i = p.ra + (int)rem;
    } else {
      const long long q = o - tri;
      j = p.rb + (int)(q / n);
      i = p.ra + (int)(q % n);
    }
    *oi = i;
    *oj = j;
    const long long k = i - p.r0;
    *crow = k * p.N - (k * (i + p.r0 - 1)) / 2 + (j - i);
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

#ifndef HK_UPDATE_MINBLOCKS
#define HK_UPDATE_MINBLOCKS 3
#endif
template <int UC>
__global__ void __launch_bounds__(UNT + 32, HK_UPDATE_MINBLOCKS) k_update(const __grid_constant__ UpdParams p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int NS = p.nst;
  const unsigned long long wlim = p.wait_ns > 0 ? (unsigned long long)p.wait_ns : WAIT_LIMIT_NS;
  const int XPADR = xpadr(p.upc), YPADL = ypadl(UC, p.upc), YPADR = ypadr(UC);
  const int Xsz = ((p.cx + XPADR + 3) / 4) * 4;
  const int Ysz = ((YPADL + p.cy + YPADR + 3) / 4) * 4;
  uint32_t *bufs = reinterpret_cast<uint32_t *>(smem_raw);
  uint64_t *full = reinterpret_cast<uint64_t *>(smem_raw + (size_t)NS * (Xsz + Ysz) * 4);
  uint64_t *empty = full + NS;
  int *sneg = reinterpret_cast<int *>(empty + NS);  // sign of the stage's product
  volatile int *abort_flag = sneg + NS;

  if (block_status(p.st) != ST_OK) return;  // an earlier step failed: nothing to do
  if (!HK_CHECK(p.st, (size_t)NS * (Xsz + Ysz) * 4 + 2 * NS * 8 + 4 * (NS + 4) <= dynamic_smem_bytes(),
                1, (size_t)NS * (Xsz + Ysz) * 4, dynamic_smem_bytes()))
    return;

  const int o = blockIdx.y;
  int oi, oj;
  long long crow;
  decode_output(p, o, &oi, &oj, &crow);
  int tb = p.t0 + blockIdx.z * p.tchunk;
  int te = min(p.t1, tb + p.tchunk);
  if (p.mode == M_GEMV_FWD) te = min(te, oi);       // t < i
  if (p.mode == M_GEMV_BACK) tb = max(tb, oi + 1);  // t > i
  const int nt = te - tb;
  if (nt <= 0) return;

  // zero the pads of the stages in use (TMA writes only the operand entries)
  const int used = min(nt, NS);
  for (int s = 0; s < used; s++) {
    uint32_t *xs = bufs + (size_t)s * (Xsz + Ysz);
    for (int k = threadIdx.x; k < Xsz - p.cx; k += blockDim.x) xs[p.cx + k] = 0;
    uint32_t *ys = xs + Xsz;
    for (int k = threadIdx.x; k < YPADL; k += blockDim.x) ys[k] = 0;
    for (int k = threadIdx.x; k < Ysz - YPADL - p.cy; k += blockDim.x) ys[YPADL + p.cy + k] = 0;
  }
  if (threadIdx.x == 0) {
    for (int s = 0; s < NS; s++) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], UNT / 32);
    }
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // operand window of this block (whole entries when nxb = 0)
  const int wlo = p.nxb ? p.xlo[blockIdx.x] : 0;
  const uint32_t bytesX = (uint32_t)(p.nxb ? p.xlen[blockIdx.x] : p.cx) * 4u;
  const uint32_t bytesY = (uint32_t)(p.nxb ? p.xlen[blockIdx.x] : p.cy) * 4u;

  if (warp == UNT / 32) {
    // ---------------- producer warp ----------------
    if (lane == 0) {
      int issued = 0;
      int s = 0, rnd = 0;  // stage of `it` and how often the ring has wrapped
      for (int it = 0; it < nt; it++, s = (s + 1 == NS) ? 0 : s + 1, rnd += (s == 0)) {
        if (rnd > 0) {
          if (!mbar_wait(&empty[s], (rnd - 1) & 1, wlim)) {
            raise_timeout(p.st);
            *abort_flag = 1;
            break;
          }
        }
        if (*abort_flag) break;
        const Operands op = operands(p, oi, oj, tb + it);
#ifdef HK_CHECKED
        {
          const uint32_t *bx = p.mode == M_DOT ? p.Vx : p.A;
          const long long lx = p.mode == M_DOT ? p.vx_len : p.a_len;
          const uint32_t *by = p.mode == M_FACTOR ? p.A : p.mode == M_LDLT ? p.B : (p.mode == M_DOT && oj == 0 ? p.Vx : p.Vy);
          const long long ly = (p.mode == M_FACTOR || p.mode == M_LDLT) ? p.a_len : (p.mode == M_DOT && oj == 0 ? p.vx_len : p.vy_len);
          const long long ox = op.x + wlo - bx, oy = op.y + wlo - by;
          if (!HK_CHECK(p.st, ox >= 0 && ox + bytesX / 4 <= lx, 2, ox, lx) ||
              !HK_CHECK(p.st, oy >= 0 && oy + bytesY / 4 <= ly, 3, oy, ly) ||
              !HK_CHECK(p.st, ((uintptr_t)(op.x + wlo) & 15) == 0 && ((uintptr_t)(op.y + wlo) & 15) == 0 &&
                                  (bytesX & 15) == 0 && (bytesY & 15) == 0 && bytesX <= 4u * p.cx &&
                                  bytesY <= 4u * p.cy,
                        4, (long long)((uintptr_t)(op.x + wlo) & 15), (long long)bytesX)) {
            *abort_flag = 1;
            break;
          }
        }
#endif
        uint32_t *xs = bufs + (size_t)s * (Xsz + Ysz);
        uint32_t *ys = xs + Xsz + YPADL;
        sneg[s] = op.neg;
        mbar_expect_tx(&full[s], bytesX + bytesY);
        bulk_g2s(xs, op.x + wlo, bytesX, &full[s]);
        bulk_g2s(ys, op.y + wlo, bytesY, &full[s]);
        issued = it + 1;
      }
      if (*abort_flag) {
        // wait (bounded) for our own copies in flight before leaving
        for (int it = max(0, issued - NS); it < issued; it++)
          mbar_wait(&full[it % NS], (it / NS) & 1, wlim);
      }
    }
    return;
  }

  // ---------------- compute warps ----------------
  const int u = blockIdx.x * UNT + threadIdx.x;
  bool active = u < p.nunits;
  const Unit un = active ? p.units[u] : Unit{0, 0};
  const int sp = (un.d0 >> 24) & 0xff;
  const int d0 = un.d0 & 0xffffff;
  // stripe 8: chunk start in bits 0..15, its length in groups of eight p-steps
  // in bits 16..23; other stripes: chunks of p.upc
  const int p0 = UC == 8 ? (un.p0 & 0xffff) : un.p0;
  const int ngrp = UC == 8 ? ((un.p0 >> 16) & 0xff) : p.upc / UC;
  // a unit table entry must name one of this launch's sub-problems (always
  // checked: a bad entry would index the operand tiles with wrong offsets)
  if (active && sp >= p.nsub) active = check_fail(p.st, 5, sp, p.nsub);
  const int xoff = p.sub[active ? sp : 0].xoff - wlo, yoff = p.sub[active ? sp : 0].yoff - wlo;
  // stripe-8 units read X four limbs at a time: chunk starts and piece
  // offsets are multiples of four limbs (always checked)
  if (UC == 8 && active && ((p0 | xoff) & 3)) active = check_fail(p.st, 10, p0, xoff);
#ifdef HK_CHECKED
  if (active) {
    // every shared-memory word the unit reads lies in its stage's X or Y tile
    // (inside the block's operand window when it has one)
    const long long xlim = p.nxb ? p.xlen[blockIdx.x] : Xsz;
    const long long ymin = p.nxb ? YPADL : 0, ylim = p.nxb ? YPADL + p.xlen[blockIdx.x] : Ysz;
    const long long xlo = xoff + p0, xhi = xoff + p0 + ngrp * UC - 1;
    const long long ylo = YPADL + yoff + d0 - p0 - ngrp * UC + 1, yhi = YPADL + yoff + d0 - p0 + UC - 1;
    if (!HK_CHECK(p.st, xlo >= 0 && xhi < xlim, 6, xhi, xlim) ||
        !HK_CHECK(p.st, ylo >= ymin && yhi < ylim, 7, ylo < ymin ? ylo : yhi, ylim) ||
        !HK_CHECK(p.st, crow * p.C + p.C <= p.colsum_len, 8, crow * p.C + p.C, p.colsum_len))
      active = false;
  }
#endif
  uint32_t c0[UC], c1[UC], c2[UC];
#pragma unroll
  for (int m = 0; m < UC; m++) c0[m] = c1[m] = c2[m] = 0;

  int s = 0, rnd = 0;  // stage of `it` and how often the ring has wrapped
  for (int it = 0; it < nt; it++, s = (s + 1 == NS) ? 0 : s + 1, rnd += (s == 0)) {
    if (!mbar_wait(&full[s], rnd & 1, wlim)) {
      if (lane == 0) raise_timeout(p.st);
      *abort_flag = 1;
      break;
    }
    if (*abort_flag) break;
    const uint32_t *X = bufs + (size_t)s * (Xsz + Ysz) + xoff;
    const uint32_t *Y = bufs + (size_t)s * (Xsz + Ysz) + Xsz + YPADL + yoff;
    const int neg = sneg[s];
    if (UC == 8 && active) {
      // X read as aligned quads: two 128-bit shared loads per eight p-steps
      // (the window below stays scalar: quads at the stripes' stride of eight
      // limbs measured slower)
      uint32_t wb[UC];
#pragma unroll
      for (int m = 1; m < UC; m++) wb[m] = Y[d0 + m - p0];
      if (!neg) {
#pragma unroll 1
        for (int b = 0; b < ngrp; b++) {
          const int pb = p0 + b * UC;
          const uint4 xa = *reinterpret_cast<const uint4 *>(X + pb);
          const uint4 xb = *reinterpret_cast<const uint4 *>(X + pb + 4);
          const uint32_t xq[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
          for (int j = 0; j < UC; j++) {
            wb[(UC - j) % UC] = Y[d0 - pb - j];
#pragma unroll
            for (int m = 0; m < UC; m++) mp::mac3(c0[m], c1[m], c2[m], xq[j % 8], wb[(m - j + UC) % UC]);
          }
        }
      } else {
#pragma unroll 1
        for (int b = 0; b < ngrp; b++) {
          const int pb = p0 + b * UC;
          const uint4 xa = *reinterpret_cast<const uint4 *>(X + pb);
          const uint4 xb = *reinterpret_cast<const uint4 *>(X + pb + 4);
          const uint32_t xq[8] = {xa.x, xa.y, xa.z, xa.w, xb.x, xb.y, xb.z, xb.w};
#pragma unroll
          for (int j = 0; j < UC; j++) {
            wb[(UC - j) % UC] = Y[d0 - pb - j];
#pragma unroll
            for (int m = 0; m < UC; m++) mp::msub3(c0[m], c1[m], c2[m], xq[j % 8], wb[(m - j + UC) % UC]);
          }
        }
      }
    } else if (active) {
      uint32_t wb[UC];
#pragma unroll
      for (int m = 1; m < UC; m++) wb[m] = Y[d0 + m - p0];
      if (!neg) {
#pragma unroll 1
        for (int b = 0; b < p.upc / UC; b++) {
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
        for (int b = 0; b < p.upc / UC; b++) {
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
  // at every (offset, sign) term of the sub-problem
  long long v[UC + 2];
#pragma unroll
  for (int m = 0; m < UC + 2; m++) {
    long long x = 0;
    if (m < UC) x += (long long)c0[m];
    if (m >= 1 && m <= UC) x += (long long)c1[m - 1];
    if (m >= 2) x += (long long)(int32_t)c2[m - 2];
    v[m] = x;
  }
  const int nterm = p.sub[sp].nterm;
  for (int k = 0; k < nterm; k++) {
    const int base = d0 + p.sub[sp].toff[k];
    const long long sg = p.sub[sp].tsign[k];
    unsigned long long *dst = reinterpret_cast<unsigned long long *>(p.colsum + crow * p.C + base);
    const int lim = p.C - base;
#pragma unroll
    for (int m = 0; m < UC + 2; m++)
      if (v[m] != 0 && m < lim) atomicAdd(dst + m, (unsigned long long)(sg * v[m]));
  }
}

// Failure-detection self-test: one block arms an mbarrier for a transaction
// that never comes (no copy is issued, nothing arrives) and waits on it with
// the same bounded routine as the update kernel.  The wait runs out after the
// limit, the block records the timeout and returns; nothing hangs and no
// fault is raised.
__global__ void k_wait_selftest(DevStatus *st, long long wait_ns) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned long long lim = wait_ns > 0 ? (unsigned long long)wait_ns : WAIT_LIMIT_NS;
    if (!mbar_wait(&bar, 0, lim)) raise_timeout(st);
  }
}

}  // namespace

// ---------------------------------------------------------------------------
// host-side schedule helpers
// ---------------------------------------------------------------------------

cudaError_t allow_dynamic_smem(const void *fn) {
  static std::mutex mu;
  static std::set<std::pair<const void *, int>> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lock(mu);
  if (done.count({fn, dev})) return cudaSuccess;
  int optin = 0;
  e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  cudaFuncAttributes fa;
  e = cudaFuncGetAttributes(&fa, fn);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, optin - (int)fa.sharedSizeBytes);
  if (e != cudaSuccess) return e;
  done.insert({fn, dev});
  return cudaSuccess;
}

void kar_layout(int W, int levels, int gap, KarLayout *kl) {
  KarLayout k{};
  levels = std::max(0, std::min(levels, MAX_KAR));
  if (W < 64) levels = std::min(levels, 3);  // the expansion's temporaries need W >= 64 at four levels
  k.levels = levels;
  k.W = W;
  k.G = ((gap + 3) / 4) * 4;
  // widths level by level: piece u of a level splits at (w_u + 1) / 2 into
  // pieces 3u (lo), 3u + 1 (hi) and 3u + 2 (lo + hi, one limb wider)
  std::vector<int> w{W};
  for (int lv = 1; lv <= levels; lv++) {
    std::vector<int> nw;
    for (size_t u = 0; u < w.size(); u++) {
      const int m = (w[u] + 1) / 2;
      k.ms[split_base(lv) + (int)u] = m;
      nw.push_back(m);
      nw.push_back(w[u] - m);
      nw.push_back(std::max(m, w[u] - m) + 1);
    }
    w.swap(nw);
  }
  const int n = (int)w.size();
  k.npieces = n;
  int off = k.G;
  for (int i = 0; i < n; i++) {
    k.w[i] = w[i];
    k.off[i] = off;
    off += ((w[i] + 3) / 4) * 4 + k.G;
  }
  k.stride = ((off + 3) / 4) * 4;
  *kl = k;
}

// Coefficients of the Karatsuba combination: the contraction of the lo, hi or
// lo+hi pieces of a split at m is added at these offsets (limbs) and signs.
static int coef(int which, int m, int *off, int *sg) {
  if (which == 0) {  // lo*lo: +1 at 0, -1 at m
    off[0] = 0;
    sg[0] = 1;
    off[1] = m;
    sg[1] = -1;
    return 2;
  }
  if (which == 1) {  // hi*hi: +1 at 2m, -1 at m
    off[0] = 2 * m;
    sg[0] = 1;
    off[1] = m;
    sg[1] = -1;
    return 2;
  }
  off[0] = m;  // sum*sum: +1 at m
  sg[0] = 1;
  return 1;
}

int kar_subprobs(const KarLayout &kl, SubProb *sub) {
  if (kl.levels <= 0) {
    SubProb s{};
    s.xoff = s.yoff = 0;
    s.wx = s.wy = kl.W;
    s.nterm = 1;
    s.toff[0] = 0;
    s.tsign[0] = 1;
    sub[0] = s;
    return 1;
  }
  for (int i = 0; i < kl.npieces; i++) {
    SubProb s{};
    s.xoff = s.yoff = kl.off[i];
    s.wx = s.wy = kl.w[i];
    // the terms multiply out level by level: digit d_l of the piece's path
    // picks the (offset, sign) list of its split at that level
    s.nterm = 1;
    s.toff[0] = 0;
    s.tsign[0] = 1;
    int parent = 0;  // index of the piece's ancestor within its level
    for (int lv = 1; lv <= kl.levels; lv++) {
      int div = 1;
      for (int r = lv; r < kl.levels; r++) div *= 3;
      const int digit = (i / div) % 3;
      const int m = kl.ms[split_base(lv) + parent];
      int o[2], sg[2];
      const int nc = coef(digit, m, o, sg);
      int toff[MAX_TERMS], tsign[MAX_TERMS], n = 0;
      for (int a = 0; a < s.nterm; a++)
        for (int b = 0; b < nc; b++) {
          toff[n] = s.toff[a] + o[b];
          tsign[n] = s.tsign[a] * sg[b];
          n++;
        }
      s.nterm = n;
      for (int a = 0; a < n; a++) {
        s.toff[a] = toff[a];
        s.tsign[a] = tsign[a];
      }
      parent = 3 * parent + digit;
    }
    sub[i] = s;
  }
  return kl.npieces;
}

// column sums needed: every stripe of every sub-problem, flushed two columns
// past its end, at every term offset
int colsum_width(const SubProb *sub, int nsub, int uc) {
  int c = 0;
  for (int k = 0; k < nsub; k++) {
    const int S = (sub[k].wx + sub[k].wy - 1 + uc - 1) / uc;
    for (int t = 0; t < sub[k].nterm; t++) c = std::max(c, sub[k].toff[t] + S * uc + 2);
  }
  return ((c + 3) / 4) * 4;
}

// Units in chunk-major order per sub-problem: for chunk k, consecutive
// stripes, so that the threads of a warp read X[p] at one address (or stride
// uc) and Y with stride uc (uc odd: no shared-memory bank conflicts).
int build_units(const SubProb *sub, int nsub, int uc, int upc, Unit *out, int cap) {
  int n = 0;
  for (int q = 0; q < nsub; q++) {
    const int Wx = sub[q].wx, Wy = sub[q].wy;
    const int S = (Wx + Wy - 1 + uc - 1) / uc;
    std::vector<int> plo(S), len(S);
    int kmax = 0;
    for (int s = 0; s < S; s++) {
      const int d0 = s * uc;
      int lo = std::max(0, d0 - Wy + 1);
      const int hi = std::min(Wx - 1, d0 + uc - 1);
      // stripe 8 reads X in aligned quads: start the chunks up to three limbs
      // early (those products pair X with Y past the piece, in its zero gap)
      if (uc == 8) lo &= ~3;
      plo[s] = lo;
      len[s] = hi >= lo ? hi - lo + 1 : 0;
      kmax = std::max(kmax, (len[s] + upc - 1) / upc);
    }
    if (uc != 8) {
      for (int k = 0; k < kmax; k++)
        for (int s = 0; s < S; s++)
          if (k * upc < len[s]) {
            if (out && n < cap) out[n] = Unit{(q << 24) | (s * uc), plo[s] + k * upc};
            n++;
          }
      continue;
    }
    // stripe 8: full chunks of upc p-steps, then each stripe's remainder as a
    // shorter chunk rounded up to eight steps (its length in bits 16..23 of
    // p0, in groups of eight); the remainders follow the full chunks, longest
    // first, so that the lanes of a warp mostly share one length
    for (int k = 0; k < kmax; k++)
      for (int s = 0; s < S; s++)
        if ((k + 1) * upc <= len[s]) {
          if (out && n < cap) out[n] = Unit{(q << 24) | (s * uc), (plo[s] + k * upc) | ((upc / 8) << 16)};
          n++;
        }
    for (int r = upc; r > 0; r -= 8)
      for (int s = 0; s < S; s++) {
        const int rem = len[s] % upc;
        if (rem > 0 && (rem + 7) / 8 * 8 == r) {
          if (out && n < cap) out[n] = Unit{(q << 24) | (s * uc), (plo[s] + (len[s] / upc) * upc) | ((r / 8) << 16)};
          n++;
        }
      }
  }
  if (uc == 8 && out && n <= cap) {
    // within each block (its units keep their operand window), longest units
    // first, so that a warp's lanes share one length
    for (int b0 = 0; b0 < n; b0 += UNT)
      std::stable_sort(out + b0, out + std::min(n, b0 + UNT),
                       [](const Unit &a, const Unit &b) { return ((a.p0 >> 16) & 0xff) > ((b.p0 >> 16) & 0xff); });
  }
  return n;
}

int operand_windows(const SubProb *sub, int nsub, const Unit *units, int n, int gap, int stride, int *xlo,
                    int *xlen) {
  const int nb = (n + UNT - 1) / UNT;
  if (nsub <= 1 || nb > MAX_XB || n <= 0) return 0;
  int maxlen = 0;
  for (int b = 0; b < nb; b++) {
    int lo = INT_MAX, hi = 0;
    for (int u = b * UNT; u < std::min(n, (b + 1) * UNT); u++) {
      const int q = (units[u].d0 >> 24) & 0xff;
      lo = std::min(lo, sub[q].xoff - gap);
      hi = std::max(hi, sub[q].xoff + ((sub[q].wx + 3) / 4) * 4 + gap);
    }
    lo = std::max(0, lo & ~3);
    hi = std::min(stride, (hi + 3) & ~3);
    xlo[b] = lo;
    xlen[b] = hi - lo;
    maxlen = std::max(maxlen, hi - lo);
  }
  return maxlen;
}

// Modelled cost of a schedule: thread-products per t including the idle
// threads of the last block, plus a per-unit cost (window load, stage
// bookkeeping) in slots per stripe column, over the relative limb-product
// slot rate of the stripe width.  Rates and unit cost are fitted to
// factorisation timings on GB300 (N = 1000, W = 804, two Karatsuba levels,
// seven (stripe, chunk) schedules).
static const int kUcs[4] = {7, 8, 9, 11};
static const double kSpeed[4] = {41.7, 52.8, 45.9, 45.1};
static double schedule_cost(const SubProb *sub, int nsub, int ui, int upc) {
  const int uc = kUcs[ui];
  const int n = build_units(sub, nsub, uc, upc, nullptr, 0);
  if (uc == 8) {
    // chunks of their own lengths: a warp costs its longest lane; idle
    // warps of the last block cost nothing (the other blocks of the SM fill
    // the integer pipe)
    std::vector<Unit> h(n);
    build_units(sub, nsub, uc, upc, h.data(), n);
    double slots = 0;
    for (int w0 = 0; w0 < n; w0 += 32) {
      int mx = 0;
      for (int u = w0; u < std::min(n, w0 + 32); u++) mx = std::max(mx, (h[u].p0 >> 16) & 0xff);
      slots += 32.0 * mx * 8 * uc;
    }
    return (slots + (double)n * 1.75 * uc) / kSpeed[ui];
  }
  const int blocks = (n + UNT - 1) / UNT;
  return ((double)blocks * UNT * upc * uc + (double)n * 1.75 * uc) / kSpeed[ui];
}

// Schedule: stripe width and chunk length (a multiple of it, at most upc_cap)
// of least modelled cost; chunks of one stripe width measured slower than the
// model says, so chunks start at two.  HK_UC / HK_UPC override (tuning runs).
static double best_schedule(const SubProb *sub, int nsub, int upc_cap, int *uc_out, int *upc_out) {
  int uc_force = 0, upc_force = 0;
  if (const char *e = getenv("HK_UC")) uc_force = atoi(e);
  if (const char *e = getenv("HK_UPC")) upc_force = atoi(e);
  int best_uc = UC, best_upc = 4 * UC;
  double best = 1e300;
  for (int ui = 0; ui < 4; ui++) {
    const int uc = kUcs[ui];
    if (uc_force && uc != uc_force) continue;
    for (int upc = 2 * uc; upc <= 8 * uc && upc <= upc_cap; upc += uc) {
      if (upc_force && upc != upc_force) continue;
      const double cost = schedule_cost(sub, nsub, ui, upc);
      if (cost < best) {
        best = cost;
        best_uc = uc;
        best_upc = upc;
      }
    }
  }
  *uc_out = best_uc;
  *upc_out = best_upc;
  return best;
}

void choose_schedule(const SubProb *sub, int nsub, int upc_cap, int *uc_out, int *upc_out) {
  best_schedule(sub, nsub, upc_cap, uc_out, upc_out);
}

// Shared memory of one update block for the schedule (uc, upc) of a
// Karatsuba launch: the default ring of USTAGES stages of the longest block
// operand window (as launch_uc sizes it).
static size_t staged_bytes(const SubProb *sub, int nsub, int uc, int upc, const KarLayout &kl) {
  const int n = build_units(sub, nsub, uc, upc, nullptr, 0);
  std::vector<Unit> h(n);
  build_units(sub, nsub, uc, upc, h.data(), n);
  int xlo[MAX_XB], xlen[MAX_XB];
  int len = operand_windows(sub, nsub, h.data(), n, kl.G, kl.stride, xlo, xlen);
  if (len <= 0) len = kl.stride;  // whole entries staged
  const int Xsz = ((len + xpadr(upc) + 3) / 4) * 4;
  const int Ysz = ((ypadl(uc, upc) + len + ypadr(uc) + 3) / 4) * 4;
  return (size_t)USTAGES * (Xsz + Ysz) * 4 + 2 * USTAGES * 8 + 4 * (USTAGES + 4);
}

// Karatsuba depth for a window of W limbs: the level count whose best
// schedule has the least modelled cost (the model of choose_schedule, which
// counts every thread slot of the unit grid, so narrow pieces pay for their
// idle slots and per-unit overhead).  The model sees neither the staged
// operand windows, which grow with the zero gaps between pieces, nor the
// expansion of every new entry into 81 pieces on the panel chain: four
// levels are considered only when allowed (large factorisations) and where
// three update blocks still fit an SM (about W >= 580; at W = 300 a
// four-level block would stage 114 KB).
int choose_levels(int W, int gap, bool allow4) {
  int best_lv = 0;
  double best = 1e300;
  for (int lv = 0; lv <= MAX_KAR; lv++) {
    if (lv == 4 && !allow4) break;
    KarLayout kl;
    kar_layout(W, lv, gap, &kl);
    if (kl.levels != lv) break;
    SubProb sub[MAX_SUB];
    const int nsub = kar_subprobs(kl, sub);
    int uc = 0, upc = 0;
    const double cost = best_schedule(sub, nsub, lv > 0 ? kl.G - 11 : 8 * UC_MAX, &uc, &upc);
    if (lv == 4 && staged_bytes(sub, nsub, uc, upc, kl) > 72 * 1024) break;
    if (cost < best * 0.98) {  // a deeper level must win by 2% (more expansion work per entry)
      best = cost;
      best_lv = lv;
    }
  }
  return best_lv;
}

namespace {

template <int UCT>
cudaError_t launch_uc(const UpdParams &p, cudaStream_t s) {
  const int Xsz = ((p.cx + xpadr(p.upc) + 3) / 4) * 4;
  const int Ysz = ((ypadl(UCT, p.upc) + p.cy + ypadr(UCT) + 3) / 4) * 4;
  // pipeline depth: the configured ring (HK_USTAGES, default USTAGES); a ring
  // deeper than the default shrinks (not below it) until three blocks still
  // fit in an SM's shared memory
  static const int want = [] {
    const char *e = getenv("HK_USTAGES");
    return e ? std::max(2, std::min(USTAGES_MAX, atoi(e))) : USTAGES;
  }();
  const size_t stage = (size_t)(Xsz + Ysz) * 4 + 8 * 2 + 4;
  int nst = want;
  while (nst > USTAGES && nst * stage + 64 > 72 * 1024) nst--;
  UpdParams q = p;
  q.nst = nst;
  const size_t smem = (size_t)nst * (Xsz + Ysz) * 4 + 2 * nst * 8 + 4 * (nst + 4);
  if (smem > 48 * 1024) {
    cudaError_t e = allow_dynamic_smem((const void *)k_update<UCT>);
    if (e != cudaSuccess) return e;
  }
  const int nz = (p.t1 - p.t0 + p.tchunk - 1) / p.tchunk;
  dim3 grid((p.nunits + UNT - 1) / UNT, p.nout, nz);
  k_update<UCT><<<grid, UNT + 32, smem, s>>>(q);
  const cudaError_t e = cudaGetLastError();
#ifdef HK_CHECKED
  if (e != cudaSuccess)
    fprintf(stderr, "[hk checked] k_update<%d> mode %d grid (%u,%u,%u) smem %zu cx %d cy %d uc %d upc %d nsub %d nxb %d: %s\n",
            UCT, p.mode, grid.x, grid.y, grid.z, smem, p.cx, p.cy, p.uc, p.upc, p.nsub, p.nxb, cudaGetErrorString(e));
#endif
  return e;
}

}  // namespace

cudaError_t launch_wait_selftest(DevStatus *st, long long wait_ns, cudaStream_t s) {
  k_wait_selftest<<<1, 32, 0, s>>>(st, wait_ns);
  return cudaGetLastError();
}

cudaError_t launch_update(const UpdParams &p, cudaStream_t s) {
  if (p.nout <= 0 || p.t1 <= p.t0 || p.nunits <= 0) return cudaSuccess;
  if (p.upc % p.uc != 0 || p.nsub < 1 || p.nsub > MAX_SUB) return cudaErrorInvalidValue;
  switch (p.uc) {
    case 7: return launch_uc<7>(p, s);
    case 8: return launch_uc<8>(p, s);
    case 9: return launch_uc<9>(p, s);
    case 11: return launch_uc<11>(p, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace hk
