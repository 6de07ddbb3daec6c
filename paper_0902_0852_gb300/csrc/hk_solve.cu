// Inverse iteration kernels: one entry of a triangular solve, vector
// alignment, the Rayleigh estimate and power-of-two rescaling.
//
//   forward  y_i = RNE(RNE(v_i - sum_{k<i} R_ki y_k) / R_ii)
//   back     w_i = RNE(RNE(y_i - sum_{k>i} R_ik w_k) / R_ii)
//   lambda   = RNE(RNE(<v,v>) / RNE(<v,w>))  (inverse Rayleigh quotient of M^-1;
//              section "M is extremely ill-conditioned" bounds the spectrum
//              with the Rayleigh quotient)
//   v        = w 2^-E, E = max_i (exp(w_i) + P)
// The sums arrive exactly as column sums from the update kernel (modes
// GEMV_FWD / GEMV_BACK / DOT) on a binary grid chosen by the host.
#include "hk_internal.h"
#include "hk_kar.cuh"
#include "hk_mp.cuh"

namespace hk {

namespace {

constexpr int NT_SOLVE = 512;
constexpr int NT_LAM = 512;

struct SSmem {
  mp::Red *red;
  long long *cs;
  uint32_t *tmp, *Z, *mant, *big, *q, *V, *rm, *res;
  uint32_t *nb[6];
  int cap, cap4;
};

__host__ __device__ inline size_t scarve(unsigned char *base, int L, int C, bool with_recip, SSmem *out) {
  SSmem s;
  const int a0 = C + L + 24, b0 = 4 * L + 64;
  s.cap = ((a0 > b0 ? a0 : b0) + 3) / 4 * 4;
  s.cap4 = ((4 * L + 64) + 3) / 4 * 4;
  size_t off = 0;
  auto at = [&](size_t bytes) {
    unsigned char *r = base ? base + off : nullptr;
    off += (bytes + 15) / 16 * 16;
    return r;
  };
  s.red = reinterpret_cast<mp::Red *>(at(sizeof(mp::Red)));
  s.cs = reinterpret_cast<long long *>(at(8 * (size_t)s.cap));
  auto take = [&](int n) { return reinterpret_cast<uint32_t *>(at(4 * (size_t)n)); };
  s.tmp = take(s.cap);
  s.Z = take(s.cap);
  s.mant = take(L + 8);
  s.q = take(L + 8);
  s.V = take(L + 8);
  s.rm = take(L + 8);
  s.res = take(L + 8);
  s.big = take(s.cap4);
  for (int k = 0; k < 6; k++) s.nb[k] = with_recip ? take(s.cap4) : nullptr;
  if (out) *out = s;
  return off;
}

__host__ __device__ inline size_t ssmem_size(int L, int C, bool with_recip) {
  return scarve(nullptr, L, C, with_recip, nullptr);
}

HK_DEV mp::Work swork(SSmem &s) {
  mp::Work w;
  w.cs = s.cs;
  w.tmp = s.tmp;
  w.r = s.red;
  return w;
}

// Z = (-1)^sv * v * 2^(ev - G) - colsum   (magnitude in s.Z); 0 on range failure
template <int NT>
HK_DEV int form_exact_s(SSmem &s, const long long *colrow, int C, int32_t sv, long long ev,
                        const uint32_t *vl, int L, long long G, DevStatus *st, int *nZ_out) {
  // v == 0? (each thread tests a strided part of the limbs; one barrier)
  uint32_t nzl = 0;
  for (int l = threadIdx.x; l < L; l += NT) nzl |= vl[l];
  const bool vz = __syncthreads_or(nzl != 0) == 0;
  long long sh = ev - G;
  if (vz) sh = 0;
  if (sh < 0) {
    if (threadIdx.x == 0) raise_range(st, -sh);
    return 0;
  }
  const long long q = sh >> 5;
  const int b = (int)(sh & 31);
  if (!vz && q >= C + 2) {
    // the sum (|sum| < 2^(32(C+1)), column sums below 2^63) lies more than 32
    // bits below the lowest bit of the P-bit value v, i.e. under ulp(v)/2^32:
    // RNE(v - sum) = v exactly.  Return v itself (no wide buffer needed).
    for (int l = threadIdx.x; l < L; l += NT) s.Z[l] = vl[l];
    for (int l = L + threadIdx.x; l < L + 2; l += NT) s.Z[l] = 0;
    __syncthreads();
    *nZ_out = -L;  // marker: s.Z holds v's mantissa, exponent ev
    return sv ? -1 : 1;
  }
  const int nm = vz ? 0 : (int)(q + L + 1);
  const int nZ = max(C, nm);
  if (nZ + 2 > s.cap) {
    if (threadIdx.x == 0) raise_range(st, 32LL * (nZ + 2 - s.cap));
    return 0;
  }
  for (int d = threadIdx.x; d < nZ; d += NT) {
    uint32_t mv = 0;
    if (!vz) {
      const long long li = d - q;
      const uint32_t a = mp::limb_at(vl, L, li), c = mp::limb_at(vl, L, li - 1);
      mv = b ? ((a << b) | (c >> (32 - b))) : a;
    }
    const long long cv = d < C ? colrow[d] : 0;
    s.cs[d] = (sv ? -(long long)mv : (long long)mv) - cv;
  }
  __syncthreads();
  const bool neg = mp::resolve<NT>(s.cs, nZ, s.Z, *s.red);
  *nZ_out = nZ + 2;
  return neg ? -1 : 1;
}

// one solve entry i: out_i = RNE(RNE(rhs_i - sum) / R_ii); aligned copy in vecA[i]
template <int NT>
__global__ void __launch_bounds__(NT) k_solve_entry(SolveParams p, int i) {
  if (block_status(p.st) != ST_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SSmem s;
  if (!HK_CHECK(p.st, ssmem_size(p.L, p.C, false) <= dynamic_smem_bytes(), 21, ssmem_size(p.L, p.C, false),
                dynamic_smem_bytes()) ||
      !HK_CHECK(p.st, (long long)(i - p.r0 + 1) * p.C <= p.colsum_len && i >= p.r0, 22,
                (long long)(i - p.r0 + 1) * p.C, p.colsum_len) ||
      !HK_CHECK(p.st, p.nosum || (long long)(i + 1) * p.Wv <= p.vec_len, 23, (long long)(i + 1) * p.Wv, p.vec_len))
    return;
  scarve(smem_raw, p.L, p.C, false, &s);
  mp::Work w = swork(s);
  const int L = p.L, N = p.N;
  const long long gi = p.colU[i] - 32LL * p.W;
  long long G = p.back ? p.h : gi + p.h;
  if (p.nosum) G = p.rhs.exp[i];
  const long long *colrow = p.colsum + (long long)(i - p.r0) * p.C;
  int nZ = 0;
  const int sgn = form_exact_s<NT>(s, colrow, p.C, p.rhs.sign[i], p.rhs.exp[i],
                                         p.rhs.limbs + (long long)i * L, L, G, p.st, &nZ);
  if (sgn == 0) return;
  // nZ < 0: the sum was negligible and s.Z holds the rhs mantissa itself
  const mp::Rounded S = nZ < 0 ? mp::round_rne<NT>(s.Z, L, p.rhs.exp[i], L, s.mant, w)
                               : mp::round_rne<NT>(s.Z, nZ, G, L, s.mant, w);
  uint32_t *outl = p.out.limbs + (long long)i * L;
  uint32_t *va = p.vecA + (long long)i * p.Wv;
  if (!S.nonzero) {
    for (int l = threadIdx.x; l < L; l += NT) outl[l] = 0;
    if (!p.nosum)
      for (int l = threadIdx.x; l < p.Wv; l += NT) va[l] = 0;
    if (!p.nosum && p.kl.levels > 0)
      for (int l = threadIdx.x; l < p.kl.stride; l += NT) p.vecAexp[(long long)i * p.kl.stride + l] = 0;
    if (threadIdx.x == 0) {
      p.out.sign[i] = 0;
      p.out.exp[i] = 0;
      p.vecAsign[i] = 0;
    }
    return;
  }
  const long long iidx = tri_idx(i, i, N);
  for (int l = threadIdx.x; l < L; l += NT) s.rm[l] = p.R.limbs[iidx * L + l];
  for (int l = threadIdx.x; l < recip_limbs(L); l += NT) s.V[l] = p.recip[(long long)i * recip_limbs(L) + l];
  __syncthreads();
  bool ok = true;
  const mp::Rounded Q =
      mp::div_rne<NT>(s.mant, S.exp, s.rm, p.R.exp[iidx], s.V, L, s.res, w, s.big, s.q, &ok, RECIP_EXTRA);
  for (int l = threadIdx.x; l < L; l += NT) outl[l] = s.res[l];
  if (threadIdx.x == 0) {
    p.out.sign[i] = sgn < 0 ? 1 : 0;
    p.out.exp[i] = Q.exp;
    p.vecAsign[i] = sgn < 0 ? 1 : 0;
    if (!ok) atomicAdd(&p.st->timeout, 1);
  }
  // aligned copy on grid h; in the back solve the entry is scaled by 2^g_i
  if (p.nosum) return;
  const long long e = Q.exp + (p.back ? gi : 0);
  const long long sh = e - p.h;
  const long long P = 32LL * L;
  if (sh < 0 || sh + P > 32LL * p.Wv) {
    if (threadIdx.x == 0) raise_range(p.st, sh < 0 ? -sh : sh + P - 32LL * p.Wv);
    return;
  }
  mp::shl<NT>(s.res, L, sh, va, p.Wv);
  if (p.kl.levels > 0) {
    __syncthreads();
    expand_entry<NT>(va, p.kl, p.vecAexp + (long long)i * p.kl.stride, s.cs, s.Z, s.big, *s.red);
  }
}

// A whole block of solve rows in one launch (low precision, where the per-row
// launches dominate): rows [B0, B1) in solve order, each
//   out_i = RNE(RNE(rhs_i - colsum_i - sum_{k earlier in the block} R.. y_k) / R_ii)
// with colsum_i the exact sum over the earlier blocks (one GEMV launch) and the
// in-block terms computed here, exactly, from the block's aligned entries kept
// in shared memory.  Same arithmetic as k_solve_entry + the in-block updates.
struct BlockSmem {
  uint32_t *Ys, *Xs;        // aligned in-block entries [nb][Wv]; staged R entries [nb][W]
  int *Ysg, *Xsg;           // their signs
  long long *cs2;           // in-block column sums [W + Wv + 4]
};

__host__ __device__ inline size_t block_smem_size(int L, int C, int W, int Wv, int nb, BlockSmem *out,
                                                  unsigned char *base) {
  size_t off = (scarve(nullptr, L, C, false, nullptr) + 15) / 16 * 16;
  auto at = [&](size_t bytes) {
    unsigned char *r = base ? base + off : nullptr;
    off += (bytes + 15) / 16 * 16;
    return r;
  };
  BlockSmem b;
  b.Ys = reinterpret_cast<uint32_t *>(at(4 * (size_t)nb * Wv));
  b.Xs = reinterpret_cast<uint32_t *>(at(4 * (size_t)nb * W));
  b.Ysg = reinterpret_cast<int *>(at(4 * (size_t)nb));
  b.Xsg = reinterpret_cast<int *>(at(4 * (size_t)nb));
  b.cs2 = reinterpret_cast<long long *>(at(8 * (size_t)(W + Wv + 4)));
  if (out) *out = b;
  return off;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_solve_block(SolveParams p, const uint32_t *A, const int32_t *Asign,
                                                          int B0, int B1) {
  if (block_status(p.st) != ST_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int L = p.L, N = p.N, W = p.W, Wv = p.Wv, nb = B1 - B0;
  if (!HK_CHECK(p.st, block_smem_size(L, p.C, W, Wv, nb, nullptr, nullptr) <= dynamic_smem_bytes(), 24,
                block_smem_size(L, p.C, W, Wv, nb, nullptr, nullptr), dynamic_smem_bytes()) ||
      !HK_CHECK(p.st, (long long)nb * p.C <= p.colsum_len && p.C >= W + Wv + 4, 25, (long long)nb * p.C,
                p.colsum_len))
    return;
  SSmem s;
  scarve(smem_raw, L, p.C, false, &s);
  BlockSmem b;
  block_smem_size(L, p.C, W, Wv, nb, &b, smem_raw);
  mp::Work w = swork(s);
  const long long P = 32LL * L;
  const int ncol = W + Wv + 2;
  for (int step = 0; step < nb; step++) {
    const int i = p.back ? B1 - 1 - step : B0 + step;
    // in-block terms: sum over the earlier entries k of this block of R y_k
    // (forward: R_ki on column i's grid; back: R_ik on column k's grid, with
    // y_k scaled by 2^g_k), exact, as column sums on the row's grid
    for (int d = threadIdx.x; d < ncol + 2; d += NT) b.cs2[d] = 0;
    for (int q = 0; q < step; q++) {
      const int k = p.back ? B1 - 1 - q : B0 + q;
      const long long aidx = p.back ? tri_idx(i, k, N) : tri_idx(k, i, N);
      for (int l = threadIdx.x; l < W; l += NT) b.Xs[q * W + l] = A[aidx * W + l];
      if (threadIdx.x == 0) b.Xsg[q] = Asign[aidx] ^ b.Ysg[q];
    }
    __syncthreads();
    if (step > 0) {
      unsigned long long *cu = reinterpret_cast<unsigned long long *>(b.cs2);
      for (int d = threadIdx.x; d < W + Wv - 1; d += NT) {
        uint32_t p0 = 0, p1 = 0, p2 = 0, n0 = 0, n1 = 0, n2 = 0;
        const int plo = max(0, d - Wv + 1), phi = min(W - 1, d);
        for (int q = 0; q < step; q++) {
          const uint32_t *X = b.Xs + q * W, *Y = b.Ys + q * Wv;
          if (b.Xsg[q]) {
            for (int pp = plo; pp <= phi; pp++) mp::mac3(n0, n1, n2, X[pp], Y[d - pp]);
          } else {
            for (int pp = plo; pp <= phi; pp++) mp::mac3(p0, p1, p2, X[pp], Y[d - pp]);
          }
        }
        // positive minus negative words, added at columns d, d+1, d+2
        const long long v0 = (long long)p0 - (long long)n0, v1 = (long long)p1 - (long long)n1,
                        v2 = (long long)p2 - (long long)n2;
        if (v0) atomicAdd(cu + d, (unsigned long long)v0);
        if (v1) atomicAdd(cu + d + 1, (unsigned long long)v1);
        if (v2) atomicAdd(cu + d + 2, (unsigned long long)v2);
      }
      __syncthreads();
    }
    // the entry itself (as k_solve_entry, with the in-block sums added)
    const long long gi = p.colU[i] - 32LL * W;
    long long G = p.back ? p.h : gi + p.h;
    if (p.nosum) G = p.rhs.exp[i];
    const long long *colrow = p.colsum + (long long)(i - p.r0) * p.C;
    const uint32_t *vl = p.rhs.limbs + (long long)i * L;
    uint32_t nzl = 0;
    for (int l = threadIdx.x; l < L; l += NT) nzl |= vl[l];
    const bool vz = __syncthreads_or(nzl != 0) == 0;
    long long sh0 = p.rhs.exp[i] - G;
    if (vz) sh0 = 0;
    if (sh0 < 0) {
      if (threadIdx.x == 0) raise_range(p.st, -sh0);
      return;
    }
    const long long q0 = sh0 >> 5;
    const int b0 = (int)(sh0 & 31);
    const bool small_sum = !vz && q0 >= max(p.C, ncol + 2) + 2;  // RNE(v - sum) = v exactly
    const int nm = vz ? 0 : (int)(q0 + L + 1);
    const int nZ0 = small_sum ? L : max(p.C, nm);
    if (!small_sum && nZ0 + 2 > s.cap) {
      if (threadIdx.x == 0) raise_range(p.st, 32LL * (nZ0 + 2 - s.cap));
      return;
    }
    const int32_t sv = p.rhs.sign[i];
    for (int d = threadIdx.x; d < nZ0; d += NT) {
      if (small_sum) {
        s.cs[d] = (long long)vl[d];  // the rhs mantissa itself
        continue;
      }
      uint32_t mv = 0;
      if (!vz) {
        const long long li = d - q0;
        const uint32_t a = mp::limb_at(vl, L, li), c = mp::limb_at(vl, L, li - 1);
        mv = b0 ? ((a << b0) | (c >> (32 - b0))) : a;
      }
      const long long cv = (d < p.C ? colrow[d] : 0) + (d < ncol + 2 ? b.cs2[d] : 0);
      s.cs[d] = (sv ? -(long long)mv : (long long)mv) - cv;
    }
    __syncthreads();
    const bool neg = small_sum ? sv != 0 : mp::resolve<NT>(s.cs, nZ0, s.Z, *s.red);
    if (small_sum) {
      for (int l = threadIdx.x; l < L + 2; l += NT) s.Z[l] = l < L ? vl[l] : 0;
      __syncthreads();
    }
    const int sgn = neg ? -1 : 1;
    const mp::Rounded S = small_sum ? mp::round_rne<NT>(s.Z, L, p.rhs.exp[i], L, s.mant, w)
                                    : mp::round_rne<NT>(s.Z, nZ0 + 2, G, L, s.mant, w);
    uint32_t *outl = p.out.limbs + (long long)i * L;
    uint32_t *ya = b.Ys + step * Wv;
    if (!S.nonzero) {
      for (int l = threadIdx.x; l < L; l += NT) outl[l] = 0;
      for (int l = threadIdx.x; l < Wv; l += NT) ya[l] = 0;
      if (threadIdx.x == 0) {
        p.out.sign[i] = 0;
        p.out.exp[i] = 0;
        b.Ysg[step] = 0;
      }
      __syncthreads();
      continue;
    }
    const long long iidx = tri_idx(i, i, N);
    for (int l = threadIdx.x; l < L; l += NT) s.rm[l] = p.R.limbs[iidx * L + l];
    for (int l = threadIdx.x; l < recip_limbs(L); l += NT) s.V[l] = p.recip[(long long)i * recip_limbs(L) + l];
    __syncthreads();
    bool ok = true;
    const mp::Rounded Q =
        mp::div_rne<NT>(s.mant, S.exp, s.rm, p.R.exp[iidx], s.V, L, s.res, w, s.big, s.q, &ok, RECIP_EXTRA);
    for (int l = threadIdx.x; l < L; l += NT) outl[l] = s.res[l];
    if (threadIdx.x == 0) {
      p.out.sign[i] = sgn < 0 ? 1 : 0;
      p.out.exp[i] = Q.exp;
      b.Ysg[step] = sgn < 0 ? 1 : 0;
      if (!ok) atomicAdd(&p.st->timeout, 1);
    }
    // aligned copy (shared memory only: later blocks re-align from `out`)
    if (step + 1 < nb && !p.nosum) {
      const long long sh = Q.exp + (p.back ? gi : 0) - p.h;
      if (sh < 0 || sh + P > 32LL * Wv) {
        if (threadIdx.x == 0) raise_range(p.st, sh < 0 ? -sh : sh + P - 32LL * Wv);
        return;
      }
      mp::shl<NT>(s.res, L, sh, ya, Wv);
    }
    __syncthreads();
  }
}

// Karatsuba expansion of aligned vector entries (one block per entry)
constexpr int NT_EXP = 128;
__global__ void __launch_bounds__(NT_EXP) k_vec_expand(int n0, const uint32_t *vecA, KarLayout kl, uint32_t *dst) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int k = n0 + blockIdx.x;
  const int h1 = kl.W / 2 + 8;  // level-1 sum width + normalize room
  mp::Red *red = reinterpret_cast<mp::Red *>(smem_raw);
  long long *cs = reinterpret_cast<long long *>(smem_raw + ((sizeof(mp::Red) + 15) / 16) * 16);
  uint32_t *t1 = reinterpret_cast<uint32_t *>(cs + h1);
  uint32_t *t2 = t1 + h1;
  expand_entry<NT_EXP>(vecA + (long long)k * kl.W, kl, dst + (long long)k * kl.stride, cs, t1, t2, *red);
}

// min lsb exponent and max top exponent over the nonzero entries [0, n)
// (optionally scaled by 2^g_k, g_k = colU[k] - 32 W passed as off)
__global__ void k_vec_exprange(int n, MpArr v, int L, const long long *off, long long *out2) {
  __shared__ long long lo_s[32], hi_s[32];
  long long lo = LLONG_MAX, hi = LLONG_MIN;
  const long long P = 32LL * L;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    bool nz = false;
    for (int l = 0; l < L && !nz; l++) nz = v.limbs[(long long)k * L + l] != 0;
    if (!nz) continue;
    const long long e = v.exp[k] + (off ? off[k] : 0);
    lo = min(lo, e);
    hi = max(hi, e + P);
  }
  for (int o = 16; o; o >>= 1) {
    lo = min(lo, (long long)__shfl_xor_sync(0xffffffffu, lo, o));
    hi = max(hi, (long long)__shfl_xor_sync(0xffffffffu, hi, o));
  }
  if ((threadIdx.x & 31) == 0) {
    lo_s[threadIdx.x >> 5] = lo;
    hi_s[threadIdx.x >> 5] = hi;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < (int)(blockDim.x >> 5); w++) {
      lo = min(lo, lo_s[w]);
      hi = max(hi, hi_s[w]);
    }
    out2[0] = lo;
    out2[1] = hi;
  }
}

// vecA[k] = v_k * 2^(e_k + off_k - h) as Wv limbs, k in [n0, n1) (one block per entry)
__global__ void k_vec_align(int n0, MpArr v, int L, const long long *off, long long h, int Wv,
                            uint32_t *vecA, int32_t *vecAsign, DevStatus *st, long long vec_len) {
  const int k = n0 + blockIdx.x;
  if (!HK_CHECK(st, (long long)(k + 1) * Wv <= vec_len, 41, (long long)(k + 1) * Wv, vec_len)) return;
  const uint32_t *src = v.limbs + (long long)k * L;
  uint32_t *dst = vecA + (long long)k * Wv;
  __shared__ int nz_s;
  if (threadIdx.x == 0) nz_s = 0;
  __syncthreads();
  for (int l = threadIdx.x; l < L; l += blockDim.x)
    if (src[l]) nz_s = 1;
  __syncthreads();
  if (!nz_s) {
    for (int l = threadIdx.x; l < Wv; l += blockDim.x) dst[l] = 0;
    if (threadIdx.x == 0) vecAsign[k] = 0;
    return;
  }
  const long long P = 32LL * L;
  const long long sh = v.exp[k] + (off ? off[k] : 0) - h;
  if (sh < 0 || sh + P > 32LL * Wv) {
    if (threadIdx.x == 0) raise_range(st, sh < 0 ? -sh : sh + P - 32LL * Wv);
    return;
  }
  const long long q = sh >> 5;
  const int b = (int)(sh & 31);
  for (int l = threadIdx.x; l < Wv; l += blockDim.x) {
    const uint32_t a = mp::limb_at(src, L, l - q), c = mp::limb_at(src, L, l - q - 1);
    dst[l] = b ? ((a << b) | (c >> (32 - b))) : a;
  }
  if (threadIdx.x == 0) vecAsign[k] = v.sign[k];
}

// lambda = RNE(RNE(vv 2^(2 hv)) / RNE(vw 2^(hv + hw))) from the two DOT outputs
__global__ void __launch_bounds__(NT_LAM) k_lambda(int L, const long long *colsum, int C, long long hv,
                                                   long long hw, MpArr lam, int slot, DevStatus *st,
                                                   long long colsum_len) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SSmem s;
  if (!HK_CHECK(st, ssmem_size(L, C, true) <= dynamic_smem_bytes(), 31, ssmem_size(L, C, true),
                dynamic_smem_bytes()) ||
      !HK_CHECK(st, 2LL * C <= colsum_len, 32, 2LL * C, colsum_len))
    return;
  scarve(smem_raw, L, C, true, &s);
  mp::Work w = swork(s);
  // RNE(<v,w>) -> s.rm (divisor)
  for (int d = threadIdx.x; d < C; d += NT_LAM) s.cs[d] = colsum[C + d];
  __syncthreads();
  const bool vwneg = mp::resolve<NT_LAM>(s.cs, C, s.Z, *s.red);
  const mp::Rounded VW = mp::round_rne<NT_LAM>(s.Z, C + 2, hv + hw, L, s.rm, w);
  if (!VW.nonzero || vwneg) {
    if (threadIdx.x == 0) {
      atomicMin(&st->bad_row, -1);
      atomicCAS(&st->code, ST_OK, ST_NOT_PD);
    }
    return;
  }
  // RNE(<v,v>) -> s.mant
  for (int d = threadIdx.x; d < C; d += NT_LAM) s.cs[d] = colsum[d];
  __syncthreads();
  mp::resolve<NT_LAM>(s.cs, C, s.Z, *s.red);
  const mp::Rounded VV = mp::round_rne<NT_LAM>(s.Z, C + 2, 2 * hv, L, s.mant, w);
  mp::NBufs B;
  for (int t = 0; t < 6; t++) (&B.a)[t] = s.nb[t];
  B.cap = s.cap4;
  bool ok = mp::recip<NT_LAM>(s.rm, L, s.V, w, B, RECIP_EXTRA);
  bool ok2 = true;
  const mp::Rounded Q = mp::div_rne<NT_LAM>(s.mant, VV.exp, s.rm, VW.exp, s.V, L, s.res, w, s.big, s.q, &ok2, RECIP_EXTRA);
  for (int l = threadIdx.x; l < L; l += NT_LAM) lam.limbs[(long long)slot * L + l] = s.res[l];
  if (threadIdx.x == 0) {
    lam.sign[slot] = 0;
    lam.exp[slot] = Q.exp;
    if (!ok || !ok2) atomicAdd(&st->timeout, 1);
  }
}

// v = w * 2^-E with E = max_k (exp(w_k) + P) over nonzero w_k; single block
__global__ void k_vec_normalise(int n, MpArr w, MpArr v, int L) {
  __shared__ long long red[32];
  const long long P = 32LL * L;
  long long E = LLONG_MIN;
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    bool nz = false;
    for (int l = 0; l < L && !nz; l++) nz = w.limbs[(long long)k * L + l] != 0;
    if (nz) E = max(E, w.exp[k] + P);
  }
  for (int o = 16; o; o >>= 1) E = max(E, (long long)__shfl_xor_sync(0xffffffffu, E, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = E;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int q = 1; q < (int)(blockDim.x >> 5); q++) E = max(E, red[q]);
    red[0] = E == LLONG_MIN ? 0 : E;
  }
  __syncthreads();
  E = red[0];
  for (long long x = threadIdx.x; x < (long long)n * L; x += blockDim.x) v.limbs[x] = w.limbs[x];
  for (int k = threadIdx.x; k < n; k += blockDim.x) {
    bool nz = false;
    for (int l = 0; l < L && !nz; l++) nz = w.limbs[(long long)k * L + l] != 0;
    v.sign[k] = nz ? w.sign[k] : 0;
    v.exp[k] = nz ? w.exp[k] - E : 0;
  }
}

__global__ void k_set_ones(int n, MpArr v, int L) {
  const long long P = 32LL * L;
  for (long long x = blockIdx.x * blockDim.x + threadIdx.x; x < (long long)n * L; x += gridDim.x * blockDim.x) {
    const int l = (int)(x % L);
    v.limbs[x] = (l == L - 1) ? 0x80000000u : 0u;
  }
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    v.sign[k] = 0;
    v.exp[k] = -(P - 1);
  }
}

cudaError_t set_smem(const void *fn, size_t bytes) {
  return bytes > 48 * 1024 ? allow_dynamic_smem(fn) : cudaSuccess;
}

}  // namespace

// the single-CTA solve kernels run NT_SOLVE threads (fewer threads measured
// slower at every precision: the work of an entry is parallel over its result
// columns)
cudaError_t launch_solve_entry(const SolveParams &p, int i, cudaStream_t s) {
  const size_t smem = ssmem_size(p.L, p.C, false);
  cudaError_t e = set_smem((const void *)k_solve_entry<NT_SOLVE>, smem);
  if (e != cudaSuccess) return e;
  k_solve_entry<NT_SOLVE><<<1, NT_SOLVE, smem, s>>>(p, i);
  return cudaGetLastError();
}

size_t solve_block_smem(int L, int C, int W, int Wv, int nb) {
  return block_smem_size(L, C, W, Wv, nb, nullptr, nullptr);
}

cudaError_t launch_solve_block(const SolveParams &p, const uint32_t *A, const int32_t *Asign, int B0, int B1,
                               cudaStream_t s) {
  const size_t smem = block_smem_size(p.L, p.C, p.W, p.Wv, B1 - B0, nullptr, nullptr);
  cudaError_t e = set_smem((const void *)k_solve_block<NT_SOLVE>, smem);
  if (e != cudaSuccess) return e;
  k_solve_block<NT_SOLVE><<<1, NT_SOLVE, smem, s>>>(p, A, Asign, B0, B1);
  return cudaGetLastError();
}

cudaError_t launch_vec_exprange(int n, MpArr v, int L, const long long *off, int scaled, long long *out2,
                                cudaStream_t s) {
  k_vec_exprange<<<1, 256, 0, s>>>(n, v, L, scaled ? off : nullptr, out2);
  return cudaGetLastError();
}

cudaError_t launch_vec_align(int n0, int n1, MpArr v, int L, const long long *off, int scaled, long long h,
                             int Wv, uint32_t *vecA, int32_t *vecAsign, DevStatus *st, long long vec_len,
                             cudaStream_t s) {
  if (n1 <= n0) return cudaSuccess;
  k_vec_align<<<n1 - n0, 128, 0, s>>>(n0, v, L, scaled ? off : nullptr, h, Wv, vecA, vecAsign, st, vec_len);
  return cudaGetLastError();
}

cudaError_t launch_lambda(int L, const long long *colsum, int C, long long hv, long long hw, MpArr lam,
                          int slot, DevStatus *st, long long colsum_len, cudaStream_t s) {
  const size_t smem = ssmem_size(L, C, true);
  cudaError_t e = set_smem((const void *)k_lambda, smem);
  if (e != cudaSuccess) return e;
  k_lambda<<<1, NT_LAM, smem, s>>>(L, colsum, C, hv, hw, lam, slot, st, colsum_len);
  return cudaGetLastError();
}

cudaError_t launch_vec_normalise(int n, MpArr w, MpArr v, int L, cudaStream_t s) {
  k_vec_normalise<<<1, 1024, 0, s>>>(n, w, v, L);
  return cudaGetLastError();
}

cudaError_t launch_vec_expand(int n0, int n1, const uint32_t *vecA, const KarLayout &kl, uint32_t *dst,
                              cudaStream_t s) {
  if (n1 <= n0) return cudaSuccess;
  const int h1 = kl.W / 2 + 8;
  const size_t smem = ((sizeof(mp::Red) + 15) / 16) * 16 + (size_t)h1 * 8 + (size_t)h1 * 4 * 2;
  cudaError_t e = set_smem((const void *)k_vec_expand, smem);
  if (e != cudaSuccess) return e;
  k_vec_expand<<<n1 - n0, NT_EXP, smem, s>>>(n0, vecA, kl, dst);
  return cudaGetLastError();
}

cudaError_t launch_set_ones(int n, MpArr v, int L, cudaStream_t s) {
  k_set_ones<<<64, 256, 0, s>>>(n, v, L);
  return cudaGetLastError();
}

}  // namespace hk
