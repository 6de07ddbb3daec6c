// Device multiprecision library: exact big-integer operations executed by one
// thread block (CTA) cooperatively on numbers held in shared memory.
//
// Numbers are little-endian arrays of 32-bit limbs.  Signed intermediate
// values are formed as signed 64-bit "column sums" cs[d] (value
// sum_d cs[d] 2^(32 d)) and resolved into limbs by `normalize`, a carry
// look-ahead over carries in {-1, 0, +1}: every thread owns a contiguous run of
// limbs, composes the carry-transfer functions of its run, and a block-wide
// scan (warp shuffles, then one warp over the warp totals) gives each run its
// carry-in.  Products use product scanning: one thread per output column sums
// the 64-bit limb products of that column exactly in three 32-bit words
// (mad.lo.cc / madc.hi.cc / addc), then the columns are resolved as above.
//
// Division and square root are correctly rounded: Newton iterations with
// precision doubling produce an approximation, an exact remainder then fixes
// it to the floor, and the remainder supplies the sticky bit of the rounding.
#pragma once
#include "hk_common.cuh"
#include <climits>

namespace hk {
namespace mp {

constexpr unsigned FULL = 0xffffffffu;

// (c0, c1, c2) += a * b  -- exact 96-bit accumulation of one limb product
HK_DEV void mac3(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t a, uint32_t b) {
  asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
      "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
      "addc.u32 %2, %2, 0;"
      : "+r"(c0), "+r"(c1), "+r"(c2) : "r"(a), "r"(b));
}

// (c0, c1, c2) -= a * b  (96-bit two's complement)
HK_DEV void msub3(uint32_t &c0, uint32_t &c1, uint32_t &c2, uint32_t a, uint32_t b) {
  uint32_t lo, hi;
  asm("mul.lo.u32 %3, %5, %6;\n\t"
      "mul.hi.u32 %4, %5, %6;\n\t"
      "sub.cc.u32 %0, %0, %3;\n\t"
      "subc.cc.u32 %1, %1, %4;\n\t"
      "subc.u32 %2, %2, 0;"
      : "+r"(c0), "+r"(c1), "+r"(c2), "=r"(lo), "=r"(hi) : "r"(a), "r"(b));
}

// ---- carry-transfer functions ---------------------------------------------
// f maps a carry-in in {-1, 0, 1} to a carry-out in {-1, 0, 1}; stored as three
// 2-bit fields holding (value + 1), field c+1 for carry-in c.
constexpr unsigned FID = 0u | (1u << 2) | (2u << 4);

// transfer function of one limb digit y in [-1, 2^32]
HK_DEV unsigned fdig(long long y) {
  unsigned f = 0;
#pragma unroll
  for (int c = -1; c <= 1; c++) {
    long long v = y + c;
    int co = v < 0 ? -1 : (int)(v >> 32);
    f |= (unsigned)(co + 1) << (2 * (c + 1));
  }
  return f;
}
HK_DEV int fapply(unsigned f, int c) { return (int)((f >> (2 * (c + 1))) & 3u) - 1; }
// g after f
HK_DEV unsigned fcompose(unsigned g, unsigned f) {
  unsigned r = 0;
#pragma unroll
  for (int c = 0; c < 3; c++) {
    unsigned fv = (f >> (2 * c)) & 3u;
    r |= ((g >> (2 * fv)) & 3u) << (2 * c);
  }
  return r;
}

// block-wide reduction / scan scratch (shared memory)
struct Red {
  long long v[33];
  unsigned f[33];
};

template <int NT>
HK_DEV long long cta_max(long long x, Red &r) {
  static_assert(NT % 32 == 0 && NT <= 1024, "block size");
#pragma unroll
  for (int o = 16; o; o >>= 1) x = max(x, (long long)__shfl_xor_sync(FULL, x, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) r.v[w] = x;
  __syncthreads();
  if (w == 0) {
    long long y = l < NT / 32 ? r.v[l] : LLONG_MIN;
#pragma unroll
    for (int o = 16; o; o >>= 1) y = max(y, (long long)__shfl_xor_sync(FULL, y, o));
    if (l == 0) r.v[32] = y;
  }
  __syncthreads();
  return r.v[32];
}

template <int NT>
HK_DEV unsigned cta_or(unsigned x, Red &r) {
  x = __reduce_or_sync(FULL, x);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) r.f[w] = x;
  __syncthreads();
  if (w == 0) {
    unsigned y = l < NT / 32 ? r.f[l] : 0u;
    y = __reduce_or_sync(FULL, y);
    if (l == 0) r.f[32] = y;
  }
  __syncthreads();
  return r.f[32];
}

// exclusive scan of carry-transfer functions in thread order: returns the
// composition of the functions of all lower threads (identity for thread 0)
template <int NT>
HK_DEV unsigned cta_excl_fn(unsigned F, Red &r) {
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  unsigned inc = F;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    unsigned other = __shfl_up_sync(FULL, inc, o);
    if (l >= o) inc = fcompose(inc, other);
  }
  __syncthreads();
  if (l == 31) r.f[w] = inc;
  __syncthreads();
  if (w == 0) {
    unsigned wt = l < NT / 32 ? r.f[l] : FID;
    unsigned winc = wt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      unsigned other = __shfl_up_sync(FULL, winc, o);
      if (l >= o) winc = fcompose(winc, other);
    }
    unsigned wex = __shfl_up_sync(FULL, winc, 1);
    if (l == 0) wex = FID;
    if (l < NT / 32) r.f[l] = wex;
  }
  __syncthreads();
  unsigned lex = __shfl_up_sync(FULL, inc, 1);
  if (l == 0) lex = FID;
  return fcompose(lex, r.f[w]);
}

// ---- limb access -------------------------------------------------------------
HK_DEV uint32_t limb_at(const uint32_t *x, int n, long long i) {
  return (i >= 0 && i < n) ? x[i] : 0u;
}
HK_DEV long long cs_at(const long long *cs, int n, int x) {
  return (x >= 0 && x < n) ? cs[x] : 0;
}
HK_DEV long long tdig(const long long *cs, int n, int x) {
  if (x < 0) return 0;
  const long long a = cs_at(cs, n, x), b = cs_at(cs, n, x - 1);
  return (long long)(uint32_t)a + (b >> 32);
}
HK_DEV long long ydig(const long long *cs, int n, int d) {
  const long long t = tdig(cs, n, d), tm = tdig(cs, n, d - 1);
  return (long long)(uint32_t)t + (tm >> 32);
}

// Resolve column sums cs[0..n) into n+2 limbs of two's complement in out.
// Requires |value| < 2^(32(n+1)).  Returns true when the value is negative.
template <int NT>
HK_DEV bool normalize(const long long *cs, int n, uint32_t *out, Red &r) {
  const int m = n + 2;
  const int k = (m + NT - 1) / NT;
  const int lo = threadIdx.x * k, hi = min(lo + k, m);
  unsigned F = FID;
  for (int d = lo; d < hi; d++) F = fcompose(fdig(ydig(cs, n, d)), F);
  const unsigned pre = cta_excl_fn<NT>(F, r);
  int c = fapply(pre, 0);
  for (int d = lo; d < hi; d++) {
    const long long v = ydig(cs, n, d) + c;
    out[d] = (uint32_t)v;
    c = v < 0 ? -1 : (int)(v >> 32);
  }
  __syncthreads();
  return (out[m - 1] >> 31) != 0;
}

// Magnitude and sign: out[0..n+2) = |value|; cs is negated in place when the
// value is negative.  Returns true for a negative value.
template <int NT>
HK_DEV bool resolve(long long *cs, int n, uint32_t *out, Red &r) {
  const bool neg = normalize<NT>(cs, n, out, r);
  if (neg) {
    for (int d = threadIdx.x; d < n; d += NT) cs[d] = -cs[d];
    __syncthreads();
    normalize<NT>(cs, n, out, r);
  }
  return neg;
}

// Work areas for the operations below (shared or global memory).
struct Work {
  long long *cs;            // column sums, capacity >= largest product columns + 4
  uint32_t *tmp;            // capacity >= L + 4
  Red *r;
};

// Column sums of the product x * y restricted to columns [dlo, dhi): column d
// holds sum_{p+q=d} x_p y_q.  One thread per output column sums its limb
// products exactly in three words, then adds the words into the 64-bit column
// sums of columns d, d+1, d+2 (shared-memory atomics).  cs[k] is the sum of
// column dlo + k; cs has dhi - dlo + 2 entries.
template <int NT>
HK_DEV void mul_cols(const uint32_t *x, int nx, const uint32_t *y, int ny, int dlo, int dhi, Work &w) {
  const int n = dhi - dlo;
  for (int d = threadIdx.x; d < n + 2; d += NT) w.cs[d] = 0;
  __syncthreads();
  unsigned long long *cu = reinterpret_cast<unsigned long long *>(w.cs);
  for (int k = threadIdx.x; k < n; k += NT) {
    const int d = dlo + k;
    uint32_t c0 = 0, c1 = 0, c2 = 0;
    const int plo = max(0, d - ny + 1), phi = min(nx - 1, d);
    for (int p = plo; p <= phi; p++) mac3(c0, c1, c2, x[p], y[d - p]);
    if (c0) atomicAdd(cu + k, (unsigned long long)c0);
    if (c1) atomicAdd(cu + k + 1, (unsigned long long)c1);
    if (c2) atomicAdd(cu + k + 2, (unsigned long long)c2);
  }
  __syncthreads();
}

// out[0..nx+ny+2) = x[0..nx) * y[0..ny)   (x, y >= 0); the top column holds a
// single product, so column nx+ny stays zero.
template <int NT>
HK_DEV void mul(const uint32_t *x, int nx, const uint32_t *y, int ny, uint32_t *out, Work &w) {
  const int nc = nx + ny;
  mul_cols<NT>(x, nx, y, ny, 0, nc, w);
  normalize<NT>(w.cs, nc, out, *w.r);
}

// out[0..nout) = floor(x / 2^s), s >= 0
template <int NT>
HK_DEV void shr(const uint32_t *x, int nx, long long s, uint32_t *out, int nout) {
  const long long q = s >> 5;
  const int b = (int)(s & 31);
  for (int l = threadIdx.x; l < nout; l += NT) {
    const uint32_t a = limb_at(x, nx, l + q), c = limb_at(x, nx, l + q + 1);
    out[l] = b ? ((a >> b) | (c << (32 - b))) : a;
  }
}

// out[0..nout) = x * 2^s (truncated to nout limbs), s >= 0
template <int NT>
HK_DEV void shl(const uint32_t *x, int nx, long long s, uint32_t *out, int nout) {
  const long long q = s >> 5;
  const int b = (int)(s & 31);
  for (int l = threadIdx.x; l < nout; l += NT) {
    const uint32_t a = limb_at(x, nx, l - q), c = limb_at(x, nx, l - q - 1);
    out[l] = b ? ((a << b) | (c >> (32 - b))) : a;
  }
}

template <int NT>
HK_DEV void copy(const uint32_t *x, int nx, uint32_t *out, int nout) {
  for (int l = threadIdx.x; l < nout; l += NT) out[l] = limb_at(x, nx, l);
}

// number of significant bits (0 for zero)
template <int NT>
HK_DEV long long bitlen(const uint32_t *x, int n, Red &r) {
  long long b = 0;
  for (int l = threadIdx.x; l < n; l += NT)
    if (x[l]) b = max(b, 32LL * l + 32 - __clz(x[l]));
  return cta_max<NT>(b, r);
}

HK_DEV bool bit_at(const uint32_t *x, int n, long long s) {
  return s >= 0 && ((limb_at(x, n, s >> 5) >> (s & 31)) & 1u);
}

// any set bit at positions < s
template <int NT>
HK_DEV bool any_below(const uint32_t *x, int n, long long s, Red &r) {
  unsigned f = 0;
  if (s > 0) {
    const long long full = s >> 5;
    const int b = (int)(s & 31);
    for (int l = threadIdx.x; l < n && l <= full; l += NT) {
      uint32_t v = x[l];
      if (l == full) v = b ? (v & ((1u << b) - 1u)) : 0u;
      f |= (v != 0);
    }
  }
  (void)r;
  return __syncthreads_or(f != 0) != 0;
}

// leading (up to) 64 bits of x as a double: x ~= return * 2^(*e); bl = bitlen(x)
HK_DEV double lead_double(const uint32_t *x, int n, long long bl, long long *e) {
  if (bl == 0) { *e = 0; return 0.0; }
  const long long s = bl > 64 ? bl - 64 : 0;
  const long long q = s >> 5;
  const int b = (int)(s & 31);
  const uint32_t l0 = limb_at(x, n, q), l1 = limb_at(x, n, q + 1), l2 = limb_at(x, n, q + 2);
  const unsigned long long lo = ((unsigned long long)l1 << 32) | l0;
  const unsigned long long top = b ? ((lo >> b) | ((unsigned long long)l2 << (64 - b))) : lo;
  *e = s;
  return (double)top;
}

struct Rounded {
  bool nonzero;
  long long exp;
};

// mant[0..L) , exponent = RNE_{32L}( x * 2^G ) for the magnitude x[0..n)
template <int NT>
HK_DEV Rounded round_rne(const uint32_t *x, int n, long long G, int L, uint32_t *mant, Work &w) {
  const long long P = 32LL * L;
  const long long bl = bitlen<NT>(x, n, *w.r);
  if (bl == 0) {
    for (int l = threadIdx.x; l < L; l += NT) mant[l] = 0;
    __syncthreads();
    return {false, 0};
  }
  if (bl <= P) {
    shl<NT>(x, n, P - bl, mant, L);
    __syncthreads();
    return {true, G - (P - bl)};
  }
  long long sh = bl - P;
  const bool guard = bit_at(x, n, sh - 1);
  const bool sticky = any_below<NT>(x, n, sh - 1, *w.r);
  shr<NT>(x, n, sh, mant, L);
  __syncthreads();
  const bool up = guard && (sticky || (mant[0] & 1u));
  if (up) {
    for (int l = threadIdx.x; l < L; l += NT) w.cs[l] = (long long)mant[l] + (l == 0 ? 1 : 0);
    __syncthreads();
    normalize<NT>(w.cs, L, w.tmp, *w.r);
    const bool ovf = w.tmp[L] != 0;
    for (int l = threadIdx.x; l < L; l += NT) mant[l] = ovf ? (l == L - 1 ? 0x80000000u : 0u) : w.tmp[l];
    if (ovf) sh += 1;
    __syncthreads();
  }
  return {true, G + sh};
}

// ---- Newton reciprocal --------------------------------------------------------
// Buffers for recip / isqrt: each of capacity `cap` limbs (>= 4L + 64); the
// Work column array needs the same capacity.
struct NBufs {
  uint32_t *a, *b, *c, *d, *e, *f;
  int cap;
};

// cs[0..n) = sa*x + sb*y (limbwise, x and y zero-extended), then resolve into
// out[0..n+2); returns negative?
template <int NT>
HK_DEV bool lincomb(const uint32_t *x, int nx, int sa, const uint32_t *y, int ny, int sb, int n,
                    uint32_t *out, Work &w) {
  for (int d = threadIdx.x; d < n; d += NT)
    w.cs[d] = (long long)sa * limb_at(x, nx, d) + (long long)sb * limb_at(y, ny, d);
  __syncthreads();
  return resolve<NT>(w.cs, n, out, *w.r);
}

HK_DEV int limbs_for(long long bits) { return (int)((bits + 31) >> 5); }

// V[0..L+2+extra/32) = floor(2^(2P+1+extra) / D) for D[0..L) with its top bit
// set, P = 32 L, extra a multiple of 32 (guard bits for div_rne's fast path).
// Returns false when the exact correction did not settle (never expected).
template <int NT>
HK_DEV bool recip(const uint32_t *D, int L, uint32_t *V, Work &w, NBufs &B, int extra = 0) {
  const long long P = 32LL * L;
  const long long P2 = P + extra;  // Newton target: X ~ 2^(n + P) / D at precision n
  uint32_t *X = B.a, *X0 = B.b, *Dk = B.c, *prod = B.d, *E = B.e, *corr = B.f;
  // seed: n = 32, X = floor((2^64 - 1) / top32(D)) ~ 2^64 / D32
  long long n = 32;
  if (threadIdx.x == 0) {
    const unsigned long long d32 = D[L - 1];
    const unsigned long long x = 0xffffffffffffffffull / d32;
    X[0] = (uint32_t)x;
    X[1] = (uint32_t)(x >> 32);
    X[2] = 0;
  }
  int nX = 3;
  __syncthreads();
  while (n < P2) {
    const long long n2 = min(2 * n - 8, P2);
    const int nD = limbs_for(n2), nX0 = limbs_for(n2 + 3);
    // Dk = D 2^(n2 - P): its top n2 bits (exactly D shifted up past P)
    if (n2 <= P)
      shr<NT>(D, L, P - n2, Dk, nD);
    else
      shl<NT>(D, L, n2 - P, Dk, nD);
    shl<NT>(X, nX, n2 - n, X0, nX0);
    __syncthreads();
    // only the top bits of E = 2^(2 n2) - Dk X0 matter: corr = (X0 |E|) >> 2 n2
    // with |E| ~ 2^(2 n2 - n); dropping the low se bits of E changes corr by
    // less than one unit.  The product is formed from its columns >= D0 only:
    // the dropped columns sum to less than 2^(32 D0 + 44) (at most 2^12
    // products of 64 bits per column, P <= 32768), below 2^(se - 20), which
    // moves |E| >> se by at most one more unit.
    const long long se = max(0LL, n2 - 16);
    const int D0 = max(0, (int)(se >> 5) - 2);
    const int nPr = nD + nX0;
    mul_cols<NT>(Dk, nD, X0, nX0, D0, nPr, w);
    const int nE = nPr - D0 + 2;
    // E / 2^(32 D0) = 2^(2 n2 - 32 D0) - columns
    for (int d = threadIdx.x; d < nE; d += NT) {
      long long v = -w.cs[d];
      if (d == (int)((2 * n2) >> 5) - D0) v += 1LL << ((2 * n2) & 31);
      w.cs[d] = v;
    }
    __syncthreads();
    const bool eneg = resolve<NT>(w.cs, nE, E, *w.r);
    shr<NT>(E, nE + 2, se - 32LL * D0, corr, nE + 2);
    __syncthreads();
    const long long eb = bitlen<NT>(corr, nE + 2, *w.r);
    const int nEm = max(1, limbs_for(eb));
    mul<NT>(X0, nX0, corr, nEm, prod, w);
    const int nP = nX0 + nEm + 2;
    shr<NT>(prod, nP, 2 * n2 - se, corr, nX0 + 1);
    __syncthreads();
    lincomb<NT>(X0, nX0, 1, corr, nX0 + 1, eneg ? -1 : 1, nX0 + 1, X, w);
    nX = nX0 + 1;
    n = n2;
  }
  // V0 = 2X ~ 2^(2P+1+extra)/D ; exact correction
  const int nV = L + 2 + extra / 32;
  const long long E2 = 2 * P + 1 + extra;
  shl<NT>(X, nX, 1, X0, nV);
  __syncthreads();
  bool ok = false;
  for (int it = 0; it < 6 && !ok; it++) {
    // rem = 2^E2 - D*V0
    mul<NT>(D, L, X0, nV, prod, w);
    const int nR = L + nV + 2;
    for (int d = threadIdx.x; d < nR; d += NT) {
      long long v = -(long long)prod[d];
      if (d == (int)(E2 >> 5)) v += 1LL << (E2 & 31);
      w.cs[d] = v;
    }
    __syncthreads();
    const bool rneg = resolve<NT>(w.cs, nR, E, *w.r);
    // compare |rem| with D
    const bool ge = !lincomb<NT>(E, nR, 1, D, L, -1, nR, corr, w);  // |rem| - D >= 0
    if (!rneg && !ge) { ok = true; break; }
    // estimate delta = rem / D (|delta| small), adjust V0 by it (at least 1)
    const long long rb = bitlen<NT>(E, nR, *w.r);
    long long re_, de_;
    const double rm = lead_double(E, nR, rb, &re_);
    const double dm = lead_double(D, L, P, &de_);
    double q = ldexp(rm / dm, (int)(re_ - de_));
    long long delta = (long long)floor(q);
    if (rneg) delta = -(long long)ceil(q);
    if (delta == 0) delta = rneg ? -1 : 1;
    if (delta > (1LL << 30)) delta = 1LL << 30;
    if (delta < -(1LL << 30)) delta = -(1LL << 30);
    for (int d = threadIdx.x; d < nV; d += NT) w.cs[d] = (long long)X0[d] + (d == 0 ? delta : 0);
    __syncthreads();
    normalize<NT>(w.cs, nV, corr, *w.r);
    copy<NT>(corr, nV, X0, nV);
    __syncthreads();
  }
  copy<NT>(X0, nV, V, nV);
  __syncthreads();
  return ok;
}

// X = floor(sqrt(A)) for A[0..nA) != 0, written to X[0..nX) (nX >= bits/2/32 + 2).
// Returns (via *exact) whether A is a perfect square.  False on failure.
template <int NT>
HK_DEV bool isqrt(const uint32_t *A, int nA, uint32_t *X, int nX, bool *exact, Work &w, NBufs &B) {
  uint32_t *Y = B.a, *Y0 = B.b, *A2 = B.c, *t1 = B.d, *t2 = B.e, *t3 = B.f;
  const long long ab = bitlen<NT>(A, nA, *w.r);
  const long long m = (ab + 1) / 2;  // A < 2^(2m), A >= 2^(2m-2)
  long long n;
  int nY;
  if (m <= 26) {
    n = m;
    if (threadIdx.x == 0) {
      // A < 2^52: exact enough in double; refined by the exact correction below
      const double a = (double)(((unsigned long long)limb_at(A, nA, 1) << 32) | limb_at(A, nA, 0));
      const unsigned long long y = (unsigned long long)floor(ldexp(1.0, (int)(2 * m)) / sqrt(a));
      Y[0] = (uint32_t)y;
      Y[1] = (uint32_t)(y >> 32);
      Y[2] = 0;
    }
    nY = 3;
  } else {
    n = 26;
    shr<NT>(A, nA, 2 * m - 52, t1, 2);
    __syncthreads();
    if (threadIdx.x == 0) {
      const double a = (double)(((unsigned long long)t1[1] << 32) | t1[0]);
      const unsigned long long y = (unsigned long long)floor(ldexp(1.0, 52) / sqrt(a));
      Y[0] = (uint32_t)y;
      Y[1] = (uint32_t)(y >> 32);
      Y[2] = 0;
    }
    nY = 3;
  }
  __syncthreads();
  while (n < m) {
    const long long n2 = min(2 * n - 8, m);
    const int nA2 = limbs_for(2 * n2), nY0 = limbs_for(n2 + 3);
    shr<NT>(A, nA, 2 * m - 2 * n2, A2, nA2);
    shl<NT>(Y, nY, n2 - n, Y0, nY0);
    __syncthreads();
    mul<NT>(Y0, nY0, Y0, nY0, t1, w);          // 2 nY0 + 2
    // corr = (Y0 |E|) >> (4 n2 + 1) with E = 2^(4 n2) - A2 Y0^2, |E| ~ 2^(4 n2 - n):
    // keep only the bits of E from se up; the product A2 Y0^2 is formed from its
    // columns >= D0 only (dropped part below 2^(32 D0 + 44) <= 2^(se - 20), as in recip)
    const long long se = max(0LL, 3 * n2 - 16);
    const int D0 = max(0, (int)(se >> 5) - 2);
    const int nPr = nA2 + 2 * nY0;
    mul_cols<NT>(A2, nA2, t1, 2 * nY0, D0, nPr, w);
    const int nE = nPr - D0 + 2;
    for (int d = threadIdx.x; d < nE; d += NT) {
      long long v = -w.cs[d];
      if (d == (int)((4 * n2) >> 5) - D0) v += 1LL << ((4 * n2) & 31);
      w.cs[d] = v;
    }
    __syncthreads();
    const bool eneg = resolve<NT>(w.cs, nE, t3, *w.r);
    shr<NT>(t3, nE + 2, se - 32LL * D0, t2, nE + 2);
    __syncthreads();
    const long long eb = bitlen<NT>(t2, nE + 2, *w.r);
    const int nEm = max(1, limbs_for(eb));
    mul<NT>(Y0, nY0, t2, nEm, t1, w);
    shr<NT>(t1, nY0 + nEm + 2, 4 * n2 + 1 - se, t2, nY0 + 1);
    __syncthreads();
    lincomb<NT>(Y0, nY0, 1, t2, nY0 + 1, eneg ? -1 : 1, nY0 + 1, Y, w);
    nY = nY0 + 1;
    n = n2;
  }
  // X ~ A * Y / 2^(2m), from the product's columns >= D1 (the dropped part,
  // below 2^(32 D1 + 44) <= 2^(2m - 20), moves X by at most one unit; the
  // exact correction below settles X)
  {
    const int D1 = max(0, (int)((2 * m) >> 5) - 2);
    mul_cols<NT>(A, nA, Y, nY, D1, nA + nY, w);
    normalize<NT>(w.cs, nA + nY - D1, t1, *w.r);
    shr<NT>(t1, nA + nY - D1 + 2, 2 * m - 32LL * D1, X, nX);
    __syncthreads();
  }
  bool ok = false;
  for (int it = 0; it < 8 && !ok; it++) {
    // rem = A - X^2
    mul<NT>(X, nX, X, nX, t1, w);
    const int nR = max(nA, 2 * nX + 2);
    const bool rneg = lincomb<NT>(A, nA, 1, t1, 2 * nX + 2, -1, nR, t2, w);
    // twice X plus one
    for (int d = threadIdx.x; d < nX + 1; d += NT) w.cs[d] = 2LL * limb_at(X, nX, d) + (d == 0 ? 1 : 0);
    __syncthreads();
    normalize<NT>(w.cs, nX + 1, t3, *w.r);  // 2X + 1
    if (!rneg) {
      // need rem < 2X + 1
      const bool ge = !lincomb<NT>(t2, nR + 2, 1, t3, nX + 3, -1, nR + 2, Y0, w);
      if (!ge) {
        *exact = bitlen<NT>(t2, nR + 2, *w.r) == 0;
        ok = true;
        break;
      }
    }
    // delta ~ rem / (2X), at least 1 in magnitude
    const long long rb = bitlen<NT>(t2, nR + 2, *w.r);
    const long long xb = bitlen<NT>(t3, nX + 3, *w.r);
    long long re_, xe_;
    const double rm = lead_double(t2, nR + 2, rb, &re_);
    const double xm = lead_double(t3, nX + 3, xb, &xe_);
    const double q = ldexp(rm / xm, (int)(re_ - xe_));
    long long delta = rneg ? -(long long)ceil(q) : (long long)floor(q);
    if (delta == 0) delta = rneg ? -1 : 1;
    if (delta > (1LL << 30)) delta = 1LL << 30;
    if (delta < -(1LL << 30)) delta = -(1LL << 30);
    for (int d = threadIdx.x; d < nX; d += NT) w.cs[d] = (long long)X[d] + (d == 0 ? delta : 0);
    __syncthreads();
    normalize<NT>(w.cs, nX, t1, *w.r);
    copy<NT>(t1, nX, X, nX);
    __syncthreads();
  }
  return ok;
}

// mant, exponent of RNE_P(sqrt(s * 2^e)) for a normalised P-bit s[0..L).
// Work buffers: B (capacity >= 4L + 64 each), big (capacity >= 2L + 16), xs (L + 4).
template <int NT>
HK_DEV Rounded sqrt_rne(const uint32_t *s, int L, long long e, uint32_t *mant, Work &w, NBufs &B,
                        uint32_t *big, uint32_t *xs, bool *ok) {
  const long long P = 32LL * L;
  const long long j = P / 2 + 2;
  long long e2 = e;
  long long sh = 2 * j;
  if (e & 1) { sh += 1; e2 -= 1; }
  const int nA = limbs_for(P + 1 + 2 * j) + 1;
  shl<NT>(s, L, sh, big, nA);
  __syncthreads();
  const int nX = L + 2;
  bool exact = false;
  *ok = isqrt<NT>(big, nA, xs, nX, &exact, w, B);
  // X2 = 2X + sticky at exponent (e2 - 2j)/2 - 1
  for (int d = threadIdx.x; d < nX + 1; d += NT)
    w.cs[d] = 2LL * limb_at(xs, nX, d) + ((d == 0 && !exact) ? 1 : 0);
  __syncthreads();
  normalize<NT>(w.cs, nX + 1, big, *w.r);
  return round_rne<NT>(big, nX + 3, (e2 - 2 * j) / 2 - 1, L, mant, w);
}

// mant, exponent of RNE_P(|num| 2^ne / (den 2^de)) where V = floor(2^(2P+1+vx)/den)
// (L + 2 + vx/32 limbs, vx a multiple of 32).  num, den: normalised P-bit
// mantissas.  big: capacity >= 2L + 16; q: L + 4 + vx/32.
// Q = floor(num 2^(P+1+vx) / den) (P+1+vx or P+2+vx bits) comes from the
// columns >= L-2 of num * V only: the dropped columns sum to less than
// (L-2) 2^(32(L-1)) < 2^(32L), one unit of Q, and the Barrett estimate is at
// most one unit low, so Q0 <= Q <= Q0 + 2.
// Fast path (vx > 0): when the k = bitlen(Q0) - P - 1 >= vx bits of Q0 below
// its guard bit hold a value T with 1 <= T <= 2^k - 3, adding up to 2 carries
// into neither the guard bit nor the mantissa and leaves the low bits nonzero:
// RNE_P(Q) = RNE_P(2 Q0 + 1) with the sticky bit set, no remainder needed.
// Otherwise (exact or near-exact quotients) the remainder
// num 2^(P+1+vx) - Q0 den lies in [0, 3 den) and is computed exactly from the
// low L+3 limbs of Q0 * den; the correction then raises Q0 to Q.
template <int NT>
HK_DEV Rounded div_rne(const uint32_t *num, long long ne, const uint32_t *den, long long de,
                       const uint32_t *V, int L, uint32_t *mant, Work &w, uint32_t *big,
                       uint32_t *q, bool *ok, int vx = 0) {
  const long long P = 32LL * L;
  const int nV = L + 2 + vx / 32;
  const int nQ = L + 3 + vx / 32;
  // high columns of num * V: value sum_{d >= L-2} col_d 2^(32 d)
  const int dlo = max(0, L - 2), dhi = L + nV;
  mul_cols<NT>(num, L, V, nV, dlo, dhi, w);
  normalize<NT>(w.cs, dhi - dlo, big, *w.r);  // big = that sum / 2^(32 dlo)
  // Q0 = floor(sum / 2^P)
  shr<NT>(big, dhi - dlo + 2, 32LL * (L - dlo), q, nQ);
  __syncthreads();
  if (vx > 0) {
    if (threadIdx.x == 0) {
      int top = nQ - 1;
      while (top > 0 && q[top] == 0) top--;
      const long long b = 32LL * top + 32 - __clz(q[top]);
      const int k = (int)(b - P - 1);  // bits below the guard bit
      const int kq = k >> 5, kr = k & 31;
      const uint32_t mask = kr ? (1u << kr) - 1u : 0u;
      bool zero = (q[kq] & mask) == 0, ones = (q[kq] & mask) == mask;
      for (int l = 0; l < kq; l++) {
        zero &= q[l] == 0;
        ones &= (l == 0 ? (q[0] | 1u) : q[l]) == 0xffffffffu;
      }
      w.r->f[32] = (k >= vx && !zero && !ones) ? 1u : 0u;
    }
    __syncthreads();
    const bool fast = w.r->f[32] != 0;
    __syncthreads();
    if (fast) {
      // 2 Q0 + 1 (a shift and a set bit: no carries)
      for (int d = threadIdx.x; d < nQ + 1; d += NT)
        big[d] = (limb_at(q, nQ, d) << 1) | (d == 0 ? 1u : (limb_at(q, nQ, d - 1) >> 31));
      __syncthreads();
      *ok = true;
      return round_rne<NT>(big, nQ + 1, ne - de - P - 2 - vx, L, mant, w);
    }
  }
  // rem = num 2^(P+1+vx) - Q0 den  mod 2^(32 nR), exact since 0 <= rem < 3 den
  const int nR = L + 3;
  mul_cols<NT>(q, nQ, den, L, 0, nR, w);
  const long long pos = P + 1 + vx;
  for (int d = threadIdx.x; d < nR; d += NT) {
    const uint32_t a = limb_at(num, L, d - (int)(pos >> 5));
    const uint32_t b = limb_at(num, L, d - (int)(pos >> 5) - 1);
    const int bb = (int)(pos & 31);
    const uint32_t sv = bb ? ((a << bb) | (b >> (32 - bb))) : a;
    w.cs[d] = (long long)sv - w.cs[d];
  }
  __syncthreads();
  // resolve modulo 2^(32 nR): the true value is non-negative and < 2^(32 nR)
  normalize<NT>(w.cs, nR, big, *w.r);  // big[0..nR) = rem (limbs above nR are the wrap)
  bool done = false;
  bool sticky = true;
  int adj = 0;
  for (int it = 0; it < 4 && !done; it++) {
    // rem >= den ?
    for (int d = threadIdx.x; d < nR; d += NT) w.cs[d] = (long long)big[d] - (long long)limb_at(den, L, d);
    __syncthreads();
    const bool neg = normalize<NT>(w.cs, nR, big + (nR + 4), *w.r);
    // two's complement in nR+2 limbs: negative means rem < den
    if (neg) {
      sticky = bitlen<NT>(big, nR, *w.r) != 0;
      done = true;
    } else {
      copy<NT>(big + (nR + 4), nR, big, nR);
      __syncthreads();
      adj++;
    }
  }
  *ok = done;
  // Q = Q0 + adj; result value (2Q + sticky) 2^(ne - de - P - 2 - vx)
  for (int d = threadIdx.x; d < nQ + 1; d += NT)
    w.cs[d] = 2LL * limb_at(q, nQ, d) + (d == 0 ? 2LL * adj + (sticky ? 1 : 0) : 0);
  __syncthreads();
  normalize<NT>(w.cs, nQ + 1, big, *w.r);
  return round_rne<NT>(big, nQ + 3, ne - de - P - 2 - vx, L, mant, w);
}

}  // namespace mp
}  // namespace hk
