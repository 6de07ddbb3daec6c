// The paper's own determinant and root finder on the device.
//
// Section "The LDL^T Determinant Algorithm" evaluates P(x) = det(M - xI) by a
// submatrix-order LDL^T: for each column t the pivot D_t (x subtracted on the
// diagonal), the column C_t[r] of the trailing matrix and CDivDiag
// Q_t[r] = C_t[r] / D_t, then the rank-1 update M[r][c] -= C_t[c] Q_t[r] of the
// trailing matrix, the determinant being the product of the pivots.  Here, as
// in the Cholesky factorisation of this library, every trailing sum is
// accumulated exactly and rounded once:
//   D_t    = RNE(m_2t - x - sum_{s<t} C_s[t] Q_s[t])
//   C_t[r] = RNE(m_{t+r} - sum_{s<t} C_s[t] Q_s[r])        (r > t)
//   Q_t[r] = RNE(C_t[r] / D_t)                              (correctly rounded)
//   det    = RNE(... RNE(RNE(D_0 D_1) D_2) ... D_{N-1})     (running product)
// with negative pivots allowed (above lambda_1 the matrix is indefinite) and a
// zero pivot ending the factorisation with det = 0.
//
// The sums run on the update kernel (mode M_LDLT: C entries against Q
// entries).  Its operands are written as integers on per-column binary grids
// shifted by a per-row exponent h_t = floor(top bit of |D_t| / 2):
//   C_t[r] = c 2^(g_r + h_t),   Q_t[r] = q 2^(g_r - h_t),
// so every product C_s[i] Q_s[j] lands on the output's grid 2^(g_i + g_j)
// whatever s, and c, q have the magnitudes of the Cholesky factor's aligned
// entries (C_t[r] ~ R_tt R_tr, Q_t[r] ~ R_tr / R_tt, 2^h_t ~ R_tt).
//
// The Secant recurrence of section "The Secant Algorithm" runs on the same
// device values: one single-block kernel per step forms
//   x3 = RNE(x2 - RNE(RNE(RNE(x2 - x1) / RNE(p2 - p1)) * p2))
// and the stopping tests; section "Interval Verification" is taken as the
// inertia of the shifted LDL^T just below and just above the root.
#include "hk_internal.h"
#include "hk_kar.cuh"
#include "hk_mp.cuh"
#include "hk_panel.cuh"

namespace hk {

namespace {

constexpr int NT_LD = 512;  // pivot kernel (sequential Newton reciprocal, as the Cholesky diagonal)
constexpr int NT_LR = 256;  // row kernel (one block per entry)
constexpr int NT_SC = 256;  // scalar kernels of the Secant recurrence

HK_DEV uint32_t shifted_limb(const uint32_t *x, int n, long long d, long long q, int b) {
  const uint32_t a = mp::limb_at(x, n, d - q), c = mp::limb_at(x, n, d - q - 1);
  return b ? ((a << b) | (c >> (32 - b))) : a;
}

// Z = (-1)^sm m 2^em - (-1)^sx x 2^ex - colsum 2^G exactly, as a magnitude in
// s.Z on the grid *Gz = min(G, ex) (x's low bits may lie below the column-sum
// grid); returns the sign (+1 / -1), or 0 on a range failure (recorded).
template <int NT>
HK_DEV int form_shifted(RowSmem &s, const long long *colrow, int C, int32_t sm, long long em, const uint32_t *ml,
                        int32_t sx, long long ex, const uint32_t *xl, bool xz, int L, long long G, DevStatus *st,
                        int *nZ_out, long long *Gz) {
  const long long Gp = (xz || ex >= G) ? G : ex;
  const long long shm = em - Gp;
  if (shm < 0) {
    if (threadIdx.x == 0) raise_range(st, -shm);
    return 0;
  }
  const long long qm = shm >> 5;
  const int bm = (int)(shm & 31);
  const long long shx = xz ? 0 : ex - Gp;
  const long long qx = shx >> 5;
  const int bx = (int)(shx & 31);
  const long long shc = G - Gp;  // > 0 only when x reaches below the column-sum grid
  const long long qc = shc >> 5;
  const int bc = (int)(shc & 31);
  long long nZl = qm + L + 1;
  if (!xz) nZl = max(nZl, qx + L + 1);
  nZl = max(nZl, shc ? qc + C + 3 : (long long)C);
  if (nZl + 2 > s.cap) {
    if (threadIdx.x == 0) raise_range(st, 32LL * (nZl + 2 - s.cap));
    return 0;
  }
  const int nZ = (int)nZl;
  bool negc = false;
  if (shc) {
    // resolve the column sums into one signed integer first, then shift it
    for (int d = threadIdx.x; d < C; d += NT) s.cs[d] = colrow[d];
    __syncthreads();
    negc = mp::resolve<NT>(s.cs, C, s.tmp, *s.red);  // |colsum| in s.tmp[0 .. C+2)
    __syncthreads();
  }
  for (int d = threadIdx.x; d < nZ; d += NT) {
    const long long mv = shifted_limb(ml, L, d, qm, bm);
    const long long xv = xz ? 0 : shifted_limb(xl, L, d, qx, bx);
    long long cv;
    if (shc) {
      const long long c = shifted_limb(s.tmp, C + 2, d, qc, bc);
      cv = negc ? -c : c;
    } else {
      cv = d < C ? colrow[d] : 0;
    }
    s.cs[d] = (sm ? -mv : mv) - (sx ? -xv : xv) - cv;
  }
  __syncthreads();
  const bool neg = mp::resolve<NT>(s.cs, nZ, s.Z, *s.red);
  *nZ_out = nZ + 2;
  *Gz = Gp;
  return neg ? -1 : 1;
}

// Pivot of row i: D_i, its row shift h_i, the running determinant, the
// negative-pivot count, and the reciprocal of |D_i|'s mantissa for the
// quotients of the row.
template <int NT>
__global__ void __launch_bounds__(NT) k_ldl_pivot(LdlParams q, int i) {
  const PanelParams &p = q.pp;
  if (block_status(p.st) != ST_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RowSmem s;
  if (!HK_CHECK(p.st, carve(nullptr, p.L, p.C, true, nullptr) <= dynamic_smem_bytes(), 21,
                carve(nullptr, p.L, p.C, true, nullptr), dynamic_smem_bytes()))
    return;
  carve(smem_raw, p.L, p.C, true, &s);
  mp::Work w = work_of(s);
  const int L = p.L, N = p.N;
  const long long P = 32LL * L;
  const long long gi = p.colU[i] - 32LL * p.W;
  const long long k = i - p.r0;
  const long long crow = k * N - (k * (i + p.r0 - 1)) / 2;
  const long long *colrow = p.colsum + crow * p.C;
  const int mk = 2 * i;
  int nZ = 0;
  long long Gz = 0;
  bool xnz = false;  // x = 0 is read from its limbs (an iterate may be zero)
  for (int l = threadIdx.x; l < L; l += NT) xnz |= q.x.limbs[l] != 0;
  const bool xz = q.xzero != 0 || !__syncthreads_or(xnz);
  const long long G = 2 * gi;  // grid of the diagonal's column sums
  const uint32_t *mlimbs = p.mom.limbs + (long long)mk * L;
  int sgn = 0;
  bool exact = true;
  if (!xz && q.x.exp[0] + P <= G) {
    // x lies wholly below the grid (|x| < 2^G).  When the rest of the sum,
    // Z0 = m_2i - colsum, is at least 2^(G + P + 1) in magnitude, the P-bit
    // result's ulp is at least 2^(G + 1): every representable value and every
    // rounding midpoint is a multiple of 2^G, and x moves the exact sum by
    // less than 2^G, so any stand-in of x's sign and of magnitude below 2^G
    // gives the same RNE(D_i).  The stand-in 2^(G - 1) costs one bit of grid
    // where x itself would need the whole gap down to its last bit.
    sgn = form_shifted<NT>(s, colrow, p.C, p.mom.sign[mk], p.mom.exp[mk], mlimbs, 0, 0, q.x.limbs, true, L, G,
                           p.st, &nZ, &Gz);
    if (sgn != 0 && nZ + 1 <= s.cap && mp::bitlen<NT>(s.Z, nZ, *s.red) >= P + 2) {
      exact = false;
      // |Z0| 2^G - sign(x) 2^(G-1) = (2|Z0| -+ 1) 2^(G-1), of Z0's sign
      for (int d = threadIdx.x; d <= nZ; d += NT) {
        const uint32_t hi = d < nZ ? s.Z[d] : 0u, lo = d >= 1 ? s.Z[d - 1] : 0u;
        s.tmp[d] = (hi << 1) | (lo >> 31);
      }
      __syncthreads();
      for (int d = threadIdx.x; d <= nZ; d += NT) s.Z[d] = s.tmp[d];
      __syncthreads();
      const bool same = (sgn > 0) == (q.x.sign[0] == 0);  // x has Z0's sign: the magnitude shrinks
      if (!same) {
        if (threadIdx.x == 0) s.Z[0] |= 1u;  // bit 0 is clear after the shift
      } else {
        // subtract one: borrow through the zero limbs below the lowest
        // nonzero one (the value is at least 2^(P+2), so one exists)
        __shared__ int low_nz;
        if (threadIdx.x == 0) low_nz = nZ;
        __syncthreads();
        for (int d = threadIdx.x; d <= nZ; d += NT)
          if (s.Z[d] != 0) atomicMin(&low_nz, d);
        __syncthreads();
        const int j = low_nz;
        for (int d = threadIdx.x; d < j; d += NT) s.Z[d] = 0xffffffffu;
        if (threadIdx.x == 0) s.Z[j] -= 1u;
      }
      __syncthreads();
      nZ += 1;
      Gz = G - 1;
    }
  }
  if (exact)
    sgn = form_shifted<NT>(s, colrow, p.C, p.mom.sign[mk], p.mom.exp[mk], mlimbs, q.x.sign[0], q.x.exp[0],
                           q.x.limbs, xz, L, G, p.st, &nZ, &Gz);
  if (sgn == 0) {
    if (threadIdx.x == 0) atomicMin(&p.st->range_row, i);
    return;
  }
  const mp::Rounded D = mp::round_rne<NT>(s.Z, nZ, Gz, L, s.mant, w);
  const long long idx = tri_idx(i, i, N);
  const int neg = (D.nonzero && sgn < 0) ? 1 : 0;
  for (int l = threadIdx.x; l < L; l += NT) p.R.limbs[idx * L + l] = s.mant[l];
  if (threadIdx.x == 0) {
    p.R.sign[idx] = neg;
    p.R.exp[idx] = D.nonzero ? D.exp : 0;
    p.Asign[idx] = neg;
  }
  if (!D.nonzero) {
    // a zero pivot: det(M - xI) = 0; the factorisation stops here
    if (threadIdx.x == 0) {
      atomicMin(q.zero_row, i);
      for (int l = 0; l < L; l++) q.det.limbs[l] = 0;
      q.det.sign[0] = 0;
      q.det.exp[0] = 0;
      atomicCAS(&p.st->code, ST_OK, ST_ZERO);
    }
    return;
  }
  if (threadIdx.x == 0) {
    q.h[i] = (D.exp + P) >> 1;  // floor of half the top-bit exponent of |D_i|
    if (neg) *q.negcount += 1;
  }
  // running determinant: det <- RNE(det * D_i)
  if (i == 0) {
    for (int l = threadIdx.x; l < L; l += NT) q.det.limbs[l] = s.mant[l];
    if (threadIdx.x == 0) {
      q.det.sign[0] = neg;
      q.det.exp[0] = D.exp;
    }
    __syncthreads();
  } else {
    mp::mul<NT>(q.det.limbs, L, s.mant, L, s.big, w);
    __syncthreads();
    const long long de = q.det.exp[0];
    const mp::Rounded r = mp::round_rne<NT>(s.big, 2 * L + 2, de + D.exp, L, s.res, w);
    for (int l = threadIdx.x; l < L; l += NT) q.det.limbs[l] = s.res[l];
    __syncthreads();
    if (threadIdx.x == 0) {
      q.det.sign[0] ^= neg;
      q.det.exp[0] = r.exp;
    }
  }
  mp::NBufs B;
  for (int t = 0; t < 6; t++) (&B.a)[t] = s.nb[t];
  B.cap = s.cap4;
  const bool ok = mp::recip<NT>(s.mant, L, s.V, w, B, RECIP_EXTRA);
  for (int l = threadIdx.x; l < recip_limbs(L); l += NT) p.recip[(long long)i * recip_limbs(L) + l] = s.V[l];
  if (threadIdx.x == 0 && !ok) raise_timeout(p.st);
}

// Row i, column j = i + 1 + blockIdx.x: C_i[j], Q_i[j] = C_i[j] / D_i, both
// aligned (column grid shifted by -+ h_i) and expanded for later updates.
template <int NT>
__global__ void __launch_bounds__(NT) k_ldl_row(LdlParams q, int i) {
  const PanelParams &p = q.pp;
  if (block_status(p.st) != ST_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RowSmem s;
  if (!HK_CHECK(p.st, carve(nullptr, p.L, p.C, false, nullptr) <= dynamic_smem_bytes(), 22,
                carve(nullptr, p.L, p.C, false, nullptr), dynamic_smem_bytes()))
    return;
  carve(smem_raw, p.L, p.C, false, &s);
  mp::Work w = work_of(s);
  const int L = p.L, N = p.N, W = p.W;
  const int j = i + 1 + blockIdx.x;
  const long long gi = p.colU[i] - 32LL * W;
  const long long gj = p.colU[j] - 32LL * W;
  const long long k = i - p.r0;
  const long long crow = k * N - (k * (i + p.r0 - 1)) / 2 + (j - i);
  const long long *colrow = p.colsum + crow * p.C;
  const int mk = i + j;
  int nZ = 0;
  const int sgn = form_exact<NT>(s, colrow, p.C, p.mom.sign[mk], p.mom.exp[mk], p.mom.limbs + (long long)mk * L, L,
                                 gi + gj, p.st, &nZ);
  if (sgn == 0) {
    if (threadIdx.x == 0) atomicMin(&p.st->range_row, i);
    return;
  }
  const mp::Rounded Cr = mp::round_rne<NT>(s.Z, nZ, gi + gj, L, s.mant, w);
  const long long idx = tri_idx(i, j, N);
  const long long iidx = tri_idx(i, i, N);
  if (!Cr.nonzero) {
    for (int l = threadIdx.x; l < L; l += NT) p.R.limbs[idx * L + l] = q.Q.limbs[idx * L + l] = 0;
    for (int l = threadIdx.x; l < W; l += NT) p.A[idx * W + l] = q.B[idx * W + l] = 0;
    if (p.kl.levels > 0)
      for (int l = threadIdx.x; l < p.kl.stride; l += NT)
        p.Aexp[idx * p.kl.stride + l] = q.Bexp[idx * p.kl.stride + l] = 0;
    if (threadIdx.x == 0) {
      p.R.sign[idx] = q.Q.sign[idx] = 0;
      p.R.exp[idx] = q.Q.exp[idx] = 0;
      p.Asign[idx] = q.Bsign[idx] = 0;
    }
    return;
  }
  const int cneg = sgn < 0 ? 1 : 0;
  const int qneg = cneg ^ (p.R.sign[iidx] ? 1 : 0);
  for (int l = threadIdx.x; l < L; l += NT) {
    p.R.limbs[idx * L + l] = s.mant[l];
    s.rm[l] = p.R.limbs[iidx * L + l];
  }
  for (int l = threadIdx.x; l < recip_limbs(L); l += NT) s.V[l] = p.recip[(long long)i * recip_limbs(L) + l];
  if (threadIdx.x == 0) {
    p.R.sign[idx] = cneg;
    p.R.exp[idx] = Cr.exp;
    p.Asign[idx] = cneg;
  }
  __syncthreads();
  bool ok = true;
  const mp::Rounded Qr =
      mp::div_rne<NT>(s.mant, Cr.exp, s.rm, p.R.exp[iidx], s.V, L, s.res, w, s.big, s.q, &ok, RECIP_EXTRA);
  for (int l = threadIdx.x; l < L; l += NT) q.Q.limbs[idx * L + l] = s.res[l];
  if (threadIdx.x == 0) {
    q.Q.sign[idx] = qneg;
    q.Q.exp[idx] = Qr.exp;
    q.Bsign[idx] = qneg;
    if (!ok) raise_timeout(p.st);
  }
  const long long hi = q.h[i];
  const bool fc = align_entry<NT>(s.mant, L, Cr.exp, false, gj + hi, W, p.A + idx * W, p.st);
  const bool fq = align_entry<NT>(s.res, L, Qr.exp, false, gj - hi, W, q.B + idx * W, p.st);
  if (!(fc && fq)) {
    if (threadIdx.x == 0) atomicMin(&p.st->range_row, i);
    return;
  }
  if (p.kl.levels > 0) {
    __syncthreads();
    expand_entry<NT>(p.A + idx * W, p.kl, p.Aexp + idx * p.kl.stride, s.cs, s.Z, s.big, *s.red);
    __syncthreads();
    expand_entry<NT>(q.B + idx * W, p.kl, q.Bexp + idx * p.kl.stride, s.cs, s.Z, s.big, *s.red);
  }
}

// ---------------------------------------------------------------------------
// scalar P-bit arithmetic of the Secant recurrence (single block, work areas
// in global memory)
// ---------------------------------------------------------------------------

struct ScalarWork {
  long long *cs;
  uint32_t *tmp, *big, *q, *V, *t1, *t2, *t3;
  uint32_t *nb[6];
  int cap;
};

HK_DEV bool is_zero(const MpArr &a, int k, int L) {
  bool z = true;
  for (int l = 0; l < L; l++) z &= a.limbs[(long long)k * L + l] == 0;
  return z;
}

// exact comparison of two P-bit values (sign, exponent, normalised mantissa):
// -1, 0, +1 for a < b, a = b, a > b (thread-serial)
HK_DEV int cmp_val(const MpArr &a, int ka, const MpArr &b, int kb, int L) {
  const bool za = is_zero(a, ka, L), zb = is_zero(b, kb, L);
  const int sa = za ? 0 : (a.sign[ka] ? -1 : 1), sb = zb ? 0 : (b.sign[kb] ? -1 : 1);
  if (sa != sb) return sa < sb ? -1 : 1;
  if (sa == 0) return 0;
  int mag = 0;  // |a| vs |b|
  if (a.exp[ka] != b.exp[kb]) {
    mag = a.exp[ka] < b.exp[kb] ? -1 : 1;
  } else {
    for (int l = L - 1; l >= 0 && mag == 0; l--) {
      const uint32_t x = a.limbs[(long long)ka * L + l], y = b.limbs[(long long)kb * L + l];
      if (x != y) mag = x < y ? -1 : 1;
    }
  }
  return sa > 0 ? mag : -mag;
}

// out[ko] = RNE(a[ka] + (-1)^negb b[kb]); exact sum on the grid of the smaller
// exponent, the smaller operand replaced by a sticky unit when it lies more
// than P + 64 bits below the larger
template <int NT>
HK_DEV void add_rne(const MpArr &a, int ka, const MpArr &b, int kb, int negb, const MpArr &out, int ko, int L,
                    ScalarWork &sw, mp::Work &w) {
  __shared__ int zs[2];
  if (threadIdx.x == 0) {
    zs[0] = is_zero(a, ka, L);
    zs[1] = is_zero(b, kb, L);
  }
  __syncthreads();
  const bool za = zs[0], zb = zs[1];
  const long long P = 32LL * L;
  if (za || zb) {
    const MpArr &src = za ? b : a;
    const int ks = za ? kb : ka;
    const int flip = za ? negb : 0;
    for (int l = threadIdx.x; l < L; l += NT) out.limbs[(long long)ko * L + l] = (za && zb) ? 0 : src.limbs[(long long)ks * L + l];
    __syncthreads();
    if (threadIdx.x == 0) {
      out.sign[ko] = (za && zb) ? 0 : (src.sign[ks] ^ flip);
      out.exp[ko] = (za && zb) ? 0 : src.exp[ks];
    }
    __syncthreads();
    return;
  }
  const long long ea = a.exp[ka], eb = b.exp[kb];
  const int sa = a.sign[ka] ? -1 : 1, sb = (b.sign[kb] ^ negb) ? -1 : 1;
  const long long hi = max(ea, eb);
  long long lo = min(ea, eb);
  const bool sticky = hi - lo > P + 64;
  if (sticky) lo = hi - P - 64;
  // columns of (-1) a 2^(ea - lo) + (-1) b 2^(eb - lo)
  const long long qa = (ea - lo) >> 5, qb = (eb - lo) >> 5;
  const int ba = (int)((ea - lo) & 31), bb = (int)((eb - lo) & 31);
  const int n = (int)(max(qa, qb) + L + 2);
  const uint32_t *al = a.limbs + (long long)ka * L, *bl = b.limbs + (long long)kb * L;
  for (int d = threadIdx.x; d < n; d += NT) {
    long long v = 0;
    if (!(sticky && ea < eb)) v += sa * (long long)shifted_limb(al, L, d, qa, ba);
    if (!(sticky && eb < ea)) v += sb * (long long)shifted_limb(bl, L, d, qb, bb);
    sw.cs[d] = v;
  }
  __syncthreads();
  if (sticky && threadIdx.x == 0) sw.cs[0] += (ea < eb ? sa : sb);  // the dropped operand's sign, one unit
  __syncthreads();
  const bool neg = mp::resolve<NT>(sw.cs, n, sw.big, *w.r);
  const mp::Rounded r = mp::round_rne<NT>(sw.big, n + 2, lo, L, sw.t1, w);
  for (int l = threadIdx.x; l < L; l += NT) out.limbs[(long long)ko * L + l] = sw.t1[l];
  __syncthreads();
  if (threadIdx.x == 0) {
    out.sign[ko] = (r.nonzero && neg) ? 1 : 0;
    out.exp[ko] = r.nonzero ? r.exp : 0;
  }
  __syncthreads();
}

template <int NT>
HK_DEV void mul_rne(const MpArr &a, int ka, const MpArr &b, int kb, const MpArr &out, int ko, int L, ScalarWork &sw,
                    mp::Work &w) {
  mp::mul<NT>(a.limbs + (long long)ka * L, L, b.limbs + (long long)kb * L, L, sw.big, w);
  __syncthreads();
  const mp::Rounded r = mp::round_rne<NT>(sw.big, 2 * L + 2, a.exp[ka] + b.exp[kb], L, sw.t1, w);
  for (int l = threadIdx.x; l < L; l += NT) out.limbs[(long long)ko * L + l] = sw.t1[l];
  __syncthreads();
  if (threadIdx.x == 0) {
    out.sign[ko] = r.nonzero ? (a.sign[ka] ^ b.sign[kb]) : 0;
    out.exp[ko] = r.nonzero ? r.exp : 0;
  }
  __syncthreads();
}

template <int NT>
HK_DEV bool div_rne_val(const MpArr &a, int ka, const MpArr &b, int kb, const MpArr &out, int ko, int L,
                        ScalarWork &sw, mp::Work &w) {
  __shared__ int za;
  if (threadIdx.x == 0) za = is_zero(a, ka, L);
  __syncthreads();
  if (za) {  // zero numerator: the quotient is +0
    for (int l = threadIdx.x; l < L; l += NT) out.limbs[(long long)ko * L + l] = 0;
    __syncthreads();
    if (threadIdx.x == 0) {
      out.sign[ko] = 0;
      out.exp[ko] = 0;
    }
    __syncthreads();
    return true;
  }
  mp::NBufs B;
  for (int t = 0; t < 6; t++) (&B.a)[t] = sw.nb[t];
  B.cap = sw.cap;
  bool ok = mp::recip<NT>(b.limbs + (long long)kb * L, L, sw.V, w, B, RECIP_EXTRA);
  bool ok2 = true;
  const mp::Rounded r = mp::div_rne<NT>(a.limbs + (long long)ka * L, a.exp[ka], b.limbs + (long long)kb * L, b.exp[kb],
                                        sw.V, L, sw.t1, w, sw.big, sw.q, &ok2, RECIP_EXTRA);
  for (int l = threadIdx.x; l < L; l += NT) out.limbs[(long long)ko * L + l] = sw.t1[l];
  __syncthreads();
  if (threadIdx.x == 0) {
    out.sign[ko] = r.nonzero ? (a.sign[ka] ^ b.sign[kb]) : 0;
    out.exp[ko] = r.nonzero ? r.exp : 0;
  }
  __syncthreads();
  return ok && ok2;
}

// One step of the Secant recurrence on device values (section "The Secant
// Algorithm"): from x1 = xs[k1], x2 = xs[k2] and P(x1) = ps[k1], P(x2) = ps[k2]
//   flags[0] = 1 when P(x2) = P(x1) (no secant: stop);
//   otherwise step = RNE(RNE(RNE(x2 - x1) / RNE(p2 - p1)) * p2),
//   x3 = RNE(x2 - step) into xs[k3], |step| into tmpv[3];
//   flags[1] = 1 when a previous step size exists (have_last) and
//     |step| >= that size (tmpv[4]) with k >= 3: the rounding noise of P(x) is
//     reached, keep x2;
//   flags[2] = 1 when |x3 - x2| <= 2^-136 |x3| exactly (converged);
//   flags[3] = 1 when a multiprecision correction did not settle.
// tmpv holds five scratch values (0..2 intermediates, 3 the new size, 4 the
// last size).
template <int NT>
__global__ void __launch_bounds__(NT) k_secant_step(MpArr xs, MpArr ps, MpArr tmpv, int k1, int k2, int k3, int kstep,
                                                    int have_last, int L, ScalarWork sw, int *flags) {
  __shared__ mp::Red red;
  mp::Work w;
  w.cs = sw.cs;
  w.tmp = sw.tmp;
  w.r = &red;
  __shared__ int stop;
  if (threadIdx.x == 0) {
    flags[0] = flags[1] = flags[2] = flags[3] = 0;
    stop = cmp_val(ps, k2, ps, k1, L) == 0 && ps.sign[k2] == ps.sign[k1];
    if (stop) flags[0] = 1;
  }
  __syncthreads();
  if (stop) return;
  add_rne<NT>(xs, k2, xs, k1, 1, tmpv, 0, L, sw, w);   // RNE(x2 - x1)
  add_rne<NT>(ps, k2, ps, k1, 1, tmpv, 1, L, sw, w);   // RNE(p2 - p1)
  const bool ok = div_rne_val<NT>(tmpv, 0, tmpv, 1, tmpv, 2, L, sw, w);  // quotient
  mul_rne<NT>(tmpv, 2, ps, k2, tmpv, 3, L, sw, w);     // step
  add_rne<NT>(xs, k2, tmpv, 3, 1, xs, k3, L, sw, w);   // x3 = RNE(x2 - step)
  if (threadIdx.x == 0) {
    if (!ok) flags[3] = 1;
    tmpv.sign[3] = 0;  // |step|
    if (kstep >= 3 && have_last && cmp_val(tmpv, 3, tmpv, 4, L) >= 0) flags[1] = 1;
  }
  __syncthreads();
  // convergence: exact |x3 - x2| 2^136 <= |x3|; only possible when x3 and x2
  // share their sign and their exponents differ by at most one
  __shared__ int conv;
  if (threadIdx.x == 0) {
    const bool z3 = is_zero(xs, k3, L), z2 = is_zero(xs, k2, L);
    conv = -1;  // -1: decide below
    if (z3) conv = z2 ? 1 : 0;
    else if (z2 || xs.sign[k3] != xs.sign[k2]) conv = 0;
    else {
      const long long d = xs.exp[k3] - xs.exp[k2];
      if (d > 1 || d < -1) conv = 0;
    }
  }
  __syncthreads();
  if (conv < 0) {
    const long long e3 = xs.exp[k3], e2 = xs.exp[k2];
    const long long lo = min(e3, e2);
    const uint32_t *l3 = xs.limbs + (long long)k3 * L, *l2 = xs.limbs + (long long)k2 * L;
    // |x3| - |x2| on the grid 2^lo (same signs), then 2^136 |diff| - |x3|
    const int n = L + 2;
    for (int d = threadIdx.x; d < n; d += NT)
      sw.cs[d] = (long long)shifted_limb(l3, L, d, 0, (int)(e3 - lo)) - (long long)shifted_limb(l2, L, d, 0, (int)(e2 - lo));
    __syncthreads();
    mp::resolve<NT>(sw.cs, n, sw.t2, red);  // |diff| in t2[0 .. n+2)
    // 2^136 |diff| = |diff| shifted by 4 limbs and 8 bits; |x3| on grid lo
    const int m = n + 2 + 6;
    for (int d = threadIdx.x; d < m; d += NT)
      sw.cs[d] = (long long)shifted_limb(sw.t2, n + 2, d, 4, 8) - (long long)shifted_limb(l3, L, d, 0, (int)(e3 - lo));
    __syncthreads();
    const bool below = mp::resolve<NT>(sw.cs, m, sw.t3, red);  // 2^136|diff| - |x3| < 0 ?
    // equal counts as converged: test the magnitude for zero
    __shared__ int nz;
    if (threadIdx.x == 0) nz = 0;
    __syncthreads();
    bool any = false;
    for (int d = threadIdx.x; d < m + 2; d += NT) any |= sw.t3[d] != 0;
    if (any) atomicOr(&nz, 1);
    __syncthreads();
    if (threadIdx.x == 0) conv = (below || !nz) ? 1 : 0;
    __syncthreads();
  }
  if (threadIdx.x == 0) flags[2] = conv;
}

// Self-test of the Secant step's scalar operations on one pair of values:
// op 0: RNE(a - b), 1: RNE(a * b), 2: RNE(a / b) (b nonzero), 3: the exact
// comparison of a and b (-1, 0, 1 in flags[0]).
template <int NT>
__global__ void __launch_bounds__(NT) k_scalar_selftest(int op, MpArr a, MpArr b, MpArr out, int L, ScalarWork sw,
                                                        int *flags) {
  __shared__ mp::Red red;
  mp::Work w;
  w.cs = sw.cs;
  w.tmp = sw.tmp;
  w.r = &red;
  if (op == 0) add_rne<NT>(a, 0, b, 0, 1, out, 0, L, sw, w);
  if (op == 1) mul_rne<NT>(a, 0, b, 0, out, 0, L, sw, w);
  if (op == 2) {
    const bool ok = div_rne_val<NT>(a, 0, b, 0, out, 0, L, sw, w);
    if (threadIdx.x == 0) flags[1] = ok ? 0 : 1;
  }
  if (op == 3 && threadIdx.x == 0) flags[0] = cmp_val(a, 0, b, 0, L);
}

// Smallest pivot (reading of the paper's start x_1 < 0): dst[kd] = -min_t D_t
// over the diagonal of the packed triangle R (exact comparisons).
template <int NT>
__global__ void __launch_bounds__(NT) k_neg_min_pivot(MpArr R, int N, int L, MpArr dst, int kd) {
  __shared__ int best[NT];
  int b = -1;
  for (int t = threadIdx.x; t < N; t += NT) {
    const int kt = (int)tri_idx(t, t, N);
    if (b < 0 || cmp_val(R, kt, R, b, L) < 0) b = kt;
  }
  best[threadIdx.x] = b;
  __syncthreads();
  for (int st = NT / 2; st > 0; st >>= 1) {
    if (threadIdx.x < st) {
      const int o = best[threadIdx.x + st];
      const int c = best[threadIdx.x];
      if (o >= 0 && (c < 0 || cmp_val(R, o, R, c, L) < 0)) best[threadIdx.x] = o;
    }
    __syncthreads();
  }
  const int kb = best[0];
  for (int l = threadIdx.x; l < L; l += NT) dst.limbs[(long long)kd * L + l] = R.limbs[(long long)kb * L + l];
  if (threadIdx.x == 0) {
    const bool z = is_zero(R, kb, L);
    dst.sign[kd] = z ? 0 : (R.sign[kb] ^ 1);
    dst.exp[kd] = z ? 0 : R.exp[kb];
  }
}

// dst[kd] = src[ks] (1 - 2^-bits) (sgn = -1) or (1 + 2^-bits) (sgn = +1),
// exactly: the source is a P-bit value, the result has L2 limbs with
// 32 L2 >= 32 L + bits + 1 (the verification points of the root)
__global__ void k_scale_pm(MpArr src, int ks, int L, int bits, int sgn, MpArr dst, int kd, int L2) {
  // magnitude m (2^bits + sgn) as an L2-limb integer, top-aligned, exponent adjusted
  extern __shared__ long long colv[];
  const uint32_t *m = src.limbs + (long long)ks * L;
  const int n = L2 + 2;
  for (int d = threadIdx.x; d < n; d += blockDim.x) {
    // columns of m 2^bits + sgn m, on the grid of m
    const long long qb = bits >> 5;
    const int bb = bits & 31;
    colv[d] = (long long)shifted_limb(m, L, d, qb, bb) + sgn * (long long)mp::limb_at(m, L, d);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    // resolve carries (non-negative result: m 2^bits > m)
    long long c = 0;
    for (int d = 0; d < n; d++) {
      const long long v = colv[d] + c;
      colv[d] = v & 0xffffffffLL;
      c = v >> 32;
    }
    int top = n - 1;
    while (top > 0 && colv[top] == 0) top--;
    const int b = 32 * top + 32 - __clz((uint32_t)colv[top]);
    // normalise to 32 L2 bits: shift left by 32 L2 - b (>= 0 by the size rule)
    const int sh = 32 * L2 - b;
    for (int l = L2 - 1; l >= 0; l--) {
      const long long bit = (long long)32 * l - sh;  // source bit of limb l's bit 0
      uint32_t v = 0;
      const long long qq = bit >> 5;
      const int rr = (int)(bit & 31);
      const uint32_t lo = (qq >= 0 && qq < n) ? (uint32_t)colv[qq] : 0;
      const uint32_t hi = (qq + 1 >= 0 && qq + 1 < n) ? (uint32_t)colv[qq + 1] : 0;
      v = rr ? ((lo >> rr) | (hi << (32 - rr))) : lo;
      dst.limbs[(long long)kd * L2 + l] = v;
    }
    dst.sign[kd] = src.sign[ks];
    dst.exp[kd] = src.exp[ks] - bits - sh;
  }
}

// Moments of precision L (src) zero-extended to L2 >= L limbs (exact).
__global__ void k_widen(MpArr src, int n, int L, MpArr dst, int L2) {
  const long long k = blockIdx.x;
  if (k >= n) return;
  const int d = L2 - L;
  for (int l = threadIdx.x; l < L2; l += blockDim.x)
    dst.limbs[k * L2 + l] = l < d ? 0 : src.limbs[k * L + l - d];
  if (threadIdx.x == 0) {
    dst.sign[k] = src.sign[k];
    bool z = true;
    for (int l = 0; l < L; l++) z &= src.limbs[k * L + l] == 0;
    dst.exp[k] = z ? 0 : src.exp[k] - 32LL * d;
  }
}

}  // namespace

size_t ldl_smem_pivot(int L, int C) { return carve_size(L, C, true); }
size_t ldl_smem_row(int L, int C) { return carve_size(L, C, false); }
size_t scalar_work_limbs(int L) { return 4 * (size_t)L + 64; }

static cudaError_t set_smem_ld(const void *fn, size_t bytes) {
  return bytes > 48 * 1024 ? allow_dynamic_smem(fn) : cudaSuccess;
}

cudaError_t launch_ldl_pivot(const LdlParams &q, int i, cudaStream_t s) {
  const size_t smem = ldl_smem_pivot(q.pp.L, q.pp.C);
  cudaError_t e = set_smem_ld((const void *)k_ldl_pivot<NT_LD>, smem);
  if (e != cudaSuccess) return e;
  k_ldl_pivot<NT_LD><<<1, NT_LD, smem, s>>>(q, i);
  return cudaGetLastError();
}

cudaError_t launch_ldl_row(const LdlParams &q, int i, cudaStream_t s) {
  if (i + 1 >= q.pp.N) return cudaSuccess;
  const size_t smem = ldl_smem_row(q.pp.L, q.pp.C);
  cudaError_t e = set_smem_ld((const void *)k_ldl_row<NT_LR>, smem);
  if (e != cudaSuccess) return e;
  k_ldl_row<NT_LR><<<q.pp.N - i - 1, NT_LR, smem, s>>>(q, i);
  return cudaGetLastError();
}

// work area of the scalar kernels: `base` of scalar_work_bytes(L) bytes
size_t scalar_work_bytes(int L) {
  const size_t cap = scalar_work_limbs(L);
  return cap * 8 + cap * 4 * 13;
}

static ScalarWork scalar_work(void *base, int L) {
  ScalarWork sw;
  const size_t cap = scalar_work_limbs(L);
  sw.cap = (int)cap;
  sw.cs = reinterpret_cast<long long *>(base);
  uint32_t *u = reinterpret_cast<uint32_t *>(sw.cs + cap);
  sw.tmp = u;
  sw.big = u + cap;
  sw.q = u + 2 * cap;
  sw.V = u + 3 * cap;
  sw.t1 = u + 4 * cap;
  sw.t2 = u + 5 * cap;
  sw.t3 = u + 6 * cap;
  for (int t = 0; t < 6; t++) sw.nb[t] = u + (7 + t) * cap;
  return sw;
}

cudaError_t launch_secant_step(MpArr xs, MpArr ps, MpArr tmpv, int k1, int k2, int k3, int kstep, int have_last,
                               int L, void *work, int *flags, cudaStream_t s) {
  k_secant_step<NT_SC><<<1, NT_SC, 0, s>>>(xs, ps, tmpv, k1, k2, k3, kstep, have_last, L, scalar_work(work, L), flags);
  return cudaGetLastError();
}

cudaError_t launch_scalar_selftest(int op, MpArr a, MpArr b, MpArr out, int L, void *work, int *flags,
                                  cudaStream_t s) {
  k_scalar_selftest<NT_SC><<<1, NT_SC, 0, s>>>(op, a, b, out, L, scalar_work(work, L), flags);
  return cudaGetLastError();
}

cudaError_t launch_neg_min_pivot(MpArr R, int N, int L, MpArr dst, int kd, cudaStream_t s) {
  k_neg_min_pivot<NT_SC><<<1, NT_SC, 0, s>>>(R, N, L, dst, kd);
  return cudaGetLastError();
}

cudaError_t launch_scale_pm(MpArr src, int ks, int L, int bits, int sgn, MpArr dst, int kd, int L2, cudaStream_t s) {
  const size_t smem = (size_t)(L2 + 2) * 8;
  cudaError_t e = set_smem_ld((const void *)k_scale_pm, smem);
  if (e != cudaSuccess) return e;
  k_scale_pm<<<1, 128, smem, s>>>(src, ks, L, bits, sgn, dst, kd, L2);
  return cudaGetLastError();
}

cudaError_t launch_widen(MpArr src, int n, int L, MpArr dst, int L2, cudaStream_t s) {
  k_widen<<<n, 128, 0, s>>>(src, n, L, dst, L2);
  return cudaGetLastError();
}

}  // namespace hk
