// Shared-memory layout and exact-formation helpers of the single-block row
// kernels (Cholesky panel in hk_panel.cu, shifted LDL^T in hk_ldlt.cu): the
// exact value m 2^e - sum (column sums from the update kernel) on a binary
// grid, and the alignment of a finished entry on its column grid.
#pragma once
#include "hk_internal.h"
#include "hk_mp.cuh"

namespace hk {

struct RowSmem {
  mp::Red *red;
  long long *cs;
  uint32_t *tmp, *Z, *mant, *big, *q, *V, *rm, *res;
  uint32_t *nb[6];
  uint32_t *xs;
  int cap, cap4;
};

__host__ __device__ inline int row_cap(int L, int C) {
  const int a = C + L + 24, b = 4 * L + 64;
  return ((a > b ? a : b) + 3) / 4 * 4;
}

// Lays out the buffers from `base` (or only measures them when base is null);
// returns the number of bytes used.
__host__ __device__ inline size_t carve(unsigned char *base, int L, int C, bool diag, RowSmem *out) {
  RowSmem s;
  s.cap = row_cap(L, C);
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
  s.big = take(s.cap4);
  s.q = take(L + 8);
  s.V = take(L + 8);
  s.rm = take(L + 8);
  s.res = take(L + 8);
  if (diag) {
    for (int k = 0; k < 6; k++) s.nb[k] = take(s.cap4);
    s.xs = take(L + 8);
  } else {
    for (int k = 0; k < 6; k++) s.nb[k] = nullptr;
    s.xs = nullptr;
  }
  if (out) *out = s;
  return off;
}

__host__ __device__ inline size_t carve_size(int L, int C, bool diag) { return carve(nullptr, L, C, diag, nullptr); }

HK_DEV mp::Work work_of(RowSmem &s) {
  mp::Work w;
  w.cs = s.cs;
  w.tmp = s.tmp;
  w.r = s.red;
  return w;
}

// Z = (-1)^sm * m * 2^(em - G) - colsum  as magnitude in s.Z, returns
// sign (+1 / -1) or 0 when the window is too narrow (range failure recorded).
template <int NT>
HK_DEV int form_exact(RowSmem &s, const long long *colrow, int C, int32_t sm, long long em,
                      const uint32_t *ml, int L, long long G, DevStatus *st, int *nZ_out) {
  const long long sh = em - G;
  if (sh < 0) {
    if (threadIdx.x == 0) raise_range(st, -sh);
    return 0;
  }
  const long long q = sh >> 5;
  const int b = (int)(sh & 31);
  const int nm = (int)(q + L + 1);
  const int nZ = max(C, nm);
  if (nZ + 2 > s.cap) {
    if (threadIdx.x == 0) raise_range(st, 32LL * (nZ + 2 - s.cap));
    return 0;
  }
  for (int d = threadIdx.x; d < nZ; d += NT) {
    const long long li = d - q;
    const uint32_t a = mp::limb_at(ml, L, li), c = mp::limb_at(ml, L, li - 1);
    const uint32_t mv = b ? ((a << b) | (c >> (32 - b))) : a;
    const long long cv = d < C ? colrow[d] : 0;
    s.cs[d] = (sm ? -(long long)mv : (long long)mv) - cv;
  }
  __syncthreads();
  const bool neg = mp::resolve<NT>(s.cs, nZ, s.Z, *s.red);
  *nZ_out = nZ + 2;
  return neg ? -1 : 1;
}

// write value (sign, mant, exp) on column grid g as W limbs; false on range failure
template <int NT>
HK_DEV bool align_entry(const uint32_t *mant, int L, long long e, bool zero, long long g, int W,
                        uint32_t *dst, DevStatus *st) {
  if (zero) {
    for (int l = threadIdx.x; l < W; l += NT) dst[l] = 0;
    return true;
  }
  const long long sh = e - g;
  const long long P = 32LL * L;
  if (sh < 0 || sh + P > 32LL * W) {
    if (threadIdx.x == 0) raise_range(st, sh < 0 ? -sh : sh + P - 32LL * W);
    return false;
  }
  mp::shl<NT>(mant, L, sh, dst, W);
  return true;
}

}  // namespace hk
