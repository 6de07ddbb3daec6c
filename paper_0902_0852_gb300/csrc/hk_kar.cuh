// Karatsuba expansion of aligned entries (shared by the panel kernels, which
// expand each new R entry, and the solve kernels, which expand the entries of
// the solution vector): an entry a[0..W) is written as the pieces of a one- to
// three-level split at the layout's split points -- lo, hi and lo + hi, each in
// its own slot with zero gaps -- so that the update kernel contracts the
// pieces (Karatsuba on the whole dot product, see hk_update.cu).
#pragma once
#include "hk_internal.h"
#include "hk_mp.cuh"

namespace hk {

// cs[0..ws) = lo + hi limbwise for the split of src[0..w) at m (ws = max(m,
// w - m) + 1), resolved into out[0..ws + 2) (the top two limbs are zero)
template <int NT>
HK_DEV void split_sum(const uint32_t *src, int w, int m, long long *cs, uint32_t *out, mp::Red &r) {
  const int ws = max(m, w - m) + 1;
  for (int l = threadIdx.x; l < ws; l += NT)
    cs[l] = (long long)mp::limb_at(src, m, l) + (long long)mp::limb_at(src + m, w - m, l);
  __syncthreads();
  mp::normalize<NT>(cs, ws, out, r);
}

// Karatsuba expansion of the aligned entry a[0..W) (global, just written by
// this block): pieces lo, hi and lo+hi of the split at m1, and for more
// levels the same split of each piece, written into their slots of dst (zero
// gaps).  t1 holds the level-1 sum, t2 the level-2 sum of the piece in hand
// (each at least W/2 + 8 limbs); the level-3 sums are resolved straight into
// their slots (their two carry limbs are zero and land in the gap).
template <int NT>
HK_DEV void expand_entry(const uint32_t *a, const KarLayout &kl, uint32_t *dst, long long *cs, uint32_t *t1,
                         uint32_t *t2, mp::Red &r) {
  for (int l = threadIdx.x; l < kl.stride; l += NT) dst[l] = 0;
  __syncthreads();
  const int W = kl.W, m1 = kl.m1;
  const int l1[3] = {m1, W - m1, max(m1, W - m1) + 1};
  split_sum<NT>(a, W, m1, cs, t1, r);
  if (kl.levels == 1) {
    for (int l = threadIdx.x; l < l1[0]; l += NT) dst[kl.off[0] + l] = a[l];
    for (int l = threadIdx.x; l < l1[1]; l += NT) dst[kl.off[1] + l] = a[m1 + l];
    for (int l = threadIdx.x; l < l1[2]; l += NT) dst[kl.off[2] + l] = t1[l];
    return;
  }
  for (int u = 0; u < 3; u++) {
    const uint32_t *src = u == 0 ? a : (u == 1 ? a + m1 : t1);
    const int wu = l1[u], m2 = kl.m2[u];
    split_sum<NT>(src, wu, m2, cs, t2, r);
    if (kl.levels == 2) {
      for (int l = threadIdx.x; l < m2; l += NT) dst[kl.off[3 * u] + l] = src[l];
      for (int l = threadIdx.x; l < wu - m2; l += NT) dst[kl.off[3 * u + 1] + l] = src[m2 + l];
      for (int l = threadIdx.x; l < kl.w[3 * u + 2]; l += NT) dst[kl.off[3 * u + 2] + l] = t2[l];
      __syncthreads();
      continue;
    }
    const int l2[3] = {m2, wu - m2, max(m2, wu - m2) + 1};
    for (int v = 0; v < 3; v++) {
      const uint32_t *s2 = v == 0 ? src : (v == 1 ? src + m2 : t2);
      const int w2 = l2[v], m3 = kl.m3[3 * u + v], base = 9 * u + 3 * v;
      for (int l = threadIdx.x; l < m3; l += NT) dst[kl.off[base] + l] = s2[l];
      for (int l = threadIdx.x; l < w2 - m3; l += NT) dst[kl.off[base + 1] + l] = s2[m3 + l];
      split_sum<NT>(s2, w2, m3, cs, dst + kl.off[base + 2], r);
    }
  }
}

}  // namespace hk
