// Karatsuba expansion of aligned entries (shared by the panel kernels, which
// expand each new R entry, and the solve kernels, which expand the entries of
// the solution vector): an entry a[0..W) is written as the pieces of a one- to
// four-level split at the layout's split points -- lo, hi and lo + hi, each in
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

// The last level's split of a piece src[0..w) at m: lo and hi copied into the
// slots base and base + 1 of dst, lo + hi resolved straight into slot base + 2
// (its two carry limbs are zero and land in the gap after the slot).
template <int NT>
HK_DEV void leaf_split(const uint32_t *src, int w, int m, const KarLayout &kl, int base, uint32_t *dst,
                       long long *cs, mp::Red &r) {
  for (int l = threadIdx.x; l < m; l += NT) dst[kl.off[base] + l] = src[l];
  for (int l = threadIdx.x; l < w - m; l += NT) dst[kl.off[base + 1] + l] = src[m + l];
  split_sum<NT>(src, w, m, cs, dst + kl.off[base + 2], r);
}

// Karatsuba expansion of the aligned entry a[0..W) (global, just written by
// this block): pieces lo, hi and lo+hi of the split at the level-1 point, and
// for more levels the same split of each piece, written into their slots of
// dst (zero gaps).  t1 holds the level-1 sum (at least W/2 + 8 limbs), t2 the
// level-2 sum of the piece in hand and, behind it, the level-3 sum (t2 holds
// at least W/2 + 8 limbs: the level-2 sum needs at most W/4 + 5, the level-3
// sum at most W/8 + 5 from offset W/4 + 8, which fits for W >= 64, the
// smallest window kar_layout gives four levels).  Every split of a piece of
// width w is at m = (w + 1)/2; the sum piece is max(m, w - m) + 1 limbs.
template <int NT>
HK_DEV void expand_entry(const uint32_t *a, const KarLayout &kl, uint32_t *dst, long long *cs, uint32_t *t1,
                         uint32_t *t2, mp::Red &r) {
  for (int l = threadIdx.x; l < kl.stride; l += NT) dst[l] = 0;
  __syncthreads();
  const int W = kl.W, lv = kl.levels;
  const int m1 = kl.ms[0];
  if (lv == 1) {
    leaf_split<NT>(a, W, m1, kl, 0, dst, cs, r);
    return;
  }
  uint32_t *t3 = t2 + (W + 3) / 4 + 8;
  split_sum<NT>(a, W, m1, cs, t1, r);
  const int l1[3] = {m1, W - m1, max(m1, W - m1) + 1};
  for (int u = 0; u < 3; u++) {
    const uint32_t *s1 = u == 0 ? a : (u == 1 ? a + m1 : t1);
    const int w1 = l1[u], m2 = kl.ms[split_base(2) + u];
    if (lv == 2) {
      leaf_split<NT>(s1, w1, m2, kl, 3 * u, dst, cs, r);
      continue;
    }
    split_sum<NT>(s1, w1, m2, cs, t2, r);
    const int l2[3] = {m2, w1 - m2, max(m2, w1 - m2) + 1};
    for (int v = 0; v < 3; v++) {
      const uint32_t *s2 = v == 0 ? s1 : (v == 1 ? s1 + m2 : t2);
      const int w2 = l2[v], m3 = kl.ms[split_base(3) + 3 * u + v];
      if (lv == 3) {
        leaf_split<NT>(s2, w2, m3, kl, 9 * u + 3 * v, dst, cs, r);
        continue;
      }
      split_sum<NT>(s2, w2, m3, cs, t3, r);
      const int l3[3] = {m3, w2 - m3, max(m3, w2 - m3) + 1};
      for (int z = 0; z < 3; z++) {
        const uint32_t *s3 = z == 0 ? s2 : (z == 1 ? s2 + m3 : t3);
        const int m4 = kl.ms[split_base(4) + 9 * u + 3 * v + z];
        leaf_split<NT>(s3, l3[z], m4, kl, 27 * u + 9 * v + 3 * z, dst, cs, r);
      }
    }
  }
}

}  // namespace hk
