// Karatsuba expansion of aligned entries (shared by the panel kernels, which
// expand each new R entry, and the solve kernels, which expand the entries of
// the solution vector): an entry a[0..W) is written as the pieces of a one- or
// two-level split at the layout's split points -- lo, hi and lo + hi, each in
// its own slot with zero gaps -- so that the update kernel contracts the
// pieces (Karatsuba on the whole dot product, see hk_update.cu).
#pragma once
#include "hk_internal.h"
#include "hk_mp.cuh"

namespace hk {

// Karatsuba expansion of the aligned entry a[0..W) (global, just written by
// this block): pieces lo, hi and lo+hi of the split at m1, and for two levels
// the same split of each of those, written into their slots of dst (zero gaps).
template <int NT>
HK_DEV void expand_entry(const uint32_t *a, const KarLayout &kl, uint32_t *dst, long long *cs, uint32_t *t1,
                         uint32_t *t2, mp::Red &r) {
  for (int l = threadIdx.x; l < kl.stride; l += NT) dst[l] = 0;
  __syncthreads();
  const int W = kl.W, m1 = kl.m1;
  const int l1[3] = {m1, W - m1, max(m1, W - m1) + 1};
  // level-1 sum lo + hi into t1
  for (int l = threadIdx.x; l < l1[2]; l += NT)
    cs[l] = (long long)mp::limb_at(a, m1, l) + (long long)mp::limb_at(a + m1, W - m1, l);
  __syncthreads();
  mp::normalize<NT>(cs, l1[2], t1, r);
  if (kl.levels == 1) {
    for (int l = threadIdx.x; l < l1[0]; l += NT) dst[kl.off[0] + l] = a[l];
    for (int l = threadIdx.x; l < l1[1]; l += NT) dst[kl.off[1] + l] = a[m1 + l];
    for (int l = threadIdx.x; l < l1[2]; l += NT) dst[kl.off[2] + l] = t1[l];
    return;
  }
  for (int u = 0; u < 3; u++) {
    const uint32_t *src = u == 0 ? a : (u == 1 ? a + m1 : t1);
    const int wu = l1[u], m2 = kl.m2[u];
    for (int l = threadIdx.x; l < m2; l += NT) dst[kl.off[3 * u] + l] = src[l];
    for (int l = threadIdx.x; l < wu - m2; l += NT) dst[kl.off[3 * u + 1] + l] = src[m2 + l];
    const int ws = kl.w[3 * u + 2];
    for (int l = threadIdx.x; l < ws; l += NT)
      cs[l] = (long long)mp::limb_at(src, m2, l) + (long long)mp::limb_at(src + m2, wu - m2, l);
    __syncthreads();
    mp::normalize<NT>(cs, ws, t2, r);
    for (int l = threadIdx.x; l < ws; l += NT) dst[kl.off[3 * u + 2] + l] = t2[l];
    __syncthreads();
  }
}

}  // namespace hk
