// Panel kernels of the factorisation: for row i of R
//   S_ij = RNE_P(m_{i+j} - sum_{t<i} R_ti R_tj)   (the sum arrives exactly as
//          column sums from the update kernel, on the grid g_i + g_j)
//   R_ii = RNE_P(sqrt(S_ii)),  R_ij = RNE_P(S_ij / R_ii)
// (section "The LDL^T Determinant Algorithm": the diagonal entry, then the
// column divided by it, CDivDiag[row] = M[row][pc] / M[pc][pc]; here with the
// square root of the Cholesky form).  Each new entry is also written on the
// binary grid of its column for the next updates ("alignment").
#include "hk_internal.h"
#include "hk_kar.cuh"
#include "hk_mp.cuh"
#include "hk_panel.cuh"

namespace hk {

namespace {

constexpr int NT_DIAG = 512;
constexpr int NT_ROW = 256;

// a priori top bit bound of column j: |R_tj| <= sqrt(m_2j) < 2^U_j
__global__ void k_col_tops(int N, int L, MpArr mom, long long *colU, long long top_margin) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  const long long P = 32LL * L;
  const int k = 2 * j;
  long long e = mom.exp[k];
  bool nz = false;
  for (int l = 0; l < L; l++) nz |= mom.limbs[(long long)k * L + l] != 0;
  if (!nz && k > 0) e = mom.exp[k - 1];  // degenerate moment: borrow a neighbour's scale
  colU[j] = ((e + P + 1) >> 1) + 2 + top_margin;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_diag(PanelParams p, int i) {
  if (block_status(p.st) != ST_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RowSmem s;
  if (!HK_CHECK(p.st, carve(nullptr, p.L, p.C, true, nullptr) <= dynamic_smem_bytes(), 11,
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
  if (!HK_CHECK(p.st, crow >= 0 && crow * p.C + p.C <= p.colsum_len, 12, crow * p.C + p.C, p.colsum_len) ||
      !HK_CHECK(p.st, p.kl.levels == 0 || (tri_idx(i, i, N) + 1) * p.kl.stride <= p.aexp_len, 13,
                (tri_idx(i, i, N) + 1) * p.kl.stride, p.aexp_len))
    return;
  int nZ = 0;
  const int sgn = form_exact<NT>(s, colrow, p.C, p.mom.sign[mk], p.mom.exp[mk],
                                      p.mom.limbs + (long long)mk * L, L, 2 * gi, p.st, &nZ);
  if (sgn == 0) {
    if (threadIdx.x == 0) atomicMin(&p.st->range_row, i);
    return;
  }
  const mp::Rounded S = mp::round_rne<NT>(s.Z, nZ, 2 * gi, L, s.mant, w);
  if (!S.nonzero || sgn < 0) {
    if (threadIdx.x == 0) {
      atomicMin(&p.st->bad_row, i);
      atomicCAS(&p.st->code, ST_OK, ST_NOT_PD);
    }
    return;
  }
  mp::NBufs B;
  for (int t = 0; t < 6; t++) (&B.a)[t] = s.nb[t];
  B.cap = s.cap4;
  bool ok = true;
  const mp::Rounded Rr = mp::sqrt_rne<NT>(s.mant, L, S.exp, s.rm, w, B, s.big, s.xs, &ok);
  const long long idx = tri_idx(i, i, N);
  for (int l = threadIdx.x; l < L; l += NT) p.R.limbs[idx * L + l] = s.rm[l];
  if (threadIdx.x == 0) {
    p.R.sign[idx] = 0;
    p.R.exp[idx] = Rr.exp;
    p.Asign[idx] = 0;
    if (!ok) atomicAdd(&p.st->timeout, 1);
  }
  if (!align_entry<NT>(s.rm, L, Rr.exp, false, gi, p.W, p.A + idx * p.W, p.st) && threadIdx.x == 0)
    atomicMin(&p.st->range_row, i);
  __syncthreads();
  if (p.kl.levels > 0)
    expand_entry<NT>(p.A + idx * p.W, p.kl, p.Aexp + idx * p.kl.stride, s.cs, s.Z, s.big, *s.red);
  __syncthreads();
  ok = mp::recip<NT>(s.rm, L, s.V, w, B, RECIP_EXTRA);
  for (int l = threadIdx.x; l < recip_limbs(L); l += NT) p.recip[(long long)i * recip_limbs(L) + l] = s.V[l];
  if (threadIdx.x == 0 && !ok) atomicAdd(&p.st->timeout, 1);
  (void)P;
}

template <int NT>
__global__ void __launch_bounds__(NT) k_offdiag(PanelParams p, int i) {
  if (block_status(p.st) != ST_OK) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  RowSmem s;
  if (!HK_CHECK(p.st, carve(nullptr, p.L, p.C, false, nullptr) <= dynamic_smem_bytes(), 14,
                carve(nullptr, p.L, p.C, false, nullptr), dynamic_smem_bytes()))
    return;
  carve(smem_raw, p.L, p.C, false, &s);
  mp::Work w = work_of(s);
  const int L = p.L, N = p.N;
  const int j = i + 1 + blockIdx.x;
  const long long gi = p.colU[i] - 32LL * p.W;
  const long long gj = p.colU[j] - 32LL * p.W;
  const long long k = i - p.r0;
  const long long crow = k * N - (k * (i + p.r0 - 1)) / 2 + (j - i);
  const long long *colrow = p.colsum + crow * p.C;
  const int mk = i + j;
  if (!HK_CHECK(p.st, j < N, 15, j, N) ||
      !HK_CHECK(p.st, crow >= 0 && crow * p.C + p.C <= p.colsum_len, 16, crow * p.C + p.C, p.colsum_len) ||
      !HK_CHECK(p.st, p.kl.levels == 0 || (tri_idx(i, j, N) + 1) * p.kl.stride <= p.aexp_len, 17,
                (tri_idx(i, j, N) + 1) * p.kl.stride, p.aexp_len))
    return;
  int nZ = 0;
  const int sgn = form_exact<NT>(s, colrow, p.C, p.mom.sign[mk], p.mom.exp[mk],
                                     p.mom.limbs + (long long)mk * L, L, gi + gj, p.st, &nZ);
  if (sgn == 0) {
    if (threadIdx.x == 0) atomicMin(&p.st->range_row, i);
    return;
  }
  const mp::Rounded S = mp::round_rne<NT>(s.Z, nZ, gi + gj, L, s.mant, w);
  const long long idx = tri_idx(i, j, N);
  const long long iidx = tri_idx(i, i, N);
  if (!S.nonzero) {
    for (int l = threadIdx.x; l < L; l += NT) p.R.limbs[idx * L + l] = 0;
    for (int l = threadIdx.x; l < p.W; l += NT) p.A[idx * p.W + l] = 0;
    if (p.kl.levels > 0)
      for (int l = threadIdx.x; l < p.kl.stride; l += NT) p.Aexp[idx * p.kl.stride + l] = 0;
    if (threadIdx.x == 0) {
      p.R.sign[idx] = 0;
      p.R.exp[idx] = 0;
      p.Asign[idx] = 0;
    }
    return;
  }
  for (int l = threadIdx.x; l < L; l += NT) s.rm[l] = p.R.limbs[iidx * L + l];
  for (int l = threadIdx.x; l < recip_limbs(L); l += NT) s.V[l] = p.recip[(long long)i * recip_limbs(L) + l];
  __syncthreads();
  bool ok = true;
  const mp::Rounded Q = mp::div_rne<NT>(s.mant, S.exp, s.rm, p.R.exp[iidx], s.V, L, s.res, w, s.big, s.q, &ok, RECIP_EXTRA);
  for (int l = threadIdx.x; l < L; l += NT) p.R.limbs[idx * L + l] = s.res[l];
  if (threadIdx.x == 0) {
    p.R.sign[idx] = sgn < 0 ? 1 : 0;
    p.R.exp[idx] = Q.exp;
    p.Asign[idx] = sgn < 0 ? 1 : 0;
    if (!ok) atomicAdd(&p.st->timeout, 1);
  }
  const bool fits = align_entry<NT>(s.res, L, Q.exp, false, gj, p.W, p.A + idx * p.W, p.st);
  if (!fits && threadIdx.x == 0) atomicMin(&p.st->range_row, i);
  if (fits && p.kl.levels > 0) {
    __syncthreads();
    expand_entry<NT>(p.A + idx * p.W, p.kl, p.Aexp + idx * p.kl.stride, s.cs, s.Z, s.big, *s.red);
  }
}

// Re-writes the finished entries of rows t < r0 (packed indices [0, E)) on the
// column grids of a widened window: aligned from the floating-point R, then
// expanded.  Lets a window failure resume at its block instead of restarting.
constexpr int NT_RA = 128;
__global__ void __launch_bounds__(NT_RA) k_realign(PanelParams p, long long E) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int t_s;
  const long long e = blockIdx.x;
  if (e >= E) return;
  const int N = p.N, L = p.L;
  if (threadIdx.x == 0) {  // row of packed index e: largest t with tri_idx(t, t) <= e
    int lo = 0, hi = N - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) / 2;
      if (tri_idx(mid, mid, N) <= e) lo = mid; else hi = mid - 1;
    }
    t_s = lo;
  }
  __syncthreads();
  const int t = t_s;
  const int j = (int)(e - tri_idx(t, t, N)) + t;
  const uint32_t *mant = p.R.limbs + e * L;
  bool zero = true;
  for (int l = 0; l < L; l++) zero &= (mant[l] == 0);
  const long long gj = p.colU[j] - 32LL * p.W;
  if (!align_entry<NT_RA>(mant, L, p.R.exp[e], zero, gj, p.W, p.A + e * p.W, p.st)) {
    if (threadIdx.x == 0) atomicMin(&p.st->range_row, t);
    return;
  }
  if (threadIdx.x == 0) p.Asign[e] = p.R.sign[e];
  if (p.kl.levels > 0) {
    __syncthreads();
    const int h1 = p.W / 2 + 8;
    mp::Red *red = reinterpret_cast<mp::Red *>(smem_raw);
    long long *cs = reinterpret_cast<long long *>(smem_raw + ((sizeof(mp::Red) + 15) / 16) * 16);
    uint32_t *t1 = reinterpret_cast<uint32_t *>(cs + h1);
    expand_entry<NT_RA>(p.A + e * p.W, p.kl, p.Aexp + e * p.kl.stride, cs, t1, t1 + h1, *red);
  }
}

}  // namespace

size_t panel_smem_diag(int L, int C) { return carve_size(L, C, true); }
size_t panel_smem_row(int L, int C) { return carve_size(L, C, false); }

cudaError_t launch_col_tops(int N, int L, long long top_margin, MpArr mom, long long *colU, DevStatus *st,
                            cudaStream_t s) {
  (void)st;
  k_col_tops<<<(N + 127) / 128, 128, 0, s>>>(N, L, mom, colU, top_margin);
  return cudaGetLastError();
}

static cudaError_t set_smem(const void *fn, size_t bytes) {
  return bytes > 48 * 1024 ? allow_dynamic_smem(fn) : cudaSuccess;
}

// one CTA of NT_DIAG threads per row (256 and 128 threads measured slower:
// the work of each phase is parallel over result columns)
cudaError_t launch_diag(const PanelParams &p, int i, cudaStream_t s) {
  const size_t smem = panel_smem_diag(p.L, p.C);
  cudaError_t e = set_smem((const void *)k_diag<NT_DIAG>, smem);
  if (e != cudaSuccess) return e;
  k_diag<NT_DIAG><<<1, NT_DIAG, smem, s>>>(p, i);
  return cudaGetLastError();
}

template <int NT>
static cudaError_t launch_offdiag_t(const PanelParams &p, int i, cudaStream_t s) {
  const size_t smem = panel_smem_row(p.L, p.C);
  cudaError_t e = set_smem((const void *)k_offdiag<NT>, smem);
  if (e != cudaSuccess) return e;
  k_offdiag<NT><<<p.N - i - 1, NT, smem, s>>>(p, i);
  return cudaGetLastError();
}

cudaError_t launch_offdiag(const PanelParams &p, int i, cudaStream_t s) {
  if (i + 1 >= p.N) return cudaSuccess;
  return launch_offdiag_t<NT_ROW>(p, i, s);
}

cudaError_t launch_realign(const PanelParams &p, int r0, cudaStream_t s) {
  const long long E = tri_idx(r0, r0, p.N);
  if (r0 <= 0 || E <= 0) return cudaSuccess;
  const int h1 = p.W / 2 + 8;
  const size_t smem = ((sizeof(mp::Red) + 15) / 16) * 16 + (size_t)h1 * 8 + (size_t)h1 * 4 * 2;
  cudaError_t e = set_smem((const void *)k_realign, smem);
  if (e != cudaSuccess) return e;
  k_realign<<<(unsigned)E, NT_RA, smem, s>>>(p, E);
  return cudaGetLastError();
}

}  // namespace hk
