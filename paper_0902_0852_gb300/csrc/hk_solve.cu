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
  bool vz = true;
  for (int l = 0; l < L; l++) vz &= (vl[l] == 0);
  long long sh = ev - G;
  if (vz) sh = 0;
  if (sh < 0) {
    if (threadIdx.x == 0) raise_range(st, -sh);
    return 0;
  }
  const long long q = sh >> 5;
  const int b = (int)(sh & 31);
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
__global__ void __launch_bounds__(NT_SOLVE) k_solve_entry(SolveParams p, int i) {
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
  const int sgn = form_exact_s<NT_SOLVE>(s, colrow, p.C, p.rhs.sign[i], p.rhs.exp[i],
                                         p.rhs.limbs + (long long)i * L, L, G, p.st, &nZ);
  if (sgn == 0) return;
  const mp::Rounded S = mp::round_rne<NT_SOLVE>(s.Z, nZ, G, L, s.mant, w);
  uint32_t *outl = p.out.limbs + (long long)i * L;
  uint32_t *va = p.vecA + (long long)i * p.Wv;
  if (!S.nonzero) {
    for (int l = threadIdx.x; l < L; l += NT_SOLVE) outl[l] = 0;
    if (!p.nosum)
      for (int l = threadIdx.x; l < p.Wv; l += NT_SOLVE) va[l] = 0;
    if (threadIdx.x == 0) {
      p.out.sign[i] = 0;
      p.out.exp[i] = 0;
      p.vecAsign[i] = 0;
    }
    return;
  }
  const long long iidx = tri_idx(i, i, N);
  for (int l = threadIdx.x; l < L; l += NT_SOLVE) s.rm[l] = p.R.limbs[iidx * L + l];
  for (int l = threadIdx.x; l < L + 2; l += NT_SOLVE) s.V[l] = p.recip[(long long)i * (L + 2) + l];
  __syncthreads();
  bool ok = true;
  const mp::Rounded Q =
      mp::div_rne<NT_SOLVE>(s.mant, S.exp, s.rm, p.R.exp[iidx], s.V, L, s.res, w, s.big, s.q, &ok);
  for (int l = threadIdx.x; l < L; l += NT_SOLVE) outl[l] = s.res[l];
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
  mp::shl<NT_SOLVE>(s.res, L, sh, va, p.Wv);
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
  bool ok = mp::recip<NT_LAM>(s.rm, L, s.V, w, B);
  bool ok2 = true;
  const mp::Rounded Q = mp::div_rne<NT_LAM>(s.mant, VV.exp, s.rm, VW.exp, s.V, L, s.res, w, s.big, s.q, &ok2);
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

cudaError_t launch_solve_entry(const SolveParams &p, int i, cudaStream_t s) {
  const size_t smem = ssmem_size(p.L, p.C, false);
  cudaError_t e = set_smem((const void *)k_solve_entry, smem);
  if (e != cudaSuccess) return e;
  k_solve_entry<<<1, NT_SOLVE, smem, s>>>(p, i);
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

cudaError_t launch_set_ones(int n, MpArr v, int L, cudaStream_t s) {
  k_set_ones<<<64, 256, 0, s>>>(n, v, L);
  return cudaGetLastError();
}

}  // namespace hk
