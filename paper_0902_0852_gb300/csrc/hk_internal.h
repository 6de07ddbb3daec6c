// Host-side declarations shared by the libhk translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "hk_common.cuh"

namespace hk {

// Let kernel `fn` use all the opt-in shared memory of the current device, once
// per (kernel, device) under a process-wide lock.  Launchers call it instead of
// setting the limit to their own size: with several host threads launching the
// same kernel with different sizes, per-size updates would race (one thread
// lowering the limit while another launches with more).
cudaError_t allow_dynamic_smem(const void *fn);

// ---- exact contraction (hk_update.cu) ----------------------------------------
// Stripe width (columns per thread) and p-steps per work unit.
constexpr int UC = 9;          // default stripe width (result columns per thread)
constexpr int UC_MAX = 13;
constexpr int UPC = 36;        // default p-steps per unit (a multiple of the stripe width)
constexpr int UNT = 256;       // compute threads per CTA
constexpr int USTAGES = 4;     // default shared-memory pipeline depth
constexpr int USTAGES_MAX = 8; // deepest ring a launch may use
constexpr int MAX_KAR = 4;     // Karatsuba levels of the expansion
constexpr int MAX_SUB = 81;    // sub-contractions per launch (3^levels)
constexpr int MAX_TERMS = 16;  // result positions a sub-contraction is added to (2^levels)
constexpr int MAX_SPLITS = 40; // split points of all levels (1 + 3 + 9 + 27)
// first split of level lv (1-based) in KarLayout::ms: (3^(lv-1) - 1) / 2
__host__ __device__ inline int split_base(int lv) {
  int b = 0, n = 1;
  for (int l = 1; l < lv; l++, n *= 3) b += n;
  return b;
}
constexpr int MAX_XB = 64;     // blocks per output with their own operand window
// Guard bits of the stored row reciprocals floor(2^(2P+1+RECIP_EXTRA)/mant(R_ii)):
// with them a correctly rounded division rarely needs its exact remainder.
constexpr int RECIP_EXTRA = 64;
__host__ __device__ inline int recip_limbs(int L) { return L + 2 + RECIP_EXTRA / 32; }

struct Unit {
  int d0;  // first column of the stripe, sub-contraction index in bits 24..31
  int p0;  // first p (limb index of the X operand)
};

// M_LDLT: the shifted LDL^T of the paper's determinant -- X from the aligned
// columns C (A, Asign), Y from the aligned quotients CDivDiag (B, Bsign)
enum UpdMode { M_FACTOR = 0, M_GEMV_FWD = 1, M_GEMV_BACK = 2, M_DOT = 3, M_LDLT = 4 };

// One integer contraction sum_t X_t[xoff..xoff+wx) * Y_t[yoff..yoff+wy), added
// to the output's column sums at each (column offset, sign) term.
struct SubProb {
  int xoff, yoff;          // limb offset of the operand pieces inside an entry
  int wx, wy;              // widths of the pieces in limbs
  int nterm;
  int toff[MAX_TERMS];
  int tsign[MAX_TERMS];
};

// Karatsuba expansion of an aligned entry of W limbs (levels 0 to 4):
// pieces lo, hi, lo+hi (recursively), each stored in its own slot with zero
// gaps of G limbs on both sides, so that one entry is one contiguous copy.
// Piece k of the last level is the base-3 path (lo = 0, hi = 1, lo+hi = 2)
// through the levels, most significant digit first.
struct KarLayout {
  int levels;
  int W;
  int npieces;
  int ms[MAX_SPLITS];      // split points: level lv's piece u splits at ms[split_base(lv) + u]
  int off[MAX_SUB];        // slot offsets (limbs)
  int w[MAX_SUB];          // piece widths
  int G;                   // gap (limbs)
  int stride;              // expanded entry size (limbs)
};

struct UpdParams {
  int mode;
  int N;
  const uint32_t *A;       // R entries (plain, or expanded), packed upper triangle
  const int32_t *Asign;
  const uint32_t *B;       // M_LDLT: the second operand triangle (same layout as A)
  const int32_t *Bsign;
  int astride;             // limbs per A entry
  const uint32_t *Vx;      // aligned vectors
  const int32_t *Vxsign;
  const uint32_t *Vy;
  const int32_t *Vysign;
  int vstride;             // limbs per vector entry
  int cx, cy;              // limbs copied per X / Y entry
  int uc;                  // stripe width of the unit table (7, 9, 11 or 13)
  int upc;                 // p-steps per unit (a multiple of uc)
  int nsub;
  int r0;                  // first row of the current block (output indexing)
  int ra, rb;              // output rows [ra, rb)
  int nout;                // number of outputs
  int t0, t1;              // contraction range [t0, t1)
  int tchunk;              // t per CTA (z dimension)
  int nst;                 // pipeline stages of the launch (2..USTAGES_MAX; set by the launcher)
  long long wait_ns;       // limit of each bounded device wait (0: the default, 2 s)
  long long *colsum;       // [outputs][C] signed 64-bit column sums (accumulated)
  int C;
  long long a_len, vx_len, vy_len, colsum_len;  // buffer sizes (limbs / entries), for checked builds
  const Unit *units;
  int nunits;
  DevStatus *st;
  // Per-block operand windows (Karatsuba launches): block x stages only limbs
  // [xlo[x], xlo[x] + xlen[x]) of each expanded entry -- the pieces its units
  // read plus one zero gap on each side.  nxb = 0: whole entries (cx, cy).
  int nxb;
  int xlo[MAX_XB], xlen[MAX_XB];
  // the sub-contractions, in the launch parameters (about 12 KB at 81 pieces),
  // last so that every other field keeps a small offset: the unit loop reads
  // them through the constant cache; a table in device memory measured 10%
  // slower, one packed into 16-bit fields 12% slower
  SubProb sub[MAX_SUB];
};

// Host-side schedule helpers.
void kar_layout(int W, int levels, int gap, KarLayout *kl);
int kar_subprobs(const KarLayout &kl, SubProb *sub);   // returns the count
int build_units(const SubProb *sub, int nsub, int uc, int upc, Unit *host_out, int cap);
// Operand windows of the blocks of a Karatsuba launch (pieces separated by
// zero gaps of `gap` limbs inside entries of `stride` limbs): fills xlo/xlen
// for the (n + 255) / 256 blocks and returns the longest window, or 0 when the
// launch has one sub-problem or too many blocks (whole entries are staged).
int operand_windows(const SubProb *sub, int nsub, const Unit *units, int n, int gap, int stride, int *xlo,
                    int *xlen);
void choose_schedule(const SubProb *sub, int nsub, int upc_cap, int *uc, int *upc);
int choose_levels(int W, int gap, bool allow4);  // Karatsuba depth of least modelled update cost
int colsum_width(const SubProb *sub, int nsub, int uc);
cudaError_t launch_update(const UpdParams &p, cudaStream_t s);
// One block waits (bounded by wait_ns, 0 = default) on an mbarrier that nothing
// arrives at, with the update kernel's wait routine; records the timeout in st.
cudaError_t launch_wait_selftest(DevStatus *st, long long wait_ns, cudaStream_t s);
// INT8 tensor-core (mma.sync u8) form of the FACTOR update, plain entries
cudaError_t launch_update_i8(const UpdParams &p, cudaStream_t s);
size_t update_i8_smem(int W);

// ---- panel kernels (hk_panel.cu) ------------------------------------------------
struct PanelParams {
  int N, L, W, C;
  KarLayout kl;            // expansion written next to each aligned entry (levels > 0)
  uint32_t *Aexp;
  MpArr mom;               // moments (2N-1)
  const long long *colU;   // column top bounds U_j  (grid g_j = U_j - 32 W)
  MpArr R;                 // R in floating form (packed)
  uint32_t *A;             // aligned entries (packed), W limbs
  int32_t *Asign;
  uint32_t *recip;         // [N][recip_limbs(L)] floor(2^(2P+1+RECIP_EXTRA)/mant(R_ii))
  const long long *colsum; // [block outputs][C]
  int r0;                  // block base row
  DevStatus *st;
  long long colsum_len, aexp_len;  // buffer sizes, for checked builds
};
cudaError_t launch_col_tops(int N, int L, long long top_margin, MpArr mom, long long *colU, DevStatus *st,
                            cudaStream_t s);
cudaError_t launch_diag(const PanelParams &p, int i, cudaStream_t s);
cudaError_t launch_offdiag(const PanelParams &p, int i, cudaStream_t s);
// Re-align (and expand) the finished entries of rows t < r0 on the current
// column grids, from the floating-point R.
cudaError_t launch_realign(const PanelParams &p, int r0, cudaStream_t s);
size_t panel_smem_diag(int L, int C);
size_t panel_smem_row(int L, int C);

// ---- shifted LDL^T, Secant and verification (hk_ldlt.cu) ------------------------
struct LdlParams {
  PanelParams pp;          // moments, grids, C entries (R slots; D_t on the diagonal), aligned
                           // and expanded C (A, Aexp), reciprocals of |D_t|, column sums
  MpArr Q;                 // CDivDiag Q_t[r] in floating form (packed, off-diagonal)
  uint32_t *B;             // Q aligned on the column grids shifted by -h_t (W limbs)
  int32_t *Bsign;
  uint32_t *Bexp;          // Karatsuba expansion of B
  long long *h;            // row shifts h_t
  MpArr x;                 // the shift (one entry)
  int xzero;               // x = 0
  MpArr det;               // running determinant (one entry)
  int *negcount;           // negative pivots so far
  int *zero_row;           // first zero pivot (atomicMin)
};
cudaError_t launch_ldl_pivot(const LdlParams &q, int i, cudaStream_t s);
cudaError_t launch_ldl_row(const LdlParams &q, int i, cudaStream_t s);
size_t scalar_work_bytes(int L);
cudaError_t launch_secant_step(MpArr xs, MpArr ps, MpArr tmpv, int k1, int k2, int k3, int kstep, int have_last,
                               int L, void *work, int *flags, cudaStream_t s);
cudaError_t launch_neg_min_pivot(MpArr R, int N, int L, MpArr dst, int kd, cudaStream_t s);
cudaError_t launch_scale_pm(MpArr src, int ks, int L, int bits, int sgn, MpArr dst, int kd, int L2, cudaStream_t s);
cudaError_t launch_widen(MpArr src, int n, int L, MpArr dst, int L2, cudaStream_t s);
cudaError_t launch_scalar_selftest(int op, MpArr a, MpArr b, MpArr out, int L, void *work, int *flags,
                                  cudaStream_t s);

// ---- solve kernels (hk_solve.cu) -------------------------------------------------
struct SolveParams {
  int N, L, W, C, Wv;
  MpArr R;
  const uint32_t *recip;
  const long long *colU;
  MpArr rhs;               // v (forward) or y (back)
  MpArr out;               // y (forward) or w (back)
  uint32_t *vecA;          // aligned solution entries [N][Wv]
  int32_t *vecAsign;
  long long h;             // grid exponent of vecA
  const long long *colsum; // [block rows][C]
  int r0;
  int back;                // 0 forward, 1 back
  int nosum;               // first entry of a solve: no sum, no aligned copy
  DevStatus *st;
  long long vec_len, colsum_len;  // buffer sizes, for checked builds
  KarLayout kl;            // levels > 0: also write the Karatsuba expansion of the aligned copy
  uint32_t *vecAexp;       // [N][kl.stride] expanded aligned entries (Wv = kl.W)
};
cudaError_t launch_solve_entry(const SolveParams &p, int i, cudaStream_t s);
// All rows [B0, B1) of a solve block in one single-CTA launch, in-block terms
// from the plain aligned entries A (W limbs) and their signs (low precision).
cudaError_t launch_solve_block(const SolveParams &p, const uint32_t *A, const int32_t *Asign, int B0, int B1,
                               cudaStream_t s);
size_t solve_block_smem(int L, int C, int W, int Wv, int nb);
cudaError_t launch_vec_exprange(int n, MpArr v, int L, const long long *colU, int scaled,
                                long long *out2, cudaStream_t s);
cudaError_t launch_vec_align(int n0, int n1, MpArr v, int L, const long long *colU, int scaled,
                             long long h, int Wv, uint32_t *vecA, int32_t *vecAsign,
                             DevStatus *st, long long vec_len, cudaStream_t s);
cudaError_t launch_lambda(int L, const long long *colsum, int C, long long hv, long long hw,
                          MpArr lam, int slot, DevStatus *st, long long colsum_len, cudaStream_t s);
cudaError_t launch_vec_normalise(int n, MpArr w, MpArr v, int L, cudaStream_t s);
// Karatsuba expansion of aligned vector entries [n0, n1) (kl.W limbs each) into
// dst (kl.stride limbs each).
cudaError_t launch_vec_expand(int n0, int n1, const uint32_t *vecA, const KarLayout &kl, uint32_t *dst,
                              cudaStream_t s);
cudaError_t launch_set_ones(int n, MpArr v, int L, cudaStream_t s);

// ---- self test (hk_selftest.cu) ---------------------------------------------------
int selftest_mp(int op, int L, const uint32_t *x, int nx, int64_t ex, const uint32_t *y, int ny,
                int64_t ey, uint32_t *out, int64_t *eo);

}  // namespace hk
