// Host-side declarations shared by the libhk translation units.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "hk_common.cuh"

namespace hk {

// ---- exact contraction (hk_update.cu) ----------------------------------------
// Stripe width (columns per thread) and p-steps per work unit.
constexpr int UC = 9;
constexpr int UPC = 36;
constexpr int UNT = 256;      // compute threads per CTA
constexpr int USTAGES = 4;    // shared-memory pipeline depth

struct Unit {
  int d0;  // first column of the stripe
  int p0;  // first p (limb index of the X operand)
};

enum UpdMode { M_FACTOR = 0, M_GEMV_FWD = 1, M_GEMV_BACK = 2, M_DOT = 3 };

struct UpdParams {
  int mode;
  int N;
  const uint32_t *A;       // aligned R entries, W limbs each (packed upper triangle)
  const int32_t *Asign;
  int W;
  const uint32_t *Vx;      // aligned vectors, Wv limbs per entry
  const int32_t *Vxsign;
  const uint32_t *Vy;
  const int32_t *Vysign;
  int Wv;
  int Wx, Wy;              // operand widths of this launch
  int r0;                  // first row of the current block (output indexing)
  int ra, rb;              // output rows [ra, rb)
  int nout;                // number of outputs
  int t0, t1;              // contraction range [t0, t1)
  int tchunk;              // t per CTA (z dimension)
  long long *colsum;       // [outputs][C] signed 64-bit column sums (accumulated)
  int C;
  const Unit *units;
  int nunits;
  DevStatus *st;
};

// Number of work units and the unit table for operand widths (Wx, Wy).
int build_units(int Wx, int Wy, Unit *host_out, int cap);
int colsum_width(int Wx, int Wy);
cudaError_t launch_update(const UpdParams &p, cudaStream_t s);

// ---- panel kernels (hk_panel.cu) ------------------------------------------------
struct PanelParams {
  int N, L, W, C;
  MpArr mom;               // moments (2N-1)
  const long long *colU;   // column top bounds U_j  (grid g_j = U_j - 32 W)
  MpArr R;                 // R in floating form (packed)
  uint32_t *A;             // aligned entries (packed), W limbs
  int32_t *Asign;
  uint32_t *recip;         // [N][L+2] floor(2^(2P+1)/mant(R_ii))
  const long long *colsum; // [block outputs][C]
  int r0;                  // block base row
  DevStatus *st;
};
cudaError_t launch_col_tops(int N, int L, long long top_margin, MpArr mom, long long *colU, DevStatus *st,
                            cudaStream_t s);
cudaError_t launch_diag(const PanelParams &p, int i, cudaStream_t s);
cudaError_t launch_offdiag(const PanelParams &p, int i, cudaStream_t s);
size_t panel_smem_diag(int L, int C);
size_t panel_smem_row(int L, int C);

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
};
cudaError_t launch_solve_entry(const SolveParams &p, int i, cudaStream_t s);
cudaError_t launch_vec_exprange(int n, MpArr v, int L, const long long *colU, int scaled,
                                long long *out2, cudaStream_t s);
cudaError_t launch_vec_align(int n0, int n1, MpArr v, int L, const long long *colU, int scaled,
                             long long h, int Wv, uint32_t *vecA, int32_t *vecAsign,
                             DevStatus *st, cudaStream_t s);
cudaError_t launch_lambda(int L, const long long *colsum, int C, long long hv, long long hw,
                          MpArr lam, int slot, DevStatus *st, cudaStream_t s);
cudaError_t launch_vec_normalise(int n, MpArr w, MpArr v, int L, cudaStream_t s);
cudaError_t launch_set_ones(int n, MpArr v, int L, cudaStream_t s);

// ---- self test (hk_selftest.cu) ---------------------------------------------------
int selftest_mp(int op, int L, const uint32_t *x, int nx, int64_t ex, const uint32_t *y, int ny,
                int64_t ey, uint32_t *out, int64_t *eo);

}  // namespace hk
