// libhk C ABI: context, device memory, and the order of kernel launches of the
// factorisation and of inverse iteration.  All arithmetic of the method runs
// in the kernels (hk_update.cu, hk_panel.cu, hk_solve.cu); this file only
// sequences launches, sizes exact-accumulation windows and moves data.
#include "hk.h"
#include "hk_internal.h"

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <climits>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <utility>
#include <vector>

using namespace hk;

// largest precision whose panel work areas fit in one block's shared memory
static const int HK_MAX_P = 32768;
static const int HK_MAX_WV = 12000;  // widest solve vector window (limbs) the update tiles can stage

namespace {

struct Arena {
  char *base = nullptr;  // caller workspace (bump allocation) or null
  size_t cap = 0, used = 0;
  std::vector<void *> owned;
  cudaError_t get(void **p, size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    if (bytes == 0) bytes = 256;
    if (base) {
      if (used + bytes > cap) return cudaErrorMemoryAllocation;
      *p = base + used;
      used += bytes;
      return cudaSuccess;
    }
    cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) owned.push_back(*p);
    return e;
  }
  void release() {
    for (void *p : owned) cudaFree(p);
    owned.clear();
  }
};

struct EvPair {
  cudaEvent_t a = nullptr, b = nullptr;
};

// unit table and schedule of the update kernel for one operand shape
struct Sched {
  Unit *units;
  int n, uc, upc;
  int nsub;
  SubProb sub[MAX_SUB];
  int C;  // column sums per output
  int nxb, maxlen;  // per-block operand windows (Karatsuba), see UpdParams
  int xlo[MAX_XB], xlen[MAX_XB];
};

// gap between Karatsuba pieces: covers the zero padding a unit reads past a
// piece (stripe width + chunk length)
constexpr int KAR_GAP = 64;

}  // namespace

struct hk_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Arena base_arena, fac_arena, sol_arena;
  Arena res_arena;          // R, its signs and the reciprocals: kept across window widenings
  int res_N = 0, res_L = 0;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  // problem
  int N = 0, L = 0, P = 0, bnum = 1, bden = 1;
  bool loaded = false, factored = false;
  int W = 0, C = 0, nb = 16, nbs = 16;
  MpArr mom{};
  long long *colU = nullptr, *colG = nullptr;
  DevStatus *st = nullptr;
  long long *d_range = nullptr;
  // factor buffers
  MpArr R{};
  uint32_t *A = nullptr;
  uint32_t *Aexp = nullptr;  // Karatsuba expansion of A (levels > 0)
  KarLayout kl{};
  int kar_levels = -1;       // Karatsuba levels of the factor update (-1: chosen per window)
  int lv_W = -1, lv_auto = 0;  // cached automatic choice for window lv_W
  bool lv_big = false;         // ... and for a factorisation of at least 768 rows
  int update_path = 0;       // 0: IMAD product scanning, 1: INT8 mma.sync
  bool use_graph = false;    // capture each factorisation in a CUDA graph
  cudaStream_t cap_stream = nullptr;  // capture stream when `stream` is a default stream
  int max_iters = 200;       // step cap of hk_smallest_eig(iters = 0)
  long long wait_ns = 0;     // limit of each bounded device wait (0: the kernels' default, 2 s)
  float *pred_params = nullptr;  // predictor network on the device (hk_set_predictor)
  double pred_scales[10] = {0};
  float *pred_buf = nullptr;     // inputs and outputs of hk_predict
  int pred_cap = 0;
  long long fuse_ww = 160000;  // solve blocks run in one launch when W * Wv is at most this
  long long solve_margin = 256;  // first-attempt margin of a solve block's vector window (bits)
  long long wv_max = 0, wv_sum = 0, wv_count = 0;  // solve window widths of the last eig
  int eig_converged = 0;     // last hk_smallest_eig(iters = 0) met the convergence test
  bool autotune = false;     // time candidate update schedules per shape
  long long graph_launches = 0;
  int32_t *Asign = nullptr;
  uint32_t *recip = nullptr;
  long long *colsum = nullptr;
  long long A_len = 0, Aexp_len = 0, colsum_len = 0;  // sizes of A, Aexp (limbs) and colsum (entries)
  int fac_N = 0, fac_L = 0, fac_W = 0, fac_levels = -1;  // shape of the factor buffers
  std::map<std::pair<long long, long long>, Sched> sched_cache;
  // solve buffers
  MpArr v{}, y{}, w{}, hist{};
  int hist_cap = 0, hist_count = 0;
  uint32_t *vecA = nullptr, *vecB = nullptr;
  // second vector set of the solve lookahead: the next block's far GEMV is
  // prepared in it while the current block's entries are computed
  uint32_t *vecA2 = nullptr, *vecA2exp = nullptr;
  int32_t *vecA2sign = nullptr;
  long long *colsum_s2 = nullptr;
  long long pf_hits = 0, pf_miss = 0;  // prepared GEMVs used / dropped in the last eig
  long long pf_ctas = 0;  // blocks per prepared GEMV launch (0: as the block's own GEMV)
  uint32_t *vecAexp = nullptr;  // Karatsuba expansion of vecA (solves on the factor's window)
  size_t vecAexp_cap = 0;       // limbs
  int32_t *vecAsign = nullptr, *vecBsign = nullptr;
  size_t vec_cap = 0;  // limbs per vector buffer
  long long *colsum_s = nullptr;
  size_t colsum_s_cap = 0;  // int64 entries
  bool sol_ready = false;
  // timing / stats
  std::vector<EvPair> evpool;
  size_t evused = 0;
  std::vector<int> evkind;  // 0 update, 1 panel, 2 solve
  double t_phase[3] = {0, 0, 0};
  double t_factor = 0, t_eig = 0;
  long long launches = 0;
  int widenings = 0;
  int resumes = 0;  // widenings that resumed at a later block instead of restarting
  long long top_margin = 0;  // extra bits above the a priori column bounds
  bool timing = true;
  // lookahead: the far part of the next block's update (rows two blocks back and
  // earlier) runs on a low-priority stream while the current block's
  // sequential panel chain runs on a high-priority one; in the solves, the next
  // block's GEMV against all but the current block's entries
  bool lookahead = true;
  cudaStream_t la_hi = nullptr, la_lo = nullptr;
  std::vector<cudaEvent_t> la_ev;
  cudaEvent_t sv_fork = nullptr, sv_done = nullptr, sv_join = nullptr;
  // shifted LDL^T of M - xI (the paper's determinant), Secant and verification
  bool ldl_mode = false;     // the factor driver runs the LDL^T instead of Cholesky
  Arena ldl_arena, ldl_small;
  MpArr Qf{};                // CDivDiag in floating form
  uint32_t *B = nullptr, *Bexp = nullptr;  // aligned (and expanded) CDivDiag
  int32_t *Bsign = nullptr;
  long long *hrow = nullptr;  // row shifts h_t
  MpArr ldl_x{}, ldl_det{};  // the shift and the determinant (one entry each)
  int *ldl_cnt = nullptr;    // [0] negative pivots, [1] first zero pivot
  int ldl_N = 0, ldl_L = 0, ldl_W = 0, ldl_levels = -1, ldl_sL = 0;
  int ldl_xzero = 1;
  bool ldl_ready = false;    // R slots hold the last LDL^T (hk_get_ldlt_flat)
  Arena sec_arena;
  MpArr sec_x{}, sec_p{}, sec_t{};  // iterates, determinants, scratch values
  void *sec_work = nullptr;
  int *sec_flags = nullptr;
  int sec_cap = 0, sec_L = 0, sec_count = 0;
};

namespace {

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HK_OK;
  if (e == cudaErrorMemoryAllocation) return HK_ERR_OOM;
  return HK_ERR_CUDA;
}

#ifdef HK_CHECKED
#define CK(x)                                                                                 \
  do {                                                                                        \
    cudaError_t e_ = (x);                                                                     \
    if (e_ != cudaSuccess) {                                                                  \
      fprintf(stderr, "[hk checked] %s:%d %s -> %s\n", __FILE__, __LINE__, #x, cudaGetErrorString(e_)); \
      return cuda_status(e_);                                                                 \
    }                                                                                         \
  } while (0)
#else
#define CK(x)                                  \
  do {                                         \
    cudaError_t e_ = (x);                      \
    if (e_ != cudaSuccess) return cuda_status(e_); \
  } while (0)
#endif

#ifdef HK_CHECKED
// Checked build: after every launch, wait for it and report a fault or a
// failed bounds check with the launch that caused it (stderr), then stop.
int dbg_after(hk_ctx *c, const char *what, long long a, long long b) {
  const cudaError_t e = cudaStreamSynchronize(c->stream);
  const cudaError_t l = cudaGetLastError();
  DevStatus s{};
  if (e == cudaSuccess) {
    cudaMemcpyAsync(&s, c->st, sizeof(s), cudaMemcpyDeviceToHost, c->stream);
    cudaStreamSynchronize(c->stream);
  }
  if (e != cudaSuccess || l != cudaSuccess || s.check_site) {
    fprintf(stderr,
            "[hk checked] %s (%lld, %lld) N=%d L=%d W=%d: sync=%s last=%s check_site=%d a=%lld b=%lld\n", what,
            a, b, c->N, c->L, c->W, cudaGetErrorString(e), cudaGetErrorString(l), s.check_site, s.check_a,
            s.check_b);
    return e != cudaSuccess || l != cudaSuccess ? HK_ERR_CUDA : HK_ERR_RANGE;
  }
  return HK_OK;
}
#define DBG(c, what, a, b)                               \
  do {                                                   \
    const int r_ = dbg_after((c), (what), (a), (b));     \
    if (r_ != HK_OK) return r_;                          \
  } while (0)
#else
#define DBG(c, what, a, b) \
  do {                     \
  } while (0)
#endif

cudaError_t arena_get(hk_ctx *c, Arena &a, void **p, size_t bytes) {
  if (c->ws) {
    // all arenas share the caller workspace through the base arena
    return c->base_arena.get(p, bytes);
  }
  return a.get(p, bytes);
}

template <typename T>
cudaError_t alloc(hk_ctx *c, Arena &a, T **p, size_t count) {
  void *q = nullptr;
  cudaError_t e = arena_get(c, a, &q, count * sizeof(T));
  *p = reinterpret_cast<T *>(q);
  return e;
}

cudaError_t alloc_mp(hk_ctx *c, Arena &a, MpArr *m, size_t count, int L) {
  cudaError_t e = alloc(c, a, &m->sign, count);
  if (e == cudaSuccess) e = alloc(c, a, &m->exp, count);
  if (e == cudaSuccess) e = alloc(c, a, &m->limbs, count * (size_t)L);
  return e;
}

int round4(long long x) { return (int)((x + 3) / 4 * 4); }

// --- event timing ---------------------------------------------------------------
void ev_begin(hk_ctx *c, int kind, cudaStream_t s);
void ev_end(hk_ctx *c, cudaStream_t s);
void ev_begin(hk_ctx *c, int kind) { ev_begin(c, kind, c->stream); }
void ev_end(hk_ctx *c) { ev_end(c, c->stream); }
void ev_begin(hk_ctx *c, int kind, cudaStream_t s) {
  if (!c->timing) return;
  if (c->evused == c->evpool.size()) {
    EvPair p;
    if (cudaEventCreate(&p.a) != cudaSuccess || cudaEventCreate(&p.b) != cudaSuccess) {
      // no more events: stop timing this context rather than record on a bad handle
      if (p.a) cudaEventDestroy(p.a);
      c->timing = false;
      return;
    }
    c->evpool.push_back(p);
  }
  if (c->evkind.size() < c->evpool.size()) c->evkind.resize(c->evpool.size());
  c->evkind[c->evused] = kind;
  cudaEventRecord(c->evpool[c->evused].a, s);
}
void ev_end(hk_ctx *c, cudaStream_t s) {
  if (!c->timing || c->evused >= c->evpool.size()) return;
  cudaEventRecord(c->evpool[c->evused].b, s);
  c->evused++;
}
void ev_collect(hk_ctx *c) {
  for (size_t k = 0; k < c->evused; k++) {
    float ms = 0;
    cudaEventElapsedTime(&ms, c->evpool[k].a, c->evpool[k].b);
    c->t_phase[c->evkind[k]] += ms;
  }
  c->evused = 0;
}

// ---- autotuner ---------------------------------------------------------------
// Measured best (stripe width, chunk length) of the factor update per operand
// shape, shared by all contexts of the process.
std::mutex g_tune_mu;
std::map<std::pair<long long, long long>, std::pair<int, int>> g_tune;

__global__ void k_fill_random(uint32_t *x, size_t n, uint32_t seed) {
  for (size_t k = blockIdx.x * (size_t)blockDim.x + threadIdx.x; k < n; k += (size_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)k * 2654435761u ^ seed;
    h ^= h >> 16;
    h *= 0x7feb352du;
    h ^= h >> 15;
    x[k] = h;
  }
}

// Times every candidate schedule on a synthetic update (random operands; the
// result is discarded) of the same sub-problem shapes: rows 64..79 of an
// 80-row packed triangle against its first 64 rows.  Returns false on error.
bool autotune_schedule(hk_ctx *c, const SubProb *sub, int nsub, int stride, int upc_cap, int *uc_out,
                       int *upc_out) {
  const int Nt = 80, r0 = 64, r1 = 80;
  const size_t NTt = (size_t)Nt * (Nt + 1) / 2;
  uint32_t *A = nullptr;
  int32_t *Asign = nullptr;
  long long *cs = nullptr;
  DevStatus *st = nullptr;
  Unit *units = nullptr;
  const int C = colsum_width(sub, nsub, 7) + 64;
  long long nout = 0;
  for (int i = r0; i < r1; i++) nout += Nt - i;
  bool ok = cudaMalloc(&A, NTt * stride * 4) == cudaSuccess && cudaMalloc(&Asign, NTt * 4) == cudaSuccess &&
            cudaMalloc(&cs, (size_t)nout * C * 8 * 2) == cudaSuccess && cudaMalloc(&st, sizeof(DevStatus)) == cudaSuccess;
  const int cap = build_units(sub, nsub, 7, 14, nullptr, 0) + 16;  // the most units of any candidate
  ok = ok && cudaMalloc(&units, (size_t)cap * sizeof(Unit)) == cudaSuccess;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (ok) {
    k_fill_random<<<256, 256, 0, c->stream>>>(A, NTt * stride, 12345u);
    cudaMemsetAsync(Asign, 0, NTt * 4, c->stream);
    cudaMemsetAsync(st, 0, sizeof(DevStatus), c->stream);
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
  }
  float best = 1e30f;
  const int ucs[4] = {7, 8, 9, 11};
  for (int ui = 0; ui < 4 && ok; ui++) {
    const int uc = ucs[ui];
    for (int upc = 2 * uc; upc <= 8 * uc && upc <= upc_cap && ok; upc += uc) {
      const int n = build_units(sub, nsub, uc, upc, nullptr, 0);
      if (n > cap) continue;
      std::vector<Unit> h(n);
      build_units(sub, nsub, uc, upc, h.data(), n);
      ok = cudaMemcpyAsync(units, h.data(), sizeof(Unit) * n, cudaMemcpyHostToDevice, c->stream) == cudaSuccess;
      UpdParams up;
      std::memset(&up, 0, sizeof(up));
      up.wait_ns = c->wait_ns;
      const int maxlen = operand_windows(sub, nsub, h.data(), n, ((KAR_GAP + 3) / 4) * 4, stride, up.xlo, up.xlen);
      up.nxb = maxlen > 0 ? (n + UNT - 1) / UNT : 0;
      up.mode = M_FACTOR;
      up.N = Nt;
      up.A = A;
      up.Asign = Asign;
      up.astride = stride;
      up.cx = up.cy = up.nxb ? maxlen : stride;
      up.uc = uc;
      up.upc = upc;
      up.nsub = nsub;
      for (int k = 0; k < nsub; k++) up.sub[k] = sub[k];
      up.r0 = r0;
      up.ra = r0;
      up.rb = r1;
      up.nout = (int)nout;
      up.t0 = 0;
      up.t1 = r0;
      up.tchunk = r0;
      up.colsum = cs;
      up.C = C;
      up.a_len = (long long)NTt * stride;
      up.colsum_len = nout * C * 2;
      up.units = units;
      up.nunits = n;
      up.st = st;
      float t_best = 1e30f;
      for (int rep = 0; rep < 3 && ok; rep++) {
        cudaEventRecord(e0, c->stream);
        ok = launch_update(up, c->stream) == cudaSuccess;
        cudaEventRecord(e1, c->stream);
        ok = ok && cudaEventSynchronize(e1) == cudaSuccess;
        float ms = 0;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) t_best = std::min(t_best, ms);
      }
      if (ok && t_best < best) {
        best = t_best;
        *uc_out = uc;
        *upc_out = upc;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(A);
  cudaFree(Asign);
  cudaFree(cs);
  cudaFree(st);
  cudaFree(units);
  return ok && best < 1e30f;
}

// host part of a schedule (no device work): the sub-contractions of an update
// of widths (Wx, Wy) -- the Karatsuba pieces of the factor shape when
// levels > 0 (then Wx == Wy) -- and the longest chunk a unit may take
struct SubPlan {
  KarLayout kl;
  SubProb sub[MAX_SUB];
  int nsub;
  int upc_cap;
};

void plan_subprobs(int Wx, int Wy, int levels, SubPlan *sp) {
  *sp = SubPlan{};
  sp->upc_cap = 8 * UC_MAX;
  if (levels > 0) {
    kar_layout(Wx, levels, KAR_GAP, &sp->kl);
    sp->nsub = kar_subprobs(sp->kl, sp->sub);
    sp->upc_cap = sp->kl.G - 11;  // a unit may read up to stripe + chunk limbs past its piece
  } else {
    sp->nsub = 1;
    sp->sub[0] = SubProb{};
    sp->sub[0].wx = Wx;
    sp->sub[0].wy = Wy;
    sp->sub[0].nterm = 1;
    sp->sub[0].tsign[0] = 1;
  }
}

// unit table, operand windows and column-sum width of schedule (uc, upc)
void plan_units(const SubPlan &sp, int Wx, int Wy, int levels, int uc, int upc, Sched *sc, std::vector<Unit> *h) {
  sc->uc = uc;
  sc->upc = upc;
  sc->nsub = sp.nsub;
  for (int k = 0; k < sp.nsub; k++) sc->sub[k] = sp.sub[k];
  sc->C = std::max(colsum_width(sp.sub, sp.nsub, uc), ((Wx + Wy + 8 + 3) / 4) * 4);
  sc->n = build_units(sp.sub, sp.nsub, uc, upc, nullptr, 0);
  h->assign(sc->n, Unit{0, 0});
  build_units(sp.sub, sp.nsub, uc, upc, h->data(), sc->n);
  sc->nxb = 0;
  sc->maxlen = 0;
  if (levels > 0) {
    sc->maxlen = operand_windows(sp.sub, sp.nsub, h->data(), sc->n, sp.kl.G, sp.kl.stride, sc->xlo, sc->xlen);
    if (sc->maxlen > 0) sc->nxb = (sc->n + UNT - 1) / UNT;
  }
}

// schedule of an update launch: the Karatsuba-expanded factor update
// (levels > 0) or a plain contraction of widths (Wx, Wy)
cudaError_t sched_for(hk_ctx *c, int Wx, int Wy, int levels, Sched *out) {
  const auto key = std::make_pair(((long long)Wx << 32) | (long long)(unsigned)Wy, (long long)levels);
  auto it = c->sched_cache.find(key);
  if (it != c->sched_cache.end()) {
    *out = it->second;
    return cudaSuccess;
  }
  SubPlan sp;
  plan_subprobs(Wx, Wy, levels, &sp);
  int uc = 0, upc = 0;
  choose_schedule(sp.sub, sp.nsub, sp.upc_cap, &uc, &upc);
  if (c->autotune && !c->ws && Wx == Wy) {
    // measured choice for factor-update shapes (cached for the process)
    const auto tkey = std::make_pair((long long)Wx, (long long)levels);
    bool have = false;
    {
      std::lock_guard<std::mutex> lock(g_tune_mu);
      auto t = g_tune.find(tkey);
      if (t != g_tune.end()) {
        uc = t->second.first;
        upc = t->second.second;
        have = true;
      }
    }
    if (!have) {
      int tuc = uc, tupc = upc;
      if (autotune_schedule(c, sp.sub, sp.nsub, levels > 0 ? sp.kl.stride : Wx, sp.upc_cap, &tuc, &tupc)) {
        uc = tuc;
        upc = tupc;
        std::lock_guard<std::mutex> lock(g_tune_mu);
        g_tune[tkey] = std::make_pair(uc, upc);
      }
    }
  }
  Sched sc{};
  std::vector<Unit> h;
  plan_units(sp, Wx, Wy, levels, uc, upc, &sc, &h);
  cudaError_t e = alloc(c, c->base_arena, &sc.units, (size_t)sc.n);
  if (e != cudaSuccess) return e;
  // on the context's stream: a plain cudaMemcpy runs on the legacy default
  // stream, which a non-blocking context stream does not wait for, and for
  // pageable memory it returns before the transfer has landed
  e = cudaMemcpyAsync(sc.units, h.data(), sizeof(Unit) * sc.n, cudaMemcpyHostToDevice, c->stream);
  if (e != cudaSuccess) return e;
  c->sched_cache[key] = sc;
  *out = sc;
  return cudaSuccess;
}

void fill_sched(UpdParams &up, const Sched &sc) {
  up.units = sc.units;
  up.nunits = sc.n;
  up.uc = sc.uc;
  up.upc = sc.upc;
  up.nsub = sc.nsub;
  for (int k = 0; k < sc.nsub; k++) up.sub[k] = sc.sub[k];
  up.C = sc.C;
  up.nxb = sc.nxb;
  for (int k = 0; k < sc.nxb; k++) {
    up.xlo[k] = sc.xlo[k];
    up.xlen[k] = sc.xlen[k];
  }
  if (sc.nxb > 0) up.cx = up.cy = sc.maxlen;  // stage size: the longest block window
}

int sm_count(hk_ctx *c) {
  int n = 0;
  cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, c->device);
  return n > 0 ? n : 1;
}

// t per CTA so that a launch has roughly `target` blocks
int pick_tchunk(int trange, long long blocks_per_chunk, long long target) {
  if (trange <= 0) return 1;
  long long nchunks = (target + blocks_per_chunk - 1) / std::max(1LL, blocks_per_chunk);
  nchunks = std::max(1LL, std::min<long long>(nchunks, trange));
  return (int)((trange + nchunks - 1) / nchunks);
}

long long rows_outputs(int N, int a, int b) {
  long long s = 0;
  for (int i = a; i < b; i++) s += N - i;
  return s;
}

DevStatus read_status(hk_ctx *c) {
  DevStatus s;
  cudaMemcpyAsync(&s, c->st, sizeof(DevStatus), cudaMemcpyDeviceToHost, c->stream);
  cudaStreamSynchronize(c->stream);
  return s;
}

cudaError_t reset_status(hk_ctx *c) {
  DevStatus s;
  std::memset(&s, 0, sizeof(s));
  s.bad_row = INT_MAX;
  s.range_row = INT_MAX;
  return cudaMemcpyAsync(c->st, &s, sizeof(s), cudaMemcpyHostToDevice, c->stream);
}

__global__ void k_col_grid(int N, const long long *colU, int W, long long *colG) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < N) colG[j] = colU[j] - 32LL * W;
}

// one attempt of the blocked factorisation with window width c->W
int factor_enqueue(hk_ctx *c, const Sched &sc, int r_start);
cudaError_t ensure_la_streams(hk_ctx *c);

// Karatsuba depth of the factor update for the current window: the option's
// value, or the depth of least modelled update cost for W
int factor_levels(hk_ctx *c) {
  if (c->update_path == 1) return 0;
  if (c->kar_levels >= 0) return c->kar_levels;
  const bool big = c->N >= 768;
  if (c->lv_W != c->W || c->lv_big != big) {
    // four levels only for large factorisations: the expansion of each new
    // entry into 81 pieces sits on the panel chain (N^2/2 entries) and pays
    // off against the update's N^3/6 products from about N = 768 (measured at
    // P = 24576: 2% slower at N = 512, faster at N = 1000)
    c->lv_auto = choose_levels(c->W, KAR_GAP, big);
    c->lv_W = c->W;
    c->lv_big = big;
  }
  return c->lv_auto;
}

// one attempt of the factorisation from block row r_start (> 0: resume after a
// window widening; rows above it are final and only re-aligned)
int factor_attempt(hk_ctx *c, int r_start) {
  const int N = c->N, L = c->L, W = c->W, nb = c->nb;
  const size_t NT = (size_t)N * (N + 1) / 2;
  const int levels = factor_levels(c);
  kar_layout(W, levels, KAR_GAP, &c->kl);
  Sched sc;
  CK(sched_for(c, W, W, levels, &sc));
  c->C = sc.C;
  const long long maxout = rows_outputs(N, 0, std::min(nb, N));
  if (c->res_N != N || c->res_L != L) {
    // R (floating form), signs and reciprocals depend on (N, P) only: they
    // survive a widening of the window, which then resumes instead of restarting
    c->res_arena.release();
    c->res_N = c->res_L = 0;
    CK(alloc_mp(c, c->res_arena, &c->R, NT, L));
    CK(alloc(c, c->res_arena, &c->Asign, NT));
    CK(alloc(c, c->res_arena, &c->recip, (size_t)N * recip_limbs(L)));
    c->res_N = N;
    c->res_L = L;
  }
  if (c->fac_N != N || c->fac_L != L || c->fac_W != W || c->fac_levels != levels) {
    // (re)allocate only when the shape changed; in caller-workspace mode the
    // bump arena keeps the old region (a widening costs one more copy)
    c->fac_arena.release();
    c->fac_N = c->fac_L = c->fac_W = 0;
    CK(alloc(c, c->fac_arena, &c->A, NT * (size_t)W));
    CK(alloc(c, c->fac_arena, &c->colsum, 2 * (size_t)maxout * c->C));  // two blocks in flight
    c->Aexp = nullptr;
    if (levels > 0) CK(alloc(c, c->fac_arena, &c->Aexp, NT * (size_t)c->kl.stride));
    c->A_len = (long long)NT * W;
    c->Aexp_len = levels > 0 ? (long long)NT * c->kl.stride : 0;
    c->colsum_len = maxout * c->C;
    c->fac_N = N;
    c->fac_L = L;
    c->fac_W = W;
    c->fac_levels = levels;
  }
  if (c->ldl_mode && (c->ldl_N != N || c->ldl_L != L || c->ldl_W != W || c->ldl_levels != levels)) {
    c->ldl_arena.release();
    c->ldl_N = c->ldl_L = c->ldl_W = 0;
    CK(alloc_mp(c, c->ldl_arena, &c->Qf, NT, L));
    CK(alloc(c, c->ldl_arena, &c->B, NT * (size_t)W));
    CK(alloc(c, c->ldl_arena, &c->Bsign, NT));
    CK(alloc(c, c->ldl_arena, &c->hrow, (size_t)N));
    c->Bexp = nullptr;
    if (levels > 0) CK(alloc(c, c->ldl_arena, &c->Bexp, NT * (size_t)c->kl.stride));
    c->ldl_N = N;
    c->ldl_L = L;
    c->ldl_W = W;
    c->ldl_levels = levels;
  }
  CK(reset_status(c));
  if (!c->use_graph || c->ldl_mode) return factor_enqueue(c, sc, r_start);
  // capture the whole launch sequence of this factorisation in a CUDA graph
  // and replay it (no host synchronisation happens inside the sequence)
  const bool timing = c->timing;
  c->timing = false;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  // the legacy and per-thread default streams cannot be captured: record on a
  // private stream and launch the graph on the context's stream (recording
  // runs nothing, so stream order is the launch's)
  const cudaStream_t run = c->stream;
  if (run == nullptr || run == cudaStreamLegacy || run == cudaStreamPerThread) {
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking));
    c->stream = c->cap_stream;
  }
  const cudaError_t be = cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal);
  if (be != cudaSuccess) {
    c->stream = run;
    c->timing = timing;
    return HK_ERR_CUDA;
  }
  const int rc = factor_enqueue(c, sc, r_start);
  const cudaError_t ce = cudaStreamEndCapture(c->stream, &graph);
  c->stream = run;
  c->timing = timing;
  if (rc != HK_OK) {
    if (graph) cudaGraphDestroy(graph);
    return rc;
  }
  CK(ce);
  cudaError_t e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, c->stream);
  if (exec) cudaGraphExecDestroy(exec);
  cudaGraphDestroy(graph);
  CK(e);
  c->graph_launches++;
  return HK_OK;
}

// the factorisation's launch sequence (asynchronous on the context stream)
int factor_enqueue(hk_ctx *c, const Sched &sc, int r_start) {
  const int N = c->N, L = c->L, W = c->W, nb = c->nb;
  const int levels = c->fac_levels;  // set by factor_attempt for this window
  CK(launch_col_tops(N, L, c->top_margin, c->mom, c->colU, c->st, c->stream));
  DBG(c, "col_tops", N, L);
  k_col_grid<<<(N + 127) / 128, 128, 0, c->stream>>>(N, c->colU, W, c->colG);
  DBG(c, "col_grid", N, W);
  CK(cudaGetLastError());
  c->launches += 2;

  PanelParams pp;
  pp.N = N;
  pp.L = L;
  pp.W = W;
  pp.C = c->C;
  pp.mom = c->mom;
  pp.colU = c->colU;
  pp.R = c->R;
  pp.A = c->A;
  pp.Asign = c->Asign;
  pp.recip = c->recip;
  pp.colsum = c->colsum;
  pp.colsum_len = c->colsum_len;
  pp.aexp_len = c->Aexp_len;
  pp.st = c->st;
  pp.kl = c->kl;
  pp.Aexp = c->Aexp;

  UpdParams up;
  std::memset(&up, 0, sizeof(up));
  up.wait_ns = c->wait_ns;
  up.mode = M_FACTOR;
  up.N = N;
  up.A = levels > 0 ? c->Aexp : c->A;
  up.Asign = c->Asign;
  up.astride = levels > 0 ? c->kl.stride : W;
  up.cx = up.cy = up.astride;
  up.colsum = c->colsum;
  up.a_len = levels > 0 ? c->Aexp_len : c->A_len;
  up.colsum_len = c->colsum_len;
  fill_sched(up, sc);
  up.st = c->st;
  const long long cta_per_out = (sc.n + UNT - 1) / UNT;
  const long long target = 6LL * sm_count(c) * 3;

  LdlParams lq;
  std::memset(&lq, 0, sizeof(lq));
  if (c->ldl_mode) {
    lq.pp = pp;
    lq.Q = c->Qf;
    lq.B = c->B;
    lq.Bsign = c->Bsign;
    lq.Bexp = c->Bexp;
    lq.h = c->hrow;
    lq.x = c->ldl_x;
    lq.xzero = c->ldl_xzero;
    lq.det = c->ldl_det;
    lq.negcount = c->ldl_cnt;
    lq.zero_row = c->ldl_cnt + 1;
    up.mode = M_LDLT;
    up.B = levels > 0 ? c->Bexp : c->B;
    up.Bsign = c->Bsign;
    const int init[2] = {0, INT_MAX};
    CK(cudaMemcpyAsync(c->ldl_cnt, init, sizeof(init), cudaMemcpyHostToDevice, c->stream));
    r_start = 0;  // an LDL^T restarts after a widening (no re-alignment of its two triangles)
  }
  if (r_start > 0) {
    CK(launch_realign(pp, r_start, c->stream));
    DBG(c, "realign", r_start, W);
    c->launches++;
  }
  // streams: the panel chain (and the near update) on sP, the far updates on
  // sU; without lookahead both are the context's stream
  cudaStream_t sP = c->stream, sU = c->stream;
  const int nblk = (N - r_start + nb - 1) / nb;
  const bool la = c->lookahead && nblk > 2;
  if (la) {
    CK(ensure_la_streams(c));
    const size_t need = 3 * (size_t)nblk + 3;
    while (c->la_ev.size() < need) {
      cudaEvent_t e;
      CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
      c->la_ev.push_back(e);
    }
    // fork from the context's stream (and its realignment, if any)
    CK(cudaEventRecord(c->la_ev[0], c->stream));
    CK(cudaStreamWaitEvent(c->la_hi, c->la_ev[0], 0));
    CK(cudaStreamWaitEvent(c->la_lo, c->la_ev[0], 0));
    sP = c->la_hi;
    sU = c->la_lo;
  }
  auto ev_panel = [&](int b) { return c->la_ev[3 + 3 * b]; };
  auto ev_zero = [&](int b) { return c->la_ev[3 + 3 * b + 1]; };
  auto ev_far = [&](int b) { return c->la_ev[3 + 3 * b + 2]; };
  const size_t cs_block = (size_t)rows_outputs(N, 0, std::min(nb, N)) * c->C;
  for (int b = 0, r0 = r_start; r0 < N; b++, r0 += nb) {
    const int r1 = std::min(N, r0 + nb);
    const long long nout = rows_outputs(N, r0, r1);
    long long *cs = c->colsum + (b % 2) * cs_block;
    pp.colsum = cs;
    up.colsum = cs;
    lq.pp.colsum = cs;
    pp.r0 = r0;
    up.r0 = r0;
    // far update on sU: rows t < r0 - nb, final once block b - 2 is done (or
    // before the first block when resuming); it shares the column sums with
    // the near update below
    if (la && b >= 2) CK(cudaStreamWaitEvent(sU, ev_panel(b - 2), 0));
    CK(cudaMemsetAsync(cs, 0, sizeof(long long) * nout * c->C, sU));
    if (la) CK(cudaEventRecord(ev_zero(b), sU));
    const int tfar = la ? std::max(0, r0 - nb) : r0;
    if (tfar > 0) {
      up.ra = r0;
      up.rb = r1;
      up.nout = (int)nout;
      up.t0 = 0;
      up.t1 = tfar;
      up.tchunk = pick_tchunk(tfar, cta_per_out * nout, target);
      ev_begin(c, 0, sU);
      CK((c->update_path == 1 && !c->ldl_mode) ? launch_update_i8(up, sU) : launch_update(up, sU));
      DBG(c, "factor update", up.ra, up.t1);
      ev_end(c, sU);
      c->launches++;
    }
    if (la) {
      CK(cudaEventRecord(ev_far(b), sU));
      // near update on sP: the previous block's rows (after its panel chain)
      CK(cudaStreamWaitEvent(sP, ev_zero(b), 0));
      if (r0 > tfar) {
        up.ra = r0;
        up.rb = r1;
        up.nout = (int)nout;
        up.t0 = tfar;
        up.t1 = r0;
        up.tchunk = pick_tchunk(r0 - tfar, cta_per_out * nout, target);
        ev_begin(c, 0, sP);
        CK((c->update_path == 1 && !c->ldl_mode) ? launch_update_i8(up, sP) : launch_update(up, sP));
        DBG(c, "factor update", up.ra, up.t1);
        ev_end(c, sP);
        c->launches++;
      }
      CK(cudaStreamWaitEvent(sP, ev_far(b), 0));
    }
    for (int i = r0; i < r1; i++) {
      ev_begin(c, 1, sP);
      if (c->ldl_mode) {
        lq.pp.r0 = r0;
        CK(launch_ldl_pivot(lq, i, sP));
        DBG(c, "ldl pivot", i, 0);
        CK(launch_ldl_row(lq, i, sP));
        DBG(c, "ldl row", i, 0);
      } else {
        CK(launch_diag(pp, i, sP));
        DBG(c, "diag", i, 0);
        CK(launch_offdiag(pp, i, sP));
        DBG(c, "offdiag", i, 0);
      }
      ev_end(c, sP);
      c->launches += (i + 1 < N) ? 2 : 1;
      if (i + 1 < r1) {
        up.ra = i + 1;
        up.rb = r1;
        up.nout = (int)rows_outputs(N, i + 1, r1);
        up.t0 = i;
        up.t1 = i + 1;
        up.tchunk = 1;
        ev_begin(c, 0, sP);
        CK((c->update_path == 1 && !c->ldl_mode) ? launch_update_i8(up, sP) : launch_update(up, sP));
        DBG(c, "factor update", up.ra, up.t1);
        ev_end(c, sP);
        c->launches++;
      }
    }
    if (la) CK(cudaEventRecord(ev_panel(b), sP));
  }
  if (la) {
    // join both streams back into the context's stream
    CK(cudaEventRecord(c->la_ev[1], sU));
    CK(cudaEventRecord(c->la_ev[2], sP));
    CK(cudaStreamWaitEvent(c->stream, c->la_ev[1], 0));
    CK(cudaStreamWaitEvent(c->stream, c->la_ev[2], 0));
  }
  return HK_OK;
}

int ensure_solve_buffers(hk_ctx *c, int hist_need) {
  const int N = c->N, L = c->L;
  if (!c->sol_ready) {
    CK(alloc_mp(c, c->sol_arena, &c->v, N, L));
    CK(alloc_mp(c, c->sol_arena, &c->y, N, L));
    CK(alloc_mp(c, c->sol_arena, &c->w, N, L));
    c->sol_ready = true;
  }
  if (hist_need > c->hist_cap) {
    const int cap = std::max(hist_need, 64);
    CK(alloc_mp(c, c->sol_arena, &c->hist, cap, L));
    c->hist_cap = cap;
  }
  return HK_OK;
}

// Vector buffers of the solves (both sets of the lookahead, same capacities).
// A growth allocates new buffers; the old ones stay allocated until the
// context's solve arena is released, so a set prepared before a growth stays
// valid.
int ensure_vec(hk_ctx *c, int Wv, int Cs, int rows, int kar_stride = 0) {
  const size_t need = (size_t)c->N * Wv;
  if (need > c->vec_cap) {
    const size_t cap = need + need / 4 + 1024;
    CK(alloc(c, c->sol_arena, &c->vecA, cap));
    CK(alloc(c, c->sol_arena, &c->vecB, cap));
    CK(alloc(c, c->sol_arena, &c->vecA2, cap));
    CK(alloc(c, c->sol_arena, &c->vecAsign, (size_t)c->N));
    CK(alloc(c, c->sol_arena, &c->vecBsign, (size_t)c->N));
    CK(alloc(c, c->sol_arena, &c->vecA2sign, (size_t)c->N));
    c->vec_cap = cap;
  }
  if (kar_stride > 0 && (size_t)c->N * kar_stride > c->vecAexp_cap) {
    const size_t cap = (size_t)c->N * kar_stride;
    CK(alloc(c, c->sol_arena, &c->vecAexp, cap));
    CK(alloc(c, c->sol_arena, &c->vecA2exp, cap));
    c->vecAexp_cap = cap;
  }
  const size_t cneed = (size_t)rows * Cs;
  if (cneed > c->colsum_s_cap) {
    const size_t cap = cneed + cneed / 4 + 1024;
    CK(alloc(c, c->sol_arena, &c->colsum_s, cap));
    CK(alloc(c, c->sol_arena, &c->colsum_s2, cap));
    c->colsum_s_cap = cap;
  }
  return HK_OK;
}

int exprange(hk_ctx *c, int n, MpArr v, bool scaled, long long *lo, long long *hi) {
  CK(launch_vec_exprange(n, v, c->L, c->colG, scaled ? 1 : 0, c->d_range, c->stream));
  c->launches++;
  long long h[2];
  CK(cudaMemcpyAsync(h, c->d_range, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  *lo = h[0];
  *hi = h[1];
  return HK_OK;
}

// streams of the factor and solve lookahead (created on first use)
cudaError_t ensure_la_streams(hk_ctx *c) {
  if (c->sv_join) return cudaSuccess;
  int lo = 0, hi = 0;
  cudaError_t e = cudaDeviceGetStreamPriorityRange(&lo, &hi);
  if (e == cudaSuccess && !c->la_hi) e = cudaStreamCreateWithPriority(&c->la_hi, cudaStreamNonBlocking, hi);
  if (e == cudaSuccess && !c->la_lo) e = cudaStreamCreateWithPriority(&c->la_lo, cudaStreamNonBlocking, lo);
  if (e == cudaSuccess && !c->sv_fork) e = cudaEventCreateWithFlags(&c->sv_fork, cudaEventDisableTiming);
  if (e == cudaSuccess && !c->sv_done) e = cudaEventCreateWithFlags(&c->sv_done, cudaEventDisableTiming);
  if (e == cudaSuccess && !c->sv_join) e = cudaEventCreateWithFlags(&c->sv_join, cudaEventDisableTiming);
  return e;
}

// One vector set of a solve block: the known entries aligned to the block's
// grid, their Karatsuba expansion and signs, and the block's column sums
// (pointers and capacities as allocated when the set was taken).
struct VecSet {
  uint32_t *A = nullptr, *Aexp = nullptr;
  int32_t *sign = nullptr;
  long long *colsum = nullptr;
  long long A_len = 0, Aexp_len = 0, colsum_len = 0;
};

VecSet vec_set(hk_ctx *c, int id) {
  VecSet s;
  s.A = id ? c->vecA2 : c->vecA;
  s.Aexp = id ? c->vecA2exp : c->vecAexp;
  s.sign = id ? c->vecA2sign : c->vecAsign;
  s.colsum = id ? c->colsum_s2 : c->colsum_s;
  s.A_len = (long long)c->vec_cap;
  s.Aexp_len = (long long)c->vecAexp_cap;
  s.colsum_len = (long long)c->colsum_s_cap;
  return s;
}

// Grid of a solve block: vector entries on [h, h + 32 Wv), Karatsuba depth lv
// of its GEMV (0: schoolbook), the schedules of the GEMV and of the in-block
// updates, and the column-sum row width serving both.
struct SolveGrid {
  long long h = 0;
  int Wv = 0, lv = 0, Cs = 0;
  Sched sc{}, sc0{};
};

int solve_grid(hk_ctx *c, long long h, long long top, SolveGrid *g) {
  const int W = c->W;
  // Karatsuba on the factor's split points when the vector fits the factor's
  // window W: the block's GEMV contracts the expanded R entries with the known
  // vector entries, expanded for this block's grid in one parallel launch.
  // The in-block updates (one new entry at a time) use the plain aligned
  // operands, so no expansion sits on the per-entry chain.
  const int Wv_need = std::max(4, round4((top - h + 31) / 32));
  const bool kar_ok = c->fac_levels > 0 && c->Aexp && c->update_path == 0;
  g->lv = kar_ok && Wv_need <= W ? c->fac_levels : 0;
  g->Wv = g->lv > 0 ? W : Wv_need;
  g->h = h;
  if (g->Wv > HK_MAX_WV) return HK_ERR_RANGE;  // no shared-memory tile could hold it
  CK(sched_for(c, W, g->Wv, g->lv, &g->sc));
  g->sc0 = g->sc;
  if (g->lv > 0) CK(sched_for(c, W, g->Wv, 0, &g->sc0));
  g->Cs = std::max(g->sc.C, g->sc0.C);
  return HK_OK;
}

// update parameters of a solve GEMV (gemv) or of the in-block updates
UpdParams solve_upd(hk_ctx *c, const SolveGrid &g, const VecSet &vs, bool back, bool gemv) {
  const bool kar = gemv && g.lv > 0;
  UpdParams up;
  std::memset(&up, 0, sizeof(up));
  up.wait_ns = c->wait_ns;
  up.mode = back ? M_GEMV_BACK : M_GEMV_FWD;
  up.N = c->N;
  up.A = kar ? c->Aexp : c->A;
  up.Asign = c->Asign;
  up.astride = kar ? c->kl.stride : c->W;
  up.Vy = kar ? vs.Aexp : vs.A;
  up.Vysign = vs.sign;
  up.vstride = kar ? c->kl.stride : g.Wv;
  up.cx = up.astride;
  up.cy = up.vstride;
  up.colsum = vs.colsum;
  up.a_len = kar ? c->Aexp_len : c->A_len;
  up.vy_len = kar ? vs.Aexp_len : vs.A_len;
  up.colsum_len = vs.colsum_len;
  fill_sched(up, kar ? g.sc : g.sc0);
  up.C = g.Cs;
  up.st = c->st;
  return up;
}

// Enqueue on stream s the exact GEMV of rows [B0, B1) against known entries
// [t0, t1): align those entries to the grid (and expand them), then contract.
// The column sums accumulate (the caller zeroes them once per block).
int solve_gemv(hk_ctx *c, const SolveGrid &g, const VecSet &vs, MpArr out, bool back, int B0, int B1, int t0,
               int t1, long long target, cudaStream_t s) {
  if (t1 <= t0) return HK_OK;
  CK(launch_vec_align(t0, t1, out, c->L, c->colG, back ? 1 : 0, g.h, g.Wv, vs.A, vs.sign, c->st, vs.A_len, s));
  DBG(c, "solve vec_align", B0, g.Wv);
  c->launches++;
  if (g.lv > 0) {
    CK(launch_vec_expand(t0, t1, vs.A, c->kl, vs.Aexp, s));
    DBG(c, "solve vec_expand", B0, g.Wv);
    c->launches++;
  }
  UpdParams up = solve_upd(c, g, vs, back, true);
  const long long cta_per_out = (g.sc.n + UNT - 1) / UNT;
  up.r0 = B0;
  up.ra = B0;
  up.rb = B1;
  up.nout = B1 - B0;
  up.t0 = t0;
  up.t1 = t1;
  up.tchunk = pick_tchunk(t1 - t0, cta_per_out * (B1 - B0), target);
  CK(launch_update(up, s));
  DBG(c, "gemv/dot update", up.ra, up.t0);
  c->launches++;
  return HK_OK;
}

// The solve's launches run on the high-priority lookahead stream, forked from
// and joined back to the context's stream (also on an early return).
struct SolveStreams {
  hk_ctx *c;
  cudaStream_t orig;
  bool on = false;
  SolveStreams(hk_ctx *ctx) : c(ctx), orig(ctx->stream) {}
  cudaError_t fork() {
    cudaError_t e = cudaEventRecord(c->sv_fork, orig);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->la_hi, c->sv_fork, 0);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(c->la_lo, c->sv_fork, 0);
    if (e != cudaSuccess) return e;
    c->stream = c->la_hi;
    on = true;
    return cudaSuccess;
  }
  ~SolveStreams() {
    if (!on) return;
    cudaEventRecord(c->sv_join, c->la_lo);
    cudaStreamWaitEvent(orig, c->sv_join, 0);
    cudaEventRecord(c->sv_join, c->la_hi);
    cudaStreamWaitEvent(orig, c->sv_join, 0);
    c->stream = orig;
  }
};

// one triangular solve: forward (R^T out = rhs) or back (R out = rhs)
//
// Blocks of nbs rows; block b's column sums are the exact GEMV of its rows
// against every known entry, followed by its entries one at a time.  With the
// lookahead on, the GEMV of block b+1 against the entries known before block b
// (all but block b's own) runs on a low-priority stream while block b's
// sequential entry chain runs; block b+1 then adds only block b's rows.  That
// grid is chosen before block b's entries exist: it is block b's range widened
// by twice the last block's growth; when block b+1's range does not fit it,
// the prepared sums are dropped and block b+1 runs in full on its own grid.
// Either way every column sum is exact, so the entries are the same bits.
int solve(hk_ctx *c, MpArr rhs, MpArr out, bool back) {
  const int N = c->N, L = c->L, nbs = c->nbs;
  const long long P = 32LL * L;
  std::vector<std::pair<int, int>> blocks;  // [B0, B1) in processing order
  if (!back) {
    blocks.push_back({0, 1});
    for (int b = 1; b < N; b += nbs) blocks.push_back({b, std::min(N, b + nbs)});
  } else {
    blocks.push_back({N - 1, N});
    for (int b = N - 1; b > 0; b -= nbs) blocks.push_back({std::max(0, b - nbs), b});
  }
  const bool la = c->lookahead && blocks.size() > 3;
  SolveStreams ss(c);
  if (la) {
    CK(ensure_la_streams(c));
    CK(ss.fork());
  }
  SolveParams sp;
  std::memset(&sp, 0, sizeof(sp));
  sp.N = N;
  sp.L = L;
  sp.W = c->W;
  sp.R = c->R;
  sp.recip = c->recip;
  sp.colU = c->colU;
  sp.rhs = rhs;
  sp.out = out;
  sp.back = back ? 1 : 0;
  sp.st = c->st;
  // the prepared GEMV of the next block
  struct {
    bool live = false;
    int B0 = 0, t0 = 0, t1 = 0;  // the block it serves, the entries it contracted
    int set = 0;
    SolveGrid g;
    VecSet vs;
  } pf;
  int cur = 0;  // vector set of the current block
  long long margin = c->solve_margin;  // bits above and below the known entries' range
  long long prev_lo = LLONG_MAX, prev_hi = LLONG_MIN;  // range known before the last block
  long long grow_lo = 0, grow_hi = 0;                  // its growth over that block
  for (size_t bi = 0; bi < blocks.size(); bi++) {
    const int B0 = blocks[bi].first, B1 = blocks[bi].second;
    const int k0 = back ? B1 : 0, k1 = back ? N : B0;  // known entries
    for (int attempt = 0;; attempt++) {
      if (attempt > 6) return HK_ERR_RANGE;
      long long h, top, lo = 0, hi = 0;
      const bool have_known = k1 > k0;
      if (have_known) {
        // exact exponent range of the known entries (scaled by 2^g_k in the back solve)
        MpArr sub = out;
        sub.sign += k0;
        sub.exp += k0;
        sub.limbs += (size_t)k0 * L;
        CK(launch_vec_exprange(k1 - k0, sub, L, c->colG + k0, back ? 1 : 0, c->d_range, c->stream));
        DBG(c, "solve exprange", B0, k1 - k0);
        c->launches++;
        long long hh[2];
        CK(cudaMemcpyAsync(hh, c->d_range, sizeof(hh), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        lo = hh[0];
        hi = hh[1];
        if (lo == LLONG_MAX) {  // all known entries are zero
          lo = 0;
          hi = P;
        }
        h = lo - margin;
        top = hi + margin;
      } else {
        h = 0;
        top = 4 * 32;
      }
      // the prepared GEMV serves this block when its grid holds this block's range
      const bool use_pf = pf.live && pf.B0 == B0 && have_known && pf.g.h <= h &&
                          top <= pf.g.h + 32LL * pf.g.Wv;
      if (pf.live) {
        // its launches (and status writes) precede everything below
        CK(cudaEventRecord(c->sv_done, c->la_lo));
        CK(cudaStreamWaitEvent(c->stream, c->sv_done, 0));
        pf.live = false;
        (use_pf ? c->pf_hits : c->pf_miss)++;
      }
      SolveGrid g;
      VecSet vs;
      if (use_pf) {
        g = pf.g;
        vs = pf.vs;
        cur = pf.set;
      } else {
        int rc = solve_grid(c, h, top, &g);
        if (rc) return rc;
        rc = ensure_vec(c, g.Wv, g.Cs, nbs, g.lv > 0 ? c->kl.stride : 0);
        if (rc) return rc;
        vs = vec_set(c, cur);
      }
      if (have_known) {
        c->wv_max = std::max<long long>(c->wv_max, g.Wv);
        c->wv_sum += g.Wv;
        c->wv_count++;
      }
      // prepare the next block's GEMV against the entries known now
      const bool prep = la && have_known && bi + 1 < blocks.size();
      SolveGrid gn;
      VecSet vn;
      if (prep) {
        // the next block's range: this one's, widened by twice the growth
        // the last block brought (at least 64 bits on each side)
        const long long lo_n = lo - 2 * std::max(grow_lo, 64LL);
        const long long hi_n = hi + 2 * std::max(grow_hi, 64LL);
        long long hn = lo_n - margin, topn = hi_n + margin;
        int rc = solve_grid(c, hn, topn, &gn);
        if (rc) return rc;
        if (gn.lv > 0) gn.h -= (32LL * gn.Wv - (topn - hn)) / 2;  // centre the spare room of the window
        rc = ensure_vec(c, std::max(g.Wv, gn.Wv), std::max(g.Cs, gn.Cs), nbs,
                        (g.lv > 0 || gn.lv > 0) ? c->kl.stride : 0);
        if (rc) return rc;
        if (!use_pf) vs = vec_set(c, cur);  // a growth replaced the buffers (the old ones stay allocated)
        vn = vec_set(c, 1 - cur);
      }
      if (!use_pf)
        CK(cudaMemsetAsync(vs.colsum, 0, sizeof(long long) * (size_t)(B1 - B0) * g.Cs, c->stream));
      if (prep) {
        const int nB0 = blocks[bi + 1].first, nB1 = blocks[bi + 1].second;
        CK(cudaEventRecord(c->sv_fork, c->stream));
        CK(cudaStreamWaitEvent(c->la_lo, c->sv_fork, 0));
        CK(cudaMemsetAsync(vn.colsum, 0, sizeof(long long) * (size_t)(nB1 - nB0) * gn.Cs, c->la_lo));
        int rc = solve_gemv(c, gn, vn, out, back, nB0, nB1, k0, k1,
                            c->pf_ctas > 0 ? c->pf_ctas : 6LL * sm_count(c) * 3, c->la_lo);
        if (rc) return rc;
      }
      ev_begin(c, 2);
      if (use_pf) {
        // only the entries the prepared GEMV has not seen: the last block's
        const int na = pf.t0 == k0 ? pf.t1 : k0, nb = pf.t0 == k0 ? k1 : pf.t0;
        int rc = solve_gemv(c, g, vs, out, back, B0, B1, na, nb, 6LL * sm_count(c) * 3, c->stream);
        if (rc) return rc;
      } else if (have_known) {
        int rc = solve_gemv(c, g, vs, out, back, B0, B1, k0, k1, 6LL * sm_count(c) * 3, c->stream);
        if (rc) return rc;
      }
      if (prep) {
        pf.live = true;
        pf.B0 = blocks[bi + 1].first;
        pf.t0 = k0;
        pf.t1 = k1;
        pf.set = 1 - cur;
        pf.g = gn;
        pf.vs = vn;
      }
      sp.kl = c->kl;
      sp.kl.levels = 0;  // solve entries write only their aligned form
      sp.vecAexp = vs.Aexp;
      sp.vecA = vs.A;
      sp.vecAsign = vs.sign;
      sp.Wv = g.Wv;
      sp.C = g.Cs;
      sp.h = g.h;
      sp.colsum = vs.colsum;
      sp.colsum_len = vs.colsum_len;
      sp.vec_len = vs.A_len;
      sp.r0 = B0;
      sp.nosum = have_known ? 0 : 1;
      UpdParams upi = solve_upd(c, g, vs, back, false);  // in-block updates
      upi.r0 = B0;
      // low precision: the whole block in one launch (its per-row launches
      // would cost more than their work); high precision: entry by entry with
      // many-CTA in-block updates
      const bool fused = (long long)c->W * g.Wv <= c->fuse_ww && g.Cs >= c->W + g.Wv + 4 &&
                         solve_block_smem(L, g.Cs, c->W, g.Wv, B1 - B0) <= 160 * 1024;
      if (fused) {
        CK(launch_solve_block(sp, c->A, c->Asign, B0, B1, c->stream));
        DBG(c, "solve block", B0, g.Wv);
        c->launches++;
      }
      for (int s = 0; s < B1 - B0 && !fused; s++) {
        const int i = back ? B1 - 1 - s : B0 + s;
        // the first entry of each solve has no sum: the kernel takes G from the rhs
        CK(launch_solve_entry(sp, i, c->stream));
        DBG(c, "solve entry", i, g.Wv);
        c->launches++;
        const bool more = back ? (i > B0) : (i + 1 < B1);
        if (more) {
          if (back) {
            upi.ra = B0;
            upi.rb = i;
          } else {
            upi.ra = i + 1;
            upi.rb = B1;
          }
          upi.nout = upi.rb - upi.ra;
          upi.t0 = i;
          upi.t1 = i + 1;
          upi.tchunk = 1;
          CK(launch_update(upi, c->stream));
          DBG(c, "gemv/dot update", upi.ra, upi.t0);
          c->launches++;
        }
      }
      ev_end(c);
      DevStatus st = read_status(c);
      ev_collect(c);  // the stream is idle: fold the block's events into the phase times
      if (st.timeout) return HK_ERR_TIMEOUT;
      if (st.range_fail) {
        margin = margin * 4 + st.need_bits;
        if (pf.live) {
          // the prepared GEMV used the old margin: wait for it and drop it
          CK(cudaStreamSynchronize(c->la_lo));
          pf.live = false;
          c->pf_miss++;
        }
        CK(reset_status(c));
        continue;
      }
      if (st.code != ST_OK) {
#ifdef HK_CHECKED
        fprintf(stderr, "[hk checked] solve block %d status code %d check_site %d\n", B0, st.code, st.check_site);
#endif
        return st.code == ST_NOT_PD ? HK_ERR_NOT_PD : HK_ERR_CUDA;
      }
      if (have_known) {
        if (prev_lo != LLONG_MAX) {
          grow_lo = prev_lo - lo;
          grow_hi = hi - prev_hi;
        }
        prev_lo = lo;
        prev_hi = hi;
      }
      break;
    }
  }
  return HK_OK;
}

// lambda_t from <v,v> and <v,w>
int rayleigh(hk_ctx *c, int slot) {
  const int N = c->N, L = c->L;
  long long lov, hiv, low, hiw;
  int rc = exprange(c, N, c->v, false, &lov, &hiv);
  if (rc) return rc;
  rc = exprange(c, N, c->w, false, &low, &hiw);
  if (rc) return rc;
  if (lov == LLONG_MAX || low == LLONG_MAX) return HK_ERR_NOT_PD;
  const int Wd = std::max(4, round4(std::max((hiv - lov + 31) / 32, (hiw - low + 31) / 32)));
  Sched sc;
  CK(sched_for(c, Wd, Wd, 0, &sc));
  const int Cd = sc.C;
  rc = ensure_vec(c, Wd, Cd, 2);
  if (rc) return rc;
  ev_begin(c, 2);
  CK(launch_vec_align(0, N, c->v, L, nullptr, 0, lov, Wd, c->vecA, c->vecAsign, c->st, (long long)c->vec_cap,
                      c->stream));
  DBG(c, "lambda vec_align v", N, Wd);
  CK(launch_vec_align(0, N, c->w, L, nullptr, 0, low, Wd, c->vecB, c->vecBsign, c->st, (long long)c->vec_cap,
                      c->stream));
  DBG(c, "lambda vec_align w", N, Wd);
  CK(cudaMemsetAsync(c->colsum_s, 0, sizeof(long long) * 2 * Cd, c->stream));
  UpdParams up;
  std::memset(&up, 0, sizeof(up));
  up.wait_ns = c->wait_ns;
  up.mode = M_DOT;
  up.N = N;
  up.Vx = c->vecA;
  up.Vxsign = c->vecAsign;
  up.Vy = c->vecB;
  up.Vysign = c->vecBsign;
  up.vstride = Wd;
  up.cx = up.cy = Wd;
  up.nout = 2;
  up.t0 = 0;
  up.t1 = N;
  up.colsum = c->colsum_s;
  up.vx_len = up.vy_len = (long long)c->vec_cap;
  up.colsum_len = (long long)c->colsum_s_cap;
  fill_sched(up, sc);
  up.st = c->st;
  const long long cta_per_out = (sc.n + UNT - 1) / UNT;
  up.tchunk = pick_tchunk(N, cta_per_out * 2, 6LL * sm_count(c) * 3);
  CK(launch_update(up, c->stream));
  DBG(c, "gemv/dot update", up.ra, up.t0);
  CK(launch_lambda(L, c->colsum_s, Cd, lov, low, c->hist, slot, c->st, (long long)c->colsum_s_cap, c->stream));
  DBG(c, "lambda", slot, Cd);
  ev_end(c);
  c->launches += 4;
  return HK_OK;
}

// |a - b| <= 2^-136 a for positive normalised P-bit values (stopping rule
// of the run-until-converged mode; exact host comparison of two mantissas)
bool converged(long long ea, const uint32_t *la, long long eb, const uint32_t *lb, int L) {
  if (ea - eb > 1 || eb - ea > 1) return false;
  std::vector<uint32_t> A(L + 1, 0), B(L + 1, 0);
  for (int l = 0; l < L; l++) {
    A[l] = la[l];
    B[l] = lb[l];
  }
  long long e = std::min(ea, eb);
  auto dbl = [&](std::vector<uint32_t> &X) {
    uint32_t carry = 0;
    for (int l = 0; l <= L; l++) {
      const uint32_t nc = X[l] >> 31;
      X[l] = (X[l] << 1) | carry;
      carry = nc;
    }
  };
  if (ea > eb) dbl(A);
  if (eb > ea) dbl(B);
  bool ge = true;
  for (int l = L; l >= 0; l--)
    if (A[l] != B[l]) {
      ge = A[l] > B[l];
      break;
    }
  std::vector<uint32_t> D(L + 1, 0);
  const std::vector<uint32_t> &X = ge ? A : B, &Y = ge ? B : A;
  long long borrow = 0;
  for (int l = 0; l <= L; l++) {
    long long v = (long long)X[l] - (long long)Y[l] - borrow;
    borrow = v < 0;
    D[l] = (uint32_t)(v + (borrow ? (1LL << 32) : 0));
  }
  long long bl = 0;
  for (int l = L; l >= 0; l--)
    if (D[l]) {
      bl = 32LL * l + 32 - __builtin_clz(D[l]);
      break;
    }
  if (bl == 0) return true;
  const long long P = 32LL * L;
  return bl + e <= P + ea - 137;
}

}  // namespace

// ============================== C ABI =========================================

extern "C" {

int hk_batch_solve_impl(hk_ctx *parent, int device, const long long *opts, int count, const int *N,
                        const int *bnum, const int *bden, const int *P, const hk_mp *const *moments, int iters,
                        int nthreads, hk_mp *lambda_out, int *status_out, int *iters_out);

const char *hk_strerror(int code) {
  switch (code) {
    case HK_OK: return "ok";
    case HK_ERR_ARG: return "invalid argument";
    case HK_ERR_NOT_PD: return "rounded pivot <= 0 (matrix not positive definite at this precision)";
    case HK_ERR_CUDA: return "CUDA runtime error";
    case HK_ERR_OOM: return "out of device memory";
    case HK_ERR_TIMEOUT: return "bounded device wait ran out";
    case HK_ERR_STATE: return "call out of order";
    case HK_ERR_RANGE: return "exact-accumulation window exhausted";
    default: return "unknown status";
  }
}

int hk_create(hk_ctx **out, int device, void *cuda_stream) {
  if (!out) return HK_ERR_ARG;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) return HK_ERR_ARG;
  hk_ctx *c = new (std::nothrow) hk_ctx();
  if (!c) return HK_ERR_OOM;
  c->device = device;
  c->stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  if (cudaSetDevice(device) != cudaSuccess) {
    delete c;
    return HK_ERR_CUDA;
  }
  *out = c;
  return HK_OK;
}

void hk_destroy(hk_ctx *c) {
  if (!c) return;
  cudaSetDevice(c->device);
  cudaStreamSynchronize(c->stream);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  if (c->la_hi) cudaStreamDestroy(c->la_hi);
  if (c->la_lo) cudaStreamDestroy(c->la_lo);
  for (cudaEvent_t e : c->la_ev) cudaEventDestroy(e);
  for (cudaEvent_t e : {c->sv_fork, c->sv_done, c->sv_join})
    if (e) cudaEventDestroy(e);
  c->sol_arena.release();
  c->fac_arena.release();
  c->res_arena.release();
  c->ldl_arena.release();
  c->ldl_small.release();
  c->sec_arena.release();
  c->base_arena.release();
  if (c->pred_params) cudaFree(c->pred_params);
  if (c->pred_buf) cudaFree(c->pred_buf);
  for (auto &p : c->evpool) {
    if (p.a) cudaEventDestroy(p.a);
    if (p.b) cudaEventDestroy(p.b);
  }
  delete c;
}

int hk_workspace_bytes(int N, int P, size_t *bytes) {
  if (N < 1 || P < 32 || P % 32 || P > HK_MAX_P || !bytes) return HK_ERR_ARG;
  const long long L = P / 32;
  const long long W = round4(L + (N + 128 + 31) / 32) + 64;  // one widening included
  const long long NT = (long long)N * (N + 1) / 2;
  long long kstride = 0;  // the widest Karatsuba expansion any depth may use
  for (int lv = 1; lv <= MAX_KAR; lv++) {
    KarLayout kl;
    kar_layout((int)W, lv, KAR_GAP, &kl);
    kstride = std::max<long long>(kstride, kl.stride);
  }
  const long long C = 2 * W + 64;
  long long b = 0;
  b += (2LL * N) * (16 + 4 * L);          // moments
  b += 3LL * N * 8 + 4096;                // tops, grids, status
  b += NT * (16 + 4 * L);                 // R
  b += NT * (4 * W + 4);                  // aligned R
  b += NT * 4LL * kstride;                // its Karatsuba expansion
  b += (long long)N * recip_limbs((int)L) * 4;  // reciprocals
  b += 2LL * 16 * N * C * 8;              // column sums of two blocks (lookahead)
  b += 3LL * N * (16 + 4 * L) + 256LL * (16 + 4 * L);  // v, y, w, history
  const long long Wv = 2 * W + (long long)N;  // vector window (generous)
  // solves: three aligned vectors (two sets of the lookahead and the Rayleigh
  // quotient's second operand), two Karatsuba expansions, two column-sum blocks
  b += 3LL * N * (4 * Wv + 4) * 5 / 4 + 2LL * N * 4 * kstride + 2LL * 16 * (W + Wv + 64) * 8 * 5 / 4;
  b += 8LL << 20;                         // unit tables, alignment slack
  *bytes = (size_t)b * 2;                 // two widenings of slack for the bump allocator
  return HK_OK;
}

int hk_set_workspace(hk_ctx *c, void *dev_ptr, size_t bytes) {
  if (!c || (!dev_ptr && bytes)) return HK_ERR_ARG;
  cudaSetDevice(c->device);
  c->sol_arena.release();
  c->fac_arena.release();
  c->res_arena.release();
  c->base_arena.release();
  c->res_N = c->res_L = 0;
  c->fac_N = c->fac_L = c->fac_W = 0;
  c->ws = reinterpret_cast<char *>(dev_ptr);
  c->ws_bytes = bytes;
  c->base_arena.base = c->ws;
  c->base_arena.cap = bytes;
  c->base_arena.used = 0;
  c->loaded = c->factored = c->sol_ready = false;
  c->hist_cap = 0;
  c->vec_cap = 0;
  c->vecAexp_cap = 0;
  c->colsum_s_cap = 0;
  c->fac_N = c->fac_L = c->fac_W = 0;
  c->mom = MpArr{};
  c->sched_cache.clear();
  return HK_OK;
}

int hk_load_moments_flat(hk_ctx *c, int N, int bnum, int bden, int P, const int32_t *sign,
                         const int64_t *exp, const uint32_t *limbs, int on_device) {
  if (!c || N < 1 || P < 32 || P % 32 || P > HK_MAX_P || !sign || !exp || !limbs) return HK_ERR_ARG;
  if ((long long)N * (N + 1) / 2 > (1LL << 40)) return HK_ERR_ARG;
  cudaSetDevice(c->device);
  const int L = P / 32;
  const int M = 2 * N - 1;
  if (!on_device) {
    for (int k = 0; k < M; k++) {
      const uint32_t *m = limbs + (size_t)k * L;
      bool nz = false;
      for (int l = 0; l < L; l++) nz |= m[l] != 0;
      if (sign[k] != 0 && sign[k] != 1) return HK_ERR_ARG;
      if (nz && !(m[L - 1] & 0x80000000u)) return HK_ERR_ARG;
      if (!nz && (sign[k] != 0 || exp[k] != 0)) return HK_ERR_ARG;
    }
  }
  cudaStreamSynchronize(c->stream);
  const bool same = c->mom.limbs != nullptr && c->N == N && c->P == P;
  c->loaded = c->factored = false;
  c->hist_count = 0;
  c->bnum = bnum;
  c->bden = bden;
  if (!same) {
    c->sol_arena.release();
    c->fac_arena.release();
    c->res_arena.release();
    c->res_N = c->res_L = 0;
    c->base_arena.release();
    if (c->ws) {
      c->base_arena.base = c->ws;
      c->base_arena.cap = c->ws_bytes;
      c->base_arena.used = 0;
    }
    c->sched_cache.clear();
    c->sol_ready = false;
    c->hist_cap = 0;
    c->vec_cap = 0;
    c->vecAexp_cap = 0;
    c->colsum_s_cap = 0;
    c->fac_N = c->fac_L = c->fac_W = 0;
    c->ldl_arena.release();
    c->ldl_small.release();
    c->sec_arena.release();
    c->ldl_N = c->ldl_L = c->ldl_W = 0;
    c->ldl_sL = 0;
    c->ldl_x = MpArr{};
    c->sec_cap = c->sec_L = c->sec_count = 0;
    c->ldl_ready = false;
    c->mom = MpArr{};
    c->N = N;
    c->L = L;
    c->P = P;
    CK(alloc_mp(c, c->base_arena, &c->mom, M, L));
    CK(alloc(c, c->base_arena, &c->colU, (size_t)N));
    CK(alloc(c, c->base_arena, &c->colG, (size_t)N));
    CK(alloc(c, c->base_arena, &c->st, 1));
    CK(alloc(c, c->base_arena, &c->d_range, 2));
  }
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CK(cudaMemcpyAsync(c->mom.sign, sign, sizeof(int32_t) * M, kind, c->stream));
  CK(cudaMemcpyAsync(c->mom.exp, exp, sizeof(long long) * M, kind, c->stream));
  CK(cudaMemcpyAsync(c->mom.limbs, limbs, sizeof(uint32_t) * (size_t)M * L, kind, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->loaded = true;
  c->ldl_ready = false;
  c->sec_count = 0;
  return HK_OK;
}

int hk_load_moments(hk_ctx *c, int N, int bnum, int bden, int P, const hk_mp *moments) {
  if (!c || N < 1 || P < 32 || P % 32 || !moments) return HK_ERR_ARG;
  const int L = P / 32, M = 2 * N - 1;
  std::vector<int32_t> s(M);
  std::vector<int64_t> e(M);
  std::vector<uint32_t> l((size_t)M * L);
  for (int k = 0; k < M; k++) {
    if (!moments[k].limbs) return HK_ERR_ARG;
    s[k] = moments[k].sign;
    e[k] = moments[k].exp;
    std::memcpy(&l[(size_t)k * L], moments[k].limbs, sizeof(uint32_t) * L);
  }
  return hk_load_moments_flat(c, N, bnum, bden, P, s.data(), e.data(), l.data(), 0);
}

}  // extern "C"

// The blocked factorisation with its window widenings: the Cholesky of M, or
// (c->ldl_mode) the shifted LDL^T of M - xI.
static int factor_run(hk_ctx *c, int *bad_row) {
  cudaSetDevice(c->device);
  c->factored = false;
  c->ldl_ready = false;
  c->launches = 0;
  c->widenings = 0;
  c->resumes = 0;
  c->t_phase[0] = c->t_phase[1] = c->t_phase[2] = 0;
  // window: P bits plus the spread of a column (at most about N bits for
  // beta = 1) plus 128; HK_WINDOW_SLACK overrides the extra bits (tests)
  long long slack = c->N + 128;
  if (const char *e = getenv("HK_WINDOW_SLACK")) slack = std::max(0LL, atoll(e));
  c->W = round4(c->L + (slack + 31) / 32);
  // the LDL^T operands are the Cholesky factor's within a factor of two
  c->top_margin = c->ldl_mode ? 2 : 0;
  if (const char *e = getenv("HK_NB")) c->nb = std::max(1, atoi(e));  // panel block rows (tuning)
  if (const char *e = getenv("HK_LOOKAHEAD")) c->lookahead = atoi(e) != 0;  // (tuning)
  if (const char *e = getenv("HK_KARATSUBA")) c->kar_levels = std::min(MAX_KAR, std::max(-1, atoi(e)));  // (tuning)
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int result = HK_ERR_RANGE;
  int r_start = 0;
  c->t_factor = 0;
  for (int attempt = 0; attempt < 6; attempt++) {
    c->evused = 0;
    cudaEventRecord(e0, c->stream);
    int rc = factor_attempt(c, r_start);
    cudaEventRecord(e1, c->stream);
    if (rc != HK_OK) {
      result = rc;
      break;
    }
    DevStatus st = read_status(c);
    cudaEventSynchronize(e1);
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    c->t_factor += ms;  // every attempt counts
    ev_collect(c);
    if (st.timeout) {
      result = HK_ERR_TIMEOUT;
      break;
    }
    // a window failure stops the sequence at its launch: widen the window
    // below and above, re-align the finished rows above the failing block and
    // resume there (rows above it are final in floating form)
    if (st.range_fail) {
      // the sequence stops at the first failing launch, so the shortfall seen
      // is a lower bound for the rows after it: widen generously (twice the
      // shortfall, at least N/2 bits) so that one resumption usually suffices
      const long long want = std::max(2 * st.need_bits, (long long)c->N / 2) + 64;
      const long long delta = (want + 31) / 32 * 32;
      c->top_margin += delta;
      c->W = round4(c->W + 2 * delta / 32);
      c->widenings++;
      const int row = st.range_row;
      r_start = (row != INT_MAX && row >= 0 && row < c->N) ? (row / c->nb) * c->nb : 0;
      if (r_start > 0 && (c->use_graph || c->ldl_mode)) r_start = 0;  // whole factorisations only
      if (r_start > 0) c->resumes++;
      continue;
    }
    if (st.code == ST_NOT_PD) {
      if (bad_row) *bad_row = st.bad_row;
      result = HK_ERR_NOT_PD;
      break;
    }
    if (st.code != ST_OK && !(c->ldl_mode && st.code == ST_ZERO)) {  // a failed device check
      result = HK_ERR_CUDA;
      break;
    }
    if (c->ldl_mode)
      c->ldl_ready = true;  // a zero pivot is a result (det = 0), not an error
    else
      c->factored = true;
    result = HK_OK;
    break;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return result;
}

extern "C" {

int hk_factor(hk_ctx *c, int *bad_row) {
  if (!c) return HK_ERR_ARG;
  if (!c->loaded) return HK_ERR_STATE;
  c->ldl_mode = false;
  return factor_run(c, bad_row);
}

int hk_selftest_wait(hk_ctx *c) {
  if (!c) return HK_ERR_ARG;
  if (!c->loaded) return HK_ERR_STATE;
  CK(reset_status(c));
  CK(launch_wait_selftest(c->st, c->wait_ns, c->stream));
  const DevStatus st = read_status(c);
  CK(cudaGetLastError());
  // the wait touched nothing but the status word: clear it so that the
  // context (and a factorisation it holds) stays usable
  CK(reset_status(c));
  CK(cudaStreamSynchronize(c->stream));
  return (st.timeout > 0 && st.code == ST_TIMEOUT) ? HK_ERR_TIMEOUT : HK_OK;
}

int hk_set_option(hk_ctx *c, int option, long long value) {
  if (!c) return HK_ERR_ARG;
  switch (option) {
    case 0:  // update path
      return hk_set_update_path(c, (int)value);
    case 1:  // Karatsuba levels of the factor update (-1: chosen per window)
      if (value < -1 || value > MAX_KAR) return HK_ERR_ARG;
      c->kar_levels = (int)value;
      break;
    case 2:  // capture factorisations in CUDA graphs
      c->use_graph = value != 0;
      break;
    case 3:  // autotune update schedules
      c->autotune = value != 0;
      c->sched_cache.clear();
      break;
    case 4:  // panel block rows
      if (value < 1 || value > 256) return HK_ERR_ARG;
      c->nb = (int)value;
      break;
    case 5:  // step cap of the converging inverse iteration (R stays valid)
      if (value < 1 || value > 100000) return HK_ERR_ARG;
      c->max_iters = (int)value;
      return HK_OK;
    case 6:  // limit of each bounded device wait, ns (R stays valid)
      if (value < 1000 || value > 60000000000LL) return HK_ERR_ARG;
      c->wait_ns = value;
      return HK_OK;
    case 7:  // lookahead: far updates overlap the panel chain on a second stream
      c->lookahead = value != 0;
      return HK_OK;
    default:
      return HK_ERR_ARG;
  }
  c->factored = false;
  return HK_OK;
}

int hk_batch_solve(hk_ctx *c, int count, const int *N, const int *beta_num, const int *beta_den, const int *P,
                   const hk_mp *const *moments, int iters, int nthreads, hk_mp *lambda_out, int *status_out,
                   int *iters_out) {
  if (!c || iters < 0) return HK_ERR_ARG;
  const long long opts[6] = {c->update_path, c->kar_levels, c->use_graph ? 1 : 0, c->autotune ? 1 : 0, c->nb,
                            c->max_iters};
  return hk_batch_solve_impl(c, c->device, opts, count, N, beta_num, beta_den, P, moments, iters,
                             nthreads > 0 ? nthreads : 16, lambda_out, status_out, iters_out);
}

int hk_set_update_path(hk_ctx *c, int path) {
  if (!c || path < 0 || path > 1) return HK_ERR_ARG;
  c->update_path = path;
  c->factored = false;
  return HK_OK;
}

int hk_get_R_flat(hk_ctx *c, int32_t *sign, int64_t *exp, uint32_t *limbs) {
  if (!c || !sign || !exp || !limbs) return HK_ERR_ARG;
  if (!c->factored) return HK_ERR_STATE;
  cudaSetDevice(c->device);
  const size_t NT = (size_t)c->N * (c->N + 1) / 2;
  CK(cudaMemcpyAsync(sign, c->R.sign, sizeof(int32_t) * NT, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(exp, c->R.exp, sizeof(int64_t) * NT, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(limbs, c->R.limbs, sizeof(uint32_t) * NT * c->L, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HK_OK;
}

int hk_get_R(hk_ctx *c, hk_mp *R) {
  if (!c || !R) return HK_ERR_ARG;
  if (!c->factored) return HK_ERR_STATE;
  const size_t NT = (size_t)c->N * (c->N + 1) / 2;
  std::vector<int32_t> s(NT);
  std::vector<int64_t> e(NT);
  std::vector<uint32_t> l(NT * c->L);
  int rc = hk_get_R_flat(c, s.data(), e.data(), l.data());
  if (rc) return rc;
  for (size_t k = 0; k < NT; k++) {
    if (!R[k].limbs) return HK_ERR_ARG;
    R[k].sign = s[k];
    R[k].exp = e[k];
    std::memcpy(R[k].limbs, &l[k * c->L], sizeof(uint32_t) * c->L);
  }
  return HK_OK;
}

int hk_smallest_eig(hk_ctx *c, int iters, hk_mp *lambda_min, int *iters_used) {
  if (!c || iters < 0) return HK_ERR_ARG;
  if (!c->factored) return HK_ERR_STATE;
  cudaSetDevice(c->device);
  const int T = iters > 0 ? iters : c->max_iters;
  if (const char *e = getenv("HK_FUSE_WW")) c->fuse_ww = atoll(e);  // (tuning and tests)
  if (const char *e = getenv("HK_SOLVE_MARGIN")) c->solve_margin = std::max(32LL, atoll(e));  // (tuning)
  if (const char *e = getenv("HK_SOLVE_PF_CTAS")) c->pf_ctas = std::max(0LL, atoll(e));  // (tuning)
  c->eig_converged = 0;
  c->wv_max = c->wv_sum = c->wv_count = 0;
  c->pf_hits = c->pf_miss = 0;
  int rc = ensure_solve_buffers(c, T);
  if (rc) return rc;
  c->t_phase[2] = 0;
  c->evused = 0;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c->stream);
  CK(launch_set_ones(c->N, c->v, c->L, c->stream));
  c->launches++;
  CK(reset_status(c));
  const int L = c->L;
  std::vector<uint32_t> prev(L), cur(L);
  long long eprev = 0, ecur = 0;
  int32_t sprev = 0, scur = 0;
  int t = 0;
  for (t = 0; t < T; t++) {
    rc = solve(c, c->v, c->y, false);
    if (rc) break;
    rc = solve(c, c->y, c->w, true);
    if (rc) break;
    rc = rayleigh(c, t);
    if (rc) break;
    rc = cuda_status(launch_vec_normalise(c->N, c->w, c->v, L, c->stream));
    c->launches++;
    if (rc) break;
    if (iters == 0) {
      CK(cudaMemcpyAsync(cur.data(), c->hist.limbs + (size_t)t * L, 4 * (size_t)L, cudaMemcpyDeviceToHost,
                         c->stream));
      CK(cudaMemcpyAsync(&ecur, c->hist.exp + t, 8, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemcpyAsync(&scur, c->hist.sign + t, 4, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaStreamSynchronize(c->stream));
      if (t > 0 && converged(ecur, cur.data(), eprev, prev.data(), L)) {
        c->eig_converged = 1;
        t++;
        break;
      }
      prev = cur;
      eprev = ecur;
      sprev = scur;
    }
  }
  (void)sprev;
  cudaEventRecord(e1, c->stream);
  cudaEventSynchronize(e1);
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  c->t_eig = ms;
  ev_collect(c);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  DevStatus st = read_status(c);
  if (st.code == ST_NOT_PD) return HK_ERR_NOT_PD;
  if (st.timeout) return HK_ERR_TIMEOUT;
  if (st.range_fail) return HK_ERR_RANGE;
  if (st.code != ST_OK) return HK_ERR_CUDA;
  const int used = std::min(t, T);
  c->hist_count = used;
  if (iters_used) *iters_used = used;
  if (lambda_min && used > 0) {
    if (!lambda_min->limbs) return HK_ERR_ARG;
    const int k = used - 1;
    CK(cudaMemcpyAsync(lambda_min->limbs, c->hist.limbs + (size_t)k * L, 4 * (size_t)L,
                       cudaMemcpyDeviceToHost, c->stream));
    long long e = 0;
    int32_t s = 0;
    CK(cudaMemcpyAsync(&e, c->hist.exp + k, 8, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(&s, c->hist.sign + k, 4, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    lambda_min->exp = e;
    lambda_min->sign = s;
  }
  return HK_OK;
}

int hk_get_history_flat(hk_ctx *c, int count, int32_t *sign, int64_t *exp, uint32_t *limbs) {
  if (!c || count < 0 || !sign || !exp || !limbs) return HK_ERR_ARG;
  if (count > c->hist_count) return HK_ERR_ARG;
  if (count == 0) return HK_OK;
  CK(cudaMemcpyAsync(sign, c->hist.sign, 4 * (size_t)count, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(exp, c->hist.exp, 8 * (size_t)count, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(limbs, c->hist.limbs, 4 * (size_t)count * c->L, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HK_OK;
}

int hk_get_timings(hk_ctx *c, double *out, int n) {
  if (!c || !out || n < 0) return HK_ERR_ARG;
  const double v[5] = {c->t_phase[0], c->t_phase[1], c->t_phase[2], c->t_factor, c->t_eig};
  for (int k = 0; k < n && k < 5; k++) out[k] = v[k];
  for (int k = 5; k < n; k++) out[k] = 0;
  return HK_OK;
}

int hk_get_stats(hk_ctx *c, int64_t *out, int n) {
  if (!c || !out || n < 0) return HK_ERR_ARG;
  // limb products the factor's update kernel executes per P-bit MAC (sum of
  // the sub-contraction areas; W^2 without Karatsuba)
  SubProb sub[MAX_SUB];
  KarLayout kl;
  const int lv = c->fac_levels >= 0 ? c->fac_levels : factor_levels(c);
  kar_layout(c->W, lv, KAR_GAP, &kl);
  const int ns = kar_subprobs(kl, sub);
  int64_t per_mac = 0;
  for (int k = 0; k < ns; k++) per_mac += (int64_t)sub[k].wx * sub[k].wy;
  const int64_t v[11] = {c->launches,
                        c->W,
                        c->widenings,
                        lv,
                        per_mac,
                        c->eig_converged,
                        c->wv_max,
                        c->wv_count ? c->wv_sum / c->wv_count : 0,
                        c->resumes,
                        c->pf_hits,
                        c->pf_miss};
  for (int k = 0; k < n && k < 11; k++) out[k] = v[k];
  for (int k = 11; k < n; k++) out[k] = 0;
  return HK_OK;
}

int hk_selftest_mp(int op, int L, const uint32_t *x, int nx, int64_t ex, const uint32_t *y, int ny,
                   int64_t ey, uint32_t *out, int64_t *eo) {
  if (!x || !out || !eo || (ny > 0 && !y)) return HK_ERR_ARG;
  const int rc = hk::selftest_mp(op, L, x, nx, ex, y, ny, ey, out, eo);
  return rc == 0 ? HK_OK : (rc == 1 ? HK_ERR_ARG : HK_ERR_CUDA);
}

int hk_update_plan(int W, int levels, int64_t *info, int32_t *splits, int32_t *pieces, int32_t *terms,
                   int32_t *units, int64_t ucap, int32_t *win) {
  if (W < 1 || W > (1 << 20) || levels < -1 || levels > MAX_KAR || !info) return HK_ERR_ARG;
  const int lv = levels < 0 ? choose_levels(W, KAR_GAP, true) : levels;
  SubPlan sp;
  plan_subprobs(W, W, lv, &sp);
  int uc = 0, upc = 0;
  choose_schedule(sp.sub, sp.nsub, sp.upc_cap, &uc, &upc);
  Sched sc{};
  std::vector<Unit> h;
  plan_units(sp, W, W, lv, uc, upc, &sc, &h);
  if (units && ucap < sc.n) return HK_ERR_ARG;
  const int64_t v[9] = {lv > 0 ? sp.kl.levels : 0, sc.nsub, lv > 0 ? sp.kl.stride : W, lv > 0 ? sp.kl.G : 0,
                        uc, upc, sc.n, sc.nxb, sc.C};
  for (int k = 0; k < 9; k++) info[k] = v[k];
  if (splits) {
    for (int k = 0; k < MAX_SPLITS; k++) splits[k] = sp.kl.ms[k];
  }
  for (int k = 0; k < sc.nsub; k++) {
    if (pieces) {
      pieces[3 * k] = sc.sub[k].xoff;
      pieces[3 * k + 1] = sc.sub[k].wx;
      pieces[3 * k + 2] = sc.sub[k].nterm;
    }
    if (terms)
      for (int t = 0; t < sc.sub[k].nterm; t++) {
        terms[2 * (MAX_TERMS * k + t)] = sc.sub[k].toff[t];
        terms[2 * (MAX_TERMS * k + t) + 1] = sc.sub[k].tsign[t];
      }
  }
  if (units)
    for (int u = 0; u < sc.n; u++) {
      units[2 * u] = h[u].d0;
      units[2 * u + 1] = h[u].p0;
    }
  if (win)
    for (int b = 0; b < sc.nxb; b++) {
      win[2 * b] = sc.xlo[b];
      win[2 * b + 1] = sc.xlen[b];
    }
  return HK_OK;
}

int hk_set_predictor(hk_ctx *c, const float *params, const double *scales) {
  if (!c || !params || !scales) return HK_ERR_ARG;
  for (int k = 0; k < 10; k++)
    if (!std::isfinite(scales[k]) || ((k == 2 || k == 3 || k >= 7) && scales[k] <= 0)) return HK_ERR_ARG;
  cudaSetDevice(c->device);
  if (!c->pred_params) CK(cudaMalloc(&c->pred_params, sizeof(float) * HK_MLP_NPARAMS));
  CK(cudaMemcpyAsync(c->pred_params, params, sizeof(float) * HK_MLP_NPARAMS, cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < 10; k++) c->pred_scales[k] = scales[k];
  return HK_OK;
}

int hk_predict(hk_ctx *c, int count, const double *N, const double *beta, float *out3) {
  if (!c || count < 0 || (count > 0 && (!N || !beta || !out3))) return HK_ERR_ARG;
  if (!c->pred_params) return HK_ERR_STATE;
  if (count == 0) return HK_OK;
  cudaSetDevice(c->device);
  const double *sc = c->pred_scales;  // x mean[2], x std[2], y mean[3], y std[3]
  std::vector<float> x((size_t)count * 2), y((size_t)count * 3);
  for (int k = 0; k < count; k++) {
    if (!(N[k] >= 1) || !(beta[k] > 0)) return HK_ERR_ARG;
    x[2 * k] = (float)((std::log2(N[k]) - 8.0 - sc[0]) / sc[2]);
    x[2 * k + 1] = (float)((std::log2(beta[k]) - sc[1]) / sc[3]);
  }
  if (count > c->pred_cap) {
    if (c->pred_buf) cudaFree(c->pred_buf);
    c->pred_buf = nullptr;
    c->pred_cap = 0;
    CK(cudaMalloc(&c->pred_buf, sizeof(float) * 5 * (size_t)count));
    c->pred_cap = count;
  }
  float *dx = c->pred_buf, *dy = c->pred_buf + 2 * (size_t)count;
  CK(cudaMemcpyAsync(dx, x.data(), sizeof(float) * x.size(), cudaMemcpyHostToDevice, c->stream));
  const int rc = hk_mlp_forward(c->pred_params, dx, count, dy, c->stream);
  if (rc) return rc;
  CK(cudaMemcpyAsync(y.data(), dy, sizeof(float) * y.size(), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < count; k++) {
    const double t0 = y[3 * k] * sc[7] + sc[4], t1 = y[3 * k + 1] * sc[8] + sc[5], t2 = y[3 * k + 2] * sc[9] + sc[6];
    out3[3 * k] = (float)(t0 * N[k] + 128.0);  // (bits - 128) / N
    out3[3 * k + 1] = (float)(t1 * N[k]);      // log2(lambda_min) / N
    out3[3 * k + 2] = (float)std::exp2(t2);    // log2(iterations)
  }
  return HK_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// The paper's own method: P(x) = det(M - xI) by the shifted LDL^T, the Secant
// recurrence on it, and the inertia on both sides of the root
// ---------------------------------------------------------------------------
namespace {

cudaError_t ensure_ldl_small(hk_ctx *c) {
  if (c->ldl_sL == c->L && c->ldl_x.limbs) return cudaSuccess;
  c->ldl_small.release();
  c->ldl_sL = 0;
  cudaError_t e = alloc_mp(c, c->ldl_small, &c->ldl_x, 1, c->L);
  if (e == cudaSuccess) e = alloc_mp(c, c->ldl_small, &c->ldl_det, 1, c->L);
  if (e == cudaSuccess) e = alloc(c, c->ldl_small, &c->ldl_cnt, 2);
  if (e == cudaSuccess) c->ldl_sL = c->L;
  return e;
}

cudaError_t copy_entry(MpArr dst, int kd, MpArr src, int ks, int L, cudaMemcpyKind kind, cudaStream_t s) {
  cudaError_t e = cudaMemcpyAsync(dst.limbs + (size_t)kd * L, src.limbs + (size_t)ks * L, 4 * (size_t)L, kind, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst.sign + kd, src.sign + ks, 4, kind, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(dst.exp + kd, src.exp + ks, 8, kind, s);
  return e;
}

// the shifted LDL^T with x = xs[kx] (device); its determinant into dst[kd]
int ldlt_dev(hk_ctx *c, MpArr xs, int kx, MpArr dst, int kd) {
  CK(ensure_ldl_small(c));
  CK(copy_entry(c->ldl_x, 0, xs, kx, c->L, cudaMemcpyDeviceToDevice, c->stream));
  c->ldl_xzero = 0;
  c->ldl_mode = true;
  const int rc = factor_run(c, nullptr);
  c->ldl_mode = false;
  if (rc != HK_OK) return rc;
  if (dst.limbs) CK(copy_entry(dst, kd, c->ldl_det, 0, c->L, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return HK_OK;
}

int read_counts(hk_ctx *c, int *neg, int *zero_row) {
  int h[2] = {0, INT_MAX};
  CK(cudaMemcpyAsync(h, c->ldl_cnt, sizeof(h), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (neg) *neg = h[0];
  if (zero_row) *zero_row = h[1] == INT_MAX ? -1 : h[1];
  return HK_OK;
}

// sign of the determinant held in ldl_det: 1, -1, or 0 (zero)
int det_sign(hk_ctx *c, int *sgn) {
  std::vector<uint32_t> l(c->L);
  int32_t sg = 0;
  CK(cudaMemcpyAsync(l.data(), c->ldl_det.limbs, 4 * (size_t)c->L, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&sg, c->ldl_det.sign, 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  bool z = true;
  for (uint32_t v : l) z &= v == 0;
  *sgn = z ? 0 : (sg ? -1 : 1);
  return HK_OK;
}

bool mp_ok(const hk_mp *v) { return v && v->limbs && (v->sign == 0 || v->sign == 1); }

}  // namespace

extern "C" {

int hk_ldlt_det(hk_ctx *c, const hk_mp *x, hk_mp *det, int *neg_pivots, int *zero_row) {
  if (!c || !mp_ok(x) || !det || !det->limbs) return HK_ERR_ARG;
  if (!c->loaded) return HK_ERR_STATE;
  cudaSetDevice(c->device);
  CK(ensure_ldl_small(c));
  const int L = c->L;
  bool z = true;
  for (int l = 0; l < L; l++) z &= x->limbs[l] == 0;
  if (!z && !(x->limbs[L - 1] >> 31)) return HK_ERR_ARG;  // not normalised
  const int32_t sg = z ? 0 : x->sign;
  const long long ex = z ? 0 : x->exp;
  CK(cudaMemcpyAsync(c->ldl_x.limbs, x->limbs, 4 * (size_t)L, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->ldl_x.sign, &sg, 4, cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(c->ldl_x.exp, &ex, 8, cudaMemcpyHostToDevice, c->stream));
  c->ldl_xzero = z ? 1 : 0;
  c->ldl_mode = true;
  const int rc = factor_run(c, nullptr);
  c->ldl_mode = false;
  if (rc != HK_OK) return rc;
  int32_t dsg = 0;
  long long dex = 0;
  CK(cudaMemcpyAsync(det->limbs, c->ldl_det.limbs, 4 * (size_t)L, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&dsg, c->ldl_det.sign, 4, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&dex, c->ldl_det.exp, 8, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  det->sign = dsg;
  det->exp = dex;
  return read_counts(c, neg_pivots, zero_row);
}

int hk_get_ldlt_flat(hk_ctx *c, int which, int32_t *sign, int64_t *exp, uint32_t *limbs) {
  if (!c || which < 0 || which > 2 || !sign || !exp || !limbs) return HK_ERR_ARG;
  if (!c->ldl_ready) return HK_ERR_STATE;
  const int N = c->N, L = c->L;
  const size_t NT = (size_t)N * (N + 1) / 2;
  if (which == 0) {
    for (int t = 0; t < N; t++) {
      const size_t k = tri_idx(t, t, N);
      CK(cudaMemcpyAsync(limbs + (size_t)t * L, c->R.limbs + k * L, 4 * (size_t)L, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemcpyAsync(sign + t, c->R.sign + k, 4, cudaMemcpyDeviceToHost, c->stream));
      CK(cudaMemcpyAsync(exp + t, c->R.exp + k, 8, cudaMemcpyDeviceToHost, c->stream));
    }
  } else {
    const MpArr &m = which == 1 ? c->R : c->Qf;
    CK(cudaMemcpyAsync(limbs, m.limbs, 4 * NT * L, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(sign, m.sign, 4 * NT, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaMemcpyAsync(exp, m.exp, 8 * NT, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  if (which == 2)  // CDivDiag has no diagonal entries
    for (int t = 0; t < N; t++) {
      const size_t k = tri_idx(t, t, N);
      sign[k] = 0;
      exp[k] = 0;
      std::memset(limbs + k * L, 0, 4 * (size_t)L);
    }
  return HK_OK;
}

int hk_secant(hk_ctx *c, int max_steps, hk_mp *root, int *dets_used) {
  if (!c || max_steps < 0 || max_steps > 10000 || !root || !root->limbs) return HK_ERR_ARG;
  if (!c->loaded) return HK_ERR_STATE;
  cudaSetDevice(c->device);
  const int L = c->L, N = c->N;
  const int cap = max_steps + 3;
  if (c->sec_cap < cap || c->sec_L != L) {
    c->sec_arena.release();
    c->sec_cap = c->sec_L = 0;
    CK(alloc_mp(c, c->sec_arena, &c->sec_x, cap, L));
    CK(alloc_mp(c, c->sec_arena, &c->sec_p, cap, L));
    CK(alloc_mp(c, c->sec_arena, &c->sec_t, 5, L));
    CK(alloc(c, c->sec_arena, reinterpret_cast<unsigned char **>(&c->sec_work), scalar_work_bytes(L)));
    CK(alloc(c, c->sec_arena, &c->sec_flags, 4));
    c->sec_cap = cap;
    c->sec_L = L;
  }
  c->sec_count = 0;
  // x_2 = 0: P(0) = det M, whose pivots give x_1 = -min_t D_t
  CK(cudaMemsetAsync(c->sec_x.limbs + L, 0, 4 * (size_t)L, c->stream));
  CK(cudaMemsetAsync(c->sec_x.sign + 1, 0, 4, c->stream));
  CK(cudaMemsetAsync(c->sec_x.exp + 1, 0, 8, c->stream));
  int rc = ldlt_dev(c, c->sec_x, 1, c->sec_p, 1);
  if (rc != HK_OK) return rc;
  CK(launch_neg_min_pivot(c->R, N, L, c->sec_x, 0, c->stream));
  rc = ldlt_dev(c, c->sec_x, 0, c->sec_p, 0);
  if (rc != HK_OK) return rc;
  int count = 2, have_last = 0;
  for (int k = 0; k < max_steps; k++) {
    CK(launch_secant_step(c->sec_x, c->sec_p, c->sec_t, count - 2, count - 1, count, k, have_last, L, c->sec_work,
                          c->sec_flags, c->stream));
    int f[4] = {0, 0, 0, 0};
    CK(cudaMemcpyAsync(f, c->sec_flags, sizeof(f), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (f[3]) return HK_ERR_TIMEOUT;  // a correction loop did not settle
    if (f[0] || f[1]) break;          // no secant, or the step stopped shrinking
    rc = ldlt_dev(c, c->sec_x, count, c->sec_p, count);
    if (rc != HK_OK) return rc;
    count++;
    CK(copy_entry(c->sec_t, 4, c->sec_t, 3, L, cudaMemcpyDeviceToDevice, c->stream));
    have_last = 1;
    if (f[2]) break;  // converged
  }
  c->sec_count = count;
  MpArr host{&root->sign, reinterpret_cast<long long *>(&root->exp), root->limbs};
  CK(copy_entry(host, 0, c->sec_x, count - 1, L, cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (dets_used) *dets_used = count;
  return HK_OK;
}

int hk_get_secant_flat(hk_ctx *c, int count, int32_t *xsign, int64_t *xexp, uint32_t *xlimbs, int32_t *psign,
                       int64_t *pexp, uint32_t *plimbs) {
  if (!c || count < 0 || !xsign || !xexp || !xlimbs || !psign || !pexp || !plimbs) return HK_ERR_ARG;
  if (count > c->sec_count) return HK_ERR_STATE;
  const int L = c->L;
  for (int k = 0; k < count; k++) {
    MpArr hx{xsign + k, reinterpret_cast<long long *>(xexp + k), xlimbs + (size_t)k * L};
    MpArr hp{psign + k, reinterpret_cast<long long *>(pexp + k), plimbs + (size_t)k * L};
    CK(copy_entry(hx, 0, c->sec_x, k, L, cudaMemcpyDeviceToHost, c->stream));
    CK(copy_entry(hp, 0, c->sec_p, k, L, cudaMemcpyDeviceToHost, c->stream));
  }
  CK(cudaStreamSynchronize(c->stream));
  return HK_OK;
}

int hk_secant_verify(hk_ctx *c, const hk_mp *x, int bits, int P2, int *out4) {
  if (!c || !mp_ok(x) || !out4 || bits < 1 || bits > 1024 || P2 % 32 || P2 > HK_MAX_P) return HK_ERR_ARG;
  if (!c->loaded) return HK_ERR_STATE;
  if ((long long)P2 < (long long)c->P + bits + 1) return HK_ERR_ARG;
  cudaSetDevice(c->device);
  const int N = c->N, L = c->L, L2 = P2 / 32, M = 2 * N - 1;
  bool z = true;
  for (int l = 0; l < L; l++) z &= x->limbs[l] == 0;
  if (z || !(x->limbs[L - 1] >> 31)) return HK_ERR_ARG;  // a nonzero, normalised root
  hk_ctx *c2 = nullptr;
  int rc = hk_create(&c2, c->device, c->stream);
  if (rc != HK_OK) return rc;
  Arena tmp;
  MpArr wm{}, xt{}, xv{};
  cudaError_t e = alloc_mp(c, tmp, &wm, M, L2);
  if (e == cudaSuccess) e = alloc_mp(c, tmp, &xt, 1, L);
  if (e == cudaSuccess) e = alloc_mp(c, tmp, &xv, 2, L2);
  if (e == cudaSuccess) e = launch_widen(c->mom, M, L, wm, L2, c->stream);
  if (e == cudaSuccess) {
    MpArr hx{const_cast<int32_t *>(&x->sign), reinterpret_cast<long long *>(const_cast<int64_t *>(&x->exp)),
             const_cast<uint32_t *>(x->limbs)};
    e = copy_entry(xt, 0, hx, 0, L, cudaMemcpyHostToDevice, c->stream);
  }
  if (e == cudaSuccess) e = launch_scale_pm(xt, 0, L, bits, -1, xv, 0, L2, c->stream);
  if (e == cudaSuccess) e = launch_scale_pm(xt, 0, L, bits, +1, xv, 1, L2, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  rc = e == cudaSuccess ? HK_OK : cuda_status(e);
  if (rc == HK_OK) rc = hk_load_moments_flat(c2, N, c->bnum, c->bden, P2, wm.sign, reinterpret_cast<int64_t *>(wm.exp),
                                             wm.limbs, 1);
  for (int side = 0; side < 2 && rc == HK_OK; side++) {
    rc = ldlt_dev(c2, xv, side, MpArr{}, 0);
    int sg = 0;
    if (rc == HK_OK) rc = read_counts(c2, &out4[side], nullptr);
    if (rc == HK_OK) rc = det_sign(c2, &sg);
    out4[2 + side] = sg;
  }
  tmp.release();
  hk_destroy(c2);
  return rc;
}


int hk_time_update_slice(hk_ctx *c, int tsteps, double *ms, double *macs) {
  if (!c || tsteps < 1 || !ms || !macs) return HK_ERR_ARG;
  if (!c->factored) return HK_ERR_STATE;
  cudaSetDevice(c->device);
  const int N = c->N, nb = c->nb, W = c->W;
  const int ts = std::min(tsteps, N);
  const int levels = c->fac_levels;
  Sched sc;
  CK(sched_for(c, W, W, levels, &sc));
  UpdParams up;
  std::memset(&up, 0, sizeof(up));
  up.wait_ns = c->wait_ns;
  up.mode = M_FACTOR;
  up.N = N;
  up.A = levels > 0 ? c->Aexp : c->A;
  up.Asign = c->Asign;
  up.astride = levels > 0 ? c->kl.stride : W;
  up.cx = up.cy = up.astride;
  up.colsum = c->colsum;
  up.a_len = levels > 0 ? c->Aexp_len : c->A_len;
  up.colsum_len = c->colsum_len;
  fill_sched(up, sc);
  up.st = c->st;
  const long long cta_per_out = (sc.n + UNT - 1) / UNT;
  const long long target = 6LL * sm_count(c) * 3;
  CK(reset_status(c));
  cudaEvent_t e0, e1;
  CK(cudaEventCreate(&e0));
  CK(cudaEventCreate(&e1));
  CK(cudaEventRecord(e0, c->stream));
  long long m = 0;
  // the contributions of the first `ts` rows (panel steps) to every later
  // entry: rows i < ts take t < i, later rows all t < ts; the result goes to
  // the factor's column-sum scratch and is discarded
  for (int r0 = 0; r0 < N; r0 += nb) {
    const int r1 = std::min(N, r0 + nb);
    for (int i = r0; i < r1;) {
      const bool early = i < ts;
      const int ra = i, rb = early ? i + 1 : r1;
      const int tend = early ? i : ts;
      i = rb;
      if (tend <= 0) continue;
      up.r0 = r0;
      up.ra = ra;
      up.rb = rb;
      up.nout = (int)rows_outputs(N, ra, rb);
      up.t0 = 0;
      up.t1 = tend;
      up.tchunk = pick_tchunk(tend, cta_per_out * up.nout, target);
      CK(launch_update(up, c->stream));
      m += (long long)tend * up.nout;
    }
  }
  CK(cudaEventRecord(e1, c->stream));
  CK(cudaEventSynchronize(e1));
  float t = 0;
  cudaEventElapsedTime(&t, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const DevStatus st = read_status(c);
  if (st.timeout) return HK_ERR_TIMEOUT;
  *ms = t;
  *macs = (double)m;
  return HK_OK;
}


int hk_selftest_scalar(int op, int L, const hk_mp *a, const hk_mp *b, hk_mp *out, int *cmp) {
  if (op < 0 || op > 3 || L < 1 || L > HK_MAX_P / 32 || !mp_ok(a) || !mp_ok(b)) return HK_ERR_ARG;
  if (op < 3 && (!out || !out->limbs)) return HK_ERR_ARG;
  if (op == 3 && !cmp) return HK_ERR_ARG;
  cudaStream_t s = nullptr;
  if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return HK_ERR_CUDA;
  MpArr da{}, db{}, dout{};
  void *work = nullptr;
  int *flags = nullptr;
  std::vector<void *> owned;
  auto get = [&](void **p, size_t bytes) {
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e == cudaSuccess) owned.push_back(*p);
    return e;
  };
  cudaError_t e = cudaSuccess;
  for (MpArr *m : {&da, &db, &dout}) {
    if (e == cudaSuccess) e = get(reinterpret_cast<void **>(&m->sign), 4);
    if (e == cudaSuccess) e = get(reinterpret_cast<void **>(&m->exp), 8);
    if (e == cudaSuccess) e = get(reinterpret_cast<void **>(&m->limbs), 4 * (size_t)L);
  }
  if (e == cudaSuccess) e = get(&work, scalar_work_bytes(L));
  if (e == cudaSuccess) e = get(reinterpret_cast<void **>(&flags), 16);
  if (e == cudaSuccess) e = cudaMemsetAsync(flags, 0, 16, s);
  MpArr ha{const_cast<int32_t *>(&a->sign), reinterpret_cast<long long *>(const_cast<int64_t *>(&a->exp)),
           const_cast<uint32_t *>(a->limbs)};
  MpArr hb{const_cast<int32_t *>(&b->sign), reinterpret_cast<long long *>(const_cast<int64_t *>(&b->exp)),
           const_cast<uint32_t *>(b->limbs)};
  if (e == cudaSuccess) e = copy_entry(da, 0, ha, 0, L, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = copy_entry(db, 0, hb, 0, L, cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = launch_scalar_selftest(op, da, db, dout, L, work, flags, s);
  int hf[4] = {0, 0, 0, 0};
  if (e == cudaSuccess && op < 3) {
    MpArr ho{&out->sign, reinterpret_cast<long long *>(&out->exp), out->limbs};
    e = copy_entry(ho, 0, dout, 0, L, cudaMemcpyDeviceToHost, s);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(hf, flags, 16, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  for (void *p : owned) cudaFree(p);
  cudaStreamDestroy(s);
  if (e != cudaSuccess) return HK_ERR_CUDA;
  if (op == 3) *cmp = hf[0];
  return hf[1] ? HK_ERR_TIMEOUT : HK_OK;
}

}  // extern "C"
