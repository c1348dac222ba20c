// C ABI of the deflated-CG library (declarations and contracts in include/dcg.h).
//
// A context owns its device workspace and a CUDA graph of one whole solve of
// Algorithm 1: the start-of-solve product and E = W^T A W, the initial
// projection and the first direction, then a device-side WHILE node over the
// iteration (operator, the fused iteration kernel, an IF node for the
// true-residual check / refinement and the direction update), an
// IF node for the final true residual, and the finishing kernel. The graph is built once per operator and
// replayed for every solve; kernels read the per-solve values (k, warm start,
// tolerances) from the device state, so nothing is re-captured between solves.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "dcg_kernels.cuh"

using namespace dcg;

enum OpKind { OP_NONE = 0, OP_DENSE = 1, OP_RBF = 2 };

struct dcg_ctx {
  dcg_config cfg;
  cudaStream_t stream = nullptr;
  cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
  int device = 0;
  int num_sms = 0;
  std::string err;
  std::vector<void*> allocs;

  Ws w{};
  DevState* st = nullptr;     // device
  DevState* h_st = nullptr;   // pinned host copy
  int* h_small = nullptr;     // pinned: ritz k_out, status
  double* gramE_part = nullptr;

  // harmonic Ritz buffers
  double *F = nullptr, *G = nullptr, *Vd = nullptr, *Vd2 = nullptr, *theta = nullptr, *ritz_part = nullptr, *colscale = nullptr;
  float *Vj = nullptr, *U = nullptr, *Wout = nullptr;
  int *k_out = nullptr, *ritz_status = nullptr;
  int k_active = 0;
  int m_last = 0;        // number of harmonic Ritz values of the last update
  int m_pencil = 0;      // order of the last update's pencil F, G (columns of Z)
  bool have_solve = false;
  bool ritz_pending = false;  // an update was enqueued and its result not yet read
  int last_iters = 0;

  int test_barrier_polls = 0;  // > 0: the next solve withholds a grid-barrier arrival (test hook)
  float* lap_v32 = nullptr;    // Laplace Newton step: float32 copies of c or a (n)
  float* lap_kv = nullptr;     // and the GEMV result K c or K a (n)
  bool dense_sym = false;      // stored operator given as its upper triangle (symmetric matvec)
  float* sym_rowpart = nullptr;
  float* sym_colpart = nullptr;
  int* sym_sched = nullptr;        // symmetric matvec: the item counter, then the items largest first
  int sym_nitems = 0;
  bool fg_sparse_used = false;     // the last extraction formed F, G from the recorded scalars
  // symmetric matrix-free matvec: row sums, column sums of the tile pairs,
  // the row-block counter
  float* mf_rowpart = nullptr;
  float* mf_colpart = nullptr;
  unsigned int* mf_ctr = nullptr;
  // tensor-core block product (k_apply_tc): A's map (set with the stored
  // operator) and the map of W (columns 1.. of XW, fixed at create)
  CUtensorMap tmap_ab{};
  CUtensorMap tmap_w{};
  bool ab_tc = false;               // tmap_ab holds the current operator
  bool w_tc = false;                // tmap_w is valid

  // operator
  int op = OP_NONE;
  const float* A = nullptr;
  int64_t lda = 0;
  CUtensorMap tmap;
  // matrix-free RBF operator (owned copies of the points)
  int n_pad = 0;             // n rounded up to the 128-row tile
  int rbf_d = 0, rbf_xformat = 0;
  float* Xr = nullptr;       // n x 64 capacity, rounded points
  void* Xt = nullptr;        // n_pad x 128 bytes tensor-core tiles
  float* nsq = nullptr;      // n_pad
  float* vcol = nullptr;     // n_pad
  RbfParams* prm = nullptr;
  // exact-form residual: transposed points, |x_i|^2 split on the anchor grid,
  // per-split partial sums
  float* XrT = nullptr;      // 64 x n_pad
  double* n64 = nullptr;     // n_pad
  unsigned int* nmax = nullptr;
  float* nh = nullptr;       // n_pad
  float* nl = nullptr;       // n_pad
  float* resid_part = nullptr;  // 3 x resid_splits x n
  int resid_splits = 1;
  float* pmv = nullptr;      // n_pad: padded copy of a caller's p (single-step matvec)
  float* pmvb = nullptr;     // rbf_block_nc() x n_pad: padded W columns of one multi-column pass
  double rbf_l = 0.0, rbf_s2 = 0.0, rbf_noise = 0.0;  // current hyperparameters (host copy)
  double* dth_partials = nullptr;  // derivative forms: 3 * kMaxDthetaPairs per CTA
  double* dth_out = nullptr;       // 3 * kMaxDthetaPairs
  unsigned int* dth_ticket = nullptr;
  CUtensorMap rbf_tmap[2];   // tile copies of the points: I-tile rows, J-tile rows
  int rbf_grid = 1;

  // split-K partials of the block product
  float* block_scratch = nullptr;

  // lockstep solves of several right-hand sides (dcg_solve_multi): per-system
  // vectors and states, allocated by the first call that needs them
  int mr_cap = 0;              // systems the buffers hold
  size_t mr_vs = 0;            // stride of the per-system vectors (n rounded up to 64)
  std::vector<void*> mr_allocs;
  float* mr_p = nullptr;       // mr_cap x n_pad directions (zero tails)
  float *mr_xh = nullptr, *mr_xl = nullptr, *mr_r = nullptr, *mr_b = nullptr;  // mr_cap x n
  double *mr_xd = nullptr, *mr_xbest = nullptr;                                  // mr_cap x n
  double* mr_small = nullptr;  // mr_cap x 4 kk: h, hp, mu, gamma
  float* mr_small_f = nullptr; // mr_cap x 2 kk: mu_f, gamma_f
  float *mr_P = nullptr, *mr_Q = nullptr;  // gathered directions and their products, mr_ld x (mr_cap rounded up to 8)
  float* mr_resid_part = nullptr;  // matrix-free residuals of EX_NL systems per pass: EX_NL x 3 x splits x n
  uint16_t* mr_phl = nullptr;  // float16 parts of the gathered directions (rbf_p16_halfs(n_pad))
  float* mr_pscale = nullptr;  // their power-of-two column scales (32)
  CUtensorMap mr_pmaps[2];     // maps of mr_phl for 16 and 32 columns
  bool mr_tc = false;          // the maps are valid: the block product contracts on the tensor cores
  DevState* mr_st = nullptr;   // mr_cap + 1 states; the last records timeouts of the shared kernels
  DevState* mr_hst = nullptr;  // pinned copies

  // standalone matvec scratch
  double* mv_partials = nullptr;
  double* mv_result = nullptr;
  unsigned int* mv_ticket = nullptr;

  // solve graph
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool graph_valid = false;
  Handles h{};
  int grid_rows = 1, grid_iter = 1;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr, ev2 = nullptr;
};

// Message of the last failed call made without a context, per host thread
// (calls on different threads do not overwrite each other's message).
static thread_local std::string g_create_err;
static std::mutex g_mu;
static EncodeTiledFn g_encode = nullptr;

static dcg_status fail(dcg_ctx* c, dcg_status s, const std::string& msg) {
  if (c)
    c->err = msg;
  else
    g_create_err = msg;
  return s;
}

static dcg_status finish_update(dcg_ctx* c);  // waits for a pending asynchronous update

static dcg_status cuda_fail(dcg_ctx* c, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) return fail(c, DCG_ERR_NOMEM, m);
  return fail(c, DCG_ERR_CUDA, m);
}

#define CK(call)                                         \
  do {                                                   \
    cudaError_t e_ = (call);                             \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
  } while (0)

static EncodeTiledFn get_encode() {
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_encode) {
    void* fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  return g_encode;
}

template <typename T>
static cudaError_t dalloc(dcg_ctx* c, T** p, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T) + 16);
  if (e != cudaSuccess) return e;
  c->allocs.push_back(v);
  *p = static_cast<T*>(v);
  return cudaMemsetAsync(v, 0, count * sizeof(T) + 16, c->stream);
}

extern "C" const char* dcg_status_string(dcg_status s) {
  switch (s) {
    case DCG_OK: return "ok";
    case DCG_ERR_INVALID_ARG: return "invalid argument";
    case DCG_ERR_NOMEM: return "out of device memory";
    case DCG_ERR_CUDA: return "CUDA error";
    case DCG_ERR_BREAKDOWN: return "breakdown: p^T A p <= 0 (operator not SPD)";
    case DCG_ERR_SUBSPACE_SINGULAR: return "deflation subspace singular";
    case DCG_ERR_MAXITER: return "maximum iterations reached";
    case DCG_ERR_TIMEOUT: return "device-side wait timed out";
    case DCG_ERR_STATE: return "call out of order";
    case DCG_ERR_UNSUPPORTED: return "unsupported configuration";
    case DCG_ERR_STAGNATION: return "stagnation: the true residual stopped decreasing above tol";
  }
  return "unknown status";
}

extern "C" const char* dcg_last_error(const dcg_ctx* c) {
  return c ? c->err.c_str() : g_create_err.c_str();
}

static void destroy_graph(dcg_ctx* c) {
  if (c->exec) cudaGraphExecDestroy(c->exec);
  if (c->graph) cudaGraphDestroy(c->graph);
  c->exec = nullptr;
  c->graph = nullptr;
  c->graph_valid = false;
}

extern "C" dcg_status dcg_destroy(dcg_ctx* c) {
  if (!c) return DCG_OK;
  cudaStreamSynchronize(c->stream);
  destroy_graph(c);
  for (void* p : c->allocs) cudaFree(p);
  for (void* p : c->mr_allocs) cudaFree(p);
  if (c->mr_hst) cudaFreeHost(c->mr_hst);
  if (c->h_st) cudaFreeHost(c->h_st);
  if (c->h_small) cudaFreeHost(c->h_small);
  for (auto& s : c->cap)
    if (s) cudaStreamDestroy(s);
  if (c->ev0) cudaEventDestroy(c->ev0);
  if (c->ev1) cudaEventDestroy(c->ev1);
  if (c->ev2) cudaEventDestroy(c->ev2);
  delete c;
  return DCG_OK;
}

extern "C" dcg_status dcg_create(const dcg_config* cfg, void* stream, dcg_ctx** out) {
  if (!cfg || !out) return fail(nullptr, DCG_ERR_INVALID_ARG, "cfg and out must not be NULL");
  *out = nullptr;
  const dcg_config& g = *cfg;
  for (int i = 0; i < 4; ++i)
    if (g.reserved[i]) return fail(nullptr, DCG_ERR_INVALID_ARG, "reserved fields must be zero");
  if (g.host_loop != 0 && g.host_loop != 1) return fail(nullptr, DCG_ERR_INVALID_ARG, "host_loop must be 0 or 1");
  if (g.n < 1 || g.n > (int64_t(1) << 30)) return fail(nullptr, DCG_ERR_INVALID_ARG, "n out of range");
  {
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) == cudaSuccess &&
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) == cudaSuccess && sms > 0 &&
        g.n > iter_max_n(sms))
      return fail(nullptr, DCG_ERR_UNSUPPORTED,
                  "n above " + std::to_string(iter_max_n(sms)) + " (one co-resident CTA per SM, at most 32 passes of 128 rows each)");
  }
  if (g.k < 0 || g.ell < 0 || g.k > g.n || g.ell > g.n) return fail(nullptr, DCG_ERR_INVALID_ARG, "k, ell out of range");
  if (g.max_iter < 1) return fail(nullptr, DCG_ERR_INVALID_ARG, "max_iter must be >= 1");
  if (!(g.tol > 0.0)) return fail(nullptr, DCG_ERR_INVALID_ARG, "tol must be > 0");
  if (g.window != DCG_WINDOW_FIRST && g.window != DCG_WINDOW_LAST)
    return fail(nullptr, DCG_ERR_INVALID_ARG, "bad window");
  if (g.select != DCG_SELECT_LARGEST && g.select != DCG_SELECT_SMALLEST)
    return fail(nullptr, DCG_ERR_INVALID_ARG, "bad select");
  if (g.extraction != DCG_EXTRACT_HARMONIC && g.extraction != DCG_EXTRACT_RITZ)
    return fail(nullptr, DCG_ERR_INVALID_ARG, "bad extraction");
  if (g.fg_form != DCG_FG_EXPLICIT && g.fg_form != DCG_FG_SPARSE)
    return fail(nullptr, DCG_ERR_INVALID_ARG, "bad fg_form");
  if (g.fg_form == DCG_FG_SPARSE && g.extraction != DCG_EXTRACT_HARMONIC)
    return fail(nullptr, DCG_ERR_INVALID_ARG, "fg_form sparse needs the harmonic extraction");
  if (g.refine_every < 0) return fail(nullptr, DCG_ERR_INVALID_ARG, "refine_every must be >= 0");
  if (g.k > kMaxK || g.ell > kMaxEll)
    return fail(nullptr, DCG_ERR_UNSUPPORTED, "k <= 96 and ell <= 128 in this build");

  dcg_ctx* c = new dcg_ctx();
  c->cfg = g;
  c->stream = static_cast<cudaStream_t>(stream);
  c->err.clear();
  auto bail = [&](dcg_status s) {
    g_create_err = c->err;
    dcg_destroy(c);
    return s;
  };
#define CKC(call)                                              \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) return bail(cuda_fail(c, e_, #call)); \
  } while (0)
  CKC(cudaGetDevice(&c->device));
  CKC(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device));
  for (auto& s : c->cap) CKC(cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking));
  CKC(cudaEventCreate(&c->ev0));
  CKC(cudaEventCreate(&c->ev1));
  CKC(cudaEventCreate(&c->ev2));
  CKC(rowop_configure());
  CKC(symv_configure());
  CKC(apply_tc_configure());
  CKC(apply_block_configure());
  CKC(iter_configure());
  CKC(rbf_mv_configure());
  CKC(rbf_mv_sym_configure());
  CKC(rbf_mv_tc_configure());
  CKC(chol_configure(96));
  CKC(ritz_configure());

  const int n = int(g.n), kmax = g.k, ellmax = g.ell;
  c->grid_rows = rowop_grid(n, c->num_sms);
  c->grid_iter = std::max(1, std::min(c->num_sms, (n + 63) / 64));
  Ws& w = c->w;
  w.n = n;
  w.kmax = kmax;
  w.ellmax = ellmax;
  w.tol = g.tol;
  CKC(dalloc(c, &w.XW, size_t(n) * (1 + kmax)));
  CKC(dalloc(c, &w.Y, size_t(n) * (1 + kmax)));
  CKC(dalloc(c, &w.xd, size_t(n)));
  CKC(dalloc(c, &w.xbest, size_t(n)));
  CKC(dalloc(c, &w.xh, size_t(n)));
  CKC(dalloc(c, &w.xl, size_t(n)));
  CKC(dalloc(c, &w.r, size_t(n)));
  c->n_pad = (n + 127) / 128 * 128;
  CKC(dalloc(c, &w.p, size_t(c->n_pad)));  // zero tail: the matrix-free kernel reads whole 128-row tiles
  CKC(dalloc(c, &w.q, size_t(n)));
  CKC(dalloc(c, &w.b, size_t(n)));
  CKC(dalloc(c, &w.P, size_t(n) * std::max(ellmax, 1)));
  CKC(dalloc(c, &w.Q, size_t(n) * std::max(ellmax, 1)));
  const int kk = std::max(kmax, 1);
  CKC(dalloc(c, &w.E, size_t(kk) * kk));
  CKC(dalloc(c, &w.Linv, size_t(kk) * kk));
  CKC(dalloc(c, &w.GW, size_t(kk) * kk));
  CKC(dalloc(c, &w.Einv, size_t(kk) * kk));
  CKC(dalloc(c, &w.N, size_t(kk) * kk));
  CKC(dalloc(c, &w.NT, size_t(kk) * kk));
  CKC(dalloc(c, &w.mats2, size_t(3) * kk * kk));
  CKC(dalloc(c, &w.M, size_t(kk) * kk));
  CKC(dalloc(c, &w.h, size_t(kk)));
  CKC(dalloc(c, &w.hp, size_t(kk)));
  CKC(dalloc(c, &w.mu, size_t(kk)));
  CKC(dalloc(c, &w.gamma, size_t(kk)));
  CKC(dalloc(c, &w.mu_f, size_t(kk)));
  CKC(dalloc(c, &w.gamma_f, size_t(kk)));
  CKC(dalloc(c, &w.partials, size_t(std::max(c->grid_iter, c->grid_rows)) * kReduceSlots));
  const int hist_cap = g.record_history ? g.max_iter + 2 : 1;
  CKC(dalloc(c, &w.hist, size_t(hist_cap)));
  if (ellmax > 0) CKC(dalloc(c, &w.fg, fg_doubles(ellmax, kmax)));
  CKC(dalloc(c, &c->st, 1));
  w.st = c->st;
  CKC(dalloc(c, &c->gramE_part, gram_partials_doubles(n, kk, c->num_sms)));
  const int m = kmax + ellmax;
  const int mm = std::max(m, 1);
  CKC(dalloc(c, &c->F, size_t(mm) * mm));
  CKC(dalloc(c, &c->G, size_t(mm) * mm));
  CKC(dalloc(c, &c->Vd, size_t(mm) * mm));
  CKC(dalloc(c, &c->Vd2, size_t(mm) * mm));
  CKC(dalloc(c, &c->Vj, size_t(mm) * (mm + 1)));
  CKC(dalloc(c, &c->theta, size_t(mm)));
  CKC(dalloc(c, &c->U, size_t(mm) * kk));
  CKC(dalloc(c, &c->Wout, size_t(n) * kk));
  CKC(dalloc(c, &c->colscale, size_t(kk)));
  CKC(dalloc(c, &c->k_out, 2));
  CKC(dalloc(c, &c->ritz_status, 1));
  CKC(dalloc(c, &c->ritz_part, gram_partials_doubles(n, mm, c->num_sms)));
  CKC(dalloc(c, &c->mv_partials,
              2 * size_t(std::max(std::max(c->grid_rows, 2 * c->num_sms),
                                  std::max(rbf_exact_grid(n), symv_fin_grid(n, c->num_sms)))) + 2));
  {
    const size_t bs = std::max(apply_block_scratch_floats(n, kMaxBlockCols, c->num_sms),
                               apply_tc_scratch_floats(n, kMaxBlockCols, c->num_sms));
    if (bs) CKC(dalloc(c, &c->block_scratch, bs));
  }
  if (kmax > 0 && apply_tc_supported(n, kmax) && apply_tc_preferred(kmax)) {
    EncodeTiledFn enc = get_encode();
    c->w_tc = enc && make_apply_tc_tmaps(nullptr, &c->tmap_w, nullptr, 0, w.XW + n, n, kmax, enc);
  }
  CKC(dalloc(c, &c->mv_result, 2));
  CKC(dalloc(c, &c->mv_ticket, 1));
  CKC(cudaMallocHost(&c->h_st, sizeof(DevState)));
  CKC(cudaMallocHost(&c->h_small, 4 * sizeof(int)));
  memset(c->h_st, 0, sizeof(DevState));
  CKC(cudaStreamSynchronize(c->stream));
#undef CKC
  *out = c;
  return DCG_OK;
}

// ---------------------------------------------------------------------------
// Operators
// ---------------------------------------------------------------------------
static dcg_status set_dense(dcg_ctx* c, const float* A, int64_t lda, bool sym) {
  if (!c) return DCG_ERR_INVALID_ARG;
  if (!A) return fail(c, DCG_ERR_INVALID_ARG, "A is NULL");
  if (lda < c->cfg.n || (lda % 4) != 0) return fail(c, DCG_ERR_INVALID_ARG, "lda must be >= n and a multiple of 4");
  if ((reinterpret_cast<uintptr_t>(A) & 15) != 0) return fail(c, DCG_ERR_INVALID_ARG, "A must be 16-byte aligned");
  EncodeTiledFn enc = get_encode();
  if (!enc) return fail(c, DCG_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  if (sym && !c->sym_rowpart) {
    CK(dalloc(c, &c->sym_rowpart, symv_rowpart_floats(c->w.n)));
    CK(dalloc(c, &c->sym_colpart, symv_colpart_floats(c->w.n)));
    std::vector<int> items;
    symv_schedule(c->w.n, items);
    CK(dalloc(c, &c->sym_sched, 1 + items.size()));  // zeroed: the counter starts at 0
    CK(cudaMemcpyAsync(c->sym_sched + 1, items.data(), items.size() * sizeof(int), cudaMemcpyHostToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->sym_nitems = int(items.size());
  }
  const bool same = (c->op == OP_DENSE && c->A == A && c->lda == lda && c->dense_sym == sym);
  if (!same) {
    CUtensorMap m;
    if (!make_rowop_tmap(&m, A, c->cfg.n, lda, enc)) return fail(c, DCG_ERR_INVALID_ARG, "tensor map encode failed");
    c->tmap = m;
    c->A = A;
    c->lda = lda;
    c->op = OP_DENSE;
    c->dense_sym = sym;
    c->ab_tc = apply_tc_supported(c->cfg.n, std::max(c->w.kmax, 1)) &&
               make_apply_tc_tmaps(&c->tmap_ab, nullptr, A, lda, nullptr, c->cfg.n, 0, enc);
    destroy_graph(c);
  }
  return DCG_OK;
}

extern "C" dcg_status dcg_set_operator_dense(dcg_ctx* c, const float* A, int64_t lda) {
  return set_dense(c, A, lda, false);
}

extern "C" dcg_status dcg_set_operator_dense_sym(dcg_ctx* c, const float* A, int64_t lda) {
  return set_dense(c, A, lda, true);
}

extern "C" dcg_status dcg_set_operator_rbf(dcg_ctx* c, const float* X, int32_t d, int32_t xformat, double l,
                                           double s2, double noise) {
  if (!c) return DCG_ERR_INVALID_ARG;
  if (!X) return fail(c, DCG_ERR_INVALID_ARG, "X is NULL");
  if (!(l > 0.0) || !(s2 > 0.0) || !(noise >= 0.0)) return fail(c, DCG_ERR_INVALID_ARG, "bad RBF parameters");
  if (xformat != DCG_X_BF16 && xformat != DCG_X_TF32 && xformat != DCG_X_FP32)
    return fail(c, DCG_ERR_INVALID_ARG, "matrix-free operator: unknown xformat");
  if (d < 1 || d > rbf_max_d(xformat))
    return fail(c, DCG_ERR_UNSUPPORTED, "matrix-free operator: d <= " + std::to_string(rbf_max_d(DCG_X_BF16)) +
                                            " (BF16), " + std::to_string(rbf_max_d(DCG_X_TF32)) + " (TF32) or " +
                                            std::to_string(rbf_max_d(DCG_X_FP32)) + " (FP32)");
  EncodeTiledFn enc = get_encode();
  if (!enc) return fail(c, DCG_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  const int n = c->w.n, n_pad = c->n_pad;
  if (!c->Xr) {
    CK(dalloc(c, &c->Xr, size_t(n) * 64));
    CK(dalloc(c, reinterpret_cast<unsigned char**>(&c->Xt), size_t(2) * n_pad * 128));
    CK(dalloc(c, &c->nsq, size_t(n_pad)));
    CK(dalloc(c, &c->vcol, size_t(n_pad)));
    CK(dalloc(c, &c->prm, 1));
    CK(dalloc(c, &c->pmv, size_t(n_pad)));
    CK(dalloc(c, &c->pmvb, size_t(rbf_block_nc()) * n_pad));
    CK(dalloc(c, &c->mf_rowpart, size_t(n_pad)));
    CK(dalloc(c, &c->mf_colpart, rbf_mv_sym_colpart_floats(n_pad)));
    CK(dalloc(c, &c->mf_ctr, 1));  // zeroed: the counter starts at 0
    c->resid_splits = rbf_resid_splits(n, c->num_sms);
    CK(dalloc(c, &c->XrT, size_t(64) * n_pad));
    CK(dalloc(c, &c->n64, size_t(n_pad)));
    CK(dalloc(c, &c->nmax, 1));
    CK(dalloc(c, &c->nh, size_t(n_pad)));
    CK(dalloc(c, &c->nl, size_t(n_pad)));
    CK(dalloc(c, &c->resid_part, size_t(3) * c->resid_splits * n));
  }
  CK(launch_rbf_prep(X, n, n_pad, d, xformat, c->Xr, c->Xt, c->nsq, c->stream));
  CK(launch_rbf_anchor(c->Xr, n, n_pad, d, c->n64, c->nmax, c->prm, c->nh, c->nl, c->XrT, c->stream));
  CK(launch_rbf_params(c->nsq, n, n_pad, d, l, s2, noise, c->vcol, c->prm, c->stream));
  CUtensorMap m[2];
  if (!make_rbf_tmap(m, c->Xt, n_pad, xformat, d, enc)) return fail(c, DCG_ERR_INVALID_ARG, "tensor map encode failed");
  c->rbf_tmap[0] = m[0];
  c->rbf_tmap[1] = m[1];
  c->rbf_d = d;
  c->rbf_xformat = xformat;
  c->rbf_l = l;
  c->rbf_s2 = s2;
  c->rbf_noise = noise;
  c->rbf_grid = rbf_mv_grid(n_pad / 128, c->num_sms);
  c->op = OP_RBF;
  c->A = nullptr;
  destroy_graph(c);
  return DCG_OK;
}

extern "C" dcg_status dcg_set_rbf_params(dcg_ctx* c, double l, double s2, double noise) {
  if (!c) return DCG_ERR_INVALID_ARG;
  if (c->op != OP_RBF) return fail(c, DCG_ERR_STATE, "no matrix-free operator set");
  if (!(l > 0.0) || !(s2 > 0.0) || !(noise >= 0.0)) return fail(c, DCG_ERR_INVALID_ARG, "bad RBF parameters");
  CK(launch_rbf_params(c->nsq, c->w.n, c->n_pad, c->rbf_d, l, s2, noise, c->vcol, c->prm, c->stream));
  c->rbf_l = l;
  c->rbf_s2 = s2;
  c->rbf_noise = noise;
  return DCG_OK;
}

// u_p^T (dA/dtheta) v_p for theta = (l, s^2, noise) of the current matrix-free
// operator, from the kernel's SD, SE, SI forms: dA/dl = s^2 E .* D / l^3,
// dA/ds^2 = E, dA/dnoise = I.
extern "C" dcg_status dcg_rbf_dtheta(dcg_ctx* c, const float* U, const float* V, int32_t npairs, double* out) {
  if (!c) return DCG_ERR_INVALID_ARG;
  if (c->op != OP_RBF) return fail(c, DCG_ERR_STATE, "no matrix-free operator set");
  if (!U || !V || !out) return fail(c, DCG_ERR_INVALID_ARG, "U, V and out are required");
  if (npairs < 1 || npairs > kMaxDthetaPairs)
    return fail(c, DCG_ERR_INVALID_ARG, "npairs must be in [1, " + std::to_string(kMaxDthetaPairs) + "]");
  const int n = c->w.n;
  if (!c->dth_partials) {
    CK(dalloc(c, &c->dth_partials, size_t(3) * kMaxDthetaPairs * rbf_dtheta_grid(n)));
    CK(dalloc(c, &c->dth_out, size_t(3) * kMaxDthetaPairs));
    CK(dalloc(c, &c->dth_ticket, 1));
  }
  RbfDthetaArgs a{};
  a.Xr = c->Xr;
  a.n = n;
  a.d = c->rbf_d;
  a.prm = c->prm;
  a.U = U;
  a.V = V;
  a.npairs = npairs;
  a.partials = c->dth_partials;
  a.ticket = c->dth_ticket;
  a.out = c->dth_out;
  CK(launch_rbf_dtheta(a, c->stream));
  std::vector<double> raw(size_t(3) * npairs);
  CK(cudaMemcpyAsync(raw.data(), c->dth_out, raw.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  const double l = c->rbf_l, s2 = c->rbf_s2;
  for (int p = 0; p < npairs; ++p) {
    out[3 * p] = s2 * raw[3 * p] / (l * l * l);
    out[3 * p + 1] = raw[3 * p + 1];
    out[3 * p + 2] = raw[3 * p + 2];
  }
  return DCG_OK;
}

extern "C" dcg_status dcg_form_rbf_dense(const float* X, int64_t n, int32_t d, double l, double s2, double noise,
                                         float* A, int64_t lda, void* stream) {
  if (!X || !A) return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_form_rbf_dense: X and A are required");
  if (n < 1 || n > (int64_t(1) << 30) || lda < n)
    return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_form_rbf_dense: need 1 <= n <= 2^30 and lda >= n");
  if (d < 1 || d > 4096) return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_form_rbf_dense: d must be in [1, 4096]");
  if (!(l > 0.0) || !std::isfinite(l) || !std::isfinite(s2) || !std::isfinite(noise))
    return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_form_rbf_dense: lengthscale > 0 and finite parameters");
  cudaError_t e = launch_form_rbf(X, int(n), d, l, s2, noise, A, lda, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return fail(nullptr, DCG_ERR_CUDA, std::string("dcg_form_rbf_dense: ") + cudaGetErrorString(e));
  return DCG_OK;
}

// q = A p and p^T q for a dense operator with no context: the matvec kernel
// of dcg_matvec on the library's fixed scratch instead of context buffers.
extern "C" dcg_status dcg_matvec_dense_noalloc(const float* A, int64_t n, int64_t lda, const float* p, float* q,
                                               double* pAp, void* stream) {
  if (!A || !p || !q) return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_matvec_dense_noalloc: A, p and q are required");
  if (n < 1 || n > (int64_t(1) << 30))
    return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_matvec_dense_noalloc: n out of range [1, 2^30]");
  if (lda < n || (lda % 4) != 0)
    return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_matvec_dense_noalloc: lda must be >= n and a multiple of 4");
  if ((reinterpret_cast<uintptr_t>(A) & 15) != 0 || (reinterpret_cast<uintptr_t>(p) & 15) != 0)
    return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_matvec_dense_noalloc: A and p must be 16-byte aligned");
  dcg_ctx* c = nullptr;  // errors below are reported without a context
  int dev = 0, sms = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = rowop_grid(int(n), sms);
  if (grid > noalloc_max_ctas())
    return fail(nullptr, DCG_ERR_UNSUPPORTED,
                "dcg_matvec_dense_noalloc: this device needs " + std::to_string(grid) +
                    " reduction slots; the fixed scratch holds " + std::to_string(noalloc_max_ctas()));
  void* scratch = nullptr;
  CK(noalloc_scratch(&scratch));
  EncodeTiledFn enc = get_encode();
  if (!enc) return fail(nullptr, DCG_ERR_CUDA, "dcg_matvec_dense_noalloc: cuTensorMapEncodeTiled unavailable");
  CUtensorMap m;
  if (!make_rowop_tmap(&m, A, n, lda, enc))
    return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_matvec_dense_noalloc: tensor map encode failed");
  CK(launch_matvec_noalloc(&m, p, q, int(n), pAp, grid, scratch, static_cast<cudaStream_t>(stream)));
  return DCG_OK;
}

// ---------------------------------------------------------------------------
// Operator launches (one place per operator kind)
// ---------------------------------------------------------------------------
static cudaError_t op_matvec(dcg_ctx* c, const float* p, float* q, double* result, double* partials,
                             unsigned int* ticket, DevState* st, cudaStream_t s) {
  if (c->op == OP_RBF) {
    RbfMvArgs a{};
    a.p = p;  // n_pad floats with a zero tail
    a.vcol = c->vcol;
    a.q = q;
    a.n = c->w.n;
    a.n_tiles = c->n_pad / 128;
    a.d = c->rbf_d;
    a.xformat = c->rbf_xformat;
    a.prm = c->prm;
    a.partials = partials;
    a.ticket = ticket;
    a.result = result;
    a.st = st;
    a.skip_if_done = st ? 1 : 0;
    a.col_idx = -1;
    a.rowpart = c->mf_rowpart;
    a.colpart = c->mf_colpart;
    a.sched_ctr = c->mf_ctr;
    return launch_rbf_mv_sym(c->rbf_tmap, a, c->rbf_grid, s);
  }
  if (c->dense_sym) {
    SymvArgs a{};
    a.p = p;
    a.q = q;
    a.n = c->w.n;
    a.rowpart = c->sym_rowpart;
    a.colpart = c->sym_colpart;
    a.sched_ctr = reinterpret_cast<unsigned int*>(c->sym_sched);
    a.sched_items = c->sym_sched + 1;
    a.nitems = c->sym_nitems;
    a.partials = partials;
    a.ticket = ticket;
    a.result = result;
    a.st = st;
    a.skip_if_done = st ? 1 : 0;
    return launch_symv(&c->tmap, a, c->num_sms, s);
  }
  RowOpArgs a{};
  a.v = p;
  a.out = q;
  a.n = c->w.n;
  a.partials = partials;
  a.ticket = ticket;
  a.result = result;
  a.st = st;
  a.skip_if_done = st ? 1 : 0;
  return launch_rowop(&c->tmap, a, false, c->grid_rows, s);
}

// Arguments of the matrix-free exact-form residual shared by the solve and
// dcg_residual.
static RbfExactArgs rbf_resid_args(dcg_ctx* c) {
  RbfExactArgs a{};
  a.Xr = c->Xr;
  a.XrT = c->XrT;
  a.nh = c->nh;
  a.nl = c->nl;
  a.n = c->w.n;
  a.n_pad = c->n_pad;
  a.d = c->rbf_d;
  a.prm = c->prm;
  a.partials_f = c->resid_part;
  a.partials = c->mv_partials;
  return a;
}

// r = b - A x for the float64 iterate (compensated sums), with the state's
// check / refinement bookkeeping; mode as in RowOpArgs::resid_mode.
// w: the workspace of the solve (the context's, or one system of a lockstep
// multi-right-hand-side solve).
static cudaError_t op_resid_w(dcg_ctx* c, const Ws& w, int mode, int skip_if_done, cudaStream_t s) {
  cudaError_t e = launch_split_x(w, c->grid_iter, skip_if_done, s);
  if (e != cudaSuccess) return e;
  if (c->op == OP_RBF) {
    RbfExactArgs a = rbf_resid_args(c);
    a.xh = w.xh;
    a.xl = w.xl;
    a.b = w.b;
    a.r = w.r;
    a.ticket = &w.st->ticket[T_CHECK_RES];
    a.st = w.st;
    a.skip_if_done = skip_if_done;
    a.resid_mode = mode;
    return launch_rbf_resid(a, c->resid_splits, s);
  }
  RowOpArgs a{};
  a.xh = w.xh;
  a.xl = w.xl;
  a.out = w.r;
  a.b = w.b;
  a.n = w.n;
  a.partials = c->mv_partials;
  a.ticket = &w.st->ticket[T_CHECK_RES];
  a.result = nullptr;
  a.st = w.st;
  a.skip_if_done = skip_if_done;
  a.resid_mode = mode;
  return launch_rowop(&c->tmap, a, true, c->grid_rows, s);
}

static cudaError_t op_resid(dcg_ctx* c, int mode, int skip_if_done, cudaStream_t s) {
  return op_resid_w(c, c->w, mode, skip_if_done, s);
}

// st: the solve's state (start-of-solve product AW, k = st->k columns of W);
// null for a plain block of ncols columns, whose bounded waits record a
// timeout in tst (the context's state if null).
static cudaError_t op_block(dcg_ctx* c, const float* V, int ncols, float* Y, DevState* st, cudaStream_t s,
                            DevState* tst = nullptr) {
  if (c->op == OP_RBF && st) {
    // Start of a solve: AW with the same tensor-core operator the iteration
    // applies, so that the deflation (E, mu, the re-deflation of r) is
    // consistent with the Krylov recursion; passes of rbf_block_nc() columns,
    // each entry's exponential formed once per pass.
    const int nc = rbf_block_nc();
    for (int col0 = 0; col0 < c->w.kmax; col0 += nc) {
      cudaError_t e = launch_copy_cols(V + int64_t(1 + col0) * c->w.n, c->pmvb, c->w.n, c->n_pad, col0, nc, st, s);
      if (e != cudaSuccess) return e;
      RbfMvArgs a{};
      a.p = c->pmvb;
      a.ldp = c->n_pad;
      a.vcol = c->vcol;
      a.q = Y + int64_t(1 + col0) * c->w.n;
      a.ldq = c->w.n;
      a.ncols = nc;
      a.n = c->w.n;
      a.n_tiles = c->n_pad / 128;
      a.d = c->rbf_d;
      a.xformat = c->rbf_xformat;
      a.prm = c->prm;
      a.st = st;
      a.skip_if_done = 1;
      a.col_idx = col0;
      if ((e = launch_rbf_mv_block(c->rbf_tmap, a, c->rbf_grid, s)) != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  if (c->op == OP_RBF) {
    RbfExactArgs a{};
    a.Xr = c->Xr;
    a.n = c->w.n;
    a.d = c->rbf_d;
    a.prm = c->prm;
    a.V = V;
    a.Y = Y;
    a.ncols = ncols;
    a.st = st;
    a.skip_if_done = st ? 1 : 0;
    return launch_rbf_block(a, st ? c->w.kmax : ncols, s);
  }
  ApplyBlockArgs a{};
  a.A = c->A;
  a.lda = c->lda;
  a.V = V;
  a.Y = Y;
  a.n = c->w.n;
  a.c = ncols;
  a.st = st;
  a.skip_if_done = st ? 1 : 0;
  // tensor cores (split TF32) where the operands allow TMA and there are more
  // than 16 columns; the FP32-pipe kernel otherwise
  if (c->ab_tc && apply_tc_preferred(st ? c->w.kmax : ncols)) {
    if (st && c->w_tc)
      return launch_apply_tc(&c->tmap_ab, &c->tmap_w, a, c->w.kmax, c->block_scratch, st, c->num_sms, s);
    if (!st && apply_tc_supported(c->w.n, ncols) && (reinterpret_cast<uintptr_t>(V) & 15) == 0) {
      EncodeTiledFn enc = get_encode();
      CUtensorMap mv;
      if (enc && make_apply_tc_tmaps(nullptr, &mv, nullptr, 0, V, c->w.n, ncols, enc))
        return launch_apply_tc(&c->tmap_ab, &mv, a, ncols, c->block_scratch, tst ? tst : c->st, c->num_sms, s);
    }
  }
  return launch_apply_block(a, st ? c->w.kmax : ncols, c->block_scratch, c->num_sms, s);
}

// ---------------------------------------------------------------------------
// Solve graph
// ---------------------------------------------------------------------------
static cudaError_t add_conditional(cudaStream_t s, cudaGraphConditionalHandle h, cudaGraphConditionalNodeType type,
                                   cudaGraph_t* body) {
  cudaStreamCaptureStatus cs;
  cudaGraph_t cg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t ndeps = 0;
  cudaError_t e = cudaStreamGetCaptureInfo(s, &cs, nullptr, &cg, &deps, nullptr, &ndeps);
  if (e != cudaSuccess) return e;
  std::vector<cudaGraphNode_t> d(deps, deps + ndeps);
  cudaGraphNodeParams prm = {cudaGraphNodeTypeConditional};
  prm.conditional.handle = h;
  prm.conditional.type = type;
  prm.conditional.size = 1;
  cudaGraphNode_t node;
  e = cudaGraphAddNode(&node, cg, d.data(), nullptr, d.size(), &prm);
  if (e != cudaSuccess) return e;
  *body = prm.conditional.phGraph_out[0];
  return cudaStreamUpdateCaptureDependencies(s, &node, nullptr, 1, cudaStreamSetCaptureDependencies);
}

// The check / refinement branch: r = b - A x (float64 accumulation); if the
// solve is not finished, re-deflate x, r against W and refresh rho, beta, mu.
static cudaError_t capture_check_branch(dcg_ctx* c, cudaStream_t s, int pre_loop) {
  cudaError_t e;
  if ((e = op_resid(c, -1, 1, s)) != cudaSuccess) return e;
  if ((e = launch_check_dots(c->w, c->grid_iter, s)) != cudaSuccess) return e;
  return launch_check_update(c->w, c->grid_iter, pre_loop, 0, c->h, s);
}

static dcg_status build_graph(dcg_ctx* c) {
  destroy_graph(c);
  CK(cudaGraphCreate(&c->graph, 0));
  Handles& h = c->h;
  CK(cudaGraphConditionalHandleCreate(&h.pre, c->graph, 0, cudaGraphCondAssignDefault));
  CK(cudaGraphConditionalHandleCreate(&h.loop, c->graph, 1, cudaGraphCondAssignDefault));
  CK(cudaGraphConditionalHandleCreate(&h.chk, c->graph, 0, cudaGraphCondAssignDefault));
  CK(cudaGraphConditionalHandleCreate(&h.fin, c->graph, 0, cudaGraphCondAssignDefault));
  Ws& w = c->w;
  cudaStream_t s0 = c->cap[0], s1 = c->cap[1], s2 = c->cap[2];
  CK(cudaStreamBeginCaptureToGraph(s0, c->graph, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = cudaSuccess;
  auto run = [&](cudaError_t r) {
    if (e == cudaSuccess) e = r;
  };
  // Start of solve: AW, r_{-1} (warm start), E and its factor, x_0, p_0.
  run(op_block(c, w.XW, 0, w.Y, c->st, s0));
  run(op_resid(c, 0, 1, s0));
  run(launch_setup_r(w, c->grid_iter, s0));
  run(launch_gram_E(w, c->gramE_part, c->num_sms, s0));
  run(launch_gram_GW(w, c->gramE_part, c->num_sms, s0));
  run(launch_chol_E(w, s0));
  run(launch_small_prods(w, s0));
  run(launch_check_dots(w, c->grid_iter, s0));
  run(launch_check_update(w, c->grid_iter, 0, 1, h, s0));
  run(launch_phase2_setup(w, c->grid_iter, s0));
  // IF |r_0| <= tol |b|: confirm with the true residual.
  cudaGraph_t body = nullptr;
  run(add_conditional(s0, h.pre, cudaGraphCondTypeIf, &body));
  if (e == cudaSuccess) {
    run(cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    run(capture_check_branch(c, s1, 1));
    cudaGraph_t tmp;
    run(cudaStreamEndCapture(s1, &tmp));
  }
  run(launch_loop_gate(w, h, s0));
  // WHILE not done: one iteration with its direction store.
  run(add_conditional(s0, h.loop, cudaGraphCondTypeWhile, &body));
  if (e == cudaSuccess) {
    run(cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    run(op_matvec(c, w.p, w.q, &c->st->d, c->mv_partials, &c->st->ticket[T_MATVEC], c->st, s1));
    run(launch_iter_fused(w, c->num_sms, h, s1));
    // IF a convergence check or a replacement is due: the true residual, the
    // replacement and the direction update (which the fused kernel then skipped)
    cudaGraph_t inner = nullptr;
    run(add_conditional(s1, h.chk, cudaGraphCondTypeIf, &inner));
    if (e == cudaSuccess) {
      run(cudaStreamBeginCaptureToGraph(s2, inner, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
      run(capture_check_branch(c, s2, 0));
      run(launch_phase2(w, c->grid_iter, h, s2));
      cudaGraph_t tmp;
      run(cudaStreamEndCapture(s2, &tmp));
    }
    cudaGraph_t tmp;
    run(cudaStreamEndCapture(s1, &tmp));
  }
  // IF the final iterate has no true residual yet (max_iter, breakdown): form it.
  run(launch_final_gate(w, h, s0));
  run(add_conditional(s0, h.fin, cudaGraphCondTypeIf, &body));
  if (e == cudaSuccess) {
    run(cudaStreamBeginCaptureToGraph(s1, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
    run(op_resid(c, 3, 0, s1));
    cudaGraph_t tmp;
    run(cudaStreamEndCapture(s1, &tmp));
  }
  run(launch_finalize(w, c->grid_iter, s0));
  cudaGraph_t g2 = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(s0, &g2);
  if (e != cudaSuccess) return cuda_fail(c, e, "capturing the solve graph");
  if (e2 != cudaSuccess) return cuda_fail(c, e2, "cudaStreamEndCapture");
  CK(cudaGraphInstantiate(&c->exec, c->graph, 0));
  c->graph_valid = true;
  return DCG_OK;
}

// The solve graph's kernels in the same order, launched from the host. Each
// conditional node becomes a host decision on the state the kernels wrote:
// the pre-loop check when |r_0| met tol (mode 1 after setup), the loop while
// not done, the in-loop check branch (true residual, replacement, direction update)
// when the fused iteration kernel chose a check (mode != 0), the final
// residual when the last iterate has none.
static dcg_status run_host_loop(dcg_ctx* c, cudaStream_t s) {
  Handles h0{};  // no graph: the kernels set no conditionals
  Ws& w = c->w;
  DevState* hs = c->h_st;
  auto read_state = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(hs, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    return e != cudaSuccess ? e : cudaStreamSynchronize(s);
  };
  CK(op_block(c, w.XW, 0, w.Y, c->st, s));
  CK(op_resid(c, 0, 1, s));
  CK(launch_setup_r(w, c->grid_iter, s));
  CK(launch_gram_E(w, c->gramE_part, c->num_sms, s));
  CK(launch_gram_GW(w, c->gramE_part, c->num_sms, s));
  CK(launch_chol_E(w, s));
  CK(launch_small_prods(w, s));
  CK(launch_check_dots(w, c->grid_iter, s));
  CK(launch_check_update(w, c->grid_iter, 0, 1, h0, s));
  CK(launch_phase2_setup(w, c->grid_iter, s));
  CK(read_state());
  if (hs->mode == 1) {
    CK(op_resid(c, -1, 1, s));
    CK(launch_check_dots(w, c->grid_iter, s));
    CK(launch_check_update(w, c->grid_iter, 1, 0, h0, s));
    CK(read_state());
  }
  while (!hs->done) {
    CK(op_matvec(c, w.p, w.q, &c->st->d, c->mv_partials, &c->st->ticket[T_MATVEC], c->st, s));
    CK(launch_iter_fused(w, c->num_sms, h0, s));
    CK(read_state());
    if (hs->mode != 0 && !hs->done) {
      CK(op_resid(c, -1, 1, s));
      CK(launch_check_dots(w, c->grid_iter, s));
      CK(launch_check_update(w, c->grid_iter, 0, 0, h0, s));
      CK(launch_phase2(w, c->grid_iter, h0, s));
      CK(read_state());
    }
  }
  if (!hs->true_valid && !hs->zero_rhs) CK(op_resid(c, 3, 0, s));
  CK(launch_finalize(w, c->grid_iter, s));
  return DCG_OK;
}

// Which bounded device-side wait gave up (DevState::timeout_site).
static const char* timeout_site_name(int site) {
  switch (site) {
    case 1: return "site 1, TMA tile wait of the stored-operator matvec";
    case 2: return "site 2, TMA tile wait of the stored-operator true residual";
    case 3: return "site 3, pipeline wait of the matrix-free matvec";
    case 4: return "site 4, grid barrier of the fused iteration kernel";
    case 5: return "site 5, staged k x k matrices of the fused iteration kernel";
    case 6: return "site 6, pipeline wait of the tensor-core block product";
    default: return "unknown site";
  }
}

// The solver state at the start of a solve. store: the solve keeps its
// directions for the next extraction and its residual history (dcg_solve);
// the systems of a lockstep multi-right-hand-side solve keep neither.
static void init_state(const dcg_ctx* c, DevState* hs, bool store) {
  memset(hs, 0, sizeof(DevState));
  hs->max_iter = c->cfg.max_iter;
  hs->refine_every = c->cfg.refine_every;
  hs->k = c->k_active;
  hs->ell = store ? c->cfg.ell : 0;
  hs->window = c->cfg.window;
  hs->reproject = c->cfg.reproject;
  hs->hist_on = store ? c->cfg.record_history : 0;
  hs->hist_cap = hs->hist_on ? c->cfg.max_iter + 2 : 0;
  hs->warm_start = c->cfg.warm_start;
  hs->status = DCG_OK;
}

static void fill_info(const DevState* hs, float ms, dcg_solve_info* info) {
  memset(info, 0, sizeof(*info));
  info->status = hs->status;
  info->iters = hs->iter;
  info->matvecs_loop = hs->iter;
  info->matvecs_setup = hs->k + hs->warm_start;
  info->matvecs_check = hs->matvecs_check;
  info->k_used = hs->k;
  info->stored = hs->nstored;
  info->relres_recursive = hs->bnorm2 > 0.0 ? sqrt(hs->rho / hs->bnorm2) : 0.0;
  info->relres_true = hs->relres_true;
  info->ms_total = ms;
}

// ---------------------------------------------------------------------------
// Solve
// ---------------------------------------------------------------------------
extern "C" dcg_status dcg_solve(dcg_ctx* c, const float* b, double* x, dcg_solve_info* info) {
  if (!c) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  if (!b || !x) return fail(c, DCG_ERR_INVALID_ARG, "b and x must not be NULL");
  if (c->op == OP_NONE) return fail(c, DCG_ERR_STATE, "no operator set");
  if (!c->cfg.host_loop && !c->graph_valid) {
    dcg_status s = build_graph(c);
    if (s != DCG_OK) return s;
  }
  const int n = c->w.n;
  DevState* hs = c->h_st;
  init_state(c, hs, true);
  if (c->test_barrier_polls > 0) {  // one-shot failure-handling test hook
    hs->test_skip_arrival = 1;
    hs->spin_limit = c->test_barrier_polls;
    c->test_barrier_polls = 0;
  }
  cudaStream_t s = c->stream;
  CK(cudaMemcpyAsync(c->st, hs, sizeof(DevState), cudaMemcpyHostToDevice, s));
  CK(cudaMemcpyAsync(c->w.b, b, size_t(n) * 4, cudaMemcpyDeviceToDevice, s));
  if (c->cfg.warm_start)
    CK(cudaMemcpyAsync(c->w.xd, x, size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
  else
    CK(cudaMemsetAsync(c->w.xd, 0, size_t(n) * 8, s));
  CK(cudaEventRecord(c->ev0, s));
  if (c->cfg.host_loop) {
    dcg_status hst = run_host_loop(c, s);
    if (hst != DCG_OK) return hst;
  } else {
    CK(cudaGraphLaunch(c->exec, s));
  }
  CK(cudaEventRecord(c->ev1, s));
  CK(cudaMemcpyAsync(x, c->w.xd, size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
  CK(cudaMemcpyAsync(hs, c->st, sizeof(DevState), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  c->have_solve = (hs->status == DCG_OK || hs->status == DCG_ERR_MAXITER);
  c->last_iters = hs->iter;
  if (info) fill_info(hs, ms, info);
  if (hs->status != DCG_OK) {
    char buf[256];
    std::string where;
    if (hs->status == DCG_ERR_TIMEOUT) where = std::string(" (bounded wait gave up: ") + timeout_site_name(hs->timeout_site) + ")";
    snprintf(buf, sizeof(buf), "solve ended with status %d (%s) after %d iterations%s", hs->status,
             dcg_status_string(dcg_status(hs->status)), hs->iter, where.c_str());
    c->err = buf;
  }
  return dcg_status(hs->status);
}

// ---------------------------------------------------------------------------
// Lockstep solves of several right-hand sides (dcg_solve_multi)
// ---------------------------------------------------------------------------
template <typename T>
static cudaError_t mr_alloc(dcg_ctx* c, T** p, size_t count) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, count * sizeof(T) + 16);
  if (e != cudaSuccess) return e;
  c->mr_allocs.push_back(v);
  *p = static_cast<T*>(v);
  return cudaMemsetAsync(v, 0, count * sizeof(T) + 16, c->stream);
}

// Per-system buffers for cap systems (replacing smaller ones).
static dcg_status mr_reserve(dcg_ctx* c, int cap) {
  if (cap <= c->mr_cap) return DCG_OK;
  CK(cudaStreamSynchronize(c->stream));
  for (void* p : c->mr_allocs) cudaFree(p);
  c->mr_allocs.clear();
  if (c->mr_hst) cudaFreeHost(c->mr_hst);
  c->mr_hst = nullptr;
  c->mr_cap = 0;
  const size_t n = size_t(c->w.n), np = size_t(c->n_pad), vs = (n + 63) / 64 * 64;
  const size_t kk = size_t(std::max(c->w.kmax, 1)), ncap = size_t(cap), cap8 = (ncap + 7) / 8 * 8;
  CK(mr_alloc(c, &c->mr_p, ncap * np));
  CK(mr_alloc(c, &c->mr_xh, ncap * vs));
  CK(mr_alloc(c, &c->mr_xl, ncap * vs));
  CK(mr_alloc(c, &c->mr_r, ncap * vs));
  CK(mr_alloc(c, &c->mr_b, ncap * vs));
  CK(mr_alloc(c, &c->mr_xd, ncap * vs));
  CK(mr_alloc(c, &c->mr_xbest, ncap * vs));
  CK(mr_alloc(c, &c->mr_small, ncap * 4 * kk));
  CK(mr_alloc(c, &c->mr_small_f, ncap * 2 * kk));
  CK(mr_alloc(c, &c->mr_P, cap8 * np));
  CK(mr_alloc(c, &c->mr_Q, cap8 * np));
  CK(mr_alloc(c, &c->mr_resid_part, size_t(EX_NL) * 3 * size_t(rbf_resid_splits(c->w.n, c->num_sms)) * n));
  CK(mr_alloc(c, &c->mr_phl, rbf_p16_halfs(c->n_pad)));
  CK(mr_alloc(c, &c->mr_pscale, size_t(DCG_MAX_RHS)));
  CK(mr_alloc(c, &c->mr_st, ncap + 1));
  CK(cudaMallocHost(&c->mr_hst, sizeof(DevState) * (ncap + 1)));
  {
    EncodeTiledFn enc = get_encode();
    c->mr_tc = enc && make_rbf_p16_tmap(&c->mr_pmaps[0], c->mr_phl, c->n_pad, 16, enc) &&
               make_rbf_p16_tmap(&c->mr_pmaps[1], c->mr_phl, c->n_pad, 32, enc);
  }
  c->mr_vs = vs;
  c->mr_cap = cap;
  return DCG_OK;
}

// The workspace of system j: its own vectors and state; W, AW, E and the
// small matrices of the context; no direction store, no history.
static Ws mr_lane_ws(const dcg_ctx* c, int j) {
  Ws w = c->w;
  const size_t vs = c->mr_vs, kk = size_t(std::max(c->w.kmax, 1));
  w.xd = c->mr_xd + j * vs;
  w.xbest = c->mr_xbest + j * vs;
  w.xh = c->mr_xh + j * vs;
  w.xl = c->mr_xl + j * vs;
  w.r = c->mr_r + j * vs;
  w.b = c->mr_b + j * vs;
  w.p = c->mr_p + j * size_t(c->n_pad);
  w.q = c->mr_Q + j * size_t(c->n_pad);  // set to the system's column of the block in each iteration
  w.P = nullptr;
  w.Q = nullptr;
  w.ellmax = 0;
  w.fg = nullptr;
  w.h = c->mr_small + j * 4 * kk;
  w.hp = w.h + kk;
  w.mu = w.h + 2 * kk;
  w.gamma = w.h + 3 * kk;
  w.mu_f = c->mr_small_f + j * 2 * kk;
  w.gamma_f = w.mu_f + kk;
  w.st = c->mr_st + j;
  return w;
}

// r = b - A x for the systems js of a lockstep solve (mode, skip_if_done as
// in op_resid). The matrix-free operator forms each exact-form entry once per
// EX_NL systems (k_rbf_resid_multi), then finishes each system on its own;
// the stored operator takes one compensated residual per system.
static cudaError_t op_resid_lanes(dcg_ctx* c, const std::vector<Ws>& w, const std::vector<int>& js, int mode,
                                  int skip_if_done, cudaStream_t s) {
  cudaError_t e = cudaSuccess;
  if (c->op != OP_RBF || js.size() == 1) {
    for (int j : js)
      if ((e = op_resid_w(c, w[j], mode, skip_if_done, s)) != cudaSuccess) return e;
    return e;
  }
  const int n = c->w.n, splits = c->resid_splits;
  for (int j : js)
    if ((e = launch_split_x(w[j], c->grid_iter, skip_if_done, s)) != cudaSuccess) return e;
  for (size_t g0 = 0; g0 < js.size(); g0 += EX_NL) {
    RbfResidMultiArgs m{};
    m.base = rbf_resid_args(c);
    m.nl = int(std::min(js.size() - g0, size_t(EX_NL)));
    for (int l = 0; l < m.nl; ++l) {
      const Ws& wj = w[js[g0 + l]];
      m.xh[l] = wj.xh;
      m.xl[l] = wj.xl;
      m.part[l] = c->mr_resid_part + size_t(l) * 3 * splits * n;
    }
    if ((e = launch_rbf_resid_multi(m, splits, s)) != cudaSuccess) return e;
    for (int l = 0; l < m.nl; ++l) {
      const Ws& wj = w[js[g0 + l]];
      RbfExactArgs a = rbf_resid_args(c);
      a.partials_f = m.part[l];
      a.xh = wj.xh;
      a.xl = wj.xl;
      a.b = wj.b;
      a.r = wj.r;
      a.ticket = &wj.st->ticket[T_CHECK_RES];
      a.st = wj.st;
      a.skip_if_done = skip_if_done;
      a.resid_mode = mode;
      if ((e = launch_rbf_resid_fin(a, splits, s)) != cudaSuccess) return e;
    }
  }
  return e;
}

// Q[:, j] = A P[:, j] for the na gathered directions (leading dimension ld):
// the operator pass the systems of a lockstep solve share. The matrix-free
// operator forms the loop's tensor-core entries once for all na <= 32
// columns and contracts them on the tensor cores (k_rbf_mv_tc; k_rbf_mv<8>
// passes if its float16 maps could not be made); a bounded wait that gives
// up records a timeout in the shared state (the last of mr_st).
static cudaError_t op_multi(dcg_ctx* c, int na, int64_t ld, cudaStream_t s) {
  DevState* tst = c->mr_st + c->mr_cap;
  if (c->op == OP_RBF && c->mr_tc) {
    // one pass for all na <= 32 columns, the contraction on the tensor cores
    RbfMvArgs a{};
    a.p = c->mr_P;
    a.ldp = ld;
    a.vcol = c->vcol;
    a.q = c->mr_Q;
    a.ldq = ld;
    a.ncols = na;
    a.n = c->w.n;
    a.n_tiles = c->n_pad / 128;
    a.d = c->rbf_d;
    a.xformat = c->rbf_xformat;
    a.prm = c->prm;
    a.st = tst;
    a.skip_if_done = 0;
    a.col_idx = -1;
    return launch_rbf_mv_tc(c->rbf_tmap, c->mr_pmaps, a, c->mr_phl, c->mr_pscale, c->rbf_grid, s);
  }
  if (c->op == OP_RBF) {
    const int nc = rbf_block_nc();
    for (int j0 = 0; j0 < na; j0 += nc) {
      RbfMvArgs a{};
      a.p = c->mr_P + j0 * ld;
      a.ldp = ld;
      a.vcol = c->vcol;
      a.q = c->mr_Q + j0 * ld;
      a.ldq = ld;
      a.ncols = std::min(nc, na - j0);
      a.n = c->w.n;
      a.n_tiles = c->n_pad / 128;
      a.d = c->rbf_d;
      a.xformat = c->rbf_xformat;
      a.prm = c->prm;
      a.st = tst;  // never done; col_idx < 0: all ncols columns are written
      a.skip_if_done = 0;
      a.col_idx = -1;
      cudaError_t e = launch_rbf_mv_block(c->rbf_tmap, a, c->rbf_grid, s);
      if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
  }
  return op_block(c, c->mr_P, na, c->mr_Q, nullptr, s, tst);
}

extern "C" dcg_status dcg_solve_multi(dcg_ctx* c, int nrhs, const float* B, double* X, dcg_solve_info* infos) {
  if (!c) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  if (!B || !X) return fail(c, DCG_ERR_INVALID_ARG, "B and X must not be NULL");
  if (nrhs < 1 || nrhs > DCG_MAX_RHS)
    return fail(c, DCG_ERR_INVALID_ARG, "nrhs must lie in [1, " + std::to_string(DCG_MAX_RHS) + "]");
  if (c->op == OP_NONE) return fail(c, DCG_ERR_STATE, "no operator set");
  { const dcg_status r = mr_reserve(c, nrhs); if (r != DCG_OK) return r; }
  // AW and E are recomputed below: the directions of the last dcg_solve no
  // longer belong to the context's AW
  c->have_solve = false;
  const int n = c->w.n;
  const int64_t ld = c->op == OP_RBF ? c->n_pad : n;  // the stored block product takes leading dimension n
  const int rows = c->op == OP_RBF ? c->n_pad : n;
  const int sh = c->mr_cap;  // index of the shared state
  cudaStream_t s = c->stream;
  Handles h0{};
  DevState* hs = c->mr_hst;
  for (int j = 0; j < nrhs; ++j) init_state(c, hs + j, false);
  memset(hs + sh, 0, sizeof(DevState));
  hs[sh].status = DCG_OK;
  CK(cudaMemcpyAsync(c->mr_st, hs, sizeof(DevState) * size_t(sh + 1), cudaMemcpyHostToDevice, s));
  std::vector<Ws> w(nrhs);
  for (int j = 0; j < nrhs; ++j) {
    w[j] = mr_lane_ws(c, j);
    CK(cudaMemcpyAsync(w[j].b, B + int64_t(j) * n, size_t(n) * 4, cudaMemcpyDeviceToDevice, s));
    if (c->cfg.warm_start)
      CK(cudaMemcpyAsync(w[j].xd, X + int64_t(j) * n, size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
    else
      CK(cudaMemsetAsync(w[j].xd, 0, size_t(n) * 8, s));
  }
  auto read_states = [&]() -> cudaError_t {
    cudaError_t e = cudaMemcpyAsync(hs, c->mr_st, sizeof(DevState) * size_t(sh + 1), cudaMemcpyDeviceToHost, s);
    return e != cudaSuccess ? e : cudaStreamSynchronize(s);
  };
  CK(cudaEventRecord(c->ev0, s));
  // Start of the solves: AW, E = W^T AW, its factor and the small products,
  // once for all systems (through system 0's state, before any system can be
  // done); a singular E ends every system.
  CK(op_block(c, c->w.XW, 0, c->w.Y, w[0].st, s));
  CK(launch_gram_E(w[0], c->gramE_part, c->num_sms, s));
  CK(launch_gram_GW(w[0], c->gramE_part, c->num_sms, s));
  CK(launch_chol_E(w[0], s));
  CK(launch_small_prods(w[0], s));
  CK(read_states());
  int shared_status = hs[0].status;
  std::vector<char> hit(nrhs, shared_status != DCG_OK ? 1 : 0);  // systems a shared failure ended
  if (shared_status == DCG_OK) {
    // per system: r_{-1}, the initial projection and the first direction
    std::vector<int> js;
    if (c->cfg.warm_start) {
      for (int j = 0; j < nrhs; ++j) js.push_back(j);
      CK(op_resid_lanes(c, w, js, 0, 1, s));
    }
    for (int j = 0; j < nrhs; ++j) {
      CK(launch_setup_r(w[j], c->grid_iter, s));
      CK(launch_check_dots(w[j], c->grid_iter, s));
      CK(launch_check_update(w[j], c->grid_iter, 0, 1, h0, s));
      CK(launch_phase2_setup(w[j], c->grid_iter, s));
    }
    CK(read_states());
    js.clear();
    for (int j = 0; j < nrhs; ++j)
      if (hs[j].mode == 1) js.push_back(j);
    if (!js.empty()) {
      CK(op_resid_lanes(c, w, js, -1, 1, s));
      for (int j : js) {
        CK(launch_check_dots(w[j], c->grid_iter, s));
        CK(launch_check_update(w[j], c->grid_iter, 1, 0, h0, s));
      }
      CK(read_states());
    }
    MultiLanes lanes{};
    for (;;) {
      if (hs[sh].status != DCG_OK) {  // a wait of the shared block product gave up
        shared_status = hs[sh].status;
        for (int j = 0; j < nrhs; ++j) hit[j] = !hs[j].done;
        break;
      }
      int na = 0;
      for (int j = 0; j < nrhs; ++j)
        if (!hs[j].done) lanes.idx[na++] = j;
      if (na == 0) break;
      CK(launch_multi_gather(c->mr_p, c->n_pad, lanes, na, rows, c->mr_P, ld, s));
      CK(op_multi(c, na, ld, s));
      CK(launch_multi_pq(c->mr_P, c->mr_Q, ld, n, lanes, na, c->mr_st, s));
      for (int a = 0; a < na; ++a) {
        Ws& wj = w[lanes.idx[a]];
        wj.q = c->mr_Q + int64_t(a) * ld;
        CK(launch_iter_fused(wj, c->num_sms, h0, s));
      }
      CK(read_states());
      // the systems whose check or replacement is due: their true residuals
      // in shared passes, then each one's check branch
      js.clear();
      for (int a = 0; a < na; ++a) {
        const int j = lanes.idx[a];
        if (hs[j].mode != 0 && !hs[j].done) js.push_back(j);
      }
      if (!js.empty()) {
        CK(op_resid_lanes(c, w, js, -1, 1, s));
        for (int j : js) {
          CK(launch_check_dots(w[j], c->grid_iter, s));
          CK(launch_check_update(w[j], c->grid_iter, 0, 0, h0, s));
          CK(launch_phase2(w[j], c->grid_iter, h0, s));
        }
        CK(read_states());
      }
    }
    js.clear();
    for (int j = 0; j < nrhs; ++j)
      if (shared_status == DCG_OK && !hs[j].true_valid && !hs[j].zero_rhs) js.push_back(j);
    if (!js.empty()) CK(op_resid_lanes(c, w, js, 3, 0, s));
    for (int j = 0; j < nrhs; ++j) CK(launch_finalize(w[j], c->grid_iter, s));
  }
  CK(cudaEventRecord(c->ev1, s));
  for (int j = 0; j < nrhs; ++j)
    CK(cudaMemcpyAsync(X + int64_t(j) * n, w[j].xd, size_t(n) * 8, cudaMemcpyDeviceToDevice, s));
  CK(read_states());
  float ms = 0.f;
  cudaEventElapsedTime(&ms, c->ev0, c->ev1);
  dcg_status first = DCG_OK;
  int first_j = -1;
  for (int j = 0; j < nrhs; ++j) {
    // a failure of the shared steps (E singular, a wait of the block product)
    // is the status of every system it ended
    if (hit[j]) hs[j].status = shared_status;
    if (infos) fill_info(hs + j, ms, infos + j);
    if (first == DCG_OK && hs[j].status != DCG_OK) {
      first = dcg_status(hs[j].status);
      first_j = j;
    }
  }
  if (first != DCG_OK) {
    char buf[256];
    const DevState& f = hs[first_j];
    std::string where;
    const int site = f.timeout_site ? f.timeout_site : hs[sh].timeout_site;
    if (f.status == DCG_ERR_TIMEOUT) where = std::string(" (bounded wait gave up: ") + timeout_site_name(site) + ")";
    snprintf(buf, sizeof(buf), "system %d of %d ended with status %d (%s) after %d iterations%s", first_j, nrhs,
             f.status, dcg_status_string(first), f.iter, where.c_str());
    c->err = buf;
  }
  return first;
}

// Enqueues the harmonic-Ritz update on the context's stream (no host wait).
static dcg_status enqueue_update(dcg_ctx* c) {
  const int kk = c->k_active, ns = c->h_st->nstored;
  RitzArgs a{};
  a.n = c->w.n;
  a.k_act = kk;
  a.nstored = ns;
  a.k_want = c->cfg.k;
  a.select = c->cfg.select;
  a.extraction = c->cfg.extraction;
  a.fg_form = c->cfg.fg_form;
  if (a.fg_form == DCG_FG_SPARSE) {
    // The sparse forms need what their identities assume. A replacement
    // inside the window (reading R13) breaks the coupling of the directions
    // around it. A solve without W is plain CG, whose float32 directions lose
    // orthogonality as soon as a Ritz value converges: the tridiagonal model
    // then carries ghost copies of that value (measured: four kept values
    // equal to 5 digits, the Gram products giving four distinct ones) and
    // the next W would be singular. Either way this extraction takes the
    // Gram products.
    const DevState* hs = c->h_st;
    const bool broken = kk == 0 || (c->cfg.window == DCG_WINDOW_FIRST ? (hs->repl_first > 0 && hs->repl_first < ns)
                                                                      : (hs->repl_last > hs->iter - ns));
    if (broken) a.fg_form = DCG_FG_EXPLICIT;
    c->fg_sparse_used = !broken;
  } else {
    c->fg_sparse_used = false;
  }
  a.fg = c->w.fg;
  a.ellmax = c->w.ellmax;
  a.kmax = c->w.kmax;
  a.E = c->w.E;
  a.GW = c->w.GW;
  a.W = c->w.XW + c->w.n;
  a.AW = c->w.Y + c->w.n;
  a.P = c->w.P;
  a.Q = c->w.Q;
  a.F = c->F;
  a.G = c->G;
  a.part = c->ritz_part;
  a.Vj = c->Vj;
  a.Vd = c->Vd;
  a.Vd2 = c->Vd2;
  a.theta = c->theta;
  a.U = c->U;
  a.Wout = c->Wout;
  a.k_out = c->k_out;
  a.status = c->ritz_status;
  a.colscale = c->colscale;
  cudaStream_t s = c->stream;
  CK(launch_ritz(a, c->num_sms, c->w.XW + c->w.n, s));
  c->m_pencil = kk + ns;
  CK(cudaMemcpyAsync(c->h_small, c->k_out, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  CK(cudaMemcpyAsync(c->h_small + 2, c->ritz_status, sizeof(int), cudaMemcpyDeviceToHost, s));
  c->have_solve = false;
  c->ritz_pending = true;
  return DCG_OK;
}

// Waits for an enqueued update and applies its result (new k, Ritz count);
// returns the update's status.
static dcg_status finish_update(dcg_ctx* c) {
  if (!c->ritz_pending) return DCG_OK;
  c->ritz_pending = false;
  CK(cudaStreamSynchronize(c->stream));
  if (c->h_small[2] != DCG_OK) {
    c->m_last = 0;
    return fail(c, dcg_status(c->h_small[2]), "Ritz extraction: F not positive definite");
  }
  c->k_active = c->h_small[0];
  c->m_last = c->h_small[1];
  return DCG_OK;
}

// Common checks of both update calls; *skip is set when there is nothing to
// extract (k = 0 or no columns in Z).
static dcg_status begin_update(dcg_ctx* c, bool* skip) {
  *skip = false;
  dcg_status st = finish_update(c);
  if (st != DCG_OK) return st;
  if (!c->have_solve) return fail(c, DCG_ERR_STATE, "no completed solve since the last update");
  const int m = c->k_active + c->h_st->nstored;
  if (c->cfg.k == 0 || m == 0) {
    c->have_solve = false;
    c->m_last = 0;
    *skip = true;
  }
  return DCG_OK;
}

extern "C" dcg_status dcg_update_subspace(dcg_ctx* c, int32_t* k_new) {
  if (!c) return DCG_ERR_INVALID_ARG;
  bool skip = false;
  dcg_status st = begin_update(c, &skip);
  if (st != DCG_OK) return st;
  if (!skip) {
    if ((st = enqueue_update(c)) != DCG_OK) return st;
    if ((st = finish_update(c)) != DCG_OK) return st;
  }
  if (k_new) *k_new = c->k_active;
  return DCG_OK;
}

extern "C" dcg_status dcg_update_subspace_async(dcg_ctx* c) {
  if (!c) return DCG_ERR_INVALID_ARG;
  bool skip = false;
  dcg_status st = begin_update(c, &skip);
  if (st != DCG_OK || skip) return st;
  return enqueue_update(c);
}

extern "C" dcg_status dcg_get_ritz_values(dcg_ctx* c, double* theta, int32_t cap, int32_t* m) {
  if (!c) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  if (m) *m = c->m_last;
  if (!theta || cap <= 0 || c->m_last == 0) return DCG_OK;
  const int cnt = std::min(cap, c->m_last);
  CK(cudaMemcpyAsync(theta, c->theta, size_t(cnt) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DCG_OK;
}

extern "C" dcg_status dcg_get_pencil(dcg_ctx* c, double* F, double* G, int32_t cap, int32_t* m) {
  if (!c) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  const int mp = c->m_last > 0 ? c->m_pencil : 0;
  if (m) *m = mp;
  if (mp == 0 || !F || !G) return DCG_OK;
  if (cap < mp * mp) return fail(c, DCG_ERR_INVALID_ARG, "cap is below m * m");
  CK(cudaMemcpyAsync(F, c->F, size_t(mp) * mp * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(G, c->G, size_t(mp) * mp * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return DCG_OK;
}

extern "C" dcg_status dcg_get_pencil_form(dcg_ctx* c, int32_t* form) {
  if (!c || !form) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  *form = (c->m_last > 0 && c->fg_sparse_used) ? DCG_FG_SPARSE : DCG_FG_EXPLICIT;
  return DCG_OK;
}

extern "C" dcg_status dcg_set_subspace(dcg_ctx* c, const float* W, int32_t k) {
  if (!c) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  if (k < 0 || k > c->cfg.k) return fail(c, DCG_ERR_INVALID_ARG, "k must be in [0, cfg.k]");
  if (k > 0 && !W) return fail(c, DCG_ERR_INVALID_ARG, "W is NULL");
  if (k > 0)
    CK(cudaMemcpyAsync(c->w.XW + c->w.n, W, size_t(c->w.n) * k * 4, cudaMemcpyDeviceToDevice, c->stream));
  c->k_active = k;
  c->have_solve = false;
  return DCG_OK;
}

extern "C" dcg_status dcg_get_subspace(dcg_ctx* c, float* W, int32_t* k) {
  if (!c) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  if (k) *k = c->k_active;
  if (W && c->k_active > 0) {
    CK(cudaMemcpyAsync(W, c->w.XW + c->w.n, size_t(c->w.n) * c->k_active * 4, cudaMemcpyDeviceToDevice,
                       c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return DCG_OK;
}

extern "C" dcg_status dcg_get_history(dcg_ctx* c, double* relres, int32_t cap, int32_t* count) {
  if (!c) return DCG_ERR_INVALID_ARG;
  if (!c->cfg.record_history) return fail(c, DCG_ERR_STATE, "record_history is off");
  const int cnt = std::min(cap, c->last_iters + 1);
  if (count) *count = c->last_iters + 1;
  if (relres && cnt > 0) {
    CK(cudaMemcpyAsync(relres, c->w.hist, size_t(cnt) * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return DCG_OK;
}

extern "C" dcg_status dcg_matvec(dcg_ctx* c, const float* p, float* q, double* pAp) {
  if (!c) return DCG_ERR_INVALID_ARG;
  if (c->op == OP_NONE) return fail(c, DCG_ERR_STATE, "no operator set");
  if (!p || !q || (reinterpret_cast<uintptr_t>(p) & 15)) return fail(c, DCG_ERR_INVALID_ARG, "p, q: 16-byte aligned device vectors");
  const float* pin = p;
  if (c->op == OP_RBF) {  // the tile kernel reads whole 128-row tiles of p
    CK(cudaMemcpyAsync(c->pmv, p, size_t(c->w.n) * 4, cudaMemcpyDeviceToDevice, c->stream));
    pin = c->pmv;
  }
  CK(op_matvec(c, pin, q, c->mv_result, c->mv_partials, c->mv_ticket, nullptr, c->stream));
  if (pAp) {
    CK(cudaMemcpyAsync(pAp, c->mv_result, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return DCG_OK;
}

extern "C" dcg_status dcg_residual(dcg_ctx* c, const float* b, const double* x, float* r, double* rnorm2,
                                   double* err) {
  if (!c) return DCG_ERR_INVALID_ARG;
  if (c->op == OP_NONE) return fail(c, DCG_ERR_STATE, "no operator set");
  if (!b || !x || !r) return fail(c, DCG_ERR_INVALID_ARG, "b, x and r are required");
  cudaStream_t s = c->stream;
  // x goes through the solver's iterate buffer and its float32 split
  CK(cudaMemcpyAsync(c->w.xd, x, size_t(c->w.n) * 8, cudaMemcpyDeviceToDevice, s));
  CK(launch_split_x(c->w, c->grid_iter, 0, s));
  CK(cudaMemsetAsync(c->mv_result, 0, 2 * sizeof(double), s));
  if (c->op == OP_RBF) {
    RbfExactArgs a = rbf_resid_args(c);
    a.xh = c->w.xh;
    a.xl = c->w.xl;
    a.b = b;
    a.r = r;
    a.ticket = c->mv_ticket;
    a.result = c->mv_result;
    a.result_err = c->mv_result + 1;
    CK(launch_rbf_resid(a, c->resid_splits, s));
  } else {
    RowOpArgs a{};
    a.xh = c->w.xh;
    a.xl = c->w.xl;
    a.out = r;
    a.b = b;
    a.n = c->w.n;
    a.partials = c->mv_partials;
    a.ticket = c->mv_ticket;
    a.result = c->mv_result;
    CK(launch_rowop(&c->tmap, a, true, c->grid_rows, s));
  }
  double h[2] = {0.0, 0.0};
  CK(cudaMemcpyAsync(h, c->mv_result, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  CK(cudaStreamSynchronize(s));
  if (rnorm2) *rnorm2 = h[0];
  if (err) *err = h[1];
  return DCG_OK;
}

extern "C" dcg_status dcg_apply_block(dcg_ctx* c, const float* V, int32_t ncols, float* Y) {
  if (!c) return DCG_ERR_INVALID_ARG;
  if (c->op == OP_NONE) return fail(c, DCG_ERR_STATE, "no operator set");
  if (!V || !Y || ncols < 1 || ncols > kMaxBlockCols) return fail(c, DCG_ERR_INVALID_ARG, "bad block arguments");
  CK(op_block(c, V, ncols, Y, nullptr, c->stream));
  return DCG_OK;
}

extern "C" dcg_status dcg_debug_arm_barrier_timeout(dcg_ctx* c, int32_t polls) {
  if (!c) return DCG_ERR_INVALID_ARG;
  if (polls < 1 || polls > (1 << 22)) return fail(c, DCG_ERR_INVALID_ARG, "polls must lie in [1, 2^22]");
  if (c->op == OP_NONE) return fail(c, DCG_ERR_STATE, "no operator set");
  c->test_barrier_polls = polls;
  return DCG_OK;
}

extern "C" dcg_status dcg_measure_ex2_rate(void* stream, double* per_second, double* per_clock_per_sm) {
  dcg_ctx* c = nullptr;  // errors below are reported without a context
  if (!per_second) return fail(nullptr, DCG_ERR_INVALID_ARG, "dcg_measure_ex2_rate: per_second is required");
  int dev = 0, sms = 0, khz = 0;
  CK(cudaGetDevice(&dev));
  CK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  CK(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = 4 * sms, iters = 4096;
  float* out = nullptr;
  CK(cudaMalloc(&out, size_t(blocks) * 512 * sizeof(float)));
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  double count = 0.0;
  float best = 0.f;
  for (int rep = 0; rep < 3 && e == cudaSuccess; ++rep) {  // the first run warms up
    if ((e = cudaEventRecord(e0, s)) != cudaSuccess) break;
    if ((e = launch_ex2_rate(out, blocks, iters, &count, s)) != cudaSuccess) break;
    if ((e = cudaEventRecord(e1, s)) != cudaSuccess) break;
    if ((e = cudaEventSynchronize(e1)) != cudaSuccess) break;
    float ms = 0.f;
    if ((e = cudaEventElapsedTime(&ms, e0, e1)) != cudaSuccess) break;
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaFree(out);
  CK(e);
  *per_second = count / (double(best) * 1e-3);
  if (per_clock_per_sm) *per_clock_per_sm = *per_second / (double(sms) * double(khz) * 1e3);
  return DCG_OK;
}

// ---------------------------------------------------------------------------
// Newton step of the Laplace approximation (the Sec. 3 experiment)
// ---------------------------------------------------------------------------
static dcg_status lap_check(dcg_ctx* c, const float* K, int64_t ldk) {
  if (!K) return fail(c, DCG_ERR_INVALID_ARG, "K is NULL");
  if (ldk < c->w.n || (ldk % 4) != 0) return fail(c, DCG_ERR_INVALID_ARG, "ldk must be >= n and a multiple of 4");
  if ((reinterpret_cast<uintptr_t>(K) & 15) != 0) return fail(c, DCG_ERR_INVALID_ARG, "K must be 16-byte aligned");
  if (!c->lap_v32) {
    CK(dalloc(c, &c->lap_v32, size_t(c->w.n)));
    CK(dalloc(c, &c->lap_kv, size_t(c->w.n)));
  }
  return DCG_OK;
}

// out = K v (float32 stored K, the row-band TMA GEMV)
static dcg_status lap_gemv(dcg_ctx* c, const float* K, int64_t ldk, const float* v, float* out) {
  EncodeTiledFn enc = get_encode();
  if (!enc) return fail(c, DCG_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
  CUtensorMap m;
  if (!make_rowop_tmap(&m, K, c->w.n, ldk, enc)) return fail(c, DCG_ERR_INVALID_ARG, "tensor map encode failed");
  RowOpArgs a{};
  a.v = v;
  a.out = out;
  a.n = c->w.n;
  a.partials = c->mv_partials;
  a.ticket = c->mv_ticket;
  a.result = c->mv_result;
  CK(launch_rowop(&m, a, false, c->grid_rows, c->stream));
  return DCG_OK;
}

extern "C" dcg_status dcg_laplace_system(dcg_ctx* c, const float* K, int64_t ldk, const float* y, const double* f,
                                         float* A, int64_t lda, float* b, double* cvec, float* s) {
  if (!c) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  if (!y || !f || !A || !b || !cvec || !s) return fail(c, DCG_ERR_INVALID_ARG, "y, f, A, b, c and s are required");
  if (lda < c->w.n || (lda % 4) != 0) return fail(c, DCG_ERR_INVALID_ARG, "lda must be >= n and a multiple of 4");
  if ((reinterpret_cast<uintptr_t>(A) & 15) != 0) return fail(c, DCG_ERR_INVALID_ARG, "A must be 16-byte aligned");
  dcg_status st = lap_check(c, K, ldk);
  if (st != DCG_OK) return st;
  const int n = c->w.n, grid = lap_grid(n, c->num_sms);
  CK(launch_lap_prep(y, f, n, s, cvec, c->lap_v32, grid, c->stream));
  if ((st = lap_gemv(c, K, ldk, c->lap_v32, c->lap_kv)) != DCG_OK) return st;
  CK(launch_lap_scale(s, c->lap_kv, n, b, grid, c->stream));
  CK(launch_lap_form(K, ldk, s, n, A, lda, c->stream));
  return DCG_OK;
}

extern "C" dcg_status dcg_laplace_update(dcg_ctx* c, const float* K, int64_t ldk, const float* y, const double* cvec,
                                         const float* s, const double* x, double* f, double* a, double* psi) {
  if (!c) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  if (!y || !cvec || !s || !x || !f || !a) return fail(c, DCG_ERR_INVALID_ARG, "y, c, s, x, f and a are required");
  dcg_status st = lap_check(c, K, ldk);
  if (st != DCG_OK) return st;
  const int n = c->w.n, grid = lap_grid(n, c->num_sms);
  CK(launch_lap_a(cvec, s, x, n, a, c->lap_v32, grid, c->stream));
  if ((st = lap_gemv(c, K, ldk, c->lap_v32, c->lap_kv)) != DCG_OK) return st;
  CK(launch_lap_psi(y, c->lap_kv, a, n, f, c->mv_partials, c->mv_ticket, c->mv_result + 1, grid, c->stream));
  if (psi) {
    CK(cudaMemcpyAsync(psi, c->mv_result + 1, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  return DCG_OK;
}

extern "C" dcg_status dcg_sync(dcg_ctx* c) {
  if (!c) return DCG_ERR_INVALID_ARG;
  { const dcg_status pend = finish_update(c); if (pend != DCG_OK) return pend; }
  CK(cudaStreamSynchronize(c->stream));
  return DCG_OK;
}
