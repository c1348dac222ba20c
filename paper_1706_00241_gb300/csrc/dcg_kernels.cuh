// Kernel argument structs and host-side launchers shared between the CUDA
// translation units of the library. Every launcher enqueues on the given
// stream and returns the launch error (no synchronisation).
#pragma once

#include <type_traits>
#include <vector>

#include "dcg_common.cuh"

namespace dcg {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Context workspace as seen by the kernels. Column c of W is XW + (1 + c) n,
// column 0 of XW is the iterate x; Y mirrors it with A x_{-1} and AW.
struct Ws {
  int n;
  int kmax;
  int ellmax;
  float* XW;       // n x (1 + kmax); column 0 unused, W from column 1
  double* xd;      // the iterate x, float64
  double* xbest;   // the iterate with the smallest true residual seen by a check
  float* xh;       // x split for the compensated residual: x = xh + xl
  float* xl;
  float* Y;        // n x (1 + kmax)
  float* r;
  float* p;
  float* q;
  float* b;
  float* P;        // n x ellmax stored directions
  float* Q;        // n x ellmax stored A p
  double* E;       // kmax x kmax, W^T A W
  double* Linv;    // kmax x kmax, inverse Cholesky factor of E (row-major, lower)
  double* GW;      // kmax x kmax, (AW)^T (AW)
  double* Einv;    // kmax x kmax, E^{-1}
  double* N;       // kmax x kmax, G_W E^{-1}
  double* NT;      // its transpose E^{-1} G_W
  double* M;       // kmax x kmax, E^{-1} G_W E^{-1}
  float2* mats2;   // [E^{-1} | M | N^T] as float pairs (hi, lo), k x k each, contiguous
  double* h;       // kmax: (AW)^T r
  double* hp;      // kmax: (AW)^T p
  double* mu;      // kmax
  double* gamma;   // kmax
  float* mu_f;     // kmax
  float* gamma_f;  // kmax
  double* partials;  // grid x kReduceSlots
  double* hist;    // hist_cap
  double* fg;      // fg_doubles(ellmax, kmax): scalars of the stored directions (null if ellmax = 0)
  DevState* st;
  double tol;
};

// Scalars the fused iteration kernel records per stored direction p_j for the
// sparse F, G of Sec. 2.3 (Saad et al.): slot s of the direction ring holds
//   fg[FG_REC s + 0..4] = d_j, alpha_j, |r_j|^2, |r'_{j+1}|^2, j,
// (AW)^T r_j at fg_ha(s) and (AW)^T r'_{j+1} at fg_hb(s), where r_j is the
// residual the iteration starts from and r'_{j+1} = r_j - alpha_j A p_j the
// one it forms (before the float32 re-deflation), so that
// A p_j = (r_j - r'_{j+1}) / alpha_j. After the slots, fg_hprev holds
// (AW)^T r of the residual the next iteration starts from.
constexpr int FG_REC = 5;
__host__ __device__ inline size_t fg_doubles(int ellmax, int kmax) {
  return size_t(ellmax) * (FG_REC + 2 * size_t(kmax)) + size_t(kmax);
}
__host__ __device__ inline double* fg_ha(double* fg, int ellmax, int kmax, int s) {
  return fg + size_t(ellmax) * FG_REC + size_t(s) * kmax;
}
__host__ __device__ inline double* fg_hb(double* fg, int ellmax, int kmax, int s) {
  return fg + size_t(ellmax) * (FG_REC + kmax) + size_t(s) * kmax;
}
__host__ __device__ inline double* fg_hprev(double* fg, int ellmax, int kmax) {
  return fg + size_t(ellmax) * (FG_REC + 2 * size_t(kmax));
}

// Conditional-node handles of the solve graph (see dcg_api.cu).
struct Handles {
  cudaGraphConditionalHandle pre;    // IF: convergence check before the loop
  cudaGraphConditionalHandle loop;   // WHILE: the iteration
  cudaGraphConditionalHandle chk;    // IF inside the loop: check / refinement
  cudaGraphConditionalHandle fin;    // IF after the loop: final true residual
};

struct RowOpArgs {
  const float* v;        // p (matvec)
  const float* xh;       // x (residual), high float32 part
  const float* xl;       // x (residual), low float32 part
  float* out;            // q (matvec) or r (residual)
  const float* b;        // residual only
  int n;
  double* partials;      // >= grid doubles
  unsigned int* ticket;
  double* result;        // matvec: p^T q; residual without state: |r|^2
  DevState* st;          // residual: updates rho_true etc.; may be null
  int skip_if_done;
  int resid_mode;        // 0 warm-start setup, 1 check, 2 refinement, 3 final, -1: read st->mode
  int* abort_word;       // without a state (context-free matvec): set to the wait site
                         // when a bounded wait gives up; the CTA's rows of out and
                         // *result are then NaN. May be null.
};

// Symmetric stored matvec (upper triangle read once): see k_dense.cu.
struct SymvArgs {
  const float* p;
  float* q;
  int n;
  int nbands;          // set by launch_symv
  int nchunks;         // set by launch_symv
  int ns;              // row stride of the partial buffers, set by launch_symv
  float* rowpart;      // symv_rowpart_floats(n)
  float* colpart;      // symv_colpart_floats(n)
  unsigned int* sched_ctr;  // item counter (zero between launches; k_symv_fin rewinds it)
  const int* sched_items;   // the items, largest first (symv_schedule), device
  int nitems;
  double* partials;    // >= symv_fin_grid(n) doubles
  unsigned int* ticket;
  double* result;      // p^T q
  DevState* st;
  int skip_if_done;
};

struct ApplyBlockArgs {
  const float* A;
  int64_t lda;
  const float* V;
  float* Y;
  int n;
  int c;
  DevState* st;          // if set: c = st->k, V and Y point at column 0 (W starts at column 1)
  int skip_if_done;
};

// ---- matrix-free RBF operator (k_rbf.cu)
struct RbfParams {
  float c2;          // 2 log2(e) / (2 l^2)
  float l2s;         // log2(s^2)
  float s2;          // s^2
  float noise;       // diagonal shift
  float neg_inv2l2;  // -1 / (2 l^2), rounded
  float neg_inv2l2_lo;  // its rounding error
  float s2_lo;       // s^2 - float(s^2)
  double noise_d;    // diagonal shift in double (residual recomputation)
  float g_anchor;    // grid of the residual's distance sums (see k_rbf.cu)
  float sigma_anchor;  // 1.5 2^23 g
  float err_dist;    // distance part of the residual entries' error model (units of u^2)
};

struct RbfMvArgs {
  const float* p;      // n_pad floats, zero beyond n
  const float* vcol;   // n_pad floats: -c |x_j|^2, -inf beyond n
  float* q;
  int n;
  int n_tiles;         // n_pad / 128
  int d;
  int xformat;
  const RbfParams* prm;
  double* partials;
  unsigned int* ticket;
  double* result;      // p^T q
  DevState* st;
  int skip_if_done;
  int col_idx;         // >= 0: column of W in a start-of-solve product (skipped if >= st->k)
  int64_t ldp;         // multi-column product: leading dimension of the padded columns in p
  int64_t ldq;         // multi-column product: leading dimension of q
  int ncols;           // multi-column product: columns to write
  float* rowpart;      // symmetric matvec: row sums (n_pad floats)
  float* colpart;      // symmetric matvec: column sums, n_tiles x n_pad floats
  unsigned int* sched_ctr;  // symmetric matvec: row-block counter (zero between launches)
};

struct RbfExactArgs {
  const float* Xr;     // n x d points of the operator
  const float* XrT;    // residual: the points transposed, d x n_pad (zero padded)
  const float* nh;     // residual: |x_i|^2 = nh + nl, nh on the anchor grid (n_pad)
  const float* nl;
  int n;
  int n_pad;
  int d;
  const RbfParams* prm;
  const float* xh;     // residual: x = xh + xl
  const float* xl;
  const float* b;
  float* r;
  const float* V;      // block: n x ncols column-major
  float* Y;
  int ncols;
  float* partials_f;   // residual: 3 x splits x n per-split sums
  double* partials;    // residual: 2 x rows / 128 CTA sums
  unsigned int* ticket;
  double* result;      // residual without a state: |r|^2
  double* result_err;  // residual without a state: the entry-error estimate of |r|
  DevState* st;
  int skip_if_done;
  int resid_mode;
};

// Hyperparameter derivative forms of the matrix-free operator for column pairs
// (u_p, v_p): out[3p] = sum_ij u_pi E_ij D_ij v_pj, out[3p+1] = sum_ij u_pi
// E_ij v_pj, out[3p+2] = sum_i u_pi v_pi, E_ij = exp(-D_ij / (2 l^2)).
struct RbfDthetaArgs {
  const float* Xr;     // n x d rounded points
  int n;
  int d;
  const RbfParams* prm;
  const float* U;      // n x npairs column-major
  const float* V;      // n x npairs column-major
  int npairs;
  double* partials;    // >= 3 * npairs * grid doubles
  unsigned int* ticket;
  double* out;         // 3 * npairs doubles
};
constexpr int kMaxDthetaPairs = 64;
int rbf_dtheta_grid(int n);
cudaError_t launch_rbf_dtheta(const RbfDthetaArgs& a, cudaStream_t s);

cudaError_t launch_rbf_prep(const float* X, int n, int n_pad, int d, int xformat, float* Xr, void* Xt, float* nsq,
                            cudaStream_t s);
cudaError_t launch_rbf_params(const float* nsq, int n, int n_pad, int d, double l, double s2, double noise,
                              float* vcol, RbfParams* prm, cudaStream_t s);
cudaError_t launch_rbf_anchor(const float* Xr, int n, int n_pad, int d, double* n64, unsigned int* maxbits,
                              RbfParams* prm, float* nh, float* nl, float* XrT, cudaStream_t s);
int rbf_resid_splits(int n, int num_sms);
cudaError_t launch_ex2_rate(float* out, int blocks, int iters, double* count, cudaStream_t s);
bool make_rbf_tmap(CUtensorMap* map, const void* Xt, int n_pad, int xformat, int d, EncodeTiledFn encode);  // map[2]
int rbf_max_d(int xformat);
__host__ __device__ int rbf_row_bytes(int xformat, int d);
cudaError_t rbf_mv_configure();
int rbf_mv_grid(int n_tiles, int num_sms);
cudaError_t launch_rbf_mv(const CUtensorMap* tmap, const RbfMvArgs& a, int grid, cudaStream_t s);
// q = A p from the tile pairs (I, J >= I), each formed once (k_rbf_mv_sym + k_rbf_mv_fin)
cudaError_t rbf_mv_sym_configure();
size_t rbf_mv_sym_colpart_floats(int n_pad);
cudaError_t launch_rbf_mv_sym(const CUtensorMap* tmap, const RbfMvArgs& a, int grid, cudaStream_t s);  // tmap[2]
int rbf_exact_grid(int n);
cudaError_t launch_copy_cols(const float* src, float* dst, int n, int64_t ldd, int col0, int nc, const DevState* st,
                             cudaStream_t s);
cudaError_t launch_rbf_mv_block(const CUtensorMap* tmap, const RbfMvArgs& a, int grid, cudaStream_t s);
// Q = A P for up to 32 columns with the contraction on the tensor cores
// (k_rbf_p16 + k_rbf_mv_tc): PHL holds rbf_p16_halfs(n_pad) float16, pmaps[0],
// [1] its maps for 16 and 32 columns (make_rbf_p16_tmap), pscale 32 floats.
cudaError_t rbf_mv_tc_configure();
bool make_rbf_p16_tmap(CUtensorMap* map, const void* PHL, int n_pad, int ncp, EncodeTiledFn encode);
size_t rbf_p16_halfs(int n_pad);
cudaError_t launch_rbf_mv_tc(const CUtensorMap* tmap, const CUtensorMap* pmaps, const RbfMvArgs& a, void* PHL,
                             float* pscale, int grid, cudaStream_t s);
int rbf_block_nc();
cudaError_t launch_rbf_resid(const RbfExactArgs& a, int splits, cudaStream_t s);
// Residual sums of up to EX_NL systems in one pass over the exact-form
// entries (k_rbf_resid_multi): base carries the operator (points, norms,
// parameters); system l reads x = xh[l] + xl[l] and writes its per-split
// partials to part[l] (3 x splits x n floats), which launch_rbf_resid_fin
// (with a.partials_f = part[l] and the system's b, r, state) turns into r.
constexpr int EX_NL = 8;
struct RbfResidMultiArgs {
  RbfExactArgs base;
  int nl;
  const float* xh[EX_NL];
  const float* xl[EX_NL];
  float* part[EX_NL];
};
cudaError_t launch_rbf_resid_multi(const RbfResidMultiArgs& m, int splits, cudaStream_t s);
cudaError_t launch_rbf_resid_fin(const RbfExactArgs& a, int splits, cudaStream_t s);
cudaError_t launch_rbf_block(const RbfExactArgs& a, int cmax, cudaStream_t s);

// ---- dense operator (k_dense.cu)
cudaError_t rowop_configure();
int rowop_grid(int n, int num_sms);
bool make_rowop_tmap(CUtensorMap* map, const float* A, int64_t n, int64_t lda, EncodeTiledFn encode);
cudaError_t launch_rowop(const CUtensorMap* tmap, const RowOpArgs& a, bool resid, int grid, cudaStream_t s);
size_t symv_rowpart_floats(int n);
size_t symv_colpart_floats(int n);
int symv_fin_grid(int n, int num_sms);
cudaError_t symv_configure();
cudaError_t launch_symv(const CUtensorMap* tmap, SymvArgs a, int num_sms, cudaStream_t s);
void symv_schedule(int n, std::vector<int>& items);
// Context-free q = A p on the library's fixed scratch (no allocation).
int noalloc_max_ctas();
cudaError_t noalloc_scratch(void** base);
cudaError_t launch_matvec_noalloc(const CUtensorMap* tmap, const float* p, float* q, int n, double* pAp, int grid,
                                  void* scratch, cudaStream_t s);
cudaError_t launch_apply_block(const ApplyBlockArgs& a, int cmax, float* scratch, int num_sms, cudaStream_t s);
size_t apply_block_scratch_floats(int n, int cmax, int num_sms);
cudaError_t apply_block_configure();
// Y = A V on the tensor cores (split TF32, k_apply_tc): usable when n % 4 == 0,
// n >= 32 and cmax <= 160; V column-major with leading dimension n, 16-byte
// aligned. The maps come from make_apply_tc_tmaps (A: the operator; V: the
// block, cols = cmax columns). tst: where a timeout is recorded when b.st is null.
bool apply_tc_supported(int n, int cmax);
bool apply_tc_preferred(int cmax);
size_t apply_tc_scratch_floats(int n, int cmax, int num_sms);
bool make_apply_tc_tmaps(CUtensorMap* ma, CUtensorMap* mv, const float* A, int64_t lda, const float* V, int n,
                         int cols, EncodeTiledFn encode);
cudaError_t apply_tc_configure();
cudaError_t launch_apply_tc(const CUtensorMap* ma, const CUtensorMap* mv, const ApplyBlockArgs& b, int cmax,
                            float* scratch, DevState* tst, int num_sms, cudaStream_t s);
cudaError_t launch_form_rbf(const float* X, int n, int d, double l, double s2, double noise, float* A, int64_t lda,
                            cudaStream_t s);

// ---- Laplace-approximation Newton step of the Sec. 3 experiment (k_laplace.cu)
int lap_grid(int n, int num_sms);
cudaError_t launch_lap_prep(const float* y, const double* f, int n, float* s, double* c, float* c32, int grid,
                            cudaStream_t st);
cudaError_t launch_lap_scale(const float* s, const float* v, int n, float* out, int grid, cudaStream_t st);
cudaError_t launch_lap_form(const float* K, int64_t ldk, const float* s, int n, float* A, int64_t lda,
                            cudaStream_t st);
cudaError_t launch_lap_a(const double* c, const float* s, const double* x, int n, double* a, float* a32, int grid,
                         cudaStream_t st);
cudaError_t launch_lap_psi(const float* y, const float* f32, const double* a, int n, double* f, double* partials,
                           unsigned int* ticket, double* psi, int grid, cudaStream_t st);

// ---- iteration kernels (k_iter.cu)
cudaError_t launch_setup_r(const Ws& w, int grid, cudaStream_t s);
cudaError_t launch_gram_E(const Ws& w, double* part, int num_sms, cudaStream_t s);
cudaError_t launch_gram_GW(const Ws& w, double* part, int num_sms, cudaStream_t s);
cudaError_t launch_chol_E(const Ws& w, cudaStream_t s);
cudaError_t launch_small_prods(const Ws& w, cudaStream_t s);
cudaError_t launch_check_dots(const Ws& w, int grid, cudaStream_t s);
cudaError_t launch_check_update(const Ws& w, int grid, int pre_loop, int setup, Handles h, cudaStream_t s);
cudaError_t launch_iter_fused(const Ws& w, int grid, Handles h, cudaStream_t s);
int64_t iter_max_n(int num_sms);
cudaError_t iter_configure();
cudaError_t launch_phase2(const Ws& w, int grid, Handles h, cudaStream_t s);
cudaError_t launch_phase2_setup(const Ws& w, int grid, cudaStream_t s);
cudaError_t launch_loop_gate(const Ws& w, Handles h, cudaStream_t s);
cudaError_t launch_final_gate(const Ws& w, Handles h, cudaStream_t s);
cudaError_t launch_finalize(const Ws& w, int grid, cudaStream_t s);
cudaError_t launch_split_x(const Ws& w, int grid, int skip_if_done, cudaStream_t s);

// ---- lockstep multi-right-hand-side solves (k_multi.cu)
// Systems of one block, by column: column j holds system idx[j].
struct MultiLanes {
  int idx[DCG_MAX_RHS];
};
cudaError_t launch_multi_gather(const float* src, int64_t lds, const MultiLanes& lanes, int na, int rows, float* dst,
                                int64_t ldd, cudaStream_t s);
cudaError_t launch_multi_pq(const float* P, const float* Q, int64_t ld, int n, const MultiLanes& lanes, int na,
                            DevState* states, cudaStream_t s);

// ---- harmonic Ritz (k_ritz.cu)
struct RitzArgs {
  int n;
  int k_act;        // columns of W in Z
  int nstored;      // columns of P in Z
  int k_want;
  int select;       // dcg_select
  int extraction;   // dcg_extraction: which pencil F, G hold
  int fg_form;      // dcg_fg_form: Gram products, or the recorded scalars (harmonic only)
  double* fg;       // the scalars (Ws::fg), ring of ellmax slots, kmax-wide h records
  int ellmax, kmax;
  const double* E;  // k_act x k_act, W^T A W of the solve
  const double* GW; // k_act x k_act, (AW)^T AW of the solve
  const float* W;   // n x k_act
  const float* AW;
  const float* P;   // n x nstored
  const float* Q;
  double* F;        // m x m: Z^T AZ (harmonic) or Z^T Z (Ritz)
  double* G;        // m x m: AZ^T AZ (harmonic) or Z^T AZ (Ritz)
  double* part;     // gram partials
  float* Vj;        // m x m eigenvector rows (float32) when they do not fit in shared memory
  double* Vd;       // m x m float64 scratch
  double* Vd2;      // m x m float64 scratch
  double* theta;    // m, descending
  float* U;         // m x k_want (column-major, leading dimension m)
  float* Wout;      // n x k_want
  int* k_out;       // device int: columns produced
  int* status;      // device int: dcg_status of the extraction
  double* colscale; // k_want: 1 / |w_j| with sign
};
size_t gram_partials_doubles(int n, int m, int num_sms);
cudaError_t launch_ritz(const RitzArgs& a, int num_sms, float* dstW, cudaStream_t s);
cudaError_t ritz_configure();
cudaError_t chol_configure(int kmax);

}  // namespace dcg
