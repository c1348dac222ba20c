// Small dense kernels:
//   * Gram products C = A^T B of tall column blocks (E = W^T (AW) for the initial
//     projection of Algorithm 1; F = Z^T (AZ) and G = (AZ)^T (AZ) for Eq. 7, or Z^T Z and
//     Z^T (AZ) for the orthogonal projection), float32
//     products summed in float32 over short row runs and in float64 across them.
//   * Cholesky factor of E and its inverse (float64, one CTA).
//   * Harmonic Ritz extraction (Sec. 2.3, Eq. 7), or the orthogonal
//     projection Z^T A Z u = theta Z^T Z u (the same pencil solver with
//     F = Z^T Z, G = Z^T AZ): diagonal scaling, Cholesky
//     reduction C = L^{-1} G L^{-T}, symmetric eigen-solve of C (Householder
//     tridiagonalisation, bisection, inverse iteration),
//     selection of k values (reading R4), U = S L^{-T} V, W = Z U with unit
//     columns whose largest-magnitude entry is positive (reading R5).
#include <algorithm>

#include "dcg_kernels.cuh"

namespace dcg {

// --------------------------------------------------------------------------
// Gram products
// --------------------------------------------------------------------------
struct GramArgs {
  int n;
  const float* a1; int ka1; const float* a2; int ka2;   // A-side columns
  const float* b1; int kb1; const float* b2; int kb2;   // B-side columns
  double* part;    // splits x ma x mb
  int chunk;       // rows per split
  DevState* st;    // E mode: ka1 = kb1 = st->k
};

constexpr int GR_T = 32;     // output tile edge
constexpr int GR_RUN = 256;  // rows summed in float32 before a float64 flush

__device__ __forceinline__ const float* gram_col(const float* c1, int k1, const float* c2, int j, int n) {
  return j < k1 ? c1 + int64_t(j) * n : c2 + int64_t(j - k1) * n;
}

__global__ void __launch_bounds__(256) k_gram(GramArgs g) {
  __shared__ float As[GR_T][GR_T + 1];
  __shared__ float Bs[GR_T][GR_T + 1];
  int ka1 = g.ka1, ka2 = g.ka2, kb1 = g.kb1, kb2 = g.kb2;
  if (g.st) {
    if (g.st->done) return;
    ka1 = kb1 = g.st->k;
    ka2 = kb2 = 0;
  }
  const int ma = ka1 + ka2, mb = kb1 + kb2;
  const int tb_count = (mb + GR_T - 1) / GR_T;
  const int ta = blockIdx.x / max(tb_count, 1), tb = blockIdx.x % max(tb_count, 1);
  if (ma == 0 || mb == 0 || ta * GR_T >= ma) return;
  const int n = g.n;
  const int r0 = blockIdx.y * g.chunk, r1 = min(n, r0 + g.chunk);
  const int t = threadIdx.x;
  const int oi = t / 8, oj = (t % 8) * 4;  // 32 x 32 outputs, 4 per thread
  double accd[4] = {0.0, 0.0, 0.0, 0.0};
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  int run = 0;
  for (int rb = r0; rb < r1; rb += GR_T) {
    for (int idx = t; idx < GR_T * GR_T; idx += 256) {
      const int c = idx / GR_T, rr = idx % GR_T;
      const int row = rb + rr;
      const int ja = ta * GR_T + c, jb = tb * GR_T + c;
      As[rr][c] = (row < r1 && ja < ma) ? gram_col(g.a1, ka1, g.a2, ja, n)[row] : 0.f;
      Bs[rr][c] = (row < r1 && jb < mb) ? gram_col(g.b1, kb1, g.b2, jb, n)[row] : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < GR_T; ++rr) {
      const float av = As[rr][oi];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fmaf(av, Bs[rr][oj + q], acc[q]);
    }
    __syncthreads();
    run += GR_T;
    if (run >= GR_RUN) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        accd[q] += double(acc[q]);
        acc[q] = 0.f;
      }
      run = 0;
    }
  }
  const int i = ta * GR_T + oi;
  double* out = g.part + int64_t(blockIdx.y) * ma * mb;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int j = tb * GR_T + oj + q;
    if (i < ma && j < mb) out[int64_t(i) * mb + j] = accd[q] + double(acc[q]);
  }
}

// out[i*mb + j] = sum over splits (fixed order: lane l adds splits l, l + 32,
// ..., then a shuffle tree); one warp per output; E mode reads the size from st.
__global__ void k_gram_reduce(const double* part, int splits, int ma, int mb, double* out, const DevState* st) {
  if (st) {
    if (st->done) return;
    ma = mb = st->k;
  }
  const int total = ma * mb;
  const int lane = threadIdx.x & 31;
  const int wstride = (gridDim.x * blockDim.x) >> 5;
  for (int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; idx < total; idx += wstride) {
    double s = 0.0;
    for (int sp = lane; sp < splits; sp += 32) s += part[int64_t(sp) * total + idx];
    s = warp_sum(s);
    if (lane == 0) out[idx] = s;
  }
}

// Row splits of a Gram product: about eight CTAs per SM in total (each split
// then covers a few 32-row blocks), at most 256 splits.
static int gram_splits(int n, int tiles, int num_sms) {
  int splits = (8 * num_sms + tiles - 1) / max(tiles, 1);
  if (splits > 256) splits = 256;
  const int max_splits = (n + GR_T - 1) / GR_T;
  if (splits > max_splits) splits = max_splits;
  return splits < 1 ? 1 : splits;
}

size_t gram_partials_doubles(int n, int m, int num_sms) {
  const int tiles = ((m + GR_T - 1) / GR_T) * ((m + GR_T - 1) / GR_T);
  return size_t(gram_splits(n, tiles, num_sms)) * m * m;
}

static cudaError_t launch_gram(const GramArgs& g0, int ma_max, int mb_max, int num_sms, double* out,
                               const DevState* st, cudaStream_t s) {
  GramArgs g = g0;
  const int tiles = ((ma_max + GR_T - 1) / GR_T) * ((mb_max + GR_T - 1) / GR_T);
  const int splits = gram_splits(g.n, tiles, num_sms);
  int chunk = (g.n + splits - 1) / splits;
  chunk = (chunk + GR_T - 1) / GR_T * GR_T;
  g.chunk = chunk;
  const int used = (g.n + chunk - 1) / chunk;
  k_gram<<<dim3(tiles, used), 256, 0, s>>>(g);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int red_blocks = std::min(1024, (ma_max * mb_max + 7) / 8);  // 8 warps per block, warp per output
  k_gram_reduce<<<std::max(red_blocks, 1), 256, 0, s>>>(g.part, used, ma_max, mb_max, out, st);
  return cudaGetLastError();
}

// E = W^T (AW), k read from the device state (graph launch, per-solve k).
cudaError_t launch_gram_E(const Ws& w, double* part, int num_sms, cudaStream_t s) {
  GramArgs g{};
  g.n = w.n;
  g.a1 = w.XW + w.n;
  g.b1 = w.Y + w.n;
  g.part = part;
  g.st = w.st;
  if (w.kmax == 0) return cudaSuccess;
  return launch_gram(g, w.kmax, w.kmax, num_sms, w.E, w.st, s);
}

// G_W = (AW)^T (AW): used to re-deflate the residual every iteration.
cudaError_t launch_gram_GW(const Ws& w, double* part, int num_sms, cudaStream_t s) {
  GramArgs g{};
  g.n = w.n;
  g.a1 = w.Y + w.n;
  g.b1 = w.Y + w.n;
  g.part = part;
  g.st = w.st;
  if (w.kmax == 0) return cudaSuccess;
  return launch_gram(g, w.kmax, w.kmax, num_sms, w.GW, w.st, s);
}

// --------------------------------------------------------------------------
// Cholesky E = L L^T (symmetrised) and Linv = L^{-1}; float64, one CTA.
// Right-looking: step j subtracts E(i, j) E(l, j) / d_j from the trailing lower
// triangle (j < l <= i) and leaves column j unscaled, so a step needs one
// barrier; column j is scaled by 1 / sqrt(d_j) at the end. 1 / sqrt(d_j) is a
// float estimate refined by two Newton steps y <- y (3 - d y^2) / 2 (relative
// error ~2^-22 -> ~2^-43 -> float64 rounding). Linv row by row, eight lanes per
// entry sharing its dot product.
// --------------------------------------------------------------------------
__device__ __forceinline__ double rsqrt_newton(double d) {
  const float fd = float(d);
  double y = (fd > 1e-30f && fd < 1e30f) ? double(rsqrtf(fd)) : 1.0 / sqrt(d);
  y = y * fma(-0.5 * d * y, y, 1.5);
  y = y * fma(-0.5 * d * y, y, 1.5);
  return y;
}

__global__ void __launch_bounds__(256) k_chol_E(Ws w) {
  DevState* st = w.st;
  if (st->done) return;
  const int k = st->k;
  if (k == 0) return;
  extern __shared__ double shd[];
  double* L = shd;          // k x k
  double* X = shd + k * k;  // k x k, inverse
  __shared__ double rsd[kMaxK];  // 1 / L(j, j)
  __shared__ int s_fail;
  const int t = threadIdx.x;
  if (t == 0) s_fail = 0;
  for (int idx = t; idx < k * k; idx += blockDim.x) {
    const int i = idx / k, j = idx % k;
    L[idx] = 0.5 * (w.E[i * k + j] + w.E[j * k + i]);
    X[idx] = 0.0;
  }
  __syncthreads();
  for (int j = 0; j < k; ++j) {
    const double dj = L[j * k + j];
    const bool bad = !(dj > 0.0) || !isfinite(dj);
    const double y = rsqrt_newton(bad ? 1.0 : dj);
    if (t == 0) {
      rsd[j] = y;
      if (bad) s_fail = 1;
    }
    const double inv_d = y * y;
    const int m = k - j - 1;
    for (int idx = t; idx < m * m; idx += blockDim.x) {
      const int i = j + 1 + idx / m, l = j + 1 + idx % m;
      if (l <= i) L[i * k + l] = fma(-L[i * k + j] * inv_d, L[l * k + j], L[i * k + l]);
    }
    __syncthreads();
  }
  if (s_fail) {
    if (t == 0) {
      st->status = DCG_ERR_SUBSPACE_SINGULAR;
      st->done = 1;
    }
    return;
  }
  for (int idx = t; idx < k * k; idx += blockDim.x) {
    const int i = idx / k, j = idx % k;
    if (j < i) L[idx] *= rsd[j];
    else if (j == i) L[idx] *= rsd[j];  // d_j / sqrt(d_j)
  }
  __syncthreads();
  // X(i, c) = -(1 / L(i, i)) sum_{c <= j < i} L(i, j) X(j, c), X(i, i) = 1 / L(i, i)
  const int grp = t >> 3, sub = t & 7;
  for (int i = 0; i < k; ++i) {
    for (int cb = 0; cb <= i; cb += 32) {  // trip count uniform across the CTA
      const int c = cb + grp;
      double sacc = 0.0;
      if (c < i)
        for (int j = c + sub; j < i; j += 8) sacc = fma(L[i * k + j], X[j * k + c], sacc);
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 4);
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 2);
      sacc += __shfl_xor_sync(0xffffffffu, sacc, 1);
      if (sub == 0 && c <= i) X[i * k + c] = (c == i) ? rsd[i] : -sacc * rsd[i];
    }
    __syncthreads();
  }
  for (int idx = t; idx < k * k; idx += blockDim.x) w.Linv[idx] = X[idx];
}

cudaError_t launch_chol_E(const Ws& w, cudaStream_t s) {
  if (w.kmax == 0) return cudaSuccess;
  const size_t smem = size_t(2) * w.kmax * w.kmax * sizeof(double);
  k_chol_E<<<1, 256, smem, s>>>(w);
  return cudaGetLastError();
}

cudaError_t chol_configure(int kmax) {
  const size_t smem = size_t(2) * kmax * kmax * sizeof(double);
  return cudaFuncSetAttribute(k_chol_E, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
}

// --------------------------------------------------------------------------
// Harmonic Ritz eigen-solve (one CTA of 1024 threads).
// F, G: m x m float64 (row-major) from the Gram kernels. Float32 work arrays
// in the float64 scratch buffers: F' (then the compacted Cholesky factor L)
// and G'. Shared memory holds the pivoted Cholesky rows, then G' reduced in
// place to C = L^{-1} G' L^{-T}, then the Householder vectors of C.
// --------------------------------------------------------------------------
constexpr int EIG_THREADS = 1024;
constexpr int EIG_SMEM_MAX = 200 * 1024;  // dynamic shared memory of the eigen kernel
constexpr int TS_P = 32;                  // panel rows of the blocked triangular solves
constexpr int TS_CWMAX = (kMaxM + 31) / 32;  // 32-column blocks of a panel update, at most

// Forward substitution L X = B in place. L: n x n lower triangular (global,
// leading dimension ldl); B: n x ncols (shared, leading dimension ldb, odd).
// Panels of 32 rows: a panel is first reduced by the rows solved before it
// (one warp per panel row, lanes over columns), then solved by one warp per
// column with lanes over the panel's rows and the panel's diagonal block
// (reciprocal diagonal) in shared memory. Two barriers per panel.
template <int CW>  // live 32-column blocks (ncols <= 32 CW)
__device__ void trsm_lower_panels(const float* L, int ldl, float* B, int ldb, int n, int ncols,
                                  float (*Ld)[TS_P + 1]) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, nw = blockDim.x >> 5;
  for (int i0 = 0; i0 < n; i0 += TS_P) {
    const int pr = min(TS_P, n - i0);
    for (int idx = t; idx < TS_P * TS_P; idx += blockDim.x) {
      const int r = idx / TS_P, q = idx % TS_P;
      float v = 0.f;
      if (r < pr && q <= r) {
        v = L[(i0 + r) * ldl + i0 + q];
        if (q == r) v = 1.f / v;
      }
      Ld[r][q] = v;
    }
    if (i0 > 0) {
      for (int rr = warp; rr < pr; rr += nw) {
        const float* lrow = L + (i0 + rr) * ldl;
        float acc[CW];
#pragma unroll
        for (int q = 0; q < CW; ++q) acc[q] = 0.f;
#pragma unroll 4
        for (int j = 0; j < i0; ++j) {
          const float l = lrow[j];
          const float* bj = B + j * ldb + lane;
#pragma unroll
          for (int q = 0; q < CW; ++q)
            if (lane + 32 * q < ncols) acc[q] = fmaf(l, bj[32 * q], acc[q]);
        }
        float* brow = B + (i0 + rr) * ldb + lane;
#pragma unroll
        for (int q = 0; q < CW; ++q)
          if (lane + 32 * q < ncols) brow[32 * q] -= acc[q];
      }
    }
    __syncthreads();
    for (int c = warp; c < ncols; c += nw) {
      float x = lane < pr ? B[(i0 + lane) * ldb + c] : 0.f;
      for (int jj = 0; jj < pr; ++jj) {
        const float y = __shfl_sync(0xffffffffu, x, jj) * Ld[jj][jj];
        if (lane == jj) x = y;
        else if (lane > jj) x = fmaf(-Ld[lane][jj], y, x);
      }
      if (lane < pr) B[(i0 + lane) * ldb + c] = x;
    }
    __syncthreads();
  }
}

// Back substitution L^T X = B in place (same layouts as trsm_lower_panels),
// panels from the bottom.
template <int CW>  // live 32-column blocks (ncols <= 32 CW)
__device__ void trsm_lower_t_panels(const float* L, int ldl, float* B, int ldb, int n, int ncols,
                                    float (*Ld)[TS_P + 1]) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31, nw = blockDim.x >> 5;
  for (int i1 = n; i1 > 0; i1 -= TS_P) {
    const int i0 = max(0, i1 - TS_P), pr = i1 - i0;
    // Ld[r][q] = L^T(i0 + r, i0 + q) = L(i0 + q, i0 + r), q >= r
    for (int idx = t; idx < TS_P * TS_P; idx += blockDim.x) {
      const int r = idx / TS_P, q = idx % TS_P;
      float v = 0.f;
      if (q < pr && r <= q) {
        v = L[(i0 + q) * ldl + i0 + r];
        if (q == r) v = 1.f / v;
      }
      Ld[r][q] = v;
    }
    if (i1 < n) {
      for (int rr = warp; rr < pr; rr += nw) {
        const int i = i0 + rr;
        float acc[CW];
#pragma unroll
        for (int q = 0; q < CW; ++q) acc[q] = 0.f;
#pragma unroll 4
        for (int j = i1; j < n; ++j) {
          const float l = L[j * ldl + i];
          const float* bj = B + j * ldb + lane;
#pragma unroll
          for (int q = 0; q < CW; ++q)
            if (lane + 32 * q < ncols) acc[q] = fmaf(l, bj[32 * q], acc[q]);
        }
        float* brow = B + i * ldb + lane;
#pragma unroll
        for (int q = 0; q < CW; ++q)
          if (lane + 32 * q < ncols) brow[32 * q] -= acc[q];
      }
    }
    __syncthreads();
    for (int c = warp; c < ncols; c += nw) {
      float x = lane < pr ? B[(i0 + lane) * ldb + c] : 0.f;
      for (int jj = pr - 1; jj >= 0; --jj) {
        const float y = __shfl_sync(0xffffffffu, x, jj) * Ld[jj][jj];
        if (lane == jj) x = y;
        else if (lane < jj) x = fmaf(-Ld[lane][jj], y, x);
      }
      if (lane < pr) B[(i0 + lane) * ldb + c] = x;
    }
    __syncthreads();
  }
}

// Dispatch on the number of live 32-column blocks (CTA-uniform).
__device__ void trsm_lower(const float* L, int ldl, float* B, int ldb, int n, int ncols, float (*Ld)[TS_P + 1]) {
  switch ((ncols + 31) / 32) {
    case 1: trsm_lower_panels<1>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 2: trsm_lower_panels<2>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 3: trsm_lower_panels<3>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 4: trsm_lower_panels<4>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 5: trsm_lower_panels<5>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 6: trsm_lower_panels<6>(L, ldl, B, ldb, n, ncols, Ld); break;
    default: trsm_lower_panels<TS_CWMAX>(L, ldl, B, ldb, n, ncols, Ld); break;
  }
}
__device__ void trsm_lower_t(const float* L, int ldl, float* B, int ldb, int n, int ncols, float (*Ld)[TS_P + 1]) {
  switch ((ncols + 31) / 32) {
    case 1: trsm_lower_t_panels<1>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 2: trsm_lower_t_panels<2>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 3: trsm_lower_t_panels<3>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 4: trsm_lower_t_panels<4>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 5: trsm_lower_t_panels<5>(L, ldl, B, ldb, n, ncols, Ld); break;
    case 6: trsm_lower_t_panels<6>(L, ldl, B, ldb, n, ncols, Ld); break;
    default: trsm_lower_t_panels<TS_CWMAX>(L, ldl, B, ldb, n, ncols, Ld); break;
  }
}

// One Householder step of the tridiagonalisation (column j, rows j+1 ..
// j+Lh of C, Lh <= 32 NQ): every warp forms the reflector of column j itself
// (v_k for k = lane + 32 q in registers), then one warp per row forms
// p = tau A' v; after a barrier every warp forms K = tau/2 p^T v and updates
// its rows of A' -= v w^T + w v^T with w = p - K v. Column j is not read after
// step j; warp 0 stores the scaled v_j into it at the start of step j + 1.
// NQ is the number of live 32-blocks, so no iteration is issued for entries
// beyond the active part (32 warps; the caller dispatches on NQ).
template <int NQ>
__device__ __forceinline__ void tridiag_step(float* C, int ldc, int j, int Lh, float* dT, float* eT, float* tauH,
                                             float* hw, float& scal_prev) {
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  float x[NQ];
  float part = 0.f;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int i = lane + 32 * q;
    x[q] = i < Lh ? C[(j + 1 + i) * ldc + j] : 0.f;
    if (i > 0) part = fmaf(x[q], x[q], part);
  }
  const float sigma = warp_sum(part);
  const float x0 = __shfl_sync(0xffffffffu, x[0], 0);
  float tau = 0.f, scal = 0.f, beta = x0;
  if (sigma != 0.f) {
    const float mu = sqrtf(fmaf(x0, x0, sigma));
    beta = x0 <= 0.f ? mu : -mu;
    tau = (beta - x0) / beta;
    scal = 1.f / (x0 - beta);
  }
  if (t == 0) {
    dT[j] = C[j * ldc + j];
    eT[j] = beta;
    tauH[j] = tau;
  }
  scal_prev = scal;
  float v[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) v[q] = (lane + 32 * q == 0) ? 1.f : x[q] * scal;
  if (tau == 0.f) {   // uniform: every warp computed the same tau
    __syncthreads();  // column j is read by every warp before warp 0 scales it
    return;
  }
  float dd[NQ];
#pragma unroll
  for (int r = 0; r < NQ; ++r) {
    const int i = warp + 32 * r;
    dd[r] = 0.f;
    if (i < Lh) {
      const float* row = C + (j + 1 + i) * ldc + (j + 1);
#pragma unroll
      for (int q = 0; q < NQ; ++q)
        if (lane + 32 * q < Lh) dd[r] = fmaf(row[lane + 32 * q], v[q], dd[r]);
    }
  }
#pragma unroll
  for (int r = 0; r < NQ; ++r)
    if (warp + 32 * r < Lh) {
      const float s_ = warp_sum(dd[r]);
      if (lane == 0) hw[warp + 32 * r] = tau * s_;
    }
  __syncthreads();
  float pv = 0.f, w[NQ];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int k = lane + 32 * q;
    w[q] = k < Lh ? hw[k] : 0.f;
    pv = fmaf(w[q], v[q], pv);
  }
  const float K = 0.5f * tau * warp_sum(pv);
#pragma unroll
  for (int q = 0; q < NQ; ++q) w[q] = fmaf(-K, v[q], w[q]);
#pragma unroll
  for (int r = 0; r < NQ; ++r) {
    const int i = warp + 32 * r;
    if (i < Lh) {
      const float vi = i == 0 ? 1.f : C[(j + 1 + i) * ldc + j] * scal;
      const float wi = fmaf(-K, vi, hw[i]);
      float* crow = C + (j + 1 + i) * ldc + (j + 1);
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int k = lane + 32 * q;
        if (k < Lh) crow[k] = fmaf(-vi, w[q], fmaf(-wi, v[q], crow[k]));
      }
    }
  }
  __syncthreads();
}

// Harmonic Ritz eigen-solve of Eq. 7 (one CTA of 1024 threads).
// The pencil is scaled to unit diagonal F' = S F S (S = diag(F_jj^{-1/2})); in
// that scaling the columns of Z are nearly A-conjugate, so F' is close to the
// identity and the reduction runs in float32: F' = L L^T, C = L^{-1} G' L^{-T},
// symmetric eigen-solve of C, u = S L^{-T} v. (Float64 on this part has a
// ~57x lower throughput and long dependent-chain latency on GB300; the float32
// eigenvectors only set the deflation basis, whose accuracy is that of the
// float32 directions anyway.)
__global__ void __launch_bounds__(EIG_THREADS, 1) k_ritz_eig(RitzArgs a, int m, int k_new) {
  extern __shared__ float C[];  // Cholesky rows; then C (m x ldc); then V^T when it fits
  __shared__ float scale[kMaxM];
  __shared__ int pos[kMaxM], orig[kMaxM];
  __shared__ float th[kMaxM];
  __shared__ float Ld[TS_P][TS_P + 1];
  const int t = threadIdx.x;
  const int warp = t / 32, lane = t % 32, nw = blockDim.x / 32;
  // float32 work arrays in the float64 scratch buffers
  float* Ff = reinterpret_cast<float*>(a.Vd);   // the compacted Cholesky factor L
  float* Gf = reinterpret_cast<float*>(a.Vd2);  // G' (m x m)
  float* Xc = Gf + m * m;                       // inverse-iteration pivots
  // 1. diagonal scaling and symmetrisation (float64 sums rounded to float32
  //    once, the rest in float32): F' (lower triangle) into shared memory as
  //    S (leading dimension lds, odd), G' into global memory
  const int lds = m | 1;
  float* S = C;
  for (int j = t; j < m; j += blockDim.x) {
    const double f = a.F[j * m + j];
    scale[j] = f > 0.0 ? float(1.0 / sqrt(f)) : 0.f;
  }
  __syncthreads();
  for (int i = warp; i < m; i += nw)
    for (int j = lane; j <= i; j += 32) {
      const float sij = scale[i] * scale[j];
      S[i * lds + j] = 0.5f * (float(a.F[i * m + j]) + float(a.F[j * m + i])) * sij;
      const float g = 0.5f * (float(a.G[i * m + j]) + float(a.G[j * m + i])) * sij;
      Gf[i * m + j] = g;
      Gf[j * m + i] = g;
    }
  __syncthreads();
  // 2. Diagonally pivoted Cholesky of F' (rank revealing): step k eliminates
  //    the column with the largest remaining Schur-complement diagonal and
  //    stops when that falls below 1e-4. The dropped columns then lie within
  //    1e-2 (A-norm, relative) of the span of the kept ones (rank-deficient Z,
  //    reading R6), and cond(F') of the kept part stays ~1e4, which the float32
  //    reduction handles; late float32 CG directions do lose A-conjugacy and
  //    can make F' indefinite. Right-looking on the lower triangle of S: step k
  //    with pivot c subtracts S(i, c) S(j, c) / S(c, c) from the remaining
  //    entries and leaves column c as it is, so that afterwards
  //    L(q_a, q_b) = S(orig[q_a], orig[q_b]) / L(q_b, q_b) (pivot order).
  //    Every warp takes the pivot itself (same data, same order), and the
  //    remaining diagonal alternates between two arrays (eliminated columns
  //    hold -inf), so a step needs one barrier.
  __shared__ float dgb[2][kMaxM], lkk[kMaxM];
  for (int j = t; j < m; j += blockDim.x) dgb[0][j] = S[j * lds + j];
  __syncthreads();
  int mk = 0;
  for (int k = 0; k < m; ++k) {
    const float* dgc = dgb[k & 1];
    float* dgn = dgb[(k + 1) & 1];
    float best = -1.f;  // argmax of the remaining diagonal (ties: lower index)
    int bi = m;
    for (int j = lane; j < m; j += 32)
      if (dgc[j] > best) {
        best = dgc[j];
        bi = j;
      }
    for (int o = 16; o > 0; o >>= 1) {
      const float ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ob > best || (ob == best && oi < bi)) {
        best = ob;
        bi = oi;
      }
    }
    if (!(best >= 1e-4f && isfinite(best))) break;
    const int c = bi;
    const float rb = 1.f / best;
    for (int i = warp; i < m; i += nw) {
      const float di = dgc[i];
      if (i == c || di == -INFINITY) {
        if (lane == 0) dgn[i] = -INFINITY;
        continue;
      }
      const float sic = (i > c ? S[i * lds + c] : S[c * lds + i]) * rb;
      float* srow = S + i * lds;
      for (int j = lane; j <= i; j += 32) {
        if (j == c || dgc[j] == -INFINITY) continue;
        const float v = fmaf(-sic, j > c ? S[j * lds + c] : S[c * lds + j], srow[j]);
        srow[j] = v;
        if (j == i) dgn[i] = v;
      }
    }
    if (t == 0) {
      orig[k] = c;
      lkk[k] = sqrtf(best);
    }
    mk = k + 1;
    __syncthreads();
  }
  if (mk == 0) {
    if (t == 0) {
      *a.status = DCG_ERR_SUBSPACE_SINGULAR;
      a.k_out[0] = 0;
      a.k_out[1] = 0;
    }
    return;
  }
  for (int j = t; j < m; j += blockDim.x) pos[j] = -1;
  __syncthreads();
  for (int q = t; q < mk; q += blockDim.x) pos[orig[q]] = q;
  // compact L (mk x mk, lower, pivot order) into Ff
  for (int idx = t; idx < mk * mk; idx += blockDim.x) {
    const int qa = idx / mk, qb = idx % mk;
    float v = 0.f;
    if (qb == qa) {
      v = lkk[qa];
    } else if (qb < qa) {
      const int ia = orig[qa], ib = orig[qb];
      v = (ia > ib ? S[ia * lds + ib] : S[ib * lds + ia]) / lkk[qb];
    }
    Ff[idx] = v;
  }
  const int m_full = m;
  m = mk;  // size of the reduced pencil
  if (k_new > m) k_new = m;
  // C (float32, odd leading dimension ldc so that column sweeps are free of
  // bank conflicts) and V^T (row p holds column p of V) in shared memory when
  // both fit, V^T in global memory otherwise.
  const int ldc = m | 1;
  float* Vt = (2 * m * ldc * int(sizeof(float)) <= EIG_SMEM_MAX) ? C + m * ldc : a.Vj;
  __syncthreads();
  // G' in pivot order into shared memory
  for (int i = warp; i < m; i += nw)
    for (int j = lane; j < m; j += 32) C[i * ldc + j] = Gf[orig[i] * m_full + orig[j]];
  __syncthreads();
  // 3. Y = L^{-1} G'; 4. C = L^{-1} Y^T = L^{-1} G' L^{-T}, symmetrised
  trsm_lower(Ff, m, C, ldc, m, m, Ld);
  for (int i = warp; i < m; i += nw)
    for (int j = i + 1 + lane; j < m; j += 32) {
      const float u = C[i * ldc + j];
      C[i * ldc + j] = C[j * ldc + i];
      C[j * ldc + i] = u;
    }
  __syncthreads();
  trsm_lower(Ff, m, C, ldc, m, m, Ld);
  for (int i = warp; i < m; i += nw)
    for (int j = i + 1 + lane; j < m; j += 32) {
      const float s = 0.5f * (C[i * ldc + j] + C[j * ldc + i]);
      C[i * ldc + j] = s;
      C[j * ldc + i] = s;
    }
  __syncthreads();

  // 5. Symmetric eigen-solve of C in three stages (one CTA):
  //    a. Householder tridiagonalisation C = Q T Q^T, Q = H_0 ... H_{m-3},
  //       H_j = I - tau_j v_j v_j^T with v_j(j+1) = 1; v_j is kept below the
  //       subdiagonal of column j for the back-transformation;
  //    b. all m eigenvalues of T by multisection on Sturm counts (a group of
  //       threads per eigenvalue evaluates the count at evenly spaced points);
  //    c. the selected eigenvectors of T by inverse iteration (thread per
  //       vector), made orthonormal by Gram-Schmidt in selection order
  //       (near-equal values), then z = Q y by applying the reflectors.
  __shared__ float dT[kMaxM], eT[kMaxM], e2[kMaxM], tauH[kMaxM], hw[kMaxM];
  // a. tridiagonalisation, one tridiag_step per column
  static_assert(EIG_THREADS == 1024, "tridiagonalisation assumes 32 warps");
  float scal_prev = 0.f;
  for (int j = 0; j + 2 < m; ++j) {
    const int Lh = m - j - 1;  // rows j+1 .. m-1
    if (warp == 0 && j > 0) {
      const int jp = j - 1, Lp = Lh + 1;
      for (int i = lane + 1; i < Lp; i += 32) C[(jp + 1 + i) * ldc + jp] *= scal_prev;
    }
    switch ((Lh + 31) / 32) {  // CTA-uniform: the step unrolled for the live 32-blocks only
      case 1: tridiag_step<1>(C, ldc, j, Lh, dT, eT, tauH, hw, scal_prev); break;
      case 2: tridiag_step<2>(C, ldc, j, Lh, dT, eT, tauH, hw, scal_prev); break;
      case 3: tridiag_step<3>(C, ldc, j, Lh, dT, eT, tauH, hw, scal_prev); break;
      case 4: tridiag_step<4>(C, ldc, j, Lh, dT, eT, tauH, hw, scal_prev); break;
      case 5: tridiag_step<5>(C, ldc, j, Lh, dT, eT, tauH, hw, scal_prev); break;
      case 6: tridiag_step<6>(C, ldc, j, Lh, dT, eT, tauH, hw, scal_prev); break;
      default: tridiag_step<7>(C, ldc, j, Lh, dT, eT, tauH, hw, scal_prev); break;
    }
  }
  __syncthreads();
  if (warp == 0 && m >= 3) {  // scaled v of the last reflector
    const int jp = m - 3, Lp = 2;
    for (int i = lane + 1; i < Lp; i += 32) C[(jp + 1 + i) * ldc + jp] *= scal_prev;
  }
  if (t == 0) {
    if (m >= 2) {
      dT[m - 2] = C[(m - 2) * ldc + (m - 2)];
      eT[m - 2] = C[(m - 1) * ldc + (m - 2)];
    }
    dT[m - 1] = C[(m - 1) * ldc + (m - 1)];
  }
  __syncthreads();
  for (int i = t; i + 1 < m; i += blockDim.x) e2[i] = eT[i] * eT[i];
  __shared__ float s_lo, s_hi;
  if (warp == 0) {  // Gershgorin bounds
    float lo = 3.4e38f, hi = -3.4e38f;
    for (int i = lane; i < m; i += 32) {
      const float r = (i > 0 ? fabsf(eT[i - 1]) : 0.f) + (i + 1 < m ? fabsf(eT[i]) : 0.f);
      lo = fminf(lo, dT[i] - r);
      hi = fmaxf(hi, dT[i] + r);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if (lane == 0) {
      const float pad = 1e-6f * fmaxf(fabsf(lo), fabsf(hi)) + 1e-30f;
      s_lo = lo - pad;
      s_hi = hi + pad;
    }
  }
  __syncthreads();
  // b. eigenvalue r (ascending) in [elo[r], ehi[r]]: count(x) = #{lambda < x}
  __shared__ float elo[kMaxM], ehi[kMaxM];
  __shared__ unsigned char cnt_le[EIG_THREADS];
  const int grp = max(1, int(blockDim.x) / m);  // threads per eigenvalue
  for (int r = t; r < m; r += blockDim.x) {
    elo[r] = s_lo;
    ehi[r] = s_hi;
  }
  __syncthreads();
  const float tiny = 1e-30f;
  auto sturm = [&](float x) -> int {
    float q = dT[0] - x;
    int c = q < 0.f;
    for (int i = 1; i < m; ++i) {
      const float qq = fabsf(q) < tiny ? -tiny : q;
      q = (dT[i] - x) - __fdividef(e2[i - 1], qq);
      c += q < 0.f;
    }
    return c;
  };
  const int my_r = t / grp, my_s = t - my_r * grp;
  for (int round = 0; round < 64; ++round) {
    if (my_r < m) {
      const float lo = elo[my_r], hi = ehi[my_r];
      const float x = lo + (hi - lo) * float(my_s + 1) / float(grp + 1);
      cnt_le[t] = sturm(x) <= my_r ? 1 : 0;  // lambda_r >= x
    }
    __syncthreads();
    __shared__ int s_more;
    if (t == 0) s_more = 0;
    __syncthreads();
    if (my_r < m && my_s == 0) {
      const float lo = elo[my_r], hi = ehi[my_r];
      float nlo = lo, nhi = hi;
      for (int q = 0; q < grp; ++q) {
        const float x = lo + (hi - lo) * float(q + 1) / float(grp + 1);
        if (cnt_le[my_r * grp + q]) {
          nlo = x;
        } else {
          nhi = x;
          break;
        }
      }
      elo[my_r] = nlo;
      ehi[my_r] = nhi;
      if (nhi - nlo > 1e-7f * (fabsf(nlo) + fabsf(nhi)) + 2e-7f * fmaxf(fabsf(s_lo), fabsf(s_hi))) s_more = 1;
    }
    __syncthreads();
    if (!s_more) break;
  }
  for (int i = t; i < m; i += blockDim.x) {
    th[i] = 0.5f * (elo[i] + ehi[i]);
    a.theta[m - 1 - i] = double(th[i]);  // descending
  }
  __syncthreads();
  // c. eigenvectors of T for the selected indices (rows of Vt): the c-th
  //    selected vector is the eigenvalue of ascending index c (smallest) or
  //    m-1-c (largest).
  const bool smallest = a.select == DCG_SELECT_SMALLEST;
  auto vrow = [&](int c) -> float* { return Vt + (smallest ? c : (m - 1 - c)) * ldc; };
  const float piv_tiny = 1e-7f * fmaxf(fabsf(s_lo), fabsf(s_hi)) + 1e-30f;  // eps |T|
  // reciprocal pivots of T - lam I, interleaved (entry i of vector c at
  // i * k_new + c, so the threads of a warp touch consecutive words): in
  // shared memory after C and V^T when they fit, in global memory otherwise
  const int used_f = (Vt == a.Vj ? 1 : 2) * m * ldc;
  float* rub = (used_f + k_new * m) * int(sizeof(float)) <= EIG_SMEM_MAX ? C + used_f : Xc;
  for (int c = t; c < k_new; c += blockDim.x) {
    const float lam = th[smallest ? c : (m - 1 - c)];
    float* __restrict__ y = vrow(c);
    float* __restrict__ ru = rub + c;  // ru[i * k_new]
    // LU of T - lam I without pivoting (tiny pivots perturbed), computed once;
    // l_i = e_{i-1} / u_{i-1}
    float ui = dT[0] - lam;
    if (fabsf(ui) < piv_tiny) ui = piv_tiny;
    float rprev = 1.f / ui;
    ru[0] = rprev;
    for (int i = 1; i < m; ++i) {
      const float l = eT[i - 1] * rprev;
      ui = fmaf(-l, eT[i - 1], dT[i] - lam);
      if (fabsf(ui) < piv_tiny) ui = piv_tiny;
      rprev = 1.f / ui;
      ru[i * k_new] = rprev;
    }
    for (int i = 0; i < m; ++i) y[i] = 1.f + 0.0137f * float((i * 7 + c * 3) % 11);
    for (int itn = 0; itn < 3; ++itn) {  // forward and back substitution, normalise
      float yp = y[0];
      for (int i = 1; i < m; ++i) {
        yp = fmaf(-eT[i - 1] * ru[(i - 1) * k_new], yp, y[i]);
        y[i] = yp;
      }
      float yn = y[m - 1] * ru[(m - 1) * k_new];
      y[m - 1] = yn;
      float nrm = yn * yn;
      for (int i = m - 2; i >= 0; --i) {
        yn = fmaf(-eT[i], yn, y[i]) * ru[i * k_new];
        y[i] = yn;
        nrm = fmaf(yn, yn, nrm);
      }
      const float inv = nrm > 0.f && isfinite(nrm) ? rsqrtf(nrm) : 0.f;
      for (int i = 0; i < m; ++i) y[i] *= inv;
    }
  }
  __syncthreads();
  // Gram-Schmidt over the selected vectors in selection order, normalisation
  // deferred: step c takes the dot products of y_c with every earlier vector
  // (and |y_{c-1}|^2), then subtracts (y_c . y_c2) / |y_c2|^2 y_c2; two
  // barriers per step.
  __shared__ float s_dot[kMaxM], s_inv2[kMaxM];
  for (int c = 1; c < k_new; ++c) {
    float* y = vrow(c);
    for (int c2 = warp; c2 < c; c2 += nw) {
      const float* y2 = vrow(c2);
      float sdot = 0.f;
      for (int i = lane; i < m; i += 32) sdot = fmaf(y[i], y2[i], sdot);
      sdot = warp_sum(sdot);
      if (lane == 0) s_dot[c2] = sdot;
    }
    if (warp == nw - 1) {
      const float* y1 = vrow(c - 1);
      float nn = 0.f;
      for (int i = lane; i < m; i += 32) nn = fmaf(y1[i], y1[i], nn);
      nn = warp_sum(nn);
      if (lane == 0) s_inv2[c - 1] = nn > 0.f ? 1.f / nn : 0.f;
    }
    __syncthreads();
    for (int i = t; i < m; i += blockDim.x) {
      float v = y[i];
      for (int c2 = 0; c2 < c; ++c2) v = fmaf(-s_dot[c2] * s_inv2[c2], vrow(c2)[i], v);
      y[i] = v;
    }
    __syncthreads();
  }
  for (int c = warp; c < k_new; c += nw) {
    float* y = vrow(c);
    float nn = 0.f;
    for (int i = lane; i < m; i += 32) nn = fmaf(y[i], y[i], nn);
    nn = warp_sum(nn);
    const float inv = nn > 0.f ? rsqrtf(nn) : 0.f;
    for (int i = lane; i < m; i += 32) y[i] *= inv;
  }
  __syncthreads();
  // z = H_0 H_1 ... H_{m-3} y: apply H_{m-3} first; one warp per vector
  for (int c = warp; c < k_new; c += nw) {
    float* y = vrow(c);
    for (int j = m - 3; j >= 0; --j) {
      const float tau = tauH[j];
      if (tau == 0.f) continue;
      const int Lh = m - j - 1;
      float sdot = 0.f;
      for (int i = lane; i < Lh; i += 32) {
        const float v = i == 0 ? 1.f : C[(j + 1 + i) * ldc + j];
        sdot = fmaf(v, y[j + 1 + i], sdot);
      }
      sdot = warp_sum(sdot) * tau;
      for (int i = lane; i < Lh; i += 32) {
        const float v = i == 0 ? 1.f : C[(j + 1 + i) * ldc + j];
        y[j + 1 + i] = fmaf(-sdot, v, y[j + 1 + i]);
      }
      __syncwarp();
    }
  }
  __syncthreads();
  // 7. U[:, c] = S L^{-T} v_sel(c) on the kept rows (dropped rows are zero):
  //    back substitution L^T Y = [v_sel(0) ...] with Y (m x k_new, odd leading
  //    dimension) in the shared memory that held C, then scale
  const int m_orig = a.k_act + a.nstored;
  const int ldb = k_new | 1;
  float* Y = C;
  for (int i = warp; i < m; i += nw)
    for (int c = lane; c < k_new; c += 32) Y[i * ldb + c] = vrow(c)[i];
  __syncthreads();
  trsm_lower_t(Ff, m, Y, ldb, m, k_new, Ld);
  for (int c = warp; c < k_new; c += nw)
    for (int i = lane; i < m_orig; i += 32) {
      const int ci = pos[i];
      a.U[int64_t(c) * m_orig + i] = ci >= 0 ? scale[i] * Y[ci * ldb + c] : 0.f;
    }
  __syncthreads();
  if (t == 0) {
    *a.status = DCG_OK;
    a.k_out[0] = k_new;
    a.k_out[1] = m;
  }
}

// Float64 refinement of the kept (harmonic) Ritz values: for every selected
// coefficient vector u = U[:, c] (float32 from the eigen-solve above) the
// pencil's Rayleigh quotient theta = (u^T G u) / (u^T F u) in float64, with
// F and G the float64 matrices of Eq. 7 (or of the orthogonal projection).
// For the symmetric pencil the quotient's error is quadratic in the vector's
// (a float32 vector good to ~1e-5 gives theta to ~1e-10), so the values the
// selection keeps are float64-accurate; the basis W itself is that of the
// float32 vectors. One CTA per selected vector; the quadratic forms see the
// symmetric part of F and G whatever the rounding of their two triangles.
__global__ void __launch_bounds__(256) k_ritz_rq(RitzArgs a, int m_orig) {
  if (*a.status != DCG_OK) return;
  const int k_new = a.k_out[0], m = a.k_out[1];
  const int c = blockIdx.x;
  if (c >= k_new) return;
  __shared__ double u[kMaxM];
  for (int i = threadIdx.x; i < m_orig; i += blockDim.x) u[i] = double(a.U[int64_t(c) * m_orig + i]);
  __syncthreads();
  double sf = 0.0, sg = 0.0;
  for (int idx = threadIdx.x; idx < m_orig * m_orig; idx += blockDim.x) {
    const int i = idx / m_orig, j = idx % m_orig;
    const double w = u[i] * u[j];
    sf = fma(w, a.F[idx], sf);
    sg = fma(w, a.G[idx], sg);
  }
  __shared__ double s_f[8], s_g[8];
  sf = warp_sum(sf);
  sg = warp_sum(sg);
  if ((threadIdx.x & 31) == 0) {
    s_f[threadIdx.x >> 5] = sf;
    s_g[threadIdx.x >> 5] = sg;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tf = 0.0, tg = 0.0;
    for (int w = 0; w < 8; ++w) {
      tf += s_f[w];
      tg += s_g[w];
    }
    // the c-th selected value: descending index c (largest) or m - 1 - c
    const int idx = a.select == DCG_SELECT_SMALLEST ? m - 1 - c : c;
    if (tf > 0.0) a.theta[idx] = tg / tf;
  }
}

// W_out[:, c] = Z U[:, c] for c < k_new (Z = [W | P]); thread per row, 32
// output columns per pass.
__global__ void __launch_bounds__(256) k_zu(RitzArgs a, int m, int k_new) {
  extern __shared__ float Us[];  // m x 32
  if (*a.status != DCG_OK) return;
  k_new = min(k_new, a.k_out[0]);
  const int n = a.n;
  for (int c0 = 0; c0 < k_new; c0 += 32) {
    const int cw = min(32, k_new - c0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < m * 32; idx += blockDim.x) {
      const int i = idx / 32, c = idx % 32;
      Us[idx] = c < cw ? a.U[int64_t(c0 + c) * m + i] : 0.f;
    }
    __syncthreads();
    for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < n; row += gridDim.x * blockDim.x) {
      float acc[32];
#pragma unroll
      for (int c = 0; c < 32; ++c) acc[c] = 0.f;
      for (int i = 0; i < m; ++i) {
        const float z = gram_col(a.W, a.k_act, a.P, i, n)[row];
#pragma unroll
        for (int c = 0; c < 32; ++c) acc[c] = fmaf(z, Us[i * 32 + c], acc[c]);
      }
      for (int c = 0; c < cw; ++c) a.Wout[int64_t(c0 + c) * n + row] = acc[c];
    }
  }
}

// Column norm and sign pivot (largest magnitude, lowest index) of W_out[:, c].
__global__ void __launch_bounds__(256) k_colnorm(RitzArgs a) {
  if (*a.status != DCG_OK || int(blockIdx.x) >= a.k_out[0]) return;
  const int c = blockIdx.x, n = a.n;
  const float* col = a.Wout + int64_t(c) * n;
  double ss = 0.0;
  float best = -1.f;
  int bi = 0x7fffffff;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const float v = col[i];
    ss += double(v) * double(v);
    const float av = fabsf(v);
    if (av > best || (av == best && i < bi)) {
      best = av;
      bi = i;
    }
  }
  __shared__ double s_ss[256];
  __shared__ float s_b[256];
  __shared__ int s_i[256];
  s_ss[threadIdx.x] = ss;
  s_b[threadIdx.x] = best;
  s_i[threadIdx.x] = bi;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      s_ss[threadIdx.x] += s_ss[threadIdx.x + o];
      const float b2 = s_b[threadIdx.x + o];
      const int i2 = s_i[threadIdx.x + o];
      if (b2 > s_b[threadIdx.x] || (b2 == s_b[threadIdx.x] && i2 < s_i[threadIdx.x])) {
        s_b[threadIdx.x] = b2;
        s_i[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double nrm = sqrt(s_ss[0]);
    const double sgn = col[s_i[0]] < 0.f ? -1.0 : 1.0;
    a.colscale[c] = nrm > 0.0 ? sgn / nrm : 0.0;
  }
}

// W (columns 1.. of XW) <- W_out * colscale
__global__ void __launch_bounds__(256) k_colscale(RitzArgs a, float* dstW, int k_new) {
  if (*a.status != DCG_OK) return;
  k_new = min(k_new, a.k_out[0]);
  const int n = a.n;
  const int64_t total = int64_t(n) * k_new;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(idx / n);
    dstW[idx] = float(double(a.Wout[idx]) * a.colscale[c]);
  }
}

cudaError_t ritz_configure() {
  const int smem = EIG_SMEM_MAX;
  cudaError_t e = cudaFuncSetAttribute(k_ritz_eig, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_zu, cudaFuncAttributeMaxDynamicSharedMemorySize, kMaxM * 32 * 4);
}

// F and G of Eq. 7 from the scalars the solve recorded (the sparse forms of
// Saad et al. that Sec. 2.3 refers to), instead of the Gram products over
// Z = [W, P] and AZ = [AW, AP]. Columns: W (k_act), then the direction slots
// in ring order. With A-conjugate directions ((AW)^T p_j = 0 and
// p_i^T A p_j = 0) and mutually orthogonal residuals:
//   F = diag(E, d_j);
//   G_WW = (AW)^T AW, G_{W,j} = (AW)^T A p_j = ((AW)^T r_j - (AW)^T r'_{j+1}) / alpha_j,
//   G_{jj} = (|r_j|^2 + |r'_{j+1}|^2) / alpha_j^2,
//   G_{j,j+1} = -|r'_{j+1}|^2 / (alpha_j alpha_{j+1}) for consecutive stored
//   directions, zero between others.
// E and G_W are symmetrised as the Gram path's products are. One CTA.
__global__ void __launch_bounds__(256) k_fg_sparse(RitzArgs a) {
  const int k = a.k_act, ns = a.nstored, m = k + ns;
  const int t = threadIdx.x;
  const double* rec = a.fg;
  for (int idx = t; idx < m * m; idx += blockDim.x) {
    const int i = idx / m, j = idx - i * m;
    double f = 0.0, g = 0.0;
    if (i < k && j < k) {
      f = 0.5 * (a.E[i * k + j] + a.E[j * k + i]);
      g = 0.5 * (a.GW[i * k + j] + a.GW[j * k + i]);
    }
    a.F[idx] = f;
    a.G[idx] = g;
  }
  __syncthreads();
  for (int sl = t; sl < ns; sl += blockDim.x) {
    const double d = rec[sl * FG_REC + 0], al = rec[sl * FG_REC + 1];
    const double ra = rec[sl * FG_REC + 2], rb = rec[sl * FG_REC + 3], jj = rec[sl * FG_REC + 4];
    const int c = k + sl;
    a.F[int64_t(c) * m + c] = d;
    a.G[int64_t(c) * m + c] = (ra + rb) / (al * al);
    for (int s2 = 0; s2 < ns; ++s2) {
      if (rec[s2 * FG_REC + 4] == jj + 1.0) {  // the next direction is stored too
        const double v = -rb / (al * rec[s2 * FG_REC + 1]);
        a.G[int64_t(c) * m + (k + s2)] = v;
        a.G[int64_t(k + s2) * m + c] = v;
      }
    }
  }
  for (int idx = t; idx < k * ns; idx += blockDim.x) {
    const int sl = idx / k, cw = idx - sl * k;
    const double al = rec[sl * FG_REC + 1];
    const double v = (fg_ha(a.fg, a.ellmax, a.kmax, sl)[cw] - fg_hb(a.fg, a.ellmax, a.kmax, sl)[cw]) / al;
    a.G[int64_t(cw) * m + (k + sl)] = v;
    a.G[int64_t(k + sl) * m + cw] = v;
  }
}

cudaError_t launch_ritz(const RitzArgs& a, int num_sms, float* dstW, cudaStream_t s) {
  const int m = a.k_act + a.nstored;
  const int k_new = min(a.k_want, m);
  if (m == 0 || k_new == 0) return cudaSuccess;
  GramArgs g{};
  g.n = a.n;
  g.part = a.part;
  cudaError_t e;
  if (a.extraction == DCG_EXTRACT_RITZ) {
    // orthogonal projection: F = Z^T Z, G = Z^T (AZ)
    g.a1 = a.W; g.ka1 = a.k_act; g.a2 = a.P; g.ka2 = a.nstored;
    g.b1 = a.W; g.kb1 = a.k_act; g.b2 = a.P; g.kb2 = a.nstored;
    e = launch_gram(g, m, m, num_sms, a.F, nullptr, s);
    if (e != cudaSuccess) return e;
    g.b1 = a.AW; g.b2 = a.Q;
    e = launch_gram(g, m, m, num_sms, a.G, nullptr, s);
    if (e != cudaSuccess) return e;
  } else if (a.fg_form == DCG_FG_SPARSE) {
    // harmonic projection (Eq. 7) from the recorded scalars
    k_fg_sparse<<<1, 256, 0, s>>>(a);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  } else {
    // harmonic projection (Eq. 7): F = Z^T (AZ), G = (AZ)^T (AZ)
    g.a1 = a.W; g.ka1 = a.k_act; g.a2 = a.P; g.ka2 = a.nstored;
    g.b1 = a.AW; g.kb1 = a.k_act; g.b2 = a.Q; g.kb2 = a.nstored;
    e = launch_gram(g, m, m, num_sms, a.F, nullptr, s);
    if (e != cudaSuccess) return e;
    g.a1 = a.AW; g.a2 = a.Q;
    e = launch_gram(g, m, m, num_sms, a.G, nullptr, s);
    if (e != cudaSuccess) return e;
  }
  k_ritz_eig<<<1, EIG_THREADS, EIG_SMEM_MAX, s>>>(a, m, k_new);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_ritz_rq<<<k_new, 256, 0, s>>>(a, m);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_zu<<<num_sms, 256, size_t(m) * 32 * sizeof(float), s>>>(a, m, k_new);  // k_new is an upper bound; k_zu reads k_out
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_colnorm<<<k_new, 256, 0, s>>>(a);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_colscale<<<num_sms * 2, 256, 0, s>>>(a, dstW, k_new);
  return cudaGetLastError();
}

}  // namespace dcg
