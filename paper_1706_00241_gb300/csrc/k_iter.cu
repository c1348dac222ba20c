// Per-iteration kernels of Deflated-CG (Algorithm 1, Sec. 2.2).
//
// Each kernel owns a contiguous band of rows per CTA. Reductions are two-level:
// float32 sums inside a CTA, float64 partials across CTAs, summed in a fixed
// order by the last CTA to arrive (no CTA waits on another). The last CTA also
// does the small float64 work that needs the full sums (alpha, beta, the k x k
// solve for mu or gamma) and the control decisions of the solve graph.
#include "dcg_kernels.cuh"

namespace dcg {

__device__ __forceinline__ void band_of(int n, int& i0, int& i1) {
  i0 = int((long long)blockIdx.x * n / gridDim.x);
  i1 = int((long long)(blockIdx.x + 1) * n / gridDim.x);
}

// Partial sums live slot-major: slot c of CTA b at partials[c * gridDim.x + b],
// so the last CTA reads each slot with coalesced loads.
__device__ __forceinline__ double* my_slots(double* partials) { return partials + blockIdx.x; }

// Dot products of k columns (column c at cols + c n) with a band vector held in
// shared memory; warp w takes columns w, w + nwarps, ...; writes float64
// partials to slots out[c * gridDim.x].
__device__ void band_col_dots(const float* __restrict__ cols, int k, int n, int i0, int len, const float* vs,
                              double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  const int G = gridDim.x;
  for (int c = warp; c < k; c += nw) {
    const float* col = cols + int64_t(c) * n + i0;
    float s = 0.f;
    for (int i = lane; i < len; i += 32) s = fmaf(__ldg(col + i), vs[i], s);
    s = warp_sum(s);
    if (lane == 0) out[int64_t(c) * G] = double(s);
  }
}

// Block-wide float sum of one value per thread (result valid in thread 0).
__device__ float block_sum(float v) {
  __shared__ float s[32];
  v = warp_sum(v);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) s[warp] = v;
  __syncthreads();
  float t = 0.f;
  if (threadIdx.x < 32) {
    t = (lane < (int)(blockDim.x >> 5)) ? s[lane] : 0.f;
    t = warp_sum(t);
  }
  return t;
}

// Last CTA: sums `count` float64 slots over all CTAs into dst (fixed order:
// lane-strided partial sums, then a warp tree). One warp per slot, four slots
// in flight per warp so that the loads overlap.
__device__ void reduce_partials(const double* partials, int count, double* dst) {
  const int G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c0 = warp * 4; c0 < count; c0 += nw * 4) {
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    for (int b = lane; b < G; b += 32) {
#pragma unroll
      for (int u = 0; u < 4; ++u)
        if (c0 + u < count) s[u] += __ldcg(partials + int64_t(c0 + u) * G + b);
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const double v = warp_sum(s[u]);
      if (lane == 0 && c0 + u < count) dst[c0 + u] = v;
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// r_{-1} = b for a cold start (a warm start has r_{-1} = b - A x_{-1} from the
// compensated residual kernel already); |b|^2 and the stopping threshold
// (reading R2: tol relative to |b|).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_setup_r(Ws w) {
  DevState* st = w.st;
  const int n = w.n;
  const int warm = st->warm_start;
  float acc = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float bi = w.b[i];
    if (!warm) w.r[i] = bi;
    acc = fmaf(bi, bi, acc);
  }
  const float s = block_sum(acc);
  if (threadIdx.x == 0) my_slots(w.partials)[0] = double(s);
  if (!arrive_last(&st->ticket[T_SETUP_G])) return;
  __shared__ double tot;
  reduce_partials(w.partials, 1, &tot);
  if (threadIdx.x == 0) {
    st->bnorm2 = tot;
    st->thresh2 = w.tol * w.tol * tot;
    if (!(tot > 0.0)) {  // b = 0: x = 0 with no iterations (reading R2)
      st->zero_rhs = 1;
      st->done = 1;
      st->true_valid = 1;
      st->relres_true = 0.0;
    }
  }
}

cudaError_t launch_setup_r(const Ws& w, int grid, cudaStream_t s) {
  k_setup_r<<<grid, 256, 0, s>>>(w);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// g = W^T r, then (last CTA) gamma = E^{-1} g: the correction of line 3 (and of
// the re-deflation after a residual replacement, reading R13).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_check_dots(Ws w) {
  DevState* st = w.st;
  if (st->done) return;
  const int k = st->k;
  if (k == 0) return;
  extern __shared__ float sh[];
  const int n = w.n;
  int i0, i1;
  band_of(n, i0, i1);
  const int len = i1 - i0;
  for (int i = threadIdx.x; i < len; i += blockDim.x) sh[i] = w.r[i0 + i];
  __syncthreads();
  double* part = my_slots(w.partials);
  band_col_dots(w.XW + n, k, n, i0, len, sh, part);
  if (!arrive_last(&st->ticket[T_CHECK_G])) return;
  __shared__ double g[kMaxK], tmp[kMaxK], y[kMaxK];
  reduce_partials(w.partials, k, g);
  if (threadIdx.x < 32) apply_Einv_warp(w.Linv, k, g, tmp, y);
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    w.gamma[c] = y[c];
    w.gamma_f[c] = float(y[c]);
  }
}

cudaError_t launch_check_dots(const Ws& w, int grid, cudaStream_t s) {
  const int band = (w.n + grid - 1) / grid + 1;
  k_check_dots<<<grid, 256, size_t(band) * sizeof(float), s>>>(w);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// x += W gamma, r -= (AW) gamma (line 3 / reading R13), then rho = r^T r,
// h = (AW)^T r, hp = (AW)^T p. The last CTA finishes according to the place of
// the kernel in the solve graph:
//   setup:    mu_0 = E^{-1} h (line 4), beta = 0, arms the pre-loop check if
//             |r_0| <= tol |b|;
//   pre_loop: after a failed initial check only rho is refreshed;
//   in loop:  beta = rho_rec / rho from the recursion's own |r_{j+1}|^2
//             (st->rho_new, written by phase 1), rho = |r_true|^2 after the
//             replacement, and mu = E^{-1}(h + beta hp), which re-projects
//             p_{j+1} against W (R13: keep beta, recompute rho). Where the
//             true residual sits far above the recursive one (an inexact
//             iteration operator at its accuracy floor) beta stays <= 1 and
//             the step acts as a restart instead of amplifying p.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_check_update(Ws w, int pre_loop, int setup, Handles hd) {
  DevState* st = w.st;
  if (st->done) return;
  extern __shared__ float sh[];
  const int n = w.n, k = st->k;
  int i0, i1;
  band_of(n, i0, i1);
  const int len = i1 - i0;
  float* rs = sh;
  float* ps = sh + len;
  __shared__ float gsh[kMaxK];
  for (int c = threadIdx.x; c < k; c += blockDim.x) gsh[c] = w.gamma_f[c];
  __syncthreads();
  const bool save_best = st->save_best != 0;  // this check found the best iterate so far
  float acc = 0.f;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const int gi = i0 + i;
    if (save_best) w.xbest[gi] = w.xd[gi];
    float dx = 0.f, ri = w.r[gi];
    for (int c = 0; c < k; ++c) {
      const float g = gsh[c];
      dx = fmaf(w.XW[int64_t(c + 1) * n + gi], g, dx);
      ri = fmaf(-w.Y[int64_t(c + 1) * n + gi], g, ri);
    }
    if (k) {
      w.xd[gi] += double(dx);
      w.r[gi] = ri;
    }
    rs[i] = ri;
    ps[i] = w.p[gi];
    acc = fmaf(ri, ri, acc);
  }
  const float rho_part = block_sum(acc);
  const int G = gridDim.x;
  double* part = my_slots(w.partials);
  if (threadIdx.x == 0) part[0] = double(rho_part);
  band_col_dots(w.Y + n, k, n, i0, len, rs, part + G);
  if (!setup && !pre_loop) band_col_dots(w.Y + n, k, n, i0, len, ps, part + int64_t(1 + k) * G);
  if (!arrive_last(&st->ticket[setup ? T_SETUP_H : T_CHECK_H])) return;

  __shared__ double red[1 + 2 * kMaxK], tmp[kMaxK], y[kMaxK];
  reduce_partials(w.partials, (setup || pre_loop) ? 1 + k : 1 + 2 * k, red);
  const double rho_new = red[0];
  __shared__ double s_beta;
  if (threadIdx.x == 0) {
    if (setup) {
      s_beta = 0.0;
    } else {
      s_beta = st->rho > 0.0 ? st->rho_new / st->rho : 0.0;
    }
  }
  __syncthreads();
  if (!pre_loop) {
    const double beta = s_beta;
    if (!setup)
      for (int c = threadIdx.x; c < k; c += blockDim.x) red[1 + c] += beta * red[1 + k + c];
    __syncthreads();
    if (threadIdx.x < 32) apply_Einv_warp(w.Linv, k, red + 1, tmp, y);
    __syncthreads();
    for (int c = threadIdx.x; c < k; c += blockDim.x) {
      w.mu[c] = y[c];
      w.mu_f[c] = float(y[c]);
    }
  }
  for (int c = threadIdx.x; c < k; c += blockDim.x) {  // gamma is applied: phase 2 must not repeat it
    w.gamma[c] = 0.0;
    w.gamma_f[c] = 0.f;
  }
  if (threadIdx.x == 0) {
    st->save_best = 0;
    st->rho = rho_new;
    st->rho_new = rho_new;
    if (k) st->true_valid = 0;
    if (setup) {
      st->beta = 0.0;
      if (st->hist_on && st->hist_cap > 0) w.hist[0] = sqrt(rho_new / st->bnorm2);
      const int arm = rho_new <= st->thresh2 ? 1 : 0;
      st->mode = arm;
      if (hd.pre) cudaGraphSetConditional(hd.pre, arm);
    } else {
      st->beta = s_beta;
      st->mode = 0;
      if (!pre_loop && st->iter >= st->max_iter) {
        st->status = DCG_ERR_MAXITER;
        st->done = 1;
      }
    }
  }
}

cudaError_t launch_check_update(const Ws& w, int grid, int pre_loop, int setup, Handles h, cudaStream_t s) {
  const int band = (w.n + grid - 1) / grid + 1;
  k_check_update<<<grid, 256, size_t(2 * band) * sizeof(float), s>>>(w, pre_loop, setup, h);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Phase 1 of an iteration (lines 6-10 and 13-14 of Algorithm 1), after q = A p
// and d = p^T q have been formed by the operator kernel:
//   alpha = rho / d, x += alpha p, r -= alpha q, store (p, q) in the window,
//   rho' = r^T r, h = (AW)^T r, g = W^T r [, hp = (AW)^T p];
// last CTA: the convergence / refinement decision and the IF-node value for
// the check branch; otherwise beta and mu (line 11, reading R1) for phase 2.
//
// Float32 re-deflation: in exact arithmetic W^T r_j = 0 for all j (Eq. 5), so
// gamma = E^{-1} W^T r is zero. In float32 the rounding of mu leaves p slightly
// A-non-conjugate to W, and r then drifts along W by ~eps32 * lambda(W) per
// step; CG never removes that drift and the recursive residual stalls. Phase 2
// therefore applies x += W gamma, r -= AW gamma every iteration (a no-op in
// exact arithmetic). With r~ = r - AW gamma:
//   |r~|^2 = rho' - 2 gamma^T h + gamma^T G_W gamma,   G_W = (AW)^T AW,
//   mu = E^{-1} ((AW)^T r~ + beta hp) = E^{-1} h - M g + beta E^{-1} hp,
// with E^{-1}, N = G_W E^{-1} and M = E^{-1} N formed once per solve, so the
// last CTA only does k x k float64 matrix-vector products in parallel.
//
// Layout: one row per thread (the grid covers n with 256-row CTAs, rows
// strided when n > 256 * grid); dot products are accumulated per thread for
// 32 columns at a time and reduced through shared memory.
// ---------------------------------------------------------------------------
constexpr int P1_THREADS = 256;
constexpr int P1_CHUNK = 32;

// Block reduction of P1_CHUNK per-thread values; column c of the result goes
// to out[c * gridDim.x] (cw columns valid).
__device__ void chunk_reduce(const float* acc, int cw, float (*red)[P1_CHUNK + 1], double* out) {
  const int G = gridDim.x, t = threadIdx.x;
  __shared__ float part8[P1_THREADS / P1_CHUNK][P1_CHUNK];
#pragma unroll
  for (int c = 0; c < P1_CHUNK; ++c) red[t][c] = acc[c];
  __syncthreads();
  {
    const int c = t % P1_CHUNK, q = t / P1_CHUNK;
    float s = 0.f;
    for (int i = q * 32; i < q * 32 + 32; ++i) s += red[i][c];
    part8[q][c] = s;
  }
  __syncthreads();
  if (t < cw) {
    float s = 0.f;
    for (int q = 0; q < P1_THREADS / P1_CHUNK; ++q) s += part8[q][t];
    out[int64_t(t) * G] = double(s);
  }
  __syncthreads();
}

// Per-CTA partial dot products h = (AW)^T r, g = W^T r and (optionally)
// hp = (AW)^T p over the thread's rows, in one pass over AW and W per block of
// P1_CHUNK columns. Slots: h at out_h[c * G], g at out_g[c * G], hp at out_hp[c * G].
__device__ void phase1_dots(const float* __restrict__ AW, const float* __restrict__ W, int k, int n,
                            const int* rows, int nrows, const float* rv, const float* pv, bool do_hp,
                            float (*red)[P1_CHUNK + 1], double* out_h, double* out_g, double* out_hp) {
  const int G = gridDim.x;
  for (int c0 = 0; c0 < k; c0 += P1_CHUNK) {
    const int cw = min(P1_CHUNK, k - c0);
    float ah[P1_CHUNK], ag[P1_CHUNK], ap[P1_CHUNK];
#pragma unroll
    for (int c = 0; c < P1_CHUNK; ++c) ah[c] = ag[c] = ap[c] = 0.f;
    for (int j = 0; j < nrows; ++j) {
      const float* aw = AW + int64_t(c0) * n + rows[j];
      const float* ww = W + int64_t(c0) * n + rows[j];
      const float r = rv[j], p = pv[j];
#pragma unroll
      for (int c = 0; c < P1_CHUNK; ++c) {
        if (c < cw) {
          const float a = __ldg(aw + int64_t(c) * n);
          const float wv = __ldg(ww + int64_t(c) * n);
          ah[c] = fmaf(a, r, ah[c]);
          ap[c] = fmaf(a, p, ap[c]);
          ag[c] = fmaf(wv, r, ag[c]);
        }
      }
    }
    chunk_reduce(ah, cw, red, out_h + int64_t(c0) * G);
    chunk_reduce(ag, cw, red, out_g + int64_t(c0) * G);
    if (do_hp) chunk_reduce(ap, cw, red, out_hp + int64_t(c0) * G);
  }
}

constexpr int P1_MAX_ROWS = 8;  // rows per thread (n <= 8 * 256 * grid)

__global__ void __launch_bounds__(P1_THREADS) k_phase1(Ws w, Handles hd) {
  DevState* st = w.st;
  if (st->done) return;
  __shared__ float red[P1_THREADS][P1_CHUNK + 1];
  const int n = w.n, k = st->k;
  const double d = st->d;
  const bool ok = (d > 0.0) && isfinite(d);
  const double alpha_d = ok ? st->rho / d : 0.0;
  const float alpha = float(alpha_d);
  int slot = -1;
  if (st->ell > 0) {
    if (st->window == DCG_WINDOW_FIRST) {
      if (st->iter < st->ell) slot = st->iter;
    } else {
      slot = st->head;
    }
  }
  const int reproj = st->reproject;
  int rows[P1_MAX_ROWS];
  float rv[P1_MAX_ROWS], pv[P1_MAX_ROWS];
  int nrows = 0;
  float acc = 0.f;
  const int stride = gridDim.x * P1_THREADS;
  for (int gi = blockIdx.x * P1_THREADS + threadIdx.x; gi < n && nrows < P1_MAX_ROWS; gi += stride) {
    const float pi = w.p[gi], qi = w.q[gi];
    float ri = w.r[gi];
    if (ok) {
      w.xd[gi] += alpha_d * double(pi);
      ri = fmaf(-alpha, qi, ri);
      w.r[gi] = ri;
      if (slot >= 0) {
        w.P[int64_t(slot) * n + gi] = pi;
        w.Q[int64_t(slot) * n + gi] = qi;
      }
    }
    rows[nrows] = gi;
    rv[nrows] = ri;
    pv[nrows] = pi;
    ++nrows;
    acc = fmaf(ri, ri, acc);
  }
  const float rho_part = block_sum(acc);
  const int G = gridDim.x;
  double* part = my_slots(w.partials);
  if (threadIdx.x == 0) part[0] = double(rho_part);
  if (ok && k > 0)
    phase1_dots(w.Y + n, w.XW + n, k, n, rows, nrows, rv, pv, reproj != 0, red, part + G,
                part + int64_t(1 + k) * G, part + int64_t(1 + 2 * k) * G);
  if (!arrive_last(&st->ticket[T_PHASE1])) return;

  __shared__ double sred[1 + 3 * kMaxK], gam[kMaxK], av[kMaxK], bv[kMaxK], uv[kMaxK];
  __shared__ int s_mode;
  __shared__ double s_beta;
  if (!ok) {
    if (threadIdx.x == 0) {
      st->status = DCG_ERR_BREAKDOWN;
      st->done = 1;
      if (hd.chk) cudaGraphSetConditional(hd.chk, 0);
    }
    return;
  }
  reduce_partials(w.partials, 1 + (reproj ? 3 : 2) * k, sred);
  const double* h = sred + 1;
  const double* g = sred + 1 + k;
  const double* hp = sred + 1 + 2 * k;
  // gamma = E^{-1} g, a = E^{-1} h - M g, b = E^{-1} hp, u = N g = G_W gamma
  for (int o = threadIdx.x; o < 4 * k; o += blockDim.x) {
    const int which = o / k, c = o % k;
    double s = 0.0;
    const double* Ei = w.Einv + c * k;
    if (which == 0) {
      for (int j = 0; j < k; ++j) s = fma(Ei[j], g[j], s);
      gam[c] = s;
    } else if (which == 1) {
      const double* Mi = w.M + c * k;
      for (int j = 0; j < k; ++j) s = fma(Ei[j], h[j], fma(-Mi[j], g[j], s));
      av[c] = s;
    } else if (which == 2) {
      if (reproj)
        for (int j = 0; j < k; ++j) s = fma(Ei[j], hp[j], s);
      bv[c] = s;
    } else {
      const double* Ni = w.N + c * k;
      for (int j = 0; j < k; ++j) s = fma(Ni[j], g[j], s);
      uv[c] = s;
    }
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double corr = 0.0;
    for (int c = threadIdx.x; c < k; c += 32) corr += gam[c] * (uv[c] - 2.0 * h[c]);
    corr = warp_sum(corr);
    if (threadIdx.x == 0) {
      double rho_new = sred[0] + corr;
      if (!(rho_new > 0.0)) rho_new = sred[0];
      const int iter = st->iter + 1;
      st->iter = iter;
      st->alpha = alpha_d;
      if (st->ell > 0) {
        if (st->window == DCG_WINDOW_FIRST) {
          st->nstored = min(iter, st->ell);
        } else {
          st->head = (st->head + 1) % st->ell;
          st->nstored = min(st->nstored + 1, st->ell);
        }
      }
      if (st->hist_on && iter < st->hist_cap) w.hist[iter] = sqrt(rho_new / st->bnorm2);
      st->rho_new = rho_new;
      st->true_valid = 0;
      int mode = 0;
      if (rho_new <= st->thresh2)
        mode = 1;
      else if (st->refine_every > 0 && iter % st->refine_every == 0)
        mode = 2;
      st->mode = mode;
      s_mode = mode;
      s_beta = rho_new / st->rho;
      if (mode == 0) {
        st->beta = s_beta;
        st->rho = rho_new;
        if (iter >= st->max_iter) {
          st->status = DCG_ERR_MAXITER;
          st->done = 1;
        }
      }
      if (hd.chk) cudaGraphSetConditional(hd.chk, mode != 0 ? 1 : 0);
    }
  }
  __syncthreads();
  if (s_mode != 0) return;  // the check branch recomputes gamma, beta and mu
  const double beta = s_beta;
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    const double mu = av[c] + beta * bv[c];
    w.mu[c] = mu;
    w.mu_f[c] = float(mu);
    w.gamma[c] = gam[c];
    w.gamma_f[c] = float(gam[c]);
  }
}

int phase1_grid(int n, int num_sms) {
  int g = (n + P1_THREADS - 1) / P1_THREADS;
  if (g > num_sms) g = num_sms;
  while (int64_t(g) * P1_THREADS * P1_MAX_ROWS < n) ++g;
  return g < 1 ? 1 : g;
}

cudaError_t launch_phase1(const Ws& w, int grid, Handles h, cudaStream_t s) {
  k_phase1<<<phase1_grid(w.n, grid), P1_THREADS, 0, s>>>(w, h);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// E^{-1} = Linv^T Linv, N = G_W E^{-1}, M = E^{-1} N (float64, k x k, once
// per solve): the small matrices phase 1 applies every iteration. One CTA per
// output row, one thread per column.
// ---------------------------------------------------------------------------
__global__ void k_small_prods(Ws w, int which) {
  const DevState* st = w.st;
  if (st->done) return;
  const int k = st->k, i = blockIdx.x;
  if (i >= k) return;
  for (int j = threadIdx.x; j < k; j += blockDim.x) {
    double s = 0.0;
    if (which == 0) {         // Einv[i][j] = sum_l Linv[l][i] Linv[l][j], l >= max(i, j)
      for (int l = max(i, j); l < k; ++l) s = fma(w.Linv[l * k + i], w.Linv[l * k + j], s);
      w.Einv[i * k + j] = s;
    } else if (which == 1) {  // N = G_W Einv
      for (int l = 0; l < k; ++l) s = fma(w.GW[i * k + l], w.Einv[l * k + j], s);
      w.N[i * k + j] = s;
    } else {                  // M = Einv N
      for (int l = 0; l < k; ++l) s = fma(w.Einv[i * k + l], w.N[l * k + j], s);
      w.M[i * k + j] = s;
    }
  }
}

cudaError_t launch_small_prods(const Ws& w, cudaStream_t s) {
  if (w.kmax == 0) return cudaSuccess;
  for (int which = 0; which < 3; ++which) {
    k_small_prods<<<w.kmax, 128, 0, s>>>(w, which);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Phase 2 (line 12): x += W gamma, r -= AW gamma (float32 re-deflation, zero
// in exact arithmetic), then p = beta p + r - W mu. In the loop body it also
// ends the while node once the solve is done.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_phase2(Ws w, Handles hd, int set_loop) {
  DevState* st = w.st;
  if (st->done) {
    if (set_loop && hd.loop && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hd.loop, 0);
    return;
  }
  const int n = w.n, k = st->k;
  __shared__ float msh[kMaxK], gsh[kMaxK];
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    msh[c] = w.mu_f[c];
    gsh[c] = w.gamma_f[c];
  }
  __syncthreads();
  const float beta = float(st->beta);
  int i0, i1;
  band_of(n, i0, i1);
  for (int gi = i0 + threadIdx.x; gi < i1; gi += blockDim.x) {
    float ri = w.r[gi], dx = 0.f, wm = 0.f;
    for (int c0 = 0; c0 < k; c0 += 16) {  // 32 loads in flight per thread
      float wc[16], ac[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        wc[c] = c0 + c < k ? __ldg(w.XW + int64_t(c0 + c + 1) * n + gi) : 0.f;
        ac[c] = c0 + c < k ? __ldg(w.Y + int64_t(c0 + c + 1) * n + gi) : 0.f;
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        if (c0 + c < k) {
          dx = fmaf(wc[c], gsh[c0 + c], dx);
          wm = fmaf(wc[c], msh[c0 + c], wm);
          ri = fmaf(-ac[c], gsh[c0 + c], ri);
        }
      }
    }
    if (k) {
      w.xd[gi] += double(dx);
      w.r[gi] = ri;
    }
    // beta = 0 starts a fresh direction without reading the old p (a
    // non-finite p left by an earlier failed solve must not leak in)
    w.p[gi] = (beta != 0.f ? fmaf(beta, w.p[gi], ri) : ri) - wm;
  }
}

cudaError_t launch_phase2(const Ws& w, int grid, Handles h, cudaStream_t s) {
  k_phase2<<<grid, 256, 0, s>>>(w, h, 1);
  return cudaGetLastError();
}

cudaError_t launch_phase2_setup(const Ws& w, int grid, cudaStream_t s) {
  Handles h{};
  k_phase2<<<grid, 256, 0, s>>>(w, h, 0);
  return cudaGetLastError();
}

__global__ void k_loop_gate(Ws w, Handles hd) {
  if (w.st->done && hd.loop) cudaGraphSetConditional(hd.loop, 0);
}

cudaError_t launch_loop_gate(const Ws& w, Handles h, cudaStream_t s) {
  k_loop_gate<<<1, 1, 0, s>>>(w, h);
  return cudaGetLastError();
}

__global__ void k_final_gate(Ws w, Handles hd) {
  const DevState* st = w.st;
  if (hd.fin) cudaGraphSetConditional(hd.fin, (!st->true_valid && !st->zero_rhs) ? 1 : 0);
}

cudaError_t launch_final_gate(const Ws& w, Handles h, cudaStream_t s) {
  k_final_gate<<<1, 1, 0, s>>>(w, h);
  return cudaGetLastError();
}

// b = 0 returns x = 0; a stagnated solve returns the iterate with the
// smallest true residual seen, with that residual.
__global__ void __launch_bounds__(256) k_finalize(Ws w) {
  DevState* st = w.st;
  const bool restore = !st->zero_rhs && st->status == DCG_ERR_STAGNATION && st->rho_best > 0.0;
  if (!st->zero_rhs && !restore) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x)
    w.xd[i] = restore ? w.xbest[i] : 0.0;
  if (restore && blockIdx.x == 0 && threadIdx.x == 0) {
    st->rho_true = st->rho_best;
    st->relres_true = st->bnorm2 > 0.0 ? sqrt(st->rho_best / st->bnorm2) : sqrt(st->rho_best);
  }
}

// x = xh + xl with xh = fl32(x), xl = fl32(x - xh): the float32 pair the
// compensated residual kernel multiplies with the float32 operator.
__global__ void __launch_bounds__(256) k_split_x(Ws w, int skip_if_done) {
  if (skip_if_done && w.st->done) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x) {
    const double x = w.xd[i];
    const float hi = float(x);
    w.xh[i] = hi;
    w.xl[i] = float(x - double(hi));
  }
}

cudaError_t launch_split_x(const Ws& w, int grid, int skip_if_done, cudaStream_t s) {
  k_split_x<<<grid, 256, 0, s>>>(w, skip_if_done);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Ws& w, int grid, cudaStream_t s) {
  k_finalize<<<grid, 256, 0, s>>>(w);
  return cudaGetLastError();
}

}  // namespace dcg
