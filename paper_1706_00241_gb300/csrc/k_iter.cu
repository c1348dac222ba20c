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

// Dot products of k columns (column c at cols + c n) with a band vector held in
// shared memory; warp w takes columns w, w + nwarps, ...; writes float64
// partials out[c].
__device__ void band_col_dots(const float* __restrict__ cols, int k, int n, int i0, int len, const float* vs,
                              double* out) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = warp; c < k; c += nw) {
    const float* col = cols + int64_t(c) * n + i0;
    float s = 0.f;
    for (int i = lane; i < len; i += 32) s = fmaf(__ldg(col + i), vs[i], s);
    s = warp_sum(s);
    if (lane == 0) out[c] = double(s);
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

// Last CTA: sums `count` float64 partial columns over all CTAs into dst.
__device__ void reduce_partials(const double* partials, int stride, int count, double* dst) {
  const int G = gridDim.x;
  for (int c = threadIdx.x; c < count; c += blockDim.x) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += partials[int64_t(b) * stride + c];
    dst[c] = s;
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// r_{-1} = b - A x_{-1} (A x_{-1} from the start-of-solve product, or 0 for a
// cold start); |b|^2 and the stopping threshold (reading R2: tol relative to |b|).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_setup_r(Ws w) {
  DevState* st = w.st;
  const int n = w.n;
  const int warm = st->warm_start;
  float acc = 0.f;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const float bi = w.b[i];
    w.r[i] = warm ? bi - w.Y[i] : bi;
    acc = fmaf(bi, bi, acc);
  }
  const float s = block_sum(acc);
  if (threadIdx.x == 0) w.partials[blockIdx.x * kReduceSlots] = double(s);
  if (!arrive_last(&st->ticket[T_SETUP_G])) return;
  __shared__ double tot;
  reduce_partials(w.partials, kReduceSlots, 1, &tot);
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
  double* part = w.partials + int64_t(blockIdx.x) * kReduceSlots;
  band_col_dots(w.XW + n, k, n, i0, len, sh, part);
  if (!arrive_last(&st->ticket[T_CHECK_G])) return;
  __shared__ double g[kMaxK], tmp[kMaxK], y[kMaxK];
  reduce_partials(w.partials, kReduceSlots, k, g);
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
//   in loop:  beta = rho_new / rho and mu = E^{-1}(h + beta hp), which
//             re-projects p_{j+1} against W after the replacement (R13).
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
  float acc = 0.f;
  for (int i = threadIdx.x; i < len; i += blockDim.x) {
    const int gi = i0 + i;
    float xi = w.XW[gi], ri = w.r[gi];
    for (int c = 0; c < k; ++c) {
      const float g = gsh[c];
      xi = fmaf(w.XW[int64_t(c + 1) * n + gi], g, xi);
      ri = fmaf(-w.Y[int64_t(c + 1) * n + gi], g, ri);
    }
    if (k) {
      w.XW[gi] = xi;
      w.r[gi] = ri;
    }
    rs[i] = ri;
    ps[i] = w.p[gi];
    acc = fmaf(ri, ri, acc);
  }
  const float rho_part = block_sum(acc);
  double* part = w.partials + int64_t(blockIdx.x) * kReduceSlots;
  if (threadIdx.x == 0) part[0] = double(rho_part);
  band_col_dots(w.Y + n, k, n, i0, len, rs, part + 1);
  if (!setup && !pre_loop) band_col_dots(w.Y + n, k, n, i0, len, ps, part + 1 + k);
  if (!arrive_last(&st->ticket[setup ? T_SETUP_H : T_CHECK_H])) return;

  __shared__ double red[1 + 2 * kMaxK], tmp[kMaxK], y[kMaxK];
  reduce_partials(w.partials, kReduceSlots, (setup || pre_loop) ? 1 + k : 1 + 2 * k, red);
  const double rho_new = red[0];
  __shared__ double s_beta;
  if (threadIdx.x == 0) {
    if (setup) {
      s_beta = 0.0;
    } else {
      s_beta = st->rho > 0.0 ? rho_new / st->rho : 0.0;
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
  if (threadIdx.x == 0) {
    st->rho = rho_new;
    st->rho_new = rho_new;
    if (k) st->true_valid = 0;
    if (setup) {
      st->beta = 0.0;
      if (st->hist_on && st->hist_cap > 0) w.hist[0] = sqrt(rho_new / st->bnorm2);
      const int arm = rho_new <= st->thresh2 ? 1 : 0;
      st->mode = arm;
      cudaGraphSetConditional(hd.pre, arm);
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
//   rho' = r^T r, h = (AW)^T r [, hp = (AW)^T p];
// last CTA: beta = rho' / rho, mu = E^{-1} h (line 11, reading R1), the
// convergence / refinement decision and the IF-node value for the check branch.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_phase1(Ws w, Handles hd) {
  DevState* st = w.st;
  if (st->done) return;
  extern __shared__ float sh[];
  const int n = w.n, k = st->k;
  const double d = st->d;
  const bool ok = (d > 0.0) && isfinite(d);
  const float alpha = ok ? float(st->rho / d) : 0.f;
  int slot = -1;
  if (st->ell > 0) {
    if (st->window == DCG_WINDOW_FIRST) {
      if (st->iter < st->ell) slot = st->iter;
    } else {
      slot = st->head;
    }
  }
  const int reproj = st->reproject;
  int i0, i1;
  band_of(n, i0, i1);
  const int len = i1 - i0;
  float* rs = sh;
  float* ps = sh + len;
  float acc = 0.f;
  if (ok) {
    for (int i = threadIdx.x; i < len; i += blockDim.x) {
      const int gi = i0 + i;
      const float pi = w.p[gi], qi = w.q[gi];
      const float xi = fmaf(alpha, pi, w.XW[gi]);
      const float ri = fmaf(-alpha, qi, w.r[gi]);
      w.XW[gi] = xi;
      w.r[gi] = ri;
      if (slot >= 0) {
        w.P[int64_t(slot) * n + gi] = pi;
        w.Q[int64_t(slot) * n + gi] = qi;
      }
      rs[i] = ri;
      ps[i] = pi;
      acc = fmaf(ri, ri, acc);
    }
  }
  const float rho_part = block_sum(acc);
  double* part = w.partials + int64_t(blockIdx.x) * kReduceSlots;
  if (threadIdx.x == 0) part[0] = double(rho_part);
  if (ok) {
    band_col_dots(w.Y + n, k, n, i0, len, rs, part + 1);
    if (reproj) band_col_dots(w.Y + n, k, n, i0, len, ps, part + 1 + k);
  }
  if (!arrive_last(&st->ticket[T_PHASE1])) return;

  __shared__ double red[1 + 2 * kMaxK], tmp[kMaxK], y[kMaxK];
  __shared__ int s_mode;
  __shared__ double s_beta;
  if (!ok) {
    if (threadIdx.x == 0) {
      st->status = DCG_ERR_BREAKDOWN;
      st->done = 1;
      cudaGraphSetConditional(hd.chk, 0);
    }
    return;
  }
  reduce_partials(w.partials, kReduceSlots, reproj ? 1 + 2 * k : 1 + k, red);
  if (threadIdx.x == 0) {
    const double rho_new = red[0];
    const int iter = st->iter + 1;
    st->iter = iter;
    st->alpha = double(alpha);
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
    cudaGraphSetConditional(hd.chk, mode != 0 ? 1 : 0);
  }
  __syncthreads();
  if (s_mode != 0) return;  // beta and mu follow the replaced residual
  if (reproj) {
    const double beta = s_beta;
    for (int c = threadIdx.x; c < k; c += blockDim.x) red[1 + c] += beta * red[1 + k + c];
    __syncthreads();
  }
  if (threadIdx.x < 32) apply_Einv_warp(w.Linv, k, red + 1, tmp, y);
  __syncthreads();
  for (int c = threadIdx.x; c < k; c += blockDim.x) {
    w.mu[c] = y[c];
    w.mu_f[c] = float(y[c]);
  }
}

cudaError_t launch_phase1(const Ws& w, int grid, Handles h, cudaStream_t s) {
  const int band = (w.n + grid - 1) / grid + 1;
  k_phase1<<<grid, 256, size_t(2 * band) * sizeof(float), s>>>(w, h);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Phase 2 (line 12): p = beta p + r - W mu. In the loop body it also ends the
// while node once the solve is done.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_phase2(Ws w, Handles hd, int set_loop) {
  DevState* st = w.st;
  if (st->done) {
    if (set_loop && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hd.loop, 0);
    return;
  }
  const int n = w.n, k = st->k;
  __shared__ float msh[kMaxK];
  for (int c = threadIdx.x; c < k; c += blockDim.x) msh[c] = w.mu_f[c];
  __syncthreads();
  const float beta = float(st->beta);
  int i0, i1;
  band_of(n, i0, i1);
  for (int gi = i0 + threadIdx.x; gi < i1; gi += blockDim.x) {
    float s = fmaf(beta, w.p[gi], w.r[gi]);
    for (int c = 0; c < k; ++c) s = fmaf(-w.XW[int64_t(c + 1) * n + gi], msh[c], s);
    w.p[gi] = s;
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
  if (w.st->done) cudaGraphSetConditional(hd.loop, 0);
}

cudaError_t launch_loop_gate(const Ws& w, Handles h, cudaStream_t s) {
  k_loop_gate<<<1, 1, 0, s>>>(w, h);
  return cudaGetLastError();
}

__global__ void k_final_gate(Ws w, Handles hd) {
  const DevState* st = w.st;
  cudaGraphSetConditional(hd.fin, (!st->true_valid && !st->zero_rhs) ? 1 : 0);
}

cudaError_t launch_final_gate(const Ws& w, Handles h, cudaStream_t s) {
  k_final_gate<<<1, 1, 0, s>>>(w, h);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_finalize(Ws w) {
  if (!w.st->zero_rhs) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < w.n; i += gridDim.x * blockDim.x) w.XW[i] = 0.f;
}

cudaError_t launch_finalize(const Ws& w, int grid, cudaStream_t s) {
  k_finalize<<<grid, 256, 0, s>>>(w);
  return cudaGetLastError();
}

}  // namespace dcg
