// Per-iteration kernels of Deflated-CG (Algorithm 1, Sec. 2.2).
//
// Each kernel owns a contiguous band of rows per CTA. Reductions are two-level:
// float32 sums inside a CTA, float64 partials across CTAs, summed in a fixed
// order by the last CTA to arrive (no CTA waits on another). The last CTA also
// does the small float64 work that needs the full sums (alpha, beta, the k x k
// solve for mu or gamma) and the control decisions of the solve graph.
#include "dcg_kernels.cuh"
#include "tc.cuh"

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
// g = W^T r, then (last CTA) gamma = E^{-1} g: the correction of the initial
// projection of Algorithm 1 (and of the re-deflation after a residual
// replacement, reading R13).
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
// x += W gamma, r -= (AW) gamma (initial projection / reading R13), then rho = r^T r,
// h = (AW)^T r, hp = (AW)^T p. The last CTA finishes according to the place of
// the kernel in the solve graph:
//   setup:    mu_0 = E^{-1} h (first direction), beta = 0, arms the pre-loop check if
//             |r_0| <= tol |b|;
//   pre_loop: after a failed initial check only rho is refreshed;
//   in loop:  beta = rho_rec / rho from the recursion's own |r_{j+1}|^2
//             (st->rho_new, written by the fused iteration kernel), rho = |r_true|^2 after the
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
  // (AW)^T r of the residual the next direction starts from (sparse F, G)
  if (w.fg) {
    double* hprev = fg_hprev(w.fg, w.ellmax, w.kmax);
    for (int c = threadIdx.x; c < k; c += blockDim.x) hprev[c] = red[1 + c];
  }
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
      if (!pre_loop) {
        if (st->repl_first == 0) st->repl_first = st->iter;
        st->repl_last = st->iter;
      }
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
// Float32 re-deflation: in exact arithmetic W^T r_j = 0 for all j (Eq. 5), so
// gamma = E^{-1} W^T r is zero. In float32 the rounding of mu leaves p slightly
// A-non-conjugate to W, and r then drifts along W by ~eps32 * lambda(W) per
// step; CG never removes that drift and the recursive residual stalls. Every
// iteration therefore applies x += W gamma, r -= AW gamma (a no-op in exact
// arithmetic). With r~ = r - AW gamma:
//   |r~|^2 = rho' - 2 gamma^T h + gamma^T G_W gamma,   G_W = (AW)^T AW,
//   mu = E^{-1} ((AW)^T r~ + beta hp) = E^{-1} h - M g + beta E^{-1} hp,
// with E^{-1}, N = G_W E^{-1} and M = E^{-1} N formed once per solve.
// ---------------------------------------------------------------------------

// Grid barrier for a cooperative launch (all CTAs co-resident): one 64-bit
// arrival counter that only grows within a solve (the solver state is zeroed
// at the start of every solve). After the block barrier, thread 0 of each CTA
// adds 1 with release semantics; its barrier completes when the counter
// reaches the next multiple of gridDim.x above its ticket, which it polls with
// acquire loads (bounded wait). Returns false if the wait gave up (the kernel
// then records a timeout). With the state's test hook armed, CTA 0 reads the
// counter instead of adding to it, so that no CTA's wait can complete, and the
// wait gives up after st->spin_limit polls.
__device__ bool grid_barrier(DevState* st) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long* cnt = &st->bar_count;
    unsigned long long ticket;
    const bool withhold = st->test_skip_arrival != 0 && blockIdx.x == 0;
    const long long limit = st->spin_limit > 0 ? st->spin_limit : kSpinLimit;
    if (withhold)
      asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(ticket) : "l"(cnt) : "memory");
    else
      asm volatile("atom.add.release.gpu.u64 %0, [%1], 1;" : "=l"(ticket) : "l"(cnt) : "memory");
    const unsigned long long target = (ticket / gridDim.x + 1) * gridDim.x;
    int ok = 1;
    long long i = 0;
    for (;;) {
      unsigned long long v;
      asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(v) : "l"(cnt) : "memory");
      if (v >= target) break;
      __nanosleep(32);
      if (++i >= limit) {
        ok = 0;
        break;
      }
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

constexpr int IT_THREADS = 256;
constexpr int IT_WARPS = IT_THREADS / 32;
constexpr int IT_ROWS = IT_THREADS / 2;  // rows per CTA pass: the two halves of a CTA split the columns
constexpr int IT_MAX_PASSES = 32;         // row passes per CTA (n <= 32 * 128 * grid)
constexpr int IT_RED_U = 13;              // partial sums each warp reduces per round

// One iteration of Algorithm 1 after q = A p, with its direction store, as one
// cooperative launch with one CTA per SM. A CTA owns rows
// b * 128 + i + j * 128 * grid (i < 128); threads t and t + 128 share row i and
// split every 32-column block of W and AW into halves of 16 columns:
//   A. x += alpha p, r -= alpha q, store (p, q) in the window, rho' = r^T r
//      (first half); then per-CTA partials of h = (AW)^T r, g = W^T r
//      [, hp = (AW)^T p] (each half its 16 columns, warp transpose sums);
//   grid barrier;
//   B. every CTA reduces all partials in the same fixed order (the values of
//      a warp step through the shuffle tree together) and forms
//      gamma = E^{-1} g, a = E^{-1} h - M g, b = E^{-1} hp and u = N g (E^{-1}
//      and M symmetric, N read through its transpose, so every read is
//      coalesced): warp 0 takes gamma, u and the correction gamma^T (u - 2 h)
//      to rho', one lane per output, then the mode (convergence check,
//      periodic replacement, or neither) and beta, while the other warps form
//      a and b with two lanes per output. CTA 0 alone writes the solver state
//      and the IF-node value of the check branch;
//   C. if no check follows, every CTA applies the direction update to its rows:
//      x += W gamma, r -= AW gamma, p = beta p + r - W mu, mu = a + beta b
//      (each half sums its columns; the second half hands its sums to the
//      first through shared memory).
// Every CTA reads the state it needs before the barrier, so CTA 0's writes
// after it cannot race with them. Float32 re-deflation (gamma): see the
// note above.
// Double-float arithmetic on float32 pairs (hi, lo), |lo| <= ulp(hi) / 2, for
// the per-iteration reductions and k x k products: float64 on GB300 issues at
// ~1/64 of the float32 rate, so a warp-wide float64 instruction occupies the
// pipe ~17 cycles; the pairs keep ~44 bits on the float32 pipe. TwoSum and the
// FMA-exact product are the standard error-free transformations (Knuth;
// Dekker; Ogita, Rump & Oishi 2005).
struct df {
  float hi, lo;
};
__device__ __forceinline__ df df_add(df a, df b) {
  const float s = __fadd_rn(a.hi, b.hi);
  const float v = __fsub_rn(s, a.hi);
  float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, v)), __fsub_rn(b.hi, v));
  e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
  const float h = __fadd_rn(s, e);
  return {h, __fsub_rn(e, __fsub_rn(h, s))};
}
// acc + x * y
__device__ __forceinline__ df df_fma(df acc, float2 x, df y) {
  const float p = __fmul_rn(x.x, y.hi);
  float pe = __fmaf_rn(x.x, y.hi, -p);
  pe = __fmaf_rn(x.x, y.lo, pe);
  pe = __fmaf_rn(x.y, y.hi, pe);
  return df_add(acc, df{p, pe});
}
// a * b (FMA-exact product of the high parts, cross terms in float32)
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float hh = __fadd_rn(p, e);
  return {hh, __fsub_rn(e, __fsub_rn(hh, p))};
}
__device__ __forceinline__ df df_shfl_xor(df a, int m) {
  return {__shfl_xor_sync(0xffffffffu, a.hi, m), __shfl_xor_sync(0xffffffffu, a.lo, m)};
}
__device__ __forceinline__ double df_to_double(df a) { return double(a.hi) + double(a.lo); }

constexpr int IT_MAX_GRID = 160;   // the unrolled partial reduction covers <= 160 CTAs
constexpr int IT_STAGE_KMAX = 64;  // E^{-1}, M, N^T staged in shared memory up to this k

__host__ __device__ constexpr uint32_t it_mat_bytes(int k) { return uint32_t((3 * k * k * 8 + 15) & ~15); }

// Column sums of 16 per-lane values across a warp: afterwards lanes l and
// l + 16 hold in v[0] the warp's sum of column l (l < 16).
__device__ __forceinline__ void warp_transpose_sum16(float (&v)[16], int lane) {
#pragma unroll
  for (int s = 8; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
  v[0] += __shfl_xor_sync(0xffffffffu, v[0], 16);
}

__global__ void __launch_bounds__(IT_THREADS) k_iter_fused(Ws w, Handles hd, int stage) {
  DevState* st = w.st;
  if (st->done) {
    if (hd.loop && blockIdx.x == 0 && threadIdx.x == 0) cudaGraphSetConditional(hd.loop, 0);
    return;
  }
  const int n = w.n, k = st->k;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int half = t / IT_ROWS, rt = t % IT_ROWS;  // column half, row slot
  const double d = st->d;
  const bool ok = (d > 0.0) && isfinite(d);
  const double rho_old = st->rho;
  const double alpha_d = ok ? rho_old / d : 0.0;
  const float alpha = float(alpha_d);
  // 1 / rho_old for beta, formed early by the one thread that needs it
  const double inv_rho_old = t == 0 ? 1.0 / rho_old : 0.0;
  const int iter = st->iter + 1;
  const int ell = st->ell, window = st->window, head = st->head, nstored = st->nstored;
  const double thresh2 = st->thresh2, bnorm2 = st->bnorm2;
  const int refine_every = st->refine_every, max_iter = st->max_iter;
  const int hist_on = st->hist_on, hist_cap = st->hist_cap;
  const int reproj = st->reproject;
  int slot = -1;
  if (ell > 0) {
    if (window == DCG_WINDOW_FIRST) {
      if (iter - 1 < ell) slot = iter - 1;
    } else {
      slot = head;
    }
  }
  if (!ok) {  // breakdown: every CTA sees the same d
    if (blockIdx.x == 0 && t == 0) {
      st->status = DCG_ERR_BREAKDOWN;
      st->done = 1;
      if (hd.chk) cudaGraphSetConditional(hd.chk, 0);
      if (hd.loop) cudaGraphSetConditional(hd.loop, 0);
    }
    return;
  }
  // E^{-1}, M and N^T (read by phase B) arrive in shared memory by bulk copies
  // while phase A runs
  extern __shared__ __align__(16) float2 smat[];
  __shared__ __align__(8) uint64_t mat_bar;
  const bool staged = stage && k > 0 && k <= IT_STAGE_KMAX;
  const uint32_t mbytes = it_mat_bytes(k);
  if (staged && t == 0) {
    mbar_init(&mat_bar, 1);
    fence_mbarrier_init();
    mbar_arrive_expect_tx(&mat_bar, mbytes);
    tc::bulk_load(smat, w.mats2, mbytes, &mat_bar);
  }
  const int G = gridDim.x;
  const int stride = G * IT_ROWS;
  const int row0 = blockIdx.x * IT_ROWS + rt;
  // (AW)^T r of the residual this iteration starts from, for the record of
  // the stored direction (sparse F, G): loaded now, used after the barrier
  const bool record = blockIdx.x == 0 && slot >= 0 && w.fg != nullptr;
  __shared__ double s_hprev[kMaxK];
  if (record)
    for (int c = t; c < k; c += IT_THREADS) s_hprev[c] = fg_hprev(w.fg, w.ellmax, w.kmax)[c];

  // ---- A. x, r update, window store, rho' ----
  float acc = 0.f;
  if (half == 0) {
    for (int gi = row0; gi < n; gi += stride) {
      const float pi = w.p[gi], qi = w.q[gi];
      w.xd[gi] += alpha_d * double(pi);
      const float ri = fmaf(-alpha, qi, w.r[gi]);
      w.r[gi] = ri;
      if (slot >= 0) {
        w.P[int64_t(slot) * n + gi] = pi;
        w.Q[int64_t(slot) * n + gi] = qi;
      }
      acc = fmaf(ri, ri, acc);
    }
  }
  // per-warp column sums of the dots; warp 4 h + j (half h) writes slot j
  __shared__ float wsum[IT_WARPS / 2][1 + 3 * kMaxK];
  const int wj = warp % (IT_WARPS / 2);
  if (half == 0) {
    const float rs = warp_sum(acc);
    if (lane == 0) wsum[wj][0] = rs;
  }
  __syncthreads();  // r' of this CTA's rows, written by the first half, read by both
  for (int c0 = 0; c0 < k; c0 += 32) {
    const int cb = c0 + 16 * half;
    const int cw = min(16, k - cb);  // warp-uniform
    if (cw <= 0) continue;
    float vh[16], vg[16], vp[16];
#pragma unroll
    for (int c = 0; c < 16; ++c) vh[c] = vg[c] = vp[c] = 0.f;
    for (int gi = row0; gi < n; gi += stride) {
      const float ri = w.r[gi], pi = w.p[gi];
      const float* aw = w.Y + int64_t(1 + cb) * n + gi;
      const float* ww = w.XW + int64_t(1 + cb) * n + gi;
      float av_[16], wv_[16];
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        av_[c] = c < cw ? __ldg(aw + int64_t(c) * n) : 0.f;
        wv_[c] = c < cw ? __ldg(ww + int64_t(c) * n) : 0.f;
      }
#pragma unroll
      for (int c = 0; c < 16; ++c) {
        vh[c] = fmaf(av_[c], ri, vh[c]);
        vp[c] = fmaf(av_[c], pi, vp[c]);
        vg[c] = fmaf(wv_[c], ri, vg[c]);
      }
    }
    warp_transpose_sum16(vh, lane);
    warp_transpose_sum16(vg, lane);
    if (reproj) warp_transpose_sum16(vp, lane);
    if (lane < cw) {
      wsum[wj][1 + cb + lane] = vh[0];
      wsum[wj][1 + k + cb + lane] = vg[0];
      if (reproj) wsum[wj][1 + 2 * k + cb + lane] = vp[0];
    }
  }
  __syncthreads();
  const int nd = reproj ? 3 : 2;  // h, g [, hp]
  const int count = 1 + nd * k;
  float* partf = reinterpret_cast<float*>(w.partials);  // float slots [v * G + b]
  for (int v = t; v < count; v += IT_THREADS) {
    float sum = 0.f;
#pragma unroll
    for (int q = 0; q < IT_WARPS / 2; ++q) sum += wsum[q][v];
    partf[int64_t(v) * G + blockIdx.x] = sum;
  }
  if (!grid_barrier(st)) {
    if (t == 0) {
      // the bulk copy of the k x k matrices may still be landing in shared
      // memory: wait for it (bounded) before the CTA leaves
      if (staged) mbar_wait_bounded(&mat_bar, 0);
      st->status = DCG_ERR_TIMEOUT;
      st->timeout_site = 4;
      st->done = 1;
      if (hd.chk) cudaGraphSetConditional(hd.chk, 0);
      if (hd.loop) cudaGraphSetConditional(hd.loop, 0);
    }
    return;
  }

  // ---- B. the same reduction and k x k products in every CTA ----
  // warp w reduces values w * 13 .. w * 13 + 12 of each round of 104, all
  // their loads in flight at once
  __shared__ df sred[1 + 3 * kMaxK];
  __shared__ double gam[kMaxK], av[kMaxK], bv[kMaxK], uu[kMaxK];
  __shared__ int s_mode, s_done;
  __shared__ double s_beta;
  for (int v0 = warp * IT_RED_U; v0 < count; v0 += IT_WARPS * IT_RED_U) {
    float ld[IT_RED_U][IT_MAX_GRID / 32];
#pragma unroll
    for (int u = 0; u < IT_RED_U; ++u)
#pragma unroll
      for (int i = 0; i < IT_MAX_GRID / 32; ++i) {
        const int b = lane + 32 * i;
        ld[u][i] = (b < G && v0 + u < count) ? __ldcg(partf + int64_t(v0 + u) * G + b) : 0.f;
      }
    // the values' sums advance level by level together (independent chains
    // interleave instead of running one value after another)
    df sv[IT_RED_U];
#pragma unroll
    for (int u = 0; u < IT_RED_U; ++u) sv[u] = df{ld[u][0], 0.f};
#pragma unroll
    for (int i = 1; i < IT_MAX_GRID / 32; ++i)
#pragma unroll
      for (int u = 0; u < IT_RED_U; ++u) sv[u] = df_add(sv[u], df{ld[u][i], 0.f});
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1)
#pragma unroll
      for (int u = 0; u < IT_RED_U; ++u) sv[u] = df_add(sv[u], df_shfl_xor(sv[u], m));
#pragma unroll
    for (int u = 0; u < IT_RED_U; ++u)
      if (lane == 0 && v0 + u < count) sred[v0 + u] = sv[u];
  }
  __syncthreads();
  const df* h = sred + 1;
  const df* g = sred + 1 + k;
  const df* hp = sred + 1 + 2 * k;
  const float2* Ei = w.mats2;
  if (staged) {
    __shared__ int s_mat_ok;
    if (t == 0) s_mat_ok = mbar_wait_bounded(&mat_bar, 0) ? 1 : 0;
    __syncthreads();
    if (s_mat_ok) {
      Ei = smat;
    } else if (t == 0) {
      st->status = DCG_ERR_TIMEOUT;   // the copy never landed: read from global, end the solve
      st->timeout_site = 5;
      st->done = 1;
    }
  }
  const float2* Mm = Ei + k * k;
  const float2* Nt = Ei + 2 * k * k;
  // Warp 0: gamma_c = (E^{-1} g)_c, u_c = (N g)_c and the correction
  // gamma^T (u - 2 h) to rho', one lane per output (even and odd j in
  // separate sums), then straight on to the scalar tail. Warps 1..: a_c and
  // b_c, two lanes per output (warp-uniform trip count for the pair
  // shuffles). One block barrier afterwards.
  if (warp == 0) {
    df corr = {0.f, 0.f};
    for (int c = lane; c < k; c += 32) {
      df s0 = {0.f, 0.f}, s1 = {0.f, 0.f}, s2 = {0.f, 0.f}, s3 = {0.f, 0.f};
      for (int j = 0; j < k; j += 2) {
        s0 = df_fma(s0, Ei[j * k + c], g[j]);
        s1 = df_fma(s1, Nt[j * k + c], g[j]);
        if (j + 1 < k) {
          s2 = df_fma(s2, Ei[(j + 1) * k + c], g[j + 1]);
          s3 = df_fma(s3, Nt[(j + 1) * k + c], g[j + 1]);
        }
      }
      s0 = df_add(s0, s2);
      s1 = df_add(s1, s3);
      gam[c] = df_to_double(s0);
      uu[c] = df_to_double(s1);
      const df hm2 = {-2.f * h[c].hi, -2.f * h[c].lo};  // exact scaling
      corr = df_add(corr, df_mul(s0, df_add(s1, hm2)));
    }
#pragma unroll
    for (int m = 16; m >= 1; m >>= 1) corr = df_add(corr, df_shfl_xor(corr, m));
    if (lane == 0) {
      const double rho_raw = df_to_double(sred[0]);
      double rho_new = df_to_double(df_add(sred[0], corr));
      if (!(rho_new > 0.0)) rho_new = rho_raw;
      int mode = 0;
      if (rho_new <= thresh2)
        mode = 1;
      else if (refine_every > 0 && iter % refine_every == 0)
        mode = 2;
      const int done = (mode == 0 && iter >= max_iter) ? 1 : 0;
      s_mode = mode;
      s_done = done;
      s_beta = rho_new * inv_rho_old;
      if (blockIdx.x == 0) {
        st->iter = iter;
        st->alpha = alpha_d;
        if (ell > 0) {
          if (window == DCG_WINDOW_FIRST) {
            st->nstored = min(iter, ell);
          } else {
            st->head = (head + 1) % ell;
            st->nstored = min(nstored + 1, ell);
          }
        }
        if (hist_on && iter < hist_cap) w.hist[iter] = sqrt(rho_new / bnorm2);
        st->rho_new = rho_new;
        st->true_valid = 0;
        st->mode = mode;
        if (mode == 0) {
          st->beta = s_beta;
          st->rho = rho_new;
          if (done) {
            st->status = DCG_ERR_MAXITER;
            st->done = 1;
          }
        }
        if (hd.chk) cudaGraphSetConditional(hd.chk, mode != 0 ? 1 : 0);
        if (done && hd.loop) cudaGraphSetConditional(hd.loop, 0);
      }
    }
  } else {
    for (int ob = (warp - 1) * 32; ob < 4 * k; ob += (IT_WARPS - 1) * 32) {
      const int o2 = ob + lane;
      const bool act = o2 < 4 * k;
      const int o = o2 >> 1, par = o2 & 1;
      const int which = act ? o / k : 2, c = act ? o - which * k : 0;
      df s0 = {0.f, 0.f}, s1 = {0.f, 0.f}, s2 = {0.f, 0.f}, s3 = {0.f, 0.f};
      if (which == 0) {
        for (int j = par; j < k; j += 4) {
          s0 = df_fma(s0, Ei[j * k + c], h[j]);
          s1 = df_fma(s1, Mm[j * k + c], g[j]);
          if (j + 2 < k) {
            s2 = df_fma(s2, Ei[(j + 2) * k + c], h[j + 2]);
            s3 = df_fma(s3, Mm[(j + 2) * k + c], g[j + 2]);
          }
        }
      } else if (which == 1 && reproj) {
        for (int j = par; j < k; j += 4) {
          s0 = df_fma(s0, Ei[j * k + c], hp[j]);
          if (j + 2 < k) s2 = df_fma(s2, Ei[(j + 2) * k + c], hp[j + 2]);
        }
      }
      s0 = df_add(s0, s2);
      s1 = df_add(s1, s3);
      s0 = df_add(s0, df_shfl_xor(s0, 1));
      s1 = df_add(s1, df_shfl_xor(s1, 1));
      if (act && par == 0) {
        if (which == 0) av[c] = df_to_double(s0) - df_to_double(s1);
        else bv[c] = df_to_double(s0);
      }
    }
  }
  __syncthreads();
  // scalars of the stored direction for the sparse F, G (Sec. 2.3); the
  // residual the next iteration starts from is r~ = r' - AW gamma, with
  // (AW)^T r~ = h - G_W gamma = h - u (a check that follows overwrites it)
  if (record) {
    double* ha = fg_ha(w.fg, w.ellmax, w.kmax, slot);
    double* hb = fg_hb(w.fg, w.ellmax, w.kmax, slot);
    double* hprev = fg_hprev(w.fg, w.ellmax, w.kmax);
    if (t == 0) {
      double* rec = w.fg + slot * FG_REC;
      rec[0] = d;
      rec[1] = alpha_d;
      rec[2] = rho_old;
      rec[3] = df_to_double(sred[0]);
      rec[4] = double(iter - 1);
    }
    for (int c = t; c < k; c += IT_THREADS) {
      const double hc = df_to_double(h[c]);
      ha[c] = s_hprev[c];
      hb[c] = hc;
      hprev[c] = hc - uu[c];
    }
  }
  if (s_mode != 0 || s_done) return;  // the check branch recomputes gamma, beta and mu

  // ---- C. the direction update on this CTA's rows ----
  __shared__ float msh[kMaxK], gsh[kMaxK];
  __shared__ float xch[3][IT_ROWS];  // second half's sums: W gamma, AW gamma, W mu
  const double beta_d = s_beta;
  for (int c = t; c < k; c += IT_THREADS) {
    msh[c] = float(av[c] + beta_d * bv[c]);
    gsh[c] = float(gam[c]);
  }
  __syncthreads();
  const float beta = float(beta_d);
  const int npass = (n - blockIdx.x * IT_ROWS + stride - 1) / stride;  // CTA-uniform
  for (int pass = 0; pass < npass; ++pass) {
    const int gi = row0 + pass * stride;
    const bool live = gi < n;
    float dx = 0.f, wm = 0.f, ra = 0.f;
    if (live) {
      for (int c0 = 16 * half; c0 < k; c0 += 32) {
        const int cw = min(16, k - c0);
        float wc[16], ac[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          wc[c] = c < cw ? __ldg(w.XW + int64_t(c0 + c + 1) * n + gi) : 0.f;
          ac[c] = c < cw ? __ldg(w.Y + int64_t(c0 + c + 1) * n + gi) : 0.f;
        }
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          if (c < cw) {
            dx = fmaf(wc[c], gsh[c0 + c], dx);
            wm = fmaf(wc[c], msh[c0 + c], wm);
            ra = fmaf(ac[c], gsh[c0 + c], ra);
          }
        }
      }
    }
    if (half == 1) {
      xch[0][rt] = dx;
      xch[1][rt] = ra;
      xch[2][rt] = wm;
    }
    __syncthreads();
    if (half == 0 && live) {
      dx += xch[0][rt];
      ra += xch[1][rt];
      wm += xch[2][rt];
      const float ri = w.r[gi] - ra;
      if (k) {
        w.xd[gi] += double(dx);
        w.r[gi] = ri;
      }
      const float pi = w.p[gi];
      w.p[gi] = (beta != 0.f ? fmaf(beta, pi, ri) : ri) - wm;
    }
    __syncthreads();
  }
}

// Largest n the fused iteration kernel covers with one co-resident CTA per SM.
int64_t iter_max_n(int num_sms) {
  return int64_t(num_sms < IT_MAX_GRID ? num_sms : IT_MAX_GRID) * IT_ROWS * IT_MAX_PASSES;
}


// Cooperative launch: the grid barrier needs every CTA resident at once (the
// grid is at most one CTA per SM for the sizes this library accepts).
static size_t iter_dyn_smem(int kmax) { return kmax <= IT_STAGE_KMAX ? size_t(it_mat_bytes(kmax)) : 0; }

// The attribute is per device, not per context: always allow the largest
// staging size, so contexts with different k never lower it for each other.
cudaError_t iter_configure() {
  return cudaFuncSetAttribute(k_iter_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(iter_dyn_smem(IT_STAGE_KMAX)));
}

cudaError_t launch_iter_fused(const Ws& w, int num_sms, Handles h, cudaStream_t s) {
  int grid = (w.n + IT_ROWS - 1) / IT_ROWS;
  if (grid > num_sms) grid = num_sms;
  if (grid > IT_MAX_GRID) grid = IT_MAX_GRID;
  if (grid < 1) grid = 1;
  if (int64_t(grid) * IT_ROWS * IT_MAX_PASSES < w.n) return cudaErrorInvalidValue;
  const size_t dyn = iter_dyn_smem(w.kmax);
  cudaLaunchConfig_t cfg{};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(IT_THREADS);
  cfg.dynamicSmemBytes = dyn;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, k_iter_fused, w, h, dyn > 0 ? 1 : 0);
}

// ---------------------------------------------------------------------------
// E^{-1} = Linv^T Linv, N = G_W E^{-1}, M = E^{-1} N (float64, k x k, once
// per solve): the small matrices the fused iteration kernel applies every
// iteration (as float pairs, staged in its shared memory). One CTA per
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
    } else if (which == 1) {  // N = G_W Einv (and its transpose, read by columns)
      for (int l = 0; l < k; ++l) s = fma(w.GW[i * k + l], w.Einv[l * k + j], s);
      w.N[i * k + j] = s;
      w.NT[j * k + i] = s;
    } else if (which == 2) {  // M = Einv N
      for (int l = 0; l < k; ++l) s = fma(w.Einv[i * k + l], w.N[l * k + j], s);
      w.M[i * k + j] = s;
    } else {                  // float pairs of Einv, M, N^T for the fused iteration kernel
      const int kk = k * k, ij = i * k + j;
      const double src[3] = {w.Einv[ij], w.M[ij], w.NT[ij]};
#pragma unroll
      for (int m = 0; m < 3; ++m) {
        const float hi = float(src[m]);
        w.mats2[m * kk + ij] = make_float2(hi, float(src[m] - double(hi)));
      }
    }
  }
}

cudaError_t launch_small_prods(const Ws& w, cudaStream_t s) {
  if (w.kmax == 0) return cudaSuccess;
  for (int which = 0; which < 4; ++which) {
    k_small_prods<<<w.kmax, 128, 0, s>>>(w, which);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// ---------------------------------------------------------------------------
// Phase 2 (the direction update): x += W gamma, r -= AW gamma (float32 re-deflation, zero
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
