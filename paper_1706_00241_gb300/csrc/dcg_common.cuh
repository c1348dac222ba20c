// Shared device-side definitions of the deflated-CG library: the per-context
// device state, bounded mbarrier/TMA helpers (inline PTX for sm_103a) and
// block reductions. Host orchestration lives in dcg_api.cu.
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "dcg.h"  // include/ is on the include path

namespace dcg {

constexpr int kMaxK = 96;         // deflation vectors (columns of W)
constexpr int kMaxEll = 128;      // stored directions
constexpr int kMaxM = kMaxK + kMaxEll;  // 224: the float32 m x m reduced pencil fits in 200 KB of shared memory
constexpr int kMaxBlockCols = 129;  // columns of one multi-vector product
constexpr int kReduceSlots = 3 * kMaxK + 8;  // per-CTA partial sums of one reduction
constexpr long long kSpinLimit = 1ll << 22;  // bounded waits: polls before giving up

// Ticket counters for the "last CTA finishes the reduction" pattern, one per
// reduction site so that consecutive kernels never share a counter.
enum Ticket : int {
  T_MATVEC = 0, T_SETUP_G, T_SETUP_H, T_PHASE1, T_CHECK_RES, T_CHECK_G, T_CHECK_H,
  T_FINAL, T_GALERKIN, T_COUNT
};

// Device-resident solver state. Written only by kernels (and once per solve
// by the host, before the graph launch).
struct DevState {
  double rho;        // r^T r of the current residual
  double rho_new;    // r^T r after the x, r update of this iteration
  double d;          // p^T A p of the current direction (Algorithm 1)
  double alpha;
  double beta;
  double bnorm2;     // |b|^2
  double thresh2;    // (tol |b|)^2
  double rho_true;   // |b - A x|^2 of the last true-residual evaluation
  double relres_true;
  int iter;          // completed iterations
  int max_iter;
  int status;        // dcg_status
  int done;          // 1 once the loop must stop
  int mode;          // 0 none, 1 convergence check, 2 periodic refinement
  int refine_every;
  int k;             // active deflation vectors this solve
  int ell;
  int window;        // dcg_window
  int nstored;       // directions stored in this solve (<= ell)
  int head;          // next ring slot (window LAST)
  int matvecs_check;
  int reproject;
  int hist_on;
  int hist_cap;
  int true_valid;    // relres_true describes the final x
  int warm_start;
  int zero_rhs;
  int timeout_site;  // nonzero: which bounded wait gave up
  int stall;         // consecutive true-residual checks without progress
  int save_best;     // 1: the check-update kernel copies x to the best iterate
  double rho_best;   // smallest true |r|^2 seen by a check (0: none yet)
  double rho_prev_chk;  // true |r|^2 of the previous check
  unsigned int ticket[T_COUNT];
  unsigned long long bar_count;  // grid barrier of the fused iteration kernel: arrivals in this solve
  // Failure-handling test hook (dcg_debug_arm_barrier_timeout), zero otherwise:
  // CTA 0 withholds its arrival at the fused kernel's grid barrier and every
  // CTA gives up after spin_limit polls.
  int test_skip_arrival;
  long long spin_limit;
  // residual replacements inside the loop (reading R13): the iteration index
  // of the first and of the last in this solve, 0 if none. The sparse F, G
  // of Sec. 2.3 hold only while no replacement falls inside the window.
  int repl_first, repl_last;
};

// --------------------------------------------------------------------------
// Reductions
// --------------------------------------------------------------------------

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Column sums of 32 per-lane values across a warp (reduce-scatter by
// halving): afterwards lane l holds in v[0] the warp's sum of column l.
__device__ __forceinline__ void warp_transpose_sum(float (&v)[32], int lane) {
#pragma unroll
  for (int s = 16; s >= 1; s >>= 1) {
    const bool up = (lane & s) != 0;
#pragma unroll
    for (int i = 0; i < s; ++i) {
      const float send = up ? v[i] : v[i + s];
      const float keep = up ? v[i + s] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, s);
    }
  }
}

// Last-CTA detection: every CTA calls this after writing its partials with a
// __threadfence(); exactly one CTA (the last to arrive) gets true and resets
// the counter for the next launch. No CTA waits on another.
__device__ __forceinline__ bool arrive_last(unsigned int* counter) {
  __shared__ unsigned int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    unsigned int prev = atomicAdd(counter, 1u);
    s_last = (prev == gridDim.x * gridDim.y * gridDim.z - 1) ? 1u : 0u;
    if (s_last) *counter = 0u;
  }
  __syncthreads();
  if (s_last) __threadfence();
  return s_last != 0;
}

// Progress of the true residual over the checks of a solve (mode 1: the
// recursive residual met tol but the true one did not; mode 2: periodic
// replacement). The iterate with the smallest true residual is kept
// (save_best asks the check-update kernel to copy x). A check is a stall if it
// does not halve the best true residual and either is a failed convergence
// check or shows a true residual that rose since the previous check.
// kStallChecks consecutive stalls end the solve with DCG_ERR_STAGNATION (tol
// lies below the accuracy the iteration reaches, and iterating on lets the
// iterate drift); the solve then returns the best iterate.
constexpr int kStallChecks = 8;
__device__ __forceinline__ void note_check(DevState* st, double rho_true, int mode) {
  const bool first = st->rho_best == 0.0;
  const bool halved = first || rho_true < 0.25 * st->rho_best;
  if (first || rho_true < st->rho_best) {
    st->rho_best = rho_true;
    st->save_best = 1;
  }
  if (halved) {
    st->stall = 0;
  } else if (mode == 1 || rho_true > st->rho_prev_chk) {
    if (++st->stall >= kStallChecks) {
      st->status = DCG_ERR_STAGNATION;
      st->done = 1;
    }
  }
  st->rho_prev_chk = rho_true;
}

// Nearest TF32 value of a finite float32 (ties to even at 10 mantissa bits):
// the element format of kind::tf32 tensor-core operands.
__device__ __forceinline__ float round_tf32(float x) {
  uint32_t u = __float_as_uint(x);
  const uint32_t lsb = (u >> 13) & 1u;
  u = (u + 0xFFFu + lsb) & 0xFFFFE000u;
  return __uint_as_float(u);
}

// --------------------------------------------------------------------------
// mbarrier and TMA (bulk tensor copy) helpers, sm_90+ PTX used on sm_103a
// --------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbarrier_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t phase) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Waits for the given phase parity; gives up after kSpinLimit polls and
// returns false (the caller records a timeout and leaves).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t phase) {
  for (long long i = 0; i < kSpinLimit; ++i)
    if (mbar_try_wait(bar, phase)) return true;
  return false;
}

// L2 cache policy for data read once per launch (the stored operator): its
// lines are evicted first, so streaming a 1 GiB matrix through the 129 MB L2
// does not displace the few MB the iteration kernels reuse (x, r, p, q, W, AW,
// the k x k matrices).
__device__ __forceinline__ uint64_t l2_policy_evict_first() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}

// As tma_load_2d, with an L2 cache policy (l2_policy_evict_first).
__device__ __forceinline__ void tma_load_2d_hint(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int x0,
                                                 int y0, uint64_t pol) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1, {%3, "
      "%4}], [%2], %5;" ::"r"(smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x0), "r"(y0), "l"(pol)
      : "memory");
}

// 2-D tiled TMA load of box {x, y} at coordinates (x0, y0) into shared memory,
// completing on an mbarrier. x0 * sizeof(elem) must be a multiple of 16 bytes.
__device__ __forceinline__ void tma_load_2d(void* smem_dst, const CUtensorMap* map, uint64_t* bar, int x0,
                                            int y0) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cta.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::"r"(
          smem_u32(smem_dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(x0), "r"(y0)
      : "memory");
}

__device__ __forceinline__ void prefetch_tensormap(const CUtensorMap* map) {
  asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

// --------------------------------------------------------------------------
// Small float64 helpers shared by the iteration kernels
// --------------------------------------------------------------------------

// y = L^{-T} (L^{-1} h) with Linv the lower-triangular inverse Cholesky factor
// of E (k x k, row-major). Run by one warp; h, y in shared memory; k <= kMaxK.
__device__ __forceinline__ void apply_Einv_warp(const double* __restrict__ Linv, int k, const double* h,
                                                double* tmp, double* y) {
  const int lane = threadIdx.x & 31;
  for (int i = lane; i < k; i += 32) {  // tmp = Linv h
    double s = 0.0;
    for (int j = 0; j <= i; ++j) s = fma(Linv[i * k + j], h[j], s);
    tmp[i] = s;
  }
  __syncwarp();
  for (int i = lane; i < k; i += 32) {  // y = Linv^T tmp
    double s = 0.0;
    for (int j = i; j < k; ++j) s = fma(Linv[j * k + i], tmp[j], s);
    y[i] = s;
  }
  __syncwarp();
}

}  // namespace dcg
