// Stored-operator kernels (dense row-major float32 A):
//   * k_rowop_tma: q = A p with the fused p^T q of Algorithm 1, or the
//     true residual r = b - A x for the float64 iterate x with compensated
//     (Dot2) accumulation (the stopping test of the Sec. 3 experiments and the
//     residual replacement). A streams through a
//     shared-memory ring filled by 2-D TMA tiles (cp.async.bulk.tensor) and
//     completed on mbarriers; one CTA per SM owns a contiguous band of rows.
//   * k_apply_block: Y = A V for up to 129 columns in one pass (the start-of-
//     solve product AW of Algorithm 1).
//   * k_form_rbf: A = K + noise I for the Sec. 3 RBF kernel.
#include <algorithm>
#include <mutex>
#include <vector>

#include "dcg_kernels.cuh"
#include "tc.cuh"

namespace dcg {

// Tile geometry of the TMA row-band kernel.
constexpr int RB_ROWS = 8;                      // rows per stage (box height): 8 KB TMA boxes
constexpr int RB_BOXW = 256;                    // floats per box row (1 KB)
constexpr int RB_BOXES = 8;                     // boxes per stage
constexpr int RB_CHUNK = RB_BOXW * RB_BOXES;    // 2048 columns per stage
constexpr int RB_STAGES = 3;
constexpr int RB_STAGE_FLOATS = RB_ROWS * RB_CHUNK;
constexpr int RB_STAGE_BYTES = RB_STAGE_FLOATS * 4;  // 64 KB
constexpr int RB_CONSUMER_WARPS = 8;            // one warp per box
constexpr int RB_THREADS = (RB_CONSUMER_WARPS + 1) * 32;
constexpr size_t RB_SMEM = size_t(RB_STAGES) * RB_STAGE_BYTES + 2 * RB_STAGES * sizeof(uint64_t) + 1024;

__device__ __forceinline__ void record_timeout(DevState* st, int site) {
  if (st) {
    st->status = DCG_ERR_TIMEOUT;
    st->timeout_site = site;
    st->done = 1;
  }
}

// Compensated dot-product step (Ogita, Rump & Oishi, "Accurate sum and dot
// product", SIAM J. Sci. Comput. 26, 2005, algorithm Dot2): the product
// a * xh is split exactly into p + e with one FMA, (s, p) is summed exactly
// into s + t (Knuth's TwoSum), and the rounding terms collect in c. The low
// part xl of the float64 iterate (x = xh + xl) is added into c directly: its
// contribution is ~eps32 of the total, so float32 accuracy suffices for it.
// Explicit _rn intrinsics keep the compiler from contracting the splits.
__device__ __forceinline__ void dot2_step(float& s, float& c, float a, float xh, float xl) {
  const float p = __fmul_rn(a, xh);
  const float e = __fmaf_rn(a, xh, -p);
  const float s2 = __fadd_rn(s, p);
  const float z = __fsub_rn(s2, s);
  const float t = __fadd_rn(__fsub_rn(s, __fsub_rn(s2, z)), __fsub_rn(p, z));
  s = s2;
  c = __fadd_rn(c, __fadd_rn(t, e));
  c = __fmaf_rn(a, xl, c);
}

// (s1, c1) += (s2, c2) for compensated partial sums.
__device__ __forceinline__ void dot2_merge(float& s1, float& c1, float s2, float c2) {
  const float s = __fadd_rn(s1, s2);
  const float z = __fsub_rn(s, s1);
  const float t = __fadd_rn(__fsub_rn(s1, __fsub_rn(s, z)), __fsub_rn(s2, z));
  s1 = s;
  c1 = __fadd_rn(c1, __fadd_rn(c2, t));
}

// One CTA streams rows [RB_ROWS*g_lo, RB_ROWS*g_hi) of A. Warp w of the
// consumers owns box w of every stage (256 columns); lane l owns float4 slots
// l and l + 32 of each box row, so each thread keeps RB_ROWS accumulators
// (RB_ROWS compensated pairs for the residual).
template <bool RESID, bool COMPQ>
__global__ void __launch_bounds__(RB_THREADS, 1)
    k_rowop_tma(const __grid_constant__ CUtensorMap tmap, RowOpArgs a) {
  constexpr bool COMP = RESID || COMPQ;  // compensated (Dot2) accumulation
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* tiles = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(RB_STAGES) * RB_STAGE_BYTES);
  uint64_t* empty = full + RB_STAGES;
  __shared__ float red[RB_CONSUMER_WARPS][RB_ROWS];
  __shared__ float redc[RB_CONSUMER_WARPS][RB_ROWS];
  __shared__ int s_abort;
  __shared__ int s_issued;
  __shared__ int s_consumed[RB_CONSUMER_WARPS];
  __shared__ double s_part[RB_CONSUMER_WARPS];

  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  if (RESID && st && a.resid_mode == 0 && !st->warm_start) return;  // setup: cold start needs no A x

  const int n = a.n;
  const int ngroups = (n + RB_ROWS - 1) / RB_ROWS;
  const int G = gridDim.x, b = blockIdx.x;
  const int g_lo = int((long long)b * ngroups / G);
  const int g_hi = int((long long)(b + 1) * ngroups / G);
  const int nchunks = (n + RB_CHUNK - 1) / RB_CHUNK;
  const int total = (g_hi - g_lo) * nchunks;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

  if (threadIdx.x == 0) {
    for (int s = 0; s < RB_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], RB_CONSUMER_WARPS);
    }
    fence_mbarrier_init();
    s_abort = 0;
    s_issued = 0;
  }
  __syncthreads();

  double my_part = 0.0;  // p^T q (matvec) or |r|^2 (residual) over this CTA's rows

  if (warp == RB_CONSUMER_WARPS) {
    // ---------------- producer: one elected lane issues the TMA tiles -------
    if (lane == 0) {
      prefetch_tensormap(&tmap);
      const uint64_t pol = l2_policy_evict_first();  // A is read once per launch
      int it = 0;
      for (; it < total; ++it) {
        const int s = it % RB_STAGES;
        if (it >= RB_STAGES && !mbar_wait_bounded(&empty[s], ((it / RB_STAGES) - 1) & 1)) {
          s_abort = 1;
          break;
        }
        if (*(volatile int*)&s_abort) break;
        const int g = g_lo + it / nchunks, c = it % nchunks;
        const int nb = min(RB_BOXES, (n - c * RB_CHUNK + RB_BOXW - 1) / RB_BOXW);
        mbar_arrive_expect_tx(&full[s], uint32_t(nb) * RB_ROWS * RB_BOXW * 4);
        for (int bx = 0; bx < nb; ++bx)
          tma_load_2d_hint(tiles + size_t(s) * RB_STAGE_FLOATS + bx * RB_ROWS * RB_BOXW, &tmap, &full[s],
                           c * RB_CHUNK + bx * RB_BOXW, g * RB_ROWS, pol);
      }
      s_issued = it;
    }
  } else {
    // ---------------- consumers ---------------------------------------------
    float acc[RB_ROWS], cmp[RB_ROWS];
#pragma unroll
    for (int r = 0; r < RB_ROWS; ++r) acc[r] = cmp[r] = 0.f;
    // The vector slice of a stage (v, or the split x = xh + xl) does not depend
    // on the tile: the slice of stage it + 1 is loaded before the wait for tile
    // it, so its L2 latency overlaps the current stage.
    constexpr int VW = RESID ? 8 : 4;  // floats per slot: xh[4] xl[4], or v[4]
    auto load_vec = [&](int itv, float (&dstv)[2][VW]) {
      const int cv = itv % nchunks;
      const int c0 = cv * RB_CHUNK + warp * RB_BOXW;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int j = c0 + 4 * (lane + 32 * h);
        if (j + 3 < n) {
          if constexpr (RESID) {
            const float4 u = __ldg(reinterpret_cast<const float4*>(a.xh + j));
            const float4 l = __ldg(reinterpret_cast<const float4*>(a.xl + j));
            dstv[h][0] = u.x; dstv[h][1] = u.y; dstv[h][2] = u.z; dstv[h][3] = u.w;
            dstv[h][4] = l.x; dstv[h][5] = l.y; dstv[h][6] = l.z; dstv[h][7] = l.w;
          } else {
            const float4 v = __ldg(reinterpret_cast<const float4*>(a.v + j));
            dstv[h][0] = v.x; dstv[h][1] = v.y; dstv[h][2] = v.z; dstv[h][3] = v.w;
          }
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            if constexpr (RESID) {
              dstv[h][e] = j + e < n ? __ldg(a.xh + j + e) : 0.f;
              dstv[h][4 + e] = j + e < n ? __ldg(a.xl + j + e) : 0.f;
            } else {
              dstv[h][e] = j + e < n ? __ldg(a.v + j + e) : 0.f;
            }
          }
        }
      }
    };
    float vcur[2][VW], vnxt[2][VW];
    if (total > 0) load_vec(0, vcur);
    int it = 0;
    for (; it < total; ++it) {
      const int s = it % RB_STAGES;
      if (it + 1 < total) load_vec(it + 1, vnxt);
      if (!mbar_wait_bounded(&full[s], (it / RB_STAGES) & 1)) {
        s_abort = 1;
        break;
      }
      const int g = g_lo + it / nchunks, c = it % nchunks;
      const int col0 = c * RB_CHUNK + warp * RB_BOXW;
      if (col0 < n) {
        const float* box = tiles + size_t(s) * RB_STAGE_FLOATS + warp * RB_ROWS * RB_BOXW;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int slot = lane + 32 * h;
          if constexpr (RESID) {
#pragma unroll
            for (int r = 0; r < RB_ROWS; ++r) {
              const float4 av = reinterpret_cast<const float4*>(box + r * RB_BOXW)[slot];
              dot2_step(acc[r], cmp[r], av.x, vcur[h][0], vcur[h][4]);
              dot2_step(acc[r], cmp[r], av.y, vcur[h][1], vcur[h][5]);
              dot2_step(acc[r], cmp[r], av.z, vcur[h][2], vcur[h][6]);
              dot2_step(acc[r], cmp[r], av.w, vcur[h][3], vcur[h][7]);
            }
          } else {
#pragma unroll
            for (int r = 0; r < RB_ROWS; ++r) {
              const float4 av = reinterpret_cast<const float4*>(box + r * RB_BOXW)[slot];
              if constexpr (COMPQ) {
                dot2_step(acc[r], cmp[r], av.x, vcur[h][0], 0.f);
                dot2_step(acc[r], cmp[r], av.y, vcur[h][1], 0.f);
                dot2_step(acc[r], cmp[r], av.z, vcur[h][2], 0.f);
                dot2_step(acc[r], cmp[r], av.w, vcur[h][3], 0.f);
              } else {
                acc[r] = fmaf(av.x, vcur[h][0], acc[r]);
                acc[r] = fmaf(av.y, vcur[h][1], acc[r]);
                acc[r] = fmaf(av.z, vcur[h][2], acc[r]);
                acc[r] = fmaf(av.w, vcur[h][3], acc[r]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int e = 0; e < VW; ++e) vcur[h][e] = vnxt[h][e];
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (c == nchunks - 1) {
        // end of a row group: reduce the RB_ROWS accumulators over the CTA
#pragma unroll
        for (int r = 0; r < RB_ROWS; ++r) {
          if constexpr (COMP) {
            float sv = acc[r], cv = cmp[r];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
              const float s2 = __shfl_xor_sync(0xffffffffu, sv, o);
              const float c2 = __shfl_xor_sync(0xffffffffu, cv, o);
              dot2_merge(sv, cv, s2, c2);
            }
            if (lane == 0) {
              red[warp][r] = sv;
              redc[warp][r] = cv;
            }
          } else {
            const float v = warp_sum(acc[r]);
            if (lane == 0) red[warp][r] = v;
          }
          acc[r] = cmp[r] = 0.f;
        }
        asm volatile("bar.sync 1, %0;" ::"r"(RB_CONSUMER_WARPS * 32));
        if (threadIdx.x < RB_ROWS) {
          const int row = g * RB_ROWS + threadIdx.x;
          if (row < n) {
            if constexpr (RESID) {
              double tot = 0.0;
#pragma unroll
              for (int w = 0; w < RB_CONSUMER_WARPS; ++w)
                tot += double(red[w][threadIdx.x]) + double(redc[w][threadIdx.x]);
              const double rr = double(a.b[row]) - tot;
              a.out[row] = float(rr);
              my_part += rr * rr;
            } else if constexpr (COMPQ) {
              double tot = 0.0;
#pragma unroll
              for (int w = 0; w < RB_CONSUMER_WARPS; ++w)
                tot += double(red[w][threadIdx.x]) + double(redc[w][threadIdx.x]);
              const float qv = float(tot);
              a.out[row] = qv;
              my_part += double(a.v[row]) * double(qv);
            } else {
              float sum = 0.f;
#pragma unroll
              for (int w = 0; w < RB_CONSUMER_WARPS; ++w) sum += red[w][threadIdx.x];
              a.out[row] = sum;
              my_part += double(a.v[row]) * double(sum);
            }
          }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(RB_CONSUMER_WARPS * 32));
      }
    }
    if (lane == 0) s_consumed[warp] = it;
  }
  __syncthreads();

  // Drain: after a timeout, wait (bounded) for tiles still in flight so that no
  // TMA write lands in shared memory after this CTA has left.
  if (s_abort && threadIdx.x == 0) {
    int lo = s_issued;
    for (int w = 0; w < RB_CONSUMER_WARPS; ++w) lo = min(lo, s_consumed[w]);
    for (int it = lo; it < s_issued; ++it) mbar_wait_bounded(&full[it % RB_STAGES], (it / RB_STAGES) & 1);
    record_timeout(st, RESID ? 2 : 1);
    if (a.abort_word) atomicExch(a.abort_word, RESID ? 2 : 1);
  }
  // Without a solver state nothing else records the timeout: the rows of this
  // CTA's band are overwritten with NaN (some were never computed) and the
  // last CTA reports a NaN sum.
  if (a.abort_word) {
    __syncthreads();
    if (s_abort) {
      const float qnan = __int_as_float(0x7fc00000);
      for (int row = g_lo * RB_ROWS + int(threadIdx.x); row < min(g_hi * RB_ROWS, n); row += RB_THREADS)
        a.out[row] = qnan;
    }
  }

  // CTA partial -> last CTA sums all partials in float64 (fixed order).
  if (warp < RB_CONSUMER_WARPS) {
    double v = warp_sum(my_part);
    if (lane == 0) s_part[warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < RB_CONSUMER_WARPS; ++w) s += s_part[w];
    a.partials[b] = s;
  }
  if (!arrive_last(a.ticket)) return;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = lane; i < G; i += 32) s += a.partials[i];
    s = warp_sum(s);
    if (lane == 0) {
      if (a.abort_word && *reinterpret_cast<volatile int*>(a.abort_word) != 0) s = __longlong_as_double(0x7ff8000000000000ll);
      if (!RESID || !st) {
        if (a.result) *a.result = s;
      } else if (a.resid_mode != 0) {
        st->rho_true = s;
        st->matvecs_check += 1;
        st->relres_true = st->bnorm2 > 0.0 ? sqrt(s / st->bnorm2) : sqrt(s);
        st->true_valid = 1;
        const int mode = a.resid_mode >= 0 ? a.resid_mode : st->mode;
        if (mode == 1 && st->status == DCG_OK) {
          if (s <= st->thresh2)
            st->done = 1;
          else
            note_check(st, s, 1);
        } else if (mode == 2 && st->status == DCG_OK) {
          note_check(st, s, 2);
        }
      }
    }
  }
}

// Compensated accumulation for q = A p as well (COMPQ) was measured on GB300:
// the 11-instruction Dot2 step per element makes the kernel issue-bound
// (243 us instead of 174 us at n = 16384, 64 % of HBM) while cutting CG
// iterations by only 2 % (float32 vector rounding, not the matvec sum,
// separates float32 from float64 CG here). The plain float32 sum is used.
constexpr bool kCompensatedMatvec = false;

cudaError_t launch_rowop(const CUtensorMap* tmap, const RowOpArgs& a, bool resid, int grid, cudaStream_t s) {
  if (resid) {
    k_rowop_tma<true, false><<<grid, RB_THREADS, RB_SMEM, s>>>(*tmap, a);
  } else {
    k_rowop_tma<false, kCompensatedMatvec><<<grid, RB_THREADS, RB_SMEM, s>>>(*tmap, a);
  }
  return cudaGetLastError();
}

cudaError_t rowop_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_rowop_tma<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       int(RB_SMEM));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rowop_tma<false, kCompensatedMatvec>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(RB_SMEM));
}

int rowop_grid(int n, int num_sms) {
  const int ngroups = (n + RB_ROWS - 1) / RB_ROWS;
  return ngroups < num_sms ? ngroups : num_sms;
}

// ---------------------------------------------------------------------------
// Symmetric stored matvec q = A p reading the upper triangle only (entries
// j >= i), about half of the 4 n^2 bytes of the full GEMV: the stored kernel
// is HBM-bound, so the bytes are the time.
//   Work item (b, c): rows [256 b, 256 b + 256) (a band) x the columns of
//   chunk c ([512 c, 512 c + 512)) at or right of column 256 b; only the TMA
//   boxes (256 columns x 8 rows) that reach column 256 b are loaded. A stage
//   is 32 rows x 512 columns (4 x 2 boxes, 64 KB), an item at most 8 stages.
//   Scheduling is dynamic: the items, sorted by size (largest first, built on
//   the host once per n), are taken from a global counter by each CTA's
//   producer, so a CTA that runs faster takes more of them and the SMs finish
//   together (greedy list scheduling; a static assignment balanced the
//   modelled cost but left the busiest SM ~10 % behind the mean).
//   Element (i, j), j >= 256 b: the row sum takes A_ij p_j when j >= i, and
//   the transposed contribution A_ij p_i goes to q_j when j > i. The masks
//   matter only in stages whose rows meet the warp's columns, and in the last
//   band, where rows at or past n are not loaded (their shared memory holds
//   stale data and must not enter the column sums).
//   Consumer warp w owns columns 64 w .. 64 w + 63 of the chunk for all 32
//   rows of a stage (two per lane): its transposed sums over the band's 256
//   rows stay in registers, four chains of 64 rows each (colpart[b ns + j]). The 32 row sums of a stage
//   are reduced over the lanes by a transposing shuffle tree and over the 8
//   warps by the last warp to finish the stage (a shared counter per slot; no
//   warp waits for another): rowpart[c ns + i]. k_symv_fin adds the partials
//   in a fixed order (deterministic):
//   q_i = sum_{c >= c0(b_i)} rowpart + sum_{b <= b_i} colpart, and p^T q.
// ---------------------------------------------------------------------------
constexpr int SY_H = 256;                       // rows per band
constexpr int SY_W = 512;                       // columns per chunk
constexpr int SY_BX = SY_W / RB_BOXW;           // column boxes per stage row: 2
constexpr int SY_RG = RB_BOXES / SY_BX;         // row boxes per stage: 4
constexpr int SY_SROWS = SY_RG * RB_ROWS;       // rows per stage: 32
constexpr int SY_GROUPS = SY_H / SY_SROWS;      // stages per item: 8
constexpr int SY_WCOLS = SY_W / RB_CONSUMER_WARPS;  // columns per consumer warp: 64
static_assert(SY_WCOLS == 64 && SY_SROWS == 32 && SY_GROUPS == 8, "lane layout of k_symv_tma");
static_assert(RB_BOXW % SY_WCOLS == 0, "a warp's columns lie in one box");

__host__ __device__ __forceinline__ int symv_c_lo(int b) { return (b * SY_H) / SY_W; }
// padded row stride of the partial buffers (float4 loads in k_symv_fin)
__host__ __device__ __forceinline__ int symv_stride(int n) { return (n + 127) / 128 * 128; }

// Boxes of item (b, c) that reach column 256 b and start before column n,
// and its stages (row groups of 32 that start before row n).
struct SymvItem {
  int b, c, bx_lo, bx_hi, groups;
};
__host__ __device__ __forceinline__ SymvItem symv_item(int item, int n, int nc) {
  SymvItem it;
  it.b = item / nc;
  it.c = item % nc;
  const int lo = (it.b * SY_H - it.c * SY_W) / RB_BOXW;
  it.bx_lo = lo > 0 ? lo : 0;
  const int hi = (n - it.c * SY_W + RB_BOXW - 1) / RB_BOXW;
  it.bx_hi = hi < SY_BX ? hi : SY_BX;
  const int g = (n - it.b * SY_H + SY_SROWS - 1) / SY_SROWS;
  it.groups = g < SY_GROUPS ? g : SY_GROUPS;
  return it;
}

__global__ void __launch_bounds__(RB_THREADS, 1) k_symv_tma(const __grid_constant__ CUtensorMap tmap, SymvArgs a) {
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* tiles = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(RB_STAGES) * RB_STAGE_BYTES);
  uint64_t* empty = full + RB_STAGES;
  // row sums of a stage: one value per warp and row, summed by the last warp
  // to arrive (a counter per slot; no warp waits for another)
  __shared__ float red[RB_STAGES][RB_CONSUMER_WARPS][SY_SROWS];
  __shared__ unsigned int red_cnt[RB_STAGES];
  // what a slot holds: item * 8 + stage of the item, or -1 (no more items)
  __shared__ int s_code[RB_STAGES];
  __shared__ int s_abort;
  __shared__ int s_issued;
  __shared__ int s_consumed[RB_CONSUMER_WARPS];

  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  const int n = a.n, nc = a.nchunks, ns = a.ns, nitems = a.nitems;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < RB_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], RB_CONSUMER_WARPS);
      red_cnt[s] = 0u;
    }
    fence_mbarrier_init();
    s_abort = 0;
    s_issued = 0;
  }
  __syncthreads();

  if (warp == RB_CONSUMER_WARPS) {
    // ---------------- producer: one elected lane takes items, issues boxes --
    if (lane == 0) {
      prefetch_tensormap(&tmap);
      const uint64_t pol = l2_policy_evict_first();
      int it = 0;
      bool stop = false;
      int t = int(atomicAdd(a.sched_ctr, 1u));
      while (t < nitems && !stop) {
        const int item = a.sched_items[t];
        const SymvItem w = symv_item(item, n, nc);
        int t_next = nitems;
        for (int g = 0; g < w.groups; ++g, ++it) {
          // the next ticket is taken as the item's last stage is issued: its
          // latency overlaps the wait for a free slot
          if (g == w.groups - 1) t_next = int(atomicAdd(a.sched_ctr, 1u));
          const int s = it % RB_STAGES;
          if (it >= RB_STAGES && !mbar_wait_bounded(&empty[s], ((it / RB_STAGES) - 1) & 1)) {
            s_abort = 1;
            stop = true;
            break;
          }
          if (*(volatile int*)&s_abort) {
            stop = true;
            break;
          }
          const int row0 = w.b * SY_H + g * SY_SROWS;
          const int nrg = min(SY_RG, (n - row0 + RB_ROWS - 1) / RB_ROWS);  // row boxes before row n
          s_code[s] = item * SY_GROUPS + g;
          mbar_arrive_expect_tx(&full[s], uint32_t(nrg * (w.bx_hi - w.bx_lo)) * RB_ROWS * RB_BOXW * 4);
          for (int rg = 0; rg < nrg; ++rg)
            for (int bx = w.bx_lo; bx < w.bx_hi; ++bx)
              tma_load_2d_hint(tiles + size_t(s) * RB_STAGE_FLOATS + (rg * SY_BX + bx) * RB_ROWS * RB_BOXW, &tmap,
                               &full[s], w.c * SY_W + bx * RB_BOXW, row0 + rg * RB_ROWS, pol);
        }
        t = t_next;
      }
      if (!stop) {
        // no more items: a slot whose code says so, completed by a plain arrival
        const int s = it % RB_STAGES;
        if (it < RB_STAGES || mbar_wait_bounded(&empty[s], ((it / RB_STAGES) - 1) & 1)) {
          s_code[s] = -1;
          mbar_arrive(&full[s]);
        } else {
          s_abort = 1;
        }
      }
      s_issued = it;
    }
  } else {
    // ---------------- consumers: warp w owns columns 64 w .. 64 w + 63 ------
    const int bxw = warp / (RB_BOXW / SY_WCOLS);                  // the warp's column box
    const int ccol = SY_WCOLS * (warp % (RB_BOXW / SY_WCOLS)) + 2 * lane;  // its first column in the box
    int it = 0;
    float pj0 = 0.f, pj1 = 0.f;            // p at the lane's two columns
    float cs0[4] = {0.f, 0.f, 0.f, 0.f}, cs1[4] = {0.f, 0.f, 0.f, 0.f};  // column sums, rows r % 4 apart
    float p_pref = 0.f;                    // p at row row_pref + lane, loaded one stage ahead
    int row_pref = -1;
    while (true) {
      const int s = it % RB_STAGES;
      if (!mbar_wait_bounded(&full[s], (it / RB_STAGES) & 1)) {
        s_abort = 1;
        break;
      }
      const int code = *(volatile int*)&s_code[s];
      if (code < 0) break;
      const SymvItem w = symv_item(code / SY_GROUPS, n, nc);
      const int g = code % SY_GROUPS;
      const int row0 = w.b * SY_H + g * SY_SROWS;
      const int band0 = w.b * SY_H;
      const int j0 = w.c * SY_W + bxw * RB_BOXW + ccol;  // the lane's columns j0, j0 + 1
      const int wj0 = j0 - 2 * lane;                     // the warp's first column
      const bool active = bxw >= w.bx_lo && bxw < w.bx_hi;
      if (g == 0) {
        pj0 = (j0 >= band0 && j0 < n) ? __ldg(a.p + j0) : 0.f;
        pj1 = (j0 + 1 >= band0 && j0 + 1 < n) ? __ldg(a.p + j0 + 1) : 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) cs0[u] = cs1[u] = 0.f;
      }
      float my_p;
      if (row_pref == row0) {
        my_p = p_pref;
      } else {
        my_p = row0 + lane < n ? __ldg(a.p + row0 + lane) : 0.f;
      }
      if (g + 1 < w.groups) {
        row_pref = row0 + SY_SROWS;
        p_pref = row_pref + lane < n ? __ldg(a.p + row_pref + lane) : 0.f;
      } else {
        row_pref = -1;
      }
      float racc[SY_SROWS];
#pragma unroll
      for (int r = 0; r < SY_SROWS; ++r) racc[r] = 0.f;
      if (active) {
        const float* base = tiles + size_t(s) * RB_STAGE_FLOATS + bxw * RB_ROWS * RB_BOXW + ccol;
        // warp-uniform cases (the shuffles below need the whole warp)
        if (wj0 >= row0 + SY_SROWS && row0 + SY_SROWS <= n) {
          // right of every row of the stage, every row before n: no masks
#pragma unroll
          for (int r = 0; r < SY_SROWS; ++r) {
            const float2 av =
                *reinterpret_cast<const float2*>(base + (r / RB_ROWS) * SY_BX * RB_ROWS * RB_BOXW + (r % RB_ROWS) * RB_BOXW);
            const float pi = __shfl_sync(0xffffffffu, my_p, r);
            racc[r] = fmaf(av.x, pj0, av.y * pj1);
            cs0[r & 3] = fmaf(av.x, pi, cs0[r & 3]);
            cs1[r & 3] = fmaf(av.y, pi, cs1[r & 3]);
          }
        } else if (wj0 + SY_WCOLS - 1 >= row0) {
          // meets the stage's rows, or rows at or past n: masks
#pragma unroll
          for (int r = 0; r < SY_SROWS; ++r) {
            const int i = row0 + r;
            const float2 av =
                *reinterpret_cast<const float2*>(base + (r / RB_ROWS) * SY_BX * RB_ROWS * RB_BOXW + (r % RB_ROWS) * RB_BOXW);
            const float pi = __shfl_sync(0xffffffffu, my_p, r);
            const bool row_in = i < n;
            racc[r] = row_in ? fmaf(j0 >= i ? av.x : 0.f, pj0, (j0 + 1 >= i ? av.y : 0.f) * pj1) : 0.f;
            const float cx = (row_in && j0 > i) ? av.x : 0.f;
            const float cy = (row_in && j0 + 1 > i) ? av.y : 0.f;
            cs0[r & 3] = fmaf(cx, pi, cs0[r & 3]);
            cs1[r & 3] = fmaf(cy, pi, cs1[r & 3]);
          }
        }  // else: left of every row of the stage, nothing
      }
      // row sums of the warp's 64 columns: lane l gets row row0 + l
      warp_transpose_sum(racc, lane);
      red[s][warp][lane] = racc[0];
      __syncwarp();
      unsigned int last = 0u;
      if (lane == 0) {
        __threadfence_block();
        last = atomicAdd(&red_cnt[s], 1u) == RB_CONSUMER_WARPS - 1 ? 1u : 0u;
        if (last) {
          __threadfence_block();
          red_cnt[s] = 0u;
        }
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last && row0 + lane < n) {
        __threadfence_block();
        float tsum = 0.f;
#pragma unroll
        for (int q = 0; q < RB_CONSUMER_WARPS; ++q) tsum += *reinterpret_cast<volatile float*>(&red[s][q][lane]);
        a.rowpart[int64_t(w.c) * ns + row0 + lane] = tsum;
      }
      // the item's last stage: the column sums over its rows
      if (g == w.groups - 1 && active) {
        if (j0 >= band0 && j0 < n) a.colpart[int64_t(w.b) * ns + j0] = (cs0[0] + cs0[1]) + (cs0[2] + cs0[3]);
        if (j0 + 1 >= band0 && j0 + 1 < n)
          a.colpart[int64_t(w.b) * ns + j0 + 1] = (cs1[0] + cs1[1]) + (cs1[2] + cs1[3]);
      }
      // the slot (tile and row sums) is released only now: the producer
      // refills it, and the warps reuse its row-sum buffer, after every warp
      // has finished this stage
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      ++it;
    }
    if (lane == 0) s_consumed[warp] = it;
  }
  __syncthreads();
  // Drain: after a timeout, wait (bounded) for boxes still in flight.
  if (s_abort && threadIdx.x == 0) {
    int lo = s_issued;
    for (int w = 0; w < RB_CONSUMER_WARPS; ++w) lo = min(lo, s_consumed[w]);
    for (int it = lo; it < s_issued; ++it) mbar_wait_bounded(&full[it % RB_STAGES], (it / RB_STAGES) & 1);
    record_timeout(st, 1);
  }
}

// q_i = sum_{c >= c0(b_i)} rowpart[c ns + i] + sum_{b <= b_i} colpart[b ns + i]
// and p^T q. A CTA takes 128 consecutive rows (a lane four of them, float4
// loads) and its 8 warps split the partial list of those rows (warp w:
// entries w, w + 8, ...), four loads in flight per warp; the warps' sums are
// combined in shared memory in a fixed order (the result does not depend on
// scheduling). Float32 sums over at most n / 256 + n / 512 + 1 terms. The
// first thread also rewinds the item counter of k_symv_tma, which has
// finished (stream order), for the next launch.
constexpr int SYF_ROWS = 128;  // rows per CTA of the finishing kernel (256 threads)
static_assert(SY_H % SYF_ROWS == 0, "the rows of a finishing CTA lie in one band");
__global__ void __launch_bounds__(256) k_symv_fin(SymvArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.sched_ctr = 0u;
  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  const int n = a.n, nc = a.nchunks, ns = a.ns;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int row0 = blockIdx.x * SYF_ROWS;
  const int b = row0 / SY_H;
  const int c0 = symv_c_lo(b);
  const int nr = nc - c0, total = nr + b + 1;
  // rows row0 + 4 lane .. + 3; the buffers' stride is a multiple of 128 and
  // rows up to the stride are allocated (those past n are not used)
  const int64_t off = row0 + 4 * lane;
  auto src = [&](int t) -> float4 {
    const float* p = t < nr ? a.rowpart + int64_t(c0 + t) * ns : a.colpart + int64_t(t - nr) * ns;
    return __ldcg(reinterpret_cast<const float4*>(p + off));
  };
  float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
  int t = warp;
  for (; t + 24 < total; t += 32) {
    const float4 v0 = src(t), v1 = src(t + 8), v2 = src(t + 16), v3 = src(t + 24);
    s0.x += v0.x; s0.y += v0.y; s0.z += v0.z; s0.w += v0.w;
    s1.x += v1.x; s1.y += v1.y; s1.z += v1.z; s1.w += v1.w;
    s2.x += v2.x; s2.y += v2.y; s2.z += v2.z; s2.w += v2.w;
    s3.x += v3.x; s3.y += v3.y; s3.z += v3.z; s3.w += v3.w;
  }
  for (; t < total; t += 8) {
    const float4 v = src(t);
    s0.x += v.x; s0.y += v.y; s0.z += v.z; s0.w += v.w;
  }
  __shared__ float4 red[8][32];
  red[warp][lane] = make_float4((s0.x + s1.x) + (s2.x + s3.x), (s0.y + s1.y) + (s2.y + s3.y),
                                (s0.z + s1.z) + (s2.z + s3.z), (s0.w + s1.w) + (s2.w + s3.w));
  __syncthreads();
  double my = 0.0;
  if (threadIdx.x < SYF_ROWS) {
    const int l = threadIdx.x >> 2, e = threadIdx.x & 3;  // row row0 + 4 l + e = row0 + threadIdx.x
    const int i = row0 + threadIdx.x;
    float q = 0.f;
#pragma unroll
    for (int w = 0; w < 8; ++w) q += reinterpret_cast<const float*>(&red[w][l])[e];
    if (i < n) {
      a.q[i] = q;
      my = double(a.p[i]) * double(q);
    }
  }
  __shared__ double s_part[4];
  if (warp < 4) {
    const double v = warp_sum(my);
    if (lane == 0) s_part[warp] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) a.partials[blockIdx.x] = (s_part[0] + s_part[1]) + (s_part[2] + s_part[3]);
  if (!arrive_last(a.ticket)) return;
  if (threadIdx.x < 32) {
    double tt = 0.0;
    for (int j = threadIdx.x; j < int(gridDim.x); j += 32) tt += __ldcg(a.partials + j);
    tt = warp_sum(tt);
    if (threadIdx.x == 0 && a.result) *a.result = tt;
  }
}

size_t symv_rowpart_floats(int n) { return size_t((n + SY_W - 1) / SY_W) * symv_stride(n); }
size_t symv_colpart_floats(int n) { return size_t((n + SY_H - 1) / SY_H) * symv_stride(n); }
int symv_fin_grid(int n, int) { return (n + SYF_ROWS - 1) / SYF_ROWS; }

cudaError_t symv_configure() {
  return cudaFuncSetAttribute(k_symv_tma, cudaFuncAttributeMaxDynamicSharedMemorySize, int(RB_SMEM));
}

// Work items (b, c) of the symmetric matvec, largest first (the size of an
// item is the boxes it loads; ties in item order), as b * nchunks + c. The
// CTAs take them in this order from the counter, so the last items to start
// are the smallest.
void symv_schedule(int n, std::vector<int>& items) {
  const int nb = (n + SY_H - 1) / SY_H, nc = (n + SY_W - 1) / SY_W;
  std::vector<std::pair<long long, int>> all;  // (boxes, item)
  for (int b = 0; b < nb; ++b)
    for (int c = symv_c_lo(b); c < nc; ++c) {
      const SymvItem w = symv_item(b * nc + c, n, nc);
      long long boxes = 0;
      for (int g = 0; g < w.groups; ++g) {
        const int row0 = b * SY_H + g * SY_SROWS;
        boxes += (long long)std::min(SY_RG, (n - row0 + RB_ROWS - 1) / RB_ROWS) * (w.bx_hi - w.bx_lo);
      }
      all.push_back({boxes, b * nc + c});
    }
  std::stable_sort(all.begin(), all.end(), [](const auto& x, const auto& y) { return x.first > y.first; });
  items.clear();
  for (const auto& it : all) items.push_back(it.second);
}

cudaError_t launch_symv(const CUtensorMap* tmap, SymvArgs a, int num_sms, cudaStream_t s) {
  a.nbands = (a.n + SY_H - 1) / SY_H;
  a.nchunks = (a.n + SY_W - 1) / SY_W;
  a.ns = symv_stride(a.n);
  k_symv_tma<<<num_sms, RB_THREADS, RB_SMEM, s>>>(*tmap, a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_symv_fin<<<symv_fin_grid(a.n, num_sms), 256, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Fixed scratch of the context-free matvec (dcg_matvec_dense_noalloc), which
// allocates no device memory: the arrival counter of the last-CTA reduction
// at byte 0 and the timeout word at byte 4 (both must be zero when a launch
// starts; the launcher clears the two on the stream before every launch), and
// one double partial per CTA from byte 256. The grid is min(ceil(n / RB_ROWS), SMs), so kNoallocMaxCtas slots
// cover every device with up to 512 SMs (GB300: 152).
// ---------------------------------------------------------------------------
constexpr int kNoallocMaxCtas = 512;
constexpr size_t kNoallocScratchBytes = 256 + sizeof(double) * kNoallocMaxCtas;  // 4352 bytes
constexpr int kNoallocMaxDevices = 64;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

int noalloc_max_ctas() { return kNoallocMaxCtas; }

// Device address of the scratch for the current device, looked up with
// cudaGetSymbolAddress once per device (with that device current) and cached;
// the first lookup also sets the matvec kernel's shared-memory attribute.
cudaError_t noalloc_scratch(void** base) {
  static std::mutex mu;
  static void* addr[kNoallocMaxDevices] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kNoallocMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(mu);
  if (!addr[dev]) {
    void* a = nullptr;
    if ((e = cudaGetSymbolAddress(&a, g_noalloc_scratch)) != cudaSuccess) return e;
    if ((e = rowop_configure()) != cudaSuccess) return e;
    addr[dev] = a;
  }
  *base = addr[dev];
  return cudaSuccess;
}

cudaError_t launch_matvec_noalloc(const CUtensorMap* tmap, const float* p, float* q, int n, double* pAp, int grid,
                                  void* scratch, cudaStream_t s) {
  if (grid < 1 || grid > kNoallocMaxCtas) return cudaErrorInvalidValue;
  unsigned int* counter = static_cast<unsigned int*>(scratch);
  cudaError_t e = cudaMemsetAsync(counter, 0, 2 * sizeof(unsigned int), s);  // counter and timeout word
  if (e != cudaSuccess) return e;
  RowOpArgs a{};
  a.v = p;
  a.out = q;
  a.n = n;
  a.partials = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + 256);
  a.ticket = counter;
  a.abort_word = reinterpret_cast<int*>(counter + 1);
  a.result = pAp;
  return launch_rowop(tmap, a, false, grid, s);
}

// Tensor map over row-major A (n x n, leading dimension lda floats): box of
// RB_BOXW columns x RB_ROWS rows; out-of-range elements read as zero.
bool make_rowop_tmap(CUtensorMap* map, const float* A, int64_t n, int64_t lda, EncodeTiledFn encode) {
  cuuint64_t gdim[2] = {cuuint64_t(n), cuuint64_t(n)};
  cuuint64_t gstride[1] = {cuuint64_t(lda) * 4};
  cuuint32_t box[2] = {RB_BOXW, RB_ROWS};
  cuuint32_t estride[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), gdim, gstride, box, estride,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// Y = A V, V and Y column-major n x c (leading dimension n), c <= 129.
// A CTA computes 256 rows x CB columns of Y over a K range (blockIdx.y; the
// split partials are summed in a fixed order by k_block_reduce: no atomics,
// deterministic). CB is 8, 16 or 32, the narrowest that covers the launch's
// largest column count (wider counts take several blocks of 32), so that a
// few columns stream A at its read rate instead of paying for 32. Per K-step
// of 32, the A tile (256 rows x 32, row-major, row stride 36 floats) and the
// V tile (CB columns x 32, stride 36) arrive in shared memory by asynchronous
// copies (cp.async, 16 bytes for A, 4 bytes for V, whose columns need not be
// 16-byte aligned), two stages in flight.
// 128 threads; thread t computes rows rg, rg + 64, rg + 128, rg + 192 (rg =
// t % 64; at a row stride of 36 floats, 8 consecutive lanes read 8 different
// 16-byte bank groups) and the CB / 2 columns of half cg = t / 64 (a
// broadcast within the warp): per 4 K-values, 4 float4 loads of A and CB / 2
// of V feed 8 CB FMAs. (Measured at n = 16384, 32 columns: 408 us, against
// 440 us for 8 columns per thread with 256 threads and 438 us for a 4-stage
// pipeline of 16-wide K-steps.)
// In a solve (st set) the columns are the k active columns of W.
// ---------------------------------------------------------------------------
constexpr int AB_ROWS = 256;
constexpr int AB_K = 32;
constexpr int AB_LD = AB_K + 4;  // row stride of both tiles (floats)
constexpr int AB_THREADS = 128;
__host__ __device__ constexpr int ab_stage_floats(int cb) { return AB_ROWS * AB_LD + cb * AB_LD; }
__host__ __device__ constexpr size_t ab_smem(int cb) { return size_t(2) * ab_stage_floats(cb) * sizeof(float); }
// Column block of a launch whose largest column count is cmax.
static int ab_cb(int cmax) { return cmax <= 8 ? 8 : (cmax <= 16 ? 16 : 32); }

__device__ __forceinline__ void cp_async16(float* dst, const float* src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async4(float* dst, const float* src, int src_bytes) {
  const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;" ::"r"(d), "l"(src), "r"(src_bytes) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

template <int CB>
__global__ void __launch_bounds__(AB_THREADS, 2) k_apply_block(ApplyBlockArgs a, int kchunk, float* part) {
  constexpr int CPT = CB / 2;  // columns per thread
  constexpr int STAGE = ab_stage_floats(CB);
  extern __shared__ __align__(16) float ab_smem_raw[];
  int c = a.c;
  const float* V = a.V;
  float* Y = a.Y;
  if (a.st) {
    if (a.skip_if_done && a.st->done) return;
    c = a.st->k;
    V += a.n;
    Y += a.n;
  }
  const int n = a.n;
  const int col0 = blockIdx.z * CB;
  if (col0 >= c) return;
  const int cw = min(CB, c - col0);
  const int row0 = blockIdx.x * AB_ROWS;
  const int k_lo = blockIdx.y * kchunk, k_hi = min(n, k_lo + kchunk);
  const int t = threadIdx.x;
  const int rg = t & 63, cg = t >> 6;  // cg in {0, 1}: columns CPT cg ..
  const int64_t lda = a.lda;
  // copies of one K-step into stage b: A chunk idx = q * 128 + t is row idx / 8,
  // 16-byte column chunk idx % 8; V element idx = q * 128 + t is column idx / 32,
  // K offset idx % 32. Out-of-range parts are zero-filled (source size 0 .. 16).
  auto issue = [&](int b, int k0) {
    float* as = ab_smem_raw + b * STAGE;
    float* vs = as + AB_ROWS * AB_LD;
#pragma unroll
    for (int q = 0; q < (AB_ROWS * AB_K / 4) / AB_THREADS; ++q) {
      const int idx = q * AB_THREADS + t;
      const int r = idx >> 3, c4 = idx & 7;
      const int gr = row0 + r, gk = k0 + 4 * c4;
      const int nb = (gr < n) ? 4 * max(0, min(4, k_hi - gk)) : 0;
      const float* src = nb > 0 ? a.A + int64_t(gr) * lda + gk : a.A;
      cp_async16(as + r * AB_LD + 4 * c4, src, nb);
    }
#pragma unroll
    for (int q = 0; q < (CB * AB_K) / AB_THREADS; ++q) {
      const int idx = q * AB_THREADS + t;
      const int j = idx >> 5, kk = idx & 31;
      const int gk = k0 + kk;
      const bool ok = j < cw && gk < k_hi;
      cp_async4(vs + j * AB_LD + kk, ok ? V + int64_t(col0 + j) * n + gk : V, ok ? 4 : 0);
    }
    cp_async_commit();
  };

  float acc[4][CPT];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < CPT; ++j) acc[i][j] = 0.f;
  const int nsteps = k_lo < k_hi ? (k_hi - k_lo + AB_K - 1) / AB_K : 0;
  if (nsteps > 0) issue(0, k_lo);
  for (int s = 0; s < nsteps; ++s) {
    if (s + 1 < nsteps) {
      issue((s + 1) & 1, k_lo + (s + 1) * AB_K);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncthreads();
    const float* as = ab_smem_raw + (s & 1) * STAGE;
    const float* vs = as + AB_ROWS * AB_LD;
#pragma unroll 1
    for (int kq = 0; kq < AB_K; kq += 4) {
      float4 a4[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a4[i] = *reinterpret_cast<const float4*>(as + (rg + 64 * i) * AB_LD + kq);
#pragma unroll
      for (int j = 0; j < CPT; ++j) {
        const float4 v4 = *reinterpret_cast<const float4*>(vs + (CPT * cg + j) * AB_LD + kq);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          acc[i][j] = fmaf(a4[i].x, v4.x, acc[i][j]);
          acc[i][j] = fmaf(a4[i].y, v4.y, acc[i][j]);
          acc[i][j] = fmaf(a4[i].z, v4.z, acc[i][j]);
          acc[i][j] = fmaf(a4[i].w, v4.w, acc[i][j]);
        }
      }
    }
    __syncthreads();
  }
  float* dst = Y;
  if (gridDim.y > 1) dst = part + int64_t(blockIdx.y) * (int64_t(gridDim.z) * CB) * n;
#pragma unroll
  for (int j = 0; j < CPT; ++j) {
    const int cj = CPT * cg + j;
    if (cj >= cw) continue;
    float* colp = dst + int64_t(col0 + cj) * n;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int gr = row0 + rg + 64 * i;
      if (gr < n) colp[gr] = acc[i][j];
    }
  }
}

cudaError_t apply_block_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_apply_block<8>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ab_smem(8)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_apply_block<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ab_smem(16)));
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_apply_block<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(ab_smem(32)));
  return e;
}

// Y[:, j] = sum over the K splits of the partials (fixed order); split sp of
// column j, row i is part[sp * sstride + j * n + i].
__global__ void __launch_bounds__(256) k_block_reduce(ApplyBlockArgs a, int splits, int64_t sstride, const float* part) {
  int c = a.c;
  float* Y = a.Y;
  if (a.st) {
    if (a.skip_if_done && a.st->done) return;
    c = a.st->k;
    Y += a.n;
  }
  const int64_t total = int64_t(c) * a.n;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    float s = 0.f;
    for (int sp = 0; sp < splits; ++sp) s += part[sp * sstride + idx];
    Y[idx] = s;
  }
}

// K splits: the CTA count (row blocks x column blocks x splits) is chosen to
// fill whole waves of two CTAs per SM (the smallest split count within 2% of
// the best wave efficiency), with at least 8 K-steps per split, at most 16.
int apply_block_splits(int n, int cmax, int num_sms) {
  const int cb = ab_cb(cmax);
  const int rowblocks = (n + AB_ROWS - 1) / AB_ROWS;
  const int colblocks = (cmax + cb - 1) / cb;
  const int base = rowblocks * colblocks;
  const int slots = 2 * num_sms;
  int kmax_splits = (n + AB_K * 8 - 1) / (AB_K * 8);
  if (kmax_splits > 16) kmax_splits = 16;
  if (kmax_splits < 1) kmax_splits = 1;
  double eff[17] = {0.0};
  double best = 0.0;
  for (int sp = 1; sp <= kmax_splits; ++sp) {
    const long long ctas = (long long)base * sp;
    const long long waves = (ctas + slots - 1) / slots;
    eff[sp] = double(ctas) / double(waves * slots);
    best = std::max(best, eff[sp]);
  }
  for (int sp = 1; sp <= kmax_splits; ++sp)
    if (eff[sp] >= best - 0.02) return sp;
  return 1;
}

// Largest split-K partial buffer any column count up to cmax can need.
size_t apply_block_scratch_floats(int n, int cmax, int num_sms) {
  size_t best = 0;
  for (int c = 1; c <= cmax; ++c) {
    const int cb = ab_cb(c);
    const int splits = apply_block_splits(n, c, num_sms);
    if (splits > 1) best = std::max(best, size_t(splits) * size_t((c + cb - 1) / cb) * cb * size_t(n));
  }
  return best;
}

cudaError_t launch_apply_block(const ApplyBlockArgs& a, int cmax, float* scratch, int num_sms, cudaStream_t s) {
  if (cmax <= 0) return cudaSuccess;
  const int n = a.n;
  const int cb = ab_cb(cmax);
  const int splits = scratch ? apply_block_splits(n, cmax, num_sms) : 1;
  int kchunk = (n + splits - 1) / splits;
  kchunk = (kchunk + AB_K - 1) / AB_K * AB_K;
  const int used = (n + kchunk - 1) / kchunk;
  const int colblocks = (cmax + cb - 1) / cb;
  dim3 grid((n + AB_ROWS - 1) / AB_ROWS, used, colblocks);
  if (cb == 8)
    k_apply_block<8><<<grid, AB_THREADS, ab_smem(8), s>>>(a, kchunk, scratch);
  else if (cb == 16)
    k_apply_block<16><<<grid, AB_THREADS, ab_smem(16), s>>>(a, kchunk, scratch);
  else
    k_apply_block<32><<<grid, AB_THREADS, ab_smem(32), s>>>(a, kchunk, scratch);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || used == 1) return e;
  k_block_reduce<<<2 * num_sms, 256, 0, s>>>(a, used, int64_t(colblocks) * cb * n, scratch);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Y = A V on the tensor cores (the start-of-solve product A W of Algorithm 1
// and dcg_apply_block), split TF32 so that the product keeps float32
// accuracy: A = A_hi + A_lo and V = V_hi + V_lo with A_hi = tf32(A),
// A_lo = tf32(A - A_hi) (both rounded to nearest; A - A_hi is exact in
// float32), so that A V = A_hi V_hi + A_hi V_lo + A_lo V_hi + O(2^-22) per
// product, three kind::tf32 MMAs per K step. The hardware accumulates one
// MMA chain with a bias that grows with its length (measured ~2e-8 per step
// over long chains), so each 32-column K stage (4 K steps x 3 MMAs) goes to
// its own TMEM accumulator and is added into float32 registers, rounded to
// nearest, by the epilogue: the bias is bounded by one stage.
//   Persistent CTAs take work items (128-row block, K range) in a fixed
// stride; a K range's result goes to Y directly (one range) or to a partial
// buffer that k_block_reduce sums in a fixed order. Roles (14 warps):
//   warp 0   TMA: A box 32 x 128 and V box 32 x NPAD (128-byte swizzle) per stage;
//   warp 1   MMA issue (one thread), TMEM owner;
//   warps 2-5   split the stage in shared memory: hi in place, lo beside it
//               (elementwise, so the swizzle does not matter), then a proxy
//               fence so that the tensor core sees the generic stores;
//   warps 6-13  read the stage's accumulator (two warps per TMEM lane quarter,
//               each half of the columns) and add it into registers.
// Every wait is bounded; a CTA that gives up fills its outputs with NaN and
// records a timeout in the state given.
// ---------------------------------------------------------------------------
constexpr int AT_M = 128;                 // rows per item (MMA M)
constexpr int AT_K = 32;                  // K per stage: one 128-byte swizzle row of float32
constexpr int AT_CONV_WARPS = 4;
constexpr int AT_EPI_WARPS = 8;
constexpr int AT_THREADS = (2 + AT_CONV_WARPS + AT_EPI_WARPS) * 32;
constexpr int AT_A_BYTES = AT_M * AT_K * 4;   // 16 KB
constexpr int AT_MAX_NPAD = 160;          // columns of V (c <= 129) rounded up to 32
__host__ __device__ constexpr int at_stage_bytes(int npad) { return 2 * AT_A_BYTES + 2 * npad * AT_K * 4; }
__host__ __device__ constexpr int at_stages(int npad) { return npad <= 32 ? 5 : (npad <= 64 ? 4 : 3); }
__host__ __device__ constexpr size_t at_smem(int npad) {
  return 1024 + size_t(at_stages(npad)) * at_stage_bytes(npad) + 256;
}
__host__ __device__ constexpr uint32_t at_tmem_cols(int npad) {
  return 2 * npad <= 64 ? 64u : (2 * npad <= 128 ? 128u : (2 * npad <= 256 ? 256u : 512u));
}

struct ApplyTcArgs {
  int n;
  int c;              // columns written (c <= NPAD); with st: read from st->k
  int splits;         // K ranges per row block
  int kchunk;         // K per range (multiple of AT_K)
  int items;          // row blocks x splits
  float* Y;           // column-major, leading dimension n (column 0 of the output)
  float* part;        // splits > 1: part[r * NPAD * n + col * n + row]
  DevState* st;       // in a solve: the state (k, done); also where a timeout is recorded
  DevState* tst;      // where a timeout is recorded when st is null (may be null)
  int skip_if_done;
};

__device__ __forceinline__ void at_split4(float4& hi, float4& lo) {
  float4 h;
  h.x = round_tf32(hi.x);
  h.y = round_tf32(hi.y);
  h.z = round_tf32(hi.z);
  h.w = round_tf32(hi.w);
  lo.x = round_tf32(hi.x - h.x);
  lo.y = round_tf32(hi.y - h.y);
  lo.z = round_tf32(hi.z - h.z);
  lo.w = round_tf32(hi.w - h.w);
  hi = h;
}

template <int NPAD>
__global__ void __launch_bounds__(AT_THREADS, 1)
    k_apply_tc(const __grid_constant__ CUtensorMap tmap_a, const __grid_constant__ CUtensorMap tmap_v, ApplyTcArgs a) {
  constexpr int ST = at_stages(NPAD);
  constexpr int SB = at_stage_bytes(NPAD);
  constexpr int V_BYTES = NPAD * AT_K * 4;
  constexpr int HC = NPAD / 2;              // columns per epilogue warp
  static_assert(NPAD % 32 == 0 && NPAD <= AT_MAX_NPAD && HC % 16 == 0, "column tiling");
  static_assert(AT_A_BYTES % 1024 == 0 && V_BYTES % 1024 == 0, "1024-byte aligned operand tiles");
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint64_t* bars = reinterpret_cast<uint64_t*>(base + size_t(ST) * SB);
  uint64_t* full = bars;             // [ST] TMA landed
  uint64_t* conv = full + ST;        // [ST] split done
  uint64_t* empty = conv + ST;       // [ST] MMAs done with the stage
  uint64_t* tfull = empty + ST;      // [2] accumulator ready
  uint64_t* tempty = tfull + 2;      // [2] accumulator read
  uint64_t* mdone = tempty + 2;      // all MMAs retired
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int s_issued;
  __shared__ int s_cprog[AT_CONV_WARPS];  // stages each split warp has taken, for the drain

  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  const int c = st ? st->k : a.c;
  if (c <= 0) return;
  const int n = a.n, S = a.splits, G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int s = 0; s < ST; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], AT_CONV_WARPS);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], AT_EPI_WARPS);
    }
    mbar_init(mdone, 1);
    fence_mbarrier_init();
    s_abort = 0;
    s_issued = 0;
  }
  if (warp == 1) tc::tmem_alloc(&s_tmem, at_tmem_cols(NPAD));
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  auto steps_of = [&](int item) {
    const int sp = item % S;
    const int k0 = sp * a.kchunk;
    const int k1 = min(n, k0 + a.kchunk);
    return k0 < k1 ? (k1 - k0 + AT_K - 1) / AT_K : 0;
  };

  if (warp == 0) {
    // ---------------- TMA producer ----------------
    if (lane == 0) {
      prefetch_tensormap(&tmap_a);
      prefetch_tensormap(&tmap_v);
      const uint64_t pol = l2_policy_evict_first();
      int it = 0;
      bool stop = false;
      for (int item = blockIdx.x; item < a.items && !stop; item += G) {
        const int rb = item / S, k0 = (item % S) * a.kchunk, ns = steps_of(item);
        for (int j = 0; j < ns; ++j, ++it) {
          const int s = it % ST;
          if (it >= ST && !mbar_wait_bounded(&empty[s], ((it / ST) - 1) & 1)) {
            s_abort = 1;
            stop = true;
            break;
          }
          if (*(volatile int*)&s_abort) {
            stop = true;
            break;
          }
          unsigned char* stg = base + size_t(s) * SB;
          mbar_arrive_expect_tx(&full[s], uint32_t(AT_A_BYTES + V_BYTES));
          tma_load_2d_hint(stg, &tmap_a, &full[s], k0 + AT_K * j, rb * AT_M, pol);
          tma_load_2d(stg + 2 * AT_A_BYTES, &tmap_v, &full[s], k0 + AT_K * j, 0);
        }
      }
      s_issued = it;
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      const uint32_t idesc = tc::instr_desc(tc::kFmtTF32, AT_M, NPAD);
      int it = 0;
      bool stop = false;
      for (int item = blockIdx.x; item < a.items && !stop; item += G) {
        const int ns = steps_of(item);
        for (int j = 0; j < ns; ++j, ++it) {
          const int s = it % ST, b = it & 1;
          if (!mbar_wait_bounded(&conv[s], (it / ST) & 1) ||
              (it >= 2 && !mbar_wait_bounded(&tempty[b], ((it >> 1) - 1) & 1))) {
            s_abort = 1;
            stop = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t sa = smem_u32(base + size_t(s) * SB);
          const uint32_t d = tmem + uint32_t(b * NPAD);
#pragma unroll
          for (int kk = 0; kk < AT_K / 8; ++kk) {
            const uint64_t ahi = tc::smem_desc_kmajor(sa + 32 * kk, 128);
            const uint64_t alo = tc::smem_desc_kmajor(sa + AT_A_BYTES + 32 * kk, 128);
            const uint64_t vhi = tc::smem_desc_kmajor(sa + 2 * AT_A_BYTES + 32 * kk, 128);
            const uint64_t vlo = tc::smem_desc_kmajor(sa + 2 * AT_A_BYTES + V_BYTES + 32 * kk, 128);
            tc::mma_tf32(d, ahi, vhi, idesc, kk > 0);
            tc::mma_tf32(d, ahi, vlo, idesc, 1);
            tc::mma_tf32(d, alo, vhi, idesc, 1);
          }
          tc::mma_commit(&empty[s]);
          tc::mma_commit(&tfull[b]);
        }
      }
      tc::mma_commit(mdone);  // arrives once every MMA issued above has completed
    }
  } else if (warp < 2 + AT_CONV_WARPS) {
    // ---------------- split into hi and lo ----------------
    const int t = threadIdx.x - 64;
    int it = 0;
    bool stop = false;
    for (int item = blockIdx.x; item < a.items && !stop; item += G) {
      const int ns = steps_of(item);
      for (int j = 0; j < ns; ++j, ++it) {
        const int s = it % ST;
        if (!mbar_wait_bounded(&full[s], (it / ST) & 1)) {
          s_abort = 1;
          stop = true;
          break;
        }
        unsigned char* stg = base + size_t(s) * SB;
        float4* ah = reinterpret_cast<float4*>(stg);
        float4* al = reinterpret_cast<float4*>(stg + AT_A_BYTES);
#pragma unroll
        for (int q = t; q < AT_A_BYTES / 16; q += AT_CONV_WARPS * 32) {
          float4 h = ah[q], l;
          at_split4(h, l);
          ah[q] = h;
          al[q] = l;
        }
        float4* vh = reinterpret_cast<float4*>(stg + 2 * AT_A_BYTES);
        float4* vl = reinterpret_cast<float4*>(stg + 2 * AT_A_BYTES + V_BYTES);
#pragma unroll
        for (int q = t; q < V_BYTES / 16; q += AT_CONV_WARPS * 32) {
          float4 h = vh[q], l;
          at_split4(h, l);
          vh[q] = h;
          vl[q] = l;
        }
        fence_proxy_async_smem();  // the tensor core (async proxy) reads what these stores wrote
        __syncwarp();
        if (lane == 0) mbar_arrive(&conv[s]);
      }
    }
    if (lane == 0) s_cprog[warp - 2] = it;
  } else {
    // ---------------- epilogue: accumulate the stages in registers ----------------
    const int e = warp - (2 + AT_CONV_WARPS);
    const int quarter = warp & 3;                // TMEM lanes this warp may read
    const int col0 = (e / 4) * HC;
    const uint32_t lane_off = uint32_t(quarter * 32) << 16;
    int it = 0;
    bool stop = false;
    for (int item = blockIdx.x; item < a.items && !stop; item += G) {
      const int rb = item / S, sp = item % S, ns = steps_of(item);
      float acc[HC];
#pragma unroll
      for (int q = 0; q < HC; ++q) acc[q] = 0.f;
      for (int j = 0; j < ns; ++j, ++it) {
        const int b = it & 1;
        if (!mbar_wait_bounded(&tfull[b], (it >> 1) & 1)) {
          s_abort = 1;
          stop = true;
          break;
        }
        tc::fence_after_sync();
#pragma unroll
        for (int q = 0; q < HC; q += 16) {
          uint32_t r[16];
          tc::tmem_ld16_nowait(tmem + lane_off + uint32_t(b * NPAD + col0 + q), r);
          tc::tmem_wait_ld16(r);
#pragma unroll
          for (int u = 0; u < 16; ++u) acc[q + u] += __uint_as_float(r[u]);
        }
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
      }
      if (stop) break;
      const int row = rb * AT_M + quarter * 32 + lane;
      float* dst = S > 1 ? a.part + int64_t(sp) * NPAD * n : a.Y;
      if (row < n) {
#pragma unroll
        for (int q = 0; q < HC; ++q)
          if (col0 + q < c) dst[int64_t(col0 + q) * n + row] = acc[q];
      }
    }
  }
  __syncthreads();
  if (s_abort) {
    // drain: wait (bounded) for the copies still in flight (issued, not yet
    // taken by every split warp), then fill every output of this CTA's items
    // with NaN and record the timeout
    if (threadIdx.x == 0) {
      int lo = s_issued;
      for (int w = 0; w < AT_CONV_WARPS; ++w) lo = min(lo, s_cprog[w]);
      for (int it = lo; it < s_issued; ++it) mbar_wait_bounded(&full[it % ST], (it / ST) & 1);
      record_timeout(st ? st : a.tst, 6);
    }
    for (int item = blockIdx.x; item < a.items; item += G) {
      const int rb = item / S, sp = item % S;
      float* dst = S > 1 ? a.part + int64_t(sp) * NPAD * n : a.Y;
      for (int idx = threadIdx.x; idx < AT_M * c; idx += blockDim.x) {
        const int row = rb * AT_M + idx % AT_M, col = idx / AT_M;
        if (row < n) dst[int64_t(col) * n + row] = __int_as_float(0x7fc00000);
      }
    }
  }
  if (warp == 1) {
    if (lane == 0) mbar_wait_bounded(mdone, 0);
    __syncwarp();
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, at_tmem_cols(NPAD));
  }
}

// K ranges per 128-row block for the tensor-core product: persistent CTAs
// (one per SM) take items (row block, K range) in a fixed stride, so the
// item count should fill whole rounds of CTAs; the smallest count within 2 %
// of the best round efficiency, at least 8 stages per range, at most 8
// ranges (the partial buffer holds ranges x NPAD x n floats).
int apply_tc_splits(int n, int num_sms) {
  const int rowblocks = (n + AT_M - 1) / AT_M;
  int smax = (n + AT_K * 8 - 1) / (AT_K * 8);
  smax = std::max(1, std::min(smax, 8));
  double eff[9] = {0.0};
  double best = 0.0;
  for (int sp = 1; sp <= smax; ++sp) {
    const long long items = (long long)rowblocks * sp;
    const long long rounds = (items + num_sms - 1) / num_sms;
    eff[sp] = double(items) / double(rounds * num_sms);
    best = std::max(best, eff[sp]);
  }
  for (int sp = 1; sp <= smax; ++sp)
    if (eff[sp] >= best - 0.02) return sp;
  return 1;
}

int apply_tc_npad(int c) { return (c + 31) / 32 * 32; }

bool apply_tc_supported(int n, int cmax) { return n % 4 == 0 && n >= AT_K && apply_tc_npad(cmax) <= AT_MAX_NPAD; }

// Up to 16 columns the FP32-pipe kernel's 8- and 16-column blocks stream A
// faster than the tensor-core kernel, whose W operand is padded to 32 columns
// (measured at n = 16384, 8 columns: 0.21 against 0.35 ms).
bool apply_tc_preferred(int cmax) { return cmax > 16; }

size_t apply_tc_scratch_floats(int n, int cmax, int num_sms) {
  if (!apply_tc_supported(n, cmax)) return 0;
  const int s = apply_tc_splits(n, num_sms);
  return s > 1 ? size_t(s) * apply_tc_npad(cmax) * size_t(n) : 0;
}

// Tensor maps of the two operands: A (row-major, leading dimension lda) in
// boxes of 32 columns x 128 rows, V (column-major n x cols, leading dimension
// n, i.e. rows of n floats) in boxes of 32 x npad; 128-byte swizzle, zero
// fill outside the matrices.
bool make_apply_tc_tmaps(CUtensorMap* ma, CUtensorMap* mv, const float* A, int64_t lda, const float* V, int n,
                         int cols, EncodeTiledFn encode) {
  if (A) {
    cuuint64_t gdim[2] = {cuuint64_t(n), cuuint64_t(n)};
    cuuint64_t gstride[1] = {cuuint64_t(lda) * 4};
    cuuint32_t box[2] = {AT_K, AT_M};
    cuuint32_t estride[2] = {1, 1};
    if (encode(ma, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(A), gdim, gstride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  if (V) {
    cuuint64_t gdim[2] = {cuuint64_t(n), cuuint64_t(cols)};
    cuuint64_t gstride[1] = {cuuint64_t(n) * 4};
    cuuint32_t box[2] = {AT_K, cuuint32_t(apply_tc_npad(cols))};
    cuuint32_t estride[2] = {1, 1};
    if (encode(mv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(V), gdim, gstride, box, estride,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return false;
  }
  return true;
}

cudaError_t apply_tc_configure() {
  cudaError_t e;
  if ((e = cudaFuncSetAttribute(k_apply_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(at_smem(32)))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_apply_tc<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(at_smem(64)))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_apply_tc<96>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(at_smem(96)))) != cudaSuccess) return e;
  if ((e = cudaFuncSetAttribute(k_apply_tc<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(at_smem(128)))) != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_apply_tc<160>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(at_smem(160)));
}

// Y = A V with the maps above; cmax: the column count the maps were made for
// (in a solve the kernel reads the active count from the state). scratch:
// apply_tc_scratch_floats(n, cmax) floats (or null with one K range).
cudaError_t launch_apply_tc(const CUtensorMap* ma, const CUtensorMap* mv, const ApplyBlockArgs& b, int cmax,
                            float* scratch, DevState* tst, int num_sms, cudaStream_t s) {
  const int n = b.n;
  const int npad = apply_tc_npad(cmax);
  int splits = scratch ? apply_tc_splits(n, num_sms) : 1;
  int kchunk = (n + splits - 1) / splits;
  kchunk = (kchunk + AT_K - 1) / AT_K * AT_K;
  splits = (n + kchunk - 1) / kchunk;
  ApplyTcArgs a{};
  a.n = n;
  a.c = b.c;
  a.splits = splits;
  a.kchunk = kchunk;
  a.items = ((n + AT_M - 1) / AT_M) * splits;
  a.Y = b.st ? b.Y + b.n : b.Y;
  a.part = scratch;
  a.st = b.st;
  a.tst = tst;
  a.skip_if_done = b.skip_if_done;
  const int grid = std::min(a.items, num_sms);
  switch (npad) {
    case 32: k_apply_tc<32><<<grid, AT_THREADS, at_smem(32), s>>>(*ma, *mv, a); break;
    case 64: k_apply_tc<64><<<grid, AT_THREADS, at_smem(64), s>>>(*ma, *mv, a); break;
    case 96: k_apply_tc<96><<<grid, AT_THREADS, at_smem(96), s>>>(*ma, *mv, a); break;
    case 128: k_apply_tc<128><<<grid, AT_THREADS, at_smem(128), s>>>(*ma, *mv, a); break;
    case 160: k_apply_tc<160><<<grid, AT_THREADS, at_smem(160), s>>>(*ma, *mv, a); break;
    default: return cudaErrorInvalidValue;
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || splits == 1) return e;
  ApplyBlockArgs r = b;
  k_block_reduce<<<2 * num_sms, 256, 0, s>>>(r, splits, int64_t(npad) * r.n, scratch);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// A = s^2 exp(-|x_i - x_j|^2 / (2 l^2)) + noise [i == j]  (Sec. 3 RBF kernel)
// 128 x 128 output tiles, 256 threads, 8 x 8 entries per thread (rows
// 8 ty .. 8 ty + 7, columns 4 tx .. 4 tx + 3 and 64 + 4 tx .. 64 + 4 tx + 3, so
// that each store instruction writes 256 contiguous bytes of two rows). The X
// rows of the tile are staged transposed in shared memory, 16 dimensions per
// pass. Squared distances in float32 difference form, two entries per packed
// f32x2 subtract and fused multiply-add; exp(z) = 2^(z log2 e) on the
// hardware ex2 (about 2 ulp), evaluated on the float32 argument as expf would be.
// ---------------------------------------------------------------------------
constexpr int FR_T = 128;          // output tile edge
constexpr int FR_DC = 16;          // dimensions per pass
constexpr int FR_LD = FR_T + 4;    // padded row of the transposed X tiles

__device__ __forceinline__ unsigned long long f2_pack(float lo, float hi) {
  return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}
__device__ __forceinline__ float2 f2_unpack(unsigned long long v) {
  return make_float2(__uint_as_float(unsigned(v)), __uint_as_float(unsigned(v >> 32)));
}
// acc += (u - v) * (u - v), lane-wise on float pairs
__device__ __forceinline__ void f2_sqdiff_acc(unsigned long long& acc, unsigned long long u, unsigned long long v) {
  unsigned long long df;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(df) : "l"(u), "l"(v));
  asm("fma.rn.f32x2 %0, %1, %1, %0;" : "+l"(acc) : "l"(df));
}
__device__ __forceinline__ float ex2_approx(float x) {
  float y;
  asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}

__global__ void __launch_bounds__(256, 2) k_form_rbf(const float* __restrict__ X, int n, int d, float c_exp2,
                                                     float s2, float noise, float* __restrict__ A, int64_t lda) {
  __shared__ __align__(16) float xiT[FR_DC][FR_LD];
  __shared__ __align__(16) float xjT[FR_DC][FR_LD];
  const int t = threadIdx.x, ty = t / 16, tx = t % 16;
  if (blockIdx.x < blockIdx.y) return;  // A is symmetric: the tile above the diagonal writes both
  const int i0 = blockIdx.y * FR_T, j0 = blockIdx.x * FR_T;
  unsigned long long sq[8][4];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int p = 0; p < 4; ++p) sq[a][p] = 0ull;
  for (int m0 = 0; m0 < d; m0 += FR_DC) {
    const int dc = min(FR_DC, d - m0);
    if (m0 > 0) __syncthreads();
    for (int idx = t; idx < FR_T * FR_DC; idx += 256) {
      const int r = idx / FR_DC, mm = idx % FR_DC;
      const bool okm = mm < dc;
      xiT[mm][r] = (okm && i0 + r < n) ? X[int64_t(i0 + r) * d + m0 + mm] : 0.f;
      xjT[mm][r] = (okm && j0 + r < n) ? X[int64_t(j0 + r) * d + m0 + mm] : 0.f;
    }
    __syncthreads();
    for (int mm = 0; mm < dc; ++mm) {
      const float4 ua = *reinterpret_cast<const float4*>(&xiT[mm][8 * ty]);
      const float4 ub = *reinterpret_cast<const float4*>(&xiT[mm][8 * ty + 4]);
      const float4 va = *reinterpret_cast<const float4*>(&xjT[mm][4 * tx]);
      const float4 vb = *reinterpret_cast<const float4*>(&xjT[mm][64 + 4 * tx]);
      const unsigned long long v2[4] = {f2_pack(va.x, va.y), f2_pack(va.z, va.w), f2_pack(vb.x, vb.y),
                                        f2_pack(vb.z, vb.w)};
      const float u[8] = {ua.x, ua.y, ua.z, ua.w, ub.x, ub.y, ub.z, ub.w};
#pragma unroll
      for (int a = 0; a < 8; ++a) {
        const unsigned long long uu = f2_pack(u[a], u[a]);
#pragma unroll
        for (int p = 0; p < 4; ++p) f2_sqdiff_acc(sq[a][p], uu, v2[p]);
      }
    }
  }
  const bool diag_tile = blockIdx.x == blockIdx.y;
  const bool vec_ok = (lda % 4) == 0 && (reinterpret_cast<uintptr_t>(A) % 16) == 0;
  // entry values, val[a][cc] for row 8 ty + a and column 64 (cc / 4) + 4 tx + cc % 4
  float val[8][8];
#pragma unroll
  for (int a = 0; a < 8; ++a)
#pragma unroll
    for (int pp = 0; pp < 4; ++pp) {
      const float2 q = f2_unpack(sq[a][pp]);
      val[a][2 * pp] = s2 * ex2_approx(q.x * c_exp2);
      val[a][2 * pp + 1] = s2 * ex2_approx(q.y * c_exp2);
    }
  if (diag_tile) {
#pragma unroll
    for (int a = 0; a < 8; ++a)
#pragma unroll
      for (int cc = 0; cc < 8; ++cc)
        if (8 * ty + a == 64 * (cc / 4) + 4 * tx + cc % 4) val[a][cc] += noise;
  }
  // the tile (rows i0.., columns j0..)
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int i = i0 + 8 * ty + a;
    if (i >= n) continue;
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int j = j0 + 64 * g + 4 * tx;
      float* dst = A + int64_t(i) * lda + j;
      if (vec_ok && j + 3 < n) {
        *reinterpret_cast<float4*>(dst) = make_float4(val[a][4 * g], val[a][4 * g + 1], val[a][4 * g + 2], val[a][4 * g + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c)
          if (j + c < n) dst[c] = val[a][4 * g + c];
      }
    }
  }
  if (diag_tile) return;
  // its mirror (rows j0.., columns i0..): each lane writes 8 consecutive
  // floats (one 32-byte run) of a row
  const int ic = i0 + 8 * ty;
#pragma unroll
  for (int cc = 0; cc < 8; ++cc) {
    const int jr = j0 + 64 * (cc / 4) + 4 * tx + cc % 4;
    if (jr >= n) continue;
    float* dst = A + int64_t(jr) * lda + ic;
    if (vec_ok && ic + 7 < n) {
      *reinterpret_cast<float4*>(dst) = make_float4(val[0][cc], val[1][cc], val[2][cc], val[3][cc]);
      *reinterpret_cast<float4*>(dst + 4) = make_float4(val[4][cc], val[5][cc], val[6][cc], val[7][cc]);
    } else {
#pragma unroll
      for (int a = 0; a < 8; ++a)
        if (ic + a < n) dst[a] = val[a][cc];
    }
  }
}

cudaError_t launch_form_rbf(const float* X, int n, int d, double l, double s2, double noise, float* A, int64_t lda,
                            cudaStream_t s) {
  dim3 grid((n + FR_T - 1) / FR_T, (n + FR_T - 1) / FR_T);
  // exp(-sq / (2 l^2)) = 2^(sq * c), c = -log2(e) / (2 l^2)
  const float c_exp2 = float(-1.4426950408889634 / (2.0 * l * l));
  k_form_rbf<<<grid, 256, 0, s>>>(X, n, d, c_exp2, float(s2), float(noise), A, lda);
  return cudaGetLastError();
}

}  // namespace dcg
