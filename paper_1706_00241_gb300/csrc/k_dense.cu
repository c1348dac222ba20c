// Stored-operator kernels (dense row-major float32 A):
//   * k_rowop_tma: q = A p with the fused p^T q of Algorithm 1 line 6, or the
//     true residual r = b - A x with float64 accumulation (the stopping test of
//     the Sec. 3 experiments and the residual replacement). A streams through a
//     shared-memory ring filled by 2-D TMA tiles (cp.async.bulk.tensor) and
//     completed on mbarriers; one CTA per SM owns a contiguous band of rows.
//   * k_apply_block: Y = A V for up to 129 columns in one pass (the start-of-
//     solve product A [x_{-1} | W] of Algorithm 1 line 3).
//   * k_form_rbf: A = K + noise I for the Sec. 3 RBF kernel.
#include "dcg_kernels.cuh"

namespace dcg {

// Tile geometry of the TMA row-band kernel.
constexpr int RB_ROWS = 4;                      // rows per stage (box height)
constexpr int RB_BOXW = 256;                    // floats per box row (1 KB)
constexpr int RB_BOXES = 8;                     // boxes per stage
constexpr int RB_CHUNK = RB_BOXW * RB_BOXES;    // 2048 columns per stage
constexpr int RB_STAGES = 6;
constexpr int RB_STAGE_FLOATS = RB_ROWS * RB_CHUNK;
constexpr int RB_STAGE_BYTES = RB_STAGE_FLOATS * 4;  // 32 KB
constexpr int RB_CONSUMER_WARPS = 8;            // one warp per box
constexpr int RB_THREADS = (RB_CONSUMER_WARPS + 1) * 32;
constexpr size_t RB_SMEM = size_t(RB_STAGES) * RB_STAGE_BYTES + 2 * RB_STAGES * sizeof(uint64_t) + 1024;

size_t rowop_smem_bytes() { return RB_SMEM; }

__device__ __forceinline__ void record_timeout(DevState* st, int site) {
  if (st) {
    st->status = DCG_ERR_TIMEOUT;
    st->timeout_site = site;
    st->done = 1;
  }
}

// One CTA streams rows [RB_ROWS*g_lo, RB_ROWS*g_hi) of A. Warp w of the
// consumers owns box w of every stage (256 columns); lane l owns float4 slots
// l and l + 32 of each box row, so each thread keeps RB_ROWS accumulators.
template <bool RESID>
__global__ void __launch_bounds__(RB_THREADS, 1)
    k_rowop_tma(const __grid_constant__ CUtensorMap tmap, RowOpArgs a) {
  using Acc = typename std::conditional<RESID, double, float>::type;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  float* tiles = reinterpret_cast<float*>(smem);
  uint64_t* full = reinterpret_cast<uint64_t*>(smem + size_t(RB_STAGES) * RB_STAGE_BYTES);
  uint64_t* empty = full + RB_STAGES;
  __shared__ Acc red[RB_CONSUMER_WARPS][RB_ROWS];
  __shared__ int s_abort;
  __shared__ int s_issued;
  __shared__ int s_consumed[RB_CONSUMER_WARPS];
  __shared__ double s_part[RB_CONSUMER_WARPS];

  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;

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
          tma_load_2d(tiles + size_t(s) * RB_STAGE_FLOATS + bx * RB_ROWS * RB_BOXW, &tmap, &full[s],
                      c * RB_CHUNK + bx * RB_BOXW, g * RB_ROWS);
      }
      s_issued = it;
    }
  } else {
    // ---------------- consumers ---------------------------------------------
    Acc acc[RB_ROWS];
#pragma unroll
    for (int r = 0; r < RB_ROWS; ++r) acc[r] = Acc(0);
    int it = 0;
    for (; it < total; ++it) {
      const int s = it % RB_STAGES;
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
          const int j = col0 + 4 * slot;
          float4 v;
          if (j + 3 < n) {
            v = __ldg(reinterpret_cast<const float4*>(a.v + j));
          } else {
            v.x = j < n ? __ldg(a.v + j) : 0.f;
            v.y = j + 1 < n ? __ldg(a.v + j + 1) : 0.f;
            v.z = j + 2 < n ? __ldg(a.v + j + 2) : 0.f;
            v.w = 0.f;
          }
#pragma unroll
          for (int r = 0; r < RB_ROWS; ++r) {
            const float4 av = reinterpret_cast<const float4*>(box + r * RB_BOXW)[slot];
            if constexpr (RESID) {
              acc[r] = fma(double(av.x), double(v.x), acc[r]);
              acc[r] = fma(double(av.y), double(v.y), acc[r]);
              acc[r] = fma(double(av.z), double(v.z), acc[r]);
              acc[r] = fma(double(av.w), double(v.w), acc[r]);
            } else {
              acc[r] = fmaf(av.x, v.x, acc[r]);
              acc[r] = fmaf(av.y, v.y, acc[r]);
              acc[r] = fmaf(av.z, v.z, acc[r]);
              acc[r] = fmaf(av.w, v.w, acc[r]);
            }
          }
        }
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(&empty[s]);
      if (c == nchunks - 1) {
        // end of a row group: reduce the RB_ROWS accumulators over the CTA
#pragma unroll
        for (int r = 0; r < RB_ROWS; ++r) {
          Acc v = warp_sum(acc[r]);
          if (lane == 0) red[warp][r] = v;
          acc[r] = Acc(0);
        }
        asm volatile("bar.sync 1, %0;" ::"r"(RB_CONSUMER_WARPS * 32));
        if (threadIdx.x < RB_ROWS) {
          const int row = g * RB_ROWS + threadIdx.x;
          Acc s = Acc(0);
#pragma unroll
          for (int w = 0; w < RB_CONSUMER_WARPS; ++w) s += red[w][threadIdx.x];
          if (row < n) {
            if constexpr (RESID) {
              const double rr = double(a.b[row]) - double(s);
              a.out[row] = float(rr);
              my_part += rr * rr;
            } else {
              a.out[row] = float(s);
              my_part += double(a.v[row]) * double(float(s));
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
      if (!RESID) {
        *a.result = s;
      } else if (st) {
        st->rho_true = s;
        st->matvecs_check += 1;
        st->relres_true = st->bnorm2 > 0.0 ? sqrt(s / st->bnorm2) : sqrt(s);
        st->true_valid = 1;
        const int mode = a.resid_mode >= 0 ? a.resid_mode : st->mode;
        if (mode == 1 && s <= st->thresh2 && st->status == DCG_OK) {
          st->done = 1;
        }
      } else {
        *a.result = s;
      }
    }
  }
}

cudaError_t launch_rowop(const CUtensorMap* tmap, const RowOpArgs& a, bool resid, int grid, cudaStream_t s) {
  if (resid) {
    k_rowop_tma<true><<<grid, RB_THREADS, RB_SMEM, s>>>(*tmap, a);
  } else {
    k_rowop_tma<false><<<grid, RB_THREADS, RB_SMEM, s>>>(*tmap, a);
  }
  return cudaGetLastError();
}

cudaError_t rowop_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_rowop_tma<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(RB_SMEM));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rowop_tma<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(RB_SMEM));
}

int rowop_grid(int n, int num_sms) {
  const int ngroups = (n + RB_ROWS - 1) / RB_ROWS;
  return ngroups < num_sms ? ngroups : num_sms;
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
// Y = A V, V and Y column-major n x c (leading dimension n). CUDA-core tiles of
// 64 rows x BN columns, K-steps of 32; each thread owns a 4 x (BN/16) block.
// The column count is read from the device state when cstate is set (graph
// launches with a per-solve k), otherwise from the argument.
// ---------------------------------------------------------------------------
template <int BN>
__global__ void __launch_bounds__(256) k_apply_block(ApplyBlockArgs a) {
  constexpr int BM = 64, BK = 32, TN = BN / 16;
  __shared__ float As[BK][BM + 4];
  __shared__ float Vs[BK][BN + 4];
  int c = a.c;
  const float* V = a.V;
  float* Y = a.Y;
  if (a.st) {
    if (a.skip_if_done && a.st->done) return;
    const int warm = a.st->warm_start;
    c = a.st->k + warm;
    if (!warm) {
      V += a.n;
      Y += a.n;
    }
  }
  const int n = a.n;
  const int row0 = blockIdx.x * BM, col0 = blockIdx.y * BN;
  if (col0 >= c) return;
  const int t = threadIdx.x, ty = t / 16, tx = t % 16;
  float acc[4][TN];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = 0.f;
  const bool vec_ok = (a.lda % 4) == 0;
  for (int k0 = 0; k0 < n; k0 += BK) {
    // A tile: 64 rows x 32 cols, stored transposed As[kk][row]
    for (int idx = t; idx < BM * (BK / 4); idx += 256) {
      const int r = idx / (BK / 4), c4 = idx % (BK / 4);
      const int gr = row0 + r, gk = k0 + 4 * c4;
      float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
      if (gr < n) {
        const float* src = a.A + int64_t(gr) * a.lda + gk;
        if (vec_ok && gk + 3 < n) {
          v = __ldg(reinterpret_cast<const float4*>(src));
        } else {
          v.x = gk < n ? __ldg(src) : 0.f;
          v.y = gk + 1 < n ? __ldg(src + 1) : 0.f;
          v.z = gk + 2 < n ? __ldg(src + 2) : 0.f;
          v.w = gk + 3 < n ? __ldg(src + 3) : 0.f;
        }
      }
      As[4 * c4 + 0][r] = v.x;
      As[4 * c4 + 1][r] = v.y;
      As[4 * c4 + 2][r] = v.z;
      As[4 * c4 + 3][r] = v.w;
    }
    // V tile: 32 rows (k) x BN cols, Vs[kk][col]
    for (int idx = t; idx < BK * BN; idx += 256) {
      const int j = idx / BK, kk = idx % BK;
      const int gj = col0 + j, gk = k0 + kk;
      Vs[kk][j] = (gj < c && gk < n) ? __ldg(V + int64_t(gj) * n + gk) : 0.f;
    }
    __syncthreads();
#pragma unroll 8
    for (int kk = 0; kk < BK; ++kk) {
      const float4 av = *reinterpret_cast<const float4*>(&As[kk][4 * ty]);
      float vv[TN];
#pragma unroll
      for (int j = 0; j < TN; ++j) vv[j] = Vs[kk][tx + 16 * j];
#pragma unroll
      for (int j = 0; j < TN; ++j) {
        acc[0][j] = fmaf(av.x, vv[j], acc[0][j]);
        acc[1][j] = fmaf(av.y, vv[j], acc[1][j]);
        acc[2][j] = fmaf(av.z, vv[j], acc[2][j]);
        acc[3][j] = fmaf(av.w, vv[j], acc[3][j]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gr = row0 + 4 * ty + i;
    if (gr >= n) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gj = col0 + tx + 16 * j;
      if (gj < c) Y[int64_t(gj) * n + gr] = acc[i][j];
    }
  }
}

cudaError_t launch_apply_block(const ApplyBlockArgs& a, int cmax, cudaStream_t s) {
  if (cmax <= 0) return cudaSuccess;
  if (cmax <= 32) {
    dim3 grid((a.n + 63) / 64, 1);
    k_apply_block<32><<<grid, 256, 0, s>>>(a);
  } else {
    dim3 grid((a.n + 63) / 64, (cmax + 63) / 64);
    k_apply_block<64><<<grid, 256, 0, s>>>(a);
  }
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// A = s^2 exp(-|x_i - x_j|^2 / (2 l^2)) + noise [i == j]  (Sec. 3 RBF kernel)
// 64 x 64 output tiles; X rows of the tile staged in shared memory; float32
// difference-form squared distances.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_form_rbf(const float* __restrict__ X, int n, int d, float neg_inv2l2,
                                                  float s2, float noise, float* __restrict__ A, int64_t lda) {
  extern __shared__ float xs[];  // [2][64][d]
  float* xi = xs;
  float* xj = xs + 64 * d;
  const int i0 = blockIdx.y * 64, j0 = blockIdx.x * 64;
  for (int idx = threadIdx.x; idx < 64 * d; idx += 256) {
    const int r = idx / d, m = idx % d;
    xi[idx] = (i0 + r < n) ? X[int64_t(i0 + r) * d + m] : 0.f;
    xj[idx] = (j0 + r < n) ? X[int64_t(j0 + r) * d + m] : 0.f;
  }
  __syncthreads();
  const int ty = threadIdx.x / 16, tx = threadIdx.x % 16;
  float sq[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 4; ++c) sq[a][c] = 0.f;
  for (int m = 0; m < d; ++m) {
    float u[4], v[4];
#pragma unroll
    for (int a = 0; a < 4; ++a) u[a] = xi[(4 * ty + a) * d + m];
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = xj[(4 * tx + c) * d + m];
#pragma unroll
    for (int a = 0; a < 4; ++a)
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const float df = u[a] - v[c];
        sq[a][c] = fmaf(df, df, sq[a][c]);
      }
  }
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = i0 + 4 * ty + a;
    if (i >= n) continue;
    float out[4];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = j0 + 4 * tx + c;
      out[c] = s2 * expf(sq[a][c] * neg_inv2l2) + (i == j ? noise : 0.f);
    }
    const int j = j0 + 4 * tx;
    float* dst = A + int64_t(i) * lda + j;
    if (j + 3 < n && (lda % 4) == 0) {
      *reinterpret_cast<float4*>(dst) = make_float4(out[0], out[1], out[2], out[3]);
    } else {
      for (int c = 0; c < 4; ++c)
        if (j + c < n) dst[c] = out[c];
    }
  }
}

cudaError_t launch_form_rbf(const float* X, int n, int d, double l, double s2, double noise, float* A, int64_t lda,
                            cudaStream_t s) {
  dim3 grid((n + 63) / 64, (n + 63) / 64);
  const size_t smem = size_t(2) * 64 * d * sizeof(float);
  const float neg_inv2l2 = float(-1.0 / (2.0 * l * l));
  k_form_rbf<<<grid, 256, smem, s>>>(X, n, d, neg_inv2l2, float(s2), float(noise), A, lda);
  return cudaGetLastError();
}

}  // namespace dcg
