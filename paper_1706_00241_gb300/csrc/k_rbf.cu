// Matrix-free RBF operator A = K + noise I, K_ij = s^2 exp(-|x_i - x_j|^2 / (2 l^2))
// (the Sec. 3 kernel), never stored.
//
//   * k_rbf_mv<1>: q = A p with the fused p^T q (Algorithm 1).
//     Persistent, warp-specialised: a TMA warp streams J tiles (128 rows,
//     swizzled) with p_J by a bulk copy; one thread issues tcgen05.mma (BF16
//     or TF32 inputs, float32 accumulation) for S~_ij = x_i . x_j - |x_j|^2 / 2
//     (augmented tile rows, below) into one of four TMEM buffers; sixteen
//     epilogue warps read S~ with
//     tcgen05.ld and accumulate q_i += exp2(2c S~_ij + u_i) p_j with the
//     exponential on the SFU (ex2.approx), c = log2(e) / (2 l^2),
//     u_i = log2(s^2) - c |x_i|^2: one packed FMA per two exponents. Padded
//     columns carry -|x_j|^2/2 = -2^100 (K = 0).
//   * k_rbf_mv<8>: the start-of-solve product A W, eight columns of W per
//     pass, each entry's exponential formed once and contracted with all
//     eight (the same entries as the loop's matvec).
//   * k_rbf_resid + k_rbf_resid_fin: the true residual b - A x on CUDA
//     cores, entries as float32 pairs from distances that are exact up to a
//     small remainder (Gram sums on a fixed grid, see below), a
//     table-driven exponential pair and compensated (Dot2) sums with
//     x = xh + xl; the convergence test includes the entry-error bound.
//     k_rbf_block: the block product A V (dcg_apply_block), entries to ~2 ulp.
//     The tensor-core tiles carry ~1e-5 relative error on close pairs (BF16,
//     TF32 operands); the residual recomputation in the exact form is the
//     refinement that wins the accuracy back.
#include <cuda_bf16.h>
#include <cuda_fp16.h>

#include "dcg_kernels.cuh"
#include "tc.cuh"

namespace dcg {

// ---------------------------------------------------------------------------
// Preparation: rounded X (the operator's points), padded tensor-core copy,
// squared norms; v_j for the current lengthscale.
// ---------------------------------------------------------------------------
__device__ __forceinline__ float round_bf16(float x) { return __bfloat162float(__float2bfloat16_rn(x)); }


// Xr (n x d float32): the operator's points, X rounded to the chosen element
// format (BF16, TF32) or X itself (FP32). Xt: two 128-byte-per-row tile
// copies (BF16: 64 elements, TF32 and FP32: 32 float32 elements holding
// TF32 values) of n_pad rows each, the operands of the tensor-core product
//   S~_ij = x_i . x_j - |x_j|^2 / 2,
// so that the exponent of an entry is one FMA, 2c S~_ij + (log2 s^2 - c |x_i|^2)
// with c = log2(e) / (2 l^2), and S~ does not depend on l:
//   BF16, TF32:  I rows [x_i, 1, 1, 1, 0 ...], J rows [x_j, h_j, m_j, l_j, 0 ...];
//   FP32 (split TF32: x = x_hi + x_lo, x_hi = tf32(x), x_lo = tf32(x - x_hi)):
//                I rows [x_hi, x_hi, x_lo, 1, 1, 1, 0 ...],
//                J rows [x_hi, x_lo, x_hi, h, m, l, 0 ...],
//     so that x_i . x_j = hi.hi + hi.lo + lo.hi to ~2^-21 (the dropped lo.lo
//     and x - x_hi - x_lo are ~2^-22 relative);
// h + m + l = -|x_j|^2 / 2 split into three pieces of the element format (24
// bits for BF16, 33 for TF32); padding rows j >= n carry h = -2^100, so that
// their entries vanish. nsq[i] = |xr_i|^2 (float64 sum, rounded).
constexpr int kRbfAug = 3;  // extra coordinates of the tile copies

// Coordinates of a tile row before the kRbfAug pieces: d, or 3 d for the
// split-TF32 copy of float32 points.
__host__ __device__ int rbf_tile_coords(int xformat, int d) { return xformat == DCG_X_FP32 ? 3 * d : d; }

__global__ void k_rbf_prep(const float* __restrict__ X, int n, int n_pad, int d, int xformat, float* Xr,
                           void* Xt, float* nsq) {
  const int dc = rbf_tile_coords(xformat, d);
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
    double ss = 0.0;
    float va[64], vb[64];   // the tile rows' coordinates (I copy, J copy)
    for (int m = 0; m < d; ++m) {
      float x = 0.f;
      if (i < n) {
        const float x0 = X[int64_t(i) * d + m];
        x = xformat == DCG_X_BF16 ? round_bf16(x0) : (xformat == DCG_X_TF32 ? round_tf32(x0) : x0);
        Xr[int64_t(i) * d + m] = x;
        ss += double(x) * double(x);
      }
      if (xformat == DCG_X_FP32) {
        const float hi = round_tf32(x), lo = round_tf32(x - hi);
        va[m] = hi;  va[d + m] = hi;  va[2 * d + m] = lo;
        vb[m] = hi;  vb[d + m] = lo;  vb[2 * d + m] = hi;
      } else {
        va[m] = vb[m] = x;
      }
    }
    // -|x_i|^2 / 2 in three pieces of the element format
    float piece[kRbfAug];
    double rest = -0.5 * ss;
    for (int k = 0; k < kRbfAug; ++k) {
      piece[k] = xformat == DCG_X_BF16 ? round_bf16(float(rest)) : round_tf32(float(rest));
      rest -= double(piece[k]);
    }
    if (i >= n) {
      piece[0] = -0x1p100f;
      piece[1] = piece[2] = 0.f;
    }
    const int width = xformat == DCG_X_BF16 ? 64 : 32;
    for (int m = 0; m < width; ++m) {
      const bool coord = m < dc, aug = m >= dc && m < dc + kRbfAug;
      const float a = coord ? va[m] : (aug ? 1.f : 0.f);
      const float b = coord ? vb[m] : (aug ? piece[m - dc] : 0.f);
      if (xformat == DCG_X_BF16) {
        reinterpret_cast<__nv_bfloat16*>(Xt)[int64_t(i) * 64 + m] = __float2bfloat16_rn(a);
        reinterpret_cast<__nv_bfloat16*>(Xt)[int64_t(n_pad + i) * 64 + m] = __float2bfloat16_rn(b);
      } else {
        reinterpret_cast<float*>(Xt)[int64_t(i) * 32 + m] = a;
        reinterpret_cast<float*>(Xt)[int64_t(n_pad + i) * 32 + m] = b;
      }
    }
    nsq[i] = float(ss);
  }
}

// vcol[i] = -c nsq[i] (c = log2(e) / (2 l^2)), the row term of the exponent
// (padded rows: -inf). Also writes the scalar parameters.
__global__ void k_rbf_params(const float* nsq, int n, int n_pad, int d, double l, double s2, double noise,
                             float* vcol, RbfParams* prm) {
  const double c = 1.4426950408889634 / (2.0 * l * l);
  for (int j = blockIdx.x * blockDim.x + threadIdx.x; j < n_pad; j += gridDim.x * blockDim.x)
    vcol[j] = j < n ? float(-c * double(nsq[j])) : -INFINITY;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    prm->c2 = float(2.0 * c);
    prm->l2s = float(log2(s2));
    prm->s2 = float(s2);
    prm->noise = float(noise);
    prm->neg_inv2l2 = float(-1.0 / (2.0 * l * l));
    prm->neg_inv2l2_lo = float(-1.0 / (2.0 * l * l) - double(prm->neg_inv2l2));
    prm->s2_lo = float(s2 - double(prm->s2));
    prm->noise_d = noise;
    // distance part of the residual entries' error model (units of u^2,
    // u = 2^-24): (0.87 d + 1) g / (2 l^2) / u, g the anchor grid
    prm->err_dist = float((0.87 * d + 1.0) * double(prm->g_anchor) / (2.0 * l * l) * 16777216.0);
  }
}

cudaError_t launch_rbf_prep(const float* X, int n, int n_pad, int d, int xformat, float* Xr, void* Xt, float* nsq,
                            cudaStream_t s) {
  k_rbf_prep<<<(n_pad + 255) / 256, 256, 0, s>>>(X, n, n_pad, d, xformat, Xr, Xt, nsq);
  return cudaGetLastError();
}

cudaError_t launch_rbf_params(const float* nsq, int n, int n_pad, int d, double l, double s2, double noise,
                              float* vcol, RbfParams* prm, cudaStream_t s) {
  k_rbf_params<<<(n_pad + 255) / 256, 256, 0, s>>>(nsq, n, n_pad, d, l, s2, noise, vcol, prm);
  return cudaGetLastError();
}

// Bytes of one X row the MMA reads: the d coordinates rounded up to a 32, 64
// or 128 byte swizzle row. Loading only these (not the full 128-byte packed
// row) cuts the L2 -> shared traffic, which bounds this kernel: every J tile is
// fetched once per I block.
__host__ __device__ int rbf_row_bytes(int xformat, int d) {
  const int bytes = d * (xformat == DCG_X_BF16 ? 2 : 4);
  return bytes <= 32 ? 32 : (bytes <= 64 ? 64 : 128);
}

static bool make_rbf_tmap_one(CUtensorMap* map, const void* Xt, int n_pad, int xformat, int d,
                              EncodeTiledFn encode);

// Tensor maps of the two tile copies (map[0]: I-tile rows, map[1]: J-tile
// rows), boxes of 128 rows x the row bytes the MMA reads (d + kRbfAug
// coordinates).
bool make_rbf_tmap(CUtensorMap* map, const void* Xt, int n_pad, int xformat, int d, EncodeTiledFn encode) {
  for (int half = 0; half < 2; ++half) {
    const void* base = static_cast<const unsigned char*>(Xt) + size_t(half) * n_pad * 128;
    if (!make_rbf_tmap_one(&map[half], base, n_pad, xformat, rbf_tile_coords(xformat, d) + kRbfAug, encode))
      return false;
  }
  return true;
}

int rbf_max_d(int xformat) {
  const int room = (xformat == DCG_X_BF16 ? 64 : 32) - kRbfAug;
  return xformat == DCG_X_FP32 ? room / 3 : room;
}

static bool make_rbf_tmap_one(CUtensorMap* map, const void* Xt, int n_pad, int xformat, int d, EncodeTiledFn encode) {
  const bool bf = xformat == DCG_X_BF16;
  const int row_bytes = rbf_row_bytes(xformat, d);
  const int esize = bf ? 2 : 4;
  cuuint64_t gdim[2] = {cuuint64_t(bf ? 64 : 32), cuuint64_t(n_pad)};
  cuuint64_t gstride[1] = {128};
  cuuint32_t box[2] = {cuuint32_t(row_bytes / esize), 128};
  cuuint32_t estride[2] = {1, 1};
  const CUtensorMapSwizzle swz = row_bytes == 128 ? CU_TENSOR_MAP_SWIZZLE_128B
                                 : row_bytes == 64 ? CU_TENSOR_MAP_SWIZZLE_64B
                                                   : CU_TENSOR_MAP_SWIZZLE_32B;
  CUresult r = encode(map, bf ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
                      const_cast<void*>(Xt), gdim, gstride, box, estride, CU_TENSOR_MAP_INTERLEAVE_NONE, swz,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

// ---------------------------------------------------------------------------
// Tensor-core matvec
// ---------------------------------------------------------------------------
constexpr int MV_TILE = 128;                // rows of an I block and columns of a J tile
constexpr int MV_STAGES = 6;
constexpr int MV_TILE_BYTES = MV_TILE * 128;  // 16 KB: 128 rows x 128 bytes
constexpr int MV_EPI_WARPS = 16;            // four per SMSP: latency hiding for the exp chains
constexpr int MV_THREADS = (2 + MV_EPI_WARPS) * 32;
constexpr int MV_TBUF = 4;                    // TMEM accumulator buffers (tiles in flight)
constexpr int MV_TMEM_COLS = MV_TBUF * MV_TILE;  // all 512 columns: one CTA per SM
// shared memory: X_I tile, stages of {X_J tile, the NC vector columns p_J
// (column-major, 128 floats each), v_J}, barriers; stages 1024-aligned for
// the swizzled X tiles
constexpr int MV_BLOCK_NC = 8;  // columns per pass of the multi-column product
__host__ __device__ constexpr int mv_stage_bytes(int nc) {
  return (MV_TILE_BYTES + nc * MV_TILE * 4 + 1023) / 1024 * 1024;
}
__host__ __device__ constexpr size_t mv_smem(int nc) {
  return 1024 + MV_TILE_BYTES + size_t(MV_STAGES) * mv_stage_bytes(nc) + 256;
}
constexpr size_t MV_SMEM = mv_smem(1);

// 16 entries of one row (lane) of the matvec epilogue: exponents from the
// Gram values h (float bits) as 2c S~ + u in packed pairs, exponentials on the
// SFU, contraction with p_j into two packed sums (entries j = 0, 1 mod 4 and
// 2, 3 mod 4).
__device__ __forceinline__ void mv_half(const uint32_t (&h)[16], const float* pj, unsigned long long c2x2,
                                        unsigned long long uu, unsigned long long& sA, unsigned long long& sB) {
#pragma unroll
  for (int j = 0; j < 16; j += 4) {
    const float4 p4 = *reinterpret_cast<const float4*>(pj + j);
    const unsigned long long g01 =
        tc::f2fma(c2x2, tc::f2pk(__uint_as_float(h[j + 0]), __uint_as_float(h[j + 1])), uu);
    const unsigned long long g23 =
        tc::f2fma(c2x2, tc::f2pk(__uint_as_float(h[j + 2]), __uint_as_float(h[j + 3])), uu);
    const unsigned long long e01 = tc::f2pk(tc::ex2_approx(tc::f2lo(g01)), tc::ex2_approx(tc::f2hi(g01)));
    const unsigned long long e23 = tc::f2pk(tc::ex2_approx(tc::f2lo(g23)), tc::ex2_approx(tc::f2hi(g23)));
    sA = tc::f2fma(e01, tc::f2pk(p4.x, p4.y), sA);
    sB = tc::f2fma(e23, tc::f2pk(p4.z, p4.w), sB);
  }
}

// NC = 1: q = A p with the fused p^T q. NC > 1 (the start-of-solve product):
// Y[:, col0 + c] = A V[:, col0 + c] for the NC columns of a group, each
// entry's exponential formed once and contracted with all NC columns
// (columns at or beyond k are read but not written).
template <int NC>
__global__ void __launch_bounds__(MV_THREADS, 1)
    k_rbf_mv(const __grid_constant__ CUtensorMap tmap_i, const __grid_constant__ CUtensorMap tmap_j, RbfMvArgs a) {
  constexpr int MV_STAGE_BYTES = mv_stage_bytes(NC);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* xi_tile = base;                                   // 1024-aligned
  unsigned char* stages = base + MV_TILE_BYTES;                    // each stage 1024-aligned (16 KB + 1 KB)
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + size_t(MV_STAGES) * MV_STAGE_BYTES);
  uint64_t* full = bars;                       // [MV_STAGES]
  uint64_t* empty = full + MV_STAGES;          // [MV_STAGES]
  uint64_t* tfull = empty + MV_STAGES;         // [MV_TBUF]
  uint64_t* tempty = tfull + MV_TBUF;          // [MV_TBUF]
  uint64_t* xi_full = tempty + MV_TBUF;
  uint64_t* xi_empty = xi_full + 1;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ float s_slice[3][MV_TILE];
  __shared__ double s_part[MV_EPI_WARPS];

  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  if (st && a.col_idx >= 0 && a.col_idx >= st->k) return;
  const int ncw = (st && a.col_idx >= 0) ? min(NC, st->k - a.col_idx) : a.ncols;  // columns written

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, n_tiles = a.n_tiles;
  const int kind_tf32 = a.xformat != DCG_X_BF16;
  const int dk = rbf_tile_coords(a.xformat, a.d) + kRbfAug;         // coordinates of the tile rows
  const int ksteps = kind_tf32 ? (dk + 7) / 8 : (dk + 15) / 16;     // 32-byte K steps
  const uint32_t row_bytes = uint32_t(rbf_row_bytes(a.xformat, dk));
  const uint32_t tile_bytes = MV_TILE * row_bytes;                  // bytes of one X tile in use
  const uint32_t idesc = tc::instr_desc(kind_tf32 ? tc::kFmtTF32 : tc::kFmtBF16, MV_TILE, MV_TILE);

  if (threadIdx.x == 0) {
    for (int s = 0; s < MV_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], MV_EPI_WARPS);
    }
    for (int b = 0; b < MV_TBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], MV_EPI_WARPS);
    }
    mbar_init(xi_full, 1);
    mbar_init(xi_empty, 1);
    fence_mbarrier_init();
    s_abort = 0;
  }
  if (warp == 1) tc::tmem_alloc(&s_tmem, MV_TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  double my_part = 0.0;
  if (warp == 0) {
    // -------------------------------- producer ------------------------------
    if (lane == 0) {
      prefetch_tensormap(&tmap_i);
      prefetch_tensormap(&tmap_j);
      long long it = 0;
      int rbc = 0;
      for (int rb = blockIdx.x; rb < n_tiles && !s_abort; rb += gridDim.x, ++rbc) {
        if (rbc > 0 && !mbar_wait_bounded(xi_empty, (rbc - 1) & 1)) { s_abort = 1; break; }
        mbar_arrive_expect_tx(xi_full, tile_bytes);
        tma_load_2d(xi_tile, &tmap_i, xi_full, 0, rb * MV_TILE);
        for (int J = 0; J < n_tiles; ++J, ++it) {
          const int s = int(it % MV_STAGES);
          if (it >= MV_STAGES && !mbar_wait_bounded(&empty[s], uint32_t((it / MV_STAGES) - 1) & 1)) {
            s_abort = 1;
            break;
          }
          unsigned char* stg = stages + size_t(s) * MV_STAGE_BYTES;
          mbar_arrive_expect_tx(&full[s], tile_bytes + NC * MV_TILE * 4);
          tma_load_2d(stg, &tmap_j, &full[s], 0, J * MV_TILE);
#pragma unroll 1
          for (int c = 0; c < NC; ++c)
            tc::bulk_load(stg + MV_TILE_BYTES + c * MV_TILE * 4, a.p + size_t(c) * a.ldp + size_t(J) * MV_TILE,
                          MV_TILE * 4, &full[s]);
        }
      }
    }
  } else if (warp == 1) {
    // -------------------------------- MMA issuer -----------------------------
    if (lane == 0) {
      long long it = 0;
      int rbc = 0;
      const uint32_t a_base = smem_u32(xi_tile);
      for (int rb = blockIdx.x; rb < n_tiles && !s_abort; rb += gridDim.x, ++rbc) {
        if (!mbar_wait_bounded(xi_full, rbc & 1)) { s_abort = 1; break; }
        tc::fence_after_sync();
        for (int J = 0; J < n_tiles; ++J, ++it) {
          const int s = int(it % MV_STAGES);
          const int b = int(it % MV_TBUF);
          if (!mbar_wait_bounded(&full[s], uint32_t(it / MV_STAGES) & 1)) { s_abort = 1; break; }
          if (it >= MV_TBUF && !mbar_wait_bounded(&tempty[b], uint32_t((it / MV_TBUF) - 1) & 1)) {
            s_abort = 1;
            break;
          }
          tc::fence_after_sync();
          const uint32_t b_base = smem_u32(stages + size_t(s) * MV_STAGE_BYTES);
          const uint32_t d_tmem = tmem + uint32_t(b * MV_TILE);
          for (int kk = 0; kk < ksteps; ++kk) {
            const uint64_t ad = tc::smem_desc_kmajor(a_base + 32 * kk, row_bytes);
            const uint64_t bd = tc::smem_desc_kmajor(b_base + 32 * kk, row_bytes);
            if (kind_tf32)
              tc::mma_tf32(d_tmem, ad, bd, idesc, kk > 0);
            else
              tc::mma_bf16(d_tmem, ad, bd, idesc, kk > 0);
          }
          tc::mma_commit(&tfull[b]);
        }
        tc::mma_commit(xi_empty);
      }
    }
  } else {
    // -------------------------------- epilogue -------------------------------
    const int ew = warp - 2;                  // 0..15
    const int quarter = warp & 3;             // TMEM lane quarter this warp may access
    const int slice = ew >> 2;                // 32-column slice of the tile
    const int row_l = quarter * 32 + lane;    // row within the I block
    const float c2 = a.prm->c2, l2s = a.prm->l2s, noise = a.prm->noise;
    long long it = 0;
    for (int rb = blockIdx.x; rb < n_tiles; rb += gridDim.x) {
      const int row = rb * MV_TILE + row_l;
      // exponent of an entry: c2 S~_ij + u_i, u_i = log2 s^2 - c |x_i|^2
      const float u = l2s + a.vcol[row];        // vcol has n_pad entries
      float acc[NC], comp[NC];                  // Kahan sums of per-tile partials
#pragma unroll
      for (int c = 0; c < NC; ++c) acc[c] = comp[c] = 0.f;
      bool aborted = false;
      if constexpr (NC == 1) {
        // Software-pipelined in half slices of 16 columns: the TMEM load of
        // the next half (or of the next tile's first half) is in flight while
        // the current half is processed.
        const unsigned long long c2x2 = tc::f2pk(c2, c2), uu = tc::f2pk(u, u);
        const uint32_t lane_off = uint32_t(quarter * 32) << 16;
        uint32_t ha[16], hb[16];
        {
          const int b = int(it % MV_TBUF);
          if (!mbar_wait_bounded(&tfull[b], uint32_t(it / MV_TBUF) & 1)) {
            s_abort = 1;
            aborted = true;
          } else {
            tc::fence_after_sync();
            tc::tmem_ld16_nowait(tmem + lane_off + uint32_t(b * MV_TILE + slice * 32), ha);
            tc::tmem_wait_ld16(ha);
          }
        }
        for (int J = 0; J < n_tiles && !aborted; ++J, ++it) {
          const int s = int(it % MV_STAGES);
          const int b = int(it % MV_TBUF);
          const float* pj =
              reinterpret_cast<const float*>(stages + size_t(s) * MV_STAGE_BYTES + MV_TILE_BYTES) + slice * 32;
          tc::tmem_ld16_nowait(tmem + lane_off + uint32_t(b * MV_TILE + slice * 32 + 16), hb);
          unsigned long long s0 = 0ull, s1 = 0ull, s2 = 0ull, s3 = 0ull;
          mv_half(ha, pj, c2x2, uu, s0, s1);
          tc::tmem_wait_ld16(hb);
          // the whole slice is in registers: the accumulator goes back to the
          // MMA warp (the stage with p is released after the math)
          tc::fence_before_sync();
          __syncwarp();
          if (lane == 0) mbar_arrive(&tempty[b]);
          const bool next = J + 1 < n_tiles;
          if (next) {
            const int b2 = int((it + 1) % MV_TBUF);
            if (!mbar_wait_bounded(&tfull[b2], uint32_t((it + 1) / MV_TBUF) & 1)) {
              s_abort = 1;
              aborted = true;
            } else {
              tc::fence_after_sync();
              tc::tmem_ld16_nowait(tmem + lane_off + uint32_t(b2 * MV_TILE + slice * 32), ha);
            }
          }
          mv_half(hb, pj + 16, c2x2, uu, s2, s3);
          __syncwarp();
          if (lane == 0) mbar_arrive(&empty[s]);
          if (next && !aborted) tc::tmem_wait_ld16(ha);
          const float part = ((tc::f2lo(s0) + tc::f2hi(s0)) + (tc::f2lo(s1) + tc::f2hi(s1))) +
                             ((tc::f2lo(s2) + tc::f2hi(s2)) + (tc::f2lo(s3) + tc::f2hi(s3)));
          const float y = part - comp[0];
          const float t = acc[0] + y;
          comp[0] = (t - acc[0]) - y;
          acc[0] = t;
        }
      } else {
      for (int J = 0; J < n_tiles; ++J, ++it) {
        const int s = int(it % MV_STAGES);
        const int b = int(it % MV_TBUF);
        if (!mbar_wait_bounded(&tfull[b], uint32_t(it / MV_TBUF) & 1)) { s_abort = 1; aborted = true; break; }
        tc::fence_after_sync();
        const unsigned char* stg = stages + size_t(s) * MV_STAGE_BYTES;
        const float* pj = reinterpret_cast<const float*>(stg + MV_TILE_BYTES) + slice * 32;
        float sv[32];
        tc::tmem_ld32(tmem + (uint32_t(quarter * 32) << 16) + uint32_t(b * MV_TILE + slice * 32), sv);
        // the values are in registers: hand the accumulator back to the MMA
        // warp before the math (the stage with p is released after it)
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
        {
          // the entries, once, as packed pairs (j, j + 1); then per column two
          // packed sums (pairs 0, 2 mod 4 and 1, 3 mod 4): one FMA
          // instruction per two entries
          const unsigned long long c2x2 = tc::f2pk(c2, c2), uu = tc::f2pk(u, u);
          unsigned long long e2[16];
#pragma unroll
          for (int j = 0; j < 32; j += 2) {
            const unsigned long long g = tc::f2fma(c2x2, tc::f2pk(sv[j], sv[j + 1]), uu);
            e2[j / 2] = tc::f2pk(tc::ex2_approx(tc::f2lo(g)), tc::ex2_approx(tc::f2hi(g)));
          }
#pragma unroll
          for (int c = 0; c < NC; ++c) {  // contracted with every column
            const float* pc = pj + c * MV_TILE;
            unsigned long long s0 = 0ull, s1 = 0ull;
#pragma unroll
            for (int j = 0; j < 32; j += 8) {
              const float4 pa4 = *reinterpret_cast<const float4*>(pc + j);
              const float4 pb4 = *reinterpret_cast<const float4*>(pc + j + 4);
              s0 = tc::f2fma(e2[j / 2 + 0], tc::f2pk(pa4.x, pa4.y), s0);
              s1 = tc::f2fma(e2[j / 2 + 1], tc::f2pk(pa4.z, pa4.w), s1);
              s0 = tc::f2fma(e2[j / 2 + 2], tc::f2pk(pb4.x, pb4.y), s0);
              s1 = tc::f2fma(e2[j / 2 + 3], tc::f2pk(pb4.z, pb4.w), s1);
            }
            const float y = ((tc::f2lo(s0) + tc::f2hi(s0)) + (tc::f2lo(s1) + tc::f2hi(s1))) - comp[c];
            const float t = acc[c] + y;
            comp[c] = (t - acc[c]) - y;
            acc[c] = t;
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
      }
      }
      if (aborted) break;
      // combine the four column slices of each row (named barrier: epilogue warps)
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if (slice > 0) s_slice[slice - 1][row_l] = acc[c];
        asm volatile("bar.sync 1, %0;" ::"r"(MV_EPI_WARPS * 32));
        if (slice == 0 && row < n) {
          const float tot = acc[c] + ((s_slice[0][row_l] + s_slice[1][row_l]) + s_slice[2][row_l]);
          if constexpr (NC == 1) {
            const float pi = a.p[row];
            const float q = tot + noise * pi;
            a.q[row] = q;
            my_part += double(pi) * double(q);
          } else {
            if (c < ncw) a.q[int64_t(c) * a.ldq + row] = tot + noise * a.p[int64_t(c) * a.ldp + row];
          }
        }
        asm volatile("bar.sync 1, %0;" ::"r"(MV_EPI_WARPS * 32));
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, MV_TMEM_COLS);
  }
  if (s_abort && threadIdx.x == 0 && st) {
    st->status = DCG_ERR_TIMEOUT;
    st->timeout_site = 3;
    st->done = 1;
  }
  if constexpr (NC > 1) return;
  // p^T q: CTA partial, then the last CTA sums in a fixed order
  if (warp >= 2) {
    const double v = warp_sum(my_part);
    if (lane == 0) s_part[warp - 2] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < MV_EPI_WARPS; ++w) s += s_part[w];
    a.partials[blockIdx.x] = s;
  }
  if (!arrive_last(a.ticket)) return;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = lane; i < int(gridDim.x); i += 32) s += a.partials[i];
    s = warp_sum(s);
    if (lane == 0 && a.result) *a.result = s;
  }
}


// ---------------------------------------------------------------------------
// Block product Q = A P for up to 32 columns with the contraction on the
// tensor cores (k_rbf_mv_tc): the systems of a lockstep solve share one pass
// over the kernel entries per iteration. k_rbf_mv<8> contracts the entries
// with the columns of P on the FP32 pipe, where every p_j reaches the 32 rows
// of a warp as a shared-memory broadcast (one wavefront per float per warp,
// 4096 per 128 x 128 tile for 8 columns: the pass is bound by the shared
// memory pipe). Here the entries go to shared memory once and a second MMA
// contracts them with all columns:
//   MMA 1  S~ = X_I X_J^T (as in k_rbf_mv) into one of three TMEM buffers;
//   epilogue  E_ij = exp2(c2 S~_ij + u'_i) = K_ij / s^2 (in [0, 1]), split
//          E = E_hi + E_lo into two float16 parts (E_hi = fp16(E) rounded to
//          nearest, E_lo = fp16(E - E_hi); E - E_hi is exact in float32) and
//          stored as the A operand (K-major, 128-byte swizzle, two 64-column
//          halves per part);
//   MMA 2  D += E_hi P_hi + E_hi P_lo + E_lo P_hi over the 128 columns of the
//          tile (K = 16 per MMA; per K step one MMA of N = 2 NCP against
//          [P_hi; P_lo] stacked as one operand and one of N = NCP against
//          P_hi: 16 MMAs), D (128 x 2 NCP float32: [E_hi P_hi + E_lo P_hi |
//          E_hi P_lo]) in one of two TMEM buffers; P = P_hi + P_lo is each
//          column of P scaled by a power of two sigma_c (max |p| sigma_c in
//          [1/2, 1)) and split like E (k_rbf_p16, once per pass);
//   flush  each epilogue warp reads its NCP / 4 columns of both groups of D
//          one tile behind, adds the groups and adds the sum into float32
//          registers (Kahan), so the tensor core accumulates one tile (8 K
//          steps) at a time;
//   end    q_c = s^2 / sigma_c (D sum) + noise p_c per row.
// The dropped E_lo P_lo term and the float16 roundings of the parts leave
// ~2^-22 relative per product plus 2^-25 absolute (E_lo below the float16
// normal range), far inside the BF16 and TF32 tiles' own entry errors.
// ---------------------------------------------------------------------------
constexpr int TC_SBUF = 3;                    // TMEM buffers of S~
constexpr int TC_STAGES = 4;
constexpr int TC_MAXC = 32;                   // columns per pass (NCP = 16 or 32)
constexpr int TC_E_PART = 2 * MV_TILE * 128;  // one part of E: two halves of 128 rows x 128 bytes = 32 KB
__host__ __device__ constexpr int tc_stage_bytes(int ncp) { return MV_TILE_BYTES + 4 * ncp * 128; }
__host__ __device__ constexpr size_t tc_smem(int ncp) {
  return 1024 + MV_TILE_BYTES + size_t(TC_STAGES) * tc_stage_bytes(ncp) + 2 * size_t(TC_E_PART) + 256;
}

namespace tc {
// 32 lanes x 4 / 8 consecutive 32-bit columns (lane l: row lane base + l).
__device__ __forceinline__ void tmem_ld4(uint32_t taddr, float (&v)[4]) {
  uint32_t r[4];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0, %1, %2, %3}, [%4];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 4; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}
constexpr uint32_t kFmtF16 = 0;  // A / B format code of kind::f16 for float16
}  // namespace tc

// P (ncols columns of length n_pad, leading dimension ldp, zero beyond n) to
// the float16 parts of the contraction's B operand: rows c of PHL hold
// fp16(sigma_c p_c), rows TC_MAXC + c fp16(sigma_c p_c - that), rows of
// columns >= ncols zero; sigma_c = 2^-e with max_j |p_cj| = f 2^e, f in
// [1/2, 1) (1 for a zero column), into pscale[c]. One CTA per column.
__global__ void __launch_bounds__(1024) k_rbf_p16(const float* __restrict__ P, int64_t ldp, int ncols, int n_pad,
                                                  __half* __restrict__ PHL, float* __restrict__ pscale) {
  __shared__ float red[32];
  const int c = blockIdx.x;
  __half* hi = PHL + int64_t(c) * n_pad;
  __half* lo = PHL + int64_t(TC_MAXC + c) * n_pad;
  if (c >= ncols) {
    for (int j = threadIdx.x; j < n_pad; j += blockDim.x) hi[j] = lo[j] = __float2half_rn(0.f);
    if (threadIdx.x == 0) pscale[c] = 1.f;
    return;
  }
  const float* p = P + int64_t(c) * ldp;
  float m = 0.f;
  for (int j = threadIdx.x; j < n_pad; j += blockDim.x) m = fmaxf(m, fabsf(p[j]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < int(blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    if (threadIdx.x == 0) {
      int e = 0;
      if (v > 0.f && isfinite(v)) frexpf(v, &e);
      red[0] = ldexpf(1.f, -e);
    }
  }
  __syncthreads();
  const float sigma = red[0];
  for (int j = threadIdx.x; j < n_pad; j += blockDim.x) {
    const float v = p[j] * sigma;  // exact: a power of two
    const __half h = __float2half_rn(v);
    hi[j] = h;
    lo[j] = __float2half_rn(v - __half2float(h));
  }
  if (threadIdx.x == 0) pscale[c] = sigma;
}

// Roles as in k_rbf_mv: warp 0 TMA (X_I per row block; per tile X_J and the
// four float16 boxes of P_J), warp 1 MMA issue (MMA 1 up to two tiles ahead of
// MMA 2), warps 2..17 epilogue (TMEM lane quarter warp % 4, 32-column slice
// (warp - 2) / 4; D columns slice * NCP / 4 .. + NCP / 4). Every wait is
// bounded; a CTA that gives up records a timeout in a.st (site 3).
template <int NCP>
__global__ void __launch_bounds__(MV_THREADS, 1)
    k_rbf_mv_tc(const __grid_constant__ CUtensorMap tmap_i, const __grid_constant__ CUtensorMap tmap_j,
                const __grid_constant__ CUtensorMap tmap_p, RbfMvArgs a, const float* __restrict__ pscale) {
  constexpr int SB = tc_stage_bytes(NCP);
  constexpr int PB = NCP * 128;  // one box of P_J: NCP rows x 64 float16 (128 bytes)
  constexpr int CPW = NCP / 4;   // D columns per epilogue warp
  // TMEM column of the first D buffer; buffers 64 apart, each 2 NCP columns:
  // [E_hi P_hi + E_lo P_hi | E_hi P_lo]
  constexpr uint32_t D_COL = TC_SBUF * MV_TILE;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* xi_tile = base;
  unsigned char* stages = base + MV_TILE_BYTES;
  unsigned char* e_tile = stages + size_t(TC_STAGES) * SB;  // E_hi halves 0, 1, then E_lo halves 0, 1
  uint64_t* bars = reinterpret_cast<uint64_t*>(e_tile + 2 * TC_E_PART);
  uint64_t* full = bars;                 // [TC_STAGES]
  uint64_t* empty = full + TC_STAGES;    // [TC_STAGES] released by MMA 2 of the tile
  uint64_t* tfull = empty + TC_STAGES;   // [TC_SBUF]
  uint64_t* tempty = tfull + TC_SBUF;    // [TC_SBUF]
  uint64_t* efull = tempty + TC_SBUF;    // E of the tile written
  uint64_t* eempty = efull + 1;          // MMA 2 done with E
  uint64_t* dfull = eempty + 1;          // [2]
  uint64_t* dempty = dfull + 2;          // [2]
  uint64_t* xi_full = dempty + 2;
  uint64_t* xi_empty = xi_full + 1;
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;

  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n = a.n, n_tiles = a.n_tiles;
  const int nrb = int(blockIdx.x) < n_tiles ? (n_tiles - 1 - int(blockIdx.x)) / int(gridDim.x) + 1 : 0;
  const long long T = (long long)nrb * n_tiles;  // tiles of this CTA
  const int kind_tf32 = a.xformat != DCG_X_BF16;
  const int dk = rbf_tile_coords(a.xformat, a.d) + kRbfAug;
  const int ksteps = kind_tf32 ? (dk + 7) / 8 : (dk + 15) / 16;
  const uint32_t row_bytes = uint32_t(rbf_row_bytes(a.xformat, dk));
  const uint32_t tile_bytes = MV_TILE * row_bytes;
  const uint32_t idesc1 = tc::instr_desc(kind_tf32 ? tc::kFmtTF32 : tc::kFmtBF16, MV_TILE, MV_TILE);
  const uint32_t idesc2 = tc::instr_desc(tc::kFmtF16, MV_TILE, NCP);       // E_lo P_hi
  const uint32_t idesc2w = tc::instr_desc(tc::kFmtF16, MV_TILE, 2 * NCP);  // E_hi [P_hi | P_lo]

  if (threadIdx.x == 0) {
    for (int s = 0; s < TC_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < TC_SBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], MV_EPI_WARPS);
    }
    mbar_init(efull, MV_EPI_WARPS);
    mbar_init(eempty, 1);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&dfull[b], 1);
      mbar_init(&dempty[b], MV_EPI_WARPS);
    }
    mbar_init(xi_full, 1);
    mbar_init(xi_empty, 1);
    fence_mbarrier_init();
    s_abort = 0;
  }
  if (warp == 1) tc::tmem_alloc(&s_tmem, MV_TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    // -------------------------------- producer ------------------------------
    if (lane == 0) {
      prefetch_tensormap(&tmap_i);
      prefetch_tensormap(&tmap_j);
      prefetch_tensormap(&tmap_p);
      long long t = 0;
      for (int rbc = 0; rbc < nrb && !s_abort; ++rbc) {
        const int rb = int(blockIdx.x) + rbc * int(gridDim.x);
        if (rbc > 0 && !mbar_wait_bounded(xi_empty, uint32_t(rbc - 1) & 1)) { s_abort = 1; break; }
        mbar_arrive_expect_tx(xi_full, tile_bytes);
        tma_load_2d(xi_tile, &tmap_i, xi_full, 0, rb * MV_TILE);
        bool stop = false;
        for (int J = 0; J < n_tiles; ++J, ++t) {
          const int s = int(t % TC_STAGES);
          if (t >= TC_STAGES && !mbar_wait_bounded(&empty[s], uint32_t((t / TC_STAGES) - 1) & 1)) {
            s_abort = 1;
            stop = true;
            break;
          }
          unsigned char* stg = stages + size_t(s) * SB;
          mbar_arrive_expect_tx(&full[s], tile_bytes + 4 * PB);
          tma_load_2d(stg, &tmap_j, &full[s], 0, J * MV_TILE);
          // per half of the tile's columns, P_hi then P_lo: one B operand of 2 NCP rows
          tma_load_2d(stg + MV_TILE_BYTES, &tmap_p, &full[s], J * MV_TILE, 0);                    // P_hi j 0..63
          tma_load_2d(stg + MV_TILE_BYTES + PB, &tmap_p, &full[s], J * MV_TILE, TC_MAXC);         // P_lo j 0..63
          tma_load_2d(stg + MV_TILE_BYTES + 2 * PB, &tmap_p, &full[s], J * MV_TILE + 64, 0);      // P_hi j 64..127
          tma_load_2d(stg + MV_TILE_BYTES + 3 * PB, &tmap_p, &full[s], J * MV_TILE + 64, TC_MAXC);
        }
        if (stop) break;
      }
    }
  } else if (warp == 1) {
    // -------------------------------- MMA issuer -----------------------------
    if (lane == 0) {
      const uint32_t a1 = smem_u32(xi_tile);
      const uint32_t e_base = smem_u32(e_tile);
      long long m1 = 0;  // next tile of MMA 1
      for (long long u = 0; u < T; ++u) {
        bool ok = true;
        // MMA 1 (the Gram tile S~) up to TC_SBUF - 1 tiles ahead of MMA 2
        while (ok && m1 < T && m1 <= u + TC_SBUF - 1) {
          const int J = int(m1 % n_tiles), rbc = int(m1 / n_tiles);
          const int s = int(m1 % TC_STAGES), b = int(m1 % TC_SBUF);
          if ((J == 0 && !mbar_wait_bounded(xi_full, uint32_t(rbc) & 1)) ||
              !mbar_wait_bounded(&full[s], uint32_t(m1 / TC_STAGES) & 1) ||
              (m1 >= TC_SBUF && !mbar_wait_bounded(&tempty[b], uint32_t((m1 / TC_SBUF) - 1) & 1))) {
            ok = false;
            break;
          }
          tc::fence_after_sync();
          const uint32_t b1 = smem_u32(stages + size_t(s) * SB);
          const uint32_t d1 = tmem + uint32_t(b * MV_TILE);
          for (int kk = 0; kk < ksteps; ++kk) {
            const uint64_t ad = tc::smem_desc_kmajor(a1 + 32 * kk, row_bytes);
            const uint64_t bd = tc::smem_desc_kmajor(b1 + 32 * kk, row_bytes);
            if (kind_tf32)
              tc::mma_tf32(d1, ad, bd, idesc1, kk > 0);
            else
              tc::mma_bf16(d1, ad, bd, idesc1, kk > 0);
          }
          tc::mma_commit(&tfull[b]);
          if (J == n_tiles - 1) tc::mma_commit(xi_empty);
          ++m1;
        }
        if (!ok) { s_abort = 1; break; }
        // MMA 2 of tile u: D = E_hi P_hi + E_hi P_lo + E_lo P_hi over its 128 columns
        const int s = int(u % TC_STAGES), bd = int(u & 1);
        if (!mbar_wait_bounded(efull, uint32_t(u & 1)) ||
            (u >= 2 && !mbar_wait_bounded(&dempty[bd], uint32_t((u >> 1) - 1) & 1))) {
          s_abort = 1;
          break;
        }
        tc::fence_after_sync();
        const uint32_t pb = smem_u32(stages + size_t(s) * SB + MV_TILE_BYTES);
        const uint32_t d2 = tmem + D_COL + uint32_t(bd * 64);
#pragma unroll 1
        for (int kk = 0; kk < 8; ++kk) {
          const uint32_t h = uint32_t(kk >> 2), ko = uint32_t(kk & 3) * 32;
          const uint64_t eh = tc::smem_desc_kmajor(e_base + h * (MV_TILE * 128) + ko, 128);
          const uint64_t el = tc::smem_desc_kmajor(e_base + TC_E_PART + h * (MV_TILE * 128) + ko, 128);
          const uint64_t phl = tc::smem_desc_kmajor(pb + h * (2 * PB) + ko, 128);  // [P_hi; P_lo], 2 NCP rows
          tc::mma_bf16(d2, eh, phl, idesc2w, kk > 0);  // kind::f16; the formats come from the descriptor
          tc::mma_bf16(d2, el, phl, idesc2, 1);        // the first NCP rows of the same operand: P_hi
        }
        tc::mma_commit(&empty[s]);
        tc::mma_commit(eempty);
        tc::mma_commit(&dfull[bd]);
      }
    }
  } else {
    // -------------------------------- epilogue -------------------------------
    const int ew = warp - 2;
    const int quarter = warp & 3;
    const int slice = ew >> 2;
    const int row_l = quarter * 32 + lane;
    const float c2 = a.prm->c2, s2 = a.prm->s2, noise = a.prm->noise;
    const unsigned long long c2x2 = tc::f2pk(c2, c2);
    const uint32_t lane_off = uint32_t(quarter * 32) << 16;
    // this row's 128-byte line of E_hi in the half holding the slice's columns
    // (E_lo TC_E_PART further); 16-byte chunk m of the slice lands at chunk
    // ((slice & 1) * 4 + m) ^ (row & 7) (128-byte swizzle)
    unsigned char* e_row = e_tile + (slice >> 1) * (MV_TILE * 128) + row_l * 128;
    const int ch0 = (slice & 1) * 4, sw = row_l & 7;
    float acc[CPW], comp[CPW];
    // adds D of tile tt (its NCP / 4 columns of this warp) into acc
    auto flush = [&](long long tt) -> bool {
      const int bd = int(tt & 1);
      if (!mbar_wait_bounded(&dfull[bd], uint32_t(tt >> 1) & 1)) return false;
      tc::fence_after_sync();
      float dv[CPW], dw[CPW];
      const uint32_t ta = tmem + lane_off + D_COL + uint32_t(bd * 64 + slice * CPW);
      if constexpr (CPW == 4) {
        tc::tmem_ld4(ta, dv);
        tc::tmem_ld4(ta + NCP, dw);
      } else {
        tc::tmem_ld8(ta, dv);
        tc::tmem_ld8(ta + NCP, dw);
      }
#pragma unroll
      for (int k = 0; k < CPW; ++k) dv[k] += dw[k];  // + E_hi P_lo
      tc::fence_before_sync();
      __syncwarp();
      if (lane == 0) mbar_arrive(&dempty[bd]);
#pragma unroll
      for (int k = 0; k < CPW; ++k) {
        const float y = dv[k] - comp[k];
        const float t2 = acc[k] + y;
        comp[k] = (t2 - acc[k]) - y;
        acc[k] = t2;
      }
      return true;
    };
    long long t = 0;
    bool aborted = false;
    for (int rbc = 0; rbc < nrb && !aborted; ++rbc) {
      const int rb = int(blockIdx.x) + rbc * int(gridDim.x);
      const int row = rb * MV_TILE + row_l;
      const float u = a.vcol[row];  // -c |x_i|^2 (n_pad entries, -inf beyond n): E = K / s^2
      const unsigned long long uu = tc::f2pk(u, u);
#pragma unroll
      for (int k = 0; k < CPW; ++k) acc[k] = comp[k] = 0.f;
      for (int J = 0; J < n_tiles; ++J, ++t) {
        const int b = int(t % TC_SBUF);
        if (!mbar_wait_bounded(&tfull[b], uint32_t(t / TC_SBUF) & 1)) { aborted = true; break; }
        tc::fence_after_sync();
        float sv[32];
        tc::tmem_ld32(tmem + lane_off + uint32_t(b * MV_TILE + slice * 32), sv);
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
        // the entries of the row's 32 columns, split into float16 parts
        uint32_t hi2[16], lo2[16];
#pragma unroll
        for (int k = 0; k < 16; ++k) {
          const unsigned long long g = tc::f2fma(c2x2, tc::f2pk(sv[2 * k], sv[2 * k + 1]), uu);
          const float e0 = tc::ex2_approx(tc::f2lo(g)), e1 = tc::ex2_approx(tc::f2hi(g));
          const __half2 h = __floats2half2_rn(e0, e1);
          const float2 hf = __half22float2(h);
          const __half2 l = __floats2half2_rn(e0 - hf.x, e1 - hf.y);  // exact differences
          hi2[k] = *reinterpret_cast<const uint32_t*>(&h);
          lo2[k] = *reinterpret_cast<const uint32_t*>(&l);
        }
        // E of the previous tile has been read by its MMA 2
        if (t > 0 && !mbar_wait_bounded(eempty, uint32_t(t - 1) & 1)) { aborted = true; break; }
        tc::fence_after_sync();
#pragma unroll
        for (int m = 0; m < 4; ++m) {
          const int ch = (ch0 + m) ^ sw;
          *reinterpret_cast<uint4*>(e_row + ch * 16) =
              make_uint4(hi2[4 * m], hi2[4 * m + 1], hi2[4 * m + 2], hi2[4 * m + 3]);
          *reinterpret_cast<uint4*>(e_row + TC_E_PART + ch * 16) =
              make_uint4(lo2[4 * m], lo2[4 * m + 1], lo2[4 * m + 2], lo2[4 * m + 3]);
        }
        fence_proxy_async_smem();  // the stores, visible to the tensor core's reads
        __syncwarp();
        if (lane == 0) mbar_arrive(efull);
        // D of the previous tile of this row block (one tile behind, so that
        // MMA 2 of it has long finished)
        if (J > 0 && !flush(t - 1)) { aborted = true; break; }
      }
      if (aborted) break;
      if (!flush(t - 1)) { aborted = true; break; }  // the row block's last tile
      if (row < n) {
#pragma unroll
        for (int k = 0; k < CPW; ++k) {
          const int c = slice * CPW + k;
          if (c < a.ncols)
            a.q[int64_t(c) * a.ldq + row] = acc[k] * (s2 / pscale[c]) + noise * a.p[int64_t(c) * a.ldp + row];
        }
      }
    }
    if (aborted) s_abort = 1;
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, MV_TMEM_COLS);
  }
  if (s_abort && threadIdx.x == 0 && st) {
    st->status = DCG_ERR_TIMEOUT;
    st->timeout_site = 3;
    st->done = 1;
  }
}

cudaError_t rbf_mv_tc_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_rbf_mv_tc<16>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tc_smem(16)));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rbf_mv_tc<32>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(tc_smem(32)));
}

// The float16 parts of P for the contraction: 2 TC_MAXC rows of n_pad float16
// (rows c: the high parts, rows TC_MAXC + c: the low parts), row-major; boxes of
// 64 x ncp (128 bytes x ncp rows) with 128-byte swizzle, the B operand layout.
bool make_rbf_p16_tmap(CUtensorMap* map, const void* PHL, int n_pad, int ncp, EncodeTiledFn encode) {
  cuuint64_t gdim[2] = {cuuint64_t(n_pad), cuuint64_t(2 * TC_MAXC)};
  cuuint64_t gstride[1] = {cuuint64_t(n_pad) * 2};
  cuuint32_t box[2] = {64, cuuint32_t(ncp)};
  cuuint32_t estride[2] = {1, 1};
  CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<void*>(PHL), gdim, gstride, box, estride,
                      CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                      CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS;
}

size_t rbf_p16_halfs(int n_pad) { return size_t(2) * TC_MAXC * n_pad; }

// Q[:, c] = A P[:, c] for c < a.ncols <= 32 (a.p, a.ldp: the columns, zero
// beyond n; a.q, a.ldq): k_rbf_p16 then one k_rbf_mv_tc pass. pmaps[0], [1]:
// the maps of PHL for 16 and 32 columns; pscale: TC_MAXC floats.
cudaError_t launch_rbf_mv_tc(const CUtensorMap* tmap, const CUtensorMap* pmaps, const RbfMvArgs& a, void* PHL,
                             float* pscale, int grid, cudaStream_t s) {
  if (a.ncols < 1 || a.ncols > TC_MAXC) return cudaErrorInvalidValue;
  const int ncp = a.ncols <= 16 ? 16 : 32;
  const int n_pad = a.n_tiles * MV_TILE;
  k_rbf_p16<<<ncp, 1024, 0, s>>>(a.p, a.ldp, a.ncols, n_pad, static_cast<__half*>(PHL), pscale);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (ncp == 16)
    k_rbf_mv_tc<16><<<grid, MV_THREADS, tc_smem(16), s>>>(tmap[0], tmap[1], pmaps[0], a, pscale);
  else
    k_rbf_mv_tc<32><<<grid, MV_THREADS, tc_smem(32), s>>>(tmap[0], tmap[1], pmaps[1], a, pscale);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Symmetric matrix-free matvec: each pair of tiles (I, J), J >= I, is formed
// once (one MMA chain, one exponential per entry) and used twice: the row
// sums q_I += E_IJ p_J as in k_rbf_mv, and, off the diagonal, the column sums
// q_J += E_IJ^T p_I. The entry is exp2(2c S~_ij + u_i) with
// S~_ij = x_i.x_j - |x_j|^2 / 2 and u_i = log2 s^2 - c |x_i|^2, i.e.
// s^2 exp(-c' |x_i - x_j|^2): the same value for (i, j) and (j, i) up to
// rounding, so the operator applied is exactly symmetric.
//   Row blocks I (128 rows) are taken from a global counter in order, the
// largest (most J tiles) first; every CTA then sweeps J = I .. n_tiles - 1.
// The row sums of a block go to rowpart, the column sums of tile (I, J) to
// colpart[I n_pad + j]: per warp (32 rows x 32 columns) a transposing
// shuffle tree, then the four warps of a column slice (the TMEM lane
// quarters) are added by the last of them to arrive (a counter per ring slot
// and slice; no warp waits for another). k_rbf_mv_fin adds, per row, its row
// part and the column parts of the blocks before its own in a fixed order,
// the noise term and p^T q, and rewinds the counter.
// ---------------------------------------------------------------------------
constexpr int MVS_RB_RING = 8;   // row-block ids published ahead (producer <= 5 blocks ahead)
constexpr int MVS_RED_RING = 8;  // column-sum slots (warps <= 4 tiles apart)

// 16 entries of one row (lane): as mv_half, and the column contributions
// c[k] = (entries 2k, 2k + 1) * p_i as packed pairs.
__device__ __forceinline__ void mv_half_sym(const uint32_t (&h)[16], const float* pj, unsigned long long c2x2,
                                            unsigned long long uu, unsigned long long pii, unsigned long long& sA,
                                            unsigned long long& sB, unsigned long long (&c)[8], bool cols) {
#pragma unroll
  for (int j = 0; j < 16; j += 4) {
    const float4 p4 = *reinterpret_cast<const float4*>(pj + j);
    const unsigned long long g01 =
        tc::f2fma(c2x2, tc::f2pk(__uint_as_float(h[j + 0]), __uint_as_float(h[j + 1])), uu);
    const unsigned long long g23 =
        tc::f2fma(c2x2, tc::f2pk(__uint_as_float(h[j + 2]), __uint_as_float(h[j + 3])), uu);
    const unsigned long long e01 = tc::f2pk(tc::ex2_approx(tc::f2lo(g01)), tc::ex2_approx(tc::f2hi(g01)));
    const unsigned long long e23 = tc::f2pk(tc::ex2_approx(tc::f2lo(g23)), tc::ex2_approx(tc::f2hi(g23)));
    sA = tc::f2fma(e01, tc::f2pk(p4.x, p4.y), sA);
    sB = tc::f2fma(e23, tc::f2pk(p4.z, p4.w), sB);
    if (cols) {
      c[j / 2] = tc::f2mul(e01, pii);
      c[j / 2 + 1] = tc::f2mul(e23, pii);
    }
  }
}

__global__ void __launch_bounds__(MV_THREADS, 1)
    k_rbf_mv_sym(const __grid_constant__ CUtensorMap tmap_i, const __grid_constant__ CUtensorMap tmap_j, RbfMvArgs a) {
  constexpr int SB = mv_stage_bytes(1);
  extern __shared__ unsigned char smem_raw[];
  unsigned char* base = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  unsigned char* xi_tile = base;
  unsigned char* stages = base + MV_TILE_BYTES;
  uint64_t* bars = reinterpret_cast<uint64_t*>(stages + size_t(MV_STAGES) * SB);
  uint64_t* full = bars;                       // [MV_STAGES]
  uint64_t* empty = full + MV_STAGES;          // [MV_STAGES]
  uint64_t* tfull = empty + MV_STAGES;         // [MV_TBUF]
  uint64_t* tempty = tfull + MV_TBUF;          // [MV_TBUF]
  uint64_t* xi_full = tempty + MV_TBUF;
  uint64_t* xi_empty = xi_full + 1;
  uint64_t* rbfull = xi_empty + 1;             // [MVS_RB_RING] a row-block id is published
  __shared__ uint32_t s_tmem;
  __shared__ int s_abort;
  __shared__ int s_rb[MVS_RB_RING];
  __shared__ float s_red[MVS_RED_RING][4][MV_TILE];     // column sums: [slot][TMEM lane quarter][column]
  __shared__ unsigned int s_red_cnt[MVS_RED_RING][4];    // [slot][column slice]
  __shared__ float s_rowred[MVS_RED_RING][4][MV_TILE];  // row sums: [slot][column slice][row]
  __shared__ unsigned int s_row_cnt[MVS_RED_RING][4];    // [slot][TMEM lane quarter]

  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int n_tiles = a.n_tiles;
  const int64_t ldc = int64_t(n_tiles) * MV_TILE;  // n_pad: row stride of colpart
  const int kind_tf32 = a.xformat != DCG_X_BF16;
  const int dk = rbf_tile_coords(a.xformat, a.d) + kRbfAug;
  const int ksteps = kind_tf32 ? (dk + 7) / 8 : (dk + 15) / 16;
  const uint32_t row_bytes = uint32_t(rbf_row_bytes(a.xformat, dk));
  const uint32_t tile_bytes = MV_TILE * row_bytes;
  const uint32_t idesc = tc::instr_desc(kind_tf32 ? tc::kFmtTF32 : tc::kFmtBF16, MV_TILE, MV_TILE);

  if (threadIdx.x == 0) {
    for (int s = 0; s < MV_STAGES; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], MV_EPI_WARPS);
    }
    for (int b = 0; b < MV_TBUF; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], MV_EPI_WARPS);
    }
    mbar_init(xi_full, 1);
    mbar_init(xi_empty, 1);
    for (int r = 0; r < MVS_RB_RING; ++r) mbar_init(&rbfull[r], 1);
    fence_mbarrier_init();
    s_abort = 0;
  }
  for (int idx = threadIdx.x; idx < MVS_RED_RING * 4; idx += blockDim.x) {
    s_red_cnt[idx / 4][idx % 4] = 0u;
    s_row_cnt[idx / 4][idx % 4] = 0u;
  }
  if (warp == 1) tc::tmem_alloc(&s_tmem, MV_TMEM_COLS);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = s_tmem;

  if (warp == 0) {
    // ---------------- producer: takes row blocks, publishes their ids ----------------
    if (lane == 0) {
      prefetch_tensormap(&tmap_i);
      prefetch_tensormap(&tmap_j);
      long long it = 0;
      int rbc = 0;
      while (true) {
        int rb = int(atomicAdd(a.sched_ctr, 1u));
        if (rb >= n_tiles) rb = -1;
        // the X_I slot is free once the MMAs of the previous block are done
        if (rb >= 0 && rbc > 0 && !mbar_wait_bounded(xi_empty, (rbc - 1) & 1)) {
          s_abort = 1;
          rb = -1;
        }
        s_rb[rbc % MVS_RB_RING] = rb;   // -1: no more blocks (the consumers leave)
        mbar_arrive(&rbfull[rbc % MVS_RB_RING]);
        if (rb < 0) break;
        mbar_arrive_expect_tx(xi_full, tile_bytes);
        tma_load_2d(xi_tile, &tmap_i, xi_full, 0, rb * MV_TILE);
        bool stop = false;
        for (int J = rb; J < n_tiles; ++J, ++it) {
          const int s = int(it % MV_STAGES);
          if (it >= MV_STAGES && !mbar_wait_bounded(&empty[s], uint32_t((it / MV_STAGES) - 1) & 1)) {
            s_abort = 1;
            stop = true;
            break;
          }
          unsigned char* stg = stages + size_t(s) * SB;
          mbar_arrive_expect_tx(&full[s], tile_bytes + MV_TILE * 4);
          tma_load_2d(stg, &tmap_j, &full[s], 0, J * MV_TILE);
          tc::bulk_load(stg + MV_TILE_BYTES, a.p + size_t(J) * MV_TILE, MV_TILE * 4, &full[s]);
        }
        ++rbc;
        if (stop) {
          s_rb[rbc % MVS_RB_RING] = -1;
          mbar_arrive(&rbfull[rbc % MVS_RB_RING]);
          break;
        }
      }
    }
  } else if (warp == 1) {
    // ---------------- MMA issuer ----------------
    if (lane == 0) {
      long long it = 0;
      const uint32_t a_base = smem_u32(xi_tile);
      for (int rbc = 0;; ++rbc) {
        if (!mbar_wait_bounded(&rbfull[rbc % MVS_RB_RING], (rbc / MVS_RB_RING) & 1)) { s_abort = 1; break; }
        const int rb = *(volatile int*)&s_rb[rbc % MVS_RB_RING];
        if (rb < 0) break;
        if (!mbar_wait_bounded(xi_full, rbc & 1)) { s_abort = 1; break; }
        tc::fence_after_sync();
        bool stop = false;
        for (int J = rb; J < n_tiles; ++J, ++it) {
          const int s = int(it % MV_STAGES);
          const int b = int(it % MV_TBUF);
          if (!mbar_wait_bounded(&full[s], uint32_t(it / MV_STAGES) & 1) ||
              (it >= MV_TBUF && !mbar_wait_bounded(&tempty[b], uint32_t((it / MV_TBUF) - 1) & 1))) {
            s_abort = 1;
            stop = true;
            break;
          }
          tc::fence_after_sync();
          const uint32_t b_base = smem_u32(stages + size_t(s) * SB);
          const uint32_t d_tmem = tmem + uint32_t(b * MV_TILE);
          for (int kk = 0; kk < ksteps; ++kk) {
            const uint64_t ad = tc::smem_desc_kmajor(a_base + 32 * kk, row_bytes);
            const uint64_t bd = tc::smem_desc_kmajor(b_base + 32 * kk, row_bytes);
            if (kind_tf32)
              tc::mma_tf32(d_tmem, ad, bd, idesc, kk > 0);
            else
              tc::mma_bf16(d_tmem, ad, bd, idesc, kk > 0);
          }
          tc::mma_commit(&tfull[b]);
        }
        tc::mma_commit(xi_empty);
        if (stop) break;
      }
    }
  } else {
    // ---------------- epilogue ----------------
    const int ew = warp - 2;                  // 0..15
    const int quarter = warp & 3;             // TMEM lane quarter this warp may read
    const int slice = ew >> 2;                // 32-column slice of the tile
    const int row_l = quarter * 32 + lane;    // row within the I block
    const float c2 = a.prm->c2, l2s = a.prm->l2s;
    const unsigned long long c2x2 = tc::f2pk(c2, c2);
    const uint32_t lane_off = uint32_t(quarter * 32) << 16;
    long long it = 0;
    bool aborted = false;
    for (int rbc = 0; !aborted; ++rbc) {
      if (!mbar_wait_bounded(&rbfull[rbc % MVS_RB_RING], (rbc / MVS_RB_RING) & 1)) { s_abort = 1; break; }
      const int rb = *(volatile int*)&s_rb[rbc % MVS_RB_RING];
      if (rb < 0) break;
      const int row = rb * MV_TILE + row_l;
      const float u = l2s + a.vcol[row];        // vcol has n_pad entries
      const float pi = a.p[row];                // p has n_pad entries, zero beyond n
      const unsigned long long uu = tc::f2pk(u, u), pii = tc::f2pk(pi, pi);
      float acc = 0.f, comp = 0.f;              // Kahan sum of the row's per-tile partials
      uint32_t ha[16], hb[16];
      {
        const int b = int(it % MV_TBUF);
        if (!mbar_wait_bounded(&tfull[b], uint32_t(it / MV_TBUF) & 1)) {
          s_abort = 1;
          aborted = true;
        } else {
          tc::fence_after_sync();
          tc::tmem_ld16_nowait(tmem + lane_off + uint32_t(b * MV_TILE + slice * 32), ha);
          tc::tmem_wait_ld16(ha);
        }
      }
      for (int J = rb; J < n_tiles && !aborted; ++J, ++it) {
        const int s = int(it % MV_STAGES);
        const int b = int(it % MV_TBUF);
        const bool cols = J > rb;               // off the diagonal: the transposed part too
        const float* pj =
            reinterpret_cast<const float*>(stages + size_t(s) * SB + MV_TILE_BYTES) + slice * 32;
        tc::tmem_ld16_nowait(tmem + lane_off + uint32_t(b * MV_TILE + slice * 32 + 16), hb);
        unsigned long long s0 = 0ull, s1 = 0ull, s2 = 0ull, s3 = 0ull;
        unsigned long long cA[8], cB[8];
        mv_half_sym(ha, pj, c2x2, uu, pii, s0, s1, cA, cols);
        tc::tmem_wait_ld16(hb);
        tc::fence_before_sync();
        __syncwarp();
        if (lane == 0) mbar_arrive(&tempty[b]);
        const bool next = J + 1 < n_tiles;
        if (next) {
          const int b2 = int((it + 1) % MV_TBUF);
          if (!mbar_wait_bounded(&tfull[b2], uint32_t((it + 1) / MV_TBUF) & 1)) {
            s_abort = 1;
            aborted = true;
          } else {
            tc::fence_after_sync();
            tc::tmem_ld16_nowait(tmem + lane_off + uint32_t(b2 * MV_TILE + slice * 32), ha);
          }
        }
        mv_half_sym(hb, pj + 16, c2x2, uu, pii, s2, s3, cB, cols);
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (next && !aborted) tc::tmem_wait_ld16(ha);
        const float part = ((tc::f2lo(s0) + tc::f2hi(s0)) + (tc::f2lo(s1) + tc::f2hi(s1))) +
                           ((tc::f2lo(s2) + tc::f2hi(s2)) + (tc::f2lo(s3) + tc::f2hi(s3)));
        const float y = part - comp;
        const float tt = acc + y;
        comp = (tt - acc) - y;
        acc = tt;
        if (cols) {
          // column sums of the warp's 32 rows: lane l ends with column 32 slice + l
          float v[32];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            v[2 * k] = tc::f2lo(cA[k]);
            v[2 * k + 1] = tc::f2hi(cA[k]);
            v[16 + 2 * k] = tc::f2lo(cB[k]);
            v[16 + 2 * k + 1] = tc::f2hi(cB[k]);
          }
          warp_transpose_sum(v, lane);
          const int slot = int(it % MVS_RED_RING);
          s_red[slot][quarter][slice * 32 + lane] = v[0];
          __syncwarp();
          unsigned int last = 0u;
          if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&s_red_cnt[slot][slice], 1u) == 3u ? 1u : 0u;
            if (last) {
              __threadfence_block();
              s_red_cnt[slot][slice] = 0u;
            }
          }
          last = __shfl_sync(0xffffffffu, last, 0);
          if (last) {
            __threadfence_block();
            const int col = slice * 32 + lane;
            float t4 = 0.f;
#pragma unroll
            for (int q4 = 0; q4 < 4; ++q4) t4 += *reinterpret_cast<volatile float*>(&s_red[slot][q4][col]);
            a.colpart[int64_t(rb) * ldc + int64_t(J) * MV_TILE + col] = t4;
          }
        }
      }
      if (aborted) break;
      // the four column slices of each row, added by the last of the four
      // warps of the lane quarter to arrive (no warp waits for another)
      const int rslot = rbc % MVS_RED_RING;
      s_rowred[rslot][slice][row_l] = acc;
      __syncwarp();
      unsigned int lastr = 0u;
      if (lane == 0) {
        __threadfence_block();
        lastr = atomicAdd(&s_row_cnt[rslot][quarter], 1u) == 3u ? 1u : 0u;
        if (lastr) {
          __threadfence_block();
          s_row_cnt[rslot][quarter] = 0u;
        }
      }
      lastr = __shfl_sync(0xffffffffu, lastr, 0);
      if (lastr) {
        __threadfence_block();
        const volatile float* rr = &s_rowred[rslot][0][row_l];
        a.rowpart[row] = (rr[0] + rr[MV_TILE]) + (rr[2 * MV_TILE] + rr[3 * MV_TILE]);
      }
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  if (warp == 1) {
    tc::fence_after_sync();
    tc::tmem_dealloc(tmem, MV_TMEM_COLS);
  }
  if (s_abort && threadIdx.x == 0 && st) {
    st->status = DCG_ERR_TIMEOUT;
    st->timeout_site = 3;
    st->done = 1;
  }
}

// q_i = rowpart_i + sum_{I' < I(i)} colpart[I' n_pad + i] + noise p_i and p^T q.
// One CTA per row block (128 rows, a lane four of them, float4 loads); its
// 16 warps split the column parts of the blocks before it (warp w: w, w + 16,
// ...), four loads in flight per warp, combined in a fixed order. The first
// thread rewinds the row-block counter of k_rbf_mv_sym, which has finished.
constexpr int MVF_WARPS = 16;
__global__ void __launch_bounds__(MVF_WARPS * 32) k_rbf_mv_fin(RbfMvArgs a) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *a.sched_ctr = 0u;
  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  const int n = a.n;
  const int64_t ldc = int64_t(a.n_tiles) * MV_TILE;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int I = blockIdx.x;
  const int64_t off = int64_t(I) * MV_TILE + 4 * lane;
  auto ld = [&](int t) { return __ldcg(reinterpret_cast<const float4*>(a.colpart + int64_t(t) * ldc + off)); };
  float4 s0 = make_float4(0.f, 0.f, 0.f, 0.f), s1 = s0, s2 = s0, s3 = s0;
  int t = warp;
  for (; t + 3 * MVF_WARPS < I; t += 4 * MVF_WARPS) {
    const float4 v0 = ld(t), v1 = ld(t + MVF_WARPS), v2 = ld(t + 2 * MVF_WARPS), v3 = ld(t + 3 * MVF_WARPS);
    s0.x += v0.x; s0.y += v0.y; s0.z += v0.z; s0.w += v0.w;
    s1.x += v1.x; s1.y += v1.y; s1.z += v1.z; s1.w += v1.w;
    s2.x += v2.x; s2.y += v2.y; s2.z += v2.z; s2.w += v2.w;
    s3.x += v3.x; s3.y += v3.y; s3.z += v3.z; s3.w += v3.w;
  }
  for (; t < I; t += MVF_WARPS) {
    const float4 v = ld(t);
    s0.x += v.x; s0.y += v.y; s0.z += v.z; s0.w += v.w;
  }
  __shared__ float4 red[MVF_WARPS][32];
  red[warp][lane] = make_float4((s0.x + s1.x) + (s2.x + s3.x), (s0.y + s1.y) + (s2.y + s3.y),
                                (s0.z + s1.z) + (s2.z + s3.z), (s0.w + s1.w) + (s2.w + s3.w));
  __syncthreads();
  double my = 0.0;
  if (threadIdx.x < MV_TILE) {
    const int l = threadIdx.x >> 2, e = threadIdx.x & 3;
    const int row = I * MV_TILE + threadIdx.x;
    float cs = 0.f;
#pragma unroll
    for (int w = 0; w < MVF_WARPS; ++w) cs += reinterpret_cast<const float*>(&red[w][l])[e];
    if (row < n) {
      const float pi = a.p[row];
      const float q = (a.rowpart[row] + cs) + a.prm->noise * pi;
      a.q[row] = q;
      my = double(pi) * double(q);
    }
  }
  __shared__ double s_part[MV_TILE / 32];
  if (warp < MV_TILE / 32) {
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

constexpr size_t MVS_SMEM = MV_SMEM + 256;  // the row-block ring's barriers

cudaError_t rbf_mv_sym_configure() {
  return cudaFuncSetAttribute(k_rbf_mv_sym, cudaFuncAttributeMaxDynamicSharedMemorySize, int(MVS_SMEM));
}

size_t rbf_mv_sym_colpart_floats(int n_pad) { return size_t(n_pad / MV_TILE) * size_t(n_pad); }

// q = A p with the symmetric tile pairs; a.rowpart (n_pad floats), a.colpart
// (rbf_mv_sym_colpart_floats), a.sched_ctr (zero between launches) and
// a.partials (>= n_tiles doubles) set by the caller.
cudaError_t launch_rbf_mv_sym(const CUtensorMap* tmap, const RbfMvArgs& a, int grid, cudaStream_t s) {
  k_rbf_mv_sym<<<grid, MV_THREADS, MVS_SMEM, s>>>(tmap[0], tmap[1], a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rbf_mv_fin<<<a.n_tiles, MVF_WARPS * 32, 0, s>>>(a);
  return cudaGetLastError();
}

cudaError_t rbf_mv_configure() {
  cudaError_t e = cudaFuncSetAttribute(k_rbf_mv<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(MV_SMEM));
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_rbf_mv<MV_BLOCK_NC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              int(mv_smem(MV_BLOCK_NC)));
}

// Persistent grid, one CTA per SM: each CTA holds all 512 TMEM columns (four
// accumulator buffers), and its register use keeps a second CTA off the SM.
int rbf_mv_grid(int n_tiles, int num_sms) { return n_tiles < num_sms ? n_tiles : num_sms; }

cudaError_t launch_rbf_mv(const CUtensorMap* tmap, const RbfMvArgs& a, int grid, cudaStream_t s) {
  k_rbf_mv<1><<<grid, MV_THREADS, MV_SMEM, s>>>(tmap[0], tmap[1], a);
  return cudaGetLastError();
}

int rbf_block_nc() { return MV_BLOCK_NC; }

// One pass of the multi-column product over columns col0 .. col0 + NC - 1:
// a.p = NC padded columns (leading dimension a.ldp = n_pad, zero beyond n),
// a.q = the first output column (leading dimension a.ldq), a.ncols = columns
// to write (a.col_idx = col0 with a solver state: the pass is skipped when
// col0 >= k, and columns at or beyond k are not written).
cudaError_t launch_rbf_mv_block(const CUtensorMap* tmap, const RbfMvArgs& a, int grid, cudaStream_t s) {
  k_rbf_mv<MV_BLOCK_NC><<<grid, MV_THREADS, mv_smem(MV_BLOCK_NC), s>>>(tmap[0], tmap[1], a);
  return cudaGetLastError();
}

// dst[c * ldd + i] = src[c * n + i] for i < n and the columns col0 + c < k
// (all NC columns without a solver state); the tails beyond n are left as
// they are (zero in the caller's padded buffer).
__global__ void k_copy_cols(const float* src, float* dst, int n, int64_t ldd, int col0, int nc, const DevState* st) {
  int kv = nc;
  if (st) {
    if (st->done) return;
    kv = min(nc, st->k - col0);
  }
  const int64_t total = int64_t(kv) * n;
  for (int64_t idx = int64_t(blockIdx.x) * blockDim.x + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int c = int(idx / n), i = int(idx - int64_t(c) * n);
    dst[c * ldd + i] = src[int64_t(c) * n + i];
  }
}

cudaError_t launch_copy_cols(const float* src, float* dst, int n, int64_t ldd, int col0, int nc, const DevState* st,
                             cudaStream_t s) {
  k_copy_cols<<<256, 256, 0, s>>>(src, dst, n, ldd, col0, nc, st);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Exact-form operator on CUDA cores (128 rows per CTA, one per thread, x_i in
// registers; J tiles of 64 points staged in shared memory):
//   * k_rbf_resid + k_rbf_resid_fin: r = b - A x for the float64 iterate
//     x = xh + xl, the true residual of the refinement. Entries are float32
//     pairs, the sums compensated (Dot2); the J range is split over grid.y so
//     that the grid fills whole waves, and the finishing kernel merges the
//     per-split pairs in a fixed order.
//   * k_rbf_block: Y[:, c] = A V[:, c] (dcg_apply_block), entries to ~2 ulp.
//
// Distances of the residual kernel, Gram form D_ij = n_i + n_j - 2 G_ij with
// G_ij = sum_m x_im x_jm summed onto a fixed grid (the error-free extraction
// onto a grid of Rump, Ogita and Oishi, "Accurate floating-point summation",
// SIAM J. Sci. Comput. 31, 2008): T starts at the anchor sigma = 1.5 2^23 g,
// whose float32 neighbours are spaced g apart, and every partial sum of G is
// below 2^22 g in magnitude (g = 2^(E - 22) with max_i |x_i|^2 < 2^E). Each
// step T' = fma(x_im, x_jm, T) rounds the product onto the grid; the step
// T' - T is exact (both lie in [2^23 g, 2^24 g)), and so is what the rounding
// dropped, e = fma(x_im, x_jm, -(T' - T)), |e| <= g / 2 (BF16 and TF32
// products fit in float32; for float32 points e carries one rounding of
// size u g / 2). Hence G = (T - sigma) + sum_m e_m: the first part exact on
// the grid, the second summed in float32. With |x_i|^2 = nh_i + nl_i, nh_i on
// the grid, D_hi = nh_i + nh_j - 2 (T - sigma) is exact in float32 (all terms
// are multiples of g below 2^24 g) and D_lo = nl_i + nl_j - 2 sum e carries
// the rest. Two entries go through each packed f32x2 instruction: four per
// coordinate and pair.
//
// Error model of one residual entry K_ij in units of u^2 = 2^-48:
//   * distance: the float32 sum of the d remainders (each <= g/2, rounding
//     errors growing like sqrt(d) u |sum e| ~ d u g / sqrt(12), taken three
//     times for a probabilistic bound) and nl's rounding: relative error of
//     K_ij <= (0.87 d + 1) g c / u with c = 1 / (2 l^2);
//   * the exponent a = -D c as a pair (2 |a|), exp after Tang (emulated
//     against 200-bit arithmetic over a in [-103, 0]: <= 2 + |a| from the
//     exponent's own representation), the s^2 pair and one Dot2 step (~4).
//   Relative error of the entry: <= (8 + 3 |a| + (0.87 d + 1) g c / u) u^2.
// ---------------------------------------------------------------------------
constexpr int EX_ROWS = 128;
constexpr double kU2 = 3.552713678800501e-15;  // 2^-48
constexpr float kEntryErrC0 = 8.f;
constexpr int EX_J = 64;
constexpr int EX_MAXD = 64;
constexpr int EX_CB = 16;
constexpr int EX_MAX_SPLITS = 16;  // J-range splits of the residual kernel (grid.y)
// Smallest exponent the residual kernel evaluates: below it exp(a) < 1.7e-38
// (near the smallest normal float32) and the entry is dropped, which changes
// a row's sum by less than n 1.7e-38 max|x|. From a >= -87 the binary
// exponent of exp_tang is >= -126, so 2^m is a normal float32.
constexpr float kExpMinArg = -87.0f;

// |x_i|^2 in float64 (exact squares, float64 sums) and the largest of them as
// float bits rounded up (positive floats order like their bit patterns).
__global__ void k_rbf_norms(const float* __restrict__ Xr, int n, int d, double* n64, unsigned int* maxbits) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double ss = 0.0;
    for (int m = 0; m < d; ++m) {
      const double v = Xr[int64_t(i) * d + m];
      ss = fma(v, v, ss);
    }
    n64[i] = ss;
    atomicMax(maxbits, __float_as_uint(__double2float_ru(ss)));
  }
}

// The grid of the distance sums: g = 2^(E - 22) with max |x_i|^2 < 2^E,
// sigma = 1.5 2^23 g; nh_i = |x_i|^2 rounded to a multiple of g (below
// 2^24 g, so exact in float32), nl_i = the rest, rounded. Rows beyond n get
// zeros. XrT: the points transposed (d x n_pad, zero padded) for coalesced
// staging of the J tiles.
__global__ void k_rbf_anchor(const double* __restrict__ n64, const float* __restrict__ Xr, int n, int n_pad, int d,
                             const unsigned int* maxbits, RbfParams* prm, float* nh, float* nl, float* XrT) {
  const float mx = __uint_as_float(*maxbits);
  int E = 0;
  frexpf(mx > 0.f ? mx : 1.f, &E);  // mx < 2^E
  const double g = ldexp(1.0, E - 22);
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    prm->g_anchor = float(g);
    prm->sigma_anchor = float(1.5 * ldexp(1.0, 23) * g);
  }
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n_pad; i += gridDim.x * blockDim.x) {
    float h = 0.f, l = 0.f;
    if (i < n) {
      const double q = rint(n64[i] / g);
      h = float(q * g);
      l = float(n64[i] - q * g);
    }
    nh[i] = h;
    nl[i] = l;
    for (int m = 0; m < d; ++m) XrT[int64_t(m) * n_pad + i] = i < n ? Xr[int64_t(i) * d + m] : 0.f;
  }
}

cudaError_t launch_rbf_anchor(const float* Xr, int n, int n_pad, int d, double* n64, unsigned int* maxbits,
                              RbfParams* prm, float* nh, float* nl, float* XrT, cudaStream_t s) {
  cudaError_t e = cudaMemsetAsync(maxbits, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess) return e;
  k_rbf_norms<<<(n + 255) / 256, 256, 0, s>>>(Xr, n, d, n64, maxbits);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  k_rbf_anchor<<<(n_pad + 255) / 256, 256, 0, s>>>(n64, Xr, n, n_pad, d, maxbits, prm, nh, nl, XrT);
  return cudaGetLastError();
}

__device__ __forceinline__ void two_sum_add(float& s, float& c, float v) {
  const float s2 = __fadd_rn(s, v);
  const float z = __fsub_rn(s2, s);
  c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(s2, z)), __fsub_rn(v, z)));
  s = s2;
}

// ln 2 / 64 = kL1 + kL2 + kL3 to ~2^-70 relative: kL1 has 10 significant bits
// so that k kL1 is exact for |k| < 2^14; kL2 and kL3 are the next float32
// pieces. k64L = 64 / ln 2 rounded (only used to pick k).
constexpr float kL1 = 0x1.63p-7f;
constexpr float kL2 = -0x1.bd0106p-19f;
constexpr float kL3 = 0x1.cf79acp-46f;
constexpr float k64L = 0x1.715476p+6f;

// exp(a_hi + a_lo) for -103 <= a <= 0 as 2^m (e_hi + e_lo). Table-driven
// reduction (Tang's method): a = k ln2/64 + r, k = 64 m + j, |r| <= ln2/128,
// exp(a) = 2^m 2^(j/64) exp(r). r is formed as a float32 pair from the exact
// product k kL1 and the FMA-exact error of k kL2. exp(r) - 1 = r + r^2/2 +
// r^3 c(r) with c the Taylor terms to r^5 (truncation r^6/720 < 4e-17); r and
// r^2/2 are carried as pairs, the cubic tail (< 3e-8) in float32. tab[j] =
// 2^(j/64) as a float32 pair.
__device__ __forceinline__ void exp_tang(float a_hi, float a_lo, const float2* tab, float& e_hi, float& e_lo,
                                         int& m) {
  const float kf = rintf(__fmul_rn(a_hi, k64L));
  const float t1 = __fmaf_rn(-kf, kL1, a_hi);  // exact
  const float p2 = __fmul_rn(kf, kL2);
  const float e2 = __fmaf_rn(kf, kL2, -p2);    // exact error of k kL2
  const float p3 = __fmul_rn(kf, kL3);
  // (r_hi, r_lo) = t1 - p2 by TwoSum, plus the low-order terms
  float r_hi = __fsub_rn(t1, p2);
  const float z = __fsub_rn(r_hi, t1);
  float r_lo = __fadd_rn(__fsub_rn(t1, __fsub_rn(r_hi, z)), __fsub_rn(-p2, z));
  r_lo = __fadd_rn(r_lo, __fsub_rn(__fsub_rn(a_lo, e2), p3));
  {
    const float s = __fadd_rn(r_hi, r_lo);
    r_lo = __fsub_rn(r_lo, __fsub_rn(s, r_hi));
    r_hi = s;
  }
  const float sq = __fmul_rn(r_hi, r_hi);
  const float sq_e = __fmaf_rn(r_hi, r_hi, -sq);
  const float h = 0.5f * sq;                                   // exact
  const float h_lo = __fmaf_rn(r_hi, r_lo, 0.5f * sq_e);
  const float c = __fmul_rn(__fmul_rn(sq, r_hi),
                            __fmaf_rn(r_hi, __fmaf_rn(r_hi, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f));
  const float s_hi = __fadd_rn(r_hi, h);                       // |r_hi| >= |h|
  const float s_e = __fsub_rn(h, __fsub_rn(s_hi, r_hi));
  const float lo = __fadd_rn(__fadd_rn(s_e, r_lo), __fadd_rn(h_lo, c));
  const float e1 = __fadd_rn(1.f, s_hi);                       // 1 >= |s_hi|
  const float e1_e = __fsub_rn(s_hi, __fsub_rn(e1, 1.f));
  const float e1_lo = __fadd_rn(e1_e, lo);
  const int ki = int(kf);
  const int j = ki & 63;
  m = (ki - j) / 64;  // exact: ki - j is a multiple of 64
  const float2 t = tab[j];
  e_hi = __fmul_rn(t.x, e1);
  e_lo = __fadd_rn(__fmaf_rn(t.x, e1, -e_hi), __fmaf_rn(t.x, e1_lo, __fmul_rn(t.y, e1)));
}

// One grid step for two entries at once: T' = fma(x, y, T), e = the part of
// x y the rounding onto the grid dropped, L += e (packed f32x2).
__device__ __forceinline__ void anchored_step2(unsigned long long& T, unsigned long long& L, unsigned long long x,
                                               unsigned long long y) {
  unsigned long long Tn, ndt, e;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(Tn) : "l"(x), "l"(y), "l"(T));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(ndt) : "l"(T), "l"(Tn));  // -(T' - T), exact
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(e) : "l"(x), "l"(y), "l"(ndt));
  asm("add.rn.f32x2 %0, %0, %1;" : "+l"(L) : "l"(e));
  T = Tn;
}

// Partial residual sums of one row over the J tiles of split blockIdx.y:
// part[(y * 3 + 0) * n + i] = s, [1] = c (the Dot2 pair of sum_j K_ij x_j),
// [2] = sum_j (e_ij K_ij x_j)^2 (entry-error estimate, units of u^2).
// Resident CTAs per SM the register budget is set for: x_i lives in
// registers, so the budget grows with DMAX; more CTAs than the kernel's own
// register need allows trades the unrolled inner loop for occupancy.
__host__ __device__ constexpr int ex_resid_min_blocks(int dmax) {
  return dmax <= 8 ? 6 : (dmax <= 16 ? 4 : (dmax <= 32 ? 3 : 2));
}

template <int DMAX>
__global__ void __launch_bounds__(EX_ROWS, ex_resid_min_blocks(DMAX)) k_rbf_resid(RbfExactArgs a) {
  __shared__ __align__(16) float xs[DMAX][EX_J];
  __shared__ __align__(16) float sh_xh[EX_J], sh_xl[EX_J], sh_nh[EX_J], sh_nl[EX_J];
  __shared__ float2 exp_tab[64];
  if (threadIdx.x < 64) {
    const double t = exp2(double(threadIdx.x) / 64.0);
    exp_tab[threadIdx.x] = make_float2(float(t), float(t - double(float(t))));
  }
  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  if (st && a.resid_mode == 0 && !st->warm_start) return;
  const int n = a.n, d = a.d, n_pad = a.n_pad;
  const int i = blockIdx.x * EX_ROWS + threadIdx.x;
  const float k_hi = a.prm->neg_inv2l2, k_lo = a.prm->neg_inv2l2_lo;
  const float s2 = a.prm->s2, s2_lo = a.prm->s2_lo;
  const float sigma = a.prm->sigma_anchor;
  const float err0 = kEntryErrC0 + a.prm->err_dist;
  float xi[DMAX];
#pragma unroll
  for (int m = 0; m < DMAX; ++m) xi[m] = (i < n && m < d) ? a.XrT[int64_t(m) * n_pad + i] : 0.f;
  const float nh_i = a.nh[min(i, n_pad - 1)], nl_i = a.nl[min(i, n_pad - 1)];
  float acc = 0.f, cmp = 0.f, esq = 0.f;
  // tiles of this split: J tiles t with t % gridDim.y == blockIdx.y
  const int ntiles = (n + EX_J - 1) / EX_J;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int j0 = tile * EX_J;
    __syncthreads();
    for (int idx = threadIdx.x; idx < d * (EX_J / 4); idx += EX_ROWS) {
      const int m = idx / (EX_J / 4), q = idx % (EX_J / 4);
      *reinterpret_cast<float4*>(&xs[m][4 * q]) =
          *reinterpret_cast<const float4*>(a.XrT + int64_t(m) * n_pad + j0 + 4 * q);
    }
    if (threadIdx.x < EX_J) {
      const int j = j0 + threadIdx.x;
      const bool in = j < n;
      sh_xh[threadIdx.x] = in ? a.xh[j] : 0.f;
      sh_xl[threadIdx.x] = in ? a.xl[j] : 0.f;
      sh_nh[threadIdx.x] = a.nh[j];  // j < n_pad: zero beyond n
      sh_nl[threadIdx.x] = a.nl[j];
    }
    __syncthreads();
    const int jn = min(EX_J, n - j0);
    for (int jq = 0; jq < jn; jq += 4) {
      unsigned long long T01 = tc::f2pk(sigma, sigma), T23 = T01, L01 = 0ull, L23 = 0ull;
#pragma unroll
      for (int m = 0; m < DMAX; ++m) {
        if (m < d) {
          const float4 x4 = *reinterpret_cast<const float4*>(&xs[m][jq]);
          const unsigned long long xx = tc::f2pk(xi[m], xi[m]);
          anchored_step2(T01, L01, xx, tc::f2pk(x4.x, x4.y));
          anchored_step2(T23, L23, xx, tc::f2pk(x4.z, x4.w));
        }
      }
      const float Tv[4] = {__uint_as_float(unsigned(T01)), __uint_as_float(unsigned(T01 >> 32)),
                           __uint_as_float(unsigned(T23)), __uint_as_float(unsigned(T23 >> 32))};
      const float Lv[4] = {__uint_as_float(unsigned(L01)), __uint_as_float(unsigned(L01 >> 32)),
                           __uint_as_float(unsigned(L23)), __uint_as_float(unsigned(L23 >> 32))};
#pragma unroll
      for (int e4 = 0; e4 < 4; ++e4) {
        const int jj = jq + e4;
        if (jj >= jn) break;
        const float ghi = __fsub_rn(Tv[e4], sigma);                            // exact
        const float dh = __fmaf_rn(-2.f, ghi, __fadd_rn(nh_i, sh_nh[jj]));   // exact
        const float dl = __fmaf_rn(-2.f, Lv[e4], __fadd_rn(nl_i, sh_nl[jj]));
        // exponent a = -(dh + dl) / (2 l^2) as a_hi + a_lo (exact product error by FMA)
        const float a_hi = __fmul_rn(dh, k_hi);
        const float a_lo = __fmaf_rn(dh, k_hi, -a_hi) + dl * k_hi + dh * k_lo;
        // exp(a) < 2^-126 (K below the smallest normal float32): K = 0. Above
        // it the binary exponent m of exp_tang lies in [-126, 0], and 2^m is
        // a normal float32 built from its bits.
        if (a_hi < kExpMinArg) continue;
        float e_hi, e_lo;
        int k2;
        exp_tang(a_hi, a_lo, exp_tab, e_hi, e_lo, k2);
        const float m_hi = __fmul_rn(s2, e_hi);
        const float m_lo = __fmaf_rn(s2, e_hi, -m_hi) + __fmaf_rn(s2, e_lo, s2_lo * e_hi);
        const float scale = __int_as_float((k2 + 127) << 23);
        const float kv_hi = __fmul_rn(m_hi, scale), kv_lo = __fmul_rn(m_lo, scale);
        const float xhv = sh_xh[jj];
        const float p = __fmul_rn(kv_hi, xhv);
        const float pe = __fmaf_rn(kv_hi, xhv, -p);
        two_sum_add(acc, cmp, p);
        cmp = __fadd_rn(cmp, pe);
        cmp = __fmaf_rn(kv_hi, sh_xl[jj], __fmaf_rn(kv_lo, xhv, cmp));
        const float e_ij = fmaf(3.f, fabsf(a_hi), err0) * p;
        esq = fmaf(e_ij, e_ij, esq);
      }
    }
  }
  if (i < n) {
    float* part = a.partials_f + int64_t(blockIdx.y) * 3 * n;
    part[i] = acc;
    part[n + i] = cmp;
    part[2 * n + i] = esq;
  }
}

// r_i = b_i - (A x)_i from the per-split pairs (merged in split order, so the
// result does not depend on scheduling), |r|^2 and the entry-error sum
// reduced by the last CTA, and the true-residual bookkeeping of the solve.
__global__ void __launch_bounds__(EX_ROWS) k_rbf_resid_fin(RbfExactArgs a, int splits) {
  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  if (st && a.resid_mode == 0 && !st->warm_start) return;
  const int n = a.n;
  const int i = blockIdx.x * EX_ROWS + threadIdx.x;
  double my = 0.0, my_e = 0.0;
  if (i < n) {
    float s = 0.f, c = 0.f;
    double se = 0.0;
    for (int y = 0; y < splits; ++y) {
      const float* part = a.partials_f + int64_t(y) * 3 * n;
      const float ps = part[i], pc = part[n + i];
      const float t = __fadd_rn(s, ps);
      const float z = __fsub_rn(t, s);
      const float err = __fadd_rn(__fsub_rn(s, __fsub_rn(t, z)), __fsub_rn(ps, z));
      s = t;
      c = __fadd_rn(c, __fadd_rn(pc, err));
      se += double(part[2 * n + i]);
    }
    const double x = double(a.xh[i]) + double(a.xl[i]);
    const double ax = double(s) + double(c) + a.prm->noise_d * x;
    const double rr = double(a.b[i]) - ax;
    a.r[i] = float(rr);
    my = rr * rr;
    my_e = se;
  }
  // |r|^2 and e^2 = sum_ij (e_ij K_ij x_j)^2: CTA partials -> last CTA
  __shared__ double s_part[2][EX_ROWS / 32];
  const double v = warp_sum(my), ve = warp_sum(my_e);
  if ((threadIdx.x & 31) == 0) {
    s_part[0][threadIdx.x >> 5] = v;
    s_part[1][threadIdx.x >> 5] = ve;
  }
  __syncthreads();
  const int G = gridDim.x;
  if (threadIdx.x == 0) {
    double s = 0.0, se = 0.0;
    for (int w = 0; w < EX_ROWS / 32; ++w) {
      s += s_part[0][w];
      se += s_part[1][w];
    }
    a.partials[blockIdx.x] = s;
    a.partials[G + blockIdx.x] = se;
  }
  if (!arrive_last(a.ticket)) return;
  if (threadIdx.x < 32) {
    double s = 0.0, se = 0.0;
    for (int b = threadIdx.x; b < G; b += 32) {
      s += __ldcg(a.partials + b);
      se += __ldcg(a.partials + G + b);
    }
    s = warp_sum(s);
    se = warp_sum(se);
    if (threadIdx.x == 0) {
      if (!st) {
        if (a.result) *a.result = s;
        if (a.result_err) *a.result_err = 3.0 * kU2 * sqrt(se);
      } else if (a.resid_mode != 0) {
        // Entry K_ij carries a relative error <= e_ij u^2 (the model above).
        // The errors of different entries are independent, so the error of
        // the computed residual is ~u^2 sqrt(sum_ij (e_ij K_ij x_j)^2)
        // (probabilistic rounding-error model, Higham & Mary 2019); the
        // worst-case sum of |K_ij x_j| overstates it by orders of magnitude
        // because b - A x cancels heavily. Convergence is accepted only if the
        // residual plus three times that estimate meets tol.
        const double err = 3.0 * kU2 * sqrt(se);
        st->rho_true = s;
        st->matvecs_check += 1;
        st->relres_true = st->bnorm2 > 0.0 ? sqrt(s / st->bnorm2) : sqrt(s);
        st->true_valid = 1;
        const int mode = a.resid_mode >= 0 ? a.resid_mode : st->mode;
        const double lim = sqrt(st->thresh2) - err;
        if (mode == 1 && st->status == DCG_OK) {
          if (lim > 0.0 && s <= lim * lim)
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

// Y[:, c] = A V[:, c] for c < ncols, EX_CB columns per blockIdx.y: distances
// in the difference form as float32 pairs (exact differences by TwoDiff,
// exact squares by FMA, compensated sum), entries s^2 expf(a_hi) (1 + a_lo)
// (~2 ulp).
__global__ void __launch_bounds__(EX_ROWS) k_rbf_block(RbfExactArgs a) {
  __shared__ float xj[EX_J][EX_MAXD + 1];
  __shared__ float vj[EX_J][EX_CB + 1];
  DevState* st = a.st;
  if (st && a.skip_if_done && st->done) return;
  const int n = a.n, d = a.d;
  int ncols = a.ncols;
  const float* V = a.V;
  float* Y = a.Y;
  if (st) {  // start of a solve: AW for the active columns of W
    ncols = st->k;
    V += n;
    Y += n;
  }
  const int col0 = blockIdx.y * EX_CB;
  if (col0 >= ncols) return;
  const int cw = min(EX_CB, ncols - col0);
  const int i = blockIdx.x * EX_ROWS + threadIdx.x;
  const float neg_inv2l2 = a.prm->neg_inv2l2, neg_inv2l2_lo = a.prm->neg_inv2l2_lo;
  const float s2 = a.prm->s2, noise = a.prm->noise;
  float xi[EX_MAXD];
#pragma unroll
  for (int m = 0; m < EX_MAXD; ++m) xi[m] = (i < n && m < d) ? a.Xr[int64_t(i) * d + m] : 0.f;
  float acc[EX_CB];
#pragma unroll
  for (int c = 0; c < EX_CB; ++c) acc[c] = 0.f;
  for (int j0 = 0; j0 < n; j0 += EX_J) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < EX_J * d; idx += EX_ROWS) {
      const int jj = idx / d, m = idx % d;
      xj[jj][m] = (j0 + jj < n) ? a.Xr[int64_t(j0 + jj) * d + m] : 0.f;
    }
    for (int idx = threadIdx.x; idx < EX_J * EX_CB; idx += EX_ROWS) {
      const int c = idx / EX_J, jj = idx % EX_J;
      vj[jj][c] = (c < cw && j0 + jj < n) ? V[int64_t(col0 + c) * n + j0 + jj] : 0.f;
    }
    __syncthreads();
    const int jn = min(EX_J, n - j0);
    for (int jj = 0; jj < jn; ++jj) {
      float dh = 0.f, dl = 0.f;
#pragma unroll
      for (int m = 0; m < EX_MAXD; ++m) {
        if (m < d) {
          const float u = xi[m], v = xj[jj][m];
          const float df = __fsub_rn(u, v);
          const float dz = __fsub_rn(df, u);
          const float df_lo = __fadd_rn(__fsub_rn(u, __fsub_rn(df, dz)), __fsub_rn(-v, dz));
          const float sq = __fmul_rn(df, df);
          dl = __fadd_rn(dl, __fmaf_rn(2.f * df, df_lo, __fmaf_rn(df, df, -sq)));
          const float hi = fmaxf(dh, sq), lo = fminf(dh, sq);
          const float t = __fadd_rn(hi, lo);
          dl = __fadd_rn(dl, __fsub_rn(lo, __fsub_rn(t, hi)));
          dh = t;
        }
      }
      const float a_hi = __fmul_rn(dh, neg_inv2l2);
      const float a_lo = __fmaf_rn(dh, neg_inv2l2, -a_hi) + dl * neg_inv2l2 + dh * neg_inv2l2_lo;
      const float kij = s2 * expf(a_hi) * (1.f + a_lo);
#pragma unroll
      for (int c = 0; c < EX_CB; ++c) acc[c] = fmaf(kij, vj[jj][c], acc[c]);
    }
  }
  if (i < n) {
#pragma unroll
    for (int c = 0; c < EX_CB; ++c)
      if (c < cw) Y[int64_t(col0 + c) * n + i] = acc[c] + noise * V[int64_t(col0 + c) * n + i];
  }
}

// ---------------------------------------------------------------------------
// Derivative forms for the hyperparameter gradient (RBF kernel of Sec. 3):
// for pairs (u_p, v_p), in one pass over the n^2 entries,
//   SD_p = sum_ij u_pi E_ij D_ij v_pj,  SE_p = sum_ij u_pi E_ij v_pj,
//   SI_p = sum_i u_pi v_pi,  E_ij = exp(-D_ij / (2 l^2)), D_ij = |x_i - x_j|^2,
// so that u^T (dA/dl) v = s^2 SD / l^3, u^T (dA/ds^2) v = SE and
// u^T (dA/dnoise) v = SI. 128 rows per CTA (one per thread), PB pairs per
// blockIdx.y, 64-point column tiles in shared memory; float32 sums over a
// tile, float64 across tiles and rows; the last CTA reduces the per-CTA
// partials in a fixed order.
// ---------------------------------------------------------------------------
constexpr int DT_ROWS = 128;
constexpr int DT_J = 64;

template <int DMAX, int PB>
__global__ void __launch_bounds__(DT_ROWS) k_rbf_dtheta(RbfDthetaArgs a) {
  __shared__ float xj[DT_J][DMAX + 1];
  __shared__ float vj[DT_J][PB + 1];
  __shared__ double s_part[DT_ROWS / 32][3 * PB];
  const int n = a.n, d = a.d;
  const int p0 = blockIdx.y * PB;
  const int pw = min(PB, a.npairs - p0);
  const int i = blockIdx.x * DT_ROWS + threadIdx.x;
  const float cexp = -0.5f * a.prm->c2;  // exp(-D / (2 l^2)) = exp2(cexp D)
  float xi[DMAX];
#pragma unroll
  for (int m = 0; m < DMAX; ++m) xi[m] = (i < n && m < d) ? a.Xr[int64_t(i) * d + m] : 0.f;
  double accE[PB], accD[PB];
#pragma unroll
  for (int c = 0; c < PB; ++c) accE[c] = accD[c] = 0.0;
  for (int j0 = 0; j0 < n; j0 += DT_J) {
    __syncthreads();
    for (int idx = threadIdx.x; idx < DT_J * d; idx += DT_ROWS) {
      const int jj = idx / d, m = idx % d;
      xj[jj][m] = (j0 + jj < n) ? a.Xr[int64_t(j0 + jj) * d + m] : 0.f;
    }
    for (int idx = threadIdx.x; idx < DT_J * PB; idx += DT_ROWS) {
      const int c = idx / DT_J, jj = idx % DT_J;
      vj[jj][c] = (c < pw && j0 + jj < n) ? a.V[int64_t(p0 + c) * n + j0 + jj] : 0.f;
    }
    __syncthreads();
    const int jn = min(DT_J, n - j0);
    float tE[PB], tD[PB];
#pragma unroll
    for (int c = 0; c < PB; ++c) tE[c] = tD[c] = 0.f;
    for (int jj = 0; jj < jn; ++jj) {
      float D = 0.f;
#pragma unroll
      for (int m = 0; m < DMAX; ++m) {
        if (m < d) {
          const float df = xi[m] - xj[jj][m];
          D = fmaf(df, df, D);
        }
      }
      const float E = tc::ex2_approx(cexp * D);
      const float ED = E * D;
#pragma unroll
      for (int c = 0; c < PB; ++c) {
        tE[c] = fmaf(E, vj[jj][c], tE[c]);
        tD[c] = fmaf(ED, vj[jj][c], tD[c]);
      }
    }
#pragma unroll
    for (int c = 0; c < PB; ++c) {
      accE[c] += double(tE[c]);
      accD[c] += double(tD[c]);
    }
  }
  // row i's contributions, reduced over the CTA
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int c = 0; c < PB; ++c) {
    double ui = 0.0, vi = 0.0;
    if (i < n && c < pw) {
      ui = double(a.U[int64_t(p0 + c) * n + i]);
      vi = double(a.V[int64_t(p0 + c) * n + i]);
    }
    const double sd = warp_sum(ui * accD[c]);
    const double se = warp_sum(ui * accE[c]);
    const double si = warp_sum(ui * vi);
    if (lane == 0) {
      s_part[warp][3 * c] = sd;
      s_part[warp][3 * c + 1] = se;
      s_part[warp][3 * c + 2] = si;
    }
  }
  __syncthreads();
  const int G = gridDim.x;
  for (int v = threadIdx.x; v < 3 * pw; v += DT_ROWS) {
    double s = 0.0;
    for (int w = 0; w < DT_ROWS / 32; ++w) s += s_part[w][v];
    a.partials[int64_t(3 * p0 + v) * G + blockIdx.x] = s;
  }
  if (!arrive_last(a.ticket)) return;
  for (int v = threadIdx.x; v < 3 * a.npairs; v += DT_ROWS) {
    double s = 0.0;
    for (int b = 0; b < G; ++b) s += __ldcg(a.partials + int64_t(v) * G + b);
    a.out[v] = s;
  }
}

int rbf_dtheta_grid(int n) { return (n + DT_ROWS - 1) / DT_ROWS; }

cudaError_t launch_rbf_dtheta(const RbfDthetaArgs& a, cudaStream_t s) {
  if (a.npairs < 1 || a.npairs > kMaxDthetaPairs || a.d < 1 || a.d > EX_MAXD) return cudaErrorInvalidValue;
  const int gx = rbf_dtheta_grid(a.n);
  if (a.npairs == 1) {
    if (a.d <= 16)
      k_rbf_dtheta<16, 1><<<dim3(gx, 1), DT_ROWS, 0, s>>>(a);
    else
      k_rbf_dtheta<EX_MAXD, 1><<<dim3(gx, 1), DT_ROWS, 0, s>>>(a);
  } else {
    const dim3 grid(gx, (a.npairs + 15) / 16);
    if (a.d <= 16)
      k_rbf_dtheta<16, 16><<<grid, DT_ROWS, 0, s>>>(a);
    else
      k_rbf_dtheta<EX_MAXD, 16><<<grid, DT_ROWS, 0, s>>>(a);
  }
  return cudaGetLastError();
}

int rbf_exact_grid(int n) { return (n + EX_ROWS - 1) / EX_ROWS; }

// J-range splits of the residual kernel (grid.y): enough CTAs for about four
// waves at four resident CTAs per SM, at most one split per J tile.
int rbf_resid_splits(int n, int num_sms) {
  const int rows = rbf_exact_grid(n);
  const int ntiles = (n + EX_J - 1) / EX_J;
  const int want = (16 * num_sms + rows - 1) / rows;
  return max(1, min(min(want, EX_MAX_SPLITS), ntiles));
}

cudaError_t launch_rbf_resid(const RbfExactArgs& a, int splits, cudaStream_t s) {
  if (splits < 1 || splits > EX_MAX_SPLITS || a.d < 1 || a.d > EX_MAXD) return cudaErrorInvalidValue;
  const dim3 grid(rbf_exact_grid(a.n), splits);
  if (a.d <= 8)
    k_rbf_resid<8><<<grid, EX_ROWS, 0, s>>>(a);
  else if (a.d <= 16)
    k_rbf_resid<16><<<grid, EX_ROWS, 0, s>>>(a);
  else if (a.d <= 32)
    k_rbf_resid<32><<<grid, EX_ROWS, 0, s>>>(a);
  else
    k_rbf_resid<64><<<grid, EX_ROWS, 0, s>>>(a);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_rbf_resid_fin<<<rbf_exact_grid(a.n), EX_ROWS, 0, s>>>(a, splits);
  return cudaGetLastError();
}

// Residuals of several systems in one pass over the exact-form entries (the
// checks of a lockstep multi-right-hand-side solve): each entry K_ij is formed
// once, as in k_rbf_resid, and contracted with the iterates of up to EX_NL
// systems, each with its own Dot2 pair, entry-error sum and per-split
// partials; k_rbf_resid_fin then finishes each system on its own. The entry
// costs ~65 float32 instructions at d = 8 and each system ~13 more, so eight
// systems take about a third of eight separate passes.
__host__ __device__ constexpr int ex_resid_multi_min_blocks(int dmax) {
  return dmax <= 8 ? 4 : (dmax <= 16 ? 3 : (dmax <= 32 ? 2 : 1));
}

template <int DMAX>
__global__ void __launch_bounds__(EX_ROWS, ex_resid_multi_min_blocks(DMAX)) k_rbf_resid_multi(RbfResidMultiArgs m) {
  __shared__ __align__(16) float xs[DMAX][EX_J];
  __shared__ __align__(16) float sh_xh[EX_NL][EX_J], sh_xl[EX_NL][EX_J];
  __shared__ __align__(16) float sh_nh[EX_J], sh_nl[EX_J];
  __shared__ float2 exp_tab[64];
  if (threadIdx.x < 64) {
    const double t = exp2(double(threadIdx.x) / 64.0);
    exp_tab[threadIdx.x] = make_float2(float(t), float(t - double(float(t))));
  }
  const RbfExactArgs& a = m.base;
  const int nl = m.nl;
  const int n = a.n, d = a.d, n_pad = a.n_pad;
  const int i = blockIdx.x * EX_ROWS + threadIdx.x;
  const float k_hi = a.prm->neg_inv2l2, k_lo = a.prm->neg_inv2l2_lo;
  const float s2 = a.prm->s2, s2_lo = a.prm->s2_lo;
  const float sigma = a.prm->sigma_anchor;
  const float err0 = kEntryErrC0 + a.prm->err_dist;
  float xi[DMAX];
#pragma unroll
  for (int mm = 0; mm < DMAX; ++mm) xi[mm] = (i < n && mm < d) ? a.XrT[int64_t(mm) * n_pad + i] : 0.f;
  const float nh_i = a.nh[min(i, n_pad - 1)], nl_i = a.nl[min(i, n_pad - 1)];
  float acc[EX_NL], cmp[EX_NL], esq[EX_NL];
#pragma unroll
  for (int l = 0; l < EX_NL; ++l) acc[l] = cmp[l] = esq[l] = 0.f;
  const int ntiles = (n + EX_J - 1) / EX_J;
  for (int tile = blockIdx.y; tile < ntiles; tile += gridDim.y) {
    const int j0 = tile * EX_J;
    __syncthreads();
    for (int idx = threadIdx.x; idx < d * (EX_J / 4); idx += EX_ROWS) {
      const int mm = idx / (EX_J / 4), q = idx % (EX_J / 4);
      *reinterpret_cast<float4*>(&xs[mm][4 * q]) =
          *reinterpret_cast<const float4*>(a.XrT + int64_t(mm) * n_pad + j0 + 4 * q);
    }
    if (threadIdx.x < EX_J) {
      const int j = j0 + threadIdx.x;
      const bool in = j < n;
#pragma unroll
      for (int l = 0; l < EX_NL; ++l) {
        if (l < nl) {
          sh_xh[l][threadIdx.x] = in ? m.xh[l][j] : 0.f;
          sh_xl[l][threadIdx.x] = in ? m.xl[l][j] : 0.f;
        }
      }
      sh_nh[threadIdx.x] = a.nh[j];  // j < n_pad: zero beyond n
      sh_nl[threadIdx.x] = a.nl[j];
    }
    __syncthreads();
    const int jn = min(EX_J, n - j0);
    for (int jq = 0; jq < jn; jq += 4) {
      unsigned long long T01 = tc::f2pk(sigma, sigma), T23 = T01, L01 = 0ull, L23 = 0ull;
#pragma unroll
      for (int mm = 0; mm < DMAX; ++mm) {
        if (mm < d) {
          const float4 x4 = *reinterpret_cast<const float4*>(&xs[mm][jq]);
          const unsigned long long xx = tc::f2pk(xi[mm], xi[mm]);
          anchored_step2(T01, L01, xx, tc::f2pk(x4.x, x4.y));
          anchored_step2(T23, L23, xx, tc::f2pk(x4.z, x4.w));
        }
      }
      const float Tv[4] = {__uint_as_float(unsigned(T01)), __uint_as_float(unsigned(T01 >> 32)),
                           __uint_as_float(unsigned(T23)), __uint_as_float(unsigned(T23 >> 32))};
      const float Lv[4] = {__uint_as_float(unsigned(L01)), __uint_as_float(unsigned(L01 >> 32)),
                           __uint_as_float(unsigned(L23)), __uint_as_float(unsigned(L23 >> 32))};
#pragma unroll
      for (int e4 = 0; e4 < 4; ++e4) {
        const int jj = jq + e4;
        if (jj >= jn) break;
        const float ghi = __fsub_rn(Tv[e4], sigma);
        const float dh = __fmaf_rn(-2.f, ghi, __fadd_rn(nh_i, sh_nh[jj]));
        const float dl = __fmaf_rn(-2.f, Lv[e4], __fadd_rn(nl_i, sh_nl[jj]));
        const float a_hi = __fmul_rn(dh, k_hi);
        const float a_lo = __fmaf_rn(dh, k_hi, -a_hi) + dl * k_hi + dh * k_lo;
        if (a_hi < kExpMinArg) continue;
        float e_hi, e_lo;
        int k2;
        exp_tang(a_hi, a_lo, exp_tab, e_hi, e_lo, k2);
        const float m_hi = __fmul_rn(s2, e_hi);
        const float m_lo = __fmaf_rn(s2, e_hi, -m_hi) + __fmaf_rn(s2, e_lo, s2_lo * e_hi);
        const float scale = __int_as_float((k2 + 127) << 23);
        const float kv_hi = __fmul_rn(m_hi, scale), kv_lo = __fmul_rn(m_lo, scale);
        const float fac = fmaf(3.f, fabsf(a_hi), err0);
#pragma unroll
        for (int l = 0; l < EX_NL; ++l) {
          if (l < nl) {
            const float xhv = sh_xh[l][jj];
            const float p = __fmul_rn(kv_hi, xhv);
            const float pe = __fmaf_rn(kv_hi, xhv, -p);
            two_sum_add(acc[l], cmp[l], p);
            cmp[l] = __fadd_rn(cmp[l], pe);
            cmp[l] = __fmaf_rn(kv_hi, sh_xl[l][jj], __fmaf_rn(kv_lo, xhv, cmp[l]));
            const float e_ij = fac * p;
            esq[l] = fmaf(e_ij, e_ij, esq[l]);
          }
        }
      }
    }
  }
  if (i < n) {
#pragma unroll
    for (int l = 0; l < EX_NL; ++l) {
      if (l < nl) {
        float* part = m.part[l] + int64_t(blockIdx.y) * 3 * n;
        part[i] = acc[l];
        part[n + i] = cmp[l];
        part[2 * n + i] = esq[l];
      }
    }
  }
}

cudaError_t launch_rbf_resid_multi(const RbfResidMultiArgs& m, int splits, cudaStream_t s) {
  const RbfExactArgs& a = m.base;
  if (splits < 1 || splits > EX_MAX_SPLITS || a.d < 1 || a.d > EX_MAXD || m.nl < 1 || m.nl > EX_NL)
    return cudaErrorInvalidValue;
  const dim3 grid(rbf_exact_grid(a.n), splits);
  if (a.d <= 8)
    k_rbf_resid_multi<8><<<grid, EX_ROWS, 0, s>>>(m);
  else if (a.d <= 16)
    k_rbf_resid_multi<16><<<grid, EX_ROWS, 0, s>>>(m);
  else if (a.d <= 32)
    k_rbf_resid_multi<32><<<grid, EX_ROWS, 0, s>>>(m);
  else
    k_rbf_resid_multi<64><<<grid, EX_ROWS, 0, s>>>(m);
  return cudaGetLastError();
}

cudaError_t launch_rbf_resid_fin(const RbfExactArgs& a, int splits, cudaStream_t s) {
  if (splits < 1 || splits > EX_MAX_SPLITS) return cudaErrorInvalidValue;
  k_rbf_resid_fin<<<rbf_exact_grid(a.n), EX_ROWS, 0, s>>>(a, splits);
  return cudaGetLastError();
}

cudaError_t launch_rbf_block(const RbfExactArgs& a, int cmax, cudaStream_t s) {
  if (cmax <= 0) return cudaSuccess;
  dim3 grid(rbf_exact_grid(a.n), (cmax + EX_CB - 1) / EX_CB);
  k_rbf_block<<<grid, EX_ROWS, 0, s>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Throughput of ex2.approx (the special-function unit), the pipe that binds
// the matrix-free matvec for small d: every thread runs 8 independent chains
// v <- 2^v - 1 (one exponential and one add each), 2048 threads per SM.
// ---------------------------------------------------------------------------
constexpr int EXR_CHAINS = 8;
__global__ void __launch_bounds__(512) k_ex2_rate(float* out, int iters) {
  float v[EXR_CHAINS];
#pragma unroll
  for (int i = 0; i < EXR_CHAINS; ++i) v[i] = -0.001f * float(threadIdx.x + i);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < EXR_CHAINS; ++i) v[i] = tc::ex2_approx(v[i]) - 1.0f;
  }
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < EXR_CHAINS; ++i) s += v[i];
  out[int64_t(blockIdx.x) * blockDim.x + threadIdx.x] = s;
}

// out: blocks * 512 floats. Returns the number of exponentials executed.
cudaError_t launch_ex2_rate(float* out, int blocks, int iters, double* count, cudaStream_t s) {
  k_ex2_rate<<<blocks, 512, 0, s>>>(out, iters);
  *count = double(blocks) * 512.0 * double(iters) * EXR_CHAINS;
  return cudaGetLastError();
}

}  // namespace dcg
