// Lockstep solves of several right-hand sides (dcg_solve_multi): each system
// keeps its own iterate, residual, direction and solver state and runs the
// kernels of a single solve (Algorithm 1); what the systems share is the
// operator pass. Per iteration:
//   k_multi_gather  copies the directions p of the systems still running into
//                   the columns of one block (the matrix-free product reads
//                   whole 128-row tiles: the padded length, zero beyond n);
//   (block product  Q = A P: k_rbf_p16 + k_rbf_mv_tc for the matrix-free
//                   operator, the stored block product otherwise)
//   k_multi_pq      p^T q of every column into its system's state, the d of
//                   Algorithm 1 that the fused iteration kernel divides by.
#include <algorithm>

#include "dcg_kernels.cuh"

namespace dcg {

__global__ void __launch_bounds__(256) k_multi_gather(const float* __restrict__ src, int64_t lds, MultiLanes lanes,
                                                      int rows, float* __restrict__ dst, int64_t ldd) {
  const int j = blockIdx.y;
  const float* s = src + int64_t(lanes.idx[j]) * lds;
  float* d = dst + int64_t(j) * ldd;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < rows; i += gridDim.x * blockDim.x) d[i] = s[i];
}

cudaError_t launch_multi_gather(const float* src, int64_t lds, const MultiLanes& lanes, int na, int rows, float* dst,
                                int64_t ldd, cudaStream_t s) {
  if (na < 1 || na > DCG_MAX_RHS) return cudaErrorInvalidValue;
  const dim3 grid(std::max(1, std::min(64, (rows + 1023) / 1024)), na);
  k_multi_gather<<<grid, 256, 0, s>>>(src, lds, lanes, rows, dst, ldd);
  return cudaGetLastError();
}

// One CTA per column: the float64 sum of p_i q_i over its rows, strided per
// thread, then a warp tree and the warps in order (the same order every
// call), written to the state of system lanes.idx[j].
constexpr int MPQ_THREADS = 512;

__global__ void __launch_bounds__(MPQ_THREADS) k_multi_pq(const float* __restrict__ P, const float* __restrict__ Q,
                                                          int64_t ld, int n, MultiLanes lanes, DevState* states) {
  __shared__ double red[MPQ_THREADS / 32];
  const int j = blockIdx.x;
  const float* p = P + int64_t(j) * ld;
  const float* q = Q + int64_t(j) * ld;
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += MPQ_THREADS) s = fma(double(p[i]), double(q[i]), s);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  s = warp_sum(s);
  if (lane == 0) red[warp] = s;
  __syncthreads();
  if (warp == 0) {
    double v = lane < MPQ_THREADS / 32 ? red[lane] : 0.0;
    v = warp_sum(v);
    if (lane == 0) states[lanes.idx[j]].d = v;
  }
}

cudaError_t launch_multi_pq(const float* P, const float* Q, int64_t ld, int n, const MultiLanes& lanes, int na,
                            DevState* states, cudaStream_t s) {
  if (na < 1 || na > DCG_MAX_RHS) return cudaErrorInvalidValue;
  k_multi_pq<<<na, MPQ_THREADS, 0, s>>>(P, Q, ld, n, lanes, states);
  return cudaGetLastError();
}

}  // namespace dcg
