// The paper's own workload (Sec. 3): the Newton loop of the Laplace
// approximation for binary GP classification with the logistic likelihood
// p(y_i | f_i) = sigma(y_i f_i). One Newton step at the latent f (Eq. obj,
// Eq. linsys, the restructured form of Kuss and Rasmussen):
//   pi = sigma(f), H = diag(pi (1 - pi)), s = H^{1/2},
//   c = H f + grad log p(y | f) = H f + (y + 1) / 2 - pi,
//   A = I + S K S,  b = S K c            (the system def-CG solves),
//   a = c - S x,    f_new = K a,  Psi = log p(y | f_new) - 1/2 f_new^T a.
// The elementwise steps run here in float64 (n values); A is written from
// the stored K in one HBM pass; the products K c and K a go through the
// stored-operator GEMV.
#include <algorithm>

#include "dcg_kernels.cuh"

namespace dcg {

// log sigma(z) = -log(1 + exp(-z)), without overflow for large |z|
__device__ __forceinline__ double log_sigmoid(double z) {
  return z >= 0.0 ? -log1p(exp(-z)) : z - log1p(exp(z));
}

__global__ void k_lap_prep(const float* __restrict__ y, const double* __restrict__ f, int n, float* s, double* c,
                           float* c32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double fi = f[i];
    const double pi = fi >= 0.0 ? 1.0 / (1.0 + exp(-fi)) : exp(fi) / (1.0 + exp(fi));
    const double h = pi * (1.0 - pi);
    const double ci = h * fi + (0.5 * (double(y[i]) + 1.0) - pi);
    s[i] = float(sqrt(h));
    c[i] = ci;
    c32[i] = float(ci);
  }
}

__global__ void k_lap_scale(const float* __restrict__ s, const float* __restrict__ v, int n, float* out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) out[i] = s[i] * v[i];
}

// A = I + S K S, row-major, four columns per thread (lda and ldk multiples of 4)
__global__ void k_lap_form(const float* __restrict__ K, int64_t ldk, const float* __restrict__ s, int n, float* A,
                           int64_t lda) {
  const int nq = (n + 3) / 4;
  for (int row = blockIdx.y; row < n; row += gridDim.y) {
    const float si = s[row];
    const float4* krow = reinterpret_cast<const float4*>(K + int64_t(row) * ldk);
    float4* arow = reinterpret_cast<float4*>(A + int64_t(row) * lda);
    for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += gridDim.x * blockDim.x) {
      const int j = 4 * q;
      const float4 k4 = __ldcs(krow + q);
      float4 o;
      // (s_i s_j) K_ij: the product of the scales commutes exactly, so A is
      // exactly symmetric when K is
      o.x = j + 0 < n ? (si * s[j + 0]) * k4.x + (j + 0 == row ? 1.f : 0.f) : 0.f;
      o.y = j + 1 < n ? (si * s[j + 1]) * k4.y + (j + 1 == row ? 1.f : 0.f) : 0.f;
      o.z = j + 2 < n ? (si * s[j + 2]) * k4.z + (j + 2 == row ? 1.f : 0.f) : 0.f;
      o.w = j + 3 < n ? (si * s[j + 3]) * k4.w + (j + 3 == row ? 1.f : 0.f) : 0.f;
      arow[q] = o;
    }
  }
}

__global__ void k_lap_a(const double* __restrict__ c, const float* __restrict__ s, const double* __restrict__ x, int n,
                        double* a, float* a32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double ai = c[i] - double(s[i]) * x[i];
    a[i] = ai;
    a32[i] = float(ai);
  }
}

// f = float64(K a); Psi = sum_i log sigma(y_i f_i) - 1/2 sum_i f_i a_i, CTA
// partials and a fixed-order sum by the last CTA
__global__ void __launch_bounds__(256) k_lap_psi(const float* __restrict__ y, const float* __restrict__ f32,
                                                 const double* __restrict__ a, int n, double* f, double* partials,
                                                 unsigned int* ticket, double* psi) {
  double acc = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double fi = double(f32[i]);
    f[i] = fi;
    acc += log_sigmoid(double(y[i]) * fi) - 0.5 * fi * a[i];
  }
  __shared__ double s_part[8];
  const double v = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) s_part[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += s_part[w];
    partials[blockIdx.x] = t;
  }
  if (!arrive_last(ticket)) return;
  if (threadIdx.x < 32) {
    double t = 0.0;
    for (int b = threadIdx.x; b < int(gridDim.x); b += 32) t += __ldcg(partials + b);
    t = warp_sum(t);
    if (threadIdx.x == 0) *psi = t;
  }
}

int lap_grid(int n, int num_sms) { return std::min((n + 255) / 256, 2 * num_sms); }

cudaError_t launch_lap_prep(const float* y, const double* f, int n, float* s, double* c, float* c32, int grid,
                            cudaStream_t st) {
  k_lap_prep<<<grid, 256, 0, st>>>(y, f, n, s, c, c32);
  return cudaGetLastError();
}

cudaError_t launch_lap_scale(const float* s, const float* v, int n, float* out, int grid, cudaStream_t st) {
  k_lap_scale<<<grid, 256, 0, st>>>(s, v, n, out);
  return cudaGetLastError();
}

cudaError_t launch_lap_form(const float* K, int64_t ldk, const float* s, int n, float* A, int64_t lda,
                            cudaStream_t st) {
  const int nq = (n + 3) / 4;
  const dim3 grid(std::max(1, std::min((nq + 255) / 256, 8)), std::min(n, 65535));
  k_lap_form<<<grid, 256, 0, st>>>(K, ldk, s, n, A, lda);
  return cudaGetLastError();
}

cudaError_t launch_lap_a(const double* c, const float* s, const double* x, int n, double* a, float* a32, int grid,
                         cudaStream_t st) {
  k_lap_a<<<grid, 256, 0, st>>>(c, s, x, n, a, a32);
  return cudaGetLastError();
}

cudaError_t launch_lap_psi(const float* y, const float* f32, const double* a, int n, double* f, double* partials,
                           unsigned int* ticket, double* psi, int grid, cudaStream_t st) {
  k_lap_psi<<<grid, 256, 0, st>>>(y, f32, a, n, f, partials, ticket, psi);
  return cudaGetLastError();
}

}  // namespace dcg
