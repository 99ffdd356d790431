// Tensor-product weights (Sec. 6.2, Eq. kronweight): when the weight array is a tensor product
// W = w_1 (x) w_2 (x) w_3, X^T W X theta = H(<X_j^T W_j X_j>, theta), so the inner PG loop needs
// only the p_j x p_j matrices M_j = X_j^T diag(w_j) X_j and p-sized arrays.  These kernels find
// the factors of W (and check that W is one), and form the M_j in FP64.
#include <algorithm>

#include "glam_internal.cuh"

namespace glam {
namespace {

// Factors read off W (C-order (n3, n2, n1)): w1(i1) = W(0, 0, i1), w2(i2) = W(0, i2, 0) / W(0, 0, 0),
// w3(i3) = W(i3, 0, 0) / W(0, 0, 0), so that w1(i1) w2(i2) w3(i3) = W whenever W is a tensor product
// with W(0, 0, 0) > 0.
template <typename T>
__global__ void kron_factor_kernel(int64_t n1, int64_t n2, int64_t n3, const T* __restrict__ W,
                                   double* __restrict__ w1, double* __restrict__ w2,
                                   double* __restrict__ w3) {
  const double w000 = (double)W[0];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n1) w1[i] = (double)W[i];
  if (i < n2) w2[i] = (double)W[i * n1] / w000;
  if (i < n3) w3[i] = (double)W[i * n1 * n2] / w000;
}

// out[0] = max_i |W_i - w1 w2 w3|, out[1] = max_i |W_i| (atomic maxima of non-negative doubles)
template <typename T>
__global__ void kron_check_kernel(int64_t n1, int64_t n2, int64_t n, const T* __restrict__ W,
                                  const double* __restrict__ w1, const double* __restrict__ w2,
                                  const double* __restrict__ w3, unsigned long long* out) {
  double dev = 0.0, mx = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i1 = i % n1, r = i / n1, i2 = r % n2, i3 = r / n2;
    const double w = (double)W[i];
    dev = fmax(dev, fabs(w - w1[i1] * w2[i2] * w3[i3]));
    mx = fmax(mx, fabs(w));
  }
  for (int o = 16; o > 0; o >>= 1) {
    dev = fmax(dev, __shfl_xor_sync(0xffffffffu, dev, o));
    mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  }
  if ((threadIdx.x & 31) == 0) {
    atomicMax(&out[0], (unsigned long long)__double_as_longlong(dev));
    atomicMax(&out[1], (unsigned long long)__double_as_longlong(mx));
  }
}

// M[a][b] = sum_i X(i, a) w(i) X(i, b) for a marginal design stored as XT (p_j, n_j), FP64
__global__ void weighted_gram_kernel(int nj, int pj, const double* __restrict__ XT,
                                     const double* __restrict__ w, double* __restrict__ M) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= pj * pj) return;
  const int a = e / pj, b = e - a * pj;
  double s = 0.0;
  for (int i = 0; i < nj; ++i) s += XT[(int64_t)a * nj + i] * w[i] * XT[(int64_t)b * nj + i];
  M[e] = s;
}

}  // namespace

template <typename T>
cudaError_t launch_kron_factors(int64_t n1, int64_t n2, int64_t n3, const T* W, double* w1, double* w2,
                                double* w3, unsigned long long* check, cudaStream_t s) {
  const int64_t m = std::max(n1, std::max(n2, n3));
  kron_factor_kernel<T><<<(unsigned)((m + 255) / 256), 256, 0, s>>>(n1, n2, n3, W, w1, w2, w3);
  count_launches(1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = cudaMemsetAsync(check, 0, 2 * sizeof(unsigned long long), s);
  if (e != cudaSuccess) return e;
  const int64_t n = n1 * n2 * n3;
  int64_t blocks = (n + 255) / 256;
  if (blocks > 4 * (int64_t)num_sms()) blocks = 4 * (int64_t)num_sms();
  kron_check_kernel<T><<<(unsigned)blocks, 256, 0, s>>>(n1, n2, n, W, w1, w2, w3, check);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_weighted_gram(int nj, int pj, const double* XT, const double* w, double* M,
                                 cudaStream_t s) {
  weighted_gram_kernel<<<(pj * pj + 127) / 128, 128, 0, s>>>(nj, pj, XT, w, M);
  count_launches(1);
  return cudaGetLastError();
}

template cudaError_t launch_kron_factors<float>(int64_t, int64_t, int64_t, const float*, double*, double*,
                                                double*, unsigned long long*, cudaStream_t);
template cudaError_t launch_kron_factors<double>(int64_t, int64_t, int64_t, const double*, double*,
                                                 double*, double*, unsigned long long*, cudaStream_t);

}  // namespace glam
