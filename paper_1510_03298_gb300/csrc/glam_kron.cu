// Tensor-product weights (Sec. 6.2, Eq. kronweight): when the weight array is a tensor product
// W = w_1 (x) w_2 (x) w_3, X^T W X theta = H(<X_j^T W_j X_j>, theta), so the inner PG loop needs
// only the p_j x p_j matrices M_j = X_j^T diag(w_j) X_j and p-sized arrays.  These kernels find
// the factors of W (and check that W is one), form the M_j in FP64, and apply H(<M_j>, d) to the
// correction of every inner iteration in one launch.
#include <cuda_bf16.h>

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

// Q = H(<M_j>, d) for p-sized arrays (d, Q: (p3, p2, p1) C-order; M_j symmetric p_j x p_j),
// one CTA per output slab j3: the CTA copies all of d into shared memory by asynchronous copies
// (every copy in flight at once: one memory round trip), forms A = sum_k3 M_3(j3, k3) d(k3),
// then B = M_2 A and Q(j3) = B M_1^T.  skip: the inner loop's stop flag (the kernel returns when
// it is set, as every kernel of a captured chunk does).
template <typename T>
__global__ void __launch_bounds__(256)
kron_product_kernel(int p1, int p2, int p3, const T* __restrict__ M1, const T* __restrict__ M2,
                    const T* __restrict__ M3, const T* __restrict__ d, T* __restrict__ Q,
                    const int* __restrict__ skip) {
  if (skip != nullptr && *skip) return;
  extern __shared__ float4 kron_smem[];
  const int P21 = p1 * p2, P = p3 * P21, tid = threadIdx.x, j3 = blockIdx.x;
  T* ds = reinterpret_cast<T*>(kron_smem);  // [p3][P21]
  T* As = ds + ((P + 3) / 4) * 4;            // [P21]
  T* Bs = As + P21;                          // [P21]
  T* m1 = Bs + P21;                          // [p1][p1]
  T* m2 = m1 + p1 * p1;                      // [p2][p2]
  T* m3 = m2 + p2 * p2;                      // [p3]  row j3 of M_3
  constexpr int kVec = 16 / sizeof(T);
  const bool vec = (P % kVec == 0) && ((reinterpret_cast<uintptr_t>(d) & 15) == 0);
  if (vec) {
    for (int i = tid; i < P / kVec; i += 256)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                       static_cast<uint32_t>(__cvta_generic_to_shared(ds + i * kVec))),
                   "l"(d + i * kVec)
                   : "memory");
  } else {
    for (int i = tid; i < P; i += 256)
      asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(
                       static_cast<uint32_t>(__cvta_generic_to_shared(ds + i))),
                   "l"(d + i), "n"(sizeof(T))
                   : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  for (int i = tid; i < p1 * p1; i += 256) m1[i] = M1[i];
  for (int i = tid; i < p2 * p2; i += 256) m2[i] = M2[i];
  for (int i = tid; i < p3; i += 256) m3[i] = M3[(int64_t)j3 * p3 + i];
  asm volatile("cp.async.wait_all;" ::: "memory");
  __syncthreads();
  for (int m = tid; m < P21; m += 256) {
    T a = T(0);
    for (int k3 = 0; k3 < p3; ++k3) a = fma(m3[k3], ds[k3 * P21 + m], a);
    As[m] = a;
  }
  __syncthreads();
  for (int e = tid; e < P21; e += 256) {
    const int j2 = e / p1, k1 = e - j2 * p1;
    T b = T(0);
    for (int k2 = 0; k2 < p2; ++k2) b = fma(m2[j2 * p2 + k2], As[k2 * p1 + k1], b);
    Bs[e] = b;
  }
  __syncthreads();
  for (int e = tid; e < P21; e += 256) {
    const int j2 = e / p1, j1 = e - j2 * p1;
    T q = T(0);
    for (int k1 = 0; k1 < p1; ++k1) q = fma(Bs[j2 * p1 + k1], m1[j1 * p1 + k1], q);
    Q[(int64_t)j3 * P21 + e] = q;
  }
}

template <typename T>
size_t kron_product_smem(int p1, int p2, int p3) {
  const int64_t P21 = (int64_t)p1 * p2, P = P21 * p3;
  return sizeof(T) * (size_t)((P + 3) / 4 * 4 + 2 * P21 + (int64_t)p1 * p1 + (int64_t)p2 * p2 + p3);
}

// ---- geometric-mean tensor approximation of a weight array V (Sec. 6.2, "tensor approximation")
// v_j(i) = exp(mean of log V over the cells of slice i of mode j - mean of log V over all cells),
// the means taken over the cells with V > 0 (a masked cell carries no weight to approximate).
// Pass 1: CTA i3 sums log V over its slab per i1 (over i2) and per i2 (over i1), with counts, in
// a fixed order.  V is C-order (n3, n2, n1).
template <typename TV>
__device__ __forceinline__ double geo_log(TV v, int& cnt) {
  const double x = (double)v;
  if (x > 0.0) {
    ++cnt;
    return log(x);
  }
  return 0.0;
}
template <typename TV>
__global__ void geo_slab_kernel(int n1, int n2, const TV* __restrict__ V, double* __restrict__ s1p,
                                int* __restrict__ c1p, double* __restrict__ s2p, int* __restrict__ c2p) {
  const int i3 = blockIdx.x;
  const TV* Vs = V + (int64_t)i3 * n1 * n2;
  for (int i1 = threadIdx.x; i1 < n1; i1 += blockDim.x) {  // per i1: over i2 in order
    double s = 0.0;
    int c = 0;
    for (int i2 = 0; i2 < n2; ++i2) s += geo_log(Vs[(int64_t)i2 * n1 + i1], c);
    s1p[(int64_t)i3 * n1 + i1] = s;
    c1p[(int64_t)i3 * n1 + i1] = c;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int i2 = warp; i2 < n2; i2 += nw) {  // per i2: lane-strided over i1, then a fixed tree
    double s = 0.0;
    int c = 0;
    for (int i1 = lane; i1 < n1; i1 += 32) s += geo_log(Vs[(int64_t)i2 * n1 + i1], c);
    for (int o = 16; o > 0; o >>= 1) {
      s += __shfl_xor_sync(0xffffffffu, s, o);
      c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    if (lane == 0) {
      s2p[(int64_t)i3 * n2 + i2] = s;
      c2p[(int64_t)i3 * n2 + i2] = c;
    }
  }
}
// Pass 2: per index of each mode, the sum of the slab partials in slab order (mode 3: of its own
// slab's per-i2 partials in i2 order); sums go to s[n1 + n2 + n3], counts to c[...].
__global__ void geo_mode_kernel(int n1, int n2, int n3, const double* __restrict__ s1p, const int* __restrict__ c1p,
                                const double* __restrict__ s2p, const int* __restrict__ c2p,
                                double* __restrict__ s, int* __restrict__ c) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  double a = 0.0;
  int k = 0;
  if (t < n1) {
    for (int i3 = 0; i3 < n3; ++i3) a += s1p[(int64_t)i3 * n1 + t], k += c1p[(int64_t)i3 * n1 + t];
  } else if (t < n1 + n2) {
    const int i2 = t - n1;
    for (int i3 = 0; i3 < n3; ++i3) a += s2p[(int64_t)i3 * n2 + i2], k += c2p[(int64_t)i3 * n2 + i2];
  } else if (t < n1 + n2 + n3) {
    const int i3 = t - n1 - n2;
    for (int i2 = 0; i2 < n2; ++i2) a += s2p[(int64_t)i3 * n2 + i2], k += c2p[(int64_t)i3 * n2 + i2];
  } else {
    return;
  }
  s[t] = a;
  c[t] = k;
}
// Pass 3 (one CTA): the overall mean of log V (the slab sums in slab order), then the factors;
// a slice without a positive cell gets the neutral factor 1.  scaled multiplies v_1 by the
// overall geometric mean, so that the product reproduces a tensor-product V exactly.
__global__ void geo_factor_kernel(int n1, int n2, int n3, const double* __restrict__ s, const int* __restrict__ c,
                                  int scaled, double* __restrict__ v1, double* __restrict__ v2,
                                  double* __restrict__ v3) {
  __shared__ double mean_all;
  if (threadIdx.x == 0) {
    double a = 0.0;
    long long k = 0;
    for (int i3 = 0; i3 < n3; ++i3) a += s[n1 + n2 + i3], k += c[n1 + n2 + i3];
    mean_all = k > 0 ? a / (double)k : 0.0;
  }
  __syncthreads();
  const double lm = mean_all;
  for (int t = threadIdx.x; t < n1 + n2 + n3; t += blockDim.x) {
    const double f = c[t] > 0 ? exp(s[t] / (double)c[t] - lm) : 1.0;
    if (t < n1) v1[t] = scaled ? f * exp(lm) : f;
    else if (t < n1 + n2) v2[t - n1] = f;
    else v3[t - n1 - n2] = f;
  }
}

}  // namespace

template <typename T>
int kron_product_supported(int p1, int p2, int p3) {
  return kron_product_smem<T>(p1, p2, p3) <= 200 * 1024 ? 1 : 0;
}

template <typename T>
cudaError_t kron_product_prepare(int p1, int p2, int p3) {
  if (!kron_product_supported<T>(p1, p2, p3)) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(kron_product_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)kron_product_smem<T>(p1, p2, p3));
}

template <typename T>
cudaError_t launch_kron_product(int p1, int p2, int p3, const T* M1, const T* M2, const T* M3,
                                const T* d, T* Q, const int* skip, cudaStream_t s) {
  if (!kron_product_supported<T>(p1, p2, p3)) return cudaErrorInvalidValue;
  const size_t smem = kron_product_smem<T>(p1, p2, p3);
  kron_product_kernel<T><<<p3, 256, smem, s>>>(p1, p2, p3, M1, M2, M3, d, Q, skip);
  count_launches(1);
  return cudaGetLastError();
}

template int kron_product_supported<float>(int, int, int);
template cudaError_t kron_product_prepare<float>(int, int, int);
template cudaError_t kron_product_prepare<double>(int, int, int);
template int kron_product_supported<double>(int, int, int);
template cudaError_t launch_kron_product<float>(int, int, int, const float*, const float*, const float*,
                                                const float*, float*, const int*, cudaStream_t);
template cudaError_t launch_kron_product<double>(int, int, int, const double*, const double*,
                                                 const double*, const double*, double*, const int*,
                                                 cudaStream_t);

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

template <typename TV>
cudaError_t launch_geo_factors(int n1, int n2, int n3, const TV* V, int scaled, double* scratch, double* v1,
                               double* v2, double* v3, cudaStream_t s) {
  // scratch: (n1 + n2) n3 doubles and as many ints, then n1 + n2 + n3 doubles and ints
  double* s1p = scratch;
  double* s2p = s1p + (int64_t)n1 * n3;
  int* c1p = reinterpret_cast<int*>(s2p + (int64_t)n2 * n3);
  int* c2p = c1p + (int64_t)n1 * n3;
  double* sm = reinterpret_cast<double*>(c2p + (int64_t)n2 * n3 + ((int64_t)(n1 + n2) * n3 % 2));
  int* cm = reinterpret_cast<int*>(sm + n1 + n2 + n3);
  geo_slab_kernel<TV><<<n3, 256, 0, s>>>(n1, n2, V, s1p, c1p, s2p, c2p);
  const int m = n1 + n2 + n3;
  geo_mode_kernel<<<(m + 127) / 128, 128, 0, s>>>(n1, n2, n3, s1p, c1p, s2p, c2p, sm, cm);
  geo_factor_kernel<<<1, 256, 0, s>>>(n1, n2, n3, sm, cm, scaled, v1, v2, v3);
  count_launches(3);
  return cudaGetLastError();
}
int64_t geo_scratch_doubles(int64_t n1, int64_t n2, int64_t n3) {
  return (n1 + n2) * n3 * 2 + 1 + (n1 + n2 + n3) * 2;
}
template cudaError_t launch_geo_factors<float>(int, int, int, const float*, int, double*, double*, double*,
                                               double*, cudaStream_t);
template cudaError_t launch_geo_factors<double>(int, int, int, const double*, int, double*, double*, double*,
                                                double*, cudaStream_t);
template cudaError_t launch_geo_factors<__nv_bfloat16>(int, int, int, const __nv_bfloat16*, int, double*,
                                                       double*, double*, double*, cudaStream_t);

template cudaError_t launch_kron_factors<float>(int64_t, int64_t, int64_t, const float*, double*, double*,
                                                double*, unsigned long long*, cudaStream_t);
template cudaError_t launch_kron_factors<double>(int64_t, int64_t, int64_t, const double*, double*,
                                                 double*, double*, unsigned long long*, cudaStream_t);

}  // namespace glam
