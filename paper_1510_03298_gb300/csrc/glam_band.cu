// Banded mode products (a specialisation for marginal designs with at most kBand consecutive
// nonzeros per row, as cubic B-spline bases have; the paper's method takes dense designs, Sec.
// 6.1).  A design X (n rows, p columns) is held as start(i) and the kBand values of row i from
// column start(i); starts are nondecreasing, so the rows touching column j form the range
// [lo(j), hi(j)).  One mode product of rho (App. A) on an array In[A][C_in][B]:
//   forward (H):  Out[a][i][b] = sum_t X(i, start(i) + t) In[a][start(i) + t][b]
//   adjoint (G):  Out[a][j][b] = sum_{i = lo(j)}^{hi(j) - 1} X(i, j) In[a][i][b]
// one thread per output, the terms in a fixed order, FP64.
#include "glam_internal.cuh"

namespace glam {
namespace {

__global__ void band_fwd_kernel(int64_t A, int Cin, int Cout, int64_t B, const int* __restrict__ start,
                                const double* __restrict__ val, const double* __restrict__ In, double* __restrict__ Out) {
  const int64_t total = A * Cout * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e % B, r = e / B;
    const int i = (int)(r % Cout);
    const int64_t a = r / Cout;
    const int s = start[i];
    double acc = 0.0;
#pragma unroll
    for (int t = 0; t < kBand; ++t)
      if (s + t < Cin) acc = fma(val[i * kBand + t], In[(a * Cin + s + t) * B + b], acc);
    Out[e] = acc;
  }
}

__global__ void band_adj_kernel(int64_t A, int Cin, int Cout, int64_t B, const int* __restrict__ start,
                                const double* __restrict__ val, const int* __restrict__ lo, const int* __restrict__ hi,
                                const double* __restrict__ In, double* __restrict__ Out) {
  const int64_t total = A * Cout * B;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e % B, r = e / B;
    const int j = (int)(r % Cout);
    const int64_t a = r / Cout;
    double acc = 0.0;
    for (int i = lo[j]; i < hi[j]; ++i) acc = fma(val[i * kBand + (j - start[i])], In[(a * Cin + i) * B + b], acc);
    Out[e] = acc;
  }
}

int band_grid(int64_t total) {
  int64_t g = (total + 255) / 256;
  const int64_t cap = 8 * (int64_t)num_sms();
  return (int)(g < 1 ? 1 : (g > cap ? cap : g));
}

}  // namespace

cudaError_t launch_band_fwd(int64_t A, int Cin, int Cout, int64_t B, const BandDesign& X, const double* In,
                            double* Out, cudaStream_t s) {
  band_fwd_kernel<<<band_grid(A * Cout * B), 256, 0, s>>>(A, Cin, Cout, B, X.start, X.val, In, Out);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_band_adj(int64_t A, int Cin, int Cout, int64_t B, const BandDesign& X, const double* In,
                            double* Out, cudaStream_t s) {
  band_adj_kernel<<<band_grid(A * Cout * B), 256, 0, s>>>(A, Cin, Cout, B, X.start, X.val, X.lo, X.hi, In, Out);
  count_launches(1);
  return cudaGetLastError();
}

// Host side: the band form of X^T (p x n, row-major, i.e. X column-major n x p) when every row has
// its nonzeros within kBand consecutive columns and the first columns do not decrease; false
// otherwise.
bool band_form(const double* XT, int n, int p, std::vector<int>& start, std::vector<double>& val,
               std::vector<int>& lo, std::vector<int>& hi) {
  start.assign(n, 0);
  val.assign((size_t)n * kBand, 0.0);
  int prev = 0;
  for (int i = 0; i < n; ++i) {
    int first = -1, last = -1;
    for (int j = 0; j < p; ++j)
      if (XT[(size_t)j * n + i] != 0.0) {
        if (first < 0) first = j;
        last = j;
      }
    if (first < 0) first = last = prev;  // an all-zero row keeps the previous start
    int s = first;
    if (s + kBand > p) s = p - kBand > 0 ? p - kBand : 0;
    if (last - s >= kBand || s < prev) return false;
    for (int t = 0; t < kBand && s + t < p; ++t) val[(size_t)i * kBand + t] = XT[(size_t)(s + t) * n + i];
    start[i] = s;
    prev = s;
  }
  lo.assign(p, 0);
  hi.assign(p, 0);
  for (int j = 0; j < p; ++j) {  // rows i with start(i) <= j < start(i) + kBand: a contiguous range
    int a = 0;
    while (a < n && start[a] + kBand <= j) ++a;
    int b = a;
    while (b < n && start[b] <= j) ++b;
    lo[j] = a;
    hi[j] = b;
  }
  return true;
}

}  // namespace glam
