// The bottleneck of GD-PG (Sec. 6.2): X^T W X theta = G(V (.) H(Theta)) (Sec. 6.1, Eq.
// twentysixnew), with the last two stages of H and the first two stages of G fused per slab.
//
// Mode order: H contracts mode 3 first (T_a = rho over X_3, computed by the GEMM kernel), then
// mode 1 and mode 2 inside this kernel; G contracts mode 2, then mode 1 inside this kernel, and
// mode 3 last (GEMM kernel).  For one slab i3 (a contiguous n2 x n1 block of V):
//   T_b  (p2 x n1) = T_a[i3] (p2 x p1) . X_1^T        phase 1
//   eta  (n2 x n1) = X_2 (n2 x p2) . T_b              phase 2 (registers only)
//   r            = V[i3] (.) eta                      phase 2
//   S    (p2 x n1) = X_2^T . r                        phase 2 (registers, then shared memory)
//   S_b[i3] (p2 x p1) = S . X_1                       phase 3
// eta and r never leave the SM: per inner iteration the kernel streams V once from memory and
// touches only the small T_a / S_b slabs otherwise.
//
// Phase 2 mapping: lanes walk the unit-stride index i1 (coalesced V loads), warps split the
// columns into 32-wide tiles and the rows i2 into RG groups.  Each lane holds its column of T_b
// and its column of S (P values each) in registers; the X_2 row is read from shared memory with
// 16-byte broadcast loads and used twice (for eta and for S).
#include "glam_internal.cuh"

namespace glam {
namespace {

template <typename T>
struct Vec16;
template <>
struct Vec16<float> {
  using type = float4;
  static constexpr int width = 4;
};
template <>
struct Vec16<double> {
  using type = double2;
  static constexpr int width = 2;
};

template <typename T, int P>
__device__ __forceinline__ void load_row(const T* __restrict__ src, T (&dst)[P]) {
  using V = typename Vec16<T>::type;
  constexpr int W = Vec16<T>::width;
  const V* s = reinterpret_cast<const V*>(src);
#pragma unroll
  for (int q = 0; q < P / W; ++q) {
    V v = s[q];
    if constexpr (W == 4) {
      dst[4 * q + 0] = v.x;
      dst[4 * q + 1] = v.y;
      dst[4 * q + 2] = v.z;
      dst[4 * q + 3] = v.w;
    } else {
      dst[2 * q + 0] = v.x;
      dst[2 * q + 1] = v.y;
    }
  }
}

struct SlabShape {
  int n1, n2, n3, p1, p2, CT, RG, LD;
};

template <typename T, int P>
__global__ void __launch_bounds__(256)
fused_slab_kernel(SlabShape sh, const T* __restrict__ X1T, const T* __restrict__ X2T,
                  const T* __restrict__ Ta, const T* __restrict__ V, T* __restrict__ Sb,
                  const int* __restrict__ skip) {
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int n1 = sh.n1, n2 = sh.n2, p1 = sh.p1, p2 = sh.p2, LD = sh.LD;
  T* X2s = reinterpret_cast<T*>(smem_raw);        // [n2][P]   X2s[i2][j2] = X_2(i2, j2)
  T* X1s = X2s + n2 * P;                          // [p1][LD]  X1s[j1][i1] = X_1(i1, j1)
  T* Tas = X1s + p1 * LD;                         // [p2 * p1] (rounded up to 4)
  T* Tbs = Tas + ((p2 * p1 + 3) & ~3);            // [P][LD]
  T* Sred = Tbs + P * LD;                         // [RG][P][LD]
  const int tid = threadIdx.x, nth = blockDim.x;
  const int i3 = blockIdx.x;

  for (int idx = tid; idx < n2 * P; idx += nth) {
    const int i2 = idx / P, j2 = idx - i2 * P;
    X2s[idx] = (j2 < p2) ? X2T[(int64_t)j2 * n2 + i2] : T(0);
  }
  for (int idx = tid; idx < p1 * n1; idx += nth) {
    const int j1 = idx / n1, i1 = idx - j1 * n1;
    X1s[j1 * LD + i1] = X1T[idx];
  }
  const T* ta = Ta + (int64_t)i3 * p2 * p1;
  for (int idx = tid; idx < p2 * p1; idx += nth) Tas[idx] = ta[idx];
  __syncthreads();

  // phase 1: T_b = T_a[i3] . X_1^T  (mode-1 product of the slab)
  for (int idx = tid; idx < P * n1; idx += nth) {
    const int j2 = idx / n1, c = idx - j2 * n1;
    T acc = T(0);
    if (j2 < p2) {
      for (int j1 = 0; j1 < p1; ++j1) acc = fma(Tas[j2 * p1 + j1], X1s[j1 * LD + c], acc);
    }
    Tbs[j2 * LD + c] = acc;
  }
  __syncthreads();

  // phase 2: eta = X_2 T_b, r = V (.) eta, S = X_2^T r  (fused mode-2 products)
  const int warp = tid >> 5, lane = tid & 31, nwarps = nth >> 5;
  const T* Vs = V + (int64_t)i3 * n2 * n1;
  for (int task = warp; task < sh.CT * sh.RG; task += nwarps) {
    const int ct = task % sh.CT, rg = task / sh.CT;
    const int c = ct * 32 + lane;
    const bool valid = c < n1;
    const int r0 = (int)(((int64_t)n2 * rg) / sh.RG);
    const int r1 = (int)(((int64_t)n2 * (rg + 1)) / sh.RG);
    T tb[P], s[P];
#pragma unroll
    for (int j = 0; j < P; ++j) {
      tb[j] = valid ? Tbs[j * LD + c] : T(0);
      s[j] = T(0);
    }
    const T* vcol = Vs + (valid ? c : 0);
#pragma unroll 2
    for (int i2 = r0; i2 < r1; ++i2) {
      T x2[P];
      load_row<T, P>(X2s + i2 * P, x2);
      T e0 = T(0), e1 = T(0), e2 = T(0), e3 = T(0);
#pragma unroll
      for (int j = 0; j < P; j += 4) {
        e0 = fma(x2[j + 0], tb[j + 0], e0);
        e1 = fma(x2[j + 1], tb[j + 1], e1);
        e2 = fma(x2[j + 2], tb[j + 2], e2);
        e3 = fma(x2[j + 3], tb[j + 3], e3);
      }
      const T v = valid ? vcol[(int64_t)i2 * n1] : T(0);
      const T r = v * ((e0 + e1) + (e2 + e3));
#pragma unroll
      for (int j = 0; j < P; ++j) s[j] = fma(x2[j], r, s[j]);
    }
    if (valid) {
#pragma unroll
      for (int j = 0; j < P; ++j) Sred[(rg * P + j) * LD + c] = s[j];
    }
  }
  __syncthreads();
  if (sh.RG > 1) {
    for (int idx = tid; idx < p2 * n1; idx += nth) {
      const int j2 = idx / n1, c = idx - j2 * n1;
      T acc = Sred[j2 * LD + c];
      for (int rg = 1; rg < sh.RG; ++rg) acc += Sred[(rg * P + j2) * LD + c];
      Sred[j2 * LD + c] = acc;
    }
    __syncthreads();
  }

  // phase 3: S_b[i3] = S . X_1  (mode-1 product back to p1)
  T* out = Sb + (int64_t)i3 * p2 * p1;
  for (int o = tid; o < p2 * p1; o += nth) {
    const int j2 = o / p1, j1 = o - j2 * p1;
    const T* srow = Sred + j2 * LD;
    const T* xrow = X1s + j1 * LD;
    T a0 = T(0), a1 = T(0);
    int c = 0;
    for (; c + 1 < n1; c += 2) {
      a0 = fma(srow[c], xrow[c], a0);
      a1 = fma(srow[c + 1], xrow[c + 1], a1);
    }
    if (c < n1) a0 = fma(srow[c], xrow[c], a0);
    out[o] = a0 + a1;
  }
}

constexpr int kPs[] = {8, 12, 16, 20, 24, 28, 32};

int pick_P(int p2) {
  for (int P : kPs)
    if (p2 <= P) return P;
  return 0;
}

void slab_config(int n1, int n2, int p1, int p2, SlabShape& sh, int& threads) {
  sh.n1 = n1;
  sh.n2 = n2;
  sh.p1 = p1;
  sh.p2 = p2;
  sh.CT = (n1 + 31) / 32;
  sh.RG = sh.CT >= 8 ? 1 : 8 / sh.CT;
  if (sh.RG > n2) sh.RG = n2 > 0 ? n2 : 1;
  sh.LD = n1 + 1;
  threads = 32 * sh.CT * sh.RG;
}

size_t slab_smem(const SlabShape& sh, int P, int elem) {
  size_t e = (size_t)sh.n2 * P + (size_t)sh.p1 * sh.LD + (((size_t)sh.p2 * sh.p1 + 3) & ~(size_t)3) +
             (size_t)P * sh.LD * (1 + sh.RG);
  return e * elem;
}

template <typename T, int P>
cudaError_t launch_P(const SlabShape& sh, int threads, size_t smem, int n3, const T* X1T,
                     const T* X2T, const T* Ta, const T* V, T* Sb, cudaStream_t s,
                     const int* skip) {
  fused_slab_kernel<T, P><<<n3, threads, smem, s>>>(sh, X1T, X2T, Ta, V, Sb, skip);
  return cudaGetLastError();
}

template <typename T, int P>
cudaError_t prepare_P() {
  return cudaFuncSetAttribute(fused_slab_kernel<T, P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              227 * 1024);
}

template <typename T>
cudaError_t prepare_T() {
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = prepare_P<T, 8>();
  if (e == cudaSuccess) e = prepare_P<T, 12>();
  if (e == cudaSuccess) e = prepare_P<T, 16>();
  if (e == cudaSuccess) e = prepare_P<T, 20>();
  if (e == cudaSuccess) e = prepare_P<T, 24>();
  if (e == cudaSuccess) e = prepare_P<T, 28>();
  if (e == cudaSuccess) e = prepare_P<T, 32>();
  return e;
}

}  // namespace

// Raise the dynamic shared-memory limit of every fused-slab instantiation on the current
// device (called once per plan, outside any stream capture).
cudaError_t fused_prepare() {
  cudaError_t e = prepare_T<float>();
  if (e == cudaSuccess) e = prepare_T<double>();
  return e;
}

int fused_slab_supported(int n1, int n2, int p1, int p2, int elem_bytes) {
  if (n1 <= 0 || n2 <= 0 || p1 <= 0 || p2 <= 0) return 0;
  if (n1 > 256) return 0;
  const int P = pick_P(p2);
  if (P == 0) return 0;
  SlabShape sh;
  int threads;
  slab_config(n1, n2, p1, p2, sh, threads);
  if (threads > 256) return 0;
  return slab_smem(sh, P, elem_bytes) <= 227 * 1024 ? 1 : 0;
}

template <typename T>
cudaError_t launch_fused_slab(int n1, int n2, int n3, int p1, int p2, const T* X1T, const T* X2T,
                              const T* Ta, const T* V, T* Sb, cudaStream_t s, const int* skip) {
  if (!fused_slab_supported(n1, n2, p1, p2, (int)sizeof(T))) return cudaErrorInvalidValue;
  if (n3 <= 0) return cudaSuccess;
  SlabShape sh;
  int threads;
  slab_config(n1, n2, p1, p2, sh, threads);
  sh.n3 = n3;
  const int P = pick_P(p2);
  const size_t smem = slab_smem(sh, P, (int)sizeof(T));
  switch (P) {
    case 8: return launch_P<T, 8>(sh, threads, smem, n3, X1T, X2T, Ta, V, Sb, s, skip);
    case 12: return launch_P<T, 12>(sh, threads, smem, n3, X1T, X2T, Ta, V, Sb, s, skip);
    case 16: return launch_P<T, 16>(sh, threads, smem, n3, X1T, X2T, Ta, V, Sb, s, skip);
    case 20: return launch_P<T, 20>(sh, threads, smem, n3, X1T, X2T, Ta, V, Sb, s, skip);
    case 24: return launch_P<T, 24>(sh, threads, smem, n3, X1T, X2T, Ta, V, Sb, s, skip);
    case 28: return launch_P<T, 28>(sh, threads, smem, n3, X1T, X2T, Ta, V, Sb, s, skip);
    case 32: return launch_P<T, 32>(sh, threads, smem, n3, X1T, X2T, Ta, V, Sb, s, skip);
    default: return cudaErrorInvalidValue;
  }
}

template cudaError_t launch_fused_slab<float>(int, int, int, int, int, const float*, const float*,
                                              const float*, const float*, float*, cudaStream_t,
                                              const int*);
template cudaError_t launch_fused_slab<double>(int, int, int, int, int, const double*,
                                               const double*, const double*, const double*,
                                               double*, cudaStream_t, const int*);

}  // namespace glam
