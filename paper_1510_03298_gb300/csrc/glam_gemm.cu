// Mode products of the rotated H-transform (App. A, rho) as one strided, batched, split-K
// SIMT GEMM.  A mode-j product of a (D3, D2, D1) C-order array is a GEMM whose contracted
// index is the j-th axis; keeping every axis in place (instead of rotating it to the end as
// rho does) makes the rotation pure index bookkeeping in the strides, so it costs no pass
// over memory.
//
//   mode 3: C (o x D2 D1)        = M (o x D3) . A (D3 x D2 D1)
//   mode 2: C[b] (o x D1)        = M (o x D2) . A[b] (D2 x D1),   b < D3
//   mode 1: C (D3 D2 x o)        = A (D3 D2 x D1) . M^T (D1 x o)
//
// Tiles of 64 x 64 outputs, 16-deep K slices staged in shared memory, 4 x 4 outputs per
// thread laid out with a 16-thread stride so that shared-memory reads are conflict-free and
// global stores are coalesced.  The operand loads pick the thread mapping that walks the
// unit-stride index, so every tensor operand is read with coalesced accesses.
#include <type_traits>

#include "glam_internal.cuh"

namespace glam {
namespace {


// TB is the storage type of the B operand.  With EXTRAP the operand is formed on load as
// B + omega (B - Bp) - Bs (Bp, Bs optional), in double when TB is double, then rounded to T:
// the FISTA extrapolation y = x + omega (x - x_prev) of Sec. 3.2, minus the anchor theta_k.
// Tiles of (16 TM) x (16 TN) outputs; 256 threads with TM x TN outputs each.
// BK is the K depth staged per step: 32 or 64 when the contraction fits in one step (all operand
// loads of the tile are then in flight together), else 16.
template <typename T, typename TB, bool EXTRAP, int TM, int TN, int BK>
__global__ void __launch_bounds__(256)
gemm_kernel(GemmDesc d, const T* __restrict__ A, const TB* __restrict__ B, T* __restrict__ C,
            const TB* __restrict__ Bp, const TB* __restrict__ Bs, const InnerCtl* __restrict__ ctl,
            double omega_h, const int* __restrict__ skip) {
  constexpr int BM = 16 * TM, BN = 16 * TN;
  if (skip != nullptr && *skip) return;
  __shared__ T As[BK][BM + 4];
  __shared__ T Bsm[BK][BN + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int bz = blockIdx.z;
  const int batch = bz / d.ksplit;
  const int split = bz - batch * d.ksplit;
  const int m0 = blockIdx.y * BM, n0 = blockIdx.x * BN;
  const int kper = (d.K + d.ksplit - 1) / d.ksplit;
  const int kbeg = split * kper;
  const int kend = min(d.K, kbeg + kper);
  A += batch * d.sAb;
  B += batch * d.sBb;
  C += batch * d.sCb + split * d.sCsplit;
  if (EXTRAP && Bp != nullptr) Bp += batch * d.sBb;
  if (EXTRAP && Bs != nullptr) Bs += batch * d.sBb;
  TB omega = TB(omega_h);
  if (EXTRAP && ctl != nullptr) {
    const int l = ctl->l;  // omega_l = (l - 1) / (l + 2), Sec. 3.2
    omega = TB(l - 1) / TB(l + 2);
  }
  T acc[TM][TN];
#pragma unroll
  for (int i = 0; i < TM; ++i)
#pragma unroll
    for (int j = 0; j < TN; ++j) acc[i][j] = T(0);

  const bool a_m_unit = (d.sAm == 1);
  const bool b_n_unit = (d.sBn == 1);
  for (int k0 = kbeg; k0 < kend; k0 += BK) {
#pragma unroll
    for (int r = 0; r < (BM * BK) / 256; ++r) {
      const int idx = tid + r * 256;
      int mm, ka;
      if (a_m_unit) {
        mm = idx % BM;
        ka = idx / BM;
      } else {
        ka = idx % BK;
        mm = idx / BK;
      }
      const int gm = m0 + mm, gk = k0 + ka;
      T v = T(0);
      if (gm < d.M && gk < kend) v = A[(int64_t)gm * d.sAm + (int64_t)gk * d.sAk];
      As[ka][mm] = v;
    }
#pragma unroll
    for (int r = 0; r < (BN * BK) / 256; ++r) {
      const int idx = tid + r * 256;
      int nn, kb;
      if (b_n_unit) {
        nn = idx % BN;
        kb = idx / BN;
      } else {
        kb = idx % BK;
        nn = idx / BK;
      }
      const int gn = n0 + nn, gkb = k0 + kb;
      T w = T(0);
      if (gn < d.N && gkb < kend) {
        const int64_t off = (int64_t)gkb * d.sBk + (int64_t)gn * d.sBn;
        TB v = B[off];
        if (EXTRAP) {
          if (Bp != nullptr) v = v + omega * (v - Bp[off]);  // y = x + omega (x - x_prev)
          if (Bs != nullptr) v = v - Bs[off];                // minus the anchor
        }
        w = T(v);
      }
      Bsm[kb][nn] = w;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < BK; ++kk) {
      T a[TM], b[TN];
#pragma unroll
      for (int i = 0; i < TM; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < TN; ++j) b[j] = Bsm[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < TM; ++i)
#pragma unroll
        for (int j = 0; j < TN; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < TM; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= d.M) continue;
#pragma unroll
    for (int j = 0; j < TN; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn < d.N) C[(int64_t)gm * d.sCm + (int64_t)gn * d.sCn] = acc[i][j];
    }
  }
}

template <typename T, typename TB, bool EXTRAP, int BK>
void launch_bk(const GemmDesc& d, dim3 grid, int tm, int tn, const T* A, const TB* B, T* C,
               cudaStream_t s, const TB* Bp, const TB* Bs, const InnerCtl* ctl, double omega,
               const int* skip) {
  if (tm == 4 && tn == 4)
    gemm_kernel<T, TB, EXTRAP, 4, 4, BK><<<grid, 256, 0, s>>>(d, A, B, C, Bp, Bs, ctl, omega, skip);
  else if (tm == 2 && tn == 4)
    gemm_kernel<T, TB, EXTRAP, 2, 4, BK><<<grid, 256, 0, s>>>(d, A, B, C, Bp, Bs, ctl, omega, skip);
  else if (tm == 4 && tn == 2)
    gemm_kernel<T, TB, EXTRAP, 4, 2, BK><<<grid, 256, 0, s>>>(d, A, B, C, Bp, Bs, ctl, omega, skip);
  else
    gemm_kernel<T, TB, EXTRAP, 2, 2, BK><<<grid, 256, 0, s>>>(d, A, B, C, Bp, Bs, ctl, omega, skip);
}

template <typename T, typename TB, bool EXTRAP>
cudaError_t launch_tiles(const GemmDesc& d, int tm, int tn, const T* A, const TB* B, T* C,
                         cudaStream_t s, const TB* Bp, const TB* Bs, const InnerCtl* ctl,
                         double omega, const int* skip) {
  dim3 grid((d.N + 16 * tn - 1) / (16 * tn), (d.M + 16 * tm - 1) / (16 * tm), d.batch * d.ksplit);
  if (grid.y > 65535) return cudaErrorInvalidValue;
  const int kper = (d.K + d.ksplit - 1) / d.ksplit;
  // one 64-deep step when the split's contraction fits in it (single-precision tiles only: the
  // FP64 tiles would need 2 x 64 x 68 x 8 = 70 KB of static shared memory at TM = TN = 4)
  if constexpr (sizeof(T) == 4) {
    // one staged step deep enough for the split's contraction, wasting at most half of it
    if (kper > 32 && kper <= 64) {
      launch_bk<T, TB, EXTRAP, 64>(d, grid, tm, tn, A, B, C, s, Bp, Bs, ctl, omega, skip);
      return cudaSuccess;
    }
    if (kper > 16 && kper <= 32) {
      launch_bk<T, TB, EXTRAP, 32>(d, grid, tm, tn, A, B, C, s, Bp, Bs, ctl, omega, skip);
      return cudaSuccess;
    }
  }
  launch_bk<T, TB, EXTRAP, 16>(d, grid, tm, tn, A, B, C, s, Bp, Bs, ctl, omega, skip);
  return cudaSuccess;
}

int64_t ctas(const GemmDesc& d, int tm, int tn) {
  return (int64_t)((d.N + 16 * tn - 1) / (16 * tn)) * ((d.M + 16 * tm - 1) / (16 * tm)) * d.batch * d.ksplit;
}

// Largest tile whose grid still fills the GPU (about 1.5 CTAs per SM), else the smallest.
void pick_tile(const GemmDesc& d, int& tm, int& tn) {
  const int64_t want = (3 * num_sms()) / 2;
  const int cand[4][2] = {{4, 4}, {2, 4}, {4, 2}, {2, 2}};
  for (auto& c : cand) {
    if (ctas(d, c[0], c[1]) >= want) {
      tm = c[0];
      tn = c[1];
      return;
    }
  }
  tm = 2;
  tn = 2;
}


}  // namespace

template <typename T, typename TB>
cudaError_t launch_gemm(const GemmDesc& d, const T* A, const TB* B, T* C, cudaStream_t s,
                        const TB* Bprev, const TB* Bsub, const InnerCtl* ctl, double omega,
                        const int* skip) {
  if (d.M <= 0 || d.N <= 0 || d.batch <= 0) return cudaSuccess;
  if (d.K <= 0 || d.ksplit < 1 || (int64_t)d.batch * d.ksplit > 65535) return cudaErrorInvalidValue;
  int tm = 4, tn = 4;
  pick_tile(d, tm, tn);
  cudaError_t e;
  if (Bprev != nullptr || Bsub != nullptr || ctl != nullptr || !std::is_same<T, TB>::value)
    e = launch_tiles<T, TB, true>(d, tm, tn, A, B, C, s, Bprev, Bsub, ctl, omega, skip);
  else
    e = launch_tiles<T, TB, false>(d, tm, tn, A, B, C, s, nullptr, nullptr, nullptr, 0.0, skip);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

#define GLAM_GEMM_INST(T, TB)                                                                  \
  template cudaError_t launch_gemm<T, TB>(const GemmDesc&, const T*, const TB*, T*, cudaStream_t, \
                                          const TB*, const TB*, const InnerCtl*, double, const int*);
GLAM_GEMM_INST(float, float)
GLAM_GEMM_INST(double, double)
GLAM_GEMM_INST(float, double)
#undef GLAM_GEMM_INST

}  // namespace glam
