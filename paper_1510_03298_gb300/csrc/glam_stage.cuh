// Cooperative loads of a CTA's small operands from global memory.  A grid-stride loop with one
// load per trip waits a full memory round trip per element; these helpers keep U loads in flight
// per thread, so a prologue of a few thousand elements costs one or two round trips.
#pragma once

#include <cstdint>

namespace glam {
namespace stage {

// store(i, src[i]) for every i in [0, total), U loads in flight per thread.
template <int U, typename T, typename F>
__device__ __forceinline__ void load_each(int total, const T* __restrict__ src, F&& store) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int base = 0; base < total; base += nth * U) {
    T v[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * nth + tid;
      v[u] = i < total ? src[i] : T(0);
    }
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int i = base + u * nth + tid;
      if (i < total) store(i, v[u]);
    }
  }
}

// The first H stage for the CTA's slabs: TaAll[k][n] = sum_j3 X3r[k][j3] D[j3][n] (App. A,
// mode 3 of Eq. eighteen), for k < kcta (the rows of X_3 of those slabs are X3r, kcta x p3, in
// shared memory) and n < P21.  Columns n over the threads, two columns per thread at a time,
// U rows of D in flight per column; every sum runs in j3 order.
template <int U, typename T>
__device__ __forceinline__ void form_ta(int kcta, int p3, int P21, const T* __restrict__ D,
                                        const T* X3r, T* TaAll) {
  const int tid = threadIdx.x, nth = blockDim.x;
  for (int nb = tid; nb < P21; nb += 2 * nth) {
    const int nc[2] = {nb, nb + nth};
    const bool on1 = nc[1] < P21;
    for (int k0 = 0; k0 < kcta; k0 += 4) {
      T acc[2][4];
#pragma unroll
      for (int c = 0; c < 2; ++c)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[c][r] = T(0);
      const T* xr = X3r + (int64_t)k0 * p3;
      for (int j0 = 0; j0 < p3; j0 += U) {
        T dv[2][U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const bool in = j0 + u < p3;
          dv[0][u] = in ? D[(int64_t)(j0 + u) * P21 + nc[0]] : T(0);
          dv[1][u] = (in && on1) ? D[(int64_t)(j0 + u) * P21 + nc[1]] : T(0);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) {
          const int j3 = j0 + u;
          if (j3 < p3) {
#pragma unroll
            for (int r = 0; r < 4; ++r) {
              if (k0 + r < kcta) {
                const T x = xr[(int64_t)r * p3 + j3];
                acc[0][r] = fma(x, dv[0][u], acc[0][r]);
                acc[1][r] = fma(x, dv[1][u], acc[1][r]);
              }
            }
          }
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        if (k0 + r < kcta) {
          TaAll[(int64_t)(k0 + r) * P21 + nc[0]] = acc[0][r];
          if (on1) TaAll[(int64_t)(k0 + r) * P21 + nc[1]] = acc[1][r];
        }
      }
    }
  }
}

}  // namespace stage
}  // namespace glam
