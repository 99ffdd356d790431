// The bottleneck of GD-PG (Sec. 6.2): X^T W X theta = G(V (.) H(Theta)) (Sec. 6.1, Eq.
// twentysixnew), with the last two stages of H and the first two stages of G fused per slab.
//
// Mode order: H contracts mode 3 first (T_a = rho over X_3, computed by the GEMM kernel), then
// mode 1 and mode 2 inside this kernel; G contracts mode 2, then mode 1 inside this kernel, and
// mode 3 last (GEMM kernel).  For one slab i3 (a contiguous n2 x n1 block of V):
//   T_b  (p2 x n1) = T_a[i3] (p2 x p1) . X_1^T        (per thread, registers)
//   eta  (n2 x n1) = X_2 (n2 x p2) . T_b              (registers only)
//   r            = V[i3] (.) eta
//   S    (p2 x n1) = X_2^T . r                        (registers, then shared memory)
//   S_b[i3] (p2 x p1) = S . X_1                       (shared memory -> global)
// eta and r never leave the SM: per inner iteration the kernel streams V once and touches only
// the small T_a / S_b slabs otherwise.
//
// Schedule: a persistent grid (one CTA per SM) walks the slabs i3 = blockIdx.x + k gridDim.x.
// With STAGE, the V slabs are double-buffered in shared memory by 1-D TMA bulk copies
// (cp.async.bulk with an mbarrier transaction count): slab k + 2 is in flight while slab k is
// computed.  Every mbarrier wait is bounded (about two seconds of %globaltimer); a wait that
// runs out sets *err and the CTA leaves the loop together.
//
// Thread mapping: lanes walk the unit-stride index i1 (conflict-free shared reads of V and
// X_1), warps split the columns into 32-wide tiles (CT of them) and the rows i2 into RG groups.
// Each lane forms its own column of T_b (P values) from T_a and X_1, then for each of its rows
// loads the X_2 row with 16-byte broadcast reads and uses it twice (for eta and for S).
#include <cstdint>

#include "glam_internal.cuh"
#include "glam_stage.cuh"
#include "glam_tma.cuh"

namespace glam {
namespace {

using namespace tma;

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

// Block size cap: 16 warps for FP32; 8 for FP64, whose register arrays take twice the space.
template <typename T>
constexpr int max_threads() {
  return sizeof(T) == 8 ? 256 : 512;
}

struct SlabShape {
  int n1, n2, n3, p1, p2, p3, CT, RG, LD;
  uint32_t vbytes;  // n2 * n1 * sizeof(T) (bulk copy size)
};

// Row pitch (elements) of the row-per-column arrays S[c][*] and X_1[c][*]: 16-byte rows whose
// pitch keeps the 8 lanes of one 128-bit shared-memory wavefront on distinct banks.
__host__ __device__ constexpr int row_pitch(int w) { return (w % 8 == 0) ? w + 4 : w; }

// Shared-memory layout of one CTA, in elements.  Every section starts on a 32-byte boundary
// (16-byte vector reads of X_2, T_a, S and X_1 rows and the bulk-copy destinations need 16).
struct SlabLayout {
  int64_t vbuf, x2, x1, x1c, ta, tb, sred, taall, x3r, total;
  int sp, q1, q1p;  // S row pitch, p1 rounded up to 4, X_1 row pitch
  int kcta;         // slabs per CTA (TAD)
};

__host__ __device__ inline int64_t align_up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline SlabLayout slab_layout(const SlabShape& sh, int P, int elem, bool stage,
                                                  bool tad = false, int kcta = 0) {
  const int64_t A = 32 / elem;
  SlabLayout L;
  L.sp = row_pitch(P);
  L.q1 = (sh.p1 + 3) / 4 * 4;
  L.q1p = row_pitch(L.q1);
  int64_t off = 0;
  L.vbuf = off;
  off = align_up(off + (stage ? 2 * (int64_t)sh.n2 * sh.n1 : 0), A);
  L.x2 = off;                                   // [n2][P]
  off = align_up(off + (int64_t)sh.n2 * P, A);
  L.x1 = off;                                   // [p1][LD]
  off = align_up(off + (int64_t)sh.p1 * sh.LD, A);
  L.x1c = off;                                  // [n1][q1p]
  off = align_up(off + (int64_t)sh.n1 * L.q1p, A);
  L.ta = off;                                   // [p1][P]
  off = align_up(off + (int64_t)sh.p1 * P, A);
  L.tb = off;                                   // [P][LD]
  off = align_up(off + (int64_t)P * sh.LD, A);
  L.sred = off;                                 // [RG][n1][sp]
  off = align_up(off + (int64_t)sh.RG * sh.n1 * L.sp, A);
  L.kcta = tad ? kcta : 0;
  L.taall = off;                                // [kcta][p2 p1]  (TAD)
  off = align_up(off + (tad ? (int64_t)kcta * sh.p2 * sh.p1 : 0), A);
  L.x3r = off;                                  // [kcta][p3]     (TAD)
  off += tad ? (int64_t)kcta * sh.p3 : 0;
  L.total = off;
  return L;
}

template <typename T>
__device__ __forceinline__ void load4(const T* src, T (&d)[4]) {
  using V = typename Vec16<T>::type;
  if constexpr (Vec16<T>::width == 4) {
    const V v = *reinterpret_cast<const V*>(src);
    d[0] = v.x; d[1] = v.y; d[2] = v.z; d[3] = v.w;
  } else {
    const V a = reinterpret_cast<const V*>(src)[0];
    const V b = reinterpret_cast<const V*>(src)[1];
    d[0] = a.x; d[1] = a.y; d[2] = b.x; d[3] = b.y;
  }
}

template <typename T>
__device__ __forceinline__ void store4(T* dst, T a, T b, T c, T d) {
  using V = typename Vec16<T>::type;
  if constexpr (Vec16<T>::width == 4) {
    *reinterpret_cast<V*>(dst) = V{a, b, c, d};
  } else {
    reinterpret_cast<V*>(dst)[0] = V{a, b};
    reinterpret_cast<V*>(dst)[1] = V{c, d};
  }
}

// TAD: instead of reading T_a (n3 x p2p1) from memory, the CTA forms it for its own slabs at
// the start, T_a(i3, :) = sum_j3 X_3(i3, j3) d(j3, :), from the correction d (p3 x p2p1, `Ta`
// then points at d) and X_3^T (p3 x n3): the first H stage folded into this kernel.
template <typename T, int P, bool STAGE, bool TAD>
__global__ void __launch_bounds__(max_threads<T>(), 1)
fused_slab_kernel(SlabShape sh, const T* __restrict__ X1T, const T* __restrict__ X2T,
                  const T* __restrict__ Ta, const T* __restrict__ V, T* __restrict__ Sb,
                  const int* __restrict__ skip, int* __restrict__ err, const T* __restrict__ X3T) {
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t mbar[2];
  __shared__ int timed_out;
  const int n1 = sh.n1, n2 = sh.n2, n3 = sh.n3, p1 = sh.p1, p2 = sh.p2, LD = sh.LD, RG = sh.RG;
  const int nv = n2 * n1;
  const int kcta = TAD ? (n3 - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x : 0;
  const SlabLayout L = slab_layout(sh, P, (int)sizeof(T), STAGE, TAD,
                                   TAD ? (n3 + (int)gridDim.x - 1) / (int)gridDim.x : 0);
  const int SP = L.sp, Q1 = L.q1, Q1P = L.q1p;
  T* const base = reinterpret_cast<T*>(smem_raw);
  T* Vbuf = base + L.vbuf;  // [2][n2 * n1]   (STAGE only)
  T* X2s = base + L.x2;     // [n2][P]    X2s[i2][j2] = X_2(i2, j2)
  T* X1s = base + L.x1;     // [p1][LD]   X1s[j1][i1] = X_1(i1, j1)
  T* X1c = base + L.x1c;    // [n1][Q1P]  X1c[i1][j1] = X_1(i1, j1)
  T* TaT = base + L.ta;     // [p1][P]    TaT[j1][j2] = T_a[i3](j2, j1)
  T* Tbs = base + L.tb;     // [P][LD]    Tbs[j2][i1] = T_b(j2, i1)
  T* Sred = base + L.sred;  // [RG][n1][SP] Sred[g][i1][j2] = partial S(j2, i1) of row group g
  const int tid = threadIdx.x, nth = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31;

  // the first two V slabs are requested before the prologue, so they arrive while it runs
  if (tid == 0) {
    timed_out = 0;
    if (STAGE) {
      mbar_init(&mbar[0], 1);
      mbar_init(&mbar[1], 1);
      fence_mbar_init();
      for (int b = 0; b < 2; ++b) {
        const int s0 = blockIdx.x + b * gridDim.x;
        if (s0 < n3) {
          mbar_expect_tx(&mbar[b], sh.vbytes);
          bulk_g2s(Vbuf + b * nv, V + (int64_t)s0 * nv, sh.vbytes, &mbar[b]);
        }
      }
    }
  }
  stage::load_each<8>(p2 * n2, X2T, [&](int idx, T x) {  // coalesced read of X_2^T rows
    const int j2 = idx / n2, i2 = idx - j2 * n2;
    X2s[i2 * P + j2] = x;
  });
  for (int idx = tid; idx < n2 * (P - p2); idx += nth) {
    const int i2 = idx / (P - p2), j2 = p2 + idx - i2 * (P - p2);
    X2s[i2 * P + j2] = T(0);
  }
  stage::load_each<8>(p1 * n1, X1T, [&](int idx, T x) {
    const int j1 = idx / n1, i1 = idx - j1 * n1;
    X1s[j1 * LD + i1] = x;
    X1c[i1 * Q1P + j1] = x;
  });
  for (int idx = tid; idx < n1 * (Q1 - p1); idx += nth) {
    const int i1 = idx / (Q1 - p1), j1 = p1 + idx - i1 * (Q1 - p1);
    X1c[i1 * Q1P + j1] = T(0);
  }
  T* TaAll = base + L.taall;  // [kcta][p2 p1]  T_a of this CTA's slabs (TAD)
  T* X3r = base + L.x3r;      // [kcta][p3]     their rows of X_3 (TAD)
  if (TAD) {
    const int p3 = sh.p3, P21 = p2 * p1;
    for (int idx = tid; idx < kcta * p3; idx += nth) {
      const int kk = idx / p3, j3 = idx - kk * p3;
      X3r[idx] = X3T[(int64_t)j3 * n3 + blockIdx.x + (int64_t)kk * gridDim.x];
    }
    __syncthreads();
    // T_a(s_k, n) = sum_j3 X_3(s_k, j3) d(j3, n): columns n over the threads, slabs in chunks of 4
    stage::form_ta<16>(kcta, p3, P21, Ta, X3r, TaAll);
    __syncthreads();
  }
  // T_a of the first slab
  if ((int)blockIdx.x < n3) {
    const T* ta = TAD ? TaAll : Ta + (int64_t)blockIdx.x * p2 * p1;
    for (int idx = tid; idx < p1 * P; idx += nth) {
      const int j1 = idx / P, j2 = idx - j1 * P;
      TaT[idx] = (j2 < p2) ? ta[j2 * p1 + j1] : T(0);
    }
  }
  __syncthreads();

  // warp roles in phase 2: column tile ct (32 columns i1), row group rg (rows i2 in [r0, r1))
  const int ct = warp % sh.CT, rg = warp / sh.CT;
  const int c = ct * 32 + lane;
  const bool valid = (c < n1) && (rg < RG);
  const int r0 = (int)(((int64_t)n2 * rg) / RG);
  const int r1 = (int)(((int64_t)n2 * (rg + 1)) / RG);
  // phase-3 roles: 4 x 4 output blocks (jb2, jb1), 16 lanes split the columns c
  const int NB1 = Q1 / 4, NB = (P / 4) * NB1;
  const int q = lane & 15;
  // T_a elements this thread prefetches for the next slab
  constexpr int kTaPer = (32 * P + 255) / 256;  // >= ceil(p1 * P / blockDim) for p1 <= 64, 256+ threads

  int k = 0;
  for (int slab = blockIdx.x; slab < n3; slab += gridDim.x, ++k) {
    const int b = k & 1;
    // ---- phase 1: T_b(j2, c) = sum_j1 T_a(j2, j1) X_1(c, j1); task = (column tile, 4 rows j2) ----
    {
      const int ntask = sh.CT * (P / 4);
      for (int task = warp; task < ntask; task += (nth >> 5)) {
        const int ct1 = task % sh.CT, jb = task / sh.CT;
        const int c1 = ct1 * 32 + lane;
        if (c1 < n1) {
          T a0 = T(0), a1 = T(0), a2 = T(0), a3 = T(0);
          for (int j1 = 0; j1 < p1; ++j1) {
            const T x1 = X1s[j1 * LD + c1];
            T t4[4];
            load4<T>(TaT + j1 * P + 4 * jb, t4);
            a0 = fma(t4[0], x1, a0);
            a1 = fma(t4[1], x1, a1);
            a2 = fma(t4[2], x1, a2);
            a3 = fma(t4[3], x1, a3);
          }
          Tbs[(4 * jb + 0) * LD + c1] = a0;
          Tbs[(4 * jb + 1) * LD + c1] = a1;
          Tbs[(4 * jb + 2) * LD + c1] = a2;
          Tbs[(4 * jb + 3) * LD + c1] = a3;
        }
      }
    }
    const T* Vs;
    if (STAGE) {
      bool ok = true;
      if (valid || tid == 0) ok = mbar_wait_bounded(&mbar[b], (uint32_t)((k >> 1) & 1));
      if (!ok) atomicOr(&timed_out, 1);
      Vs = Vbuf + b * nv;
    } else {
      Vs = V + (int64_t)slab * nv;
    }
    __syncthreads();  // (1) T_b complete; the previous slab's phase 3 is done with Sred
    if (STAGE && timed_out) break;

    // prefetch the next slab's T_a into registers (stored after phase 2)
    T ta_next[kTaPer];
    const int nxt_slab = slab + gridDim.x;
#pragma unroll
    for (int r = 0; r < kTaPer; ++r) {
      const int idx = tid + r * nth;
      ta_next[r] = T(0);
      if (nxt_slab < n3 && idx < p1 * P) {
        const int j1 = idx / P, j2 = idx - j1 * P;
        if (j2 < p2)
          ta_next[r] = TAD ? TaAll[(int64_t)(k + 1) * p2 * p1 + j2 * p1 + j1]
                           : Ta[(int64_t)nxt_slab * p2 * p1 + j2 * p1 + j1];
      }
    }

    // ---- phase 2: eta = X_2 T_b, r = V (.) eta, S = X_2^T r over this warp's rows ----
    if (valid) {
      T tb[P], sacc[P];
#pragma unroll
      for (int j = 0; j < P; ++j) {
        tb[j] = Tbs[j * LD + c];
        sacc[j] = T(0);
      }
      const T* vcol = Vs + c;
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
        const T rr = vcol[(int64_t)i2 * n1] * ((e0 + e1) + (e2 + e3));
#pragma unroll
        for (int j = 0; j < P; ++j) sacc[j] = fma(x2[j], rr, sacc[j]);
      }
      T* srow = Sred + ((int64_t)rg * n1 + c) * SP;
#pragma unroll
      for (int j = 0; j < P; j += 4) store4<T>(srow + j, sacc[j], sacc[j + 1], sacc[j + 2], sacc[j + 3]);
    }
#pragma unroll
    for (int r = 0; r < kTaPer; ++r) {
      const int idx = tid + r * nth;
      if (nxt_slab < n3 && idx < p1 * P) TaT[idx] = ta_next[r];
    }
    __syncthreads();  // (2) partial S complete; this V buffer and T_a are free
    if (STAGE && tid == 0) {
      const int nxt = slab + 2 * gridDim.x;
      if (nxt < n3) {
        fence_proxy_async();
        mbar_expect_tx(&mbar[b], sh.vbytes);
        bulk_g2s(Vbuf + b * nv, V + (int64_t)nxt * nv, sh.vbytes, &mbar[b]);
      }
    }
    if (RG > 1) {
      const int nq = n1 * (P / 4);
      for (int idx = tid; idx < nq; idx += nth) {
        const int cc = idx / (P / 4), j = 4 * (idx - cc * (P / 4));
        T a[4], t[4];
        load4<T>(Sred + (int64_t)cc * SP + j, a);
        for (int g = 1; g < RG; ++g) {
          load4<T>(Sred + ((int64_t)g * n1 + cc) * SP + j, t);
          a[0] += t[0]; a[1] += t[1]; a[2] += t[2]; a[3] += t[3];
        }
        store4<T>(Sred + (int64_t)cc * SP + j, a[0], a[1], a[2], a[3]);
      }
      __syncthreads();  // (3) S complete in Sred[0]
    }

    // ---- phase 3: S_b(j2, j1) = sum_c S(j2, c) X_1(c, j1), 4 x 4 blocks, 16 lanes over c ----
    T* out = Sb + (int64_t)slab * p2 * p1;
    const int nwarps = nth >> 5;
    for (int pair = warp; 2 * pair < NB; pair += nwarps) {
      const int blk = 2 * pair + (lane >> 4);
      const bool act = blk < NB;
      const int jb2 = act ? blk / NB1 : 0, jb1 = act ? blk - jb2 * NB1 : 0;
      T acc[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = T(0);
      if (act) {
        for (int cc = q; cc < n1; cc += 16) {
          T sv[4], xv[4];
          load4<T>(Sred + (int64_t)cc * SP + 4 * jb2, sv);
          load4<T>(X1c + (int64_t)cc * Q1P + 4 * jb1, xv);
#pragma unroll
          for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int v = 0; v < 4; ++v) acc[u][v] = fma(sv[u], xv[v], acc[u][v]);
        }
      }
#pragma unroll
      for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          T t = acc[u][v];
          t += __shfl_xor_sync(0xffffffffu, t, 1);
          t += __shfl_xor_sync(0xffffffffu, t, 2);
          t += __shfl_xor_sync(0xffffffffu, t, 4);
          t += __shfl_xor_sync(0xffffffffu, t, 8);
          acc[u][v] = t;
        }
      if (act && q == 0) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int j2 = 4 * jb2 + u;
          if (j2 >= p2) continue;
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const int j1 = 4 * jb1 + v;
            if (j1 < p1) out[j2 * p1 + j1] = acc[u][v];
          }
        }
      }
    }
  }
  if (STAGE && timed_out) {
    if (tid == 0) {
      atomicOr(err, 1);
      // give copies still in flight a bounded chance to land before the CTA leaves
      mbar_wait_bounded(&mbar[0], 0u);
      mbar_wait_bounded(&mbar[1], 0u);
    }
  }
}

constexpr int kPs[] = {8, 12, 16, 20, 24, 28, 32};

int pick_P(int p2) {
  for (int P : kPs)
    if (p2 <= P) return P;
  return 0;
}

size_t smem_bytes(const SlabShape& sh, int P, int elem, bool stage, bool tad = false, int kcta = 0) {
  return (size_t)slab_layout(sh, P, elem, stage, tad, kcta).total * elem;
}

// Dynamic shared-memory budget of one CTA: the device's opt-in limit minus room for the
// kernels' static shared variables (set by fused_prepare).
size_t g_smem_budget = 227 * 1024 - 256;

// Shape, block size and shared-memory plan; stage = false plans direct V loads.
bool configure(int n1, int n2, int p1, int p2, int elem, bool stage, SlabShape& sh, int& threads,
               size_t& smem, bool tad = false, int kcta = 0, int p3 = 1) {
  const int P = pick_P(p2);
  if (P == 0 || n1 <= 0 || n2 <= 0 || p1 <= 0 || n1 > 256 || p1 > 64) return false;
  if (elem == 8 && P > 24) return false;  // FP64 register arrays beyond this spill
  sh.n1 = n1;
  sh.n2 = n2;
  sh.n3 = 0;
  sh.p3 = p3;
  sh.p1 = p1;
  sh.p2 = p2;
  sh.CT = (n1 + 31) / 32;
  sh.LD = n1 + 1;
  const int max_warps = (elem == 8 ? 256 : 512) / 32;
  if (sh.CT > max_warps) return false;
  sh.RG = max_warps / sh.CT;
  if (sh.RG < 1) sh.RG = 1;
  if (sh.RG > n2) sh.RG = n2;
  sh.vbytes = (uint32_t)((size_t)n1 * n2 * elem);
  while (true) {
    smem = smem_bytes(sh, P, elem, stage, tad, kcta);
    if (smem <= g_smem_budget) break;
    if (sh.RG > 1) {
      sh.RG = sh.RG / 2;
      continue;
    }
    return false;
  }
  threads = 32 * sh.CT * sh.RG;
  // the next slab's T_a (p1 x P values) is prefetched with ceil(32 P / 256) values per thread
  if ((int64_t)threads * ((32 * P + 255) / 256) < (int64_t)p1 * P) return false;
  return threads <= (elem == 8 ? 256 : 512);
}

struct FusedArgs {
  const void* X1T;
  const void* X2T;
  const void* Ta;   // T_a (n3 x p2p1), or the correction d (p3 x p2p1) with TAD
  const void* V;
  void* Sb;
  const int* skip;
  int* err;
  const void* X3T;  // TAD only
};

template <typename T, int P, bool STAGE, bool TAD>
cudaError_t launch_P(const SlabShape& sh, int grid, int threads, size_t smem, const FusedArgs& a,
                     cudaStream_t s) {
  fused_slab_kernel<T, P, STAGE, TAD><<<grid, threads, smem, s>>>(
      sh, (const T*)a.X1T, (const T*)a.X2T, (const T*)a.Ta, (const T*)a.V, (T*)a.Sb, a.skip, a.err,
      (const T*)a.X3T);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T, bool STAGE, bool TAD>
cudaError_t launch_S(int P, const SlabShape& sh, int grid, int threads, size_t smem,
                     const FusedArgs& a, cudaStream_t s) {
  switch (P) {
    case 8: return launch_P<T, 8, STAGE, TAD>(sh, grid, threads, smem, a, s);
    case 12: return launch_P<T, 12, STAGE, TAD>(sh, grid, threads, smem, a, s);
    case 16: return launch_P<T, 16, STAGE, TAD>(sh, grid, threads, smem, a, s);
    case 20: return launch_P<T, 20, STAGE, TAD>(sh, grid, threads, smem, a, s);
    case 24: return launch_P<T, 24, STAGE, TAD>(sh, grid, threads, smem, a, s);
    case 28: return launch_P<T, 28, STAGE, TAD>(sh, grid, threads, smem, a, s);
    case 32: return launch_P<T, 32, STAGE, TAD>(sh, grid, threads, smem, a, s);
    default: return cudaErrorInvalidValue;
  }
}

template <typename T, int P, bool STAGE, bool TAD>
cudaError_t prepare_P() {
  return cudaFuncSetAttribute(fused_slab_kernel<T, P, STAGE, TAD>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_smem_budget);
}

template <typename T, bool STAGE, bool TAD>
cudaError_t prepare_TS() {
  cudaError_t e = prepare_P<T, 8, STAGE, TAD>();
  if (e == cudaSuccess) e = prepare_P<T, 12, STAGE, TAD>();
  if (e == cudaSuccess) e = prepare_P<T, 16, STAGE, TAD>();
  if (e == cudaSuccess) e = prepare_P<T, 20, STAGE, TAD>();
  if (e == cudaSuccess) e = prepare_P<T, 24, STAGE, TAD>();
  if (e == cudaSuccess) e = prepare_P<T, 28, STAGE, TAD>();
  if (e == cudaSuccess) e = prepare_P<T, 32, STAGE, TAD>();
  return e;
}

// Staging needs a 16-byte aligned slab start and a slab size that is a multiple of 16 bytes
// (the rules of cp.async.bulk), and is used for FP32 only: the FP64 path is bound by FP64 ALU
// throughput, not by the V stream.
bool can_stage(int n1, int n2, int elem, const void* V) {
  const size_t bytes = (size_t)n1 * n2 * elem;
  return elem == 4 && bytes % 16 == 0 && bytes < (1u << 20) &&
         (reinterpret_cast<uintptr_t>(V) % 16) == 0;
}

}  // namespace

// Raise the dynamic shared-memory limit of every fused-slab instantiation on the current
// device (called once per plan, outside any stream capture).
cudaError_t fused_prepare() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  g_smem_budget = optin > 1024 ? (size_t)optin - 1024 : 0;  // 1 KB kept for static variables
  e = prepare_TS<float, true, false>();
  if (e == cudaSuccess) e = prepare_TS<float, false, false>();
  if (e == cudaSuccess) e = prepare_TS<double, false, false>();
  if (e == cudaSuccess) e = prepare_TS<float, true, true>();
  if (e == cudaSuccess) e = prepare_TS<float, false, true>();
  if (e == cudaSuccess) e = prepare_TS<double, false, true>();
  return e;
}

int fused_slab_supported(int n1, int n2, int p1, int p2, int elem_bytes) {
  SlabShape sh;
  int threads;
  size_t smem;
  return configure(n1, n2, p1, p2, elem_bytes, false, sh, threads, smem) ? 1 : 0;
}

template <typename T>
cudaError_t launch_fused_slab(int n1, int n2, int n3, int p1, int p2, const T* X1T, const T* X2T,
                              const T* Ta, const T* V, T* Sb, cudaStream_t s, const int* skip,
                              int* err, const T* X3T, int p3) {
  if (n3 <= 0) return cudaSuccess;
  const bool tad = X3T != nullptr;
  SlabShape sh;
  int threads;
  size_t smem;
  bool stage = sizeof(T) == 4 && can_stage(n1, n2, (int)sizeof(T), V);
  const int grid_stage = n3 < num_sms() ? n3 : num_sms();
  const int grid_plain = n3 < 2 * num_sms() ? n3 : 2 * num_sms();
  const int kcta_stage = (n3 + grid_stage - 1) / grid_stage;
  const int kcta_plain = (n3 + grid_plain - 1) / grid_plain;
  if (stage && !configure(n1, n2, p1, p2, (int)sizeof(T), true, sh, threads, smem, tad, kcta_stage, p3))
    stage = false;
  if (!stage && !configure(n1, n2, p1, p2, (int)sizeof(T), false, sh, threads, smem, tad, kcta_plain, p3))
    return cudaErrorInvalidValue;
  sh.n3 = n3;
  const int grid = stage ? grid_stage : grid_plain;
  const int P = pick_P(p2);
  const FusedArgs a{X1T, X2T, Ta, V, Sb, skip, err, X3T};
  if constexpr (sizeof(T) == 4) {
    if (stage)
      return tad ? launch_S<T, true, true>(P, sh, grid, threads, smem, a, s)
                 : launch_S<T, true, false>(P, sh, grid, threads, smem, a, s);
  }
  return tad ? launch_S<T, false, true>(P, sh, grid, threads, smem, a, s)
             : launch_S<T, false, false>(P, sh, grid, threads, smem, a, s);
}

template cudaError_t launch_fused_slab<float>(int, int, int, int, int, const float*, const float*,
                                              const float*, const float*, float*, cudaStream_t,
                                              const int*, int*, const float*, int);
template cudaError_t launch_fused_slab<double>(int, int, int, int, int, const double*,
                                               const double*, const double*, const double*,
                                               double*, cudaStream_t, const int*, int*,
                                               const double*, int);

}  // namespace glam
