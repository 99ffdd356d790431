// Tensor-core (TF32) version of the fused bottleneck G(V (.) H(d)) of Sec. 6.2 (Eq.
// twentysixnew), used by GLAM_TF32 plans.
//
// Per slab i3 the four contractions run as warp-level TF32 MMAs (mma.sync m16n8k8, FP32
// accumulation):
//   MMA0  T_b^T (c x j2)  = X_1 (c x j1) . T_a^T (j1 x j2)           (mode 1 of the slab)
//   MMA1  eta^T (c x i2)  = T_b^T . X_2^T (j2 x i2)                   (mode 2)
//         r = V (.) eta                                               (IRLS weights)
//   MMA2  S (j2 x c)      = X_2^T (j2 x i2) . r (i2 x c)              (mode 2 adjoint)
//   MMA3  S_b (j2 x j1)   = S . X_1 (c x j1)                          (mode 1 adjoint)
// with c = i1.  MMA0 runs once per slab (one 16-row tile of c per warp, its X_1 operand held
// in registers for the whole launch) and leaves T_b^T in shared memory in the fragment order
// of MMA1's A operand.  Each warp then owns 16 NCT columns c and a range of 8-row blocks of
// i2; MMA1's accumulator becomes MMA2's B operand after the multiply by V, and MMA2's
// accumulator becomes MMA3's A operand, without leaving registers.  That reuse works because
// the next product contracts over the accumulator's column index: the accumulator holds
// columns (2t, 2t+1) of a lane where an operand wants K indices (t, t+4), so those K indices
// are permuted (k = t <-> 2t, k = t + 4 <-> 2t + 1) and the other operand of the product is
// read with the same permutation.  The per-warp S_b partials are summed in warp order (the
// same bits on every run).
//
// V slabs are double-buffered in shared memory with bounded mbarrier waits.  A slab arrives as
// n1/32 tiled TMA copies (a 3-D tensor map over V, one box of 32 columns x n2 rows per copy)
// with the 128-byte swizzle: in each 1 KB atom the 16-byte chunk k of row r lands at chunk
// k ^ (r mod 8), which spreads the fragment reads of V (four rows 2t, 2t+1 apart, one column)
// over all 32 banks.  T_a = X_3 d for the CTA's slabs is formed at kernel start (the first H
// stage).  Every other shared array has a pitch that keeps its fragment reads free of bank
// conflicts.
//
// Shapes: n1 % 32 == 0 (NCT = 4 when n1 % 64 == 0), n2 % 8 == 0, n2 <= 256, p1, p2 <= 32,
// n1 n2 4 < 2^20 bytes; other shapes use the FP32 SIMT kernel.
#include <cuda.h>
#include <cudaTypedefs.h>

#include <cstdint>
#include <mutex>

#include "glam_internal.cuh"
#include "glam_tma.cuh"

namespace glam {
namespace {

using namespace tma;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// D += A B for one 16 x 8 x 8 tile: A row-major 16 x 8, B column-major 8 x 8 (TF32), D FP32
__device__ __forceinline__ void mma_tf32(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2,
                                         uint32_t a3, uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// An MMA operand element as TF32 bits: the rounded value alone (SPLIT = 1), or the pair
// hi + lo of the 3xTF32 form (SPLIT = 3): hi = tf32(x), lo = tf32(x - hi), so hi + lo carries about
// 21 significant bits of x.
template <int SPLIT>
struct Tf {
  uint32_t h, l;
};
// from an FP32 value
template <int SPLIT>
__device__ __forceinline__ Tf<SPLIT> tf_of(float x) {
  Tf<SPLIT> r;
  r.h = to_tf32(x);
  r.l = SPLIT == 3 ? to_tf32(x - __uint_as_float(r.h)) : 0u;
  return r;
}
// from a value stored in shared memory: already TF32 when SPLIT = 1, FP32 when SPLIT = 3
template <int SPLIT>
__device__ __forceinline__ Tf<SPLIT> tf_stored(float x) {
  if constexpr (SPLIT == 1) {
    Tf<SPLIT> r;
    r.h = __float_as_uint(x);
    r.l = 0u;
    return r;
  } else {
    return tf_of<SPLIT>(x);
  }
}
// shared-memory form of a constant operand
template <int SPLIT>
__device__ __forceinline__ float tf_store(float x) {
  return SPLIT == 1 ? __uint_as_float(to_tf32(x)) : x;
}
// D += A B.  The 3xTF32 form adds hi hi' to D and the two cross terms hi lo' + lo hi' to a
// second accumulator X, which the caller adds to D when the sum is complete (two independent
// chains of MMAs instead of one three times as long); the lo lo' term, below 2^-22 of the
// product, is dropped.  X is untouched when SPLIT = 1.
template <int SPLIT>
__device__ __forceinline__ void mma_x(float (&d)[4], float (&x)[4], const Tf<SPLIT>& a0,
                                      const Tf<SPLIT>& a1, const Tf<SPLIT>& a2, const Tf<SPLIT>& a3,
                                      const Tf<SPLIT>& b0, const Tf<SPLIT>& b1) {
  if constexpr (SPLIT == 3) {
    mma_tf32(x, a0.h, a1.h, a2.h, a3.h, b0.l, b1.l);
    mma_tf32(x, a0.l, a1.l, a2.l, a3.l, b0.h, b1.h);
  }
  mma_tf32(d, a0.h, a1.h, a2.h, a3.h, b0.h, b1.h);
}
// D += X (the cross terms of the 3xTF32 form), once a sum is complete
template <int SPLIT>
__device__ __forceinline__ void fold_cross(float (&d)[4], const float (&x)[4]) {
  if constexpr (SPLIT == 3) {
#pragma unroll
    for (int e = 0; e < 4; ++e) d[e] += x[e];
  }
}

struct TcShape {
  int n1, n2, n3, p1, p2, p3;
  int CG, IG;  // column groups (16 NCT columns each) and row groups of the warps
  int kmax;    // slabs per CTA, at most
  int R;       // rows of d per staged chunk of the prologue
  int v4d;     // 1: V's tensor map is 4-D and a slab is one copy; 0: 3-D, one copy per strip
};

// pitch >= w with pitch = 8 (mod 16): 64-bit fragment reads whose half warp touches rows
// g = 0..3 at offsets 2t hit 16 distinct bank pairs
__host__ __device__ constexpr int pitch8(int w) { return w <= 8 ? 8 : ((w - 8 + 15) / 16) * 16 + 8; }
// pitch >= w with pitch = 4 (mod 8): 32-bit fragment reads of rows g = 0..7 at offsets t
__host__ __device__ constexpr int pitch4(int w) { return ((w + 3) / 8) * 8 + 4; }

struct TcLayout {
  int64_t vbuf, x2t, x2n, x1s, tas, tbf, pbuf, x3r, total;  // offsets in floats
  int64_t sd;     // prologue staging of a chunk of d, inside vbuf
  int64_t cst_n;  // floats of the constant block [x2t, x2n, x1s], copied whole from global memory
  int KP, NP, LDc, QT;   // pitches in floats
};

// The dynamic shared memory is used from its first 1 KB boundary on (the swizzle atoms of the
// V buffers are 1 KB aligned), so a launch asks for kTcAlignSlack bytes more than the layout.
constexpr int kTcAlignSlack = 1024;

__host__ __device__ inline int64_t al8(int64_t v) { return (v + 7) / 8 * 8; }
__host__ __device__ inline int64_t al4(int64_t v) { return (v + 3) / 4 * 4; }

template <int NB>
__host__ __device__ inline TcLayout tc_layout(const TcShape& sh, int nwarps) {
  constexpr int K8 = 8 * NB, MT = (K8 + 15) / 16;
  TcLayout L;
  L.KP = pitch8(K8);
  L.NP = pitch8(sh.n2);
  L.LDc = pitch8(sh.n1);
  L.QT = pitch4(K8);
  int64_t off = 0;
  // vbuf, tbf and pbuf come first: nothing else touches them during the prologue, which uses
  // their union [0, x2t) to stage its copies
  L.vbuf = off;                                   // [2][n1/32][n2][32] V slabs, swizzled
  off = al8(off + 2 * (int64_t)sh.n2 * sh.n1);
  L.tbf = off;                                    // [n1/16][NB][32][4]  T_b^T fragments
  off = al8(off + (int64_t)(sh.n1 / 16) * NB * 128);
  L.pbuf = off;                                   // [nwarps][p2 p1] partial S_b
  off = al8(off + (int64_t)nwarps * sh.p2 * sh.p1);
  L.x2t = off;                                    // [n2][KP]        X_2(i2, j2)
  off = al8(off + (int64_t)sh.n2 * L.KP);
  L.x2n = off;                                    // [16 MT][NP]     X_2(i2, j2) by rows j2
  off = al8(off + 16 * MT * (int64_t)L.NP);
  L.x1s = off;                                    // [K8][LDc]       X_1(c, j1) by rows j1
  off = al8(off + (int64_t)K8 * L.LDc);
  L.tas = off;                                    // [kmax][K8][QT]  T_a(j2, j1) of the CTA's slabs
  off = al8(off + (int64_t)sh.kmax * K8 * L.QT);
  L.x3r = off;                                    // [p3][KQ]        X_3(slab_k, j3) at [j3][k]
  off += (int64_t)sh.p3 * ((sh.kmax + 3) / 4 * 4);
  L.total = off;
  L.sd = L.vbuf;
  L.cst_n = L.tas - L.x2t;  // a multiple of 8 floats
  return L;
}

// One V slab into buffer b (called by one thread): the byte count of the slab is posted, then
// the copies.  With the 4-D map (dims: 32 columns, n2 rows, n1/32 strips, n3 slabs) one box
// {32, n2, n1/32, 1} lands as [strip][row][32]; with the 3-D map (32-column boxes of the
// (n3, n2, n1) array) one copy per strip, box {32, n2, 1} at {32 s, 0, slab}.
__device__ __forceinline__ void issue_slab(float* vbuf_b, const CUtensorMap* tmap, int v4d, int slab,
                                           int n1, int n2, uint64_t* bar) {
  fence_proxy_async();
  mbar_expect_tx(bar, (uint32_t)n1 * (uint32_t)n2 * 4u);
  if (v4d) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(smem_u32(vbuf_b)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(0), "r"(0), "r"(0), "r"(slab), "r"(smem_u32(bar))
        : "memory");
    return;
  }
  for (int s = 0; s < n1 / 32; ++s) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(vbuf_b + (int64_t)s * n2 * 32)),
        "l"(reinterpret_cast<uint64_t>(tmap)), "r"(32 * s), "r"(0), "r"(slab), "r"(smem_u32(bar))
        : "memory");
  }
}

// block size limit of a tiling: the 3xTF32 form keeps hi and lo of the register operands, so it
// runs with at most 256 threads (255 registers each)
template <int NCT, int SPLIT>
constexpr int tc_max_threads() {
  return SPLIT == 3 ? 256 : (NCT == 4 ? 256 : (NCT == 2 ? 384 : 512));
}

template <int NB, int NCT, int SPLIT>
__global__ void __launch_bounds__(tc_max_threads<NCT, SPLIT>(), 1)
fused_slab_tc_kernel(TcShape sh, const float* __restrict__ Cst, const float* __restrict__ D,
                     const __grid_constant__ CUtensorMap tmapV,
                     float* __restrict__ Sb, const int* __restrict__ skip, int* __restrict__ err,
                     const float* __restrict__ X3T) {
  constexpr int K8 = 8 * NB, MT = (K8 + 15) / 16;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t mbar[3];  // V buffers 0 and 1, prologue copies
  __shared__ int timed_out;
  const int n1 = sh.n1, n2 = sh.n2, n3 = sh.n3, p1 = sh.p1, p2 = sh.p2, p3 = sh.p3;
  const int nv = n2 * n1, P21 = p2 * p1;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int warp = tid >> 5, lane = tid & 31, nwarps = nth >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int kcta = (n3 - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  const TcLayout L = tc_layout<NB>(sh, nwarps);
  float* const base = reinterpret_cast<float*>(
      smem_raw + ((kTcAlignSlack - (smem_u32(smem_raw) & (kTcAlignSlack - 1))) & (kTcAlignSlack - 1)));
  float* Vbuf = base + L.vbuf;
  float* X2t = base + L.x2t;
  float* X2n = base + L.x2n;
  float* X1s = base + L.x1s;
  float* TaS = base + L.tas;
  float4* TbF = reinterpret_cast<float4*>(base + L.tbf);
  float* Pbuf = base + L.pbuf;
  float* X3r = base + L.x3r;
  float* sD = base + L.sd;
  const int KP = L.KP, NP = L.NP, LDc = L.LDc, QT = L.QT;
  const int R = sh.R, nchunk = (p3 + R - 1) / R;

  // ---- prologue: the constant operands (X_2 and X_1 in their shared-memory layouts, prepared
  // once per fit by tc_const_kernel) and the first rows of d arrive by bulk copies (one memory
  // round trip), the X_3 entries of the CTA's slabs by one gather ----
  if (tid == 0) {
    // the descriptor of V's tensor map is fetched now, not at the first V request
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmapV)) : "memory");
    timed_out = 0;
    mbar_init(&mbar[0], 1);
    mbar_init(&mbar[1], 1);
    mbar_init(&mbar[2], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto chunk_rows = [&](int c) { return (c + 1) * R < p3 ? R : p3 - c * R; };
  // a chunk of d moves as its 16-byte multiple; the last < 4 floats (odd p2 p1) by plain loads
  auto chunk_bulk = [&](int c) { return (uint32_t)(((int64_t)chunk_rows(c) * P21) / 4 * 16); };
  if (tid == 0) {
    const uint32_t bc = (uint32_t)L.cst_n * 4u;
    mbar_expect_tx(&mbar[2], bc + chunk_bulk(0));
    bulk_g2s(X2t, Cst, bc, &mbar[2]);
    if (chunk_bulk(0) > 0) bulk_g2s(sD, D, chunk_bulk(0), &mbar[2]);
  }
  const int KQ = (sh.kmax + 3) / 4 * 4;  // slabs of X3r rounded up to float4 groups
  for (int idx = tid; idx < p3 * KQ; idx += nth) {  // X_3 entries of this CTA's slabs, [j3][k]
    const int j3 = idx / KQ, kk = idx - j3 * KQ;
    X3r[idx] = kk < kcta ? X3T[(int64_t)j3 * n3 + blockIdx.x + (int64_t)kk * gridDim.x] : 0.f;
  }
  for (int idx = tid; idx < sh.kmax * K8 * QT; idx += nth) TaS[idx] = 0.f;
  bool ok0 = mbar_wait_bounded(&mbar[2], 0u);
  if (!ok0) atomicOr(&timed_out, 1);
  __syncthreads();
  // MMA0's A operand X_1(c, j1) for this warp's 16-row tile of c, kept in registers (X1s holds
  // zeros in the rows j1 >= p1)
  const bool mma0_warp = warp < n1 / 16;
  Tf<SPLIT> xa[NB][4];
#pragma unroll
  for (int s = 0; s < NB; ++s) {
    const int c = 16 * warp + g, j0 = 8 * s + t, j4 = j0 + 4;
    xa[s][0] = tf_stored<SPLIT>(mma0_warp ? X1s[j0 * LDc + c] : 0.f);
    xa[s][1] = tf_stored<SPLIT>(mma0_warp ? X1s[j0 * LDc + c + 8] : 0.f);
    xa[s][2] = tf_stored<SPLIT>(mma0_warp ? X1s[j4 * LDc + c] : 0.f);
    xa[s][3] = tf_stored<SPLIT>(mma0_warp ? X1s[j4 * LDc + c + 8] : 0.f);
  }
  // ---- first H stage for this CTA's slabs: T_a(s_k, :) = sum_j3 X_3(s_k, j3) d(j3, :), summed
  // in j3 order into TaS (FP32), chunk by chunk of staged rows of d ----
  // (timed_out is read only right after a barrier that follows every write to it, so all threads
  // of the CTA take the same branch)
  for (int c = 0; c < nchunk; ++c) {
    const int j0 = c * R, rows = chunk_rows(c);
    if (c > 0) {
      __syncthreads();  // every thread is done with the previous chunk
      if (tid == 0) {
        fence_proxy_async();
        mbar_expect_tx(&mbar[2], chunk_bulk(c));
        if (chunk_bulk(c) > 0) bulk_g2s(sD, D + (int64_t)j0 * P21, chunk_bulk(c), &mbar[2]);
      }
      bool okc = mbar_wait_bounded(&mbar[2], (uint32_t)(c & 1));
      if (!okc) atomicOr(&timed_out, 1);
    }
    for (int i = (int)(chunk_bulk(c) / 4) + tid; i < rows * P21; i += nth) sD[i] = D[(int64_t)j0 * P21 + i];
    __syncthreads();  // the chunk (and its tail) is in place
    if (timed_out) break;
    // task = (2 consecutive columns n, 4 slabs k): one float2 of d and one float4 of X_3 per row
    const int nq = (P21 + 1) / 2, nkg = (kcta + 3) / 4;
    const bool vec = (P21 % 2) == 0;
    for (int task = tid; task < nq * nkg; task += nth) {
      const int q = task % nq, k0 = 4 * (task / nq), n0 = 2 * q;
      int eo[2];  // TaS offsets of the two columns (within a slab)
      bool in[2];
#pragma unroll
      for (int cc = 0; cc < 2; ++cc) {
        const int n = n0 + cc, j2 = n / p1;
        in[cc] = n < P21;
        eo[cc] = j2 * QT + (n - j2 * p1);
      }
      float a[4][2];
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc)
          a[r][cc] = (c > 0 && k0 + r < kcta && in[cc]) ? TaS[(k0 + r) * K8 * QT + eo[cc]] : 0.f;
#pragma unroll 4
      for (int j = 0; j < rows; ++j) {
        float dv[2];
        if (vec) {
          const float2 d2 = *reinterpret_cast<const float2*>(sD + j * P21 + n0);
          dv[0] = d2.x;
          dv[1] = d2.y;
        } else {
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) dv[cc] = in[cc] ? sD[j * P21 + n0 + cc] : 0.f;
        }
        const float4 x4 = *reinterpret_cast<const float4*>(X3r + (j0 + j) * KQ + k0);
        const float xv[4] = {x4.x, x4.y, x4.z, x4.w};
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int cc = 0; cc < 2; ++cc) a[r][cc] = fmaf(xv[r], dv[cc], a[r][cc]);
      }
      const bool last = c == nchunk - 1;  // the last chunk stores T_a in its operand form
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int cc = 0; cc < 2; ++cc)
          if (k0 + r < kcta && in[cc]) TaS[(k0 + r) * K8 * QT + eo[cc]] = last ? tf_store<SPLIT>(a[r][cc]) : a[r][cc];
    }
  }
  __syncthreads();  // every chunk is summed: T_a is in place and the V buffers are free
  if (tid == 0 && !timed_out) {
    fence_proxy_async();
    for (int b = 0; b < 2; ++b) {
      const int s0 = blockIdx.x + b * gridDim.x;
      if (s0 < n3) issue_slab(Vbuf + (int64_t)b * nv, &tmapV, sh.v4d, s0, n1, n2, &mbar[b]);
    }
  }

  // warp roles in the slab: columns c0w .. c0w + 16 NCT - 1, row blocks [ib0, ib1) of i2
  const int cg = warp % sh.CG, ig = warp / sh.CG;
  const int c0w = 16 * NCT * cg;
  const int NI = n2 / 8;
  const int ib0 = (NI * ig) / sh.IG, ib1 = (NI * (ig + 1)) / sh.IG;
  const int nact = sh.CG * sh.IG;  // warps of the main phase; any others only run MMA0
  const bool main_warp = warp < nact;
  // swizzled V offsets of this lane: the element (row r, column 16 (cti & 1) + g + 8 h) of a
  // 32-column strip (cti = c0w / 16 + ct) sits at r * 32 + (((g / 4 + 4 (cti & 1) + 2 h) ^ (r mod 8))
  // * 4 + g mod 4), and the rows read are r = i0 + 2t + rr with i0 a multiple of 8.  With NCT even
  // cti & 1 = ct & 1; with NCT = 1 the warp's one tile may be the second half of a strip (kb).
  const int kb = (NCT == 1) ? 2 * ((c0w >> 4) & 1) : 0;
  int vofs[4][2];
#pragma unroll
  for (int kq = 0; kq < 4; ++kq)
#pragma unroll
    for (int rr = 0; rr < 2; ++rr)
      vofs[kq][rr] = ((((g >> 2) + 2 * ((kq + kb) & 3)) ^ (2 * t + rr)) << 2) | (g & 3);

  // MMA0: the 16 x K8 tile of T_b^T of this warp for slab k, stored as MMA1 A fragments
  auto mma0 = [&](int kk) {
    if (!mma0_warp) return;
    const float* TaK = TaS + kk * K8 * QT;
#pragma unroll
    for (int nb = 0; nb < NB; ++nb) {
      float acc[4] = {0.f, 0.f, 0.f, 0.f}, accx[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
      for (int s = 0; s < NB; ++s) {
        const float* tb = TaK + (8 * nb + g) * QT + 8 * s + t;
        mma_x<SPLIT>(acc, accx, xa[s][0], xa[s][1], xa[s][2], xa[s][3], tf_stored<SPLIT>(tb[0]),
                     tf_stored<SPLIT>(tb[4]));
      }
      fold_cross<SPLIT>(acc, accx);
      // C (c, j2 = 8 nb + {2t, 2t+1}) -> A (c, K slot t <-> 2t, slot t + 4 <-> 2t + 1)
      TbF[(warp * NB + nb) * 32 + lane] = make_float4(tf_store<SPLIT>(acc[0]), tf_store<SPLIT>(acc[2]),
                                                      tf_store<SPLIT>(acc[1]), tf_store<SPLIT>(acc[3]));
    }
  };
  if (!timed_out) mma0(0);

  int k = 0;
  for (int slab = blockIdx.x; slab < n3; slab += gridDim.x, ++k) {
    const int b = k & 1;
    const bool ok = mbar_wait_bounded(&mbar[b], (uint32_t)((k >> 1) & 1));
    if (!ok) atomicOr(&timed_out, 1);
    // (S2) T_b^T fragments of slab k complete, its V slab landed, the reduction of slab k - 1
    // is done with Pbuf
    __syncthreads();
    if (timed_out) break;
    const float* Vs = Vbuf + (int64_t)b * nv;
    if (main_warp) {
    Tf<SPLIT> a1f[NCT][NB][4];
#pragma unroll
    for (int ct = 0; ct < NCT; ++ct)
#pragma unroll
      for (int nb = 0; nb < NB; ++nb) {
        const float4 f = TbF[((c0w / 16 + ct) * NB + nb) * 32 + lane];
        a1f[ct][nb][0] = tf_stored<SPLIT>(f.x);
        a1f[ct][nb][1] = tf_stored<SPLIT>(f.y);
        a1f[ct][nb][2] = tf_stored<SPLIT>(f.z);
        a1f[ct][nb][3] = tf_stored<SPLIT>(f.w);
      }
    float c2[MT][NCT][2][4];  // S(j2, c): [j2 tile][column tile][column half][fragment]
    float c2x[SPLIT == 3 ? MT : 1][NCT][2][4];  // its 3xTF32 cross terms
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int ct = 0; ct < NCT; ++ct)
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            c2[mt][ct][h][e] = 0.f;
            if (SPLIT == 3) c2x[SPLIT == 3 ? mt : 0][ct][h][e] = 0.f;
          }

#pragma unroll (NCT == 1 ? 2 : 1)
    for (int ib = ib0; ib < ib1; ++ib) {
      const int i0 = 8 * ib;
      // ---- MMA1: eta^T(c, i0 .. i0 + 7); B = X_2(i2, j2) with the permuted K = j2 ----
      float c1[NCT][4], c1x[NCT][4];
#pragma unroll
      for (int ct = 0; ct < NCT; ++ct)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          c1[ct][e] = 0.f;
          c1x[ct][e] = 0.f;
        }
#pragma unroll
      for (int ks = 0; ks < NB; ++ks) {
        const float2 bv = *reinterpret_cast<const float2*>(X2t + (i0 + g) * KP + 8 * ks + 2 * t);
        const Tf<SPLIT> b0 = tf_stored<SPLIT>(bv.x), b1 = tf_stored<SPLIT>(bv.y);
#pragma unroll
        for (int ct = 0; ct < NCT; ++ct)
          mma_x<SPLIT>(c1[ct], c1x[ct], a1f[ct][ks][0], a1f[ct][ks][1], a1f[ct][ks][2], a1f[ct][ks][3],
                       b0, b1);
      }
#pragma unroll
      for (int ct = 0; ct < NCT; ++ct) fold_cross<SPLIT>(c1[ct], c1x[ct]);
      // ---- r = V (.) eta as MMA2 B fragments (K = i2 permuted, N = c) ----
      Tf<SPLIT> b2f[NCT][2][2];
      const float* vrow = Vs + (int64_t)(c0w >> 5) * n2 * 32 + (i0 + 2 * t) * 32;
#pragma unroll
      for (int ct = 0; ct < NCT; ++ct) {
        const float* vs = vrow + (int64_t)(ct >> 1) * n2 * 32;
        const int kq = 2 * (ct & 1);
        b2f[ct][0][0] = tf_of<SPLIT>(vs[vofs[kq][0]] * c1[ct][0]);           // (c,     i0 + 2t)
        b2f[ct][0][1] = tf_of<SPLIT>(vs[32 + vofs[kq][1]] * c1[ct][1]);      // (c,     i0 + 2t + 1)
        b2f[ct][1][0] = tf_of<SPLIT>(vs[vofs[kq + 1][0]] * c1[ct][2]);       // (c + 8, i0 + 2t)
        b2f[ct][1][1] = tf_of<SPLIT>(vs[32 + vofs[kq + 1][1]] * c1[ct][3]);  // (c + 8, i0 + 2t + 1)
      }
      // ---- MMA2: S(j2, c) += X_2^T(j2, i2) r(i2, c) ----
#pragma unroll
      for (int mt = 0; mt < MT; ++mt) {
        const float2 lo = *reinterpret_cast<const float2*>(X2n + (16 * mt + g) * NP + i0 + 2 * t);
        const float2 hi = *reinterpret_cast<const float2*>(X2n + (16 * mt + g + 8) * NP + i0 + 2 * t);
        const Tf<SPLIT> a0 = tf_stored<SPLIT>(lo.x), a2 = tf_stored<SPLIT>(lo.y);
        const Tf<SPLIT> a1 = tf_stored<SPLIT>(hi.x), a3 = tf_stored<SPLIT>(hi.y);
#pragma unroll
        for (int ct = 0; ct < NCT; ++ct)
#pragma unroll
          for (int h = 0; h < 2; ++h)
            mma_x<SPLIT>(c2[mt][ct][h], c2x[SPLIT == 3 ? mt : 0][ct][h], a0, a1, a2, a3, b2f[ct][h][0],
                         b2f[ct][h][1]);
      }
    }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int ct = 0; ct < NCT; ++ct)
#pragma unroll
        for (int h = 0; h < 2; ++h) fold_cross<SPLIT>(c2[mt][ct][h], c2x[SPLIT == 3 ? mt : 0][ct][h]);
    // ---- MMA3: S_b(j2, j1) += S(j2, c) X_1(c, j1); A from S with the permuted K = c ----
    float c3[MT][NB][4], c3x[MT][NB][4];
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nj = 0; nj < NB; ++nj)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          c3[mt][nj][e] = 0.f;
          c3x[mt][nj][e] = 0.f;
        }
#pragma unroll
    for (int ct = 0; ct < NCT; ++ct)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int cb = c0w + 16 * ct + 8 * h + 2 * t;
        Tf<SPLIT> bx[NB][2];
#pragma unroll
        for (int nj = 0; nj < NB; ++nj) {
          const float2 bv = *reinterpret_cast<const float2*>(X1s + (8 * nj + g) * LDc + cb);
          bx[nj][0] = tf_stored<SPLIT>(bv.x);
          bx[nj][1] = tf_stored<SPLIT>(bv.y);
        }
#pragma unroll
        for (int mt = 0; mt < MT; ++mt) {
          const Tf<SPLIT> a0 = tf_of<SPLIT>(c2[mt][ct][h][0]), a1 = tf_of<SPLIT>(c2[mt][ct][h][2]);
          const Tf<SPLIT> a2 = tf_of<SPLIT>(c2[mt][ct][h][1]), a3 = tf_of<SPLIT>(c2[mt][ct][h][3]);
#pragma unroll
          for (int nj = 0; nj < NB; ++nj)
            mma_x<SPLIT>(c3[mt][nj], c3x[mt][nj], a0, a1, a2, a3, bx[nj][0], bx[nj][1]);
        }
      }
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nj = 0; nj < NB; ++nj) fold_cross<SPLIT>(c3[mt][nj], c3x[mt][nj]);
    // this warp's partial S_b (rows j2 < p2, columns j1 < p1)
    float* pw = Pbuf + (int64_t)warp * P21;
#pragma unroll
    for (int mt = 0; mt < MT; ++mt)
#pragma unroll
      for (int nj = 0; nj < NB; ++nj)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int j2 = 16 * mt + g + (e >= 2 ? 8 : 0);
          const int j1 = 8 * nj + 2 * t + (e & 1);
          if (j2 < p2 && j1 < p1) pw[j2 * p1 + j1] = c3[mt][nj][e];
        }
    }  // main_warp
    __syncthreads();  // (S3) partials complete; every thread is done with this V buffer and TbF
    if (tid == 0) {
      const int nxt = slab + 2 * gridDim.x;
      if (nxt < n3) issue_slab(Vbuf + (int64_t)b * nv, &tmapV, sh.v4d, nxt, n1, n2, &mbar[b]);
    }
    if (k + 1 < kcta) mma0(k + 1);  // overlaps the reduction below
    // sum of the partials in warp order
    float* out = Sb + (int64_t)slab * P21;
    for (int o = tid; o < P21; o += nth) {
      float acc = 0.f;
      for (int w = 0; w < nact; ++w) acc += Pbuf[(int64_t)w * P21 + o];
      out[o] = acc;
    }
  }
  if (timed_out && tid == 0) {
    atomicOr(err, 1);
    // give copies still in flight a bounded chance to land before the CTA leaves
    mbar_wait_bounded(&mbar[0], 0u);
    mbar_wait_bounded(&mbar[1], 0u);
    mbar_wait_bounded(&mbar[2], (uint32_t)((nchunk - 1) & 1));
  }
}

// Positions of the constant block [x2t, x2n, x1s] of the kernel's shared-memory layout.
struct CstLayout {
  int n1, n2, p1, p2, KP, NP, LDc, K8, M16;
  int64_t o2n, o1s, total;
};

// The constant block in global memory, element for element as the kernel keeps it in shared
// memory: X_2(i2, j2) at [i2][KP], X_2 by rows j2 at [16 MT][NP], X_1 by rows j1 at [K8][LDc],
// zeros in every padding entry; TF32-rounded for the TF32 form, FP32 for the 3xTF32 form.
__global__ void tc_const_kernel(CstLayout c, const float* __restrict__ X1T,
                                const float* __restrict__ X2T, float* __restrict__ out, int split) {
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < c.total;
       e += (int64_t)gridDim.x * blockDim.x) {
    float v = 0.f;
    if (e < (int64_t)c.n2 * c.KP) {
      const int i2 = (int)(e / c.KP), j2 = (int)(e % c.KP);
      if (j2 < c.p2) v = X2T[(int64_t)j2 * c.n2 + i2];
    } else if (e >= c.o2n && e < c.o2n + (int64_t)c.M16 * c.NP) {
      const int64_t f = e - c.o2n;
      const int j2 = (int)(f / c.NP), i2 = (int)(f % c.NP);
      if (j2 < c.p2 && i2 < c.n2) v = X2T[(int64_t)j2 * c.n2 + i2];
    } else if (e >= c.o1s && e < c.o1s + (int64_t)c.K8 * c.LDc) {
      const int64_t f = e - c.o1s;
      const int j1 = (int)(f / c.LDc), i1 = (int)(f % c.LDc);
      if (j1 < c.p1 && i1 < c.n1) v = X1T[(int64_t)j1 * c.n1 + i1];
    }
    out[e] = split == 1 ? __uint_as_float(to_tf32(v)) : v;
  }
}

template <int NB>
CstLayout cst_layout_nb(int n1, int n2, int p1, int p2) {
  TcShape sh{};
  sh.n1 = n1;
  sh.n2 = n2;
  sh.p1 = p1;
  sh.p2 = p2;
  const TcLayout L = tc_layout<NB>(sh, 1);  // the constant block does not depend on the warps
  CstLayout c;
  c.n1 = n1;
  c.n2 = n2;
  c.p1 = p1;
  c.p2 = p2;
  c.KP = L.KP;
  c.NP = L.NP;
  c.LDc = L.LDc;
  c.K8 = 8 * NB;
  c.M16 = 16 * ((8 * NB + 15) / 16);
  c.o2n = L.x2n - L.x2t;
  c.o1s = L.x1s - L.x2t;
  c.total = L.cst_n;
  return c;
}

bool cst_layout(int n1, int n2, int p1, int p2, CstLayout& c) {
  switch (((p1 > p2 ? p1 : p2) + 7) / 8) {
    case 1: c = cst_layout_nb<1>(n1, n2, p1, p2); return true;
    case 2: c = cst_layout_nb<2>(n1, n2, p1, p2); return true;
    case 3: c = cst_layout_nb<3>(n1, n2, p1, p2); return true;
    case 4: c = cst_layout_nb<4>(n1, n2, p1, p2); return true;
    default: return false;
  }
}

size_t g_tc_budget = 227 * 1024 - 1024;

size_t tc_smem_bytes(int NB, const TcShape& sh, int nwarps) {
  switch (NB) {
    case 1: return (size_t)tc_layout<1>(sh, nwarps).total * 4;
    case 2: return (size_t)tc_layout<2>(sh, nwarps).total * 4;
    case 3: return (size_t)tc_layout<3>(sh, nwarps).total * 4;
    case 4: return (size_t)tc_layout<4>(sh, nwarps).total * 4;
    default: return (size_t)-1;
  }
}

// Shape, block size and shared-memory plan of the tensor-core kernel for the warp tiling
// (NCT column tiles of 16 per warp, IG row groups; IG = 0 takes as many as the block allows);
// false when the shape is outside the kernel's domain.
bool tc_configure_with(int n1, int n2, int n3, int p1, int p2, int p3, int grid, int NCT, int IGreq,
                       int split, TcShape& sh, int& threads, size_t& smem, int& NB) {
  if (split != 1 && split != 3) return false;
  if (n1 < 32 || n2 < 8 || n3 < 1 || p1 < 1 || p2 < 1 || p3 < 1 || n1 % 32 != 0 || n2 % 8 != 0 ||
      n2 > 256 || p1 > 32 || p2 > 32 || grid < 1 || !(NCT == 1 || NCT == 2 || NCT == 4) ||
      n1 % (16 * NCT) != 0)
    return false;
  if ((int64_t)n1 * n2 * 4 >= (1 << 20)) return false;  // one slab's bytes in an mbarrier tx count
  NB = ((p1 > p2 ? p1 : p2) + 7) / 8;
  sh.n1 = n1;
  sh.n2 = n2;
  sh.n3 = n3;
  sh.p1 = p1;
  sh.p2 = p2;
  sh.p3 = p3;
  sh.CG = n1 / (16 * NCT);
  const int max_warps = (split == 3 ? 256 : (NCT == 4 ? 256 : (NCT == 2 ? 384 : 512))) / 32;
  if (sh.CG > max_warps) return false;
  sh.IG = IGreq > 0 ? IGreq : max_warps / sh.CG;
  if (sh.IG > n2 / 8) sh.IG = n2 / 8;
  if (sh.IG < 1) return false;
  // MMA0 takes one 16-row tile of c per warp: small n2 adds warps that only run MMA0
  const int nwarps = sh.CG * sh.IG > n1 / 16 ? sh.CG * sh.IG : n1 / 16;
  if (nwarps > max_warps) return false;
  sh.kmax = (n3 + grid - 1) / grid;
  threads = 32 * nwarps;
  {  // rows of d per prologue chunk: what fits in the staging area after X_1^T and X_2^T
    const int64_t P21 = (int64_t)p1 * p2;
    const int64_t sd = 0;  // d is staged from the start of the V buffers
    const int64_t stage_end = al8(al8(2LL * n1 * n2) + (int64_t)(n1 / 16) * NB * 128) +
                              (int64_t)nwarps * P21;  // the start of x2t
    const int64_t avail = stage_end - sd;
    int64_t R = avail > 0 ? avail / P21 : 0;
    if (R >= p3) R = p3;
    else if (P21 % 4 != 0) R = R / 4 * 4;  // chunk starts stay 16-byte aligned
    if (R < 1) return false;
    sh.R = (int)R;
  }
  sh.v4d = 0;
  smem = tc_smem_bytes(NB, sh, nwarps) + kTcAlignSlack;
  return smem <= g_tc_budget;
}

// The tiling the kernel runs with: 64 or 32 columns per warp for TF32; 32 for 3xTF32, whose
// register operands are twice as large.
bool tc_configure(int n1, int n2, int n3, int p1, int p2, int p3, int grid, int split, TcShape& sh,
                  int& threads, size_t& smem, int& NB, int& NCT) {
  NCT = split == 3 ? 2 : ((n1 % 64 == 0) ? 4 : 2);
  return tc_configure_with(n1, n2, n3, p1, p2, p3, grid, NCT, 0, split, sh, threads, smem, NB);
}

template <int NB, int NCT, int SPLIT>
cudaError_t tc_launch(const TcShape& sh, int grid, int threads, size_t smem, const float* Cst,
                      const float* D, const CUtensorMap& tmapV, float* Sb, cudaStream_t s,
                      const int* skip, int* err, const float* X3T) {
  fused_slab_tc_kernel<NB, NCT, SPLIT><<<grid, threads, smem, s>>>(sh, Cst, D, tmapV, Sb, skip, err, X3T);
  count_launches(1);
  return cudaGetLastError();
}

// cuTensorMapEncodeTiled of the driver, looked up once through the runtime (no link to libcuda)
PFN_cuTensorMapEncodeTiled_v12000 encode_tiled() {
  static std::once_flag once;
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  std::call_once(once, [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

// V's tensor map with the 128-byte swizzle: 4-D (32 columns, n2 rows, n1/32 strips, n3 slabs;
// strides n1 * 4, 128 and n1 n2 * 4 bytes) so that one box {32, n2, n1/32, 1} moves a slab; if
// the driver does not take that map, the 3-D map of the (n3, n2, n1) array with boxes
// {32, n2, 1}.  Returns 4, 3, or 0 when neither map can be made.
int encode_v_map(CUtensorMap* m, const float* V, int n1, int n2, int n3) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (fn == nullptr) return 0;
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  {
    const cuuint64_t dims[4] = {32, (cuuint64_t)n2, (cuuint64_t)(n1 / 32), (cuuint64_t)n3};
    const cuuint64_t strides[3] = {(cuuint64_t)n1 * 4, 128, (cuuint64_t)n1 * n2 * 4};
    const cuuint32_t box[4] = {32, (cuuint32_t)n2, (cuuint32_t)(n1 / 32), 1};
    if (fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, const_cast<float*>(V), dims, strides, box, estr,
           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS)
      return 4;
  }
  const cuuint64_t dims[3] = {(cuuint64_t)n1, (cuuint64_t)n2, (cuuint64_t)n3};
  const cuuint64_t strides[2] = {(cuuint64_t)n1 * 4, (cuuint64_t)n1 * n2 * 4};
  const cuuint32_t box[3] = {32, (cuuint32_t)n2, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<float*>(V), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS
             ? 3
             : 0;
}

template <int NB, int NCT, int SPLIT>
cudaError_t tc_prepare_one() {
  return cudaFuncSetAttribute(fused_slab_tc_kernel<NB, NCT, SPLIT>,
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_tc_budget);
}

}  // namespace

// Raise the dynamic shared-memory limit of every tensor-core instantiation on the current
// device (called once per plan, outside any stream capture).
cudaError_t fused_tc_prepare() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  g_tc_budget = optin > 1024 ? (size_t)optin - 1024 : 0;  // 1 KB kept for static variables
  if (e == cudaSuccess) e = tc_prepare_one<1, 1, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<2, 1, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<3, 1, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<4, 1, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<1, 2, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<2, 2, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<3, 2, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<4, 2, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<1, 4, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<2, 4, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<3, 4, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<4, 4, 1>();
  if (e == cudaSuccess) e = tc_prepare_one<1, 2, 3>();
  if (e == cudaSuccess) e = tc_prepare_one<2, 2, 3>();
  if (e == cudaSuccess) e = tc_prepare_one<3, 2, 3>();
  if (e == cudaSuccess) e = tc_prepare_one<4, 2, 3>();
  return e;
}

int fused_tc_supported(int n1, int n2, int n3, int p1, int p2, int p3, int split) {
  TcShape sh;
  int threads, NB, NCT;
  size_t smem;
  const int grid = n3 < num_sms() ? n3 : num_sms();
  return tc_configure(n1, n2, n3, p1, p2, p3, grid, split, sh, threads, smem, NB, NCT) ? 1 : 0;
}

int encode_map_2d(CUtensorMap* m, const float* base, uint64_t dim0, uint64_t dim1, uint64_t stride1,
                  uint32_t box0, uint32_t box1) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_tiled();
  if (fn == nullptr) return 0;
  const cuuint64_t dims[2] = {dim0, dim1};
  const cuuint64_t strides[1] = {stride1};
  const cuuint32_t box[2] = {box0, box1};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS
             ? 1
             : 0;
}

int fused_tc_pointers_ok(const float* Cst, const float* D, const float* V) {
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) % 16) == 0; };
  return al16(Cst) && al16(D) && al16(V) ? 1 : 0;
}

int64_t fused_tc_const_floats(int n1, int n2, int p1, int p2) {
  CstLayout c;
  return cst_layout(n1, n2, p1, p2, c) ? c.total : 0;
}

cudaError_t launch_fused_tc_const(int n1, int n2, int p1, int p2, const float* X1T, const float* X2T,
                                  float* Cst, int split, cudaStream_t s) {
  CstLayout c;
  if (!cst_layout(n1, n2, p1, p2, c)) return cudaErrorInvalidValue;
  int blocks = (int)((c.total + 255) / 256);
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
  tc_const_kernel<<<blocks, 256, 0, s>>>(c, X1T, X2T, Cst, split);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fused_slab_tc(int n1, int n2, int n3, int p1, int p2, int p3, const float* Cst,
                                 const float* D, const float* V, float* Sb,
                                 cudaStream_t s, const int* skip, int* err, const float* X3T,
                                 int split) {
  if (n3 <= 0) return cudaSuccess;
  if (!fused_tc_pointers_ok(Cst, D, V)) return cudaErrorInvalidValue;
  const int grid = n3 < num_sms() ? n3 : num_sms();
  TcShape sh;
  int threads, NB, NCT;
  size_t smem;
  if (!tc_configure(n1, n2, n3, p1, p2, p3, grid, split, sh, threads, smem, NB, NCT))
    return cudaErrorInvalidValue;
  alignas(64) CUtensorMap tmapV;
  const int rank = encode_v_map(&tmapV, V, n1, n2, n3);
  if (rank == 0) return cudaErrorInvalidValue;
  sh.v4d = rank == 4 ? 1 : 0;
  const int key = (split * 8 + NB) * 8 + NCT;
  switch (key) {
    case (1 * 8 + 1) * 8 + 1:
      return tc_launch<1, 1, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 2) * 8 + 1:
      return tc_launch<2, 1, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 3) * 8 + 1:
      return tc_launch<3, 1, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 4) * 8 + 1:
      return tc_launch<4, 1, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 1) * 8 + 2:
      return tc_launch<1, 2, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 2) * 8 + 2:
      return tc_launch<2, 2, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 3) * 8 + 2:
      return tc_launch<3, 2, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 4) * 8 + 2:
      return tc_launch<4, 2, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 1) * 8 + 4:
      return tc_launch<1, 4, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 2) * 8 + 4:
      return tc_launch<2, 4, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 3) * 8 + 4:
      return tc_launch<3, 4, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (1 * 8 + 4) * 8 + 4:
      return tc_launch<4, 4, 1>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (3 * 8 + 1) * 8 + 2:
      return tc_launch<1, 2, 3>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (3 * 8 + 2) * 8 + 2:
      return tc_launch<2, 2, 3>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (3 * 8 + 3) * 8 + 2:
      return tc_launch<3, 2, 3>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    case (3 * 8 + 4) * 8 + 2:
      return tc_launch<4, 2, 3>(sh, grid, threads, smem, Cst, D, tmapV, Sb, s, skip, err, X3T);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace glam
