// Linear predictor eta = H(<X_j>, Theta) (Sec. 6.1, Eq. eighteen; rho of App. A) for FP32 plans.
//
// H contracts mode 3 first (T_a = X_3 Theta, n3 x p2p1 outputs, mode3_rows_kernel), then modes 1
// and 2 per slab i3 in predict_tile_kernel:
//   T_b[i3] (p2 x n1) = T_a[i3] (p2 x p1) . X_1^T (p1 x n1)          (mode 1)
//   eta[i3] (n2 x n1) = X_2 (n2 x p2) . T_b[i3] (p2 x n1)            (mode 2)
// T_b never leaves shared memory, so the only n-sized traffic is the eta write (4n bytes): the
// kernel is bound by that store stream and by the FP32 FMAs of the mode-2 product
// (2 n p2 FLOPs).  Work items are 128 x 128 tiles (rows i2, columns i1) of a slab; each of the
// 256 threads owns 8 rows x 8 columns (two groups of 4 adjacent columns 64 apart), so the mode-2
// operands come from shared memory as float4 loads (X_2 rows broadcast within a warp, T_b rows
// conflict-free) and each warp stores two full 256-byte row segments per instruction.
// Persistent grid of two CTAs per SM; the X_1 / X_2 tiles stay in shared memory while
// consecutive work items of a CTA share the same (i2, i1) block.
#include <algorithm>

#include "glam_internal.cuh"
#include "glam_tma.cuh"

namespace glam {
namespace {

constexpr int kTile = 128;  // tile side: rows i2 and columns i1
constexpr int kPMax = 32;   // p1, p2 at most this (shared-memory operand tiles)

// Shared-memory layout of predict_tile_kernel<MODE>: X_1^T, X_2^T and T_b blocks of LD = kTile
// columns, T_a, then (MODE 1) the staged eta tile (kTile x kTile, dense, so that a tile whose rows
// are contiguous in eta leaves in one bulk copy), every part 16-byte aligned.
struct PredLayout {
  int64_t x1s, x2s, tbs, tas, es, total;  // floats
};
__host__ __device__ inline PredLayout pred_layout(int p1, int p2, int mode) {
  PredLayout L;
  int64_t off = 0;
  L.x1s = off;
  off += (int64_t)p1 * kTile;
  L.x2s = off;
  off += (int64_t)p2 * kTile;
  L.tbs = off;
  off += (int64_t)p2 * kTile;
  L.tas = off;  // two buffers: the current work item's T_a and the next one's, in flight
  off += 2 * (((int64_t)p1 * p2 + 3) / 4 * 4);
  L.es = off;
  if (mode >= 1) off += (int64_t)kTile * kTile;
  L.total = off;
  return L;
}

// Mode-3 product T_a (n3 x P21) = X_3 (n3 x p3) . Theta (p3 x P21), the first stage of H.  A CTA
// owns 16 rows i3 and 128 columns m: every thread issues all of its loads of the X_3 and Theta
// blocks before the first use (one memory round trip), then computes 2 rows x 4 columns.
constexpr int kM3Rows = 16, kM3Cols = 128, kM3KMax = 64;

__global__ void __launch_bounds__(256)
mode3_rows_kernel(int n3, int p3, int P21, const float* __restrict__ XT3,
                  const float* __restrict__ Theta, float* __restrict__ Ta) {
  __shared__ float Th[kM3KMax][kM3Cols];
  __shared__ float X3s[kM3KMax][kM3Rows];
  // the tile kernel that consumes T_a may be launched now (it waits for this grid's results
  // before reading them)
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
  const int tid = threadIdx.x;
  const int r0 = blockIdx.y * kM3Rows, m0 = blockIdx.x * kM3Cols;
  constexpr int kThLoads = kM3KMax * kM3Cols / 256, kXLoads = kM3KMax * kM3Rows / 256;
  float tv[kThLoads], xv[kXLoads];
#pragma unroll
  for (int q = 0; q < kThLoads; ++q) {
    const int idx = tid + q * 256, k = idx / kM3Cols, c = idx - k * kM3Cols;
    tv[q] = (k < p3 && m0 + c < P21) ? Theta[(int64_t)k * P21 + m0 + c] : 0.f;
  }
#pragma unroll
  for (int q = 0; q < kXLoads; ++q) {
    const int idx = tid + q * 256, k = idx / kM3Rows, r = idx - k * kM3Rows;
    xv[q] = (k < p3 && r0 + r < n3) ? XT3[(int64_t)k * n3 + r0 + r] : 0.f;
  }
#pragma unroll
  for (int q = 0; q < kThLoads; ++q) {
    const int idx = tid + q * 256;
    Th[idx / kM3Cols][idx % kM3Cols] = tv[q];
  }
#pragma unroll
  for (int q = 0; q < kXLoads; ++q) {
    const int idx = tid + q * 256;
    X3s[idx / kM3Rows][idx % kM3Rows] = xv[q];
  }
  __syncthreads();
  const int cq = tid & 31, rp = tid >> 5;  // 4 columns 4cq.., rows 2rp, 2rp + 1
  float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll 8
  for (int k = 0; k < p3; ++k) {
    const float4 t = *reinterpret_cast<const float4*>(&Th[k][4 * cq]);
    const float x0 = X3s[k][2 * rp], x1 = X3s[k][2 * rp + 1];
    a0[0] = fmaf(x0, t.x, a0[0]); a0[1] = fmaf(x0, t.y, a0[1]);
    a0[2] = fmaf(x0, t.z, a0[2]); a0[3] = fmaf(x0, t.w, a0[3]);
    a1[0] = fmaf(x1, t.x, a1[0]); a1[1] = fmaf(x1, t.y, a1[1]);
    a1[2] = fmaf(x1, t.z, a1[2]); a1[3] = fmaf(x1, t.w, a1[3]);
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int m = m0 + 4 * cq + j;
    if (m >= P21) break;
    if (r0 + 2 * rp < n3) Ta[(int64_t)(r0 + 2 * rp) * P21 + m] = a0[j];
    if (r0 + 2 * rp + 1 < n3) Ta[(int64_t)(r0 + 2 * rp + 1) * P21 + m] = a1[j];
  }
}

// MODE 0: every thread stores its outputs directly.  MODE 1: eta tiles staged in shared memory
// and written by bulk copies (n1 % 4 == 0, eta 16-byte aligned), so the stores of one tile
// proceed while the next one is computed.
template <int MODE>
__global__ void __launch_bounds__(256, 2)
predict_tile_kernel(int n1, int n2, int n3, int p1, int p2, const float* __restrict__ XT1,
                    const float* __restrict__ XT2, const float* __restrict__ Ta,
                    float* __restrict__ eta) {
  constexpr bool BULK = MODE >= 1;
  extern __shared__ float4 smem_f4[];
  const PredLayout L = pred_layout(p1, p2, MODE);
  constexpr int LD = kTile;
  float* sm = reinterpret_cast<float*>(smem_f4);
  float* X1s = sm + L.x1s;  // [p1][LD]   X_1^T columns of the block
  float* X2s = sm + L.x2s;  // [p2][LD]   X_2^T columns of the block
  float* Tbs = sm + L.tbs;  // [p2][LD]   T_b of the tile
  float* Tas0 = sm + L.tas;  // [2][p2][p1] T_a of the slab (double-buffered)
  float* Es = sm + L.es;    // [kTile][kTile] eta tile (BULK)
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int nb1 = (n1 + kTile - 1) / kTile, nb2 = (n2 + kTile - 1) / kTile;
  const int64_t ntiles = (int64_t)n3 * nb1 * nb2;
  const int P21 = p1 * p2;
  const int TaStride = (P21 + 3) / 4 * 4;
  // T_a of work item t into buffer b by asynchronous 4-byte copies (completed by cp.async.wait_all)
  auto fetch_ta = [&](int64_t t, int b) {
    if (t >= ntiles) return;
    const float* src = Ta + (t % n3) * (int64_t)P21;
    float* dst = Tas0 + b * TaStride;
    for (int idx = tid; idx < P21; idx += 256)
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(tma::smem_u32(dst + idx)),
                   "l"(src + idx)
                   : "memory");
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  // every load of the two operand blocks of block blk is issued before the first store, so a
  // block costs one memory round trip
  auto load_blocks = [&](int blk) {
    const int r0 = (blk / nb1) * kTile, c0 = (blk - (blk / nb1) * nb1) * kTile;
    constexpr int kBlkRegs = kPMax * kTile / 256;
    float v1[kBlkRegs], v2[kBlkRegs];
#pragma unroll
    for (int q = 0; q < kBlkRegs; ++q) {
      const int idx = tid + q * 256, k = idx / kTile, c = idx - k * kTile;
      v1[q] = (k < p1 && c0 + c < n1) ? XT1[(int64_t)k * n1 + c0 + c] : 0.f;
      v2[q] = (k < p2 && r0 + c < n2) ? XT2[(int64_t)k * n2 + r0 + c] : 0.f;
    }
#pragma unroll
    for (int q = 0; q < kBlkRegs; ++q) {
      const int idx = tid + q * 256, k = idx / kTile, c = idx - k * kTile;
      if (k < p1) X1s[k * LD + c] = v1[q];
      if (k < p2) X2s[k * LD + c] = v2[q];
    }
  };
  int cur_blk = -1;
  if ((int64_t)blockIdx.x < ntiles) {
    cur_blk = (int)((int64_t)blockIdx.x / n3);
    load_blocks(cur_blk);
  }
  // T_a is written by the mode-3 kernel launched just before: with a programmatic launch this
  // kernel starts early, loads its operand blocks, and waits here for that grid's results
  asm volatile("griddepcontrol.wait;" ::: "memory");
  fetch_ta(blockIdx.x, 0);
  int buf = 0;
  for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, buf ^= 1) {
    const int blk = (int)(t / n3);
    const int i3 = (int)(t - (int64_t)blk * n3);
    const int b2 = blk / nb1, b1 = blk - b2 * nb1;
    const int r0 = b2 * kTile, c0 = b1 * kTile;
    __syncthreads();  // every reader of the previous work item's shared arrays is done
    if (blk != cur_blk) {
      load_blocks(blk);
      cur_blk = blk;
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();  // T_a of this work item is in buffer buf; the other buffer is free
    fetch_ta(t + gridDim.x, buf ^ 1);
    const float* Tas = Tas0 + buf * TaStride;

    // mode 1: T_b[k2][c] = sum_k1 T_a[k2][k1] X_1[c][k1]; a thread owns rows k2 = 2kp, 2kp + 1
    // and the columns 4cx.. and 64 + 4cx.. (float4 operand loads, conflict-free)
    {
      const int kp = tid >> 4, cx = tid & 15;
      if (2 * kp < p2) {
        const bool two = 2 * kp + 1 < p2;
        const float* ta0 = Tas + 2 * kp * p1;
        const float* ta1 = two ? ta0 + p1 : ta0;
        float s0[8], s1[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) s0[j] = s1[j] = 0.f;
#pragma unroll 4
        for (int k1 = 0; k1 < p1; ++k1) {
          const float4 u0 = *reinterpret_cast<const float4*>(X1s + k1 * LD + 4 * cx);
          const float4 u1 = *reinterpret_cast<const float4*>(X1s + k1 * LD + 64 + 4 * cx);
          const float x[8] = {u0.x, u0.y, u0.z, u0.w, u1.x, u1.y, u1.z, u1.w};
          const float w0 = ta0[k1], w1 = ta1[k1];
#pragma unroll
          for (int j = 0; j < 8; ++j) {
            s0[j] = fmaf(w0, x[j], s0[j]);
            s1[j] = fmaf(w1, x[j], s1[j]);
          }
        }
        float* tb0 = Tbs + 2 * kp * LD;
        *reinterpret_cast<float4*>(tb0 + 4 * cx) = make_float4(s0[0], s0[1], s0[2], s0[3]);
        *reinterpret_cast<float4*>(tb0 + 64 + 4 * cx) = make_float4(s0[4], s0[5], s0[6], s0[7]);
        if (two) {
          float* tb1 = tb0 + LD;
          *reinterpret_cast<float4*>(tb1 + 4 * cx) = make_float4(s1[0], s1[1], s1[2], s1[3]);
          *reinterpret_cast<float4*>(tb1 + 64 + 4 * cx) = make_float4(s1[4], s1[5], s1[6], s1[7]);
        }
      }
    }
    __syncthreads();

    float* out = eta + (int64_t)i3 * n2 * n1;
    // mode 2: eta[r][c] = sum_k2 X_2[r][k2] T_b[k2][c] for the thread's 8 x 8 outputs
    float acc[8][8];
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) acc[i][j] = 0.f;
#pragma unroll 4
    for (int k = 0; k < p2; ++k) {
      const float4 a0 = *reinterpret_cast<const float4*>(X2s + k * LD + ty * 8);
      const float4 a1 = *reinterpret_cast<const float4*>(X2s + k * LD + ty * 8 + 4);
      const float4 v0 = *reinterpret_cast<const float4*>(Tbs + k * LD + tx * 4);
      const float4 v1 = *reinterpret_cast<const float4*>(Tbs + k * LD + 64 + tx * 4);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      const float b[8] = {v0.x, v0.y, v0.z, v0.w, v1.x, v1.y, v1.z, v1.w};
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    if (BULK) {
      if (tid < 32) tma::bulk_wait_read_all();  // the previous tile's copies have read Es
      __syncthreads();
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        float* er = Es + (ty * 8 + i) * kTile + tx * 4;
        *reinterpret_cast<float4*>(er) = make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]);
        *reinterpret_cast<float4*>(er + 64) = make_float4(acc[i][4], acc[i][5], acc[i][6], acc[i][7]);
      }
    } else {
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int r = r0 + ty * 8 + i;
        if (r >= n2) break;
        float* row = out + (int64_t)r * n1;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int cc = c0 + h * 64 + tx * 4;
#pragma unroll
          for (int j = 0; j < 4; ++j)
            if (cc + j < n1) row[cc + j] = acc[i][4 * h + j];
        }
      }
    }
    if (BULK) {
      tma::fence_proxy_async();
      __syncthreads();
      if (tid < 32) {
        const int rows = min(kTile, n2 - r0), cols = min(kTile, n1 - c0);
        if (cols == kTile && n1 == kTile) {
          // the tile's rows are contiguous in eta and in Es: one copy
          if (tid == 0) tma::bulk_s2g(out + (int64_t)r0 * n1, Es, (uint32_t)(rows * kTile * 4));
        } else {
          for (int r = tid; r < rows; r += 32)
            tma::bulk_s2g(out + (int64_t)(r0 + r) * n1 + c0, Es + r * kTile, (uint32_t)(cols * 4));
        }
        tma::bulk_commit();
      }
    }
  }
  // bulk copies must finish before the CTA (and its shared memory) is released
  if (BULK && tid < 32) tma::bulk_wait_all();
}

}  // namespace

int predict_tiles_supported(int p1, int p2) {
  return p1 >= 1 && p2 >= 1 && p1 <= kPMax && p2 <= kPMax;
}

int mode3_rows_supported(int p3) { return p3 >= 1 && p3 <= kM3KMax; }

cudaError_t launch_mode3_rows(int n3, int p3, int P21, const float* XT3, const float* Theta,
                              float* Ta, cudaStream_t s) {
  if (!mode3_rows_supported(p3)) return cudaErrorInvalidValue;
  if (n3 <= 0 || P21 <= 0) return cudaSuccess;
  const dim3 grid((P21 + kM3Cols - 1) / kM3Cols, (n3 + kM3Rows - 1) / kM3Rows);
  mode3_rows_kernel<<<grid, 256, 0, s>>>(n3, p3, P21, XT3, Theta, Ta);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_predict_tiles(int n1, int n2, int n3, int p1, int p2, const float* XT1,
                                 const float* XT2, const float* Ta, float* eta, cudaStream_t s) {
  if (!predict_tiles_supported(p1, p2)) return cudaErrorInvalidValue;
  const int64_t ntiles = (int64_t)n3 * ((n1 + kTile - 1) / kTile) * ((n2 + kTile - 1) / kTile);
  if (ntiles <= 0) return cudaSuccess;
  const bool bulk = (n1 % 4 == 0) && ((reinterpret_cast<uintptr_t>(eta) & 15) == 0);
  const int mode = bulk ? 1 : 0;
  const size_t smem = sizeof(float) * (size_t)pred_layout(p1, p2, mode).total;
  auto kern = mode == 1 ? predict_tile_kernel<1> : predict_tile_kernel<0>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  const int grid = (int)std::min<int64_t>(ntiles, (int64_t)per_sm * num_sms());
  // programmatic dependent launch: the kernel may start while the mode-3 kernel before it on the
  // stream finishes; it waits (griddepcontrol.wait) before it reads T_a
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(256);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  e = cudaLaunchKernelEx(&cfg, kern, n1, n2, n3, p1, p2, XT1, XT2, Ta, eta);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace glam
