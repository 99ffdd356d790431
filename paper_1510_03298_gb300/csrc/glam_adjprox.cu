// The last G stage and the inner PG step of the fit path in one kernel.
//
// After the fused slab kernel has left S_b (n3 x p2p1, FP32), one inner iteration of Sec. 3.2
// still needs Q = X_3^T S_b (mode 3 of Eq. nineteen) and the prox step on every coordinate
// m = (j3, n):  g = g_k + Q / n,  y = x + omega_l (x - x_prev),  x+ = soft(y - delta g,
// delta lambda w_m)  (Sec. 6.3), the next correction x+ + omega_{l+1} (x+ - x) - theta_k, and the
// stop criterion max |x+ - y|.  Each CTA owns a tile of TJ rows j3 x 32 columns n of Q and sums
// it over every i3 itself, so no split partials go through memory and no second kernel is
// launched.  The i3 range streams through shared memory in chunks of up to 256 rows: a 2-D
// tensor copy of S_b (box 32 x KC) and one of X_3^T (box KC x TJ) per chunk, three buffers (up to
// three chunks in flight from the start), with bounded mbarrier waits.  Lane = column, warp = an eighth of each chunk's rows; the eight
// warp partials are added in warp order in FP64 (the same bits on every run).  The operands of
// the prox step and the loop state are loaded at kernel start, behind the chunk copies.  The
// criterion ends in the last-block-done protocol of the prox kernel (glam_elementwise.cu) on the
// same control block.
#include <cuda.h>

#include <atomic>
#include <cstdint>

#include "glam_internal.cuh"
#include "glam_tma.cuh"

namespace glam {
namespace {

using namespace tma;

constexpr int kAPThreads = 256;
constexpr int kAPWarps = kAPThreads / 32;
constexpr int kAPMaxRows = 8;   // rows j3 of a tile, at most
constexpr int kAPMaxChunk = 256;  // rows i3 of a chunk, at most (tensor-copy box limit)
constexpr int kAPBufs = 3;        // chunk buffers: up to three chunks in flight at once
constexpr int kAPMaxSmem = kAPBufs * (kAPMaxChunk * 32 + kAPMaxChunk * kAPMaxRows) * 4;

struct APShape {
  int n3, p3, P21;
  int TJ;      // rows j3 of a tile
  int nx;      // column tiles
  int KC;      // rows i3 per chunk (a multiple of 8 warps x 4)
  int nchunk;  // chunks of the i3 range
};

__device__ double ap_block_max(double v) {
  __shared__ double sh[kAPWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < kAPWarps; ++w) m = fmax(m, sh[w]);
  return m;
}

template <int TJ>
__global__ void __launch_bounds__(kAPThreads)
adjprox_kernel(APShape sh, const __grid_constant__ CUtensorMap mapS, const __grid_constant__ CUtensorMap mapX,
               const double* __restrict__ gk, const double* __restrict__ x, const double* xp,
               const double* __restrict__ pen, double* out, float* __restrict__ dnext,
               const double* __restrict__ anchor, double inv_n, InnerCtl* ctl, int* err,
               const int* __restrict__ rows) {
  // with a programmatic dependent launch this kernel may start before the preceding one ends:
  // nothing is read or written before it has
  griddep_wait();
  // written by the preceding kernels: the same value in every thread; tested once the first
  // copies are under way, so its load overlaps their issue
  const int done = ctl->done;
  // the loop state of this iteration; the last CTA changes it only after every CTA has arrived
  const int l = ctl->l;
  const double delta = ctl->delta, lam = ctl->lambda, pl1 = ctl->pen_l1, pl2 = ctl->pen_l2;
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ uint64_t mbar[kAPBufs];
  __shared__ int timed_out;
  __shared__ bool is_last;
  float* const base = reinterpret_cast<float*>(smem_raw);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int KC = sh.KC, P21 = sh.P21;
  const int tn = blockIdx.x % sh.nx, tj = blockIdx.x / sh.nx;
  const int n0 = 32 * tn, j0 = TJ * tj;
  // the rows i3 where this tile's rows of X_3 have nonzero entries (from rows[]: per j3 the first
  // and one past the last nonzero i3), the start rounded down to 4 (16-byte copy coordinates);
  // the other rows add exact zeros
  int i_lo = 0, i_hi = sh.n3;
  if (rows != nullptr) {
    i_lo = sh.n3;
    i_hi = 0;
    for (int j = j0; j < j0 + TJ && j < sh.p3; ++j) {
      i_lo = min(i_lo, rows[2 * j]);
      i_hi = max(i_hi, rows[2 * j + 1]);
    }
    i_lo &= ~3;
    if (i_hi < i_lo) i_hi = i_lo;
  }
  const int nchunk = (i_hi - i_lo + KC - 1) / KC;
  const int stage = KC * 32 + KC * TJ;  // floats per buffer: S chunk [KC][32], X chunk [TJ][KC]
  const uint32_t bytes = (uint32_t)stage * 4u;
  if (tid == 0) {
    timed_out = 0;
    for (int b = 0; b < kAPBufs; ++b) mbar_init(&mbar[b], 1);
    fence_mbar_init();
  }
  __syncthreads();
  auto issue = [&](int c, int b) {  // called by thread 0
    float* dst = base + (int64_t)b * stage;
    fence_proxy_async();
    mbar_expect_tx(&mbar[b], bytes);
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(&mapS)), "r"(n0), "r"(i_lo + c * KC), "r"(smem_u32(&mbar[b]))
        : "memory");
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
        "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst + KC * 32)),
        "l"(reinterpret_cast<uint64_t>(&mapX)), "r"(i_lo + c * KC), "r"(j0), "r"(smem_u32(&mbar[b]))
        : "memory");
  };
  const int nfirst = nchunk < kAPBufs ? nchunk : kAPBufs;
  if (tid == 0)
    for (int c = 0; c < nfirst; ++c) issue(c, c);
  if (done) {  // the loop has stopped: nothing to compute; the copies land before the CTA leaves
    if (tid == 0)
      for (int c = 0; c < nfirst; ++c) mbar_wait_bounded(&mbar[c], 0u);
    return;
  }
  // the prox operands of this thread's coordinate (at most one: TJ x 32 <= 256), loaded now
  const int jo = tid / 32, co = tid - jo * 32;
  const int j3o = j0 + jo, no = n0 + co;
  const bool mine = tid < TJ * 32 && j3o < sh.p3 && no < P21;
  const int64_t mo = (int64_t)j3o * P21 + no;
  double xm = 0.0, xpm = 0.0, gm = 0.0, pm = 0.0, am = 0.0;
  if (mine) {
    xm = x[mo];
    xpm = xp[mo];
    gm = gk[mo];
    pm = pen[mo];
    am = anchor[mo];
  }
  // ---- Q(j0 + j, n0 + lane) over this warp's rows of every chunk (rows past n3 read zeros) ----
  float acc[TJ];
#pragma unroll
  for (int j = 0; j < TJ; ++j) acc[j] = 0.f;
  const int RW = KC / kAPWarps;  // rows of a chunk per warp (a multiple of 4)
  for (int c = 0; c < nchunk; ++c) {
    const int b = c % kAPBufs;
    if (!mbar_wait_bounded(&mbar[b], (uint32_t)((c / kAPBufs) & 1))) atomicOr(&timed_out, 1);
    __syncthreads();
    if (timed_out) break;  // read after the barrier that follows every write to it
    const float* Sc = base + (int64_t)b * stage;
    const float* Xc = Sc + KC * 32;
    const int r0 = warp * RW;
    // four rows i3 per step: their S_b values for this lane's column, and for each j3 the four
    // X_3 entries as one broadcast float4; the sums run in row order
#pragma unroll 2
    for (int r = r0; r < r0 + RW; r += 4) {
      const float s0 = Sc[r * 32 + lane], s1 = Sc[(r + 1) * 32 + lane];
      const float s2 = Sc[(r + 2) * 32 + lane], s3 = Sc[(r + 3) * 32 + lane];
#pragma unroll
      for (int j = 0; j < TJ; ++j) {
        const float4 xv = *reinterpret_cast<const float4*>(Xc + j * KC + r);
        acc[j] = fmaf(xv.x, s0, acc[j]);
        acc[j] = fmaf(xv.y, s1, acc[j]);
        acc[j] = fmaf(xv.z, s2, acc[j]);
        acc[j] = fmaf(xv.w, s3, acc[j]);
      }
    }
    __syncthreads();  // every warp is done with buffer b
    if (tid == 0 && c + kAPBufs < nchunk) issue(c + kAPBufs, b);
  }
  // ---- the warp partials, added in warp order (FP64), then the prox step per coordinate ----
  float* red = base;  // [warp][TJ][32], over buffer 0 (free after the loop's last barrier)
#pragma unroll
  for (int j = 0; j < TJ; ++j) red[(warp * TJ + j) * 32 + lane] = acc[j];
  __shared__ double om_s[2];  // the extrapolation weights, divided once per CTA (FP64 is slow here)
  if (tid == 0) {
    om_s[0] = double(l - 1) / double(l + 2);
    om_s[1] = double(l) / double(l + 3);
  }
  __syncthreads();
  const double omega = om_s[0], omega_next = om_s[1];
  double crit = 0.0;
  if (!timed_out && mine) {
    // the warp partials (FP32 sums themselves) added in warp order in FP32: FP64 is slow here
    float qs = 0.f;
    for (int w = 0; w < kAPWarps; ++w) qs += red[(w * TJ + jo) * 32 + co];
    const double q = (double)qs;
    const double g = gm + q * inv_n;            // gradient of the quadratic model
    const double y = xm + omega * (xm - xpm);   // extrapolation, Sec. 3.2
    const double z = y - delta * g;
    const double gam = delta * lam * pm;
    const double az = fabs(z) - gam * pl1;  // soft threshold, Sec. 6.3, then the ridge shrinkage
    double xn = az > 0.0 ? copysign(az, z) : 0.0;
    if (pl2 != 0.0) xn /= 1.0 + 2.0 * gam * pl2;  // the ridge part (no division for the lasso)
    out[mo] = xn;
    dnext[mo] = (float)(xn + omega_next * (xn - xm) - am);
    crit = fabs(xn - y);
  }
  // ---- stop criterion: the prox kernel's last-block-done protocol on the same control block ----
  const double bm = ap_block_max(crit);
  if (tid == 0) {
    if (timed_out) atomicOr(err, 1);
    atomicMax(&ctl->crit_bits, (unsigned long long)__double_as_longlong(bm));
    __threadfence();
    is_last = (atomicAdd(&ctl->counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && tid == 0)
    ctl_finish_iteration(ctl, __longlong_as_double((long long)atomicAdd(&ctl->crit_bits, 0ull)));
  if (timed_out && tid == 0)  // copies still in flight land before the CTA leaves
    for (int b = 0; b < nfirst; ++b) mbar_wait_bounded(&mbar[b], 0u);
}

// rows[2 j3] = the first i3 with X_3(i3, j3) != 0 (n3 if none), rows[2 j3 + 1] = one past the last
__global__ void x3_rows_kernel(int n3, const float* __restrict__ X3T, int* __restrict__ rows) {
  __shared__ int lo, hi;
  if (threadIdx.x == 0) {
    lo = n3;
    hi = 0;
  }
  __syncthreads();
  const float* r = X3T + (int64_t)blockIdx.x * n3;
  int a = n3, b = 0;
  for (int i = threadIdx.x; i < n3; i += blockDim.x)
    if (r[i] != 0.f) {
      a = min(a, i);
      b = max(b, i + 1);
    }
  atomicMin(&lo, a);
  atomicMax(&hi, b);
  __syncthreads();
  if (threadIdx.x == 0) {
    rows[2 * blockIdx.x] = lo;
    rows[2 * blockIdx.x + 1] = hi;
  }
}

bool ap_configure(int n3, int p3, int P21, APShape& sh, size_t& smem) {
  if (n3 < 1 || p3 < 1 || P21 < 1 || P21 % 4 != 0 || n3 % 4 != 0) return false;
  sh.n3 = n3;
  sh.p3 = p3;
  sh.P21 = P21;
  sh.nx = (P21 + 31) / 32;
  int gy = num_sms() / sh.nx;  // at most one tile per SM: a second CTA on an SM ends last
  if (gy > p3) gy = p3;
  if (gy < 1) gy = 1;
  sh.TJ = (p3 + gy - 1) / gy;
  if (sh.TJ > kAPMaxRows) sh.TJ = kAPMaxRows;
  // chunks of a multiple of 32 rows (every warp's share stays whole), as few as the buffers allow
  const int per = (n3 + kAPBufs - 1) / kAPBufs;
  const int kc = ((per + 31) / 32) * 32;
  sh.KC = kc < kAPMaxChunk ? kc : kAPMaxChunk;
  sh.nchunk = (n3 + sh.KC - 1) / sh.KC;
  smem = (size_t)kAPBufs * (sh.KC * 32 + sh.KC * sh.TJ) * 4;
  return true;
}

std::atomic<int> g_ap_ready{0};

template <int TJ>
cudaError_t ap_prepare_one() {
  cudaError_t e =
      cudaFuncSetAttribute(adjprox_kernel<TJ>, cudaFuncAttributeMaxDynamicSharedMemorySize, kAPMaxSmem);
  // the largest shared-memory carveout, so that two CTAs fit on an SM and the grid (about one
  // tile per SM, a few more than the SMs) runs as one wave
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(adjprox_kernel<TJ>, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
  return e;
}

}  // namespace

int adjprox_supported(int n3, int p3, int P21, const float* X3T, const float* Sb) {
  APShape sh;
  size_t smem;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) % 16) == 0; };
  return ap_configure(n3, p3, P21, sh, smem) && al16(X3T) && al16(Sb) ? 1 : 0;
}

cudaError_t launch_adjprox(int n3, int p3, int P21, const float* X3T, const float* Sb, const double* gk,
                           const double* x, const double* xp, const double* pen, double* out,
                           float* dnext, const double* anchor, double inv_n, InnerCtl* ctl, int* err,
                           cudaStream_t s, bool pdl, const int* x3_rows) {
  APShape sh;
  size_t smem;
  if (!adjprox_supported(n3, p3, P21, X3T, Sb) || !ap_configure(n3, p3, P21, sh, smem))
    return cudaErrorInvalidValue;
  if (!g_ap_ready) {  // the largest tile any shape can ask for: three chunks of 256 rows, 8 rows j3
    cudaError_t e = ap_prepare_one<1>();
    if (e == cudaSuccess) e = ap_prepare_one<2>();
    if (e == cudaSuccess) e = ap_prepare_one<3>();
    if (e == cudaSuccess) e = ap_prepare_one<4>();
    if (e == cudaSuccess) e = ap_prepare_one<5>();
    if (e == cudaSuccess) e = ap_prepare_one<6>();
    if (e == cudaSuccess) e = ap_prepare_one<7>();
    if (e == cudaSuccess) e = ap_prepare_one<8>();
    if (e != cudaSuccess) return e;
    g_ap_ready = 1;
  }
  alignas(64) CUtensorMap mapS, mapX;
  // S_b: rows i3 of p2p1 floats, boxes of 32 columns x KC rows; X_3^T: rows j3 of n3 floats,
  // boxes of KC columns x TJ rows
  if (!encode_map_2d(&mapS, Sb, (uint64_t)P21, (uint64_t)n3, (uint64_t)P21 * 4, 32, (uint32_t)sh.KC) ||
      !encode_map_2d(&mapX, X3T, (uint64_t)n3, (uint64_t)p3, (uint64_t)n3 * 4, (uint32_t)sh.KC,
                     (uint32_t)sh.TJ))
    return cudaErrorInvalidValue;
  const int blocks = sh.nx * ((p3 + sh.TJ - 1) / sh.TJ);
  cudaError_t e = cudaSuccess;
  switch (sh.TJ) {
#define GLAM_AP(tj)                                                                                  \
  case tj:                                                                                           \
    e = launch_pdl(adjprox_kernel<tj>, dim3(blocks), dim3(kAPThreads), smem, s, pdl, sh, mapS, mapX, gk, \
                   x, xp, pen, out, dnext, anchor, inv_n, ctl, err, x3_rows);                        \
    break;
    GLAM_AP(1) GLAM_AP(2) GLAM_AP(3) GLAM_AP(4) GLAM_AP(5) GLAM_AP(6) GLAM_AP(7) GLAM_AP(8)
#undef GLAM_AP
    default: return cudaErrorInvalidValue;
  }
  count_launches(1);
  return e != cudaSuccess ? e : cudaGetLastError();
}

cudaError_t launch_x3_rows(int n3, int p3, const float* X3T, int* rows, cudaStream_t s) {
  x3_rows_kernel<<<p3, 256, 0, s>>>(n3, X3T, rows);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace glam
