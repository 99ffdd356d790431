// The bottleneck product G(V (.) H(d)) of Sec. 6.2 (Eq. twentysixnew) on the 5th-generation
// tensor cores (tcgen05), with the accumulators and the reused operands in tensor memory (TMEM).
//
// Per slab i3 (c = i1 along the 128 TMEM lanes, padded with zero rows when n1 < 128):
//   first H stage  T_a = X_3 d for the CTA's slabs (once per launch, FP32, from d staged by bulk
//                  copies)
//   MMA0 (SIMT)    T_b^T (c x j2) = X_1 (c x j1) T_a^T (j1 x j2)  exact FP32 FMAs on the compute
//                  warps, written to TMEM as the A operand of MMA1
//   MMA1 (tcgen05) eta^T (c x i2) = T_b^T X_2^T                     A from TMEM, B X_2 (i2 rows) in
//                  shared memory, D in TMEM
//   r = V (.) eta  on the compute warps, in place in TMEM (the V chunk staged by TMA)
//   MMA2 (tcgen05) P (c x j2) = r^T X_2                              A = r from TMEM, B X_2^T (j2
//                  rows) in shared memory
//   MMA3 (tcgen05) S_b^T (j1 x j2) = X_1^T P                         P goes through shared memory
//                  (the one transposition of the chain: it contracts the lane index c), M = 64
// and S_b (p2 x p1) is written to global memory for the mode-3 adjoint.  Only eta's 128 x n2 tile
// is ever formed, and only in TMEM.
//
// Arithmetic forms: FORM 1 (TF32 operands rounded to nearest, FP32 accumulation), FORM 3
// (3xTF32: every operand split into hi = tf32(x) and lo = tf32(x - hi); each product as
// hi hi' + hi lo' + lo hi', about FP32 accuracy), FORM 16 (BF16 operands rounded to nearest, FP32
// accumulation).  V is read as FP32, or as BF16 (TV) by the BF16 fit path.
//
// Warp roles (320 threads): warps 0-7 compute (two warpgroups; warp w reaches TMEM lanes
// 32 (w mod 4) .. + 31, i.e. rows c = 32 (w mod 4) + lane), warp 8 issues the MMAs (one thread)
// and owns the TMEM allocation, warp 9 streams V by TMA through a ring of 32-row chunks.  The roles
// meet at mbarriers; every wait is bounded (a kernel parameter, default 2 s) and a wait that runs
// out sets an error flag, after which every role leaves its loop, the copies and MMAs already issued
// are waited for (bounded by at least 2 s), the TMEM is freed and the CTA exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <cstdint>

#include "glam_internal.cuh"
#include "glam_tma.cuh"
#include "glam_umma.cuh"

namespace glam {
namespace {

using namespace tma;

constexpr int kUmThreads = 320;
constexpr int kUmCompute = 256;     // warps 0-7
constexpr int kUmMmaWarp = 8;
constexpr int kUmTmaWarp = 9;
constexpr uint32_t kUmTmemCols = 512;
constexpr int kUmMaxSlots = 16;
constexpr uint64_t kDrainNs = 2000000000ull;

enum : int { kFormTF32 = 1, kForm3x = 3, kFormBF16 = 16 };

// Shape and shared-memory plan (byte offsets from the 1 KB aligned base).
struct UmShape {
  int n1, n2, n3, p1, p2, p3;
  int NB1;     // 8-column blocks of j1 (p1 <= 8 NB1)
  int K1;      // K of MMA1 (j2, padded): multiple of 8 (TF32) or 16 (BF16)
  int N2;      // N of MMA2 (j2, padded to 16)
  int N3;      // N of MMA3 (j2, padded to 8)
  int KA1;     // K atoms of MMA3 (i1): 32 (TF32) or 64 (BF16) elements each
  int KA2;     // K atoms of MMA2 (i2)
  int nchunk;  // V chunks of 32 rows i2 per slab
  int nslot;   // V ring slots
  int kmax;    // slabs per CTA, at most
  int R;       // rows of d per staging round
  int parts;   // 2 for the 3xTF32 form (hi, lo), else 1
  int64_t o_cst, o_xt1, o_x2t, o_x2, cst_bytes;  // constant block: [XT1 parts][X2T parts][X2 parts]
  int64_t xt1_part, x2t_part, x2_part;
  int64_t o_stage, stage_bytes;  // d staging: the last bytes of the V ring and the P tile
  int64_t o_ptile, ptile_part;
  int64_t o_ring, slot_bytes;
  int64_t o_tas, o_x3r, total;
  // TMEM columns
  uint32_t c_eta, c_rlo, c_rb, c_tb, c_tblo, c_p, c_sb;
};

__host__ __device__ inline int64_t up(int64_t v, int64_t a) { return (v + a - 1) / a * a; }

// element size of the operands of a form
__host__ __device__ inline int um_esz(int form) { return form == kFormBF16 ? 2 : 4; }

// ---------------------------------------------------------------- device helpers
__device__ __forceinline__ uint32_t rna_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half), .y = hi
  return *reinterpret_cast<const uint32_t*>(&v);
}
template <typename TV>
__device__ __forceinline__ float vload(const TV* p);
template <>
__device__ __forceinline__ float vload<float>(const float* p) {
  return *p;
}
template <>
__device__ __forceinline__ float vload<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}

__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// Bounded wait with a caller-given limit (0: give up at once unless the phase has completed).
__device__ __forceinline__ bool wait_for(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  if (limit_ns == 0) return false;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait(bar, parity)) return true;
    if (globaltimer_ns() - t0 > limit_ns) return false;
  }
}
// The same, taken by every lane of a warp with one outcome for the whole warp (a time-out seen by
// any lane is a time-out for all, so the warp never splits before a warp-collective instruction).
__device__ __forceinline__ bool warp_wait(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  const bool ok = wait_for(bar, parity, limit_ns);
  return __all_sync(0xffffffffu, ok) != 0;
}
// one arrival per warp on a barrier counting warps
__device__ __forceinline__ void warp_arrive(uint64_t* bar) {
  __syncwarp();
  if ((threadIdx.x & 31) == 0)
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

// The mbarriers of the kernel, in static shared memory.
struct UmBars {
  uint64_t full[kUmMaxSlots], empty[kUmMaxSlots];
  uint64_t cst, stage, stage_free;
  uint64_t tb_ready, eta_ready, r_ready, p_ready, pt_ready, sb_ready;
};

template <int FORM, typename TV>
__global__ void __launch_bounds__(kUmThreads, 1)
fused_slab_umma_kernel(UmShape sh, const unsigned char* __restrict__ Cst, const float* __restrict__ D,
                       const float* __restrict__ X1T, const float* __restrict__ X3T,
                       const __grid_constant__ CUtensorMap tmapV, float* __restrict__ Sb,
                       const int* __restrict__ skip, int* __restrict__ err, uint64_t wait_ns) {
  constexpr int PARTS = FORM == kForm3x ? 2 : 1;
  constexpr uint32_t kType = FORM == kFormBF16 ? umma::kTypeBF16 : umma::kTypeTF32;
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ UmBars bars;
  __shared__ uint32_t tmem_base_s;
  __shared__ int timed_out;
  const int n1 = sh.n1, n2 = sh.n2, n3 = sh.n3, p1 = sh.p1, p2 = sh.p2, p3 = sh.p3;
  const int P21 = p1 * p2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kcta = (n3 - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  unsigned char* const base =
      smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(base);
  float* const TaS = reinterpret_cast<float*>(base + sh.o_tas);   // [kmax][K1][8 NB1]
  float* const X3r = reinterpret_cast<float*>(base + sh.o_x3r);   // [p3][KQ]
  float* const stage = reinterpret_cast<float*>(base + sh.o_stage);
  const int P1P = 8 * sh.NB1;
  const int KQ = (sh.kmax + 3) / 4 * 4;

  // ---------------------------------------------------------------- set-up
  if (tid == 0) {
    timed_out = 0;
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmapV)) : "memory");
    for (int s = 0; s < sh.nslot; ++s) {
      mbar_init(&bars.full[s], 1);
      mbar_init(&bars.empty[s], 4);  // the four warps of the warpgroup that consumes the chunk
    }
    mbar_init(&bars.cst, 1);
    mbar_init(&bars.stage, 1);
    mbar_init(&bars.stage_free, 1);
    mbar_init(&bars.tb_ready, 8);
    mbar_init(&bars.eta_ready, 1);
    mbar_init(&bars.r_ready, 8);
    mbar_init(&bars.p_ready, 1);
    mbar_init(&bars.pt_ready, 8);
    mbar_init(&bars.sb_ready, 1);
    fence_mbar_init();
  }
  if (warp == kUmMmaWarp) {
    umma::tmem_alloc(&tmem_base_s, kUmTmemCols);
    umma::tmem_relinquish();
  }
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tb = tmem_base_s;

  // ---------------------------------------------------------------- V producer (warp 9)
  if (warp == kUmTmaWarp) {
    if (lane == 0) {
      const int total = kcta * sh.nchunk;
      const uint32_t bytes = (uint32_t)(32 * n1 * (int)sizeof(TV));
      // slots that overlap the d staging area wait until the first H stage is done with it
      bool stage_released = false;
      int issued = 0;
      bool ok = true;
      for (int g = 0; g < total && ok; ++g) {
        const int slot = g % sh.nslot;
        if (g >= sh.nslot) {
          ok = wait_for(&bars.empty[slot], (uint32_t)(((g / sh.nslot) - 1) & 1), wait_ns);
        } else if (!stage_released && sh.o_ring + (int64_t)(slot + 1) * sh.slot_bytes > sh.o_stage) {
          ok = wait_for(&bars.stage_free, 0u, wait_ns);
          stage_released = true;
        }
        if (!ok || *(volatile int*)&timed_out) break;
        const int k = g / sh.nchunk, c = g - k * sh.nchunk;
        const int slab = (int)blockIdx.x + k * (int)gridDim.x;
        unsigned char* dst = base + sh.o_ring + (int64_t)slot * sh.slot_bytes;
        mbar_expect_tx(&bars.full[slot], bytes);
        asm volatile(
            "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes "
            "[%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(dst)),
            "l"(reinterpret_cast<uint64_t>(&tmapV)), "r"(0), "r"(slab * n2 + 32 * c),
            "r"(smem_u32(&bars.full[slot]))
            : "memory");
        ++issued;
      }
      if (!ok) atomicOr(&timed_out, 1);
      // copies still in flight land before the CTA leaves: every issued chunk whose arrival was
      // not consumed (a consumed one has completed its phase, so the wait returns at once)
      for (int g = issued - sh.nslot > 0 ? issued - sh.nslot : 0; g < issued; ++g)
        wait_for(&bars.full[g % sh.nslot], (uint32_t)((g / sh.nslot) & 1),
                 wait_ns > kDrainNs ? wait_ns : kDrainNs);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- prologue (warps 0-8)
    const int nth = kUmCompute + 32, ptid = tid;  // 288 threads
    if (tid == 0) {
      mbar_expect_tx(&bars.cst, (uint32_t)sh.cst_bytes);
      bulk_g2s(base + sh.o_cst, Cst, (uint32_t)sh.cst_bytes, &bars.cst);
    }
    // X_3 entries of this CTA's slabs, [j3][k]
    for (int idx = ptid; idx < p3 * KQ; idx += nth) {
      const int j3 = idx / KQ, kk = idx - j3 * KQ;
      X3r[idx] = kk < kcta ? X3T[(int64_t)j3 * n3 + blockIdx.x + (int64_t)kk * gridDim.x] : 0.f;
    }
    for (int idx = ptid; idx < sh.kmax * sh.K1 * P1P; idx += nth) TaS[idx] = 0.f;
    // first H stage: T_a(s_k, j2, j1) = sum_j3 X_3(s_k, j3) d(j3, j2, j1), in j3 order, R rows of
    // d per round (a bulk copy of their 16-byte multiple; the tail by plain loads)
    const int nround = (p3 + sh.R - 1) / sh.R;
    int rounds_issued = 0;  // thread 0's count of staging copies
    for (int rd = 0; rd < nround; ++rd) {
      const int j0 = rd * sh.R, rows = (j0 + sh.R < p3) ? sh.R : p3 - j0;
      const uint32_t bulk = (uint32_t)(((int64_t)rows * P21) / 4 * 16);
      named_sync(1, nth);  // every thread is done with the previous round (and TaS is zeroed)
      if (tid == 0) {
        fence_proxy_async();
        mbar_expect_tx(&bars.stage, bulk);
        if (bulk > 0) bulk_g2s(stage, D + (int64_t)j0 * P21, bulk, &bars.stage);
        ++rounds_issued;
      }
      for (int i = (int)(bulk / 4) + ptid; i < rows * P21; i += nth) stage[i] = D[(int64_t)j0 * P21 + i];
      if (!wait_for(&bars.stage, (uint32_t)(rd & 1), wait_ns)) atomicOr(&timed_out, 1);
      named_sync(1, nth);
      if (*(volatile int*)&timed_out) break;
      // task = (one column n, 4 slabs k)
      const int nkg = (kcta + 3) / 4;
      for (int task = ptid; task < P21 * nkg; task += nth) {
        const int nn = task % P21, k0 = 4 * (task / P21);
        const int j2 = nn / p1, j1 = nn - j2 * p1;
        float a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = (k0 + r < kcta) ? TaS[((k0 + r) * sh.K1 + j2) * P1P + j1] : 0.f;
#pragma unroll 4
        for (int j = 0; j < rows; ++j) {
          const float dv = stage[j * P21 + nn];
          const float4 x4 = *reinterpret_cast<const float4*>(X3r + (j0 + j) * KQ + k0);
          a[0] = fmaf(x4.x, dv, a[0]);
          a[1] = fmaf(x4.y, dv, a[1]);
          a[2] = fmaf(x4.z, dv, a[2]);
          a[3] = fmaf(x4.w, dv, a[3]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (k0 + r < kcta) TaS[((k0 + r) * sh.K1 + j2) * P1P + j1] = a[r];
      }
    }
    // after a time-out the last staging copy may still be in flight: it lands before the area is
    // handed to the V ring
    if (tid == 0 && rounds_issued > 0)
      wait_for(&bars.stage, (uint32_t)((rounds_issued - 1) & 1), wait_ns > kDrainNs ? wait_ns : kDrainNs);
    named_sync(1, nth);  // T_a complete; the staging area is free
    if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars.stage_free)) : "memory");

    if (warp == kUmMmaWarp) {
      // ---------------------------------------------------------------- MMA issue (warp 8)
      if (lane == 0) {
        bool ok = !*(volatile int*)&timed_out && wait_for(&bars.cst, 0u, wait_ns);
        const uint32_t x1b = sbase + (uint32_t)sh.o_xt1, x2tb = sbase + (uint32_t)sh.o_x2t,
                       x2b = sbase + (uint32_t)sh.o_x2, ptb = sbase + (uint32_t)sh.o_ptile;
        const uint32_t id1 = umma::idesc(128, (uint32_t)n2, kType, kType, 0, 0);
        const uint32_t id2 = umma::idesc(128, (uint32_t)sh.N2, kType, kType, 0, 0);
        const uint32_t id3 = umma::idesc(64, (uint32_t)sh.N3, kType, kType, 0, 0);
        const int ks1 = FORM == kFormBF16 ? sh.K1 / 16 : sh.K1 / 8;
        const int ks2 = FORM == kFormBF16 ? n2 / 16 : n2 / 8;
        const int ks3 = 4 * sh.KA1;
        const uint32_t a_r = tb + (FORM == kFormBF16 ? sh.c_rb : sh.c_eta);
        // MMA1: eta^T = T_b^T X_2^T (A in TMEM, 8 columns per K step; B rows i2, 32 bytes per step)
        auto mma1 = [&]() {
          for (int s = 0; s < ks1; ++s)
            for (int t = 0; t < (PARTS == 2 ? 3 : 1); ++t) {
              // the three products of the split form: hi hi', hi lo', lo hi'
              const uint32_t ac = (t == 2 ? sh.c_tblo : sh.c_tb) + 8u * s;
              const uint64_t bd = umma::sdesc(x2tb + (t == 1 ? (uint32_t)sh.x2t_part : 0u) + 32u * s, 16,
                                              1024, umma::kSwizzle128B);
              if (FORM == kFormBF16) umma::mma_f16_ts(tb + sh.c_eta, tb + ac, bd, id1, (s | t) != 0);
              else umma::mma_tf32_ts(tb + sh.c_eta, tb + ac, bd, id1, (s | t) != 0);
            }
        };
        // MMA2: P = r^T X_2 (A = r in TMEM; B rows j2, K atoms of 128 bytes)
        auto mma2 = [&]() {
          for (int s = 0; s < ks2; ++s)
            for (int t = 0; t < (PARTS == 2 ? 3 : 1); ++t) {
              const uint32_t ac = (t == 2 ? sh.c_rlo : (a_r - tb)) + 8u * s;
              const uint32_t bo = (uint32_t)((s >> 2) * sh.N2 * 128 + (s & 3) * 32);
              const uint64_t bd = umma::sdesc(x2b + (t == 1 ? (uint32_t)sh.x2_part : 0u) + bo, 16, 1024,
                                              umma::kSwizzle128B);
              if (FORM == kFormBF16) umma::mma_f16_ts(tb + sh.c_p, tb + ac, bd, id2, (s | t) != 0);
              else umma::mma_tf32_ts(tb + sh.c_p, tb + ac, bd, id2, (s | t) != 0);
            }
        };
        // MMA3: S_b^T = X_1^T P (M = 64: A reads 64 rows j1 of 32-row atoms, rows past p1 unused)
        auto mma3 = [&]() {
          for (int s = 0; s < ks3; ++s)
            for (int t = 0; t < (PARTS == 2 ? 3 : 1); ++t) {
              const uint32_t ao = (uint32_t)((s >> 2) * 4096 + (s & 3) * 32);
              const uint32_t bo = (uint32_t)((s >> 2) * sh.N3 * 128 + (s & 3) * 32);
              const uint64_t ad = umma::sdesc(x1b + (t == 2 ? (uint32_t)sh.xt1_part : 0u) + ao, 16, 1024,
                                              umma::kSwizzle128B);
              const uint64_t bd = umma::sdesc(ptb + (t == 1 ? (uint32_t)sh.ptile_part : 0u) + bo, 16, 1024,
                                              umma::kSwizzle128B);
              if (FORM == kFormBF16) umma::mma_f16_ss(tb + sh.c_sb, ad, bd, id3, (s | t) != 0);
              else umma::mma_tf32_ss(tb + sh.c_sb, ad, bd, id3, (s | t) != 0);
            }
        };
        int committed = 0;  // commits issued (the last one is drained before the TMEM is freed)
        uint64_t* last_bar = nullptr;
        uint32_t last_par = 0;
        auto commit_to = [&](uint64_t* bar, uint32_t par) {
          umma::commit(bar);
          last_bar = bar;
          last_par = par;
          ++committed;
        };
        for (int k = 0; k < kcta && ok; ++k) {
          const uint32_t par = (uint32_t)(k & 1);
          if (k == 0) {
            ok = wait_for(&bars.tb_ready, 0u, wait_ns);
            if (!ok) break;
            umma::fence_after_sync();
            mma1();
            commit_to(&bars.eta_ready, 0u);
          }
          ok = wait_for(&bars.r_ready, par, wait_ns);
          if (!ok) break;
          umma::fence_after_sync();
          mma2();
          commit_to(&bars.p_ready, par);
          if (k + 1 < kcta) {
            ok = wait_for(&bars.tb_ready, (uint32_t)((k + 1) & 1), wait_ns);
            if (!ok) break;
            umma::fence_after_sync();
            mma1();  // in issue order after MMA2 of slab k, which read the r columns it overwrites
            commit_to(&bars.eta_ready, (uint32_t)((k + 1) & 1));
          }
          ok = wait_for(&bars.pt_ready, par, wait_ns);
          if (!ok) break;
          umma::fence_after_sync();
          mma3();
          commit_to(&bars.sb_ready, par);
        }
        if (!ok) atomicOr(&timed_out, 1);
        // every MMA issued has completed before the TMEM is released (the last commit covers all)
        if (committed > 0) wait_for(last_bar, last_par, wait_ns > kDrainNs ? wait_ns : kDrainNs);
      }
      __syncwarp();
    } else {
      // ---------------------------------------------------------------- compute warps 0-7
      const int q = warp & 3, wg = warp >> 2;
      const int c = 32 * q + lane;  // TMEM lane = row i1
      const bool rowok = c < n1;
      const uint32_t lq = (uint32_t)(32 * q) << 16;
      // this thread's row of X_1 (FP32), zero past p1 and past n1
      float x1[32];
#pragma unroll
      for (int j = 0; j < 32; ++j) x1[j] = (rowok && j < p1) ? X1T[(int64_t)j * n1 + c] : 0.f;
      bool ok = __all_sync(0xffffffffu, !*(volatile int*)&timed_out) != 0;
      // MMA0 on the compute warps: T_b^T(c, j2) = sum_j1 X_1(c, j1) T_a(k, j2, j1), written as the
      // A operand of MMA1 (warpgroup wg takes the 8- or 16-column groups wg, wg + 2, ...)
      auto mma0 = [&](int kk) {
        const float* ta = TaS + (int64_t)kk * sh.K1 * P1P;
        constexpr int GW = FORM == kFormBF16 ? 16 : 8;  // j2 per group (8 TMEM columns)
        for (int g0 = wg; g0 < sh.K1 / GW; g0 += 2) {
          float acc[GW];
#pragma unroll
          for (int u = 0; u < GW; ++u) {
            const float* row = ta + (g0 * GW + u) * P1P;
            float s = 0.f;
#pragma unroll
            for (int j = 0; j < 32; j += 4) {
              if (j < P1P) {
                const float4 t4 = *reinterpret_cast<const float4*>(row + j);
                s = fmaf(x1[j], t4.x, s);
                s = fmaf(x1[j + 1], t4.y, s);
                s = fmaf(x1[j + 2], t4.z, s);
                s = fmaf(x1[j + 3], t4.w, s);
              }
            }
            acc[u] = s;
          }
          uint32_t hi[8], lo[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (FORM == kFormBF16) {
              hi[u] = pack_bf16(acc[2 * u], acc[2 * u + 1 < GW ? 2 * u + 1 : 0]);
            } else {
              hi[u] = rna_tf32(acc[u]);
              lo[u] = rna_tf32(acc[u] - __uint_as_float(hi[u]));
            }
          }
          umma::st_x8(tb + lq + sh.c_tb + 8u * g0, hi);
          if (PARTS == 2) umma::st_x8(tb + lq + sh.c_tblo + 8u * g0, lo);
        }
        umma::wait_st();
        umma::fence_before_sync();
        warp_arrive(&bars.tb_ready);
      };
      if (ok) mma0(0);
      for (int k = 0; k < kcta && ok; ++k) {
        const uint32_t par = (uint32_t)(k & 1);
        const int slab = (int)blockIdx.x + k * (int)gridDim.x;
        // ---- r = V (.) eta over this warpgroup's chunks of 32 columns i2 (wg, wg + 2, ...)
        ok = warp_wait(&bars.eta_ready, par, wait_ns);
        if (!ok) break;
        umma::fence_after_sync();
        for (int ch = wg; ch < sh.nchunk; ch += 2) {
          const int g = k * sh.nchunk + ch, slot = g % sh.nslot;
          ok = warp_wait(&bars.full[slot], (uint32_t)((g / sh.nslot) & 1), wait_ns);
          if (!ok) break;
          const TV* vs = reinterpret_cast<const TV*>(base + sh.o_ring + (int64_t)slot * sh.slot_bytes);
#pragma unroll
          for (int h = 0; h < 2; ++h) {  // two halves of 16 columns
            uint32_t e[16];
            umma::ld_x16(tb + lq + sh.c_eta + 32u * ch + 16u * h, e);
            float v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = rowok ? vload<TV>(vs + (16 * h + u) * n1 + c) : 0.f;
            umma::wait_ld();
            if (FORM == kFormBF16) {
              uint32_t pk[8];
#pragma unroll
              for (int u = 0; u < 8; ++u)
                pk[u] = pack_bf16(v[2 * u] * __uint_as_float(e[2 * u]), v[2 * u + 1] * __uint_as_float(e[2 * u + 1]));
              umma::st_x8(tb + lq + sh.c_rb + 16u * ch + 8u * h, pk);
            } else {
              uint32_t hi[16], lo[16];
#pragma unroll
              for (int u = 0; u < 16; ++u) {
                const float r = v[u] * __uint_as_float(e[u]);
                hi[u] = rna_tf32(r);
                lo[u] = rna_tf32(r - __uint_as_float(hi[u]));
              }
              umma::st_x16(tb + lq + sh.c_eta + 32u * ch + 16u * h, hi);
              if (PARTS == 2) umma::st_x16(tb + lq + sh.c_rlo + 32u * ch + 16u * h, lo);
            }
          }
          warp_arrive(&bars.empty[slot]);
        }
        if (!ok) break;
        umma::wait_st();
        umma::fence_before_sync();
        warp_arrive(&bars.r_ready);
        // ---- MMA0 of the next slab while MMA2 of this one runs
        if (k + 1 < kcta) mma0(k + 1);
        // ---- P (c, j2) from TMEM into the B operand of MMA3 (K-major rows j2, K = c; warp q
        // writes K atom q of 32 rows c (TF32) or half of atom q / 2 (BF16))
        ok = warp_wait(&bars.p_ready, par, wait_ns);
        if (!ok) break;
        umma::fence_after_sync();
        for (int g0 = wg; g0 < sh.N3 / 8; g0 += 2) {
          uint32_t pv[8];
          umma::ld_x8(tb + lq + sh.c_p + 8u * g0, pv);
          umma::wait_ld();
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int j2 = 8 * g0 + u;
            const float x = __uint_as_float(pv[u]);
            if (FORM == kFormBF16) {
              if ((c >> 6) >= sh.KA1) continue;  // rows past the last K atom: MMA3 does not read them
              const uint32_t off = (uint32_t)((c >> 6) * sh.N3 * 128) + umma::sw128_k2((uint32_t)j2, (uint32_t)(c & 63));
              *reinterpret_cast<__nv_bfloat16*>(base + sh.o_ptile + off) = __float2bfloat16_rn(x);
            } else {
              if (q >= sh.KA1) continue;
              const uint32_t off = (uint32_t)(q * sh.N3 * 128) + umma::sw128_k4((uint32_t)j2, (uint32_t)lane);
              const uint32_t h = rna_tf32(x);
              *reinterpret_cast<uint32_t*>(base + sh.o_ptile + off) = h;
              if (PARTS == 2)
                *reinterpret_cast<uint32_t*>(base + sh.o_ptile + sh.ptile_part + off) =
                    rna_tf32(x - __uint_as_float(h));
            }
          }
        }
        fence_proxy_async();
        warp_arrive(&bars.pt_ready);
        // ---- S_b^T (j1, j2) from TMEM (M = 64 layout: rows 0-15 in lanes 0-15 of warp 0, rows
        // 16-31 in lanes 0-15 of warp 1) to global memory
        if (warp < 2) {
          ok = warp_wait(&bars.sb_ready, par, wait_ns);
          if (!ok) break;
          umma::fence_after_sync();
          const int j1 = 16 * warp + lane;
          float* out = Sb + (int64_t)slab * P21;
          for (int g0 = 0; g0 < sh.N3 / 8; ++g0) {
            uint32_t sv[8];
            umma::ld_x8(tb + lq + sh.c_sb + 8u * g0, sv);
            umma::wait_ld();
            if (lane < 16 && j1 < p1) {
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int j2 = 8 * g0 + u;
                if (j2 < p2) out[j2 * p1 + j1] = __uint_as_float(sv[u]);
              }
            }
          }
        }
      }
      if (!ok) atomicOr(&timed_out, 1);
      umma::fence_before_sync();
      // the constant block's copy has landed before the CTA leaves (at once in a normal run)
      if (tid == 0) wait_for(&bars.cst, 0u, wait_ns > kDrainNs ? wait_ns : kDrainNs);
    }
  }
  __syncthreads();
  if (timed_out && tid == 0) atomicOr(err, 1);
  if (warp == kUmMmaWarp) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tb, kUmTmemCols);
  }
}

// ---------------------------------------------------------------- constant block
// The operand tiles of X_1 and X_2 as they sit in shared memory (K-major, 128-byte swizzle), in
// the kernel's element type, with the hi / lo parts of the 3xTF32 form; zeros in all padding:
//   XT1: MMA3's A, rows j1 (32 per atom), K = i1 (KA1 atoms of 4 KB)
//   X2T: MMA1's B, rows i2 (n2), K = j2 (one atom row)
//   X2 : MMA2's B, rows j2 (N2), K = i2 (KA2 atoms of N2 x 128 bytes)
__global__ void umma_const_kernel(UmShape sh, int form, const float* __restrict__ X1T,
                                  const float* __restrict__ X2T, unsigned char* __restrict__ out) {
  const int esz = form == kFormBF16 ? 2 : 4;
  const int epr = 128 / esz;  // elements per 128-byte row
  const int64_t nel = sh.cst_bytes / esz;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nel; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e * esz;  // byte offset in the block
    int part = 0;
    int64_t off = 0;
    float v = 0.f;
    // locate (region, part, row, k) from the byte offset by inverting the swizzle of its atom
    auto inv = [&](int64_t o, int64_t atom_bytes, int& atom, int& row, int& k) {
      atom = (int)(o / atom_bytes);
      const int64_t w = o - (int64_t)atom * atom_bytes;
      row = (int)(w / 128);
      const int chunk = (int)((w % 128) / 16) ^ (row & 7);
      k = chunk * (16 / esz) + (int)((w % 16) / esz);
    };
    if (b < sh.o_x2t - sh.o_xt1) {  // XT1
      part = (int)(b / sh.xt1_part);
      off = b - part * sh.xt1_part;
      int atom, row, k;
      inv(off, 4096, atom, row, k);
      const int j1 = row, i1 = atom * epr + k;
      if (j1 < sh.p1 && i1 < sh.n1) v = X1T[(int64_t)j1 * sh.n1 + i1];
    } else if (b < sh.o_x2 - sh.o_xt1) {  // X2T
      const int64_t bb = b - (sh.o_x2t - sh.o_xt1);
      part = (int)(bb / sh.x2t_part);
      off = bb - part * sh.x2t_part;
      int atom, row, k;
      inv(off, (int64_t)sh.n2 * 128, atom, row, k);
      const int i2 = row, j2 = k;
      if (j2 < sh.p2) v = X2T[(int64_t)j2 * sh.n2 + i2];
    } else {  // X2
      const int64_t bb = b - (sh.o_x2 - sh.o_xt1);
      part = (int)(bb / sh.x2_part);
      off = bb - part * sh.x2_part;
      int atom, row, k;
      inv(off, (int64_t)sh.N2 * 128, atom, row, k);
      const int j2 = row, i2 = atom * epr + k;
      if (j2 < sh.p2 && i2 < sh.n2) v = X2T[(int64_t)j2 * sh.n2 + i2];
    }
    if (form == kFormBF16) {
      reinterpret_cast<__nv_bfloat16*>(out)[e] = __float2bfloat16_rn(v);
    } else {
      const uint32_t h = rna_tf32(v);
      const uint32_t l = rna_tf32(v - __uint_as_float(h));
      reinterpret_cast<uint32_t*>(out)[e] = part == 0 ? h : l;
    }
  }
}

size_t g_um_budget = 227 * 1024 - 1024;

// The kernel's plan for a shape and form; false outside its domain.
bool um_configure(int n1, int n2, int n3, int p1, int p2, int p3, int grid, int form, bool v_bf16, UmShape& s) {
  if (!(form == kFormTF32 || form == kForm3x || form == kFormBF16)) return false;
  if (v_bf16 && form != kFormBF16) return false;
  const int vesz = v_bf16 ? 2 : 4;  // bytes of a V element (the ring slots hold V as it is stored)
  if (n1 < 4 || n1 > 128 || n1 % (form == kFormBF16 ? 8 : 4) != 0 || n2 < 32 || n2 % 32 != 0 || n3 < 1 || p1 < 1 || p1 > 32 ||
      p2 < 1 || p2 > 32 || p3 < 1 || grid < 1)
    return false;
  const int parts = form == kForm3x ? 2 : 1;
  const int esz = um_esz(form);
  if (n2 > (form == kForm3x ? 128 : 256)) return false;
  s.n1 = n1; s.n2 = n2; s.n3 = n3; s.p1 = p1; s.p2 = p2; s.p3 = p3;
  s.parts = parts;
  s.NB1 = (p1 + 7) / 8;
  s.K1 = form == kFormBF16 ? (int)up(p2, 16) : (int)up(p2, 8);
  s.N2 = (int)up(p2, 16);
  s.N3 = (int)up(p2, 8);
  const int epr = 128 / esz;
  s.KA1 = (n1 + epr - 1) / epr;
  s.KA2 = (n2 + epr - 1) / epr;
  s.nchunk = n2 / 32;
  s.kmax = (n3 + grid - 1) / grid;
  // constant block
  s.xt1_part = (int64_t)s.KA1 * 4096;
  s.x2t_part = (int64_t)n2 * 128;
  s.x2_part = (int64_t)s.KA2 * s.N2 * 128;
  int64_t o = 0;
  s.o_cst = o;
  s.o_xt1 = o;
  o += parts * s.xt1_part;
  s.o_x2t = o;
  o += parts * s.x2t_part;
  s.o_x2 = o;
  o += parts * s.x2_part;
  s.cst_bytes = o - s.o_cst;
  // MMA3 reads 64 rows of each 32-row XT1 atom: the last atom's reads run 4 KB past the XT1 parts,
  // into the X2T tile (n2 >= 32 rows of 128 bytes)
  o = up(o, 1024);
  // the V ring, then the P tile; d is staged for the first H stage in the last bytes of the two
  // (so that the first V chunks, in the first slots, can be in flight while T_a is formed)
  s.o_ring = o;
  s.slot_bytes = up((int64_t)32 * n1 * vesz, 1024);
  s.ptile_part = (int64_t)s.KA1 * s.N3 * 128;
  const int64_t ptile_bytes = up(parts * s.ptile_part, 1024);
  const int KQ = (s.kmax + 3) / 4 * 4;
  const int64_t tas_bytes = up((int64_t)s.kmax * s.K1 * 8 * s.NB1 * 4, 16);
  const int64_t tail = ptile_bytes + tas_bytes + (int64_t)p3 * KQ * 4;
  const int64_t room = (int64_t)g_um_budget - 1024 - o - tail;
  int slots = (int)(room / s.slot_bytes);
  if (slots > kUmMaxSlots) slots = kUmMaxSlots;
  if (slots > 2 * s.nchunk) slots = 2 * s.nchunk > 2 ? 2 * s.nchunk : 2;
  if (slots < 2) return false;
  s.nslot = slots;
  o += (int64_t)slots * s.slot_bytes;
  s.o_ptile = o;
  o += ptile_bytes;
  const int64_t stage_end = o, stage_cap = o - s.o_ring;
  s.o_tas = o;
  o += tas_bytes;
  s.o_x3r = o;
  o += (int64_t)p3 * KQ * 4;
  s.total = up(o, 16);
  // rows of d per staging round (16-byte aligned round starts when p2 p1 is not a multiple of 4)
  const int64_t P21 = (int64_t)p1 * p2;
  int64_t R = stage_cap / (P21 * 4);
  if (R >= p3) R = p3;
  else if (P21 % 4 != 0) R = R / 4 * 4;
  if (R < 1) return false;
  s.R = (int)R;
  s.stage_bytes = up(R * P21 * 4, 16);
  s.o_stage = stage_end - s.stage_bytes;
  // TMEM columns (each region starts on a multiple of 32)
  uint32_t col = 0;
  s.c_eta = col;
  col += (uint32_t)up(n2, 32);
  s.c_rlo = col;
  s.c_rb = col;
  if (form == kForm3x) col += (uint32_t)up(n2, 32);
  if (form == kFormBF16) col += (uint32_t)up(n2 / 2, 32);
  s.c_tb = col;
  col += 32;
  s.c_tblo = col;
  if (form == kForm3x) col += 32;
  s.c_p = col;
  col += 32;
  s.c_sb = col;
  col += 32;
  if (col > kUmTmemCols) return false;
  return (size_t)(s.total + 1024) <= g_um_budget;
}

PFN_cuTensorMapEncodeTiled_v12000 um_encode() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool done = false;
  if (!done) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    done = true;
  }
  return fn;
}

// V as a 2-D tensor (n1 columns, n2 n3 rows) with boxes of 32 rows, no swizzle.
bool um_encode_v(CUtensorMap* m, const void* V, int n1, int64_t rows, bool bf16) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = um_encode();
  if (fn == nullptr) return false;
  const int esz = bf16 ? 2 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)n1, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n1 * esz};
  const cuuint32_t box[2] = {(cuuint32_t)n1, 32};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<void*>(V),
            dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

template <int FORM, typename TV>
cudaError_t um_prepare_one() {
  return cudaFuncSetAttribute(fused_slab_umma_kernel<FORM, TV>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)g_um_budget);
}

int um_grid(int n3) { return n3 < num_sms() ? n3 : num_sms(); }

}  // namespace

cudaError_t fused_umma_prepare() {
  int dev = 0, optin = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  g_um_budget = optin > 2048 ? (size_t)optin - 2048 : 0;  // room for the kernel's static variables
  if (e == cudaSuccess) e = um_prepare_one<kFormTF32, float>();
  if (e == cudaSuccess) e = um_prepare_one<kForm3x, float>();
  if (e == cudaSuccess) e = um_prepare_one<kFormBF16, float>();
  if (e == cudaSuccess) e = um_prepare_one<kFormBF16, __nv_bfloat16>();
  return e;
}

int fused_umma_supported(int n1, int n2, int n3, int p1, int p2, int p3, int form) {
  UmShape s;
  // both V element types of the form (the BF16 form takes BF16 V in the fit path, FP32 elsewhere)
  return um_configure(n1, n2, n3, p1, p2, p3, um_grid(n3), form, false, s) &&
                 (form != kFormBF16 || um_configure(n1, n2, n3, p1, p2, p3, um_grid(n3), form, true, s))
             ? 1
             : 0;
}

int64_t fused_umma_const_bytes(int n1, int n2, int n3, int p1, int p2, int p3, int form) {
  UmShape s;
  return um_configure(n1, n2, n3, p1, p2, p3, um_grid(n3), form, false, s) ? s.cst_bytes : 0;
}

cudaError_t launch_fused_umma_const(int n1, int n2, int n3, int p1, int p2, int p3, int form,
                                    const float* X1T, const float* X2T, void* Cst, cudaStream_t st) {
  UmShape s;
  if (!um_configure(n1, n2, n3, p1, p2, p3, um_grid(n3), form, false, s)) return cudaErrorInvalidValue;
  const int64_t nel = s.cst_bytes / um_esz(form);
  int blocks = (int)((nel + 255) / 256);
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
  umma_const_kernel<<<blocks, 256, 0, st>>>(s, form, X1T, X2T, static_cast<unsigned char*>(Cst));
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_fused_umma(int n1, int n2, int n3, int p1, int p2, int p3, int form, bool v_bf16,
                              const void* Cst, const float* D, const float* X1T, const float* X3T,
                              const void* V, float* Sb, cudaStream_t st, const int* skip, int* err,
                              uint64_t wait_ns) {
  UmShape s;
  const int grid = um_grid(n3);
  if (!um_configure(n1, n2, n3, p1, p2, p3, grid, form, v_bf16, s)) return cudaErrorInvalidValue;
  auto al16 = [](const void* q) { return (reinterpret_cast<uintptr_t>(q) % 16) == 0; };
  if (!al16(Cst) || !al16(D) || !al16(V)) return cudaErrorInvalidValue;
  alignas(64) CUtensorMap tmapV;
  if (!um_encode_v(&tmapV, V, n1, (int64_t)n2 * n3, v_bf16)) return cudaErrorInvalidValue;
  // at least half of the shared memory of an SM: one CTA per SM, so two CTAs never queue on the
  // TMEM allocation of 512 columns
  size_t smem = (size_t)s.total + 1024;
  if (smem < g_um_budget / 2 + 1024) smem = g_um_budget / 2 + 1024;
  const unsigned char* c = static_cast<const unsigned char*>(Cst);
  if (form == kFormTF32)
    fused_slab_umma_kernel<kFormTF32, float><<<grid, kUmThreads, smem, st>>>(s, c, D, X1T, X3T, tmapV, Sb, skip,
                                                                            err, wait_ns);
  else if (form == kForm3x)
    fused_slab_umma_kernel<kForm3x, float><<<grid, kUmThreads, smem, st>>>(s, c, D, X1T, X3T, tmapV, Sb, skip,
                                                                          err, wait_ns);
  else if (v_bf16)
    fused_slab_umma_kernel<kFormBF16, __nv_bfloat16><<<grid, kUmThreads, smem, st>>>(s, c, D, X1T, X3T, tmapV, Sb,
                                                                                    skip, err, wait_ns);
  else
    fused_slab_umma_kernel<kFormBF16, float><<<grid, kUmThreads, smem, st>>>(s, c, D, X1T, X3T, tmapV, Sb, skip,
                                                                            err, wait_ns);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace glam
