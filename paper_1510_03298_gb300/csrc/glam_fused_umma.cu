// The bottleneck product G(V (.) H(d)) of Sec. 6.2 (Eq. twentysixnew) on the 5th-generation
// tensor cores (tcgen05), with the accumulators and the reused operands in tensor memory (TMEM).
//
// Per slab i3 (c = i1 along the 128 TMEM lanes, padded with zero rows when n1 < 128):
//   first H stage  T_a = X_3 d for the CTA's slabs (once per launch, FP32; only the rows j3 where
//                  the CTA's rows of X_3 are nonzero enter the sums, which skips exact zeros)
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
// Issue.  A tcgen05.mma of the small N used here costs its issuing thread about 100 cycles
// whatever N is (measured on this GPU), while several threads issuing at once overlap; so the MMAs
// are issued by three threads and the operand splits of the 3xTF32 form share instructions where
// an operand is common: the hi and lo parts of the constant operand sit side by side along N
// (hi hi' and hi lo' in one instruction of twice the N), leaving hi' lo as the third.
//
// Warp roles (320 threads).  Warps 0-7 compute in two warpgroups; warp w reaches TMEM lanes
// 32 (w mod 4) .. + 31 (rows c = 32 (w mod 4) + lane).  Warpgroup g owns the i2 columns
// [g n2/2, (g+1) n2/2): its leader (warp 4g + 3, lane 0) issues MMA1 for those columns and, chunk
// by chunk as r is formed, MMA2 over those columns into the warpgroup's own partial P (summed when
// P is read); issuing both keeps every reuse of the group's TMEM columns in issue order on one
// thread.  Warp 8 issues MMA3 and owns the TMEM allocation; warp 9 streams V by TMA through a ring
// of 16-row chunks.  The roles meet at mbarriers; every wait is bounded (a kernel parameter,
// default 2 s) and a wait that runs out sets an error flag, after which every role leaves its
// loop, the copies and MMAs already issued are waited for (bounded by at least 2 s), the TMEM is
// freed and the CTA exits.
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
constexpr int kUmRows = 16;         // rows i2 of a V chunk (one 16-column TMEM load per thread)
constexpr uint32_t kUmTmemCols = 512;
constexpr int kUmMaxSlots = 24;
constexpr uint64_t kDrainNs = 2000000000ull;

enum : int { kFormTF32 = 1, kForm3x = 3, kFormBF16 = 16 };

// Shape and shared-memory plan (byte offsets from the 1 KB aligned base).
struct UmShape {
  int n1, n2, n3, p1, p2, p3;
  int K1;      // K of MMA1 (j2, padded): multiple of 8 (TF32) or 16 (BF16)
  int N2;      // N of MMA2 per part (j2, padded to 16)
  int N3;      // N of MMA3 per part (j2, padded to 8)
  int KA1;     // K atoms of MMA3 (i1): 32 (TF32) or 64 (BF16) elements each
  int KA2;     // K atoms of MMA2 (i2)
  int nchunk;  // V chunks of kUmRows rows i2 per slab (each warpgroup takes half)
  int nslot;   // V ring slots
  int kmax;    // slabs per CTA, at most
  int R;       // rows of d per staging round
  int parts;   // 2 for the 3xTF32 form (hi, lo), else 1
  int64_t o_cst, o_xt1, o_x2t, o_x2, cst_bytes;  // constant block: [XT1 parts][X2T parts][X2]
  int64_t xt1_part, x2t_part, x2_atom;           // X2: KA2 atoms of [hi rows N2][lo rows N2]
  int64_t o_stage, stage_bytes;  // d staging: the last bytes of the V ring and the P tile
  int64_t o_ptile, ptile_atom;   // P tile: KA1 atoms of [hi rows N3][lo rows N3]
  int64_t o_ring, slot_bytes;
  int64_t o_tas, o_x3r, o_rows, total;
  // TMEM columns
  uint32_t c_eta, c_rlo, c_rb, c_tb, c_tblo, c_p, pw, c_sb;
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
// named barrier that also returns the AND of `ok` over its threads (the same value in every one)
__device__ __forceinline__ bool named_sync_and(int id, int n, bool ok) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p, q;\n\tsetp.ne.u32 p, %1, 0;\n\tbarrier.red.and.pred q, %2, %3, p;\n\t"
      "selp.u32 %0, 1, 0, q;\n\t}"
      : "=r"(r)
      : "r"((uint32_t)ok), "r"(id), "r"(n)
      : "memory");
  return r != 0;
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
  uint64_t tb_ready, pt_ready, sb_ready;
  uint64_t eta_ready[2], p_ready[2];  // per warpgroup
};

// One tcgen05.mma whose A operand sits in TMEM (TS) or shared memory (SS), by form.
template <int FORM>
__device__ __forceinline__ void mma_ts(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (FORM == kFormBF16) umma::mma_f16_ts(d, a, b, id, acc);
  else umma::mma_tf32_ts(d, a, b, id, acc);
}
template <int FORM>
__device__ __forceinline__ void mma_ss(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
  if (FORM == kFormBF16) umma::mma_f16_ss(d, a, b, id, acc);
  else umma::mma_tf32_ss(d, a, b, id, acc);
}

template <int FORM, typename TV>
__global__ void __launch_bounds__(kUmThreads, 1)
fused_slab_umma_kernel(UmShape sh, const unsigned char* __restrict__ Cst, const float* __restrict__ D,
                       const float* __restrict__ X1T, const float* __restrict__ X3T,
                       const __grid_constant__ CUtensorMap tmapV, float* __restrict__ Sb,
                       const int* __restrict__ skip, int* __restrict__ err, uint64_t wait_ns) {
  constexpr int PARTS = FORM == kForm3x ? 2 : 1;
  constexpr uint32_t kType = FORM == kFormBF16 ? umma::kTypeBF16 : umma::kTypeTF32;
  constexpr uint32_t KS = FORM == kFormBF16 ? 16 : 8;  // K elements of one MMA (32 bytes)
  if (skip != nullptr && *skip) return;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ UmBars bars;
  __shared__ uint32_t tmem_base_s;
  __shared__ int timed_out, nrows_s;
  const int n1 = sh.n1, n2 = sh.n2, n3 = sh.n3, p1 = sh.p1, p2 = sh.p2, p3 = sh.p3;
  const int P21 = p1 * p2, K1 = sh.K1;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kcta = (n3 - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  unsigned char* const base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(base);
  float* const TaS = reinterpret_cast<float*>(base + sh.o_tas);   // [kmax][p1][K1]: T_a(k, j2, j1) at [k][j1][j2]
  float* const X3r = reinterpret_cast<float*>(base + sh.o_x3r);   // [p3][KQ]
  int* const rowlist = reinterpret_cast<int*>(base + sh.o_rows);  // rows j3 with a nonzero X_3 entry
  float* const stage = reinterpret_cast<float*>(base + sh.o_stage);
  const int KQ = (sh.kmax + 3) / 4 * 4;
  const uint64_t drain_ns = wait_ns > kDrainNs ? wait_ns : kDrainNs;

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
    mbar_init(&bars.pt_ready, 8);
    mbar_init(&bars.sb_ready, 1);
    for (int g = 0; g < 2; ++g) {
      mbar_init(&bars.eta_ready[g], 1);
      mbar_init(&bars.p_ready[g], 1);
    }
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
  const int nround = (p3 + sh.R - 1) / sh.R;

  // ---------------------------------------------------------------- V producer (warp 9)
  if (warp == kUmTmaWarp) {
    if (lane == 0) {
      const int total = kcta * sh.nchunk;
      const uint32_t bytes = (uint32_t)(kUmRows * n1 * (int)sizeof(TV));
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
            "l"(reinterpret_cast<uint64_t>(&tmapV)), "r"(0), "r"(slab * n2 + kUmRows * c),
            "r"(smem_u32(&bars.full[slot]))
            : "memory");
        ++issued;
      }
      if (!ok) atomicOr(&timed_out, 1);
      // copies still in flight land before the CTA leaves: every issued chunk whose arrival was
      // not consumed (a consumed one has completed its phase, so the wait returns at once)
      for (int g = issued - sh.nslot > 0 ? issued - sh.nslot : 0; g < issued; ++g)
        wait_for(&bars.full[g % sh.nslot], (uint32_t)((g / sh.nslot) & 1), drain_ns);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- prologue (warps 0-8)
    const int nth = kUmCompute + 32, ptid = tid;  // 288 threads
    int rounds_issued = 0;                        // thread 0's count of staging copies
    auto issue_round = [&](int rd) {              // thread 0: R rows of d (16-byte multiple)
      const int j0 = rd * sh.R, rows = (j0 + sh.R < p3) ? sh.R : p3 - j0;
      const uint32_t bulk = (uint32_t)(((int64_t)rows * P21) / 4 * 16);
      fence_proxy_async();
      mbar_expect_tx(&bars.stage, bulk);
      if (bulk > 0) bulk_g2s(stage, D + (int64_t)j0 * P21, bulk, &bars.stage);
      ++rounds_issued;
    };
    if (tid == 0) {
      mbar_expect_tx(&bars.cst, (uint32_t)sh.cst_bytes);
      bulk_g2s(base + sh.o_cst, Cst, (uint32_t)sh.cst_bytes, &bars.cst);
      issue_round(0);
    }
    // the compute warps' rows of X_1 (FP32), zero past p1 and past n1, loaded behind the copies
    const int q = warp & 3, wg = warp >> 2;
    const int c = 32 * q + lane;  // TMEM lane = row i1
    const bool rowok = c < n1;
    float x1[32];
#pragma unroll
    for (int j = 0; j < 32; ++j) x1[j] = (warp < 8 && rowok && j < p1) ? X1T[(int64_t)j * n1 + c] : 0.f;
    // X_3 entries of this CTA's slabs, [j3][k]
    for (int idx = ptid; idx < p3 * KQ; idx += nth) {
      const int j3 = idx / KQ, kk = idx - j3 * KQ;
      X3r[idx] = kk < kcta ? X3T[(int64_t)j3 * n3 + blockIdx.x + (int64_t)kk * gridDim.x] : 0.f;
    }
    for (int idx = ptid; idx < sh.kmax * p1 * K1; idx += nth) TaS[idx] = 0.f;
    named_sync(1, nth);
    // the rows j3 whose X_3 entries are not all zero for this CTA's slabs, in increasing order (a
    // zero row adds exactly nothing to the sums of the first H stage)
    if (warp == 0) {
      int cnt = 0;
      for (int j0 = 0; j0 < p3; j0 += 32) {
        const int j3 = j0 + lane;
        bool nz = false;
        if (j3 < p3)
          for (int kk = 0; kk < kcta; ++kk) nz |= X3r[j3 * KQ + kk] != 0.f;
        const unsigned m = __ballot_sync(0xffffffffu, nz);
        if (nz) rowlist[cnt + __popc(m & ((1u << lane) - 1u))] = j3;
        cnt += __popc(m);
      }
      if (lane == 0) nrows_s = cnt;
    }
    // first H stage: T_a(s_k, j2, j1) = sum_j3 X_3(s_k, j3) d(j3, j2, j1), in j3 order, R rows of
    // d per round (a bulk copy of their 16-byte multiple; the tail by plain loads)
    int rl = 0;  // first entry of rowlist not yet summed
    for (int rd = 0; rd < nround; ++rd) {
      const int j0 = rd * sh.R, rows = (j0 + sh.R < p3) ? sh.R : p3 - j0;
      const uint32_t bulk = (uint32_t)(((int64_t)rows * P21) / 4 * 16);
      if (rd > 0) {
        named_sync(1, nth);  // every thread is done with the previous round
        if (tid == 0) issue_round(rd);
      }
      for (int i = (int)(bulk / 4) + ptid; i < rows * P21; i += nth) stage[i] = D[(int64_t)j0 * P21 + i];
      if (!wait_for(&bars.stage, (uint32_t)(rd & 1), wait_ns)) atomicOr(&timed_out, 1);
      named_sync(1, nth);
      if (*(volatile int*)&timed_out) break;
      int re = rl;
      const int nr = nrows_s;
      while (re < nr && rowlist[re] < j0 + rows) ++re;
      // task = (one column n, 4 slabs k)
      const int nkg = (kcta + 3) / 4;
      for (int task = ptid; task < P21 * nkg; task += nth) {
        const int nn = task % P21, k0 = 4 * (task / P21);
        const int j2 = nn / p1, j1 = nn - j2 * p1;
        float a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = (k0 + r < kcta) ? TaS[((k0 + r) * p1 + j1) * K1 + j2] : 0.f;
#pragma unroll 4
        for (int t = rl; t < re; ++t) {
          const int j3 = rowlist[t];
          const float dv = stage[(j3 - j0) * P21 + nn];
          const float4 x4 = *reinterpret_cast<const float4*>(X3r + j3 * KQ + k0);
          a[0] = fmaf(x4.x, dv, a[0]);
          a[1] = fmaf(x4.y, dv, a[1]);
          a[2] = fmaf(x4.z, dv, a[2]);
          a[3] = fmaf(x4.w, dv, a[3]);
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (k0 + r < kcta) TaS[((k0 + r) * p1 + j1) * K1 + j2] = a[r];
      }
      rl = re;
    }
    // after a time-out the last staging copy may still be in flight: it lands before the area is
    // handed to the V ring
    if (tid == 0 && rounds_issued > 0)
      wait_for(&bars.stage, (uint32_t)((rounds_issued - 1) & 1), drain_ns);
    named_sync(1, nth);  // T_a complete; the staging area is free
    if (tid == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&bars.stage_free)) : "memory");

    const uint32_t x1b = sbase + (uint32_t)sh.o_xt1, x2tb = sbase + (uint32_t)sh.o_x2t,
                   x2b = sbase + (uint32_t)sh.o_x2, ptb = sbase + (uint32_t)sh.o_ptile;
    if (warp == kUmMmaWarp) {
      // ---------------------------------------------------------------- MMA3 issue (warp 8)
      if (lane == 0) {
        bool ok = !*(volatile int*)&timed_out && wait_for(&bars.cst, 0u, wait_ns);
        const uint32_t id3 = umma::idesc(64, (uint32_t)(PARTS * sh.N3), kType, kType, 0, 0);
        const uint32_t id3h = umma::idesc(64, (uint32_t)sh.N3, kType, kType, 0, 0);
        const uint64_t ad0 = umma::sdesc(x1b, 16, 1024, umma::kSwizzle128B);
        const uint64_t ad1 = umma::sdesc(x1b + (uint32_t)sh.xt1_part, 16, 1024, umma::kSwizzle128B);
        const uint64_t bd0 = umma::sdesc(ptb, 16, 1024, umma::kSwizzle128B);
        const uint32_t da = (uint32_t)(4096 >> 4), db = (uint32_t)(sh.ptile_atom >> 4);  // atom steps
        int committed = 0;
        for (int k = 0; k < kcta && ok; ++k) {
          const uint32_t par = (uint32_t)(k & 1);
          ok = wait_for(&bars.pt_ready, par, wait_ns);
          if (!ok) break;
          umma::fence_after_sync();
          // S_b^T = X_1^T P: A reads 64 rows j1 of the 32-row atoms (rows past p1 unused); in the
          // split form the first instruction takes B = [P_hi | P_lo] (hi hi' and hi lo'), the second
          // A = X_1 lo with B = P_hi
          for (int ka = 0; ka < sh.KA1; ++ka)
#pragma unroll
            for (int s4 = 0; s4 < 4; ++s4) {
              const uint64_t off = (uint64_t)(2 * s4);
              mma_ss<FORM>(tb + sh.c_sb, ad0 + ka * da + off, bd0 + ka * db + off, id3, (ka | s4) != 0);
              if (PARTS == 2) mma_ss<FORM>(tb + sh.c_sb, ad1 + ka * da + off, bd0 + ka * db + off, id3h, 1u);
            }
          umma::commit(&bars.sb_ready);
          ++committed;
        }
        if (!ok) atomicOr(&timed_out, 1);
        // every MMA issued has completed before the TMEM is released (the last commit covers all)
        if (committed > 0) wait_for(&bars.sb_ready, (uint32_t)((committed - 1) & 1), drain_ns);
      }
      __syncwarp();
    } else {
      // ---------------------------------------------------------------- compute warps 0-7
      const uint32_t lq = (uint32_t)(32 * q) << 16;
      const int half = sh.nchunk / 2;                 // chunks of this warpgroup
      const int ncw = n2 / 2;                         // i2 columns of this warpgroup
      const bool leader_warp = q == 3;                // issues this warpgroup's MMA1 and MMA2
      const bool issuer = leader_warp && lane == 0;
      const uint32_t pcol = sh.c_p + (uint32_t)wg * sh.pw;  // this warpgroup's partial P
      // MMA1 for this warpgroup's columns: eta^T(:, wg ncw .. + ncw) = T_b^T X_2^T
      const uint32_t id1 = umma::idesc(128, (uint32_t)ncw, kType, kType, 0, 0);
      const uint64_t b1h = umma::sdesc(x2tb + (uint32_t)(wg * ncw * 128), 16, 1024, umma::kSwizzle128B);
      const uint64_t b1l = umma::sdesc(x2tb + (uint32_t)sh.x2t_part + (uint32_t)(wg * ncw * 128), 16, 1024,
                                       umma::kSwizzle128B);
      const uint32_t d1 = tb + sh.c_eta + (uint32_t)(wg * ncw);
      auto mma1 = [&]() {
        for (int s = 0; s < K1 / (int)KS; ++s) {
          const uint64_t off = (uint64_t)(2 * s);  // 32 bytes of K
          mma_ts<FORM>(d1, tb + sh.c_tb + 8u * s, b1h + off, id1, s != 0);
          if (PARTS == 2) {
            mma_ts<FORM>(d1, tb + sh.c_tb + 8u * s, b1l + off, id1, 1u);
            mma_ts<FORM>(d1, tb + sh.c_tblo + 8u * s, b1h + off, id1, 1u);
          }
        }
      };
      // MMA2 for one chunk (kUmRows columns i2 = one or two K steps): P_g (+)= r^T X_2
      const uint32_t id2 = umma::idesc(128, (uint32_t)(PARTS * sh.N2), kType, kType, 0, 0);
      const uint32_t id2h = umma::idesc(128, (uint32_t)sh.N2, kType, kType, 0, 0);
      const uint64_t b2 = umma::sdesc(x2b, 16, 1024, umma::kSwizzle128B);
      auto mma2 = [&](int ch, bool first) {
        for (int u = 0; u < kUmRows / (int)KS; ++u) {
          const int s = ch * (kUmRows / (int)KS) + u;  // global K step over i2
          const uint64_t bd = b2 + (uint64_t)(((s >> 2) * sh.x2_atom + (s & 3) * 32) >> 4);
          const uint32_t ar = FORM == kFormBF16 ? tb + sh.c_rb + 8u * s : tb + sh.c_eta + 8u * s;
          mma_ts<FORM>(tb + pcol, ar, bd, id2, (first && u == 0) ? 0u : 1u);
          if (PARTS == 2) mma_ts<FORM>(tb + pcol, tb + sh.c_rlo + 8u * s, bd, id2h, 1u);
        }
      };
      bool ok = __all_sync(0xffffffffu, !*(volatile int*)&timed_out) != 0;
      // MMA0 on the compute warps: T_b^T(c, j2) = sum_j1 X_1(c, j1) T_a(k, j2, j1), written as the
      // A operand of MMA1 (warpgroup wg takes the 8- or 16-column groups wg, wg + 2, ...); each
      // thread keeps one independent FMA chain per column of its group
      auto mma0 = [&](int kk) {
        constexpr int GW = FORM == kFormBF16 ? 16 : 8;  // j2 per group (8 TMEM columns)
        for (int g0 = wg; g0 < K1 / GW; g0 += 2) {
          float acc[GW];
#pragma unroll
          for (int u = 0; u < GW; ++u) acc[u] = 0.f;
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            if (j < p1) {
              const float4* t4 = reinterpret_cast<const float4*>(TaS + ((int64_t)kk * p1 + j) * K1 + g0 * GW);
#pragma unroll
              for (int v = 0; v < GW / 4; ++v) {
                const float4 t = t4[v];
                acc[4 * v + 0] = fmaf(x1[j], t.x, acc[4 * v + 0]);
                acc[4 * v + 1] = fmaf(x1[j], t.y, acc[4 * v + 1]);
                acc[4 * v + 2] = fmaf(x1[j], t.z, acc[4 * v + 2]);
                acc[4 * v + 3] = fmaf(x1[j], t.w, acc[4 * v + 3]);
              }
            }
          }
          uint32_t hi[8], lo[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            if (FORM == kFormBF16) {
              hi[u] = pack_bf16(acc[2 * u], acc[(2 * u + 1) % GW]);
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
      // the leader issues MMA1 of slab kk once every warp has written T_b^T (tb_ready) and the
      // constant tiles have landed; its commit tells the warpgroup that eta is in TMEM
      auto issue_mma1 = [&](int kk) -> bool {
        bool lok = true;
        if (issuer) {
          lok = wait_for(&bars.tb_ready, (uint32_t)(kk & 1), wait_ns) && (kk > 0 || wait_for(&bars.cst, 0u, wait_ns));
          if (lok) {
            umma::fence_after_sync();
            mma1();
            umma::commit(&bars.eta_ready[wg]);
          }
        }
        __syncwarp();
        return __all_sync(0xffffffffu, lok) != 0;
      };
      int committed = 0;  // this issuer's commits (eta_ready and p_ready alternate: 2 per slab)
      if (ok) mma0(0);
      if (ok && leader_warp) ok = issue_mma1(0);
      if (issuer && ok) committed = 1;
      // Every warp of a warpgroup passes that group's named barrier (2 + wg) exactly once per chunk
      // until the group leaves its loop together: the barrier ANDs the warps' status, and it is the
      // only place a warp leaves the loop.  Elsewhere a wait that runs out only clears `ok`, which
      // skips the remaining work and reaches the next chunk barrier.
      for (int k = 0; k < kcta; ++k) {
        const uint32_t par = (uint32_t)(k & 1);
        // ---- r = V (.) eta over this warpgroup's chunks; MMA2 of each chunk as soon as it is in TMEM
        ok = ok && warp_wait(&bars.eta_ready[wg], par, wait_ns);
        umma::fence_after_sync();
        // P_g is overwritten by this slab's MMA2: every warp has read the last slab's (pt_ready)
        if (leader_warp && k > 0) ok = ok && warp_wait(&bars.pt_ready, (uint32_t)((k - 1) & 1), wait_ns);
        for (int i = 0; i < half; ++i) {
          const int ch = wg * half + i;
          const int g = k * sh.nchunk + ch, slot = g % sh.nslot;
          const bool okc = ok && warp_wait(&bars.full[slot], (uint32_t)((g / sh.nslot) & 1), wait_ns);
          if (okc) {
            const TV* vs = reinterpret_cast<const TV*>(base + sh.o_ring + (int64_t)slot * sh.slot_bytes);
            uint32_t e[16];
            umma::ld_x16(tb + lq + sh.c_eta + (uint32_t)(kUmRows * ch), e);
            float v[16];
#pragma unroll
            for (int u = 0; u < 16; ++u) v[u] = rowok ? vload<TV>(vs + u * n1 + c) : 0.f;
            umma::wait_ld();
            if (FORM == kFormBF16) {
              uint32_t pk[8];
#pragma unroll
              for (int u = 0; u < 8; ++u)
                pk[u] = pack_bf16(v[2 * u] * __uint_as_float(e[2 * u]), v[2 * u + 1] * __uint_as_float(e[2 * u + 1]));
              umma::st_x8(tb + lq + sh.c_rb + (uint32_t)(8 * ch), pk);
            } else {
              uint32_t hi[16], lo[16];
#pragma unroll
              for (int u = 0; u < 16; ++u) {
                const float r = v[u] * __uint_as_float(e[u]);
                hi[u] = rna_tf32(r);
                lo[u] = rna_tf32(r - __uint_as_float(hi[u]));
              }
              umma::st_x16(tb + lq + sh.c_eta + (uint32_t)(kUmRows * ch), hi);
              if (PARTS == 2) umma::st_x16(tb + lq + sh.c_rlo + (uint32_t)(kUmRows * ch), lo);
            }
            warp_arrive(&bars.empty[slot]);
            umma::wait_st();
          }
          umma::fence_before_sync();
          // the chunk's r is in TMEM for all 128 rows
          ok = named_sync_and(2 + wg, 128, okc);
          if (!ok) break;
          if (issuer) {
            umma::fence_after_sync();
            mma2(ch, i == 0);
            if (i == half - 1) umma::commit(&bars.p_ready[wg]);
          }
          __syncwarp();
        }
        if (!ok) break;  // the whole warpgroup (the barrier's AND)
        if (issuer) ++committed;
        // ---- MMA0 of the next slab (T_b^T is free once both warpgroups' MMA1 of this slab ran)
        if (k + 1 < kcta) {
          ok = ok && warp_wait(&bars.eta_ready[wg ^ 1], par, wait_ns);
          if (ok) mma0(k + 1);
          if (ok && leader_warp) {
            ok = issue_mma1(k + 1);
            if (ok && issuer) ++committed;
          }
        }
        // ---- P = P_0 + P_1 from TMEM into the B operand of MMA3 (K-major rows j2, K = c; warp q
        // writes K atom q of 32 rows c (TF32) or half of atom q / 2 (BF16); the split form stores
        // hi in rows j2 and lo in rows N3 + j2 of the atom).  The tile is free once MMA3 of the last
        // slab ran (sb_ready), whose S_b warps 0 and 1 write out first.
        ok = ok && warp_wait(&bars.p_ready[0], par, wait_ns) && warp_wait(&bars.p_ready[1], par, wait_ns);
        if (k > 0) ok = ok && warp_wait(&bars.sb_ready, (uint32_t)((k - 1) & 1), wait_ns);
        umma::fence_after_sync();
        auto write_sb = [&](int kk) {  // S_b^T (M = 64 layout: rows 0-15 in lanes 0-15 of warps 0, 1)
          const int j1 = 16 * warp + lane;
          float* out = Sb + (int64_t)((int)blockIdx.x + kk * (int)gridDim.x) * P21;
          for (int g0 = 0; g0 < sh.N3 / 8; ++g0) {
            uint32_t sv[8], sl[8];
            umma::ld_x8(tb + lq + sh.c_sb + 8u * g0, sv);
            if (PARTS == 2) umma::ld_x8(tb + lq + sh.c_sb + (uint32_t)sh.N3 + 8u * g0, sl);
            umma::wait_ld();
            if (lane < 16 && j1 < p1) {
#pragma unroll
              for (int u = 0; u < 8; ++u) {
                const int j2 = 8 * g0 + u;
                const float x = PARTS == 2 ? __uint_as_float(sv[u]) + __uint_as_float(sl[u]) : __uint_as_float(sv[u]);
                if (j2 < p2) out[j2 * p1 + j1] = x;
              }
            }
          }
        };
        if (ok) {
          if (k > 0 && warp < 2) write_sb(k - 1);
          for (int g0 = wg; g0 < sh.N3 / 8; g0 += 2) {
            uint32_t a0[8], a1[8], b0[8], b1[8];
            umma::ld_x8(tb + lq + sh.c_p + 8u * g0, a0);
            umma::ld_x8(tb + lq + sh.c_p + sh.pw + 8u * g0, a1);
            if (PARTS == 2) {
              umma::ld_x8(tb + lq + sh.c_p + (uint32_t)sh.N2 + 8u * g0, b0);
              umma::ld_x8(tb + lq + sh.c_p + sh.pw + (uint32_t)sh.N2 + 8u * g0, b1);
            }
            umma::wait_ld();
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int j2 = 8 * g0 + u;
              float x = __uint_as_float(a0[u]) + __uint_as_float(a1[u]);
              if (PARTS == 2) x += __uint_as_float(b0[u]) + __uint_as_float(b1[u]);
              if (FORM == kFormBF16) {
                if ((c >> 6) >= sh.KA1) continue;  // rows past the last K atom: MMA3 does not read them
                const uint32_t off =
                    (uint32_t)((c >> 6) * sh.ptile_atom) + umma::sw128_k2((uint32_t)j2, (uint32_t)(c & 63));
                *reinterpret_cast<__nv_bfloat16*>(base + sh.o_ptile + off) = __float2bfloat16_rn(x);
              } else {
                if (q >= sh.KA1) continue;
                const uint32_t off = (uint32_t)(q * sh.ptile_atom);
                const uint32_t h = rna_tf32(x);
                *reinterpret_cast<uint32_t*>(base + sh.o_ptile + off + umma::sw128_k4((uint32_t)j2, (uint32_t)lane)) = h;
                if (PARTS == 2)
                  *reinterpret_cast<uint32_t*>(base + sh.o_ptile + off +
                                               umma::sw128_k4((uint32_t)(sh.N3 + j2), (uint32_t)lane)) =
                      rna_tf32(x - __uint_as_float(h));
              }
            }
          }
          fence_proxy_async();
          warp_arrive(&bars.pt_ready);
          if (k == kcta - 1 && warp < 2) {
            ok = warp_wait(&bars.sb_ready, par, wait_ns);
            umma::fence_after_sync();
            if (ok) write_sb(k);
          }
        }
      }
      if (!ok) atomicOr(&timed_out, 1);
      // this issuer's MMAs have completed before the TMEM is released: its last commit was on
      // eta_ready (slab k + 1's MMA1) or p_ready (slab k's last chunk); each covers all earlier ones
      if (issuer && committed > 0) {
        wait_for(&bars.eta_ready[wg], (uint32_t)(((committed + 1) / 2 - 1) & 1), drain_ns);
        if (committed >= 2) wait_for(&bars.p_ready[wg], (uint32_t)((committed / 2 - 1) & 1), drain_ns);
      }
      umma::fence_before_sync();
      // the constant block's copy has landed before the CTA leaves (at once in a normal run)
      if (tid == 0) wait_for(&bars.cst, 0u, drain_ns);
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
//   XT1: MMA3's A, rows j1 (32 per atom), K = i1 (KA1 atoms of 4 KB), parts [hi][lo]
//   X2T: MMA1's B, rows i2 (n2), K = j2 (one atom row), parts [hi][lo]
//   X2 : MMA2's B, rows j2, K = i2: KA2 atoms, each [hi rows 0 .. N2-1][lo rows N2 .. 2 N2 - 1]
__global__ void umma_const_kernel(UmShape sh, int form, const float* __restrict__ X1T,
                                  const float* __restrict__ X2T, unsigned char* __restrict__ out) {
  const int esz = form == kFormBF16 ? 2 : 4;
  const int epr = 128 / esz;  // elements per 128-byte row
  const int64_t nel = sh.cst_bytes / esz;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < nel; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t b = e * esz;  // byte offset in the block
    int part = 0;
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
      int atom, row, k;
      inv(b - part * sh.xt1_part, 4096, atom, row, k);
      const int j1 = row, i1 = atom * epr + k;
      if (j1 < sh.p1 && i1 < sh.n1) v = X1T[(int64_t)j1 * sh.n1 + i1];
    } else if (b < sh.o_x2 - sh.o_xt1) {  // X2T
      const int64_t bb = b - (sh.o_x2t - sh.o_xt1);
      part = (int)(bb / sh.x2t_part);
      int atom, row, k;
      inv(bb - part * sh.x2t_part, (int64_t)sh.n2 * 128, atom, row, k);
      const int i2 = row, j2 = k;
      if (j2 < sh.p2) v = X2T[(int64_t)j2 * sh.n2 + i2];
    } else {  // X2
      int atom, row, k;
      inv(b - (sh.o_x2 - sh.o_xt1), sh.x2_atom, atom, row, k);
      part = row / sh.N2;
      const int j2 = row - part * sh.N2, i2 = atom * epr + k;
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

size_t g_um_budget = 227 * 1024 - 2048;

// The kernel's plan for a shape and form; false outside its domain.
bool um_configure(int n1, int n2, int n3, int p1, int p2, int p3, int grid, int form, bool v_bf16, UmShape& s) {
  if (!(form == kFormTF32 || form == kForm3x || form == kFormBF16)) return false;
  if (v_bf16 && form != kFormBF16) return false;
  const int vesz = v_bf16 ? 2 : 4;  // bytes of a V element (the ring slots hold V as it is stored)
  if (n1 < 4 || n1 > 128 || n1 % (form == kFormBF16 ? 8 : 4) != 0 || n2 < 32 || n2 % 32 != 0 || n3 < 1 ||
      p1 < 1 || p1 > 32 || p2 < 1 || p2 > 32 || p3 < 1 || grid < 1)
    return false;
  const int parts = form == kForm3x ? 2 : 1;
  const int esz = um_esz(form);
  if (n2 > (form == kForm3x ? 128 : 256)) return false;
  s.n1 = n1; s.n2 = n2; s.n3 = n3; s.p1 = p1; s.p2 = p2; s.p3 = p3;
  s.parts = parts;
  s.K1 = form == kFormBF16 ? (int)up(p2, 16) : (int)up(p2, 8);
  s.N2 = (int)up(p2, 16);
  s.N3 = (int)up(p2, 8);
  const int epr = 128 / esz;
  s.KA1 = (n1 + epr - 1) / epr;
  s.KA2 = (n2 + epr - 1) / epr;
  s.nchunk = n2 / kUmRows;
  s.kmax = (n3 + grid - 1) / grid;
  // constant block
  s.xt1_part = (int64_t)s.KA1 * 4096;
  s.x2t_part = (int64_t)n2 * 128;
  s.x2_atom = (int64_t)parts * s.N2 * 128;
  int64_t o = 0;
  s.o_cst = o;
  s.o_xt1 = o;
  o += parts * s.xt1_part;
  s.o_x2t = o;
  o += parts * s.x2t_part;
  s.o_x2 = o;
  o += (int64_t)s.KA2 * s.x2_atom;
  s.cst_bytes = o - s.o_cst;
  // MMA3 reads 64 rows of each 32-row XT1 atom: the last atom's reads run 4 KB past the XT1 parts,
  // into the X2T tile (n2 >= 32 rows of 128 bytes)
  o = up(o, 1024);
  // the V ring, then the P tile; d is staged for the first H stage in the last bytes of the two
  // (so that the first V chunks, in the first slots, can be in flight while T_a is formed)
  s.o_ring = o;
  s.slot_bytes = up((int64_t)kUmRows * n1 * vesz, 1024);
  s.ptile_atom = (int64_t)parts * s.N3 * 128;
  const int64_t ptile_bytes = up((int64_t)s.KA1 * s.ptile_atom, 1024);
  const int KQ = (s.kmax + 3) / 4 * 4;
  const int64_t tas_bytes = up((int64_t)s.kmax * p1 * s.K1 * 4, 16);
  const int64_t tail = ptile_bytes + tas_bytes + up((int64_t)p3 * KQ * 4, 16) + up((int64_t)p3 * 4, 16);
  const int64_t room = (int64_t)g_um_budget - 1024 - o - tail;
  int slots = (int)(room / s.slot_bytes);
  if (slots > kUmMaxSlots) slots = kUmMaxSlots;
  if (slots > 3 * s.nchunk) slots = 3 * s.nchunk;
  if (slots < 2) return false;
  s.nslot = slots;
  o += (int64_t)slots * s.slot_bytes;
  s.o_ptile = o;
  o += ptile_bytes;
  const int64_t stage_end = o, stage_cap = o - s.o_ring;
  s.o_tas = o;
  o += tas_bytes;
  s.o_x3r = o;
  o += up((int64_t)p3 * KQ * 4, 16);
  s.o_rows = o;
  o += up((int64_t)p3 * 4, 16);
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
  // TMEM columns (each region starts on a multiple of 32): eta (r in place for TF32 forms), r lo
  // (3xTF32) or packed r (BF16), T_b^T hi and lo, the two warpgroups' partial P, S_b
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
  s.pw = (uint32_t)up(parts * s.N2, 32);
  col += 2 * s.pw;
  s.c_sb = col;
  col += (uint32_t)up(parts * s.N3, 32);
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

// V as a 2-D tensor (n1 columns, n2 n3 rows) with boxes of kUmRows rows (one ring slot), no swizzle.
bool um_encode_v(CUtensorMap* m, const void* V, int n1, int64_t rows, bool bf16) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = um_encode();
  if (fn == nullptr) return false;
  const int esz = bf16 ? 2 : 4;
  const cuuint64_t dims[2] = {(cuuint64_t)n1, (cuuint64_t)rows};
  const cuuint64_t strides[1] = {(cuuint64_t)n1 * esz};
  const cuuint32_t box[2] = {(cuuint32_t)n1, (cuuint32_t)kUmRows};
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
