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
//                  (the one transposition of the chain: it contracts the lane index c), M = 128
//                  so that row j1 of S_b^T sits in TMEM lane j1
// and S_b (p2 x p1) is written to global memory for the mode-3 adjoint.  Only eta's 128 x n2 tile
// is ever formed, and only in TMEM.
//
// Arithmetic forms: FORM 1 (TF32 operands rounded to nearest, FP32 accumulation), FORM 3
// (3xTF32: every operand split into hi = tf32(x) and lo = tf32(x - hi); each product as
// hi hi' + hi lo' + lo hi', about FP32 accuracy), FORM 16 (BF16 operands rounded to nearest, FP32
// accumulation).  V is read as FP32, or as BF16 (TV) by the BF16 fit path.
//
// Issue.  A tcgen05.mma of the small N used here costs its issuing thread about 100 cycles
// whatever N is (measured on this GPU), while threads of different warps issuing at once overlap;
// so the MMAs are issued by three threads of three warps that do nothing else, and the operand
// splits of the 3xTF32 form share instructions where an operand is common: the hi and lo parts of
// the constant operand sit side by side along N (hi hi' and hi lo' in one instruction of twice the
// N), leaving hi' lo as the third.
//
// Warp roles (384 threads).  Warps 0-7 compute in two warpgroups; warp w reaches TMEM lanes
// 32 (w mod 4) .. + 31 (rows c = 32 (w mod 4) + lane).  Warpgroup g owns the i2 columns
// [g n2/2, (g+1) n2/2) and its issuer warp 10 + g (lane 0) issues MMA1 for those columns and,
// chunk by chunk as the warpgroup signals that r is in TMEM, MMA2 over those columns into the
// group's own partial P (summed when P is read); one thread issuing both keeps every reuse of the
// group's TMEM columns in issue order.  Warp 8 issues MMA3, writes S_b out and owns the TMEM
// allocation; warp 9 streams V by TMA through a ring of 16-row chunks.  The roles meet only at
// mbarriers; every wait is bounded (a kernel parameter, default 2 s) and a wait that runs out sets
// an error flag, after which every role leaves its loop, the copies and MMAs already issued are
// waited for (bounded by at least 2 s), the TMEM is freed and the CTA exits.

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

constexpr int kUmThreads = 384;
constexpr int kUmMmaWarp = 8;       // MMA3, S_b out, TMEM owner
constexpr int kUmTmaWarp = 9;       // V producer
constexpr int kUmIssWarp = 10;      // MMA1 / MMA2 issuers of warpgroups 0 and 1: warps 10, 11
constexpr int kUmRows = 16;         // rows i2 of a V chunk (one 16-column TMEM load per thread)
constexpr uint32_t kUmTmemCols = 512;
constexpr int kUmMaxSlots = 24;
constexpr int kUmMaxHalf = 8;       // chunks of a warpgroup per slab, at most (n2 <= 256)
constexpr uint64_t kDrainNs = 2000000000ull;

enum : int { kFormTF32 = 1, kForm3x = 3, kFormBF16 = 16 };

// Shape and shared-memory plan (byte offsets from the 1 KB aligned base).
struct UmShape {
  int n1, n2, n3, p1, p2, p3;
  int K1;      // K of MMA1 (j2, padded): multiple of 8 (TF32) or 16 (BF16)
  int N2;      // N of MMA2 per part (j2, padded to 16)
  int N3;      // N of MMA3 per part (j2, padded to 8 in the split form, else 16)
  int P1P;     // rows j1 of a slab's T_a in shared memory (p1 padded to 4 with zero rows)
  int KA1;     // K atoms of MMA3 (i1): 32 (TF32) or 64 (BF16) elements each
  int KA2;     // K atoms of MMA2 (i2)
  int nchunk;  // V chunks of kUmRows rows i2 per slab (each warpgroup takes half)
  int nslot;   // V ring slots
  int kmax;    // slabs per CTA, at most
  int R;       // rows of d per staging round
  int parts;   // 2 for the 3xTF32 form (hi, lo), else 1
  int64_t o_cst, o_xt1, o_x2t, o_x2, cst_bytes;  // constant block: [XT1 parts][X2T parts][X2]
                                                 // (copied in two pieces: X2T and X2 first)
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
// x rounded to TF32 (10 mantissa bits), to nearest with ties away from zero, on the bit pattern:
// half a TF32 unit (bit 12) is added to the magnitude and the 13 low bits cleared; a carry moves
// into the exponent as rounding requires (finite inputs; integer operations at full rate)
__device__ __forceinline__ uint32_t rna_tf32(float x) {
  return (__float_as_uint(x) + 0x1000u) & 0xffffe000u;
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
// Between checks of the clock the thread sleeps in the barrier's wait (up to kSleepNs), so that
// waiting roles take no issue slots or shared-memory bandwidth from the working ones.
constexpr uint32_t kSleepNs = 1000;
__device__ __forceinline__ bool wait_for(uint64_t* bar, uint32_t parity, uint64_t limit_ns) {
  if (mbar_try_wait(bar, parity)) return true;
  if (limit_ns == 0) return false;
  const uint64_t t0 = globaltimer_ns();
  while (true) {
    if (mbar_try_wait_sleep(bar, parity, kSleepNs)) return true;
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
  uint64_t cst, cst1, stage, stage_free;  // cst: X2T and X2 tiles; cst1: XT1 tiles
  uint64_t tb_ready, pt_ready, sb_ready;
  uint64_t eta_ready[2], p_ready[2];      // per warpgroup
  uint64_t r_ready[2][kUmMaxHalf];        // per warpgroup and chunk of a slab: r is in TMEM
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

// The FMA core of MMA0 for one thread (row c): acc[4 v + u] += sum_j1 X_1(c, j1) T(j1, 4 v + u)
// over NV groups of four columns; the rows j1 go four at a time (rows past p1 are zero in T), the
// four X_1 values through L1 and the 4 NV loads of T issued together.  A rolled loop: the kernel's
// roles run different code at once, so its hot loops are kept small for the instruction cache.
template <int NV>
__device__ __forceinline__ void mma0_fma(const float* __restrict__ tk, int K1, int p1, const float* __restrict__ x1c,
                                         int n1, bool rowok, float (&acc)[16]) {
#pragma unroll 1
  for (int j0 = 0; j0 < p1; j0 += 4) {
    float x[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) x[u] = (rowok && j0 + u < p1) ? __ldg(x1c + (int64_t)(j0 + u) * n1) : 0.f;
    float4 t[4][NV];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v) t[u][v] = reinterpret_cast<const float4*>(tk + (j0 + u) * K1)[v];
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int v = 0; v < NV; ++v) {
        acc[4 * v + 0] = fmaf(x[u], t[u][v].x, acc[4 * v + 0]);
        acc[4 * v + 1] = fmaf(x[u], t[u][v].y, acc[4 * v + 1]);
        acc[4 * v + 2] = fmaf(x[u], t[u][v].z, acc[4 * v + 2]);
        acc[4 * v + 3] = fmaf(x[u], t[u][v].w, acc[4 * v + 3]);
      }
  }
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
  float* const TaS = reinterpret_cast<float*>(base + sh.o_tas);   // [kmax][P1P][K1]: T_a(k, j2, j1) at [k][j1][j2]
  float* const X3r = reinterpret_cast<float*>(base + sh.o_x3r);   // [p3][KQ]
  int* const rowlist = reinterpret_cast<int*>(base + sh.o_rows);  // rows j3 with a nonzero X_3 entry
  float* const stage = reinterpret_cast<float*>(base + sh.o_stage);
  const int KQ = (sh.kmax + 3) / 4 * 4;
  const int P1P = sh.P1P;
  const uint64_t drain_ns = wait_ns > kDrainNs ? wait_ns : kDrainNs;
  const int half = sh.nchunk / 2;  // chunks of a warpgroup per slab

  // ---------------------------------------------------------------- set-up
  if (tid == 0) {
    timed_out = 0;
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmapV)) : "memory");
    for (int s = 0; s < sh.nslot; ++s) {
      mbar_init(&bars.full[s], 1);
      mbar_init(&bars.empty[s], 4);  // the four warps of the warpgroup that consumes the chunk
    }
    mbar_init(&bars.cst, 1);
    mbar_init(&bars.cst1, 1);
    mbar_init(&bars.stage, 1);
    mbar_init(&bars.stage_free, 1);
    mbar_init(&bars.tb_ready, 8);
    mbar_init(&bars.pt_ready, 8);
    mbar_init(&bars.sb_ready, 1);
    for (int g = 0; g < 2; ++g) {
      mbar_init(&bars.eta_ready[g], 1);
      mbar_init(&bars.p_ready[g], 1);
      for (int i = 0; i < kUmMaxHalf; ++i) mbar_init(&bars.r_ready[g][i], 4);
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
    // ---------------------------------------------------------------- prologue (every warp but 9)
    const int nth = kUmThreads - 32;                     // 352 threads
    const int ptid = warp < kUmTmaWarp ? tid : tid - 32;
    int rounds_issued = 0;                               // thread 0's count of staging copies
    auto issue_round = [&](int rd) {                     // thread 0: R rows of d (16-byte multiple)
      const int j0 = rd * sh.R, rows = (j0 + sh.R < p3) ? sh.R : p3 - j0;
      const uint32_t bulk = (uint32_t)(((int64_t)rows * P21) / 4 * 16);
      fence_proxy_async();
      mbar_expect_tx(&bars.stage, bulk);
      if (bulk > 0) bulk_g2s(stage, D + (int64_t)j0 * P21, bulk, &bars.stage);
      ++rounds_issued;
    };
    if (tid == 0) {  // the operands of MMA1 and MMA2 first, X_1's tiles (MMA3 needs them last) next
      const uint32_t b23 = (uint32_t)(sh.cst_bytes - sh.o_x2t);
      mbar_expect_tx(&bars.cst, b23);
      bulk_g2s(base + sh.o_cst + sh.o_x2t, Cst + sh.o_x2t, b23, &bars.cst);
      mbar_expect_tx(&bars.cst1, (uint32_t)sh.o_x2t);
      bulk_g2s(base + sh.o_cst, Cst, (uint32_t)sh.o_x2t, &bars.cst1);
    }
    // X_3 entries of this CTA's slabs, [j3][k]
    for (int idx = ptid; idx < p3 * KQ; idx += nth) {
      const int j3 = idx / KQ, kk = idx - j3 * KQ;
      X3r[idx] = kk < kcta ? X3T[(int64_t)j3 * n3 + blockIdx.x + (int64_t)kk * gridDim.x] : 0.f;
    }
    // d and S_b belong to the preceding kernels of the fit loop: with a programmatic dependent
    // launch everything above may overlap them, nothing below
    griddep_wait();
    if (tid == 0) issue_round(0);
    // T_a starts at zero, rows j1 >= p1 stay zero (MMA0 reads them in groups of four), and the
    // slack after it is finite
    for (int idx = ptid; idx < sh.kmax * P1P * K1 + 16; idx += nth) TaS[idx] = 0.f;
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
      // one decision for all the threads (the flag may be raised by the producer at any time)
      if (!named_sync_and(1, nth, !*(volatile int*)&timed_out)) break;
      int re = rl;
      const int nr = nrows_s;
      while (re < nr && rowlist[re] < j0 + rows) ++re;
      // task = (one column n, 4 slabs k); the rows are taken eight at a time with their loads
      // issued together (past the last row the d value is zero, which adds exactly nothing)
      const int nkg = (kcta + 3) / 4;
      for (int task = ptid; task < P21 * nkg; task += nth) {
        const int nn = task % P21, k0 = 4 * (task / P21);
        const int j2 = nn / p1, j1 = nn - j2 * p1;
        float a[4];
#pragma unroll
        for (int r = 0; r < 4; ++r) a[r] = (k0 + r < kcta) ? TaS[((k0 + r) * P1P + j1) * K1 + j2] : 0.f;
        for (int t0 = rl; t0 < re; t0 += 8) {
          int jr[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) jr[u] = rowlist[t0 + u < re ? t0 + u : re - 1];
          float dv[8];
          float4 xv[8];
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            dv[u] = t0 + u < re ? stage[(jr[u] - j0) * P21 + nn] : 0.f;
            xv[u] = *reinterpret_cast<const float4*>(X3r + jr[u] * KQ + k0);
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            a[0] = fmaf(xv[u].x, dv[u], a[0]);
            a[1] = fmaf(xv[u].y, dv[u], a[1]);
            a[2] = fmaf(xv[u].z, dv[u], a[2]);
            a[3] = fmaf(xv[u].w, dv[u], a[3]);
          }
        }
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (k0 + r < kcta) TaS[((k0 + r) * P1P + j1) * K1 + j2] = a[r];
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
      // ---------------------------------------------------------------- MMA3 and S_b (warp 8)
      // S_b^T = X_1^T P with M = 128: A reads 128 rows j1 from each 32-row K atom of XT1 (the rows
      // past the atom belong to the next atoms or the tiles after them; their outputs, TMEM lanes
      // 32 .. 127, are never read).  In the split form both instructions take B = [P_hi | P_lo]:
      // X_1 hi with it gives hi hi' and hi lo', X_1 lo gives lo hi' (and lo lo', a smaller term).
      const uint32_t id3 = umma::idesc(128, (uint32_t)(PARTS * sh.N3), kType, kType, 0, 0);
      const uint64_t ad0 = umma::sdesc(x1b, 16, 1024, umma::kSwizzle128B);
      const uint64_t ad1 = umma::sdesc(x1b + (uint32_t)sh.xt1_part, 16, 1024, umma::kSwizzle128B);
      const uint64_t bd0 = umma::sdesc(ptb, 16, 1024, umma::kSwizzle128B);
      const uint32_t da = (uint32_t)(4096 >> 4), db = (uint32_t)(sh.ptile_atom >> 4);  // atom steps
      int committed = 0;
      bool ok = true;
      if (lane == 0) ok = !*(volatile int*)&timed_out && wait_for(&bars.cst1, 0u, wait_ns);
      ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
      for (int k = 0; k < kcta && ok; ++k) {
        const uint32_t par = (uint32_t)(k & 1);
        if (lane == 0) {
          ok = wait_for(&bars.pt_ready, par, wait_ns);
          if (ok) {
            umma::fence_after_sync();
            for (int ka = 0; ka < sh.KA1; ++ka)
#pragma unroll
              for (int s4 = 0; s4 < 4; ++s4) {
                const uint64_t off = (uint64_t)(2 * s4);
                mma_ss<FORM>(tb + sh.c_sb, ad0 + ka * da + off, bd0 + ka * db + off, id3, (ka | s4) != 0);
                if (PARTS == 2) mma_ss<FORM>(tb + sh.c_sb, ad1 + ka * da + off, bd0 + ka * db + off, id3, 1u);
              }
            umma::commit(&bars.sb_ready);
            ++committed;
          }
        }
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (!ok) break;
        ok = warp_wait(&bars.sb_ready, par, wait_ns);
        if (!ok) break;
        umma::fence_after_sync();
        // row j1 of S_b^T in lane j1; S_b(s, j2, j1) is stored with j1 fastest
        float* out = Sb + (int64_t)((int)blockIdx.x + k * (int)gridDim.x) * P21;
        for (int g0 = 0; g0 < sh.N3 / 8; ++g0) {
          uint32_t sv[8], sl[8];
          umma::ld_x8(tb + sh.c_sb + 8u * g0, sv);
          if (PARTS == 2) umma::ld_x8(tb + sh.c_sb + (uint32_t)sh.N3 + 8u * g0, sl);
          umma::wait_ld();
          umma::ld_done(sv);
          if (PARTS == 2) umma::ld_done(sl);
          if (lane < p1) {
#pragma unroll
            for (int u = 0; u < 8; ++u) {
              const int j2 = 8 * g0 + u;
              const float x = PARTS == 2 ? __uint_as_float(sv[u]) + __uint_as_float(sl[u]) : __uint_as_float(sv[u]);
              if (j2 < p2) out[j2 * p1 + lane] = x;
            }
          }
        }
      }
      if (!ok) atomicOr(&timed_out, 1);
      // every MMA issued has completed before the TMEM is released (the last commit covers all)
      if (lane == 0 && committed > 0) wait_for(&bars.sb_ready, (uint32_t)((committed - 1) & 1), drain_ns);
      __syncwarp();
    } else if (warp >= kUmIssWarp) {
      // ---------------------------------------------------------------- MMA1 / MMA2 issue (warps 10, 11)
      const int g = warp - kUmIssWarp;  // the warpgroup served
      if (lane == 0) {
        const int ncw = n2 / 2;         // i2 columns of the warpgroup
        // MMA1: eta^T(:, g ncw .. + ncw) = T_b^T X_2^T
        const uint32_t id1 = umma::idesc(128, (uint32_t)ncw, kType, kType, 0, 0);
        const uint64_t b1h = umma::sdesc(x2tb + (uint32_t)(g * ncw * 128), 16, 1024, umma::kSwizzle128B);
        const uint64_t b1l = umma::sdesc(x2tb + (uint32_t)sh.x2t_part + (uint32_t)(g * ncw * 128), 16, 1024,
                                         umma::kSwizzle128B);
        const uint32_t d1 = tb + sh.c_eta + (uint32_t)(g * ncw);
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
        const uint32_t pcol = tb + sh.c_p + (uint32_t)g * sh.pw;
        auto mma2 = [&](int ch, bool first) {
          for (int u = 0; u < kUmRows / (int)KS; ++u) {
            const int s = ch * (kUmRows / (int)KS) + u;  // global K step over i2
            const uint64_t bd = b2 + (uint64_t)(((s >> 2) * sh.x2_atom + (s & 3) * 32) >> 4);
            const uint32_t ar = FORM == kFormBF16 ? tb + sh.c_rb + 8u * s : tb + sh.c_eta + 8u * s;
            mma_ts<FORM>(pcol, ar, bd, id2, (first && u == 0) ? 0u : 1u);
            if (PARTS == 2) mma_ts<FORM>(pcol, tb + sh.c_rlo + 8u * s, bd, id2h, 1u);
          }
        };
        int ne = 0, np = 0;  // commits on eta_ready[g] and p_ready[g]
        bool ok = !*(volatile int*)&timed_out && wait_for(&bars.cst, 0u, wait_ns) &&
                  wait_for(&bars.tb_ready, 0u, wait_ns);
        if (ok) {
          umma::fence_after_sync();
          mma1();
          umma::commit(&bars.eta_ready[g]);
          ++ne;
        }
        for (int k = 0; k < kcta && ok; ++k) {
          for (int i = 0; i < half && ok; ++i) {
            ok = wait_for(&bars.r_ready[g][i], (uint32_t)(k & 1), wait_ns);
            // P_g is overwritten by this slab's first MMA2: every compute warp has read the last
            // slab's (pt_ready)
            if (ok && i == 0 && k > 0) ok = wait_for(&bars.pt_ready, (uint32_t)((k - 1) & 1), wait_ns);
            if (!ok) break;
            umma::fence_after_sync();
            mma2(g * half + i, i == 0);
          }
          if (!ok) break;
          umma::commit(&bars.p_ready[g]);
          ++np;
          if (k + 1 < kcta) {
            // MMA1 of the next slab once every compute warp has written its T_b^T
            ok = wait_for(&bars.tb_ready, (uint32_t)((k + 1) & 1), wait_ns);
            if (!ok) break;
            umma::fence_after_sync();
            mma1();
            umma::commit(&bars.eta_ready[g]);
            ++ne;
          }
        }
        if (!ok) atomicOr(&timed_out, 1);
        // this issuer's MMAs have completed before the TMEM is released
        if (ne > 0) wait_for(&bars.eta_ready[g], (uint32_t)((ne - 1) & 1), drain_ns);
        if (np > 0) wait_for(&bars.p_ready[g], (uint32_t)((np - 1) & 1), drain_ns);
      }
      __syncwarp();
    } else {
      // ---------------------------------------------------------------- compute warps 0-7
      const int q = warp & 3, wg = warp >> 2;
      const int c = 32 * q + lane;  // TMEM lane = row i1
      const bool rowok = c < n1;
      const uint32_t lq = (uint32_t)(32 * q) << 16;
      const int hw = K1 / 2;        // columns j2 of T_b^T this warpgroup forms
      bool ok = __all_sync(0xffffffffu, !*(volatile int*)&timed_out) != 0;
      // MMA0 on the compute warps: T_b^T(c, j2) = sum_j1 X_1(c, j1) T_a(k, j2, j1) for this
      // warpgroup's columns j2 in [wg hw, wg hw + hw), written as the A operand of MMA1
      const float* const x1c = X1T + (rowok ? c : 0);
      auto mma0 = [&](int kk) {
        const float* tk = TaS + (int64_t)kk * P1P * K1 + wg * hw;
        float acc[16];
#pragma unroll
        for (int u = 0; u < 16; ++u) acc[u] = 0.f;
        switch (hw >> 2) {
          case 1: mma0_fma<1>(tk, K1, p1, x1c, n1, rowok, acc); break;
          case 2: mma0_fma<2>(tk, K1, p1, x1c, n1, rowok, acc); break;
          case 3: mma0_fma<3>(tk, K1, p1, x1c, n1, rowok, acc); break;
          default: mma0_fma<4>(tk, K1, p1, x1c, n1, rowok, acc); break;
        }
        if (FORM == kFormBF16) {
#pragma unroll
          for (int q8 = 0; q8 < 2; ++q8)
            if (8 * q8 < hw) {
              uint32_t pk[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) pk[u] = pack_bf16(acc[8 * q8 + 2 * u], acc[8 * q8 + 2 * u + 1]);
              umma::st_x4(tb + lq + sh.c_tb + (uint32_t)((wg * hw + 8 * q8) / 2), pk);
            }
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v)
            if (4 * v < hw) {
              uint32_t hi[4], lo[4];
#pragma unroll
              for (int u = 0; u < 4; ++u) {
                hi[u] = rna_tf32(acc[4 * v + u]);
                lo[u] = rna_tf32(acc[4 * v + u] - __uint_as_float(hi[u]));
              }
              umma::st_x4(tb + lq + sh.c_tb + (uint32_t)(wg * hw + 4 * v), hi);
              if (PARTS == 2) umma::st_x4(tb + lq + sh.c_tblo + (uint32_t)(wg * hw + 4 * v), lo);
            }
        }
        umma::wait_st();
        umma::fence_before_sync();
        warp_arrive(&bars.tb_ready);
      };
      // the chunks whose r stores are in flight: their r_ready arrivals wait until the next chunks'
      // loads have been issued, so the store latency overlaps them
      auto r_done = [&](int i, int m) {
        umma::wait_st();
        umma::fence_before_sync();
        warp_arrive(&bars.r_ready[wg][i]);
        if (m == 2) warp_arrive(&bars.r_ready[wg][i + 1]);
      };
      // r = V (.) eta for one chunk: eta from e, V from the slot; r (split or packed) to TMEM
      auto v_load = [&](int s, float (&v)[16]) {
        const TV* vs = reinterpret_cast<const TV*>(base + sh.o_ring + (int64_t)s * sh.slot_bytes);
#pragma unroll
        for (int u = 0; u < 16; ++u) v[u] = rowok ? vload<TV>(vs + u * n1 + c) : 0.f;
      };
      auto r_chunk = [&](int ch, const float (&v)[16], uint32_t (&e)[16]) {
        if (FORM == kFormBF16) {
          uint32_t pk[8];
#pragma unroll
          for (int u = 0; u < 8; ++u)
            pk[u] = pack_bf16(v[2 * u] * __uint_as_float(e[2 * u]), v[2 * u + 1] * __uint_as_float(e[2 * u + 1]));
          umma::st_x8(tb + lq + sh.c_rb + (uint32_t)(8 * ch), pk);
        } else {
          uint32_t lo[16];
#pragma unroll
          for (int u = 0; u < 16; ++u) {
            const float r = v[u] * __uint_as_float(e[u]);
            e[u] = rna_tf32(r);
            lo[u] = rna_tf32(r - __uint_as_float(e[u]));
          }
          umma::st_x16(tb + lq + sh.c_eta + (uint32_t)(kUmRows * ch), e);
          if (PARTS == 2) umma::st_x16(tb + lq + sh.c_rlo + (uint32_t)(kUmRows * ch), lo);
        }
      };
      if (ok) mma0(0);
      for (int k = 0; k < kcta && ok; ++k) {
        const uint32_t par = (uint32_t)(k & 1);
        // ---- r = V (.) eta over this warpgroup's chunks, two at a time (both chunks' loads issued
        // before one wait), each chunk signalled to the issuer when in TMEM
        ok = warp_wait(&bars.eta_ready[wg], par, wait_ns);
        if (!ok) break;
        umma::fence_after_sync();
        const int g0 = k * sh.nchunk + wg * half;  // ring position of the first chunk
        int slot = g0 % sh.nslot;
        uint32_t ph = (uint32_t)((g0 / sh.nslot) & 1);
        int pend = -1, pm = 0;
        for (int i = 0; i < half; i += 2) {
          const int m = i + 1 < half ? 2 : 1;
          const int ch = wg * half + i;
          const int s0 = slot;
          const uint32_t ph0 = ph;
          if (++slot == sh.nslot) slot = 0, ph ^= 1u;
          const int s1 = slot;
          const uint32_t ph1 = ph;
          if (m == 2 && ++slot == sh.nslot) slot = 0, ph ^= 1u;
          ok = warp_wait(&bars.full[s0], ph0, wait_ns) && (m == 1 || warp_wait(&bars.full[s1], ph1, wait_ns));
          if (!ok) break;
          uint32_t e0[16], e1[16];
          float v0[16], v1[16];
          umma::ld_x16(tb + lq + sh.c_eta + (uint32_t)(kUmRows * ch), e0);
          if (m == 2) umma::ld_x16(tb + lq + sh.c_eta + (uint32_t)(kUmRows * (ch + 1)), e1);
          v_load(s0, v0);
          if (m == 2) v_load(s1, v1);
          if (pend >= 0) r_done(pend, pm);
          umma::wait_ld();
          umma::ld_done(e0);
          umma::ld_done(e1);
          warp_arrive(&bars.empty[s0]);  // the slots' data is in registers
          if (m == 2) warp_arrive(&bars.empty[s1]);
          r_chunk(ch, v0, e0);
          if (m == 2) r_chunk(ch + 1, v1, e1);
          pend = i;
          pm = m;
        }
        if (!ok) break;
        r_done(pend, pm);
        // ---- MMA0 of the next slab (T_b^T is free once both warpgroups' MMA1 of this slab ran)
        if (k + 1 < kcta) {
          ok = warp_wait(&bars.eta_ready[wg ^ 1], par, wait_ns);
          if (!ok) break;
          umma::fence_after_sync();
          mma0(k + 1);
        }
        // ---- P = P_0 + P_1 from TMEM into the B operand of MMA3 (K-major rows j2, K = c; warp q
        // writes K atom q of 32 rows c (TF32) or half of atom q / 2 (BF16); the split form stores
        // hi in rows j2 and lo in rows N3 + j2 of the atom).  The tile is free once MMA3 of the last
        // slab ran (sb_ready).
        ok = warp_wait(&bars.p_ready[0], par, wait_ns) && warp_wait(&bars.p_ready[1], par, wait_ns);
        if (ok && k > 0) ok = warp_wait(&bars.sb_ready, (uint32_t)((k - 1) & 1), wait_ns);
        if (!ok) break;
        umma::fence_after_sync();
        for (int g4 = wg; g4 < sh.N3 / 4; g4 += 2) {
          uint32_t a0[4], a1[4], b0[4], b1[4];
          umma::ld_x4(tb + lq + sh.c_p + 4u * g4, a0);
          umma::ld_x4(tb + lq + sh.c_p + sh.pw + 4u * g4, a1);
          if (PARTS == 2) {
            umma::ld_x4(tb + lq + sh.c_p + (uint32_t)sh.N2 + 4u * g4, b0);
            umma::ld_x4(tb + lq + sh.c_p + sh.pw + (uint32_t)sh.N2 + 4u * g4, b1);
          }
          umma::wait_ld();
          umma::ld_done(a0);
          umma::ld_done(a1);
          if (PARTS == 2) {
            umma::ld_done(b0);
            umma::ld_done(b1);
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int j2 = 4 * g4 + u;
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
        umma::fence_before_sync();
        fence_proxy_async();
        warp_arrive(&bars.pt_ready);
      }
      if (!ok) atomicOr(&timed_out, 1);
      umma::wait_st();  // after a time-out, r stores may still be in flight
    }
    umma::fence_before_sync();
    // the constant block's copies have landed before the CTA leaves (at once in a normal run)
    if (tid == 0) {
      wait_for(&bars.cst, 0u, drain_ns);
      wait_for(&bars.cst1, 0u, drain_ns);
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
  s.N3 = parts == 2 ? (int)up(p2, 8) : (int)up(p2, 16);  // MMA3 (M = 128) takes N = parts N3, a multiple of 16
  s.P1P = (int)up(p1, 4);
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
  o = up(o, 1024);
  // the V ring, then the P tile; d is staged for the first H stage in the last bytes of the two
  // (so that the first V chunks, in the first slots, can be in flight while T_a is formed)
  s.o_ring = o;
  s.slot_bytes = up((int64_t)kUmRows * n1 * vesz, 1024);
  s.ptile_atom = (int64_t)parts * s.N3 * 128;
  const int64_t ptile_bytes = up((int64_t)s.KA1 * s.ptile_atom, 1024);
  const int KQ = (s.kmax + 3) / 4 * 4;
  const int64_t tas_bytes = up(((int64_t)s.kmax * s.P1P * s.K1 + 16) * 4, 16);  // + slack read by MMA0
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
  // MMA3 reads 128 rows from each 32-row XT1 atom: the last atom's reads run 12 KB past the XT1
  // parts, into the tiles after them, which must lie inside the allocation
  if (s.total < parts * s.xt1_part + 12288) s.total = parts * s.xt1_part + 12288;
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

// ---------------------------------------------------------------- the H-transform on tcgen05
// eta = H(<X_j>, Theta) (Sec. 6.1, Eq. eighteen) for glam_predict and the other single-precision
// products of the linear predictor, one CTA per SM over the slabs i3 it owns:
//   first H stage  T_a = X_3 Theta for the CTA's slabs (FP32; zero rows of X_3 skipped), Theta
//                  staged in shared memory in rounds of rows j3
//   MMA0 (SIMT)    T_b^T (c x j2) = X_1 (c x j1) T_a^T, exact FP32 FMAs, split hi/lo into TMEM
//   MMA1 (tcgen05) eta^T (c x i2) = T_b^T X_2^T in the 3xTF32 form (about FP32 accuracy), A from
//                  TMEM, B = X_2 (hi and lo tiles formed in shared memory by the CTA), D in one of
//                  two TMEM buffers
//   write-out      the compute warps read eta^T from TMEM (lane = i1) and store it with
//                  coalesced global stores while MMA1 of the next slab fills the other buffer.
// Warps 0-7 compute (two warpgroups split the i2 columns of the write-out), warp 8 issues MMA1
// and owns the TMEM.  Every wait is bounded; a wait that runs out sets *err and the CTA drains and
// exits (eta is then incomplete).
constexpr int kPuThreads = 288;
constexpr int kPuIssuer = 8;

struct PuShape {
  int n1, n2, n3, p1, p2, p3;
  int K1, P1P, kmax, R;  // K of MMA1 (p2 padded to 8), p1 padded to 4, slabs per CTA, rows j3 per round
  int64_t o_x2t, x2t_part, o_tas, o_x3r, o_rows, o_stage, stage_floats, total;
  uint32_t c_eta, c_tb, c_tblo;  // TMEM: two eta buffers of n2 columns, T_b^T hi and lo
};

bool pu_configure(int n1, int n2, int n3, int p1, int p2, int p3, int grid, PuShape& s) {
  if (n1 < 4 || n1 > 128 || n1 % 4 != 0 || n2 < 32 || n2 % 32 != 0 || n2 > 224 || n3 < 1 || p1 < 1 ||
      p1 > 32 || p2 < 1 || p2 > 32 || p3 < 1 || grid < 1)
    return false;
  s.n1 = n1; s.n2 = n2; s.n3 = n3; s.p1 = p1; s.p2 = p2; s.p3 = p3;
  s.K1 = (int)up(p2, 8);
  s.P1P = (int)up(p1, 4);
  s.kmax = (n3 + grid - 1) / grid;
  const int KQ = (s.kmax + 3) / 4 * 4;
  int64_t o = 0;
  s.o_x2t = o;
  s.x2t_part = (int64_t)n2 * 128;  // rows i2 of 128 bytes (K = j2 <= 32 TF32 values), 1 KB groups
  o += 2 * s.x2t_part;
  s.o_tas = o;
  o += up(((int64_t)s.kmax * s.P1P * s.K1 + 16) * 4, 16);
  s.o_x3r = o;
  o += up((int64_t)p3 * KQ * 4, 16);
  s.o_rows = o;
  o += up((int64_t)p3 * 4, 16);
  s.o_stage = o;
  const int64_t P21 = (int64_t)p1 * p2;
  const int64_t room = (int64_t)g_um_budget - 1024 - o;
  int64_t R = room / (P21 * 4);
  if (R > p3) R = p3;
  if (R < 1) return false;
  s.R = (int)R;
  s.stage_floats = R * P21;
  o += up(s.stage_floats * 4, 16);
  s.total = up(o, 16);
  s.c_eta = 0;
  s.c_tb = (uint32_t)(2 * n2);
  s.c_tblo = s.c_tb + 32;
  if (s.c_tblo + 32 > kUmTmemCols) return false;
  return (size_t)(s.total + 1024) <= g_um_budget;
}

__global__ void __launch_bounds__(kPuThreads, 1)
predict_umma_kernel(PuShape sh, const float* __restrict__ X1T, const float* __restrict__ X2T,
                    const float* __restrict__ X3T, const float* __restrict__ Theta, float* __restrict__ eta,
                    int* __restrict__ err, uint64_t wait_ns) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ uint64_t tb_ready, eta_ready[2], eta_free[2];
  __shared__ uint32_t tmem_base_s;
  __shared__ int timed_out, nrows_s;
  const int n1 = sh.n1, n2 = sh.n2, n3 = sh.n3, p1 = sh.p1, p2 = sh.p2, p3 = sh.p3;
  const int P21 = p1 * p2, K1 = sh.K1, P1P = sh.P1P;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int kcta = (n3 - (int)blockIdx.x + (int)gridDim.x - 1) / (int)gridDim.x;
  unsigned char* const base = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  const uint32_t sbase = smem_u32(base);
  float* const TaS = reinterpret_cast<float*>(base + sh.o_tas);
  float* const X3r = reinterpret_cast<float*>(base + sh.o_x3r);
  int* const rowlist = reinterpret_cast<int*>(base + sh.o_rows);
  float* const stage = reinterpret_cast<float*>(base + sh.o_stage);
  const int KQ = (sh.kmax + 3) / 4 * 4;
  const uint64_t drain_ns = wait_ns > kDrainNs ? wait_ns : kDrainNs;
  if (tid == 0) {
    timed_out = 0;
    mbar_init(&tb_ready, 8);
    for (int b = 0; b < 2; ++b) {
      mbar_init(&eta_ready[b], 1);
      mbar_init(&eta_free[b], 8);
    }
    fence_mbar_init();
  }
  if (warp == kPuIssuer) {
    umma::tmem_alloc(&tmem_base_s, kUmTmemCols);
    umma::tmem_relinquish();
  }
  // X_2 as MMA1's B operand (rows i2, K = j2, 128-byte swizzle), hi and lo TF32 parts; each
  // thread loads 8 entries before it stores any
  for (int e0 = 0; e0 < n2 * 32; e0 += 8 * kPuThreads) {
    float v[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kPuThreads + tid, i2 = e >> 5, j2 = e & 31;
      v[u] = (e < n2 * 32 && j2 < p2) ? X2T[(int64_t)j2 * n2 + i2] : 0.f;
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const int e = e0 + u * kPuThreads + tid, i2 = e >> 5, j2 = e & 31;
      if (e >= n2 * 32) break;
      const uint32_t h = rna_tf32(v[u]);
      const uint32_t off = umma::sw128_k4((uint32_t)i2, (uint32_t)j2);
      *reinterpret_cast<uint32_t*>(base + sh.o_x2t + off) = h;
      *reinterpret_cast<uint32_t*>(base + sh.o_x2t + sh.x2t_part + off) = rna_tf32(v[u] - __uint_as_float(h));
    }
  }
  // X_3 entries of this CTA's slabs, [j3][k]; T_a starts at zero (rows j1 >= p1 stay zero)
  for (int idx = tid; idx < p3 * KQ; idx += kPuThreads) {
    const int j3 = idx / KQ, kk = idx - j3 * KQ;
    X3r[idx] = kk < kcta ? X3T[(int64_t)j3 * n3 + blockIdx.x + (int64_t)kk * gridDim.x] : 0.f;
  }
  for (int idx = tid; idx < sh.kmax * P1P * K1 + 16; idx += kPuThreads) TaS[idx] = 0.f;
  fence_proxy_async();  // the B tiles were written by plain stores; MMA1 reads them
  umma::fence_before_sync();
  __syncthreads();
  umma::fence_after_sync();
  const uint32_t tb = tmem_base_s;
  if (warp == 0) {  // rows j3 with a nonzero X_3 entry for this CTA's slabs, in increasing order
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
  __syncthreads();
  // first H stage: T_a(s_k, j2, j1) = sum_j3 X_3(s_k, j3) Theta(j3, j2, j1) over the listed rows,
  // in j3 order, Theta staged R rows at a time (only the listed rows are copied)
  const int nr = nrows_s;
  for (int rl = 0; rl < nr;) {
    int re = rl;
    while (re < nr && rowlist[re] - rowlist[rl] < sh.R) ++re;
    const int j0 = rowlist[rl];
    // the round's listed rows of Theta by asynchronous 4-byte copies, all in flight at once
    for (int idx = tid; idx < (re - rl) * P21; idx += kPuThreads) {
      const int t = idx / P21, i = idx - t * P21;
      const int j3 = rowlist[rl + t];
      asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(stage + (j3 - j0) * P21 + i)),
                   "l"(Theta + (int64_t)j3 * P21 + i)
                   : "memory");
    }
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    const int nkg = (kcta + 3) / 4;
    for (int task = tid; task < P21 * nkg; task += kPuThreads) {
      const int nn = task % P21, k0 = 4 * (task / P21);
      const int j2 = nn / p1, j1 = nn - j2 * p1;
      float a[4];
#pragma unroll
      for (int r = 0; r < 4; ++r) a[r] = (k0 + r < kcta) ? TaS[((k0 + r) * P1P + j1) * K1 + j2] : 0.f;
      for (int t0 = rl; t0 < re; t0 += 8) {
        int jr[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) jr[u] = rowlist[t0 + u < re ? t0 + u : re - 1];
        float dv[8];
        float4 xv[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          dv[u] = t0 + u < re ? stage[(jr[u] - j0) * P21 + nn] : 0.f;
          xv[u] = *reinterpret_cast<const float4*>(X3r + jr[u] * KQ + k0);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          a[0] = fmaf(xv[u].x, dv[u], a[0]);
          a[1] = fmaf(xv[u].y, dv[u], a[1]);
          a[2] = fmaf(xv[u].z, dv[u], a[2]);
          a[3] = fmaf(xv[u].w, dv[u], a[3]);
        }
      }
#pragma unroll
      for (int r = 0; r < 4; ++r)
        if (k0 + r < kcta) TaS[((k0 + r) * P1P + j1) * K1 + j2] = a[r];
    }
    __syncthreads();
    rl = re;
  }
  if (warp == kPuIssuer) {
    // ---------------------------------------------------------------- MMA1 issue (warp 8)
    if (lane == 0) {
      const uint32_t id1 = umma::idesc(128, (uint32_t)n2, umma::kTypeTF32, umma::kTypeTF32, 0, 0);
      const uint64_t bh = umma::sdesc(sbase + (uint32_t)sh.o_x2t, 16, 1024, umma::kSwizzle128B);
      const uint64_t bl = umma::sdesc(sbase + (uint32_t)(sh.o_x2t + sh.x2t_part), 16, 1024, umma::kSwizzle128B);
      int ne0 = 0, ne1 = 0;  // commits on eta_ready[0] and [1]
      bool ok = true;
      for (int k = 0; k < kcta && ok; ++k) {
        const int b = k & 1;
        ok = wait_for(&tb_ready, (uint32_t)(k & 1), wait_ns);
        if (ok && k >= 2) ok = wait_for(&eta_free[b], (uint32_t)(((k - 2) >> 1) & 1), wait_ns);
        if (!ok) break;
        umma::fence_after_sync();
        const uint32_t d = tb + sh.c_eta + (uint32_t)(b * n2);
        for (int s = 0; s < K1 / 8; ++s) {
          const uint64_t off = (uint64_t)(2 * s);  // 32 bytes of K
          umma::mma_tf32_ts(d, tb + sh.c_tb + 8u * s, bh + off, id1, s != 0);
          umma::mma_tf32_ts(d, tb + sh.c_tb + 8u * s, bl + off, id1, 1u);
          umma::mma_tf32_ts(d, tb + sh.c_tblo + 8u * s, bh + off, id1, 1u);
        }
        umma::commit(&eta_ready[b]);
        if (b == 0) ++ne0;
        else ++ne1;
      }
      if (!ok) atomicOr(&timed_out, 1);
      // every MMA has completed before the TMEM is released
      if (ne0 > 0) wait_for(&eta_ready[0], (uint32_t)((ne0 - 1) & 1), drain_ns);
      if (ne1 > 0) wait_for(&eta_ready[1], (uint32_t)((ne1 - 1) & 1), drain_ns);
    }
    __syncwarp();
  } else {
    // ---------------------------------------------------------------- compute warps 0-7
    const int q = warp & 3, wg = warp >> 2;
    const int c = 32 * q + lane;  // TMEM lane = row i1
    const bool rowok = c < n1;
    const uint32_t lq = (uint32_t)(32 * q) << 16;
    const int hw = K1 / 2;
    const float* const x1c = X1T + (rowok ? c : 0);
    auto mma0 = [&](int kk) {  // T_b^T(c, j2) for this warpgroup's columns j2, hi and lo parts
      const float* tk = TaS + (int64_t)kk * P1P * K1 + wg * hw;
      float acc[16];
#pragma unroll
      for (int u = 0; u < 16; ++u) acc[u] = 0.f;
      switch (hw >> 2) {
        case 1: mma0_fma<1>(tk, K1, p1, x1c, n1, rowok, acc); break;
        case 2: mma0_fma<2>(tk, K1, p1, x1c, n1, rowok, acc); break;
        case 3: mma0_fma<3>(tk, K1, p1, x1c, n1, rowok, acc); break;
        default: mma0_fma<4>(tk, K1, p1, x1c, n1, rowok, acc); break;
      }
#pragma unroll
      for (int v = 0; v < 4; ++v)
        if (4 * v < hw) {
          uint32_t hi[4], lo[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            hi[u] = rna_tf32(acc[4 * v + u]);
            lo[u] = rna_tf32(acc[4 * v + u] - __uint_as_float(hi[u]));
          }
          umma::st_x4(tb + lq + sh.c_tb + (uint32_t)(wg * hw + 4 * v), hi);
          umma::st_x4(tb + lq + sh.c_tblo + (uint32_t)(wg * hw + 4 * v), lo);
        }
      umma::wait_st();
      umma::fence_before_sync();
      warp_arrive(&tb_ready);
    };
    bool ok = __all_sync(0xffffffffu, !*(volatile int*)&timed_out) != 0;
    if (ok) mma0(0);
    const int half = n2 / 32;  // 16-column chunks of this warpgroup
    for (int k = 0; k < kcta && ok; ++k) {
      const int b = k & 1;
      ok = warp_wait(&eta_ready[b], (uint32_t)((k >> 1) & 1), wait_ns);
      if (!ok) break;
      umma::fence_after_sync();
      // T_b^T is free once MMA1 of slab k has completed: the next slab's goes in now, so that its
      // MMA1 runs while this slab is written out
      if (k + 1 < kcta) mma0(k + 1);
      float* out = eta + (int64_t)((int)blockIdx.x + k * (int)gridDim.x) * n2 * n1 + c;
      const uint32_t src = tb + lq + sh.c_eta + (uint32_t)(b * n2);
      for (int i = 0; i < half; i += 2) {  // two chunks per load round
        const int ch = wg * half + i;
        const bool two = i + 1 < half;
        uint32_t e0[16], e1[16];
        umma::ld_x16(src + (uint32_t)(16 * ch), e0);
        if (two) umma::ld_x16(src + (uint32_t)(16 * (ch + 1)), e1);
        umma::wait_ld();
        umma::ld_done(e0);
        umma::ld_done(e1);
        if (rowok) {
#pragma unroll
          for (int u = 0; u < 16; ++u) __stcs(out + (int64_t)(16 * ch + u) * n1, __uint_as_float(e0[u]));
          if (two) {
#pragma unroll
            for (int u = 0; u < 16; ++u) __stcs(out + (int64_t)(16 * (ch + 1) + u) * n1, __uint_as_float(e1[u]));
          }
        }
      }
      umma::fence_before_sync();
      warp_arrive(&eta_free[b]);
    }
    if (!ok) atomicOr(&timed_out, 1);
  }
  __syncthreads();
  if (timed_out && tid == 0) atomicOr(err, 1);
  if (warp == kPuIssuer) {
    umma::fence_after_sync();
    umma::tmem_dealloc(tb, kUmTmemCols);
  }
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
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(predict_umma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g_um_budget);
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
                              uint64_t wait_ns, bool pdl) {
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
  const dim3 g(grid), b(kUmThreads);
  cudaError_t e;
  if (form == kFormTF32)
    e = launch_pdl(fused_slab_umma_kernel<kFormTF32, float>, g, b, smem, st, pdl, s, c, D, X1T, X3T, tmapV, Sb,
                   skip, err, wait_ns);
  else if (form == kForm3x)
    e = launch_pdl(fused_slab_umma_kernel<kForm3x, float>, g, b, smem, st, pdl, s, c, D, X1T, X3T, tmapV, Sb,
                   skip, err, wait_ns);
  else if (v_bf16)
    e = launch_pdl(fused_slab_umma_kernel<kFormBF16, __nv_bfloat16>, g, b, smem, st, pdl, s, c, D, X1T, X3T,
                   tmapV, Sb, skip, err, wait_ns);
  else
    e = launch_pdl(fused_slab_umma_kernel<kFormBF16, float>, g, b, smem, st, pdl, s, c, D, X1T, X3T, tmapV, Sb,
                   skip, err, wait_ns);
  if (e != cudaSuccess) return e;
  count_launches(1);
  return cudaGetLastError();
}

int predict_umma_supported(int n1, int n2, int n3, int p1, int p2, int p3) {
  PuShape s;
  return pu_configure(n1, n2, n3, p1, p2, p3, um_grid(n3), s) ? 1 : 0;
}

cudaError_t launch_predict_umma(int n1, int n2, int n3, int p1, int p2, int p3, const float* X1T, const float* X2T,
                                const float* X3T, const float* Theta, float* eta, int* err, cudaStream_t st) {
  PuShape s;
  const int grid = um_grid(n3);
  if (!pu_configure(n1, n2, n3, p1, p2, p3, grid, s)) return cudaErrorInvalidValue;
  // at least half of the shared memory of an SM: one CTA per SM (the TMEM allocation is 512 columns)
  size_t smem = (size_t)s.total + 1024;
  if (smem < g_um_budget / 2 + 1024) smem = g_um_budget / 2 + 1024;
  predict_umma_kernel<<<grid, kPuThreads, smem, st>>>(s, X1T, X2T, X3T, Theta, eta, err, kDrainNs);
  count_launches(1);
  return cudaGetLastError();
}

}  // namespace glam
