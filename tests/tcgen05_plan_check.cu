// Host-side check of the shared-memory and TMEM plans of the two tcgen05 kernels over a sweep of
// shapes: the bottleneck kernel's plan (um_configure; TF32, 3xTF32 and BF16 forms, FP32 or BF16 V)
// and the H-transform kernel's plan (pu_configure).  For every accepted shape: each shared-memory
// region lies inside the allocation, after the one before it and aligned as its use needs (1 KB
// for 128-byte-swizzled operand atoms, 16 bytes for bulk and tensor copies); the MMA shapes are
// legal for M = 128 (N a multiple of 16 in [16, 256], K a multiple of the instruction's K); the TMEM
// regions start on multiples of 32 columns, do not overlap and fit the 512 allocated columns; the
// V chunk's tensor-copy box has an inner extent of a multiple of 16 bytes; the slabs of the grid
// cover n3.  The program launches nothing: tests/test_tcgen05_plans.py compiles it with nvcc and
// runs it on the host.
#include "../paper_1510_03298_gb300/csrc/glam_fused_umma.cu"

#include <cstdio>

namespace glam {
int num_sms() { return 152; }
void count_launches(int64_t) {}
}  // namespace glam

using namespace glam;

namespace {

long g_fail = 0, g_um_ok = 0, g_pu_ok = 0;

#define REQ(c)                                                                                         \
  do {                                                                                                 \
    if (!(c)) {                                                                                        \
      if (g_fail < 20)                                                                                 \
        std::printf("FAIL %s: %s (form %d, n %d %d %d, p %d %d %d)\n", what, #c, form, n1, n2, n3, p1, \
                    p2, p3);                                                                           \
      ++g_fail;                                                                                        \
      return;                                                                                          \
    }                                                                                                  \
  } while (0)

bool legal_n(int64_t N) { return N % 16 == 0 && N >= 16 && N <= 256; }

void check_um(int form, bool vb, int n1, int n2, int n3, int p1, int p2, int p3) {
  const char* what = vb ? "fused (BF16 V)" : "fused";
  UmShape s{};
  const int grid = n3 < 152 ? n3 : 152;
  if (!um_configure(n1, n2, n3, p1, p2, p3, grid, form, vb, s)) return;
  ++g_um_ok;
  const int vesz = vb ? 2 : 4, esz = um_esz(form), parts = form == kForm3x ? 2 : 1, epr = 128 / esz;
  // the documented domain
  REQ(n1 >= 4 && n1 <= 128 && n1 % (form == kFormBF16 ? 8 : 4) == 0);
  REQ(n2 >= 32 && n2 % 32 == 0 && n2 <= (form == kForm3x ? 128 : 256));
  REQ(p1 >= 1 && p1 <= 32 && p2 >= 1 && p2 <= 32 && s.parts == parts);
  REQ(!vb || form == kFormBF16);
  // the V chunk's tensor-copy box (n1 elements x 16 rows)
  REQ((int64_t)n1 * vesz % 16 == 0);
  // MMA shapes: MMA1 (N = i2), MMA2 (N = hi/lo parts of j2), MMA3 (N = parts of j2)
  REQ(legal_n(n2) && legal_n((int64_t)parts * s.N2) && legal_n((int64_t)parts * s.N3));
  REQ(s.K1 >= p2 && s.K1 <= 32 && s.K1 % (form == kFormBF16 ? 16 : 8) == 0);
  REQ(s.N2 >= p2 && s.N3 >= p2 && s.P1P >= p1 && s.P1P % 4 == 0);
  REQ((int64_t)s.KA1 * epr >= n1 && (int64_t)(s.KA1 - 1) * epr < n1);
  REQ((int64_t)s.KA2 * epr >= n2 && (int64_t)(s.KA2 - 1) * epr < n2);
  REQ(s.nchunk * kUmRows == n2 && s.nchunk % 2 == 0 && s.nchunk / 2 <= kUmMaxHalf);
  REQ((int64_t)s.kmax * grid >= n3 && (int64_t)(s.kmax - 1) * grid < n3);
  // constant block: [XT1 parts][X2T parts][X2 atoms], every swizzled atom on a 1 KB boundary
  REQ(s.o_cst == 0 && s.o_xt1 == 0 && s.xt1_part % 1024 == 0 && s.x2t_part % 1024 == 0 &&
      s.x2_atom % 1024 == 0);
  REQ(s.xt1_part >= (int64_t)s.KA1 * 32 * 128);  // KA1 atoms of 32 rows j1 x 128 bytes
  REQ(s.x2t_part >= (int64_t)n2 * 128 && s.x2_atom >= (int64_t)parts * s.N2 * 128);
  REQ(s.o_x2t >= parts * s.xt1_part && s.o_x2 >= s.o_x2t + parts * s.x2t_part);
  REQ(s.cst_bytes >= s.o_x2 + (int64_t)s.KA2 * s.x2_atom && s.cst_bytes % 16 == 0);
  // the V ring, the P tile, T_a, X3's entries, the row list
  REQ(s.o_ring >= s.cst_bytes && s.o_ring % 1024 == 0);
  REQ(s.slot_bytes % 1024 == 0 && s.slot_bytes >= (int64_t)kUmRows * n1 * vesz);
  REQ(s.nslot >= 2 && s.nslot <= kUmMaxSlots && s.nslot <= 3 * s.nchunk);
  REQ(s.o_ptile >= s.o_ring + (int64_t)s.nslot * s.slot_bytes && s.o_ptile % 1024 == 0);
  REQ(s.ptile_atom % 1024 == 0 && s.ptile_atom >= (int64_t)parts * s.N3 * 128);
  const int64_t ptile_end = s.o_ptile + (int64_t)s.KA1 * s.ptile_atom;
  REQ(s.o_tas >= ptile_end && s.o_tas % 16 == 0);
  const int KQ = (s.kmax + 3) / 4 * 4;
  REQ(s.o_x3r >= s.o_tas + ((int64_t)s.kmax * s.P1P * s.K1 + 16) * 4 && s.o_x3r % 16 == 0);
  REQ(s.o_rows >= s.o_x3r + (int64_t)p3 * KQ * 4 && s.o_rows % 16 == 0);
  REQ(s.total >= s.o_rows + (int64_t)p3 * 4 && s.total % 16 == 0);
  // MMA3 reads 128 rows of 128 bytes from the start of each 32-row XT1 atom
  REQ(s.total >= (int64_t)parts * s.xt1_part + 16384 - 4096);
  REQ(s.total + 1024 <= (int64_t)g_um_budget);
  // descriptor start addresses hold (address >> 4) in 14 bits
  REQ(s.total + 1024 < (int64_t)1 << 18);
  // staging rounds of d: inside the ring and P tile, ending where T_a starts, 16-byte round starts
  const int64_t P21 = (int64_t)p1 * p2;
  REQ(s.R >= 1 && s.R <= p3 && s.stage_bytes >= (int64_t)s.R * P21 * 4 && s.stage_bytes % 16 == 0);
  REQ(s.o_stage >= s.o_ring && s.o_stage % 16 == 0 && s.o_stage + s.stage_bytes <= s.o_tas);
  REQ(s.R == p3 || ((int64_t)s.R * P21 * 4) % 16 == 0);
  // TMEM: eta (r in place for the TF32 forms), r lo or packed r, T_b^T (and lo), two partial P, S_b
  const uint32_t rcols =
      form == kForm3x ? (uint32_t)up(n2, 32) : (form == kFormBF16 ? (uint32_t)up(n2 / 2, 32) : 0u);
  REQ(s.c_eta == 0 && s.c_rlo >= s.c_eta + (uint32_t)n2 && s.c_rlo % 32 == 0 && s.c_rb == s.c_rlo);
  REQ(s.c_tb >= s.c_rlo + rcols && s.c_tb % 32 == 0);
  REQ(s.c_tblo >= s.c_tb + (uint32_t)s.K1 && s.c_tblo % 32 == 0);
  REQ(s.c_p >= (form == kForm3x ? s.c_tblo + (uint32_t)s.K1 : s.c_tb + (uint32_t)s.K1) && s.c_p % 32 == 0);
  REQ(s.pw >= (uint32_t)(parts * s.N2) && s.pw % 32 == 0);
  REQ(s.c_sb >= s.c_p + 2 * s.pw && s.c_sb % 32 == 0);
  REQ(s.c_sb + (uint32_t)(parts * s.N3) <= kUmTmemCols);
}

void check_pu(int n1, int n2, int n3, int p1, int p2, int p3) {
  const char* what = "predict";
  const int form = 3;
  PuShape s{};
  const int grid = n3 < 152 ? n3 : 152;
  if (!pu_configure(n1, n2, n3, p1, p2, p3, grid, s)) return;
  ++g_pu_ok;
  REQ(n1 >= 4 && n1 <= 128 && n1 % 4 == 0 && n2 >= 32 && n2 % 32 == 0 && n2 <= 224);
  REQ(p1 >= 1 && p1 <= 32 && p2 >= 1 && p2 <= 32);
  REQ(legal_n(n2));  // MMA1: eta^T, N = i2
  REQ(s.K1 >= p2 && s.K1 <= 32 && s.K1 % 8 == 0 && s.P1P >= p1 && s.P1P % 4 == 0);
  REQ((int64_t)s.kmax * grid >= n3 && (int64_t)(s.kmax - 1) * grid < n3);
  // X2 hi and lo tiles (rows i2 of 128 bytes, 1 KB swizzle atoms), T_a, X3's entries, rows, staging
  REQ(s.o_x2t == 0 && s.x2t_part >= (int64_t)n2 * 128 && s.x2t_part % 1024 == 0);
  REQ(s.o_tas >= 2 * s.x2t_part && s.o_tas % 16 == 0);
  const int KQ = (s.kmax + 3) / 4 * 4;
  REQ(s.o_x3r >= s.o_tas + ((int64_t)s.kmax * s.P1P * s.K1 + 16) * 4 && s.o_x3r % 16 == 0);
  REQ(s.o_rows >= s.o_x3r + (int64_t)p3 * KQ * 4 && s.o_rows % 16 == 0);
  REQ(s.o_stage >= s.o_rows + (int64_t)p3 * 4 && s.o_stage % 16 == 0);
  REQ(s.R >= 1 && s.R <= p3 && s.stage_floats == (int64_t)s.R * p1 * p2);
  REQ(s.total >= s.o_stage + s.stage_floats * 4 && s.total % 16 == 0);
  REQ(s.total + 1024 <= (int64_t)g_um_budget && s.total + 1024 < (int64_t)1 << 18);
  // TMEM: two eta buffers of n2 columns, T_b^T hi and lo
  REQ(s.c_eta == 0 && s.c_tb >= 2u * (uint32_t)n2 && s.c_tb % 32 == 0);
  REQ(s.c_tblo >= s.c_tb + (uint32_t)s.K1 && s.c_tblo % 32 == 0 && s.c_tblo + (uint32_t)s.K1 <= kUmTmemCols);
}

}  // namespace

int main() {
  g_um_budget = 232448 - 2048;  // the GB300's opt-in shared memory per block, less the static part
  const int n3s[] = {1, 2, 5, 151, 152, 153, 365, 600, 2000};
  const int p3s[] = {1, 3, 12, 60, 200, 2000};
  const int ps[] = {1, 2, 3, 4, 5, 7, 8, 9, 15, 16, 17, 20, 24, 30, 31, 32, 33};
  const int forms[] = {kFormTF32, kForm3x, kFormBF16};
  for (int n1 = 4; n1 <= 132; n1 += 4)
    for (int n2 = 16; n2 <= 288; n2 += 16)
      for (int p1 : ps)
        for (int p2 : ps)
          for (int n3 : n3s)
            for (int p3 : p3s) {
              for (int form : forms) check_um(form, false, n1, n2, n3, p1, p2, p3);
              check_um(kFormBF16, true, n1, n2, n3, p1, p2, p3);
              check_pu(n1, n2, n3, p1, p2, p3);
            }
  UmShape s{};
  if (um_configure(128, 128, 600, 20, 20, 60, 152, kForm3x, false, s))
    std::printf("128x128x600 3xTF32: %lld B of shared memory, %d V slots, TMEM to column %u\n",
                (long long)s.total + 1024, s.nslot, s.c_sb + 2 * s.N3);
  std::printf("accepted: %ld bottleneck plans, %ld H-transform plans; failures %ld\n", g_um_ok, g_pu_ok, g_fail);
  return g_fail != 0 || g_um_ok == 0 || g_pu_ok == 0 ? 1 : 0;
}
