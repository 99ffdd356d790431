// Host driver of band_form, the band description of a marginal design used by the banded mode
// products: reads "n p" and then X^T (p rows of n values, row-major) from standard input and prints
// "banded 0|1", then (when banded) per row i "row start v0 v1 v2 v3" and per column j "col lo hi".
// Launches nothing: tests/test_band_form.py compiles it with nvcc and runs it on the host.
#include "../paper_1510_03298_gb300/csrc/glam_band.cu"

#include <cstdio>

namespace glam {
int num_sms() { return 152; }
void count_launches(int64_t) {}
}  // namespace glam

int main() {
  int n = 0, p = 0;
  if (std::scanf("%d %d", &n, &p) != 2 || n < 1 || p < 1) return 2;
  std::vector<double> XT((size_t)n * p);
  for (auto& v : XT)
    if (std::scanf("%lf", &v) != 1) return 2;
  std::vector<int> start, lo, hi;
  std::vector<double> val;
  const bool ok = glam::band_form(XT.data(), n, p, start, val, lo, hi);
  std::printf("banded %d\n", ok ? 1 : 0);
  if (!ok) return 0;
  for (int i = 0; i < n; ++i) {
    std::printf("row %d", start[i]);
    for (int t = 0; t < glam::kBand; ++t) std::printf(" %.17g", val[(size_t)i * glam::kBand + t]);
    std::printf("\n");
  }
  for (int j = 0; j < p; ++j) std::printf("col %d %d\n", lo[j], hi[j]);
  return 0;
}
