// Host driver of jacobi_spectral_radius (the rho(X_j^T X_j) of Prop. 1 in the plan set-up): reads
// matrices "m" followed by m x m values (row-major) from standard input until end of input and
// prints the spectral radius of each.  tests/test_jacobi.py builds it with the host C++ compiler.
#include <cstdio>
#include <vector>

#include "glam_host_math.h"

int main() {
  int m = 0;
  while (std::scanf("%d", &m) == 1) {
    if (m < 1) return 2;
    std::vector<double> A((size_t)m * m);
    for (auto& v : A)
      if (std::scanf("%lf", &v) != 1) return 2;
    std::printf("%.17g\n", glam::jacobi_spectral_radius(A, m));
  }
  return 0;
}
