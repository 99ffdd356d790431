// Host-side numerics of the plan set-up, kept free of CUDA so that they compile with any C++
// compiler (the library includes this header; so does a host test of it).
#pragma once

#include <cmath>
#include <cstddef>
#include <vector>

namespace glam {

// Largest eigenvalue magnitude of a symmetric m x m matrix (row-major) by the cyclic Jacobi
// method: rotations zero each off-diagonal entry in turn until the off-diagonal mass is below
// 1e-30 of the diagonal's (or 100 sweeps); the spectral radius rho(X_j^T X_j) of Prop. 1 comes
// from it.  The matrix is taken by value and consumed.
inline double jacobi_spectral_radius(std::vector<double> A, int m) {
  auto at = [&](int i, int j) -> double& { return A[(size_t)i * m + j]; };
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < m; ++i) {
      diag += at(i, i) * at(i, i);
      for (int j = i + 1; j < m; ++j) off += at(i, j) * at(i, j);
    }
    if (off <= 1e-30 * (diag + 1e-300)) break;
    for (int p = 0; p < m - 1; ++p) {
      for (int q = p + 1; q < m; ++q) {
        const double apq = at(p, q);
        if (apq == 0.0) continue;
        const double theta = (at(q, q) - at(p, p)) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), s = t * c;
        for (int k = 0; k < m; ++k) {
          const double akp = at(k, p), akq = at(k, q);
          at(k, p) = c * akp - s * akq;
          at(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < m; ++k) {
          const double apk = at(p, k), aqk = at(q, k);
          at(p, k) = c * apk - s * aqk;
          at(q, k) = s * apk + c * aqk;
        }
      }
    }
  }
  double r = 0.0;
  for (int i = 0; i < m; ++i) r = std::fmax(r, std::fabs(at(i, i)));
  return r;
}

}  // namespace glam
