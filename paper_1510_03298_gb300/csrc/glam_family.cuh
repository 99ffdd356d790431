// Per-cell quantities of the exponential families of App. B, shared by every kernel that
// evaluates them (the family pass, the loss reductions, the line search, the penalized NLL and
// the allocation-free loss), so that each computes the same terms with the same overflow clamp.
#pragma once

#include <cuda_runtime.h>

#include "glam.h"

namespace glam {
namespace {

template <typename T>
__device__ __forceinline__ T poisson_clamp();
template <>
__device__ __forceinline__ float poisson_clamp<float>() {
  return 80.0f;  // exp(80) ~ 5.5e34 < FLT_MAX
}
template <>
__device__ __forceinline__ double poisson_clamp<double>() {
  return 700.0;
}

template <typename T>
__device__ __forceinline__ T t_exp(T x);
template <>
__device__ __forceinline__ float t_exp<float>(float x) {
  return expf(x);
}
template <>
__device__ __forceinline__ double t_exp<double>(double x) {
  return exp(x);
}
template <typename T>
__device__ __forceinline__ T t_expm1(T x);
template <>
__device__ __forceinline__ float t_expm1<float>(float x) {
  return expm1f(x);
}
template <>
__device__ __forceinline__ double t_expm1<double>(double x) {
  return expm1(x);
}

template <typename T>
__device__ __forceinline__ T t_log1p(T x);
template <>
__device__ __forceinline__ float t_log1p<float>(float x) {
  return log1pf(x);
}
template <>
__device__ __forceinline__ double t_log1p<double>(double x) {
  return log1p(x);
}

// The per-cell quantities of App. B at eta = e for response y and observation weight a:
//   u  the score a theta'(e) (y - g^-1(e))                       (Eq. four)
//   w  the IRLS weight a theta'(e) (g^-1)'(e)                     (Eq. weights, times a)
//   l  the cell's term of n f, f = -(1/n) l(eta) + constants      (Eq. two)
//   dy the derivative of l in y
// Gaussian/identity, Poisson/log, binomial/logit (y a proportion of a trials) and Gamma/log
// (dispersion 1; the link is not canonical: theta(e) = -exp(-e)).  bad is set where e had to be
// clamped to keep the mean finite.
template <typename T>
struct CellTerms {
  T u, w, l, dy;
};
template <typename T>
__device__ __forceinline__ CellTerms<T> family_cell(int family, T e, T y, T a, int& bad) {
  CellTerms<T> c;
  if (family == GLAM_GAUSSIAN_IDENTITY) {
    const T r = y - e;              // identity link: mu = eta
    c.u = a * r;
    c.w = a;                        // theta' = (g^-1)' = 1
    c.l = T(0.5) * a * r * r;
    c.dy = a * r;
  } else if (family == GLAM_POISSON_LOG) {
    T ec = e;
    if (ec > poisson_clamp<T>()) {
      ec = poisson_clamp<T>();
      bad = 1;
    }
    const T mu = t_exp<T>(ec);      // log link: mu = exp(eta)
    c.u = a * (y - mu);
    c.w = a * mu;                   // (g^-1)' = exp(eta)
    c.l = a * (mu - y * e);
    c.dy = -a * e;
  } else if (family == GLAM_BINOMIAL_LOGIT) {
    const T ex = t_exp<T>(-fabs(e));  // in (0, 1]: no overflow on either side
    const T mu = e >= T(0) ? T(1) / (T(1) + ex) : ex / (T(1) + ex);
    c.u = a * (y - mu);
    c.w = a * mu * (T(1) - mu);     // (g^-1)' = mu (1 - mu)
    c.l = a * (fmax(e, T(0)) + t_log1p<T>(ex) - y * e);  // log(1 + e^eta) - y eta
    c.dy = -a * e;
  } else {                          // GLAM_GAMMA_LOG
    T ec = e;
    if (ec < -poisson_clamp<T>()) {
      ec = -poisson_clamp<T>();
      bad = 1;
    }
    const T ie = t_exp<T>(-ec);     // 1 / mu
    c.u = a * (y * ie - T(1));      // theta'(eta) = exp(-eta)
    c.w = a;                        // theta' (g^-1)' = exp(-eta) exp(eta)
    c.l = a * (y * ie + e);
    c.dy = a * ie;
  }
  return c;
}

}  // namespace
}  // namespace glam
