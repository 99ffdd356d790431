// Entrywise steps and reductions of GD-PG.
//
//  * family pass (Sec. 6.1 step 2; App. B Eqs. four, weights, tennew; Gaussian, Poisson, binomial
//    and Gamma families, family_cell): from eta, Y and the
//    observation weights a it writes V = w, V (.) Z = u + w eta and optionally U, and reduces the
//    loss f(eta) (FP64 accumulation) and max(w) (for the step size of Prop. 1);
//  * proximal step (Sec. 3.2, Sec. 6.3): y = x + omega (x - x_prev), g = (Q - b)/n,
//    x+ = soft(y - delta g, delta lambda w_m), with the inner stopping reduction;
//  * Armijo rule (Sec. 5): Delta_k and the loss change at several trial steps in one pass over
//    the cells, using eta(theta + alpha d) = eta + alpha (eta~ - eta) (linearity of H);
//  * KKT residual, lambda_max (Sec. 6.4), penalty, conversions, Gram matrices (Prop. 1).
//
// Reductions: per-thread partials in the working precision over a few elements, FP64 across
// threads and blocks, and a deterministic final sum in block order by the last block to finish
// (no floating-point atomics, so every run gives the same bits).
#include <cuda_bf16.h>

#include <atomic>
#include <cfloat>
#include <type_traits>

#include "glam_family.cuh"
#include "glam_internal.cuh"

namespace glam {
namespace {

constexpr int kEPT = 8;  // elements per thread per tile of a streaming reduction

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide sums of NV values; result valid in thread 0.
template <int NV>
__device__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) v[k] = warp_sum(v[k]);
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; ++k) sh[k][warp] = v[k];
  __syncthreads();
  if (warp == 0) {
#pragma unroll
    for (int k = 0; k < NV; ++k) {
      double t = lane < nw ? sh[k][lane] : 0.0;
      v[k] = warp_sum(t);
    }
  }
  __syncthreads();
}

__device__ double block_max(double v) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
  v = warp_max(v);
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double t = lane < nw ? sh[lane] : 0.0;
    v = warp_max(t);
  }
  __syncthreads();
  return v;
}

// Last-block-done: returns true in every thread of the block that finished last.  Partials
// written before the call are visible to that block (threadfence before the ticket).
__device__ bool last_block(unsigned int* counter) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned int ticket = atomicAdd(counter, 1u);
    is_last = (ticket == gridDim.x - 1);
  }
  __syncthreads();
  return is_last;
}

int red_blocks(int64_t n, int per_thread) {
  const int64_t per_block = (int64_t)kThreads * per_thread;
  int64_t b = (n + per_block - 1) / per_block;
  const int cap = 4 * num_sms();
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  if (b > kMaxRedBlocks) b = kMaxRedBlocks;
  return (int)b;
}

// ---------------------------------------------------------------- family pass
// The stored IRLS weight in the type the inner-loop product reads (BF16 rounds to nearest).
template <typename TV, typename T>
__device__ __forceinline__ TV to_weight(T w) {
  if constexpr (std::is_same<TV, __nv_bfloat16>::value) {
    if constexpr (sizeof(T) == 8) return __double2bfloat16(w);
    else return __float2bfloat16_rn(w);
  } else {
    return TV(w);
  }
}

template <typename T, typename TV>
__global__ void __launch_bounds__(kThreads)
family_kernel(int family, int64_t n, const T* __restrict__ eta, const T* __restrict__ Y,
              const T* __restrict__ A, TV* __restrict__ V, T* __restrict__ VZ, T* __restrict__ U,
              double rho_prod, DevScalars* sc, RedScratch red) {
  double lsum = 0.0, wmax = 0.0;
  int bad = 0;
  const int64_t tile = (int64_t)gridDim.x * blockDim.x * kEPT;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kEPT; base < n; base += tile) {
    T lpart = T(0);
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int64_t i = base + (int64_t)k * blockDim.x + threadIdx.x;
      if (i >= n) break;
      const T e = eta[i], y = Y[i], a = A[i];
      const CellTerms<T> c = family_cell<T>(family, e, y, a, bad);
      const T u = c.u, w = c.w, l = c.l;
      if (!(isfinite(e) && isfinite(y) && isfinite(a))) bad = 1;
      if (V != nullptr) V[i] = to_weight<TV>(w);
      if (VZ != nullptr) VZ[i] = u + w * e;  // V (.) Z with Z = W^-1 u + eta (Eq. ten)
      if (U != nullptr) U[i] = u;
      lpart += l;
      wmax = fmax(wmax, (double)w);
    }
    lsum += (double)lpart;
  }
  double v[1] = {lsum};
  block_sum<1>(v);
  const double m = block_max(wmax);
  if (threadIdx.x == 0) {
    red.partial[blockIdx.x * 2 + 0] = v[0];
    red.partial[blockIdx.x * 2 + 1] = m;
    if (bad) atomicOr(&sc->nonfinite, 1);
  }
  if (last_block(red.counter)) {
    if (threadIdx.x == 0) {
      double s = 0.0, mx = 0.0;
      for (unsigned int b = 0; b < gridDim.x; ++b) {
        s += __ldcg(&red.partial[b * 2 + 0]);
        mx = fmax(mx, __ldcg(&red.partial[b * 2 + 1]));
      }
      sc->loss = s / (double)n;
      sc->maxw = mx;
      sc->Lhat = mx / (double)n * rho_prod;  // Prop. 1, Eq. (nineteennew); rho_prod sums over the components
      *red.counter = 0u;
    }
  }
}

// ---------------------------------------------------------------- loss only
template <typename T>
__global__ void __launch_bounds__(kThreads)
loss_kernel(int family, int64_t n, const T* __restrict__ eta, const T* __restrict__ Y,
            const T* __restrict__ A, double* out, RedScratch red) {
  double lsum = 0.0;
  const int64_t tile = (int64_t)gridDim.x * blockDim.x * kEPT;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kEPT; base < n; base += tile) {
    T lpart = T(0);
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int64_t i = base + (int64_t)k * blockDim.x + threadIdx.x;
      if (i >= n) break;
      int bad = 0;
      lpart += family_cell<T>(family, eta[i], Y[i], A[i], bad).l;
    }
    lsum += (double)lpart;
  }
  double v[1] = {lsum};
  block_sum<1>(v);
  if (threadIdx.x == 0) red.partial[blockIdx.x] = v[0];
  if (last_block(red.counter)) {
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (unsigned int b = 0; b < gridDim.x; ++b) s += __ldcg(&red.partial[b]);
      *out = s / (double)n;
      *red.counter = 0u;
    }
  }
}

// ---------------------------------------------------------------- penalized NLL and its VJP
// Cells pass of the penalized negative log-likelihood (Sec. 2, Eqs. two/three; App. B): reduces
// f(eta) and, for the vector-Jacobian product with the upstream scalar g (*gout, 1 if NULL),
// writes U = -(g/n) u (so that G(U) = g grad_theta f, Eq. nineteen) and GY = g df/dy, with the
// per-cell terms of family_cell.
template <typename T>
__global__ void __launch_bounds__(kThreads)
nll_cells_kernel(int family, int64_t n, const T* __restrict__ eta, const T* __restrict__ Y,
                 const T* __restrict__ A, const double* __restrict__ gout, T* __restrict__ U,
                 T* __restrict__ GY, DevScalars* sc, RedScratch red) {
  const double g = gout ? *gout : 1.0;
  const T su = T(-g / (double)n), sy = T(g / (double)n);
  double lsum = 0.0;
  int bad = 0;
  const int64_t tile = (int64_t)gridDim.x * blockDim.x * kEPT;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kEPT; base < n; base += tile) {
    T lpart = T(0);
#pragma unroll
    for (int k = 0; k < kEPT; ++k) {
      const int64_t i = base + (int64_t)k * blockDim.x + threadIdx.x;
      if (i >= n) break;
      const T e = eta[i], y = Y[i], a = A[i];
      const CellTerms<T> c = family_cell<T>(family, e, y, a, bad);
      lpart += c.l;
      if (!(isfinite(e) && isfinite(y) && isfinite(a))) bad = 1;
      if (U != nullptr) U[i] = su * c.u;
      if (GY != nullptr) GY[i] = sy * c.dy;
    }
    lsum += (double)lpart;
  }
  double v[1] = {lsum};
  block_sum<1>(v);
  if (threadIdx.x == 0) {
    red.partial[blockIdx.x] = v[0];
    if (bad) atomicOr(&sc->nonfinite, 1);
  }
  if (last_block(red.counter)) {
    if (threadIdx.x == 0) {
      double s = 0.0;
      for (unsigned int b = 0; b < gridDim.x; ++b) s += __ldcg(&red.partial[b]);
      sc->loss = s / (double)n;
      *red.counter = 0u;
    }
  }
}

// Coefficient pass: J(theta) = sum_m w_m |theta_m| (FP64), F = f + lambda J, and the penalty part
// of the VJP, grad[m] = Q[m] + g lambda w_m sign(theta_m) (sign(0) = 0; Q = g grad f from G).
template <typename T>
__global__ void __launch_bounds__(kThreads)
nll_coef_kernel(int64_t p, const T* __restrict__ th, const T* __restrict__ pw, double lambda,
                const double* __restrict__ gout, const T* __restrict__ Q, T* __restrict__ grad,
                double* F, DevScalars* sc, RedScratch red) {
  const double g = gout ? *gout : 1.0;
  double acc[1] = {0.0};
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < p;
       m += (int64_t)gridDim.x * blockDim.x) {
    const double t = (double)th[m], w = (double)pw[m];
    acc[0] += w * fabs(t);
    if (grad != nullptr) {
      const double sg = t > 0.0 ? 1.0 : (t < 0.0 ? -1.0 : 0.0);
      grad[m] = T((double)Q[m] + g * lambda * w * sg);
    }
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) red.partial[blockIdx.x] = acc[0];
  if (last_block(red.counter)) {
    if (threadIdx.x == 0) {
      double pen = 0.0;
      for (unsigned int b = 0; b < gridDim.x; ++b) pen += __ldcg(&red.partial[b]);
      sc->pen = pen;
      if (F != nullptr) *F = sc->loss + lambda * pen;
      *red.counter = 0u;
    }
  }
}

// ---------------------------------------------------------------- SCAD weights
// Weights of step s >= 1 of the multistep adaptive lasso for the SCAD penalty: the local linear
// approximation at theta, w[m] = base[m] p'_lambda(|theta_m|) / lambda with p'_lambda(t) = lambda
// for t <= lambda and (a lambda - t)_+ / (a - 1) beyond.
__global__ void scad_weights_kernel(int64_t p, const double* __restrict__ th,
                                    const double* __restrict__ base, double lambda, double a,
                                    double* __restrict__ w) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < p;
       m += (int64_t)gridDim.x * blockDim.x) {
    const double t = fabs(th[m]);
    const double d = t <= lambda ? lambda : fmax(a * lambda - t, 0.0) / (a - 1.0);
    w[m] = base[m] * (d / lambda);
  }
}

// ---------------------------------------------------------------- scale / convert / finite
template <typename T>
__global__ void scale_kernel(int64_t n, const T* __restrict__ in, T* __restrict__ out, T scale) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = in[i] * scale;
}

template <typename TI, typename TO>
__global__ void convert_kernel(int64_t n, const TI* __restrict__ in, TO* __restrict__ out) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    out[i] = (TO)in[i];
}

// y = x + omega (x - x_prev) (the FISTA extrapolation of Sec. 3.2), x_prev may be NULL
template <typename T>
__global__ void extrap_kernel(int64_t n, const T* __restrict__ x, const T* __restrict__ xp,
                              double omega, T* __restrict__ y) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] = xp ? (T)((double)x[i] + omega * ((double)x[i] - (double)xp[i])) : x[i];
}

template <typename T>
__global__ void sum_splits_kernel(int64_t p, int ksplit, const T* __restrict__ part, T* __restrict__ out) {
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < p;
       m += (int64_t)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int s = 0; s < ksplit; ++s) acc += part[(int64_t)s * p + m];
    out[m] = acc;
  }
}

template <typename T>
__global__ void vmul_kernel(int64_t n, const T* __restrict__ V, T* x, const int* skip) {
  if (skip != nullptr && *skip) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    x[i] = V[i] * x[i];
}

// y += x (the sum over the components of a model with c > 1, Eq. eighteen)
template <typename T>
__global__ void add_kernel(int64_t n, const T* __restrict__ x, T* y, const int* skip) {
  if (skip != nullptr && *skip) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

template <typename T>
__global__ void finite_kernel(int64_t n, const T* __restrict__ x, DevScalars* sc) {
  int bad = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(x[i])) bad = 1;
  if (__syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&sc->nonfinite, 1);
}

// ---------------------------------------------------------------- proximal step
// out[m] = soft(y_m - delta g_m, delta lambda w_m), y = x + omega (x - x_prev) (Sec. 3.2, 6.3),
// with the gradient of the quadratic model written as g = lin_scale * lin[m] + (sum_s Qpart[s]) / n:
//   lin = b = X^T W z, lin_scale = -1/n:   g = (X^T W X y - X^T W z) / n     (Eq. twentyfive)
//   lin = grad f(theta_k), lin_scale = 1:  g = grad f(theta_k) + X^T W X (y - theta_k) / n
// (the same function of y; the second form needs the products only for the correction).
// With a control block, omega, delta and lambda come from it, the kernel reduces
// max_m |x+_m - y_m| and the last block decides whether the inner loop stops.
// With dnext, the kernel also writes the operand of the next iteration's first mode product,
// dnext = y(l+1) - anchor = x+ + omega_{l+1} (x+ - x) - anchor, rounded to Tq.
template <typename Tq, typename TP>
__global__ void __launch_bounds__(kThreads)
prox_kernel(int64_t p, int ksplit, const Tq* __restrict__ Qpart, const TP* __restrict__ lin,
            TP lin_scale, const TP* __restrict__ x, const TP* xprev, const TP* __restrict__ pen_w,
            TP* out, TP inv_n, InnerCtl* ctl, TP omega_h, TP delta_h, TP lambda_h, const double* Lhat,
            Tq* __restrict__ dnext, const TP* __restrict__ anchor) {
  // The element loads of the first grid-stride step are issued before the control block is
  // read (they do not depend on it), so the two memory round trips overlap.
  const int64_t m0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  TP q0 = TP(0), lin0 = TP(0), x0 = TP(0), xp0 = TP(0), pw0 = TP(0), an0 = TP(0);
  if (m0 < p) {
    // every split partial is loaded before the first add (one memory round trip); the adds
    // then run in split order
    Tq qv[kMaxSplits];
#pragma unroll
    for (int s = 0; s < kMaxSplits; ++s) qv[s] = s < ksplit ? Qpart[(int64_t)s * p + m0] : Tq(0);
#pragma unroll
    for (int s = 0; s < kMaxSplits; ++s)
      if (s < ksplit) q0 += TP(qv[s]);
    lin0 = lin[m0];
    x0 = x[m0];
    xp0 = xprev[m0];
    pw0 = pen_w[m0];
    if (dnext != nullptr) an0 = anchor[m0];
  }
  TP omega, delta, lam, omega_next = TP(0), pl1 = TP(1), pl2 = TP(0);
  if (ctl != nullptr) {
    const int done = ctl->done;
    const int l = ctl->l;
    const double cdelta = ctl->delta, clambda = ctl->lambda, cl1 = ctl->pen_l1, cl2 = ctl->pen_l2;
    if (done) return;
    omega = TP(l - 1) / TP(l + 2);
    omega_next = TP(l) / TP(l + 3);
    delta = TP(cdelta);
    lam = TP(clambda);
    pl1 = TP(cl1);
    pl2 = TP(cl2);
  } else {
    omega = omega_h;
    delta = delta_h > TP(0) ? delta_h : TP(1.0 / *Lhat);
    lam = lambda_h;
  }
  double crit = 0.0;
  for (int64_t m = m0; m < p; m += stride) {
    TP q, lm, xm, xpm, pwm, anm;
    if (m == m0) {
      q = q0; lm = lin0; xm = x0; xpm = xp0; pwm = pw0; anm = an0;
    } else {
      q = TP(0);
      for (int s = 0; s < ksplit; ++s) q += TP(Qpart[(int64_t)s * p + m]);
      lm = lin[m]; xm = x[m]; xpm = xprev[m]; pwm = pen_w[m];
      anm = dnext != nullptr ? anchor[m] : TP(0);
    }
    const TP g = lin_scale * lm + q * inv_n;    // gradient of the quadratic model
    const TP y = xm + omega * (xm - xpm);       // extrapolation, Sec. 3.2
    const TP z = y - delta * g;
    const TP gam = delta * lam * pwm;
    const TP az = fabs(z) - gam * pl1;          // soft threshold, Sec. 6.3
    // then the ridge shrinkage of the elastic-net / ridge prox (Sec. 6.3)
    const TP xn = (az > TP(0) ? copysign(az, z) : TP(0)) / (TP(1) + TP(2) * gam * pl2);
    out[m] = xn;
    if (dnext != nullptr) dnext[m] = Tq(xn + omega_next * (xn - xm) - anm);
    crit = fmax(crit, (double)fabs(xn - y));
  }
  if (ctl == nullptr) return;
  const double bm = block_max(crit);
  if (threadIdx.x == 0) atomicMax(&ctl->crit_bits, (unsigned long long)__double_as_longlong(bm));
  if (last_block(&ctl->counter)) {
    if (threadIdx.x == 0)
      ctl_finish_iteration(ctl, __longlong_as_double((long long)atomicAdd(&ctl->crit_bits, 0ull)));
  }
}

// ---------------------------------------------------------------- Armijo (Sec. 5)
// sums[0] = sum_i u_i d_i;  sums[1 + j] = sum_i a_i (l_i(eta + alpha_j d) - l_i(eta)), d = eta~ - eta
// with l_i the per-cell loss, written as a difference so that small steps keep their digits:
//   Gaussian: t (t/2 - (y - eta)),  Poisson: exp(eta) expm1(t) - y t,   t = alpha_j (eta~ - eta).
template <typename TE, typename T>
__global__ void __launch_bounds__(kThreads)
armijo_stream_kernel(int family, int64_t n, const TE* __restrict__ eta, const T* __restrict__ deta,
                     const TE* __restrict__ Y, const TE* __restrict__ A, double alpha0, double bfac,
                     int j0, DevScalars* sc, RedScratch red) {
  double acc[kTrials + 1];
#pragma unroll
  for (int k = 0; k <= kTrials; ++k) acc[k] = 0.0;
  T alpha[kTrials];
  {
    double a = alpha0;
    for (int j = 0; j < j0; ++j) a *= bfac;
#pragma unroll
    for (int j = 0; j < kTrials; ++j) {
      alpha[j] = T(a);
      a *= bfac;
    }
  }
  const int64_t tile = (int64_t)gridDim.x * blockDim.x * kEPT;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kEPT; base < n; base += tile) {
    T part[kTrials + 1];
#pragma unroll
    for (int k = 0; k <= kTrials; ++k) part[k] = T(0);
#pragma unroll 2
    for (int k = 0; k < kEPT; ++k) {
      const int64_t i = base + (int64_t)k * blockDim.x + threadIdx.x;
      if (i >= n) break;
      const T e = T(eta[i]), y = T(Y[i]), a = T(A[i]);
      const T d = deta[i];  // eta(theta~) - eta(theta) = H(theta~ - theta)
      // part[0]: <u, d>; part[1 + j]: the cell's loss change at the step alpha_j d, each written
      // as a difference that keeps its digits for small steps (expm1, log1p)
      if (family == GLAM_GAUSSIAN_IDENTITY) {
        const T r = T(Y[i] - eta[i]);
        part[0] += a * r * d;
#pragma unroll
        for (int j = 0; j < kTrials; ++j) {
          const T t = alpha[j] * d;
          part[1 + j] += a * (t * (T(0.5) * t - r));
        }
      } else if (family == GLAM_POISSON_LOG) {
        const T mu = t_exp<T>(e);
        part[0] += a * (y - mu) * d;
#pragma unroll
        for (int j = 0; j < kTrials; ++j) {
          const T t = alpha[j] * d;
          part[1 + j] += a * (mu * t_expm1<T>(t) - y * t);
        }
      } else if (family == GLAM_BINOMIAL_LOGIT) {
        // log(1 + e^(eta + t)) - log(1 + e^eta) = log1p(mu expm1(t))
        const T ex = t_exp<T>(-fabs(e));
        const T mu = e >= T(0) ? T(1) / (T(1) + ex) : ex / (T(1) + ex);
        part[0] += a * (y - mu) * d;
#pragma unroll
        for (int j = 0; j < kTrials; ++j) {
          const T t = alpha[j] * d;
          part[1 + j] += a * (t_log1p<T>(mu * t_expm1<T>(t)) - y * t);
        }
      } else {  // Gamma, log link: l = y e^-eta + eta
        const T ie = t_exp<T>(-e);
        part[0] += a * (y * ie - T(1)) * d;
#pragma unroll
        for (int j = 0; j < kTrials; ++j) {
          const T t = alpha[j] * d;
          part[1 + j] += a * (y * ie * t_expm1<T>(-t) + t);
        }
      }
    }
#pragma unroll
    for (int k = 0; k <= kTrials; ++k) acc[k] += (double)part[k];
  }
  block_sum<kTrials + 1>(acc);
  if (threadIdx.x == 0)
    for (int k = 0; k <= kTrials; ++k) red.partial[blockIdx.x * (kTrials + 1) + k] = acc[k];
  if (last_block(red.counter)) {
    if (threadIdx.x < kTrials + 1) {
      const int k = threadIdx.x;
      double s = 0.0;
      for (unsigned int b = 0; b < gridDim.x; ++b) s += __ldcg(&red.partial[b * (kTrials + 1) + k]);
      if (k == 0)
        sc->dir = -s / (double)n;
      else
        sc->data_diff[k - 1] = s / (double)n;
    }
    __syncthreads();
    if (threadIdx.x == 0) *red.counter = 0u;
  }
}

// pen_diff[j] = J(theta + alpha_j d) - J(theta); pen_tilde_diff = J(theta~) - J(theta);
// pen = J(theta).
template <typename T>
__global__ void __launch_bounds__(kThreads)
armijo_penalty_kernel(int64_t p, const T* __restrict__ th, const T* __restrict__ tt,
                      const T* __restrict__ pw, double alpha0, double bfac, int j0, DevScalars* sc,
                      RedScratch red, double l1, double l2) {
  constexpr int NV = kTrials + 2;
  double acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.0;
  double alpha[kTrials];
  {
    double a = alpha0;
    for (int j = 0; j < j0; ++j) a *= bfac;
    for (int j = 0; j < kTrials; ++j) {
      alpha[j] = a;
      a *= bfac;
    }
  }
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < p;
       m += (int64_t)gridDim.x * blockDim.x) {
    const double t0 = (double)th[m], t1 = (double)tt[m], w = (double)pw[m];
    const double d = t1 - t0;
    const double a0 = fabs(t0);
    // J = sum w (l1 |t| + l2 t^2); the changes use t^2 - t0^2 = s (2 t0 + s), s = t - t0
    acc[0] += w * (l1 * a0 + l2 * t0 * t0);
    acc[1] += w * (l1 * (fabs(t1) - a0) + l2 * d * (2.0 * t0 + d));
#pragma unroll
    for (int j = 0; j < kTrials; ++j) {
      const double sj = alpha[j] * d;
      acc[2 + j] += w * (l1 * (fabs(t0 + sj) - a0) + l2 * sj * (2.0 * t0 + sj));
    }
  }
  block_sum<NV>(acc);
  if (threadIdx.x == 0)
    for (int k = 0; k < NV; ++k) red.partial[blockIdx.x * NV + k] = acc[k];
  if (last_block(red.counter)) {
    if (threadIdx.x < NV) {
      const int k = threadIdx.x;
      double s = 0.0;
      for (unsigned int b = 0; b < gridDim.x; ++b) s += __ldcg(&red.partial[b * NV + k]);
      if (k == 0)
        sc->pen = s;
      else if (k == 1)
        sc->pen_tilde_diff = s;
      else
        sc->pen_diff[k - 2] = s;
    }
    __syncthreads();
    if (threadIdx.x == 0) *red.counter = 0u;
  }
}

// Smallest j with F(theta + alpha_j d) - F(theta) <= alpha_j v Delta_k, where
// Delta_k = -(1/n) u^T X d + lambda (J(theta~) - J(theta)).
__global__ void armijo_select_kernel(double lambda, double v, double alpha0, double bfac, int j0,
                                     DevScalars* sc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double Delta = sc->dir + lambda * sc->pen_tilde_diff;
  double a = alpha0;
  for (int j = 0; j < j0; ++j) a *= bfac;
  sc->accepted = -1;
  for (int j = 0; j < kTrials; ++j) {
    const double dF = sc->data_diff[j] + lambda * sc->pen_diff[j];
    if (dF <= a * v * Delta) {
      sc->accepted = j0 + j;
      sc->alpha = a;
      sc->F_new = sc->F + dF;
      return;
    }
    a *= bfac;
  }
  sc->alpha = 0.0;
}

template <typename T>
__global__ void armijo_update_kernel(int64_t p, T* __restrict__ th, const T* __restrict__ tt,
                                     const DevScalars* __restrict__ sc) {
  if (sc->accepted < 0) return;
  const double alpha = sc->alpha;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < p;
       m += (int64_t)gridDim.x * blockDim.x) {
    if (alpha == 1.0)
      th[m] = tt[m];
    else
      th[m] = T((double)th[m] + alpha * ((double)tt[m] - (double)th[m]));
  }
}

// ---------------------------------------------------------------- KKT / penalty / lambda_max
template <typename T>
__global__ void __launch_bounds__(kThreads)
kkt_kernel(int64_t p, const double* __restrict__ g, const T* __restrict__ th,
           const T* __restrict__ pw, double lambda, DevScalars* sc, RedScratch red, double l1,
           double l2) {
  double rmax = 0.0;
  double acc[2] = {0.0, 0.0};  // J(theta), nnz
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < p;
       m += (int64_t)gridDim.x * blockDim.x) {
    const double t = (double)th[m], thr = lambda * (double)pw[m], gm = g[m];
    double r;
    if (t != 0.0) {  // distance of -g to lambda dJ: J = sum w (l1 |t| + l2 t^2)
      r = fabs(gm + thr * (copysign(l1, t) + 2.0 * l2 * t));
      acc[1] += 1.0;
    } else {
      r = fmax(0.0, fabs(gm) - thr * l1);
    }
    rmax = fmax(rmax, r);
    acc[0] += (double)pw[m] * (l1 * fabs(t) + l2 * t * t);
  }
  block_sum<2>(acc);
  const double bm = block_max(rmax);
  if (threadIdx.x == 0) {
    red.partial[blockIdx.x * 3 + 0] = bm;
    red.partial[blockIdx.x * 3 + 1] = acc[0];
    red.partial[blockIdx.x * 3 + 2] = acc[1];
  }
  if (last_block(red.counter)) {
    if (threadIdx.x == 0) {
      double mx = 0.0, pen = 0.0, nnz = 0.0;
      for (unsigned int b = 0; b < gridDim.x; ++b) {
        mx = fmax(mx, __ldcg(&red.partial[b * 3 + 0]));
        pen += __ldcg(&red.partial[b * 3 + 1]);
        nnz += __ldcg(&red.partial[b * 3 + 2]);
      }
      sc->kkt_max = mx;
      sc->pen = pen;
      sc->nnz = (int)nnz;
      *red.counter = 0u;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kThreads)
lmax_kernel(int64_t p, const double* __restrict__ g0, const T* __restrict__ pw, DevScalars* sc,
            RedScratch red) {
  double mx = 0.0;
  for (int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; m < p;
       m += (int64_t)gridDim.x * blockDim.x)
    mx = fmax(mx, fabs(g0[m]) / (double)pw[m]);
  const double bm = block_max(mx);
  if (threadIdx.x == 0) red.partial[blockIdx.x] = bm;
  if (last_block(red.counter)) {
    if (threadIdx.x == 0) {
      double m2 = 0.0;
      for (unsigned int b = 0; b < gridDim.x; ++b) m2 = fmax(m2, __ldcg(&red.partial[b]));
      sc->lmax = m2;
      *red.counter = 0u;
    }
  }
}

__global__ void gram_kernel(int nj, int pj, const double* __restrict__ XT, double* __restrict__ gram) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= pj * pj) return;
  const int a = idx / pj, b = idx - a * pj;
  const double* xa = XT + (int64_t)a * nj;
  const double* xb = XT + (int64_t)b * nj;
  double s = 0.0;
  for (int i = 0; i < nj; ++i) s = fma(xa[i], xb[i], s);
  gram[idx] = s;
}

int grid_for(int64_t n) {
  int64_t b = (n + kThreads - 1) / kThreads;
  const int cap = 8 * num_sms();
  if (b > cap) b = cap;
  if (b < 1) b = 1;
  return (int)b;
}

}  // namespace

namespace {
std::atomic<int64_t> g_launches{0};
// a stream capture runs in one host thread; fits of a batch capture from several threads at once
thread_local int g_capturing = 0;
}  // namespace

void count_launches(int64_t k) {
  if (g_capturing == 0) g_launches.fetch_add(k, std::memory_order_relaxed);
}
int64_t launch_count() { return g_launches.load(); }
void set_capturing(bool on) { g_capturing = on ? 1 : 0; }

int num_sms() {
  static int cached = 0;
  if (cached == 0) {
    int dev = 0, v = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v <= 0)
      v = 152;
    cached = v;
  }
  return cached;
}

template <typename T, typename TV>
cudaError_t launch_family(int family, int64_t n, const T* eta, const T* Y, const T* A, TV* V, T* VZ,
                          T* U, double rho_prod, DevScalars* sc, RedScratch red, cudaStream_t s) {
  family_kernel<T, TV><<<red_blocks(n, kEPT), kThreads, 0, s>>>(family, n, eta, Y, A, V, VZ, U,
                                                                rho_prod, sc, red);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_loss_only(int family, int64_t n, const T* eta, const T* Y, const T* A,
                             double* out, RedScratch red, cudaStream_t s) {
  loss_kernel<T><<<red_blocks(n, kEPT), kThreads, 0, s>>>(family, n, eta, Y, A, out, red);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nll_cells(int family, int64_t n, const T* eta, const T* Y, const T* A,
                             const double* gout, T* U, T* GY, DevScalars* sc, RedScratch red,
                             cudaStream_t s) {
  nll_cells_kernel<T><<<red_blocks(n, kEPT), kThreads, 0, s>>>(family, n, eta, Y, A, gout, U, GY,
                                                               sc, red);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_nll_coef(int64_t p, const T* theta, const T* pen_w, double lambda,
                            const double* gout, const T* Q, T* grad, double* F, DevScalars* sc,
                            RedScratch red, cudaStream_t s) {
  nll_coef_kernel<T><<<red_blocks(p, 1), kThreads, 0, s>>>(p, theta, pen_w, lambda, gout, Q, grad,
                                                           F, sc, red);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_scale(int64_t n, const T* in, T* out, double scale, cudaStream_t s) {
  scale_kernel<T><<<grid_for(n), kThreads, 0, s>>>(n, in, out, T(scale));
  count_launches(1);
  return cudaGetLastError();
}

template <typename TI, typename TO>
cudaError_t launch_convert(int64_t n, const TI* in, TO* out, cudaStream_t s) {
  convert_kernel<TI, TO><<<grid_for(n), kThreads, 0, s>>>(n, in, out);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_extrap(int64_t n, const T* x, const T* xp, double omega, T* y, cudaStream_t s) {
  extrap_kernel<T><<<grid_for(n), kThreads, 0, s>>>(n, x, xp, omega, y);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_sum_splits(int64_t p, int ksplit, const T* part, T* out, cudaStream_t s) {
  sum_splits_kernel<T><<<grid_for(p), kThreads, 0, s>>>(p, ksplit, part, out);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_vmul(int64_t n, const T* V, T* x, const int* skip, cudaStream_t s) {
  vmul_kernel<T><<<grid_for(n), kThreads, 0, s>>>(n, V, x, skip);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_add(int64_t n, const T* x, T* y, const int* skip, cudaStream_t s) {
  add_kernel<T><<<grid_for(n), kThreads, 0, s>>>(n, x, y, skip);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_check_finite(int64_t n, const T* x, DevScalars* sc, cudaStream_t s) {
  finite_kernel<T><<<grid_for(n), kThreads, 0, s>>>(n, x, sc);
  count_launches(1);
  return cudaGetLastError();
}

template <typename Tq, typename TP>
cudaError_t launch_prox(int64_t p, int ksplit, const Tq* Qpart, const TP* lin, double lin_scale,
                        const TP* x, const TP* xprev, const TP* pen_w, TP* out, double inv_n,
                        InnerCtl* ctl, double omega, double delta, double lambda,
                        const double* Lhat, cudaStream_t s, Tq* dnext, const TP* anchor) {
  if (ksplit < 1 || ksplit > kMaxSplits) return cudaErrorInvalidValue;
  int blocks = (int)((p + kThreads - 1) / kThreads);
  if (blocks < 1) blocks = 1;
  if (blocks > 4 * num_sms()) blocks = 4 * num_sms();
  prox_kernel<Tq, TP><<<blocks, kThreads, 0, s>>>(p, ksplit, Qpart, lin, TP(lin_scale), x, xprev,
                                                  pen_w, out, TP(inv_n), ctl, TP(omega), TP(delta),
                                                  TP(lambda), Lhat, dnext, anchor);
  count_launches(1);
  return cudaGetLastError();
}

template <typename TE, typename T>
cudaError_t launch_armijo_stream(int family, int64_t n, const TE* eta, const T* deta, const TE* Y,
                                 const TE* A, double alpha0, double b, int j0, DevScalars* sc,
                                 RedScratch red, cudaStream_t s) {
  armijo_stream_kernel<TE, T><<<red_blocks(n, kEPT), kThreads, 0, s>>>(family, n, eta, deta, Y, A,
                                                                       alpha0, b, j0, sc, red);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_armijo_penalty(int64_t p, const T* theta, const T* theta_t, const T* pen_w,
                                  double alpha0, double b, int j0, DevScalars* sc, RedScratch red,
                                  cudaStream_t s, double l1, double l2) {
  armijo_penalty_kernel<T><<<red_blocks(p, 1), kThreads, 0, s>>>(p, theta, theta_t, pen_w, alpha0,
                                                                 b, j0, sc, red, l1, l2);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_armijo_select(double lambda, double v, double alpha0, double b, int j0,
                                 DevScalars* sc, cudaStream_t s) {
  armijo_select_kernel<<<1, 32, 0, s>>>(lambda, v, alpha0, b, j0, sc);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_armijo_update(int64_t p, T* theta, const T* theta_t, const DevScalars* sc,
                                 cudaStream_t s) {
  armijo_update_kernel<T><<<grid_for(p), kThreads, 0, s>>>(p, theta, theta_t, sc);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_kkt(int64_t p, const double* g, const T* theta, const T* pen_w, double lambda,
                       DevScalars* sc, RedScratch red, cudaStream_t s, double l1, double l2) {
  kkt_kernel<T><<<red_blocks(p, 1), kThreads, 0, s>>>(p, g, theta, pen_w, lambda, sc, red, l1, l2);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_penalty(int64_t p, const T* theta, const T* pen_w, DevScalars* sc,
                           RedScratch red, cudaStream_t s, double l1, double l2) {
  // J(theta) only: reuse the Armijo penalty kernel with theta~ = theta.
  armijo_penalty_kernel<T><<<red_blocks(p, 1), kThreads, 0, s>>>(p, theta, theta, pen_w, 1.0, 0.5,
                                                                 0, sc, red, l1, l2);
  count_launches(1);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lambda_max(int64_t p, const double* g0, const T* pen_w, DevScalars* sc,
                              RedScratch red, cudaStream_t s) {
  lmax_kernel<T><<<red_blocks(p, 1), kThreads, 0, s>>>(p, g0, pen_w, sc, red);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scad_weights(int64_t p, const double* theta, const double* base, double lambda,
                                double a, double* w, cudaStream_t s) {
  scad_weights_kernel<<<grid_for(p), kThreads, 0, s>>>(p, theta, base, lambda, a, w);
  count_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_gram(int nj, int pj, const double* XT, double* gram, cudaStream_t s) {
  const int tot = pj * pj;
  gram_kernel<<<(tot + kThreads - 1) / kThreads, kThreads, 0, s>>>(nj, pj, XT, gram);
  count_launches(1);
  return cudaGetLastError();
}

#define GLAM_INST(T)                                                                              \
  template cudaError_t launch_loss_only<T>(int, int64_t, const T*, const T*, const T*, double*,   \
                                           RedScratch, cudaStream_t);                             \
  template cudaError_t launch_scale<T>(int64_t, const T*, T*, double, cudaStream_t);              \
  template cudaError_t launch_nll_cells<T>(int, int64_t, const T*, const T*, const T*,           \
                                           const double*, T*, T*, DevScalars*, RedScratch,         \
                                           cudaStream_t);                                          \
  template cudaError_t launch_nll_coef<T>(int64_t, const T*, const T*, double, const double*,     \
                                          const T*, T*, double*, DevScalars*, RedScratch,          \
                                          cudaStream_t);                                           \
  template cudaError_t launch_check_finite<T>(int64_t, const T*, DevScalars*, cudaStream_t);      \
  template cudaError_t launch_vmul<T>(int64_t, const T*, T*, const int*, cudaStream_t);           \
  template cudaError_t launch_add<T>(int64_t, const T*, T*, const int*, cudaStream_t);            \
  template cudaError_t launch_sum_splits<T>(int64_t, int, const T*, T*, cudaStream_t);            \
  template cudaError_t launch_armijo_penalty<T>(int64_t, const T*, const T*, const T*, double,    \
                                                double, int, DevScalars*, RedScratch,             \
                                                cudaStream_t, double, double);                    \
  template cudaError_t launch_armijo_update<T>(int64_t, T*, const T*, const DevScalars*,          \
                                               cudaStream_t);                                     \
  template cudaError_t launch_kkt<T>(int64_t, const double*, const T*, const T*, double,          \
                                     DevScalars*, RedScratch, cudaStream_t, double, double);      \
  template cudaError_t launch_penalty<T>(int64_t, const T*, const T*, DevScalars*, RedScratch,    \
                                         cudaStream_t, double, double);                           \
  template cudaError_t launch_lambda_max<T>(int64_t, const double*, const T*, DevScalars*,        \
                                            RedScratch, cudaStream_t);

GLAM_INST(float)
GLAM_INST(double)
#undef GLAM_INST

template cudaError_t launch_family<float, float>(int, int64_t, const float*, const float*,
                                                 const float*, float*, float*, float*, double,
                                                 DevScalars*, RedScratch, cudaStream_t);
template cudaError_t launch_family<double, double>(int, int64_t, const double*, const double*,
                                                   const double*, double*, double*, double*, double,
                                                   DevScalars*, RedScratch, cudaStream_t);
template cudaError_t launch_family<double, float>(int, int64_t, const double*, const double*,
                                                  const double*, float*, double*, double*, double,
                                                  DevScalars*, RedScratch, cudaStream_t);
template cudaError_t launch_family<double, __nv_bfloat16>(int, int64_t, const double*, const double*,
                                                          const double*, __nv_bfloat16*, double*, double*,
                                                          double, DevScalars*, RedScratch, cudaStream_t);
#define GLAM_PROX_INST(Tq, TP)                                                                  \
  template cudaError_t launch_prox<Tq, TP>(int64_t, int, const Tq*, const TP*, double, const TP*,  \
                                           const TP*, const TP*, TP*, double, InnerCtl*, double,  \
                                           double, double, const double*, cudaStream_t, Tq*,      \
                                           const TP*);
GLAM_PROX_INST(float, float)
GLAM_PROX_INST(double, double)
GLAM_PROX_INST(float, double)
#undef GLAM_PROX_INST
template cudaError_t launch_armijo_stream<double, float>(int, int64_t, const double*, const float*,
                                                         const double*, const double*, double,
                                                         double, int, DevScalars*, RedScratch,
                                                         cudaStream_t);
template cudaError_t launch_armijo_stream<double, double>(int, int64_t, const double*,
                                                          const double*, const double*,
                                                          const double*, double, double, int,
                                                          DevScalars*, RedScratch, cudaStream_t);

template cudaError_t launch_convert<float, double>(int64_t, const float*, double*, cudaStream_t);
template cudaError_t launch_convert<double, float>(int64_t, const double*, float*, cudaStream_t);
template cudaError_t launch_convert<double, double>(int64_t, const double*, double*, cudaStream_t);
template cudaError_t launch_convert<float, float>(int64_t, const float*, float*, cudaStream_t);
template cudaError_t launch_extrap<float>(int64_t, const float*, const float*, double, float*, cudaStream_t);

}  // namespace glam
