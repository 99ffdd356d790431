// C ABI of libglam (include/glam.h): plans, the array transforms H and G, the standalone
// entry points and the warm-started GD-PG lambda path (Alg. 1, Sec. 3; Sec. 6.1 and 6.4).
//
// Mode order (the Kronecker algebra of App. A leaves it free): H contracts mode 3, then mode 1,
// then mode 2; G runs the reverse.  Mode 2 is the fused mode of the bottleneck kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "glam_host_math.h"
#include "glam_internal.cuh"

using namespace glam;

namespace {

thread_local std::string g_thread_err;
constexpr uint64_t kDefaultWaitNs = 2000000000ull;  // bounded device waits: 2 s unless a fit says otherwise

template <typename T>
struct Work {
  T *Ta = nullptr, *Tb = nullptr, *Sb = nullptr, *Qpart = nullptr;
  T *eta = nullptr, *eta_bar = nullptr, *V = nullptr, *VZ = nullptr, *U = nullptr;
  T *x0 = nullptr, *x1 = nullptr, *theta = nullptr, *theta_t = nullptr, *b = nullptr,
    *grad = nullptr;
  T* Xc[3] = {nullptr, nullptr, nullptr};  // converted copies of the marginal designs
  T *Yc = nullptr, *Wc = nullptr, *penc = nullptr;
  T* one = nullptr;                        // the 1 x 1 design of a d = 2 problem
  T* dn = nullptr;                         // y - theta_k of the next inner iteration (p)
  T* yx = nullptr;                         // extrapolated point of a standalone prox step (p)
  // tensor-product weights (Sec. 6.2): M_j = X_j^T W_j X_j in the working precision and the
  // p-space intermediates of H(<M_j>, d)
  T* Mk[3] = {nullptr, nullptr, nullptr};
  T *kTa = nullptr, *kTb = nullptr, *kQ = nullptr;
  bool ready = false;
};

}  // namespace

constexpr int kMaxComp = 8;  // components of a plan of the model with c > 1 (Eq. fivenew), at most

struct glam_plan {
  int device = 0;
  // c > 1 components: the transforms of component r run on the single-component plan sub[r]
  // (its own workspace); this plan holds the n-space arrays and the concatenated p-space state,
  // component r's coefficients at [poff[r], poff[r + 1])
  int nc = 1;
  glam_plan* sub[kMaxComp] = {};
  int64_t poff[kMaxComp + 1] = {};
  cudaStream_t stream = nullptr;   // caller's stream
  cudaStream_t work = nullptr;     // private stream (graph capture needs a capturable stream)
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  glam_dims dims{};
  int family = 0, precision = 0;
  int64_t n1 = 1, n2 = 1, n3 = 1, p1 = 1, p2 = 1, p3 = 1, n = 1, p = 1;
  int ksplit = 1;
  bool fused[2] = {false, false};  // [float, double]: the fused slab kernel applies
  // form of the tensor-core fused kernel for this plan: 1 (TF32 plans: TF32 operands), 3 (FP32
  // plans: 3xTF32, about FP32 accuracy), 0 when the shape is outside its domain or the plan is FP64
  int tc_split = 0;
  float* tc_cst = nullptr;  // the tensor-core kernel's constant block (X_1, X_2 in its layouts)
  // form of the tcgen05 kernel of the inner-loop product (1 TF32, 3 3xTF32, 16 BF16), 0 when the
  // shape is outside its domain (the warp-level tensor-core kernel above, or SIMT, serves then)
  int um_form = 0;
  void* um_cst = nullptr;          // its constant block
  __nv_bfloat16* Vb = nullptr;     // BF16 plans: the IRLS weights of the fit path in BF16 (n)
  std::string err;
  Work<float> wf;
  Work<double> wd;
  // p-space state of the fit path, always FP64: theta, the two FISTA buffers, grad f(theta_k),
  // the penalty weights and a scratch vector
  double *th = nullptr, *x0 = nullptr, *x1 = nullptr, *gk = nullptr, *pen = nullptr, *ptmp = nullptr;
  InnerCtl* ctl = nullptr;
  DevScalars* sc = nullptr;
  RedScratch red{};
  InnerCtl* h_ctl = nullptr;
  DevScalars* h_sc = nullptr;
  double* h_gram = nullptr;
  double* d_gram = nullptr;        // p_j x p_j Gram scratch (p_j <= 64)
  double* kfac[3] = {nullptr, nullptr, nullptr};  // factors of a tensor-product W (n_j each)
  double* kgram = nullptr;         // the FP64 weighted Gram matrices, p1^2 + p2^2 + p3^2
  double* pen_base = nullptr;      // the caller's penalty weights during a SCAD fit (p)
  unsigned long long* kcheck = nullptr;
  double* geo = nullptr;           // scratch of the geometric-mean weight factors
  // banded form of the marginal designs, used by the FP64 transforms while a fit that asked for it
  // (glam_opts.exploit_bands) runs
  bool band_on = false;
  BandDesign band[3];
  int* x3rows = nullptr;           // per row j3 of X_3^T the range of its nonzero entries (2 p3)
  std::vector<void*> allocs;
};

namespace {

int fail(glam_plan* pl, int code, const std::string& msg) {
  if (pl)
    pl->err = msg;
  else
    g_thread_err = msg;
  return code;
}

#define CK(...)                                                                             \
  do {                                                                                      \
    cudaError_t e_ = (__VA_ARGS__);                                                         \
    if (e_ != cudaSuccess)                                                                  \
      return fail(pl, GLAM_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define CKS(call)                                 \
  do {                                            \
    int s_ = (call);                              \
    if (s_ != GLAM_OK) return s_;                 \
  } while (0)

template <typename T>
int dalloc(glam_plan* pl, T** ptr, size_t count) {
  if (count == 0) count = 1;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(pl, GLAM_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  pl->allocs.push_back(p);
  *ptr = static_cast<T*>(p);
  return GLAM_OK;
}

// ---------------------------------------------------------------- GEMM descriptors (rho)
GemmDesc mk(int M, int N, int K, int batch, int ksplit, int64_t sAb, int64_t sAm, int64_t sAk,
            int64_t sBb, int64_t sBk, int64_t sBn, int64_t sCb, int64_t sCm, int64_t sCn,
            int64_t sCs) {
  GemmDesc d;
  d.M = M; d.N = N; d.K = K; d.batch = batch; d.ksplit = ksplit;
  d.sAb = sAb; d.sAm = sAm; d.sAk = sAk;
  d.sBb = sBb; d.sBk = sBk; d.sBn = sBn;
  d.sCb = sCb; d.sCm = sCm; d.sCn = sCn; d.sCsplit = sCs;
  return d;
}
// H stage 1: T_a (n3 x p2p1) = X_3 (n3 x p3) . Theta (p3 x p2p1)
GemmDesc d_mode3_fwd(const glam_plan* pl) {
  const int64_t P21 = pl->p2 * pl->p1;
  return mk((int)pl->n3, (int)P21, (int)pl->p3, 1, 1, 0, 1, pl->n3, 0, P21, 1, 0, P21, 1, 0);
}
// H stage 2: T_b (n3 p2 x n1) = T_a (n3 p2 x p1) . X_1^T (p1 x n1)
GemmDesc d_mode1_fwd(const glam_plan* pl) {
  return mk((int)(pl->n3 * pl->p2), (int)pl->n1, (int)pl->p1, 1, 1, 0, pl->p1, 1, 0, pl->n1, 1, 0,
            pl->n1, 1, 0);
}
// H stage 3: eta[i3] (n2 x n1) = X_2 (n2 x p2) . T_b[i3] (p2 x n1)
GemmDesc d_mode2_fwd(const glam_plan* pl) {
  return mk((int)pl->n2, (int)pl->n1, (int)pl->p2, (int)pl->n3, 1, 0, 1, pl->n2, pl->p2 * pl->n1,
            pl->n1, 1, pl->n2 * pl->n1, pl->n1, 1, 0);
}
// G stage 1: S[i3] (p2 x n1) = X_2^T (p2 x n2) . U[i3] (n2 x n1)
GemmDesc d_mode2_adj(const glam_plan* pl) {
  return mk((int)pl->p2, (int)pl->n1, (int)pl->n2, (int)pl->n3, 1, 0, pl->n2, 1, pl->n2 * pl->n1,
            pl->n1, 1, pl->p2 * pl->n1, pl->n1, 1, 0);
}
// G stage 2: S_b (n3 p2 x p1) = S (n3 p2 x n1) . X_1 (n1 x p1)
GemmDesc d_mode1_adj(const glam_plan* pl) {
  return mk((int)(pl->n3 * pl->p2), (int)pl->p1, (int)pl->n1, 1, 1, 0, pl->n1, 1, 0, 1, pl->n1, 0,
            pl->p1, 1, 0);
}
// G stage 3: Q (p3 x p2p1) = X_3^T (p3 x n3) . S_b (n3 x p2p1), optionally split over i3
GemmDesc d_mode3_adj(const glam_plan* pl, int ksplit) {
  const int64_t P21 = pl->p2 * pl->p1;
  return mk((int)pl->p3, (int)P21, (int)pl->n3, 1, ksplit, 0, pl->n3, 1, 0, P21, 1, 0, P21, 1,
            pl->p3 * P21);
}

// H(<M_j>, d) with the p_j x p_j matrices M_j of tensor-product weights: the three forward
// stages above with every n_j replaced by p_j (M_j is stored like a design, as (p_j, p_j))
GemmDesc k_mode3_fwd(const glam_plan* pl) {
  const int64_t P21 = pl->p2 * pl->p1;
  return mk((int)pl->p3, (int)P21, (int)pl->p3, 1, 1, 0, 1, pl->p3, 0, P21, 1, 0, P21, 1, 0);
}
GemmDesc k_mode1_fwd(const glam_plan* pl) {
  return mk((int)(pl->p3 * pl->p2), (int)pl->p1, (int)pl->p1, 1, 1, 0, pl->p1, 1, 0, pl->p1, 1, 0,
            pl->p1, 1, 0);
}
GemmDesc k_mode2_fwd(const glam_plan* pl) {
  return mk((int)pl->p2, (int)pl->p1, (int)pl->p2, (int)pl->p3, 1, 0, 1, pl->p2, pl->p2 * pl->p1,
            pl->p1, 1, pl->p2 * pl->p1, pl->p1, 1, 0);
}

template <typename T>
Work<T>& work_of(glam_plan* pl);
template <>
Work<float>& work_of<float>(glam_plan* pl) { return pl->wf; }
template <>
Work<double>& work_of<double>(glam_plan* pl) { return pl->wd; }

template <typename T>
struct Ops {
  glam_plan* pl;
  Work<T>& w;
  cudaStream_t s;
  const T* X[3 * kMaxComp];  // 3 designs per component

  Ops(glam_plan* p, cudaStream_t st, const void* const Xin[3])
      : pl(p), w(work_of<T>(p)), s(st) {
    for (int r = 0; r < pl->nc; ++r) {
      for (int j = 0; j < 3; ++j) X[3 * r + j] = static_cast<const T*>(Xin[3 * r + j]);
      if (X[3 * r + 2] == nullptr) X[3 * r + 2] = pl->nc > 1 ? work_of<T>(pl->sub[r]).one : w.one;
    }
  }
  // the transforms of component r (c > 1): its own plan, designs and workspace
  Ops sub(int r) const { return Ops(pl->sub[r], s, reinterpret_cast<const void* const*>(X + 3 * r)); }

  // eta = H(<X_j>, Theta)   (Sec. 6.1, Eq. eighteen); c > 1: the sum over the components, each
  // component's term formed in its own plan's n-array and added
  int H(const T* theta, T* eta) {
    if constexpr (sizeof(T) == 8) {
      if (pl->band_on) {  // modes 3, 1, 2 as banded products (4 terms per output)
        const int64_t P21 = pl->p2 * pl->p1;
        CK(launch_band_fwd(1, (int)pl->p3, (int)pl->n3, P21, pl->band[2], theta, w.Ta, s));
        CK(launch_band_fwd(pl->n3 * pl->p2, (int)pl->p1, (int)pl->n1, 1, pl->band[0], w.Ta, w.Tb, s));
        CK(launch_band_fwd(pl->n3, (int)pl->p2, (int)pl->n2, pl->n1, pl->band[1], w.Tb, eta, s));
        return GLAM_OK;
      }
    }
    if (pl->nc > 1) {
      for (int r = 0; r < pl->nc; ++r) {
        Ops o = sub(r);
        T* dst = r == 0 ? eta : o.w.eta;
        CKS(o.H(theta + pl->poff[r], dst));
        if (r > 0) CK(launch_add<T>(pl->n, dst, eta, nullptr, s));
      }
      return GLAM_OK;
    }
    if constexpr (sizeof(T) == 4) {
      if (predict_umma_supported((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2, (int)pl->p3)) {
        CK(launch_predict_umma((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2, (int)pl->p3, X[0],
                               X[1], X[2], theta, eta, &pl->sc->timeout, s));
        return GLAM_OK;
      }
      if (predict_tiles_supported((int)pl->p1, (int)pl->p2) && mode3_rows_supported((int)pl->p3)) {
        CK(launch_mode3_rows((int)pl->n3, (int)pl->p3, (int)(pl->p2 * pl->p1), X[2], theta, w.Ta, s));
        CK(launch_predict_tiles((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2,
                                X[0], X[1], w.Ta, eta, s));
        return GLAM_OK;
      }
    }
    CK(launch_gemm<T, T>(d_mode3_fwd(pl), X[2], theta, w.Ta, s));
    CK(launch_gemm<T, T>(d_mode1_fwd(pl), w.Ta, X[0], w.Tb, s));
    CK(launch_gemm<T, T>(d_mode2_fwd(pl), X[1], w.Tb, eta, s));
    return GLAM_OK;
  }
  // out = G(<X_j>, U)   (Sec. 6.1, Eq. nineteen); c > 1: component r's block at poff[r]
  int G(const T* U, T* out) {
    if constexpr (sizeof(T) == 8) {
      if (pl->band_on) {  // modes 2, 1, 3 as banded adjoint products
        const int64_t P21 = pl->p2 * pl->p1;
        CK(launch_band_adj(pl->n3, (int)pl->n2, (int)pl->p2, pl->n1, pl->band[1], U, w.Tb, s));
        CK(launch_band_adj(pl->n3 * pl->p2, (int)pl->n1, (int)pl->p1, 1, pl->band[0], w.Tb, w.Sb, s));
        CK(launch_band_adj(1, (int)pl->n3, (int)pl->p3, P21, pl->band[2], w.Sb, out, s));
        return GLAM_OK;
      }
    }
    if (pl->nc > 1) {
      for (int r = 0; r < pl->nc; ++r) CKS(sub(r).G(U, out + pl->poff[r]));
      return GLAM_OK;
    }
    CK(launch_gemm<T, T>(d_mode2_adj(pl), X[1], U, w.Tb, s));
    CK(launch_gemm<T, T>(d_mode1_adj(pl), w.Tb, X[0], w.Sb, s));
    if (pl->ksplit > 1) {
      CK(launch_gemm<T, T>(d_mode3_adj(pl, pl->ksplit), X[2], w.Sb, w.Qpart, s));
      CK(launch_sum_splits<T>(pl->p, pl->ksplit, w.Qpart, out, s));
    } else {
      CK(launch_gemm<T, T>(d_mode3_adj(pl, 1), X[2], w.Sb, out, s));
    }
    return GLAM_OK;
  }
  // eta = H(<X_j>, x - sub) for a parameter array held in TB (the correction of a refinement)
  template <typename TB>
  int H_diff(const TB* x, const TB* sub, T* eta) {
    if (pl->nc > 1) {
      for (int r = 0; r < pl->nc; ++r) {
        Ops o = this->sub(r);
        T* dst = r == 0 ? eta : o.w.eta;
        CKS(o.H_diff(x + pl->poff[r], sub + pl->poff[r], dst));
        if (r > 0) CK(launch_add<T>(pl->n, dst, eta, nullptr, s));
      }
      return GLAM_OK;
    }
    CK(launch_gemm<T, TB>(d_mode3_fwd(pl), X[2], x, w.Ta, s, nullptr, sub, nullptr, 0.0, nullptr));
    CK(launch_gemm<T, T>(d_mode1_fwd(pl), w.Ta, X[0], w.Tb, s));
    CK(launch_gemm<T, T>(d_mode2_fwd(pl), X[1], w.Tb, eta, s));
    return GLAM_OK;
  }
  // Qpart = partial sums of G(V (.) H(y - sub)), y = x + omega (x - x_prev)  (Eq. twentysixnew);
  // with xp = sub = nullptr the operand x is used as it is.
  template <typename TB>
  int XtWX(const TB* x, const TB* xp, const TB* sub, const T* V, const InnerCtl* ctl,
           double omega, const int* skip) {
    if (pl->nc > 1) {
      // c > 1 (Eq. twentysixnew with r = 1..c): eta = sum_r H_r(y_r - sub_r) in this plan's
      // n-array, V (.) eta, then G_r of it into component r's block of Qpart (ksplit = 1)
      T* acc = w.eta_bar;
      for (int r = 0; r < pl->nc; ++r) {
        Ops o = this->sub(r);
        glam_plan* q = pl->sub[r];
        const int64_t off = pl->poff[r];
        T* dst = r == 0 ? acc : o.w.eta_bar;
        CK(launch_gemm<T, TB>(d_mode3_fwd(q), o.X[2], x + off, o.w.Ta, s, xp ? xp + off : nullptr,
                              sub ? sub + off : nullptr, ctl, omega, skip));
        CK(launch_gemm<T, T>(d_mode1_fwd(q), o.w.Ta, o.X[0], o.w.Tb, s, nullptr, nullptr, nullptr, 0.0, skip));
        CK(launch_gemm<T, T>(d_mode2_fwd(q), o.X[1], o.w.Tb, dst, s, nullptr, nullptr, nullptr, 0.0, skip));
        if (r > 0) CK(launch_add<T>(pl->n, dst, acc, skip, s));
      }
      CK(launch_vmul<T>(pl->n, V, acc, skip, s));
      for (int r = 0; r < pl->nc; ++r) {
        Ops o = this->sub(r);
        glam_plan* q = pl->sub[r];
        CK(launch_gemm<T, T>(d_mode2_adj(q), o.X[1], acc, o.w.Tb, s, nullptr, nullptr, nullptr, 0.0, skip));
        CK(launch_gemm<T, T>(d_mode1_adj(q), o.w.Tb, o.X[0], o.w.Sb, s, nullptr, nullptr, nullptr, 0.0, skip));
        CK(launch_gemm<T, T>(d_mode3_adj(q, q->ksplit), o.X[2], o.w.Sb, o.w.Qpart, s, nullptr, nullptr,
                             nullptr, 0.0, skip));
        CK(launch_sum_splits<T>(q->p, q->ksplit, o.w.Qpart, w.Qpart + pl->poff[r], s));
      }
      return GLAM_OK;
    }
    if constexpr (sizeof(T) == 4 && sizeof(TB) == 4) {
      if (pl->um_form && sub == nullptr && ctl == nullptr && fused_tc_pointers_ok((const float*)pl->um_cst, w.yx, V)) {
        // tcgen05 kernel: it forms T_a = X_3 y from the extrapolated point itself
        CK(launch_extrap<T>(pl->p, x, xp, omega, w.yx, s));
        CK(launch_fused_umma_const((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2,
                                   (int)pl->p3, pl->um_form, X[0], X[1], pl->um_cst, s));
        CK(launch_fused_umma((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2, (int)pl->p3,
                             pl->um_form, false, pl->um_cst, w.yx, X[0], X[2], V, w.Sb, s, skip,
                             &pl->sc->timeout, kDefaultWaitNs));
        CK(launch_gemm<T, T>(d_mode3_adj(pl, pl->ksplit), X[2], w.Sb, w.Qpart, s, nullptr, nullptr,
                             nullptr, 0.0, skip));
        return GLAM_OK;
      }
      if (pl->tc_split && sub == nullptr && ctl == nullptr && fused_tc_pointers_ok(pl->tc_cst, w.yx, V)) {
        // tensor-core kernel: it forms T_a = X_3 y from the extrapolated point itself
        CK(launch_extrap<T>(pl->p, x, xp, omega, w.yx, s));
        CK(launch_fused_tc_const((int)pl->n1, (int)pl->n2, (int)pl->p1, (int)pl->p2, X[0], X[1],
                                 pl->tc_cst, pl->tc_split, s));
        CK(launch_fused_slab_tc((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2,
                                (int)pl->p3, pl->tc_cst, w.yx, V, w.Sb, s, skip, &pl->sc->timeout,
                                X[2], pl->tc_split));
        CK(launch_gemm<T, T>(d_mode3_adj(pl, pl->ksplit), X[2], w.Sb, w.Qpart, s, nullptr, nullptr,
                             nullptr, 0.0, skip));
        return GLAM_OK;
      }
    }
    CK(launch_gemm<T, TB>(d_mode3_fwd(pl), X[2], x, w.Ta, s, xp, sub, ctl, omega, skip));
    if (pl->fused[sizeof(T) == 8 ? 1 : 0]) {
      CK(launch_fused_slab<T>((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2,
                              X[0], X[1], w.Ta, V, w.Sb, s, skip, &pl->sc->timeout));
    } else {
      T* tmp = w.eta_bar;
      CK(launch_gemm<T, T>(d_mode1_fwd(pl), w.Ta, X[0], w.Tb, s, nullptr, nullptr, nullptr, 0.0, skip));
      CK(launch_gemm<T, T>(d_mode2_fwd(pl), X[1], w.Tb, tmp, s, nullptr, nullptr, nullptr, 0.0, skip));
      CK(launch_vmul<T>(pl->n, V, tmp, skip, s));
      CK(launch_gemm<T, T>(d_mode2_adj(pl), X[1], tmp, w.Tb, s, nullptr, nullptr, nullptr, 0.0, skip));
      CK(launch_gemm<T, T>(d_mode1_adj(pl), w.Tb, X[0], w.Sb, s, nullptr, nullptr, nullptr, 0.0, skip));
    }
    CK(launch_gemm<T, T>(d_mode3_adj(pl, pl->ksplit), X[2], w.Sb, w.Qpart, s, nullptr, nullptr,
                         nullptr, 0.0, skip));
    return GLAM_OK;
  }
};

template <typename T>
int alloc_work(glam_plan* pl, Work<T>& w, bool full) {
  const int64_t n = pl->n, p = pl->p;
  const int64_t ta = pl->n3 * pl->p2 * pl->p1;
  const int64_t tb = pl->n3 * pl->p2 * pl->n1;
  CKS(dalloc(pl, &w.Ta, ta));
  CKS(dalloc(pl, &w.Tb, tb));
  CKS(dalloc(pl, &w.Sb, ta));
  CKS(dalloc(pl, &w.Qpart, (size_t)pl->ksplit * p));
  CKS(dalloc(pl, &w.eta, n));
  CKS(dalloc(pl, &w.U, n));
  CKS(dalloc(pl, &w.theta, p));
  CKS(dalloc(pl, &w.grad, p));
  CKS(dalloc(pl, &w.dn, p));
  CKS(dalloc(pl, &w.yx, p));
  CKS(dalloc(pl, &w.one, 1));
  const T one = T(1);
  CK(cudaMemcpy(w.one, &one, sizeof(T), cudaMemcpyHostToDevice));
  if (full) {
    CKS(dalloc(pl, &w.eta_bar, n));
    CKS(dalloc(pl, &w.V, n));
    CKS(dalloc(pl, &w.VZ, n));
    CKS(dalloc(pl, &w.x0, p));
    CKS(dalloc(pl, &w.x1, p));
    CKS(dalloc(pl, &w.theta_t, p));
    CKS(dalloc(pl, &w.b, p));
  }
  w.ready = true;
  return GLAM_OK;
}

// X holds 3 design pointers per component (X_r1, X_r2, X_r3 of component r at 3r .. 3r + 2)
int validate_X(glam_plan* pl, const void* const X[3]) {
  if (X == nullptr) return fail(pl, GLAM_EINVAL, "X: NULL design pointer");
  for (int r = 0; r < pl->nc; ++r) {
    if (X[3 * r] == nullptr || X[3 * r + 1] == nullptr) return fail(pl, GLAM_EINVAL, "X: NULL design pointer");
    if (pl->dims.d == 3 && X[3 * r + 2] == nullptr) return fail(pl, GLAM_EINVAL, "X: NULL X_3 with d = 3");
  }
  return GLAM_OK;
}

// entry points that take one component only
int single_component(glam_plan* pl, const char* what) {
  if (pl->nc > 1)
    return fail(pl, GLAM_EINVAL, std::string(what) + ": not available for a plan with c > 1 components");
  return GLAM_OK;
}

int check_plan(glam_plan* pl) {
  if (pl == nullptr) return fail(nullptr, GLAM_EINVAL, "NULL plan");
  pl->err.clear();
  return GLAM_OK;
}

}  // namespace

namespace glam {
int thread_fail(int code, const std::string& msg) { return fail(nullptr, code, msg); }
int plan_components(const glam_plan* pl) { return pl->nc; }
}  // namespace glam

// ======================================================================== ABI
// (every entry point is declared extern "C" in glam.h, so these definitions have C linkage)

int glam_opts_default(glam_opts* o) {
  if (o == nullptr) return fail(nullptr, GLAM_EINVAL, "glam_opts_default: NULL");
  std::memset(o, 0, sizeof(*o));
  o->tol = 1e-6;
  o->lambda_min_ratio = 1e-3;
  o->inner_forcing = 1e-2;
  o->inner_floor = 0.1;
  o->armijo_alpha0 = 1.0;
  o->armijo_b = 0.5;
  o->armijo_v = 0.1;
  o->max_inner = 50000;
  o->max_outer = 50;
  o->max_linesearch = 30;
  o->check_every = 32;
  o->iwls = GLAM_IWLS_EXACT;
  o->penalty = GLAM_PENALTY_LASSO;
  o->steps = 1;
  o->wait_limit_s = 2.0;
  o->nu = 1.0;
  return GLAM_OK;
}

int glam_plan_create(const glam_dims* dims, int family, int precision, void* stream,
                     glam_plan** out) {
  glam_plan* pl = nullptr;
  if (out == nullptr || dims == nullptr) return fail(nullptr, GLAM_EINVAL, "glam_plan_create: NULL argument");
  *out = nullptr;
  if (!(dims->d == 2 || dims->d == 3)) return fail(nullptr, GLAM_EINVAL, "dims.d must be 2 or 3");
  for (int j = 0; j < 3; ++j)
    if (dims->n[j] < 1 || dims->p[j] < 1)
      return fail(nullptr, GLAM_EINVAL, "dims: every n_j and p_j must be >= 1");
  if (dims->d == 2 && (dims->n[2] != 1 || dims->p[2] != 1))
    return fail(nullptr, GLAM_EINVAL, "dims: d = 2 needs n3 = p3 = 1");
  if (family != GLAM_GAUSSIAN_IDENTITY && family != GLAM_POISSON_LOG && family != GLAM_BINOMIAL_LOGIT &&
      family != GLAM_GAMMA_LOG)
    return fail(nullptr, GLAM_EINVAL, "unknown family");
  if (precision != GLAM_FP64 && precision != GLAM_FP32 && precision != GLAM_TF32 && precision != GLAM_BF16)
    return fail(nullptr, GLAM_EINVAL, "precision: GLAM_FP64, GLAM_FP32, GLAM_TF32 or GLAM_BF16");
  // the products are formed only once each factor is known to keep them below 2^40 (no int64
  // overflow can slip a huge shape past the limit)
  const int64_t kLim = (int64_t)1 << 40;
  int64_t n = 1, p = 1;
  for (int j = 0; j < 3; ++j) {
    if (dims->n[j] > kLim / n || dims->p[j] > kLim / p)
      return fail(nullptr, GLAM_EINVAL, "dims too large: n1 n2 n3 and p1 p2 p3 must not exceed 2^40");
    n *= dims->n[j];
    p *= dims->p[j];
  }
  if (dims->n[2] > 65535 || dims->n[2] * dims->p[1] > 65535LL * 64)
    return fail(nullptr, GLAM_EINVAL, "dims too large");
  pl = new (std::nothrow) glam_plan();
  if (pl == nullptr) return fail(nullptr, GLAM_ENOMEM, "host allocation failed");
  pl->dims = *dims;
  pl->family = family;
  pl->precision = precision;
  pl->stream = static_cast<cudaStream_t>(stream);
  pl->n1 = dims->n[0]; pl->n2 = dims->n[1]; pl->n3 = dims->n[2];
  pl->p1 = dims->p[0]; pl->p2 = dims->p[1]; pl->p3 = dims->p[2];
  pl->n = n;
  pl->p = p;
  auto bail = [&](int code) {
    std::string m = pl->err;
    glam_plan_destroy(pl);
    g_thread_err = m;
    return code;
  };
  if (cudaGetDevice(&pl->device) != cudaSuccess) { pl->err = "cudaGetDevice failed"; return bail(GLAM_ECUDA); }
  {
    const cudaError_t e = fused_prepare();
    if (e != cudaSuccess) {
      pl->err = std::string("fused kernel set-up (cudaFuncSetAttribute): ") + cudaGetErrorString(e);
      return bail(GLAM_ECUDA);
    }
  }
  // split of the last G stage over i3 so that the small p3 x p2p1 output still fills the GPU
  {
    int64_t ks = (pl->n3 + 63) / 64;  // at most 64 rows of i3 per split: one staged K step
    if (ks < 1) ks = 1;
    if (ks > kMaxSplits) ks = kMaxSplits;
    pl->ksplit = (int)ks;
  }
  pl->fused[0] = fused_slab_supported((int)pl->n1, (int)pl->n2, (int)pl->p1, (int)pl->p2, 4) != 0;
  pl->fused[1] = fused_slab_supported((int)pl->n1, (int)pl->n2, (int)pl->p1, (int)pl->p2, 8) != 0;
  if (precision != GLAM_FP64) {
    const cudaError_t e = fused_tc_prepare();
    if (e != cudaSuccess) {
      pl->err = std::string("tensor-core kernel set-up (cudaFuncSetAttribute): ") + cudaGetErrorString(e);
      return bail(GLAM_ECUDA);
    }
    const cudaError_t e2 = fused_umma_prepare();
    if (e2 != cudaSuccess) {
      pl->err = std::string("tcgen05 kernel set-up (cudaFuncSetAttribute): ") + cudaGetErrorString(e2);
      return bail(GLAM_ECUDA);
    }
    // the tcgen05 kernel where the shape allows; otherwise the warp-level tensor-core kernel (TF32
    // operands for TF32 and BF16 plans, 3xTF32 for FP32 plans) or the FP32 SIMT kernel
    const int form = precision == GLAM_TF32 ? 1 : (precision == GLAM_BF16 ? 16 : 3);
    if (fused_umma_supported((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2, (int)pl->p3, form)) {
      pl->um_form = form;
    } else {
      const int split = precision == GLAM_FP32 ? 3 : 1;
      if (fused_tc_supported((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2, (int)pl->p3,
                             split))
        pl->tc_split = split;
    }
  }
  int st;
  if (precision == GLAM_FP64) {
    if ((st = alloc_work<double>(pl, pl->wd, true)) != GLAM_OK) return bail(st);
  } else {
    if ((st = alloc_work<float>(pl, pl->wf, true)) != GLAM_OK) return bail(st);
    if ((st = alloc_work<double>(pl, pl->wd, true)) != GLAM_OK) return bail(st);
    for (int j = 0; j < 3; ++j)
      if ((st = dalloc(pl, &pl->wd.Xc[j], (size_t)dims->n[j] * dims->p[j])) != GLAM_OK) return bail(st);
    if ((st = dalloc(pl, &pl->wd.Yc, n)) != GLAM_OK) return bail(st);
    if ((st = dalloc(pl, &pl->wd.Wc, n)) != GLAM_OK) return bail(st);
  }
  for (double** v : {&pl->th, &pl->x0, &pl->x1, &pl->gk, &pl->pen, &pl->ptmp})
    if ((st = dalloc(pl, v, p)) != GLAM_OK) return bail(st);
  if ((st = dalloc(pl, &pl->d_gram, 4096)) != GLAM_OK) return bail(st);
  if (pl->tc_split) {
    const int64_t nc = fused_tc_const_floats((int)pl->n1, (int)pl->n2, (int)pl->p1, (int)pl->p2);
    if (nc <= 0) {
      pl->tc_split = 0;
    } else if ((st = dalloc(pl, &pl->tc_cst, (size_t)nc)) != GLAM_OK) {
      return bail(st);
    }
  }

  if (pl->um_form) {
    const int64_t nb = fused_umma_const_bytes((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2,
                                              (int)pl->p3, pl->um_form);
    unsigned char* c = nullptr;
    if ((st = dalloc(pl, &c, (size_t)nb)) != GLAM_OK) return bail(st);
    pl->um_cst = c;
    if (pl->um_form == 16 && (st = dalloc(pl, &pl->Vb, (size_t)n)) != GLAM_OK) return bail(st);
  }
  if ((st = dalloc(pl, &pl->ctl, 1)) != GLAM_OK) return bail(st);
  if ((st = dalloc(pl, &pl->sc, 1)) != GLAM_OK) return bail(st);
  if ((st = dalloc(pl, &pl->red.partial, (size_t)kMaxRedBlocks * kRedSlots)) != GLAM_OK) return bail(st);
  if ((st = dalloc(pl, &pl->red.counter, 1)) != GLAM_OK) return bail(st);
  if (cudaMemset(pl->red.counter, 0, sizeof(unsigned int)) != cudaSuccess ||
      cudaMemset(pl->ctl, 0, sizeof(InnerCtl)) != cudaSuccess ||
      cudaMemset(pl->sc, 0, sizeof(DevScalars)) != cudaSuccess) {
    pl->err = "cudaMemset failed";
    return bail(GLAM_ECUDA);
  }
  if (cudaMallocHost(&pl->h_ctl, sizeof(InnerCtl)) != cudaSuccess ||
      cudaMallocHost(&pl->h_sc, sizeof(DevScalars)) != cudaSuccess ||
      cudaMallocHost(&pl->h_gram, sizeof(double) * 3 * 4096) != cudaSuccess) {
    pl->err = "cudaMallocHost failed";
    return bail(GLAM_ENOMEM);
  }
  if (cudaStreamCreateWithFlags(&pl->work, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->ev_in, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&pl->ev_out, cudaEventDisableTiming) != cudaSuccess) {
    pl->err = "stream/event creation failed";
    return bail(GLAM_ECUDA);
  }
  if (cudaDeviceSynchronize() != cudaSuccess) { pl->err = "cudaDeviceSynchronize failed"; return bail(GLAM_ECUDA); }
  *out = pl;
  return GLAM_OK;
}

int glam_plan_destroy(glam_plan* pl) {
  if (pl == nullptr) return GLAM_OK;
  for (int r = 0; r < kMaxComp; ++r)
    if (pl->sub[r] != nullptr) glam_plan_destroy(pl->sub[r]);
  if (pl->stream) cudaStreamSynchronize(pl->stream);
  if (pl->work) cudaStreamSynchronize(pl->work);
  for (void* p : pl->allocs) cudaFree(p);
  if (pl->h_ctl) cudaFreeHost(pl->h_ctl);
  if (pl->h_sc) cudaFreeHost(pl->h_sc);
  if (pl->h_gram) cudaFreeHost(pl->h_gram);
  if (pl->ev_in) cudaEventDestroy(pl->ev_in);
  if (pl->ev_out) cudaEventDestroy(pl->ev_out);
  if (pl->work) cudaStreamDestroy(pl->work);
  delete pl;
  return GLAM_OK;
}

int glam_plan_set_stream(glam_plan* pl, void* stream) {
  CKS(check_plan(pl));
  pl->stream = static_cast<cudaStream_t>(stream);
  for (int r = 0; r < kMaxComp; ++r)
    if (pl->sub[r] != nullptr) pl->sub[r]->stream = pl->stream;
  return GLAM_OK;
}

int glam_plan_create_components(int d, const int64_t n[3], int c, const int64_t* p, int family, int precision,
                                void* stream, glam_plan** out) {
  if (out == nullptr || n == nullptr || p == nullptr)
    return fail(nullptr, GLAM_EINVAL, "glam_plan_create_components: NULL argument");
  *out = nullptr;
  if (c < 1 || c > kMaxComp) return fail(nullptr, GLAM_EINVAL, "c must be in [1, 8]");
  glam_dims dr{};
  dr.d = d;
  for (int j = 0; j < 3; ++j) dr.n[j] = n[j];
  if (c == 1) {
    for (int j = 0; j < 3; ++j) dr.p[j] = p[j];
    return glam_plan_create(&dr, family, precision, stream, out);
  }
  int64_t ptot = 0;
  const int64_t kLim = (int64_t)1 << 40;
  for (int r = 0; r < c; ++r) {
    if (p[3 * r] < 1 || p[3 * r + 1] < 1 || p[3 * r + 2] < 1)
      return fail(nullptr, GLAM_EINVAL, "every p_rj must be >= 1");
    int64_t pr = 1;
    for (int j = 0; j < 3; ++j) {
      if (p[3 * r + j] > kLim / pr) return fail(nullptr, GLAM_EINVAL, "component coefficients too many");
      pr *= p[3 * r + j];
    }
    if (pr > kLim - ptot) return fail(nullptr, GLAM_EINVAL, "component coefficients too many");
    ptot += pr;
  }
  // this plan: the grid's n-space arrays and the concatenated p-space state (its own transforms
  // are never used: the components' plans do them)
  glam_dims dp = dr;
  dp.p[0] = ptot;
  dp.p[1] = 1;
  dp.p[2] = 1;
  glam_plan* pl = nullptr;
  CKS(glam_plan_create(&dp, family, precision, stream, &pl));
  pl->nc = c;
  pl->ksplit = 1;
  pl->fused[0] = pl->fused[1] = false;
  pl->um_form = 0;
  pl->tc_split = 0;
  pl->Vb = nullptr;  // the generic inner product reads the weights in the working precision
  pl->poff[0] = 0;
  for (int r = 0; r < c; ++r) {
    for (int j = 0; j < 3; ++j) dr.p[j] = p[3 * r + j];
    const int st = glam_plan_create(&dr, family, precision, stream, &pl->sub[r]);
    if (st != GLAM_OK) {
      const std::string m = g_thread_err;
      glam_plan_destroy(pl);
      return fail(nullptr, st, "component " + std::to_string(r) + ": " + m);
    }
    pl->poff[r + 1] = pl->poff[r] + pl->sub[r]->p;
  }
  *out = pl;
  return GLAM_OK;
}

const char* glam_last_error(const glam_plan* pl) {
  return pl ? pl->err.c_str() : g_thread_err.c_str();
}

int glam_predict(glam_plan* pl, const void* const X[3], const void* Theta, void* eta) {
  CKS(check_plan(pl));
  CKS(validate_X(pl, X));
  if (Theta == nullptr || eta == nullptr) return fail(pl, GLAM_EINVAL, "glam_predict: NULL array");
  if (pl->precision == GLAM_FP64) {
    Ops<double> op(pl, pl->stream, X);
    return op.H(static_cast<const double*>(Theta), static_cast<double*>(eta));
  }
  Ops<float> op(pl, pl->stream, X);
  return op.H(static_cast<const float*>(Theta), static_cast<float*>(eta));
}

namespace {
template <typename T>
int gradient_impl(glam_plan* pl, const void* const X[3], const T* Theta, const T* Y, const T* W,
                  T* grad, double* loss) {
  Ops<T> op(pl, pl->stream, X);
  CKS(op.H(Theta, op.w.eta));
  CK(launch_family<T, T>(pl->family, pl->n, op.w.eta, Y, W, nullptr, nullptr, op.w.U, 1.0, pl->sc,
                         pl->red, pl->stream));
  CKS(op.G(op.w.U, op.w.grad));
  CK(launch_scale<T>(pl->p, op.w.grad, grad, -1.0 / (double)pl->n, pl->stream));
  if (loss != nullptr)
    CK(cudaMemcpyAsync(loss, &pl->sc->loss, sizeof(double), cudaMemcpyDeviceToDevice, pl->stream));
  return GLAM_OK;
}
}  // namespace

int glam_gradient(glam_plan* pl, const void* const X[3], const void* Theta, const void* Y,
                  const void* W, void* grad, double* loss_or_null) {
  CKS(check_plan(pl));
  CKS(validate_X(pl, X));
  if (!Theta || !Y || !W || !grad) return fail(pl, GLAM_EINVAL, "glam_gradient: NULL array");
  if (pl->precision == GLAM_FP64)
    return gradient_impl<double>(pl, X, (const double*)Theta, (const double*)Y, (const double*)W,
                                 (double*)grad, loss_or_null);
  return gradient_impl<float>(pl, X, (const float*)Theta, (const float*)Y, (const float*)W,
                              (float*)grad, loss_or_null);
}

namespace {
template <typename T>
int loss_impl(glam_plan* pl, const void* const X[3], const T* Theta, const T* Y, const T* W,
              double* out) {
  Ops<T> op(pl, pl->stream, X);
  CKS(op.H(Theta, op.w.eta));
  CK(launch_loss_only<T>(pl->family, pl->n, op.w.eta, Y, W, out, pl->red, pl->stream));
  return GLAM_OK;
}
}  // namespace

int glam_loss(glam_plan* pl, const void* const X[3], const void* Theta, const void* Y,
              const void* W, double* out) {
  CKS(check_plan(pl));
  CKS(validate_X(pl, X));
  if (!Theta || !Y || !W || !out) return fail(pl, GLAM_EINVAL, "glam_loss: NULL array");
  if (pl->precision == GLAM_FP64)
    return loss_impl<double>(pl, X, (const double*)Theta, (const double*)Y, (const double*)W, out);
  return loss_impl<float>(pl, X, (const float*)Theta, (const float*)Y, (const float*)W, out);
}

namespace {
template <typename T>
int nll_impl(glam_plan* pl, const void* const X[3], const T* Theta, const T* Y, const T* W,
             double lambda, const T* pen_w, const double* gout, double* F, T* gTheta, T* gY) {
  Ops<T> op(pl, pl->stream, X);
  const bool vjp_theta = gTheta != nullptr;
  CKS(op.H(Theta, op.w.eta));
  CK(launch_nll_cells<T>(pl->family, pl->n, op.w.eta, Y, W, gout, vjp_theta ? op.w.U : nullptr, gY,
                         pl->sc, pl->red, pl->stream));
  if (vjp_theta) CKS(op.G(op.w.U, op.w.grad));
  CK(launch_nll_coef<T>(pl->p, Theta, pen_w, lambda, gout, op.w.grad, gTheta, F, pl->sc, pl->red,
                        pl->stream));
  return GLAM_OK;
}
}  // namespace

int glam_penalized_nll(glam_plan* pl, const void* const X[3], const void* Theta, const void* Y,
                       const void* W, double lambda, const void* pen_w, const double* gout,
                       double* F, void* grad_Theta, void* grad_Y) {
  CKS(check_plan(pl));
  CKS(single_component(pl, "glam_penalized_nll"));
  CKS(validate_X(pl, X));
  if (!Theta || !Y || !W || !pen_w) return fail(pl, GLAM_EINVAL, "glam_penalized_nll: NULL array");
  if (!F && !grad_Theta && !grad_Y)
    return fail(pl, GLAM_EINVAL, "glam_penalized_nll: no output requested");
  if (!(lambda >= 0.0) || !std::isfinite(lambda))
    return fail(pl, GLAM_EINVAL, "glam_penalized_nll: lambda must be finite and >= 0");
  if (pl->precision == GLAM_FP64)
    return nll_impl<double>(pl, X, (const double*)Theta, (const double*)Y, (const double*)W, lambda,
                            (const double*)pen_w, gout, F, (double*)grad_Theta, (double*)grad_Y);
  return nll_impl<float>(pl, X, (const float*)Theta, (const float*)Y, (const float*)W, lambda,
                         (const float*)pen_w, gout, F, (float*)grad_Theta, (float*)grad_Y);
}

namespace {


template <typename T>
int quad_impl(glam_plan* pl, const void* const X[3], const T* Theta, const T* Y, const T* W,
              const glam_quad* q, double rho_prod) {
  Ops<T> op(pl, pl->stream, X);
  CKS(op.H(Theta, op.w.eta));
  CK(launch_family<T, T>(pl->family, pl->n, op.w.eta, Y, W, (T*)q->V, (T*)q->VZ, nullptr, rho_prod,
                         pl->sc, pl->red, pl->stream));
  CKS(op.G((const T*)q->VZ, (T*)q->b));
  CK(cudaMemcpyAsync(q->Lhat, &pl->sc->Lhat, sizeof(double), cudaMemcpyDeviceToDevice, pl->stream));
  return GLAM_OK;
}

// prod_j varrho(X_j^T X_j) (Prop. 1): FP64 Gram matrices on the device, eigenvalues on the host.
template <typename T>
int rho_product_from(glam_plan* pl, const T* const X[3], cudaStream_t s, double& out) {
  double prod = 1.0;
  const int d = pl->dims.d;
  for (int j = 0; j < d; ++j) {
    const int nj = (int)pl->dims.n[j], pj = (int)pl->dims.p[j];
    if ((int64_t)pj * pj > 4096) return fail(pl, GLAM_EINVAL, "p_j > 64 is not supported by the step-size setup");
    const double* X64;
    if (sizeof(T) == 8) {
      X64 = reinterpret_cast<const double*>(X[j]);
    } else {
      CK(launch_convert<float, double>((int64_t)nj * pj, reinterpret_cast<const float*>(X[j]),
                                       pl->wd.Xc[j], s));
      X64 = pl->wd.Xc[j];
    }
    CK(launch_gram(nj, pj, X64, pl->d_gram, s));
    CK(cudaMemcpyAsync(pl->h_gram, pl->d_gram, sizeof(double) * pj * pj, cudaMemcpyDeviceToHost, s));
    CK(cudaStreamSynchronize(s));
    std::vector<double> A(pl->h_gram, pl->h_gram + (size_t)pj * pj);
    prod *= jacobi_spectral_radius(A, pj);
  }
  out = prod;
  return GLAM_OK;
}

}  // namespace

int glam_quad_build(glam_plan* pl, const void* const X[3], const void* Theta_k, const void* Y,
                    const void* W, const glam_quad* q) {
  CKS(check_plan(pl));
  CKS(single_component(pl, "glam_quad_build"));
  CKS(validate_X(pl, X));
  if (!Theta_k || !Y || !W || !q || !q->V || !q->VZ || !q->b || !q->Lhat)
    return fail(pl, GLAM_EINVAL, "glam_quad_build: NULL argument");
  double rp = 1.0;
  if (pl->precision == GLAM_FP64) {
    const double* Xd[3] = {(const double*)X[0], (const double*)X[1], (const double*)X[2]};
    if (Xd[2] == nullptr) Xd[2] = pl->wd.one;
    CKS(rho_product_from<double>(pl, Xd, pl->stream, rp));
    return quad_impl<double>(pl, X, (const double*)Theta_k, (const double*)Y, (const double*)W, q, rp);
  }
  const float* Xf[3] = {(const float*)X[0], (const float*)X[1], (const float*)X[2]};
  if (Xf[2] == nullptr) Xf[2] = pl->wf.one;
  CKS(rho_product_from<float>(pl, Xf, pl->stream, rp));
  return quad_impl<float>(pl, X, (const float*)Theta_k, (const float*)Y, (const float*)W, q, rp);
}

namespace {
template <typename T>
int prox_impl(glam_plan* pl, const void* const X[3], const glam_quad* q, const T* x, const T* xp,
              double omega, double delta, double lambda, const T* pen_w, T* x_next) {
  Ops<T> op(pl, pl->stream, X);
  CKS(op.template XtWX<T>(x, xp, nullptr, (const T*)q->V, nullptr, omega, nullptr));
  CK(launch_prox<T, T>(pl->p, pl->ksplit, op.w.Qpart, (const T*)q->b, -1.0 / (double)pl->n, x, xp,
                       pen_w, x_next, 1.0 / (double)pl->n, nullptr, omega, delta, lambda, q->Lhat,
                       pl->stream));
  return GLAM_OK;
}
}  // namespace

int glam_prox_step(glam_plan* pl, const void* const X[3], const glam_quad* q, const void* x,
                   const void* x_prev, double omega, double delta, double lambda, const void* pen_w,
                   void* x_next) {
  CKS(check_plan(pl));
  CKS(single_component(pl, "glam_prox_step"));
  CKS(validate_X(pl, X));
  if (!q || !q->V || !q->b || !q->Lhat || !x || !x_prev || !pen_w || !x_next)
    return fail(pl, GLAM_EINVAL, "glam_prox_step: NULL argument");
  if (x_next == x || x_next == x_prev) return fail(pl, GLAM_EINVAL, "glam_prox_step: x_next aliases an input");
  if (pl->precision == GLAM_FP64)
    return prox_impl<double>(pl, X, q, (const double*)x, (const double*)x_prev, omega, delta,
                             lambda, (const double*)pen_w, (double*)x_next);
  return prox_impl<float>(pl, X, q, (const float*)x, (const float*)x_prev, omega, delta, lambda,
                          (const float*)pen_w, (float*)x_next);
}


// ======================================================================== fit path
//
// Mixed-precision refinement form of Alg. 1.  Per outer iteration k:
//   FP64 pass:  eta = H(theta_k), u, w (App. B), g_k = grad f(theta_k) = -(1/n) G(u), the KKT
//               residual (the convergence test of step 6) and F(theta_k), all in FP64;
//               V = w is written in the plan's working precision;
//   inner loop: FISTA (Sec. 3.2) on the quadratic model h with
//               grad h(y) = g_k + (1/n) X^T W X (y - theta_k)        (= Eq. twentyfive)
//               p-space vectors in FP64, mode products in the working precision acting on the
//               correction y - theta_k only;
//   line search: Armijo rule (Sec. 5) on d = theta~ - theta_k with eta(theta_k + alpha d) =
//               eta + alpha H(d) (linearity of H), all trial steps evaluated in one pass.
// The mode products only ever see corrections, so their rounding error shrinks with the
// correction and the iteration converges to FP64 accuracy in theta and in the KKT residual.
namespace {

// Step 3 of Alg. 1 and the package's nu (Sec. 6.4): delta = 1 / L_hat for nu = 1, 1 / (nu L_hat)
// for nu in (0, 1), 1 for nu = 0; delta_cap > 0 (a restart after divergence) caps it, but not
// below 1 / L_hat.  Steps larger than 1 / L_hat arm the divergence test of the prox kernels.
__global__ void ctl_init_kernel(InnerCtl* ctl, const DevScalars* sc, double lambda, double stop_rel,
                                int max_iter, double l1, double l2, double nu, double delta_cap) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double safe = 1.0 / sc->Lhat;
  double delta = nu >= 1.0 ? safe : (nu > 0.0 ? 1.0 / (nu * sc->Lhat) : 1.0);
  if (delta_cap > 0.0 && delta > delta_cap) delta = delta_cap > safe ? delta_cap : safe;
  ctl->div_factor = delta > safe ? kInnerDivFactor : 0.0;
  ctl->crit_first = 0.0;
  ctl->l = 1;
  ctl->done = 0;
  ctl->max_iter = max_iter;
  ctl->iters_run = 0;
  ctl->counter = 0u;
  ctl->stop_reason = 0;
  ctl->crit_bits = 0ull;
  ctl->delta = delta;
  ctl->lambda = lambda;
  ctl->stop_abs = stop_rel * sc->lmax * delta;
  ctl->crit = 0.0;
  ctl->pen_l1 = l1;
  ctl->pen_l2 = l2;
}

__global__ void objective_kernel(DevScalars* sc, double lambda) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc->F = sc->loss + lambda * sc->pen;
}

__global__ void set_lhat_kernel(DevScalars* sc, double L) {
  if (threadIdx.x == 0 && blockIdx.x == 0) sc->Lhat = L;
}

template <typename T>
struct Fit {
  glam_plan* pl = nullptr;
  glam_opts o{};
  cudaStream_t s = nullptr;
  double rho_prod = 1.0;
  double lmax = 0.0;
  const void* Xw[3 * kMaxComp] = {};   // designs in the working precision (3 per component)
  const void* X64[3 * kMaxComp] = {};  // designs in FP64
  const double* Y64 = nullptr;
  const double* W64 = nullptr;
  cudaGraphExec_t graph = nullptr;
  int64_t graph_kernels = 0;
  bool kron = false;  // inner loop on the tensor-product form H(<M_j>, .) (Sec. 6.2)
  bool kron_geo = false;  // ... with the M_j of the geometric-mean approximation of V, per pass
  int restarts = 0;       // inner solves restarted with a halved step (nu < 1), this lambda
  double l1 = 1.0, l2 = 0.0;  // penalty J = sum_m w_m (l1 |theta_m| + l2 theta_m^2) (Sec. 6.3)
  // eta, U, V, the loss and g_k in the plan describe the current theta: set by a full FP64 pass,
  // cleared whenever theta moves (a new lambda starts where the last one stopped, so its first
  // pass needs only the lambda-dependent KKT residual and objective)
  bool grad_fresh = false;
  uint64_t wait_ns = kDefaultWaitNs;  // limit of every bounded device wait of the inner loop
  ~Fit() {
    if (graph) cudaGraphExecDestroy(graph);
  }
};

// The FP64 pass at theta (see above).  Fills r (scaled KKT residual), F, nnz.
template <typename T>
int kron_refresh_geo(Fit<T>& f);

template <typename T>
int fp64_pass(Fit<T>& f, double lambda, double& r, double& F, int& nnz, bool& nonfinite) {
  glam_plan* pl = f.pl;
  Ops<double> op(pl, f.s, f.X64);
  Work<T>& w = work_of<T>(pl);
  if (!f.grad_fresh) {
    CKS(op.H(pl->th, pl->wd.eta));
    if (pl->Vb != nullptr)  // BF16 plans: the inner product streams the weights in BF16
      CK(launch_family<double, __nv_bfloat16>(pl->family, pl->n, pl->wd.eta, f.Y64, f.W64, pl->Vb, nullptr,
                                              pl->wd.U, f.rho_prod, pl->sc, pl->red, f.s));
    else
      CK(launch_family<double, T>(pl->family, pl->n, pl->wd.eta, f.Y64, f.W64, w.V, nullptr, pl->wd.U,
                                  f.rho_prod, pl->sc, pl->red, f.s));
    CKS(op.G(pl->wd.U, pl->gk));
    CK(launch_scale<double>(pl->p, pl->gk, pl->gk, -1.0 / (double)pl->n, f.s));
    if (f.kron_geo) CKS(kron_refresh_geo<T>(f));
  }
  CK(launch_kkt<double>(pl->p, pl->gk, pl->th, pl->pen, lambda, pl->sc, pl->red, f.s, f.l1, f.l2));
  objective_kernel<<<1, 32, 0, f.s>>>(pl->sc, lambda);
  CK(cudaGetLastError());
  count_launches(1);
  CK(cudaMemcpyAsync(pl->h_sc, pl->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, f.s));
  CK(cudaStreamSynchronize(f.s));
  r = pl->h_sc->kkt_max / f.lmax;
  F = pl->h_sc->F;
  nnz = pl->h_sc->nnz;
  nonfinite = pl->h_sc->nonfinite != 0 || !std::isfinite(F) || !std::isfinite(r);
  f.grad_fresh = true;
  return GLAM_OK;
}

template <typename T>
int capture_chunk(Fit<T>& f) {
  glam_plan* pl = f.pl;
  Ops<T> op(pl, f.s, f.Xw);
  const int C = f.o.check_every;
  cudaGraph_t g = nullptr;
  CK(cudaStreamBeginCapture(f.s, cudaStreamCaptureModeThreadLocal));
  set_capturing(true);
  int st = GLAM_OK;
  for (int it = 0; it < C && st == GLAM_OK; ++it) {
    double* x = (it % 2 == 0) ? pl->x0 : pl->x1;
    double* xp = (it % 2 == 0) ? pl->x1 : pl->x0;
    if (f.kron) {
      // X^T W X d = H(<M_j>, d) on p-sized arrays (Sec. 6.2, Eq. kronweight), then the prox step
      Work<T>& w = op.w;
      const int* skip = &pl->ctl->done;
      cudaError_t e = cudaSuccess;
      if (kron_product_supported<T>((int)pl->p1, (int)pl->p2, (int)pl->p3)) {
        e = launch_kron_product<T>((int)pl->p1, (int)pl->p2, (int)pl->p3, w.Mk[0], w.Mk[1], w.Mk[2],
                                   w.dn, w.kQ, skip, f.s);
      } else {
        e = launch_gemm<T, T>(k_mode3_fwd(pl), w.Mk[2], w.dn, w.kTa, f.s, nullptr, nullptr, nullptr,
                              0.0, skip);
        if (e == cudaSuccess)
          e = launch_gemm<T, T>(k_mode1_fwd(pl), w.kTa, w.Mk[0], w.kTb, f.s, nullptr, nullptr, nullptr,
                                0.0, skip);
        if (e == cudaSuccess)
          e = launch_gemm<T, T>(k_mode2_fwd(pl), w.Mk[1], w.kTb, w.kQ, f.s, nullptr, nullptr, nullptr,
                                0.0, skip);
      }
      if (e == cudaSuccess)
        e = launch_prox<T, double>(pl->p, 1, w.kQ, pl->gk, 1.0, x, xp, pl->pen, xp, 1.0 / (double)pl->n,
                                   pl->ctl, 0.0, 0.0, 0.0, nullptr, f.s, w.dn, pl->th);
      if (e != cudaSuccess) st = fail(pl, GLAM_ECUDA, std::string("inner iteration launch: ") + cudaGetErrorString(e));
      continue;
    }
    bool use_tc = false, use_ap = false, use_um = false;
    const void* Vin = pl->Vb != nullptr ? (const void*)pl->Vb : (const void*)op.w.V;
    if constexpr (sizeof(T) == 4) {
      use_um = pl->um_form && fused_tc_pointers_ok((const float*)pl->um_cst, op.w.dn, (const float*)Vin);
      use_tc = !use_um && pl->tc_split && fused_tc_pointers_ok(pl->tc_cst, op.w.dn, op.w.V);
      use_ap = pl->nc == 1 && adjprox_supported((int)pl->n3, (int)pl->p3, (int)(pl->p2 * pl->p1),
                                                (const float*)op.X[2], (const float*)op.w.Sb) != 0;
    }
    const bool fused = pl->fused[sizeof(T) == 8 ? 1 : 0] || use_tc || use_um;
    if (fused) {
      // the fused kernel forms T_a = X_3 d from the correction itself, then the adjoint
      cudaError_t e = cudaSuccess;
      // the tensor-core kernel and the adjoint + prox kernel alternate: each launch may overlap the
      // end of the one before it (programmatic dependent launch), which writes nothing the overlapped
      // part of the next reads (V, X_1, X_3 and the constant block stay fixed inside this loop)
      const bool pdl = use_um && use_ap;
      if constexpr (sizeof(T) == 4) {
        if (use_um)
          e = launch_fused_umma((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2, (int)pl->p3,
                                pl->um_form, pl->Vb != nullptr, pl->um_cst, op.w.dn, op.X[0], op.X[2], Vin,
                                op.w.Sb, f.s, &pl->ctl->done, &pl->sc->timeout, f.wait_ns, pdl && it > 0);
        else if (use_tc)
          e = launch_fused_slab_tc((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2,
                                   (int)pl->p3, pl->tc_cst, op.w.dn, op.w.V, op.w.Sb, f.s,
                                   &pl->ctl->done, &pl->sc->timeout, op.X[2], pl->tc_split);
      }
      if (!use_tc && !use_um)
        e = launch_fused_slab<T>((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2,
                                 op.X[0], op.X[1], op.w.dn, op.w.V, op.w.Sb, f.s, &pl->ctl->done,
                                 &pl->sc->timeout, op.X[2], (int)pl->p3);
      if constexpr (sizeof(T) == 4) {
        if (e == cudaSuccess && use_ap)  // mode-3 adjoint and prox step in one kernel
          e = launch_adjprox((int)pl->n3, (int)pl->p3, (int)(pl->p2 * pl->p1), op.X[2], op.w.Sb, pl->gk,
                             x, xp, pl->pen, xp, op.w.dn, pl->th, 1.0 / (double)pl->n, pl->ctl,
                             &pl->sc->timeout, f.s, pdl, pl->x3rows);
      }
      if (e == cudaSuccess && !use_ap)
        e = launch_gemm<T, T>(d_mode3_adj(pl, pl->ksplit), op.X[2], op.w.Sb, op.w.Qpart, f.s, nullptr,
                              nullptr, nullptr, 0.0, &pl->ctl->done);
      if (e != cudaSuccess) st = fail(pl, GLAM_ECUDA, std::string("inner iteration launch: ") + cudaGetErrorString(e));
    } else {
      st = op.template XtWX<T>(op.w.dn, nullptr, nullptr, op.w.V, nullptr, 0.0, &pl->ctl->done);
    }
    if (st == GLAM_OK && !(fused && use_ap)) {
      cudaError_t e = launch_prox<T, double>(pl->p, pl->ksplit, op.w.Qpart, pl->gk, 1.0, x, xp,
                                             pl->pen, xp, 1.0 / (double)pl->n, pl->ctl, 0.0, 0.0,
                                             0.0, nullptr, f.s, op.w.dn, pl->th);
      if (e != cudaSuccess) st = fail(pl, GLAM_ECUDA, std::string("prox launch: ") + cudaGetErrorString(e));
    }
  }
  cudaError_t e = cudaStreamEndCapture(f.s, &g);
  set_capturing(false);
  if (st != GLAM_OK) {
    if (g) cudaGraphDestroy(g);
    return st;
  }
  if (e != cudaSuccess) return fail(pl, GLAM_ECUDA, std::string("cudaStreamEndCapture: ") + cudaGetErrorString(e));
  size_t nodes = 0;
  if (g) cudaGraphGetNodes(g, nullptr, &nodes);
  f.graph_kernels = (int64_t)nodes;
  e = cudaGraphInstantiate(&f.graph, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(pl, GLAM_ECUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
  return GLAM_OK;
}

// Inner PG loop of Sec. 3.2 from x(0) = x(1) = theta_k; *xout receives the last iterate.
template <typename T>
int run_inner_once(Fit<T>& f, double lambda, double stop_rel, int max_iter, double** xout, int& iters,
                   int& reason, double delta_cap) {
  glam_plan* pl = f.pl;
  CK(cudaMemcpyAsync(pl->x0, pl->th, sizeof(double) * pl->p, cudaMemcpyDeviceToDevice, f.s));
  CK(cudaMemcpyAsync(pl->x1, pl->th, sizeof(double) * pl->p, cudaMemcpyDeviceToDevice, f.s));
  CK(cudaMemsetAsync(work_of<T>(pl).dn, 0, sizeof(T) * pl->p, f.s));  // y(1) - theta_k = 0
  CK(cudaMemsetAsync(&pl->sc->timeout, 0, sizeof(int), f.s));
  ctl_init_kernel<<<1, 32, 0, f.s>>>(pl->ctl, pl->sc, lambda, stop_rel, max_iter, f.l1, f.l2, f.o.nu, delta_cap);
  CK(cudaGetLastError());
  count_launches(1);
  if (f.graph == nullptr) CKS(capture_chunk<T>(f));
  const int C = f.o.check_every;
  const int max_chunks = max_iter / C + 2;
  bool done = false;
  for (int c = 0; c < max_chunks && !done; ++c) {
    CK(cudaGraphLaunch(f.graph, f.s));
    count_launches(f.graph_kernels);
    CK(cudaMemcpyAsync(pl->h_ctl, pl->ctl, sizeof(InnerCtl), cudaMemcpyDeviceToHost, f.s));
    CK(cudaMemcpyAsync(&pl->h_sc->timeout, &pl->sc->timeout, sizeof(int), cudaMemcpyDeviceToHost, f.s));
    CK(cudaStreamSynchronize(f.s));
    done = pl->h_ctl->done != 0;
    if (pl->h_sc->timeout) return fail(pl, GLAM_ETIMEOUT, "a bounded device-side wait ran out");
  }
  if (!done) return fail(pl, GLAM_ETIMEOUT, "inner loop did not stop within its iteration cap");
  CK(cudaMemcpyAsync(pl->h_sc, pl->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, f.s));
  CK(cudaStreamSynchronize(f.s));
  if (pl->h_sc->timeout) return fail(pl, GLAM_ETIMEOUT, "a bounded device-side wait ran out");
  iters = pl->h_ctl->iters_run;
  reason = pl->h_ctl->stop_reason;
  *xout = (iters % 2 == 1) ? pl->x1 : pl->x0;
  return GLAM_OK;
}

// With nu < 1 a solve that diverges (stop reason 3) starts again from theta_k with the step
// halved, until it reaches 1 / L_hat (where the test is off); the iterations of the abandoned
// solves count in iters.
template <typename T>
int run_inner(Fit<T>& f, double lambda, double stop_rel, int max_iter, double** xout, int& iters,
              int& reason) {
  double cap = 0.0;
  int total = 0;
  for (;;) {
    CKS(run_inner_once<T>(f, lambda, stop_rel, max_iter, xout, iters, reason, cap));
    total += iters;
    if (reason != 3) break;
    f.restarts += 1;
    cap = 0.5 * f.pl->h_ctl->delta;
  }
  iters = total;
  return GLAM_OK;
}

struct LamOut {
  int outer = 0, inner = 0, passes = 0, backtracks = 0, nnz = 0;
  double kkt = 1e300, F = 0.0;
  bool converged = false, nonfinite = false;
};

template <typename T>
int solve_lambda(Fit<T>& f, double lambda, LamOut& lo) {
  glam_plan* pl = f.pl;
  Ops<T> op(pl, f.s, f.Xw);
  Work<T>& w = op.w;
  for (int k = 0;; ++k) {
    double r = 0.0, F = 0.0;
    int nnz = 0;
    bool nonfinite = false;
    const bool full = !f.grad_fresh;
    CKS(fp64_pass<T>(f, lambda, r, F, nnz, nonfinite));
    if (full) lo.passes += 1;
    lo.kkt = r;
    lo.F = F;
    lo.nnz = nnz;
    if (nonfinite) {
      lo.nonfinite = true;
      return GLAM_OK;
    }
    if (r <= f.o.tol) {
      lo.converged = true;
      return GLAM_OK;
    }
    if (k >= f.o.max_outer) return GLAM_OK;
    // inner PG loop, solved to a fraction of the current residual (floor: inner_floor * tol)
    double stop_rel = f.o.inner_forcing * r;
    if (stop_rel < f.o.inner_floor * f.o.tol) stop_rel = f.o.inner_floor * f.o.tol;
    double* xt = nullptr;
    int iters = 0, reason = 0;
    CKS(run_inner<T>(f, lambda, stop_rel, f.o.max_inner, &xt, iters, reason));
    lo.inner += iters;
    lo.outer += 1;
    // Armijo rule along d = theta~ - theta_k
    CKS(op.template H_diff<double>(xt, pl->th, w.eta_bar));
    int accepted = -1;
    for (int j0 = 0; j0 < f.o.max_linesearch && accepted < 0; j0 += kTrials) {
      CK(launch_armijo_stream<double, T>(pl->family, pl->n, pl->wd.eta, w.eta_bar, f.Y64, f.W64,
                                         f.o.armijo_alpha0, f.o.armijo_b, j0, pl->sc, pl->red, f.s));
      CK(launch_armijo_penalty<double>(pl->p, pl->th, xt, pl->pen, f.o.armijo_alpha0, f.o.armijo_b,
                                       j0, pl->sc, pl->red, f.s, f.l1, f.l2));
      CK(launch_armijo_select(lambda, f.o.armijo_v, f.o.armijo_alpha0, f.o.armijo_b, j0, pl->sc, f.s));
      CK(cudaMemcpyAsync(pl->h_sc, pl->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, f.s));
      CK(cudaStreamSynchronize(f.s));
      accepted = pl->h_sc->accepted;
    }
    if (accepted < 0) return GLAM_OK;  // no descent left: report the current residual
    lo.backtracks += accepted;
    CK(launch_armijo_update<double>(pl->p, pl->th, xt, pl->sc, f.s));
    f.grad_fresh = false;
  }
}

// The range of the nonzero entries of each row j3 of X_3^T, read by the adjoint + prox kernel.
int x3_rows_setup(glam_plan* pl, const float* X3T, cudaStream_t s) {
  if (pl->x3rows == nullptr) CKS(dalloc(pl, &pl->x3rows, 2 * pl->p3));
  CK(launch_x3_rows((int)pl->n3, (int)pl->p3, X3T, pl->x3rows, s));
  return GLAM_OK;
}

// The banded form of the FP64 marginal designs of this fit (glam_opts.exploit_bands): every X_j
// must have at most kBand consecutive nonzeros per row with nondecreasing first columns.
template <typename T>
int band_setup(Fit<T>& f) {
  glam_plan* pl = f.pl;
  if (pl->nc > 1) return fail(pl, GLAM_EINVAL, "exploit_bands: takes one component (c = 1)");
  const int64_t nj[3] = {pl->n1, pl->n2, pl->n3}, pj[3] = {pl->p1, pl->p2, pl->p3};
  for (int j = 0; j < 3; ++j) {
    const double* Xd = (const double*)f.X64[j];
    if (Xd == nullptr) Xd = pl->wd.one;  // d = 2: the 1 x 1 design
    std::vector<double> XT((size_t)(nj[j] * pj[j]));
    CK(cudaMemcpyAsync(XT.data(), Xd, sizeof(double) * XT.size(), cudaMemcpyDeviceToHost, f.s));
    CK(cudaStreamSynchronize(f.s));
    std::vector<int> st, lo, hi;
    std::vector<double> val;
    if (!band_form(XT.data(), (int)nj[j], (int)pj[j], st, val, lo, hi))
      return fail(pl, GLAM_EINVAL,
                  "exploit_bands: X_" + std::to_string(j + 1) + " has a row with more than 4 consecutive nonzeros "
                  "or first columns that decrease");
    BandDesign& b = pl->band[j];
    if (b.start == nullptr) {
      CKS(dalloc(pl, &b.start, nj[j]));
      CKS(dalloc(pl, &b.val, nj[j] * kBand));
      CKS(dalloc(pl, &b.lo, pj[j]));
      CKS(dalloc(pl, &b.hi, pj[j]));
    }
    CK(cudaMemcpyAsync(b.start, st.data(), sizeof(int) * st.size(), cudaMemcpyHostToDevice, f.s));
    CK(cudaMemcpyAsync(b.val, val.data(), sizeof(double) * val.size(), cudaMemcpyHostToDevice, f.s));
    CK(cudaMemcpyAsync(b.lo, lo.data(), sizeof(int) * lo.size(), cudaMemcpyHostToDevice, f.s));
    CK(cudaMemcpyAsync(b.hi, hi.data(), sizeof(int) * hi.size(), cudaMemcpyHostToDevice, f.s));
    CK(cudaStreamSynchronize(f.s));  // the host vectors go out of scope
  }
  pl->band_on = true;
  return GLAM_OK;
}

// Buffers of the tensor-product form: the factors w_j, the FP64 and working-precision M_j, the
// p-sized intermediates of H(<M_j>, d), and the scratch of the geometric-mean factors.
template <typename T>
int kron_alloc(glam_plan* pl) {
  Work<T>& w = work_of<T>(pl);
  const int64_t pj[3] = {pl->p1, pl->p2, pl->p3};
  const int64_t nj[3] = {pl->n1, pl->n2, pl->n3};
  if (pl->kgram == nullptr) {
    for (int j = 0; j < 3; ++j) CKS(dalloc(pl, &pl->kfac[j], nj[j]));
    CKS(dalloc(pl, &pl->kgram, pj[0] * pj[0] + pj[1] * pj[1] + pj[2] * pj[2]));
    CKS(dalloc(pl, &pl->kcheck, 2));
  }
  if (pl->geo == nullptr) CKS(dalloc(pl, &pl->geo, geo_scratch_doubles(nj[0], nj[1], nj[2])));
  if (w.kQ == nullptr) {
    for (int j = 0; j < 3; ++j) CKS(dalloc(pl, &w.Mk[j], pj[j] * pj[j]));
    CKS(dalloc(pl, &w.kTa, pl->p));
    CKS(dalloc(pl, &w.kTb, pl->p));
    CKS(dalloc(pl, &w.kQ, pl->p));
  }
  return GLAM_OK;
}

// M_j = X_j^T diag(kfac_j) X_j in FP64 and in the working precision, and prod_j varrho(M_j)
// (host Jacobi on the FP64 matrices; p_j <= 64).
template <typename T>
int kron_grams(Fit<T>& f, double& rho_kron) {
  glam_plan* pl = f.pl;
  Work<T>& w = work_of<T>(pl);
  const int64_t pj[3] = {pl->p1, pl->p2, pl->p3};
  const int64_t nj[3] = {pl->n1, pl->n2, pl->n3};
  rho_kron = 1.0;
  if (kron_product_supported<T>((int)pl->p1, (int)pl->p2, (int)pl->p3))
    CK(kron_product_prepare<T>((int)pl->p1, (int)pl->p2, (int)pl->p3));
  int64_t off = 0;
  for (int j = 0; j < 3; ++j) {
    const double* Xd = (const double*)f.X64[j];
    if (Xd == nullptr) Xd = pl->wd.one;  // d = 2: the 1 x 1 design
    CK(launch_weighted_gram((int)nj[j], (int)pj[j], Xd, pl->kfac[j], pl->kgram + off, f.s));
    CK(launch_convert<double, T>(pj[j] * pj[j], pl->kgram + off, w.Mk[j], f.s));
    std::vector<double> M((size_t)(pj[j] * pj[j]));
    CK(cudaMemcpyAsync(M.data(), pl->kgram + off, sizeof(double) * M.size(), cudaMemcpyDeviceToHost, f.s));
    CK(cudaStreamSynchronize(f.s));
    rho_kron *= jacobi_spectral_radius(M, (int)pj[j]);
    off += pj[j] * pj[j];
  }
  return GLAM_OK;
}

// Set-up of the tensor-product form (Sec. 6.2): checks that the weight array of the inner problem
// is a tensor product (for the Gaussian family it is W itself), forms M_j = X_j^T diag(w_j) X_j in
// FP64 and in the working precision, and returns prod_j varrho(M_j), which times 1/n is the exact
// Lipschitz constant of the inner problem (Sec. 5, the case of tensor-product weights).
template <typename T>
int kron_setup(Fit<T>& f, const T* W, double& rho_kron, double& wmax) {
  glam_plan* pl = f.pl;
  // the IRLS weight is the observation weight itself for the Gaussian family and for the Gamma
  // family with log link; for the others it varies with eta and is not a tensor product
  if (pl->family != GLAM_GAUSSIAN_IDENTITY && pl->family != GLAM_GAMMA_LOG)
    return fail(pl, GLAM_EINVAL,
                "iwls = GLAM_IWLS_KRON needs tensor-product IRLS weights: the Gaussian or Gamma family");
  Work<T>& w = work_of<T>(pl);
  const int64_t nj[3] = {pl->n1, pl->n2, pl->n3};
  CKS(kron_alloc<T>(pl));
  CK(launch_kron_factors<T>(pl->n1, pl->n2, pl->n3, W, pl->kfac[0], pl->kfac[1], pl->kfac[2],
                            pl->kcheck, f.s));
  unsigned long long chk[2] = {0ull, 0ull};
  double w000 = 0.0;
  CK(cudaMemcpyAsync(chk, pl->kcheck, sizeof(chk), cudaMemcpyDeviceToHost, f.s));
  CK(cudaMemcpyAsync(&w000, f.W64, sizeof(double), cudaMemcpyDeviceToHost, f.s));
  CK(cudaStreamSynchronize(f.s));
  double dev_max, w_max;
  std::memcpy(&dev_max, &chk[0], sizeof(double));
  std::memcpy(&w_max, &chk[1], sizeof(double));
  if (!(w000 > 0.0) || !(dev_max <= 1e-6 * w_max))
    return fail(pl, GLAM_EINVAL, "iwls = GLAM_IWLS_KRON needs W = w1 (x) w2 (x) w3 with W(0,0,0) > 0");
  wmax = w_max;
  return kron_grams<T>(f, rho_kron);
}

// The geometric-mean tensor approximation of this outer iteration's weights V (Sec. 6.2, the
// iwls options kron1 / kron2): factors v_j from V, M_j = X_j^T diag(v_j) X_j, and the exact
// Lipschitz constant prod_j varrho(M_j) / n of the approximated problem in place of Prop. 1's
// bound (the family pass has just written V and L_hat).
template <typename T>
int kron_refresh_geo(Fit<T>& f) {
  glam_plan* pl = f.pl;
  Work<T>& w = work_of<T>(pl);
  const int scaled = f.o.iwls == GLAM_IWLS_KRON2 ? 1 : 0;
  if (pl->Vb != nullptr)
    CK(launch_geo_factors<__nv_bfloat16>((int)pl->n1, (int)pl->n2, (int)pl->n3, pl->Vb, scaled, pl->geo,
                                         pl->kfac[0], pl->kfac[1], pl->kfac[2], f.s));
  else
    CK(launch_geo_factors<T>((int)pl->n1, (int)pl->n2, (int)pl->n3, w.V, scaled, pl->geo, pl->kfac[0],
                             pl->kfac[1], pl->kfac[2], f.s));
  double rho_kron = 1.0;
  CKS(kron_grams<T>(f, rho_kron));
  set_lhat_kernel<<<1, 1, 0, f.s>>>(pl->sc, rho_kron / (double)pl->n);
  CK(cudaGetLastError());
  count_launches(1);
  return GLAM_OK;
}

constexpr double kScadA = 3.7;  // the SCAD shape parameter (Fan and Li's choice)

template <typename T>
int fit_impl(glam_plan* pl, const void* const X[3], const T* Y, const T* W, const double* pen,
             int nlambda, double* lambda, const glam_opts& o, const double* Theta0, double* path,
             glam_stats* stats, int* nfit) {
  Fit<T> f;
  f.pl = pl;
  f.o = o;
  f.s = pl->work;
  CK(cudaEventRecord(pl->ev_in, pl->stream));
  CK(cudaStreamWaitEvent(f.s, pl->ev_in, 0));
  const int nx = 3 * pl->nc;
  for (int j = 0; j < nx; ++j) f.Xw[j] = X[j];
  f.wait_ns = (uint64_t)(o.wait_limit_s * 1e9);
  if (sizeof(T) == 4 && pl->um_form)  // the tcgen05 kernel's constant block, once per fit
    CK(launch_fused_umma_const((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2, (int)pl->p3,
                               pl->um_form, (const float*)X[0], (const float*)X[1], pl->um_cst, f.s));
  if (sizeof(T) == 4 && pl->nc == 1)  // the nonzero range of each row of X_3, once per fit
    CKS(x3_rows_setup(pl, X[2] != nullptr ? (const float*)X[2] : pl->wf.one, f.s));
  if (sizeof(T) == 4 && pl->tc_split)  // the tensor-core kernel's constant block, once per fit
    CK(launch_fused_tc_const((int)pl->n1, (int)pl->n2, (int)pl->p1, (int)pl->p2, (const float*)X[0],
                             (const float*)X[1], pl->tc_cst, pl->tc_split, f.s));
  if (sizeof(T) == 8) {
    for (int j = 0; j < nx; ++j) f.X64[j] = X[j];
    f.Y64 = (const double*)Y;
    f.W64 = (const double*)W;
  } else {
    for (int r = 0; r < pl->nc; ++r) {
      glam_plan* q = pl->nc > 1 ? pl->sub[r] : pl;  // the FP64 copies live in each component's plan
      for (int j = 0; j < 3; ++j) {
        if (X[3 * r + j] == nullptr) continue;
        CK(launch_convert<float, double>(q->dims.n[j] * q->dims.p[j], (const float*)X[3 * r + j], q->wd.Xc[j], f.s));
        f.X64[3 * r + j] = q->wd.Xc[j];
      }
    }
    CK(launch_convert<float, double>(pl->n, (const float*)Y, pl->wd.Yc, f.s));
    CK(launch_convert<float, double>(pl->n, (const float*)W, pl->wd.Wc, f.s));
    f.Y64 = pl->wd.Yc;
    f.W64 = pl->wd.Wc;
  }
  CK(cudaMemcpyAsync(pl->pen, pen, sizeof(double) * pl->p, cudaMemcpyDeviceToDevice, f.s));
  const bool scad = o.penalty == GLAM_PENALTY_SCAD;
  if (o.penalty == GLAM_PENALTY_ENET) {
    f.l1 = 1.0;
    f.l2 = o.enet_alpha;
  } else if (o.penalty == GLAM_PENALTY_RIDGE) {
    f.l1 = 0.0;
    f.l2 = 1.0;
  }
  if (scad) {
    if (pl->pen_base == nullptr) CKS(dalloc(pl, &pl->pen_base, pl->p));
    CK(cudaMemcpyAsync(pl->pen_base, pen, sizeof(double) * pl->p, cudaMemcpyDeviceToDevice, f.s));
  }
  // input checks
  CK(cudaMemsetAsync(&pl->sc->nonfinite, 0, sizeof(int), f.s));
  CK(launch_check_finite<double>(pl->n, f.Y64, pl->sc, f.s));
  CK(launch_check_finite<double>(pl->n, f.W64, pl->sc, f.s));
  CK(launch_check_finite<double>(pl->p, pl->pen, pl->sc, f.s));
  if (Theta0) CK(launch_check_finite<double>(pl->p, Theta0, pl->sc, f.s));
  CK(cudaMemcpyAsync(pl->h_sc, pl->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, f.s));
  CK(cudaStreamSynchronize(f.s));
  if (pl->h_sc->nonfinite) return fail(pl, GLAM_ENONFINITE, "non-finite value in Y, W, pen_w or Theta0");
  // Prop. 1: sum over the components of prod_j varrho(X_rj^T X_rj) (Eq. nineteennew)
  f.rho_prod = 0.0;
  for (int r = 0; r < pl->nc; ++r) {
    glam_plan* q = pl->nc > 1 ? pl->sub[r] : pl;
    const double* Xd[3] = {(const double*)f.X64[3 * r], (const double*)f.X64[3 * r + 1],
                           (const double*)f.X64[3 * r + 2]};
    if (Xd[2] == nullptr) Xd[2] = q->wd.one;
    double rr = 1.0;
    CKS(rho_product_from<double>(q, Xd, f.s, rr));
    f.rho_prod += rr;
  }
  if (pl->nc > 1 && o.iwls != GLAM_IWLS_EXACT)
    return fail(pl, GLAM_EINVAL, "iwls: the tensor-product forms take one component (c = 1)");
  struct BandOff {  // the banded form serves this fit only
    glam_plan* p;
    ~BandOff() { p->band_on = false; }
  } band_off{pl};
  if (o.exploit_bands) CKS(band_setup<T>(f));
  if (o.iwls == GLAM_IWLS_KRON1 || o.iwls == GLAM_IWLS_KRON2) {
    // the factors, the M_j and L are formed from V in every full FP64 pass
    CKS(kron_alloc<T>(pl));
    f.kron = true;
    f.kron_geo = true;
  }
  if (o.iwls == GLAM_IWLS_KRON) {
    // the family pass sets L_hat = max(w)/n * rho_prod with w = W here; with rho_prod =
    // prod_j varrho(M_j) / max(W) it is the exact constant prod_j varrho(M_j) / n of
    // tensor-product weights
    double rho_kron = 1.0, wmax = 1.0;
    CKS(kron_setup<T>(f, W, rho_kron, wmax));
    f.kron = true;
    f.rho_prod = rho_kron / wmax;
  }
  // lambda_max (Sec. 6.4): g(0) = -(1/n) G(U(eta = 0)), in FP64
  {
    Ops<double> op(pl, f.s, f.X64);
    CK(cudaMemsetAsync(pl->wd.eta, 0, sizeof(double) * pl->n, f.s));
    CK(launch_family<double, double>(pl->family, pl->n, pl->wd.eta, f.Y64, f.W64, nullptr, nullptr,
                                     pl->wd.U, 1.0, pl->sc, pl->red, f.s));
    CKS(op.G(pl->wd.U, pl->ptmp));
    CK(launch_scale<double>(pl->p, pl->ptmp, pl->ptmp, -1.0 / (double)pl->n, f.s));
    CK(launch_lambda_max<double>(pl->p, pl->ptmp, pl->pen, pl->sc, pl->red, f.s));
    CK(cudaMemcpyAsync(pl->h_sc, pl->sc, sizeof(DevScalars), cudaMemcpyDeviceToHost, f.s));
    CK(cudaStreamSynchronize(f.s));
    f.lmax = pl->h_sc->lmax;
  }
  if (!(f.lmax > 0.0)) return fail(pl, GLAM_EINVAL, "lambda_max is zero: the zero fit is exact");
  CK(cudaMemcpyAsync(&pl->sc->lmax, &f.lmax, sizeof(double), cudaMemcpyHostToDevice, f.s));
  std::vector<double> lams(nlambda);
  if (lambda[0] < 0) {
    for (int k = 0; k < nlambda; ++k)
      lams[k] = nlambda == 1 ? f.lmax : f.lmax * std::pow(o.lambda_min_ratio, (double)k / (nlambda - 1));
    for (int k = 0; k < nlambda; ++k) lambda[k] = lams[k];
  } else {
    for (int k = 0; k < nlambda; ++k) lams[k] = lambda[k];
  }
  if (Theta0)
    CK(cudaMemcpyAsync(pl->th, Theta0, sizeof(double) * pl->p, cudaMemcpyDeviceToDevice, f.s));
  else
    CK(cudaMemsetAsync(pl->th, 0, sizeof(double) * pl->p, f.s));
  int status = GLAM_OK;
  *nfit = 0;
  for (int k = 0; k < nlambda; ++k) {
    const auto t0 = std::chrono::steady_clock::now();
    LamOut lo;
    f.restarts = 0;
    CK(cudaMemsetAsync(&pl->sc->nonfinite, 0, sizeof(int), f.s));
    const int nsteps = scad ? o.steps : 1;
    for (int st = 0; st < nsteps; ++st) {
      // SCAD by the multistep adaptive lasso (Sec. 6.4): step 0 with the caller's weights, step
      // st >= 1 with the local linear approximation at the previous step's solution
      if (scad)
        CK(st == 0 ? cudaMemcpyAsync(pl->pen, pl->pen_base, sizeof(double) * pl->p,
                                     cudaMemcpyDeviceToDevice, f.s)
                   : launch_scad_weights(pl->p, pl->th, pl->pen_base, lams[k], kScadA, pl->pen, f.s));
      LamOut ls;
      CKS(solve_lambda<T>(f, lams[k], ls));
      lo.outer += ls.outer;
      lo.inner += ls.inner;
      lo.passes += ls.passes;
      lo.backtracks += ls.backtracks;
      lo.nnz = ls.nnz;
      lo.kkt = ls.kkt;
      lo.F = ls.F;
      lo.converged = ls.converged;
      lo.nonfinite = ls.nonfinite;
      if (!ls.converged) break;
    }
    CK(cudaMemcpyAsync(path + (size_t)k * pl->p, pl->th, sizeof(double) * pl->p, cudaMemcpyDeviceToDevice, f.s));
    CK(cudaStreamSynchronize(f.s));
    const double ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    const int lam_status = lo.converged ? GLAM_OK : (lo.nonfinite ? GLAM_ENONFINITE : GLAM_ENOCONV);
    if (stats) {
      glam_stats& s = stats[k];
      s.lambda = lams[k];
      s.objective = lo.F;
      s.kkt = lo.kkt;
      s.time_ms = ms;
      s.outer_iters = lo.outer;
      s.inner_iters = lo.inner;
      s.fp64_passes = lo.passes;
      s.armijo_backtracks = lo.backtracks;
      s.nnz = lo.nnz;
      s.status = lam_status;
      s.inner_restarts = f.restarts;
      s.reserved0 = 0;
    }
    if (lam_status != GLAM_OK) {
      status = lam_status;
      char buf[160];
      std::snprintf(buf, sizeof(buf), "lambda %d (%.6g): %s, KKT %.3g", k, lams[k],
                    lo.nonfinite ? "non-finite iterate" : "no convergence", lo.kkt);
      fail(pl, status, buf);
      break;
    }
    *nfit = k + 1;
  }
  CK(cudaEventRecord(pl->ev_out, f.s));
  CK(cudaStreamWaitEvent(pl->stream, pl->ev_out, 0));
  return status;
}

}  // namespace

int glam_kron_weights(glam_plan* pl, const double* V, int scaled, double* v1, double* v2, double* v3) {
  CKS(check_plan(pl));
  if (!V || !v1 || !v2 || !v3) return fail(pl, GLAM_EINVAL, "glam_kron_weights: NULL argument");
  if (pl->geo == nullptr) CKS(dalloc(pl, &pl->geo, geo_scratch_doubles(pl->n1, pl->n2, pl->n3)));
  CK(launch_geo_factors<double>((int)pl->n1, (int)pl->n2, (int)pl->n3, V, scaled ? 1 : 0, pl->geo, v1, v2, v3,
                                pl->stream));
  return GLAM_OK;
}

// longest captured chunk of inner iterations (each iteration adds two to four kernel nodes)
constexpr int kMaxCheckEvery = 4096;

int glam_fit_path(glam_plan* pl, const void* const X[3], const void* Y, const void* W,
                  const void* pen_w, int nlambda, double* lambda, const glam_opts* opts,
                  const double* Theta0, double* Theta_path, glam_stats* stats, int* nfit) {
  CKS(check_plan(pl));
  CKS(validate_X(pl, X));
  if (!Y || !W || !pen_w || !lambda || !Theta_path || !nfit)
    return fail(pl, GLAM_EINVAL, "glam_fit_path: NULL argument");
  if (nlambda < 1) return fail(pl, GLAM_EINVAL, "glam_fit_path: nlambda must be >= 1");
  glam_opts o;
  if (opts)
    o = *opts;
  else
    glam_opts_default(&o);
  if (o.check_every > kMaxCheckEvery)
    return fail(pl, GLAM_EINVAL, "glam_fit_path: check_every above 4096 (the captured chunk holds that many iterations)");
  if (o.check_every < 2) o.check_every = 2;
  if (o.check_every % 2) o.check_every += 1;
  if (o.max_inner < 1 || o.max_outer < 1 || o.max_linesearch < 1 || !(o.tol > 0) ||
      !(o.inner_forcing > 0) || !(o.inner_floor > 0) || !(o.armijo_b > 0 && o.armijo_b < 1) ||
      !(o.armijo_v > 0 && o.armijo_v < 1) || !(o.armijo_alpha0 > 0) ||
      !(o.iwls >= GLAM_IWLS_EXACT && o.iwls <= GLAM_IWLS_KRON2) || !(o.nu >= 0.0 && o.nu <= 1.0) ||
      !(o.penalty >= GLAM_PENALTY_LASSO && o.penalty <= GLAM_PENALTY_RIDGE) || o.steps < 1 ||
      !(o.enet_alpha >= 0.0 && std::isfinite(o.enet_alpha)) ||
      !(o.wait_limit_s >= 0.0 && o.wait_limit_s <= 3600.0))
    return fail(pl, GLAM_EINVAL, "glam_fit_path: bad options");
  if (std::isnan(lambda[0])) return fail(pl, GLAM_EINVAL, "glam_fit_path: lambda[0] is NaN");
  if (lambda[0] >= 0) {
    for (int k = 0; k < nlambda; ++k)
      if (!(lambda[k] >= 0)) return fail(pl, GLAM_EINVAL, "glam_fit_path: negative lambda");
  } else if (!(o.lambda_min_ratio > 0.0 && o.lambda_min_ratio <= 1.0)) {
    return fail(pl, GLAM_EINVAL, "glam_fit_path: lambda_min_ratio must be in (0, 1]");
  }
  if (pl->precision == GLAM_FP64)
    return fit_impl<double>(pl, X, (const double*)Y, (const double*)W, (const double*)pen_w, nlambda,
                            lambda, o, Theta0, Theta_path, stats, nfit);
  return fit_impl<float>(pl, X, (const float*)Y, (const float*)W, (const double*)pen_w, nlambda,
                         lambda, o, Theta0, Theta_path, stats, nfit);
}

// ======================================================================== diagnostics
int64_t glam_launch_count(void) { return launch_count(); }

namespace {
template <typename T>
int time_inner_impl(glam_plan* pl, const void* const X[3], const glam_quad* q, int reps, double* ms) {
  Ops<T> op(pl, pl->stream, X);
  const T* V = (const T*)q->V;
  cudaEvent_t a, b;
  CK(cudaEventCreate(&a));
  CK(cudaEventCreate(&b));
  const int slot = sizeof(T) == 8 ? 1 : 0;
  if constexpr (sizeof(T) == 4) {
    if (pl->um_form)
      CK(launch_fused_umma_const((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2, (int)pl->p3,
                                 pl->um_form, op.X[0], op.X[1], pl->um_cst, pl->stream));
    if (pl->tc_split)
      CK(launch_fused_tc_const((int)pl->n1, (int)pl->n2, (int)pl->p1, (int)pl->p2, op.X[0], op.X[1],
                               pl->tc_cst, pl->tc_split, pl->stream));
  }
  // the fused adjoint + prox kernel updates a control block; the timing runs use one of their
  // own that never reports convergence
  InnerCtl* tctl = nullptr;
  bool use_ap = false;
  if constexpr (sizeof(T) == 4) {
    use_ap = adjprox_supported((int)pl->n3, (int)pl->p3, (int)(pl->p2 * pl->p1), op.X[2], op.w.Sb) != 0;
    if (use_ap) {
      CKS(x3_rows_setup(pl, op.X[2], pl->stream));
      CK(cudaMalloc(&tctl, sizeof(InnerCtl)));
      InnerCtl h{};
      h.l = 1;
      h.max_iter = 1 << 30;
      h.delta = 1e-3;
      h.stop_abs = -1.0;
      CK(cudaMemcpy(tctl, &h, sizeof(InnerCtl), cudaMemcpyHostToDevice));
    }
  }
  auto timed = [&](int which) -> int {
    ms[which] = 0.0;
    bool use_tc = false, use_um = false;
    // the weights as the fit reads them: BF16 plans stream their own BF16 copy
    const void* Vin = pl->Vb != nullptr ? (const void*)pl->Vb : (const void*)V;
    if constexpr (sizeof(T) == 4) {
      use_um = pl->um_form && fused_tc_pointers_ok((const float*)pl->um_cst, op.w.dn, (const float*)Vin);
      use_tc = !use_um && pl->tc_split && fused_tc_pointers_ok(pl->tc_cst, op.w.dn, V);
    }
    const bool fused = pl->fused[slot] || use_tc || use_um;
    if (which == 0 && !fused) return GLAM_OK;
    if (which == 3 && fused && use_ap) return GLAM_OK;  // part of ms[2]
    for (int r = -2; r < reps; ++r) {
      if (r == 0) CK(cudaEventRecord(a, pl->stream));
      switch (which) {
        case 0:
          if constexpr (sizeof(T) == 4) {
            if (use_um) {
              CK(launch_fused_umma((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2, (int)pl->p3,
                                   pl->um_form, pl->Vb != nullptr, pl->um_cst, op.w.dn, op.X[0], op.X[2], Vin,
                                   op.w.Sb, pl->stream, nullptr, &pl->sc->timeout, kDefaultWaitNs,
                                   r > -2));  // programmatic dependent launches, as in the fit path
              break;
            }
            if (use_tc) {
              CK(launch_fused_slab_tc((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1,
                                      (int)pl->p2, (int)pl->p3, pl->tc_cst, op.w.dn, V,
                                      op.w.Sb, pl->stream, nullptr, &pl->sc->timeout, op.X[2],
                                      pl->tc_split));
              break;
            }
          }
          CK(launch_fused_slab<T>((int)pl->n1, (int)pl->n2, (int)pl->n3, (int)pl->p1, (int)pl->p2,
                                  op.X[0], op.X[1], op.w.dn, V, op.w.Sb, pl->stream, nullptr,
                                  &pl->sc->timeout, op.X[2], (int)pl->p3));
          break;
        case 1:
          if (fused) return GLAM_OK;  // folded into the fused kernel
          CK(launch_gemm<T, T>(d_mode3_fwd(pl), op.X[2], op.w.dn, op.w.Ta, pl->stream));
          break;
        case 2:
          if constexpr (sizeof(T) == 4) {
            if (fused && use_ap) {
              CK(launch_adjprox((int)pl->n3, (int)pl->p3, (int)(pl->p2 * pl->p1), op.X[2], op.w.Sb,
                                pl->gk, pl->x0, pl->x1, pl->pen, pl->ptmp, op.w.grad, pl->th,
                                1.0 / (double)pl->n, tctl, &pl->sc->timeout, pl->stream, false, pl->x3rows));
              break;
            }
          }
          CK(launch_gemm<T, T>(d_mode3_adj(pl, pl->ksplit), op.X[2], op.w.Sb, op.w.Qpart, pl->stream));
          break;
        default:
          CK(launch_prox<T, double>(pl->p, pl->ksplit, op.w.Qpart, pl->gk, 1.0, pl->x0, pl->x1,
                                    pl->pen, pl->ptmp, 1.0 / (double)pl->n, nullptr, 0.5, 1e-3, 0.0,
                                    nullptr, pl->stream, op.w.grad, pl->th));
      }
    }
    CK(cudaEventRecord(b, pl->stream));
    CK(cudaEventSynchronize(b));
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, a, b));
    ms[which] = (double)t / reps;
    return GLAM_OK;
  };
  int st = GLAM_OK;
  for (int k = 0; k < 4 && st == GLAM_OK; ++k) st = timed(k);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (tctl) cudaFree(tctl);
  return st;
}
}  // namespace

int glam_time_inner_kernels(glam_plan* pl, const void* const X[3], const glam_quad* q, int reps,
                            double* ms) {
  CKS(check_plan(pl));
  CKS(single_component(pl, "glam_time_inner_kernels"));
  CKS(validate_X(pl, X));
  if (!q || !q->V || !ms || reps < 1) return fail(pl, GLAM_EINVAL, "glam_time_inner_kernels: bad argument");
  if (pl->precision == GLAM_FP64) return time_inner_impl<double>(pl, X, q, reps, ms);
  return time_inner_impl<float>(pl, X, q, reps, ms);
}
