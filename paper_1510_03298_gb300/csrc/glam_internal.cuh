// Internal declarations of libglam (not part of the ABI).
//
// Layout: paper arrays n1 x n2 x n3 are C-order (n3, n2, n1) buffers (vec of App. A);
// Theta is (p3, p2, p1); a marginal design X_j is the C-order (p_j, n_j) buffer XT_j
// (column-major n_j x p_j).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "glam.h"

namespace glam {


// Launches kernel k; with pdl the launch may begin while the preceding kernel of the stream is
// still running (programmatic dependent launch): k then must execute griddep_wait() before it
// reads anything that kernel writes or writes anything it reads.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*k)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, bool pdl,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = pdl ? at : nullptr;
  cfg.numAttrs = pdl ? 1u : 0u;
  return cudaLaunchKernelEx(&cfg, k, args...);
}

#ifdef __CUDACC__
// Waits until the preceding kernel of the stream has completed and its writes are visible (at
// once when this launch was not a programmatic dependent one), then lets the next kernel of the
// stream begin launching.
__device__ __forceinline__ void griddep_wait() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

constexpr int kThreads = 256;
constexpr int kTrials = 8;          // Armijo trial step sizes evaluated per n-stream pass
constexpr int kMaxRedBlocks = 1216; // 8 x 152 SMs: upper bound of blocks in a reduction grid
constexpr int kRedSlots = 2 * kTrials + 4;
constexpr int kMaxSplits = 16;      // split-K partials of the last G stage (mode 3), at most

// ------------------------------------------------------------------------------------
// Device-resident control of the inner PG loop (Sec. 3.2).  One instance per plan; every
// kernel of an inner iteration reads `done` first and returns when it is set, so a captured
// chunk of iterations costs nothing after convergence.
// ------------------------------------------------------------------------------------
struct InnerCtl {
  int l;                       // iteration index of the paper (1-based): omega_l = (l-1)/(l+2)
  int done;                    // nonzero: the loop has stopped
  int max_iter;                // cap on l
  int iters_run;               // iterations executed since the last reset
  unsigned int counter;        // last-block-done counter of the prox kernel
  int stop_reason;             // 1 converged, 2 cap
  unsigned long long crit_bits;  // atomicMax accumulator: max_m |x+_m - y_m| (double bits, >= 0)
  double delta;                // step size
  double lambda;               // penalty parameter
  double stop_abs;             // stop when max_m |x+_m - y_m| <= stop_abs
  double crit;                 // last criterion value
  double pen_l1, pen_l2;       // penalty J = sum_m w_m (pen_l1 |theta_m| + pen_l2 theta_m^2)
  double crit_first;           // criterion of the first iteration
  double div_factor;           // > 0: stop as diverged when crit > div_factor * crit_first
};

// A step larger than 1 / L_hat (opts.nu < 1) is given up when the step max_m |x+_m - y_m| grows
// past this multiple of its first value, or is not finite.
constexpr double kInnerDivFactor = 10.0;

#ifdef __CUDACC__
// End of an inner iteration, run once by the last block of the prox kernel: the stop criterion
// (1 converged, 2 iteration cap, 3 diverged) and the advance of the loop state.
__device__ __forceinline__ void ctl_finish_iteration(InnerCtl* ctl, double c) {
  ctl->crit = c;
  ctl->iters_run += 1;
  if (ctl->l == 1) ctl->crit_first = c;
  if (c <= ctl->stop_abs) {
    ctl->done = 1;
    ctl->stop_reason = 1;
  } else if (ctl->div_factor > 0.0 && !(c <= ctl->div_factor * ctl->crit_first)) {
    ctl->done = 1;
    ctl->stop_reason = 3;
  } else if (ctl->l >= ctl->max_iter) {
    ctl->done = 1;
    ctl->stop_reason = 2;
  }
  ctl->l += 1;
  ctl->crit_bits = 0ull;
  ctl->counter = 0u;
}
#endif

// Scalars produced by reductions and consumed by later kernels (all device-resident).
struct DevScalars {
  double loss;                 // f(eta) of the last family pass (already divided by n)
  double maxw;                 // max_i w_i of the last family pass
  double Lhat;                 // Prop. 1 bound for the last family pass
  double pen;                  // J(theta) (weighted l1) of the last penalty pass
  double F;                    // objective at the current outer iterate
  double dir;                  // -(1/n) <U, eta_bar - eta>
  double data_diff[kTrials];   // (1/n) sum a (l(eta + alpha_j d_eta) - l(eta))
  double pen_diff[kTrials];    // J(theta + alpha_j d) - J(theta)
  double pen_tilde_diff;       // J(theta~) - J(theta)
  double alpha;                // accepted Armijo step (0 if none)
  double F_new;
  double kkt_max;              // max_m r_m (unscaled)
  double lmax;                 // lambda_max
  int accepted;                // index j of the accepted trial, -1 if none in this pass
  int nnz;
  int nonfinite;               // set by kernels that meet a non-finite value
  int timeout;                 // set by a kernel whose bounded wait ran out
};

struct RedScratch {
  double* partial;             // kMaxRedBlocks * kRedSlots doubles
  unsigned int* counter;       // one counter (reset by the last block)
};

// ------------------------------------------------------------------------------------
// Generic strided, batched, split-K SIMT GEMM used for the mode products (App. A rho):
//   C[b, split][m, n] = sum_{k in split} A[b][m, k] * B[b][k, n]
// Optional B-operand extrapolation y = x + omega (x - x_prev) (Sec. 3.2) applied on load.
// ------------------------------------------------------------------------------------
struct GemmDesc {
  int M, N, K, batch, ksplit;
  int64_t sAb, sAm, sAk;
  int64_t sBb, sBk, sBn;
  int64_t sCb, sCm, sCn;
  int64_t sCsplit;
};

template <typename T, typename TB>
cudaError_t launch_gemm(const GemmDesc& d, const T* A, const TB* B, T* C, cudaStream_t s,
                        const TB* Bprev = nullptr, const TB* Bsub = nullptr,
                        const InnerCtl* ctl = nullptr, double omega = 0.0,
                        const int* skip = nullptr);

// ------------------------------------------------------------------------------------
// Fused bottleneck of Sec. 6.2: per slab i3, S_b[i3] = X2^T (V[i3] (.) (X2 (T_a[i3] X1^T))) X1
// (the last H stage and the first G stage on-chip; eta never reaches memory).  With X3T given,
// `Ta` is the correction d (p3 x p2p1) and the kernel forms T_a = X_3 d itself.
// ------------------------------------------------------------------------------------
template <typename T>
cudaError_t launch_fused_slab(int n1, int n2, int n3, int p1, int p2, const T* X1T, const T* X2T,
                              const T* Ta, const T* V, T* Sb, cudaStream_t s, const int* skip,
                              int* err, const T* X3T = nullptr, int p3 = 1);
int fused_slab_supported(int n1, int n2, int p1, int p2, int elem_bytes);
cudaError_t fused_prepare();

// The same product on tensor cores with FP32 accumulation, always forming T_a = X_3 d from the
// correction D (p3 x p2p1): split = 1 rounds every operand to TF32; split = 3 is the 3xTF32
// form (each operand as hi + lo, three MMAs per product: about FP32 accuracy).  Cst is the
// constant block of fused_tc_const_floats floats written by launch_fused_tc_const from X_1^T and
// X_2^T (once per set of designs).  fused_tc_supported tells whether the shape is in the
// kernel's domain for that form.
cudaError_t launch_fused_slab_tc(int n1, int n2, int n3, int p1, int p2, int p3, const float* Cst,
                                 const float* D, const float* V, float* Sb, cudaStream_t s,
                                 const int* skip, int* err, const float* X3T, int split);
cudaError_t launch_fused_tc_const(int n1, int n2, int p1, int p2, const float* X1T, const float* X2T,
                                  float* Cst, int split, cudaStream_t s);
int64_t fused_tc_const_floats(int n1, int n2, int p1, int p2);
int fused_tc_supported(int n1, int n2, int n3, int p1, int p2, int p3, int split);
// Cst, D and V are bulk-copied by the kernel: each must start on a 16-byte boundary
int fused_tc_pointers_ok(const float* Cst, const float* D, const float* V);
cudaError_t fused_tc_prepare();

// The same product on the 5th-generation tensor cores (tcgen05, accumulators in tensor memory):
// form 1 TF32, 3 3xTF32 (about FP32 accuracy), 16 BF16 operands, FP32 accumulation throughout.  T_a
// = X_3 D is formed in the kernel from the correction D (p3 x p2p1, FP32).  Cst is the constant
// block (fused_umma_const_bytes bytes, written by launch_fused_umma_const from X_1^T and X_2^T
// once per set of designs); V is FP32, or BF16 for form 16 with v_bf16.  Every wait of the
// kernel gives up after wait_ns nanoseconds and sets *err.  With pdl the launch may overlap the
// preceding kernel of the stream: the kernel reads D (and writes Sb) only after that kernel has
// completed, and reads V, X_1, X_3 and the constant block before, so the preceding kernel must not
// write those.  fused_umma_supported tells whether
// the shape is in the kernel's domain (n1 <= 128, n1 a multiple of 4 (8 for BF16), n2 a multiple
// of 32 up to 128 (3xTF32) or 256, p1, p2 <= 32).
cudaError_t fused_umma_prepare();
// eta = H(<X_j>, Theta) for single-precision plans on the tcgen05 kernel (first H stage and MMA0
// in FP32 FMAs, MMA1 in 3xTF32), one CTA per SM, eta written with coalesced stores; after
// fused_umma_prepare.  Domain: n1 <= 128, n1 % 4 == 0, n2 % 32 == 0, n2 <= 224, p1, p2 <= 32.  A
// device wait that runs out (bounded by 2 s) sets *err.
int predict_umma_supported(int n1, int n2, int n3, int p1, int p2, int p3);
cudaError_t launch_predict_umma(int n1, int n2, int n3, int p1, int p2, int p3, const float* X1T, const float* X2T,
                                const float* X3T, const float* Theta, float* eta, int* err, cudaStream_t st);
int fused_umma_supported(int n1, int n2, int n3, int p1, int p2, int p3, int form);
int64_t fused_umma_const_bytes(int n1, int n2, int n3, int p1, int p2, int p3, int form);
cudaError_t launch_fused_umma_const(int n1, int n2, int n3, int p1, int p2, int p3, int form,
                                    const float* X1T, const float* X2T, void* Cst, cudaStream_t st);
cudaError_t launch_fused_umma(int n1, int n2, int n3, int p1, int p2, int p3, int form, bool v_bf16,
                              const void* Cst, const float* D, const float* X1T, const float* X3T,
                              const void* V, float* Sb, cudaStream_t st, const int* skip, int* err,
                              uint64_t wait_ns, bool pdl = false);

// The last two stages of H for FP32 (modes 1 and 2, Sec. 6.1, Eq. eighteen) in one kernel:
// eta[i3] = X_2 (T_a[i3] X_1^T) per slab, T_a (n3 x p2p1) from the mode-3 product.
int predict_tiles_supported(int p1, int p2);
cudaError_t launch_predict_tiles(int n1, int n2, int n3, int p1, int p2, const float* XT1,
                                 const float* XT2, const float* Ta, float* eta, cudaStream_t s);
// Its first stage, T_a (n3 x P21) = X_3 (n3 x p3) . Theta (p3 x P21), for p3 <= 64.
int mode3_rows_supported(int p3);
cudaError_t launch_mode3_rows(int n3, int p3, int P21, const float* XT3, const float* Theta,
                              float* Ta, cudaStream_t s);

// A 2-D FP32 tensor map without swizzle (dims {dim0, dim1}, row stride stride1 bytes, box
// {box0, box1}; elements outside the tensor read as zero); 1 on success, 0 otherwise.
int encode_map_2d(CUtensorMap* m, const float* base, uint64_t dim0, uint64_t dim1, uint64_t stride1,
                  uint32_t box0, uint32_t box1);

// ------------------------------------------------------------------------------------
// Last G stage (mode 3 of Eq. nineteen) and the inner PG step of Sec. 3.2 in one kernel, for the
// FP32 products of the fit path: Q = X_3^T S_b (p3 x p2p1, every i3 summed in the CTA that owns
// the entry), then the prox step of launch_prox with lin = g_k, lin_scale = 1 and the anchor
// theta_k (x, xp, out, gk, pen, anchor FP64; dnext FP32).  With pdl the launch may overlap the
// preceding kernel of the stream; the kernel touches no memory before that kernel has completed.
// adjprox_supported tells whether the
// shape and pointers allow its tensor copies.
// ------------------------------------------------------------------------------------
int adjprox_supported(int n3, int p3, int P21, const float* X3T, const float* Sb);
cudaError_t launch_adjprox(int n3, int p3, int P21, const float* X3T, const float* Sb, const double* gk,
                           const double* x, const double* xp, const double* pen, double* out,
                           float* dnext, const double* anchor, double inv_n, InnerCtl* ctl, int* err,
                           cudaStream_t s, bool pdl = false, const int* x3_rows = nullptr);
// For each row j3 of X_3^T (p3 x n3), the range [first, last + 1) of its nonzero entries (n3, 0 when
// none): with it launch_adjprox reads only the rows i3 of S_b that meet a nonzero entry.
cudaError_t launch_x3_rows(int n3, int p3, const float* X3T, int* rows, cudaStream_t s);

// Tensor-product weights (Sec. 6.2, Eq. kronweight): the factors w1 (n1), w2 (n2), w3 (n3) of W
// read off its first row, column and tube, and check[0] = max |W - w1 w2 w3|, check[1] = max |W|
// (doubles as bits); the FP64 weighted Gram matrix M = X_j^T diag(w) X_j (pj x pj).
template <typename T>
cudaError_t launch_kron_factors(int64_t n1, int64_t n2, int64_t n3, const T* W, double* w1, double* w2,
                                double* w3, unsigned long long* check, cudaStream_t s);
cudaError_t launch_weighted_gram(int nj, int pj, const double* XT, const double* w, double* M,
                                 cudaStream_t s);
// The geometric-mean tensor approximation of a weight array V (C-order (n3, n2, n1), Sec. 6.2):
// v_j(i) = exp(mean of log V over slice i of mode j - mean of log V over all cells), the means
// over the cells with V > 0 (1 for a slice with none), summed in a fixed order; scaled != 0
// multiplies v_1 by the overall geometric mean.  scratch holds geo_scratch_doubles(n1, n2, n3).
template <typename TV>
cudaError_t launch_geo_factors(int n1, int n2, int n3, const TV* V, int scaled, double* scratch, double* v1,
                               double* v2, double* v3, cudaStream_t s);
int64_t geo_scratch_doubles(int64_t n1, int64_t n2, int64_t n3);
// Q = H(<M_j>, d) on p-sized arrays in one launch (one CTA per slab j3, d staged in shared memory);
// supported when d and the M_j fit in shared memory; kron_product_prepare sets the kernel's
// shared-memory limit (call it outside any stream capture, before the first launch).
template <typename T>
int kron_product_supported(int p1, int p2, int p3);
template <typename T>
cudaError_t kron_product_prepare(int p1, int p2, int p3);
template <typename T>
cudaError_t launch_kron_product(int p1, int p2, int p3, const T* M1, const T* M2, const T* M3,
                                const T* d, T* Q, const int* skip, cudaStream_t s);

// ------------------------------------------------------------------------------------
// Elementwise / reduction kernels.
// ------------------------------------------------------------------------------------
template <typename T, typename TV>
cudaError_t launch_family(int family, int64_t n, const T* eta, const T* Y, const T* A, TV* V, T* VZ,
                          T* U, double rho_prod, DevScalars* sc, RedScratch red, cudaStream_t s);

template <typename T>
cudaError_t launch_scale(int64_t n, const T* in, T* out, double scale, cudaStream_t s);

template <typename Tq, typename TP>
cudaError_t launch_prox(int64_t p, int ksplit, const Tq* Qpart, const TP* lin, double lin_scale,
                        const TP* x, const TP* xprev, const TP* pen_w, TP* out, double inv_n,
                        InnerCtl* ctl, double omega, double delta, double lambda,
                        const double* Lhat, cudaStream_t s, Tq* dnext = nullptr,
                        const TP* anchor = nullptr);

template <typename TE, typename T>
cudaError_t launch_armijo_stream(int family, int64_t n, const TE* eta, const T* deta, const TE* Y,
                                 const TE* A, double alpha0, double b, int j0, DevScalars* sc,
                                 RedScratch red, cudaStream_t s);

// penalty J = sum_m w_m (l1 |theta_m| + l2 theta_m^2) in the three kernels below
template <typename T>
cudaError_t launch_armijo_penalty(int64_t p, const T* theta, const T* theta_t, const T* pen_w,
                                  double alpha0, double b, int j0, DevScalars* sc, RedScratch red,
                                  cudaStream_t s, double l1 = 1.0, double l2 = 0.0);

cudaError_t launch_armijo_select(double lambda, double v, double alpha0, double b, int j0,
                                 DevScalars* sc, cudaStream_t s);

template <typename T>
cudaError_t launch_armijo_update(int64_t p, T* theta, const T* theta_t, const DevScalars* sc,
                                 cudaStream_t s);

template <typename T>
cudaError_t launch_kkt(int64_t p, const double* g, const T* theta, const T* pen_w, double lambda,
                       DevScalars* sc, RedScratch red, cudaStream_t s, double l1 = 1.0,
                       double l2 = 0.0);

template <typename T>
cudaError_t launch_penalty(int64_t p, const T* theta, const T* pen_w, DevScalars* sc,
                           RedScratch red, cudaStream_t s, double l1 = 1.0, double l2 = 0.0);

template <typename T>
cudaError_t launch_lambda_max(int64_t p, const double* g0, const T* pen_w, DevScalars* sc,
                              RedScratch red, cudaStream_t s);

template <typename TI, typename TO>
cudaError_t launch_convert(int64_t n, const TI* in, TO* out, cudaStream_t s);

template <typename T>
cudaError_t launch_extrap(int64_t n, const T* x, const T* xp, double omega, T* y, cudaStream_t s);

cudaError_t launch_gram(int nj, int pj, const double* XT, double* gram, cudaStream_t s);

// Multistep-adaptive-lasso weights of the SCAD penalty: w = base * p'_lambda(|theta|) / lambda.
cudaError_t launch_scad_weights(int64_t p, const double* theta, const double* base, double lambda,
                                double a, double* w, cudaStream_t s);

template <typename T>
cudaError_t launch_sum_splits(int64_t p, int ksplit, const T* part, T* out, cudaStream_t s);

template <typename T>
cudaError_t launch_vmul(int64_t n, const T* V, T* x, const int* skip, cudaStream_t s);
template <typename T>
cudaError_t launch_add(int64_t n, const T* x, T* y, const int* skip, cudaStream_t s);

template <typename T>
cudaError_t launch_check_finite(int64_t n, const T* x, DevScalars* sc, cudaStream_t s);

// Penalized negative log-likelihood and its vector-Jacobian product (glam_penalized_nll): the
// cells pass (loss f into sc->loss, U = -(g/n) u, GY = g df/dy) and the coefficient pass
// (J(theta) into sc->pen, F = f + lambda J, grad = Q + g lambda w sign(theta)); g = *gout or 1.
template <typename T>
cudaError_t launch_nll_cells(int family, int64_t n, const T* eta, const T* Y, const T* A,
                             const double* gout, T* U, T* GY, DevScalars* sc, RedScratch red,
                             cudaStream_t s);
template <typename T>
cudaError_t launch_nll_coef(int64_t p, const T* theta, const T* pen_w, double lambda,
                            const double* gout, const T* Q, T* grad, double* F, DevScalars* sc,
                            RedScratch red, cudaStream_t s);

template <typename T>
cudaError_t launch_loss_only(int family, int64_t n, const T* eta, const T* Y, const T* A,
                             double* out, RedScratch red, cudaStream_t s);

int num_sms();

// Record msg as the calling thread's last error (read by glam_last_error(NULL)); returns code.
int thread_fail(int code, const std::string& msg);
// ---- banded marginal designs (glam_band.cu): at most kBand consecutive nonzeros per row
constexpr int kBand = 4;
struct BandDesign {
  int* start = nullptr;   // n: first column of row i
  double* val = nullptr;  // n x kBand: X(i, start(i) + t)
  int* lo = nullptr;      // p: the rows touching column j are [lo(j), hi(j))
  int* hi = nullptr;
};
cudaError_t launch_band_fwd(int64_t A, int Cin, int Cout, int64_t B, const BandDesign& X, const double* In,
                            double* Out, cudaStream_t s);
cudaError_t launch_band_adj(int64_t A, int Cin, int Cout, int64_t B, const BandDesign& X, const double* In,
                            double* Out, cudaStream_t s);
bool band_form(const double* XT, int n, int p, std::vector<int>& start, std::vector<double>& val,
               std::vector<int>& lo, std::vector<int>& hi);

// Number of model components c of a plan (1, or c > 1 for glam_plan_create_components).
int plan_components(const glam_plan* pl);

// Process-wide count of kernels launched by the library (graph replays add their kernel nodes).
void count_launches(int64_t k);
int64_t launch_count();
void set_capturing(bool on);

}  // namespace glam
