// glam_loss_eta_noalloc: the loss reduction f(eta) for callers that cannot allocate device
// memory.
//
// Some callers cannot call cudaMalloc at the point where they need the objective: code running
// while a stream is being captured into a CUDA graph (allocation calls are not capturable),
// hosts that own every byte of device memory through their own pool and forbid allocations
// behind their back, and real-time or signal-handler contexts where an allocation could block.
// The plan-based glam_loss keeps its reduction scratch in plan workspace that glam_plan_create
// allocates; this variant keeps it in one file-scope __device__ array of fixed size instead,
// and takes eta (computed by the caller, e.g. with glam_predict) rather than Theta, so it needs
// no other workspace.
//
// Scratch: kNoAllocBlocks FP64 partial sums followed by a completion counter, 8448 bytes in
// total, held by every GPU that loads the library until the process exits.  Every call shares
// it: calls whose kernels overlap on the GPU (different streams, or host threads on the same
// device) race on it, so issue them in one stream or serialize them.  The counter is cleared
// by each call (cudaMemsetAsync on the call's stream) and again by the kernel's last block.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "glam_family.cuh"
#include "glam_internal.cuh"

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocPerThread = 8;           // elements per thread per tile
constexpr int kNoAllocBlocks = 1024;           // maximum reduction grid (one partial per block)
// Largest accepted n: the cell limit of glam_plan_create, chosen for the interface.  The scratch
// does not depend on n (the grid is capped at kNoAllocBlocks blocks that stride over the cells).
constexpr int64_t kNoAllocMaxCells = (int64_t)1 << 40;
constexpr size_t kCounterOffset = (size_t)kNoAllocBlocks * sizeof(double);
constexpr size_t kScratchBytes = kCounterOffset + 256;

static __device__ __align__(256) unsigned char g_loss_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_loss_scratch on the current device, looked up once per device.
cudaError_t scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lk(g_mu);
  if (g_scratch_ptr[dev] == nullptr) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_loss_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return cudaSuccess;
}

// f(eta) = (1/n) sum_i a_i l_i (Sec. 2, Eq. two with the constants of glam.h), each cell's term
// from the same per-cell code as glam_loss (family_cell: App. B, with its clamp of eta before the
// exponential, so that a large eta gives the same finite term there and here, and a masked cell
// contributes exactly zero); every term is added to an FP64 accumulator, FP64 across threads and
// blocks, final sum in block order by the last block (the same bits on every run).
template <typename T>
__global__ void __launch_bounds__(kNoAllocThreads)
loss_noalloc_kernel(int family, int64_t n, const T* __restrict__ eta, const T* __restrict__ Y,
                    const T* __restrict__ A, double* __restrict__ out, unsigned char* scratch) {
  double* partial = reinterpret_cast<double*>(scratch);
  unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kCounterOffset);
  __shared__ double warp_part[kNoAllocThreads / 32];
  __shared__ bool is_last;
  double acc = 0.0;
  const int64_t tile = (int64_t)gridDim.x * blockDim.x * kNoAllocPerThread;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x * kNoAllocPerThread; base < n; base += tile) {
#pragma unroll
    for (int k = 0; k < kNoAllocPerThread; ++k) {
      const int64_t i = base + (int64_t)k * blockDim.x + threadIdx.x;
      if (i >= n) break;
      int clamped = 0;
      acc += (double)glam::family_cell<T>(family, eta[i], Y[i], A[i], clamped).l;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) warp_part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) b += warp_part[w];
    partial[blockIdx.x] = b;
    __threadfence();
    is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (is_last && threadIdx.x == 0) {
    double s = 0.0;
    for (unsigned int b = 0; b < gridDim.x; ++b) s += __ldcg(&partial[b]);
    *out = s / (double)n;
    *counter = 0u;
  }
}

}  // namespace

int glam_loss_eta_noalloc(int family, int precision, int64_t n, const void* eta, const void* Y,
                          const void* W, double* out, void* stream) {
  if (family != GLAM_GAUSSIAN_IDENTITY && family != GLAM_POISSON_LOG && family != GLAM_BINOMIAL_LOGIT &&
      family != GLAM_GAMMA_LOG)
    return glam::thread_fail(GLAM_EINVAL, "glam_loss_eta_noalloc: unknown family");
  if (precision != GLAM_FP64 && precision != GLAM_FP32)
    return glam::thread_fail(GLAM_EINVAL, "glam_loss_eta_noalloc: precision must be GLAM_FP64 or GLAM_FP32");
  if (n < 1 || n > kNoAllocMaxCells)
    return glam::thread_fail(GLAM_EINVAL,
                             "glam_loss_eta_noalloc: n must be in [1, 2^40] (a limit of the interface, "
                             "the same as a plan's; the scratch does not depend on n)");
  if (!eta || !Y || !W || !out) return glam::thread_fail(GLAM_EINVAL, "glam_loss_eta_noalloc: NULL array");
  void* scratch = nullptr;
  cudaError_t e = scratch_address(&scratch);
  if (e != cudaSuccess)
    return glam::thread_fail(GLAM_ECUDA, std::string("glam_loss_eta_noalloc: cudaGetSymbolAddress: ") +
                                             cudaGetErrorString(e));
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int64_t blocks = (n + (int64_t)kNoAllocThreads * kNoAllocPerThread - 1) /
                   ((int64_t)kNoAllocThreads * kNoAllocPerThread);
  if (blocks > kNoAllocBlocks) blocks = kNoAllocBlocks;
  if (blocks < 1) blocks = 1;
  unsigned char* sp = static_cast<unsigned char*>(scratch);
  e = cudaMemsetAsync(sp + kCounterOffset, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess)
    return glam::thread_fail(GLAM_ECUDA, std::string("glam_loss_eta_noalloc: ") + cudaGetErrorString(e));
  if (precision == GLAM_FP64)
    loss_noalloc_kernel<double><<<(int)blocks, kNoAllocThreads, 0, s>>>(
        family, n, static_cast<const double*>(eta), static_cast<const double*>(Y),
        static_cast<const double*>(W), out, sp);
  else
    loss_noalloc_kernel<float><<<(int)blocks, kNoAllocThreads, 0, s>>>(
        family, n, static_cast<const float*>(eta), static_cast<const float*>(Y),
        static_cast<const float*>(W), out, sp);
  glam::count_launches(1);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return glam::thread_fail(GLAM_ECUDA, std::string("glam_loss_eta_noalloc: launch: ") + cudaGetErrorString(e));
  return GLAM_OK;
}
