// acopf_objective_noalloc: the generation-cost objective for callers that
// must not allocate device memory.
//
// Its scratch (one partial sum per block and the blocks' arrival counter)
// lives in a file-scope static device array, so the call itself allocates
// nothing: no cudaMalloc, no cudaFree, no allocating library routine.  The
// array exists on every GPU that loads this library, from load until the
// process exits.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "../../include/acopf.h"

namespace acopf {
void set_last_error(const std::string& msg);  // capi.cpp: the message acopf_last_error returns

namespace {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocMaxBlocks = 1024;
constexpr int64_t kNoAllocMaxTerms = int64_t(1) << 24;
constexpr int kMaxDevices = 64;

struct NoAllocScratch {
  double part[kNoAllocMaxBlocks];  // block sums of the current call
  unsigned int ticket;             // blocks that have finished (must start at 0)
};

static __device__ __align__(256) NoAllocScratch g_noalloc_scratch;

// Device address of g_noalloc_scratch per device, taken with that device
// current and kept once the lookup has succeeded (a failed lookup, such as
// one that met an error left over from earlier work, is retried by the next
// call).  In host code the symbol's name is only a host-side handle, never a
// device address.
NoAllocScratch* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu[kMaxDevices];

// f = sum_g c2 pg^2 + c1 pg + c0: each thread sums its terms in index order
// (grid stride), each block reduces in a fixed tree order, and the last
// block to arrive adds the block sums in block order, so the value does not
// depend on scheduling.
__global__ void __launch_bounds__(kNoAllocThreads) k_objective_noalloc(
    int n, const double* __restrict__ pg, const double* __restrict__ c2,
    const double* __restrict__ c1, const double* __restrict__ c0, double* f,
    NoAllocScratch* scratch) {
  double v = 0.0;
  for (int g = blockIdx.x * kNoAllocThreads + threadIdx.x; g < n; g += gridDim.x * kNoAllocThreads)
    v += fma(fma(__ldg(c2 + g), __ldg(pg + g), __ldg(c1 + g)), __ldg(pg + g), __ldg(c0 + g));
  __shared__ double sh[kNoAllocThreads / 32];
  __shared__ int last;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kNoAllocThreads / 32; ++k) s += sh[k];
    scratch->part[blockIdx.x] = s;
    __threadfence();
    const unsigned int t = atomicAdd(&scratch->ticket, 1u);
    last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (last && threadIdx.x < 32) {
    __threadfence();
    double r = 0.0;
    for (int k = threadIdx.x; k < static_cast<int>(gridDim.x); k += 32)
      r += __ldcg(&scratch->part[k]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r += __shfl_down_sync(0xffffffffu, r, o);
    if (threadIdx.x == 0) {
      *f = r;
      scratch->ticket = 0u;
    }
  }
}

acopf_status fail(acopf_status s, const std::string& m) {
  set_last_error(m);
  return s;
}

}  // namespace
}  // namespace acopf

extern "C" acopf_status acopf_objective_noalloc(int64_t n_gen, const double* pg, const double* c2,
                                                const double* c1, const double* c0, double* f_dev,
                                                acopf_stream stream) {
  using namespace acopf;
  if (n_gen < 0 || n_gen > kNoAllocMaxTerms)
    return fail(ACOPF_E_INVALID_ARG,
                "acopf_objective_noalloc: n_gen must be in [0, 16777216] (static scratch limit)");
  if (!f_dev || (n_gen > 0 && (!pg || !c2 || !c1 || !c0)))
    return fail(ACOPF_E_INVALID_ARG, "acopf_objective_noalloc: null pointer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return fail(ACOPF_E_CUDA, "acopf_objective_noalloc: no usable current device");
  // First successful call on this device: resolve the static array's device
  // address.
  NoAllocScratch* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mu[dev]);
    if (!g_scratch_addr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess || !p) {
        if (e == cudaSuccess) e = cudaErrorInvalidSymbol;
        return fail(ACOPF_E_CUDA, std::string("acopf_objective_noalloc: cudaGetSymbolAddress: ") +
                                      cudaGetErrorString(e));
      }
      g_scratch_addr[dev] = static_cast<NoAllocScratch*>(p);
    }
    scratch = g_scratch_addr[dev];
  }
  cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
  // The arrival counter must start at zero; the array keeps what the last
  // call left, so clear it in stream order before the launch.
  e = cudaMemsetAsync(&scratch->ticket, 0, sizeof(unsigned int), s);
  if (e != cudaSuccess)
    return fail(ACOPF_E_CUDA, std::string("acopf_objective_noalloc: ") + cudaGetErrorString(e));
  int blocks = static_cast<int>((n_gen + kNoAllocThreads - 1) / kNoAllocThreads);
  if (blocks < 1) blocks = 1;
  if (blocks > kNoAllocMaxBlocks) blocks = kNoAllocMaxBlocks;
  k_objective_noalloc<<<blocks, kNoAllocThreads, 0, s>>>(static_cast<int>(n_gen), pg, c2, c1, c0,
                                                          f_dev, scratch);
  e = cudaGetLastError();
  if (e != cudaSuccess)
    return fail(ACOPF_E_CUDA, std::string("acopf_objective_noalloc: ") + cudaGetErrorString(e));
  return ACOPF_OK;
}
