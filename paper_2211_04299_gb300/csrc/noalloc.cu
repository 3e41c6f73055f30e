// Bellman sweep that allocates no memory: bellman_apply_ell_noalloc_dev.
//
// Some callers cannot allocate device memory while they run: a server or control loop that
// hands the whole device to its own pooling allocator up front (a second allocator's
// cudaMalloc would fail or fragment that pool), or latency-critical code where cudaMalloc /
// cudaFree, which can synchronise the whole device, would stall every other stream.  For
// them this entry point takes the MDP, v and the outputs as caller-owned device arrays in the
// caller's own layout and keeps its only scratch (the per-block partial maxima and the
// done-counter of the grid reduction) in a fixed array that is part of the library's device
// image.  The paper has no counterpart; it is an interface convenience of this library.
#include "mdp_internal.cuh"

#include <math.h>
#include <mutex>

namespace {

constexpr int NA_THREADS = 256;
constexpr int NA_MAX_BLOCKS = (int)(MDP_NOALLOC_MAX_STATES / NA_THREADS);
// [0, NA_MAX_BLOCKS): block maxima of |Tv - v|; then the done-counter and a bad-column flag
constexpr int NA_CTRL = NA_MAX_BLOCKS;

}  // namespace

// Fixed scratch: every GPU that loads the library holds these 33 KiB until the process exits.
// All calls share it; it keeps the last call's contents.
static __device__ __align__(256) double g_noalloc_scratch[NA_MAX_BLOCKS + 32];

namespace {

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mu;
void* g_na_ptr[NA_MAX_DEVICES];  // device address of g_noalloc_scratch, per device

// One thread per state: Q(s,a) = g(s,a) + gamma sum_j val[a][s][j] v[col[a][s][j]] for every
// a, lowest-index argmin, Tv(s), and the grid maximum of |Tv - v| (Sec. 2 Bellman operator).
__global__ void __launch_bounds__(NA_THREADS)
noalloc_sweep_kernel(int64_t S, int A, int k, const int32_t* __restrict__ col,
                     const double* __restrict__ val, const double* __restrict__ g, double gamma,
                     const double* __restrict__ v, double* __restrict__ Tv,
                     int32_t* __restrict__ pi, double* __restrict__ res_inf, double* scratch) {
  unsigned* counter = reinterpret_cast<unsigned*>(scratch + NA_CTRL);
  unsigned* bad_flag = counter + 1;
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double phi = 0.0;
  int bad = 0;
  if (s < S) {
    double best = 0.0;
    int abest = 0;
    for (int a = 0; a < A; ++a) {
      const int64_t base = ((int64_t)a * S + s) * k;
      double acc = 0.0;
      for (int j = 0; j < k; ++j) {
        const int32_t c = col[base + j];
        if (c < 0 || (int64_t)c >= S) {  // skip the access, report through res_inf
          bad = 1;
          continue;
        }
        acc = fma(val[base + j], v[c], acc);
      }
      const double q = fma(gamma, acc, g[(int64_t)a * S + s]);
      if (a == 0 || q < best) {
        best = q;
        abest = a;
      }
    }
    Tv[s] = best;
    pi[s] = abest;
    phi = fabs(best - v[s]);
  }
  if (bad) atomicOr(bad_flag, 1u);
  __shared__ double sh[32];
  const double bm = mdp::block_max(phi, sh);
  if (threadIdx.x == 0) scratch[blockIdx.x] = bm;
  if (!mdp::arrive_last(counter)) return;
  double m = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) m = max(m, __ldcg(scratch + b));
  m = mdp::block_max(m, sh);
  if (threadIdx.x == 0) {
    const unsigned flagged = atomicExch(bad_flag, 0u);
    *res_inf = flagged ? __longlong_as_double(0x7ff8000000000000LL) : m;
  }
}

}  // namespace

extern "C" int bellman_apply_ell_noalloc_dev(int64_t S, int32_t A, int32_t k, const int32_t* col,
                                             const double* val, const double* g, double gamma,
                                             const double* v, double* Tv, int32_t* pi,
                                             double* res_inf, void* stream) {
  if (S < 1 || A < 1 || k < 1 || (int64_t)k > S || !(gamma > 0.0 && gamma < 1.0)) return MDP_EINVAL;
  if (!col || !val || !g || !v || !Tv || !pi || !res_inf) return MDP_EINVAL;
  if (S > (int64_t)MDP_NOALLOC_MAX_STATES) return MDP_EINVAL;  // beyond the fixed scratch
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return MDP_EDEVICE;
  if (dev < 0 || dev >= NA_MAX_DEVICES) return MDP_EINVAL;
  void* scratch = nullptr;
  {
    // first call on this device: look up the scratch's device address (no allocation)
    std::lock_guard<std::mutex> lock(g_na_mu);
    scratch = g_na_ptr[dev];
    if (!scratch) {
      if (cudaGetSymbolAddress(&scratch, g_noalloc_scratch) != cudaSuccess || !scratch)
        return MDP_EDEVICE;
      g_na_ptr[dev] = scratch;
    }
  }
  cudaStream_t st = (cudaStream_t)stream;
  // the done-counter and the bad-column flag must start at zero
  if (cudaMemsetAsync((double*)scratch + NA_CTRL, 0, 2 * sizeof(unsigned), st) != cudaSuccess)
    return MDP_EDEVICE;
  const int blocks = (int)((S + NA_THREADS - 1) / NA_THREADS);
  noalloc_sweep_kernel<<<blocks, NA_THREADS, 0, st>>>(S, A, k, col, val, g, gamma, v, Tv, pi,
                                                      res_inf, (double*)scratch);
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}
