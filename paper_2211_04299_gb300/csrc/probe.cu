// Diagnostics: the arithmetic-rate probe mdp_probe_alu and the bounded-wait self-test
// mdp_selftest_wait.
//
// The plain FP64 form of the solver accumulates every transition entry with an FP64 FMA, and
// GB300's FP64 pipe is a small fraction of its FP32 pipe, so that form's Bellman sweep can be
// bound by FP64 arithmetic rather than by HBM.  This probe measures the FMA rate of the GPU it
// runs on, so that such a kernel's roofline is stated against a measured peak: every thread
// keeps eight independent FMA chains (no dependency stalls between them), the grid covers
// every SM several times over, and the rate is 2 flops per FMA over the best of three timed
// launches (CUDA events on a private stream, after one warm-up launch).
#include "mdp_internal.cuh"

namespace {

constexpr int PR_THREADS = 256;
constexpr int PR_CHAINS = 8;

template <typename T>
__global__ void __launch_bounds__(PR_THREADS)
fma_chains_kernel(int iters, T m, T a, T* out) {
  T x[PR_CHAINS];
#pragma unroll
  for (int c = 0; c < PR_CHAINS; ++c) x[c] = (T)(threadIdx.x + c) * (T)1e-3;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) x[c] = fma(x[c], m, a);
  }
  T s = 0;
#pragma unroll
  for (int c = 0; c < PR_CHAINS; ++c) s += x[c];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;  // keeps the chains live
}

template <typename T>
int probe(int iters, double* tflops) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return mdp::set_error(MDP_EDEVICE, "mdp_probe_alu: no device");
  const int blocks = sms * 8;
  T* out = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int r = MDP_OK;
  if (cudaMalloc(&out, (size_t)blocks * PR_THREADS * sizeof(T)) != cudaSuccess)
    return mdp::set_error(MDP_ENOMEM, "mdp_probe_alu: cudaMalloc failed");
  if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    r = mdp::set_error(MDP_EDEVICE, "mdp_probe_alu: stream or event creation failed");
  }
  float best = 0.f;
  for (int rep = 0; rep < 4 && r == MDP_OK; ++rep) {
    cudaEventRecord(e0, st);
    fma_chains_kernel<T><<<blocks, PR_THREADS, 0, st>>>(iters, (T)0.999999, (T)1e-7, out);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
      r = mdp::set_error(MDP_EDEVICE, "mdp_probe_alu: launch failed");
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0 && (best == 0.f || ms < best)) best = ms;  // rep 0 is the warm-up
  }
  if (r == MDP_OK) {
    const double flops = 2.0 * PR_CHAINS * (double)iters * blocks * PR_THREADS;
    *tflops = flops / (best * 1e-3) / 1e12;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (st) cudaStreamDestroy(st);
  cudaFree(out);
  return r;
}

// One thread waits, through the pipelines' bounded-wait helper, on an mbarrier that expects one
// arrival; with arrive = 0 nothing arrives (and no copy is in flight), so the wait runs out after
// `limit` clock cycles and raises the error flag; with arrive = 1 the thread arrives first.
__global__ void wait_selftest_kernel(long long limit, int arrive, int* err) {
  __shared__ __align__(8) uint64_t bar;
  mdp::mbar_init(&bar, 1);
  mdp::mbar_fence_init();
  if (arrive) mdp::mbar_arrive(&bar);
  mdp::mbar_wait(&bar, 0, err, limit);
}

}  // namespace

extern "C" int mdp_selftest_wait(int64_t limit_cycles, int32_t arrive) {
  if (limit_cycles < 1 || limit_cycles > mdp::MBAR_WAIT_CYCLES || (arrive != 0 && arrive != 1))
    return mdp::set_error(MDP_EINVAL, "mdp_selftest_wait: limit must lie in [1, 2^31], arrive 0 or 1");
  int* err = nullptr;
  if (cudaMalloc(&err, sizeof(int)) != cudaSuccess)
    return mdp::set_error(MDP_ENOMEM, "mdp_selftest_wait: cudaMalloc failed");
  int h = 0;
  cudaMemset(err, 0, sizeof(int));
  wait_selftest_kernel<<<1, 1>>>((long long)limit_cycles, arrive, err);
  const cudaError_t e = cudaMemcpy(&h, err, sizeof(int), cudaMemcpyDeviceToHost);
  cudaFree(err);
  if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return mdp::set_error(MDP_EDEVICE, "mdp_selftest_wait: launch failed");
  return h ? mdp::set_error(MDP_ETIMEOUT, "bounded device wait ran out (self-test)") : MDP_OK;
}

extern "C" int mdp_probe_alu(int32_t dtype, double* tflops) {
  if (!tflops) return mdp::set_error(MDP_EINVAL, "mdp_probe_alu: null output");
  if (dtype == MDP_F64) return probe<double>(20000, tflops);
  if (dtype == MDP_F32) return probe<float>(400000, tflops);
  return mdp::set_error(MDP_EINVAL, "mdp_probe_alu: dtype must be MDP_F32 or MDP_F64");
}
