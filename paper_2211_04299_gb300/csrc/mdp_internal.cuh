// Internal declarations shared by the CUDA translation units of libmdpgpu.
//
// Device data layout (chosen at upload, independent of the caller's layout):
//   dense P : [S][A][ld]   state-major, ld = S rounded up to 32 elements (128-byte rows),
//                          pad columns zero; a state's A rows are one contiguous stream.
//   ELL     : val, col [S][A][kp], kp = k rounded up to 4; pad entries val 0, col 0.
//   g       : [S][A] FP64, plus a double-float copy [S][A] for the mixed path.
//   mask    : [S][A] bytes or null.
// Value vectors of the FP64 path are double[ldv]; of the mixed path float2 (hi, lo)
// double-float pairs.  Krylov vectors are double (FP64 path) or float (mixed path),
// [W+1][ldq] with ldq a multiple of 32 elements.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mdpgpu.h"

namespace mdp {

constexpr int WMAX = 64;          // largest GMRES restart length
constexpr int RED_THREADS = 256;  // threads of every reduction-carrying kernel
constexpr int MAX_RED_BLOCKS = 2048;

enum Kind { KIND_DENSE = 0, KIND_ELL = 1 };

// Read-only view of a handle's transition data on the device.
struct DevMDP {
  int64_t S;
  int32_t A;
  int32_t k;
  int32_t kp;      // padded ELL row length
  int64_t ld;      // padded dense row length
  int32_t kind;
  int32_t pdt;     // MDP_F32 / MDP_F64
  double gamma;
  float gamma_hi, gamma_lo;
  const void* P;       // dense P or ELL val
  const int32_t* col;  // ELL columns
  const double* g64;   // [S][A]
  const float2* gdf;   // [S][A] double-float copy (FP32 P only)
  const uint8_t* mask; // [S][A] or null
  int64_t span;        // ELL: max |col - s| over the stored entries (set by validation); -1 unknown
};

// ------------------------------------------------------------------ double-float arithmetic
// Error-free transforms (Knuth's TwoSum, Dekker's Fast2Sum, FMA-based TwoProduct) and the
// double-word sum/product of Joldes, Muller & Popescu (ACM TOMS 2017).  The *_rn
// intrinsics keep the compiler from contracting the steps into FMAs.
struct dfl { float hi, lo; };

__device__ __forceinline__ dfl two_sum(float a, float b) {
  float s = __fadd_rn(a, b);
  float bb = __fsub_rn(s, a);
  float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  return {s, e};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {  // needs |a| >= |b| or a == 0
  float s = __fadd_rn(a, b);
  float e = __fsub_rn(b, __fsub_rn(s, a));
  return {s, e};
}
__device__ __forceinline__ dfl two_prod(float a, float b) {
  float p = __fmul_rn(a, b);
  return {p, __fmaf_rn(a, b, -p)};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
  dfl s = two_sum(x.hi, y.hi);
  dfl t = two_sum(x.lo, y.lo);
  dfl v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}
__device__ __forceinline__ dfl df_neg(dfl x) { return {-x.hi, -x.lo}; }
__device__ __forceinline__ dfl df_sub(dfl x, dfl y) { return df_add(x, df_neg(y)); }
__device__ __forceinline__ dfl df_mul(dfl x, dfl y) {
  dfl c = two_prod(x.hi, y.hi);
  float t = __fmaf_rn(x.lo, y.hi, __fmul_rn(x.hi, y.lo));
  return fast_two_sum(c.hi, __fadd_rn(c.lo, t));
}
__device__ __forceinline__ dfl df_mul_f(dfl x, float b) {  // double-float times float
  dfl c = two_prod(x.hi, b);
  return fast_two_sum(c.hi, __fmaf_rn(x.lo, b, c.lo));
}
__device__ __forceinline__ bool df_lt(dfl a, dfl b) {
  return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
}
__device__ __forceinline__ double df_to_d(dfl x) { return (double)x.hi + (double)x.lo; }
__device__ __forceinline__ dfl d_to_df(double d) {
  float hi = (float)d;
  return {hi, (float)(d - (double)hi)};
}
__device__ __forceinline__ dfl shfl_xor_df(dfl x, int off) {
  return {__shfl_xor_sync(0xffffffffu, x.hi, off), __shfl_xor_sync(0xffffffffu, x.lo, off)};
}

// Packed pairs of FP32 values in one 64-bit register and the paired FP32 instructions of this
// architecture (add / sub / mul / fma .rn.f32x2: two IEEE round-to-nearest operations per
// instruction, never contracted), so two independent error-free transforms issue as one.
typedef unsigned long long f2x;
__device__ __forceinline__ f2x f2_pack(float a, float b) {
  f2x r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void f2_unpack(f2x x, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(x));
}
__device__ __forceinline__ f2x f2_add(f2x a, f2x b) {
  f2x r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x f2_sub(f2x a, f2x b) {
  f2x r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x f2_mul(f2x a, f2x b) {
  f2x r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ f2x f2_fma(f2x a, f2x b, f2x c) {
  f2x r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
// Two running sums, each of products p * (vh + vl), in the manner of AccDF below but on packed
// pairs: with nvh = -vh (exact), the product's high part is -(p * nvh) and its error
// fma(p, vh, p * nvh); TwoSum of the high parts is written with the negated term, so every step is
// exact as in the scalar form.  sh holds the two high sums, sl their error terms.
__device__ __forceinline__ void f2_acc(f2x& sh, f2x& sl, f2x p, f2x vh, f2x nvh, f2x vl) {
  const f2x nph = f2_mul(p, nvh);          // -(p * vh) rounded
  const f2x pe = f2_fma(p, vh, nph);       // exact error of the product
  const f2x s = f2_sub(sh, nph);           // sh + p * vh rounded
  const f2x bb = f2_sub(s, sh);
  const f2x t2 = f2_sub(sh, f2_sub(s, bb));
  const f2x e = f2_sub(t2, f2_add(nph, bb));  // TwoSum error: (sh - (s - bb)) + (ph - bb)
  sl = f2_add(sl, f2_add(e, f2_fma(p, vl, pe)));
  sh = s;
}

// The double-float value of a packed pair of running sums (hi pair sh, error pair sl): TwoSum of
// the two high words, the two error words and its error added in FP32, then Fast2Sum.
__device__ __forceinline__ dfl f2_to_df(f2x sh, f2x sl) {
  float h0, h1, l0, l1;
  f2_unpack(sh, h0, h1);
  f2_unpack(sl, l0, l1);
  const dfl t = two_sum(h0, h1);
  return fast_two_sum(t.hi, __fadd_rn(t.lo, __fadd_rn(l0, l1)));
}

// Running sum of products p * v with p FP32 and v double-float, accurate to about 2^-48
// relative: each product is split exactly (TwoProduct), the high parts are added with
// TwoSum and every error term goes to a low word; every 32 terms the chunk is folded into
// a double-word total so the low word never grows long.
struct AccDF {
  float sh, sl;
  dfl tot;
  int n;
  __device__ __forceinline__ void init() { sh = 0.f; sl = 0.f; tot = {0.f, 0.f}; n = 0; }
  __device__ __forceinline__ void add(float p, float2 v) {
    float ph = __fmul_rn(p, v.x);
    float pe = __fmaf_rn(p, v.x, -ph);
    dfl s = two_sum(sh, ph);
    sh = s.hi;
    sl = __fadd_rn(sl, __fadd_rn(s.lo, __fmaf_rn(p, v.y, pe)));
  }
  __device__ __forceinline__ void tick() {
    if (++n == 8) fold();
  }
  __device__ __forceinline__ void fold() {
    tot = df_add(tot, two_sum(sh, sl));
    sh = 0.f; sl = 0.f; n = 0;
  }
  __device__ __forceinline__ dfl result() {
    fold();
    return tot;
  }
};

// ------------------------------------------------------------------ L2 cache policy
// Gathered vectors (v, x: a few MB, read many times) are loaded with an evict-last L2
// policy so the multi-GB transition streams (evict-first, ld.cs) do not push them out.
__device__ __forceinline__ uint64_t l2_keep_policy() {
  uint64_t pol;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
  return pol;
}
__device__ __forceinline__ float2 ld_keep(const float2* p, uint64_t pol) {
  float2 r;
  asm volatile("ld.global.nc.L2::cache_hint.v2.f32 {%0, %1}, [%2], %3;"
               : "=f"(r.x), "=f"(r.y) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ double ld_keep(const double* p, uint64_t pol) {
  double r;
  asm volatile("ld.global.nc.L2::cache_hint.f64 %0, [%1], %2;" : "=d"(r) : "l"(p), "l"(pol));
  return r;
}
__device__ __forceinline__ float ld_keep(const float* p, uint64_t pol) {
  float r;
  asm volatile("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(r) : "l"(p), "l"(pol));
  return r;
}

// ------------------------------------------------------------------ small helpers
template <typename T> __device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
template <typename T> __device__ __forceinline__ T warp_max(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = max(x, __shfl_xor_sync(0xffffffffu, x, o));
  return x;
}

// Block-wide sum/max of one value per thread (blockDim.x == RED_THREADS); result valid in
// every thread.  Uses sh[32].
template <typename T> __device__ __forceinline__ T block_sum(T x, T* sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  x = warp_sum(x);
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  T r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : T(0);
  if (wid == 0) r = warp_sum(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}
template <typename T> __device__ __forceinline__ T block_max(T x, T* sh) {
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  x = warp_max(x);
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  T r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : T(0);
  if (wid == 0) r = warp_max(r);
  if (threadIdx.x == 0) sh[0] = r;
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

// "Last block done" detection for single-pass grid reductions: every block stores its
// partial results, then calls this; it returns true in exactly one block (the last to
// arrive), which may then read all partials.  That block resets the counter to zero, so a
// counter that starts at zero is zero again after every launch.
// nb = number of blocks taking part (gridDim.x for a plain launch, the instance's block
// count inside a batched launch).
__device__ __forceinline__ bool arrive_last(unsigned* counter, int nb) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned t = atomicAdd(counter, 1u);
    am_last = (t == (unsigned)nb - 1u);
    if (am_last) *counter = 0u;
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}
__device__ __forceinline__ bool arrive_last(unsigned* counter) { return arrive_last(counter, gridDim.x); }

// Position of a block within the blocks that work on one instance: (blockIdx.x, gridDim.x)
// for a plain launch; inside a batched launch, the block's index among its instance's
// blocks and that instance's block count.
struct GridPos {
  int bid;
  int nb;
};
__device__ __forceinline__ GridPos this_grid() { return GridPos{(int)blockIdx.x, (int)gridDim.x}; }

// ------------------------------------------------------------------ bulk-copy pipeline
// cp.async.bulk (TMA, untiled) global -> shared copies completing on an mbarrier, and the
// mbarrier operations of a producer/consumer ring.  Every wait is bounded: after about a
// second of spinning it raises *err and returns false, so a kernel never hangs the GPU.
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_fence_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(b)),
               "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(b)) : "memory");
}
// try_wait with a suspend-time hint: the warp sleeps in hardware until the phase completes
// (or about 20 us pass) instead of spinning through issue slots.
__device__ __forceinline__ bool mbar_test(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_addr(b)), "r"(parity), "r"(20000u)
      : "memory");
  return ok != 0;
}
constexpr long long MBAR_WAIT_CYCLES = 1LL << 31;  // about one second at the SM clock
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, int* err,
                                          long long limit = MBAR_WAIT_CYCLES) {
  if (mbar_test(b, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_test(b, parity)) {
    if (clock64() - t0 > limit) {
      if (err) atomicExch(err, 1);
      return false;
    }
  }
  return true;
}
// bytes and both addresses must be multiples of 16
__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// ------------------------------------------------------------------ GMRES control block
// Modes of the device-resident inner-solver state machine.  Each kernel of an Arnoldi step
// runs only in the modes listed beside it and returns at once otherwise, so a whole step
// can be enqueued (or replayed from a graph) without the host looking at the state.
enum GmresMode {
  GM_STEP = 0,      // matvec + CGS2 + Givens of step i are due
  GM_EST = 1,       // Givens estimate passed the gate: estimate ||r||_inf from Q z
  GM_CHECK = 2,     // estimate passed: form the candidate and test the true residual
  GM_RESTART = 3,   // cycle full: form the candidate, restart from its true residual
  GM_FINISH = 4,    // breakdown or step cap: form the candidate and stop
  GM_DONE = 5,      // candidate accepted (ctl.status says why)
  GM_IDLE = 6
};

enum GmresStatus { GS_RUNNING = 0, GS_CONVERGED = 1, GS_BREAKDOWN = 2, GS_CAP = 3 };

// Scalars produced by the Bellman sweep and by reduction kernels.
struct SweepOut {
  double res_inf;   // ||Phi||_inf
  double res_nrm2;  // ||Phi||_2
};

struct GmresCtl {
  int mode;
  int status;
  int i;            // current Arnoldi index: Q_0..Q_i exist, Q_i is normalised
  int W;            // restart length
  int steps;        // Arnoldi steps so far (all cycles)
  int max_steps;
  int restarts;
  int dsel;         // delta_base = dbuf[dsel], candidate = dbuf[1 - dsel]
  int from_rhs;     // step 0 of a cycle reads its start vector from rbuf (scaled by 1/beta)
  int est_runs, checks, loop_iters;
  double thr;       // target on the inf-norm of the residual
  double sqrtS;
  double beta;      // 2-norm of the cycle's start residual
  double rho;       // |gv[i+1]| = least-squares residual estimate
  double hnext;     // H[i+1][i]
  double xscale;    // scale of the vector the next matvec reads (1/beta or 1/hnext)
  double last_inf;  // last inf-norm computed (estimate or true residual)
  double last_nrm2;
  double thr_saved; // threshold of the current outer iteration (kept for a resumed solve)
  int accept_est;   // accept on the Arnoldi-relation estimate (the caller verifies exactly)
  int resumed;
  int est_last;     // steps at the last estimate pass
  double est_ratio; // ||r||_inf / ||r||_2 last observed (start residual, estimate or restart)
  double H[(WMAX + 1) * WMAX];  // column-major, leading dimension WMAX+1
  double cs[WMAX], sn[WMAX];
  double gv[WMAX + 1];
  double y[WMAX];
  double z[WMAX + 1];
  double c1[WMAX + 1], c2[WMAX + 1];  // CGS2 coefficients of pass 1 and pass 2
  float c1f[WMAX + 1], c2f[WMAX + 1], yf[WMAX], zf[WMAX + 1];
  float xscalef;
  int once;         // this step needs no second projection (set by the first pass)
};

// Right-hand side of the inexact stopping rule for outer residual res = ||Phi_k||_inf
// (Sec. 3): alpha ||Phi_k||_inf with the constant alpha of Alg. 2 (forcing_c = 0), or
// alpha_k ||Phi_k||_inf with the forcing sequence alpha_k = min(alpha, forcing_c res), kept at
// or above floor.  Host and device evaluate the same expression.
__host__ __device__ inline double inexact_threshold(double alpha, double forcing_c, double res,
                                                    double floor) {
  if (forcing_c > 0.0) {
    const double ak = alpha < forcing_c * res ? alpha : forcing_c * res;
    const double t = ak * res;
    return t > floor ? t : floor;
  }
  return alpha * res;
}

__device__ __forceinline__ void gmres_set_scale(GmresCtl* c, double s) {
  c->xscale = s;
  c->xscalef = (float)s;
}

// Start an inner solve of J^pi delta = r (Krylov init, Sec. 2.2): beta = ||r||_2 from the
// norms of r, threshold alpha ||r||_inf (or thr when alpha == 0; the saved threshold when
// resuming), first basis vector r / beta.  A start that already meets the threshold ends at
// once with delta = 0.
__device__ inline void gmres_init_ctl(GmresCtl* c, double thr, double alpha, double sqrtS, int W,
                                      int max_steps, const SweepOut* rhs, int resume,
                                      int accept_est, double forcing_c = 0.0,
                                      double thr_floor = 0.0) {
  c->W = W;
  c->max_steps = max_steps;
  c->sqrtS = sqrtS;
  c->steps = 0;
  c->restarts = 0;
  c->est_runs = 0;
  c->checks = 0;
  c->loop_iters = 0;
  c->i = 0;
  c->dsel = 0;
  c->from_rhs = 1;
  c->status = GS_RUNNING;
  c->last_inf = rhs->res_inf;
  c->last_nrm2 = 0.0;
  if (resume) {
    c->thr = c->thr_saved;
  } else {
    c->thr = alpha > 0.0 ? inexact_threshold(alpha, forcing_c, rhs->res_inf, thr_floor) : thr;
    c->thr_saved = c->thr;
  }
  c->accept_est = accept_est;
  c->resumed = resume;
  const double beta = rhs->res_nrm2;
  c->beta = beta;
  c->est_last = 0;
  c->est_ratio = beta > 0.0 ? rhs->res_inf / beta : 1.0;
  for (int j = 0; j <= WMAX; ++j) c->gv[j] = 0.0;
  c->gv[0] = beta;
  gmres_set_scale(c, beta > 0.0 ? 1.0 / beta : 0.0);
  if (!(rhs->res_inf > c->thr) || beta == 0.0) {
    c->mode = GM_DONE;
    c->status = GS_CONVERGED;
  } else {
    c->mode = GM_STEP;
  }
}

// ------------------------------------------------------------------ launch descriptors
struct SweepLaunch {
  DevMDP d;
  int arith;            // 0: FP64, 1: double-float (needs FP32 P)
  const void* v;        // value vector (double or float2)
  const int32_t* pi_in; // optional: evaluate only row pi_in(s) (T^pi v)
  int32_t* pi_out;
  void* tv_out;         // same type as v
  double* tv64_out;
  void* phi_out;        // Krylov type: double (arith 0) or float (arith 1)
  double* margin_out;
  const int32_t* pi_ref;// optional: residual of this policy at v
  void* rref_out;       // Krylov type: g^pi_ref + gamma P^pi_ref v - v
  SweepOut* out;
  SweepOut* ref_out;    // norms of rref_out
  void* partials;       // >= MAX_RED_BLOCKS * 4 doubles
  unsigned* counter;
  int lanes;            // ELL lanes per row (1,2,4,8); 0 = choose
  int grid;             // 0 = choose
  int* err;             // raised by a bounded wait that ran out (bulk-copy kernels)
  int no_tma;           // force the register-streaming kernel
  int no_window;        // ELL: force the global-gather kernel even for banded columns
};

int launch_sweep(const SweepLaunch& L, cudaStream_t st);

struct MatvecLaunch {
  DevMDP d;
  int kt;               // Krylov type: 0 double, 1 float
  const int32_t* pi;
  const void* x;        // input vector (kt), scaled by *xscale_d / *xscale_f if given
  const GmresCtl* ctl;  // when set: gate on ctl->mode and take x / scale from the control
  int gate_mode;        // run only if ctl->mode == gate_mode (or gate_mode2)
  int gate_mode2;
  const void* x_rhs;    // cycle start vector (ctl->from_rhs)
  const void* x_w0;     // previous step's w, buffer for even steps
  const void* x_w1;     // ... odd steps
  void* qbase;          // Krylov basis [W+1][ldq]: the normalised input is written to Q_i
  int64_t ldq;
  double a, b, c;       // out = a*x + b*u + c*(P^pi x)
  const void* u;
  void* out;            // or chosen by parity when ctl is set
  void* out0;
  void* out1;
  SweepOut* norms;      // optional inf/2-norm of out
  GmresCtl* ctl_rw;     // when set (with gate CHECK/RESTART): finalise the check
  void* partials;
  unsigned* counter;
  int lanes;
  int grid;
  int* err;
  int no_tma;
  const void* x_pre;    // gate STEP with a preconditioner: multiply this vector (M^{-1} Q_i,
                        // already formed) with scale 1 and leave Q_i alone
  int no_window;        // ELL: force the global-gather kernel even for banded columns
};

int launch_matvec(const MatvecLaunch& L, cudaStream_t st);

struct KrylovBufs {
  int kt;         // 0 double, 1 float
  int64_t S;
  int64_t ldq;
  void* Q;        // [W+1][ldq]
  void* w0;       // w buffers (parity of i)
  void* w1;
  void* rbuf;     // cycle start residual
  void* d0;       // delta buffers
  void* d1;
  void* partials;
  unsigned* counter;
  GmresCtl* ctl;
  int grid;
  int maxm;       // column capacity of the tall-skinny kernels (>= restart + 1)
  const void* ec = nullptr;  // two-level preconditioner: coarse part of the candidate, added
  int lb = 0;                // to each state of its block (block = 2^lb states)
};

// One Arnoldi step after the matvec: Gram-Schmidt (one or two projections) + norm + Givens +
// mode decision.
int launch_cgs2_givens(const KrylovBufs& B, cudaStream_t st);
// Gated on EST/RESTART/FINISH: candidate = delta_base + Q_{0..i} y and, in EST mode, the
// Arnoldi-relation bound ||Q_{0..i} z + z_{i+1} w / hnext||_inf that decides CHECK or not.
int launch_estimate(const KrylovBufs& B, cudaStream_t st);
// Body-end kernel of the graph-resident inner loop: keeps the WHILE node looping while the
// solve is not done and fewer than cap iterations have run (a hard guard on the loop).
int launch_loop_cond(cudaGraphConditionalHandle hc, GmresCtl* ctl, int cap, cudaStream_t st);
// Initialise the control block for a new inner solve (device side, no host copy).
// resume != 0 keeps the threshold of the previous solve (ctl->thr_saved); accept_est != 0
// ends the solve as soon as the Arnoldi-relation estimate meets the threshold, leaving the
// exact test to the caller (the next Bellman sweep).
int launch_gmres_init(const KrylovBufs& B, double thr, double sqrtS, int W, int max_steps,
                      const SweepOut* rhs_norms, double alpha, cudaStream_t st, int resume = 0,
                      int accept_est = 0, double forcing_c = 0.0, double thr_floor = 0.0);

// Two-level preconditioner (right preconditioning of the inner solve): restriction to blocks
// of 2^lb consecutive states by averaging, prolongation by copying, Galerkin coarse operator
// J_c = R J^pi Pr, M^{-1} q = q + Pr J_c^{-1} R q.
struct PrecondK {
  const GmresCtl* ctl;
  int64_t S, nc;        // states, coarse blocks
  int64_t ldq, ldc;     // leading dimensions of Q (states) and of E and J_c^{-1} (blocks, % 4 == 0)
  int lb;
  const void* rbuf;     // Arnoldi-step inputs, as the matvec reads them
  const void* w0;
  const void* w1;
  void* Q;              // [W+1][ldq] Krylov basis (Q_i written here)
  void* E;              // [W][ldc]: E_i = J_c^{-1} R Q_i
  void* ec;             // [ldc]: sum_j y_j E_j
  void* z;              // [ldq]: Q_i + Pr E_i
  float* f;             // [ldc]: R Q_i (zero past nc)
  float* inv;           // [nc][ldc]: J_c^{-1} (zero past nc in each row)
};
// Per-policy setup buffers: the rows of J_c with their row sums and off-diagonal sums, then
// its LU (nc * (2 bw + 3) floats), and the coefficients of the triangular solves with L and U
// ([nc][32] floats each, dinv [nc]).
struct PrecondScratch {
  float* band;
  float* cl;
  float* cu;
  float* dinv;
};
constexpr int PC_BW_MAX = 31;  // coarse half-bandwidth handled (one warp lane per band entry)
// Largest |block(col) - block(s)| over all ELL entries, atomically maxed into *bw (zeroed first).
int launch_coarse_bandwidth(const DevMDP& d, int lb, int* bw, cudaStream_t st);
// Per policy: band of J_c, its banded LU in place, the solve coefficients, J_c^{-1} into p.inv.
int launch_coarse_setup(const DevMDP& d, const int32_t* pi, const PrecondK& p, int bw,
                        const PrecondScratch& w, cudaStream_t st);
// Per Arnoldi step (gated on STEP): Q_i and R Q_i, E_i, z = Q_i + Pr E_i.
int launch_coarse_step(const PrecondK& p, int kt, cudaStream_t st);
// *count += number of s in [0, S) with pi[s] != ref[s]
int launch_count_changed(const int32_t* pi, const int32_t* ref, int64_t S, int* count, cudaStream_t st);
// Gated on EST / RESTART / FINISH: ec = sum_{j <= i} y_j E_j.
int launch_coarse_combine(const PrecondK& p, int kt, cudaStream_t st);

// Value update v += delta (double or double-float), delta = chosen by ctl (or given).
int launch_value_update(int kt, void* v, const void* d0, const void* d1, const GmresCtl* ctl,
                        const void* delta, int64_t S, cudaStream_t st);
// Conversions between double and double-float vectors, and fills.
int launch_d_to_df(const double* in, float2* out, int64_t n, cudaStream_t st);
int launch_df_to_d(const float2* in, double* out, int64_t n, cudaStream_t st);
int launch_fill_zero(void* p, size_t bytes, cudaStream_t st);
// Transpose [A][S] -> [S][A] for g (and produce the double-float copy when gdf != null).
int launch_cost_transpose(const double* gAS, double* gSA, float2* gdf, int64_t S, int32_t A,
                          cudaStream_t st);
// Device-side validation of uploaded data: error flags into flags[0..4] (values, columns, row
// sums, costs, allowed actions) and, for ELL, the largest |col - s| into flags[6] (atomicMax).
int launch_validate(const DevMDP& d, int* flags, cudaStream_t st);
// After launch_validate on the same stream: reorder the nonzeros within each row of banded ELL
// data (validation's flags clean, column reach within the windowed sweep's) so that the
// windowed sweep's shared-memory gathers spread over the banks (sweep.cu).  val and col are
// the handle's own copies of d.P and d.col.
int launch_ell_bank_order(const DevMDP& d, void* val, int32_t* col, const int* flags,
                          cudaStream_t st);
// flags[5] |= 1 when a policy entry is out of range or disallowed by the mask.
int launch_check_policy(const int32_t* pi, int64_t S, int32_t A, const uint8_t* mask, int* flags,
                        cudaStream_t st);

// ------------------------------------------------------------------ batched iGMRES-PI
// A batch solves many independent ELL MDPs (FP32 P, mixed precision) with one graph launch.
// Each instance runs Alg. 2 as a device-side state machine:
//   SWEEP0 (first Bellman sweep) -> INNER (Arnoldi steps; GmresCtl.mode) -> SWEEPV (the
//   sweep that gives pi_{k+1}, Phi_{k+1} and the exact inner residual of pi_k) -> INNER ... -> DONE
// One loop iteration runs every kernel once over the instances that are in the matching
// phase.  An instance is cut into "virtual blocks" per kernel family; a batched kernel walks
// the virtual blocks of a compacted list of instances with a grid-stride loop, and each
// virtual block runs the same kernel body as a single-instance launch whose grid has that
// instance's block count, so results do not depend on the batch.
enum BatchPhase { BP_SWEEP0 = 0, BP_INNER = 1, BP_SWEEPV = 2, BP_DONE = 3, BP_FREE = 4 };
constexpr int BATCH_CLASSES = 4;  // ELL lanes per row 1, 2, 4, 8 (class = log2)

struct BatchInst {
  DevMDP d;
  int64_t ldq;
  float2* v;        // V_k (double-float)
  float2* tv;       // T V_k
  float* phi;       // Phi_k = T V_k - V_k
  float* rref;      // exact residual of pi_k at V_{k+1}
  float* Q;         // Krylov basis [W+1][ldq]
  float* w0;
  float* w1;
  float* rbuf;
  float* d0;
  float* d1;
  int32_t* pib[2];  // policy double buffer: pi_k = pib[cur]
  GmresCtl* ctl;
  SweepOut* sout;   // [4]
  void* partials;
  unsigned* counter;
  double sqrtS;
  int nb_sw, nb_mv, nb_ts, nb_ew;  // virtual blocks per kernel family
  int cls_sw, cls_mv;              // ELL lane class of the sweep / matvec
  // state
  int phase, cur, k, reps, status, starting, rhs_sel;
  int inner, restarts, checks, sweeps, loops, breakdowns;
  double thr, res;
};

struct BatchList {  // active instances of one kernel family, with block prefix sums
  int* inst;        // [n]
  int* first;       // [n + 1]; the blocks of inst[j] are first[j] .. first[j+1]-1
  int* count;       // number of listed instances
};

struct BatchDev {
  BatchInst* insts;
  int n;
  double alpha, tol;
  double forcing_c, thr_floor;  // forcing sequence of the inner stopping rule
  int W, max_steps, max_outer;
  BatchList sw;                 // sweeps due
  BatchList mv;                 // inner solves running (matvec blocks)
  BatchList ts;                 // inner solves running (tall-skinny kernels)
  BatchList ew;                 // inner solves running (element-wise kernels)
  BatchList all;                // every instance (element-wise kernels)
  double** vout;                // [n] output T(V_K) per instance
  int32_t** pout;               // [n] output pi_K per instance
  int* ctr;                     // [0] instances not done, [1] loop iterations, [2] guard hit
  int max_iters;
};

// Position of a block among the virtual blocks of one instance (binary search in first[]).
__device__ __forceinline__ int batch_slot(const int* first, int cnt, int vb) {
  int lo = 0, hi = cnt - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (first[mid] <= vb) lo = mid; else hi = mid - 1;
  }
  return lo;
}

// Copy an instance record into shared memory with every thread of the block (one word per
// thread, so the loads overlap), then wait for the copy.
__device__ __forceinline__ void batch_stage_inst(const BatchInst* g, BatchInst* s) {
  static_assert(sizeof(BatchInst) % 4 == 0, "BatchInst is copied in 4-byte words");
  constexpr int NW = (int)(sizeof(BatchInst) / 4);
  const uint32_t* src = reinterpret_cast<const uint32_t*>(g);
  uint32_t* dst = reinterpret_cast<uint32_t*>(s);
  for (int i = threadIdx.x; i < NW; i += blockDim.x) dst[i] = src[i];
  __syncthreads();
}

// Run f(instance, GridPos) for every virtual block of list L (grid-stride over blocks).
template <class F>
__device__ __forceinline__ void batch_for_each(const BatchList& L, F&& f) {
  const int cnt = *(volatile const int*)L.count;
  if (cnt <= 0) return;
  const int total = L.first[cnt];
  for (int vb = blockIdx.x; vb < total; vb += gridDim.x) {
    const int j = batch_slot(L.first, cnt, vb);
    const int f0 = L.first[j];
    f(L.inst[j], GridPos{vb - f0, L.first[j + 1] - f0});
    __syncthreads();
  }
}

// Batched kernel families (sweep.cu, krylov.cu).  grid = physical blocks.  Each virtual
// block runs the kernel body for its instance's lane count (cls_sw / cls_mv), so one launch
// serves instances of every shape.
int launch_batch_sweep(const BatchDev& B, int grid, cudaStream_t st);
int batch_sweep_grid();
// which: 0 Arnoldi-step matvec, 1 true-residual matvec (CHECK / RESTART), 2 timing only
int launch_batch_matvec(const BatchDev& B, int which, int grid, cudaStream_t st);
int batch_matvec_grid();
int launch_batch_cgs(const BatchDev& B, int maxm, int grid, cudaStream_t st);
int launch_batch_estimate(const BatchDev& B, int maxm, int grid, cudaStream_t st);
int batch_ts_grid(int maxm);
// Block counts of the single-instance ELL kernels (library choice), shared with the batch.
int ell_sweep_lanes_default(const DevMDP& d);
int ell_matvec_lanes_default(const DevMDP& d);
int krylov_blocks(int64_t S);

// Shared by the batch and the server drivers (batch.cu).
struct BatchGrids {
  int sw, mv, ts, ew;  // physical blocks of the sweep, matvec, tall-skinny, element-wise kernels
};
// Instance record for data d: geometry, lane classes and the workspace carved from base (a
// 256-byte aligned block of batch_workspace_bytes(d, W) bytes, zeroed by the caller).
size_t batch_workspace_bytes(const DevMDP& d, int W);
void batch_setup_inst(const DevMDP& d, int W, char* base, BatchInst& I);
// Reset an instance record to the start of a solve (phase SWEEP0, counters zero).
void batch_reset_state(BatchInst& I);
// Enqueue one loop iteration (with_cond: end with cudaGraphSetConditional on hc).
int batch_enqueue_iteration(const BatchDev& B, const BatchGrids& g, int maxm, cudaStream_t st,
                            cudaGraphConditionalHandle hc, int with_cond);
// Start of a launch of loop iterations: zero the iteration counter, rebuild the sweep list
// (instances activated since the last launch join it).
int batch_enqueue_relist(const BatchDev& B, cudaStream_t st);
// T(V_K) as double and pi_K of the instance whose record is at rec (device) into vo / po.
int batch_enqueue_output_one(const BatchInst* rec, int64_t S, double* vo, int32_t* po,
                             cudaStream_t st);
BatchGrids batch_max_grids(int maxm);

// Handle access for the batch driver (api.cu): the device view of a handle's data, its
// device, and the thread-local error message of mdp_last_error.
const DevMDP* handle_view(mdp_t h);
// Wait for a load enqueued by mdp_load_*_async on the handle (its stream only), check it.
int handle_finish_pending(mdp_t h);
int handle_device(mdp_t h);
int set_error(int code, const char* msg);

int num_sms();

}  // namespace mdp
