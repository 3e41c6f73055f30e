// Batched iGMRES-PI (Alg. 2) over many independent ELL MDPs in one CUDA-graph launch.
//
// Every instance runs the outer loop of Alg. 2 as a device-side state machine (BatchInst):
//   SWEEP0  first Bellman sweep at V_0: pi_0, T V_0, Phi_0 and ||Phi_0||
//   INNER   GMRES(W) on J^{pi_k} delta = Phi_k (or, when resumed, on the exact residual),
//           one Arnoldi step per loop iteration, accepted on the Arnoldi-relation estimate
//   SWEEPV  Bellman sweep at V_{k+1}: pi_{k+1}, Phi_{k+1}, and the exact residual of pi_k,
//           which either confirms the inner stopping rule or resumes the inner solve
//   DONE    ||Phi_k||_inf <= tol, or k = max_outer
// The graph is: init, then a WHILE node whose body is one loop iteration (sweeps due,
// controller, inner-solve prologue, Arnoldi step kernels, value update, loop condition),
// then the output conversion.  Control decisions are taken on the device by one block
// (a thread per instance), which also rebuilds the compacted lists of instances each
// kernel family serves next, so idle instances cost no blocks.
#include "mdp_internal.cuh"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

using namespace mdp;

namespace {

constexpr int CTRL_THREADS = 1024;
constexpr int EW_THREADS = 256;

// ------------------------------------------------------------------ list building
// Exclusive block scan of (count, blocks) pairs; blockDim.x == CTRL_THREADS.
__device__ int2 scan_pairs(int2 x, int2* tot) {
  __shared__ int2 ws[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int2 inc = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int a = __shfl_up_sync(0xffffffffu, inc.x, o);
    const int b = __shfl_up_sync(0xffffffffu, inc.y, o);
    if (lane >= o) { inc.x += a; inc.y += b; }
  }
  if (lane == 31) ws[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    const int nw = blockDim.x >> 5;
    int2 t = lane < nw ? ws[lane] : make_int2(0, 0);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int a = __shfl_up_sync(0xffffffffu, t.x, o);
      const int b = __shfl_up_sync(0xffffffffu, t.y, o);
      if (lane >= o) { t.x += a; t.y += b; }
    }
    ws[lane] = t;
  }
  __syncthreads();
  const int2 pre = wid > 0 ? ws[wid - 1] : make_int2(0, 0);
  *tot = ws[(blockDim.x >> 5) - 1];
  __syncthreads();
  return make_int2(pre.x + inc.x - x.x, pre.y + inc.y - x.y);
}

// L = the instances j < n with pred(j), in index order, with prefix sums of nbf(j).
template <class Pred, class NB>
__device__ void build_list(const BatchList& L, int n, Pred pred, NB nbf) {
  int2 base = make_int2(0, 0);
  for (int c0 = 0; c0 < n; c0 += blockDim.x) {
    const int j = c0 + threadIdx.x;
    const bool on = j < n && pred(j);
    const int2 x = make_int2(on ? 1 : 0, on ? nbf(j) : 0);
    int2 tot;
    const int2 ex = scan_pairs(x, &tot);
    if (on) {
      L.inst[base.x + ex.x] = j;
      L.first[base.x + ex.x] = base.y + ex.y;
    }
    base.x += tot.x;
    base.y += tot.y;
  }
  if (threadIdx.x == 0) {
    L.first[base.x] = base.y;
    *L.count = base.x;
  }
}

__device__ void build_sweep_lists(const BatchDev& B) {
  build_list(
      B.sw, B.n,
      [&](int j) {
        const BatchInst& I = B.insts[j];
        return I.phase == BP_SWEEP0 || I.phase == BP_SWEEPV;
      },
      [&](int j) { return B.insts[j].nb_sw; });
}

__device__ void build_inner_lists(const BatchDev& B) {
  build_list(B.mv, B.n, [&](int j) { return B.insts[j].phase == BP_INNER; },
             [&](int j) { return B.insts[j].nb_mv; });
  build_list(B.ts, B.n, [&](int j) { return B.insts[j].phase == BP_INNER; },
             [&](int j) { return B.insts[j].nb_ts; });
  build_list(B.ew, B.n, [&](int j) { return B.insts[j].phase == BP_INNER; },
             [&](int j) { return B.insts[j].nb_ew; });
}

// ------------------------------------------------------------------ control kernels
__global__ void __launch_bounds__(CTRL_THREADS) batch_init_kernel(BatchDev B) {
  for (int j = threadIdx.x; j < B.n; j += blockDim.x) {
    BatchInst& I = B.insts[j];
    I.phase = BP_SWEEP0;
    I.cur = 0;
    I.k = 0;
    I.reps = 0;
    I.status = MDP_ENOCONV;
    I.starting = 0;
    I.rhs_sel = 0;
    I.inner = I.restarts = I.checks = I.sweeps = I.loops = I.breakdowns = 0;
    I.thr = 0.0;
    I.res = 0.0;
    I.ctl->mode = GM_IDLE;
  }
  __syncthreads();
  build_sweep_lists(B);
  if (threadIdx.x == 0) {
    *B.mv.count = 0;
    *B.ts.count = 0;
    *B.ew.count = 0;
    B.ctr[0] = B.n;
    B.ctr[1] = 0;
    B.ctr[2] = 0;
  }
}

__device__ void start_inner(const BatchDev& B, BatchInst& I, int variant) {
  I.phase = BP_INNER;
  I.starting = 1;
  I.rhs_sel = variant;
  // variant 0: J delta = Phi_k (norms sout[0]), threshold alpha ||Phi_k||_inf;
  // variant 1: resumed on the exact residual (norms sout[2]) with the same threshold
  gmres_init_ctl(I.ctl, 0.0, B.alpha, I.sqrtS, B.W, B.max_steps, I.sout + (variant ? 2 : 0),
                 variant, 1, B.forcing_c, B.thr_floor);
}

// The decisions of the outer loop of Alg. 2 after a sweep, one thread per instance.
__global__ void __launch_bounds__(CTRL_THREADS) batch_ctrl_kernel(BatchDev B) {
  for (int j = threadIdx.x; j < B.n; j += blockDim.x) {
    BatchInst& I = B.insts[j];
    I.starting = 0;
    const int ph = I.phase;
    if (ph != BP_SWEEP0 && ph != BP_SWEEPV) continue;
    I.sweeps += 1;
    if (ph == BP_SWEEPV) {
      const GmresCtl* c = I.ctl;
      I.inner += c->steps;
      I.restarts += c->restarts;
      I.checks += c->checks;
      I.loops += 1;
      if (c->status == GS_BREAKDOWN) I.breakdowns += 1;
      if (c->mode != GM_DONE) {  // cannot happen: SWEEPV follows a finished solve
        I.status = MDP_ETIMEOUT;
        I.phase = BP_DONE;
        continue;
      }
      // exact stopping test of Alg. 2 on the residual of pi_k at V_{k+1} (breakdown or the
      // step cap also end the inner solve; at most 8 resumptions)
      const double sref = I.sout[2].res_inf;
      const bool ok = !(sref > I.thr) || c->status == GS_BREAKDOWN || c->status == GS_CAP ||
                      I.reps >= 8;
      if (!ok) {
        I.reps += 1;
        I.restarts += 1;
        start_inner(B, I, 1);
        continue;
      }
      I.cur = 1 - I.cur;  // pi_{k+1} = GreedyPolicy(V_{k+1})
    }
    const double res = I.sout[0].res_inf;
    I.res = res;
    if (res <= B.tol) {
      I.status = MDP_OK;
      I.phase = BP_DONE;
    } else if (I.k >= B.max_outer) {
      I.status = MDP_ENOCONV;
      I.phase = BP_DONE;
    } else {
      I.thr = inexact_threshold(B.alpha, B.forcing_c, res, B.thr_floor);
      I.k += 1;
      I.reps = 0;
      start_inner(B, I, 0);
    }
  }
  __syncthreads();
  build_inner_lists(B);
}

// Rows [r0, r1) of an instance's virtual block in the element-wise kernels.
__device__ __forceinline__ void ew_rows(int64_t S, GridPos gp, int64_t& r0, int64_t& r1) {
  const int64_t per = (S + gp.nb - 1) / gp.nb;
  r0 = (int64_t)gp.bid * per;
  r1 = min(S, r0 + per);
}

// Start of an inner solve: the start residual goes to rbuf, the correction base to zero.
__global__ void __launch_bounds__(EW_THREADS) batch_prologue_kernel(BatchDev B) {
  batch_for_each(B.ew, [&](int j, GridPos gp) {
    const BatchInst& I = B.insts[j];
    if (!I.starting) return;
    const float* rhs = I.rhs_sel ? I.rref : I.phi;
    int64_t r0, r1;
    ew_rows(I.d.S, gp, r0, r1);
    for (int64_t s = r0 + threadIdx.x; s < r1; s += blockDim.x) {
      I.rbuf[s] = rhs[s];
      I.d0[s] = 0.f;
    }
  });
}

// V_{k+1} = V_k + delta once the inner solve is done (double-float sum).
__global__ void __launch_bounds__(EW_THREADS) batch_value_update_kernel(BatchDev B) {
  batch_for_each(B.ew, [&](int j, GridPos gp) {
    const BatchInst& I = B.insts[j];
    const GmresCtl* c = I.ctl;
    if (c->mode != GM_DONE) return;
    const float* dl = c->dsel ? I.d1 : I.d0;
    int64_t r0, r1;
    ew_rows(I.d.S, gp, r0, r1);
    for (int64_t s = r0 + threadIdx.x; s < r1; s += blockDim.x) {
      const float2 x = I.v[s];
      const dfl r = df_add({x.x, x.y}, {dl[s], 0.f});
      I.v[s] = make_float2(r.hi, r.lo);
    }
  });
}

// Loop condition: finished inner solves move to their verifying sweep; the WHILE node runs
// again while some instance is not done (and the iteration guard allows).
__global__ void __launch_bounds__(CTRL_THREADS) batch_loop_kernel(BatchDev B,
                                                                  cudaGraphConditionalHandle hc,
                                                                  int with_cond) {
  __shared__ int active;
  if (threadIdx.x == 0) active = 0;
  __syncthreads();
  int a = 0;
  for (int j = threadIdx.x; j < B.n; j += blockDim.x) {
    BatchInst& I = B.insts[j];
    if (I.phase == BP_INNER && I.ctl->mode == GM_DONE) I.phase = BP_SWEEPV;
    if (I.phase != BP_DONE && I.phase != BP_FREE) a += 1;
  }
  if (a) atomicAdd(&active, a);
  __syncthreads();
  build_sweep_lists(B);
  if (threadIdx.x == 0) {
    const int it = ++B.ctr[1];
    B.ctr[0] = active;
    const bool more = active > 0 && it < B.max_iters;
    if (active > 0 && !more) B.ctr[2] = 1;
    B.ctr[3] = more ? 1 : 0;
    if (with_cond) cudaGraphSetConditional(hc, more ? 1u : 0u);
  }
}

__global__ void __launch_bounds__(CTRL_THREADS) batch_relist_kernel(BatchDev B) {
  if (threadIdx.x == 0) B.ctr[1] = 0;
  build_sweep_lists(B);
}

__global__ void batch_output_one_kernel(const BatchInst* rec, int64_t S, double* vo, int32_t* po) {
  const float2* tv = rec->tv;
  const int32_t* pi = rec->pib[rec->cur];
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x) {
    const float2 x = tv[s];
    vo[s] = (double)x.x + (double)x.y;
    po[s] = pi[s];
  }
}

// One Bellman sweep of every instance at its current V (mdp_batch_bellman): every instance
// gets phase SWEEP0 (its policy buffer pib[cur] receives GreedyPolicy(V)).
__global__ void __launch_bounds__(CTRL_THREADS) batch_sweep_all_kernel(BatchDev B) {
  for (int j = threadIdx.x; j < B.n; j += blockDim.x) B.insts[j].phase = BP_SWEEP0;
  __syncthreads();
  build_sweep_lists(B);
}

__global__ void __launch_bounds__(EW_THREADS) batch_zero_v_kernel(BatchDev B) {
  batch_for_each(B.all, [&](int j, GridPos gp) {
    const BatchInst& I = B.insts[j];
    int64_t r0, r1;
    ew_rows(I.d.S, gp, r0, r1);
    for (int64_t s = r0 + threadIdx.x; s < r1; s += blockDim.x) I.v[s] = make_float2(0.f, 0.f);
  });
}

// Results: v = T(V_K) as double, pi = pi_K.
__global__ void __launch_bounds__(EW_THREADS) batch_output_kernel(BatchDev B) {
  batch_for_each(B.all, [&](int j, GridPos gp) {
    const BatchInst& I = B.insts[j];
    double* vo = B.vout[j];
    int32_t* po = B.pout[j];
    const int32_t* pi = I.pib[I.cur];
    int64_t r0, r1;
    ew_rows(I.d.S, gp, r0, r1);
    for (int64_t s = r0 + threadIdx.x; s < r1; s += blockDim.x) {
      const float2 x = I.tv[s];
      vo[s] = (double)x.x + (double)x.y;
      po[s] = pi[s];
    }
  });
}

inline size_t align256(size_t x) { return (x + 255) / 256 * 256; }
inline int ilog2(int x) { int r = 0; while ((1 << r) < x) ++r; return r; }

}  // namespace

// ------------------------------------------------------------------ host side
struct mdp_batch_s {
  int n = 0;
  std::vector<mdp_t> hs;
  mdp_opts o{};
  int device = 0;
  cudaStream_t stream = nullptr;
  cudaStream_t own = nullptr;
  cudaStream_t cap = nullptr;
  char* pool = nullptr;       // workspaces of every instance
  size_t pool_bytes = 0;
  char* outpool = nullptr;    // device results for host-pointer solves
  size_t out_bytes = 0;
  char* h_out = nullptr;      // pinned staging of outpool
  std::vector<size_t> vo_off, po_off;
  BatchInst* d_insts = nullptr;
  BatchInst* h_insts = nullptr;  // pinned: static table / readback
  std::vector<BatchInst> table;  // static table as built at creation (or by the tuner)
  int* d_lists = nullptr;
  int* d_ctr = nullptr;
  int* h_ctr = nullptr;          // pinned
  void** d_outp = nullptr;       // [2n] device pointer table (vout, pout)
  void** h_outp = nullptr;       // pinned staging
  BatchDev B{};
  int grid_sw = 0, grid_mv = 0;
  int grid_ts = 0, grid_ew = 0, grid_all = 0;
  int launches_per_iter = 0;
  cudaGraphExec_t exec = nullptr;
};

namespace {

#define BCK(x)                                                                        \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess)                                                            \
      return set_error(MDP_EDEVICE, (std::string(#x) + ": " + cudaGetErrorString(e_)).c_str()); \
  } while (0)
#define BRK(x)                                                                        \
  do {                                                                                \
    int r_ = (x);                                                                     \
    if (r_ != MDP_OK) return r_ == MDP_EDEVICE ? set_error(r_, #x) : r_;              \
  } while (0)

void free_batch(mdp_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  void* dp[] = {b->pool, b->outpool, b->d_insts, b->d_lists, b->d_ctr, b->d_outp};
  for (void* p : dp)
    if (p) cudaFree(p);
  void* hp[] = {b->h_out, b->h_insts, b->h_ctr, b->h_outp};
  for (void* p : hp)
    if (p) cudaFreeHost(p);
  if (b->cap) cudaStreamDestroy(b->cap);
  if (b->own) cudaStreamDestroy(b->own);
}

// Physical grids: the occupancy limit of each batched kernel, capped by the most virtual
// blocks the family can have in one launch.
void set_grids(mdp_batch_s* b) {
  int64_t tsw = 0, tmv = 0, tts = 0, tew = 0;
  for (const BatchInst& I : b->table) {
    tsw += I.nb_sw;
    tmv += I.nb_mv;
    tts += I.nb_ts;
    tew += I.nb_ew;
  }
  // sweep, ctrl, prologue, two matvecs, three CGS2 kernels, estimate, value update, loop
  b->launches_per_iter = 11;
  b->grid_sw = (int)std::max<int64_t>(1, std::min<int64_t>(batch_sweep_grid(), tsw));
  b->grid_mv = (int)std::max<int64_t>(1, std::min<int64_t>(batch_matvec_grid(), tmv));
  b->grid_ts = (int)std::max<int64_t>(1, std::min<int64_t>(batch_ts_grid(b->o.restart + 1), tts));
  b->grid_ew = (int)std::max<int64_t>(1, std::min<int64_t>((int64_t)num_sms() * 8, tew));
  b->grid_all = b->grid_ew;
}

int upload_table(mdp_batch_s* b) {
  std::memcpy(b->h_insts, b->table.data(), sizeof(BatchInst) * b->n);
  BCK(cudaMemcpyAsync(b->d_insts, b->h_insts, sizeof(BatchInst) * b->n, cudaMemcpyHostToDevice,
                      b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  return MDP_OK;
}

// The static list of all instances (element-wise families) is built on the host.
int upload_all_list(mdp_batch_s* b) {
  std::vector<int> inst(b->n), first(b->n + 1);
  int acc = 0;
  for (int j = 0; j < b->n; ++j) {
    inst[j] = j;
    first[j] = acc;
    acc += b->table[j].nb_ew;
  }
  first[b->n] = acc;
  const int cnt = b->n;
  BCK(cudaMemcpy(b->B.all.inst, inst.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->B.all.first, first.data(), sizeof(int) * (b->n + 1), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(b->B.all.count, &cnt, sizeof(int), cudaMemcpyHostToDevice));
  return MDP_OK;
}

// Kernels of the batch: the prologue (state reset, V_0 = 0), one loop iteration, and the
// output conversion.  Every launch goes to stream st (a capturing stream when building the
// graph).
int enqueue_init(mdp_batch_s* b, cudaStream_t st) {
  batch_init_kernel<<<1, CTRL_THREADS, 0, st>>>(b->B);
  batch_zero_v_kernel<<<b->grid_all, EW_THREADS, 0, st>>>(b->B);
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}

int enqueue_iteration(mdp_batch_s* b, cudaStream_t st, cudaGraphConditionalHandle hc, int with_cond) {
  const BatchGrids g{b->grid_sw, b->grid_mv, b->grid_ts, b->grid_ew};
  return batch_enqueue_iteration(b->B, g, b->o.restart + 1, st, hc, with_cond);
}

int enqueue_output(mdp_batch_s* b, cudaStream_t st) {
  batch_output_kernel<<<b->grid_all, EW_THREADS, 0, st>>>(b->B);
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}

// The whole solve as one graph: prologue, WHILE node over one loop iteration, outputs.
int build_graph(mdp_batch_s* b) {
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  if (!b->cap) BCK(cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  BCK(cudaGraphCreate(&g, 0));
  auto abort_capture = [&](const char* what) {
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(b->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(b->cap, &junk);
    }
    const std::string msg = std::string("batch graph: ") + what + ": " +
                            cudaGetErrorString(cudaGetLastError());
    cudaGraphDestroy(g);
    return set_error(MDP_EDEVICE, msg.c_str());
  };
  if (cudaStreamBeginCaptureToGraph(b->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return abort_capture("capture start");
  if (enqueue_init(b, b->cap) != MDP_OK) return abort_capture("init launches");
  cudaStreamCaptureStatus cst;
  cudaGraph_t capg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(b->cap, &cst, nullptr, &capg, &deps, nullptr, &nd) != cudaSuccess)
    return abort_capture("capture info");
  cudaGraphConditionalHandle hc;
  if (cudaGraphConditionalHandleCreate(&hc, capg, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return abort_capture("conditional handle");
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hc;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t cn;
  if (cudaGraphAddNode(&cn, capg, deps, nullptr, nd, &np) != cudaSuccess)
    return abort_capture("conditional node");
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(b->cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return abort_capture("capture dependencies");
  if (enqueue_output(b, b->cap) != MDP_OK) return abort_capture("output launch");
  cudaGraph_t g2 = nullptr;
  if (cudaStreamEndCapture(b->cap, &g2) != cudaSuccess) return abort_capture("end capture");
  // loop body: one iteration of every instance's state machine
  if (cudaStreamBeginCaptureToGraph(b->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return abort_capture("body capture start");
  if (enqueue_iteration(b, b->cap, hc, 1) != MDP_OK) return abort_capture("body launches");
  cudaGraph_t b2 = nullptr;
  if (cudaStreamEndCapture(b->cap, &b2) != cudaSuccess) return abort_capture("end body capture");
  if (cudaGraphInstantiate(&b->exec, g, 0) != cudaSuccess) {
    b->exec = nullptr;
    return abort_capture("instantiate");
  }
  cudaGraphDestroy(g);
  return MDP_OK;
}

// The same kernels enqueued from the host, one loop iteration at a time (the host reads
// the loop condition after each), for tools that cannot follow conditional graph nodes.
int run_host_loop(mdp_batch_s* b) {
  BRK(enqueue_init(b, b->stream));
  for (int it = 0; it < b->B.max_iters; ++it) {
    BRK(enqueue_iteration(b, b->stream, 0, 0));
    BCK(cudaMemcpyAsync(b->h_ctr, b->d_ctr, 4 * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    if (!b->h_ctr[3]) break;
  }
  return enqueue_output(b, b->stream);
}

int check_batch_opts(const mdp_opts& o) {
  if (o.restart < 1 || o.restart > WMAX) return set_error(MDP_EINVAL, "restart must be in 1..64");
  if (!(o.alpha > 0.0 && o.alpha < 1.0)) return set_error(MDP_EINVAL, "alpha must be in (0, 1)");
  if (!(o.tol >= 0.0)) return set_error(MDP_EINVAL, "tol must be >= 0");
  if (!(o.forcing_c >= 0.0 && o.forcing_c < INFINITY)) return set_error(MDP_EINVAL, "forcing_c must be finite and >= 0");
  if (o.precond_block != 0) return set_error(MDP_EINVAL, "precond_block applies to ipi_solve only");
  if (o.max_outer < 0 || o.max_inner < 1) return set_error(MDP_EINVAL, "bad iteration caps");
  if (o.precision != MDP_PREC_MIXED) return set_error(MDP_EINVAL, "a batch runs in MDP_PREC_MIXED");
  if (o.v0) return set_error(MDP_EINVAL, "a batch starts from V_0 = 0 (v0 must be NULL)");
  return MDP_OK;
}

int create_batch(const mdp_t* hs, int32_t n, const mdp_opts* opts, mdp_batch_s* b) {
  if (!hs || n < 1) return set_error(MDP_EINVAL, "need n >= 1 handles");
  b->o = opts ? *opts : mdp_opts_default();
  BRK(check_batch_opts(b->o));
  BCK(cudaGetDevice(&b->device));
  b->n = n;
  b->hs.assign(hs, hs + n);
  for (int j = 0; j < n; ++j) {
    const DevMDP* d = handle_view(hs[j]);
    if (!d) return set_error(MDP_EINVAL, "null handle in batch");
    BRK(handle_finish_pending(hs[j]));
    if (d->kind != KIND_ELL || d->pdt != MDP_F32)
      return set_error(MDP_EINVAL, "a batch takes ELL handles with FP32 transition data");
    if (handle_device(hs[j]) != b->device)
      return set_error(MDP_EINVAL, "every handle of a batch must live on the current device");
  }
  BCK(cudaStreamCreateWithFlags(&b->own, cudaStreamNonBlocking));
  b->stream = b->own;
  const int W = b->o.restart;
  // workspaces, instance by instance, in one allocation
  b->table.assign(n, BatchInst{});
  std::vector<size_t> off(n);
  size_t tot = 0, otot = 0;
  b->vo_off.resize(n);
  b->po_off.resize(n);
  for (int j = 0; j < n; ++j) {
    const DevMDP& d = *handle_view(hs[j]);
    off[j] = tot;
    tot += batch_workspace_bytes(d, W);
    b->vo_off[j] = otot;
    otot += align256((size_t)d.S * 8);
    b->po_off[j] = otot;
    otot += align256((size_t)d.S * 4);
  }
  if (cudaMalloc(&b->pool, tot) != cudaSuccess) {
    cudaGetLastError();
    return set_error(MDP_ENOMEM, ("batch workspace of " + std::to_string(tot) + " bytes").c_str());
  }
  b->pool_bytes = tot;
  BCK(cudaMemset(b->pool, 0, tot));
  if (cudaMalloc(&b->outpool, otot) != cudaSuccess) {
    cudaGetLastError();
    return set_error(MDP_ENOMEM, "batch output buffers");
  }
  b->out_bytes = otot;
  for (int j = 0; j < n; ++j) {
    batch_setup_inst(*handle_view(hs[j]), W, b->pool + off[j], b->table[j]);
    b->table[j].phase = BP_DONE;
  }
  // device tables
  BCK(cudaMalloc((void**)&b->d_insts, sizeof(BatchInst) * n));
  BCK(cudaMallocHost((void**)&b->h_insts, sizeof(BatchInst) * n));
  const int nlists = 5;
  const size_t per_list = (size_t)2 * n + 2;
  BCK(cudaMalloc((void**)&b->d_lists, sizeof(int) * per_list * nlists));
  BCK(cudaMemset(b->d_lists, 0, sizeof(int) * per_list * nlists));
  BCK(cudaMalloc((void**)&b->d_ctr, 64));
  BCK(cudaMemset(b->d_ctr, 0, 64));
  BCK(cudaMallocHost((void**)&b->h_ctr, 64));
  BCK(cudaMalloc((void**)&b->d_outp, sizeof(void*) * 2 * n));
  BCK(cudaMallocHost((void**)&b->h_outp, sizeof(void*) * 2 * n));
  auto list_at = [&](int li) {
    int* base = b->d_lists + per_list * li;
    return BatchList{base, base + n, base + 2 * n + 1};
  };
  BatchDev& B = b->B;
  B.insts = b->d_insts;
  B.n = n;
  B.alpha = b->o.alpha;
  B.tol = b->o.tol;
  B.forcing_c = b->o.forcing_c;
  B.thr_floor = 0.1 * b->o.tol;
  B.W = W;
  B.max_steps = b->o.max_inner;
  B.max_outer = b->o.max_outer;
  B.sw = list_at(0);
  B.mv = list_at(1);
  B.ts = list_at(2);
  B.ew = list_at(3);
  B.all = list_at(4);
  B.vout = (double**)b->d_outp;
  B.pout = (int32_t**)(b->d_outp + n);
  B.ctr = b->d_ctr;
  // guard on loop iterations: every instance's own caps end it far earlier
  const double guard = (double)(b->o.max_outer + 2) * 9.0 * (double)(b->o.max_inner + 2);
  B.max_iters = (int)std::min(guard, 1.0e9);
  BRK(upload_table(b));
  BRK(upload_all_list(b));
  set_grids(b);
  return MDP_OK;
}

int run_batch(mdp_batch_s* b, double* const* v_out, int32_t* const* pi_out, mdp_stats* st,
              bool device_out) {
  if (!b) return set_error(MDP_EINVAL, "null batch");
  if (!v_out || !pi_out) return set_error(MDP_EINVAL, "null output arrays");
  const int n = b->n;
  for (int j = 0; j < n; ++j) {
    if (!v_out[j] || !pi_out[j]) return set_error(MDP_EINVAL, "null output pointer");
    b->h_outp[j] = device_out ? (void*)v_out[j] : (void*)(b->outpool + b->vo_off[j]);
    b->h_outp[n + j] = device_out ? (void*)pi_out[j] : (void*)(b->outpool + b->po_off[j]);
  }
  // loads enqueued with mdp_load_*_async on the batch's handles must have landed (and passed
  // validation) before the batch reads their data
  for (mdp_t h : b->hs) BRK(handle_finish_pending(h));
  const bool host_loop = (b->o.flags & MDP_FLAG_HOST_LOOP) != 0;
  if (!host_loop && !b->exec) BRK(build_graph(b));
  BCK(cudaMemcpyAsync(b->d_outp, b->h_outp, sizeof(void*) * 2 * n, cudaMemcpyHostToDevice, b->stream));
  if (host_loop) BRK(run_host_loop(b));
  else BCK(cudaGraphLaunch(b->exec, b->stream));
  BCK(cudaMemcpyAsync(b->h_ctr, b->d_ctr, 3 * sizeof(int), cudaMemcpyDeviceToHost, b->stream));
  BCK(cudaMemcpyAsync(b->h_insts, b->d_insts, sizeof(BatchInst) * n, cudaMemcpyDeviceToHost, b->stream));
  if (!device_out) {
    if (!b->h_out) BCK(cudaMallocHost((void**)&b->h_out, b->out_bytes));
    BCK(cudaMemcpyAsync(b->h_out, b->outpool, b->out_bytes, cudaMemcpyDeviceToHost, b->stream));
  }
  BCK(cudaStreamSynchronize(b->stream));
  if (!device_out)
    for (int j = 0; j < n; ++j) {
      const int64_t S = b->table[j].d.S;
      std::memcpy(v_out[j], b->h_out + b->vo_off[j], (size_t)S * 8);
      std::memcpy(pi_out[j], b->h_out + b->po_off[j], (size_t)S * 4);
    }
  const int iters = b->h_ctr[1];
  int status = MDP_OK;
  for (int j = 0; j < n; ++j) {
    const BatchInst& I = b->h_insts[j];
    mdp_stats s{};
    s.outer = I.k;
    s.inner = I.inner;
    s.restarts = I.restarts;
    s.sweeps = I.sweeps;
    s.matvecs = I.inner + I.checks;
    s.breakdowns = I.breakdowns;
    s.status = I.phase == BP_DONE ? I.status : MDP_ETIMEOUT;
    s.residual_inf = I.res;
    s.launches = 3 + iters * b->launches_per_iter;
    if (st) st[j] = s;
    if (s.status == MDP_ETIMEOUT) status = MDP_ETIMEOUT;
    else if (s.status != MDP_OK && status == MDP_OK) status = s.status;
  }
  if (b->h_ctr[2]) return set_error(MDP_ETIMEOUT, "batch loop guard ended the launch");
  if (status == MDP_ENOCONV) set_error(MDP_ENOCONV, "some instances reached max_outer");
  return status;
}

// Time fn() on the batch stream: one warm-up, best of three.
template <class F>
float time_best(mdp_batch_s* b, F fn) {
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {
    cudaEventRecord(e0, b->stream);
    fn();
    cudaEventRecord(e1, b->stream);
    cudaEventSynchronize(e1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep > 0) best = std::min(best, ms);
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}

// Host-built list of the given instances into list L.
int upload_list(mdp_batch_s* b, const BatchList& L, const std::vector<int>& ids, bool sweep) {
  std::vector<int> first(ids.size() + 1);
  int acc = 0;
  for (size_t i = 0; i < ids.size(); ++i) {
    first[i] = acc;
    acc += sweep ? b->table[ids[i]].nb_sw : b->table[ids[i]].nb_mv;
  }
  first[ids.size()] = acc;
  const int cnt = (int)ids.size();
  BCK(cudaMemcpy(L.inst, ids.data(), sizeof(int) * ids.size(), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(L.first, first.data(), sizeof(int) * first.size(), cudaMemcpyHostToDevice));
  BCK(cudaMemcpy(L.count, &cnt, sizeof(int), cudaMemcpyHostToDevice));
  return MDP_OK;
}

}  // namespace
namespace mdp {
static size_t partial_bytes(const BatchInst& I);
static void batch_geometry(const DevMDP& d, BatchInst& I);
}  // namespace mdp
namespace {

int tune_batch(mdp_batch_s* b) {
  // group instances by padded ELL row length
  std::vector<int> kps;
  for (const BatchInst& I : b->table)
    if (std::find(kps.begin(), kps.end(), I.d.kp) == kps.end()) kps.push_back(I.d.kp);
  std::vector<BatchInst> saved = b->table;
  for (BatchInst& I : b->table) {  // tuning launches run ungated: a valid phase and policy
    I.phase = BP_SWEEP0;
    I.cur = 0;
  }
  for (int kp : kps) {
    std::vector<int> ids;
    for (int j = 0; j < b->n; ++j)
      if (b->table[j].d.kp == kp) ids.push_back(j);
    for (int fam = 0; fam < 2; ++fam) {
      float best = 1e30f;
      int best_c = 0;
      const BatchList& L = fam == 0 ? b->B.sw : b->B.mv;
      BRK(upload_list(b, L, ids, fam == 0));
      int64_t tot = 0;
      for (int j : ids) tot += fam == 0 ? b->table[j].nb_sw : b->table[j].nb_mv;
      const int grid = (int)std::min<int64_t>(fam == 0 ? batch_sweep_grid() : batch_matvec_grid(), tot);
      for (int c = 0; c < BATCH_CLASSES; ++c) {
        for (int j : ids) (fam == 0 ? b->table[j].cls_sw : b->table[j].cls_mv) = c;
        BRK(upload_table(b));
        int r = MDP_OK;
        const float ms = time_best(b, [&]() {
          if (r != MDP_OK) return;
          r = fam == 0 ? launch_batch_sweep(b->B, grid, b->stream)
                       : launch_batch_matvec(b->B, 2, grid, b->stream);
        });
        BRK(r);
        BCK(cudaGetLastError());
        if (ms < best) {
          best = ms;
          best_c = c;
        }
      }
      for (int j : ids) (fam == 0 ? saved[j].cls_sw : saved[j].cls_mv) = best_c;
      for (int j : ids) (fam == 0 ? b->table[j].cls_sw : b->table[j].cls_mv) = best_c;
      // row tiles of the chosen lane class: the library's states per virtual block scaled by
      // 1, 1/2, 2 and 4 (block counts scaled inversely); a candidate whose matvec partial sums
      // would not fit the instance's workspace is skipped
      std::vector<int> base(ids.size());
      for (size_t i = 0; i < ids.size(); ++i)
        base[i] = fam == 0 ? b->table[ids[i]].nb_sw : b->table[ids[i]].nb_mv;
      const double scales[4] = {1.0, 0.5, 2.0, 4.0};
      float best_t = 1e30f;
      int best_s = 0;
      for (int si = 0; si < 4; ++si) {
        bool fits = true;
        int64_t tot_s = 0;
        for (size_t i = 0; i < ids.size(); ++i) {
          BatchInst& I = b->table[ids[i]];
          const int nb = (int)std::max<int64_t>(
              1, std::min<int64_t>(MAX_RED_BLOCKS, (int64_t)std::ceil(base[i] / scales[si])));
          if (fam == 0) {
            I.nb_sw = nb;
          } else {
            BatchInst t = I, t0 = I;  // t0: the create-time geometry the workspace was sized for
            batch_geometry(t0.d, t0);
            t.nb_mv = nb;
            if (partial_bytes(t) > partial_bytes(t0)) fits = false;
            I.nb_mv = nb;
          }
          tot_s += nb;
        }
        if (!fits) continue;
        BRK(upload_table(b));
        BRK(upload_list(b, L, ids, fam == 0));
        const int g2 = (int)std::min<int64_t>(fam == 0 ? batch_sweep_grid() : batch_matvec_grid(), tot_s);
        int r = MDP_OK;
        const float ms = time_best(b, [&]() {
          if (r != MDP_OK) return;
          r = fam == 0 ? launch_batch_sweep(b->B, g2, b->stream)
                       : launch_batch_matvec(b->B, 2, g2, b->stream);
        });
        BRK(r);
        BCK(cudaGetLastError());
        if (ms < best_t) {
          best_t = ms;
          best_s = si;
        }
      }
      for (size_t i = 0; i < ids.size(); ++i) {
        const int nb = (int)std::max<int64_t>(
            1, std::min<int64_t>(MAX_RED_BLOCKS, (int64_t)std::ceil(base[i] / scales[best_s])));
        BatchInst& I = b->table[ids[i]];
        BatchInst& Sv = saved[ids[i]];
        if (fam == 0) I.nb_sw = Sv.nb_sw = nb;
        else I.nb_mv = Sv.nb_mv = nb;
      }
      const int empty = 0;
      BCK(cudaMemcpy(L.count, &empty, sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  b->table = saved;
  BRK(upload_table(b));
  set_grids(b);
  if (b->exec) {
    cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
  }
  return MDP_OK;
}

}  // namespace

extern "C" {

int mdp_batch_create(const mdp_t* hs, int32_t n, const mdp_opts* opts, mdp_batch_t* out) {
  if (!out) return set_error(MDP_EINVAL, "null output handle");
  *out = nullptr;
  mdp_batch_s* b = new mdp_batch_s();
  const int r = create_batch(hs, n, opts, b);
  if (r != MDP_OK) {
    free_batch(b);
    delete b;
    return r;
  }
  *out = b;
  return MDP_OK;
}

void mdp_batch_destroy(mdp_batch_t b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  free_batch(b);
  delete b;
}

int mdp_batch_set_stream(mdp_batch_t b, void* stream) {
  if (!b) return set_error(MDP_EINVAL, "null batch");
  b->stream = stream ? (cudaStream_t)stream : b->own;
  return MDP_OK;
}

int mdp_batch_tune(mdp_batch_t b) {
  if (!b) return set_error(MDP_EINVAL, "null batch");
  return tune_batch(b);
}

int mdp_batch_geometry(mdp_batch_t b, int32_t i, int32_t* lanes_sweep, int32_t* lanes_matvec,
                       int32_t* sweep_blocks, int32_t* matvec_blocks, int32_t* krylov_blocks_out) {
  if (!b || i < 0 || i >= b->n) return set_error(MDP_EINVAL, "bad batch or instance index");
  const BatchInst& I = b->table[i];
  if (lanes_sweep) *lanes_sweep = 1 << I.cls_sw;
  if (lanes_matvec) *lanes_matvec = 1 << I.cls_mv;
  if (sweep_blocks) *sweep_blocks = I.nb_sw;
  if (matvec_blocks) *matvec_blocks = I.nb_mv;
  if (krylov_blocks_out) *krylov_blocks_out = I.nb_ts;
  return MDP_OK;
}

int64_t mdp_batch_device_bytes(mdp_batch_t b) {
  if (!b) return 0;
  return (int64_t)(b->pool_bytes + b->out_bytes);
}

int mdp_batch_bellman(mdp_batch_t b, double* res_inf) {
  if (!b) return set_error(MDP_EINVAL, "null batch");
  batch_sweep_all_kernel<<<1, CTRL_THREADS, 0, b->stream>>>(b->B);
  BCK(cudaGetLastError());
  BRK(launch_batch_sweep(b->B, b->grid_sw, b->stream));
  if (!res_inf) return MDP_OK;
  BCK(cudaMemcpyAsync(b->h_insts, b->d_insts, sizeof(BatchInst) * b->n, cudaMemcpyDeviceToHost,
                      b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  std::vector<SweepOut> so(b->n);
  for (int j = 0; j < b->n; ++j)
    BCK(cudaMemcpyAsync(&so[j], b->h_insts[j].sout, sizeof(SweepOut), cudaMemcpyDeviceToHost,
                        b->stream));
  BCK(cudaStreamSynchronize(b->stream));
  for (int j = 0; j < b->n; ++j) res_inf[j] = so[j].res_inf;
  return MDP_OK;
}

int mdp_batch_solve(mdp_batch_t b, double* const* v_out, int32_t* const* pi_out, mdp_stats* stats) {
  return run_batch(b, v_out, pi_out, stats, false);
}

int mdp_batch_solve_dev(mdp_batch_t b, double* const* v_out, int32_t* const* pi_out,
                        mdp_stats* stats) {
  return run_batch(b, v_out, pi_out, stats, true);
}

int ipi_solve_batch(const mdp_t* hs, int32_t n, const mdp_opts* opts, double* const* v_out,
                    int32_t* const* pi_out, mdp_stats* stats) {
  mdp_batch_t b = nullptr;
  int r = mdp_batch_create(hs, n, opts, &b);
  if (r != MDP_OK) return r;
  r = run_batch(b, v_out, pi_out, stats, false);
  mdp_batch_destroy(b);
  return r;
}

}  // extern "C"

// ------------------------------------------------------------------ shared with the server
namespace mdp {

// Virtual blocks per kernel family: a sweep block streams about 512 KB of P, a matvec block
// about 256 KB, a Krylov block 4096 rows, an element-wise block 8192 rows.  Each virtual
// block ends with a block-wide reduction, so larger blocks amortise it; the batch supplies
// the parallelism that small instances lack.
static void batch_geometry(const DevMDP& d, BatchInst& I) {
  const int64_t S = d.S;
  const int64_t row_b = (int64_t)d.kp * 8;
  auto clampb = [](int64_t x) { return (int)std::max<int64_t>(1, std::min<int64_t>(x, MAX_RED_BLOCKS)); };
  const int64_t st_sw = std::max<int64_t>(8, 524288 / std::max<int64_t>(1, row_b * d.A));
  const int64_t st_mv = std::max<int64_t>(32, 262144 / std::max<int64_t>(1, row_b));
  I.nb_sw = clampb((S + st_sw - 1) / st_sw);
  I.nb_mv = clampb((S + st_mv - 1) / st_mv);
  I.nb_ts = clampb((S + 4095) / 4096);
  I.nb_ew = clampb((S + 8191) / 8192);
}

static size_t partial_bytes(const BatchInst& I) {
  return std::max<size_t>((size_t)MAX_RED_BLOCKS * 32,
                          (size_t)I.nb_ts * (WMAX + 1) * 4 + 2 * (size_t)I.nb_mv * 4);
}

size_t batch_workspace_bytes(const DevMDP& d, int W) {
  BatchInst I{};
  I.d = d;
  I.ldq = (d.S + 31) / 32 * 32;
  batch_geometry(d, I);
  const size_t f = align256((size_t)I.ldq * 4), f2 = align256((size_t)I.ldq * 8);
  return 2 * f2 + 7 * f + align256((size_t)(W + 1) * I.ldq * 4) + 2 * f +
         align256(sizeof(GmresCtl)) + align256(4 * sizeof(SweepOut)) + align256(partial_bytes(I)) +
         256;
}

void batch_setup_inst(const DevMDP& d, int W, char* base, BatchInst& I) {
  I = BatchInst{};
  I.d = d;
  I.ldq = (d.S + 31) / 32 * 32;
  I.sqrtS = std::sqrt((double)d.S);
  batch_geometry(d, I);
  I.cls_sw = ilog2(ell_sweep_lanes_default(d));
  I.cls_mv = ilog2(ell_matvec_lanes_default(d));
  char* p = base;
  auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
  const size_t f = (size_t)I.ldq * 4, f2 = (size_t)I.ldq * 8;
  I.v = (float2*)take(f2);
  I.tv = (float2*)take(f2);
  I.phi = (float*)take(f);
  I.rref = (float*)take(f);
  I.w0 = (float*)take(f);
  I.w1 = (float*)take(f);
  I.rbuf = (float*)take(f);
  I.d0 = (float*)take(f);
  I.d1 = (float*)take(f);
  I.Q = (float*)take((size_t)(W + 1) * I.ldq * 4);
  I.pib[0] = (int32_t*)take(f);
  I.pib[1] = (int32_t*)take(f);
  I.ctl = (GmresCtl*)take(sizeof(GmresCtl));
  I.sout = (SweepOut*)take(4 * sizeof(SweepOut));
  I.partials = take(partial_bytes(I));
  I.counter = (unsigned*)take(256);
  batch_reset_state(I);
}

void batch_reset_state(BatchInst& I) {
  I.phase = BP_SWEEP0;
  I.cur = 0;
  I.k = 0;
  I.reps = 0;
  I.status = MDP_ENOCONV;
  I.starting = 0;
  I.rhs_sel = 0;
  I.inner = I.restarts = I.checks = I.sweeps = I.loops = I.breakdowns = 0;
  I.thr = 0.0;
  I.res = 0.0;
}

int batch_enqueue_iteration(const BatchDev& B, const BatchGrids& g, int maxm, cudaStream_t st,
                            cudaGraphConditionalHandle hc, int with_cond) {
  int r = launch_batch_sweep(B, g.sw, st);
  if (r != MDP_OK) return r;
  batch_ctrl_kernel<<<1, CTRL_THREADS, 0, st>>>(B);
  batch_prologue_kernel<<<g.ew, EW_THREADS, 0, st>>>(B);
  r = launch_batch_matvec(B, 0, g.mv, st);
  if (r == MDP_OK) r = launch_batch_cgs(B, maxm, g.ts, st);
  if (r == MDP_OK) r = launch_batch_estimate(B, maxm, g.ts, st);
  if (r == MDP_OK) r = launch_batch_matvec(B, 1, g.mv, st);
  if (r != MDP_OK) return r;
  batch_value_update_kernel<<<g.ew, EW_THREADS, 0, st>>>(B);
  batch_loop_kernel<<<1, CTRL_THREADS, 0, st>>>(B, hc, with_cond);
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}

int batch_enqueue_relist(const BatchDev& B, cudaStream_t st) {
  batch_relist_kernel<<<1, CTRL_THREADS, 0, st>>>(B);
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}

int batch_enqueue_output_one(const BatchInst* rec, int64_t S, double* vo, int32_t* po,
                             cudaStream_t st) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((S + 255) / 256, (int64_t)num_sms() * 4));
  batch_output_one_kernel<<<grid, 256, 0, st>>>(rec, S, vo, po);
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}

BatchGrids batch_max_grids(int maxm) {
  return BatchGrids{batch_sweep_grid(), batch_matvec_grid(), batch_ts_grid(maxm), num_sms() * 8};
}

}  // namespace mdp
