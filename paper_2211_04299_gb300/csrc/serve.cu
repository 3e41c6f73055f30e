// Serving loop: continuous batching of iGMRES-PI solve requests on one GPU.
//
// A request (an ELL MDP with FP32 P, given as host arrays) goes through
//   PENDING    queued on the host, in arrival order
//   UPLOADING  admitted: a slot is reserved and one stream-ordered device allocation holds
//              its P, g, workspace and result staging; the data is copied and laid out on the
//              upload stream, then validated on the device
//   ACTIVE     its record is written into a slot of the device table; the loop kernels of the
//              batch engine (batch.cu) now serve it together with every other active slot
//   RETIRING   its state machine reached DONE: v = T(V_K) and pi_K are converted and copied to
//              the caller's buffers, then the allocation is freed (stream-ordered) and the slot
//              is released
// Admission needs a free slot and room in the HBM budget (bytes of all admitted requests).
// The device runs the loop in launches of a fixed number of iterations (one CUDA graph with a
// WHILE node, guard = iterations per launch); between launches the host retires finished
// slots and activates uploaded ones, so requests that arrive while others are solving join
// the running mix at the next launch boundary.  Each slot's arithmetic is the batch engine's,
// which does not depend on the other slots: a request's result is the same alone or in a mix.
#include "mdp_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <deque>
#include <string>
#include <vector>

using namespace mdp;

namespace {

constexpr int FLAG_INTS = 16;

enum ReqState { RQ_PENDING = 0, RQ_UPLOADING = 1, RQ_ACTIVE = 2, RQ_RETIRING = 3 };

struct Req {
  int64_t id = 0;
  int64_t S = 0;
  int32_t A = 0, k = 0;
  double gamma = 0.0;
  const int32_t* col = nullptr;
  const float* val = nullptr;
  const double* g = nullptr;
  double* v_out = nullptr;
  int32_t* pi_out = nullptr;
  double t_submit = 0.0;
  size_t bytes = 0;
  char* blk = nullptr;
  int slot = -1;
  int state = RQ_PENDING;
  cudaEvent_t ev = nullptr;
  DevMDP d{};
  char* ws = nullptr;     // workspace inside blk
  double* vo = nullptr;   // result staging inside blk
  int32_t* po = nullptr;
  int* flags = nullptr;   // validation flags inside blk
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

inline size_t al256(size_t x) { return (x + 255) / 256 * 256; }

}  // namespace

struct mdp_server_s {
  mdp_server_opts o{};
  int device = 0;
  cudaStream_t ms = nullptr;  // loop launches, activation, retirement
  cudaStream_t us = nullptr;  // uploads
  cudaStream_t cap = nullptr;
  int n = 0;                  // slots
  BatchInst* d_insts = nullptr;
  BatchInst* h_table = nullptr;  // pinned readback after each launch
  BatchInst* h_stage = nullptr;  // pinned activation records, one per slot
  int* h_flags = nullptr;        // pinned validation flags, one row per slot
  int* d_lists = nullptr;
  int* d_ctr = nullptr;
  BatchDev B{};
  BatchGrids grids{};
  cudaGraphExec_t exec = nullptr;
  cudaEvent_t chunk_ev = nullptr;
  bool chunk_in_flight = false;
  std::deque<Req*> pending;
  std::vector<Req*> slots;       // request holding each slot (any state but PENDING)
  std::vector<int> free_slots;
  int64_t bytes_in_use = 0;
  int64_t next_id = 1;
  std::deque<std::pair<int64_t, mdp_stats>> done;
  std::vector<cudaEvent_t> ev_pool;
  int64_t launches = 0;
  int64_t iterations_launched = 0;
};

namespace {

#define SCK(x)                                                                        \
  do {                                                                                \
    cudaError_t e_ = (x);                                                             \
    if (e_ != cudaSuccess)                                                            \
      return set_error(MDP_EDEVICE, (std::string(#x) + ": " + cudaGetErrorString(e_)).c_str()); \
  } while (0)
#define SRK(x)                                                                        \
  do {                                                                                \
    int r_ = (x);                                                                     \
    if (r_ != MDP_OK) return r_ == MDP_EDEVICE ? set_error(r_, #x) : r_;              \
  } while (0)

cudaEvent_t get_event(mdp_server_s* s) {
  if (!s->ev_pool.empty()) {
    cudaEvent_t e = s->ev_pool.back();
    s->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  return e;
}

void put_event(mdp_server_s* s, cudaEvent_t e) {
  if (e) s->ev_pool.push_back(e);
}

// Device bytes of one request: ELL values and columns [S][A][kp], costs (FP64, double-float
// and a staging copy), the batch workspace, result staging and validation flags.
size_t request_bytes(const DevMDP& d, int W) {
  const size_t rows = (size_t)d.S * d.A;
  return al256(rows * d.kp * 4) * 2 + al256(rows * 8) * 3 + batch_workspace_bytes(d, W) +
         al256((size_t)d.S * 8) + al256((size_t)d.S * 4) + 256;
}

DevMDP request_view(int64_t S, int32_t A, int32_t k, double gamma) {
  DevMDP d{};
  d.S = S;
  d.A = A;
  d.k = k;
  d.kp = (k + 3) / 4 * 4;
  d.ld = 0;
  d.kind = KIND_ELL;
  d.pdt = MDP_F32;
  d.gamma = gamma;
  d.gamma_hi = (float)gamma;
  d.gamma_lo = (float)(gamma - (double)d.gamma_hi);
  d.span = -1;
  return d;
}

void finish(mdp_server_s* s, Req* r, int status, const mdp_stats* st) {
  mdp_stats out{};
  if (st) out = *st;
  out.status = status;
  out.seconds = now_s() - r->t_submit;
  s->done.emplace_back(r->id, out);
  put_event(s, r->ev);
  delete r;
}

// Admission: reserve a slot, allocate, upload and lay out the data, validate (upload stream).
int start_upload(mdp_server_s* s, Req* r) {
  const int W = s->o.solver.restart;
  r->d = request_view(r->S, r->A, r->k, r->gamma);
  r->bytes = request_bytes(r->d, W);
  if (cudaMallocAsync((void**)&r->blk, r->bytes, s->us) != cudaSuccess) {
    // the device is out of memory despite the budget: fail this request, keep serving
    cudaGetLastError();
    r->blk = nullptr;
    r->bytes = 0;
    s->slots[r->slot] = nullptr;
    s->free_slots.push_back(r->slot);
    finish(s, r, MDP_ENOMEM, nullptr);
    return MDP_OK;
  }
  char* p = r->blk;
  auto take = [&](size_t b) { char* q = p; p += al256(b); return q; };
  const DevMDP& d = r->d;
  const size_t rows = (size_t)d.S * d.A;
  float* val = (float*)take(rows * d.kp * 4);
  int32_t* col = (int32_t*)take(rows * d.kp * 4);
  double* g64 = (double*)take(rows * 8);
  float2* gdf = (float2*)take(rows * 8);
  double* gst = (double*)take(rows * 8);
  r->ws = take(batch_workspace_bytes(d, W));
  r->vo = (double*)take((size_t)d.S * 8);
  r->po = (int32_t*)take((size_t)d.S * 4);
  r->flags = (int*)take(FLAG_INTS * sizeof(int));
  r->d.P = val;
  r->d.col = col;
  r->d.g64 = g64;
  r->d.gdf = gdf;
  r->d.mask = nullptr;
  // workspace zero (V_0 = 0, zero pads of the Krylov vectors, reduction counters)
  SCK(cudaMemsetAsync(r->ws, 0, batch_workspace_bytes(d, W), s->us));
  if (d.kp != d.k) {  // pad entries k..kp-1 of every row: value 0, column 0
    SCK(cudaMemset2DAsync(val + d.k, (size_t)d.kp * 4, 0, (size_t)(d.kp - d.k) * 4, rows, s->us));
    SCK(cudaMemset2DAsync(col + d.k, (size_t)d.kp * 4, 0, (size_t)(d.kp - d.k) * 4, rows, s->us));
  }
  for (int a = 0; a < d.A; ++a) {
    SCK(cudaMemcpy2DAsync(val + (size_t)a * d.kp, (size_t)d.A * d.kp * 4, r->val + (size_t)a * d.S * d.k,
                          (size_t)d.k * 4, (size_t)d.k * 4, (size_t)d.S, cudaMemcpyDefault, s->us));
    SCK(cudaMemcpy2DAsync(col + (size_t)a * d.kp, (size_t)d.A * d.kp * 4, r->col + (size_t)a * d.S * d.k,
                          (size_t)d.k * 4, (size_t)d.k * 4, (size_t)d.S, cudaMemcpyDefault, s->us));
  }
  SCK(cudaMemcpyAsync(gst, r->g, rows * 8, cudaMemcpyDefault, s->us));
  SRK(launch_cost_transpose(gst, g64, gdf, d.S, d.A, s->us));
  SCK(cudaMemsetAsync(r->flags, 0, FLAG_INTS * sizeof(int), s->us));
  SRK(launch_validate(d, r->flags, s->us));
  SRK(launch_ell_bank_order(d, val, col, r->flags, s->us));  // the handles' order, bit for bit
  SCK(cudaMemcpyAsync(s->h_flags + (size_t)r->slot * FLAG_INTS, r->flags, FLAG_INTS * sizeof(int),
                      cudaMemcpyDeviceToHost, s->us));
  r->ev = get_event(s);
  if (!r->ev) return set_error(MDP_EDEVICE, "cudaEventCreate failed");
  SCK(cudaEventRecord(r->ev, s->us));
  r->state = RQ_UPLOADING;
  s->bytes_in_use += (int64_t)r->bytes;
  return MDP_OK;
}

void release(mdp_server_s* s, Req* r, cudaStream_t st) {
  if (r->blk) cudaFreeAsync(r->blk, st);
  s->bytes_in_use -= (int64_t)r->bytes;
  if (r->slot >= 0) {
    s->slots[r->slot] = nullptr;
    s->free_slots.push_back(r->slot);
  }
}

// Uploaded and valid: write the slot's record (main stream, between launches).
int activate(mdp_server_s* s, Req* r) {
  const int* f = s->h_flags + (size_t)r->slot * FLAG_INTS;
  if (f[0] || f[1] || f[2] || f[3] || f[4]) {
    release(s, r, s->us);
    finish(s, r, MDP_EINVAL, nullptr);
    return MDP_OK;
  }
  BatchInst& I = s->h_stage[r->slot];
  batch_setup_inst(r->d, s->o.solver.restart, r->ws, I);
  SCK(cudaMemcpyAsync(s->d_insts + r->slot, &I, sizeof(BatchInst), cudaMemcpyHostToDevice, s->ms));
  r->state = RQ_ACTIVE;
  return MDP_OK;
}

// Finished on the device: convert and copy the results out (main stream).
int retire(mdp_server_s* s, Req* r) {
  SRK(batch_enqueue_output_one(s->d_insts + r->slot, r->S, r->vo, r->po, s->ms));
  SCK(cudaMemcpyAsync(r->v_out, r->vo, (size_t)r->S * 8, cudaMemcpyDefault, s->ms));
  SCK(cudaMemcpyAsync(r->pi_out, r->po, (size_t)r->S * 4, cudaMemcpyDefault, s->ms));
  SCK(cudaEventRecord(r->ev, s->ms));
  r->state = RQ_RETIRING;
  return MDP_OK;
}

int build_server_graph(mdp_server_s* s) {
  if (!s->cap) SCK(cudaStreamCreateWithFlags(&s->cap, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  SCK(cudaGraphCreate(&g, 0));
  auto abort_capture = [&](const char* what) {
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(s->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(s->cap, &junk);
    }
    const std::string msg = std::string("server graph: ") + what + ": " +
                            cudaGetErrorString(cudaGetLastError());
    cudaGraphDestroy(g);
    return set_error(MDP_EDEVICE, msg.c_str());
  };
  if (cudaStreamBeginCaptureToGraph(s->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return abort_capture("capture start");
  if (batch_enqueue_relist(s->B, s->cap) != MDP_OK) return abort_capture("relist");
  cudaStreamCaptureStatus cst;
  cudaGraph_t capg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(s->cap, &cst, nullptr, &capg, &deps, nullptr, &nd) != cudaSuccess)
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
  cudaGraph_t g2 = nullptr;
  if (cudaStreamEndCapture(s->cap, &g2) != cudaSuccess) return abort_capture("end capture");
  if (cudaStreamBeginCaptureToGraph(s->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return abort_capture("body capture start");
  if (batch_enqueue_iteration(s->B, s->grids, s->o.solver.restart + 1, s->cap, hc, 1) != MDP_OK)
    return abort_capture("body launches");
  cudaGraph_t b2 = nullptr;
  if (cudaStreamEndCapture(s->cap, &b2) != cudaSuccess) return abort_capture("end body capture");
  if (cudaGraphInstantiate(&s->exec, g, 0) != cudaSuccess) {
    s->exec = nullptr;
    return abort_capture("instantiate");
  }
  cudaGraphDestroy(g);
  return MDP_OK;
}

void free_server(mdp_server_s* s) {
  if (s->ms) cudaStreamSynchronize(s->ms);
  if (s->us) cudaStreamSynchronize(s->us);
  for (Req* r : s->slots)
    if (r) {
      if (r->blk) cudaFree(r->blk);
      if (r->ev) cudaEventDestroy(r->ev);
      delete r;
    }
  for (Req* r : s->pending) delete r;
  for (cudaEvent_t e : s->ev_pool) cudaEventDestroy(e);
  if (s->exec) cudaGraphExecDestroy(s->exec);
  if (s->chunk_ev) cudaEventDestroy(s->chunk_ev);
  void* dp[] = {s->d_insts, s->d_lists, s->d_ctr};
  for (void* p : dp)
    if (p) cudaFree(p);
  void* hp[] = {s->h_table, s->h_stage, s->h_flags};
  for (void* p : hp)
    if (p) cudaFreeHost(p);
  if (s->cap) cudaStreamDestroy(s->cap);
  if (s->us) cudaStreamDestroy(s->us);
  if (s->ms) cudaStreamDestroy(s->ms);
}

int create_server(const mdp_server_opts* opts, mdp_server_s* s) {
  s->o = opts ? *opts : mdp_server_opts_default();
  const mdp_opts& so = s->o.solver;
  if (s->o.max_slots < 1 || s->o.max_slots > 4096) return set_error(MDP_EINVAL, "max_slots must be in 1..4096");
  if (s->o.iters_per_launch < 1) return set_error(MDP_EINVAL, "iters_per_launch must be >= 1");
  if (s->o.hbm_budget_bytes <= 0) return set_error(MDP_EINVAL, "hbm_budget_bytes must be > 0");
  if (so.restart < 1 || so.restart > WMAX) return set_error(MDP_EINVAL, "restart must be in 1..64");
  if (!(so.alpha > 0.0 && so.alpha < 1.0)) return set_error(MDP_EINVAL, "alpha must be in (0, 1)");
  if (!(so.tol >= 0.0)) return set_error(MDP_EINVAL, "tol must be >= 0");
  if (!(so.forcing_c >= 0.0 && so.forcing_c < INFINITY))
    return set_error(MDP_EINVAL, "forcing_c must be finite and >= 0");
  if (so.precond_block != 0) return set_error(MDP_EINVAL, "precond_block applies to ipi_solve only");
  if (so.max_outer < 0 || so.max_inner < 1) return set_error(MDP_EINVAL, "bad iteration caps");
  if (so.precision != MDP_PREC_MIXED) return set_error(MDP_EINVAL, "the server runs in MDP_PREC_MIXED");
  if (so.v0) return set_error(MDP_EINVAL, "requests start from V_0 = 0 (v0 must be NULL)");
  SCK(cudaGetDevice(&s->device));
  SCK(cudaStreamCreateWithFlags(&s->ms, cudaStreamNonBlocking));
  SCK(cudaStreamCreateWithFlags(&s->us, cudaStreamNonBlocking));
  SCK(cudaEventCreateWithFlags(&s->chunk_ev, cudaEventDisableTiming));
  // keep freed request memory in the pool instead of returning it to the driver
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, s->device) == cudaSuccess) {
    uint64_t thr = UINT64_MAX;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
  }
  const int n = s->o.max_slots;
  s->n = n;
  SCK(cudaMalloc((void**)&s->d_insts, sizeof(BatchInst) * n));
  SCK(cudaMallocHost((void**)&s->h_table, sizeof(BatchInst) * n));
  SCK(cudaMallocHost((void**)&s->h_stage, sizeof(BatchInst) * n));
  SCK(cudaMallocHost((void**)&s->h_flags, sizeof(int) * FLAG_INTS * n));
  for (int j = 0; j < n; ++j) {
    s->h_stage[j] = BatchInst{};
    s->h_stage[j].phase = BP_FREE;
  }
  SCK(cudaMemcpy(s->d_insts, s->h_stage, sizeof(BatchInst) * n, cudaMemcpyHostToDevice));
  const int nlists = 5;
  const size_t per_list = (size_t)2 * n + 2;
  SCK(cudaMalloc((void**)&s->d_lists, sizeof(int) * per_list * nlists));
  SCK(cudaMemset(s->d_lists, 0, sizeof(int) * per_list * nlists));
  SCK(cudaMalloc((void**)&s->d_ctr, 64));
  SCK(cudaMemset(s->d_ctr, 0, 64));
  auto list_at = [&](int li) {
    int* base = s->d_lists + per_list * li;
    return BatchList{base, base + n, base + 2 * n + 1};
  };
  BatchDev& B = s->B;
  B.insts = s->d_insts;
  B.n = n;
  B.alpha = so.alpha;
  B.tol = so.tol;
  B.forcing_c = so.forcing_c;
  B.thr_floor = 0.1 * so.tol;
  B.W = so.restart;
  B.max_steps = so.max_inner;
  B.max_outer = so.max_outer;
  B.sw = list_at(0);
  B.mv = list_at(1);
  B.ts = list_at(2);
  B.ew = list_at(3);
  B.all = list_at(4);
  B.vout = nullptr;
  B.pout = nullptr;
  B.ctr = s->d_ctr;
  B.max_iters = s->o.iters_per_launch;
  s->grids = batch_max_grids(so.restart + 1);
  s->slots.assign(n, nullptr);
  for (int j = n - 1; j >= 0; --j) s->free_slots.push_back(j);
  SRK(build_server_graph(s));
  return MDP_OK;
}

// One step of the server: retire finished work, admit and activate requests, keep the
// device loop running.  Never waits for the device.
int server_step(mdp_server_s* s) {
  // 1. the last launch of loop iterations finished: retire instances that are done
  if (s->chunk_in_flight) {
    const cudaError_t q = cudaEventQuery(s->chunk_ev);
    if (q == cudaSuccess) {
      s->chunk_in_flight = false;
      for (int j = 0; j < s->n; ++j) {
        Req* r = s->slots[j];
        if (r && r->state == RQ_ACTIVE && s->h_table[j].phase == BP_DONE) SRK(retire(s, r));
      }
    } else if (q != cudaErrorNotReady) {
      return set_error(MDP_EDEVICE, cudaGetErrorString(q));
    }
  }
  // 2. retirement copies that completed: report, free memory and the slot
  for (int j = 0; j < s->n; ++j) {
    Req* r = s->slots[j];
    if (!r || r->state != RQ_RETIRING) continue;
    const cudaError_t q = cudaEventQuery(r->ev);
    if (q == cudaErrorNotReady) continue;
    if (q != cudaSuccess) return set_error(MDP_EDEVICE, cudaGetErrorString(q));
    const BatchInst& I = s->h_table[j];
    mdp_stats st{};
    st.outer = I.k;
    st.inner = I.inner;
    st.restarts = I.restarts;
    st.sweeps = I.sweeps;
    st.matvecs = I.inner + I.checks;
    st.breakdowns = I.breakdowns;
    st.residual_inf = I.res;
    const int status = I.status;
    release(s, r, s->ms);
    finish(s, r, status, &st);
  }
  // 3. admission in arrival order: a free slot and room in the HBM budget
  while (!s->pending.empty() && !s->free_slots.empty()) {
    Req* r = s->pending.front();
    const size_t need = request_bytes(request_view(r->S, r->A, r->k, r->gamma), s->o.solver.restart);
    if ((int64_t)need > s->o.hbm_budget_bytes) {
      s->pending.pop_front();
      finish(s, r, MDP_ENOMEM, nullptr);
      continue;
    }
    if (s->bytes_in_use + (int64_t)need > s->o.hbm_budget_bytes) break;
    s->pending.pop_front();
    r->slot = s->free_slots.back();
    s->free_slots.pop_back();
    s->slots[r->slot] = r;
    const int rc = start_upload(s, r);
    if (rc != MDP_OK) return rc;
  }
  // 4. between launches: activate uploaded requests, then launch the next iterations
  if (!s->chunk_in_flight) {
    bool any = false;
    for (int j = 0; j < s->n; ++j) {
      Req* r = s->slots[j];
      if (!r) continue;
      if (r->state == RQ_UPLOADING) {
        const cudaError_t q = cudaEventQuery(r->ev);
        if (q == cudaErrorNotReady) continue;
        if (q != cudaSuccess) return set_error(MDP_EDEVICE, cudaGetErrorString(q));
        SRK(activate(s, r));
        r = s->slots[j];
      }
      if (r && r->state == RQ_ACTIVE) any = true;
    }
    if (any) {
      SCK(cudaGraphLaunch(s->exec, s->ms));
      SCK(cudaMemcpyAsync(s->h_table, s->d_insts, sizeof(BatchInst) * s->n, cudaMemcpyDeviceToHost, s->ms));
      SCK(cudaEventRecord(s->chunk_ev, s->ms));
      s->chunk_in_flight = true;
      s->launches += 1;
    }
  }
  return MDP_OK;
}

int take_done(mdp_server_s* s, int64_t* ids, mdp_stats* stats, int32_t max_done, int32_t* n_done) {
  int32_t m = 0;
  while (m < max_done && !s->done.empty()) {
    if (ids) ids[m] = s->done.front().first;
    if (stats) stats[m] = s->done.front().second;
    s->done.pop_front();
    ++m;
  }
  if (n_done) *n_done = m;
  return MDP_OK;
}

bool idle(const mdp_server_s* s) {
  if (!s->pending.empty() || s->chunk_in_flight) return false;
  for (const Req* r : s->slots)
    if (r) return false;
  return true;
}

}  // namespace

extern "C" {

mdp_server_opts mdp_server_opts_default(void) {
  mdp_server_opts o{};
  o.hbm_budget_bytes = (int64_t)120 << 30;
  o.max_slots = 256;
  o.iters_per_launch = 4;
  o.solver = mdp_opts_default();
  return o;
}

int mdp_server_create(const mdp_server_opts* opts, mdp_server_t* out) {
  if (!out) return set_error(MDP_EINVAL, "null output handle");
  *out = nullptr;
  mdp_server_s* s = new mdp_server_s();
  const int r = create_server(opts, s);
  if (r != MDP_OK) {
    free_server(s);
    delete s;
    return r;
  }
  *out = s;
  return MDP_OK;
}

void mdp_server_destroy(mdp_server_t s) {
  if (!s) return;
  free_server(s);
  delete s;
}

int mdp_server_submit(mdp_server_t s, int64_t S, int32_t A, int32_t k, const int32_t* col,
                      const float* val, const double* g, double gamma, double* v_out,
                      int32_t* pi_out, int64_t* request_id) {
  if (!s) return set_error(MDP_EINVAL, "null server");
  if (S < 1 || S > (int64_t)INT32_MAX - 64) return set_error(MDP_EINVAL, "S must be in 1..2^31-65");
  if (A < 1) return set_error(MDP_EINVAL, "A must be >= 1");
  if (k < 1 || (int64_t)k > S) return set_error(MDP_EINVAL, "k must be in 1..S");
  if (!(gamma > 0.0 && gamma < 1.0)) return set_error(MDP_EINVAL, "gamma must be in (0, 1)");
  if (!col || !val || !g || !v_out || !pi_out) return set_error(MDP_EINVAL, "null request array");
  Req* r = new Req();
  r->id = s->next_id++;
  r->S = S;
  r->A = A;
  r->k = k;
  r->gamma = gamma;
  r->col = col;
  r->val = val;
  r->g = g;
  r->v_out = v_out;
  r->pi_out = pi_out;
  r->t_submit = now_s();
  s->pending.push_back(r);
  if (request_id) *request_id = r->id;
  return server_step(s);
}

int mdp_server_poll(mdp_server_t s, int64_t* ids, mdp_stats* stats, int32_t max_done,
                    int32_t* n_done) {
  if (!s) return set_error(MDP_EINVAL, "null server");
  if (max_done < 0) return set_error(MDP_EINVAL, "max_done must be >= 0");
  SRK(server_step(s));
  return take_done(s, ids, stats, max_done, n_done);
}

int mdp_server_drain(mdp_server_t s) {
  if (!s) return set_error(MDP_EINVAL, "null server");
  while (!idle(s)) SRK(server_step(s));
  return MDP_OK;
}

int mdp_server_info(mdp_server_t s, int32_t* active, int32_t* pending, int64_t* bytes_in_use,
                    int64_t* launches) {
  if (!s) return set_error(MDP_EINVAL, "null server");
  int32_t a = 0;
  for (const Req* r : s->slots)
    if (r) ++a;
  if (active) *active = a;
  if (pending) *pending = (int32_t)s->pending.size();
  if (bytes_in_use) *bytes_in_use = s->bytes_in_use;
  if (launches) *launches = s->launches;
  return MDP_OK;
}

}  // extern "C"
