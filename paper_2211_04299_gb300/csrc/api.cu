// C ABI of libmdpgpu: handle management, validation and the host drivers of the solvers.
// Every arithmetic step runs in the kernels of sweep.cu and krylov.cu; the host only
// enqueues launches and reads back the scalars that decide control flow.
#include "mdp_internal.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

using namespace mdp;

namespace {

thread_local std::string g_err;

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

#define CK(x)                                                                          \
  do {                                                                                 \
    cudaError_t e_ = (x);                                                              \
    if (e_ != cudaSuccess) return fail(MDP_EDEVICE, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)
#define RK(x)                                                                          \
  do {                                                                                 \
    int r_ = (x);                                                                      \
    if (r_ != MDP_OK) {                                                                \
      if (r_ == MDP_EDEVICE) return fail(r_, std::string(#x) + ": " + cudaGetErrorString(cudaGetLastError())); \
      if (g_err.empty()) g_err = #x;                                                   \
      return r_;                                                                       \
    }                                                                                  \
  } while (0)

inline int64_t round_up(int64_t x, int64_t m) { return (x + m - 1) / m * m; }

struct HostCtl {  // leading fields of GmresCtl read back by the host
  int mode, status, i, W, steps, max_steps, restarts, dsel, from_rhs, est_runs, checks, loop_iters;
};

struct Workspace {
  int kt = -1;
  int W = 0;
  int64_t ldq = 0;
  void* Q = nullptr;
  void* w0 = nullptr;
  void* w1 = nullptr;
  void* rbuf = nullptr;
  void* d0 = nullptr;
  void* d1 = nullptr;
  void* phi = nullptr;
  void* rref = nullptr;  // residual of the previous policy at the new iterate (Krylov type)
  void* v = nullptr;   // value vector (double or float2)
  void* tv = nullptr;
  double* stage64 = nullptr;
  int32_t* pi = nullptr;
  int32_t* pi2 = nullptr;
  GmresCtl* ctl = nullptr;
  SweepOut* sout = nullptr;  // [4]
  void* partials = nullptr;
  unsigned* counter = nullptr;
  int* flags = nullptr;
  SweepOut* h_sout = nullptr;  // pinned
  HostCtl* h_ctl = nullptr;    // pinned
  size_t bytes = 0;
};

}  // namespace

struct mdp_s {
  DevMDP d{};
  void* P = nullptr;
  int32_t* col = nullptr;
  double* g64 = nullptr;
  float2* gdf = nullptr;
  uint8_t* mask = nullptr;
  double* gstage = nullptr;
  int* vflags = nullptr;   // validation flags of mdp_create / mdp_load
  int* h_vflags = nullptr; // pinned copy of them
  int vpending = 0;        // an enqueued load not yet checked (mdp_load_*_async)
  cudaStream_t stream = nullptr;
  cudaStream_t own = nullptr;
  int device = 0;
  int timing = 0;
  int lanes_sweep = 0;   // ELL lanes per row (0 = library choice)
  int lanes_matvec = 0;
  int grid_sweep = 0;    // blocks per launch (0 = library choice)
  int grid_matvec = 0;
  int grid_krylov = 0;
  double forcing_c = 0.0;  // forcing sequence of the current ipi_solve (mdp_opts.forcing_c)
  double thr_floor = 0.0;  // and its floor on the inner threshold (tol / 10)
  size_t data_bytes = 0;
  Workspace ws;
  // two-level preconditioner of ipi_solve (mdp_opts.precond_block): per-policy coarse data
  struct Precond {
    int kt = -1, W = 0, lb = -1, bw = -1;
    int bw_lb = -1;        // aggregation the cached bandwidth was measured for (-1: none)
    int bw_cached = -1;
    int64_t nc = 0, ldc = 0;
    float* band = nullptr;
    float* cl = nullptr;
    float* cu = nullptr;
    float* dinv = nullptr;
    float* inv = nullptr;
    void* E = nullptr;
    void* ec = nullptr;
    void* z = nullptr;
    float* f = nullptr;
    int32_t* pi_built = nullptr;  // the policy the current coarse factors were built for
    int* nchanged = nullptr;      // states whose action differs from pi_built (device)
    int* h_nchanged = nullptr;    // pinned copy
    int built = 0;                // factors valid for the current solve
    int* bwbuf = nullptr;
    size_t bytes = 0;
  } pc;
  int pc_on = 0;           // the current solve applies the preconditioner
  int no_window = 0;       // the current solve asked for the global-gather ELL sweep
  int64_t last_span = -2;  // column reach of the data the inner graphs were captured for
  // graph-resident inner GMRES loops of ipi_solve: [0] a fresh solve on Phi_k, [1] a solve
  // resumed on the exact residual found by the verifying sweep (rebuilt when parameters change)
  struct InnerGraph {
    cudaGraphExec_t exec = nullptr;
    int kt = -1, W = 0, steps = 0;
    double alpha = -1.0, forcing_c = -1.0, thr_floor = -1.0;
    const void* ws = nullptr;
    const void* pcz = nullptr;  // preconditioner buffers the graph was captured with (or null)
    int nowin = -1;             // MDP_FLAG_NO_WINDOW at capture (selects the matvec kernel)
  } ig[2];
  cudaStream_t cap = nullptr;
  std::vector<cudaEvent_t> ev;   // event pool (pairs)
  std::vector<int> ev_kind;      // 0 sweep, 1 matvec
  size_t ev_used = 0;
  int launches = 0;
};

namespace {

void free_ws(Workspace& w) {
  void* ptrs[] = {w.Q, w.w0, w.w1, w.rbuf, w.d0, w.d1, w.phi, w.rref, w.v, w.tv, w.stage64, w.pi, w.pi2,
                  w.ctl, w.sout, w.partials, w.counter, w.flags};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (w.h_sout) cudaFreeHost(w.h_sout);
  if (w.h_ctl) cudaFreeHost(w.h_ctl);
  w = Workspace{};
}

void free_pc(mdp_s::Precond& p) {
  void* ptrs[] = {p.band, p.cl, p.cu, p.dinv, p.inv, p.E, p.ec, p.z, p.f, p.pi_built, p.nchanged};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (p.h_nchanged) cudaFreeHost(p.h_nchanged);
  int* keep = p.bwbuf;
  const int bl = p.bw_lb, bc = p.bw_cached;
  p = mdp_s::Precond{};
  p.bwbuf = keep;
  p.bw_lb = bl;
  p.bw_cached = bc;
}

int alloc0(void** p, size_t bytes, size_t& acc) {
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(MDP_ENOMEM, "cudaMalloc of " + std::to_string(bytes) + " bytes failed");
  }
  acc += bytes;
  if (cudaMemset(*p, 0, bytes) != cudaSuccess) return fail(MDP_EDEVICE, "cudaMemset failed");
  return MDP_OK;
}

// kt: 0 double Krylov / double values, 1 float Krylov / double-float values
int ensure_ws(mdp_t h, int kt, int W) {
  Workspace& w = h->ws;
  if (w.kt == kt && w.W >= W && w.ctl) return MDP_OK;
  if (w.ctl) CK(cudaStreamSynchronize(h->stream));
  free_ws(w);
  const int64_t S = h->d.S;
  w.kt = kt;
  w.W = W;
  w.ldq = round_up(std::max<int64_t>(S, h->d.ld), 32);
  const size_t ek = kt ? 4 : 8;
  const size_t vec = (size_t)w.ldq * ek;
  size_t& acc = w.bytes;
  RK(alloc0(&w.Q, vec * (W + 1), acc));
  RK(alloc0(&w.w0, vec, acc));
  RK(alloc0(&w.w1, vec, acc));
  RK(alloc0(&w.rbuf, vec, acc));
  RK(alloc0(&w.d0, vec, acc));
  RK(alloc0(&w.d1, vec, acc));
  RK(alloc0(&w.phi, vec, acc));
  RK(alloc0(&w.rref, vec, acc));
  RK(alloc0(&w.v, (size_t)w.ldq * 8, acc));
  RK(alloc0(&w.tv, (size_t)w.ldq * 8, acc));
  RK(alloc0((void**)&w.stage64, (size_t)w.ldq * 8, acc));
  RK(alloc0((void**)&w.pi, (size_t)w.ldq * 4, acc));
  RK(alloc0((void**)&w.pi2, (size_t)w.ldq * 4, acc));
  RK(alloc0((void**)&w.ctl, sizeof(GmresCtl), acc));
  RK(alloc0((void**)&w.sout, 4 * sizeof(SweepOut), acc));
  RK(alloc0(&w.partials, (size_t)MAX_RED_BLOCKS * (WMAX + 1) * 8, acc));
  RK(alloc0((void**)&w.counter, 64, acc));
  RK(alloc0((void**)&w.flags, 64, acc));
  CK(cudaMallocHost((void**)&w.h_sout, 4 * sizeof(SweepOut)));
  CK(cudaMallocHost((void**)&w.h_ctl, sizeof(HostCtl)));
  return MDP_OK;
}

// Blocks of the tall-skinny Krylov kernels (mdp_set_geometry may fix them).
int krylov_grid(mdp_t h) { return h->grid_krylov > 0 ? h->grid_krylov : krylov_blocks(h->d.S); }

KrylovBufs kbufs(mdp_t h) {
  Workspace& w = h->ws;
  KrylovBufs B;
  B.kt = w.kt;
  B.S = h->d.S;
  B.ldq = w.ldq;
  B.Q = w.Q;
  B.w0 = w.w0;
  B.w1 = w.w1;
  B.rbuf = w.rbuf;
  B.d0 = w.d0;
  B.d1 = w.d1;
  B.partials = w.partials;
  B.counter = w.counter;
  B.ctl = w.ctl;
  B.grid = krylov_grid(h);
  B.maxm = w.W + 1;
  if (h->pc_on) {
    B.ec = h->pc.ec;
    B.lb = h->pc.lb;
  }
  return B;
}

constexpr int64_t PC_NC_MAX = 8192;  // coarse blocks (J_c^{-1} is nc^2 FP32 values)

// Coarse half-bandwidth of the transition data for blocks of 2^lb states (cached until the
// data is reloaded).  When the upload's validation measured the column reach r = max |col - s|,
// the bound |block(col) - block(s)| <= (r + b - 1) / b (b = 2^lb) is used without a pass over
// the columns: a band a block wider than the data needs only holds zeros, which the GTH
// elimination and the inverse carry through unchanged.
int coarse_bandwidth(mdp_t h, int lb, int* bw) {
  auto& p = h->pc;
  if (p.bw_lb == lb) {
    *bw = p.bw_cached;
    return MDP_OK;
  }
  if (h->d.span >= 0) {
    const int64_t b = (int64_t)1 << lb;
    const int64_t hb = (h->d.span + b - 1) >> lb;
    p.bw_lb = lb;
    p.bw_cached = (int)std::min<int64_t>(hb, INT32_MAX);
    *bw = p.bw_cached;
    return MDP_OK;
  }
  if (!p.bwbuf) {
    size_t acc = 0;
    if (cudaMalloc((void**)&p.bwbuf, 64) != cudaSuccess) {
      cudaGetLastError();
      p.bwbuf = nullptr;
      return fail(MDP_ENOMEM, "cudaMalloc failed");
    }
    (void)acc;
  }
  CK(cudaMemsetAsync(p.bwbuf, 0, sizeof(int), h->stream));
  RK(launch_coarse_bandwidth(h->d, lb, p.bwbuf, h->stream));
  int hb = 0;
  CK(cudaMemcpyAsync(&hb, p.bwbuf, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  p.bw_lb = lb;
  p.bw_cached = hb;
  *bw = hb;
  return MDP_OK;
}

// Buffers of the two-level preconditioner for Krylov type kt, restart W and blocks of
// 2^lb states (after ensure_ws).
int ensure_pc(mdp_t h, int kt, int W, int lb) {
  auto& p = h->pc;
  if (h->d.kind != KIND_ELL) return fail(MDP_EINVAL, "the two-level preconditioner needs ELL data");
  const int64_t S = h->d.S;
  const int64_t nc = (S + ((int64_t)1 << lb) - 1) >> lb;
  if (nc > PC_NC_MAX)
    return fail(MDP_EINVAL, "precond_block too small: more than 8192 coarse blocks");
  int bw = 0;
  RK(coarse_bandwidth(h, lb, &bw));
  if (bw > PC_BW_MAX)
    return fail(MDP_EINVAL, "transitions reach more than 31 aggregation blocks away: "
                            "use a larger precond_block");
  if (p.kt == kt && p.W >= W && p.lb == lb && p.bw == bw && p.inv) return MDP_OK;
  if (p.inv) CK(cudaStreamSynchronize(h->stream));
  free_pc(p);
  p.kt = kt;
  p.W = W;
  p.lb = lb;
  p.bw = bw;
  p.nc = nc;
  p.ldc = round_up(nc, 4);
  const size_t ek = kt ? 4 : 8;
  size_t& acc = p.bytes;
  RK(alloc0((void**)&p.band, (size_t)nc * (2 * bw + 2) * 4, acc));
  RK(alloc0((void**)&p.cl, (size_t)nc * 32 * 4, acc));
  RK(alloc0((void**)&p.cu, (size_t)nc * 32 * 4, acc));
  RK(alloc0((void**)&p.dinv, (size_t)nc * 4, acc));
  RK(alloc0((void**)&p.inv, (size_t)nc * p.ldc * 4, acc));
  RK(alloc0(&p.E, (size_t)W * p.ldc * ek, acc));
  RK(alloc0(&p.ec, (size_t)p.ldc * ek, acc));
  RK(alloc0(&p.z, (size_t)h->ws.ldq * ek, acc));
  RK(alloc0((void**)&p.f, (size_t)p.ldc * 4, acc));
  RK(alloc0((void**)&p.pi_built, (size_t)S * 4, acc));
  RK(alloc0((void**)&p.nchanged, 64, acc));
  if (cudaMallocHost((void**)&p.h_nchanged, 64) != cudaSuccess) {
    p.h_nchanged = nullptr;
    return fail(MDP_ENOMEM, "cudaMallocHost failed");
  }
  return MDP_OK;
}

PrecondK pck(mdp_t h) {
  const Workspace& w = h->ws;
  const auto& p = h->pc;
  PrecondK k;
  k.ctl = w.ctl;
  k.S = h->d.S;
  k.nc = p.nc;
  k.ldq = w.ldq;
  k.ldc = p.ldc;
  k.lb = p.lb;
  k.rbuf = w.rbuf;
  k.w0 = w.w0;
  k.w1 = w.w1;
  k.Q = w.Q;
  k.E = p.E;
  k.ec = p.ec;
  k.z = p.z;
  k.f = p.f;
  k.inv = p.inv;
  return k;
}

// ---------------------------------------------------------------- event timing
int tic(mdp_t h, int kind) {
  if (!h->timing) return -1;
  if (h->ev_used + 2 > h->ev.size()) {
    for (int i = 0; i < 256; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      h->ev.push_back(e);
    }
    h->ev_kind.resize(h->ev.size() / 2 + 1);
  }
  int idx = (int)h->ev_used;
  h->ev_used += 2;
  h->ev_kind[idx / 2] = kind;
  cudaEventRecord(h->ev[idx], h->stream);
  return idx;
}
void toc(mdp_t h, int idx) {
  if (idx >= 0) cudaEventRecord(h->ev[idx + 1], h->stream);
}
void collect_times(mdp_t h, mdp_stats* st) {
  if (!h->timing) return;
  for (size_t i = 0; i + 1 < h->ev_used; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, h->ev[i], h->ev[i + 1]) != cudaSuccess) {
      cudaGetLastError();
      continue;
    }
    if (st) {
      if (h->ev_kind[i / 2] == 0) { st->sweep_ms += ms; st->timed_sweeps += 1; }
      else { st->matvec_ms += ms; st->timed_matvecs += 1; }
    }
  }
  h->ev_used = 0;
}

// ---------------------------------------------------------------- algorithmic bytes
double sweep_bytes(mdp_t h, bool policy_only, int arith) {
  const DevMDP& d = h->d;
  const double eb = d.pdt == MDP_F32 ? 4.0 : 8.0;
  const double rows = policy_only ? (double)d.S : (double)d.S * d.A;
  double b = d.kind == KIND_DENSE ? rows * (double)d.S * eb : rows * (double)d.k * (eb + 4.0);
  b += rows * (arith ? 8.0 : 8.0);         // g (double or double-float)
  b += (double)d.S * 8.0;                  // v
  b += (double)d.S * (4.0 + 8.0 + (arith ? 4.0 : 8.0));  // pi, Tv, Phi writes
  return b;
}
double matvec_bytes(mdp_t h, int kt) {
  const DevMDP& d = h->d;
  const double eb = d.pdt == MDP_F32 ? 4.0 : 8.0;
  const double ek = kt ? 4.0 : 8.0;
  double b = d.kind == KIND_DENSE ? (double)d.S * d.S * eb : (double)d.S * d.k * (eb + 4.0);
  return b + (double)d.S * (4.0 + 3.0 * ek);
}

// ---------------------------------------------------------------- launch helpers
int sweep(mdp_t h, int arith, const void* v, const int32_t* pi_in, int32_t* pi_out, void* tv_out,
          double* tv64_out, void* phi_out, double* margin_out, SweepOut* out, mdp_stats* st,
          const int32_t* pi_ref = nullptr, void* rref_out = nullptr, SweepOut* ref_out = nullptr) {
  SweepLaunch L{};
  L.pi_ref = pi_ref;
  L.rref_out = rref_out;
  L.ref_out = ref_out;
  L.d = h->d;
  L.arith = arith;
  L.v = v;
  L.pi_in = pi_in;
  L.pi_out = pi_out;
  L.tv_out = tv_out;
  L.tv64_out = tv64_out;
  L.phi_out = phi_out;
  L.margin_out = margin_out;
  L.out = out;
  L.partials = h->ws.partials;
  L.counter = h->ws.counter;
  L.err = h->ws.flags + 8;
  L.lanes = h->lanes_sweep;
  L.grid = pi_in ? 0 : h->grid_sweep;
  L.no_window = h->no_window || h->grid_sweep > 0;  // a fixed geometry is the batch's
  int t = tic(h, pi_in ? 1 : 0);
  int r = launch_sweep(L, h->stream);
  toc(h, t);
  h->launches += 1;
  if (st) {
    if (pi_in) st->matvecs += 1; else st->sweeps += 1;
    st->bytes += sweep_bytes(h, pi_in != nullptr, arith);
  }
  return r == MDP_EDEVICE ? fail(r, std::string("sweep launch: ") + cudaGetErrorString(cudaGetLastError())) : r;
}

int read_sout(mdp_t h, int slot, SweepOut* out) {
  CK(cudaMemcpyAsync(h->ws.h_sout + slot, h->ws.sout + slot, sizeof(SweepOut),
                     cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *out = h->ws.h_sout[slot];
  return MDP_OK;
}

int read_ctl(mdp_t h, HostCtl* c) {
  CK(cudaMemcpyAsync(h->ws.h_ctl, h->ws.ctl, sizeof(HostCtl), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  *c = *h->ws.h_ctl;
  return MDP_OK;
}

// Bounded device waits that ran out raise flags[8]; report and clear it.
int check_device_error(mdp_t h) {
  int e = 0;
  CK(cudaMemcpyAsync(&e, h->ws.flags + 8, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (e) {
    cudaMemsetAsync(h->ws.flags + 8, 0, sizeof(int), h->stream);
    return fail(MDP_ETIMEOUT, "a bounded device wait ran out (bulk-copy pipeline)");
  }
  return MDP_OK;
}

// Load an initial value vector (double, host or device; null = 0) into the workspace.
int load_v(mdp_t h, const double* v0, int arith) {
  Workspace& w = h->ws;
  const int64_t S = h->d.S;
  CK(cudaMemsetAsync(w.v, 0, (size_t)w.ldq * 8, h->stream));
  if (!v0) return MDP_OK;
  if (arith) {
    CK(cudaMemcpyAsync(w.stage64, v0, (size_t)S * 8, cudaMemcpyDefault, h->stream));
    RK(launch_d_to_df(w.stage64, (float2*)w.v, S, h->stream));
  } else {
    CK(cudaMemcpyAsync(w.v, v0, (size_t)S * 8, cudaMemcpyDefault, h->stream));
  }
  return MDP_OK;
}

int store_v(mdp_t h, const void* src, double* dst, int arith) {
  const int64_t S = h->d.S;
  if (arith) {
    RK(launch_df_to_d((const float2*)src, h->ws.stage64, S, h->stream));
    CK(cudaMemcpyAsync(dst, h->ws.stage64, (size_t)S * 8, cudaMemcpyDefault, h->stream));
  } else {
    CK(cudaMemcpyAsync(dst, src, (size_t)S * 8, cudaMemcpyDefault, h->stream));
  }
  return MDP_OK;
}

int enqueue_step(mdp_t h, const int32_t* pi_dev, const void* rhs, cudaStream_t st);
// Kernels per Arnoldi step as enqueue_step issues them (loop-condition kernel not included).
int step_launches(mdp_t h) { return h->pc_on ? 10 : 6; }

// One inner solve (Alg. 2 inner loop) on J^pi delta = rhs (rhs already in ws.phi, its norms
// in ws.sout[slot]), with pi in ws.pi (or pi_dev).  thr: absolute target when alpha == 0.
// On return delta is added to ws.v.
int inner_gmres(mdp_t h, const int32_t* pi_dev, int slot, double alpha, double thr, int W,
                int max_steps, mdp_stats* st, int* status_out, const void* rhs = nullptr,
                int resume = 0, int accept_est = 0) {
  Workspace& w = h->ws;
  const int kt = w.kt;
  const int64_t S = h->d.S;
  const size_t ek = kt ? 4 : 8;
  KrylovBufs B = kbufs(h);
  CK(cudaMemcpyAsync(w.rbuf, rhs ? rhs : w.phi, (size_t)S * ek, cudaMemcpyDeviceToDevice, h->stream));
  CK(cudaMemsetAsync(w.d0, 0, (size_t)S * ek, h->stream));
  RK(launch_gmres_init(B, thr, std::sqrt((double)S), W, max_steps, w.sout + slot, alpha,
                       h->stream, resume, accept_est, h->forcing_c, h->thr_floor));
  h->launches += 1;
  HostCtl hc{};
  RK(read_ctl(h, &hc));
  for (int it = 0; it <= max_steps + 1 && hc.mode != GM_DONE; ++it) {
    RK(enqueue_step(h, pi_dev, rhs ? rhs : w.phi, h->stream));
    h->launches += step_launches(h);
    RK(read_ctl(h, &hc));
  }
  if (hc.mode != GM_DONE) return fail(MDP_ETIMEOUT, "inner GMRES did not reach a final state");
  RK(launch_value_update(kt, w.v, w.d0, w.d1, w.ctl, nullptr, S, h->stream));
  h->launches += 1;
  if (st) {
    st->inner += hc.steps;
    st->restarts += hc.restarts;
    st->matvecs += hc.steps + hc.checks;
    const double ek2 = (double)ek;
    st->bytes += (double)(hc.steps + hc.checks) * matvec_bytes(h, kt);
    // CGS2: three passes over Q_0..Q_i plus w traffic, per step (i averaged over the cycle)
    const double avg_m = std::min<double>(W, hc.steps) * 0.5 + 1.0;
    st->bytes += hc.steps * (3.0 * avg_m + 6.0) * (double)S * ek2;
    if (hc.status == GS_BREAKDOWN) st->breakdowns += 1;
  }
  if (status_out) *status_out = hc.status;
  return MDP_OK;
}

// The Arnoldi step as enqueued kernels (matvec, CGS2 + Givens, estimate + candidate, true
// check); every kernel is gated on the device-resident mode.  rhs is the right-hand side of
// the solve (Phi_k, or the exact residual when a solve resumes), used by the true-residual
// matvec.
int enqueue_step(mdp_t h, const int32_t* pi_dev, const void* rhs, cudaStream_t st) {
  Workspace& w = h->ws;
  KrylovBufs B = kbufs(h);
  MatvecLaunch M{};
  M.d = h->d;
  M.kt = w.kt;
  M.pi = pi_dev;
  M.ctl = w.ctl;
  M.gate_mode = GM_STEP;
  M.gate_mode2 = GM_STEP;
  M.x_rhs = w.rbuf;
  M.x_w0 = w.w0;
  M.x_w1 = w.w1;
  M.qbase = w.Q;
  M.ldq = w.ldq;
  M.a = 1.0;
  M.b = 0.0;
  M.c = -h->d.gamma;
  M.out0 = w.w0;
  M.out1 = w.w1;
  M.partials = w.partials;
  M.counter = w.counter;
  M.err = w.flags + 8;
  M.lanes = h->lanes_matvec;
  M.grid = h->grid_matvec;
  M.no_window = h->no_window;
  MatvecLaunch C = M;
  C.gate_mode = GM_CHECK;
  C.gate_mode2 = GM_RESTART;
  C.ctl = nullptr;
  C.ctl_rw = w.ctl;
  C.x_w0 = w.d0;
  C.x_w1 = w.d1;
  C.a = -1.0;
  C.b = 1.0;
  C.c = h->d.gamma;
  C.u = rhs;
  C.out = w.rbuf;
  C.qbase = nullptr;
  if (h->pc_on) {
    // right preconditioning: Q_i, R Q_i, E_i = J_c^{-1} R Q_i and z = M^{-1} Q_i first
    RK(launch_coarse_step(pck(h), w.kt, st));
    M.x_pre = h->pc.z;
  }
  RK(launch_matvec(M, st));
  RK(launch_cgs2_givens(B, st));
  if (h->pc_on) RK(launch_coarse_combine(pck(h), w.kt, st));
  RK(launch_estimate(B, st));
  RK(launch_matvec(C, st));
  return MDP_OK;
}


// Build the graph of one inner solve: prologue (start vector, zero correction, control
// block), a WHILE node whose body is one Arnoldi step plus the loop-condition kernel, and the
// value update V <- V + delta.  No host decision is needed inside.  Variant 0 starts from
// Phi_k (norms in sout[0], threshold alpha ||Phi_k||_inf); variant 1 resumes from the exact
// residual of the same policy (rref, norms in sout[2]) with the saved threshold.  Both accept
// on the Arnoldi-relation estimate: the next Bellman sweep tests the exact residual.
int build_inner_graph(mdp_t h, int variant, const int32_t* pi_dev, double alpha, int W,
                      int max_steps) {
  Workspace& w = h->ws;
  auto& gg = h->ig[variant];
  if (gg.exec) {
    cudaGraphExecDestroy(gg.exec);
    gg.exec = nullptr;
  }
  if (!h->cap) CK(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
  const int64_t S = h->d.S;
  const size_t ek = w.kt ? 4 : 8;
  KrylovBufs B = kbufs(h);
  cudaGraph_t g = nullptr;
  CK(cudaGraphCreate(&g, 0));
  auto fail_graph = [&](int code) {
    cudaStreamCaptureStatus cs;
    if (cudaStreamIsCapturing(h->cap, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
      cudaGraph_t junk = nullptr;
      cudaStreamEndCapture(h->cap, &junk);
    }
    cudaGetLastError();
    cudaGraphDestroy(g);
    return code;
  };
  if (cudaStreamBeginCaptureToGraph(h->cap, g, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return fail_graph(fail(MDP_EDEVICE, "graph capture could not start"));
  int r = MDP_OK;
  const void* rhs = variant == 0 ? w.phi : w.rref;
  if (cudaMemcpyAsync(w.rbuf, rhs, (size_t)S * ek, cudaMemcpyDeviceToDevice, h->cap) != cudaSuccess ||
      cudaMemsetAsync(w.d0, 0, (size_t)S * ek, h->cap) != cudaSuccess)
    return fail_graph(fail(MDP_EDEVICE, "graph prologue copy"));
  r = launch_gmres_init(B, 0.0, std::sqrt((double)S), W, max_steps, w.sout + (variant == 0 ? 0 : 2),
                        alpha, h->cap, variant, 1, h->forcing_c, h->thr_floor);
  if (r != MDP_OK) return fail_graph(r);
  cudaStreamCaptureStatus cst;
  cudaGraph_t capg = nullptr;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  if (cudaStreamGetCaptureInfo(h->cap, &cst, nullptr, &capg, &deps, nullptr, &nd) != cudaSuccess)
    return fail_graph(fail(MDP_EDEVICE, "capture info"));
  cudaGraphConditionalHandle hc;
  if (cudaGraphConditionalHandleCreate(&hc, capg, 1, cudaGraphCondAssignDefault) != cudaSuccess)
    return fail_graph(fail(MDP_EDEVICE, "conditional handle"));
  cudaGraphNodeParams np = {};
  np.type = cudaGraphNodeTypeConditional;
  np.conditional.handle = hc;
  np.conditional.type = cudaGraphCondTypeWhile;
  np.conditional.size = 1;
  cudaGraphNode_t cn;
  if (cudaGraphAddNode(&cn, capg, deps, nullptr, nd, &np) != cudaSuccess)
    return fail_graph(fail(MDP_EDEVICE, "conditional node"));
  cudaGraph_t body = np.conditional.phGraph_out[0];
  if (cudaStreamUpdateCaptureDependencies(h->cap, &cn, nullptr, 1, cudaStreamSetCaptureDependencies) != cudaSuccess)
    return fail_graph(fail(MDP_EDEVICE, "capture dependencies"));
  r = launch_value_update(w.kt, w.v, w.d0, w.d1, w.ctl, nullptr, S, h->cap);
  if (r != MDP_OK) return fail_graph(r);
  cudaGraph_t g2 = nullptr;
  if (cudaStreamEndCapture(h->cap, &g2) != cudaSuccess) return fail_graph(fail(MDP_EDEVICE, "end capture"));
  // loop body
  if (cudaStreamBeginCaptureToGraph(h->cap, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed) != cudaSuccess)
    return fail_graph(fail(MDP_EDEVICE, "body capture could not start"));
  r = enqueue_step(h, pi_dev, rhs, h->cap);
  if (r == MDP_OK) r = launch_loop_cond(hc, w.ctl, max_steps + 8, h->cap);
  if (r != MDP_OK) return fail_graph(r);
  cudaGraph_t b2 = nullptr;
  if (cudaStreamEndCapture(h->cap, &b2) != cudaSuccess) return fail_graph(fail(MDP_EDEVICE, "end body capture"));
  if (cudaGraphInstantiate(&gg.exec, g, 0) != cudaSuccess) {
    gg.exec = nullptr;
    return fail_graph(fail(MDP_EDEVICE, "graph instantiate"));
  }
  cudaGraphDestroy(g);
  gg.kt = w.kt;
  gg.W = W;
  gg.steps = max_steps;
  gg.alpha = alpha;
  gg.forcing_c = h->forcing_c;
  gg.thr_floor = h->thr_floor;
  gg.ws = w.ctl;
  gg.pcz = h->pc_on ? h->pc.z : nullptr;
  gg.nowin = h->no_window;
  return MDP_OK;
}

// The inner graphs always use ws.pi as the policy (the driver copies pi_{k} there).
int launch_inner_graph(mdp_t h, int variant, double alpha, int W, int max_steps) {
  Workspace& w = h->ws;
  auto& gg = h->ig[variant];
  if (!gg.exec || gg.kt != w.kt || gg.W != W || gg.steps != max_steps || gg.alpha != alpha ||
      gg.forcing_c != h->forcing_c || gg.thr_floor != h->thr_floor ||
      gg.ws != w.ctl || gg.pcz != (h->pc_on ? h->pc.z : nullptr) || gg.nowin != h->no_window)
    RK(build_inner_graph(h, variant, w.pi, alpha, W, max_steps));
  CK(cudaGraphLaunch(gg.exec, h->stream));
  return MDP_OK;
}

mdp_opts normalise(const mdp_opts* o) {
  mdp_opts r = o ? *o : mdp_opts_default();
  return r;
}

int check_opts(mdp_t h, const mdp_opts& o) {
  if (!h) return fail(MDP_EINVAL, "null handle");
  if (o.restart < 1 || o.restart > WMAX) return fail(MDP_EINVAL, "restart must be in 1..64");
  if (!(o.alpha >= 0.0 && o.alpha < 1.0)) return fail(MDP_EINVAL, "alpha must be in [0, 1)");
  if (!(o.forcing_c >= 0.0 && o.forcing_c < INFINITY))
    return fail(MDP_EINVAL, "forcing_c must be finite and >= 0");
  if (!(o.tol >= 0.0)) return fail(MDP_EINVAL, "tol must be >= 0");
  if (o.max_outer < 0 || o.max_inner < 1) return fail(MDP_EINVAL, "bad iteration caps");
  if (o.precision != MDP_PREC_FP64 && o.precision != MDP_PREC_MIXED)
    return fail(MDP_EINVAL, "unknown precision");
  if (o.precision == MDP_PREC_MIXED && h->d.pdt != MDP_F32)
    return fail(MDP_EINVAL, "mixed precision needs FP32 transition data");
  if (o.precond_block != 0 &&
      (o.precond_block < 4 || o.precond_block > (1 << 20) || (o.precond_block & (o.precond_block - 1))))
    return fail(MDP_EINVAL, "precond_block must be 0 or a power of two in [4, 2^20]");
  return MDP_OK;
}

int log2_exact(int x) {
  int l = 0;
  while ((1 << l) < x) ++l;
  return l;
}

// Clears the per-solve switches of a handle when a solve leaves, on every path.
struct PcGuard {
  mdp_t h;
  ~PcGuard() { h->pc_on = 0; h->no_window = 0; }
};

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// ---------------------------------------------------------------- solvers (device buffers)
enum Method { METH_IPI = 0, METH_VI = 1, METH_PI = 2, METH_OPI = 3, METH_IPI_VI = 4 };

// Policy evaluation to an absolute target by repeated inner solves on the current residual
// (one solve in FP64; in FP32 Krylov each solve cuts the residual by up to 1e-5 and the
// next residual is recomputed in double-float).
int eval_policy(mdp_t h, const int32_t* pi_dev, int arith, double target, const mdp_opts& o,
                mdp_stats* st, double* final_res, int* last_status = nullptr) {
  Workspace& w = h->ws;
  const double floor_rel = arith ? 1e-5 : 0.0;
  double res = INFINITY, prev = INFINITY;
  for (int rep = 0; rep < 50; ++rep) {
    // residual of pi at v: T^pi v - v (into phi) and its norms
    RK(sweep(h, arith, w.v, pi_dev, nullptr, nullptr, nullptr, w.phi, nullptr, w.sout + 1, st));
    SweepOut so;
    RK(read_sout(h, 1, &so));
    res = so.res_inf;
    if (!(res > target)) break;
    if (rep > 0 && !(res < 0.5 * prev)) break;  // stagnated at the arithmetic's floor
    prev = res;
    const double thr = std::max(target, floor_rel * res);
    int status = 0;
    RK(inner_gmres(h, pi_dev, 1, 0.0, thr, o.restart, o.max_inner, st, &status));
    if (last_status) *last_status = status;
    if (status == GS_CAP && !arith) break;
  }
  if (final_res) *final_res = res;
  return MDP_OK;
}

// iGMRES-PI, Alg. 2.  Outer iteration k: the inner GMRES(W) solve of J^{pi_k} delta = Phi_k
// runs as one graph launch and stops when the Arnoldi-relation estimate of
// ||g^{pi_k} - J^{pi_k} V_{k+1}||_inf meets alpha ||Phi_k||_inf; the next Bellman sweep then
// gives pi_{k+1}, Phi_{k+1} and, for the reference policy pi_k, the exact residual at V_{k+1}
// (double-float or FP64).  If that exact residual is above the threshold, the inner solve
// resumes from it (a restart from the current iterate) and the sweep is repeated, so the
// stopping rule of Alg. 2 always holds on the exact residual.
int run_ipi(mdp_t h, const mdp_opts& o, double* v_out, int32_t* pi_out, mdp_stats* st_user) {
  const double t0 = now_s();
  mdp_stats st{};
  h->launches = 0;
  const int arith = o.precision == MDP_PREC_MIXED ? 1 : 0;
  RK(ensure_ws(h, arith, o.restart));
  Workspace& w = h->ws;
  const int64_t S = h->d.S;
  h->forcing_c = o.forcing_c;
  h->thr_floor = 0.1 * o.tol;
  PcGuard pc_guard{h};
  if (o.precond_block) {
    RK(ensure_pc(h, arith, o.restart, log2_exact(o.precond_block)));
    h->pc_on = 1;
    h->pc.built = 0;
  }
  RK(load_v(h, o.v0, arith));
  int status = MDP_ENOCONV;
  SweepOut so{};
  int k = 0;
  RK(sweep(h, arith, w.v, nullptr, w.pi, w.tv, nullptr, w.phi, nullptr, w.sout, &st));
  RK(read_sout(h, 0, &so));
  while (true) {
    if (so.res_inf <= o.tol) { status = MDP_OK; break; }
    if (k >= o.max_outer) break;
    const double thr = inexact_threshold(o.alpha, o.forcing_c, so.res_inf, h->thr_floor);
    const bool host_loop = (o.flags & MDP_FLAG_HOST_LOOP) != 0;
    if (h->pc_on) {  // coarse operator of the policy pi_k: band, LU, explicit inverse
      auto& pc = h->pc;
      bool rebuild = !pc.built || (o.flags & MDP_FLAG_PC_REBUILD);
      if (!rebuild) {  // factors of a nearby policy remain a valid right preconditioner
        CK(cudaMemsetAsync(pc.nchanged, 0, sizeof(int), h->stream));
        RK(launch_count_changed(w.pi, pc.pi_built, S, pc.nchanged, h->stream));
        CK(cudaMemcpyAsync(pc.h_nchanged, pc.nchanged, sizeof(int), cudaMemcpyDeviceToHost, h->stream));
        CK(cudaStreamSynchronize(h->stream));
        rebuild = (int64_t)*pc.h_nchanged * 1000 > S;
        h->launches += 1;
      }
      if (rebuild) {
        RK(launch_coarse_setup(h->d, w.pi, pck(h), pc.bw,
                               PrecondScratch{pc.band, pc.cl, pc.cu, pc.dinv}, h->stream));
        CK(cudaMemcpyAsync(pc.pi_built, w.pi, (size_t)S * 4, cudaMemcpyDeviceToDevice, h->stream));
        pc.built = 1;
        h->launches += 4;
      }
    }
    if (host_loop) RK(inner_gmres(h, w.pi, 0, o.alpha, 0.0, o.restart, o.max_inner, nullptr, nullptr,
                                  w.phi, 0, 1));
    else RK(launch_inner_graph(h, 0, o.alpha, o.restart, o.max_inner));
    ++k;
    for (int rep = 0;; ++rep) {
      RK(sweep(h, arith, w.v, nullptr, w.pi2, w.tv, nullptr, w.phi, nullptr, w.sout, &st, w.pi,
               w.rref, w.sout + 2));
      CK(cudaMemcpyAsync(w.h_ctl, w.ctl, sizeof(HostCtl), cudaMemcpyDeviceToHost, h->stream));
      CK(cudaMemcpyAsync(w.h_sout + 2, w.sout + 2, sizeof(SweepOut), cudaMemcpyDeviceToHost, h->stream));
      RK(read_sout(h, 0, &so));
      const HostCtl hc = *w.h_ctl;
      const SweepOut sref = w.h_sout[2];
      if (hc.mode != GM_DONE) return fail(MDP_ETIMEOUT, "inner GMRES loop ended without a final state");
      st.inner += hc.steps;
      st.restarts += hc.restarts;
      st.matvecs += hc.steps + hc.checks;
      if (hc.status == GS_BREAKDOWN) st.breakdowns += 1;
      st.bytes += (double)(hc.steps + hc.checks) * matvec_bytes(h, w.kt);
      const double avg_m = std::min<double>(o.restart, hc.steps) * 0.5 + 1.0;
      st.bytes += hc.steps * (3.0 * avg_m + 6.0) * (double)S * (w.kt ? 4.0 : 8.0);
      h->launches += host_loop ? 0 : 4 + (step_launches(h) + 1) * hc.loop_iters;
      // exact stopping test of Alg. 2 (breakdown or the step cap also end the inner loop)
      if (!(sref.res_inf > thr) || hc.status == GS_BREAKDOWN || hc.status == GS_CAP || rep >= 8) break;
      st.restarts += 1;
      if (host_loop) RK(inner_gmres(h, w.pi, 2, o.alpha, 0.0, o.restart, o.max_inner, nullptr,
                                    nullptr, w.rref, 1, 1));
      else RK(launch_inner_graph(h, 1, o.alpha, o.restart, o.max_inner));
    }
    // pi_{k+1} = GreedyPolicy(V_{k+1}) becomes the current policy
    CK(cudaMemcpyAsync(w.pi, w.pi2, (size_t)S * 4, cudaMemcpyDeviceToDevice, h->stream));
  }
  st.outer = k;
  st.residual_inf = so.res_inf;
  RK(store_v(h, w.tv, v_out, arith));
  if (pi_out) CK(cudaMemcpyAsync(pi_out, w.pi, (size_t)S * 4, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  RK(check_device_error(h));
  collect_times(h, &st);
  st.status = status;
  st.launches = h->launches;
  st.seconds = now_s() - t0;
  if (st_user) *st_user = st;
  if (status != MDP_OK) g_err = "iteration cap reached before ||T(v)-v||_inf <= tol";
  return status;
}

int run_solver(mdp_t h, int method, const mdp_opts& o, double* v_out, int32_t* pi_out,
               mdp_stats* st_user) {
  const double t0 = now_s();
  mdp_stats st{};
  h->launches = 0;
  const int arith = o.precision == MDP_PREC_MIXED ? 1 : 0;
  RK(ensure_ws(h, arith, o.restart));
  Workspace& w = h->ws;
  RK(load_v(h, o.v0, arith));
  int status = MDP_ENOCONV;
  SweepOut so{};
  int k = 0;
  for (k = 0; k <= o.max_outer; ++k) {
    // pi_k = GreedyPolicy(V_k), T V_k, Phi_k = T V_k - V_k and ||Phi_k||_inf
    RK(sweep(h, arith, w.v, nullptr, w.pi, w.tv, nullptr, w.phi, nullptr, w.sout, &st));
    RK(read_sout(h, 0, &so));
    if (so.res_inf <= o.tol) { status = MDP_OK; break; }
    if (k == o.max_outer) break;
    if (method == METH_VI) {
      std::swap(w.v, w.tv);
    } else if (method == METH_OPI) {
      std::swap(w.v, w.tv);  // first application of T^{pi_k} is T V_k
      for (int j = 1; j < o.opi_W; ++j) {
        RK(sweep(h, arith, w.v, w.pi, nullptr, w.tv, nullptr, nullptr, nullptr, w.sout + 2, &st));
        std::swap(w.v, w.tv);
      }
    } else if (method == METH_IPI_VI) {
      // Alg. 1 with VI as the inner solver: V <- T^{pi_k} V while the residual of pi_k,
      // ||g^{pi_k} - J^{pi_k} V||_inf = ||T^{pi_k} V - V||_inf, is above alpha_k ||Phi_k||_inf.
      // The first step is T V_k of the greedy sweep; each further policy sweep gives the
      // residual at the current V and T^{pi_k} V together.
      const double thr = inexact_threshold(o.alpha, o.forcing_c, so.res_inf, 0.1 * o.tol);
      std::swap(w.v, w.tv);
      int j = 1;
      for (; j < o.max_inner; ++j) {
        RK(sweep(h, arith, w.v, w.pi, nullptr, w.tv, nullptr, nullptr, nullptr, w.sout + 2, &st));
        SweepOut sr{};
        RK(read_sout(h, 2, &sr));
        if (!(sr.res_inf > thr)) break;
        std::swap(w.v, w.tv);
      }
      st.inner += j;
    } else {  // PI: evaluate pi_k "exactly" (relative 10^-x of ||Phi_k||)
      const double target = so.res_inf * std::pow(10.0, -(double)o.pi_inner_tol_exp);
      double r = 0;
      RK(eval_policy(h, w.pi, arith, target, o, &st, &r));
    }
  }
  st.outer = k;
  st.residual_inf = so.res_inf;
  // v = T(V_K) of the last sweep, pi = GreedyPolicy(V_K)
  RK(store_v(h, w.tv, v_out, arith));
  if (pi_out) CK(cudaMemcpyAsync(pi_out, w.pi, (size_t)h->d.S * 4, cudaMemcpyDefault, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  RK(check_device_error(h));
  collect_times(h, &st);
  st.status = status;
  st.launches = h->launches;
  st.seconds = now_s() - t0;
  if (st_user) *st_user = st;
  if (status != MDP_OK) g_err = "iteration cap reached before ||T(v)-v||_inf <= tol";
  return status;
}

// ---------------------------------------------------------------- creation
int validate_args(int64_t S, int32_t A, int32_t k, int kind, int dt, double gamma,
                  const void* P, const int32_t* col, const double* g) {
  if (S < 1 || S > (int64_t)INT32_MAX - 64) return fail(MDP_EINVAL, "S must be in 1..2^31-65");
  if (A < 1) return fail(MDP_EINVAL, "A must be >= 1");
  if (kind == KIND_ELL && (k < 1 || (int64_t)k > S)) return fail(MDP_EINVAL, "k must be in 1..S");
  if (dt != MDP_F32 && dt != MDP_F64) return fail(MDP_EINVAL, "dtype must be MDP_F32 or MDP_F64");
  if (!(gamma > 0.0 && gamma < 1.0)) return fail(MDP_EINVAL, "gamma must be in (0, 1)");
  if (!P || !g || (kind == KIND_ELL && !col)) return fail(MDP_EINVAL, "null input array");
  return MDP_OK;
}

// Enqueue the upload of P (and columns), g and the mask on the handle's stream, the cost
// layout change and the device validation, whose flags are copied to pinned host memory.
int enqueue_upload(mdp_t h, const void* P, const int32_t* col, const double* g,
                   const uint8_t* mask) {
  DevMDP& d = h->d;
  const size_t eb = d.pdt == MDP_F32 ? 4 : 8;
  cudaStream_t s = h->stream;
  h->pc.bw_lb = -1;  // new data: the coarse bandwidth is measured again
  d.span = -1;
  if (d.kind == KIND_DENSE) {
    // zero only the pad columns S..ld-1 of every row; the copies below write the rest
    if (d.ld > d.S)
      CK(cudaMemset2DAsync((char*)h->P + (size_t)d.S * eb, (size_t)d.ld * eb, 0,
                           (size_t)(d.ld - d.S) * eb, (size_t)d.S * d.A, s));
    for (int a = 0; a < d.A; ++a) {
      const char* src = (const char*)P + (size_t)a * d.S * d.S * eb;
      char* dst = (char*)h->P + (size_t)a * d.ld * eb;
      CK(cudaMemcpy2DAsync(dst, (size_t)d.A * d.ld * eb, src, (size_t)d.S * eb, (size_t)d.S * eb,
                           (size_t)d.S, cudaMemcpyDefault, s));
    }
  } else {
    if (d.kp > d.k) {  // pad entries k..kp-1 of every row: value 0, column 0
      CK(cudaMemset2DAsync((char*)h->P + (size_t)d.k * eb, (size_t)d.kp * eb, 0,
                           (size_t)(d.kp - d.k) * eb, (size_t)d.S * d.A, s));
      CK(cudaMemset2DAsync((char*)h->col + (size_t)d.k * 4, (size_t)d.kp * 4, 0,
                           (size_t)(d.kp - d.k) * 4, (size_t)d.S * d.A, s));
    }
    for (int a = 0; a < d.A; ++a) {
      const char* src = (const char*)P + (size_t)a * d.S * d.k * eb;
      char* dst = (char*)h->P + (size_t)a * d.kp * eb;
      CK(cudaMemcpy2DAsync(dst, (size_t)d.A * d.kp * eb, src, (size_t)d.k * eb, (size_t)d.k * eb,
                           (size_t)d.S, cudaMemcpyDefault, s));
      const char* srcc = (const char*)col + (size_t)a * d.S * d.k * 4;
      char* dstc = (char*)h->col + (size_t)a * d.kp * 4;
      CK(cudaMemcpy2DAsync(dstc, (size_t)d.A * d.kp * 4, srcc, (size_t)d.k * 4, (size_t)d.k * 4,
                           (size_t)d.S, cudaMemcpyDefault, s));
    }
  }
  CK(cudaMemcpyAsync(h->gstage, g, (size_t)d.S * d.A * 8, cudaMemcpyDefault, s));
  RK(launch_cost_transpose(h->gstage, h->g64, h->gdf, d.S, d.A, s));
  if (mask) CK(cudaMemcpyAsync(h->mask, mask, (size_t)d.S * d.A, cudaMemcpyDefault, s));
  // validate on the device
  int* flags = h->vflags;  // allocated with the handle (a per-load cudaFree would stall the device)
  CK(cudaMemsetAsync(flags, 0, 8 * sizeof(int), s));
  RK(launch_validate(d, flags, s));
  RK(launch_ell_bank_order(d, h->P, h->col, flags, s));
  CK(cudaMemcpyAsync(h->h_vflags, flags, 8 * sizeof(int), cudaMemcpyDeviceToHost, s));
  h->vpending = 1;
  return MDP_OK;
}

// Wait for an enqueued upload (this handle's stream only) and report its validation.
int finish_upload(mdp_t h) {
  if (!h->vpending) return MDP_OK;
  h->vpending = 0;
  const cudaError_t e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) return fail(MDP_EDEVICE, std::string("upload: ") + cudaGetErrorString(e));
  const int* hf = h->h_vflags;
  if (hf[0]) return fail(MDP_EINVAL, "transition probabilities must be finite and >= 0");
  if (hf[1]) return fail(MDP_EINVAL, "ELL column index out of range [0, S)");
  if (hf[2]) return fail(MDP_EINVAL, "a transition row does not sum to 1 within tolerance");
  if (hf[3]) return fail(MDP_EINVAL, "costs must be finite");
  if (hf[4]) return fail(MDP_EINVAL, "every state needs at least one allowed action");
  const int64_t span = h->d.kind == KIND_ELL ? hf[6] : -1;  // column reach: banded data windowed
  if (span != h->last_span) {
    // inner-loop graphs hold the DevMDP (and so the kernel choice) they were captured with
    for (auto& gg : h->ig)
      if (gg.exec) {
        cudaGraphExecDestroy(gg.exec);
        gg.exec = nullptr;
      }
    h->last_span = span;
  }
  h->d.span = span;
  return MDP_OK;
}

int create_common(int64_t S, int32_t A, int32_t k, int kind, const void* P, int dt,
                  const int32_t* col, const double* g, double gamma, const uint8_t* mask,
                  mdp_t* out) {
  g_err.clear();
  if (!out) return fail(MDP_EINVAL, "null output handle pointer");
  *out = nullptr;
  RK(validate_args(S, A, k, kind, dt, gamma, P, col, g));
  mdp_t h = new (std::nothrow) mdp_s();
  if (!h) return fail(MDP_ENOMEM, "host allocation failed");
  cudaGetDevice(&h->device);
  if (cudaStreamCreateWithFlags(&h->own, cudaStreamNonBlocking) != cudaSuccess) {
    delete h;
    return fail(MDP_EDEVICE, "cudaStreamCreate failed");
  }
  h->stream = h->own;
  DevMDP& d = h->d;
  d.S = S;
  d.A = A;
  d.k = kind == KIND_ELL ? k : (int32_t)std::min<int64_t>(S, INT32_MAX);
  d.kp = kind == KIND_ELL ? (int32_t)round_up(k, 4) : 0;
  d.ld = kind == KIND_DENSE ? round_up(S, 32) : 0;  // 128-byte aligned rows
  d.kind = kind;
  d.pdt = dt;
  d.gamma = gamma;
  d.gamma_hi = (float)gamma;
  d.gamma_lo = (float)(gamma - (double)d.gamma_hi);
  d.span = -1;  // measured by the validation of each upload
  const size_t eb = dt == MDP_F32 ? 4 : 8;
  size_t acc = 0;
  int r = MDP_OK;
  auto bail = [&](int code) {
    mdp_destroy(h);
    return code;
  };
  if (kind == KIND_DENSE) r = alloc0(&h->P, (size_t)S * A * d.ld * eb, acc);
  else {
    r = alloc0(&h->P, (size_t)S * A * d.kp * eb, acc);
    if (r == MDP_OK) r = alloc0((void**)&h->col, (size_t)S * A * d.kp * 4, acc);
  }
  if (r == MDP_OK) r = alloc0((void**)&h->g64, (size_t)S * A * 8, acc);
  if (r == MDP_OK && dt == MDP_F32) r = alloc0((void**)&h->gdf, (size_t)S * A * 8, acc);
  if (r == MDP_OK) r = alloc0((void**)&h->gstage, (size_t)S * A * 8, acc);
  if (r == MDP_OK) r = alloc0((void**)&h->vflags, 8 * sizeof(int), acc);
  if (r == MDP_OK && cudaMallocHost((void**)&h->h_vflags, 8 * sizeof(int)) != cudaSuccess)
    r = fail(MDP_ENOMEM, "cudaMallocHost of the validation flags failed");
  if (r == MDP_OK && mask) r = alloc0((void**)&h->mask, (size_t)S * A, acc);
  if (r != MDP_OK) return bail(r);
  h->data_bytes = acc;
  d.P = h->P;
  d.col = h->col;
  d.g64 = h->g64;
  d.gdf = h->gdf;
  d.mask = h->mask;
  r = enqueue_upload(h, P, col, g, mask);
  if (r == MDP_OK) r = finish_upload(h);
  if (r != MDP_OK) return bail(r);
  *out = h;
  return MDP_OK;
}

}  // namespace

// ====================================================================== C ABI
namespace mdp {
const DevMDP* handle_view(mdp_t h) { return h ? &h->d : nullptr; }
int handle_finish_pending(mdp_t h) { return h ? finish_upload(h) : MDP_OK; }
int handle_device(mdp_t h) { return h ? h->device : -1; }
int set_error(int code, const char* msg) { return fail(code, msg); }
}  // namespace mdp

extern "C" {

mdp_opts mdp_opts_default(void) {
  mdp_opts o;
  o.alpha = 0.1;
  o.tol = 1e-8;
  o.restart = 30;
  o.max_outer = 100;
  o.max_inner = 3000;
  o.precision = MDP_PREC_MIXED;
  o.opi_W = 50;
  o.pi_inner_tol_exp = 13;
  o.flags = 0;
  o.v0 = nullptr;
  o.forcing_c = 0.0;
  o.precond_block = 0;
  return o;
}

const char* mdp_last_error(void) { return g_err.c_str(); }
const char* mdp_version(void) { return "mdpgpu 0.1 (sm_103a)"; }

int mdp_create_dense(int64_t S, int32_t A, const void* P, int p_dtype, const double* g,
                     double gamma, const uint8_t* mask, mdp_t* out) {
  return create_common(S, A, 0, KIND_DENSE, P, p_dtype, nullptr, g, gamma, mask, out);
}
int mdp_create_ell(int64_t S, int32_t A, int32_t k, const int32_t* col, const void* val,
                   int val_dtype, const double* g, double gamma, const uint8_t* mask,
                   mdp_t* out) {
  return create_common(S, A, k, KIND_ELL, val, val_dtype, col, g, gamma, mask, out);
}
int mdp_create_dense_dev(int64_t S, int32_t A, const void* P, int p_dtype, const double* g,
                         double gamma, const uint8_t* mask, mdp_t* out) {
  return create_common(S, A, 0, KIND_DENSE, P, p_dtype, nullptr, g, gamma, mask, out);
}
int mdp_create_ell_dev(int64_t S, int32_t A, int32_t k, const int32_t* col, const void* val,
                       int val_dtype, const double* g, double gamma, const uint8_t* mask,
                       mdp_t* out) {
  return create_common(S, A, k, KIND_ELL, val, val_dtype, col, g, gamma, mask, out);
}

int mdp_load_dense_async(mdp_t h, const void* P, const double* g) {
  g_err.clear();
  if (!h || h->d.kind != KIND_DENSE || !P || !g) return fail(MDP_EINVAL, "bad handle or input");
  RK(finish_upload(h));
  return enqueue_upload(h, P, nullptr, g, nullptr);
}
int mdp_load_ell_async(mdp_t h, const int32_t* col, const void* val, const double* g) {
  g_err.clear();
  if (!h || h->d.kind != KIND_ELL || !col || !val || !g) return fail(MDP_EINVAL, "bad handle or input");
  RK(finish_upload(h));
  return enqueue_upload(h, val, col, g, nullptr);
}
int mdp_load_dense(mdp_t h, const void* P, const double* g) {
  RK(mdp_load_dense_async(h, P, g));
  return finish_upload(h);
}
int mdp_load_ell(mdp_t h, const int32_t* col, const void* val, const double* g) {
  RK(mdp_load_ell_async(h, col, val, g));
  return finish_upload(h);
}

void mdp_destroy(mdp_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  free_ws(h->ws);
  free_pc(h->pc);
  if (h->pc.bwbuf) cudaFree(h->pc.bwbuf);
  void* ptrs[] = {h->P, h->col, h->g64, h->gdf, h->mask, h->gstage, h->vflags};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (h->h_vflags) cudaFreeHost(h->h_vflags);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  for (auto& gg : h->ig)
    if (gg.exec) cudaGraphExecDestroy(gg.exec);
  if (h->cap) cudaStreamDestroy(h->cap);
  if (h->own) cudaStreamDestroy(h->own);
  delete h;
}

int mdp_set_stream(mdp_t h, void* stream) {
  if (!h) return fail(MDP_EINVAL, "null handle");
  RK(finish_upload(h));
  CK(cudaStreamSynchronize(h->stream));
  h->stream = stream ? (cudaStream_t)stream : h->own;
  return MDP_OK;
}

int mdp_set_tuning(mdp_t h, int32_t ell_lanes_sweep, int32_t ell_lanes_matvec) {
  if (!h) return fail(MDP_EINVAL, "null handle");
  auto ok = [](int x) { return x == 0 || x == 1 || x == 2 || x == 4 || x == 8; };
  if (!ok(ell_lanes_sweep) || !ok(ell_lanes_matvec)) return fail(MDP_EINVAL, "lanes must be 0, 1, 2, 4 or 8");
  h->lanes_sweep = ell_lanes_sweep;
  h->lanes_matvec = ell_lanes_matvec;
  for (auto& gg : h->ig)  // captured graphs hold the old shapes
    if (gg.exec) {
      cudaGraphExecDestroy(gg.exec);
      gg.exec = nullptr;
    }
  return MDP_OK;
}

int mdp_set_geometry(mdp_t h, int32_t sweep_blocks, int32_t matvec_blocks, int32_t krylov_blocks) {
  if (!h) return fail(MDP_EINVAL, "null handle");
  if (h->d.kind != KIND_ELL) return fail(MDP_EINVAL, "block geometry applies to ELL handles");
  const int32_t lim = MAX_RED_BLOCKS;
  if (sweep_blocks < 0 || matvec_blocks < 0 || krylov_blocks < 0 || sweep_blocks > lim ||
      matvec_blocks > lim || krylov_blocks > lim)
    return fail(MDP_EINVAL, "block counts must be in 0..2048");
  h->grid_sweep = sweep_blocks;
  h->grid_matvec = matvec_blocks;
  h->grid_krylov = krylov_blocks;
  for (auto& gg : h->ig) {
    if (gg.exec) cudaGraphExecDestroy(gg.exec);
    gg.exec = nullptr;
  }
  return MDP_OK;
}

int mdp_set_timing(mdp_t h, int on) {
  if (!h) return fail(MDP_EINVAL, "null handle");
  h->timing = on ? 1 : 0;
  return MDP_OK;
}

int mdp_info(mdp_t h, int64_t* S, int32_t* A, int32_t* k, int32_t* kind, int32_t* dtype,
             double* gamma) {
  if (!h) return fail(MDP_EINVAL, "null handle");
  if (S) *S = h->d.S;
  if (A) *A = h->d.A;
  if (k) *k = h->d.kind == KIND_ELL ? h->d.k : 0;
  if (kind) *kind = h->d.kind;
  if (dtype) *dtype = h->d.pdt;
  if (gamma) *gamma = h->d.gamma;
  return MDP_OK;
}

int64_t mdp_device_bytes(mdp_t h) {
  if (!h) return -1;
  return (int64_t)(h->data_bytes + h->ws.bytes + h->pc.bytes);
}

int bellman_apply_dev(mdp_t h, const double* v, double* Tv, int32_t* pi, double* margin,
                      double* res_inf, int32_t precision) {
  if (h && h->vpending) RK(finish_upload(h));
  g_err.clear();
  if (!h || !v) return fail(MDP_EINVAL, "null handle or v");
  const int arith = precision == MDP_PREC_MIXED ? 1 : 0;
  if (arith && h->d.pdt != MDP_F32) return fail(MDP_EINVAL, "mixed precision needs FP32 data");
  RK(ensure_ws(h, arith, h->ws.W > 0 ? h->ws.W : 30));
  RK(load_v(h, v, arith));
  RK(sweep(h, arith, h->ws.v, nullptr, pi, nullptr, Tv, nullptr, margin, h->ws.sout, nullptr));
  if (res_inf) {
    SweepOut so;
    RK(read_sout(h, 0, &so));
    *res_inf = so.res_inf;
  }
  return res_inf ? check_device_error(h) : MDP_OK;
}

int bellman_apply(mdp_t h, const double* v, double* Tv, int32_t* pi, double* res_inf,
                  int32_t precision) {
  if (h && h->vpending) RK(finish_upload(h));
  g_err.clear();
  if (!h || !v) return fail(MDP_EINVAL, "null handle or v");
  const int arith = precision == MDP_PREC_MIXED ? 1 : 0;
  if (arith && h->d.pdt != MDP_F32) return fail(MDP_EINVAL, "mixed precision needs FP32 data");
  RK(ensure_ws(h, arith, h->ws.W > 0 ? h->ws.W : 30));
  Workspace& w = h->ws;
  const int64_t S = h->d.S;
  RK(load_v(h, v, arith));
  RK(sweep(h, arith, w.v, nullptr, w.pi2, nullptr, w.stage64, nullptr, nullptr, w.sout, nullptr));
  if (Tv) CK(cudaMemcpyAsync(Tv, w.stage64, (size_t)S * 8, cudaMemcpyDeviceToHost, h->stream));
  if (pi) CK(cudaMemcpyAsync(pi, w.pi2, (size_t)S * 4, cudaMemcpyDeviceToHost, h->stream));
  SweepOut so;
  RK(read_sout(h, 0, &so));
  if (res_inf) *res_inf = so.res_inf;
  return check_device_error(h);
}

int policy_eval_gmres_dev(mdp_t h, const int32_t* pi, const double* v0, double target_inf,
                          const mdp_opts* opts, double* v_out, mdp_stats* stats) {
  if (h && h->vpending) RK(finish_upload(h));
  g_err.clear();
  mdp_opts o = normalise(opts);
  RK(check_opts(h, o));
  if (!pi || !v_out) return fail(MDP_EINVAL, "null pi or v_out");
  if (o.precond_block != 0) return fail(MDP_EINVAL, "precond_block applies to ipi_solve only");
  if (!(target_inf >= 0.0)) return fail(MDP_EINVAL, "target must be >= 0");
  PcGuard guard{h};
  h->no_window = (o.flags & MDP_FLAG_NO_WINDOW) != 0;
  const double t0 = now_s();
  mdp_stats st{};
  h->launches = 0;
  const int arith = o.precision == MDP_PREC_MIXED ? 1 : 0;
  RK(ensure_ws(h, arith, o.restart));
  Workspace& w = h->ws;
  CK(cudaMemcpyAsync(w.pi2, pi, (size_t)h->d.S * 4, cudaMemcpyDefault, h->stream));
  {
    CK(cudaMemsetAsync(w.flags, 0, 64, h->stream));
    RK(launch_check_policy(w.pi2, h->d.S, h->d.A, h->d.mask, w.flags, h->stream));
    int hf[16] = {0};
    CK(cudaMemcpyAsync(hf, w.flags, 64, cudaMemcpyDeviceToHost, h->stream));
    CK(cudaStreamSynchronize(h->stream));
    if (hf[5]) return fail(MDP_EINVAL, "policy entry out of range or not an allowed action");
  }
  RK(load_v(h, v0, arith));
  double res = 0;
  int last = GS_RUNNING;
  RK(eval_policy(h, w.pi2, arith, target_inf, o, &st, &res, &last));
  RK(store_v(h, w.v, v_out, arith));
  CK(cudaStreamSynchronize(h->stream));
  RK(check_device_error(h));
  collect_times(h, &st);
  st.residual_inf = res;
  st.status = res <= target_inf ? (last == GS_BREAKDOWN ? MDP_EBREAKDOWN_INFO : MDP_OK)
                                 : MDP_ENOCONV;
  st.launches = h->launches;
  st.seconds = now_s() - t0;
  if (stats) *stats = st;
  if (st.status == MDP_ENOCONV) g_err = "policy evaluation did not reach the target";
  return st.status;
}

int policy_eval_gmres(mdp_t h, const int32_t* pi, const double* v0, double target_inf,
                      const mdp_opts* opts, double* v_out, mdp_stats* stats) {
  // host pointers: cudaMemcpyDefault handles them through the same path
  return policy_eval_gmres_dev(h, pi, v0, target_inf, opts, v_out, stats);
}

// Coarse inverse of the two-level preconditioner for a given policy, copied to the host: the
// same band build, GTH-form LU and explicit FP32 inverse that ipi_solve runs once per policy.
int mdp_precond_coarse_inverse(mdp_t h, const int32_t* pi, int32_t block, float* inv_out,
                               int64_t* nc_out, int32_t* bw_out) {
  if (h && h->vpending) RK(finish_upload(h));
  g_err.clear();
  if (!h || !pi) return fail(MDP_EINVAL, "null handle or policy");
  if (h->d.kind != KIND_ELL) return fail(MDP_EINVAL, "the two-level preconditioner needs ELL data");
  if (block < 2 || (block & (block - 1)) != 0 || (int64_t)block > h->d.S)
    return fail(MDP_EINVAL, "block must be a power of two in [2, S]");
  const int kt = h->d.pdt == MDP_F32 ? 1 : 0;
  RK(ensure_ws(h, kt, 1));
  RK(ensure_pc(h, kt, 1, log2_exact(block)));
  Workspace& w = h->ws;
  auto& p = h->pc;
  CK(cudaMemcpyAsync(w.pi2, pi, (size_t)h->d.S * 4, cudaMemcpyDefault, h->stream));
  CK(cudaMemsetAsync(w.flags, 0, 64, h->stream));
  RK(launch_check_policy(w.pi2, h->d.S, h->d.A, h->d.mask, w.flags, h->stream));
  int hf[16] = {0};
  CK(cudaMemcpyAsync(hf, w.flags, 64, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  if (hf[5]) return fail(MDP_EINVAL, "policy entry out of range or not an allowed action");
  RK(launch_coarse_setup(h->d, w.pi2, pck(h), p.bw,
                         PrecondScratch{p.band, p.cl, p.cu, p.dinv}, h->stream));
  if (inv_out)
    CK(cudaMemcpy2DAsync(inv_out, (size_t)p.nc * 4, p.inv, (size_t)p.ldc * 4, (size_t)p.nc * 4,
                         (size_t)p.nc, cudaMemcpyDeviceToHost, h->stream));
  CK(cudaStreamSynchronize(h->stream));
  RK(check_device_error(h));
  if (nc_out) *nc_out = p.nc;
  if (bw_out) *bw_out = p.bw;
  return MDP_OK;
}

#define SOLVER(name, method)                                                            \
  int name##_dev(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out,         \
                 mdp_stats* stats) {                                                    \
    g_err.clear();                                                                      \
    mdp_opts o = normalise(opts);                                                       \
    RK(check_opts(h, o));                                                               \
    RK(finish_upload(h));                                                               \
    if (!v_out) return fail(MDP_EINVAL, "null v_out");                                  \
    if (method == METH_OPI && o.opi_W < 1) return fail(MDP_EINVAL, "opi_W must be >= 1");  \
    if (method != METH_IPI && o.precond_block != 0)                                     \
      return fail(MDP_EINVAL, "precond_block applies to ipi_solve only");               \
    PcGuard guard{h};                                                                   \
    h->no_window = (o.flags & MDP_FLAG_NO_WINDOW) != 0;                                 \
    if (method == METH_IPI) return run_ipi(h, o, v_out, pi_out, stats);                 \
    return run_solver(h, method, o, v_out, pi_out, stats);                              \
  }                                                                                     \
  int name(mdp_t h, const mdp_opts* opts, double* v_out, int32_t* pi_out, mdp_stats* stats) { \
    return name##_dev(h, opts, v_out, pi_out, stats);                                   \
  }

SOLVER(ipi_solve, METH_IPI)
SOLVER(vi_solve, METH_VI)
SOLVER(pi_solve, METH_PI)
SOLVER(opi_solve, METH_OPI)
SOLVER(ipi_vi_solve, METH_IPI_VI)

}  // extern "C"
