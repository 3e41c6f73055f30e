// Row-sharded iGMRES-PI: one MDP whose state rows are split over several GPUs (processes),
// the parallel/distributed form of the method that the paper names as future work (Sec. 5).
//
// Rank r holds rows [row0, row0 + rows) of every P_a and g_a (ELL, global column indices), and
// the matching slices of V, T V, Phi, pi and of the Krylov vectors.  The steps of Alg. 2 need
// three kinds of exchange, all done through caller-supplied host collectives (mdp_comm):
//   * all-gather of a vector whose entries the local rows own (V before a Bellman sweep, the
//     Arnoldi vector Q_i before the P^pi matvec, a candidate iterate before its true residual);
//   * allreduce-max of ||Phi||_inf and of the true residual's inf-norm (stopping rules);
//   * allreduce-sum of ||Phi||_2^2, of the CGS2 projections Q^T w (two passes) and of ||w||_2^2.
// The Hessenberg matrix and its Givens rotations are replicated: every rank applies the same
// FP64 operations to the same reduced values, and each accept / restart decision is also
// agreed by an allreduce-max, so the ranks never take different branches.
//
// Arithmetic: P stored as FP32 or FP64 and every sum accumulated in FP64, one FMA per entry;
// the Krylov basis is FP64.  Kernels: a warp per state for the sweep (lane a forms Q(s, a) over
// the row's k entries, then a warp argmin with the lowest index on ties), a thread per state for
// the P^pi products, block partial sums reduced in a fixed order (no atomics), so a run is
// reproducible and the reduced values are the same on every rank.
#include "mdp_internal.cuh"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <string>
#include <vector>

namespace mdp {
namespace {

constexpr int SH_THREADS = 256;
constexpr int SH_NP = 2 * WMAX + 8;  // partial-sum slots per block
constexpr int SH_MAX_BLOCKS = 1024;

struct ShardView {
  int64_t S, row0, rows;
  int A, k, pdt;
  double gamma;
  const void* val;     // [rows][A][k]
  const int32_t* col;  // [rows][A][k], global columns
  const double* g;     // [rows][A]
};

template <class PT>
__device__ __forceinline__ double row_dot(const ShardView& d, int64_t s, int a, const double* x) {
  const int64_t base = (s * d.A + a) * (int64_t)d.k;
  const PT* val = (const PT*)d.val;
  double acc = 0.0;
  for (int j = 0; j < d.k; ++j) acc = fma((double)val[base + j], x[d.col[base + j]], acc);
  return acc;
}

// Block partials: slot 0 = max of |phi|, slot 1 = sum of phi^2.
template <class PT>
__global__ void __launch_bounds__(SH_THREADS) shard_sweep_kernel(ShardView d, const double* vglob,
                                                                 double* tv, double* phi,
                                                                 int32_t* pi, double* part) {
  __shared__ double shm[32];
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  double mx = 0.0, sq = 0.0;
  for (int64_t s = wid; s < d.rows; s += nw) {
    double best = INFINITY;
    int abest = 0x7fffffff;
    for (int a = lane; a < d.A; a += 32) {
      const double q = fma(d.gamma, row_dot<PT>(d, s, a, vglob), d.g[s * d.A + a]);
      if (q < best) { best = q; abest = a; }  // a grows: the lowest index keeps a tie
    }
#pragma unroll
    for (int off = 16; off > 0; off >>= 1) {
      const double qo = __shfl_xor_sync(0xffffffffu, best, off);
      const int ao = __shfl_xor_sync(0xffffffffu, abest, off);
      if (qo < best || (qo == best && ao < abest)) { best = qo; abest = ao; }
    }
    if (lane == 0) {
      const double f = best - vglob[d.row0 + s];
      tv[s] = best;
      pi[s] = abest;
      phi[s] = f;
      mx = fmax(mx, fabs(f));
      sq = fma(f, f, sq);
    }
  }
  mx = block_max(mx, shm);
  sq = block_sum(sq, shm);
  if (threadIdx.x == 0) {
    part[(int64_t)blockIdx.x * SH_NP + 0] = mx;
    part[(int64_t)blockIdx.x * SH_NP + 1] = sq;
  }
}

// mode 0: w = x_own - gamma P^pi x            (J^pi x, Arnoldi step); slot 0 = sum w^2
// mode 1: w = g^pi - (x_own - gamma P^pi x)   (true residual);        slot 0 = max |w|, 1 = sum w^2
template <class PT>
__global__ void __launch_bounds__(SH_THREADS) shard_matvec_kernel(ShardView d, const int32_t* pi,
                                                                  const double* xglob, double* w,
                                                                  int mode, double* part) {
  __shared__ double shm[32];
  double mx = 0.0, sq = 0.0;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < d.rows;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int a = pi[s];
    const double jx = fma(-d.gamma, row_dot<PT>(d, s, a, xglob), xglob[d.row0 + s]);
    const double y = mode == 0 ? jx : d.g[s * d.A + a] - jx;
    w[s] = y;
    mx = fmax(mx, fabs(y));
    sq = fma(y, y, sq);
  }
  mx = block_max(mx, shm);
  sq = block_sum(sq, shm);
  if (threadIdx.x == 0) {
    part[(int64_t)blockIdx.x * SH_NP + 0] = mode == 0 ? sq : mx;
    part[(int64_t)blockIdx.x * SH_NP + 1] = sq;
  }
}

// Block partials of h_j = Q_j . w for j = 0..m-1.
__global__ void __launch_bounds__(SH_THREADS) shard_dots_kernel(const double* Q, int64_t ldq, int m,
                                                                const double* w, int64_t rows,
                                                                double* part) {
  __shared__ double shm[32];
  for (int j = 0; j < m; ++j) {
    const double* q = Q + (int64_t)j * ldq;
    double t = 0.0;
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < rows;
         s += (int64_t)gridDim.x * blockDim.x)
      t = fma(q[s], w[s], t);
    t = block_sum(t, shm);
    if (threadIdx.x == 0) part[(int64_t)blockIdx.x * SH_NP + j] = t;
  }
}

// out = base + sign * sum_j c_j Q_j (c in device memory); slot 0 = sum out^2.
__global__ void __launch_bounds__(SH_THREADS) shard_combine_kernel(const double* Q, int64_t ldq, int m,
                                                                   const double* c, double sign,
                                                                   const double* base, double* out,
                                                                   int64_t rows, double* part) {
  __shared__ double shm[32];
  double sq = 0.0;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < rows;
       s += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int j = 0; j < m; ++j) t = fma(c[j], Q[(int64_t)j * ldq + s], t);
    const double y = fma(sign, t, base[s]);
    out[s] = y;
    sq = fma(y, y, sq);
  }
  sq = block_sum(sq, shm);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.x * SH_NP] = sq;
}

__global__ void shard_scale_kernel(const double* x, double a, double* y, int64_t rows) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < rows;
       s += (int64_t)gridDim.x * blockDim.x)
    y[s] = a * x[s];
}

// red[j] = sum (or max, for j < nmax) over blocks of part[b][j], in block order.
__global__ void shard_finalize_kernel(const double* part, int nblk, int n, int nmax, double* red) {
  const int j = threadIdx.x;
  if (j >= n) return;
  double t = 0.0;
  for (int b = 0; b < nblk; ++b) {
    const double x = part[(int64_t)b * SH_NP + j];
    t = j < nmax ? fmax(t, x) : t + x;
  }
  red[j] = t;
}

}  // namespace
}  // namespace mdp

using namespace mdp;

struct mdp_shard_s {
  ShardView d{};
  int device = 0;
  cudaStream_t stream = nullptr;
  void* val = nullptr;
  int32_t* col = nullptr;
  double* g = nullptr;
  // workspace (restart length W)
  int W = 0;
  int64_t ldq = 0;
  double *vglob = nullptr, *xglob = nullptr;
  double *v = nullptr, *tv = nullptr, *phi = nullptr, *w = nullptr, *x0 = nullptr, *r = nullptr,
         *cand = nullptr, *Q = nullptr, *part = nullptr, *red = nullptr, *coef = nullptr;
  int32_t* pi = nullptr;
  double *h_loc = nullptr, *h_glob = nullptr, *h_red = nullptr;
  int nblk = 1;
};

namespace {

int sfail(int code, const char* msg) { return set_error(code, msg); }

void shard_free_ws(mdp_shard_t h) {
  void* dev[] = {h->vglob, h->xglob, h->v, h->tv, h->phi, h->w, h->x0, h->r, h->cand, h->Q,
                 h->part, h->red, h->coef, h->pi};
  for (void* p : dev)
    if (p) cudaFree(p);
  void* host[] = {h->h_loc, h->h_glob, h->h_red};
  for (void* p : host)
    if (p) cudaFreeHost(p);
  h->vglob = h->xglob = h->v = h->tv = h->phi = h->w = h->x0 = h->r = h->cand = h->Q = nullptr;
  h->part = h->red = h->coef = nullptr;
  h->pi = nullptr;
  h->h_loc = h->h_glob = h->h_red = nullptr;
  h->W = 0;
}

int shard_ensure_ws(mdp_shard_t h, int W) {
  if (h->W >= W) return MDP_OK;
  shard_free_ws(h);
  const int64_t S = h->d.S, n = std::max<int64_t>(h->d.rows, 1);
  h->ldq = (n + 31) / 32 * 32;
  bool ok = true;
  auto dal = [&](void** p, size_t bytes) {
    if (ok && cudaMalloc(p, bytes) != cudaSuccess) ok = false;
    if (ok) cudaMemsetAsync(*p, 0, bytes, h->stream);
  };
  dal((void**)&h->vglob, (size_t)S * 8);
  dal((void**)&h->xglob, (size_t)S * 8);
  for (double** p : {&h->v, &h->tv, &h->phi, &h->w, &h->x0, &h->r, &h->cand})
    dal((void**)p, (size_t)h->ldq * 8);
  dal((void**)&h->Q, (size_t)(W + 1) * h->ldq * 8);
  dal((void**)&h->part, (size_t)SH_MAX_BLOCKS * SH_NP * 8);
  dal((void**)&h->red, (size_t)SH_NP * 8);
  dal((void**)&h->coef, (size_t)SH_NP * 8);
  dal((void**)&h->pi, (size_t)h->ldq * 4);
  if (ok && (cudaMallocHost((void**)&h->h_loc, (size_t)n * 8) != cudaSuccess ||
             cudaMallocHost((void**)&h->h_glob, (size_t)S * 8) != cudaSuccess ||
             cudaMallocHost((void**)&h->h_red, (size_t)SH_NP * 8) != cudaSuccess))
    ok = false;
  if (!ok) {
    shard_free_ws(h);
    return sfail(MDP_ENOMEM, "shard workspace allocation failed");
  }
  h->W = W;
  h->nblk = (int)std::max<int64_t>(1, std::min<int64_t>((h->d.rows + SH_THREADS - 1) / SH_THREADS,
                                                        (int64_t)std::min(num_sms() * 4, SH_MAX_BLOCKS)));
  return MDP_OK;
}

#define SK(x)                                                                       \
  do {                                                                              \
    const cudaError_t e_ = (x);                                                     \
    if (e_ != cudaSuccess) return sfail(MDP_EDEVICE, cudaGetErrorString(e_));       \
  } while (0)
#define SR(x)                    \
  do {                           \
    const int r_ = (x);          \
    if (r_ != MDP_OK) return r_; \
  } while (0)

// Reduced values of the last kernel's block partials to the host: n slots, the first nmax by max.
int reduce_local(mdp_shard_t h, int nblk, int n, int nmax, double* out) {
  shard_finalize_kernel<<<1, 32 * ((n + 31) / 32), 0, h->stream>>>(h->part, nblk, n, nmax, h->red);
  SK(cudaGetLastError());
  SK(cudaMemcpyAsync(h->h_red, h->red, (size_t)n * 8, cudaMemcpyDeviceToHost, h->stream));
  SK(cudaStreamSynchronize(h->stream));
  for (int j = 0; j < n; ++j) out[j] = h->h_red[j];
  return MDP_OK;
}

struct Exchange {
  const mdp_comm* c;
  mdp_shard_t h;
  // global[S] (device) <- every rank's rows of local (device)
  int allgather(const double* local, double* global) {
    SK(cudaMemcpyAsync(h->h_loc, local, (size_t)h->d.rows * 8, cudaMemcpyDeviceToHost, h->stream));
    SK(cudaStreamSynchronize(h->stream));
    if (c->allgather(c->ctx, h->h_loc, h->h_glob, 8) != 0)
      return sfail(MDP_EDEVICE, "mdp_comm.allgather failed");
    SK(cudaMemcpyAsync(global, h->h_glob, (size_t)h->d.S * 8, cudaMemcpyHostToDevice, h->stream));
    return MDP_OK;
  }
  int allreduce(double* vals, int n, int op) {
    if (c->allreduce(c->ctx, vals, n, op) != 0) return sfail(MDP_EDEVICE, "mdp_comm.allreduce failed");
    return MDP_OK;
  }
  // every rank takes the largest decision code
  int agree(int* code) {
    double x = (double)*code;
    SR(allreduce(&x, 1, 1));
    *code = (int)x;
    return MDP_OK;
  }
};

template <class PT>
int shard_launch_sweep(mdp_shard_t h) {
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((h->d.rows + 7) / 8, h->nblk));
  shard_sweep_kernel<PT><<<grid, SH_THREADS, 0, h->stream>>>(h->d, h->vglob, h->tv, h->phi, h->pi, h->part);
  SK(cudaGetLastError());
  return grid;
}
template <class PT>
int shard_launch_matvec(mdp_shard_t h, const double* xglob, double* out, int mode) {
  shard_matvec_kernel<PT><<<h->nblk, SH_THREADS, 0, h->stream>>>(h->d, h->pi, xglob, out, mode, h->part);
  SK(cudaGetLastError());
  return MDP_OK;
}

// One Bellman sweep at V (allgathered): pi, T V, Phi and the global ||Phi||_inf, ||Phi||_2.
template <class PT>
int shard_bellman(mdp_shard_t h, Exchange& ex, double* res_inf, double* res_nrm2) {
  SR(ex.allgather(h->v, h->vglob));
  const int grid = shard_launch_sweep<PT>(h);
  if (grid < 0) return grid;
  double loc[2];
  SR(reduce_local(h, grid, 2, 1, loc));
  double mx = loc[0], sq = loc[1];
  SR(ex.allreduce(&mx, 1, 1));
  SR(ex.allreduce(&sq, 1, 0));
  *res_inf = mx;
  *res_nrm2 = sqrt(sq);
  return MDP_OK;
}

// The inner loop of Alg. 2 for pi_k: restarted GMRES(W) on J^pi delta = Phi_k in correction
// form (the iterate is x0 + Q y), CGS2 orthogonalisation, Givens rotations on the replicated
// Hessenberg matrix.  The true inf-norm residual is formed (all-gather, matvec, allreduce-max)
// when the Givens estimate ||r||_2 (an upper bound of ||r||_inf) comes within sqrt(S) of the
// threshold, at the end of a cycle, at a breakdown and at the step cap; the solve ends when it
// meets the threshold (or at a breakdown or the cap).  Leaves V_{k+1} in h->v.
template <class PT>
int shard_inner(mdp_shard_t h, Exchange& ex, double beta, double thr, int W, int max_steps,
                mdp_stats& st) {
  const int64_t n = h->d.rows;
  const double sqrtS = sqrt((double)h->d.S);
  const int g1 = h->nblk;
  std::vector<double> H((size_t)(W + 1) * W), cs(W), sn(W), gv(W + 1), y(W), hv(W + 1), h2(W + 1);
  SK(cudaMemcpyAsync(h->x0, h->v, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->stream));
  SK(cudaMemcpyAsync(h->r, h->phi, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->stream));
  int steps = 0;
  while (true) {  // one restart cycle
    if (!(beta > 0.0)) {  // the base solves the system exactly
      SK(cudaMemcpyAsync(h->v, h->x0, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->stream));
      return MDP_OK;
    }
    shard_scale_kernel<<<g1, SH_THREADS, 0, h->stream>>>(h->r, 1.0 / beta, h->Q, n);
    std::fill(H.begin(), H.end(), 0.0);
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    for (int i = 0; i < W; ++i) {
      double* qi = h->Q + (int64_t)i * h->ldq;
      // w = J^pi Q_i, with ||J^pi Q_i||_2 as the breakdown reference
      SR(ex.allgather(qi, h->xglob));
      SR(shard_launch_matvec<PT>(h, h->xglob, h->w, 0));
      double jq2;
      SR(reduce_local(h, g1, 1, 0, &jq2));
      SR(ex.allreduce(&jq2, 1, 0));
      // CGS2: two projections on Q_0..Q_i, then ||w||_2
      const int m = i + 1;
      for (int pass = 0; pass < 2; ++pass) {
        double* hp = pass ? h2.data() : hv.data();
        shard_dots_kernel<<<g1, SH_THREADS, 0, h->stream>>>(h->Q, h->ldq, m, h->w, n, h->part);
        SK(cudaGetLastError());
        SR(reduce_local(h, g1, m, 0, hp));
        SR(ex.allreduce(hp, m, 0));
        SK(cudaMemcpyAsync(h->coef, hp, (size_t)m * 8, cudaMemcpyHostToDevice, h->stream));
        shard_combine_kernel<<<g1, SH_THREADS, 0, h->stream>>>(h->Q, h->ldq, m, h->coef, -1.0, h->w,
                                                               h->w, n, h->part);
        SK(cudaGetLastError());
      }
      double wn2;
      SR(reduce_local(h, g1, 1, 0, &wn2));
      SR(ex.allreduce(&wn2, 1, 0));
      const double hnext = sqrt(wn2);
      for (int j = 0; j < m; ++j) H[(size_t)j * W + i] = hv[j] + h2[j];
      H[(size_t)m * W + i] = hnext;
      // Givens rotations (replicated): previous ones on column i, then a new one
      for (int j = 0; j < i; ++j) {
        const double a = H[(size_t)j * W + i], b = H[(size_t)(j + 1) * W + i];
        H[(size_t)j * W + i] = cs[j] * a + sn[j] * b;
        H[(size_t)(j + 1) * W + i] = -sn[j] * a + cs[j] * b;
      }
      const double a = H[(size_t)i * W + i], b = H[(size_t)m * W + i];
      const double rr = hypot(a, b);
      cs[i] = rr > 0.0 ? a / rr : 1.0;
      sn[i] = rr > 0.0 ? b / rr : 0.0;
      H[(size_t)i * W + i] = rr;
      H[(size_t)m * W + i] = 0.0;
      gv[m] = -sn[i] * gv[i];
      gv[i] = cs[i] * gv[i];
      ++steps;
      st.inner += 1;
      st.matvecs += 1;
      const bool breakdown = !(hnext > 1e-14 * sqrt(jq2));
      if (!breakdown)
        shard_scale_kernel<<<g1, SH_THREADS, 0, h->stream>>>(h->w, 1.0 / hnext,
                                                             h->Q + (int64_t)m * h->ldq, n);
      const bool cap = steps >= max_steps;
      const double est = fabs(gv[m]);
      if (!(breakdown || cap || i == W - 1 || est <= sqrtS * thr)) continue;
      // candidate x0 + Q y (y from the triangular system of the rotated Hessenberg matrix)
      for (int r = m - 1; r >= 0; --r) {
        double t = gv[r];
        for (int c2 = r + 1; c2 < m; ++c2) t -= H[(size_t)r * W + c2] * y[c2];
        y[r] = t / H[(size_t)r * W + r];
      }
      SK(cudaMemcpyAsync(h->coef, y.data(), (size_t)m * 8, cudaMemcpyHostToDevice, h->stream));
      shard_combine_kernel<<<g1, SH_THREADS, 0, h->stream>>>(h->Q, h->ldq, m, h->coef, 1.0, h->x0,
                                                             h->cand, n, h->part);
      SK(cudaGetLastError());
      SR(ex.allgather(h->cand, h->xglob));
      SR(shard_launch_matvec<PT>(h, h->xglob, h->r, 1));
      st.matvecs += 1;
      double rl[2];
      SR(reduce_local(h, g1, 2, 1, rl));
      double rmax = rl[0], rsq = rl[1];
      SR(ex.allreduce(&rmax, 1, 1));
      SR(ex.allreduce(&rsq, 1, 0));
      // 2 = accept (residual met, breakdown or cap), 1 = restart, 0 = continue the cycle
      int code = (!(rmax > thr) || breakdown || cap) ? 2 : (i == W - 1 ? 1 : 0);
      SR(ex.agree(&code));
      if (breakdown) st.breakdowns += 1;
      if (code == 2) {
        SK(cudaMemcpyAsync(h->v, h->cand, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->stream));
        return MDP_OK;
      }
      if (code == 1) {  // restart from the candidate and its true residual
        SK(cudaMemcpyAsync(h->x0, h->cand, (size_t)n * 8, cudaMemcpyDeviceToDevice, h->stream));
        beta = sqrt(rsq);
        st.restarts += 1;
        break;
      }
    }
  }
}

template <class PT>
int shard_ipi(mdp_shard_t h, const mdp_comm* comm, const mdp_opts& o, double* v_out,
              int32_t* pi_out, mdp_stats* st_user) {
  mdp_stats st{};
  const auto t0 = std::chrono::steady_clock::now();
  SR(shard_ensure_ws(h, o.restart));
  const int64_t n = h->d.rows;
  Exchange ex{comm, h};
  if (o.v0) SK(cudaMemcpyAsync(h->v, o.v0, (size_t)n * 8, cudaMemcpyDefault, h->stream));
  else SK(cudaMemsetAsync(h->v, 0, (size_t)n * 8, h->stream));
  int status = MDP_ENOCONV;
  double res = 0.0, nrm2 = 0.0;
  for (int k = 0;; ++k) {
    SR(shard_bellman<PT>(h, ex, &res, &nrm2));
    st.sweeps += 1;
    if (res <= o.tol) { status = MDP_OK; break; }
    if (k >= o.max_outer) break;
    const double thr = inexact_threshold(o.alpha, o.forcing_c, res, 0.1 * o.tol);
    SR(shard_inner<PT>(h, ex, nrm2, thr, o.restart, o.max_inner, st));
    st.outer += 1;
  }
  SK(cudaMemcpyAsync(v_out, h->tv, (size_t)n * 8, cudaMemcpyDefault, h->stream));
  if (pi_out) SK(cudaMemcpyAsync(pi_out, h->pi, (size_t)n * 4, cudaMemcpyDefault, h->stream));
  SK(cudaStreamSynchronize(h->stream));
  st.residual_inf = res;
  st.status = status;
  st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (st_user) *st_user = st;
  if (status != MDP_OK) set_error(status, "iteration cap reached before ||T(v)-v||_inf <= tol");
  return status;
}

}  // namespace

extern "C" {

int mdp_shard_create(int64_t S, int64_t row0, int64_t rows, int32_t A, int32_t k, const int32_t* col,
                     const void* val, int val_dtype, const double* g, double gamma,
                     mdp_shard_t* out) {
  if (!out) return sfail(MDP_EINVAL, "null output handle");
  *out = nullptr;
  if (S < 1 || row0 < 0 || rows < 1 || row0 + rows > S || A < 1 || k < 1 || (int64_t)k > S)
    return sfail(MDP_EINVAL, "bad sizes: need 1 <= rows, row0 + rows <= S, 1 <= k <= S, A >= 1");
  if (!(gamma > 0.0 && gamma < 1.0)) return sfail(MDP_EINVAL, "gamma must lie in (0, 1)");
  if (!col || !val || !g) return sfail(MDP_EINVAL, "null input array");
  if (val_dtype != MDP_F32 && val_dtype != MDP_F64) return sfail(MDP_EINVAL, "bad value dtype");
  const size_t eb = val_dtype == MDP_F32 ? 4 : 8;
  // host validation and transposition [A][rows][k] -> [rows][A][k]
  const int64_t nnz = rows * A * (int64_t)k;
  std::vector<int32_t> ct((size_t)nnz);
  std::vector<unsigned char> vt((size_t)nnz * eb);
  std::vector<double> gt((size_t)rows * A);
  for (int a = 0; a < A; ++a)
    for (int64_t s = 0; s < rows; ++s) {
      double sum = 0.0;
      const int64_t src = ((int64_t)a * rows + s) * k, dst = (s * A + a) * (int64_t)k;
      for (int j = 0; j < k; ++j) {
        const int32_t c = col[src + j];
        const double x = val_dtype == MDP_F32 ? (double)((const float*)val)[src + j]
                                              : ((const double*)val)[src + j];
        if (c < 0 || (int64_t)c >= S) return sfail(MDP_EINVAL, "column index out of range");
        if (!(x >= 0.0) || !std::isfinite(x)) return sfail(MDP_EINVAL, "negative or non-finite probability");
        sum += x;
        ct[(size_t)(dst + j)] = c;
        memcpy(&vt[(size_t)(dst + j) * eb], (const unsigned char*)val + (size_t)(src + j) * eb, eb);
      }
      if (!(fabs(sum - 1.0) <= 1e-5)) return sfail(MDP_EINVAL, "row does not sum to 1");
      const double gv = g[(int64_t)a * rows + s];
      if (!std::isfinite(gv)) return sfail(MDP_EINVAL, "non-finite cost");
      gt[(size_t)(s * A + a)] = gv;
    }
  mdp_shard_t h = new mdp_shard_s();
  cudaGetDevice(&h->device);
  auto bail = [&](int code, const char* msg) {
    mdp_shard_destroy(h);
    return sfail(code, msg);
  };
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess)
    return bail(MDP_EDEVICE, "stream creation failed");
  if (cudaMalloc(&h->val, (size_t)nnz * eb) != cudaSuccess ||
      cudaMalloc((void**)&h->col, (size_t)nnz * 4) != cudaSuccess ||
      cudaMalloc((void**)&h->g, (size_t)rows * A * 8) != cudaSuccess)
    return bail(MDP_ENOMEM, "shard data allocation failed");
  if (cudaMemcpy(h->val, vt.data(), (size_t)nnz * eb, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->col, ct.data(), (size_t)nnz * 4, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(h->g, gt.data(), (size_t)rows * A * 8, cudaMemcpyHostToDevice) != cudaSuccess)
    return bail(MDP_EDEVICE, "shard upload failed");
  h->d = ShardView{S, row0, rows, A, k, val_dtype, gamma, h->val, h->col, h->g};
  *out = h;
  return MDP_OK;
}

void mdp_shard_destroy(mdp_shard_t h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  shard_free_ws(h);
  if (h->val) cudaFree(h->val);
  if (h->col) cudaFree(h->col);
  if (h->g) cudaFree(h->g);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int ipi_solve_sharded(mdp_shard_t h, const mdp_comm* comm, const mdp_opts* opts, double* v_out,
                      int32_t* pi_out, mdp_stats* stats) {
  if (!h || !comm || !v_out || !comm->allgather || !comm->allreduce || !comm->row_begin)
    return sfail(MDP_EINVAL, "null shard, communicator, callback or output");
  if (comm->world < 1 || comm->rank < 0 || comm->rank >= comm->world ||
      comm->row_begin[0] != 0 || comm->row_begin[comm->world] != h->d.S ||
      comm->row_begin[comm->rank] != h->d.row0 ||
      comm->row_begin[comm->rank + 1] - comm->row_begin[comm->rank] != h->d.rows)
    return sfail(MDP_EINVAL, "the communicator's row partition does not match the shard");
  const mdp_opts o = opts ? *opts : mdp_opts_default();
  if (!(o.alpha > 0.0 && o.alpha < 1.0) || !(o.tol > 0.0) || o.restart < 1 || o.restart > WMAX ||
      o.max_outer < 0 || o.max_inner < 1 || o.precond_block != 0)
    return sfail(MDP_EINVAL, "bad options (0 < alpha < 1, tol > 0, 1 <= restart <= 64, no precond_block)");
  cudaSetDevice(h->device);
  return h->d.pdt == MDP_F32 ? shard_ipi<float>(h, comm, o, v_out, pi_out, stats)
                             : shard_ipi<double>(h, comm, o, v_out, pi_out, stats);
}

}  // extern "C"
