// Two-level preconditioner for the inexact policy evaluation (right preconditioning of the
// GMRES solve of J^pi delta = r, J^pi = I - gamma P^pi; the paper names preconditioning as
// future work in Sec. 5).
//
// States are aggregated into consecutive blocks of b = 2^lb states; R averages a vector over
// each block and Pr copies a block value to its states (R Pr = I).  The coarse operator is the
// Galerkin product J_c = R J^pi Pr = I - gamma P_c, P_c row-stochastic, so J_c is a strictly
// diagonally dominant M-matrix that factors without pivoting.  For transitions that stay within
// +-bw blocks J_c is banded.  Once per outer iteration (the policy is fixed): build the band,
// factor it (banded LU, one block), and form J_c^{-1} explicitly in FP32 (one warp per row,
// solving J_c^T z = e_i with the transposed factors), so that applying the coarse correction in
// an Arnoldi step is a small dense matvec instead of a sequential triangular solve.  Per step:
// restrict (write Q_i and its block means), coarse apply (E_i = J_c^{-1} R Q_i), prolong
// (z = Q_i + Pr E_i, the vector the matvec multiplies).  The candidate iterate adds
// Pr (sum_j y_j E_j), so M^{-1} is never applied to it separately.
#include "mdp_internal.cuh"

#include <algorithm>

namespace mdp {

namespace {

constexpr int PC_THREADS = 256;

// Largest |block(col) - block(s)| over every ELL entry of every action (atomicMax).
template <class PT>
__global__ void coarse_bandwidth_kernel(DevMDP d, int lb, int* bw) {
  int m = 0;
  const int64_t n = d.S * d.A * (int64_t)d.kp;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / ((int64_t)d.A * d.kp);
    const int j = (int)(e % d.kp);
    if (j >= d.k) continue;
    const int dlt = (int)((d.col[e] >> lb) - (s >> lb));
    m = max(m, dlt < 0 ? -dlt : dlt);
  }
  m = warp_max(m);
  if ((threadIdx.x & 31) == 0 && m > 0) atomicMax(bw, m);
}

// Band of J_c for coarse row I (one block per coarse row):
// band[I][t], t = J - I + bw, = delta_{t,bw} - gamma / |I| * sum_{s in I} sum_{c in J} p(s, c).
// Offsets are summed 8 at a time, each thread over its states in a fixed order and the block
// by fixed-order reductions, so the band is the same on every run.
template <class PT>
__global__ void __launch_bounds__(PC_THREADS) coarse_build_kernel(DevMDP d, const int32_t* pi, int lb,
                                                                  int bw, double* band) {
  __shared__ double red[PC_THREADS / 32][8];
  const int W = 2 * bw + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t I = blockIdx.x;
  const int64_t s0 = I << lb;
  const int64_t cnt = min((int64_t)1 << lb, d.S - s0);
  const PT* val = (const PT*)d.P;
  for (int t0 = 0; t0 < W; t0 += 8) {
    double part[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) part[q] = 0.0;
    for (int64_t u = threadIdx.x; u < cnt; u += blockDim.x) {
      const int64_t s = s0 + u;
      const int64_t base = (s * d.A + pi[s]) * d.kp;
      for (int j = 0; j < d.k; ++j) {
        const int t = (int)((d.col[base + j] >> lb) - I) + bw - t0;
        const double x = (double)val[base + j];
#pragma unroll
        for (int q = 0; q < 8; ++q) part[q] += (t == q) ? x : 0.0;
      }
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const double x = warp_sum(part[q]);
      if (lane == 0) red[wid][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < 8 && t0 + (int)threadIdx.x < W) {
      double acc = 0.0;
      for (int w = 0; w < PC_THREADS / 32; ++w) acc += red[w][threadIdx.x];
      const int t = t0 + threadIdx.x;
      band[I * W + t] = (t == bw ? 1.0 : 0.0) - d.gamma * acc / (double)cnt;
    }
    __syncthreads();
  }
}

// In-place banded LU without pivoting (unit lower L below the diagonal, U on and above);
// band[i][j - i + bw] holds A[i][j] and no fill leaves the band.  One block; rows k..k+bw live
// in a shared-memory ring while pivot k is eliminated, and row k is written back when done.
__global__ void __launch_bounds__(PC_THREADS) coarse_lu_kernel(double* band, int nc, int bw) {
  extern __shared__ double win[];
  const int W = 2 * bw + 1, R = bw + 1;
  for (int e = threadIdx.x; e < R * W; e += blockDim.x) {
    const int r = e / W;
    if (r < nc) win[e] = band[(int64_t)r * W + e % W];
  }
  __syncthreads();
  for (int k = 0; k < nc; ++k) {
    const int m = min(bw, nc - 1 - k);  // rows / columns of the trailing window
    double* rk = win + (k % R) * W;
    const double piv = rk[bw];
    for (int r = threadIdx.x; r < m; r += blockDim.x) win[((k + 1 + r) % R) * W + (bw - 1 - r)] /= piv;
    __syncthreads();
    for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
      const int i = k + 1 + e / m, j = k + 1 + e % m;
      double* ri = win + (i % R) * W;
      ri[j - i + bw] -= ri[k - i + bw] * rk[j - k + bw];
    }
    __syncthreads();
    for (int t = threadIdx.x; t < W; t += blockDim.x) {
      band[(int64_t)k * W + t] = rk[t];
      if (k + R < nc) rk[t] = band[(int64_t)(k + R) * W + t];
    }
    __syncthreads();
  }
}

// Row i of J_c^{-1} is z^T with J_c^T z = e_i; J_c^T = U^T L^T, so first U^T w = e_i (forward,
// w[k] = 0 for k < i), then L^T z = w (backward).  One warp per row: lane q keeps the value bw
// steps back that band entry q multiplies, so a step is one warp sum and one shuffle.  The
// forward values are kept in FP64 scratch (row i) for the backward pass; z is stored in FP32.
__global__ void __launch_bounds__(PC_THREADS) coarse_inverse_kernel(const double* band, int nc, int bw,
                                                                    float* inv, double* scratch) {
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const int W = 2 * bw + 1;
  for (int64_t ii = wid; ii < nc; ii += nw) {
    const int i = (int)ii;
    double* w = scratch + ii * nc;
    double r = 0.0;  // lane q: w[k - 1 - q]
    for (int k = i; k < nc; ++k) {
      const int j = k - 1 - lane;
      double t = (lane < bw && j >= i) ? band[(int64_t)j * W + (k - j + bw)] * r : 0.0;
      t = warp_sum(t);
      const double nv = ((k == i ? 1.0 : 0.0) - t) / band[(int64_t)k * W + bw];
      r = __shfl_up_sync(0xffffffffu, r, 1);
      if (lane == 0) {
        r = nv;
        w[k] = nv;
      }
    }
    r = 0.0;  // lane q: z[k + 1 + q]
    for (int k = nc - 1; k >= 0; --k) {
      const int j = k + 1 + lane;
      double t = (lane < bw && j < nc) ? band[(int64_t)j * W + (k - j + bw)] * r : 0.0;
      t = warp_sum(t);
      r = __shfl_up_sync(0xffffffffu, r, 1);
      if (lane == 0) {
        const double nv = (k >= i ? w[k] : 0.0) - t;
        r = nv;
        inv[ii * nc + k] = (float)nv;
      }
    }
  }
}

// Arnoldi step (mode STEP): Q_i = x * scale (x = start residual or previous w) and its block
// means f[I] (one block per coarse block).
template <class KT>
__global__ void __launch_bounds__(PC_THREADS) coarse_restrict_kernel(PrecondK p) {
  const GmresCtl* c = p.ctl;
  if (*(volatile const int*)&c->mode != GM_STEP) return;
  const int i = c->i;
  const KT* x = (const KT*)(c->from_rhs ? p.rbuf : ((i - 1) & 1 ? p.w1 : p.w0));
  const KT scale = sizeof(KT) == 4 ? (KT)c->xscalef : (KT)c->xscale;
  KT* q = (KT*)p.Q + (int64_t)i * p.ldq;
  const int64_t I = blockIdx.x;
  const int64_t s0 = I << p.lb;
  const int64_t cnt = min((int64_t)1 << p.lb, p.S - s0);
  double sum = 0.0;
  for (int64_t u = threadIdx.x; u < cnt; u += blockDim.x) {
    const KT qs = x[s0 + u] * scale;
    q[s0 + u] = qs;
    sum += (double)qs;
  }
  __shared__ double red[32];
  sum = block_sum(sum, red);
  if (threadIdx.x == 0) p.f[I] = sum / (double)cnt;
}

// E_i[I] = sum_J J_c^{-1}[I][J] f[J] (one warp per coarse row).
template <class KT>
__global__ void __launch_bounds__(PC_THREADS) coarse_apply_kernel(PrecondK p) {
  const GmresCtl* c = p.ctl;
  if (*(volatile const int*)&c->mode != GM_STEP) return;
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  KT* e = (KT*)p.E + (int64_t)c->i * p.ldc;
  for (int64_t I = wid; I < p.nc; I += nw) {
    const float* row = p.inv + I * (int64_t)p.nc;
    double t = 0.0;
    for (int64_t J = lane; J < p.nc; J += 32) t += (double)__ldg(row + J) * p.f[J];
    t = warp_sum(t);
    if (lane == 0) e[I] = (KT)t;
  }
}

// z = Q_i + Pr E_i (the vector the Arnoldi-step matvec multiplies).
template <class KT>
__global__ void coarse_prolong_kernel(PrecondK p) {
  const GmresCtl* c = p.ctl;
  if (*(volatile const int*)&c->mode != GM_STEP) return;
  const KT* q = (const KT*)p.Q + (int64_t)c->i * p.ldq;
  const KT* e = (const KT*)p.E + (int64_t)c->i * p.ldc;
  KT* z = (KT*)p.z;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < p.S;
       s += (int64_t)gridDim.x * blockDim.x)
    z[s] = q[s] + e[s >> p.lb];
}

// ec[I] = sum_{j <= i} y_j E_j[I]: the coarse part of M^{-1} Q y for the candidate iterate
// (modes EST, RESTART, FINISH, where the estimate kernel forms the candidate).
template <class KT>
__global__ void coarse_combine_kernel(PrecondK p) {
  const GmresCtl* c = p.ctl;
  const int mode = *(volatile const int*)&c->mode;
  if (mode != GM_EST && mode != GM_RESTART && mode != GM_FINISH) return;
  const int m = c->i + 1;
  for (int64_t I = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; I < p.nc;
       I += (int64_t)gridDim.x * blockDim.x) {
    double t = 0.0;
    for (int j = 0; j < m; ++j) t += c->y[j] * (double)((const KT*)p.E)[(int64_t)j * p.ldc + I];
    ((KT*)p.ec)[I] = (KT)t;
  }
}

inline int pc_grid(int64_t n, int per_block) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block,
                                                     (int64_t)num_sms() * 8));
}

inline int ok() { return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE; }

}  // namespace

int launch_coarse_bandwidth(const DevMDP& d, int lb, int* bw, cudaStream_t st) {
  const int64_t n = d.S * d.A * (int64_t)d.kp;
  if (d.pdt == MDP_F32) coarse_bandwidth_kernel<float><<<pc_grid(n, 256), 256, 0, st>>>(d, lb, bw);
  else coarse_bandwidth_kernel<double><<<pc_grid(n, 256), 256, 0, st>>>(d, lb, bw);
  return ok();
}

int launch_coarse_setup(const DevMDP& d, const int32_t* pi, const PrecondK& p, int bw,
                        double* band, double* scratch, cudaStream_t st) {
  if (d.pdt == MDP_F32)
    coarse_build_kernel<float><<<(int)p.nc, PC_THREADS, 0, st>>>(d, pi, p.lb, bw, band);
  else
    coarse_build_kernel<double><<<(int)p.nc, PC_THREADS, 0, st>>>(d, pi, p.lb, bw, band);
  const size_t lu_smem = (size_t)(bw + 1) * (2 * bw + 1) * sizeof(double);
  coarse_lu_kernel<<<1, PC_THREADS, lu_smem, st>>>(band, (int)p.nc, bw);
  const int grid = (int)std::max<int64_t>(1, (p.nc * 32 + PC_THREADS - 1) / PC_THREADS);
  coarse_inverse_kernel<<<grid, PC_THREADS, 0, st>>>(band, (int)p.nc, bw, p.inv, scratch);
  return ok();
}

int launch_coarse_step(const PrecondK& p, int kt, cudaStream_t st) {
  const int gapply = (int)std::min<int64_t>((p.nc * 32 + PC_THREADS - 1) / PC_THREADS,
                                            (int64_t)num_sms() * 8);
  if (kt == 1) {
    coarse_restrict_kernel<float><<<(int)p.nc, PC_THREADS, 0, st>>>(p);
    coarse_apply_kernel<float><<<std::max(1, gapply), PC_THREADS, 0, st>>>(p);
    coarse_prolong_kernel<float><<<pc_grid(p.S, 256), 256, 0, st>>>(p);
  } else {
    coarse_restrict_kernel<double><<<(int)p.nc, PC_THREADS, 0, st>>>(p);
    coarse_apply_kernel<double><<<std::max(1, gapply), PC_THREADS, 0, st>>>(p);
    coarse_prolong_kernel<double><<<pc_grid(p.S, 256), 256, 0, st>>>(p);
  }
  return ok();
}

int launch_coarse_combine(const PrecondK& p, int kt, cudaStream_t st) {
  if (kt == 1) coarse_combine_kernel<float><<<pc_grid(p.nc, 256), 256, 0, st>>>(p);
  else coarse_combine_kernel<double><<<pc_grid(p.nc, 256), 256, 0, st>>>(p);
  return ok();
}

}  // namespace mdp
