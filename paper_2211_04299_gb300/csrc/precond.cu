// Two-level preconditioner for the inexact policy evaluation (right preconditioning of the
// GMRES solve of J^pi delta = r, J^pi = I - gamma P^pi; the paper names preconditioning as
// future work in Sec. 5).
//
// States are aggregated into consecutive blocks of b = 2^lb states; R averages a vector over
// each block and Pr copies a block value to its states (R Pr = I).  The coarse operator is the
// Galerkin product J_c = R J^pi Pr = I - gamma P_c, P_c row-stochastic, so J_c is a strictly
// diagonally dominant M-matrix that factors without pivoting.  For transitions that stay within
// +-bw blocks J_c is banded.  Once per outer iteration (the policy is fixed): build the band,
// factor it (banded LU in FP64, one block), and form J_c^{-1} explicitly in FP32 (one warp per
// row, solving J_c^T z = e_i with the transposed factors), so that the coarse correction in an
// Arnoldi step is a small dense matvec instead of a sequential triangular solve.  Per step:
// restrict (write Q_i and its block means), coarse apply (E_i = J_c^{-1} R Q_i), prolong
// (z = Q_i + Pr E_i, the vector the matvec multiplies).  The candidate iterate adds
// Pr (sum_j y_j E_j), the same E_j the Arnoldi process used, so the accuracy of J_c^{-1} only
// sets how fast the solve converges, never what it converges to.
//
// Precision: the band and its LU are FP64 (the pivots of a nearly singular J_c come from
// cancellation); the triangular solves of the inverse run in FP32, where the M-matrix factors
// give sums of terms of one sign.  Per-step work is FP32: FP64 throughput is low on this part.
#include "mdp_internal.cuh"

#include <algorithm>

namespace mdp {

namespace {

constexpr int PC_THREADS = 256;
constexpr int LU_CHUNK = 32;  // rows per cp.async-staged chunk of the banded LU

__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_ahead() {  // all but the newest LU1_AHEAD - 1 groups
  asm volatile("cp.async.wait_group 7;" ::: "memory");
}

// Largest |block(col) - block(s)| over every ELL entry of every action (atomicMax).
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

// Row I of the coarse operator (one block per coarse row), stored as Wp = 2 bw + 2 floats:
//   band[I][t], t = J - I + bw < W:  J_c[I][J] = delta_{IJ} - gamma / |I| * sum_{s in I} sum_{c in J} p(s, c)
//   band[I][W]:      s_I = row sum of J_c = (1 - gamma) + gamma * mean_{s in I} (1 - sum_c p(s, c))
// (the LU forms each pivot from s_I and the row's final upper entries, never from the diagonal).
// The row sum is formed from each state's deficit 1 - sum_c p(s, c) (compensated sum), not by
// cancelling 1 against the row's entries.  A team of PC_TEAM lanes reads one state's row (16-byte
// loads, as the matvec does); offsets are summed 8 at a time, each lane over its entries in a
// fixed order, each warp by a fixed shuffle tree, the warps in FP64 in a fixed order, so the
// row is the same on every run.
constexpr int PC_TEAM = 8;
template <class PT>
__global__ void __launch_bounds__(PC_THREADS) coarse_build_kernel(DevMDP d, const int32_t* pi, int lb,
                                                                  int bw, float* band) {
  __shared__ float red[PC_THREADS / 32][9];
  const int W = 2 * bw + 1, Wp = W + 1;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int team = threadIdx.x / PC_TEAM, tl = threadIdx.x % PC_TEAM;
  const int nteams = PC_THREADS / PC_TEAM;
  const int64_t I = blockIdx.x;
  const int64_t s0 = I << lb;
  const int64_t cnt = min((int64_t)1 << lb, d.S - s0);
  const PT* val = (const PT*)d.P;
  const int nvec = d.kp >> 2;
  for (int t0 = 0; t0 < W; t0 += 8) {
    float part[9];  // 8 offsets, and the states' deficits in the first pass
#pragma unroll
    for (int q = 0; q < 9; ++q) part[q] = 0.f;
    for (int64_t ub = 0; ub < cnt; ub += nteams) {  // uniform trip count: shuffles below
      const int64_t u = ub + team;
      const bool act = u < cnt;
      float sh = 0.f, sl = 0.f;  // sum_c p(s, c) over this lane's entries (TwoSum cascade)
      double s64 = 0.0;
      if (act) {
        const int64_t s = s0 + u;
        const int64_t base = (s * d.A + pi[s]) * d.kp;
        for (int q4 = tl; q4 < nvec; q4 += PC_TEAM) {
          const int4 c4 = *reinterpret_cast<const int4*>(d.col + base + 4 * q4);
          PT v[4];
          if constexpr (sizeof(PT) == 4) {
            const float4 x = *reinterpret_cast<const float4*>(val + base + 4 * q4);
            v[0] = x.x; v[1] = x.y; v[2] = x.z; v[3] = x.w;
          } else {
            const double2 x0 = *reinterpret_cast<const double2*>(val + base + 4 * q4);
            const double2 x1 = *(reinterpret_cast<const double2*>(val + base + 4 * q4) + 1);
            v[0] = x0.x; v[1] = x0.y; v[2] = x1.x; v[3] = x1.y;
          }
          const int cc[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int t = (int)((cc[e] >> lb) - I) + bw - t0;
            const float x = (float)v[e];
#pragma unroll
            for (int q = 0; q < 8; ++q) part[q] += (t == q) ? x : 0.f;
            if (t0 == 0) {
              if constexpr (sizeof(PT) == 8) {
                s64 += v[e];
              } else {
                const dfl ts = two_sum(sh, x);
                sh = ts.hi;
                sl += ts.lo;
              }
            }
          }
        }
      }
      if (t0 == 0) {  // the team's row sum, then the state's deficit 1 - sum
#pragma unroll
        for (int o = PC_TEAM / 2; o > 0; o >>= 1) {
          if constexpr (sizeof(PT) == 8) {
            s64 += __shfl_xor_sync(0xffffffffu, s64, o);
          } else {
            const float h2 = __shfl_xor_sync(0xffffffffu, sh, o);
            const float l2 = __shfl_xor_sync(0xffffffffu, sl, o);
            const dfl ts = two_sum(sh, h2);
            sh = ts.hi;
            sl = sl + l2 + ts.lo;
          }
        }
        if (act && tl == 0) {
          if constexpr (sizeof(PT) == 8) {
            part[8] += (float)(1.0 - s64);
          } else {
            const dfl ts = two_sum(1.f, -sh);
            part[8] += ts.hi + (ts.lo - sl);
          }
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      const float x = warp_sum(part[q]);
      if (lane == 0) red[wid][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < 9) {
      const int q = threadIdx.x, t = t0 + q;
      double acc = 0.0;
      for (int w = 0; w < PC_THREADS / 32; ++w) acc += (double)red[w][q];
      if (q < 8 && t < W) band[I * Wp + t] = (float)((t == bw ? 1.0 : 0.0) - d.gamma * acc / (double)cnt);
      if (q == 8 && t0 == 0)
        band[I * Wp + W] = (float)((1.0 - d.gamma) + d.gamma * acc / (double)cnt);
    }
    __syncthreads();
  }
}

// In-place banded LU without pivoting (unit lower L below the diagonal, U on and above) of the
// M-matrix J_c, in the manner of Grassmann, Taksar and Heyman: every row carries its row sum s
// over the Schur complement, and the pivot is formed as u_kk = s_k + sum_{j>k} |u_kj| (the
// magnitudes of the row's final upper entries), so every quantity is a sum of terms of one sign
// and FP32 keeps its relative accuracy however close J_c is to singular.  Eliminating pivot k,
// for the rows i = k+1..k+bw:  l_ik = S_ik / u_kk,  s_i += |l_ik| s_k,  S_ij -= l_ik u_kj
// (i != j; diagonals are never formed by subtraction).
// One warp: rows k..k+bw live in a shared-memory ring while pivot k is eliminated, lane r owning
// row k+1+r, so a pivot needs one warp barrier; row k is written back when done and row
// k+bw+1 taken from a staging buffer that cp.async fills a chunk of rows ahead.
__global__ void __launch_bounds__(32) coarse_lu_kernel(float* band, int nc, int bw) {
  extern __shared__ float sm[];
  const int W = 2 * bw + 1, Wp = W + 1, R = bw + 1;
  const int lane = threadIdx.x;
  float* win = sm;             // [R][Wp] ring, row r in slot r % R
  float* stg = sm + R * Wp;    // [2][LU_CHUNK][Wp]; chunk c holds rows R + c*LU_CHUNK ...
  const int nstage = nc > R ? (nc - R + LU_CHUNK - 1) / LU_CHUNK : 0;
  auto issue = [&](int c) {
    if (c < nstage) {
      const int r0 = R + c * LU_CHUNK;
      float* dst = stg + (c & 1) * LU_CHUNK * Wp;
      for (int rr = 0; rr < LU_CHUNK && r0 + rr < nc; ++rr)
        for (int t = lane; t < Wp; t += 32)
          cp_async4(dst + rr * Wp + t, band + (int64_t)(r0 + rr) * Wp + t);
    }
    cp_async_commit();  // possibly empty: every lane keeps the same group count
  };
  for (int r = 0; r < R && r < nc; ++r)
    for (int t = lane; t < Wp; t += 32) win[r * Wp + t] = band[(int64_t)r * Wp + t];
  issue(0);
  issue(1);
  __syncwarp();
  int slot = 0;  // k % R
  for (int k = 0; k < nc; ++k) {
    const int m = min(bw, nc - 1 - k);  // rows / columns of the trailing window
    float* rk = win + slot * Wp;
    const float sk = rk[W];
    // pivot: row sum plus the magnitudes of row k's final upper entries (lanes < bw)
    const float u = sk + warp_sum(lane < bw ? -rk[bw + 1 + lane] : 0.f);
    if (lane < m) {
      int si = slot + 1 + lane;
      if (si >= R) si -= R;
      float* ri = win + si * Wp;
      const float sik = ri[bw - 1 - lane];  // S_ik <= 0
      const float l = sik / u;              // l_ik <= 0
      ri[bw - 1 - lane] = l;
      ri[W] = fmaf(-l, sk, ri[W]);
      // row i = k+1+lane, column j = k+1+c: offset c - lane + bw in row i, c + 1 + bw in row k
      for (int c = 0; c < m; ++c)
        if (c != lane) ri[c - lane + bw] = fmaf(-l, rk[c + 1 + bw], ri[c - lane + bw]);
    }
    if (lane == 0) rk[bw] = u;
    __syncwarp();
    if (k + R < nc) {
      const int c = k / LU_CHUNK, o = k % LU_CHUNK;
      if (o == 0) {  // first row of chunk c: its copies (all but the newest group) are done
        cp_async_wait1();
        __syncwarp();
      }
      const float* src = stg + (c & 1) * LU_CHUNK * Wp + o * Wp;
      for (int t = lane; t < Wp; t += 32) {
        band[(int64_t)k * Wp + t] = rk[t];
        rk[t] = src[t];
      }
      __syncwarp();
      if (o == LU_CHUNK - 1) issue(c + 2);  // chunk c's buffer is free now
    } else {
      for (int t = lane; t < Wp; t += 32) band[(int64_t)k * Wp + t] = rk[t];
      __syncwarp();
    }
    if (++slot == R) slot = 0;
  }
  cp_async_wait0();
}

// Reciprocal without branches: the approximate hardware reciprocal refined by one Newton-Raphson
// step x' = x + x (1 - u x), which roughly doubles its number of correct bits.  The factors it
// feeds are checked as a whole: the device's J_c^{-1} against the oracle's FP64 inverse of the
// Galerkin operator, within 5e-6 of its largest entry up to gamma = 0.9999 (GPU test).
__device__ __forceinline__ float rcp_nr(float u) {
  float x;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(x) : "f"(u));
  return fmaf(x, fmaf(-u, x, 1.f), x);
}

// Single-thread banded LU for a narrow band (bw = BW <= 8), same elimination (GTH form) as
// coarse_lu_kernel.  Rows k..k+BW stay in registers in band form (slot i mod R holds row i:
// b[slot][t] = A[i][i - BW + t]), so advancing the pivot moves no data: the pivot loop is
// unrolled by R = BW + 1 and every slot index is static.  A finished row leaves in one
// contiguous store; the next row enters its slot from a shared-memory ring that cp.async fills
// LU1_AHEAD rows ahead.  The main loop has no branches (the scheduler interleaves the
// independent row updates of consecutive pivots); the last pivots run with range guards.
constexpr int LU1_AHEAD = 8;

template <int BW, bool GUARD>
__device__ __forceinline__ void lu1_pivot(float (&b)[BW + 1][2 * BW + 1], float (&sr)[BW + 1],
                                          float (*ring)[2 * BW + 2], int j, int k, int nc,
                                          float* band) {
  constexpr int W = 2 * BW + 1, Wp = W + 1, R = BW + 1, NS = LU1_AHEAD + 1;
  float osum = 0.f;  // magnitudes of row k's final upper entries (all <= 0 in the band)
#pragma unroll
  for (int c = 1; c <= BW; ++c) osum -= b[j][BW + c];
  const float u = sr[j] + osum;
  const float rcp = rcp_nr(u);
  b[j][BW] = u;
#pragma unroll
  for (int r = 1; r <= BW; ++r) {
    const int q = (j + r) % R;  // static after unrolling
    if (!GUARD || k + r < nc) {
      const float sik = b[q][BW - r];  // S_{k+r,k} <= 0
      const float l = sik * rcp;
      b[q][BW - r] = l;
      sr[q] = fmaf(-l, sr[j], sr[q]);
#pragma unroll
      for (int c = 1; c <= BW; ++c)
        if (c != r) b[q][c - r + BW] = fmaf(-l, b[j][BW + c], b[q][c - r + BW]);
    }
  }
  float* rowk = band + (int64_t)k * Wp;
#pragma unroll
  for (int t = 0; t < W; ++t) rowk[t] = b[j][t];
  const int i = k + R;  // the row entering slot j
  if (!GUARD || i < nc) {
    cp_async_wait_ahead();  // row i's group (the oldest pending) is complete
    const float* src = ring[(i - R) % NS];
#pragma unroll
    for (int t = 0; t < W; ++t) b[j][t] = src[t];
    sr[j] = src[W];
    const int in = i + LU1_AHEAD;  // into the slot read one pivot ago
    if (!GUARD || in < nc) {
      float* dst = ring[(in - R) % NS];
#pragma unroll
      for (int t = 0; t < Wp; ++t) cp_async4(dst + t, band + (int64_t)in * Wp + t);
    }
    cp_async_commit();
  }
}

template <int BW>
__global__ void __launch_bounds__(1) coarse_lu1_kernel(float* band, int nc) {
  constexpr int W = 2 * BW + 1, Wp = W + 1, R = BW + 1, NS = LU1_AHEAD + 1;
  __shared__ float ring[NS][Wp];
  float b[R][W];
  float sr[R];  // row sum of each slot's row over its Schur complement
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const bool in = r < nc;
#pragma unroll
    for (int t = 0; t < W; ++t) b[r][t] = in ? band[(int64_t)r * Wp + t] : 0.f;
    sr[r] = in ? band[(int64_t)r * Wp + W] : 1.f;
  }
  for (int q = 0; q < LU1_AHEAD; ++q) {
    const int i = R + q;
    if (i < nc) {
#pragma unroll
      for (int t = 0; t < Wp; ++t) cp_async4(&ring[(i - R) % NS][t], band + (int64_t)i * Wp + t);
    }
    cp_async_commit();
  }
  int k0 = 0;
  // every row a pivot of this round touches exists, and so does every row it prefetches
  for (; k0 + 2 * R + LU1_AHEAD + BW <= nc; k0 += R) {
#pragma unroll
    for (int j = 0; j < R; ++j) lu1_pivot<BW, false>(b, sr, ring, j, k0 + j, nc, band);
  }
  for (; k0 < nc; k0 += R) {
#pragma unroll
    for (int j = 0; j < R; ++j)
      if (k0 + j < nc) lu1_pivot<BW, true>(b, sr, ring, j, k0 + j, nc, band);
  }
  cp_async_wait0();
}

// Coefficients of the two triangular solves of J_c x = e_j = L U x, row k of each in a
// [nc][32] layout (FP32), zero for q >= bw and outside the matrix:
//   forward  L y = e_j:  y[k] = delta_{kj} + sum_q cl[k][q] y[k-1-q],   cl[k][q] = -L[k][k-1-q]
//   backward U x = y:    x[k] = dinv[k] y[k] + sum_q cu[k][q] x[k+1+q], cu[k][q] = -U[k][k+1+q] dinv[k]
__global__ void coarse_prep_kernel(const float* band, int nc, int bw, float* cl, float* cu, float* dinv) {
  const int W = 2 * bw + 1, Wp = W + 1;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < (int64_t)nc * 32;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e >> 5), q = (int)(e & 31);
    const float* rk = band + (int64_t)k * Wp;
    const float dk = 1.f / rk[bw];
    float f = 0.f, b = 0.f;
    if (q < bw) {
      if (k - 1 - q >= 0) f = -rk[bw - 1 - q];
      if (k + 1 + q < nc) b = -rk[bw + 1 + q] * dk;
    }
    cl[e] = f;
    cu[e] = b;
    if (q == 0) dinv[k] = dk;
  }
}

// Columns of J_c^{-1}: lane j of a warp solves J_c x = e_j for column j = 32 * warp + lane, so
// all lanes step through k together and read the same coefficients (broadcast), each lane
// keeping the last RW values of its own recurrence in registers (RW a power of two >= bw; steps
// are unrolled in blocks of 32 so the ring index is static).  The newest value enters each step
// through one FMA, so the recurrence runs at FMA latency.  y is parked in inv[k][j] (stores
// coalesced across lanes) for the backward pass, which reads it a block of 32 steps ahead and
// overwrites it with x.  With STAGED the block (one warp) first copies the coefficients it
// needs into shared memory.
template <int RW, bool STAGED>
__global__ void __launch_bounds__(32) coarse_inverse_kernel(const float* cl, const float* cu,
                                                            const float* dinv, int nc, int64_t ldi,
                                                            float* inv) {
  extern __shared__ float csm[];  // STAGED: [nc][RW] coefficients, then dinv [nc]
  const int lane = threadIdx.x;
  const int64_t j0 = (int64_t)blockIdx.x * 32;
  const int64_t j = j0 + lane;
  const bool own = j < nc;
  auto stage = [&](const float* src, bool with_d) {
    __syncwarp();
    for (int64_t e = lane; e < (int64_t)nc * RW; e += 32) csm[e] = src[(e / RW) * 32 + e % RW];
    if (with_d)
      for (int64_t e = lane; e < nc; e += 32) csm[(int64_t)nc * RW + e] = dinv[e];
    __syncwarp();
  };
  // the RW coefficients of step k as vector loads (rows are 16-byte aligned for RW >= 4)
  auto coefs = [&](const float* g, int64_t k, float (&c)[RW]) {
    const float* src = STAGED ? csm + k * RW : g + k * 32;
    if constexpr (RW >= 4) {
#pragma unroll
      for (int i = 0; i < RW / 4; ++i) {
        const float4 v = STAGED ? reinterpret_cast<const float4*>(src)[i]
                                : __ldg(reinterpret_cast<const float4*>(src) + i);
        c[4 * i] = v.x; c[4 * i + 1] = v.y; c[4 * i + 2] = v.z; c[4 * i + 3] = v.w;
      }
    } else {
      const float2 v = STAGED ? *reinterpret_cast<const float2*>(src)
                              : __ldg(reinterpret_cast<const float2*>(src));
      c[0] = v.x; c[1] = v.y;
    }
  };
  auto dk = [&](int64_t k) -> float {
    if constexpr (STAGED) return csm[(int64_t)nc * RW + k];
    else return __ldg(dinv + k);
  };
  if constexpr (STAGED) stage(cl, false);
  float h[RW];
#pragma unroll
  for (int q = 0; q < RW; ++q) h[q] = 0.f;
  // forward: k = j0 .. nc-1 (y[k] = 0 below the warp's first column); full blocks of 32
  // steps have no branches, so the scheduler overlaps consecutive steps' older terms
  auto fstep = [&](int s, int64_t k) {
    float c[RW];
    coefs(cl, k, c);
    float part = (k == j) ? 1.f : 0.f;
#pragma unroll
    for (int q = 1; q < RW; ++q) part = fmaf(c[q], h[(s - 1 - q) & (RW - 1)], part);
    const float y = fmaf(c[0], h[(s - 1) & (RW - 1)], part);
    h[s & (RW - 1)] = y;
    if (own) inv[k * ldi + j] = y;
  };
  int64_t kb = j0;
  for (; kb + 32 <= nc; kb += 32) {
#pragma unroll
    for (int s = 0; s < 32; ++s) fstep(s, kb + s);
  }
#pragma unroll
  for (int s = 0; s < 32; ++s)
    if (kb + s < nc) fstep(s, kb + s);
  if constexpr (STAGED) stage(cu, true);
  __syncwarp();
#pragma unroll
  for (int q = 0; q < RW; ++q) h[q] = 0.f;
  // backward: k = nc-1 .. 0, with h[(s - 1 - q) mod RW] holding x[k+1+q]
  float yb[32];
  auto load_y = [&](int64_t kb, float (&dst)[32]) {
#pragma unroll
    for (int s = 0; s < 32; ++s) {
      const int64_t k = kb - s;
      dst[s] = (k >= j0 && own) ? inv[k * ldi + j] : 0.f;
    }
  };
  auto bstep = [&](int s, int64_t k) {
    float c[RW];
    coefs(cu, k, c);
    float part = yb[s] * dk(k);
#pragma unroll
    for (int q = 1; q < RW; ++q) part = fmaf(c[q], h[(s - 1 - q) & (RW - 1)], part);
    const float x = fmaf(c[0], h[(s - 1) & (RW - 1)], part);
    h[s & (RW - 1)] = x;
    if (own) inv[k * ldi + j] = x;
  };
  load_y(nc - 1, yb);
  int64_t kd = nc - 1;
  for (; kd - 31 >= 0; kd -= 32) {
    float yn[32];
    load_y(kd - 32, yn);  // the next block, in flight while this one runs
#pragma unroll
    for (int s = 0; s < 32; ++s) bstep(s, kd - s);
#pragma unroll
    for (int s = 0; s < 32; ++s) yb[s] = yn[s];
  }
#pragma unroll
  for (int s = 0; s < 32; ++s)
    if (kd - s >= 0) bstep(s, kd - s);
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
  float sum = 0.f;
  for (int64_t u = threadIdx.x; u < cnt; u += blockDim.x) {
    const KT qs = x[s0 + u] * scale;
    q[s0 + u] = qs;
    sum += (float)qs;
  }
  __shared__ float red[32];
  sum = block_sum(sum, red);
  if (threadIdx.x == 0) p.f[I] = sum / (float)cnt;
}

// E_i[I] = sum_J J_c^{-1}[I][J] f[J] (one warp per coarse row; rows padded to ldc with zeros).
template <class KT>
__global__ void __launch_bounds__(PC_THREADS) coarse_apply_kernel(PrecondK p) {
  const GmresCtl* c = p.ctl;
  if (*(volatile const int*)&c->mode != GM_STEP) return;
  const int lane = threadIdx.x & 31;
  const int64_t wid = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  KT* e = (KT*)p.E + (int64_t)c->i * p.ldc;
  const float4* f4 = reinterpret_cast<const float4*>(p.f);
  const int64_t n4 = p.ldc >> 2;
  for (int64_t I = wid; I < p.nc; I += nw) {
    const float4* row = reinterpret_cast<const float4*>(p.inv + I * p.ldc);
    float t = 0.f;
    for (int64_t J = lane; J < n4; J += 32) {
      const float4 a = __ldg(row + J), b = f4[J];
      t = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, t))));
    }
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
    KT t = 0;
    for (int j = 0; j < m; ++j)
      t += (sizeof(KT) == 4 ? (KT)c->yf[j] : (KT)c->y[j]) * ((const KT*)p.E)[(int64_t)j * p.ldc + I];
    ((KT*)p.ec)[I] = t;
  }
}

// Number of states whose action differs between two policies (block sums, one atomic per block).
__global__ void count_changed_kernel(const int32_t* pi, const int32_t* ref, int64_t S, int* count) {
  __shared__ int red[32];
  int c = 0;
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x)
    c += pi[s] != ref[s];
  c = block_sum(c, red);
  if (threadIdx.x == 0 && c) atomicAdd(count, c);
}

inline int pc_grid(int64_t n, int per_block) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + per_block - 1) / per_block,
                                                     (int64_t)num_sms() * 8));
}

inline int ok() { return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE; }

// Shared memory the staged inverse kernel needs: coefficients [nc][RW] and dinv [nc].
inline size_t inverse_smem(int64_t nc, int rw) { return (size_t)nc * (rw + 1) * sizeof(float); }
constexpr size_t INV_SMEM_MAX = 200 * 1024;

template <int RW>
int launch_inverse(const PrecondScratch& w, const PrecondK& p, cudaStream_t st) {
  const int grid = (int)((p.nc + 31) / 32);  // one warp (block) per 32 columns
  const size_t smem = inverse_smem(p.nc, RW);
  if (smem <= INV_SMEM_MAX) {
    auto k = coarse_inverse_kernel<RW, true>;
    if (smem > 48 * 1024 &&
        cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
      return MDP_EDEVICE;
    k<<<grid, 32, smem, st>>>(w.cl, w.cu, w.dinv, (int)p.nc, p.ldc, p.inv);
  } else {
    coarse_inverse_kernel<RW, false><<<grid, 32, 0, st>>>(w.cl, w.cu, w.dinv, (int)p.nc, p.ldc, p.inv);
  }
  return MDP_OK;
}

}  // namespace

int launch_coarse_bandwidth(const DevMDP& d, int lb, int* bw, cudaStream_t st) {
  const int64_t n = d.S * d.A * (int64_t)d.kp;
  coarse_bandwidth_kernel<<<pc_grid(n, 256), 256, 0, st>>>(d, lb, bw);
  return ok();
}

size_t coarse_lu_smem(int bw) { return (size_t)(bw + 1 + 2 * LU_CHUNK) * (2 * bw + 2) * sizeof(float); }

int launch_coarse_setup(const DevMDP& d, const int32_t* pi, const PrecondK& p, int bw,
                        const PrecondScratch& w, cudaStream_t st) {
  if (d.pdt == MDP_F32)
    coarse_build_kernel<float><<<(int)p.nc, PC_THREADS, 0, st>>>(d, pi, p.lb, bw, w.band);
  else
    coarse_build_kernel<double><<<(int)p.nc, PC_THREADS, 0, st>>>(d, pi, p.lb, bw, w.band);
  switch (bw) {  // a narrow band factors in one thread's registers
    case 1: coarse_lu1_kernel<1><<<1, 1, 0, st>>>(w.band, (int)p.nc); break;
    case 2: coarse_lu1_kernel<2><<<1, 1, 0, st>>>(w.band, (int)p.nc); break;
    case 3: coarse_lu1_kernel<3><<<1, 1, 0, st>>>(w.band, (int)p.nc); break;
    case 4: coarse_lu1_kernel<4><<<1, 1, 0, st>>>(w.band, (int)p.nc); break;
    case 5: coarse_lu1_kernel<5><<<1, 1, 0, st>>>(w.band, (int)p.nc); break;
    case 6: coarse_lu1_kernel<6><<<1, 1, 0, st>>>(w.band, (int)p.nc); break;
    case 7: coarse_lu1_kernel<7><<<1, 1, 0, st>>>(w.band, (int)p.nc); break;
    case 8: coarse_lu1_kernel<8><<<1, 1, 0, st>>>(w.band, (int)p.nc); break;
    default: coarse_lu_kernel<<<1, 32, coarse_lu_smem(bw), st>>>(w.band, (int)p.nc, bw);
  }
  coarse_prep_kernel<<<pc_grid(p.nc * 32, 256), 256, 0, st>>>(w.band, (int)p.nc, bw, w.cl, w.cu, w.dinv);
  int r;
  if (bw <= 2) r = launch_inverse<2>(w, p, st);
  else if (bw <= 4) r = launch_inverse<4>(w, p, st);
  else if (bw <= 8) r = launch_inverse<8>(w, p, st);
  else if (bw <= 16) r = launch_inverse<16>(w, p, st);
  else r = launch_inverse<32>(w, p, st);
  if (r != MDP_OK) return r;
  return ok();
}

int launch_coarse_step(const PrecondK& p, int kt, cudaStream_t st) {
  const int gapply = (int)std::max<int64_t>(1, std::min<int64_t>((p.nc * 32 + PC_THREADS - 1) / PC_THREADS,
                                                                  (int64_t)num_sms() * 8));
  if (kt == 1) {
    coarse_restrict_kernel<float><<<(int)p.nc, PC_THREADS, 0, st>>>(p);
    coarse_apply_kernel<float><<<gapply, PC_THREADS, 0, st>>>(p);
    coarse_prolong_kernel<float><<<pc_grid(p.S, 256), 256, 0, st>>>(p);
  } else {
    coarse_restrict_kernel<double><<<(int)p.nc, PC_THREADS, 0, st>>>(p);
    coarse_apply_kernel<double><<<gapply, PC_THREADS, 0, st>>>(p);
    coarse_prolong_kernel<double><<<pc_grid(p.S, 256), 256, 0, st>>>(p);
  }
  return ok();
}

int launch_count_changed(const int32_t* pi, const int32_t* ref, int64_t S, int* count,
                         cudaStream_t st) {
  count_changed_kernel<<<pc_grid(S, 256), 256, 0, st>>>(pi, ref, S, count);
  return ok();
}

int launch_coarse_combine(const PrecondK& p, int kt, cudaStream_t st) {
  if (kt == 1) coarse_combine_kernel<float><<<pc_grid(p.nc, 256), 256, 0, st>>>(p);
  else coarse_combine_kernel<double><<<pc_grid(p.nc, 256), 256, 0, st>>>(p);
  return ok();
}

}  // namespace mdp
