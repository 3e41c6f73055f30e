// Restarted GMRES(W) for the inexact policy evaluation of Alg. 2 (paper Sec. 2.2, 3.1):
//
//   P^pi matvec   w = J^pi q = q - gamma P^pi q, rows of P_{pi(s)} gathered on the fly
//   Arnoldi       classical Gram-Schmidt, re-orthogonalised once (CGS2) when the first projection
//                 cancelled more than half of the norm, the Hessenberg
//                 column H[0..i+1][i] in FP64
//   least squares Givens rotations on H in FP64, |gv[i+1]| = ||beta e1 - H y||_2
//   stopping rule ||g^pi - J^pi V||_inf <= thr, tested on the true residual; a cheap bound
//                 from the Arnoldi relation decides when the true test is worth a matvec
//
// The inner solver is a device-resident state machine (GmresCtl.mode): every kernel of an
// Arnoldi step checks the mode and returns at once when it is not due, and only the last
// block of a grid (after all blocks have read the mode) changes it.
#include "mdp_internal.cuh"

#include <algorithm>
#include <math.h>

namespace mdp {

namespace {

template <class KT> __device__ __forceinline__ KT coef(const double* d, const float* f, int j);
template <> __device__ __forceinline__ double coef<double>(const double* d, const float*, int j) {
  return d[j];
}
template <> __device__ __forceinline__ float coef<float>(const double*, const float* f, int j) {
  return f[j];
}
template <class KT> __device__ __forceinline__ KT scale_of(const GmresCtl* c);
template <> __device__ __forceinline__ double scale_of<double>(const GmresCtl* c) { return c->xscale; }
template <> __device__ __forceinline__ float scale_of<float>(const GmresCtl* c) { return c->xscalef; }

__device__ __forceinline__ void set_scale(GmresCtl* c, double s) { gmres_set_scale(c, s); }

// Move to the next Arnoldi step of the cycle, or to a restart when the cycle is full.
__device__ __forceinline__ void advance(GmresCtl* c) {
  if (c->i >= c->W - 1) {
    c->mode = GM_RESTART;
  } else {
    c->i += 1;
    c->from_rhs = 0;
    set_scale(c, 1.0 / c->hnext);
    c->mode = GM_STEP;
  }
}

// ------------------------------------------------------------------ P^pi matvec
struct MatvecK {
  DevMDP d;
  const int32_t* pi;
  const void* x;
  GmresCtl* ctl;
  int gate_mode, gate_mode2;
  const void* x_rhs;
  const void* x_w0;
  const void* x_w1;
  void* qbase;
  int64_t ldq;
  double a, b, c;
  const void* u;
  void* out;
  void* out0;
  void* out1;
  SweepOut* norms;
  int finalize_check;
  void* partials;
  unsigned* counter;
  const void* x_pre;  // preconditioned STEP: the vector M^{-1} Q_i to multiply (scale 1)
};

// Resolved per launch (uniform over the grid): input, its scale, output and side output.
template <class KT> struct MvIO {
  const KT* x;
  KT scale;
  KT* out;
  KT* qside;
  bool run;
};

template <class KT>
__device__ __forceinline__ MvIO<KT> resolve(const MatvecK& p) {
  MvIO<KT> io;
  io.run = true;
  io.x = (const KT*)p.x;
  io.scale = KT(1);
  io.out = (KT*)p.out;
  io.qside = nullptr;
  if (p.ctl) {
    const GmresCtl* c = p.ctl;
    int mode = *(volatile const int*)&c->mode;
    io.run = (mode == p.gate_mode || mode == p.gate_mode2);
    if (p.gate_mode == GM_STEP) {
      const int i = c->i;
      io.out = (KT*)((i & 1) ? p.out1 : p.out0);
      if (p.x_pre) {  // Q_i was written by the preconditioner's restriction kernel
        io.x = (const KT*)p.x_pre;
      } else {
        io.x = c->from_rhs ? (const KT*)p.x_rhs : (const KT*)((i - 1) & 1 ? p.x_w1 : p.x_w0);
        io.scale = scale_of<KT>(c);
        io.qside = (KT*)p.qbase + (int64_t)i * p.ldq;
      }
    } else {
      io.x = (const KT*)(c->dsel ? p.x_w0 : p.x_w1);  // candidate = dbuf[1 - dsel]
    }
  }
  return io;
}

template <class KT>
__device__ __forceinline__ void matvec_finish(const MatvecK& p, KT mx, KT ss,
                                              GridPos gp = this_grid()) {
  __shared__ KT shr[32];
  KT bm = block_max(mx, shr);
  KT bs = block_sum(ss, shr);
  KT* part = (KT*)p.partials;
  if (threadIdx.x == 0) {
    part[2 * gp.bid] = bm;
    part[2 * gp.bid + 1] = bs;
  }
  if (!arrive_last(p.counter, gp.nb)) return;
  KT m = 0, t = 0;
  for (int b = threadIdx.x; b < gp.nb; b += blockDim.x) {
    m = max(m, __ldcg(part + 2 * b));
    t += __ldcg(part + 2 * b + 1);
  }
  m = block_max(m, shr);
  t = block_sum(t, shr);
  if (threadIdx.x != 0) return;
  const double rinf = (double)m, rn2 = sqrt((double)t);
  if (p.norms) {
    p.norms->res_inf = rinf;
    p.norms->res_nrm2 = rn2;
  }
  if (!p.ctl) return;
  GmresCtl* c = p.ctl;
  if (p.gate_mode == GM_STEP) {
    c->last_nrm2 = rn2;  // ||J q_i||_2 before orthogonalisation (breakdown reference)
    return;
  }
  // true-residual check of the candidate (CHECK) or restart from it (RESTART)
  c->checks += 1;
  c->last_inf = rinf;
  const int mode = c->mode;
  if (rinf <= c->thr) {
    c->mode = GM_DONE;
    c->status = GS_CONVERGED;
    c->dsel = 1 - c->dsel;  // the candidate becomes the result
    return;
  }
  if (mode == GM_CHECK && c->i < c->W - 1) {
    advance(c);
    return;
  }
  // restart (Alg. 2: cycle full) from the candidate and its true residual (now in rbuf)
  c->dsel = 1 - c->dsel;
  c->restarts += 1;
  c->beta = rn2;
  c->est_ratio = rn2 > 0.0 ? rinf / rn2 : 1.0;
  for (int j = 0; j <= WMAX; ++j) c->gv[j] = 0.0;
  c->gv[0] = rn2;
  c->i = 0;
  c->from_rhs = 1;
  set_scale(c, rn2 > 0.0 ? 1.0 / rn2 : 0.0);
  c->mode = (rn2 > 0.0) ? GM_STEP : GM_DONE;
  if (rn2 == 0.0) c->status = GS_CONVERGED;
}

template <class PT, class KT, int T>
__device__ __forceinline__ void matvec_ell_body(const MatvecK& p, GridPos gp) {
  const MvIO<KT> io = resolve<KT>(p);
  if (!io.run) return;
  const DevMDP& d = p.d;
  const int nteams = blockDim.x / T;
  const int team = threadIdx.x / T, tl = threadIdx.x % T;
  const PT* val = (const PT*)d.P;
  const int nvec = d.kp >> 2;
  const KT* u = (const KT*)p.u;
  const KT ca = (KT)p.a, cb = (KT)p.b, cc = (KT)p.c;
  const uint64_t pol = l2_keep_policy();
  KT mx = 0, ss = 0;
  const int64_t nteam_total = (int64_t)gp.nb * nteams;
  for (int64_t sb = (int64_t)gp.bid * nteams; sb < d.S; sb += nteam_total) {
    const int64_t s = sb + team;
    const bool act = s < d.S;
    KT acc = 0;
    if (act) {
      const int64_t base = ((int64_t)s * d.A + p.pi[s]) * d.kp;
      for (int q = tl; q < nvec; q += T) {
        float4 vv;
        KT v0, v1, v2, v3;
        if constexpr (sizeof(PT) == 4) {
          vv = __ldcs(reinterpret_cast<const float4*>(val + base) + q);
          v0 = (KT)vv.x; v1 = (KT)vv.y; v2 = (KT)vv.z; v3 = (KT)vv.w;
        } else {
          double2 t0 = __ldcs(reinterpret_cast<const double2*>(val + base + 4 * q));
          double2 t1 = __ldcs(reinterpret_cast<const double2*>(val + base + 4 * q) + 1);
          v0 = (KT)t0.x; v1 = (KT)t0.y; v2 = (KT)t1.x; v3 = (KT)t1.y;
        }
        int4 c4 = __ldcs(reinterpret_cast<const int4*>(d.col + base) + q);
        acc = fma(v0, ld_keep(io.x + c4.x, pol), acc);
        acc = fma(v1, ld_keep(io.x + c4.y, pol), acc);
        acc = fma(v2, ld_keep(io.x + c4.z, pol), acc);
        acc = fma(v3, ld_keep(io.x + c4.w, pol), acc);
      }
    }
#pragma unroll
    for (int o = T >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (act && tl == 0) {
      const KT xs = io.x[s] * io.scale;
      KT r = ca * xs + cc * (acc * io.scale);
      if (u) r += cb * u[s];
      io.out[s] = r;
      if (io.qside) io.qside[s] = xs;
      mx = max(mx, (KT)fabs(r));
      ss += r * r;
    }
  }
  matvec_finish<KT>(p, mx, ss, gp);
}

template <class PT, class KT, int T>
__global__ void __launch_bounds__(256) matvec_ell_kernel(MatvecK p) {
  matvec_ell_body<PT, KT, T>(p, this_grid());
}

// Banded columns (every column within d.span of its state): a block walks contiguous steps of
// MV_NB states and gathers x from a shared-memory ring that cp.async refills a step ahead, as
// the windowed Bellman sweep does.  Same per-row arithmetic as matvec_ell_body.
constexpr int MV_RING = 4096;
constexpr int MV_NB = 256;
constexpr int64_t MV_SPAN_MAX = (MV_RING - 2 * MV_NB) / 2;

template <class KT>
__device__ __forceinline__ void mv_cp_async(KT* smem, const KT* gmem) {
  if constexpr (sizeof(KT) == 4)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}

template <class PT, class KT, int T>
__global__ void __launch_bounds__(256) matvec_ell_window_kernel(MatvecK p) {
  __shared__ KT ring[MV_RING];
  const MvIO<KT> io = resolve<KT>(p);
  if (!io.run) return;  // uniform over the grid
  const DevMDP& d = p.d;
  const int nteams = blockDim.x / T;
  const int team = threadIdx.x / T, tl = threadIdx.x % T;
  const PT* val = (const PT*)d.P;
  const int nvec = d.kp >> 2;
  const KT* u = (const KT*)p.u;
  const KT ca = (KT)p.a, cb = (KT)p.b, cc = (KT)p.c;
  const int64_t span = d.span;
  // this block's states: an equal share of the 32-state units, walked in steps of MV_NB
  const int64_t nu = (d.S + 31) >> 5;
  const int64_t sb = 32 * (nu * blockIdx.x / gridDim.x);
  const int64_t se = min(d.S, 32 * (nu * (blockIdx.x + 1) / gridDim.x));
  auto fill = [&](int64_t x0, int64_t x1) {
    const int64_t a0 = max(x0, (int64_t)0), a1 = min(x1, d.S);
    for (int64_t x = a0 + threadIdx.x; x < a1; x += blockDim.x) mv_cp_async(ring + (x & (MV_RING - 1)), io.x + x);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  KT mx = 0, ss = 0;
  if (sb < se) {
    fill(sb - span, min(sb + MV_NB, se) + span);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int64_t s_lo = sb; s_lo < se; s_lo += MV_NB) {
      const int64_t s_hi = min(s_lo + MV_NB, se);
      if (s_hi < se) fill(s_hi + span, min(s_hi + MV_NB, se) + span);
      for (int64_t s1 = s_lo; s1 < s_hi; s1 += nteams) {
        const int64_t s = s1 + team;
        const bool act = s < s_hi;
        KT acc = 0;
        if (act) {
          const int64_t base = ((int64_t)s * d.A + p.pi[s]) * d.kp;
          for (int q = tl; q < nvec; q += T) {
            float4 vv;
            KT v0, v1, v2, v3;
            if constexpr (sizeof(PT) == 4) {
              vv = __ldcs(reinterpret_cast<const float4*>(val + base) + q);
              v0 = (KT)vv.x; v1 = (KT)vv.y; v2 = (KT)vv.z; v3 = (KT)vv.w;
            } else {
              double2 t0 = __ldcs(reinterpret_cast<const double2*>(val + base + 4 * q));
              double2 t1 = __ldcs(reinterpret_cast<const double2*>(val + base + 4 * q) + 1);
              v0 = (KT)t0.x; v1 = (KT)t0.y; v2 = (KT)t1.x; v3 = (KT)t1.y;
            }
            int4 c4 = __ldcs(reinterpret_cast<const int4*>(d.col + base) + q);
            acc = fma(v0, ring[c4.x & (MV_RING - 1)], acc);
            acc = fma(v1, ring[c4.y & (MV_RING - 1)], acc);
            acc = fma(v2, ring[c4.z & (MV_RING - 1)], acc);
            acc = fma(v3, ring[c4.w & (MV_RING - 1)], acc);
          }
        }
#pragma unroll
        for (int o = T >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (act && tl == 0) {
          const KT xs = io.x[s] * io.scale;
          KT r = ca * xs + cc * (acc * io.scale);
          if (u) r += cb * u[s];
          io.out[s] = r;
          if (io.qside) io.qside[s] = xs;
          mx = max(mx, (KT)fabs(r));
          ss += r * r;
        }
      }
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncthreads();
    }
  }
  matvec_finish<KT>(p, mx, ss, this_grid());
}

template <class PT, class KT>
__global__ void __launch_bounds__(256) matvec_dense_kernel(MatvecK p) {
  const MvIO<KT> io = resolve<KT>(p);
  if (!io.run) return;
  const DevMDP& d = p.d;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const PT* P = (const PT*)d.P;
  const KT* u = (const KT*)p.u;
  const KT ca = (KT)p.a, cb = (KT)p.b, cc = (KT)p.c;
  KT mx = 0, ss = 0;
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < d.S; s += nw) {
    const PT* row = P + ((int64_t)s * d.A + p.pi[s]) * d.ld;
    KT acc0 = 0, acc1 = 0;
    int64_t c = 4 * lane;
    for (; c + 128 < d.ld; c += 256) {
      KT xa[4], xb[4], pa[4], pb[4];
      if constexpr (sizeof(KT) == 4) {
        float4 t = __ldg(reinterpret_cast<const float4*>(io.x + c));
        float4 t2 = __ldg(reinterpret_cast<const float4*>(io.x + c + 128));
        xa[0] = t.x; xa[1] = t.y; xa[2] = t.z; xa[3] = t.w;
        xb[0] = t2.x; xb[1] = t2.y; xb[2] = t2.z; xb[3] = t2.w;
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) { xa[e] = __ldg(io.x + c + e); xb[e] = __ldg(io.x + c + 128 + e); }
      }
      if constexpr (sizeof(PT) == 4) {
        float4 t = __ldcs(reinterpret_cast<const float4*>(row + c));
        float4 t2 = __ldcs(reinterpret_cast<const float4*>(row + c + 128));
        pa[0] = t.x; pa[1] = t.y; pa[2] = t.z; pa[3] = t.w;
        pb[0] = t2.x; pb[1] = t2.y; pb[2] = t2.z; pb[3] = t2.w;
      } else {
        double2 t0 = __ldcs(reinterpret_cast<const double2*>(row + c));
        double2 t1 = __ldcs(reinterpret_cast<const double2*>(row + c) + 1);
        double2 t2 = __ldcs(reinterpret_cast<const double2*>(row + c + 128));
        double2 t3 = __ldcs(reinterpret_cast<const double2*>(row + c + 128) + 1);
        pa[0] = t0.x; pa[1] = t0.y; pa[2] = t1.x; pa[3] = t1.y;
        pb[0] = t2.x; pb[1] = t2.y; pb[2] = t3.x; pb[3] = t3.y;
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) { acc0 = fma(pa[e], xa[e], acc0); acc1 = fma(pb[e], xb[e], acc1); }
    }
    for (; c < d.ld; c += 128) {
#pragma unroll
      for (int e = 0; e < 4; ++e) acc0 = fma((KT)row[c + e], __ldg(io.x + c + e), acc0);
    }
    KT acc = warp_sum(acc0 + acc1);
    if (lane == 0) {
      const KT xs = io.x[s] * io.scale;
      KT r = ca * xs + cc * (acc * io.scale);
      if (u) r += cb * u[s];
      io.out[s] = r;
      if (io.qside) io.qside[s] = xs;
      mx = max(mx, (KT)fabs(r));
      ss += r * r;
    }
  }
  matvec_finish<KT>(p, mx, ss);
}

// ------------------------------------------------------------------ dense, bulk-copy pipeline
// FP32 P^pi matvec: warp 8 (one elected thread) streams row pi(s) of every state in chunks of
// TM_CW columns into a ring of shared-memory stages with cp.async.bulk; warps 0..7 take four
// float4 quads of each chunk against the input vector, which stays resident in shared memory;
// the last warp to finish a state combines the eight partial sums in a fixed order.
constexpr int TM_WARPS = 8;
constexpr int TM_THREADS = (TM_WARPS + 1) * 32;
constexpr int TM_CW = 4096;
constexpr int TM_NBUF = 16;  // > stages + 2

struct TmaMvLayout {
  size_t x_off, stg_off, bar_off, red_off, cnt_off, total;
};

__host__ __device__ inline size_t align_up_mv(size_t x, size_t a) { return (x + a - 1) / a * a; }

__host__ __device__ inline TmaMvLayout tma_mv_layout(int64_t ld, int ns) {
  TmaMvLayout L;
  L.x_off = 0;
  L.stg_off = align_up_mv((size_t)ld * 4, 128);
  L.bar_off = L.stg_off + (size_t)ns * TM_CW * 4;
  L.red_off = align_up_mv(L.bar_off + (size_t)(2 * ns + 1) * 8, 16);
  L.cnt_off = L.red_off + (size_t)TM_NBUF * TM_WARPS * sizeof(float);
  L.total = align_up_mv(L.cnt_off + TM_NBUF * sizeof(int), 128);
  return L;
}

__global__ void __launch_bounds__(TM_THREADS, 2) matvec_dense_tma_kernel(MatvecK p, int ns, int* err) {
  const MvIO<float> io = resolve<float>(p);
  if (!io.run) return;
  extern __shared__ __align__(128) unsigned char sm[];
  const DevMDP& d = p.d;
  const int64_t ld = d.ld;
  const TmaMvLayout L = tma_mv_layout(ld, ns);
  float* xres = reinterpret_cast<float*>(sm + L.x_off);
  float* stg = reinterpret_cast<float*>(sm + L.stg_off);
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar_off);
  uint64_t* empty = full + ns;
  uint64_t* xbar = empty + ns;
  float* red = reinterpret_cast<float*>(sm + L.red_off);
  int* cnt = reinterpret_cast<int*>(sm + L.cnt_off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = (int)((ld + TM_CW - 1) / TM_CW);
  if (threadIdx.x == 0) {
    for (int st = 0; st < ns; ++st) {
      mbar_init(full + st, 1);
      mbar_init(empty + st, TM_WARPS);
    }
    mbar_init(xbar, 1);
    mbar_fence_init();
  }
  if (threadIdx.x < TM_NBUF) cnt[threadIdx.x] = 0;
  __syncthreads();
  const float* P = (const float*)d.P;
  const float* u = (const float*)p.u;
  const float ca = (float)p.a, cb = (float)p.b, cc = (float)p.c;
  float mx = 0.f, ss = 0.f;
  if (warp == TM_WARPS) {
    if (lane == 0) {
      const size_t xbytes = (size_t)ld * 4;
      mbar_expect_tx(xbar, (uint32_t)xbytes);
      for (size_t o = 0; o < xbytes; o += 32768)
        bulk_load((char*)xres + o, (const char*)io.x + o, (uint32_t)min((size_t)32768, xbytes - o), xbar);
      int n = 0;
      bool ok = true;
      int a_cur = blockIdx.x < d.S ? p.pi[blockIdx.x] : 0;
      for (int64_t s = blockIdx.x; s < d.S && ok; s += gridDim.x) {
        const float* row = P + ((int64_t)s * d.A + a_cur) * ld;
        // the next state's action is loaded now and used one state later
        const int64_t s2 = s + gridDim.x;
        const int a_next = s2 < d.S ? p.pi[s2] : 0;
        for (int ch = 0; ch < nch; ++ch, ++n) {
          const int st = n % ns;
          if (!mbar_wait(empty + st, (uint32_t)(((n / ns) & 1) ^ 1), err)) { ok = false; break; }
          const int64_t c0 = (int64_t)ch * TM_CW;
          const int cw = (int)((ld - c0) < (int64_t)TM_CW ? (ld - c0) : (int64_t)TM_CW);
          mbar_expect_tx(full + st, (uint32_t)cw * 4u);
          bulk_load(stg + (size_t)st * TM_CW, row + c0, (uint32_t)cw * 4u, full + st);
        }
        a_cur = a_next;
      }
      for (int k = 1; k <= ns && n - k >= 0; ++k) {
        const int m = n - k;
        mbar_wait(full + (m % ns), (uint32_t)((m / ns) & 1), err);
      }
    }
  } else {
    const int t = threadIdx.x;
    const int ldi = (int)ld;
    bool ok = mbar_wait(xbar, 0, err);
    int st = 0, ri = 0;
    uint32_t ph = 0;
    for (int64_t s = blockIdx.x; s < d.S && ok; s += gridDim.x) {
      float acc0 = 0.f, acc1 = 0.f;
      for (int c0 = 0; c0 < ldi; c0 += TM_CW) {
        if (!mbar_wait(full + st, ph, err)) { ok = false; break; }
        const int cw = ldi - c0;
        const float* sg = stg + (size_t)st * TM_CW;
#pragma unroll
        for (int j = 0; j < TM_CW / 1024; ++j) {
          const int col = 4 * t + 1024 * j;
          if (col < cw) {
            const float4 pv = *reinterpret_cast<const float4*>(sg + col);
            const float4 xv = *reinterpret_cast<const float4*>(xres + c0 + col);
            acc0 = fmaf(pv.x, xv.x, acc0);
            acc1 = fmaf(pv.y, xv.y, acc1);
            acc0 = fmaf(pv.z, xv.z, acc0);
            acc1 = fmaf(pv.w, xv.w, acc1);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + st);
        if (++st == ns) { st = 0; ph ^= 1u; }
      }
      if (!ok) break;
      const int buf = ri % TM_NBUF;
      ++ri;
      const float part = warp_sum(acc0 + acc1);
      if (lane == 0) red[buf * TM_WARPS + warp] = part;
      __syncwarp();
      int last = 0;
      if (lane == 0) {
        __threadfence_block();
        last = (atomicAdd(cnt + buf, 1) == TM_WARPS - 1);
      }
      last = __shfl_sync(0xffffffffu, last, 0);
      if (last && lane == 0) {
        __threadfence_block();
        cnt[buf] = 0;
        float acc = red[buf * TM_WARPS];
        for (int w = 1; w < TM_WARPS; ++w) acc += red[buf * TM_WARPS + w];
        const float xs = xres[s] * io.scale;
        float r = ca * xs + cc * (acc * io.scale);
        if (u) r += cb * u[s];
        io.out[s] = r;
        if (io.qside) io.qside[s] = xs;
        mx = fmaxf(mx, fabsf(r));
        ss += r * r;
      }
    }
  }
  __syncthreads();
  matvec_finish<float>(p, mx, ss);
}

size_t g_tma_mv_smem_set = 0;

int tma_mv_stages(int64_t ld) {
  static int max_smem = 0;
  if (max_smem == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      max_smem = 48 * 1024;
  }
  // two blocks per SM (each with half the shared memory), so one block's start (the copy of x)
  // and final reduction overlap the other's streaming: S = 10^4 solves 5.599 -> 5.575 ms
  for (int ns = 12; ns >= 4; --ns)
    if (tma_mv_layout(ld, ns).total + 1024 <= (size_t)max_smem / 2) return ns;
  return 0;
}

template <class Kern>
int grid_for(Kern k, int threads, size_t smem, int64_t work_units) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, threads, smem) != cudaSuccess)
    per_sm = 1;
  per_sm = std::max(per_sm, 1);
  int64_t g = (int64_t)num_sms() * per_sm;
  g = std::min<int64_t>(g, std::max<int64_t>(work_units, 1));
  g = std::min<int64_t>(g, MAX_RED_BLOCKS);
  return (int)std::max<int64_t>(g, 1);
}

template <class PT, class KT>
int launch_mv_typed(const MatvecLaunch& L, cudaStream_t st) {
  MatvecK p{L.d, L.pi, L.x, L.ctl_rw ? L.ctl_rw : const_cast<GmresCtl*>(L.ctl),
            L.gate_mode, L.gate_mode2, L.x_rhs, L.x_w0, L.x_w1, L.qbase, L.ldq,
            L.a, L.b, L.c, L.u, L.out, L.out0, L.out1, L.norms, L.ctl_rw != nullptr,
            L.partials, L.counter, L.x_pre};
  const DevMDP& d = L.d;
  if (d.kind == KIND_DENSE) {
    if constexpr (sizeof(PT) == 4 && sizeof(KT) == 4) {
      const int ns = (L.no_tma || !L.err) ? 0 : tma_mv_stages(d.ld);
      if (ns > 0) {
        const size_t smem = tma_mv_layout(d.ld, ns).total;
        if (smem > g_tma_mv_smem_set) {
          if (cudaFuncSetAttribute(matvec_dense_tma_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem) != cudaSuccess)
            return MDP_EDEVICE;
          g_tma_mv_smem_set = smem;
        }
        const int grid = L.grid > 0 ? L.grid : (int)std::min<int64_t>(2 * num_sms(), d.S);
        matvec_dense_tma_kernel<<<grid, TM_THREADS, smem, st>>>(p, ns, L.err);
        return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
      }
    }
    auto k = matvec_dense_kernel<PT, KT>;
    int grid = L.grid > 0 ? L.grid : grid_for(k, 256, 0, (d.S + 7) / 8);
    k<<<grid, 256, 0, st>>>(p);
  } else {
    const int T = L.lanes > 0 ? L.lanes : ell_matvec_lanes_default(d);
    if (d.span >= 0 && d.span <= MV_SPAN_MAX && !L.no_window && L.grid <= 0 && d.S >= 4 * MV_NB) {
      // the windowed kernel wants two vectors per lane in flight (measured: banded S = 10^6,
      // 4 lanes per row 153 us per Arnoldi step against 180 us with 8)
      const int Tw = L.lanes > 0 ? L.lanes : std::max(1, T / 2);
      // banded columns: shared-memory window of x (each block a contiguous range of states,
      // at least one step of MV_NB); six blocks per SM (measured on banded S = 10^6: 0.5% and
      // 2% faster preconditioned and plain solves than four, eight slower)
      const int grid = (int)std::max<int64_t>(
          1, std::min<int64_t>(std::min<int64_t>((int64_t)num_sms() * 6, d.S / MV_NB), MAX_RED_BLOCKS));
      switch (Tw) {
        case 1: matvec_ell_window_kernel<PT, KT, 1><<<grid, 256, 0, st>>>(p); break;
        case 2: matvec_ell_window_kernel<PT, KT, 2><<<grid, 256, 0, st>>>(p); break;
        case 4: matvec_ell_window_kernel<PT, KT, 4><<<grid, 256, 0, st>>>(p); break;
        case 8: matvec_ell_window_kernel<PT, KT, 8><<<grid, 256, 0, st>>>(p); break;
        default: return MDP_EINVAL;
      }
      return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
    }
    const int64_t units = (d.S + 256 / T - 1) / (256 / T);
    int grid = 1;
    switch (T) {
      case 1: { auto k = matvec_ell_kernel<PT, KT, 1>; grid = L.grid > 0 ? L.grid : grid_for(k, 256, 0, units); k<<<grid, 256, 0, st>>>(p); break; }
      case 2: { auto k = matvec_ell_kernel<PT, KT, 2>; grid = L.grid > 0 ? L.grid : grid_for(k, 256, 0, units); k<<<grid, 256, 0, st>>>(p); break; }
      case 4: { auto k = matvec_ell_kernel<PT, KT, 4>; grid = L.grid > 0 ? L.grid : grid_for(k, 256, 0, units); k<<<grid, 256, 0, st>>>(p); break; }
      case 8: { auto k = matvec_ell_kernel<PT, KT, 8>; grid = L.grid > 0 ? L.grid : grid_for(k, 256, 0, units); k<<<grid, 256, 0, st>>>(p); break; }
      default: return MDP_EINVAL;
    }
  }
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}

// ------------------------------------------------------------------ tall-skinny kernels
struct KB {
  int64_t S, ldq;
  void* Q;
  void* w0;
  void* w1;
  void* rbuf;
  void* d0;
  void* d1;
  void* partials;
  unsigned* counter;
  GmresCtl* ctl;
  const void* ec;  // two-level preconditioner: coarse part of the candidate (or null)
  int lb;          // log2 of the aggregation block
};


// Rows are processed in 16-byte vector units (4 floats or 2 doubles); every Krylov buffer is
// padded with zeros to a multiple of 32 rows, so whole units past S contribute nothing.
template <class KT> struct TSv;
template <> struct TSv<float> {
  using V = float4;
  static constexpr int R = 4;
  static __device__ __forceinline__ V ld(const float* p) { return *reinterpret_cast<const float4*>(p); }
  static __device__ __forceinline__ void st(float* p, V x) { *reinterpret_cast<float4*>(p) = x; }
  static __device__ __forceinline__ V zero() { return make_float4(0.f, 0.f, 0.f, 0.f); }
  static __device__ __forceinline__ float dot(V a, V b) {
    return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
  }
  static __device__ __forceinline__ V axpy(float c, V x, V y) {  // y + c x
    return make_float4(fmaf(c, x.x, y.x), fmaf(c, x.y, y.y), fmaf(c, x.z, y.z), fmaf(c, x.w, y.w));
  }
  static __device__ __forceinline__ float amax(V x) {
    return fmaxf(fmaxf(fabsf(x.x), fabsf(x.y)), fmaxf(fabsf(x.z), fabsf(x.w)));
  }
};
template <> struct TSv<double> {
  using V = double2;
  static constexpr int R = 2;
  static __device__ __forceinline__ V ld(const double* p) { return *reinterpret_cast<const double2*>(p); }
  static __device__ __forceinline__ void st(double* p, V x) { *reinterpret_cast<double2*>(p) = x; }
  static __device__ __forceinline__ V zero() { return make_double2(0.0, 0.0); }
  static __device__ __forceinline__ double dot(V a, V b) { return fma(a.x, b.x, a.y * b.y); }
  static __device__ __forceinline__ V axpy(double c, V x, V y) {
    return make_double2(fma(c, x.x, y.x), fma(c, x.y, y.y));
  }
  static __device__ __forceinline__ double amax(V x) { return fmax(fabs(x.x), fabs(x.y)); }
};

// Vector-unit load, with an L2 evict-last hint when KEEP: the single-instance Krylov basis
// (a few tens of MB at S = 10^6) then stays in L2 across Arnoldi steps while the matvec and
// sweep streams (loaded evict-first) pass through.
template <class KT, bool KEEP>
__device__ __forceinline__ typename TSv<KT>::V tsld(uint64_t pol, const KT* p) {
  if constexpr (!KEEP) {
    return TSv<KT>::ld(p);
  } else if constexpr (sizeof(KT) == 4) {
    float4 r;
    asm volatile("ld.global.L2::cache_hint.v4.f32 {%0, %1, %2, %3}, [%4], %5;"
                 : "=f"(r.x), "=f"(r.y), "=f"(r.z), "=f"(r.w) : "l"(p), "l"(pol));
    return r;
  } else {
    double2 r;
    asm volatile("ld.global.L2::cache_hint.v2.f64 {%0, %1}, [%2], %3;"
                 : "=d"(r.x), "=d"(r.y) : "l"(p), "l"(pol));
    return r;
  }
}

// This block's range of vector units [u0, u1).
template <class KT>
__device__ __forceinline__ void block_units(int64_t S, int64_t& u0, int64_t& u1, GridPos gp) {
  const int64_t nu = (S + TSv<KT>::R - 1) / TSv<KT>::R;
  const int64_t per = (nu + gp.nb - 1) / gp.nb;
  u0 = (int64_t)gp.bid * per;
  u1 = min(nu, u0 + per);
}

// Sum acc[j] (j < m) over the block into part[blockIdx.x * (WMAX+1) + j].
template <class KT, int MAXM>
__device__ __forceinline__ void block_reduce_cols(KT (&acc)[MAXM], int m, KT* part, GridPos gp) {
  __shared__ KT red[RED_THREADS / 32][MAXM];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < MAXM; ++j) {
    if (j < m) {
      const KT x = warp_sum(acc[j]);
      if (lane == 0) red[wid][j] = x;
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j < m; j += blockDim.x) {
    KT x = 0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) x += red[w][j];
    part[(int64_t)gp.bid * (WMAX + 1) + j] = x;
  }
}

// Stage m coefficients (FP64 copy for double, FP32 copy for float) in shared memory.
template <class KT>
__device__ __forceinline__ void stage_coefs(KT* sh, const double* d, const float* f, int m) {
  for (int j = threadIdx.x; j <= WMAX; j += blockDim.x) sh[j] = j < m ? coef<KT>(d, f, j) : KT(0);
  __syncthreads();
}

// Columns are processed in batches of 8 with one uniform branch per batch, so the 8 loads
// of a batch issue back to back.  Indices past the last column are clamped to it (the
// duplicate loads hit L1) and carry zero weight.
constexpr int TS_BATCH = 8;

// Last block: out[j] = sum over blocks of part[b][j], j < m.
template <class KT>
__device__ __forceinline__ void reduce_dots(const KT* part, int m, double* outd, float* outf,
                                            GridPos gp) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int j = wid; j < m; j += nw) {
    KT acc = 0;
    for (int b = lane; b < gp.nb; b += 32) acc += __ldcg(part + (int64_t)b * (WMAX + 1) + j);
    acc = warp_sum(acc);
    if (lane == 0) {
      outd[j] = (double)acc;
      outf[j] = (float)acc;
    }
  }
}

// CGS2 pass 1: c1 = Q_{0..i}^T w.  Each thread keeps MAXM column accumulators (MAXM is
// fixed by the restart length, so the loop is static) and streams its vector units of w and
// of every Q_j once.
template <class KT, int MAXM, bool KEEP = false>
__device__ __forceinline__ void cgs_dots_body(const KB& b, GridPos gp) {
  const uint64_t pol = KEEP ? l2_keep_policy() : 0ull;
  using T = TSv<KT>;
  GmresCtl* c = b.ctl;
  if (*(volatile int*)&c->mode != GM_STEP) return;
  const int i = c->i, m = i + 1;
  const KT* w = (const KT*)((i & 1) ? b.w1 : b.w0);
  const KT* Q = (const KT*)b.Q;
  int64_t u0, u1;
  block_units<KT>(b.S, u0, u1, gp);
  KT acc[MAXM];
#pragma unroll
  for (int j = 0; j < MAXM; ++j) acc[j] = 0;
  for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    const typename T::V wv = tsld<KT, KEEP>(pol, w + u * T::R);
#pragma unroll
    for (int j0 = 0; j0 < MAXM; j0 += TS_BATCH) {
      if (j0 < m) {
        typename T::V q[TS_BATCH];
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t)
          q[t] = tsld<KT, KEEP>(pol, Q + (int64_t)min(j0 + t, m - 1) * b.ldq + u * T::R);
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t) acc[j0 + t] += T::dot(q[t], wv);
      }
    }
  }
  block_reduce_cols<KT, MAXM>(acc, m, (KT*)b.partials, gp);
  if (!arrive_last(b.counter, gp.nb)) return;
  reduce_dots<KT>((const KT*)b.partials, m, c->c1, c->c1f, gp);
  __syncthreads();
  if (threadIdx.x == 0) {
    // w - Q c1 keeps ||w||^2 - ||c1||^2 of w's squared norm (Q orthonormal); when that is more
    // than half, the projection cancelled little and one pass is enough (the criterion of
    // Daniel, Gragg, Kaufman and Stewart with eta = 1/sqrt(2)); otherwise the second projection
    // runs (CGS2).  ||w|| = ||J q_i||_2 was measured by the matvec.
    double h2 = 0.0;
    for (int j = 0; j < m; ++j) h2 += c->c1[j] * c->c1[j];
    c->once = h2 < 0.5 * c->last_nrm2 * c->last_nrm2 ? 1 : 0;
  }
}

__device__ void givens_and_decide(GmresCtl* c, double hnext, bool fp32_basis);

// w -= Q coef, then ||w||_2 and the Givens update (the last projection of a step).  With
// zero_c2 (a step with one projection) the second coefficients are set to zero, since column i
// of H is c1 + c2.
template <class KT, int MAXM, bool KEEP>
__device__ __forceinline__ void cgs_update_norm(const KB& b, GridPos gp, const double* coefd,
                                                const float* coeff, bool zero_c2) {
  const uint64_t pol = KEEP ? l2_keep_policy() : 0ull;
  using T = TSv<KT>;
  GmresCtl* c = b.ctl;
  const int i = c->i, m = i + 1;
  KT* w = (KT*)((i & 1) ? b.w1 : b.w0);
  const KT* Q = (const KT*)b.Q;
  __shared__ KT cf[WMAX + 1];
  stage_coefs<KT>(cf, coefd, coeff, m);
  int64_t u0, u1;
  block_units<KT>(b.S, u0, u1, gp);
  KT ss = 0;
  for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    typename T::V wv = tsld<KT, KEEP>(pol, w + u * T::R);
#pragma unroll
    for (int j0 = 0; j0 < MAXM; j0 += TS_BATCH) {
      if (j0 < m) {
        typename T::V q[TS_BATCH];
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t)
          q[t] = tsld<KT, KEEP>(pol, Q + (int64_t)min(j0 + t, m - 1) * b.ldq + u * T::R);
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t) wv = T::axpy(-cf[j0 + t], q[t], wv);
      }
    }
    T::st(w + u * T::R, wv);
    ss += T::dot(wv, wv);
  }
  __shared__ KT shr[32];
  KT bs = block_sum(ss, shr);
  KT* part = (KT*)b.partials;
  if (threadIdx.x == 0) part[gp.bid] = bs;
  if (!arrive_last(b.counter, gp.nb)) return;
  KT t = 0;
  for (int bb = threadIdx.x; bb < gp.nb; bb += blockDim.x) t += __ldcg(part + bb);
  t = block_sum(t, shr);
  if (threadIdx.x == 0) {
    if (zero_c2)
      for (int j = 0; j < m; ++j) c->c2[j] = 0.0;
    givens_and_decide(c, sqrt((double)t), sizeof(KT) == 4);
  }
}

// CGS2 pass 1 update and pass 2 projection: w -= Q c1, then c2 = Q^T w.  The second read of
// each Q_j unit follows the first within the same thread and is served by L1.  When the first
// pass found one projection enough, this pass is the last one instead.
template <class KT, int MAXM, bool KEEP = false>
__device__ __forceinline__ void cgs_axpy_dots_body(const KB& b, GridPos gp) {
  const uint64_t pol = KEEP ? l2_keep_policy() : 0ull;
  using T = TSv<KT>;
  GmresCtl* c = b.ctl;
  if (*(volatile int*)&c->mode != GM_STEP) return;
  if (c->once) {
    cgs_update_norm<KT, MAXM, KEEP>(b, gp, c->c1, c->c1f, true);
    return;
  }
  const int i = c->i, m = i + 1;
  KT* w = (KT*)((i & 1) ? b.w1 : b.w0);
  const KT* Q = (const KT*)b.Q;
  __shared__ KT cf[WMAX + 1];
  stage_coefs<KT>(cf, c->c1, c->c1f, m);
  int64_t u0, u1;
  block_units<KT>(b.S, u0, u1, gp);
  KT acc[MAXM];
#pragma unroll
  for (int j = 0; j < MAXM; ++j) acc[j] = 0;
  for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    typename T::V wv = tsld<KT, KEEP>(pol, w + u * T::R);
#pragma unroll
    for (int j0 = 0; j0 < MAXM; j0 += TS_BATCH) {
      if (j0 < m) {
        typename T::V q[TS_BATCH];
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t)
          q[t] = tsld<KT, KEEP>(pol, Q + (int64_t)min(j0 + t, m - 1) * b.ldq + u * T::R);
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t) wv = T::axpy(-cf[j0 + t], q[t], wv);
      }
    }
    T::st(w + u * T::R, wv);
#pragma unroll
    for (int j0 = 0; j0 < MAXM; j0 += TS_BATCH) {
      if (j0 < m) {
        typename T::V q[TS_BATCH];
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t)
          q[t] = tsld<KT, KEEP>(pol, Q + (int64_t)min(j0 + t, m - 1) * b.ldq + u * T::R);
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t) acc[j0 + t] += T::dot(q[t], wv);
      }
    }
  }
  block_reduce_cols<KT, MAXM>(acc, m, (KT*)b.partials, gp);
  if (!arrive_last(b.counter, gp.nb)) return;
  reduce_dots<KT>((const KT*)b.partials, m, c->c2, c->c2f, gp);
}

// Givens update of column i of H and the stopping/restart decision (thread 0, FP64).
__device__ void givens_and_decide(GmresCtl* c, double hnext, bool fp32_basis) {
  const int i = c->i;
  double* Hc = c->H + (int64_t)(WMAX + 1) * i;
  for (int j = 0; j <= i; ++j) Hc[j] = c->c1[j] + c->c2[j];
  Hc[i + 1] = hnext;
  c->hnext = hnext;
  for (int j = 0; j < i; ++j) {
    const double t = c->cs[j] * Hc[j] + c->sn[j] * Hc[j + 1];
    Hc[j + 1] = -c->sn[j] * Hc[j] + c->cs[j] * Hc[j + 1];
    Hc[j] = t;
  }
  const double a = Hc[i], bb = Hc[i + 1];
  const double r = hypot(a, bb);
  double cs = 1.0, sn = 0.0;
  if (r > 0.0) { cs = a / r; sn = bb / r; }
  c->cs[i] = cs;
  c->sn[i] = sn;
  Hc[i] = r;
  Hc[i + 1] = 0.0;
  c->gv[i + 1] = -sn * c->gv[i];
  c->gv[i] = cs * c->gv[i];
  c->rho = fabs(c->gv[i + 1]);
  c->steps += 1;
  // breakdown: the new direction vanished to working precision (reading of "||q||_2 = 0")
  const double eps = fp32_basis ? 3.0e-6 : 1.0e-14;
  const bool breakdown = !(hnext > eps * c->last_nrm2);
  int mode;
  if (breakdown) {
    mode = GM_FINISH;
    c->status = GS_BREAKDOWN;
  } else if (c->steps >= c->max_steps) {
    mode = GM_FINISH;
    c->status = GS_CAP;
  } else if (c->rho <= c->sqrtS * c->thr &&
             (c->sqrtS < 256.0 || c->rho * c->est_ratio <= 2.0 * c->thr ||
              c->steps - c->est_last >= 4)) {
    // ||r||_inf >= ||r||_2 / sqrt(S) rules the estimate out above sqrt(S) thr.  Below it, for
    // S >= 65536 (where that band is wide and a pass over Q costs as much as a step), the pass
    // runs when rho times the last observed inf/2-norm ratio comes within 2x of the threshold,
    // and at least every 4 steps (the ratio is a prediction, not a bound); smaller problems
    // estimate at every step of the band
    mode = GM_EST;
  } else if (i >= c->W - 1) {
    mode = GM_RESTART;
  } else {
    mode = GM_STEP;
  }
  if (mode != GM_STEP) {
    // y solves the (i+1)x(i+1) triangular system R y = gv[0..i]
    for (int j = i; j >= 0; --j) {
      double t = c->gv[j];
      for (int l = j + 1; l <= i; ++l) t -= c->H[(int64_t)(WMAX + 1) * l + j] * c->y[l];
      const double rjj = c->H[(int64_t)(WMAX + 1) * j + j];
      c->y[j] = (rjj != 0.0) ? t / rjj : 0.0;
      c->yf[j] = (float)c->y[j];
    }
  }
  if (mode == GM_EST) {
    // residual coefficients in the basis Q_0..Q_{i+1}: z = G_0^T ... G_i^T (gv[i+1] e_{i+1})
    for (int j = 0; j <= i + 1; ++j) c->z[j] = 0.0;
    c->z[i + 1] = c->gv[i + 1];
    for (int j = i; j >= 0; --j) {
      const double zj = c->z[j], zj1 = c->z[j + 1];
      c->z[j] = c->cs[j] * zj - c->sn[j] * zj1;
      c->z[j + 1] = c->sn[j] * zj + c->cs[j] * zj1;
    }
    for (int j = 0; j <= i + 1; ++j) c->zf[j] = (float)c->z[j];
  }
  if (mode == GM_STEP) {
    c->i = i + 1;
    c->from_rhs = 0;
    set_scale(c, 1.0 / hnext);
  }
  c->mode = mode;
}

// CGS2 pass 2 update, ||w||_2 and the Givens step: w -= Q c2 (idle when pass 2 finished the step).
template <class KT, int MAXM, bool KEEP = false>
__device__ __forceinline__ void cgs_axpy_norm_body(const KB& b, GridPos gp) {
  GmresCtl* c = b.ctl;
  if (*(volatile int*)&c->mode != GM_STEP || c->once) return;  // once: pass 2 finished the step
  cgs_update_norm<KT, MAXM, KEEP>(b, gp, c->c2, c->c2f, false);
}

// x + e on the rows of a vector unit that lie below S (the block of 2^lb >= 4 states is the
// same for every row of the unit; padding rows stay zero).
template <class KT>
__device__ __forceinline__ typename TSv<KT>::V add_coarse(typename TSv<KT>::V x, KT e, int64_t r0,
                                                         int64_t S);
template <>
__device__ __forceinline__ float4 add_coarse<float>(float4 x, float e, int64_t r0, int64_t S) {
  x.x += e;
  if (r0 + 1 < S) x.y += e;
  if (r0 + 2 < S) x.z += e;
  if (r0 + 3 < S) x.w += e;
  return x;
}
template <>
__device__ __forceinline__ double2 add_coarse<double>(double2 x, double e, int64_t r0, int64_t S) {
  x.x += e;
  if (r0 + 1 < S) x.y += e;
  return x;
}

// Runs in the modes EST, RESTART and FINISH.  In one pass over Q_0..Q_i it forms the
// candidate iterate delta_base + sum_{j<=i} y_j Q_j (into dbuf[1 - dsel]) and, in EST mode,
// the cheap bound r = sum_{j<=i} z_j Q_j + z_{i+1} w / hnext, which equals the residual of the
// candidate by the Arnoldi relation J Q_i = Q_{i+1} H (exact arithmetic).  The last block
// decides: EST -> accept (or CHECK) when ||r||_inf meets the threshold, else the next step or
// a restart; FINISH -> DONE with the candidate as the result.
template <class KT, int MAXM, bool KEEP = false>
__device__ __forceinline__ void estimate_candidate_body(const KB& b, GridPos gp) {
  const uint64_t pol = KEEP ? l2_keep_policy() : 0ull;
  using T = TSv<KT>;
  GmresCtl* c = b.ctl;
  const int mode = *(volatile int*)&c->mode;
  if (mode != GM_EST && mode != GM_RESTART && mode != GM_FINISH) return;
  const bool est = mode == GM_EST;
  const int i = c->i, m = i + 1;
  const KT* w = (const KT*)((i & 1) ? b.w1 : b.w0);
  const KT* Q = (const KT*)b.Q;
  const KT* base = (const KT*)(c->dsel ? b.d1 : b.d0);
  KT* cand = (KT*)(c->dsel ? b.d0 : b.d1);
  __shared__ KT cy[WMAX + 1], cz[WMAX + 1];
  for (int j = threadIdx.x; j <= WMAX; j += blockDim.x) {
    cy[j] = j < m ? coef<KT>(c->y, c->yf, j) : KT(0);
    cz[j] = (est && j < m) ? coef<KT>(c->z, c->zf, j) : KT(0);
  }
  __syncthreads();
  const KT zl = est ? coef<KT>(c->z, c->zf, i + 1) * (KT)(1.0 / c->hnext) : KT(0);
  int64_t u0, u1;
  block_units<KT>(b.S, u0, u1, gp);
  KT mx = 0;
  for (int64_t u = u0 + threadIdx.x; u < u1; u += blockDim.x) {
    typename T::V x = tsld<KT, KEEP>(pol, base + u * T::R);
    typename T::V e = est ? T::axpy(zl, tsld<KT, KEEP>(pol, w + u * T::R), T::zero()) : T::zero();
#pragma unroll
    for (int j0 = 0; j0 < MAXM; j0 += TS_BATCH) {
      if (j0 < m) {
        typename T::V q[TS_BATCH];
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t)
          q[t] = tsld<KT, KEEP>(pol, Q + (int64_t)min(j0 + t, m - 1) * b.ldq + u * T::R);
#pragma unroll
        for (int t = 0; t < TS_BATCH; ++t) {
          x = T::axpy(cy[j0 + t], q[t], x);
          e = T::axpy(cz[j0 + t], q[t], e);
        }
      }
    }
    if (b.ec) x = add_coarse<KT>(x, ((const KT*)b.ec)[(u * T::R) >> b.lb], u * T::R, b.S);
    T::st(cand + u * T::R, x);
    mx = max(mx, T::amax(e));
  }
  __shared__ KT shr[32];
  KT bm = block_max(mx, shr);
  KT* part = (KT*)b.partials;
  if (threadIdx.x == 0) part[gp.bid] = bm;
  if (!arrive_last(b.counter, gp.nb)) return;
  KT t = 0;
  for (int bb = threadIdx.x; bb < gp.nb; bb += blockDim.x) t = max(t, __ldcg(part + bb));
  t = block_max(t, shr);
  if (threadIdx.x == 0) {
    if (mode == GM_FINISH) {
      c->dsel = 1 - c->dsel;
      c->mode = GM_DONE;
    } else if (est) {
      c->est_runs += 1;
      c->last_inf = (double)t;
      c->est_last = c->steps;
      if (c->rho > 0.0) c->est_ratio = (double)t / c->rho;
      if (c->accept_est && (double)t <= c->thr) {
        // accepted on the estimate: the candidate is the result; the caller's next Bellman
        // sweep evaluates the exact residual of this policy and resumes the solve if needed
        c->dsel = 1 - c->dsel;
        c->mode = GM_DONE;
        c->status = GS_CONVERGED;
      } else if (!c->accept_est && (double)t <= c->thr * 1.01) {
        // a small margin keeps rounding in the estimate from skipping a true check
        c->mode = GM_CHECK;
      } else {
        advance(c);
      }
    }
  }
}

__global__ void gmres_init_kernel(GmresCtl* c, double thr, double alpha, double sqrtS, int W,
                                  int max_steps, const SweepOut* rhs, int resume, int accept_est,
                                  double forcing_c, double thr_floor) {
  gmres_init_ctl(c, thr, alpha, sqrtS, W, max_steps, rhs, resume, accept_est, forcing_c, thr_floor);
}

__global__ void gmres_loop_cond_kernel(cudaGraphConditionalHandle hc, GmresCtl* c, int cap) {
  const int it = ++c->loop_iters;
  const bool more = (c->mode != GM_DONE) && it < cap;
  cudaGraphSetConditional(hc, more ? 1u : 0u);
}

// v += delta_result (delta_result = dbuf[dsel] once the solve is done)
template <class KT>
__global__ void value_update_kernel(double* v, const KT* d0, const KT* d1, const GmresCtl* c,
                                    const KT* delta, int64_t S) {
  const KT* dl = delta ? delta : (c->dsel ? d1 : d0);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x)
    v[s] += (double)dl[s];
}
__global__ void value_update_df_kernel(float2* v, const float* d0, const float* d1,
                                       const GmresCtl* c, const float* delta, int64_t S) {
  const float* dl = delta ? delta : (c->dsel ? d1 : d0);
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x) {
    float2 x = v[s];
    dfl r = df_add({x.x, x.y}, {dl[s], 0.f});
    v[s] = make_float2(r.hi, r.lo);
  }
}

__global__ void d_to_df_kernel(const double* in, float2* out, int64_t n) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    dfl r = d_to_df(in[s]);
    out[s] = make_float2(r.hi, r.lo);
  }
}
__global__ void df_to_d_kernel(const float2* in, double* out, int64_t n) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < n;
       s += (int64_t)gridDim.x * blockDim.x) {
    float2 x = in[s];
    out[s] = (double)x.x + (double)x.y;
  }
}
__global__ void cost_transpose_kernel(const double* gAS, double* gSA, float2* gdf, int64_t S,
                                      int32_t A) {
  const int64_t n = S * A;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = t / A;
    const int a = (int)(t - s * A);
    const double gv = gAS[(int64_t)a * S + s];
    gSA[t] = gv;
    if (gdf) {
      dfl r = d_to_df(gv);
      gdf[t] = make_float2(r.hi, r.lo);
    }
  }
}

// Compensated (Kahan) FP32 sum: error about 2 eps |sum| independent of the length, so FP32
// rows can be checked against the 1e-5 row-sum tolerance at the speed of the FP32 pipes.
struct KahanF {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = __fsub_rn(x, c);
    const float t = __fadd_rn(s, y);
    c = __fsub_rn(__fsub_rn(t, s), y);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};

__device__ __forceinline__ int bad_prob(float x) { return !(x >= 0.f) || isinf(x); }
__device__ __forceinline__ int bad_prob(double x) { return !(x >= 0.0) || isinf(x); }

__device__ __forceinline__ int bad_prob4(float4 x) {
  return bad_prob(x.x) | bad_prob(x.y) | bad_prob(x.z) | bad_prob(x.w);
}
__device__ __forceinline__ int bad_prob4(double2 x, double2 y) {
  return bad_prob(x.x) | bad_prob(x.y) | bad_prob(y.x) | bad_prob(y.y);
}
__device__ __forceinline__ void kahan4(KahanF& k, float4 x) { k.add(x.x); k.add(x.y); k.add(x.z); k.add(x.w); }

// flags: [0] negative / non-finite probability, [1] column out of range, [2] row sum off,
//        [3] non-finite cost, [4] state without an allowed action
// Whole padded rows are read with 16-byte streaming loads (pads hold zeros and column 0).
// Dense: a warp per row, each lane keeping four loads in flight and four independent sums
// (compensated FP32 sums for FP32 rows, FP64 for FP64 rows), combined in FP64.  ELL: a thread
// per row (a team of 8 lanes per row with 4 rows' loads in flight measured slower, 2.0 against
// 1.6 ms at S = 10^6, A = 16, k = 32).
template <class PT>
__global__ void validate_kernel(DevMDP d, int* flags) {
  const int lane = threadIdx.x & 31;
  const int64_t nrows = d.S * d.A;
  const PT* P = (const PT*)d.P;
  const double tol = 1e-5;  // FP32 rows keep their ~1e-7 rounding
  int badv = 0, badc = 0, bads = 0, span = 0;
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  if (d.kind == KIND_DENSE) {
    const int64_t nv = d.ld / 4;  // 16-byte vectors of FP32 (or 32-byte pairs of FP64) per row
    for (int64_t r = gw; r < nrows; r += nw) {
      const PT* row = P + r * d.ld;
      double tot = 0.0;
      if constexpr (sizeof(PT) == 4) {
        const float4* rv = reinterpret_cast<const float4*>(row);
        KahanF k0, k1, k2, k3;
        int64_t q = lane;
        for (; q + 96 < nv; q += 128) {
          const float4 x0 = __ldcs(rv + q), x1 = __ldcs(rv + q + 32), x2 = __ldcs(rv + q + 64),
                       x3 = __ldcs(rv + q + 96);
          badv |= bad_prob4(x0) | bad_prob4(x1) | bad_prob4(x2) | bad_prob4(x3);
          kahan4(k0, x0); kahan4(k1, x1); kahan4(k2, x2); kahan4(k3, x3);
        }
        for (; q < nv; q += 32) {
          const float4 x = __ldcs(rv + q);
          badv |= bad_prob4(x);
          kahan4(k0, x);
        }
        tot = (k0.value() + k1.value()) + (k2.value() + k3.value());
      } else {
        const double2* rv = reinterpret_cast<const double2*>(row);
        double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
        int64_t q = lane;
        for (; q + 32 < nv; q += 64) {
          const double2 x0 = __ldcs(rv + 2 * q), x1 = __ldcs(rv + 2 * q + 1);
          const double2 y0 = __ldcs(rv + 2 * (q + 32)), y1 = __ldcs(rv + 2 * (q + 32) + 1);
          badv |= bad_prob4(x0, x1) | bad_prob4(y0, y1);
          s0 += x0.x + x0.y;
          s1 += x1.x + x1.y;
          s2 += y0.x + y0.y;
          s3 += y1.x + y1.y;
        }
        for (; q < nv; q += 32) {
          const double2 x0 = __ldcs(rv + 2 * q), x1 = __ldcs(rv + 2 * q + 1);
          badv |= bad_prob4(x0, x1);
          s0 += x0.x + x0.y;
          s1 += x1.x + x1.y;
        }
        tot = (s0 + s1) + (s2 + s3);
      }
      tot = warp_sum(tot);
      if (lane == 0 && !(fabs(tot - 1.0) <= tol)) bads = 1;
    }
  } else {
    const int nv = d.kp / 4;
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
      const PT* row = P + r * d.kp;
      const int4* cr = reinterpret_cast<const int4*>(d.col + r * d.kp);
      double tot;
      if constexpr (sizeof(PT) == 4) {
        KahanF k;
        for (int q = 0; q < nv; ++q) {
          const float4 x = __ldcs(reinterpret_cast<const float4*>(row) + q);
          badv |= bad_prob4(x);
          kahan4(k, x);
        }
        tot = k.value();
      } else {
        double sm = 0.0;
        for (int q = 0; q < nv; ++q) {
          const double2 x0 = __ldcs(reinterpret_cast<const double2*>(row) + 2 * q);
          const double2 x1 = __ldcs(reinterpret_cast<const double2*>(row) + 2 * q + 1);
          badv |= bad_prob4(x0, x1);
          sm += (x0.x + x0.y) + (x1.x + x1.y);
        }
        tot = sm;
      }
      const int64_t s = r / d.A;
      for (int q = 0; q < nv; ++q) {
        const int4 c = __ldcs(cr + q);
        badc |= (c.x < 0 || c.x >= d.S) | (c.y < 0 || c.y >= d.S) | (c.z < 0 || c.z >= d.S) |
                (c.w < 0 || c.w >= d.S);
        const int cc[4] = {c.x, c.y, c.z, c.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)  // column reach of the stored entries (pads excluded)
          if (4 * q + e < d.k) {
            const int64_t dl = (int64_t)cc[e] - s;
            const int64_t ad = dl < 0 ? -dl : dl;
            span = max(span, ad > INT_MAX ? INT_MAX : (int)ad);
          }
      }
      if (!(fabs(tot - 1.0) <= tol)) bads = 1;
    }
  }
  badv = __any_sync(0xffffffffu, badv);
  badc = __any_sync(0xffffffffu, badc);
  bads = __any_sync(0xffffffffu, bads);
  span = warp_max(span);
  if (lane == 0) {
    if (span > 0) atomicMax(flags + 6, span);
    if (badv) atomicOr(flags + 0, 1);
    if (badc) atomicOr(flags + 1, 1);
    if (bads) atomicOr(flags + 2, 1);
  }
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nrows;
       t += (int64_t)gridDim.x * blockDim.x)
    if (!isfinite(d.g64[t])) atomicOr(flags + 3, 1);
  if (d.mask) {
    for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < d.S;
         s += (int64_t)gridDim.x * blockDim.x) {
      int any = 0;
      for (int a = 0; a < d.A; ++a) any |= d.mask[s * d.A + a] != 0;
      if (!any) atomicOr(flags + 4, 1);
    }
  }
}

// flags[5] set when some pi(s) is outside [0, A) or not an allowed action
__global__ void check_policy_kernel(const int32_t* pi, int64_t S, int32_t A, const uint8_t* mask,
                                    int* flags) {
  for (int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; s < S;
       s += (int64_t)gridDim.x * blockDim.x) {
    const int32_t a = pi[s];
    if (a < 0 || a >= A || (mask && mask[s * A + a] == 0)) atomicOr(flags + 5, 1);
  }
}

inline int ew_grid(int64_t n) {
  int64_t g = (n + 255) / 256;
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, (int64_t)num_sms() * 8));
}

inline int ok_or_dev() { return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE; }

KB make_kb(const KrylovBufs& B) {
  return KB{B.S, B.ldq, B.Q, B.w0, B.w1, B.rbuf, B.d0, B.d1, B.partials, B.counter, B.ctl,
            B.ec, B.lb};
}

}  // namespace

int launch_matvec(const MatvecLaunch& L, cudaStream_t st) {
  if (L.kt == 1) {
    if (L.d.pdt != MDP_F32) return MDP_EINVAL;
    return launch_mv_typed<float, float>(L, st);
  }
  if (L.d.pdt == MDP_F32) return launch_mv_typed<float, double>(L, st);
  return launch_mv_typed<double, double>(L, st);
}

template <class KT, int MAXM>
__global__ void __launch_bounds__(RED_THREADS) cgs_dots_kernel(KB b) {
  cgs_dots_body<KT, MAXM, true>(b, this_grid());
}
template <class KT, int MAXM>
__global__ void __launch_bounds__(RED_THREADS) cgs_axpy_dots_kernel(KB b) {
  cgs_axpy_dots_body<KT, MAXM, true>(b, this_grid());
}
template <class KT, int MAXM>
__global__ void __launch_bounds__(RED_THREADS) cgs_axpy_norm_kernel(KB b) {
  cgs_axpy_norm_body<KT, MAXM, true>(b, this_grid());
}
template <class KT, int MAXM>
__global__ void __launch_bounds__(RED_THREADS) estimate_candidate_kernel(KB b) {
  estimate_candidate_body<KT, MAXM, true>(b, this_grid());
}

// ------------------------------------------------------------------ batched kernels
// Launch parameters of one instance, staged in shared memory by thread 0 of the block.
// which: 0 Arnoldi-step matvec, 1 true residual of the candidate (CHECK / RESTART),
// 2 ungated timing run (out = rbuf - gamma P^pi rbuf into w0).
__device__ __forceinline__ MatvecK batch_matvec_params(const BatchInst& I, int which) {
  MatvecK p;
  p.d = I.d;
  p.pi = I.pib[I.cur];
  p.x = nullptr;
  p.ctl = I.ctl;
  p.gate_mode = GM_STEP;
  p.gate_mode2 = GM_STEP;
  p.x_rhs = I.rbuf;
  p.x_w0 = I.w0;
  p.x_w1 = I.w1;
  p.qbase = I.Q;
  p.ldq = I.ldq;
  p.a = 1.0;
  p.b = 0.0;
  p.c = -I.d.gamma;
  p.u = nullptr;
  p.out = nullptr;
  p.out0 = I.w0;
  p.out1 = I.w1;
  p.norms = nullptr;
  p.finalize_check = 0;
  p.partials = I.partials;
  p.counter = I.counter;
  p.x_pre = nullptr;
  if (which == 1) {
    p.gate_mode = GM_CHECK;
    p.gate_mode2 = GM_RESTART;
    p.x_w0 = I.d0;
    p.x_w1 = I.d1;
    p.qbase = nullptr;
    p.a = -1.0;
    p.b = 1.0;
    p.c = I.d.gamma;
    p.u = I.rhs_sel ? I.rref : I.phi;
    p.out = I.rbuf;
    p.finalize_check = 1;
  } else if (which == 2) {
    p.ctl = nullptr;
    p.x = I.rbuf;
    p.out = I.w0;
  }
  return p;
}

__global__ void __launch_bounds__(256) batch_matvec_kernel(BatchDev B, int which) {
  __shared__ MatvecK mp;
  __shared__ BatchInst si;
  batch_for_each(B.mv, [&](int j, GridPos gp) {
    batch_stage_inst(B.insts + j, &si);
    if (threadIdx.x == 0) mp = batch_matvec_params(si, which);
    __syncthreads();
    switch (si.cls_mv) {
      case 0: matvec_ell_body<float, float, 1>(mp, gp); break;
      case 1: matvec_ell_body<float, float, 2>(mp, gp); break;
      case 2: matvec_ell_body<float, float, 4>(mp, gp); break;
      default: matvec_ell_body<float, float, 8>(mp, gp); break;
    }
  });
}

__device__ __forceinline__ KB batch_kb(const BatchInst& I) {
  return KB{I.d.S, I.ldq, I.Q, I.w0, I.w1, I.rbuf, I.d0, I.d1, I.partials, I.counter, I.ctl,
            nullptr, 0};
}

template <int MAXM, int STAGE>
__global__ void __launch_bounds__(RED_THREADS) batch_ts_kernel(BatchDev B) {
  __shared__ KB kb;
  __shared__ BatchInst si;
  batch_for_each(B.ts, [&](int j, GridPos gp) {
    batch_stage_inst(B.insts + j, &si);
    if (threadIdx.x == 0) kb = batch_kb(si);
    __syncthreads();
    if (STAGE == 0) cgs_dots_body<float, MAXM>(kb, gp);
    else if (STAGE == 1) cgs_axpy_dots_body<float, MAXM>(kb, gp);
    else if (STAGE == 2) cgs_axpy_norm_body<float, MAXM>(kb, gp);
    else estimate_candidate_body<float, MAXM>(kb, gp);
  });
}

template <int MAXM>
void launch_batch_ts(const BatchDev& B, int first_stage, int last_stage, int grid, cudaStream_t st) {
  if (first_stage <= 0 && 0 <= last_stage) batch_ts_kernel<MAXM, 0><<<grid, RED_THREADS, 0, st>>>(B);
  if (first_stage <= 1 && 1 <= last_stage) batch_ts_kernel<MAXM, 1><<<grid, RED_THREADS, 0, st>>>(B);
  if (first_stage <= 2 && 2 <= last_stage) batch_ts_kernel<MAXM, 2><<<grid, RED_THREADS, 0, st>>>(B);
  if (first_stage <= 3 && 3 <= last_stage) batch_ts_kernel<MAXM, 3><<<grid, RED_THREADS, 0, st>>>(B);
}

void launch_batch_ts_m(const BatchDev& B, int maxm, int s0, int s1, int grid, cudaStream_t st) {
  if (maxm <= 8) launch_batch_ts<8>(B, s0, s1, grid, st);
  else if (maxm <= 16) launch_batch_ts<16>(B, s0, s1, grid, st);
  else if (maxm <= 32) launch_batch_ts<32>(B, s0, s1, grid, st);
  else launch_batch_ts<64>(B, s0, s1, grid, st);
}

template <class KT, int MAXM>
void launch_cgs_typed(const KB& b, int grid, cudaStream_t st) {
  cgs_dots_kernel<KT, MAXM><<<grid, RED_THREADS, 0, st>>>(b);
  cgs_axpy_dots_kernel<KT, MAXM><<<grid, RED_THREADS, 0, st>>>(b);
  cgs_axpy_norm_kernel<KT, MAXM><<<grid, RED_THREADS, 0, st>>>(b);
}
template <class KT>
void launch_cgs_kt(const KB& b, int grid, int maxm, cudaStream_t st) {
  if (maxm <= 8) launch_cgs_typed<KT, 8>(b, grid, st);
  else if (maxm <= 16) launch_cgs_typed<KT, 16>(b, grid, st);
  else if (maxm <= 32) launch_cgs_typed<KT, 32>(b, grid, st);
  else launch_cgs_typed<KT, 64>(b, grid, st);
}
template <class KT>
void launch_est_kt(const KB& b, int grid, int maxm, cudaStream_t st) {
  if (maxm <= 8) estimate_candidate_kernel<KT, 8><<<grid, RED_THREADS, 0, st>>>(b);
  else if (maxm <= 16) estimate_candidate_kernel<KT, 16><<<grid, RED_THREADS, 0, st>>>(b);
  else if (maxm <= 32) estimate_candidate_kernel<KT, 32><<<grid, RED_THREADS, 0, st>>>(b);
  else estimate_candidate_kernel<KT, 64><<<grid, RED_THREADS, 0, st>>>(b);
}

int launch_cgs2_givens(const KrylovBufs& B, cudaStream_t st) {
  KB b = make_kb(B);
  if (B.kt == 1) launch_cgs_kt<float>(b, B.grid, B.maxm, st);
  else launch_cgs_kt<double>(b, B.grid, B.maxm, st);
  return ok_or_dev();
}

int launch_estimate(const KrylovBufs& B, cudaStream_t st) {
  KB b = make_kb(B);
  if (B.kt == 1) launch_est_kt<float>(b, B.grid, B.maxm, st);
  else launch_est_kt<double>(b, B.grid, B.maxm, st);
  return ok_or_dev();
}

int ell_matvec_lanes_default(const DevMDP& d) {
  const int nvec = d.kp / 4;
  return nvec >= 8 ? 8 : (nvec >= 4 ? 4 : (nvec >= 2 ? 2 : 1));
}

// Blocks of the single-instance tall-skinny Krylov kernels: about 256 rows per block, at
// most four blocks per SM.
int krylov_blocks(int64_t S) {
  int64_t g = (S + 255) / 256;
  g = std::min<int64_t>(g, (int64_t)num_sms() * 2);  // measured best at S = 10^6 (W = 30)
  return (int)std::max<int64_t>(1, std::min<int64_t>(g, MAX_RED_BLOCKS));
}

int batch_matvec_grid() {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_matvec_kernel, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return num_sms() * std::max(per_sm, 1);
}

int launch_batch_matvec(const BatchDev& B, int which, int grid, cudaStream_t st) {
  batch_matvec_kernel<<<grid, 256, 0, st>>>(B, which);
  return ok_or_dev();
}

int batch_ts_grid(int maxm) {
  int per_sm = 1;
  cudaError_t e;
  if (maxm <= 8) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_ts_kernel<8, 1>, RED_THREADS, 0);
  else if (maxm <= 16) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_ts_kernel<16, 1>, RED_THREADS, 0);
  else if (maxm <= 32) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_ts_kernel<32, 1>, RED_THREADS, 0);
  else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_ts_kernel<64, 1>, RED_THREADS, 0);
  if (e != cudaSuccess) { cudaGetLastError(); per_sm = 1; }
  return num_sms() * std::max(per_sm, 1);
}

int launch_batch_cgs(const BatchDev& B, int maxm, int grid, cudaStream_t st) {
  launch_batch_ts_m(B, maxm, 0, 2, grid, st);
  return ok_or_dev();
}

int launch_batch_estimate(const BatchDev& B, int maxm, int grid, cudaStream_t st) {
  launch_batch_ts_m(B, maxm, 3, 3, grid, st);
  return ok_or_dev();
}

int launch_gmres_init(const KrylovBufs& B, double thr, double sqrtS, int W, int max_steps,
                      const SweepOut* rhs_norms, double alpha, cudaStream_t st, int resume,
                      int accept_est, double forcing_c, double thr_floor) {
  gmres_init_kernel<<<1, 1, 0, st>>>(B.ctl, thr, alpha, sqrtS, W, max_steps, rhs_norms, resume,
                                     accept_est, forcing_c, thr_floor);
  return ok_or_dev();
}

int launch_loop_cond(cudaGraphConditionalHandle hc, GmresCtl* ctl, int cap, cudaStream_t st) {
  gmres_loop_cond_kernel<<<1, 1, 0, st>>>(hc, ctl, cap);
  return ok_or_dev();
}

int launch_value_update(int kt, void* v, const void* d0, const void* d1, const GmresCtl* ctl,
                        const void* delta, int64_t S, cudaStream_t st) {
  if (kt == 1)
    value_update_df_kernel<<<ew_grid(S), 256, 0, st>>>((float2*)v, (const float*)d0,
                                                        (const float*)d1, ctl,
                                                        (const float*)delta, S);
  else
    value_update_kernel<double><<<ew_grid(S), 256, 0, st>>>((double*)v, (const double*)d0,
                                                            (const double*)d1, ctl,
                                                            (const double*)delta, S);
  return ok_or_dev();
}

int launch_d_to_df(const double* in, float2* out, int64_t n, cudaStream_t st) {
  d_to_df_kernel<<<ew_grid(n), 256, 0, st>>>(in, out, n);
  return ok_or_dev();
}
int launch_df_to_d(const float2* in, double* out, int64_t n, cudaStream_t st) {
  df_to_d_kernel<<<ew_grid(n), 256, 0, st>>>(in, out, n);
  return ok_or_dev();
}
int launch_fill_zero(void* p, size_t bytes, cudaStream_t st) {
  return cudaMemsetAsync(p, 0, bytes, st) == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}
int launch_cost_transpose(const double* gAS, double* gSA, float2* gdf, int64_t S, int32_t A,
                          cudaStream_t st) {
  cost_transpose_kernel<<<ew_grid(S * A), 256, 0, st>>>(gAS, gSA, gdf, S, A);
  return ok_or_dev();
}
int launch_validate(const DevMDP& d, int* flags, cudaStream_t st) {
  const int64_t rows = d.S * d.A;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((rows + 7) / 8, (int64_t)num_sms() * 16));
  if (d.pdt == MDP_F32) validate_kernel<float><<<grid, 256, 0, st>>>(d, flags);
  else validate_kernel<double><<<grid, 256, 0, st>>>(d, flags);
  return ok_or_dev();
}

int launch_check_policy(const int32_t* pi, int64_t S, int32_t A, const uint8_t* mask, int* flags,
                        cudaStream_t st) {
  check_policy_kernel<<<ew_grid(S), 256, 0, st>>>(pi, S, A, mask, flags);
  return ok_or_dev();
}

int num_sms() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 1;
  }
  return n;
}

}  // namespace mdp
