// Fused Bellman sweep (paper Sec. 2, Bellman operators T^pi and T; Alg. 2 steps
// "pi_k <- GreedyPolicy(V_k)" and "Phi_k <- g^pi_k - J^pi_k V_k"):
//
//   Q(s,a) = g(s,a) + gamma * sum_s' p_ss'(a) v(s')
//   pi(s)  = lowest a in A(s) with minimal Q(s,a),  Tv(s) = Q(s, pi(s)),
//   Phi(s) = Tv(s) - v(s),   ||Phi||_inf, ||Phi||_2,   margin(s) = Q2(s) - Q1(s)
//
// One pass over every P_a row.  With pi_in set the sweep evaluates only row pi_in(s)
// (T^pi v).  Two arithmetics: FP64 (P in FP32 or FP64, v double) and double-float (P FP32,
// v as float2 hi/lo pairs, all sums on the FP32 pipes, ~2^-48 relative).
#include "mdp_internal.cuh"

#include <algorithm>
#include <type_traits>

namespace mdp {

namespace {

// ------------------------------------------------------------------ arithmetic traits
struct ArF64 {
  using V = double;   // value vector element
  using Qt = double;  // Q value
  using K = double;   // Krylov element
  using R = double;   // reduction type
  struct Acc {
    double s;
    __device__ __forceinline__ void init() { s = 0.0; }
    __device__ __forceinline__ void add(double p, double v) { s = fma(p, v, s); }
    __device__ __forceinline__ void add(float p, double v) { s = fma((double)p, v, s); }
    __device__ __forceinline__ void fold() {}
    __device__ __forceinline__ void tick2() {}
    __device__ __forceinline__ double result() { return s; }
  };
  static __device__ __forceinline__ Qt reduce_team(Qt x, int T) {
    for (int o = T >> 1; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    return x;
  }
  static __device__ __forceinline__ Qt qval(const DevMDP& d, int64_t s, int a, Qt sum) {
    return fma(d.gamma, sum, d.g64[s * d.A + a]);
  }
  // the cost, loaded before a row's sum (so its latency overlaps the row) and applied after
  using G = double;
  static __device__ __forceinline__ G gload(const DevMDP& d, int64_t s, int a) { return __ldg(d.g64 + s * d.A + a); }
  static __device__ __forceinline__ Qt qval_g(const DevMDP& d, G g, Qt sum) { return fma(d.gamma, sum, g); }
  static __device__ __forceinline__ Qt inf() { return __longlong_as_double(0x7ff0000000000000LL); }
  static __device__ __forceinline__ bool lt(Qt a, Qt b) { return a < b; }
  static __device__ __forceinline__ Qt sub(Qt a, V b) { return a - b; }
  static __device__ __forceinline__ Qt subq(Qt a, Qt b) { return a - b; }
  static __device__ __forceinline__ double to_d(Qt a) { return a; }
  static __device__ __forceinline__ K to_k(Qt a) { return a; }
  static __device__ __forceinline__ V to_v(Qt a) { return a; }
  static __device__ __forceinline__ R absr(Qt a) { return fabs(a); }
  static __device__ __forceinline__ V load_v(const V* v, int64_t i) { return __ldg(v + i); }
  // running maximum of |Phi| (exact comparison in the arithmetic's own precision)
  using MaxT = double;
  static __device__ __forceinline__ MaxT max0() { return 0.0; }
  static __device__ __forceinline__ MaxT absq(Qt a) { return fabs(a); }
  static __device__ __forceinline__ MaxT mmax(MaxT a, MaxT b) { return max(a, b); }
  static __device__ __forceinline__ MaxT shfl(MaxT a, int o) { return __shfl_xor_sync(0xffffffffu, a, o); }
  static __device__ __forceinline__ double mtod(MaxT a) { return a; }
};

struct ArDF {
  using V = float2;
  using Qt = dfl;
  using K = float;
  using R = float;
  struct Acc {
    AccDF a;
    __device__ __forceinline__ void init() { a.init(); }
    __device__ __forceinline__ void add(float p, float2 v) { a.add(p, v); }
    __device__ __forceinline__ void fold() { a.fold(); }
    __device__ __forceinline__ void tick2() {  // called every 8 terms: fold every 32
      if (++a.n == 4) a.fold();
    }
    __device__ __forceinline__ dfl result() { return a.result(); }
  };
  static __device__ __forceinline__ Qt reduce_team(Qt x, int T) {
    for (int o = T >> 1; o > 0; o >>= 1) x = df_add(x, shfl_xor_df(x, o));
    return x;
  }
  static __device__ __forceinline__ Qt qval(const DevMDP& d, int64_t s, int a, Qt sum) {
    float2 g = __ldg(d.gdf + s * d.A + a);
    return df_add({g.x, g.y}, df_mul(dfl{d.gamma_hi, d.gamma_lo}, sum));
  }
  using G = float2;
  static __device__ __forceinline__ G gload(const DevMDP& d, int64_t s, int a) { return __ldg(d.gdf + s * d.A + a); }
  static __device__ __forceinline__ Qt qval_g(const DevMDP& d, G g, Qt sum) {
    return df_add({g.x, g.y}, df_mul(dfl{d.gamma_hi, d.gamma_lo}, sum));
  }
  static __device__ __forceinline__ Qt inf() { return {__int_as_float(0x7f800000), 0.f}; }
  static __device__ __forceinline__ bool lt(Qt a, Qt b) { return df_lt(a, b); }
  static __device__ __forceinline__ Qt sub(Qt a, V b) { return df_sub(a, dfl{b.x, b.y}); }
  static __device__ __forceinline__ Qt subq(Qt a, Qt b) { return df_sub(a, b); }
  static __device__ __forceinline__ double to_d(Qt a) { return df_to_d(a); }
  static __device__ __forceinline__ K to_k(Qt a) { return __fadd_rn(a.hi, a.lo); }
  static __device__ __forceinline__ V to_v(Qt a) { return make_float2(a.hi, a.lo); }
  static __device__ __forceinline__ R absr(Qt a) { return fabsf(__fadd_rn(a.hi, a.lo)); }
  static __device__ __forceinline__ V load_v(const V* v, int64_t i) { return __ldg(v + i); }
  using MaxT = dfl;
  static __device__ __forceinline__ MaxT max0() { return {0.f, 0.f}; }
  static __device__ __forceinline__ MaxT absq(Qt a) { return a.hi < 0.f ? df_neg(a) : a; }
  static __device__ __forceinline__ MaxT mmax(MaxT a, MaxT b) { return df_lt(a, b) ? b : a; }
  static __device__ __forceinline__ MaxT shfl(MaxT a, int o) { return shfl_xor_df(a, o); }
  static __device__ __forceinline__ double mtod(MaxT a) { return df_to_d(a); }
};

struct SweepK {
  DevMDP d;
  const void* v;
  const int32_t* pi_in;
  int32_t* pi_out;
  void* tv_out;
  double* tv64_out;
  void* phi_out;
  double* margin_out;
  const int32_t* pi_ref;
  void* rref_out;
  SweepOut* out;
  SweepOut* ref_out;
  void* partials;
  unsigned* counter;
};

// Running norms of Phi = Tv - v and of the reference-policy residual.
template <class AR> struct Norms {
  typename AR::MaxT mx, mx2;
  typename AR::R ss, ss2;
  __device__ __forceinline__ void init() {
    mx = AR::max0();
    mx2 = AR::max0();
    ss = 0;
    ss2 = 0;
  }
};

// Running argmin over the actions of one state, lowest index on exact ties.
template <class AR> struct Pick {
  typename AR::Qt best, second, qref;
  int abest;
  __device__ __forceinline__ void init() {
    best = AR::inf(); second = AR::inf(); qref = AR::inf(); abest = -1;
  }
  __device__ __forceinline__ void consider(int a, typename AR::Qt q, bool allowed, int aref) {
    if (a == aref) qref = q;
    if (!allowed) return;
    if (AR::lt(q, best) || abest < 0) {
      second = best; best = q; abest = a;
    } else if (AR::lt(q, second)) {
      second = q;
    }
  }
};

__device__ __forceinline__ dfl shfl_idx_df(dfl x, int src) {
  return {__shfl_sync(0xffffffffu, x.hi, src), __shfl_sync(0xffffffffu, x.lo, src)};
}

template <class AR> __device__ __forceinline__ typename AR::Qt shfl_xor_q(typename AR::Qt x, int off);
template <> __device__ __forceinline__ double shfl_xor_q<ArF64>(double x, int off) {
  return __shfl_xor_sync(0xffffffffu, x, off);
}
template <> __device__ __forceinline__ dfl shfl_xor_q<ArDF>(dfl x, int off) { return shfl_xor_df(x, off); }

template <class AR> __device__ __forceinline__ typename AR::Qt shfl_q(typename AR::Qt x, int src);
template <> __device__ __forceinline__ double shfl_q<ArF64>(double x, int src) {
  return __shfl_sync(0xffffffffu, x, src);
}
template <> __device__ __forceinline__ dfl shfl_q<ArDF>(dfl x, int src) { return shfl_idx_df(x, src); }

// Per-state outputs of a sweep given v(s): pi, Tv, Phi, margin, the residual of the
// reference policy (g(s, pi_ref(s)) + gamma p_s.(pi_ref(s)) v - v(s)), and running norms.
template <class AR>
__device__ __forceinline__ void emit_state_v(const SweepK& p, int64_t s, const Pick<AR>& pk,
                                             typename AR::V vs, Norms<AR>& nm) {
  using V = typename AR::V;
  using K = typename AR::K;
  const typename AR::Qt phi = AR::sub(pk.best, vs);
  int a = pk.abest < 0 ? 0 : pk.abest;
  if (p.pi_in) a = p.pi_in[s];
  if (p.pi_out) p.pi_out[s] = a;
  if (p.tv_out) ((V*)p.tv_out)[s] = AR::to_v(pk.best);
  if (p.tv64_out) p.tv64_out[s] = AR::to_d(pk.best);
  if (p.phi_out) ((K*)p.phi_out)[s] = AR::to_k(phi);
  if (p.margin_out) {
    double m = AR::to_d(pk.second);
    p.margin_out[s] = isinf(m) ? m : AR::to_d(AR::subq(pk.second, pk.best));
  }
  if (p.rref_out) {
    const typename AR::Qt rr = AR::sub(pk.qref, vs);
    ((K*)p.rref_out)[s] = AR::to_k(rr);
    const typename AR::R r2 = AR::absr(rr);
    nm.mx2 = AR::mmax(nm.mx2, AR::absq(rr));
    nm.ss2 += r2 * r2;
  }
  const typename AR::R r = AR::absr(phi);
  nm.mx = AR::mmax(nm.mx, AR::absq(phi));
  nm.ss += r * r;
}

template <class AR>
__device__ __forceinline__ void emit_state(const SweepK& p, int64_t s, const Pick<AR>& pk,
                                           Norms<AR>& nm) {
  emit_state_v<AR>(p, s, pk, AR::load_v((const typename AR::V*)p.v, s), nm);
}

template <class AR>
__device__ __forceinline__ typename AR::MaxT block_maxq(typename AR::MaxT x, typename AR::MaxT* sh) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x = AR::mmax(x, AR::shfl(x, o));
  __syncthreads();
  if (lane == 0) sh[wid] = x;
  __syncthreads();
  typename AR::MaxT r = (threadIdx.x < (blockDim.x >> 5)) ? sh[threadIdx.x] : AR::max0();
  if (wid == 0) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) r = AR::mmax(r, AR::shfl(r, o));
    if (lane == 0) sh[0] = r;
  }
  __syncthreads();
  r = sh[0];
  __syncthreads();
  return r;
}

template <class AR>
__device__ __forceinline__ typename AR::MaxT load_maxt(const typename AR::MaxT* pm, int b) {
  if constexpr (sizeof(typename AR::MaxT) == 8 && sizeof(typename AR::R) == 8) {
    return __ldcg((const double*)pm + b);
  } else {
    const float2 f = __ldcg((const float2*)pm + b);
    return typename AR::MaxT{f.x, f.y};
  }
}

// Block partials -> last block -> out (norms of Phi) and ref_out (norms of the reference
// residual).  Partials: four arrays of MAX_RED_BLOCKS slots of 8 bytes.
template <class AR>
__device__ __forceinline__ void finish_norms(const SweepK& p, const Norms<AR>& nm,
                                             GridPos gp = this_grid()) {
  using R = typename AR::R;
  using M = typename AR::MaxT;
  __shared__ M shm[32];
  __shared__ R shr[32];
  const M bm = block_maxq<AR>(nm.mx, shm);
  const R bs = block_sum(nm.ss, shr);
  const M bm2 = block_maxq<AR>(nm.mx2, shm);
  const R bs2 = block_sum(nm.ss2, shr);
  M* pm = (M*)p.partials;
  M* pm2 = (M*)((char*)p.partials + (size_t)MAX_RED_BLOCKS * 8);
  R* ps = (R*)((char*)p.partials + (size_t)MAX_RED_BLOCKS * 16);
  R* ps2 = (R*)((char*)p.partials + (size_t)MAX_RED_BLOCKS * 24);
  if (threadIdx.x == 0) {
    pm[gp.bid] = bm;
    ps[gp.bid] = bs;
    pm2[gp.bid] = bm2;
    ps2[gp.bid] = bs2;
  }
  if (!arrive_last(p.counter, gp.nb)) return;
  M m = AR::max0(), m2 = AR::max0();
  R t = 0, t2 = 0;
  for (int b = threadIdx.x; b < gp.nb; b += blockDim.x) {
    m = AR::mmax(m, load_maxt<AR>(pm, b));
    m2 = AR::mmax(m2, load_maxt<AR>(pm2, b));
    t += __ldcg(ps + b);
    t2 += __ldcg(ps2 + b);
  }
  m = block_maxq<AR>(m, shm);
  t = block_sum(t, shr);
  m2 = block_maxq<AR>(m2, shm);
  t2 = block_sum(t2, shr);
  if (threadIdx.x == 0) {
    if (p.out) {
      p.out->res_inf = AR::mtod(m);
      p.out->res_nrm2 = sqrt((double)t);
    }
    if (p.ref_out) {
      p.ref_out->res_inf = AR::mtod(m2);
      p.ref_out->res_nrm2 = sqrt((double)t2);
    }
  }
}

// ------------------------------------------------------------------ dense: warp per state
template <class PT> struct Vec4;
// load(): streaming (evict-first) 16-byte loads.  load_cached(): read-only loads with the
// default cache policy, for the windowed ELL sweep, whose lane teams consume each 128-byte line
// of values and columns over two loop iterations: with streaming hints (or with L1 bypassed) L2
// dropped some lines between the two halves, 12% more DRAM reads than the data at S = 10^6.
template <> struct Vec4<float> {
  float e[4];
  __device__ __forceinline__ void load(const float* p) {
    float4 t = __ldcs(reinterpret_cast<const float4*>(p));
    e[0] = t.x; e[1] = t.y; e[2] = t.z; e[3] = t.w;
  }
  __device__ __forceinline__ void load_cached(const float* p) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    e[0] = t.x; e[1] = t.y; e[2] = t.z; e[3] = t.w;
  }
};
template <> struct Vec4<double> {
  double e[4];
  __device__ __forceinline__ void load(const double* p) {
    double2 t0 = __ldcs(reinterpret_cast<const double2*>(p));
    double2 t1 = __ldcs(reinterpret_cast<const double2*>(p) + 1);
    e[0] = t0.x; e[1] = t0.y; e[2] = t1.x; e[3] = t1.y;
  }
  __device__ __forceinline__ void load_cached(const double* p) {
    double2 t0 = __ldg(reinterpret_cast<const double2*>(p));
    double2 t1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    e[0] = t0.x; e[1] = t0.y; e[2] = t1.x; e[3] = t1.y;
  }
};

template <class V> struct VLoad4;
template <> struct VLoad4<double> {
  double e[4];
  __device__ __forceinline__ void load(const double* v) {
    double2 t0 = __ldg(reinterpret_cast<const double2*>(v));
    double2 t1 = __ldg(reinterpret_cast<const double2*>(v) + 1);
    e[0] = t0.x; e[1] = t0.y; e[2] = t1.x; e[3] = t1.y;
  }
};
template <> struct VLoad4<float2> {
  float2 e[4];
  __device__ __forceinline__ void load(const float2* v) {
    float4 t0 = __ldg(reinterpret_cast<const float4*>(v));
    float4 t1 = __ldg(reinterpret_cast<const float4*>(v) + 1);
    e[0] = make_float2(t0.x, t0.y); e[1] = make_float2(t0.z, t0.w);
    e[2] = make_float2(t1.x, t1.y); e[3] = make_float2(t1.z, t1.w);
  }
};

template <class PT, class AR, int AG>
__global__ void __launch_bounds__(256) sweep_dense_kernel(SweepK p) {
  using V = typename AR::V;
  using Qt = typename AR::Qt;
  const DevMDP& d = p.d;
  const int lane = threadIdx.x & 31;
  const int64_t nw = (int64_t)gridDim.x * (blockDim.x >> 5);
  const int R = p.pi_in ? 1 : d.A;
  const PT* P = (const PT*)d.P;
  const V* v = (const V*)p.v;
  Norms<AR> nm;
  nm.init();
  for (int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; s < d.S; s += nw) {
    Pick<AR> pk;
    pk.init();
    const int aref = p.pi_ref ? p.pi_ref[s] : -1;
    for (int a0 = 0; a0 < R; a0 += AG) {
      const int na = min(AG, R - a0);
      const PT* row[AG];
#pragma unroll
      for (int g = 0; g < AG; ++g) {
        int a = p.pi_in ? p.pi_in[s] : min(a0 + g, d.A - 1);
        row[g] = P + ((int64_t)s * d.A + a) * d.ld;
      }
      typename AR::Acc acc[AG];
#pragma unroll
      for (int g = 0; g < AG; ++g) acc[g].init();
      int it = 0;
      for (int64_t c = 4 * lane; c < d.ld; c += 128) {
        VLoad4<V> vv;
        vv.load(v + c);
        Vec4<PT> pv[AG];
#pragma unroll
        for (int g = 0; g < AG; ++g)
          if (g < na) pv[g].load(row[g] + c);
#pragma unroll
        for (int g = 0; g < AG; ++g) {
          if (g < na) {
#pragma unroll
            for (int e = 0; e < 4; ++e) acc[g].add(pv[g].e[e], vv.e[e]);
          }
        }
        if ((++it & 7) == 0) {
#pragma unroll
          for (int g = 0; g < AG; ++g) acc[g].fold();
        }
      }
#pragma unroll
      for (int g = 0; g < AG; ++g) {
        Qt sum = AR::reduce_team(acc[g].result(), 32);
        if (g < na) {
          int a = p.pi_in ? p.pi_in[s] : a0 + g;
          bool allowed = p.pi_in ? true : (d.mask ? d.mask[s * d.A + a] != 0 : true);
          pk.consider(a, AR::qval(d, s, a, sum), allowed, aref);
        }
      }
    }
    if (lane == 0) emit_state<AR>(p, s, pk, nm);
  }
  finish_norms<AR>(p, nm);
}

// ------------------------------------------------------------------ dense, bulk-copy pipeline
// Warp-specialised sweep for FP32 P in double-float arithmetic, A <= 8.
//   warp 16 (producer, one elected thread): streams each state's A row segments of TS_CW
//            columns into a ring of NS shared-memory stages with cp.async.bulk;
//   warps 0..15 (consumers): two columns of every stage for all A rows, against v resident in
//            shared memory; at the end of a state each warp reduce-scatters its A partial sums
//            and hands them over through a small mbarrier-guarded buffer;
//   warp 17 (epilogue): prefetches g, v(s) for the next state, then combines the 16 warps'
//            partials in a fixed order, forms Q = g + gamma * sum, the argmin and the outputs.
// Consumers never stall on global memory; every wait is bounded.
constexpr int TC_WARPS = 16;
constexpr int TC_THREADS = (TC_WARPS + 2) * 32;
constexpr int TS_PRODUCER = TC_WARPS;
constexpr int TS_EPILOGUE = TC_WARPS + 1;
constexpr int TS_CW = 1024;   // columns per stage = 2 per consumer thread
constexpr int TS_RMAX = 8;
constexpr int TS_NBUF = 8;    // partial-sum buffers between consumers and the epilogue warp

struct TmaSweepLayout {
  size_t stage_bytes, vpart, bar_off, red_off, total;
  int ns;
};

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Each stage holds TS_RMAX row segments of TS_CW floats; the consumers read their two
// double-float entries of v from L2 into registers one stage ahead.
__host__ __device__ inline TmaSweepLayout tma_sweep_layout(int64_t /*ld*/, int ns) {
  TmaSweepLayout L;
  L.ns = ns;
  L.vpart = 0;
  L.stage_bytes = (size_t)TS_RMAX * TS_CW * 4;
  L.bar_off = (size_t)ns * L.stage_bytes;
  // full[ns], empty[ns], done[NBUF], free[NBUF]
  L.red_off = align_up(L.bar_off + (size_t)(2 * ns + 2 * TS_NBUF) * 8, 16);
  L.total = align_up(L.red_off + (size_t)TS_NBUF * TC_WARPS * TS_RMAX * sizeof(dfl), 128);
  return L;
}

// Double-word sum with TwoSum on the high words only (the low words are added): error about
// 2^-48 (|x| + |y|), enough for partial sums bounded by ||v||_inf.
__device__ __forceinline__ dfl df_add_fast(dfl x, dfl y) {
  const dfl s = two_sum(x.hi, y.hi);
  return fast_two_sum(s.hi, __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo)));
}

// Sum 8 double-float values per lane over the warp by recursive halving: afterwards the
// lanes with (lane & 3) == 0 hold the warp total of row ((lane>>4)&1)*4 + ((lane>>3)&1)*2 +
// ((lane>>2)&1).  Nine double-float additions per lane instead of forty.
__device__ __forceinline__ dfl warp_reduce_scatter8(const dfl (&a)[TS_RMAX], int lane) {
  dfl b[4], c[2];
  const bool u1 = lane & 16, u2 = lane & 8, u3 = lane & 4;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const dfl snd = u1 ? a[j] : a[j + 4];
    const dfl kep = u1 ? a[j + 4] : a[j];
    b[j] = df_add_fast(kep, shfl_xor_df(snd, 16));
  }
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const dfl snd = u2 ? b[j] : b[j + 2];
    const dfl kep = u2 ? b[j + 2] : b[j];
    c[j] = df_add_fast(kep, shfl_xor_df(snd, 8));
  }
  const dfl snd = u3 ? c[0] : c[1];
  const dfl kep = u3 ? c[1] : c[0];
  dfl d = df_add_fast(kep, shfl_xor_df(snd, 4));
  d = df_add_fast(d, shfl_xor_df(d, 2));
  d = df_add_fast(d, shfl_xor_df(d, 1));
  return d;
}

template <int R>
__global__ void __launch_bounds__(TC_THREADS, 1) sweep_dense_tma_kernel(SweepK p, int ns, int* err) {
  extern __shared__ __align__(128) unsigned char sm[];
  const DevMDP& d = p.d;
  const int64_t ld = d.ld;
  const TmaSweepLayout L = tma_sweep_layout(ld, ns);
  unsigned char* stg = sm;
  uint64_t* full = reinterpret_cast<uint64_t*>(sm + L.bar_off);
  uint64_t* empty = full + ns;
  uint64_t* done = empty + ns;
  uint64_t* freeb = done + TS_NBUF;
  dfl* red = reinterpret_cast<dfl*>(sm + L.red_off);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nch = (int)((ld + TS_CW - 1) / TS_CW);
  if (threadIdx.x == 0) {
    for (int st = 0; st < ns; ++st) {
      mbar_init(full + st, 1);
      mbar_init(empty + st, TC_WARPS);
    }
    for (int b = 0; b < TS_NBUF; ++b) {
      mbar_init(done + b, TC_WARPS);
      mbar_init(freeb + b, 1);
    }
    mbar_fence_init();
  }
  __syncthreads();
  Norms<ArDF> nm;
  nm.init();
  const float* P = (const float*)d.P;
  if (warp == TS_PRODUCER) {
    if (lane == 0) {
      int n = 0;
      bool ok = true;
      for (int64_t s = blockIdx.x; s < d.S && ok; s += gridDim.x) {
        const float* rowbase = P + (int64_t)s * d.A * ld;
        for (int ch = 0; ch < nch; ++ch, ++n) {
          const int st = n % ns;
          if (!mbar_wait(empty + st, (uint32_t)(((n / ns) & 1) ^ 1), err)) { ok = false; break; }
          const int64_t c0 = (int64_t)ch * TS_CW;
          const int cc = (int)((ld - c0) < (int64_t)TS_CW ? (ld - c0) : (int64_t)TS_CW);
          unsigned char* sg = stg + (size_t)st * L.stage_bytes;
          mbar_expect_tx(full + st, (uint32_t)(R * cc * 4));
          for (int r = 0; r < R; ++r)
            bulk_load(sg + (size_t)r * TS_CW * 4, rowbase + (int64_t)r * ld + c0, (uint32_t)cc * 4u,
                      full + st);
        }
      }
      // every issued copy has landed before the block can exit
      for (int k = 1; k <= ns && n - k >= 0; ++k) {
        const int m = n - k;
        mbar_wait(full + (m % ns), (uint32_t)((m / ns) & 1), err);
      }
    }
  } else if (warp == TS_EPILOGUE) {
    int ri = 0;
    int64_t s = blockIdx.x;
    // prefetch the first state's costs, mask and v(s)
    float2 gq = make_float2(0.f, 0.f);
    uint8_t mk = 1;
    float2 vs = make_float2(0.f, 0.f);
    if (s < d.S) {
      if (lane < R) {
        gq = __ldg(d.gdf + s * d.A + lane);
        if (d.mask) mk = d.mask[s * d.A + lane];
      }
      vs = __ldg((const float2*)p.v + s);
    }
    for (; s < d.S; s += gridDim.x, ++ri) {
      const int buf = ri % TS_NBUF;
      // next state's inputs, loaded while this state's partials are still being produced
      const int64_t s2 = s + gridDim.x;
      float2 gq2 = make_float2(0.f, 0.f);
      uint8_t mk2 = 1;
      float2 vs2 = make_float2(0.f, 0.f);
      if (s2 < d.S) {
        if (lane < R) {
          gq2 = __ldg(d.gdf + s2 * d.A + lane);
          if (d.mask) mk2 = d.mask[s2 * d.A + lane];
        }
        vs2 = __ldg((const float2*)p.v + s2);
      }
      if (!mbar_wait(done + buf, (uint32_t)((ri / TS_NBUF) & 1), err)) break;
      dfl q = {0.f, 0.f};
      if (lane < R) {
        q = red[((size_t)buf * TC_WARPS + 0) * TS_RMAX + lane];
        for (int w = 1; w < TC_WARPS; ++w) q = df_add(q, red[((size_t)buf * TC_WARPS + w) * TS_RMAX + lane]);
        q = df_add(dfl{gq.x, gq.y}, df_mul(dfl{d.gamma_hi, d.gamma_lo}, q));
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(freeb + buf);
      Pick<ArDF> pk;
      pk.init();
      const int aref = p.pi_ref ? p.pi_ref[s] : -1;
      for (int a = 0; a < R; ++a) {
        const dfl qa = shfl_idx_df(q, a);
        const int ma = __shfl_sync(0xffffffffu, (int)mk, a);
        pk.consider(a, qa, ma != 0, aref);
      }
      if (lane == 0) emit_state_v<ArDF>(p, s, pk, vs, nm);
      gq = gq2;
      mk = mk2;
      vs = vs2;
    }
  } else {
    // ---------------- consumers
    // Per row two (hi, lo) pairs, for the even and the odd column of the thread, held as packed
    // FP32 pairs (f2_acc): the hi parts gather the high halves of the exact products p*vh with
    // TwoSum, every error term (product error, p*vl, TwoSum error) goes to lo.  Each pair adds
    // one term per stage and row, so up to 16 stages a lo word holds at most 16 error terms;
    // then the pairs are folded into a double-word total.
    const int t = threadIdx.x;  // 0..511
    const int col = 2 * t;
    const int ldi = (int)ld;
    const float4* vq = reinterpret_cast<const float4*>(p.v);  // two double-float entries
    bool ok = true;
    int st = 0, ri = 0;
    uint32_t ph = 0;
    float4 vnext = col < ldi ? __ldg(vq + t) : make_float4(0.f, 0.f, 0.f, 0.f);
    for (int64_t s = blockIdx.x; s < d.S && ok; s += gridDim.x, ++ri) {
      f2x sh[R], sl[R];
      dfl tot[R];
#pragma unroll
      for (int g = 0; g < R; ++g) { sh[g] = 0ull; sl[g] = 0ull; tot[g] = {0.f, 0.f}; }
      for (int c0 = 0, ch = 0; c0 < ldi; c0 += TS_CW, ++ch) {
        const float4 vv = vnext;  // (hi, lo) of columns col and col + 1
        {  // the v entries of the next stage (wrapping to the next state's first chunk)
          const int cn = (c0 + TS_CW < ldi) ? c0 + TS_CW : 0;
          vnext = (cn + col < ldi) ? __ldg(vq + ((cn + col) >> 1)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        if (!mbar_wait(full + st, ph, err)) { ok = false; break; }
        const unsigned char* sg = stg + (size_t)st * L.stage_bytes;
        if (col < ldi - c0) {
          const float* pp = reinterpret_cast<const float*>(sg) + col;
          const f2x vh = f2_pack(vv.x, vv.z), vl = f2_pack(vv.y, vv.w);
          const f2x nvh = f2_pack(-vv.x, -vv.z);
#pragma unroll
          for (int g = 0; g < R; ++g) {
            const f2x pv = *reinterpret_cast<const f2x*>(pp + g * TS_CW);  // p of both columns
            f2_acc(sh[g], sl[g], pv, vh, nvh, vl);
          }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(empty + st);
        if (++st == ns) { st = 0; ph ^= 1u; }
        if ((ch & 15) == 15) {
#pragma unroll
          for (int g = 0; g < R; ++g) {
            tot[g] = df_add(tot[g], f2_to_df(sh[g], sl[g]));
            sh[g] = 0ull;
            sl[g] = 0ull;
          }
        }
      }
      if (!ok) break;
      dfl parts[TS_RMAX];
      const bool folded = ldi > 16 * TS_CW;
#pragma unroll
      for (int g = 0; g < TS_RMAX; ++g) {
        if (g < R) {
          parts[g] = f2_to_df(sh[g], sl[g]);
          if (folded) parts[g] = df_add(tot[g], parts[g]);
        } else {
          parts[g] = {0.f, 0.f};
        }
      }
      const dfl wsum = warp_reduce_scatter8(parts, lane);
      const int buf = ri % TS_NBUF;
      if (!mbar_wait(freeb + buf, (uint32_t)(((ri / TS_NBUF) & 1) ^ 1), err)) break;
      if ((lane & 3) == 0) {
        const int row = ((lane >> 4) & 1) * 4 + ((lane >> 3) & 1) * 2 + ((lane >> 2) & 1);
        red[((size_t)buf * TC_WARPS + warp) * TS_RMAX + row] = wsum;
      }
      __syncwarp();
      if (lane == 0) mbar_arrive(done + buf);
    }
  }
  __syncthreads();
  finish_norms<ArDF>(p, nm);
}

size_t g_tma_sweep_smem_set = 0;

// Stages that fit next to the resident v (0 = the pipeline does not apply).
int tma_sweep_stages(int64_t ld) {
  static int max_smem = 0;
  if (max_smem == 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess)
      max_smem = 48 * 1024;
  }
  for (int ns = 7; ns >= 3; --ns)
    if (tma_sweep_layout(ld, ns).total <= (size_t)max_smem) return ns;
  return 0;
}

// ------------------------------------------------------------------ ELL, warp per state group
// T lanes share a row.  A state's R rows are padded to Rp (a power of two) row slots; a warp
// pass covers 32/T row slots: G = (32/T)/Rp whole states, or one state in ceil(R/(32/T))
// passes when it does not fit.  Each lane issues all loads of a batch of vectors (values,
// columns), then their gathers of v (L2 evict-last), then the arithmetic.  The argmin over a
// state's rows is a butterfly over the lanes that hold them, ordered by (Q, action) so the
// lowest action index wins exact ties; it also carries the second-best Q for the margin.
// No shared memory and no block barrier until the final norm reduction.
template <class AR> struct Cand {
  typename AR::Qt q, q2;  // best and second-best Q
  int a;                  // action of the best (INT_MAX when none)
};

template <class AR>
__device__ __forceinline__ Cand<AR> cand_merge(const Cand<AR>& x, const Cand<AR>& y) {
  const bool xfirst = AR::lt(x.q, y.q) || (!AR::lt(y.q, x.q) && x.a < y.a);
  Cand<AR> r;
  r.q = xfirst ? x.q : y.q;
  r.a = xfirst ? x.a : y.a;
  const typename AR::Qt loser = xfirst ? y.q : x.q;
  typename AR::Qt s2 = AR::lt(x.q2, y.q2) ? x.q2 : y.q2;
  r.q2 = AR::lt(loser, s2) ? loser : s2;
  return r;
}

template <class AR>
__device__ __forceinline__ Cand<AR> cand_shfl(const Cand<AR>& x, int off) {
  Cand<AR> r;
  r.q = shfl_xor_q<AR>(x.q, off);
  r.q2 = shfl_xor_q<AR>(x.q2, off);
  r.a = __shfl_xor_sync(0xffffffffu, x.a, off);
  return r;
}

// Lane roles of the ELL sweep (fixed for a launch).
struct EllLanes {
  int R, Rp, G, npass, rr, tl, g, leader, nvec, T;
};

template <int T>
__device__ __forceinline__ EllLanes ell_lanes(const SweepK& p) {
  EllLanes L;
  const int lane = threadIdx.x & 31;
  L.R = p.pi_in ? 1 : p.d.A;
  constexpr int RPI = 32 / T;                      // row slots per pass
  L.Rp = 1;
  while (L.Rp < L.R && L.Rp < RPI) L.Rp <<= 1;     // row slots of one state per pass
  L.G = RPI / L.Rp;                                // states per pass
  L.npass = (L.R + RPI - 1) / RPI;                 // passes per state
  const int row_slot = lane / T;
  L.tl = lane % T;
  L.g = row_slot / L.Rp;
  L.rr = row_slot % L.Rp;
  L.leader = L.g * L.Rp * T;
  L.nvec = p.d.kp >> 2;
  L.T = T;
  return L;
}

// Gathers of v at a column: from global memory with an L2 evict-last hint, or from a block's
// shared-memory window of v.
template <class AR> struct GatherGlobal {
  static constexpr bool kWindow = false;
  const typename AR::V* v;
  uint64_t pol;
  __device__ __forceinline__ typename AR::V operator()(int c) const { return ld_keep(v + c, pol); }
};
template <class AR> struct GatherRing {
  static constexpr bool kWindow = true;
  const typename AR::V* ring;
  int mask;
  __device__ __forceinline__ typename AR::V operator()(int c) const { return ring[c & mask]; }
};

// Merge without the second-best value (when no margin is asked for).
template <class AR>
__device__ __forceinline__ Cand<AR> cand_merge1(const Cand<AR>& x, const Cand<AR>& y) {
  const bool xfirst = AR::lt(x.q, y.q) || (!AR::lt(y.q, x.q) && x.a < y.a);
  Cand<AR> r;
  r.q = xfirst ? x.q : y.q;
  r.a = xfirst ? x.a : y.a;
  r.q2 = x.q2;
  return r;
}
template <class AR>
__device__ __forceinline__ Cand<AR> cand_shfl1(const Cand<AR>& x, int off) {
  Cand<AR> r;
  r.q = shfl_xor_q<AR>(x.q, off);
  r.q2 = x.q2;
  r.a = __shfl_xor_sync(0xffffffffu, x.a, off);
  return r;
}

// One group of G states starting at s0 (every lane of the warp takes part): the Q-values of
// their rows and the argmin.  Returns the state's pick in every lane of its row group.
template <class PT, class AR, int T, class Gather>
__device__ __forceinline__ Pick<AR> ell_state_group(const SweepK& p, const EllLanes& L, int64_t s0,
                                                    const Gather& gather) {
  using Qt = typename AR::Qt;
  using V = typename AR::V;
  const DevMDP& d = p.d;
  constexpr int RPI = 32 / T;
  const PT* val = (const PT*)d.P;
  const int32_t* col = d.col;
  const int64_t s = s0 + L.g;
  const bool st_ok = s < d.S;
  const bool need_q2 = p.margin_out != nullptr;
  Cand<AR> run;
  run.q = AR::inf(); run.q2 = AR::inf(); run.a = 0x7fffffff;
  Qt qref = AR::inf();
  const int aref = (p.pi_ref && st_ok) ? p.pi_ref[s] : -1;
  for (int pass = 0; pass < L.npass; ++pass) {
    const int a_local = pass * RPI + L.rr;
    const bool act = st_ok && a_local < L.R;
    const int a = act ? (p.pi_in ? p.pi_in[s] : a_local) : 0;
    typename AR::Acc acc;
    acc.init();
    typename AR::G gq{};  // windowed sweep: the cost is loaded before the row's sum, so its
                          // latency overlaps the row (the L1-bound global-gather sweeps load it
                          // after the sum, which measured faster there)
    if (act) {
      if constexpr (Gather::kWindow) gq = AR::gload(d, s, a);
      const int64_t base = ((int64_t)s * d.A + a) * d.kp;
      for (int q0 = L.tl; q0 < L.nvec; q0 += 2 * T) {
        Vec4<PT> pv[2];
        int4 c4[2];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          const int q = q0 + b * T;
          if (q < L.nvec) {
            if constexpr (Gather::kWindow) {  // v from shared memory: L1 holds the rows
              pv[b].load_cached(val + base + 4 * q);
              c4[b] = __ldg(reinterpret_cast<const int4*>(col + base) + q);
            } else {                          // v gathered through L1: stream the rows
              pv[b].load(val + base + 4 * q);
              c4[b] = __ldcs(reinterpret_cast<const int4*>(col + base) + q);
            }
          } else {
            c4[b] = make_int4(0, 0, 0, 0);
#pragma unroll
            for (int e = 0; e < 4; ++e) pv[b].e[e] = PT(0);
          }
        }
        V x[8];
#pragma unroll
        for (int b = 0; b < 2; ++b) {
          x[4 * b + 0] = gather(c4[b].x);
          x[4 * b + 1] = gather(c4[b].y);
          x[4 * b + 2] = gather(c4[b].z);
          x[4 * b + 3] = gather(c4[b].w);
        }
#pragma unroll
        for (int b = 0; b < 2; ++b) {
#pragma unroll
          for (int e = 0; e < 4; ++e) acc.add(pv[b].e[e], x[4 * b + e]);
        }
        acc.tick2();
      }
    }
    const Qt sum = AR::reduce_team(acc.result(), T);
    Qt q = AR::inf();
    if (act) {
      if constexpr (Gather::kWindow) q = AR::qval_g(d, gq, sum);
      else q = AR::qval(d, s, a, sum);
    }
    const bool allowed = act && (p.pi_in ? true : (d.mask ? d.mask[s * d.A + a] != 0 : true));
    // reference-policy row of this pass (when it lies here): its lane holds qref.  Every
    // lane takes part in the shuffle; only lanes whose reference row is in this pass keep it.
    if (p.pi_ref) {
      const int aoff = aref - pass * RPI;
      const bool here = aref >= 0 && aoff >= 0 && aoff < L.Rp && aref < L.R;
      const Qt qs = shfl_q<AR>(q, L.leader + (here ? aoff : 0) * T);
      if (here) qref = qs;
    }
    Cand<AR> c;
    c.q = allowed ? q : AR::inf();
    c.q2 = AR::inf();
    c.a = allowed ? a : 0x7fffffff;
    if (need_q2) {
      for (int off = T; off < L.Rp * T; off <<= 1) c = cand_merge<AR>(c, cand_shfl<AR>(c, off));
      run = cand_merge<AR>(run, c);
    } else if constexpr (Gather::kWindow) {
      // the least Q of the pass by a butterfly on Q alone, then the lowest lane of this state
      // group that holds it exactly, allowed rows first (lanes run in action order): the pick of
      // cand_merge1 (lowest action among the exact minima) with a third of its shuffles, which
      // share the L1 data pipe with the window gathers.  A NaN anywhere in the warp takes the
      // full merge.
      Qt m = c.q;
      for (int off = T; off < L.Rp * T; off <<= 1) {
        const Qt o = shfl_xor_q<AR>(m, off);
        m = AR::lt(o, m) ? o : m;
      }
      const int width = L.Rp * T;
      const unsigned grp = width >= 32 ? 0xffffffffu : (((1u << width) - 1u) << L.leader);
      const bool eq = !AR::lt(c.q, m) && !AR::lt(m, c.q);
      const unsigned hit_allowed = __ballot_sync(0xffffffffu, eq && c.a != 0x7fffffff) & grp;
      const unsigned hit_any = __ballot_sync(0xffffffffu, eq) & grp;
      if (__any_sync(0xffffffffu, hit_any == 0u)) {
        for (int off = T; off < L.Rp * T; off <<= 1) c = cand_merge1<AR>(c, cand_shfl1<AR>(c, off));
      } else {
        const unsigned hit = hit_allowed ? hit_allowed : hit_any;
        c.a = __shfl_sync(0xffffffffu, c.a, __ffs(hit) - 1);
        c.q = m;
      }
      run = cand_merge1<AR>(run, c);
    } else {
      for (int off = T; off < L.Rp * T; off <<= 1) c = cand_merge1<AR>(c, cand_shfl1<AR>(c, off));
      run = cand_merge1<AR>(run, c);
    }
  }
  Pick<AR> pk;
  pk.best = run.q;
  pk.second = run.q2;
  pk.abest = p.pi_in ? (st_ok ? p.pi_in[s] : 0) : (run.a == 0x7fffffff ? -1 : run.a);
  pk.qref = qref;
  return pk;
}

// Per-state outputs leave 32 states at a time: each group's pick is handed to one lane of
// the warp (in order), and when every lane holds one the warp writes them in parallel
// (consecutive lanes, mostly consecutive states) instead of one lane writing per state.
template <class AR>
struct EmitQueue {
  Pick<AR> pk;
  int64_t s;
  int n;
  __device__ __forceinline__ void init() { s = -1; n = 0; }
  __device__ __forceinline__ void flush(const SweepK& p, Norms<AR>& nm) {
    if (s >= 0 && s < p.d.S) emit_state<AR>(p, s, pk, nm);
    s = -1;
    n = 0;
  }
  __device__ __forceinline__ void push(const SweepK& p, const EllLanes& L, int64_t s0,
                                       const Pick<AR>& in, Norms<AR>& nm) {
    const int lane = threadIdx.x & 31;
    for (int g = 0; g < L.G; ++g) {
      const int src = g * L.Rp * L.T;
      Pick<AR> x;
      x.best = shfl_q<AR>(in.best, src);
      x.second = p.margin_out ? shfl_q<AR>(in.second, src) : in.second;
      x.qref = p.pi_ref ? shfl_q<AR>(in.qref, src) : in.qref;
      x.abest = __shfl_sync(0xffffffffu, in.abest, src);
      if (lane == n) {
        pk = x;
        s = s0 + g;
      }
      if (++n == 32) flush(p, nm);
    }
  }
};

// QUEUE: hand the outputs to the emit queue (fewer instructions, ~10 more registers), or
// write each group's outputs from its leader lane right away (the batched kernel, whose
// staged instance record leaves no registers to spare).
template <class PT, class AR, int T, bool QUEUE = true>
__device__ __forceinline__ void sweep_ell_body(const SweepK& p, GridPos gp) {
  const EllLanes L = ell_lanes<T>(p);
  const int lane = threadIdx.x & 31;
  const int64_t gw = ((int64_t)gp.bid * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = (int64_t)gp.nb * (blockDim.x >> 5);
  const GatherGlobal<AR> gather{(const typename AR::V*)p.v, l2_keep_policy()};
  Norms<AR> nm;
  nm.init();
  if constexpr (QUEUE) {
    EmitQueue<AR> eq;
    eq.init();
    for (int64_t s0 = gw * L.G; s0 < p.d.S; s0 += nw * L.G)
      eq.push(p, L, s0, ell_state_group<PT, AR, T>(p, L, s0, gather), nm);
    eq.flush(p, nm);
  } else {
    for (int64_t s0 = gw * L.G; s0 < p.d.S; s0 += nw * L.G) {
      const Pick<AR> pk = ell_state_group<PT, AR, T>(p, L, s0, gather);
      const int64_t s = s0 + L.g;
      if (lane == L.leader && s < p.d.S) emit_state<AR>(p, s, pk, nm);
    }
  }
  finish_norms<AR>(p, nm, gp);
}

template <class PT, class AR, int T, bool QUEUE>
__global__ void __launch_bounds__(256, 3) sweep_ell_warp_kernel(SweepK p) {
  sweep_ell_body<PT, AR, T, QUEUE>(p, this_grid());
}

// ------------------------------------------------------------------ ELL, banded columns
// When every column lies within d.span states of its row's state, a block walks a contiguous
// range of states in steps of WIN_NB, keeping v over [step - span, step + WIN_NB + span) in a
// shared-memory ring that cp.async refills one step ahead.  The gathers then cost a few
// shared-memory wavefronts instead of one L1 tag lookup per distinct line (a warp's 32 random
// columns within +-span touch ~30 lines, which bounds the global-gather kernel).  Each block
// takes an equal share of the 32-state units of S, so every SM (four blocks each) gets the same
// work; rows are bank-ordered at upload (ell_bank_order_kernel) and the argmin shuffles Q alone.
constexpr int WIN_RING = 4096;  // entries of v per block (8 bytes each)
constexpr int WIN_NB = 256;     // states per step; span <= (WIN_RING - 2 WIN_NB) / 2
constexpr int64_t WIN_SPAN_MAX = (WIN_RING - 2 * WIN_NB) / 2;

__device__ __forceinline__ void win_cp8(void* smem, const void* gmem) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_addr(smem)), "l"(gmem) : "memory");
}

template <class PT, class AR, int T>
__global__ void __launch_bounds__(256, 4) sweep_ell_window_kernel(SweepK p) {
  using V = typename AR::V;
  static_assert(sizeof(V) == 8, "window entries are 8 bytes");
  __shared__ V ring[WIN_RING];
  const DevMDP& d = p.d;
  const EllLanes L = ell_lanes<T>(p);
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int64_t span = d.span;
  // this block's states: an equal share of the 32-state units (so every SM, holding the same
  // number of blocks, gets the same work), walked in steps of WIN_NB
  const int64_t nu = (d.S + 31) >> 5;
  const int64_t sb = 32 * (nu * blockIdx.x / gridDim.x);
  const int64_t se = min(d.S, 32 * (nu * (blockIdx.x + 1) / gridDim.x));
  const V* v = (const V*)p.v;
  auto fill = [&](int64_t x0, int64_t x1) {  // v[x], x in [x0, x1) and in [0, S), one group
    const int64_t a0 = max(x0, (int64_t)0), a1 = min(x1, d.S);
    for (int64_t x = a0 + threadIdx.x; x < a1; x += blockDim.x) win_cp8(ring + (x & (WIN_RING - 1)), v + x);
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  const GatherRing<AR> gather{ring, WIN_RING - 1};
  Norms<AR> nm;
  nm.init();
  if (sb < se) {
    fill(sb - span, min(sb + WIN_NB, se) + span);
    asm volatile("cp.async.wait_group 0;" ::: "memory");
    __syncthreads();
    for (int64_t s_lo = sb; s_lo < se; s_lo += WIN_NB) {
      const int64_t s_hi = min(s_lo + WIN_NB, se);
      // the next step's new entries go where entries below s_lo - span were (the ring holds
      // 2 WIN_NB + 2 span entries, so they never overwrite this step's window)
      if (s_hi < se) fill(s_hi + span, min(s_hi + WIN_NB, se) + span);
      // each state's outputs leave from its leader lane (the emit queue's shuffles cost more
      // here than its coalesced stores save: 0.954 against 0.919 ms at S = 10^6)
      for (int64_t s0 = s_lo + warp * L.G; s0 < s_hi; s0 += nwarp * L.G) {
        const Pick<AR> pk = ell_state_group<PT, AR, T>(p, L, s0, gather);
        const int64_t s = s0 + L.g;
        if (lane == L.leader && s < d.S) emit_state<AR>(p, s, pk, nm);
      }
      asm volatile("cp.async.wait_group 0;" ::: "memory");
      __syncthreads();
    }
  }
  finish_norms<AR>(p, nm, this_grid());
}

// ------------------------------------------------------------------ ELL bank order (upload)
// The windowed sweep gathers v from a shared-memory ring of 8-byte entries.  Entry c sits in
// bank pair c mod 16 (up to a constant offset), and a 64-bit shared-memory load is served half
// a warp at a time in as many wavefronts as the most distinct entries that one bank pair holds,
// so 16 random columns take about 3 wavefronts.  The order of the nonzeros within a row is free
// (it changes only the order of the row's sum, and every kernel reads the same stored order),
// so after validation, banded data is reordered for the sweep's lane layout (ell_lanes with the
// default lane count): the rows whose lanes form one half-warp are visited in lane order, and
// each nonzero of a row, in stored order, moves to a free slot of its row whose gather
// instruction has so far the fewest entries in the nonzero's bank pair (ties: the lowest
// instruction, then the lowest lane).  On banded S = 10^6 data (16 actions, 32 entries per
// row) this greedy placement takes the wavefronts of a gather instruction from 6.13 to 3.99
// (ncu), as good as a full assignment per row by the Hungarian method in a CPU emulation, and
// costs 5.9 ms once per upload of the 4.2 GB.  Layouts whose rows span more than 16 gather
// instructions (more than 16 entries at one lane per row, more than 32 at two) keep their order.
//
// One thread per half-warp group.  Per bank pair r it keeps a word of sixteen 4-bit counters,
// one per gather instruction (saturating at 14); the instructions without a free slot read as
// 15, and the first instruction holding the least count is found with the zero-nibble test
// ((y - 0x11..1) & ~y & 0x88..8 flags the lowest nibble of y that is zero exactly).
constexpr int BO_KPMAX = 32;
constexpr int BO_JMAX = 16;
constexpr int BO_THREADS = 64;
constexpr uint64_t BO_ONES = 0x1111111111111111ull;

template <class PT, int T>
__global__ void __launch_bounds__(BO_THREADS) ell_bank_order_kernel(DevMDP d, PT* val, int32_t* col,
                                                                    const int* flags, int64_t span_max) {
  __shared__ uint64_t cnt[16][BO_THREADS];   // [bank pair][thread]: counters per instruction
  __shared__ int32_t sc[BO_KPMAX][BO_THREADS];
  __shared__ PT sv[BO_KPMAX][BO_THREADS];
  if (flags[0] | flags[1] | flags[2] | flags[3] | flags[4]) return;  // invalid data: left as is
  if ((int64_t)flags[6] > span_max) return;  // not banded: the global-gather sweeps take it
  constexpr int RPI = 32 / T;
  int Rp = 1;
  while (Rp < d.A && Rp < RPI) Rp <<= 1;
  const int G = RPI / Rp;
  const int npass = (d.A + RPI - 1) / RPI;
  const int kp = d.kp, nvec = kp >> 2;
  // free slots per instruction j = 4 m + e of a fresh row: the lanes tl < T with tl + T m < nvec
  uint64_t F0 = 0;
  for (int j = 0; j < BO_JMAX; ++j) {
    const int m = j >> 2;
    int n = 0;
    for (int tl = 0; tl < T; ++tl) n += (tl + T * m < nvec) ? 1 : 0;
    F0 |= (uint64_t)n << (4 * j);
  }
  const int tid = threadIdx.x;
  const int64_t nblk = (d.S + G - 1) / G;
  const int64_t ngroups = nblk * npass * 2;
  for (int64_t gi = (int64_t)blockIdx.x * blockDim.x + tid; gi < ngroups;
       gi += (int64_t)gridDim.x * blockDim.x) {
    const int hw = (int)(gi & 1);
    const int pass = (int)((gi >> 1) % npass);
    const int64_t blk = (gi >> 1) / npass;
#pragma unroll
    for (int r = 0; r < 16; ++r) cnt[r][tid] = 0;
    for (int rs = hw * 16 / T; rs < (hw + 1) * 16 / T; ++rs) {  // row slots of this half-warp
      const int g = rs / Rp, rr = rs % Rp;
      const int64_t s = blk * G + g;
      const int a = pass * RPI + rr;
      if (s >= d.S || a >= d.A) continue;
      PT* rv = val + (s * d.A + a) * kp;
      int32_t* rc = col + (s * d.A + a) * kp;
      int32_t c[BO_KPMAX];
      PT v[BO_KPMAX];
#pragma unroll
      for (int q = 0; q < BO_KPMAX / 4; ++q) {
        if (q < nvec) {
          const int4 c4 = reinterpret_cast<const int4*>(rc)[q];
          c[4 * q] = c4.x; c[4 * q + 1] = c4.y; c[4 * q + 2] = c4.z; c[4 * q + 3] = c4.w;
          Vec4<PT> v4;
          v4.load_cached(rv + 4 * q);
#pragma unroll
          for (int e = 0; e < 4; ++e) v[4 * q + e] = v4.e[e];
        } else {
#pragma unroll
          for (int e = 0; e < 4; ++e) { c[4 * q + e] = 0; v[4 * q + e] = PT(0); }
        }
      }
      uint64_t F = F0;                       // free slots left per instruction
      uint32_t freem = kp >= 32 ? 0xffffffffu : ((1u << kp) - 1u);
#pragma unroll
      for (int i = 0; i < BO_KPMAX; ++i) {
        if (i < kp) {
          const int r = c[i] & 15;
          const uint64_t x = cnt[r][tid];
          uint64_t nz = F | (F >> 1) | (F >> 2) | (F >> 3);
          nz &= BO_ONES;                       // 1 in the nibbles with a free slot
          const uint64_t fm = nz * 15ull;      // 0xF there
          const uint64_t xs = (x & fm) | ~fm;  // counters, 15 where no slot is free
          int js = 0;
          for (int t = 0; t < 15; ++t) {
            const uint64_t y = xs ^ (BO_ONES * (uint64_t)t);
            const uint64_t z = (y - BO_ONES) & ~y & (BO_ONES * 8ull);
            if (z) {
              js = __ffsll((long long)z) >> 2;  // bit 4j+3 set -> ffs = 4j+4
              js -= 1;
              break;
            }
          }
          const int m = js >> 2, e = js & 3;
          int idx = 4 * (T * m) + e;           // lane tl = 0 of instruction js
#pragma unroll
          for (int tl = 0; tl < T; ++tl) {
            const int id2 = 4 * (tl + T * m) + e;
            if (id2 < kp && ((freem >> id2) & 1u)) { idx = id2; break; }
          }
          freem &= ~(1u << idx);
          sc[idx][tid] = c[i];
          sv[idx][tid] = v[i];
          if (((x >> (4 * js)) & 15ull) < 14ull) cnt[r][tid] = x + (1ull << (4 * js));
          F -= 1ull << (4 * js);
        }
      }
#pragma unroll
      for (int q = 0; q < BO_KPMAX / 4; ++q) {
        if (q < nvec) {
          reinterpret_cast<int4*>(rc)[q] =
              make_int4(sc[4 * q][tid], sc[4 * q + 1][tid], sc[4 * q + 2][tid], sc[4 * q + 3][tid]);
#pragma unroll
          for (int e = 0; e < 4; ++e) rv[4 * q + e] = sv[4 * q + e][tid];
        }
      }
    }
  }
}

// Batched sweep: the virtual blocks of every instance whose sweep is due.  The instance
// record is staged in shared memory; thread 0 assembles the launch parameters.  Phase SWEEP0
// writes pi_k; phase SWEEPV writes the candidate pi_{k+1} into the other policy buffer and
// the exact residual of pi_k (the reference policy) into rref.
__global__ void __launch_bounds__(256, 3) batch_sweep_kernel(BatchDev B) {
  __shared__ SweepK sp;
  __shared__ BatchInst si;
  batch_for_each(B.sw, [&](int j, GridPos gp) {
    batch_stage_inst(B.insts + j, &si);
    if (threadIdx.x == 0) {
      const BatchInst& I = si;
      const bool verify = I.phase == BP_SWEEPV;
      SweepK p;
      p.d = I.d;
      p.v = I.v;
      p.pi_in = nullptr;
      p.pi_out = I.pib[verify ? 1 - I.cur : I.cur];
      p.tv_out = I.tv;
      p.tv64_out = nullptr;
      p.phi_out = I.phi;
      p.margin_out = nullptr;
      p.pi_ref = verify ? I.pib[I.cur] : nullptr;
      p.rref_out = verify ? (void*)I.rref : nullptr;
      p.out = I.sout;
      p.ref_out = verify ? I.sout + 2 : nullptr;
      p.partials = I.partials;
      p.counter = I.counter;
      sp = p;
    }
    __syncthreads();
    switch (si.cls_sw) {
      case 0: sweep_ell_body<float, ArDF, 1, false>(sp, gp); break;
      case 1: sweep_ell_body<float, ArDF, 2, false>(sp, gp); break;
      case 2: sweep_ell_body<float, ArDF, 4, false>(sp, gp); break;
      default: sweep_ell_body<float, ArDF, 8, false>(sp, gp); break;
    }
  });
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

template <class PT, class AR>
int launch_typed(const SweepLaunch& L, cudaStream_t st) {
  SweepK p{L.d, L.v, L.pi_in, L.pi_out, L.tv_out, L.tv64_out, L.phi_out, L.margin_out,
           L.pi_ref, L.rref_out, L.out, L.ref_out, L.partials, L.counter};
  const DevMDP& d = L.d;
  if (d.kind == KIND_DENSE) {
    if constexpr (std::is_same<AR, ArDF>::value) {
      const int ns = (L.pi_in || L.no_tma || d.A > TS_RMAX || !L.err) ? 0 : tma_sweep_stages(d.ld);
      if (ns > 0) {
        const size_t smem = tma_sweep_layout(d.ld, ns).total;
        if (smem > g_tma_sweep_smem_set) {
          const void* ks[8] = {(const void*)sweep_dense_tma_kernel<1>, (const void*)sweep_dense_tma_kernel<2>,
                               (const void*)sweep_dense_tma_kernel<3>, (const void*)sweep_dense_tma_kernel<4>,
                               (const void*)sweep_dense_tma_kernel<5>, (const void*)sweep_dense_tma_kernel<6>,
                               (const void*)sweep_dense_tma_kernel<7>, (const void*)sweep_dense_tma_kernel<8>};
          for (const void* kf : ks)
            if (cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
              return MDP_EDEVICE;
          g_tma_sweep_smem_set = smem;
        }
        const int grid = L.grid > 0 ? L.grid : (int)std::min<int64_t>(num_sms(), d.S);
        switch (d.A) {
          case 1: sweep_dense_tma_kernel<1><<<grid, TC_THREADS, smem, st>>>(p, ns, L.err); break;
          case 2: sweep_dense_tma_kernel<2><<<grid, TC_THREADS, smem, st>>>(p, ns, L.err); break;
          case 3: sweep_dense_tma_kernel<3><<<grid, TC_THREADS, smem, st>>>(p, ns, L.err); break;
          case 4: sweep_dense_tma_kernel<4><<<grid, TC_THREADS, smem, st>>>(p, ns, L.err); break;
          case 5: sweep_dense_tma_kernel<5><<<grid, TC_THREADS, smem, st>>>(p, ns, L.err); break;
          case 6: sweep_dense_tma_kernel<6><<<grid, TC_THREADS, smem, st>>>(p, ns, L.err); break;
          case 7: sweep_dense_tma_kernel<7><<<grid, TC_THREADS, smem, st>>>(p, ns, L.err); break;
          default: sweep_dense_tma_kernel<8><<<grid, TC_THREADS, smem, st>>>(p, ns, L.err); break;
        }
        return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
      }
    }
    auto k = sweep_dense_kernel<PT, AR, 8>;
    int grid = L.grid > 0 ? L.grid : grid_for(k, 256, 0, (d.S + 7) / 8);
    k<<<grid, 256, 0, st>>>(p);
  } else {
    const int T = L.lanes > 0 ? L.lanes : ell_sweep_lanes_default(d);
    if (d.span >= 0 && d.span <= WIN_SPAN_MAX && !L.no_window && d.S >= 4 * WIN_NB) {
      // banded columns: shared-memory window of v (each block a contiguous range of states,
      // at least one step of WIN_NB)
      int64_t blocks = L.grid > 0 ? L.grid : (int64_t)num_sms() * 4;
      blocks = std::max<int64_t>(1, std::min<int64_t>(blocks, d.S / WIN_NB));
      const int grid = (int)std::min<int64_t>(blocks, MAX_RED_BLOCKS);
      switch (T) {
        case 1: sweep_ell_window_kernel<PT, AR, 1><<<grid, 256, 0, st>>>(p); break;
        case 2: sweep_ell_window_kernel<PT, AR, 2><<<grid, 256, 0, st>>>(p); break;
        case 4: sweep_ell_window_kernel<PT, AR, 4><<<grid, 256, 0, st>>>(p); break;
        case 8: sweep_ell_window_kernel<PT, AR, 8><<<grid, 256, 0, st>>>(p); break;
        default: return MDP_EINVAL;
      }
      return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
    }
    const int64_t units = (d.S + 7) / 8;
    // a geometry fixed by the caller reproduces the batched kernel's grouping of the norm
    // partial sums as well (outputs from the group leaders, no emit queue)
    if (L.grid > 0) {
      switch (T) {
        case 1: sweep_ell_warp_kernel<PT, AR, 1, false><<<L.grid, 256, 0, st>>>(p); break;
        case 2: sweep_ell_warp_kernel<PT, AR, 2, false><<<L.grid, 256, 0, st>>>(p); break;
        case 4: sweep_ell_warp_kernel<PT, AR, 4, false><<<L.grid, 256, 0, st>>>(p); break;
        case 8: sweep_ell_warp_kernel<PT, AR, 8, false><<<L.grid, 256, 0, st>>>(p); break;
        default: return MDP_EINVAL;
      }
      return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
    }
    switch (T) {
      case 1: { auto k = sweep_ell_warp_kernel<PT, AR, 1, true>;
        k<<<grid_for(k, 256, 0, units), 256, 0, st>>>(p); break; }
      case 2: { auto k = sweep_ell_warp_kernel<PT, AR, 2, true>;
        k<<<grid_for(k, 256, 0, units), 256, 0, st>>>(p); break; }
      case 4: { auto k = sweep_ell_warp_kernel<PT, AR, 4, true>;
        k<<<grid_for(k, 256, 0, units), 256, 0, st>>>(p); break; }
      case 8: { auto k = sweep_ell_warp_kernel<PT, AR, 8, true>;
        k<<<grid_for(k, 256, 0, units), 256, 0, st>>>(p); break; }
      default: return MDP_EINVAL;
    }
  }
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}

}  // namespace

int ell_sweep_lanes_default(const DevMDP& d) { return (d.kp / 4) >= 8 ? 2 : 1; }

int batch_sweep_grid() {
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_sweep_kernel, 256, 0) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return num_sms() * std::max(per_sm, 1);
}

int launch_ell_bank_order(const DevMDP& d, void* val, int32_t* col, const int* flags,
                          cudaStream_t st) {
  if (d.kind != KIND_ELL || d.S < 4 * WIN_NB || d.kp > BO_KPMAX) return MDP_OK;
  const int T = ell_sweep_lanes_default(d);
  if (T > 2 || 4 * ((d.kp / 4 + T - 1) / T) > BO_JMAX) return MDP_OK;
  const int RPI = 32 / T;
  int Rp = 1;
  while (Rp < d.A && Rp < RPI) Rp <<= 1;
  const int64_t groups = (d.S + RPI / Rp - 1) / (RPI / Rp) * ((d.A + RPI - 1) / RPI) * 2;
  const int grid = (int)std::max<int64_t>(
      1, std::min<int64_t>((groups + BO_THREADS - 1) / BO_THREADS, (int64_t)num_sms() * 32));
  auto go = [&](auto tag) {
    using PT = decltype(tag);
    if (T == 1) ell_bank_order_kernel<PT, 1><<<grid, BO_THREADS, 0, st>>>(d, (PT*)val, col, flags, WIN_SPAN_MAX);
    else ell_bank_order_kernel<PT, 2><<<grid, BO_THREADS, 0, st>>>(d, (PT*)val, col, flags, WIN_SPAN_MAX);
  };
  if (d.pdt == MDP_F32) go(float{});
  else go(double{});
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}

int launch_batch_sweep(const BatchDev& B, int grid, cudaStream_t st) {
  batch_sweep_kernel<<<grid, 256, 0, st>>>(B);
  return cudaGetLastError() == cudaSuccess ? MDP_OK : MDP_EDEVICE;
}

int launch_sweep(const SweepLaunch& L, cudaStream_t st) {
  if (L.arith == 1) {
    if (L.d.pdt != MDP_F32) return MDP_EINVAL;
    return launch_typed<float, ArDF>(L, st);
  }
  if (L.d.pdt == MDP_F32) return launch_typed<float, ArF64>(L, st);
  return launch_typed<double, ArF64>(L, st);
}

}  // namespace mdp
