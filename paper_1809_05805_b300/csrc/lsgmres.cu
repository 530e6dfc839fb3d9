// B300-native restarted GMRES(m) with plain MGS and one-reduce (lagged
// normalization, compact-WY) MGS orthogonalization, FP64.
//
// Method: Swirydowicz, Langou, Ananthan, Yang, Thomas, "Low synchronization
// GMRES algorithms" (arXiv:1809.05805): Algorithm 6 (MGS-GMRES), Algorithm 4
// (Level-2 MGS with R normalization lag), Algorithm 7 (one-synchronization
// MGS-GMRES), the compact-WY T recurrence of Section II, and the fused mass
// inner product / MAXPY of Section IV.
//
// Design for sm_103a (B300):
//  * FP64 issue rate, not HBM, bounds the FP64 Arnoldi step on this part
//    (about 2 DFMA per clock per SM against ~6 TB/s of HBM), so the kernels
//    spend DFMAs only on the method's own products, keep every scale factor
//    out of the inner loops, and reduce across threads once per kernel.
//  * The basis is stored unnormalized: column k holds u_k and scale[k] = 1/||u_k||,
//    so v_k = scale[k] * u_k is never written. Scales are folded into the
//    coefficients of the dot products and of the MAXPY.
//  * One grid-wide reduction per kernel: per-CTA partial sums go to global
//    memory, an atomic ticket elects the last CTA (of each group of 16 CTAs,
//    then of the groups, when the sum is long), which sums the partials in
//    CTA order (deterministic) and runs the small dense epilogue (lagged norm,
//    Givens rotation, T row, T s, MAXPY coefficients) in shared memory.
//  * The step kernel's CSR reaches the SpMV through shared memory: the
//    bulk-copy engine brings each tile's rowptr slice, indices and values in
//    while the previous tile is computed (mbarrier completion, bounded waits);
//    cycles with a BF16 basis stage the tile's basis columns the same way. The instantiations
//    of the step kernel live in step.cuh and the step_*.cu units.
//  * Kernels read the step index and the stop flag from device state, so a
//    cycle is a fixed launch sequence; once the epilogue marks the cycle done,
//    the remaining kernels of the cycle return immediately.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <type_traits>
#include <utility>
#include <vector>

#include "lsgmres.h"
#include "common.cuh"
#include "step.cuh"

namespace {

// --------------------------------------------------------------------------
// Second projection of Algorithm 5 (cgs2_lvl2) in Arnoldi form
// --------------------------------------------------------------------------
// After step j and its MAXPY, column j+1 holds z = A v_j - V_{j+1} r. One more
// grid reduction gives a_k = u_k^T z (k <= j) with the same fused tile block
// dot (no SpMV); the last CTA forms s2_k = v_k^T z = scale_k a_k, adds s2 to
// H(0:j, j) and writes the coefficients of z -= V_{j+1} s2, which the in-place
// MAXPY (MAXPY_REORTH) applies.
template <int MAXC>
__global__ void __launch_bounds__(kThreads, 2)
k_reorth(const double* __restrict__ V, int64_t ldv, int64_t n, Small s) {
  __shared__ double su[2 * kThreads];
  __shared__ double sw[2 * kThreads];
  __shared__ double red[2 * (kMaxM + 1) + 2];
  __shared__ int s_jj, s_skip;
  DevState* st = s.st;
  if (threadIdx.x == 0) {
    s_skip = __ldcg(&st->done);
    s_jj = __ldcg(&st->step);  // j + 1: z is column j + 1, projected on columns 0..j
  }
  __syncthreads();
  if (s_skip) return;
  const int jj = s_jj;
  const double* z = V + (size_t)jj * ldv;
  const int J8 = jj / kWarps, r8 = jj % kWarps;
  double acc_a[MAXC], acc_c[MAXC], rem_a[kWarps - 1], rem_c[kWarps - 1];
#pragma unroll
  for (int c = 0; c < MAXC; ++c) acc_a[c] = acc_c[c] = 0.0;
#pragma unroll
  for (int c = 0; c < kWarps - 1; ++c) rem_a[c] = rem_c[c] = 0.0;
  double sig = 0.0, dd = 0.0;
  const int64_t ntiles = (n + kThreads - 1) / kThreads;
  if (ntiles >= 4 * (int64_t)gridDim.x) {
    const int64_t npairs = (ntiles + 1) / 2;
    for (int64_t pp = blockIdx.x; pp < npairs; pp += gridDim.x)
      tile_pair_block_dot<MAXC, double, double>(pp, n, nullptr, nullptr, nullptr, V, ldv, z, z, nullptr, false, false, J8,
                                        r8, su, sw, acc_a, acc_c, rem_a, rem_c, sig, dd);
  } else {
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
      tile_block_dot<MAXC, double, double>(t, n, nullptr, nullptr, nullptr, V, ldv, z, z, nullptr, false, false, J8, r8, su,
                                   sw, acc_a, acc_c, rem_a, rem_c, sig, dd);
  }
  cta_partials<MAXC, double>(acc_a, acc_c, rem_a, rem_c, sig, dd, jj, J8, r8, red);
  if (!grid_reduce_last(s, red, 2 * jj + 2)) return;
  const int ld = s.ldh;
  for (int k = threadIdx.x; k < jj; k += blockDim.x) {
    const double sk = __ldcg(&s.scale[k]);
    const double s2 = red[k] * sk;
    s.H[(size_t)(jj - 1) * ld + k] += s2;
    s.coef[1 + k] = -s2 * sk;
  }
  if (threadIdx.x == 0) {
    s.coef[0] = 1.0;
    st->grid_syncs += 1;
  }
}

// --------------------------------------------------------------------------
// MAXPY: out = alpha * y_in + sum_{k<K} c_k V[:, k]
// --------------------------------------------------------------------------
enum { MAXPY_ARNOLDI = 0, MAXPY_XUPDATE = 1, MAXPY_STANDALONE = 2, MAXPY_REORTH = 3 };

template <typename T>
struct Vec16;  // a 16-byte vector of T
template <>
struct Vec16<double> {
  using type = double2;
};
template <>
struct Vec16<float> {
  using type = float4;
};

// VT: basis type, YT: type of y_in / y_out, CT: arithmetic type. Arnoldi mode
// needs VT == YT (the output is a basis column); the FP32 solution update of
// GMRES-IR uses VT = float, YT = CT = double. MAXPY_REORTH (the second
// projection of Algorithm 5) updates the new basis column in place:
// u_{j+1} += sum_k c_k u_k (y_in and y_out are that column; no Givens CTA).
template <typename VT, typename YT, typename CT>
__global__ void __launch_bounds__(kThreads, 4)
k_maxpy(const VT* __restrict__ V, int64_t ldv, const YT* y_in, YT* y_out, int64_t n, Small s, int mode,
        int K_arg) {
  __shared__ double sc[kMaxM + 3];
  __shared__ CT scc[kMaxM + 3];
  __shared__ int sK, s_skip, s_colk;
  __shared__ YT* s_out;
  DevState* st = s.st;
  if (threadIdx.x == 0) {
    s_skip = 0;
    s_out = y_out;
    s_colk = -1;
    if (mode == MAXPY_ARNOLDI || mode == MAXPY_REORTH) {
      s_skip = __ldcg(&st->done);
      sK = __ldcg(&st->maxpy_k);
      if constexpr (std::is_same<VT, YT>::value) {
        s_colk = __ldcg(&st->step);
        s_out = const_cast<VT*>(V) + (size_t)s_colk * ldv;
      }
    } else if (mode == MAXPY_XUPDATE) {
      sK = __ldcg(&st->k);
    } else {
      sK = K_arg;
    }
  }
  __syncthreads();
  if (s_skip) return;
  const int K = sK;
  const double* cf = (mode == MAXPY_XUPDATE) ? s.coefx : s.coef;
  for (int i = threadIdx.x; i <= K; i += blockDim.x) {
    sc[i] = __ldcg(cf + i);
    scc[i] = (CT)sc[i];
  }
  __syncthreads();
  if (mode == MAXPY_ARNOLDI && blockIdx.x == 0) {
    // The first CTA of an Arnoldi MAXPY finishes column j-1 of H (Givens,
    // residual estimate, stop decision) while the other CTAs stream (first,
    // so that it starts with them rather than after the first wave).
    const int j = __ldcg(&st->step) - 1;
    if (j >= 1) {
      const double h = __ldcg(&s.H[(size_t)(j - 1) * s.ldh + j]);
      const int stop = finish_completed(s, j - 1, h, false);
      if (threadIdx.x == 0) {
        st->grid_syncs += 1;
        if (stop) st->done = 1;
      }
    }
    return;
  }
  const int ndata = gridDim.x - (mode == MAXPY_ARNOLDI ? 1 : 0);  // CTAs that stream
  const int bdata = (int)blockIdx.x - (mode == MAXPY_ARNOLDI ? 1 : 0);  // this CTA among them
  YT* out = s_out;
  // FP64 basis column written: its exponent bound for the fixed-point block dot
  constexpr bool kNote = std::is_same<VT, double>::value && std::is_same<YT, double>::value;
  uint32_t emax = 0;
  if (mode == MAXPY_REORTH) y_in = out;  // in place: each element is read, then written, by one thread
  const CT alpha = scc[0];
  const int64_t stride = (int64_t)ndata * blockDim.x;
  const int64_t gid = (int64_t)bdata * blockDim.x + threadIdx.x;
  int64_t done_rows = 0;
  if constexpr (std::is_same<VT, YT>::value) {
    constexpr int E = 16 / (int)sizeof(VT);
    using V16 = typename Vec16<VT>::type;
    union U {
      V16 v;
      VT e[E];
    };
    const bool vec = ((reinterpret_cast<uintptr_t>(y_in) | reinterpret_cast<uintptr_t>(out) |
                       reinterpret_cast<uintptr_t>(V)) & 15) == 0 && (ldv % E) == 0;
    if (vec) {
      const int64_t nE = n / E;
      for (int64_t i = gid; i < nE; i += stride) {
        U y;
        y.v = reinterpret_cast<const V16*>(y_in)[i];
        CT a[E];
#pragma unroll
        for (int e = 0; e < E; ++e) a[e] = alpha * (CT)y.e[e];
        int k = 0;
        for (; k + 4 <= K; k += 4) {  // four independent loads in flight per thread
          U v[4];
#pragma unroll
          for (int u2 = 0; u2 < 4; ++u2) v[u2].v = __ldg(reinterpret_cast<const V16*>(V + (size_t)(k + u2) * ldv) + i);
#pragma unroll
          for (int u2 = 0; u2 < 4; ++u2)
#pragma unroll
            for (int e = 0; e < E; ++e) a[e] = fma(scc[1 + k + u2], (CT)v[u2].e[e], a[e]);
        }
        for (; k < K; ++k) {
          U v;
          v.v = __ldg(reinterpret_cast<const V16*>(V + (size_t)k * ldv) + i);
#pragma unroll
          for (int e = 0; e < E; ++e) a[e] = fma(scc[1 + k], (CT)v.e[e], a[e]);
        }
        U o;
#pragma unroll
        for (int e = 0; e < E; ++e) {
          o.e[e] = (VT)a[e];
          if constexpr (kNote) emax = max(emax, fx_hi_field(o.e[e]));
        }
        reinterpret_cast<V16*>(out)[i] = o.v;
      }
      done_rows = nE * E;
      for (int64_t i = done_rows + gid; i < n; i += stride) {  // ragged tail
        CT a0 = alpha * (CT)y_in[i];
        for (int k = 0; k < K; ++k) a0 = fma(scc[1 + k], (CT)V[(size_t)k * ldv + i], a0);
        out[i] = (YT)a0;
        if constexpr (kNote) emax = max(emax, fx_hi_field(a0));
      }
      if constexpr (kNote)
        if (s_colk >= 0) fx_note_max(s.ecol, s_colk, emax);
      return;
    }
  }
  for (int64_t i = done_rows + gid; i < n; i += stride) {
    CT a0 = alpha * (CT)y_in[i];
    for (int k = 0; k < K; ++k) a0 = fma(scc[1 + k], (CT)V[(size_t)k * ldv + i], a0);
    out[i] = (YT)a0;
    if constexpr (kNote) emax = max(emax, fx_hi_field((double)a0));
  }
  if constexpr (kNote)
    if (s_colk >= 0) fx_note_max(s.ecol, s_colk, emax);
}

// Arnoldi MAXPY of FP64 cycles with the column products on the integer
// pipes: u_{j+1} = alpha w + sum_{k<K} c_k u_k (Section IV's MAXPY; the
// coefficients fold the lagged normalization and T s of Algorithm 4). The
// sum over the basis columns is formed exactly in integers and rounded to
// FP64 once per row, then alpha w is added with one FMA:
//  * each basis value is the integer X within one unit of u 2^(58 - E_k)
//    from its column's stored bound (Small::ecol), in 29-bit limbs, as the
//    step kernel stored them (Small::VL, fx_split);
//  * each coefficient becomes an integer C_k = round(c_k 2^e_k) scaled so
//    that every product C_k X_k shares one scale and |C_k| <= 2^57 (2^56 from
//    64 columns, 2^55 from 128), split in C_k = Ch 2^29 + Cl;
//  * per row, hh = sum Ch Xh and mid = sum (Ch Xl + Cl Xh) in 64-bit integers
//    (mid folded into hh every 16 columns), Cl Xl (below 2^-56 of the
//    largest product) dropped.
// The first CTA finishes column j-1 of H meanwhile, as in k_maxpy.
// mode MAXPY_XUPDATE: the cycle's solution update x += sum_{k<K} c_k u_k the
// same way (K = the cycle's steps, c from Small::coefx, w = xout = x, in
// place: each element is read, then written, by one thread; no Givens CTA).
__global__ void __launch_bounds__(kThreads, 4)
k_maxpy_fx(const double* __restrict__ V, int64_t ldv, const double* w, int64_t n, Small s, int mode,
           double* xout) {
  __shared__ int4 sC[kMaxM + 1];  // (Ch, Cl, 5 + column bound field, 0) per column
  __shared__ uint32_t s_p[kWarps];
  __shared__ int sK, s_skip, s_colk, s_bad, s_ps;
  __shared__ double s_alpha;
  DevState* st = s.st;
  const bool arn = mode == MAXPY_ARNOLDI;
  const double* cf = arn ? s.coef : s.coefx;
  if (threadIdx.x == 0) {
    s_skip = arn ? __ldcg(&st->done) : 0;
    sK = __ldcg(arn ? &st->maxpy_k : &st->k);
    s_colk = arn ? __ldcg(&st->step) : -1;
    s_alpha = __ldcg(cf);
    s_bad = 0;
  }
  __syncthreads();
  if (s_skip) return;
  const int K = sK;
  if (arn && blockIdx.x == 0) {
    // column j-1 of H: Givens, residual estimate, stop decision (the first
    // CTA, so that it starts with the streaming ones)
    const int j = s_colk - 1;
    if (j >= 1) {
      const double h = __ldcg(&s.H[(size_t)(j - 1) * s.ldh + j]);
      const int stop = finish_completed(s, j - 1, h, false);
      if (threadIdx.x == 0) {
        st->grid_syncs += 1;
        if (stop) st->done = 1;
      }
    }
    return;
  }
  // the coefficients' common scale: P = max_k (field(c_k) + field bound of column k)
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double ck = 0.0;
  int fk = (int)kFxMinField, pk = 0;
  if ((int)threadIdx.x < K) {
    ck = __ldcg(cf + 1 + threadIdx.x);
    fk = (int)max(kFxMinField, __ldcg(s.ecol + threadIdx.x) >> 20);
    const int gk = (int)fx_field(ck);
    if (gk == 0x7FF || fk == 0x7FF) s_bad = 1;  // NaN or Inf among the inputs
    pk = (ck != 0.0) ? gk + fk : 0;
  }
  uint32_t pm = __reduce_max_sync(0xffffffffu, (uint32_t)pk);
  if (lane == 0) s_p[wid] = pm;
  __syncthreads();
  if (threadIdx.x == 0) {
    uint32_t q = 0;
    for (int v = 0; v < kWarps; ++v) q = max(q, s_p[v]);
    s_ps = (int)q;
  }
  __syncthreads();
  const int P = s_ps;
  // |C| <= 2^cbits and |Xh| <= 2^29: the high sum gathers K products of at most
  // 2^cbits, below 2^63 for K < 2^(63 - cbits)
  const int cbits = K < 64 ? 57 : (K < 128 ? 56 : 55);
  if ((int)threadIdx.x < K) {
    long long C = 0;
    if (ck != 0.0 && P > 0) {
      // |c_k| 2^e < 2^(cbits + field(c_k) + f_k - P) <= 2^cbits
      const int e = cbits + 1022 - P + fk;
      C = __double2ll_rn(scalbn(ck, e));
    }
    sC[threadIdx.x] = make_int4((int)(C >> 29), (int)(C & 0x1FFFFFFFll), 5 + fk, 0);
  }
  __syncthreads();
  const bool bad = s_bad != 0;
  const double alpha = s_alpha;
  double* out = arn ? const_cast<double*>(V) + (size_t)s_colk * ldv : xout;
  const int ndata = gridDim.x - (arn ? 1 : 0);
  const int64_t stride = (int64_t)ndata * blockDim.x;
  const int64_t gid = (int64_t)(blockIdx.x - (arn ? 1 : 0)) * blockDim.x + threadIdx.x;
  const int e2 = P - 2044 - cbits;  // sum = (hh + mid / 2^29) 2^(P - 2044 - cbits)
  uint32_t emax = 0;
  const int64_t nE = n / 2;
  // two rows per thread (16-byte loads); ldv is even and the columns 16-byte aligned
  for (int64_t i = gid; i < nE; i += stride) {
    long long hh0 = 0, md0 = 0, hh1 = 0, md1 = 0;
    int k = 0;
    for (; k < K; k += 8) {
      int4 x[8];  // the stored limbs of rows 2i, 2i + 1 of columns k .. k + 7
#pragma unroll
      for (int u2 = 0; u2 < 8; ++u2)
        x[u2] = (k + u2 < K) ? __ldg(reinterpret_cast<const int4*>(s.VL + (size_t)(k + u2) * s.ldl) + i)
                             : make_int4(0, 0, 0, 0);
#pragma unroll
      for (int u2 = 0; u2 < 8; ++u2) {
        if (k + u2 < K) {
          const int4 c = sC[k + u2];
          const int2 a = make_int2(x[u2].x, x[u2].y), b = make_int2(x[u2].z, x[u2].w);
          hh0 = fx_madw(c.x, a.x, hh0);
          md0 = fx_madw(c.x, a.y, md0);
          md0 = fx_madw(c.y, a.x, md0);
          hh1 = fx_madw(c.x, b.x, hh1);
          md1 = fx_madw(c.x, b.y, md1);
          md1 = fx_madw(c.y, b.x, md1);
        }
      }
      if ((k & 15) == 8) {  // every 16 columns: carry mid's high part into hh
        hh0 += md0 >> 29;
        md0 &= 0x1FFFFFFFll;
        hh1 += md1 >> 29;
        md1 &= 0x1FFFFFFFll;
      }
    }
    const double2 wv = __ldg(reinterpret_cast<const double2*>(w) + i);
    double2 o;
    o.x = fma(alpha, wv.x, fx_to_double(hh0 + (md0 >> 29), e2));
    o.y = fma(alpha, wv.y, fx_to_double(hh1 + (md1 >> 29), e2));
    if (bad) o.x = o.y = __longlong_as_double(0x7ff8000000000000ll);
    reinterpret_cast<double2*>(out)[i] = o;
    emax = max(emax, max(fx_hi_field(o.x), fx_hi_field(o.y)));
  }
  for (int64_t i = 2 * nE + gid; i < n; i += stride) {  // odd last row
    long long hh = 0, md = 0;
    for (int k = 0; k < K; ++k) {
      const int4 c = sC[k];
      const int2 a = __ldg(s.VL + (size_t)k * s.ldl + i);
      hh = fx_madw(c.x, a.x, hh);
      md = fx_madw(c.x, a.y, md);
      md = fx_madw(c.y, a.x, md);
      if ((k & 15) == 15) {
        hh += md >> 29;
        md &= 0x1FFFFFFFll;
      }
    }
    double o = fma(alpha, w[i], fx_to_double(hh + (md >> 29), e2));
    if (bad) o = __longlong_as_double(0x7ff8000000000000ll);
    out[i] = o;
    emax = max(emax, fx_hi_field(o));
  }
  if (s_colk >= 0) fx_note_max(s.ecol, s_colk, emax);
}

// Arnoldi MAXPY of GMRES-IR with BF16 basis storage: u_{j+1} = alpha w +
// sum_k c_k u_k computed in FP32 (w in FP32, the basis widened from BF16, the
// coefficients rounded to FP32) and rounded to BF16 (nearest, ties to even)
// as it is stored; eight BF16 values per 16-byte access. The first CTA
// finishes column j-1 of H as in k_maxpy.
__global__ void __launch_bounds__(kThreads, 4)
k_maxpy_bf16(__nv_bfloat16* __restrict__ V, int64_t ldv, const float* __restrict__ w, int64_t n, Small s) {
  __shared__ float scc[kMaxM + 3];
  __shared__ int sK, s_skip, s_step;
  DevState* st = s.st;
  if (threadIdx.x == 0) {
    s_skip = __ldcg(&st->done);
    sK = __ldcg(&st->maxpy_k);
    s_step = __ldcg(&st->step);
  }
  __syncthreads();
  if (s_skip) return;
  const int K = sK;
  for (int i = threadIdx.x; i <= K; i += blockDim.x) scc[i] = (float)__ldcg(s.coef + i);
  __syncthreads();
  if (blockIdx.x == 0) {  // column j-1 of H, beside the streaming CTAs
    const int j = s_step - 1;
    if (j >= 1) {
      const double h = __ldcg(&s.H[(size_t)(j - 1) * s.ldh + j]);
      const int stop = finish_completed(s, j - 1, h, false);
      if (threadIdx.x == 0) {
        st->grid_syncs += 1;
        if (stop) st->done = 1;
      }
    }
    return;
  }
  __nv_bfloat16* out = V + (size_t)s_step * ldv;
  const int ndata = gridDim.x - 1;
  const int64_t stride = (int64_t)ndata * blockDim.x;
  const int64_t gid = (int64_t)(blockIdx.x - 1) * blockDim.x + threadIdx.x;
  const float alpha = scc[0];
  const int64_t n8 = n / 8;  // columns start on 16-byte boundaries (ldv is a multiple of 32)
  for (int64_t i = gid; i < n8; i += stride) {
    const float4 w0 = reinterpret_cast<const float4*>(w)[2 * i];
    const float4 w1 = reinterpret_cast<const float4*>(w)[2 * i + 1];
    float a[8] = {alpha * w0.x, alpha * w0.y, alpha * w0.z, alpha * w0.w,
                  alpha * w1.x, alpha * w1.y, alpha * w1.z, alpha * w1.w};
    for (int k = 0; k < K; ++k) {
      union {
        uint4 v;
        __nv_bfloat162 h[4];
      } x;
      x.v = __ldg(reinterpret_cast<const uint4*>(V + (size_t)k * ldv) + i);
      const float c = scc[1 + k];
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 f = __bfloat1622float2(x.h[q]);
        a[2 * q] = fmaf(c, f.x, a[2 * q]);
        a[2 * q + 1] = fmaf(c, f.y, a[2 * q + 1]);
      }
    }
    union {
      uint4 v;
      __nv_bfloat162 h[4];
    } o;
#pragma unroll
    for (int q = 0; q < 4; ++q) o.h[q] = __floats2bfloat162_rn(a[2 * q], a[2 * q + 1]);
    reinterpret_cast<uint4*>(out)[i] = o.v;
  }
  for (int64_t i = 8 * n8 + gid; i < n; i += stride) {  // ragged tail
    float a0 = alpha * w[i];
    for (int k = 0; k < K; ++k) a0 = fmaf(scc[1 + k], __bfloat162float(V[(size_t)k * ldv + i]), a0);
    out[i] = __float2bfloat16_rn(a0);
  }
}

// --------------------------------------------------------------------------
// MGS-GMRES kernels (Algorithm 6)
// --------------------------------------------------------------------------
// Step i, first kernel: w = A v_i = scale_i * (A u_i) written into column i+1,
// fused with the first inner product p = u_0^T w; the epilogue sets
// h_0 = scale_0 p = H(0, i).
__global__ void __launch_bounds__(kThreads, 2)
k_mgs_spmv(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
           const double* __restrict__ val, double* __restrict__ V, int64_t ldv, int64_t n, Small s) {
  __shared__ double sbuf[kWarps];
  __shared__ double red[2];
  __shared__ int s_i, s_skip;
  __shared__ double s_si;
  DevState* st = s.st;
  if (threadIdx.x == 0) {
    s_skip = __ldcg(&st->done);
    s_i = __ldcg(&st->step);
    s_si = __ldcg(&s.scale[s_i]);
  }
  __syncthreads();
  if (s_skip) return;
  const int i = s_i;
  const double si = s_si;
  const double* u = V + (size_t)i * ldv;
  double* w = V + (size_t)(i + 1) * ldv;
  const double* u0 = V;
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const double wr = si * csr_row(rowptr, col, val, u, r);
    w[r] = wr;
    acc = fma(wr, u0[r], acc);
  }
  const double tot = block_sum(acc, sbuf);
  if (threadIdx.x == 0) red[0] = tot;
  __syncthreads();
  if (!grid_reduce_last(s, red, 1)) return;
  if (threadIdx.x == 0) {
    st->grid_syncs += 1;
    const double h = s.scale[0] * red[0];
    s.H[(size_t)i * s.ldh + 0] = h;
    st->mgs_coef = h * s.scale[0];
    st->inner = 0;
  }
}

// Step i, inner kernel k: w -= h_k v_k, fused with the next reduction:
// h_{k+1} = v_{k+1}^T w (k < i) or ||w||^2 (k == i). The last inner kernel
// completes column i of H, rotates it, tests convergence and stores
// scale[i+1] = 1 / ||w||, so column i+1 becomes v_{i+1} without a rewrite.
__global__ void __launch_bounds__(kThreads, 2)
k_mgs_axpy_dot(double* __restrict__ V, int64_t ldv, int64_t n, Small s) {
  __shared__ double sbuf[kWarps];
  __shared__ double red[2];
  __shared__ int s_i, s_k, s_skip;
  __shared__ double s_cf;
  DevState* st = s.st;
  if (threadIdx.x == 0) {
    s_skip = __ldcg(&st->done);
    s_i = __ldcg(&st->step);
    s_k = __ldcg(&st->inner);
    s_cf = __ldcg(&st->mgs_coef);
  }
  __syncthreads();
  if (s_skip) return;
  const int i = s_i, k = s_k;
  const double cf = s_cf;
  double* w = V + (size_t)(i + 1) * ldv;
  const double* uk = V + (size_t)k * ldv;
  const bool last = (k == i);
  const double* un = last ? w : V + (size_t)(k + 1) * ldv;
  double acc = 0.0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    const double wr = fma(-cf, uk[r], w[r]);
    w[r] = wr;
    acc = fma(wr, last ? wr : un[r], acc);
  }
  const double tot = block_sum(acc, sbuf);
  if (threadIdx.x == 0) red[0] = tot;
  __syncthreads();
  if (!grid_reduce_last(s, red, 1)) return;
  const int ld = s.ldh;
  if (!last) {
    if (threadIdx.x == 0) {
      st->grid_syncs += 1;
      const double sc = __ldcg(&s.scale[k + 1]);
      const double h = sc * red[0];
      s.H[(size_t)i * ld + k + 1] = h;
      st->mgs_coef = h * sc;
      st->inner = k + 1;
    }
    return;
  }
  __shared__ double s_hn;
  if (threadIdx.x == 0) {
    st->grid_syncs += 1;
    const double hn = sqrt(red[0]);
    s.H[(size_t)i * ld + i + 1] = hn;
    s.scale[i + 1] = 1.0 / hn;
    s_hn = hn;
  }
  __syncthreads();
  const int stop = finish_column(s, i, s_hn, i + 1 == __ldcg(&st->kmax));
  if (threadIdx.x == 0) {
    st->step = i + 1;
    st->inner = 0;
    if (stop) st->done = 1;
  }
}

// --------------------------------------------------------------------------
// One whole restart cycle in one launch (small systems: latency-bound)
// --------------------------------------------------------------------------
// A software grid barrier for a cooperative launch (every CTA resident):
// bar[0] counts arrivals, bar[1] is the generation. Thread 0 of each CTA reads
// the generation, arrives, and the last arrival resets the count and advances
// the generation; the others wait for it to advance. Every wait is bounded
// (about one second of SM clocks, as the staging waits): a CTA that gives up,
// or sees that another gave up, marks the state stalled and returns false, so
// every CTA leaves the kernel within a few seconds and the solve reports
// GMRES_ERR_TIMEOUT. `extra` (testing) raises the arrival count the barrier
// waits for, so that it never completes.
__device__ bool grid_barrier(unsigned int* bar, unsigned int nblocks, unsigned int extra, DevState* st) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vgen = bar + 1;
    const unsigned int g = *vgen;
    __threadfence();
    int ok = 1;
    if (atomicAdd(bar, 1u) == nblocks + extra - 1) {
      bar[0] = 0u;
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      const long long t0 = clock64();
      while (*vgen == g) {
        if (*reinterpret_cast<volatile int*>(&st->stalled)) {
          ok = 0;
          break;
        }
        if (clock64() - t0 > (1ll << 31)) {
          atomicExch(&st->stalled, 1);
          ok = 0;
          break;
        }
        __nanosleep(64);
      }
      __threadfence();
    }
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// The one-launch cycle's wait for a step's epilogue: bar[2] counts the
// epilogues published in this launch; every CTA waits until it reaches
// `epoch` (bounded as grid_barrier's waits). The CTA that ran the epilogue has
// made its writes visible (__threadfence) before raising the count, so after
// the wait its coefficients and state may be read through L2. This replaces a
// grid barrier: every CTA's arrival is already implied by the grid reduction
// that elected the epilogue's CTA.
__device__ bool wait_epilogue(unsigned int* bar, unsigned int epoch, DevState* st) {
  __shared__ int s_ok;
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned int* vf = bar + 2;
    int ok = 1;
    const long long t0 = clock64();
    while (*vf < epoch) {
      if (*reinterpret_cast<volatile int*>(&st->stalled)) {
        ok = 0;
        break;
      }
      if (clock64() - t0 > (1ll << 31)) {
        atomicExch(&st->stalled, 1);
        ok = 0;
        break;
      }
      __nanosleep(32);
    }
    __threadfence();
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Basis reads of the one-launch cycle go through L2 (__ldcg): the columns are
// written during the launch by other CTAs, so neither the read-only path nor
// a possibly stale L1 line may serve them.
struct CoherentCols {
  const double* V;
  int64_t ldv;
  int64_t r0;
  template <typename VT>
  __device__ VT ld(int k, int i) const {
    return __ldcg(V + (size_t)k * ldv + r0 + i);
  }
};

// Row i of A times x (FMA chain in column order, as csr_row), x through L2.
__device__ __forceinline__ double csr_row_cg(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                             const double* __restrict__ val, const double* x, int64_t i) {
  double acc = 0.0;
  for (int p = __ldg(rowptr + i), e = __ldg(rowptr + i + 1); p < e; ++p)
    acc = fma(__ldg(val + p), __ldcg(x + __ldg(col + p)), acc);
  return acc;
}

// Every Arnoldi step of a cycle (Algorithm 7 on Algorithm 4), with the same
// arithmetic and device functions as the per-step launches (the fused SpMV +
// block dot on single tiles, the last-CTA grid reduction and epilogue, the
// Arnoldi MAXPY, the Givens rotations). The grid is Pw work CTAs and one
// Givens CTA (the last). Per step j:
//   phase A: the work CTAs run the fused SpMV + block dot over their tiles
//            and publish their partial sums; the last to arrive sums them and
//            runs the epilogue (lagged norm, T row, r = T s, MAXPY
//            coefficients). Meanwhile the Givens CTA applies the stored
//            rotations to column j-1, whose first j entries the previous
//            step's epilogue wrote (the lagged H(j, j-1) is still to come);
//   wait for the epilogue (wait_epilogue: a count the epilogue's CTA raises;
//            every CTA's arrival is implied by the grid reduction);
//   phase B: the work CTAs run the MAXPY over their rows; the Givens CTA forms
//            rotation j-1 from the new H(j, j-1) and takes the convergence
//            decision (in the L = 2 pipeline: the rotations of Algorithm 8's
//            column pairs, as the per-step launches do);
//   barrier 2 (the next SpMV reads the new column everywhere).
// One grid reduction and one grid barrier per step (two launches per step
// would synchronize twice), and the Givens chain off the critical path.
// Needs a cooperative launch (every CTA resident) and (m+1)^2 + (m+1) doubles
// of dynamic shared memory for the epilogue.
template <int MAXC>
__global__ void __launch_bounds__(kThreads, 2)
k_cycle_persistent(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                   const double* __restrict__ val, double* V, int64_t ldv, double* w, int64_t n, Small s,
                   unsigned int* bar, unsigned int bar_extra) {
  __shared__ double su[kThreads];
  __shared__ double sw[kThreads];
  __shared__ double red[2 * (kMaxM + 1) + 2];
  __shared__ double scf[kMaxM + 3];
  __shared__ PreRot s_pr;
  __shared__ int s_j, s_tail, s_done, s_K, s_out, s_pipe2;
  DevState* st = s.st;
  const unsigned int P = gridDim.x;
  const int Pw = (int)P - 1;  // work CTAs; CTA Pw rotates
  const bool givens = (int)blockIdx.x == Pw;
  const int64_t ntiles = (n + kThreads - 1) / kThreads;
  if (threadIdx.x == 0) s_pipe2 = __ldcg(&st->pipe2);
  unsigned int epoch = 0;  // steps of this launch whose epilogue has been waited for
  for (;;) {
    if (threadIdx.x == 0) {
      s_done = __ldcg(&st->done) | __ldcg(&st->stalled);
      s_j = __ldcg(&st->step);
      s_tail = (s_j == __ldcg(&st->kmax));
    }
    __syncthreads();
    if (s_done) return;
    const int j = s_j;
    const bool tail = s_tail;
    const double* u = V + (size_t)j * ldv;
    // ---- phase A ----
    if (givens) {
      if (j >= 1 && !tail && !s_pipe2) prerotate_column(s, j - 1, &s_pr);
    } else {
      const int J8 = j / kWarps, r8 = j % kWarps;
      double acc_a[MAXC], acc_c[MAXC], rem_a[kWarps - 1], rem_c[kWarps - 1];
#pragma unroll
      for (int c = 0; c < MAXC; ++c) acc_a[c] = acc_c[c] = 0.0;
#pragma unroll
      for (int c = 0; c < kWarps - 1; ++c) rem_a[c] = rem_c[c] = 0.0;
      double sig = 0.0, dd = 0.0;
      for (int64_t t = blockIdx.x; t < ntiles; t += Pw) {
        const int64_t row = t * kThreads + threadIdx.x;
        double ur = 0.0, wr = 0.0;
        if (row < n) {
          ur = __ldcg(u + row);
          if (!tail) {
            wr = csr_row_cg(rowptr, col, val, u, row);
            w[row] = wr;
          }
        }
        tile_dot_rows_cols<MAXC, double, double>(t, n, CoherentCols{V, ldv, t * kThreads}, !tail, J8, r8, ur, wr,
                                                 su, sw, acc_a, acc_c, rem_a, rem_c, sig, dd, NoHook{}, NoHook{},
                                                 NoHook{});
      }
      cta_partials<MAXC, double>(acc_a, acc_c, rem_a, rem_c, sig, dd, j, J8, r8, red);
      if (grid_reduce_last(s, red, 2 * j + 2, Pw)) {
        epilogue_one_reduce(s, red, j, tail);
        __syncthreads();  // every thread's epilogue writes are issued
        if (threadIdx.x == 0) {
          __threadfence();
          atomicAdd(bar + 2, 1u);
        }
      }
    }
    ++epoch;
    if (!wait_epilogue(bar, epoch + (bar_extra >> 1), st)) return;
    if (threadIdx.x == 0) {
      s_done = __ldcg(&st->done);
      s_K = __ldcg(&st->maxpy_k);
      s_out = __ldcg(&st->step);
    }
    __syncthreads();
    if (s_done) return;
    // ---- phase B ----
    if (givens) {
      if (j >= 1) {
        const double h = __ldcg(&s.H[(size_t)(j - 1) * s.ldh + j]);
        const int stop = s_pipe2 ? finish_completed(s, j - 1, h, false)
                                 : finish_prerotated(s, j - 1, h, &s_pr, false);
        if (threadIdx.x == 0) {
          atomicAdd(reinterpret_cast<unsigned long long*>(&st->grid_syncs), 1ull);
          if (stop) st->done = 1;
        }
      }
    } else {
      const int K = s_K;
      for (int i = threadIdx.x; i <= K; i += blockDim.x) scf[i] = __ldcg(s.coef + i);
      __syncthreads();
      double* out = V + (size_t)s_out * ldv;
      for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)Pw * blockDim.x) {
        double a0 = scf[0] * __ldcg(w + i);
        for (int k = 0; k < K; ++k) a0 = fma(scf[1 + k], __ldcg(V + (size_t)k * ldv + i), a0);
        out[i] = a0;
      }
    }
    if (!grid_barrier(bar, P, bar_extra & 1u, st)) return;
  }
}

using CycleKernel = void (*)(const int32_t*, const int32_t*, const double*, double*, int64_t, double*, int64_t,
                             Small, unsigned int*, unsigned int);
CycleKernel cycle_kernel_for(int m) {
  switch (std::max(1, m / kWarps)) {
    case 1: return k_cycle_persistent<1>;
    case 2: return k_cycle_persistent<2>;
    case 3: return k_cycle_persistent<3>;
    case 4: return k_cycle_persistent<4>;
    case 5: return k_cycle_persistent<5>;
    case 6: return k_cycle_persistent<6>;
    case 7: return k_cycle_persistent<7>;
    case 8: return k_cycle_persistent<8>;
    case 9: case 10: case 11: case 12: return k_cycle_persistent<12>;
    default: return k_cycle_persistent<16>;
  }
}

// Exponent bounds of the first j columns of a caller's basis (the standalone
// block dot): ecol[k] = largest (hi word & 0x7FF00000) in column k; ecol
// cleared before. Grid: (x, j).
__global__ void k_col_fields(const double* __restrict__ V, int64_t ldv, int64_t n, unsigned int* ecol) {
  const int k = blockIdx.y;
  uint32_t emax = 0;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    emax = max(emax, fx_hi_field(V[(size_t)k * ldv + i]));
  fx_note_max(ecol, k, emax);
}

// The first j columns of a caller's basis as fixed-point limbs (fx_split
// against the bounds k_col_fields measured) into VL, for the standalone block
// dot of staging mode 6. Grid: (x, j).
__global__ void k_col_limbs(const double* __restrict__ V, int64_t ldv, int64_t n, const unsigned int* ecol,
                            int2* __restrict__ VL, int64_t ldl) {
  const int k = blockIdx.y;
  const int kf = 5 + (int)max(kFxMinField, ecol[k] >> 20);
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
    VL[(size_t)k * ldl + i] = fx_split(V[(size_t)k * ldv + i], kf);
}

// mode RES_BNORM:    ||b|| -> st->bnorm
// mode RES_RESIDUAL: r = b - A x -> column 0, ||r|| -> st->rnorm, and the
//                    cycle state is reset (x == nullptr means x = 0).
// mode RES_START:    column 0 = b (a given start vector), ||b|| -> bnorm and rnorm.
__global__ void __launch_bounds__(kThreads, 2)
k_residual(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
           const double* __restrict__ val, const double* __restrict__ b, const double* __restrict__ x,
           double* __restrict__ V0, int64_t n, Small s, int mode, int kmax) {
  __shared__ double sbuf[kWarps];
  __shared__ double red[2];
  double acc = 0.0;
  uint32_t emax = 0;  // exponent bound of column 0 for the fixed-point block dot
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    double v = b[r];
    if (mode == RES_RESIDUAL && x) v -= csr_row(rowptr, col, val, x, r);
    if (mode != RES_BNORM) {
      V0[r] = v;
      emax = max(emax, fx_hi_field(v));
    }
    acc = fma(v, v, acc);
  }
  if (mode != RES_BNORM) fx_note_max(s.ecol, 0, emax);
  const double tot = block_sum(acc, sbuf);
  if (threadIdx.x == 0) red[0] = tot;
  __syncthreads();
  if (!grid_reduce_last(s, red, 1)) return;
  if (threadIdx.x == 0) residual_finish(s, red[0], mode, kmax);
}

// Start of an FP32 (GMRES-IR) cycle: column 0 of the FP32 (or BF16) basis =
// r / ||r|| rounded to FP32 (then BF16) (normalized in FP64 first, so the FP32
// cycle works on a unit-scale right-hand side); the estimate and the
// correction of this cycle are scaled back by ||r||.
__device__ __forceinline__ void store_narrow(float* p, double x) { *p = (float)x; }
__device__ __forceinline__ void store_narrow(__nv_bfloat16* p, double x) { *p = __float2bfloat16_rn((float)x); }

template <typename OT>
__global__ void k_round_scaled(const double* __restrict__ r, OT* __restrict__ out, int64_t n, Small s) {
  const double rn = __ldcg(&s.st->rnorm);
  const double ir = 1.0 / rn;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) store_narrow(out + i, r[i] * ir);
  if (blockIdx.x == 0 && threadIdx.x == 0) s.st->cycle_scale = rn;
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (float)a[i];
}

__global__ void k_lsq(Small s) { lsq_system(s); }

// V_out[:, k] = scale[k] * V[:, k] for k <= kk (normalized basis export; an
// FP32 or BF16 basis is widened exactly before the scaling).
template <typename SV>
__global__ void k_export_basis(const SV* __restrict__ V, int64_t ldv, double* __restrict__ Vo,
                               int64_t n, int kk, Small s) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k <= kk; ++k) {
    const double sc = s.scale[k];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride)
      if constexpr (std::is_same<SV, double>::value)
        Vo[(size_t)k * n + r] = sc * V[(size_t)k * ldv + r];
      else
        Vo[(size_t)k * n + r] = sc * (double)ld_as<float>(V + (size_t)k * ldv + r);
  }
}

__global__ void k_spmv(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                       const double* __restrict__ val, const double* __restrict__ x, double* __restrict__ y,
                       int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride)
    y[r] = csr_row(rowptr, col, val, x, r);
}


// --------------------------------------------------------------------------
// scratch for lsg_block_dot_noalloc
// --------------------------------------------------------------------------
// The grid reduction of the fused SpMV + block-dot kernel needs scratch: one
// row of partial sums per CTA and the last-CTA ticket. gmres_create allocates
// it per handle; lsg_block_dot_noalloc instead uses this fixed array, which is
// part of the library image and so exists on every device that loads the
// library, from load until process exit. Layout: a DevState (holds the ticket)
// followed by kNoAllocMaxCtas rows of kNoAllocNv doubles.
constexpr int kNoAllocMaxJ = 64;                       // largest j (block-dot columns)
constexpr int kNoAllocMaxCtas = 296;                   // largest grid of the reduction
constexpr int kNoAllocNv = 2 * kNoAllocMaxJ + 2;       // sums per CTA
constexpr size_t kNoAllocStateBytes = 512;             // DevState, padded
constexpr size_t kNoAllocBytes =
    kNoAllocStateBytes +
    sizeof(double) * (size_t)(kNoAllocMaxCtas + (kNoAllocMaxCtas + kGridGroup - 1) / kGridGroup) * kNoAllocNv;
static_assert(sizeof(DevState) <= kNoAllocStateBytes, "DevState outgrew its slot");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

using ReorthKernel = void (*)(const double*, int64_t, int64_t, Small);

ReorthKernel reorth_kernel_for(int m) {
  switch (std::max(1, m / kWarps)) {
    case 1: return k_reorth<1>;
    case 2: return k_reorth<2>;
    case 3: return k_reorth<3>;
    case 4: return k_reorth<4>;
    case 5: return k_reorth<5>;
    case 6: return k_reorth<6>;
    case 7: return k_reorth<7>;
    case 8: return k_reorth<8>;
    case 9: case 10: case 11: case 12: return k_reorth<12>;
    default: return k_reorth<16>;
  }
}

// Step kernels of a restart length m and staging mode (the instantiations
// live in the step_<type>_s<stage>.cu translation units).
StepKernel<double> step64_for(int m, int stage = 0) {
  return reinterpret_cast<StepKernel<double>>(const_cast<void*>(lsg_steps::step_kernel_f64(m, stage)));
}
// The FP64 step kernel of a handle: staging mode 2 runs as mode 6 (the same
// kernel with the fixed-point block dot) unless the handle turned that off.
int fx_stage(int stage, int dot_fx) { return (dot_fx && stage == 2) ? 6 : stage; }

StepKernel<float> step32_for(int m, int stage = 0) {
  return reinterpret_cast<StepKernel<float>>(const_cast<void*>(lsg_steps::step_kernel_f32(m, stage)));
}
StepKernel<float, __nv_bfloat16> step16_for(int m, int stage = 0) {
  return reinterpret_cast<StepKernel<float, __nv_bfloat16>>(const_cast<void*>(lsg_steps::step_kernel_bf16(m, stage)));
}

}  // namespace

// ==========================================================================
// host side
// ==========================================================================
namespace {
// Raise (never lower) a kernel's dynamic shared-memory limit. The attribute
// belongs to the function and the device, process-wide, and handles of
// different shapes launch the same kernels with different amounts: lowering it
// for one handle would make another's launches fail.
cudaError_t raise_smem_limit(const void* f, size_t bytes) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> cur;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& c = cur[{dev, f}];
  if (bytes <= c) return cudaSuccess;
  e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e == cudaSuccess) c = bytes;
  return e;
}

}  // namespace

struct gmres_ctx {
  int64_t n = 0, nnz = 0;
  int m = 0;
  double tol = 0.0;
  int max_iter = 0;
  int ortho = GMRES_ONE_REDUCE_MGS;
  int prec = GMRES_FP64;
  int device = 0;
  int nsm = 0;
  int P = 0;          // CTAs of reduction kernels
  int P32 = 0;        // CTAs of the FP32-cycle step kernel (3 resident per SM)
  int P16 = 0;        // CTAs of the BF16-basis step kernel (3 per SM; 2 in staging modes 3 and 4)
  int grid_stream = 0;// CTAs of streaming kernels
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  double* V = nullptr;
  int2* VL = nullptr;  // the basis as fixed-point limbs (Small::VL; staging mode 6 only)
  int64_t ldv = 0;
  double* w = nullptr;
  char* small = nullptr;
  Small s{};
  DevState* h_st = nullptr;  // pinned mirror
  cudaStream_t stream = nullptr;
  StepKernel<double> step = nullptr;
  ReorthKernel reorth = nullptr;
  StepKernel<float> step32 = nullptr;
  StepKernel<float, __nv_bfloat16> step16 = nullptr;
  // GMRES-IR (FP32 cycles): FP32 (or BF16) basis, FP32 SpMV result and matrix
  // values, and the FP64 restart residual; allocated by gmres_set
  float* V32 = nullptr;
  __nv_bfloat16* V16 = nullptr;
  float* w32 = nullptr;
  float* val32 = nullptr;
  double* r64 = nullptr;
  size_t step_smem = 0;  // dynamic shared memory of the step kernel (T and scales)
  // Staged CSR of the step kernels (FP64 cycles; FP32 cycles): mode 0 off,
  // 1 tiles, 2 tile pairs; entry capacity; dynamic shared memory at launch.
  int stage64 = 0, cap64 = 0, stage32 = 0, cap32 = 0, stage16 = 0, cap16 = 0;
  int stall_test = 0;  // gmres_test_stall_staging
  // FP64 block dot of staging mode 2 on the integer pipes (mode 6; on by
  // default, gmres_set_block_dot)
  int dot_fx = 1;
  // whole cycles in one cooperative launch (gmres_set_persistent): -1 auto,
  // 0 off, 1 on; the kernel, whether it fits the device at once, its grid
  // barrier words (in the small block) and the barrier test switch
  int persist = -1;
  CycleKernel cyc = nullptr;
  bool cyc_ok = false;
  unsigned int* bar = nullptr;
  unsigned int bar_extra = 0;
  size_t smem64 = 0, smem32 = 0, smem16 = 0;
  size_t lsq_smem = 0;   // dynamic shared memory of k_lsq (rotated Hessenberg)
  std::vector<double> hist;
  int hist_len = 0;
  double* h_b = nullptr;  // pinned staging for gmres_solve_host
  double* h_x = nullptr;
  double* d_b = nullptr;  // device staging for gmres_solve_host
  double* d_x = nullptr;
  int64_t launches = 0;
  std::string err;
  // per-kernel timing (gmres_set_profile)
  struct ProfRec {
    int cls, j, i;
    cudaEvent_t a, b;
  };
  bool prof_on = false;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  std::vector<ProfRec> recs;
  // CUDA graphs of whole cycles (captured once per scheme, kmax and profiling
  // mode; used when the handle has a non-default stream)
  struct CycleGraph {
    int ortho, prec, kmax;
    bool prof;
    cudaGraphExec_t exec;
    int64_t nlaunch;
    std::vector<ProfRec> recs;
    std::vector<cudaEvent_t> events;
  };
  std::vector<CycleGraph> graphs;
  bool capturing = false;
  bool graph_prof_ok = true;  // false once a capture with timing events has failed
  CycleGraph* cap = nullptr;
  size_t cap_ev_used = 0;
  double prof_ms[GMRES_PROFILE_CLASSES] = {};
  double prof_bytes[GMRES_PROFILE_CLASSES] = {};
  double prof_flops[GMRES_PROFILE_CLASSES] = {};
  int64_t prof_cnt[GMRES_PROFILE_CLASSES] = {};
};

namespace {

// Handle-less errors (failed create, the no-alloc entry point): one string per
// host thread, so concurrent callers never share or tear it.
thread_local std::string g_create_err;

// Device address of g_noalloc_scratch, looked up once per device (the host
// symbol is only a stand-in and must never be passed to a kernel).
constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
int g_noalloc_nsm[kNoAllocMaxDevices] = {};


gmres_status fail(gmres_ctx* h, gmres_status st, const std::string& msg) {
  if (h)
    h->err = msg;
  else
    g_create_err = msg;
  return st;
}

#define CUDA_TRY(h, call)                                                                        \
  do {                                                                                           \
    cudaError_t e_ = (call);                                                                     \
    if (e_ != cudaSuccess)                                                                       \
      return fail(h, e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA,           \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                           \
  } while (0)

#define LAUNCH_CHECK(h)                                                                          \
  do {                                                                                           \
    cudaError_t e_ = cudaGetLastError();                                                         \
    if (e_ != cudaSuccess) return fail(h, GMRES_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e_)); \
  } while (0)


void destroy_graphs(gmres_ctx* h);

// Staging mode 6 keeps the basis a second time as fixed-point limbs
// (Small::VL, 8 bytes per entry, m + 1 columns): allocated when the mode is
// first chosen.
cudaError_t ensure_limbs(gmres_ctx* h) {
  if (fx_stage(h->stage64, h->dot_fx) != 6 || h->VL) return cudaSuccess;
  const size_t bytes = sizeof(int2) * (size_t)h->ldv * (h->m + 1);
  cudaError_t e = cudaMalloc(&h->VL, bytes);
  if (e == cudaSuccess) e = cudaMemset(h->VL, 0, bytes);
  if (e != cudaSuccess) {
    cudaFree(h->VL);
    h->VL = nullptr;
    return e;
  }
  h->s.VL = h->VL;
  h->s.ldl = h->ldv;
  return cudaSuccess;
}

gmres_status alloc_small(gmres_ctx* h) {
  destroy_graphs(h);  // captured graphs hold pointers into the old block
  const int m = h->m, ld = m + 1;
  const int nvmax = 2 * (m + 1) + 2;
  h->s.m = m;
  h->s.ldh = ld;
  h->s.nvmax = nvmax;
  h->s.hist_cap = h->max_iter + m + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    size_t o = off;
    off = align_up(off + bytes, 256);
    return o;
  };
  const size_t o_st = take(sizeof(DevState));
  const size_t o_H = take(sizeof(double) * ld * m);
  const size_t o_R = take(sizeof(double) * ld * m);
  const size_t o_cs = take(sizeof(double) * (m + 1));
  const size_t o_sn = take(sizeof(double) * (m + 1));
  const size_t o_g = take(sizeof(double) * (m + 2));
  const size_t o_T = take(sizeof(double) * ld * ld);
  const size_t o_sc = take(sizeof(double) * (m + 2));
  const size_t o_cf = take(sizeof(double) * (m + 3));
  const size_t o_cx = take(sizeof(double) * (m + 3));
  const size_t o_hi = take(sizeof(double) * h->s.hist_cap);
  const int Pmax = std::max({h->P, h->P32, h->P16});  // rows: one per CTA, then one per group of 16 CTAs
  const size_t o_pa = take(sizeof(double) * (size_t)(Pmax + (Pmax + kGridGroup - 1) / kGridGroup) * nvmax);
  const size_t o_raw = take(sizeof(double) * nvmax);
  const size_t o_ec = take(sizeof(unsigned int) * (m + 2));
  const size_t o_bar = take(sizeof(unsigned int) * 3);
  if (h->small) cudaFree(h->small);
  h->small = nullptr;
  CUDA_TRY(h, cudaMalloc(&h->small, off));
  CUDA_TRY(h, cudaMemset(h->small, 0, off));
  char* b = h->small;
  h->s.st = reinterpret_cast<DevState*>(b + o_st);
  h->s.H = reinterpret_cast<double*>(b + o_H);
  h->s.Rg = reinterpret_cast<double*>(b + o_R);
  h->s.cs = reinterpret_cast<double*>(b + o_cs);
  h->s.sn = reinterpret_cast<double*>(b + o_sn);
  h->s.g = reinterpret_cast<double*>(b + o_g);
  h->s.T = reinterpret_cast<double*>(b + o_T);
  h->s.scale = reinterpret_cast<double*>(b + o_sc);
  h->s.coef = reinterpret_cast<double*>(b + o_cf);
  h->s.coefx = reinterpret_cast<double*>(b + o_cx);
  h->s.hist = reinterpret_cast<double*>(b + o_hi);
  h->s.partials = reinterpret_cast<double*>(b + o_pa);
  h->s.raw = reinterpret_cast<double*>(b + o_raw);
  h->s.ecol = reinterpret_cast<unsigned int*>(b + o_ec);
  h->bar = reinterpret_cast<unsigned int*>(b + o_bar);
  h->hist.assign(h->s.hist_cap, 0.0);
  return GMRES_OK;
}

gmres_status read_state(gmres_ctx* h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->h_st, h->s.st, sizeof(DevState), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return GMRES_OK;
}

gmres_status write_state(gmres_ctx* h) {
  CUDA_TRY(h, cudaMemcpyAsync(h->s.st, h->h_st, sizeof(DevState), cudaMemcpyHostToDevice, h->stream));
  return GMRES_OK;
}

int prof_begin(gmres_ctx* h, int cls, int j, int i);
void prof_end(gmres_ctx* h, int idx);

// Launch the kernels of one cycle of kmax steps (the state was reset by the
// residual kernel). Kernels past the end of the cycle return at once.
gmres_status launch_cycle(gmres_ctx* h, int kmax) {
  const int P = h->P;
  if (h->ortho != GMRES_MGS) {  // one-reduce, its L = 2 pipeline, and cgs2_lvl2
    for (int j = 0; j <= kmax; ++j) {
      int pr = prof_begin(h, 0, j, kmax);
      if (h->prec == GMRES_IR_FP32)
        h->step32<<<h->P32, kThreads, h->smem32, h->stream>>>(h->rowptr, h->col, h->val32, h->V32, h->ldv, nullptr,
                                                              h->w32, h->n, h->s, 0, 1, nullptr, h->stage32,
                                                              h->cap32);
      else if (h->prec == GMRES_IR_BF16)
        h->step16<<<h->P16, kThreads, h->smem16, h->stream>>>(h->rowptr, h->col, h->val32, h->V16, h->ldv, nullptr,
                                                              h->w32, h->n, h->s, 0, 1, nullptr, h->stage16,
                                                              h->cap16);
      else
        h->step<<<P, kThreads, h->smem64, h->stream>>>(h->rowptr, h->col, h->val, h->V, h->ldv, nullptr, h->w, h->n,
                                                       h->s, 0, 1, nullptr, h->stage64, h->cap64);
      prof_end(h, pr);
      ++h->launches;
      if (j < kmax) {
        pr = prof_begin(h, 1, j, kmax);
        if (h->prec == GMRES_IR_FP32)
          k_maxpy<float, float, float><<<h->grid_stream + 1, kThreads, 0, h->stream>>>(
              h->V32, h->ldv, h->w32, nullptr, h->n, h->s, MAXPY_ARNOLDI, 0);
        else if (h->prec == GMRES_IR_BF16)
          k_maxpy_bf16<<<h->grid_stream + 1, kThreads, 0, h->stream>>>(h->V16, h->ldv, h->w32, h->n, h->s);
        else if (fx_stage(h->stage64, h->dot_fx) == 6)  // large systems: the fixed-point form with the step's
          k_maxpy_fx<<<h->grid_stream + 1, kThreads, 0, h->stream>>>(h->V, h->ldv, h->w, h->n, h->s,
                                                                     MAXPY_ARNOLDI, nullptr);
        else
          k_maxpy<double, double, double><<<h->grid_stream + 1, kThreads, 0, h->stream>>>(
              h->V, h->ldv, h->w, nullptr, h->n, h->s, MAXPY_ARNOLDI, 0);
        prof_end(h, pr);
        ++h->launches;
        if (h->ortho == GMRES_CGS2_LVL2) {  // Algorithm 5's second reduction and projection
          pr = prof_begin(h, PC_REORTH, j, kmax);
          h->reorth<<<P, kThreads, 0, h->stream>>>(h->V, h->ldv, h->n, h->s);
          prof_end(h, pr);
          pr = prof_begin(h, PC_REORTH_MAXPY, j, kmax);
          k_maxpy<double, double, double><<<h->grid_stream, kThreads, 0, h->stream>>>(
              h->V, h->ldv, nullptr, nullptr, h->n, h->s, MAXPY_REORTH, 0);
          prof_end(h, pr);
          h->launches += 2;
        }
      }
    }
  } else {
    for (int i = 0; i < kmax; ++i) {
      int pr = prof_begin(h, 2, i, 0);
      k_mgs_spmv<<<P, kThreads, 0, h->stream>>>(h->rowptr, h->col, h->val, h->V, h->ldv, h->n, h->s);
      prof_end(h, pr);
      ++h->launches;
      for (int k = 0; k <= i; ++k) {
        pr = prof_begin(h, 3, i, k);
        k_mgs_axpy_dot<<<P, kThreads, 0, h->stream>>>(h->V, h->ldv, h->n, h->s);
        prof_end(h, pr);
        ++h->launches;
      }
    }
  }
  LAUNCH_CHECK(h);
  return GMRES_OK;
}

gmres_status check_ptr(gmres_ctx* h, const void* p, const char* what) {
  if (!p) return fail(h, GMRES_ERR_ARG, std::string(what) + " is NULL");
  if (reinterpret_cast<uintptr_t>(p) & 7) return fail(h, GMRES_ERR_ARG, std::string(what) + " is not 8-byte aligned");
  return GMRES_OK;
}


// Record an event pair around the next launch (no-op unless profiling).
int prof_begin(gmres_ctx* h, int cls, int j, int i) {
  if (!h->prof_on) return -1;
  if (h->capturing) {  // events pre-created for the graph being captured
    if (h->cap_ev_used + 2 > h->cap->events.size()) return -1;
    gmres_ctx::ProfRec r{cls, j, i, h->cap->events[h->cap_ev_used], h->cap->events[h->cap_ev_used + 1]};
    h->cap_ev_used += 2;
    cudaEventRecordWithFlags(r.a, h->stream, cudaEventRecordExternal);  // a timing node in the graph
    h->cap->recs.push_back(r);
    return (int)h->cap->recs.size() - 1;
  }
  while (h->ev_used + 2 > h->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    h->ev_pool.push_back(e);
  }
  gmres_ctx::ProfRec r{cls, j, i, h->ev_pool[h->ev_used], h->ev_pool[h->ev_used + 1]};
  h->ev_used += 2;
  cudaEventRecord(r.a, h->stream);
  h->recs.push_back(r);
  return (int)h->recs.size() - 1;
}

void prof_end(gmres_ctx* h, int idx) {
  if (idx < 0) return;
  if (h->capturing)
    cudaEventRecordWithFlags(h->cap->recs[idx].b, h->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(h->recs[idx].b, h->stream);
}

void destroy_graphs(gmres_ctx* h) {
  for (auto& g : h->graphs) {
    cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : g.events) cudaEventDestroy(e);
  }
  h->graphs.clear();
}

gmres_status launch_cycle(gmres_ctx* h, int kmax);

// One cycle of kmax steps. With a non-default stream the cycle's fixed launch
// sequence is captured once into a CUDA graph (per scheme, kmax and profiling
// mode) and replayed; kernels read their step index from device state, so the
// same graph serves every cycle. On the legacy default stream (which cannot be
// captured) the kernels are launched one by one.
// Whether the next cycle runs as one cooperative launch (gmres_set_persistent).
// CTAs of the one-launch cycle: up to two per SM of work CTAs (the reduction
// grid, one fewer) and the Givens CTA.
int persistent_grid(const gmres_ctx* h) {
  const int64_t ntiles = (h->n + kThreads - 1) / kThreads;
  return (int)std::min<int64_t>(2 * (int64_t)h->nsm - 1, ntiles) + 1;
}

bool use_persistent(const gmres_ctx* h) {
  if (!h->cyc_ok || h->prec != GMRES_FP64 || h->persist == 0) return false;
  if (h->ortho != GMRES_ONE_REDUCE_MGS && h->ortho != GMRES_ONE_REDUCE_PIPE2) return false;
  const int64_t ntiles = (h->n + kThreads - 1) / kThreads;
  return h->persist == 1 || ntiles < 2 * (int64_t)h->nsm;
}

// Whether the solution update of an FP64 cycle can run in fixed point on the
// basis limbs: the cycle ran the mode-6 step kernel (which stores the limbs of
// every column it uses; the persistent cycle and plain MGS do not), and x is
// 16-byte aligned for the kernel's two-row loads and stores.
bool xupdate_fx(const gmres_ctx* h, const double* x) {
  return h->prec == GMRES_FP64 && h->ortho != GMRES_MGS && fx_stage(h->stage64, h->dot_fx) == 6 &&
         !use_persistent(h) && (reinterpret_cast<uintptr_t>(x) & 15) == 0;
}

// One cycle of kmax steps in one cooperative launch (k_cycle_persistent).
gmres_status launch_persistent(gmres_ctx* h, int kmax) {
  CUDA_TRY(h, cudaMemsetAsync(h->bar, 0, 3 * sizeof(unsigned int), h->stream));
  const int pr = prof_begin(h, PC_CYCLE, 0, kmax);
  void* args[] = {&h->rowptr, &h->col, &h->val, &h->V, &h->ldv, &h->w, &h->n, &h->s, &h->bar, &h->bar_extra};
  CUDA_TRY(h, cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(h->cyc), dim3(persistent_grid(h)),
                                          dim3(kThreads), args, h->step_smem, h->stream));
  prof_end(h, pr);
  ++h->launches;
  LAUNCH_CHECK(h);
  return GMRES_OK;
}

gmres_status run_cycle(gmres_ctx* h, int kmax) {
  if (use_persistent(h)) return launch_persistent(h, kmax);
  if (h->stream == nullptr || (h->prof_on && !h->graph_prof_ok)) return launch_cycle(h, kmax);
  gmres_ctx::CycleGraph* g = nullptr;
  for (auto& c : h->graphs)
    if (c.ortho == h->ortho && c.prec == h->prec && c.kmax == kmax && c.prof == h->prof_on) g = &c;
  if (!g) {
    h->graphs.emplace_back();
    g = &h->graphs.back();
    g->ortho = h->ortho;
    g->prec = h->prec;
    g->kmax = kmax;
    g->prof = h->prof_on;
    g->exec = nullptr;
    const int64_t nl = (h->ortho == GMRES_MGS)         ? (int64_t)kmax + (int64_t)kmax * (kmax + 1) / 2
                       : (h->ortho == GMRES_CGS2_LVL2) ? 4 * (int64_t)kmax + 1
                                                       : 2 * (int64_t)kmax + 1;
    if (h->prof_on) {
      g->events.resize(2 * nl);
      for (auto& e : g->events) CUDA_TRY(h, cudaEventCreate(&e));
    }
    const int64_t before = h->launches;
    h->capturing = true;
    h->cap = g;
    h->cap_ev_used = 0;
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal);
    gmres_status st = GMRES_OK;
    if (e == cudaSuccess) st = launch_cycle(h, kmax);
    cudaError_t e2 = cudaStreamEndCapture(h->stream, &graph);
    h->capturing = false;
    h->cap = nullptr;
    g->nlaunch = h->launches - before;
    h->launches = before;
    if (e != cudaSuccess || e2 != cudaSuccess || st != GMRES_OK) {
      if (graph) cudaGraphDestroy(graph);
      for (cudaEvent_t ev : g->events) cudaEventDestroy(ev);
      h->graphs.pop_back();
      cudaGetLastError();
      if (!h->prof_on)
        return fail(h, GMRES_ERR_CUDA, std::string("cycle graph capture failed: ") +
                                            cudaGetErrorString(e != cudaSuccess ? e : e2));
      h->graph_prof_ok = false;  // timed launches are not capturable here: launch them directly
      h->err.clear();
      return launch_cycle(h, kmax);
    }
    e = cudaGraphInstantiate(&g->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
      h->graphs.pop_back();
      return fail(h, GMRES_ERR_CUDA, std::string("cudaGraphInstantiate: ") + cudaGetErrorString(e));
    }
  }
  CUDA_TRY(h, cudaGraphLaunch(g->exec, h->stream));
  h->launches += g->nlaunch;
  if (h->prof_on)
    for (const auto& r : g->recs) h->recs.push_back(r);
  return GMRES_OK;
}

// Algorithmic traffic and flops of one launch that did work (FP64: 8-byte
// values, 4-byte indices; a vector read once counts once).
void alg_model(const gmres_ctx* h, const gmres_ctx::ProfRec& r, int kx, double* bytes, double* flops) {
  const double n = (double)h->n, nnz = (double)h->nnz;
  // FP32 cycles: 4-byte values and w; basis vectors 4 bytes (FP32) or 2 (BF16)
  const bool f32 = h->prec == GMRES_IR_FP32 || h->prec == GMRES_IR_BF16;
  const double wb = f32 ? 4.0 : 8.0;
  const double vb = h->prec == GMRES_IR_BF16 ? 2.0 : wb;
  const double csr = 4.0 * (n + 1) + (4.0 + (f32 && (r.cls == PC_STEP) ? 4.0 : 8.0)) * nnz;
  switch (r.cls) {
    case PC_STEP:
      if (r.j == r.i) {  // tail: u and V_j, no SpMV (r.i carries kmax)
        *bytes = vb * n * (r.j + 1);
        *flops = 2.0 * n * (r.j + 1);
      } else {
        *bytes = csr + vb * n * (r.j + 1) + wb * n;  // u (gathered), j basis columns, w written
        *flops = 2.0 * nnz + 2.0 * n * (2.0 * r.j + 2.0);
      }
      break;
    case PC_CYCLE: {  // every step and MAXPY of a cycle that completed k columns (tail at kmax)
      double by = 0.0, fl = 0.0;
      for (int jj = 0; jj <= std::min(kx, r.i); ++jj) {
        const bool tl = (jj == r.i);
        by += tl ? vb * n * (jj + 1) : csr + vb * n * (jj + 1) + wb * n;
        fl += tl ? 2.0 * n * (jj + 1) : 2.0 * nnz + 2.0 * n * (2.0 * jj + 2.0);
        if (jj < kx && jj < r.i) {
          by += wb * n + vb * n * (jj + 2);
          fl += 2.0 * n * (jj + 1) + n;
        }
      }
      *bytes = by;
      *flops = fl;
      break;
    }
    case PC_MAXPY:  // w and j+1 columns read, one column written
      *bytes = wb * n + vb * n * (r.j + 2);
      *flops = 2.0 * n * (r.j + 1) + n;
      break;
    case PC_REORTH:  // z and j+1 basis columns read
      *bytes = 8.0 * n * (r.j + 2);
      *flops = 2.0 * n * (r.j + 2);
      break;
    case PC_REORTH_MAXPY:  // z and j+1 columns read, z written
      *bytes = 8.0 * n * (r.j + 3);
      *flops = 2.0 * n * (r.j + 1) + n;
      break;
    case PC_MGS_SPMV:  // u_i gathered, u_0 read, w written
      *bytes = csr + 24.0 * n;
      *flops = 2.0 * nnz + 3.0 * n;
      break;
    case PC_MGS_AXPY:  // w read+written, u_k, u_{k+1} read (the last reads only u_k)
      *bytes = (r.i == r.j) ? 24.0 * n : 32.0 * n;
      *flops = 4.0 * n;
      break;
    case PC_RES:
      *bytes = (r.j == 0) ? 8.0 * n : csr + 24.0 * n;
      *flops = (r.j == 0) ? 2.0 * n : 2.0 * nnz + 3.0 * n;
      break;
    case PC_XUPD:  // x read and written (FP64), kx basis columns
      *bytes = 16.0 * n + vb * n * kx;
      *flops = 2.0 * n * kx + n;
      break;
    default:
      *bytes = 0.0;
      *flops = 0.0;
  }
}

// After the stream is synchronized: attribute the recorded launches of one
// cycle that completed k columns (work or no-op) and recycle the events.
void prof_settle(gmres_ctx* h, int k) {
  if (!h->prof_on) return;
  for (const auto& r : h->recs) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    bool work = true;
    if (r.cls == PC_STEP) work = r.j <= k;
    else if (r.cls == PC_MAXPY) work = r.j <= k && r.j < r.i;  // also runs after the stopping step
    else if (r.cls == PC_MGS_SPMV || r.cls == PC_MGS_AXPY || r.cls == PC_REORTH || r.cls == PC_REORTH_MAXPY)
      work = r.j < k;
    const int c = work ? r.cls : PC_NOOP;
    h->prof_ms[c] += ms;
    h->prof_cnt[c] += 1;
    if (work) {
      double by, fl;
      alg_model(h, r, k, &by, &fl);
      h->prof_bytes[c] += by;
      h->prof_flops[c] += fl;
    }
  }
  h->recs.clear();
  h->ev_used = 0;
}

void prof_reset(gmres_ctx* h) {
  for (int c = 0; c < GMRES_PROFILE_CLASSES; ++c) {
    h->prof_ms[c] = h->prof_bytes[c] = h->prof_flops[c] = 0.0;
    h->prof_cnt[c] = 0;
  }
  h->recs.clear();
  h->ev_used = 0;
}

}  // namespace

extern "C" {

extern "C++" {
// Largest staged entry range of a 256-row tile and of a 512-row tile pair
// (the range [rowptr[first] rounded down, rowptr[last + 1] rounded up to 4),
// as the step kernel copies it). rp is padded past n with nnz.
static void csr_stage_caps(const std::vector<int32_t>& rp, int64_t n, int& cap_tile, int& cap_pair) {
  cap_tile = cap_pair = 0;
  for (int U : {kThreads, 2 * kThreads}) {
    int64_t best = 0;
    for (int64_t r = 0; r < n; r += U) {
      const int64_t lo = rp[r] & ~3, hi = ((int64_t)rp[r + U] + 3) & ~3;
      best = std::max(best, hi - lo);
    }
    (U == kThreads ? cap_tile : cap_pair) = (int)std::min<int64_t>(best, 1 << 30);
  }
}

// Staging of a step kernel with values of vb bytes, launched on P CTAs of
// which `per_sm` must stay resident per SM: tile pairs when the unstaged kernel
// would take pairs (ntiles >= 4 P) and their buffer fits, else single tiles if
// theirs fits, else off. With v3_bytes > 0 (the basis columns of a tile, BF16
// basis), modes with the unit's basis columns staged too are tried next (first
// when the kernel has no column ring), at two CTAs per SM: 4 (tile pairs: bulk
// copies of twice the size, half as many), then 3 (single tiles); *P is then
// lowered to two CTAs per SM. kernel_for(stage)
// gives the kernel of a mode; the dynamic shared memory is the larger of the
// epilogue's (t_smem) and the staging buffer's (plus pair_extra bytes behind
// a tile pair's CSR in mode 2: the kernel's column ring; mode 5 is the same
// tile-pair kernel without it). Sets the kernel's
// shared-memory limit.
template <typename KernelFor>
static gmres_status choose_stage(KernelFor kernel_for, size_t vb, int per_sm, int* P, int nsm, int64_t ntiles,
                                 int cap_tile, int cap_pair, size_t t_smem, size_t v3_bytes, size_t pair_extra,
                                 int& mode, int& cap, size_t& smem) {
  const bool pairs = ntiles >= 4 * (int64_t)*P;
  // a kernel with the column ring (pair_extra > 0) takes tile pairs at per_sm
  // CTAs per SM first (at 256^3 7-point the BF16 basis streamed through the
  // ring, 0.523 s, beat its bulk-copy staging, mode 4, 0.583 s), then tile
  // pairs without the ring (mode 5: where the pair CSR leaves no room for it)
  const int order_ring[5] = {2, 5, 4, 3, 1}, order_bulk[5] = {4, 3, 2, 1, 0};
  for (int cand : (pair_extra > 0 ? order_ring : order_bulk)) {
    if (cand == 0) continue;
    const bool sv = cand == 3 || cand == 4;  // basis columns staged too
    // staged basis: at least 4 tiles per CTA at two CTAs per SM
    if (sv && (v3_bytes == 0 || ntiles < 4 * 2 * (int64_t)nsm)) continue;
    if ((cand == 2 || cand == 5) && !pairs) continue;
    const bool pr = cand == 2 || cand == 4 || cand == 5;
    const int U = pr ? 2 * kThreads : kThreads;
    const int c = pr ? cap_pair : cap_tile;
    const size_t need = std::max(t_smem, (size_t)(U + 4) * 4 + (size_t)c * (4 + vb) +
                                             (sv ? (pr ? 2 : 1) * v3_bytes : 0) + (cand == 2 ? pair_extra : 0));
    if (need > 200 * 1024) continue;
    const void* k = reinterpret_cast<const void*>(kernel_for(cand));
    if (raise_smem_limit(k, need) != cudaSuccess)
      return GMRES_ERR_CUDA;
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, kThreads, need) != cudaSuccess) return GMRES_ERR_CUDA;
    if (nb >= (sv ? 2 : per_sm)) {
      mode = cand;
      cap = c;
      smem = need;
      if (sv) *P = (int)std::min<int64_t>(2 * (int64_t)nsm, cand == 4 ? (ntiles + 1) / 2 : ntiles);
      return GMRES_OK;
    }
  }
  mode = 0;
  cap = 0;
  smem = t_smem;
  if (raise_smem_limit(reinterpret_cast<const void*>(kernel_for(0)), t_smem) != cudaSuccess)
    return GMRES_ERR_CUDA;
  return GMRES_OK;
}
}  // extern "C++"

gmres_status gmres_create(const gmres_csr* A, int m_restart, double tol, gmres_handle* out) {
  if (!out) return fail(nullptr, GMRES_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!A || !A->rowptr || (A->nnz > 0 && (!A->col || !A->val)))
    return fail(nullptr, GMRES_ERR_ARG, "A or its arrays are NULL");
  if (A->n <= 0 || A->nnz < 0 || A->nnz >= (int64_t)INT32_MAX || A->n >= (int64_t)INT32_MAX)
    return fail(nullptr, GMRES_ERR_ARG, "n must be in [1, 2^31) and nnz in [0, 2^31)");
  if (m_restart < 1 || m_restart > kMaxM) return fail(nullptr, GMRES_ERR_ARG, "m_restart must be in [1, 128]");
  if (!(tol >= 0.0)) return fail(nullptr, GMRES_ERR_ARG, "tol must be >= 0");
  const int64_t n = A->n, nnz = A->nnz;
  // host copies for validation
  std::vector<int32_t> rp(n + 1), cl(nnz);
  std::vector<double> vl(nnz);
  if (A->on_device) {
    if (cudaMemcpy(rp.data(), A->rowptr, sizeof(int32_t) * (n + 1), cudaMemcpyDeviceToHost) != cudaSuccess ||
        (nnz && cudaMemcpy(cl.data(), A->col, sizeof(int32_t) * nnz, cudaMemcpyDeviceToHost) != cudaSuccess) ||
        (nnz && cudaMemcpy(vl.data(), A->val, sizeof(double) * nnz, cudaMemcpyDeviceToHost) != cudaSuccess))
      return fail(nullptr, GMRES_ERR_CUDA, "cannot read device CSR arrays");
  } else {
    std::memcpy(rp.data(), A->rowptr, sizeof(int32_t) * (n + 1));
    if (nnz) {
      std::memcpy(cl.data(), A->col, sizeof(int32_t) * nnz);
      std::memcpy(vl.data(), A->val, sizeof(double) * nnz);
    }
  }
  if (rp[0] != 0 || rp[n] != nnz) return fail(nullptr, GMRES_ERR_ARG, "rowptr[0] must be 0 and rowptr[n] = nnz");
  for (int64_t i = 0; i < n; ++i)
    if (rp[i + 1] < rp[i]) return fail(nullptr, GMRES_ERR_ARG, "rowptr is not nondecreasing");
  for (int64_t p = 0; p < nnz; ++p)
    if (cl[p] < 0 || cl[p] >= n) return fail(nullptr, GMRES_ERR_ARG, "column index out of range");
  for (int64_t p = 0; p < nnz; ++p)
    if (!std::isfinite(vl[p])) return fail(nullptr, GMRES_ERR_NONFINITE, "non-finite matrix value");

  gmres_ctx* h = new gmres_ctx();
  h->n = n;
  h->nnz = nnz;
  h->m = m_restart;
  h->tol = tol;
  h->max_iter = 10 * m_restart;
  auto bail = [&](gmres_status st) {
    g_create_err = h->err;
    gmres_destroy(h);
    return st;
  };
#define CREATE_TRY(call)                                                               \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      h->err = std::string(#call) + ": " + cudaGetErrorString(e_);                     \
      return bail(e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA);   \
    }                                                                                  \
  } while (0)
  CREATE_TRY(cudaGetDevice(&h->device));
  CREATE_TRY(cudaDeviceGetAttribute(&h->nsm, cudaDevAttrMultiProcessorCount, h->device));
  const int64_t ntiles = (n + kThreads - 1) / kThreads;
  h->P = (int)std::min<int64_t>(2 * (int64_t)h->nsm, ntiles);
  h->P32 = (int)std::min<int64_t>(3 * (int64_t)h->nsm, ntiles);
  h->P16 = h->P32;
  h->grid_stream = (int)std::min<int64_t>(4 * (int64_t)h->nsm, std::max<int64_t>(1, (n / 2 + kThreads - 1) / kThreads));
  const int64_t nnz_pad = align_up(std::max<int64_t>(nnz, 1), 4);
  // rowptr is padded with nnz to a whole number of 512-row tile pairs + 8, so
  // that a staged unit's rowptr slice (U + 4 entries) is always in bounds
  const int64_t rp_len = (int64_t)align_up((size_t)n, 2 * kThreads) + 8;
  rp.resize(rp_len, (int32_t)nnz);
  CREATE_TRY(cudaMalloc(&h->rowptr, sizeof(int32_t) * rp_len));
  CREATE_TRY(cudaMalloc(&h->col, sizeof(int32_t) * nnz_pad));
  CREATE_TRY(cudaMalloc(&h->val, sizeof(double) * nnz_pad));
  CREATE_TRY(cudaMemset(h->col, 0, sizeof(int32_t) * nnz_pad));
  CREATE_TRY(cudaMemset(h->val, 0, sizeof(double) * nnz_pad));
  CREATE_TRY(cudaMemcpy(h->rowptr, rp.data(), sizeof(int32_t) * rp_len, cudaMemcpyHostToDevice));
  if (nnz) {
    CREATE_TRY(cudaMemcpy(h->col, cl.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemcpy(h->val, vl.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice));
  }
  // whole tile pairs: a staged copy of a tile's slice of a basis column stays
  // inside its column
  h->ldv = (int64_t)align_up((size_t)n, 2 * kThreads);
  CREATE_TRY(cudaMalloc(&h->V, sizeof(double) * (size_t)h->ldv * (m_restart + 1)));
  CREATE_TRY(cudaMemset(h->V, 0, sizeof(double) * (size_t)h->ldv * (m_restart + 1)));
  CREATE_TRY(cudaMalloc(&h->w, sizeof(double) * (size_t)h->ldv));
  CREATE_TRY(cudaMemset(h->w, 0, sizeof(double) * (size_t)h->ldv));
  CREATE_TRY(cudaMallocHost(&h->h_st, sizeof(DevState)));
  std::memset(h->h_st, 0, sizeof(DevState));
  if (alloc_small(h) != GMRES_OK) return bail(GMRES_ERR_CUDA);
  h->reorth = reorth_kernel_for(m_restart);
  h->step_smem = sizeof(double) * ((size_t)(m_restart + 1) * (m_restart + 1) + (m_restart + 1));
  h->lsq_smem = sizeof(double) * (size_t)(m_restart + 1) * m_restart;
  {
    int cap_tile = 0, cap_pair = 0;
    csr_stage_caps(rp, n, cap_tile, cap_pair);
    const int m = m_restart;
    gmres_status sst = choose_stage([m](int sg) { return step64_for(m, sg); }, sizeof(double), 2, &h->P, h->nsm,
                                    ntiles, cap_tile, cap_pair, h->step_smem, 0, pf_ring_bytes<double>(), h->stage64,
                                    h->cap64, h->smem64);
    if (sst == GMRES_OK)
      // FP32 basis: no mode 3 (measured: equal at 192^3 27-point, 16% slower at 256^3
      // 7-point than three CTAs per SM reading the basis themselves); the BF16
      // basis, whose 2-byte loads use sectors poorly, gains from it (31% at 192^3)
      sst = choose_stage([m](int sg) { return step32_for(m, sg); }, sizeof(float), 3, &h->P32, h->nsm, ntiles,
                         cap_tile, cap_pair, h->step_smem, 0, pf_ring_bytes<float>(),
                         h->stage32, h->cap32, h->smem32);
    if (sst == GMRES_OK)
      sst = choose_stage([m](int sg) { return step16_for(m, sg); }, sizeof(float), 3, &h->P16, h->nsm, ntiles,
                         cap_tile, cap_pair, h->step_smem, (size_t)m * kThreads * sizeof(__nv_bfloat16),
                         pf_ring_bytes<__nv_bfloat16>(),
                         h->stage16, h->cap16, h->smem16);
    if (sst != GMRES_OK) {
      h->err = "cudaFuncSetAttribute / occupancy query of the step kernels failed";
      return bail(GMRES_ERR_CUDA);
    }
    if ((h->stage64 == 2 &&
         raise_smem_limit(reinterpret_cast<const void*>(step64_for(m, 6)), h->smem64) != cudaSuccess) ||
        raise_smem_limit(reinterpret_cast<const void*>(step64_for(m, 0)), h->step_smem) != cudaSuccess) {
      h->err = "cudaFuncSetAttribute of the fixed-point or unstaged step kernel failed";
      return bail(GMRES_ERR_CUDA);
    }
    if (cudaError_t e = ensure_limbs(h); e == cudaErrorMemoryAllocation) {
      // no room for the limb copy beside the basis: the handle starts with
      // FP64 products (gmres_set_block_dot reports which form is active)
      cudaGetLastError();
      h->dot_fx = 0;
    } else if (e != cudaSuccess) {
      h->err = std::string("limb copy of the basis: ") + cudaGetErrorString(e);
      return bail(GMRES_ERR_CUDA);
    }
    h->step = step64_for(m, fx_stage(h->stage64, h->dot_fx));
    h->step32 = step32_for(m, h->stage32);
    h->step16 = step16_for(m, h->stage16);
  }
  {  // whole cycles in one launch: needs cooperative launches and the grid resident at once
    h->cyc = cycle_kernel_for(h->m);
    int coop = 0, nb = 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, h->device) == cudaSuccess && coop &&
        raise_smem_limit(reinterpret_cast<const void*>(h->cyc), h->step_smem) == cudaSuccess &&
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, h->cyc, kThreads, h->step_smem) == cudaSuccess)
      h->cyc_ok = (int64_t)nb * h->nsm >= (int64_t)persistent_grid(h);
    cudaGetLastError();
  }
  CREATE_TRY(raise_smem_limit(reinterpret_cast<const void*>(k_lsq), h->lsq_smem));
#undef CREATE_TRY
  *out = h;
  return GMRES_OK;
}

gmres_status gmres_set(gmres_handle h, gmres_ortho ortho, gmres_prec prec, int max_iter) {
  if (!h) return GMRES_ERR_ARG;
  if (ortho != GMRES_MGS && ortho != GMRES_ONE_REDUCE_MGS && ortho != GMRES_CGS2_LVL2 &&
      ortho != GMRES_ONE_REDUCE_PIPE2)
    return fail(h, GMRES_ERR_ARG, "unknown ortho");
  if (prec != GMRES_FP64 && prec != GMRES_IR_FP32 && prec != GMRES_IR_BF16)
    return fail(h, GMRES_ERR_ARG, "precision must be GMRES_FP64, GMRES_IR_FP32 or GMRES_IR_BF16");
  if (prec != GMRES_FP64 && ortho != GMRES_ONE_REDUCE_MGS)
    return fail(h, GMRES_ERR_ARG, "GMRES-IR runs the one-reduce scheme only");
  if (max_iter < 0) return fail(h, GMRES_ERR_ARG, "max_iter < 0");
  if (prec == GMRES_IR_BF16 && !h->V16) {  // BF16 basis
    CUDA_TRY(h, cudaSetDevice(h->device));
    CUDA_TRY(h, cudaMalloc(&h->V16, sizeof(__nv_bfloat16) * (size_t)h->ldv * (h->m + 1)));
    CUDA_TRY(h, cudaMemset(h->V16, 0, sizeof(__nv_bfloat16) * (size_t)h->ldv * (h->m + 1)));
  }
  if (prec == GMRES_IR_FP32 && !h->V32) {  // FP32 basis
    CUDA_TRY(h, cudaSetDevice(h->device));
    CUDA_TRY(h, cudaMalloc(&h->V32, sizeof(float) * (size_t)h->ldv * (h->m + 1)));
    CUDA_TRY(h, cudaMemset(h->V32, 0, sizeof(float) * (size_t)h->ldv * (h->m + 1)));
  }
  if (prec != GMRES_FP64 && !h->w32) {  // FP32 values, SpMV result and the FP64 restart residual
    CUDA_TRY(h, cudaSetDevice(h->device));
    const int64_t nnz_pad = (int64_t)align_up((size_t)std::max<int64_t>(h->nnz, 1), 4);
    CUDA_TRY(h, cudaMalloc(&h->w32, sizeof(float) * (size_t)h->ldv));
    CUDA_TRY(h, cudaMemset(h->w32, 0, sizeof(float) * (size_t)h->ldv));
    CUDA_TRY(h, cudaMalloc(&h->val32, sizeof(float) * (size_t)nnz_pad));
    CUDA_TRY(h, cudaMemset(h->val32, 0, sizeof(float) * (size_t)nnz_pad));
    CUDA_TRY(h, cudaMalloc(&h->r64, sizeof(double) * (size_t)h->ldv));
    k_to_float<<<h->grid_stream, kThreads>>>(h->val, h->val32, h->nnz);
    LAUNCH_CHECK(h);
    CUDA_TRY(h, cudaDeviceSynchronize());
  }
  h->ortho = ortho;
  h->prec = prec;
  if (max_iter != h->max_iter) {
    h->max_iter = max_iter;
    gmres_status st = alloc_small(h);
    if (st != GMRES_OK) return st;
  }
  return GMRES_OK;
}

gmres_status gmres_set_tol(gmres_handle h, double tol) {
  if (!h) return GMRES_ERR_ARG;
  if (!(tol >= 0.0)) return fail(h, GMRES_ERR_ARG, "tol must be >= 0");
  h->tol = tol;
  return GMRES_OK;
}

gmres_status gmres_set_stream(gmres_handle h, void* stream) {
  if (!h) return GMRES_ERR_ARG;
  h->stream = reinterpret_cast<cudaStream_t>(stream);
  return GMRES_OK;
}

gmres_status gmres_solve(gmres_handle h, const double* b, double* x, gmres_info* info) {
  if (!h) return GMRES_ERR_ARG;
  gmres_status st;
  if ((st = check_ptr(h, b, "b")) != GMRES_OK) return st;
  if ((st = check_ptr(h, x, "x")) != GMRES_OK) return st;
  CUDA_TRY(h, cudaSetDevice(h->device));
  const auto t0 = std::chrono::steady_clock::now();
  h->launches = 0;
  // fresh state
  std::memset(h->h_st, 0, sizeof(DevState));
  h->h_st->tol = h->tol;
  h->h_st->pipe2 = h->ortho == GMRES_ONE_REDUCE_PIPE2;
  h->h_st->stall_test = h->stall_test;
  if ((st = write_state(h)) != GMRES_OK) return st;
  const int P = h->P;
  prof_reset(h);
  int pr = prof_begin(h, PC_RES, 0, 0);
  k_residual<<<P, kThreads, 0, h->stream>>>(h->rowptr, h->col, h->val, b, nullptr, nullptr, h->n, h->s, RES_BNORM, 0);
  prof_end(h, pr);
  ++h->launches;
  LAUNCH_CHECK(h);
  if ((st = read_state(h)) != GMRES_OK) return st;
  const double bnorm = h->h_st->bnorm;
  gmres_status result = GMRES_OK;
  h->hist_len = 0;
  if (!std::isfinite(bnorm)) {
    result = GMRES_ERR_NONFINITE;
    fail(h, result, "b contains NaN or Inf");
  } else if (bnorm == 0.0) {
    CUDA_TRY(h, cudaMemsetAsync(x, 0, sizeof(double) * h->n, h->stream));
    CUDA_TRY(h, cudaStreamSynchronize(h->stream));
    h->h_st->rnorm = 0.0;
  } else {
    int prev_total = 0, cycles = 0;
    for (;;) {
      pr = prof_begin(h, PC_RES, 1, 0);
      // a new cycle rewrites every basis column: clear their exponent bounds
      CUDA_TRY(h, cudaMemsetAsync(h->s.ecol, 0, sizeof(unsigned int) * (h->m + 2), h->stream));
      k_residual<<<P, kThreads, 0, h->stream>>>(h->rowptr, h->col, h->val, b, x,
                                                 h->prec != GMRES_FP64 ? h->r64 : h->V, h->n, h->s,
                                                 RES_RESIDUAL, 0);
      prof_end(h, pr);
      ++h->launches;
      LAUNCH_CHECK(h);
      if ((st = read_state(h)) != GMRES_OK) return st;
      const DevState& hs = *h->h_st;
      prof_settle(h, hs.total_iters - prev_total);
      if (hs.stalled) {  // (a cycle that gave up waiting may have completed no column)
        result = GMRES_ERR_TIMEOUT;
        fail(h, result, "a bounded device-side wait (staged CSR data or the one-launch cycle's grid barrier) "
                        "gave up");
        break;
      }
      if (cycles > 0 && hs.total_iters == prev_total) {  // every cycle completes >= 1 column
        result = GMRES_ERR_CUDA;
        fail(h, result, "internal: a cycle completed no column");
        break;
      }
      prev_total = hs.total_iters;
      ++cycles;
      if (!std::isfinite(hs.rnorm) || hs.nonfinite) {
        result = GMRES_ERR_NONFINITE;
        fail(h, result, "non-finite residual (NaN or Inf in x0 or the iteration)");
        break;
      }
      if (hs.rnorm / bnorm <= h->tol) {
        result = GMRES_OK;
        break;
      }
      if (hs.total_iters >= h->max_iter) {
        result = GMRES_MAXITER;
        break;
      }
      const int kmax = std::min(h->m, h->max_iter - hs.total_iters);
      h->h_st->kmax = kmax;
      // only kmax changes on the host side; write it without touching the rest
      CUDA_TRY(h, cudaMemcpyAsync(&h->s.st->kmax, &h->h_st->kmax, sizeof(int), cudaMemcpyHostToDevice, h->stream));
      if (h->prec == GMRES_IR_BF16) {
        k_round_scaled<<<h->grid_stream, kThreads, 0, h->stream>>>(h->r64, h->V16, h->n, h->s);
        ++h->launches;
        LAUNCH_CHECK(h);
      } else if (h->prec == GMRES_IR_FP32) {
        k_round_scaled<<<h->grid_stream, kThreads, 0, h->stream>>>(h->r64, h->V32, h->n, h->s);
        ++h->launches;
        LAUNCH_CHECK(h);
      }
      if ((st = run_cycle(h, kmax)) != GMRES_OK) return st;
      pr = prof_begin(h, PC_LSQ, 0, 0);
      k_lsq<<<1, 128, h->lsq_smem, h->stream>>>(h->s);
      prof_end(h, pr);
      pr = prof_begin(h, PC_XUPD, 0, 0);
      if (h->prec == GMRES_IR_BF16)
        k_maxpy<__nv_bfloat16, double, double><<<h->grid_stream, kThreads, 0, h->stream>>>(h->V16, h->ldv, x, x,
                                                                                           h->n, h->s,
                                                                                           MAXPY_XUPDATE, 0);
      else if (h->prec == GMRES_IR_FP32)
        k_maxpy<float, double, double><<<h->grid_stream, kThreads, 0, h->stream>>>(h->V32, h->ldv, x, x, h->n, h->s,
                                                                                  MAXPY_XUPDATE, 0);
      else if (xupdate_fx(h, x))  // the cycle stored the limbs of every column it used
        k_maxpy_fx<<<h->grid_stream, kThreads, 0, h->stream>>>(h->V, h->ldv, x, h->n, h->s, MAXPY_XUPDATE, x);
      else
        k_maxpy<double, double, double><<<h->grid_stream, kThreads, 0, h->stream>>>(h->V, h->ldv, x, x, h->n, h->s,
                                                                                   MAXPY_XUPDATE, 0);
      prof_end(h, pr);
      h->launches += 2;
      LAUNCH_CHECK(h);
    }
  }
  if ((st = read_state(h)) != GMRES_OK) return st;
  const DevState& hs = *h->h_st;
  h->hist_len = std::min(hs.total_iters, h->s.hist_cap);
  if (h->hist_len > 0)
    CUDA_TRY(h, cudaMemcpy(h->hist.data(), h->s.hist, sizeof(double) * h->hist_len, cudaMemcpyDeviceToHost));
  const auto t1 = std::chrono::steady_clock::now();
  if (info) {
    std::memset(info, 0, sizeof(*info));
    info->iters = hs.total_iters;
    info->restarts = hs.restarts;
    info->status = result;
    info->breakdowns = hs.breakdowns;
    info->rel_resid_true = bnorm > 0.0 ? hs.rnorm / bnorm : 0.0;
    info->rel_resid_est = hs.est;
    info->reductions = hs.reductions;
    info->grid_syncs = hs.grid_syncs;
    info->kernel_launches = h->launches;
    info->seconds = std::chrono::duration<double>(t1 - t0).count();
  }
  return result;
}

gmres_status gmres_solve_host(gmres_handle h, const double* b_host, double* x_host, gmres_info* info) {
  if (!h) return GMRES_ERR_ARG;
  if (!b_host || !x_host) return fail(h, GMRES_ERR_ARG, "b_host or x_host is NULL");
  const size_t bytes = sizeof(double) * h->n;
  if (!h->d_b) {
    CUDA_TRY(h, cudaMalloc(&h->d_b, bytes));
    CUDA_TRY(h, cudaMalloc(&h->d_x, bytes));
  }
  CUDA_TRY(h, cudaMemcpyAsync(h->d_b, b_host, bytes, cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(h->d_x, x_host, bytes, cudaMemcpyHostToDevice, h->stream));
  gmres_status st = gmres_solve(h, h->d_b, h->d_x, info);
  CUDA_TRY(h, cudaMemcpyAsync(x_host, h->d_x, bytes, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return st;
}

gmres_status gmres_history(gmres_handle h, double* host_buf, int cap, int* len) {
  if (!h) return GMRES_ERR_ARG;
  if (len) *len = h->hist_len;
  if (host_buf && cap > 0) std::memcpy(host_buf, h->hist.data(), sizeof(double) * std::min(cap, h->hist_len));
  return GMRES_OK;
}

gmres_status gmres_destroy(gmres_handle h) {
  if (!h) return GMRES_OK;
  cudaFree(h->rowptr);
  cudaFree(h->col);
  cudaFree(h->val);
  cudaFree(h->V);
  cudaFree(h->VL);
  cudaFree(h->w);
  cudaFree(h->small);
  cudaFree(h->d_b);
  cudaFree(h->d_x);
  cudaFree(h->V32);
  cudaFree(h->V16);
  cudaFree(h->w32);
  cudaFree(h->val32);
  cudaFree(h->r64);
  if (h->h_st) cudaFreeHost(h->h_st);
  for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
  destroy_graphs(h);
  delete h;
  return GMRES_OK;
}

const char* gmres_last_error(gmres_handle h) { return h ? h->err.c_str() : g_create_err.c_str(); }

gmres_status gmres_set_persistent(gmres_handle h, int mode, int* active) {
  if (!h) return GMRES_ERR_ARG;
  h->persist = mode < 0 ? -1 : (mode ? 1 : 0);
  if (active) *active = use_persistent(h);
  return GMRES_OK;
}

gmres_status gmres_test_stall_barrier(gmres_handle h, int on) {
  if (!h) return GMRES_ERR_ARG;
  if (on < 0 || on > 2) return fail(h, GMRES_ERR_ARG, "stall test mode must be 0, 1 or 2");
  h->bar_extra = (unsigned int)on;  // bit 0: the grid barrier; bit 1: the epilogue wait
  return GMRES_OK;
}

gmres_status gmres_set_block_dot(gmres_handle h, int fixed_point, int* active) {
  if (!h) return GMRES_ERR_ARG;
  h->dot_fx = fixed_point ? 1 : 0;
  CUDA_TRY(h, cudaSetDevice(h->device));
  if (cudaError_t e = ensure_limbs(h); e != cudaSuccess) {
    h->dot_fx = 0;  // the kernel in use stays the FP64 one
    return fail(h, e == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA,
                std::string("limb basis: ") + cudaGetErrorString(e));
  }
  auto k = step64_for(h->m, fx_stage(h->stage64, h->dot_fx));
  if (k != h->step) {
    destroy_graphs(h);  // captured cycles hold the other kernel
    h->step = k;
  }
  if (active) *active = fx_stage(h->stage64, h->dot_fx) == 6;
  return GMRES_OK;
}

gmres_status gmres_set_reproducible(gmres_handle h, int on) {
  if (!h) return GMRES_ERR_ARG;
  const int v = on ? 1 : 0;
  if (h->s.fixed_order != v) {
    destroy_graphs(h);  // captured cycles hold the kernels' Small by value
    h->s.fixed_order = v;
  }
  return GMRES_OK;
}

gmres_status gmres_test_stall_staging(gmres_handle h, int on, int* staged) {
  if (!h) return GMRES_ERR_ARG;
  h->stall_test = on ? 1 : 0;
  if (staged) *staged = h->stage64 != 0;
  return GMRES_OK;
}

gmres_status gmres_set_profile(gmres_handle h, int on) {
  if (!h) return GMRES_ERR_ARG;
  h->prof_on = on != 0;
  prof_reset(h);
  return GMRES_OK;
}

gmres_status gmres_profile(gmres_handle h, int cls, double* total_ms, int64_t* launches, double* alg_bytes,
                           double* alg_flops) {
  if (!h) return GMRES_ERR_ARG;
  if (cls < 0 || cls >= GMRES_PROFILE_CLASSES) return fail(h, GMRES_ERR_ARG, "profile class out of range");
  if (total_ms) *total_ms = h->prof_ms[cls];
  if (launches) *launches = h->prof_cnt[cls];
  if (alg_bytes) *alg_bytes = h->prof_bytes[cls];
  if (alg_flops) *alg_flops = h->prof_flops[cls];
  return GMRES_OK;
}

gmres_status lsg_spmv(gmres_handle h, const double* x, double* y) {
  if (!h) return GMRES_ERR_ARG;
  gmres_status st;
  if ((st = check_ptr(h, x, "x")) != GMRES_OK) return st;
  if ((st = check_ptr(h, y, "y")) != GMRES_OK) return st;
  k_spmv<<<h->grid_stream, kThreads, 0, h->stream>>>(h->rowptr, h->col, h->val, x, y, h->n);
  LAUNCH_CHECK(h);
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return GMRES_OK;
}

gmres_status lsg_block_dot(gmres_handle h, const double* V, int64_t ldv, int j, const double* u, double* w,
                           int use_spmv, double* X) {
  if (!h) return GMRES_ERR_ARG;
  if (j < 0 || j > h->m) return fail(h, GMRES_ERR_ARG, "j must be in [0, m]");
  if ((j > 0 && (!V || ldv < h->n)) || !u || !w || !X) return fail(h, GMRES_ERR_ARG, "bad pointer or ldv");
  CUDA_TRY(h, cudaSetDevice(h->device));
  if (j > 0) {  // the caller's columns carry no stored exponent bounds: measure them
    CUDA_TRY(h, cudaMemsetAsync(h->s.ecol, 0, sizeof(unsigned int) * (h->m + 2), h->stream));
    k_col_fields<<<dim3((unsigned)std::max(1, h->grid_stream / std::max(1, j)), (unsigned)j), kThreads, 0,
                   h->stream>>>(V, ldv, h->n, h->s.ecol);
    LAUNCH_CHECK(h);
  }
  // The staged kernels copy basis slices with 16-byte asynchronous copies,
  // which need 16-byte aligned columns: a caller's basis with an odd leading
  // dimension or an unaligned base goes through the kernel that loads the
  // basis with plain loads (staging mode 0, FP64 products).
  const bool aligned = ((reinterpret_cast<uintptr_t>(V) & 15) == 0 && (ldv & 1) == 0) || j == 0;
  if (aligned && j > 0 && use_spmv && fx_stage(h->stage64, h->dot_fx) == 6) {
    // mode 6 reads the columns as limbs: split the caller's columns once
    k_col_limbs<<<dim3((unsigned)std::max(1, h->grid_stream / std::max(1, j)), (unsigned)j), kThreads, 0,
                  h->stream>>>(V, ldv, h->n, h->s.ecol, h->VL, h->ldv);
    LAUNCH_CHECK(h);
  }
  if (aligned)
    h->step<<<h->P, kThreads, h->smem64, h->stream>>>(h->rowptr, h->col, h->val, V, ldv, u, w, h->n, h->s, j,
                                                       use_spmv, h->s.raw, h->stage64, h->cap64);
  else
    step64_for(h->m, 0)<<<h->P, kThreads, h->step_smem, h->stream>>>(h->rowptr, h->col, h->val, V, ldv, u, w, h->n,
                                                                     h->s, j, use_spmv, h->s.raw, 0, 0);
  LAUNCH_CHECK(h);
  CUDA_TRY(h, cudaMemcpyAsync(X, h->s.raw, sizeof(double) * (2 * j + 2), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return GMRES_OK;
}

gmres_status lsg_maxpy(gmres_handle h, const double* V, int64_t ldv, int K, const double* c, double alpha,
                       const double* y_in, double* y_out) {
  if (!h) return GMRES_ERR_ARG;
  if (K < 0 || K > h->m + 1) return fail(h, GMRES_ERR_ARG, "K must be in [0, m+1]");
  if ((K > 0 && (!V || !c || ldv < h->n)) || !y_in || !y_out) return fail(h, GMRES_ERR_ARG, "bad pointer or ldv");
  std::vector<double> cf(K + 1);
  cf[0] = alpha;
  for (int k = 0; k < K; ++k) cf[1 + k] = c[k];
  CUDA_TRY(h, cudaMemcpyAsync(h->s.coef, cf.data(), sizeof(double) * (K + 1), cudaMemcpyHostToDevice, h->stream));
  k_maxpy<double, double, double><<<h->grid_stream, kThreads, 0, h->stream>>>(V, ldv, y_in, y_out, h->n, h->s,
                                                                               MAXPY_STANDALONE, K);
  LAUNCH_CHECK(h);
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  return GMRES_OK;
}

gmres_status lsg_block_dot_noalloc(const int32_t* rowptr, const int32_t* col, const double* val, int64_t n,
                                   const double* V, int64_t ldv, int j, const double* u, double* w,
                                   int use_spmv, double* X, void* cuda_stream) {
  if (n <= 0 || n >= (int64_t)INT32_MAX) return fail(nullptr, GMRES_ERR_ARG, "n must be in [1, 2^31)");
  if (j < 0 || j > kNoAllocMaxJ)
    return fail(nullptr, GMRES_ERR_ARG,
                "lsg_block_dot_noalloc: j = " + std::to_string(j) + " exceeds the fixed scratch limit of " +
                    std::to_string(kNoAllocMaxJ) + " columns");
  if (!u || !w || !X || (use_spmv && (!rowptr || !col || !val)) || (j > 0 && (!V || ldv < n)))
    return fail(nullptr, GMRES_ERR_ARG, "lsg_block_dot_noalloc: NULL pointer or ldv < n");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices)
    return fail(nullptr, GMRES_ERR_CUDA, "lsg_block_dot_noalloc: no usable current device");
  void* scratch = nullptr;
  int nsm = 0;
  {
    std::lock_guard<std::mutex> lock(g_noalloc_mu);
    if (!g_noalloc_ptr[dev]) {  // first call on this device: look up the array's device address
      cudaError_t e = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
      if (e != cudaSuccess) {
        g_noalloc_ptr[dev] = nullptr;
        return fail(nullptr, GMRES_ERR_CUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
      e = cudaDeviceGetAttribute(&g_noalloc_nsm[dev], cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) {
        g_noalloc_ptr[dev] = nullptr;
        return fail(nullptr, GMRES_ERR_CUDA, std::string("cudaDeviceGetAttribute: ") + cudaGetErrorString(e));
      }
    }
    scratch = g_noalloc_ptr[dev];
    nsm = g_noalloc_nsm[dev];
  }
  cudaStream_t stream = reinterpret_cast<cudaStream_t>(cuda_stream);
  Small sm{};
  sm.st = reinterpret_cast<DevState*>(scratch);
  sm.partials = reinterpret_cast<double*>(static_cast<unsigned char*>(scratch) + kNoAllocStateBytes);
  sm.nvmax = kNoAllocNv;
  const int64_t ntiles = (n + kThreads - 1) / kThreads;
  const int P = (int)std::min<int64_t>(std::min<int64_t>(kNoAllocMaxCtas, 2 * (int64_t)nsm), ntiles);
  // the ticket must start at zero; a memset allocates nothing
  cudaError_t e = cudaMemsetAsync(scratch, 0, sizeof(DevState), stream);
  if (e != cudaSuccess) return fail(nullptr, GMRES_ERR_CUDA, std::string("cudaMemsetAsync: ") + cudaGetErrorString(e));
  step64_for(kNoAllocMaxJ)<<<P, kThreads, 0, stream>>>(rowptr, col, val, V, ldv, u, w, n, sm, j, use_spmv, X, 0, 0);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail(nullptr, GMRES_ERR_CUDA, std::string("launch: ") + cudaGetErrorString(e));
  return GMRES_OK;
}

gmres_status gmres_arnoldi(gmres_handle h, const double* r0, int k, double* V_out, double* H_out, double* T_out,
                           int* k_done) {
  if (!h) return GMRES_ERR_ARG;
  gmres_status st;
  if ((st = check_ptr(h, r0, "r0")) != GMRES_OK) return st;
  if (k < 1 || k > h->m) return fail(h, GMRES_ERR_ARG, "k must be in [1, m]");
  CUDA_TRY(h, cudaSetDevice(h->device));
  std::memset(h->h_st, 0, sizeof(DevState));
  h->h_st->tol = 0.0;
  h->h_st->pipe2 = h->ortho == GMRES_ONE_REDUCE_PIPE2;
  h->h_st->stall_test = h->stall_test;
  if ((st = write_state(h)) != GMRES_OK) return st;
  CUDA_TRY(h, cudaMemsetAsync(h->s.H, 0, sizeof(double) * h->s.ldh * h->m, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->s.T, 0, sizeof(double) * h->s.ldh * h->s.ldh, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->s.ecol, 0, sizeof(unsigned int) * (h->m + 2), h->stream));
  k_residual<<<h->P, kThreads, 0, h->stream>>>(h->rowptr, h->col, h->val, r0, nullptr,
                                               h->prec != GMRES_FP64 ? h->r64 : h->V, h->n, h->s, RES_START, k);
  LAUNCH_CHECK(h);
  // a GMRES-IR cycle starts from r0 / ||r0|| rounded to its basis type, as in gmres_solve
  if (h->prec == GMRES_IR_BF16)
    k_round_scaled<<<h->grid_stream, kThreads, 0, h->stream>>>(h->r64, h->V16, h->n, h->s);
  else if (h->prec == GMRES_IR_FP32)
    k_round_scaled<<<h->grid_stream, kThreads, 0, h->stream>>>(h->r64, h->V32, h->n, h->s);
  LAUNCH_CHECK(h);
  if ((st = launch_cycle(h, k)) != GMRES_OK) return st;
  if ((st = read_state(h)) != GMRES_OK) return st;
  const int kk = h->h_st->k;
  if (h->h_st->stalled) return fail(h, GMRES_ERR_TIMEOUT, "a bounded device-side wait for staged CSR data gave up");
  if (h->h_st->nonfinite) return fail(h, GMRES_ERR_NONFINITE, "non-finite value in the Arnoldi process");
  if (k_done) *k_done = kk;
  if (V_out) {
    if (h->prec == GMRES_IR_BF16)
      k_export_basis<<<h->grid_stream, kThreads, 0, h->stream>>>(h->V16, h->ldv, V_out, h->n, kk, h->s);
    else if (h->prec == GMRES_IR_FP32)
      k_export_basis<<<h->grid_stream, kThreads, 0, h->stream>>>(h->V32, h->ldv, V_out, h->n, kk, h->s);
    else
      k_export_basis<<<h->grid_stream, kThreads, 0, h->stream>>>(h->V, h->ldv, V_out, h->n, kk, h->s);
    LAUNCH_CHECK(h);
  }
  const int ld = h->s.ldh;
  std::vector<double> Hd((size_t)ld * h->m), Td((size_t)ld * ld);
  CUDA_TRY(h, cudaMemcpyAsync(Hd.data(), h->s.H, sizeof(double) * Hd.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaMemcpyAsync(Td.data(), h->s.T, sizeof(double) * Td.size(), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(h, cudaStreamSynchronize(h->stream));
  if (H_out)
    for (int c = 0; c < k; ++c)
      for (int r = 0; r <= k; ++r) H_out[r + (size_t)c * (k + 1)] = (c < kk) ? Hd[r + (size_t)c * ld] : 0.0;
  if (T_out)
    for (int c = 0; c <= k; ++c)
      for (int r = 0; r <= k; ++r)
        T_out[r + (size_t)c * (k + 1)] =
            (h->ortho != GMRES_MGS && r <= kk && c <= kk) ? Td[r + (size_t)c * ld] : 0.0;
  return GMRES_OK;
}

}  // extern "C"
