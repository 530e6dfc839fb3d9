// Batched engine: restarted one-reduce MGS-GMRES(m) (Algorithm 7 on the
// lagged-normalization MGS of Algorithm 4, Sections III-IV of Swirydowicz et
// al., arXiv:1809.05805) on many independent systems at once, FP64 or with
// FP32 cycles inside FP64 restarts (GMRES-IR). It backs the batch API
// (gmres_batch_*: a fixed set of systems solved together) and the serving loop
// (gmres_server_*: systems admitted and retired while others iterate).
//
// Layout. Each system owns a region of a shared row arena (its rows padded to
// whole 512-row tile pairs) in every basis column, in w, b, x (and r for
// GMRES-IR), plus its own CSR (local indices) in a CSR pool; both are
// first-fit allocations. A per-slot descriptor tells the kernels where.
//
// Work split. The host lists the tiles (256 rows) of the systems still
// iterating, system by system; CTA c of a reduction kernel takes the
// contiguous range [c Ta / Pe, (c+1) Ta / Pe) of the Ta listed tiles
// (Pe = min(grid, Ta)). Whenever its range moves to another system it
// publishes that system's partial sums in the system's slot for this CTA and
// takes the system's ticket; the last CTA to arrive for a system sums the
// system's slots in slot order and runs its epilogue (deterministic for a given
// listing and grid). On B300 every cross-lane FP64 reduction is expensive (a
// dependent DADD costs a warp-instruction slot of the SM's small FP64 pipe),
// so the split keeps them to about one per CTA per system touched.
//
// Cycles. A cycle of every iterating system is the fixed launch sequence
// step(0), maxpy(0), ..., maxpy(K-1), step(K) with K the largest step budget
// of the cycle; systems with a smaller budget, or that stopped inside the
// cycle, are skipped by the kernels (state in device memory). On a
// non-default stream each cycle shape is captured once into a CUDA graph and
// replayed. The host acts only at cycle boundaries: residual pass, decisions
// (converged, max_iter, non-finite), admissions and retirements.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "lsgmres.h"
#include "common.cuh"
#include "engine.cuh"

namespace {

template <typename VT>
struct Vec16T;
template <>
struct Vec16T<double> {
  using type = double2;
  static constexpr int E = 2;
};
template <>
struct Vec16T<float> {
  using type = float4;
  static constexpr int E = 4;
};

// The run of one system's tiles that starts at position it of this CTA's range
// [it, hi): its slot and its length.
__device__ __forceinline__ int64_t tile_run(const EngDev& e, int64_t it, int64_t hi, int* sy) {
  const int s = __ldg(e.act_sys + it);
  const int64_t t0 = __ldg(e.act_tiles + it);
  const SysDesc* d = e.desc + s;
  const int64_t tend = (d->row0 + d->n + kThreads - 1) / kThreads;  // one past the system's last tile
  *sy = s;
  return min(hi - it, tend - t0);
}

// Arnoldi MAXPY of step j for every listed system: CTAs < ndata stream the
// runs of one system's tiles in their range (16-byte loads, four basis columns
// in flight, the system's coefficients staged once per run; FP32 cycles
// compute in FP32); CTA ndata + i rotates column j-1 of the i-th listed
// system's Hessenberg matrix and tests convergence while the others stream.
template <typename VT>
__global__ void __launch_bounds__(kThreads, 4)
ke_maxpy(VT* __restrict__ V, int64_t ldv, const VT* __restrict__ w, EngDev e, int j, int ndata) {
  __shared__ VT sc[kMaxM + 3];
  __shared__ int sK, s_on;
  __shared__ const double* s_coef;
  if ((int)blockIdx.x >= ndata) {
    const int i = (int)blockIdx.x - ndata;
    if (i >= *e.n_slots) return;
    const Small sm = e.smalls[__ldg(e.act_slots + i)];
    if (threadIdx.x == 0) s_on = !__ldcg(&sm.st->done) && j >= 1 && j < __ldcg(&sm.st->kmax);
    __syncthreads();
    if (s_on) {
      const double h = __ldcg(&sm.H[(size_t)(j - 1) * sm.ldh + j]);
      const int stop = finish_column(sm, j - 1, h, false);
      if (threadIdx.x == 0) {
        sm.st->grid_syncs += 1;
        if (stop) sm.st->done = 1;
      }
    }
    return;
  }
  int64_t lo, hi;
  if (!cta_tile_range(e, ndata, lo, hi)) return;
  using V16 = typename Vec16T<VT>::type;
  constexpr int E = Vec16T<VT>::E;
  union U {
    V16 v;
    VT e[E];
  };
  const V16* w16 = reinterpret_cast<const V16*>(w);
  V16* out16 = reinterpret_cast<V16*>(V + (size_t)(j + 1) * ldv);
  const V16* V16p = reinterpret_cast<const V16*>(V);
  const int64_t ldv16 = ldv / E;
  for (int64_t it = lo; it < hi;) {
    int sy;
    const int64_t run = tile_run(e, it, hi, &sy);
    const int64_t t0 = __ldg(e.act_tiles + it);
    __syncthreads();  // every warp is done with the previous run's flags and coefficients
    if (threadIdx.x == 0) {
      const Small sm = e.smalls[sy];
      s_on = !__ldcg(&sm.st->done) && j < __ldcg(&sm.st->kmax);
      sK = __ldcg(&sm.st->maxpy_k);
      s_coef = sm.coef;
    }
    __syncthreads();
    it += run;
    if (!s_on) continue;
    const int K = sK;
    for (int i = threadIdx.x; i <= K; i += blockDim.x) sc[i] = (VT)__ldcg(s_coef + i);
    __syncthreads();
    const int64_t q1 = (t0 + run) * (kThreads / E);
    for (int64_t q0 = t0 * (kThreads / E) + threadIdx.x; q0 < q1; q0 += blockDim.x) {
      U y, o;
      y.v = w16[q0];
      VT a[E];
#pragma unroll
      for (int t = 0; t < E; ++t) a[t] = sc[0] * y.e[t];
      int k = 0;
      for (; k + 4 <= K; k += 4) {
        U v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q].v = __ldg(V16p + (size_t)(k + q) * ldv16 + q0);
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int t = 0; t < E; ++t) a[t] = fma(sc[1 + k + q], v[q].e[t], a[t]);
      }
      for (; k < K; ++k) {
        U v;
        v.v = __ldg(V16p + (size_t)k * ldv16 + q0);
#pragma unroll
        for (int t = 0; t < E; ++t) a[t] = fma(sc[1 + k], v.e[t], a[t]);
      }
#pragma unroll
      for (int t = 0; t < E; ++t) o.e[t] = a[t];
      out16[q0] = o.v;
    }
  }
}

// Arnoldi MAXPY of FP64 cycles for every listed system with the column
// products on the integer pipes (the single-system k_maxpy_fx, per run of one
// system's tiles): the system's coefficients become integers C_k on one
// common scale chosen from its basis exponent bounds (Small::ecol), each basis
// value a 58-bit integer relative to its column's bound, read as the limbs the
// step kernel stored (EngDev::VL; rows past a system's end hold limbs of
// whatever the arena held, their outputs are zeroed); per row the sum over
// the columns is exact in 64-bit integers (hi-hi and mid limb products, the
// low-low product dropped) and rounded to FP64 once, then alpha w is added by
// one FMA. Rows of the run past the system's last row (its last tile's
// padding) are stored as zeros. The writers note column j+1's exponent bound.
// CTA ndata + i rotates column j-1 of the i-th listed system, as in ke_maxpy.
__global__ void __launch_bounds__(kThreads, 4)
ke_maxpy_fx(double* __restrict__ V, int64_t ldv, const double* __restrict__ w, EngDev e, int j, int ndata) {
  __shared__ int4 sC[kMaxM + 1];  // (Ch, Cl, 5 + column bound field, 0) per column
  __shared__ uint32_t s_p[kWarps];
  __shared__ int sK, s_on, s_bad;
  __shared__ double s_alpha;
  __shared__ int64_t s_end;
  __shared__ const double* s_coef;
  __shared__ unsigned int* s_ecol;
  if ((int)blockIdx.x >= ndata) {
    const int i = (int)blockIdx.x - ndata;
    if (i >= *e.n_slots) return;
    const Small sm = e.smalls[__ldg(e.act_slots + i)];
    if (threadIdx.x == 0) s_on = !__ldcg(&sm.st->done) && j >= 1 && j < __ldcg(&sm.st->kmax);
    __syncthreads();
    if (s_on) {
      const double h = __ldcg(&sm.H[(size_t)(j - 1) * sm.ldh + j]);
      const int stop = finish_column(sm, j - 1, h, false);
      if (threadIdx.x == 0) {
        sm.st->grid_syncs += 1;
        if (stop) sm.st->done = 1;
      }
    }
    return;
  }
  int64_t lo, hi;
  if (!cta_tile_range(e, ndata, lo, hi)) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  double2* out2 = reinterpret_cast<double2*>(V + (size_t)(j + 1) * ldv);
  const double2* w2 = reinterpret_cast<const double2*>(w);
  for (int64_t it = lo; it < hi;) {
    int sy;
    const int64_t run = tile_run(e, it, hi, &sy);
    const int64_t t0 = __ldg(e.act_tiles + it);
    __syncthreads();  // every warp is done with the previous run's flags and coefficients
    if (threadIdx.x == 0) {
      const Small sm = e.smalls[sy];
      s_on = !__ldcg(&sm.st->done) && j < __ldcg(&sm.st->kmax);
      sK = __ldcg(&sm.st->maxpy_k);
      s_coef = sm.coef;
      s_ecol = sm.ecol;
      s_alpha = __ldcg(sm.coef);
      s_bad = 0;
      s_end = e.desc[sy].row0 + e.desc[sy].n;
    }
    __syncthreads();
    it += run;
    if (!s_on) continue;
    const int K = sK;
    // the coefficients' common scale: P = max_k (field(c_k) + field bound of column k)
    double ck = 0.0;
    int fk = (int)kFxMinField, pk = 0;
    if ((int)threadIdx.x < K) {
      ck = __ldcg(s_coef + 1 + threadIdx.x);
      fk = (int)max(kFxMinField, __ldcg(s_ecol + threadIdx.x) >> 20);
      const int gk = (int)fx_field(ck);
      if (gk == 0x7FF || fk == 0x7FF) s_bad = 1;  // NaN or Inf among the inputs
      pk = (ck != 0.0) ? gk + fk : 0;
    }
    const uint32_t pm = __reduce_max_sync(0xffffffffu, (uint32_t)pk);
    if (lane == 0) s_p[wid] = pm;
    __syncthreads();
    uint32_t q = 0;
#pragma unroll
    for (int v = 0; v < kWarps; ++v) q = max(q, s_p[v]);
    const int P = (int)q;
    // |C| <= 2^cbits and |Xh| <= 2^29: the high sum gathers K products of at most
    // 2^cbits, below 2^63 for K < 2^(63 - cbits)
    const int cbits = K < 64 ? 57 : (K < 128 ? 56 : 55);
    if ((int)threadIdx.x < K) {
      long long C = 0;
      if (ck != 0.0 && P > 0) C = __double2ll_rn(scalbn(ck, cbits + 1022 - P + fk));  // |C| < 2^cbits
      sC[threadIdx.x] = make_int4((int)(C >> 29), (int)(C & 0x1FFFFFFFll), 5 + fk, 0);
    }
    __syncthreads();
    const bool bad = s_bad != 0;
    const double alpha = s_alpha;
    const int e2 = P - 2044 - cbits;  // sum = (hh + mid / 2^29) 2^(P - 2044 - cbits)
    const int64_t end = s_end;
    uint32_t emax = 0;
    // two rows per thread (16-byte loads): arena rows are even-aligned and ldv is a multiple of 512
    const int64_t q1 = (t0 + run) * (kThreads / 2);
    for (int64_t i = t0 * (kThreads / 2) + threadIdx.x; i < q1; i += blockDim.x) {
      long long hh0 = 0, md0 = 0, hh1 = 0, md1 = 0;
      for (int k = 0; k < K; k += 8) {
        int4 x[8];  // the stored limbs of rows 2i, 2i + 1 of columns k .. k + 7
#pragma unroll
        for (int u2 = 0; u2 < 8; ++u2)
          x[u2] = (k + u2 < K) ? __ldg(reinterpret_cast<const int4*>(e.VL + (size_t)(k + u2) * ldv) + i)
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
      const double2 wv = __ldg(w2 + i);
      double2 o;
      o.x = fma(alpha, wv.x, fx_to_double(hh0 + (md0 >> 29), e2));
      o.y = fma(alpha, wv.y, fx_to_double(hh1 + (md1 >> 29), e2));
      if (bad) o.x = o.y = __longlong_as_double(0x7ff8000000000000ll);
      if (2 * i >= end) o.x = 0.0;
      if (2 * i + 1 >= end) o.y = 0.0;
      out2[i] = o;
      emax = max(emax, max(fx_hi_field(o.x), fx_hi_field(o.y)));
    }
    fx_note_max(s_ecol, j + 1, emax);
  }
}

// Cycle start of every listed system: r = b - A x over its rows (FP64, local
// CSR), written to out (basis column 0 for FP64 cycles, the FP64 residual
// vector for FP32 cycles), with the sums of r^2 and b^2; the CTA completing a
// system finishes ||r|| (and ||b|| on the system's first pass) and resets the
// cycle state.
__global__ void __launch_bounds__(kThreads, 2)
ke_residual(const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ out, EngDev e) {
  __shared__ double sbuf[kWarps];
  __shared__ double red[2];
  __shared__ int s_on;
  __shared__ SysDesc s_d;
  int64_t lo, hi;
  if (!cta_tile_range(e, (int)gridDim.x, lo, hi)) return;
  int cur = -1;
  double rr = 0.0, bb = 0.0;
  uint32_t emax = 0;  // exponent bound of basis column 0 (FP64 cycles; Small::ecol is null otherwise)
  for (int64_t it = lo; it <= hi; ++it) {
    const int64_t t = (it < hi) ? __ldg(e.act_tiles + it) : -1;
    const int snext = (it < hi) ? __ldg(e.act_sys + it) : -1;
    if (snext != cur) {  // CTA-uniform
      if (cur >= 0 && s_on) {
        fx_note_max(e.smalls[cur].ecol, 0, emax);
        const double trr = block_sum(rr, sbuf);
        const double tbb = block_sum(bb, sbuf);
        if (threadIdx.x == 0) {
          red[0] = trr;
          red[1] = tbb;
        }
        __syncthreads();
        if (sys_publish(e, cur, red, 2) && threadIdx.x == 0) {
          const Small sm = e.smalls[cur];
          DevState* st = sm.st;
          st->reductions += 1;
          if (st->fresh) {
            residual_finish(sm, red[1], RES_BNORM, 0);
            st->fresh = 0;
          }
          residual_finish(sm, red[0], RES_RESIDUAL, 0);
        }
      }
      if (snext < 0) break;
      cur = snext;
      rr = bb = 0.0;
      emax = 0;
      __syncthreads();
      if (threadIdx.x == 0) {
        s_on = __ldcg(&e.smalls[cur].st->kmax) >= 0;  // a retired system is left untouched
        s_d = e.desc[cur];
      }
      __syncthreads();
    }
    if (!s_on) continue;
    const int64_t row = t * kThreads + threadIdx.x;
    if (row < s_d.row0 + s_d.n) {
      const double bv = b[row];
      const double v = bv - csr_row(s_d.rowptr - s_d.row0, s_d.col, s_d.val, x + s_d.row0, row);
      out[row] = v;
      emax = max(emax, fx_hi_field(v));
      rr = fma(v, v, rr);
      bb = fma(bv, bv, bb);
    }
  }
}

// Start of an FP32 cycle for every listed system: basis column 0 = r / ||r||
// rounded to FP32 (normalized in FP64 first); the cycle's estimates and its
// correction are scaled back by ||r||.
__global__ void __launch_bounds__(kThreads, 4)
ke_round_scaled(const double* __restrict__ r, float* __restrict__ out, EngDev e) {
  int64_t lo, hi;
  if (!cta_tile_range(e, (int)gridDim.x, lo, hi)) return;
  for (int64_t it = lo; it < hi;) {
    int sy;
    const int64_t run = tile_run(e, it, hi, &sy);
    const int64_t t0 = __ldg(e.act_tiles + it);
    it += run;
    const Small sm = e.smalls[sy];
    if (__ldcg(&sm.st->kmax) <= 0) continue;
    const double rn = __ldcg(&sm.st->rnorm);
    const double ir = 1.0 / rn;
    for (int64_t row = t0 * kThreads + threadIdx.x; row < (t0 + run) * kThreads; row += blockDim.x)
      out[row] = (float)(r[row] * ir);
    if (t0 * kThreads == e.desc[sy].row0 && threadIdx.x == 0) sm.st->cycle_scale = rn;  // the system's first tile
  }
}

// Back substitution and cycle totals, one CTA per listed system in this cycle.
__global__ void ke_lsq(EngDev e) {
  if ((int)blockIdx.x >= *e.n_slots) return;
  const Small sm = e.smalls[__ldg(e.act_slots + blockIdx.x)];
  if (__ldcg(&sm.st->kmax) <= 0) return;
  lsq_system(sm);
}

// x += V_k y for every listed system (FP64 accumulation; an FP32 basis is
// widened exactly).
template <typename VT>
__global__ void __launch_bounds__(kThreads, 4)
ke_xupdate(const VT* __restrict__ V, int64_t ldv, double* __restrict__ x, EngDev e) {
  __shared__ double sc[kMaxM + 3];
  __shared__ int sK;
  __shared__ const double* s_coef;
  int64_t lo, hi;
  if (!cta_tile_range(e, (int)gridDim.x, lo, hi)) return;
  for (int64_t it = lo; it < hi;) {
    int sy;
    const int64_t run = tile_run(e, it, hi, &sy);
    const int64_t t0 = __ldg(e.act_tiles + it);
    it += run;
    __syncthreads();
    if (threadIdx.x == 0) {
      const Small sm = e.smalls[sy];
      sK = (__ldcg(&sm.st->kmax) > 0) ? __ldcg(&sm.st->k) : 0;
      s_coef = sm.coefx;
    }
    __syncthreads();
    const int K = sK;
    if (K <= 0) continue;
    for (int i = threadIdx.x; i <= K; i += blockDim.x) sc[i] = __ldcg(s_coef + i);
    __syncthreads();
    for (int64_t row = t0 * kThreads + threadIdx.x; row < (t0 + run) * kThreads; row += blockDim.x) {
      double a = sc[0] * x[row];
      for (int k = 0; k < K; ++k) a = fma(sc[1 + k], (double)__ldg(V + (size_t)k * ldv + row), a);
      x[row] = a;
    }
  }
}

__global__ void ke_fill_i32(int32_t* __restrict__ a, int64_t n, int32_t v) {
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) a[i] = v;
}

__global__ void ke_to_float(const double* __restrict__ a, float* __restrict__ out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (float)a[i];
}

// Engine step kernels (instantiated in engine_step_f64.cu and engine_step_f32.cu).
template <typename VT>
EngStepKernel<VT> eng_step_for(int m, bool pairs, int fx);
template <>
EngStepKernel<double> eng_step_for<double>(int m, bool pairs, int fx) {
  return reinterpret_cast<EngStepKernel<double>>(const_cast<void*>(lsg_engine::eng_step_f64(m, pairs, fx)));
}
template <>
EngStepKernel<float> eng_step_for<float>(int m, bool pairs, int fx) {
  return reinterpret_cast<EngStepKernel<float>>(const_cast<void*>(lsg_engine::eng_step_f32(m, pairs, fx)));
}

// ==========================================================================
// host side
// ==========================================================================

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


// First-fit allocator of unit ranges [0, cap) (free ranges kept merged).
class RangeAlloc {
 public:
  void reset(int64_t cap) {
    free_.clear();
    cap_ = cap;
    used_ = 0;
    if (cap > 0) free_[0] = cap;
  }
  int64_t alloc(int64_t len) {  // start, or -1
    for (auto it = free_.begin(); it != free_.end(); ++it)
      if (it->second >= len) {
        const int64_t s = it->first, l = it->second;
        free_.erase(it);
        if (l > len) free_[s + len] = l - len;
        used_ += len;
        return s;
      }
    return -1;
  }
  void release(int64_t s, int64_t len) {
    used_ -= len;
    auto nx = free_.lower_bound(s);
    if (nx != free_.end() && s + len == nx->first) {
      len += nx->second;
      nx = free_.erase(nx);
    }
    if (nx != free_.begin()) {
      auto pv = std::prev(nx);
      if (pv->first + pv->second == s) {
        pv->second += len;
        return;
      }
    }
    free_[s] = len;
  }
  int64_t used() const { return used_; }
  int64_t cap() const { return cap_; }
  int64_t largest() const {
    int64_t b = 0;
    for (auto& f : free_) b = std::max(b, f.second);
    return b;
  }

 private:
  std::map<int64_t, int64_t> free_;
  int64_t cap_ = 0, used_ = 0;
};

struct EngineConfig {
  int m = 30;
  int prec = GMRES_FP64;    // GMRES_FP64 or GMRES_IR_FP32
  int64_t rows = 0;         // arena capacity in rows
  int64_t csr_bytes = 0;    // CSR pool capacity
  int max_systems = 1;
  int max_iter_cap = 1;     // longest per-system step budget (sizes the histories)
};

// One batched solver instance (one precision, one stream).
struct Engine {
  EngineConfig cfg;
  std::string err;
  int device = 0, nsm = 0, P = 0, nvmax = 0, hist_cap = 0;
  bool pairs = true;
  bool fx = true;  // FP64 tile pairs: block dot and MAXPY products on the integer pipes
  // the step kernel with the column ring over the epilogue's shared memory
  // (FP64: fixed-point products; FP32: FMA products): its CSR staging
  // capacity and dynamic shared memory, and whether the listed systems' tile
  // pairs fit that capacity
  int ring_cap = 0;
  size_t ring_smem = 0;
  bool ring_ok = false;
  bool no_ring = false;  // gmres_batch_set_block_dot(-1): fixed point with direct basis loads
  int64_t R = 0, ldv = 0;
  size_t vb = 8;
  // arena
  void* V = nullptr;
  int2* VL = nullptr;  // FP64 cycles: the basis as fixed-point limbs (EngDev::VL)
  void* w = nullptr;
  double* bv = nullptr;
  double* xv = nullptr;
  double* r64 = nullptr;  // FP32 cycles: FP64 residual
  char* csr_pool = nullptr;
  // per slot
  SysDesc* d_desc = nullptr;
  Small* d_smalls = nullptr;
  DevState* d_states = nullptr;
  char* d_blk = nullptr;
  unsigned int* d_tickets = nullptr;
  unsigned int* d_ecol = nullptr;  // FP64 cycles: basis exponent bounds, m + 2 per slot
  // listing
  int32_t* d_tiles = nullptr;  // act_tiles (R / 256) | act_sys (R / 256)
  int32_t* d_act = nullptr;    // act_slots (S) | sys_b0 (S) | sys_nslot (S) | sys_slot0 (S) | n_slots | bounds (act_len - 4 S - 1)
  int64_t* d_nact = nullptr;
  double* d_partials = nullptr;
  int64_t tile_cap = 0, slot_cap = 0;
  size_t act_len = 0;  // entries of d_act / h_act
  // pinned host mirrors
  DevState* h_states = nullptr;
  int32_t* h_tiles = nullptr;
  int32_t* h_act = nullptr;
  int64_t* h_nact = nullptr;
  SysDesc* h_desc = nullptr;
  std::vector<Small> smalls;
  size_t small_stride = 0;
  // allocators and slots
  RangeAlloc rows, csr;
  struct Slot {
    bool used = false, listed = false;
    int64_t n = 0, nnz = 0, row0 = 0, npairs = 0, csr_off = 0, csr_units = 0;
    double tol = 0.0, bnorm = 0.0;
    int max_iter = 0, status = GMRES_OK, it_prev = -1;
    bool finished = true;
  };
  std::vector<Slot> slot;
  std::vector<int> free_slots;
  std::vector<int> listed;  // slots in the current device listing
  bool listing_dirty = true;
  // launch
  cudaStream_t stream = nullptr;
  size_t step_smem = 0, lsq_smem = 0;
  int stage_cap = 0;  // entries of the step kernel's CSR staging buffer
  struct G {
    int kmax;
    bool prof;
    int fxm;  // the step kernel's fixed-point mode when captured
    cudaGraphExec_t exec;
    std::vector<cudaEvent_t> events;
    std::vector<int> rec_cls, rec_j;
  };
  std::vector<G> graphs;
  G* cap = nullptr;
  int64_t launches = 0;
  // profiling
  struct Rec {
    int cls, j;
    cudaEvent_t a, b;
    double bytes, flops;
    int64_t tiles;
  };
  bool prof_on = false;
  std::vector<Rec> pending;
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double prof_ms[GMRES_PROFILE_CLASSES] = {}, prof_bytes[GMRES_PROFILE_CLASSES] = {},
         prof_flops[GMRES_PROFILE_CLASSES] = {};
  int64_t prof_cnt[GMRES_PROFILE_CLASSES] = {};
  struct LogEntry {
    int cls, j;
    int64_t tiles;
    float ms;
    double flops;
  };
  std::vector<LogEntry> log;
  std::vector<int> cyc_kmax, cyc_it0;

  ~Engine() { release(); }

  gmres_status fail(gmres_status st, const std::string& m) {
    err = m;
    return st;
  }

#define ETRY(call)                                                                           \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return fail(e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA,          \
                  std::string(#call) + ": " + cudaGetErrorString(e_));                       \
  } while (0)

  bool ir() const { return cfg.prec == GMRES_IR_FP32; }

  // Device bytes per arena row: the basis (m + 1 columns) and w, b and x;
  // FP32 cycles add the FP64 residual, FP64 cycles the basis limbs.
  static size_t row_bytes(const EngineConfig& c) {
    const size_t vbytes = c.prec == GMRES_IR_FP32 ? 4 : 8;
    return vbytes * (c.m + 2) + 16 + (c.prec == GMRES_IR_FP32 ? 8 : 8 * (size_t)(c.m + 1));
  }
  // Device bytes the engine holds for `rows` arena rows and `csr_bytes` of CSR.
  static size_t footprint(const EngineConfig& c) { return row_bytes(c) * (size_t)c.rows + (size_t)c.csr_bytes; }

  gmres_status init(const EngineConfig& c) {
    cfg = c;
    if (cfg.m < 1 || cfg.m > kMaxM) return fail(GMRES_ERR_ARG, "m_restart must be in [1, 128]");
    ETRY(cudaGetDevice(&device));
    ETRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device));
    vb = ir() ? 4 : 8;
    R = std::max<int64_t>(kPairRows, (cfg.rows + kPairRows - 1) / kPairRows * kPairRows);
    ldv = R;
    const int m = cfg.m, ld = m + 1, S = std::max(1, cfg.max_systems);
    ETRY(cudaMalloc(&V, vb * (size_t)R * (m + 1)));
    if (!ir()) {  // rows no system has written read as zero limbs
      ETRY(cudaMalloc(&VL, sizeof(int2) * (size_t)R * (m + 1)));
      ETRY(cudaMemset(VL, 0, sizeof(int2) * (size_t)R * (m + 1)));
    }
    ETRY(cudaMalloc(&w, vb * (size_t)R));
    ETRY(cudaMalloc(&bv, 8 * (size_t)R));
    ETRY(cudaMalloc(&xv, 8 * (size_t)R));
    if (ir()) ETRY(cudaMalloc(&r64, 8 * (size_t)R));
    const int64_t csr_units = std::max<int64_t>(1, (cfg.csr_bytes + 255) / 256);
    ETRY(cudaMalloc(&csr_pool, 256 * (size_t)csr_units));
    rows.reset(R / kPairRows);
    csr.reset(csr_units);
    // listing: every arena tile at most once; a reduction grid of P CTAs
    // touches at most P + S - 1 (CTA, system) pairs
    tile_cap = R / kThreads;
    slot_cap = (int64_t)kMaxGridPerSm * nsm + S + 1;
    nvmax = 2 * (m + 1) + 2;
    ETRY(cudaMalloc(&d_tiles, sizeof(int32_t) * 2 * (size_t)tile_cap));
    act_len = 4 * (size_t)S + 1 + (size_t)kMaxGridPerSm * nsm + 2;
    ETRY(cudaMalloc(&d_act, sizeof(int32_t) * act_len));
    ETRY(cudaMalloc(&d_nact, sizeof(int64_t)));
    ETRY(cudaMalloc(&d_partials, sizeof(double) * (size_t)slot_cap * nvmax));
    ETRY(cudaMallocHost(&h_tiles, sizeof(int32_t) * 2 * (size_t)tile_cap));
    ETRY(cudaMallocHost(&h_act, sizeof(int32_t) * act_len));
    ETRY(cudaMallocHost(&h_nact, sizeof(int64_t)));
    *h_nact = 0;
    ETRY(cudaMalloc(&d_tickets, sizeof(unsigned int) * S));
    ETRY(cudaMemset(d_tickets, 0, sizeof(unsigned int) * S));
    ETRY(cudaMalloc(&d_desc, sizeof(SysDesc) * S));
    ETRY(cudaMallocHost(&h_desc, sizeof(SysDesc) * S));
    std::memset(h_desc, 0, sizeof(SysDesc) * S);
    // per-slot dense state
    hist_cap = cfg.max_iter_cap + m + 1;
    size_t off = 0;
    auto take = [&](size_t bytes) {
      size_t o = off;
      off = align_up(off + bytes, 256);
      return o;
    };
    const size_t oH = take(sizeof(double) * ld * m), oR = take(sizeof(double) * ld * m),
                 ocs = take(sizeof(double) * (m + 1)), osn = take(sizeof(double) * (m + 1)),
                 og = take(sizeof(double) * (m + 2)), oT = take(sizeof(double) * ld * ld),
                 osc = take(sizeof(double) * (m + 2)), ocf = take(sizeof(double) * (m + 3)),
                 ocx = take(sizeof(double) * (m + 3)), ohi = take(sizeof(double) * hist_cap);
    small_stride = off;
    ETRY(cudaMalloc(&d_blk, off * S));
    ETRY(cudaMemset(d_blk, 0, off * S));
    ETRY(cudaMalloc(&d_states, sizeof(DevState) * S));
    ETRY(cudaMemset(d_states, 0, sizeof(DevState) * S));
    if (!ir()) {
      ETRY(cudaMalloc(&d_ecol, sizeof(unsigned int) * (size_t)(m + 2) * S));
      ETRY(cudaMemset(d_ecol, 0, sizeof(unsigned int) * (size_t)(m + 2) * S));
    }
    ETRY(cudaMallocHost(&h_states, sizeof(DevState) * S));
    std::memset(h_states, 0, sizeof(DevState) * S);
    smalls.resize(S);
    for (int i = 0; i < S; ++i) {
      char* base = d_blk + off * i;
      Small& sm = smalls[i];
      sm.st = d_states + i;
      sm.H = reinterpret_cast<double*>(base + oH);
      sm.Rg = reinterpret_cast<double*>(base + oR);
      sm.cs = reinterpret_cast<double*>(base + ocs);
      sm.sn = reinterpret_cast<double*>(base + osn);
      sm.g = reinterpret_cast<double*>(base + og);
      sm.T = reinterpret_cast<double*>(base + oT);
      sm.scale = reinterpret_cast<double*>(base + osc);
      sm.coef = reinterpret_cast<double*>(base + ocf);
      sm.coefx = reinterpret_cast<double*>(base + ocx);
      sm.hist = reinterpret_cast<double*>(base + ohi);
      sm.ecol = d_ecol ? d_ecol + (size_t)(m + 2) * i : nullptr;
      sm.partials = nullptr;
      sm.raw = nullptr;
      sm.m = m;
      sm.ldh = ld;
      sm.nvmax = nvmax;
      sm.hist_cap = hist_cap;
    }
    ETRY(cudaMalloc(&d_smalls, sizeof(Small) * S));
    ETRY(cudaMemcpy(d_smalls, smalls.data(), sizeof(Small) * S, cudaMemcpyHostToDevice));
    slot.assign(S, Slot());
    free_slots.clear();
    for (int i = S - 1; i >= 0; --i) free_slots.push_back(i);
    cyc_kmax.assign(S, -1);
    cyc_it0.assign(S, 0);
    lsq_smem = sizeof(double) * (size_t)ld * m;
    // The step kernel's dynamic shared memory: the CSR staging buffer (rowptr
    // slice of a tile pair, then stage_cap indices and values) followed by the
    // epilogue's T and scales. stage_cap is the largest multiple of 256 entries
    // (at most 16,384) that keeps the kernel's resident CTAs per SM.
    {
      const size_t vb = ir() ? sizeof(float) : sizeof(double);
      const size_t epi = sizeof(double) * ((size_t)ld * ld + ld);
      const int per_sm = ir() ? 3 : 2;
      stage_cap = 0;
      for (int cap = 16384; cap >= 256 && stage_cap == 0; cap -= 256) {
        const size_t need = (size_t)(2 * kThreads + 4) * 4 + (size_t)cap * (4 + vb) + epi;
        bool ok = true;
        for (int v = 0; v < 3; ++v) {  // one row per thread, tile pairs, tile pairs with fixed-point products
          const bool pr = v > 0;
          const int fv = v == 2 ? 1 : 0;
          const void* f = ir() ? reinterpret_cast<const void*>(eng_step_for<float>(m, pr, fv))
                               : reinterpret_cast<const void*>(eng_step_for<double>(m, pr, fv));
          int nb = 0;
          if (raise_smem_limit(f, need) != cudaSuccess ||
              cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, need) != cudaSuccess || nb < per_sm)
            ok = false;
        }
        if (ok) {
          stage_cap = cap;
          step_smem = need;
        }
      }
      // the ring variant: the ring shares the epilogue's region (it is live only inside a unit's block dot)
      {
        const void* f = ir() ? reinterpret_cast<const void*>(eng_step_for<float>(m, true, 3))
                             : reinterpret_cast<const void*>(eng_step_for<double>(m, true, 2));
        const size_t ring = ir() ? pf_ring_bytes<float>() : kEngRingBytes;
        for (int cap = 16384; cap >= 256 && ring_cap == 0; cap -= 256) {
          const size_t need = (size_t)(2 * kThreads + 4) * 4 + (size_t)cap * (4 + vb) + std::max(epi, ring);
          int nb = 0;
          if (raise_smem_limit(f, need) == cudaSuccess &&
              cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, f, kThreads, need) == cudaSuccess && nb >= per_sm) {
            ring_cap = cap;
            ring_smem = need;
          }
        }
      }
      (void)cudaGetLastError();  // sizes above the per-block limit were refused; that is not an error here
      if (stage_cap == 0) return fail(GMRES_ERR_CUDA, "no shared-memory size keeps the step kernel resident");
    }
    ETRY(raise_smem_limit(reinterpret_cast<const void*>(ke_lsq), lsq_smem));
    P = (ir() ? 3 : 2) * nsm;  // resident CTAs per SM of the step kernel
    pairs = true;
    return GMRES_OK;
  }

  void release() {
    drop_graphs();
    for (void* p : {V, (void*)VL, w, (void*)bv, (void*)xv, (void*)r64, (void*)csr_pool, (void*)d_desc, (void*)d_smalls,
                    (void*)d_states, (void*)d_blk, (void*)d_tickets, (void*)d_ecol, (void*)d_tiles, (void*)d_act,
                    (void*)d_nact, (void*)d_partials})
      if (p) cudaFree(p);
    for (void* p : {(void*)h_states, (void*)h_tiles, (void*)h_act, (void*)h_nact, (void*)h_desc})
      if (p) cudaFreeHost(p);
    for (cudaEvent_t e : ev_pool) cudaEventDestroy(e);
    ev_pool.clear();
    V = w = nullptr;
    bv = xv = r64 = nullptr;
    csr_pool = nullptr;
    d_desc = nullptr;
    d_smalls = nullptr;
    d_states = nullptr;
    d_blk = nullptr;
    d_tickets = nullptr;
    d_ecol = nullptr;
    d_tiles = d_act = nullptr;
    d_nact = nullptr;
    d_partials = nullptr;
    h_states = nullptr;
    h_tiles = h_act = nullptr;
    h_nact = nullptr;
    h_desc = nullptr;
  }

  void drop_graphs() {
    for (auto& g : graphs) {
      cudaGraphExecDestroy(g.exec);
      for (cudaEvent_t e : g.events) cudaEventDestroy(e);
    }
    graphs.clear();
  }

  EngDev dev() const {
    EngDev d{};
    const int S = (int)slot.size();
    d.desc = d_desc;
    d.smalls = d_smalls;
    d.act_tiles = d_tiles;
    d.act_sys = d_tiles + tile_cap;
    d.n_act = d_nact;
    d.act_slots = d_act;
    d.sys_b0 = d_act + S;
    d.sys_nslot = d_act + 2 * S;
    d.sys_slot0 = d_act + 3 * S;
    d.n_slots = d_act + 4 * S;
    d.bounds = d_act + 4 * S + 1;
    d.nb = P;
    d.partials = d_partials;
    d.tickets = d_tickets;
    d.nvmax = nvmax;
    d.VL = VL;
    return d;
  }

  int stream_grid() const { return 4 * nsm; }
  // rowptr entries kept per system: padded with nnz to whole tile pairs + 8,
  // so that every staged rowptr slice of the step kernel is in bounds
  static int64_t rp_entries(int64_t n) { return (n + kPairRows - 1) / kPairRows * kPairRows + 8; }
  int64_t csr_bytes_for(int64_t n, int64_t nnz) const {
    return (int64_t)align_up(4 * (size_t)rp_entries(n), 256) + (int64_t)align_up(4 * (size_t)std::max<int64_t>(nnz, 1), 256) +
           (int64_t)align_up(8 * (size_t)std::max<int64_t>(nnz, 1), 256) +
           (ir() ? (int64_t)align_up(4 * (size_t)std::max<int64_t>(nnz, 1), 256) : 0);
  }
  bool fits_ever(int64_t n, int64_t nnz) const {
    return (n + kPairRows - 1) / kPairRows <= rows.cap() && (csr_bytes_for(n, nnz) + 255) / 256 <= csr.cap();
  }
  bool fits_now(int64_t n, int64_t nnz) const {
    return !free_slots.empty() && (n + kPairRows - 1) / kPairRows <= rows.largest() &&
           (csr_bytes_for(n, nnz) + 255) / 256 <= csr.largest();
  }

  // Place a system (host or device CSR, validated by the caller) into a free
  // slot: arena rows, CSR pool space, descriptor. Returns the slot or -1 (no
  // room now). Copies are queued on the engine's stream.
  int add(const gmres_csr& a) {
    if (!fits_now(a.n, a.nnz)) return -1;
    const int s = free_slots.back();
    const int64_t np = (a.n + kPairRows - 1) / kPairRows;
    const int64_t units = (csr_bytes_for(a.n, a.nnz) + 255) / 256;
    const int64_t r0 = rows.alloc(np);
    const int64_t c0 = csr.alloc(units);
    if (r0 < 0 || c0 < 0) {
      if (r0 >= 0) rows.release(r0, np);
      if (c0 >= 0) csr.release(c0, units);
      return -1;
    }
    free_slots.pop_back();
    Slot& sl = slot[s];
    sl = Slot();
    sl.used = true;
    sl.n = a.n;
    sl.nnz = a.nnz;
    sl.row0 = r0 * kPairRows;
    sl.npairs = np;
    sl.csr_off = c0;
    sl.csr_units = units;
    char* base = csr_pool + 256 * (size_t)c0;
    const size_t o_col = align_up(4 * (size_t)rp_entries(a.n), 256);
    const size_t o_val = o_col + align_up(4 * (size_t)std::max<int64_t>(a.nnz, 1), 256);
    const size_t o_v32 = o_val + align_up(8 * (size_t)std::max<int64_t>(a.nnz, 1), 256);
    SysDesc& d = h_desc[s];
    d.rowptr = reinterpret_cast<const int32_t*>(base);
    d.col = reinterpret_cast<const int32_t*>(base + o_col);
    d.val = reinterpret_cast<const double*>(base + o_val);
    d.val32 = ir() ? reinterpret_cast<const float*>(base + o_v32) : nullptr;
    d.row0 = sl.row0;
    d.n = a.n;
    const cudaMemcpyKind k = cudaMemcpyDefault;
    cudaMemcpyAsync((void*)d.rowptr, a.rowptr, 4 * (size_t)(a.n + 1), k, stream);
    ke_fill_i32<<<1, kThreads, 0, stream>>>(const_cast<int32_t*>(d.rowptr) + a.n + 1, rp_entries(a.n) - (a.n + 1),
                                           (int32_t)a.nnz);
    if (a.nnz > 0) {
      cudaMemcpyAsync((void*)d.col, a.col, 4 * (size_t)a.nnz, k, stream);
      cudaMemcpyAsync((void*)d.val, a.val, 8 * (size_t)a.nnz, k, stream);
      if (ir()) ke_to_float<<<64, kThreads, 0, stream>>>(d.val, const_cast<float*>(d.val32), a.nnz);
    }
    cudaMemcpyAsync(d_desc + s, &h_desc[s], sizeof(SysDesc), cudaMemcpyHostToDevice, stream);
    return s;
  }

  void remove(int s) {
    Slot& sl = slot[s];
    if (!sl.used) return;
    rows.release(sl.row0 / kPairRows, sl.npairs);
    csr.release(sl.csr_off, sl.csr_units);
    sl = Slot();
    free_slots.push_back(s);
    listing_dirty = true;
  }

  // Start a solve of slot s: b and x0 (device or host pointers; x0 may be
  // NULL for zero) are copied into the arena; the state is reset.
  gmres_status activate(int s, const double* b, const double* x0, double tol, int max_iter) {
    Slot& sl = slot[s];
    ETRY(cudaMemcpyAsync(bv + sl.row0, b, 8 * (size_t)sl.n, cudaMemcpyDefault, stream));
    if (x0)
      ETRY(cudaMemcpyAsync(xv + sl.row0, x0, 8 * (size_t)sl.n, cudaMemcpyDefault, stream));
    else
      ETRY(cudaMemsetAsync(xv + sl.row0, 0, 8 * (size_t)sl.n, stream));
    sl.tol = tol;
    sl.max_iter = std::min(max_iter, cfg.max_iter_cap);
    sl.status = GMRES_OK;
    sl.finished = false;
    sl.it_prev = -1;
    sl.bnorm = 0.0;
    DevState& hs = h_states[s];
    std::memset(&hs, 0, sizeof(DevState));
    hs.tol = tol;
    hs.fresh = 1;
    ETRY(cudaMemcpyAsync(d_states + s, &hs, sizeof(DevState), cudaMemcpyHostToDevice, stream));
    listing_dirty = true;
    return GMRES_OK;
  }

  // Slots being solved (not finished), in slot order.
  void active_slots(std::vector<int>& out) const {
    out.clear();
    for (int i = 0; i < (int)slot.size(); ++i)
      if (slot[i].used && !slot[i].finished) out.push_back(i);
  }

  // Device listing of the slots in `ls`: their tiles (system by system), and
  // per slot the first CTA of the reduction grid (P CTAs, CTA c taking
  // [c Ta / Pe, (c+1) Ta / Pe), Pe = min(P, Ta)) whose range touches it, the
  // number of such CTAs and its first partial-sum slot. Staging is pinned; the
  // caller has synchronized the stream since the staging was last used.
  gmres_status write_listing(const std::vector<int>& ls) {
    const int S = (int)slot.size();
    int32_t* at = h_tiles;
    int32_t* as = h_tiles + tile_cap;
    int32_t* act = h_act;
    int32_t* b0 = h_act + S;
    int32_t* ns = h_act + 2 * S;
    int32_t* s0 = h_act + 3 * S;
    int64_t Ta = 0;
    for (int k = 0; k < (int)ls.size(); ++k) {
      const int s = ls[k];
      const Slot& sl = slot[s];
      const int64_t ft = sl.row0 / kThreads, ntile = (sl.n + kThreads - 1) / kThreads;
      act[k] = s;
      for (int64_t q = 0; q < ntile; ++q) {
        at[Ta] = (int32_t)(ft + q);
        as[Ta] = s;
        ++Ta;
      }
      b0[s] = INT32_MAX;
      ns[s] = 0;
    }
    const int Pe = (int)std::min<int64_t>(P, Ta);
    // The reduction grid's ranges, balanced by estimated cost: a tile costs 1,
    // and a system costs kSysCost more (its switch, publish and, in the CTA
    // that completes it, its epilogue: measured at 3-4 tiles' time), charged
    // at its first tile. Boundary c goes where the cumulative cost first
    // reaches c / Pe of the total, moved one tile on so that it does not split
    // a tile pair where it can, and kept strictly increasing (every range
    // non-empty).
    int32_t* bnd = h_act + 4 * S + 1;
    {
      constexpr double kSysCost = 3.5;
      std::vector<double> cum((size_t)Ta + 1, 0.0);
      for (int64_t i = 0; i < Ta; ++i)
        cum[i + 1] = cum[i] + 1.0 + ((i == 0 || as[i] != as[i - 1]) ? kSysCost : 0.0);
      bnd[0] = Pe;
      bnd[1] = 0;
      int64_t prev = 0;
      for (int c = 1; c < Pe; ++c) {
        const double target = cum[Ta] * c / Pe;
        int64_t b = std::lower_bound(cum.begin(), cum.end(), target) - cum.begin();
        // odd tile with its pair partner just before it in the same system: cut after it instead
        if (b < Ta && b > 0 && (at[b] & 1) && as[b - 1] == as[b]) ++b;
        b = std::max<int64_t>(b, prev + 1);
        b = std::min<int64_t>(b, Ta - (Pe - c));
        bnd[1 + c] = (int32_t)b;
        prev = b;
      }
      bnd[1 + Pe] = (int32_t)Ta;
    }
    std::vector<int32_t> b1(S, -1);
    for (int c = 0; c < Pe; ++c) {
      const int64_t lo = bnd[1 + c], hi = bnd[2 + c];
      for (int64_t it = lo; it < hi; ++it) {
        const int s = as[it];
        b0[s] = std::min(b0[s], c);
        b1[s] = std::max(b1[s], c);
      }
    }
    int64_t tot = 0;
    for (int s : ls) {
      ns[s] = b1[s] - b0[s] + 1;
      s0[s] = (int32_t)tot;
      tot += ns[s];
    }
    if (tot > slot_cap) return fail(GMRES_ERR_ARG, "internal: slot capacity");
    // the ring variant keeps the tile pairs' CSR staged when a pair's entries
    // (estimated from each system's mean row length, with 5% and the copies'
    // 16-byte rounding to spare) fit its smaller staging capacity
    bool fits = ring_cap > 0;
    for (int s : ls) {
      const Slot& sl = slot[s];
      const double per_pair = (double)kPairRows * (double)sl.nnz / (double)std::max<int64_t>(sl.n, 1);
      if (per_pair * 1.05 + 16.0 > (double)ring_cap) fits = false;
    }
    ring_ok = fits;
    act[4 * S] = (int32_t)ls.size();  // n_slots
    *h_nact = Ta;
    if (Ta > 0) {
      ETRY(cudaMemcpyAsync(d_tiles, at, sizeof(int32_t) * Ta, cudaMemcpyHostToDevice, stream));
      ETRY(cudaMemcpyAsync(d_tiles + tile_cap, as, sizeof(int32_t) * Ta, cudaMemcpyHostToDevice, stream));
    }
    ETRY(cudaMemcpyAsync(d_act, h_act, sizeof(int32_t) * (4 * (size_t)S + 2 + (size_t)Pe + 1), cudaMemcpyHostToDevice,
                         stream));
    ETRY(cudaMemcpyAsync(d_nact, h_nact, sizeof(int64_t), cudaMemcpyHostToDevice, stream));
    listed = ls;
    listing_dirty = false;
    return GMRES_OK;
  }

  // ---- profiling
  int prof_begin(int cls, int j, double bytes = -1.0, double flops = -1.0) {
    if (!prof_on) return -1;
    if (cap) {
      const size_t u = 2 * cap->rec_cls.size();
      if (u + 2 > cap->events.size()) return -1;
      cudaEventRecordWithFlags(cap->events[u], stream, cudaEventRecordExternal);
      cap->rec_cls.push_back(cls);
      cap->rec_j.push_back(j);
      return 1;
    }
    while (ev_used + 2 > ev_pool.size()) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return -1;
      ev_pool.push_back(e);
    }
    Rec r{cls, j, ev_pool[ev_used], ev_pool[ev_used + 1], bytes, flops, *h_nact};
    ev_used += 2;
    cudaEventRecord(r.a, stream);
    pending.push_back(r);
    return 0;
  }
  void prof_end(int tok) {
    if (tok < 0) return;
    if (tok == 1)
      cudaEventRecordWithFlags(cap->events[2 * cap->rec_cls.size() - 1], stream, cudaEventRecordExternal);
    else
      cudaEventRecord(pending.back().b, stream);
  }
  void prof_reset() {
    pending.clear();
    ev_used = 0;
    log.clear();
    for (int c = 0; c < GMRES_PROFILE_CLASSES; ++c) {
      prof_ms[c] = prof_bytes[c] = prof_flops[c] = 0.0;
      prof_cnt[c] = 0;
    }
  }
  // Algorithmic bytes / flops of a launch, summed over the systems it did work
  // for (per-system model of the single-system solver; a cycle of k columns
  // ran steps 0..k).
  void alg_model(const Rec& r, const std::vector<int>& kcol, double* bytes, double* flops) const {
    double by = 0.0, fl = 0.0;
    const double v = (double)vb;
    for (size_t i = 0; i < slot.size(); ++i) {
      const int km = cyc_kmax[i], k = kcol[i];
      if (km < 0) continue;
      const double n = (double)slot[i].n, nnz = (double)slot[i].nnz;
      const double csrb = 4.0 * (n + 1) + (4.0 + v) * nnz;
      const int j = r.j;
      if (r.cls == PC_STEP && j <= k) {
        if (j == km) {
          by += v * n * (j + 1);
          fl += 2.0 * n * (j + 1);
        } else {
          by += csrb + v * n * (j + 2);
          fl += 2.0 * nnz + 2.0 * n * (2.0 * j + 2.0);
        }
      } else if (r.cls == PC_MAXPY && j <= k && j < km) {
        by += v * n * (j + 3);
        fl += 2.0 * n * (j + 1) + n;
      } else if (r.cls == PC_XUPD) {
        by += 16.0 * n + v * n * k;
        fl += 2.0 * n * k + n;
      }
    }
    *bytes = by;
    *flops = fl;
  }
  void prof_settle() {
    if (!prof_on) return;
    std::vector<int> kcol(slot.size(), 0);
    for (size_t i = 0; i < slot.size(); ++i)
      if (cyc_kmax[i] >= 0) kcol[i] = h_states[i].total_iters - cyc_it0[i];
    for (const auto& r : pending) {
      float ms = 0.f;
      cudaEventElapsedTime(&ms, r.a, r.b);
      double by = r.bytes, fl = r.flops;
      if (by < 0.0) alg_model(r, kcol, &by, &fl);
      const int c = (by > 0.0 || r.cls == PC_LSQ) ? r.cls : PC_NOOP;
      prof_ms[c] += ms;
      prof_cnt[c] += 1;
      prof_bytes[c] += by;
      prof_flops[c] += fl;
      log.push_back({c, r.j, r.tiles, ms, fl});
    }
    pending.clear();
    ev_used = 0;
    std::fill(cyc_kmax.begin(), cyc_kmax.end(), -1);
  }

  // ---- launches
  gmres_status launch_cycle(int KM) {
    const EngDev d = dev();
    const int fxm = fx_mode();
    const int nd = stream_grid();
    const int S = (int)slot.size();
    for (int j = 0; j <= KM; ++j) {
      int pr = prof_begin(PC_STEP, j);
      if (ir())
        eng_step_for<float>(cfg.m, pairs, fxm)<<<P, kThreads, fxm == 3 ? ring_smem : step_smem, stream>>>(
            static_cast<const float*>(V), ldv, static_cast<float*>(w), d, j, fxm == 3 ? ring_cap : stage_cap);
      else
        eng_step_for<double>(cfg.m, pairs, fxm)<<<P, kThreads, fxm == 2 ? ring_smem : step_smem, stream>>>(
            static_cast<const double*>(V), ldv, static_cast<double*>(w), d, j, fxm == 2 ? ring_cap : stage_cap);
      prof_end(pr);
      if (j < KM) {
        pr = prof_begin(PC_MAXPY, j);
        if (ir())
          ke_maxpy<float><<<nd + S, kThreads, 0, stream>>>(static_cast<float*>(V), ldv, static_cast<const float*>(w),
                                                           d, j, nd);
        else if (fx_active())
          ke_maxpy_fx<<<nd + S, kThreads, 0, stream>>>(static_cast<double*>(V), ldv, static_cast<const double*>(w), d,
                                                       j, nd);
        else
          ke_maxpy<double><<<nd + S, kThreads, 0, stream>>>(static_cast<double*>(V), ldv,
                                                            static_cast<const double*>(w), d, j, nd);
        prof_end(pr);
      }
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GMRES_ERR_CUDA, std::string("cycle launch: ") + cudaGetErrorString(e));
    return GMRES_OK;
  }

  gmres_status run_cycle(int KM) {
    launches += 2 * (int64_t)KM + 1;
    if (stream == nullptr) return launch_cycle(KM);
    G* hit = nullptr;
    for (auto& g : graphs)
      if (g.kmax == KM && g.prof == prof_on && g.fxm == fx_mode()) hit = &g;
    if (!hit) {
      G g{KM, prof_on, fx_mode(), nullptr, {}, {}, {}};
      if (prof_on) {
        g.events.resize(2 * (2 * (size_t)KM + 1));
        for (auto& ev : g.events) ETRY(cudaEventCreate(&ev));
      }
      graphs.push_back(std::move(g));
      hit = &graphs.back();
      cudaGraph_t graph = nullptr;
      ETRY(cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal));
      cap = hit;
      gmres_status st = launch_cycle(KM);
      cap = nullptr;
      cudaError_t e = cudaStreamEndCapture(stream, &graph);
      if (st == GMRES_OK && e == cudaSuccess) e = cudaGraphInstantiate(&hit->exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (st != GMRES_OK || e != cudaSuccess || !hit->exec) {
        for (cudaEvent_t ev : hit->events) cudaEventDestroy(ev);
        graphs.pop_back();
        return fail(GMRES_ERR_CUDA, std::string("cycle graph: ") + cudaGetErrorString(e));
      }
    }
    ETRY(cudaGraphLaunch(hit->exec, stream));
    if (prof_on)
      for (size_t r = 0; r < hit->rec_cls.size(); ++r)
        pending.push_back({hit->rec_cls[r], hit->rec_j[r], hit->events[2 * r], hit->events[2 * r + 1], -1.0, -1.0,
                           *h_nact});
    return GMRES_OK;
  }

  // One cycle boundary for every active slot: (re)list, residual pass, and
  // the decisions (synchronizes the stream). Slots whose solve ended are
  // marked finished (their x is final in the arena) and returned in `ended`;
  // the others, with their step budgets set, in `go`.
  gmres_status residual_decide(std::vector<int>& ended, std::vector<int>& go) {
    ended.clear();
    go.clear();
    std::vector<int> act;
    active_slots(act);
    if (act.empty()) return GMRES_OK;
    gmres_status st;
    if (listing_dirty || act != listed) {
      ETRY(cudaStreamSynchronize(stream));  // the staging may still feed a queued copy
      if ((st = write_listing(act)) != GMRES_OK) return st;
    }
    const EngDev d = dev();
    double rby = 0.0, rfl = 0.0;
    for (int s : act) {
      const double n = (double)slot[s].n, nnz = (double)slot[s].nnz;
      rby += 4.0 * (n + 1) + 12.0 * nnz + 24.0 * n;
      rfl += 2.0 * nnz + 5.0 * n;
    }
    if (d_ecol)  // the new cycle's basis bounds start from column 0, noted by the residual pass
      ETRY(cudaMemsetAsync(d_ecol, 0, sizeof(unsigned int) * (size_t)(cfg.m + 2) * slot.size(), stream));
    int pr = prof_begin(PC_RES, 1, rby, rfl);
    ke_residual<<<P, kThreads, 0, stream>>>(bv, xv, ir() ? r64 : static_cast<double*>(V), d);
    prof_end(pr);
    ++launches;
    ETRY(cudaGetLastError());
    ETRY(cudaMemcpyAsync(h_states, d_states, sizeof(DevState) * slot.size(), cudaMemcpyDeviceToHost, stream));
    ETRY(cudaStreamSynchronize(stream));
    prof_settle();
    for (int s : act) {
      Slot& sl = slot[s];
      DevState& hs = h_states[s];
      bool end = true;
      if (sl.it_prev < 0) sl.bnorm = hs.bnorm;
      if (!std::isfinite(sl.bnorm)) {
        sl.status = GMRES_ERR_NONFINITE;
      } else if (sl.bnorm == 0.0) {
        ETRY(cudaMemsetAsync(xv + sl.row0, 0, 8 * (size_t)sl.n, stream));
        hs.rnorm = 0.0;
        sl.status = GMRES_OK;
      } else if (sl.it_prev >= 0 && hs.total_iters == sl.it_prev) {  // every cycle completes >= 1 column
        sl.status = GMRES_ERR_CUDA;
      } else if (!std::isfinite(hs.rnorm) || hs.nonfinite) {
        sl.status = GMRES_ERR_NONFINITE;
      } else if (hs.rnorm / sl.bnorm <= sl.tol) {
        sl.status = GMRES_OK;
      } else if (hs.total_iters >= sl.max_iter) {
        sl.status = GMRES_MAXITER;
      } else {
        end = false;
      }
      if (end) {
        sl.finished = true;
        hs.done = 1;
        hs.kmax = -1;
        ended.push_back(s);
      } else {
        hs.kmax = std::min(cfg.m, sl.max_iter - hs.total_iters);
        sl.it_prev = hs.total_iters;
        cyc_kmax[s] = hs.kmax;
        cyc_it0[s] = hs.total_iters;
        go.push_back(s);
      }
    }
    // the stream is idle and h_states mirrors the device: write back the
    // host's decisions (kmax, done) in one copy
    ETRY(cudaMemcpyAsync(d_states, h_states, sizeof(DevState) * slot.size(), cudaMemcpyHostToDevice, stream));
    return GMRES_OK;
  }

  // Queue the cycle of the slots in `go` (as returned by residual_decide, the
  // stream not used since): listing, FP32 start vector, the cycle's steps,
  // least squares and solution update. Not synchronized.
  gmres_status launch_next(const std::vector<int>& go) {
    if (go.empty()) return GMRES_OK;
    gmres_status st;
    int KM = 0;
    for (int s : go) KM = std::max(KM, h_states[s].kmax);
    if (go != listed && (st = write_listing(go)) != GMRES_OK) return st;
    const EngDev d2 = dev();
    const int ng = stream_grid();
    if (ir()) {
      ke_round_scaled<<<ng, kThreads, 0, stream>>>(r64, static_cast<float*>(V), d2);
      ++launches;
    }
    if ((st = run_cycle(KM)) != GMRES_OK) return st;
    int pr = prof_begin(PC_LSQ, 0, 0.0, 0.0);
    ke_lsq<<<(int)slot.size(), 128, lsq_smem, stream>>>(d2);
    prof_end(pr);
    pr = prof_begin(PC_XUPD, 0);
    if (ir())
      ke_xupdate<float><<<ng, kThreads, 0, stream>>>(static_cast<const float*>(V), ldv, xv, d2);
    else
      ke_xupdate<double><<<ng, kThreads, 0, stream>>>(static_cast<const double*>(V), ldv, xv, d2);
    prof_end(pr);
    launches += 2;
    ETRY(cudaGetLastError());
    return GMRES_OK;
  }

  // Result of a finished slot.
  void info_of(int s, gmres_info* in) const {
    const Slot& sl = slot[s];
    const DevState& hs = h_states[s];
    std::memset(in, 0, sizeof(*in));
    in->iters = hs.total_iters;
    in->restarts = hs.restarts;
    in->status = sl.status;
    in->breakdowns = hs.breakdowns;
    in->rel_resid_true = sl.bnorm > 0.0 ? hs.rnorm / sl.bnorm : 0.0;
    in->rel_resid_est = hs.est;
    in->reductions = hs.reductions;
    in->grid_syncs = hs.grid_syncs;
    in->kernel_launches = launches;
  }

  gmres_status history(int s, std::vector<double>& out) {
    const int len = std::min(h_states[s].total_iters, hist_cap);
    out.resize(len);
    if (len > 0) ETRY(cudaMemcpy(out.data(), smalls[s].hist, sizeof(double) * len, cudaMemcpyDeviceToHost));
    return GMRES_OK;
  }

  // Time one mid-cycle step of every slot in use (zeroed basis, all systems
  // active) for grids of 1, 2 and 3 CTAs per SM with one and two rows per
  // thread; keep the fastest.
  gmres_status autotune() {
    std::vector<int> all;
    for (int i = 0; i < (int)slot.size(); ++i)
      if (slot[i].used) all.push_back(i);
    if (all.empty()) return GMRES_OK;
    gmres_status st;
    ETRY(cudaStreamSynchronize(stream));
    ETRY(cudaMemsetAsync(V, 0, vb * (size_t)R * (cfg.m + 1), stream));
    ETRY(cudaMemsetAsync(w, 0, vb * (size_t)R, stream));
    if ((st = write_listing(all)) != GMRES_OK) return st;
    const int j = std::max(1, cfg.m / 2);
    cudaEvent_t e0, e1;
    ETRY(cudaEventCreate(&e0));
    ETRY(cudaEventCreate(&e1));
    float best = 1e30f;
    int bestP = (ir() ? 3 : 2) * nsm;
    bool bestPairs = true;
    const bool pairs0 = pairs;
    st = GMRES_OK;
    for (int pr = 0; pr < 2 && st == GMRES_OK; ++pr)
      for (int k = 1; k <= 3 && st == GMRES_OK; ++k) {
        const int Pc = k * nsm;
        P = Pc;
        ETRY(cudaStreamSynchronize(stream));
        if ((st = write_listing(all)) != GMRES_OK) break;
        float tb = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
          for (int s : all) {
            DevState& hs = h_states[s];
            std::memset(&hs, 0, sizeof(DevState));
            hs.kmax = cfg.m;
            hs.bnorm = hs.inv_bnorm = hs.cycle_scale = 1.0;
          }
          cudaError_t e = cudaMemcpyAsync(d_states, h_states, sizeof(DevState) * slot.size(), cudaMemcpyHostToDevice,
                                          stream);
          if (e == cudaSuccess) e = cudaEventRecord(e0, stream);
          if (e == cudaSuccess) {
            if (ir()) {
              pairs = pr == 1;
              const int fxm = fx_mode();
              eng_step_for<float>(cfg.m, pairs, fxm)<<<Pc, kThreads, fxm == 3 ? ring_smem : step_smem, stream>>>(
                  static_cast<const float*>(V), ldv, static_cast<float*>(w), dev(), j,
                  fxm == 3 ? ring_cap : stage_cap);
            } else {
              pairs = pr == 1;  // fx_mode() follows the shape being timed
              const int fxm = fx_mode();
              eng_step_for<double>(cfg.m, pairs, fxm)<<<Pc, kThreads, fxm == 2 ? ring_smem : step_smem, stream>>>(
                  static_cast<const double*>(V), ldv, static_cast<double*>(w), dev(), j,
                  fxm == 2 ? ring_cap : stage_cap);
            }
            e = cudaGetLastError();
          }
          if (e == cudaSuccess) e = cudaEventRecord(e1, stream);
          if (e == cudaSuccess) e = cudaEventSynchronize(e1);
          float ms = 0.f;
          if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
          if (e != cudaSuccess) {
            st = fail(GMRES_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            break;
          }
          if (rep > 0) tb = std::min(tb, ms);
        }
        if (st == GMRES_OK && tb < best) {
          best = tb;
          bestP = Pc;
          bestPairs = pr == 1;
        }
      }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    for (int s : all) std::memset(&h_states[s], 0, sizeof(DevState));
    cudaMemcpy(d_states, h_states, sizeof(DevState) * slot.size(), cudaMemcpyHostToDevice);
    if (st != GMRES_OK) {
      pairs = pairs0;
      return st;
    }
    set_shape(bestP, bestPairs);
    return GMRES_OK;
  }

  // FP64 tile pairs with fixed-point block-dot and MAXPY products
  bool fx_active() const { return fx && pairs && !ir(); }
  // the step kernel's fixed-point mode: 0 none, 1 direct basis loads, 2 the column ring
  // (FP32 cycles: 3 with the column ring, else 0)
  int fx_mode() const {
    if (ir()) return (pairs && ring_ok && !no_ring) ? 3 : 0;
    return !fx_active() ? 0 : (ring_ok && !no_ring) ? 2 : 1;
  }

  void set_shape(int ctas, bool pr) {
    P = ctas;
    pairs = pr;
    listing_dirty = true;  // the reduction slots depend on the grid
    drop_graphs();
  }
};

std::string validate_csr(const gmres_csr& a, int i) {
  const std::string who = "matrix " + std::to_string(i) + ": ";
  if (a.on_device || !a.rowptr || a.n <= 0 || a.nnz < 0 || (a.nnz > 0 && (!a.col || !a.val)))
    return who + "need host CSR arrays with n > 0";
  if (a.n >= (int64_t)INT32_MAX || a.nnz >= (int64_t)INT32_MAX) return who + "too large for 32-bit indices";
  if (a.rowptr[0] != 0 || a.rowptr[a.n] != a.nnz) return who + "rowptr[0] must be 0 and rowptr[n] = nnz";
  for (int64_t r = 0; r < a.n; ++r)
    if (a.rowptr[r + 1] < a.rowptr[r]) return who + "rowptr is not nondecreasing";
  for (int64_t p = 0; p < a.nnz; ++p)
    if (a.col[p] < 0 || a.col[p] >= a.n || !std::isfinite(a.val[p]))
      return who + "column out of range or non-finite value";
  return "";
}

}  // namespace

// ==========================================================================
// batch API
// ==========================================================================
struct gmres_batch_ctx {
  Engine eng;
  int S = 0, max_iter = 0;
  double tol = 0.0;
  std::vector<int> slots;  // system i -> engine slot
  std::vector<std::vector<double>> hist;
  std::string err;
};

namespace {

thread_local std::string g_batch_err;  // handle-less errors, one string per host thread

gmres_status bfail(gmres_batch_ctx* b, gmres_status st, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_batch_err = msg;
  return st;
}

gmres_status beng(gmres_batch_ctx* b, gmres_status st) {
  if (st != GMRES_OK) b->err = b->eng.err;
  return st;
}

gmres_status batch_solve(gmres_batch b, const double* const* bv, double* const* xv, gmres_info* info) {
  if (!bv || !xv) return bfail(b, GMRES_ERR_ARG, "b or x array is NULL");
  for (int i = 0; i < b->S; ++i)
    if (!bv[i] || !xv[i] || (reinterpret_cast<uintptr_t>(bv[i]) & 7) || (reinterpret_cast<uintptr_t>(xv[i]) & 7))
      return bfail(b, GMRES_ERR_ARG, "b[" + std::to_string(i) + "] or x[" + std::to_string(i) +
                                         "] is NULL or not 8-byte aligned");
  Engine& e = b->eng;
  if (cudaSetDevice(e.device) != cudaSuccess) return bfail(b, GMRES_ERR_CUDA, "cudaSetDevice failed");
  const auto t0 = std::chrono::steady_clock::now();
  e.launches = 0;
  e.prof_reset();
  std::fill(e.cyc_kmax.begin(), e.cyc_kmax.end(), -1);
  gmres_status st;
  for (int i = 0; i < b->S; ++i)
    if ((st = beng(b, e.activate(b->slots[i], bv[i], xv[i], b->tol, b->max_iter))) != GMRES_OK) return st;
  std::vector<int> ended, go;
  do {
    if ((st = beng(b, e.residual_decide(ended, go))) != GMRES_OK) return st;
    if ((st = beng(b, e.launch_next(go))) != GMRES_OK) return st;
  } while (!go.empty());
  for (int i = 0; i < b->S; ++i) {
    const Engine::Slot& sl = e.slot[b->slots[i]];
    if (cudaMemcpyAsync(xv[i], e.xv + sl.row0, 8 * (size_t)sl.n, cudaMemcpyDefault, e.stream) != cudaSuccess)
      return bfail(b, GMRES_ERR_CUDA, "copy of x failed");
  }
  if (cudaStreamSynchronize(e.stream) != cudaSuccess) return bfail(b, GMRES_ERR_CUDA, "stream synchronize failed");
  const auto t1 = std::chrono::steady_clock::now();
  gmres_status result = GMRES_OK;
  for (int i = 0; i < b->S; ++i) {
    const int s = b->slots[i];
    if ((st = beng(b, e.history(s, b->hist[i]))) != GMRES_OK) return st;
    const int si = e.slot[s].status;
    if (si < 0 && result >= 0) result = (gmres_status)si;
    if (si == GMRES_MAXITER && result == GMRES_OK) result = GMRES_MAXITER;
    if (info) {
      e.info_of(s, &info[i]);
      info[i].seconds = std::chrono::duration<double>(t1 - t0).count();
    }
  }
  if (result < 0) b->err = "a system reported status " + std::to_string((int)result) + " (see its info entry)";
  return result;
}

}  // namespace

extern "C" {

gmres_status gmres_batch_destroy(gmres_batch b) {
  if (!b) return GMRES_OK;
  delete b;
  return GMRES_OK;
}

const char* gmres_batch_last_error(gmres_batch b) { return b ? b->err.c_str() : g_batch_err.c_str(); }

gmres_status gmres_batch_create(const gmres_csr* A, int count, int m_restart, double tol, int max_iter,
                                gmres_batch* out) {
  if (!out) return bfail(nullptr, GMRES_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!A || count < 1) return bfail(nullptr, GMRES_ERR_ARG, "need count >= 1 matrices");
  if (m_restart < 1 || m_restart > kMaxM) return bfail(nullptr, GMRES_ERR_ARG, "m_restart must be in [1, 128]");
  if (!(tol >= 0.0) || max_iter < 0) return bfail(nullptr, GMRES_ERR_ARG, "tol must be >= 0 and max_iter >= 0");
  EngineConfig c;
  c.m = m_restart;
  c.prec = GMRES_FP64;
  c.max_systems = count;
  c.max_iter_cap = max_iter;
  for (int i = 0; i < count; ++i) {
    const std::string v = validate_csr(A[i], i);
    if (!v.empty()) return bfail(nullptr, GMRES_ERR_ARG, v);
    c.rows += (A[i].n + kPairRows - 1) / kPairRows * kPairRows;
  }
  gmres_batch_ctx* b = new gmres_batch_ctx();
  b->S = count;
  b->tol = tol;
  b->max_iter = max_iter;
  // CSR pool: exactly what the systems need
  for (int i = 0; i < count; ++i) c.csr_bytes += Engine::rp_entries(A[i].n) * 4 + A[i].nnz * 12 + 3 * 256 + 256;
  if (b->eng.init(c) != GMRES_OK) {
    g_batch_err = b->eng.err;
    const gmres_status st = b->eng.err.find("cudaErrorMemoryAllocation") != std::string::npos ||
                                    b->eng.err.find("out of memory") != std::string::npos
                                ? GMRES_ERR_OOM
                                : GMRES_ERR_CUDA;
    delete b;
    return st;
  }
  for (int i = 0; i < count; ++i) {
    const int s = b->eng.add(A[i]);
    if (s < 0) {
      g_batch_err = "internal: batch arena too small";
      delete b;
      return GMRES_ERR_CUDA;
    }
    b->slots.push_back(s);
  }
  if (cudaStreamSynchronize(nullptr) != cudaSuccess || b->eng.autotune() != GMRES_OK) {
    g_batch_err = "batch setup: " + b->eng.err;
    delete b;
    return GMRES_ERR_CUDA;
  }
  b->hist.assign(count, std::vector<double>());
  *out = b;
  return GMRES_OK;
}

gmres_status gmres_batch_set_grid(gmres_batch b, int ctas) {
  if (!b) return GMRES_ERR_ARG;
  Engine& e = b->eng;
  if (ctas == 0) return beng(b, e.autotune());
  const int mx = kMaxGridPerSm * e.nsm;
  if (ctas < 0 || ctas > mx) return bfail(b, GMRES_ERR_ARG, "ctas must be in [0, " + std::to_string(mx) + "]");
  e.set_shape(ctas, e.pairs);
  return GMRES_OK;
}

gmres_status gmres_batch_get_grid(gmres_batch b, int* ctas) {
  if (!b || !ctas) return GMRES_ERR_ARG;
  *ctas = b->eng.P;
  return GMRES_OK;
}

gmres_status gmres_batch_set_rows_per_thread(gmres_batch b, int rows) {
  if (!b) return GMRES_ERR_ARG;
  if (rows != 1 && rows != 2) return bfail(b, GMRES_ERR_ARG, "rows per thread must be 1 or 2");
  b->eng.set_shape(b->eng.P, rows == 2);
  return GMRES_OK;
}

gmres_status gmres_batch_set_block_dot(gmres_batch b, int fixed_point, int* active) {
  if (!b) return GMRES_ERR_ARG;
  b->eng.fx = fixed_point != 0;
  b->eng.no_ring = fixed_point < 0;
  b->eng.drop_graphs();
  if (active) *active = b->eng.fx_mode();
  return GMRES_OK;
}

gmres_status gmres_batch_get_rows_per_thread(gmres_batch b, int* rows) {
  if (!b || !rows) return GMRES_ERR_ARG;
  *rows = b->eng.pairs ? 2 : 1;
  return GMRES_OK;
}

gmres_status gmres_batch_set_stream(gmres_batch b, void* stream) {
  if (!b) return GMRES_ERR_ARG;
  b->eng.stream = reinterpret_cast<cudaStream_t>(stream);
  b->eng.drop_graphs();
  return GMRES_OK;
}

gmres_status gmres_batch_solve(gmres_batch b, const double* const* bv, double* const* xv, gmres_info* info) {
  if (!b) return GMRES_ERR_ARG;
  return batch_solve(b, bv, xv, info);
}

gmres_status gmres_batch_solve_host(gmres_batch b, const double* const* bv, double* const* xv, gmres_info* info) {
  if (!b) return GMRES_ERR_ARG;
  return batch_solve(b, bv, xv, info);
}

gmres_status gmres_batch_set_profile(gmres_batch b, int on) {
  if (!b) return GMRES_ERR_ARG;
  b->eng.prof_on = on != 0;
  return GMRES_OK;
}

gmres_status gmres_batch_profile(gmres_batch b, int cls, double* total_ms, int64_t* launches, double* alg_bytes,
                                 double* alg_flops) {
  if (!b) return GMRES_ERR_ARG;
  if (cls < 0 || cls >= GMRES_PROFILE_CLASSES) return bfail(b, GMRES_ERR_ARG, "profile class out of range");
  const Engine& e = b->eng;
  if (total_ms) *total_ms = e.prof_ms[cls];
  if (launches) *launches = e.prof_cnt[cls];
  if (alg_bytes) *alg_bytes = e.prof_bytes[cls];
  if (alg_flops) *alg_flops = e.prof_flops[cls];
  return GMRES_OK;
}

gmres_status gmres_batch_launch_log(gmres_batch b, int cap, int* cls, int* step, int64_t* active_tiles, float* ms,
                                    double* alg_flops, int* count) {
  if (!b || cap < 0) return GMRES_ERR_ARG;
  const auto& log = b->eng.log;
  if (count) *count = (int)log.size();
  const int k = std::min<int>(cap, (int)log.size());
  for (int i = 0; i < k; ++i) {
    if (cls) cls[i] = log[i].cls;
    if (step) step[i] = log[i].j;
    if (active_tiles) active_tiles[i] = log[i].tiles;
    if (ms) ms[i] = log[i].ms;
    if (alg_flops) alg_flops[i] = log[i].flops;
  }
  return GMRES_OK;
}

gmres_status gmres_batch_history(gmres_batch b, int i, double* buf, int cap, int* len) {
  if (!b || i < 0 || i >= b->S) return GMRES_ERR_ARG;
  const auto& h = b->hist[i];
  if (len) *len = (int)h.size();
  if (buf && cap > 0) std::memcpy(buf, h.data(), sizeof(double) * std::min<size_t>(cap, h.size()));
  return GMRES_OK;
}

}  // extern "C"

// ==========================================================================
// serving loop
// ==========================================================================
// Two engines (FP64 cycles, FP32 cycles inside FP64 restarts), each with its
// own stream and worker thread, so their launches overlap on the device. A
// worker repeats: residual pass and decisions for its iterating requests;
// copy the finished ones' solutions out and complete them; queue the next
// cycle; then, while that cycle runs, admit queued requests (first come,
// first served) as long as its arena rows, CSR pool and slots allow: they join
// at the next cycle boundary. The device footprint of each engine is fixed at
// create from the byte budget, so admission never allocates.
namespace {

struct Request {
  int64_t id = 0;
  gmres_csr A{};
  const double* b = nullptr;
  const double* x0 = nullptr;
  double* x_out = nullptr;
  double tol = 0.0;
  int prec = GMRES_FP64;
  int max_iter = 0;
  int slot = -1;
  bool done = false;
  gmres_info info{};
  std::chrono::steady_clock::time_point t_submit, t_admit, t_done;
};

struct Worker {
  Engine eng;
  std::thread th;
  std::deque<Request*> queue;
  std::vector<Request*> running;  // by slot
  int64_t admitted = 0, completed = 0, cycles = 0, peak_rows = 0, peak_csr_units = 0, peak_running = 0;
  double busy_s = 0.0;
};

}  // namespace

struct gmres_server_ctx {
  gmres_server_config cfg{};
  Worker w[2];  // 0: FP64, 1: GMRES-IR FP32
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  int64_t next_id = 1, submitted = 0, rejected = 0;
  std::map<int64_t, std::unique_ptr<Request>> reqs;
  std::vector<double> latencies;  // seconds, completion order
  std::string err, worker_err;
  int device = 0;
  std::chrono::steady_clock::time_point t0;
};

namespace {

thread_local std::string g_server_err;  // handle-less errors, one string per host thread

gmres_status sfail(gmres_server_ctx* sv, gmres_status st, const std::string& m) {
  if (sv)
    sv->err = m;
  else
    g_server_err = m;
  return st;
}

// Admit queued requests of worker k, first come first served, while the head
// fits (called by the worker with the lock released; only the worker touches
// its engine). The full CSR check runs here, off the submitting thread.
void admit(gmres_server_ctx* sv, int k) {
  Worker& W = sv->w[k];
  Engine& e = W.eng;
  for (;;) {
    Request* r;
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      if (W.queue.empty()) break;
      r = W.queue.front();
      if (!e.fits_now(r->A.n, r->A.nnz)) break;  // wait for room
      W.queue.pop_front();
    }
    const std::string bad = validate_csr(r->A, 0);
    int s = -1;
    gmres_status st = GMRES_ERR_ARG;
    if (bad.empty()) {
      s = e.add(r->A);
      st = s < 0 ? GMRES_ERR_CUDA : e.activate(s, r->b, r->x0, r->tol, r->max_iter);
    }
    std::lock_guard<std::mutex> lk(sv->mu);
    if (st != GMRES_OK) {
      if (s >= 0) e.remove(s);
      if (!bad.empty()) sv->err = bad;
      r->info.status = st;
      r->done = true;
      r->t_done = std::chrono::steady_clock::now();
      sv->cv_done.notify_all();
      continue;
    }
    r->slot = s;
    r->t_admit = std::chrono::steady_clock::now();
    W.running[s] = r;
    ++W.admitted;
    W.peak_rows = std::max(W.peak_rows, e.rows.used());
    W.peak_csr_units = std::max(W.peak_csr_units, e.csr.used());
    int64_t nrun = 0;
    for (Request* q : W.running) nrun += q != nullptr;
    W.peak_running = std::max(W.peak_running, nrun);
  }
}

void worker_loop(gmres_server_ctx* sv, int k) {
  Worker& W = sv->w[k];
  Engine& e = W.eng;
  cudaSetDevice(sv->device);
  std::vector<int> ended, go;
  for (;;) {
    admit(sv, k);
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      bool any = false;
      for (Request* q : W.running) any |= q != nullptr;
      if (!any) {
        if (sv->stop) return;
        sv->cv_work.wait(lk, [&] { return sv->stop || !W.queue.empty(); });
        continue;
      }
    }
    const auto tb = std::chrono::steady_clock::now();
    gmres_status st = e.residual_decide(ended, go);
    // solutions of the finished requests go out before the next cycle is queued
    for (int s : ended) {
      Request* r = W.running[s];
      cudaMemcpyAsync(r->x_out, e.xv + e.slot[s].row0, 8 * (size_t)e.slot[s].n, cudaMemcpyDefault, e.stream);
    }
    if (!ended.empty()) cudaStreamSynchronize(e.stream);
    const auto td = std::chrono::steady_clock::now();
    if (st == GMRES_OK) st = e.launch_next(go);
    {
      std::lock_guard<std::mutex> lk(sv->mu);
      for (int s : ended) {
        Request* r = W.running[s];
        e.info_of(s, &r->info);
        r->t_done = td;
        r->info.seconds = std::chrono::duration<double>(td - r->t_submit).count();
        r->done = true;
        sv->latencies.push_back(r->info.seconds);
        W.running[s] = nullptr;
        e.remove(s);
        ++W.completed;
      }
      if (!go.empty()) ++W.cycles;
      if (st != GMRES_OK) {  // a CUDA failure ends every request of this engine
        sv->worker_err = e.err;
        for (Request*& q : W.running)
          if (q) {
            q->info.status = st;
            q->done = true;
            e.remove(q->slot);
            q = nullptr;
          }
      }
      W.busy_s += std::chrono::duration<double>(std::chrono::steady_clock::now() - tb).count();
    }
    sv->cv_done.notify_all();
    // the loop's next admit() runs while the queued cycle executes (its copies
    // are ordered after the cycle on the engine's stream)
  }
}

}  // namespace

extern "C" {

const char* gmres_server_last_error(gmres_server sv) { return sv ? sv->err.c_str() : g_server_err.c_str(); }

gmres_status gmres_server_destroy(gmres_server sv) {
  if (!sv) return GMRES_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    for (Worker& W : sv->w) W.queue.clear();
  }
  sv->cv_work.notify_all();
  for (Worker& W : sv->w)
    if (W.th.joinable()) W.th.join();
  for (Worker& W : sv->w)
    if (W.eng.stream) cudaStreamDestroy(W.eng.stream);
  delete sv;
  return GMRES_OK;
}

gmres_status gmres_server_create(const gmres_server_config* cfg, gmres_server* out) {
  if (!out) return sfail(nullptr, GMRES_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return sfail(nullptr, GMRES_ERR_ARG, "cfg is NULL");
  if (cfg->m_restart < 1 || cfg->m_restart > kMaxM) return sfail(nullptr, GMRES_ERR_ARG, "m_restart must be in [1, 128]");
  if (cfg->max_iter < 1 || cfg->max_requests < 1 || cfg->hbm_budget_bytes <= 0 || !(cfg->ir_share >= 0.0) ||
      cfg->ir_share > 1.0 || cfg->nnz_per_row_hint < 1)
    return sfail(nullptr, GMRES_ERR_ARG,
                 "need max_iter >= 1, max_requests >= 1, hbm_budget_bytes > 0, 0 <= ir_share <= 1, "
                 "nnz_per_row_hint >= 1");
  gmres_server_ctx* sv = new gmres_server_ctx();
  sv->cfg = *cfg;
  sv->t0 = std::chrono::steady_clock::now();
  int nsm = 0;
  if (cudaGetDevice(&sv->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, sv->device) != cudaSuccess) {
    delete sv;
    return sfail(nullptr, GMRES_ERR_CUDA, "no CUDA device");
  }
  for (int k = 0; k < 2; ++k) {
    const double share = k == 0 ? 1.0 - cfg->ir_share : cfg->ir_share;
    const int64_t budget = (int64_t)(share * (double)cfg->hbm_budget_bytes);
    EngineConfig c;
    c.m = cfg->m_restart;
    c.prec = k == 0 ? GMRES_FP64 : GMRES_IR_FP32;
    c.max_systems = cfg->max_requests;
    c.max_iter_cap = cfg->max_iter;
    // fixed per-slot state, then rows and CSR in proportion to a row's needs
    const int ld = c.m + 1;
    const int64_t per_slot = 8 * (int64_t)(2 * ld * c.m + ld * ld + 6 * ld + c.max_iter_cap + ld) + 256 * 12;
    const int64_t per_row = (int64_t)Engine::row_bytes(c);
    const int64_t csr_row = 4 + cfg->nnz_per_row_hint * (12 + (k == 1 ? 4 : 0));
    // reduction slots: (largest grid + slots) rows of 2 (m+1) + 2 partial sums
    const int64_t partials = 8 * ((int64_t)kMaxGridPerSm * nsm + c.max_systems + 1) * (2 * ld + 2);
    const int64_t avail = budget - per_slot * c.max_systems - partials;
    if (share > 0.0 && avail > (per_row + csr_row) * kPairRows) {
      c.rows = avail / (per_row + csr_row) / kPairRows * kPairRows;
      c.csr_bytes = c.rows * csr_row;
    } else {
      c.rows = 0;  // this engine takes no requests
    }
    Worker& W = sv->w[k];
    if (c.rows > 0) {
      if (W.eng.init(c) != GMRES_OK) {
        g_server_err = "engine " + std::to_string(k) + ": " + W.eng.err;
        gmres_server_destroy(sv);
        return GMRES_ERR_OOM;
      }
      cudaStreamCreateWithFlags(&W.eng.stream, cudaStreamNonBlocking);
      W.running.assign(c.max_systems, nullptr);
      W.th = std::thread(worker_loop, sv, k);
    }
  }
  *out = sv;
  return GMRES_OK;
}

gmres_status gmres_server_submit(gmres_server sv, const gmres_csr* A, const double* b, const double* x0,
                                 double* x_out, double tol, int prec, int max_iter, int64_t* id) {
  if (!sv) return GMRES_ERR_ARG;
  if (!A || !b || !x_out || !id) return sfail(sv, GMRES_ERR_ARG, "A, b, x_out and id must not be NULL");
  if (prec != GMRES_FP64 && prec != GMRES_IR_FP32) return sfail(sv, GMRES_ERR_ARG, "prec must be FP64 or IR_FP32");
  if (!(tol >= 0.0) || max_iter < 0 || max_iter > sv->cfg.max_iter)
    return sfail(sv, GMRES_ERR_ARG, "need tol >= 0 and 0 <= max_iter <= the server's max_iter");
  // O(1) checks here; the full CSR scan runs at admission, on the worker
  if (A->on_device || !A->rowptr || A->n <= 0 || A->nnz < 0 || (A->nnz > 0 && (!A->col || !A->val)) ||
      A->n >= (int64_t)INT32_MAX || A->nnz >= (int64_t)INT32_MAX || A->rowptr[0] != 0 || A->rowptr[A->n] != A->nnz)
    return sfail(sv, GMRES_ERR_ARG, "need a host CSR with n > 0, rowptr[0] = 0 and rowptr[n] = nnz");
  const int k = prec == GMRES_FP64 ? 0 : 1;
  Worker& W = sv->w[k];
  if (W.eng.R == 0 || !W.eng.fits_ever(A->n, A->nnz)) {
    std::lock_guard<std::mutex> lk(sv->mu);
    ++sv->rejected;
    return sfail(sv, GMRES_ERR_OOM, "request larger than its engine's share of the byte budget");
  }
  auto r = std::make_unique<Request>();
  r->A = *A;
  r->b = b;
  r->x0 = x0;
  r->x_out = x_out;
  r->tol = tol;
  r->prec = prec;
  r->max_iter = max_iter;
  r->t_submit = std::chrono::steady_clock::now();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    r->id = sv->next_id++;
    *id = r->id;
    W.queue.push_back(r.get());
    sv->reqs[r->id] = std::move(r);
    ++sv->submitted;
  }
  sv->cv_work.notify_all();
  return GMRES_OK;
}

gmres_status gmres_server_poll(gmres_server sv, int64_t id, int* done, gmres_info* info) {
  if (!sv || !done) return GMRES_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return sfail(sv, GMRES_ERR_ARG, "unknown request id");
  *done = it->second->done;
  if (*done && info) *info = it->second->info;
  return GMRES_OK;
}

gmres_status gmres_server_wait(gmres_server sv, int64_t id, double timeout_s, gmres_info* info) {
  if (!sv) return GMRES_ERR_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return sfail(sv, GMRES_ERR_ARG, "unknown request id");
  Request* r = it->second.get();
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                                            std::chrono::duration<double>(std::max(0.0, timeout_s)));
  if (!sv->cv_done.wait_until(lk, until, [&] { return r->done; })) return GMRES_ERR_TIMEOUT;
  if (info) *info = r->info;
  return (gmres_status)(r->info.status < 0 ? r->info.status : GMRES_OK);
}

gmres_status gmres_server_drain(gmres_server sv, double timeout_s) {
  if (!sv) return GMRES_ERR_ARG;
  std::unique_lock<std::mutex> lk(sv->mu);
  const auto until = std::chrono::steady_clock::now() + std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                                                            std::chrono::duration<double>(std::max(0.0, timeout_s)));
  const bool ok = sv->cv_done.wait_until(lk, until, [&] {
    for (auto& kv : sv->reqs)
      if (!kv.second->done) return false;
    return true;
  });
  return ok ? GMRES_OK : GMRES_ERR_TIMEOUT;
}

gmres_status gmres_server_release(gmres_server sv, int64_t id) {
  if (!sv) return GMRES_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(id);
  if (it == sv->reqs.end()) return sfail(sv, GMRES_ERR_ARG, "unknown request id");
  if (!it->second->done) return sfail(sv, GMRES_ERR_ARG, "request still in flight");
  sv->reqs.erase(it);
  return GMRES_OK;
}

gmres_status gmres_server_stats(gmres_server sv, gmres_server_counters* st) {
  if (!sv || !st) return GMRES_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  std::memset(st, 0, sizeof(*st));
  st->submitted = sv->submitted;
  st->rejected = sv->rejected;
  for (int k = 0; k < 2; ++k) {
    const Worker& W = sv->w[k];
    const Engine& e = W.eng;
    st->admitted[k] = W.admitted;
    st->completed[k] = W.completed;
    st->queued[k] = (int64_t)W.queue.size();
    int64_t nrun = 0;
    for (Request* q : W.running) nrun += q != nullptr;
    st->running[k] = nrun;
    st->peak_running[k] = W.peak_running;
    st->cycles[k] = W.cycles;
    st->busy_seconds[k] = W.busy_s;
    st->kernel_launches[k] = e.launches;
    const int64_t row_bytes = (int64_t)Engine::row_bytes(e.cfg);
    st->engine_bytes[k] = e.R > 0 ? (int64_t)Engine::footprint(e.cfg) : 0;
    st->peak_bytes_in_use[k] = W.peak_rows * kPairRows * row_bytes + W.peak_csr_units * 256;
    st->arena_rows[k] = e.R;
  }
  st->wall_seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - sv->t0).count();
  return GMRES_OK;
}

gmres_status gmres_server_set_profile(gmres_server sv, int on) {
  if (!sv) return GMRES_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  for (Worker& W : sv->w) {
    bool busy = !W.queue.empty();
    for (Request* q : W.running) busy |= q != nullptr;
    if (busy) return sfail(sv, GMRES_ERR_ARG, "profiling can be switched only while the server is idle");
  }
  for (Worker& W : sv->w) {
    W.eng.prof_on = on != 0;
    W.eng.prof_reset();
  }
  return GMRES_OK;
}

gmres_status gmres_server_profile(gmres_server sv, int engine, int cls, double* total_ms, int64_t* launches,
                                  double* alg_bytes, double* alg_flops) {
  if (!sv || engine < 0 || engine > 1) return GMRES_ERR_ARG;
  if (cls < 0 || cls >= GMRES_PROFILE_CLASSES) return sfail(sv, GMRES_ERR_ARG, "profile class out of range");
  std::lock_guard<std::mutex> lk(sv->mu);
  const Engine& e = sv->w[engine].eng;
  if (total_ms) *total_ms = e.prof_ms[cls];
  if (launches) *launches = e.prof_cnt[cls];
  if (alg_bytes) *alg_bytes = e.prof_bytes[cls];
  if (alg_flops) *alg_flops = e.prof_flops[cls];
  return GMRES_OK;
}

gmres_status gmres_server_latencies(gmres_server sv, double* buf, int cap, int* len) {
  if (!sv) return GMRES_ERR_ARG;
  std::lock_guard<std::mutex> lk(sv->mu);
  if (len) *len = (int)sv->latencies.size();
  if (buf && cap > 0)
    std::memcpy(buf, sv->latencies.data(), sizeof(double) * std::min<size_t>(cap, sv->latencies.size()));
  return GMRES_OK;
}

}  // extern "C"
