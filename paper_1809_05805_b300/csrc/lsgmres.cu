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
//    memory, an atomic ticket elects the last CTA, which sums the partials in
//    CTA order (deterministic) and runs the small dense epilogue (lagged norm,
//    Givens rotation, T row, T s, MAXPY coefficients) in shared memory.
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
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "lsgmres.h"

namespace {

constexpr int kThreads = 256;                // CTA size; also rows per tile
constexpr int kWarps = kThreads / 32;        // 8
constexpr int kRowsPerLane = kThreads / 32;  // rows of a tile handled by one lane in the dot phase
constexpr int kMaxM = 128;                   // largest restart length
constexpr double kEps = 2.220446049250313e-16;
constexpr double kBreakdownFactor = 16.0;

// --------------------------------------------------------------------------
// device state
// --------------------------------------------------------------------------
struct DevState {
  double bnorm;        // ||b|| (or ||r0|| for gmres_arnoldi)
  double inv_bnorm;    // 1 / bnorm (the residual estimate multiplies; FP64 division is slow)
  double cycle_scale;  // norm the cycle's right-hand side was divided by (FP32 cycles), else 1
  double rnorm;        // last true-residual norm
  double tol;
  double est;          // last Givens estimate (relative)
  int step;            // next Arnoldi step of the cycle
  int inner;           // MGS: next inner-product index within the step
  int kmax;            // steps allowed in this cycle
  int k;               // Hessenberg columns completed in this cycle
  int done;            // cycle finished
  int converged;
  int breakdown;
  int nonfinite;
  int maxpy_k;         // columns of the pending Arnoldi MAXPY
  int total_iters;     // over all cycles
  int restarts;
  int breakdowns;
  unsigned int ticket; // last-CTA election
  int pad;
  long long reductions;
  long long grid_syncs;
  double mgs_coef;     // MGS: coefficient of the pending axpy
};

// Device pointers into the small dense arrays (one allocation).
struct Small {
  DevState* st;
  double* H;        // (m+1) x m, unrotated, column-major, ld = m+1
  double* Rg;       // (m+1) x m, rotated
  double* cs;       // m+1
  double* sn;       // m+1
  double* g;        // m+2
  double* T;        // (m+1) x (m+1), lower, ld = m+1
  double* scale;    // m+2: 1/||u_k||
  double* coef;     // m+3: [alpha, c_0 .. c_m] of the pending Arnoldi MAXPY
  double* coefx;    // m+3: [1, y_0 s_0 .. ] of the solution update
  double* hist;     // hist_cap
  double* partials; // P x nvmax
  double* raw;      // nvmax: standalone block-dot output
  int m;
  int ldh;          // m + 1
  int nvmax;        // 2 (m + 1) + 2
  int hist_cap;
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Butterfly reduce-scatter of 32 per-lane values over the warp: 31 adds
// (16 + 8 + 4 + 2 + 1), each lane keeping the half its lane bit selects at
// every level. On return lane l holds the sum over the 32 lanes of slot l
// (also returned). Fixed order: bitwise reproducible.
template <typename T>
__device__ __forceinline__ T warp_reduce_scatter32(T* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const T send = up ? v[i] : v[i + o];
      const T keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0];
}

// Sum one value over the CTA (fixed order); result valid in thread 0.
__device__ __forceinline__ double block_sum(double v, double* sbuf /* kWarps */) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  if (lane == 0) sbuf[wid] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0) {
    for (int i = 0; i < kWarps; ++i) t += sbuf[i];
  }
  __syncthreads();
  return t;
}

// Row i of A times x (CSR, FP64 FMA chain in column order). The loads of up
// to 8 entries are issued together (predicated), so a stencil row costs two
// dependent memory latencies (indices, then the gather) instead of two per entry.
template <typename VT>
__device__ __forceinline__ VT csr_row(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                          const VT* __restrict__ val, const VT* __restrict__ x,
                                          int64_t i) {
  constexpr int kW = 8;
  const int p0 = __ldg(rowptr + i), p1 = __ldg(rowptr + i + 1);
  VT s = VT(0);
  for (int p = p0; p < p1; p += kW) {
    int c[kW];
    VT v[kW], xv[kW];
#pragma unroll
    for (int e = 0; e < kW; ++e) {
      const bool ok = p + e < p1;
      c[e] = ok ? __ldg(col + p + e) : 0;
      v[e] = ok ? __ldg(val + p + e) : VT(0);
    }
#pragma unroll
    for (int e = 0; e < kW; ++e) xv[e] = (p + e < p1) ? __ldg(x + c[e]) : VT(0);
#pragma unroll
    for (int e = 0; e < kW; ++e)
      if (p + e < p1) s = fma(v[e], xv[e], s);
  }
  return s;
}

// Rows r0 and r1 of A times x with the loads of both rows in flight together
// (rows of up to 8 entries; longer rows use csr_row). Rows >= n give 0.
template <typename VT>
__device__ __forceinline__ void csr_row2(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                         const VT* __restrict__ val, const VT* __restrict__ x,
                                         int64_t r0, int64_t r1, int64_t n, VT& y0, VT& y1) {
  constexpr int kW = 8;
  const int a0 = r0 < n ? __ldg(rowptr + r0) : 0, b0 = r0 < n ? __ldg(rowptr + r0 + 1) : 0;
  const int a1 = r1 < n ? __ldg(rowptr + r1) : 0, b1 = r1 < n ? __ldg(rowptr + r1 + 1) : 0;
  if (b0 - a0 <= kW && b1 - a1 <= kW) {
    int c0[kW], c1[kW];
    VT v0[kW], v1[kW];
#pragma unroll
    for (int e = 0; e < kW; ++e) {
      c0[e] = (a0 + e < b0) ? __ldg(col + a0 + e) : 0;
      v0[e] = (a0 + e < b0) ? __ldg(val + a0 + e) : VT(0);
      c1[e] = (a1 + e < b1) ? __ldg(col + a1 + e) : 0;
      v1[e] = (a1 + e < b1) ? __ldg(val + a1 + e) : VT(0);
    }
    VT x0[kW], x1[kW];
#pragma unroll
    for (int e = 0; e < kW; ++e) {
      x0[e] = (a0 + e < b0) ? __ldg(x + c0[e]) : VT(0);
      x1[e] = (a1 + e < b1) ? __ldg(x + c1[e]) : VT(0);
    }
    VT s0 = VT(0), s1 = VT(0);
#pragma unroll
    for (int e = 0; e < kW; ++e) {
      if (a0 + e < b0) s0 = fma(v0[e], x0[e], s0);
      if (a1 + e < b1) s1 = fma(v1[e], x1[e], s1);
    }
    y0 = s0;
    y1 = s1;
  } else {
    y0 = r0 < n ? csr_row(rowptr, col, val, x, r0) : VT(0);
    y1 = r1 < n ? csr_row(rowptr, col, val, x, r1) : VT(0);
  }
}

// Sum nslot rows of partial sums (slots slot0 .. slot0+nslot-1, row stride
// nvmax) into red[0 .. nv), all threads of the CTA: S threads per value (S a
// power of two, S * nv <= blockDim) sum slots seg, seg + S, ... in order; the S
// sums are combined by a fixed xor tree (and, for S > 32, across warps in warp
// order). The order is independent of timing: results are bitwise reproducible.
__device__ void reduce_slots(const double* partials, int64_t slot0, int nslot, int nvmax, double* red, int nv) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  int S = 1;
  while (2 * S * nv <= (int)blockDim.x && S < (int)blockDim.x) S *= 2;
  const int Sw = S < 32 ? S : 32;
  __shared__ double wred[kThreads / 32];
  for (int base = 0; base < nv * S; base += blockDim.x) {
    const int t = base + threadIdx.x;
    const int v = t / S, seg = t % S;
    double acc = 0.0;
    if (v < nv) {
#pragma unroll 8
      for (int b = seg; b < nslot; b += S) acc += __ldcg(partials + (size_t)(slot0 + b) * nvmax + v);
    }
    for (int o = Sw >> 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (S > 32) {  // one pass only (S * nv <= blockDim): combine the warps of each value
      if (lane == 0) wred[wid] = acc;
      __syncthreads();
      if ((int)threadIdx.x < nv) {
        double t2 = 0.0;
        for (int w = threadIdx.x * (S / 32); w < ((int)threadIdx.x + 1) * (S / 32); ++w) t2 += wred[w];
        red[threadIdx.x] = t2;
      }
    } else if (v < nv && seg == 0) {
      red[v] = acc;
    }
  }
  __syncthreads();
}

// Publish this CTA's row `slot` of partial sums (red[0 .. nv)) and take a
// ticket; returns true in every thread of the CTA that arrived last of
// `expected`, after which red holds the totals over slots slot0 .. slot0 +
// expected - 1, and the ticket is reset for the next kernel.
__device__ bool publish_and_reduce(double* partials, int nvmax, int64_t slot, int64_t slot0, int expected,
                                   unsigned int* ticket, double* red, int nv) {
  __shared__ int s_last;
  for (int v = threadIdx.x; v < nv; v += blockDim.x) partials[(size_t)slot * nvmax + v] = red[v];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) s_last = (atomicAdd(ticket, 1u) == (unsigned)expected - 1);
  __syncthreads();
  if (!s_last) return false;
  __threadfence();
  reduce_slots(partials, slot0, expected, nvmax, red, nv);
  if (threadIdx.x == 0) *ticket = 0u;
  return true;
}

// Grid-wide form: every CTA of the grid publishes one slot (its block index).
__device__ bool grid_reduce_last(Small s, double* red, int nv) {
  if (!publish_and_reduce(s.partials, s.nvmax, blockIdx.x, 0, gridDim.x, &s.st->ticket, red, nv)) return false;
  if (threadIdx.x == 0) s.st->reductions += 1;
  return true;
}

// Column j of H is complete (entries 0..j+1 in global memory). Run by the
// whole CTA: the column and the stored rotations are staged in shared memory
// with parallel loads, then thread 0 rotates the column, forms rotation j,
// updates g, records the residual estimate and decides whether the cycle
// stops (breakdown, convergence, non-finite, or the last allowed column).
// Returns the stop decision (0/1) in every thread.
__device__ int finish_column(Small s, int j, double h, bool last_allowed) {
  __shared__ double sh_col[kMaxM + 2], sh_c[kMaxM + 1], sh_s[kMaxM + 1];
  __shared__ int s_res;
  const int ld = s.ldh;
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) sh_col[i] = s.H[(size_t)j * ld + i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    sh_c[i] = s.cs[i];
    sh_s[i] = s.sn[i];
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    DevState* st = s.st;
    double hn2 = 0.0;  // ||Hbar(0:j+1, j)||^2 for the breakdown test
    for (int i = 0; i <= j + 1; ++i) hn2 += sh_col[i] * sh_col[i];
    double* R = sh_col;
    for (int i = 0; i < j; ++i) {
      const double c = sh_c[i], sn = sh_s[i];
      const double t = c * R[i] + sn * R[i + 1];
      R[i + 1] = -sn * R[i] + c * R[i + 1];
      R[i] = t;
    }
    double c = 1.0, sn = 0.0;
    if (R[j + 1] != 0.0) {
      const double irho = 1.0 / hypot(R[j], R[j + 1]);
      c = R[j] * irho;
      sn = R[j + 1] * irho;
    }
    R[j] = c * R[j] + sn * R[j + 1];
    R[j + 1] = 0.0;
    double* Rg = s.Rg + (size_t)j * ld;
    for (int i = 0; i <= j + 1; ++i) Rg[i] = R[i];
    s.cs[j] = c;
    s.sn[j] = sn;
    const double gj = s.g[j];
    s.g[j + 1] = -sn * gj;
    s.g[j] = c * gj;
    const double est = fabs(sn * gj) * st->cycle_scale * st->inv_bnorm;
    const int it = st->total_iters + j;
    if (it < s.hist_cap) s.hist[it] = est;
    st->k = j + 1;
    st->est = est;
    int stop = 0;
    if (!isfinite(est)) {
      st->nonfinite = 1;
      stop = 1;
    } else if (h <= kBreakdownFactor * kEps * sqrt(hn2)) {
      st->breakdown = 1;
      stop = 1;
    } else if (est <= st->tol) {
      st->converged = 1;
      stop = 1;
    } else if (last_allowed) {
      stop = 1;
    }
    s_res = stop;
  }
  __syncthreads();
  return s_res;
}

// --------------------------------------------------------------------------
// one-reduce step: fused SpMV + block dot + epilogue
// --------------------------------------------------------------------------
// Step j of a cycle (u_j = column j, not yet normalized; V_{j} = columns 0..j-1):
//   w = A u_j;
//   X = [a = U_j^T u_j, c = U_j^T w, sigma = u_j^T u_j, d = u_j^T w]  (one reduction)
// where U_j holds the unnormalized columns; the epilogue applies scale[k].
// At j == kmax (the tail) the SpMV and c, d are skipped.
// Standalone mode (raw_out != nullptr): j is j_arg, w may be an input
// (use_spmv == 0), and the totals go to raw_out without the GMRES epilogue.
// One 256-row tile t of the fused SpMV + block dot (one row per thread in the
// SpMV, the block-dot work split over the 8 warps), accumulated into the
// caller's per-thread sums.
template <int MAXC, typename VT>
__device__ __forceinline__ void tile_block_dot(int64_t t, int64_t n, const int32_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col, const VT* __restrict__ val,
                                               const VT* __restrict__ V, int64_t ldv, const VT* __restrict__ u,
                                               VT* __restrict__ w, bool spmv, bool need_w, int J8, int r8, VT* su,
                                               VT* sw, VT (&acc_a)[MAXC], VT (&acc_c)[MAXC],
                                               VT (&rem_a)[kWarps - 1], VT (&rem_c)[kWarps - 1], VT& sig,
                                               VT& dd) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row = t * kThreads + threadIdx.x;
  VT ur = VT(0), wr = VT(0);
  if (row < n) {
    ur = u[row];
    if (spmv) {
      wr = csr_row(rowptr, col, val, u, row);
      w[row] = wr;
    } else if (need_w) {
      wr = w[row];
    }
  }
  sig = fma(ur, ur, sig);
  dd = fma(ur, wr, dd);
  su[threadIdx.x] = ur;
  sw[threadIdx.x] = wr;
  __syncthreads();
  const int64_t base = t * kThreads + lane;
  VT ru[kRowsPerLane], rw[kRowsPerLane];
#pragma unroll
  for (int q = 0; q < kRowsPerLane; ++q) {
    ru[q] = su[lane + 32 * q];
    rw[q] = sw[lane + 32 * q];
  }
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    if (c < J8) {  // warp-uniform
      const int k = wid + c * kWarps;
      const VT* vk = V + (size_t)k * ldv + base;
      VT x[kRowsPerLane];
#pragma unroll
      for (int q = 0; q < kRowsPerLane; ++q) x[q] = (base + 32 * q < n) ? __ldg(vk + 32 * q) : VT(0);
#pragma unroll
      for (int q = 0; q < kRowsPerLane; ++q) acc_a[c] = fma(x[q], ru[q], acc_a[c]);
      if (need_w) {  // the cycle's tail needs only V^T u
#pragma unroll
        for (int q = 0; q < kRowsPerLane; ++q) acc_c[c] = fma(x[q], rw[q], acc_c[c]);
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kWarps - 1; ++c) {
    if (c < r8) {  // block-uniform
      const VT x = (row < n) ? __ldg(V + (size_t)(J8 * kWarps + c) * ldv + row) : VT(0);
      rem_a[c] = fma(x, ur, rem_a[c]);
      if (need_w) rem_c[c] = fma(x, wr, rem_c[c]);
    }
  }
  __syncthreads();
}

// Tiles 2 pp and 2 pp + 1 (rows 512 pp .. 512 pp + 511) of the fused SpMV +
// block dot, two rows per thread: the CSR loads of both rows are in flight
// together, halving the latency-bound SpMV phases per row. su, sw hold 512
// values.
template <int MAXC, typename VT>
__device__ __forceinline__ void tile_pair_block_dot(int64_t pp, int64_t n, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                    const VT* __restrict__ V, int64_t ldv, const VT* __restrict__ u,
                                                    VT* __restrict__ w, bool spmv, bool need_w, int J8, int r8,
                                                    VT* su, VT* sw, VT (&acc_a)[MAXC], VT (&acc_c)[MAXC],
                                                    VT (&rem_a)[kWarps - 1], VT (&rem_c)[kWarps - 1], VT& sig,
                                                    VT& dd) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row0 = pp * (2 * kThreads) + threadIdx.x, row1 = row0 + kThreads;
  VT ur0 = VT(0), wr0 = VT(0), ur1 = VT(0), wr1 = VT(0);
  if (row0 < n) ur0 = u[row0];
  if (row1 < n) ur1 = u[row1];
  if (spmv) {
    csr_row2(rowptr, col, val, u, row0, row1, n, wr0, wr1);
    if (row0 < n) w[row0] = wr0;
    if (row1 < n) w[row1] = wr1;
  } else if (need_w) {
    if (row0 < n) wr0 = w[row0];
    if (row1 < n) wr1 = w[row1];
  }
  sig = fma(ur0, ur0, sig);
  dd = fma(ur0, wr0, dd);
  sig = fma(ur1, ur1, sig);
  dd = fma(ur1, wr1, dd);
  su[threadIdx.x] = ur0;
  sw[threadIdx.x] = wr0;
  su[kThreads + threadIdx.x] = ur1;
  sw[kThreads + threadIdx.x] = wr1;
  __syncthreads();
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t base = pp * (2 * kThreads) + h * kThreads + lane;
    VT ru[kRowsPerLane], rw[kRowsPerLane];
#pragma unroll
    for (int q = 0; q < kRowsPerLane; ++q) {
      ru[q] = su[h * kThreads + lane + 32 * q];
      rw[q] = sw[h * kThreads + lane + 32 * q];
    }
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
      if (c < J8) {  // warp-uniform
        const int k = wid + c * kWarps;
        const VT* vk = V + (size_t)k * ldv + base;
        VT x[kRowsPerLane];
#pragma unroll
        for (int q = 0; q < kRowsPerLane; ++q) x[q] = (base + 32 * q < n) ? __ldg(vk + 32 * q) : VT(0);
#pragma unroll
        for (int q = 0; q < kRowsPerLane; ++q) acc_a[c] = fma(x[q], ru[q], acc_a[c]);
        if (need_w) {  // the cycle's tail needs only V^T u
#pragma unroll
          for (int q = 0; q < kRowsPerLane; ++q) acc_c[c] = fma(x[q], rw[q], acc_c[c]);
        }
      }
    }
  }
#pragma unroll
  for (int c = 0; c < kWarps - 1; ++c) {
    if (c < r8) {  // block-uniform
      const VT* vk = V + (size_t)(J8 * kWarps + c) * ldv;
      const VT x0 = (row0 < n) ? __ldg(vk + row0) : VT(0);
      const VT x1 = (row1 < n) ? __ldg(vk + row1) : VT(0);
      rem_a[c] = fma(x0, ur0, rem_a[c]);
      rem_a[c] = fma(x1, ur1, rem_a[c]);
      if (need_w) {
        rem_c[c] = fma(x0, wr0, rem_c[c]);
        rem_c[c] = fma(x1, wr1, rem_c[c]);
      }
    }
  }
  __syncthreads();
}

// Reduce the per-thread block-dot sums of the CTA into red[0 .. 2j+2).
template <int MAXC, typename VT>
__device__ __forceinline__ void cta_partials(VT (&acc_a)[MAXC], VT (&acc_c)[MAXC], VT (&rem_a)[kWarps - 1],
                                             VT (&rem_c)[kWarps - 1], VT sig, VT dd, int j, int J8, int r8,
                                             double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // CTA partials: red[0:j] = a, red[j:2j] = c, red[2j] = sigma, red[2j+1] = d.
  // Each lane's accumulators are packed into 32-slot chunks and reduced across
  // the warp by a butterfly reduce-scatter (31 adds per chunk instead of 5 per
  // value): lane l then holds the warp total of slot l.
  constexpr int kSlots = 2 * MAXC + 2 * (kWarps - 1) + 2;
  constexpr int kChunks = (kSlots + 31) / 32;
  VT v[kChunks * 32];
#pragma unroll
  for (int i = 0; i < kChunks * 32; ++i) v[i] = VT(0);
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    v[c] = acc_a[c];
    v[MAXC + c] = acc_c[c];
  }
#pragma unroll
  for (int c = 0; c < kWarps - 1; ++c) {
    v[2 * MAXC + c] = rem_a[c];
    v[2 * MAXC + kWarps - 1 + c] = rem_c[c];
  }
  v[kSlots - 2] = sig;
  v[kSlots - 1] = dd;
  __shared__ VT scross[kSlots - 2 * MAXC][kWarps];  // slots summed across warps
#pragma unroll
  for (int ch = 0; ch < kChunks; ++ch) {
    const VT tot = warp_reduce_scatter32(v + 32 * ch);
    const int slot = 32 * ch + lane;
    if (slot < MAXC) {
      if (slot < J8) red[wid + slot * kWarps] = tot;  // column wid + 8 slot belongs to this warp
    } else if (slot < 2 * MAXC) {
      if (slot - MAXC < J8) red[j + wid + (slot - MAXC) * kWarps] = tot;
    } else if (slot < kSlots) {
      scross[slot - 2 * MAXC][wid] = tot;
    }
  }
  __syncthreads();
  // remainder columns and the two norms: sum the 8 warps in warp order
  if ((int)threadIdx.x < kSlots - 2 * MAXC) {
    const int q = threadIdx.x;
    double t2 = 0.0;
    for (int w2 = 0; w2 < kWarps; ++w2) t2 += scross[q][w2];
    if (q < kWarps - 1) {
      if (q < r8) red[J8 * kWarps + q] = t2;
    } else if (q < 2 * (kWarps - 1)) {
      if (q - (kWarps - 1) < r8) red[j + J8 * kWarps + q - (kWarps - 1)] = t2;
    } else {
      red[2 * j + (q - 2 * (kWarps - 1))] = t2;
    }
  }
  __syncthreads();
}

// The one-reduce epilogue (last CTA), given the grid totals red[0 .. 2j+2) of
// step j: lagged norm, completion of column j-1 at the tail, T row, r = T s,
// the new Hessenberg column and the MAXPY coefficients.
__device__ void epilogue_one_reduce(Small s, double* red, int j, bool tail) {
  DevState* st = s.st;
  // ---------------- epilogue (last CTA) ----------------
  // stop: 0 = continue the cycle; 1 = cycle done after the T row (converged
  // or tail); 2 = cycle done now (breakdown, zero or non-finite norm); 3 =
  // exact breakdown found, column j-1 still to be finished (then 2).
  // T (rows and columns 0..j-1) and scale[0..j-1] are staged in shared memory
  // (dynamic, (m+1)^2 + (m+1) doubles) so the O(j^2) work reads no global memory.
  extern __shared__ double dyn[];
  const int ld = s.ldh;
  double* sT = dyn;                       // (m+1) x (m+1), column-major, ld
  double* sScale = dyn + (size_t)ld * ld; // m+1
  __shared__ double s_beta;
  __shared__ int s_stop;
  for (int e = threadIdx.x; e < j * j; e += blockDim.x) {
    const int k = e / j, i = e % j;  // column k, row i
    if (i >= k) sT[(size_t)k * ld + i] = s.T[(size_t)k * ld + i];
  }
  for (int i = threadIdx.x; i < j; i += blockDim.x) sScale[i] = s.scale[i];
  if (threadIdx.x == 0) {
    st->grid_syncs += 1;
    const double beta = sqrt(red[2 * j]);
    int stop = 0;
    if (!isfinite(beta)) {
      st->nonfinite = 1;
      stop = 2;
    } else if (j == 0) {
      if (beta == 0.0) stop = 2;  // r0 = 0: the host never starts such a cycle
      else s.g[0] = beta;
    } else {
      s.H[(size_t)(j - 1) * ld + j] = beta;  // H(j, j-1): the lagged norm completes column j-1
    }
    if (isfinite(beta) && beta != 0.0) s.scale[j] = 1.0 / beta;
    s_beta = beta;
    s_stop = stop;
  }
  __syncthreads();
  // exact breakdown (u_j = 0): column j-1 is still rotated (its h = 0 makes the
  // estimate exact), then the cycle ends without forming v_j (no 1/0)
  if (threadIdx.x == 0 && s_stop == 0 && j > 0 && s_beta == 0.0) s_stop = 3;
  __syncthreads();
  // Column j-1 is now complete. Except at the cycle's tail (or an exact
  // breakdown), its Givens rotation and the convergence test run in the
  // following MAXPY launch (one extra CTA beside the streaming CTAs): they are a
  // chain of dependent FP64 operations at ~64 cycles each on this part and are
  // not needed by the MAXPY.
  if (j > 0 && (s_stop == 3 || (s_stop == 0 && tail))) {
    const bool exact = (s_stop == 3);
    const int fin = finish_column(s, j - 1, s_beta, tail);
    if (threadIdx.x == 0) {
      if (exact || st->breakdown || st->nonfinite) s_stop = 2;
      else if (fin) s_stop = 1;
    }
    __syncthreads();
  }
  if (s_stop == 2) {
    if (threadIdx.x == 0) st->done = 1;
    return;
  }
  const double ib = 1.0 / s_beta;
  if (threadIdx.x == 0) sScale[j] = ib;
  // ell = (U_j^T u_j) scaled to v_k^T v_j
  for (int i = threadIdx.x; i < j; i += blockDim.x) red[i] = red[i] * sScale[i] * ib;
  __syncthreads();
  // row j of T = (I + L)^{-1}: T(j, k) = -sum_{i=k}^{j-1} ell_i T(i, k). Each sum
  // is split into 4 interleaved partial sums on different warps (shorter
  // dependent FP64 chains), combined in a fixed order.
  __shared__ double spart[4][kMaxM + 1];
  for (int t = threadIdx.x; t < 4 * j; t += blockDim.x) {
    const int seg = t / j, k = t % j;
    double p = 0.0;
    for (int i = k + seg; i < j; i += 4) p = fma(red[i], sT[(size_t)k * ld + i], p);
    spart[seg][k] = p;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < j; k += blockDim.x) {
    const double t = -(((spart[0][k] + spart[1][k]) + spart[2][k]) + spart[3][k]);
    sT[(size_t)k * ld + j] = t;
    s.T[(size_t)k * ld + j] = t;
  }
  if (threadIdx.x == 0) {
    sT[(size_t)j * ld + j] = 1.0;
    s.T[(size_t)j * ld + j] = 1.0;
  }
  __syncthreads();
  if (s_stop) {
    if (threadIdx.x == 0) st->done = 1;
    return;
  }
  // s = [c * scale / beta ; d / beta^2]
  __shared__ double sv[kMaxM + 1];
  for (int i = threadIdx.x; i <= j; i += blockDim.x)
    sv[i] = (i < j) ? red[j + i] * sScale[i] * ib : red[2 * j + 1] * ib * ib;
  __syncthreads();
  // r = T s (4 interleaved partial sums per entry); H(0:j, j) = r; MAXPY coefficients
  for (int t = threadIdx.x; t < 4 * (j + 1); t += blockDim.x) {
    const int seg = t / (j + 1), i = t % (j + 1);
    double p = 0.0;
    for (int k = seg; k <= i; k += 4) p = fma(sT[(size_t)k * ld + i], sv[k], p);
    spart[seg][i] = p;
  }
  __syncthreads();
  for (int i = threadIdx.x; i <= j; i += blockDim.x) {
    const double t = ((spart[0][i] + spart[1][i]) + spart[2][i]) + spart[3][i];
    s.H[(size_t)j * ld + i] = t;
    s.coef[1 + i] = -t * sScale[i];
  }
  if (threadIdx.x == 0) {
    s.coef[0] = ib;
    st->maxpy_k = j + 1;
    st->step = j + 1;
  }}

template <int MAXC, typename VT>
__global__ void __launch_bounds__(kThreads, 2)
k_one_reduce_step(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                  const VT* __restrict__ val, const VT* __restrict__ V, int64_t ldv,
                  const VT* __restrict__ u_arg, VT* __restrict__ w, int64_t n, Small s,
                  int j_arg, int use_spmv, double* raw_out) {
  __shared__ VT su[2 * kThreads];
  __shared__ VT sw[2 * kThreads];
  __shared__ double red[2 * (kMaxM + 1) + 2];
  __shared__ int s_j, s_tail, s_skip;
  DevState* st = s.st;
  if (threadIdx.x == 0) {
    if (raw_out) {
      s_j = j_arg;
      s_tail = 0;
      s_skip = 0;
    } else {
      s_skip = __ldcg(&st->done);
      s_j = __ldcg(&st->step);
      s_tail = (s_j == __ldcg(&st->kmax));
    }
  }
  __syncthreads();
  if (s_skip) return;
  const int j = s_j;
  const bool tail = s_tail;
  const bool spmv = raw_out ? (use_spmv != 0) : !tail;
  const bool need_w = raw_out ? true : !tail;
  const VT* u = raw_out ? u_arg : V + (size_t)j * ldv;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;

  // Work split of the block dot over a tile of 256 rows (8 row groups of 32):
  // the first 8*J8 columns go to warps whole (warp w owns columns w, w+8, ...,
  // all 8 row groups); the r8 = j mod 8 remaining columns are split by rows,
  // each warp taking its own row group. Every warp issues the same DFMAs.
  const int J8 = j / kWarps, r8 = j % kWarps;
  VT acc_a[MAXC], acc_c[MAXC];
  VT rem_a[kWarps - 1], rem_c[kWarps - 1];
#pragma unroll
  for (int c = 0; c < MAXC; ++c) acc_a[c] = acc_c[c] = VT(0);
#pragma unroll
  for (int c = 0; c < kWarps - 1; ++c) rem_a[c] = rem_c[c] = VT(0);
  VT sig = VT(0), dd = VT(0);

  const int64_t ntiles = (n + kThreads - 1) / kThreads;
  // Large problems take tiles in pairs (the CSR loads of two rows per thread are
  // in flight together, halving the latency-bound SpMV phases per row); small
  // ones keep one tile per CTA iteration so that every SM gets work.
  if (ntiles >= 4 * (int64_t)gridDim.x) {
    const int64_t npairs = (ntiles + 1) / 2;
    for (int64_t pp = blockIdx.x; pp < npairs; pp += gridDim.x)
      tile_pair_block_dot<MAXC, VT>(pp, n, rowptr, col, val, V, ldv, u, w, spmv, need_w, J8, r8, su, sw, acc_a, acc_c,
                                    rem_a, rem_c, sig, dd);
  } else {
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
      tile_block_dot<MAXC, VT>(t, n, rowptr, col, val, V, ldv, u, w, spmv, need_w, J8, r8, su, sw, acc_a, acc_c, rem_a,
                               rem_c, sig, dd);
  }

  cta_partials<MAXC, VT>(acc_a, acc_c, rem_a, rem_c, sig, dd, j, J8, r8, red);
  const int nv = 2 * j + 2;
  if (!grid_reduce_last(s, red, nv)) return;

  if (raw_out) {
    for (int v = threadIdx.x; v < nv; v += blockDim.x) raw_out[v] = red[v];
    return;
  }

  epilogue_one_reduce(s, red, j, tail);
}

// --------------------------------------------------------------------------
// MAXPY: out = alpha * y_in + sum_{k<K} c_k V[:, k]
// --------------------------------------------------------------------------
enum { MAXPY_ARNOLDI = 0, MAXPY_XUPDATE = 1, MAXPY_STANDALONE = 2 };

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
// GMRES-IR uses VT = float, YT = CT = double.
template <typename VT, typename YT, typename CT>
__global__ void __launch_bounds__(kThreads, 4)
k_maxpy(const VT* __restrict__ V, int64_t ldv, const YT* y_in, YT* y_out, int64_t n, Small s, int mode,
        int K_arg) {
  __shared__ double sc[kMaxM + 3];
  __shared__ CT scc[kMaxM + 3];
  __shared__ int sK, s_skip;
  __shared__ YT* s_out;
  DevState* st = s.st;
  if (threadIdx.x == 0) {
    s_skip = 0;
    s_out = y_out;
    if (mode == MAXPY_ARNOLDI) {
      s_skip = __ldcg(&st->done);
      sK = __ldcg(&st->maxpy_k);
      if constexpr (std::is_same<VT, YT>::value)
        s_out = const_cast<VT*>(V) + (size_t)__ldcg(&st->step) * ldv;
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
  if (mode == MAXPY_ARNOLDI && blockIdx.x == gridDim.x - 1) {
    // The last CTA of an Arnoldi MAXPY finishes column j-1 of H (Givens,
    // residual estimate, stop decision) while the other CTAs stream.
    const int j = __ldcg(&st->step) - 1;
    if (j >= 1) {
      const double h = __ldcg(&s.H[(size_t)(j - 1) * s.ldh + j]);
      const int stop = finish_column(s, j - 1, h, false);
      if (threadIdx.x == 0) {
        st->grid_syncs += 1;
        if (stop) st->done = 1;
      }
    }
    return;
  }
  const int ndata = gridDim.x - (mode == MAXPY_ARNOLDI ? 1 : 0);  // CTAs that stream
  YT* out = s_out;
  const CT alpha = scc[0];
  const int64_t stride = (int64_t)ndata * blockDim.x;
  const int64_t gid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
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
        for (int e = 0; e < E; ++e) o.e[e] = (VT)a[e];
        reinterpret_cast<V16*>(out)[i] = o.v;
      }
      done_rows = nE * E;
      for (int64_t i = done_rows + gid; i < n; i += stride) {  // ragged tail
        CT a0 = alpha * (CT)y_in[i];
        for (int k = 0; k < K; ++k) a0 = fma(scc[1 + k], (CT)V[(size_t)k * ldv + i], a0);
        out[i] = (YT)a0;
      }
      return;
    }
  }
  for (int64_t i = done_rows + gid; i < n; i += stride) {
    CT a0 = alpha * (CT)y_in[i];
    for (int k = 0; k < K; ++k) a0 = fma(scc[1 + k], (CT)V[(size_t)k * ldv + i], a0);
    out[i] = (YT)a0;
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
// residual, norms, least squares, export
// --------------------------------------------------------------------------
enum { RES_BNORM = 0, RES_RESIDUAL = 1, RES_START = 2 };

// End of a residual / norm kernel for one system (thread 0): store the norm
// and, for a cycle start, reset the cycle state.
__device__ void residual_finish(Small s, double sumsq, int mode, int kmax) {
  DevState* st = s.st;
  st->grid_syncs += 1;
  const double nr = sqrt(sumsq);
  if (mode == RES_BNORM) {
    st->bnorm = nr;
    st->inv_bnorm = 1.0 / nr;
    return;
  }
  if (mode == RES_START) {
    st->bnorm = nr;
    st->inv_bnorm = 1.0 / nr;
  }
  st->rnorm = nr;
  st->cycle_scale = 1.0;
  st->step = 0;
  st->inner = 0;
  st->kmax = kmax;
  st->k = 0;
  st->done = 0;
  st->converged = 0;
  st->breakdown = 0;
  st->nonfinite = isfinite(nr) ? 0 : 1;
  st->maxpy_k = 0;
  s.g[0] = nr;
  s.scale[0] = 1.0 / nr;
  for (int i = 1; i <= s.m + 1; ++i) s.g[i] = 0.0;
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
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
    double v = b[r];
    if (mode == RES_RESIDUAL && x) v -= csr_row(rowptr, col, val, x, r);
    if (mode != RES_BNORM) V0[r] = v;
    acc = fma(v, v, acc);
  }
  const double tot = block_sum(acc, sbuf);
  if (threadIdx.x == 0) red[0] = tot;
  __syncthreads();
  if (!grid_reduce_last(s, red, 1)) return;
  if (threadIdx.x == 0) residual_finish(s, red[0], mode, kmax);
}

// Start of an FP32 (GMRES-IR) cycle: column 0 of the FP32 basis = r / ||r||
// rounded to FP32 (normalized in FP64 first, so the FP32 cycle works on a
// unit-scale right-hand side); the estimate and the correction of this cycle
// are scaled back by ||r||.
__global__ void k_round_scaled(const double* __restrict__ r, float* __restrict__ out, int64_t n, Small s) {
  const double rn = __ldcg(&s.st->rnorm);
  const double ir = 1.0 / rn;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (float)(r[i] * ir);
  if (blockIdx.x == 0 && threadIdx.x == 0) s.st->cycle_scale = rn;
}

__global__ void k_to_float(const double* __restrict__ a, float* __restrict__ out, int64_t n) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) out[i] = (float)a[i];
}

// Back substitution R(0:k,0:k) y = g(0:k) (column-oriented), then the
// coefficients of x += V_k y in the unnormalized basis, and the cycle totals.
// The k x k triangle of the rotated Hessenberg is staged in shared memory
// (dynamic, (m+1) x m doubles) so each of the k sequential steps is a
// shared-memory update, not a global-memory round trip.
__device__ void lsq_system(Small s) {
  extern __shared__ double sR[];
  __shared__ double y[kMaxM + 1];
  __shared__ int sk;
  DevState* st = s.st;
  if (threadIdx.x == 0) sk = st->k;
  __syncthreads();
  const int k = sk;
  const int ld = s.ldh;
  for (int e = threadIdx.x; e < k * ld; e += blockDim.x) sR[e] = s.Rg[e];
  __shared__ double rinv[kMaxM + 1];
  for (int l = threadIdx.x; l < k; l += blockDim.x) y[l] = s.g[l];
  __syncthreads();
  for (int l = threadIdx.x; l < k; l += blockDim.x) rinv[l] = 1.0 / sR[(size_t)l * ld + l];
  __syncthreads();
  for (int i = k - 1; i >= 0; --i) {
    if (threadIdx.x == 0) y[i] = y[i] * rinv[i];
    __syncthreads();
    const double yi = y[i];
    for (int l = threadIdx.x; l < i; l += blockDim.x) y[l] = fma(-sR[(size_t)i * ld + l], yi, y[l]);
    __syncthreads();
  }
  const double cs = st->cycle_scale;
  for (int l = threadIdx.x; l < k; l += blockDim.x) s.coefx[1 + l] = y[l] * s.scale[l] * cs;
  if (threadIdx.x == 0) {
    s.coefx[0] = 1.0;
    st->total_iters += k;
    st->restarts += 1;
    st->breakdowns += st->breakdown;
  }
}

__global__ void k_lsq(Small s) { lsq_system(s); }

// V_out[:, k] = scale[k] * V[:, k] for k <= kk (normalized basis export).
__global__ void k_export_basis(const double* __restrict__ V, int64_t ldv, double* __restrict__ Vo,
                               int64_t n, int kk, Small s) {
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int k = 0; k <= kk; ++k) {
    const double sc = s.scale[k];
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride)
      Vo[(size_t)k * n + r] = sc * V[(size_t)k * ldv + r];
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
constexpr size_t kNoAllocStateBytes = 256;             // DevState, padded
constexpr size_t kNoAllocBytes = kNoAllocStateBytes + sizeof(double) * (size_t)kNoAllocMaxCtas * kNoAllocNv;
static_assert(sizeof(DevState) <= kNoAllocStateBytes, "DevState outgrew its slot");
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// ==========================================================================
// batched solves: lock-step cycles over many independent systems
// ==========================================================================
// The systems' rows are concatenated, each padded to whole 256-row tiles, into
// one block-diagonal CSR and one basis (a tile never straddles two systems).
// The tiles of the systems still iterating are listed, system by system, in
// act_tiles (Ta entries; rebuilt by the host at cycle boundaries, so the grid
// always spreads over the remaining work). CTA b of a batched reduction kernel
// takes the contiguous range [b Ta / P, (b+1) Ta / P) of that list; when its
// range moves on to another system it
// publishes that system's partial sums into the system's slot for CTA b, and
// the last CTA to arrive for a system (per-system ticket) reduces the system's
// slots in slot order and runs that system's epilogue. Every active system
// takes step j of the cycle in the same launch; systems that finished their
// cycle (or the solve) are skipped.
struct BatchDev {
  const int32_t* tile_sys;   // T: system of each tile
  const int32_t* sys_tile1;  // S: one past the last tile of each system
  const int32_t* act_tiles;  // Ta: tiles of the active systems, system by system
  const int64_t* n_act;      // Ta (device scalar)
  const int32_t* sys_b0;     // S: first CTA whose tile range touches the system
  const int32_t* sys_nslot;  // S: number of CTAs touching it
  const int64_t* sys_slot0;  // S: first partial-sum slot of the system
  const Small* smalls;       // S: per-system dense state
  double* partials;          // slots x nvmax
  unsigned int* tickets;     // S
  int64_t ntiles;
  int nsys;
  int nvmax;
};

// This CTA's range [lo, hi) of the active-tile list: the first Pe = min(grid,
// Ta) CTAs split the list evenly (every range non-empty, so the CTAs touching
// a system are consecutive); the others get an empty range.
__device__ __forceinline__ void cta_tile_range(const BatchDev& bd, int64_t& lo, int64_t& hi) {
  const int64_t Ta = *bd.n_act;
  const int64_t Pe = Ta < (int64_t)gridDim.x ? Ta : (int64_t)gridDim.x;
  lo = hi = 0;
  if ((int64_t)blockIdx.x >= Pe) return;
  lo = (int64_t)blockIdx.x * Ta / Pe;
  hi = ((int64_t)blockIdx.x + 1) * Ta / Pe;
}

// Step j of the current cycle for every active system of the batch. PAIRS:
// two consecutive tiles of one system are processed together (two rows per
// thread) wherever the CTA's range allows.
template <int MAXC, bool PAIRS>
__global__ void __launch_bounds__(kThreads, 2)
kb_step(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const double* __restrict__ val,
        const double* __restrict__ V, int64_t ldv, double* __restrict__ w, int64_t NT, BatchDev bd, int j) {
  __shared__ double su[PAIRS ? 2 * kThreads : kThreads];
  __shared__ double sw[PAIRS ? 2 * kThreads : kThreads];
  __shared__ double red[2 * (kMaxM + 1) + 2];
  __shared__ int s_active, s_tail;
  const int J8 = j / kWarps, r8 = j % kWarps;
  const double* u = V + (size_t)j * ldv;
  double acc_a[MAXC], acc_c[MAXC], rem_a[kWarps - 1], rem_c[kWarps - 1];
  double sig = 0.0, dd = 0.0;
  int64_t lo, hi;
  cta_tile_range(bd, lo, hi);
  if (lo >= hi) return;  // no tiles (fewer active tiles than CTAs): no slot, no ticket
  int cur = -1;
  for (int64_t it = lo; it <= hi;) {
    const int64_t t = (it < hi) ? bd.act_tiles[it] : -1;
    const int snext = (it < hi) ? __ldg(bd.tile_sys + t) : -1;
    if (snext != cur) {  // CTA-uniform
      if (cur >= 0 && s_active) {  // this CTA is done with system cur: publish its sums
        cta_partials<MAXC, double>(acc_a, acc_c, rem_a, rem_c, sig, dd, j, J8, r8, red);
        const int64_t slot0 = bd.sys_slot0[cur];
        if (publish_and_reduce(bd.partials, bd.nvmax, slot0 + ((int)blockIdx.x - bd.sys_b0[cur]), slot0,
                               bd.sys_nslot[cur], bd.tickets + cur, red, 2 * j + 2)) {
          const Small sm = bd.smalls[cur];
          if (threadIdx.x == 0) sm.st->reductions += 1;
          epilogue_one_reduce(sm, red, j, s_tail);
        }
        __syncthreads();
      }
      if (snext < 0) break;
      cur = snext;
      __syncthreads();  // every warp is done reading the previous system's flags
      if (threadIdx.x == 0) {
        const DevState* st = bd.smalls[cur].st;
        const int kmax = __ldcg(&st->kmax);
        s_active = !__ldcg(&st->done) && j <= kmax;
        s_tail = (j == kmax);
      }
      __syncthreads();
#pragma unroll
      for (int c = 0; c < MAXC; ++c) acc_a[c] = acc_c[c] = 0.0;
#pragma unroll
      for (int c = 0; c < kWarps - 1; ++c) rem_a[c] = rem_c[c] = 0.0;
      sig = dd = 0.0;
    }
    // a system's tiles are consecutive in the list and in memory: tiles t and
    // t + 1 form the pair t / 2 when t is even
    if (PAIRS && (t & 1) == 0 && it + 1 < hi && __ldg(bd.tile_sys + t + 1) == cur) {
      if (s_active)
        tile_pair_block_dot<MAXC, double>(t >> 1, NT, rowptr, col, val, V, ldv, u, w, !s_tail, !s_tail, J8, r8, su,
                                          sw, acc_a, acc_c, rem_a, rem_c, sig, dd);
      it += 2;
      continue;
    }
    if (s_active)
      tile_block_dot<MAXC, double>(t, NT, rowptr, col, val, V, ldv, u, w, !s_tail, !s_tail, J8, r8, su, sw, acc_a,
                                   acc_c, rem_a, rem_c, sig, dd);
    ++it;
  }
}

// Arnoldi MAXPY of step j for every active system: the first Pe = min(ndata,
// Ta) CTAs take contiguous ranges of the active-tile list and stream each run
// of one system's tiles (consecutive rows) with 16-byte loads, four basis
// columns in flight, the system's coefficients staged in shared memory once per
// run. One CTA per system (block index >= ndata) finishes column j-1 of that
// system's Hessenberg matrix while the others stream.
__global__ void __launch_bounds__(kThreads, 4)
kb_maxpy(double* __restrict__ V, int64_t ldv, const double* __restrict__ w, BatchDev bd, int j, int ndata) {
  __shared__ double sc[kMaxM + 3];
  __shared__ int sK, s_on;
  __shared__ const double* s_coef;
  if ((int)blockIdx.x >= ndata) {
    const Small sm = bd.smalls[blockIdx.x - ndata];
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
  const int64_t Ta = *bd.n_act;
  const int64_t Pe = Ta < (int64_t)ndata ? Ta : (int64_t)ndata;
  if ((int64_t)blockIdx.x >= Pe) return;
  const int64_t lo = (int64_t)blockIdx.x * Ta / Pe, hi = ((int64_t)blockIdx.x + 1) * Ta / Pe;
  const double2* w2 = reinterpret_cast<const double2*>(w);
  double2* out2 = reinterpret_cast<double2*>(V + (size_t)(j + 1) * ldv);
  const int64_t ldv2 = ldv / 2;
  const double2* V2 = reinterpret_cast<const double2*>(V);
  for (int64_t it = lo; it < hi;) {
    const int64_t t0 = bd.act_tiles[it];
    const int sy = __ldg(bd.tile_sys + t0);
    const int64_t run = min(hi - it, (int64_t)__ldg(bd.sys_tile1 + sy) - t0);  // this system's tiles in range
    __syncthreads();  // every warp is done with the previous run's flags and coefficients
    if (threadIdx.x == 0) {
      const Small sm = bd.smalls[sy];
      s_on = !__ldcg(&sm.st->done) && j < __ldcg(&sm.st->kmax);
      sK = __ldcg(&sm.st->maxpy_k);
      s_coef = sm.coef;
    }
    __syncthreads();
    if (s_on) {
      const int K = sK;
      for (int i = threadIdx.x; i <= K; i += blockDim.x) sc[i] = __ldcg(s_coef + i);
      __syncthreads();
      const int64_t e0 = t0 * (kThreads / 2), e1 = (t0 + run) * (kThreads / 2);  // double2 elements
      for (int64_t e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const double2 y = w2[e];
        double a0 = sc[0] * y.x, a1 = sc[0] * y.y;
        int k = 0;
        for (; k + 4 <= K; k += 4) {
          double2 v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = __ldg(V2 + (size_t)(k + q) * ldv2 + e);
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            a0 = fma(sc[1 + k + q], v[q].x, a0);
            a1 = fma(sc[1 + k + q], v[q].y, a1);
          }
        }
        for (; k < K; ++k) {
          const double2 v = __ldg(V2 + (size_t)k * ldv2 + e);
          a0 = fma(sc[1 + k], v.x, a0);
          a1 = fma(sc[1 + k], v.y, a1);
        }
        out2[e] = make_double2(a0, a1);
      }
    }
    it += run;
  }
}

// Residual r = b - A x (or ||b||) of every system not yet retired: one norm
// reduction per system, then the cycle-start bookkeeping of residual_finish.
__global__ void __launch_bounds__(kThreads, 2)
kb_residual(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col, const double* __restrict__ val,
            const double* __restrict__ b, const double* __restrict__ x, double* __restrict__ V0, BatchDev bd,
            int mode) {
  __shared__ double sbuf[kWarps];
  __shared__ double red[2];
  __shared__ int s_on;
  int64_t lo, hi;
  cta_tile_range(bd, lo, hi);
  if (lo >= hi) return;  // no tiles (fewer active tiles than CTAs): no slot, no ticket
  int cur = -1;
  double acc = 0.0;
  for (int64_t it = lo; it <= hi; ++it) {
    const int64_t t = (it < hi) ? bd.act_tiles[it] : -1;
    const int snext = (it < hi) ? __ldg(bd.tile_sys + t) : -1;
    if (snext != cur) {  // CTA-uniform
      if (cur >= 0 && s_on) {
        const double tot = block_sum(acc, sbuf);
        if (threadIdx.x == 0) red[0] = tot;
        __syncthreads();
        const int64_t slot0 = bd.sys_slot0[cur];
        if (publish_and_reduce(bd.partials, bd.nvmax, slot0 + ((int)blockIdx.x - bd.sys_b0[cur]), slot0,
                               bd.sys_nslot[cur], bd.tickets + cur, red, 1)) {
          if (threadIdx.x == 0) {
            const Small sm = bd.smalls[cur];
            sm.st->reductions += 1;
            residual_finish(sm, red[0], mode, 0);
          }
        }
        __syncthreads();
      }
      if (snext < 0) break;
      cur = snext;
      acc = 0.0;
      __syncthreads();  // every warp is done reading the previous system's flag
      // a system the host has retired (kmax < 0) is left untouched
      if (threadIdx.x == 0) s_on = __ldcg(&bd.smalls[cur].st->kmax) >= 0;
      __syncthreads();
    }
    if (!s_on) continue;
    const int64_t row = t * kThreads + threadIdx.x;
    double v = b[row];
    if (mode == RES_RESIDUAL) v -= csr_row(rowptr, col, val, x, row);
    if (mode != RES_BNORM) V0[row] = v;
    acc = fma(v, v, acc);
  }
}

// Back substitution and cycle totals, one CTA per system active in this cycle.
__global__ void kb_lsq(BatchDev bd) {
  const Small sm = bd.smalls[blockIdx.x];
  if (__ldcg(&sm.st->kmax) <= 0) return;  // not active in this cycle
  lsq_system(sm);
}

// x += V_k y for every system active in this cycle (x padded like the basis).
__global__ void __launch_bounds__(kThreads, 4)
kb_xupdate(const double* __restrict__ V, int64_t ldv, double* __restrict__ x, BatchDev bd) {
  __shared__ double sc[kMaxM + 3];
  __shared__ int sK;
  __shared__ const double* s_coef;
  const int64_t Ta = *bd.n_act;
  for (int64_t it = blockIdx.x; it < Ta; it += gridDim.x) {
    const int64_t t = bd.act_tiles[it];
    if (threadIdx.x == 0) {
      const Small sm = bd.smalls[__ldg(bd.tile_sys + t)];
      sK = (__ldcg(&sm.st->kmax) > 0) ? __ldcg(&sm.st->k) : 0;
      s_coef = sm.coefx;
    }
    __syncthreads();
    const int K = sK;
    if (K > 0) {
      for (int i = threadIdx.x; i <= K; i += blockDim.x) sc[i] = __ldcg(s_coef + i);
      __syncthreads();
      const int64_t row = t * kThreads + threadIdx.x;
      double a = x[row];
      for (int k = 0; k < K; ++k) a = fma(sc[1 + k], __ldg(V + (size_t)k * ldv + row), a);
      x[row] = a;
    }
    __syncthreads();
  }
}

using BatchStepKernel = void (*)(const int32_t*, const int32_t*, const double*, const double*, int64_t, double*,
                                 int64_t, BatchDev, int);

template <bool PAIRS>
BatchStepKernel batch_step_kernel_sel(int m) {
  switch (std::max(1, m / kWarps)) {
    case 1: return kb_step<1, PAIRS>;
    case 2: return kb_step<2, PAIRS>;
    case 3: return kb_step<3, PAIRS>;
    case 4: return kb_step<4, PAIRS>;
    case 5: return kb_step<5, PAIRS>;
    case 6: return kb_step<6, PAIRS>;
    case 7: return kb_step<7, PAIRS>;
    case 8: return kb_step<8, PAIRS>;
    case 9: case 10: case 11: case 12: return kb_step<12, PAIRS>;
    default: return kb_step<16, PAIRS>;
  }
}

BatchStepKernel batch_step_kernel_for(int m, bool pairs) {
  return pairs ? batch_step_kernel_sel<true>(m) : batch_step_kernel_sel<false>(m);
}

template <typename VT>
using StepKernel = void (*)(const int32_t*, const int32_t*, const VT*, const VT*, int64_t, const VT*, VT*, int64_t,
                            Small, int, int, double*);

// MAXC = floor(m / 8) whole columns per warp (j <= m), at least 1.
template <typename VT>
StepKernel<VT> step_kernel_for(int m) {
  switch (std::max(1, m / kWarps)) {
    case 1: return k_one_reduce_step<1, VT>;
    case 2: return k_one_reduce_step<2, VT>;
    case 3: return k_one_reduce_step<3, VT>;
    case 4: return k_one_reduce_step<4, VT>;
    case 5: return k_one_reduce_step<5, VT>;
    case 6: return k_one_reduce_step<6, VT>;
    case 7: return k_one_reduce_step<7, VT>;
    case 8: return k_one_reduce_step<8, VT>;
    case 9: case 10: case 11: case 12: return k_one_reduce_step<12, VT>;
    default: return k_one_reduce_step<16, VT>;
  }
}

}  // namespace

// ==========================================================================
// host side
// ==========================================================================
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
  int grid_stream = 0;// CTAs of streaming kernels
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  double* V = nullptr;
  int64_t ldv = 0;
  double* w = nullptr;
  char* small = nullptr;
  Small s{};
  DevState* h_st = nullptr;  // pinned mirror
  cudaStream_t stream = nullptr;
  StepKernel<double> step = nullptr;
  StepKernel<float> step32 = nullptr;
  // GMRES-IR (FP32 cycles): FP32 basis, SpMV result and matrix values, and the
  // FP64 restart residual; allocated by gmres_set(GMRES_IR_FP32)
  float* V32 = nullptr;
  float* w32 = nullptr;
  float* val32 = nullptr;
  double* r64 = nullptr;
  size_t step_smem = 0;  // dynamic shared memory of the step kernel (T and scales)
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

std::string g_create_err;

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

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

void destroy_graphs(gmres_ctx* h);

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
  const size_t o_pa = take(sizeof(double) * (size_t)h->P * nvmax);
  const size_t o_raw = take(sizeof(double) * nvmax);
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
  if (h->ortho == GMRES_ONE_REDUCE_MGS) {
    for (int j = 0; j <= kmax; ++j) {
      int pr = prof_begin(h, 0, j, kmax);
      if (h->prec == GMRES_IR_FP32)
        h->step32<<<P, kThreads, h->step_smem, h->stream>>>(h->rowptr, h->col, h->val32, h->V32, h->ldv, nullptr,
                                                            h->w32, h->n, h->s, 0, 1, nullptr);
      else
        h->step<<<P, kThreads, h->step_smem, h->stream>>>(h->rowptr, h->col, h->val, h->V, h->ldv, nullptr, h->w,
                                                          h->n, h->s, 0, 1, nullptr);
      prof_end(h, pr);
      ++h->launches;
      if (j < kmax) {
        pr = prof_begin(h, 1, j, kmax);
        if (h->prec == GMRES_IR_FP32)
          k_maxpy<float, float, float><<<h->grid_stream + 1, kThreads, 0, h->stream>>>(
              h->V32, h->ldv, h->w32, nullptr, h->n, h->s, MAXPY_ARNOLDI, 0);
        else
          k_maxpy<double, double, double><<<h->grid_stream + 1, kThreads, 0, h->stream>>>(
              h->V, h->ldv, h->w, nullptr, h->n, h->s, MAXPY_ARNOLDI, 0);
        prof_end(h, pr);
        ++h->launches;
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

enum { PC_STEP = 0, PC_MAXPY = 1, PC_MGS_SPMV = 2, PC_MGS_AXPY = 3, PC_RES = 4, PC_LSQ = 5, PC_XUPD = 6,
       PC_NOOP = 7 };

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
gmres_status run_cycle(gmres_ctx* h, int kmax) {
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
    const int64_t nl = (h->ortho == GMRES_ONE_REDUCE_MGS) ? 2 * (int64_t)kmax + 1
                                                          : (int64_t)kmax + (int64_t)kmax * (kmax + 1) / 2;
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
  const bool f32 = h->prec == GMRES_IR_FP32;          // FP32 cycle: 4-byte vectors and values
  const double vb = f32 ? 4.0 : 8.0;
  const double csr = 4.0 * (n + 1) + (4.0 + (f32 && (r.cls == PC_STEP) ? 4.0 : 8.0)) * nnz;
  switch (r.cls) {
    case PC_STEP:
      if (r.j == r.i) {  // tail: u and V_j, no SpMV (r.i carries kmax)
        *bytes = vb * n * (r.j + 1);
        *flops = 2.0 * n * (r.j + 1);
      } else {
        *bytes = csr + vb * n * (r.j + 2);  // u (gathered), j basis columns, w written
        *flops = 2.0 * nnz + 2.0 * n * (2.0 * r.j + 2.0);
      }
      break;
    case PC_MAXPY:  // w, j+1 columns read, one column written
      *bytes = vb * n * (r.j + 3);
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
    else if (r.cls == PC_MGS_SPMV || r.cls == PC_MGS_AXPY) work = r.j < k;
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
  h->grid_stream = (int)std::min<int64_t>(4 * (int64_t)h->nsm, std::max<int64_t>(1, (n / 2 + kThreads - 1) / kThreads));
  const int64_t nnz_pad = align_up(std::max<int64_t>(nnz, 1), 4);
  CREATE_TRY(cudaMalloc(&h->rowptr, sizeof(int32_t) * (n + 1)));
  CREATE_TRY(cudaMalloc(&h->col, sizeof(int32_t) * nnz_pad));
  CREATE_TRY(cudaMalloc(&h->val, sizeof(double) * nnz_pad));
  CREATE_TRY(cudaMemset(h->col, 0, sizeof(int32_t) * nnz_pad));
  CREATE_TRY(cudaMemset(h->val, 0, sizeof(double) * nnz_pad));
  CREATE_TRY(cudaMemcpy(h->rowptr, rp.data(), sizeof(int32_t) * (n + 1), cudaMemcpyHostToDevice));
  if (nnz) {
    CREATE_TRY(cudaMemcpy(h->col, cl.data(), sizeof(int32_t) * nnz, cudaMemcpyHostToDevice));
    CREATE_TRY(cudaMemcpy(h->val, vl.data(), sizeof(double) * nnz, cudaMemcpyHostToDevice));
  }
  h->ldv = (int64_t)align_up((size_t)n, 32);
  CREATE_TRY(cudaMalloc(&h->V, sizeof(double) * (size_t)h->ldv * (m_restart + 1)));
  CREATE_TRY(cudaMemset(h->V, 0, sizeof(double) * (size_t)h->ldv * (m_restart + 1)));
  CREATE_TRY(cudaMalloc(&h->w, sizeof(double) * (size_t)h->ldv));
  CREATE_TRY(cudaMemset(h->w, 0, sizeof(double) * (size_t)h->ldv));
  CREATE_TRY(cudaMallocHost(&h->h_st, sizeof(DevState)));
  std::memset(h->h_st, 0, sizeof(DevState));
  if (alloc_small(h) != GMRES_OK) return bail(GMRES_ERR_CUDA);
  h->step = step_kernel_for<double>(m_restart);
  h->step32 = step_kernel_for<float>(m_restart);
  h->step_smem = sizeof(double) * ((size_t)(m_restart + 1) * (m_restart + 1) + (m_restart + 1));
  h->lsq_smem = sizeof(double) * (size_t)(m_restart + 1) * m_restart;
  CREATE_TRY(cudaFuncSetAttribute(reinterpret_cast<const void*>(h->step),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->step_smem));
  CREATE_TRY(cudaFuncSetAttribute(reinterpret_cast<const void*>(h->step32),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->step_smem));
  CREATE_TRY(cudaFuncSetAttribute(reinterpret_cast<const void*>(k_lsq),
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h->lsq_smem));
#undef CREATE_TRY
  *out = h;
  return GMRES_OK;
}

gmres_status gmres_set(gmres_handle h, gmres_ortho ortho, gmres_prec prec, int max_iter) {
  if (!h) return GMRES_ERR_ARG;
  if (ortho != GMRES_MGS && ortho != GMRES_ONE_REDUCE_MGS) return fail(h, GMRES_ERR_ARG, "unknown ortho");
  if (prec != GMRES_FP64 && prec != GMRES_IR_FP32)
    return fail(h, GMRES_ERR_ARG, "precision must be GMRES_FP64 or GMRES_IR_FP32");
  if (prec == GMRES_IR_FP32 && ortho != GMRES_ONE_REDUCE_MGS)
    return fail(h, GMRES_ERR_ARG, "GMRES_IR_FP32 runs the one-reduce scheme only");
  if (max_iter < 0) return fail(h, GMRES_ERR_ARG, "max_iter < 0");
  if (prec == GMRES_IR_FP32 && !h->V32) {  // FP32 copies for the inner cycles
    CUDA_TRY(h, cudaSetDevice(h->device));
    const int64_t nnz_pad = (int64_t)align_up((size_t)std::max<int64_t>(h->nnz, 1), 4);
    CUDA_TRY(h, cudaMalloc(&h->V32, sizeof(float) * (size_t)h->ldv * (h->m + 1)));
    CUDA_TRY(h, cudaMemset(h->V32, 0, sizeof(float) * (size_t)h->ldv * (h->m + 1)));
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
      k_residual<<<P, kThreads, 0, h->stream>>>(h->rowptr, h->col, h->val, b, x,
                                                 h->prec == GMRES_IR_FP32 ? h->r64 : h->V, h->n, h->s,
                                                 RES_RESIDUAL, 0);
      prof_end(h, pr);
      ++h->launches;
      LAUNCH_CHECK(h);
      if ((st = read_state(h)) != GMRES_OK) return st;
      const DevState& hs = *h->h_st;
      prof_settle(h, hs.total_iters - prev_total);
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
      if (h->prec == GMRES_IR_FP32) {
        k_round_scaled<<<h->grid_stream, kThreads, 0, h->stream>>>(h->r64, h->V32, h->n, h->s);
        ++h->launches;
        LAUNCH_CHECK(h);
      }
      if ((st = run_cycle(h, kmax)) != GMRES_OK) return st;
      pr = prof_begin(h, PC_LSQ, 0, 0);
      k_lsq<<<1, 128, h->lsq_smem, h->stream>>>(h->s);
      prof_end(h, pr);
      pr = prof_begin(h, PC_XUPD, 0, 0);
      if (h->prec == GMRES_IR_FP32)
        k_maxpy<float, double, double><<<h->grid_stream, kThreads, 0, h->stream>>>(h->V32, h->ldv, x, x, h->n, h->s,
                                                                                  MAXPY_XUPDATE, 0);
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
  cudaFree(h->w);
  cudaFree(h->small);
  cudaFree(h->d_b);
  cudaFree(h->d_x);
  cudaFree(h->V32);
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
  h->step<<<h->P, kThreads, h->step_smem, h->stream>>>(h->rowptr, h->col, h->val, V, ldv, u, w, h->n, h->s, j,
                                                        use_spmv, h->s.raw);
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
  k_one_reduce_step<kNoAllocMaxJ / kWarps, double><<<P, kThreads, 0, stream>>>(rowptr, col, val, V, ldv, u, w, n, sm, j,
                                                                      use_spmv, X);
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
  if (h->prec != GMRES_FP64) return fail(h, GMRES_ERR_ARG, "gmres_arnoldi runs the FP64 cycle only");
  CUDA_TRY(h, cudaSetDevice(h->device));
  std::memset(h->h_st, 0, sizeof(DevState));
  h->h_st->tol = 0.0;
  if ((st = write_state(h)) != GMRES_OK) return st;
  CUDA_TRY(h, cudaMemsetAsync(h->s.H, 0, sizeof(double) * h->s.ldh * h->m, h->stream));
  CUDA_TRY(h, cudaMemsetAsync(h->s.T, 0, sizeof(double) * h->s.ldh * h->s.ldh, h->stream));
  k_residual<<<h->P, kThreads, 0, h->stream>>>(h->rowptr, h->col, h->val, r0, nullptr, h->V, h->n, h->s, RES_START, k);
  LAUNCH_CHECK(h);
  if ((st = launch_cycle(h, k)) != GMRES_OK) return st;
  if ((st = read_state(h)) != GMRES_OK) return st;
  const int kk = h->h_st->k;
  if (h->h_st->nonfinite) return fail(h, GMRES_ERR_NONFINITE, "non-finite value in the Arnoldi process");
  if (k_done) *k_done = kk;
  if (V_out) {
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
            (h->ortho == GMRES_ONE_REDUCE_MGS && r <= kk && c <= kk) ? Td[r + (size_t)c * ld] : 0.0;
  return GMRES_OK;
}

}  // extern "C"

// ==========================================================================
// batched solves: host side
// ==========================================================================
struct gmres_batch_ctx {
  int S = 0, m = 0, max_iter = 0;
  double tol = 0.0;
  int device = 0, nsm = 0, P = 0, nvmax = 0, hist_cap = 0;
  int64_t NT = 0, T = 0, ldv = 0, total_slots = 0;
  std::vector<int64_t> n, row0, tile0, ntile;
  std::vector<int32_t> h_tile_sys;
  std::vector<char> layout_active;  // active set of the current device layout
  int32_t* rowptr = nullptr;
  int32_t* col = nullptr;
  double* val = nullptr;
  double* V = nullptr;
  double* w = nullptr;
  double* bcat = nullptr;
  double* xcat = nullptr;
  int32_t* tile_sys = nullptr;
  int32_t* sys_tile1 = nullptr;
  // device layout: active-tile list and per-system reduction slots
  int32_t* act_tiles = nullptr;
  int64_t* n_act = nullptr;
  int32_t* sys_b0 = nullptr;
  int32_t* sys_nslot = nullptr;
  int64_t* sys_slot0 = nullptr;
  // pinned staging of the layout (T + 2 S int32, S + 1 int64)
  char* h_layout = nullptr;
  int32_t* h_act = nullptr;
  int32_t* h_b0 = nullptr;
  int32_t* h_ns = nullptr;
  int64_t* h_s0 = nullptr;
  int64_t* h_nact = nullptr;
  Small* smalls_dev = nullptr;
  double* partials = nullptr;
  unsigned int* tickets = nullptr;
  char* blk = nullptr;
  DevState* states = nullptr;
  DevState* h_states = nullptr;  // pinned mirror of all systems' states
  std::vector<Small> smalls;
  size_t small_stride = 0;
  size_t step_smem = 0, lsq_smem = 0;
  BatchStepKernel step = nullptr;
  bool pairs = false;  // step kernel takes tile pairs (two rows per thread)
  cudaStream_t stream = nullptr;
  // profiling (events around each launch; graphs captured with timing nodes)
  struct Rec {
    int cls, j;
    cudaEvent_t a, b;
    double bytes, flops;  // bytes < 0: attributed when the cycle's columns are known
    int64_t tiles;        // active tiles at launch
  };
  struct LogEntry {
    int cls, j;
    int64_t tiles;
    float ms;
    double bytes, flops;
  };
  std::vector<LogEntry> log;  // every launch of the last profiled solve
  struct G {
    int kmax;
    bool prof;
    cudaGraphExec_t exec;
    std::vector<cudaEvent_t> events;
    std::vector<Rec> recs;
  };
  std::vector<G> graphs;
  G* cap = nullptr;          // graph being captured
  bool prof_on = false;
  std::vector<Rec> pending;  // launched, not yet attributed
  std::vector<cudaEvent_t> ev_pool;
  size_t ev_used = 0;
  double prof_ms[GMRES_PROFILE_CLASSES] = {}, prof_bytes[GMRES_PROFILE_CLASSES] = {},
         prof_flops[GMRES_PROFILE_CLASSES] = {};
  int64_t prof_cnt[GMRES_PROFILE_CLASSES] = {};
  std::vector<int64_t> nnz;
  std::vector<int> cyc_kmax, cyc_it0;  // per system: the cycle in flight (-1: not in it)
  std::vector<std::vector<double>> hist;
  std::vector<int> hist_len;
  std::string err;
};

namespace {

std::string g_batch_err;

gmres_status bfail(gmres_batch_ctx* b, gmres_status st, const std::string& msg) {
  if (b)
    b->err = msg;
  else
    g_batch_err = msg;
  return st;
}

#define BCUDA(b, call)                                                                                 \
  do {                                                                                                 \
    cudaError_t e_ = (call);                                                                           \
    if (e_ != cudaSuccess)                                                                             \
      return bfail(b, e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA,                \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                                \
  } while (0)

// Largest grid of the batched reduction kernels, in CTAs per SM.
constexpr int kBatchMaxCtasPerSm = 8;

int batch_max_grid(const gmres_batch_ctx* b) {
  return (int)std::min<int64_t>((int64_t)kBatchMaxCtasPerSm * b->nsm, b->T);
}

// CTAs of the streaming batched kernels (MAXPY, solution update).
int batch_stream_grid(const gmres_batch_ctx* b) { return (int)std::min<int64_t>(4 * (int64_t)b->nsm, b->T); }

BatchDev batch_dev(gmres_batch_ctx* b) {
  BatchDev d{};
  d.tile_sys = b->tile_sys;
  d.sys_tile1 = b->sys_tile1;
  d.act_tiles = b->act_tiles;
  d.n_act = b->n_act;
  d.sys_b0 = b->sys_b0;
  d.sys_nslot = b->sys_nslot;
  d.sys_slot0 = b->sys_slot0;
  d.smalls = b->smalls_dev;
  d.partials = b->partials;
  d.tickets = b->tickets;
  d.ntiles = b->T;
  d.nsys = b->S;
  d.nvmax = b->nvmax;
  return d;
}

// Device layout for the systems with active[i] != 0 and grid b->P: the list of
// their tiles (system by system) and, per system, the first CTA whose range
// [c Ta / Pe, (c+1) Ta / Pe) of the list touches it (Pe = min(P, Ta)), the
// number of such CTAs and its first partial-sum slot. Queued on `sm` from pinned staging (the caller
// has synchronized since the staging was last used).
gmres_status batch_layout(gmres_batch_ctx* b, const std::vector<char>& active, cudaStream_t sm) {
  const int S = b->S, P = b->P;
  int64_t Ta = 0;
  for (int i = 0; i < S; ++i)
    if (active[i])
      for (int64_t t = b->tile0[i]; t < b->tile0[i] + b->ntile[i]; ++t) b->h_act[Ta++] = (int32_t)t;
  std::vector<int32_t> b1(S, -1);
  for (int i = 0; i < S; ++i) b->h_b0[i] = INT32_MAX;
  const int Pe = (int)std::min<int64_t>(P, Ta);  // as cta_tile_range
  for (int c = 0; c < Pe; ++c) {
    const int64_t lo = (int64_t)c * Ta / Pe, hi = ((int64_t)c + 1) * Ta / Pe;
    for (int64_t it = lo; it < hi; ++it) {
      const int sy = b->h_tile_sys[b->h_act[it]];
      b->h_b0[sy] = std::min(b->h_b0[sy], c);
      b1[sy] = std::max(b1[sy], c);
    }
  }
  int64_t tot = 0;
  for (int i = 0; i < S; ++i) {
    if (b1[i] < 0) {  // not in the list
      b->h_b0[i] = 0;
      b->h_ns[i] = 0;
      b->h_s0[i] = 0;
      continue;
    }
    b->h_ns[i] = b1[i] - b->h_b0[i] + 1;
    b->h_s0[i] = tot;
    tot += b->h_ns[i];
  }
  if (tot > b->total_slots) return bfail(b, GMRES_ERR_ARG, "internal: slot capacity");
  *b->h_nact = Ta;
  if (Ta > 0) BCUDA(b, cudaMemcpyAsync(b->act_tiles, b->h_act, sizeof(int32_t) * Ta, cudaMemcpyHostToDevice, sm));
  BCUDA(b, cudaMemcpyAsync(b->n_act, b->h_nact, sizeof(int64_t), cudaMemcpyHostToDevice, sm));
  BCUDA(b, cudaMemcpyAsync(b->sys_b0, b->h_b0, sizeof(int32_t) * S, cudaMemcpyHostToDevice, sm));
  BCUDA(b, cudaMemcpyAsync(b->sys_nslot, b->h_ns, sizeof(int32_t) * S, cudaMemcpyHostToDevice, sm));
  BCUDA(b, cudaMemcpyAsync(b->sys_slot0, b->h_s0, sizeof(int64_t) * S, cudaMemcpyHostToDevice, sm));
  b->layout_active = active;
  return GMRES_OK;
}

void batch_drop_graphs(gmres_batch_ctx* b) {
  for (auto& g : b->graphs) {
    cudaGraphExecDestroy(g.exec);
    for (cudaEvent_t e : g.events) cudaEventDestroy(e);
  }
  b->graphs.clear();
}

// ---- profiling: an event pair around a launch (no-op unless profiling)
int batch_prof_begin(gmres_batch_ctx* b, int cls, int j, double bytes = -1.0, double flops = -1.0) {
  if (!b->prof_on) return -1;
  gmres_batch_ctx::Rec r{cls, j, nullptr, nullptr, bytes, flops, *b->h_nact};
  if (b->cap) {  // timing nodes of the graph being captured
    gmres_batch_ctx::G* g = b->cap;
    const size_t u = 2 * g->recs.size();
    if (u + 2 > g->events.size()) return -1;
    r.a = g->events[u];
    r.b = g->events[u + 1];
    cudaEventRecordWithFlags(r.a, b->stream, cudaEventRecordExternal);
    g->recs.push_back(r);
    return 1;
  }
  while (b->ev_used + 2 > b->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    b->ev_pool.push_back(e);
  }
  r.a = b->ev_pool[b->ev_used];
  r.b = b->ev_pool[b->ev_used + 1];
  b->ev_used += 2;
  cudaEventRecord(r.a, b->stream);
  b->pending.push_back(r);
  return 0;
}

void batch_prof_end(gmres_batch_ctx* b, int tok) {
  if (tok < 0) return;
  if (tok == 1)
    cudaEventRecordWithFlags(b->cap->recs.back().b, b->stream, cudaEventRecordExternal);
  else
    cudaEventRecord(b->pending.back().b, b->stream);
}

// Algorithmic bytes and flops of one batched launch, summed over the systems
// it did work for (the same per-system model as the single-system solver; a
// system's cycle of k columns ran steps 0..k).
void batch_alg_model(const gmres_batch_ctx* b, const gmres_batch_ctx::Rec& r, const std::vector<int>& kcol,
                     double* bytes, double* flops) {
  double by = 0.0, fl = 0.0;
  for (int i = 0; i < b->S; ++i) {
    const int km = b->cyc_kmax[i], k = kcol[i];
    if (km < 0) continue;
    const double n = (double)b->n[i], nnz = (double)b->nnz[i], csr = 4.0 * (n + 1) + 12.0 * nnz;
    const int j = r.j;
    if (r.cls == PC_STEP && j <= k) {
      if (j == km) {
        by += 8.0 * n * (j + 1);
        fl += 2.0 * n * (j + 1);
      } else {
        by += csr + 8.0 * n * (j + 2);
        fl += 2.0 * nnz + 2.0 * n * (2.0 * j + 2.0);
      }
    } else if (r.cls == PC_MAXPY && j <= k && j < km) {
      by += 8.0 * n * (j + 3);
      fl += 2.0 * n * (j + 1) + n;
    } else if (r.cls == PC_XUPD) {
      by += 16.0 * n + 8.0 * n * k;
      fl += 2.0 * n * k + n;
    }
  }
  *bytes = by;
  *flops = fl;
}

// After a stream synchronization: attribute every pending launch. its_now[i]
// is system i's step total now; the cycle in flight (if any) did its_now -
// cyc_it0 columns.
void batch_prof_settle(gmres_batch_ctx* b) {
  if (!b->prof_on) return;
  std::vector<int> kcol(b->S, 0);
  for (int i = 0; i < b->S; ++i)
    if (b->cyc_kmax[i] >= 0) kcol[i] = b->h_states[i].total_iters - b->cyc_it0[i];
  for (const auto& r : b->pending) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, r.a, r.b);
    double by = r.bytes, fl = r.flops;
    if (by < 0.0) batch_alg_model(b, r, kcol, &by, &fl);
    const int c = (by > 0.0 || r.cls == PC_LSQ) ? r.cls : PC_NOOP;
    b->prof_ms[c] += ms;
    b->prof_cnt[c] += 1;
    b->prof_bytes[c] += by;
    b->prof_flops[c] += fl;
    b->log.push_back({c, r.j, r.tiles, ms, by, fl});
  }
  b->pending.clear();
  b->ev_used = 0;
  std::fill(b->cyc_kmax.begin(), b->cyc_kmax.end(), -1);
}

gmres_status batch_set_grid(gmres_batch_ctx* b, int P, bool pairs) {
  b->P = P;
  b->pairs = pairs;
  b->step = batch_step_kernel_for(b->m, pairs);
  b->layout_active.clear();  // the next solve lays out again
  batch_drop_graphs(b);
  return GMRES_OK;
}

gmres_status batch_launch_cycle(gmres_batch_ctx* b, int KM) {
  const BatchDev d = batch_dev(b);
  const int ndata = batch_stream_grid(b);
  for (int j = 0; j <= KM; ++j) {
    int pr = batch_prof_begin(b, PC_STEP, j);
    b->step<<<b->P, kThreads, b->step_smem, b->stream>>>(b->rowptr, b->col, b->val, b->V, b->ldv, b->w, b->NT, d, j);
    batch_prof_end(b, pr);
    if (j < KM) {
      pr = batch_prof_begin(b, PC_MAXPY, j);
      kb_maxpy<<<ndata + b->S, kThreads, 0, b->stream>>>(b->V, b->ldv, b->w, d, j, ndata);
      batch_prof_end(b, pr);
    }
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return bfail(b, GMRES_ERR_CUDA, std::string("batch launch: ") + cudaGetErrorString(e));
  return GMRES_OK;
}

// One cycle of KM steps: direct launches on the legacy stream, else a CUDA
// graph per KM (kernel arguments are fixed; the layout and the states they
// read live in device memory).
gmres_status batch_run_cycle(gmres_batch_ctx* b, int KM) {
  if (b->stream == nullptr) return batch_launch_cycle(b, KM);
  gmres_batch_ctx::G* hit = nullptr;
  for (auto& g : b->graphs)
    if (g.kmax == KM && g.prof == b->prof_on) hit = &g;
  if (!hit) {
    gmres_batch_ctx::G g{KM, b->prof_on, nullptr, {}, {}};
    if (b->prof_on) {
      g.events.resize(2 * (2 * (size_t)KM + 1));
      for (auto& e : g.events) BCUDA(b, cudaEventCreate(&e));
    }
    b->graphs.push_back(std::move(g));
    hit = &b->graphs.back();
    cudaGraph_t graph = nullptr;
    BCUDA(b, cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    b->cap = hit;
    gmres_status st = batch_launch_cycle(b, KM);
    b->cap = nullptr;
    cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
    if (st == GMRES_OK && e == cudaSuccess) e = cudaGraphInstantiate(&hit->exec, graph, 0);
    if (graph) cudaGraphDestroy(graph);
    if (st != GMRES_OK || e != cudaSuccess || !hit->exec) {
      for (cudaEvent_t ev : hit->events) cudaEventDestroy(ev);
      b->graphs.pop_back();
      return bfail(b, GMRES_ERR_CUDA, std::string("batch cycle graph: ") + cudaGetErrorString(e));
    }
  }
  BCUDA(b, cudaGraphLaunch(hit->exec, b->stream));
  if (b->prof_on)
    for (auto r : hit->recs) {
      r.tiles = *b->h_nact;
      b->pending.push_back(r);
    }
  return GMRES_OK;
}

// Pick the launch shape of the batched step kernel: time one mid-cycle
// batched step (all systems active, on the zeroed basis) for grids of 1, 2
// and 3 CTAs per SM (clamped to the tile count), each with one and with two
// rows per thread, best of two timed repeats each. The states it dirties are
// reset by every solve.
gmres_status batch_autotune(gmres_batch_ctx* b) {
  std::vector<std::pair<int, bool>> cand;
  for (int pr = 0; pr < 2; ++pr)
    for (int k = 1; k <= 3; ++k) {
      const int P = (int)std::min<int64_t>((int64_t)k * b->nsm, b->T);
      if (cand.empty() || cand.back() != std::make_pair(P, pr == 1)) cand.emplace_back(P, pr == 1);
    }
  cudaEvent_t e0, e1;
  BCUDA(b, cudaEventCreate(&e0));
  BCUDA(b, cudaEventCreate(&e1));
  const int j = std::max(1, b->m / 2);
  const std::vector<char> all(b->S, 1);
  float best = 1e30f;
  auto bestc = cand.front();
  gmres_status st = GMRES_OK;
  for (auto c : cand) {
    const int P = c.first;
    batch_set_grid(b, P, c.second);
    if ((st = batch_layout(b, all, 0)) != GMRES_OK) break;
    float t_best = 1e30f;
    for (int rep = 0; rep < 3 && st == GMRES_OK; ++rep) {
      for (int i = 0; i < b->S; ++i) {
        std::memset(&b->h_states[i], 0, sizeof(DevState));
        b->h_states[i].kmax = b->m;
        b->h_states[i].bnorm = b->h_states[i].inv_bnorm = b->h_states[i].cycle_scale = 1.0;
      }
      cudaError_t e = cudaMemcpy(b->states, b->h_states, sizeof(DevState) * b->S, cudaMemcpyHostToDevice);
      if (e == cudaSuccess) e = cudaEventRecord(e0, 0);
      if (e == cudaSuccess) {
        b->step<<<P, kThreads, b->step_smem, 0>>>(b->rowptr, b->col, b->val, b->V, b->ldv, b->w, b->NT,
                                                  batch_dev(b), j);
        e = cudaGetLastError();
      }
      if (e == cudaSuccess) e = cudaEventRecord(e1, 0);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      float ms = 0.f;
      if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
      if (e != cudaSuccess) st = bfail(b, GMRES_ERR_CUDA, std::string("batch autotune: ") + cudaGetErrorString(e));
      if (rep > 0) t_best = std::min(t_best, ms);
    }
    if (st != GMRES_OK) break;
    if (t_best < best) {
      best = t_best;
      bestc = c;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != GMRES_OK) return st;
  return batch_set_grid(b, bestc.first, bestc.second);
}

}  // namespace

extern "C" {

gmres_status gmres_batch_destroy(gmres_batch b) {
  if (!b) return GMRES_OK;
  batch_drop_graphs(b);
  cudaFree(b->rowptr);
  cudaFree(b->col);
  cudaFree(b->val);
  cudaFree(b->V);
  cudaFree(b->w);
  cudaFree(b->bcat);
  cudaFree(b->xcat);
  cudaFree(b->tile_sys);
  cudaFree(b->sys_tile1);
  cudaFree(b->act_tiles);
  cudaFree(b->n_act);
  cudaFree(b->sys_b0);
  cudaFree(b->sys_nslot);
  cudaFree(b->sys_slot0);
  cudaFree(b->smalls_dev);
  cudaFree(b->partials);
  cudaFree(b->tickets);
  cudaFree(b->blk);
  cudaFree(b->states);
  if (b->h_states) cudaFreeHost(b->h_states);
  if (b->h_layout) cudaFreeHost(b->h_layout);
  for (cudaEvent_t e : b->ev_pool) cudaEventDestroy(e);
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
  gmres_batch_ctx* b = new gmres_batch_ctx();
  auto bail = [&](gmres_status st) {
    g_batch_err = b->err;
    gmres_batch_destroy(b);
    return st;
  };
  b->S = count;
  b->m = m_restart;
  b->tol = tol;
  b->max_iter = max_iter;
  b->n.resize(count);
  b->nnz.resize(count);
  b->row0.resize(count);
  b->tile0.resize(count);
  b->ntile.resize(count);
  // validate and concatenate (block-diagonal, each system padded to whole tiles)
  int64_t NT = 0, nnz_tot = 0;
  for (int i = 0; i < count; ++i) {
    const gmres_csr& a = A[i];
    if (a.on_device || !a.rowptr || a.n <= 0 || a.nnz < 0 || (a.nnz > 0 && (!a.col || !a.val))) {
      b->err = "matrix " + std::to_string(i) + ": need host CSR arrays with n > 0";
      return bail(GMRES_ERR_ARG);
    }
    if (a.rowptr[0] != 0 || a.rowptr[a.n] != a.nnz) {
      b->err = "matrix " + std::to_string(i) + ": rowptr[0] must be 0 and rowptr[n] = nnz";
      return bail(GMRES_ERR_ARG);
    }
    for (int64_t r = 0; r < a.n; ++r)
      if (a.rowptr[r + 1] < a.rowptr[r]) {
        b->err = "matrix " + std::to_string(i) + ": rowptr is not nondecreasing";
        return bail(GMRES_ERR_ARG);
      }
    for (int64_t p = 0; p < a.nnz; ++p)
      if (a.col[p] < 0 || a.col[p] >= a.n || !std::isfinite(a.val[p])) {
        b->err = "matrix " + std::to_string(i) + ": column out of range or non-finite value";
        return bail(GMRES_ERR_ARG);
      }
    b->n[i] = a.n;
    b->nnz[i] = a.nnz;
    b->row0[i] = NT;
    b->tile0[i] = NT / kThreads;
    b->ntile[i] = (int64_t)align_up((size_t)a.n, kThreads) / kThreads;
    NT += (int64_t)align_up((size_t)a.n, kThreads);
    nnz_tot += a.nnz;
  }
  if (NT >= (int64_t)INT32_MAX || nnz_tot >= (int64_t)INT32_MAX) {
    b->err = "batch too large for 32-bit indices";
    return bail(GMRES_ERR_ARG);
  }
  b->NT = NT;
  b->T = NT / kThreads;
  b->ldv = NT;
  std::vector<int32_t> rp(NT + 1, 0), cl(std::max<int64_t>(nnz_tot, 1));
  std::vector<double> vl(std::max<int64_t>(nnz_tot, 1));
  b->h_tile_sys.resize(b->T);
  int64_t pos = 0;
  for (int i = 0; i < count; ++i) {
    const gmres_csr& a = A[i];
    const int64_t r0 = b->row0[i], np = b->ntile[i] * kThreads;
    for (int64_t t = b->tile0[i]; t < b->tile0[i] + b->ntile[i]; ++t) b->h_tile_sys[t] = i;
    for (int64_t r = 0; r < np; ++r) {
      if (r < a.n)
        for (int64_t p = a.rowptr[r]; p < a.rowptr[r + 1]; ++p) {
          cl[pos] = (int32_t)(a.col[p] + r0);
          vl[pos] = a.val[p];
          ++pos;
        }
      rp[r0 + r + 1] = (int32_t)pos;
    }
  }
#define BTRY(call)                                                                   \
  do {                                                                               \
    cudaError_t e_ = (call);                                                         \
    if (e_ != cudaSuccess) {                                                         \
      b->err = std::string(#call) + ": " + cudaGetErrorString(e_);                   \
      return bail(e_ == cudaErrorMemoryAllocation ? GMRES_ERR_OOM : GMRES_ERR_CUDA); \
    }                                                                                \
  } while (0)
  BTRY(cudaGetDevice(&b->device));
  BTRY(cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, b->device));
  BTRY(cudaMalloc(&b->rowptr, sizeof(int32_t) * (NT + 1)));
  BTRY(cudaMalloc(&b->col, sizeof(int32_t) * cl.size()));
  BTRY(cudaMalloc(&b->val, sizeof(double) * vl.size()));
  BTRY(cudaMemcpy(b->rowptr, rp.data(), sizeof(int32_t) * (NT + 1), cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(b->col, cl.data(), sizeof(int32_t) * cl.size(), cudaMemcpyHostToDevice));
  BTRY(cudaMemcpy(b->val, vl.data(), sizeof(double) * vl.size(), cudaMemcpyHostToDevice));
  BTRY(cudaMalloc(&b->V, sizeof(double) * (size_t)NT * (m_restart + 1)));
  BTRY(cudaMemset(b->V, 0, sizeof(double) * (size_t)NT * (m_restart + 1)));
  for (double** p : {&b->w, &b->bcat, &b->xcat}) {
    BTRY(cudaMalloc(p, sizeof(double) * NT));
    BTRY(cudaMemset(*p, 0, sizeof(double) * NT));
  }
  BTRY(cudaMalloc(&b->tile_sys, sizeof(int32_t) * b->T));
  BTRY(cudaMemcpy(b->tile_sys, b->h_tile_sys.data(), sizeof(int32_t) * b->T, cudaMemcpyHostToDevice));
  {
    std::vector<int32_t> t1(count);
    for (int i = 0; i < count; ++i) t1[i] = (int32_t)(b->tile0[i] + b->ntile[i]);
    BTRY(cudaMalloc(&b->sys_tile1, sizeof(int32_t) * count));
    BTRY(cudaMemcpy(b->sys_tile1, t1.data(), sizeof(int32_t) * count, cudaMemcpyHostToDevice));
  }
  BTRY(cudaMalloc(&b->act_tiles, sizeof(int32_t) * b->T));
  BTRY(cudaMalloc(&b->n_act, sizeof(int64_t)));
  BTRY(cudaMalloc(&b->sys_b0, sizeof(int32_t) * count));
  BTRY(cudaMalloc(&b->sys_nslot, sizeof(int32_t) * count));
  BTRY(cudaMalloc(&b->sys_slot0, sizeof(int64_t) * count));
  {
    const size_t i32 = sizeof(int32_t) * ((size_t)b->T + 2 * (size_t)count);
    BTRY(cudaMallocHost(&b->h_layout, align_up(i32, 8) + sizeof(int64_t) * ((size_t)count + 1)));
    b->h_act = reinterpret_cast<int32_t*>(b->h_layout);
    b->h_b0 = b->h_act + b->T;
    b->h_ns = b->h_b0 + count;
    b->h_s0 = reinterpret_cast<int64_t*>(b->h_layout + align_up(i32, 8));
    b->h_nact = b->h_s0 + count;
  }
  BTRY(cudaMalloc(&b->tickets, sizeof(unsigned int) * count));
  BTRY(cudaMemset(b->tickets, 0, sizeof(unsigned int) * count));
  // per-system dense state: DevState array + one block of arrays per system
  const int m = m_restart, ld = m + 1;
  b->nvmax = 2 * (m + 1) + 2;
  b->hist_cap = max_iter + m + 1;
  // slots: each CTA of the grid contributes one slot per system its range
  // touches, so at most P + S - 1 slots
  b->total_slots = (int64_t)kBatchMaxCtasPerSm * b->nsm + count + 1;
  BTRY(cudaMalloc(&b->partials, sizeof(double) * (size_t)b->total_slots * b->nvmax));
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
               ocx = take(sizeof(double) * (m + 3)), ohi = take(sizeof(double) * b->hist_cap);
  b->small_stride = off;
  BTRY(cudaMalloc(&b->blk, off * count));
  BTRY(cudaMemset(b->blk, 0, off * count));
  BTRY(cudaMalloc(&b->states, sizeof(DevState) * count));
  BTRY(cudaMallocHost(&b->h_states, sizeof(DevState) * count));
  b->smalls.resize(count);
  for (int i = 0; i < count; ++i) {
    char* base = b->blk + off * i;
    Small& sm = b->smalls[i];
    sm.st = b->states + i;
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
    sm.partials = nullptr;
    sm.raw = nullptr;
    sm.m = m;
    sm.ldh = ld;
    sm.nvmax = b->nvmax;
    sm.hist_cap = b->hist_cap;
  }
  BTRY(cudaMalloc(&b->smalls_dev, sizeof(Small) * count));
  BTRY(cudaMemcpy(b->smalls_dev, b->smalls.data(), sizeof(Small) * count, cudaMemcpyHostToDevice));
  b->step_smem = sizeof(double) * ((size_t)ld * ld + ld);
  b->lsq_smem = sizeof(double) * (size_t)ld * m;
  for (bool pr : {false, true})
    BTRY(cudaFuncSetAttribute(reinterpret_cast<const void*>(batch_step_kernel_for(m, pr)),
                              cudaFuncAttributeMaxDynamicSharedMemorySize, (int)b->step_smem));
  BTRY(cudaFuncSetAttribute(reinterpret_cast<const void*>(kb_lsq), cudaFuncAttributeMaxDynamicSharedMemorySize,
                            (int)b->lsq_smem));
#undef BTRY
  gmres_status st = batch_autotune(b);
  if (st != GMRES_OK) return bail(st);
  b->hist.assign(count, std::vector<double>());
  b->hist_len.assign(count, 0);
  *out = b;
  return GMRES_OK;
}

gmres_status gmres_batch_set_grid(gmres_batch b, int ctas) {
  if (!b) return GMRES_ERR_ARG;
  BCUDA(b, cudaSetDevice(b->device));
  if (ctas == 0) return batch_autotune(b);
  if (ctas < 0 || ctas > batch_max_grid(b))
    return bfail(b, GMRES_ERR_ARG, "ctas must be in [0, " + std::to_string(batch_max_grid(b)) + "]");
  return batch_set_grid(b, ctas, b->pairs);
}

gmres_status gmres_batch_set_rows_per_thread(gmres_batch b, int rows) {
  if (!b) return GMRES_ERR_ARG;
  if (rows != 1 && rows != 2) return bfail(b, GMRES_ERR_ARG, "rows per thread must be 1 or 2");
  return batch_set_grid(b, b->P, rows == 2);
}

gmres_status gmres_batch_get_rows_per_thread(gmres_batch b, int* rows) {
  if (!b || !rows) return GMRES_ERR_ARG;
  *rows = b->pairs ? 2 : 1;
  return GMRES_OK;
}

gmres_status gmres_batch_get_grid(gmres_batch b, int* ctas) {
  if (!b || !ctas) return GMRES_ERR_ARG;
  *ctas = b->P;
  return GMRES_OK;
}

gmres_status gmres_batch_set_stream(gmres_batch b, void* stream) {
  if (!b) return GMRES_ERR_ARG;
  b->stream = reinterpret_cast<cudaStream_t>(stream);
  return GMRES_OK;
}

}  // extern "C"

namespace {

// Shared body of gmres_batch_solve (device vectors) and gmres_batch_solve_host
// (host vectors): the gather into and the scatter out of the padded layout use
// cudaMemcpyDefault, so either kind of pointer works.
gmres_status batch_solve(gmres_batch b, const double* const* bv, double* const* xv, gmres_info* info) {
  if (!bv || !xv) return bfail(b, GMRES_ERR_ARG, "b or x array is NULL");
  for (int i = 0; i < b->S; ++i)
    if (!bv[i] || !xv[i] || (reinterpret_cast<uintptr_t>(bv[i]) & 7) || (reinterpret_cast<uintptr_t>(xv[i]) & 7))
      return bfail(b, GMRES_ERR_ARG, "b[" + std::to_string(i) + "] or x[" + std::to_string(i) +
                                         "] is NULL or not 8-byte aligned");
  BCUDA(b, cudaSetDevice(b->device));
  const auto t0 = std::chrono::steady_clock::now();
  const int S = b->S;
  cudaStream_t sm = b->stream;
  int64_t launches = 0;
  b->pending.clear();
  b->ev_used = 0;
  b->cyc_kmax.assign(S, -1);
  b->cyc_it0.assign(S, 0);
  for (int c = 0; c < GMRES_PROFILE_CLASSES; ++c) {
    b->prof_ms[c] = b->prof_bytes[c] = b->prof_flops[c] = 0.0;
    b->prof_cnt[c] = 0;
  }
  b->log.clear();
  // gather b and x0 into the padded layout (padding rows stay 0 throughout)
  BCUDA(b, cudaMemsetAsync(b->bcat, 0, sizeof(double) * b->NT, sm));
  BCUDA(b, cudaMemsetAsync(b->xcat, 0, sizeof(double) * b->NT, sm));
  for (int i = 0; i < S; ++i) {
    BCUDA(b, cudaMemcpyAsync(b->bcat + b->row0[i], bv[i], sizeof(double) * b->n[i], cudaMemcpyDefault, sm));
    BCUDA(b, cudaMemcpyAsync(b->xcat + b->row0[i], xv[i], sizeof(double) * b->n[i], cudaMemcpyDefault, sm));
  }
  for (int i = 0; i < S; ++i) {
    std::memset(&b->h_states[i], 0, sizeof(DevState));
    b->h_states[i].tol = b->tol;
  }
  BCUDA(b, cudaMemcpyAsync(b->states, b->h_states, sizeof(DevState) * S, cudaMemcpyHostToDevice, sm));
  std::vector<char> active(S, 1);
  gmres_status st = batch_layout(b, active, sm);
  if (st != GMRES_OK) return st;
  const BatchDev d = batch_dev(b);
  const int ngrid = batch_stream_grid(b);
  auto res_model = [&](int mode, double* by, double* fl) {
    *by = *fl = 0.0;
    for (int i = 0; i < S; ++i)
      if (active[i]) {
        const double n = (double)b->n[i], nnz = (double)b->nnz[i];
        *by += (mode == RES_BNORM) ? 8.0 * n : 4.0 * (n + 1) + 12.0 * nnz + 24.0 * n;
        *fl += (mode == RES_BNORM) ? 2.0 * n : 2.0 * nnz + 3.0 * n;
      }
  };
  double rby, rfl;
  res_model(RES_BNORM, &rby, &rfl);
  int pr = batch_prof_begin(b, PC_RES, 0, rby, rfl);
  kb_residual<<<b->P, kThreads, 0, sm>>>(b->rowptr, b->col, b->val, b->bcat, nullptr, nullptr, d, RES_BNORM);
  batch_prof_end(b, pr);
  ++launches;
  BCUDA(b, cudaGetLastError());
  BCUDA(b, cudaMemcpyAsync(b->h_states, b->states, sizeof(DevState) * S, cudaMemcpyDeviceToHost, sm));
  BCUDA(b, cudaStreamSynchronize(sm));
  batch_prof_settle(b);
  std::vector<int> status(S, GMRES_OK), it_prev(S, -1);
  std::vector<double> bnorm(S);
  for (int i = 0; i < S; ++i) {
    bnorm[i] = b->h_states[i].bnorm;
    if (!std::isfinite(bnorm[i])) {
      status[i] = GMRES_ERR_NONFINITE;
      active[i] = 0;
    } else if (bnorm[i] == 0.0) {
      BCUDA(b, cudaMemsetAsync(b->xcat + b->row0[i], 0, sizeof(double) * b->n[i], sm));
      b->h_states[i].rnorm = 0.0;
      active[i] = 0;
    }
    if (!active[i]) {  // retired before the first cycle: no residual, no steps
      b->h_states[i].done = 1;
      b->h_states[i].kmax = -1;
    }
  }
  BCUDA(b, cudaMemcpyAsync(b->states, b->h_states, sizeof(DevState) * S, cudaMemcpyHostToDevice, sm));
  if (active != b->layout_active && (st = batch_layout(b, active, sm)) != GMRES_OK) return st;
  while (*b->h_nact > 0) {
    res_model(RES_RESIDUAL, &rby, &rfl);
    pr = batch_prof_begin(b, PC_RES, 1, rby, rfl);
    kb_residual<<<b->P, kThreads, 0, sm>>>(b->rowptr, b->col, b->val, b->bcat, b->xcat, b->V, d, RES_RESIDUAL);
    batch_prof_end(b, pr);
    ++launches;
    BCUDA(b, cudaGetLastError());
    BCUDA(b, cudaMemcpyAsync(b->h_states, b->states, sizeof(DevState) * S, cudaMemcpyDeviceToHost, sm));
    BCUDA(b, cudaStreamSynchronize(sm));
    batch_prof_settle(b);
    int KM = 0;
    for (int i = 0; i < S; ++i) {
      // a retired system's state was not touched on the device since its retirement
      DevState& hs = b->h_states[i];
      if (active[i]) {
        if (it_prev[i] >= 0 && hs.total_iters == it_prev[i]) {  // every cycle completes >= 1 column
          status[i] = GMRES_ERR_CUDA;
          active[i] = 0;
        } else if (!std::isfinite(hs.rnorm) || hs.nonfinite) {
          status[i] = GMRES_ERR_NONFINITE;
          active[i] = 0;
        } else if (hs.rnorm / bnorm[i] <= b->tol) {
          status[i] = GMRES_OK;
          active[i] = 0;
        } else if (hs.total_iters >= b->max_iter) {
          status[i] = GMRES_MAXITER;
          active[i] = 0;
        }
      }
      if (!active[i]) {
        hs.done = 1;
        hs.kmax = -1;
      } else {
        hs.kmax = std::min(b->m, b->max_iter - hs.total_iters);
        KM = std::max(KM, hs.kmax);
        b->cyc_kmax[i] = hs.kmax;
        b->cyc_it0[i] = hs.total_iters;
        it_prev[i] = hs.total_iters;
      }
    }
    if (KM == 0) break;
    BCUDA(b, cudaMemcpyAsync(b->states, b->h_states, sizeof(DevState) * S, cudaMemcpyHostToDevice, sm));
    if (active != b->layout_active && (st = batch_layout(b, active, sm)) != GMRES_OK) return st;
    if ((st = batch_run_cycle(b, KM)) != GMRES_OK) return st;
    pr = batch_prof_begin(b, PC_LSQ, 0, 0.0, 0.0);
    kb_lsq<<<S, 128, b->lsq_smem, sm>>>(d);
    batch_prof_end(b, pr);
    pr = batch_prof_begin(b, PC_XUPD, 0);
    kb_xupdate<<<ngrid, kThreads, 0, sm>>>(b->V, b->ldv, b->xcat, d);
    batch_prof_end(b, pr);
    launches += 2 * (int64_t)KM + 1 + 2;
    BCUDA(b, cudaGetLastError());
  }
  for (int i = 0; i < S; ++i)
    BCUDA(b, cudaMemcpyAsync(xv[i], b->xcat + b->row0[i], sizeof(double) * b->n[i], cudaMemcpyDefault, sm));
  BCUDA(b, cudaStreamSynchronize(sm));
  const auto t1 = std::chrono::steady_clock::now();
  gmres_status result = GMRES_OK;
  for (int i = 0; i < S; ++i) {
    const DevState& hs = b->h_states[i];
    const int len = std::min(hs.total_iters, b->hist_cap);
    b->hist[i].resize(len);
    b->hist_len[i] = len;
    if (len > 0)
      BCUDA(b, cudaMemcpy(b->hist[i].data(), b->smalls[i].hist, sizeof(double) * len, cudaMemcpyDeviceToHost));
    if (status[i] < 0 && result >= 0) result = (gmres_status)status[i];
    if (status[i] == GMRES_MAXITER && result == GMRES_OK) result = GMRES_MAXITER;
    if (info) {
      gmres_info& in = info[i];
      std::memset(&in, 0, sizeof(in));
      in.iters = hs.total_iters;
      in.restarts = hs.restarts;
      in.status = status[i];
      in.breakdowns = hs.breakdowns;
      in.rel_resid_true = bnorm[i] > 0.0 ? hs.rnorm / bnorm[i] : 0.0;
      in.rel_resid_est = hs.est;
      in.reductions = hs.reductions;
      in.grid_syncs = hs.grid_syncs;
      in.kernel_launches = launches;
      in.seconds = std::chrono::duration<double>(t1 - t0).count();
    }
  }
  if (result < 0) b->err = "a system reported status " + std::to_string((int)result) + " (see its info entry)";
  return result;
}

}  // namespace

extern "C" {

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
  b->prof_on = on != 0;
  return GMRES_OK;
}

gmres_status gmres_batch_launch_log(gmres_batch b, int cap, int* cls, int* step, int64_t* active_tiles, float* ms,
                                    double* alg_flops, int* count) {
  if (!b || cap < 0) return GMRES_ERR_ARG;
  if (count) *count = (int)b->log.size();
  const int k = std::min<int>(cap, (int)b->log.size());
  for (int i = 0; i < k; ++i) {
    const auto& e = b->log[i];
    if (cls) cls[i] = e.cls;
    if (step) step[i] = e.j;
    if (active_tiles) active_tiles[i] = e.tiles;
    if (ms) ms[i] = e.ms;
    if (alg_flops) alg_flops[i] = e.flops;
  }
  return GMRES_OK;
}

gmres_status gmres_batch_profile(gmres_batch b, int cls, double* total_ms, int64_t* launches, double* alg_bytes,
                                 double* alg_flops) {
  if (!b) return GMRES_ERR_ARG;
  if (cls < 0 || cls >= GMRES_PROFILE_CLASSES) return bfail(b, GMRES_ERR_ARG, "profile class out of range");
  if (total_ms) *total_ms = b->prof_ms[cls];
  if (launches) *launches = b->prof_cnt[cls];
  if (alg_bytes) *alg_bytes = b->prof_bytes[cls];
  if (alg_flops) *alg_flops = b->prof_flops[cls];
  return GMRES_OK;
}

gmres_status gmres_batch_history(gmres_batch b, int i, double* buf, int cap, int* len) {
  if (!b || i < 0 || i >= b->S) return GMRES_ERR_ARG;
  if (len) *len = b->hist_len[i];
  if (buf && cap > 0) std::memcpy(buf, b->hist[i].data(), sizeof(double) * std::min(cap, b->hist_len[i]));
  return GMRES_OK;
}

}  // extern "C"
