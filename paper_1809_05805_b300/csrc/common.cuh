// Device code shared by the single-system solver (lsgmres.cu, step.cuh) and the
// batched engine (batch.cu, engine_step.cuh): constants, the per-system state,
// CSR rows (from global memory, or staged in shared memory by bulk copies
// with mbarrier completion), the fused tile block dot, the deterministic grid
// reduction, and the small dense epilogues of one-reduce MGS-GMRES (Algorithm 7
// on Algorithm 4, Sections II-IV of Swirydowicz et al., arXiv:1809.05805).
// Internal linkage: each translation unit gets its own copy.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <type_traits>

namespace {

constexpr int kThreads = 256;                // CTA size; also rows per tile
constexpr int kWarps = kThreads / 32;        // 8
constexpr int kRowsPerLane = kThreads / 32;  // rows of a tile handled by one lane in the dot phase
constexpr int kRemBatch = 4;                 // remainder columns of the block dot loaded together
constexpr int kGridGroup = 16;               // CTAs per group of a two-level grid reduction
constexpr int kGridGroupsMax = 32;           // groups a two-level grid reduction supports (grids <= 512)
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
  unsigned int gticket[kGridGroupsMax];  // per CTA group, two-level grid reductions
  int fresh;           // batched engine: the next residual pass also sets bnorm
  int pipe2;           // Givens rotations on column pairs (the L = 2 pipeline)
  int stalled;         // a bounded device-side wait for staged CSR data gave up
  int stall_test;      // testing: staged copies announce 16 bytes more than they bring
  unsigned int unit_ctr;  // step kernel (mode 6): units handed out beyond the first per CTA; 0 between launches
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
  // m + 2: per basis column, the largest (hi word & 0x7FF00000) its writer
  // stored (atomicMax; cleared at each cycle start): the bound of the
  // fixed-point block dot. Unused (may be NULL) elsewhere.
  unsigned int* ecol;
  // Staging mode 6: the basis columns as fixed-point limbs (fx_split against
  // the column's stored bound ecol[k]), m + 1 columns of leading dimension
  // ldl. The step kernel writes column j when it is the step's u; later steps'
  // block dots read the limbs instead of splitting the FP64 values again.
  // NULL (and unused) elsewhere.
  int2* VL;
  int64_t ldl;
  // Staging mode 6: 1 assigns tile pairs to CTAs by a fixed stride (results
  // bitwise reproducible for a given grid), 0 hands them out by a counter.
  int fixed_order;
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

// The same over 16 slots: four halving levels on lane bits 3..0, then one add
// across bit 4 (16 adds instead of 31); lanes l and l + 16 both return the
// warp total of slot l mod 16. Fixed order: bitwise reproducible.
template <typename T>
__device__ __forceinline__ T warp_reduce_scatter16(T* v) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) {
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < o; ++i) {
      const T send = up ? v[i] : v[i + o];
      const T keep = up ? v[i + o] : v[i];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
  return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
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

// Load a stored value through the read-only path, widened to the compute type
// CT (the identity when the storage type is CT; BF16 storage widens exactly).
template <typename CT, typename ST>
__device__ __forceinline__ CT ld_as(const ST* p) {
  return (CT)__ldg(p);
}
template <>
__device__ __forceinline__ float ld_as<float, __nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(__ldg(p));
}

// Row i of A times x (CSR, FMA chain in column order, in the type of val; x
// may be stored narrower). The loads of up to 8 entries are issued together
// (predicated), so a stencil row costs two dependent memory latencies
// (indices, then the gather) instead of two per entry. Longer rows are taken
// in rounds of 8 with the index and value loads of the next round issued
// beside the gathers of the current one, so that a row of R rounds costs R + 1
// latencies instead of 2 R.
template <typename VT, typename XT>
__device__ __forceinline__ VT csr_row(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                          const VT* __restrict__ val, const XT* __restrict__ x,
                                          int64_t i) {
  constexpr int kW = 8;
  const int p0 = __ldg(rowptr + i), p1 = __ldg(rowptr + i + 1);
  int c[kW];
  VT v[kW];
#pragma unroll
  for (int e = 0; e < kW; ++e) {
    const bool ok = p0 + e < p1;
    c[e] = ok ? __ldg(col + p0 + e) : 0;
    v[e] = ok ? __ldg(val + p0 + e) : VT(0);
  }
  VT s = VT(0);
  for (int p = p0; p < p1; p += kW) {
    VT xv[kW], vc[kW];
#pragma unroll
    for (int e = 0; e < kW; ++e) {
      xv[e] = (p + e < p1) ? ld_as<VT>(x + c[e]) : VT(0);
      vc[e] = v[e];
    }
    const int q = p + kW;
    if (q < p1) {  // next round's indices and values, in flight with this round's gathers
#pragma unroll
      for (int e = 0; e < kW; ++e) {
        const bool ok = q + e < p1;
        c[e] = ok ? __ldg(col + q + e) : 0;
        v[e] = ok ? __ldg(val + q + e) : VT(0);
      }
    }
#pragma unroll
    for (int e = 0; e < kW; ++e)
      if (p + e < p1) s = fma(vc[e], xv[e], s);
  }
  return s;
}

// ---------------------------------------------------------------------------
// CSR staging in shared memory: the bulk-copy (TMA) engine moves a tile's
// rowptr slice, column indices and values into shared memory while the CTA
// works on the previous tile; completion is signalled on an mbarrier
// (transaction bytes). Every wait is bounded.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// Global -> shared bulk copy (16-byte aligned addresses, size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
// Per-thread asynchronous 16-byte copy global -> shared through L2; bytes
// past src_bytes (0..16) are zero-filled and not read. Completion is per
// thread: commit groups, then wait until at most N of them are pending.
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for the phase of the given parity to complete; false after ~1 s
// (2^31 SM clocks) without completion.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  while (!mbar_try_wait(bar, parity))
    if (clock64() - t0 > (1LL << 31)) return false;
  return true;
}

// A CTA's staging buffer for the CSR of one unit of U rows (a tile, U = 256,
// or a tile pair, U = 512): rp holds rowptr[U u .. U u + U + 4), col and val
// hold entries [lo, hi) with lo = rowptr[U u] rounded down and hi =
// rowptr[U u + U] rounded up to a multiple of 4 (16-byte copies), at most cap
// entries. rowptr must be readable up to U * units + 4 entries (padded with
// nnz past n) and col, val up to nnz rounded up to 4. A unit with more than
// cap entries copies rowptr only and is read from global memory.
template <typename VT>
struct CsrStage {
  int32_t* rp;
  int32_t* col;
  VT* val;
  uint64_t* bar;
  int cap;
  int U;
  __device__ static int lo_of(int p) { return p & ~3; }
  __device__ static int hi_of(int p) { return (p + 3) & ~3; }
  // Thread 0: start the copies of unit u with entry range [lo, hi).
  __device__ void issue(const int32_t* g_rp, const int32_t* g_col, const VT* g_val, int64_t u, int lo, int hi,
                        uint32_t extra = 0) const {
    issue_at(g_rp + u * U, g_col, g_val, U, lo, hi, extra);
  }
  // Thread 0: start the copies of a unit of nrows rows whose rowptr slice
  // starts at rp_src (16-byte aligned), with entry range [lo, hi). `extra`
  // bytes are announced on top of the copies' (0 except in the test of the
  // bounded waits, where they never arrive).
  __device__ void issue_at(const int32_t* rp_src, const int32_t* g_col, const VT* g_val, int nrows, int lo, int hi,
                           uint32_t extra = 0) const {
    // order this CTA's earlier shared-memory reads of the buffer before the
    // asynchronous writes into it
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    const uint32_t brp = (uint32_t)(nrows + 4) * 4;
    const bool fits = hi - lo <= cap;
    const uint32_t bcol = fits ? (uint32_t)(hi - lo) * 4u : 0u;
    const uint32_t bval = fits ? (uint32_t)(hi - lo) * (uint32_t)sizeof(VT) : 0u;
    mbar_arrive_expect_tx(bar, brp + bcol + bval + extra);
    bulk_g2s(rp, rp_src, brp, bar);
    if (bcol) {
      bulk_g2s(col, g_col + lo, bcol, bar);
      bulk_g2s(val, g_val + lo, bval, bar);
    }
  }
};

// Row of A times x from staged entries p0 .. p1 (relative to the staged base):
// gathers in rounds of kW issued together, FMA chain in column order (the
// same sums as csr_row).
template <int kW, typename VT, typename XT>
__device__ __forceinline__ VT csr_row_staged(const int32_t* s_col, const VT* s_val, const XT* __restrict__ x,
                                             int p0, int p1) {
  VT s = VT(0);
  for (int p = p0; p < p1; p += kW) {
    VT xv[kW];
#pragma unroll
    for (int e = 0; e < kW; ++e) xv[e] = (p + e < p1) ? ld_as<VT>(x + s_col[p + e]) : VT(0);
#pragma unroll
    for (int e = 0; e < kW; ++e)
      if (p + e < p1) s = fma(s_val[p + e], xv[e], s);
  }
  return s;
}

// Two staged rows with the gathers of both in flight together (rows of up to
// kW entries each; longer rows one after the other).
template <int kW, typename VT, typename XT>
__device__ __forceinline__ void csr_row2_staged(const int32_t* s_col, const VT* s_val, const XT* __restrict__ x,
                                                int a0, int b0, int a1, int b1, VT& y0, VT& y1) {
  if (b0 - a0 <= kW && b1 - a1 <= kW) {
    VT x0[kW], x1[kW];
#pragma unroll
    for (int e = 0; e < kW; ++e) {
      x0[e] = (a0 + e < b0) ? ld_as<VT>(x + s_col[a0 + e]) : VT(0);
      x1[e] = (a1 + e < b1) ? ld_as<VT>(x + s_col[a1 + e]) : VT(0);
    }
    VT s0 = VT(0), s1 = VT(0);
#pragma unroll
    for (int e = 0; e < kW; ++e) {
      if (a0 + e < b0) s0 = fma(s_val[a0 + e], x0[e], s0);
      if (a1 + e < b1) s1 = fma(s_val[a1 + e], x1[e], s1);
    }
    y0 = s0;
    y1 = s1;
  } else {
    y0 = csr_row_staged<kW>(s_col, s_val, x, a0, b0);
    y1 = csr_row_staged<kW>(s_col, s_val, x, a1, b1);
  }
}

// Rows r0 and r1 of A times x with the loads of both rows in flight together
// (rows of up to 8 entries; longer rows use csr_row). Rows >= n give 0.
template <typename VT, typename XT>
__device__ __forceinline__ void csr_row2(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                         const VT* __restrict__ val, const XT* __restrict__ x,
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
      x0[e] = (a0 + e < b0) ? ld_as<VT>(x + c0[e]) : VT(0);
      x1[e] = (a1 + e < b1) ? ld_as<VT>(x + c1[e]) : VT(0);
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
      // this thread's slots seg, seg + S, ... in chunks of 16: the chunk's
      // loads issued together, then summed as a fixed pairwise tree (four
      // dependent FP64 adds instead of sixteen), the chunks in order
      constexpr int C = 16;
      for (int b0 = seg; b0 < nslot; b0 += C * S) {
        double x[C];
#pragma unroll
        for (int i = 0; i < C; ++i) {
          const int b = b0 + i * S;
          x[i] = b < nslot ? __ldcg(partials + (size_t)(slot0 + b) * nvmax + v) : 0.0;
        }
#pragma unroll
        for (int h = C / 2; h > 0; h >>= 1)
#pragma unroll
          for (int i = 0; i < h; ++i) x[i] += x[i + h];
        acc += x[0];
      }
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
// The last CTA sums the slots with S threads per value; when that leaves more
// than 64 slots per thread (many CTAs and many values: each thread's loads
// come in rounds of 16, one round per chunk sum), the reduction takes two
// levels instead: the last CTA of each group of 16
// consecutive CTAs sums its group's slots into row P + group, and the last
// group sums the group rows. Both levels sum in a fixed order (deterministic
// for a given grid). Needs P + ceil(P / 16) rows of partials.
__device__ bool grid_reduce_last(Small s, double* red, int nv, int nctas = 0) {
  const int P = nctas > 0 ? nctas : (int)gridDim.x;  // CTAs taking part (the first nctas of the grid)
  int S = 1;
  while (2 * S * nv <= (int)blockDim.x && S < (int)blockDim.x) S *= 2;
  const int NG = (P + kGridGroup - 1) / kGridGroup;
  if ((P + S - 1) / S <= 64 || NG > kGridGroupsMax) {
    if (!publish_and_reduce(s.partials, s.nvmax, blockIdx.x, 0, P, &s.st->ticket, red, nv)) return false;
  } else {
    const int g = (int)blockIdx.x / kGridGroup, g0 = g * kGridGroup;
    const int gn = (P - g0 < kGridGroup) ? P - g0 : kGridGroup;
    if (!publish_and_reduce(s.partials, s.nvmax, blockIdx.x, g0, gn, &s.st->gticket[g], red, nv)) return false;
    if (!publish_and_reduce(s.partials, s.nvmax, P + g, P, NG, &s.st->ticket, red, nv)) return false;
  }
  if (threadIdx.x == 0) atomicAdd(reinterpret_cast<unsigned long long*>(&s.st->reductions), 1ull);
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
  // state written by other CTAs of the same launch (the one-launch cycle) is
  // read through L2 (__ldcg): their writes are not visible in this SM's L1
  for (int i = threadIdx.x; i <= j + 1; i += blockDim.x) sh_col[i] = __ldcg(&s.H[(size_t)j * ld + i]);
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    sh_c[i] = __ldcg(&s.cs[i]);
    sh_s[i] = __ldcg(&s.sn[i]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    DevState* st = s.st;
    // every global input first: the stores below may alias them, so a load
    // placed after a store would wait for it
    const double gj = __ldcg(&s.g[j]);
    const double cyc_scale = __ldcg(&st->cycle_scale), inv_bnorm = __ldcg(&st->inv_bnorm), tol = __ldcg(&st->tol);
    const int it0 = __ldcg(&st->total_iters);
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
    s.g[j + 1] = -sn * gj;
    s.g[j] = c * gj;
    const double est = fabs(sn * gj) * cyc_scale * inv_bnorm;
    const int it = it0 + j;
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
    } else if (est <= tol) {
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

// What prerotate_column leaves for finish_prerotated (in the caller's shared
// memory): the column's squared norm so far, rotated entry c, and the scalars
// the finish reads (fixed for the rest of the cycle), so that the finish
// itself reads nothing but h from global memory.
struct PreRot {
  double hn2, rc, gj, cyc_scale, inv_bnorm, tol;
  int it0;
};

// finish_column in two parts, for a caller that knows column c's first c+1
// entries one step before its last one (the one-launch cycle): prerotate_column
// applies the stored rotations 0 .. c-1 to H(0:c, c) and keeps the result in
// Rg(:, c) (rows 0 .. c, row c not yet final), and the column's squared norm
// and rotated entry c in *pr; finish_prerotated then forms rotation c from
// that entry and h = H(c+1, c), as finish_column does, with the same
// operations in the same order (bitwise the same results). Thread 0 works; the
// whole CTA calls both.
__device__ void prerotate_column(Small s, int c, PreRot* pr) {
  __shared__ double sh_col[kMaxM + 2], sh_c[kMaxM + 1], sh_s[kMaxM + 1];
  const int ld = s.ldh;
  for (int i = threadIdx.x; i <= c; i += blockDim.x) sh_col[i] = __ldcg(&s.H[(size_t)c * ld + i]);
  for (int i = threadIdx.x; i < c; i += blockDim.x) {
    sh_c[i] = __ldcg(&s.cs[i]);
    sh_s[i] = __ldcg(&s.sn[i]);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    DevState* st = s.st;
    pr->gj = __ldcg(&s.g[c]);  // g(c) is final once rotation c-1 is
    pr->cyc_scale = __ldcg(&st->cycle_scale);
    pr->inv_bnorm = __ldcg(&st->inv_bnorm);
    pr->tol = __ldcg(&st->tol);
    pr->it0 = __ldcg(&st->total_iters);
    double hn2 = 0.0;
    for (int i = 0; i <= c; ++i) hn2 += sh_col[i] * sh_col[i];
    pr->hn2 = hn2;
    double* R = sh_col;
    for (int i = 0; i < c; ++i) {
      const double cc = sh_c[i], sn = sh_s[i];
      const double t = cc * R[i] + sn * R[i + 1];
      R[i + 1] = -sn * R[i] + cc * R[i + 1];
      R[i] = t;
    }
    double* Rg = s.Rg + (size_t)c * ld;
    for (int i = 0; i <= c; ++i) Rg[i] = R[i];
    pr->rc = R[c];
  }
  __syncthreads();
}

// *pr from prerotate_column (the same thread 0); h = H(c+1, c). Returns the
// stop decision in every thread, as finish_column.
__device__ int finish_prerotated(Small s, int c, double h, const PreRot* pr, bool last_allowed) {
  __shared__ int s_res;
  if (threadIdx.x == 0) {
    DevState* st = s.st;
    const int ld = s.ldh;
    double* Rg = s.Rg + (size_t)c * ld;
    const double hn2 = pr->hn2 + h * h;
    const double gj = pr->gj;
    double R0 = pr->rc, R1 = h;
    double cc = 1.0, sn = 0.0;
    if (R1 != 0.0) {
      const double irho = 1.0 / hypot(R0, R1);
      cc = R0 * irho;
      sn = R1 * irho;
    }
    Rg[c] = cc * R0 + sn * R1;
    Rg[c + 1] = 0.0;
    s.cs[c] = cc;
    s.sn[c] = sn;
    s.g[c + 1] = -sn * gj;
    s.g[c] = cc * gj;
    const double est = fabs(sn * gj) * pr->cyc_scale * pr->inv_bnorm;
    const int it = pr->it0 + c;
    if (it < s.hist_cap) s.hist[it] = est;
    st->k = c + 1;
    st->est = est;
    int stop = 0;
    if (!isfinite(est)) {
      st->nonfinite = 1;
      stop = 1;
    } else if (h <= kBreakdownFactor * kEps * sqrt(hn2)) {
      st->breakdown = 1;
      stop = 1;
    } else if (est <= pr->tol) {
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

// Column c of H is complete (h = H(c+1, c)). Normally it is rotated at once
// (finish_column). In the L = 2 pipeline (Algorithm 8, st->pipe2) column 0 is
// rotated alone and afterwards columns are rotated in pairs: an odd column
// waits for the next even one, unless it is the cycle's last (tail) or its
// new direction vanished (breakdown test on the unrotated column), in which
// case everything pending is rotated now. Returns the stop decision of the
// last rotation (0 when nothing was rotated). Run by the whole CTA.
__device__ int finish_completed(Small s, int c, double h, bool tail) {
  DevState* st = s.st;
  if (!__ldcg(&st->pipe2)) return finish_column(s, c, h, tail);
  __shared__ double sbuf[kWarps];
  __shared__ int s_rot, s_first;
  double v = 0.0;
  for (int i = threadIdx.x; i <= c + 1; i += blockDim.x) {
    const double x = (i == c + 1) ? h : __ldcg(&s.H[(size_t)c * s.ldh + i]);
    v = fma(x, x, v);
  }
  const double hn2 = block_sum(v, sbuf);
  if (threadIdx.x == 0) {
    const bool brk = h <= kBreakdownFactor * kEps * sqrt(hn2);
    s_rot = (c == 0 || (c & 1) == 0 || tail || brk);
    s_first = __ldcg(&st->k);  // columns rotated so far in this cycle
  }
  __syncthreads();
  if (!s_rot) return 0;
  int stop = 0;
  for (int q = s_first; q <= c; ++q) {
    const double hq = (q == c) ? h : __ldcg(&s.H[(size_t)q * s.ldh + q + 1]);
    stop |= finish_column(s, q, hq, tail && q == c);
  }
  return stop;
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
// Where the block dot of a 256-row tile t reads basis column k: GlobalCols
// reads the basis in global memory (row 256 t of column k at V + k ldv + r0);
// SharedCols a copy of the unit's columns in shared memory (column k at
// s + ld_s k).
// ld(k, i) reads entry i of the tile's slice of column k (global memory goes
// through the read-only path, which takes global addresses only; shared
// memory through plain loads).
template <typename SV>
struct GlobalCols {
  const SV* V;
  int64_t ldv;
  int64_t r0;
  template <typename VT>
  __device__ VT ld(int k, int i) const {
    return ld_as<VT>(V + (size_t)k * ldv + r0 + i);
  }
};
template <typename SV>
struct SharedCols {
  const SV* s;
  int ld_s;  // values per staged column slice (the unit's rows)
  template <typename VT>
  __device__ VT ld(int k, int i) const {
    if constexpr (std::is_same<SV, __nv_bfloat16>::value)
      return __bfloat162float(s[(size_t)k * ld_s + i]);
    else
      return (VT)s[(size_t)k * ld_s + i];
  }
};

// The block-dot half of one 256-row tile t, given this thread's row values
// ur = u[row], wr = w[row] (zero for rows >= n): accumulates sigma and d,
// stages u and w of the tile in shared memory, calls hook() once every thread
// of the CTA is past its SpMV (the staged CSR of the tile is no longer read)
// and before() ahead of the first basis read, then splits the block dot over
// the 8 warps: warp w owns columns w, w+8, ... over all 8 row groups, and the
// r8 = j mod 8 remainder columns are split by rows; after() runs once every
// thread is done with the tile's basis columns.
struct NoHook {
  __device__ void operator()() const {}
};
template <int MAXC, typename SV, typename VT, typename Cols, typename Hook, typename Before, typename After>
__device__ __forceinline__ void tile_dot_rows_cols(int64_t t, int64_t n, Cols cols, bool need_w, int J8, int r8,
                                                   VT ur, VT wr, VT* su, VT* sw, VT (&acc_a)[MAXC],
                                                   VT (&acc_c)[MAXC], VT (&rem_a)[kWarps - 1],
                                                   VT (&rem_c)[kWarps - 1], VT& sig, VT& dd, Hook hook,
                                                   Before before, After after) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row = t * kThreads + threadIdx.x;
  sig = fma(ur, ur, sig);
  dd = fma(ur, wr, dd);
  su[threadIdx.x] = ur;
  sw[threadIdx.x] = wr;
  __syncthreads();
  hook();
  before();
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
      VT x[kRowsPerLane];
#pragma unroll
      for (int q = 0; q < kRowsPerLane; ++q)
        x[q] = (base + 32 * q < n) ? cols.template ld<VT>(k, lane + 32 * q) : VT(0);
#pragma unroll
      for (int q = 0; q < kRowsPerLane; ++q) acc_a[c] = fma(x[q], ru[q], acc_a[c]);
      if (need_w) {  // the cycle's tail needs only V^T u
#pragma unroll
        for (int q = 0; q < kRowsPerLane; ++q) acc_c[c] = fma(x[q], rw[q], acc_c[c]);
      }
    }
  }
  // The r8 remainder columns, four at a time: their loads are issued together
  // (one memory latency per four columns instead of one per column).
#pragma unroll
  for (int c0 = 0; c0 < kWarps - 1; c0 += kRemBatch) {
    if (c0 < r8) {  // block-uniform
      VT x[kRemBatch];
#pragma unroll
      for (int b = 0; b < kRemBatch; ++b) {
        const int c = c0 + b;
        x[b] = (c < r8 && row < n) ? cols.template ld<VT>(J8 * kWarps + c, (int)threadIdx.x) : VT(0);
      }
#pragma unroll
      for (int b = 0; b < kRemBatch; ++b) {
        const int c = c0 + b;
        if (c < kWarps - 1 && c < r8) {
          rem_a[c] = fma(x[b], ur, rem_a[c]);
          if (need_w) rem_c[c] = fma(x[b], wr, rem_c[c]);
        }
      }
    }
  }
  __syncthreads();
  after();
}

// The block-dot half of one tile with the basis read from global memory.
template <int MAXC, typename SV, typename VT, typename Hook>
__device__ __forceinline__ void tile_dot_rows(int64_t t, int64_t n, const SV* __restrict__ V, int64_t ldv,
                                              bool need_w, int J8, int r8, VT ur, VT wr, VT* su, VT* sw,
                                              VT (&acc_a)[MAXC], VT (&acc_c)[MAXC], VT (&rem_a)[kWarps - 1],
                                              VT (&rem_c)[kWarps - 1], VT& sig, VT& dd, Hook hook) {
  tile_dot_rows_cols<MAXC, SV, VT>(t, n, GlobalCols<SV>{V, ldv, t * kThreads}, need_w, J8, r8, ur, wr, su, sw,
                                   acc_a, acc_c, rem_a, rem_c, sig, dd, hook, NoHook{}, NoHook{});
}

// The block-dot half of the tile pair pp (rows 512 pp .. 512 pp + 511, two
// per thread: row0 = 512 pp + tid and row1 = row0 + 256), as tile_dot_rows_cols;
// cols.ld(k, i) reads row 512 pp + i of column k. su, sw hold 512 values.
template <int MAXC, typename SV, typename VT, typename Cols, typename Hook, typename Before, typename After>
__device__ __forceinline__ void tile_pair_dot_rows_cols(int64_t pp, int64_t n, Cols cols, bool need_w, int J8,
                                                        int r8, VT ur0, VT wr0, VT ur1, VT wr1, VT* su, VT* sw,
                                                        VT (&acc_a)[MAXC], VT (&acc_c)[MAXC],
                                                        VT (&rem_a)[kWarps - 1], VT (&rem_c)[kWarps - 1], VT& sig,
                                                        VT& dd, Hook hook, Before before, After after) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row0 = pp * (2 * kThreads) + threadIdx.x, row1 = row0 + kThreads;
  sig = fma(ur0, ur0, sig);
  dd = fma(ur0, wr0, dd);
  sig = fma(ur1, ur1, sig);
  dd = fma(ur1, wr1, dd);
  su[threadIdx.x] = ur0;
  sw[threadIdx.x] = wr0;
  su[kThreads + threadIdx.x] = ur1;
  sw[kThreads + threadIdx.x] = wr1;
  __syncthreads();
  hook();
  before();
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
        VT x[kRowsPerLane];
#pragma unroll
        for (int q = 0; q < kRowsPerLane; ++q)
          x[q] = (base + 32 * q < n) ? cols.template ld<VT>(k, h * kThreads + lane + 32 * q) : VT(0);
#pragma unroll
        for (int q = 0; q < kRowsPerLane; ++q) acc_a[c] = fma(x[q], ru[q], acc_a[c]);
        if (need_w) {  // the cycle's tail needs only V^T u
#pragma unroll
          for (int q = 0; q < kRowsPerLane; ++q) acc_c[c] = fma(x[q], rw[q], acc_c[c]);
        }
      }
    }
  }
  // The r8 remainder columns, four at a time (loads issued together).
#pragma unroll
  for (int c0 = 0; c0 < kWarps - 1; c0 += kRemBatch) {
    if (c0 < r8) {  // block-uniform
      VT x0[kRemBatch], x1[kRemBatch];
#pragma unroll
      for (int b = 0; b < kRemBatch; ++b) {
        const int c = c0 + b;
        x0[b] = (c < r8 && row0 < n) ? cols.template ld<VT>(J8 * kWarps + c, (int)threadIdx.x) : VT(0);
        x1[b] = (c < r8 && row1 < n) ? cols.template ld<VT>(J8 * kWarps + c, kThreads + (int)threadIdx.x) : VT(0);
      }
#pragma unroll
      for (int b = 0; b < kRemBatch; ++b) {
        const int c = c0 + b;
        if (c < kWarps - 1 && c < r8) {
          rem_a[c] = fma(x0[b], ur0, rem_a[c]);
          rem_a[c] = fma(x1[b], ur1, rem_a[c]);
          if (need_w) {
            rem_c[c] = fma(x0[b], wr0, rem_c[c]);
            rem_c[c] = fma(x1[b], wr1, rem_c[c]);
          }
        }
      }
    }
  }
  __syncthreads();
  after();
}

// The tile pair pp with the basis (FP64, FP32 or BF16) read from global memory
// through a per-warp ring of pf_stages<SV>() column slices in shared memory,
// filled by per-thread asynchronous 16-byte copies pf_stages - 1 columns ahead
// of use: the bytes in flight cost shared memory instead of registers (with
// register loads a lane kept one column's 8 loads in flight). Each lane
// copies and reads only its own rows (half h: rows 256 h + 32 R q + R lane +
// e, R = 16 / sizeof(SV) rows per copy, q < 8 / R, e < R), so no barrier
// orders the ring; a slot is refilled only after the FMAs that consumed it
// were issued. Rows >= n are zero-filled. Same sums as tile_pair_dot_rows in
// another row order; the remainder columns are read directly as there.
// ring: kWarps * pf_stages<SV>() * 256 values of SV (24 KB for FP32 and BF16,
// 48 KB for FP64).
template <typename SV>
__host__ __device__ constexpr int pf_stages() { return sizeof(SV) == 2 ? 6 : 3; }
template <typename SV>
__host__ __device__ constexpr size_t pf_ring_bytes() { return (size_t)kWarps * pf_stages<SV>() * kThreads * sizeof(SV); }
template <int MAXC, typename SV, typename VT, typename Hook>
__device__ __forceinline__ void tile_pair_dot_rows_pf(int64_t pp, int64_t n, const SV* __restrict__ V,
                                                      int64_t ldv, bool need_w, int J8, int r8, VT ur0, VT wr0,
                                                      VT ur1, VT wr1, VT* su, VT* sw, SV* ring,
                                                      VT (&acc_a)[MAXC], VT (&acc_c)[MAXC],
                                                      VT (&rem_a)[kWarps - 1], VT (&rem_c)[kWarps - 1], VT& sig,
                                                      VT& dd, Hook hook) {
  constexpr int S = pf_stages<SV>();
  constexpr int R = 16 / (int)sizeof(SV);  // rows per 16-byte copy
  constexpr int NQ = kRowsPerLane / R;     // copies per lane per column half
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t row0 = pp * (2 * kThreads) + threadIdx.x, row1 = row0 + kThreads;
  sig = fma(ur0, ur0, sig);
  dd = fma(ur0, wr0, dd);
  sig = fma(ur1, ur1, sig);
  dd = fma(ur1, wr1, dd);
  su[threadIdx.x] = ur0;
  sw[threadIdx.x] = wr0;
  su[kThreads + threadIdx.x] = ur1;
  sw[kThreads + threadIdx.x] = wr1;
  __syncthreads();
  hook();
  SV* wring = ring + wid * (S * kThreads);
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int64_t hb = pp * (2 * kThreads) + h * kThreads;  // first row of the half
    VT ru[kRowsPerLane], rw[kRowsPerLane];
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      if constexpr (sizeof(VT) == 4) {
#pragma unroll
        for (int e = 0; e < R; e += 4) {
          const int o = h * kThreads + 32 * R * q + R * lane + e;
          const float4 a = *reinterpret_cast<const float4*>(su + o);
          const float4 b = *reinterpret_cast<const float4*>(sw + o);
          ru[R * q + e] = a.x, ru[R * q + e + 1] = a.y, ru[R * q + e + 2] = a.z, ru[R * q + e + 3] = a.w;
          rw[R * q + e] = b.x, rw[R * q + e + 1] = b.y, rw[R * q + e + 2] = b.z, rw[R * q + e + 3] = b.w;
        }
      } else {  // FP64: two rows per copy
        const int o = h * kThreads + 32 * R * q + R * lane;
        const double2 a = *reinterpret_cast<const double2*>(su + o);
        const double2 b = *reinterpret_cast<const double2*>(sw + o);
        ru[R * q] = a.x, ru[R * q + 1] = a.y;
        rw[R * q] = b.x, rw[R * q + 1] = b.y;
      }
    }
    // this lane's rows of column wid + 8 c into ring slot `slot`
    auto issue = [&](int c, int slot) {
      const SV* colp = V + (size_t)(wid + c * kWarps) * ldv;
#pragma unroll
      for (int q = 0; q < NQ; ++q) {
        const int64_t r = hb + 32 * R * q + R * lane;
        const int64_t left = n - r;
        const int bytes = left >= R ? 16 : (left > 0 ? (int)left * (int)sizeof(SV) : 0);
        cp_async16(wring + slot * kThreads + 32 * R * q + R * lane, colp + (bytes ? r : 0), bytes);
      }
    };
#pragma unroll
    for (int c = 0; c < S - 1; ++c) {
      if (c < J8) issue(c, c);  // warp-uniform
      cp_async_commit();
    }
#pragma unroll
    for (int c = 0; c < MAXC; ++c) {
      if (c < J8) {  // warp-uniform
        if (c + S - 1 < J8) issue(c + S - 1, (c + S - 1) % S);
        cp_async_commit();
        cp_async_wait<S - 1>();  // column c's copies are done
        const SV* sl = wring + (c % S) * kThreads;
        VT x[kRowsPerLane];
#pragma unroll
        for (int q = 0; q < NQ; ++q) {
          const uint4 v = *reinterpret_cast<const uint4*>(sl + 32 * R * q + R * lane);
          if constexpr (sizeof(SV) == 8) {
            x[R * q] = __hiloint2double((int)v.y, (int)v.x);
            x[R * q + 1] = __hiloint2double((int)v.w, (int)v.z);
          } else if constexpr (sizeof(SV) == 4) {
            x[R * q] = __uint_as_float(v.x), x[R * q + 1] = __uint_as_float(v.y);
            x[R * q + 2] = __uint_as_float(v.z), x[R * q + 3] = __uint_as_float(v.w);
          } else {  // BF16 widened exactly: its bits are the high half of the FP32 value
            const uint32_t wds[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
            for (int t = 0; t < 4; ++t) {
              x[R * q + 2 * t] = __uint_as_float(wds[t] << 16);
              x[R * q + 2 * t + 1] = __uint_as_float(wds[t] & 0xffff0000u);
            }
          }
        }
#pragma unroll
        for (int i = 0; i < kRowsPerLane; ++i) acc_a[c] = fma(x[i], ru[i], acc_a[c]);
        if (need_w) {
#pragma unroll
          for (int i = 0; i < kRowsPerLane; ++i) acc_c[c] = fma(x[i], rw[i], acc_c[c]);
        }
      }
    }
    cp_async_wait<0>();
  }
  // The r8 remainder columns, four at a time (loads issued together).
#pragma unroll
  for (int c0 = 0; c0 < kWarps - 1; c0 += kRemBatch) {
    if (c0 < r8) {  // block-uniform
      VT x0[kRemBatch], x1[kRemBatch];
#pragma unroll
      for (int b = 0; b < kRemBatch; ++b) {
        const int c = c0 + b;
        const SV* colp = V + (size_t)(J8 * kWarps + c) * ldv;
        x0[b] = (c < r8 && row0 < n) ? ld_as<VT>(colp + row0) : VT(0);
        x1[b] = (c < r8 && row1 < n) ? ld_as<VT>(colp + row1) : VT(0);
      }
#pragma unroll
      for (int b = 0; b < kRemBatch; ++b) {
        const int c = c0 + b;
        if (c < kWarps - 1 && c < r8) {
          rem_a[c] = fma(x0[b], ur0, rem_a[c]);
          rem_a[c] = fma(x1[b], ur1, rem_a[c]);
          if (need_w) {
            rem_c[c] = fma(x0[b], wr0, rem_c[c]);
            rem_c[c] = fma(x1[b], wr1, rem_c[c]);
          }
        }
      }
    }
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// FP64 block dot on the integer pipes (exact fixed-point products).
// ---------------------------------------------------------------------------
// On B300 an SM retires about 1.8 DFMA per clock but 64 IMAD/LOP3/SHF and 25
// 32x32->64-bit IMAD.WIDE, so the FP64 block dot, at 2 DFMA per basis element,
// is bound by the FP64 pipe at ~40% of HBM bandwidth. Here the products of the
// full columns run as integer arithmetic instead, at FP64 accuracy:
//  * each value x of a vector with bound |x| < 2^(f - 1022) (f: a biased
//    exponent at least that of its largest entry) becomes an integer X within
//    one unit of x 2^(58 - f + 1022), |X| <= 2^58, split into two 29-bit limbs
//    X = Xh 2^29 + Xl, Xh signed, Xl >= 0 (the error is at most 2^-58 of the
//    bound, 32 times finer than FP64 rounding of the largest entry);
//  * X Y = Xh Yh 2^58 + (Xh Yl + Xl Yh) 2^29 + Xl Yl: the first two parts are
//    summed exactly in 64-bit integers (three mad.wide.s32 per product), the
//    last (below 2^-58 of the largest product) is dropped;
//  * each lane sums the 16 products of one column over one tile pair exactly,
//    then converts the sum to FP64 once and adds it to its FP64 accumulator.
// The bounds: basis columns carry the largest exponent their writer stored
// (Small::ecol, kept by the residual and MAXPY kernels); u and w get theirs
// per tile pair from the CTA's own rows. The sums differ from FP64 DFMA sums
// only by rounding, within the same classical bounds.
// Record the largest exponent field among the values a warp stored into
// column k (per thread: emax = max over its values of the hi word & 0x7FF00000).
__device__ __forceinline__ void fx_note_max(unsigned int* ecol, int k, uint32_t emax) {
  emax = __reduce_max_sync(0xffffffffu, emax);
  if (ecol && (threadIdx.x & 31) == 0 && emax) atomicMax(ecol + k, emax);
}
__device__ __forceinline__ uint32_t fx_hi_field(double x) { return (uint32_t)__double2hiint(x) & 0x7FF00000u; }

constexpr uint32_t kFxMinField = 64;  // bounds below 2^-958 are raised to it (values that small count as 0)

__device__ __forceinline__ uint32_t fx_field(double x) {
  return ((uint32_t)__double2hiint(x) >> 20) & 0x7FFu;
}

// x -> (Xh, Xl) for the bound of biased exponent f, given kf = 5 + f (the
// right shift that takes x's 63-bit aligned significand to X).
__device__ __forceinline__ int2 fx_split(double x, int kf) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int sh = kf - (int)((hi >> 20) & 0x7FFu);  // >= 5 in bound; >= 69 for zero and subnormals
  // M: the significand with its leading one at bit 62, or, for negative x,
  // its ones' complement ~M = -M - 1; the arithmetic shift then gives
  // floor(M / 2^sh) or -floor(M / 2^sh) - 1, within one unit of x 2^(58 - f + 1022)
  // either way (shifts past 64 give 0 or -1)
  const uint32_t sg = (uint32_t)((int)hi >> 31);
  const uint32_t mh = ((__funnelshift_l(lo, hi, 10) & 0x3FFFFFFFu) | 0x40000000u) ^ sg;
  const long long M = (long long)(((unsigned long long)mh << 32) | (unsigned long long)((lo << 10) ^ sg));
  long long X;
  asm("shr.s64 %0, %1, %2;" : "=l"(X) : "l"(M), "r"(sh));
  // X = Xh 2^29 + Xl with Xh = floor(X / 2^29) in [-2^29, 2^29) and Xl in [0, 2^29)
  return make_int2((int)(X >> 29), (int)((uint32_t)X & 0x1FFFFFFFu));
}

__device__ __forceinline__ long long fx_madw(int a, int b, long long c) {
  long long d;
  asm("mad.wide.s32 %0, %1, %2, %3;" : "=l"(d) : "r"(a), "r"(b), "l"(c));
  return d;
}

// t * 2^e2 rounded to the nearest FP64 value (ties away from zero), |t| < 2^63,
// assembled from the binary64 layout with integer instructions (the FP64
// conversion instructions run at the FP64 pipe's rate on this part). Results
// below the normal range flush to zero, above it give infinity.
__device__ __forceinline__ double fx_to_double(long long t, int e2) {
  if (t == 0) return 0.0;
  const unsigned long long sgn = (unsigned long long)t & 0x8000000000000000ull;
  unsigned long long a = t < 0 ? 0ull - (unsigned long long)t : (unsigned long long)t;
  const int lz = __clzll((long long)a);
  a <<= lz;                                                    // leading one at bit 63
  const unsigned long long m = (a >> 11) + ((a >> 10) & 1ull);  // 53 bits, rounded; 2^53 carries into the exponent
  const int ef = 1022 + 63 - lz + e2;                           // biased exponent - 1 (the significand adds 1)
  if (ef < 0) return __longlong_as_double((long long)sgn);
  if (ef >= 2046) return __longlong_as_double((long long)(0x7ff0000000000000ull | sgn));
  return __longlong_as_double((long long)((((unsigned long long)ef) << 52) + m | sgn));
}

// The FP64 block dot of tile pair pp on the integer pipes, with the same ring
// of column slices as tile_pair_dot_rows_pf. The ring streams half-column
// slices (256 rows of one column): warp w takes both halves of its full
// columns w + 8 c (c < J8) and the remainder half-columns r = w and r = w + 8
// of the r8 = j mod 8 last columns (half-column r: column 8 J8 + r / 2, half
// r mod 2), so that no warp does more than half a column more than another.
// Each lane sums a column's 16 products (8 for a remainder half-column)
// exactly, then converts the sum to FP64 once (one FP64 add per column and
// tile pair). kf[c] = 5 + f of column w + 8 c, kfr[q] of remainder slot q
// (f: its stored exponent bound). The u and w values of the pair are replaced
// in su, sw by their limbs (int2 per row) relative to the pair's own bounds;
// s_ex holds 2 kWarps words. w may be absent (need_w false: the cycle's tail,
// which needs only V^T u); then wr0 = wr1 = 0.
//
// S: ring slices per warp (S - 1 slices in flight ahead of use). RING = false
// (no room for a ring): each lane loads its two rows of a slice directly
// (16-byte loads through the read-only path), and only pair rows in
// [rlo, rhi) (relative to the pair's first row) take part: a unit that is one
// tile of a pair, or a system's ragged end. With the ring, rows past n read as
// zeros and a caller masks rows below n by passing zero u and w there.
//
// LIMBS: V holds each column's limbs already (int2 per row, (Xh, Xl) as
// fx_split gives them against the column's bound; Small::VL), read through the
// same 8-byte-per-row copies, so the per-value split drops out of the loop.
template <int MAXC, bool RING = true, int S = pf_stages<double>(), bool LIMBS = false, typename Hook>
__device__ __forceinline__ void tile_pair_dot_rows_fx(int64_t pp, int64_t n,
                                                      const double* __restrict__ V, int64_t ldv, bool need_w, int J8,
                                                      int r8, double ur0, double wr0, double ur1, double wr1,
                                                      double* su, double* sw, double* ring, const int (&kf)[MAXC],
                                                      const int (&kfr)[2], double (&acc_a)[MAXC],
                                                      double (&acc_c)[MAXC], double (&rem_a)[2],
                                                      double (&rem_c)[2], double& sig, double& dd, uint32_t* s_ex,
                                                      Hook hook, int rlo = 0, int rhi = 2 * kThreads) {
  static_assert(S >= 2, "the ring needs a slice in flight beside the one in use");
  constexpr int R = 2;                    // rows per 16-byte copy
  constexpr int NQ = kRowsPerLane / R;    // copies per lane per slice
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  sig = fma(ur0, ur0, sig);
  dd = fma(ur0, wr0, dd);
  sig = fma(ur1, ur1, sig);
  dd = fma(ur1, wr1, dd);
  // the pair's bounds for u and w: largest exponent field over its 512 rows
  uint32_t eu = max(fx_field(ur0), fx_field(ur1)), ew = max(fx_field(wr0), fx_field(wr1));
  eu = __reduce_max_sync(0xffffffffu, eu);
  ew = __reduce_max_sync(0xffffffffu, ew);
  if (lane == 0) {
    s_ex[wid] = eu;
    s_ex[kWarps + wid] = ew;
  }
  __syncthreads();
  hook();
  uint32_t fu = kFxMinField, fw = kFxMinField;
#pragma unroll
  for (int q = 0; q < kWarps; ++q) {
    fu = max(fu, s_ex[q]);
    fw = max(fw, s_ex[kWarps + q]);
  }
  int2* lu = reinterpret_cast<int2*>(su);
  int2* lw = reinterpret_cast<int2*>(sw);
  lu[threadIdx.x] = fx_split(ur0, 5 + (int)fu);
  lu[kThreads + threadIdx.x] = fx_split(ur1, 5 + (int)fu);
  lw[threadIdx.x] = fx_split(wr0, 5 + (int)fw);
  lw[kThreads + threadIdx.x] = fx_split(wr1, 5 + (int)fw);
  __syncthreads();
  const bool bad = fu == 0x7FFu || fw == 0x7FFu;  // NaN or Inf among the pair's u, w
  // x u = (Xh Uh + (Xh Ul + Xl Uh) / 2^29) 2^(f_x + f_u - 2102): the flush scales
  const int ea = (int)fu - 2102, ec = (int)fw - 2102;
  double* wring = RING ? ring + wid * (S * kThreads) : nullptr;  // this warp's ring slices
  const int nr = (wid < 2 * r8 ? 1 : 0) + (wid + kWarps < 2 * r8 ? 1 : 0);  // remainder half-columns of this warp
  const int nsl = 2 * J8 + nr;  // slices this warp streams
  // column and half of this warp's slice sl
  auto locate = [&](int sl, int& col, int& h) {
    if (sl < 2 * J8) {
      col = wid + (sl >> 1) * kWarps;
      h = sl & 1;
    } else {
      const int r = wid + (sl - 2 * J8) * kWarps;
      col = J8 * kWarps + (r >> 1);
      h = r & 1;
    }
  };
  auto issue = [&](int sl, int slot) {
    int col, h;
    locate(sl, col, h);
    const double* colp = V + (size_t)col * ldv;
    const int64_t hb = pp * (2 * kThreads) + h * kThreads;
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int64_t r = hb + 32 * R * q + R * lane;
      const int64_t left = n - r;
      const int bytes = left >= R ? 16 : (left > 0 ? (int)left * 8 : 0);
      cp_async16(wring + slot * kThreads + 32 * R * q + R * lane, colp + (bytes ? r : 0), bytes);
    }
  };
  // the products of slice sl (half h of a column with shift kfc) into the
  // exact sums ah, am (x u) and ch, cm (x w)
  auto slice = [&](int sl, int h, int kfc, long long& ah, long long& am, long long& ch, long long& cm) {
    const double* slp = nullptr;
    const double* colg = nullptr;
    if constexpr (RING) {
      if (sl + S - 1 < nsl) issue(sl + S - 1, (sl + S - 1) % S);
      cp_async_commit();
      cp_async_wait<S - 1>();  // slice sl's copies are done
      slp = wring + (sl % S) * kThreads;
    } else {
      int col, hh;
      locate(sl, col, hh);
      colg = V + (size_t)col * ldv + pp * (2 * kThreads);
    }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      const int r = h * kThreads + 32 * R * q + R * lane;       // row within the pair
      double2 xv;
      if constexpr (RING) {
        xv = *reinterpret_cast<const double2*>(slp + 32 * R * q + R * lane);
      } else {
        xv = (r >= rlo && r + 1 < rhi) ? __ldg(reinterpret_cast<const double2*>(colg + r)) : make_double2(0.0, 0.0);
        if (r >= rlo && r < rhi && r + 1 >= rhi) xv.x = __ldg(colg + r);  // the range's last row, alone
      }
      const int4 uu = *reinterpret_cast<const int4*>(lu + r);  // limbs of rows r, r + 1
      int2 x0, x1;
      if constexpr (LIMBS) {  // the stored (Xh, Xl) of rows r, r + 1
        x0 = make_int2(__double2loint(xv.x), __double2hiint(xv.x));
        x1 = make_int2(__double2loint(xv.y), __double2hiint(xv.y));
      } else {
        x0 = fx_split(xv.x, kfc);
        x1 = fx_split(xv.y, kfc);
      }
      ah = fx_madw(x0.x, uu.x, ah);
      am = fx_madw(x0.x, uu.y, am);
      am = fx_madw(x0.y, uu.x, am);
      ah = fx_madw(x1.x, uu.z, ah);
      am = fx_madw(x1.x, uu.w, am);
      am = fx_madw(x1.y, uu.z, am);
      if (need_w) {
        const int4 ww = *reinterpret_cast<const int4*>(lw + r);
        ch = fx_madw(x0.x, ww.x, ch);
        cm = fx_madw(x0.x, ww.y, cm);
        cm = fx_madw(x0.y, ww.x, cm);
        ch = fx_madw(x1.x, ww.z, ch);
        cm = fx_madw(x1.x, ww.w, cm);
        cm = fx_madw(x1.y, ww.z, cm);
      }
    }
  };
  auto flush = [&](int kfc, long long ah, long long am, long long ch, long long cm, double& a, double& c) {
    const int fx = kfc - 5;
    const bool nan = bad || fx == 0x7FF;
    const double qnan = __longlong_as_double(0x7ff8000000000000ll);
    a += nan ? qnan : fx_to_double(ah + (am >> 29), ea + fx);
    if (need_w) c += nan ? qnan : fx_to_double(ch + (cm >> 29), ec + fx);
  };
  if constexpr (RING) {
#pragma unroll
    for (int sl = 0; sl < S - 1; ++sl) {
      if (sl < nsl) issue(sl, sl);  // warp-uniform
      cp_async_commit();
    }
  }
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    if (c < J8) {  // warp-uniform
      long long ah = 0, am = 0, ch = 0, cm = 0;
      slice(2 * c, 0, kf[c], ah, am, ch, cm);
      slice(2 * c + 1, 1, kf[c], ah, am, ch, cm);
      flush(kf[c], ah, am, ch, cm, acc_a[c], acc_c[c]);
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    if (q < nr) {  // warp-uniform
      const int r = wid + q * kWarps;
      long long ah = 0, am = 0, ch = 0, cm = 0;
      slice(2 * J8 + q, r & 1, kfr[q], ah, am, ch, cm);
      flush(kfr[q], ah, am, ch, cm, rem_a[q], rem_c[q]);
    }
  }
  // No closing barrier: each thread's ring copies are complete here; the
  // limbs in su, sw and the bounds in s_ex are next written after the next
  // pair's first barrier, which no warp passes before every warp has left
  // this pair's column loop; a caller's own shared state after the call is
  // ordered by its own barriers.
  if constexpr (RING) cp_async_wait<0>();
}

// The CTA's partial sums of the fixed-point block dot (tile_pair_dot_rows_fx):
// red[0:j] = a, red[j:2j] = c, red[2j] = sigma, red[2j+1] = d. Full column
// wid + 8 c comes from warp wid alone; remainder column 8 J8 + q from the two
// warps holding its halves (half-columns 2q and 2q + 1: warps 2q mod 8 and
// 2q + 1 mod 8, slot q / 4), added in that order. Warp totals by the
// butterfly reduce-scatter; fixed order throughout.
template <int MAXC>
__device__ __forceinline__ void cta_partials_fx(double (&acc_a)[MAXC], double (&acc_c)[MAXC], double (&rem_a)[2],
                                                double (&rem_c)[2], double sig, double dd, int j, int J8, int r8,
                                                double* red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int kSlots = 2 * MAXC + 4 + 2;
  constexpr int kChunks = (kSlots + 31) / 32;
  double v[kChunks * 32];
#pragma unroll
  for (int i = 0; i < kChunks * 32; ++i) v[i] = 0.0;
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    v[c] = acc_a[c];
    v[MAXC + c] = acc_c[c];
  }
  v[2 * MAXC] = rem_a[0];
  v[2 * MAXC + 1] = rem_a[1];
  v[2 * MAXC + 2] = rem_c[0];
  v[2 * MAXC + 3] = rem_c[1];
  v[kSlots - 2] = sig;
  v[kSlots - 1] = dd;
  __shared__ double sx[6][kWarps];  // per warp: rem_a[0..1], rem_c[0..1], sigma, d
#pragma unroll
  for (int ch = 0; ch < kChunks; ++ch) {
    const double tot = warp_reduce_scatter32(v + 32 * ch);
    const int slot = 32 * ch + lane;
    if (slot < MAXC) {
      if (slot < J8) red[wid + slot * kWarps] = tot;  // column wid + 8 slot belongs to this warp
    } else if (slot < 2 * MAXC) {
      if (slot - MAXC < J8) red[j + wid + (slot - MAXC) * kWarps] = tot;
    } else if (slot < kSlots) {
      sx[slot - 2 * MAXC][wid] = tot;
    }
  }
  __syncthreads();
  const int t = threadIdx.x;
  if (t < 2 * r8) {  // remainder column q = t mod r8, a (t < r8) or c
    const int q = t < r8 ? t : t - r8;
    const int base = t < r8 ? 0 : 2;  // rem_a or rem_c slots
    const int h0 = 2 * q, h1 = 2 * q + 1;  // its half-columns
    const double x0 = sx[base + h0 / kWarps][h0 % kWarps], x1 = sx[base + h1 / kWarps][h1 % kWarps];
    red[(t < r8 ? 0 : j) + J8 * kWarps + q] = x0 + x1;
  } else if (t == 2 * r8 || t == 2 * r8 + 1) {  // sigma, d: the 8 warps in warp order
    const int k = 4 + (t - 2 * r8);
    double s2 = 0.0;
    for (int w2 = 0; w2 < kWarps; ++w2) s2 += sx[k][w2];
    red[2 * j + (t - 2 * r8)] = s2;
  }
  __syncthreads();
}

// The tile pair with the basis read from global memory.
template <int MAXC, typename SV, typename VT, typename Hook>
__device__ __forceinline__ void tile_pair_dot_rows(int64_t pp, int64_t n, const SV* __restrict__ V, int64_t ldv,
                                                   bool need_w, int J8, int r8, VT ur0, VT wr0, VT ur1, VT wr1,
                                                   VT* su, VT* sw, VT (&acc_a)[MAXC], VT (&acc_c)[MAXC],
                                                   VT (&rem_a)[kWarps - 1], VT (&rem_c)[kWarps - 1], VT& sig,
                                                   VT& dd, Hook hook) {
  tile_pair_dot_rows_cols<MAXC, SV, VT>(pp, n, GlobalCols<SV>{V, ldv, pp * (2 * kThreads)}, need_w, J8, r8, ur0,
                                        wr0, ur1, wr1, su, sw, acc_a, acc_c, rem_a, rem_c, sig, dd, hook, NoHook{},
                                        NoHook{});
}

// One 256-row tile t of the fused SpMV + block dot (one row per thread in the
// SpMV), accumulated into the caller's per-thread sums. Rows >= n count as
// zero. Row i of the SpMV is rowptr[i] .. rowptr[i+1] of col/val, gathering
// xg[col] (a single system passes xg = u; a system stored at rows row0.. of a
// shared arena passes its own CSR shifted by -row0 and xg = u + row0).
template <int MAXC, typename SV, typename VT = SV>
__device__ __forceinline__ void tile_block_dot(int64_t t, int64_t n, const int32_t* __restrict__ rowptr,
                                               const int32_t* __restrict__ col, const VT* __restrict__ val,
                                               const SV* __restrict__ V, int64_t ldv, const SV* __restrict__ u,
                                               const SV* __restrict__ xg, VT* __restrict__ w, bool spmv,
                                               bool need_w, int J8, int r8, VT* su,
                                               VT* sw, VT (&acc_a)[MAXC], VT (&acc_c)[MAXC],
                                               VT (&rem_a)[kWarps - 1], VT (&rem_c)[kWarps - 1], VT& sig,
                                               VT& dd) {
  const int64_t row = t * kThreads + threadIdx.x;
  VT ur = VT(0), wr = VT(0);
  if (row < n) {
    ur = ld_as<VT>(u + row);
    if (spmv) {
      wr = csr_row(rowptr, col, val, xg, row);
      w[row] = wr;
    } else if (need_w) {
      wr = w[row];
    }
  }
  tile_dot_rows<MAXC, SV, VT>(t, n, V, ldv, need_w, J8, r8, ur, wr, su, sw, acc_a, acc_c, rem_a, rem_c, sig, dd,
                              NoHook{});
}

// Tiles 2 pp and 2 pp + 1 (rows 512 pp .. 512 pp + 511) of the fused SpMV +
// block dot, two rows per thread: the CSR loads of both rows are in flight
// together, halving the latency-bound SpMV phases per row. su, sw hold 512
// values.
template <int MAXC, typename SV, typename VT = SV>
__device__ __forceinline__ void tile_pair_block_dot(int64_t pp, int64_t n, const int32_t* __restrict__ rowptr,
                                                    const int32_t* __restrict__ col, const VT* __restrict__ val,
                                                    const SV* __restrict__ V, int64_t ldv, const SV* __restrict__ u,
                                                    const SV* __restrict__ xg, VT* __restrict__ w, bool spmv,
                                                    bool need_w, int J8, int r8,
                                                    VT* su, VT* sw, VT (&acc_a)[MAXC], VT (&acc_c)[MAXC],
                                                    VT (&rem_a)[kWarps - 1], VT (&rem_c)[kWarps - 1], VT& sig,
                                                    VT& dd) {
  const int64_t row0 = pp * (2 * kThreads) + threadIdx.x, row1 = row0 + kThreads;
  VT ur0 = VT(0), wr0 = VT(0), ur1 = VT(0), wr1 = VT(0);
  if (row0 < n) ur0 = ld_as<VT>(u + row0);
  if (row1 < n) ur1 = ld_as<VT>(u + row1);
  if (spmv) {
    csr_row2(rowptr, col, val, xg, row0, row1, n, wr0, wr1);
    if (row0 < n) w[row0] = wr0;
    if (row1 < n) w[row1] = wr1;
  } else if (need_w) {
    if (row0 < n) wr0 = w[row0];
    if (row1 < n) wr1 = w[row1];
  }
  tile_pair_dot_rows<MAXC, SV, VT>(pp, n, V, ldv, need_w, J8, r8, ur0, wr0, ur1, wr1, su, sw, acc_a, acc_c, rem_a,
                                   rem_c, sig, dd, NoHook{});
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
  // value): lane l then holds the warp total of slot l. When every used slot
  // lies below 16, a 16-slot reduce-scatter takes the place of the 32-slot one.
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
  // cross-warp slots q = slot - 2 MAXC: sigma, d, then remainder columns a, c
  // interleaved (so that few remainder columns leave the high slots empty)
  v[2 * MAXC] = sig;
  v[2 * MAXC + 1] = dd;
#pragma unroll
  for (int c = 0; c < kWarps - 1; ++c) {
    v[2 * MAXC + 2 + 2 * c] = rem_a[c];
    v[2 * MAXC + 3 + 2 * c] = rem_c[c];
  }
  __shared__ VT scross[kSlots - 2 * MAXC][kWarps];  // slots summed across warps
  // all used slots below 16: a 16-slot reduce-scatter (16 FP64 adds instead of 31)
  const bool short16 = kSlots > 16 && 2 * MAXC + 2 + 2 * r8 <= 16;
  if (short16) {
    const VT tot = warp_reduce_scatter16(v);
    const int slot = lane;
    if (lane < 16) {
      if (slot < MAXC) {
        if (slot < J8) red[wid + slot * kWarps] = tot;
      } else if (slot < 2 * MAXC) {
        if (slot - MAXC < J8) red[j + wid + (slot - MAXC) * kWarps] = tot;
      } else {
        scross[slot - 2 * MAXC][wid] = tot;
      }
    }
  } else {
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
  }
  __syncthreads();
  // remainder columns and the two norms: sum the 8 warps in warp order
  if ((int)threadIdx.x < 2 + 2 * r8) {
    const int q = threadIdx.x;
    double t2 = 0.0;
    for (int w2 = 0; w2 < kWarps; ++w2) t2 += scross[q][w2];
    if (q < 2) {
      red[2 * j + q] = t2;
    } else {
      const int c = (q - 2) >> 1;
      red[((q - 2) & 1 ? j : 0) + J8 * kWarps + c] = t2;
    }
  }
  __syncthreads();
}

// The one-reduce epilogue (last CTA), given the grid totals red[0 .. 2j+2) of
// step j: lagged norm, completion of column j-1 at the tail, T row, r = T s,
// the new Hessenberg column and the MAXPY coefficients.
__device__ void epilogue_one_reduce(Small s, double* red, int j, bool tail, size_t dyn_off = 0) {
  DevState* st = s.st;
  // ---------------- epilogue (last CTA) ----------------
  // stop: 0 = continue the cycle; 1 = cycle done after the T row (converged
  // or tail); 2 = cycle done now (breakdown, zero or non-finite norm); 3 =
  // exact breakdown found, column j-1 still to be finished (then 2).
  // T (rows and columns 0..j-1) and scale[0..j-1] are staged in shared memory
  // (dynamic, (m+1)^2 + (m+1) doubles from byte dyn_off on) so the O(j^2) work
  // reads no global memory.
  extern __shared__ __align__(16) double dyn[];
  const int ld = s.ldh;
  double* sT = dyn + dyn_off / sizeof(double);  // (m+1) x (m+1), column-major, ld
  double* sScale = sT + (size_t)ld * ld;         // m+1
  __shared__ double s_beta;
  __shared__ int s_stop;
  for (int e = threadIdx.x; e < j * j; e += blockDim.x) {
    const int k = e / j, i = e % j;  // column k, row i
    if (i >= k) sT[(size_t)k * ld + i] = __ldcg(&s.T[(size_t)k * ld + i]);
  }
  for (int i = threadIdx.x; i < j; i += blockDim.x) sScale[i] = __ldcg(&s.scale[i]);
  if (threadIdx.x == 0) {
    atomicAdd(reinterpret_cast<unsigned long long*>(&st->grid_syncs), 1ull);
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
    const int fin = finish_completed(s, j - 1, s_beta, tail);
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

// Back substitution R(0:k,0:k) y = g(0:k) (column-oriented), then the
// coefficients of x += V_k y in the unnormalized basis, and the cycle totals.
// The k x k triangle of the rotated Hessenberg is staged in shared memory
// (dynamic, (m+1) x m doubles) so each of the k sequential steps is a
// shared-memory update, not a global-memory round trip.
__device__ void lsq_system(Small s) {
  extern __shared__ __align__(16) double sR[];
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

// Kernel classes of the per-launch profiles (gmres_profile, gmres_batch_profile).
enum { PC_STEP = 0, PC_MAXPY = 1, PC_MGS_SPMV = 2, PC_MGS_AXPY = 3, PC_RES = 4, PC_LSQ = 5, PC_XUPD = 6,
       PC_NOOP = 7, PC_REORTH = 8, PC_REORTH_MAXPY = 9, PC_CYCLE = 10 };

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace
