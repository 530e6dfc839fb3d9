// The one-reduce Arnoldi step kernel (Algorithm 7's loop body with the
// fused reduction of Algorithm 4), templated on the block-dot width, the
// arithmetic and basis storage types and the CSR staging mode. Its
// instantiations are compiled in step_<type>_s<stage>.cu (one translation unit
// per type and staging mode, built in parallel) and reached through
// lsg_steps::step_kernel_*.
#pragma once

#include "common.cuh"

namespace lsg_steps {
// Host stub of the step kernel for restart length m and staging mode (0 off,
// 1 tiles, 2 tile pairs with the block dot's column ring, 3 tiles with their
// basis columns, 4 tile pairs with theirs, 5 tile pairs without the ring, 6
// mode 2 with the fixed-point block dot; 3 and 4 for the BF16 basis only, 6
// for FP64 only); callers cast it to their StepKernel type.
const void* step_kernel_f64_s0(int m);
const void* step_kernel_f64_s1(int m);
const void* step_kernel_f64_s2(int m);
const void* step_kernel_f64_s5(int m);
const void* step_kernel_f64_s6(int m);
const void* step_kernel_f32_s0(int m);
const void* step_kernel_f32_s1(int m);
const void* step_kernel_f32_s2(int m);
const void* step_kernel_f32_s5(int m);
const void* step_kernel_bf16_s0(int m);
const void* step_kernel_bf16_s1(int m);
const void* step_kernel_bf16_s2(int m);
const void* step_kernel_bf16_s5(int m);
const void* step_kernel_bf16_s3(int m);
const void* step_kernel_bf16_s4(int m);
// Modes 3 and 4 are built for the BF16 basis only: the FP64 basis tile does not fit
// beside two resident CTAs, and FP32 cycles ran faster at three CTAs per SM
// reading the basis themselves than at two with it staged. Mode 6 is FP64
// only: mode 2 with the block dot's full columns on the integer pipes
// (exact fixed-point products, tile_pair_dot_rows_fx).
inline const void* step_kernel_f64(int m, int stage) {
  return stage == 6   ? step_kernel_f64_s6(m)
         : stage == 5 ? step_kernel_f64_s5(m)
         : stage == 2 ? step_kernel_f64_s2(m)
         : stage == 1 ? step_kernel_f64_s1(m)
                      : step_kernel_f64_s0(m);
}
inline const void* step_kernel_f32(int m, int stage) {
  return stage == 5   ? step_kernel_f32_s5(m)
         : stage == 2 ? step_kernel_f32_s2(m)
         : stage == 1 ? step_kernel_f32_s1(m)
                      : step_kernel_f32_s0(m);
}
inline const void* step_kernel_bf16(int m, int stage) {
  return stage == 5   ? step_kernel_bf16_s5(m)
         : stage == 4 ? step_kernel_bf16_s4(m)
         : stage == 3 ? step_kernel_bf16_s3(m)
         : stage == 2 ? step_kernel_bf16_s2(m)
         : stage == 1 ? step_kernel_bf16_s1(m)
                      : step_kernel_bf16_s0(m);
}
}  // namespace lsg_steps

namespace {

template <typename VT, typename SV = VT>
using StepKernel = void (*)(const int32_t*, const int32_t*, const VT*, const SV*, int64_t, const SV*, VT*, int64_t,
                            Small, int, int, double*, int, int);

// VT: arithmetic type (and of A's values and w); SV: storage type of the
// basis (VT, or BF16 for GMRES-IR with BF16 storage, widened exactly on load).
// FP32 cycles run three CTAs per SM (FP64: two): the FP32 step is bound by
// memory latency, and the extra resident warps hide more of it (measured on
// the 192^3 27-point GMRES-IR solve: 2.9 -> 3.4 TB/s; four per SM spill and
// lose).
template <int MAXC, typename VT, typename SV = VT, int STAGE = 0>
__global__ void __launch_bounds__(kThreads, (sizeof(VT) == 4 && STAGE != 3 && STAGE != 4) ? 3 : 2)
k_one_reduce_step(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                  const VT* __restrict__ val, const SV* __restrict__ V, int64_t ldv,
                  const SV* __restrict__ u_arg, VT* __restrict__ w, int64_t n, Small s,
                  int j_arg, int use_spmv, double* raw_out, int stage, int stage_cap) {
  __shared__ __align__(16) VT su[2 * kThreads];
  __shared__ __align__(16) VT sw[2 * kThreads];
  __shared__ double red[2 * (kMaxM + 1) + 2];
  __shared__ int s_j, s_tail, s_skip, s_stage_off;
  __shared__ uint64_t s_bar, s_barV;
  __shared__ uint32_t s_extra;
  __shared__ uint32_t s_ex[2 * kWarps];  // STAGE 6: per-warp exponent maxima of u and w
  __shared__ int64_t s_nx[2];            // STAGE 6: the CTA's next unit (by iteration parity)
  DevState* st = s.st;
  if (threadIdx.x == 0) {
    if (raw_out) {
      s_j = j_arg;
      s_tail = 0;
      s_skip = 0;
      s_extra = 0;
    } else {
      s_skip = __ldcg(&st->done);
      s_j = __ldcg(&st->step);
      s_tail = (s_j == __ldcg(&st->kmax));
      s_extra = __ldcg(&st->stall_test) ? 16u : 0u;
    }
  }
  __syncthreads();
  if (s_skip) return;
  // STAGES 3 and 4 copy basis columns of the handle's own basis; the
  // standalone block dot (raw_out) never runs them
  if ((STAGE == 3 || STAGE == 4) && raw_out) return;
  const int j = s_j;
  const bool tail = s_tail;
  const bool spmv = raw_out ? (use_spmv != 0) : !tail;
  const bool need_w = raw_out ? true : !tail;
  const SV* u = raw_out ? u_arg : V + (size_t)j * ldv;

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
  // STAGE 6: 5 + the stored exponent bound of each full column this warp owns
  // and of its remainder half-columns (slots q = 0, 1: half-column wid + 8 q of
  // columns 8 J8 ..), and their FP64 sums
  int kf[MAXC], kfr[2];
  double fr_a[2] = {0.0, 0.0}, fr_c[2] = {0.0, 0.0};
  // STAGE 6: u's limbs go to Small::VL column j against u's stored bound (not
  // for the standalone block dot, whose u is the caller's, nor at the tail,
  // whose column no later step reads)
  const bool put_limbs = STAGE == 6 && !raw_out && !tail;
  const int kf_u = put_limbs ? 5 + (int)max(kFxMinField, __ldcg(s.ecol + j) >> 20) : 0;
#pragma unroll
  for (int c = 0; c < MAXC; ++c) {
    kf[c] = 5 + (int)kFxMinField;
    if constexpr (STAGE == 6) {
      const int k = (threadIdx.x >> 5) + c * kWarps;
      if (c < J8) kf[c] = 5 + (int)max(kFxMinField, __ldcg(s.ecol + k) >> 20);
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    kfr[q] = 5 + (int)kFxMinField;
    if constexpr (STAGE == 6) {
      const int r = (threadIdx.x >> 5) + q * kWarps;
      if (r < 2 * r8) kfr[q] = 5 + (int)max(kFxMinField, __ldcg(s.ecol + J8 * kWarps + (r >> 1)) >> 20);
    }
  }

  const int64_t ntiles = (n + kThreads - 1) / kThreads;
  if constexpr (STAGE != 0) {
    // Staged CSR (STAGE 1: one tile per unit, 2: tile pairs, 5: the same
    // without the block dot's column ring, 6: STAGE 2 with the full columns'
    // products in exact fixed point on the integer pipes; 3: one tile per unit, and the
    // tile's basis columns too; 4: tile pairs and their basis columns): the bulk-copy engine fetches the next unit's rowptr slice,
    // indices and values into shared memory while this one's block dot runs
    // (and, for STAGES 3 and 4, the next unit's basis columns while this
    // one's SpMV runs). The global CSR is never
    // read by this instantiation: a unit whose copy did not arrive in time, or
    // that does not fit the buffer (the host sizes it for the largest unit),
    // sets the stalled flag and contributes a zero SpMV.
    constexpr bool kPairs = STAGE == 2 || STAGE == 4 || STAGE == 5 || STAGE == 6;  // units of two tiles
    constexpr bool kStageV = STAGE == 3 || STAGE == 4;               // basis columns staged too
    const int U = kPairs ? 2 * kThreads : kThreads;
    const int64_t units = (n + U - 1) / U;
    if (spmv) {
      extern __shared__ __align__(16) double dyn[];
      constexpr int kWs = kPairs ? 8 : 14;  // gathers in flight per staged row
      CsrStage<VT> cs;
      cs.rp = reinterpret_cast<int32_t*>(dyn);
      cs.col = cs.rp + (U + 4);
      cs.val = reinterpret_cast<VT*>(cs.col + stage_cap);
      cs.bar = &s_bar;
      cs.cap = stage_cap;
      cs.U = U;
      // STAGES 3 and 4 also stage the unit's basis columns 0 .. j-1 (after the
      // CSR; U values each)
      SV* sV = reinterpret_cast<SV*>(cs.val + stage_cap);
      if (threadIdx.x == 0) {
        s_stage_off = 0;
        mbar_init(&s_bar, 1);
        if (kStageV) mbar_init(&s_barV, 1);
      }
      __syncthreads();
      uint32_t phase = 0, pend_phase = 0, vphase = 0, vpend_phase = 0;
      bool pending = false;   // thread 0: a CSR copy was issued and not yet seen complete (phase pend_phase)
      bool vpending = false;  // the same for the basis copies
      // thread 0: pend_phase (vpend_phase) is that of the copy a failed wait
      // left in flight; no copy is issued after a failed wait, so the first
      // one recorded is the last one
      bool held = false, vheld = false;
      // thread 0: bulk copies of unit tu's slices of basis columns 0 .. j-1
      // (in bounds: ldv is a whole number of tile pairs)
      auto issue_cols = [&](int64_t tu) {
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        const uint32_t bytes = (uint32_t)(U * sizeof(SV));
        mbar_arrive_expect_tx(&s_barV, (uint32_t)j * bytes + s_extra);
        for (int k = 0; k < j; ++k) bulk_g2s(sV + (size_t)k * U, V + (size_t)k * ldv + tu * U, bytes, &s_barV);
      };
      int64_t unit = blockIdx.x;
      if (threadIdx.x == 0 && unit < units) {
        cs.issue(rowptr, col, val, unit, CsrStage<VT>::lo_of(__ldg(rowptr + unit * U)),
                 CsrStage<VT>::hi_of(__ldg(rowptr + unit * U + U)), s_extra);
        pending = true;
        if (kStageV) {
          issue_cols(unit);
          vpending = true;
        }
      }
      int par = 0;
      for (; unit < units; par ^= 1) {
        // The next unit: fixed stride, or (STAGE 6 unless s.fixed_order) the
        // next one not yet taken, from a counter (CTAs that run faster take
        // more units, so the launch does not wait for the slowest one's last
        // units; which CTA sums which unit then varies from run to run); the
        // counter is reset by the CTA that completes the grid reduction.
        int64_t nx = unit + gridDim.x;
        if constexpr (STAGE == 6) {
          if (threadIdx.x == 0) {
            if (!s.fixed_order) nx = (int64_t)gridDim.x + (int64_t)atomicAdd(&st->unit_ctr, 1u);
            s_nx[par] = nx;
          }
        }
        int nlo = 0, nhi = 0;  // thread 0: the next unit's entry range, loaded ahead of its use
        if (threadIdx.x == 0 && nx < units) {
          nlo = CsrStage<VT>::lo_of(__ldg(rowptr + nx * U));
          nhi = CsrStage<VT>::hi_of(__ldg(rowptr + nx * U + U));
        }
        const int64_t row0 = unit * U + threadIdx.x, row1 = row0 + kThreads;
        VT ur0 = VT(0), ur1 = VT(0), wr0 = VT(0), wr1 = VT(0);
        if (row0 < n) ur0 = ld_as<VT>(u + row0);
        if (kPairs && row1 < n) ur1 = ld_as<VT>(u + row1);
        if constexpr (STAGE == 6) {
          // u is basis column j: its limbs, for the block dots of the
          // cycle's later steps (rows past n stay zero)
          if (put_limbs) {
            int2* vl = s.VL + (size_t)j * s.ldl;
            if (row0 < n) vl[row0] = fx_split((double)ur0, kf_u);
            if (row1 < n) vl[row1] = fx_split((double)ur1, kf_u);
          }
        }
        bool staged = !s_stage_off;
        if (staged) {
          staged = mbar_wait_bounded(&s_bar, phase);
          if (!staged) s_stage_off = 1;
        }
        if (threadIdx.x == 0) {
          if (staged) {
            pending = false;
          } else if (pending && !held) {
            pend_phase = phase;
            held = true;
          }
        }
        phase ^= 1u;
        int lo = 0;
        if (staged) {
          lo = CsrStage<VT>::lo_of(cs.rp[0]);
          staged = CsrStage<VT>::hi_of(cs.rp[U]) - lo <= stage_cap;
        }
        if (!staged) atomicExch(&st->stalled, 1);
        if (kPairs) {
          if (staged)
            csr_row2_staged<kWs>(cs.col, cs.val, u, cs.rp[threadIdx.x] - lo, cs.rp[threadIdx.x + 1] - lo,
                                 cs.rp[kThreads + threadIdx.x] - lo, cs.rp[kThreads + threadIdx.x + 1] - lo, wr0,
                                 wr1);
          if (row0 < n) w[row0] = wr0;
          if (row1 < n) w[row1] = wr1;
        } else if (row0 < n) {
          if (staged)
            wr0 = csr_row_staged<kWs>(cs.col, cs.val, u, cs.rp[threadIdx.x] - lo, cs.rp[threadIdx.x + 1] - lo);
          w[row0] = wr0;
        }
        // once every thread is past its SpMV, the buffer takes the next unit
        auto next = [&]() {
          if (threadIdx.x == 0 && nx < units && !s_stage_off) {
            cs.issue(rowptr, col, val, nx, nlo, nhi, s_extra);
            pending = true;
          }
        };
        if constexpr (kStageV) {
          // the unit's basis columns: waited for after the SpMV, refilled for
          // the next unit once every thread is done with them
          auto before = [&]() {
            bool ok = !s_stage_off;
            if (ok) {
              ok = mbar_wait_bounded(&s_barV, vphase);
              if (!ok) {
                s_stage_off = 1;
                atomicExch(&st->stalled, 1);
              }
            }
            if (threadIdx.x == 0) {
              if (ok) {
                vpending = false;
              } else if (vpending && !vheld) {
                vpend_phase = vphase;
                vheld = true;
              }
            }
            vphase ^= 1u;
          };
          auto after = [&]() {
            if (threadIdx.x == 0 && nx < units && !s_stage_off) {
              issue_cols(nx);
              vpending = true;
            }
          };
          if constexpr (kPairs)
            tile_pair_dot_rows_cols<MAXC, SV, VT>(unit, n, SharedCols<SV>{sV, U}, need_w, J8, r8, ur0, wr0, ur1,
                                                  wr1, su, sw, acc_a, acc_c, rem_a, rem_c, sig, dd, next, before,
                                                  after);
          else
            tile_dot_rows_cols<MAXC, SV, VT>(unit, n, SharedCols<SV>{sV, U}, need_w, J8, r8, ur0, wr0, su, sw,
                                             acc_a, acc_c, rem_a, rem_c, sig, dd, next, before, after);
        } else if (kPairs) {
          if constexpr (STAGE == 2)
            // the column slices stream through a per-warp ring behind the
            // CSR buffer
            tile_pair_dot_rows_pf<MAXC, SV>(unit, n, V, ldv, need_w, J8, r8, ur0, wr0, ur1, wr1, su, sw,
                                            reinterpret_cast<SV*>(cs.val + stage_cap), acc_a, acc_c, rem_a, rem_c,
                                            sig, dd, next);
          else if constexpr (STAGE == 6)
            // the same ring over the columns' stored limbs; every column's
            // products on the integer pipes
            tile_pair_dot_rows_fx<MAXC, true, pf_stages<double>(), true>(
                unit, n, reinterpret_cast<const double*>(s.VL), s.ldl, need_w, J8, r8, ur0, wr0, ur1, wr1, su, sw,
                reinterpret_cast<double*>(cs.val + stage_cap), kf, kfr, acc_a, acc_c, fr_a, fr_c, sig, dd, s_ex,
                next);
          else
            tile_pair_dot_rows<MAXC, SV, VT>(unit, n, V, ldv, need_w, J8, r8, ur0, wr0, ur1, wr1, su, sw, acc_a,
                                             acc_c, rem_a, rem_c, sig, dd, next);
        } else {
          tile_dot_rows<MAXC, SV, VT>(unit, n, V, ldv, need_w, J8, r8, ur0, wr0, su, sw, acc_a, acc_c, rem_a,
                                      rem_c, sig, dd, next);
        }
        if constexpr (STAGE == 6)
          unit = s_nx[par];  // written by thread 0 before this unit's barriers
        else
          unit += gridDim.x;
      }
      // no copy may still be landing in shared memory when the CTA moves on
      if (threadIdx.x == 0 && pending) mbar_wait_bounded(&s_bar, pend_phase);
      if (kStageV && threadIdx.x == 0 && vpending) mbar_wait_bounded(&s_barV, vpend_phase);
      __syncthreads();
    } else {
      // no SpMV (the cycle's tail, or a standalone block dot with w given)
      for (int64_t unit = blockIdx.x; unit < units; unit += gridDim.x) {
        const int64_t row0 = unit * U + threadIdx.x, row1 = row0 + kThreads;
        VT ur0 = VT(0), ur1 = VT(0), wr0 = VT(0), wr1 = VT(0);
        if (row0 < n) {
          ur0 = ld_as<VT>(u + row0);
          if (need_w) wr0 = w[row0];
        }
        if (kPairs && row1 < n) {
          ur1 = ld_as<VT>(u + row1);
          if (need_w) wr1 = w[row1];
        }
        if constexpr (STAGE == 6) {
          // the ring sits where the SpMV launches keep it, behind the CSR buffer
          extern __shared__ __align__(16) double dyn6[];
          double* ring = reinterpret_cast<double*>(reinterpret_cast<int32_t*>(dyn6) + (U + 4) + stage_cap) +
                         stage_cap;
          tile_pair_dot_rows_fx<MAXC>(unit, n, V, ldv, need_w,
                                      J8, r8, ur0, wr0, ur1, wr1, su, sw, ring, kf, kfr, acc_a, acc_c, fr_a, fr_c,
                                      sig, dd, s_ex, NoHook{});
        } else if (kPairs)
          tile_pair_dot_rows<MAXC, SV, VT>(unit, n, V, ldv, need_w, J8, r8, ur0, wr0, ur1, wr1, su, sw, acc_a,
                                           acc_c, rem_a, rem_c, sig, dd, NoHook{});
        else
          tile_dot_rows<MAXC, SV, VT>(unit, n, V, ldv, need_w, J8, r8, ur0, wr0, su, sw, acc_a, acc_c, rem_a,
                                      rem_c, sig, dd, NoHook{});
      }
    }
  } else if (ntiles >= 4 * (int64_t)gridDim.x) {
    // Large problems take tiles in pairs (the CSR loads of two rows per thread
    // are in flight together, halving the latency-bound SpMV phases per row);
    // small ones keep one tile per CTA iteration so that every SM gets work.
    const int64_t npairs = (ntiles + 1) / 2;
    for (int64_t pp = blockIdx.x; pp < npairs; pp += gridDim.x)
      tile_pair_block_dot<MAXC, SV, VT>(pp, n, rowptr, col, val, V, ldv, u, u, w, spmv, need_w, J8, r8, su, sw,
                                        acc_a, acc_c, rem_a, rem_c, sig, dd);
  } else {
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x)
      tile_block_dot<MAXC, SV, VT>(t, n, rowptr, col, val, V, ldv, u, u, w, spmv, need_w, J8, r8, su, sw, acc_a,
                                   acc_c, rem_a, rem_c, sig, dd);
  }

  if constexpr (STAGE == 6)
    cta_partials_fx<MAXC>(acc_a, acc_c, fr_a, fr_c, sig, dd, j, J8, r8, red);
  else
    cta_partials<MAXC, VT>(acc_a, acc_c, rem_a, rem_c, sig, dd, j, J8, r8, red);
  const int nv = 2 * j + 2;
  if (!grid_reduce_last(s, red, nv)) return;
  if (STAGE == 6 && threadIdx.x == 0) st->unit_ctr = 0u;  // every CTA has taken its last unit

  if (raw_out) {
    for (int v = threadIdx.x; v < nv; v += blockDim.x) raw_out[v] = red[v];
    return;
  }

  epilogue_one_reduce(s, red, j, tail);
}

// MAXC = floor(m / 8) whole columns per warp (j <= m), at least 1; STAGE as
// in k_one_reduce_step.
template <typename VT, typename SV, int STAGE>
StepKernel<VT, SV> step_kernel_staged(int m) {
  switch (std::max(1, m / kWarps)) {
    case 1: return k_one_reduce_step<1, VT, SV, STAGE>;
    case 2: return k_one_reduce_step<2, VT, SV, STAGE>;
    case 3: return k_one_reduce_step<3, VT, SV, STAGE>;
    case 4: return k_one_reduce_step<4, VT, SV, STAGE>;
    case 5: return k_one_reduce_step<5, VT, SV, STAGE>;
    case 6: return k_one_reduce_step<6, VT, SV, STAGE>;
    case 7: return k_one_reduce_step<7, VT, SV, STAGE>;
    case 8: return k_one_reduce_step<8, VT, SV, STAGE>;
    case 9: case 10: case 11: case 12: return k_one_reduce_step<12, VT, SV, STAGE>;
    default: return k_one_reduce_step<16, VT, SV, STAGE>;
  }
}

}  // namespace
