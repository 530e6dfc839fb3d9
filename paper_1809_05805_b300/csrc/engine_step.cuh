// The engine's step kernel (Algorithm 7's loop body for every listed system)
// and its instantiation table.
#pragma once

#include "engine.cuh"

namespace {

// The copies of one staged unit: its rowptr slice, the system's indices and
// values, the unit's rows and entry range.
template <typename VT>
struct StageCopy {
  const int32_t* rp;
  const int32_t* col;
  const VT* val;
  int nrows, lo, hi;
};

// Rows of one system's CSR times x, one entry at a time from global memory
// (local row indices; the same FMA order as csr_row): the engine step's path
// for a unit whose staged range exceeds the buffer.
template <typename VT, typename XT>
__device__ __noinline__ VT csr_row_plain(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                         const VT* __restrict__ val, const XT* __restrict__ x, int64_t i) {
  VT s = VT(0);
  for (int p = __ldg(rowptr + i), e = __ldg(rowptr + i + 1); p < e; ++p) s = fma(__ldg(val + p), ld_as<VT>(x + __ldg(col + p)), s);
  return s;
}

// Step j of the current cycle for every listed system: the CTA walks its
// range of listed tiles (pairs of consecutive tiles of one system, two rows
// per thread, when PAIRS); whenever the range moves to another system it
// publishes that system's sums, and the CTA completing a system runs the
// system's reduction and epilogue. Each unit's CSR (rowptr slice, indices,
// values; per-system local indices) is staged in shared memory by bulk copies
// issued while the previous unit's block dot runs (as in the single-system
// step kernel); the epilogue's shared memory follows the staging buffer
// (cap entries), since a system's epilogue can run while the next unit lands.
// Each system's rowptr is padded with nnz to whole tile pairs + 8.
// FP64 cycles on tile pairs with FXM = 1 or 2: the block dot's products as exact
// fixed-point integers on the integer pipes (tile_pair_dot_rows_fx, the
// system's basis exponent bounds from its Small::ecol), as the single-system
// solver's staging mode 6, on the limbs each basis column got at the step
// whose u it was (EngDev::VL); a unit that is one tile of a pair runs as that pair
// with the other tile's rows masked. FXM = 1 loads the basis directly;
// FXM = 2 streams it through a per-warp ring of kEngRing half-column slices
// filled by cp.async, placed over the epilogue's shared memory (the epilogue
// runs between units, the ring only inside a unit's block dot, which waits
// for all of its copies before it returns). FP32 cycles on tile pairs with
// FXM = 3: FMA products with the basis through the single-system kernels'
// column ring (tile_pair_dot_rows_pf, pf_stages<float>() column slices per
// warp), laid over the epilogue's shared memory in the same way.
template <int MAXC, bool PAIRS, typename VT, int FXM>
__global__ void __launch_bounds__(kThreads, sizeof(VT) == 4 ? 3 : 2)
ke_step(const VT* __restrict__ V, int64_t ldv, VT* __restrict__ w, EngDev e, int j, int cap) {
  constexpr bool FX = FXM == 1 || FXM == 2;
  static_assert(!FX || (PAIRS && std::is_same<VT, double>::value), "fixed-point products need FP64 tile pairs");
  static_assert(FXM != 3 || (PAIRS && std::is_same<VT, float>::value), "the FP32 ring variant is for FP32 tile pairs");
  __shared__ __align__(16) VT su[PAIRS ? 2 * kThreads : kThreads];
  __shared__ __align__(16) VT sw[PAIRS ? 2 * kThreads : kThreads];
  __shared__ uint32_t s_ex[2 * kWarps];
  __shared__ double red[2 * (kMaxM + 1) + 2];
  __shared__ int s_active, s_tail, s_stage_off;
  __shared__ SysDesc s_d;
  __shared__ uint64_t s_bar;
  __shared__ StageCopy<VT> s_nc;
  extern __shared__ __align__(16) double dyn[];
  int64_t lo, hi;
  if (!cta_tile_range(e, (int)gridDim.x, lo, hi)) return;
  const int J8 = j / kWarps, r8 = j % kWarps;
  const VT* u = V + (size_t)j * ldv;
  constexpr int kRpRows = 2 * kThreads;  // the rowptr slice holds up to a tile pair
  constexpr int kWs = 10;                // gathers in flight per staged row
  CsrStage<VT> cs;
  cs.rp = reinterpret_cast<int32_t*>(dyn);
  cs.col = cs.rp + (kRpRows + 4);
  cs.val = reinterpret_cast<VT*>(cs.col + cap);
  cs.bar = &s_bar;
  cs.cap = cap;
  cs.U = kRpRows;
  const size_t epi_off = (size_t)(kRpRows + 4) * 4 + (size_t)cap * (4 + sizeof(VT));
  if (threadIdx.x == 0) {
    s_stage_off = 0;
    mbar_init(&s_bar, 1);
  }
  __syncthreads();
  // thread 0: the unit at list position p (a pair when PAIRS and the tile is
  // even with its partner next in this CTA's range) and its copies
  auto unit_at = [&](int64_t p, int64_t& t, int& sy, bool& pair) {
    t = __ldg(e.act_tiles + p);
    sy = __ldg(e.act_sys + p);
    pair = PAIRS && (t & 1) == 0 && p + 1 < hi && __ldg(e.act_sys + p + 1) == sy;
  };
  auto copy_of = [&](int64_t t, int sy, bool pair) {
    const SysDesc* d = e.desc + sy;
    StageCopy<VT> c;
    c.rp = d->rowptr + (t * kThreads - d->row0);
    c.col = d->col;
    c.val = desc_val<VT>(*d);
    c.nrows = pair ? 2 * kThreads : kThreads;
    c.lo = CsrStage<VT>::lo_of(__ldg(c.rp));
    c.hi = CsrStage<VT>::hi_of(__ldg(c.rp + c.nrows));
    return c;
  };
  uint32_t phase = 0, pend_phase = 0;
  bool pending = false;  // thread 0: a copy was issued and not yet seen complete (phase pend_phase)
  bool held = false;     // thread 0: pend_phase is that of the copy left in flight by a failed wait
  if (threadIdx.x == 0 && lo < hi) {
    int64_t t0;
    int sy0;
    bool pr0;
    unit_at(lo, t0, sy0, pr0);
    const StageCopy<VT> c = copy_of(t0, sy0, pr0);
    cs.issue_at(c.rp, c.col, c.val, c.nrows, c.lo, c.hi);
    pending = true;
  }
  VT acc_a[MAXC], acc_c[MAXC], rem_a[kWarps - 1], rem_c[kWarps - 1];
  VT sig = VT(0), dd = VT(0);
  double fr_a[2] = {0.0, 0.0}, fr_c[2] = {0.0, 0.0};  // FX: remainder half-columns
  int kf[MAXC], kfr[2];                               // FX: 5 + the current system's column bounds
  int kf_u = 0;                                       // FX: 5 + the bound of its column j (u)
  int cur = -1;
  // Within a system the listing is the system's tiles in order, so the next
  // unit's tile follows from the current one (t_next) while it is at most the
  // system's last tile (t_last); the listing is read only where a system starts.
  int64_t t_next = -1, t_last = -1;
  // the current system's CSR (registers: the next unit's description reads no memory)
  const int32_t* cur_rp = nullptr;
  const int32_t* cur_col = nullptr;
  const VT* cur_val = nullptr;
  int64_t cur_row0 = 0;
  for (int64_t it = lo; it <= hi;) {
    int64_t t;
    int snext;
    if (it < hi && cur >= 0 && t_next <= t_last) {  // CTA-uniform
      t = t_next;
      snext = cur;
    } else {
      t = (it < hi) ? __ldg(e.act_tiles + it) : -1;
      snext = (it < hi) ? __ldg(e.act_sys + it) : -1;
    }
    if (snext != cur) {  // CTA-uniform
      if (snext < 0) {   // end of the range: no copy may still land in the buffer
        if (threadIdx.x == 0 && pending) mbar_wait_bounded(&s_bar, pend_phase);
        __syncthreads();
      }
      if (cur >= 0 && s_active) {  // done with system cur: publish its sums
        if constexpr (FX)
          cta_partials_fx<MAXC>(acc_a, acc_c, fr_a, fr_c, sig, dd, j, J8, r8, red);
        else
          cta_partials<MAXC, VT>(acc_a, acc_c, rem_a, rem_c, sig, dd, j, J8, r8, red);
        if (sys_publish(e, cur, red, 2 * j + 2)) {
          const Small sm = e.smalls[cur];
          if (threadIdx.x == 0) sm.st->reductions += 1;
          epilogue_one_reduce(sm, red, j, s_tail, epi_off);
        }
      }
      if (snext < 0) break;
      cur = snext;
      __syncthreads();  // every warp is done with the previous system's shared state
      if (threadIdx.x == 0) {
        const DevState* st = e.smalls[cur].st;
        const int kmax = __ldcg(&st->kmax);
        s_active = !__ldcg(&st->done) && j <= kmax;
        s_tail = (j == kmax);
        s_d = e.desc[cur];
      }
      __syncthreads();
      t_last = (s_d.row0 + s_d.n - 1) / kThreads;
      cur_rp = s_d.rowptr;
      cur_col = s_d.col;
      cur_val = desc_val<VT>(s_d);
      cur_row0 = s_d.row0;
#pragma unroll
      for (int c = 0; c < MAXC; ++c) acc_a[c] = acc_c[c] = VT(0);
#pragma unroll
      for (int c = 0; c < kWarps - 1; ++c) rem_a[c] = rem_c[c] = VT(0);
      sig = dd = VT(0);
      if constexpr (FX) {
        fr_a[0] = fr_a[1] = fr_c[0] = fr_c[1] = 0.0;
        const unsigned int* ec = e.smalls[cur].ecol;
        const int wid = threadIdx.x >> 5;
#pragma unroll
        for (int c = 0; c < MAXC; ++c)
          kf[c] = 5 + (int)max(kFxMinField, c < J8 ? __ldcg(ec + wid + c * kWarps) >> 20 : 0u);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const int r = wid + q * kWarps;
          kfr[q] = 5 + (int)max(kFxMinField, r < 2 * r8 ? __ldcg(ec + J8 * kWarps + (r >> 1)) >> 20 : 0u);
        }
        kf_u = 5 + (int)max(kFxMinField, __ldcg(ec + j) >> 20);
      }
    }
    const bool tail = s_tail;
    // a system's tiles are consecutive in the list and in the arena (its
    // region starts on a tile pair): tiles t, t + 1 form the pair t / 2
    const bool pair = PAIRS && (t & 1) == 0 && it + 1 < hi && t + 1 <= t_last;
    const int64_t it_next = it + (pair ? 2 : 1);
    t_next = t + (pair ? 2 : 1);
    // thread 0: the next unit's copies, described ahead of their issue (kept
    // in shared memory). A unit of the current system takes its descriptor
    // from s_d (no loads); the two rowptr bounds are loaded here and first
    // used when the copies are issued, after this unit's SpMV, which hides
    // their latency.
    int nlo_raw = 0, nhi_raw = 0;
    if (threadIdx.x == 0) {
      s_nc.nrows = 0;
      if (it_next < hi && t_next <= t_last) {  // the current system's next tile
        const int nr = (PAIRS && (t_next & 1) == 0 && it_next + 1 < hi && t_next + 1 <= t_last) ? 2 * kThreads
                                                                                               : kThreads;
        const int32_t* rp = cur_rp + (t_next * kThreads - cur_row0);
        nlo_raw = __ldg(rp);
        nhi_raw = __ldg(rp + nr);
        s_nc.rp = rp;
        s_nc.col = cur_col;
        s_nc.val = cur_val;
        s_nc.nrows = nr;
      } else if (it_next < hi) {  // the first tile of the next system
        int64_t t1;
        int sy1;
        bool pr1;
        unit_at(it_next, t1, sy1, pr1);
        const SysDesc* d = e.desc + sy1;
        StageCopy<VT> c;
        c.rp = d->rowptr + (t1 * kThreads - d->row0);
        c.col = d->col;
        c.val = desc_val<VT>(*d);
        c.nrows = pr1 ? 2 * kThreads : kThreads;
        c.lo = c.hi = 0;  // set from nlo_raw, nhi_raw at the issue
        nlo_raw = __ldg(c.rp);
        nhi_raw = __ldg(c.rp + c.nrows);
        s_nc = c;
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
      } else if (pending && !held) {  // no copy is issued after this one: keep its phase
        pend_phase = phase;
        held = true;
      }
    }
    phase ^= 1u;
    // once every thread is past this unit's SpMV, the buffer takes the next unit
    auto next = [&]() {
      if (threadIdx.x == 0 && s_nc.nrows > 0 && !s_stage_off) {
        cs.issue_at(s_nc.rp, s_nc.col, s_nc.val, s_nc.nrows, CsrStage<VT>::lo_of(nlo_raw),
                    CsrStage<VT>::hi_of(nhi_raw));
        pending = true;
      }
    };
    if (s_active) {
      const int64_t lim = s_d.row0 + s_d.n;
      const VT* val = desc_val<VT>(s_d);
      const VT* xg = u + s_d.row0;
      const int U = pair ? 2 * kThreads : kThreads;
      const int64_t row0 = t * kThreads + threadIdx.x, row1 = row0 + kThreads;  // arena rows
      const int32_t* rpl = s_d.rowptr - s_d.row0;  // indexed by arena row
      int slo = 0;
      if (staged) {
        slo = CsrStage<VT>::lo_of(cs.rp[0]);
        staged = CsrStage<VT>::hi_of(cs.rp[U]) - slo <= cap;
      }
      VT ur0 = VT(0), ur1 = VT(0), wr0 = VT(0), wr1 = VT(0);
      if (row0 < lim) ur0 = ld_as<VT>(u + row0);
      if (pair && row1 < lim) ur1 = ld_as<VT>(u + row1);
      if constexpr (FX) {
        // u is the system's basis column j: its limbs, for the block dots of
        // the cycle's later steps and the MAXPY (not at the tail, whose
        // column nothing reads again)
        if (!tail) {
          int2* vl = e.VL + (size_t)j * ldv;
          if (row0 < lim) vl[row0] = fx_split((double)ur0, kf_u);
          if (pair && row1 < lim) vl[row1] = fx_split((double)ur1, kf_u);
        }
      }
      if (!tail) {
        if (pair) {
          if (staged)
            csr_row2_staged<kWs>(cs.col, cs.val, xg, cs.rp[threadIdx.x] - slo, cs.rp[threadIdx.x + 1] - slo,
                                 cs.rp[kThreads + threadIdx.x] - slo, cs.rp[kThreads + threadIdx.x + 1] - slo, wr0,
                                 wr1);
          else {
            if (row0 < lim) wr0 = csr_row_plain(rpl, s_d.col, val, xg, row0);
            if (row1 < lim) wr1 = csr_row_plain(rpl, s_d.col, val, xg, row1);
          }
          if (row0 < lim) w[row0] = wr0;
          if (row1 < lim) w[row1] = wr1;
        } else if (row0 < lim) {
          wr0 = staged ? csr_row_staged<kWs>(cs.col, cs.val, xg, cs.rp[threadIdx.x] - slo,
                                             cs.rp[threadIdx.x + 1] - slo)
                       : csr_row_plain(rpl, s_d.col, val, xg, row0);
          w[row0] = wr0;
        }
      }
      if constexpr (FX) {
        // the pair t / 2: both tiles, or (a single tile) the one this unit holds
        const int64_t pb = (t >> 1) * (2 * kThreads);  // the pair's first arena row
        const bool second = !pair && (t & 1);
        const int rlo = (int)(max(s_d.row0, second ? pb + kThreads : pb) - pb);
        const int rhi = (int)(min(lim, pair || second ? pb + 2 * kThreads : pb + kThreads) - pb);
        double* ring = FXM == 2 ? reinterpret_cast<double*>(reinterpret_cast<char*>(dyn) + epi_off) : nullptr;
        // the basis columns as the limbs stored at their own steps
        const double* VLd = reinterpret_cast<const double*>(e.VL);
        if (second)
          tile_pair_dot_rows_fx<MAXC, FXM == 2, kEngRing, true>(t >> 1, lim, VLd, ldv, !tail, J8, r8, 0.0, 0.0, ur0,
                                                                wr0, su, sw, ring, kf, kfr, acc_a, acc_c, fr_a, fr_c,
                                                                sig, dd, s_ex, next, rlo, rhi);
        else
          tile_pair_dot_rows_fx<MAXC, FXM == 2, kEngRing, true>(t >> 1, lim, VLd, ldv, !tail, J8, r8, ur0, wr0, ur1,
                                                                wr1, su, sw, ring, kf, kfr, acc_a, acc_c, fr_a, fr_c,
                                                                sig, dd, s_ex, next, rlo, rhi);
      } else if constexpr (FXM == 3) {
        // FP32 tile pairs with the basis through the per-warp cp.async ring
        // (over the epilogue's shared memory); a single tile runs as its pair
        // with the absent tile's u and w zero
        VT* ring = reinterpret_cast<VT*>(reinterpret_cast<char*>(dyn) + epi_off);
        if (!pair && (t & 1))
          tile_pair_dot_rows_pf<MAXC, VT, VT>(t >> 1, lim, V, ldv, !tail, J8, r8, VT(0), VT(0), ur0, wr0, su, sw,
                                              ring, acc_a, acc_c, rem_a, rem_c, sig, dd, next);
        else
          tile_pair_dot_rows_pf<MAXC, VT, VT>(t >> 1, lim, V, ldv, !tail, J8, r8, ur0, wr0, ur1, wr1, su, sw, ring,
                                              acc_a, acc_c, rem_a, rem_c, sig, dd, next);
      } else if (pair)
        tile_pair_dot_rows<MAXC, VT, VT>(t >> 1, lim, V, ldv, !tail, J8, r8, ur0, wr0, ur1, wr1, su, sw, acc_a, acc_c,
                                         rem_a, rem_c, sig, dd, next);
      else
        tile_dot_rows<MAXC, VT, VT>(t, lim, V, ldv, !tail, J8, r8, ur0, wr0, su, sw, acc_a, acc_c, rem_a, rem_c, sig,
                                    dd, next);
    } else {
      __syncthreads();  // every thread is past its wait for this unit
      next();
    }
    it = it_next;
  }
}

template <bool PAIRS, typename VT, int FX>
EngStepKernel<VT> eng_step_sel(int m) {
  switch (std::max(1, m / kWarps)) {
    case 1: return ke_step<1, PAIRS, VT, FX>;
    case 2: return ke_step<2, PAIRS, VT, FX>;
    case 3: return ke_step<3, PAIRS, VT, FX>;
    case 4: return ke_step<4, PAIRS, VT, FX>;
    case 5: return ke_step<5, PAIRS, VT, FX>;
    case 6: return ke_step<6, PAIRS, VT, FX>;
    case 7: return ke_step<7, PAIRS, VT, FX>;
    case 8: return ke_step<8, PAIRS, VT, FX>;
    case 9: case 10: case 11: case 12: return ke_step<12, PAIRS, VT, FX>;
    default: return ke_step<16, PAIRS, VT, FX>;
  }
}

// The step kernel for restart length m, one or two rows per thread, and (FP64
// tile pairs only) fixed-point block-dot products: fx = 1 direct basis loads,
// fx = 2 the column ring; (FP32 tile pairs only) fx = 3 the column ring.
template <typename VT>
EngStepKernel<VT> eng_step_table(int m, bool pairs, int fx) {
  if constexpr (std::is_same<VT, double>::value) {
    if (pairs && fx == 1) return eng_step_sel<true, VT, 1>(m);
    if (pairs && fx == 2) return eng_step_sel<true, VT, 2>(m);
  } else {
    if (pairs && fx == 3) return eng_step_sel<true, VT, 3>(m);
  }
  return pairs ? eng_step_sel<true, VT, 0>(m) : eng_step_sel<false, VT, 0>(m);
}

}  // namespace
