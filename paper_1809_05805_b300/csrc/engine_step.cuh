// The engine's step kernel (Algorithm 7's loop body for every listed system)
// and its instantiation table.
#pragma once

#include "engine.cuh"

namespace {

// Step j of the current cycle for every listed system: the CTA walks its
// range of listed tiles (pairs of consecutive tiles of one system, two rows
// per thread, when PAIRS); whenever the range moves to another system it
// publishes that system's sums, and the CTA completing a system runs the
// system's reduction and epilogue.
template <int MAXC, bool PAIRS, typename VT>
__global__ void __launch_bounds__(kThreads, sizeof(VT) == 4 ? 3 : 2)
ke_step(const VT* __restrict__ V, int64_t ldv, VT* __restrict__ w, EngDev e, int j) {
  __shared__ VT su[PAIRS ? 2 * kThreads : kThreads];
  __shared__ VT sw[PAIRS ? 2 * kThreads : kThreads];
  __shared__ double red[2 * (kMaxM + 1) + 2];
  __shared__ int s_active, s_tail;
  __shared__ SysDesc s_d;
  int64_t lo, hi;
  if (!cta_tile_range(e, (int)gridDim.x, lo, hi)) return;
  const int J8 = j / kWarps, r8 = j % kWarps;
  const VT* u = V + (size_t)j * ldv;
  VT acc_a[MAXC], acc_c[MAXC], rem_a[kWarps - 1], rem_c[kWarps - 1];
  VT sig = VT(0), dd = VT(0);
  int cur = -1;
  for (int64_t it = lo; it <= hi;) {
    const int64_t t = (it < hi) ? __ldg(e.act_tiles + it) : -1;
    const int snext = (it < hi) ? __ldg(e.act_sys + it) : -1;
    if (snext != cur) {  // CTA-uniform
      if (cur >= 0 && s_active) {  // done with system cur: publish its sums
        cta_partials<MAXC, VT>(acc_a, acc_c, rem_a, rem_c, sig, dd, j, J8, r8, red);
        if (sys_publish(e, cur, red, 2 * j + 2)) {
          const Small sm = e.smalls[cur];
          if (threadIdx.x == 0) sm.st->reductions += 1;
          epilogue_one_reduce(sm, red, j, s_tail);
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
#pragma unroll
      for (int c = 0; c < MAXC; ++c) acc_a[c] = acc_c[c] = VT(0);
#pragma unroll
      for (int c = 0; c < kWarps - 1; ++c) rem_a[c] = rem_c[c] = VT(0);
      sig = dd = VT(0);
    }
    const bool tail = s_tail;
    const int64_t lim = s_d.row0 + s_d.n;
    const int32_t* rp = s_d.rowptr - s_d.row0;  // indexed by arena row
    const VT* val = desc_val<VT>(s_d);
    const VT* xg = u + s_d.row0;
    // a system's tiles are consecutive in the list and in the arena (its
    // region starts on a tile pair): tiles t, t + 1 form the pair t / 2
    if (PAIRS && (t & 1) == 0 && it + 1 < hi && __ldg(e.act_sys + it + 1) == cur) {
      if (s_active)
        tile_pair_block_dot<MAXC, VT>(t >> 1, lim, rp, s_d.col, val, V, ldv, u, xg, w, !tail, !tail, J8, r8, su, sw,
                                      acc_a, acc_c, rem_a, rem_c, sig, dd);
      it += 2;
      continue;
    }
    if (s_active)
      tile_block_dot<MAXC, VT>(t, lim, rp, s_d.col, val, V, ldv, u, xg, w, !tail, !tail, J8, r8, su, sw, acc_a, acc_c,
                               rem_a, rem_c, sig, dd);
    ++it;
  }
}

template <bool PAIRS, typename VT>
EngStepKernel<VT> eng_step_sel(int m) {
  switch (std::max(1, m / kWarps)) {
    case 1: return ke_step<1, PAIRS, VT>;
    case 2: return ke_step<2, PAIRS, VT>;
    case 3: return ke_step<3, PAIRS, VT>;
    case 4: return ke_step<4, PAIRS, VT>;
    case 5: return ke_step<5, PAIRS, VT>;
    case 6: return ke_step<6, PAIRS, VT>;
    case 7: return ke_step<7, PAIRS, VT>;
    case 8: return ke_step<8, PAIRS, VT>;
    case 9: case 10: case 11: case 12: return ke_step<12, PAIRS, VT>;
    default: return ke_step<16, PAIRS, VT>;
  }
}

template <typename VT>
EngStepKernel<VT> eng_step_table(int m, bool pairs) {
  return pairs ? eng_step_sel<true, VT>(m) : eng_step_sel<false, VT>(m);
}

}  // namespace
