// Device-side layout of the batched engine (system descriptors, the listing
// of active tiles, per-system reduction slots) and its step kernel. The step
// kernel's instantiations are compiled in engine_step_f64.cu and
// engine_step_f32.cu (built in parallel) and reached through
// lsg_engine::eng_step_*.
#pragma once

#include "common.cuh"

namespace lsg_engine {
// Host stub of the engine step kernel for restart length m, with or without
// tile pairs, with fixed-point block-dot products (FP64 tile pairs only;
// ignored otherwise: fx = 1 direct basis loads, 2 the column ring) or not
// (fx = 0); callers cast it to their EngStepKernel type.
const void* eng_step_f64(int m, bool pairs, int fx);
const void* eng_step_f32(int m, bool pairs, int fx);
}  // namespace lsg_engine

namespace {

constexpr int kPairRows = 2 * kThreads;  // arena regions are whole tile pairs
constexpr int kMaxGridPerSm = 8;         // largest grid of any engine kernel, per SM
constexpr int kEngRing = 2;              // half-column slices per warp in the step kernel's column ring
constexpr size_t kEngRingBytes = (size_t)kWarps * kEngRing * kThreads * sizeof(double);

// Where one system lives.
struct SysDesc {
  const int32_t* rowptr;  // n + 1 entries (local)
  const int32_t* col;     // local column indices
  const double* val;      // FP64 values
  const float* val32;     // FP32 values (GMRES-IR), else null
  int64_t row0;           // first arena row (multiple of kPairRows)
  int64_t n;              // rows
};

struct EngDev {
  const SysDesc* desc;       // per slot
  const Small* smalls;       // per slot
  const int32_t* act_tiles;  // Ta: arena tiles of the listed systems, system by system
  const int32_t* act_sys;    // Ta: slot of each listed tile
  const int64_t* n_act;      // Ta (device scalar)
  const int32_t* act_slots;  // listed systems
  const int32_t* n_slots;    // their number (device scalar)
  const int32_t* sys_b0;     // per slot: first CTA (of the reduction grid) whose range touches it
  const int32_t* sys_nslot;  // per slot: number of such CTAs
  const int32_t* sys_slot0;  // per slot: its first partial-sum slot
  double* partials;          // one row of nvmax per (CTA, system) pair
  unsigned int* tickets;     // per slot
  // The reduction grid's ranges of the listing: bounds[0] = Pe (CTAs with a
  // range), CTA c < Pe takes [bounds[1 + c], bounds[2 + c]); built by the host
  // with the listing for a grid of nb CTAs.
  const int32_t* bounds;
  int nb;
  int nvmax;
  // FP64 cycles: the arena's basis a second time as fixed-point limbs (same
  // rows and leading dimension; each system's column j written by the step
  // kernel when it is the step's u, read by later steps' block dots and by
  // the MAXPY); null for FP32 cycles
  int2* VL;
};

// This CTA's range [lo, hi) of the listed tiles when `grid` CTAs share them.
// For the reduction grid (grid == nb) the ranges are the host's (balanced by
// estimated cost: each tile, plus a fixed charge for each system whose first
// tile the range holds, for its switch and epilogue); otherwise the first
// Pe = min(grid, Ta) CTAs split the list evenly. Either way every range is
// non-empty (so the CTAs touching a system are consecutive) and the other
// CTAs get none.
__device__ __forceinline__ bool cta_tile_range(const EngDev& e, int grid, int64_t& lo, int64_t& hi) {
  if (grid == e.nb) {
    const int pe = __ldg(e.bounds);
    if ((int)blockIdx.x >= pe) return false;
    lo = __ldg(e.bounds + 1 + blockIdx.x);
    hi = __ldg(e.bounds + 2 + blockIdx.x);
    return true;
  }
  const int64_t Ta = *e.n_act;
  const int64_t Pe = Ta < (int64_t)grid ? Ta : (int64_t)grid;
  if ((int64_t)blockIdx.x >= Pe) return false;
  lo = (int64_t)blockIdx.x * Ta / Pe;
  hi = ((int64_t)blockIdx.x + 1) * Ta / Pe;
  return true;
}

// Publish this CTA's sums for system sy (red[0 .. nv)) in its (CTA, system)
// slot and take the system's ticket; true in every thread of the CTA that
// arrived last, after which red holds the system's totals (summed over its
// slots in slot order: deterministic for a given listing and grid).
__device__ __forceinline__ bool sys_publish(const EngDev& e, int sy, double* red, int nv) {
  const int64_t slot0 = __ldg(e.sys_slot0 + sy);
  return publish_and_reduce(e.partials, e.nvmax, slot0 + ((int)blockIdx.x - __ldg(e.sys_b0 + sy)), slot0,
                            __ldg(e.sys_nslot + sy), e.tickets + sy, red, nv);
}

template <typename VT>
__device__ __forceinline__ const VT* desc_val(const SysDesc& d);
template <>
__device__ __forceinline__ const double* desc_val<double>(const SysDesc& d) {
  return d.val;
}
template <>
__device__ __forceinline__ const float* desc_val<float>(const SysDesc& d) {
  return d.val32;
}

template <typename VT>
using EngStepKernel = void (*)(const VT*, int64_t, VT*, EngDev, int, int);

}  // namespace
