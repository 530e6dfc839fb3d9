// Instruction-throughput probe: how many instructions of one kind an SM
// retires per clock when every warp slot it can hold issues nothing else.
//
// The roofline of the FP64 Arnoldi step is set on B300 by the FP64 pipe, not
// by HBM (2 DFMA per basis element in the block dot against ~2 DFMA per clock
// per SM), so the peak the step is measured against has to be measured too.
// The same probe measures the integer and conversion instructions that an
// FP64 product can be emulated with, which decides where such emulation pays.
//
// Each thread runs kChains independent dependency chains of the instruction
// (so the pipe, not its latency, is the limit) for `iters` rounds; one thread
// per CTA stamps the SM clock before and after (with a CTA barrier on both
// sides), and the host times the launch with CUDA events. Operands come from
// a kernel argument and the chains feed one another, so the compiler can fold
// nothing; every chain ends in a store that never happens unless the value
// equals a key the host never passes (no dead-code elimination).
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "lsgmres.h"

namespace {

constexpr int kProbeThreads = 256;
constexpr int kChains = 8;
constexpr int kUnroll = 4;  // rounds of kChains instructions per loop trip

template <int OP>
__device__ __forceinline__ void probe_round(uint64_t (&x)[kChains], uint32_t a, uint32_t b) {
#pragma unroll
  for (int c = 0; c < kChains; ++c) {
    uint64_t& v = x[c];
    const uint64_t nb = x[(c + 1) % kChains];
    if constexpr (OP == LSG_PROBE_DFMA) {
      double d = __longlong_as_double((long long)v);
      asm volatile("fma.rn.f64 %0, %0, %1, %2;" : "+d"(d) : "d"(__longlong_as_double((long long)a | 0x3fe0000000000000ull)), "d"(0.5));
      v = (uint64_t)__double_as_longlong(d);
    } else if constexpr (OP == LSG_PROBE_DADD) {
      double d = __longlong_as_double((long long)v);
      asm volatile("add.rn.f64 %0, %0, %1;" : "+d"(d) : "d"(__longlong_as_double((long long)b | 0x3ff0000000000000ull)));
      v = (uint64_t)__double_as_longlong(d);
    } else if constexpr (OP == LSG_PROBE_FFMA) {
      float f = __uint_as_float((uint32_t)v);
      asm volatile("fma.rn.f32 %0, %0, %1, %2;" : "+f"(f) : "f"(__uint_as_float((a & 0x7fffffu) | 0x3f000000u)), "f"(0.5f));
      v = __float_as_uint(f);
    } else if constexpr (OP == LSG_PROBE_IMAD) {
      uint32_t r = (uint32_t)v;
      asm volatile("mad.lo.u32 %0, %0, %1, %2;" : "+r"(r) : "r"(a), "r"((uint32_t)nb));
      v = r;
    } else if constexpr (OP == LSG_PROBE_IMAD_WIDE) {
      asm volatile("mad.wide.u32 %0, %1, %2, %0;" : "+l"(v) : "r"((uint32_t)nb), "r"(a));
    } else if constexpr (OP == LSG_PROBE_IMAD_HI) {
      uint32_t r = (uint32_t)v;
      asm volatile("mad.hi.u32 %0, %0, %1, %2;" : "+r"(r) : "r"(a), "r"((uint32_t)nb));
      v = r;
    } else if constexpr (OP == LSG_PROBE_IADD) {
      uint32_t r = (uint32_t)v;
      asm volatile("add.u32 %0, %0, %1;" : "+r"(r) : "r"((uint32_t)nb));
      v = r;
    } else if constexpr (OP == LSG_PROBE_LOP3) {
      uint32_t r = (uint32_t)v;
      asm volatile("lop3.b32 %0, %0, %1, %2, 0x96;" : "+r"(r) : "r"((uint32_t)nb), "r"(b));
      v = r;
    } else if constexpr (OP == LSG_PROBE_SHF) {
      uint32_t r = (uint32_t)v;
      asm volatile("shf.l.wrap.b32 %0, %0, %1, %2;" : "+r"(r) : "r"((uint32_t)nb), "r"(a));
      v = r;
    } else if constexpr (OP == LSG_PROBE_I2F_F64) {
      double d;
      asm volatile("cvt.rn.f64.s64 %0, %1;" : "=d"(d) : "l"(v ^ nb));
      v = (uint64_t)__double_as_longlong(d);
    } else if constexpr (OP == LSG_PROBE_F2I_F64) {
      long long r;
      asm volatile("cvt.rni.s64.f64 %0, %1;" : "=l"(r) : "d"(__longlong_as_double((long long)((v & 0xfffffffffffffull) | 0x4300000000000000ull))));
      v = (uint64_t)r ^ nb;
    } else if constexpr (OP == LSG_PROBE_F2F_F32_F64) {
      float f;
      asm volatile("cvt.rn.f32.f64 %0, %1;" : "=f"(f) : "d"(__longlong_as_double((long long)((v & 0xfffffffffffffull) | 0x3ff0000000000000ull))));
      v = (uint64_t)__float_as_uint(f) ^ nb;
    } else if constexpr (OP == LSG_PROBE_I2F_F32) {
      float f;
      asm volatile("cvt.rn.f32.s32 %0, %1;" : "=f"(f) : "r"((uint32_t)(v ^ nb)));
      v = __float_as_uint(f);
    } else if constexpr (OP == LSG_PROBE_FLO) {
      uint32_t r;
      asm volatile("clz.b32 %0, %1;" : "=r"(r) : "r"((uint32_t)(v ^ nb)));
      v = r + b;
    }
  }
}

template <int OP>
__global__ void __launch_bounds__(kProbeThreads) k_probe(int iters, uint32_t a, uint32_t b, uint64_t key,
                                                        uint64_t* sink, unsigned long long* cycles) {
  __shared__ unsigned long long t0;
  uint64_t x[kChains];
#pragma unroll
  for (int c = 0; c < kChains; ++c) x[c] = (uint64_t)(threadIdx.x * kChains + c) * 0x9e3779b97f4a7c15ull + a;
  __syncthreads();
  if (threadIdx.x == 0) t0 = clock64();
  __syncthreads();
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int u = 0; u < kUnroll; ++u) probe_round<OP>(x, a, b);
  }
  __syncthreads();
  if (threadIdx.x == 0) cycles[blockIdx.x] = clock64() - t0;
  uint64_t acc = 0;
#pragma unroll
  for (int c = 0; c < kChains; ++c) acc ^= x[c];
  if (acc == key) sink[blockIdx.x * blockDim.x + threadIdx.x] = acc;
}

using ProbeKernel = void (*)(int, uint32_t, uint32_t, uint64_t, uint64_t*, unsigned long long*);

ProbeKernel probe_kernel(int op) {
  switch (op) {
    case LSG_PROBE_DFMA: return k_probe<LSG_PROBE_DFMA>;
    case LSG_PROBE_DADD: return k_probe<LSG_PROBE_DADD>;
    case LSG_PROBE_FFMA: return k_probe<LSG_PROBE_FFMA>;
    case LSG_PROBE_IMAD: return k_probe<LSG_PROBE_IMAD>;
    case LSG_PROBE_IMAD_WIDE: return k_probe<LSG_PROBE_IMAD_WIDE>;
    case LSG_PROBE_IMAD_HI: return k_probe<LSG_PROBE_IMAD_HI>;
    case LSG_PROBE_IADD: return k_probe<LSG_PROBE_IADD>;
    case LSG_PROBE_LOP3: return k_probe<LSG_PROBE_LOP3>;
    case LSG_PROBE_SHF: return k_probe<LSG_PROBE_SHF>;
    case LSG_PROBE_I2F_F64: return k_probe<LSG_PROBE_I2F_F64>;
    case LSG_PROBE_F2I_F64: return k_probe<LSG_PROBE_F2I_F64>;
    case LSG_PROBE_F2F_F32_F64: return k_probe<LSG_PROBE_F2F_F32_F64>;
    case LSG_PROBE_I2F_F32: return k_probe<LSG_PROBE_I2F_F32>;
    case LSG_PROBE_FLO: return k_probe<LSG_PROBE_FLO>;
    default: return nullptr;
  }
}

thread_local std::string g_probe_err;  // one message per host thread

gmres_status probe_fail(gmres_status st, const std::string& msg) {
  g_probe_err = msg;
  return st;
}

}  // namespace

extern "C" {

gmres_status lsg_probe_pipe(int op, int ctas_per_sm, int iters, lsg_probe_result* out) {
  ProbeKernel k = probe_kernel(op);
  if (!k) return probe_fail(GMRES_ERR_ARG, "unknown probe op");
  if (ctas_per_sm < 1 || ctas_per_sm > 8 || iters < 1 || iters > (1 << 24) || !out)
    return probe_fail(GMRES_ERR_ARG, "ctas_per_sm must be in [1, 8], iters in [1, 2^24], out non-NULL");
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return probe_fail(GMRES_ERR_CUDA, std::string("device query: ") + cudaGetErrorString(e));
  const int grid = nsm * ctas_per_sm;
  uint64_t* sink = nullptr;
  unsigned long long* cyc = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  std::vector<unsigned long long> hc(grid);
  float ms = 0.f;
  auto cleanup = [&]() {
    cudaFree(sink);
    cudaFree(cyc);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
  };
#define PROBE_TRY(call)                                                                        \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess) {                                                                   \
      cleanup();                                                                               \
      return probe_fail(GMRES_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_));  \
    }                                                                                          \
  } while (0)
  PROBE_TRY(cudaMalloc(&sink, sizeof(uint64_t) * grid * kProbeThreads));
  PROBE_TRY(cudaMalloc(&cyc, sizeof(unsigned long long) * grid));
  PROBE_TRY(cudaEventCreate(&e0));
  PROBE_TRY(cudaEventCreate(&e1));
  // one short warm-up launch (clocks ramp, instruction cache), then the timed one
  k<<<grid, kProbeThreads>>>(iters / 8 + 1, 0x9e3779b9u, 0x7f4a7c15u, 0x1ull, sink, cyc);
  PROBE_TRY(cudaGetLastError());
  PROBE_TRY(cudaEventRecord(e0));
  k<<<grid, kProbeThreads>>>(iters, 0x9e3779b9u, 0x7f4a7c15u, 0x1ull, sink, cyc);
  PROBE_TRY(cudaGetLastError());
  PROBE_TRY(cudaEventRecord(e1));
  PROBE_TRY(cudaEventSynchronize(e1));
  PROBE_TRY(cudaEventElapsedTime(&ms, e0, e1));
  PROBE_TRY(cudaMemcpy(hc.data(), cyc, sizeof(unsigned long long) * grid, cudaMemcpyDeviceToHost));
  cleanup();
#undef PROBE_TRY
  unsigned long long cmax = 0;
  for (unsigned long long c : hc) cmax = c > cmax ? c : cmax;
  const double per_thread = (double)iters * kUnroll * kChains;
  const double per_sm = per_thread * kProbeThreads * ctas_per_sm;
  out->ops_per_clk_per_sm = cmax ? per_sm / (double)cmax : 0.0;
  out->ops_per_s = per_sm * nsm / (ms * 1e-3);
  out->sm_mhz = cmax / (ms * 1e-3) / 1e6;
  out->seconds = ms * 1e-3;
  out->sms = nsm;
  return GMRES_OK;
}

const char* lsg_probe_last_error(void) { return g_probe_err.c_str(); }

}  // extern "C"
