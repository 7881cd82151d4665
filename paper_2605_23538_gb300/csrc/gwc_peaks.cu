// gwc_peaks.cu -- throughput probes of the GPU's arithmetic units (measurement only).
//
// The likelihood kernels are bound by arithmetic, not by memory: their roofline is the
// FP32 pipe (adds, multiplies, fused multiply-adds) and the special-function unit (the
// ex2/lg2/rcp/rsqrt approximations).  These probes measure what each unit sustains on
// the device at hand, so that the roofline fractions the benchmark reports rest on
// measured peaks.  Each probe is one kernel in which every thread runs CHAINS independent
// dependency chains of one operation for `iters` iterations; enough warps are resident
// to hide the operation's latency, so the time is set by the unit's issue rate.
#include <cstdint>
#include <string>

#include "../../include/gwc.h"
#include "gwc_kernels.h"

using namespace gwc;

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int CHAINS = 8;

// written only when a chain reaches a value it never reaches, so the work stays live
__device__ float g_probe_sink_f;
__device__ double g_probe_sink_d;

__device__ __forceinline__ float p_ex2(float x) {
  float y;
  asm volatile("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float p_lg2(float x) {
  float y;
  asm volatile("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float p_rcp(float x) {
  float y;
  asm volatile("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
__device__ __forceinline__ float p_rsqrt(float x) {
  float y;
  asm volatile("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
  return y;
}
// packed pair FMA (two FP32 lanes per instruction)
__device__ __forceinline__ unsigned long long p_fma2(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm volatile("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  return (unsigned long long)__float_as_uint(lo) | ((unsigned long long)__float_as_uint(hi) << 32);
}

template <int UNIT>
__global__ void __launch_bounds__(PROBE_THREADS) k_probe(int iters) {
  const float seed = 1e-3f * (float)(threadIdx.x & 7);
  if constexpr (UNIT == GWC_UNIT_DFMA || UNIT == GWC_UNIT_DFMA_LANE1) {
    double a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = 0.5 + seed + 0.01 * c;
    // DFMA_LANE1: only lane 0 of each warp runs the chains (does the FP64 pipe charge a
    // warp-instruction by its active lanes or as a whole?)
    if (UNIT == GWC_UNIT_DFMA || (threadIdx.x & 31) == 0) {
      for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int c = 0; c < CHAINS; ++c) a[c] = fma(a[c], 0.999, 1e-3);
      }
    }
    double s = 0.0;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += a[c];
    if (s == -1.25) g_probe_sink_d = s;
  } else if constexpr (UNIT == GWC_UNIT_FFMA2) {
    unsigned long long a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = pack2(0.5f + seed + 0.01f * c, 0.25f + seed + 0.01f * c);
    const unsigned long long b = pack2(0.999f, 0.998f), d = pack2(1e-3f, 2e-3f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) a[c] = p_fma2(a[c], b, d);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += __uint_as_float((unsigned)a[c]) + __uint_as_float((unsigned)(a[c] >> 32));
    if (s == -1.25f) g_probe_sink_f = s;
  } else {
    float a[CHAINS];
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = (UNIT == GWC_UNIT_EX2 ? -0.5f : 1.5f) + seed + 0.01f * c;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
      for (int c = 0; c < CHAINS; ++c) {
        // each chain stays bounded: ex2(a) - 1 in (-1, 0], lg2(a) + 1.5 near 3.1,
        // rcp(a) + 1 near 1.6, rsqrt(a) + 1 near 1.75, the FMA's fixed point 1
        if constexpr (UNIT == GWC_UNIT_FFMA) a[c] = fmaf(a[c], 0.999f, 1e-3f);
        else if constexpr (UNIT == GWC_UNIT_EX2) a[c] = p_ex2(a[c]) - 1.f;
        else if constexpr (UNIT == GWC_UNIT_LG2) a[c] = p_lg2(a[c]) + 1.5f;
        else if constexpr (UNIT == GWC_UNIT_RCP) a[c] = p_rcp(a[c]) + 1.f;
        else a[c] = p_rsqrt(a[c]) + 1.f;
      }
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) s += a[c];
    if (s == -1.25f) g_probe_sink_f = s;
  }
}

gwc_status probe_err(gwc_status s, const std::string& m) {
  set_thread_error(m);
  return s;
}

}  // namespace

extern "C" gwc_status gwc_alu_probe(int32_t unit, int32_t blocks, int32_t iters, double* ops, void* stream) {
  if (blocks < 1 || blocks > (1 << 20) || iters < 1) return probe_err(GWC_E_INVALID, "blocks or iters out of range");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  double per_op = 1.0;
  switch (unit) {
    case GWC_UNIT_FFMA: k_probe<GWC_UNIT_FFMA><<<blocks, PROBE_THREADS, 0, s>>>(iters); break;
    case GWC_UNIT_FFMA2: k_probe<GWC_UNIT_FFMA2><<<blocks, PROBE_THREADS, 0, s>>>(iters); per_op = 2.0; break;
    case GWC_UNIT_EX2: k_probe<GWC_UNIT_EX2><<<blocks, PROBE_THREADS, 0, s>>>(iters); break;
    case GWC_UNIT_LG2: k_probe<GWC_UNIT_LG2><<<blocks, PROBE_THREADS, 0, s>>>(iters); break;
    case GWC_UNIT_RCP: k_probe<GWC_UNIT_RCP><<<blocks, PROBE_THREADS, 0, s>>>(iters); break;
    case GWC_UNIT_RSQRT: k_probe<GWC_UNIT_RSQRT><<<blocks, PROBE_THREADS, 0, s>>>(iters); break;
    case GWC_UNIT_DFMA: k_probe<GWC_UNIT_DFMA><<<blocks, PROBE_THREADS, 0, s>>>(iters); break;
    case GWC_UNIT_DFMA_LANE1:
      k_probe<GWC_UNIT_DFMA_LANE1><<<blocks, PROBE_THREADS, 0, s>>>(iters);
      per_op = 1.0 / 32.0;   // one lane of 32 works
      break;
    default: return probe_err(GWC_E_INVALID, "unknown unit");
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return probe_err(GWC_E_CUDA, std::string("probe launch: ") + cudaGetErrorString(e));
  if (ops) *ops = (double)blocks * PROBE_THREADS * CHAINS * (double)iters * per_op;
  return GWC_OK;
}
