// Measured FP32 FMA throughput of the device: the denominator of the roofline of the kernels that
// are bound by FP32 FMA issue (the matrix-free tap kernel of long-range hopping).  Every thread
// runs eight independent FMA chains, so the pipe is limited by issue, not by the 4-cycle FMA
// latency; the packed form issues f32x2 FMAs (two FMAs per lane and instruction), the form the
// tap kernel uses.  The chains start from kernel arguments and end in a store that a run with
// finite inputs never takes, so the compiler keeps all of them.
#include <cuda_runtime.h>

#include <algorithm>

#include "tbpm_internal.cuh"

namespace tbpm {

constexpr int kPeakThreads = 256;
constexpr int kPeakChains = 8;

template <bool PACKED>
__global__ void __launch_bounds__(kPeakThreads) k_fma_peak(float a, float b, int iters, float* sink) {
  const float x0 = a + 1e-7f * (float)threadIdx.x;
  if constexpr (PACKED) {
    float2 v[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) v[c] = make_float2(x0 + c, x0 - c);
    const float2 m = make_float2(a, a), d = make_float2(b, -b);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) v[c] = __ffma2_rn(v[c], m, d);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += v[c].x + v[c].y;
    if (!(s == s)) sink[threadIdx.x] = s;  // NaN only: never for finite a, b with |a| < 1
  } else {
    float v[kPeakChains];
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) v[c] = x0 + c;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
      for (int c = 0; c < kPeakChains; ++c) v[c] = fmaf(v[c], a, b);
    }
    float s = 0.f;
#pragma unroll
    for (int c = 0; c < kPeakChains; ++c) s += v[c];
    if (!(s == s)) sink[threadIdx.x] = s;
  }
}

}  // namespace tbpm

using namespace tbpm;

// Times both forms with CUDA events on the context stream (one warm-up launch each, then the
// best of three) and returns TFLOP/s with an FMA counted as two flops.
extern "C" int tbpm_fp32_fma_peak(tbpm_ctx* ctx, double* tflops_scalar, double* tflops_packed) {
  clear_error();
  if (!ctx || !tflops_scalar || !tflops_packed) {
    set_error("tbpm_fp32_fma_peak: NULL argument");
    return TBPM_EINVAL;
  }
  TBPM_TRY(ensure(ctx, ctx->ws_aux, sizeof(float) * kPeakThreads));
  float* sink = (float*)ctx->ws_aux.p;
  const int blocks = ctx->num_sms * 8;  // 64 warps per SM
  const int iters = 1 << 14;
  cudaEvent_t e0, e1;
  TBPM_CK(cudaEventCreate(&e0));
  TBPM_CK(cudaEventCreate(&e1));
  double out[2] = {0.0, 0.0};
  int r = TBPM_OK;
  for (int packed = 0; packed < 2 && r == TBPM_OK; ++packed) {
    void* fn = packed ? (void*)k_fma_peak<true> : (void*)k_fma_peak<false>;
    float a = 0.999f, b = 1e-3f;
    int it = iters;
    void* args[] = {&a, &b, &it, &sink};
    float best = 1e30f;
    for (int rep = 0; rep < 4 && r == TBPM_OK; ++rep) {
      cudaEventRecord(e0, ctx->stream);
      cudaError_t e = cudaLaunchKernel(fn, dim3(blocks), dim3(kPeakThreads), args, 0, ctx->stream);
      ctx->launches++;
      cudaEventRecord(e1, ctx->stream);
      if (e == cudaSuccess) e = cudaEventSynchronize(e1);
      if (e != cudaSuccess) {
        set_error("tbpm_fp32_fma_peak: %s", cudaGetErrorString(e));
        r = TBPM_ECUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (rep > 0) best = std::min(best, ms);  // launch 0 warms up
    }
    const double fmas = (double)blocks * kPeakThreads * iters * kPeakChains * (packed ? 2.0 : 1.0);
    out[packed] = 2.0 * fmas / (best * 1e-3) / 1e12;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TBPM_TRY(r);
  *tflops_scalar = out[0];
  *tflops_packed = out[1];
  return TBPM_OK;
}
