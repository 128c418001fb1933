// Device building blocks shared by the recurrence kernels (csrc/cheb.cu) and the batched
// serving kernel (csrc/serve.cu): 16-byte state packs, FP32/FP64 partial sums, the
// deterministic grid reduction, and the matrix-free stencil neighbour offsets along x-lines.
#pragma once

#include <cuda_runtime.h>

#include "tbpm_internal.cuh"

namespace tbpm {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

// ------------------------------------------------------------------ 16-byte state packs
template <typename R, int SPT>
struct Pack {
  R v[2 * SPT];
};

template <typename R, int SPT>
__device__ __forceinline__ Pack<R, SPT> ld(const Pack<R, SPT>* p) {
  Pack<R, SPT> r;
  if constexpr (sizeof(Pack<R, SPT>) == 16) {
    if constexpr (sizeof(R) == 4) {
      const float4 q = __ldg(reinterpret_cast<const float4*>(p));
      r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
    } else {
      const double2 q = __ldg(reinterpret_cast<const double2*>(p));
      r.v[0] = q.x; r.v[1] = q.y;
    }
  } else {
    const float2 q = __ldg(reinterpret_cast<const float2*>(p));
    r.v[0] = q.x; r.v[1] = q.y;
  }
  return r;
}

template <typename R, int SPT>
__device__ __forceinline__ Pack<R, SPT> ld_stream(const Pack<R, SPT>* p) {
  Pack<R, SPT> r;
  if constexpr (sizeof(Pack<R, SPT>) == 16) {
    if constexpr (sizeof(R) == 4) {
      const float4 q = __ldcs(reinterpret_cast<const float4*>(p));
      r.v[0] = q.x; r.v[1] = q.y; r.v[2] = q.z; r.v[3] = q.w;
    } else {
      const double2 q = __ldcs(reinterpret_cast<const double2*>(p));
      r.v[0] = q.x; r.v[1] = q.y;
    }
  } else {
    const float2 q = __ldcs(reinterpret_cast<const float2*>(p));
    r.v[0] = q.x; r.v[1] = q.y;
  }
  return r;
}

template <typename R, int SPT>
__device__ __forceinline__ void st(Pack<R, SPT>* p, const Pack<R, SPT>& r) {
  if constexpr (sizeof(Pack<R, SPT>) == 16) {
    if constexpr (sizeof(R) == 4) {
      *reinterpret_cast<float4*>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    } else {
      *reinterpret_cast<double2*>(p) = make_double2(r.v[0], r.v[1]);
    }
  } else {
    *reinterpret_cast<float2*>(p) = make_float2(r.v[0], r.v[1]);
  }
}

template <typename R, int SPT>
__device__ __forceinline__ void st_stream(Pack<R, SPT>* p, const Pack<R, SPT>& r) {
  if constexpr (sizeof(Pack<R, SPT>) == 16) {
    if constexpr (sizeof(R) == 4) {
      __stcs(reinterpret_cast<float4*>(p), make_float4(r.v[0], r.v[1], r.v[2], r.v[3]));
    } else {
      __stcs(reinterpret_cast<double2*>(p), make_double2(r.v[0], r.v[1]));
    }
  } else {
    __stcs(reinterpret_cast<float2*>(p), make_float2(r.v[0], r.v[1]));
  }
}

// ------------------------------------------------------------------ accumulators
// Neumaier-compensated FP32 sum (complex64 path) or plain FP64 sum (complex128 path).
template <typename R>
struct Acc;

template <>
struct Acc<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = s + x;
    c += (fabsf(s) >= fabsf(x)) ? ((s - t) + x) : ((x - t) + s);
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s + (double)c; }
};

template <>
struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

// ------------------------------------------------------------------ grid reduction
// Every thread holds NV values for its states (states p*SPT .. p*SPT+SPT-1, C values each,
// p = threadIdx.x % P).  Sums them over the grid and calls fin(q, total) for q = s*C + c in
// the last block.  Deterministic: fixed trees and a fixed block order.
template <int NV, int SPT, int C, typename Fin>
__device__ __forceinline__ void grid_reduce(double (&v)[NV], int P, int S, double* partials,
                                            unsigned* counter, int nblocks, Fin fin) {
  static_assert(NV == SPT * C, "values per thread");
  __shared__ double red[kWarps][32][NV];
  __shared__ unsigned ticket;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    for (int off = 16; off >= P; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  }
  if (lane < P) {
#pragma unroll
    for (int k = 0; k < NV; ++k) red[warp][lane][k] = v[k];
  }
  __syncthreads();
  const int SC = S * C;
  if (threadIdx.x < SC) {
    const int q = threadIdx.x, s = q / C, c = q - s * C;
    const int p = s / SPT, k = (s - p * SPT) * C + c;
    double acc = 0.0;
    for (int w = 0; w < kWarps; ++w) acc += red[w][p][k];
    partials[(size_t)blockIdx.x * SC + q] = acc;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(counter, 1u);
  __syncthreads();
  if (ticket != (unsigned)(nblocks - 1)) return;
  // last block: sum the partials in block order, one warp per output value
  __threadfence();
  for (int q = warp; q < SC; q += kWarps) {
    double acc = 0.0;
    for (int b = lane; b < nblocks; b += 32) acc += __ldcg(partials + (size_t)b * SC + q);
    for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (lane == 0) fin(q, acc);
  }
  if (threadIdx.x == 0) *counter = 0u;
}


// Recurrence coefficients t/|H| and D (clean lattices) for the first (x1) or a regular (x2)
// term, in the kernel's precision.
template <typename R>
__device__ __forceinline__ R coef_th(const RecurrenceArgs& a, bool first);
template <>
__device__ __forceinline__ float coef_th<float>(const RecurrenceArgs& a, bool first) {
  return first ? a.th1f : a.th2f;
}
template <>
__device__ __forceinline__ double coef_th<double>(const RecurrenceArgs& a, bool first) {
  return first ? a.thop : 2.0 * a.thop;
}
template <typename R>
__device__ __forceinline__ R coef_dc(const RecurrenceArgs& a, bool first);
template <>
__device__ __forceinline__ float coef_dc<float>(const RecurrenceArgs& a, bool first) {
  return first ? a.dc1f : a.dc2f;
}
template <>
__device__ __forceinline__ double coef_dc<double>(const RecurrenceArgs& a, bool first) {
  return first ? a.diag_const : 2.0 * a.diag_const;
}

// ------------------------------------------------------------------ stencil lines
template <typename R>
struct Partial;
template <>
struct Partial<float> {
  float f = 0.f;
  double d = 0.0;
  __device__ __forceinline__ void add(float x) { f += x; }
  __device__ __forceinline__ void fold() { d += (double)f; f = 0.f; }
  __device__ __forceinline__ double value() const { return d + (double)f; }
};
template <>
struct Partial<double> {
  double d = 0.0;
  __device__ __forceinline__ void add(double x) { d += x; }
  __device__ __forceinline__ void fold() {}
  __device__ __forceinline__ double value() const { return d; }
};

// Unit bases of the line and of its neighbouring lines (-1 when an open boundary drops them).
struct LineBases {
  int64_t own, up, dn, zup, zdn;
};

template <int KIND>
__device__ __forceinline__ LineBases line_bases(const Geom& g, int64_t row, int64_t upr) {
  LineBases b;
  int64_t y = row, zc = 0;
  if constexpr (KIND == TBPM_CUBIC) {
    // rows = Ly*Lz < 2^31 on any lattice that fits the device: 32-bit division
    const uint32_t r32 = (uint32_t)row, ly = (uint32_t)g.Ly;
    const uint32_t z32 = r32 / ly;
    zc = z32;
    y = r32 - z32 * ly;
  }
  b.own = row * upr;
  int64_t r;
  r = (y + 1 < g.Ly) ? row + 1 : (g.pbc_y ? row + 1 - g.Ly : -1);
  b.up = r >= 0 ? r * upr : -1;
  r = (y > 0) ? row - 1 : (g.pbc_y ? row - 1 + g.Ly : -1);
  b.dn = r >= 0 ? r * upr : -1;
  b.zup = b.zdn = -1;
  if constexpr (KIND == TBPM_CUBIC) {
    const int64_t plane = g.Ly, vol = g.Ly * g.Lz;
    r = (zc + 1 < g.Lz) ? row + plane : (g.pbc_z ? row + plane - vol : -1);
    b.zup = r >= 0 ? r * upr : -1;
    r = (zc > 0) ? row - plane : (g.pbc_z ? row - plane + vol : -1);
    b.zdn = r >= 0 ? r * upr : -1;
  }
  return b;
}

// Neighbour unit offsets of in-line unit u (absolute, -1 = none); returns the count.
template <int KIND>
__device__ __forceinline__ int stencil_neighbours(const Geom& g, const LineBases& b, int u, int P, int logP,
                                                  int p, int upr, int64_t (&nb)[6]) {
  const int64_t Lx = g.Lx;
  if constexpr (KIND == TBPM_HONEYCOMB) {
    const int sir = u >> logP, s = sir & 1, xc = sir >> 1;
    nb[0] = b.own + (u ^ P);
    if (s) {
      nb[1] = (xc < Lx - 1) ? b.own + u + P : (g.pbc_x ? b.own + p : -1);
      nb[2] = b.up >= 0 ? b.up + u - P : -1;
    } else {
      nb[1] = (xc > 0) ? b.own + u - P : (g.pbc_x ? b.own + u - P + upr : -1);
      nb[2] = b.dn >= 0 ? b.dn + u + P : -1;
    }
    return 3;
  } else {
    const int xc = u >> logP;
    nb[0] = (xc < Lx - 1) ? b.own + u + P : (g.pbc_x ? b.own + p : -1);
    nb[1] = (xc > 0) ? b.own + u - P : (g.pbc_x ? b.own + u - P + upr : -1);
    nb[2] = b.up >= 0 ? b.up + u : -1;
    nb[3] = b.dn >= 0 ? b.dn + u : -1;
    if constexpr (KIND == TBPM_CUBIC) {
      nb[4] = b.zup >= 0 ? b.zup + u : -1;
      nb[5] = b.zdn >= 0 ? b.zdn + u : -1;
      return 6;
    }
    return 4;
  }
}


}  // namespace tbpm
