// C ABI of the library: context, lattice construction on the device, initial states, and
// the drivers of the three propagation forms of Sec. II.A (sequential, moment-based,
// state-based with time blocks) and of the spectra of Sec. III.
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <functional>
#include <vector>

#include "tbpm_internal.cuh"

namespace tbpm {

static thread_local char g_err[1024];

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}
void clear_error() { g_err[0] = 0; }

int ensure(tbpm_ctx* ctx, DevBuf& b, size_t bytes) {
  if (bytes <= b.cap) return TBPM_OK;
  if (b.p) {
    TBPM_CK(cudaFreeAsync(b.p, ctx->stream));
    b.p = nullptr;
    b.cap = 0;
  }
  const size_t want = std::max<size_t>(256, bytes + (bytes >> 4));
  cudaError_t e = cudaMallocAsync(&b.p, want, ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    set_error("device allocation of %zu bytes failed: %s", want, cudaGetErrorString(e));
    return TBPM_ENOMEM;
  }
  b.cap = want;
  return TBPM_OK;
}

static cudaEvent_t take_event(tbpm_ctx* ctx) {
  if (!ctx->event_pool.empty()) {
    cudaEvent_t e = ctx->event_pool.back();
    ctx->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

int phase_begin(tbpm_ctx* ctx, int kind) {
  static const char* const kNames[3] = {"recurrence", "reconstruction", "fused passes"};
  ctx->nvtx_open.push_back(nvtxRangeStartA(kNames[kind >= 0 && kind < 3 ? kind : 0]));
  if (!ctx->profiling) return -1;
  tbpm_ctx::Phase ph;
  ph.a = take_event(ctx);
  ph.b = take_event(ctx);
  ph.kind = kind;
  ph.launches = ctx->launches;
  cudaEventRecord(ph.a, ctx->stream);
  ctx->phases.push_back(ph);
  return (int)ctx->phases.size() - 1;
}

void phase_end(tbpm_ctx* ctx, int token) {
  if (!ctx->nvtx_open.empty()) {
    nvtxRangeEnd(ctx->nvtx_open.back());
    ctx->nvtx_open.pop_back();
  }
  if (token < 0 || token >= (int)ctx->phases.size()) return;
  tbpm_ctx::Phase& ph = ctx->phases[token];
  ph.launches = ctx->launches - ph.launches;
  cudaEventRecord(ph.b, ctx->stream);
}

static void release(tbpm_ctx* ctx, DevBuf& b) {
  if (b.p) cudaFreeAsync(b.p, ctx->stream);
  b.p = nullptr;
  b.cap = 0;
}

template <typename T>
static int dev_alloc(tbpm_ctx* ctx, T** p, size_t count) {
  cudaError_t e = cudaMallocAsync((void**)p, std::max<size_t>(1, count) * sizeof(T), ctx->stream);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    set_error("device allocation of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
    return TBPM_ENOMEM;
  }
  return TBPM_OK;
}

static int grid_for(tbpm_ctx* ctx, int64_t n, int threads, int per_sm = 16) {
  const int64_t b = (n + threads - 1) / threads;
  return (int)std::max<int64_t>(1, std::min<int64_t>(b, (int64_t)ctx->num_sms * per_sm));
}

// ------------------------------------------------------------------ lattice kernels
constexpr int kT = 256;

__device__ __forceinline__ double disorder_value(uint64_t seed, double W, int64_t i) {
  const uint32_t u = draw_u32(seed, (uint64_t)i, STREAM_DISORDER, 0);
  return W * ((double)(u >> 8) * 0x1p-24 - 0.5);
}

__device__ __forceinline__ bool vacant(uint64_t seed, uint64_t thr, int64_t i) {
  return (uint64_t)draw_u32(seed, (uint64_t)i, STREAM_VACANCY, 0) < thr;
}

struct Bounds3 {
  double emax, emin, deg;
};

__device__ __forceinline__ void block_bounds(Bounds3 v, Bounds3* part) {
  __shared__ Bounds3 sh[kT / 32];
  for (int off = 16; off >= 1; off >>= 1) {
    v.emax = fmax(v.emax, __shfl_xor_sync(0xffffffffu, v.emax, off));
    v.emin = fmin(v.emin, __shfl_xor_sync(0xffffffffu, v.emin, off));
    v.deg += __shfl_xor_sync(0xffffffffu, v.deg, off);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    Bounds3 r = sh[0];
    for (int w = 1; w < kT / 32; ++w) {
      r.emax = fmax(r.emax, sh[w].emax);
      r.emin = fmin(r.emin, sh[w].emin);
      r.deg += sh[w].deg;
    }
    part[blockIdx.x] = r;
  }
}

// Stencil path: V_i (FP64), degree and Gershgorin terms for every site.
__global__ void __launch_bounds__(kT) k_lattice_stencil(Geom g, uint64_t seed, double W, double abs_t,
                                                        double* v64, Bounds3* part) {
  Bounds3 acc{-INFINITY, INFINITY, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * kT + threadIdx.x; i < g.n_full; i += (int64_t)gridDim.x * kT) {
    int deg = 0;
    for (int d = 0; d < g.z; ++d) deg += neighbour_full(g, i, d) >= 0;
    const double v = (W != 0.0) ? disorder_value(seed, W, i) : 0.0;
    if (v64) v64[i] = v;
    acc.emax = fmax(acc.emax, v + deg * abs_t);
    acc.emin = fmin(acc.emin, v - deg * abs_t);
    acc.deg += deg;
  }
  block_bounds(acc, part);
}

__global__ void k_bounds_final(const Bounds3* part, int n, double* out) {
  __shared__ Bounds3 sh[kT];
  Bounds3 acc{-INFINITY, INFINITY, 0.0};
  for (int i = threadIdx.x; i < n; i += kT) {
    acc.emax = fmax(acc.emax, part[i].emax);
    acc.emin = fmin(acc.emin, part[i].emin);
    acc.deg += part[i].deg;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    Bounds3 r = sh[0];
    for (int w = 1; w < kT; ++w) {
      r.emax = fmax(r.emax, sh[w].emax);
      r.emin = fmin(r.emin, sh[w].emin);
      r.deg += sh[w].deg;
    }
    out[0] = r.emax;
    out[1] = r.emin;
    out[2] = r.deg;
  }
}

// CSR path, pass 1: active-site counts per chunk of kChunk sites.
constexpr int kPer = 16;
constexpr int kChunk = kT * kPer;

__global__ void __launch_bounds__(kT) k_count_active(int64_t n_full, uint64_t seed, uint64_t thr,
                                                     int64_t* counts) {
  __shared__ int64_t sh[kT / 32];
  const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kPer;
  int64_t c = 0;
  for (int q = 0; q < kPer; ++q) {
    const int64_t i = base + q;
    if (i < n_full && !vacant(seed, thr, i)) ++c;
  }
  for (int off = 16; off >= 1; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = c;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kT / 32; ++w) t += sh[w];
    counts[blockIdx.x] = t;
  }
}

// Exclusive scan of the chunk counts by one block: offs[0..n], offs[n] = total.
__global__ void k_scan_counts(const int64_t* counts, int64_t n, int64_t* offs) {
  __shared__ int64_t sh[1024];
  const int64_t per = (n + 1023) / 1024;
  const int64_t lo = threadIdx.x * per, hi = std::min<int64_t>(n, lo + per);
  int64_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += counts[i];
  sh[threadIdx.x] = s;
  __syncthreads();
  for (int off = 1; off < 1024; off <<= 1) {
    const int64_t v = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t run = sh[threadIdx.x] - s;  // exclusive prefix of this thread's segment
  for (int64_t i = lo; i < hi; ++i) {
    offs[i] = run;
    run += counts[i];
  }
  if (threadIdx.x == 1023) offs[n] = sh[1023];
}

// CSR path, pass 2: compact index of every site (-1 if vacant) and full index of every active site.
__global__ void __launch_bounds__(kT) k_compact(int64_t n_full, uint64_t seed, uint64_t thr,
                                                const int64_t* offs, int64_t* compact, int64_t* full_of) {
  __shared__ int64_t sh[kT];
  const int64_t base = (int64_t)blockIdx.x * kChunk + (int64_t)threadIdx.x * kPer;
  unsigned flags = 0;
  int c = 0;
  for (int q = 0; q < kPer; ++q) {
    const int64_t i = base + q;
    if (i < n_full && !vacant(seed, thr, i)) {
      flags |= 1u << q;
      ++c;
    }
  }
  sh[threadIdx.x] = c;
  __syncthreads();
  for (int off = 1; off < kT; off <<= 1) {
    const int64_t v = threadIdx.x >= off ? sh[threadIdx.x - off] : 0;
    __syncthreads();
    sh[threadIdx.x] += v;
    __syncthreads();
  }
  int64_t k = offs[blockIdx.x] + sh[threadIdx.x] - c;
  for (int q = 0; q < kPer; ++q) {
    const int64_t i = base + q;
    if (i >= n_full) break;
    if (flags & (1u << q)) {
      compact[i] = k;
      full_of[k] = i;
      ++k;
    } else {
      compact[i] = -1;
    }
  }
}

// CSR path, pass 3: ELL neighbour lists, V_i and Gershgorin terms of every active site.
__global__ void __launch_bounds__(kT) k_build_ell(Geom g, int64_t n, const int64_t* full_of,
                                                  const int64_t* compact, uint64_t seed, double W,
                                                  double abs_t, int32_t* ell, double* v64, Bounds3* part) {
  Bounds3 acc{-INFINITY, INFINITY, 0.0};
  for (int64_t k = (int64_t)blockIdx.x * kT + threadIdx.x; k < n; k += (int64_t)gridDim.x * kT) {
    const int64_t i = full_of[k];
    int deg = 0;
    for (int d = 0; d < g.z; ++d) {
      const int64_t j = neighbour_full(g, i, d);
      const int64_t cj = j >= 0 ? compact[j] : -1;
      ell[k * g.z + d] = (int32_t)cj;
      deg += cj >= 0;
    }
    const double v = (W != 0.0) ? disorder_value(seed, W, i) : 0.0;
    if (v64) v64[k] = v;
    acc.emax = fmax(acc.emax, v + deg * abs_t);
    acc.emin = fmin(acc.emin, v - deg * abs_t);
    acc.deg += deg;
  }
  block_bounds(acc, part);
}

// Long-range lattices, pass 3: ELL lists from the taps (dx, dy, dz, ds) of sublattice 0; a
// honeycomb B site takes every tap mirrored, (x-dx, y-dy) of sublattice 1-ds, so slot d has the
// same length and weight on both sublattices.  Periodic directions wrap by modulo, open ones
// drop the tap.  Gershgorin radius = sum of |t_d| over the slots that reach active sites.
__global__ void __launch_bounds__(kT) k_build_ell_taps(Geom g, int64_t n, const int64_t* full_of,
                                                       const int64_t* compact, const int4* taps, const double* tabs,
                                                       uint64_t seed, double W, int32_t* ell, double* v64,
                                                       Bounds3* part) {
  Bounds3 acc{-INFINITY, INFINITY, 0.0};
  const bool hc = g.kind == TBPM_HONEYCOMB;
  auto wrap = [](int64_t v, int64_t L, int periodic, bool* ok) -> int64_t {
    if (v >= 0 && v < L) return v;
    if (!periodic) { *ok = false; return 0; }
    const int64_t r = v % L;
    return r < 0 ? r + L : r;
  };
  for (int64_t k = (int64_t)blockIdx.x * kT + threadIdx.x; k < n; k += (int64_t)gridDim.x * kT) {
    const int64_t i = full_of[k];
    int64_t x, y, zc = 0;
    int s = 0;
    if (hc) {
      s = (int)(i & 1);
      const int64_t c = i >> 1;
      x = c % g.Lx;
      y = c / g.Lx;
    } else {
      x = i % g.Lx;
      y = (i / g.Lx) % g.Ly;
      zc = i / (g.Lx * g.Ly);
    }
    const int64_t sg = s ? -1 : 1;
    double rad = 0.0;
    int deg = 0;
    for (int d = 0; d < g.z; ++d) {
      const int4 tp = taps[d];
      bool ok = true;
      const int64_t tx = wrap(x + sg * tp.x, g.Lx, g.pbc_x, &ok);
      const int64_t ty = wrap(y + sg * tp.y, g.Ly, g.pbc_y, &ok);
      const int64_t tz = wrap(zc + sg * tp.z, g.Lz, g.pbc_z, &ok);
      int64_t cj = -1;
      if (ok) {
        const int64_t j = hc ? 2 * (ty * g.Lx + tx) + (s ? 1 - tp.w : tp.w) : (tz * g.Ly + ty) * g.Lx + tx;
        cj = compact[j];
      }
      if (ell) ell[k * g.z + d] = (int32_t)cj;
      if (cj >= 0) {
        rad += tabs[d];
        ++deg;
      }
    }
    const double v = (W != 0.0) ? disorder_value(seed, W, i) : 0.0;
    if (v64) v64[k] = v;
    acc.emax = fmax(acc.emax, v + rad);
    acc.emin = fmin(acc.emin, v - rad);
    acc.deg += deg;
  }
  block_bounds(acc, part);
}

// D_i = (V_i - H0)/|H| in FP64 and rounded once to FP32.
__global__ void k_make_diag(int64_t n, const double* v64, double H0, double half, double* d64, float* d32) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const double d = (v64[i] - H0) / half;
    if (d64) d64[i] = d;
    if (d32) d32[i] = (float)d;
  }
}

// ------------------------------------------------------------------ initial states
// Random phases psi_i = exp(2 pi i u / 2^32) / sqrt(N), u = Philox(state_seed; i, 2, s).
template <typename R>
__global__ void k_init_random(int64_t n, int Spad, int logS, int S, int s0, uint64_t seed, const int64_t* full_of,
                              double inv_sqrt_n, R* out, uint32_t* draws) {
  const int64_t total = n * Spad;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total;
       e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = e >> logS;
    const int s = (int)(e & (Spad - 1));
    R re = R(0), im = R(0);
    if (s < S) {
      const int64_t f = full_of ? full_of[k] : k;
      const uint32_t u = draw_u32(seed, (uint64_t)f, STREAM_PHASE, (uint32_t)(s0 + s));
      double sn, cs;
      sincospi((double)u * 0x1p-31, &sn, &cs);
      re = (R)(cs * inv_sqrt_n);
      im = (R)(sn * inv_sqrt_n);
      if (draws) draws[(int64_t)s * n + k] = u;
    }
    out[2 * e] = re;
    out[2 * e + 1] = im;
  }
}

template <typename R>
__global__ void k_init_sites(int64_t n, int Spad, int S, const int64_t* sites, R* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= S) return;
  out[2 * (sites[s] * Spad + s)] = R(1);
}

}  // namespace tbpm

using namespace tbpm;

// ====================================================================== C ABI
extern "C" {

const char* tbpm_last_error(void) { return g_err; }

int tbpm_create(tbpm_ctx** out, int device) {
  clear_error();
  if (!out) {
    set_error("tbpm_create: out is NULL");
    return TBPM_EINVAL;
  }
  *out = nullptr;
  int count = 0;
  TBPM_CK(cudaGetDeviceCount(&count));
  if (device < 0 || device >= count) {
    set_error("tbpm_create: device %d out of range (%d devices)", device, count);
    return TBPM_EINVAL;
  }
  TBPM_CK(cudaSetDevice(device));
  tbpm_ctx* ctx = new tbpm_ctx();
  ctx->device = device;
  cudaError_t e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaMallocHost((void**)&ctx->pinned, 4096);
  if (e == cudaSuccess) {
    // keep memory freed by stream-ordered frees in the pool instead of returning it to the
    // system at every synchronisation (re-mapping it made later allocations expensive)
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, device) == cudaSuccess) {
      uint64_t keep = UINT64_MAX;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    cudaGetLastError();
  }
  if (e != cudaSuccess) {
    set_error("tbpm_create: %s", cudaGetErrorString(e));
    delete ctx;
    return TBPM_ECUDA;
  }
  ctx->pinned_cap = 4096;
  memset(ctx->pinned, 0, ctx->pinned_cap);
  *out = ctx;
  return TBPM_OK;
}

int tbpm_destroy(tbpm_ctx* ctx) {
  clear_error();
  if (!ctx) return TBPM_OK;
  cudaSetDevice(ctx->device);
  DevBuf* bufs[] = {&ctx->ws_phi[0], &ctx->ws_phi[1], &ctx->ws_psi, &ctx->ws_acc, &ctx->ws_partials,
                    &ctx->ws_counter, &ctx->ws_mu, &ctx->ws_table, &ctx->ws_aux, &ctx->ws_out,
                    &ctx->ws_energies, &ctx->ws_recon, &ctx->ws_phi2[0], &ctx->ws_phi2[1],
                    &ctx->ws_fused_partials, &ctx->ws_qe, &ctx->ws_qe_coef, &ctx->ws_xdot, &ctx->ws_blk, &ctx->ws_blk_coef,
                    &ctx->ws_jpsi, &ctx->ws_ec, &ctx->ws_fermi};
  for (DevBuf* b : bufs) release(ctx, *b);
  cudaStreamSynchronize(ctx->stream);
  for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
  ctx->graphs.clear();
  for (auto& ph : ctx->phases) {
    cudaEventDestroy(ph.a);
    cudaEventDestroy(ph.b);
  }
  for (cudaEvent_t e : ctx->event_pool) cudaEventDestroy(e);
  for (cudaEvent_t e : ctx->queue_ev)
    if (e) cudaEventDestroy(e);
  if (ctx->pinned) cudaFreeHost(ctx->pinned);
  cudaStreamDestroy(ctx->stream);
  delete ctx;
  return TBPM_OK;
}

void* tbpm_stream(tbpm_ctx* ctx) { return ctx ? (void*)ctx->stream : nullptr; }

int tbpm_sync(tbpm_ctx* ctx) {
  clear_error();
  if (!ctx) {
    set_error("tbpm_sync: ctx is NULL");
    return TBPM_EINVAL;
  }
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return sweep_status(ctx);  // a fused sweep's bounded wait that expired since the last check
}

int64_t tbpm_launch_count(const tbpm_ctx* ctx) { return ctx ? ctx->launches : -1; }

int tbpm_set_fusion(tbpm_ctx* ctx, int enable) {
  clear_error();
  if (!ctx) {
    set_error("tbpm_set_fusion: ctx is NULL");
    return TBPM_EINVAL;
  }
  if (enable < -1 || enable > 10) {
    set_error("tbpm_set_fusion: mode %d unknown (-1..10)", enable);
    return TBPM_EINVAL;
  }
  ctx->fusion = enable;
  return TBPM_OK;
}

int tbpm_set_block_buffering(tbpm_ctx* ctx, int enable) {
  clear_error();
  if (!ctx) {
    set_error("tbpm_set_block_buffering: ctx is NULL");
    return TBPM_EINVAL;
  }
  ctx->buffer_blocks = enable != 0;
  return TBPM_OK;
}

int tbpm_set_graphs(tbpm_ctx* ctx, int enable) {
  clear_error();
  if (!ctx) {
    set_error("tbpm_set_graphs: ctx is NULL");
    return TBPM_EINVAL;
  }
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  ctx->use_graphs = enable != 0;
  if (!ctx->use_graphs) {
    for (auto& g : ctx->graphs) cudaGraphExecDestroy(g.exec);
    ctx->graphs.clear();
    ctx->graph_seen.clear();
  }
  return TBPM_OK;
}

int tbpm_fusion_report(tbpm_ctx* ctx, double ms_per_step[16]) {
  clear_error();
  if (!ctx || !ms_per_step) {
    set_error("tbpm_fusion_report: invalid argument");
    return TBPM_EINVAL;
  }
  for (int m = 0; m < 16; ++m) ms_per_step[m] = -1.0;
  for (auto& t : ctx->fusion_timings)
    if (t.first >= 0 && t.first < 16) ms_per_step[t.first] = t.second;
  return TBPM_OK;
}

int tbpm_set_pass_states(tbpm_ctx* ctx, int max_states) {
  clear_error();
  if (!ctx || max_states < 0) {
    set_error("tbpm_set_pass_states: invalid argument");
    return TBPM_EINVAL;
  }
  ctx->max_pass_states = max_states;
  return TBPM_OK;
}

int tbpm_profile(tbpm_ctx* ctx, int enable) {
  clear_error();
  if (!ctx) {
    set_error("tbpm_profile: ctx is NULL");
    return TBPM_EINVAL;
  }
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  for (auto& ph : ctx->phases) {
    ctx->event_pool.push_back(ph.a);
    ctx->event_pool.push_back(ph.b);
  }
  ctx->phases.clear();
  ctx->profiling = enable != 0;
  return TBPM_OK;
}

int tbpm_profile_read(tbpm_ctx* ctx, double out[6]) {
  clear_error();
  if (!ctx || !out) {
    set_error("tbpm_profile_read: NULL argument");
    return TBPM_EINVAL;
  }
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  for (int k = 0; k < 6; ++k) out[k] = 0.0;
  for (auto& ph : ctx->phases) {
    float ms = 0.f;
    TBPM_CK(cudaEventElapsedTime(&ms, ph.a, ph.b));
    out[2 * ph.kind] += ms;
    out[2 * ph.kind + 1] += (double)ph.launches;
  }
  return TBPM_OK;
}

int64_t tbpm_truncation_order(double tau) { return truncation_order_host(tau); }

}  // extern "C"

// ------------------------------------------------------------------ lattice construction
// Taps of a long-range lattice: every (dx, dy, dz, ds) from a site of sublattice 0 with
// 0 < r <= cutoff, in (dz, dy, dx, ds) order, and its weight t(r)/t = exp(-(r - 1)/decay).
// r^2 is exact in FP64 for these integer and half-integer coordinates.
static int make_taps(const tbpm_lattice_desc& d, std::vector<int>& off, std::vector<double>& wrel) {
  const bool hc = d.kind == TBPM_HONEYCOMB, cu = d.kind == TBPM_CUBIC;
  const int R = (int)ceil(d.cutoff) + 2;
  const double c2 = d.cutoff * d.cutoff;
  off.clear();
  wrel.clear();
  for (int dz = cu ? -R : 0; dz <= (cu ? R : 0); ++dz)
    for (int dy = -R; dy <= R; ++dy)
      for (int dx = -R; dx <= R; ++dx)
        for (int ds = 0; ds <= (hc ? 1 : 0); ++ds) {
          double r2;
          if (hc) {
            const double u = 1.5 * (dx + dy) + ds, v = (double)(dx - dy);
            r2 = u * u + 0.75 * v * v;
          } else {
            r2 = (double)dx * dx + (double)dy * dy + (double)dz * dz;
          }
          if (r2 == 0.0 || r2 > c2) continue;
          off.insert(off.end(), {dx, dy, dz, ds});
          wrel.push_back(exp(-(sqrt(r2) - 1.0) / d.decay));
        }
  if (wrel.empty()) {
    set_error("cutoff %g keeps no neighbour (nearest-neighbour distance is 1)", d.cutoff);
    return TBPM_EINVAL;
  }
  if (wrel.size() > 1024) {
    set_error("cutoff %g gives %zu neighbours per site (at most 1024)", d.cutoff, wrel.size());
    return TBPM_EUNSUPPORTED;
  }
  return TBPM_OK;
}

static int build_lattice(tbpm_ctx* ctx, tbpm_lattice* lat) {
  const tbpm_lattice_desc& d = lat->desc;
  Geom& g = lat->geom;
  g.kind = d.kind;
  g.Lx = d.L[0];
  g.Ly = d.kind == TBPM_CUBIC || d.kind == TBPM_SQUARE || d.kind == TBPM_HONEYCOMB ? d.L[1] : 1;
  g.Lz = d.kind == TBPM_CUBIC ? d.L[2] : 1;
  g.pbc_x = d.pbc[0] != 0;
  g.pbc_y = d.pbc[1] != 0;
  g.pbc_z = d.pbc[2] != 0;
  g.z = d.kind == TBPM_SQUARE ? 4 : d.kind == TBPM_HONEYCOMB ? 3 : 6;
  g.row_sites = d.kind == TBPM_HONEYCOMB ? 2 * g.Lx : g.Lx;
  g.n_rows = g.Ly * g.Lz;
  g.n_full = g.row_sites * g.n_rows;
  const double abs_t = fabs(d.t);
  const bool vac = d.vacancy_frac > 0.0;
  const bool lr = d.cutoff > 0.0;
  lat->path = (d.path == TBPM_PATH_AUTO) ? (vac || lr ? TBPM_PATH_CSR : TBPM_PATH_STENCIL) : d.path;
  if (vac && lat->path == TBPM_PATH_STENCIL) {
    set_error("vacancies need the CSR path");
    return TBPM_EINVAL;
  }
  if (lr && lat->path == TBPM_PATH_STENCIL) {
    set_error("long-range hopping runs on the CSR path");
    return TBPM_EINVAL;
  }
  std::vector<double> wrel;
  int4* d_taps = nullptr;
  double* d_tabs = nullptr;
  struct Release {  // frees the tap tables on every return path
    cudaStream_t st;
    int4** a;
    double** b;
    ~Release() {
      if (*a) cudaFreeAsync(*a, st);
      if (*b) cudaFreeAsync(*b, st);
    }
  } release{ctx->stream, &d_taps, &d_tabs};
  if (lr) {
    TBPM_TRY(make_taps(d, lat->tap_off, wrel));
    g.z = (int)wrel.size();
    lat->tap_t.resize(wrel.size());
    std::vector<double> tabs(wrel.size());
    std::vector<float> w32(wrel.size());
    for (size_t k = 0; k < wrel.size(); ++k) {
      lat->tap_t[k] = d.t * wrel[k];
      tabs[k] = abs_t * wrel[k];
      w32[k] = (float)wrel[k];
    }
    const size_t z = wrel.size();
    // current-operator weights t_k (r_j - r_i)_a per direction and sublattice; a honeycomb B site
    // takes every tap mirrored, so its bond vectors are the negatives
    std::vector<double> jw(6 * z);
    const double h = sqrt(3.0) / 2.0;
    for (size_t k = 0; k < z; ++k) {
      const int* o = &lat->tap_off[4 * k];
      double dv[3];
      if (d.kind == TBPM_HONEYCOMB) {
        dv[0] = 1.5 * (o[0] + o[1]) + o[3];
        dv[1] = h * (o[0] - o[1]);
        dv[2] = 0.0;
      } else {
        dv[0] = o[0];
        dv[1] = o[1];
        dv[2] = o[2];
      }
      for (int a = 0; a < 3; ++a) {
        jw[(a * 2 + 0) * z + k] = lat->tap_t[k] * dv[a];
        jw[(a * 2 + 1) * z + k] = (d.kind == TBPM_HONEYCOMB ? -1.0 : 1.0) * lat->tap_t[k] * dv[a];
      }
    }
    TBPM_TRY(dev_alloc(ctx, &lat->jw, 6 * z));
    TBPM_CK(cudaMemcpyAsync(lat->jw, jw.data(), 6 * z * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    TBPM_TRY(dev_alloc(ctx, &lat->wrel64, z));
    TBPM_TRY(dev_alloc(ctx, &lat->wrel32, z));
    TBPM_TRY(dev_alloc(ctx, &d_taps, z));
    TBPM_TRY(dev_alloc(ctx, &d_tabs, z));
    TBPM_CK(cudaMemcpyAsync(lat->wrel64, wrel.data(), z * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    TBPM_CK(cudaMemcpyAsync(lat->wrel32, w32.data(), z * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
    TBPM_CK(cudaMemcpyAsync(d_taps, lat->tap_off.data(), z * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream));
    TBPM_CK(cudaMemcpyAsync(d_tabs, tabs.data(), z * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
    // the pageable sources above must outlive the copies
    TBPM_CK(cudaStreamSynchronize(ctx->stream));
  }
  lat->has_v = d.W != 0.0;
  const uint64_t thr = vac ? (uint64_t)floor(d.vacancy_frac * 4294967296.0) : 0;

  TBPM_TRY(ensure(ctx, ctx->ws_aux, sizeof(Bounds3) * (size_t)ctx->num_sms * 16 + 64));
  Bounds3* part = (Bounds3*)ctx->ws_aux.p;
  int nb = 0;
  if (lat->path == TBPM_PATH_STENCIL) {
    lat->n_sites = g.n_full;
    if (lat->has_v) TBPM_TRY(dev_alloc(ctx, &lat->v64, lat->n_sites));
    nb = grid_for(ctx, g.n_full, kT);
    k_lattice_stencil<<<nb, kT, 0, ctx->stream>>>(g, d.seed, d.W, abs_t, lat->v64, part);
    TBPM_CK_LAUNCH(ctx);
  } else {
    const int64_t nchunks = (g.n_full + kChunk - 1) / kChunk;
    int64_t *counts = nullptr, *offs = nullptr;
    TBPM_TRY(dev_alloc(ctx, &counts, nchunks));
    TBPM_TRY(dev_alloc(ctx, &offs, nchunks + 1));
    k_count_active<<<(unsigned)nchunks, kT, 0, ctx->stream>>>(g.n_full, d.seed, thr, counts);
    TBPM_CK_LAUNCH(ctx);
    k_scan_counts<<<1, 1024, 0, ctx->stream>>>(counts, nchunks, offs);
    TBPM_CK_LAUNCH(ctx);
    int64_t n_active = 0;
    TBPM_CK(cudaMemcpyAsync(&n_active, offs + nchunks, sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    TBPM_CK(cudaStreamSynchronize(ctx->stream));
    if (n_active <= 0) {
      cudaFreeAsync(counts, ctx->stream);
      cudaFreeAsync(offs, ctx->stream);
      set_error("lattice has no active sites");
      return TBPM_EINVAL;
    }
    if (n_active >= (int64_t)INT32_MAX) {
      set_error("CSR path supports fewer than 2^31 active sites");
      return TBPM_EUNSUPPORTED;
    }
    lat->n_sites = n_active;
    TBPM_TRY(dev_alloc(ctx, &lat->compact, g.n_full));
    TBPM_TRY(dev_alloc(ctx, &lat->full_of, n_active));
    // clean long-range lattices that the tap kernel serves build their ELL lists only when a
    // pass needs them (complex128, one state, exports): at D_H ~ 230 they outweigh the states
    const bool lazy_ell = lr && d.path == TBPM_PATH_AUTO && !vac && d.kind != TBPM_CUBIC;
    if (!lazy_ell) TBPM_TRY(dev_alloc(ctx, &lat->ell, (size_t)n_active * g.z));
    if (lat->has_v) TBPM_TRY(dev_alloc(ctx, &lat->v64, n_active));
    k_compact<<<(unsigned)nchunks, kT, 0, ctx->stream>>>(g.n_full, d.seed, thr, offs, lat->compact, lat->full_of);
    TBPM_CK_LAUNCH(ctx);
    cudaFreeAsync(counts, ctx->stream);
    cudaFreeAsync(offs, ctx->stream);
    nb = grid_for(ctx, n_active, kT);
    if (lr) {
      k_build_ell_taps<<<nb, kT, 0, ctx->stream>>>(g, n_active, lat->full_of, lat->compact, d_taps, d_tabs, d.seed,
                                                    d.W, lat->ell, lat->v64, part);
      TBPM_CK_LAUNCH(ctx);
    } else {
      k_build_ell<<<nb, kT, 0, ctx->stream>>>(g, n_active, lat->full_of, lat->compact, d.seed, d.W, abs_t,
                                               lat->ell, lat->v64, part);
      TBPM_CK_LAUNCH(ctx);
    }
  }
  if (lr && d.path == TBPM_PATH_AUTO) TBPM_TRY(build_tap_chunks(ctx, lat));
  double* res = (double*)((char*)ctx->ws_aux.p + sizeof(Bounds3) * (size_t)ctx->num_sms * 16);
  k_bounds_final<<<1, kT, 0, ctx->stream>>>(part, nb, res);
  TBPM_CK_LAUNCH(ctx);
  TBPM_CK(cudaMemcpyAsync(ctx->pinned, res, 3 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  lat->E_max = ctx->pinned[0];
  lat->E_min = ctx->pinned[1];
  lat->n_bonds = (int64_t)ctx->pinned[2];
  if (!(lat->E_max > lat->E_min)) {
    set_error("degenerate spectrum (no hopping between active sites)");
    return TBPM_EINVAL;
  }
  lat->H0 = (lat->E_max + lat->E_min) / 2.0;
  lat->half = (1.0 + 0.01) * (lat->E_max - lat->E_min) / 2.0;
  if (lat->has_v) {
    TBPM_TRY(dev_alloc(ctx, &lat->d32, lat->n_sites));
    k_make_diag<<<grid_for(ctx, lat->n_sites, kT), kT, 0, ctx->stream>>>(lat->n_sites, lat->v64, lat->H0,
                                                                        lat->half, nullptr, lat->d32);
    TBPM_CK_LAUNCH(ctx);
  }
  return TBPM_OK;
}

// ELL lists of a long-range lattice built on first need (see build_lattice).
int tbpm::ensure_ell(tbpm_ctx* ctx, tbpm_lattice* lat) {
  if (lat->ell || lat->tap_t.empty()) return TBPM_OK;
  const Geom& g = lat->geom;
  const size_t z = lat->tap_t.size();
  std::vector<double> tabs(z);
  for (size_t k = 0; k < z; ++k) tabs[k] = fabs(lat->tap_t[k]);
  const int nb = grid_for(ctx, lat->n_sites, kT);
  int4* d_taps = nullptr;
  double* d_tabs = nullptr;
  Bounds3* part = nullptr;
  int r = dev_alloc(ctx, &lat->ell, (size_t)lat->n_sites * g.z);
  if (r == TBPM_OK) r = dev_alloc(ctx, &d_taps, z);
  if (r == TBPM_OK) r = dev_alloc(ctx, &d_tabs, z);
  if (r == TBPM_OK) r = dev_alloc(ctx, &part, (size_t)nb);
  if (r == TBPM_OK) {
    cudaMemcpyAsync(d_taps, lat->tap_off.data(), z * sizeof(int4), cudaMemcpyHostToDevice, ctx->stream);
    cudaMemcpyAsync(d_tabs, tabs.data(), z * sizeof(double), cudaMemcpyHostToDevice, ctx->stream);
    k_build_ell_taps<<<nb, kT, 0, ctx->stream>>>(g, lat->n_sites, lat->full_of, lat->compact, d_taps, d_tabs,
                                                  lat->desc.seed, lat->desc.W, lat->ell, nullptr, part);
    ctx->launches++;
    const cudaError_t e = cudaGetLastError();
    const cudaError_t es = cudaStreamSynchronize(ctx->stream);  // the host tables must outlive the copies
    if (e != cudaSuccess || es != cudaSuccess) {
      set_error("ELL build: %s", cudaGetErrorString(e != cudaSuccess ? e : es));
      r = TBPM_ECUDA;
    }
  }
  for (void* q : {(void*)d_taps, (void*)d_tabs, (void*)part})
    if (q) cudaFreeAsync(q, ctx->stream);
  if (r != TBPM_OK && lat->ell) {
    cudaFreeAsync(lat->ell, ctx->stream);
    lat->ell = nullptr;
  }
  return r;
}

static int ensure_d64(tbpm_lattice* lat) {
  if (!lat->has_v || lat->d64) return TBPM_OK;
  tbpm_ctx* ctx = lat->ctx;
  TBPM_TRY(dev_alloc(ctx, &lat->d64, lat->n_sites));
  k_make_diag<<<grid_for(ctx, lat->n_sites, kT), kT, 0, ctx->stream>>>(lat->n_sites, lat->v64, lat->H0, lat->half,
                                                                      lat->d64, nullptr);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

static void free_lattice_mem(tbpm_lattice* lat) {
  tbpm_ctx* ctx = lat->ctx;
  void* ps[] = {lat->d32, lat->d64, lat->v64, lat->ell, lat->compact, lat->full_of, lat->wrel32, lat->wrel64,
                lat->chunks, lat->jw};
  for (void* p : ps)
    if (p) cudaFreeAsync(p, ctx->stream);
}

extern "C" {

int tbpm_lattice_create(tbpm_ctx* ctx, const tbpm_lattice_desc* desc, tbpm_lattice** out) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !desc || !out) {
    set_error("tbpm_lattice_create: NULL argument");
    return TBPM_EINVAL;
  }
  *out = nullptr;
  const tbpm_lattice_desc& d = *desc;
  if (d.kind < TBPM_SQUARE || d.kind > TBPM_CUBIC) {
    set_error("unknown lattice kind %d", d.kind);
    return TBPM_EINVAL;
  }
  const int dims = d.kind == TBPM_CUBIC ? 3 : 2;
  for (int k = 0; k < dims; ++k)
    if (d.L[k] < 1 || d.L[k] > (1LL << 31)) {
      set_error("lattice size L[%d] = %lld out of range", k, (long long)d.L[k]);
      return TBPM_EINVAL;
    }
  if (!(d.t == d.t) || d.t == 0.0 || !isfinite(d.t) || !isfinite(d.W) || d.W < 0.0) {
    set_error("hopping t must be finite and non-zero, W finite and >= 0");
    return TBPM_EINVAL;
  }
  if (!(d.vacancy_frac >= 0.0 && d.vacancy_frac < 1.0)) {
    set_error("vacancy_frac must lie in [0, 1)");
    return TBPM_EINVAL;
  }
  if (!(d.cutoff >= 0.0 && d.cutoff <= 12.0) || (d.cutoff > 0.0 && !(d.decay > 0.0 && isfinite(d.decay)))) {
    set_error("cutoff must lie in [0, 12], and decay be finite and > 0 when cutoff > 0");
    return TBPM_EINVAL;
  }
  if (d.path < TBPM_PATH_AUTO || d.path > TBPM_PATH_CSR) {
    set_error("unknown path %d", d.path);
    return TBPM_EINVAL;
  }
  if (d.kind == TBPM_CUBIC && (double)d.L[1] * (double)d.L[2] >= 2147483648.0) {
    set_error("cubic lattice: Ly*Lz must be below 2^31");
    return TBPM_EINVAL;
  }
  double nf = (double)d.L[0] * (double)d.L[1] * (d.kind == TBPM_CUBIC ? (double)d.L[2] : 1.0) *
              (d.kind == TBPM_HONEYCOMB ? 2.0 : 1.0);
  if (nf > 4.0e9) {
    set_error("lattice too large (%.3g sites)", nf);
    return TBPM_EINVAL;
  }
  TBPM_CK(cudaSetDevice(ctx->device));
  tbpm_lattice* lat = new tbpm_lattice();
  lat->ctx = ctx;
  lat->desc = d;
  if (d.kind != TBPM_CUBIC) lat->desc.L[2] = 1;
  int r = build_lattice(ctx, lat);
  if (r != TBPM_OK) {
    free_lattice_mem(lat);
    delete lat;
    return r;
  }
  *out = lat;
  return TBPM_OK;
}

int tbpm_lattice_destroy(tbpm_lattice* lat) {
  clear_error();
  if (!lat) return TBPM_OK;
  tbpm_ctx* ctx = lat->ctx;
  cudaSetDevice(ctx->device);
  free_lattice_mem(lat);
  cudaStreamSynchronize(lat->ctx->stream);
  delete lat;
  return TBPM_OK;
}

int tbpm_lattice_info(const tbpm_lattice* lat, tbpm_lattice_props* out) {
  clear_error();
  if (!lat || !out) {
    set_error("tbpm_lattice_info: NULL argument");
    return TBPM_EINVAL;
  }
  out->n_full = lat->geom.n_full;
  out->n_sites = lat->n_sites;
  out->n_bonds = lat->n_bonds;
  out->path = lat->path;
  out->coordination = lat->geom.z;
  out->E_min = lat->E_min;
  out->E_max = lat->E_max;
  out->H0 = lat->H0;
  out->half_width = lat->half;
  return TBPM_OK;
}

int tbpm_lattice_export(const tbpm_lattice* lat, int64_t* compact, double* V, int32_t* nbr) {
  clear_error();
  if (!lat) {
    set_error("tbpm_lattice_export: NULL lattice");
    return TBPM_EINVAL;
  }
  tbpm_ctx* ctx = lat->ctx;
  TBPM_CK(cudaSetDevice(ctx->device));
  const int64_t n = lat->n_sites, nf = lat->geom.n_full;
  const int z = lat->geom.z;
  if (compact) {
    if (lat->compact) {
      TBPM_CK(cudaMemcpyAsync(compact, lat->compact, nf * sizeof(int64_t), cudaMemcpyDeviceToHost, ctx->stream));
    } else {
      for (int64_t i = 0; i < nf; ++i) compact[i] = i;
    }
  }
  if (V) {
    if (lat->v64) {
      TBPM_CK(cudaMemcpyAsync(V, lat->v64, n * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    } else {
      for (int64_t i = 0; i < n; ++i) V[i] = 0.0;
    }
  }
  if (nbr) {
    TBPM_TRY(ensure_ell(ctx, const_cast<tbpm_lattice*>(lat)));
    if (lat->ell) {
      TBPM_CK(cudaMemcpyAsync(nbr, lat->ell, n * z * sizeof(int32_t), cudaMemcpyDeviceToHost, ctx->stream));
    } else {
      for (int64_t i = 0; i < n; ++i)
        for (int d = 0; d < z; ++d) nbr[i * z + d] = (int32_t)neighbour_full(lat->geom, i, d);
    }
  }
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return TBPM_OK;
}

int tbpm_debug_status(tbpm_ctx* ctx, uint64_t words[3]) {
  clear_error();
  if (!ctx || !words) {
    set_error("tbpm_debug_status: NULL argument");
    return TBPM_EINVAL;
  }
#ifdef TBPM_DEBUG
  TBPM_CK(cudaSetDevice(ctx->device));
  TBPM_CK(cudaDeviceSynchronize());
  words[0] = debug_take_cheb();
  words[1] = debug_take_sweep();
  words[2] = debug_take_serve();
  return TBPM_OK;
#else
  words[0] = words[1] = words[2] = 0;
  set_error("tbpm_debug_status: this library was built without TBPM_DEBUG (use libtbpm_debug.so)");
  return TBPM_EUNSUPPORTED;
#endif
}

int tbpm_lattice_taps(const tbpm_lattice* lat, int32_t* offsets, double* t) {
  clear_error();
  if (!lat) {
    set_error("tbpm_lattice_taps: NULL lattice");
    return TBPM_EINVAL;
  }
  const int z = lat->geom.z;
  if (!lat->tap_t.empty()) {
    if (offsets)
      for (int k = 0; k < 4 * z; ++k) offsets[k] = lat->tap_off[k];
    if (t)
      for (int k = 0; k < z; ++k) t[k] = lat->tap_t[k];
    return TBPM_OK;
  }
  // nearest-neighbour lattices: the fixed neighbour order of a sublattice-0 site
  static const int sq[4][4] = {{1, 0, 0, 0}, {-1, 0, 0, 0}, {0, 1, 0, 0}, {0, -1, 0, 0}};
  static const int hc[3][4] = {{0, 0, 0, 1}, {-1, 0, 0, 1}, {0, -1, 0, 1}};
  static const int cu[6][4] = {{1, 0, 0, 0}, {-1, 0, 0, 0}, {0, 1, 0, 0}, {0, -1, 0, 0}, {0, 0, 1, 0}, {0, 0, -1, 0}};
  const int(*tab)[4] = lat->geom.kind == TBPM_SQUARE ? sq : lat->geom.kind == TBPM_HONEYCOMB ? hc : cu;
  for (int d = 0; d < z; ++d) {
    if (offsets)
      for (int c = 0; c < 4; ++c) offsets[4 * d + c] = tab[d][c];
    if (t) t[d] = lat->desc.t;
  }
  return TBPM_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ request plumbing
namespace {

struct Plan {
  int precision;
  int S, Spad, logS, spt, P, logP;
  size_t elem;        // bytes per complex element
  size_t state_bytes; // one block of Spad states
  double tau;
  int s0;             // index of the block's first state among the request's states (Philox sub-stream)
};

int ilog2(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

int make_plan(const tbpm_lattice* lat, const tbpm_request* req, Plan* pl) {
  if (!lat || !req) {
    set_error("NULL lattice or request");
    return TBPM_EINVAL;
  }
  if (req->precision != TBPM_C64 && req->precision != TBPM_C128) {
    set_error("unknown precision %d", req->precision);
    return TBPM_EINVAL;
  }
  if (req->n_states < 1 || req->n_states > 32) {
    set_error("n_states must lie in [1, 32] (got %d)", req->n_states);
    return TBPM_EINVAL;
  }
  if (req->states == TBPM_STATES_SITES) {
    if (!req->sites) {
      set_error("site states need a site list");
      return TBPM_EINVAL;
    }
    for (int s = 0; s < req->n_states; ++s)
      if (req->sites[s] < 0 || req->sites[s] >= lat->n_sites) {
        set_error("site %lld out of range", (long long)req->sites[s]);
        return TBPM_EINVAL;
      }
  } else if (req->states != TBPM_STATES_RANDOM) {
    set_error("unknown state kind %d", req->states);
    return TBPM_EINVAL;
  }
  pl->precision = req->precision;
  pl->S = req->n_states;
  pl->logS = ilog2(pl->S);
  pl->Spad = 1 << pl->logS;
  pl->spt = (req->precision == TBPM_C64 && pl->Spad >= 2) ? 2 : 1;
  pl->P = pl->Spad / pl->spt;
  pl->logP = ilog2(pl->P);
  pl->elem = req->precision == TBPM_C64 ? 8 : 16;
  pl->state_bytes = (size_t)lat->n_sites * pl->Spad * pl->elem;
  pl->tau = req->tau == 0.0 ? M_PI : req->tau;
  pl->s0 = 0;
  if (!(pl->tau > 0.0) || !isfinite(pl->tau)) {
    set_error("tau must be positive");
    return TBPM_EINVAL;
  }
  return TBPM_OK;
}

int init_states(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, void* dst,
                uint32_t* draws) {
  const int64_t n = lat->n_sites;
  if (req->states == TBPM_STATES_RANDOM) {
    const double inv = 1.0 / sqrt((double)n);
    const int nb = grid_for(ctx, n * pl.Spad, kT, 32);
    if (pl.precision == TBPM_C64)
      k_init_random<float><<<nb, kT, 0, ctx->stream>>>(n, pl.Spad, pl.logS, pl.S, pl.s0, req->state_seed, lat->full_of,
                                                       inv, (float*)dst, draws);
    else
      k_init_random<double><<<nb, kT, 0, ctx->stream>>>(n, pl.Spad, pl.logS, pl.S, pl.s0, req->state_seed, lat->full_of,
                                                        inv, (double*)dst, draws);
    TBPM_CK_LAUNCH(ctx);
  } else {
    TBPM_CK(cudaMemsetAsync(dst, 0, pl.state_bytes, ctx->stream));
    TBPM_TRY(ensure(ctx, ctx->ws_aux, sizeof(int64_t) * 32));
    TBPM_CK(cudaMemcpyAsync(ctx->ws_aux.p, req->sites, sizeof(int64_t) * pl.S, cudaMemcpyHostToDevice, ctx->stream));
    if (pl.precision == TBPM_C64)
      k_init_sites<float><<<1, 32, 0, ctx->stream>>>(n, pl.Spad, pl.S, (const int64_t*)ctx->ws_aux.p, (float*)dst);
    else
      k_init_sites<double><<<1, 32, 0, ctx->stream>>>(n, pl.Spad, pl.S, (const int64_t*)ctx->ws_aux.p, (double*)dst);
    TBPM_CK_LAUNCH(ctx);
  }
  return TBPM_OK;
}

int64_t tiles_of(const tbpm_lattice* lat, const Plan& pl) {
  if (lat->path == TBPM_PATH_CSR) return (lat->n_sites * pl.P + 255) / 256;
  return lat->geom.n_rows * ((lat->geom.row_sites * pl.P + 255) / 256);
}

int base_args(tbpm_ctx* ctx, tbpm_lattice* lat, const Plan& pl, RecurrenceArgs* a, int comps) {
  memset(a, 0, sizeof(*a));
  a->geom = lat->geom;
  a->path = lat->path;
  a->wrel = lat->wrel64 ? (pl.precision == TBPM_C128 ? (const void*)lat->wrel64 : (const void*)lat->wrel32) : nullptr;
  if (lat->chunks && pl.precision == TBPM_C64 && pl.Spad >= 2) {
    a->taps = lat->chunks;
    a->taps_n0 = lat->n_chunks[0];
    a->taps_n1 = lat->n_chunks[1];
    a->taps_rx = lat->halo_x;
    a->taps_ry = lat->halo_y;
    a->taps_exact = lat->tap_exact ? 1 : 0;
  }
  if (!a->taps) TBPM_TRY(ensure_ell(ctx, lat));
  a->ell = lat->ell;
  if (lat->has_v) {
    if (pl.precision == TBPM_C128) TBPM_TRY(ensure_d64(lat));
    a->diag = pl.precision == TBPM_C128 ? (const void*)lat->d64 : (const void*)lat->d32;
  } else {
    a->diag = nullptr;
  }
  a->diag_const = (0.0 - lat->H0) / lat->half;
  a->thop = lat->desc.t / lat->half;
  set_float_coefficients(a);
  a->n_sites = lat->n_sites;
  a->S = pl.Spad;
  a->P = pl.P;
  a->logP = pl.logP;
  a->n_tiles = tiles_of(lat, pl);
  a->nblocks = recurrence_blocks(ctx, pl.precision, pl.Spad);
  TBPM_TRY(ensure(ctx, ctx->ws_partials, sizeof(double) * (size_t)a->nblocks * pl.Spad * comps));
  a->partials = (double*)ctx->ws_partials.p;
  if (!ctx->ws_counter.p) {
    TBPM_TRY(ensure(ctx, ctx->ws_counter, 256));
    TBPM_CK(cudaMemsetAsync(ctx->ws_counter.p, 0, ctx->ws_counter.cap, ctx->stream));
  }
  a->counter = (unsigned*)ctx->ws_counter.p;
  if (a->taps) {
    TBPM_TRY(ensure(ctx, ctx->ws_fused_partials, taps_partials_bytes(*a)));
    a->tap_partials = (double*)ctx->ws_fused_partials.p;
  }
  return TBPM_OK;
}

// Fusion mode for a moment request: ctx->fusion, or under -1 the fastest mode measured on this
// lattice shape (a few passes of each applicable mode on scratch buffers; cached per shape).
int choose_fusion(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, int64_t M, int* mode) {
  if (ctx->fusion >= 0) {
    *mode = ctx->fusion;
    return TBPM_OK;
  }
  *mode = 0;
  if (!fused_applicable(lat, pl.precision, pl.Spad) || M / 2 < 64) return TBPM_OK;
  const Geom& g = lat->geom;
  const std::vector<int64_t> key = {g.kind, g.Lx, g.Ly, g.Lz, g.pbc_x | (g.pbc_y << 1) | (g.pbc_z << 2), lat->path,
                                    pl.Spad, pl.precision, lat->has_v ? 1 : 0};
  for (auto& kv : ctx->fusion_choice)
    if (kv.first == key) {
      *mode = kv.second;
      return TBPM_OK;
    }
  TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi2[0], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi2[1], pl.state_bytes));
  const int Ms = 64;  // scratch moments: steps 1 .. 31
  TBPM_TRY(ensure(ctx, ctx->ws_aux, sizeof(double) * 2 * (size_t)Ms * pl.Spad));
  TBPM_CK(cudaMemsetAsync(ctx->ws_aux.p, 0, sizeof(double) * 2 * (size_t)Ms * pl.Spad, ctx->stream));
  TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_phi[0].p, nullptr));
  TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_phi[1].p, nullptr));
  RecurrenceArgs a;
  TBPM_TRY(base_args(ctx, lat, pl, &a, 3));
  a.mu = (double*)ctx->ws_aux.p;
  a.M = Ms;
  cudaEvent_t e0, e1;
  TBPM_CK(cudaEventCreate(&e0));
  TBPM_CK(cudaEventCreate(&e1));
  const int modes[] = {0, 4, 5, 8};
  double best_ms = 1e300;
  ctx->fusion_timings.clear();
  // 24 steps per mode after 8 warm-up steps (multiples of every mode's steps per pass)
  int r = TBPM_OK;
  for (int m : modes) {
    const int K = m == 0 ? 1 : fused_steps(m);
    const int passes = 24 / K;  // 24 steps per measurement, after 8 warm-up steps
    float ms = 0.f;
    for (int rep = 0; rep < 2 && r == TBPM_OK; ++rep) {
      const int np = rep == 0 ? 8 / K : passes;
      if (rep == 1) cudaEventRecord(e0, ctx->stream);
      for (int i = 0; i < np && r == TBPM_OK; ++i) {
        if (m == 0) {
          a.cur = ctx->ws_phi[0].p;
          a.prev_out = ctx->ws_phi[1].p;
          a.step = 1 + (i % 16);
          r = launch_moment_step(ctx, a, pl.precision, false);
        } else {
          r = launch_fused_pass(ctx, lat, a, ctx->ws_phi[0].p, ctx->ws_phi[1].p, ctx->ws_phi2[0].p, ctx->ws_phi2[1].p,
                                1 + (i % 8) * K, m);
        }
      }
      if (rep == 1) cudaEventRecord(e1, ctx->stream);
    }
    if (r != TBPM_OK) break;
    if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    const double per_step = ms / 24.0;
    ctx->fusion_timings.push_back({m, per_step});
    if (per_step < best_ms) {
      best_ms = per_step;
      *mode = m;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  TBPM_TRY(r);
  ctx->fusion_choice.push_back({key, *mode});
  return TBPM_OK;
}

// Bounded launch queue (ctx->max_queue > 0, never while a graph is being captured): every 64
// launches record an event and wait for the one recorded 64 launches before.
void throttle_queue(tbpm_ctx* ctx, bool capturing) {
  if (ctx->max_queue <= 0 || capturing) return;
  if (++ctx->queue_count % 64 != 0) return;
  const int k = (int)((ctx->queue_count / 64) & 1);
  if (!ctx->queue_ev[k]) cudaEventCreateWithFlags(&ctx->queue_ev[k], cudaEventDisableTiming);
  if (ctx->queue_live[k]) cudaEventSynchronize(ctx->queue_ev[k]);
  cudaEventRecord(ctx->queue_ev[k], ctx->stream);
  ctx->queue_live[k] = true;
}

// Moments of all Spad states into d_mu [Spad][M][2].
int run_moments(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, int64_t M,
                double* d_mu) {
  if (M < 2 || (M & 1)) {
    set_error("n_moments must be even and >= 2 (got %lld)", (long long)M);
    return TBPM_EINVAL;
  }
  TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pl.state_bytes));
  TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_phi[0].p, nullptr));
  RecurrenceArgs a;
  TBPM_TRY(base_args(ctx, lat, pl, &a, 3));
  a.mu = d_mu;
  a.M = (int)M;
  int fmode = 0;
  TBPM_TRY(choose_fusion(ctx, lat, req, pl, M, &fmode));
  const int K = fused_steps(fmode);
  const bool fuse = fmode > 0 && fused_applicable(lat, pl.precision, pl.Spad) && M / 2 - 1 >= K;
  if (fuse) {
    TBPM_TRY(ensure(ctx, ctx->ws_phi2[0], pl.state_bytes));
    TBPM_TRY(ensure(ctx, ctx->ws_phi2[1], pl.state_bytes));
  }
  // the pass sequence: step n reads cur = phi_n and overwrites prev (phi_{n-1}) with phi_{n+1}
  bool capturing = false;
  auto body = [&]() -> int {
    void* cur = ctx->ws_phi[0].p;
    void* prev = ctx->ws_phi[1].p;
    int64_t n = 0;
    auto unfused = [&]() -> int {
      a.cur = cur;
      a.prev_out = prev;
      a.step = (int)n;
      TBPM_TRY(launch_moment_step(ctx, a, pl.precision, n == 0));
      throttle_queue(ctx, capturing);
      std::swap(cur, prev);
      ++n;
      return TBPM_OK;
    };
    TBPM_TRY(unfused());  // phi_1 = H~ phi_0, m_0, m_1
    if (fuse) {
      const int ftok = phase_begin(ctx, 2);
      void* pair_out[2] = {ctx->ws_phi2[0].p, ctx->ws_phi2[1].p};
      while (n + K <= M / 2) {
        TBPM_TRY(launch_fused_pass(ctx, lat, a, prev, cur, pair_out[0], pair_out[1], (int)n, fmode));
        throttle_queue(ctx, capturing);
        void* old_prev = prev;
        void* old_cur = cur;
        prev = pair_out[0];
        cur = pair_out[1];
        pair_out[0] = old_prev;
        pair_out[1] = old_cur;
        n += K;
      }
      phase_end(ctx, ftok);
    }
    while (n < M / 2) TBPM_TRY(unfused());
    return TBPM_OK;
  };
  const int tok = phase_begin(ctx, 0);
  if (!ctx->use_graphs || ctx->profiling) {
    TBPM_TRY(body());
  } else {
    auto bits = [](double v) {
      uint64_t u;
      memcpy(&u, &v, 8);
      return u;
    };
    const Geom& g = lat->geom;
    // every device pointer the captured passes read must be part of the key: a graph replays
    // only where those same addresses are allocated again (a lattice created anew at the same
    // addresses holds the same data there); a missing one would replay freed memory
    const std::vector<uint64_t> key = {
        (uint64_t)ctx->ws_phi[0].p, (uint64_t)ctx->ws_phi[1].p, (uint64_t)ctx->ws_phi2[0].p,
        (uint64_t)ctx->ws_phi2[1].p, (uint64_t)d_mu, (uint64_t)lat, (uint64_t)lat->d32, (uint64_t)lat->d64,
        (uint64_t)lat->ell, (uint64_t)a.partials, (uint64_t)a.counter, (uint64_t)ctx->ws_fused_partials.p,
        (uint64_t)M, (uint64_t)fmode, (uint64_t)pl.precision, (uint64_t)pl.Spad, bits(a.thop), bits(a.diag_const),
        (uint64_t)g.Lx, (uint64_t)g.Ly, (uint64_t)g.Lz, (uint64_t)g.kind,
        (uint64_t)(g.pbc_x | (g.pbc_y << 1) | (g.pbc_z << 2)), (uint64_t)lat->path, (uint64_t)lat->n_sites,
        (uint64_t)lat->chunks, (uint64_t)a.taps_rx, (uint64_t)a.taps_ry, (uint64_t)a.taps_n0, (uint64_t)a.taps_n1,
        (uint64_t)a.taps_exact,
        (uint64_t)lat->wrel32, (uint64_t)lat->wrel64};
    tbpm_ctx::Graph* hit = nullptr;
    for (auto& e : ctx->graphs)
      if (e.key == key) hit = &e;
    if (!hit) {
      bool seen = false;
      for (auto& k : ctx->graph_seen) seen = seen || k == key;
      if (!seen) {
        // first time: run eagerly (this also sizes every workspace the sequence touches)
        if (ctx->graph_seen.size() >= 16) ctx->graph_seen.erase(ctx->graph_seen.begin());
        ctx->graph_seen.push_back(key);
        TBPM_TRY(body());
      } else {
        cudaGraph_t graph = nullptr;
        const int64_t l0 = ctx->launches;
        TBPM_CK(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
        capturing = true;
        const int r = body();
        capturing = false;
        const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
        const int64_t kernels = ctx->launches - l0;
        ctx->launches = l0;
        if (r != TBPM_OK) {
          if (graph) cudaGraphDestroy(graph);
          return r;
        }
        TBPM_CK(ec);
        cudaGraphExec_t exec = nullptr;
        const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        TBPM_CK(ei);
        if (ctx->graphs.size() >= 8) {
          cudaGraphExecDestroy(ctx->graphs.front().exec);
          ctx->graphs.erase(ctx->graphs.begin());
        }
        ctx->graphs.push_back({key, exec, kernels});
        hit = &ctx->graphs.back();
      }
    }
    if (hit) {
      TBPM_CK(cudaGraphLaunch(hit->exec, ctx->stream));
      ctx->launches += hit->kernels;
    }
  }
  phase_end(ctx, tok);
  return TBPM_OK;
}

// Coefficient table of one time block of bb steps: coef[n][j] = exp(-i shift (j+1) tau) c_n((j+1) tau),
// zero once n >= N((j+1) tau).  n_per[j] = N((j+1) tau).
void block_coefficients(double tau, double shift, int bb, std::vector<double>* coef, std::vector<int>* n_per) {
  n_per->resize(bb);
  for (int j = 0; j < bb; ++j) (*n_per)[j] = (int)truncation_order_host((j + 1) * tau);
  const int nt = *std::max_element(n_per->begin(), n_per->end());
  coef->assign((size_t)nt * bb * 2, 0.0);
  std::vector<double> J(nt + 1);
  for (int j = 0; j < bb; ++j) {
    const double x = (j + 1) * tau;
    bessel_j_host(x, nt, J.data());
    double ps, pc;
    sincos(-shift * x, &ps, &pc);
    for (int n = 0; n < (*n_per)[j]; ++n) {
      const double a = n == 0 ? J[0] : 2.0 * J[n];
      double cr = 0, ci = 0;
      switch (n & 3) {
        case 0: cr = a; break;
        case 1: ci = -a; break;
        case 2: cr = -a; break;
        default: ci = a; break;
      }
      (*coef)[((size_t)n * bb + j) * 2] = pc * cr - ps * ci;
      (*coef)[((size_t)n * bb + j) * 2 + 1] = pc * ci + ps * cr;
    }
  }
}

// Largest b whose accumulators fit in 80% of the free device memory (and <= 256, <= n_steps).
int64_t block_cap(const Plan& pl, int64_t n_steps) {
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  const int64_t by_mem = (int64_t)std::max<double>(1.0, 0.8 * (double)free_b / (double)pl.state_bytes - 4.0 - 34.0);
  return std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(by_mem, 256), n_steps));
}

// Measured per-pass costs of the state-based form (Sec. II.B: "obtained via benchmarking prior
// to the main calculation"): t_amxsy = one recurrence pass with no accumulator open,
// t_axpy = the extra time per open accumulator.  Times in milliseconds.
int measure_pass_costs(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, int k_acc,
                       double* t_amxsy, double* t_axpy) {
  TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_psi, pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_acc, pl.state_bytes * (size_t)k_acc));
  TBPM_TRY(ensure(ctx, ctx->ws_table, sizeof(double) * 2 * (size_t)k_acc));
  TBPM_CK(cudaMemsetAsync(ctx->ws_table.p, 0, sizeof(double) * 2 * (size_t)k_acc, ctx->stream));
  TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_phi[0].p, nullptr));
  TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_phi[1].p, nullptr));
  TBPM_CK(cudaMemsetAsync(ctx->ws_acc.p, 0, pl.state_bytes * (size_t)k_acc, ctx->stream));
  AccumArgs g;
  memset(&g, 0, sizeof(g));
  TBPM_TRY(base_args(ctx, lat, pl, &g.r, 3));
  g.acc = ctx->ws_acc.p;
  g.acc_stride = lat->n_sites * (int64_t)pl.Spad;
  g.coef = (const double*)ctx->ws_table.p;
  g.psi = ctx->ws_psi.p;
  g.j_done = -1;
  g.r.cur = ctx->ws_phi[0].p;
  g.r.prev_out = ctx->ws_phi[1].p;
  cudaEvent_t e[3];
  for (auto& x : e) TBPM_CK(cudaEventCreate(&x));
  const int reps = 3;
  float ms0 = 0.f, ms1 = 0.f;
  int r = TBPM_OK;
  for (int pass = 0; pass < 2 && r == TBPM_OK; ++pass) {   // pass 0 warms up
    g.b = 0;
    g.j_lo = 0;
    cudaEventRecord(e[0], ctx->stream);
    for (int i = 0; i < reps && r == TBPM_OK; ++i) r = launch_accum_step(ctx, g, pl.precision, ACC_REGULAR);
    cudaEventRecord(e[1], ctx->stream);
    g.b = k_acc;
    for (int i = 0; i < reps && r == TBPM_OK; ++i) r = launch_accum_step(ctx, g, pl.precision, ACC_REGULAR);
    cudaEventRecord(e[2], ctx->stream);
  }
  if (r == TBPM_OK && cudaEventSynchronize(e[2]) == cudaSuccess) {
    cudaEventElapsedTime(&ms0, e[0], e[1]);
    cudaEventElapsedTime(&ms1, e[1], e[2]);
  }
  *t_amxsy = ms0 / reps;
  *t_axpy = std::max(1e-6, (double)(ms1 - ms0) / reps / k_acc);
  // buffered blocks: a step is the recurrence into a buffer slot plus its share of the flush's
  // slot reads; an accumulator update is the flush's extra cost per accumulator and term
  const int Tm = 8;
  if (r == TBPM_OK && ctx->buffer_blocks && k_acc >= 2 &&
      ensure(ctx, ctx->ws_blk, pl.state_bytes * (size_t)Tm) == TBPM_OK &&
      ensure(ctx, ctx->ws_blk_coef, sizeof(double) * 2 * (size_t)Tm * k_acc) == TBPM_OK) {
    if (cudaMemsetAsync(ctx->ws_blk_coef.p, 0, sizeof(double) * 2 * (size_t)Tm * k_acc, ctx->stream) !=
            cudaSuccess ||
        cudaMemsetAsync(ctx->ws_blk.p, 0, pl.state_bytes * (size_t)Tm, ctx->stream) != cudaSuccess) {
      set_error("measure_pass_costs: %s", cudaGetErrorString(cudaGetLastError()));
      r = TBPM_ECUDA;
    }
    float m[3] = {0.f, 0.f, 0.f};
    for (int pass = 0; pass < 2 && r == TBPM_OK; ++pass) {
      g.b = 0;
      g.j_lo = 0;
      g.r.next = ctx->ws_blk.p;
      cudaEventRecord(e[0], ctx->stream);
      for (int i = 0; i < reps && r == TBPM_OK; ++i) r = launch_accum_step(ctx, g, pl.precision, ACC_REGULAR);
      cudaEventRecord(e[1], ctx->stream);
      // both flushes in the 16-accumulator tile of the block sizes being chosen between, so that
      // the difference is the cost of the extra accumulators, not of another kernel
      for (int i = 0; i < reps && r == TBPM_OK; ++i)
        r = launch_block_flush(ctx, g.r, pl.precision, ctx->ws_blk.p, Tm, ctx->ws_acc.p, 1,
                               (const double*)ctx->ws_blk_coef.p, 16);
      cudaEventRecord(e[2], ctx->stream);
      for (int i = 0; i < reps && r == TBPM_OK; ++i)
        r = launch_block_flush(ctx, g.r, pl.precision, ctx->ws_blk.p, Tm, ctx->ws_acc.p, k_acc,
                               (const double*)ctx->ws_blk_coef.p, 16);
      cudaEvent_t e3;
      cudaEventCreate(&e3);
      cudaEventRecord(e3, ctx->stream);
      if (r == TBPM_OK && cudaEventSynchronize(e3) == cudaSuccess) {
        cudaEventElapsedTime(&m[0], e[0], e[1]);
        cudaEventElapsedTime(&m[1], e[1], e[2]);
        cudaEventElapsedTime(&m[2], e[2], e3);
      }
      cudaEventDestroy(e3);
    }
    g.r.next = nullptr;
    if (r == TBPM_OK) {
      const double rec = m[0] / reps, f1 = m[1] / reps, fk = m[2] / reps;
      *t_amxsy = rec + f1 / Tm;
      *t_axpy = std::max(1e-6, (fk - f1) / ((double)(k_acc - 1) * Tm));
    }
  }
  for (auto& x : e) cudaEventDestroy(x);
  TBPM_TRY(r);
  return TBPM_OK;
}

// b_opt = argmin_b C(b) with measured costs (Sec. II.B), capped by memory.
int choose_block(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, int64_t n_steps,
                 int64_t* b, double* t_amxsy, double* t_axpy) {
  int64_t cap = block_cap(pl, n_steps);
  // buffered blocks: one flush serves 16 accumulators per pass over the buffer; past that every
  // further 16 re-read the buffer, which the linear cost model does not see
  if (ctx->buffer_blocks) cap = std::min<int64_t>(cap, 16);
  double ta = 0, tx = 0;
  TBPM_TRY(measure_pass_costs(ctx, lat, req, pl, (int)std::min<int64_t>(cap, 8), &ta, &tx));
  if (t_amxsy) *t_amxsy = ta;
  if (t_axpy) *t_axpy = tx;
  *b = tbpm_block_opt(n_steps, pl.tau, ta, tx, cap);
  return TBPM_OK;
}

// State-based propagation in blocks of b steps; b = 1 is the sequential form.
// d_C [Spad][n_steps+1][2].  The hook sees each finished time block: psi(t_{start+1}) ..
// psi(t_{start+bb}) as bb consecutive state blocks.  init (device, optional) replaces the
// request's initial states.
using BlockHook = std::function<int(int64_t /*start*/, int /*bb*/, const void* /*first state block*/)>;

int run_blocks(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, int64_t n_steps,
               int64_t b, double* d_C, double tau_signed = 0.0, const BlockHook& hook = nullptr,
               const void* init = nullptr, bool corr = true) {
  const double tau = tau_signed != 0.0 ? tau_signed : pl.tau;
  if (n_steps < 1) {
    set_error("n_steps must be >= 1");
    return TBPM_EINVAL;
  }
  b = std::max<int64_t>(1, std::min<int64_t>(b, n_steps));
  if (corr) TBPM_TRY(ensure(ctx, ctx->ws_psi, pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_acc, pl.state_bytes * (size_t)b));
  if (corr) {
    if (init)
      TBPM_CK(cudaMemcpyAsync(ctx->ws_psi.p, init, pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    else
      TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_psi.p, nullptr));
    TBPM_CK(cudaMemcpyAsync(ctx->ws_phi[0].p, ctx->ws_psi.p, pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  } else if (!init) {
    TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_phi[0].p, nullptr));
  } else if (init != ctx->ws_phi[0].p) {
    TBPM_CK(cudaMemcpyAsync(ctx->ws_phi[0].p, init, pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  }

  AccumArgs g;
  memset(&g, 0, sizeof(g));
  TBPM_TRY(base_args(ctx, lat, pl, &g.r, 3));
  const int C_len = (int)(n_steps + 1);
  // C(0) = <psi|psi>
  if (corr) TBPM_TRY(launch_dot(ctx, g.r, pl.precision, ctx->ws_psi.p, ctx->ws_psi.p, d_C, C_len));

  const double shift = lat->H0 / lat->half;
  std::vector<double> coef_full, coef_last;
  std::vector<int> nper_full, nper_last;
  block_coefficients(tau, shift, (int)b, &coef_full, &nper_full);
  const int64_t last_len = n_steps % b;
  if (last_len) block_coefficients(tau, shift, (int)last_len, &coef_last, &nper_last);
  const size_t tab_bytes = (coef_full.size() + coef_last.size()) * sizeof(double);
  TBPM_TRY(ensure(ctx, ctx->ws_table, tab_bytes));
  double* tab_full = (double*)ctx->ws_table.p;
  double* tab_last = tab_full + coef_full.size();
  TBPM_CK(cudaMemcpyAsync(tab_full, coef_full.data(), coef_full.size() * sizeof(double), cudaMemcpyHostToDevice,
                          ctx->stream));
  if (last_len)
    TBPM_CK(cudaMemcpyAsync(tab_last, coef_last.data(), coef_last.size() * sizeof(double), cudaMemcpyHostToDevice,
                            ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));  // host vectors go out of scope below

  g.acc = ctx->ws_acc.p;
  g.acc_stride = lat->n_sites * (int64_t)pl.Spad;
  g.psi = corr ? ctx->ws_psi.p : nullptr;
  g.C = corr ? d_C : nullptr;
  g.C_len = C_len;

  // Buffered accumulation: the recurrence writes phi_n into a window of T buffer slots, and
  // every T terms one flush adds sum_t c_t(j) phi_t to every accumulator of the block (each
  // accumulator crosses HBM once per T terms instead of once per term); C(t_j) = <psi|acc_j>
  // for the whole block comes from one block inner product at its end.  Slots 0 and 1 carry the
  // two latest vectors of the previous window, slot 2 + k holds term n0 + k.  Where the register
  // sweep applies, four terms at a time come from one window pass (phi_n and phi_{n-1} read once
  // for four slots), which pays even for b = 1: the sequential form then buffers too; otherwise
  // the sequential form keeps its fused one-accumulator pass.
  const bool sweep_win = sweep_window_applicable(lat, pl.precision, pl.Spad);
  int T = 0;
  if (ctx->buffer_blocks && (b >= 2 || sweep_win)) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const int64_t fit = (int64_t)(0.5 * (double)free_b / (double)pl.state_bytes) - 2;
    const int Nb_full = *std::max_element(nper_full.begin(), nper_full.end());
    T = (int)std::min<int64_t>(std::min<int64_t>(qe_flush_max_terms(), fit), (int64_t)Nb_full);
  }
  if (T >= 4) {
    TBPM_TRY(ensure(ctx, ctx->ws_blk, pl.state_bytes * (size_t)(T + 2)));
    // coefficient tables with the terms past N(j tau~) set to zero, full block then last block
    std::vector<double> cz;
    auto zeroed = [&](const std::vector<double>& cf, const std::vector<int>& np, int bb) {
      const int Nb = *std::max_element(np.begin(), np.end());
      const size_t base = cz.size();
      cz.insert(cz.end(), cf.begin(), cf.begin() + (size_t)Nb * bb * 2);
      for (int n = 0; n < Nb; ++n)
        for (int j = 0; j < bb; ++j)
          if (n >= np[j]) cz[base + ((size_t)n * bb + j) * 2] = cz[base + ((size_t)n * bb + j) * 2 + 1] = 0.0;
      return base;
    };
    const size_t off_full = zeroed(coef_full, nper_full, (int)b);
    const size_t off_last = last_len ? zeroed(coef_last, nper_last, (int)last_len) : 0;
    TBPM_TRY(ensure(ctx, ctx->ws_blk_coef, cz.size() * sizeof(double)));
    TBPM_CK(cudaMemcpyAsync(ctx->ws_blk_coef.p, cz.data(), cz.size() * sizeof(double), cudaMemcpyHostToDevice,
                            ctx->stream));
    TBPM_CK(cudaStreamSynchronize(ctx->stream));
    char* slots = (char*)ctx->ws_blk.p;
    auto slot = [&](int k) { return (void*)(slots + (size_t)k * pl.state_bytes); };
    AccumArgs gr = g;
    gr.b = 0;
    gr.j_lo = 0;
    gr.j_done = -1;
    gr.first_term = 0;
    int64_t start = 0;
    while (start < n_steps) {
      const int bb = (int)std::min<int64_t>(b, n_steps - start);
      const std::vector<int>& nper = (bb == b) ? nper_full : nper_last;
      const double* cf = (const double*)ctx->ws_blk_coef.p + ((bb == b) ? off_full : off_last);
      const int Nb = *std::max_element(nper.begin(), nper.end());
      TBPM_CK(cudaMemsetAsync(ctx->ws_acc.p, 0, pl.state_bytes * (size_t)bb, ctx->stream));
      TBPM_CK(cudaMemcpyAsync(slot(2), ctx->ws_phi[0].p, pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      int n0 = 0;
      auto slot_of = [&](int m) { return m >= n0 ? slot(2 + (m - n0)) : (m == n0 - 1 ? slot(1) : slot(0)); };
      for (int n = 1; n < Nb; ++n) {
        if (n - n0 == T) {
          TBPM_TRY(launch_block_flush(ctx, gr.r, pl.precision, slot(2), T, ctx->ws_acc.p, bb,
                                      cf + (size_t)n0 * bb * 2));
          TBPM_CK(cudaMemcpyAsync(slot(0), slot(T), pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
          TBPM_CK(cudaMemcpyAsync(slot(1), slot(T + 1), pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
          n0 = n;
        }
        if (sweep_win && n >= 2 && n + 3 < Nb && n - n0 + 4 <= T) {  // terms n .. n+3 in one pass
          void* const w[4] = {slot_of(n), slot_of(n + 1), slot_of(n + 2), slot_of(n + 3)};
          TBPM_TRY(launch_sweep_window(ctx, lat, gr.r, slot_of(n - 2), slot_of(n - 1), w));
          n += 3;
          continue;
        }
        gr.r.cur = slot_of(n - 1);
        gr.r.prev_out = n >= 2 ? slot_of(n - 2) : slot_of(n - 1);  // not read by the first step
        gr.r.next = slot_of(n);
        TBPM_TRY(launch_accum_step(ctx, gr, pl.precision, n == 1 ? ACC_FIRST : ACC_REGULAR));
      }
      TBPM_TRY(launch_block_flush(ctx, gr.r, pl.precision, slot(2), Nb - n0, ctx->ws_acc.p, bb,
                                  cf + (size_t)n0 * bb * 2));
      if (corr)
        TBPM_TRY(launch_xdot(ctx, pl.precision, pl.Spad, lat->n_sites, ctx->ws_psi.p, 1, ctx->ws_acc.p, bb, d_C,
                             C_len, 0, 1, start + 1));
      if (hook) TBPM_TRY(hook(start, bb, ctx->ws_acc.p));
      const char* last = (const char*)ctx->ws_acc.p + (size_t)(bb - 1) * pl.state_bytes;
      TBPM_CK(cudaMemcpyAsync(ctx->ws_phi[0].p, last, pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      start += bb;
    }
    return TBPM_OK;
  }

  int64_t start = 0;
  while (start < n_steps) {
    const int bb = (int)std::min<int64_t>(b, n_steps - start);
    const std::vector<int>& nper = (bb == b) ? nper_full : nper_last;
    const double* tab = (bb == b) ? tab_full : tab_last;
    const int Nb = *std::max_element(nper.begin(), nper.end());
    g.b = bb;
    for (int n = 0; n < Nb; ++n) {
      int j_lo = 0;
      while (j_lo < bb && nper[j_lo] <= n) ++j_lo;
      std::vector<int> done;
      for (int j = j_lo; j < bb; ++j)
        if (nper[j] - 1 == n) done.push_back(j);
      const int mode = (n == Nb - 1) ? ACC_NOSPMV : (n == 0 ? ACC_FIRST : ACC_REGULAR);
      g.r.cur = ctx->ws_phi[n & 1].p;
      g.r.prev_out = ctx->ws_phi[(n + 1) & 1].p;
      g.coef = tab + (size_t)n * bb * 2;
      g.j_lo = j_lo;
      g.first_term = n == 0;
      if (!corr) done.clear();
      g.j_done = done.empty() ? -1 : done[0];
      g.j_global = done.empty() ? 0 : (int)(start + done[0] + 1);
      TBPM_TRY(launch_accum_step(ctx, g, pl.precision, mode));
      for (size_t q = 1; q < done.size(); ++q) {
        const int j = done[q];
        const char* accj = (const char*)ctx->ws_acc.p + (size_t)j * pl.state_bytes;
        TBPM_TRY(launch_dot(ctx, g.r, pl.precision, ctx->ws_psi.p, accj, d_C + (start + j + 1) * 2, C_len));
      }
    }
    if (hook) TBPM_TRY(hook(start, bb, ctx->ws_acc.p));
    // the block's last state starts the next block
    const char* last = (const char*)ctx->ws_acc.p + (size_t)(bb - 1) * pl.state_bytes;
    TBPM_CK(cudaMemcpyAsync(ctx->ws_phi[0].p, last, pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    start += bb;
  }
  return TBPM_OK;
}

// Correlation of all Spad states into d_C [Spad][n_steps+1][2].
int run_correlation(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, double* d_C) {
  const int64_t n_steps = req->n_steps;
  if (n_steps < 1 || n_steps > (1 << 24)) {
    set_error("n_steps out of range");
    return TBPM_EINVAL;
  }
  if (req->form == TBPM_CONCURRENT_M) {
    const int64_t need = truncation_order_host(n_steps * pl.tau);
    int64_t M = std::max<int64_t>(req->n_moments, need);
    M += (M & 1);
    TBPM_TRY(ensure(ctx, ctx->ws_mu, sizeof(double) * 2 * (size_t)M * pl.Spad));
    double* mu = (double*)ctx->ws_mu.p;
    TBPM_TRY(run_moments(ctx, lat, req, pl, M, mu));
    const int n_terms = (int)need + 8;
    const size_t tab = sizeof(double) * (size_t)n_terms * (n_steps + 1);
    TBPM_TRY(ensure(ctx, ctx->ws_table, tab + sizeof(int) * (n_steps + 1)));
    double* table = (double*)ctx->ws_table.p;
    int* nper = (int*)((char*)ctx->ws_table.p + tab);
    TBPM_TRY(launch_bessel_table(ctx, pl.tau, (int)n_steps, n_terms, table, nper));
    TBPM_TRY(launch_corr_from_moments(ctx, table, nper, (int)n_steps, n_terms, mu, pl.Spad, (int)M,
                                      lat->H0 / lat->half, pl.tau, d_C));
    return TBPM_OK;
  }
  if (req->form == TBPM_SEQUENTIAL) return run_blocks(ctx, lat, req, pl, n_steps, 1, d_C);
  if (req->form == TBPM_CONCURRENT_S) {
    int64_t b = req->time_block;
    if (b <= 0) TBPM_TRY(choose_block(ctx, lat, req, pl, n_steps, &b, nullptr, nullptr));
    return run_blocks(ctx, lat, req, pl, n_steps, b, d_C);
  }
  set_error("unknown form %d", req->form);
  return TBPM_EINVAL;
}

// Quasi-eigenstates (Sec. IV) of all Spad states into ws_qe: [nE][n_sites][Spad].
int run_qe(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, const double* d_E, int nE) {
  const int64_t n_steps = req->n_steps;
  if (n_steps < 1 || n_steps > (1 << 22) || nE < 1 || nE > 4096) {
    set_error("quasi-eigenstates need 1 <= n_steps and 1 <= n_energies <= 4096");
    return TBPM_EINVAL;
  }
  const double tphys = pl.tau / lat->half;
  TBPM_TRY(ensure(ctx, ctx->ws_qe, pl.state_bytes * (size_t)nE));
  const size_t phase_bytes = sizeof(double) * 2 * (size_t)nE * (n_steps + 1);
  if (req->form == TBPM_CONCURRENT_E) {
    const int64_t need = truncation_order_host(n_steps * pl.tau);
    const int n_table = (int)need + 8;
    const size_t tab = sizeof(double) * (size_t)n_table * (n_steps + 1);
    TBPM_TRY(ensure(ctx, ctx->ws_table, tab + sizeof(int) * (n_steps + 1)));
    TBPM_TRY(ensure(ctx, ctx->ws_qe_coef, phase_bytes + sizeof(double) * 2 * (size_t)need * nE));
    double* table = (double*)ctx->ws_table.p;
    int* nper = (int*)((char*)ctx->ws_table.p + tab);
    double* phase = (double*)ctx->ws_qe_coef.p;
    double* coef = phase + 2 * (size_t)nE * (n_steps + 1);
    TBPM_TRY(launch_bessel_table(ctx, pl.tau, (int)n_steps, n_table, table, nper));
    TBPM_TRY(launch_qe_coefficients(ctx, table, (int)n_steps, (int)need, d_E, nE, lat->H0, tphys, phase, coef));
    TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
    TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pl.state_bytes));
    TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_phi[0].p, nullptr));
    // buffered accumulation: each pass also copies phi_n into slot n % T of a buffer of T states,
    // and every T terms one flush adds sum_t C_t(E) phi_t to all N_E accumulators
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const int T = (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(qe_flush_max_terms(), need),
                                                               (int64_t)(0.5 * (double)free_b / pl.state_bytes)));
    TBPM_TRY(ensure(ctx, ctx->ws_acc, pl.state_bytes * (size_t)T));
    TBPM_TRY(ensure(ctx, ctx->ws_aux, 2 * sizeof(double)));
    const double one[2] = {1.0, 0.0};
    TBPM_CK(cudaMemcpyAsync(ctx->ws_aux.p, one, sizeof(one), cudaMemcpyHostToDevice, ctx->stream));
    TBPM_CK(cudaMemsetAsync(ctx->ws_qe.p, 0, pl.state_bytes * (size_t)nE, ctx->stream));
    AccumArgs g;
    memset(&g, 0, sizeof(g));
    TBPM_TRY(base_args(ctx, lat, pl, &g.r, 3));
    g.acc_stride = lat->n_sites * (int64_t)pl.Spad;
    g.b = 1;
    g.j_lo = 0;
    g.j_done = -1;
    g.first_term = 1;  // the buffer slot is written, not accumulated
    g.coef = (const double*)ctx->ws_aux.p;
    const int tok = phase_begin(ctx, 0);
    for (int64_t n = 0; n < need; ++n) {
      const int mode = (n == need - 1) ? ACC_NOSPMV : (n == 0 ? ACC_FIRST : ACC_REGULAR);
      g.r.cur = ctx->ws_phi[n & 1].p;
      g.r.prev_out = ctx->ws_phi[(n + 1) & 1].p;
      g.acc = (char*)ctx->ws_acc.p + (size_t)(n % T) * pl.state_bytes;
      TBPM_TRY(launch_accum_step(ctx, g, pl.precision, mode));
      if ((n + 1) % T == 0 || n == need - 1) {
        const int nt = (int)(n % T) + 1;
        TBPM_TRY(launch_qe_flush(ctx, g.r, pl.precision, ctx->ws_acc.p, nt, ctx->ws_qe.p, nE, coef, (int)(n + 1 - nt)));
      }
    }
    phase_end(ctx, tok);
    return TBPM_OK;
  }
  if (req->form != TBPM_SEQUENTIAL && req->form != TBPM_CONCURRENT_S) {
    set_error("quasi-eigenstates: form must be SEQUENTIAL, CONCURRENT_S or CONCURRENT_E");
    return TBPM_EINVAL;
  }
  // explicit states psi(+-t_j), each folded into the N_E accumulators with (tau/2pi) e^{+-i E t_j}
  TBPM_TRY(ensure(ctx, ctx->ws_qe_coef, phase_bytes));
  double* phase = (double*)ctx->ws_qe_coef.p;
  {
    const int64_t tot = (int64_t)nE * (n_steps + 1);
    (void)tot;
    TBPM_TRY(launch_qe_coefficients_phase_only(ctx, d_E, nE, tphys, (int)n_steps, phase));
  }
  TBPM_CK(cudaMemsetAsync(ctx->ws_qe.p, 0, pl.state_bytes * (size_t)nE, ctx->stream));
  RecurrenceArgs ra;
  TBPM_TRY(base_args(ctx, lat, pl, &ra, 3));
  const int width = (int)(n_steps + 1);
  const double scale = tphys / (2.0 * M_PI);
  int64_t b = req->form == TBPM_SEQUENTIAL ? 1 : req->time_block;
  if (b <= 0) TBPM_TRY(choose_block(ctx, lat, req, pl, n_steps, &b, nullptr, nullptr));
  TBPM_TRY(ensure(ctx, ctx->ws_psi, pl.state_bytes));
  TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_psi.p, nullptr));
  for (int dir = 0; dir < 2; ++dir) {
    const double sgn = dir == 0 ? 1.0 : -1.0;
    BlockHook hook = [&](int64_t start, int bb, const void* first) -> int {
      for (int j = 0; j < bb; ++j)
        TBPM_TRY(launch_qe_axpy(ctx, ra, pl.precision, (const char*)first + (size_t)j * pl.state_bytes,
                                ctx->ws_qe.p, phase, width, (int)(start + j + 1), sgn, scale, nE));
      return TBPM_OK;
    };
    TBPM_TRY(run_blocks(ctx, lat, req, pl, n_steps, b, nullptr, sgn * pl.tau, hook, ctx->ws_psi.p, false));
    if (dir == 0)  // j = 0 term, tau a(E,0) psi, once
      TBPM_TRY(launch_qe_axpy(ctx, ra, pl.precision, ctx->ws_psi.p, ctx->ws_qe.p, phase, width, 0, 1.0, scale, nE));
  }
  return TBPM_OK;
}

// Electronic conductivity (Sec. V) along `direction` for all Spad states and nE energies.
// Leaves C(t_j, E_k) in ws_out as [Spad][nE][n_steps+1][2] and sigma in ws_ec (after the
// 2*Spad*nE norms) as [Spad][nE].  Returns the sigma pointer through *d_sigma.
int run_ec(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, const double* d_E, int nE,
           int direction, double** d_C_out, double** d_sigma) {
  const int64_t n_steps = req->n_steps;
  const int dims = lat->desc.kind == TBPM_CUBIC ? 3 : 2;
  if (direction < 0 || direction >= dims) {
    set_error("direction %d out of range for a %d-dimensional lattice", direction, dims);
    return TBPM_EINVAL;
  }
  if (req->form != TBPM_SEQUENTIAL && req->form != TBPM_CONCURRENT_S && req->form != TBPM_CONCURRENT_M) {
    set_error("conductivity: form must be SEQUENTIAL, CONCURRENT_S or CONCURRENT_M");
    return TBPM_EINVAL;
  }
  if (n_steps < 1 || n_steps > (1 << 20) || nE < 1 || nE > 4096 || (int64_t)nE * pl.Spad > 65536) {
    set_error("conductivity needs 1 <= n_steps <= 2^20, 1 <= n_energies <= 4096 and n_energies * states <= 65536");
    return TBPM_EINVAL;
  }
  // quasi-eigenstates: energy-based form for few energies, state-based otherwise (Sec. IV)
  tbpm_request qreq = *req;
  qreq.form = nE <= 200 ? TBPM_CONCURRENT_E : TBPM_CONCURRENT_S;
  qreq.time_block = 0;
  TBPM_TRY(run_qe(ctx, lat, &qreq, pl, d_E, nE));
  const int rows = pl.Spad * nE;
  const int64_t W = n_steps + 1;
  TBPM_TRY(ensure(ctx, ctx->ws_ec, sizeof(double) * 3 * (size_t)rows));
  double* nrm = (double*)ctx->ws_ec.p;
  double* sigma = nrm + 2 * (size_t)rows;
  TBPM_TRY(ensure(ctx, ctx->ws_psi, pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_jpsi, pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pl.state_bytes));
  TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_psi.p, nullptr));
  const int64_t n = lat->n_sites;
  // <psi|Psi(E)> before the kets are overwritten
  TBPM_TRY(launch_xdot(ctx, pl.precision, pl.Spad, n, ctx->ws_psi.p, 1, ctx->ws_qe.p, nE, nrm, nE, 0, 1, 0));
  // |psi_2(E)> = J |Psi(E)> in place (through one scratch block), |psi_1> = J |psi>
  for (int k = 0; k < nE; ++k) {
    char* qk = (char*)ctx->ws_qe.p + (size_t)k * pl.state_bytes;
    TBPM_TRY(launch_current(ctx, lat, pl.precision, pl.Spad, direction, qk, ctx->ws_phi[0].p));
    TBPM_CK(cudaMemcpyAsync(qk, ctx->ws_phi[0].p, pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
  }
  TBPM_TRY(launch_current(ctx, lat, pl.precision, pl.Spad, direction, ctx->ws_psi.p, ctx->ws_jpsi.p));
  const void* kets = ctx->ws_qe.p;
  TBPM_TRY(ensure(ctx, ctx->ws_out, sizeof(double) * 2 * (size_t)rows * W));
  double* C = (double*)ctx->ws_out.p;
  const int tok = phase_begin(ctx, 0);
  if (req->form == TBPM_CONCURRENT_M) {
    // m_n(E) = <J psi|T_n(H~)|J Psi(E)> (Eq. dc_mom), n < N(t~_tot)
    const int64_t Nn = truncation_order_host(n_steps * pl.tau);
    TBPM_TRY(ensure(ctx, ctx->ws_mu, sizeof(double) * 2 * (size_t)rows * Nn));
    double* m = (double*)ctx->ws_mu.p;
    TBPM_CK(cudaMemcpyAsync(ctx->ws_phi[0].p, ctx->ws_jpsi.p, pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    AccumArgs g;
    memset(&g, 0, sizeof(g));
    TBPM_TRY(base_args(ctx, lat, pl, &g.r, 3));
    g.b = 0;
    g.j_done = -1;
    // buffered: the recurrence fills a window of up to 32 slots and one block inner product
    // gives the window's moments against all kets (each ket read once per window, not per term);
    // slots 0 and 1 carry the previous window's last two vectors, slot 2 + a holds term n0 + a
    int T = 0;
    if (ctx->buffer_blocks) {
      size_t free_b = 0, total_b = 0;
      cudaMemGetInfo(&free_b, &total_b);
      const int64_t fit = (int64_t)(0.5 * (double)free_b / (double)pl.state_bytes) - 2;
      T = (int)std::min<int64_t>(std::min<int64_t>(qe_flush_max_terms(), fit), Nn);
    }
    if (T >= 4) {
      TBPM_TRY(ensure(ctx, ctx->ws_blk, pl.state_bytes * (size_t)(T + 2)));
      char* slots = (char*)ctx->ws_blk.p;
      auto slot = [&](int64_t k) { return (void*)(slots + (size_t)k * pl.state_bytes); };
      int64_t n0 = 0;
      auto slot_of = [&](int64_t t) { return t >= n0 ? slot(2 + (t - n0)) : (t == n0 - 1 ? slot(1) : slot(0)); };
      TBPM_CK(cudaMemcpyAsync(slot(2), ctx->ws_jpsi.p, pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
      const bool sweep_win = sweep_window_applicable(lat, pl.precision, pl.Spad);
      for (int64_t k = 1; k < Nn; ++k) {
        if (k - n0 == T) {
          TBPM_TRY(launch_xdot(ctx, pl.precision, pl.Spad, n, slot(2), T, kets, nE, m, (int64_t)nE * Nn, 1, Nn, n0));
          TBPM_CK(cudaMemcpyAsync(slot(0), slot(T), pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
          TBPM_CK(cudaMemcpyAsync(slot(1), slot(T + 1), pl.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
          n0 = k;
        }
        if (sweep_win && k >= 2 && k + 3 < Nn && k - n0 + 4 <= T) {  // terms k .. k+3 in one pass
          void* const w[4] = {slot_of(k), slot_of(k + 1), slot_of(k + 2), slot_of(k + 3)};
          TBPM_TRY(launch_sweep_window(ctx, lat, g.r, slot_of(k - 2), slot_of(k - 1), w));
          k += 3;
          continue;
        }
        g.r.cur = slot_of(k - 1);
        g.r.prev_out = k >= 2 ? slot_of(k - 2) : slot_of(k - 1);  // not read by the first step
        g.r.next = slot_of(k);
        TBPM_TRY(launch_accum_step(ctx, g, pl.precision, k == 1 ? ACC_FIRST : ACC_REGULAR));
      }
      TBPM_TRY(launch_xdot(ctx, pl.precision, pl.Spad, n, slot(2), (int)(Nn - n0), kets, nE, m, (int64_t)nE * Nn, 1,
                           Nn, n0));
      g.r.next = nullptr;
    } else {
    TBPM_TRY(launch_xdot(ctx, pl.precision, pl.Spad, n, ctx->ws_phi[0].p, 1, kets, nE, m, (int64_t)nE * Nn, 0, Nn, 0));
    for (int64_t k = 0; k + 1 < Nn; ++k) {
      g.r.cur = ctx->ws_phi[k & 1].p;
      g.r.prev_out = ctx->ws_phi[(k + 1) & 1].p;
      TBPM_TRY(launch_accum_step(ctx, g, pl.precision, k == 0 ? ACC_FIRST : ACC_REGULAR));
      TBPM_TRY(launch_xdot(ctx, pl.precision, pl.Spad, n, ctx->ws_phi[(k + 1) & 1].p, 1, kets, nE, m,
                           (int64_t)nE * Nn, 0, Nn, k + 1));
    }
    }
    phase_end(ctx, tok);
    const int n_table = (int)Nn + 8;
    const size_t tab = sizeof(double) * (size_t)n_table * W;
    TBPM_TRY(ensure(ctx, ctx->ws_table, tab + sizeof(int) * (size_t)W));
    double* table = (double*)ctx->ws_table.p;
    int* nper = (int*)((char*)ctx->ws_table.p + tab);
    TBPM_TRY(launch_bessel_table(ctx, pl.tau, (int)n_steps, n_table, table, nper));
    TBPM_TRY(launch_ec_corr_from_moments(ctx, table, nper, (int)n_steps, m, rows, (int)Nn, lat->H0 / lat->half,
                                         pl.tau, C));
  } else {
    // psi_1(t_j) = e^{-iHt_j} J psi in time blocks; each block's b states meet all N_E kets at once
    int64_t b = req->form == TBPM_SEQUENTIAL ? 1 : req->time_block;
    if (b <= 0) TBPM_TRY(choose_block(ctx, lat, req, pl, n_steps, &b, nullptr, nullptr));
    BlockHook hook = [&](int64_t start, int bb, const void* first) -> int {
      return launch_xdot(ctx, pl.precision, pl.Spad, n, first, bb, kets, nE, C, (int64_t)nE * W, 1, W, start + 1);
    };
    TBPM_TRY(run_blocks(ctx, lat, req, pl, n_steps, b, nullptr, 0.0, hook, ctx->ws_jpsi.p, false));
    TBPM_TRY(launch_xdot(ctx, pl.precision, pl.Spad, n, ctx->ws_jpsi.p, 1, kets, nE, C, (int64_t)nE * W, 0, W, 0));
    phase_end(ctx, tok);
  }
  const double area = lat->desc.kind == TBPM_HONEYCOMB ? 3.0 * sqrt(3.0) / 4.0 : 1.0;
  TBPM_TRY(launch_ec_finish(ctx, C, nrm, d_E, nE, rows, (int)n_steps, pl.tau / lat->half, area, sigma));
  *d_C_out = C;
  *d_sigma = sigma;
  return TBPM_OK;
}

// Chebyshev coefficients of the Fermi-Dirac function (or its square root) on the lattice's
// spectral window into ws_fermi; *coef = device complex table [n_terms][2], truncated at
// 1 + max{n : |a_n| > 1e-14} within n_cap = min(2^14, 12|H|/kT + 64) orders.
int fermi_series(tbpm_ctx* ctx, const tbpm_lattice* lat, double mu, double kT, int sqrt_f, const double** coef,
                 int* n_terms) {
  if (!(kT > 0.0) || !isfinite(kT) || !isfinite(mu)) {
    set_error("Fermi-Dirac operator needs kT > 0 and a finite mu");
    return TBPM_EINVAL;
  }
  const double want = 12.0 * lat->half / kT + 64.0;
  const int n_cap = (int)std::min<double>(16384.0, std::max<double>(64.0, ceil(want)));
  const int K = std::max(2 * n_cap, 1024);
  TBPM_TRY(ensure(ctx, ctx->ws_fermi, sizeof(double) * ((size_t)K + 2 * (size_t)n_cap)));
  double* scratch = (double*)ctx->ws_fermi.p;
  double* table = scratch + K;
  TBPM_TRY(launch_fermi_coefficients(ctx, mu, kT, lat->H0, lat->half, sqrt_f, n_cap, K, scratch, table));
  std::vector<double> h(2 * (size_t)n_cap);
  TBPM_CK(cudaMemcpyAsync(h.data(), table, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  int last = 0;
  for (int n = n_cap - 1; n >= 0; --n)
    if (fabs(h[2 * (size_t)n]) > 1e-14) {
      last = n;
      break;
    }
  *coef = table;
  *n_terms = last + 1;
  return TBPM_OK;
}

// out = sum_{n < n_terms} coef_n T_n(H~) X for one state block of plan pc.  The recurrence runs
// in b0 (which holds X on entry and is overwritten) and b1; out is distinct from both.
int apply_series_bufs(tbpm_ctx* ctx, tbpm_lattice* lat, const Plan& pc, void* b0, void* b1, void* out,
                      const double* coef, int n_terms) {
  AccumArgs g;
  memset(&g, 0, sizeof(g));
  TBPM_TRY(base_args(ctx, lat, pc, &g.r, 3));
  g.acc = out;
  g.acc_stride = lat->n_sites * (int64_t)pc.Spad;
  g.b = 1;
  g.j_lo = 0;
  g.j_done = -1;
  // buffered: terms go into a window of up to 32 slots and one flush adds sum_n a_n T_n phi to
  // the output per window (the same bookkeeping as the buffered time blocks)
  int T = 0;
  if (ctx->buffer_blocks) {
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const int64_t fit = (int64_t)(0.5 * (double)free_b / (double)pc.state_bytes) - 2;
    T = (int)std::min<int64_t>(std::min<int64_t>(qe_flush_max_terms(), fit), (int64_t)n_terms);
  }
  if (T >= 4) {
    TBPM_TRY(ensure(ctx, ctx->ws_blk, pc.state_bytes * (size_t)(T + 2)));
    char* slots = (char*)ctx->ws_blk.p;
    auto slot = [&](int k) { return (void*)(slots + (size_t)k * pc.state_bytes); };
    int n0 = 0;
    auto slot_of = [&](int t) { return t >= n0 ? slot(2 + (t - n0)) : (t == n0 - 1 ? slot(1) : slot(0)); };
    TBPM_CK(cudaMemsetAsync(out, 0, pc.state_bytes, ctx->stream));
    TBPM_CK(cudaMemcpyAsync(slot(2), b0, pc.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
    g.b = 0;
    const bool sweep_win = sweep_window_applicable(lat, pc.precision, pc.Spad);
    for (int n = 1; n < n_terms; ++n) {
      if (n - n0 == T) {
        TBPM_TRY(launch_block_flush(ctx, g.r, pc.precision, slot(2), T, out, 1, coef + 2 * (size_t)n0));
        TBPM_CK(cudaMemcpyAsync(slot(0), slot(T), pc.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        TBPM_CK(cudaMemcpyAsync(slot(1), slot(T + 1), pc.state_bytes, cudaMemcpyDeviceToDevice, ctx->stream));
        n0 = n;
      }
      if (sweep_win && n >= 2 && n + 3 < n_terms && n - n0 + 4 <= T) {  // terms n .. n+3 in one pass
        void* const w[4] = {slot_of(n), slot_of(n + 1), slot_of(n + 2), slot_of(n + 3)};
        TBPM_TRY(launch_sweep_window(ctx, lat, g.r, slot_of(n - 2), slot_of(n - 1), w));
        n += 3;
        continue;
      }
      g.r.cur = slot_of(n - 1);
      g.r.prev_out = n >= 2 ? slot_of(n - 2) : slot_of(n - 1);  // not read by the first step
      g.r.next = slot_of(n);
      TBPM_TRY(launch_accum_step(ctx, g, pc.precision, n == 1 ? ACC_FIRST : ACC_REGULAR));
    }
    TBPM_TRY(launch_block_flush(ctx, g.r, pc.precision, slot(2), n_terms - n0, out, 1, coef + 2 * (size_t)n0));
    release(ctx, ctx->ws_blk);  // the callers' next step sizes its blocks by the free memory
    return TBPM_OK;
  }
  void* buf[2] = {b0, b1};
  for (int n = 0; n < n_terms; ++n) {
    const int mode = (n == n_terms - 1) ? ACC_NOSPMV : (n == 0 ? ACC_FIRST : ACC_REGULAR);
    g.r.cur = buf[n & 1];
    g.r.prev_out = buf[(n + 1) & 1];
    g.coef = coef + 2 * (size_t)n;
    g.first_term = n == 0;
    TBPM_TRY(launch_accum_step(ctx, g, pc.precision, mode));
  }
  return TBPM_OK;
}

// Largest power-of-two number of states per pass (<= cap) for which `blocks` state blocks of
// that width fit in 85% of the free device memory; 0 when not even one state fits.
int states_per_pass(const tbpm_lattice* lat, size_t elem, int cap, double blocks) {
  size_t free_b = 0, total_b = 0;
  cudaMemGetInfo(&free_b, &total_b);
  int k = cap;
  while (k >= 1 && blocks * (double)lat->n_sites * k * elem > 0.85 * (double)free_b) k >>= 1;
  return k;
}

// Optical conductivity (op 0: X = J_alpha, O = J_beta) or dynamical polarization (op 1:
// X = rho(q), O = rho(-q)) correlation C(t_j) = <psi_1(t_j)|X|psi_2(t_j)> of the plan's Sh states
// (the request's states pl.s0 .. pl.s0 + S - 1) into ws_out [Sh][n_steps+1][2]; the pair plan's
// time step is returned in *tphys.  Live memory: three pair blocks during the Fermi-Dirac series,
// 2 + b during the propagation.
int run_response(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, int op, int alpha,
                 int beta, const double q[3], double mu, double kT, double** d_C, double* tphys) {
  const int64_t n_steps = req->n_steps;
  const int Sh = pl.Spad;
  tbpm_request rc = *req;
  rc.n_states = 2 * Sh;
  rc.states = TBPM_STATES_RANDOM;
  Plan pc;
  TBPM_TRY(make_plan(lat, &rc, &pc));
  pc.tau = req->tau == 0.0 ? M_PI / 2 : req->tau;
  *tphys = pc.tau / lat->half;
  const int64_t n = lat->n_sites;
  const double* coef = nullptr;
  int nf = 0;
  TBPM_TRY(fermi_series(ctx, lat, mu, kT, 0, &coef, &nf));
  const double2* phase = nullptr;
  if (op == 1) {
    TBPM_TRY(ensure(ctx, ctx->ws_ec, sizeof(double2) * (size_t)n));
    phase = (const double2*)ctx->ws_ec.p;
    TBPM_TRY(launch_density_phases(ctx, lat, q, (double2*)ctx->ws_ec.p));
  }
  // O psi, formed from psi (twice: before the series and for the split after it)
  auto make_states = [&]() -> int {
    TBPM_TRY(ensure(ctx, ctx->ws_psi, pl.state_bytes));
    TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_psi.p, nullptr));
    if (op == 0) {
      TBPM_TRY(ensure(ctx, ctx->ws_jpsi, pl.state_bytes));
      TBPM_TRY(launch_current(ctx, lat, pl.precision, Sh, beta, ctx->ws_psi.p, ctx->ws_jpsi.p));
    }
    return TBPM_OK;
  };
  TBPM_TRY(make_states());
  TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pc.state_bytes));
  TBPM_TRY(launch_pair_init(ctx, pl.precision, n, Sh, ctx->ws_psi.p, op == 0 ? ctx->ws_jpsi.p : nullptr, phase,
                            ctx->ws_phi[0].p));
  release(ctx, ctx->ws_psi);
  release(ctx, ctx->ws_jpsi);
  TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pc.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi2[1], pc.state_bytes));
  // F = f(H) X, consuming X in ws_phi[0]
  TBPM_TRY(apply_series_bufs(ctx, lat, pc, ctx->ws_phi[0].p, ctx->ws_phi[1].p, ctx->ws_phi2[1].p, coef, nf));
  release(ctx, ctx->ws_phi[0]);
  TBPM_TRY(make_states());
  TBPM_TRY(launch_pair_split(ctx, pl.precision, n, Sh, ctx->ws_psi.p, op == 0 ? ctx->ws_jpsi.p : nullptr, phase,
                             ctx->ws_phi2[1].p));
  release(ctx, ctx->ws_psi);
  release(ctx, ctx->ws_jpsi);
  release(ctx, ctx->ws_phi2[0]);
  std::swap(ctx->ws_phi[0], ctx->ws_phi2[1]);  // Y(0) = [f psi | (1 - f) O psi] starts the propagation
  const int64_t W = n_steps + 1;
  TBPM_TRY(ensure(ctx, ctx->ws_out, sizeof(double) * 2 * (size_t)W * Sh));
  double* C = (double*)ctx->ws_out.p;
  const int tok = phase_begin(ctx, 0);
  TBPM_TRY(launch_xmy(ctx, lat, pl.precision, Sh, alpha, phase, ctx->ws_phi[0].p, 1, pc.state_bytes, C, W, 0));
  int64_t b = req->form == TBPM_SEQUENTIAL ? 1 : req->time_block;
  if (b <= 0) {
    // time the passes on copies, leaving Y(0) in ws_phi[0] untouched
    std::swap(ctx->ws_phi[0], ctx->ws_phi2[0]);
    const int r = choose_block(ctx, lat, &rc, pc, n_steps, &b, nullptr, nullptr);
    std::swap(ctx->ws_phi[0], ctx->ws_phi2[0]);
    release(ctx, ctx->ws_phi2[0]);
    release(ctx, ctx->ws_psi);
    TBPM_TRY(r);
  }
  BlockHook hook = [&](int64_t start, int bb, const void* first) -> int {
    return launch_xmy(ctx, lat, pl.precision, Sh, alpha, phase, first, bb, pc.state_bytes, C, W, start + 1);
  };
  TBPM_TRY(run_blocks(ctx, lat, &rc, pc, n_steps, b, nullptr, 0.0, hook, ctx->ws_phi[0].p, false));
  phase_end(ctx, tok);
  *d_C = C;
  return TBPM_OK;
}

int copy_rows(tbpm_ctx* ctx, double* dst, const double* src, int S, size_t row_doubles, cudaMemcpyKind kind) {
  TBPM_CK(cudaMemcpyAsync(dst, src, sizeof(double) * row_doubles * S, kind, ctx->stream));
  return TBPM_OK;
}

int run_dos(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, const Plan& pl, const double* d_E,
            int64_t nE, double* d_D) {
  if (nE < 1) {
    set_error("n_energies must be >= 1");
    return TBPM_EINVAL;
  }
  if (req->dos_method == TBPM_DOS_JACKSON) {
    const int64_t M = req->n_moments;
    TBPM_TRY(ensure(ctx, ctx->ws_mu, sizeof(double) * 2 * (size_t)std::max<int64_t>(M, 2) * pl.Spad));
    double* mu = (double*)ctx->ws_mu.p;
    TBPM_TRY(run_moments(ctx, lat, req, pl, M, mu));
    const int tok = phase_begin(ctx, 1);
    const int r = (req->recon == TBPM_RECON_TENSOR)
                      ? launch_dos_jackson_tensor(ctx, mu, pl.S, (int)M, d_E, nE, lat->H0, lat->half, d_D)
                      : launch_dos_jackson_fp64(ctx, mu, pl.S, (int)M, d_E, nE, lat->H0, lat->half, d_D);
    phase_end(ctx, tok);
    return r;
  }
  if (req->dos_method == TBPM_DOS_FOURIER) {
    TBPM_TRY(ensure(ctx, ctx->ws_out, sizeof(double) * 2 * (size_t)(req->n_steps + 1) * pl.Spad));
    double* C = (double*)ctx->ws_out.p;
    TBPM_TRY(run_correlation(ctx, lat, req, pl, C));
    return launch_dos_fourier(ctx, C, pl.S, (int)req->n_steps, d_E, nE, pl.tau / lat->half, req->window, d_D);
  }
  set_error("unknown dos_method %d", req->dos_method);
  return TBPM_EINVAL;
}

}  // namespace

namespace tbpm {
int lattice_ensure_d64(tbpm_lattice* lat) {
  TBPM_TRY(ensure_d64(lat));
  TBPM_CK(cudaStreamSynchronize(lat->ctx->stream));
  return TBPM_OK;
}

int init_request_states(tbpm_ctx* ctx, const tbpm_lattice* lat, const tbpm_request* req, void* dst) {
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  return init_states(ctx, lat, req, pl, dst, nullptr);
}
}  // namespace tbpm

// ====================================================================== C ABI: hot path
extern "C" {

int tbpm_states_export(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, void* out,
                       uint32_t* draws) {
  clear_error();
  if (!ctx) {
    set_error("NULL context");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  const int64_t n = lat->n_sites;
  TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
  uint32_t* d_draws = nullptr;
  if (draws && req->states == TBPM_STATES_RANDOM) {
    TBPM_TRY(ensure(ctx, ctx->ws_out, sizeof(uint32_t) * (size_t)n * pl.Spad));
    d_draws = (uint32_t*)ctx->ws_out.p;
  }
  TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_phi[0].p, d_draws));
  if (out) {
    for (int s = 0; s < pl.S; ++s)
      TBPM_CK(cudaMemcpy2DAsync((char*)out + (size_t)s * n * pl.elem, pl.elem, (const char*)ctx->ws_phi[0].p + s * pl.elem,
                                pl.Spad * pl.elem, pl.elem, n, cudaMemcpyDeviceToHost, ctx->stream));
  }
  if (d_draws)
    TBPM_CK(cudaMemcpyAsync(draws, d_draws, sizeof(uint32_t) * n * pl.S, cudaMemcpyDeviceToHost, ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return TBPM_OK;
}

int tbpm_moment_pass_kind(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, int* kind) {
  clear_error();
  if (!ctx || !lat_c || !req || !kind) {
    set_error("tbpm_moment_pass_kind: NULL argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  if (lat->chunks && pl.precision == TBPM_C64 && pl.Spad >= 2) {
    *kind = TBPM_PASS_TAPS;
    return TBPM_OK;
  }
  const int m = ctx->fusion;  // -1: autotuned on first use, reported as the mode it would time first
  const int64_t M = req->n_moments > 0 ? req->n_moments : truncation_order_host(req->n_steps * pl.tau);
  if (m > 0 && fused_applicable(lat, pl.precision, pl.Spad) && M / 2 - 1 >= fused_steps(m)) {
    const int band = (m == 8 ? 128 : m == 9 ? 192 : 256) / (pl.Spad / 2);
    *kind = (m >= 8 && m <= 10 && lat->geom.Lx >= band) ? TBPM_PASS_SWEEP
            : (m >= 3) ? TBPM_PASS_ROWS : TBPM_PASS_TILES;
    return TBPM_OK;
  }
  *kind = lat->path == TBPM_PATH_CSR ? TBPM_PASS_ELL : TBPM_PASS_STENCIL;
  return TBPM_OK;
}

int tbpm_moments_device(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, double* d_mu) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !d_mu) {
    set_error("NULL argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  const int64_t M = req->n_moments;
  if (pl.Spad == pl.S) return run_moments(ctx, lat, req, pl, M, d_mu);
  TBPM_TRY(ensure(ctx, ctx->ws_mu, sizeof(double) * 2 * (size_t)std::max<int64_t>(M, 2) * pl.Spad));
  TBPM_TRY(run_moments(ctx, lat, req, pl, M, (double*)ctx->ws_mu.p));
  return copy_rows(ctx, d_mu, (double*)ctx->ws_mu.p, pl.S, 2 * (size_t)M, cudaMemcpyDeviceToDevice);
}

int tbpm_moments(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, double* mu) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !mu) {
    set_error("NULL argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  const int64_t M = req->n_moments;
  TBPM_TRY(ensure(ctx, ctx->ws_mu, sizeof(double) * 2 * (size_t)std::max<int64_t>(M, 2) * pl.Spad));
  TBPM_TRY(run_moments(ctx, lat, req, pl, M, (double*)ctx->ws_mu.p));
  TBPM_TRY(copy_rows(ctx, mu, (double*)ctx->ws_mu.p, pl.S, 2 * (size_t)M, cudaMemcpyDeviceToHost));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return sweep_status(ctx);
}

int tbpm_correlation_device(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, double* d_C) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !d_C) {
    set_error("NULL argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  const size_t row = 2 * (size_t)(req->n_steps + 1);
  if (pl.Spad == pl.S) return run_correlation(ctx, lat, req, pl, d_C);
  TBPM_TRY(ensure(ctx, ctx->ws_out, sizeof(double) * row * pl.Spad));
  TBPM_TRY(run_correlation(ctx, lat, req, pl, (double*)ctx->ws_out.p));
  return copy_rows(ctx, d_C, (double*)ctx->ws_out.p, pl.S, row, cudaMemcpyDeviceToDevice);
}

int tbpm_correlation(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, double* C) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !C) {
    set_error("NULL argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  if (req->n_steps < 1) {
    set_error("n_steps must be >= 1");
    return TBPM_EINVAL;
  }
  const size_t row = 2 * (size_t)(req->n_steps + 1);
  TBPM_TRY(ensure(ctx, ctx->ws_out, sizeof(double) * row * pl.Spad));
  TBPM_TRY(run_correlation(ctx, lat, req, pl, (double*)ctx->ws_out.p));
  TBPM_TRY(copy_rows(ctx, C, (double*)ctx->ws_out.p, pl.S, row, cudaMemcpyDeviceToHost));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return TBPM_OK;
}

int tbpm_dos_device(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, const double* d_E,
                    int64_t nE, double* d_D) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !d_E || !d_D) {
    set_error("NULL argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  return run_dos(ctx, lat, req, pl, d_E, nE, d_D);
}

int tbpm_dos(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, const double* energies,
             int64_t nE, double* D) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !energies || !D) {
    set_error("NULL argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  if (nE < 1) {
    set_error("n_energies must be >= 1");
    return TBPM_EINVAL;
  }
  TBPM_TRY(ensure(ctx, ctx->ws_energies, sizeof(double) * (size_t)nE * (1 + pl.S)));
  double* dE = (double*)ctx->ws_energies.p;
  double* dD = dE + nE;
  TBPM_CK(cudaMemcpyAsync(dE, energies, sizeof(double) * nE, cudaMemcpyHostToDevice, ctx->stream));
  TBPM_TRY(run_dos(ctx, lat, req, pl, dE, nE, dD));
  TBPM_CK(cudaMemcpyAsync(D, dD, sizeof(double) * nE * pl.S, cudaMemcpyDeviceToHost, ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return sweep_status(ctx);
}

// Adjacency operator y_i = sum_{j in nbr(i)} x_j through the hot-path recurrence kernel
// (first-term mode with zero diagonal and unit hopping); debug export for exact index tests.
int tbpm_apply_hopping(tbpm_ctx* ctx, const tbpm_lattice* lat_c, int precision, int n_states, const void* x,
                       void* y) {
  clear_error();
  if (!ctx || !lat_c || !x || !y) {
    set_error("NULL argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  tbpm_request req;
  memset(&req, 0, sizeof(req));
  req.precision = precision;
  req.n_states = n_states;
  req.states = TBPM_STATES_RANDOM;
  Plan pl;
  TBPM_TRY(make_plan(lat, &req, &pl));
  if (pl.Spad != pl.S) {
    set_error("tbpm_apply_hopping needs a power-of-two number of states");
    return TBPM_EINVAL;
  }
  TBPM_CK(cudaSetDevice(ctx->device));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_mu, sizeof(double) * 4 * pl.Spad));
  TBPM_CK(cudaMemcpyAsync(ctx->ws_phi[0].p, x, pl.state_bytes, cudaMemcpyHostToDevice, ctx->stream));
  RecurrenceArgs a;
  TBPM_TRY(base_args(ctx, lat, pl, &a, 3));
  a.diag = nullptr;
  a.diag_const = 0.0;
  a.thop = 1.0;
  set_float_coefficients(&a);
  a.mu = (double*)ctx->ws_mu.p;
  a.M = 2;
  a.cur = ctx->ws_phi[0].p;
  a.prev_out = ctx->ws_phi[1].p;
  TBPM_TRY(launch_moment_step(ctx, a, pl.precision, true));
  TBPM_CK(cudaMemcpyAsync(y, ctx->ws_phi[1].p, pl.state_bytes, cudaMemcpyDeviceToHost, ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return TBPM_OK;
}

// Block-size autotuner: measures t_amxsy and t_axpy on this lattice and request, then minimises
// the Tab. I cost model (Sec. II.B) under the memory cap.
int tbpm_block_autotune(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, int64_t n_steps,
                        int64_t* b_opt, double times_ms[2]) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !lat_c || !req || !b_opt || n_steps < 1) {
    set_error("tbpm_block_autotune: invalid argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  double ta = 0, tx = 0;
  TBPM_TRY(choose_block(ctx, lat, req, pl, n_steps, b_opt, &ta, &tx));
  if (times_ms) {
    times_ms[0] = ta;
    times_ms[1] = tx;
  }
  return TBPM_OK;
}

int tbpm_quasi_eigenstates(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, const double* energies,
                           int64_t nE, void* out) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !energies || !out || nE < 1) {
    set_error("tbpm_quasi_eigenstates: invalid argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  TBPM_TRY(ensure(ctx, ctx->ws_energies, sizeof(double) * (size_t)nE));
  TBPM_CK(cudaMemcpyAsync(ctx->ws_energies.p, energies, sizeof(double) * nE, cudaMemcpyHostToDevice, ctx->stream));
  TBPM_TRY(run_qe(ctx, lat, req, pl, (const double*)ctx->ws_energies.p, (int)nE));
  const int64_t n = lat->n_sites;
  for (int64_t k = 0; k < nE; ++k)
    for (int s = 0; s < pl.S; ++s)
      TBPM_CK(cudaMemcpy2DAsync((char*)out + ((size_t)k * pl.S + s) * n * pl.elem, pl.elem,
                                (const char*)ctx->ws_qe.p + (size_t)k * pl.state_bytes + s * pl.elem,
                                pl.Spad * pl.elem, pl.elem, n, cudaMemcpyDeviceToHost, ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return TBPM_OK;
}

int tbpm_conductivity(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, int direction,
                      const double* energies, int64_t nE, double* C, double* sigma) {
  return tbpm_conductivity_overlap(ctx, lat_c, req, direction, energies, nE, C, sigma, nullptr);
}

int tbpm_conductivity_overlap(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, int direction,
                              const double* energies, int64_t nE, double* C, double* sigma, double* overlap) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !energies || !sigma || nE < 1 || nE > 4096) {
    set_error("tbpm_conductivity: invalid argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  if (lat) TBPM_TRY(ensure_ell(ctx, lat));  // the current operator reads the ELL lists
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  TBPM_TRY(ensure(ctx, ctx->ws_energies, sizeof(double) * (size_t)nE));
  TBPM_CK(cudaMemcpyAsync(ctx->ws_energies.p, energies, sizeof(double) * nE, cudaMemcpyHostToDevice, ctx->stream));
  double *d_C = nullptr, *d_sigma = nullptr;
  TBPM_TRY(run_ec(ctx, lat, req, pl, (const double*)ctx->ws_energies.p, (int)nE, direction, &d_C, &d_sigma));
  // rows s*nE + k of the first S states are contiguous
  const size_t rows = (size_t)pl.S * nE;
  if (C)
    TBPM_CK(cudaMemcpyAsync(C, d_C, sizeof(double) * 2 * rows * (req->n_steps + 1), cudaMemcpyDeviceToHost,
                            ctx->stream));
  TBPM_CK(cudaMemcpyAsync(sigma, d_sigma, sizeof(double) * rows, cudaMemcpyDeviceToHost, ctx->stream));
  // <psi|Psi(E)> of every state and energy, [Spad][nE][2] at the head of the EC workspace
  if (overlap)
    TBPM_CK(cudaMemcpyAsync(overlap, ctx->ws_ec.p, sizeof(double) * 2 * rows, cudaMemcpyDeviceToHost, ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return TBPM_OK;
}

int tbpm_fermi_apply(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, double mu, double kT,
                     int sqrt_f, void* out) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !out) {
    set_error("tbpm_fermi_apply: invalid argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  TBPM_CK(cudaSetDevice(ctx->device));
  const double* coef = nullptr;
  int nf = 0;
  TBPM_TRY(fermi_series(ctx, lat, mu, kT, sqrt_f ? 1 : 0, &coef, &nf));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pl.state_bytes));
  TBPM_TRY(ensure(ctx, ctx->ws_phi2[0], pl.state_bytes));
  TBPM_TRY(init_states(ctx, lat, req, pl, ctx->ws_phi[0].p, nullptr));
  TBPM_TRY(apply_series_bufs(ctx, lat, pl, ctx->ws_phi[0].p, ctx->ws_phi[1].p, ctx->ws_phi2[0].p, coef, nf));
  const int64_t n = lat->n_sites;
  for (int s = 0; s < pl.S; ++s)
    TBPM_CK(cudaMemcpy2DAsync((char*)out + (size_t)s * n * pl.elem, pl.elem,
                              (const char*)ctx->ws_phi2[0].p + s * pl.elem, pl.Spad * pl.elem, pl.elem, n,
                              cudaMemcpyDeviceToHost, ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));
  return TBPM_OK;
}

namespace {
// Shared checks and the state-chunk loop of the OC, DP and CD entry points: `pass` runs the
// request's states s0 .. s0 + k - 1 with the chunk's plan.
int response_chunks(tbpm_ctx* ctx, tbpm_lattice* lat, const tbpm_request* req, int64_t min_steps,
                    double pair_blocks, const std::function<int(const tbpm_request*, const Plan&)>& pass) {
  Plan pl;
  TBPM_TRY(make_plan(lat, req, &pl));
  if (req->n_steps < min_steps || req->n_steps > (1 << 22)) {
    set_error("n_steps must lie in [%lld, 2^22]", (long long)min_steps);
    return TBPM_EINVAL;
  }
  if (req->form != TBPM_SEQUENTIAL && req->form != TBPM_CONCURRENT_S) {
    set_error("this quantity takes the SEQUENTIAL or CONCURRENT_S form");
    return TBPM_EINVAL;
  }
  int cap = std::min(pl.Spad, 16);
  if (ctx->max_pass_states > 0)
    while (cap > ctx->max_pass_states) cap >>= 1;
  const int k = states_per_pass(lat, pl.elem, cap, pair_blocks);
  if (k < 1) {
    set_error("not enough device memory for one state of %lld sites", (long long)lat->n_sites);
    return TBPM_ENOMEM;
  }
  for (int s0 = 0; s0 < pl.S; s0 += k) {
    tbpm_request rq = *req;
    rq.n_states = std::min(k, pl.S - s0);
    if (req->states == TBPM_STATES_SITES) rq.sites = req->sites + s0;
    Plan pk;
    TBPM_TRY(make_plan(lat, &rq, &pk));
    pk.s0 = s0;
    TBPM_TRY(pass(&rq, pk));
  }
  return TBPM_OK;
}
}  // namespace

int tbpm_optical_conductivity(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, int alpha,
                              int beta, double mu, double kT, double omega_max, int64_t n_omega, double* C,
                              double* sigma) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !req || !sigma || n_omega < 2 || n_omega > (1 << 20) || !(omega_max > 0.0)) {
    set_error("tbpm_optical_conductivity: invalid argument (n_omega in [2, 2^20], omega_max > 0)");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  if (!lat) {
    set_error("tbpm_optical_conductivity: lattice is NULL");
    return TBPM_EINVAL;
  }
  TBPM_TRY(ensure_ell(ctx, lat));  // the current operator reads the ELL lists
  const int dims = lat->desc.kind == TBPM_CUBIC ? 3 : 2;
  if (alpha < 0 || alpha >= dims || beta < 0 || beta >= dims) {
    set_error("directions must lie in [0, %d)", dims);
    return TBPM_EINVAL;
  }
  TBPM_CK(cudaSetDevice(ctx->device));
  const double area = lat->desc.kind == TBPM_HONEYCOMB ? 3.0 * sqrt(3.0) / 4.0 : 1.0;
  const int64_t W = req->n_steps + 1;
  const double q0[3] = {0, 0, 0};
  // 3 pair blocks = 6 single blocks live at a time, plus room for b >= 2 accumulators
  return response_chunks(ctx, lat, req, 1, 8.0, [&](const tbpm_request* rq, const Plan& pk) -> int {
    double* d_C = nullptr;
    double tphys = 0.0;
    TBPM_TRY(run_response(ctx, lat, rq, pk, 0, alpha, beta, q0, mu, kT, &d_C, &tphys));
    TBPM_TRY(ensure(ctx, ctx->ws_recon, sizeof(double) * 2 * (size_t)n_omega * pk.S));
    double* d_sig = (double*)ctx->ws_recon.p;
    TBPM_TRY(launch_oc_spectrum(ctx, d_C, pk.S, (int)rq->n_steps, omega_max / (double)(n_omega - 1), (int)n_omega,
                                kT, tphys, area, rq->window, d_sig));
    if (C)
      TBPM_CK(cudaMemcpyAsync(C + 2 * (size_t)pk.s0 * W, d_C, sizeof(double) * 2 * (size_t)pk.S * W,
                              cudaMemcpyDeviceToHost, ctx->stream));
    TBPM_CK(cudaMemcpyAsync(sigma + 2 * (size_t)pk.s0 * n_omega, d_sig, sizeof(double) * 2 * (size_t)pk.S * n_omega,
                            cudaMemcpyDeviceToHost, ctx->stream));
    TBPM_CK(cudaStreamSynchronize(ctx->stream));
    return TBPM_OK;
  });
}

int tbpm_polarization(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, const double q[3], double mu,
                      double kT, const double* omegas, int64_t n_omega, double* C, double* Pi) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !req || !q || !omegas || !Pi || n_omega < 1 || n_omega > (1 << 20)) {
    set_error("tbpm_polarization: invalid argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  TBPM_CK(cudaSetDevice(ctx->device));
  const double area = lat->desc.kind == TBPM_HONEYCOMB ? 3.0 * sqrt(3.0) / 4.0 : 1.0;
  const int64_t W = req->n_steps + 1;
  return response_chunks(ctx, lat, req, 1, 8.0, [&](const tbpm_request* rq, const Plan& pk) -> int {
    double* d_C = nullptr;
    double tphys = 0.0;
    TBPM_TRY(run_response(ctx, lat, rq, pk, 1, 0, 0, q, mu, kT, &d_C, &tphys));
    TBPM_TRY(ensure(ctx, ctx->ws_energies, sizeof(double) * (size_t)n_omega));
    TBPM_CK(cudaMemcpyAsync(ctx->ws_energies.p, omegas, sizeof(double) * n_omega, cudaMemcpyHostToDevice,
                            ctx->stream));
    TBPM_TRY(ensure(ctx, ctx->ws_recon, sizeof(double) * 2 * (size_t)n_omega * pk.S));
    double* d_pi = (double*)ctx->ws_recon.p;
    TBPM_TRY(launch_dp_spectrum(ctx, d_C, pk.S, (int)rq->n_steps, (const double*)ctx->ws_energies.p, (int)n_omega,
                                tphys, area, rq->window, d_pi));
    if (C)
      TBPM_CK(cudaMemcpyAsync(C + 2 * (size_t)pk.s0 * W, d_C, sizeof(double) * 2 * (size_t)pk.S * W,
                              cudaMemcpyDeviceToHost, ctx->stream));
    TBPM_CK(cudaMemcpyAsync(Pi + 2 * (size_t)pk.s0 * n_omega, d_pi, sizeof(double) * 2 * (size_t)pk.S * n_omega,
                            cudaMemcpyDeviceToHost, ctx->stream));
    TBPM_CK(cudaStreamSynchronize(ctx->stream));
    return TBPM_OK;
  });
}

int tbpm_charge_density(tbpm_ctx* ctx, const tbpm_lattice* lat_c, const tbpm_request* req, double mu, double kT,
                        double* rho) {
  clear_error();
  TBPM_NVTX_CALL(ctx);
  if (!ctx || !req || !rho) {
    set_error("tbpm_charge_density: invalid argument");
    return TBPM_EINVAL;
  }
  tbpm_lattice* lat = const_cast<tbpm_lattice*>(lat_c);
  TBPM_CK(cudaSetDevice(ctx->device));
  double tau = req->tau;
  if (tau == 0.0) {
    const double occ = std::min(lat->E_max, mu + 20.0 * kT) - lat->E_min;
    if (!(occ > 0.0)) {
      set_error("charge density: no occupied states below mu");
      return TBPM_EINVAL;
    }
    tau = M_PI * lat->half / occ;
  }
  const int64_t n = lat->n_sites;
  // live: three state blocks in the series, then 2 + b blocks and the FP64 accumulator (2 blocks)
  return response_chunks(ctx, lat, req, 0, 6.0, [&](const tbpm_request* rq, const Plan& pl) -> int {
    Plan pc = pl;
    pc.tau = tau;
    const double* coef = nullptr;
    int nf = 0;
    TBPM_TRY(fermi_series(ctx, lat, mu, kT, 1, &coef, &nf));
    TBPM_TRY(ensure(ctx, ctx->ws_phi[0], pl.state_bytes));
    TBPM_TRY(ensure(ctx, ctx->ws_phi[1], pl.state_bytes));
    TBPM_TRY(ensure(ctx, ctx->ws_phi2[0], pl.state_bytes));
    TBPM_TRY(init_states(ctx, lat, rq, pl, ctx->ws_phi[0].p, nullptr));
    // phi = f^{1/2}(H) psi into ws_phi2[0], consuming psi in ws_phi[0]
    TBPM_TRY(apply_series_bufs(ctx, lat, pl, ctx->ws_phi[0].p, ctx->ws_phi[1].p, ctx->ws_phi2[0].p, coef, nf));
    std::swap(ctx->ws_phi[0], ctx->ws_phi2[0]);
    release(ctx, ctx->ws_phi2[0]);
    const int64_t elems = n * pl.Spad;
    TBPM_TRY(ensure(ctx, ctx->ws_ec, sizeof(double) * (size_t)elems));
    double* z = (double*)ctx->ws_ec.p;
    TBPM_CK(cudaMemsetAsync(z, 0, sizeof(double) * (size_t)elems, ctx->stream));
    const int tok = phase_begin(ctx, 0);
    TBPM_TRY(launch_abs2py(ctx, pl.precision, ctx->ws_phi[0].p, 1, pl.state_bytes, elems, 0.5, z));
    if (rq->n_steps >= 1) {
      int64_t b = rq->form == TBPM_SEQUENTIAL ? 1 : rq->time_block;
      if (b <= 0) {
        std::swap(ctx->ws_phi[0], ctx->ws_phi2[0]);
        const int r = choose_block(ctx, lat, rq, pc, rq->n_steps, &b, nullptr, nullptr);
        std::swap(ctx->ws_phi[0], ctx->ws_phi2[0]);
        release(ctx, ctx->ws_phi2[0]);
        release(ctx, ctx->ws_psi);
        TBPM_TRY(r);
      }
      BlockHook hook = [&](int64_t, int bb, const void* first) -> int {
        return launch_abs2py(ctx, pl.precision, first, bb, pl.state_bytes, elems, 1.0, z);
      };
      TBPM_TRY(run_blocks(ctx, lat, rq, pc, rq->n_steps, b, nullptr, 0.0, hook, ctx->ws_phi[0].p, false));
    }
    phase_end(ctx, tok);
    TBPM_TRY(ensure(ctx, ctx->ws_out, sizeof(double) * (size_t)n * pl.S));
    const double wsum = 0.5 + (double)rq->n_steps;
    TBPM_TRY(launch_cd_finish(ctx, z, n, pl.S, pl.Spad, (double)n / wsum, (double*)ctx->ws_out.p));
    TBPM_CK(cudaMemcpyAsync(rho + (size_t)pl.s0 * n, ctx->ws_out.p, sizeof(double) * (size_t)n * pl.S,
                            cudaMemcpyDeviceToHost, ctx->stream));
    TBPM_CK(cudaStreamSynchronize(ctx->stream));
    return TBPM_OK;
  });
}

// ---------------------------------------------------------------- cost model (Sec. II.B, Tab. I)
int tbpm_block_counts(int64_t n_steps, int64_t b, double tau, int64_t out[3]) {
  clear_error();
  if (n_steps < 1 || b < 1 || !out || !(tau > 0)) {
    set_error("tbpm_block_counts: invalid argument");
    return TBPM_EINVAL;
  }
  int64_t amxsy = 0, axpy = 0;
  std::vector<int64_t> N(std::min(b, n_steps) + 1);
  for (int64_t j = 1; j <= std::min(b, n_steps); ++j) N[j] = truncation_order_host(j * tau);
  for (int64_t start = 0; start < n_steps; start += b) {
    const int64_t bb = std::min(b, n_steps - start);
    int64_t mx = 0;
    for (int64_t j = 1; j <= bb; ++j) {
      axpy += N[j];
      mx = std::max(mx, N[j]);
    }
    amxsy += mx;
  }
  out[0] = amxsy;
  out[1] = axpy;
  out[2] = n_steps;
  return TBPM_OK;
}

int64_t tbpm_block_opt(int64_t n_steps, double tau, double t_amxsy, double t_axpy, int64_t b_max) {
  clear_error();
  if (n_steps < 1 || !(tau > 0)) return 1;
  b_max = std::max<int64_t>(1, std::min(b_max, n_steps));
  std::vector<int64_t> N(b_max + 1), pre(b_max + 1, 0);
  for (int64_t j = 1; j <= b_max; ++j) {
    N[j] = truncation_order_host(j * tau);
    pre[j] = pre[j - 1] + N[j];
  }
  int64_t best = 1;
  double best_c = -1;
  for (int64_t b = 1; b <= b_max; ++b) {
    const int64_t full = n_steps / b, rest = n_steps % b;
    const double am = (double)full * N[b] + (rest ? (double)N[rest] : 0.0);
    const double ax = (double)full * pre[b] + (rest ? (double)pre[rest] : 0.0);
    const double c = am * t_amxsy + ax * t_axpy;
    if (best_c < 0 || c < best_c) {
      best_c = c;
      best = b;
    }
  }
  return best;
}

}  // extern "C"
