// Serving: continuous batching of DOS / LDOS requests, one kernel launch per Chebyshev step.
//
// A scheduler thread admits queued requests by their HBM footprint, keeps their state blocks
// resident, and advances every active request by one Chebyshev step (moment-based form with
// the cost halving of Eq. cheby_prod) per launch of k_serve_step.  Requests of different
// lattice kinds, sizes, state counts and moment counts share that launch: the grid walks a
// global list of tiles, each tile belongs to one request and is processed with that request's
// stencil or ELL neighbour rule.  Every tile writes its own FP64 partial sums and the last tile
// of a request sums them in tile order, so a request's moments do not depend on what else is in
// the batch: results are bit-identical alone and in any mix.  A request that has produced its
// M moments leaves the batch, its DOS is reconstructed (Jackson kernel) and copied to pinned
// host memory, and its memory is released for the next admission.
//
// Requests large enough to fill the GPU with one step on their own (at least kLaneSiteStates
// site-states) do not join the batched kernel: each gets a direct lane, a context of its own
// whose stream runs the direct path's moment passes (the fused sweep where it applies, the
// one-step stencil or ELL pass otherwise) and the reconstruction, overlapping the batch and the
// other lanes on the device.  Which way a request goes depends only on the request, and both
// ways are deterministic, so a result is the same alone and in any mix.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "stencil.cuh"
#include "tbpm_internal.cuh"

namespace tbpm {

constexpr int kServeTU = 32 * kThreads;  // largest tile (32 units per thread, FP32 partial sums)
constexpr int64_t kLaneSiteStates = 1 << 21;  // full sites x padded states of a direct-lane request

// Units per tile of a request with `units` thread units: 32 per thread (the per-tile reduction
// and bookkeeping amortised) unless the request would get fewer than 64 tiles, then fewer.
// Depends only on the request, so its partial sums (and results) are the same alone and in any mix.
__host__ __device__ inline int serve_tile_units(int64_t units) {
  int upt = 1;
  while (upt < 32 && (int64_t)upt * kThreads * 64 < units) upt <<= 1;
  return upt * kThreads;
}

struct ServeItem {
  Geom geom;
  int path;
  const int32_t* ell;
  int precision, spt, S, P, logP;
  const void* diag;
  double diag_const, thop;
  float th1f, th2f, dc1f, dc2f;
  void* buf0;
  void* buf1;
  int64_t n_sites;
  int upr;              // units per x-line (stencil)
  int tiles_per_line;   // > 0: tiles are segments of one line
  int lines_per_tile;   // > 0: tiles hold whole short lines
  uint32_t line_magic;  // ceil(2^32 / upr), for u / upr with u < tu <= kServeTU
  int tu;               // units per tile (a multiple of kThreads, <= kServeTU)
  int64_t n_tiles, tile_begin;
  double* tile_partials;  // [n_tiles][S][3]
  unsigned* counter;
  double* mu;
  int M;
  int step;
};

// One unit: neighbour sum, output, and the unit's terms of A, B.
template <int KIND, bool CSR, typename R, int SPT>
__device__ __forceinline__ void serve_unit(const ServeItem& it, const Pack<R, SPT>* __restrict__ cur,
                                           Pack<R, SPT>* __restrict__ po, const LineBases& b, int64_t site_unit,
                                           int u, int p, bool first, R th, R dc, R (&acc)[3 * SPT]) {
  using PK = Pack<R, SPT>;
  constexpr int Z = CSR ? 6 : (KIND == TBPM_HONEYCOMB ? 3 : (KIND == TBPM_SQUARE ? 4 : 6));
  const int64_t own = site_unit;
  const PK ph = ld(cur + own);
  PK h;
#pragma unroll
  for (int w = 0; w < 2 * SPT; ++w) h.v[w] = R(0);
  if constexpr (CSR) {
    const int64_t site = own >> it.logP;
    const int z = it.geom.z;
    for (int d = 0; d < z; ++d) {
      const int64_t j = (int64_t)__ldg(it.ell + site * z + d);
      if (j >= 0) {
        const PK t = ld(cur + j * it.P + p);
#pragma unroll
        for (int w = 0; w < 2 * SPT; ++w) h.v[w] += t.v[w];
      }
    }
  } else {
    int64_t nb[6];
    stencil_neighbours<KIND>(it.geom, b, u, it.P, it.logP, p, it.upr, nb);
#pragma unroll
    for (int q = 0; q < Z; ++q) {
      if (q < 6 && nb[q] >= 0 && TBPM_DBG_OK(nb[q], it.n_sites * it.P, TBPM_DBG_SERVE)) {
        const PK t = ld(cur + nb[q]);
#pragma unroll
        for (int w = 0; w < 2 * SPT; ++w) h.v[w] += t.v[w];
      }
    }
  }
  R d = dc;
  if (it.diag) {
    const R dd = __ldg(reinterpret_cast<const R*>(it.diag) + (own >> it.logP));
    d = first ? dd : dd + dd;
  }
  PK o;
#pragma unroll
  for (int w = 0; w < 2 * SPT; ++w) o.v[w] = d * ph.v[w] + th * h.v[w];
  if (!first) {
    const PK pv = ld_stream(po + own);
#pragma unroll
    for (int w = 0; w < 2 * SPT; ++w) o.v[w] -= pv.v[w];
  }
  st(po + own, o);
#pragma unroll
  for (int q = 0; q < SPT; ++q) {
    const R pr = ph.v[2 * q], pi = ph.v[2 * q + 1], orr = o.v[2 * q], oi = o.v[2 * q + 1];
    acc[3 * q] += pr * pr + pi * pi;
    acc[3 * q + 1] += orr * pr + oi * pi;
    acc[3 * q + 2] += orr * pi - oi * pr;
  }
}

// One tile of one request; the last tile of the request finishes its step.
// `it` is the block's shared-memory copy; `git` the item in global memory, whose step field the
// last tile advances for the next launch.
template <int KIND, bool CSR, typename R, int SPT>
__device__ void serve_tile(const ServeItem* itp, ServeItem* git, int64_t lt, double (*red)[32][6], unsigned& ticket) {
  using PK = Pack<R, SPT>;
  const ServeItem& it = *itp;
  const int step = it.step;
  const bool first = step == 0;
  const PK* cur = reinterpret_cast<const PK*>((step & 1) ? it.buf1 : it.buf0);
  PK* po = reinterpret_cast<PK*>((step & 1) ? it.buf0 : it.buf1);
  const int P = it.P, p = threadIdx.x & (P - 1);
  R th, dc;
  if constexpr (sizeof(R) == 4) {
    th = first ? it.th1f : it.th2f;
    dc = first ? it.dc1f : it.dc2f;
  } else {
    th = first ? it.thop : 2.0 * it.thop;
    dc = first ? it.diag_const : 2.0 * it.diag_const;
  }
  R acc[3 * SPT];
#pragma unroll
  for (int k = 0; k < 3 * SPT; ++k) acc[k] = R(0);

  if constexpr (CSR) {
    const int64_t n_units = it.n_sites * P;
    const LineBases b{};
#pragma unroll 4
    for (int k = 0; k < it.tu / kThreads; ++k) {
      const int64_t u = lt * it.tu + k * kThreads + threadIdx.x;
      if (u < n_units) serve_unit<KIND, CSR, R, SPT>(it, cur, po, b, u, 0, p, first, th, dc, acc);
    }
  } else if (it.tiles_per_line > 0) {
    const int64_t line = lt / it.tiles_per_line;
    const int seg = (int)(lt - line * it.tiles_per_line);
    const LineBases b = line_bases<KIND>(it.geom, line, it.upr);
#pragma unroll 4
    for (int k = 0; k < it.tu / kThreads; ++k) {
      const int u = seg * it.tu + k * kThreads + threadIdx.x;
      if (u < it.upr) serve_unit<KIND, CSR, R, SPT>(it, cur, po, b, b.own + u, u, p, first, th, dc, acc);
    }
  } else {
    const int L = it.lines_per_tile;
    const int64_t line0 = lt * L;
#pragma unroll 4
    for (int k = 0; k < it.tu / kThreads; ++k) {
      const uint32_t uu = (uint32_t)(k * kThreads + threadIdx.x);
      const uint32_t lo = (uint32_t)(((uint64_t)uu * it.line_magic) >> 32);
      const int u = (int)(uu - lo * (uint32_t)it.upr);
      const int64_t line = line0 + lo;
      if ((int)lo < L && line < it.geom.n_rows) {
        const LineBases b = line_bases<KIND>(it.geom, line, it.upr);
        serve_unit<KIND, CSR, R, SPT>(it, cur, po, b, b.own + u, u, p, first, th, dc, acc);
      }
    }
  }

  // tile partial sums: FP32 (at most 32 units per thread) -> FP64 warp and block trees
  double v[3 * SPT];
#pragma unroll
  for (int k = 0; k < 3 * SPT; ++k) v[k] = (double)acc[k];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 3 * SPT; ++k)
    for (int off = 16; off >= P; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  if (lane < P) {
#pragma unroll
    for (int k = 0; k < 3 * SPT; ++k) red[warp][lane][k] = v[k];
  }
  __syncthreads();
  const int SC = it.S * 3;
  if (threadIdx.x < SC) {
    const int q = threadIdx.x, s = q / 3, c = q - 3 * s;
    const int pp = s / SPT, k = (s - pp * SPT) * 3 + c;
    double a = 0.0;
    for (int w = 0; w < kWarps; ++w) a += red[w][pp][k];
    it.tile_partials[(size_t)lt * SC + q] = a;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(it.counter, 1u);
  __syncthreads();
  if (ticket == (unsigned)(it.n_tiles - 1)) {
    __threadfence();
    for (int q = warp; q < SC; q += kWarps) {
      double a = 0.0;
      for (int64_t t = lane; t < it.n_tiles; t += 32) a += __ldcg(it.tile_partials + (size_t)t * SC + q);
      for (int off = 16; off >= 1; off >>= 1) a += __shfl_xor_sync(0xffffffffu, a, off);
      if (lane == 0) {
        const int s = q / 3, c = q - 3 * s;
        double* ms = it.mu + (size_t)s * it.M * 2;
        if (first) {
          if (c == 0) { ms[0] = a; ms[1] = 0.0; }
          else if (c == 1) ms[2] = a;
          else ms[3] = a;
        } else {
          if (c == 0) { ms[4 * step] = 2.0 * a - ms[0]; ms[4 * step + 1] = -ms[1]; }
          else if (c == 1) ms[4 * step + 2] = 2.0 * a - ms[2];
          else ms[4 * step + 3] = 2.0 * a - ms[3];
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      *it.counter = 0u;
      git->step = step + 1;
    }
  }
  __syncthreads();
}

template <int KIND, bool CSR>
__device__ __forceinline__ void serve_dispatch_prec(const ServeItem* it, ServeItem* git, int64_t lt,
                                                    double (*red)[32][6], unsigned& ticket) {
  if (it->precision == TBPM_C128) serve_tile<KIND, CSR, double, 1>(it, git, lt, red, ticket);
  else if (it->spt == 2) serve_tile<KIND, CSR, float, 2>(it, git, lt, red, ticket);
  else serve_tile<KIND, CSR, float, 1>(it, git, lt, red, ticket);
}

__global__ void __launch_bounds__(kThreads, 4) k_serve_step(ServeItem* items, int n_items, int64_t total_tiles) {
  __shared__ double red[kWarps][32][6];
  __shared__ unsigned ticket;
  __shared__ ServeItem sit;  // the tile's work item, staged once per tile
  __shared__ int sit_index;
  if (threadIdx.x == 0) sit_index = -1;
  __syncthreads();
  for (int64_t t = blockIdx.x; t < total_tiles; t += gridDim.x) {
    int lo = 0, hi = n_items - 1;
    while (lo < hi) {  // last item with tile_begin <= t
      const int mid = (lo + hi + 1) >> 1;
      if (items[mid].tile_begin <= t) lo = mid;
      else hi = mid - 1;
    }
    if (lo != sit_index) {
      __syncthreads();
      constexpr int W = sizeof(ServeItem) / sizeof(int);
      static_assert(sizeof(ServeItem) % sizeof(int) == 0, "item size");
      for (int w = threadIdx.x; w < W; w += blockDim.x)
        reinterpret_cast<int*>(&sit)[w] = reinterpret_cast<const int*>(items + lo)[w];
      if (threadIdx.x == 0) sit_index = lo;
      __syncthreads();
    }
    const int64_t lt = t - sit.tile_begin;
    if (sit.path == TBPM_PATH_CSR) serve_dispatch_prec<0, true>(&sit, items + lo, lt, red, ticket);
    else if (sit.geom.kind == TBPM_HONEYCOMB) serve_dispatch_prec<TBPM_HONEYCOMB, false>(&sit, items + lo, lt, red, ticket);
    else if (sit.geom.kind == TBPM_SQUARE) serve_dispatch_prec<TBPM_SQUARE, false>(&sit, items + lo, lt, red, ticket);
    else serve_dispatch_prec<TBPM_CUBIC, false>(&sit, items + lo, lt, red, ticket);
  }
}

}  // namespace tbpm

// ====================================================================== host scheduler
using namespace tbpm;
using Clock = std::chrono::steady_clock;

namespace {

enum { JOB_PENDING = 0, JOB_ACTIVE = 1, JOB_FINISHING = 2, JOB_DONE = 3 };

struct ServeJob {
  uint64_t ticket = 0;
  tbpm_lattice_desc ldesc{};
  tbpm_request req{};
  std::vector<int64_t> sites;
  std::vector<double> energies;
  Clock::time_point t_submit, t_admit, t_done;
  tbpm_lattice* lat = nullptr;
  void* buf[2] = {nullptr, nullptr};
  double* mu = nullptr;
  double* tile_partials = nullptr;
  unsigned* counter = nullptr;
  double* dE = nullptr;
  double* dD = nullptr;
  double* hD = nullptr;
  int* h_err = nullptr;
  size_t footprint = 0;
  int64_t steps_total = 0, steps_done = 0;
  int status = JOB_PENDING;
  int result = TBPM_OK;
  std::string message;
  cudaEvent_t done_ev = nullptr;
  ServeItem item{};
  int S = 1, Spad = 1, spt = 1, P = 1, logP = 0;
  size_t elem = 8, state_bytes = 0;
  int64_t n_tiles = 0;
  bool lane = false;            // direct lane: own context and stream, the direct path's kernels
  tbpm_ctx* lane_ctx = nullptr;
  std::thread lane_thread;      // enqueues the lane's work (may block on a full launch queue)
  std::atomic<int> lane_state{0};  // 0 enqueueing, 1 enqueued, 2 failed
  int lane_result = TBPM_OK;
};

int ilog2i(int v) {
  int r = 0;
  while ((1 << r) < v) ++r;
  return r;
}

}  // namespace

struct tbpm_server {
  tbpm_ctx* ctx = nullptr;      // compute stream of the scheduler
  tbpm_ctx* builder = nullptr;  // lattice construction (synchronises only its own stream)
  tbpm_server_config cfg{};
  size_t budget = 0, used = 0;
  std::thread th;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<ServeJob*> pending;
  std::vector<ServeJob*> active, finishing, lanes;
  std::unordered_map<uint64_t, ServeJob*> jobs;
  bool stop = false;
  uint64_t next_ticket = 1;
  ServeItem* d_items = nullptr;
  ServeItem* h_items[2] = {nullptr, nullptr};
  cudaEvent_t items_ev[2] = {nullptr, nullptr};
  int items_cap = 0, items_slot = 0;
  std::vector<cudaEvent_t> inflight;      // end of each in-flight launch (timed)
  std::vector<cudaEvent_t> inflight_beg;  // start of each in-flight launch
  std::vector<char> inflight_live;
  size_t inflight_head = 0;
  int64_t launches = 0, completed = 0;
  double gpu_ms = 0.0;  // summed device time of the batched launches
};

static size_t job_footprint(const ServeJob* j, int64_t n_sites, int64_t n_full, int z) {
  size_t lat = (size_t)n_sites * (8 + 4 + 8) + (j->ldesc.vacancy_frac > 0 ? (size_t)n_full * 8 + (size_t)n_sites * (8 + 4 * z) : 0);
  // a direct lane holds up to four state blocks (the fused passes write a second pair) and the
  // partial sums of its passes
  const size_t states = j->lane ? 4 * j->state_bytes + (16u << 20) : 2 * j->state_bytes;
  return lat + states + (size_t)j->n_tiles * j->Spad * 3 * 8 + (size_t)j->Spad * j->req.n_moments * 16 +
         j->energies.size() * 8 * (1 + j->S) + 4096;
}

static int64_t full_sites(const tbpm_lattice_desc& d) {
  const int64_t Lz = d.kind == TBPM_CUBIC ? d.L[2] : 1;
  return d.L[0] * d.L[1] * Lz * (d.kind == TBPM_HONEYCOMB ? 2 : 1);
}

// geometry-only tiling, identical alone and in a mix
static void plan_tiles(ServeJob* j, int64_t n_sites, const Geom& g, int path) {
  const int tu = serve_tile_units(n_sites * j->P);
  j->item.tu = tu;
  if (path == TBPM_PATH_CSR) {
    j->n_tiles = (n_sites * j->P + tu - 1) / tu;
    j->item.upr = 0;
    j->item.tiles_per_line = 0;
    j->item.lines_per_tile = 0;
    return;
  }
  const int upr = (int)(g.row_sites * j->P);
  j->item.upr = upr;
  if (upr >= tu) {
    j->item.tiles_per_line = (upr + tu - 1) / tu;
    j->item.lines_per_tile = 0;
    j->n_tiles = g.n_rows * j->item.tiles_per_line;
  } else {
    j->item.tiles_per_line = 0;
    j->item.lines_per_tile = tu / upr;
    j->item.line_magic = (uint32_t)(((1ull << 32) + upr - 1) / upr);
    j->n_tiles = (g.n_rows + j->item.lines_per_tile - 1) / j->item.lines_per_tile;
  }
}

static void fail_job(tbpm_server* srv, ServeJob* j, int code) {
  j->result = code;
  j->message = tbpm_last_error();
  j->status = JOB_DONE;
  j->t_done = Clock::now();
  (void)srv;
}

static void release_job(tbpm_server* srv, ServeJob* j) {
  cudaStream_t st = j->lane_ctx ? j->lane_ctx->stream : srv->ctx->stream;
  void* ps[] = {j->buf[0], j->buf[1], j->mu, j->tile_partials, j->counter, j->dE, j->dD};
  for (void* p : ps)
    if (p) cudaFreeAsync(p, st);
  j->buf[0] = j->buf[1] = nullptr;
  j->mu = j->tile_partials = j->dE = j->dD = nullptr;
  j->counter = nullptr;
  if (j->lat) {
    tbpm_lattice_destroy(j->lat);
    j->lat = nullptr;
  }
  if (j->done_ev) {
    cudaEventDestroy(j->done_ev);
    j->done_ev = nullptr;
  }
  if (j->lane_ctx) {  // waits for the lane's stream, frees its workspaces
    srv->launches += tbpm_launch_count(j->lane_ctx);
    tbpm_destroy(j->lane_ctx);
    j->lane_ctx = nullptr;
  }
}

// A direct lane: lattice (builder stream), buffers, then the whole request -- moment passes,
// reconstruction, copy of the DOS to pinned host memory -- enqueued on the lane's own stream.
static int setup_lane_job(tbpm_server* srv, ServeJob* j) {
  TBPM_TRY(tbpm_create(&j->lane_ctx, srv->ctx->device));
  tbpm_ctx* c = j->lane_ctx;
  c->max_queue = 128;  // the lane's thread waits instead of filling the launch queue
  TBPM_TRY(tbpm_lattice_create(c, &j->ldesc, &j->lat));
  tbpm_lattice* lat = j->lat;
  if (j->req.precision == TBPM_C128) TBPM_TRY(lattice_ensure_d64(lat));
  cudaStream_t st = c->stream;
  const int64_t M = j->req.n_moments, nE = (int64_t)j->energies.size();
  auto alloc = [&](void** p, size_t bytes) -> int {
    if (cudaMallocAsync(p, std::max<size_t>(bytes, 256), st) != cudaSuccess) {
      cudaGetLastError();
      set_error("serving: device allocation of %zu bytes failed", bytes);
      return TBPM_ENOMEM;
    }
    return TBPM_OK;
  };
  TBPM_TRY(alloc((void**)&j->mu, sizeof(double) * 2 * (size_t)M * j->Spad));
  TBPM_TRY(alloc((void**)&j->dE, sizeof(double) * nE));
  TBPM_TRY(alloc((void**)&j->dD, sizeof(double) * nE * j->S));
  TBPM_CK(cudaMemcpyAsync(j->dE, j->energies.data(), sizeof(double) * nE, cudaMemcpyHostToDevice, st));
  TBPM_CK(cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming));
  tbpm_request rq = j->req;
  rq.sites = j->sites.empty() ? nullptr : j->sites.data();
  TBPM_TRY(tbpm_moments_device(c, lat, &rq, j->mu));
  int r;
  if (srv->cfg.recon == TBPM_RECON_TENSOR)
    r = launch_dos_jackson_tensor_async(c, j->mu, j->S, (int)M, j->dE, nE, lat->H0, lat->half, j->dD, j->h_err);
  else
    r = launch_dos_jackson_fp64(c, j->mu, j->S, (int)M, j->dE, nE, lat->H0, lat->half, j->dD);
  TBPM_TRY(r);
  TBPM_CK(cudaMemcpyAsync(j->hD, j->dD, sizeof(double) * nE * j->S, cudaMemcpyDeviceToHost, st));
  TBPM_CK(cudaEventRecord(j->done_ev, st));
  return TBPM_OK;
}

// Device set-up of an admitted job: lattice (builder stream), buffers, initial states.
static int setup_job(tbpm_server* srv, ServeJob* j) {
  if (j->lane) return setup_lane_job(srv, j);
  tbpm_ctx* ctx = srv->ctx;
  TBPM_TRY(tbpm_lattice_create(srv->builder, &j->ldesc, &j->lat));
  tbpm_lattice* lat = j->lat;
  if (j->req.precision == TBPM_C128) TBPM_TRY(lattice_ensure_d64(lat));
  TBPM_CK(cudaStreamSynchronize(srv->builder->stream));
  plan_tiles(j, lat->n_sites, lat->geom, lat->path);
  j->state_bytes = (size_t)lat->n_sites * j->Spad * j->elem;
  cudaStream_t st = ctx->stream;
  const int64_t M = j->req.n_moments;
  auto alloc = [&](void** p, size_t bytes) -> int {
    if (cudaMallocAsync(p, std::max<size_t>(bytes, 256), st) != cudaSuccess) {
      cudaGetLastError();
      set_error("serving: device allocation of %zu bytes failed", bytes);
      return TBPM_ENOMEM;
    }
    return TBPM_OK;
  };
  TBPM_TRY(alloc(&j->buf[0], j->state_bytes));
  TBPM_TRY(alloc(&j->buf[1], j->state_bytes));
  TBPM_TRY(alloc((void**)&j->mu, sizeof(double) * 2 * (size_t)M * j->Spad));
  TBPM_TRY(alloc((void**)&j->tile_partials, sizeof(double) * 3 * (size_t)j->Spad * j->n_tiles));
  TBPM_TRY(alloc((void**)&j->counter, 256));
  TBPM_TRY(alloc((void**)&j->dE, sizeof(double) * j->energies.size()));
  TBPM_TRY(alloc((void**)&j->dD, sizeof(double) * j->energies.size() * j->S));
  TBPM_CK(cudaMemsetAsync(j->counter, 0, 256, st));
  TBPM_CK(cudaMemcpyAsync(j->dE, j->energies.data(), sizeof(double) * j->energies.size(), cudaMemcpyHostToDevice, st));
  TBPM_CK(cudaEventCreateWithFlags(&j->done_ev, cudaEventDisableTiming));
  tbpm_request rq = j->req;
  rq.sites = j->sites.empty() ? nullptr : j->sites.data();
  TBPM_TRY(init_request_states(ctx, lat, &rq, j->buf[0]));

  ServeItem& it = j->item;
  it.geom = lat->geom;
  it.path = lat->path;
  it.ell = lat->ell;
  it.precision = j->req.precision;
  it.spt = j->spt;
  it.S = j->Spad;
  it.P = j->P;
  it.logP = j->logP;
  it.diag = lat->has_v ? (j->req.precision == TBPM_C128 ? (const void*)lat->d64 : (const void*)lat->d32) : nullptr;
  it.diag_const = (0.0 - lat->H0) / lat->half;
  it.thop = lat->desc.t / lat->half;
  it.th1f = (float)it.thop;
  it.th2f = (float)(2.0 * it.thop);
  it.dc1f = (float)it.diag_const;
  it.dc2f = (float)(2.0 * it.diag_const);
  it.buf0 = j->buf[0];
  it.buf1 = j->buf[1];
  it.n_sites = lat->n_sites;
  it.n_tiles = j->n_tiles;
  it.tile_partials = j->tile_partials;
  it.counter = j->counter;
  it.mu = j->mu;
  it.M = (int)M;
  it.step = 0;
  return TBPM_OK;
}

static int upload_items(tbpm_server* srv) {
  const int n = (int)srv->active.size();
  if (n > srv->items_cap) {
    int cap = std::max(16, 2 * n);
    if (srv->d_items) cudaFreeAsync(srv->d_items, srv->ctx->stream);
    for (int k = 0; k < 2; ++k) {
      if (srv->h_items[k]) {
        cudaEventSynchronize(srv->items_ev[k]);
        cudaFreeHost(srv->h_items[k]);
      }
      TBPM_CK(cudaMallocHost((void**)&srv->h_items[k], sizeof(ServeItem) * cap));
    }
    TBPM_CK(cudaMallocAsync((void**)&srv->d_items, sizeof(ServeItem) * cap, srv->ctx->stream));
    srv->items_cap = cap;
  }
  const int slot = srv->items_slot;
  srv->items_slot ^= 1;
  TBPM_CK(cudaEventSynchronize(srv->items_ev[slot]));  // the copy that last used this slot is done
  int64_t begin = 0;
  for (int k = 0; k < n; ++k) {
    ServeJob* j = srv->active[k];
    j->item.tile_begin = begin;
    j->item.step = (int)j->steps_done;
    srv->h_items[slot][k] = j->item;
    begin += j->n_tiles;
  }
  TBPM_CK(cudaMemcpyAsync(srv->d_items, srv->h_items[slot], sizeof(ServeItem) * n, cudaMemcpyHostToDevice,
                          srv->ctx->stream));
  TBPM_CK(cudaEventRecord(srv->items_ev[slot], srv->ctx->stream));
  return TBPM_OK;
}

static int finish_job(tbpm_server* srv, ServeJob* j) {
  tbpm_ctx* ctx = srv->ctx;
  const int64_t nE = (int64_t)j->energies.size();
  const int M = (int)j->req.n_moments;
  int r;
  if (srv->cfg.recon == TBPM_RECON_TENSOR)
    r = launch_dos_jackson_tensor_async(ctx, j->mu, j->S, M, j->dE, nE, j->lat->H0, j->lat->half, j->dD, j->h_err);
  else
    r = launch_dos_jackson_fp64(ctx, j->mu, j->S, M, j->dE, nE, j->lat->H0, j->lat->half, j->dD);
  TBPM_TRY(r);
  TBPM_CK(cudaMemcpyAsync(j->hD, j->dD, sizeof(double) * nE * j->S, cudaMemcpyDeviceToHost, ctx->stream));
  TBPM_CK(cudaEventRecord(j->done_ev, ctx->stream));
  return TBPM_OK;
}

static void scheduler(tbpm_server* srv) {
  cudaSetDevice(srv->ctx->device);
  bool dirty = true;
  const size_t depth = 4;
  // a lane job's set-up and enqueue run on a thread of their own, so that the batch keeps going
  auto start_lane = [srv](ServeJob* j) {
    j->lane_thread = std::thread([srv, j] {
      cudaSetDevice(srv->ctx->device);
      const int r = setup_lane_job(srv, j);
      if (r != TBPM_OK) j->message = tbpm_last_error();
      j->lane_result = r;
      j->lane_state.store(r == TBPM_OK ? 1 : 2);
    });
  };
  while (true) {
    std::vector<ServeJob*> admitted;
    {
      std::unique_lock<std::mutex> lk(srv->mu);
      if (srv->stop) break;
      while (!srv->pending.empty() && (int)srv->active.size() + (int)admitted.size() < srv->cfg.max_active) {
        ServeJob* j = srv->pending.front();
        if (j->footprint > srv->budget) {
          srv->pending.pop_front();
          set_error("request footprint %zu B exceeds the serving HBM budget %zu B", j->footprint, srv->budget);
          fail_job(srv, j, TBPM_ENOMEM);
          srv->cv_done.notify_all();
          continue;
        }
        if (srv->used + j->footprint > srv->budget) break;  // FIFO: wait for memory to free up
        srv->pending.pop_front();
        srv->used += j->footprint;
        j->status = JOB_ACTIVE;
        j->t_admit = Clock::now();
        admitted.push_back(j);
      }
      if (admitted.empty() && srv->active.empty() && srv->finishing.empty() && srv->lanes.empty()) {
        srv->cv_work.wait_for(lk, std::chrono::milliseconds(2));
        continue;
      }
    }
    for (ServeJob* j : admitted) {
      if (j->lane) {
        start_lane(j);
        srv->lanes.push_back(j);
        continue;
      }
      int r = setup_job(srv, j);
      std::lock_guard<std::mutex> lk(srv->mu);
      if (r != TBPM_OK) {
        fail_job(srv, j, r);
        release_job(srv, j);
        srv->used -= j->footprint;
        srv->cv_done.notify_all();
      } else {
        srv->active.push_back(j);
        dirty = true;
      }
    }
    if (!srv->active.empty()) {
      if (dirty) {
        if (upload_items(srv) != TBPM_OK) {
          std::lock_guard<std::mutex> lk(srv->mu);
          for (ServeJob* j : srv->active) fail_job(srv, j, TBPM_ECUDA);
          srv->active.clear();
          srv->cv_done.notify_all();
          continue;
        }
        dirty = false;
      }
      int64_t total = 0;
      for (ServeJob* j : srv->active) total += j->n_tiles;
      // bound the queue depth so completion times and admission follow the device
      const size_t h = srv->inflight_head;
      if (srv->inflight.size() < depth) {
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        srv->inflight_beg.push_back(e0);
        srv->inflight.push_back(e1);
        srv->inflight_live.push_back(0);
      } else if (srv->inflight_live[h]) {
        cudaEventSynchronize(srv->inflight[h]);
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, srv->inflight_beg[h], srv->inflight[h]) == cudaSuccess) srv->gpu_ms += ms;
        srv->inflight_live[h] = 0;
      }
      const int grid = (int)std::min<int64_t>(total, (int64_t)srv->ctx->num_sms * 4);
      cudaEventRecord(srv->inflight_beg[h], srv->ctx->stream);
      k_serve_step<<<grid, kThreads, 0, srv->ctx->stream>>>(srv->d_items, (int)srv->active.size(), total);
      cudaEventRecord(srv->inflight[h], srv->ctx->stream);
      srv->inflight_live[h] = 1;
      srv->ctx->launches++;
      srv->launches++;
      srv->inflight_head = (h + 1) % depth;
      std::vector<ServeJob*> still;
      for (ServeJob* j : srv->active) {
        j->steps_done++;
        if (j->steps_done >= j->steps_total) {
          int r = finish_job(srv, j);
          std::lock_guard<std::mutex> lk(srv->mu);
          if (r != TBPM_OK) {
            fail_job(srv, j, r);
            release_job(srv, j);
            srv->used -= j->footprint;
            srv->cv_done.notify_all();
          } else {
            j->status = JOB_FINISHING;
            srv->finishing.push_back(j);
          }
          dirty = true;
        } else {
          still.push_back(j);
        }
      }
      srv->active.swap(still);
    }
    // direct lanes: set-up failures and completed streams
    {
      std::vector<ServeJob*> keep;
      for (ServeJob* j : srv->lanes) {
        const int st = j->lane_state.load();
        if (st == 0 || (st == 1 && cudaEventQuery(j->done_ev) != cudaSuccess)) {
          keep.push_back(j);
          continue;
        }
        j->lane_thread.join();
        std::lock_guard<std::mutex> lk(srv->mu);
        if (st == 2) {
          j->result = j->lane_result;
          j->status = JOB_DONE;
          j->t_done = Clock::now();
        } else {
          j->t_done = Clock::now();
          if (j->h_err && *j->h_err) {
            j->result = TBPM_ETIMEOUT;
            j->message = "tensor-core reconstruction: bounded wait expired";
          }
          j->status = JOB_DONE;
          srv->completed++;
        }
        release_job(srv, j);
        srv->used -= j->footprint;
        srv->cv_done.notify_all();
      }
      srv->lanes.swap(keep);
    }
    // completions
    std::vector<ServeJob*> left;
    for (ServeJob* j : srv->finishing) {
      if (cudaEventQuery(j->done_ev) == cudaSuccess) {
        std::lock_guard<std::mutex> lk(srv->mu);
        j->t_done = Clock::now();
        if (j->h_err && *j->h_err) {
          j->result = TBPM_ETIMEOUT;
          j->message = "tensor-core reconstruction: bounded wait expired";
        }
        release_job(srv, j);
        srv->used -= j->footprint;
        j->status = JOB_DONE;
        srv->completed++;
        srv->cv_done.notify_all();
      } else {
        left.push_back(j);
      }
    }
    srv->finishing.swap(left);
    if (srv->active.empty() && (!srv->finishing.empty() || !srv->lanes.empty()))
      std::this_thread::sleep_for(std::chrono::microseconds(20));
  }
  // shutdown: cancel everything still queued or running (a lane that is enqueued runs to its end)
  for (ServeJob* j : srv->lanes)
    if (j->lane_thread.joinable()) j->lane_thread.join();
  cudaStreamSynchronize(srv->ctx->stream);
  std::lock_guard<std::mutex> lk(srv->mu);
  for (ServeJob* j : srv->pending) {
    j->result = TBPM_ECANCELLED;
    j->status = JOB_DONE;
  }
  srv->pending.clear();
  for (auto* v : {&srv->active, &srv->finishing, &srv->lanes}) {
    for (ServeJob* j : *v) {
      release_job(srv, j);
      j->result = j->status == JOB_FINISHING ? TBPM_OK : TBPM_ECANCELLED;
      j->t_done = Clock::now();
      j->status = JOB_DONE;
    }
    v->clear();
  }
  srv->cv_done.notify_all();
}

extern "C" {

int tbpm_server_create(tbpm_ctx* ctx, const tbpm_server_config* cfg, tbpm_server** out) {
  clear_error();
  if (!ctx || !out) {
    set_error("tbpm_server_create: NULL argument");
    return TBPM_EINVAL;
  }
  *out = nullptr;
  tbpm_server* srv = new tbpm_server();
  if (cfg) srv->cfg = *cfg;
  if (srv->cfg.max_active <= 0) srv->cfg.max_active = 64;
  if (srv->cfg.max_queue <= 0) srv->cfg.max_queue = 4096;
  int r = tbpm_create(&srv->ctx, ctx->device);
  if (r == TBPM_OK) r = tbpm_create(&srv->builder, ctx->device);
  if (r == TBPM_OK) {
    // the batch (small requests) runs at the highest stream priority, so its kernels take SMs as
    // soon as the direct lanes' passes free them
    int least = 0, greatest = 0;
    cudaStream_t hi = nullptr;
    if (cudaDeviceGetStreamPriorityRange(&least, &greatest) == cudaSuccess &&
        cudaStreamCreateWithPriority(&hi, cudaStreamNonBlocking, greatest) == cudaSuccess) {
      cudaStreamSynchronize(srv->ctx->stream);
      cudaStreamDestroy(srv->ctx->stream);
      srv->ctx->stream = hi;
    }
    cudaGetLastError();
  }
  if (r != TBPM_OK) {
    if (srv->ctx) tbpm_destroy(srv->ctx);
    delete srv;
    return r;
  }
  size_t free_b = 0, total_b = 0;
  cudaSetDevice(ctx->device);
  cudaMemGetInfo(&free_b, &total_b);
  srv->budget = srv->cfg.hbm_budget_bytes ? srv->cfg.hbm_budget_bytes : (size_t)(0.7 * (double)free_b);
  for (int k = 0; k < 2; ++k) cudaEventCreateWithFlags(&srv->items_ev[k], cudaEventDisableTiming);
  srv->th = std::thread(scheduler, srv);
  *out = srv;
  return TBPM_OK;
}

int tbpm_server_destroy(tbpm_server* srv) {
  clear_error();
  if (!srv) return TBPM_OK;
  {
    std::lock_guard<std::mutex> lk(srv->mu);
    srv->stop = true;
  }
  srv->cv_work.notify_all();
  if (srv->th.joinable()) srv->th.join();
  cudaSetDevice(srv->ctx->device);
  cudaStreamSynchronize(srv->ctx->stream);
  for (auto& kv : srv->jobs) {
    release_job(srv, kv.second);
    if (kv.second->hD) cudaFreeHost(kv.second->hD);
    if (kv.second->h_err) cudaFreeHost(kv.second->h_err);
    delete kv.second;
  }
  for (int k = 0; k < 2; ++k) {
    if (srv->h_items[k]) cudaFreeHost(srv->h_items[k]);
    if (srv->items_ev[k]) cudaEventDestroy(srv->items_ev[k]);
  }
  for (cudaEvent_t e : srv->inflight) cudaEventDestroy(e);
  for (cudaEvent_t e : srv->inflight_beg) cudaEventDestroy(e);
  if (srv->d_items) cudaFreeAsync(srv->d_items, srv->ctx->stream);
  tbpm_destroy(srv->builder);
  tbpm_destroy(srv->ctx);
  delete srv;
  return TBPM_OK;
}

int tbpm_submit(tbpm_server* srv, const tbpm_lattice_desc* ldesc, const tbpm_request* req, const double* energies,
                int64_t n_energies, uint64_t* ticket) {
  clear_error();
  if (!srv || !ldesc || !req || !energies || !ticket || n_energies < 1) {
    set_error("tbpm_submit: invalid argument");
    return TBPM_EINVAL;
  }
  if (req->n_moments < 2 || (req->n_moments & 1) || req->n_states < 1 || req->n_states > 32 ||
      (req->precision != TBPM_C64 && req->precision != TBPM_C128) ||
      (req->states == TBPM_STATES_SITES && !req->sites)) {
    set_error("tbpm_submit: request needs even n_moments >= 2, 1 <= n_states <= 32, a known precision");
    return TBPM_EINVAL;
  }
  if (ldesc->kind < TBPM_SQUARE || ldesc->kind > TBPM_CUBIC || ldesc->L[0] < 1 || ldesc->L[1] < 1 ||
      (ldesc->kind == TBPM_CUBIC && ldesc->L[2] < 1)) {
    set_error("tbpm_submit: invalid lattice");
    return TBPM_EINVAL;
  }
  if (ldesc->cutoff != 0.0) {
    set_error("tbpm_submit: long-range hopping lattices are not served");
    return TBPM_EUNSUPPORTED;
  }
  ServeJob* j = new ServeJob();
  j->ldesc = *ldesc;
  if (j->ldesc.kind != TBPM_CUBIC) j->ldesc.L[2] = 1;
  j->req = *req;
  j->S = req->n_states;
  j->logP = 0;
  const int lg = ilog2i(j->S);
  j->Spad = 1 << lg;
  j->spt = (req->precision == TBPM_C64 && j->Spad >= 2) ? 2 : 1;
  j->P = j->Spad / j->spt;
  j->logP = ilog2i(j->P);
  j->elem = req->precision == TBPM_C64 ? 8 : 16;
  if (req->states == TBPM_STATES_SITES) j->sites.assign(req->sites, req->sites + req->n_states);
  j->req.sites = nullptr;
  j->energies.assign(energies, energies + n_energies);
  j->steps_total = req->n_moments / 2;
  const int64_t nf = full_sites(j->ldesc);
  const int z = ldesc->kind == TBPM_SQUARE ? 4 : ldesc->kind == TBPM_HONEYCOMB ? 3 : 6;
  j->state_bytes = (size_t)nf * j->Spad * j->elem;
  j->lane = nf * j->Spad >= kLaneSiteStates;
  const int tu = serve_tile_units(nf * j->P);
  j->n_tiles = j->lane ? 0 : (nf * j->P + tu - 1) / tu + (ldesc->L[1] * (ldesc->kind == TBPM_CUBIC ? ldesc->L[2] : 1));
  j->footprint = job_footprint(j, nf, nf, z);
  if (cudaMallocHost((void**)&j->hD, sizeof(double) * n_energies * j->S) != cudaSuccess ||
      cudaMallocHost((void**)&j->h_err, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    if (j->hD) cudaFreeHost(j->hD);
    delete j;
    set_error("tbpm_submit: pinned host allocation failed");
    return TBPM_ENOMEM;
  }
  *j->h_err = 0;
  std::lock_guard<std::mutex> lk(srv->mu);
  if ((int)srv->pending.size() >= srv->cfg.max_queue) {
    cudaFreeHost(j->hD);
    cudaFreeHost(j->h_err);
    delete j;
    set_error("tbpm_submit: queue full");
    return TBPM_EBUSY;
  }
  j->ticket = srv->next_ticket++;
  j->t_submit = Clock::now();
  srv->jobs[j->ticket] = j;
  srv->pending.push_back(j);
  *ticket = j->ticket;
  srv->cv_work.notify_all();
  return TBPM_OK;
}

int tbpm_wait(tbpm_server* srv, uint64_t ticket, int64_t timeout_us, double* D, size_t D_len, double* latency_us) {
  clear_error();
  if (!srv) {
    set_error("tbpm_wait: NULL server");
    return TBPM_EINVAL;
  }
  std::unique_lock<std::mutex> lk(srv->mu);
  auto it = srv->jobs.find(ticket);
  if (it == srv->jobs.end()) {
    set_error("tbpm_wait: unknown ticket %llu", (unsigned long long)ticket);
    return TBPM_EINVAL;
  }
  ServeJob* j = it->second;
  auto done = [&] { return j->status == JOB_DONE; };
  if (timeout_us < 0) {
    srv->cv_done.wait(lk, done);
  } else if (!srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), done)) {
    set_error("tbpm_wait: request %llu not finished within %lld us", (unsigned long long)ticket,
              (long long)timeout_us);
    return TBPM_ETIMEOUT;
  }
  const int result = j->result;
  if (result == TBPM_OK) {
    const size_t need = j->energies.size() * j->S;
    if (D && D_len >= need) memcpy(D, j->hD, sizeof(double) * need);
    else if (D) {
      set_error("tbpm_wait: output buffer holds %zu values, %zu needed", D_len, need);
      return TBPM_EINVAL;
    }
  } else {
    set_error("%s", j->message.empty() ? "request failed" : j->message.c_str());
  }
  if (latency_us) {
    using us = std::chrono::duration<double, std::micro>;
    latency_us[0] = us(j->t_admit - j->t_submit).count();
    latency_us[1] = us(j->t_done - j->t_admit).count();
    latency_us[2] = us(j->t_done - j->t_submit).count();
  }
  srv->jobs.erase(it);
  cudaFreeHost(j->hD);
  cudaFreeHost(j->h_err);
  delete j;
  return result;
}

int tbpm_server_stats(tbpm_server* srv, int64_t out[7]) {
  clear_error();
  if (!srv || !out) {
    set_error("tbpm_server_stats: NULL argument");
    return TBPM_EINVAL;
  }
  std::lock_guard<std::mutex> lk(srv->mu);
  out[0] = (int64_t)srv->pending.size();
  out[1] = (int64_t)(srv->active.size() + srv->lanes.size());
  out[2] = srv->completed;
  out[3] = srv->launches;
  out[4] = (int64_t)srv->used;
  out[5] = (int64_t)srv->budget;
  out[6] = (int64_t)(srv->gpu_ms * 1000.0);
  return TBPM_OK;
}

}  // extern "C"

TBPM_DEBUG_UNIT(serve)
