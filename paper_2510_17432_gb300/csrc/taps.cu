// Matrix-free moment pass for clean long-range lattices (square and honeycomb): H applied
// from the lattice's taps, every neighbour within the cutoff with t(r) = t exp(-(r-1)/decay),
// fused with the moments of the cost-halving identity (Sec. II.A, Eq. cheby_prod):
//     phi_{n+1} = 2 H~ phi_n - phi_{n-1},  A_n = <phi_n|phi_n>,  B_n = <phi_{n+1}|phi_n>.
//
// The paper's test Hamiltonians are dense (D_H up to 230 non-zeros per row, Sec. IV); with a
// few states the CSR/ELL form of such a matrix reads ~4 D_H bytes of indices per site and
// step, more than the states themselves.  Here the taps are the same for every site, so no
// index is stored: a CTA stages a halo'd tile of phi_n (one 16-byte pack = two complex64
// states per site; 64 honeycomb or 128 square cells by 32 rows) in shared memory and each
// thread computes 16 consecutive rows of one column of cells.  The taps of one destination
// sublattice, grouped by (dx, source sublattice), form runs along y; a run piece of n <= 8
// taps is applied to the 16 rows as a sliding window, so each shared load feeds up to 4n FMAs
// and the pass is bound by FP32 FMA issue rather than by HBM (2 (D_H - 1) FMAs per
// site-update against 24 bytes).
//
// Reductions follow the other moment kernels: Neumaier-compensated FP32 per thread, an FP64
// tree per CTA, per-CTA partials and a fixed-order sum by the last CTA to finish.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <vector>

#include "tbpm_internal.cuh"
#include "stencil.cuh"

namespace tbpm {
namespace {

// row blocks of 16 rows per CTA (4 warps each); two give 8-warp CTAs, two per SM
#ifndef TBPM_TAPS_RB
#define TBPM_TAPS_RB 2
#endif

// build-time variants (on the D_H = 235 workload the table read through L1 took 284 us per
// launch against 256 us staged in shared memory; the prefetch is off by default):
//   TBPM_TAPS_PREFETCH    1 = prefetch phi_{n-1} into L2 before the taps run
//   TBPM_TAPS_TABLE_SMEM  1 = chunk table staged in shared memory, 0 = read through L1
#ifndef TBPM_TAPS_PREFETCH
#define TBPM_TAPS_PREFETCH 0
#endif
#ifndef TBPM_TAPS_TABLE_SMEM
#define TBPM_TAPS_TABLE_SMEM 1
#endif

constexpr int kTapOY = 16;                       // output rows per thread
constexpr int kTapRB = TBPM_TAPS_RB;
constexpr int kTapTY = kTapOY * kTapRB;          // rows per tile
constexpr int kTapThreads = 128 * kTapRB;
constexpr int kTapMinBlocks = kTapRB == 1 ? 3 : 2;
constexpr int kTapMaxSmem = 227 * 1024;

// cells per tile along x: 64 (two warps per sublattice) on the honeycomb, 128 on the square
template <int NSUB>
struct TapShape {
  static constexpr int XS = 4 / NSUB;
  static constexpr int TX = 32 * XS;
};

__device__ __forceinline__ int64_t tap_wrap(int64_t v, int64_t L, int periodic, bool* ok) {
  if (v >= 0 && v < L) return v;
  if (!periodic) {
    *ok = false;
    return 0;
  }
  const int64_t r = v % L;
  return r < 0 ? r + L : r;
}

// acc[o] += sum_k w[k] col[(o + k) rs] for the 16 rows o: a sliding window over NW + 15 rows.
// The two states of a pack are two FP32 pairs (lo, hi); each pair takes one packed f32x2 FMA
// with the tap weight duplicated in both halves.
template <int NW>
__device__ __forceinline__ void tap_piece(float2 (&lo)[kTapOY], float2 (&hi)[kTapOY], const float4* col, int rs,
                                          const float* w) {
  float2 w2[NW];
#pragma unroll
  for (int k = 0; k < NW; ++k) {
#if TBPM_TAPS_TABLE_SMEM
    const float wk = w[k];
#else
    const float wk = __ldg(w + k);
#endif
    w2[k] = make_float2(wk, wk);
  }
#pragma unroll
  for (int j = 0; j < kTapOY + NW - 1; ++j) {
    const float4 v = col[j * rs];
    const float2 vl = make_float2(v.x, v.y), vh = make_float2(v.z, v.w);
#pragma unroll
    for (int k = 0; k < NW; ++k) {
      const int o = j - k;
      if (o >= 0 && o < kTapOY) {
        lo[o] = __ffma2_rn(w2[k], vl, lo[o]);
        hi[o] = __ffma2_rn(w2[k], vh, hi[o]);
      }
    }
  }
}

// MOM: fuse the moment sums (moment pass); without it the kernel is the plain recurrence step
// that the accumulation passes pair with an accumulate-only pass.
// EXACT: run pieces of every length 1..8 (fewer, longer pieces; best below D_H ~ 180), else
// pieces of 8, 4, 2 and 1 taps (fewer kernel variants in the dispatch; best at D_H = 235)
template <int NSUB, bool FIRST, bool MOM, bool EXACT>
__global__ void __launch_bounds__(kTapThreads, kTapMinBlocks) k_taps_moment(RecurrenceArgs a) {
  constexpr int TX = TapShape<NSUB>::TX;
  extern __shared__ float4 smem[];
  const int RX = a.taps_rx, RY = a.taps_ry;
  const int TW = TX + 2 * RX, TH = kTapTY + 2 * RY, RS = NSUB * TW;
  float4* tile = smem;
  const int nch = a.taps_n0 + (NSUB == 2 ? a.taps_n1 : 0);
  static_assert(sizeof(TapChunk) == 48, "chunk = 3 float4");
#if TBPM_TAPS_TABLE_SMEM
  TapChunk* ch = reinterpret_cast<TapChunk*>(smem + (size_t)TH * RS);
  for (int i = threadIdx.x; i < 3 * nch; i += kTapThreads) {
    const unsigned dst = (unsigned)__cvta_generic_to_shared(reinterpret_cast<float4*>(ch) + i);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst),
                 "l"(reinterpret_cast<const float4*>(a.taps) + i)
                 : "memory");
  }
#else
  const TapChunk* ch = a.taps;
#endif

  const int P = a.P;
  const int p = (int)(blockIdx.x % (unsigned)P);
  const int64_t tile_id = blockIdx.x / (unsigned)P;
  const int64_t Lx = a.geom.Lx, Ly = a.geom.Ly;
  const int64_t ntx = (Lx + TX - 1) / TX;
  const int64_t x0 = (tile_id % ntx) * TX, y0 = (tile_id / ntx) * kTapTY;
  const float4* cur = reinterpret_cast<const float4*>(a.cur);
  float4* po = reinterpret_cast<float4*>(a.prev_out);

  // stage phi_n of the tile and its halo (wrapped on periodic sides, zero on open ones) with
  // asynchronous 16-byte copies, all in flight at once
  // (one column (tx, s) per thread, walked down the rows: the column's wrap is computed once)
  for (int e = threadIdx.x; e < NSUB * TW; e += kTapThreads) {
    const int s = NSUB == 2 ? (e & 1) : 0;
    const int tx = NSUB == 2 ? (e >> 1) : e;
    bool okx = true;
    const int64_t gx = tap_wrap(x0 - RX + tx, Lx, a.geom.pbc_x, &okx);
    const float4* colsrc = cur + (gx * NSUB + s) * P + p;
    const int64_t rstride = Lx * NSUB * P;
    unsigned dst = (unsigned)__cvta_generic_to_shared(tile + s * TW + tx);
    for (int ty = 0; ty < TH; ++ty, dst += (unsigned)(RS * sizeof(float4))) {
      bool ok = okx;
      const int64_t gy = tap_wrap(y0 - RY + ty, Ly, a.geom.pbc_y, &ok);
      const float4* src = ok ? colsrc + gy * rstride : cur;
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(ok ? 16 : 0)
                   : "memory");
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lw = warp & 3, rb = warp >> 2;  // warp within its row block, row block
  const int sub = NSUB == 2 ? (lw & 1) : 0;
  const int xl = (NSUB == 2 ? (lw >> 1) : lw) * 32 + lane;
  const int r0 = RY + rb * kTapOY;          // tile row of this thread's first output row
#if TBPM_TAPS_PREFETCH
  // pull this thread's phi_{n-1} lines towards L2 while the taps run
  if (!FIRST && x0 + xl < Lx) {
#pragma unroll 4
    for (int o = 0; o < kTapOY; ++o) {
      const int64_t y = y0 + rb * kTapOY + o;
      if (y < Ly) asm volatile("prefetch.global.L2 [%0];" ::"l"(po + ((y * Lx + x0 + xl) * NSUB + sub) * P + p));
    }
  }
#endif
  float2 lo[kTapOY], hi[kTapOY];
#pragma unroll
  for (int o = 0; o < kTapOY; ++o) lo[o] = hi[o] = make_float2(0.f, 0.f);
  const int c_lo = sub == 0 ? 0 : a.taps_n0, c_hi = sub == 0 ? a.taps_n0 : nch;
  for (int c = c_lo; c < c_hi; ++c) {
#if TBPM_TAPS_TABLE_SMEM
    const int4 hd = *reinterpret_cast<const int4*>(ch + c);  // dx, dy0, ds, n
#else
    const int4 hd = __ldg(reinterpret_cast<const int4*>(ch + c));
#endif
    const float4* col = tile + (r0 + hd.y) * RS + hd.z * TW + RX + xl + hd.x;
    const float* w = ch[c].w;
    if constexpr (EXACT) {
      switch (hd.w) {
        case 8: tap_piece<8>(lo, hi, col, RS, w); break;
        case 7: tap_piece<7>(lo, hi, col, RS, w); break;
        case 6: tap_piece<6>(lo, hi, col, RS, w); break;
        case 5: tap_piece<5>(lo, hi, col, RS, w); break;
        case 4: tap_piece<4>(lo, hi, col, RS, w); break;
        case 3: tap_piece<3>(lo, hi, col, RS, w); break;
        case 2: tap_piece<2>(lo, hi, col, RS, w); break;
        default: tap_piece<1>(lo, hi, col, RS, w); break;
      }
    } else {
      switch (hd.w) {
        case 8: tap_piece<8>(lo, hi, col, RS, w); break;
        case 4: tap_piece<4>(lo, hi, col, RS, w); break;
        case 2: tap_piece<2>(lo, hi, col, RS, w); break;
        default: tap_piece<1>(lo, hi, col, RS, w); break;
      }
    }
  }

  // phi_{n+1} = d phi_n + th h (- phi_{n-1}) and the moment sums of the two states
  const float th = FIRST ? a.th1f : a.th2f;
  Acc<float> A0, A1, R0, R1, I0, I1;
  const int64_t x = x0 + xl;
#pragma unroll
  for (int o = 0; o < kTapOY; ++o) {
    const int64_t y = y0 + rb * kTapOY + o;
    if (x < Lx && y < Ly) {
      const int64_t site = (y * Lx + x) * NSUB + sub;
      const int64_t off = site * P + p;
      const float4 ph = tile[(r0 + o) * RS + sub * TW + RX + xl];
      float d = a.diag ? __ldg(reinterpret_cast<const float*>(a.diag) + site) : a.dc1f;
      if (!FIRST) d = d + d;
      float4 out;
      out.x = d * ph.x + th * lo[o].x;
      out.y = d * ph.y + th * lo[o].y;
      out.z = d * ph.z + th * hi[o].x;
      out.w = d * ph.w + th * hi[o].y;
      if (!FIRST) {
        const float4 pv = __ldcs(po + off);
        out.x -= pv.x;
        out.y -= pv.y;
        out.z -= pv.z;
        out.w -= pv.w;
      }
      (a.next ? reinterpret_cast<float4*>(a.next) : po)[off] = out;
      if constexpr (MOM) {
        A0.add(ph.x * ph.x + ph.y * ph.y);
        R0.add(out.x * ph.x + out.y * ph.y);
        I0.add(out.x * ph.y - out.y * ph.x);
        A1.add(ph.z * ph.z + ph.w * ph.w);
        R1.add(out.z * ph.z + out.w * ph.w);
        I1.add(out.z * ph.w - out.w * ph.z);
      }
    }
  }
  if constexpr (!MOM) return;

  // CTA sums (fixed trees), per-CTA partials, the last CTA sums them in CTA order
  double v[6] = {A0.value(), R0.value(), I0.value(), A1.value(), R1.value(), I1.value()};
#pragma unroll
  for (int k = 0; k < 6; ++k)
    for (int off = 16; off >= 1; off >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], off);
  __shared__ double red[kTapThreads / 32][6];
  __shared__ unsigned ticket;
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 6; ++k) red[warp][k] = v[k];
  __syncthreads();
  if (threadIdx.x < 6) {
    double s = 0.0;
    for (int w = 0; w < kTapThreads / 32; ++w) s += red[w][threadIdx.x];
    a.tap_partials[(size_t)blockIdx.x * 6 + threadIdx.x] = s;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(a.counter, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  const int64_t ntiles = gridDim.x / (unsigned)P;
  double* mu = a.mu;
  const int M = a.M, n = a.step;
  for (int q = warp; q < 6 * P; q += kTapThreads / 32) {
    const int pp = q / 6, k = q - 6 * pp;
    double s = 0.0;
    for (int64_t t = lane; t < ntiles; t += 32) s += __ldcg(a.tap_partials + (size_t)(t * P + pp) * 6 + k);
    for (int off = 16; off >= 1; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (lane == 0) {
      const int st = 2 * pp + k / 3, c = k % 3;
      double* ms = mu + (size_t)st * M * 2;
      if (FIRST) {
        if (c == 0) {
          ms[0] = s;
          ms[1] = 0.0;
        } else if (c == 1) {
          ms[2] = s;
        } else {
          ms[3] = s;
        }
      } else {
        if (c == 0) {
          ms[4 * n] = 2.0 * s - ms[0];
          ms[4 * n + 1] = -ms[1];
        } else if (c == 1) {
          ms[4 * n + 2] = 2.0 * s - ms[2];
        } else {
          ms[4 * n + 3] = 2.0 * s - ms[3];
        }
      }
    }
  }
  if (threadIdx.x == 0) *a.counter = 0u;
}

template <int NSUB>
int64_t tap_grid(const RecurrenceArgs& a) {
  constexpr int TX = TapShape<NSUB>::TX;
  return ((a.geom.Lx + TX - 1) / TX) * ((a.geom.Ly + kTapTY - 1) / kTapTY) * a.P;
}

template <int NSUB>
size_t tap_smem(int rx, int ry, int nch) {
  constexpr int TX = TapShape<NSUB>::TX;
  return (size_t)(kTapTY + 2 * ry) * NSUB * (TX + 2 * rx) * 16 + (TBPM_TAPS_TABLE_SMEM ? (size_t)nch * sizeof(TapChunk) : 0);
}

}  // namespace

size_t taps_partials_bytes(const RecurrenceArgs& a) {
  const int64_t g = a.geom.kind == TBPM_HONEYCOMB ? tap_grid<2>(a) : tap_grid<1>(a);
  return sizeof(double) * 6 * (size_t)g;
}

static int launch_taps(tbpm_ctx* ctx, const RecurrenceArgs& a, bool first, bool mom) {
  const bool hc = a.geom.kind == TBPM_HONEYCOMB;
  const int nch = a.taps_n0 + (hc ? a.taps_n1 : 0);
  const size_t smem = hc ? tap_smem<2>(a.taps_rx, a.taps_ry, nch) : tap_smem<1>(a.taps_rx, a.taps_ry, nch);
  const int64_t grid = hc ? tap_grid<2>(a) : tap_grid<1>(a);
  if (grid <= 0 || grid >= (1LL << 31) || smem > (size_t)kTapMaxSmem) {
    set_error("tap kernel: grid %lld or shared memory %zu out of range", (long long)grid, smem);
    return TBPM_EUNSUPPORTED;
  }
  // [exact][honeycomb][first][moments]
  static void* const fns[2][2][2][2] = {
      {{{(void*)k_taps_moment<1, false, false, false>, (void*)k_taps_moment<1, false, true, false>},
        {(void*)k_taps_moment<1, true, false, false>, (void*)k_taps_moment<1, true, true, false>}},
       {{(void*)k_taps_moment<2, false, false, false>, (void*)k_taps_moment<2, false, true, false>},
        {(void*)k_taps_moment<2, true, false, false>, (void*)k_taps_moment<2, true, true, false>}}},
      {{{(void*)k_taps_moment<1, false, false, true>, (void*)k_taps_moment<1, false, true, true>},
        {(void*)k_taps_moment<1, true, false, true>, (void*)k_taps_moment<1, true, true, true>}},
       {{(void*)k_taps_moment<2, false, false, true>, (void*)k_taps_moment<2, false, true, true>},
        {(void*)k_taps_moment<2, true, false, true>, (void*)k_taps_moment<2, true, true, true>}}}};
  void* fn = fns[a.taps_exact ? 1 : 0][hc ? 1 : 0][first ? 1 : 0][mom ? 1 : 0];
  TBPM_CK(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  RecurrenceArgs aa = a;
  void* args[] = {&aa};
  const cudaError_t e = cudaLaunchKernel(fn, dim3((unsigned)grid), dim3(kTapThreads), args, smem, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("tap kernel launch: %s", cudaGetErrorString(e));
    return TBPM_ECUDA;
  }
  return TBPM_OK;
}

int launch_taps_moment(tbpm_ctx* ctx, const RecurrenceArgs& a, bool first) { return launch_taps(ctx, a, first, true); }

int launch_taps_step(tbpm_ctx* ctx, const RecurrenceArgs& a, bool first) { return launch_taps(ctx, a, first, false); }

// Column-run pieces of the taps of every destination sublattice.  Sublattice 1 of the honeycomb
// takes each tap mirrored, (-dx, -dy, 1-ds), as the ELL builder does.  A run of one (dx, ds)
// spans its lowest to highest dy (holes weigh 0) and is cut into pieces of 8 taps and then one
// piece of the 1..7 that remain (below 180 taps per site, measured faster there: 141 against
// 152 us at D_H = 61) or pieces of 4, 2 and 1 (247 against 251 us at D_H = 235), so the tile
// halo is the largest |dx| and |dy| of any tap.  Lattices whose tile would not fit shared
// memory, cubic lattices and lattices with vacancies keep the ELL path only.
int build_tap_chunks(tbpm_ctx* ctx, tbpm_lattice* lat) {
  const tbpm_lattice_desc& d = lat->desc;
  if (lat->tap_t.empty() || d.kind == TBPM_CUBIC || d.vacancy_frac > 0.0) return TBPM_OK;
  const int nsub = d.kind == TBPM_HONEYCOMB ? 2 : 1;
  const size_t z = lat->tap_t.size();
  const bool exact = z < 180;
  std::vector<TapChunk> out;
  int rx = 0, ry = 0;
  for (int sub = 0; sub < nsub; ++sub) {
    std::map<std::pair<int, int>, std::map<int, float>> runs;  // (dx, ds) -> dy -> weight
    for (size_t k = 0; k < z; ++k) {
      int dx = lat->tap_off[4 * k], dy = lat->tap_off[4 * k + 1], ds = lat->tap_off[4 * k + 3];
      if (sub == 1) {
        dx = -dx;
        dy = -dy;
        ds = 1 - ds;
      }
      runs[{dx, ds}][dy] += (float)(lat->tap_t[k] / d.t);
    }
    int count = 0;
    for (auto& kv : runs) {
      const int lo = kv.second.begin()->first, hi = kv.second.rbegin()->first;
      for (int pos = lo; pos <= hi;) {
        TapChunk c;
        memset(&c, 0, sizeof(c));
        c.dx = kv.first.first;
        c.ds = kv.first.second;
        const int left = hi - pos + 1;
        c.n = exact ? std::min(8, left) : (left >= 8 ? 8 : left >= 4 ? 4 : left >= 2 ? 2 : 1);
        c.dy0 = pos;
        for (int k = 0; k < c.n; ++k) {
          auto it = kv.second.find(c.dy0 + k);
          c.w[k] = (c.dy0 + k < pos || it == kv.second.end()) ? 0.f : it->second;
        }
        rx = std::max(rx, std::abs(c.dx));
        ry = std::max(ry, std::max(std::abs(c.dy0), std::abs(c.dy0 + c.n - 1)));
        out.push_back(c);
        ++count;
        pos += c.n;
      }
    }
    lat->n_chunks[sub] = count;
  }
  const size_t smem = nsub == 2 ? tap_smem<2>(rx, ry, (int)out.size()) : tap_smem<1>(rx, ry, (int)out.size());
  if (smem > (size_t)kTapMaxSmem) {
    lat->n_chunks[0] = lat->n_chunks[1] = 0;
    return TBPM_OK;
  }
  lat->halo_x = rx;
  lat->halo_y = ry;
  lat->tap_exact = exact;
  TBPM_CK(cudaMallocAsync((void**)&lat->chunks, out.size() * sizeof(TapChunk), ctx->stream));
  TBPM_CK(cudaMemcpyAsync(lat->chunks, out.data(), out.size() * sizeof(TapChunk), cudaMemcpyHostToDevice,
                          ctx->stream));
  TBPM_CK(cudaStreamSynchronize(ctx->stream));  // the pageable source must outlive the copy
  return TBPM_OK;
}

}  // namespace tbpm
