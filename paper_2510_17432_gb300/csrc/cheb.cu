// Chebyshev recurrence kernels for blocks of S states (App. B, Eq. cheb_relation):
//     phi_1 = H~ phi_0,   phi_{n+1} = 2 H~ phi_n - phi_{n-1},   H~ = (H - H0)/|H|,
// with H applied matrix-free on square / honeycomb / simple-cubic stencils, or from
// compact ELL neighbour lists on vacancy and long-range lattices (CSR/ELL path; long-range
// lattices carry one weight t_d/t per neighbour slot d).
//
// States are interleaved [site][state] so one thread unit moves 16 bytes (two complex64
// states, or one complex128 state) and the neighbour loads of all S states of a site are
// contiguous.  Each pass is fused with the inner products the method needs:
//   * moment pass (Sec. II.A, moment-based form, cost halving of Eq. cheby_prod):
//       A_n = <phi_n|phi_n>, B_n = <phi_{n+1}|phi_n>  ->  m_{2n} = 2A_n - m_0, m_{2n+1} = 2B_n - m_1;
//   * accumulation pass (Sec. II.A Eq. TE, time blocks of Sec. II.B; b = 1 is the sequential
//     form): acc_j += c_n(j tau~) phi_n for every step j of the block still open at term n,
//     and C(t_j) = <psi|acc_j> when term n closes step j.
// Reductions are deterministic: compensated FP32 (Neumaier) per thread for complex64,
// then FP64 warp and block trees, per-block partials, and a fixed-order sum by the last
// block to finish.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <type_traits>
#include <unordered_map>

#include "tbpm_internal.cuh"
#include "stencil.cuh"

namespace tbpm {

// ------------------------------------------------------------------ H~ phi for one unit
// Computes hphi = sum over neighbours of phi_j and the per-site diagonal term.
template <int KIND, bool CSR, typename R, int SPT>
struct Row {
  int64_t base, up, dn, zup, zdn;
  int32_t nb[6];  // ELL path, nearest-neighbour lists: the unit's indices, loaded one unit ahead
};

template <int KIND, bool CSR, typename R, int SPT>
__device__ __forceinline__ void neighbour_sum(const RecurrenceArgs& a, const Pack<R, SPT>* cur,
                                              int64_t site, int64_t x, int64_t sir, const Row<KIND, CSR, R, SPT>& rw,
                                              int p, Pack<R, SPT>& h) {
#pragma unroll
  for (int k = 0; k < 2 * SPT; ++k) h.v[k] = R(0);
  auto add = [&](int64_t j) {
    if (j >= 0 && TBPM_DBG_OK(j, a.n_sites, TBPM_DBG_ELL)) {
      const Pack<R, SPT> q = ld(cur + j * a.P + p);
#pragma unroll
      for (int k = 0; k < 2 * SPT; ++k) h.v[k] += q.v[k];
    }
  };
  if constexpr (CSR) {
    const int z = a.geom.z;
    const int32_t* row = a.ell + site * z;
    if (!a.wrel && z <= 6) {  // indices prefetched by the walk (for_each_unit)
#pragma unroll
      for (int d = 0; d < 6; ++d)
        if (d < z) add((int64_t)rw.nb[d]);
    } else if (a.wrel) {
      // long-range hopping: slot d carries the weight t_d / t
      const R* w = reinterpret_cast<const R*>(a.wrel);
      for (int d = 0; d < z; ++d) {
        const int32_t j = __ldg(row + d);
        if (j >= 0 && TBPM_DBG_OK(j, a.n_sites, TBPM_DBG_ELL)) {
          const R wd = __ldg(w + d);
          const Pack<R, SPT> q = ld(cur + (int64_t)j * a.P + p);
#pragma unroll
          for (int k = 0; k < 2 * SPT; ++k) h.v[k] = fma(wd, q.v[k], h.v[k]);
        }
      }
    } else {
      for (int d = 0; d < z; ++d) add((int64_t)__ldg(row + d));
    }
  } else if constexpr (KIND == TBPM_HONEYCOMB) {
    const int64_t Lx = a.geom.Lx;
    const int64_t xc = sir >> 1;
    const int s = (int)(sir & 1);
    add(rw.base + (sir ^ 1));                         // partner in the same cell
    int64_t xn = xc + (s ? 1 : -1);                   // A: B(x-1,y); B: A(x+1,y)
    bool ok = true;
    xn = wrap_coord(xn, Lx, a.geom.pbc_x, &ok);
    add(ok ? rw.base + 2 * xn + (1 - s) : -1);
    const int64_t nrow = s ? rw.up : rw.dn;           // A: B(x,y-1); B: A(x,y+1)
    add(nrow >= 0 ? nrow + 2 * xc + (1 - s) : -1);
  } else {
    const int64_t Lx = a.geom.Lx;
    bool ok = true;
    int64_t xp = wrap_coord(x + 1, Lx, a.geom.pbc_x, &ok);
    add(ok ? rw.base + xp : -1);
    ok = true;
    int64_t xm = wrap_coord(x - 1, Lx, a.geom.pbc_x, &ok);
    add(ok ? rw.base + xm : -1);
    add(rw.up >= 0 ? rw.up + x : -1);
    add(rw.dn >= 0 ? rw.dn + x : -1);
    if constexpr (KIND == TBPM_CUBIC) {
      add(rw.zup >= 0 ? rw.zup + x : -1);
      add(rw.zdn >= 0 ? rw.zdn + x : -1);
    }
  }
}

// Site base index of the row (y, z) and of its neighbouring rows (-1 when dropped).
template <int KIND, bool CSR, typename R, int SPT>
__device__ __forceinline__ Row<KIND, CSR, R, SPT> row_info(const Geom& g, int64_t row) {
  Row<KIND, CSR, R, SPT> rw{};
  const int64_t rs = g.row_sites;
  int64_t y = row, zc = 0;
  if constexpr (KIND == TBPM_CUBIC) {
    y = row % g.Ly;
    zc = row / g.Ly;
  }
  rw.base = row * rs;
  bool ok = true;
  int64_t yy = wrap_coord(y + 1, g.Ly, g.pbc_y, &ok);
  rw.up = ok ? (zc * g.Ly + yy) * rs : -1;
  ok = true;
  yy = wrap_coord(y - 1, g.Ly, g.pbc_y, &ok);
  rw.dn = ok ? (zc * g.Ly + yy) * rs : -1;
  if constexpr (KIND == TBPM_CUBIC) {
    ok = true;
    int64_t zz = wrap_coord(zc + 1, g.Lz, g.pbc_z, &ok);
    rw.zup = ok ? (zz * g.Ly + y) * rs : -1;
    ok = true;
    zz = wrap_coord(zc - 1, g.Lz, g.pbc_z, &ok);
    rw.zdn = ok ? (zz * g.Ly + y) * rs : -1;
  }
  return rw;
}

// Iterates over the thread's units: f(site, x, sir, row) for every valid unit.
// Stencil: tiles of kThreads units along one x-line; CSR: linear tiles.
template <int KIND, bool CSR, typename R, int SPT, typename F>
__device__ __forceinline__ void for_each_unit(const RecurrenceArgs& a, F f) {
  const int tid = threadIdx.x;
  if constexpr (CSR) {
    // nearest-neighbour ELL lists: the indices of the next unit are loaded before the current
    // unit's neighbours are gathered, so that the two dependent loads of a unit overlap with the
    // previous unit's instead of following each other
    const int64_t n_units = a.n_sites * a.P;
    const int64_t n_tiles = (n_units + kThreads - 1) / kThreads;
    const int z = a.geom.z;
    const bool pre = a.wrel == nullptr && z <= 6;
    auto load_idx = [&](int64_t u, int32_t* dst) {
      const int32_t* row = a.ell + (u >> a.logP) * z;
#pragma unroll
      for (int d = 0; d < 6; ++d) dst[d] = d < z ? __ldg(row + d) : -1;
    };
    Row<KIND, CSR, R, SPT> rw{};
    int64_t t = blockIdx.x;
    if (pre && t < n_tiles && t * kThreads + tid < n_units) load_idx(t * kThreads + tid, rw.nb);
    for (; t < n_tiles; t += gridDim.x) {
      const int64_t u = t * kThreads + tid;
      const int64_t un = (t + gridDim.x) * kThreads + tid;
      int32_t nxt[6] = {-1, -1, -1, -1, -1, -1};
      if (pre && t + gridDim.x < n_tiles && un < n_units) load_idx(un, nxt);
      if (u < n_units) f(u >> a.logP, (int64_t)0, (int64_t)0, rw);
#pragma unroll
      for (int d = 0; d < 6; ++d) rw.nb[d] = nxt[d];
    }
  } else {
    const int64_t upr = a.geom.row_sites * a.P;
    const int64_t tpr = (upr + kThreads - 1) / kThreads;
    const int64_t n_tiles = a.geom.n_rows * tpr;
    for (int64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
      const int64_t row = t / tpr;
      const int64_t u = (t - row * tpr) * kThreads + tid;
      if (u < upr) {
        const Row<KIND, CSR, R, SPT> rw = row_info<KIND, CSR, R, SPT>(a.geom, row);
        const int64_t sir = u >> a.logP;
        const int64_t x = (KIND == TBPM_HONEYCOMB) ? (sir >> 1) : sir;
        f(rw.base + sir, x, sir, rw);
      }
    }
  }
}

template <typename R>
__device__ __forceinline__ R site_diag(const RecurrenceArgs& a, int64_t site) {
  if (a.diag == nullptr) return coef_dc<R>(a, true);
  return __ldg(reinterpret_cast<const R*>(a.diag) + site);
}

// ------------------------------------------------------------------ moment pass
template <int KIND, bool CSR, typename R, int SPT, bool FIRST>
__global__ void __launch_bounds__(kThreads) k_moment_step(RecurrenceArgs a) {
  using PK = Pack<R, SPT>;
  const PK* cur = reinterpret_cast<const PK*>(a.cur);
  PK* po = reinterpret_cast<PK*>(a.prev_out);
  const int p = threadIdx.x & (a.P - 1);
  const R th = coef_th<R>(a, FIRST);
  Acc<R> A[SPT], Br[SPT], Bi[SPT];

  for_each_unit<KIND, CSR, R, SPT>(a, [&](int64_t site, int64_t x, int64_t sir,
                                          const Row<KIND, CSR, R, SPT>& rw) {
    const int64_t off = site * a.P + p;
    const PK ph = ld(cur + off);
    PK h;
    neighbour_sum<KIND, CSR, R, SPT>(a, cur, site, x, sir, rw, p, h);
    R d = site_diag<R>(a, site);
    if (!FIRST) d = d + d;
    PK o;
    if constexpr (FIRST) {
#pragma unroll
      for (int k = 0; k < 2 * SPT; ++k) o.v[k] = d * ph.v[k] + th * h.v[k];
    } else {
      const PK pv = ld_stream(po + off);
#pragma unroll
      for (int k = 0; k < 2 * SPT; ++k) o.v[k] = d * ph.v[k] + th * h.v[k] - pv.v[k];
    }
    st(po + off, o);
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
      const R pr = ph.v[2 * k], pi = ph.v[2 * k + 1], orr = o.v[2 * k], oi = o.v[2 * k + 1];
      A[k].add(pr * pr + pi * pi);
      Br[k].add(orr * pr + oi * pi);
      Bi[k].add(orr * pi - oi * pr);
    }
  });

  double v[3 * SPT];
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    v[3 * k] = A[k].value();
    v[3 * k + 1] = Br[k].value();
    v[3 * k + 2] = Bi[k].value();
  }
  double* mu = a.mu;
  const int M = a.M, n = a.step;
  grid_reduce<3 * SPT, SPT, 3>(v, a.P, a.S, a.partials, a.counter, a.nblocks, [&](int q, double val) {
    const int s = q / 3, c = q - 3 * s;
    double* ms = mu + (size_t)s * M * 2;
    if (FIRST) {
      if (c == 0) { ms[0] = val; ms[1] = 0.0; }
      else if (c == 1) ms[2] = val;
      else ms[3] = val;
    } else {
      if (c == 0) { ms[4 * n] = 2.0 * val - ms[0]; ms[4 * n + 1] = -ms[1]; }
      else if (c == 1) ms[4 * n + 2] = 2.0 * val - ms[2];
      else ms[4 * n + 3] = 2.0 * val - ms[3];
    }
  });
}

// ------------------------------------------------------------------ stencil moment pass (fast path)
// Launch shape of the pass: units per thread per super-tile and the CTAs per SM the register
// budget is sized for (overridable at build time for sweeps).
#ifndef TBPM_STENCIL_UPT
#define TBPM_STENCIL_UPT 2
#endif
#ifndef TBPM_STENCIL_MINB
#define TBPM_STENCIL_MINB 4
#endif
constexpr int kStencilUPT = TBPM_STENCIL_UPT;
constexpr int kStencilMinBlocks = TBPM_STENCIL_MINB;

// Matrix-free stencil version of the moment pass.  Work is walked in super-tiles of UPT x 256
// thread units along one x-line, so each thread keeps UPT independent units in flight; the
// line index advances incrementally (no division per unit) and neighbour offsets inside a
// line are 32-bit.  The inner products are summed in FP32 over at most 32 units per thread
// and then folded into FP64 (GB300 issues only 2 FP64 operations per clock per SM, so FP64
// work per unit is kept to a fraction of an operation).
template <int KIND, typename R, int SPT, bool FIRST>
__global__ void __launch_bounds__(kThreads, kStencilMinBlocks) k_moment_stencil(RecurrenceArgs a) {
  using PK = Pack<R, SPT>;
  constexpr int Z = KIND == TBPM_HONEYCOMB ? 3 : (KIND == TBPM_SQUARE ? 4 : 6);
  constexpr int TU = kStencilUPT * kThreads;
  const PK* __restrict__ cur = reinterpret_cast<const PK*>(a.cur);
  PK* __restrict__ po = reinterpret_cast<PK*>(a.prev_out);
  const R* __restrict__ diag = reinterpret_cast<const R*>(a.diag);
  const Geom g = a.geom;
  const int P = a.P, logP = a.logP, p = threadIdx.x & (P - 1);
  const int upr = (int)(g.row_sites * P);
  const int stpr = (upr + TU - 1) / TU;
  const R th = coef_th<R>(a, FIRST);
  const R dc = coef_dc<R>(a, FIRST);
  Partial<R> A[SPT], Br[SPT], Bi[SPT];

  int64_t row = blockIdx.x / stpr;
  int chunk = (int)(blockIdx.x - row * stpr);
  const int64_t gq = gridDim.x / stpr;
  const int gr = (int)(gridDim.x - gq * stpr);
  int64_t cached = -1;
  LineBases b{};
  int fold = 0;
  while (row < g.n_rows) {
    if (row != cached) {
      b = line_bases<KIND>(g, row, upr);
      cached = row;
    }
    PK ph[kStencilUPT], h[kStencilUPT], pv[kStencilUPT];
    bool valid[kStencilUPT];
    int64_t own[kStencilUPT];
    R d[kStencilUPT];
#pragma unroll
    for (int k = 0; k < kStencilUPT; ++k) {
      const int u = chunk * TU + k * kThreads + threadIdx.x;
      valid[k] = u < upr && TBPM_DBG_OK(b.own + u, g.n_full * P, TBPM_DBG_STENCIL);
#pragma unroll
      for (int q = 0; q < 2 * SPT; ++q) h[k].v[q] = R(0);
      if (valid[k]) {
        own[k] = b.own + u;
        ph[k] = ld(cur + own[k]);
        int64_t nb[6];
        stencil_neighbours<KIND>(g, b, u, P, logP, p, upr, nb);
#pragma unroll
        for (int q = 0; q < Z; ++q) {
          if (nb[q] >= 0 && TBPM_DBG_OK(nb[q], g.n_full * P, TBPM_DBG_STENCIL)) {
            const PK t = ld(cur + nb[q]);
#pragma unroll
            for (int w = 0; w < 2 * SPT; ++w) h[k].v[w] += t.v[w];
          }
        }
        if (!FIRST) pv[k] = ld_stream(po + own[k]);
        d[k] = dc;
        if (diag) {
          const R dd = __ldg(diag + (own[k] >> logP));
          d[k] = FIRST ? dd : dd + dd;
        }
      }
    }
#pragma unroll
    for (int k = 0; k < kStencilUPT; ++k) {
      if (!valid[k]) continue;
      PK o;
#pragma unroll
      for (int w = 0; w < 2 * SPT; ++w) {
        o.v[w] = d[k] * ph[k].v[w] + th * h[k].v[w];
        if (!FIRST) o.v[w] -= pv[k].v[w];
      }
      st_stream(po + own[k], o);
#pragma unroll
      for (int q = 0; q < SPT; ++q) {
        const R pr = ph[k].v[2 * q], pi = ph[k].v[2 * q + 1], orr = o.v[2 * q], oi = o.v[2 * q + 1];
        A[q].add(pr * pr + pi * pi);
        Br[q].add(orr * pr + oi * pi);
        Bi[q].add(orr * pi - oi * pr);
      }
    }
    if (++fold == 32 / kStencilUPT) {
      fold = 0;
#pragma unroll
      for (int q = 0; q < SPT; ++q) {
        A[q].fold();
        Br[q].fold();
        Bi[q].fold();
      }
    }
    chunk += gr;
    row += gq;
    if (chunk >= stpr) {
      chunk -= stpr;
      ++row;
    }
  }

  double v[3 * SPT];
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    v[3 * k] = A[k].value();
    v[3 * k + 1] = Br[k].value();
    v[3 * k + 2] = Bi[k].value();
  }
  double* mu = a.mu;
  const int M = a.M, n = a.step;
  grid_reduce<3 * SPT, SPT, 3>(v, a.P, a.S, a.partials, a.counter, a.nblocks, [&](int q, double val) {
    const int s = q / 3, c = q - 3 * s;
    double* ms = mu + (size_t)s * M * 2;
    if (FIRST) {
      if (c == 0) { ms[0] = val; ms[1] = 0.0; }
      else if (c == 1) ms[2] = val;
      else ms[3] = val;
    } else {
      if (c == 0) { ms[4 * n] = 2.0 * val - ms[0]; ms[4 * n + 1] = -ms[1]; }
      else if (c == 1) ms[4 * n + 2] = 2.0 * val - ms[2];
      else ms[4 * n + 3] = 2.0 * val - ms[3];
    }
  });
}

// ------------------------------------------------------------------ stencil accumulation pass (fast path)
// Same walk as k_moment_stencil (one unit per thread per tile); MODE as in k_accum_step.
template <int KIND, typename R, int SPT, int MODE>
__global__ void __launch_bounds__(kThreads, 4) k_accum_stencil(AccumArgs gargs) {
  using PK = Pack<R, SPT>;
  constexpr int Z = KIND == TBPM_HONEYCOMB ? 3 : (KIND == TBPM_SQUARE ? 4 : 6);
  const RecurrenceArgs& a = gargs.r;
  const PK* __restrict__ cur = reinterpret_cast<const PK*>(a.cur);
  PK* __restrict__ po = reinterpret_cast<PK*>(a.prev_out);
  PK* __restrict__ acc = reinterpret_cast<PK*>(gargs.acc);
  const PK* __restrict__ psi = reinterpret_cast<const PK*>(gargs.psi);
  const R* __restrict__ diag = reinterpret_cast<const R*>(a.diag);
  const Geom g = a.geom;
  const int P = a.P, logP = a.logP, p = threadIdx.x & (P - 1);
  const int upr = (int)(g.row_sites * P);
  const int tpr = (upr + kThreads - 1) / kThreads;
  const R th = coef_th<R>(a, MODE == ACC_FIRST);
  const R dc = coef_dc<R>(a, MODE == ACC_FIRST);
  const int64_t astr = gargs.acc_stride / SPT;
  const int jlo = gargs.j_lo, jb = gargs.b, jdone = gargs.j_done;
  const bool first_term = gargs.first_term != 0;
  Partial<R> Cr[SPT], Ci[SPT];

  int64_t row = blockIdx.x / tpr;
  int chunk = (int)(blockIdx.x - row * tpr);
  const int64_t gq = gridDim.x / tpr;
  const int gr = (int)(gridDim.x - gq * tpr);
  int64_t cached = -1;
  LineBases b{};
  int fold = 0;
  while (row < g.n_rows) {
    if (row != cached) {
      b = line_bases<KIND>(g, row, upr);
      cached = row;
    }
    const int u = chunk * kThreads + threadIdx.x;
    if (u < upr) {
      const int64_t own = b.own + u;
      const PK ph = ld(cur + own);
      if constexpr (MODE != ACC_NOSPMV) {
        PK h;
#pragma unroll
        for (int w = 0; w < 2 * SPT; ++w) h.v[w] = R(0);
        int64_t nb[6];
        stencil_neighbours<KIND>(g, b, u, P, logP, p, upr, nb);
#pragma unroll
        for (int q = 0; q < Z; ++q) {
          if (nb[q] >= 0) {
            const PK t = ld(cur + nb[q]);
#pragma unroll
            for (int w = 0; w < 2 * SPT; ++w) h.v[w] += t.v[w];
          }
        }
        R d = dc;
        if (diag) {
          const R dd = __ldg(diag + (own >> logP));
          d = (MODE == ACC_FIRST) ? dd : dd + dd;
        }
        PK o;
        if constexpr (MODE == ACC_FIRST) {
#pragma unroll
          for (int w = 0; w < 2 * SPT; ++w) o.v[w] = d * ph.v[w] + th * h.v[w];
        } else {
          const PK pv = ld_stream(po + own);
#pragma unroll
          for (int w = 0; w < 2 * SPT; ++w) o.v[w] = d * ph.v[w] + th * h.v[w] - pv.v[w];
        }
        st((a.next ? reinterpret_cast<PK*>(a.next) : po) + own, o);
      }
      for (int j = jlo; j < jb; ++j) {
        const R cr = (R)__ldg(gargs.coef + 2 * j), ci = (R)__ldg(gargs.coef + 2 * j + 1);
        PK* aj = acc + (int64_t)j * astr + own;
        PK av;
        if (first_term) {
#pragma unroll
          for (int w = 0; w < 2 * SPT; ++w) av.v[w] = R(0);
        } else {
          av = ld_stream(aj);
        }
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
          const R pr = ph.v[2 * q], pi = ph.v[2 * q + 1];
          av.v[2 * q] += cr * pr - ci * pi;
          av.v[2 * q + 1] += cr * pi + ci * pr;
        }
        st_stream(aj, av);
        if (j == jdone) {
          const PK s0 = ld(psi + own);
#pragma unroll
          for (int q = 0; q < SPT; ++q) {
            const R sr = s0.v[2 * q], si = s0.v[2 * q + 1];
            Cr[q].add(sr * av.v[2 * q] + si * av.v[2 * q + 1]);
            Ci[q].add(sr * av.v[2 * q + 1] - si * av.v[2 * q]);
          }
        }
      }
    }
    if (++fold == 32) {
      fold = 0;
#pragma unroll
      for (int q = 0; q < SPT; ++q) {
        Cr[q].fold();
        Ci[q].fold();
      }
    }
    chunk += gr;
    row += gq;
    if (chunk >= tpr) {
      chunk -= tpr;
      ++row;
    }
  }

  if (jdone < 0) return;
  double v[2 * SPT];
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    v[2 * k] = Cr[k].value();
    v[2 * k + 1] = Ci[k].value();
  }
  double* C = gargs.C;
  const int len = gargs.C_len, jg = gargs.j_global;
  grid_reduce<2 * SPT, SPT, 2>(v, a.P, a.S, a.partials, a.counter, a.nblocks, [&](int q, double val) {
    const int s = q >> 1, c = q & 1;
    C[((size_t)s * len + jg) * 2 + c] = val;
  });
}

// ------------------------------------------------------------------ accumulation pass
// MODE: ACC_FIRST (phi_1 = H~ phi_0), ACC_REGULAR, ACC_NOSPMV (last term: accumulate only).
template <int KIND, bool CSR, typename R, int SPT, int MODE>
__global__ void __launch_bounds__(kThreads) k_accum_step(AccumArgs g) {
  using PK = Pack<R, SPT>;
  const RecurrenceArgs& a = g.r;
  const PK* cur = reinterpret_cast<const PK*>(a.cur);
  PK* po = reinterpret_cast<PK*>(a.prev_out);
  PK* acc = reinterpret_cast<PK*>(g.acc);
  const PK* psi = reinterpret_cast<const PK*>(g.psi);
  const int p = threadIdx.x & (a.P - 1);
  const R th = coef_th<R>(a, MODE == ACC_FIRST);
  const int64_t astr = g.acc_stride / SPT;  // in packs
  Acc<R> Cr[SPT], Ci[SPT];

  for_each_unit<KIND, CSR, R, SPT>(a, [&](int64_t site, int64_t x, int64_t sir,
                                          const Row<KIND, CSR, R, SPT>& rw) {
    const int64_t off = site * a.P + p;
    const PK ph = ld(cur + off);
    if constexpr (MODE != ACC_NOSPMV) {
      PK h;
      neighbour_sum<KIND, CSR, R, SPT>(a, cur, site, x, sir, rw, p, h);
      R d = site_diag<R>(a, site);
      if (MODE != ACC_FIRST) d = d + d;
      PK o;
      if constexpr (MODE == ACC_FIRST) {
#pragma unroll
        for (int k = 0; k < 2 * SPT; ++k) o.v[k] = d * ph.v[k] + th * h.v[k];
      } else {
        const PK pv = ld_stream(po + off);
#pragma unroll
        for (int k = 0; k < 2 * SPT; ++k) o.v[k] = d * ph.v[k] + th * h.v[k] - pv.v[k];
      }
      st((a.next ? reinterpret_cast<PK*>(a.next) : po) + off, o);
    }
    for (int j = g.j_lo; j < g.b; ++j) {
      const R cr = (R)__ldg(g.coef + 2 * j), ci = (R)__ldg(g.coef + 2 * j + 1);
      PK* aj = acc + (int64_t)j * astr + off;
      PK av;
      if (g.first_term) {
#pragma unroll
        for (int k = 0; k < 2 * SPT; ++k) av.v[k] = R(0);
      } else {
        av = ld(aj);
      }
#pragma unroll
      for (int k = 0; k < SPT; ++k) {
        const R pr = ph.v[2 * k], pi = ph.v[2 * k + 1];
        av.v[2 * k] += cr * pr - ci * pi;
        av.v[2 * k + 1] += cr * pi + ci * pr;
      }
      st(aj, av);
      if (j == g.j_done) {
        const PK s0 = ld(psi + off);
#pragma unroll
        for (int k = 0; k < SPT; ++k) {
          const R sr = s0.v[2 * k], si = s0.v[2 * k + 1];
          Cr[k].add(sr * av.v[2 * k] + si * av.v[2 * k + 1]);
          Ci[k].add(sr * av.v[2 * k + 1] - si * av.v[2 * k]);
        }
      }
    }
  });

  if (g.j_done < 0) return;
  double v[2 * SPT];
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    v[2 * k] = Cr[k].value();
    v[2 * k + 1] = Ci[k].value();
  }
  double* C = g.C;
  const int len = g.C_len, jg = g.j_global;
  grid_reduce<2 * SPT, SPT, 2>(v, a.P, a.S, a.partials, a.counter, a.nblocks, [&](int q, double val) {
    const int s = q >> 1, c = q & 1;
    C[((size_t)s * len + jg) * 2 + c] = val;
  });
}

// ------------------------------------------------------------------ nearest-neighbour ELL step
// One Chebyshev step phi_{n+1} = 2 H~ phi_n - phi_{n-1} (phi_1 = H~ phi_0) on the compact ELL
// lists of a nearest-neighbour lattice with vacancies: with no accumulator and no inner product
// (MOM = false: the recurrence pass of the buffered time blocks and of the sequential form), or
// with the moment inner products of k_moment_step (MOM = true; FP32 partial sums over at most 32
// units per thread folded into FP64, then the deterministic grid reduction).  A CTA takes tiles
// of UPT x 256 units; thread t owns units t, t + 256, ... of the tile, so every load and store of
// a warp is one contiguous run.  All z index loads of the UPT units are issued first, then the
// own, previous and diagonal loads, then all z gathers, and only then the arithmetic: UPT (z + 3)
// independent loads in flight per thread, where the generic walk has two dependent rounds per
// unit; the index loads of the next tile are issued before the gathers of the current one.  Unit
// offsets are 32-bit (the host takes this kernel only below 2^31 - 2^24 units).
constexpr int kEllUPT = 4;

template <typename R, int SPT, int Z, bool FIRST, bool MOM>
__global__ void __launch_bounds__(kThreads) k_ell_step(RecurrenceArgs a) {
  using PK = Pack<R, SPT>;
  constexpr int UPT = kEllUPT, TU = UPT * kThreads;
  const PK* __restrict__ cur = reinterpret_cast<const PK*>(a.cur);
  const PK* prev = reinterpret_cast<const PK*>(a.prev_out);  // may be the output (in place)
  PK* out = reinterpret_cast<PK*>(a.next ? a.next : a.prev_out);
  const R* __restrict__ diag = reinterpret_cast<const R*>(a.diag);
  const int32_t* __restrict__ ell = a.ell;
  const int logP = a.logP, p = threadIdx.x & (a.P - 1);
  const int n_units = (int)(a.n_sites << logP);
  const R th = coef_th<R>(a, FIRST);
  const R dc = coef_dc<R>(a, true);
  Partial<R> A[SPT], Br[SPT], Bi[SPT];
  int fold = 0;
  const int stride = gridDim.x * TU;
  // the index lists of a tile are loaded one tile ahead, so that their round trip overlaps with
  // the gathers of the tile before
  auto load_idx = [&](int b0, int (&nbo)[UPT][Z], int (&so)[UPT]) {
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
      const int u = b0 + k * kThreads + (int)threadIdx.x;
      so[k] = u < n_units ? (u >> logP) : -1;
#pragma unroll
      for (int d = 0; d < Z; ++d) nbo[k][d] = so[k] >= 0 ? __ldg(ell + (int64_t)so[k] * Z + d) : -1;
    }
  };
  int nb[UPT][Z];
  int site[UPT];
  load_idx(blockIdx.x * TU, nb, site);
  for (int base = blockIdx.x * TU; base < n_units; base += stride) {
    int nbn[UPT][Z];
    int siten[UPT];
    load_idx(base + stride, nbn, siten);  // base + stride < 2^31: the host bounds the unit count
    PK ph[UPT], pv[UPT];
    R dd[UPT];
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
      const int u = base + k * kThreads + (int)threadIdx.x;
      if (site[k] >= 0) {
        ph[k] = ld(cur + u);
        if (!FIRST) pv[k] = ld_stream(prev + u);
        dd[k] = diag ? __ldg(diag + site[k]) : dc;
      }
    }
    PK h[UPT];
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
#pragma unroll
      for (int q = 0; q < 2 * SPT; ++q) h[k].v[q] = R(0);
#pragma unroll
      for (int d = 0; d < Z; ++d) {
        const int j = nb[k][d];
        if (j >= 0 && TBPM_DBG_OK(j, a.n_sites, TBPM_DBG_ELL)) {
          const PK q = ld(cur + (((int64_t)j << logP) + p));
#pragma unroll
          for (int c = 0; c < 2 * SPT; ++c) h[k].v[c] += q.v[c];
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
      if (site[k] < 0) continue;
      const int u = base + k * kThreads + (int)threadIdx.x;
      R d = dd[k];
      if (!FIRST) d = d + d;
      PK o;
      if constexpr (FIRST) {
#pragma unroll
        for (int c = 0; c < 2 * SPT; ++c) o.v[c] = d * ph[k].v[c] + th * h[k].v[c];
      } else {
#pragma unroll
        for (int c = 0; c < 2 * SPT; ++c) o.v[c] = d * ph[k].v[c] + th * h[k].v[c] - pv[k].v[c];
      }
      st(out + u, o);
      if constexpr (MOM) {
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
          const R pr = ph[k].v[2 * q], pi = ph[k].v[2 * q + 1], orr = o.v[2 * q], oi = o.v[2 * q + 1];
          A[q].add(pr * pr + pi * pi);
          Br[q].add(orr * pr + oi * pi);
          Bi[q].add(orr * pi - oi * pr);
        }
      }
    }
#pragma unroll
    for (int k = 0; k < UPT; ++k) {
      site[k] = siten[k];
#pragma unroll
      for (int d = 0; d < Z; ++d) nb[k][d] = nbn[k][d];
    }
    if constexpr (MOM) {
      if (++fold == 32 / UPT) {
        fold = 0;
#pragma unroll
        for (int q = 0; q < SPT; ++q) {
          A[q].fold();
          Br[q].fold();
          Bi[q].fold();
        }
      }
    }
  }
  if constexpr (MOM) {
    double v[3 * SPT];
#pragma unroll
    for (int q = 0; q < SPT; ++q) {
      v[3 * q] = A[q].value();
      v[3 * q + 1] = Br[q].value();
      v[3 * q + 2] = Bi[q].value();
    }
    double* mu = a.mu;
    const int M = a.M, n = a.step;
    grid_reduce<3 * SPT, SPT, 3>(v, a.P, a.S, a.partials, a.counter, a.nblocks, [&](int q, double val) {
      const int s = q / 3, c = q - 3 * s;
      double* ms = mu + (size_t)s * M * 2;
      if (FIRST) {
        if (c == 0) { ms[0] = val; ms[1] = 0.0; }
        else if (c == 1) ms[2] = val;
        else ms[3] = val;
      } else {
        if (c == 0) { ms[4 * n] = 2.0 * val - ms[0]; ms[4 * n + 1] = -ms[1]; }
        else if (c == 1) ms[4 * n + 2] = 2.0 * val - ms[2];
        else ms[4 * n + 3] = 2.0 * val - ms[3];
      }
    });
  }
}

// ------------------------------------------------------------------ plain dot <x|y> per state
template <typename R, int SPT>
__global__ void __launch_bounds__(kThreads) k_dot(RecurrenceArgs a, const void* xv, const void* yv,
                                                  double* out, int out_stride) {
  using PK = Pack<R, SPT>;
  const PK* X = reinterpret_cast<const PK*>(xv);
  const PK* Y = reinterpret_cast<const PK*>(yv);
  Acc<R> Cr[SPT], Ci[SPT];
  const int64_t n_units = a.n_sites * a.P;
  for (int64_t u = (int64_t)blockIdx.x * kThreads + threadIdx.x; u < n_units;
       u += (int64_t)gridDim.x * kThreads) {
    const PK xs = ld(X + u), ys = ld(Y + u);
#pragma unroll
    for (int k = 0; k < SPT; ++k) {
      Cr[k].add(xs.v[2 * k] * ys.v[2 * k] + xs.v[2 * k + 1] * ys.v[2 * k + 1]);
      Ci[k].add(xs.v[2 * k] * ys.v[2 * k + 1] - xs.v[2 * k + 1] * ys.v[2 * k]);
    }
  }
  double v[2 * SPT];
#pragma unroll
  for (int k = 0; k < SPT; ++k) {
    v[2 * k] = Cr[k].value();
    v[2 * k + 1] = Ci[k].value();
  }
  grid_reduce<2 * SPT, SPT, 2>(v, a.P, a.S, a.partials, a.counter, a.nblocks, [&](int q, double val) {
    const int s = q >> 1, c = q & 1;
    out[(size_t)s * out_stride * 2 + c] = val;
  });
}

// ------------------------------------------------------------------ quasi-eigenstate accumulation
// qe[k] += w_k x for k < nE with w_k = scale (cos, sgn sin)(theta_kj) from phase[k][j] = (cos, sin):
// the N_E axpy of the sequential and state-based quasi-eigenstate forms (Tab. I, QE rows).
template <typename R, int SPT>
__global__ void __launch_bounds__(kThreads) k_qe_axpy(const void* xv, void* qev, int64_t stride_packs, int64_t n_units,
                                                      const double* phase, int width, int j, double sgn, double scale,
                                                      int nE) {
  using PK = Pack<R, SPT>;
  const PK* X = reinterpret_cast<const PK*>(xv);
  PK* Q = reinterpret_cast<PK*>(qev);
  for (int64_t u = (int64_t)blockIdx.x * kThreads + threadIdx.x; u < n_units; u += (int64_t)gridDim.x * kThreads) {
    const PK x = ld(X + u);
    for (int k = 0; k < nE; ++k) {
      const double* ph = phase + ((int64_t)k * width + j) * 2;
      const R wr = (R)(scale * __ldg(ph)), wi = (R)(scale * sgn * __ldg(ph + 1));
      PK q = ld_stream(Q + k * stride_packs + u);
#pragma unroll
      for (int s = 0; s < SPT; ++s) {
        q.v[2 * s] += wr * x.v[2 * s] - wi * x.v[2 * s + 1];
        q.v[2 * s + 1] += wr * x.v[2 * s + 1] + wi * x.v[2 * s];
      }
      st_stream(Q + k * stride_packs + u, q);
    }
  }
}

// Buffered form of the energy-based quasi-eigenstate accumulation (Sec. IV, Eq. form2_concurrent):
// the recurrence writes T Chebyshev states phi_{n0} .. phi_{n0+T-1} once into a buffer, and one
// pass then adds sum_t C_{n0+t}(E) phi_{n0+t} to every accumulator, so each accumulator is read and
// written once per T terms instead of once per term.  grid (energy tiles of kQeEB, unit blocks):
// the energy tiles of one unit block run side by side and share the buffered states through L2.
constexpr int kQeEB = 16;
constexpr int kQeMaxT = 32;
template <typename R, int SPT>
__global__ void __launch_bounds__(kThreads) k_qe_flush(const void* phiv, int T, int64_t stride_packs, void* qev,
                                                       int nE, const double* coef, int n0, int64_t n_units) {
  using PK = Pack<R, SPT>;
  __shared__ R cs[kQeMaxT][kQeEB];
  const int e0 = blockIdx.x * kQeEB;
  const int ne = min(kQeEB, nE - e0);
  for (int i = threadIdx.x; i < T * kQeEB; i += kThreads) {
    const int t = i / kQeEB, e = i - t * kQeEB;
    cs[t][e] = e < ne ? (R)coef[((int64_t)(n0 + t) * nE + e0 + e) * 2] : R(0);  // C_n(E) is real
  }
  __syncthreads();
  const PK* Phi = reinterpret_cast<const PK*>(phiv);
  PK* Q = reinterpret_cast<PK*>(qev);
  for (int64_t u = (int64_t)blockIdx.y * kThreads + threadIdx.x; u < n_units; u += (int64_t)gridDim.y * kThreads) {
    PK acc[kQeEB];
#pragma unroll
    for (int e = 0; e < kQeEB; ++e) {
      if (e < ne) acc[e] = ld(Q + (int64_t)(e0 + e) * stride_packs + u);
      else
#pragma unroll
        for (int k = 0; k < 2 * SPT; ++k) acc[e].v[k] = R(0);
    }
    for (int t = 0; t < T; ++t) {
      const PK x = ld(Phi + (int64_t)t * stride_packs + u);
#pragma unroll
      for (int e = 0; e < kQeEB; ++e) {
        const R c = cs[t][e];
#pragma unroll
        for (int k = 0; k < 2 * SPT; ++k) acc[e].v[k] += c * x.v[k];
      }
    }
#pragma unroll
    for (int e = 0; e < kQeEB; ++e)
      if (e < ne) st(Q + (int64_t)(e0 + e) * stride_packs + u, acc[e]);
  }
}

// Complex64 form of k_qe_flush: the real weights C_n(E) of two energies sit in one shared quad
// (C_e, C_e, C_{e+1}, C_{e+1}), so one broadcast load feeds one packed f32x2 FMA per state and
// energy, (q_re, q_im) += C (x_re, x_im); each thread reads TB buffered terms before their FMAs.
template <int SPT, int TB>
__global__ void __launch_bounds__(kThreads, 2) k_qe_flush_c64(const void* phiv, int T, int64_t stride_packs,
                                                              void* qev, int nE, const double* coef, int n0,
                                                              int64_t n_units) {
  using PK = Pack<float, SPT>;
  constexpr int EB = kQeEB;
  __shared__ float4 cs[kQeMaxT][EB / 2];
  const int e0 = blockIdx.x * EB;
  const int ne = min(EB, nE - e0);
  for (int i = threadIdx.x; i < T * (EB / 2); i += kThreads) {
    const int t = i / (EB / 2), e = 2 * (i - t * (EB / 2));
    const float c0 = e < ne ? (float)coef[((int64_t)(n0 + t) * nE + e0 + e) * 2] : 0.f;  // C_n(E) is real
    const float c1 = e + 1 < ne ? (float)coef[((int64_t)(n0 + t) * nE + e0 + e + 1) * 2] : 0.f;
    cs[t][e / 2] = make_float4(c0, c0, c1, c1);
  }
  __syncthreads();
  const PK* Phi = reinterpret_cast<const PK*>(phiv);
  PK* Q = reinterpret_cast<PK*>(qev);
  for (int64_t u = (int64_t)blockIdx.y * kThreads + threadIdx.x; u < n_units; u += (int64_t)gridDim.y * kThreads) {
    float2 ac[EB][SPT];
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      PK q;
      if (e < ne) q = ld(Q + (int64_t)(e0 + e) * stride_packs + u);
      else
#pragma unroll
        for (int c = 0; c < 2 * SPT; ++c) q.v[c] = 0.f;
#pragma unroll
      for (int s = 0; s < SPT; ++s) ac[e][s] = make_float2(q.v[2 * s], q.v[2 * s + 1]);
    }
    for (int t0 = 0; t0 < T; t0 += TB) {
      PK x[TB];
#pragma unroll
      for (int j = 0; j < TB; ++j) {
        if (t0 + j < T) x[j] = ld(Phi + (int64_t)(t0 + j) * stride_packs + u);
        else
#pragma unroll
          for (int c = 0; c < 2 * SPT; ++c) x[j].v[c] = 0.f;
      }
#pragma unroll
      for (int j = 0; j < TB; ++j) {
        if (t0 + j >= T) break;  // uniform
#pragma unroll
        for (int e = 0; e < EB; e += 2) {
          if (e < ne) {  // uniform
            const float4 c = cs[t0 + j][e / 2];
            const float2 c0 = make_float2(c.x, c.y), c1 = make_float2(c.z, c.w);
#pragma unroll
            for (int s = 0; s < SPT; ++s) {
              const float2 xv = make_float2(x[j].v[2 * s], x[j].v[2 * s + 1]);
              ac[e][s] = __ffma2_rn(c0, xv, ac[e][s]);
              ac[e + 1][s] = __ffma2_rn(c1, xv, ac[e + 1][s]);
            }
          }
        }
      }
    }
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      if (e < ne) {
        PK q;
#pragma unroll
        for (int s = 0; s < SPT; ++s) {
          q.v[2 * s] = ac[e][s].x;
          q.v[2 * s + 1] = ac[e][s].y;
        }
        st(Q + (int64_t)(e0 + e) * stride_packs + u, q);
      }
    }
  }
}

// Buffered time-block accumulation: acc_j += sum_{t < T} c_t(j) phi_t for the open
// accumulators of a time block, with T buffered Chebyshev vectors phi_t (consecutive state
// blocks) and complex coefficients c_t(j) = coef[(t * nb + j) * 2 + {0, 1}] (zero once term t is
// past N(j tau~)).  Each accumulator is read and written once per T terms instead of once per
// term.  grid: (accumulator tiles of EB, unit blocks); EB = 1, 4 or 16 accumulators per tile
// (the registers of a tile's accumulators limit how many threads, and so how many buffer loads,
// an SM keeps in flight: a one-accumulator flush, the sequential form's, runs at full occupancy).
// Buffer loads in flight per thread: 8 for the small tiles, 4 for 16 accumulators (whose registers
// already bound the occupancy).
template <int EB>
struct FlushUnroll {
  static constexpr int value = EB >= 16 ? 4 : 8;
};

template <typename R, int SPT, int EB>
__global__ void __launch_bounds__(kThreads) k_block_flush(const void* phiv, int T, int64_t stride_packs, void* accv,
                                                          int nb, const double* coef, int64_t n_units) {
  using PK = Pack<R, SPT>;
  __shared__ R cr[kQeMaxT][EB], ci[kQeMaxT][EB];
  const int e0 = blockIdx.x * EB;
  const int ne = min(EB, nb - e0);
  for (int i = threadIdx.x; i < T * EB; i += kThreads) {
    const int t = i / EB, e = i - t * EB;
    const bool ok = e < ne;
    cr[t][e] = ok ? (R)coef[((int64_t)t * nb + e0 + e) * 2] : R(0);
    ci[t][e] = ok ? (R)coef[((int64_t)t * nb + e0 + e) * 2 + 1] : R(0);
  }
  __syncthreads();
  const PK* Phi = reinterpret_cast<const PK*>(phiv);
  PK* Q = reinterpret_cast<PK*>(accv);
  for (int64_t u = (int64_t)blockIdx.y * kThreads + threadIdx.x; u < n_units; u += (int64_t)gridDim.y * kThreads) {
    PK acc[EB];
#pragma unroll
    for (int e = 0; e < EB; ++e) {
      if (e < ne) acc[e] = ld(Q + (int64_t)(e0 + e) * stride_packs + u);
      else
#pragma unroll
        for (int k = 0; k < 2 * SPT; ++k) acc[e].v[k] = R(0);
    }
#pragma unroll (FlushUnroll<EB>::value)
    for (int t = 0; t < T; ++t) {  // unrolled so that several buffer loads are in flight
      const PK x = ld(Phi + (int64_t)t * stride_packs + u);
#pragma unroll
      for (int e = 0; e < EB; ++e) {
        if (e < ne) {  // uniform: a tile of fewer accumulators does no work for the rest
          const R a = cr[t][e], b = ci[t][e];
#pragma unroll
          for (int q = 0; q < SPT; ++q) {
            const R xr = x.v[2 * q], xi = x.v[2 * q + 1];
            acc[e].v[2 * q] += a * xr - b * xi;
            acc[e].v[2 * q + 1] += a * xi + b * xr;
          }
        }
      }
    }
#pragma unroll
    for (int e = 0; e < EB; ++e)
      if (e < ne) st(Q + (int64_t)(e0 + e) * stride_packs + u, acc[e]);
  }
}

// Complex64 flush of a tile of EB >= 4 accumulators with packed f32x2 FMAs.  The coefficient
// table holds (Re c, Re c, Im c, Im c) per term and accumulator, so one broadcast shared load
// feeds every state of the thread's U units, each with two packed FMAs:
//   (acc_re, acc_im) += Re c (x_re, x_im) + Im c (-x_im, x_re).
// Per term and accumulator that is 2 SPT U FMA instructions and 1 / (SPT U) shared loads per
// state, where the scalar flush above issues 4 FMAs and 2 shared loads per state (measured on a
// 32-term, 16-accumulator flush: 31 % fewer instructions than the same kernel with scalar FMAs).
template <int SPT, int EB, int U, int TB>
__global__ void __launch_bounds__(kThreads, 2) k_block_flush_c64(const void* phiv, int T, int64_t stride_packs,
                                                              void* accv, int nb, const double* coef,
                                                              int64_t n_units) {
  using PK = Pack<float, SPT>;
  __shared__ float4 cf[kQeMaxT][EB];
  const int e0 = blockIdx.x * EB;
  const int ne = min(EB, nb - e0);
  for (int i = threadIdx.x; i < T * EB; i += kThreads) {
    const int t = i / EB, e = i - t * EB;
    const bool ok = e < ne;
    const float cr = ok ? (float)coef[((int64_t)t * nb + e0 + e) * 2] : 0.f;
    const float ci = ok ? (float)coef[((int64_t)t * nb + e0 + e) * 2 + 1] : 0.f;
    cf[t][e] = make_float4(cr, cr, ci, ci);
  }
  __syncthreads();
  const PK* Phi = reinterpret_cast<const PK*>(phiv);
  PK* Q = reinterpret_cast<PK*>(accv);
  const int64_t step = (int64_t)gridDim.y * kThreads * U;
  for (int64_t ub = (int64_t)blockIdx.y * kThreads * U + threadIdx.x; ub < n_units; ub += step) {
    bool valid[U];
    float2 ac[U][EB][SPT];
#pragma unroll
    for (int k = 0; k < U; ++k) {
      valid[k] = ub + k * kThreads < n_units;
#pragma unroll
      for (int e = 0; e < EB; ++e) {
        PK q;
        if (valid[k] && e < ne) q = ld(Q + (int64_t)(e0 + e) * stride_packs + ub + k * kThreads);
        else
#pragma unroll
          for (int c = 0; c < 2 * SPT; ++c) q.v[c] = 0.f;
#pragma unroll
        for (int s = 0; s < SPT; ++s) ac[k][e][s] = make_float2(q.v[2 * s], q.v[2 * s + 1]);
      }
    }
    // the buffered vectors are read TB terms at a time, all loads issued before the FMAs, so
    // that TB loads per thread are in flight (the flush streams T + 2 ne state blocks)
    for (int t0 = 0; t0 < T; t0 += TB) {
      PK x[TB][U];
#pragma unroll
      for (int j = 0; j < TB; ++j)
#pragma unroll
        for (int k = 0; k < U; ++k) {
          if (valid[k] && t0 + j < T) x[j][k] = ld(Phi + (int64_t)(t0 + j) * stride_packs + ub + k * kThreads);
          else
#pragma unroll
            for (int c = 0; c < 2 * SPT; ++c) x[j][k].v[c] = 0.f;
        }
#pragma unroll
      for (int j = 0; j < TB; ++j) {
        if (t0 + j >= T) break;  // uniform
        float2 xs[U][SPT], xw[U][SPT];
#pragma unroll
        for (int k = 0; k < U; ++k)
#pragma unroll
          for (int s = 0; s < SPT; ++s) {
            xs[k][s] = make_float2(x[j][k].v[2 * s], x[j][k].v[2 * s + 1]);
            xw[k][s] = make_float2(-x[j][k].v[2 * s + 1], x[j][k].v[2 * s]);
          }
#pragma unroll
        for (int e = 0; e < EB; ++e) {
          if (e < ne) {  // uniform: a tile of fewer accumulators does no work for the rest
            const float4 c = cf[t0 + j][e];
            const float2 cre = make_float2(c.x, c.y), cim = make_float2(c.z, c.w);
#pragma unroll
            for (int k = 0; k < U; ++k)
#pragma unroll
              for (int s = 0; s < SPT; ++s) {
                ac[k][e][s] = __ffma2_rn(cre, xs[k][s], ac[k][e][s]);
                ac[k][e][s] = __ffma2_rn(cim, xw[k][s], ac[k][e][s]);
              }
          }
        }
      }
    }
#pragma unroll
    for (int k = 0; k < U; ++k) {
      if (!valid[k]) continue;
#pragma unroll
      for (int e = 0; e < EB; ++e) {
        if (e < ne) {
          PK q;
#pragma unroll
          for (int s = 0; s < SPT; ++s) {
            q.v[2 * s] = ac[k][e][s].x;
            q.v[2 * s + 1] = ac[k][e][s].y;
          }
          st(Q + (int64_t)(e0 + e) * stride_packs + ub + k * kThreads, q);
        }
      }
    }
  }
}

// ------------------------------------------------------------------ dispatch
template <typename R, int SPT>
static void* moment_kernel(int kind, bool csr, bool first) {
  if (csr) return first ? (void*)k_moment_step<0, true, R, SPT, true> : (void*)k_moment_step<0, true, R, SPT, false>;
  switch (kind) {
    case TBPM_SQUARE:
      return first ? (void*)k_moment_stencil<TBPM_SQUARE, R, SPT, true>
                   : (void*)k_moment_stencil<TBPM_SQUARE, R, SPT, false>;
    case TBPM_HONEYCOMB:
      return first ? (void*)k_moment_stencil<TBPM_HONEYCOMB, R, SPT, true>
                   : (void*)k_moment_stencil<TBPM_HONEYCOMB, R, SPT, false>;
    default:
      return first ? (void*)k_moment_stencil<TBPM_CUBIC, R, SPT, true>
                   : (void*)k_moment_stencil<TBPM_CUBIC, R, SPT, false>;
  }
}

// super-tiles of the stencil moment pass (2 x 256 units along one line)
static int64_t stencil_supertiles(const Geom& g, int P) {
  const int64_t upr = g.row_sites * P;
  return g.n_rows * ((upr + kStencilUPT * kThreads - 1) / (kStencilUPT * kThreads));
}

template <typename R, int SPT, int MODE>
static void* accum_kernel_m(int kind, bool csr) {
  if (csr) return (void*)k_accum_step<0, true, R, SPT, MODE>;
  switch (kind) {
    case TBPM_SQUARE: return (void*)k_accum_stencil<TBPM_SQUARE, R, SPT, MODE>;
    case TBPM_HONEYCOMB: return (void*)k_accum_stencil<TBPM_HONEYCOMB, R, SPT, MODE>;
    default: return (void*)k_accum_stencil<TBPM_CUBIC, R, SPT, MODE>;
  }
}

template <typename R, int SPT, bool MOM>
static void* ell_step_kernel(int z, bool first) {
  if (z == 3) return first ? (void*)k_ell_step<R, SPT, 3, true, MOM> : (void*)k_ell_step<R, SPT, 3, false, MOM>;
  if (z == 4) return first ? (void*)k_ell_step<R, SPT, 4, true, MOM> : (void*)k_ell_step<R, SPT, 4, false, MOM>;
  return first ? (void*)k_ell_step<R, SPT, 6, true, MOM> : (void*)k_ell_step<R, SPT, 6, false, MOM>;
}

// the batched nearest-neighbour ELL kernel applies: ELL lists without per-slot weights, z of
// 3, 4 or 6, fewer than 2^31 - 2^24 units
static bool ell_batched(const RecurrenceArgs& a) {
  const int z = a.geom.z;
  return a.path == TBPM_PATH_CSR && !a.wrel && (z == 3 || z == 4 || z == 6) &&
         a.n_sites * a.P < (int64_t)INT32_MAX - (int64_t)(1 << 24);
}


template <typename R, int SPT>
static void* accum_kernel(int kind, bool csr, int mode) {
  if (mode == ACC_FIRST) return accum_kernel_m<R, SPT, ACC_FIRST>(kind, csr);
  if (mode == ACC_REGULAR) return accum_kernel_m<R, SPT, ACC_REGULAR>(kind, csr);
  return accum_kernel_m<R, SPT, ACC_NOSPMV>(kind, csr);
}

static int spt_of(int precision, int S) { return (precision == TBPM_C64 && S >= 2) ? 2 : 1; }

// Upper bound of the persistent grid (partials are sized for it).
int recurrence_blocks(tbpm_ctx* ctx, int precision, int S) {
  (void)precision;
  (void)S;
  return ctx->num_sms * 8;
}

// Resident 256-thread blocks per SM of one kernel (occupancy API, cached per kernel).
static int resident_per_sm(void* fn) {
  static std::mutex mu;
  static std::unordered_map<void*, int> cache;
  std::lock_guard<std::mutex> lock(mu);
  auto it = cache.find(fn);
  if (it != cache.end()) return it->second;
  int nb = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, fn, kThreads, 0) != cudaSuccess || nb < 1) {
    cudaGetLastError();
    nb = 1;
  }
  nb = nb > 8 ? 8 : nb;
  cache[fn] = nb;
  return nb;
}

// Persistent grid: every resident slot filled once, never more blocks than tiles.
static int persistent_grid(tbpm_ctx* ctx, void* fn, int64_t n_tiles) {
  const int64_t g = (int64_t)ctx->num_sms * resident_per_sm(fn);
  return (int)(n_tiles < g ? (n_tiles > 0 ? n_tiles : 1) : g);
}

static int launch(tbpm_ctx* ctx, void* fn, int nblocks, void** args) {
  cudaError_t e = cudaLaunchKernel(fn, dim3(nblocks), dim3(kThreads), args, 0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("kernel launch: %s", cudaGetErrorString(e));
    return TBPM_ECUDA;
  }
  return TBPM_OK;
}

template <bool MOM>
static int launch_ell(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, bool first) {
  const int spt = spt_of(precision, a.S);
  void* fe;
  if (precision == TBPM_C128) fe = ell_step_kernel<double, 1, MOM>(a.geom.z, first);
  else if (spt == 2) fe = ell_step_kernel<float, 2, MOM>(a.geom.z, first);
  else fe = ell_step_kernel<float, 1, MOM>(a.geom.z, first);
  RecurrenceArgs ra = a;
  // the moment partials are sized for recurrence_blocks() CTAs
  ra.nblocks = persistent_grid(ctx, fe, (a.n_sites * a.P + kEllUPT * kThreads - 1) / (kEllUPT * kThreads));
  void* args[] = {&ra};
  return launch(ctx, fe, ra.nblocks, args);
}

int launch_moment_step(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, bool first) {
  const bool csr = a.path == TBPM_PATH_CSR;
  const int spt = spt_of(precision, a.S);
  if (a.taps && precision == TBPM_C64 && spt == 2) return launch_taps_moment(ctx, a, first);
  if (ell_batched(a)) return launch_ell<true>(ctx, a, precision, first);
  void* fn;
  if (precision == TBPM_C128) fn = moment_kernel<double, 1>(a.geom.kind, csr, first);
  else if (spt == 2) fn = moment_kernel<float, 2>(a.geom.kind, csr, first);
  else fn = moment_kernel<float, 1>(a.geom.kind, csr, first);
  RecurrenceArgs aa = a;
  aa.nblocks = persistent_grid(ctx, fn, csr ? a.n_tiles : stencil_supertiles(a.geom, a.P));
  void* args[] = {&aa};
  return launch(ctx, fn, aa.nblocks, args);
}

int launch_accum_step(tbpm_ctx* ctx, const AccumArgs& g, int precision, int mode) {
  const bool csr = g.r.path == TBPM_PATH_CSR;
  const int spt = spt_of(precision, g.r.S);
  if (g.r.taps && precision == TBPM_C64 && spt == 2 && mode != ACC_NOSPMV) {
    // long-range lattices: the matrix-free recurrence step, then the accumulate-only pass on phi_n
    TBPM_TRY(launch_taps_step(ctx, g.r, mode == ACC_FIRST));
    if (g.j_lo >= g.b && g.j_done < 0) return TBPM_OK;
    mode = ACC_NOSPMV;
  }
  if (mode != ACC_NOSPMV && g.j_lo >= g.b && g.j_done < 0 && ell_batched(g.r))
    return launch_ell<false>(ctx, g.r, precision, mode == ACC_FIRST);  // a plain step, loads batched
  void* fn;
  if (precision == TBPM_C128) fn = accum_kernel<double, 1>(g.r.geom.kind, csr, mode);
  else if (spt == 2) fn = accum_kernel<float, 2>(g.r.geom.kind, csr, mode);
  else fn = accum_kernel<float, 1>(g.r.geom.kind, csr, mode);
  AccumArgs gg = g;
  gg.r.nblocks = persistent_grid(ctx, fn, g.r.n_tiles);  // stencil: tiles of 256 units along a line
  void* args[] = {&gg};
  return launch(ctx, fn, gg.r.nblocks, args);
}

int launch_qe_axpy(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, const void* x, void* qe,
                   const double* phase, int width, int j, double sgn, double scale, int nE) {
  const int spt = spt_of(precision, a.S);
  const int64_t n_units = a.n_sites * a.P;
  const int grid = (int)std::min<int64_t>((n_units + kThreads - 1) / kThreads, (int64_t)ctx->num_sms * 8);
  void* fn;
  if (precision == TBPM_C128) fn = (void*)k_qe_axpy<double, 1>;
  else if (spt == 2) fn = (void*)k_qe_axpy<float, 2>;
  else fn = (void*)k_qe_axpy<float, 1>;
  int64_t stride = n_units;
  int64_t nu = n_units;
  void* args[] = {(void*)&x, &qe, &stride, &nu, (void*)&phase, &width, &j, &sgn, &scale, &nE};
  return launch(ctx, fn, grid, args);
}

int qe_flush_max_terms() { return kQeMaxT; }

int launch_qe_flush(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, const void* phi, int T, void* qe, int nE,
                    const double* coef, int n0) {
  if (T < 1 || T > kQeMaxT) {
    set_error("quasi-eigenstate flush of %d terms", T);
    return TBPM_EINVAL;
  }
  const int spt = spt_of(precision, a.S);
  const int64_t n_units = a.n_sites * a.P;
  const int etiles = (nE + kQeEB - 1) / kQeEB;
  const int64_t want = std::max<int64_t>(1, (int64_t)ctx->num_sms * 8 / etiles);
  const int ublocks = (int)std::min<int64_t>(std::min<int64_t>(want, (n_units + kThreads - 1) / kThreads), 65535);
  void* fn;
  if (precision == TBPM_C128) fn = (void*)k_qe_flush<double, 1>;
  else if (spt == 2) fn = (void*)k_qe_flush_c64<2, 2>;
  else fn = (void*)k_qe_flush_c64<1, 8>;
  int64_t stride = n_units;
  int64_t nu = n_units;
  void* args[] = {(void*)&phi, &T, &stride, &qe, &nE, (void*)&coef, &n0, &nu};
  cudaError_t e = cudaLaunchKernel(fn, dim3(etiles, ublocks), dim3(kThreads), args, 0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("kernel launch: %s", cudaGetErrorString(e));
    return TBPM_ECUDA;
  }
  return TBPM_OK;
}

int launch_block_flush(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, const void* phi, int T, void* acc,
                       int nb, const double* coef, int tile) {
  if (T < 1 || T > kQeMaxT || nb < 1) {
    set_error("block flush of %d terms into %d accumulators", T, nb);
    return TBPM_EINVAL;
  }
  const int spt = spt_of(precision, a.S);
  const int64_t n_units = a.n_sites * a.P;
  const int eb = tile > 0 ? tile : (nb == 1 ? 1 : nb <= 4 ? 4 : 16);
  const int etiles = (nb + eb - 1) / eb;
  const int64_t want = std::max<int64_t>(1, (int64_t)ctx->num_sms * (eb == 16 ? 8 : 16) / etiles);
  const int ublocks = (int)std::min<int64_t>(std::min<int64_t>(want, (n_units + kThreads - 1) / kThreads), 65535);
  void* fn;
  auto pick = [&](auto eb_tag) -> void* {
    constexpr int E = decltype(eb_tag)::value;
    if (precision == TBPM_C128) return (void*)k_block_flush<double, 1, E>;
    if constexpr (E >= 4) {  // complex64: packed FMAs
      if (spt == 2) return (void*)k_block_flush_c64<2, E, 1, 2>;
      return (void*)k_block_flush_c64<1, E, 1, 8>;
    }
    if (spt == 2) return (void*)k_block_flush<float, 2, E>;
    return (void*)k_block_flush<float, 1, E>;
  };
  if (eb == 1) fn = pick(std::integral_constant<int, 1>());
  else if (eb == 4) fn = pick(std::integral_constant<int, 4>());
  else fn = pick(std::integral_constant<int, 16>());
  int64_t stride = n_units;
  int64_t nu = n_units;
  void* args[] = {(void*)&phi, &T, &stride, &acc, &nb, (void*)&coef, &nu};
  cudaError_t e = cudaLaunchKernel(fn, dim3(etiles, ublocks), dim3(kThreads), args, 0, ctx->stream);
  ctx->launches++;
  if (e != cudaSuccess) {
    set_error("kernel launch: %s", cudaGetErrorString(e));
    return TBPM_ECUDA;
  }
  return TBPM_OK;
}

int launch_dot(tbpm_ctx* ctx, const RecurrenceArgs& a, int precision, const void* x, const void* y,
               double* out, int out_stride) {
  const int spt = spt_of(precision, a.S);
  void* fn;
  if (precision == TBPM_C128) fn = (void*)k_dot<double, 1>;
  else if (spt == 2) fn = (void*)k_dot<float, 2>;
  else fn = (void*)k_dot<float, 1>;
  RecurrenceArgs aa = a;
  aa.nblocks = persistent_grid(ctx, fn, (a.n_sites * a.P + kThreads - 1) / kThreads);
  void* args[] = {&aa, &x, &y, &out, &out_stride};
  return launch(ctx, fn, aa.nblocks, args);
}

}  // namespace tbpm

// ====================================================================== allocation-free moment step
// Some callers cannot let a library allocate device memory: applications that reserve nearly
// all HBM up front in their own arena (a cudaMalloc from the library would fail or fragment
// it), latency-critical loops where cudaMalloc/cudaFree may synchronise the device and stall
// other streams, and plugin hosts that hand buffers to their plugins but forbid them to
// allocate.  tbpm_moment_step_noalloc serves them: it runs one pass of the moment kernel on a
// matrix-free stencil with every state buffer supplied by the caller, and keeps the kernel's
// only scratch (per-block partial sums and the last-block counter) in the fixed array below.
namespace tbpm {

// Scratch of the allocation-free entry point: 256 bytes for the completion counter, then the
// per-block FP64 partial sums.  Every GPU that loads the library holds this array until the
// process exits.
constexpr size_t kNoAllocScratchBytes = 1u << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

// Device address of g_noalloc_scratch, looked up once per device with that device current.
static int noalloc_scratch_address(int device, unsigned char** out) {
  static std::mutex mu;
  static std::unordered_map<int, unsigned char*> addr;
  std::lock_guard<std::mutex> lock(mu);
  auto it = addr.find(device);
  if (it != addr.end()) {
    *out = it->second;
    return TBPM_OK;
  }
  void* p = nullptr;
  cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
  if (e != cudaSuccess || p == nullptr) {
    set_error("cudaGetSymbolAddress(g_noalloc_scratch) failed: %s", cudaGetErrorString(e));
    return TBPM_ECUDA;
  }
  addr[device] = (unsigned char*)p;
  *out = (unsigned char*)p;
  return TBPM_OK;
}

}  // namespace tbpm

extern "C" int tbpm_moment_step_noalloc(int kind, const int64_t L[3], const int32_t pbc[3], double t_scaled,
                                        double diag_const, const void* d_diag, int precision, int n_states,
                                        const void* d_cur, void* d_prev_out, double* d_mu, int64_t n_moments,
                                        int64_t step, void* stream) {
  using namespace tbpm;
  clear_error();
  if (!L || !pbc || !d_cur || !d_prev_out || !d_mu) {
    set_error("tbpm_moment_step_noalloc: NULL argument");
    return TBPM_EINVAL;
  }
  if (kind < TBPM_SQUARE || kind > TBPM_CUBIC || (precision != TBPM_C64 && precision != TBPM_C128)) {
    set_error("tbpm_moment_step_noalloc: unknown lattice kind or precision");
    return TBPM_EINVAL;
  }
  if (n_states < 1 || n_states > 32 || (n_states & (n_states - 1))) {
    set_error("tbpm_moment_step_noalloc: n_states must be a power of two <= 32 (got %d)", n_states);
    return TBPM_EINVAL;
  }
  if (n_moments < 2 || (n_moments & 1) || n_moments > INT32_MAX || step < 0 || step >= n_moments / 2) {
    set_error("tbpm_moment_step_noalloc: need even n_moments >= 2 and 0 <= step < n_moments/2");
    return TBPM_EINVAL;
  }
  Geom g{};
  g.kind = kind;
  g.Lx = L[0];
  g.Ly = L[1];
  g.Lz = kind == TBPM_CUBIC ? L[2] : 1;
  if (g.Lx < 1 || g.Ly < 1 || g.Lz < 1 || (double)g.Ly * (double)g.Lz >= 2147483648.0) {
    set_error("tbpm_moment_step_noalloc: lattice sizes must be >= 1 with Ly*Lz below 2^31");
    return TBPM_EINVAL;
  }
  g.pbc_x = pbc[0] != 0;
  g.pbc_y = pbc[1] != 0;
  g.pbc_z = kind == TBPM_CUBIC ? pbc[2] != 0 : 1;  // a 2-D caller may pass a two-entry pbc array
  g.z = kind == TBPM_SQUARE ? 4 : kind == TBPM_HONEYCOMB ? 3 : 6;
  g.row_sites = kind == TBPM_HONEYCOMB ? 2 * g.Lx : g.Lx;
  g.n_rows = g.Ly * g.Lz;
  g.n_full = g.row_sites * g.n_rows;

  int device = 0, n_sms = 0;
  cudaError_t e = cudaGetDevice(&device);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&n_sms, cudaDevAttrMultiProcessorCount, device);
  if (e != cudaSuccess) {
    set_error("tbpm_moment_step_noalloc: %s", cudaGetErrorString(e));
    return TBPM_ECUDA;
  }
  unsigned char* scratch = nullptr;
  TBPM_TRY(noalloc_scratch_address(device, &scratch));

  RecurrenceArgs a;
  memset(&a, 0, sizeof(a));
  a.cur = d_cur;
  a.prev_out = d_prev_out;
  a.geom = g;
  a.path = TBPM_PATH_STENCIL;
  a.diag = d_diag;
  a.diag_const = diag_const;
  a.thop = t_scaled;
  set_float_coefficients(&a);
  a.n_sites = g.n_full;
  const int spt = (precision == TBPM_C64 && n_states >= 2) ? 2 : 1;
  a.S = n_states;
  a.P = n_states / spt;
  a.logP = 0;
  while ((1 << a.logP) < a.P) ++a.logP;
  a.n_tiles = g.n_rows * ((g.row_sites * a.P + kThreads - 1) / kThreads);
  a.mu = d_mu;
  a.M = (int)n_moments;
  a.step = (int)step;
  const bool first = step == 0;
  void* fn;
  if (precision == TBPM_C128) fn = moment_kernel<double, 1>(kind, false, first);
  else if (spt == 2) fn = moment_kernel<float, 2>(kind, false, first);
  else fn = moment_kernel<float, 1>(kind, false, first);

  // grid: the persistent grid, shrunk until its partial sums fit the fixed scratch
  const size_t per_block = sizeof(double) * 3 * (size_t)n_states;
  const int64_t fit = (int64_t)((kNoAllocScratchBytes - 256) / per_block);
  int64_t grid = (int64_t)n_sms * resident_per_sm(fn);
  const int64_t supertiles = stencil_supertiles(g, a.P);
  if (grid > supertiles) grid = supertiles;
  if (grid > fit) grid = fit;
  if (grid < 1) {
    set_error("tbpm_moment_step_noalloc: %d states need more than the %zu-byte scratch", n_states,
              kNoAllocScratchBytes);
    return TBPM_EINVAL;
  }
  a.nblocks = (int)grid;
  a.counter = reinterpret_cast<unsigned*>(scratch);
  a.partials = reinterpret_cast<double*>(scratch + 256);
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  // the completion counter must start at zero; the partial sums are fully overwritten
  e = cudaMemsetAsync(scratch, 0, sizeof(unsigned), st);
  if (e == cudaSuccess) {
    void* args[] = {&a};
    e = cudaLaunchKernel(fn, dim3(a.nblocks), dim3(kThreads), args, 0, st);
  }
  if (e != cudaSuccess) {
    set_error("tbpm_moment_step_noalloc: %s", cudaGetErrorString(e));
    return TBPM_ECUDA;
  }
  return TBPM_OK;
}

TBPM_DEBUG_UNIT(cheb)
