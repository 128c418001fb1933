// Electronic (DC) conductivity, Sec. V: the current operator, the block inner products
// <A_a|B_b> between two families of state blocks, and the reconstruction of the EC
// correlation function and of sigma(E) (Eq. DC).
//
//  * Current operator (Sec. V): J_alpha = i[H, P_alpha] with P_alpha = -sum_i r_alpha,i |i><i|,
//    so every bond i-j carries (J_alpha)_ij = -i H_ij (r_j - r_i)_alpha (hbar = e = 1).  Bond
//    vectors are those of the library's lattices: unit-spaced square and cubic lattices; graphene
//    with C-C distance 1, A -> B bonds (1,0), (-1/2,-sqrt3/2), (-1/2,sqrt3/2) in the fixed
//    neighbour order, B -> A their negatives.  Periodic bonds use the nearest image.  On
//    long-range lattices every tap carries its own bond vector (negated on the B sublattice).
//  * Block inner products: out[s][a][b] = sum_i conj(A_a[i][s]) B_b[i][s] for nA x nB pairs of
//    state blocks in one pass; each CTA owns a TA x TB tile of pairs and walks chunks of the
//    site range, FP32 products (complex64 states) summed over 16 units per thread, folded into
//    FP64 per chunk in a fixed warp order; chunk groups are summed in order by a second kernel.
//    Deterministic for fixed sizes.  This one primitive gives <psi|Psi(E)>, the moment-form
//    m_n(E) = <J psi|T_n(H~)|J Psi(E)> (Eq. dc_mom, nA = 1) and, for a time block of b states
//    psi_1(t_j), all b x N_E correlation values at once (the state-based form).
//  * Moment form (Eq. dc_mom and the sum after it):
//        C(t_j, E) = e^{i H0 t_j} sum_{n < N(j tau~)} c_n^*(j tau~) m_n(E) / |<psi|Psi(E)>|,
//    c_n^* = a_n i^n, a_0 = J_0, a_n = 2 J_n; the phase e^{i H0 t} undoes the spectral shift.
//  * sigma(E) = D(E)/A int_0^{t_tot} Re[e^{-iEt} C(t,E)] dt (Eq. DC) with D(E) = N Re<psi|Psi(E)>
//    and A = N x (area per site), weights (2 - delta_j0)/2 on t_j = j tau.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "stencil.cuh"
#include "tbpm_internal.cuh"

namespace tbpm {

namespace {

constexpr int kXIter = 16;                       // units per thread per chunk
constexpr int kXChunk = kXIter * kThreads;       // units per chunk

struct CurArgs {
  Geom g;
  int path;
  const int32_t* ell;
  const int64_t* full_of;
  int64_t n_sites;
  int P, logP;
  double kw[2][6];  // t (r_j - r_i)_alpha per sublattice and neighbour slot
  const double* kwl;  // long-range lattices: the same per slot on the device, [2][z] (else null)
};

// y = J_alpha x for one block of states [n_sites][S].
template <typename R, int SPT>
__global__ void __launch_bounds__(kThreads) k_current(CurArgs c, const void* xv, void* yv) {
  using PK = Pack<R, SPT>;
  const PK* X = reinterpret_cast<const PK*>(xv);
  PK* Y = reinterpret_cast<PK*>(yv);
  const int64_t n_units = c.n_sites * c.P;
  const bool csr = c.path == TBPM_PATH_CSR;
  for (int64_t u = (int64_t)blockIdx.x * kThreads + threadIdx.x; u < n_units; u += (int64_t)gridDim.x * kThreads) {
    const int64_t i = u >> c.logP;
    const int p = (int)(u & (c.P - 1));
    int sub = 0;
    if (c.g.kind == TBPM_HONEYCOMB) sub = (int)((csr ? c.full_of[i] : i) & 1);
    PK o;
#pragma unroll
    for (int k = 0; k < 2 * SPT; ++k) o.v[k] = R(0);
    for (int d = 0; d < c.g.z; ++d) {
      const int64_t j = csr ? (int64_t)c.ell[i * c.g.z + d] : neighbour_full(c.g, i, d);
      if (j < 0) continue;
      const R w = c.kwl ? (R)__ldg(c.kwl + sub * c.g.z + d) : (R)c.kw[sub][d];
      const PK x = ld(X + j * c.P + p);
#pragma unroll
      for (int k = 0; k < SPT; ++k) {  // -i w (xr + i xi) = w xi - i w xr
        o.v[2 * k] += w * x.v[2 * k + 1];
        o.v[2 * k + 1] -= w * x.v[2 * k];
      }
    }
    st(Y + u, o);
  }
}

struct XdotArgs {
  const void* A;
  int64_t a_stride;  // packs between blocks of A
  int nA;
  const void* B;
  int64_t b_stride;
  int nB;
  int64_t n_units;
  int P;
  int S;             // padded states per block
  int64_t n_chunks;
  double* partials;  // [gridDim.y][nA][nB][S][2]
};

template <typename R>
struct XAcc { using T = float; };
template <>
struct XAcc<double> { using T = double; };

// grid (a_tiles * b_tiles, chunk groups); 256 threads.
template <typename R, int SPT, int TA, int TB>
__global__ void __launch_bounds__(kThreads, 2) k_xdot(XdotArgs x) {
  using PK = Pack<R, SPT>;
  using T = typename XAcc<R>::T;
  constexpr int V = TA * TB * SPT * 2;
  __shared__ double tot[32 * TA * TB * 2];
  const PK* A = reinterpret_cast<const PK*>(x.A);
  const PK* B = reinterpret_cast<const PK*>(x.B);
  const int b_tiles = (x.nB + TB - 1) / TB;
  const int at = blockIdx.x / b_tiles, bt = blockIdx.x - at * b_tiles;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int PV = x.P * V;
  for (int q = threadIdx.x; q < PV; q += kThreads) tot[q] = 0.0;
  const PK* pa[TA];
  const PK* pb[TB];
#pragma unroll
  for (int k = 0; k < TA; ++k) pa[k] = A + (int64_t)min(at * TA + k, x.nA - 1) * x.a_stride;
#pragma unroll
  for (int l = 0; l < TB; ++l) pb[l] = B + (int64_t)min(bt * TB + l, x.nB - 1) * x.b_stride;
  __syncthreads();

  for (int64_t chunk = blockIdx.y; chunk < x.n_chunks; chunk += gridDim.y) {
    T acc[V];
#pragma unroll
    for (int v = 0; v < V; ++v) acc[v] = T(0);
    const int64_t u0 = chunk * kXChunk + threadIdx.x;
#pragma unroll 2
    for (int it = 0; it < kXIter; ++it) {
      const int64_t u = u0 + (int64_t)it * kThreads;
      if (u >= x.n_units) break;
      PK a[TA], b[TB];
#pragma unroll
      for (int k = 0; k < TA; ++k) a[k] = ld(pa[k] + u);
#pragma unroll
      for (int l = 0; l < TB; ++l) b[l] = ld(pb[l] + u);
#pragma unroll
      for (int k = 0; k < TA; ++k)
#pragma unroll
        for (int l = 0; l < TB; ++l)
#pragma unroll
          for (int s = 0; s < SPT; ++s) {
            const T ar = a[k].v[2 * s], ai = a[k].v[2 * s + 1];
            const T br = b[l].v[2 * s], bi = b[l].v[2 * s + 1];
            T* o = acc + ((k * TB + l) * SPT + s) * 2;
            o[0] += ar * br + ai * bi;
            o[1] += ar * bi - ai * br;
          }
    }
    // lanes with the same state group p = lane % P
#pragma unroll
    for (int v = 0; v < V; ++v)
      for (int off = 16; off >= x.P; off >>= 1) acc[v] += __shfl_xor_sync(0xffffffffu, acc[v], off);
    for (int w = 0; w < kThreads / 32; ++w) {
      if (warp == w && lane < x.P) {
#pragma unroll
        for (int v = 0; v < V; ++v) tot[lane * V + v] += (double)acc[v];
      }
      __syncthreads();
    }
  }
  for (int q = threadIdx.x; q < PV; q += kThreads) {
    const int p = q / V, v = q - p * V;
    const int c = v & 1, s = (v >> 1) % SPT, kl = (v >> 1) / SPT;
    const int k = kl / TB, l = kl - k * TB;
    const int ia = at * TA + k, ib = bt * TB + l;
    if (ia < x.nA && ib < x.nB)
      x.partials[((((int64_t)blockIdx.y * x.nA + ia) * x.nB + ib) * x.S + p * SPT + s) * 2 + c] = tot[q];
  }
}

// out[(s*os + a*oa + b*ob + off)*2 + c] = sum over chunk groups, in order.
__global__ void k_xdot_reduce(const double* partials, int G, int nA, int nB, int S, double* out, int64_t os,
                              int64_t oa, int64_t ob, int64_t off) {
  const int64_t per = (int64_t)nA * nB * S * 2;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < per; q += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int g = 0; g < G; ++g) acc += partials[(int64_t)g * per + q];
    const int c = (int)(q & 1);
    const int64_t r = q >> 1;
    const int s = (int)(r % S);
    const int64_t ab = r / S;
    const int b = (int)(ab % nB), a = (int)(ab / nB);
    out[(s * os + a * oa + b * ob + off) * 2 + c] = acc;
  }
}

__device__ __forceinline__ double block_sum256(double v, double* sh) {
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) r += sh[w];
  return r;  // valid in thread 0
}

// grid (n_steps+1, ceil(rows/8)).  m [rows][Nn][2]; C [rows][n_steps+1][2] (not yet normalised).
constexpr int kEcRows = 8;
__global__ void __launch_bounds__(256) k_ec_corr_m(const double* table, const int* n_per_step, int n_steps,
                                                   const double* m, int rows, int Nn, double shift, double tau,
                                                   double* C) {
  __shared__ double sh[8];
  const int j = blockIdx.x, r0 = blockIdx.y * kEcRows;
  const int64_t width = n_steps + 1;
  const int nj = min(n_per_step[j], Nn);
  double re[kEcRows], im[kEcRows];
#pragma unroll
  for (int q = 0; q < kEcRows; ++q) re[q] = im[q] = 0.0;
  for (int n = threadIdx.x; n < nj; n += blockDim.x) {
    const double Jn = table[(int64_t)n * width + j];
    const double a = (n == 0) ? Jn : 2.0 * Jn;
    double cr, ci;  // c_n^* = a i^n
    switch (n & 3) {
      case 0: cr = a; ci = 0.0; break;
      case 1: cr = 0.0; ci = a; break;
      case 2: cr = -a; ci = 0.0; break;
      default: cr = 0.0; ci = -a; break;
    }
#pragma unroll
    for (int q = 0; q < kEcRows; ++q) {
      if (r0 + q < rows) {
        const double* mr = m + ((int64_t)(r0 + q) * Nn + n) * 2;
        re[q] += cr * mr[0] - ci * mr[1];
        im[q] += cr * mr[1] + ci * mr[0];
      }
    }
  }
  double sn, cs;
  sincos(shift * (double)j * tau, &sn, &cs);  // e^{+i H0 t_j}
  for (int q = 0; q < kEcRows && r0 + q < rows; ++q) {
    const double R = block_sum256(re[q], sh);
    const double I = block_sum256(im[q], sh);
    if (threadIdx.x == 0) {
      C[((int64_t)(r0 + q) * width + j) * 2] = cs * R - sn * I;
      C[((int64_t)(r0 + q) * width + j) * 2 + 1] = cs * I + sn * R;
    }
  }
}

// One block per row = s*nE + k: C /= |<psi|Psi(E_k)>| and sigma from Eq. DC.
__global__ void __launch_bounds__(256) k_ec_finish(double* C, const double* nrm, const double* energies, int nE,
                                                   int n_steps, double tphys, double area, double* sigma) {
  __shared__ double sh[8];
  const int row = blockIdx.x, k = row % nE;
  const int64_t width = n_steps + 1;
  const double nr = nrm[2 * row], ni = nrm[2 * row + 1];
  const double mag = hypot(nr, ni);
  const double inv = mag > 0.0 ? 1.0 / mag : 0.0;
  const double E = energies[k];
  double* Cr = C + (int64_t)row * width * 2;
  double acc = 0.0;
  for (int j = threadIdx.x; j <= n_steps; j += blockDim.x) {
    const double cr = Cr[2 * j] * inv, ci = Cr[2 * j + 1] * inv;
    Cr[2 * j] = cr;
    Cr[2 * j + 1] = ci;
    double sn, cs;
    sincos(-E * (double)j * tphys, &sn, &cs);
    acc += (j == 0 ? 0.5 : 1.0) * (cs * cr - sn * ci);
  }
  const double tot = block_sum256(acc, sh);
  if (threadIdx.x == 0) sigma[row] = mag > 0.0 ? nr / area * tphys * tot : 0.0;
}

int spt_for(int precision, int S) { return (precision == TBPM_C64 && S >= 2) ? 2 : 1; }

template <typename R, int SPT, int TA, int TB>
int xdot_launch(tbpm_ctx* ctx, const XdotArgs& xa0, int G) {
  XdotArgs xa = xa0;
  const int pairs = ((xa.nA + TA - 1) / TA) * ((xa.nB + TB - 1) / TB);
  k_xdot<R, SPT, TA, TB><<<dim3(pairs, G), kThreads, 0, ctx->stream>>>(xa);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

}  // namespace

// Bond-vector components (r_j - r_i)_alpha per sublattice and neighbour slot, times t.
void current_weights(int kind, int direction, double t, double kw[2][6]) {
  for (int s = 0; s < 2; ++s)
    for (int d = 0; d < 6; ++d) kw[s][d] = 0.0;
  if (kind == TBPM_HONEYCOMB) {
    const double h = sqrt(3.0) / 2.0;
    const double vx[3] = {1.0, -0.5, -0.5}, vy[3] = {0.0, -h, h};
    for (int d = 0; d < 3; ++d) {
      const double c = direction == 0 ? vx[d] : direction == 1 ? vy[d] : 0.0;
      kw[0][d] = t * c;
      kw[1][d] = -t * c;
    }
  } else {
    // slots +x, -x, +y, -y, +z, -z
    for (int d = 0; d < 6; ++d) {
      const double c = (d / 2 == direction) ? ((d & 1) ? -1.0 : 1.0) : 0.0;
      kw[0][d] = kw[1][d] = t * c;
    }
  }
}

int launch_current(tbpm_ctx* ctx, const tbpm_lattice* lat, int precision, int S, int direction, const void* x,
                   void* y) {
  CurArgs c;
  c.g = lat->geom;
  c.path = lat->path;
  c.ell = lat->ell;
  c.full_of = lat->full_of;
  c.n_sites = lat->n_sites;
  const int spt = spt_for(precision, S);
  c.P = S / spt;
  c.logP = 0;
  while ((1 << c.logP) < c.P) ++c.logP;
  current_weights(lat->desc.kind, direction, lat->desc.t, c.kw);
  c.kwl = lat->jw ? lat->jw + (size_t)direction * 2 * lat->geom.z : nullptr;
  if (c.path == TBPM_PATH_CSR && !c.ell) {
    set_error("current operator: ELL lists missing");
    return TBPM_EINVAL;
  }
  const int64_t n_units = lat->n_sites * c.P;
  const int grid = (int)std::max<int64_t>(1, std::min<int64_t>((n_units + kThreads - 1) / kThreads,
                                                               (int64_t)ctx->num_sms * 8));
  if (precision == TBPM_C128)
    k_current<double, 1><<<grid, kThreads, 0, ctx->stream>>>(c, x, y);
  else if (spt == 2)
    k_current<float, 2><<<grid, kThreads, 0, ctx->stream>>>(c, x, y);
  else
    k_current<float, 1><<<grid, kThreads, 0, ctx->stream>>>(c, x, y);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

// out[(s*os + a*oa + b*ob + off)] (complex) = <A_a|B_b> for state s; blocks are [n_sites][S].
int launch_xdot(tbpm_ctx* ctx, int precision, int S, int64_t n_sites, const void* A, int nA, const void* B, int nB,
                double* out, int64_t os, int64_t oa, int64_t ob, int64_t off) {
  if (nA < 1 || nB < 1) return TBPM_OK;
  const int spt = spt_for(precision, S);
  XdotArgs xa;
  xa.A = A;
  xa.B = B;
  xa.nA = nA;
  xa.nB = nB;
  xa.P = S / spt;
  xa.S = S;
  xa.n_units = n_sites * xa.P;
  xa.a_stride = xa.n_units;
  xa.b_stride = xa.n_units;
  xa.n_chunks = (xa.n_units + kXChunk - 1) / kXChunk;
  const bool single = nA == 1;
  const int TA = single ? 1 : (spt == 2 ? 2 : 4), TB = single ? 8 : 4;
  const int64_t pairs = (int64_t)((nA + TA - 1) / TA) * ((nB + TB - 1) / TB);
  if (pairs > 2147483647LL) {
    set_error("too many state-block pairs");
    return TBPM_EUNSUPPORTED;
  }
  // enough CTAs for ~4 waves of 2 per SM, partials bounded to 64 MiB
  const int64_t per = (int64_t)nA * nB * S * 2;
  int64_t G = std::max<int64_t>(1, ((int64_t)ctx->num_sms * 8 + pairs - 1) / pairs);
  G = std::min<int64_t>(G, xa.n_chunks);
  G = std::min<int64_t>(G, std::max<int64_t>(1, (64LL << 20) / (int64_t)(per * sizeof(double))));
  G = std::min<int64_t>(G, 65535);
  TBPM_TRY(ensure(ctx, ctx->ws_xdot, sizeof(double) * (size_t)(per * G)));
  xa.partials = (double*)ctx->ws_xdot.p;
  int r;
  if (precision == TBPM_C128)
    r = single ? xdot_launch<double, 1, 1, 8>(ctx, xa, (int)G) : xdot_launch<double, 1, 4, 4>(ctx, xa, (int)G);
  else if (spt == 2)
    r = single ? xdot_launch<float, 2, 1, 8>(ctx, xa, (int)G) : xdot_launch<float, 2, 2, 4>(ctx, xa, (int)G);
  else
    r = single ? xdot_launch<float, 1, 1, 8>(ctx, xa, (int)G) : xdot_launch<float, 1, 4, 4>(ctx, xa, (int)G);
  TBPM_TRY(r);
  return launch_partial_reduce(ctx, xa.partials, (int)G, nA, nB, S, out, os, oa, ob, off);
}

int launch_partial_reduce(tbpm_ctx* ctx, const double* partials, int G, int nA, int nB, int S, double* out,
                          int64_t os, int64_t oa, int64_t ob, int64_t off) {
  const int64_t per = (int64_t)nA * nB * S * 2;
  const int rgrid = (int)std::max<int64_t>(1, std::min<int64_t>((per + 255) / 256, (int64_t)ctx->num_sms * 16));
  k_xdot_reduce<<<rgrid, 256, 0, ctx->stream>>>(partials, G, nA, nB, S, out, os, oa, ob, off);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

int launch_ec_corr_from_moments(tbpm_ctx* ctx, const double* table, const int* n_per_step, int n_steps,
                                const double* m, int rows, int Nn, double shift, double tau, double* C) {
  k_ec_corr_m<<<dim3(n_steps + 1, (rows + kEcRows - 1) / kEcRows), 256, 0, ctx->stream>>>(
      table, n_per_step, n_steps, m, rows, Nn, shift, tau, C);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

int launch_ec_finish(tbpm_ctx* ctx, double* C, const double* nrm, const double* energies, int nE, int rows,
                     int n_steps, double tphys, double area, double* sigma) {
  k_ec_finish<<<rows, 256, 0, ctx->stream>>>(C, nrm, energies, nE, n_steps, tphys, area, sigma);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

}  // namespace tbpm
