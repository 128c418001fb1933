// Fermi-Dirac filtered response functions: the Fermi-Dirac operator as a Chebyshev series,
// the optical conductivity (OC) and the dynamical polarization (DP) of the paper's OC and DP
// sections, in the sequential and the state-based (time-block) forms.
//
//  * f(H) = [1 + e^{(H-mu)/kT}]^{-1} (or its square root) = sum_n a_n T_n(H~) with
//    a_n = ((2 - delta_n0)/K) sum_k f(H0 + |H| cos th_k) cos(n th_k), th_k = pi(k + 1/2)/K
//    (Chebyshev-Gauss quadrature); the angle n th_k is reduced exactly in integers before the
//    cosine.  The series runs to 1 + max{n : |a_n| > 1e-14}.
//  * Both Fermi-filtered states of one random state travel in one state block of 2 Sh states:
//    states [0, Sh) hold psi_1 = f(H) psi, states [Sh, 2Sh) hold psi_2 = [1 - f(H)] O psi with
//    O = J_beta (OC) or rho(-q) (DP), so one recurrence pass propagates both.  1 - f is applied
//    as O psi - f(H) O psi, with O psi formed again after the series (the series consumes its
//    input block in place, so at most three pair blocks are live).
//  * xmy: C(t) = <psi_1(t)| X |psi_2(t)> with X = J_alpha (bonds, weights -i t (r_j - r_i)_alpha)
//    or rho(q) (diagonal e^{i q.r_i}), for every state of a time block in one launch.
//  * Re sigma(w) = 2 (e^{-w/kT} - 1)/(w a_site) tau sum_j w_j sin(w t_j) Im C(t_j)   (w > 0),
//    Im sigma by Kramers-Kronig on w_k = k dw with Maclaurin's rule (nodes of opposite parity,
//    weight 2 dw; w = 0 weight dw), Pi(w) = -(2/a_site) tau sum_j w_j e^{i w t_j} Im C(t_j);
//    w_j = window_j (2 - delta_j0)/2.  a_site = area (volume) per site; the sample trace N C(t)
//    over the sample area N a_site.
//  * Charge density (CD section, Eq. rho): abs2py z_i += |psi(t_j)_i|^2 over the states of each time
//    block; rho_i = N sum_j w_j |psi(t_j)_i|^2 / sum_j w_j with psi(t) = e^{-iHt} f^{1/2}(H) psi.
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "stencil.cuh"
#include "tbpm_internal.cuh"

namespace tbpm {

namespace {

// ------------------------------------------------------------------ Fermi-Dirac coefficients
__global__ void k_fermi_nodes(int K, double mu, double kT, double H0, double half, int sqrt_f, double* g) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < K; k += gridDim.x * blockDim.x) {
    const double E = H0 + half * cos(M_PI * (k + 0.5) / K);
    const double x = (E - mu) / kT;
    // 1/(1 + e^x) without overflow
    const double f = x > 0.0 ? exp(-x) / (1.0 + exp(-x)) : 1.0 / (1.0 + exp(x));
    g[k] = sqrt_f ? sqrt(f) : f;
  }
}

// One block per order n: coef[2n] = a_n, coef[2n+1] = 0.
__global__ void __launch_bounds__(256) k_fermi_coeffs(int K, const double* g, double* coef) {
  __shared__ double sh[8];
  const int n = blockIdx.x;
  const int64_t period = 4LL * K;  // n th_k = pi n (2k+1) / (2K)
  double acc = 0.0;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const int64_t m = ((int64_t)n * (2 * k + 1)) % period;
    acc += g[k] * cos(M_PI * (double)m / (2.0 * K));
  }
  for (int off = 16; off >= 1; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += sh[w];
    coef[2 * n] = (n == 0 ? 1.0 : 2.0) / K * s;
    coef[2 * n + 1] = 0.0;
  }
}

// ------------------------------------------------------------------ site geometry
struct SiteGeom {
  Geom g;
  int csr;
  const int64_t* full_of;
};

__device__ __forceinline__ int64_t full_index(const SiteGeom& sg, int64_t i) { return sg.csr ? sg.full_of[i] : i; }

// position of full site f (library geometry): square/cubic unit spacing, graphene C-C = 1
__device__ __forceinline__ void site_position(const Geom& g, int64_t f, double* r) {
  if (g.kind == TBPM_HONEYCOMB) {
    const int64_t s = f & 1, c = f >> 1;
    const double x = (double)(c % g.Lx), y = (double)(c / g.Lx);
    r[0] = 1.5 * (x + y) + (double)s;
    r[1] = 0.8660254037844386 * (x - y);
    r[2] = 0.0;
  } else if (g.kind == TBPM_SQUARE) {
    r[0] = (double)(f % g.Lx);
    r[1] = (double)(f / g.Lx);
    r[2] = 0.0;
  } else {
    r[0] = (double)(f % g.Lx);
    r[1] = (double)((f / g.Lx) % g.Ly);
    r[2] = (double)(f / (g.Lx * g.Ly));
  }
}

// phase[i] = e^{i q.r_i} (FP64)
__global__ void k_density_phases(SiteGeom sg, int64_t n, double qx, double qy, double qz, double2* phase) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    double r[3];
    site_position(sg.g, full_index(sg, i), r);
    double sn, cs;
    sincos(qx * r[0] + qy * r[1] + qz * r[2], &sn, &cs);
    phase[i] = make_double2(cs, sn);
  }
}

// ------------------------------------------------------------------ state-block helpers
template <typename R>
struct C2;
template <>
struct C2<float> { using T = float2; };
template <>
struct C2<double> { using T = double2; };

// Xc[i][s] = psi[i][s], Xc[i][Sh+s] = (O psi)[i][s]; with phase != null, O psi = conj(phase_i) psi_i.
template <typename R>
__global__ void k_pair_init(int64_t n, int Sh, const void* psi_v, const void* opsi_v, const double2* phase,
                            void* xc_v) {
  using T = typename C2<R>::T;
  const T* psi = reinterpret_cast<const T*>(psi_v);
  const T* opsi = reinterpret_cast<const T*>(opsi_v);
  T* xc = reinterpret_cast<T*>(xc_v);
  const int64_t total = n * Sh;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Sh;
    const int s = (int)(e - i * Sh);
    const T p = psi[e];
    T o;
    if (phase) {
      const double2 ph = phase[i];
      const R cr = (R)ph.x, ci = (R)-ph.y;  // e^{-i q.r}
      o.x = cr * p.x - ci * p.y;
      o.y = cr * p.y + ci * p.x;
    } else {
      o = opsi[e];
    }
    xc[i * 2 * Sh + s] = p;
    xc[i * 2 * Sh + Sh + s] = o;
  }
}

// F[i][Sh+s] = (O psi)[i][s] - F[i][Sh+s]: the second half becomes [1 - f(H)] O psi.  O psi is
// opsi, or conj(phase_i) psi_i when phase != null.
template <typename R>
__global__ void k_pair_split(int64_t n, int Sh, const void* psi_v, const void* opsi_v, const double2* phase,
                             void* f_v) {
  using T = typename C2<R>::T;
  const T* psi = reinterpret_cast<const T*>(psi_v);
  const T* opsi = reinterpret_cast<const T*>(opsi_v);
  T* f = reinterpret_cast<T*>(f_v);
  const int64_t total = n * Sh;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = e / Sh;
    const int s = (int)(e - i * Sh);
    T x;
    if (phase) {
      const T p = psi[e];
      const double2 ph = phase[i];
      const R cr = (R)ph.x, ci = (R)-ph.y;
      x.x = cr * p.x - ci * p.y;
      x.y = cr * p.y + ci * p.x;
    } else {
      x = opsi[e];
    }
    const int64_t o = i * 2 * Sh + Sh + s;
    const T y = f[o];
    f[o] = T{x.x - y.x, x.y - y.y};
  }
}

// ------------------------------------------------------------------ xmy
struct XmyArgs {
  SiteGeom sg;
  const int32_t* ell;
  double kw[2][6];       // current operator weights t (r_j - r_i)_alpha
  const double* kwl;     // long-range lattices: the same per slot on the device, [2][z] (else null)
  const double2* phase;  // density operator e^{i q.r_i}, or null for the current operator
  const void* Y;         // bb pair blocks [n][2 Sh], consecutive
  int64_t y_stride;      // elements (complex) between pair blocks
  int64_t n_sites;
  int Sh;
  int64_t n_chunks;      // chunks of kYChunk sites
  double* partials;      // [gridDim.x][bb][Sh][2]
};

constexpr int kYIter = 8;
constexpr int kYChunk = kYIter * kThreads;

__device__ __forceinline__ int64_t nb_of(const XmyArgs& a, int64_t i, int d, const int64_t* coords) {
  if (a.sg.csr) return a.ell[i * a.sg.g.z + d];
  const Geom& g = a.sg.g;
  bool ok = true;
  if (g.kind == TBPM_HONEYCOMB) {
    const int64_t s = coords[2];
    const int sg = s == 0 ? -1 : 1;
    const int64_t xx = wrap_coord(coords[0] + ((d == 1) ? sg : 0), g.Lx, g.pbc_x, &ok);
    const int64_t yy = wrap_coord(coords[1] + ((d == 2) ? sg : 0), g.Ly, g.pbc_y, &ok);
    return ok ? 2 * (yy * g.Lx + xx) + (1 - s) : -1;
  }
  const int dx = (d == 0) ? 1 : (d == 1) ? -1 : 0;
  const int dy = (d == 2) ? 1 : (d == 3) ? -1 : 0;
  const int dz = (d == 4) ? 1 : (d == 5) ? -1 : 0;
  const int64_t xx = wrap_coord(coords[0] + dx, g.Lx, g.pbc_x, &ok);
  const int64_t yy = wrap_coord(coords[1] + dy, g.Ly, g.pbc_y, &ok);
  const int64_t zz = wrap_coord(coords[2] + dz, g.Lz, g.pbc_z, &ok);
  return ok ? (zz * g.Ly + yy) * g.Lx + xx : -1;
}

// One thread per (site, state s < Sh); grid (chunk groups, bb).  CURRENT: X = J_alpha, else rho(q).
template <typename R, bool CURRENT>
__global__ void __launch_bounds__(kThreads) k_xmy(XmyArgs a) {
  using T = typename C2<R>::T;
  __shared__ double tot[32 * 2];
  const T* Y = reinterpret_cast<const T*>(a.Y) + (int64_t)blockIdx.y * a.y_stride;
  const int Sh = a.Sh, S2 = 2 * a.Sh;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < 2 * Sh; q += kThreads) tot[q] = 0.0;
  __syncthreads();
  // thread -> (site offset, state): Sh divides 256
  const int s = threadIdx.x & (Sh - 1);
  const int site_lane = threadIdx.x / Sh;
  const int sites_per_pass = kThreads / Sh;
  for (int64_t chunk = blockIdx.x; chunk < a.n_chunks; chunk += gridDim.x) {
    Partial<R> pr, pi;
    const int64_t i0 = chunk * (int64_t)kYChunk / Sh;
    for (int it = 0; it < kYIter; ++it) {
      const int64_t i = i0 + (int64_t)it * sites_per_pass + site_lane;
      if (i >= a.n_sites) break;
      const T b = Y[i * S2 + s];
      R vr = 0, vi = 0;  // (X psi_2)_i
      if constexpr (CURRENT) {
        const int64_t f = full_index(a.sg, i);
        int64_t coords[3];
        int sub = 0;
        if (a.sg.g.kind == TBPM_HONEYCOMB) {
          sub = (int)(f & 1);
          const int64_t c = f >> 1;
          coords[0] = c % a.sg.g.Lx;
          coords[1] = c / a.sg.g.Lx;
          coords[2] = sub;
        } else {
          coords[0] = f % a.sg.g.Lx;
          coords[1] = (f / a.sg.g.Lx) % a.sg.g.Ly;
          coords[2] = f / (a.sg.g.Lx * a.sg.g.Ly);
        }
        for (int d = 0; d < a.sg.g.z; ++d) {
          const int64_t j = nb_of(a, i, d, coords);
          if (j < 0) continue;
          const R w = a.kwl ? (R)__ldg(a.kwl + sub * a.sg.g.z + d) : (R)a.kw[sub][d];
          const T x = Y[j * S2 + Sh + s];
          vr += w * x.y;  // -i w x
          vi -= w * x.x;
        }
      } else {
        const double2 ph = a.phase[i];
        const T x = Y[i * S2 + Sh + s];
        const R cr = (R)ph.x, ci = (R)ph.y;
        vr = cr * x.x - ci * x.y;
        vi = cr * x.y + ci * x.x;
      }
      pr.add(b.x * vr + b.y * vi);  // conj(psi_1) (X psi_2)
      pi.add(b.x * vi - b.y * vr);
    }
    pr.fold();
    pi.fold();
    double vr = pr.value(), vi = pi.value();
    for (int off = 16; off >= Sh; off >>= 1) {
      vr += __shfl_xor_sync(0xffffffffu, vr, off);
      vi += __shfl_xor_sync(0xffffffffu, vi, off);
    }
    for (int w = 0; w < kThreads / 32; ++w) {
      if (warp == w && lane < Sh) {
        tot[2 * lane] += vr;
        tot[2 * lane + 1] += vi;
      }
      __syncthreads();
    }
  }
  for (int q = threadIdx.x; q < 2 * Sh; q += kThreads)
    a.partials[(((int64_t)blockIdx.x * gridDim.y + blockIdx.y) * Sh) * 2 + q] = tot[q];
}

// ------------------------------------------------------------------ spectra
__device__ __forceinline__ double block_sum_r(double v, double* sh) {
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int w = 0; w < 8; ++w) r += sh[w];
  return r;
}

__device__ __forceinline__ double window_weight(int window, int j, int n_steps) {
  const double w = (window == TBPM_WINDOW_HANN) ? 0.5 * (1.0 + cos(M_PI * j / (n_steps + 1.0))) : 1.0;
  return j == 0 ? 0.5 * w : w;
}

// grid (n_omega, S); out[(s*n_omega + k)*2] = Re sigma(w_k)
__global__ void __launch_bounds__(256) k_oc_real(const double* C, int n_steps, double dw, int n_omega, double kT,
                                                 double tphys, double area, int window, double* out) {
  __shared__ double sh[8];
  const int k = blockIdx.x, s = blockIdx.y;
  const double w = k * dw;
  const double* Cs = C + (int64_t)s * (n_steps + 1) * 2;
  double acc = 0.0;
  for (int j = threadIdx.x; j <= n_steps; j += blockDim.x)
    acc += window_weight(window, j, n_steps) * sin(w * (double)j * tphys) * Cs[2 * j + 1];
  const double tot = block_sum_r(acc, sh);
  if (threadIdx.x == 0) {
    double v = 0.0;
    if (k > 0) v = 2.0 * (exp(-w / kT) - 1.0) / (w * area) * tphys * tot;
    out[((int64_t)s * n_omega + k) * 2] = v;
  }
}

// Im sigma(w_k) = -(2 w_k/pi) sum_{j: j-k odd} Re sigma(w_j) c_j / (w_j^2 - w_k^2), c_0 = dw, c_j = 2 dw.
__global__ void __launch_bounds__(256) k_oc_kk(double dw, int n_omega, double* out) {
  __shared__ double sh[8];
  const int k = blockIdx.x, s = blockIdx.y;
  double* row = out + (int64_t)s * n_omega * 2;
  const double wk = k * dw;
  double acc = 0.0;
  for (int j = threadIdx.x; j < n_omega; j += blockDim.x) {
    if (((j - k) & 1) == 0) continue;
    const double wj = j * dw;
    acc += row[2 * j] * (j == 0 ? dw : 2.0 * dw) / (wj * wj - wk * wk);
  }
  const double tot = block_sum_r(acc, sh);
  if (threadIdx.x == 0) row[2 * k + 1] = -2.0 * wk / M_PI * tot;
}

// grid (n_omega, S); Pi(w_k) = -(2/a) tau sum_j w_j e^{i w t_j} Im C_j
__global__ void __launch_bounds__(256) k_dp_pi(const double* C, int n_steps, const double* omegas, int n_omega,
                                               double tphys, double area, int window, double* out) {
  __shared__ double sh[8];
  const int k = blockIdx.x, s = blockIdx.y;
  const double w = omegas[k];
  const double* Cs = C + (int64_t)s * (n_steps + 1) * 2;
  double re = 0.0, im = 0.0;
  for (int j = threadIdx.x; j <= n_steps; j += blockDim.x) {
    double sn, cs;
    sincos(w * (double)j * tphys, &sn, &cs);
    const double v = window_weight(window, j, n_steps) * Cs[2 * j + 1];
    re += cs * v;
    im += sn * v;
  }
  const double R = block_sum_r(re, sh);
  const double I = block_sum_r(im, sh);
  if (threadIdx.x == 0) {
    out[((int64_t)s * n_omega + k) * 2] = -2.0 / area * tphys * R;
    out[((int64_t)s * n_omega + k) * 2 + 1] = -2.0 / area * tphys * I;
  }
}

// abs2py (CD section): z[e] += scale sum_a |Y_a[e]|^2 over bb state blocks, e < n_elems (FP64 z).
template <typename R>
__global__ void k_abs2py(const void* yv, int bb, int64_t stride, int64_t n_elems, double scale, double* z) {
  using T = typename C2<R>::T;
  const T* Y = reinterpret_cast<const T*>(yv);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n_elems; e += (int64_t)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int a = 0; a < bb; ++a) {
      const T v = Y[(int64_t)a * stride + e];
      acc += (double)(v.x * v.x + v.y * v.y);
    }
    z[e] += scale * acc;
  }
}

// out[s][i] = factor z[i][s] for the first S of Spad states
__global__ void k_cd_finish(const double* z, int64_t n, int S, int Spad, double factor, double* out) {
  const int64_t total = n * S;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int s = (int)(e / n);
    const int64_t i = e - (int64_t)s * n;
    out[e] = factor * z[i * Spad + s];
  }
}

int grid_of(tbpm_ctx* ctx, int64_t n) {
  return (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, (int64_t)ctx->num_sms * 8));
}

}  // namespace

// Coefficients a_n (n < n_cap) of f or sqrt(f) as complex pairs into coef [n_cap][2]; node
// values go to scratch [K].
int launch_fermi_coefficients(tbpm_ctx* ctx, double mu, double kT, double H0, double half, int sqrt_f, int n_cap,
                              int K, double* scratch, double* coef) {
  k_fermi_nodes<<<grid_of(ctx, K), 256, 0, ctx->stream>>>(K, mu, kT, H0, half, sqrt_f, scratch);
  TBPM_CK_LAUNCH(ctx);
  k_fermi_coeffs<<<n_cap, 256, 0, ctx->stream>>>(K, scratch, coef);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

int launch_density_phases(tbpm_ctx* ctx, const tbpm_lattice* lat, const double q[3], double2* phase) {
  SiteGeom sg{lat->geom, lat->path == TBPM_PATH_CSR, lat->full_of};
  k_density_phases<<<grid_of(ctx, lat->n_sites), 256, 0, ctx->stream>>>(sg, lat->n_sites, q[0], q[1], q[2], phase);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

int launch_pair_init(tbpm_ctx* ctx, int precision, int64_t n, int Sh, const void* psi, const void* opsi,
                     const double2* phase, void* xc) {
  const int g = grid_of(ctx, n * Sh);
  if (precision == TBPM_C128)
    k_pair_init<double><<<g, 256, 0, ctx->stream>>>(n, Sh, psi, opsi, phase, xc);
  else
    k_pair_init<float><<<g, 256, 0, ctx->stream>>>(n, Sh, psi, opsi, phase, xc);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

int launch_pair_split(tbpm_ctx* ctx, int precision, int64_t n, int Sh, const void* psi, const void* opsi,
                      const double2* phase, void* f) {
  const int g = grid_of(ctx, n * Sh);
  if (precision == TBPM_C128)
    k_pair_split<double><<<g, 256, 0, ctx->stream>>>(n, Sh, psi, opsi, phase, f);
  else
    k_pair_split<float><<<g, 256, 0, ctx->stream>>>(n, Sh, psi, opsi, phase, f);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

// C[(s*os + a + off)] = <psi_1|X|psi_2> of pair block a (bb blocks at stride pair_bytes).
int launch_xmy(tbpm_ctx* ctx, const tbpm_lattice* lat, int precision, int Sh, int alpha, const double2* phase,
               const void* Y, int bb, size_t pair_bytes, double* C, int64_t os, int64_t off) {
  XmyArgs a;
  a.sg = SiteGeom{lat->geom, lat->path == TBPM_PATH_CSR, lat->full_of};
  a.ell = lat->ell;
  a.kwl = nullptr;
  if (!phase) {
    current_weights(lat->desc.kind, alpha, lat->desc.t, a.kw);
    a.kwl = lat->jw ? lat->jw + (size_t)alpha * 2 * lat->geom.z : nullptr;
    if (a.sg.csr && !a.ell) {
      set_error("current operator: ELL lists missing");
      return TBPM_EINVAL;
    }
  }
  a.phase = phase;
  a.Y = Y;
  a.y_stride = (int64_t)(pair_bytes / (precision == TBPM_C128 ? 16 : 8));
  a.n_sites = lat->n_sites;
  a.Sh = Sh;
  const int64_t units = lat->n_sites * Sh;
  a.n_chunks = (units + kYChunk - 1) / kYChunk;
  int64_t G = std::max<int64_t>(1, ((int64_t)ctx->num_sms * 8 + bb - 1) / bb);
  G = std::min<int64_t>(G, a.n_chunks);
  G = std::min<int64_t>(G, 65535);
  TBPM_TRY(ensure(ctx, ctx->ws_xdot, sizeof(double) * 2 * (size_t)(G * bb * Sh)));
  a.partials = (double*)ctx->ws_xdot.p;
  dim3 grid((unsigned)G, (unsigned)bb);
  const bool cur = phase == nullptr;
  if (precision == TBPM_C128) {
    if (cur) k_xmy<double, true><<<grid, kThreads, 0, ctx->stream>>>(a);
    else k_xmy<double, false><<<grid, kThreads, 0, ctx->stream>>>(a);
  } else {
    if (cur) k_xmy<float, true><<<grid, kThreads, 0, ctx->stream>>>(a);
    else k_xmy<float, false><<<grid, kThreads, 0, ctx->stream>>>(a);
  }
  TBPM_CK_LAUNCH(ctx);
  return launch_partial_reduce(ctx, a.partials, (int)G, bb, 1, Sh, C, os, 1, 0, off);
}

int launch_abs2py(tbpm_ctx* ctx, int precision, const void* Y, int bb, size_t block_bytes, int64_t n_elems,
                  double scale, double* z) {
  const int64_t stride = (int64_t)(block_bytes / (precision == TBPM_C128 ? 16 : 8));
  const int g = grid_of(ctx, n_elems);
  if (precision == TBPM_C128)
    k_abs2py<double><<<g, 256, 0, ctx->stream>>>(Y, bb, stride, n_elems, scale, z);
  else
    k_abs2py<float><<<g, 256, 0, ctx->stream>>>(Y, bb, stride, n_elems, scale, z);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

int launch_cd_finish(tbpm_ctx* ctx, const double* z, int64_t n, int S, int Spad, double factor, double* out) {
  k_cd_finish<<<grid_of(ctx, n * S), 256, 0, ctx->stream>>>(z, n, S, Spad, factor, out);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

int launch_oc_spectrum(tbpm_ctx* ctx, const double* C, int S, int n_steps, double dw, int n_omega, double kT,
                       double tphys, double area, int window, double* out) {
  k_oc_real<<<dim3(n_omega, S), 256, 0, ctx->stream>>>(C, n_steps, dw, n_omega, kT, tphys, area, window, out);
  TBPM_CK_LAUNCH(ctx);
  k_oc_kk<<<dim3(n_omega, S), 256, 0, ctx->stream>>>(dw, n_omega, out);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

int launch_dp_spectrum(tbpm_ctx* ctx, const double* C, int S, int n_steps, const double* omegas, int n_omega,
                       double tphys, double area, int window, double* out) {
  k_dp_pi<<<dim3(n_omega, S), 256, 0, ctx->stream>>>(C, n_steps, omegas, n_omega, tphys, area, window, out);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

}  // namespace tbpm
