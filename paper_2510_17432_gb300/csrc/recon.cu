// Reconstruction of correlation values and spectra from moments / correlation samples
// (FP64 on CUDA cores), and the host-side Bessel-Chebyshev coefficients.
//
//  * Bessel table J_n(j tau~), n < n_terms, j = 0..N_t, by Miller's backward recurrence
//    normalised with J_0 + 2 sum_k J_{2k} = 1 (Abramowitz & Stegun 9.1.27, 9.1.46), one thread
//    per time step; the Chebyshev coefficients of exp(-i H~ tau~) are c_0 = J_0,
//    c_n = 2(-i)^n J_n (App. B).  Truncation N(tau~) = 1 + max{n : |c_n| > 1e-14} (Sec. II.A).
//  * Moment-based correlation (Sec. III, DOS-Concurrent-M):
//       C(t_j) = exp(-i H0 t_j) sum_{n<N(j tau~)} c_n(j tau~) m_n.
//  * Jackson-damped Chebyshev DOS (kernel polynomial method, Weisse et al., Rev. Mod.
//    Phys. 78, 275 (2006), Eqs. 71 and 81):
//       D(E) = [g_0 m_0 + 2 sum_{n>=1} g_n Re m_n T_n(E~)] / (pi |H| sqrt(1 - E~^2)).
//  * Windowed Fourier DOS (Sec. III): D(E) = (tau/2pi)[w_0 C_0 + 2 Re sum_j w_j e^{iEt_j} C_j].
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "tbpm_internal.cuh"

namespace tbpm {

constexpr double kEta = 1e-14;

// ------------------------------------------------------------------ host Bessel (FP64)
void bessel_j_host(double x, int n_max, double* out) {
  for (int k = 0; k <= n_max; ++k) out[k] = 0.0;
  if (x == 0.0) {
    out[0] = 1.0;
    return;
  }
  const double ax = fabs(x);
  int m = (n_max > (int)ceil(ax) ? n_max : (int)ceil(ax)) + 40 + (int)(10.0 * cbrt(ax));
  m += (m & 1);
  double jp1 = 0.0, j = 1e-200, norm = 0.0;
  for (int k = m; k >= 1; --k) {
    const double jm1 = (2.0 * k / ax) * j - jp1;
    jp1 = j;
    j = jm1;  // j now holds J_{k-1} (unnormalised)
    if (k - 1 <= n_max) out[k - 1] = j;
    if (fabs(j) > 1e200) {
      j *= 1e-200;
      jp1 *= 1e-200;
      norm *= 1e-200;
      for (int q = k - 1; q <= n_max; ++q) out[q] *= 1e-200;
    }
    if (((k - 1) & 1) == 0 && k - 1 > 0) norm += 2.0 * j;
  }
  norm += j;
  for (int k = 0; k <= n_max; ++k) {
    out[k] /= norm;
    if (x < 0 && (k & 1)) out[k] = -out[k];
  }
}

int64_t truncation_order_host(double tau) {
  const double at = fabs(tau);
  const int scan = (int)ceil(at + 40.0 + 12.0 * cbrt(at));
  double* J = new double[scan + 1];
  bessel_j_host(at, scan, J);
  int64_t last = -1;
  for (int n = scan; n >= 0; --n) {
    const double c = (n == 0) ? fabs(J[0]) : 2.0 * fabs(J[n]);
    if (c > kEta) {
      last = n;
      break;
    }
  }
  delete[] J;
  return last + 1;
}

// ------------------------------------------------------------------ Bessel table (device)
// table[n * width + j] = J_n(j tau), width = n_steps + 1; n_per_step[j] = N(j tau).
__global__ void k_bessel_table(double tau, int n_steps, int n_terms, double* table, int* n_per_step) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j > n_steps) return;
  const int64_t width = n_steps + 1;
  const double x = j * tau;
  if (j == 0) {
    for (int n = 0; n < n_terms; ++n) table[(int64_t)n * width] = (n == 0) ? 1.0 : 0.0;
    n_per_step[0] = 1;
    return;
  }
  // orders above x + 60 + 12 x^(1/3) are below 1e-24 of the peak: stored as 0
  int top = (int)ceil(x + 60.0 + 12.0 * cbrt(x));
  int keep = top < n_terms - 1 ? top : n_terms - 1;
  for (int n = keep + 1; n < n_terms; ++n) table[(int64_t)n * width + j] = 0.0;
  int m = top + 30;
  m += (m & 1);
  double jp1 = 0.0, jc = 1e-200, norm = 0.0;
  for (int k = m; k >= 1; --k) {
    const double jm1 = (2.0 * k / x) * jc - jp1;
    jp1 = jc;
    jc = jm1;
    if (k - 1 <= keep) table[(int64_t)(k - 1) * width + j] = jc;
    if (fabs(jc) > 1e200) {
      jc *= 1e-200;
      jp1 *= 1e-200;
      norm *= 1e-200;
      for (int q = k - 1; q <= keep; ++q) table[(int64_t)q * width + j] *= 1e-200;
    }
    if (((k - 1) & 1) == 0 && k - 1 > 0) norm += 2.0 * jc;
  }
  norm += jc;
  const double inv = 1.0 / norm;
  int last = 0;
  for (int n = 0; n <= keep; ++n) {
    const double v = table[(int64_t)n * width + j] * inv;
    table[(int64_t)n * width + j] = v;
    const double c = (n == 0) ? fabs(v) : 2.0 * fabs(v);
    if (c > kEta) last = n;
  }
  n_per_step[j] = last + 1;
}

int launch_bessel_table(tbpm_ctx* ctx, double tau, int n_steps, int n_terms, double* table,
                        int* n_per_step) {
  const int threads = 64;
  const int blocks = (n_steps + 1 + threads - 1) / threads;
  k_bessel_table<<<blocks, threads, 0, ctx->stream>>>(tau, n_steps, n_terms, table, n_per_step);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

// ------------------------------------------------------------------ block reductions (FP64)
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) sh[warp] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0) {
    for (int w = 0; w < NT / 32; ++w) r += sh[w];
  }
  return r;  // valid in thread 0
}

// ------------------------------------------------------------------ C(t_j) from moments
// grid (n_steps+1, S); C[(s*(n_steps+1) + j)*2 + {0,1}]
__global__ void __launch_bounds__(256) k_corr_from_moments(const double* table, const int* n_per_step,
                                                           int n_steps, const double* mu, int M,
                                                           double shift, double tau, double* C) {
  __shared__ double sh[8];
  const int j = blockIdx.x, s = blockIdx.y;
  const int64_t width = n_steps + 1;
  const int nj = min(n_per_step[j], M);
  const double* ms = mu + (size_t)s * M * 2;
  double re = 0.0, im = 0.0;
  for (int n = threadIdx.x; n < nj; n += blockDim.x) {
    const double Jn = table[(int64_t)n * width + j];
    const double a = (n == 0) ? Jn : 2.0 * Jn;
    const double mr = ms[2 * n], mi = ms[2 * n + 1];
    // c_n = a * (-i)^n
    double cr, ci;
    switch (n & 3) {
      case 0: cr = a; ci = 0.0; break;
      case 1: cr = 0.0; ci = -a; break;
      case 2: cr = -a; ci = 0.0; break;
      default: cr = 0.0; ci = a; break;
    }
    re += cr * mr - ci * mi;
    im += cr * mi + ci * mr;
  }
  const double R = block_sum<256>(re, sh);
  const double I = block_sum<256>(im, sh);
  if (threadIdx.x == 0) {
    double sn, cs;
    sincos(-shift * (double)j * tau, &sn, &cs);
    C[((size_t)s * width + j) * 2] = cs * R - sn * I;
    C[((size_t)s * width + j) * 2 + 1] = cs * I + sn * R;
  }
}

int launch_corr_from_moments(tbpm_ctx* ctx, const double* table, const int* n_per_step, int n_steps,
                             int n_terms, const double* mu, int S, int M, double shift, double tau,
                             double* C) {
  (void)n_terms;
  k_corr_from_moments<<<dim3(n_steps + 1, S), 256, 0, ctx->stream>>>(table, n_per_step, n_steps, mu, M,
                                                                     shift, tau, C);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

// ------------------------------------------------------------------ Jackson DOS (FP64)
__global__ void k_jackson_factors(int M, double* g) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= M) return;
  const double q = M_PI / (M + 1.0);
  double sn, cs;
  sincos(q * n, &sn, &cs);
  g[n] = ((M - n + 1.0) * cs + sn * (cos(q) / sin(q))) / (M + 1.0);
}

// One block per energy; thread t owns chunks of 16 consecutive orders generated by the
// three-term recurrence from T_n0, T_n0+1 = cos(n theta).  D[s*nE + k].
constexpr int kJTerms = 16;
constexpr int kMaxS = 32;
__global__ void __launch_bounds__(256) k_dos_jackson(const double* mu, int S, int M, const double* g,
                                                     const double* energies, int64_t nE, double H0,
                                                     double half, double* D) {
  __shared__ double sh[8];
  const int64_t k = blockIdx.x;
  const double x = (energies[k] - H0) / half;
  if (!(fabs(x) < 1.0)) {
    for (int s = threadIdx.x; s < S; s += blockDim.x) D[(size_t)s * nE + k] = 0.0;
    return;
  }
  const double th = acos(x);
  double acc[kMaxS];
  for (int s = 0; s < S; ++s) acc[s] = 0.0;
  for (int n0 = threadIdx.x * kJTerms; n0 < M; n0 += blockDim.x * kJTerms) {
    double tm = cos(n0 * th), tc = cos((n0 + 1) * th);
    for (int i = 0; i < kJTerms && n0 + i < M; ++i) {
      const int n = n0 + i;
      double Tn;
      if (i == 0) {
        Tn = tm;
      } else if (i == 1) {
        Tn = tc;
      } else {
        const double tn = 2.0 * x * tc - tm;
        tm = tc;
        tc = tn;
        Tn = tn;
      }
      const double wn = g[n] * Tn * (n == 0 ? 1.0 : 2.0);
      for (int s = 0; s < S; ++s) acc[s] += wn * mu[((size_t)s * M + n) * 2];
    }
  }
  const double scale = 1.0 / (M_PI * half * sqrt(1.0 - x * x));
  for (int s = 0; s < S; ++s) {
    const double tot = block_sum<256>(acc[s], sh);
    if (threadIdx.x == 0) D[(size_t)s * nE + k] = tot * scale;
  }
}

int launch_dos_jackson_fp64(tbpm_ctx* ctx, const double* mu, int S, int M, const double* energies,
                            int64_t nE, double H0, double half, double* D) {
  if (S > kMaxS) {
    set_error("Jackson reconstruction supports S <= %d per call", kMaxS);
    return TBPM_EUNSUPPORTED;
  }
  TBPM_TRY(ensure(ctx, ctx->ws_aux, sizeof(double) * M));
  double* g = (double*)ctx->ws_aux.p;
  k_jackson_factors<<<(M + 255) / 256, 256, 0, ctx->stream>>>(M, g);
  TBPM_CK_LAUNCH(ctx);
  k_dos_jackson<<<(unsigned)nE, 256, 0, ctx->stream>>>(mu, S, M, g, energies, nE, H0, half, D);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

// ------------------------------------------------------------------ Fourier DOS (FP64)
__global__ void __launch_bounds__(256) k_dos_fourier(const double* C, int S, int n_steps,
                                                     const double* energies, int64_t nE, double tau,
                                                     int window, double* D) {
  __shared__ double sh[8];
  const int64_t k = blockIdx.x;
  const double E = energies[k];
  const int64_t width = n_steps + 1;
  for (int s = 0; s < S; ++s) {
    const double* cs_ = C + (size_t)s * width * 2;
    double acc = 0.0;
    for (int j = threadIdx.x; j <= n_steps; j += blockDim.x) {
      const double wj = (window == TBPM_WINDOW_HANN) ? 0.5 * (1.0 + cos(M_PI * j / (n_steps + 1.0))) : 1.0;
      double sn, cs;
      sincos(E * (double)j * tau, &sn, &cs);
      const double re = cs * cs_[2 * j] - sn * cs_[2 * j + 1];
      acc += (j == 0 ? 1.0 : 2.0) * wj * re;
    }
    const double tot = block_sum<256>(acc, sh);
    if (threadIdx.x == 0) D[(size_t)s * nE + k] = tau / (2.0 * M_PI) * tot;
  }
}

int launch_dos_fourier(tbpm_ctx* ctx, const double* C, int S, int n_steps, const double* energies,
                       int64_t nE, double tau_phys, int window, double* D) {
  k_dos_fourier<<<(unsigned)nE, 256, 0, ctx->stream>>>(C, S, n_steps, energies, nE, tau_phys, window, D);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

// ------------------------------------------------------------------ quasi-eigenstate coefficients
// Energy-based form of Sec. IV (Eqs. form2_concurrent, QE_coeff with a(E,t) = e^{iEt}/2pi):
//   C_0(E) = (tau/2pi) sum_j w_j 2 J_0(j tau~) cos(eps t_j),
//   C_n(E) = (tau/2pi) sum_j w_j 4 J_n(j tau~) Re[(-i)^n e^{i eps t_j}],  n >= 1,
// eps = E - H0, w_j = (2 - delta_j0)/2.  phase[k][j] = (cos, sin)(eps_k t_j).
__global__ void k_qe_phase(const double* energies, int nE, double H0, double tphys, int n_steps, double* phase) {
  const int64_t total = (int64_t)nE * (n_steps + 1);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int k = (int)(e / (n_steps + 1));
    const int j = (int)(e - (int64_t)k * (n_steps + 1));
    double sn, cs;
    sincos((energies[k] - H0) * (double)j * tphys, &sn, &cs);
    phase[2 * e] = cs;
    phase[2 * e + 1] = sn;
  }
}

// One block per (n, group of 8 energies); threads over j.  coef[(n*nE + k)*2] = C_n(E_k), imag 0.
__global__ void __launch_bounds__(256) k_qe_coeffs(const double* table, int n_steps, const double* phase, int nE,
                                                   double scale, double* coef) {
  __shared__ double sh[8];
  const int n = blockIdx.x;
  const int k0 = blockIdx.y * 8;
  const int64_t width = n_steps + 1;
  double acc[8];
  for (int q = 0; q < 8; ++q) acc[q] = 0.0;
  for (int j = threadIdx.x; j <= n_steps; j += blockDim.x) {
    const double Jn = table[(int64_t)n * width + j];
    const double w = j == 0 ? 0.5 : 1.0;
    for (int q = 0; q < 8 && k0 + q < nE; ++q) {
      const double* ph = phase + ((int64_t)(k0 + q) * width + j) * 2;
      double f;
      if (n == 0) f = 2.0 * ph[0];
      else {
        switch (n & 3) {  // 4 Re[(-i)^n (cos + i sin)]
          case 0: f = 4.0 * ph[0]; break;
          case 1: f = 4.0 * ph[1]; break;
          case 2: f = -4.0 * ph[0]; break;
          default: f = -4.0 * ph[1]; break;
        }
      }
      acc[q] += w * Jn * f;
    }
  }
  for (int q = 0; q < 8 && k0 + q < nE; ++q) {
    const double tot = block_sum<256>(acc[q], sh);
    if (threadIdx.x == 0) {
      coef[((int64_t)n * nE + k0 + q) * 2] = scale * tot;
      coef[((int64_t)n * nE + k0 + q) * 2 + 1] = 0.0;
    }
  }
}

// (cos, sin)(E_k t_j) without the H0 shift: the phases of explicitly propagated states.
int launch_qe_coefficients_phase_only(tbpm_ctx* ctx, const double* energies, int nE, double tphys, int n_steps,
                                      double* phase) {
  const int64_t tot = (int64_t)nE * (n_steps + 1);
  k_qe_phase<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, ctx->stream>>>(energies, nE, 0.0, tphys,
                                                                                      n_steps, phase);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

int launch_qe_coefficients(tbpm_ctx* ctx, const double* table, int n_steps, int n_terms, const double* energies,
                           int nE, double H0, double tphys, double* phase, double* coef) {
  const int64_t tot = (int64_t)nE * (n_steps + 1);
  k_qe_phase<<<(int)std::min<int64_t>((tot + 255) / 256, 4096), 256, 0, ctx->stream>>>(energies, nE, H0, tphys,
                                                                                      n_steps, phase);
  TBPM_CK_LAUNCH(ctx);
  k_qe_coeffs<<<dim3(n_terms, (nE + 7) / 8), 256, 0, ctx->stream>>>(table, n_steps, phase, nE,
                                                                     tphys / (2.0 * M_PI), coef);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

}  // namespace tbpm
