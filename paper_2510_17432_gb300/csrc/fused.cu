// Temporal fusion of the moment pass on the honeycomb stencil: K = 4 Chebyshev steps per pass.
//
// The recurrence phi_{n+1} = 2 H~ phi_n - phi_{n-1} (App. B) touches only nearest neighbours, so
// K steps of a 2-D tile of cells can be taken in shared memory once the tile carries a halo:
// on the honeycomb (A(x,y) ~ B(x,y), B(x-1,y), B(x,y-1); B(x,y) ~ A(x,y), A(x+1,y), A(x,y+1)) the
// region that stays exact shrinks by one cell per two steps, so a halo of K/2 cells suffices.
// Each state vector then crosses HBM twice (read phi_{n-1}, phi_n; write phi_{n+K-1}, phi_{n+K})
// per K steps instead of three times per step.  The moments of every step (A_j = <phi_j|phi_j>,
// B_j = <phi_{j+1}|phi_j>, cost halving of Eq. cheby_prod) are summed over the tile interior and
// reduced across CTAs in a fixed order.
//
// One CTA = one tile x one state pair (16 bytes per site per vector, complex64).  Reads are
// cp.async with zero fill for sites outside open boundaries (those stay zero: missing bonds);
// periodic directions wrap.  Outputs go to a second buffer pair, because neighbouring CTAs are
// still reading the inputs as their halos.
#include <cuda_runtime.h>
#include <string.h>

#include "stencil.cuh"
#include "tbpm_internal.cuh"

namespace tbpm {
namespace fused {

constexpr int K = 4;              // steps per pass
constexpr int H = K / 2;          // halo in cells
constexpr int TXC = 44, TY = 32;  // interior cells per tile
constexpr int WX = TXC + 2 * H, WY = TY + 2 * H;
constexpr int RS = 2 * WX;        // sites per tile row
constexpr int NS = RS * WY;       // sites per tile
constexpr int NT = 256;
constexpr int PER = (NS + NT - 1) / NT;  // sites per thread
constexpr int NV = K * 2 * 3;            // per-thread sums: step x state x {A, Re B, Im B}
constexpr size_t SMEM = 2 * (size_t)NS * 16;

struct FusedArgs {
  const float4* prev_in;
  const float4* cur_in;
  float4* prev_out;
  float4* cur_out;
  const float* diag;  // rescaled D_i or null
  float dc2, th2;     // regular-step coefficients 2D, 2t/|H|
  int64_t Lx, Ly;
  int pbc_x, pbc_y;
  int P;              // state pairs per site
  int S;
  int tiles_x, tiles_y;
  double* partials;   // [gridDim][NV]
  unsigned* counter;
  double* mu;
  int M;
  int step0;          // global index of the first step of this pass
};

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
  const uint32_t s = (uint32_t)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(s), "l"(gmem), "r"(bytes) : "memory");
}

__global__ void __launch_bounds__(NT, 2) k_fused_honeycomb(FusedArgs a) {
  extern __shared__ float4 sm[];
  float4* bufP = sm;       // phi_{j-1}, overwritten by phi_{j+1}
  float4* bufC = sm + NS;  // phi_j
  __shared__ double red[NT / 32][NV];
  __shared__ unsigned ticket;

  const int pair = blockIdx.x % a.P;
  const int tile = blockIdx.x / a.P;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int64_t x0 = (int64_t)tx * TXC - H, y0 = (int64_t)ty * TY - H;

  // per-thread sites: global site index (-1 = ghost outside an open boundary), interior flag
  int64_t gsite[PER];
  unsigned interior = 0;
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int q = threadIdx.x + i * NT;
    gsite[i] = -1;
    if (q < NS) {
      const int r = q / RS, c = q - r * RS, cx = c >> 1, s = c & 1;
      int64_t gx = x0 + cx, gy = y0 + r;
      const bool in_x = gx >= 0 && gx < a.Lx, in_y = gy >= 0 && gy < a.Ly;
      bool ok = true;
      if (!in_x) {
        if (a.pbc_x) gx = gx < 0 ? gx + a.Lx : gx - a.Lx;
        else ok = false;
      }
      if (!in_y) {
        if (a.pbc_y) gy = gy < 0 ? gy + a.Ly : gy - a.Ly;
        else ok = false;
      }
      if (ok) gsite[i] = 2 * (gy * a.Lx + gx) + s;
      if (cx >= H && cx < H + TXC && r >= H && r < H + TY && in_x && in_y) interior |= 1u << i;
    }
  }
  // load phi_{n-1}, phi_n of this state pair (zeros for ghosts)
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    const int q = threadIdx.x + i * NT;
    if (q < NS) {
      const int64_t off = gsite[i] >= 0 ? gsite[i] * a.P + pair : 0;
      const int bytes = gsite[i] >= 0 ? 16 : 0;
      cp_async16(bufP + q, a.prev_in + off, bytes);
      cp_async16(bufC + q, a.cur_in + off, bytes);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  float dsite[PER];
#pragma unroll
  for (int i = 0; i < PER; ++i) dsite[i] = (a.diag && gsite[i] >= 0) ? 2.0f * __ldg(a.diag + gsite[i]) : a.dc2;
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();

  float acc[NV];
#pragma unroll
  for (int k = 0; k < NV; ++k) acc[k] = 0.f;
  const float th = a.th2;
#pragma unroll
  for (int k = 0; k < K; ++k) {
#pragma unroll
    for (int i = 0; i < PER; ++i) {
      const int q = threadIdx.x + i * NT;
      if (q >= NS) continue;
      const int r = q / RS, c = q - r * RS, s = c & 1;
      const float4 own = bufC[q];
      float4 h = make_float4(0.f, 0.f, 0.f, 0.f);
      auto add = [&](int j) {
        const float4 v = bufC[j];
        h.x += v.x;
        h.y += v.y;
        h.z += v.z;
        h.w += v.w;
      };
      if (s == 0) {  // A(x,y): B(x,y), B(x-1,y), B(x,y-1)
        add(q + 1);
        if (c >= 2) add(q - 1);
        if (r >= 1) add(q - RS + 1);
      } else {  // B(x,y): A(x,y), A(x+1,y), A(x,y+1)
        add(q - 1);
        if (c + 1 < RS) add(q + 1);
        if (r + 1 < WY) add(q + RS - 1);
      }
      const float4 pv = bufP[q];
      const float d = dsite[i];
      float4 o;
      o.x = d * own.x + th * h.x - pv.x;
      o.y = d * own.y + th * h.y - pv.y;
      o.z = d * own.z + th * h.z - pv.z;
      o.w = d * own.w + th * h.w - pv.w;
      if (gsite[i] < 0) o = make_float4(0.f, 0.f, 0.f, 0.f);
      bufP[q] = o;
      if (interior & (1u << i)) {
        float* A = acc + k * 6;
        A[0] += own.x * own.x + own.y * own.y;
        A[1] += o.x * own.x + o.y * own.y;
        A[2] += o.x * own.y - o.y * own.x;
        A[3] += own.z * own.z + own.w * own.w;
        A[4] += o.z * own.z + o.w * own.w;
        A[5] += o.z * own.w - o.w * own.z;
      }
    }
    __syncthreads();
    float4* t = bufP;
    bufP = bufC;
    bufC = t;
  }
  // bufC = phi_{n+K}, bufP = phi_{n+K-1}: write the interior
#pragma unroll
  for (int i = 0; i < PER; ++i) {
    if (interior & (1u << i)) {
      const int q = threadIdx.x + i * NT;
      const int64_t off = gsite[i] * a.P + pair;
      __stcs(a.cur_out + off, bufC[q]);
      __stcs(a.prev_out + off, bufP[q]);
    }
  }

  // reduction: FP32 per thread -> FP64 warp and block trees -> per-CTA partials -> fixed-order sum
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; ++k) {
    double v = (double)acc[k];
    for (int off = 16; off >= 1; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (lane == 0) red[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < NV) {
    double v = 0.0;
    for (int w = 0; w < NT / 32; ++w) v += red[w][threadIdx.x];
    a.partials[(size_t)blockIdx.x * NV + threadIdx.x] = v;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(a.counter, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  const int n_tiles = a.tiles_x * a.tiles_y;
  const int nval = K * a.S * 3;
  for (int v = warp; v < nval; v += NT / 32) {
    const int k = v / (a.S * 3), rem = v - k * a.S * 3, s = rem / 3, comp = rem - s * 3;
    const int pr = s >> 1, sub = s & 1;
    const int idx = k * 6 + sub * 3 + comp;
    double sum = 0.0;
    for (int t = lane; t < n_tiles; t += 32) sum += __ldcg(a.partials + ((size_t)t * a.P + pr) * NV + idx);
    for (int off = 16; off >= 1; off >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, off);
    if (lane == 0) {
      const int j = a.step0 + k;
      double* ms = a.mu + (size_t)s * a.M * 2;
      if (comp == 0) {
        ms[4 * j] = 2.0 * sum - ms[0];
        ms[4 * j + 1] = -ms[1];
      } else if (comp == 1) {
        ms[4 * j + 2] = 2.0 * sum - ms[2];
      } else {
        ms[4 * j + 3] = 2.0 * sum - ms[3];
      }
    }
  }
  if (threadIdx.x == 0) *a.counter = 0u;
}

}  // namespace fused

bool fused_applicable(const tbpm_lattice* lat, int precision, int Spad) {
  const Geom& g = lat->geom;
  return lat->path == TBPM_PATH_STENCIL && g.kind == TBPM_HONEYCOMB && precision == TBPM_C64 && Spad >= 2 &&
         g.Lx >= fused::TXC + 2 * fused::H && g.Ly >= fused::TY + 2 * fused::H;
}

int fused_steps() { return fused::K; }

// One fused pass: steps step0 .. step0+K-1 from (prev_in, cur_in) into (prev_out, cur_out).
int launch_fused_pass(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                      const void* cur_in, void* prev_out, void* cur_out, int step0) {
  using namespace fused;
  static bool attr = false;
  if (!attr) {
    TBPM_CK(cudaFuncSetAttribute(k_fused_honeycomb, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMEM));
    attr = true;
  }
  FusedArgs a;
  memset(&a, 0, sizeof(a));
  a.prev_in = (const float4*)prev_in;
  a.cur_in = (const float4*)cur_in;
  a.prev_out = (float4*)prev_out;
  a.cur_out = (float4*)cur_out;
  a.diag = (const float*)ra.diag;
  a.dc2 = ra.dc2f;
  a.th2 = ra.th2f;
  a.Lx = lat->geom.Lx;
  a.Ly = lat->geom.Ly;
  a.pbc_x = lat->geom.pbc_x;
  a.pbc_y = lat->geom.pbc_y;
  a.P = ra.S / 2;
  a.S = ra.S;
  a.tiles_x = (int)((a.Lx + TXC - 1) / TXC);
  a.tiles_y = (int)((a.Ly + TY - 1) / TY);
  a.mu = ra.mu;
  a.M = ra.M;
  a.step0 = step0;
  const int64_t grid = (int64_t)a.tiles_x * a.tiles_y * a.P;
  TBPM_TRY(ensure(ctx, ctx->ws_fused_partials, sizeof(double) * NV * (size_t)grid));
  a.partials = (double*)ctx->ws_fused_partials.p;
  a.counter = ra.counter;
  k_fused_honeycomb<<<(unsigned)grid, NT, SMEM, ctx->stream>>>(a);
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

}  // namespace tbpm
