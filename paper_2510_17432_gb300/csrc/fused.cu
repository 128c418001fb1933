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

#include <mutex>

#include "stencil.cuh"
#include "tbpm_internal.cuh"

namespace tbpm {
namespace fused {

// Tile shapes: interior TXC x TY cells, halo H = KS/2 cells, NT threads; the whole tile (both
// vectors, one state pair, 16 B per site each) sits in shared memory.
template <int KS, int NT_>
struct Cfg {
  static constexpr int K = KS;
  static constexpr int H = KS / 2;
  static constexpr int TXC = 48 - 2 * H, TY = 36 - 2 * H;
  static constexpr int WX = TXC + 2 * H, WY = TY + 2 * H;  // 48 x 36 cells
  static constexpr int RS = 2 * WX;
  static constexpr int NS = RS * WY;
  static constexpr int NT = NT_;
  static constexpr int PER = (NS + NT - 1) / NT;
  static constexpr int NV = K * 2 * 3;
  static constexpr size_t SMEM = 2 * (size_t)NS * 16;
};

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

__device__ __forceinline__ float4 f4add(float4 a, float4 b) {
  return make_float4(a.x + b.x, a.y + b.y, a.z + b.z, a.w + b.w);
}

// ------------------------------------------------------------------ column-blocked fused kernel
// Shared memory holds the A and B sublattices of a WX x WY-cell tile in separate arrays with one
// zero pad line: A[y][x] (pad column x = WX, pad row y = WY), B[y+1][x+1] (pad column 0, pad row
// 0), so that every neighbour offset exists and no neighbour test is needed:
//   A(x,y) <- B(x,y), B(x-1,y), B(x,y-1)        B(x,y) <- A(x,y), A(x+1,y), A(x,y+1)
// Thread t owns column x = t % WX and the RPT consecutive rows starting at RPT * (t / WX); the
// y-neighbours inside that run come from its own registers.  Pads stay zero in both buffers;
// values next to them are wrong but lie in the halo band that the tile never writes back.
template <int KS>
struct Cfg2 {
  static constexpr int K = KS;
  static constexpr int H = KS / 2;
  static constexpr int WX = 48, WY = 32;
  static constexpr int TXC = WX - 2 * H, TY = WY - 2 * H;
  static constexpr int RPT = 4;                 // rows per thread
  static constexpr int NT = WX * (WY / RPT);    // 384 threads
  static constexpr int PITCH = WX + 1;          // padded row length (float4)
  static constexpr int PLANE = (WY + 1) * PITCH;
  static constexpr int NV = K * 6;
  static constexpr size_t SMEM = 4 * (size_t)PLANE * 16;  // {A, B} x {phi_{j-1}, phi_j}
};

template <class C, bool HAS_DIAG, bool OPEN>
__global__ void __launch_bounds__(C::NT, 2) k_fused_cols(FusedArgs a) {
  constexpr int WX = C::WX, WY = C::WY, PITCH = C::PITCH, PLANE = C::PLANE, RPT = C::RPT, H = C::H;
  constexpr int NT = C::NT, NV = C::NV;
  extern __shared__ float4 sm[];
  __shared__ float redf[NT / 32][NV];
  __shared__ unsigned ticket;
  // planes: [0] A_prev, [1] B_prev, [2] A_cur, [3] B_cur (roles of prev/cur swap every step)
  float4* Ab[2] = {sm, sm + 2 * PLANE};
  float4* Bb[2] = {sm + PLANE, sm + 3 * PLANE};

  const int pair = blockIdx.x % a.P;
  const int tile = blockIdx.x / a.P;
  const int tx = tile % a.tiles_x, ty = tile / a.tiles_x;
  const int64_t x0 = (int64_t)tx * C::TXC - H, y0 = (int64_t)ty * C::TY - H;
  const int x = threadIdx.x % WX, ybase = RPT * (threadIdx.x / WX);
  const float4 zero = make_float4(0.f, 0.f, 0.f, 0.f);

  // zero the pads of all four planes
  for (int i = threadIdx.x; i < PITCH + WY; i += NT) {
    for (int b = 0; b < 2; ++b) {
      if (i < PITCH) {
        Ab[b][WY * PITCH + i] = zero;  // A pad row
        Bb[b][i] = zero;               // B pad row
      } else {
        const int y = i - PITCH;
        Ab[b][y * PITCH + WX] = zero;  // A pad column
        Bb[b][(y + 1) * PITCH] = zero; // B pad column
      }
    }
  }
  // global coordinates of this thread's cells
  int64_t gx = x0 + x;
  const bool in_x = gx >= 0 && gx < a.Lx;
  bool ghost_x = false;
  if (!in_x) {
    if (OPEN && !a.pbc_x) ghost_x = true;
    else gx = gx < 0 ? gx + a.Lx : gx - a.Lx;
  }
  const bool int_x = x >= H && x < H + C::TXC && in_x;
  int64_t site_a[RPT];  // global index of A(x, y); B is +1; -1 = ghost
  unsigned int_rows = 0, ghost_rows = 0;
  float dA[HAS_DIAG ? RPT : 1], dB[HAS_DIAG ? RPT : 1];
#pragma unroll
  for (int k = 0; k < RPT; ++k) {
    const int y = ybase + k;
    int64_t gy = y0 + y;
    const bool in_y = gy >= 0 && gy < a.Ly;
    bool ghost = ghost_x;
    if (!in_y) {
      if (OPEN && !a.pbc_y) ghost = true;
      else gy = gy < 0 ? gy + a.Ly : gy - a.Ly;
    }
    site_a[k] = ghost ? -1 : 2 * (gy * a.Lx + gx);
    if (ghost) ghost_rows |= 1u << k;
    if (int_x && y >= H && y < H + C::TY && in_y) int_rows |= 1u << k;
    const int64_t offA = ghost ? 0 : site_a[k] * a.P + pair, offB = ghost ? 0 : (site_a[k] + 1) * a.P + pair;
    const int bytes = ghost ? 0 : 16;
    cp_async16(Ab[0] + y * PITCH + x, a.prev_in + offA, bytes);
    cp_async16(Bb[0] + (y + 1) * PITCH + x + 1, a.prev_in + offB, bytes);
    cp_async16(Ab[1] + y * PITCH + x, a.cur_in + offA, bytes);
    cp_async16(Bb[1] + (y + 1) * PITCH + x + 1, a.cur_in + offB, bytes);
    if (HAS_DIAG) {
      dA[k] = ghost ? 0.f : 2.0f * __ldg(a.diag + site_a[k]);
      dB[k] = ghost ? 0.f : 2.0f * __ldg(a.diag + site_a[k] + 1);
    }
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
  asm volatile("cp.async.wait_group 0;" ::: "memory");
  __syncthreads();

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const float th = a.th2, dc = a.dc2;
#pragma unroll
  for (int k = 0; k < C::K; ++k) {
    float4* Ap = Ab[k & 1];        // phi_{j-1}, receives phi_{j+1}
    float4* Bp = Bb[k & 1];
    const float4* Ac = Ab[(k + 1) & 1];  // phi_j
    const float4* Bc = Bb[(k + 1) & 1];
    float acc[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    // current values of the run (and the rows just outside it)
    float4 aC[RPT + 1], bC[RPT + 1];  // aC[k] = A(x, ybase+k); bC[k] = B(x, ybase+k-1)
#pragma unroll
    for (int r = 0; r <= RPT; ++r) {
      aC[r] = Ac[(ybase + r) * PITCH + x];      // row ybase+RPT may be the pad row
      bC[r] = Bc[(ybase + r) * PITCH + x + 1];  // B(x, ybase+r-1)
    }
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      const int y = ybase + r;
      const float4 bxm = Bc[(y + 1) * PITCH + x];      // B(x-1, y)
      const float4 axp = Ac[y * PITCH + x + 1];        // A(x+1, y)
      const float4 ownA = aC[r], ownB = bC[r + 1];
      const float4 pA = Ap[y * PITCH + x], pB = Bp[(y + 1) * PITCH + x + 1];
      const float4 hA = f4add(f4add(ownB, bxm), bC[r]);       // B(x,y) + B(x-1,y) + B(x,y-1)
      const float4 hB = f4add(f4add(ownA, axp), aC[r + 1]);   // A(x,y) + A(x+1,y) + A(x,y+1)
      const float da = HAS_DIAG ? dA[r] : dc, db = HAS_DIAG ? dB[r] : dc;
      float4 oA, oB;
      oA.x = da * ownA.x + th * hA.x - pA.x;
      oA.y = da * ownA.y + th * hA.y - pA.y;
      oA.z = da * ownA.z + th * hA.z - pA.z;
      oA.w = da * ownA.w + th * hA.w - pA.w;
      oB.x = db * ownB.x + th * hB.x - pB.x;
      oB.y = db * ownB.y + th * hB.y - pB.y;
      oB.z = db * ownB.z + th * hB.z - pB.z;
      oB.w = db * ownB.w + th * hB.w - pB.w;
      if (OPEN && (ghost_rows & (1u << r))) {
        oA = zero;
        oB = zero;
      }
      Ap[y * PITCH + x] = oA;
      Bp[(y + 1) * PITCH + x + 1] = oB;
      if (int_rows & (1u << r)) {
        acc[0] += ownA.x * ownA.x + ownA.y * ownA.y + ownB.x * ownB.x + ownB.y * ownB.y;
        acc[1] += oA.x * ownA.x + oA.y * ownA.y + oB.x * ownB.x + oB.y * ownB.y;
        acc[2] += oA.x * ownA.y - oA.y * ownA.x + oB.x * ownB.y - oB.y * ownB.x;
        acc[3] += ownA.z * ownA.z + ownA.w * ownA.w + ownB.z * ownB.z + ownB.w * ownB.w;
        acc[4] += oA.z * ownA.z + oA.w * ownA.w + oB.z * ownB.z + oB.w * ownB.w;
        acc[5] += oA.z * ownA.w - oA.w * ownA.z + oB.z * ownB.w - oB.w * ownB.z;
      }
    }
#pragma unroll
    for (int v = 0; v < 6; ++v) {
      float t = acc[v];
      for (int off = 16; off >= 1; off >>= 1) t += __shfl_xor_sync(0xffffffffu, t, off);
      if (lane == 0) redf[warp][k * 6 + v] = t;
    }
    __syncthreads();
  }
  // after K (even) steps: planes [0]/[1] hold phi_{n+K-1}... roles: the last step wrote index (K-1)&1
  {
    const int last = (C::K - 1) & 1;   // plane set holding phi_{n+K}
    const float4* An = Ab[last];
    const float4* Bn = Bb[last];
    const float4* Ao = Ab[last ^ 1];   // phi_{n+K-1}
    const float4* Bo = Bb[last ^ 1];
#pragma unroll
    for (int r = 0; r < RPT; ++r) {
      if (int_rows & (1u << r)) {
        const int y = ybase + r;
        const int64_t offA = site_a[r] * a.P + pair, offB = (site_a[r] + 1) * a.P + pair;
        __stcs(a.cur_out + offA, An[y * PITCH + x]);
        __stcs(a.cur_out + offB, Bn[(y + 1) * PITCH + x + 1]);
        __stcs(a.prev_out + offA, Ao[y * PITCH + x]);
        __stcs(a.prev_out + offB, Bo[(y + 1) * PITCH + x + 1]);
      }
    }
  }

  // reduction: FP32 per thread and warp -> FP64 across warps -> per-CTA partials -> fixed-order sum
  if (threadIdx.x < NV) {
    double v = 0.0;
    for (int w = 0; w < NT / 32; ++w) v += (double)redf[w][threadIdx.x];
    a.partials[(size_t)blockIdx.x * NV + threadIdx.x] = v;
    __threadfence();
  }
  __syncthreads();
  if (threadIdx.x == 0) ticket = atomicAdd(a.counter, 1u);
  __syncthreads();
  if (ticket != gridDim.x - 1) return;
  __threadfence();
  const int n_tiles = a.tiles_x * a.tiles_y;
  const int nval = C::K * a.S * 3;
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

using V1 = Cfg2<4>;  // 4 steps per pass
using V2 = Cfg2<2>;  // 2 steps per pass

}  // namespace fused

bool fused_applicable(const tbpm_lattice* lat, int precision, int Spad) {
  const Geom& g = lat->geom;
  return lat->path == TBPM_PATH_STENCIL && g.kind == TBPM_HONEYCOMB && precision == TBPM_C64 && Spad >= 2 &&
         g.Lx >= fused::V1::WX && g.Ly >= fused::V1::WY;
}

int fused_steps(int variant) { return variant == 2 ? fused::V2::K : fused::V1::K; }

template <class C, bool D, bool O>
static cudaError_t set_smem_attr() {
  return cudaFuncSetAttribute(fused::k_fused_cols<C, D, O>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)C::SMEM);
}

template <class C>
static int launch_variant(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                          const void* cur_in, void* prev_out, void* cur_out, int step0) {
  using namespace fused;
  static std::once_flag once;
  static cudaError_t attr = cudaSuccess;
  std::call_once(once, [] {
    cudaError_t e[4] = {set_smem_attr<C, false, false>(), set_smem_attr<C, false, true>(),
                        set_smem_attr<C, true, false>(), set_smem_attr<C, true, true>()};
    for (cudaError_t x : e)
      if (x != cudaSuccess) attr = x;
  });
  TBPM_CK(attr);
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
  a.tiles_x = (int)((a.Lx + C::TXC - 1) / C::TXC);
  a.tiles_y = (int)((a.Ly + C::TY - 1) / C::TY);
  a.mu = ra.mu;
  a.M = ra.M;
  a.step0 = step0;
  const int64_t grid = (int64_t)a.tiles_x * a.tiles_y * a.P;
  TBPM_TRY(ensure(ctx, ctx->ws_fused_partials, sizeof(double) * C::NV * (size_t)grid));
  a.partials = (double*)ctx->ws_fused_partials.p;
  a.counter = ra.counter;
  const bool open = !(a.pbc_x && a.pbc_y);
  const dim3 gr((unsigned)grid), bl(C::NT);
  if (a.diag) {
    if (open) k_fused_cols<C, true, true><<<gr, bl, C::SMEM, ctx->stream>>>(a);
    else k_fused_cols<C, true, false><<<gr, bl, C::SMEM, ctx->stream>>>(a);
  } else {
    if (open) k_fused_cols<C, false, true><<<gr, bl, C::SMEM, ctx->stream>>>(a);
    else k_fused_cols<C, false, false><<<gr, bl, C::SMEM, ctx->stream>>>(a);
  }
  TBPM_CK_LAUNCH(ctx);
  return TBPM_OK;
}

// One fused pass: steps step0 .. step0+K-1 from (prev_in, cur_in) into (prev_out, cur_out).
int launch_fused_pass(tbpm_ctx* ctx, const tbpm_lattice* lat, const RecurrenceArgs& ra, const void* prev_in,
                      const void* cur_in, void* prev_out, void* cur_out, int step0, int variant) {
  if (variant == 2) return launch_variant<fused::V2>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
  return launch_variant<fused::V1>(ctx, lat, ra, prev_in, cur_in, prev_out, cur_out, step0);
}

}  // namespace tbpm
